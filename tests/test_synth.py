"""Seeded input generators (no GPU): Philox known answers, unit-variance transform, the planted map."""
import numpy as np

from paper_1805_05821_gb300 import synth


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 published with Random123 (Salmon et al., SC'11)."""
    cases = [((0, 0, 0, 0, 0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 6, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for args, want in cases:
        got = tuple(int(v) for v in synth.philox4x32_10(*args))
        assert got == want


def test_irwin_hall_moments():
    r = np.arange(200000)
    words = synth.philox4x32_10(r, 0, 3, 0, 12345, synth.KEY_MODES)
    g = synth.irwin_hall4(words, np.float64, np.float64(np.sqrt(3.0)))
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert np.abs(g).max() <= 2 * np.sqrt(3.0)


def test_planted_map_generates_the_sequence():
    spec = synth.planted(300, 12, 7, seed=4)
    X = synth.snapshots(spec)
    A = synth.planted_map(spec)
    np.testing.assert_allclose(A @ X[:, :-1], X[:, 1:], rtol=0, atol=1e-12 * np.abs(X).max())
    lam = np.linalg.eigvals(spec.meta["block"])
    d = np.abs(np.sort_complex(lam) - np.sort_complex(spec.lam))
    assert d.max() < 1e-12


def test_rows_match_full_matrix_and_precisions():
    spec = synth.config5(0, G=8, N=6)
    X64 = synth.snapshots(spec, np.float64)
    X32 = synth.snapshots(spec, np.float32)
    r = np.array([0, 5, 511, 1024, spec.n - 1])
    for t in (0, 3, 5):
        np.testing.assert_array_equal(synth.rows(spec, t, r, np.float64), X64[r, t])
        np.testing.assert_array_equal(synth.rows(spec, t, r, np.float32), X32[r, t])
    assert np.abs(X32 - X64).max() <= 1e-5 * np.abs(X64).max()


def test_wave_tables_are_exact_unit_phasors():
    spec = synth.config2(0, G=64, N=4)
    for tab in spec.tables:
        np.testing.assert_allclose(tab[..., 0] ** 2 + tab[..., 1] ** 2, 1.0, atol=1e-15)
    # x_0 is a sum of unit sine waves with distinct wavevectors: mean square = M/2
    X = synth.snapshots(spec, np.float64, N=1)
    assert abs(np.mean(X[:, 0] ** 2) - spec.M / 2) < 1e-3 * spec.M


def test_config_shapes():
    assert synth.config1().n == 4096 and synth.config1().N == 32
    s2 = synth.config2()
    assert s2.n == 2 ** 20 and s2.N == 200 and len(s2.lam) == 40
    s3 = synth.config3(kappa=1e4)
    assert s3.n == 2 ** 24 and s3.N == 500
    s5 = synth.config5()
    assert s5.n == 67108864 and s5.N == 384 and s5.n_fields == 4
    streams = synth.config4(streams=8)
    for s in streams:
        assert 2 ** 14 <= s.n <= 2 ** 22 + 1 and 50 <= s.N <= 400
