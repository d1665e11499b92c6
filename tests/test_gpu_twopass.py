"""GPU parity of the two-pass push (reorth = 2) against the FP64 oracle's two-pass reading.

The two-pass push takes h_{j+1,j} from ||w'||^2 - ||s||^2 (w' after the first projection,
s = V^T w') and writes v_{j+1} while the next push streams V.  The oracle runs the same reading
(reorth = 2); in exact arithmetic both equal the CGS2 projections and norm of Alg. 1, so the FP64
case is also checked against the oracle's three-pass CGS2.  Tolerances as in test_gpu_push:
FP64 1e-10 normwise, FP32/BF16 column by column within C u_s kappa_2(X_{1:p}) <= 1e-2 (gpu_util).
"""
import numpy as np
import pytest

from gpu_util import compare_state, gaussian, match, run_gpu, run_oracle, to_device
from paper_1805_05821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


def compare(g, o, dt, k_max=None, label="two-pass"):
    """State and basis against the oracle (reading V first writes the pending column)."""
    return compare_state(g, o, dt, with_basis=True, label=label)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_two_pass_matches_oracle(dt):
    """n = 5184 (162 tiles, several stages), 28 snapshots: damped waves on a 72^2 grid for FP64 and
    FP32 (kappa_2 = 52), Gaussian snapshots for BF16 (kappa_2 = 1.16)."""
    spec = synth.config2(11, G=72, N=28)
    X = synth.snapshots(spec) if dt != "bf16" else gaussian(spec.n, 28, 11)
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, spec.n, 28, dt, reorth=2)
    o, sts = run_oracle(Xr, 28, dt, reorth=2)
    assert [s for s, _ in infos] == [0 if s[0] == "ok" else 5 for s in sts]
    for (st, inf), so in zip(infos, sts):
        if dt == "f64":
            assert abs(inf["h_last"] - so[1]) <= 1e-10 * abs(so[1])
    compare(g, o, dt, 28)


def test_two_pass_equals_cgs2_fp64():
    """In FP64 the two-pass reading and the three-pass CGS2 step agree to rounding."""
    spec = synth.config2(12, G=64, N=24)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, _ = run_gpu(Xd, spec.n, 24, "f64", reorth=2)
    o, _ = run_oracle(Xr, 24, "f64", reorth=1)
    compare(g, o, "f64", 24)


@pytest.mark.parametrize("n", [1, 31, 33, 4097, 20001])
def test_two_pass_ragged_fp64(n):
    rng = np.random.default_rng(100 + n)
    N = 16 if n > 16 else n + 1
    X = rng.standard_normal((n, N))
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, n, N, "f64", reorth=2)
    o, sts = run_oracle(Xr, N, "f64", reorth=2)
    assert [s for s, _ in infos] == [0 if s[0] == "ok" else 5 for s in sts]
    compare(g, o, "f64", N)


def test_two_pass_breakdown_planted_rank10():
    """Planted rank-10 map: the breakdown comes at push 11 on both sides; V holds 10 columns."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, spec.n, 32, "f64", reorth=2)
    o, sts = run_oracle(Xr, 32, "f64", reorth=2)
    assert len(infos) == 11 and infos[-1][0] == 5
    assert sts[-1][0] == "breakdown" and len(sts) == 11
    compare(g, o, "f64", 32)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_two_pass_basis_reads_between_pushes(dt):
    """Reading V (which writes the pending column) between pushes does not change the result
    (waves on a 48^2 grid for FP32, Gaussian snapshots for BF16)."""
    spec = synth.config2(13, G=48, N=24)
    X = synth.snapshots(spec) if dt == "f32" else gaussian(spec.n, 24, 13)
    Xr, Xd = to_device(X, dt)
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(spec.n, 24, dt, reorth=2)
    for t in range(24):
        assert g.push(Xd[t])[0] == 0
        if t % 5 == 2:
            g.basis(0, t + 1)
    o, _ = run_oracle(Xr, 24, dt, reorth=2)
    compare(g, o, dt, 24)


def test_two_pass_batch_and_full():
    """push_batch drives the same sequence; at q = k_max the last column is still written."""
    spec = synth.config2(14, G=40, N=20)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f32")
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(spec.n, 12, "f32", reorth=2)
    st, infos = g.push_batch(Xd[:15])
    assert st == 4  # EFULL after 12 pushes
    assert [i["status"] for i in infos[:12]] == ["OK"] * 12
    o, _ = run_oracle(Xr[:, :12], 12, "f32", reorth=2)
    compare(g, o, "f32", 12)


def test_two_pass_checkpoint_and_eig(tmp_path):
    """save writes the pending column; a loaded two-pass stream continues like the original,
    and the eigen path (Ritz values and modes) agrees with a three-pass stream."""
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    spec = synth.config2(15, G=64, N=24)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g1, _ = run_gpu(Xd, spec.n, 24, "f64", reorth=2)
    g2 = FoaDMD(spec.n, 24, "f64", reorth=2)
    for t in range(10):
        g2.push(Xd[t])
    path = tmp_path / "two_pass.foa"
    assert g2.save(path) == 0
    g2.close()
    g3 = FoaDMD.load(path, "f64", spec.n, 24, reorth=2)
    for t in range(10, 24):
        assert g3.push(Xd[t])[0] == 0
    o, _ = run_oracle(Xr, 24, "f64", reorth=2)
    compare(g3, o, "f64", 24)
    g4, _ = run_gpu(Xd, spec.n, 24, "f64", reorth=1)
    r1 = g1.eig(rank_tol=-1.0, n_modes=6)
    r4 = g4.eig(rank_tol=-1.0, n_modes=6)
    assert r1["status"] == r4["status"] == 0 and r1["r"] == r4["r"]
    d, perm = match(r1["lam"], r4["lam"])
    assert d.max() <= 1e-8
    P1, P4 = r1["phi"], r4["phi"]
    for k in range(P1.shape[1]):
        k4 = int(perm[k])
        if k4 >= P4.shape[1]:
            continue
        a, b = P1[:, k], P4[:, k4]
        c = np.vdot(b, a) / np.vdot(b, b)  # same mode up to the normalisation phase
        assert np.linalg.norm(a - c * b) <= 1e-6 * np.linalg.norm(a)
