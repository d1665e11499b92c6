"""GPU parity of the streaming push (the modified FOA update of Alg. 1, Alg. 4) against the FP64 oracle.

Every case runs the CUDA path through the C ABI and the oracle on the same (storage-rounded)
inputs.  Tolerances: FP64 storage 1e-10 normwise on beta and H-bar; FP32/BF16 storage column by
column, ||delta col|| / ||col|| <= C u_s kappa_2(X_{1:p}) with the fixed C of gpu_util (the error
law of Sec. 3.2.2, Eq. foabaseddmdberr), and only on inputs where that bound is at most 1e-2.
Ill-conditioned reduced-precision sequences are compared through their leading eigenvalues.
"""
import numpy as np
import pytest

from gpu_util import (U, compare_eigs, compare_state, gaussian, kappa_of, rel, run_gpu, run_oracle,
                      to_device)
from paper_1805_05821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()



def test_planted_rank10_fp64_breakdown():
    """n=4096, N=32 planted rank-10 map: breakdown at push 11 on both sides, state within 1e-10."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, spec.n, 32, "f64")
    o, sts = run_oracle(Xr, 32, "f64")
    assert len(infos) == 11 and infos[-1][0] == 5  # FOA_DMD_EBREAKDOWN at push 11
    assert sts[-1][0] == "breakdown" and len(sts) == 11
    compare_state(g, o, "f64", q_expect=10)
    Vg = g.basis(0, 10).double().cpu().numpy().T
    assert rel(Vg, o.V[:, :10]) <= 1e-10
    for (st, inf), so in zip(infos[:-1], sts[:-1]):
        assert abs(inf["h_last"] - so[1]) <= 1e-10 * abs(so[1])


@pytest.mark.parametrize("n", [1, 31, 33, 1000, 4097, 20001])
def test_ragged_fp64(n):
    """Ragged lengths (not multiples of the 32-row tile or of a pipeline stage)."""
    rng = np.random.default_rng(n)
    N = 24 if n > 24 else n + 1
    X = rng.standard_normal((n, N))
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, n, N, "f64")
    o, sts = run_oracle(Xr, N, "f64")
    assert [s[0] for s in infos] == [0 if s[0] == "ok" else 5 for s in sts]
    compare_state(g, o, "f64")


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_precision_forms(dt):
    """FP32/BF16 storage, FP32 products, FP64 blocked accumulation.  FP32: 40 undamped waves on a
    96^2 grid with 1e-3 noise (kappa_2 = 33); BF16: Gaussian snapshots of the same shape
    (kappa_2 = 1.14), since u_bf16 kappa must stay below 1e-2."""
    if dt == "f32":
        X = synth.snapshots(synth.waves(96, 2, 1, 40, 40, 2, sigma=None, noise_rel=1e-3))
    else:
        X = gaussian(9216, 40, 2)
    n = X.shape[0]
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, n, 40, dt)
    o, sts = run_oracle(Xr, 40, dt)
    assert len(infos) == len(sts) == 40
    compare_state(g, o, dt, with_basis=True, label="precision forms")


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_push_batch_is_bitwise_push(dt):
    """Alg. 4 with batch p carries out the same operations as p single pushes (Sec. 3.1)."""
    spec = synth.config2(3, G=64, N=30)
    X = synth.snapshots(spec)
    _, Xd = to_device(X, dt)
    g1, _ = run_gpu(Xd, spec.n, 30, dt)
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g2 = FoaDMD(spec.n, 30, dt)
    st, infos = g2.push_batch(Xd[:9])
    assert st == 0 and all(i["status"] == "OK" for i in infos)
    st, infos = g2.push_batch(Xd[9:30])
    assert st == 0
    q1, s1, H1, B1 = g1.state()
    q2, s2, H2, B2 = g2.state()
    assert q1 == q2 == 30
    np.testing.assert_array_equal(H1, H2)
    np.testing.assert_array_equal(B1, B2)
    assert bool((g1.basis(0, 30) == g2.basis(0, 30)).all())


def test_status_cases():
    import torch
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    n = 500
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((5, n))).cuda()
    # zero first snapshot
    g = FoaDMD(n, 4, "f64")
    st, inf = g.push(torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert st == 5 and inf["q"] == 0
    assert g.push(X[0])[0] == 6  # ESTOPPED
    # non-finite snapshot leaves the state unchanged
    g = FoaDMD(n, 3, "f64")
    assert g.push(X[0])[0] == 0 and g.push(X[1])[0] == 0
    q0, _, H0, B0 = g.state()
    bad = X[2].clone()
    bad[77] = float("nan")
    st, inf = g.push(bad)
    assert st == 7
    q1, stopped, H1, B1 = g.state()
    assert q1 == q0 == 2 and not stopped
    np.testing.assert_array_equal(H0, H1)
    np.testing.assert_array_equal(B0, B1)
    assert g.push(X[2])[0] == 0
    assert g.push(X[3])[0] == 4  # EFULL
    # linearly dependent snapshot
    g = FoaDMD(n, 5, "f64")
    g.push(X[0])
    g.push(X[1])
    st, inf = g.push(2.0 * X[0] - 0.5 * X[1])
    assert st == 5 and inf["q"] == 2
    q, stopped, H, B = g.state()
    assert stopped and q == 2 and H[2, 1] == 0.0
    assert g.push(X[3])[0] == 6


def test_push_batch_stops_at_failure():
    import torch
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    n = 300
    rng = np.random.default_rng(1)
    Xh = rng.standard_normal((6, n))
    Xh[3, 5] = np.inf
    Xd = torch.from_numpy(Xh).cuda()
    g = FoaDMD(n, 8, "f64")
    st, infos = g.push_batch(Xd)
    assert st == 7
    assert [i["status"] for i in infos] == ["OK", "OK", "OK", "ENONFINITE", "ESTOPPED", "ESTOPPED"]
    assert g.state()[0] == 3


def test_cgs1_option():
    """reorth = 0 (one classical Gram-Schmidt pass) against the oracle with the same option."""
    spec = synth.config2(4, G=48, N=20)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, _ = run_gpu(Xd, spec.n, 20, "f64", reorth=0)
    o, _ = run_oracle(Xr, 20, "f64", reorth=0)
    compare_state(g, o, "f64")


def test_checkpoint_resume_is_bitwise(tmp_path):
    """The streaming state is exactly (H, V, beta, q) (Alg. 3): save, load, continue = uninterrupted."""
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    spec = synth.config2(5, G=64, N=24)
    X = synth.snapshots(spec)
    _, Xd = to_device(X, "f32")
    g1, _ = run_gpu(Xd, spec.n, 24, "f32")
    g2 = FoaDMD(spec.n, 24, "f32")
    for t in range(10):
        g2.push(Xd[t])
    path = tmp_path / "state.foa"
    assert g2.save(path) == 0
    g2.close()
    g3 = FoaDMD.load(path, "f32", spec.n, 24)
    for t in range(10, 24):
        assert g3.push(Xd[t])[0] == 0
    a, b = g1.state(), g3.state()
    assert a[0] == b[0] == 24
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])
    assert bool((g1.basis(0, 24) == g3.basis(0, 24)).all())
    # a corrupted file is refused
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0xFF
    path.write_bytes(bytes(raw))
    with pytest.raises(RuntimeError):
        FoaDMD.load(path, "f32", spec.n, 24)


def test_device_generator_matches_host_rows():
    """The device snapshot generator equals the host evaluation bit for bit (sampled rows)."""
    import torch
    from paper_1805_05821_gb300 import foa_dmd as F
    spec = synth.config5(0, G=32, N=3)
    tabs = torch.from_numpy(np.stack(spec.tables).astype(np.float32)).cuda()
    x = torch.empty(spec.n, dtype=torch.float32, device="cuda")
    r = np.random.default_rng(0).integers(0, spec.n, 4000)
    for t in (0, 2):
        coef = torch.from_numpy(spec.T[:, :, t].astype(np.float32)).cuda()
        F.foa_synth_waves(x, "f32", spec.n, 3, 32, 4, spec.M, tabs, coef, spec.noise_scale, spec.seed_noise, t)
        torch.cuda.synchronize()
        got = x.cpu().numpy()[r]
        want = synth.rows(spec, t, r, np.float32)
        np.testing.assert_array_equal(got, want)
    sp = synth.planted(5000, 4, 9, seed=2, noise_rel=1e-5)
    coef = torch.from_numpy(sp.T[0, :, 1].astype(np.float64)).cuda()
    x64 = torch.empty(sp.n, dtype=torch.float64, device="cuda")
    F.foa_synth_gauss(x64, "f64", sp.n, sp.M, sp.seed_modes, sp.mode_scale, coef, sp.noise_scale, sp.seed_noise, 1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x64.cpu().numpy(), synth.rows(sp, 1, np.arange(sp.n), np.float64))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_waves_2d_full_size(dt):
    """1024 x 1024 grid (n = 2^20), N = 200, 20 damped waves, noise 1e-6 relative (kappa_2 = 1.8e6).
    FP64: state within the FP64 law.  FP32: u_s kappa_2(X) is far above 1e-2 (the default FP32
    breakdown test stops both sides at push 44), so the state is not comparable column by column;
    the eig truncated at rank_tol = 1e-4 (retained kappa_2 <= 1e4) is, through the 20 leading
    eigenvalues (compare_eigs)."""
    spec = synth.config2(0)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, spec.n, 200, dt)
    o, sts = run_oracle(Xr, 200, dt)
    assert len(infos) == len(sts)
    if dt == "f64":
        compare_state(g, o, dt)
        return
    rg = g.eig(rank_tol=1e-4)
    ro = o.eig(1e-4)
    assert rg["status"] == 0
    compare_eigs(rg, ro, dt, 20, label="waves 1024^2")


@pytest.mark.parametrize("dt,reorth", [("f32", 1), ("bf16", 1), ("f32", 2), ("bf16", 2)])
def test_wide_basis_register_stage(dt, reorth):
    """N = 160 on n = 9216 rows: past j = 64 a pipeline stage is one or two 32-row tiles and the
    FP32/BF16 passes with column dots hold the stage in registers.  FP32: 100 undamped waves on a
    96^2 grid with 1e-2 noise (kappa_2 = 210); BF16: Gaussian snapshots (kappa_2 = 1.3)."""
    if dt == "f32":
        X = synth.snapshots(synth.waves(96, 2, 1, 160, 100, 6, sigma=None, noise_rel=1e-2))
    else:
        X = gaussian(9216, 160, 6)
    n = X.shape[0]
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, n, 160, dt, reorth=reorth, breakdown_tol=1e-12)
    o, sts = run_oracle(Xr, 160, dt, tol=1e-12, reorth=reorth)
    assert len(infos) == len(sts) == 160
    compare_state(g, o, dt, with_basis=True, label=f"register stage reorth={reorth}")


@pytest.mark.parametrize("dt,reorth", [("f32", 1), ("f32", 2), ("bf16", 1), ("bf16", 2)])
def test_wide_basis_ragged(dt, reorth):
    """n = 9001 (a ragged last tile, snapshot rows not 16-byte aligned, so x is read from global
    memory instead of the staged slice), N = 140 Gaussian snapshots through the register-held
    passes."""
    n, N = 9001, 140
    X = np.random.default_rng(9001).standard_normal((n, N))
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, n, N, dt, reorth=reorth)
    o, sts = run_oracle(Xr, N, dt, reorth=reorth)
    assert [s[0] for s in infos] == [0] * N and all(s[0] == "ok" for s in sts)
    compare_state(g, o, dt, with_basis=True, label=f"ragged n=9001 reorth={reorth}")


@pytest.mark.parametrize("dt,reorth", [("f32", 1), ("f32", 2), ("bf16", 1)])
def test_widest_basis_register_stage(dt, reorth):
    """k_max = 440 on n = 4097 Gaussian snapshots: past j = 384 a thread's column group holds up
    to 32 columns (the widest register-held form)."""
    n, N = 4097, 440
    X = np.random.default_rng(4097).standard_normal((n, N))
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, n, N, dt, reorth=reorth)
    o, sts = run_oracle(Xr, N, dt, reorth=reorth)
    assert [s[0] for s in infos] == [0] * N and all(s[0] == "ok" for s in sts)
    compare_state(g, o, dt, with_basis=True, label=f"widest n=4097 reorth={reorth}")


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_push_host_matches_device_pushes(dt):
    """foa_dmd_push_host from pinned memory (foa_dmd_host_alloc) and from pageable host memory
    gives the state of foa_dmd_push on the same snapshots bit for bit (the host path adds only the
    staged copy and the host-side page reads); n = 9001 (ragged last tile), N = 24 Gaussian."""
    import ctypes
    import torch
    from paper_1805_05821_gb300 import foa_dmd as F
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    n, N = 9001, 24
    X = gaussian(n, N, 24)
    Xr, Xd = to_device(X, dt)
    es = 4 if dt == "f32" else 2
    gd = FoaDMD(n, N, dt)
    for t in range(N):
        gd.push(Xd[t], info=False)
    want = gd.state()
    Vd = gd.basis(0, N).cpu()
    host_rows = Xd.cpu().contiguous()
    ptr = F.foa_dmd_host_alloc(N * n * es)
    try:
        ctypes.memmove(ptr, host_rows.data_ptr(), N * n * es)
        for label, base in (("pinned", ptr), ("pageable", host_rows.data_ptr())):
            g = FoaDMD(n, N, dt)
            for t in range(N):
                st, _ = F.foa_dmd_push_host(g.h, base + t * n * es)
                assert st == 0, (label, t, st)
            q, stopped, H, B = g.state()
            assert q == want[0] == N and not stopped
            np.testing.assert_array_equal(H, want[2], err_msg=label)
            np.testing.assert_array_equal(B, want[3], err_msg=label)
            assert torch.equal(g.basis(0, N).cpu(), Vd), label
            g.close()
    finally:
        F.foa_dmd_host_free(ptr)
    gd.close()
