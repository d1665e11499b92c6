"""GPU parity of the block push (block CGS2 against V + Cholesky QR twice; the block form of the QR
view) against the oracle's block step on the same blocking.  Tolerances as in test_gpu_push:
column by column within C u_s kappa_2(X_{1:p}) <= 1e-2 (gpu_util), against the FP64 oracle on
the same storage-rounded inputs."""
import numpy as np
import pytest

from gpu_util import PARITY_C, U, compare_state, gaussian, kappa_of, rel, to_device
from paper_1805_05821_gb300 import synth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


def oracle_blocks(Xr, k_max, dt, block, tol=None):
    """First snapshot alone, then blocks of `block` (the library's blocking for (N-1) % block == 0)."""
    o = oracle.FoaOracle(Xr.shape[0], k_max, breakdown_tol=tol, storage=dt, form="qr")
    sts = [o.push(Xr[:, 0])]
    for s in range(1, Xr.shape[1], block):
        sts += o.push_block(Xr[:, s:s + block])
        if o.stopped:
            break
    return o, sts


def compare(g, o, dt, k_max=None, label="block push"):
    return compare_state(g, o, dt, with_basis=True, label=label)


@pytest.mark.parametrize("dt,block", [("f32", 4), ("f32", 2), ("bf16", 4), ("bf16", 2)])
def test_block_push_matches_oracle(dt, block):
    """n = 4900 (ragged last tile), 25 snapshots = 1 + 6 blocks of 4: damped waves on a 70^2 grid
    for FP32 (kappa_2 = 14), Gaussian snapshots for BF16."""
    spec = synth.config2(41, G=70, N=25)
    X = synth.snapshots(spec) if dt == "f32" else gaussian(spec.n, 25, 41)
    Xr, Xd = to_device(X, dt)
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(spec.n, 25, dt)
    import torch
    ld = (spec.n + 7) // 8 * 8  # rows 16-byte aligned for every storage type
    Xp = torch.zeros((25, ld), dtype=Xd.dtype, device="cuda")
    Xp[:, :spec.n] = Xd
    st, infos = g.push_block(Xp, block=block)
    assert st == 0
    o, sts = oracle_blocks(Xr, 25, dt, block)
    assert [i["status"] for i in infos] == ["OK" if s[0] == "ok" else "EBREAKDOWN" for s in sts][:len(infos)]
    compare(g, o, dt, 25)
    # the block push agrees with single pushes to the same tolerance
    g1 = FoaDMD(spec.n, 25, dt)
    for t in range(25):
        g1.push(Xd[t])
    q, _, H1, B1 = g1.state()
    kap = kappa_of(o.B, q)
    assert rel(g.state()[3][:q, :q], B1[:q, :q]) <= PARITY_C[dt] * U[dt] * kap


def test_block_push_breakdown_inside_a_block():
    """Planted rank-10 map (FP32 storage): snapshot 11 is the second column of the third block of 4;
    the library commits the block's first column and stops, like the oracle."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f32")
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(spec.n, 32, "f32")
    st, infos = g.push_block(Xd[:29], block=4)
    assert st == 5  # EBREAKDOWN
    assert [i["status"] for i in infos[:10]] == ["OK"] * 10 and infos[10]["status"] == "EBREAKDOWN"
    assert all(i["status"] == "ESTOPPED" for i in infos[11:])
    o, sts = oracle_blocks(Xr, 32, "f32", 4)
    q, stopped, H, B = g.state()
    assert q == o.q == 10 and stopped
    assert H[10, 9] == 0.0
    r = g.eig(0.0)
    from gpu_util import match
    d, _ = match(r["lam"], spec.lam)
    assert d.max() <= 1e-4


def test_block_push_on_a_two_pass_handle_and_fp64_refused():
    import torch
    from paper_1805_05821_gb300.foa_dmd import FoaDMD, FoaError
    spec = synth.config2(42, G=48, N=13)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f32")
    g = FoaDMD(spec.n, 13, "f32", reorth=2)
    for t in range(5):
        assert g.push(Xd[t])[0] == 0
    st, infos = g.push_block(Xd[5:13], block=4)
    assert st == 0 and g.state()[0] == 13
    o = oracle.FoaOracle(spec.n, 13, storage="f32", reorth=2)
    for t in range(5):
        o.push(Xr[:, t])
    o.form = "qr"
    o.push_block(Xr[:, 5:9])
    o.push_block(Xr[:, 9:13])
    compare(g, o, "f32", 13)
    g64 = FoaDMD(1000, 8, "f64")
    x = torch.zeros((4, 1000), dtype=torch.float64, device="cuda")
    assert g64.push_block(x, block=4)[0] == 1  # EINVAL


def test_block_push_stops_at_its_resolution_limit_on_fields():
    """The fields workload's structure at a small grid (4 x 16^3, n = 16384), N = 384, breakdown_tol
    1e-12: after the 96 wave dimensions every snapshot adds only its 1e-7 noise (R_ii about 7 u_fp32
    ||psi||).  Without a limit the block push lost the orthogonality of V near column 250 and
    H-bar diverged, while reporting OK.  Now the block push stops with ERESOLVE at the first
    snapshot whose R_ii < 16 u_fp32 ||psi||, having committed the columns before it (past j = 128,
    where a pipeline stage is one 32-row tile and the row sweep splits the columns into 16 groups);
    the rest go through the single push (Alg. 1 form).  V stays orthogonal and the leading Ritz
    values match the planted eigenvalues; the block part matches the oracle's block step."""
    import torch
    from scipy.optimize import linear_sum_assignment
    from paper_1805_05821_gb300.foa_dmd import ERESOLVE, FoaDMD
    spec = synth.config5(0, G=16, N=384)
    X = synth.snapshots(spec, np.float32).astype(np.float64)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).float().cuda()
    g = FoaDMD(spec.n, 384, "f32", breakdown_tol=1e-12)
    st, infos = g.push_block(Xd, block=4)
    assert st == ERESOLVE, st
    t0 = next(t for t, i in enumerate(infos) if i["status"] != "OK")
    assert all(i["status"] == "ERESOLVE" for i in infos[t0:])
    q, stopped, H, B = g.state()
    assert q == t0 and not stopped and 128 < t0 < 250, t0
    assert infos[t0]["x_norm"] > 0
    # the block part against the oracle's block step on the same blocking
    o = oracle.FoaOracle(spec.n, 384, breakdown_tol=1e-12, storage="f32", form="qr")
    o.push(X[:, 0])
    s = 1
    while s + 4 <= t0:
        o.push_block(X[:, s:s + 4])
        s += 4
    if s < t0:
        o.push_block(X[:, s:t0])
    assert o.q == t0
    Vg = g.basis(0, q).double().cpu().numpy().T
    assert np.linalg.norm(np.eye(q) - Vg.T @ Vg, 2) <= 1e-5
    # normwise within the reduced-precision law (kappa_2 is large here, so this is no tight pin:
    # the columns of the ill-conditioned part are pinned by the orthogonality check above)
    eB = np.linalg.norm(B[:q, :q] - o.B[:q, :q]) / np.linalg.norm(o.B[:q, :q])
    assert eB <= PARITY_C["f32"] * U["f32"] * kappa_of(o.B, q), (eB, kappa_of(o.B, q))
    # the rest singly: the stream was not stopped
    for t in range(t0, 384):
        assert g.push(Xd[t], info=False)[0] == 0
    q, stopped, H, B = g.state()
    assert q == 384 and not stopped
    Vg = g.basis(0, q).double().cpu().numpy().T
    orth = np.linalg.norm(np.eye(q) - Vg.T @ Vg, 2)
    assert orth <= 1e-5, orth
    r = g.eig(-1.0)
    lam = r["lam"][:32]
    D = np.abs(lam[:, None] - spec.lam[None, :])
    ri, ci = linear_sum_assignment(D)
    err = np.max(D[ri, ci] / np.abs(spec.lam[ci]))
    print(f"block push stopped at {t0}; orthogonality {orth:.2e}; leading 32 vs planted {err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("dt,block", [("f32", 4), ("f32", 2), ("bf16", 4), ("bf16", 2)])
def test_block_push_widest_basis(dt, block):
    """n = 4097 Gaussian snapshots (ragged last tile), N = 421 = 1 + 105 blocks of 4: the block
    passes run in every shape (256-thread CTAs with two, four or eight columns a thread up to
    j = 256, one 512-thread CTA per SM with eight columns a thread beyond)."""
    import torch
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    n, N = 4097, 421
    X = np.random.default_rng(421).standard_normal((n, N))
    Xr, Xd = to_device(X, dt)
    ld = (n + 7) // 8 * 8
    Xp = torch.zeros((N, ld), dtype=Xd.dtype, device="cuda")
    Xp[:, :n] = Xd
    g = FoaDMD(n, N, dt)
    st, infos = g.push_block(Xp, block=block)
    assert st == 0
    o, sts = oracle_blocks(Xr, N, dt, block)
    assert all(s[0] == "ok" for s in sts)
    compare(g, o, dt, N)
