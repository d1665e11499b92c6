"""GPU parity of the QR view of the push (form = 1) against the oracle's QR view.

The QR view orthogonalises each snapshot directly (h = V^T psi, CGS2), stores beta's column as
[h; nu] and forms the Hbar column from beta_{:,2:} = Hbar beta (Eq. matmulhbeta).  Tolerances
as in test_gpu_push: FP64 1e-10 normwise, FP32/BF16 column by column within
C u_s kappa_2(X_{1:p}) <= 1e-2 (gpu_util).
"""
import numpy as np
import pytest

from gpu_util import compare_state, gaussian, match, run_gpu, to_device
from paper_1805_05821_gb300 import synth
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


def run_oracle_qr(Xr, k_max, dt, reorth=1):
    o = oracle.FoaOracle(Xr.shape[0], k_max, storage=dt, reorth=reorth, form="qr")
    sts = []
    for t in range(Xr.shape[1]):
        st = o.push(Xr[:, t])
        sts.append(st)
        if st[0] != "ok":
            break
    return o, sts


def compare(g, o, dt, k_max=None, label="QR view"):
    return compare_state(g, o, dt, with_basis=True, label=label)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_qr_view_matches_oracle(dt):
    """Damped waves on a 72^2 grid (kappa_2 = 126) for FP64 and FP32, Gaussian snapshots of the
    same shape for BF16."""
    spec = synth.config2(21, G=72, N=28)
    X = synth.snapshots(spec) if dt != "bf16" else gaussian(spec.n, 28, 21)
    Xr, Xd = to_device(X, dt)
    g, infos = run_gpu(Xd, spec.n, 28, dt, form=1)
    o, sts = run_oracle_qr(Xr, 28, dt)
    assert [s for s, _ in infos] == [0 if s[0] == "ok" else 5 for s in sts]
    if dt == "f64":
        for (st, inf), so in zip(infos, sts):
            assert abs(inf["h_last"] - so[1]) <= 1e-10 * abs(so[1])
    compare(g, o, dt, 28)


def test_qr_view_cgs1_fp64():
    spec = synth.config2(22, G=48, N=20)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, _ = run_gpu(Xd, spec.n, 20, "f64", form=1, reorth=0)
    o, _ = run_oracle_qr(Xr, 20, "f64", reorth=0)
    compare(g, o, "f64", 20)


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_qr_view_ragged_fp64(n):
    rng = np.random.default_rng(200 + n)
    N = 12 if n > 12 else n + 1
    X = rng.standard_normal((n, N))
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, n, N, "f64", form=1)
    o, sts = run_oracle_qr(Xr, N, "f64")
    assert [s for s, _ in infos] == [0 if s[0] == "ok" else 5 for s in sts]
    compare(g, o, "f64", N)


def test_qr_view_breakdown_and_eig():
    """Planted rank-10 map: breakdown at push 11 and the planted eigenvalues from the QR view."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, infos = run_gpu(Xd, spec.n, 32, "f64", form=1)
    assert len(infos) == 11 and infos[-1][0] == 5
    o, _ = run_oracle_qr(Xr, 32, "f64")
    compare(g, o, "f64", 32)
    r = g.eig(0.0)
    d, _ = match(r["lam"], spec.lam)
    assert r["status"] == 0 and d.max() <= 1e-9


def test_qr_view_rejects_two_pass():
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    with pytest.raises(RuntimeError):
        FoaDMD(1000, 8, "f32", form=1, reorth=2)
