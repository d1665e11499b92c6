"""The failure path of the bounded device waits, made to run out without faulting anything.

Every spin of the library's kernels (pipeline mbarriers, grid barriers, cross-CTA flags) gives up
after a bounded number of clock cycles, records FOA_DMD_ETIMEOUT and returns.  Here one CTA of the
cooperative Jacobi SVD of a truncated eig returns before its first grid-barrier arrival (the test
hook foa_dmd_test_wait_fault), as a CTA that died would; the other CTAs spin for 2^22 cycles (about
2 ms), give up and return.  Nothing waits without a limit downstream: the waiting threads of each
CTA sit at a block barrier that thread 0 reaches once its bounded spin ends, and the kernels after
the SVD (rank count, projection, Hessenberg reduction, QR iteration with at most 60 sweeps per
eigenvalue, inverse iteration, ordering) run fixed loop counts.  The eig must report ETIMEOUT and
leave the stream state untouched; the next eig, and a reset followed by new pushes, must give the
oracle's results again.
"""
import numpy as np
import pytest

from gpu_util import match, run_gpu, run_oracle, to_device
from paper_1805_05821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


def test_grid_barrier_timeout_reports_and_recovers():
    from paper_1805_05821_gb300.foa_dmd import EINVAL, ETIMEOUT
    spec = synth.planted(20000, 30, 12, seed=6, noise_rel=1e-10)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f64")
    g, _ = run_gpu(Xd, spec.n, 30, "f64", breakdown_tol=1e-14)
    o, _ = run_oracle(Xr, 30, "f64", tol=1e-14)
    q0, s0, H0, B0 = g.state()
    ro = o.eig(1e-7)
    assert g.test_wait_fault(-1, 1 << 22) == EINVAL
    assert g.test_wait_fault(3, 0) == EINVAL
    assert g.test_wait_fault(3, 1 << 22) == 0
    bad = g.eig(1e-7)
    assert bad["status"] == ETIMEOUT, bad["status"]
    q1, s1, H1, B1 = g.state()
    assert q1 == q0 and s1 == s0 and np.array_equal(H1, H0) and np.array_equal(B1, B0)
    # the next eig runs normally and matches the oracle
    good = g.eig(1e-7)
    assert good["status"] == 0 and good["r"] == ro["r"] == 12
    d, _ = match(ro["lam"], good["lam"])
    assert d.max() <= 1e-9
    # and after a reset the handle streams again
    g.reset()
    for t in range(30):
        assert g.push(Xd[t], info=False)[0] == 0
    again = g.eig(1e-7)
    assert again["status"] == 0
    assert np.array_equal(again["lam"], good["lam"])
    g.close()
