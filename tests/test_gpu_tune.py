"""The launch-geometry autotuner: it times candidates on the handle's own buffers, leaves the
stream empty, and the pushes that follow still match the oracle (the modified FOA update of Alg. 1)."""
import numpy as np
import pytest

from gpu_util import compare_state, run_oracle, to_device
from paper_1805_05821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


@pytest.mark.parametrize("reorth", [1, 2])
def test_autotune_then_push(tmp_path, reorth):
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    # 40 undamped waves with 1e-3 noise on a 128^2 grid (kappa_2 well below 1e-2 / u_fp32)
    spec = synth.waves(128, 2, 1, 40, 40, 31, sigma=None, noise_rel=1e-3)
    X = synth.snapshots(spec)
    Xr, Xd = to_device(X, "f32")
    cache = tmp_path / "tune.txt"
    g = FoaDMD(spec.n, 40, "f32", reorth=reorth, breakdown_tol=1e-9)
    g.autotune(cache)
    kinds = (3, 4) if reorth == 2 else (0, 1, 2)
    cands = {16384, 32768, 65536}
    for k in kinds:
        for j in (4, 20, 39):
            t = g.tuned_geometry(k, j)
            assert t["tuned"] and t["stage_bytes"] in cands and t["ctas_per_sm"] in (1, 2)
    q, stopped, H, B = g.state()
    assert q == 0 and not stopped and not H.any() and not B.any()
    assert not g.basis(0, 40).float().abs().sum().item()
    for t in range(40):
        assert g.push(Xd[t])[0] == 0
    o, _ = run_oracle(Xr, 40, "f32", tol=1e-9, reorth=reorth)
    compare_state(g, o, "f32", with_basis=True, label=f"after autotune reorth={reorth}")
    # a second handle reads the cache instead of timing again and picks the same geometry
    g2 = FoaDMD(spec.n, 40, "f32", reorth=reorth)
    g2.autotune(cache)
    for k in kinds:
        for j in (4, 20, 39):
            assert g2.tuned_geometry(k, j) == g.tuned_geometry(k, j)
    lines = cache.read_text().strip().splitlines()
    assert all(l.startswith("foa_dmd_tune ") for l in lines)


def test_autotune_refuses_a_nonempty_stream():
    import torch
    from paper_1805_05821_gb300.foa_dmd import FoaDMD, FoaError
    g = FoaDMD(4096, 8, "f32")
    g.push(torch.ones(4096, dtype=torch.float32, device="cuda"))
    with pytest.raises(FoaError):
        g.autotune()
