"""foa_dmd_push_noalloc: the push for callers that cannot allocate device memory.

Such callers (memory arenas that own the whole device, host applications that forbid cudaMalloc
on their hot path) hand in every buffer; the library keeps its per-push scratch in a fixed
device array.  This test drives the entry point through the C ABI on caller-owned torch
buffers and checks two calls in a row against the handle-based foa_dmd_push on the same
snapshots: same launches, so the state must agree (bitwise here, within the FP64 parity
tolerance of 1e-10 at least).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_push_two_calls_in_a_row():
    import torch
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    build.build()
    spec = synth.config2(7, G=80, N=12)
    n, K = spec.n, 12
    X = torch.from_numpy(np.ascontiguousarray(synth.snapshots(spec).T)).cuda()
    # reference: the handle-based push
    g = FoaDMD(n, K, "f64")
    for t in range(K):
        assert g.push(X[t], info=False)[0] == 0
    q_ref, _, H_ref, B_ref = g.state()
    # caller-owned buffers
    nrows = (n + 31) // 32 * 32
    V = torch.zeros(nrows * K, dtype=torch.float64, device="cuda")
    H = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    w = torch.zeros(nrows, dtype=torch.float64, device="cuda")
    q = 0
    for t in range(K):
        st, info = F.foa_dmd_push_noalloc(n, K, "f64", V, H, B, q, X[t], w)
        assert st == 0, F.STATUS.get(st, st)
        assert info.q == q + 1
        q = info.q
        if t in (K - 2, K - 1):  # two calls in a row checked against the reference state
            Hn = H.cpu().numpy().T  # torch row-major (K, K) holds the column-major matrix transposed
            Bn = B.cpu().numpy().T
            g2 = FoaDMD(n, K, "f64")
            for u in range(t + 1):
                g2.push(X[u], info=False)
            _, _, Hr, Br = g2.state()
            g2.close()
            assert np.linalg.norm(Hn - Hr) <= 1e-10 * np.linalg.norm(Hr)
            assert np.linalg.norm(Bn - Br) <= 1e-10 * np.linalg.norm(Br)
    assert q == q_ref == K
    np.testing.assert_allclose(H.cpu().numpy().T, H_ref, rtol=0, atol=1e-10 * np.abs(H_ref).max())
    np.testing.assert_allclose(B.cpu().numpy().T, B_ref, rtol=0, atol=1e-10 * np.abs(B_ref).max())
    Vg = g.basis(0, K).cpu().numpy()
    Vt = V.view(nrows // 32, K, 32)
    Vn = Vt.permute(1, 0, 2).reshape(K, nrows)[:, :n].cpu().numpy()
    np.testing.assert_allclose(Vn, Vg, rtol=0, atol=1e-12)
    # sizes beyond the fixed scratch are refused
    st, _ = F.foa_dmd_push_noalloc(n, 600, "f32", V, H, B, 0, X[0], w)
    assert st == F.EINVAL
