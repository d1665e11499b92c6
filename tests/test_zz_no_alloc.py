"""foa_dmd_push_noalloc: the push for callers that cannot allocate device memory.

Such callers (memory arenas or pools that own the whole device, host applications that forbid
cudaMalloc on their hot path) hand in every buffer; the library keeps its per-push scratch in a
fixed device array.  These tests drive the entry point through the C ABI on caller-owned torch
buffers and check two calls in a row against the handle-based foa_dmd_push on the same
snapshots, for FP64 storage (within 1e-10) and for FP32 and BF16 storage (past j = 64, where
the passes hold a stage in registers and run two CTAs per SM; within the reduced-precision
parity bound C u_s kappa_2(X) of the other tests), and that a breakdown recorded in the
caller's H-bar makes the next call return ESTOPPED.  The file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}
PARITY_C = {"f32": 4.0, "bf16": 1.0}  # the reduced-precision parity constant of the other tests


def _buffers(n, K, dt):
    import torch
    sdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
    wdt = torch.float64 if dt == "f64" else torch.float32
    nrows = (n + 31) // 32 * 32
    V = torch.zeros(nrows * K, dtype=sdt, device="cuda")
    H = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    w = torch.zeros(nrows, dtype=wdt, device="cuda")
    return V, H, B, w, nrows


def _handle_state(X, n, K, dt, pushes):
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(n, K, dt)
    for u in range(pushes):
        assert g.push(X[u], info=False)[0] == 0
    q, _, Hr, Br = g.state()
    Vr = g.basis(0, q).double().cpu().numpy()
    g.close()
    return q, Hr, Br, Vr


def _tol(dt, Br, q):
    if dt == "f64":
        return 1e-10
    s = np.linalg.svd(Br[:q, :q], compute_uv=False)
    tol = PARITY_C[dt] * U[dt] * s[0] / s[-1]
    assert tol <= 1e-2
    return tol


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_noalloc_matches_push_two_calls_in_a_row(dt):
    import torch
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    if dt == "f64":
        spec = synth.config2(7, G=80, N=12)
        n, K = spec.n, 12
        Xh = synth.snapshots(spec)
    else:
        n, K = 9001, 100  # ragged last tile; j > 64 reaches the register-held passes
        Xh = np.random.default_rng(77).standard_normal((n, K))
    sdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
    X = torch.from_numpy(np.ascontiguousarray(Xh.T)).to(sdt).cuda()
    V, H, B, w, nrows = _buffers(n, K, dt)
    q = 0
    for t in range(K):
        st, info = F.foa_dmd_push_noalloc(n, K, dt, V, H, B, q, X[t], w)
        assert st == 0, F.STATUS.get(st, st)
        assert info.q == q + 1
        q = info.q
        if t in (K - 2, K - 1):  # two calls in a row checked against the handle-based push
            qr, Hr, Br, Vr = _handle_state(X, n, K, dt, t + 1)
            assert qr == q
            tol = _tol(dt, Br, q)
            Hn = H.cpu().numpy().T  # torch row-major (K, K) holds the column-major matrix transposed
            Bn = B.cpu().numpy().T
            assert np.linalg.norm(Hn - Hr) <= tol * np.linalg.norm(Hr)
            assert np.linalg.norm(Bn - Br) <= tol * np.linalg.norm(Br)
            Vt = V.view(nrows // 32, K, 32)
            Vn = Vt.permute(1, 0, 2).reshape(K, nrows)[:q, :n].double().cpu().numpy()
            assert np.linalg.norm(Vn - Vr) <= max(tol, 1e-12) * np.linalg.norm(Vr)
            print(f"{dt} call {t + 1}: bitwise equal to foa_dmd_push: "
                  f"{np.array_equal(Hn, Hr) and np.array_equal(Bn, Br) and np.array_equal(Vn, Vr)}")
    assert q == K
    # sizes beyond the fixed scratch are refused
    st, _ = F.foa_dmd_push_noalloc(n, 600, dt, V, H, B, 0, X[0], w)
    assert st == F.EINVAL


def test_noalloc_breakdown_then_stopped():
    """Planted rank-10 map (n = 4096): the 11th snapshot is dependent (EBREAKDOWN, q stays 10, h
    recorded in H-bar column 10); the next call with q = 10 returns ESTOPPED and changes nothing."""
    import torch
    from paper_1805_05821_gb300 import build, synth
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    spec = synth.config1(0)
    n, K = spec.n, 32
    X = torch.from_numpy(np.ascontiguousarray(synth.snapshots(spec).T)).cuda()
    V, H, B, w, _ = _buffers(n, K, "f64")
    q = 0
    sts = []
    for t in range(11):
        st, info = F.foa_dmd_push_noalloc(n, K, "f64", V, H, B, q, X[t], w)
        sts.append(st)
        if st == 0:
            q = info.q
    assert sts == [0] * 10 + [F.EBREAKDOWN] and q == 10
    Hb, Bb, Vb = H.clone(), B.clone(), V.clone()
    st, info = F.foa_dmd_push_noalloc(n, K, "f64", V, H, B, q, X[11], w)
    assert st == F.ESTOPPED and info.q == 10
    assert torch.equal(H, Hb) and torch.equal(B, Bb) and torch.equal(V, Vb)


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, which a stream capture does not allow: on a stream that is
    being captured it returns EINVAL before enqueueing anything, and the caller's buffers stay
    untouched (the capture itself goes on: the work after the call is captured as usual)."""
    import torch
    from paper_1805_05821_gb300 import build
    from paper_1805_05821_gb300 import foa_dmd as F
    build.build()
    n, K = 4096, 16
    V, H, B, w, _ = _buffers(n, K, "f32")
    x = torch.randn(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        st, _ = F.foa_dmd_push_noalloc(n, K, "f32", V, H, B, 0, x, w, stream=s)
        y = x * 2.0
    torch.cuda.synchronize()
    assert st == F.EINVAL
    assert int(torch.count_nonzero(H)) == 0 and int(torch.count_nonzero(B)) == 0
    assert int(torch.count_nonzero(V)) == 0 and int(torch.count_nonzero(w)) == 0
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, x * 2.0)
    # outside a capture the same call pushes
    st, info = F.foa_dmd_push_noalloc(n, K, "f32", V, H, B, 0, x, w, stream=s)
    s.synchronize()
    assert st == 0 and info.q == 1
