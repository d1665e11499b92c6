"""Batched streams (one persistent launch per push of every stream) against the FP64 oracle.

Streams of uneven n and k_max, FP32 storage, planted maps with noise (the batched workload's
recipe at small sizes, with 1e-3 instead of 1e-5 relative noise so that u_fp32 kappa_2(X) stays
below 1e-2); some streams sit out some pushes.  Each stream's beta and H-bar must match an
oracle run on the same rounded inputs column by column within C u_fp32 kappa_2(X_{1:p})
(gpu_util).
"""
import ctypes

import numpy as np
import pytest

from gpu_util import PARITY_C, PARITY_MAX_BOUND, U, compare_columns, kappa_of, rel, to_device
from paper_1805_05821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1805_05821_gb300 import build
    build.build()


def make_streams():
    rng = np.random.default_rng(3)
    out = []
    for s in range(6):
        n = int(rng.integers(500, 70000))
        N = int(rng.integers(10, 40))
        out.append(synth.planted(n, N, int(rng.integers(6, 12)) * 2, seed=100 + s, noise_rel=1e-3))
    return out


def oracle_state(Xr, k, dt="f32"):
    import oracle
    o = oracle.FoaOracle(Xr.shape[0], k, storage=dt)
    for t in range(Xr.shape[1]):
        if o.push(Xr[:, t])[0] != "ok":
            break
    return o


def run_batch(specs, skip, use_graph=False, Xs=None, dt="f32"):
    """Drive a batch round by round (graph replays or direct calls); specs give n and N, Xs (optional)
    the n x N snapshot matrices (else the specs' synthetic snapshots)."""
    import torch
    from paper_1805_05821_gb300 import foa_dmd as F
    S = len(specs)
    devs, hosts = [], []
    for i, sp in enumerate(specs):
        Xr, Xd = to_device(synth.snapshots(sp) if Xs is None else Xs[i], dt)
        hosts.append(Xr)
        devs.append(Xd)
    stream = torch.cuda.Stream()
    opts = F.foa_dmd_opts_default()
    opts.cuda_stream = stream.cuda_stream
    b = F.foa_dmd_batch_create([sp.n for sp in specs], [sp.N for sp in specs], dt, opts)
    ptrs = torch.zeros(S, dtype=torch.int64, device="cuda")
    hl = torch.zeros(S, dtype=torch.float64, device="cuda")
    T = max(sp.N for sp in specs) + 3
    pushed = [0] * S
    graph = None
    if use_graph:
        graph = torch.cuda.CUDAGraph()
    for r in range(T):
        host_ptrs = []
        for s, sp in enumerate(specs):
            if pushed[s] < sp.N and (r, s) not in skip:
                host_ptrs.append(int(devs[s][pushed[s]].data_ptr()))
                pushed[s] += 1
            else:
                host_ptrs.append(0)
        with torch.cuda.stream(stream):
            ptrs.copy_(torch.tensor(host_ptrs, dtype=torch.int64), non_blocking=False)
            if use_graph:
                if r == 0:
                    with torch.cuda.graph(graph, stream=stream):
                        rc = F.foa_dmd_batch_push(b, ptrs, hl)
                    assert rc == 0
                graph.replay()
            else:
                assert F.foa_dmd_batch_push(b, ptrs, hl) == 0
        stream.synchronize()
    return b, hosts


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_streams_match_oracle(use_graph):
    from paper_1805_05821_gb300 import foa_dmd as F
    specs = make_streams()
    skip = {(3, 1), (4, 1), (7, 4), (0, 5)}
    b, hosts = run_batch(specs, skip, use_graph)
    try:
        for s, sp in enumerate(specs):
            q, status, H, B = F.foa_dmd_batch_get_state(b, s, sp.N)
            o = oracle_state(hosts[s], sp.N)
            assert q == o.q, (s, q, o.q)
            compare_columns(q, o.m, H, B, o, "f32", label=f"stream {s} n={sp.n}")
    finally:
        F.foa_dmd_batch_destroy(b)


def test_batched_equals_single_stream_structure():
    """The same stream pushed alone (single-stream API) and inside a batch gives the same q and
    agrees to rounding (different summation orders)."""
    import torch
    from paper_1805_05821_gb300 import foa_dmd as F
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    sp = synth.planted(40000, 30, 16, seed=5, noise_rel=1e-3)
    Xr, Xd = to_device(synth.snapshots(sp), "f32")
    g = FoaDMD(sp.n, 30, "f32", breakdown_tol=1e-9)
    for t in range(30):
        assert g.push(Xd[t], info=False)[0] == 0
    opts = F.foa_dmd_opts_default()
    opts.breakdown_tol = 1e-9
    b = F.foa_dmd_batch_create([sp.n], [30], "f32", opts)
    ptrs = torch.zeros(1, dtype=torch.int64, device="cuda")
    for t in range(30):
        ptrs.fill_(int(Xd[t].data_ptr()))
        assert F.foa_dmd_batch_push(b, ptrs, None) == 0
    torch.cuda.synchronize()
    q1, _, H1, B1 = g.state()
    q2, st, H2, B2 = F.foa_dmd_batch_get_state(b, 0, 30)
    F.foa_dmd_batch_destroy(b)
    assert q1 == q2 == 30
    # two FP32 summation orders: agreement to C u_fp32 kappa_2(X), like the oracle comparisons
    tol = PARITY_C["f32"] * U["f32"] * kappa_of(B1, 30)
    assert tol <= PARITY_MAX_BOUND
    assert rel(B2, B1) <= tol and rel(H2[:30, :29], H1[:30, :29]) <= tol


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_batched_wide_bases(dt):
    """Bases up to 299 columns, so the pass items run every stage shape: R = 32 / 512 * j tiles,
    from 32 tiles (j <= 16) down to one tile (256 < j <= 299), the column groups from one per CTA to
    32 per CTA.  Gaussian snapshots (kappa_2 <= 1.5) of ragged lengths, one stream sitting out two
    rounds; against the oracle column by column (C u_s kappa_2, gpu_util)."""
    from types import SimpleNamespace
    from paper_1805_05821_gb300 import foa_dmd as F
    shapes = [(9001, 300), (4097, 140), (20000, 70), (777, 33)]
    specs = [SimpleNamespace(n=n, N=N) for n, N in shapes]
    Xs = [np.random.default_rng(50 + i).standard_normal((n, N)) for i, (n, N) in enumerate(shapes)]
    b, hosts = run_batch(specs, {(5, 2), (6, 2)}, use_graph=True, Xs=Xs, dt=dt)
    try:
        for s, sp in enumerate(specs):
            q, status, H, B = F.foa_dmd_batch_get_state(b, s, sp.N)
            o = oracle_state(hosts[s], sp.N, dt)
            assert q == o.q == sp.N, (s, q, o.q)
            import torch
            from gpu_util import torch_dtype
            Vd = torch.empty((q, sp.n), dtype=torch_dtype(dt), device="cuda")
            F.foa_dmd_batch_get_basis(b, s, 0, q, Vd, sp.n)
            V = Vd.double().cpu().numpy().T
            compare_columns(q, o.m, H, B, o, dt, V=V, label=f"batched stream {s} n={sp.n}")
    finally:
        F.foa_dmd_batch_destroy(b)


def test_batched_statuses_follow_the_oracle():
    """Per-stream statuses inside one batch (Sec. 3.2.4 and reading 4 of the breakdown test): a
    noise-free planted rank-6 map breaks down at push 7 and stays stopped while the batch goes on;
    a snapshot holding a NaN is refused (state unchanged) and the stream continues with the next
    one; a Gaussian stream is unaffected.  States against the oracle fed the same sequences (the
    oracle skips the refused snapshot as the batch does)."""
    import torch
    from types import SimpleNamespace
    from paper_1805_05821_gb300 import foa_dmd as F
    import oracle
    planted = synth.planted(6000, 12, 6, seed=77, noise_rel=0.0)
    Xp = synth.snapshots(planted)
    Xn = np.random.default_rng(78).standard_normal((5000, 12))
    Xn[123, 4] = np.nan                               # the fifth snapshot of stream 1 is refused
    Xg = np.random.default_rng(79).standard_normal((7000, 12))
    specs = [SimpleNamespace(n=6000, N=12), SimpleNamespace(n=5000, N=12), SimpleNamespace(n=7000, N=12)]
    b, hosts = run_batch(specs, set(), use_graph=True, Xs=[Xp, Xn, Xg])
    try:
        # stream 0: breakdown at push 7, q = 6, stopped (status of its last push EBREAKDOWN or ESTOPPED)
        q, status, H, B = F.foa_dmd_batch_get_state(b, 0, 12)
        o = oracle.FoaOracle(6000, 12, storage="f32")
        sts = [o.push(hosts[0][:, t])[0] for t in range(12)]
        assert sts[:6] == ["ok"] * 6 and sts[6] == "breakdown" and o.q == 6
        assert q == 6 and status in (F.EBREAKDOWN, F.ESTOPPED), (q, status)
        assert H[6, 5] == 0.0 and np.any(H[:6, 5] != 0.0)
        compare_columns(q, o.m, H, B, o, "f32", label="batched breakdown stream")
        # stream 1: the NaN snapshot is refused, the other 11 are pushed
        q, status, H, B = F.foa_dmd_batch_get_state(b, 1, 12)
        o = oracle.FoaOracle(5000, 12, storage="f32")
        sts = [o.push(hosts[1][:, t])[0] for t in range(12)]
        assert sts[4] == "nonfinite" and o.q == 11
        assert q == 11 and status == F.OK, (q, status)
        compare_columns(q, o.m, H, B, o, "f32", label="batched NaN stream")
        # stream 2: all 12
        q, status, H, B = F.foa_dmd_batch_get_state(b, 2, 12)
        o = oracle_state(hosts[2], 12)
        assert q == o.q == 12 and status == F.OK
        compare_columns(q, o.m, H, B, o, "f32", label="batched Gaussian stream")
    finally:
        F.foa_dmd_batch_destroy(b)
