"""Helpers shared by the GPU tests: device copies of host snapshots and oracle comparisons."""
import numpy as np

import oracle

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}


def torch_dtype(dt):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]


def to_device(X, dt):
    """X (n x N, float64) -> (rounded host copy in FP64, device tensor (N, n) in the storage dtype)."""
    import torch
    T = torch.from_numpy(np.ascontiguousarray(X.T)).to(torch_dtype(dt))
    Xr = T.double().numpy().T.copy()
    return Xr, T.cuda()


def kappa_of(B, q):
    s = np.linalg.svd(B[:q, :q], compute_uv=False)
    return s[0] / s[-1]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run_gpu(X_dev, n, k_max, dt, **kw):
    from paper_1805_05821_gb300.foa_dmd import FoaDMD
    g = FoaDMD(n, k_max, dt, **kw)
    infos = []
    for t in range(X_dev.shape[0]):
        st, inf = g.push(X_dev[t])
        infos.append((st, inf))
        if st != 0:
            break
    return g, infos


def run_oracle(Xr, k_max, dt, tol=None, reorth=1):
    o = oracle.FoaOracle(Xr.shape[0], k_max, breakdown_tol=tol, storage=dt, reorth=reorth)
    sts = []
    for t in range(Xr.shape[1]):
        st = o.push(Xr[:, t])
        sts.append(st)
        if st[0] != "ok":
            break
    return o, sts


def match(a, b):
    from scipy.optimize import linear_sum_assignment
    D = np.abs(a[:, None] - b[None, :])
    ri, ci = linear_sum_assignment(D)
    return D[ri, ci], ci
