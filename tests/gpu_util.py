"""Helpers shared by the GPU tests: device copies of host snapshots and oracle comparisons.

Reduced-precision parity law (FP32/BF16 storage against the FP64 oracle on the same
storage-rounded inputs).  Sec. 3.2.2 (Eq. foabaseddmdberr and App. B) bounds the error of the
projected matrix by a modest multiple of the unit roundoff times kappa_2(X).  Read column by
column: column c of beta (and of V) comes from the push of snapshot c+1, column c of H-bar from the
push of snapshot c+2, so each is compared with

    ||delta col|| / ||col||  <=  C * u_s * kappa_2(X_{1:p})          (p = the pushes it depends on)

with C = PARITY_C[dtype] (a fixed constant that does not grow with k_max), u_s the unit roundoff
of the storage type and kappa_2(X_{1:p}) the condition number of the leading p x p block of the
oracle's beta (beta's leading block is the R factor of X_{1:p}, Sec. 3.1).  C is 4 for FP32 and 1
for BF16 storage: every stored basis vector carries a rounding error of up to u_s, and with FP32
storage the FP32 products and row sweeps add errors of the same unit roundoff (measured columns
reach 1.5 u kappa), while with BF16 storage the FP32 arithmetic is 2^-16 times finer than the
storage and only the storage rounding shows (measured columns reach 0.47 u kappa).  A comparison
is only meaningful when the bound is well below one: every reduced-precision case asserts
C u_s kappa <= 1e-2 first (PARITY_MAX_BOUND), so the inputs of such cases are chosen well
conditioned.  Ill-conditioned sequences are compared through their leading eigenvalues after
rank truncation (compare_eigs), where the retained part has kappa_2 = sigma_1/sigma_r <= 1/rank_tol.

FP64 storage: normwise on beta and H-bar within max(1e-10, 4 u_64 kappa_2(X)) (fp64_tol), the
same law with the FP64 unit roundoff; the floor 1e-10 covers every well-conditioned case.
"""
import numpy as np

import oracle

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}
PARITY_C = {"f64": 4.0, "f32": 4.0, "bf16": 1.0}  # C of the law above, per storage type
PARITY_MAX_BOUND = 1e-2  # a bound above this could not catch an error of a few percent
FP64_TOL = 1e-10         # FP64 storage: floor of the normwise bound on beta and H-bar


def fp64_tol(kappa):
    """FP64-storage bound max(1e-10, C u_64 kappa_2(X)) on the normwise beta and H-bar errors."""
    return max(FP64_TOL, PARITY_C["f64"] * U["f64"] * kappa)


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


def leading_kappas(B, q):
    """kap[p] >= kappa_2 of the leading p x p block of beta, p = 1..q (kap[0] unused).

    Exact on a grid of p (every p up to 64, then every 8th, and q); between grid points the next
    grid value is used, which bounds it from above: the singular values of a leading block of R
    interlace those of the larger block, so kappa_2 never decreases with p."""
    grid = sorted(set(list(range(1, min(q, 64) + 1)) + list(range(64, q + 1, 8)) + [q]))
    vals = {p: kappa_of(B, p) for p in grid}
    kap = np.zeros(q + 1)
    nxt = q
    for p in range(q, 0, -1):
        if p in vals:
            nxt = p
        kap[p] = vals[nxt]
    return kap


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def col_rel(a, b):
    """Relative 2-norm error of every column of a against b (columns of zero norm: absolute)."""
    nb = np.linalg.norm(b, axis=0)
    return np.linalg.norm(a - b, axis=0) / np.where(nb > 0, nb, 1.0)


def compare_columns(q, m, H, B, o, dt, V=None, C=None, label=""):
    """Column-by-column parity of beta, H-bar (and V when given, n x q) with the oracle `o` under
    the reduced-precision law of this module; returns the largest error/bound ratio."""
    assert q == o.q
    C = PARITY_C[dt] if C is None else C
    kap = leading_kappas(o.B, q)
    u = U[dt]
    bB = C * u * kap[1:q + 1]                                     # beta and V column c: X_{1:c+1}
    bH = C * u * kap[np.minimum(np.arange(m) + 2, q)]             # H-bar column c: X_{1:c+2}
    worst = max(bB.max(), bH.max() if m else 0.0)
    assert worst <= PARITY_MAX_BOUND, f"{label}: bound {worst:.3g} too loose to pin anything (kappa {kap[q]:.3g})"
    eB = np.array([np.linalg.norm(B[:c + 1, c] - o.B[:c + 1, c]) / np.linalg.norm(o.B[:c + 1, c])
                   for c in range(q)])
    eH = np.array([np.linalg.norm(H[:c + 2, c] - o.H[:c + 2, c]) / max(np.linalg.norm(o.H[:c + 2, c]), 1e-300)
                   for c in range(m)])
    ratios = [np.max(eB / bB)]
    if m:
        ratios.append(np.max(eH / bH))
    bad_B = np.where(eB > bB)[0]
    bad_H = np.where(eH > bH)[0] if m else []
    msg = f"{label} {dt}: kappa {kap[q]:.3g}, max err/bound beta {ratios[0]:.3g}"
    if m:
        msg += f", H-bar {ratios[1]:.3g}"
    if V is not None:
        eV = col_rel(V[:, :q], o.V[:, :q])
        ratios.append(np.max(eV / bB))
        msg += f", V {ratios[-1]:.3g}"
        bad_V = np.where(eV > bB)[0]
    else:
        bad_V = []
    print(msg, f"(bound at the last column {bB[-1]:.3g})")
    assert len(bad_B) == 0, (label, "beta columns", bad_B[:8], eB[bad_B[:8]], bB[bad_B[:8]])
    assert len(bad_H) == 0, (label, "H-bar columns", bad_H[:8], eH[bad_H[:8]], bH[bad_H[:8]])
    assert len(bad_V) == 0, (label, "V columns", bad_V[:8])
    return max(ratios)


def compare_state(g, o, dt, k_max=None, q_expect=None, with_basis=False, label=""):
    """GPU handle g against oracle o: FP64 storage normwise within fp64_tol(kappa_2(X)); FP32/BF16
    storage column by column (compare_columns).  V is compared too when with_basis is set."""
    q, stopped, H, B = g.state()
    assert q == o.q and stopped == o.stopped
    if q_expect is not None:
        assert q == q_expect
    m = o.m
    V = g.basis(0, q).double().cpu().numpy().T if (with_basis and q > 0) else None
    if dt == "f64":
        tol = fp64_tol(kappa_of(o.B, q)) if q > 0 else FP64_TOL
        eB = rel(B[:q, :q], o.B[:q, :q])
        eH = rel(H[:m + 1, :m], o.H[:m + 1, :m]) if m >= 1 else 0.0
        assert eB <= tol, (eB, tol)
        assert eH <= tol, (eH, tol)
        if V is not None:
            assert rel(V, o.V[:, :q]) <= tol
        return max(eB, eH) / tol
    return compare_columns(q, m, H, B, o, dt, V=V, label=label)


def eig_condition(G):
    """Eigenvalues of G and their condition s_i = |y_i^H z_i| / (||y_i|| ||z_i||)."""
    import scipy.linalg
    w, vl, vr = scipy.linalg.eig(G, left=True, right=True)
    s = np.abs(np.sum(np.conj(vl) * vr, axis=0)) / (np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0))
    return w, s


def compare_eigs(res_g, res_o, dt, n_lead, C=None, label=""):
    """Leading eigenvalues (the first n_lead of the oracle's |c| order) of a truncated eig against
    the oracle's on the same rounded inputs.  First-order perturbation of a simple eigenvalue:
    |d lambda_i| <= ||dG||_2 / s_i, and the retained part of the projected matrix obeys the law
    of this module with kappa_2 = sigma_1/sigma_r of the oracle's retained singular values, so

        |d lambda_i| <= C u_s (sigma_1/sigma_r) ||G||_2 / s_i       (C u_s sigma_1/sigma_r <= 1e-2).

    Every GPU eigenvalue may match only one oracle eigenvalue (optimal assignment)."""
    C = PARITY_C[dt] if C is None else C
    u = U[dt]
    sig = res_o["sigma"]
    r = res_o["r"]
    kap_r = sig[0] / sig[r - 1] if sig is not None else 1.0
    assert C * u * kap_r <= PARITY_MAX_BOUND, (label, C * u * kap_r)
    lam_o = res_o["lam"][:n_lead]
    w, s = eig_condition(res_o["G"])
    d_w, pw = match(lam_o, w)
    s_o = s[pw]
    d, perm = match(lam_o, res_g["lam"])
    nrm = np.linalg.norm(res_o["G"], 2)
    tol = C * u * kap_r * nrm / np.maximum(s_o, 1e-300)
    print(f"{label} {dt}: leading {n_lead} eigenvalues, r {res_g['r']}/{r}, kappa_r {kap_r:.3g}, "
          f"max |dlambda|/|lambda| {np.max(d / np.abs(lam_o)):.3g}, max err/tol {np.max(d / tol):.3g}")
    assert np.all(d <= tol), (label, d, tol)
    return perm


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


def gaussian(n, N, seed):
    """n x N independent Gaussian snapshots: kappa_2(X) ~ (1 + sqrt(N/n)) / (1 - sqrt(N/n)), the
    well-conditioned input on which the BF16 law can be asserted (u_bf16 = 2^-8)."""
    return np.random.default_rng(seed).standard_normal((n, N))
