"""Pins of the FP64 CPU oracle to what the paper and the mathematics fix (no GPU).

Each test states the passage it follows.  None of them retypes the oracle's own formula: they
use closed forms derived by hand, the Arnoldi method with the generating matrix known
(Algorithm 2), LAPACK's SVD-based DMD, least-squares companion matrices, invariants of
Sec. 3.2.2 and the error law of Eq. (foabaseddmdberr).  ``test_mutants_are_caught`` plants
mistakes in copies of the oracle's C source and checks that the pins fail on them.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg
from scipy.optimize import linear_sum_assignment

import oracle
from paper_1805_05821_gb300 import synth

U64 = 2.0 ** -53


def match_eigs(a, b):
    """Optimal one-to-one matching of two eigenvalue sets; returns the matched distances."""
    D = np.abs(a[:, None] - b[None, :])
    ri, ci = linear_sum_assignment(D)
    return D[ri, ci], ci


def run_oracle(X, k_max=None, tol=None, library=None, reorth=1, form="foa"):
    return oracle.run(X, k_max, tol, "f64", reorth, library, form)


# ------------------------------------------------------------------ closed forms
def test_two_snapshot_closed_form():
    """N = 2 (Alg. 1 with one step): h11 = <p1,p2>/|p1|^2, h21 = |p2 - h11 p1|/|p1|,
    beta12 = <p1,p2>/|p1|, beta22 = |p2 - h11 p1| (derived by hand from the update of Alg. 1)."""
    rng = np.random.default_rng(7)
    p1, p2 = rng.standard_normal(1000), rng.standard_normal(1000)
    o = run_oracle(np.stack([p1, p2], axis=1))
    b = np.linalg.norm(p1)
    h11 = p1 @ p2 / b ** 2
    r = np.linalg.norm(p2 - h11 * p1)
    assert o.q == 2
    np.testing.assert_allclose(o.B[0, 0], b, rtol=1e-15)
    np.testing.assert_allclose(o.H[0, 0], h11, rtol=1e-13)
    np.testing.assert_allclose(o.H[1, 0], r / b, rtol=1e-13)
    np.testing.assert_allclose(o.B[0, 1], p1 @ p2 / b, rtol=1e-13)
    np.testing.assert_allclose(o.B[1, 1], r, rtol=1e-13)
    np.testing.assert_allclose(o.V[:, 0], p1 / b, rtol=1e-14)


def test_single_snapshot_and_zero_snapshot():
    """First snapshot of Alg. 1: beta11 = |psi1|, v1 = psi1/|psi1|; a zero snapshot cannot start a basis."""
    x = np.arange(1.0, 11.0)
    o = oracle.FoaOracle(10, 4)
    st, h, xn = o.push(x)
    assert st == "ok" and o.q == 1
    assert h == pytest.approx(np.sqrt(385.0), rel=1e-15)
    np.testing.assert_allclose(o.V[:, 0] * np.sqrt(385.0), x, rtol=1e-15)
    o2 = oracle.FoaOracle(10, 4)
    assert o2.push(np.zeros(10))[0] == "breakdown"
    assert o2.push(x)[0] == "stopped"


# ------------------------------------------------------------------ invariants (Sec. 3.2.2, App. B)
@pytest.mark.parametrize("spec_fn", [lambda: synth.config1(1), lambda: synth.config2(0, G=64, N=40)])
def test_orthogonality_and_factorisation(spec_fn):
    """||I - V^T V||_2 <= c2 eps (Eq. qrfactorth), ||X - V beta||_F <= c1 eps ||X||_F
    (Eqs. qrfactbstab/errorinfact), beta_{1:N,2:N} = Hbar_N beta_{N-1} (Eq. matmulhbeta)."""
    spec = spec_fn()
    X = synth.snapshots(spec)
    o = run_oracle(X)
    q = o.q
    k = X.shape[1]
    V, B, H = o.V[:, :q], o.B[:q, :q], o.H
    assert np.linalg.norm(np.eye(q) - V.T @ V, 2) <= 10 * k * U64
    assert np.linalg.norm(X[:, :q] - V @ B) <= 10 * k * U64 * np.linalg.norm(X[:, :q])
    Nn = q
    lhs = B[:Nn, 1:Nn]
    rhs = H[:Nn, :Nn - 1] @ B[:Nn - 1, :Nn - 1]
    gam = (Nn - 1) * U64 / (1 - (Nn - 1) * U64)
    bound = gam * np.sqrt(Nn) * np.linalg.norm(H[:Nn, :Nn - 1]) * np.linalg.norm(X[:, :Nn], 2)
    assert np.linalg.norm(lhs - rhs) <= 10 * bound
    # upper Hessenberg / upper triangular structure
    assert np.all(np.tril(o.H[:q, :q - 1], -2) == 0)
    assert np.all(np.tril(B, -1) == 0)


# ------------------------------------------------------------------ Arnoldi with A known (Alg. 2)
def arnoldi(A, v, N):
    """Algorithm 2 (Rayleigh-Ritz with Arnoldi, CGS with one reorthogonalisation), A known."""
    n = A.shape[0]
    V = np.zeros((n, N))
    H = np.zeros((N, N - 1))
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(N - 1):
        w = A @ V[:, j]
        h = V[:, :j + 1].T @ w
        w = w - V[:, :j + 1] @ h
        s = V[:, :j + 1].T @ w
        h = h + s
        w = w - V[:, :j + 1] @ s
        H[:j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def test_equals_arnoldi_with_known_map():
    """FOA-based DMD is the Arnoldi method without access to A (Sec. 3.1, Eqs. avpsijp1beta,
    betacolumnupdate): with snapshots psi_{j+1} = A psi_j both give the same H up to
    O(eps kappa_2(X)) (Eq. foabaseddmdberr)."""
    rng = np.random.default_rng(3)
    n, N = 60, 14
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    X = np.empty((n, N))
    X[:, 0] = rng.standard_normal(n)
    for t in range(1, N):
        X[:, t] = A @ X[:, t - 1]
    o = run_oracle(X)
    Va, Ha = arnoldi(A, X[:, 0], N)
    s = np.linalg.svd(X[:, :N - 1], compute_uv=False)
    kappa = s[0] / s[-1]
    m = N - 1
    err = np.linalg.norm(o.H[:m + 1, :m] - Ha[:m + 1, :m])
    assert err <= 1e3 * U64 * kappa * np.linalg.norm(Ha)
    # projection error of Eq. (foabaseddmdberr): ||V^T A V - H||_F <= C eps kappa
    V = o.V[:, :m]
    perr = np.linalg.norm(V.T @ A @ V - o.H[:m, :m])
    assert perr <= 1e3 * U64 * kappa * max(1.0, np.linalg.norm(A, 2))


# ------------------------------------------------------------------ planted low-rank map (Sec. 3.2.4)
def test_planted_map_breakdown_and_exact_eigenvalues():
    """A rank-10 map with noise-free snapshots: psi_11 is a combination of psi_1..psi_10, so
    h_{11,10} = 0, FOA stops, and the Ritz values are the planted eigenvalues (Sec. 3.2.4)."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    o = run_oracle(X)
    assert o.stopped and o.q == 10 and o.m == 10
    res = o.eig()
    d, _ = match_eigs(res["lam"], spec.lam)
    s = np.linalg.svd(X[:, :10], compute_uv=False)
    kappa = s[0] / s[-1]
    assert d.max() <= 1e3 * U64 * kappa
    np.testing.assert_array_equal(res["indicator"], 0.0)  # h_{m+1,m} = 0 at a breakdown


def test_companion_matrix_ritz_values():
    """Exact-arithmetic equivalence with the Krylov companion form (Secs. 1-2, Eq. pdmdgalprob with
    Q = X_1^{N-1}): Ritz values = eigenvalues of the companion matrix whose last column is the
    least-squares fit of psi_N by psi_1..psi_{N-1}."""
    rng = np.random.default_rng(11)
    n, N = 200, 9
    X = rng.standard_normal((n, N))
    o = run_oracle(X)
    res = o.eig()
    c, *_ = np.linalg.lstsq(X[:, :N - 1], X[:, N - 1], rcond=None)
    Cm = np.zeros((N - 1, N - 1))
    Cm[1:, :-1] = np.eye(N - 2)
    Cm[:, -1] = c
    mu = np.linalg.eigvals(Cm)
    d, _ = match_eigs(res["lam"], mu)
    assert d.max() <= 1e-10 * max(1.0, np.abs(mu).max())


def test_truncated_agrees_with_svd_dmd():
    """Rank-truncated FOA-based DMD and rank-truncated SVD-based DMD (Schmid 2010) give nearly
    the same eigenvalues (Sec. 3.2.2, after Eq. foabaseddmdrtkberr): eig(U_r^T X_2 W_r S_r^-1)."""
    rng = np.random.default_rng(5)
    n, N, r = 120, 16, 6
    spec = synth.planted(n, N, r, 9, noise_rel=1e-9)
    X = synth.snapshots(spec)
    o = oracle.FoaOracle(n, N, breakdown_tol=1e-14)
    for t in range(N):
        assert o.push(X[:, t])[0] == "ok"
    tol = 1e-6
    res = o.eig(rank_tol=tol)
    U, S, Wt = np.linalg.svd(X[:, :N - 1], full_matrices=False)
    rr = int(np.sum(S > tol * S[0]))
    assert rr == res["r"] == r
    At = U[:, :rr].T @ X[:, 1:N] @ Wt[:rr].T @ np.diag(1.0 / S[:rr])
    mu = np.linalg.eigvals(At)
    d, _ = match_eigs(res["lam"], mu)
    assert d.max() <= 1e-6
    d2, _ = match_eigs(res["lam"], spec.lam)
    assert d2.max() <= 1e-6


# ------------------------------------------------------------------ error law (Sec. 3.2.2, Fig. 2)
def test_projection_error_grows_like_kappa():
    """Vandermonde A = vander(linspace(0,1,50)) applied to a random start vector; the error
    ||V^T A V - H||_2 of the computed projection grows like eps kappa_2(X) (Fig. 2,
    Eq. foabaseddmdberr): the log-log slope over the sweep is about 1."""
    A, Xall = synth.vandermonde_sequence(40, seed=0)
    ks, es = [], []
    for N in range(4, 14):
        X = Xall[:, :N]
        o = oracle.FoaOracle(50, N, breakdown_tol=1e-300)
        for t in range(N):
            if o.push(X[:, t])[0] != "ok":
                break
        m = o.m
        if m < 2:
            continue
        V = o.V[:, :m]
        P = V.T @ A @ V
        err = np.linalg.norm(P - o.H[:m, :m], 2)
        s = np.linalg.svd(X[:, :m], compute_uv=False)
        ks.append(s[0] / s[-1])
        es.append(err)
    ks, es = np.log10(ks), np.log10(es)
    sel = ks < 14.0
    slope = np.polyfit(ks[sel], es[sel], 1)[0]
    assert 0.8 <= slope <= 1.2, slope  # measured 0.92
    # and the error stays within a modest multiple of eps kappa
    assert np.all(es[sel] <= ks[sel] + np.log10(U64) + 4)


# ------------------------------------------------------------------ indicators (Sec. 3.2.3)
def test_indicator_matches_actual_residual():
    """|h_{N,N-1}| |e^T z| equals ||A V z - lambda V z|| for a known map when kappa << 1/eps
    (Eq. errordmdvec); with truncation the truncated indicator tracks the truncated residual."""
    rng = np.random.default_rng(2)
    n, N = 80, 20
    A = rng.standard_normal((n, n)) / np.sqrt(n) * 0.9
    X = np.empty((n, N))
    X[:, 0] = rng.standard_normal(n)
    for t in range(1, N):
        X[:, t] = A @ X[:, t - 1]
    o = run_oracle(X)
    res = o.eig()
    m = res["m"]
    V = o.V[:, :m]
    for i in range(m):
        phi = V @ res["Z"][:, i]
        act = np.linalg.norm(A @ phi - res["lam"][i] * phi)
        pred = res["indicator"][i]
        assert abs(act - pred) <= 1e-8 * max(1.0, act) + 10 * act * 1e-6, (act, pred)
    # truncated form
    tol = 1e-3
    rt = o.eig(rank_tol=tol)
    Ur = rt["Ur"]
    for i in range(rt["r"]):
        phi = V @ (Ur @ rt["Z"][:, i])
        act = np.linalg.norm(A @ phi - rt["lam"][i] * phi)
        assert abs(act - rt["indicator"][i]) <= 1e-8 * max(1.0, act)


# ------------------------------------------------------------------ reconstruction (Sec. 3.2.4)
def test_amplitudes_reconstruct_snapshots():
    """psi_k = sum_i c_i lambda_i^{k-1} phi_i for k = 1..N-1 with [z]{c} = |psi_1| e_1
    (Eqs. exrecon, reconerror)."""
    rng = np.random.default_rng(4)
    n, N = 150, 12
    X = rng.standard_normal((n, N))
    o = run_oracle(X)
    res = o.eig()
    m = res["m"]
    Phi = o.V[:, :m] @ res["Z"]
    s = np.linalg.svd(X[:, :m], compute_uv=False)
    kappa = s[0] / s[-1]
    # rounding enters through the projection (u kappa_2(X)), the eigenvector basis (cond(Z)) and
    # the powers lambda^(k-1); measured errors are 1e-15 ... 6e-15 against bounds near 2e-13, so a
    # percent-level error in one amplitude fails
    condz = np.linalg.cond(res["Z"])
    growth = max(1.0, np.abs(res["lam"]).max())
    for k in range(1, N):
        rec = (Phi * (res["amp"] * res["lam"] ** (k - 1))[None, :]).sum(axis=1)
        err = np.linalg.norm(rec - X[:, k - 1]) / np.linalg.norm(X[:, k - 1])
        assert err <= 100 * U64 * kappa * condz * growth ** (k - 1), (k, err)
    # a 1% error in the largest amplitude is caught
    amp = res["amp"].copy()
    amp[0] *= 1.01
    rec = (Phi * amp[None, :]).sum(axis=1)
    assert np.linalg.norm(rec - X[:, 0]) / np.linalg.norm(X[:, 0]) > 100 * U64 * kappa * condz


def test_modes_are_eigenvectors_of_the_known_map():
    """The planted rank-10 map (exact Krylov case, breakdown at push 11): every DMD mode
    Phi_i = V U_r z_i (Alg. 1) is a unit eigenvector of A with eigenvalue lambda_i, untruncated
    and truncated (Sec. 3.2.4: a zero h_{N,N-1} makes the Ritz pairs exact)."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    A = synth.planted_map(spec)
    o = run_oracle(X, 32)
    assert o.stopped and o.m == 10
    for rank_tol in (0.0, 1e-12):
        res = o.eig(rank_tol)
        Phi = o.modes(res, res["r"])
        assert Phi.shape == (spec.n, 10)
        for i in range(10):
            ph = Phi[:, i]
            assert abs(np.linalg.norm(ph) - 1.0) <= 1e-12
            r = np.linalg.norm(A @ ph - res["lam"][i] * ph)
            assert r <= 1e-9, (rank_tol, i, r)
        # modes follow the |c| order of the eigenvalues they belong to: a swapped column fails
        sw = Phi[:, [1, 0]]
        assert np.linalg.norm(A @ sw[:, 0] - res["lam"][0] * sw[:, 0]) > 1e-3


def test_ordering_rule():
    """Ordering by |c| (Secs. 4.1, 4.2), ties by |lambda| then Im(lambda); conjugate pairs adjacent."""
    spec = synth.config1(3)
    X = synth.snapshots(spec)
    o = run_oracle(X)
    res = o.eig()
    lam, amp = res["lam"], res["amp"]
    key = np.abs(amp)
    for i in range(0, len(lam) - 1, 2):
        assert abs(lam[i] - np.conj(lam[i + 1])) <= 1e-9
        assert lam[i].imag >= 0
    pair_keys = [max(key[i], key[i + 1]) for i in range(0, len(lam), 2)]
    assert all(pair_keys[i] >= pair_keys[i + 1] for i in range(len(pair_keys) - 1))


# ------------------------------------------------------------------ streaming = batch (Sec. 3.1)
def test_streaming_equals_batch_bitwise():
    """The streaming form carries out the same floating-point operations in the same order as the
    batch form (Sec. 3.1): pushing in pieces reproduces one pass bit for bit."""
    spec = synth.config2(1, G=32, N=30)
    X = synth.snapshots(spec)
    a = run_oracle(X)
    b = oracle.FoaOracle(X.shape[0], 30)
    b.push_batch(X[:, :7])
    b.push_batch(X[:, 7:19])
    for t in range(19, 30):
        b.push(X[:, t])
    assert a.q == b.q
    np.testing.assert_array_equal(a.V, b.V)
    np.testing.assert_array_equal(a.H, b.H)
    np.testing.assert_array_equal(a.B, b.B)


def test_status_rules():
    """Duplicate snapshot -> breakdown (Sec. 3.2.4); full basis; non-finite input leaves state."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 5))
    o = oracle.FoaOracle(300, 3)
    assert o.push(X[:, 0])[0] == "ok"
    assert o.push(X[:, 1])[0] == "ok"
    bad = X[:, 2].copy()
    bad[17] = np.nan
    H0 = o.H.copy()
    assert o.push(bad)[0] == "nonfinite"
    np.testing.assert_array_equal(o.H, H0)
    assert o.push(X[:, 2])[0] == "ok"
    assert o.push(X[:, 3])[0] == "full"
    o2 = oracle.FoaOracle(300, 5)
    o2.push(X[:, 0])
    o2.push(X[:, 1])
    assert o2.push(2.0 * X[:, 0] - 0.5 * X[:, 1])[0] == "breakdown"
    assert o2.m == 2
    assert o2.H[2, 1] == 0.0


def test_two_pass_reading_agrees():
    """The two-pass reading (h_{j+1,j} from ||w||^2 - ||s||^2, w after the first projection, s = V^T w)
    is the same step in exact arithmetic (V orthonormal): on ill- and well-conditioned sequences the
    states agree to rounding, and V stays orthonormal to O(eps)."""
    for X in (np.random.default_rng(1).standard_normal((400, 20)), synth.vandermonde_sequence(12, seed=2)[1]):
        a = oracle.run(X, breakdown_tol=1e-300)
        b = oracle.run(X, breakdown_tol=1e-300, reorth=2)
        assert a.q == b.q
        q = a.q
        s = np.linalg.svd(X[:, :q], compute_uv=False)
        kap = s[0] / s[-1]
        assert np.linalg.norm(a.B[:q, :q] - b.B[:q, :q]) <= 1e3 * U64 * kap * np.linalg.norm(a.B[:q, :q])
        assert np.linalg.norm(np.eye(q) - b.V[:, :q].T @ b.V[:, :q], 2) <= 10 * X.shape[1] * U64 * 10


def test_qr_view_is_the_householder_qr():
    """The QR view (Sec. 3.1: X = V beta with V orthonormal and beta upper triangular): beta equals
    LAPACK's R of X and V its Q, once the signs are fixed so that diag(R) > 0."""
    X = np.random.default_rng(5).standard_normal((500, 24))
    o = run_oracle(X, form="qr")
    assert o.q == 24
    Q, R = np.linalg.qr(X)
    sg = np.sign(np.diag(R))
    Q, R = Q * sg[None, :], R * sg[:, None]
    assert np.linalg.norm(o.B[:24, :24] - R) <= 50 * U64 * np.linalg.norm(R)
    assert np.linalg.norm(o.V[:, :24] - Q) <= 50 * U64 * 24
    assert np.all(np.tril(o.B[:24, :24], -1) == 0.0)


def test_qr_view_equals_foa_form():
    """Eq. matmulhbeta: the Hbar the QR view forms from beta is the Hbar of Alg. 1 (equal in exact
    arithmetic); beta of the QR view is beta of Alg. 1 (both are R of X).  Checked to rounding on a
    well-conditioned and an ill-conditioned (Vandermonde) sequence, with the O(eps kappa) law."""
    for X in (np.random.default_rng(6).standard_normal((300, 16)), synth.vandermonde_sequence(10, seed=4)[1]):
        a = run_oracle(X, tol=1e-300)
        b = run_oracle(X, tol=1e-300, form="qr")
        assert a.q == b.q
        q, m = a.q, a.m
        s = np.linalg.svd(X[:, :q], compute_uv=False)
        kap = s[0] / s[-1]
        assert np.linalg.norm(a.B[:q, :q] - b.B[:q, :q]) <= 1e3 * U64 * kap * np.linalg.norm(a.B[:q, :q])
        assert np.linalg.norm(a.H[:m + 1, :m] - b.H[:m + 1, :m]) <= 1e3 * U64 * kap * np.linalg.norm(a.H[:m + 1, :m])


def test_qr_view_planted_breakdown():
    """Planted rank-10 map: the QR view also stops at push 11 and gives the planted eigenvalues."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    o = run_oracle(X, k_max=32, form="qr")
    assert o.stopped and o.q == 10 and o.m == 10
    d, _ = match_eigs(o.eig(0.0)["lam"], spec.lam)
    assert d.max() <= 1e-9


def run_blocks(X, p, k_max=None, tol=None, library=None):
    """Block pushes of p columns at a time (the first column alone)."""
    n, N = X.shape
    o = oracle.FoaOracle(n, k_max or N, breakdown_tol=tol, library=library, form="qr")
    o.push(X[:, 0])
    for s in range(1, N, p):
        st = o.push_block(X[:, s:s + p])
        if any(x[0] != "ok" for x in st):
            break
    return o


def test_block_push_is_the_householder_qr():
    """Block push (block CGS2 + Cholesky QR twice, Sec. 3.1's QR view in blocks): beta is LAPACK's R
    of X and V its Q (signs fixed), beta_{:,2:} = Hbar beta (Eq. matmulhbeta) to rounding."""
    X = np.random.default_rng(8).standard_normal((400, 21))
    for p in (2, 4):
        o = run_blocks(X, p)
        assert o.q == 21
        Q, R = np.linalg.qr(X)
        sg = np.sign(np.diag(R))
        Q, R = Q * sg[None, :], R * sg[:, None]
        assert np.linalg.norm(o.B[:21, :21] - R) <= 100 * U64 * np.linalg.norm(R)
        assert np.linalg.norm(o.V[:, :21] - Q) <= 100 * U64 * 21
        m = o.m
        assert np.linalg.norm(o.B[:m + 1, 1:m + 1] - o.H[:m + 1, :m] @ o.B[:m, :m]) <= 100 * U64 * np.linalg.norm(o.B)


def test_block_push_equals_single_pushes():
    """In exact arithmetic the block push is p single pushes: the states agree to O(eps kappa) on a
    well-conditioned and an ill-conditioned (Vandermonde) sequence, and V stays orthonormal."""
    for X in (np.random.default_rng(9).standard_normal((300, 17)), synth.vandermonde_sequence(9, seed=6)[1]):
        a = run_oracle(X, tol=1e-300, form="qr")
        b = run_blocks(X, 4, tol=1e-300)
        assert a.q == b.q
        q, m = a.q, a.m
        s = np.linalg.svd(X[:, :q], compute_uv=False)
        kap = s[0] / s[-1]
        assert np.linalg.norm(a.B[:q, :q] - b.B[:q, :q]) <= 1e3 * U64 * kap * np.linalg.norm(a.B[:q, :q])
        assert np.linalg.norm(a.H[:m + 1, :m] - b.H[:m + 1, :m]) <= 1e3 * U64 * kap * np.linalg.norm(a.H[:m + 1, :m])
        assert np.linalg.norm(np.eye(q) - b.V[:, :q].T @ b.V[:, :q], 2) <= 1e3 * U64 * max(1.0, kap * U64 * 1e8)


def test_block_push_breakdown_inside_a_block():
    """Planted rank-10 map pushed in blocks of 4: snapshot 11 (second column of the third block)
    is dependent; the block commits its first column, stops, and the planted eigenvalues follow."""
    spec = synth.config1(0)
    X = synth.snapshots(spec)
    o = oracle.FoaOracle(spec.n, 32, form="qr")
    o.push(X[:, 0])
    sts = []
    for s in range(1, 32, 4):
        sts += o.push_block(X[:, s:s + 4])
        if o.stopped:
            break
    assert [x[0] for x in sts][:10] == ["ok"] * 9 + ["breakdown"]
    assert o.stopped and o.q == 10 and o.m == 10 and o.H[10, 9] == 0.0
    d, _ = match_eigs(o.eig(0.0)["lam"], spec.lam)
    assert d.max() <= 1e-9


# ------------------------------------------------------------------ planted mistakes
MUTANTS = {
    "drop_second_projection": ("gemv_n(n, j, V, ldv, s, y);\n    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - y[r];",
                               "gemv_n(n, j, V, ldv, s, y);\n    for (int64_t r = 0; r < n; ++r) w[r] = w[r];"),
    "norm_without_sqrt": ("    nu = sqrt(dot_blocked(n, w, w, part));", "    nu = dot_blocked(n, w, w, part);"),
    "second_dot_uses_x": ("gemv_t(n, j, V, ldv, w, s, part);", "gemv_t(n, j, V, ldv, x, s, part);"),
    "beta_update_sign": ("BT(i, j) = pre[i] + h[i] * bjj;", "BT(i, j) = pre[i] - h[i] * bjj;"),
    "beta_pre_transposed": ("acc += HB(i, l) * BT(l, jc);", "acc += HB(l, i) * BT(l, jc);"),
    "beta_pre_index": ("int32_t l0 = i == 0 ? 0 : i - 1;", "int32_t l0 = i;"),
    "no_divide_by_bjj": ("w[r] = (x[r] - y[r]) / bjj;", "w[r] = (x[r] - y[r]);"),
    "diag_missing_bjj": ("BT(j, j) = nu * bjj;", "BT(j, j) = nu;"),
    "qr_hbar_sign": ("HB(i, jc) = (h[i] - acc) / bjj;", "HB(i, jc) = (h[i] + acc) / bjj;"),
    "qr_subdiag_missing_bjj": ("HB(j, jc) = nu / bjj;", "HB(j, jc) = nu;"),
    "qr_beta_diag": ("    BT(j, j) = nu;\n", "    BT(j, j) = nu * bjj;\n"),
    "qr_hbar_index": ("acc += HB(i, l) * BT(l, jc);\n    HB(i, jc) = (h[i] - acc) / bjj;",
                      "acc += HB(i, l) * BT(jc, l);\n    HB(i, jc) = (h[i] - acc) / bjj;"),
    "drop_h_plus_s": ("    /* reorthogonalisation */\n    gemv_t(n, j, V, ldv, w, s, part);\n"
                      "    for (int32_t i = 0; i < j; ++i) h[i] = h[i] + s[i];",
                      "    /* reorthogonalisation */\n    gemv_t(n, j, V, ldv, w, s, part);\n"
                      "    for (int32_t i = 0; i < j; ++i) h[i] = h[i];"),
    "qr_drop_h_plus_s": ("w[r] = x[r] - y[r];\n  if (reorth) {\n    gemv_t(n, j, V, ldv, w, s, part);\n"
                         "    for (int32_t i = 0; i < j; ++i) h[i] = h[i] + s[i];",
                         "w[r] = x[r] - y[r];\n  if (reorth) {\n    gemv_t(n, j, V, ldv, w, s, part);\n"
                         "    for (int32_t i = 0; i < j; ++i) h[i] = h[i];"),
}


def _step_from_perturbed_basis(library, form, delta=1e-6, n=60, j=8):
    """One push from a basis whose orthogonality is off by delta.  The CGS2 steps give
    psi = V beta_{:,j+1} (the QR view of Sec. 3.1: X = V beta, with the pre-vector of Alg. 1 in the
    FOA form) as an algebraic identity whatever V's orthogonality, because the second projection's
    coefficients s are added to h; without that sum the residual is beta_jj V s, of order delta.
    Returns the relative residual of psi - V beta_{:,j+1}."""
    rng = np.random.default_rng(17)
    k = j + 2
    Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    V = np.zeros((n, k), order="F")
    V[:, :j] = Q + delta * rng.standard_normal((n, j))
    H = np.zeros((k, k), order="F")
    B = np.zeros((k, k), order="F")
    B[:j, :j] = np.triu(rng.standard_normal((j, j)))
    B[np.arange(j), np.arange(j)] = 1.0 + rng.random(j)
    H[:j, :j - 1] = np.triu(rng.standard_normal((j, j - 1)), -1)
    x = rng.standard_normal(n)
    out = np.zeros(2)
    step = library.foa_oracle_qr_step if form == "qr" else library.foa_oracle_step
    st = step(n, j, oracle._ptr(V), n, oracle._ptr(H), k, oracle._ptr(B), k, oracle._ptr(x), 1e-300, 1,
              oracle._ptr(out))
    assert st == 0
    res = x - V[:, :j + 1] @ B[:j + 1, j]
    return np.linalg.norm(res) / np.linalg.norm(x)


@pytest.mark.parametrize("form", ["foa", "qr"])
def test_cgs2_identity_from_a_perturbed_basis(form):
    """psi = V beta_{:,j+1} to rounding after a push from a basis with orthogonality defect 1e-6
    (the second projection's coefficients are summed into h); a residual of order 1e-6 would mean
    the sum h + s was dropped."""
    r = _step_from_perturbed_basis(oracle.lib(), form)
    print(form, "relative residual", r)
    assert r <= 1e3 * U64


def _pins_pass(library):
    """Run a compact set of pins against an oracle library, for both forms of the push; True when
    all of them hold."""
    return _form_pins_pass(library, "foa") and _form_pins_pass(library, "qr")


def _form_pins_pass(library, form):
    try:
        rng = np.random.default_rng(3)
        n, N = 60, 12
        A = rng.standard_normal((n, n)) / np.sqrt(n)
        X = np.empty((n, N))
        X[:, 0] = rng.standard_normal(n)
        for t in range(1, N):
            X[:, t] = A @ X[:, t - 1]
        o = run_oracle(X, library=library, form=form)
        if o.q != N:
            return False
        q = o.q
        V, B = o.V[:, :q], o.B[:q, :q]
        if np.linalg.norm(np.eye(q) - V.T @ V, 2) > 10 * N * U64:
            return False
        if np.linalg.norm(X - V @ B) > 10 * N * U64 * np.linalg.norm(X):
            return False
        Va, Ha = arnoldi(A, X[:, 0], N)
        s = np.linalg.svd(X[:, :N - 1], compute_uv=False)
        if np.linalg.norm(o.H[:N, :N - 1] - Ha) > 1e3 * U64 * s[0] / s[-1] * np.linalg.norm(Ha):
            return False
        # ill-conditioned sequence (Vandermonde map): the second Gram-Schmidt pass matters here
        A2, X2 = synth.vandermonde_sequence(10, seed=1)
        o2 = oracle.FoaOracle(50, 10, breakdown_tol=1e-300, library=library, form=form)
        for t in range(10):
            o2.push(X2[:, t])
        q2 = o2.q
        V2, B2 = o2.V[:, :q2], o2.B[:q2, :q2]
        if np.linalg.norm(np.eye(q2) - V2.T @ V2, 2) > 10 * 10 * U64:
            return False
        if np.linalg.norm(X2[:, :q2] - V2 @ B2) > 10 * 10 * U64 * np.linalg.norm(X2[:, :q2]):
            return False
        if _step_from_perturbed_basis(library, form) > 1e3 * U64:
            return False
        return True
    except Exception:
        return False


BLOCK_MUTANTS = {
    "block_no_second_projection": (
        "gemv_n(n, j, V, ldv, C2, Y);\n    for (int64_t r = 0; r < n; ++r) w[r] = w[r] - Y[r];",
        "gemv_n(n, j, V, ldv, C2, Y);\n    for (int64_t r = 0; r < n; ++r) w[r] = w[r];"),
    "block_skip_first_cholesky_solve": ("    right_solve_upper(n, m1, W, R1, p);", "    (void)R1;"),
    "block_hbar_subdiag_unscaled": ("      HB(jj, jc) = R[i + i * p] / bjj;", "      HB(jj, jc) = R[i + i * p];"),
}


def _block_pins_pass(library):
    """The block push's pins: orthogonality, X = V beta and the Arnoldi Hbar (A known) on a random map,
    orthogonality and X = V beta on the Vandermonde sequence."""
    try:
        rng = np.random.default_rng(3)
        n, N = 60, 13
        A = rng.standard_normal((n, n)) / np.sqrt(n)
        X = np.empty((n, N))
        X[:, 0] = rng.standard_normal(n)
        for t in range(1, N):
            X[:, t] = A @ X[:, t - 1]
        o = run_blocks(X, 4, library=library)
        if o.q != N:
            return False
        V, B = o.V[:, :N], o.B[:N, :N]
        if np.linalg.norm(np.eye(N) - V.T @ V, 2) > 10 * N * U64:
            return False
        if np.linalg.norm(X - V @ B) > 10 * N * U64 * np.linalg.norm(X):
            return False
        Va, Ha = arnoldi(A, X[:, 0], N)
        s = np.linalg.svd(X[:, :N - 1], compute_uv=False)
        if np.linalg.norm(o.H[:N, :N - 1] - Ha) > 1e3 * U64 * s[0] / s[-1] * np.linalg.norm(Ha):
            return False
        A2, X2 = synth.vandermonde_sequence(9, seed=1)
        o2 = run_blocks(X2, 4, tol=1e-300, library=library)
        q2 = o2.q
        V2, B2 = o2.V[:, :q2], o2.B[:q2, :q2]
        if np.linalg.norm(np.eye(q2) - V2.T @ V2, 2) > 1e-6:  # Cholesky QR: O(u kappa(W)^2), measured 1e-9
            return False
        if np.linalg.norm(X2[:, :q2] - V2 @ B2) > 10 * 9 * U64 * np.linalg.norm(X2[:, :q2]):
            return False
        return True
    except Exception:
        return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(BLOCK_MUTANTS))
def test_block_mutants_are_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "foa_oracle.c")).read()
    old, new = BLOCK_MUTANTS[name]
    assert src.count(old) == 1
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(so),
                    str(path), "-lm"], check=True)
    assert _block_pins_pass(oracle.lib()), "block pins must hold on the real oracle"
    assert not _block_pins_pass(oracle.load(str(so))), f"mutant {name} was not caught"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "foa_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(so),
                    str(path), "-lm"], check=True)
    assert _pins_pass(oracle.lib()), "pins must hold on the real oracle"
    assert not _pins_pass(oracle.load(str(so))), f"mutant {name} was not caught"
