"""FP64 CPU oracle of FOA-based projected DMD (Anantharamu & Mahesh, arXiv:1805.05821).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use this package; the product path (``paper_1805_05821_gb300``) never imports it, and it
imports nothing from the product except the shared seeded input generators.

* ``FoaOracle.push`` is the streaming update of Algorithm 4 (one snapshot, p = 1) carried out by
  the plain C code in ``foa_oracle.c`` (the basis and coefficient updates of Algorithm 1, unfused,
  fixed-order sums).
* ``FoaOracle.eig`` is the eigen extraction of Algorithms 1 and 3: the projected matrix
  H_m, the optional SVD of beta_m and rank truncation, the eigenpairs (LAPACK through scipy),
  the error indicators of Sec. 3.2.3 and the amplitudes of Sec. 3.2.4, Eqs. (exrecon)/(exreconwrt).
* ``FoaOracle.modes`` forms the DMD modes V U_r z_i (Algorithm 1).

Every function names the passage it follows; where the paper is silent or ambiguous, the docstring
states the reading taken.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np
import scipy.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfoa_oracle.so")

# unit roundoffs of the storage formats (FP64, FP32, BF16)
UNIT_ROUNDOFF = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}
# machine epsilons (distance from 1 to the next number)
EPS = {"f64": 2.0 ** -52, "f32": 2.0 ** -23, "bf16": 2.0 ** -7}

OK, BREAKDOWN, NOMEM = 0, 1, 2


def build(force=False):
    """Compile foa_oracle.c with gcc (plain C, -O2, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "foa_oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load(path):
    """Load a compiled oracle library (the default one, or a copy built elsewhere by a test)."""
    L = ctypes.CDLL(path)
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
    P = ctypes.POINTER(ctypes.c_double)
    L.foa_oracle_first.argtypes = [i64, P, P, P, P]
    L.foa_oracle_first.restype = ctypes.c_int
    L.foa_oracle_step.argtypes = [i64, i32, P, i64, P, i32, P, i32, P, d, ctypes.c_int, P]
    L.foa_oracle_step.restype = ctypes.c_int
    L.foa_oracle_qr_step.argtypes = [i64, i32, P, i64, P, i32, P, i32, P, d, ctypes.c_int, P]
    L.foa_oracle_qr_step.restype = ctypes.c_int
    L.foa_oracle_block_step.argtypes = [i64, i32, i32, P, i64, P, i32, P, i32, P, i64, d, P]
    L.foa_oracle_block_step.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_breakdown_tol(storage="f64"):
    """sqrt of the storage unit roundoff (the paper only says h_{j+1,j} = 0, Sec. 3.2.4)."""
    return float(np.sqrt(UNIT_ROUNDOFF[storage]))


def auto_rank_tol(storage, n_snapshots):
    """Relative rank threshold N*eps for "numerical rank" (Sec. 4.1), relative to sigma_1."""
    return n_snapshots * EPS[storage]


class FoaOracle:
    """Streaming FOA-based DMD state (H, V, beta, q) of Algorithm 3 in FP64 on the host."""

    def __init__(self, n, k_max, breakdown_tol=None, storage="f64", reorth=1, library=None, form="foa"):
        """form: "foa" = the modified FOA update of Alg. 1; "qr" = the QR view of the same push
        (psi orthogonalised directly, beta column = [h; nu], Hbar column from Eq. matmulhbeta)."""
        assert form in ("foa", "qr")
        self.form = form
        self._L = library
        self.n, self.k_max = int(n), int(k_max)
        self.storage = storage
        self.tol = default_breakdown_tol(storage) if breakdown_tol is None else float(breakdown_tol)
        self.reorth = int(reorth)
        self.V = np.zeros((self.n, self.k_max), order="F")
        self.H = np.zeros((self.k_max, self.k_max), order="F")
        self.B = np.zeros((self.k_max, self.k_max), order="F")
        self.q = 0
        self.stopped = False
        self.h_last = []

    # Algorithm 4 with p = 1
    def push(self, x):
        """Push one snapshot; returns (status, h_last, ||x||). Status strings: ok, breakdown,
        stopped (push after a breakdown), full (q == k_max), nonfinite (state unchanged)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.n,)
        if self.stopped:
            return "stopped", float("nan"), float("nan")
        if self.q == self.k_max:
            return "full", float("nan"), float("nan")
        if not np.all(np.isfinite(x)):
            return "nonfinite", float("nan"), float("nan")
        L = self._L or lib()
        if self.q == 0:
            nrm = ctypes.c_double(0.0)
            st = L.foa_oracle_first(self.n, _ptr(self.V), _ptr(self.B), _ptr(x), ctypes.byref(nrm))
            if st == NOMEM:
                raise MemoryError
            if st == BREAKDOWN:
                self.stopped = True
                return "breakdown", 0.0, nrm.value
            self.q = 1
            self.h_last.append(nrm.value)
            return "ok", nrm.value, nrm.value
        out = np.zeros(2)
        step = L.foa_oracle_qr_step if self.form == "qr" else L.foa_oracle_step
        st = step(self.n, self.q, _ptr(self.V), self.n, _ptr(self.H), self.k_max,
                  _ptr(self.B), self.k_max, _ptr(x), self.tol, self.reorth, _ptr(out))
        if st == NOMEM:
            raise MemoryError
        if st == BREAKDOWN:
            self.stopped = True
            return "breakdown", float(out[0]), float(out[1])
        self.q += 1
        self.h_last.append(float(out[0]))
        return "ok", float(out[0]), float(out[1])

    def push_block(self, X):
        """Block push of the columns of X (n x p) at once: block CGS2 against V and Cholesky QR twice
        (the block form of the QR view); returns one status tuple per snapshot as push() does.  A
        stream with no basis yet starts with a single push of the first column."""
        X = np.asfortranarray(X, dtype=np.float64)
        n, p = X.shape
        assert n == self.n
        res = []
        t = 0
        if self.q == 0 and p > 0:
            res.append(self.push(X[:, 0]))
            t = 1
            if res[-1][0] != "ok":
                return res + [("stopped", float("nan"), float("nan"))] * (p - 1)
        if self.stopped:
            return res + [("stopped", float("nan"), float("nan"))] * (p - t)
        pb = min(p - t, self.k_max - self.q)
        if pb > 0:
            Xb = np.asfortranarray(X[:, t:t + pb])
            if not np.all(np.isfinite(Xb)):
                return res + [("nonfinite", float("nan"), float("nan"))] * (p - t)
            out = np.zeros(1 + pb)
            L = self._L or lib()
            st = L.foa_oracle_block_step(self.n, self.q, pb, _ptr(self.V), self.n, _ptr(self.H), self.k_max,
                                         _ptr(self.B), self.k_max, _ptr(Xb), self.n, self.tol, _ptr(out))
            if st == NOMEM:
                raise MemoryError
            nc = int(out[0])
            for i in range(nc):
                res.append(("ok", float(out[1 + i]), float(np.linalg.norm(Xb[:, i]))))
                self.h_last.append(float(out[1 + i]))
            self.q += nc
            if st == BREAKDOWN:
                self.stopped = True
                res.append(("breakdown", 0.0, float(np.linalg.norm(Xb[:, nc]))))
                res += [("stopped", float("nan"), float("nan"))] * (p - t - nc - 1)
                return res
            t += pb
        res += [("full", float("nan"), float("nan"))] * (p - t)
        return res

    def push_batch(self, X):
        """Algorithm 4 with p = X.shape[1]: the same per-snapshot steps in sequence."""
        res = []
        for t in range(X.shape[1]):
            res.append(self.push(X[:, t]))
            if res[-1][0] != "ok":
                break
        return res

    # the eigen extraction of Algorithms 1 and 3
    @property
    def m(self):
        """Size of the projected matrix: q-1 normally, q after a breakdown (Sec. 3.2.4)."""
        return self.q if self.stopped else self.q - 1

    def projected(self):
        m = self.m
        return self.H[:m, :m].copy(), (self.H[m, m - 1] if m < self.k_max else 0.0)

    def eig(self, rank_tol=0.0):
        """Eigenpairs of H_m (rank_tol <= 0) or of U_r^T H_m U_r (rank_tol > 0; rank_tol < 0 and
        != 0 is not used here: pass auto_rank_tol() explicitly).

        r = #{sigma_i(beta_m) > rank_tol * sigma_1} (Sec. 3.2.2 rank truncation, Sec. 4.1 rule).
        Eigenvectors have unit 2-norm, largest-magnitude entry real and positive.
        Indicators (Sec. 3.2.3, Eq. errordmdvec and its truncated form):
          untruncated: |h_{m+1,m}| |e_m^T z_i|
          truncated:   ||[(I - U_r U_r^T) H_m U_r z_i ; h_{m+1,m} e_m^T U_r z_i]||_2
        Amplitudes (Sec. 3.2.4, Eqs. exrecon/exreconwrt): [z] c = beta_11 U_r^T e_1.
        Order: |c| descending (Sec. 4.1, 4.2), then |lambda| descending, then Im(lambda)
        descending; the two members of a conjugate pair share the larger |c|.
        """
        m = self.m
        if m < 1:
            raise ValueError("need at least two snapshots (or a breakdown) for a projected matrix")
        H, hlast = self.projected()
        Bm = self.B[:m, :m]
        if rank_tol > 0.0:
            U, S, _ = np.linalg.svd(Bm)
            r = int(np.sum(S > rank_tol * S[0]))
            r = max(r, 1)
            Ur = U[:, :r]
            G = Ur.T @ H @ Ur
        else:
            S = None
            r = m
            Ur = np.eye(m)
            G = H
        lam, Z = scipy.linalg.eig(G)
        Z = normalize_eigvecs(Z)
        Y = Ur @ Z                                   # U_r z_i in the Krylov coordinates
        if rank_tol > 0.0:
            top = H @ Y
            top = top - Ur @ (Ur.T @ top)
            ind = np.sqrt(np.sum(np.abs(top) ** 2, axis=0) + np.abs(hlast * Y[m - 1, :]) ** 2)
        else:
            ind = np.abs(hlast) * np.abs(Z[m - 1, :])
        b = self.B[0, 0] * Ur[0, :]
        c = np.linalg.solve(Z, b.astype(np.complex128))
        order = mode_order(lam, c)
        return {"m": m, "r": r, "lam": lam[order], "Z": Z[:, order], "Y": Y[:, order],
                "indicator": ind[order], "amp": c[order], "Ur": Ur, "G": G, "sigma": S,
                "h_last": hlast}

    def modes(self, res, n_modes):
        """DMD modes V_{1:m} U_r z_i for the first n_modes in the returned order (Alg. 1)."""
        m = res["m"]
        return self.V[:, :m] @ res["Y"][:, :n_modes]


def normalize_eigvecs(Z):
    """Unit 2-norm columns; the entry of largest magnitude is made real and positive."""
    Z = np.array(Z, dtype=np.complex128)
    Z /= np.linalg.norm(Z, axis=0, keepdims=True)
    idx = np.argmax(np.abs(Z), axis=0)
    ph = Z[idx, np.arange(Z.shape[1])]
    Z *= (np.abs(ph) / ph)[None, :]
    return Z


def mode_order(lam, c):
    """Indices sorting by |c| desc, |lambda| desc, Im(lambda) desc; conjugate pairs share |c|."""
    key = np.abs(c).copy()
    k = len(lam)
    used = np.zeros(k, dtype=bool)
    for i in range(k):
        if used[i] or lam[i].imag == 0.0:
            continue
        d = np.abs(lam - np.conj(lam[i]))
        d[i] = np.inf
        d[used] = np.inf
        d[lam.imag == 0.0] = np.inf
        jx = int(np.argmin(d))
        if np.isfinite(d[jx]):
            mx = max(key[i], key[jx])
            key[i] = key[jx] = mx
            used[i] = used[jx] = True
    return np.lexsort((-lam.imag, -np.abs(lam), -key))


def run(X, k_max=None, breakdown_tol=None, storage="f64", reorth=1, library=None, form="foa"):
    """Algorithm 1 (batch form) as a loop of streaming updates; returns the oracle state."""
    n, N = X.shape
    o = FoaOracle(n, k_max or N, breakdown_tol, storage, reorth, library, form)
    for t in range(N):
        st, _, _ = o.push(X[:, t])
        if st != "ok":
            break
    return o
