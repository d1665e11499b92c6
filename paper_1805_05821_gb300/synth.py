"""Seeded synthetic snapshot generators shared by the FP64 oracle tests and the CUDA path.

This module holds only the inputs: it contains none of the FOA-DMD arithmetic. Every snapshot
sequence is a modal synthesis

    x_t[r] = sum_m F(r, m) * T_f(r)[m, t]  +  noise_scale * xi(t, r),        t = 0 .. N-1

where F is a spatial mode evaluated element by element, T holds time coefficients computed
once on the host in FP64, and xi is unit-variance noise.  Two spatial kinds exist:

* ``waves``: plane waves on a periodic grid of 1, 2 or 3 axes (optionally several fields
  stacked, e.g. the u, v, w, p velocity/pressure fields of a flow snapshot, Sec. 1 and
  Sec. 4.3).  The complex factor exp(i k.r) is the product of per-axis tables of
  (cos, sin) values, so the device can rebuild it without transcendental functions.
* ``gauss``: Gaussian mode vectors (a planted low-rank linear map x_{t+1} = A x_t, Sec. 2
  Eq. (2)), drawn with the Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  and an Irwin-Hall(4) sum of uniforms rescaled to unit variance.

``rows()`` evaluates chosen rows in float32 or float64 with one fixed operation order and
round-to-nearest on every operation (numpy never contracts to FMA); the CUDA generator in
``csrc/synth.cu`` applies the same operations in the same order with __fmul_rn/__fadd_rn,
so a device snapshot equals the host rows bit for bit.  Full matrices for small n come from
``snapshots()``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
KEY_MODES = 0x5EED
KEY_NOISE = 0x401E
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11), vectorised over the counter."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3)]
    k0 = np.uint64(k0) & _MASK32
    k1 = np.uint64(k1) & _MASK32
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [(hi1 ^ c[1] ^ k0) & _MASK32, lo1, (hi0 ^ c[3] ^ k1) & _MASK32, lo0]
    return [v.astype(np.uint32) for v in c]


def irwin_hall4(words, dtype, sqrt3):
    """Unit-variance sample from four 32-bit words: (u0+u1+u2+u3-2)*sqrt(3), u = (w>>8)*2^-24."""
    inv = dtype(2.0 ** -24)
    u = [dtype((w >> np.uint32(8)).astype(np.float64)) * inv for w in words]
    s = ((u[0] + u[1]) + u[2]) + u[3]
    return (s - dtype(2.0)) * sqrt3


@dataclasses.dataclass
class ModalSpec:
    """One synthetic snapshot sequence; see the module docstring for the formula."""
    name: str
    kind: str                    # "waves" or "gauss"
    n: int                       # snapshot length
    N: int                       # number of snapshots
    M: int                       # number of spatial modes (waves or Gaussian vectors)
    T: np.ndarray                # (n_fields, C, N) float64 time coefficients, C = 2M (waves) or M (gauss)
    grid: tuple = ()             # waves: (G,)*axes
    n_fields: int = 1
    tables: list = None          # waves: per axis an (M, G, 2) float64 array of (cos, sin)
    seed_modes: int = 0          # gauss: Philox key for the mode vectors
    mode_scale: float = 1.0      # gauss: factor on each mode entry (1/sqrt(n))
    seed_noise: int = 0
    noise_scale: float = 0.0
    lam: np.ndarray = None       # planted eigenvalues of the generating linear map
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_cols(self):
        return self.T.shape[1]


def _grid_index(spec, r):
    """Split flat row indices into (field, axis indices...) for the waves kind."""
    G = spec.grid[0]
    axes = len(spec.grid)
    idx = []
    rem = np.asarray(r, dtype=np.int64)
    for _ in range(axes):
        idx.append(rem % G)
        rem = rem // G
    idx.reverse()
    return rem, idx  # rem = field index


def _cmul(ar, ai, br, bi):
    return ar * br - ai * bi, ar * bi + ai * br


def rows(spec: ModalSpec, t: int, r, dtype=np.float64):
    """Rows r of snapshot t, computed in ``dtype`` arithmetic with the canonical order."""
    dtype = np.dtype(dtype).type
    r = np.asarray(r, dtype=np.int64)
    acc = np.zeros(r.shape, dtype=dtype)
    if spec.kind == "waves":
        field, idx = _grid_index(spec, r)
        tabs = [tab.astype(dtype) for tab in spec.tables]
        Tf = spec.T.astype(dtype)[:, :, t]          # (F, 2M)
        for m in range(spec.M):
            sr, si = tabs[0][m, idx[0], 0], tabs[0][m, idx[0], 1]
            for a in range(1, len(idx)):
                sr, si = _cmul(sr, si, tabs[a][m, idx[a], 0], tabs[a][m, idx[a], 1])
            acc = acc + sr * Tf[field, 2 * m]
            acc = acc + si * Tf[field, 2 * m + 1]
    elif spec.kind == "gauss":
        sqrt3 = dtype(math.sqrt(3.0))
        scale = dtype(spec.mode_scale)
        lo = (r & 0xFFFFFFFF).astype(np.uint64)
        hi = (r >> 32).astype(np.uint64)
        Tf = spec.T.astype(dtype)[0, :, t]
        for m in range(spec.M):
            words = philox4x32_10(lo, hi, np.uint64(m), np.uint64(0), spec.seed_modes, KEY_MODES)
            g = irwin_hall4(words, dtype, sqrt3) * scale
            acc = acc + g * Tf[m]
    else:
        raise ValueError(spec.kind)
    if spec.noise_scale > 0.0:
        acc = acc + dtype(spec.noise_scale) * noise(spec, t, r, dtype)
    return acc


def noise(spec, t, r, dtype=np.float64):
    dtype = np.dtype(dtype).type
    r = np.asarray(r, dtype=np.int64)
    lo = (r & 0xFFFFFFFF).astype(np.uint64)
    hi = (r >> 32).astype(np.uint64)
    words = philox4x32_10(lo, hi, np.uint64(t), np.uint64(1), spec.seed_noise, KEY_NOISE)
    return irwin_hall4(words, dtype, dtype(math.sqrt(3.0)))


def snapshots(spec: ModalSpec, dtype=np.float64, N=None, chunk=1 << 20):
    """The full n x N snapshot matrix (column t = snapshot t), for sizes the host holds.  For the
    waves kind the spatial factors of a row chunk are formed once and reused for every t; each
    element goes through the same operations in the same order as rows(), so the values are
    identical."""
    N = spec.N if N is None else N
    X = np.empty((spec.n, N), dtype=dtype, order="F")
    dt = np.dtype(dtype).type
    for r0 in range(0, spec.n, chunk):
        r = np.arange(r0, min(spec.n, r0 + chunk))
        if spec.kind != "waves":
            for t in range(N):
                X[r0:r0 + len(r), t] = rows(spec, t, r, dtype)
            continue
        field, idx = _grid_index(spec, r)
        tabs = [tab.astype(dt) for tab in spec.tables]
        SR, SI = [], []
        for m in range(spec.M):
            sr, si = tabs[0][m, idx[0], 0], tabs[0][m, idx[0], 1]
            for a in range(1, len(idx)):
                sr, si = _cmul(sr, si, tabs[a][m, idx[a], 0], tabs[a][m, idx[a], 1])
            SR.append(sr)
            SI.append(si)
        for t in range(N):
            Tf = spec.T.astype(dt)[:, :, t]
            acc = np.zeros(r.shape, dtype=dt)
            for m in range(spec.M):
                acc = acc + SR[m] * Tf[field, 2 * m]
                acc = acc + SI[m] * Tf[field, 2 * m + 1]
            if spec.noise_scale > 0.0:
                acc = acc + dt(spec.noise_scale) * noise(spec, t, r, dtype)
            X[r0:r0 + len(r), t] = acc
    return X


def mode_matrix(spec: ModalSpec, dtype=np.float64):
    """Gauss kind: the n x M matrix of mode vectors (FP64 values of the generated entries)."""
    assert spec.kind == "gauss"
    r = np.arange(spec.n, dtype=np.int64)
    lo = (r & 0xFFFFFFFF).astype(np.uint64)
    hi = (r >> 32).astype(np.uint64)
    dt = np.dtype(dtype).type
    P = np.empty((spec.n, spec.M), dtype=dtype)
    for m in range(spec.M):
        words = philox4x32_10(lo, hi, np.uint64(m), np.uint64(0), spec.seed_modes, KEY_MODES)
        P[:, m] = irwin_hall4(words, dt, dt(math.sqrt(3.0))) * dt(spec.mode_scale)
    return P


def planted_map(spec: ModalSpec):
    """Gauss kind: the linear map A = P M P^+ that advances x_t to x_{t+1} (without noise)."""
    P = mode_matrix(spec)
    Mb = spec.meta["block"]
    return P @ Mb @ np.linalg.pinv(P)


# ----------------------------------------------------------------------------------------
# Workloads.  Each follows the shapes of the paper's flow-field snapshots (Sec. 4) at the
# sizes of the five workload configurations; the paper's own datasets are not available.
# ----------------------------------------------------------------------------------------

def _axis_tables(rng_k, G):
    """(M, G, 2) (cos, sin) of 2*pi*k*i/G for integer wavenumbers k (one per wave)."""
    k = np.asarray(rng_k, dtype=np.int64)
    i = np.arange(G, dtype=np.int64)
    ph = (k[:, None] * i[None, :]) % G
    ang = 2.0 * np.pi * ph.astype(np.float64) / G
    return np.stack([np.cos(ang), np.sin(ang)], axis=-1)


def _distinct_wavevectors(rng, M, dims, kmax, kmin=1):
    seen = set()
    out = []
    while len(out) < M:
        k = tuple(int(v) for v in rng.integers(-kmax, kmax + 1, size=dims))
        nrm = math.sqrt(sum(v * v for v in k))
        if nrm < kmin or nrm > kmax:
            continue
        neg = tuple(-v for v in k)
        if k in seen or neg in seen:
            continue
        seen.add(k)
        out.append(k)
    return np.array(out, dtype=np.int64)


def planted(n, N, rank, seed, noise_rel=0.0, rho=(0.9, 1.0), name="planted"):
    """Planted low-rank linear map: rank//2 conjugate pairs (+1 real eigenvalue if rank odd).

    x_t = sum_p 2 rho_p^t (a_p cos(t th_p) - b_p sin(t th_p)) [+ lam_0^t c] (+ noise), with
    Gaussian mode entries ~ N(0, 1/n), rho ~ U[0.9, 1], th ~ U(0.05, pi-0.05) (kept off the
    real axis so no pair is nearly a double real eigenvalue); x_1 is the sum of the
    modes with unit amplitudes.  The map A = P blkdiag(rho R(th)) P^+ has these eigenvalues.
    """
    rng = np.random.default_rng([seed, 1])
    pairs, odd = rank // 2, rank % 2
    M = 2 * pairs + odd
    rh = rng.uniform(rho[0], rho[1], size=pairs + odd)
    th = rng.uniform(0.05, np.pi - 0.05, size=pairs)
    t = np.arange(N, dtype=np.float64)
    T = np.zeros((1, M, N))
    Mb = np.zeros((M, M))
    lam = []
    for p in range(pairs):
        T[0, 2 * p] = 2.0 * rh[p] ** t * np.cos(t * th[p])
        T[0, 2 * p + 1] = -2.0 * rh[p] ** t * np.sin(t * th[p])
        c, s = rh[p] * np.cos(th[p]), rh[p] * np.sin(th[p])
        Mb[2 * p:2 * p + 2, 2 * p:2 * p + 2] = [[c, s], [-s, c]]
        lam += [rh[p] * np.exp(1j * th[p]), rh[p] * np.exp(-1j * th[p])]
    if odd:
        T[0, M - 1] = rh[pairs] ** t
        Mb[M - 1, M - 1] = rh[pairs]
        lam.append(complex(rh[pairs]))
    rms = math.sqrt((4.0 * pairs + odd) / n)
    return ModalSpec(name=name, kind="gauss", n=n, N=N, M=M, T=T, seed_modes=(seed * 7919 + 17) & 0xFFFFFFFF,
                     mode_scale=1.0 / math.sqrt(n), seed_noise=(seed * 104729 + 3) & 0xFFFFFFFF,
                     noise_scale=noise_rel * rms, lam=np.array(lam), meta={"block": Mb, "rank": rank})


def config1(seed=0):
    """n=4096, N=32, FP64; rank-10 planted map (5 conjugate pairs), no noise."""
    return planted(4096, 32, 10, seed, 0.0, name="planted n=4096 N=32 rank=10")


def waves(G, axes, n_fields, N, M, seed, sigma=(-0.05, 0.0), omega=None, amp=None, kmax=64,
          noise_rel=0.0, field_coef=False, name="waves"):
    """Damped travelling waves sin/cos(k.r - w t + phi) e^{sigma t} on a periodic G^axes grid."""
    rng = np.random.default_rng([seed, 2])
    kvec = _distinct_wavevectors(rng, M, axes, kmax)
    if omega is None:
        omega = rng.uniform(0.05, np.pi - 0.05, size=M)
    sig = np.zeros(M) if sigma is None else rng.uniform(sigma[0], sigma[1], size=M)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=M)
    amp = np.ones(M) if amp is None else np.asarray(amp, dtype=np.float64)
    tables = [_axis_tables(kvec[:, a], G) for a in range(axes)]
    t = np.arange(N, dtype=np.float64)
    T = np.zeros((n_fields, 2 * M, N))
    ms = np.zeros(n_fields)
    if field_coef:
        cf = rng.standard_normal((M, n_fields)) + 1j * rng.standard_normal((M, n_fields))
        cf /= np.abs(cf).max(axis=1, keepdims=True)
    for m in range(M):
        env = amp[m] * np.exp(sig[m] * t)
        if field_coef:
            # Re(c_f exp(i(k.r - w t))) = Re S Re E - Im S Im E, E = amp e^{sig t} c_f e^{-i w t}
            for f in range(n_fields):
                E = env * cf[m, f] * np.exp(-1j * omega[m] * t)
                T[f, 2 * m] = E.real
                T[f, 2 * m + 1] = -E.imag
                ms[f] += amp[m] ** 2 * abs(cf[m, f]) ** 2 / 2.0
        else:
            # sin(k.r + phi - w t) = Re S sin(phi - w t) + Im S cos(phi - w t)
            for f in range(n_fields):
                T[f, 2 * m] = env * np.sin(phi[m] - omega[m] * t)
                T[f, 2 * m + 1] = env * np.cos(phi[m] - omega[m] * t)
                ms[f] += amp[m] ** 2 / 2.0
    lam = np.concatenate([np.exp(sig + 1j * omega), np.exp(sig - 1j * omega)])
    n = n_fields * G ** axes
    rms = math.sqrt(float(ms.mean()))
    return ModalSpec(name=name, kind="waves", n=n, N=N, M=M, T=T, grid=(G,) * axes, n_fields=n_fields,
                     tables=tables, seed_noise=(seed * 104729 + 5) & 0xFFFFFFFF, noise_scale=noise_rel * rms,
                     lam=lam, meta={"k": kvec, "omega": omega, "sigma": sig, "amp": amp})


def config2(seed=0, G=1024, N=200):
    """1024x1024 grid (n=2^20), N=200, 20 damped travelling waves, noise 1e-6 relative."""
    return waves(G, 2, 1, N, 20, seed, sigma=(-0.05, 0.0), noise_rel=1e-6,
                 name=f"waves2d n={G * G} N={N} M=20")


def config3(seed=0, kappa=1e4, G=256, N=500):
    """256^3 grid (n=2^24), N=500, 250 undamped waves with amplitudes kappa^{-(m-1)/249}."""
    M = N // 2
    omega = np.pi * (np.arange(1, M + 1) - 0.5) / M
    amp = kappa ** (-np.arange(M) / max(M - 1, 1))
    return waves(G, 3, 1, N, M, seed, sigma=None, omega=omega, amp=amp, kmax=min(64, G // 2 - 1),
                 name=f"waves3d n={G ** 3} N={N} kappa_t={kappa:g}")


def config4(seed=0, streams=256, n_range=(2 ** 14, 2 ** 22), N_range=(50, 400), r_range=(8, 32)):
    """Independent streams: n log-uniform, N uniform, planted rank-8..32 maps, noise 1e-5 relative."""
    rng = np.random.default_rng([seed, 4])
    out = []
    for s in range(streams):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        out.append(planted(n, N, r, seed * 100003 + s, noise_rel=1e-5, name=f"stream{s} n={n} N={N} r={r}"))
    return out


def config5(seed=0, G=256, N=384):
    """u, v, w, p fields on a 256^3 grid (n=4*256^3=67,108,864), N=384, 48 waves with
    amplitudes 1 -> 1e-3 and noise 1e-7 relative, so kappa_2(X) approaches 1/eps_fp32."""
    M = 48
    amp = 10.0 ** (-3.0 * np.arange(M) / (M - 1))
    return waves(G, 3, 4, N, M, seed, sigma=(-0.01, 0.0), amp=amp, kmax=min(64, G // 2 - 1),
                 noise_rel=1e-7, field_coef=True, name=f"fields4x{G}^3 n={4 * G ** 3} N={N} M=48")


def vandermonde_sequence(N, seed=0, size=50):
    """Snapshots psi_{i+1} = A psi_i with A = vander(linspace(0,1,50)) (Sec. 3.2.2, Fig. 2)."""
    A = np.vander(np.linspace(0.0, 1.0, size))
    rng = np.random.default_rng([seed, 5])
    X = np.empty((size, N))
    X[:, 0] = rng.standard_normal(size)
    for t in range(1, N):
        X[:, t] = A @ X[:, t - 1]
    return A, X
