"""Python binding of the C ABI in include/foa_dmd.h and include/foa_synth.h.

Argument marshalling only: every function forwards to the function of the same name in
libfoa_dmd.so (built for sm_103a by ``paper_1805_05821_gb300.build``).  Device buffers are torch
tensors (their data pointers are passed); results come back as Python/numpy values.  There is no
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# FOA_DMD_CHECKED=1 loads the self-checking build (build.build(checked=True)) instead
_LIB_PATH = _build.CHECKED_LIB if os.environ.get("FOA_DMD_CHECKED") == "1" else _build.LIB

F64, F32, BF16 = 0, 1, 2
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EFULL", 5: "EBREAKDOWN", 6: "ESTOPPED",
          7: "ENONFINITE", 8: "ETIMEOUT", 9: "EIO", 10: "ENOCONV", 11: "ERESOLVE"}
OK, EINVAL, ENOMEM, ECUDA, EFULL, EBREAKDOWN, ESTOPPED, ENONFINITE, ETIMEOUT, EIO, ENOCONV, ERESOLVE = range(12)


class foa_dmd_opts(ctypes.Structure):
    _fields_ = [("reorth", ctypes.c_int32), ("breakdown_tol", ctypes.c_double),
                ("indicator_every", ctypes.c_int32), ("n_lead", ctypes.c_int32),
                ("indicator_rank_tol", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("form", ctypes.c_int32)]


class foa_dmd_push_info(ctypes.Structure):
    _fields_ = [("h_last", ctypes.c_double), ("indicator", ctypes.c_double), ("x_norm", ctypes.c_double),
                ("q", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {"h_last": self.h_last, "indicator": self.indicator, "x_norm": self.x_norm, "q": self.q,
                "status": STATUS.get(self.status, self.status)}


_DP = ctypes.POINTER(ctypes.c_double)


class foa_dmd_eig_result(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int32), ("n_modes", ctypes.c_int32), ("phi_dev", ctypes.c_void_p),
                ("ld_phi", ctypes.c_int64), ("vec_re", _DP), ("vec_im", _DP), ("vec_cols", ctypes.c_int32),
                ("m", ctypes.c_int32), ("r", ctypes.c_int32), ("lam_re", _DP), ("lam_im", _DP),
                ("indicator", _DP), ("amp_re", _DP), ("amp_im", _DP), ("sigma", _DP), ("h_last", ctypes.c_double)]


class foa_dmd_kernel_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("bytes", ctypes.c_double * 4), ("launches", ctypes.c_int64 * 4),
                ("total_launches", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libfoa_dmd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "foa_dmd_opts_default": (None, [ctypes.POINTER(foa_dmd_opts)]),
            "foa_dmd_create": (ctypes.c_int, [i64, i32, i32, ctypes.POINTER(foa_dmd_opts), ctypes.POINTER(vp)]),
            "foa_dmd_push": (ctypes.c_int, [vp, vp, ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_push_batch": (ctypes.c_int, [vp, vp, i32, i64, ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_push_host": (ctypes.c_int, [vp, vp, ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_sync": (ctypes.c_int, [vp, ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_indicators": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), _DP, i32,
                                                  ctypes.POINTER(i32)]),
            "foa_dmd_eig": (ctypes.c_int, [vp, d, ctypes.POINTER(foa_dmd_eig_result)]),
            "foa_dmd_test_wait_fault": (ctypes.c_int, [vp, i32, i64]),
            "foa_dmd_check_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
            "foa_dmd_get_state": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), _DP, _DP, i32]),
            "foa_dmd_get_basis": (ctypes.c_int, [vp, i32, i32, vp, i64]),
            "foa_dmd_reset": (ctypes.c_int, [vp]),
            "foa_dmd_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
            "foa_dmd_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(foa_dmd_opts), ctypes.POINTER(vp)]),
            "foa_dmd_destroy": (None, [vp]),
            "foa_dmd_push_noalloc": (ctypes.c_int, [i64, i32, i32, vp, _DP, _DP, i32, vp, vp, d, vp,
                                                    ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "foa_dmd_profile": (ctypes.c_int, [vp, ctypes.c_int]),
            "foa_dmd_profile_read": (ctypes.c_int, [vp, ctypes.POINTER(foa_dmd_kernel_stats)]),
            "foa_dmd_autotune": (ctypes.c_int, [vp, ctypes.c_char_p, i32]),
            "foa_dmd_push_block": (ctypes.c_int, [vp, vp, i32, i64, i32, ctypes.POINTER(foa_dmd_push_info)]),
            "foa_dmd_tuned_geometry": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                                      ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "foa_dmd_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(vp)]),
            "foa_dmd_host_free": (ctypes.c_int, [vp]),
            "foa_dmd_batch_create": (ctypes.c_int, [i32, ctypes.POINTER(i64), ctypes.POINTER(i32), i32,
                                                    ctypes.POINTER(foa_dmd_opts), ctypes.POINTER(vp)]),
            "foa_dmd_batch_push": (ctypes.c_int, [vp, vp, vp]),
            "foa_dmd_batch_get_state": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), _DP, _DP,
                                                       i32]),
            "foa_dmd_batch_get_basis": (ctypes.c_int, [vp, i32, i32, i32, vp, i64]),
            "foa_dmd_batch_destroy": (None, [vp]),
            "foa_synth_waves": (ctypes.c_int, [vp, i32, i64, i32, i32, i32, i32, vp, vp, d, ctypes.c_uint32, i64,
                                               vp]),
            "foa_synth_gauss": (ctypes.c_int, [vp, i32, i64, i32, ctypes.c_uint32, d, vp, d, ctypes.c_uint32, i64,
                                               vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class FoaError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({lib().foa_dmd_strerror(status).decode()})")


def _check(status, where):
    if status != OK:
        raise FoaError(status, where)
    return status


def _ptr(t):
    return ctypes.c_void_p(int(t.data_ptr())) if t is not None else ctypes.c_void_p(0)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ------------------------------------------------------------------ functions of the C ABI
def foa_dmd_opts_default():
    o = foa_dmd_opts()
    lib().foa_dmd_opts_default(ctypes.byref(o))
    return o


def foa_dmd_create(n, k_max, dtype, opts=None):
    h = ctypes.c_void_p()
    st = lib().foa_dmd_create(int(n), int(k_max), DTYPES.get(dtype, dtype), ctypes.byref(opts) if opts else None,
                              ctypes.byref(h))
    _check(st, "foa_dmd_create")
    return h


def foa_dmd_push(h, x, want_info=True):
    info = foa_dmd_push_info()
    st = lib().foa_dmd_push(h, _ptr(x), ctypes.byref(info) if want_info else None)
    return st, (info if want_info else None)


def foa_dmd_push_batch(h, X, p, ld, want_info=True):
    infos = (foa_dmd_push_info * max(p, 1))()
    st = lib().foa_dmd_push_batch(h, _ptr(X), int(p), int(ld), infos if want_info else None)
    return st, (list(infos)[:p] if want_info else None)


def foa_dmd_push_host(h, x_host_ptr, want_info=False):
    info = foa_dmd_push_info()
    st = lib().foa_dmd_push_host(h, ctypes.c_void_p(int(x_host_ptr)), ctypes.byref(info) if want_info else None)
    return st, (info if want_info else None)


def foa_dmd_sync(h):
    info = foa_dmd_push_info()
    st = lib().foa_dmd_sync(h, ctypes.byref(info))
    return st, info


def foa_dmd_indicators(h, cap=1024):
    pi = (ctypes.c_int32 * cap)()
    mm = (ctypes.c_int32 * cap)()
    val = np.zeros(cap)
    cnt = ctypes.c_int32()
    _check(lib().foa_dmd_indicators(h, pi, mm, val.ctypes.data_as(_DP), cap, ctypes.byref(cnt)), "foa_dmd_indicators")
    k = cnt.value
    return [(int(pi[i]), int(mm[i]), float(val[i])) for i in range(k)]


def foa_dmd_get_state(h, k_max):
    q, stopped = ctypes.c_int32(), ctypes.c_int32()
    H = np.zeros((k_max, k_max), order="F")
    B = np.zeros((k_max, k_max), order="F")
    st = lib().foa_dmd_get_state(h, ctypes.byref(q), ctypes.byref(stopped), H.ctypes.data_as(_DP),
                                 B.ctypes.data_as(_DP), k_max)
    _check(st, "foa_dmd_get_state")
    return q.value, bool(stopped.value), H, B


def foa_dmd_get_basis(h, col0, ncols, dst, ld):
    return _check(lib().foa_dmd_get_basis(h, int(col0), int(ncols), _ptr(dst), int(ld)), "foa_dmd_get_basis")


def foa_dmd_eig(h, rank_tol, cap, n_modes=0, phi=None, ld_phi=0, vec_cols=0, want_sigma=True):
    res = foa_dmd_eig_result()
    arrs = {k: np.zeros(cap) for k in ("lam_re", "lam_im", "indicator", "amp_re", "amp_im", "sigma")}
    res.cap = cap
    res.n_modes = n_modes
    res.phi_dev = int(phi.data_ptr()) if phi is not None else None
    res.ld_phi = int(ld_phi)
    res.vec_cols = int(vec_cols)
    vr = vi = None
    if vec_cols:
        vr = np.zeros(cap * vec_cols)
        vi = np.zeros(cap * vec_cols)
        res.vec_re = vr.ctypes.data_as(_DP)
        res.vec_im = vi.ctypes.data_as(_DP)
    for k in ("lam_re", "lam_im", "indicator", "amp_re", "amp_im"):
        setattr(res, k, arrs[k].ctypes.data_as(_DP))
    if want_sigma:
        res.sigma = arrs["sigma"].ctypes.data_as(_DP)
    st = lib().foa_dmd_eig(h, float(rank_tol), ctypes.byref(res))
    out = {"status": st, "m": res.m, "r": res.r, "h_last": res.h_last}
    if st == OK:
        r = res.r
        out["lam"] = arrs["lam_re"][:r] + 1j * arrs["lam_im"][:r]
        out["indicator"] = arrs["indicator"][:r].copy()
        out["amp"] = arrs["amp_re"][:r] + 1j * arrs["amp_im"][:r]
        out["sigma"] = arrs["sigma"][:r].copy() if want_sigma else None
        if vec_cols:
            vc = min(vec_cols, r)
            m = res.m
            out["vec"] = (vr[:m * vc].reshape(vc, m).T + 1j * vi[:m * vc].reshape(vc, m).T)
    return out


def foa_dmd_check_status():
    """(status, bits): the device checks that failed since the last call in a self-checking build
    (status EINVAL in a normal build)."""
    bits = ctypes.c_uint32(0)
    st = lib().foa_dmd_check_status(ctypes.byref(bits))
    return st, bits.value


def foa_dmd_test_wait_fault(h, skip_cta, spin_cycles):
    return lib().foa_dmd_test_wait_fault(h, int(skip_cta), int(spin_cycles))


def foa_dmd_push_noalloc(n, k_max, dtype, V, Hbar, beta, q, x, w, breakdown_tol=0.0, stream=None):
    """V, Hbar, beta, x, w: device tensors owned by the caller (see include/foa_dmd.h)."""
    info = foa_dmd_push_info()
    st = lib().foa_dmd_push_noalloc(int(n), int(k_max), DTYPES.get(dtype, dtype), _ptr(V),
                                    ctypes.cast(ctypes.c_void_p(int(Hbar.data_ptr())), _DP),
                                    ctypes.cast(ctypes.c_void_p(int(beta.data_ptr())), _DP), int(q), _ptr(x), _ptr(w),
                                    float(breakdown_tol), _stream_ptr(stream), ctypes.byref(info))
    return st, info


def foa_dmd_reset(h):
    return _check(lib().foa_dmd_reset(h), "foa_dmd_reset")


def foa_dmd_save(h, path):
    return lib().foa_dmd_save(h, str(path).encode())


def foa_dmd_load(path, opts=None):
    h = ctypes.c_void_p()
    st = lib().foa_dmd_load(str(path).encode(), ctypes.byref(opts) if opts else None, ctypes.byref(h))
    _check(st, "foa_dmd_load")
    return h


def foa_dmd_destroy(h):
    lib().foa_dmd_destroy(h)


def foa_dmd_strerror(status):
    return lib().foa_dmd_strerror(int(status)).decode()


def foa_dmd_profile(h, enable):
    return _check(lib().foa_dmd_profile(h, int(enable)), "foa_dmd_profile")


def foa_dmd_profile_read(h):
    s = foa_dmd_kernel_stats()
    _check(lib().foa_dmd_profile_read(h, ctypes.byref(s)), "foa_dmd_profile_read")
    return {"ms": list(s.ms), "bytes": list(s.bytes), "launches": list(s.launches),
            "total_launches": int(s.total_launches)}


def foa_dmd_push_block(h, X, p, ld, block=4, info=True):
    infos = (foa_dmd_push_info * max(p, 1))() if info else None
    st = lib().foa_dmd_push_block(h, _ptr(X), int(p), int(ld), int(block), infos)
    return st, (list(infos)[:p] if info else None)


def foa_dmd_autotune(h, cache_path=None, force=False):
    path = str(cache_path).encode() if cache_path else None
    return _check(lib().foa_dmd_autotune(h, path, 1 if force else 0), "foa_dmd_autotune")


def foa_dmd_tuned_geometry(h, kind, j):
    st, inf = ctypes.c_int64(), ctypes.c_int64()
    ctas, variant, tuned = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().foa_dmd_tuned_geometry(h, int(kind), int(j), ctypes.byref(st), ctypes.byref(inf), ctypes.byref(ctas),
                                        ctypes.byref(variant), ctypes.byref(tuned)), "foa_dmd_tuned_geometry")
    return {"stage_bytes": st.value, "inflight_bytes": inf.value, "ctas_per_sm": ctas.value,
            "variant": variant.value, "tuned": bool(tuned.value)}


def foa_dmd_host_alloc(nbytes):
    p = ctypes.c_void_p()
    _check(lib().foa_dmd_host_alloc(int(nbytes), ctypes.byref(p)), "foa_dmd_host_alloc")
    return p.value


def foa_dmd_host_free(ptr):
    return _check(lib().foa_dmd_host_free(ctypes.c_void_p(ptr)), "foa_dmd_host_free")


def foa_dmd_batch_create(ns, kmaxs, dtype, opts=None):
    S = len(ns)
    n_arr = (ctypes.c_int64 * S)(*[int(v) for v in ns])
    k_arr = (ctypes.c_int32 * S)(*[int(v) for v in kmaxs])
    b = ctypes.c_void_p()
    st = lib().foa_dmd_batch_create(S, n_arr, k_arr, DTYPES.get(dtype, dtype), ctypes.byref(opts) if opts else None,
                                    ctypes.byref(b))
    _check(st, "foa_dmd_batch_create")
    return b


def foa_dmd_batch_push(b, xptrs_dev, hlast_dev):
    return lib().foa_dmd_batch_push(b, _ptr(xptrs_dev), _ptr(hlast_dev))


def foa_dmd_batch_get_state(b, s, k_max):
    q, status = ctypes.c_int32(), ctypes.c_int32()
    H = np.zeros((k_max, k_max), order="F")
    B = np.zeros((k_max, k_max), order="F")
    st = lib().foa_dmd_batch_get_state(b, int(s), ctypes.byref(q), ctypes.byref(status), H.ctypes.data_as(_DP),
                                       B.ctypes.data_as(_DP), k_max)
    _check(st, "foa_dmd_batch_get_state")
    return q.value, status.value, H, B


def foa_dmd_batch_get_basis(b, s, col0, ncols, dst, ld):
    return _check(lib().foa_dmd_batch_get_basis(b, int(s), int(col0), int(ncols), _ptr(dst), int(ld)),
                  "foa_dmd_batch_get_basis")


def foa_dmd_batch_destroy(b):
    lib().foa_dmd_batch_destroy(b)


def foa_synth_waves(x, dtype, n, axes, G, n_fields, M, tables, coef, noise_scale, seed_noise, t, stream=None):
    return _check(lib().foa_synth_waves(_ptr(x), DTYPES.get(dtype, dtype), int(n), int(axes), int(G), int(n_fields),
                                        int(M), _ptr(tables), _ptr(coef), float(noise_scale), int(seed_noise),
                                        int(t), _stream_ptr(stream)), "foa_synth_waves")


def foa_synth_gauss(x, dtype, n, M, seed_modes, mode_scale, coef, noise_scale, seed_noise, t, stream=None):
    return _check(lib().foa_synth_gauss(_ptr(x), DTYPES.get(dtype, dtype), int(n), int(M), int(seed_modes),
                                        float(mode_scale), _ptr(coef), float(noise_scale), int(seed_noise), int(t),
                                        _stream_ptr(stream)), "foa_synth_gauss")


# ------------------------------------------------------------------ convenience wrapper
class FoaDMD:
    """One snapshot stream (a handle of the C ABI) with torch tensors as device buffers."""

    def __init__(self, n, k_max, dtype="f32", reorth=1, breakdown_tol=0.0, indicator_every=0, n_lead=32,
                 indicator_rank_tol=0.0, stream=None, form=0, _handle=None):
        self.n, self.k_max, self.dtype = int(n), int(k_max), dtype
        o = foa_dmd_opts_default()
        o.reorth = reorth
        o.form = form
        o.breakdown_tol = breakdown_tol
        o.indicator_every = indicator_every
        o.n_lead = n_lead
        o.indicator_rank_tol = indicator_rank_tol
        o.cuda_stream = _stream_ptr(stream)
        self.opts = o
        self.h = _handle if _handle is not None else foa_dmd_create(n, k_max, dtype, o)

    def push(self, x, info=True):
        st, inf = foa_dmd_push(self.h, x, info)
        return st, (inf.as_dict() if inf is not None else None)

    def push_batch(self, X, info=True):
        """X: torch tensor of shape (p, ld) (row t = snapshot t, contiguous, ld >= n)."""
        p, ld = X.shape
        st, infos = foa_dmd_push_batch(self.h, X, p, ld, info)
        return st, ([i.as_dict() for i in infos] if infos is not None else None)

    def push_block(self, X, block=4, info=True):
        """X: torch tensor of shape (p, ld) (row t = snapshot t, contiguous, ld >= n)."""
        p, ld = X.shape
        st, infos = foa_dmd_push_block(self.h, X, p, ld, block, info)
        return st, ([i.as_dict() for i in infos] if infos is not None else None)

    def sync(self):
        st, inf = foa_dmd_sync(self.h)
        return st, inf.as_dict()

    def indicators(self):
        return foa_dmd_indicators(self.h)

    def state(self):
        return foa_dmd_get_state(self.h, self.k_max)

    def basis(self, col0, ncols):
        import torch
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[self.dtype]
        out = torch.empty((ncols, self.n), dtype=tdt, device="cuda")
        if ncols:
            foa_dmd_get_basis(self.h, col0, ncols, out, self.n)
        return out

    def eig(self, rank_tol=0.0, n_modes=0, vec_cols=0):
        import torch
        phi = None
        ld = 0
        if n_modes:
            tdt = torch.float64 if self.dtype == "f64" else torch.float32
            ld = (self.n + 3) // 4 * 4
            phi = torch.zeros((2 * n_modes, ld), dtype=tdt, device="cuda")
        res = foa_dmd_eig(self.h, rank_tol, self.k_max, n_modes, phi, ld, vec_cols)
        if n_modes and res["status"] == OK:
            nm = min(n_modes, res["r"])
            P = phi[:2 * nm, :self.n].double().cpu().numpy()
            res["phi"] = (P[0::2] + 1j * P[1::2]).T
        return res

    def reset(self):
        foa_dmd_reset(self.h)

    def test_wait_fault(self, skip_cta, spin_cycles):
        return foa_dmd_test_wait_fault(self.h, skip_cta, spin_cycles)

    def save(self, path):
        return foa_dmd_save(self.h, path)

    @classmethod
    def load(cls, path, dtype, n, k_max, reorth=1, breakdown_tol=0.0, stream=None, form=0):
        o = cls.__new__(cls)
        o.n, o.k_max, o.dtype = n, k_max, dtype
        o.opts = foa_dmd_opts_default()
        o.opts.reorth = reorth
        o.opts.form = form
        o.opts.breakdown_tol = breakdown_tol
        o.opts.cuda_stream = _stream_ptr(stream)
        o.h = foa_dmd_load(path, o.opts)
        return o

    def autotune(self, cache_path=None, force=False):
        return foa_dmd_autotune(self.h, cache_path, force)

    def tuned_geometry(self, kind, j):
        return foa_dmd_tuned_geometry(self.h, kind, j)

    def profile(self, enable=True):
        foa_dmd_profile(self.h, enable)

    def profile_read(self):
        return foa_dmd_profile_read(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            foa_dmd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
