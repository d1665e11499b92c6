"""The C-ABI library loads and exports every function declared in include/*.h (no GPU calls)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1805_05821_gb300 import build, foa_dmd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return foa_dmd.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(foa_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("foa_dmd_create", "foa_dmd_push", "foa_dmd_push_batch", "foa_dmd_eig", "foa_dmd_destroy",
                 "foa_dmd_batch_create", "foa_dmd_batch_push", "foa_synth_waves"):
        assert want in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_and_defaults(L):
    assert foa_dmd.foa_dmd_strerror(0) == "ok"
    assert "breakdown" in foa_dmd.foa_dmd_strerror(foa_dmd.EBREAKDOWN)
    assert foa_dmd.foa_dmd_strerror(99) == "unknown status"
    o = foa_dmd.foa_dmd_opts_default()
    assert o.reorth == 1 and o.n_lead == 32 and o.indicator_every == 0


def test_argument_checks_without_gpu(L):
    h = ctypes.c_void_p()
    assert L.foa_dmd_create(0, 8, 1, None, ctypes.byref(h)) == foa_dmd.EINVAL
    assert L.foa_dmd_create(100, 1, 1, None, ctypes.byref(h)) == foa_dmd.EINVAL
    assert L.foa_dmd_create(100, 600, 1, None, ctypes.byref(h)) == foa_dmd.EINVAL
    assert L.foa_dmd_create(100, 400, 0, None, ctypes.byref(h)) == foa_dmd.EINVAL  # FP64 limit 384
    for bad in (-1, 3):
        o = foa_dmd.foa_dmd_opts_default()
        o.reorth = bad  # 0 (CGS), 1 (CGS2) and 2 (two-pass CGS2) only
        assert L.foa_dmd_create(100, 8, 1, ctypes.byref(o), ctypes.byref(h)) == foa_dmd.EINVAL
    assert L.foa_dmd_push(None, None, None) == foa_dmd.EINVAL
    assert L.foa_dmd_eig(None, 0.0, None) == foa_dmd.EINVAL


def test_no_cpu_fallback(L):
    """Without a GPU the library refuses to create a stream; it never computes on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.foa_dmd_create(100, 8, 1, None, ctypes.byref(h)) == foa_dmd.ECUDA


def test_checked_build_translation_units_compile(tmp_path):
    """The self-checking variant (-DFOA_DMD_CHECKED) still compiles: the unit holding the check
    registry and foa_dmd_check_status, and units of the single, block and batched passes (nvcc
    cross-compiles without a GPU; the GPU test builds and runs the whole variant)."""
    import subprocess
    csrc = os.path.join(ROOT, "paper_1805_05821_gb300", "csrc")
    flags = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", csrc,
             "--expt-relaxed-constexpr", "-DFOA_DMD_CHECKED"] + build.ARCH
    for unit in ("api.cu", "pass_f32.cu", "block_pass_f32.cu", "batch.cu"):
        p = subprocess.run([build.nvcc(), "-c", os.path.join(csrc, unit), "-o", str(tmp_path / (unit + ".o"))] + flags,
                           capture_output=True, text=True)
        assert p.returncode == 0, (unit, p.stderr[-2000:])
