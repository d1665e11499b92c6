"""The self-checking build (-DFOA_DMD_CHECKED: every bulk copy checks its shared-memory destination
and its 16-byte alignment, every streaming producer its tile index) on representative workloads:
no device check fails, and every result equals the normal build's bit for bit (the checks only
add tests before the copies).  Each build runs the same script in its own process
(FOA_DMD_CHECKED selects the library)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, ".")
from paper_1805_05821_gb300 import foa_dmd as F, synth
from paper_1805_05821_gb300.foa_dmd import FoaDMD

def digest(*arrs):
    h = hashlib.sha256()
    for a in arrs:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]

def snaps(n, N, seed, dt):
    X = np.random.default_rng(seed).standard_normal((N, n))
    t = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]
    return torch.from_numpy(X).to(t).cuda()

out = {"lib": F.lib()._name.rsplit("/", 1)[-1]}
# single pushes, three storage types, ragged n; FP32 through every basis size up to the register-held stage
for dt, n, N in (("f64", 4096, 24), ("f32", 9001, 120), ("bf16", 9001, 72)):
    g = FoaDMD(n, N, dt)
    Xd = snaps(n, N, 1, dt)
    for t in range(N):
        g.push(Xd[t], info=False)
    q, st, H, B = g.state()
    out["push_" + dt] = [q, digest(H, B, g.basis(0, q).float().cpu().numpy())]
    if dt == "f32":
        r = g.eig(-1.0, n_modes=8)  # truncated eig and the tensor-core mode product
        out["eig_f32"] = [r["r"], digest(r["lam"].real, r["lam"].imag, r["phi"].real, r["phi"].imag)]
    g.close()
# two-pass push and block push (FP32)
g = FoaDMD(5000, 40, "f32", reorth=2)
Xd = snaps(5000, 40, 2, "f32")
for t in range(40):
    g.push(Xd[t], info=False)
q, st, H, B = g.state()
out["two_pass"] = [q, digest(H, B)]
g.close()
n, N = 4097, 41
Xd = snaps(n, N, 3, "f32")
Xp = torch.zeros((N, 4104), dtype=torch.float32, device="cuda")
Xp[:, :n] = Xd
g = FoaDMD(n, N, "f32")
st, infos = g.push_block(Xp, block=4)
q, stopped, H, B = g.state()
out["block"] = [int(st), q, digest(H, B)]
g.close()
# batched streams of uneven n
ns, Ns = [3001, 20000, 777], [30, 18, 25]
stream = torch.cuda.Stream()
opts = F.foa_dmd_opts_default()
opts.cuda_stream = stream.cuda_stream
b = F.foa_dmd_batch_create(ns, Ns, "f32", opts)
Xs = [snaps(ns[s], Ns[s], 10 + s, "f32") for s in range(3)]
ptrs = torch.zeros(3, dtype=torch.int64, device="cuda")
hl = torch.zeros(3, dtype=torch.float64, device="cuda")
for r in range(max(Ns)):
    with torch.cuda.stream(stream):
        ptrs.copy_(torch.tensor([int(Xs[s][r].data_ptr()) if r < Ns[s] else 0 for s in range(3)],
                                dtype=torch.int64), non_blocking=False)
        assert F.foa_dmd_batch_push(b, ptrs, hl) == 0
    stream.synchronize()
out["batched"] = []
for s in range(3):
    q, status, H, B = F.foa_dmd_batch_get_state(b, s, Ns[s])
    out["batched"].append([q, digest(H, B)])
F.foa_dmd_batch_destroy(b)
torch.cuda.synchronize()
out["check"] = list(F.foa_dmd_check_status())
print(json.dumps(out))
'''


def run(checked):
    env = dict(os.environ)
    env["FOA_DMD_CHECKED"] = "1" if checked else "0"
    p = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_checked_build_matches_the_normal_build_and_reports_nothing():
    from paper_1805_05821_gb300 import build
    from paper_1805_05821_gb300.foa_dmd import EINVAL, OK
    build.build()
    build.build(checked=True)
    normal, checked = run(False), run(True)
    print(json.dumps({"normal": normal, "checked": checked}))
    assert normal["lib"] == "libfoa_dmd.so" and checked["lib"] == "libfoa_dmd_checked.so"
    assert normal["check"] == [EINVAL, 0]
    assert checked["check"] == [OK, 0], f"device checks failed: bits {checked['check'][1]}"
    for key in normal:
        if key not in ("lib", "check"):
            assert normal[key] == checked[key], key
