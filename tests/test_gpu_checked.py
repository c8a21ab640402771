"""The index-checked build (the library compiled with -DLBM_CHECKED, built by
``__graft_entry__.build_checked()``): a stand-in for a memory checker, which
is not run on these GPUs.  In that build every population index the step
kernels compute (pulls, stores, plate writes) is tested against its buffer,
and the TMA copies' x coordinates against the 16-byte rule, before the
access; a failure is counted and the access skipped, so nothing can fault.

The check: every kernel form on small odd lattices -- the shared-memory
hold form, the TMA forms with and without walls, the FP32 and 16-bit seam
forms, the two-pass kernel, BGK, moving plates, the wetting rule and a
batch of uneven boxes -- counts no index out of range over a few steps,
and the checked build's populations equal the normal build's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (nx, ny, nz, make_params keywords); one batch entry holds a list
CASES = {
    "hold_form_tiny": (5, 7, 3, {}),
    "hold_form_tiny_walls": (5, 7, 3, dict(wall=(1, 1, 1))),
    "seam_fp32": (64, 24, 9, {}),
    "seam_fp32_zwalls": (67, 23, 11, dict(wall=(0, 0, 1), gravity=(0.0, 0.0, -1e-5))),
    "tma_xy_walls": (67, 23, 11, dict(wall=(1, 1, 0))),
    "seam16_f16": (68, 23, 11, dict(storage="f16", ref_B=1.0)),
    "seam16_bf16_zwalls": (68, 30, 9, dict(storage="bf16", ref_B=1.0, wall=(0, 0, 1))),
    "tma_f16_odd": (67, 23, 11, dict(storage="f16", ref_B=1.0)),
    "two_pass": (13, 9, 5, dict(kernel="two_pass")),
    "bgk": (35, 17, 8, dict(collision="bgk", wall=(0, 0, 1))),
    "plates": (33, 20, 4, dict(wall=(0, 2, 0), wall_u=((0.02, 0.0, 0.0), (0.02, 0.0, 0.0)))),
    "wetting": (40, 12, 10, dict(wall=(1, 1, 1), wetting=True, contact_angle_deg=60.0)),
}
BATCH = [(32, 32, 32), (48, 40, 24), (20, 16, 12)]

SCRIPT = r"""
import ctypes, json, sys
import numpy as np
import torch
from paper_1904_03618_gb300 import lbm, workloads as wl

cases = json.loads(sys.argv[1])
batch = json.loads(sys.argv[2])
outdir = sys.argv[3]
dev = torch.device("cuda:0")
base = dict(rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.1,
            A_R=0.01, A_B=0.01, beta=0.7, force=(2e-5, 0.0, 0.0))
counts = {}

def checks(ctx):
    c, n = ctypes.c_int(), ctypes.c_uint()
    assert lbm._lib.lbm_test_index_checks(ctx, ctypes.byref(c), ctypes.byref(n)) == 0
    return c.value, n.value

for name, (nx, ny, nz, kw) in cases.items():
    kw = dict(base, **kw)
    ref_B = kw.pop("ref_B", None)
    if "wall_u" in kw:
        kw["wall_u"] = tuple(tuple(v) for v in kw["wall_u"])
    for k in ("force", "gravity"):
        if k in kw:
            kw[k] = tuple(kw[k])
    kw["wall"] = tuple(kw.get("wall", (0, 0, 0)))
    p = lbm.make_params(nx, ny, nz, **kw)
    if ref_B is not None:
        p.ref_R, p.ref_B = 0.0, ref_B
    lat = lbm.Lattice(p, device=dev)
    lat.init_fields(*wl.random_fields(nx, ny, nz, seed=len(name)))
    lat.step(3)
    np.save("%s/%s.npy" % (outdir, name), lat.get_f().cpu().numpy())
    counts[name] = checks(lat.ctx)
    lat.close()

ps = [lbm.make_params(nx, ny, nz, **base) for nx, ny, nz in batch]
b = lbm.Batch(ps, device=dev)
for k, (nx, ny, nz) in enumerate(batch):
    b.init_fields(k, *wl.droplet(nx, ny, nz, 0.3 * min(nx, ny, nz), 3.0, 1.0,
                                 velocity=(0.03, 0.0, 0.01)))
b.step(3)
for k in range(len(batch)):
    np.save("%s/batch%d.npy" % (outdir, k), b.get_f(k).cpu().numpy())
counts["batch"] = checks(b.ctx)
b.close()
print(json.dumps(counts))
"""


def _run(lib, outdir):
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, json.dumps(CASES), json.dumps(BATCH),
                        str(outdir)], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_counts_no_index_out_of_range(tmp_path):
    sys.path.insert(0, ROOT)
    import __graft_entry__ as g
    checked_lib = g.build_checked()
    normal_lib = os.path.join(ROOT, "paper_1904_03618_gb300", "_lib", "liblbm.so")
    (tmp_path / "c").mkdir()
    (tmp_path / "n").mkdir()
    got = _run(checked_lib, tmp_path / "c")
    ref = _run(normal_lib, tmp_path / "n")
    names = list(CASES) + ["batch%d" % k for k in range(len(BATCH))]
    for name in list(CASES) + ["batch"]:
        assert got[name] == [1, 0], (name, got[name])   # checked build, nothing out of range
        assert ref[name] == [0, 0], (name, ref[name])   # the normal build has no checks
    for name in names:
        a = np.load(tmp_path / "c" / ("%s.npy" % name))
        b = np.load(tmp_path / "n" / ("%s.npy" % name))
        assert np.all(np.isfinite(a)), name
        # the two builds schedule the same FP32 arithmetic; where the
        # compiler contracts an operation differently, a 16-bit store can
        # round the other way: one storage ulp (2^-10 FP16, 2^-7 BF16)
        storage = CASES.get(name, (0, 0, 0, {}))[3].get("storage", "f32")
        tol = {"f32": 1e-6, "f16": 2.0 ** -10, "bf16": 2.0 ** -7}[storage]
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1.0), name
