"""The bounds-checked build (librad_checked.so, RAD_LIB=checked): every
device allocation carries canary words on both sides, verified when it is
returned and before every call returns.  A child process runs every kind of
call through it (trees, both pivotings, products of 1 to 65 columns, solves
with refinement and preconditioning, the block LU, checkpoints, the
allocation-free product, the server, a batch) and every call must come back
RAD_OK with its results equal to the ordinary build's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
import cavities as cv
import paper_2305_06891_gb300 as r
S = 5.670374419e-8
out = {"checked": r.rad_debug_bounds_checks()}
c = cv.config1()
T = np.asfortranarray(c.T[:, :1] * np.array([1.0, 0.9, 1.1]))
h = r.rad_build_htree(c.verts, 32, 1.0)
r.rad_compress_aca(h, 1e-6, 64, "partial", "f32", "f32", accurate_dtype="f32")
r.rad_htree_autotune(h)
X = np.random.default_rng(0).uniform(size=(c.n, 65))
out["y"] = [float(np.abs(r.rad_hmatvec(h, X[:, :k].astype(np.float32))).sum()) for k in (1, 3, 6, 65)]
q, i = r.rad_solve_flux(h, c.eps, T, S, tol=1e-6)
out["q"] = float(np.abs(q).sum())
q, i = r.rad_solve_flux(h, c.eps, T, S, tol=1e-8, refine=True)
out["q_refined"] = float(np.abs(q).sum())
lu = r.rad_hlu_factor(h, c.eps, 1e-4)
out["lu_x"] = float(np.abs(r.rad_hlu_solve(lu, X[:, :2])).sum())
q, i = r.rad_solve_flux(h, c.eps, T, S, tol=1e-6, precond=lu)
out["q_pre_status"] = i["status"]
lu.free()
blob = r.rad_htree_save(h)
g = r.rad_htree_load(blob)
out["y_loaded"] = float(np.abs(r.rad_hmatvec(g, X[:, :3].astype(np.float32))).sum())
g.free()
h.free()
h = r.rad_build_htree(cv.unit_cube(4), 16, 1.0)
r.rad_compress_aca(h, 1e-8, 64, "full", "f64", "f64")
out["full"] = float(np.abs(r.rad_hmatvec(h, np.ones(h.n))).sum())
h.free()
cavs = [cv.config1(), cv.config1()]
hb = r.rad_build_htree_batch(np.concatenate([k.verts for k in cavs]), [k.n for k in cavs], 32, 1.0)
r.rad_compress_aca(hb, 1e-6, 64, "partial", "f32", "f32")
yb, ib = r.rad_solve_reflection(hb, np.concatenate([k.eps for k in cavs]), np.ones(2 * c.n), tol=1e-6)
out["batch"] = float(np.abs(yb).sum())
hb.free()
srv = r.Server(slots=2, hbm_budget_bytes=8 << 30, leaf_size=32, aca_tol=1e-6, factor_dtype="f32",
               near_dtype="f32", accurate_dtype=None, tol=1e-6, refine=False, aca_scratch_mib=256)
cid = srv.add_cavity(c.verts)
tk = [srv.submit(cid, c.eps, T[:, k:k + 1], S) for k in range(3)]
out["served"] = [float(np.abs(srv.wait(t)[0]).sum()) for t in tk]
srv.close()
print(json.dumps(out))
"""


def _run(checked: bool) -> dict:
    env = dict(os.environ)
    env.pop("RAD_LIB", None)
    if checked:
        env["RAD_LIB"] = "checked"
    p = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_every_call_keeps_its_canaries_and_results():
    ref = _run(False)
    got = _run(True)
    assert ref.pop("checked") == 0 and got.pop("checked") == 1
    for k in ref:
        np.testing.assert_array_equal(np.asarray(got[k]), np.asarray(ref[k]), err_msg=k)
