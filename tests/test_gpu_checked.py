"""The bounds-checked build (FR_CHECKED, the memory-checker substitute: compute-sanitizer is not
available to these tests): the library compiled with device-side checks of every mesh-derived
gather / scatter index gives the same results as the normal build, bit for bit, and records no
failure on clean runs of the uniform and the general path; a corrupted face-point trace map
planted through the checked build's import is caught (site, index, count) without a fault, and
the normal build refuses that import.  Each library runs in a child process of its own."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import paper_2401_16632_gb300 as pkg
lib_path = sys.argv[1]
pkg.load_library(lib_path)
from workloads import make_config
from workloads.mesh import BC_FARFIELD, BC_WALL, geometric_nodes, structured_quads, uniform_nodes
out = {}

def status():
    try:
        return list(pkg.fr_checked_status())
    except pkg.HfrError as e:
        return ["unsupported", e.code]

# uniform path: a 6x6 p=3 vortex with an implicit band, one IMEX stage (residual, blocks,
# condensation, GMRES, back-substitution)
band = np.zeros((6, 6), bool)
band[2:4, :] = True
w = make_config("vortex", n=6, p=3, re=300.0, implicit=band.reshape(-1))
ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
u_n = torch.tensor(w.u0, device="cuda")
uh = ctx.hfr_initial_trace(u_n)
R_hist = ctx.empty(3, *ctx.state_shape)
us = ctx.empty(*ctx.state_shape)
ctx.imex_stage(0, 0.05, u_n, us, uh, R_hist)
st = ctx.imex_stage(1, 0.05, u_n, us, uh, R_hist, newton_tol=1e-10, gmres_rtol=1e-8, gmres_maxit=2000)
out["uniform"] = {"u": us.cpu().numpy().ravel().tolist(), "newton": st["newton_iterations"]}
out["uniform_status"] = status()
ctx.close()

# general path: a stretched wall band with mixed degree, wall and far field, FP32 stage
yn = geometric_nodes(0.02, 1.6, 0.25, 1.0)
ny = len(yn) - 1
imp = np.zeros((ny, 3), bool)
imp[:3] = True
p = np.random.default_rng(2).choice([2, 3, 4], size=3 * ny).astype(np.int32)
mesh = structured_quads(uniform_nodes(3, 0.0, 1.0), yn, periodic=(True, False), p=p, implicit=imp.reshape(-1),
                        bc_y=(BC_WALL, BC_FARFIELD))
U_INF = np.array([1.0, 0.3, 0.05, 2.6])
rng = np.random.default_rng(3)
U = [U_INF * (1 + 1e-2 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 4))) for e in range(mesh.nelem)]
phys = {"kind": "ns", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0, "u_inf": U_INF}
ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2)
u_n = torch.tensor(ctx.pack_state(U), device="cuda")
uh = ctx.hfr_initial_trace(u_n)
R_hist = ctx.empty(3, *ctx.state_shape)
us = ctx.empty(*ctx.state_shape)
ctx.imex_stage(0, 0.004, u_n, us, uh, R_hist)
st = ctx.imex_stage(1, 0.004, u_n, us, uh, R_hist, newton_tol=1e-10, gmres_rtol=1e-8, gmres_maxit=2000)
out["general"] = {"u": us.cpu().numpy().ravel().tolist(), "newton": st["newton_iterations"]}
out["general_status"] = status()
# a corrupted face-point trace map (array 64): one traced face point sent far out of range
fn = ctx.hfr_export("fnode")
bad = int(torch.nonzero(fn >= 0)[5])
fn[bad] = 1 << 30
try:
    ctx.hfr_import("fnode", fn)
    R, g = ctx.fr_residual(u_n, uh)
    torch.cuda.synchronize()
    out["corrupt"] = {"imported": True, "status": status(), "finite_call": True}
except pkg.HfrError as e:
    out["corrupt"] = {"imported": False, "code": e.code}
ctx.close()
print("RESULT " + json.dumps(out))
'''


def _run(lib):
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code, lib], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def runs():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2401_16632_gb300.build import build

    plain = build()
    checked = build(checked=True)
    return _run(plain), _run(checked)


def test_checked_build_matches_the_normal_build_and_records_nothing(runs):
    plain, checked = runs
    assert plain["uniform_status"][0] == "unsupported" and plain["general_status"][0] == "unsupported"
    assert checked["uniform_status"] == [0, 0, 0]
    assert checked["general_status"] == [0, 0, 0]
    for part in ("uniform", "general"):
        assert plain[part]["newton"] == checked[part]["newton"]
        assert np.array_equal(np.array(plain[part]["u"]), np.array(checked[part]["u"]))


def test_corrupted_trace_map_is_caught_without_a_fault(runs):
    plain, checked = runs
    import paper_2401_16632_gb300 as pkg

    # the normal build refuses to write the map; the checked build takes it and its checks report
    # the first bad index at the residual's trace read (site 1) with the planted value
    assert plain["corrupt"] == {"imported": False, "code": pkg.FR_ERR_INVALID_ARG}
    assert checked["corrupt"]["imported"]
    site, index, count = checked["corrupt"]["status"]
    assert site == 1 and index == 1 << 30 and count >= 1
