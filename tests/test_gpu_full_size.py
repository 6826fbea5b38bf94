"""Full-size parity of the bench workloads (vortex64: 64x64 quads, p = 3; vortex256: 256x256
quads, p = 4, 6,553,600 implicit DOF) in the launch configuration the bench times.

* the FP64 residual R and trace residual g of the whole mesh against the oracle's;
* element blocks A, B, C, D, right-hand sides r, s and the condensed S, A^{-1}B, A^{-1}r, t_k of
  sampled elements: a hybridized element's blocks depend only on its own state and its own
  faces' traces (every face of these meshes is a trace face), so the oracle evaluates each
  sampled element on a 3x3 periodic patch with the same element nodes, the element's state and
  the full mesh's traces on its faces;
* the stage: the GPU's converged stage-1 solution evaluated by the oracle's residual meets the
  relative Newton tolerance 1e-8, on the mixed-precision and the FP64 path, and the two
  solutions agree to what that tolerance fixes.
"""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2401_16632_gb300.build import build

    build()
    torch.cuda.set_device(0)


import paper_2401_16632_gb300 as pkg  # noqa: E402
from oracle.blocks import element_blocks  # noqa: E402
from oracle.fr import Discretisation  # noqa: E402
from oracle.physics import make_physics  # noqa: E402
from oracle.solve import condense  # noqa: E402
from oracle.stepping import TABLEAUX  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import structured_quads  # noqa: E402

DEV = "cuda"
NEWTON_TOL = 1e-8
GMRES_RTOL = 1e-4  # the bench's inner tolerance


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


_CACHE = {}


def _workload(name):
    if name not in _CACHE:
        w = make_config(name)
        _CACHE[name] = (w, Discretisation(w.mesh, make_physics(w.physics)))
    return _CACHE[name]


def _perturbed_trace(d, u0, seed=0):
    uh = d.initial_trace(u0)
    rng = np.random.default_rng(seed)
    return uh * (1.0 + 1e-3 * rng.standard_normal(uh.shape))


@pytest.mark.parametrize("name", ["vortex64", "vortex256"])
def test_full_size_residual(name):
    w, d = _workload(name)
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    uh = _perturbed_trace(d, w.u0)
    R, g = ctx.fr_residual(torch.tensor(w.u0, device=DEV), torch.tensor(uh, device=DEV))
    Ro, go = d.full_residual(w.u0, uh)
    assert _rel(R.cpu().numpy(), Ro) < 1e-11
    assert _rel(g.cpu().numpy(), go) < 1e-11


def _patch(w, e):
    """3x3 periodic patch around element e of the full structured mesh: the centre element
    (patch index 4) has e's nodes; returns the patch mesh and the patch's element ids in the
    full mesh."""
    n = w.mesh.nx
    i, j = e % n, e // n
    v = w.mesh.verts[e]
    x0, y0 = v[0]
    hx, hy = v[1, 0] - v[0, 0], v[2, 1] - v[0, 1]
    xn = x0 + hx * np.array([-1.0, 0.0, 1.0, 2.0])
    yn = y0 + hy * np.array([-1.0, 0.0, 1.0, 2.0])
    xn[1], xn[2] = v[0, 0], v[1, 0]
    yn[1], yn[2] = v[0, 1], v[2, 1]
    mesh = structured_quads(xn, yn, periodic=(True, True), p=w.p)
    ids = np.array([((i + di) % n) + n * ((j + dj) % n) for dj in (-1, 0, 1) for di in (-1, 0, 1)])
    assert np.array_equal(mesh.verts[4], v)
    return mesh, ids


SAMPLES = [0, 255, 256 * 128 + 77, 256 * 255 + 255]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_sampled_blocks_and_condensation(precision):
    w, d = _workload("vortex256")
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
    a_dt = TABLEAUX["sdirk2"]["a"][0, 0] * w.dt
    uh = _perturbed_trace(d, w.u0, 1)
    ustar = w.u0 * 0.999
    ctx.hfr_local_jacobian(torch.tensor(w.u0, device=DEV), torch.tensor(uh, device=DEV),
                           torch.tensor(ustar, device=DEV), a_dt)
    assert np.array_equal(d.imp_idx, np.arange(w.mesh.nelem))  # compact index = element id
    sel = torch.tensor(SAMPLES, device=DEV)
    got = {k: ctx.hfr_export(k)[sel].cpu().numpy().astype(np.float64) for k in ("A", "B", "C", "D", "r", "s")}
    ctx.hfr_condense(refine=0)
    cond = {k: ctx.hfr_export(k)[sel].cpu().numpy().astype(np.float64) for k in ("S", "XB", "xr", "t_k")}
    full_view = d.trace_view(uh)
    tol_blk, tol_cond = (1e-11, 1e-11) if precision == "fp64" else (3e-5, 1e-4)
    phys = make_physics(w.physics)
    for k, e in enumerate(SAMPLES):
        mesh, ids = _patch(w, e)
        dp = Discretisation(mesh, phys)
        U = w.u0[ids]
        view = full_view[ids]
        A, B, C, D = (x[4] for x in element_blocks(dp, U, None, a_dt, view=view))
        for key, ref in zip("ABCD", (A, B, C, D)):
            assert _rel(got[key][k], ref) < tol_blk, (e, key)
        R, Fn = dp.residual(U, view)
        r_ref = -(U[4] - ustar[e] - a_dt * R[4]).reshape(-1)
        s_ref = -dp.trace_weights(Fn)[4].reshape(-1)
        assert _rel(got["r"][k], r_ref) < 1e-11, e
        assert _rel(got["s"][k], s_ref) < 1e-11, e
        # condensation of the oracle's blocks with the GPU's right-hand sides
        XB, xr, S, t = condense(A[None], B[None], C[None], D[None], got["r"][k][None], got["s"][k][None])
        assert _rel(cond["S"][k], S[0]) < tol_cond, e
        assert _rel(cond["XB"][k], XB[0]) < tol_cond, e
        assert _rel(cond["xr"][k], xr[0]) < tol_cond, e
        assert _rel(cond["t_k"][k], t[0]) < tol_cond, e


def _newton_norm(d, U, uh, Ustar, a_dt):
    """Oracle evaluation of the stage residual norm sqrt(|h|^2 + |g|^2) (all elements implicit)."""
    R, g = d.full_residual(U, uh)
    h = U - Ustar - a_dt * R
    return math.sqrt(float(np.sum(h * h) + np.sum(g * g)))


def _stage(w, precision):
    ctx = pkg.Context(w.mesh, w.physics, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    u_n = torch.tensor(w.u0, device=DEV)
    uh = ctx.hfr_initial_trace(u_n)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist, newton_tol=NEWTON_TOL, gmres_rtol=GMRES_RTOL)
    st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, newton_tol=NEWTON_TOL, newton_maxit=30,
                        gmres_rtol=GMRES_RTOL, gmres_maxit=3000)
    return st, us.cpu().numpy(), uh.cpu().numpy()


@pytest.mark.parametrize("name", ["vortex64", "vortex256"])
def test_full_size_stage_meets_newton_tolerance(name):
    w, d = _workload(name)
    a_dt = TABLEAUX["sdirk2"]["a"][0, 0] * w.dt
    nrm0 = _newton_norm(d, w.u0, d.initial_trace(w.u0), w.u0, a_dt)
    out = {}
    for label, prec in (("mixed", pkg.FR_PREC_FP32), ("fp64", pkg.FR_PREC_FP64)):
        st, U, uh = _stage(w, prec)
        assert st["converged"], label
        rel = _newton_norm(d, U, uh, w.u0, a_dt) / nrm0
        assert rel <= 1.05 * NEWTON_TOL, (label, rel)
        out[label] = U
    inc = np.abs(out["fp64"] - w.u0).max()
    # both solutions are within the Newton tolerance of the discrete solution: their difference
    # is the tolerance times the conditioning of the stage Jacobian relative to the increment
    assert np.abs(out["mixed"] - out["fp64"]).max() < 1e-6 * inc


def test_full_size_mixed_precision_error_at_tight_newton_tolerance():
    """The precision error of the mixed path apart from the Newton tolerance: the FP64 and the
    mixed-precision stage of vortex256 (the benchmark workload) converged to a relative FP64
    Newton residual of 1e-11, the mixed one with 0 and with 1 FP64 refinement sweep of its local
    solves, agree to 1e-8 relative to the stage increment (the mixed-precision target)."""
    w, _ = _workload("vortex256")
    kw = dict(newton_tol=1e-11, newton_maxit=40, gmres_rtol=1e-6, gmres_maxit=5000)
    u_n = torch.tensor(w.u0, device=DEV)

    def solve(prec, refine):
        ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist, **kw)
        st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, refine=refine, **kw)
        ctx.close()
        assert st["converged"], (prec, refine, st)
        return us

    ref = solve(pkg.FR_PREC_FP64, 0)
    inc = (ref - u_n).abs().max().item()
    for refine in (0, 1):
        us = solve(pkg.FR_PREC_FP32, refine)
        rel = (us - ref).abs().max().item() / inc
        assert rel < 1e-8, (refine, rel)
