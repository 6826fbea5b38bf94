"""Parity of the interior-embedded variant EFR on the GPU (the trace continuous on the implicit
skeleton at the Gauss-Lobatto points of the trace faces, Sec. 2.2; FR_TRACE_EFR) with the EFR
oracle (oracle/efr.py), through the C ABI: periodic skewed meshes (all implicit, and an IMEX band)
and a wall band with wall and far-field faces (discontinuous boundary traces):

* residual R and node-wise trace residual g (1e-11); the initial trace (1e-14);
* element blocks A, B, C, D (FP64 1e-11, FP32 3e-5 of each element's largest entry);
* the condensed Newton step (node-assembled trace system, node-block Jacobi GMRES at rtol 1e-13)
  against the oracle's condensed step with a direct solve (1e-10);
* a converged stage against the oracle's EFR Newton stage, FP64 and mixed precision."""

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
from oracle.efr import EmbeddedDiscretisation, condensed_newton_step, newton_stage  # noqa: E402
from oracle.physics import make_physics  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import BC_FARFIELD, BC_WALL, geometric_nodes, structured_quads, uniform_nodes  # noqa: E402

DEV = "cuda"
NS_WALL = {"kind": "ns", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0}
U_INF = np.array([1.0, 0.3, 0.05, 2.6])


def _case(name):
    rng = np.random.default_rng(7)
    if name == "periodic_p3":
        w = make_config("vortex", n=4, p=3, jitter=0.12, seed=5, re=300.0)
        return w.mesh, w.physics, w.u0
    if name == "band_p2":
        n = 5
        band = np.zeros((n, n), bool)
        band[1:3, :] = True
        w = make_config("vortex", n=n, p=2, re=300.0, implicit=band.reshape(-1))
        return w.mesh, w.physics, w.u0
    if name == "wall_band_p3":
        yn = geometric_nodes(0.02, 1.6, 0.25, 1.0)
        ny = len(yn) - 1
        imp = np.zeros((ny, 3), bool)
        imp[:3] = True
        mesh = structured_quads(uniform_nodes(3, 0.0, 1.0), yn, periodic=(True, False), p=3,
                                implicit=imp.reshape(-1), bc_y=(BC_WALL, BC_FARFIELD))
        U = U_INF * (1 + 1e-2 * rng.standard_normal((mesh.nelem, 16, 4)))
        return mesh, dict(NS_WALL, u_inf=U_INF), U
    raise KeyError(name)


CASES = ["periodic_p3", "band_p2", "wall_band_p3"]


def _setup(name, precision=pkg.FR_PREC_FP64):
    mesh, phys, U = _case(name)
    ctx = pkg.Context(mesh, phys, precision=precision, tableau=pkg.FR_TAB_SDIRK2, trace_kind=pkg.FR_TRACE_EFR)
    assert ctx.general
    d = EmbeddedDiscretisation(mesh, make_physics(phys), phys.get("u_inf"))
    assert ctx.info.ntrace == d.nnode
    return ctx, d, mesh, U


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _trace(d, U, seed=0):
    rng = np.random.default_rng(seed)
    uh = d.initial_trace(U)
    return uh * (1 + 1e-3 * rng.standard_normal(uh.shape))


@pytest.mark.parametrize("name", CASES)
def test_efr_residual_trace_residual_and_initial_trace(name):
    ctx, d, mesh, U = _setup(name)
    uh = _trace(d, U)
    R, g = ctx.fr_residual(torch.tensor(U.reshape(-1), device=DEV), torch.tensor(uh.reshape(-1), device=DEV))
    Ro, go = d.full_residual(U, uh)
    assert _rel(R.cpu().numpy(), Ro.reshape(-1)) < 1e-11
    assert _rel(g.cpu().numpy(), go.reshape(-1)) < 1e-11
    uhg = ctx.hfr_initial_trace(torch.tensor(U.reshape(-1), device=DEV))
    assert _rel(uhg.cpu().numpy(), d.initial_trace(U).reshape(-1)) < 1e-14
    ctx.close()


_REF = {}


def _blocks(name, precision, a_dt=0.027):
    ctx, d, mesh, U = _setup(name, precision)
    uh = _trace(d, U, 1)
    rng = np.random.default_rng(3)
    Ustar = U * (1 + 1e-4 * rng.standard_normal(U.shape))
    ctx.hfr_local_jacobian(torch.tensor(U.reshape(-1), device=DEV), torch.tensor(uh.reshape(-1), device=DEV),
                           torch.tensor(Ustar.reshape(-1), device=DEV), a_dt)
    if name not in _REF:
        _REF[name] = element_blocks(d, U, uh, a_dt)
    return ctx, d, U, uh, Ustar, a_dt, _REF[name]


@pytest.mark.parametrize("name", CASES)
def test_efr_element_blocks_fp64(name):
    ctx, d, U, uh, Ustar, a_dt, ref = _blocks(name, pkg.FR_PREC_FP64)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(d.imp_idx):
        for key, blk in zip("ABCD", ref):
            assert _rel(got[key][k], blk[e]) < 1e-11, (e, key)
    ctx.close()


def test_efr_element_blocks_fp32():
    ctx, d, U, uh, Ustar, a_dt, ref = _blocks("wall_band_p3", pkg.FR_PREC_FP32)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(d.imp_idx):
        for key, blk in zip("ABCD", ref):
            assert _rel(got[key][k], blk[e]) < 3e-5, (e, key)
    ctx.close()


@pytest.mark.parametrize("name", CASES)
def test_efr_condensed_newton_step_fp64(name):
    ctx, d, U, uh, Ustar, a_dt, _ = _blocks(name, pkg.FR_PREC_FP64)
    ctx.hfr_condense(refine=0)
    duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-13, maxit=5000)
    assert rel <= 1e-12
    du = ctx.hfr_backsolve(duh).cpu().numpy()
    dU_ref, duh_ref = condensed_newton_step(d, U, uh, Ustar, a_dt)
    scale = max(np.abs(duh_ref).max(), np.abs(dU_ref).max())
    assert np.abs(duh.cpu().numpy() - duh_ref.reshape(-1)).max() < 1e-10 * scale
    assert np.abs(du - dU_ref[d.imp_idx].reshape(-1)).max() < 1e-10 * scale
    ctx.close()


@pytest.mark.parametrize("name,prec", [("periodic_p3", pkg.FR_PREC_FP64), ("periodic_p3", pkg.FR_PREC_FP32)])
def test_efr_stage_matches_oracle_newton(name, prec):
    """All elements implicit: the stage from u* = u_n converges to the oracle's EFR stage."""
    ctx, d, mesh, U = _setup(name, prec)
    dt = 0.2
    a11 = 1.0 - np.sqrt(2.0) / 2.0
    u_n = torch.tensor(U.reshape(-1), device=DEV)
    uh = ctx.hfr_initial_trace(u_n)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, dt, u_n, us, uh, R_hist)
    st = ctx.imex_stage(1, dt, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-10,
                        gmres_maxit=5000)
    assert st["converged"]
    Uo, _, info = newton_stage(d, U, U, d.initial_trace(U), a11 * dt, tol=1e-12)
    assert info["converged"]
    inc = np.abs(Uo - U).max()
    assert np.abs(us.cpu().numpy() - Uo.reshape(-1)).max() < 1e-9 * inc
    ctx.close()


def test_efr_graph_stage_equals_stream_stage():
    """The EFR stage as one CUDA graph gives the stream stage's result bit for bit."""
    mesh, phys, U = _case("band_p2")
    out = []
    for graph in (False, True):
        ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2,
                          trace_kind=pkg.FR_TRACE_EFR)
        if graph:
            ctx.imex_stage_set_graph(True)
        u_n = torch.tensor(U.reshape(-1), device=DEV)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, 0.05, u_n, us, uh, R_hist)
        st = ctx.imex_stage(1, 0.05, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-8,
                            gmres_maxit=5000)
        assert st["converged"]
        out.append((us.clone(), uh.clone(), st["newton_iterations"], st["gmres_iterations"]))
        ctx.close()
    assert out[0][2:] == out[1][2:]
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ full size (vortex256 mesh)
def test_full_size_efr_free_stream_and_mixed_against_fp64():
    """The EFR trace on the 256 x 256 p = 4 vortex mesh (458 752 trace nodes): a uniform state
    with its initial trace is steady (R and g vanish to rounding over all 65 536 elements), and the
    implicit stage converges on the FP64 and the mixed-precision path to the same state, to what
    the Newton tolerance fixes."""
    w = make_config("vortex256")
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2,
                      trace_kind=pkg.FR_TRACE_EFR)
    assert ctx.general and ctx.info.ntrace == 458752
    ufs = np.array([1.0, 0.5, 0.0, 1.0 / (1.4 * 0.4) + 0.125])
    U = torch.tensor(np.tile(ufs, int(ctx.info.state_values) // 4), device=DEV)
    uh = ctx.hfr_initial_trace(U)
    R, g = ctx.fr_residual(U, uh)
    assert R.abs().max().item() < 1e-10
    assert g.abs().max().item() < 1e-12
    ctx.close()
    out = {}
    for label, prec in (("fp64", pkg.FR_PREC_FP64), ("mixed", pkg.FR_PREC_FP32)):
        ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2, trace_kind=pkg.FR_TRACE_EFR)
        u_n = torch.tensor(w.u0.reshape(-1), device=DEV)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist)
        st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, newton_tol=1e-11, newton_maxit=30, gmres_rtol=1e-6,
                            gmres_maxit=5000)
        assert st["converged"], (label, st)
        out[label] = (us - u_n).cpu().numpy()
        ctx.close()
    inc = np.abs(out["fp64"]).max()
    assert np.abs(out["mixed"] - out["fp64"]).max() < 1e-9 * inc
