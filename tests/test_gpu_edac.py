"""The EDAC equations (Appendix A; hybridized stabilisation of Sec. 5.4) on the CUDA path against
the oracle: residual and trace residual, element blocks (FP64 and FP32), condensation + trace
solve + back-substitution (FP64), and whole stages / IMEX steps (FP64 and mixed, stream and
graph), on periodic and IMEX-band meshes, p = 2, 3, 4 (nv = 3: blocks 27/36, 48/48, 75/60)."""

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
from oracle.solve import backsolve, condense, solve_trace  # noqa: E402
from oracle.stepping import imex_step  # noqa: E402
from workloads import make_config  # noqa: E402

DEV = "cuda"


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _case(name):
    if name == "edac_p2":
        return make_config("edac", n=4, p=2, noise=1e-3, seed=1)
    if name == "edac_skew_p3":
        return make_config("edac", n=4, p=3, jitter=0.15, seed=2, noise=1e-3)
    if name == "edac_p4":
        return make_config("edac", n=3, p=4, noise=1e-3, seed=3)
    if name == "edac_band_p3":
        imp = np.zeros((6, 6), bool)
        imp[2:4, :] = True
        # explicit elements outside the band: a time step under their stability limit
        return make_config("edac", n=6, p=3, implicit=imp.reshape(-1), noise=1e-3, seed=4, cfl_mult=0.5)
    raise KeyError(name)


CASES = ["edac_p2", "edac_skew_p3", "edac_p4", "edac_band_p3"]


def _setup(name, precision=pkg.FR_PREC_FP64):
    w = _case(name)
    ctx = pkg.Context(w.mesh, w.physics, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    d = Discretisation(w.mesh, make_physics(w.physics))
    return w, ctx, d


@pytest.mark.parametrize("name", CASES)
def test_edac_residual(name):
    w, ctx, d = _setup(name)
    assert ctx.info.nv == 3
    uh = d.initial_trace(w.u0)
    uh = uh * (1.0 + 1e-3 * np.random.default_rng(0).standard_normal(uh.shape))
    R, g = ctx.fr_residual(torch.tensor(w.u0, device=DEV), torch.tensor(uh, device=DEV))
    Ro, go = d.full_residual(w.u0, uh)
    assert _rel(R.cpu().numpy(), Ro) < 1e-11
    assert _rel(g.cpu().numpy(), go) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_edac_blocks_and_condensation(name, precision):
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    w, ctx, d = _setup(name, prec)
    uh = d.initial_trace(w.u0)
    a_dt = 0.3 * w.dt
    ustar = w.u0 * 0.999
    ctx.hfr_local_jacobian(torch.tensor(w.u0, device=DEV), torch.tensor(uh, device=DEV),
                           torch.tensor(ustar, device=DEV), a_dt)
    A, B, C, D = element_blocks(d, w.u0, uh, a_dt)
    imp = d.imp_idx
    tb, tc = (1e-11, 1e-9) if precision == "fp64" else (3e-5, 1e-4)
    blocks = (A[imp], B[imp], C[imp], D[imp])
    for key, ref in zip("ABCD", blocks):
        assert _rel(ctx.hfr_export(key).cpu().numpy().astype(np.float64), ref) < tb, key
    ctx.hfr_condense(refine=0)
    r = ctx.hfr_export("r").cpu().numpy()
    s = ctx.hfr_export("s").cpu().numpy()
    XB, xr, S, t = condense(*blocks, r, s)
    assert _rel(ctx.hfr_export("S").cpu().numpy().astype(np.float64), S) < tc
    assert _rel(ctx.hfr_export("xr").cpu().numpy(), xr) < tc
    if precision == "fp64":
        duh_ref, _, _ = solve_trace(d, S, t, imp, method="direct")
        duh, _, rel = ctx.hfr_trace_gmres(rtol=1e-13, maxit=3000)
        assert rel <= 1e-12
        assert _rel(duh.cpu().numpy().reshape(-1), duh_ref) < 1e-9
        du = ctx.hfr_backsolve(duh, refine=0).cpu().numpy()
        dview = d.trace_view(duh_ref.reshape(d.ntrace, d.n, d.nv))[imp].reshape(len(imp), -1)
        assert _rel(du, backsolve(XB, xr, dview)) < 1e-9


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_edac_imex_step_matches_oracle(name, precision, graph):
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    w, ctx, d = _setup(name, prec)
    if graph:
        if ctx.hfr_gmres_get_mode() != pkg.FR_GMRES_FUSED:
            # face blocks without a single-launch cycle (bs = 9, 15): the graph stage is refused
            with pytest.raises(pkg.HfrError) as ei:
                ctx.imex_stage_set_graph(True)
            assert ei.value.code == pkg.FR_ERR_UNSUPPORTED
            return
        ctx.imex_stage_set_graph(True)
    # Theta = 100 puts the rounding floor of the relative stage residual near 2e-12: test at 1e-11
    U_o, _, _ = imex_step(d, w.u0, d.initial_trace(w.u0), w.dt, "sdirk2", tol=1e-11)
    u = torch.tensor(w.u0, device=DEV)
    u1, stats = ctx.imex_step(w.dt, u, ctx.hfr_initial_trace(u), newton_tol=1e-11,
                              gmres_rtol=1e-13 if precision == "fp64" else 1e-8, gmres_maxit=3000)
    inc = np.abs(U_o - w.u0).max()
    assert np.abs(u1.cpu().numpy() - U_o).max() < (1e-9 if precision == "fp64" else 1e-8) * inc


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("name", ["edac_p2", "edac_band_p3", "edac_p4"])
def test_modal_filter_matches_oracle(name, which):
    """Appendix B's modal filter on the GPU (operator built through orthonormality, V^{-1} =
    V^T W) against the oracle's (explicit Vandermonde inverse), on all, implicit or explicit
    elements."""
    from oracle.filter import apply_filter

    w, ctx, d = _setup(name)
    u = torch.tensor(w.u0, device=DEV)
    for alpha, s, ec, ratio in ((100.0, 1.0, 3, 1.0), (10.0, 2.0, 1, 0.25)):
        got = ctx.fr_modal_filter(u.clone(), alpha, s, ec, ratio, which).cpu().numpy()
        sel = {0: None, 1: d.imp_idx, 2: d.ex_idx}[which]
        ref = apply_filter(w.u0, w.p, alpha, s, ec, ratio, elements=sel)
        assert _rel(got, ref) < 1e-13
    with pytest.raises(pkg.HfrError):
        ctx.fr_modal_filter(u, -1.0, 1.0, 3)
