"""Failure detection through the C ABI, with every fault made on the host (no GPU fault, trap or
hang): a non-finite state, a singular element block planted with hfr_import, and iteration limits.
Each call must return its status code (with the failing element or iteration in fr_last_error)
and leave the context usable: a clean call on the same context succeeds afterwards."""

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
from workloads import make_config  # noqa: E402


def _ctx(precision, p=3, n=4):
    w = make_config("vortex", n=n, p=p, re=500.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    return w, ctx


def _stage(ctx, w, u_n, **kw):
    uh = ctx.hfr_initial_trace(u_n)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist)
    return ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, **kw)


@pytest.mark.parametrize("precision", [pkg.FR_PREC_FP64, pkg.FR_PREC_FP32])
def test_nan_state_reports_diverged_and_context_survives(precision):
    w, ctx = _ctx(precision)
    u = torch.tensor(w.u0, device="cuda")
    bad = u.clone()
    bad[5, 3, 1] = float("nan")
    with pytest.raises(pkg.HfrError) as ei:
        uh = torch.tensor(np.zeros(ctx.trace_shape), device="cuda")
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(1, w.dt, bad, us, uh, R_hist)
    assert ei.value.code == pkg.FR_ERR_DIVERGED
    assert ei.value.info.iteration == 0
    st = _stage(ctx, w, u)  # the same context still solves a clean stage
    assert st["converged"]
    ctx.close()


@pytest.mark.parametrize("precision", [pkg.FR_PREC_FP64, pkg.FR_PREC_FP32])
def test_singular_block_reports_its_element(precision):
    w, ctx = _ctx(precision, p=3 if precision == pkg.FR_PREC_FP64 else 4)
    u = torch.tensor(w.u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    ctx.hfr_local_jacobian(u, uh, u, 0.05)
    A = ctx.hfr_export("A")
    good = A.clone()
    k = 7
    A[k, 11, :] = 0.0  # one zero row: no pivot in that row's column elimination
    ctx.hfr_import("A", A)
    with pytest.raises(pkg.HfrError) as ei:
        ctx.hfr_condense(refine=0)
    assert ei.value.code == pkg.FR_ERR_SINGULAR
    assert ei.value.info.element == k
    ctx.hfr_import("A", good)
    ctx.hfr_condense(refine=0)  # status words were cleared: the valid blocks condense
    ctx.close()


def test_newton_iteration_limit_reports_not_converged():
    w, ctx = _ctx(pkg.FR_PREC_FP64)
    u = torch.tensor(w.u0, device="cuda")
    with pytest.raises(pkg.HfrError) as ei:
        _stage(ctx, w, u, newton_tol=1e-14, newton_maxit=1, gmres_rtol=1e-2)
    assert ei.value.code == pkg.FR_ERR_NOT_CONVERGED
    assert ei.value.info.iteration == 1
    assert _stage(ctx, w, u)["converged"]
    ctx.close()


def test_gmres_iteration_limit_reports_not_converged():
    w, ctx = _ctx(pkg.FR_PREC_FP64)
    u = torch.tensor(w.u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    ctx.hfr_local_jacobian(u, uh, u * 0.999, 0.05)
    ctx.hfr_condense(refine=0)
    with pytest.raises(pkg.HfrError) as ei:
        ctx.hfr_trace_gmres(rtol=1e-14, maxit=3)
    assert ei.value.code == pkg.FR_ERR_NOT_CONVERGED
    duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-10, maxit=3000)
    assert rel <= 1e-10
    ctx.close()
