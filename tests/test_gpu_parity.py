"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element on
seeded inputs, plus full-size checks of the bench workload by properties the oracle can
evaluate cheaply.

Tolerances.  FP64 path: the same discretisation evaluated in a different order, so agreement
is to rounding: 1e-11 relative to the magnitude of the compared array for residuals, blocks
and the condensed blocks (condition numbers of the element blocks are O(1)-O(10)), 1e-10 for the
trace solution of GMRES at rtol 1e-13 and its back-substitution, and 1e-10 relative to the stage
increment for converged stages.
FP32 blocks (mixed path): 3e-5 relative (FP32 rounding of O(n) accumulated terms); the
converged mixed-precision stage must match the FP64 stage to 1e-8 relative to the increment
(the FP64 Newton residual fixes the solution).
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
from oracle.solve import backsolve, condense, solve_trace  # noqa: E402
from oracle.stepping import TABLEAUX, imex_step, newton_stage  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import structured_quads, uniform_nodes  # noqa: E402
from workloads.states import isentropic_vortex, sample_points  # noqa: E402

DEV = "cuda"


def _band(n=8, p=2, physics="advdiff"):
    imp = np.zeros((n, n), bool)
    imp[n // 2 - 1:n // 2 + 1, :] = True
    if physics == "advdiff":
        mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=p, implicit=imp.reshape(-1))
        xy = sample_points(mesh, p)
        u0 = np.exp(-20 * ((xy[..., 0] - 0.5) ** 2 + (xy[..., 1] - 0.4) ** 2))[..., None]
        phys = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01, "lref": 1.0}
    else:
        mesh = structured_quads(uniform_nodes(n, 0, 10), uniform_nodes(n, 0, 10), p=p, implicit=imp.reshape(-1))
        u0 = isentropic_vortex(sample_points(mesh, p))
        phys = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}
    return mesh, u0, phys


CASES = {
    "advdiff8": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("advdiff8")),
    "advdiff_skew_p3": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("advdiff", n=5, p=3, jitter=0.15, seed=4)),
    "vortex_skew_p3": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("vortex", n=5, p=3, jitter=0.15, seed=9, re=200.0)),
    "vortex_p2": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("vortex", n=4, p=2, re=500.0)),
    "vortex_p4": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("vortex", n=3, p=4, re=500.0)),
    "vortex_p5": lambda: (lambda w: (w.mesh, w.u0, w.physics))(make_config("vortex", n=3, p=5, re=500.0)),
    "band_advdiff": lambda: _band(8, 2, "advdiff"),
    "band_ns": lambda: _band(6, 3, "ns"),
}


def _setup(name, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2):
    mesh, u0, phys = CASES[name]()
    ctx = pkg.Context(mesh, phys, precision=precision, tableau=tableau)
    disc = Discretisation(mesh, make_physics(phys))
    return ctx, disc, u0


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _perturbed_trace(disc, u0, seed=0):
    uh = disc.initial_trace(u0)
    rng = np.random.default_rng(seed)
    return uh * (1.0 + 1e-3 * rng.standard_normal(uh.shape))


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_trace_residual(name):
    ctx, d, u0 = _setup(name)
    uh = _perturbed_trace(d, u0)
    R, g = ctx.fr_residual(torch.tensor(u0, device=DEV), torch.tensor(uh, device=DEV))
    Ro, go = d.full_residual(u0, uh)
    assert _rel(R.cpu().numpy(), Ro) < 1e-11
    if d.ntrace:
        assert _rel(g.cpu().numpy(), go) < 1e-11


@pytest.mark.parametrize("name", ["advdiff8", "vortex_skew_p3", "band_ns"])
def test_initial_trace_and_solution_points(name):
    ctx, d, u0 = _setup(name)
    uh = ctx.hfr_initial_trace(torch.tensor(u0, device=DEV))
    assert _rel(uh.cpu().numpy(), d.initial_trace(u0)) < 1e-14
    assert _rel(ctx.solution_points().cpu().numpy(), d.geo.xy) < 1e-14


def _blocks_both(name, precision, a_dt=0.037):
    ctx, d, u0 = _setup(name, precision)
    uh = _perturbed_trace(d, u0, 1)
    ustar = u0 * 0.999
    ctx.hfr_local_jacobian(torch.tensor(u0, device=DEV), torch.tensor(uh, device=DEV),
                           torch.tensor(ustar, device=DEV), a_dt)
    A, B, C, D = element_blocks(d, u0, uh, a_dt)
    imp = d.imp_idx
    return ctx, d, u0, uh, ustar, a_dt, (A[imp], B[imp], C[imp], D[imp])


@pytest.mark.parametrize("name", ["advdiff8", "advdiff_skew_p3", "vortex_skew_p3", "vortex_p2", "vortex_p4",
                                  "vortex_p5", "band_advdiff", "band_ns"])
def test_element_blocks_fp64(name):
    ctx, d, u0, uh, ustar, a_dt, blocks = _blocks_both(name, pkg.FR_PREC_FP64)
    for key, ref in zip("ABCD", blocks):
        got = ctx.hfr_export(key).cpu().numpy()
        assert _rel(got, ref) < 1e-11, key
    # Newton right-hand sides r = -h, s = -g^k
    R, Fn = d.residual(u0, d.trace_view(uh))
    imp = d.imp_idx
    r_ref = -(u0[imp] - ustar[imp] - a_dt * R[imp]).reshape(len(imp), -1)
    s_ref = -d.trace_weights(Fn)[imp].reshape(len(imp), -1)
    assert _rel(ctx.hfr_export("r").cpu().numpy(), r_ref) < 1e-11
    assert _rel(ctx.hfr_export("s").cpu().numpy(), s_ref) < 1e-11


@pytest.mark.parametrize("name", ["vortex_skew_p3", "vortex_p4", "vortex_p5", "band_ns"])
def test_element_blocks_and_condense_fp32(name):
    ctx, d, u0, uh, ustar, a_dt, blocks = _blocks_both(name, pkg.FR_PREC_FP32)
    for key, ref in zip("ABCD", blocks):
        got = ctx.hfr_export(key).cpu().numpy().astype(np.float64)
        assert _rel(got, ref) < 3e-5, key
    # FP32 condensation of the FP32 blocks against the FP64 condensation of the oracle's blocks:
    # differences come from FP32 rounding amplified by the block condition numbers (O(1e2))
    ctx.hfr_condense(refine=0)
    A, B, C, D = blocks
    r = ctx.hfr_export("r").cpu().numpy()
    s = ctx.hfr_export("s").cpu().numpy()
    XB, xr, S, t = condense(A, B, C, D, r, s)
    assert _rel(ctx.hfr_export("S").cpu().numpy().astype(np.float64), S) < 1e-4
    assert _rel(ctx.hfr_export("XB").cpu().numpy().astype(np.float64), XB) < 1e-4
    assert _rel(ctx.hfr_export("xr").cpu().numpy(), xr) < 1e-4


@pytest.mark.parametrize("name", ["advdiff8", "vortex_skew_p3", "vortex_p4", "band_ns"])
def test_condense_gmres_backsolve_fp64(name):
    ctx, d, u0, uh, ustar, a_dt, (A, B, C, D) = _blocks_both(name, pkg.FR_PREC_FP64)
    ctx.hfr_condense(refine=0)
    r = ctx.hfr_export("r").cpu().numpy()
    s = ctx.hfr_export("s").cpu().numpy()
    XB, xr, S, t = condense(A, B, C, D, r, s)
    # FP64 path: 1e-11 for the condensed blocks (condition numbers of A are O(1)-O(10) here;
    # measured on GB300 1e-15), 1e-10 for the GMRES solution at rtol 1e-13 and its back-substitution
    # (measured 5e-14)
    assert _rel(ctx.hfr_export("S").cpu().numpy(), S) < 1e-11
    assert _rel(ctx.hfr_export("XB").cpu().numpy(), XB) < 1e-11
    assert _rel(ctx.hfr_export("xr").cpu().numpy(), xr) < 1e-11
    assert _rel(ctx.hfr_export("t_k").cpu().numpy(), t) < 1e-11
    # face-block Jacobi preconditioner blocks
    from oracle.solve import face_block_jacobi
    assert _rel(ctx.hfr_export("Pinv").cpu().numpy(), face_block_jacobi(d, S, d.imp_idx)) < 1e-11
    duh_ref, _, _ = solve_trace(d, S, t, d.imp_idx, method="direct")
    duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-13, maxit=3000)
    assert rel <= 1e-12
    assert _rel(duh.cpu().numpy().reshape(-1), duh_ref) < 1e-10
    du = ctx.hfr_backsolve(duh, refine=0).cpu().numpy()
    dview = d.trace_view(duh_ref.reshape(d.ntrace, d.n, d.nv))[d.imp_idx].reshape(len(d.imp_idx), -1)
    assert _rel(du, backsolve(XB, xr, dview)) < 1e-10


def test_fp64_refinement_sweep_is_consistent():
    """Refinement against the FP64 linearisation leaves an already exact FP64 solve unchanged
    (to rounding): checks the JVP used for refinement equals the assembled blocks."""
    ctx, d, u0, uh, ustar, a_dt, _ = _blocks_both("vortex_skew_p3", pkg.FR_PREC_FP64)
    ctx.hfr_condense(refine=0)
    duh, _, _ = ctx.hfr_trace_gmres(rtol=1e-13, maxit=3000)
    du0 = ctx.hfr_backsolve(duh, refine=0).cpu().numpy()
    du2 = ctx.hfr_backsolve(duh, refine=2).cpu().numpy()
    assert _rel(du2, du0) < 1e-10


@pytest.mark.parametrize("name,tab", [("advdiff8", "be"), ("vortex_skew_p3", "sdirk2"), ("vortex_p4", "sdirk2")])
def test_newton_stage_matches_oracle(name, tab):
    tabc = pkg.FR_TAB_BE if tab == "be" else pkg.FR_TAB_SDIRK2
    ctx, d, u0 = _setup(name, tableau=tabc)
    dt = 0.05 if tab == "be" else 0.2
    a11 = TABLEAUX[tab]["a"][0, 0]
    U_o, uh_o, info = newton_stage(d, u0, u0, d.initial_trace(u0), a11 * dt, tol=1e-13)
    u = torch.tensor(u0, device=DEV)
    uh = ctx.hfr_initial_trace(u)
    R_hist = ctx.empty(ctx.info.nstages + 1, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, dt, u, us, uh, R_hist)
    st = ctx.imex_stage(1, dt, u, us, uh, R_hist, newton_tol=1e-13, gmres_rtol=1e-14, gmres_maxit=3000)
    assert st["converged"]
    inc = np.abs(U_o - u0).max()
    assert np.abs(us.cpu().numpy() - U_o).max() < 1e-10 * inc
    assert np.abs(uh.cpu().numpy() - uh_o).max() < 1e-10 * max(inc, 1e-300) + 1e-13 * np.abs(uh_o).max()
    # the stored stage derivative is R(u_1, u^_1)
    R1, _ = d.full_residual(U_o, uh_o)
    assert _rel(R_hist[1].cpu().numpy(), R1) < 1e-8


@pytest.mark.parametrize("name", ["band_advdiff", "band_ns"])
def test_imex_step_matches_oracle(name):
    ctx, d, u0 = _setup(name, tableau=pkg.FR_TAB_SDIRK2)
    dt = 0.01 if name == "band_advdiff" else 0.02
    U_o, uh_o, _ = imex_step(d, u0, d.initial_trace(u0), dt, "sdirk2", tol=1e-13)
    u = torch.tensor(u0, device=DEV)
    uh = ctx.hfr_initial_trace(u)
    u1, stats = ctx.imex_step(dt, u, uh, newton_tol=1e-13, gmres_rtol=1e-14, gmres_maxit=3000)
    inc = np.abs(U_o - u0).max()
    assert np.abs(u1.cpu().numpy() - U_o).max() < 1e-10 * inc
    # discrete conservation across the interface on the GPU result (Sec. 4)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    m0 = np.einsum("s,es,esv->v", W, d.geo.J, u0)
    m1 = np.einsum("s,es,esv->v", W, d.geo.J, u1.cpu().numpy())
    assert np.abs(m1 - m0).max() < 1e-11 * np.abs(m0).max() + 1e-13


@pytest.mark.parametrize("refine", [0, 1])
def test_mixed_precision_stage_matches_fp64(refine):
    ctx64, d, u0 = _setup("vortex_skew_p3", pkg.FR_PREC_FP64)
    mesh, u0, phys = CASES["vortex_skew_p3"]()
    ctx32 = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2)
    dt = 0.2
    out = []
    for ctx in (ctx64, ctx32):
        u = torch.tensor(u0, device=DEV)
        uh = ctx.hfr_initial_trace(u)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, dt, u, us, uh, R_hist)
        st = ctx.imex_stage(1, dt, u, us, uh, R_hist, newton_tol=1e-11, gmres_rtol=1e-6, refine=refine)
        assert st["converged"]
        out.append(us.cpu().numpy())
    inc = np.abs(out[0] - u0).max()
    assert np.abs(out[1] - out[0]).max() < 1e-8 * inc


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["vortex_p2", "vortex_skew_p3", "vortex_p4", "band_ns"])
def test_gmres_single_launch_and_multi_kernel_cycles_agree(name, precision):
    """The cooperative single-launch cycle and the multi-kernel cycle run the same iteration:
    both reach the requested residual on the condensed system and agree with its direct
    solution (FP64: to the solve's rounding; FP32 S: to what FP32 mat-vecs allow)."""
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    ctx, d, *_ = _blocks_both(name, prec)
    ctx.hfr_condense(refine=0)
    assert ctx.hfr_gmres_get_mode() == pkg.FR_GMRES_FUSED
    S = ctx.hfr_export("S").cpu().numpy().astype(np.float64)
    t = ctx.hfr_export("t_k").cpu().numpy()
    duh_ref, _, _ = solve_trace(d, S, t, d.imp_idx, method="direct")
    rtol, tol = (1e-12, 1e-9) if precision == "fp64" else (1e-5, 2e-3)
    out, its = {}, {}
    for mode in (pkg.FR_GMRES_FUSED, pkg.FR_GMRES_MULTI):
        ctx.hfr_gmres_set_mode(mode)
        duh, it, rel = ctx.hfr_trace_gmres(rtol=rtol, maxit=3000)
        assert rel <= 10 * rtol, (mode, rel)
        out[mode] = duh.cpu().numpy().reshape(-1)
        its[mode] = it
        assert _rel(out[mode], duh_ref) < tol, mode
    assert abs(its[pkg.FR_GMRES_FUSED] - its[pkg.FR_GMRES_MULTI]) <= 1 + its[pkg.FR_GMRES_MULTI] // 10
    assert _rel(out[pkg.FR_GMRES_FUSED], out[pkg.FR_GMRES_MULTI]) < tol


def test_gmres_single_launch_restarts_and_iteration_limit():
    mesh, u0, phys = CASES["vortex_skew_p3"]()
    ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP64, gmres_restart=5)
    d = Discretisation(mesh, make_physics(phys))
    uh = _perturbed_trace(d, u0, 1)
    ctx.hfr_local_jacobian(torch.tensor(u0, device=DEV), torch.tensor(uh, device=DEV),
                           torch.tensor(u0 * 0.999, device=DEV), 0.037)
    ctx.hfr_condense(refine=0)
    S = ctx.hfr_export("S").cpu().numpy()
    t = ctx.hfr_export("t_k").cpu().numpy()
    duh_ref, _, _ = solve_trace(d, S, t, d.imp_idx, method="direct")
    for mode in (pkg.FR_GMRES_FUSED, pkg.FR_GMRES_MULTI):
        ctx.hfr_gmres_set_mode(mode)
        duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-12, maxit=5000)
        assert its > 5 and rel <= 1e-11
        assert _rel(duh.cpu().numpy().reshape(-1), duh_ref) < 1e-9
        with pytest.raises(pkg.HfrError) as ei:
            ctx.hfr_trace_gmres(rtol=1e-12, maxit=7)
        assert ei.value.code == 4 and ei.value.info.iteration == 7
    with pytest.raises(pkg.HfrError) as ei:
        ctx.hfr_gmres_set_mode(7)
    assert ei.value.code == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chord_newton_stage_reaches_the_same_solution(precision):
    """Jacobian once per stage (chord iterations reuse blocks, factors and S_k): linear instead of
    quadratic Newton convergence, same FP64 residual test, same converged stage as the oracle's
    exact Newton solve."""
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    ctx, d, u0 = _setup("vortex_skew_p3", prec)
    dt = 0.2
    a11 = TABLEAUX["sdirk2"]["a"][0, 0]
    U_o, uh_o, _ = newton_stage(d, u0, u0, d.initial_trace(u0), a11 * dt, tol=1e-13)
    ctx.imex_set_jacobian_policy(pkg.FR_JAC_ONCE_PER_STAGE)
    u = torch.tensor(u0, device=DEV)
    uh = ctx.hfr_initial_trace(u)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, dt, u, us, uh, R_hist)
    st = ctx.imex_stage(1, dt, u, us, uh, R_hist, newton_tol=1e-11, newton_maxit=60, gmres_rtol=1e-9,
                        gmres_maxit=3000)
    assert st["converged"] and st["newton_iterations"] >= 2
    inc = np.abs(U_o - u0).max()
    assert np.abs(us.cpu().numpy() - U_o).max() < 1e-8 * inc
    with pytest.raises(pkg.HfrError) as ei:
        ctx.imex_set_jacobian_policy(5)
    assert ei.value.code == 1


@pytest.mark.parametrize("name", ["vortex_p2", "vortex_skew_p3", "vortex_p4", "band_ns"])
def test_tensor_core_and_fma_condensation_agree(name):
    """FP32 blocks: the three condensation modes -- factorisation and products on the FP32 FMA
    pipes, products on the tensor cores (tcgen05, 3xTF32), both on the tensor cores (blocked
    Gauss-Jordan with rank-16 tensor-core updates) -- agree to FP32-level rounding, and each
    matches the oracle's FP64 condensation of the same blocks."""
    ctx, d, u0, uh, ustar, a_dt, (A, B, C, D) = _blocks_both(name, pkg.FR_PREC_FP32)
    assert ctx.hfr_condense_get_mode() == pkg.FR_CONDENSE_TENSOR
    out = {}
    modes = (pkg.FR_CONDENSE_TENSOR, pkg.FR_CONDENSE_TENSOR_PRODUCTS, pkg.FR_CONDENSE_FMA)
    for mode in modes:
        ctx.hfr_condense_set_mode(mode)
        ctx.hfr_condense(refine=0)
        out[mode] = {k: ctx.hfr_export(k).cpu().numpy().astype(np.float64) for k in ("S", "XB", "xr", "t_k")}
    r = ctx.hfr_export("r").cpu().numpy()
    s = ctx.hfr_export("s").cpu().numpy()
    XB, xr, S, t = condense(A, B, C, D, r, s)
    fma = out[pkg.FR_CONDENSE_FMA]
    for key, ref in (("S", S), ("XB", XB), ("xr", xr), ("t_k", t)):
        # same factorisation, different product arithmetic
        assert _rel(out[pkg.FR_CONDENSE_TENSOR_PRODUCTS][key], fma[key]) < 2e-5, key
        # different factorisation arithmetic (and possibly pivot order on near ties)
        assert _rel(out[pkg.FR_CONDENSE_TENSOR][key], fma[key]) < 5e-5, key
        for mode in modes:
            assert _rel(out[mode][key], ref) < 1e-4, (mode, key)


@pytest.mark.parametrize("name", ["vortex_skew_p3", "vortex_p4"])
def test_single_pass_tf32_condensation(name):
    """FR_CONDENSE_TENSOR_TF32: the tensor-core kernels with one TF32 product per term.  Its
    condensation is within TF32 accuracy of the oracle and visibly less accurate than 3xTF32 (the
    mode is in effect); the implicit stage still converges to the FP64 stage's solution, since the
    FP64 Newton residual decides convergence."""
    ctx, d, u0, uh, ustar, a_dt, (A, B, C, D) = _blocks_both(name, pkg.FR_PREC_FP32)
    r = ctx.hfr_export("r").cpu().numpy()
    s = ctx.hfr_export("s").cpu().numpy()
    XB, xr, S, t = condense(A, B, C, D, r, s)
    err = {}
    for mode in (pkg.FR_CONDENSE_TENSOR, pkg.FR_CONDENSE_TENSOR_TF32):
        ctx.hfr_condense_set_mode(mode)
        assert ctx.hfr_condense_get_mode() == mode
        ctx.hfr_condense(refine=0)
        got = {k: ctx.hfr_export(k).cpu().numpy().astype(np.float64) for k in ("S", "XB")}
        err[mode] = max(_rel(got["S"], S), _rel(got["XB"], XB))
    assert err[pkg.FR_CONDENSE_TENSOR] < 1e-4
    assert err[pkg.FR_CONDENSE_TENSOR_TF32] < 2e-2
    assert err[pkg.FR_CONDENSE_TENSOR_TF32] > 3 * err[pkg.FR_CONDENSE_TENSOR]
    # the stage: same FP64 Newton test, same solution
    mesh, u0, phys = CASES[name]()
    res = {}
    for prec in (pkg.FR_PREC_FP64, pkg.FR_PREC_FP32):
        c = pkg.Context(mesh, phys, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        if prec == pkg.FR_PREC_FP32:
            c.hfr_condense_set_mode(pkg.FR_CONDENSE_TENSOR_TF32)
        u = torch.tensor(u0, device=DEV)
        uhat = c.hfr_initial_trace(u)
        R_hist = c.empty(3, *c.state_shape)
        us = c.empty(*c.state_shape)
        c.imex_stage(0, 0.1, u, us, uhat, R_hist)
        st = c.imex_stage(1, 0.1, u, us, uhat, R_hist, newton_tol=1e-11, newton_maxit=60, gmres_rtol=1e-6,
                          gmres_maxit=3000)
        assert st["converged"]
        res[prec] = us.cpu().numpy()
    inc = np.abs(res[pkg.FR_PREC_FP64] - u0).max()
    assert np.abs(res[pkg.FR_PREC_FP32] - res[pkg.FR_PREC_FP64]).max() < 1e-8 * inc


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["vortex_skew_p3", "vortex_p4", "band_ns"])
def test_graph_stage_equals_stream_stage(name, precision):
    """The stage as one CUDA graph (conditional WHILE / IF nodes, device-side tests) runs the same
    kernels in the same order as the stream path: same solution, same iteration counts; a
    replay of the cached graph (same buffers) gives the same result again."""
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    mesh, u0, phys = CASES[name]()
    dt = 0.2 if name != "band_ns" else 0.02

    def run(ctx, bufs):
        u, us, uh, uh0, R_hist = bufs
        uh.copy_(uh0)
        ctx.imex_stage(0, dt, u, us, uh, R_hist)
        l0 = ctx.kernel_launches()
        st = ctx.imex_stage(1, dt, u, us, uh, R_hist, newton_tol=1e-10, gmres_rtol=1e-6, gmres_maxit=3000)
        assert st["converged"]
        return (us.cpu().numpy(), uh.cpu().numpy(), R_hist[1].cpu().numpy(), st["newton_iterations"],
                st["gmres_iterations"], ctx.kernel_launches() - l0)

    def buffers(ctx):
        u = torch.tensor(u0, device=DEV)
        uh0 = ctx.hfr_initial_trace(u)
        return u, ctx.empty(*ctx.state_shape), uh0.clone(), uh0, ctx.empty(3, *ctx.state_shape)

    ctx_s = pkg.Context(mesh, phys, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
    ref = run(ctx_s, buffers(ctx_s))
    ctx_g = pkg.Context(mesh, phys, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
    ctx_g.imex_stage_set_graph(True)
    assert ctx_g.imex_stage_get_graph() == 1
    bufs = buffers(ctx_g)
    inc = np.abs(ref[0] - u0).max()
    for _ in range(2):  # capture, then replay
        got = run(ctx_g, bufs)
        assert np.abs(got[0] - ref[0]).max() <= 1e-12 * inc
        assert _rel(got[1], ref[1]) < 1e-12
        assert _rel(got[2], ref[2]) < 1e-12
        assert got[3] == ref[3] and got[4] == ref[4]
        # kernel executions of a graph stage: the stream path's plus the device-side decisions
        assert got[5] > ref[5]


@pytest.mark.parametrize("name", ["vortex_p4", "band_ns"])
def test_autotune_picks_a_valid_configuration(name):
    """hfr_autotune times the condensation forms (and the tensor-core inverse's residency) and
    both GMRES cycle forms, keeps the fastest, and the tuned context still solves the stage."""
    mesh, u0, phys = CASES[name]()
    ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2)
    u = torch.tensor(u0, device=DEV)
    uh = ctx.hfr_initial_trace(u)
    rep = ctx.hfr_autotune(u, uh, u * 0.999, 0.05)
    assert rep["condense_mode"] == ctx.hfr_condense_get_mode()
    assert rep["gmres_mode"] == ctx.hfr_gmres_get_mode()
    assert all(rep["condense_ms"][m] > 0 for m in range(3))
    assert all(t > 0 for t in rep["inverse_ms"])
    assert rep["condense_ms"][rep["condense_mode"]] == min(rep["condense_ms"])
    assert 1 <= rep["inverse_ctas_per_sm"] or rep["condense_mode"] != pkg.FR_CONDENSE_TENSOR
    d = Discretisation(mesh, make_physics(phys))
    dt = 0.2 if name != "band_ns" else 0.02
    U_o, uh_o, _ = imex_step(d, u0, d.initial_trace(u0), dt, "sdirk2", tol=1e-12)
    u1, _ = ctx.imex_step(dt, u, ctx.hfr_initial_trace(u), newton_tol=1e-12, gmres_rtol=1e-8, gmres_maxit=3000)
    assert np.abs(u1.cpu().numpy() - U_o).max() < 1e-8 * np.abs(U_o - u0).max()


@pytest.mark.parametrize("name", ["vortex_skew_p3", "vortex_p4"])
def test_bf16_trace_operator_stage_converges_to_the_fp64_stage(name):
    """FR_PREC_BF16 stores S^k in BF16 for the GMRES mat-vecs (FP32 accumulation); the FP64 Newton
    residual still decides, so the converged stage is the FP64 one: at a 1e-12 Newton tolerance
    both agree to 1e-8 relative to the stage increment (the mixed-precision target)."""
    out = {}
    for prec in (pkg.FR_PREC_FP64, pkg.FR_PREC_BF16, pkg.FR_PREC_TF32):
        ctx, d, u0 = _setup(name, precision=prec)
        if prec == pkg.FR_PREC_BF16:
            assert ctx.hfr_gmres_get_mode() == pkg.FR_GMRES_FUSED
        u = torch.tensor(u0, device=DEV)
        uh = ctx.hfr_initial_trace(u)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, 0.2, u, us, uh, R_hist)
        st = ctx.imex_stage(1, 0.2, u, us, uh, R_hist, newton_tol=1e-12, newton_maxit=40, gmres_rtol=1e-6,
                            gmres_maxit=5000)
        assert st["converged"], (prec, st)
        out[prec] = us.cpu().numpy()
        ctx.close()
    inc = np.abs(out[pkg.FR_PREC_FP64] - u0).max()
    assert np.abs(out[pkg.FR_PREC_BF16] - out[pkg.FR_PREC_FP64]).max() < 1e-8 * inc
    assert np.abs(out[pkg.FR_PREC_TF32] - out[pkg.FR_PREC_FP64]).max() < 1e-8 * inc
