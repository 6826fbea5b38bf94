"""Several IMEX steps with the element Jacobian held across stages and steps (FR_JAC_KEEP, the
paper's practice of refreshing the Jacobian every 100 steps, Sec. 5) through the C entry
imex_steps: the chord-Newton steps reach the same discrete solution as the oracle's exact-Newton
steps (the FP64 Newton residual fixes it), the condensation is recomputed only when it must be
(first stage, a_ii dt changed, every refresh_every steps, after a public block call), and the
mixed-precision path under the same policy agrees with the FP64 path."""

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
from oracle.fr import Discretisation  # noqa: E402
from oracle.physics import make_physics  # noqa: E402
from oracle.stepping import imex_step  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import structured_quads, uniform_nodes  # noqa: E402
from workloads.states import isentropic_vortex, sample_points  # noqa: E402


def _band_ns(n=6, p=3):
    """IMEX band: the two middle element rows implicit, Navier-Stokes vortex."""
    imp = np.zeros((n, n), bool)
    imp[n // 2 - 1:n // 2 + 1, :] = True
    mesh = structured_quads(uniform_nodes(n, 0, 10), uniform_nodes(n, 0, 10), p=p, implicit=imp.reshape(-1))
    u0 = isentropic_vortex(sample_points(mesh, p))
    phys = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}
    return mesh, u0, phys


def _steps(ctx, u0, n, dt, **kw):
    u = torch.tensor(u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    st = ctx.imex_steps(n, dt, u, uh, **kw)
    return u, uh, st


def test_kept_jacobian_steps_match_the_oracle():
    mesh, u0, phys = _band_ns()
    d = Discretisation(mesh, make_physics(phys))
    dt, nsteps = 0.02, 3
    U, uh = u0, d.initial_trace(u0)
    for _ in range(nsteps):
        U, uh, _ = imex_step(d, U, uh, dt, "sdirk2", tol=1e-13)
    ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    ctx.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    u, _, st = _steps(ctx, u0, nsteps, dt, newton_tol=1e-12, newton_maxit=80, gmres_rtol=1e-13, gmres_maxit=3000)
    assert st["steps"] == nsteps and st["converged"] and st["max_rel_residual"] <= 1e-12
    # SDIRK2 has a_11 = a_22: one linearisation serves every stage of every step
    assert st["jacobian_refreshes"] == 1
    inc = np.abs(U - u0).max()
    assert np.abs(u.cpu().numpy() - U).max() < 1e-9 * inc


def test_refreshes_follow_the_policy():
    w = make_config("vortex", n=4, p=2, re=500.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    dt = 0.1
    kw = dict(newton_tol=1e-10, newton_maxit=80, gmres_rtol=1e-12, gmres_maxit=3000)
    # exact Newton: one linearisation per Newton iteration
    u_ex, _, st_ex = _steps(ctx, w.u0, 2, dt, **kw)
    assert st_ex["converged"] and st_ex["jacobian_refreshes"] == st_ex["newton_iterations"]
    ctx.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    u_k, uh, st = _steps(ctx, w.u0, 4, dt, refresh_every=2, **kw)
    assert st["converged"] and st["jacobian_refreshes"] == 2  # steps 0 and 2
    assert st["newton_iterations"] > 0
    # a new a_ii dt re-linearises once, then the new condensation is kept
    st = ctx.imex_steps(2, 0.5 * dt, u_k, uh, **kw)
    assert st["converged"] and st["jacobian_refreshes"] == 1
    # a public block call drops the held condensation; an explicit refresh asks for a new one
    ctx.hfr_local_jacobian(u_k, uh, u_k, 0.3)
    st = ctx.imex_steps(1, 0.5 * dt, u_k, uh, **kw)
    assert st["jacobian_refreshes"] == 1
    ctx.imex_refresh_jacobian()
    st = ctx.imex_steps(1, 0.5 * dt, u_k, uh, **kw)
    assert st["jacobian_refreshes"] == 1
    st = ctx.imex_steps(1, 0.5 * dt, u_k, uh, **kw)
    assert st["jacobian_refreshes"] == 0
    # the kept-Jacobian steps reach the exact-Newton steps' solution (same FP64 stopping test)
    u_k2, _, _ = _steps(ctx, w.u0, 2, dt, refresh_every=0, **kw)
    inc = (u_ex - torch.tensor(w.u0, device="cuda")).abs().max().item()
    assert (u_k2 - u_ex).abs().max().item() < 1e-8 * inc


def test_mixed_precision_kept_jacobian_matches_fp64():
    mesh, u0, phys = _band_ns()
    dt = 0.02
    kw = dict(newton_tol=1e-11, newton_maxit=80, gmres_rtol=1e-6, gmres_maxit=3000)
    ctx64 = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    u64, _, st64 = _steps(ctx64, u0, 2, dt, **kw)
    ctx32 = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2)
    ctx32.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    u32, _, st32 = _steps(ctx32, u0, 2, dt, **kw)
    assert st64["converged"] and st32["converged"] and st32["jacobian_refreshes"] == 1
    inc = (u64 - torch.tensor(u0, device="cuda")).abs().max().item()
    assert (u32 - u64).abs().max().item() < 1e-8 * inc


def test_imex_steps_rejects_bad_arguments():
    w = make_config("vortex", n=3, p=2, re=500.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    u = torch.tensor(w.u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    with pytest.raises(pkg.HfrError) as ei:
        ctx.imex_steps(1, -0.1, u, uh)
    assert ei.value.code == pkg.FR_ERR_INVALID_ARG
    with pytest.raises(pkg.HfrError) as ei:
        ctx.imex_set_jacobian_policy(7)
    assert ei.value.code == pkg.FR_ERR_INVALID_ARG
    st = ctx.imex_steps(0, 0.1, u, uh)
    assert st["steps"] == 0 and st["jacobian_refreshes"] == 0


def test_kept_jacobian_steps_conserve_across_the_interface():
    """Discrete conservation of every conserved variable over several steps on an IMEX band mesh
    (Sec. 4): it rests on the converged trace residual and the tableau (bhat_{j+1} = b_j), not on
    the Jacobian the Newton iterations used."""
    mesh, u0, phys = _band_ns()
    d = Discretisation(mesh, make_physics(phys))
    ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    ctx.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    u, _, st = _steps(ctx, u0, 3, 0.02, newton_tol=1e-12, newton_maxit=80, gmres_rtol=1e-13, gmres_maxit=3000)
    assert st["converged"] and st["jacobian_refreshes"] == 1
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    m0 = np.einsum("s,es,esv->v", W, d.geo.J, u0)
    m1 = np.einsum("s,es,esv->v", W, d.geo.J, u.cpu().numpy())
    assert np.abs(m1 - m0).max() < 1e-10 * np.abs(m0).max() + 1e-12


def _band_advdiff(n=8, p=2):
    imp = np.zeros((n, n), bool)
    imp[n // 2 - 1:n // 2 + 1, :] = True
    mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=p, implicit=imp.reshape(-1))
    xy = sample_points(mesh, p)
    u0 = np.exp(-20 * ((xy[..., 0] - 0.5) ** 2 + (xy[..., 1] - 0.4) ** 2))[..., None]
    phys = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01, "lref": 1.0}
    return mesh, u0, phys


@pytest.mark.parametrize("policy", ["every", "keep"])
def test_backward_euler_steps_match_the_oracle(policy):
    """imex_steps with backward Euler / ARS(1,2,1) on an IMEX band (advection-diffusion): two steps
    against the oracle's two steps, under exact Newton and with the Jacobian kept."""
    mesh, u0, phys = _band_advdiff()
    d = Discretisation(mesh, make_physics(phys))
    dt = 0.01
    U, uh = u0, d.initial_trace(u0)
    for _ in range(2):
        U, uh, _ = imex_step(d, U, uh, dt, "be", tol=1e-13)
    ctx = pkg.Context(mesh, phys, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_BE)
    if policy == "keep":
        ctx.imex_set_jacobian_policy(pkg.FR_JAC_KEEP)
    u, _, st = _steps(ctx, u0, 2, dt, newton_tol=1e-13, newton_maxit=80, gmres_rtol=1e-14, gmres_maxit=3000)
    assert st["converged"] and st["steps"] == 2
    # linear problem: exact Newton converges in one iteration per stage; kept blocks stay exact
    assert st["jacobian_refreshes"] == (st["newton_iterations"] if policy == "every" else 1)
    inc = np.abs(U - u0).max()
    assert np.abs(u.cpu().numpy() - U).max() < 1e-10 * inc


def test_single_pass_tf32_mode_needs_the_fp32_tensor_core_path():
    w = make_config("vortex", n=3, p=2, re=500.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    with pytest.raises(pkg.HfrError) as ei:
        ctx.hfr_condense_set_mode(pkg.FR_CONDENSE_TENSOR_TF32)
    assert ei.value.code == pkg.FR_ERR_UNSUPPORTED
    with pytest.raises(pkg.HfrError) as ei:
        ctx.hfr_condense_set_mode(9)
    assert ei.value.code == pkg.FR_ERR_INVALID_ARG
