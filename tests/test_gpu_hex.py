"""Parity of the hexahedral path (3D Navier-Stokes, the channel workload's element type) with the
FP64 hexahedral oracle (oracle/fr3d.py), through the C ABI, on small meshes: skewed periodic
hexahedra (all implicit, and an IMEX band) and a tanh-clustered channel with no-slip walls whose
wall layers are implicit and whose centre is explicit:

* residual R and trace residual g (1e-11); the initial trace (1e-14);
* element blocks A, B, C, D of every implicit element (FP64 1e-11, FP32 3e-5 of the element's
  largest entry);
* the condensed Newton step (global-memory LU of the 320 x 320 blocks, trace GMRES at rtol 1e-13,
  back-substitution) against the oracle's condensed step with a direct trace solve (1e-10);
* a converged stage against Newton iterations of the oracle's condensed step;
* at full size (64 x 32 x 48 hexahedra, p = 3, 18 432 implicit): the rest state is steady and the
  mixed-precision stage agrees with the FP64 one to what the Newton tolerance fixes."""

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
from oracle.fr3d import Discretisation3D, condensed_newton_step, element_blocks_3d  # noqa: E402
from oracle.physics import make_physics  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import BC_WALL, structured_hexes, tanh_nodes, uniform_nodes  # noqa: E402
from workloads.states import channel_state, sample_points_hex  # noqa: E402

DEV = "cuda"
NS3 = {"kind": "ns3d", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0}
BASE = np.array([1.0, 0.3, -0.2, 0.1, 2.6])


def _state(mesh, p, seed):
    rng = np.random.default_rng(seed)
    xyz = sample_points_hex(mesh, p)
    wave = 0.05 * np.sin(xyz[..., :1]) * np.cos(xyz[..., 1:2]) * np.cos(xyz[..., 2:3])
    return BASE * (1 + wave) * (1 + 1e-2 * rng.standard_normal(xyz.shape[:2] + (5,)))


def _case(name):
    if name == "periodic_p2":
        n = 3
        nodes = [uniform_nodes(n, 0, 2.0)] * 3
        mesh = structured_hexes(*nodes, periodic=(True, True, True), jitter=0.12, seed=3, p=2)
        return mesh, _state(mesh, 2, 1)
    if name == "band_p3":
        n = 3
        imp = np.zeros((n, n, n), bool)  # [k, j, i]
        imp[:, 1, :] = True
        nodes = [uniform_nodes(n, 0, 2.0)] * 3
        mesh = structured_hexes(*nodes, periodic=(True, True, True), jitter=0.1, seed=4, p=3,
                                implicit=imp.reshape(-1))
        return mesh, _state(mesh, 3, 2)
    if name == "channel_p3":  # walls at y = +-1, one implicit layer per wall, explicit centre
        nx, ny, nz = 2, 4, 2
        j = np.arange(nx * ny * nz) // nx % ny
        mesh = structured_hexes(uniform_nodes(nx, 0, 2 * np.pi), tanh_nodes(ny, 2.5), uniform_nodes(nz, 0, np.pi),
                                periodic=(True, False, True), p=3, implicit=(j == 0) | (j == ny - 1),
                                bc_y=(BC_WALL, BC_WALL))
        U = _state(mesh, 3, 5)
        U[..., 1:4] *= (1 - sample_points_hex(mesh, 3)[..., 1:2] ** 2)  # no-slip compatible
        return mesh, U
    raise KeyError(name)


CASES = ["periodic_p2", "band_p3", "channel_p3"]


def _setup(name, precision=pkg.FR_PREC_FP64):
    mesh, U = _case(name)
    ctx = pkg.Context(mesh, NS3, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    assert ctx.general and ctx.hex
    d = Discretisation3D(mesh, make_physics(NS3))
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
def test_hex_residual_and_trace_residual(name):
    ctx, d, mesh, U = _setup(name)
    uh = _trace(d, U)
    R, g = ctx.fr_residual(torch.tensor(U.reshape(-1), device=DEV), torch.tensor(uh.reshape(-1), device=DEV))
    Ro, go = d.full_residual(U, uh)
    assert _rel(R.cpu().numpy(), Ro.reshape(-1)) < 1e-11
    if d.ntrace:
        assert _rel(g.cpu().numpy(), go.reshape(-1)) < 1e-11
    uhg = ctx.hfr_initial_trace(torch.tensor(U.reshape(-1), device=DEV))
    assert _rel(uhg.cpu().numpy(), d.initial_trace(U).reshape(-1)) < 1e-14
    xyz = ctx.solution_points().cpu().numpy()
    assert _rel(xyz, d.xyz.reshape(-1)) < 1e-14
    ctx.close()


def _blocks(name, precision, a_dt=0.021):
    ctx, d, mesh, U = _setup(name, precision)
    uh = _trace(d, U, 1)
    rng = np.random.default_rng(3)
    Ustar = U * (1 + 1e-4 * rng.standard_normal(U.shape))
    ctx.hfr_local_jacobian(torch.tensor(U.reshape(-1), device=DEV), torch.tensor(uh.reshape(-1), device=DEV),
                           torch.tensor(Ustar.reshape(-1), device=DEV), a_dt)
    return ctx, d, U, uh, Ustar, a_dt


_REF = {}


def _ref_blocks(name, d, U, uh, a_dt):
    key = (name, a_dt)
    if key not in _REF:
        _REF[key] = element_blocks_3d(d, U, uh, a_dt)
    return _REF[key]


@pytest.mark.parametrize("name", ["band_p3", "channel_p3"])
def test_hex_element_blocks_fp64(name):
    ctx, d, U, uh, Ustar, a_dt = _blocks(name, pkg.FR_PREC_FP64)
    A, B, C, D = _ref_blocks(name, d, U, uh, a_dt)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(d.imp_idx):
        for key, ref in zip("ABCD", (A, B, C, D)):
            assert _rel(got[key][k], ref[e]) < 1e-11, (e, key)
    ctx.close()


def test_hex_element_blocks_fp32():
    ctx, d, U, uh, Ustar, a_dt = _blocks("channel_p3", pkg.FR_PREC_FP32)
    A, B, C, D = _ref_blocks("channel_p3", d, U, uh, a_dt)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(d.imp_idx):
        for key, ref in zip("ABCD", (A, B, C, D)):
            assert _rel(got[key][k], ref[e]) < 3e-5, (e, key)
    ctx.close()


@pytest.mark.parametrize("name", ["band_p3", "channel_p3"])
def test_hex_condensed_newton_step_fp64(name):
    ctx, d, U, uh, Ustar, a_dt = _blocks(name, pkg.FR_PREC_FP64)
    ctx.hfr_condense(refine=0)
    duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-13, maxit=5000)
    assert rel <= 1e-12
    du = ctx.hfr_backsolve(duh).cpu().numpy()
    dU_ref, duh_ref = condensed_newton_step(d, U, uh, Ustar, a_dt)
    scale = max(np.abs(duh_ref).max(), np.abs(dU_ref).max())
    assert np.abs(duh.cpu().numpy() - duh_ref.reshape(-1)).max() < 1e-10 * scale
    assert np.abs(du - dU_ref[d.imp_idx].reshape(-1)).max() < 1e-10 * scale
    ctx.close()


@pytest.mark.parametrize("prec", [pkg.FR_PREC_FP64, pkg.FR_PREC_FP32])
def test_hex_stage_matches_oracle_newton(prec):
    ctx, d, mesh, U = _setup("channel_p3", prec)
    dt = 0.01
    a11 = 1.0 - np.sqrt(2.0) / 2.0
    u_n = torch.tensor(U.reshape(-1), device=DEV)
    uh = ctx.hfr_initial_trace(u_n)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, dt, u_n, us, uh, R_hist)
    st = ctx.imex_stage(1, dt, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-10,
                        gmres_maxit=5000)
    assert st["converged"]
    # the oracle from the same start: explicit elements u_n + dt gamma R(u_n); implicit ones Newton
    uh0 = d.initial_trace(U)
    R0, _ = d.full_residual(U, uh0)
    Us = U + np.where(d.imp[:, None, None], 0.0, dt * a11 * R0)
    Uo, uho = Us.copy(), uh0.copy()
    n0 = None
    for _ in range(12):
        R, g = d.full_residual(Uo, uho)
        h = Uo[d.imp_idx] - Us[d.imp_idx] - a11 * dt * R[d.imp_idx]
        nrm = np.sqrt(np.sum(h * h) + np.sum(g * g))
        n0 = nrm if n0 is None else n0
        if nrm <= 1e-12 * n0:
            break
        dU, dh = condensed_newton_step(d, Uo, uho, Us, a11 * dt)
        Uo, uho = Uo + dU, uho + dh
    inc = np.abs(Uo - U).max()
    assert np.abs(us.cpu().numpy() - Uo.reshape(-1)).max() < 1e-9 * inc
    ctx.close()


# ------------------------------------------------------------------ full size (channel3d)
_CH = {}


def _channel():
    if "w" not in _CH:
        _CH["w"] = make_config("channel3d")
    return _CH["w"]


@pytest.mark.parametrize("prec", [pkg.FR_PREC_FP64, pkg.FR_PREC_FP32])
def test_hex_graph_stage_equals_stream_stage(prec):
    """The hexahedral stage as one CUDA graph gives the stream stage's result bit for bit, with the
    same Newton and GMRES iteration counts."""
    mesh, U = _case("channel_p3")
    out = []
    for graph in (False, True):
        ctx = pkg.Context(mesh, NS3, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        if graph:
            ctx.imex_stage_set_graph(True)
        u_n = torch.tensor(U.reshape(-1), device=DEV)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, 0.01, u_n, us, uh, R_hist)
        st = ctx.imex_stage(1, 0.01, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-10,
                            gmres_maxit=5000)
        assert st["converged"]
        out.append((us.clone(), uh.clone(), st["newton_iterations"], st["gmres_iterations"]))
        ctx.close()
    assert out[0][2:] == out[1][2:]
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_full_size_channel_rest_state_is_steady():
    w = _channel()
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP32, tableau=pkg.FR_TAB_SDIRK2)
    assert ctx.info.nimplicit == 18432 and ctx.info.nA == 320 and ctx.info.nT == 480
    rest = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / (1.4 * 0.4)])
    U = torch.tensor(np.tile(rest, int(ctx.info.state_values) // 5), device=DEV)
    uh = ctx.hfr_initial_trace(U)
    R, g = ctx.fr_residual(U, uh)
    assert R.abs().max().item() < 1e-9 and g.abs().max().item() < 1e-12
    ctx.close()


def test_full_size_channel_stage_mixed_and_fp64_agree():
    w = _channel()
    out = {}
    for label, prec in (("fp64", pkg.FR_PREC_FP64), ("mixed", pkg.FR_PREC_FP32)):
        ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        u_n = torch.tensor(w.u0.reshape(-1), device=DEV)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist)
        st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, newton_tol=1e-10, newton_maxit=30, gmres_rtol=1e-6,
                            gmres_maxit=20000)
        assert st["converged"], (label, st)
        out[label] = (us - u_n).cpu().numpy()
        ctx.close()
        del R_hist, us, uh
        torch.cuda.empty_cache()
    inc = np.abs(out["fp64"]).max()
    assert np.abs(out["mixed"] - out["fp64"]).max() < 1e-6 * inc
