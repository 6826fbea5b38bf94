"""Parity of the general-mesh path (per-element degree, faces between unequal degrees, wall and
far-field faces; the shape of the boundary-layer workload) with the FP64 mixed-degree oracle
(oracle/fr_mixed.py, oracle/blocks_mixed.py), through the C ABI, element by element on small
meshes that span several degrees, IMEX bands and both boundary kinds:

* residual R and trace residual g; the initial trace;
* element blocks A, B, C, D (FP64: 1e-11 of each element's largest entry; FP32: 3e-5);
* the condensed Newton step (condensation, GMRES at rtol 1e-13, back-substitution) against the
  oracle's hybridized step: 1e-10 relative;
* a converged implicit stage against Newton iterations of the oracle's hybridized step;
* at full size (400 x 500 quads, p in 2..5, the boundary-layer workload): the rest state is
  steady (R and g vanish to rounding) and the mixed-precision stage converges and agrees with the
  FP64 one to what the Newton tolerance fixes.

FP64 tolerances are rounding-level for the same discretisation in a different operation order;
the blocks are compared per element relative to that element's largest entry (the stretched
cells' blocks differ by orders of magnitude from one element to the next)."""

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
from oracle.blocks_mixed import element_blocks_mixed, hybridized_step, stage_residual, trace_flatten  # noqa: E402
from oracle.fr_mixed import MixedDiscretisation  # noqa: E402
from oracle.physics import make_physics  # noqa: E402
from workloads import make_config  # noqa: E402
from workloads.mesh import BC_FARFIELD, BC_WALL, geometric_nodes, structured_quads, uniform_nodes  # noqa: E402
from workloads.states import isentropic_vortex, sample_points_mixed  # noqa: E402

DEV = "cuda"
NS = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}
NS_WALL = {"kind": "ns", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0}
ADVDIFF = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01, "lref": 1.0}
U_INF = np.array([1.0, 0.3, 0.05, 2.6])


def _grid_mesh(n, L, degrees, seed, implicit, jitter=0.1):
    p = np.random.default_rng(seed).choice(degrees, size=n * n).astype(np.int32)
    return structured_quads(uniform_nodes(n, 0, L), uniform_nodes(n, 0, L), jitter=jitter, seed=seed, p=p,
                            implicit=implicit)


def _bl_mesh(nx, degrees, imp_rows, bc_y, seed, h0=0.02, ratio=1.6, jitter=0.0):
    yn = geometric_nodes(h0, ratio, 0.25, 1.0)
    ny = len(yn) - 1
    imp = np.zeros((ny, nx), bool)
    imp[imp_rows, :] = True
    p = np.random.default_rng(seed).choice(degrees, size=nx * ny).astype(np.int32)
    return structured_quads(uniform_nodes(nx, 0.0, 1.0), yn, periodic=(True, False), jitter=jitter, seed=seed, p=p,
                            implicit=imp.reshape(-1), bc_y=bc_y)


def _case(name):
    """(mesh, physics dict, state list)."""
    rng = np.random.default_rng(11)
    if name == "mixed_periodic_ns":
        mesh = _grid_mesh(4, 10.0, [2, 3, 4, 5], 3, np.ones(16, bool))
        U = [isentropic_vortex(x) for x in sample_points_mixed(mesh)]
        return mesh, NS, U
    if name == "mixed_band_ns":
        n = 5
        band = np.zeros((n, n), bool)
        band[1:3, :] = True
        mesh = _grid_mesh(n, 10.0, [2, 3, 4], 5, band.reshape(-1))
        U = [isentropic_vortex(x) for x in sample_points_mixed(mesh)]
        return mesh, NS, U
    if name == "mixed_band_advdiff":
        n = 5
        band = np.zeros((n, n), bool)
        band[2:4, :] = True
        mesh = _grid_mesh(n, 1.0, [1, 2, 3], 6, band.reshape(-1))
        U = [np.exp(-20 * ((x[:, :1] - 0.5) ** 2 + (x[:, 1:] - 0.4) ** 2)) for x in sample_points_mixed(mesh)]
        return mesh, ADVDIFF, U
    if name == "wall_band_ns":  # stretched wall band, implicit near the wall, explicit far field above
        mesh = _bl_mesh(3, [2, 3, 4, 5], [0, 1, 2], (BC_WALL, BC_FARFIELD), seed=2)
        U = [U_INF * (1 + 1e-2 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 4))) for e in range(mesh.nelem)]
        return mesh, dict(NS_WALL, u_inf=U_INF), U
    if name == "wall_channel_ns":  # all implicit, walls below, hybridized far field above
        mesh = _bl_mesh(3, [2, 3], list(range(8)), (BC_WALL, BC_FARFIELD), seed=4, jitter=0.1)
        U = [U_INF * (1 + 1e-2 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 4))) for e in range(mesh.nelem)]
        return mesh, dict(NS_WALL, u_inf=U_INF), U
    raise KeyError(name)


CASES = ["mixed_periodic_ns", "mixed_band_ns", "mixed_band_advdiff", "wall_band_ns", "wall_channel_ns"]


def _setup(name, precision=pkg.FR_PREC_FP64):
    mesh, phys, U = _case(name)
    ctx = pkg.Context(mesh, phys, precision=precision, tableau=pkg.FR_TAB_SDIRK2)
    assert ctx.general
    m = MixedDiscretisation(mesh, make_physics(phys), phys.get("u_inf"))
    return ctx, m, mesh, U


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _perturbed_trace(m, U, seed=0):
    rng = np.random.default_rng(seed)
    return [h * (1 + 1e-3 * rng.standard_normal(h.shape)) for h in m.initial_trace(U)]


@pytest.mark.parametrize("name", CASES)
def test_general_residual_and_trace_residual(name):
    ctx, m, mesh, U = _setup(name)
    uh = _perturbed_trace(m, U)
    R, g = ctx.fr_residual(torch.tensor(ctx.pack_state(U), device=DEV), torch.tensor(ctx.pack_trace(uh), device=DEV))
    Ro, go = m.full_residual(U, uh)
    assert _rel(R.cpu().numpy(), ctx.pack_state(Ro)) < 1e-11
    if m.ntrace:
        assert _rel(g.cpu().numpy(), trace_flatten(go)) < 1e-11
    ctx.close()


@pytest.mark.parametrize("name", ["mixed_band_ns", "wall_band_ns", "wall_channel_ns"])
def test_general_initial_trace_and_layout(name):
    ctx, m, mesh, U = _setup(name)
    uh = ctx.hfr_initial_trace(torch.tensor(ctx.pack_state(U), device=DEV))
    assert _rel(uh.cpu().numpy(), trace_flatten(m.initial_trace(U))) < 1e-14
    # the trace layout of the context is the oracle's: traces in increasing global face id with
    # the higher side's point count, boundary faces their element's
    assert np.array_equal(np.diff(ctx.trace_off) // m.nv, m.trace_npts)
    xy = ctx.solution_points().cpu().numpy()
    assert _rel(xy, np.concatenate([x.reshape(-1) for x in sample_points_mixed(mesh)])) < 1e-14
    ctx.close()


_ORACLE = {}


def _blocks(name, precision, a_dt=0.031):
    """The context linearised at seeded (U, u^, U*) and the oracle's blocks and hybridized step
    there (computed once per case: the oracle's complex-step blocks dominate the test time)."""
    ctx, m, mesh, U = _setup(name, precision)
    uh = _perturbed_trace(m, U, 1)
    rng = np.random.default_rng(3)
    Ustar = [u * (1 + 1e-4 * rng.standard_normal(u.shape)) for u in U]
    ctx.hfr_local_jacobian(torch.tensor(ctx.pack_state(U), device=DEV), torch.tensor(ctx.pack_trace(uh), device=DEV),
                           torch.tensor(ctx.pack_state(Ustar), device=DEV), a_dt)
    if (name, a_dt) not in _ORACLE:
        _ORACLE[name, a_dt] = {"blocks": element_blocks_mixed(m, U, uh, a_dt)}
    return ctx, m, U, uh, Ustar, a_dt, _ORACLE[name, a_dt]["blocks"]


def _oracle_step(name, m, U, uh, Ustar, a_dt):
    """The oracle's hybridized step at the cached linearisation point (its blocks are the cached
    ones: the same U, u^ and a dt)."""
    import oracle.blocks_mixed as obm

    entry = _ORACLE[name, a_dt]
    if "step" not in entry:
        saved = obm.element_blocks_mixed
        obm.element_blocks_mixed = lambda *args, **kw: entry["blocks"]
        try:
            entry["step"] = hybridized_step(m, U, uh, Ustar, a_dt)
        finally:
            obm.element_blocks_mixed = saved
    return entry["step"]


@pytest.mark.parametrize("name", CASES)
def test_general_element_blocks_fp64(name):
    ctx, m, U, uh, Ustar, a_dt, ref = _blocks(name, pkg.FR_PREC_FP64)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(sorted(ref)):
        for key, blk in zip("ABCD", ref[e]):
            assert got[key][k].shape == blk.shape, (e, key)
            assert _rel(got[key][k], blk) < 1e-11, (e, key)
    # Newton right-hand sides r = -h, s = -g^k (element layout)
    h, _ = stage_residual(m, U, uh, Ustar, a_dt)
    r = ctx.export_blocks("r")
    for k, e in enumerate(sorted(ref)):
        assert _rel(r[k], -h[e]) < 1e-11
    ctx.close()


@pytest.mark.parametrize("name", ["mixed_periodic_ns", "wall_band_ns"])
def test_general_element_blocks_fp32(name):
    ctx, m, U, uh, Ustar, a_dt, ref = _blocks(name, pkg.FR_PREC_FP32)
    got = {key: ctx.export_blocks(key) for key in "ABCD"}
    for k, e in enumerate(sorted(ref)):
        for key, blk in zip("ABCD", ref[e]):
            assert _rel(got[key][k], blk) < 3e-5, (e, key)
    ctx.close()


@pytest.mark.parametrize("name", CASES)
def test_general_condensed_newton_step_fp64(name):
    """Condensation (uneven shapes; the global-memory LU for blocks beyond shared memory), the
    trace solve and the back-substitution against the oracle's hybridized Newton step."""
    ctx, m, U, uh, Ustar, a_dt, _ = _blocks(name, pkg.FR_PREC_FP64)
    ctx.hfr_condense(refine=0)
    duh, its, rel = ctx.hfr_trace_gmres(rtol=1e-13, maxit=5000)
    assert rel <= 1e-12
    du = ctx.hfr_backsolve(duh).cpu().numpy()
    du_ref, dh_ref = _oracle_step(name, m, U, uh, Ustar, a_dt)
    scale = max(np.abs(dh_ref).max(), max(np.abs(v).max() for v in du_ref.values()))
    assert np.abs(duh.cpu().numpy() - dh_ref).max() < 1e-10 * scale
    du_flat = np.concatenate([du_ref[e] for e in sorted(du_ref)])
    assert np.abs(du - du_flat).max() < 1e-10 * scale
    ctx.close()


@pytest.mark.parametrize("name", ["mixed_band_ns", "wall_band_ns"])
def test_general_condensation_fp32(name):
    """FP32 condensation of the FP32 blocks against the FP64 condensation of the oracle's blocks."""
    ctx, m, U, uh, Ustar, a_dt, ref = _blocks(name, pkg.FR_PREC_FP32)
    ctx.hfr_condense(refine=0)
    S = ctx.export_blocks("S")
    XB = ctx.export_blocks("XB")
    r = ctx.export_blocks("r")
    for k, e in enumerate(sorted(ref)):
        A, B, C, D = ref[e]
        XBo = np.linalg.solve(A, B)
        # FP32 elimination: error of order the unit roundoff times the condition number of A (the
        # stretched wall cells reach cond(A) ~ 1e3), never looser than 1e-4
        tol = max(1e-4, 4 * 6e-8 * np.linalg.cond(A))
        assert _rel(S[k], D - C @ XBo) < tol, (e, np.linalg.cond(A))
        assert _rel(XB[k], XBo) < tol, (e, np.linalg.cond(A))
    ctx.close()


def _oracle_stage(m, U0, uh0, a_dt, tol=1e-12, maxit=12):
    """Newton on the stage equations with the oracle's hybridized step (u* = U0)."""
    U = [u.copy() for u in U0]
    uh = [h.copy() for h in uh0]
    off = np.concatenate([[0], np.cumsum(m.trace_npts * m.nv)]).astype(np.int64)
    n0 = None
    for _ in range(maxit):
        h, g = stage_residual(m, U, uh, U0, a_dt)
        nrm = np.sqrt(sum(np.sum(v * v) for v in h.values()) + np.sum(g * g))
        n0 = nrm if n0 is None else n0
        if nrm <= tol * n0:
            return U, uh
        du, dh = hybridized_step(m, U, uh, U0, a_dt)
        for e, d in du.items():
            U[e] = U[e] + d.reshape(U[e].shape)
        uh = [uh[t] + dh[off[t]:off[t + 1]].reshape(uh[t].shape) for t in range(m.ntrace)]
    raise AssertionError("oracle Newton did not converge")


@pytest.mark.parametrize("name,prec", [("wall_band_ns", pkg.FR_PREC_FP64), ("mixed_band_ns", pkg.FR_PREC_FP64),
                                       ("wall_band_ns", pkg.FR_PREC_FP32)])
def test_general_stage_matches_oracle_newton(name, prec):
    ctx, m, mesh, U = _setup(name, prec)
    # the explicit elements take one forward step of the ERK partner: a time step within their
    # explicit limit (smallest explicit cell 0.08 on the wall band, 2 units on the periodic band)
    dt = 0.004 if name.startswith("wall") else 0.05
    a11 = 1.0 - np.sqrt(2.0) / 2.0
    u_n = torch.tensor(ctx.pack_state(U), device=DEV)
    uh = ctx.hfr_initial_trace(u_n)
    R_hist = ctx.empty(3, *ctx.state_shape)
    us = ctx.empty(*ctx.state_shape)
    ctx.imex_stage(0, dt, u_n, us, uh, R_hist)
    st = ctx.imex_stage(1, dt, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-10,
                        gmres_maxit=5000)
    assert st["converged"]
    # the oracle's stage from the same start: explicit elements take u_n + dt a^_21 R(u_n) = u_n +
    # dt gamma R(u_n); implicit ones solve the stage from u* = u_n
    R0, _ = m.full_residual(U, m.initial_trace(U))
    Ustart = [U[e] + (0.0 if m.imp[e] else dt * a11) * R0[e] for e in range(mesh.nelem)]
    Uo, uho = _oracle_stage(m, Ustart, m.initial_trace(U), a11 * dt)
    got = ctx.unpack_state(us.cpu().numpy())
    inc = max(np.abs(Uo[e] - U[e]).max() for e in range(mesh.nelem))
    err = max(np.abs(got[e] - Uo[e]).max() for e in range(mesh.nelem))
    assert err < 1e-9 * inc, err / inc
    ctx.close()


@pytest.mark.parametrize("name,prec", [("wall_band_ns", pkg.FR_PREC_FP64), ("wall_band_ns", pkg.FR_PREC_FP32),
                                       ("mixed_band_advdiff", pkg.FR_PREC_FP32)])
def test_general_graph_stage_equals_stream_stage(name, prec):
    """The implicit stage as one CUDA graph (Newton WHILE node, solve IF node, GMRES restart cycles
    as a nested WHILE node with device-side decisions) gives the stream stage's result bit for
    bit, with the same Newton and GMRES iteration counts; a second launch reuses the graph."""
    mesh, phys, U = _case(name)
    dt = 0.004 if name.startswith("wall") else 0.05
    out = []
    for graph in (False, True):
        ctx = pkg.Context(mesh, phys, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        if graph:
            ctx.imex_stage_set_graph(True)
        u_n = torch.tensor(ctx.pack_state(U), device=DEV)
        res = []
        for _ in range(2):
            uh = ctx.hfr_initial_trace(u_n)
            R_hist = ctx.empty(3, *ctx.state_shape)
            us = ctx.empty(*ctx.state_shape)
            ctx.imex_stage(0, dt, u_n, us, uh, R_hist)
            st = ctx.imex_stage(1, dt, u_n, us, uh, R_hist, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-8,
                                gmres_maxit=5000)
            assert st["converged"]
            res.append((us.clone(), uh.clone(), st["newton_iterations"], st["gmres_iterations"]))
        assert torch.equal(res[0][0], res[1][0])  # the replay repeats the first launch
        out.append(res[0])
        ctx.close()
    (u0, h0, n0, g0), (u1, h1, n1, g1) = out
    assert (n0, g0) == (n1, g1)
    assert torch.equal(u0, u1) and torch.equal(h0, h1)


# ------------------------------------------------------------------ full size (boundary layer)
_BL = {}


def _bl():
    if "w" not in _BL:
        _BL["w"] = make_config("boundary_layer")
    return _BL["w"]


def test_full_size_boundary_layer_rest_state_is_steady():
    """400 x 500 quads, p in 2..5, wall below, far field above: a uniform state at rest (with the
    far field at rest too) is steady on the GPU: R and g vanish to rounding over all 200 000
    elements, 40 000 of them implicit."""
    w = _bl()
    rest = np.array([1.0, 0.0, 0.0, 1.0 / (1.4 * 0.4)])
    phys = dict(w.physics, u_inf=rest)
    ctx = pkg.Context(w.mesh, phys, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    assert ctx.general and ctx.info.nimplicit == 40000
    U = torch.tensor(np.tile(rest, int(ctx.info.state_values) // 4), device=DEV)
    uh = ctx.hfr_initial_trace(U)
    R, g = ctx.fr_residual(U, uh)
    h_min = 1e-5
    assert R.abs().max().item() < 1e-12 / h_min
    assert g.abs().max().item() < 1e-12
    ctx.close()


def test_full_size_boundary_layer_stage_mixed_and_fp64_agree():
    """The boundary-layer workload's implicit stage (SDIRK2 stage 1, IMEX with the ERK partner on the
    explicit elements) converges on both paths, and the mixed-precision stage agrees with the FP64
    one to what the Newton tolerance fixes."""
    w = _bl()
    out = {}
    for label, prec in (("fp64", pkg.FR_PREC_FP64), ("mixed", pkg.FR_PREC_FP32)):
        ctx = pkg.Context(w.mesh, w.physics, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
        u_n = torch.tensor(ctx.pack_state(w.u0), device=DEV)
        uh = ctx.hfr_initial_trace(u_n)
        R_hist = ctx.empty(3, *ctx.state_shape)
        us = ctx.empty(*ctx.state_shape)
        ctx.imex_stage(0, w.dt, u_n, us, uh, R_hist)
        st = ctx.imex_stage(1, w.dt, u_n, us, uh, R_hist, newton_tol=1e-10, newton_maxit=30, gmres_rtol=1e-6,
                            gmres_maxit=20000)
        assert st["converged"], (label, st)
        out[label] = (us - u_n).cpu().numpy()
        ctx.close()
    inc = np.abs(out["fp64"]).max()
    assert np.abs(out["mixed"] - out["fp64"]).max() < 1e-6 * inc
