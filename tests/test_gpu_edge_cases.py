"""Edge cases of the CUDA path against the oracle: meshes with no implicit element (the stage is
the explicit FR update alone), a single implicit element (no trace: the local solve is the whole
Newton step), random implicit masks on non-square meshes (ragged element and trace counts, IMEX
faces on every side, isolated implicit elements), and the bounded grid barrier's timeout path,
checked without faulting the GPU: one CTA of a cooperative launch never arrives, the others'
wait runs out, the call reports FR_ERR_TIMEOUT and the CUDA context stays usable.
"""

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
from oracle.stepping import imex_step  # noqa: E402
from workloads.mesh import structured_quads, uniform_nodes  # noqa: E402
from workloads.states import isentropic_vortex, sample_points, uniform_noise  # noqa: E402

DEV = "cuda"
NS = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _case(name):
    if name == "all_explicit":
        nx, ny, p, mask = 5, 4, 2, np.zeros(20, bool)
    elif name == "single_implicit":
        nx, ny, p = 5, 5, 3
        mask = np.zeros(25, bool)
        mask[12] = True
    elif name == "random_mask_7x5_p2":
        nx, ny, p = 7, 5, 2
        mask = np.random.default_rng(3).random(35) < 0.45
    elif name == "random_mask_6x4_p3":
        nx, ny, p = 6, 4, 3
        mask = np.random.default_rng(8).random(24) < 0.6
    elif name == "random_mask_3x5_p4":
        nx, ny, p = 3, 5, 4
        mask = np.random.default_rng(5).random(15) < 0.7
    else:
        raise KeyError(name)
    mesh = structured_quads(uniform_nodes(nx, 0.0, 10.0), uniform_nodes(ny, 0.0, 10.0), jitter=0.1, seed=2, p=p,
                            implicit=mask)
    # a weaker vortex than the bench's: these meshes are coarse, and the face values of the
    # strength-5 vortex interpolated from a few points per 2.5-unit element have negative pressure
    u0 = isentropic_vortex(sample_points(mesh, p), strength=2.0, center=(5.0, 5.0))
    u0 = u0 + uniform_noise(u0.shape, 1e-3, 11)
    return mesh, u0


CASES = ["all_explicit", "single_implicit", "random_mask_7x5_p2", "random_mask_6x4_p3", "random_mask_3x5_p4"]


@pytest.mark.parametrize("name", CASES)
def test_residual_on_edge_meshes(name):
    mesh, u0 = _case(name)
    d = Discretisation(mesh, make_physics(NS))
    ctx = pkg.Context(mesh, NS, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    assert ctx.info.nimplicit == int(mesh.implicit.sum())
    assert ctx.info.ntrace == d.ntrace
    uh = d.initial_trace(u0)
    uh_dev = torch.tensor(uh, device=DEV) if d.ntrace else None
    R, g = ctx.fr_residual(torch.tensor(u0, device=DEV), uh_dev)
    Ro, go = d.full_residual(u0, uh)
    assert _rel(R.cpu().numpy(), Ro) < 1e-11
    if d.ntrace:
        assert _rel(g.cpu().numpy(), go) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["single_implicit", "random_mask_7x5_p2", "random_mask_3x5_p4"])
def test_blocks_on_edge_meshes(name, precision):
    mesh, u0 = _case(name)
    d = Discretisation(mesh, make_physics(NS))
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    ctx = pkg.Context(mesh, NS, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
    uh = d.initial_trace(u0)
    a_dt = 0.05
    uh_dev = torch.tensor(uh, device=DEV) if d.ntrace else None
    ctx.hfr_local_jacobian(torch.tensor(u0, device=DEV), uh_dev, torch.tensor(u0, device=DEV), a_dt)
    A, B, C, D = element_blocks(d, u0, uh, a_dt)
    imp = d.imp_idx
    tol = 1e-11 if precision == "fp64" else 3e-5
    for key, ref in zip("ABCD", (A[imp], B[imp], C[imp], D[imp])):
        got = ctx.hfr_export(key).cpu().numpy().astype(np.float64)
        scale = max(np.abs(ref).max(), np.abs(A[imp]).max() * 1e-6)  # all-zero C, D when no trace
        assert np.abs(got - ref).max() <= tol * scale, key


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_imex_step_on_edge_meshes(name, precision):
    mesh, u0 = _case(name)
    d = Discretisation(mesh, make_physics(NS))
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    ctx = pkg.Context(mesh, NS, precision=prec, tableau=pkg.FR_TAB_SDIRK2)
    dt = 0.02
    U_o, _, _ = imex_step(d, u0, d.initial_trace(u0), dt, "sdirk2", tol=1e-12)
    u = torch.tensor(u0, device=DEV)
    uh = ctx.hfr_initial_trace(u)
    u1, stats = ctx.imex_step(dt, u, uh, newton_tol=1e-12, gmres_rtol=1e-13 if precision == "fp64" else 1e-6,
                              gmres_maxit=3000)
    inc = np.abs(U_o - u0).max()
    assert np.abs(u1.cpu().numpy() - U_o).max() < (1e-10 if precision == "fp64" else 1e-9) * inc


def test_barrier_timeout_is_reported_and_context_survives():
    # every CTA arrives: all barriers pass
    rc, passed = pkg.fr_barrier_selftest(64, -1, rounds=16, timeout_s=0.5)
    assert rc == pkg.FR_OK and passed == 64 * 16
    # CTA 5 never arrives: the wait of the other 63 runs out after 50 ms and is reported
    rc, passed = pkg.fr_barrier_selftest(64, 5, rounds=4, timeout_s=0.05)
    assert rc == pkg.FR_ERR_TIMEOUT and passed == 0
    # more CTAs than one cooperative launch can hold: rejected on the host
    rc, _ = pkg.fr_barrier_selftest(1 << 20, -1, rounds=1, timeout_s=0.05)
    assert rc == pkg.FR_ERR_INVALID_ARG
    torch.cuda.synchronize()
    # the context is still usable: a stage through the single-launch GMRES cycle
    mesh, u0 = _case("random_mask_6x4_p3")
    d = Discretisation(mesh, make_physics(NS))
    ctx = pkg.Context(mesh, NS, precision=pkg.FR_PREC_FP64, tableau=pkg.FR_TAB_SDIRK2)
    U_o, _, _ = imex_step(d, u0, d.initial_trace(u0), 0.02, "sdirk2", tol=1e-12)
    u = torch.tensor(u0, device=DEV)
    u1, _ = ctx.imex_step(0.02, u, ctx.hfr_initial_trace(u), newton_tol=1e-12, gmres_rtol=1e-13, gmres_maxit=3000)
    assert np.abs(u1.cpu().numpy() - U_o).max() < 1e-10 * np.abs(U_o - u0).max()
