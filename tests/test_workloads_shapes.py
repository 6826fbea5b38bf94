"""The synthetic inputs of the boundary-layer and 3D channel workloads have the stated shapes:
counts, wall-normal growth and aspect ratio, implicit fraction chosen by the stiffness indicator
E_s = |Omega| / |dOmega| (Sec. 5), degree mix, wall and far-field tags, no-slip initial velocity."""

import numpy as np

from workloads import make_config
from workloads.configs import stiffness_indicator
from workloads.mesh import BC_FARFIELD, BC_WALL


def test_stiffness_indicator_closed_forms():
    square = np.array([[[0, 0], [2, 0], [0, 2], [2, 2]]], float)  # area 4, perimeter 8
    thin = np.array([[[0, 0], [1, 0], [0, 1e-3], [1, 1e-3]]], float)
    assert np.allclose(stiffness_indicator(square), [0.5])
    assert np.allclose(stiffness_indicator(thin), [1e-3 / 2.002])


def test_boundary_layer_workload_shape():
    w = make_config("boundary_layer")
    m = w.mesh
    assert m.nelem == 200_000 and m.nx == 400 and m.ny == 500
    rows = m.verts[::400, :, 1]
    h = rows[:, 2] - rows[:, 0]
    assert abs(h[0] - 1e-5) < 1e-15 and np.all(np.diff(h) >= -1e-12) and abs(h.max() - 1e-2) < 1e-12
    assert 45 <= np.sum(h < 1e-2 - 1e-12) <= 55 and abs((1e-2 / h).max() - 1e3) < 1e-6
    assert m.implicit.mean() == 0.2
    imp_rows = np.unique(np.nonzero(m.implicit)[0] // 400)
    assert np.array_equal(imp_rows, np.arange(100))  # the stiffest (thinnest) rows, then towards the wall
    es = stiffness_indicator(m.verts)
    assert es[m.implicit].max() <= es[~m.implicit].min() * (1 + 1e-9)
    assert set(np.unique(m.p)) == {2, 3, 4, 5}
    assert np.all(m.bc[:400, 2] == BC_WALL) and np.all(m.bc[-400:, 3] == BC_FARFIELD)
    assert abs(w.dofs_implicit - 3.4e6) < 0.1e6
    assert len(w.u0) == m.nelem and w.u0[0].shape == ((m.p[0] + 1) ** 2, 4)


def test_channel3d_workload_shape():
    w = make_config("channel3d")
    m = w.mesh
    assert m.nelem == 64 * 32 * 48 and m.implicit.sum() == 18432
    assert w.u0.shape == (m.nelem, 64, 5) and w.dofs_implicit == 18432 * 64 * 5
    assert np.sum(m.bc == BC_WALL) == 2 * 64 * 48
    y = m.verts[:, :, 1]
    assert abs(y.min() + 1) < 1e-14 and abs(y.max() - 1) < 1e-14
    # velocity is M-scaled and vanishes towards the walls; density and pressure uniform
    assert np.abs(w.u0[..., 1:4]).max() <= 0.1 + 1e-12 and np.allclose(w.u0[..., 0], 1.0)
