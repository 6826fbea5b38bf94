"""The library's EFR trace-node layout (host code, no device) against the oracle's numbering,
bit-exact: all-implicit periodic meshes, implicit bands, random implicit masks (ragged skeletons,
vertices shared by one, two or four trace faces), isolated implicit elements, and the error
codes for bad connectivity and boundary faces."""

import os
import shutil

import numpy as np
import pytest

from oracle.efr import EmbeddedDiscretisation
from oracle.physics import AdvectionDiffusion
from workloads.mesh import structured_quads, uniform_nodes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2401_16632_gb300.build import build

    build()
    import paper_2401_16632_gb300 as pkg

    return pkg


def _mesh(nx, ny, p, implicit):
    return structured_quads(uniform_nodes(nx, 0, 1), uniform_nodes(ny, 0, 1), p=p, implicit=implicit)


def _cases():
    rng = np.random.default_rng(11)
    yield _mesh(4, 4, 1, None)
    yield _mesh(5, 3, 3, None)
    band = np.zeros((6, 5), bool)
    band[2:4] = True
    yield _mesh(5, 6, 2, band.reshape(-1))
    for k in range(6):
        nx, ny = int(rng.integers(3, 8)), int(rng.integers(3, 8))
        yield _mesh(nx, ny, int(rng.integers(1, 6)), rng.random(nx * ny) < 0.3 + 0.1 * k)
    yield _mesh(4, 4, 2, np.arange(16) == 5)  # one isolated implicit element: no trace


def test_library_layout_equals_the_oracle(pkg):
    ad = AdvectionDiffusion((1.0, 0.5), 0.01)
    seen_shared = set()
    for mesh in _cases():
        d = EmbeddedDiscretisation(mesh, ad)
        node_of, nvert, nnode = pkg.efr_trace_nodes(mesh.nbr, mesh.nbr_face, mesh.face_of, mesh.implicit,
                                                    int(mesh.p[0]))
        assert nvert == d.nvert and nnode == d.nnode
        assert np.array_equal(node_of, d.node_of)
        counts = np.bincount(node_of[node_of >= 0].ravel(), minlength=max(nnode, 1))
        seen_shared.update(np.unique(counts[:nvert]).tolist())
    # vertex nodes met by 1, 2 and 4 trace faces (two copies each; on a structured quad mesh the
    # implicit elements around a vertex never give exactly three trace faces)
    assert {2, 4, 8} <= seen_shared


def test_layout_errors(pkg):
    mesh = _mesh(3, 3, 2, None)
    with pytest.raises(pkg.HfrError, match="invalid"):
        pkg.efr_trace_nodes(mesh.nbr, mesh.nbr_face, mesh.face_of, mesh.implicit, 0)
    bad = mesh.nbr.copy()
    bad[0, 1] = 2  # element 1 no longer points back
    with pytest.raises(pkg.HfrError, match="invalid"):
        pkg.efr_trace_nodes(bad, mesh.nbr_face, mesh.face_of, mesh.implicit, 2)
    walls = structured_quads(uniform_nodes(3, 0, 1), uniform_nodes(3, 0, 1), periodic=(True, False), p=2)
    with pytest.raises(pkg.HfrError, match="unsupported|not"):  # boundary faces need their tags
        pkg.efr_trace_nodes(walls.nbr, walls.nbr_face, walls.face_of, walls.implicit, 2)
    bad = walls.bc.copy()
    bad[walls.nbr < 0] = 0
    with pytest.raises(pkg.HfrError, match="invalid"):
        pkg.efr_trace_nodes(walls.nbr, walls.nbr_face, walls.face_of, walls.implicit, 2, bc=bad)


def test_layout_with_wall_and_far_field_faces_equals_the_oracle(pkg):
    """Boundary faces of implicit elements carry discontinuous traces at their Gauss points,
    numbered after the interior nodes as the oracle numbers them (walls below, far field above,
    implicit wall rows and random masks)."""
    from oracle.physics import NavierStokes2D
    from workloads.mesh import BC_FARFIELD, BC_WALL

    rng = np.random.default_rng(8)
    u_inf = np.array([1.0, 0.2, 0.0, 2.5])
    for k in range(5):
        nx, ny = int(rng.integers(3, 7)), int(rng.integers(3, 7))
        imp = rng.random(nx * ny) < 0.5 + 0.1 * k
        imp[:nx] = True  # walls on implicit elements
        m = structured_quads(uniform_nodes(nx, 0, 1), uniform_nodes(ny, 0, 1), periodic=(True, False),
                             p=int(rng.integers(1, 6)), implicit=imp, bc_y=(BC_WALL, BC_FARFIELD))
        d = EmbeddedDiscretisation(m, NavierStokes2D(mu=1e-2), u_inf)
        node_of, nvert, nnode = pkg.efr_trace_nodes(m.nbr, m.nbr_face, m.face_of, m.implicit, int(m.p[0]),
                                                    bc=m.bc)
        assert nvert == d.nvert and nnode == d.nnode
        assert np.array_equal(node_of, d.node_of)


def test_mixed_degree_layout_equals_the_oracle(pkg):
    """Face point counts, trace numbering and trace offsets of mixed-degree meshes (periodic, and
    the stretched wall band with wall and far-field faces) against the mixed-degree oracle."""
    from oracle.fr_mixed import MixedDiscretisation
    from oracle.physics import NavierStokes2D
    from workloads.mesh import BC_FARFIELD, BC_WALL

    rng = np.random.default_rng(5)
    u_inf = np.array([1.0, 0.2, 0.0, 2.5])
    meshes = []
    for k in range(5):
        nx, ny = int(rng.integers(3, 7)), int(rng.integers(3, 7))
        periodic = (True, bool(k % 2))
        m = structured_quads(uniform_nodes(nx, 0, 1), uniform_nodes(ny, 0, 1), periodic=periodic, p=2,
                             implicit=rng.random(nx * ny) < 0.6, bc_y=(BC_WALL, BC_FARFIELD))
        m.p = rng.integers(1, 6, size=nx * ny).astype(np.int32)
        m.implicit[:nx] = True  # the wall row is implicit (walls on implicit elements only)
        meshes.append(m)
    for m in meshes:
        d = MixedDiscretisation(m, NavierStokes2D(mu=1e-2), u_inf)
        face_pts, trace_of, trace_off = pkg.mixed_trace_layout(m.nbr, m.nbr_face, m.face_of, m.bc, m.implicit, m.p)
        assert np.array_equal(face_pts, d.nf) and np.array_equal(trace_of, d.tr_of)
        assert np.array_equal(trace_off, np.concatenate([[0], np.cumsum(d.trace_npts)]))
    m = meshes[0]  # walls below, far field above
    assert np.any(m.nbr < 0)
    bad = m.bc.copy()
    bad[m.nbr < 0] = 0  # a boundary face with no boundary kind
    with pytest.raises(pkg.HfrError, match="invalid"):
        pkg.mixed_trace_layout(m.nbr, m.nbr_face, m.face_of, bad, m.implicit, m.p)
    with pytest.raises(pkg.HfrError, match="invalid"):
        pkg.mixed_trace_layout(m.nbr, m.nbr_face, m.face_of, m.bc, m.implicit, np.full(m.nelem, 6))
