"""Structured quadrilateral meshes (coordinates + connectivity only).

Conventions shared by every consumer of these meshes:

* element ``e = i + nx * j`` for cell column ``i`` and row ``j``;
* corner ``k = a + 2 b`` of an element sits at reference coordinates
  ``(2a - 1, 2b - 1)``, i.e. corners are listed (-1,-1), (+1,-1), (-1,+1), (+1,+1);
* local faces are 0: xi = -1, 1: xi = +1, 2: eta = -1, 3: eta = +1;
* ``face_of[e, f]`` numbers the faces of the mesh in order of first appearance
  when scanning elements in increasing ``e`` and, inside an element, faces in
  increasing ``f``;
* all elements have the same orientation, so the points of a shared face are
  met in the same order from both sides.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BC_INTERIOR = 0
BC_WALL = 1
BC_FARFIELD = 2


@dataclass
class QuadMesh:
    nx: int
    ny: int
    verts: np.ndarray  # (E, 4, 2) float64 corner coordinates
    nbr: np.ndarray  # (E, 4) int32 neighbour element or -1
    nbr_face: np.ndarray  # (E, 4) int32 neighbour's local face or -1
    bc: np.ndarray  # (E, 4) int32 boundary tag (0 on interior faces)
    face_of: np.ndarray  # (E, 4) int32 global face id
    implicit: np.ndarray  # (E,) bool
    p: np.ndarray  # (E,) int32 polynomial degree
    period: tuple = (0.0, 0.0)  # domain period in x and y (0 = not periodic)
    meta: dict = field(default_factory=dict)

    @property
    def nelem(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nface(self) -> int:
        return int(self.face_of.max()) + 1

    @property
    def dim(self) -> int:
        return 2


def uniform_nodes(n: int, lo: float, hi: float) -> np.ndarray:
    return np.linspace(lo, hi, n + 1)


def geometric_nodes(h0: float, ratio: float, hmax: float, length: float) -> np.ndarray:
    """Nodes starting at 0 with first spacing ``h0`` growing by ``ratio`` until
    the spacing reaches ``hmax``; then uniform spacing ``hmax`` up to ``length``."""
    nodes = [0.0]
    h = h0
    while nodes[-1] < length - 1e-12:
        step = min(h, hmax)
        nodes.append(min(nodes[-1] + step, length))
        h *= ratio
    return np.asarray(nodes)


def tanh_nodes(n: int, beta: float) -> np.ndarray:
    """Nodes on [-1, 1] clustered towards both ends: y_j = tanh(beta (2j/n - 1)) / tanh(beta)."""
    j = np.arange(n + 1)
    return np.tanh(beta * (2.0 * j / n - 1.0)) / np.tanh(beta)


def structured_quads(
    xn: np.ndarray,
    yn: np.ndarray,
    periodic=(True, True),
    jitter: float = 0.0,
    seed: int = 0,
    p=2,
    implicit=None,
    bc_y=(BC_WALL, BC_WALL),
) -> QuadMesh:
    """Tensor-product quad mesh on node lines ``xn`` x ``yn``.

    ``jitter`` > 0 displaces every node that is interior to the (unwrapped)
    node grid by a seeded uniform amount of ``jitter`` times the local spacing,
    which makes the cells general bilinear quadrilaterals while keeping the
    mesh conforming (periodic copies of a node move together).
    ``p`` is an int or an (E,) array; ``implicit`` an (E,) bool array or None
    (all implicit).
    """
    xn = np.asarray(xn, dtype=np.float64)
    yn = np.asarray(yn, dtype=np.float64)
    nx, ny = len(xn) - 1, len(yn) - 1
    X, Y = np.meshgrid(xn, yn, indexing="ij")  # (nx+1, ny+1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx = np.diff(xn).min()
        hy = np.diff(yn).min()
        dx = rng.uniform(-jitter, jitter, size=(nx + 1, ny + 1)) * hx
        dy = rng.uniform(-jitter, jitter, size=(nx + 1, ny + 1)) * hy
        # periodic copies move together; nodes on a non-periodic boundary stay put
        if periodic[0]:
            dx[nx, :] = dx[0, :]
            dy[nx, :] = dy[0, :]
        else:
            dx[[0, nx], :] = 0.0
            dy[[0, nx], :] = 0.0
        if periodic[1]:
            dx[:, ny] = dx[:, 0]
            dy[:, ny] = dy[:, 0]
        else:
            dx[:, [0, ny]] = 0.0
            dy[:, [0, ny]] = 0.0
        X = X + dx
        Y = Y + dy

    E = nx * ny
    verts = np.zeros((E, 4, 2))
    nbr = -np.ones((E, 4), dtype=np.int32)
    nbr_face = -np.ones((E, 4), dtype=np.int32)
    bc = np.zeros((E, 4), dtype=np.int32)
    for j in range(ny):
        for i in range(nx):
            e = i + nx * j
            for b in range(2):
                for a in range(2):
                    verts[e, a + 2 * b, 0] = X[i + a, j + b]
                    verts[e, a + 2 * b, 1] = Y[i + a, j + b]
            # xi faces
            for f, di in ((0, -1), (1, +1)):
                ii = i + di
                if 0 <= ii < nx:
                    nbr[e, f] = ii + nx * j
                elif periodic[0]:
                    nbr[e, f] = (ii % nx) + nx * j
                else:
                    bc[e, f] = BC_FARFIELD
                if nbr[e, f] >= 0:
                    nbr_face[e, f] = 1 - f
            for f, dj in ((2, -1), (3, +1)):
                jj = j + dj
                if 0 <= jj < ny:
                    nbr[e, f] = i + nx * jj
                elif periodic[1]:
                    nbr[e, f] = i + nx * (jj % ny)
                else:
                    bc[e, f] = bc_y[0] if f == 2 else bc_y[1]
                if nbr[e, f] >= 0:
                    nbr_face[e, f] = 5 - f
    face_of = number_faces(nbr, nbr_face)
    pe = np.full(E, p, dtype=np.int32) if np.isscalar(p) else np.asarray(p, dtype=np.int32)
    imp = np.ones(E, dtype=bool) if implicit is None else np.asarray(implicit, dtype=bool)
    period = (
        float(xn[-1] - xn[0]) if periodic[0] else 0.0,
        float(yn[-1] - yn[0]) if periodic[1] else 0.0,
    )
    return QuadMesh(nx, ny, verts, nbr, nbr_face, bc, face_of, imp, pe, period)


def number_faces(nbr: np.ndarray, nbr_face: np.ndarray) -> np.ndarray:
    """Global face ids in order of first appearance over (element, local face)."""
    E, NF = nbr.shape
    face_of = -np.ones((E, NF), dtype=np.int32)
    nxt = 0
    for e in range(E):
        for f in range(NF):
            if face_of[e, f] >= 0:
                continue
            face_of[e, f] = nxt
            if nbr[e, f] >= 0:
                face_of[nbr[e, f], nbr_face[e, f]] = nxt
            nxt += 1
    return face_of


@dataclass
class HexMesh:
    """Structured hexahedral mesh: element e = i + nx (j + ny k); corner a + 2 b + 4 c at reference
    (2a - 1, 2b - 1, 2c - 1); faces 0/1: xi = -1/+1, 2/3: eta = -1/+1, 4/5: zeta = -1/+1; the
    points of a face are numbered along its two tangential axes in increasing axis order (the lower
    axis fastest), the same from both sides."""

    n: tuple
    verts: np.ndarray  # (E, 8, 3)
    nbr: np.ndarray  # (E, 6) neighbour element or -1
    nbr_face: np.ndarray  # (E, 6)
    bc: np.ndarray  # (E, 6) boundary tag
    face_of: np.ndarray  # (E, 6)
    implicit: np.ndarray  # (E,)
    p: np.ndarray  # (E,)
    period: tuple = (0.0, 0.0, 0.0)

    @property
    def nelem(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nface(self) -> int:
        return int(self.face_of.max()) + 1

    @property
    def dim(self) -> int:
        return 3


def structured_hexes(xn, yn, zn, periodic=(True, False, True), jitter: float = 0.0, seed: int = 0,
                     p=3, implicit=None, bc_y=(BC_WALL, BC_WALL)) -> HexMesh:
    """Tensor-product hex mesh on node lines ``xn`` x ``yn`` x ``zn``; ``jitter`` displaces the
    nodes interior to the unwrapped grid as in ``structured_quads`` (periodic copies together)."""
    nodes = [np.asarray(v, dtype=np.float64) for v in (xn, yn, zn)]
    N = [len(v) - 1 for v in nodes]
    X = np.stack(np.meshgrid(*nodes, indexing="ij"), axis=-1)  # (nx+1, ny+1, nz+1, 3)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        h = np.array([np.diff(v).min() for v in nodes])
        dX = rng.uniform(-jitter, jitter, size=X.shape) * h
        for ax in range(3):
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[ax], sl_hi[ax] = 0, N[ax]
            if periodic[ax]:
                dX[tuple(sl_hi)] = dX[tuple(sl_lo)]
            else:
                dX[tuple(sl_lo)] = 0.0
                dX[tuple(sl_hi)] = 0.0
        X = X + dX
    nx, ny, nz = N
    E = nx * ny * nz
    verts = np.zeros((E, 8, 3))
    nbr = -np.ones((E, 6), dtype=np.int32)
    nbr_face = -np.ones((E, 6), dtype=np.int32)
    bc = np.zeros((E, 6), dtype=np.int32)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                for c in range(2):
                    for b in range(2):
                        for a in range(2):
                            verts[e, a + 2 * b + 4 * c] = X[i + a, j + b, k + c]
                ijk = [i, j, k]
                for ax in range(3):
                    for side, step in ((0, -1), (1, 1)):
                        f = 2 * ax + side
                        nn = list(ijk)
                        nn[ax] += step
                        if 0 <= nn[ax] < N[ax] or periodic[ax]:
                            nn[ax] %= N[ax]
                            nbr[e, f] = nn[0] + nx * (nn[1] + ny * nn[2])
                            nbr_face[e, f] = 2 * ax + 1 - side
                        else:
                            bc[e, f] = bc_y[side] if ax == 1 else BC_FARFIELD
    face_of = number_faces(nbr, nbr_face)
    pe = np.full(E, p, dtype=np.int32) if np.isscalar(p) else np.asarray(p, dtype=np.int32)
    imp = np.ones(E, dtype=bool) if implicit is None else np.asarray(implicit, dtype=bool)
    period = tuple(float(v[-1] - v[0]) if per else 0.0 for v, per in zip(nodes, periodic))
    return HexMesh(tuple(N), verts, nbr, nbr_face, bc, face_of, imp, pe, period)
