"""Condensation of elements of uneven block shapes in one persistent launch (hfr_condense_uneven)
against the oracle's condensation element by element: the shapes of every physics and degree
the library supports (advection-diffusion p = 2, 3; EDAC p = 2-4; Navier-Stokes p = 2-5) mixed
in one seeded batch, FP64 and FP32, plus the refused shapes and a singular element."""

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
from oracle.solve import condense  # noqa: E402

SHAPES = [(9, 12), (16, 16), (27, 36), (48, 48), (75, 60), (36, 48), (64, 64), (100, 80), (144, 96)]


def _batch(shapes, seed):
    rng = np.random.default_rng(seed)
    blocks = []
    for nA, nT in shapes:
        A = 4.0 * np.eye(nA) + rng.standard_normal((nA, nA)) / np.sqrt(nA)
        blocks.append((A, rng.standard_normal((nA, nT)), rng.standard_normal((nT, nA)),
                       rng.standard_normal((nT, nT)), rng.standard_normal(nA), rng.standard_normal(nT)))
    return blocks


def _packed(blocks, dtype):
    cat = lambda i: torch.tensor(np.concatenate([b[i].reshape(-1) for b in blocks]), dtype=dtype, device="cuda")
    vec = lambda i: torch.tensor(np.concatenate([b[i] for b in blocks]), dtype=torch.float64, device="cuda")
    return cat(0), cat(1), cat(2), cat(3), vec(4), vec(5)


def _split(x, sizes):
    out, o = [], 0
    for sz in sizes:
        out.append(x[o:o + sz])
        o += sz
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uneven_batch_matches_oracle(precision):
    rng = np.random.default_rng(7)
    allowed = [sh for sh in SHAPES if precision == "fp32" or sh != (144, 96)]
    shapes = [allowed[i] for i in rng.integers(0, len(allowed), 160)]
    blocks = _batch(shapes, 11)
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    dtype = torch.float64 if precision == "fp64" else torch.float32
    nA = [a for a, _ in shapes]
    nT = [t for _, t in shapes]
    out = pkg.hfr_condense_uneven(nA, nT, *_packed(blocks, dtype), precision=prec)
    XB = _split(out["XB"].cpu().numpy().astype(np.float64), [a * t for a, t in shapes])
    S = _split(out["S"].cpu().numpy().astype(np.float64), [t * t for t in nT])
    xr = _split(out["xr"].cpu().numpy(), nA)
    tt = _split(out["t"].cpu().numpy(), nT)
    tol = 1e-11 if precision == "fp64" else 1e-4
    for k, (b, (a, t)) in enumerate(zip(blocks, shapes)):
        XBo, xro, So, to = condense(*(x[None] for x in b))
        rel = lambda g, r: np.abs(g - r.reshape(-1)).max() / np.abs(r).max()
        assert rel(XB[k], XBo[0]) < tol, (k, a, t)
        assert rel(S[k], So[0]) < tol, (k, a, t)
        assert rel(xr[k], xro[0]) < tol, (k, a, t)
        assert rel(tt[k], to[0]) < tol, (k, a, t)


def test_uneven_global_memory_blocks_and_a_singular_element():
    # FP64 (144, 96) exceeds shared memory: the global-memory LU condenses it, and so it does
    # mixed with shared-memory shapes in one call
    shapes = [(144, 96), (36, 48), (144, 96)]
    blocks = _batch(shapes, 1)
    out = pkg.hfr_condense_uneven([a for a, _ in shapes], [t for _, t in shapes], *_packed(blocks, torch.float64),
                                  precision=pkg.FR_PREC_FP64)
    S = _split(out["S"].cpu().numpy(), [t * t for _, t in shapes])
    xr = _split(out["xr"].cpu().numpy(), [a for a, _ in shapes])
    for k, b in enumerate(blocks):
        XBo, xro, So, to = condense(*(x[None] for x in b))
        assert np.abs(S[k] - So[0].reshape(-1)).max() < 1e-11 * np.abs(So).max(), k
        assert np.abs(xr[k] - xro[0]).max() < 1e-11 * np.abs(xro).max(), k
    with pytest.raises(pkg.HfrError) as ei:  # an empty trace block is refused
        pkg.hfr_condense_uneven([36], [0], *_packed(_batch([(36, 48)], 1), torch.float64), precision=pkg.FR_PREC_FP64)
    assert ei.value.code == pkg.FR_ERR_INVALID_ARG
    shapes = [(36, 48), (64, 64), (36, 48)]
    blocks = _batch(shapes, 2)
    A1 = blocks[1][0].copy()
    A1[:, 5] = 0.0  # a zero column: no pivot in column 5
    blocks[1] = (A1,) + blocks[1][1:]
    with pytest.raises(pkg.HfrError) as ei:
        pkg.hfr_condense_uneven([36, 64, 36], [48, 64, 48], *_packed(blocks, torch.float32), precision=pkg.FR_PREC_FP32)
    assert ei.value.code == pkg.FR_ERR_SINGULAR and ei.value.failed_element == 1


def test_uneven_fp32_large_blocks_take_the_blocked_lu_and_report_a_singular_element():
    """FP32 (144, 96) blocks go to the blocked LU with the tensor-core GEMMs (3xTF32): the same
    condensation as the oracle's to FP32 accuracy, and a zero column found by the panel pivot
    search is reported with its element."""
    shapes = [(144, 96), (36, 48), (144, 96), (144, 96)]
    blocks = _batch(shapes, 5)
    out = pkg.hfr_condense_uneven([a for a, _ in shapes], [t for _, t in shapes], *_packed(blocks, torch.float32),
                                  precision=pkg.FR_PREC_FP32)
    S = _split(out["S"].cpu().numpy().astype(np.float64), [t * t for _, t in shapes])
    XB = _split(out["XB"].cpu().numpy().astype(np.float64), [a * t for a, t in shapes])
    for k, b in enumerate(blocks):
        XBo, xro, So, to = condense(*(x[None] for x in b))
        assert np.abs(S[k] - So[0].reshape(-1)).max() < 1e-5 * np.abs(So).max(), k
        assert np.abs(XB[k] - XBo[0].reshape(-1)).max() < 1e-5 * np.abs(XBo).max(), k
    A2 = blocks[2][0].copy()
    A2[:, 100] = 0.0  # no pivot in column 100 (the fourth panel)
    blocks[2] = (A2,) + blocks[2][1:]
    with pytest.raises(pkg.HfrError) as ei:
        pkg.hfr_condense_uneven([a for a, _ in shapes], [t for _, t in shapes], *_packed(blocks, torch.float32),
                                precision=pkg.FR_PREC_FP32)
    assert ei.value.code == pkg.FR_ERR_SINGULAR and ei.value.failed_element == 2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uneven_batch_of_quadrilateral_and_hexahedral_shapes(precision):
    """Element types mixed in one call: hexahedral Navier-Stokes blocks (p = 2: 135 / 270; p = 3:
    320 / 480) beside quadrilateral ones, each condensed by the form its shape takes (shared-memory
    bundles, blocked LU with the column-block solve), against the oracle's condensation."""
    shapes = [(320, 480), (36, 48), (135, 270), (100, 80), (320, 480), (64, 64)]
    blocks = _batch(shapes, 9)
    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    dtype = torch.float64 if precision == "fp64" else torch.float32
    out = pkg.hfr_condense_uneven([a for a, _ in shapes], [t for _, t in shapes], *_packed(blocks, dtype), precision=prec)
    S = _split(out["S"].cpu().numpy().astype(np.float64), [t * t for _, t in shapes])
    XB = _split(out["XB"].cpu().numpy().astype(np.float64), [a * t for a, t in shapes])
    xr = _split(out["xr"].cpu().numpy(), [a for a, _ in shapes])
    tol = 1e-11 if precision == "fp64" else 2e-5
    for k, b in enumerate(blocks):
        XBo, xro, So, to = condense(*(x[None] for x in b))
        assert np.abs(S[k] - So[0].reshape(-1)).max() < tol * np.abs(So).max(), (k, shapes[k])
        assert np.abs(XB[k] - XBo[0].reshape(-1)).max() < tol * np.abs(XBo).max(), (k, shapes[k])
        assert np.abs(xr[k] - xro[0]).max() < tol * np.abs(xro).max(), (k, shapes[k])
