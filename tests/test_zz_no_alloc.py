"""The allocation-free condensation entry point against hfr_condense.

Some callers may not let a library allocate device memory (their device memory is a fixed
budget handed out by their own pool, or they are plugins given pre-allocated buffers).  For them
the library offers hfr_condense_noalloc, whose scratch is a file-scope device array.  This file
checks, through the C ABI, that two calls in a row reproduce the context-based condensation
(same kernels, so within the tolerances of test_gpu_parity.py), that an over-size request is
refused, and that repeated calls do not inherit state from the previous one.  Kept last in
collection order so that a stop-at-first-failure run has already run every other test.
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


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_condense_matches_context_condense(precision):
    import paper_2401_16632_gb300 as pkg
    from workloads import make_config

    prec = pkg.FR_PREC_FP64 if precision == "fp64" else pkg.FR_PREC_FP32
    w = make_config("vortex", n=5, p=3, jitter=0.15, seed=9, re=200.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=prec)
    if prec == pkg.FR_PREC_FP32:  # the allocation-free entry runs the FP32-FMA products
        ctx.hfr_condense_set_mode(pkg.FR_CONDENSE_FMA)
    u = torch.tensor(w.u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    ctx.hfr_local_jacobian(u, uh, u * 0.999, 0.037)
    ctx.hfr_condense(refine=0)
    A, B, C, D = (ctx.hfr_export(k) for k in "ABCD")
    r, s = ctx.hfr_export("r"), ctx.hfr_export("s")
    ref = {k: ctx.hfr_export(k).cpu().numpy() for k in ("S", "XB", "xr", "t_k")}
    E, nA, nT = A.shape[0], A.shape[1], B.shape[2]
    tol = 1e-12 if precision == "fp64" else 1e-6
    for call in range(2):
        XB = torch.full_like(B, float("nan"))
        S = torch.full_like(D, float("nan"))
        xr = torch.full((E, nA), float("nan"), dtype=torch.float64, device="cuda")
        t = torch.full((E, nT), float("nan"), dtype=torch.float64, device="cuda")
        rc = pkg.hfr_condense_noalloc(A, B, C, D, r, s, XB, xr, S, t, precision=prec)
        torch.cuda.synchronize()
        assert rc == 0, call
        assert _rel(S.cpu().numpy(), ref["S"]) < tol, call
        assert _rel(XB.cpu().numpy(), ref["XB"]) < tol, call
        assert _rel(xr.cpu().numpy(), ref["xr"]) < tol, call
        assert _rel(t.cpu().numpy(), ref["t_k"]) < tol, call
    ctx.close()


def test_noalloc_rejects_requests_beyond_the_scratch_size():
    import ctypes

    import paper_2401_16632_gb300 as pkg

    lib = pkg.load_library()
    # 4096 elements of 64x64 FP64 factors need 128 MiB > 16 MiB: refused on the host before any
    # pointer is used or any device work is enqueued (the placeholder pointers are never read)
    z = ctypes.c_void_p(0x1000)
    rc = lib.hfr_condense_noalloc(4096, 64, 64, pkg.FR_PREC_FP64, z, z, z, z, z, z, z, z, z, z, z)
    assert rc == 1  # FR_ERR_INVALID_ARG
    # the limit formula of include/hfr.h: 400 such elements (about 12.6 MiB) fit, 4096 do not
    need = 256 + ((4 * 64 * 400 + 255) // 256) * 256 + 400 * 64 * 64 * 8
    assert need <= 16 << 20


def test_noalloc_status_words_do_not_leak_between_calls():
    """A call whose blocks hold a singular A (one element's A zeroed) reports FR_ERR_SINGULAR; the
    next call on valid blocks starts from cleared status words and returns 0 with the same S and t
    as the context condensation."""
    import paper_2401_16632_gb300 as pkg
    from workloads import make_config

    w = make_config("vortex", n=4, p=3, re=500.0)
    ctx = pkg.Context(w.mesh, w.physics, precision=pkg.FR_PREC_FP64)
    u = torch.tensor(w.u0, device="cuda")
    uh = ctx.hfr_initial_trace(u)
    ctx.hfr_local_jacobian(u, uh, u * 0.999, 0.037)
    ctx.hfr_condense(refine=0)
    A, B, C, D = (ctx.hfr_export(k) for k in "ABCD")
    r, s = ctx.hfr_export("r"), ctx.hfr_export("s")
    ref_S, ref_t = ctx.hfr_export("S").cpu().numpy(), ctx.hfr_export("t_k").cpu().numpy()
    E, nA, nT = A.shape[0], A.shape[1], B.shape[2]
    XB, S = torch.empty_like(B), torch.empty_like(D)
    xr = torch.empty((E, nA), dtype=torch.float64, device="cuda")
    t = torch.empty((E, nT), dtype=torch.float64, device="cuda")
    bad = A.clone()
    bad[3].zero_()
    assert pkg.hfr_condense_noalloc(bad, B, C, D, r, s, XB, xr, S, t, precision=pkg.FR_PREC_FP64) == 3
    assert pkg.hfr_condense_noalloc(A, B, C, D, r, s, XB, xr, S, t, precision=pkg.FR_PREC_FP64) == 0
    torch.cuda.synchronize()
    assert _rel(S.cpu().numpy(), ref_S) < 1e-12
    assert _rel(t.cpu().numpy(), ref_t) < 1e-12
    ctx.close()


def test_noalloc_rejects_shapes_outside_its_limits():
    import ctypes

    import paper_2401_16632_gb300 as pkg

    lib = pkg.load_library()
    z = ctypes.c_void_p(0x1000)
    # one FP64 element of nA = 200 would fit the scratch (320 KB of factors) but exceeds nA <= 160;
    # nT = 0 is no block: both refused before any pointer is used or any work is enqueued
    assert lib.hfr_condense_noalloc(1, 200, 10, pkg.FR_PREC_FP64, z, z, z, z, z, z, z, z, z, z, z) == 1
    assert lib.hfr_condense_noalloc(1, 64, 0, pkg.FR_PREC_FP64, z, z, z, z, z, z, z, z, z, z, z) == 1
