"""Python binding of the GB300 hybridized IMEX flux-reconstruction stage library.

Argument marshalling only: every numerical step runs in ``libhfr.so`` (CUDA, sm_103a).
PyTorch supplies device memory and the stream.  The names mirror the C ABI in
``include/hfr.h``.  Loading fails loudly when the library has not been built; there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "load_library",
    "Context",
    "HfrError",
    "FR_PREC_FP64",
    "FR_PREC_FP32",
    "FR_TAB_BE",
    "FR_TAB_SDIRK2",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhfr.so")
# the bounds-checked build (FR_CHECKED), built by build(checked=True)
LIB_CHECKED_PATH = os.path.join(HERE, "libhfr_checked.so")

FR_PREC_FP64, FR_PREC_FP32, FR_PREC_TF32, FR_PREC_BF16 = 0, 1, 2, 3
FR_TAB_BE, FR_TAB_SDIRK2 = 0, 1
FR_PHYS_ADVDIFF, FR_PHYS_NAVIER_STOKES, FR_PHYS_EDAC = 0, 1, 2
FR_GMRES_MULTI, FR_GMRES_FUSED = 0, 1
FR_BC_WALL, FR_BC_FARFIELD = 1, 2
FR_TRACE_HFR, FR_TRACE_EFR = 0, 1
FR_ELEM_QUAD, FR_ELEM_HEX = 0, 1
FR_JAC_EVERY_NEWTON, FR_JAC_ONCE_PER_STAGE, FR_JAC_KEEP = 0, 1, 2
FR_CONDENSE_FMA, FR_CONDENSE_TENSOR_PRODUCTS, FR_CONDENSE_TENSOR, FR_CONDENSE_TENSOR_TF32 = 0, 1, 2, 3
(FR_OK, FR_ERR_INVALID_ARG, FR_ERR_CUDA, FR_ERR_SINGULAR, FR_ERR_NOT_CONVERGED, FR_ERR_DIVERGED, FR_ERR_TIMEOUT,
 FR_ERR_OOM, FR_ERR_UNSUPPORTED) = range(9)
EXPORT = {"A": 0, "B": 1, "C": 2, "D": 3, "S": 4, "XB": 5, "xr": 6, "t_k": 7, "r": 8, "s": 9, "t": 10, "Pinv": 11,
          "fnode": 64}

# every symbol declared in include/hfr.h
ABI_SYMBOLS = [
    "efr_trace_nodes",
    "mixed_trace_layout",
    "fr_ctx_create",
    "fr_ctx_destroy",
    "fr_ctx_query",
    "fr_ctx_layout",
    "fr_solution_points",
    "fr_residual",
    "hfr_local_jacobian",
    "hfr_condense",
    "hfr_trace_gmres",
    "imex_set_jacobian_policy",
    "imex_refresh_jacobian",
    "hfr_gmres_set_mode",
    "hfr_gmres_get_mode",
    "hfr_condense_set_mode",
    "hfr_condense_get_mode",
    "fr_modal_filter",
    "hfr_condense_uneven",
    "hfr_autotune",
    "imex_stage_set_graph",
    "imex_stage_get_graph",
    "fr_barrier_selftest",
    "hfr_backsolve",
    "hfr_export",
    "imex_stage",
    "imex_steps",
    "hfr_initial_trace",
    "fr_profile_enable",
    "fr_profile_read",
    "fr_kernel_launches",
    "fr_checked_status",
    "hfr_condense_noalloc",
    "hfr_import",
    "fr_measure_peak",
    "fr_last_error",
    "fr_status_string",
]

PHASES = ["residual", "jacobian", "condense_factor", "trace_rhs_precond", "gmres", "backsolve", "newton",
          "refine_xr", "trace_matvec", "condense_products"]


class fr_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("nelem", ctypes.c_int),
        ("p", ctypes.c_int),
        ("verts", ctypes.POINTER(ctypes.c_double)),
        ("nbr", ctypes.POINTER(ctypes.c_int)),
        ("nbr_face", ctypes.POINTER(ctypes.c_int)),
        ("face_of", ctypes.POINTER(ctypes.c_int)),
        ("implicit", ctypes.POINTER(ctypes.c_ubyte)),
        ("p_elem", ctypes.POINTER(ctypes.c_int)),
        ("bc", ctypes.POINTER(ctypes.c_int)),
        ("elem_type", ctypes.c_int),
    ]


class fr_config(ctypes.Structure):
    _fields_ = [
        ("physics", ctypes.c_int),
        ("beta", ctypes.c_double * 2),
        ("nu", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("lref", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("tableau", ctypes.c_int),
        ("gmres_restart", ctypes.c_int),
        ("theta", ctypes.c_double),
        ("u_inf", ctypes.c_double * 5),
        ("trace_kind", ctypes.c_int),
    ]


class fr_ctx_info(ctypes.Structure):
    _fields_ = [
        ("nelem", ctypes.c_int),
        ("nimplicit", ctypes.c_int),
        ("p", ctypes.c_int),
        ("n", ctypes.c_int),
        ("ns", ctypes.c_int),
        ("nv", ctypes.c_int),
        ("nA", ctypes.c_int),
        ("nT", ctypes.c_int),
        ("ntrace", ctypes.c_int),
        ("nstages", ctypes.c_int),
        ("has_explicit", ctypes.c_int),
        ("workspace_bytes", ctypes.c_size_t),
        ("general", ctypes.c_int),
        ("state_values", ctypes.c_size_t),
        ("trace_values", ctypes.c_size_t),
        ("face_points", ctypes.c_int),
    ]


class fr_stage_stats(ctypes.Structure):
    _fields_ = [
        ("newton_iterations", ctypes.c_int),
        ("gmres_iterations", ctypes.c_int),
        ("residual0", ctypes.c_double),
        ("residual", ctypes.c_double),
        ("converged", ctypes.c_int),
    ]


class fr_steps_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int),
        ("newton_iterations", ctypes.c_int),
        ("gmres_iterations", ctypes.c_int),
        ("jacobian_refreshes", ctypes.c_int),
        ("max_rel_residual", ctypes.c_double),
        ("converged", ctypes.c_int),
    ]


class fr_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 10), ("count", ctypes.c_longlong * 10)]


class fr_tune_report(ctypes.Structure):
    _fields_ = [
        ("condense_mode", ctypes.c_int),
        ("inverse_ctas_per_sm", ctypes.c_int),
        ("gmres_mode", ctypes.c_int),
        ("condense_ms", ctypes.c_double * 3),
        ("inverse_ms", ctypes.c_double * 4),
        ("gmres_ms", ctypes.c_double * 2),
    ]


class fr_error_info(ctypes.Structure):
    _fields_ = [
        ("code", ctypes.c_int),
        ("element", ctypes.c_int),
        ("iteration", ctypes.c_int),
        ("value", ctypes.c_double),
        ("message", ctypes.c_char * 160),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhfr.so (built by ``paper_2401_16632_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2401_16632_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
    lib.fr_ctx_create.argtypes = [ctypes.POINTER(fr_mesh_desc), ctypes.POINTER(fr_config), vp, ctypes.POINTER(vp)]
    lib.fr_ctx_destroy.argtypes = [vp]
    lib.fr_ctx_destroy.restype = None
    lib.fr_ctx_query.argtypes = [vp, ctypes.POINTER(fr_ctx_info)]
    lib.fr_ctx_layout.argtypes = [vp, vp, vp, vp, vp]
    lib.fr_solution_points.argtypes = [vp, dp]
    lib.fr_residual.argtypes = [vp, dp, dp, dp, dp]
    lib.hfr_local_jacobian.argtypes = [vp, dp, dp, dp, ctypes.c_double]
    lib.hfr_condense.argtypes = [vp, ctypes.c_int]
    lib.hfr_trace_gmres.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_double)]
    lib.imex_set_jacobian_policy.argtypes = [vp, ctypes.c_int]
    lib.imex_refresh_jacobian.argtypes = [vp]
    lib.imex_steps.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(fr_steps_stats)]
    lib.hfr_gmres_set_mode.argtypes = [vp, ctypes.c_int]
    lib.hfr_gmres_get_mode.argtypes = [vp]
    lib.hfr_condense_set_mode.argtypes = [vp, ctypes.c_int]
    lib.hfr_condense_get_mode.argtypes = [vp]
    lib.hfr_condense_uneven.argtypes = [ctypes.c_int, ip, ip, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp, ip, dp, dp, dp,
                                        dp, ip, vp, ip]
    lib.fr_modal_filter.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.hfr_autotune.argtypes = [vp, dp, dp, dp, ctypes.c_double, ctypes.POINTER(fr_tune_report)]
    lib.imex_stage_set_graph.argtypes = [vp, ctypes.c_int]
    lib.imex_stage_get_graph.argtypes = [vp]
    lib.fr_barrier_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, vp]
    lib.hfr_backsolve.argtypes = [vp, dp, dp, ctypes.c_int]
    lib.hfr_export.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    lib.imex_stage.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(fr_stage_stats)]
    lib.hfr_initial_trace.argtypes = [vp, dp, dp]
    lib.fr_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.fr_profile_read.argtypes = [vp, ctypes.POINTER(fr_profile)]
    lib.fr_kernel_launches.argtypes = []
    lib.fr_kernel_launches.restype = ctypes.c_ulonglong
    lib.fr_checked_status.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.hfr_condense_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp,
                                         dp, dp, dp, dp, dp, vp]
    lib.hfr_import.argtypes = [vp, ctypes.c_int, dp, ctypes.c_size_t]
    lib.fr_measure_peak.argtypes = [ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
    lib.fr_last_error.argtypes = [vp, ctypes.POINTER(fr_error_info)]
    lib.fr_status_string.argtypes = [ctypes.c_int]
    lib.fr_status_string.restype = ctypes.c_char_p
    lib.efr_trace_nodes.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_int, vp, ip, ip]
    lib.mixed_trace_layout.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, ip]
    _lib = lib
    return lib


class HfrError(RuntimeError):
    def __init__(self, code, info=None):
        self.code = code
        self.info = info
        msg = load_library().fr_status_string(code).decode()
        if info is not None:
            msg += f" ({info.message.decode()}; element {info.element}, iteration {info.iteration}, value {info.value:g})"
        super().__init__(msg)


def efr_trace_nodes(nbr, nbr_face, face_of, implicit, p, bc=None):
    """EFR trace-node layout of a quad mesh (host arrays in, host arrays out): (node_of (E, 4, p+1)
    int32, nvert, nnode).  Raises HfrError on the library's error codes."""
    import numpy as np

    lib = load_library()
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    nbr_face = np.ascontiguousarray(nbr_face, dtype=np.int32)
    face_of = np.ascontiguousarray(face_of, dtype=np.int32)
    imp = np.ascontiguousarray(implicit, dtype=np.uint8)
    E = int(nbr.shape[0])
    for a in (nbr, nbr_face, face_of):
        if a.shape != (E, 4):
            raise ValueError("efr_trace_nodes: connectivity arrays must have shape (E, 4)")
    if imp.shape != (E,):
        raise ValueError("efr_trace_nodes: implicit must have shape (E,)")
    out = np.empty((E, 4, max(int(p), 0) + 1), dtype=np.int32)
    nvert, nnode = ctypes.c_int(), ctypes.c_int()
    bca = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
    if bca is not None and bca.shape != (E, 4):
        raise ValueError("efr_trace_nodes: bc must have shape (E, 4)")
    rc = lib.efr_trace_nodes(E, nbr.ctypes.data, nbr_face.ctypes.data, face_of.ctypes.data,
                             None if bca is None else bca.ctypes.data, imp.ctypes.data, int(p), out.ctypes.data,
                             ctypes.byref(nvert), ctypes.byref(nnode))
    if rc != 0:
        raise HfrError(rc)
    return out, nvert.value, nnode.value


def mixed_trace_layout(nbr, nbr_face, face_of, bc, implicit, p):
    """Trace layout of a mixed-degree quad mesh (host arrays): (face_pts (E, 4), trace_of (E, 4),
    trace_off (ntrace + 1,)), all int32.  Raises HfrError on the library's error codes."""
    import numpy as np

    lib = load_library()
    a = [np.ascontiguousarray(x, dtype=np.int32) for x in (nbr, nbr_face, face_of, bc)]
    imp = np.ascontiguousarray(implicit, dtype=np.uint8)
    deg = np.ascontiguousarray(p, dtype=np.int32)
    E = int(a[0].shape[0])
    if any(x.shape != (E, 4) for x in a):
        raise ValueError("mixed_trace_layout: nbr, nbr_face, face_of and bc must have shape (E, 4)")
    if imp.shape != (E,) or deg.shape != (E,):
        raise ValueError("mixed_trace_layout: implicit and p must have shape (E,)")
    face_pts = np.empty((E, 4), dtype=np.int32)
    trace_of = np.empty((E, 4), dtype=np.int32)
    trace_off = np.empty(4 * E + 1, dtype=np.int32)
    ntrace = ctypes.c_int()
    rc = lib.mixed_trace_layout(E, *(x.ctypes.data for x in a), imp.ctypes.data, deg.ctypes.data,
                                face_pts.ctypes.data, trace_of.ctypes.data, trace_off.ctypes.data,
                                ctypes.byref(ntrace))
    if rc != 0:
        raise HfrError(rc)
    return face_pts, trace_of, trace_off[:ntrace.value + 1].copy()


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def hfr_condense_noalloc(A, B, C, D, r, s, XB, xr, S, t, precision=FR_PREC_FP64, stream=None):
    """Allocation-free condensation on caller-provided device tensors (see include/hfr.h):
    shapes (E, nA, nA), (E, nA, nT), (E, nT, nA), (E, nT, nT), (E, nA), (E, nT) in, XB, xr, S, t out.
    Returns the status code (0 = ok)."""
    import torch

    lib = load_library()
    E, nA, nT = int(A.shape[0]), int(A.shape[1]), int(B.shape[2])
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib.hfr_condense_noalloc(E, nA, nT, int(precision), _ptr(A), _ptr(B), _ptr(C), _ptr(D), _ptr(r), _ptr(s),
                                    _ptr(XB), _ptr(xr), _ptr(S), _ptr(t), ctypes.c_void_p(st.cuda_stream))


def hfr_condense_uneven(nA, nT, A, B, C, D, r, s, precision=FR_PREC_FP32, stream=None):
    """Condensation of elements of uneven shapes in one launch (see include/hfr.h).  nA, nT:
    sequences of ints; A, B, C, D: packed 1-D device tensors of the block precision; r, s: packed
    FP64.  Returns the packed outputs {LU, piv, XB, xr, S, t}; raises HfrError on failure."""
    import torch

    lib = load_library()
    n = len(nA)
    na = (ctypes.c_int * n)(*[int(x) for x in nA])
    nt = (ctypes.c_int * n)(*[int(x) for x in nT])
    sa = sum(int(x) * int(x) for x in nA)
    sb = sum(int(x) * int(y) for x, y in zip(nA, nT))
    sd = sum(int(y) * int(y) for y in nT)
    dev, dt = A.device, A.dtype
    out = {"LU": torch.empty(sa, dtype=dt, device=dev), "piv": torch.empty(sum(nA), dtype=torch.int32, device=dev),
           "XB": torch.empty(sb, dtype=dt, device=dev), "xr": torch.empty(sum(nA), dtype=torch.float64, device=dev),
           "S": torch.empty(sd, dtype=dt, device=dev), "t": torch.empty(sum(nT), dtype=torch.float64, device=dev)}
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    failed = ctypes.c_int(-1)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.hfr_condense_uneven(n, na, nt, int(precision), _ptr(A), _ptr(B), _ptr(C), _ptr(D), _ptr(r), _ptr(s),
                                 _ptr(out["LU"]), ctypes.cast(_ptr(out["piv"]), ctypes.POINTER(ctypes.c_int)),
                                 _ptr(out["XB"]), _ptr(out["xr"]), _ptr(out["S"]), _ptr(out["t"]),
                                 ctypes.cast(_ptr(status), ctypes.POINTER(ctypes.c_int)),
                                 ctypes.c_void_p(st.cuda_stream), ctypes.byref(failed))
    if rc != 0:
        err = HfrError(rc)
        err.failed_element = failed.value
        raise err
    return out


def fr_checked_status():
    """Bounds-checked build (see include/hfr.h): (site, index, count) of the index failures the
    device checks recorded since the last call (site 0: none); raises HfrError (FR_ERR_UNSUPPORTED)
    in a build without the checks."""
    lib = load_library()
    first, count = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    rc = lib.fr_checked_status(ctypes.byref(first), ctypes.byref(count))
    if rc != 0:
        raise HfrError(rc)
    return int(first.value >> 48), int(first.value & ((1 << 48) - 1)), int(count.value)


def fr_measure_peak(which, stream=None):
    """Measured dense TFLOP/s of one pipe of the current device (see include/hfr.h): which 0 FP64
    FMA, 1 FP32 FMA, 2 TF32 tensor core.  Raises HfrError on failure."""
    import torch

    lib = load_library()
    out = ctypes.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.fr_measure_peak(int(which), ctypes.c_void_p(st.cuda_stream), ctypes.byref(out))
    if rc != 0:
        raise HfrError(rc)
    return out.value


def fr_barrier_selftest(nblocks, absent_block=-1, rounds=4, timeout_s=0.05, stream=None):
    """Bounded grid-barrier self-test (see include/hfr.h).  Returns (status, barriers passed)."""
    import torch

    lib = load_library()
    passed = ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.fr_barrier_selftest(int(nblocks), int(absent_block), int(rounds), float(timeout_s),
                                 ctypes.byref(passed), ctypes.c_void_p(st.cuda_stream))
    return rc, passed.value


class Context:
    """One fr_ctx on the current CUDA device and stream.

    mesh: object with verts (E,4,2), nbr, nbr_face, face_of (E,4) int arrays, implicit (E,) bool
    and p (E,) int; physics: dict (kind 'advdiff' with beta, nu or 'ns' with gamma, mu, Pr; lref).
    """

    def __init__(self, mesh, physics: dict, precision: int = FR_PREC_FP64, tableau: int = FR_TAB_SDIRK2,
                 gmres_restart: int = 30, stream=None, trace_kind: int = FR_TRACE_HFR):
        import torch

        self.torch = torch
        self.lib = load_library()
        degs = np.asarray(mesh.p).reshape(-1)
        p = int(degs[0])
        E = int(mesh.verts.shape[0])
        self.hex = int(getattr(mesh, "dim", 2)) == 3
        general = (bool(np.any(degs != p)) or bool(np.any(np.asarray(mesh.nbr) < 0)) or self.hex
                   or trace_kind == FR_TRACE_EFR)
        self._deg = np.ascontiguousarray(np.broadcast_to(degs, (E,)), dtype=np.int32)
        bc = getattr(mesh, "bc", None)
        self._bc = np.ascontiguousarray(bc if bc is not None else np.zeros_like(np.asarray(mesh.nbr)), dtype=np.int32)
        self._verts = np.ascontiguousarray(mesh.verts, dtype=np.float64)
        self._nbr = np.ascontiguousarray(mesh.nbr, dtype=np.int32)
        self._nbf = np.ascontiguousarray(mesh.nbr_face, dtype=np.int32)
        self._fid = np.ascontiguousarray(mesh.face_of, dtype=np.int32)
        self._imp = np.ascontiguousarray(mesh.implicit, dtype=np.uint8)
        md = fr_mesh_desc(
            E, p,
            self._verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            self._nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            self._nbf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            self._fid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            self._imp.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
            self._deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if general else None,
            self._bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if general else None,
            FR_ELEM_HEX if self.hex else FR_ELEM_QUAD,
        )
        cfg = fr_config()
        if physics["kind"] == "advdiff":
            cfg.physics = FR_PHYS_ADVDIFF
            cfg.beta[0], cfg.beta[1] = physics["beta"][0], physics["beta"][1]
            cfg.nu = physics["nu"]
        elif physics["kind"] == "edac":
            cfg.physics = FR_PHYS_EDAC
            cfg.theta, cfg.nu = physics["theta"], physics["nu"]
        else:
            cfg.physics = FR_PHYS_NAVIER_STOKES
            cfg.gamma, cfg.mu, cfg.Pr = physics["gamma"], physics["mu"], physics["Pr"]
        cfg.lref = physics.get("lref", 1.0)
        if physics.get("u_inf") is not None:
            ui = np.asarray(physics["u_inf"], dtype=np.float64).reshape(-1)
            for i, x in enumerate(ui[:5]):
                cfg.u_inf[i] = float(x)
        cfg.precision = precision
        cfg.trace_kind = trace_kind
        cfg.tableau = tableau
        cfg.gmres_restart = gmres_restart
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.fr_ctx_create(ctypes.byref(md), ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h))
        if rc != 0:
            raise HfrError(rc)
        self.h = h
        info = fr_ctx_info()
        self.lib.fr_ctx_query(self.h, ctypes.byref(info))
        self.info = info
        self.precision = precision
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.general = bool(info.general)
        if self.general:
            eo = np.zeros(info.nelem + 1, dtype=np.int64)
            to = np.zeros(info.ntrace + 1, dtype=np.int64)
            na = np.zeros(max(info.nimplicit, 1), dtype=np.int32)
            nt = np.zeros(max(info.nimplicit, 1), dtype=np.int32)
            self._check(self.lib.fr_ctx_layout(self.h, eo.ctypes.data, to.ctypes.data, na.ctypes.data, nt.ctypes.data))
            self.elem_off, self.trace_off = eo, to
            self.blk_nA, self.blk_nT = na[:info.nimplicit], nt[:info.nimplicit]

    # ----------------------------------------------------------------------- plumbing
    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            info = fr_error_info()
            self.lib.fr_last_error(self.h, ctypes.byref(info))
            raise HfrError(rc, info)

    def empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.torch.float64, device=self.dev)

    @property
    def trace_shape(self):
        if self.general:
            return (int(self.info.trace_values),)
        return (self.info.ntrace, self.info.n, self.info.nv)

    @property
    def state_shape(self):
        if self.general:
            return (int(self.info.state_values),)
        return (self.info.nelem, self.info.ns, self.info.nv)

    # ------------------------------------------------------- packed layouts (general path)
    def pack_state(self, U):
        """List of per-element (Ns_e, nv) arrays -> the packed state vector (numpy)."""
        return np.concatenate([np.asarray(u, dtype=np.float64).reshape(-1) for u in U])

    def unpack_state(self, x):
        x = np.asarray(x).reshape(-1)
        nv = self.info.nv
        return [x[self.elem_off[e]:self.elem_off[e + 1]].reshape(-1, nv) for e in range(self.info.nelem)]

    def pack_trace(self, H):
        return np.concatenate([np.asarray(h, dtype=np.float64).reshape(-1) for h in H]) if len(H) else np.zeros(0)

    def unpack_trace(self, x):
        x = np.asarray(x).reshape(-1)
        nv = self.info.nv
        return [x[self.trace_off[t]:self.trace_off[t + 1]].reshape(-1, nv) for t in range(self.info.ntrace)]

    def export_blocks(self, which: str):
        """General path: an exported element array split into its implicit elements (numpy list)."""
        flat = self.hfr_export(which).cpu().numpy()
        na, nt = self.blk_nA.astype(np.int64), self.blk_nT.astype(np.int64)
        shapes = {"A": (na, na), "B": (na, nt), "C": (nt, na), "D": (nt, nt), "S": (nt, nt), "XB": (na, nt),
                  "xr": (na, None), "r": (na, None), "t_k": (nt, None), "s": (nt, None)}[which]
        out, o = [], 0
        # hexahedra keep A, B, C, D column-major (S and X_B, written by the condensation, row-major)
        colmajor = self.hex and which in ("A", "B", "C", "D")
        for k in range(self.info.nimplicit):
            r = int(shapes[0][k])
            c = 1 if shapes[1] is None else int(shapes[1][k])
            blk = flat[o:o + r * c]
            if shapes[1] is not None:
                blk = blk.reshape(c, r).T if colmajor else blk.reshape(r, c)
            out.append(blk)
            o += r * c
        return out

    # -------------------------------------------------------------------- ABI calls
    def solution_points(self):
        if self.general:
            xy = self.empty((3 if self.hex else 2) * int(self.info.state_values) // self.info.nv)
        else:
            xy = self.empty(self.info.nelem, self.info.ns, 2)
        self._check(self.lib.fr_solution_points(self.h, _ptr(xy)))
        return xy

    def hfr_initial_trace(self, u):
        uh = self.empty(*self.trace_shape)
        self._check(self.lib.hfr_initial_trace(self.h, _ptr(u), _ptr(uh)))
        return uh

    def fr_residual(self, u, uhat, want_g=True):
        R = self.empty(*self.state_shape)
        g = self.empty(*self.trace_shape) if want_g else None
        self._check(self.lib.fr_residual(self.h, _ptr(u), _ptr(uhat), _ptr(R), _ptr(g)))
        return R, g

    def hfr_local_jacobian(self, u, uhat, ustar, a_dt):
        self._check(self.lib.hfr_local_jacobian(self.h, _ptr(u), _ptr(uhat), _ptr(ustar), float(a_dt)))

    def hfr_condense(self, refine=0):
        self._check(self.lib.hfr_condense(self.h, int(refine)))

    def hfr_trace_gmres(self, rtol=1e-10, maxit=1000, check=True):
        duh = self.empty(*self.trace_shape)
        its = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        rc = self.lib.hfr_trace_gmres(self.h, _ptr(duh), float(rtol), int(maxit), ctypes.byref(its), ctypes.byref(rel))
        if check:
            self._check(rc)
        return duh, its.value, rel.value

    def imex_set_jacobian_policy(self, policy: int):
        self._check(self.lib.imex_set_jacobian_policy(self.h, int(policy)))

    def imex_refresh_jacobian(self):
        self._check(self.lib.imex_refresh_jacobian(self.h))

    def hfr_gmres_set_mode(self, mode: int):
        self._check(self.lib.hfr_gmres_set_mode(self.h, int(mode)))

    def hfr_gmres_get_mode(self) -> int:
        return int(self.lib.hfr_gmres_get_mode(self.h))

    def fr_modal_filter(self, u, alpha, s, eta_c, dt_ratio=1.0, which=0):
        """In place on u (device tensor): the modal filter of Appendix B (see include/hfr.h)."""
        self._check(self.lib.fr_modal_filter(self.h, _ptr(u), float(alpha), float(s), int(eta_c), float(dt_ratio),
                                             int(which)))
        return u

    def hfr_autotune(self, u, uhat, ustar, a_dt):
        rep = fr_tune_report()
        self._check(self.lib.hfr_autotune(self.h, _ptr(u), _ptr(uhat), _ptr(ustar), float(a_dt), ctypes.byref(rep)))
        return {"condense_mode": rep.condense_mode, "inverse_ctas_per_sm": rep.inverse_ctas_per_sm,
                "gmres_mode": rep.gmres_mode, "condense_ms": list(rep.condense_ms),
                "inverse_ms": list(rep.inverse_ms), "gmres_ms": list(rep.gmres_ms)}

    def imex_stage_set_graph(self, on: bool = True):
        self._check(self.lib.imex_stage_set_graph(self.h, 1 if on else 0))

    def imex_stage_get_graph(self) -> int:
        return int(self.lib.imex_stage_get_graph(self.h))

    def hfr_condense_set_mode(self, mode: int):
        self._check(self.lib.hfr_condense_set_mode(self.h, int(mode)))

    def hfr_condense_get_mode(self) -> int:
        return int(self.lib.hfr_condense_get_mode(self.h))

    def hfr_backsolve(self, duhat, refine=0):
        if self.general:
            du = self.empty(int(np.sum(self.blk_nA)))
        else:
            du = self.empty(self.info.nimplicit, self.info.nA)
        self._check(self.lib.hfr_backsolve(self.h, _ptr(duhat), _ptr(du), int(refine)))
        return du

    def hfr_export(self, which: str):
        i = self.info
        if self.general:
            blk = self.torch.float64 if self.precision == FR_PREC_FP64 else self.torch.float32
            na, nt = self.blk_nA.astype(np.int64), self.blk_nT.astype(np.int64)
            sizes = {"A": (int(np.sum(na * na)), blk), "B": (int(np.sum(na * nt)), blk), "C": (int(np.sum(na * nt)), blk),
                     "D": (int(np.sum(nt * nt)), blk), "S": (int(np.sum(nt * nt)), blk), "XB": (int(np.sum(na * nt)), blk),
                     "xr": (int(np.sum(na)), self.torch.float64), "t_k": (int(np.sum(nt)), self.torch.float64),
                     "r": (int(np.sum(na)), self.torch.float64), "s": (int(np.sum(nt)), self.torch.float64),
                     "t": (int(i.trace_values), self.torch.float64)}
            if which == "Pinv":
                tp = np.diff(self.trace_off) // i.nv
                sizes["Pinv"] = (int(np.sum((tp * i.nv) ** 2)), blk)
            sizes["fnode"] = (int(i.face_points), self.torch.int32)
            n, dt = sizes[which]
            out = self.torch.empty(max(n, 1), dtype=dt, device=self.dev)
            self._check(self.lib.hfr_export(self.h, EXPORT[which], _ptr(out), n * out.element_size()))
            return out[:n]
        E, nA, nT = i.nimplicit, i.nA, i.nT
        blk = self.torch.float64 if self.precision == FR_PREC_FP64 else self.torch.float32
        shapes = {"A": (E, nA, nA, blk), "B": (E, nA, nT, blk), "C": (E, nT, nA, blk), "D": (E, nT, nT, blk),
                  "S": (E, nT, nT, blk), "XB": (E, nA, nT, blk), "xr": (E, nA, self.torch.float64),
                  "t_k": (E, nT, self.torch.float64), "r": (E, nA, self.torch.float64),
                  "s": (E, nT, self.torch.float64), "t": (i.ntrace * i.n * i.nv, self.torch.float64),
                  "Pinv": (i.ntrace, i.n * i.nv, i.n * i.nv, blk)}
        *shp, dt = shapes[which]
        out = self.torch.empty(*shp, dtype=dt, device=self.dev)
        self._check(self.lib.hfr_export(self.h, EXPORT[which], _ptr(out), out.numel() * out.element_size()))
        return out

    def hfr_import(self, which: str, src):
        """Overwrite a context array (A, B, C, D, S, XB, xr, t_k, r, s) with a device tensor of
        exactly its size (C entry hfr_import)."""
        self._check(self.lib.hfr_import(self.h, EXPORT[which], _ptr(src), src.numel() * src.element_size()))

    def imex_stage(self, stage, dt, u_n, u_stage, uhat, R_hist, newton_tol=1e-8, newton_maxit=20,
                   gmres_rtol=1e-3, gmres_maxit=500, refine=0):
        st = fr_stage_stats()
        rc = self.lib.imex_stage(self.h, int(stage), float(dt), _ptr(u_n), _ptr(u_stage), _ptr(uhat), _ptr(R_hist),
                                 float(newton_tol), int(newton_maxit), float(gmres_rtol), int(gmres_maxit),
                                 int(refine), ctypes.byref(st))
        self._check(rc)
        return {"newton_iterations": st.newton_iterations, "gmres_iterations": st.gmres_iterations,
                "residual0": st.residual0, "residual": st.residual, "converged": bool(st.converged)}

    def imex_steps(self, nsteps, dt, u, uhat, refresh_every=0, newton_tol=1e-8, newton_maxit=20, gmres_rtol=1e-3,
                   gmres_maxit=500, refine=0):
        """nsteps whole IMEX steps in place on u and uhat (C entry imex_steps); returns the totals."""
        R_hist = self.empty(self.info.nstages + 1, *self.state_shape)
        u_stage = self.empty(*self.state_shape)
        st = fr_steps_stats()
        rc = self.lib.imex_steps(self.h, int(nsteps), float(dt), _ptr(u), _ptr(uhat), _ptr(R_hist), _ptr(u_stage),
                                 int(refresh_every), float(newton_tol), int(newton_maxit), float(gmres_rtol),
                                 int(gmres_maxit), int(refine), ctypes.byref(st))
        self._check(rc)
        return {"steps": st.steps, "newton_iterations": st.newton_iterations, "gmres_iterations": st.gmres_iterations,
                "jacobian_refreshes": st.jacobian_refreshes, "max_rel_residual": st.max_rel_residual,
                "converged": bool(st.converged)}

    def fr_profile_enable(self, on=True):
        self._check(self.lib.fr_profile_enable(self.h, 1 if on else 0))

    def fr_profile_read(self):
        pr = fr_profile()
        self._check(self.lib.fr_profile_read(self.h, ctypes.byref(pr)))
        return {name: (pr.ms[i], pr.count[i]) for i, name in enumerate(PHASES)}

    def kernel_launches(self):
        return int(self.lib.fr_kernel_launches())

    def imex_step(self, dt, u_n, uhat, **kw):
        """All stages of one IMEX step; returns u_{n+1} (uhat updated in place)."""
        s = self.info.nstages
        R_hist = self.empty(s + 1, *self.state_shape)
        u_stage = self.empty(*self.state_shape)
        self.imex_stage(0, dt, u_n, u_stage, uhat, R_hist, **kw)
        stats = []
        for i in range(1, s + 1):
            stats.append(self.imex_stage(i, dt, u_n, u_stage, uhat, R_hist, **kw))
        u_new = self.empty(*self.state_shape)
        self.imex_stage(s + 1, dt, u_n, u_new, uhat, R_hist, **kw)
        return u_new, stats
