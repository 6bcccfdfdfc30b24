"""ctypes binding of the C ABI in include/ap.h (argument marshalling only).

The functions ``ap_*`` below carry the ABI's names and pass plain pointers,
sizes and the current CUDA stream through to libapt.so; every step of the
push runs in the library's kernels.  PyTorch only provides device memory and
streams.  If libapt.so is missing the binding raises: there is no CPU path.

Pulses are described by plain dicts of physical parameters (see
``pulse_desc``); the same dicts drive the CPU oracle in the tests.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapt.so")

AP_OK = 0
AP_ERR_ARG = -1
AP_ERR_ALIGN = -2
AP_ERR_CUDA = -3
AP_ERR_NONFINITE = -4
AP_ERR_TIMEOUT = -5
AP_ERR_WORKSPACE = -6
AP_ERR_UNSUPPORTED = -7

KINDS = {"plane": 0, "gauss": 1, "lg": 2, "flying": 3, "flying_cf": 4}
POLS = {"x": 0, "y": 1, "cp": 2, "cm": 3}
ENVS = {"sin2": 0, "gauss": 1, "sgauss": 2, "cw": 3}
PRECISIONS = {"fp64": 0, "fp32_phase64": 1, "fp32": 2, "fp32_phaseff": 2}
AP_F_LONGITUDINAL = 1
AP_F_YEE_DISP = 2
AP_F_1D3V = 4
AP_PACK_NODES = 0
AP_PACK_CELLS = 1
PACK_LAYOUTS = {"nodes": AP_PACK_NODES, "cells": AP_PACK_CELLS}
AP_NPARAM = 4
AP_OBJ_MEAN_GAMMA = 0
AP_MAX_COMP = 128
AP_MAX_SETS = 4096
AP_YEE1D_MAX_NODES = 12288
AP_LINE1D_MAX_NODES_F32 = 12288
AP_LINE1D_MAX_NODES_F64 = 6144
AP_APT1D_MAX_NODES_F32 = 8192
AP_ABI_VERSION = 3


class ApPulseDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("pol", ctypes.c_int32), ("env", ctypes.c_int32),
        ("sg_order", ctypes.c_int32), ("lg_p", ctypes.c_int32), ("lg_l", ctypes.c_int32),
        ("n_comp", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("a0", ctypes.c_double), ("omega", ctypes.c_double), ("w0", ctypes.c_double),
        ("z_focus", ctypes.c_double), ("t_focus", ctypes.c_double), ("env_len", ctypes.c_double),
        ("phase0", ctypes.c_double), ("beta_f", ctypes.c_double), ("bw_frac", ctypes.c_double),
        ("ff_length", ctypes.c_double), ("yee_dx", ctypes.c_double), ("yee_dt", ctypes.c_double),
        ("omega_p", ctypes.c_double),
    ]


class ApParticles(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
        ("ux", ctypes.c_void_p), ("uy", ctypes.c_void_p), ("uz", ctypes.c_void_p),
        ("n", ctypes.c_int64), ("set_offsets", ctypes.c_void_p), ("n_sets", ctypes.c_int32),
    ]


class ApGrid(ctypes.Structure):
    _fields_ = [
        ("f", ctypes.c_void_p * 6), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("packed", ctypes.c_void_p), ("packed_layout", ctypes.c_int32),
    ]


class ApDiag(ctypes.Structure):
    _fields_ = [
        ("lightfront_max", ctypes.c_void_p), ("gamma_hist", ctypes.c_void_p),
        ("hist_bins", ctypes.c_int32), ("hist_lo", ctypes.c_double), ("hist_hi", ctypes.c_double),
        ("set_gamma_sum", ctypes.c_void_p), ("accumulate", ctypes.c_int32),
    ]


class ApYeeGrid(ctypes.Structure):
    _fields_ = [
        ("f", ctypes.c_void_p * 6), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("f64", ctypes.c_int32),
        ("lo", ctypes.c_double * 3), ("d", ctypes.c_double * 3),
    ]


class ApYee1d(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_void_p), ("B", ctypes.c_void_p), ("nz", ctypes.c_int32),
        ("n_lines", ctypes.c_int32), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
    ]


class ApLine1d(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_void_p), ("B", ctypes.c_void_p), ("J", ctypes.c_void_p), ("wp2", ctypes.c_void_p),
        ("nz", ctypes.c_int32), ("n_lines", ctypes.c_int32), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
        ("omega_p", ctypes.c_double), ("z0", ctypes.c_double),
    ]


class ApLaunchCfg(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("grid_cache", ctypes.c_int32),
                ("pairs", ctypes.c_int32), ("tile", ctypes.c_int32)]


# every entry point declared in include/ap.h: name -> (restype, argtypes)
_vp = ctypes.c_void_p
SIGNATURES = {
    "ap_version": (ctypes.c_int, []),
    "ap_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ap_init_pulse": (ctypes.c_int, [ctypes.POINTER(ApPulseDesc), ctypes.c_int32, ctypes.POINTER(_vp)]),
    "ap_destroy": (None, [_vp]),
    "ap_set_launch": (ctypes.c_int, [_vp, ctypes.POINTER(ApLaunchCfg)]),
    "ap_grid_packed_bytes": (ctypes.c_size_t, [ctypes.POINTER(ApGrid)]),
    "ap_grid_pack": (ctypes.c_int, [ctypes.POINTER(ApGrid), _vp, _vp]),
    "ap_eval_fields": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int64, _vp, ctypes.c_int32, _vp]),
    "ap_gather_push": (ctypes.c_int, [_vp, ctypes.POINTER(ApParticles), ctypes.POINTER(ApGrid),
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.POINTER(ApDiag), _vp]),
    "ap_batch_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "ap_gather_push_batched": (ctypes.c_int, [_vp, ctypes.POINTER(ApParticles), ctypes.POINTER(ApGrid),
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.POINTER(ApDiag), _vp,
                                              ctypes.c_size_t, _vp]),
    "ap_gather_push_batched_static": (ctypes.c_int, [_vp, ctypes.POINTER(ApParticles),
                                                     ctypes.POINTER(ApGrid), ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                                     ctypes.POINTER(ApDiag), _vp]),
    "ap_batch_graph_create": (ctypes.c_int, [_vp, ctypes.POINTER(ApParticles), ctypes.POINTER(ApGrid),
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.POINTER(ApDiag), _vp, ctypes.c_size_t,
                                             _vp, ctypes.POINTER(_vp)]),
    "ap_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "ap_graph_destroy": (None, [_vp]),
    "ap_adjoint_workspace_bytes": (ctypes.c_size_t, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]),
    "ap_push_adjoint": (ctypes.c_int, [_vp, ctypes.POINTER(ApParticles), ctypes.POINTER(ApGrid),
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "ap_sync_status": (ctypes.c_int, [_vp, _vp]),
    "ap_num_sets": (ctypes.c_int, [_vp]),
    "ap_eval_nodes": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ApYeeGrid), ctypes.c_double,
                                     ctypes.c_int32, ctypes.c_int32, _vp]),
    "ap_eval_current": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ApYeeGrid), ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_int32, _vp]),
    "ap_yee1d_run": (ctypes.c_int, [ctypes.POINTER(ApYee1d), ctypes.c_int64, ctypes.c_int32, _vp]),
    "ap_plasma1d_run": (ctypes.c_int, [ctypes.POINTER(ApLine1d), ctypes.c_int64, ctypes.c_int32, _vp]),
    "ap_apt1d_run": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ApLine1d), ctypes.c_double,
                                    ctypes.c_int64, ctypes.c_int32, _vp]),
}

_lib = None
_lock = threading.Lock()


class APError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = lib().ap_status_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s failed: %s (%d)" % (fn, msg, status))


def lib():
    """Load libapt.so (raises if it has not been built: no fallback)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(
                        "libapt.so not found at %s: build it with "
                        "`python -m paper_2307_04843_gb300.build` (no CPU fallback exists)" % LIB_PATH)
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                if L.ap_version() != AP_ABI_VERSION:
                    raise RuntimeError("libapt.so has ABI version %d, the binding expects %d: rebuild it"
                                       % (L.ap_version(), AP_ABI_VERSION))
                _lib = L
    return _lib


def check(fn, rc):
    if rc != AP_OK:
        raise APError(fn, rc)
    return rc


# ---------------------------------------------------------------- marshalling

def pulse_desc(d):
    """ap_pulse_desc from a pulse dict (kind, pol, env strings; physical floats)."""
    p = ApPulseDesc()
    p.kind = KINDS[d.get("kind", "plane")]
    p.pol = POLS[d.get("pol", "x")]
    p.env = ENVS[d.get("env", "cw")]
    p.sg_order = int(d.get("sg_order", 1))
    p.lg_p = int(d.get("lg_p", 0))
    p.lg_l = int(d.get("lg_l", 0))
    p.n_comp = int(d.get("n_comp", 0))
    p.flags = (AP_F_LONGITUDINAL if d.get("longitudinal", False) else 0) | \
              (AP_F_YEE_DISP if d.get("yee", False) else 0) | \
              (AP_F_1D3V if d.get("one_d", False) else 0)
    for name in ("a0", "omega", "w0", "z_focus", "t_focus", "env_len", "phase0", "beta_f",
                 "bw_frac", "ff_length", "yee_dx", "yee_dt", "omega_p"):
        setattr(p, name, float(d.get(name, 1.0 if name == "omega" else 0.0)))
    return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def precision_id(precision):
    if isinstance(precision, int):
        return precision
    return PRECISIONS[precision]


def particles_struct(p, precision, set_offsets=None):
    """ap_particles from a dict of CUDA tensors x, y, z (float64) and ux, uy,
    uz (float64 for fp64, float32 otherwise), all contiguous and of equal length."""
    import torch
    n = p["x"].numel()
    udt = torch.float64 if precision_id(precision) == 0 else torch.float32
    for k in ("x", "y", "z"):
        t = p[k]
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError("particle array %s must be a contiguous CUDA float64 tensor of length %d" % (k, n))
    for k in ("ux", "uy", "uz"):
        t = p[k]
        if t.dtype != udt or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError("particle array %s must be a contiguous CUDA %s tensor of length %d" % (k, udt, n))
    s = ApParticles()
    s.x, s.y, s.z = p["x"].data_ptr(), p["y"].data_ptr(), p["z"].data_ptr()
    s.ux, s.uy, s.uz = p["ux"].data_ptr(), p["uy"].data_ptr(), p["uz"].data_ptr()
    s.n = n
    if set_offsets is not None:
        if set_offsets.dtype != torch.int64 or not set_offsets.is_cuda:
            raise ValueError("set_offsets must be a CUDA int64 tensor")
        s.set_offsets = set_offsets.data_ptr()
        s.n_sets = set_offsets.numel() - 1
    return s


def grid_struct(grid):
    """ap_grid from (tensor [6, nz, ny, nx] float32 CUDA, lo, hi[, packed[,
    layout]]) or None; `packed` is the copy made by ``pack_grid`` in `layout`
    ("nodes", the default, or "cells")."""
    if grid is None:
        return None
    import torch
    g, lo, hi = grid[:3]
    packed = grid[3] if len(grid) > 3 else None
    layout = PACK_LAYOUTS[grid[4]] if len(grid) > 4 else AP_PACK_NODES
    if g.dtype != torch.float32 or not g.is_cuda or not g.is_contiguous() or g.dim() != 4 or g.shape[0] != 6:
        raise ValueError("grid must be a contiguous CUDA float32 tensor [6, nz, ny, nx]")
    s = ApGrid()
    for c in range(6):
        s.f[c] = g[c].data_ptr()
    s.nz, s.ny, s.nx = int(g.shape[1]), int(g.shape[2]), int(g.shape[3])
    for a in range(3):
        s.lo[a] = float(lo[a])
        s.hi[a] = float(hi[a])
    s.packed_layout = layout
    if packed is not None:
        if packed.dtype != torch.float32 or not packed.is_cuda or packed.numel() * 4 != ap_grid_packed_bytes(s):
            raise ValueError("packed grid must be the CUDA float32 tensor made by pack_grid")
        s.packed = packed.data_ptr()
    return s


def ap_grid_packed_bytes(gs):
    return lib().ap_grid_packed_bytes(ctypes.byref(gs))


def ap_grid_pack(grid, packed, stream=None, layout="nodes"):
    gs = grid_struct(tuple(grid[:3]) + (None, layout))
    check("ap_grid_pack", lib().ap_grid_pack(ctypes.byref(gs), _ptr(packed), _stream(stream)))


def pack_grid(grid, stream=None, layout="nodes"):
    """Packed copy of a grid (g, lo, hi) in `layout` ("nodes": 32 B per node;
    "cells": per-cell trilinear coefficients, 192 B per cell); returns
    (g, lo, hi, packed, layout)."""
    import torch
    g, lo, hi = grid[:3]
    gs = grid_struct((g, lo, hi, None, layout))
    packed = torch.empty(ap_grid_packed_bytes(gs) // 4, dtype=torch.float32, device=g.device)
    ap_grid_pack((g, lo, hi), packed, stream, layout)
    return (g, lo, hi, packed, layout)


def diag_struct(diag):
    """ap_diag from a dict with optional CUDA tensors lightfront (float64),
    hist (int32, read as uint32), set_sum (float64) and hist_bins/lo/hi."""
    if not diag:
        return None
    d = ApDiag()
    if diag.get("lightfront") is not None:
        d.lightfront_max = diag["lightfront"].data_ptr()
    if diag.get("hist") is not None:
        d.gamma_hist = diag["hist"].data_ptr()
        d.hist_bins = int(diag["hist"].numel())
        d.hist_lo = float(diag["hist_lo"])
        d.hist_hi = float(diag["hist_hi"])
    if diag.get("set_sum") is not None:
        d.set_gamma_sum = diag["set_sum"].data_ptr()
    d.accumulate = 1 if diag.get("accumulate") else 0
    return d


def _ref(s):
    return ctypes.byref(s) if s is not None else None


# ------------------------------------------------------- ABI-named wrappers

def ap_version():
    return lib().ap_version()


def ap_status_string(status):
    return lib().ap_status_string(status).decode()


def ap_init_pulse(pulses):
    """Create a handle for a list of pulse dicts (one per set)."""
    if isinstance(pulses, dict):
        pulses = [pulses]
    arr = (ApPulseDesc * len(pulses))(*[pulse_desc(d) for d in pulses])
    h = ctypes.c_void_p()
    check("ap_init_pulse", lib().ap_init_pulse(arr, len(pulses), ctypes.byref(h)))
    return h


def ap_destroy(h):
    lib().ap_destroy(h)


def ap_set_launch(h, block=0, blocks_per_sm=0, grid_cache=0, pairs=0, tile=0):
    cfg = ApLaunchCfg(block, blocks_per_sm, grid_cache, pairs, tile)
    check("ap_set_launch", lib().ap_set_launch(h, ctypes.byref(cfg)))


def ap_eval_fields(h, set_index, xyzt, EB_out, precision, stream=None):
    """xyzt: CUDA float64 [4, n]; EB_out: CUDA float64 [6, n]."""
    n = xyzt.shape[1]
    check("ap_eval_fields", lib().ap_eval_fields(h, set_index, _ptr(xyzt), n, _ptr(EB_out),
                                                 precision_id(precision), _stream(stream)))


def ap_gather_push(h, particles, grid, t0, dt, n_steps, precision, diag=None, stream=None):
    ps = particles_struct(particles, precision)
    check("ap_gather_push", lib().ap_gather_push(h, ctypes.byref(ps), _ref(grid_struct(grid)), float(t0),
                                                 float(dt), int(n_steps), precision_id(precision),
                                                 _ref(diag_struct(diag)), _stream(stream)))


def ap_batch_workspace_bytes(h):
    return lib().ap_batch_workspace_bytes(h)


def ap_gather_push_batched(h, particles, set_offsets, grid, t0, dt, n_steps, precision, diag,
                           workspace, stream=None):
    ps = particles_struct(particles, precision, set_offsets)
    check("ap_gather_push_batched",
          lib().ap_gather_push_batched(h, ctypes.byref(ps), _ref(grid_struct(grid)), float(t0), float(dt),
                                       int(n_steps), precision_id(precision), _ref(diag_struct(diag)),
                                       _ptr(workspace), workspace.numel() * workspace.element_size(),
                                       _stream(stream)))


def ap_gather_push_batched_static(h, particles, set_offsets, grid, t0, dt, n_steps, precision, diag,
                                  stream=None):
    """Batched push without a caller workspace: for callers that cannot
    allocate device memory when they push (their allocator owns the GPU, or
    the step loop must not risk a synchronising or failing allocation).  The
    scratch is a static device array shared by every call on the device, so
    calls must not overlap on the GPU; the first call on a device should come
    before any stream capture."""
    ps = particles_struct(particles, precision, set_offsets)
    check("ap_gather_push_batched_static",
          lib().ap_gather_push_batched_static(h, ctypes.byref(ps), _ref(grid_struct(grid)), float(t0),
                                              float(dt), int(n_steps), precision_id(precision),
                                              _ref(diag_struct(diag)), _stream(stream)))


def ap_batch_graph_create(h, particles, set_offsets, grid, t0, dt, n_steps, precision, diag, workspace,
                          stream):
    ps = particles_struct(particles, precision, set_offsets)
    g = ctypes.c_void_p()
    check("ap_batch_graph_create",
          lib().ap_batch_graph_create(h, ctypes.byref(ps), _ref(grid_struct(grid)), float(t0), float(dt),
                                      int(n_steps), precision_id(precision), _ref(diag_struct(diag)),
                                      _ptr(workspace), workspace.numel() * workspace.element_size(),
                                      _stream(stream), ctypes.byref(g)))
    return g


def ap_graph_launch(g, stream=None):
    check("ap_graph_launch", lib().ap_graph_launch(g, _stream(stream)))


def ap_graph_destroy(g):
    lib().ap_graph_destroy(g)


def ap_adjoint_workspace_bytes(h, n, n_steps, ckpt_every):
    return lib().ap_adjoint_workspace_bytes(h, int(n), int(n_steps), int(ckpt_every))


def ap_push_adjoint(h, particles, set_offsets, grid, t0, dt, n_steps, ckpt_every, precision, dJ, J,
                    workspace, stream=None):
    ps = particles_struct(particles, precision, set_offsets)
    check("ap_push_adjoint",
          lib().ap_push_adjoint(h, ctypes.byref(ps), _ref(grid_struct(grid)), float(t0), float(dt),
                                int(n_steps), int(ckpt_every), AP_OBJ_MEAN_GAMMA, precision_id(precision),
                                _ptr(dJ), _ptr(J), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)))


def ap_sync_status(h, stream=None):
    return lib().ap_sync_status(h, _stream(stream))


def ap_num_sets(h):
    return lib().ap_num_sets(h)


def yee_grid_struct(fields, lo, d):
    """ap_yee_grid from a list of six CUDA tensors (or None) of one shape
    (nz, ny, nx) and one dtype (float32 or float64), node (0,0,0) at lo,
    spacing d."""
    import torch
    present = [f for f in fields if f is not None]
    if len(fields) != 6 or not present:
        raise ValueError("need six entries (tensor or None), at least one tensor")
    shape, dtype = present[0].shape, present[0].dtype
    for f in present:
        if f.shape != shape or f.dtype != dtype or not f.is_cuda or not f.is_contiguous():
            raise ValueError("node arrays must be contiguous CUDA tensors of one shape and dtype")
    if dtype not in (torch.float32, torch.float64) or len(shape) != 3:
        raise ValueError("node arrays must be float32 or float64 of shape (nz, ny, nx)")
    g = ApYeeGrid()
    for c in range(6):
        g.f[c] = fields[c].data_ptr() if fields[c] is not None else None
    g.nz, g.ny, g.nx = (int(v) for v in shape)
    g.f64 = 1 if dtype == torch.float64 else 0
    for a in range(3):
        g.lo[a] = float(lo[a])
        g.d[a] = float(d[a])
    return g


def ap_eval_nodes(h, set_index, fields, lo, d, t, accumulate=False, precision="fp64", stream=None):
    gs = yee_grid_struct(fields, lo, d)
    check("ap_eval_nodes", lib().ap_eval_nodes(h, set_index, ctypes.byref(gs), float(t),
                                               1 if accumulate else 0, precision_id(precision),
                                               _stream(stream)))


def ap_eval_current(h, set_index, fields, lo, d, t, accumulate=False, precision="fp64", stream=None):
    """J1 on the E nodes: fields = [Jx, Jy, Jz] tensors (or None)."""
    gs = yee_grid_struct(list(fields) + [None, None, None], lo, d)
    check("ap_eval_current", lib().ap_eval_current(h, set_index, ctypes.byref(gs), float(t),
                                                   1 if accumulate else 0, precision_id(precision),
                                                   _stream(stream)))


def ap_yee1d_run(E, B, dz, dt, n_steps, stream=None):
    """n_steps of the 1-D vacuum Yee scheme on CUDA tensors E, B of shape
    (n_lines, nz) or (nz,), float64 (AP_FP64) or float32 (AP_FP32_PHASEFF)."""
    import torch
    if E.shape != B.shape or E.dtype != B.dtype or E.dim() not in (1, 2):
        raise ValueError("E and B must have one shape (n_lines, nz) or (nz,) and one dtype")
    if not (E.is_cuda and B.is_cuda and E.is_contiguous() and B.is_contiguous()):
        raise ValueError("E and B must be contiguous CUDA tensors")
    y = ApYee1d()
    y.E, y.B = E.data_ptr(), B.data_ptr()
    y.nz = int(E.shape[-1])
    y.n_lines = int(E.shape[0]) if E.dim() == 2 else 1
    y.dz, y.dt = float(dz), float(dt)
    prec = {torch.float64: 0, torch.float32: 2}.get(E.dtype)
    if prec is None:
        raise ValueError("E and B must be float32 or float64")
    check("ap_yee1d_run", lib().ap_yee1d_run(ctypes.byref(y), int(n_steps), prec, _stream(stream)))


def line_struct(E, B, J, dz, dt, wp2=None, omega_p=0.0, z0=0.0):
    """ap_line1d from CUDA tensors E, B, J (and optional wp2) of one shape
    (n_lines, nz) or (nz,) and one dtype; returns (struct, precision id)."""
    import torch
    arrs = [E, B, J] + ([wp2] if wp2 is not None else [])
    for a in arrs:
        if a.shape != E.shape or a.dtype != E.dtype or not a.is_cuda or not a.is_contiguous():
            raise ValueError("line arrays must be contiguous CUDA tensors of one shape and dtype")
    if E.dim() not in (1, 2):
        raise ValueError("line arrays must have shape (n_lines, nz) or (nz,)")
    prec = {torch.float64: 0, torch.float32: 2}.get(E.dtype)
    if prec is None:
        raise ValueError("line arrays must be float32 or float64")
    y = ApLine1d()
    y.E, y.B, y.J = E.data_ptr(), B.data_ptr(), J.data_ptr()
    y.wp2 = wp2.data_ptr() if wp2 is not None else None
    y.nz = int(E.shape[-1])
    y.n_lines = int(E.shape[0]) if E.dim() == 2 else 1
    y.dz, y.dt, y.omega_p, y.z0 = float(dz), float(dt), float(omega_p), float(z0)
    return y, prec


def ap_plasma1d_run(E, B, J, dz, dt, n_steps, wp2=None, omega_p=0.0, stream=None):
    """n_steps of the Yee line with a linear cold-plasma current (E_x at z_k,
    B_y at z_{k+1/2}, J_x at z_k and half steps); float64 (AP_FP64) or
    float32 (AP_FP32_PHASEFF) by the arrays' dtype."""
    y, prec = line_struct(E, B, J, dz, dt, wp2, omega_p)
    check("ap_plasma1d_run", lib().ap_plasma1d_run(ctypes.byref(y), int(n_steps), prec, _stream(stream)))


def ap_apt1d_run(h, set_index, E2, B2, J, z0, dz, t0, dt, n_steps, wp2=None, omega_p=0.0, stream=None):
    """n_steps of the split line of Sec. 4 with the analytic E1 and J1 of
    set `set_index` (nodes at z0 + k dz, steps from t0)."""
    y, prec = line_struct(E2, B2, J, dz, dt, wp2, omega_p, z0)
    check("ap_apt1d_run", lib().ap_apt1d_run(h, int(set_index), ctypes.byref(y), float(t0), int(n_steps),
                                             prec, _stream(stream)))


# ------------------------------------------------------------ convenience

class Handle:
    """Owns an ap_handle for a list of pulse dicts."""

    def __init__(self, pulses):
        self.pulses = [pulses] if isinstance(pulses, dict) else list(pulses)
        self.h = ap_init_pulse(self.pulses)

    def close(self):
        if self.h is not None and _lib is not None:
            ap_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_launch(self, block=0, blocks_per_sm=0, grid_cache=0, pairs=0, tile=0):
        ap_set_launch(self.h, block, blocks_per_sm, grid_cache, pairs, tile)

    def push(self, particles, t0, dt, n_steps, precision="fp32", grid=None, diag=None, stream=None):
        ap_gather_push(self.h, particles, grid, t0, dt, n_steps, precision, diag, stream)

    def eval_fields(self, x, y, z, t, precision="fp64", set_index=0):
        import torch
        xyzt = torch.stack([torch.as_tensor(v, dtype=torch.float64, device="cuda").reshape(-1)
                            for v in torch.broadcast_tensors(*[torch.as_tensor(v, dtype=torch.float64)
                                                               for v in (x, y, z, t)])]).contiguous()
        EB = torch.empty((6, xyzt.shape[1]), dtype=torch.float64, device="cuda")
        ap_eval_fields(self.h, set_index, xyzt, EB, precision)
        return EB

    def eval_nodes(self, fields, lo, d, t, accumulate=False, precision="fp64", set_index=0, stream=None):
        """Analytic E1/B1 on the Yee-staggered nodes (see ap_eval_nodes)."""
        ap_eval_nodes(self.h, set_index, fields, lo, d, t, accumulate, precision, stream)

    def eval_current(self, fields, lo, d, t, accumulate=False, precision="fp64", set_index=0, stream=None):
        """Analytic current J1 on the E nodes (see ap_eval_current)."""
        ap_eval_current(self.h, set_index, fields, lo, d, t, accumulate, precision, stream)

    def apt1d(self, E2, B2, J, z0, dz, t0, dt, n_steps, wp2=None, omega_p=0.0, set_index=0, stream=None):
        """Split line with this handle's analytic E1 and J1 (see ap_apt1d_run)."""
        ap_apt1d_run(self.h, set_index, E2, B2, J, z0, dz, t0, dt, n_steps, wp2, omega_p, stream)

    def status(self, stream=None):
        return ap_sync_status(self.h, stream)


def to_device(particles, precision="fp32", device="cuda"):
    """Copy a dict of numpy arrays to CUDA tensors in the ABI's layout."""
    import numpy as np
    import torch
    udt = torch.float64 if precision_id(precision) == 0 else torch.float32
    out = {}
    for k in ("x", "y", "z"):
        out[k] = torch.as_tensor(np.ascontiguousarray(particles[k], dtype=np.float64)).to(device)
    for k in ("ux", "uy", "uz"):
        out[k] = torch.as_tensor(np.ascontiguousarray(particles[k], dtype=np.float64)).to(device=device, dtype=udt)
    return out


def to_host(particles):
    return {k: v.detach().double().cpu().numpy() for k, v in particles.items()}

