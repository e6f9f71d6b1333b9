"""Thin Python binding of the C ABI in include/wos.h.

Argument marshalling only: every step of the operator build, the SVD and the
reconstruction runs in the CUDA library ``_lib/libwos.so``.  There is no CPU
path: if the library cannot be loaded, every call raises.

The binding mirrors the C names (``wos_build_operator``, ``wos_op_svd``,
``wos_reconstruct``, ...).  Device arrays are torch CUDA tensors (PyTorch is
used for device memory and streams only); descriptors come from the
``workloads`` dataclasses.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from pathlib import Path

import numpy as np

MAX_VERTICES = 64
MAX_HOLES = 16
_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libwos.so"

STATUS = {
    0: "WOS_OK", 1: "WOS_INVALID_ARG", 2: "WOS_K_NOT_SPD", 3: "WOS_POINT_OUTSIDE",
    4: "WOS_EPS_BELOW_FP32_FLOOR", 5: "WOS_COUNT_OVERFLOW", 6: "WOS_STEP_CAP_HIT",
    7: "WOS_DEVICE_TIMEOUT", 8: "WOS_OOM", 9: "WOS_CUDA_ERROR",
    10: "WOS_NO_CONVERGENCE", 11: "WOS_TRUNCATION_IN_CLUSTER", 12: "WOS_NOT_READY",
    13: "WOS_NOALLOC_LIMIT",
}
WARNINGS = {6, 11}


class WosError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class WosDomain(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("outer_kind", ctypes.c_int32),
        ("center", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
        ("half", ctypes.c_double * 3),
        ("n_vertices", ctypes.c_int32),
        ("vertices", ctypes.c_double * (2 * MAX_VERTICES)),
        ("n_holes", ctypes.c_int32),
        ("hole_center", (ctypes.c_double * 3) * MAX_HOLES),
        ("hole_radius", ctypes.c_double * MAX_HOLES),
    ]


class WosPartition(ctypes.Structure):
    _fields_ = [
        ("outer_m", ctypes.c_int32),
        ("outer_theta0", ctypes.c_double),
        ("edge_m", ctypes.c_int32 * MAX_VERTICES),
        ("outer_nb", ctypes.c_int32),
        ("outer_ns", ctypes.c_int32),
        ("face_n1", ctypes.c_int32),
        ("face_n2", ctypes.c_int32),
        ("hole_m", ctypes.c_int32 * MAX_HOLES),
        ("hole_theta0", ctypes.c_double * MAX_HOLES),
        ("hole_nb", ctypes.c_int32 * MAX_HOLES),
        ("hole_ns", ctypes.c_int32 * MAX_HOLES),
        ("voronoi_n", ctypes.c_int32),
        ("voronoi_sites", ctypes.POINTER(ctypes.c_double)),
    ]


class WosOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("step_cap", ctypes.c_uint32),
        ("stream_id", ctypes.c_uint32),
        ("k0", ctypes.c_uint32),
        ("k1", ctypes.c_uint32),
        ("accumulate", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("tile_walks", ctypes.c_int32),
        ("hist_slots", ctypes.c_int32),
        ("refill_min", ctypes.c_int32),
        ("tiles_per_warp", ctypes.c_int32),
        ("trace_elem", ctypes.c_void_p),
        ("trace_steps", ctypes.c_void_p),
        ("trace_x", ctypes.c_void_p),
        ("kernel_events", ctypes.c_void_p * 2),
        ("mapped", ctypes.c_int32),
        ("group_blocks", ctypes.c_int32),
    ]


class WosProblem(ctypes.Structure):
    _fields_ = [
        ("domain", ctypes.c_void_p),
        ("partition", ctypes.c_void_p),
        ("K", ctypes.c_void_p),
        ("points", ctypes.c_void_p),
        ("M_D", ctypes.c_int32),
        ("N", ctypes.c_uint32),
        ("eps", ctypes.c_double),
        ("stream_id", ctypes.c_uint32),
        ("step_cap", ctypes.c_uint32),
        ("counts", ctypes.c_void_p),
        ("unterminated", ctypes.c_void_p),
        ("k0", ctypes.c_uint32),
        ("k1", ctypes.c_uint32),
    ]


class WosTuning(ctypes.Structure):
    _fields_ = [
        ("block_size", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("tiles_per_warp", ctypes.c_int32),
        ("hist_slots", ctypes.c_int32),
        ("refill_min", ctypes.c_int32),
        ("group_blocks", ctypes.c_int32),
        ("trials", ctypes.c_int32),
        ("best_ms", ctypes.c_float),
        ("default_ms", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class WosStats(ctypes.Structure):
    _fields_ = [
        ("walks", ctypes.c_uint64),
        ("steps", ctypes.c_uint64),
        ("unterminated", ctypes.c_uint64),
        ("max_steps", ctypes.c_uint32),
        ("grid", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("tile_walks", ctypes.c_int32),
        ("hist_slots", ctypes.c_int32),
        ("kernel_ms", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class WosSvdProblem(ctypes.Structure):
    _fields_ = [
        ("counts", ctypes.c_void_p),
        ("M_D", ctypes.c_int32),
        ("M_tot", ctypes.c_int32),
        ("N", ctypes.c_uint32),
        ("gamma1", ctypes.c_void_p),
        ("nu", ctypes.c_void_p),
        ("sigma", ctypes.c_void_p),
        ("U", ctypes.c_void_p),
        ("S", ctypes.c_void_p),
        ("V", ctypes.c_void_p),
    ]


class WosQueueOpts(ctypes.Structure):
    _fields_ = [
        ("max_inflight", ctypes.c_int32),
        ("device_budget", ctypes.c_uint64),
        ("slice_walks", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("side_streams", ctypes.c_int32),
    ]


class WosRequest(ctypes.Structure):
    _fields_ = [
        ("domain", ctypes.c_void_p),
        ("partition", ctypes.c_void_p),
        ("gamma1", ctypes.c_void_p),
        ("K", ctypes.c_void_p),
        ("points", ctypes.c_void_p),
        ("M_D", ctypes.c_int32),
        ("N", ctypes.c_uint32),
        ("eps", ctypes.c_double),
        ("stream_id", ctypes.c_uint32),
        ("nu", ctypes.c_void_p),
        ("uD", ctypes.c_void_p),
        ("u0", ctypes.c_void_p),
        ("r", ctypes.c_int32),
        ("tikhonov_alpha", ctypes.c_double),
        ("u_gamma1", ctypes.c_void_p),
        ("S", ctypes.c_void_p),
        ("counts", ctypes.c_void_p),
        ("r_used", ctypes.c_void_p),
    ]


class WosQueueStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("admitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("slices", ctypes.c_uint64),
        ("walks", ctypes.c_uint64),
        ("inflight", ctypes.c_int32),
        ("queued", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libwos.so.  Raises when it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        if not build_if_missing:
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing; build it with "
                "python -c 'import __graft_entry__ as g; g.build()'")
        from . import build as _b
        _b.build()
    L = ctypes.CDLL(str(LIB_PATH))
    vp, i32, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                              ctypes.c_uint64, ctypes.c_double)
    L.wos_create.argtypes = [i32, ctypes.POINTER(vp)]
    L.wos_destroy.argtypes = [vp]
    L.wos_kernel_launches.restype = u64
    L.wos_kernel_launches.argtypes = [vp]
    L.wos_set_svd_path.argtypes = [vp, i32]
    L.wos_measure_pipes.argtypes = [vp, vp, vp]
    L.wos_status_string.restype = ctypes.c_char_p
    L.wos_status_string.argtypes = [ctypes.c_int]
    L.wos_conductivity_sqrt.argtypes = [i32, vp, vp]
    L.wos_num_elements.restype = i32
    L.wos_num_elements.argtypes = [vp, vp]
    L.wos_element_measures.argtypes = [vp, vp, vp]
    L.wos_fp32_eps_floor.restype = dbl
    L.wos_fp32_eps_floor.argtypes = [vp]
    L.wos_check_points.argtypes = [vp, vp, i32, vp]
    L.wos_build_operator.argtypes = [vp, vp, vp, vp, i32, vp, u32, dbl, u64, vp, vp, vp,
                                     vp, vp]
    L.wos_build_operator_noalloc.argtypes = [vp, vp, vp, vp, i32, vp, u32, dbl, u64, vp,
                                             vp, vp, vp, vp]
    L.wos_build_operators_batched.argtypes = [vp, i32, vp, u64, vp, vp, vp]
    L.wos_autotune.argtypes = [vp, vp, u64, i32, u64, vp, vp]
    L.wos_autotune_reset.argtypes = [vp]
    L.wos_op_svd.argtypes = [vp, vp, i32, i32, u32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.wos_reconstruct.argtypes = [vp, vp, vp, vp, i32, i32, vp, i32, u32, vp, vp, vp, vp,
                                  vp, i32, dbl, vp, vp, vp]
    L.wos_truncation_gap.argtypes = [vp, i32, i32]
    L.wos_op_svd_batched.argtypes = [vp, i32, vp, vp, vp, vp]
    L.wos_spectral.argtypes = [vp, vp, vp, vp, i32, i32, vp, i32, u32, vp, vp, vp, vp, vp,
                               i32, vp, vp, vp, vp, vp, vp]
    L.wos_queue_create.argtypes = [vp, vp, ctypes.POINTER(vp)]
    L.wos_queue_destroy.argtypes = [vp]
    L.wos_submit.argtypes = [vp, vp, ctypes.POINTER(u64)]
    L.wos_poll.argtypes = [vp, u64]
    L.wos_wait.argtypes = [vp, u64, i32]
    L.wos_queue_get_stats.argtypes = [vp, vp]
    _lib = L
    return L


def _check(code: int, where: str, allow_warning: bool = True) -> int:
    if code == 0 or (allow_warning and code in WARNINGS):
        return code
    raise WosError(code, where)


# ---------------------------------------------------------------------------
# descriptors
# ---------------------------------------------------------------------------
_KIND = {"sphere": 1, "box": 2, "polygon": 3}


def make_domain(dom) -> WosDomain:
    D = WosDomain()
    D.dim = dom.dim
    D.outer_kind = _KIND[dom.outer]
    for a in range(3):
        D.center[a] = float(dom.center[a]) if a < len(dom.center) else 0.0
        D.half[a] = float(dom.half[a]) if a < len(dom.half) else 0.0
    D.radius = float(dom.radius)
    if dom.outer == "polygon":
        D.n_vertices = len(dom.vertices)
        for e, (x, y) in enumerate(dom.vertices):
            D.vertices[2 * e] = x
            D.vertices[2 * e + 1] = y
    D.n_holes = len(dom.holes)
    for h, (c, r) in enumerate(dom.holes):
        for a in range(3):
            D.hole_center[h][a] = float(c[a]) if a < len(c) else 0.0
        D.hole_radius[h] = float(r)
    return D


def make_partition(dom, part):
    """Returns (struct, keep-alive objects)."""
    P = WosPartition()
    keep = []
    P.outer_m = part.outer_m
    P.outer_theta0 = part.outer_theta0
    for e, m in enumerate(part.edge_m):
        P.edge_m[e] = int(m)
    P.outer_nb, P.outer_ns = part.outer_nb, part.outer_ns
    P.face_n1, P.face_n2 = part.face_n1, part.face_n2
    for h in range(len(dom.holes)):
        if part.voronoi_sites is not None:
            break  # Voronoi sites replace the per-component cells
        if dom.dim == 2:
            P.hole_m[h] = part.hole_m[h]
            P.hole_theta0[h] = part.hole_theta0[h]
        else:
            P.hole_nb[h] = part.hole_nb[h]
            P.hole_ns[h] = part.hole_ns[h]
    if part.voronoi_sites is not None:
        s = np.ascontiguousarray(part.voronoi_sites, dtype=np.float64)
        keep.append(s)
        P.voronoi_n = s.shape[0]
        P.voronoi_sites = s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return P, keep


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Context:
    """A library context on one CUDA device (owns events and settings)."""

    def __init__(self, device: int = 0):
        L = load()
        h = ctypes.c_void_p()
        _check(L.wos_create(device, ctypes.byref(h)), "wos_create", False)
        self.h = h
        self.device = device

    def kernel_launches(self) -> int:
        return int(load().wos_kernel_launches(self.h))

    def close(self):
        if self.h:
            load().wos_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wos_conductivity_sqrt(K) -> np.ndarray:
    """S = (K / lambda_max(K))^{1/2} as the library computes it (host)."""
    Kc = np.ascontiguousarray(K, dtype=np.float64)
    d = Kc.shape[0]
    S = np.zeros((d, d))
    _check(load().wos_conductivity_sqrt(d, Kc.ctypes.data, S.ctypes.data),
           "wos_conductivity_sqrt", False)
    return S


def wos_num_elements(domain, partition) -> int:
    D = make_domain(domain)
    P, keep = make_partition(domain, partition)
    return int(load().wos_num_elements(ctypes.byref(D), ctypes.byref(P)))


def wos_element_measures(domain, partition) -> np.ndarray:
    D = make_domain(domain)
    P, keep = make_partition(domain, partition)
    n = wos_num_elements(domain, partition)
    out = np.zeros(n)
    _check(load().wos_element_measures(ctypes.byref(D), ctypes.byref(P),
                                       out.ctypes.data), "wos_element_measures", False)
    return out


def wos_fp32_eps_floor(domain) -> float:
    D = make_domain(domain)
    return float(load().wos_fp32_eps_floor(ctypes.byref(D)))


def wos_check_points(domain, points: np.ndarray) -> int:
    """Returns -1 if all points are inside D, else the first offending index."""
    D = make_domain(domain)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    bad = ctypes.c_int32(-1)
    code = load().wos_check_points(ctypes.byref(D), pts.ctypes.data, len(pts),
                                   ctypes.byref(bad))
    if code == 3:
        return int(bad.value)
    _check(code, "wos_check_points", False)
    return -1


def make_opts(precision: int = 0, step_cap: int = 0, stream_id: int = 0, k0: int = 0,
              k1: int = 0, accumulate: bool = False, block_size: int = 0,
              blocks_per_sm: int = 0, tile_walks: int = 0, hist_slots: int = 0,
              refill_min: int = 0, tiles_per_warp: int = 0,
              trace_elem=None, trace_steps=None, trace_x=None,
              kernel_events=None, mapped: bool = False,
              group_blocks: int = 0) -> WosOpts:
    o = WosOpts()
    o.precision = precision
    o.step_cap = step_cap
    o.stream_id = stream_id
    o.k0, o.k1 = k0, k1
    o.accumulate = int(accumulate)
    o.block_size = block_size
    o.blocks_per_sm = blocks_per_sm
    o.tile_walks = tile_walks
    o.hist_slots = hist_slots
    o.refill_min = refill_min
    o.tiles_per_warp = tiles_per_warp
    o.trace_elem = _ptr(trace_elem)
    o.trace_steps = _ptr(trace_steps)
    o.trace_x = _ptr(trace_x)
    if kernel_events is not None:
        for q, ev in enumerate(kernel_events):
            o.kernel_events[q] = ev.cuda_event
    o.mapped = int(mapped)
    o.group_blocks = group_blocks
    return o


def _check_build_tensors(ctx: Context, where: str, points, dim: int, M_tot: int,
                         counts, unterminated) -> None:
    """The device arrays of a build must match what the library reads and
    writes: points contiguous float64 (M_D, dim); counts contiguous 32-bit
    (M_D, M_tot); unterminated (optional) contiguous 32-bit with >= M_D
    entries; all on the context's device.  Raises WosError(INVALID_ARG)
    before any launch otherwise (an undersized buffer would be written out of
    bounds)."""
    import torch

    def bad(msg):
        raise WosError(1, f"{where}: {msg}")

    want = torch.device("cuda", ctx.device)
    if not isinstance(points, torch.Tensor) or points.device != want:
        bad(f"points must be a tensor on {want}")
    if points.dtype != torch.float64 or not points.is_contiguous() or points.dim() != 2 \
            or points.shape[1] != dim or points.shape[0] < 1:
        bad(f"points must be contiguous float64 of shape (M_D, {dim})")
    M_D = int(points.shape[0])
    if not isinstance(counts, torch.Tensor) or counts.device != want:
        bad(f"counts must be a tensor on {want}")
    if counts.dtype not in (torch.int32, torch.uint32) or not counts.is_contiguous() \
            or tuple(counts.shape) != (M_D, M_tot):
        bad(f"counts must be contiguous 32-bit of shape ({M_D}, {M_tot})")
    if unterminated is not None:
        if not isinstance(unterminated, torch.Tensor) or unterminated.device != want:
            bad(f"unterminated must be a tensor on {want}")
        if unterminated.dtype not in (torch.int32, torch.uint32) \
                or not unterminated.is_contiguous() or unterminated.numel() < M_D:
            bad(f"unterminated must be contiguous 32-bit with at least {M_D} entries")


def wos_build_operator(ctx: Context, domain, K, points, partition, N: int, eps: float,
                       seed: int, opts: WosOpts | None = None, counts=None,
                       unterminated=None, stats: bool = True, stream=None):
    """MC-REM on the GPU.  ``points``: CUDA float64 tensor (M_D, dim).
    Returns (counts, unterminated, stats-dict or None); counts is an int32
    CUDA tensor holding the uint32 counts (M_D, M_tot)."""
    import torch
    L = load()
    D = make_domain(domain)
    P, keep = make_partition(domain, partition)
    M_tot = int(L.wos_num_elements(ctypes.byref(D), ctypes.byref(P)))
    if M_tot < 1:
        raise WosError(1, "wos_num_elements")
    M_D = int(points.shape[0])
    dev = points.device
    if counts is None:
        counts = torch.empty((M_D, M_tot), dtype=torch.int32, device=dev)
    if unterminated is None:
        unterminated = torch.empty(M_D, dtype=torch.int32, device=dev)
    _check_build_tensors(ctx, "wos_build_operator", points, domain.dim, M_tot, counts,
                         unterminated)
    Kc = np.ascontiguousarray(K, dtype=np.float64)
    st = WosStats() if stats else None
    code = L.wos_build_operator(ctx.h, ctypes.byref(D), Kc.ctypes.data, points.data_ptr(),
                                M_D, ctypes.byref(P), int(N), float(eps), int(seed),
                                ctypes.byref(opts) if opts is not None else None,
                                counts.data_ptr(), _ptr(unterminated),
                                ctypes.byref(st) if st is not None else None,
                                _stream(stream))
    _check(code, "wos_build_operator")
    return counts, unterminated, (st.as_dict() if st is not None else None)


def wos_build_operator_noalloc(ctx: Context, domain, K, points, partition, N: int,
                               eps: float, seed: int, counts, unterminated=None,
                               opts: WosOpts | None = None, stats: bool = True,
                               stream=None):
    """The same build as wos_build_operator for callers that cannot allocate
    device memory: the library takes its scratch from a fixed device array
    instead of allocating, and this wrapper allocates nothing either -- the
    caller passes the counts (and optional unterminated) tensors, which are
    checked against the partition's size (a host call) before the build.
    Calls on one device must not overlap on the GPU."""
    L = load()
    D = make_domain(domain)
    P, keep = make_partition(domain, partition)
    M_tot = int(L.wos_num_elements(ctypes.byref(D), ctypes.byref(P)))
    if M_tot < 1:
        raise WosError(1, "wos_num_elements")
    _check_build_tensors(ctx, "wos_build_operator_noalloc", points, domain.dim, M_tot,
                         counts, unterminated)
    Kc = np.ascontiguousarray(K, dtype=np.float64)
    st = WosStats() if stats else None
    code = L.wos_build_operator_noalloc(
        ctx.h, ctypes.byref(D), Kc.ctypes.data, points.data_ptr(), int(points.shape[0]),
        ctypes.byref(P), int(N), float(eps), int(seed),
        ctypes.byref(opts) if opts is not None else None, counts.data_ptr(),
        _ptr(unterminated), ctypes.byref(st) if st is not None else None, _stream(stream))
    _check(code, "wos_build_operator_noalloc")
    return counts, unterminated, (st.as_dict() if st is not None else None)


def wos_build_operators_batched(ctx: Context, insts, seed: int, points=None,
                                counts=None, unterminated=None, opts: WosOpts | None = None,
                                stats: bool = True, stream=None):
    """Builds the operators of many workloads.Instance objects in one launch
    per dimension.  Each instance's stream_id (its `stream`) keeps its walks
    identical to a lone build.  Returns (counts list, unterminated list,
    stats)."""
    import torch
    L = load()
    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    probs = (WosProblem * len(insts))()
    counts = list(counts) if counts is not None else []
    unterminated = list(unterminated) if unterminated is not None else []
    points = list(points) if points is not None else []
    for q, inst in enumerate(insts):
        D = make_domain(inst.domain)
        P, kp = make_partition(inst.domain, inst.partition)
        Kc = np.ascontiguousarray(inst.K, dtype=np.float64)
        keep += [D, P, kp, Kc]
        if len(points) <= q:
            points.append(torch.as_tensor(inst.points, dtype=torch.float64, device=dev))
        M_tot = int(L.wos_num_elements(ctypes.byref(D), ctypes.byref(P)))
        if len(counts) <= q:
            counts.append(torch.empty((inst.M_D, M_tot), dtype=torch.int32, device=dev))
        if len(unterminated) <= q:
            unterminated.append(torch.empty(inst.M_D, dtype=torch.int32, device=dev))
        pb = probs[q]
        pb.domain = ctypes.addressof(D)
        pb.partition = ctypes.addressof(P)
        pb.K = Kc.ctypes.data
        pb.points = points[q].data_ptr()
        pb.M_D = inst.M_D
        pb.N = int(inst.N)
        pb.eps = float(inst.eps)
        pb.stream_id = int(inst.stream)
        pb.step_cap = 0 if inst.step_cap == 1_000_000 else int(inst.step_cap)
        pb.counts = counts[q].data_ptr()
        pb.unterminated = unterminated[q].data_ptr()
    if opts is None and any(getattr(i, "mapped", False) for i in insts):
        opts = make_opts(mapped=True)
    st = WosStats() if stats else None
    code = L.wos_build_operators_batched(ctx.h, len(insts), ctypes.byref(probs), int(seed),
                                         ctypes.byref(opts) if opts is not None else None,
                                         ctypes.byref(st) if st is not None else None,
                                         _stream(stream))
    _check(code, "wos_build_operators_batched")
    return counts, unterminated, (st.as_dict() if st is not None else None)


def wos_autotune(ctx: Context, inst, seed: int | None = None, sample_walks: int = 20_000_000,
                 stream=None) -> dict:
    """Tunes the launch of `inst`'s class (precision, dim, kernel kind) on a
    bounded sample of its walks; later builds with default launch options use
    the result.  Returns the chosen configuration and the sample timings."""
    import torch
    L = load()
    dev = torch.device("cuda", torch.cuda.current_device())
    D = make_domain(inst.domain)
    P, kp = make_partition(inst.domain, inst.partition)
    Kc = np.ascontiguousarray(inst.K, dtype=np.float64)
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=dev)
    M_tot = int(L.wos_num_elements(ctypes.byref(D), ctypes.byref(P)))
    counts = torch.empty((inst.M_D, M_tot), dtype=torch.int32, device=dev)
    pb = WosProblem(ctypes.addressof(D), ctypes.addressof(P), Kc.ctypes.data, pts.data_ptr(),
                    inst.M_D, int(inst.N), float(inst.eps), int(inst.stream), 0,
                    counts.data_ptr(), None, 0, 0)
    out = WosTuning()
    code = L.wos_autotune(ctx.h, ctypes.byref(pb), int(inst.seed if seed is None else seed),
                          1 if inst.fp64 else 0, int(sample_walks), ctypes.byref(out),
                          _stream(stream))
    _check(code, "wos_autotune")
    return out.as_dict()


def wos_autotune_reset(ctx: Context) -> None:
    _check(load().wos_autotune_reset(ctx.h), "wos_autotune_reset", False)


SVD_AUTO, SVD_GRID, SVD_CLUSTER, SVD_FP64_SWEEPS = 0, 1, 2, 3
PIPES = ("ffma", "mufu", "imad_wide", "lop3", "dfma", "issue")


def wos_measure_pipes(ctx: Context, stream=None) -> dict:
    """Measured lane-operations per second of each pipe (see wos.h)."""
    out = (ctypes.c_double * len(PIPES))()
    _check(load().wos_measure_pipes(ctx.h, ctypes.byref(out), _stream(stream)),
           "wos_measure_pipes", False)
    return {k: float(out[q]) for q, k in enumerate(PIPES)}


def wos_set_svd_path(ctx: Context, path: int) -> None:
    """Kernels that factor SVD problems: SVD_AUTO (cluster kernel when the
    worked matrix fits it), SVD_GRID (grid-wide kernels), SVD_CLUSTER, or
    SVD_FP64_SWEEPS (as SVD_AUTO without the FP32 preconditioning sweeps of
    problems of more than 256 columns)."""
    _check(load().wos_set_svd_path(ctx.h, int(path)), "wos_set_svd_path", False)


def wos_op_svd(ctx: Context, counts, N: int, gamma1: np.ndarray, sigma, nu=None,
               sync: bool = True, stream=None):
    """FP64 one-sided Jacobi SVD of B = diag(nu) A_{Gamma_1} diag(sigma)^{-1/2}.
    Returns (U, S, V, sweeps) as CUDA float64 tensors."""
    import torch
    L = load()
    M_D, M_tot = int(counts.shape[0]), int(counts.shape[1])
    g1 = np.ascontiguousarray(gamma1, dtype=np.uint8)
    M_1 = int(g1.sum())
    k = min(M_D, M_1)
    dev = counts.device
    U = torch.empty((M_D, k), dtype=torch.float64, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    V = torch.empty((M_1, k), dtype=torch.float64, device=dev)
    sw = ctypes.c_int32(0)
    code = L.wos_op_svd(ctx.h, counts.data_ptr(), M_D, M_tot, int(N), g1.ctypes.data,
                        _ptr(nu), sigma.data_ptr(), U.data_ptr(), S.data_ptr(),
                        V.data_ptr(), ctypes.byref(sw) if sync else None,
                        _stream(stream))
    _check(code, "wos_op_svd", allow_warning=False)
    return U, S, V, int(sw.value)


def wos_op_svd_batched(ctx: Context, items, sync: bool = True, stream=None,
                       jacobi_events=None):
    """Many SVDs in one pass.  items: list of (counts, N, gamma1, sigma[, nu]).
    jacobi_events: optional pair of torch.cuda.Event recorded around the
    Jacobi launches.  Returns a list of (U, S, V, sweeps)."""
    import torch
    L = load()
    probs = (WosSvdProblem * len(items))()
    keep, out = [], []
    for q, it in enumerate(items):
        counts, N, gamma1, sigma = it[:4]
        nu = it[4] if len(it) > 4 else None
        M_D, M_tot = int(counts.shape[0]), int(counts.shape[1])
        g1 = np.ascontiguousarray(gamma1, dtype=np.uint8)
        M_1 = int(g1.sum())
        k = min(M_D, M_1)
        dev = counts.device
        U = torch.empty((M_D, k), dtype=torch.float64, device=dev)
        S = torch.empty(k, dtype=torch.float64, device=dev)
        V = torch.empty((M_1, k), dtype=torch.float64, device=dev)
        keep.append(g1)
        out.append([U, S, V, 0])
        pb = probs[q]
        pb.counts = counts.data_ptr()
        pb.M_D, pb.M_tot, pb.N = M_D, M_tot, int(N)
        pb.gamma1 = g1.ctypes.data
        pb.nu = _ptr(nu)
        pb.sigma = sigma.data_ptr()
        pb.U, pb.S, pb.V = U.data_ptr(), S.data_ptr(), V.data_ptr()
    sw = (ctypes.c_int32 * len(items))()
    evs = None
    if jacobi_events is not None:
        evs = (ctypes.c_void_p * 2)(jacobi_events[0].cuda_event, jacobi_events[1].cuda_event)
    code = L.wos_op_svd_batched(ctx.h, len(items), ctypes.byref(probs),
                                sw if sync else None, _stream(stream), evs)
    _check(code, "wos_op_svd_batched", allow_warning=False)
    for q in range(len(items)):
        out[q][3] = int(sw[q])
    return [tuple(o) for o in out]


def wos_reconstruct(ctx: Context, U, S, V, counts, N: int, gamma1: np.ndarray, sigma,
                    uD, r: int, u0=None, nu=None, tikhonov_alpha: float = 0.0,
                    want_uD_hat: bool = True, stream=None):
    """r-TSVD (or Tikhonov) Gamma_1 data; returns (u_gamma1, uD_hat)."""
    import torch
    L = load()
    M_D, M_tot = int(counts.shape[0]), int(counts.shape[1])
    g1 = np.ascontiguousarray(gamma1, dtype=np.uint8)
    M_1 = int(g1.sum())
    k = int(S.shape[0])
    dev = counts.device
    u1 = torch.empty(M_1, dtype=torch.float64, device=dev)
    uhat = torch.empty(M_D, dtype=torch.float64, device=dev) if want_uD_hat else None
    code = L.wos_reconstruct(ctx.h, U.data_ptr(), S.data_ptr(), V.data_ptr(), M_D, k,
                             counts.data_ptr(), M_tot, int(N), g1.ctypes.data, _ptr(nu),
                             sigma.data_ptr(), uD.data_ptr(), _ptr(u0), int(r),
                             float(tikhonov_alpha), u1.data_ptr(), _ptr(uhat),
                             _stream(stream))
    _check(code, "wos_reconstruct", allow_warning=False)
    return u1, uhat


def wos_spectral(ctx: Context, U, S, V, counts, N: int, gamma1: np.ndarray, sigma,
                 uD=None, u0=None, nu=None, r_max: int = 0, want_eigfun: bool = True,
                 stream=None) -> dict:
    """Spectral diagnostics (Sec. 5.2 items (i)-(iv)): lambda (k), eigfun
    (M_1 x k), density (M_1), and for r_max > 0 the TSVD family u_sweep
    (r_max x M_1) with its fitted interior data uD_sweep (r_max x M_D)."""
    import torch
    L = load()
    M_D, M_tot = int(counts.shape[0]), int(counts.shape[1])
    g1 = np.ascontiguousarray(gamma1, dtype=np.uint8)
    M_1 = int(g1.sum())
    k = int(S.shape[0])
    dev = counts.device
    f64 = dict(dtype=torch.float64, device=dev)
    out = dict(lambda_=torch.empty(k, **f64),
               eigfun=torch.empty((M_1, k), **f64) if want_eigfun else None,
               density=torch.empty(M_1, **f64))
    if r_max > 0:
        out["u_sweep"] = torch.empty((r_max, M_1), **f64)
        out["uD_sweep"] = torch.empty((r_max, M_D), **f64)
    code = L.wos_spectral(ctx.h, U.data_ptr(), S.data_ptr(), V.data_ptr(), M_D, k,
                          counts.data_ptr(), M_tot, int(N), g1.ctypes.data, _ptr(nu),
                          sigma.data_ptr(), _ptr(uD), _ptr(u0), int(r_max),
                          out["lambda_"].data_ptr(), _ptr(out["eigfun"]),
                          out["density"].data_ptr(), _ptr(out.get("u_sweep")),
                          _ptr(out.get("uD_sweep")), _stream(stream))
    _check(code, "wos_spectral", allow_warning=False)
    return out


def wos_truncation_gap(S: np.ndarray, r: int) -> bool:
    s = np.ascontiguousarray(S, dtype=np.float64)
    return load().wos_truncation_gap(s.ctypes.data, len(s), int(r)) == 0


# ---------------------------------------------------------------------------
# one instance end to end (the path timed by the benchmark)
# ---------------------------------------------------------------------------
@dataclass
class Solution:
    counts: object
    unterminated: object
    U: object
    S: object
    V: object
    u_gamma1: object
    uD_hat: object
    stats: dict | None
    sweeps: int


def solve_instance(ctx: Context, inst, uD, u0, r: int, points=None, sigma=None,
                   stats: bool = False, stream=None, opts: WosOpts | None = None,
                   sync_svd: bool = False) -> Solution:
    """Operator build + SVD + TSVD for one workloads.Instance (device inputs:
    uD (M_D), u0 (M_0) as CUDA float64 tensors)."""
    import torch
    dev = uD.device
    if points is None:
        points = torch.as_tensor(inst.points, dtype=torch.float64, device=dev)
    if sigma is None:
        sigma = torch.as_tensor(wos_element_measures(inst.domain, inst.partition),
                                dtype=torch.float64, device=dev)
    if opts is None:
        opts = make_opts(precision=1 if inst.fp64 else 0, stream_id=inst.stream,
                         step_cap=inst.step_cap, mapped=getattr(inst, "mapped", False))
    counts, unterm, st = wos_build_operator(ctx, inst.domain, inst.K, points,
                                            inst.partition, inst.N, inst.eps, inst.seed,
                                            opts=opts, stats=stats, stream=stream)
    U, S, V, sw = wos_op_svd(ctx, counts, inst.N, inst.partition.gamma1, sigma,
                             sync=sync_svd, stream=stream)
    u1, uhat = wos_reconstruct(ctx, U, S, V, counts, inst.N, inst.partition.gamma1,
                               sigma, uD, r, u0=u0, stream=stream)
    return Solution(counts, unterm, U, S, V, u1, uhat, st, sw)


# ---------------------------------------------------------------------------
# serving: request queue with continuous batching
# ---------------------------------------------------------------------------
@dataclass
class Ticket:
    id: int
    u_gamma1: np.ndarray
    S: np.ndarray
    counts: np.ndarray | None
    r_used: ctypes.c_int32
    keep: list


def wos_queue_create(ctx: Context, seed: int, precision: int = 0, max_inflight: int = 0,
                     device_budget: int = 0, slice_walks: int = 0,
                     side_streams: int = 0) -> ctypes.c_void_p:
    o = WosQueueOpts(int(max_inflight), int(device_budget), int(slice_walks),
                     int(precision), int(seed), int(side_streams))
    h = ctypes.c_void_p()
    _check(load().wos_queue_create(ctx.h, ctypes.byref(o), ctypes.byref(h)),
           "wos_queue_create", False)
    return h


def wos_queue_destroy(q) -> None:
    _check(load().wos_queue_destroy(q), "wos_queue_destroy", False)


def wos_submit(q, inst, uD: np.ndarray, u0: np.ndarray | None = None, r: int = 0,
               tikhonov_alpha: float = 0.0, nu: np.ndarray | None = None,
               want_counts: bool = False) -> Ticket:
    """Queues one workloads.Instance end to end (host inputs; outputs land in
    the returned Ticket's host arrays once the request completes)."""
    L = load()
    D = make_domain(inst.domain)
    P, kp = make_partition(inst.domain, inst.partition)
    Kc = np.ascontiguousarray(inst.K, dtype=np.float64)
    pts = np.ascontiguousarray(inst.points, dtype=np.float64)
    g1 = np.ascontiguousarray(inst.partition.gamma1, dtype=np.uint8)
    M_tot, M_1 = int(g1.size), int(g1.sum())
    k = min(inst.M_D, M_1)
    uDc = np.ascontiguousarray(uD, dtype=np.float64)
    u0c = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    nuc = None if nu is None else np.ascontiguousarray(nu, dtype=np.float64)
    u1 = np.zeros(M_1)
    S = np.zeros(k)
    cnt = np.zeros((inst.M_D, M_tot), dtype=np.uint32) if want_counts else None
    r_used = ctypes.c_int32(0)
    rq = WosRequest()
    rq.domain = ctypes.addressof(D)
    rq.partition = ctypes.addressof(P)
    rq.gamma1 = g1.ctypes.data
    rq.K = Kc.ctypes.data
    rq.points = pts.ctypes.data
    rq.M_D = inst.M_D
    rq.N = int(inst.N)
    rq.eps = float(inst.eps)
    rq.stream_id = int(inst.stream)
    rq.nu = None if nuc is None else nuc.ctypes.data
    rq.uD = uDc.ctypes.data
    rq.u0 = None if u0c is None else u0c.ctypes.data
    rq.r = int(r)
    rq.tikhonov_alpha = float(tikhonov_alpha)
    rq.u_gamma1 = u1.ctypes.data
    rq.S = S.ctypes.data
    rq.counts = None if cnt is None else cnt.ctypes.data
    rq.r_used = ctypes.addressof(r_used)
    t = ctypes.c_uint64(0)
    _check(L.wos_submit(q, ctypes.byref(rq), ctypes.byref(t)), "wos_submit", False)
    return Ticket(int(t.value), u1, S, cnt, r_used, [D, P, kp, rq])


def wos_poll(q, ticket: Ticket) -> bool:
    code = load().wos_poll(q, ticket.id)
    if code == 12:
        return False
    _check(code, "wos_poll", False)
    return True


def wos_wait(q, ticket: Ticket, timeout_ms: int = -1) -> bool:
    code = load().wos_wait(q, ticket.id, int(timeout_ms))
    if code == 12:
        return False
    _check(code, "wos_wait", False)
    return True


def wos_queue_get_stats(q) -> dict:
    st = WosQueueStats()
    _check(load().wos_queue_get_stats(q, ctypes.byref(st)), "wos_queue_get_stats", False)
    return st.as_dict()
