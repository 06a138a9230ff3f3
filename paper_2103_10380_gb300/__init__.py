"""Python binding of libfnr (FastNeRF cached rendering on GB300).

Argument marshalling only: every step of the render path runs in libfnr's CUDA
kernels. The names mirror the C ABI in include/fnr.h. PyTorch is used for
device memory and streams. There is no CPU fallback: importing the binding
without a built libfnr.so raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfnr.so")

FNR_OK = 0
FNR_ERR_INVALID_ARG = 1
FNR_ERR_UNSUPPORTED = 2
FNR_ERR_OOM = 3
FNR_ERR_BUDGET = 4
FNR_ERR_QUEUE_FULL = 5
FNR_ERR_NOT_READY = 6
FNR_ERR_TIMEOUT = 7
FNR_ERR_CUDA = 8
FNR_ERR_DEVICE = 9
FNR_ERR_IO = 10

FNR_PREC_FP32 = 0
FNR_PREC_FP16 = 1
FNR_PREC_FP8_E4M3 = 2
FNR_ACT_SIGMOID = 0
FNR_ACT_IDENTITY = 1
FNR_RENDER_SKIP_EMPTY = 1
FNR_RENDER_DIR_BILINEAR = 2
FNR_RENDER_VOXELS = 4
FNR_LAYOUT_DENSE = 0
FNR_LAYOUT_BRICKS = 1
FNR_SRC_ARRAYS = 1
FNR_SRC_MLP = 2
FNR_LOC_HOST = 0
FNR_LOC_DEVICE = 1

_STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "BUDGET", 5: "QUEUE_FULL",
                 6: "NOT_READY", 7: "TIMEOUT", 8: "CUDA", 9: "DEVICE", 10: "IO"}


class FnrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fnr status {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fnr_cache_desc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("D", ctypes.c_int32), ("l", ctypes.c_int32),
                ("pos_precision", ctypes.c_int32), ("dir_precision", ctypes.c_int32),
                ("occupancy_brick", ctypes.c_int32), ("layout", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("bmin", ctypes.c_float * 3), ("bmax", ctypes.c_float * 3)]


class fnr_mlp(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("pe_in", ctypes.c_int32), ("pe_freqs", ctypes.c_int32),
                ("dims", ctypes.c_int32 * 17), ("weights", ctypes.c_void_p * 16), ("biases", ctypes.c_void_p * 16)]


class fnr_cache_source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("location", ctypes.c_int32), ("sigma", ctypes.c_void_p),
                ("uvw", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("pos_mlp", ctypes.c_void_p),
                ("dir_mlp", ctypes.c_void_p)]


class fnr_cache_layout(ctypes.Structure):
    _fields_ = [("sigma_dev", ctypes.c_void_p), ("uvw_dev", ctypes.c_void_p), ("beta_dev", ctypes.c_void_p),
                ("scales_dev", ctypes.c_void_p), ("cos_theta_dev", ctypes.c_void_p),
                ("phi_key_dev", ctypes.c_void_p), ("occupancy_dev", ctypes.c_void_p),
                ("record_stride", ctypes.c_int32), ("occupancy_brick", ctypes.c_int32), ("footprint", ctypes.c_uint64),
                ("layout", ctypes.c_int32), ("reserved1", ctypes.c_int32), ("page_table_dev", ctypes.c_void_p),
                ("n_bricks", ctypes.c_uint64), ("brick_distance_dev", ctypes.c_void_p),
                ("distance_brick", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("offsets_dev", ctypes.c_void_p), ("offset_brick", ctypes.c_int32), ("offset_stride", ctypes.c_int32)]


class fnr_camera(ctypes.Structure):
    _fields_ = [("c2w", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class fnr_render_params(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int32), ("t_near", ctypes.c_float), ("t_far", ctypes.c_float),
                ("t_thr", ctypes.c_float), ("bg", ctypes.c_float * 3), ("activation", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class fnr_ray_stats(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("n_lookups", ctypes.c_int32), ("n_occupied", ctypes.c_int32),
                ("dir_cell", ctypes.c_int32)]


class fnr_request(ctypes.Structure):
    _fields_ = [("cache", ctypes.c_void_p), ("camera", fnr_camera), ("params", fnr_render_params),
                ("rgba_dev", ctypes.c_void_p), ("stats_dev", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("priority", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fnr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t_submit_ns", ctypes.c_uint64),
                ("t_admit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64), ("n_rays", ctypes.c_uint64),
                ("batch", ctypes.c_int64), ("ticket", ctypes.c_uint64)]


class fnr_serve_config(ctypes.Structure):
    _fields_ = [("queue_capacity", ctypes.c_int32), ("max_batch_requests", ctypes.c_int32),
                ("max_batch_rays", ctypes.c_int64), ("n_slots", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("idle_spin_us", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# Every symbol include/fnr.h declares, with (argtypes, restype).
_P = ctypes.c_void_p
SIGNATURES = {
    "fnr_context_create": ([ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_P)], ctypes.c_int32),
    "fnr_context_destroy": ([_P], ctypes.c_int32),
    "fnr_context_used_bytes": ([_P], ctypes.c_uint64),
    "fnr_last_error": ([], ctypes.c_char_p),
    "fnr_cache_bytes": ([ctypes.POINTER(fnr_cache_desc)], ctypes.c_uint64),
    "fnr_cache_footprint": ([ctypes.POINTER(fnr_cache_desc)], ctypes.c_uint64),
    "fnr_build_cache": ([_P, ctypes.POINTER(fnr_cache_desc), ctypes.POINTER(fnr_cache_source), _P,
                         ctypes.POINTER(_P)], ctypes.c_int32),
    "fnr_cache_free": ([_P, _P], ctypes.c_int32),
    "fnr_cache_get_layout": ([_P, ctypes.POINTER(fnr_cache_layout)], ctypes.c_int32),
    "fnr_cache_save": ([_P, ctypes.c_char_p], ctypes.c_int32),
    "fnr_render_mlp": ([_P, _P, _P, ctypes.c_int32, _P, _P, ctypes.POINTER(fnr_camera),
                        ctypes.POINTER(fnr_render_params), _P, _P, _P], ctypes.c_int32),
    "fnr_cache_load": ([_P, ctypes.c_char_p, _P, ctypes.POINTER(_P)], ctypes.c_int32),
    "fnr_render": ([_P, _P, ctypes.POINTER(fnr_camera), ctypes.c_int32, ctypes.POINTER(fnr_render_params), _P, _P,
                    _P, _P], ctypes.c_int32),
    "fnr_serve_start": ([_P, ctypes.POINTER(fnr_serve_config)], ctypes.c_int32),
    "fnr_serve_stop": ([_P], ctypes.c_int32),
    "fnr_submit": ([_P, ctypes.POINTER(fnr_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int32),
    "fnr_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(fnr_result)], ctypes.c_int32),
    "fnr_wait": ([_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(fnr_result)], ctypes.c_int32),
    "fnr_render_noalloc": ([_P, ctypes.POINTER(fnr_camera), ctypes.c_int32, ctypes.POINTER(fnr_render_params), _P,
                            _P, _P, _P], ctypes.c_int32),
    "fnr_testing_fail_allocations": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_int32),
    "fnr_testing_mlp_fault": ([ctypes.c_int64, ctypes.c_int64], ctypes.c_int32),
    "fnr_testing_mlp_cta_pair": ([ctypes.c_int32], ctypes.c_int32),
}

_lib = None


def lib():
    """Load libfnr.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfnr.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status: int):
    if status != FNR_OK:
        raise FnrError(status, lib().fnr_last_error().decode(errors="replace"))


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream) or None


# ------------------------------------------------------------------ thin wrappers (same names as the C ABI)
def fnr_context_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    out = _P()
    check(lib().fnr_context_create(device, hbm_budget_bytes, ctypes.byref(out)))
    return out.value


def fnr_context_destroy(ctx: int):
    check(lib().fnr_context_destroy(ctx))


def fnr_context_used_bytes(ctx: int) -> int:
    return lib().fnr_context_used_bytes(ctx)


def make_desc(k, D, l, pos_precision=FNR_PREC_FP32, dir_precision=FNR_PREC_FP32, bmin=(-1.5, -1.5, -1.5),
              bmax=(1.5, 1.5, 1.5), occupancy_brick=0, layout=FNR_LAYOUT_DENSE) -> fnr_cache_desc:
    d = fnr_cache_desc()
    d.k, d.D, d.l = k, D, l
    d.pos_precision, d.dir_precision = pos_precision, dir_precision
    d.occupancy_brick = int(occupancy_brick)
    d.layout = int(layout)
    d.bmin[:] = [float(v) for v in bmin]
    d.bmax[:] = [float(v) for v in bmax]
    return d


def fnr_cache_bytes(desc: fnr_cache_desc) -> int:
    return lib().fnr_cache_bytes(ctypes.byref(desc))


def fnr_cache_footprint(desc: fnr_cache_desc) -> int:
    return lib().fnr_cache_footprint(ctypes.byref(desc))


def fnr_build_cache(ctx: int, desc: fnr_cache_desc, sigma, uvw, beta, stream=None) -> int:
    """sigma/uvw/beta: float32 arrays (numpy: host source; torch CUDA tensors: device source)."""
    src = fnr_cache_source()
    src.kind = FNR_SRC_ARRAYS
    arrs = (sigma, uvw, beta)
    if all(hasattr(a, "is_cuda") and a.is_cuda for a in arrs):
        for a in arrs:
            assert a.is_contiguous() and str(a.dtype) == "torch.float32"
        src.location = FNR_LOC_DEVICE
        src.sigma, src.uvw, src.beta = (a.data_ptr() for a in arrs)
    else:
        import numpy as np
        for a in arrs:
            assert isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous
        src.location = FNR_LOC_HOST
        src.sigma, src.uvw, src.beta = (a.ctypes.data for a in arrs)
    out = _P()
    check(lib().fnr_build_cache(ctx, ctypes.byref(desc), ctypes.byref(src), _stream_handle(stream),
                                ctypes.byref(out)))
    return out.value


def make_mlp(layers, pe_freqs: int) -> fnr_mlp:
    """layers: [(W, b)] with W a CUDA tensor of bf16 bits [out][in] (int16/uint16/bfloat16), b float32 [out]."""
    m = fnr_mlp()
    m.n_layers = len(layers)
    m.pe_in = 3
    m.pe_freqs = pe_freqs
    dims = [int(layers[0][0].shape[1])] + [int(W.shape[0]) for W, _ in layers]
    for i, d in enumerate(dims):
        m.dims[i] = d
    for i, (W, b) in enumerate(layers):
        assert W.is_cuda and W.is_contiguous() and W.element_size() == 2
        assert b.is_cuda and b.is_contiguous() and str(b.dtype) == "torch.float32"
        m.weights[i] = W.data_ptr()
        m.biases[i] = b.data_ptr()
    return m


def fnr_build_cache_mlp(ctx: int, desc: fnr_cache_desc, pos_layers, dir_layers, pos_freqs: int = 10,
                        dir_freqs: int = 4, stream=None) -> int:
    """Build a cache by evaluating F_pos over the k^3 cell centres and F_dir over the l x l bin centres."""
    pm, dm = make_mlp(pos_layers, pos_freqs), make_mlp(dir_layers, dir_freqs)
    src = fnr_cache_source()
    src.kind = FNR_SRC_MLP
    src.pos_mlp = ctypes.addressof(pm)
    src.dir_mlp = ctypes.addressof(dm)
    out = _P()
    check(lib().fnr_build_cache(ctx, ctypes.byref(desc), ctypes.byref(src), _stream_handle(stream),
                                ctypes.byref(out)))
    return out.value


def fnr_render_mlp(ctx: int, pos_layers, dir_layers, D: int, cam, params: fnr_render_params, rgba, stats=None,
                   bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5), pos_freqs: int = 10, dir_freqs: int = 4,
                   stream=None):
    """The uncached render of one view: F_pos at every inside sample, F_dir per ray, Eq. 5 + Eq. 1."""
    pm, dm = make_mlp(pos_layers, pos_freqs), make_mlp(dir_layers, dir_freqs)
    c = cam if isinstance(cam, fnr_camera) else make_camera(cam)
    lo = (ctypes.c_float * 3)(*[float(v) for v in bmin])
    hi = (ctypes.c_float * 3)(*[float(v) for v in bmax])
    assert rgba.is_cuda and rgba.is_contiguous() and rgba.numel() >= 4 * c.width * c.height
    check(lib().fnr_render_mlp(ctx, ctypes.addressof(pm), ctypes.addressof(dm), int(D), ctypes.addressof(lo),
                               ctypes.addressof(hi), ctypes.byref(c), ctypes.byref(params), rgba.data_ptr(),
                               None if stats is None else stats.data_ptr(), _stream_handle(stream)))


def fnr_cache_free(ctx: int, cache: int):
    check(lib().fnr_cache_free(ctx, cache))


def fnr_cache_get_layout(cache: int) -> fnr_cache_layout:
    out = fnr_cache_layout()
    check(lib().fnr_cache_get_layout(cache, ctypes.byref(out)))
    return out


def fnr_cache_save(cache: int, path) -> None:
    check(lib().fnr_cache_save(cache, os.fsencode(path)))


def fnr_cache_load(ctx: int, path, stream=None) -> int:
    out = _P()
    check(lib().fnr_cache_load(ctx, os.fsencode(path), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def make_camera(cam: dict) -> fnr_camera:
    c = fnr_camera()
    c.c2w[:] = [float(v) for v in cam["c2w"]]
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["W"]), int(cam["H"])
    return c


def make_params(n_samples, t_near=2.0, t_far=6.0, t_thr=1e-4, bg=(1.0, 1.0, 1.0),
                activation=FNR_ACT_SIGMOID, skip_empty=False, dir_bilinear=False, voxels=False) -> fnr_render_params:
    """voxels: walk every cell the ray passes through (n_samples caps the walk; 3k covers any ray)."""
    p = fnr_render_params()
    p.n_samples, p.t_near, p.t_far, p.t_thr = int(n_samples), float(t_near), float(t_far), float(t_thr)
    p.bg[:] = [float(v) for v in bg]
    p.activation = int(activation)
    p.flags = ((FNR_RENDER_SKIP_EMPTY if skip_empty else 0) | (FNR_RENDER_DIR_BILINEAR if dir_bilinear else 0)
               | (FNR_RENDER_VOXELS if voxels else 0))
    return p


def fnr_render(ctx: int, cache: int, cams, params: fnr_render_params, rgba, stats=None, cells=None, stream=None):
    """cams: list of dicts or fnr_camera; rgba/stats/cells: CUDA tensors (caller-owned)."""
    cams = [c if isinstance(c, fnr_camera) else make_camera(c) for c in cams]
    arr = (fnr_camera * len(cams))(*cams)
    npix = sum(c.width * c.height for c in cams)
    assert rgba.is_cuda and rgba.is_contiguous() and rgba.numel() >= 4 * npix
    if stats is not None:
        assert stats.is_cuda and stats.is_contiguous() and stats.numel() >= 4 * npix
    if cells is not None:
        assert cells.is_cuda and cells.is_contiguous() and cells.numel() >= npix * params.n_samples
    check(lib().fnr_render(ctx, cache, arr, len(cams), ctypes.byref(params), rgba.data_ptr(),
                           None if stats is None else stats.data_ptr(), None if cells is None else cells.data_ptr(),
                           _stream_handle(stream)))


# ------------------------------------------------------------------ serving
def fnr_serve_start(ctx: int, queue_capacity=0, max_batch_requests=0, max_batch_rays=0, n_slots=0,
                    use_graphs=1, idle_spin_us=0):
    """idle_spin_us: how long the scheduler keeps polling after its last event (0: 5 ms; -1: always)."""
    cfg = fnr_serve_config(queue_capacity, max_batch_requests, max_batch_rays, n_slots, use_graphs, idle_spin_us, 0)
    check(lib().fnr_serve_start(ctx, ctypes.byref(cfg)))


def fnr_serve_stop(ctx: int):
    check(lib().fnr_serve_stop(ctx))


def make_request(cache: int, cam, params: fnr_render_params, rgba, stats=None, stream=None) -> fnr_request:
    """stream: the stream that produced rgba/stats (default: torch's current stream)."""
    r = fnr_request()
    r.cache = cache
    r.camera = cam if isinstance(cam, fnr_camera) else make_camera(cam)
    r.params = params
    assert rgba.is_cuda and rgba.is_contiguous() and rgba.numel() >= 4 * r.camera.width * r.camera.height
    r.rgba_dev = rgba.data_ptr()
    r.stats_dev = None if stats is None else stats.data_ptr()
    r.stream = _stream_handle(stream)
    return r


def fnr_submit(ctx: int, req: fnr_request) -> int:
    t = ctypes.c_uint64()
    check(lib().fnr_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def fnr_poll(ctx: int, ticket: int):
    """Returns fnr_result when done, None while queued or in flight."""
    out = fnr_result()
    st = lib().fnr_poll(ctx, ticket, ctypes.byref(out))
    if st == FNR_ERR_NOT_READY:
        return None
    check(st)
    return out


def fnr_wait(ctx: int, ticket: int, timeout_ms: int = 10000) -> fnr_result:
    out = fnr_result()
    check(lib().fnr_wait(ctx, ticket, timeout_ms, ctypes.byref(out)))
    return out


# ------------------------------------------------------------------ rendering without allocation
def fnr_render_noalloc(cache: int, cams, params: fnr_render_params, rgba, stats=None, done_words=None,
                       stream=None):
    """Render up to 32 views with the persistent kernel whose scratch is a static device array (for callers
    that cannot allocate device memory). Same output layout as fnr_render."""
    cams = [c if isinstance(c, fnr_camera) else make_camera(c) for c in cams]
    arr = (fnr_camera * len(cams))(*cams)
    npix = sum(c.width * c.height for c in cams)
    assert rgba.is_cuda and rgba.is_contiguous() and rgba.numel() >= 4 * npix
    if stats is not None:
        assert stats.is_cuda and stats.is_contiguous() and stats.numel() >= 4 * npix
    check(lib().fnr_render_noalloc(cache, arr, len(cams), ctypes.byref(params), rgba.data_ptr(),
                                   None if stats is None else stats.data_ptr(),
                                   None if done_words is None else done_words.data_ptr(), _stream_handle(stream)))


# ------------------------------------------------------------------ failure injection (fnr_testing.h; tests only)
def fnr_testing_fail_allocations(skip: int, count: int) -> None:
    """The library's next `skip` device allocations succeed and the `count` after them fail (0 disarms)."""
    check(lib().fnr_testing_fail_allocations(int(skip), int(count)))


def fnr_testing_mlp_fault(wait_limit: int, withhold_chunk: int = -1) -> None:
    """The next tensor-core build launch gives up its waits after wait_limit polls and, if withhold_chunk >= 0,
    each CTA's producer withholds that weight chunk; the call then returns FNR_ERR_DEVICE."""
    check(lib().fnr_testing_mlp_fault(int(wait_limit), int(withhold_chunk)))


def fnr_testing_mlp_cta_pair(on: bool) -> None:
    """Builds that follow use the CTA-pair form of the tensor-core kernel (on) or the default single-CTA form."""
    check(lib().fnr_testing_mlp_cta_pair(1 if on else 0))
