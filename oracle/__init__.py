"""FP64 CPU oracle for the FastNeRF cached rendering path (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg. The renderer package never imports it, and it
shares no code with the renderer. What each function follows in the paper is
stated in oracle.c.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

FP32, FP16, FP8 = 0, 1, 2
ACT_SIGMOID, ACT_IDENTITY = 0, 1

FIELD_FN = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class _Cache(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("D", ctypes.c_int32), ("l", ctypes.c_int32),
                ("bmin", ctypes.c_float * 3), ("bmax", ctypes.c_float * 3),
                ("pos_prec", ctypes.c_int32), ("dir_prec", ctypes.c_int32),
                ("sigma", ctypes.c_void_p), ("uvw", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("scales", ctypes.c_void_p), ("field", ctypes.c_void_p), ("field_user", ctypes.c_void_p),
                ("occ", ctypes.c_void_p), ("occ_brick", ctypes.c_int32), ("off_brick", ctypes.c_int32),
                ("offsets", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("c2w", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("W", ctypes.c_int32), ("H", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("t_near", ctypes.c_float), ("t_far", ctypes.c_float),
                ("t_thr", ctypes.c_float), ("bg", ctypes.c_float * 3), ("act", ctypes.c_int32),
                ("skip_empty", ctypes.c_int32), ("dir_bilinear", ctypes.c_int32), ("voxels", ctypes.c_int32)]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
                               "-fPIC", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        L.orc_render_pixels.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P, ctypes.c_int]
        L.orc_render_pixels.restype = ctypes.c_int
        L.orc_f16_decode.argtypes = [ctypes.c_uint16]; L.orc_f16_decode.restype = ctypes.c_double
        L.orc_f16_encode.argtypes = [ctypes.c_float]; L.orc_f16_encode.restype = ctypes.c_uint16
        L.orc_e4m3_decode.argtypes = [ctypes.c_uint8]; L.orc_e4m3_decode.restype = ctypes.c_double
        L.orc_e4m3_encode.argtypes = [ctypes.c_float]; L.orc_e4m3_encode.restype = ctypes.c_uint8
        L.orc_fp8_scale.argtypes = [ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int]
        L.orc_fp8_scale.restype = ctypes.c_float
        L.orc_quantize.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int, ctypes.c_float, P]
        L.orc_quantize.restype = None
        L.orc_fp8_offsets.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
        L.orc_fp8_offsets.restype = None
        L.orc_fp8_uvw_scale.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int]
        L.orc_fp8_uvw_scale.restype = ctypes.c_float
        L.orc_fp8_uvw_quantize.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P]
        L.orc_fp8_uvw_quantize.restype = None
        for f in ("orc_bytes_nerf",):
            getattr(L, f).argtypes = [ctypes.c_uint64] * 4
            getattr(L, f).restype = ctypes.c_uint64
        L.orc_bytes_fastnerf_pos.argtypes = [ctypes.c_uint64] * 4
        L.orc_bytes_fastnerf_pos.restype = ctypes.c_uint64
        L.orc_bytes_fastnerf_dir.argtypes = [ctypes.c_uint64] * 3
        L.orc_bytes_fastnerf_dir.restype = ctypes.c_uint64
        L.orc_ray.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P]
        L.orc_ray.restype = None
        L.orc_voxel_walk.argtypes = [ctypes.c_int32, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_int32, P, P]
        L.orc_voxel_walk.restype = ctypes.c_int32
        L.orc_phi_key.argtypes = [ctypes.c_float, ctypes.c_float]; L.orc_phi_key.restype = ctypes.c_float
        L.orc_dir_cell.argtypes = [ctypes.c_int, P, P, P]; L.orc_dir_cell.restype = None
        L.orc_dt.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int32]; L.orc_dt.restype = ctypes.c_float
        L.orc_s_thr.argtypes = [ctypes.c_float, ctypes.c_float]; L.orc_s_thr.restype = ctypes.c_int64
        L.orc_fix.argtypes = [ctypes.c_double]; L.orc_fix.restype = ctypes.c_int64
        L.orc_round_bf16.argtypes = [ctypes.c_double]; L.orc_round_bf16.restype = ctypes.c_double
        L.orc_trace_fp64.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P]
        L.orc_trace_fp64.restype = None
        L.orc_posenc.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P]
        L.orc_posenc.restype = None
        L.orc_mlp_forward.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int64, P, P, ctypes.c_int]
        L.orc_mlp_forward.restype = ctypes.c_int
        L.orc_table_field.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P]
        L.orc_beta_bilinear.argtypes = [P, P, P]
        L.orc_beta_bilinear.restype = None
        L.orc_mlp_samples.argtypes = [P, P, P, P, ctypes.c_int64, P, P, P, P, P]
        L.orc_mlp_samples.restype = None
        L.orc_table_field.restype = None
        _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _nthreads(n):
    return int(n) if n else max(1, os.cpu_count() or 1)


# ------------------------------------------------------------------ structs
class Cache:
    """A cache as the oracle reads it: stored arrays (dense, unpadded) plus metadata.

    sigma: [k^3] (float32 / uint16 FP16 bits / uint8 E4M3 codes), index (z*k + y)*k + x;
    uvw: [k^3, 3D] same dtype, channels u_1..u_D, v_1..v_D, w_1..w_D;
    beta: [l, l, D] float32 or uint16 FP16 bits, index [i_theta][i_phi];
    scales: float32 [1 + 3D] for FP8 (sigma first).
    offsets: FP8 only, uint16 binary16 bits [nbo^3, 3D] of the (u, v, w) offsets per offset brick of
    off_brick cells a side.
    field: optional (ctypes function pointer, user pointer) FP64 cell accessor
    that replaces sigma/uvw.
    """

    def __init__(self, k, D, l, sigma, uvw, beta, pos_prec=FP32, dir_prec=FP32, scales=None,
                 bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5), field=None, offsets=None, off_brick=0):
        self.k, self.D, self.l = int(k), int(D), int(l)
        self.pos_prec, self.dir_prec = pos_prec, dir_prec
        self.sigma = None if sigma is None else np.ascontiguousarray(sigma).reshape(-1)
        self.uvw = None if uvw is None else np.ascontiguousarray(uvw).reshape(-1)
        self.beta = np.ascontiguousarray(beta).reshape(-1)
        self.scales = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
        self.bmin, self.bmax = tuple(bmin), tuple(bmax)
        self.field = field
        s = _Cache()
        s.k, s.D, s.l = self.k, self.D, self.l
        s.bmin[:] = [float(v) for v in self.bmin]
        s.bmax[:] = [float(v) for v in self.bmax]
        s.pos_prec, s.dir_prec = pos_prec, dir_prec
        s.sigma = None if self.sigma is None else self.sigma.ctypes.data
        s.uvw = None if self.uvw is None else self.uvw.ctypes.data
        s.beta = self.beta.ctypes.data
        s.scales = None if self.scales is None else self.scales.ctypes.data
        self.offsets = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.uint16).reshape(-1)
        self.off_brick = int(off_brick)
        s.offsets = None if self.offsets is None else self.offsets.ctypes.data
        s.off_brick = self.off_brick
        if field is not None:
            fn, user = field
            s.field = ctypes.cast(fn, ctypes.c_void_p).value
            s.field_user = user
        self.occ = None
        self._s = s

    def set_occupancy(self, brick: int, positive: np.ndarray | None = None):
        """Brick occupancy for skip_empty renders: from the stored densities (positive_density), or from a
        given boolean [k^3] array of "sigma > 0" (e.g. for a tabled render)."""
        if positive is None:
            positive = positive_density(self)
        self.occ = brick_occupancy(self.k, int(brick), positive)
        self._s.occ = self.occ.ctypes.data
        self._s.occ_brick = int(brick)
        return self


def positive_density(cache: "Cache") -> np.ndarray:
    """bool [k^3]: the stored density, dequantised as the oracle reads it, is > 0."""
    s = cache.sigma
    if cache.pos_prec == FP16:
        h = s.view(np.uint16)
        return ((h & 0x8000) == 0) & ((h & 0x7FFF) != 0) & ((h & 0x7FFF) <= 0x7C00)
    if cache.pos_prec == FP8:
        table = e4m3_decode(np.arange(256)).astype(np.float32)
        vals = table[s.view(np.uint8)] * np.float32(cache.scales[0])  # binary32 product
        return vals > 0.0
    return s.view(np.float32) > 0.0


def brick_occupancy(k: int, B: int, positive: np.ndarray) -> np.ndarray:
    """uint8 [nb^3], nb = ceil(k / B): brick (bz, by, bx) -- the cells [bx B, bx B + B) x [by B, ...) x
    [bz B, ...) clipped to the grid -- is 1 iff one of its cells has sigma > 0. Index (bz nb + by) nb + bx."""
    nb = (k + B - 1) // B
    pos = np.asarray(positive, dtype=bool).reshape(k, k, k)
    pad = np.zeros((nb * B,) * 3, dtype=bool)
    pad[:k, :k, :k] = pos
    return np.ascontiguousarray(pad.reshape(nb, B, nb, B, nb, B).any(axis=(1, 3, 5)).astype(np.uint8).reshape(-1))


def camera_struct(cam: dict) -> _Camera:
    c = _Camera()
    c.c2w[:] = [float(v) for v in np.asarray(cam["c2w"], dtype=np.float32).reshape(12)]
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.W, c.H = int(cam["W"]), int(cam["H"])
    return c


def params_struct(N, t_near=2.0, t_far=6.0, t_thr=1e-4, bg=(1.0, 1.0, 1.0), act=ACT_SIGMOID,
                  skip_empty=False, dir_bilinear=False, voxels=False) -> _Params:
    p = _Params()
    p.N, p.t_near, p.t_far, p.t_thr = int(N), float(t_near), float(t_far), float(t_thr)
    p.bg[:] = [float(v) for v in bg]
    p.act = int(act)
    p.skip_empty = 1 if skip_empty else 0
    p.dir_bilinear = 1 if dir_bilinear else 0
    p.voxels = 1 if voxels else 0
    return p


def grid_scale(k, bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5)) -> np.ndarray:
    """s_a = k / (bmax_a - bmin_a) rounded to binary32, as the oracle's renderer uses it."""
    return np.array([np.float32(float(k) / (float(b1) - float(b0))) for b0, b1 in zip(bmin, bmax)], dtype=np.float32)


def voxel_walk(k, o, d, t_near, t_far, max_steps, bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5)):
    """The cells a ray passes through (Section 4's voxel traversal) and its length inside each:
    (cells int32 [n], delta float32 [n]) -- the walk orc_voxel_walk defines."""
    cells = np.zeros(max_steps, dtype=np.int32)
    delta = np.zeros(max_steps, dtype=np.float32)
    b = np.ascontiguousarray(bmin, dtype=np.float32)
    sc = grid_scale(k, bmin, bmax)
    o = np.ascontiguousarray(o, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    n = lib().orc_voxel_walk(int(k), _p(b), _p(sc), _p(o), _p(d), float(t_near), float(t_far), int(max_steps),
                             _p(cells), _p(delta))
    return cells[:n].copy(), delta[:n].copy()


# ------------------------------------------------------------------ rendering
def render_pixels(cache: Cache, cam: dict, params: _Params, px, py, want_cells=False, nthreads=None):
    """Render listed pixels. Returns (rgba [n,4] f64, stats [n,4] i32, cells [n,N] i32 or None)."""
    px = np.ascontiguousarray(px, dtype=np.int32).reshape(-1)
    py = np.ascontiguousarray(py, dtype=np.int32).reshape(-1)
    n = px.size
    rgba = np.zeros((n, 4))
    stats = np.zeros((n, 4), dtype=np.int32)
    cells = np.zeros((n, params.N), dtype=np.int32) if want_cells else None
    cs = camera_struct(cam)
    rc = lib().orc_render_pixels(ctypes.byref(cache._s), ctypes.byref(cs), ctypes.byref(params), n, _p(px), _p(py),
                                 _p(rgba), _p(stats), _p(cells), _nthreads(nthreads))
    if rc != 0:
        raise ValueError("orc_render_pixels rejected its arguments")
    return rgba, stats, cells


class _Table(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_void_p), ("n", ctypes.c_int64), ("cells", ctypes.c_void_p),
                ("rec", ctypes.c_void_p), ("nch", ctypes.c_int32), ("missing", ctypes.c_int64)]


def render_pixels_tabled(k, D, l, sigma, beta, records, cam: dict, params: _Params, px, py, nthreads=None,
                         bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5)):
    """render_pixels for an FP32 grid whose uvw channels are too large to hold densely.

    sigma: dense float32 [k^3]; beta: float32 [l, l, D]; records(cells) -> float32 [n, 3D], the uvw
    values of the given ascending int64 cells (e.g. the scene generator evaluated at their centres).
    First pass: the cells the rays shade (they depend on sigma alone). Second pass: the render with
    those records. Returns (rgba [n,4] f64, stats [n,4] i32, number of distinct shaded cells).
    """
    sigma = np.ascontiguousarray(sigma, dtype=np.float32).reshape(-1)
    assert sigma.size == k ** 3
    L = lib()
    fn = ctypes.cast(L.orc_table_field, ctypes.c_void_p).value
    t = _Table()
    t.sigma, t.n, t.cells, t.rec, t.nch, t.missing = sigma.ctypes.data, 0, None, None, 3 * D, 0
    c = Cache(k, D, l, None, None, beta, bmin=bmin, bmax=bmax, field=(fn, ctypes.addressof(t)))
    _, _, cells = render_pixels(c, cam, params, px, py, want_cells=True, nthreads=nthreads)
    cells = cells.reshape(-1)
    cells = cells[cells >= 0].astype(np.int64)
    cells = np.unique(cells[sigma[cells] > 0.0])
    rec = np.ascontiguousarray(records(cells), dtype=np.float32).reshape(cells.size, 3 * D)
    t.n, t.cells, t.rec, t.missing = cells.size, cells.ctypes.data, rec.ctypes.data, 0
    rgba, stats, _ = render_pixels(c, cam, params, px, py, nthreads=nthreads)
    if t.missing != 0:
        raise RuntimeError(f"{t.missing} shaded cells were missing from the record table")
    return rgba, stats, int(cells.size)


def render_image(cache: Cache, cam: dict, params: _Params, want_cells=False, nthreads=None):
    """Whole image: rgba [H,W,4], stats [H,W,4], cells [H,W,N] or None."""
    W, H = int(cam["W"]), int(cam["H"])
    py, px = np.meshgrid(np.arange(H, dtype=np.int32), np.arange(W, dtype=np.int32), indexing="ij")
    rgba, stats, cells = render_pixels(cache, cam, params, px.reshape(-1), py.reshape(-1), want_cells, nthreads)
    return (rgba.reshape(H, W, 4), stats.reshape(H, W, 4),
            None if cells is None else cells.reshape(H, W, params.N))


def ray(cam: dict, px: int, py: int):
    d = np.zeros(3, dtype=np.float32)
    o = np.zeros(3, dtype=np.float32)
    cs = camera_struct(cam)
    lib().orc_ray(ctypes.byref(cs), px, py, _p(d), _p(o))
    return d, o


def beta_bilinear(cache: Cache, d) -> np.ndarray:
    """The bilinearly interpolated direction weights (FP64) for the binary32 unit direction d."""
    d = np.ascontiguousarray(d, dtype=np.float32)
    out = np.zeros(cache.D)
    lib().orc_beta_bilinear(ctypes.byref(cache._s), _p(d), _p(out))
    return out


def render_mlp_pixels(pos_layers, dir_layers, D, cam: dict, params: _Params, px, py, pos_freqs=10, dir_freqs=4,
                      bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5), round_bf16=True, nthreads=None):
    """The uncached render of listed pixels (FP64): F_pos (layers [(W FP64, b FP64)]) at every sample inside
    the box (binary32 positions, orc_mlp_samples), F_dir at the ray direction, then Eq. 5 with the sigmoid
    and Eq. 1 with the exact integer termination on sigma rounded to binary32 (the width the renderer
    keeps it in). round_bf16: the activations between layers (and the encoded input) are rounded to bf16 as
    the tensor cores see them. Returns (rgba [n,4] f64, stats [n,4] i32: n_steps, n_lookups, n_occupied, -1)."""
    px = np.ascontiguousarray(px, dtype=np.int32).reshape(-1)
    py = np.ascontiguousarray(py, dtype=np.int32).reshape(-1)
    n, N = px.size, params.N
    pts = np.zeros((n, N, 3), np.float32)
    inside = np.zeros((n, N), np.uint8)
    dirs = np.zeros((n, 3), np.float32)
    lo, hi = np.asarray(bmin, np.float32), np.asarray(bmax, np.float32)
    cs = camera_struct(cam)
    lib().orc_mlp_samples(ctypes.byref(cs), ctypes.byref(params), _p(lo), _p(hi), n, _p(px), _p(py), _p(pts),
                          _p(inside), _p(dirs))
    mask = inside.astype(bool)
    out = mlp_eval(pos_layers, pts[mask].astype(np.float64), pos_freqs, round_bf16, nthreads)
    beta = mlp_eval(dir_layers, dirs.astype(np.float64), dir_freqs, round_bf16, nthreads)[:, :D]
    dtv = float(dt(params.t_near, params.t_far, N))
    sthr = s_thr(params.t_thr, dtv) if params.t_thr > 0 else (1 << 63) - 1
    rgba = np.zeros((n, 4))
    stats = np.zeros((n, 4), np.int32)
    j = 0
    for r in range(n):
        T, C, S = 1.0, np.zeros(3), 0
        n_steps, n_look, n_occ = N, 0, 0
        idx = np.flatnonzero(mask[r])
        for i in idx:
            o = out[j + n_look]
            n_look += 1
            sg = max(o[0], 0.0)
            if not sg > 0.0:
                continue
            n_occ += 1
            x = beta[r] @ o[1:1 + 3 * D].reshape(3, D).T  # Eq. 5: x_ch = sum_i beta_i u_ch,i
            col = x if params.act == ACT_IDENTITY else 1.0 / (1.0 + np.exp(-x))
            od = sg * dtv
            C += T * (-math.expm1(-od)) * col  # Eq. 1
            T *= math.exp(-od)
            S = min(S + fix(float(np.float32(sg))), (1 << 63) - 1)
            if S >= sthr:
                n_steps = int(i) + 1
                break
        j += int(mask[r].sum())
        rgba[r, :3] = C + T * np.asarray(params.bg[:], np.float64)
        rgba[r, 3] = 1.0 - T
        stats[r] = (n_steps, n_look, n_occ, -1)
    return rgba, stats


def dir_cell(l: int, d) -> tuple:
    d = np.ascontiguousarray(d, dtype=np.float32)
    it = ctypes.c_int32()
    ip = ctypes.c_int32()
    lib().orc_dir_cell(l, _p(d), ctypes.byref(it), ctypes.byref(ip))
    return it.value, ip.value


def phi_key(x: float, y: float) -> float:
    return lib().orc_phi_key(x, y)


def dt(t_near, t_far, N) -> float:
    return lib().orc_dt(t_near, t_far, N)


def s_thr(t_thr, dt_) -> int:
    return lib().orc_s_thr(t_thr, dt_)


def round_bf16(x) -> np.ndarray:
    """Each value rounded to binary32, then to bfloat16 (both round to nearest even), as FP64."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    return np.array([lib().orc_round_bf16(float(v)) for v in x])


def fix(sigma: float) -> int:
    return lib().orc_fix(sigma)


def trace_fp64(cache: Cache, cam: dict, params: _Params, px: int, py: int):
    N = params.N
    cells = np.zeros(N, dtype=np.int32)
    margin = np.zeros(N)
    dc = ctypes.c_int32()
    dm = ctypes.c_double()
    cs = camera_struct(cam)
    lib().orc_trace_fp64(ctypes.byref(cache._s), ctypes.byref(cs), ctypes.byref(params), px, py, _p(cells),
                         _p(margin), ctypes.byref(dc), ctypes.byref(dm))
    return cells, margin, dc.value, dm.value


# ------------------------------------------------------------------ formats and quantisation
def f16_encode(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32).reshape(-1)
    return np.array([lib().orc_f16_encode(float(v)) for v in x], dtype=np.uint16)


def f16_decode(h) -> np.ndarray:
    h = np.asarray(h, dtype=np.uint16).reshape(-1)
    return np.array([lib().orc_f16_decode(int(v)) for v in h])


def e4m3_encode(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32).reshape(-1)
    return np.array([lib().orc_e4m3_encode(float(v)) for v in x], dtype=np.uint8)


def e4m3_decode(q) -> np.ndarray:
    q = np.asarray(q, dtype=np.uint8).reshape(-1)
    return np.array([lib().orc_e4m3_decode(int(v)) for v in q])


def quantize_channel(prec: int, x: np.ndarray, clamp_nonneg: bool, scale: float = 1.0) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    dt_ = {FP32: np.float32, FP16: np.uint16, FP8: np.uint8}[prec]
    out = np.zeros(x.size, dtype=dt_)
    lib().orc_quantize(prec, x.size, 1, _p(x), int(clamp_nonneg), scale, _p(out))
    return out


def fp8_scale(x: np.ndarray, clamp_nonneg: bool) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    return lib().orc_fp8_scale(x.size, 1, _p(x), int(clamp_nonneg))


def offset_brick(k: int) -> int:
    """Side of the E4M3 offset bricks: the smallest power of two >= 4 with ceil(k / Bo) <= 64."""
    b = 4
    while (k + b - 1) // b > 64:
        b *= 2
    return b


def fp8_offsets(k, D, uvw, Bo) -> np.ndarray:
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1)
    nbo = (k + Bo - 1) // Bo
    out = np.zeros(nbo ** 3 * 3 * D, dtype=np.uint16)
    lib().orc_fp8_offsets(k, 3 * D, Bo, _p(uvw), _p(out))
    return out


def quantize_cache(k, D, l, sigma, uvw, beta, pos_prec, dir_prec) -> Cache:
    """The oracle's own quantisation of FP32 cache arrays into a stored-precision Cache."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float32).reshape(-1)
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1, 3 * D)
    beta = np.ascontiguousarray(beta, dtype=np.float32).reshape(-1)
    scales = None
    offsets, Bo = None, 0
    if pos_prec == FP8:
        Bo = offset_brick(k)
        offsets = fp8_offsets(k, D, uvw, Bo)
        scales = np.zeros(1 + 3 * D, dtype=np.float32)
        scales[0] = fp8_scale(sigma, True)
        for c in range(3 * D):
            scales[1 + c] = lib().orc_fp8_uvw_scale(k, 3 * D, Bo, _p(uvw), _p(offsets), c)
        qs = quantize_channel(FP8, sigma, True, scales[0])
        qu = np.zeros(uvw.shape, dtype=np.uint8)
        lib().orc_fp8_uvw_quantize(k, 3 * D, Bo, _p(uvw), _p(offsets), _p(np.ascontiguousarray(scales[1:])),
                                   _p(qu))
    elif pos_prec == FP16:
        qs = quantize_channel(FP16, sigma, True)
        qu = quantize_channel(FP16, uvw.reshape(-1), False).reshape(uvw.shape)
    else:
        qs = quantize_channel(FP32, sigma, True)
        qu = uvw
    qb = quantize_channel(FP16, beta, False) if dir_prec == FP16 else beta
    return Cache(k, D, l, qs, qu, qb, pos_prec=pos_prec, dir_prec=dir_prec, scales=scales, offsets=offsets,
                 off_brick=Bo)


# ------------------------------------------------------------------ cache sizes
def bytes_nerf(k, l, s_sigma_bits=16, s_rgb_bits=24) -> int:
    return int(lib().orc_bytes_nerf(k, l, s_sigma_bits, s_rgb_bits))


def bytes_fastnerf(k, l, D, s_sigma_bits=16, s_uvw_bits=48, s_beta_bits=16) -> tuple:
    """(position-cache bytes, direction-cache bytes) for a dense cache."""
    return (int(lib().orc_bytes_fastnerf_pos(k, D, s_sigma_bits, s_uvw_bits)),
            int(lib().orc_bytes_fastnerf_dir(l, D, s_beta_bits)))


# ------------------------------------------------------------------ MLPs
def posenc(x: np.ndarray, L: int, n_out: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, n_in = x.shape
    out = np.zeros((n, n_out))
    lib().orc_posenc(n, n_in, L, _p(x), n_out, _p(out))
    return out


def mlp_forward(weights, biases, x: np.ndarray, round_bf16: bool, nthreads=None) -> np.ndarray:
    """weights[i]: [out, in] FP64 (exact values of the stored bf16 weights); biases[i]: [out]."""
    n_layers = len(weights)
    dims = [weights[0].shape[1]] + [w.shape[0] for w in weights]
    dims_a = np.array(dims, dtype=np.int32)
    Ws = [np.ascontiguousarray(w, dtype=np.float64) for w in weights]
    Bs = [np.ascontiguousarray(b, dtype=np.float64) for b in biases]
    Wp = (ctypes.c_void_p * n_layers)(*[w.ctypes.data for w in Ws])
    Bp = (ctypes.c_void_p * n_layers)(*[b.ctypes.data for b in Bs])
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], dims[-1]))
    rc = lib().orc_mlp_forward(n_layers, _p(dims_a), Wp, Bp, int(round_bf16), x.shape[0], _p(x), _p(out),
                               _nthreads(nthreads))
    if rc != 0:
        raise ValueError("orc_mlp_forward rejected its arguments")
    return out


# ------------------------------------------------------------------ cache build from the MLPs (Section 3.3)
def cell_centres(k: int, cells, bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5)) -> np.ndarray:
    """FP64 grid sample of linear cell index (z*k + y)*k + x: bmin + (j + 1/2)(bmax - bmin)/k per axis."""
    cells = np.asarray(cells, dtype=np.int64)
    idx = np.stack([cells % k, (cells // k) % k, cells // (k * k)], axis=1).astype(np.float64)
    lo, hi = np.asarray(bmin, np.float64), np.asarray(bmax, np.float64)
    return lo + (idx + 0.5) * ((hi - lo) / k)


def bin_directions(l: int, bins) -> np.ndarray:
    """FP64 unit direction of bin i_theta*l + i_phi: theta = (i_theta + 1/2) pi / l from +z,
    phi = (i_phi + 1/2) 2 pi / l."""
    bins = np.asarray(bins, dtype=np.int64)
    th = (bins // l + 0.5) * (np.pi / l)
    ph = (bins % l + 0.5) * (2.0 * np.pi / l)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)


def mlp_eval(layers, x: np.ndarray, L: int, round_bf16: bool, nthreads=None) -> np.ndarray:
    """F(x): positional encoding with L frequencies, then the MLP (layers: [(W FP64 [out][in], b FP64)])."""
    enc = posenc(x, L, layers[0][0].shape[1])
    return mlp_forward([W for W, _ in layers], [b for _, b in layers], enc, round_bf16, nthreads)
