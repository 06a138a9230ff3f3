"""Seeded synthetic inputs: procedural scenes, direction fields and cameras.

This module is the one input generator that both the renderer's tests and the
oracle consume. It holds none of the rendering method's arithmetic (no ray
generation, no cache lookup, no compositing): it draws random scene parameters
from a counter-based generator and evaluates procedural fields at given points.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition. Draw order for ``make_scene`` (one generator seeded with ``seed``):

1. spheres, for each: centre x, y, z ~ U[-1, 1], radius ~ U[0.1, 0.4];
2. shells, for each: centre x, y, z ~ U[-1, 1], half-extents hx, hy, hz ~ U[0.1, 0.5];
3. deep-radiance channels c = 0 .. 3D-1 (order u_1..u_D, v_1..v_D, w_1..w_D), for
   each of ``n_terms`` sinusoids: amplitude ~ U[-1, 1]; integer frequency vector
   f ~ {-2..2}^3 drawn x, y, z as ``-2 + (next() % 5)`` and redrawn whole while
   all three are zero; phase ~ U[0, 2*pi);
4. direction weights i = 0 .. D-1, degree l = 0 .. L, order m = -l .. l: one
   real-SH coefficient ~ N(0, 1) (Box-Muller, cosine branch, two draws).

U[a, b] = a + (b - a) * u with u = (next() >> 11) * 2**-53.

Cameras (``cameras``, own generator seeded with ``seed``): per camera, z ~ U[zlo, 1]
(zlo = -1 for the full sphere, 0 for the upper hemisphere) then phi ~ U[0, 2*pi);
the eye is radius * (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z), looking at the
origin, world up +z (+y when the view axis is within 0.001 of +-z), camera looking
down its -z axis, fx = fy = W / (2 tan(fov/2)), cx = W/2, cy = H/2.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libscenegen.so")
_lib = None

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: a 64-bit counter with a fixed finalising mix per output."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        u = (self.next() >> 11) * (2.0 ** -53)
        return a + (b - a) * u

    def normal(self) -> float:
        u1 = ((self.next() >> 11) + 1) * (2.0 ** -53)  # (0, 1]
        u2 = (self.next() >> 11) * (2.0 ** -53)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def int_sym2(self) -> int:
        return -2 + (self.next() % 5)


def build_lib(force: bool = False) -> str:
    """Compile the grid-fill helper with gcc (plain C, no contraction)."""
    src = os.path.join(_HERE, "scenegen.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.sg_fill_grid.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P,
                                     ctypes.c_int, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, P, P, P, P, P, ctypes.c_int]
        lib.sg_fill_grid.restype = ctypes.c_int
        lib.sg_eval_points.argtypes = [ctypes.c_int64, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        lib.sg_eval_points.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Scene:
    """Parameters of one procedural scene (everything FP64)."""

    seed: int
    D: int
    spheres: np.ndarray          # [n, 4] cx, cy, cz, r
    shells: np.ndarray           # [n, 6] cx, cy, cz, hx, hy, hz
    amp: np.ndarray              # [3D * n_terms]
    freq: np.ndarray             # [3D * n_terms, 3] int32
    phase: np.ndarray            # [3D * n_terms]
    sh_coef: np.ndarray          # [D, (L+1)^2]
    sh_degree: int
    n_terms: int = 4
    sigma_val: float = 50.0
    thick: float = 0.02
    bmin: tuple = (-1.5, -1.5, -1.5)
    bmax: tuple = (1.5, 1.5, 1.5)
    extra: dict = field(default_factory=dict)


def make_scene(seed: int, n_spheres: int, n_shells: int, D: int, sh_degree: int, n_terms: int = 4,
               sigma_val: float = 50.0) -> Scene:
    rng = SplitMix64(seed)
    sph = np.zeros((n_spheres, 4))
    for s in range(n_spheres):
        sph[s, 0] = rng.uniform(-1, 1)
        sph[s, 1] = rng.uniform(-1, 1)
        sph[s, 2] = rng.uniform(-1, 1)
        sph[s, 3] = rng.uniform(0.1, 0.4)
    shl = np.zeros((n_shells, 6))
    for s in range(n_shells):
        for a in range(3):
            shl[s, a] = rng.uniform(-1, 1)
        for a in range(3):
            shl[s, 3 + a] = rng.uniform(0.1, 0.5)
    nt = 3 * D * n_terms
    amp = np.zeros(nt)
    freq = np.zeros((nt, 3), dtype=np.int32)
    phase = np.zeros(nt)
    for t in range(nt):
        amp[t] = rng.uniform(-1, 1)
        while True:
            f = [rng.int_sym2(), rng.int_sym2(), rng.int_sym2()]
            if any(f):
                break
        freq[t] = f
        phase[t] = rng.uniform(0.0, 2.0 * math.pi)
    nsh = (sh_degree + 1) ** 2
    coef = np.zeros((D, nsh))
    for i in range(D):
        for j in range(nsh):
            coef[i, j] = rng.normal()
    return Scene(seed=seed, D=D, spheres=sph, shells=shl, amp=amp, freq=freq, phase=phase, sh_coef=coef,
                 sh_degree=sh_degree, n_terms=n_terms, sigma_val=sigma_val)


def grid_axis(k: int, lo: float, hi: float) -> np.ndarray:
    """Grid sample coordinates along one axis: cell centres lo + (j + 1/2) (hi - lo) / k."""
    return lo + (np.arange(k, dtype=np.float64) + 0.5) * ((hi - lo) / k)


def fill_position_grid(scene: Scene, k: int, z0: int = 0, nz: int | None = None, nthreads: int | None = None,
                       with_uvw: bool = True, sigma_out=None, uvw_out=None):
    """Evaluate the scene on the k^3 grid, z-slab [z0, z0+nz).

    Returns (sigma [nz, k, k] float32, uvw [nz, k, k, 3D] float32 or None).
    Index order is [z][y][x], x fastest.
    """
    lib = _load()
    if nz is None:
        nz = k - z0
    nthreads = nthreads or max(1, os.cpu_count() or 1)
    xs = grid_axis(k, scene.bmin[0], scene.bmax[0])
    ys = grid_axis(k, scene.bmin[1], scene.bmax[1])
    zs = grid_axis(k, scene.bmin[2], scene.bmax[2])
    nch = 3 * scene.D
    sig = sigma_out if sigma_out is not None else np.empty((nz, k, k), dtype=np.float32)
    uvw = None
    if with_uvw:
        uvw = uvw_out if uvw_out is not None else np.empty((nz, k, k, nch), dtype=np.float32)
    assert sig.dtype == np.float32 and sig.flags.c_contiguous and sig.size == nz * k * k
    if uvw is not None:
        assert uvw.dtype == np.float32 and uvw.flags.c_contiguous and uvw.size == nz * k * k * nch
    sph = np.ascontiguousarray(scene.spheres, dtype=np.float64)
    shl = np.ascontiguousarray(scene.shells, dtype=np.float64)
    amp = np.ascontiguousarray(scene.amp)
    freq = np.ascontiguousarray(scene.freq, dtype=np.int32)
    phase = np.ascontiguousarray(scene.phase)
    rc = lib.sg_fill_grid(k, _ptr(xs), _ptr(ys), _ptr(zs), z0, nz, len(sph), _ptr(sph), len(shl), _ptr(shl),
                          scene.thick, scene.sigma_val, nch, scene.n_terms, _ptr(amp), _ptr(freq), _ptr(phase),
                          _ptr(sig), _ptr(uvw), nthreads)
    if rc != 0:
        raise RuntimeError("sg_fill_grid failed")
    return sig, uvw


def eval_points(scene: Scene, xyz: np.ndarray):
    """FP64 field (sigma [n], channels [n, 3D]) at arbitrary points, direct evaluation."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = xyz.shape[0]
    nch = 3 * scene.D
    sig = np.empty(n)
    ch = np.empty((n, nch))
    sph = np.ascontiguousarray(scene.spheres, dtype=np.float64)
    shl = np.ascontiguousarray(scene.shells, dtype=np.float64)
    freq = np.ascontiguousarray(scene.freq, dtype=np.int32)
    lib.sg_eval_points(n, _ptr(xyz), len(sph), _ptr(sph), len(shl), _ptr(shl), scene.thick, scene.sigma_val,
                       nch, scene.n_terms, _ptr(np.ascontiguousarray(scene.amp)), _ptr(freq),
                       _ptr(np.ascontiguousarray(scene.phase)), _ptr(sig), _ptr(ch))
    return sig, ch


# ---------------------------------------------------------------- spherical harmonics
def _assoc_legendre(L: int, x: np.ndarray) -> dict:
    """P_l^m(x) for 0 <= m <= l <= L by the standard three-term recurrences."""
    P = {}
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for m in range(L + 1):
        if m > 0:
            pmm = -pmm * (2 * m - 1) * s
        P[(m, m)] = pmm
        if m + 1 <= L:
            P[(m + 1, m)] = x * (2 * m + 1) * pmm
        for l in range(m + 2, L + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def real_sh(L: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonics Y_lm, l <= L, m = -l..l, stacked on the last axis."""
    x = np.cos(theta)
    P = _assoc_legendre(L, x)
    out = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(K * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2.0) * K * np.cos(m * phi) * P[(l, m)])
            else:
                out.append(math.sqrt(2.0) * K * np.sin(am * phi) * P[(l, am)])
    return np.stack(out, axis=-1)


def direction_grid(scene: Scene, l: int, dtype=np.float32) -> np.ndarray:
    """beta on the l x l (theta, phi) grid at cell centres: [l(theta)][l(phi)][D]."""
    th = (np.arange(l) + 0.5) * (math.pi / l)
    ph = (np.arange(l) + 0.5) * (2.0 * math.pi / l)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Y = real_sh(scene.sh_degree, TH, PH)              # [l, l, nsh]
    beta = np.einsum("abj,ij->abi", Y, scene.sh_coef)  # [l, l, D]
    return beta.astype(dtype)


# ---------------------------------------------------------------- cameras
def look_at_camera(eye, W: int, H: int, fov_deg: float = 40.0) -> dict:
    eye = np.asarray(eye, dtype=np.float64)
    back = eye / np.linalg.norm(eye)
    up_w = np.array([0.0, 0.0, 1.0])
    if abs(back[2]) > 0.999:
        up_w = np.array([0.0, 1.0, 0.0])
    right = np.cross(up_w, back)
    right /= np.linalg.norm(right)
    up = np.cross(back, right)
    c2w = np.zeros((3, 4))
    c2w[:, 0] = right
    c2w[:, 1] = up
    c2w[:, 2] = back
    c2w[:, 3] = eye
    f = 0.5 * W / math.tan(0.5 * math.radians(fov_deg))
    return dict(c2w=c2w.astype(np.float32).reshape(12), fx=np.float32(f), fy=np.float32(f),
                cx=np.float32(W / 2), cy=np.float32(H / 2), W=int(W), H=int(H))


def cameras(seed: int, n: int, W: int, H: int, radius: float = 4.0, fov_deg: float = 40.0,
            hemisphere: bool = False) -> list:
    rng = SplitMix64(seed)
    cams = []
    zlo = 0.0 if hemisphere else -1.0
    for _ in range(n):
        z = rng.uniform(zlo, 1.0)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        eye = radius * np.array([s * math.cos(ph), s * math.sin(ph), z])
        cams.append(look_at_camera(eye, W, H, fov_deg))
    return cams


# ---------------------------------------------------------------- workload presets
@dataclass
class Workload:
    name: str
    scene: Scene
    k: int
    l: int
    D: int
    W: int
    H: int
    n_samples: int
    n_cams: int
    cam_seed: int
    hemisphere: bool
    t_near: float = 2.0
    t_far: float = 6.0
    t_thr: float = 1e-4
    bg: tuple = (1.0, 1.0, 1.0)

    def cameras(self, n: int | None = None) -> list:
        return cameras(self.cam_seed, n or self.n_cams, self.W, self.H, hemisphere=self.hemisphere)


def tiny(seed: int = 0) -> Workload:
    """64^3 FP32 cache, D=8, 8 spheres, 64x64 direction grid of degree-3 SH, one 64x64 view, 64 samples."""
    sc = make_scene(seed, n_spheres=8, n_shells=0, D=8, sh_degree=3)
    return Workload("tiny-k64-D8-64x64-N64", sc, k=64, l=64, D=8, W=64, H=64, n_samples=64, n_cams=1,
                    cam_seed=seed + 1, hemisphere=False)


def scale(seed: int = 0, k: int = 512, l: int = 512, W: int = 800, H: int = 800, n_samples: int = 128,
          n_cams: int = 8) -> Workload:
    """800x800 views, 128 samples, k=512^3 FP32 cache (D=8), 32 spheres + 16 shells, 512^2 degree-4 SH."""
    sc = make_scene(seed, n_spheres=32, n_shells=16, D=8, sh_degree=4)
    return Workload(f"scale-k{k}-D8-{W}x{H}-N{n_samples}", sc, k=k, l=l, D=8, W=W, H=H, n_samples=n_samples,
                    n_cams=n_cams, cam_seed=seed + 1, hemisphere=True)


def precision(seed: int = 0) -> Workload:
    """The same scene family at k=1024^3 (D=8) with a 768^2 direction grid, 16 views of 800x800, 192 samples."""
    return scale(seed, k=1024, l=768, n_samples=192, n_cams=16)


def fill_position_grid_device(scene: Scene, k: int, sigma_dev, uvw_dev, sigma_host=None, nz: int = 16,
                              nthreads: int | None = None):
    """fill_position_grid for grids too large for host memory: z-slabs of nz are generated into a pinned
    host buffer and copied into the device tensors sigma_dev [k^3] and uvw_dev [k^3 * 3D] (float32).
    The sigma plane is also kept in sigma_host (float32 [k, k, k]) when given."""
    import torch
    nch = 3 * scene.D
    plane = k * k
    bufs = [(torch.empty(nz * plane, dtype=torch.float32, pin_memory=True),
             torch.empty(nz * plane * nch, dtype=torch.float32, pin_memory=True)) for _ in range(2)]
    done = [None, None]
    stream = torch.cuda.current_stream(sigma_dev.device)
    for i, z0 in enumerate(range(0, k, nz)):
        n = min(nz, k - z0)
        bs, bu = bufs[i & 1]
        if done[i & 1] is not None:
            done[i & 1].synchronize()  # the copy out of this buffer has finished
        fill_position_grid(scene, k, z0, n, nthreads, sigma_out=bs.numpy()[: n * plane].reshape(n, k, k),
                           uvw_out=bu.numpy()[: n * plane * nch].reshape(n, k, k, nch))
        if sigma_host is not None:
            sigma_host.reshape(k, k, k)[z0:z0 + n] = bs.numpy()[: n * plane].reshape(n, k, k)
        sigma_dev[z0 * plane:(z0 + n) * plane].copy_(bs[: n * plane], non_blocking=True)
        uvw_dev[z0 * plane * nch:(z0 + n) * plane * nch].copy_(bu[: n * plane * nch], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(stream)
        done[i & 1] = ev
    torch.cuda.synchronize(sigma_dev.device)


def cell_records(scene: Scene, k: int, cells: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """uvw channels (float32 [n, 3D]) of the grid cells with linear index (z*k + y)*k + x, evaluated at
    the cell centres: the values fill_position_grid stores for those cells."""
    from concurrent.futures import ThreadPoolExecutor
    cells = np.asarray(cells, dtype=np.int64).reshape(-1)
    axes = [grid_axis(k, scene.bmin[a], scene.bmax[a]) for a in range(3)]
    x, y, z = cells % k, (cells // k) % k, cells // (k * k)
    pts = np.stack([axes[0][x], axes[1][y], axes[2][z]], axis=1)
    out = np.empty((cells.size, 3 * scene.D), dtype=np.float32)
    nthreads = nthreads or max(1, os.cpu_count() or 1)
    chunks = np.array_split(np.arange(cells.size), max(1, min(nthreads * 4, cells.size)))

    def run(ix):
        if ix.size:
            out[ix] = eval_points(scene, pts[ix])[1].astype(np.float32)

    with ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(run, chunks))
    return out


# ---------------------------------------------------------------- MLP weights (cache-build inputs)
def bf16_bits(x: np.ndarray) -> np.ndarray:
    """binary32 -> bf16 bit patterns, round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_value(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def mlp_weights(seed: int, dims: list, bias_scale: float = 0.0) -> list:
    """He-uniform MLP weights W_i ~ U(-sqrt(6/fan_in), +sqrt(6/fan_in)), [out][in], stored as bf16 bits;
    biases U(-bias_scale, bias_scale) as float32 (0 by default). Draws: numpy PCG64(seed), layer by layer,
    weights then biases."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32)
        b = rng.uniform(-bias_scale, bias_scale, size=fan_out).astype(np.float32) if bias_scale else \
            np.zeros(fan_out, np.float32)
        out.append((bf16_bits(W), b))
    return out


FPOS_DIMS_D8 = [60, 256, 256, 256, 256, 256, 256, 256, 256, 25]   # 8 ReLU layers of 256 + linear head
FDIR_DIMS_D8 = [24, 128, 128, 128, 128, 8]                          # 4 ReLU layers of 128 + linear head
