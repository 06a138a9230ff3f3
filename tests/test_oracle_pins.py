"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: numbers the
paper prints, closed forms of Eq. 1 on homogeneous media, reductions of Eq. 5,
brute-force FP64 geometry with libm, and library number formats.
"""

import ctypes
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenegen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def axis_camera(W=64, H=64, f=80.0, eye=(0.0, 0.0, 4.0)):
    """Camera at `eye` looking at the origin; cx, cy put pixel (W//2, H//2) on the optical axis."""
    cam = scenegen.look_at_camera(eye, W, H)
    cam["fx"] = np.float32(f)
    cam["fy"] = np.float32(f)
    cam["cx"] = np.float32(W // 2 + 0.5)
    cam["cy"] = np.float32(H // 2 + 0.5)
    return cam


def const_cache(k, D, l, sigma0, uvw_vals, beta_vals, prec=oracle.FP32):
    n = k ** 3
    sig = np.full(n, sigma0, dtype=np.float32)
    uvw = np.tile(np.asarray(uvw_vals, dtype=np.float32).reshape(1, 3 * D), (n, 1))
    beta = np.tile(np.asarray(beta_vals, dtype=np.float32).reshape(1, D), (l * l, 1))
    return oracle.Cache(k, D, l, sig, uvw, beta)


# ------------------------------------------------------------------ cache sizes (printed integers)
def test_cache_sizes_match_paper():
    with open(os.path.join(GOLDEN, "cache_sizes.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        if c["formula"] == "nerf":
            assert oracle.bytes_nerf(c["k"], c["l"], c["s_sigma_bits"], c["s_rgb_bits"]) == c["bytes"], c["cite"]
        elif c["formula"] == "fastnerf":
            pos, dirb = oracle.bytes_fastnerf(c["k"], c["l"], c["D"], c["s_sigma_bits"], c["s_uvw_bits"],
                                              c["s_beta_bits"])
            assert (pos, dirb) == (c["pos_bytes"], c["dir_bytes"]), c["cite"]
        elif c["formula"] == "nerf_approx":
            v = oracle.bytes_nerf(c["k"], c["l"], c["s_sigma_bits"], c["s_rgb_bits"])
            assert abs(v / c["approx_bytes"] - 1) < c["rel_tol"], c["cite"]
        elif c["formula"] == "fastnerf_approx":
            pos, dirb = oracle.bytes_fastnerf(c["k"], c["l"], c["D"], c["s_sigma_bits"], c["s_uvw_bits"],
                                              c["s_beta_bits"])
            assert abs((pos + dirb) / c["approx_bytes"] - 1) < c["rel_tol"], c["cite"]


# ------------------------------------------------------------------ Eq. 1: homogeneous medium closed forms
@pytest.mark.parametrize("sigma0,expect_steps", [(2.0, 64), (0.5, 64), (50.0, 11), (7.0, None)])
def test_homogeneous_box_closed_form(sigma0, expect_steps):
    """All cells sigma0, colour c: C = c (1 - e^{-sigma0 m Delta}) + e^{-sigma0 m Delta} bg, m composited samples.

    Central ray of a camera at (0,0,4) looking down -z: samples t_i = 2 + (i+1/2)/16 put
    z = 2 - (i+1/2)/16, exact in binary32, inside [-1.5, 1.5) for i = 8..55 (48 samples).
    m = min(48, m_thr) with m_thr the smallest m such that m sigma0 Delta >= ln(1/T_thr).
    """
    k, D, l, N = 64, 1, 8, 64
    c = np.array([0.3, 0.5, 0.7], dtype=np.float32).astype(np.float64)  # stored binary32 values
    cache = const_cache(k, D, l, sigma0, c, [1.0])
    cam = axis_camera()
    bg = (0.9, 0.2, 0.4)
    p = oracle.params_struct(N, 2.0, 6.0, 1e-4, bg, oracle.ACT_IDENTITY)
    rgba, st, cells = oracle.render_pixels(cache, cam, p, [32], [32], want_cells=True)
    delta = 4.0 / N
    m_thr = math.ceil(math.log(1e4) / (sigma0 * delta))
    m = min(48, m_thr)
    Tm = math.exp(-sigma0 * m * delta)
    expect = c * (1 - Tm) + Tm * np.array(bg, dtype=np.float32).astype(np.float64)
    np.testing.assert_allclose(rgba[0, :3], expect, rtol=0, atol=1e-12)
    assert abs(rgba[0, 3] - (1 - Tm)) < 1e-12
    n_steps = 8 + m if m_thr <= 48 else N
    assert st[0, 0] == n_steps
    if expect_steps is not None:
        assert n_steps == expect_steps
    assert st[0, 1] == m and st[0, 2] == m


@pytest.mark.parametrize("sigma0", [2.0, 50.0])
def test_homogeneous_box_cells_single_answer(sigma0):
    """Every sample's cell, worked out by hand, with no sample near a cell face.

    Camera with the identity rotation (looking down -z) at eye = (0.01, -0.02, 4 + 1/128); the central
    pixel's ray is d = (0, 0, -1) exactly. Sample i lies at t_i = 2 + (2i + 1)/32, so
    z_i + 1.5 = (445 - 8i)/128 and the exact grid coordinate is gz_i = (445 - 8i)/6, which is never within
    1/6 of an integer (445 - 8i is odd and not divisible by 3 for any i; 445 - 8i = 1 - 2i mod 6).
    gx = 1.51 * 64/3 = 32.21 and gy = 1.48 * 64/3 = 31.57 are 0.2 cells or more from a face. So each
    sample has exactly one correct cell: (floor(gz_i) * 64 + 31) * 64 + 32 for i = 8..55, outside the box
    (-1) otherwise, -2 after termination. The colour is the closed form of the homogeneous box.
    """
    k, D, l, N = 64, 1, 8, 64
    c = np.array([0.3, 0.5, 0.7], dtype=np.float32).astype(np.float64)
    cache = const_cache(k, D, l, sigma0, c, [1.0])
    cam = dict(c2w=np.array([1, 0, 0, 0.01, 0, 1, 0, -0.02, 0, 0, 1, 4 + 1 / 128], np.float32),
               fx=np.float32(80.0), fy=np.float32(80.0), cx=np.float32(32.5), cy=np.float32(32.5), W=64, H=64)
    d, _ = oracle.ray(cam, 32, 32)
    assert list(d) == [0.0, 0.0, -1.0]
    bg = (0.9, 0.2, 0.4)
    p = oracle.params_struct(N, 2.0, 6.0, 1e-4, bg, oracle.ACT_IDENTITY)
    rgba, st, cells = oracle.render_pixels(cache, cam, p, [32], [32], want_cells=True)
    delta = 4.0 / N
    m_thr = math.ceil(math.log(1e4) / (sigma0 * delta))
    m = min(48, m_thr)
    n_steps = 8 + m if m_thr <= 48 else N
    assert st[0, 0] == n_steps and st[0, 1] == m and st[0, 2] == m
    Tm = math.exp(-sigma0 * m * delta)
    expect = c * (1 - Tm) + Tm * np.array(bg, dtype=np.float32).astype(np.float64)
    np.testing.assert_allclose(rgba[0, :3], expect, rtol=0, atol=1e-12)
    for i in range(N):
        if i >= n_steps:
            want = -2
        elif i < 8 or i > 55:
            want = -1
        else:
            assert (445 - 8 * i) % 6 != 0
            want = (((445 - 8 * i) // 6) * k + 31) * k + 32
        assert cells[0, i] == want, (i, cells[0, i], want)


def test_homogeneous_box_chord_form():
    """Continuous Beer-Lambert along the chord: |C - (c (1-e^{-sL}) + e^{-sL} bg)| <= s * Delta (|n Delta - L| <= Delta)."""
    k, N, sigma0 = 32, 256, 0.7
    c = np.array([0.2, 0.6, 0.9], dtype=np.float32).astype(np.float64)
    cache = const_cache(k, 1, 4, sigma0, c, [1.0])
    cam = axis_camera()
    bg = np.array([1.0, 1.0, 1.0])
    p = oracle.params_struct(N, 2.0, 6.0, 0.0, tuple(bg), oracle.ACT_IDENTITY)
    rgba, st, _ = oracle.render_pixels(cache, cam, p, [32], [32])
    L = 3.0
    TL = math.exp(-sigma0 * L)
    expect = c * (1 - TL) + TL * bg
    assert np.max(np.abs(rgba[0, :3] - expect)) <= sigma0 * (4.0 / N) + 1e-12
    assert st[0, 0] == N  # T_thr = 0 disables termination


def test_empty_cache_invariants(tiny_arrays):
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    cache = oracle.Cache(w.k, w.D, w.l, np.zeros_like(sig), uvw, beta)
    bg = (0.25, 0.5, 1.0)
    p = oracle.params_struct(w.n_samples, bg=bg)
    rgba, st, _ = oracle.render_image(cache, w.cameras()[0], p)
    assert np.all(rgba[..., :3] == np.array(bg))
    assert np.all(rgba[..., 3] == 0.0)
    assert np.all(st[..., 2] == 0) and np.all(st[..., 0] == w.n_samples)


def test_transmittance_invariants_and_termination(tiny_arrays):
    """0 <= 1-T <= 1; terminated rays stop at the first sample whose FP64 transmittance is <= T_thr."""
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    cache = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    p = oracle.params_struct(w.n_samples)
    cam = w.cameras()[0]
    rgba, st, cells = oracle.render_image(cache, cam, p, want_cells=True)
    A = rgba[..., 3]
    assert np.all(A >= 0) and np.all(A <= 1)
    assert np.all(rgba[..., :3] >= 0) and np.all(rgba[..., :3] <= 1 + 1e-12)  # sigmoid colours, white bg
    flat_cells = cells.reshape(-1, w.n_samples)
    sflat = sig.reshape(-1)
    dt = 4.0 / w.n_samples
    term = st[..., 0].reshape(-1) < w.n_samples
    assert term.sum() > 100
    for r in np.nonzero(term)[0][:400]:
        n = st.reshape(-1, 4)[r, 0]
        cs = flat_cells[r, :n]
        od = np.cumsum([sflat[cc] * dt if cc >= 0 else 0.0 for cc in cs])
        assert math.exp(-od[-1]) <= 1e-4 * (1 + 1e-9)
        assert n == 1 or math.exp(-od[-2]) > 1e-4
        assert abs((1 - A.reshape(-1)[r]) - math.exp(-od[-1])) < 1e-12
        assert np.all(flat_cells[r, n:] == -2)


# ------------------------------------------------------------------ Eq. 5 reductions
def test_eq5_component_pairing():
    """D=2, u=(1,0), v=(0,1), w=(0,0), beta=(b1,b2), identity: colour per sample = (b1, b2, 0)."""
    k, l, N, sigma0 = 16, 8, 64, 3.0
    b1, b2 = 0.375, -1.25
    cache = const_cache(k, 2, l, sigma0, [1, 0, 0, 1, 0, 0], [b1, b2])
    cam = axis_camera()
    p = oracle.params_struct(N, bg=(0, 0, 0), act=oracle.ACT_IDENTITY)
    rgba, _, _ = oracle.render_pixels(cache, cam, p, [32, 20, 40], [32, 31, 45])
    A = rgba[:, 3]
    np.testing.assert_allclose(rgba[:, 0], b1 * A, atol=1e-14)
    np.testing.assert_allclose(rgba[:, 1], b2 * A, atol=1e-14)
    np.testing.assert_allclose(rgba[:, 2], 0.0, atol=0)


def test_eq5_dropped_component_reduction(tiny_arrays):
    """D=2 with beta=(1, 0) renders exactly like D=1 with beta=1 on the first component."""
    sig, uvw, _ = tiny_arrays
    w = scenegen.tiny()
    D = w.D
    u1 = uvw[:, :, :, [0, D, 2 * D]].reshape(-1, 3)
    rng = np.random.default_rng(5)
    u2 = rng.standard_normal(u1.shape).astype(np.float32)
    uvw2 = np.stack([u1[:, 0], u2[:, 0], u1[:, 1], u2[:, 1], u1[:, 2], u2[:, 2]], axis=1)
    l = 16
    c1 = oracle.Cache(w.k, 1, l, sig, u1, np.ones((l, l, 1), np.float32))
    b2 = np.zeros((l, l, 2), np.float32)
    b2[..., 0] = 1
    c2 = oracle.Cache(w.k, 2, l, sig, uvw2, b2)
    p = oracle.params_struct(w.n_samples)
    cam = w.cameras()[0]
    r1, s1, _ = oracle.render_image(c1, cam, p)
    r2, s2, _ = oracle.render_image(c2, cam, p)
    assert np.array_equal(r1, r2) and np.array_equal(s1[..., :3], s2[..., :3])


def test_eq5_constant_beta_direction_permutation(tiny_arrays):
    """With direction-independent beta, permuting the direction cache leaves the image unchanged."""
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    const_b = np.tile(beta[3, 5].reshape(1, 1, -1), (w.l, w.l, 1))
    perm = np.random.default_rng(1).permutation(w.l * w.l)
    shuffled = const_b.reshape(-1, w.D)[perm].reshape(w.l, w.l, w.D)
    p = oracle.params_struct(w.n_samples)
    cam = w.cameras()[0]
    ra, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, const_b), cam, p)
    rb, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, shuffled), cam, p)
    assert np.array_equal(ra, rb)


def test_sigmoid_activation_midpoint():
    """u=v=w=0 under the sigmoid gives colour 1/2: closed form with c = 0.5."""
    k, N, sigma0 = 16, 64, 2.0
    cache = const_cache(k, 1, 4, sigma0, [0, 0, 0], [1.0])
    p = oracle.params_struct(N, bg=(0, 0, 0), act=oracle.ACT_SIGMOID)
    rgba, st, _ = oracle.render_pixels(cache, axis_camera(), p, [32], [32])
    Tm = math.exp(-sigma0 * 48 * (4.0 / N))
    np.testing.assert_allclose(rgba[0, :3], 0.5 * (1 - Tm), atol=1e-13)


def test_identity_activation_linearity(tiny_arrays):
    """Identity activation, bg = 0: the image is linear in beta (same density, same weights)."""
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    p = oracle.params_struct(w.n_samples, bg=(0, 0, 0), act=oracle.ACT_IDENTITY)
    cam = w.cameras()[0]
    b1 = (np.round(beta * 64) / 64).astype(np.float32)  # coarse values: 2 b1 - 3 b2 is exact in binary32
    b2 = np.roll(b1, 7, axis=1)
    r1, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, b1), cam, p)
    r2, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, b2), cam, p)
    r3, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, (2 * b1 - 3 * b2).astype(np.float32)),
                                   cam, p)
    np.testing.assert_allclose(r3[..., :3], 2 * r1[..., :3] - 3 * r2[..., :3], atol=1e-9)


# ------------------------------------------------------------------ direction cell vs libm FP64
def test_direction_cell_known_axes():
    l = 64
    assert oracle.dir_cell(l, [0, 0, 1]) == (0, 0)
    assert oracle.dir_cell(l, [0, 0, -1]) == (l - 1, 0)
    assert oracle.dir_cell(l, [1, 0, 0]) == (l // 2, 0)
    assert oracle.dir_cell(l, [0, 1, 0]) == (l // 2, l // 4)
    assert oracle.dir_cell(l, [-1, 0, 0]) == (l // 2, l // 2)
    assert oracle.dir_cell(l, [0, -1, 0]) == (l // 2, 3 * l // 4)
    s = math.sqrt(0.5)
    assert oracle.dir_cell(l, [s, -1e-3, s])[1] == l - 1


@pytest.mark.parametrize("l", [8, 64, 512, 768])
def test_direction_cell_vs_fp64_libm(l):
    rng = np.random.default_rng(l)
    d = rng.standard_normal((3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    dd = d.astype(np.float64)
    th = np.arccos(np.clip(dd[:, 2], -1, 1))
    ph = np.mod(np.arctan2(dd[:, 1], dd[:, 0]), 2 * np.pi)
    ut, up = th * l / np.pi, ph * l / (2 * np.pi)
    it_ref = np.minimum(np.floor(ut).astype(int), l - 1)
    ip_ref = np.floor(up).astype(int) % l
    near = (np.abs(ut - np.round(ut)) * np.pi / l < 1e-5) | (np.abs(up - np.round(up)) * 2 * np.pi / l < 1e-5)
    bad = 0
    for i in range(len(d)):
        got = oracle.dir_cell(l, d[i])
        if got != (it_ref[i], ip_ref[i]):
            assert near[i], (i, got, it_ref[i], ip_ref[i])
            bad += 1
    assert bad <= 3


def test_phi_key_monotone():
    ang = np.sort(np.random.default_rng(3).uniform(0, 2 * np.pi, 20000))
    keys = np.array([oracle.phi_key(np.float32(np.cos(a)), np.float32(np.sin(a))) for a in ang])
    assert np.all(np.diff(keys) >= 0)
    assert keys[0] >= 0 and keys[-1] <= 4


# ------------------------------------------------------------------ position cells vs FP64 geometry
def test_position_cells_vs_fp64_geometry(tiny_arrays):
    """binary32 sample cells equal the all-FP64 ones except for samples within 1e-3 cells of a face."""
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    cache = oracle.Cache(w.k, w.D, w.l, np.zeros_like(sig), uvw, beta)  # no termination: every sample visited
    p = oracle.params_struct(w.n_samples)
    cam = w.cameras()[0]
    rng = np.random.default_rng(0)
    px = rng.integers(0, w.W, 300).astype(np.int32)
    py = rng.integers(0, w.H, 300).astype(np.int32)
    _, st, cells = oracle.render_pixels(cache, cam, p, px, py, want_cells=True)
    mism = 0
    total = 0
    for i in range(len(px)):
        c64, margin, dcell, dmargin = oracle.trace_fp64(cache, cam, p, int(px[i]), int(py[i]))
        diff = c64 != cells[i]
        assert np.all(margin[diff] < 1e-3)
        mism += diff.sum()
        total += len(c64)
        if st[i, 3] != dcell:
            assert dmargin < 1e-5
    assert mism / total < 1e-3


# ------------------------------------------------------------------ termination arithmetic
def test_fixed_point_depth():
    assert oracle.fix(50.0) == 50 * 2 ** 32
    assert oracle.fix(0.0) == 0
    f = float(np.float32(0.1))
    assert oracle.fix(f) == math.floor(f * 2 ** 32)
    assert oracle.fix(3e9) == 2 ** 63 - 1
    assert oracle.dt(2.0, 6.0, 64) == 0.0625
    assert oracle.s_thr(1e-4, 0.0625) == math.ceil(math.log(1 / float(np.float32(1e-4))) / 0.0625 * 2 ** 32)
    assert oracle.s_thr(0.0, 0.0625) == 2 ** 63 - 1


# ------------------------------------------------------------------ number formats vs libraries
def test_fp16_codec_vs_numpy():
    codes = np.arange(65536, dtype=np.uint16)
    ref = codes.view(np.float16).astype(np.float64)
    got = oracle.f16_decode(codes)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin]) and np.all(np.isnan(got[np.isnan(ref)]))
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10 ** rng.uniform(-9, 5, 4000),
                        [65504, 65519.99, 65520, 1e9, -1e9, 2 ** -24, 2 ** -25, 3 * 2 ** -26, 0.0, -0.0,
                         1 + 2 ** -11, 1 + 3 * 2 ** -11]]).astype(np.float32)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(oracle.f16_encode(x), ref)


def test_e4m3_codec_vs_torch():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = oracle.e4m3_decode(codes)
    fin = ~np.isnan(ref)
    assert np.array_equal(got[fin], ref[fin]) and np.all(np.isnan(got[~fin]))
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 3000), rng.standard_normal(3000) * 2.0 ** rng.uniform(-12, 8, 3000),
                        [448, -448, 2 ** -9, 2 ** -10, 3 * 2 ** -10, 0.0, 1.0625, 1.1875, 15.5]]).astype(np.float32)
    x = x[np.abs(x) <= 448]  # torch's cast is not saturating: compare in range only
    ref_q = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.e4m3_encode(x), ref_q)
    # saturating form: beyond the largest finite value (and infinities) -> +-448
    assert list(oracle.e4m3_encode(np.array([500, -1e6, np.inf], np.float32))) == [0x7E, 0xFE, 0x7E]


def test_quantised_cache_close_to_fp32(tiny_arrays):
    """FP16 and FP8 caches render close to the FP32 one (property, any size)."""
    sig, uvw, beta = tiny_arrays
    w = scenegen.tiny()
    p = oracle.params_struct(w.n_samples)
    cam = w.cameras()[0]
    ref, _, _ = oracle.render_image(oracle.Cache(w.k, w.D, w.l, sig, uvw, beta), cam, p)
    for prec, min_psnr in ((oracle.FP16, 55.0), (oracle.FP8, 25.0)):
        q = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, oracle.FP16)
        img, _, _ = oracle.render_image(q, cam, p)
        mse = np.mean((img[..., :3] - ref[..., :3]) ** 2)
        assert 10 * math.log10(1 / mse) > min_psnr


# ------------------------------------------------------------------ MLP pieces
def test_posenc_closed_form():
    x = np.array([[0.0, 0.5, -0.25]])
    e = oracle.posenc(x, 3, 20)
    want = []
    for v in x[0]:
        for j in range(3):
            want += [math.sin(2 ** j * math.pi * v), math.cos(2 ** j * math.pi * v)]
    np.testing.assert_allclose(e[0, :18], want, atol=1e-15)
    assert np.all(e[0, 18:] == 0)
    assert e[0, 0] == 0.0 and e[0, 1] == 1.0


def test_mlp_forward_vs_numpy():
    rng = np.random.default_rng(2)
    dims = [12, 16, 16, 5]
    Ws = [rng.standard_normal((dims[i + 1], dims[i])) for i in range(3)]
    bs = [rng.standard_normal(dims[i + 1]) for i in range(3)]
    x = rng.standard_normal((40, 12))
    h = x
    for i in range(3):
        h = h @ Ws[i].T + bs[i]
        if i < 2:
            h = np.maximum(h, 0)
    np.testing.assert_allclose(oracle.mlp_forward(Ws, bs, x, False), h, rtol=1e-12, atol=1e-12)
    # bf16 rounding mode stays within bf16 error of the exact chain
    hb = oracle.mlp_forward(Ws, bs, x, True)
    assert np.max(np.abs(hb - h)) < 0.05 * np.max(np.abs(h))


def test_round_bf16_vs_torch_and_by_hand():
    """The oracle's activation rounding: binary32 first, then bfloat16, both round to nearest even.

    Hand-worked values near 1 (bf16 spacing 2^-7 there): 1 + 2^-8 is a tie between 1 and 1 + 2^-7 and goes
    to the even 1; 1 + 3 * 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6 and goes to the even 1 + 2^-6;
    1 + 2^-8 + 2^-20 lies above the tie and rounds up. An FP64 value first rounds to binary32, so
    1 + 2^-8 + 2^-40 becomes the tie 1 + 2^-8 and then 1 (direct rounding would give 1 + 2^-7).
    Then bit-for-bit against torch's float32 -> bfloat16 cast on random values, ties and subnormals."""
    torch = pytest.importorskip("torch")
    hand = [(1 + 2 ** -8, 1.0), (1 + 3 * 2 ** -8, 1 + 2 ** -6), (1 + 2 ** -8 + 2 ** -20, 1 + 2 ** -7),
            (-(1 + 3 * 2 ** -8), -(1 + 2 ** -6)), (1 + 2 ** -8 + 2 ** -40, 1.0), (2 ** -130, 2 ** -130),
            (3.0 * 2 ** -133 + 2 ** -149, 3.0 * 2 ** -133), (0.1, 0.10009765625), (-0.0, -0.0), (65504.0, 65536.0)]
    got = oracle.round_bf16([v for v, _ in hand])
    for (v, want), g in zip(hand, got):
        assert g == want and math.copysign(1, g) == math.copysign(1, want), (v, g, want)
    rng = np.random.default_rng(5)
    mant = rng.integers(0, 2 ** 23, 4000, dtype=np.uint32)
    expo = rng.integers(1, 255, 4000, dtype=np.uint32)
    sign = rng.integers(0, 2, 4000, dtype=np.uint32)
    bits = (sign << 31) | (expo << 23) | mant
    ties = (bits & ~np.uint32(0xFFFF)) | np.uint32(0x8000)      # exactly halfway between two bf16 values
    subn = rng.integers(1, 2 ** 23, 1000, dtype=np.uint32)      # binary32 subnormals
    x = np.concatenate([bits, ties, subn]).view(np.float32)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(x), ref)
    special = oracle.round_bf16([np.inf, -np.inf, np.nan])
    assert special[0] == np.inf and special[1] == -np.inf and np.isnan(special[2])


def test_mlp_rounds_input_and_hidden_but_not_head():
    """round_bf16 mode rounds the encoded input and every hidden activation to bf16, never the head's
    outputs: with identity layers, input 1 + 2^-9 reaches the head as 1 (rounded), and a head bias of 2^-12
    survives unrounded; the FP64 mode keeps everything."""
    I2 = np.eye(2)
    Ws, bs = [I2, I2], [np.zeros(2), np.array([2.0 ** -12, 0.0])]
    x = np.array([[1 + 2 ** -9, 3.0]])
    assert list(oracle.mlp_forward(Ws, bs, x, True)[0]) == [1 + 2 ** -12, 3.0]
    assert list(oracle.mlp_forward(Ws, bs, x, False)[0]) == [1 + 2 ** -9 + 2 ** -12, 3.0]
    # a hidden pre-activation that needs rounding: 1 + 2^-9 + 2^-9 = 1 + 2^-8 is a tie -> 1
    Ws2 = [np.array([[1.0, 1.0]]), np.array([[1.0]])]
    bs2 = [np.zeros(1), np.zeros(1)]
    x2 = np.array([[1.0, 2.0 ** -8]])
    assert oracle.mlp_forward(Ws2, bs2, x2, True)[0, 0] == 1.0


def test_fp8_scale_and_codes_by_definition():
    """Per-channel E4M3 quantisation (one binary32 scale per channel = absmax / 448, 1 for an all-zero
    channel; q = E4M3(x / scale), nearest even, saturating; the density channel is clamped to >= 0 first).

    Hand-worked channel {0, 1.5, -7, 3.5}: absmax 7, scale = 7/448 = 2^-6 exactly; x / scale =
    {0, 96, -448, 224} -> codes {0x00, 0x6C (1.5 * 2^6: exponent field 13, mantissa 4), 0xFE (-448),
    0x76 (1.75 * 2^7: exponent field 14, mantissa 6)}. As a density channel the -7 is clamped to 0 first:
    absmax 3.5, scale 2^-7, codes {0x00, 0x74 (192), 0x00, 0x7E (448)}."""
    ch = np.array([0.0, 1.5, -7.0, 3.5], np.float32)
    s_u = oracle.fp8_scale(ch, False)
    assert s_u == np.float32(7.0 / 448.0) == 2.0 ** -6
    assert list(oracle.quantize_channel(oracle.FP8, ch, False, s_u)) == [0x00, 0x6C, 0xFE, 0x76]
    s_s = oracle.fp8_scale(ch, True)
    assert s_s == 2.0 ** -7
    assert list(oracle.quantize_channel(oracle.FP8, ch, True, s_s)) == [0x00, 0x74, 0x00, 0x7E]
    assert oracle.fp8_scale(np.zeros(5, np.float32), False) == 1.0
    assert oracle.fp8_scale(np.array([-3.0, 0.0], np.float32), True) == 1.0  # clamped to all zero
    # random channels: the absmax element encodes to +-448, nothing else saturates, and every code
    # decodes to within half an E4M3 step of x / scale
    rng = np.random.default_rng(3)
    for trial in range(20):
        x = (rng.standard_normal(500) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        s = oracle.fp8_scale(x, False)
        assert s == np.float32(np.float32(np.max(np.abs(x))) / np.float32(448.0))
        q = oracle.quantize_channel(oracle.FP8, x, False, s)
        a = int(np.argmax(np.abs(x)))
        assert q[a] == (0xFE if x[a] < 0 else 0x7E)
        y = (x / s).astype(np.float32).astype(np.float64)
        assert np.all(np.abs(y) <= 448.0 * (1 + 2 ** -23))
        dec = oracle.e4m3_decode(q)
        step = np.where(np.abs(y) < 2 ** -6, 2.0 ** -9, 2.0 ** (np.floor(np.log2(np.maximum(np.abs(y), 2 ** -6))) - 3))
        assert np.all(np.abs(dec - y) <= step / 2 * (1 + 1e-12))


def test_fp8_cache_by_hand():
    """quantize_cache for E4M3: the density plane is clamped and scaled as one channel (no offset); each
    (u, v, w) channel is stored as the residual from its offset brick's binary16 midrange, one binary32 scale
    per channel = absmax residual / 448.

    k = 2 (one offset brick of Bo = 4 cells). Channel 0 = {0, 1.5, -7, 3.5, 0, 0, 0, 0}: midrange
    (-7 + 3.5) / 2 = -1.75, residuals {1.75, 3.25, -5.25, 5.25, 1.75, ...}, scale 5.25 / 448 = 3/256;
    r / scale = {149.33, 277.33, -448, 448, 149.33, ...} -> codes {0x71 (144: exponent field 14,
    mantissa 1), 0x79 (288: exponent field 15, mantissa 1), 0xFE, 0x7E, 0x71, ...}. Channel 1 = {-2, 0, ...}:
    midrange -1, residuals {-1, 1, ...}, scale 1/448, codes {0xFE, 0x7E, ...}. Channel 2 all zero: offset 0,
    scale 1, codes 0. The stored value of cell 0, channel 0 is -1.75 + 144 * 3/256 = -0.0625."""
    k, D, l = 2, 1, 2
    sig = np.array([0, 1.5, -7, 3.5, 0, 0, 0, 0], np.float32)
    uvw = np.zeros((8, 3), np.float32)
    uvw[:4, 0] = [0, 1.5, -7, 3.5]
    uvw[0, 1] = -2.0
    beta = np.ones((l * l, D), np.float32)
    q = oracle.quantize_cache(k, D, l, sig, uvw, beta, oracle.FP8, oracle.FP16)
    assert q.off_brick == 4
    assert list(q.offsets) == [0xBF00, 0xBC00, 0x0000]  # binary16 -1.75, -1, 0
    assert q.scales[0] == 2.0 ** -7 and q.scales[1] == 3.0 / 256 and q.scales[3] == 1.0
    assert q.scales[2] == np.float32(np.float32(1.0) / np.float32(448.0))
    assert list(np.asarray(q.sigma)) == [0x00, 0x74, 0x00, 0x7E, 0, 0, 0, 0]
    qu = np.asarray(q.uvw).reshape(8, 3)
    assert list(qu[:, 0]) == [0x71, 0x79, 0xFE, 0x7E, 0x71, 0x71, 0x71, 0x71]
    assert list(qu[:, 1]) == [0xFE] + [0x7E] * 7
    assert list(qu[:, 2]) == [0] * 8
    # the oracle renders the exact stored value: with density only in cell 0, identity activation and
    # beta = 1, a ray through cell 0 has colour (stored u, v, w of cell 0) (1 - T) + T bg
    sig1 = np.array([50, 0, 0, 0, 0, 0, 0, 0], np.float32)
    q1 = oracle.quantize_cache(k, D, l, sig1, uvw, beta, oracle.FP8, oracle.FP16)
    s1 = np.asarray(q1.scales, np.float64)
    stored = [-1.75 + s1[1] * 144, -1.0 - s1[2] * 448, 0.0]
    cam = dict(c2w=np.array([1, 0, 0, -0.75, 0, 1, 0, -0.75, 0, 0, 1, 4], np.float32), fx=np.float32(10.0),
               fy=np.float32(10.0), cx=np.float32(0.5), cy=np.float32(0.5), W=1, H=1)
    bg = (0.25, 0.5, 0.75)
    rgba, st, _ = oracle.render_pixels(q1, cam, oracle.params_struct(64, 2.0, 6.0, 0.0, bg, oracle.ACT_IDENTITY),
                                       [0], [0])
    m = st[0, 2]
    assert m == 24  # samples at z = 2 - (i + 1/2) / 16 inside [-1.5, 0): i = 32 .. 55
    sigma_stored = float(np.float32(448.0) * np.float32(s1[0]))  # binary32 product of code 0x7E and the scale
    T = math.exp(-sigma_stored * m / 16)                          # Delta = 4 / 64
    np.testing.assert_allclose(rgba[0, :3], np.array(stored) * (1 - T) + T * np.array(bg), rtol=0, atol=1e-12)
    assert oracle.offset_brick(64) == 4 and oracle.offset_brick(256) == 4 and oracle.offset_brick(512) == 8
    assert oracle.offset_brick(1024) == 16 and oracle.offset_brick(1290) == 32


def test_fp8_offsets_and_residual_bound():
    """Any grid: each offset is the binary16 value of a number between the brick's min and max (so the
    residuals of a brick straddle 0), the largest residual of each channel codes to +-448, and every stored
    value (offset + scale * e4m3(code)) is within half an E4M3 step (times the scale) of the input."""
    rng = np.random.default_rng(4)
    for k, D in ((6, 2), (9, 1), (16, 3)):
        uvw = (rng.standard_normal((k ** 3, 3 * D)) * 3 + rng.uniform(-5, 5, 3 * D)).astype(np.float32)
        sig = np.abs(rng.standard_normal(k ** 3)).astype(np.float32)
        q = oracle.quantize_cache(k, D, 4, sig, uvw, np.ones((16, D), np.float32), oracle.FP8, oracle.FP32)
        Bo = q.off_brick
        nbo = -(-k // Bo)
        off = oracle.f16_decode(q.offsets).reshape(nbo, nbo, nbo, 3 * D)
        idx = np.arange(k ** 3)
        x, y, z = idx % k, (idx // k) % k, idx // (k * k)
        m = off[z // Bo, y // Bo, x // Bo]            # [k^3, 3D] offset of each cell
        U = uvw.reshape(k, k, k, 3 * D)
        for bz in range(nbo):
            for by in range(nbo):
                for bx in range(nbo):
                    blk = U[bz * Bo:(bz + 1) * Bo, by * Bo:(by + 1) * Bo, bx * Bo:(bx + 1) * Bo].reshape(-1, 3 * D)
                    o = off[bz, by, bx]
                    assert np.all(o >= blk.min(0) - np.abs(blk.min(0)) * 2 ** -10)
                    assert np.all(o <= blk.max(0) + np.abs(blk.max(0)) * 2 ** -10)
        codes = np.asarray(q.uvw).reshape(k ** 3, 3 * D)
        dec = oracle.e4m3_decode(codes.reshape(-1)).reshape(codes.shape)
        r = (uvw - m.astype(np.float32)).astype(np.float32).astype(np.float64)
        s = q.scales[1:].astype(np.float64)
        for c in range(3 * D):
            a = int(np.argmax(np.abs(r[:, c])))
            assert codes[a, c] == (0xFE if r[a, c] < 0 else 0x7E)
        y_ = np.abs(r / s)
        step = np.where(y_ < 2 ** -6, 2.0 ** -9, 2.0 ** (np.floor(np.log2(np.maximum(y_, 2 ** -6))) - 3))
        stored = m + s * dec
        assert np.all(np.abs(stored - uvw) <= (step / 2) * s * (1 + 1e-6) + 1e-12)


def test_build_sample_points_by_hand():
    """The cache build evaluates F_pos at cell centres and F_dir at bin centres (Section 3.3; reading s5,
    s15). k = 2 on [-1.5, 1.5]^3: centres +-0.75, cell (z*2 + y)*2 + x; k = 3: centres -1, 0, 1.
    l = 2: theta centres pi/4, 3 pi/4 (from +z), phi centres pi/2, 3 pi/2; bin i_theta * 2 + i_phi."""
    c = oracle.cell_centres(2, [0, 1, 2, 4, 7])
    assert c.tolist() == [[-0.75, -0.75, -0.75], [0.75, -0.75, -0.75], [-0.75, 0.75, -0.75],
                          [-0.75, -0.75, 0.75], [0.75, 0.75, 0.75]]
    c3 = oracle.cell_centres(3, [0, 5, 13, 26])
    np.testing.assert_allclose(c3, [[-1, -1, -1], [1, 0, -1], [0, 0, 0], [1, 1, 1]], atol=1e-15)
    h = math.sqrt(0.5)
    dirs = oracle.bin_directions(2, [0, 1, 2, 3])
    np.testing.assert_allclose(dirs, [[0, h, h], [0, -h, h], [0, h, -h], [0, -h, -h]], atol=1e-15)
    # each bin centre's direction is looked up in its own bin (the lookup is pinned against libm
    # separately), for several resolutions
    for l in (2, 3, 8, 64, 512):
        bins = np.arange(l * l) if l <= 64 else np.random.default_rng(l).integers(0, l * l, 4000)
        for b, d in zip(bins, oracle.bin_directions(l, bins)):
            it, ip = oracle.dir_cell(l, d.astype(np.float32))
            assert it * l + ip == b, (l, b, it, ip)


def test_tabled_field_equals_dense(tiny_workload, tiny_arrays):
    """The cell-table accessor (dense sigma, uvw only for the cells rays shade) is storage only: it gives
    the dense FP32 render bit for bit, and asks for exactly the occupied cells that rays reach."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cam = w.cameras()[0]
    p = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    dense = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    py, px = np.meshgrid(np.arange(w.H, dtype=np.int32), np.arange(w.W, dtype=np.int32), indexing="ij")
    px, py = px.reshape(-1), py.reshape(-1)
    ref, ref_st, cells = oracle.render_pixels(dense, cam, p, px, py, want_cells=True)
    flat_uvw = uvw.reshape(-1, 3 * w.D)
    asked = []

    def records(c):
        asked.append(c.copy())
        return flat_uvw[c]

    got, st, n_cells = oracle.render_pixels_tabled(w.k, w.D, w.l, sig.reshape(-1), beta, records, cam, p, px, py)
    assert np.array_equal(got, ref) and np.array_equal(st, ref_st)
    c = cells.reshape(-1)
    c = c[c >= 0]
    expect = np.unique(c[sig.reshape(-1)[c] > 0])
    assert n_cells == expect.size > 0 and np.array_equal(asked[0], expect)
    # a cell left out of the table is counted, not rendered silently wrong
    import ctypes
    drop = expect[1:]
    rec = np.ascontiguousarray(flat_uvw[drop])
    t = oracle._Table()
    sflat = np.ascontiguousarray(sig.reshape(-1))
    t.sigma, t.n, t.cells, t.rec, t.nch, t.missing = sflat.ctypes.data, drop.size, drop.ctypes.data, \
        rec.ctypes.data, 3 * w.D, 0
    fn = ctypes.cast(oracle.lib().orc_table_field, ctypes.c_void_p).value
    c = oracle.Cache(w.k, w.D, w.l, None, None, beta, field=(fn, ctypes.addressof(t)))
    oracle.render_pixels(c, cam, p, px, py)
    assert t.missing > 0


def test_brick_occupancy_brute_force():
    """Brick occupancy against a per-brick loop over its cells, with a ragged last brick (k % B != 0)."""
    k, B = 10, 4
    rng = np.random.default_rng(5)
    pos = rng.random(k ** 3) < 0.01
    occ = oracle.brick_occupancy(k, B, pos)
    nb = 3
    P = pos.reshape(k, k, k)
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                want = any(P[z, y, x] for z in range(bz * B, min(k, bz * B + B))
                           for y in range(by * B, min(k, by * B + B)) for x in range(bx * B, min(k, bx * B + B)))
                assert occ[(bz * nb + by) * nb + bx] == int(want)


@pytest.mark.parametrize("brick", [1, 2, 4, 8])
def test_skip_empty_same_image_fewer_lookups(tiny_workload, tiny_arrays, brick):
    """Skipping samples in empty bricks changes nothing but the lookup count, which equals the number of
    visited in-box samples (the plain render's per-sample cells) whose brick holds density."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cam = w.cameras()[0]
    c = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta).set_occupancy(brick)
    p = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    ps = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg, skip_empty=True)
    ref, st, cells = oracle.render_image(c, cam, p, want_cells=True)
    got, st2, cells2 = oracle.render_image(c, cam, ps, want_cells=True)
    assert np.array_equal(got, ref)
    assert np.array_equal(st[..., [0, 2, 3]], st2[..., [0, 2, 3]]) and np.array_equal(cells, cells2)
    k, nb = w.k, (w.k + brick - 1) // brick
    cz, cy, cx = cells // (k * k), (cells // k) % k, cells % k
    b = ((cz // brick) * nb + cy // brick) * nb + cx // brick
    occ = oracle.brick_occupancy(k, brick, sig.reshape(-1) > 0)
    expect = ((cells >= 0) & (occ[np.where(cells >= 0, b, 0)] == 1)).sum(axis=-1)
    assert np.array_equal(st2[..., 1], expect)
    assert (st2[..., 1] <= st[..., 1]).all()
    if brick == 1:  # single-cell bricks: only occupied samples are looked up
        assert np.array_equal(st2[..., 1], st2[..., 2])
    assert st2[..., 1].sum() < st[..., 1].sum()


def test_unique_sector_count_brute_force(tiny_workload, tiny_arrays):
    """bench.py's unique-bytes figure against sets of sector indices built sample by sample."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cam = w.cameras()[0]
    got = bench.unique_sector_bytes(w, sig, uvw, beta, cam)
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    _, st, cells = oracle.render_image(oc, cam, oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg),
                                       want_cells=True)
    dens, recs, betas = set(), set(), set()
    sflat = sig.reshape(-1)
    for c in cells.reshape(-1).tolist():
        if c < 0:
            continue
        dens.add((4 * c) // 32)
        if sflat[c] > 0:
            for b in range(96 * c, 96 * c + 96):
                recs.add(b // 32)
    for d in st[..., 3].reshape(-1).tolist():
        for b in range(32 * d, 32 * d + 32):
            betas.add(b // 32)
    assert (got["density_sectors"], got["record_sectors"], got["beta_sectors"]) == (len(dens), len(recs), len(betas))


def _dir(theta, phi):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], dtype=np.float32)


def _angles(d):
    x, y, z = (float(v) for v in d)
    th = math.atan2(math.hypot(x, y), z)
    ph = math.atan2(y, x)
    return th, ph + 2 * math.pi if ph < 0 else ph


def test_beta_bilinear_reproduces_linear_fields_and_centres():
    """Bilinear interpolation in (theta, phi): exact at bin centres and for fields linear in the angles
    between the first and last bin centres; a field of theta alone is clamped beyond the polar centres."""
    l, D = 16, 3
    th_c = (np.arange(l) + 0.5) * np.pi / l
    ph_c = (np.arange(l) + 0.5) * 2 * np.pi / l
    coef = np.array([[0.7, -0.2, 0.1], [0.3, 0.05, -1.0], [-0.4, 0.6, 0.25]])  # beta_i = a th + b ph + c
    grid = (coef[None, None, :, 0] * th_c[:, None, None] + coef[None, None, :, 1] * ph_c[None, :, None] +
            coef[None, None, :, 2]).astype(np.float64)
    c = oracle.Cache(2, D, l, np.zeros(8, np.float32), np.zeros(8 * 3 * D, np.float32), grid.astype(np.float32))
    g32 = grid.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(8)
    for _ in range(200):
        d = _dir(rng.uniform(th_c[0], th_c[-1]), rng.uniform(ph_c[0], ph_c[-1]))
        th, ph = _angles(d)
        want = coef[:, 0] * th + coef[:, 1] * ph + coef[:, 2]
        # the grid holds binary32 values: compare with the interpolant of those
        assert np.allclose(oracle.beta_bilinear(c, d), want, atol=2e-6)
    for i, j in [(0, 0), (5, 9), (15, 15), (7, 0)]:
        got = oracle.beta_bilinear(c, _dir(th_c[i], ph_c[j]))
        assert np.allclose(got, g32[i, j], atol=1e-5)
    # theta-only field: above the first centre (towards +z) the first row is used as is
    rows = np.repeat(np.arange(l, dtype=np.float32)[:, None, None], l, axis=1).repeat(D, axis=2)
    cr = oracle.Cache(2, D, l, np.zeros(8, np.float32), np.zeros(8 * 3 * D, np.float32), rows)
    assert np.allclose(oracle.beta_bilinear(cr, _dir(0.3 * th_c[0], 1.0)), 0.0)
    assert np.allclose(oracle.beta_bilinear(cr, _dir(np.pi - 0.3 * th_c[0], 4.0)), l - 1)


def test_beta_bilinear_wraps_in_phi():
    """Between the last and the first azimuth centre the weights wrap around 2 pi."""
    l, D = 8, 1
    grid = np.zeros((l, l, D), np.float32)
    grid[:, 0, 0] = 1.0  # bin 0 in phi
    c = oracle.Cache(2, D, l, np.zeros(8, np.float32), np.zeros(8 * 3, np.float32), grid)
    th = np.pi / 2
    w = 2 * np.pi / l
    for frac in (0.1, 0.5, 0.9):  # phi between the centre of bin l-1 and 2 pi + centre of bin 0
        ph = (l - 0.5) * w + frac * w
        got = oracle.beta_bilinear(c, _dir(th, ph % (2 * np.pi)))[0]
        assert abs(got - frac) < 1e-5, (frac, got)


def test_bilinear_render_with_constant_beta_equals_nearest(tiny_workload, tiny_arrays):
    w = tiny_workload
    sig, uvw, _ = tiny_arrays
    beta = np.broadcast_to(np.linspace(-1, 1, w.D, dtype=np.float32), (w.l, w.l, w.D)).copy()
    c = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    cam = w.cameras()[0]
    a = oracle.render_image(c, cam, oracle.params_struct(w.n_samples))
    b = oracle.render_image(c, cam, oracle.params_struct(w.n_samples, dir_bilinear=True))
    assert np.array_equal(a[1], b[1]) and np.allclose(a[0], b[0], atol=1e-12)


def _const_mlp(dims, head_bias, hidden_bias=0.25):
    """An MLP with zero weights: every output is its head bias, whatever the input."""
    layers = []
    for i, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
        bias = np.full(b, hidden_bias) if i + 1 < len(dims) - 1 else np.asarray(head_bias, np.float64)
        layers.append((np.zeros((b, a)), bias))
    return layers


@pytest.mark.parametrize("round_bf16", [False, True])
def test_uncached_render_homogeneous_closed_form(round_bf16):
    """Position-independent F_pos (sigma0, constant u, v, w) and F_dir (constant beta): each ray is a
    homogeneous medium over its inside samples, C = c (1 - e^{-sigma0 m Delta}) + e^{-sigma0 m Delta} bg with
    m = the inside samples up to the integer termination and c = sigmoid(sum_i beta_i (u_i, v_i, w_i))."""
    D = 2
    sigma0 = 3.0
    head = [sigma0, 0.5, -0.25, 1.0, 0.75, -1.5, 0.125]  # sigma, u1 u2, v1 v2, w1 w2
    pos = _const_mlp([60, 32, 32, 1 + 3 * D], head)
    dirn = _const_mlp([24, 16, D], [1.0, -0.5])
    cam = scenegen.cameras(9, 1, 24, 20, fov_deg=100.0)[0]  # wide: some rays miss the box
    N, near, far, t_thr = 64, 2.0, 6.0, 1e-3
    p = oracle.params_struct(N, near, far, t_thr, (1.0, 1.0, 1.0))
    py, px = np.meshgrid(np.arange(20, dtype=np.int32), np.arange(24, dtype=np.int32), indexing="ij")
    px, py = px.reshape(-1), py.reshape(-1)
    rgba, st = oracle.render_mlp_pixels(pos, dirn, D, cam, p, px, py, round_bf16=round_bf16)
    dt = oracle.dt(near, far, N)
    sthr = oracle.s_thr(t_thr, dt)
    m_thr = -(-sthr // oracle.fix(sigma0))
    u = np.array(head[1:]).reshape(3, D)
    c = 1.0 / (1.0 + np.exp(-(u @ np.array([1.0, -0.5]))))
    pts = np.zeros((px.size, N, 3), np.float32)
    inside = np.zeros((px.size, N), np.uint8)
    dirs = np.zeros((px.size, 3), np.float32)
    lo, hi = np.full(3, -1.5, np.float32), np.full(3, 1.5, np.float32)
    oracle.lib().orc_mlp_samples(ctypes.byref(oracle.camera_struct(cam)), ctypes.byref(p), lo.ctypes.data,
                                 hi.ctypes.data, px.size, px.ctypes.data, py.ctypes.data, pts.ctypes.data,
                                 inside.ctypes.data, dirs.ctypes.data)
    n_in = inside.sum(axis=1)
    m = np.minimum(n_in, m_thr)
    ext = np.exp(-sigma0 * m * dt)
    want = c[None, :] * (1 - ext[:, None]) + ext[:, None]
    assert np.allclose(rgba[:, :3], want, atol=1e-12) and np.allclose(rgba[:, 3], 1 - ext, atol=1e-12)
    assert np.array_equal(st[:, 1], m) and np.array_equal(st[:, 2], m)
    assert (n_in > m_thr).any() and (n_in == 0).any() and ((n_in > 0) & (n_in < m_thr)).any()
    # inside counts against FP64 ray-box clipping (binary32 positions may move a boundary sample)
    for r in range(0, px.size, 7):
        d, o = dirs[r].astype(np.float64), np.asarray(cam["c2w"], np.float64).reshape(3, 4)[:, 3]
        t = near + (np.arange(N) + 0.5) * dt
        q = o[None, :] + t[:, None] * d[None, :]
        exact = int(((q >= -1.5) & (q < 1.5)).all(axis=1).sum())
        assert abs(exact - int(n_in[r])) <= 1


# ------------------------------------------------------------------ voxel walk (Section 4: every voxel visited)
def _slab_cells_fp64(k, o, d, t_near, t_far, bmin=(-1.5, -1.5, -1.5), bmax=(1.5, 1.5, 1.5)):
    """Brute force: every cell's parameter interval on the ray, FP64 slabs in world units."""
    o = np.asarray(o, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    lo_b = np.asarray(bmin, dtype=np.float64)
    h = (np.asarray(bmax, dtype=np.float64) - lo_b) / k
    out = []
    for iz in range(k):
        for iy in range(k):
            for ix in range(k):
                c = np.array([ix, iy, iz], dtype=np.float64)
                t0, t1 = t_near, t_far
                for a in range(3):
                    b0, b1 = lo_b[a] + c[a] * h[a], lo_b[a] + (c[a] + 1) * h[a]
                    if d[a] == 0.0:
                        if not (b0 <= o[a] < b1):
                            t0, t1 = 1.0, 0.0
                        continue
                    ta, tb = (b0 - o[a]) / d[a], (b1 - o[a]) / d[a]
                    t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
                if t1 > t0:
                    out.append((t0, t1 - t0, (iz * k + iy) * k + ix))
    out.sort()
    return out


@pytest.mark.parametrize("k", [5, 7])
def test_voxel_walk_vs_fp64_slabs(k):
    """The walk visits exactly the cells the FP64 ray meets, in ray order, each with its FP64 length; cells
    the ray only grazes (length < 1e-4, within rounding of a corner or an edge) may appear either way."""
    rng = np.random.default_rng(k)
    n_rays = 0
    for trial in range(300):
        if trial % 3 == 0:  # from inside the box
            o = rng.uniform(-1.4, 1.4, 3)
        else:
            o = rng.normal(size=3)
            o = 4.0 * o / np.linalg.norm(o)
        d = rng.normal(size=3)
        if trial % 10 == 1:
            d[rng.integers(0, 3)] = 0.0  # a ray parallel to a face
        d = d / np.linalg.norm(d)
        o32, d32 = o.astype(np.float32), d.astype(np.float32)
        t_near, t_far = (0.0, 10.0) if trial % 4 else (0.5, 3.5)
        cells, delta = oracle.voxel_walk(k, o32, d32, t_near, t_far, 4 * k)
        ref = _slab_cells_fp64(k, o32, d32, t_near, t_far)
        big_ref = [(c, L) for _, L, c in ref if L > 1e-4]
        big = [(c, float(dl)) for c, dl in zip(cells, delta) if dl > 1e-4]
        assert [c for c, _ in big] == [c for c, _ in big_ref], (trial, cells, ref)
        for (_, dl), (_, L) in zip(big, big_ref):
            assert abs(dl - L) < 2e-5, (trial, dl, L)
        assert abs(float(np.sum(delta[delta > 0], dtype=np.float64)) - sum(L for _, L, _ in ref)) < 5e-5
        # consecutive cells are face neighbours (one step along one axis)
        xyz = np.stack([cells % k, (cells // k) % k, cells // (k * k)], axis=1)
        if len(cells) > 1:
            assert np.all(np.abs(np.diff(xyz, axis=0)).sum(axis=1) == 1)
        n_rays += len(cells) > 0
    assert n_rays > 100


@pytest.mark.parametrize("sigma0,t_thr", [(0.7, 0.0), (3.0, 0.0), (50.0, 1e-4), (9.0, 1e-3)])
def test_voxel_homogeneous_box_closed_form(sigma0, t_thr):
    """All cells sigma0, colour c, voxel walk: C = c (1 - e^{-sigma0 L}) + e^{-sigma0 L} bg with L the sum of the
    cells' lengths (the FP64 chord through the box without termination); with termination the walk stops at
    the first cell where sum floor(fp32(sigma0 delta) 2^32) >= ceil(ln(1/T_thr) 2^32)."""
    k, D, l = 16, 1, 8
    c = np.array([0.3, 0.5, 0.7], dtype=np.float32).astype(np.float64)
    cache = const_cache(k, D, l, sigma0, c, [1.0])
    cam = scenegen.cameras(5, 1, 24, 16)[0]
    bg = np.array([0.9, 0.2, 0.4], dtype=np.float32).astype(np.float64)
    N = 3 * k
    p = oracle.params_struct(N, 2.0, 6.0, t_thr, tuple(bg), oracle.ACT_IDENTITY, voxels=True)
    rgba, st, cells = oracle.render_image(cache, cam, p, want_cells=True)
    s_thr = oracle.lib().orc_s_thr(t_thr, 1.0)
    checked = 0
    for py in range(0, 16, 3):
        for px in range(0, 24, 3):
            d, o = oracle.ray(cam, px, py)
            wc, wd = oracle.voxel_walk(k, o, d, 2.0, 6.0, N)
            m = len(wc)
            if t_thr > 0:
                S = 0
                for j in range(len(wc)):
                    S += oracle.lib().orc_fix(float(np.float32(np.float32(sigma0) * wd[j])))
                    if S >= s_thr:
                        m = j + 1
                        break
            assert st[py, px, 0] == m
            assert np.array_equal(cells[py, px, :m], wc[:m])
            L = float(np.sum(wd[:m][wd[:m] > 0], dtype=np.float64))
            s0 = float(np.float32(sigma0))  # the stored binary32 density
            TL = math.exp(-s0 * L)
            np.testing.assert_allclose(rgba[py, px, :3], c * (1 - TL) + TL * bg, rtol=0, atol=1e-12)
            if t_thr == 0.0 and m > 0:
                chord = sum(Lc for _, Lc, _ in _slab_cells_fp64(k, o, d, 2.0, 6.0))
                assert abs(L - chord) < 5e-5
            if t_thr > 0 and m < len(wc):
                assert TL < t_thr * (1 + 1e-6)
                L_prev = float(np.sum(wd[:m - 1][wd[:m - 1] > 0], dtype=np.float64))
                assert math.exp(-s0 * L_prev) >= t_thr * (1 - 1e-6)
            checked += m > 0
    assert checked > 10


def test_voxel_skip_and_empty(tiny_workload, tiny_arrays):
    """Voxel walk: skipping empty bricks changes only the lookup count; an empty cache gives T = 1 and C = bg."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, oracle.FP32, oracle.FP32).set_occupancy(4)
    cam = w.cameras()[0]
    N = 3 * w.k
    p = oracle.params_struct(N, voxels=True)
    ps = oracle.params_struct(N, voxels=True, skip_empty=True)
    a = oracle.render_image(cache, cam, p, want_cells=True)
    b = oracle.render_image(cache, cam, ps, want_cells=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[1][..., [0, 2, 3]], b[1][..., [0, 2, 3]])
    assert (b[1][..., 1] <= a[1][..., 1]).all() and (b[1][..., 1] < a[1][..., 1]).any()
    assert (a[1][..., 2] > 0).any()
    empty = oracle.quantize_cache(w.k, w.D, w.l, np.zeros_like(sig), uvw, beta, oracle.FP32, oracle.FP32)
    r = oracle.render_image(empty, cam, oracle.params_struct(N, bg=(0.25, 0.5, 1.0), voxels=True))
    assert np.all(r[0][..., :3] == np.array([0.25, 0.5, 1.0], np.float32)) and np.all(r[0][..., 3] == 0)
    assert np.all(r[1][..., 2] == 0)


def test_voxel_walk_hand_cases():
    """Walks worked out by hand in a k=4 box over [-1.5, 1.5)^3 (cells 0.75 wide): an axis-aligned ray, the
    same ray cut by [t_near, t_far], a ray starting inside the box, one along -x, and one that misses."""
    k = 4
    idx = lambda x, y, z: (z * k + y) * k + x  # noqa: E731
    # +z through x = y = 0 (cell 2 on both axes): enters at t = 3.5 (z = -1.5), four cells of 0.75
    c, d = oracle.voxel_walk(k, [0.0, 0.0, -5.0], [0.0, 0.0, 1.0], 0.0, 10.0, 16)
    assert list(c) == [idx(2, 2, z) for z in range(4)] and np.allclose(d, 0.75, atol=1e-6)
    # the same ray on [4.0, 5.5]: z from -1.0 to 0.5 -> cells z = 0 (0.25 left), 1 (0.75), 2 (0.5)
    c, d = oracle.voxel_walk(k, [0.0, 0.0, -5.0], [0.0, 0.0, 1.0], 4.0, 5.5, 16)
    assert list(c) == [idx(2, 2, z) for z in range(3)] and np.allclose(d, [0.25, 0.75, 0.5], atol=1e-6)
    # from inside the box at z = 0.1 (cell 2, exit at 0.75 after 0.65), one more cell to 1.5
    c, d = oracle.voxel_walk(k, [0.2, -0.3, 0.1], [0.0, 0.0, 1.0], 0.0, 10.0, 16)
    assert list(c) == [idx(2, 1, 2), idx(2, 1, 3)] and np.allclose(d, [0.65, 0.75], atol=1e-6)
    # -x at y = z = -1.0 (cell 0): x from 1.5 down to -1.5, cells x = 3, 2, 1, 0
    c, d = oracle.voxel_walk(k, [3.0, -1.0, -1.0], [-1.0, 0.0, 0.0], 0.0, 10.0, 16)
    assert list(c) == [idx(x, 0, 0) for x in (3, 2, 1, 0)] and np.allclose(d, 0.75, atol=1e-6)
    # parallel to the box outside it: no cells
    c, d = oracle.voxel_walk(k, [2.0, 0.0, -5.0], [0.0, 0.0, 1.0], 0.0, 10.0, 16)
    assert len(c) == 0
    # the step cap
    c, d = oracle.voxel_walk(k, [0.0, 0.0, -5.0], [0.0, 0.0, 1.0], 0.0, 10.0, 2)
    assert list(c) == [idx(2, 2, 0), idx(2, 2, 1)]
