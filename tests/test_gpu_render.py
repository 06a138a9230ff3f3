"""GPU parity of fnr_render against the FP64 oracle, through the C ABI.

Bar: cell indices, direction cells, termination steps and sample counters
bit-exact; RGBA within 1e-5 absolute per channel (binary32 accumulation of
Eq. 5 and Eq. 1 against FP64; see the tolerance derivation in the design
notes). Quantised cache bytes (FP16 / FP8 and the FP8 scales) are compared
bit-exactly with the oracle's own quantiser.
"""

import math
import os

import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fnr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2103_10380_gb300 as fnr
    torch.cuda.set_device(0)
    return fnr


@pytest.fixture(scope="module")
def ctx(fnr):
    c = fnr.fnr_context_create(0, 0)
    yield c
    fnr.fnr_context_destroy(c)


def device_bytes(ptr: int, nbytes: int):
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_View(), device="cuda").cpu().numpy()


def gpu_render(fnr, ctx, cache, cams, params, with_cells=False, stream=None):
    import torch
    npix = sum(int(c["W"]) * int(c["H"]) for c in cams)
    rgba = torch.full((npix * 4,), float("nan"), device="cuda", dtype=torch.float32)
    stats = torch.full((npix * 4,), -7, device="cuda", dtype=torch.int32)
    cells = torch.full((npix * params.n_samples,), -9, device="cuda", dtype=torch.int32) if with_cells else None
    fnr.fnr_render(ctx, cache, cams, params, rgba, stats, cells, stream=stream)
    torch.cuda.synchronize()
    out = []
    off = 0
    for c in cams:
        W, H = int(c["W"]), int(c["H"])
        n = W * H
        out.append((rgba[off * 4:(off + n) * 4].cpu().numpy().reshape(H, W, 4),
                    stats[off * 4:(off + n) * 4].cpu().numpy().reshape(H, W, 4),
                    None if cells is None else
                    cells[off * params.n_samples:(off + n) * params.n_samples].cpu().numpy().reshape(H, W, -1)))
        off += n
    return out


def oparams(p):
    return oracle.params_struct(p.n_samples, p.t_near, p.t_far, p.t_thr, tuple(p.bg), p.activation,
                                skip_empty=bool(p.flags & 1), dir_bilinear=bool(p.flags & 2))


def compare(got, ref, tol=TOL):
    (g_rgba, g_st, g_cells), (r_rgba, r_st, r_cells) = got, ref
    assert np.array_equal(g_st, r_st), f"counters differ at {np.argwhere(g_st != r_st)[:5]}"
    if r_cells is not None:
        assert np.array_equal(g_cells, r_cells), f"cells differ at {np.argwhere(g_cells != r_cells)[:5]}"
    err = np.max(np.abs(g_rgba.astype(np.float64) - r_rgba))
    assert err <= tol, f"max |rgba - oracle| = {err}"
    return err


def build(fnr, ctx, k, D, l, sig, uvw, beta, prec=0, dprec=0, on_device=False):
    desc = fnr.make_desc(k, D, l, prec, dprec)
    arrs = [np.ascontiguousarray(a, dtype=np.float32).reshape(-1) for a in (sig, uvw, beta)]
    if on_device:
        import torch
        arrs = [torch.from_numpy(a).cuda() for a in arrs]
    return fnr.fnr_build_cache(ctx, desc, *arrs)


# ------------------------------------------------------------------ tiny workload, three storage precisions
@pytest.mark.parametrize("prec,dprec,on_device", [(0, 0, False), (0, 0, True), (1, 1, False), (1, 0, True),
                                                  (2, 1, False), (2, 0, True)])
def test_tiny_parity(fnr, ctx, tiny_workload, tiny_arrays, prec, dprec, on_device):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta, prec, dprec, on_device)
    try:
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, dprec)
        # stored bytes bit-exact against the oracle's quantiser
        lay = fnr.fnr_cache_get_layout(cache)
        es = {0: 4, 1: 2, 2: 1}[prec]
        k3 = w.k ** 3
        assert np.array_equal(device_bytes(lay.sigma_dev, k3 * es), oc.sigma.view(np.uint8))
        recs = device_bytes(lay.uvw_dev, k3 * lay.record_stride).reshape(k3, lay.record_stride)
        assert np.array_equal(recs[:, :3 * w.D * es], oc.uvw.reshape(k3, -1).view(np.uint8).reshape(k3, -1))
        bes = 2 if dprec == 1 else 4
        assert np.array_equal(device_bytes(lay.beta_dev, w.l * w.l * w.D * bes), oc.beta.view(np.uint8))
        if prec == 2:
            assert np.array_equal(device_bytes(lay.scales_dev, (1 + 3 * w.D) * 4).view(np.float32), oc.scales)
            # binary16 (u, v, w) offsets per offset brick, each brick's record padded to offset_stride
            assert lay.offset_brick == oc.off_brick
            nbo3 = (-(-w.k // oc.off_brick)) ** 3
            offs = device_bytes(lay.offsets_dev, nbo3 * lay.offset_stride * 2).view(np.uint16)
            offs = offs.reshape(nbo3, lay.offset_stride)
            assert np.array_equal(offs[:, :3 * w.D], oc.offsets.reshape(nbo3, 3 * w.D))
            assert not offs[:, 3 * w.D:].any()
        cam = w.cameras()[0]
        p = fnr.make_params(w.n_samples)
        got = gpu_render(fnr, ctx, cache, [cam], p, with_cells=True)[0]
        ref = oracle.render_image(oc, cam, oparams(p), want_cells=True)
        compare(got, ref)
        assert (ref[1][..., 0] < w.n_samples).sum() > 200  # many rays terminate early
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_ragged_and_multi_frame(fnr, ctx, tiny_workload, tiny_arrays):
    """Image sizes that are not tile multiples, several frames per launch, > 32 frames (two launches)."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    try:
        sizes = [(67, 45), (1, 1), (9, 5), (8, 4), (33, 70)]
        cams = []
        for i, (W, H) in enumerate(sizes * 8):  # 40 frames
            cams.append(scenegen.cameras(100 + i, 1, W, H)[0])
        p = fnr.make_params(w.n_samples, t_thr=1e-3)
        got = gpu_render(fnr, ctx, cache, cams, p, with_cells=True)
        for i in (0, 1, 2, 3, 4, 33, 39):
            compare(got[i], oracle.render_image(oc, cams[i], oparams(p), want_cells=True))
    finally:
        fnr.fnr_cache_free(ctx, cache)


@pytest.mark.parametrize("D", [1, 3, 6, 16])
def test_component_counts(fnr, ctx, tiny_workload, D):
    """Odd record sizes (3D values padded to 16 bytes) in all three precisions."""
    w = tiny_workload
    k, l = 24, 16
    sc = scenegen.make_scene(7, n_spheres=6, n_shells=2, D=D, sh_degree=2)
    sig, uvw = scenegen.fill_position_grid(sc, k)
    beta = scenegen.direction_grid(sc, l)
    cam = scenegen.cameras(3, 1, 40, 24)[0]
    for prec in (0, 1, 2):
        cache = build(fnr, ctx, k, D, l, sig, uvw, beta, prec, 0)
        try:
            oc = oracle.quantize_cache(k, D, l, sig, uvw, beta, prec, 0)
            p = fnr.make_params(32, t_thr=1e-3)
            compare(gpu_render(fnr, ctx, cache, [cam], p, with_cells=True)[0],
                    oracle.render_image(oc, cam, oparams(p), want_cells=True))
        finally:
            fnr.fnr_cache_free(ctx, cache)


def test_degenerate_cases(fnr, ctx, tiny_workload, tiny_arrays):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cam = w.cameras()[0]
    # empty cache: RGB = background exactly, alpha 0
    cache = build(fnr, ctx, w.k, w.D, w.l, np.zeros_like(sig), uvw, beta)
    try:
        p = fnr.make_params(w.n_samples, bg=(0.25, 0.5, 1.0))
        rgba, st, _ = gpu_render(fnr, ctx, cache, [cam], p)[0]
        assert np.all(rgba[..., :3] == np.array([0.25, 0.5, 1.0], np.float32)) and np.all(rgba[..., 3] == 0)
        assert np.all(st[..., 0] == w.n_samples) and np.all(st[..., 2] == 0)
    finally:
        fnr.fnr_cache_free(ctx, cache)
    # negative / NaN densities are stored as 0
    bad = sig.copy().reshape(-1)
    bad[::7] = -3.0
    bad[::11] = np.nan
    cache = build(fnr, ctx, w.k, w.D, w.l, bad, uvw, beta)
    try:
        oc = oracle.Cache(w.k, w.D, w.l, np.where(bad > 0, bad, 0).astype(np.float32), uvw, beta)
        p = fnr.make_params(w.n_samples)
        compare(gpu_render(fnr, ctx, cache, [cam], p, with_cells=True)[0],
                oracle.render_image(oc, cam, oparams(p), want_cells=True))
    finally:
        fnr.fnr_cache_free(ctx, cache)
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    try:
        cases = [
            (cam, fnr.make_params(1)),                                   # one sample per ray
            (cam, fnr.make_params(w.n_samples, t_thr=0.0)),              # no termination
            (cam, fnr.make_params(w.n_samples, t_thr=1.0)),              # stop at the first occupied sample
            (cam, fnr.make_params(w.n_samples, activation=fnr.FNR_ACT_IDENTITY)),
            (scenegen.look_at_camera((0.1, 0.2, 0.3), 30, 20), fnr.make_params(w.n_samples, 0.0, 3.0)),  # inside box
            (scenegen.look_at_camera((0.0, 0.0, 4.0), 16, 16), fnr.make_params(w.n_samples)),  # view axis on a pole
            (scenegen.look_at_camera((0.0, 0.0, -4.0), 16, 16), fnr.make_params(w.n_samples)),
            (scenegen.look_at_camera((3.0, 0.0, 0.0), 16, 16), fnr.make_params(200, 2.0, 6.0)),  # N not / 4
        ]
        for c, p in cases:
            compare(gpu_render(fnr, ctx, cache, [c], p, with_cells=True)[0],
                    oracle.render_image(oc, c, oparams(p), want_cells=True))
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_smallest_grids(fnr, ctx):
    """k = 1 and l = 2: one position cell, four direction cells."""
    sc = scenegen.make_scene(11, n_spheres=1, n_shells=0, D=2, sh_degree=1)
    sig = np.array([3.5], np.float32)
    uvw = np.random.default_rng(0).standard_normal(6).astype(np.float32)
    beta = scenegen.direction_grid(sc, 2)
    cam = scenegen.cameras(5, 1, 20, 20)[0]
    cache = build(fnr, ctx, 1, 2, 2, sig, uvw, beta)
    try:
        p = fnr.make_params(16)
        compare(gpu_render(fnr, ctx, cache, [cam], p, with_cells=True)[0],
                oracle.render_image(oracle.Cache(1, 2, 2, sig, uvw, beta), cam, oparams(p), want_cells=True))
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_homogeneous_closed_form_on_gpu(fnr, ctx):
    """The oracle's closed-form pin, rendered by the kernel: C = c(1 - e^{-s m D}) + e^{-s m D} bg."""
    k, N, s0 = 64, 64, 50.0
    c = np.array([0.3, 0.5, 0.7], np.float32)
    sig = np.full(k ** 3, s0, np.float32)
    uvw = np.tile(c, (k ** 3, 1))
    beta = np.ones((8, 8, 1), np.float32)
    cam = scenegen.look_at_camera((0.0, 0.0, 4.0), 64, 64)
    cam.update(fx=np.float32(80), fy=np.float32(80), cx=np.float32(32.5), cy=np.float32(32.5))
    cache = build(fnr, ctx, k, 1, 8, sig, uvw, beta)
    try:
        p = fnr.make_params(N, bg=(0.9, 0.2, 0.4), activation=fnr.FNR_ACT_IDENTITY)
        rgba, st, _ = gpu_render(fnr, ctx, cache, [cam], p)[0]
        Tm = math.exp(-s0 * 3 / 16)
        expect = c.astype(np.float64) * (1 - Tm) + Tm * np.array([0.9, 0.2, 0.4], np.float32)
        assert np.max(np.abs(rgba[32, 32, :3] - expect)) < 1e-6
        assert tuple(st[32, 32, :3]) == (11, 3, 3)
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_invalid_arguments(fnr, ctx, tiny_workload, tiny_arrays):
    import ctypes
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    L = fnr.lib()
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    try:
        cam = fnr.make_camera(w.cameras()[0])
        out = torch.empty(w.W * w.H * 4, device="cuda")
        for p in (fnr.make_params(0), fnr.make_params(5000), fnr.make_params(8, 6.0, 2.0),
                  fnr.make_params(8, activation=9), fnr.make_params(8, t_near=float("nan"))):
            assert L.fnr_render(ctx, cache, ctypes.byref(cam), 1, ctypes.byref(p), out.data_ptr(), None, None,
                                None) == fnr.FNR_ERR_INVALID_ARG
        p = fnr.make_params(8)
        bad = fnr.make_camera(w.cameras()[0])
        bad.width = 0
        assert L.fnr_render(ctx, cache, ctypes.byref(bad), 1, ctypes.byref(p), out.data_ptr(), None, None,
                            None) == fnr.FNR_ERR_INVALID_ARG
        assert L.fnr_render(ctx, 12345, ctypes.byref(cam), 1, ctypes.byref(p), out.data_ptr(), None, None,
                            None) == fnr.FNR_ERR_INVALID_ARG
        assert L.fnr_render(ctx, cache, ctypes.byref(cam), 0, ctypes.byref(p), out.data_ptr(), None, None,
                            None) == fnr.FNR_ERR_INVALID_ARG
    finally:
        fnr.fnr_cache_free(ctx, cache)
    # the HBM budget refuses a cache that does not fit, and charges/uncharges exactly
    small = fnr.fnr_context_create(0, 1 << 20)
    try:
        with pytest.raises(fnr.FnrError) as ei:
            build(fnr, small, w.k, w.D, w.l, sig, uvw, beta)
        assert ei.value.status == fnr.FNR_ERR_BUDGET
        assert fnr.fnr_context_used_bytes(small) == 0
    finally:
        fnr.fnr_context_destroy(small)
    before = fnr.fnr_context_used_bytes(ctx)
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    assert fnr.fnr_context_used_bytes(ctx) - before == fnr.fnr_cache_footprint(fnr.make_desc(w.k, w.D, w.l))
    fnr.fnr_cache_free(ctx, cache)
    assert fnr.fnr_context_used_bytes(ctx) == before


def test_stream_ordering(fnr, ctx, tiny_workload, tiny_arrays):
    """Renders on a side stream match the default-stream result bit for bit."""
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    try:
        cam = w.cameras()[0]
        p = fnr.make_params(w.n_samples)
        a = gpu_render(fnr, ctx, cache, [cam], p)[0]
        s = torch.cuda.Stream()
        b = gpu_render(fnr, ctx, cache, [cam], p, stream=s)[0]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    finally:
        fnr.fnr_cache_free(ctx, cache)


# ------------------------------------------------------------------ full-size plain workload, sampled pixels
@pytest.fixture(scope="module")
def scale_arrays():
    w = scenegen.scale()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    return w, sig, uvw, beta


def test_scale_workload_sampled_parity(fnr, ctx, scale_arrays):
    """800x800, N=128, k=512^3 FP32 (13.4 GB), 8 cameras, one launch per frame (the benchmark's
    configuration); 1500 random pixels per frame checked against the oracle one by one."""
    w, sig, uvw, beta = scale_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    try:
        p = fnr.make_params(w.n_samples)
        rng = np.random.default_rng(0)
        for i, cam in enumerate(w.cameras()):
            rgba, st, _ = gpu_render(fnr, ctx, cache, [cam], p)[0]
            px = rng.integers(0, w.W, 1500).astype(np.int32)
            py = rng.integers(0, w.H, 1500).astype(np.int32)
            r_rgba, r_st, _ = oracle.render_pixels(oc, cam, oparams(p), px, py)
            assert np.array_equal(st[py, px], r_st)
            assert np.max(np.abs(rgba[py, px].astype(np.float64) - r_rgba)) <= TOL
            # whole-frame properties
            assert np.all(rgba[..., 3] >= 0) and np.all(rgba[..., 3] <= 1)
            assert np.all((st[..., 0] >= 1) & (st[..., 0] <= w.n_samples))
            assert np.all(st[..., 2] <= st[..., 1]) and np.all(st[..., 1] <= st[..., 0])
        # per-sample cells on one frame, sampled
        cam = w.cameras()[0]
        _, _, cells = gpu_render(fnr, ctx, cache, [cam], p, with_cells=True)[0]
        px = rng.integers(0, w.W, 300).astype(np.int32)
        py = rng.integers(0, w.H, 300).astype(np.int32)
        _, _, r_cells = oracle.render_pixels(oc, cam, oparams(p), px, py, want_cells=True)
        assert np.array_equal(cells[py, px], r_cells)
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_scale_workload_skip_empty(fnr, ctx, scale_arrays):
    """Empty-space skipping at the benchmark's size (k=512^3, 8-cell bricks): the image and every counter
    but the lookups equal the plain render bit for bit; the lookups and colours of sampled pixels match the
    oracle's skip mode; the brick bits equal the oracle's."""
    w, sig, uvw, beta = scale_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    lay = fnr.fnr_cache_get_layout(cache)
    assert lay.occupancy_brick == 8
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta).set_occupancy(8)
    nb3 = 64 ** 3
    words = device_bytes(lay.occupancy_dev, nb3 // 8).view(np.uint32)
    assert np.array_equal(np.unpackbits(words.view(np.uint8), bitorder="little")[:nb3], oc.occ)
    try:
        p, ps = fnr.make_params(w.n_samples), fnr.make_params(w.n_samples, skip_empty=True)
        rng = np.random.default_rng(2)
        for cam in w.cameras()[:4]:
            rgba, st, _ = gpu_render(fnr, ctx, cache, [cam], p)[0]
            rgba_s, st_s, _ = gpu_render(fnr, ctx, cache, [cam], ps)[0]
            assert np.array_equal(rgba_s, rgba)
            assert np.array_equal(st_s[..., [0, 2, 3]], st[..., [0, 2, 3]])
            assert st_s[..., 1].sum() < 0.7 * st[..., 1].sum()
            px = rng.integers(0, w.W, 1500).astype(np.int32)
            py = rng.integers(0, w.H, 1500).astype(np.int32)
            r_rgba, r_st, _ = oracle.render_pixels(oc, cam, oparams(ps), px, py)
            assert np.array_equal(st_s[py, px], r_st)
            assert np.max(np.abs(rgba_s[py, px].astype(np.float64) - r_rgba)) <= TOL
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_back_to_back_launches_keep_stream_order(fnr, ctx, tiny_workload, tiny_arrays):
    """Consecutive renders into the same buffers (launches that may overlap through programmatic
    dependent launch) leave exactly the last render's output, and a torch kernel queued after a render
    sees its complete output."""
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = build(fnr, ctx, w.k, w.D, w.l, sig, uvw, beta)
    try:
        cams = scenegen.cameras(55, 3, 256, 192)
        p = fnr.make_params(w.n_samples)
        n = 256 * 192
        ref = []
        for cam in cams:
            r = torch.zeros(n * 4, device="cuda")
            st = torch.zeros(n * 4, device="cuda", dtype=torch.int32)
            fnr.fnr_render(ctx, cache, [cam], p, r, st)
            torch.cuda.synchronize()
            ref.append((r.clone(), st.clone()))
        rgba = torch.zeros(n * 4, device="cuda")
        stats = torch.zeros(n * 4, device="cuda", dtype=torch.int32)
        sums = []
        for i in range(60):
            fnr.fnr_render(ctx, cache, [cams[i % 3]], p, rgba, stats)
            sums.append(rgba.sum())  # a torch kernel between renders reads the whole output
        torch.cuda.synchronize()
        assert torch.equal(rgba, ref[59 % 3][0]) and torch.equal(stats, ref[59 % 3][1])
        for i, v in enumerate(sums):
            assert float(v) == float(ref[i % 3][0].sum())
        for i in range(61):  # no reader in between: only the order of writes matters
            fnr.fnr_render(ctx, cache, [cams[i % 3]], p, rgba, stats)
        torch.cuda.synchronize()
        assert torch.equal(rgba, ref[60 % 3][0]) and torch.equal(stats, ref[60 % 3][1])
    finally:
        fnr.fnr_cache_free(ctx, cache)
