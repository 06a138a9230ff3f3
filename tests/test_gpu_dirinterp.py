"""Interpolated direction lookup (FNR_RENDER_DIR_BILINEAR) through the C ABI against the oracle.

The kernel computes the angles with binary32 atan2f (a few ulp), so the interpolation weights differ
from the oracle's FP64 ones by ~1e-6 relative; at l = 64 (512) a direction-weight difference of that
order moves beta by ~4e-6 (3e-5) and the colour, through sum_i beta_i u_i (|u| <~ 4, D = 8) and the
sigmoid (slope <= 1/4), by up to ~1e-5 (5e-5): the bar is 1e-4 absolute. Integer outputs are
unchanged by the mode and stay bit-exact."""

import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

TOL = 1e-4


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


def render(fnr, ctx, cache, cam, p):
    import torch
    n = int(cam["W"]) * int(cam["H"])
    rgba = torch.full((n * 4,), float("nan"), device="cuda")
    stats = torch.full((n * 4,), -7, device="cuda", dtype=torch.int32)
    fnr.fnr_render(ctx, cache, [cam], p, rgba, stats)
    torch.cuda.synchronize()
    H, W = int(cam["H"]), int(cam["W"])
    return rgba.cpu().numpy().reshape(H, W, 4), stats.cpu().numpy().reshape(H, W, 4)


def oparams(p, **kw):
    return oracle.params_struct(p.n_samples, p.t_near, p.t_far, p.t_thr, tuple(p.bg), p.activation,
                                skip_empty=bool(p.flags & 1), dir_bilinear=bool(p.flags & 2))


@pytest.mark.parametrize("prec,dprec", [(0, 0), (1, 1), (2, 1)])
def test_tiny_bilinear_parity(fnr, ctx, tiny_workload, tiny_arrays, prec, dprec):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, prec, dprec), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    try:
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, dprec)
        cams = [w.cameras()[0], scenegen.look_at_camera((0.0, 0.0, 4.0), 40, 40),  # across the +z pole
                scenegen.look_at_camera((-4.0, 0.01, 0.5), 48, 32)]                 # phi near the 2 pi seam
        for cam in cams:
            p = fnr.make_params(w.n_samples, dir_bilinear=True)
            got = render(fnr, ctx, cache, cam, p)
            ref_rgba, ref_st, _ = oracle.render_image(oc, cam, oparams(p))
            assert np.array_equal(got[1], ref_st)
            err = np.max(np.abs(got[0].astype(np.float64) - ref_rgba))
            assert err <= TOL, err
            # the mode changes colours, not counters
            plain = render(fnr, ctx, cache, cam, fnr.make_params(w.n_samples))
            assert np.array_equal(plain[1], got[1])
            # with skipping as well: the same image
            both = render(fnr, ctx, cache, cam, fnr.make_params(w.n_samples, dir_bilinear=True, skip_empty=True))
            assert np.array_equal(both[0], got[0])
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_scale_bilinear_sampled(fnr, ctx):
    w = scenegen.scale()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    try:
        oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
        p = fnr.make_params(w.n_samples, dir_bilinear=True)
        rng = np.random.default_rng(5)
        for cam in w.cameras()[:3]:
            rgba, st = render(fnr, ctx, cache, cam, p)
            px = rng.integers(0, w.W, 1500).astype(np.int32)
            py = rng.integers(0, w.H, 1500).astype(np.int32)
            r_rgba, r_st, _ = oracle.render_pixels(oc, cam, oparams(p), px, py)
            assert np.array_equal(st[py, px], r_st)
            assert np.max(np.abs(rgba[py, px].astype(np.float64) - r_rgba)) <= TOL
    finally:
        fnr.fnr_cache_free(ctx, cache)
