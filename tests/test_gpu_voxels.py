"""The voxel walk (FNR_RENDER_VOXELS) through the C ABI against the FP64 oracle's walk.

Bar: the walked cells, n_steps, n_lookups, n_occupied and the direction cell
bit-exact (the walk is a fixed binary32 sequence on both sides); RGBA within
1e-5 (1e-4 with the interpolated direction lookup). Unsupported combinations
(brick caches, served requests, fnr_render_noalloc, the uncached render)
return FNR_ERR_UNSUPPORTED.
"""

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


def render(fnr, ctx, cache, cam, p, with_cells=True):
    import torch
    n = int(cam["W"]) * int(cam["H"])
    rgba = torch.full((n * 4,), float("nan"), device="cuda")
    stats = torch.full((n * 4,), -7, device="cuda", dtype=torch.int32)
    cells = torch.full((n * p.n_samples,), -9, device="cuda", dtype=torch.int32) if with_cells else None
    fnr.fnr_render(ctx, cache, [cam], p, rgba, stats, cells)
    torch.cuda.synchronize()
    H, W = int(cam["H"]), int(cam["W"])
    return (rgba.cpu().numpy().reshape(H, W, 4), stats.cpu().numpy().reshape(H, W, 4),
            None if cells is None else cells.cpu().numpy().reshape(H, W, -1))


def oparams(p):
    return oracle.params_struct(p.n_samples, p.t_near, p.t_far, p.t_thr, tuple(p.bg), p.activation,
                                skip_empty=bool(p.flags & 1), dir_bilinear=bool(p.flags & 2),
                                voxels=bool(p.flags & 4))


def check(got, ref, tol):
    assert np.array_equal(got[1], ref[1]), f"counters differ at {np.argwhere(got[1] != ref[1])[:5]}"
    if ref[2] is not None:
        assert np.array_equal(got[2], ref[2]), f"cells differ at {np.argwhere(got[2] != ref[2])[:5]}"
    err = np.max(np.abs(got[0].astype(np.float64) - ref[0]))
    assert err <= tol, f"max |rgba - oracle| = {err}"


@pytest.mark.parametrize("prec,dprec", [(0, 0), (1, 1), (2, 1)])
def test_tiny_voxel_parity(fnr, ctx, tiny_workload, tiny_arrays, prec, dprec):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, prec, dprec, occupancy_brick=4),
                                sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    try:
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, dprec).set_occupancy(4)
        N = 3 * w.k
        cases = [(w.cameras()[0], dict()),
                 (w.cameras()[0], dict(t_thr=0.0)),
                 (scenegen.look_at_camera((0.1, 0.2, 0.3), 30, 20), dict(t_near=0.0, t_far=3.0)),  # inside the box
                 (scenegen.cameras(41, 1, 37, 29)[0], dict(t_thr=1e-3, t_near=3.0, t_far=4.5))]      # clipped, ragged
        for cam, kw in cases:
            for skip in (False, True):
                for bil in (False, True):
                    p = fnr.make_params(N, voxels=True, skip_empty=skip, dir_bilinear=bil, **kw)
                    got = render(fnr, ctx, cache, cam, p)
                    ref = oracle.render_image(oc, cam, oparams(p), want_cells=True)
                    check(got, ref, 1e-4 if bil else TOL)
                    assert (got[1][..., 2] > 0).any() or kw.get("t_near") == 3.0
    finally:
        fnr.fnr_cache_free(ctx, cache)


@pytest.mark.parametrize("D", [1, 3, 16])
def test_voxel_component_counts(fnr, ctx, D):
    k, l = 20, 12
    sc = scenegen.make_scene(9, n_spheres=6, n_shells=2, D=D, sh_degree=2)
    sig, uvw = scenegen.fill_position_grid(sc, k)
    beta = scenegen.direction_grid(sc, l)
    cam = scenegen.cameras(8, 1, 33, 21)[0]
    for prec in (0, 1, 2):
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(k, D, l, prec, 0, occupancy_brick=4), sig.reshape(-1),
                                    uvw.reshape(-1), beta.reshape(-1))
        try:
            oc = oracle.quantize_cache(k, D, l, sig, uvw, beta, prec, 0).set_occupancy(4)
            for skip in (False, True):
                p = fnr.make_params(3 * k, t_thr=1e-3, voxels=True, skip_empty=skip)
                check(render(fnr, ctx, cache, cam, p), oracle.render_image(oc, cam, oparams(p), want_cells=True), TOL)
        finally:
            fnr.fnr_cache_free(ctx, cache)


def test_voxel_walk_cap_and_degenerate(fnr, ctx, tiny_workload, tiny_arrays):
    """n_samples caps the walk (the oracle caps it the same way); an empty cache leaves T = 1 and the
    background; a camera looking away from the box walks no cell."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    empty = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), np.zeros(w.k ** 3, np.float32),
                                uvw.reshape(-1), beta.reshape(-1))
    try:
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, 0, 0)
        cam = w.cameras()[0]
        for N in (1, 7, 40):
            p = fnr.make_params(N, voxels=True, t_thr=0.0)
            got = render(fnr, ctx, cache, cam, p)
            check(got, oracle.render_image(oc, cam, oparams(p), want_cells=True), TOL)
            assert got[1][..., 0].max() <= N
        p = fnr.make_params(3 * w.k, voxels=True, bg=(0.25, 0.5, 1.0))
        rgba, st, _ = render(fnr, ctx, empty, cam, p)
        assert np.all(st[..., 2] == 0)
        assert np.all(rgba[..., :3] == np.array([0.25, 0.5, 1.0], np.float32)) and np.all(rgba[..., 3] == 0)
        away = scenegen.look_at_camera((0.0, 0.0, 4.0), 16, 16)
        m = np.asarray(away["c2w"], np.float32).reshape(3, 4).copy()
        m[:, :3] *= -1.0  # looks away from the box
        away["c2w"] = m.reshape(12)
        rgba, st, cells = render(fnr, ctx, cache, away, p)
        assert np.all(st[..., 0] == 0) and np.all(st[..., 1] == 0) and np.all(cells == -1)
        assert np.all(rgba[..., 3] == 0)
    finally:
        fnr.fnr_cache_free(ctx, cache)
        fnr.fnr_cache_free(ctx, empty)


def test_voxel_unsupported_paths(fnr, ctx, tiny_workload, tiny_arrays):
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    dense = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    bricks = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, layout=fnr.FNR_LAYOUT_BRICKS), sig.reshape(-1),
                                 uvw.reshape(-1), beta.reshape(-1))
    try:
        cam = w.cameras()[0]
        out = torch.zeros(cam["W"] * cam["H"] * 4, device="cuda")
        p = fnr.make_params(3 * w.k, voxels=True)
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render(ctx, bricks, [cam], p, out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render_noalloc(dense, [cam], p, out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_submit(ctx, fnr.make_request(dense, cam, p, out))
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        p.flags = 8  # no such flag
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render(ctx, dense, [cam], p, out)
        assert ei.value.status == fnr.FNR_ERR_INVALID_ARG
    finally:
        fnr.fnr_cache_free(ctx, dense)
        fnr.fnr_cache_free(ctx, bricks)


def test_voxel_scale_workload_sampled(fnr, ctx):
    """800x800 over the k=512^3 FP32 scene (13.4 GB), N = 3k, the benchmark's voxel-walk launch: counters of
    1000 random pixels bit-exact and colours within 1e-5 of the oracle's walk, with and without skipping."""
    w = scenegen.scale()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta).set_occupancy(8)
    try:
        rng = np.random.default_rng(5)
        cam = w.cameras()[3]
        for skip in (False, True):
            p = fnr.make_params(3 * w.k, voxels=True, skip_empty=skip)
            rgba, st, _ = render(fnr, ctx, cache, cam, p, with_cells=False)
            px = rng.integers(0, w.W, 1000).astype(np.int32)
            py = rng.integers(0, w.H, 1000).astype(np.int32)
            r_rgba, r_st, _ = oracle.render_pixels(oc, cam, oparams(p), px, py)
            assert np.array_equal(st[py, px], r_st)
            assert np.max(np.abs(rgba[py, px].astype(np.float64) - r_rgba)) <= TOL
            assert np.all(st[..., 2] <= st[..., 1]) and np.all(st[..., 1] <= st[..., 0])
    finally:
        fnr.fnr_cache_free(ctx, cache)


@pytest.mark.parametrize("prec,brick", [(0, 4), (1, 2), (2, 8)])
def test_voxel_skip_without_cells(fnr, ctx, tiny_workload, tiny_arrays, prec, brick):
    """Skipping without per-cell output: the walk passes over whole empty cubes of jump bricks in one step
    (and over the remaining cells of empty bricks without a density load); the counters (n_steps counts
    every walked cell, jumped ones included) and colours must equal the oracle's cell-by-cell walk."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, prec, 1 if prec else 0, occupancy_brick=brick),
                                sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    try:
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, 1 if prec else 0).set_occupancy(brick)
        cams = [(w.cameras()[0], dict()), (w.cameras()[0], dict(t_thr=0.0)),
                (scenegen.look_at_camera((0.1, 0.2, 0.3), 30, 20), dict(t_near=0.0, t_far=3.0)),
                (scenegen.cameras(41, 1, 37, 29)[0], dict(t_thr=1e-3, t_near=3.0, t_far=4.5)),
                (scenegen.cameras(43, 1, 29, 31)[0], dict()),
                # central rays along the main diagonal (crossings on all three axes at the same times) and
                # along -z (two axes never crossed): the one-step passes over empty cubes must break ties
                # in axis order exactly as the cell-by-cell walk does
                (scenegen.look_at_camera((2.5, 2.5, 2.5), 31, 31), dict()),
                (scenegen.look_at_camera((0.0, 0.0, 3.5), 31, 31), dict(t_thr=0.0))]
        for cam, kw in cams:
            for N in (3 * w.k, 50):
                p = fnr.make_params(N, voxels=True, skip_empty=True, **kw)
                got = render(fnr, ctx, cache, cam, p, with_cells=False)
                ref = oracle.render_image(oc, cam, oparams(p))
                check(got, ref, TOL)
    finally:
        fnr.fnr_cache_free(ctx, cache)
