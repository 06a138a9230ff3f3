"""Empty-space skipping (FNR_RENDER_SKIP_EMPTY) through the C ABI.

The cache's brick occupancy bits must equal the oracle's (bit-exact, from the
stored densities of each precision); a skip render must give the plain
render's image and counters bit for bit except the lookup count, which must
equal the oracle's skip-mode count (in-box samples in occupied bricks, up to
termination); colours within 1e-5 of the FP64 oracle. Served skip requests,
mixed with plain ones, must equal fnr_render's skip output bit for bit."""

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
                                skip_empty=bool(p.flags & 1), dir_bilinear=bool(p.flags & 2))


def occupancy_from_device(lay, k):
    B = lay.occupancy_brick
    nb = (k + B - 1) // B
    nw = (nb ** 3 + 31) // 32
    bits = np.unpackbits(device_bytes(lay.occupancy_dev, nw * 4), bitorder="little")
    return B, bits[:nb ** 3]


@pytest.mark.parametrize("prec,dprec", [(0, 0), (1, 1), (2, 1)])
@pytest.mark.parametrize("brick", [0, 1, 4, 16])
def test_tiny_skip_parity(fnr, ctx, tiny_workload, tiny_arrays, prec, dprec, brick):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    desc = fnr.make_desc(w.k, w.D, w.l, prec, dprec, occupancy_brick=brick)
    cache = fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    try:
        lay = fnr.fnr_cache_get_layout(cache)
        B, bits = occupancy_from_device(lay, w.k)
        assert B == (brick or 2)  # automatic: smallest power of two >= 2 with ceil(64 / B) <= 64
        oc = oracle.quantize_cache(w.k, w.D, w.l, sig, uvw, beta, prec, dprec).set_occupancy(B)
        assert np.array_equal(bits, oc.occ)
        cases = [(w.cameras()[0], dict()), (w.cameras()[0], dict(t_thr=0.0)),
                 (scenegen.look_at_camera((0.1, 0.2, 0.3), 30, 20), dict(t_near=0.0, t_far=3.0)),
                 (scenegen.cameras(41, 1, 37, 29)[0], dict(t_thr=1e-3))]
        for cam, kw in cases:
            p = fnr.make_params(w.n_samples, **kw)
            ps = fnr.make_params(w.n_samples, skip_empty=True, **kw)
            plain = render(fnr, ctx, cache, cam, p)
            got = render(fnr, ctx, cache, cam, ps)
            assert np.array_equal(got[0], plain[0])  # image bit for bit
            assert np.array_equal(got[1][..., [0, 2, 3]], plain[1][..., [0, 2, 3]])
            assert np.array_equal(got[2], plain[2])
            ref = oracle.render_image(oc, cam, oparams(ps), want_cells=True)
            assert np.array_equal(got[1], ref[1]), f"counters differ at {np.argwhere(got[1] != ref[1])[:5]}"
            assert np.max(np.abs(got[0].astype(np.float64) - ref[0])) <= TOL
            assert (got[1][..., 1] <= plain[1][..., 1]).all()
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_empty_cache_skips_every_lookup(fnr, ctx, tiny_workload, tiny_arrays):
    w = tiny_workload
    _, uvw, beta = tiny_arrays
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), np.zeros(w.k ** 3, np.float32),
                                uvw.reshape(-1), beta.reshape(-1))
    try:
        _, bits = occupancy_from_device(fnr.fnr_cache_get_layout(cache), w.k)
        assert not bits.any()
        rgba, st, _ = render(fnr, ctx, cache, w.cameras()[0], fnr.make_params(w.n_samples, skip_empty=True,
                                                                               bg=(0.25, 0.5, 1.0)))
        assert np.all(st[..., 1] == 0) and np.all(st[..., 2] == 0) and np.all(st[..., 0] == w.n_samples)
        assert np.all(rgba[..., :3] == np.array([0.25, 0.5, 1.0], np.float32)) and np.all(rgba[..., 3] == 0)
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_invalid_flags_and_bricks(fnr, ctx, tiny_workload, tiny_arrays):
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    for bad in (3, -2, 512):
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, occupancy_brick=bad), sig.reshape(-1),
                                uvw.reshape(-1), beta.reshape(-1))
        assert ei.value.status == fnr.FNR_ERR_INVALID_ARG
    cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                beta.reshape(-1))
    try:
        cam = w.cameras()[0]
        out = torch.zeros(cam["W"] * cam["H"] * 4, device="cuda")
        p = fnr.make_params(w.n_samples)
        p.flags = 8  # no such flag
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render(ctx, cache, [cam], p, out)
        assert ei.value.status == fnr.FNR_ERR_INVALID_ARG
        ps = fnr.make_params(w.n_samples, skip_empty=True)
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render_noalloc(cache, [cam], ps, out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
    finally:
        fnr.fnr_cache_free(ctx, cache)


def test_served_skip_requests(fnr, tiny_workload, tiny_arrays):
    """Skip and plain requests submitted together: each served result equals fnr_render's with the same
    flags, bit for bit (skip and plain requests go to different launches)."""
    import torch
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, 1, 1), sig.reshape(-1), uvw.reshape(-1),
                                    beta.reshape(-1))
        fnr.fnr_serve_start(ctx, n_slots=2, max_batch_requests=16, use_graphs=1)
        cams = scenegen.cameras(77, 12, 53, 41)
        reqs = []
        for i, cam in enumerate(cams):
            p = fnr.make_params(w.n_samples, skip_empty=(i % 2 == 0), dir_bilinear=(i % 3 == 0))
            n = cam["W"] * cam["H"]
            rgba = torch.zeros(n * 4, device="cuda")
            stats = torch.zeros(n * 4, device="cuda", dtype=torch.int32)
            reqs.append((fnr.fnr_submit(ctx, fnr.make_request(cache, cam, p, rgba, stats)), cam, p, rgba, stats))
        for t, cam, p, rgba, stats in reqs:
            assert fnr.fnr_wait(ctx, t, 20000).status == fnr.FNR_OK
            ref = render(fnr, ctx, cache, cam, p, with_cells=False)
            assert np.array_equal(rgba.cpu().numpy().reshape(ref[0].shape), ref[0])
            assert np.array_equal(stats.cpu().numpy().reshape(ref[1].shape), ref[1])
        fnr.fnr_serve_stop(ctx)
        fnr.fnr_cache_free(ctx, cache)
    finally:
        fnr.fnr_context_destroy(ctx)


@pytest.mark.parametrize("D", [1, 3, 16])
def test_component_counts_skip_bricks_bilinear(fnr, ctx, D):
    """Odd record sizes with skipping, brick caches and the interpolated direction lookup."""
    k, l = 24, 16
    sc = scenegen.make_scene(7, n_spheres=6, n_shells=2, D=D, sh_degree=2)
    sig, uvw = scenegen.fill_position_grid(sc, k)
    beta = scenegen.direction_grid(sc, l)
    cam = scenegen.cameras(3, 1, 40, 24)[0]
    arrs = (sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    for prec in (0, 1, 2):
        dense = fnr.fnr_build_cache(ctx, fnr.make_desc(k, D, l, prec, 0, occupancy_brick=4), *arrs)
        bricks = fnr.fnr_build_cache(ctx, fnr.make_desc(k, D, l, prec, 0, occupancy_brick=4,
                                                        layout=fnr.FNR_LAYOUT_BRICKS), *arrs)
        try:
            oc = oracle.quantize_cache(k, D, l, sig, uvw, beta, prec, 0).set_occupancy(4)
            for bil in (False, True):
                p = fnr.make_params(32, t_thr=1e-3, skip_empty=True, dir_bilinear=bil)
                got = render(fnr, ctx, dense, cam, p)
                got_b = render(fnr, ctx, bricks, cam, p)
                assert np.array_equal(got_b[0], got[0]) and np.array_equal(got_b[1], got[1])
                ref = oracle.render_image(oc, cam, oparams(p), want_cells=True)
                assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
                assert np.max(np.abs(got[0].astype(np.float64) - ref[0])) <= (1e-4 if bil else 1e-5)
        finally:
            fnr.fnr_cache_free(ctx, dense)
            fnr.fnr_cache_free(ctx, bricks)
