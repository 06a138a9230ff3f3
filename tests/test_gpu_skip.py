"""Empty-space skipping (FNR_RENDER_SKIP_EMPTY) through the C ABI.

The cache's brick occupancy bits must equal the oracle's (bit-exact, from the
stored densities of each precision), and its brick distance field the
brute-force Chebyshev distance to the nearest occupied brick; a skip render
must give the plain render's image and counters bit for bit except the lookup
count, which must equal the oracle's skip-mode count (in-box samples in
occupied bricks, up to termination); colours within 1e-5 of the FP64 oracle.
Without per-sample cell output the march passes over runs of samples the
distance field proves empty: those renders must equal the ones with cell
output bit for bit. Served skip requests, mixed with plain ones, must equal
fnr_render's skip output bit for bit."""

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


def chebyshev_distance(occ, nb, cap=15):
    """Brute force: per brick, min over occupied bricks of the L-infinity index distance, capped at cap + 1."""
    idx = np.stack(np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij"), -1).reshape(-1, 3)
    idx = idx[:, ::-1]  # brick (bz nb + by) nb + bx -> (bx, by, bz)
    occupied = idx[occ.astype(bool)]
    out = np.full(nb ** 3, cap + 1, np.int64)
    for lo in range(0, occupied.shape[0], 256):
        o = occupied[lo:lo + 256]
        d = np.abs(idx[:, None, :] - o[None, :, :]).max(-1).min(1)
        out = np.minimum(out, d)
    return np.minimum(out, cap + 1)


def axis_ray_camera():
    """Identity rotation (looking down -z) from (0.013, -0.021, 3.7); pixel (16, 16) of 33 x 33 has
    d = (0, 0, -1) exactly, so its x and y sample coordinates are constant."""
    return dict(c2w=np.array([1, 0, 0, 0.013, 0, 1, 0, -0.021, 0, 0, 1, 3.7], np.float32), fx=np.float32(30.0),
                fy=np.float32(30.0), cx=np.float32(16.5), cy=np.float32(16.5), W=33, H=33)


@pytest.mark.parametrize("brick", [0, 1, 4, 8])
def test_brick_distance_field(fnr, ctx, tiny_workload, tiny_arrays, brick):
    """The distance field: jump bricks J = B 2^m (smallest with ceil(k / J) <= 32), occupied iff one of their
    occupancy bricks is, each holding the capped Chebyshev distance to the nearest occupied jump brick."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    sparse = sig.copy().reshape(w.k, w.k, w.k)
    sparse[:, :, : w.k // 2] = 0  # a large empty half-space: distances up to the cap
    for s_ in (sig, sparse):
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, occupancy_brick=brick), s_.reshape(-1),
                                    uvw.reshape(-1), beta.reshape(-1))
        try:
            lay = fnr.fnr_cache_get_layout(cache)
            B, bits = occupancy_from_device(lay, w.k)
            nb = (w.k + B - 1) // B
            J = lay.distance_brick
            m = J // B
            assert J % B == 0 and m & (m - 1) == 0 and -(-w.k // J) <= 32 and (J == B or -(-w.k // (J // 2)) > 32)
            nj = -(-w.k // J)
            occ = bits.reshape(nb, nb, nb)
            coarse = np.zeros((nj, nj, nj), bool)
            for z in range(nb):
                for y in range(nb):
                    coarse[z // m, y // m] |= np.add.reduceat(occ[z, y], np.arange(0, nb, m)) > 0
            dist = device_bytes(lay.brick_distance_dev, nj ** 3).astype(np.int64)
            assert np.array_equal(dist, chebyshev_distance(coarse.reshape(-1), nj))
            assert np.array_equal(dist == 0, coarse.reshape(-1))
        finally:
            fnr.fnr_cache_free(ctx, cache)


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
                 (scenegen.cameras(41, 1, 37, 29)[0], dict(t_thr=1e-3)),
                 (axis_ray_camera(), dict(t_near=0.5, t_far=7.0)),
                 (scenegen.cameras(43, 1, 24, 24, radius=9.0)[0], dict(t_near=5.0, t_far=13.0))]
        for cam, kw in cases:
            p = fnr.make_params(w.n_samples, **kw)
            ps = fnr.make_params(w.n_samples, skip_empty=True, **kw)
            plain = render(fnr, ctx, cache, cam, p)
            got = render(fnr, ctx, cache, cam, ps)
            assert np.array_equal(got[0], plain[0])  # image bit for bit
            assert np.array_equal(got[1][..., [0, 2, 3]], plain[1][..., [0, 2, 3]])
            assert np.array_equal(got[2], plain[2])
            fast = render(fnr, ctx, cache, cam, ps, with_cells=False)  # passes over empty runs
            assert np.array_equal(fast[0], got[0]) and np.array_equal(fast[1], got[1])
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
                for c_ in (dense, bricks):  # passing over empty runs
                    fast = render(fnr, ctx, c_, cam, p, with_cells=False)
                    assert np.array_equal(fast[0], got[0]) and np.array_equal(fast[1], got[1])
                ref = oracle.render_image(oc, cam, oparams(p), want_cells=True)
                assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
                assert np.max(np.abs(got[0].astype(np.float64) - ref[0])) <= (1e-4 if bil else 1e-5)
        finally:
            fnr.fnr_cache_free(ctx, dense)
            fnr.fnr_cache_free(ctx, bricks)
