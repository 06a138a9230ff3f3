"""FNR_LAYOUT_BRICKS (sparse brick pools behind a page table) through the C ABI.

A brick cache must hold exactly the occupied bricks of the dense cache (page table = ranks of the
occupied bricks in brick-index order, pool bytes = the dense cells of each brick, zero past the grid
edge) and render bit-identically to the dense cache with FNR_RENDER_SKIP_EMPTY; counters against the
oracle's skip mode bit-exact, colour within 1e-5 (FP32)."""

import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu


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


def device_bytes(ptr, nbytes):
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_View(), device="cuda").cpu().numpy()


def render(fnr, ctx, cache, cam, p, with_cells=False):
    import torch
    n = int(cam["W"]) * int(cam["H"])
    rgba = torch.full((n * 4,), float("nan"), device="cuda")
    stats = torch.full((n * 4,), -7, device="cuda", dtype=torch.int32)
    cells = torch.full((n * p.n_samples,), -9, device="cuda", dtype=torch.int32) if with_cells else None
    fnr.fnr_render(ctx, cache, [cam], p, rgba, stats, cells)
    torch.cuda.synchronize()
    return (rgba.cpu().numpy(), stats.cpu().numpy(), None if cells is None else cells.cpu().numpy())


@pytest.mark.parametrize("prec,dprec,brick", [(0, 0, 4), (0, 0, 8), (1, 1, 2), (2, 1, 8)])
def test_bricks_match_dense(fnr, ctx, prec, dprec, brick):
    w = scenegen.tiny()
    k = 60  # not a multiple of the brick side: edge bricks are partly outside the grid
    sig, uvw = scenegen.fill_position_grid(w.scene, k)
    beta = scenegen.direction_grid(w.scene, w.l)
    arrs = (sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    dense = fnr.fnr_build_cache(ctx, fnr.make_desc(k, w.D, w.l, prec, dprec, occupancy_brick=brick), *arrs)
    bricks = fnr.fnr_build_cache(ctx, fnr.make_desc(k, w.D, w.l, prec, dprec, occupancy_brick=brick,
                                                    layout=fnr.FNR_LAYOUT_BRICKS), *arrs)
    try:
        ld, lb = fnr.fnr_cache_get_layout(dense), fnr.fnr_cache_get_layout(bricks)
        assert lb.layout == fnr.FNR_LAYOUT_BRICKS and ld.layout == fnr.FNR_LAYOUT_DENSE and not ld.page_table_dev
        nb = (k + brick - 1) // brick
        nw = (nb ** 3 + 31) // 32
        bits = np.unpackbits(device_bytes(ld.occupancy_dev, nw * 4), bitorder="little")[:nb ** 3]
        assert np.array_equal(np.unpackbits(device_bytes(lb.occupancy_dev, nw * 4), bitorder="little")[:nb ** 3],
                              bits)
        page = device_bytes(lb.page_table_dev, nb ** 3 * 4).view(np.int32)
        occ = np.flatnonzero(bits)
        assert lb.n_bricks == occ.size > 0
        expect = np.full(nb ** 3, -1, np.int32)
        expect[occ] = np.arange(occ.size, dtype=np.int32)
        assert np.array_equal(page, expect)
        assert lb.footprint < ld.footprint
        # pool bytes: every brick's cells, in brick-local order, zero past the grid edge
        es = {0: 4, 1: 2, 2: 1}[prec]
        dsig = device_bytes(ld.sigma_dev, k ** 3 * es).reshape(k, k, k, es)
        drec = device_bytes(ld.uvw_dev, k ** 3 * ld.record_stride).reshape(k, k, k, ld.record_stride)
        B3 = brick ** 3
        psig = device_bytes(lb.sigma_dev, occ.size * B3 * es).reshape(occ.size, brick, brick, brick, es)
        prec_ = device_bytes(lb.uvw_dev, occ.size * B3 * lb.record_stride).reshape(occ.size, brick, brick, brick, -1)
        for slot in np.random.default_rng(1).choice(occ.size, min(40, occ.size), replace=False):
            b = occ[slot]
            bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
            z0, y0, x0 = bz * brick, by * brick, bx * brick
            zs, ys, xs = min(brick, k - z0), min(brick, k - y0), min(brick, k - x0)
            assert np.array_equal(psig[slot, :zs, :ys, :xs], dsig[z0:z0 + zs, y0:y0 + ys, x0:x0 + xs])
            assert np.array_equal(prec_[slot, :zs, :ys, :xs], drec[z0:z0 + zs, y0:y0 + ys, x0:x0 + xs])
            assert not psig[slot, zs:].any() and not psig[slot, :, ys:].any() and not psig[slot, :, :, xs:].any()
        oc = oracle.quantize_cache(k, w.D, w.l, sig, uvw, beta, prec, dprec).set_occupancy(brick)
        cams = [w.cameras()[0], scenegen.cameras(12, 1, 37, 29)[0], scenegen.look_at_camera((0.1, 0.2, 0.3), 20, 16)]
        for cam in cams:
            for kw in (dict(), dict(dir_bilinear=True), dict(t_thr=0.0)):
                if cam["W"] == 20:
                    kw = dict(kw, t_near=0.0, t_far=3.0)
                ps = fnr.make_params(w.n_samples, skip_empty=True, **kw)
                p_plain = fnr.make_params(w.n_samples, **kw)
                ref = render(fnr, ctx, dense, cam, ps, with_cells=True)
                got = render(fnr, ctx, bricks, cam, p_plain, with_cells=True)  # bricks always skip
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
                assert np.array_equal(got[2], ref[2])
            o_rgba, o_st, _ = oracle.render_image(oc, cam, oracle.params_struct(w.n_samples, skip_empty=True))
            got = render(fnr, ctx, bricks, cam, fnr.make_params(w.n_samples))
            H, W = int(cam["H"]), int(cam["W"])
            if cam["W"] != 20:
                assert np.array_equal(got[1].reshape(H, W, 4), o_st)
                if prec == 0:
                    assert np.max(np.abs(got[0].reshape(H, W, 4).astype(np.float64) - o_rgba)) <= 1e-5
    finally:
        fnr.fnr_cache_free(ctx, dense)
        fnr.fnr_cache_free(ctx, bricks)


def test_bricks_scale_footprint_and_paths(fnr, ctx, tmp_path):
    """512^3 FP32: the brick cache is a fraction of the dense one, renders like the dense skip render,
    survives save/load and is served; the allocation-free path refuses it."""
    import torch
    w = scenegen.scale()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    arrs = (sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    dense = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), *arrs)
    bricks = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, layout=fnr.FNR_LAYOUT_BRICKS), *arrs)
    try:
        ld, lb = fnr.fnr_cache_get_layout(dense), fnr.fnr_cache_get_layout(bricks)
        print(f"dense {ld.footprint / 1e9:.2f} GB, bricks {lb.footprint / 1e9:.2f} GB ({lb.n_bricks} bricks)")
        assert lb.footprint < 0.5 * ld.footprint
        ps = fnr.make_params(w.n_samples, skip_empty=True)
        for cam in w.cameras()[:2]:
            ref = render(fnr, ctx, dense, cam, ps)
            got = render(fnr, ctx, bricks, cam, ps)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        path = tmp_path / "bricks.fnrcache"
        fnr.fnr_cache_save(bricks, path)
        again = fnr.fnr_cache_load(ctx, path)
        la = fnr.fnr_cache_get_layout(again)
        assert (la.n_bricks, la.footprint, la.layout) == (lb.n_bricks, lb.footprint, lb.layout)
        cam = w.cameras()[2]
        assert np.array_equal(render(fnr, ctx, again, cam, ps)[0], render(fnr, ctx, bricks, cam, ps)[0])
        fnr.fnr_cache_free(ctx, again)
        out = torch.zeros(w.W * w.H * 4, device="cuda")
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render_noalloc(bricks, [cam], fnr.make_params(w.n_samples), out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        # served: brick-cache requests (mixed with dense ones) equal fnr_render's output bit for bit
        fnr.fnr_serve_start(ctx, n_slots=2, max_batch_requests=8, use_graphs=1)
        reqs = []
        for i, c in enumerate(scenegen.cameras(31, 6, 320, 200, hemisphere=True)):
            cache_i = bricks if i % 2 == 0 else dense
            o = torch.zeros(320 * 200 * 4, device="cuda")
            st = torch.zeros(320 * 200 * 4, device="cuda", dtype=torch.int32)
            reqs.append((fnr.fnr_submit(ctx, fnr.make_request(cache_i, c, ps, o, st)), cache_i, c, o, st))
        for t, cache_i, c, o, st in reqs:
            assert fnr.fnr_wait(ctx, t, 20000).status == fnr.FNR_OK
            ref = render(fnr, ctx, cache_i, c, ps)
            assert np.array_equal(o.cpu().numpy(), ref[0]) and np.array_equal(st.cpu().numpy(), ref[1])
        fnr.fnr_serve_stop(ctx)
    finally:
        fnr.fnr_cache_free(ctx, dense)
        fnr.fnr_cache_free(ctx, bricks)
