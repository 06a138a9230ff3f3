"""fnr_render_noalloc: rendering for callers that cannot allocate device memory.

Such callers (a process whose HBM another allocator already owns, a render
loop that must not stall on cudaMalloc / cudaFree, a host that plans all device
memory up front) get a persistent-kernel render whose scratch lives in a static
device array. Through the C ABI, two calls in a row must reproduce the existing
fnr_render output (same tolerance as the other parity tests: RGBA within 1e-5,
counters exact), and the second call must not change the device's free memory.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

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


def render_both(fnr, ctx, cache, cams, params):
    import torch
    npix = sum(c["W"] * c["H"] for c in cams)
    ref = torch.zeros(npix * 4, device="cuda")
    ref_st = torch.zeros(npix * 4, device="cuda", dtype=torch.int32)
    fnr.fnr_render(ctx, cache, cams, params, ref, ref_st)
    outs = []
    for _ in range(2):  # two calls in a row share (and re-clear) the static scratch
        rgba = torch.full((npix * 4,), float("nan"), device="cuda")
        st = torch.full((npix * 4,), -1, device="cuda", dtype=torch.int32)
        done = torch.zeros(len(cams), device="cuda", dtype=torch.int32)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        fnr.fnr_render_noalloc(cache, cams, params, rgba, st, done)
        torch.cuda.synchronize()
        outs.append((rgba.cpu().numpy(), st.cpu().numpy(), done.cpu().numpy(), free_before,
                     torch.cuda.mem_get_info()[0]))
    return ref.cpu().numpy(), ref_st.cpu().numpy(), outs


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_fnr_render(fnr, prec):
    w = scenegen.tiny()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, prec, min(prec, 1)), sig.reshape(-1),
                                    uvw.reshape(-1), beta.reshape(-1))
        cams = [w.cameras()[0]] + scenegen.cameras(21, 2, 45, 27)  # ragged sizes, three views in one launch
        params = fnr.make_params(w.n_samples)
        ref, ref_st, outs = render_both(fnr, ctx, cache, cams, params)
        for i, (rgba, st, done, free_before, free_after) in enumerate(outs):
            assert np.array_equal(st, ref_st)
            assert np.max(np.abs(rgba - ref)) <= TOL
            assert np.all(done == 1)
            if i == 1:
                assert free_after == free_before  # the second call allocated nothing
    finally:
        fnr.fnr_context_destroy(ctx)


def test_noalloc_rejects_more_views_than_its_scratch(fnr):
    import torch
    w = scenegen.tiny()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                    beta.reshape(-1))
        cams = scenegen.cameras(3, 33, 8, 8)
        arr = (fnr.fnr_camera * 33)(*[fnr.make_camera(c) for c in cams])
        out = torch.zeros(33 * 8 * 8 * 4, device="cuda")
        p = fnr.make_params(16)
        st = fnr.lib().fnr_render_noalloc(cache, arr, 33, ctypes.byref(p), out.data_ptr(), None, None, None)
        assert st == fnr.FNR_ERR_INVALID_ARG
        assert b"at most 32 views" in fnr.lib().fnr_last_error()
    finally:
        fnr.fnr_context_destroy(ctx)
