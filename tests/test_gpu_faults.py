"""Failure paths made to run without faulting the GPU (failure detection).

- A bounded device wait that runs out: the tensor-core cache build is armed
  (through the library's test hook) with a short wait limit and a producer that
  withholds one weight chunk, so the MMA issuer's wait for that chunk expires.
  The kernel sets its error word, drains what it has in flight, frees its
  tensor memory and returns; fnr_build_cache returns FNR_ERR_DEVICE, the
  context's budget is back where it was, and the next build succeeds and equals
  an unfaulted build bit for bit.
- A device allocation that fails: every allocation of a build (and of the
  uncached render and the request loop's start) is made to fail in turn; each
  call returns FNR_ERR_OOM with nothing left charged, and the same call
  succeeds once the hook is disarmed.
"""

import numpy as np
import pytest

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
    yield fnr
    fnr.fnr_testing_fail_allocations(0, 0)


def to_device(layers):
    import torch
    return [(torch.from_numpy(W.view(np.int16)).cuda(), torch.from_numpy(b).cuda()) for W, b in layers]


def cache_bytes(fnr, cache, k, D, l):
    """The cache's stored sigma, records and beta, as bytes (FP32 cache)."""
    import torch
    lay = fnr.fnr_cache_get_layout(cache)

    def grab(ptr, n):
        class _V:
            __cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False), "version": 3}
        return torch.as_tensor(_V(), device="cuda").cpu().numpy().copy()

    return (grab(lay.sigma_dev, k ** 3 * 4), grab(lay.uvw_dev, k ** 3 * lay.record_stride),
            grab(lay.beta_dev, l * l * D * 4))


@pytest.mark.parametrize("pair", [False, True])
@pytest.mark.parametrize("withhold", [0, 3, 11])
def test_build_wait_runs_out_and_recovers(fnr, withhold, pair):
    """Single-CTA and CTA-pair forms of the build kernel: in the pair form both CTAs withhold the chunk, the
    MMA issuer's wait runs out and sets both CTAs' abort flags."""
    import torch
    fnr.fnr_testing_mlp_cta_pair(pair)
    try:
        _wait_runs_out(fnr, withhold)
    finally:
        fnr.fnr_testing_mlp_cta_pair(False)


def _wait_runs_out(fnr, withhold):
    import torch
    k, l, D = 24, 12, 8
    pos = to_device(scenegen.mlp_weights(3, scenegen.FPOS_DIMS_D8, bias_scale=0.05))
    dirn = to_device(scenegen.mlp_weights(4, scenegen.FDIR_DIMS_D8, bias_scale=0.05))
    desc = fnr.make_desc(k, D, l)
    ctx = fnr.fnr_context_create(0, 1 << 30)
    try:
        ref = fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
        want = cache_bytes(fnr, ref, k, D, l)
        used = fnr.fnr_context_used_bytes(ctx)
        fnr.fnr_testing_mlp_fault(1 << 12, withhold)
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
        assert ei.value.status == fnr.FNR_ERR_DEVICE
        assert "ran out" in str(ei.value)
        assert fnr.fnr_context_used_bytes(ctx) == used  # the failed build's cache was released
        torch.cuda.synchronize()                        # the context is still usable
        again = fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
        got = cache_bytes(fnr, again, k, D, l)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        fnr.fnr_cache_free(ctx, again)
        fnr.fnr_cache_free(ctx, ref)
        assert fnr.fnr_context_used_bytes(ctx) == 0
    finally:
        fnr.fnr_context_destroy(ctx)


def test_wait_limit_alone_does_not_corrupt(fnr):
    """A short limit without a withheld chunk either completes (equal to the unfaulted build) or reports
    FNR_ERR_DEVICE; either way the next build is correct."""
    k, l, D = 16, 8, 8
    pos = to_device(scenegen.mlp_weights(5, scenegen.FPOS_DIMS_D8, bias_scale=0.05))
    dirn = to_device(scenegen.mlp_weights(6, scenegen.FDIR_DIMS_D8, bias_scale=0.05))
    desc = fnr.make_desc(k, D, l)
    ctx = fnr.fnr_context_create(0, 0)
    try:
        ref = fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
        want = cache_bytes(fnr, ref, k, D, l)
        fnr.fnr_testing_mlp_fault(1, -1)
        try:
            c = fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
            for a, b in zip(cache_bytes(fnr, c, k, D, l), want):
                assert np.array_equal(a, b)
            fnr.fnr_cache_free(ctx, c)
        except fnr.FnrError as e:
            assert e.status == fnr.FNR_ERR_DEVICE
        c = fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn)
        for a, b in zip(cache_bytes(fnr, c, k, D, l), want):
            assert np.array_equal(a, b)
    finally:
        fnr.fnr_context_destroy(ctx)


def _fail_each_allocation(fnr, ctx, call, max_allocs=16):
    """Make allocation i of `call` fail for i = 0, 1, ... until the call makes fewer allocations than i + 1;
    every failing attempt must return FNR_ERR_OOM and leave the budget as it was."""
    failures = 0
    for i in range(max_allocs):
        used = fnr.fnr_context_used_bytes(ctx)
        fnr.fnr_testing_fail_allocations(i, 1)
        try:
            out = call()
        except fnr.FnrError as e:
            assert e.status == fnr.FNR_ERR_OOM, (i, e)
            assert fnr.fnr_context_used_bytes(ctx) == used, i
            failures += 1
            continue
        finally:
            fnr.fnr_testing_fail_allocations(0, 0)
        return failures, out
    raise AssertionError("call kept allocating")


def test_allocation_failures_leave_nothing_charged(fnr):
    import torch
    w = scenegen.tiny()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    ctx = fnr.fnr_context_create(0, 1 << 30)
    try:
        for prec, layout in ((0, fnr.FNR_LAYOUT_DENSE), (2, fnr.FNR_LAYOUT_DENSE), (1, fnr.FNR_LAYOUT_BRICKS)):
            desc = fnr.make_desc(w.k, w.D, w.l, prec, min(prec, 1), layout=layout)
            n_fail, cache = _fail_each_allocation(
                fnr, ctx, lambda: fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1)))
            assert n_fail >= 1
            # the cache built after the failures renders like one built without them
            ref = fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
            p = fnr.make_params(w.n_samples)
            a = torch.zeros(w.W * w.H * 4, device="cuda")
            b = torch.zeros_like(a)
            cam = w.cameras()[0]
            fnr.fnr_render(ctx, cache, [cam], p, a)
            fnr.fnr_render(ctx, ref, [cam], p, b)
            torch.cuda.synchronize()
            assert torch.equal(a, b)
            fnr.fnr_cache_free(ctx, cache)
            fnr.fnr_cache_free(ctx, ref)
        assert fnr.fnr_context_used_bytes(ctx) == 0
        # the tensor-core build: cache, weights, biases, error word (F_pos, then F_dir)
        pos = to_device(scenegen.mlp_weights(3, scenegen.FPOS_DIMS_D8, bias_scale=0.05))
        dirn = to_device(scenegen.mlp_weights(4, scenegen.FDIR_DIMS_D8, bias_scale=0.05))
        desc = fnr.make_desc(16, 8, 8)
        n_fail, cache = _fail_each_allocation(fnr, ctx, lambda: fnr.fnr_build_cache_mlp(ctx, desc, pos, dirn))
        assert n_fail >= 7
        fnr.fnr_cache_free(ctx, cache)
        assert fnr.fnr_context_used_bytes(ctx) == 0
        # the uncached render's scratch
        rgba = torch.zeros(32 * 24 * 4, device="cuda")
        cam = scenegen.cameras(2, 1, 32, 24)[0]
        n_fail, _ = _fail_each_allocation(
            fnr, ctx, lambda: fnr.fnr_render_mlp(ctx, pos, dirn, 8, cam, fnr.make_params(32), rgba))
        assert n_fail >= 7
        # the request loop's scratch
        n_fail, _ = _fail_each_allocation(fnr, ctx, lambda: fnr.fnr_serve_start(ctx))
        assert n_fail >= 1
        fnr.fnr_serve_stop(ctx)
    finally:
        fnr.fnr_testing_fail_allocations(0, 0)
        fnr.fnr_context_destroy(ctx)
