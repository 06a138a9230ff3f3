"""The uncached render (fnr_render_mlp) against the oracle.

Homogeneous model (zero weights, biases only): the network outputs are exact in binary32, so the
renderer must match the closed form with bit-exact counters and colour within 1e-5 (the cached
path's bar). Random He-uniform networks: the renderer evaluates bf16 layers with fp32 accumulation,
the oracle FP64 with the same bf16 rounding of inputs and activations (the cache-build tier-(i)
reading); a rounding flip can move a density across the termination threshold by one sample, so at
least 99% of the rays must have identical counters, colours of those rays within 2e-2 max / 2e-3 mean."""

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


def to_device(layers):
    import torch
    return [(torch.from_numpy(W.view(np.int16)).cuda(), torch.from_numpy(b).cuda()) for W, b in layers]


def as_fp64(layers):
    return [(scenegen.bf16_value(W).astype(np.float64), b.astype(np.float64)) for W, b in layers]


def run(fnr, pos, dirn, D, cam, p):
    import torch
    ctx = fnr.fnr_context_create(0, 0)
    try:
        n = cam["W"] * cam["H"]
        rgba = torch.full((n * 4,), float("nan"), device="cuda")
        stats = torch.full((n * 4,), -7, device="cuda", dtype=torch.int32)
        fnr.fnr_render_mlp(ctx, to_device(pos), to_device(dirn), D, cam, p, rgba, stats)
        torch.cuda.synchronize()
        assert fnr.fnr_context_used_bytes(ctx) == 0  # temporaries returned
        return rgba.cpu().numpy().reshape(-1, 4), stats.cpu().numpy().reshape(-1, 4)
    finally:
        fnr.fnr_context_destroy(ctx)


def const_layers(dims, head, hidden=0.25):
    out = []
    for i, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
        W = scenegen.bf16_bits(np.zeros((b, a), np.float32))
        bias = np.full(b, hidden, np.float32) if i + 1 < len(dims) - 1 else np.asarray(head, np.float32)
        out.append((W, bias))
    return out


def test_homogeneous_model_matches_closed_form_oracle(fnr):
    D = 8
    rng = np.random.default_rng(3)
    head = np.concatenate([[3.0], rng.uniform(-1, 1, 3 * D)]).astype(np.float32)
    pos = const_layers([60, 64, 64, 1 + 3 * D], head)
    dirn = const_layers([24, 32, D], rng.uniform(-1, 1, D).astype(np.float32))
    cam = scenegen.cameras(9, 1, 48, 40, fov_deg=100.0)[0]
    p = fnr.make_params(64, t_thr=1e-3)
    rgba, st = run(fnr, pos, dirn, D, cam, p)
    py, px = np.meshgrid(np.arange(40, dtype=np.int32), np.arange(48, dtype=np.int32), indexing="ij")
    op = oracle.params_struct(64, 2.0, 6.0, 1e-3)
    ref, ref_st = oracle.render_mlp_pixels(as_fp64(pos), as_fp64(dirn), D, cam, op, px.reshape(-1), py.reshape(-1))
    assert np.array_equal(st, ref_st)
    assert np.max(np.abs(rgba.astype(np.float64) - ref)) <= 1e-5
    assert (st[:, 0] < 64).any() and (st[:, 1] == 0).any()


def test_random_networks_sampled(fnr):
    D = 8
    pos = scenegen.mlp_weights(11, scenegen.FPOS_DIMS_D8, bias_scale=0.1)
    dirn = scenegen.mlp_weights(12, scenegen.FDIR_DIMS_D8, bias_scale=0.1)
    # a density bias keeps part of the rays inside the box terminating
    pos[-1] = (pos[-1][0], pos[-1][1] + np.concatenate([[2.0], np.zeros(3 * D)]).astype(np.float32))
    cam = scenegen.cameras(4, 1, 64, 48)[0]
    p = fnr.make_params(96, t_thr=1e-3)
    rgba, st = run(fnr, pos, dirn, D, cam, p)
    rng = np.random.default_rng(2)
    sel = rng.choice(64 * 48, 600, replace=False)
    px, py = (sel % 64).astype(np.int32), (sel // 64).astype(np.int32)
    ref, ref_st = oracle.render_mlp_pixels(as_fp64(pos), as_fp64(dirn), D, cam, oracle.params_struct(96, 2.0, 6.0, 1e-3),
                                           px, py)
    same = (st[sel] == ref_st).all(axis=1)
    assert same.mean() >= 0.99, same.mean()
    err = np.abs(rgba[sel][same].astype(np.float64) - ref[same])
    print(f"max {err.max():.2e} mean {err.mean():.2e} terminated {np.mean(ref_st[:, 0] < 96):.2f}")
    assert err.max() <= 2e-2 and err.mean() <= 2e-3
    assert (ref_st[:, 0] < 96).mean() > 0.05 and (ref_st[:, 2] > 0).mean() > 0.3


def test_uncached_rejects_bad_arguments(fnr):
    import torch
    D = 8
    pos = scenegen.mlp_weights(11, scenegen.FPOS_DIMS_D8)
    dirn = scenegen.mlp_weights(12, scenegen.FDIR_DIMS_D8)
    cam = scenegen.cameras(4, 1, 16, 16)[0]
    ctx = fnr.fnr_context_create(0, 0)
    try:
        out = torch.zeros(16 * 16 * 4, device="cuda")
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render_mlp(ctx, to_device(pos), to_device(dirn), 3, cam, fnr.make_params(32), out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_render_mlp(ctx, to_device(pos), to_device(dirn), D, cam, fnr.make_params(32, skip_empty=True), out)
        assert ei.value.status == fnr.FNR_ERR_UNSUPPORTED
        small = fnr.fnr_context_create(0, 1 << 16)
        try:
            with pytest.raises(fnr.FnrError) as ei:
                fnr.fnr_render_mlp(small, to_device(pos), to_device(dirn), D, cam, fnr.make_params(32), out)
            assert ei.value.status == fnr.FNR_ERR_BUDGET
        finally:
            fnr.fnr_context_destroy(small)
    finally:
        fnr.fnr_context_destroy(ctx)
