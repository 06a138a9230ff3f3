"""The precision workload at its full size (k=1024^3, D=8, 768^2 direction grid, 800x800, N=192):
FP16 and E4M3 position caches rendered through the C ABI in the launch configuration the benchmark
times (one view per launch), checked on sampled pixels against the FP64 oracle reading the
unquantised binary32 field.

Bars: with the FP16 cache every integer output (steps, lookups, occupied samples, direction cell) is
bit-exact, because this scene family's densities (0 and 50) are exact in FP16; colour error is the
cache quantisation error: FP16 max abs <= 5e-3 and PSNR >= 60 dB (11-bit significands on |u| <~ 4,
|beta| <~ 3, through a sigmoid). E4M3 stores each (u, v, w) value as a 4-bit-significand residual
from its offset brick's binary16 midrange; the residuals span about a third of the values' range, so
E4M3 PSNR >= 50 dB and max abs <= 2e-2 (without the offsets, per-channel scales alone gave 44.5 dB).
"""

import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

VIEWS = 4
PIX = 1500


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def test_precision_k1024_sampled_parity():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2103_10380_gb300 as fnr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = scenegen.precision()
    k, D, l = w.k, w.D, w.l
    dsig = torch.empty(k ** 3, device=dev, dtype=torch.float32)
    duvw = torch.empty(k ** 3 * 3 * D, device=dev, dtype=torch.float32)
    sig_host = np.empty(k ** 3, dtype=np.float32)
    scenegen.fill_position_grid_device(w.scene, k, dsig, duvw, sig_host)
    beta = scenegen.direction_grid(w.scene, l)
    dbeta = torch.from_numpy(beta.reshape(-1)).to(dev)
    cams = w.cameras()[:VIEWS]
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    npix = w.W * w.H
    rgba = torch.empty((VIEWS, npix * 4), device=dev, dtype=torch.float32)
    stats = torch.empty((VIEWS, npix * 4), device=dev, dtype=torch.int32)
    ctx = fnr.fnr_context_create(0, 0)
    got = {}
    try:
        for name, prec in (("fp16", fnr.FNR_PREC_FP16), ("fp8", fnr.FNR_PREC_FP8_E4M3)):
            cache = fnr.fnr_build_cache(ctx, fnr.make_desc(k, D, l, prec, fnr.FNR_PREC_FP16), dsig, duvw, dbeta)
            for i, c in enumerate(cams):
                fnr.fnr_render(ctx, cache, [fnr.make_camera(c)], params, rgba[i], stats[i])
            torch.cuda.synchronize()
            got[name] = (rgba.cpu().numpy().reshape(VIEWS, w.H, w.W, 4),
                         stats.cpu().numpy().reshape(VIEWS, w.H, w.W, 4))
            fnr.fnr_cache_free(ctx, cache)
    finally:
        fnr.fnr_context_destroy(ctx)
        del dsig, duvw
        torch.cuda.empty_cache()
    op = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    rng = np.random.default_rng(21)
    for i, cam in enumerate(cams):
        px = rng.integers(0, w.W, PIX).astype(np.int32)
        py = rng.integers(0, w.H, PIX).astype(np.int32)
        ref, ref_st, n_cells = oracle.render_pixels_tabled(
            k, D, l, sig_host, beta, lambda c: scenegen.cell_records(w.scene, k, c), cam, op, px, py)
        assert n_cells > 0
        img16, st16 = got["fp16"]
        assert np.array_equal(st16[i][py, px], ref_st), f"view {i}: FP16 integer outputs differ"
        c16 = img16[i][py, px]
        assert np.max(np.abs(c16 - ref)) <= 5e-3
        assert psnr(c16[:, :3], ref[:, :3]) >= 60.0
        img8, _ = got["fp8"]
        c8 = img8[i][py, px, :3]
        assert psnr(c8, ref[:, :3]) >= 50.0, f"view {i}: E4M3 PSNR {psnr(c8, ref[:, :3]):.2f} dB"
        assert np.max(np.abs(c8 - ref[:, :3])) <= 2e-2
