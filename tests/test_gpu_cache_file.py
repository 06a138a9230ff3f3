"""fnr_cache_save / fnr_cache_load: a saved cache, loaded into another context, renders bit-identically
(every section of the device image round-trips); damaged files are refused with FNR_ERR_IO and a load
is charged against the context's budget."""

import os

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
    return fnr


def device_bytes(ptr, nbytes):
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_View(), device="cuda").cpu().numpy()


def render(fnr, ctx, cache, cam, p):
    import torch
    n = cam["W"] * cam["H"]
    rgba = torch.zeros(n * 4, device="cuda")
    stats = torch.zeros(n * 4, device="cuda", dtype=torch.int32)
    fnr.fnr_render(ctx, cache, [cam], p, rgba, stats)
    torch.cuda.synchronize()
    return rgba.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("prec,dprec", [(0, 0), (2, 1)])
def test_save_load_round_trip(fnr, tiny_workload, tiny_arrays, tmp_path, prec, dprec):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    a, b = fnr.fnr_context_create(0, 0), fnr.fnr_context_create(0, 0)
    try:
        cache = fnr.fnr_build_cache(a, fnr.make_desc(w.k, w.D, w.l, prec, dprec, occupancy_brick=4),
                                    sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
        path = tmp_path / "scene.fnrcache"
        fnr.fnr_cache_save(cache, path)
        lay = fnr.fnr_cache_get_layout(cache)
        assert os.path.getsize(path) > lay.footprint
        loaded = fnr.fnr_cache_load(b, path)
        lay2 = fnr.fnr_cache_get_layout(loaded)
        assert (lay2.footprint, lay2.record_stride, lay2.occupancy_brick) == \
            (lay.footprint, lay.record_stride, lay.occupancy_brick)
        # the whole device image round-trips
        base1 = min(lay.sigma_dev, lay.uvw_dev, lay.beta_dev)
        base2 = min(lay2.sigma_dev, lay2.uvw_dev, lay2.beta_dev)
        assert np.array_equal(device_bytes(base1, lay.footprint), device_bytes(base2, lay2.footprint))
        assert fnr.fnr_context_used_bytes(b) == lay.footprint
        cam = w.cameras()[0]
        for p in (fnr.make_params(w.n_samples), fnr.make_params(w.n_samples, skip_empty=True, dir_bilinear=True)):
            r1, s1 = render(fnr, a, cache, cam, p)
            r2, s2 = render(fnr, b, loaded, cam, p)
            assert np.array_equal(r1, r2) and np.array_equal(s1, s2)
    finally:
        fnr.fnr_context_destroy(a)
        fnr.fnr_context_destroy(b)


def test_damaged_files_and_budget(fnr, tiny_workload, tiny_arrays, tmp_path):
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l), sig.reshape(-1), uvw.reshape(-1),
                                    beta.reshape(-1))
        good = tmp_path / "good.fnrcache"
        fnr.fnr_cache_save(cache, good)
        data = good.read_bytes()
        cases = {"missing": None, "empty": b"", "magic": b"XNRCACHE" + data[8:], "version": data[:8] + b"\x07" +
                 data[9:], "truncated": data[: len(data) // 2]}
        for name, content in cases.items():
            p = tmp_path / f"{name}.fnrcache"
            if content is not None:
                p.write_bytes(content)
            with pytest.raises(fnr.FnrError) as ei:
                fnr.fnr_cache_load(ctx, p)
            assert ei.value.status == fnr.FNR_ERR_IO, name
        used = fnr.fnr_context_used_bytes(ctx)
        small = fnr.fnr_context_create(0, 1 << 20)  # 1 MB budget: too small for the 26 MB cache
        try:
            with pytest.raises(fnr.FnrError) as ei:
                fnr.fnr_cache_load(small, good)
            assert ei.value.status == fnr.FNR_ERR_BUDGET
            assert fnr.fnr_context_used_bytes(small) == 0
        finally:
            fnr.fnr_context_destroy(small)
        assert fnr.fnr_context_used_bytes(ctx) == used
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_cache_save(cache, tmp_path / "no_such_dir" / "x.fnrcache")
        assert ei.value.status == fnr.FNR_ERR_IO
    finally:
        fnr.fnr_context_destroy(ctx)
