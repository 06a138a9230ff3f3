"""Served rendering (fnr_submit / fnr_poll / fnr_wait) through the C ABI.

Each request's result must be the same rendered alone (fnr_render, one launch)
and in a mix of requests batched into persistent launches: bit-identical,
since both paths run the same per-tile march. One served result is also checked
against the FP64 oracle (counters bit-exact, RGBA within 1e-5)."""

import ctypes
import threading

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
def scenes():
    """Two small scenes: D=8 (tiny workload) and D=4, as float32 arrays."""
    out = []
    w = scenegen.tiny()
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    out.append((w.k, w.D, w.l, sig, uvw, scenegen.direction_grid(w.scene, w.l)))
    sc = scenegen.make_scene(9, n_spheres=10, n_shells=4, D=4, sh_degree=2)
    sig2, uvw2 = scenegen.fill_position_grid(sc, 48)
    out.append((48, 4, 32, sig2, uvw2, scenegen.direction_grid(sc, 32)))
    return out


def build(fnr, ctx, sc, prec=0, dprec=0):
    k, D, l, sig, uvw, beta = sc
    return fnr.fnr_build_cache(ctx, fnr.make_desc(k, D, l, prec, dprec), sig.reshape(-1), uvw.reshape(-1),
                               beta.reshape(-1))


def alone(fnr, ctx, cache, cam, params):
    import torch
    n = cam["W"] * cam["H"]
    rgba = torch.zeros(n * 4, device="cuda")
    stats = torch.zeros(n * 4, device="cuda", dtype=torch.int32)
    fnr.fnr_render(ctx, cache, [cam], params, rgba, stats)
    torch.cuda.synchronize()
    return rgba.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("use_graphs", [1, 0])
def test_alone_equals_mix(fnr, scenes, use_graphs):
    import torch
    ctx = fnr.fnr_context_create(0, 0)
    try:
        fnr.fnr_serve_start(ctx, n_slots=2, max_batch_requests=8, use_graphs=use_graphs)
        caches = [build(fnr, ctx, scenes[0], 0, 0), build(fnr, ctx, scenes[0], 1, 1),
                  build(fnr, ctx, scenes[1], 0, 0), build(fnr, ctx, scenes[1], 2, 1)]
        # two long requests hold both slots while the mix queues up behind them
        hold = []
        for j in range(2):
            cam = scenegen.cameras(40 + j, 1, 1920, 1080)[0]
            out = torch.zeros(1920 * 1080 * 4, device="cuda")
            hold.append((fnr.fnr_submit(ctx, fnr.make_request(caches[0], cam, fnr.make_params(4096, t_thr=0.0),
                                                               out)), out))
        rng = np.random.default_rng(3)
        sizes = [(64, 64), (37, 21), (128, 72), (8, 4), (1, 1), (96, 96)]
        reqs = []
        for i in range(40):
            ci = int(rng.integers(0, len(caches)))
            W, H = sizes[int(rng.integers(0, len(sizes)))]
            cam = scenegen.cameras(500 + i, 1, W, H)[0]
            p = fnr.make_params(int(rng.choice([32, 64, 100])), t_thr=float(rng.choice([1e-4, 1e-2, 0.0])))
            rgba = torch.full((W * H * 4,), float("nan"), device="cuda")
            stats = torch.full((W * H * 4,), -1, device="cuda", dtype=torch.int32)
            r = fnr.make_request(caches[ci], cam, p, rgba, stats)
            reqs.append((fnr.fnr_submit(ctx, r), ci, cam, p, rgba, stats))
        batches = set()
        for t, ci, cam, p, rgba, stats in reqs:
            res = fnr.fnr_wait(ctx, t, 20000)
            assert res.status == fnr.FNR_OK
            assert res.t_submit_ns <= res.t_admit_ns <= res.t_done_ns
            assert res.n_rays == cam["W"] * cam["H"]
            batches.add(res.batch)
        assert len(batches) < len(reqs)  # requests really shared launches
        for t, _ in hold:
            assert fnr.fnr_wait(ctx, t, 60000).status == fnr.FNR_OK
        torch.cuda.synchronize()
        for t, ci, cam, p, rgba, stats in reqs:
            a_rgba, a_st = alone(fnr, ctx, caches[ci], cam, p)
            assert np.array_equal(a_st, stats.cpu().numpy())
            assert np.array_equal(a_rgba, rgba.cpu().numpy())
        # and one of them against the oracle
        t, ci, cam, p, rgba, stats = reqs[0]
        k, D, l, sig, uvw, beta = scenes[0 if ci < 2 else 1]
        prec, dprec = [(0, 0), (1, 1), (0, 0), (2, 1)][ci]
        oc = oracle.quantize_cache(k, D, l, sig, uvw, beta, prec, dprec)
        ref, rst, _ = oracle.render_image(oc, cam, oracle.params_struct(p.n_samples, t_thr=p.t_thr))
        W, H = cam["W"], cam["H"]
        assert np.array_equal(stats.cpu().numpy().reshape(H, W, 4), rst)
        assert np.max(np.abs(rgba.cpu().numpy().reshape(H, W, 4) - ref)) <= 1e-5
    finally:
        fnr.fnr_context_destroy(ctx)


def test_budget_admission_and_errors(fnr, scenes):
    import torch
    probe = fnr.fnr_context_create(0, 0)
    c0 = build(fnr, probe, scenes[0])
    cache_bytes = fnr.fnr_context_used_bytes(probe)
    fnr.fnr_context_destroy(probe)
    W, H = 256, 256
    out_bytes = W * H * 16
    # room for the cache plus one request's output at a time
    ctx = fnr.fnr_context_create(0, cache_bytes + out_bytes + 1024)
    try:
        cache = build(fnr, ctx, scenes[0])
        p = fnr.make_params(64)
        cams = scenegen.cameras(77, 6, W, H)
        outs = [torch.zeros(W * H * 4, device="cuda") for _ in cams]
        tickets = [fnr.fnr_submit(ctx, fnr.make_request(cache, c, p, o)) for c, o in zip(cams, outs)]
        results = [fnr.fnr_wait(ctx, t, 20000) for t in tickets]
        assert all(r.status == fnr.FNR_OK for r in results)
        # admitted one at a time: each admission after the previous completion
        for a, b in zip(results, results[1:]):
            assert b.t_admit_ns >= a.t_done_ns or b.batch == a.batch
        assert fnr.fnr_context_used_bytes(ctx) == cache_bytes
        for o, c in zip(outs, cams):
            ref, _ = alone(fnr, ctx, cache, c, p)
            assert np.array_equal(ref, o.cpu().numpy())
        # an output larger than the whole budget is refused at submit
        big = scenegen.cameras(1, 1, 2048, 2048)[0]
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_submit(ctx, fnr.make_request(cache, big, p, torch.zeros(2048 * 2048 * 4, device="cuda")))
        assert ei.value.status == fnr.FNR_ERR_BUDGET
        # unknown ticket, invalid request
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_poll(ctx, 987654321)
        assert ei.value.status == fnr.FNR_ERR_INVALID_ARG
        bad = fnr.make_request(cache, cams[0], fnr.make_params(0), outs[0])
        with pytest.raises(fnr.FnrError) as ei:
            fnr.fnr_submit(ctx, bad)
        assert ei.value.status == fnr.FNR_ERR_INVALID_ARG
        # a cache with a queued or in-flight request cannot be freed
        t = fnr.fnr_submit(ctx, fnr.make_request(cache, cams[0], fnr.make_params(4096), outs[0]))
        try:
            fnr.fnr_cache_free(ctx, cache)
            freed_early = True
        except fnr.FnrError as e:
            freed_early = False
            assert e.status == fnr.FNR_ERR_INVALID_ARG
        fnr.fnr_wait(ctx, t, 20000)
        if not freed_early:
            fnr.fnr_cache_free(ctx, cache)
    finally:
        fnr.fnr_context_destroy(ctx)


def test_wait_timeout_and_poll(fnr, scenes):
    import torch
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = build(fnr, ctx, scenes[0])
        cam = scenegen.cameras(5, 1, 1920, 1080)[0]
        out = torch.zeros(1920 * 1080 * 4, device="cuda")
        t = fnr.fnr_submit(ctx, fnr.make_request(cache, cam, fnr.make_params(4096, t_thr=0.0), out))
        res = None
        try:
            res = fnr.fnr_wait(ctx, t, 0)
        except fnr.FnrError as e:
            assert e.status == fnr.FNR_ERR_TIMEOUT
        while res is None:
            res = fnr.fnr_poll(ctx, t)
        assert res.status == fnr.FNR_OK
        with pytest.raises(fnr.FnrError):  # the ticket was consumed
            fnr.fnr_poll(ctx, t)
    finally:
        fnr.fnr_context_destroy(ctx)


def test_concurrent_submitters(fnr, scenes):
    import torch
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = build(fnr, ctx, scenes[1])
        p = fnr.make_params(48)
        errors = []
        done = []

        def worker(seed):
            try:
                cams = scenegen.cameras(seed, 10, 40, 30)
                outs = [torch.zeros(40 * 30 * 4, device="cuda") for _ in cams]
                ts = [fnr.fnr_submit(ctx, fnr.make_request(cache, c, p, o)) for c, o in zip(cams, outs)]
                for t in ts:
                    assert fnr.fnr_wait(ctx, t, 20000).status == fnr.FNR_OK
                done.append((cams, outs))
            except Exception as e:  # noqa: BLE001
                errors.append(e)

        ths = [threading.Thread(target=worker, args=(1000 + i,)) for i in range(4)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        assert not errors, errors
        torch.cuda.synchronize()
        for cams, outs in done:
            for c, o in zip(cams, outs):
                ref, _ = alone(fnr, ctx, cache, c, p)
                assert np.array_equal(ref, o.cpu().numpy())
    finally:
        fnr.fnr_context_destroy(ctx)


@pytest.mark.parametrize("idle_spin_us", [-1, 1, 0])
def test_scheduler_idle_spin(fnr, scenes, idle_spin_us):
    """The scheduler's idle policy (poll forever, poll 1 us after the last event then sleep, default)
    changes when it notices work, never what it renders: requests spaced beyond the spin window still
    complete and equal the plain render bit for bit. idle_spin_us < -1 and a non-zero reserved field
    are refused."""
    import time
    import torch
    ctx = fnr.fnr_context_create(0, 0)
    try:
        cache = build(fnr, ctx, scenes[0])
        p = fnr.make_params(48)
        for bad in ((-2, 0), (0, 1)):
            cfg = fnr.fnr_serve_config(0, 0, 0, 0, 1, bad[0], bad[1])
            st = fnr.lib().fnr_serve_start(ctx, ctypes.byref(cfg))
            assert st == fnr.FNR_ERR_INVALID_ARG
        fnr.fnr_serve_start(ctx, n_slots=2, idle_spin_us=idle_spin_us)
        cams = scenegen.cameras(321, 4, 40, 30)
        for c in cams:
            out = torch.zeros(40 * 30 * 4, device="cuda")
            t = fnr.fnr_submit(ctx, fnr.make_request(cache, c, p, out))
            assert fnr.fnr_wait(ctx, t, 20000).status == fnr.FNR_OK
            ref, _ = alone(fnr, ctx, cache, c, p)
            assert np.array_equal(ref, out.cpu().numpy())
            time.sleep(0.01)  # longer than a 1 us window: the scheduler goes to sleep in between
        fnr.fnr_serve_stop(ctx)
    finally:
        fnr.fnr_context_destroy(ctx)


EXIT_SCRIPT = r"""
import sys
import torch
import scenegen
import paper_2103_10380_gb300 as fnr
w = scenegen.tiny()
sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
beta = scenegen.direction_grid(w.scene, w.l)
desc = fnr.make_desc(w.k, w.D, w.l, 0, 0)
req_bytes = 64 * 48 * 16
# queue_full: a budget that holds the cache and leaves one byte less than a request needs, so no
# request is ever admitted and the queue fills; exit: no budget
budget = fnr.fnr_cache_footprint(desc) + req_bytes - 1 if sys.argv[1] == "queue_full" else 0
ctx = fnr.fnr_context_create(0, budget)
cache = fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
fnr.fnr_serve_start(ctx, queue_capacity=16, n_slots=1, idle_spin_us=-1)
outs = [torch.zeros(64 * 48 * 4, device="cuda") for _ in range(8)]
cams = scenegen.cameras(5, 8, 64, 48)
p = fnr.make_params(w.n_samples)
side = torch.cuda.Stream()
with torch.cuda.stream(side):
    torch.cuda._sleep(500_000_000)  # a bounded spin on the outputs' stream: the first batch waits behind it
for i in range(10000):
    fnr.fnr_submit(ctx, fnr.make_request(cache, cams[i % 8], p, outs[i % 8], stream=side))
    if i == 8 and sys.argv[1] == "exit":
        sys.exit(0)
"""


@pytest.mark.parametrize("how", ["exit", "queue_full"])
def test_process_exit_with_live_loop(fnr, how):
    """A process that ends with its request loop still running (never stopped, requests launched or
    queued) ends cleanly: by sys.exit, or by the uncaught QUEUE_FULL error of a burst that the HBM budget
    keeps from being admitted. The loop's thread is stopped before the CUDA runtime shuts down, so the
    exit status is the program's own, never a crash."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", EXIT_SCRIPT, how], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    if how == "exit":
        assert r.returncode == 0, r.stderr[-2000:]
    else:
        assert r.returncode == 1, r.stderr[-2000:]
        assert "QUEUE_FULL" in r.stderr
