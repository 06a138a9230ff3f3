"""Benchmark of the cached FastNeRF render path on GB300.

Default workload (the plain method at the paper's image scale): one 800x800
view per launch, 128 samples per ray, dense k=512^3 FP32 position cache with
D=8 (13.4 GB), 512x512 FP32 direction cache, procedural scene of 32 spheres
and 16 thin shells (seed 0), 8 cameras on the upper hemisphere. One step
renders the 8 views, one launch each. Inputs are synthetic (no dataset).

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s, 800² fps, p50/p99 ms vs FP32 plain at ≥45 dB PSNR to FP64 oracle"
UNIT = "Mrays/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fnr", choices=["fnr", "reference"])
    ap.add_argument("--k", type=int, default=512)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="only the plain FP32 render line")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="arrival window per request rate in the serving workload (its full length is 30)")
    ap.add_argument("--serve-repeats", type=int, default=2, help="runs per request rate in the serving workload")
    ap.add_argument("--only-build", action="store_true",
                    help="time only the tensor-core cache build (F_pos over k^3, F_dir over 512^2)")
    ap.add_argument("--mlp-cta-pair", action="store_true",
                    help="with --only-build: time the CTA-pair form of the build kernel (through its test hook)")
    ap.add_argument("--check-points", type=int, default=1 << 20,
                    help="random grid points of the built cache checked against the FP64 oracle (0: none)")
    ap.add_argument("--only-voxels", action="store_true",
                    help="run only the voxel-walk line (plain and skipping) over the bench views")
    ap.add_argument("--only-serve", action="store_true",
                    help="run only the serving workload (three resident k^3 scenes, Poisson arrivals)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples (every 20 ms, each with its timestamp) while the GPU runs the
    timed region; summary() keeps the samples taken between two host wall-clock times."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s: float = 3.0):
        """Return once the sampler has produced a line (or after timeout_s)."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout_s:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None, window=""):
        """Median SM clock, max clock and active slowdown reasons of the samples stamped within
        [t0, t1] (host epoch seconds, widened by one interval)."""
        import datetime
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        pad = self.INTERVAL_MS * 1e-3
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if t0 is not None and not (t0 - pad <= ts <= t1 + pad):
                    continue
                sm.append(float(parts[2]))
                mx = float(parts[3])
            except ValueError:
                continue
            for n, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        out = {"interval_ms": self.INTERVAL_MS, "window": window}
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, **out}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                **out}


def algorithmic_bytes(stats: np.ndarray, D: int, s_sigma: int, s_uvw: int, s_beta: int) -> int:
    """Bytes the method must move per frame: one density per in-box sample, 3D values per occupied
    sample, D weights per ray, 16 bytes of RGBA per ray."""
    n_look = int(stats[..., 1].astype(np.int64).sum())
    n_occ = int(stats[..., 2].astype(np.int64).sum())
    rays = stats.shape[0] * stats.shape[1]
    return n_look * s_sigma + n_occ * 3 * D * s_uvw + rays * (D * s_beta + 16)


# DRAM bytes (read + write) of one plain FP32 march launch of the default workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); reported only while the kernel sources are unchanged.
MARCH_TRAFFIC = {"sources_sha256": "19ee25ab1d8660dbfe2de8b77a67ce5ed24d22c85a3db3d06bbb04bd8b1bf71a",
                 "bytes_per_launch": 334.0e6, "k": 512}
MARCH_SOURCES = ("march_device.cuh", "march.cu", "fnr_internal.h")


def march_traffic(k: int):
    import hashlib
    h = hashlib.sha256()
    for f in MARCH_SOURCES:
        with open(os.path.join(ROOT, "paper_2103_10380_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != MARCH_TRAFFIC["sources_sha256"] or k != MARCH_TRAFFIC["k"]:
        return None
    return MARCH_TRAFFIC["bytes_per_launch"]


def unique_sector_bytes(w, sig, uvw, beta, cam):
    """Bytes of the distinct 32-byte sectors one view touches (the "unique bytes" of a frame), counted
    from the oracle's per-sample cells of every pixel: the density sectors of all in-box samples up to
    termination, the record sectors of the occupied ones, the beta sectors of the rays' direction cells,
    and the RGBA image. FP32 cache at D=8: 8 densities and exactly 3 records' worth of bytes per 3 sectors."""
    import oracle
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    p = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    _, st, cells = oracle.render_image(oc, cam, p, want_cells=True)
    c = cells.reshape(-1)
    c = c[c >= 0].astype(np.int64)
    n_sig = np.unique(c >> 3).size                      # 8 binary32 densities per sector
    occ = np.unique(c[sig.reshape(-1)[c] > 0])
    rec = 3 * w.D * 4                                   # 96 bytes: 3 whole sectors per record
    assert rec % 32 == 0
    n_rec = occ.size * (rec // 32)
    n_beta = np.unique(st[..., 3].reshape(-1)).size * ((w.D * 4 + 31) // 32)
    return {"density_sectors": int(n_sig), "record_sectors": int(n_rec), "beta_sectors": int(n_beta),
            "bytes": int(32 * (n_sig + n_rec + n_beta) + w.W * w.H * 16)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(w, sig, uvw, beta, cams, seconds: float, seed: int = 0):
    """The FP64 oracle as it stands, on every host core, over random pixels of the workload's views."""
    import oracle
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    p = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    rays = 0
    t0 = time.perf_counter()
    batch = 32768
    i = 0
    while time.perf_counter() - t0 < seconds:
        cam = cams[i % len(cams)]
        px = rng.integers(0, w.W, batch).astype(np.int32)
        py = rng.integers(0, w.H, batch).astype(np.int32)
        oracle.render_pixels(oc, cam, p, px, py, nthreads=cores)
        rays += batch
        i += 1
    dt = time.perf_counter() - t0
    return {"value": rays / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rays} random pixels ({batch} per call) of the {len(cams)} views, {dt:.1f} s, FP64",
            "seconds": dt}


RESOLUTIONS = [(256, 256), (512, 512), (800, 800), (1280, 720), (1920, 1080)]


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


def precision_forms(fnr, torch, ctx, w, sig, uvw, beta, cams, steps, rng_seed=7):
    """FP16 and FP8-E4M3 position caches (FP16 direction cache) of the same scene: render throughput and
    error against the FP64 oracle (which reads the unquantised binary32 cache) on sampled pixels."""
    import oracle
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    op = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    rng = np.random.default_rng(rng_seed)
    samples = []
    for cam in cams:
        px = rng.integers(0, w.W, 2500).astype(np.int32)
        py = rng.integers(0, w.H, 2500).astype(np.int32)
        ref, _, _ = oracle.render_pixels(oc, cam, op, px, py)
        samples.append((px, py, ref))
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    fcams = [fnr.make_camera(c) for c in cams]
    npix = w.W * w.H
    rgba = torch.empty((len(cams), npix * 4), device="cuda", dtype=torch.float32)
    out = {}
    for name, prec, dprec in (("fp32", 0, 0), ("fp16", 1, 1), ("fp8_e4m3", 2, 1)):
        desc = fnr.make_desc(w.k, w.D, w.l, prec, dprec)
        cache = fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
        stream = torch.cuda.current_stream()
        for _ in range(3):
            for i in range(len(cams)):
                fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], None, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            for i in range(len(cams)):
                fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], None, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        imgs = rgba.cpu().numpy().reshape(len(cams), w.H, w.W, 4)
        got = np.concatenate([imgs[i][py, px, :3] for i, (px, py, _) in enumerate(samples)])
        ref = np.concatenate([r[:, :3] for _, _, r in samples])
        out[name] = {"mrays_per_s": steps * len(cams) * npix / (ms * 1e-3) / 1e6,
                     "frame_ms": ms / (steps * len(cams)), "cache_bytes": fnr.fnr_cache_footprint(desc),
                     "max_abs_vs_fp64": float(np.max(np.abs(got - ref))), "psnr_db_vs_fp64": psnr(got, ref),
                     "pixels_checked": int(got.shape[0])}
        fnr.fnr_cache_free(ctx, cache)
    return out


def precision_config(fnr, torch, dev, repeats=5, pix_per_view=20000, rng_seed=7):
    """The precision workload: the scene family at k=1024^3, D=8, position cache in FP16 (53.7 GB) and in
    E4M3 with 25 per-channel scales (26.8 GB), 768x768 FP16 direction cache, 16 views of 800x800, N=192.
    Per view: max abs error and PSNR of sampled pixels against the FP64 oracle reading the unquantised
    binary32 field (the oracle's tabled render: dense sigma plane, uvw evaluated for the cells rays shade),
    plus render throughput (one view per launch). The binary32 source arrays (107 GB) live on the device
    only while the two caches are built."""
    import oracle
    import scenegen
    w = scenegen.precision()
    k, D, l = w.k, w.D, w.l
    t0 = time.perf_counter()
    dsig = torch.empty(k ** 3, device=dev, dtype=torch.float32)
    duvw = torch.empty(k ** 3 * 3 * D, device=dev, dtype=torch.float32)
    sig_host = np.empty(k ** 3, dtype=np.float32)
    scenegen.fill_position_grid_device(w.scene, k, dsig, duvw, sig_host)
    beta = scenegen.direction_grid(w.scene, l)
    dbeta = torch.from_numpy(beta.reshape(-1)).to(dev)
    t_gen = time.perf_counter() - t0
    cams = w.cameras()
    fcams = [fnr.make_camera(c) for c in cams]
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    npix = w.W * w.H
    rgba = torch.empty((len(cams), npix * 4), device=dev, dtype=torch.float32)
    stats = torch.empty((len(cams), npix * 4), device=dev, dtype=torch.int32)
    ctx = fnr.fnr_context_create(dev.index or 0, 0)
    stream = torch.cuda.current_stream(dev)
    images = {}
    out = {"workload": w.name, "k": k, "D": D, "l": l, "n_samples": w.n_samples, "views": len(cams),
           "source_generation_s": t_gen}
    for name, prec in (("fp16", fnr.FNR_PREC_FP16), ("fp8_e4m3", fnr.FNR_PREC_FP8_E4M3)):
        desc = fnr.make_desc(k, D, l, prec, fnr.FNR_PREC_FP16)
        tb = time.perf_counter()
        cache = fnr.fnr_build_cache(ctx, desc, dsig, duvw, dbeta, stream=stream)
        torch.cuda.synchronize(dev)
        t_build = time.perf_counter() - tb
        for i in range(len(cams)):
            fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], stats[i], stream=stream)
        torch.cuda.synchronize(dev)
        images[name] = (rgba.cpu().numpy().reshape(len(cams), w.H, w.W, 4),
                        stats.cpu().numpy().reshape(len(cams), w.H, w.W, 4))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(repeats * len(cams))]
        for r in range(repeats):
            for i in range(len(cams)):
                a, b = ev[r * len(cams) + i]
                a.record(stream)
                fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], None, stream=stream)
                b.record(stream)
        torch.cuda.synchronize(dev)
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        out[name] = {"cache_bytes": fnr.fnr_cache_footprint(desc), "build_s": t_build,
                     "mrays_per_s": npix / (ms.mean() * 1e-3) / 1e6, "fps": 1e3 / ms.mean(),
                     "frame_ms_p50": float(np.percentile(ms, 50)), "frame_ms_p99": float(np.percentile(ms, 99))}
        fnr.fnr_cache_free(ctx, cache)
    del dsig, duvw
    torch.cuda.empty_cache()
    fnr.fnr_context_destroy(ctx)
    # FP64 oracle on sampled pixels of every view
    to = time.perf_counter()
    rng = np.random.default_rng(rng_seed)
    op = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    per_view = {n: [] for n in images}
    stats_equal_fp16 = True
    n_cells = 0
    for i, cam in enumerate(cams):
        px = rng.integers(0, w.W, pix_per_view).astype(np.int32)
        py = rng.integers(0, w.H, pix_per_view).astype(np.int32)
        ref, ref_st, nc = oracle.render_pixels_tabled(
            k, D, l, sig_host, beta, lambda c: scenegen.cell_records(w.scene, k, c), cam, op, px, py)
        n_cells += nc
        for name, (img, st) in images.items():
            got = img[i][py, px, :3]
            per_view[name].append((float(np.max(np.abs(got - ref[:, :3]))), psnr(got, ref[:, :3])))
        # sigma is 0 or 50 in this scene family, both exact in FP16: the integer outputs must match
        stats_equal_fp16 &= bool(np.array_equal(images["fp16"][1][i][py, px], ref_st))
    for name in images:
        errs = np.array(per_view[name])
        out[name].update({"max_abs_vs_fp64": float(errs[:, 0].max()), "psnr_db_min": float(errs[:, 1].min()),
                          "psnr_db_mean": float(errs[:, 1].mean()),
                          "per_view_psnr_db": [round(float(v), 2) for v in errs[:, 1]]})
    out["fp16"]["stats_bit_exact_vs_oracle"] = stats_equal_fp16
    out["oracle"] = {"pixels_per_view": pix_per_view, "shaded_cells_evaluated": n_cells,
                     "seconds": time.perf_counter() - to, "reads": "binary32 field (unquantised)"}
    return out


def cache_build(fnr, torch, ctx, k=512, l=512, check_points=1 << 20):
    """F_pos (8x256 ReLU + head, L=10) over k^3 cell centres and F_dir (4x128 ReLU + head, L=4) over l^2 bins,
    bf16 on the tensor cores with fp32 accumulation; He-uniform weights, seed 0. The first build is also
    checked against the FP64 oracle on check_points random grid points."""
    import scenegen
    pos = scenegen.mlp_weights(0, scenegen.FPOS_DIMS_D8)
    dirn = scenegen.mlp_weights(100, scenegen.FDIR_DIMS_D8)
    dev = lambda L: [(torch.from_numpy(W.view(np.int16)).cuda(), torch.from_numpy(b).cuda()) for W, b in L]
    pl, dl = dev(pos), dev(dirn)
    flop_pt = lambda dims: 2 * sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    flops = flop_pt(scenegen.FPOS_DIMS_D8) * k ** 3 + flop_pt(scenegen.FDIR_DIMS_D8) * l * l
    desc = fnr.make_desc(k, 8, l)
    times = []
    for it in range(2):  # first call includes one-time set-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cache = fnr.fnr_build_cache_mlp(ctx, desc, pl, dl)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        if it == 0 and check_points:
            error = build_error_vs_oracle(fnr, torch, cache, k, l, 8, pos, dirn, check_points)
        fnr.fnr_cache_free(ctx, cache)
    peaks, kind = measured_peaks()
    dt = min(times)
    out = {"workload": f"F_pos over {k}^3 + F_dir over {l}^2, bf16 x bf16 -> fp32", "flops": flops,
           "seconds": dt, "tflops": flops / dt / 1e12, "peak_tflops": float(peaks["bf16_tflops"]),
           "frac": flops / dt / 1e12 / float(peaks["bf16_tflops"]),
           "peak_kind": f"{kind} cuBLAS bf16 (burst)",
           "timing": "whole fnr_build_cache call (includes the cache allocation), best of 2"}
    if check_points:
        out["error_vs_fp64_oracle"] = error
    return out


def build_error_vs_oracle(fnr, torch, cache, k, l, D, pos, dirn, n_points, seed=1):
    """Error of a built cache against the FP64 oracle MLP (same bf16 weights, bf16 rounding of the input
    and of every hidden activation) on n_points random grid cells (seed 1) and n_points / 16 random
    direction bins, per output channel relative to the channel's rms: relative L2, max, and the fraction
    of values within 1e-2 rms."""
    import oracle
    import scenegen
    lay = fnr.fnr_cache_get_layout(cache)
    rng = np.random.default_rng(seed)
    cells = rng.integers(0, k ** 3, n_points)
    bins = rng.integers(0, l * l, max(1, n_points // 16))

    def dev_view(ptr, shape, typestr):
        return torch.as_tensor(type("V", (), {"__cuda_array_interface__": {
            "shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}})(), device="cuda")

    idx = torch.from_numpy(cells).cuda()
    sig = dev_view(lay.sigma_dev, (k ** 3,), "<f4")[idx].cpu().numpy().astype(np.float64)
    rec = dev_view(lay.uvw_dev, (k ** 3, lay.record_stride // 4), "<f4")[idx].cpu().numpy()
    got = np.concatenate([sig[:, None], rec[:, :3 * D].astype(np.float64)], axis=1)
    beta = dev_view(lay.beta_dev, (l * l, D), "<f4")[torch.from_numpy(bins).cuda()].cpu().numpy()
    as64 = lambda L: [(scenegen.bf16_value(W).astype(np.float64), b.astype(np.float64)) for W, b in L]
    t0 = time.perf_counter()
    ref = oracle.mlp_eval(as64(pos), oracle.cell_centres(k, cells), 10, True)
    ref[:, 0] = np.maximum(ref[:, 0], 0.0)
    bref = oracle.mlp_eval(as64(dirn), oracle.bin_directions(l, bins), 4, True)
    t_oracle = time.perf_counter() - t0

    def stats(g, r):
        rms = np.sqrt(np.mean(r ** 2, axis=0)) + 1e-12
        e = np.abs(g - r) / rms
        return {"rel_l2_max": float(np.sqrt(np.mean(e ** 2, axis=0)).max()), "max_over_rms": float(e.max()),
                **{f"frac_within_{t:g}_rms_min": float(np.mean(e <= t, axis=0).min()) for t in (1e-2, 3e-2)}}

    return {"f_pos": {"points": int(n_points), **stats(got, ref)},
            "f_dir": {"points": int(bins.size), **stats(beta.astype(np.float64), bref)},
            "oracle_seconds": t_oracle, "oracle_cores": os.cpu_count() or 1}


def uncached_render(fnr, torch, dev, w, reps=3):
    """The uncached render (the paper's "no cache" row): one 800x800 view, N=128, F_pos (8x256 + head, L=10)
    at every inside sample and F_dir (4x128 + head, L=4) per ray on the tensor cores, random He-uniform
    weights; the per-frame time of fnr_render_mlp (samples, both MLPs, compositing) and the MLP FLOPs."""
    import scenegen
    pos = scenegen.mlp_weights(0, scenegen.FPOS_DIMS_D8)
    dirn = scenegen.mlp_weights(100, scenegen.FDIR_DIMS_D8)
    devw = lambda L: [(torch.from_numpy(W.view(np.int16)).to(dev), torch.from_numpy(b).to(dev)) for W, b in L]
    pl, dl = devw(pos), devw(dirn)
    ctx = fnr.fnr_context_create(dev.index or 0, 0)
    cam = w.cameras()[0]
    npix = w.W * w.H
    rgba = torch.empty(npix * 4, device=dev)
    stats = torch.empty(npix * 4, device=dev, dtype=torch.int32)
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    fnr.fnr_render_mlp(ctx, pl, dl, w.D, cam, params, rgba, stats)
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fnr.fnr_render_mlp(ctx, pl, dl, w.D, cam, params, rgba, None)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    fnr.fnr_context_destroy(ctx)
    # every inside sample is evaluated: count them with the oracle's sample positions (same binary32 rule)
    import ctypes
    import oracle
    py, px = np.meshgrid(np.arange(w.H, dtype=np.int32), np.arange(w.W, dtype=np.int32), indexing="ij")
    px, py = np.ascontiguousarray(px.reshape(-1)), np.ascontiguousarray(py.reshape(-1))
    op = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    pts = np.zeros((npix, w.n_samples, 3), np.float32)
    inside = np.zeros((npix, w.n_samples), np.uint8)
    dirs = np.zeros((npix, 3), np.float32)
    lo, hi = np.full(3, -1.5, np.float32), np.full(3, 1.5, np.float32)
    oracle.lib().orc_mlp_samples(ctypes.byref(oracle.camera_struct(cam)), ctypes.byref(op), lo.ctypes.data,
                                 hi.ctypes.data, npix, px.ctypes.data, py.ctypes.data, pts.ctypes.data,
                                 inside.ctypes.data, dirs.ctypes.data)
    n_pts = int(inside.sum())
    fl = lambda dims: 2 * sum(a * b for a, b in zip(dims[:-1], dims[1:]))
    flops = fl(scenegen.FPOS_DIMS_D8) * n_pts + fl(scenegen.FDIR_DIMS_D8) * npix
    dt = min(times)
    return {"workload": f"{w.W}x{w.H}, N={w.n_samples}, random He-uniform F_pos / F_dir", "frame_ms": dt * 1e3,
            "mrays_per_s": npix / dt / 1e6, "inside_samples": n_pts, "mlp_flops": flops,
            "mlp_tflops": flops / dt / 1e12,
            "timing": "whole fnr_render_mlp call (allocation, samples, F_pos over every inside sample, F_dir per "
                      "ray, compositing), best of %d" % reps}


RATES = (50.0, 100.0, 200.0, 400.0, 2000.0, 5000.0)
CLOSED_LOOP_REQUESTS = 1200


def serving_config(fnr, torch, dev, w, sig, uvw, beta, seconds, rates=RATES, seed=11, budget=120e9, repeats=2):
    """The serving workload: three resident scenes (seeds 0, 1, 2; k=512^3, D=8, 512^2 direction grid),
    each with an FP16 and an E4M3 position cache (served; FP16 direction cache) and an FP32 one (plain),
    all inside one context with a 120 GB HBM budget. Poisson arrivals at each rate for `seconds`; every
    request draws a scene, an upper-hemisphere camera and a resolution from RESOLUTIONS, N=128.
    Served: fnr_submit (continuous batching into graph launches). Plain: fnr_render, one frame per
    launch, one request at a time in arrival order (latency counts the wait for earlier requests).
    Each rate is run `repeats` times with fresh draws (p50/p99 per repeat, and their median / spread).
    The two highest rates load the GPU enough that launches batch several requests. Then closed loop
    (1200 requests drawn like the 400 req/s ones, submitted at once) for throughput."""
    import scenegen
    ctx = fnr.fnr_context_create(dev.index or 0, int(budget))
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    caches = {"fp16": [], "fp8_e4m3": [], "fp32": []}
    forms = (("fp16", fnr.FNR_PREC_FP16, fnr.FNR_PREC_FP16), ("fp8_e4m3", fnr.FNR_PREC_FP8_E4M3, fnr.FNR_PREC_FP16),
             ("fp32", fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32))
    t0 = time.perf_counter()
    for scene_seed in (0, 1, 2):
        if scene_seed == 0:
            s_, u_, b_ = sig, uvw, beta
        else:
            ws = scenegen.scale(seed=scene_seed)
            s_, u_ = scenegen.fill_position_grid(ws.scene, ws.k)
            b_ = scenegen.direction_grid(ws.scene, ws.l)
        for name, prec, dprec in forms:
            caches[name].append(fnr.fnr_build_cache(ctx, fnr.make_desc(w.k, w.D, w.l, prec, dprec),
                                                    s_.reshape(-1), u_.reshape(-1), b_.reshape(-1)))
        del s_, u_, b_
    t_setup = time.perf_counter() - t0
    resident = fnr.fnr_context_used_bytes(ctx)
    pool = {(W, H): [torch.empty(W * H * 4, device=dev) for _ in range(160)] for W, H in RESOLUTIONS}
    used = {key: 0 for key in pool}

    def out_for(cam):
        key = (cam.width, cam.height)
        t = pool[key][used[key] % len(pool[key])]
        used[key] += 1
        return t

    def workload(rate, rng, n=None):
        n = max(8, int(rate * seconds)) if n is None else n
        reqs = []
        for i in range(n):
            W, H = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
            cam = fnr.make_camera(scenegen.cameras(int(rng.integers(1, 2 ** 31)), 1, W, H, hemisphere=True)[0])
            reqs.append((int(rng.integers(0, 3)), cam))
        return reqs, np.cumsum(rng.exponential(1.0 / rate, n))

    def run_served(form, reqs, arrivals):
        tickets = []
        t0 = time.perf_counter()
        for i, (sc, cam) in enumerate(reqs):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
            tickets.append(fnr.fnr_submit(ctx, fnr.make_request(caches[form][sc], cam, params, out_for(cam))))
        lat, t_first, t_last = [], None, None
        for t in tickets:
            r = fnr.fnr_wait(ctx, t, 60000)
            if r.status != 0:
                raise RuntimeError(f"served request failed with status {r.status}")
            lat.append((r.t_done_ns - r.t_submit_ns) * 1e-6)
            t_first = r.t_submit_ns if t_first is None else min(t_first, r.t_submit_ns)
            t_last = r.t_done_ns if t_last is None else max(t_last, r.t_done_ns)
        return np.array(lat), (t_last - t_first) * 1e-9

    def run_plain(reqs, arrivals):
        lat = []
        stream = torch.cuda.current_stream(dev)
        t0 = time.perf_counter()
        for i, (sc, cam) in enumerate(reqs):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
            arrive = t0 + (arrivals[i] if arrivals is not None else 0.0)
            fnr.fnr_render(ctx, caches["fp32"][sc], [cam], params, out_for(cam), None, stream=stream)
            stream.synchronize()
            lat.append((time.perf_counter() - arrive) * 1e3)
        return np.array(lat), time.perf_counter() - t0

    def summary(lat, span, n):
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "frames_per_s": n / span}

    def combine(runs):
        """Per-repeat summaries -> the medians plus every repeat's p50 / p99."""
        out = {key: float(np.median([r[key] for r in runs])) for key in ("p50_ms", "p99_ms", "frames_per_s")}
        out["p50_ms_runs"] = [round(r["p50_ms"], 4) for r in runs]
        out["p99_ms_runs"] = [round(r["p99_ms"], 4) for r in runs]
        return out

    # the scheduler thread polls continuously while serving (lowest latency; one busy host thread)
    fnr.fnr_serve_start(ctx, n_slots=3, max_batch_requests=64, use_graphs=1, idle_spin_us=-1)
    torch.cuda.synchronize(dev)
    rng = np.random.default_rng(seed)
    # the untimed warm-up and the closed loop submit every request at once: fixed sizes within the
    # request queue's capacity (4096 pending requests), whatever the seconds per rate
    warm, _ = workload(200.0, rng, n=600)
    for form in ("fp16", "fp8_e4m3"):
        run_served(form, warm, None)  # graphs captured, kernels loaded
    run_plain(warm, None)
    res = {}
    for rate in rates:
        runs = {"served_fp16": [], "served_fp8_e4m3": [], "plain_fp32_per_frame": []}
        n_req = 0
        for _ in range(repeats):
            reqs, arrivals = workload(rate, rng)
            n_req += len(reqs)
            for form in ("fp16", "fp8_e4m3"):
                runs["served_" + form].append(summary(*run_served(form, reqs, arrivals), len(reqs)))
            runs["plain_fp32_per_frame"].append(summary(*run_plain(reqs, arrivals), len(reqs)))
        row = {"requests": n_req, "repeats": repeats, **{key: combine(v) for key, v in runs.items()}}
        res[f"{int(rate)}_req_per_s"] = row
    reqs, _ = workload(400.0, rng, n=CLOSED_LOOP_REQUESTS)
    row = {"requests": len(reqs)}
    for form in ("fp16", "fp8_e4m3"):
        row["served_" + form] = summary(*run_served(form, reqs, None), len(reqs))
    row["plain_fp32_per_frame"] = summary(*run_plain(reqs, None), len(reqs))
    res["closed_loop"] = row
    fnr.fnr_serve_stop(ctx)
    for lst in caches.values():
        for c in lst:
            fnr.fnr_cache_free(ctx, c)
    fnr.fnr_context_destroy(ctx)
    return {"scenes": 3, "hbm_budget_bytes": int(budget), "resident_cache_bytes": int(resident),
            "seconds_per_rate": seconds, "repeats": repeats, "resolutions": RESOLUTIONS, "n_samples": w.n_samples,
            "setup_s": t_setup, **res,
            "latency": "submit -> completion seen by the host (served); arrival -> frame synchronised (plain)",
            "scheduler": "fnr_serve_start(n_slots=3, max_batch_requests=64, use_graphs=1, idle_spin_us=-1): "
                         "the scheduler thread polls continuously while serving"}


def rank_views(w, rank: int) -> list:
    """Weak scaling: every rank renders its own views of the same scene (camera seed offset by rank)."""
    import scenegen
    return scenegen.cameras(w.cam_seed + 1000 * rank, w.n_cams, w.W, w.H, hemisphere=True)


def reduce_max(value: float, world: int, device=None) -> float:
    """Largest value over the ranks (the job's elapsed time is the slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, elapsed_ms: float) -> float:
    """Whole-job throughput in millions of units per second: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (elapsed_ms * 1e-3) / 1e6


def make_workload(k):
    import scenegen
    return scenegen.scale(k=k)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import scenegen
    w = make_workload(args.k)
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)
    cams = w.cameras()
    import oracle
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    p = oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    cores = os.cpu_count() or 1
    per_step = 65536  # rays per step: a bounded sample of one 800x800 view
    rng = np.random.default_rng(1)

    def step(i):
        cam = cams[i % len(cams)]
        px = rng.integers(0, w.W, per_step).astype(np.int32)
        py = rng.integers(0, w.H, per_step).astype(np.int32)
        oracle.render_pixels(oc, cam, p, px, py, nthreads=cores)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "rays_per_step": per_step, "k": w.k, "D": w.D, "l": w.l,
                      "n_samples": w.n_samples},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} random pixels of one of the 8 views per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


def voxel_walk_line(fnr, torch, ctx, cache, w, fcams, rgba, stats, stream, steps):
    """The voxel walk (FNR_RENDER_VOXELS) over the bench views, plain and with skipping: per view one launch
    with the per-ray counters (algorithmic bytes), two untimed passes, then max(3, steps / 20) timed passes."""
    occ_bytes = (((w.k + 7) // 8) ** 3 + 7) // 8
    npix = w.W * w.H
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # every cell a ray passes through, N = 3k caps nothing
    voxel_line = {}
    for vskip in (False, True):
        params_v = fnr.make_params(3 * w.k, w.t_near, w.t_far, w.t_thr, w.bg, skip_empty=vskip, voxels=True)
        rgba_v = torch.empty_like(rgba)
        stats_v = torch.empty_like(stats)
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, cache, [fcams[i]], params_v, rgba_v[i], stats_v[i], stream=stream)
        torch.cuda.synchronize()
        st_v = stats_v.cpu().numpy().reshape(w.n_cams, w.H, w.W, 4)
        alg_v = float(np.mean([algorithmic_bytes(st_v[i], w.D, 4, 4, 4) for i in range(w.n_cams)]))
        if vskip:
            alg_v += occ_bytes
        v_steps = max(3, steps // 20)
        for _ in range(2):
            for i in range(w.n_cams):
                fnr.fnr_render(ctx, cache, [fcams[i]], params_v, rgba_v[i], None, stream=stream)
        k0.record(stream)
        for s_ in range(v_steps):
            for i in range(w.n_cams):
                fnr.fnr_render(ctx, cache, [fcams[i]], params_v, rgba_v[i], None, stream=stream)
        k1.record(stream)
        torch.cuda.synchronize()
        v_ms = k0.elapsed_time(k1) / (v_steps * w.n_cams)
        voxel_line["skip_empty" if vskip else "plain"] = {
            "mrays_per_s": npix / (v_ms * 1e-3) / 1e6, "launch_ms": v_ms,
            "cells_per_ray": float(st_v[..., 0].mean()), "lookups_per_ray": float(st_v[..., 1].mean()),
            "occupied_per_ray": float(st_v[..., 2].mean()),
            "roofline_frac": alg_v / (v_ms * 1e-3) / 1e9 / float(measured_peaks()[0]["hbm_gbs"]),
            "algorithmic_bytes_per_launch": alg_v}
        del rgba_v, stats_v
    voxel_line["n_samples"] = 3 * w.k
    voxel_line["bytes"] = "densities looked up + records of composited cells + beta + RGBA (+ brick bits)"
    return voxel_line


def run_fnr(args):
    import torch
    import scenegen
    import paper_2103_10380_gb300 as fnr

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = make_workload(args.k)
    cams = rank_views(w, rank)
    sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
    beta = scenegen.direction_grid(w.scene, w.l)

    ctx = fnr.fnr_context_create(local, 0)
    desc = fnr.make_desc(w.k, w.D, w.l, fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32)
    cache = fnr.fnr_build_cache(ctx, desc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    params = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg)
    npix = w.W * w.H
    fcams = [fnr.make_camera(c) for c in cams]
    rgba = torch.empty((w.n_cams, npix * 4), device=dev, dtype=torch.float32)
    stats = torch.empty((w.n_cams, npix * 4), device=dev, dtype=torch.int32)
    stream = torch.cuda.current_stream(dev)

    # algorithmic bytes per launch, from the kernel's own per-ray counters (same counts as the oracle)
    alg = []
    for i in range(w.n_cams):
        fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], stats[i], stream=stream)
    torch.cuda.synchronize()
    st_all = stats.cpu().numpy().reshape(w.n_cams, w.H, w.W, 4)
    for i in range(w.n_cams):
        alg.append(algorithmic_bytes(st_all[i], w.D, 4, 4, 4))
    alg_per_launch = float(np.mean(alg))
    if args.only_voxels:
        print(json.dumps({"voxel_walk": voxel_walk_line(fnr, torch, ctx, cache, w, fcams, rgba, stats, stream,
                                                        args.steps), "config": {"workload": w.name}}), flush=True)
        fnr.fnr_context_destroy(ctx)
        return

    def step(events=None):
        for i in range(w.n_cams):
            if events is not None:
                events[i][0].record(stream)
            fnr.fnr_render(ctx, cache, [fcams[i]], params, rgba[i], None, stream=stream)
            if events is not None:
                events[i][1].record(stream)

    frame_events = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(w.n_cams)] for _ in range(max(5, args.steps // 4))]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat_steps = max(5, args.steps // 4)
    with ClockSampler(local) as clocks:
        clocks.wait_first()  # sampling before the timed region starts
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall0 = time.time()
        t_start.record(stream)
        for s in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
        wall1 = time.time()
        if world > 1:
            torch.distributed.barrier()
        # per-launch durations (p50/p99 frame time): a second pass with an event pair around every launch,
        # which also keeps consecutive launches from overlapping
        for s in range(lat_steps):
            step(frame_events[s])
        torch.cuda.synchronize()
        wall2 = time.time()
    clock_summary = clocks.summary(wall0, wall1, "timed steps")
    if clock_summary["samples"] < 3:  # a short timed region: the same load through the per-launch pass
        clock_summary = clocks.summary(wall0, wall2, "timed steps and the per-launch pass that follows")
    total_ms = t_start.elapsed_time(t_end)
    frame_ms = np.array([[a.elapsed_time(b) for a, b in ev] for ev in frame_events[:lat_steps]]).reshape(-1)
    total_ms = reduce_max(total_ms, world, dev)
    value = job_rate(args.steps * w.n_cams * npix, world, total_ms)

    # end to end through the public API with host buffers: camera structs go host -> device with each
    # launch, every frame's RGBA comes back to pinned host memory inside the timed region. The read-back
    # is pipelined with double-buffered outputs: a step renders its views back to back into one set of
    # buffers (consecutive launches still overlap through programmatic dependent launch; an event
    # between them would stop that), then a second stream copies that set to the host while the next
    # step renders into the other set; a set is rendered into again only once its copies have finished,
    # and the timed region ends when the last copy has.
    host_out = torch.empty((w.n_cams, npix * 4), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(20, args.steps // 10)  # enough steps that the two-set pipeline's fill and drain are small
    copy_stream = torch.cuda.Stream(dev)
    out_sets = [rgba, [torch.empty_like(rgba[i]) for i in range(w.n_cams)]]
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(j):
        b = j % 2
        if j >= 2:
            stream.wait_event(copied[b])
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, cache, [fcams[i]], params, out_sets[b][i], None, stream=stream)
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            for i in range(w.n_cams):
                host_out[i].copy_(out_sets[b][i], non_blocking=True)
        copied[b].record(copy_stream)

    for j in range(2):
        e2e_step(j)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(e2e_steps):
        e2e_step(j + 2)
    stream.wait_event(copied[(e2e_steps + 1) % 2])  # copies complete in order on copy_stream
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = e2e_steps * w.n_cams * npix * world / (e2e_ms * 1e-3) / 1e6

    # empty-space skipping (FNR_RENDER_SKIP_EMPTY): same views, density lookups only in occupied bricks
    params_skip = fnr.make_params(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg, skip_empty=True)
    rgba_skip = torch.empty_like(rgba)
    stats_skip = torch.empty_like(stats)
    for i in range(w.n_cams):
        fnr.fnr_render(ctx, cache, [fcams[i]], params_skip, rgba_skip[i], stats_skip[i], stream=stream)
    fnr.fnr_render(ctx, cache, fcams[:1], params, rgba[0], None, stream=stream)
    torch.cuda.synchronize()
    skip_identical = bool(torch.equal(rgba_skip[0], rgba[0]))
    st_skip = stats_skip.cpu().numpy().reshape(w.n_cams, w.H, w.W, 4)
    occ_bytes = (((w.k + 7) // 8) ** 3 + 7) // 8
    alg_skip = float(np.mean([algorithmic_bytes(st_skip[i], w.D, 4, 4, 4) for i in range(w.n_cams)])) + occ_bytes
    sk_steps = max(5, args.steps // 4)
    for _ in range(3):
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, cache, [fcams[i]], params_skip, rgba_skip[i], None, stream=stream)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for s_ in range(sk_steps):
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, cache, [fcams[i]], params_skip, rgba_skip[i], None, stream=stream)
    k1.record(stream)
    torch.cuda.synchronize()
    sk_launch_ms = k0.elapsed_time(k1) / (sk_steps * w.n_cams)

    # the same scene as a sparse brick cache (FNR_LAYOUT_BRICKS, always skipping)
    bdesc = fnr.make_desc(w.k, w.D, w.l, fnr.FNR_PREC_FP32, fnr.FNR_PREC_FP32, layout=fnr.FNR_LAYOUT_BRICKS)
    bcache = fnr.fnr_build_cache(ctx, bdesc, sig.reshape(-1), uvw.reshape(-1), beta.reshape(-1))
    blay = fnr.fnr_cache_get_layout(bcache)
    rgba_b = torch.empty_like(rgba)
    fnr.fnr_render(ctx, bcache, fcams[:1], params_skip, rgba_b[0], None, stream=stream)
    torch.cuda.synchronize()
    bricks_identical = bool(torch.equal(rgba_b[0], rgba_skip[0]))
    for _ in range(3):
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, bcache, [fcams[i]], params_skip, rgba_b[i], None, stream=stream)
    k0.record(stream)
    for s_ in range(sk_steps):
        for i in range(w.n_cams):
            fnr.fnr_render(ctx, bcache, [fcams[i]], params_skip, rgba_b[i], None, stream=stream)
    k1.record(stream)
    torch.cuda.synchronize()
    br_launch_ms = k0.elapsed_time(k1) / (sk_steps * w.n_cams)
    bricks_line = {"mrays_per_s": npix / (br_launch_ms * 1e-3) / 1e6, "launch_ms": br_launch_ms,
                   "cache_bytes": int(blay.footprint), "dense_cache_bytes": int(fnr.fnr_cache_footprint(desc)),
                   "bricks": int(blay.n_bricks), "brick": int(blay.occupancy_brick),
                   "image_bit_identical_to_dense_skip": bricks_identical}
    fnr.fnr_cache_free(ctx, bcache)
    del rgba_skip, stats_skip, rgba_b

    voxel_line = voxel_walk_line(fnr, torch, ctx, cache, w, fcams, rgba, stats, stream, args.steps)

    # the same 8 views in one launch (fnr_render takes several cameras): no per-launch tail
    for _ in range(3):
        fnr.fnr_render(ctx, cache, fcams, params, rgba.view(-1), None, stream=stream)
    mv_steps = max(5, args.steps // 4)
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(mv_steps):
        fnr.fnr_render(ctx, cache, fcams, params, rgba.view(-1), None, stream=stream)
    m1.record(stream)
    torch.cuda.synchronize()
    mv_ms = m0.elapsed_time(m1) / mv_steps

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        launch_ms = total_ms / (args.steps * w.n_cams)  # per launch inside the timed region (back to back)
        achieved = alg_per_launch / (launch_ms * 1e-3) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "k": w.k, "D": w.D, "l": w.l, "W": w.W, "H": w.H,
                       "n_samples": w.n_samples, "views_per_step": w.n_cams, "launch": "one view per launch",
                       "cache": "fp32 sigma plane + fp32 uvw records", "cache_bytes": fnr.fnr_cache_footprint(desc),
                       "l2": "inputs larger than L2 (13.4 GB cache, ~0.3-0.6 GB touched per view), views cycled",
                       "parallelism": f"dp{world} (independent views per GPU)"},
            "fps": w.n_cams * args.steps * world / (total_ms * 1e-3),
            "frame_ms_p50": float(np.percentile(frame_ms, 50)), "frame_ms_p99": float(np.percentile(frame_ms, 99)),
            "roofline": {"bound": "hbm", "kernel": "march_kernel<fp32, D=8>", "achieved": achieved,
                         "peak": float(peaks["hbm_gbs"]), "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]),
                         "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                         "algorithmic_bytes_per_launch": alg_per_launch, "launch_ms": launch_ms,
                         "launch_ms_isolated": float(np.mean(frame_ms)),
                         "timing": "launch_ms = timed region / launches (consecutive launches overlap through "
                                   "programmatic dependent launch); launch_ms_isolated = mean of event pairs "
                                   "around single launches",
                         "traffic": march_traffic(w.k)},
            "skip_empty": {
                "mrays_per_s": npix / (sk_launch_ms * 1e-3) / 1e6, "launch_ms": sk_launch_ms,
                "image_bit_identical_to_plain": skip_identical, "occupancy_brick": 8,
                "lookups_per_ray": float(st_skip[..., 1].mean()), "plain_lookups_per_ray": float(st_all[..., 1].mean()),
                "roofline": {"bound": "hbm", "achieved": alg_skip / (sk_launch_ms * 1e-3) / 1e9,
                             "frac": alg_skip / (sk_launch_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"]),
                             "algorithmic_bytes_per_launch": alg_skip,
                             "bytes": "densities looked up + records of occupied samples + beta + RGBA + brick bits"}},
            "bricks_layout": bricks_line,
            "voxel_walk": voxel_line,
            "all_views_one_launch": {
                "mrays_per_s": w.n_cams * npix / (mv_ms * 1e-3) / 1e6, "launch_ms": mv_ms,
                "roofline_frac": alg_per_launch * w.n_cams / (mv_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"])},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": w.n_cams * 72,
                    "d2h_bytes_per_step": w.n_cams * npix * 16,
                    "pipeline": "fnr_render per view on the render stream into one of two output sets; a step's "
                                "RGBA copied to pinned host memory on a second stream while the next step renders "
                                "into the other set"},
            "clocks": clock_summary,
            "gpu_launches": args.steps * w.n_cams,
        }
    fnr.fnr_cache_free(ctx, cache)
    if rank == 0:
        # distinct sectors the first view touches, from the oracle's cells (against the same launch time)
        ub = unique_sector_bytes(w, sig, uvw, beta, cams[0])
        out["roofline"]["unique_bytes_view0"] = ub["bytes"]
        out["roofline"]["unique_frac"] = ub["bytes"] / (out["roofline"]["launch_ms"] * 1e-3) / 1e9 / \
            out["roofline"]["peak"]
        if not args.no_extras:
            out["precision_forms"] = precision_forms(fnr, torch, ctx, w, sig, uvw, beta, cams, max(5, args.steps // 10))
            out["serving"] = serving_config(fnr, torch, dev, w, sig, uvw, beta, args.serve_seconds,
                                            repeats=args.serve_repeats)
            out["precision_k1024"] = precision_config(fnr, torch, dev)
            out["cache_build"] = cache_build(fnr, torch, ctx)
            out["uncached_render"] = uncached_render(fnr, torch, dev, w)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, sig, uvw, beta, cams, args.cpu_seconds)
        print(json.dumps(out), flush=True)
    fnr.fnr_context_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.only_build:
        import torch
        import paper_2103_10380_gb300 as fnr
        torch.cuda.set_device(0)
        ctx = fnr.fnr_context_create(0, 0)
        fnr.fnr_testing_mlp_cta_pair(args.mlp_cta_pair)
        out = cache_build(fnr, torch, ctx, k=args.k, check_points=args.check_points)
        out["kernel_form"] = "CTA pair (cta_group::2)" if args.mlp_cta_pair else "single CTA per SM"
        fnr.fnr_testing_mlp_cta_pair(False)
        print(json.dumps({"cache_build": out}), flush=True)
        fnr.fnr_context_destroy(ctx)
        return
    if args.only_serve:
        import torch
        import scenegen
        import paper_2103_10380_gb300 as fnr
        torch.cuda.set_device(0)
        w = make_workload(args.k)
        sig, uvw = scenegen.fill_position_grid(w.scene, w.k)
        beta = scenegen.direction_grid(w.scene, w.l)
        out = serving_config(fnr, torch, torch.device("cuda", 0), w, sig, uvw, beta, args.serve_seconds,
                             repeats=args.serve_repeats)
        print(json.dumps({"serving": out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fnr(args)


if __name__ == "__main__":
    main()
