"""Host-side pieces of bench.py that its reported numbers rest on: the algorithmic-bytes formula of the
roofline, the guard that reports the captured DRAM traffic only for the kernel sources it was captured
on, the oracle-counted unique sectors, the peak table's fallback, and the clock record of the timed
region."""

import numpy as np
import pytest

import bench
import oracle
import scenegen


def test_algorithmic_bytes_formula():
    """n_lookups * s_sigma + n_occupied * 3D * s_uvw + rays * (D * s_beta + 16), from per-ray counters."""
    st = np.zeros((2, 3, 4), dtype=np.int32)
    st[..., 1] = [[10, 0, 5], [7, 1, 2]]     # lookups: 25
    st[..., 2] = [[3, 0, 1], [2, 0, 0]]      # occupied: 6
    D = 8
    assert bench.algorithmic_bytes(st, D, 4, 4, 4) == 25 * 4 + 6 * 3 * D * 4 + 6 * (D * 4 + 16)
    assert bench.algorithmic_bytes(st, D, 2, 2, 2) == 25 * 2 + 6 * 3 * D * 2 + 6 * (D * 2 + 16)
    assert bench.algorithmic_bytes(st, 1, 1, 1, 2) == 25 + 6 * 3 + 6 * (2 + 16)


def test_march_traffic_only_for_the_captured_sources(monkeypatch):
    import hashlib
    import os
    h = hashlib.sha256()
    for f in bench.MARCH_SOURCES:
        with open(os.path.join(bench.ROOT, "paper_2103_10380_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    k = bench.MARCH_TRAFFIC["k"]
    monkeypatch.setitem(bench.MARCH_TRAFFIC, "sources_sha256", h.hexdigest())
    assert bench.march_traffic(k) == bench.MARCH_TRAFFIC["bytes_per_launch"]
    assert bench.march_traffic(k + 1) is None              # another workload size
    monkeypatch.setitem(bench.MARCH_TRAFFIC, "sources_sha256", "0" * 64)
    assert bench.march_traffic(k) is None                  # the kernel changed since the capture


def test_unique_sectors_bounded_by_algorithmic(tiny_workload, tiny_arrays):
    """Distinct sectors a frame touches: at least the RGBA image, at most 32 bytes per density lookup plus
    the records' sectors, beta sectors and the image (the sector-granular form of the algorithmic bytes)."""
    w = tiny_workload
    sig, uvw, beta = tiny_arrays
    cam = w.cameras()[0]
    u = bench.unique_sector_bytes(w, sig, uvw, beta, cam)
    oc = oracle.Cache(w.k, w.D, w.l, sig, uvw, beta)
    _, st, _ = oracle.render_image(oc, cam, oracle.params_struct(w.n_samples, w.t_near, w.t_far, w.t_thr, w.bg))
    rays = w.W * w.H
    n_look, n_occ = int(st[..., 1].sum()), int(st[..., 2].sum())
    assert 0 < u["density_sectors"] <= n_look
    assert 0 < u["record_sectors"] <= n_occ * 3 * w.D * 4 // 32
    assert 0 < u["beta_sectors"] <= rays
    assert u["bytes"] == 32 * (u["density_sectors"] + u["record_sectors"] + u["beta_sectors"]) + rays * 16
    upper = n_look * 32 + n_occ * 3 * w.D * 4 + rays * 32 + rays * 16
    assert rays * 16 < u["bytes"] <= upper


def test_measured_peaks_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] > 0 and peaks["bf16_tflops"] > 0


def test_clock_summary_keeps_the_timed_window():
    """The clock record reported beside the number: only samples stamped inside the timed region (widened by
    one sampling interval) count; slowdown reasons of those samples are reported, others are not."""
    import datetime
    import time
    c = bench.ClockSampler(0)
    t0 = time.time()

    def line(t, mhz, power_cap="Not Active", thermal="Not Active"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return (f"{ts}, 0, {mhz}, 2070, 812.5, 0x0000000000000000, Not Active, {thermal}, Not Active, "
                f"{power_cap}")

    c.lines = [line(t0 - 1.0, 990, thermal="Active"),        # before the window: ignored
               line(t0 + 0.010, 2070),
               line(t0 + 0.030, 2055, power_cap="Active"),
               line(t0 + 0.090, 2070),
               "garbage line",
               line(t0 + 5.0, 1200)]                          # after the window: ignored
    s = c.summary(t0, t0 + 0.08, "timed steps")
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["window"] == "timed steps"
    assert bench.ClockSampler(0).summary(t0, t0 + 1)["reasons"] == ["unsampled"]
