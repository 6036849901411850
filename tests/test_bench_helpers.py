"""Host-side helpers of bench.py that its reported numbers rest on: the exact
count of (pixel, Gaussian) pairs the backward of Sec. 3.1 evaluates, the SFU
roofline arithmetic, and the DRAM-traffic record keyed by the raster sources."""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = saved
    return mod


def test_walked_pairs_counts_each_pixels_entries_through_its_last(bench):
    # a 40 x 20 image: 3 x 2 tiles, the last column and row of tiles partial
    W, H = 40, 20
    TX, TY = 3, 2
    rng = np.random.default_rng(0)
    lens = rng.integers(0, 9, TX * TY)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    ranges = np.stack([starts, starts + lens], 1).astype(np.int32)
    last = np.empty((H, W), np.int32)
    expected = 0
    for y in range(H):
        for x in range(W):
            t = (y // 16) * TX + x // 16
            s, e = ranges[t]
            # no composited Gaussian: last = start - 1, else an entry of the tile's list
            last[y, x] = rng.integers(s - 1, e) if e > s else s - 1
            expected += last[y, x] - s + 1
    f = types.SimpleNamespace(tile_ranges=torch.tensor(ranges), last_idx=torch.tensor(last.reshape(-1)))
    cam = types.SimpleNamespace(width=W, height=H)
    assert bench.walked_pairs(f, cam, "cpu") == expected


def test_sfu_roof_charges_one_ex2_and_one_rcp_per_pair(bench):
    r = bench.sfu_roof(10**9, 1e-3, 2000.0)
    per_pair_clk = 1 / bench.MUFU_EX2_PER_SM_CLK + 1 / bench.MUFU_RCP_PER_SM_CLK
    assert r["peak"] == pytest.approx(bench.SMS * 2000e6 / per_pair_clk / 1e9)
    assert r["achieved"] == pytest.approx(1000.0)  # 1e9 pairs in 1 ms = 1000 G pairs/s
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_traffic_record_matches_only_the_current_raster_sources(bench):
    h = bench.raster_source_hash()
    assert len(h) == 64
    rec = {}
    for line in open(os.path.join(ROOT, "profiles", "roofline_traffic.txt")):
        f = line.split()
        if len(f) == 3 and not line.startswith("#"):
            rec[f[0]] = (f[1], int(f[2]))
    for k in ("k_raster_fwd", "k_raster_bwd"):
        want = rec[k][1] if rec.get(k, ("", 0))[0] == h else None
        assert bench.recorded_traffic(k) == want
    assert bench.recorded_traffic("no_such_kernel") is None


def test_clock_summary_reads_nvidia_smi_rows(bench):
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 1965, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, [N/A], 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1011.9, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1980 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == pytest.approx(1011.9)
    c.lines = ["0, 1500, 2070, [N/A], 0x8, Active, Not Active, Active, Not Active"]
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["power_w_max"] is None
    c.lines = []
    assert c.summary() is None


def test_clock_median_is_taken_inside_the_timed_regions(bench):
    import datetime
    c = bench.ClockSampler(0)
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5, 0).timestamp()

    def row(dt, mhz, cap="Not Active"):
        ts = datetime.datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"0, {mhz}, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, {cap}, {ts}"

    # idle before and between the timed regions at a lower clock, under load inside them
    c.lines = [row(0.00, 900), row(0.10, 900), row(0.50, 2010), row(0.52, 1990, "Active"), row(0.54, 2000),
               row(0.80, 1100), row(1.20, 1950), row(1.22, 1970), row(1.60, 800)]
    c.mark(t0 + 0.49, t0 + 0.55)
    c.mark(t0 + 1.19, t0 + 1.23)
    s = c.summary()
    assert s["samples"] == 5 and s["sm_mhz"] == 1990 and s["scope"] == "timed region"
    assert s["reasons"] == ["sw_power_cap"]
    # no sample stamped inside a region (or none stamped at all): every sample counts
    c.windows = [(t0 + 5.0, t0 + 6.0)]
    s = c.summary()
    assert s["samples"] == 9 and s["sm_mhz"] == 1950 and s["scope"].startswith("whole run")


def test_clock_sampler_runs_a_sampler_process_and_windows_its_rows(bench, tmp_path, monkeypatch):
    # a stand-in nvidia-smi on PATH prints one stamped row every 20 ms (SM clock 1000 MHz before the
    # timed region, 2000 MHz inside it); the sampler starts it, reads it on a thread, stops it
    import sys
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text(f"""#!{sys.executable}
import datetime, sys, time
while True:
    now = time.time()
    mhz = 2000 if open({str(tmp_path / 'load')!r}).read().strip() == "1" else 1000
    ts = datetime.datetime.fromtimestamp(now).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print(f"0, {{mhz}}, 2070, 400.0, 0x0, Not Active, Not Active, Not Active, Not Active, {{ts}}", flush=True)
    time.sleep(0.02)
""")
    fake.chmod(0o755)
    (tmp_path / "load").write_text("0")
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    with bench.ClockSampler(0) as clk:
        time.sleep(0.3)
        (tmp_path / "load").write_text("1")
        time.sleep(0.05)
        t0 = time.time()
        time.sleep(0.3)
        t1 = time.time()
        clk.mark(t0, t1)
        time.sleep(0.05)
        (tmp_path / "load").write_text("0")
        time.sleep(0.3)
    s = clk.summary()
    assert clk.proc.poll() is not None  # the sampler process was stopped
    assert s is not None and s["scope"] == "timed region" and s["sm_mhz"] == 2000 and s["samples"] >= 3
