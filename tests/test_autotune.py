"""Host logic of the autotuner (batch.autotune) with a fake gs_autotune: it
returns the fastest candidate with every candidate's time, caches the choice
per GPU name and workload key, reuses the cache without tuning again, survives
a corrupt cache file, and writes nothing when asked not to; the tuning dict
maps onto a RasterConfig (the C struct's batch-shape fields included)."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB
from paper_2312_02121_gb300 import binding as B


class _Views:
    P, T, pixels, V = 100, 40, 4096, 1


class _Renderer:
    def __init__(self):
        self.views, self.cap, self.forwards = _Views(), 900, 0
        self.p = type("P", (), {"n": 80, "means": torch.zeros(1), "opacities": None, "colors": None})()
        self.means2d = self.conics = self.isect_ids = self.tile_ranges = self.K = None

    def forward(self):
        self.forwards += 1


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    calls = []
    times = [3.0, 2.5, 1.25, 1.5]

    def fake_autotune(views, N, *args, **kw):
        cands = args[-2] if len(args) >= 9 else kw.get("candidates")
        calls.append((views.P, N))
        allc = [dict(persistent=i % 2, ctas_per_sm=0, longest_first=1, bwd_pixels=1 + (i // 2) % 2, bwd_batch=64,
                     ms=t) for i, t in enumerate(times)]
        best = min(allc, key=lambda d: d["ms"])
        return dict(best), allc

    monkeypatch.setenv("GSPLAT103_CACHE", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "Fake GB300")
    monkeypatch.setattr(B, "gs_autotune_workspace_size", lambda *a: 16)
    monkeypatch.setattr(torch, "empty", lambda *a, **kw: torch.zeros(16, dtype=torch.uint8))
    monkeypatch.setattr(B, "gs_autotune", fake_autotune)
    return calls, tmp_path


def test_picks_the_fastest_and_caches_it(fake_gpu):
    calls, tmp = fake_gpu
    r = _Renderer()
    best = GB.autotune(r, key="scene|P100|T40|K900")
    assert best["ms"] == 1.25 and best["cached"] is False and len(best["all"]) == 4
    assert (best["persistent"], best["bwd_pixels"]) == (0, 2)
    assert r.forwards == 1 and calls == [(100, 80)]
    cache = json.load(open(tmp / "tuning.json"))
    assert list(cache) == ["Fake GB300|scene|P100|T40|K900"]
    # a second call with the same key is answered from the cache: nothing is rendered or timed
    again = GB.autotune(r, key="scene|P100|T40|K900")
    assert again["cached"] is True and again["ms"] == 1.25 and len(calls) == 1 and r.forwards == 1
    # another workload key is tuned afresh and cached beside the first
    GB.autotune(r, key="other")
    assert len(calls) == 2
    assert sorted(json.load(open(tmp / "tuning.json"))) == ["Fake GB300|other", "Fake GB300|scene|P100|T40|K900"]


def test_corrupt_cache_is_ignored_and_no_cache_writes_nothing(fake_gpu):
    calls, tmp = fake_gpu
    (tmp / "tuning.json").write_text("{not json")
    best = GB.autotune(_Renderer(), key="k")
    assert best["cached"] is False
    assert "Fake GB300|k" in json.load(open(tmp / "tuning.json"))
    (tmp / "tuning.json").unlink()
    GB.autotune(_Renderer(), key="k2", use_cache=False)
    assert not (tmp / "tuning.json").exists()


def test_tuning_maps_onto_the_raster_config():
    cfg = GB.config(dict(persistent=1, ctas_per_sm=3, longest_first=1, bwd_pixels=2, bwd_batch=128), device="cpu")
    assert (cfg.c.persistent, cfg.c.ctas_per_sm, cfg.c.bwd_pixels, cfg.c.bwd_batch) == (1, 3, 2, 128)
    assert cfg.describe()["bwd_batch"] == 128
