"""Host logic of the tile-walk autotuner (batch.autotune) with a fake clock:
it keeps the fastest candidate, caches the choice per GPU name and workload
key, reuses the cache without timing again, survives a corrupt cache file, and
writes nothing when asked not to."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import batch as GB


class _Renderer:
    def __init__(self, cand):
        self.cand = cand

    def step(self):
        pass


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    made = []
    times = {(False, 0, False): 3.0, (False, 0, True): 2.5, (True, 0, True): 1.25, (True, 4, True): 1.5,
             (True, 3, True): 2.0}

    def make(cand):
        made.append(cand)
        return _Renderer(cand)

    monkeypatch.setenv("GSPLAT103_CACHE", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "Fake GB300")
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(GB, "time_steps", lambda step, n=5, warmup=2: times[(
        step.__self__.cand["persistent"], step.__self__.cand["ctas_per_sm"], step.__self__.cand["longest_first"])])
    return make, made, tmp_path


def test_picks_the_fastest_and_caches_it(fake_gpu):
    make, made, tmp = fake_gpu
    best = GB.autotune(make, key="scene|P100|T40|K900")
    assert (best["persistent"], best["ctas_per_sm"], best["longest_first"]) == (True, 0, True)
    assert best["ms"] == 1.25 and best["cached"] is False and len(best["all"]) == len(GB.CANDIDATES)
    assert len(made) == len(GB.CANDIDATES)
    cache = json.load(open(tmp / "tuning.json"))
    assert list(cache) == ["Fake GB300|scene|P100|T40|K900"]
    # a second call with the same key is answered from the cache: nothing is built or timed
    again = GB.autotune(make, key="scene|P100|T40|K900")
    assert again["cached"] is True and again["ms"] == 1.25 and len(made) == len(GB.CANDIDATES)
    # another workload key is tuned afresh and cached beside the first
    GB.autotune(make, key="other", candidates=GB.CANDIDATES[:2])
    assert len(made) == len(GB.CANDIDATES) + 2
    assert sorted(json.load(open(tmp / "tuning.json"))) == ["Fake GB300|other", "Fake GB300|scene|P100|T40|K900"]


def test_corrupt_cache_is_ignored_and_no_cache_writes_nothing(fake_gpu):
    make, made, tmp = fake_gpu
    (tmp / "tuning.json").write_text("{not json")
    best = GB.autotune(make, key="k", candidates=GB.CANDIDATES[:2])
    assert best["longest_first"] is True and best["cached"] is False
    assert "Fake GB300|k" in json.load(open(tmp / "tuning.json"))
    (tmp / "tuning.json").unlink()
    GB.autotune(make, key="k2", candidates=GB.CANDIDATES[:1], use_cache=False)
    assert not (tmp / "tuning.json").exists()
