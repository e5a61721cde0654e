"""The batch autotuner's search and cache, on the CPU, with a stand-in timer."""
import json

from paper_2201_00613_gb300 import batch as B
from paper_2201_00613_gb300 import inputs as I


def test_coordinate_search_and_cache(tmp_path, monkeypatch):
    calls = []

    def fake_time(instances, levels, threads, ctas):
        calls.append((dict(levels or {}), threads, ctas))
        lv = levels or {}
        # best: triangle level 5, carpet level 3 (vicsek untouched), 256 threads, 3 CTAs per SM
        cost = 10.0
        cost -= {5: 2.0, 6: 1.0}.get(lv.get("sierpinski_triangle"), 0.0)
        cost -= {3: 1.5}.get(lv.get("sierpinski_carpet"), 0.0)
        cost -= {256: 0.5}.get(threads, 0.0) + {3: 0.25}.get(ctas, 0.0)
        return cost

    monkeypatch.setattr(B, "_CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(B, "time_config", fake_time)
    monkeypatch.setattr(B, "_device_key", lambda: "stand-in/1")
    monkeypatch.setattr(B, "_level_candidates", lambda f, max_r: {
        "sierpinski_triangle": [4, 5, 6], "sierpinski_carpet": [1, 2, 3], "vicsek": [2, 3, 4]}[f.name])
    mix = I.batch_mix(5, 24)
    res = B.autotune(mix)
    assert res["levels"]["sierpinski_triangle"] == 5
    assert res["levels"]["sierpinski_carpet"] == 3
    assert "vicsek" not in res["levels"]          # no candidate beat the default there
    assert (res["threads"], res["ctas_per_sm"]) == (256, 3)
    assert res["seconds_per_step"] == 10.0 - 2.0 - 1.5 - 0.5 - 0.25
    assert res["trials"] == len(calls) == 1 + 9 + 11
    cached = json.load(open(tmp_path / "autotune.json"))
    assert list(cached.values())[0]["threads"] == 256
    n = len(calls)
    again = B.autotune(mix)                          # from the cache: no new timings
    assert len(calls) == n and again["levels"] == res["levels"]
    other = B.autotune(I.batch_mix(6, 24))           # another mix: tuned afresh
    assert len(calls) > n and other["threads"] == 256
