"""Host logic of the autotuner: search-space enumeration and the per-GPU cache."""
import json

from paper_2009_07174_gb300 import autotune


def test_candidates_cover_space_and_prune():
    c = list(autotune.candidates("frontier"))
    assert all(o["mode"] == "frontier" for o in c)
    assert not any(o["driver"] == "graph" and o["solo_max"] for o in c)
    assert {o["eager"] for o in c} == set(autotune.SPACE["frontier"]["eager"])
    assert len({json.dumps(o, sort_keys=True) for o in c}) == len(c)


def test_choose_precedence(tmp_path):
    path = str(tmp_path / "cache.json")
    assert autotune.choose("frontier", "w", gpu="G", path=path) == autotune.DEFAULTS["frontier"]
    autotune.save_cache({"G": {"default": {"frontier": {"opts": {"block_size": 256}, "ms": 1.0}},
                               "w": {"frontier": {"opts": {"eager": 7}, "ms": 1.0}}}}, path)
    o = autotune.choose("frontier", "w", gpu="G", path=path)
    assert o["eager"] == 7 and o["block_size"] == autotune.DEFAULTS["frontier"]["block_size"]
    o = autotune.choose("frontier", "other", gpu="G", path=path)
    assert o["block_size"] == 256
    assert autotune.choose("frontier", "w", gpu="H", path=path) == autotune.DEFAULTS["frontier"]
