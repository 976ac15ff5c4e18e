"""Host-side logic of the sweep autotuner (no GPU)."""
from paper_2606_26547_gb300 import autotune


def test_pick_fastest_and_ties():
    t = {(128, 32): 2.0, (64, 16): 1.5, (256, 16): 1.5}
    assert autotune.pick_fastest(t) == (64, 16)          # first listed among equal times
    assert autotune.pick_fastest({}) is None


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("HDC_TUNE_CACHE", str(tmp_path / "c.json"))
    autotune._store({"k": [64, 16]})
    assert autotune._load() == {"k": [64, 16]}
    monkeypatch.setenv("HDC_TUNE_CACHE", str(tmp_path / "missing" / "x.json"))
    assert autotune._load() == {}
