"""Host logic of the row-tile tuner's persisted choices (paper_1810_12357_gb300/tuning.py):
shape classes, the JSON store keyed by GPU name and shape, and its behaviour on a
missing or damaged file.  No GPU: the GPU name is replaced by a fixed string."""
import json

import pytest

from paper_1810_12357_gb300 import tuning


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuning.json"
    monkeypatch.setenv("EHC_TUNE_CACHE", str(path))
    monkeypatch.setattr(tuning, "gpu_name", lambda: "GPU A")
    return path


def test_shape_class_buckets():
    box = (361.5, 361.5, 361.5)
    a = tuning.shape_class(4_000_000, box, 4.0)
    # the same shape class within half a binary order of the atom count
    assert tuning.shape_class(4_100_000, box, 4.0) == a
    assert tuning.shape_class(8_000_000, box, 4.0) != a
    # the skin widens the cells: 84 x 84 rows of 4.3 A cells stay in the class of
    # 90 x 90 (log2 scale), 60 x 60 rows of 6 A cells do not
    assert tuning.shape_class(4_000_000, box, 4.0, skin=0.3) == a
    assert tuning.shape_class(4_000_000, box, 4.0, skin=2.0) != a
    assert tuning.shape_class(4_000_000, box, 4.0, skin=-2.0) == tuning.shape_class(4_000_000, box, 4.0, skin=2.0)
    # replicas are part of the key
    assert tuning.shape_class(4_000_000, box, 4.0, replicas=256) != a
    # 90 x 90 rows of 4.0 A cells: log2(8100) rounds to 13
    assert "_rows13_" in a and a.endswith("_rep1")
    # degenerate inputs still give a key
    assert tuning.shape_class(0, (1.0, 1.0, 1.0), 4.0).startswith("n0_rows0")


def test_store_and_lookup_round_trip(cache):
    assert tuning.lookup("k1") is None            # no file yet
    tuning.store("k1", 256, 3)
    assert cache.exists()
    assert tuning.lookup("k1") == (256, 3)
    tuning.store("k2", 128, 4)
    tuning.store("k1", 128, 2)                    # overwritten, the other key kept
    assert tuning.lookup("k1") == (128, 2)
    assert tuning.lookup("k2") == (128, 4)
    d = json.loads(cache.read_text())
    assert set(d) == {"GPU A"} and set(d["GPU A"]) == {"k1", "k2"}
    # no temporary file is left behind
    assert sorted(p.name for p in cache.parent.iterdir()) == ["tuning.json"]


def test_choices_are_kept_per_gpu(cache, monkeypatch):
    tuning.store("k", 256, 4)
    monkeypatch.setattr(tuning, "gpu_name", lambda: "GPU B")
    assert tuning.lookup("k") is None
    tuning.store("k", 128, 3)
    assert tuning.lookup("k") == (128, 3)
    monkeypatch.setattr(tuning, "gpu_name", lambda: "GPU A")
    assert tuning.lookup("k") == (256, 4)


def test_damaged_file_is_ignored_and_replaced(cache):
    cache.parent.mkdir(parents=True)
    cache.write_text("{not json")
    assert tuning.lookup("k") is None
    tuning.store("k", 256, 2)
    assert tuning.lookup("k") == (256, 2)
    assert json.loads(cache.read_text())["GPU A"]["k"] == {"tile_threads": 256, "grid_quarters": 2}


def test_default_path_under_home(monkeypatch, tmp_path):
    monkeypatch.delenv("EHC_TUNE_CACHE", raising=False)
    monkeypatch.setenv("HOME", str(tmp_path))
    assert tuning.cache_path() == str(tmp_path / ".cache" / "ehc" / "tuning.json")
