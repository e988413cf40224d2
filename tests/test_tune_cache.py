"""Wisdom cache file handling (CPU only)."""
import json

from paper_1406_5597_gb300 import tune


def test_cache_roundtrip_and_merge(tmp_path):
    p = str(tmp_path / "w.json")
    assert tune.load_cache(p) == {}
    k1 = tune.cache_key("NVIDIA GB300", (512, 512, 512), 1, 0, 0)
    k2 = tune.cache_key("NVIDIA GB300", (64, 64, 64), 4, 0, 0)
    assert k1 != k2 and "512x512x512" in k1
    tune.store_cache({k1: [8, 4, 2, 1, 1]}, p)
    tune.store_cache({k2: [0, 16, 4, 0, 1]}, p)
    data = tune.load_cache(p)
    assert data[k1] == [8, 4, 2, 1, 1] and data[k2] == [0, 16, 4, 0, 1]
    json.loads(open(p).read())


def test_corrupt_cache_reads_empty(tmp_path):
    p = tmp_path / "w.json"
    p.write_text("{not json")
    assert tune.load_cache(str(p)) == {}


def test_cache_key_separates_drivers():
    """A new driver may change the fastest kernel shape: keys differ by driver."""
    a = tune.cache_key("NVIDIA GB300", (512, 512, 512), 1, 0, 0, driver=13000)
    b = tune.cache_key("NVIDIA GB300", (512, 512, 512), 1, 0, 0, driver=13010)
    assert a != b and "drv13000" in a
    assert isinstance(tune.driver_version(), int)  # 0 where no driver is installed
