"""Autotuner bookkeeping (no GPU): workload classes and the cache."""
import paper_2109_08206_gb300.autotune as T


def test_workload_key_buckets():
    a = T.workload_key("batch", 1, 1_281_854, 3_221_081, 256)
    b = T.workload_key("batch", 1, 1_300_000, 3_300_000, 256)
    assert a == b                                   # same class
    assert a != T.workload_key("batch", 0, 1_281_854, 3_221_081, 256)   # precision
    assert a != T.workload_key("single", 1, 1_281_854, 3_221_081, 256)
    assert T.workload_key("single", 1, 100_000, 358_098) != T.workload_key("single", 1, 100_000, 1_400_000)


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(T, "_CACHE", tmp_path / "tune.json")
    key = T.workload_key("single", 1, 1000, 3000)
    assert T.cached(key) is None
    T._store(key, (512, 2), {"512x2": 1.0, "1024x1": 2.0})
    assert T.cached(key) == (512, 2)

    class Ctx:
        def set_launch(self, *s):
            self.s = s

    c = Ctx()
    assert T.apply_cached(c, "single", 1, 1000, 3000)
    assert c.s == (512, 2)
    assert not T.apply_cached(c, "batch", 1, 1000, 3000, 4)
