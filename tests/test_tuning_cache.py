"""The autotuner's JSON cache (host logic): a miss tunes and records, a hit
applies the recorded pattern and launch shape without tuning, and the key
separates what the choice depends on."""
import json

from paper_0707_1581_gb300 import flb, tuning


class Cfg:
    def __init__(self, nx, ny, nz, store=1, pattern=1, lattice=0):
        self.nx, self.ny, self.nz, self.store, self.pattern, self.lattice = nx, ny, nz, store, pattern, lattice


class FakeContext:
    """Stands in for flb.Context: records the calls the cache makes."""

    def __init__(self, cfgs, tuned=(2, 64, 2), tuned_pattern="ab"):
        self.cfgs = cfgs
        self.calls = []
        self._launch = (4, 128, 1)
        self._pattern = "aa"
        self._tuned, self._tuned_pattern = tuned, tuned_pattern

    def flb_autotune(self, trials, pattern=False):
        self.calls.append(("autotune", trials, pattern))
        self._launch = self._tuned
        if pattern:
            self._pattern = self._tuned_pattern

    def flb_get_launch(self):
        return self._launch

    def flb_set_launch(self, V, bx, by):
        self.calls.append(("set_launch", V, bx, by))
        self._launch = (V, bx, by)

    def flb_get_pattern(self):
        return self._pattern

    def flb_set_pattern(self, p):
        self.calls.append(("set_pattern", p))
        self._pattern = p


def test_miss_tunes_and_hit_applies(tmp_path, monkeypatch):
    monkeypatch.setattr(flb, "flb_version", lambda: "flb test")
    path = str(tmp_path / "tune.json")
    a = FakeContext([Cfg(64, 64, 64), Cfg(32, 32, 32)])
    r = tuning.autotune_cached(a, path, trials=3, pattern=True, device="GPU X")
    assert r == {"launch": [2, 64, 2], "pattern": "ab", "cached": False}
    assert a.calls == [("autotune", 3, True)]
    b = FakeContext([Cfg(64, 64, 64), Cfg(32, 32, 32)])
    r = tuning.autotune_cached(b, path, pattern=True, device="GPU X")
    assert r["cached"] and b.calls == [("set_pattern", "ab"), ("set_launch", 2, 64, 2)]
    assert b.flb_get_launch() == (2, 64, 2)
    assert len(json.load(open(path))) == 1


def test_key_separates_boxes_formats_devices_and_pattern_tuning(monkeypatch):
    monkeypatch.setattr(flb, "flb_version", lambda: "flb test")
    base = FakeContext([Cfg(64, 64, 64)])
    keys = {tuning.tuning_key(base, False, "A"),
            tuning.tuning_key(base, True, "A"),
            tuning.tuning_key(base, False, "B"),
            tuning.tuning_key(FakeContext([Cfg(64, 64, 32)]), False, "A"),
            tuning.tuning_key(FakeContext([Cfg(64, 64, 64, store=2)]), False, "A"),
            tuning.tuning_key(FakeContext([Cfg(64, 64, 1, lattice=1)]), False, "A")}
    assert len(keys) == 6
