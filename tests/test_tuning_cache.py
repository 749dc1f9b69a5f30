"""The autotuner's JSON cache (sph.TuningCache / sph.tune): a miss runs the
trials and stores the choice under the GPU name and the problem's signature;
a hit sets the stored options without trials; another signature misses."""
import json

from paper_2603_11868_gb300 import sph


class FakeSolver:
    def __init__(self, n):
        self.n = n
        self.options = {}
        self.trials = 0

    def tuning_signature(self):
        return {"kind": "tank", "dim": 3, "precision": 1, "n": self.n, "nw": 10, "cells": 99}

    def set_option(self, opt, value):
        self.options[opt] = value

    def autotune(self, steps):
        self.trials += 1
        return {"block": 192, "radix_bits": 9, "neighbour_list": 1, "trials": 12}


def test_cache_miss_then_hit(tmp_path):
    path = str(tmp_path / "tune.json")
    a = FakeSolver(1000)
    t = sph.tune(a, 5, cache=path)
    assert a.trials == 1 and t["block"] == 192 and not a.options
    stored = json.load(open(path))
    assert len(stored) == 1
    (key, val), = stored.items()
    assert "n=1000" in key and val == {"block": 192, "radix_bits": 9, "neighbour_list": 1}
    b = FakeSolver(1000)
    t = sph.tune(b, 5, cache=path)
    assert b.trials == 0 and t["cached"] and t["trials"] == 0
    assert b.options == {sph.SPH_OPT_BLOCK: 192, sph.SPH_OPT_RADIX_BITS: 9,
                         sph.SPH_OPT_NEIGHBOUR_LIST: 1}
    c = FakeSolver(2000)
    sph.tune(c, 5, cache=path)
    assert c.trials == 1 and len(json.load(open(path))) == 2


def test_no_cache_always_tunes():
    a = FakeSolver(10)
    sph.tune(a, 5)
    sph.tune(a, 5)
    assert a.trials == 2
