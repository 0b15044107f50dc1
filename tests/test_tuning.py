"""The autotuning cache (host logic, no GPU): a fake library stands in for
oasm_autotune / oasm_get_tuning / oasm_set_tuning."""
import ctypes
import json

import pytest

from paper_1712_03560_gb300 import binding as B
from paper_1712_03560_gb300 import tuning


class FakeLib:
    def __init__(self, classes):
        self.classes = classes
        self.settings = [dict(words=w, algo=a, groups_per_warp=1, warps=8, chunk=1024,
                              region_scale=1.0) for w, a in classes]
        self.autotunes = 0
        self.sets = 0

    def oasm_autotune(self, ctx, sample):
        self.autotunes += 1
        for s in self.settings:
            s.update(warps=16, chunk=2048, region_scale=0.5)
        return "{}"

    def oasm_get_tuning(self, ctx):
        return [dict(s) for s in self.settings]

    def oasm_set_tuning(self, ctx, entries):
        if [(e["words"], e["algo"]) for e in entries] != self.classes:
            raise B.OasmError(B.OASM_EINVAL, "class mismatch")
        self.sets += 1
        self.settings = [dict(e) for e in entries]


def test_tuning_struct_size_matches_header():
    assert ctypes.sizeof(B.oasm_tuning) == 24


def test_cache_tunes_once_then_reuses(tmp_path):
    path = str(tmp_path / "tune.json")
    pats, ks = [b"ACGTACGT", b"ACGTACGTAC", b"GATTACA"], [0, 1, 2]
    key = tuning.cache_key("GB300", pats, ks)
    a = FakeLib([(1, 1), (1, 2)])
    assert tuning.autotune_cached(a, None, None, key, path) == "tuned"
    assert a.autotunes == 1 and key in json.load(open(path))
    b = FakeLib([(1, 1), (1, 2)])
    assert tuning.autotune_cached(b, None, None, key, path) == "cached"
    assert b.autotunes == 0 and b.sets == 1
    assert b.settings == a.settings


def test_stale_entry_is_tuned_again(tmp_path):
    path = str(tmp_path / "tune.json")
    key = tuning.cache_key("GB300", [b"AAAA"], [1])
    tuning.autotune_cached(FakeLib([(1, 0)]), None, None, key, path)
    other = FakeLib([(2, 0)])  # same key, other classes: the entry does not fit
    assert tuning.autotune_cached(other, None, None, key, path) == "tuned"
    assert other.autotunes == 1
    assert json.load(open(path))[key][0]["words"] == 2


def test_key_follows_gpu_histogram_costs_and_config():
    pats, ks = [b"ACGTACGT", b"ACGTACGTAC"], [0, 1]
    k0 = tuning.cache_key("GB300", pats, ks)
    assert k0 == tuning.cache_key("GB300", [b"TTTTTTTT", b"GGGGGGGGGG"], ks)  # same lengths
    assert k0 != tuning.cache_key("B200", pats, ks)
    assert k0 != tuning.cache_key("GB300", pats, [1, 1])
    assert k0 != tuning.cache_key("GB300", pats + [b"AC"], ks + [0])
    assert k0 != tuning.cache_key("GB300", pats, ks, costs=(1, 2, 2))
    assert k0 != tuning.cache_key("GB300", pats, ks, cfg={"prefilter_piece": 1})


def test_no_path_only_tunes():
    lib = FakeLib([(1, 0)])
    assert tuning.autotune_cached(lib, None, None, "k", None) == "tuned"
    assert lib.autotunes == 1
