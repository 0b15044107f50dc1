"""CPU-side checks of the C ABI: the CUDA library builds for sm_103a, loads,
exports every function ``include/oasm.h`` declares, and rejects bad input on
the host without touching a GPU."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_1712_03560_gb300 import binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "oasm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(oasm_[a-z_]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for must in ("oasm_create", "oasm_feed", "oasm_flush", "oasm_open_stream",
                 "oasm_close_stream", "oasm_destroy", "oasm_strerror", "oasm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == sorted(declared_functions())


def test_struct_sizes_match_header():
    assert ctypes.sizeof(B.oasm_hit) == 32
    assert ctypes.sizeof(B.oasm_rules) == 20
    # oasm_config: 4+4+8+4+4+4+4+8+4+4+4+4+4, padded to 8
    assert ctypes.sizeof(B.oasm_config) == 64
    assert ctypes.sizeof(B.oasm_costs) == 12


@pytest.mark.parametrize("lens,ks", [([0], [0]), ([129], [1]), ([8], [8]), ([20], [16]), ([], [])])
def test_create_rejects_bad_patterns(lens, ks):
    pats = [b"A" * max(n, 1) for n in lens]
    lib = B.load()
    n = len(lens)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[ctypes.cast(ctypes.c_char_p(p), ctypes.c_void_p) for p in pats])
    L = (ctypes.c_uint32 * max(n, 1))(*lens)
    K = (ctypes.c_uint32 * max(n, 1))(*ks)
    ctx = ctypes.c_void_p()
    rc = lib.oasm_create(ptrs, L, K, n, None, None, ctypes.byref(ctx))
    assert rc == B.OASM_EINVAL
    assert not ctx.value
    assert lib.oasm_last_error(None)


def test_strerror_and_null_safety():
    lib = B.load()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.oasm_strerror(code)
    assert lib.oasm_destroy(None) == 0
    assert lib.oasm_step(None) == B.OASM_EINVAL
    assert lib.oasm_open_stream(None, None) == B.OASM_EINVAL
    cfg = B.oasm_config()
    assert lib.oasm_config_default(ctypes.byref(cfg)) == 0
    assert cfg.max_streams == 64 and cfg.flush_timeout_ms > 0


@pytest.mark.parametrize("field,value", [("groups_per_warp", 3), ("prefilter_piece", 2),
                                         ("prefilter_piece", 129), ("tile_warps", 17),
                                         ("full_words", 2), ("full_words", -1),
                                         ("record_order", 3), ("record_order", -1)])
def test_create_rejects_bad_config(field, value):
    """Config fields out of range are rejected on the host, before any device work."""
    lib = B.load()
    pats = [b"ACGTACGTACGT"]
    ptrs = (ctypes.c_void_p * 1)(ctypes.cast(ctypes.c_char_p(pats[0]), ctypes.c_void_p))
    L = (ctypes.c_uint32 * 1)(12)
    K = (ctypes.c_uint32 * 1)(1)
    cfg = B.oasm_config_make(**{field: value})
    ctx = ctypes.c_void_p()
    rc = lib.oasm_create(ptrs, L, K, 1, None, ctypes.byref(cfg), ctypes.byref(ctx))
    assert rc == B.OASM_EINVAL
    assert not ctx.value
    assert b"config" in lib.oasm_last_error(None)


@pytest.mark.parametrize("costs", [(0, 1, 1), (1, 0, 1), (1, 1, 0), (256, 1, 1), (1, 1, 300)])
def test_create_weighted_rejects_bad_costs(costs):
    """Edit costs outside 1..255 are rejected on the host, before any device work."""
    lib = B.load()
    pats = [b"ACGTACGTACGT"]
    ptrs = (ctypes.c_void_p * 1)(ctypes.cast(ctypes.c_char_p(pats[0]), ctypes.c_void_p))
    L = (ctypes.c_uint32 * 1)(12)
    K = (ctypes.c_uint32 * 1)(1)
    w = B.oasm_costs(*costs)
    ctx = ctypes.c_void_p()
    rc = lib.oasm_create_weighted(ptrs, L, K, 1, None, ctypes.byref(w), None, ctypes.byref(ctx))
    assert rc == B.OASM_EINVAL
    assert not ctx.value
    assert b"cost" in lib.oasm_last_error(None)


def test_config_maker_rejects_unknown_fields():
    with pytest.raises(KeyError):
        B.oasm_config_make(prefilter=4)


def test_piece_filter_choice_follows_its_rule():
    """The host-only routing query (no device): fixed piece lengths, and the
    automatic rule on a skewed byte set versus a 4-letter alphabet."""
    rng = np.random.default_rng(3)
    pats = [bytes(rng.integers(65, 69, size=m).astype(np.uint8)) for m in (8, 12, 16, 24, 32)]
    ks = [1, 2, 3, 1, 0]
    got = B.oasm_piece_filter_choice(pats, ks, 4)
    assert got.tolist() == [len(p) // (k + 1) >= 4 for p, k in zip(pats, ks)]
    assert not B.oasm_piece_filter_choice(pats, ks, 0).any()
    # automatic: a 4-letter alphabet makes 4-symbol pieces match often; the
    # same lengths over many distinct bytes make them rare
    dna = [bytes(rng.integers(65, 69, size=20).astype(np.uint8)) for _ in range(50)]
    wide = [bytes(rng.integers(0, 256, size=20).astype(np.uint8)) for _ in range(50)]
    assert not B.oasm_piece_filter_choice(dna, [3] * 50, 1).any()      # pieces of 5 over 4 letters
    assert B.oasm_piece_filter_choice(wide, [3] * 50, 1).all()         # pieces of 5 over 256 bytes
    assert B.oasm_piece_filter_choice(dna, [0] * 50, 1).all()          # one piece of 20
    with pytest.raises(B.OasmError):
        B.oasm_piece_filter_choice(pats, ks, 3)


def test_tuning_and_selftest_reject_bad_arguments_on_the_host():
    """No context or no count: rejected before any device work."""
    lib = B.load()
    n = ctypes.c_uint32(0)
    assert lib.oasm_get_tuning(None, None, 0, ctypes.byref(n)) == B.OASM_EINVAL
    assert lib.oasm_set_tuning(None, None, 0) == B.OASM_EINVAL
    assert lib.oasm_selftest_wait(0, 0, 0) == B.OASM_EINVAL
