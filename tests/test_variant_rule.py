"""The solver's choice of iteration pass and tile height (host logic, no GPU):
the rule the short-tile measurements set (a small grid spreads over more
blocks on shorter tiles while one tile per SM remains; FP64 takes the
shortest such tiles, FP32 takes 4 rows only while the blocks stay few; the
streaming pass from 448 tiles of 128x16 on), the options that override it,
and argument checks."""
import ctypes

import pytest

from paper_2604_01800_gb300 import _lib

FP64, MIXED = _lib.PPE_PREC_FP64, _lib.PPE_PREC_MIXED


def pick(prec, iter_pass, ntiles, tile_rows=0, sms=152):
    lib = _lib.load(build_if_missing=False)
    p, r = ctypes.c_int(-1), ctypes.c_int(-1)
    st = lib.ppe_debug_pick_variant(prec, iter_pass, ntiles, tile_rows, sms, ctypes.byref(p), ctypes.byref(r))
    return st, p.value, r.value


@pytest.mark.parametrize("prec,ntiles,want", [
    (MIXED, 4, (1, 4)),        # 64^2: 16 blocks of 4 rows
    (MIXED, 32, (1, 8)),       # 256^2: 64 blocks of 8 rows (128 of 4 rows measured slower)
    (MIXED, 76, (1, 8)),       # the largest count that fits twice on 152 SMs
    (MIXED, 77, (1, 16)),
    (MIXED, 128, (1, 16)),     # 512^2
    (MIXED, 447, (1, 16)),
    (MIXED, 448, (2, 16)),     # the streaming pass from 448 tiles on
    (FP64, 4, (1, 4)),
    (FP64, 32, (1, 4)),        # FP64 passes are long: the shortest tiles that fit one per SM
    (FP64, 38, (1, 4)),
    (FP64, 39, (1, 8)),
    (FP64, 77, (1, 16)),
    (FP64, 5000, (1, 16)),     # FP64 has no streaming pass
])
def test_size_rule(prec, ntiles, want):
    st, p, r = pick(prec, 0, ntiles)
    assert st == 0 and (p, r) == want


def test_options_override_the_rule():
    assert pick(MIXED, 2, 4)[1:] == (2, 16)          # streaming asked for
    assert pick(MIXED, 1, 5000)[1:] == (1, 16)       # tile-cooperative asked for, too many tiles to shorten
    assert pick(MIXED, 1, 32, tile_rows=16)[1:] == (1, 16)
    assert pick(MIXED, 0, 128, tile_rows=4)[1:] == (1, 4)
    assert pick(FP64, 2, 4, tile_rows=8)[1:] == (1, 8)   # FP64 ignores the streaming choice


def test_sm_count_scales_the_rule():
    assert pick(MIXED, 0, 32, sms=64)[1:] == (1, 8)
    assert pick(MIXED, 0, 32, sms=63)[1:] == (1, 16)
    assert pick(MIXED, 0, 4, sms=63)[1:] == (1, 8)    # 4 rows need 16 x the tile count <= SMs


@pytest.mark.parametrize("args", [(2, 0, 4, 0, 152), (MIXED, 3, 4, 0, 152), (MIXED, 0, 0, 0, 152),
                                  (MIXED, 0, 4, 12, 152), (MIXED, 0, 4, 0, 0)])
def test_bad_arguments(args):
    lib = _lib.load(build_if_missing=False)
    assert lib.ppe_debug_pick_variant(*args, None, None) == _lib.PPE_ERR_ARG
