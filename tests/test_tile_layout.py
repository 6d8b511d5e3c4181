"""The lane layout of the block tiles (phic_tile_layout, a host query: runs without a GPU).

A row of a tile is handled by L lanes of cw columns in a power-of-two group of Lp2 lanes (the row sums
are reduced by shuffles inside the group), and an idle lane of a group costs its warp's instructions all
the same.  With odd widths allowed (the single-instance series tile), a tile whose width divides by 3 or 5
takes that many columns a lane exactly when it needs fewer lane slots, Lp2 cw, than the power-of-two
widths: for the 1024^2 series (p = 4, r = 4, 20 columns) 4 lanes of 5 instead of 8 lanes for 5 live ones.
The expected layouts below are worked out from that rule by counting slots."""
import ctypes

import pytest

from paper_2509_26475_gb300 import capi

F64, F32 = 0, 1
MAX_WIDTH = 128


def layout(w, prec, odd):
    out = (ctypes.c_int32 * 5)()
    assert capi.load(build_if_missing=True).phic_tile_layout(w, prec, odd, out) == 0
    return dict(zip(("w", "ws", "cw", "L", "Lp2"), list(out)))


def slots(t):
    return t["Lp2"] * t["cw"]


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("odd", [0, 1])
def test_every_width_is_covered_by_whole_lanes(prec, odd):
    for w in range(1, MAX_WIDTH + 1):
        t = layout(w, prec, odd)
        assert t["w"] == w
        assert t["ws"] == t["L"] * t["cw"] and t["ws"] >= w, (w, t)
        assert t["Lp2"] & (t["Lp2"] - 1) == 0 and t["L"] <= t["Lp2"] < 2 * t["L"] and t["Lp2"] <= 32, (w, t)
        if t["cw"] in (3, 5):  # odd chunks: only when allowed, only for exact multiples, no padding column
            assert odd and w > 4 and w % t["cw"] == 0 and t["ws"] == w, (w, t)
        else:  # vector chunks start on their own size: the row stride is a multiple of the chunk
            assert t["cw"] in ((1, 2, 4) if prec == F64 else (1, 2, 4, 8)), (w, t)
            assert t["ws"] % t["cw"] == 0, (w, t)


@pytest.mark.parametrize("prec", [F64, F32])
def test_odd_widths_are_taken_only_when_they_save_lane_slots(prec):
    for w in range(1, MAX_WIDTH + 1):
        a, b = layout(w, prec, 0), layout(w, prec, 1)
        assert slots(b) <= slots(a), (w, a, b)
        if b["cw"] != a["cw"]:
            assert b["cw"] in (3, 5) and slots(b) < slots(a), (w, a, b)
        else:
            assert a == b, (w, a, b)


@pytest.mark.parametrize("w,prec,expect", [
    (20, F64, (5, 4, 4)),   # the 1024^2 series: 20 slots against 8 lanes of 4 (32)
    (20, F32, (5, 4, 4)),
    (12, F64, (3, 4, 4)),   # 12 against 4 lanes of 4 for 3 live ones (16)
    (10, F64, (5, 2, 2)),   # 10 against 8 lanes of 2 for 5 live ones (16)
    (24, F64, (3, 8, 8)),   # 24 against 8 lanes of 4 for 6 live ones (32)
    (35, F64, (5, 7, 8)),   # 40 against 16 lanes of 4 for 9 live ones (64; padded to 36)
    (5, F64, (5, 1, 1)),    # 5 against 4 lanes of 2 for 3 live ones (8; padded to 6)
    (15, F64, (4, 4, 4)),   # padded to 16: 16 slots beat 3 lanes of 5 (20) and 5 lanes of 3 (24)
    (8, F64, (4, 2, 2)),    # the 1024^2 recovery tile (2r = 8): nothing to gain
    (8, F32, (8, 1, 1)),
    (3, F64, (2, 2, 2)),    # narrow tiles (up to 4 columns) keep the power-of-two widths
])
def test_known_layouts(w, prec, expect):
    t = layout(w, prec, 1)
    assert (t["cw"], t["L"], t["Lp2"]) == expect, t


def test_power_of_two_layout_of_the_default_series_tile():
    t = layout(20, F64, 0)
    assert (t["cw"], t["L"], t["Lp2"]) == (4, 5, 8)


def test_invalid_arguments():
    lib = capi.load(build_if_missing=True)
    out = (ctypes.c_int32 * 5)()
    for w, prec in [(0, F64), (MAX_WIDTH + 1, F64), (8, 2), (-1, F32)]:
        assert lib.phic_tile_layout(w, prec, 0, out) == capi.PHIC_INVALID_ARG
    assert lib.phic_tile_layout(8, F64, 0, None) == capi.PHIC_INVALID_ARG
