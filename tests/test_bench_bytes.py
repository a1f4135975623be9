"""bench.py's accounting: the tile-key plan follows the library's rule for
gs_render, the per-stage algorithmic bytes add up as counted by hand, and the
launches per frame follow from the plan."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("tiles,key_bits,plan", [
    ((120, 68), 45, (2, 2, 1)),     # 1080p: (row << 8 | column), 7 row bits, column pass fused
    ((240, 135), 47, (2, 2, 1)),    # 4K: 8 row bits, 16-bit keys
    ((16, 300), 45, (4, 3, 1)),     # 300 tile rows: 17-bit (row, column) keys
    ((512, 4), 43, (2, 2, 0)),      # wider than 256 tiles: 11-bit tile ids, separate passes
    ((300, 300), 49, (4, 3, 0)),    # 90,000 tiles: 17-bit tile ids
    ((1, 1), 32, (2, 1, 1)),        # one tile: one (column) pass, inside the emission
])
def test_tile_key_plan(tiles, key_bits, plan):
    assert bench.tile_key_plan(*tiles, key_bits) == plan


def test_long_lists_sort_tile_ids_in_separate_passes():
    # From 8M key slots on, the library emits tile ids and sorts them with
    # reduce-then-scan passes, none inside the emission.
    assert bench.tile_key_plan(240, 135, 47, capacity=bench.RTS_MIN_PAIRS) == (2, 2, 0)
    assert bench.tile_key_plan(240, 135, 47, capacity=bench.RTS_MIN_PAIRS - 1) == (2, 2, 1)


def test_frame_bytes_hand_count():
    # 10 Gaussians, 4 visible, 7 keys, SH degree 0 (3 floats), 2x2 tiles, 32x32 pixels.
    fb = bench.frame_bytes(10, 4, 7, 0, 2, 2, 34, 1024)
    assert fb == {
        "project": 10 * 24 + 4 * (20 + 12) + 4 * 108,  # means + log-scales; quats, opacity, SH; 2 records + list
        "depth_sort": 4 * 24 + 4 * 4 * 24,              # gather, then four passes
        "entry_scan": 4 * 12,
        "emit": 4 * 40 + 7 * (2 + 4),                   # entries read; keys + values written once
        "tile_sort": 1 * 7 * 2 * (2 + 4),               # the row pass only (column pass fused)
        "ranges": 7 * 2 + 4 * 8,
        "blend": 7 * 4 + 4 * 48 + 1024 * 20,
    }


def test_unfused_grids_count_every_tile_pass():
    # 512 x 4 tiles: tile-id keys, both passes separate.
    fb = bench.frame_bytes(10, 4, 7, 0, 512, 4, 43, 1024)
    assert fb["tile_sort"] == 2 * 7 * 2 * (2 + 4)


def test_launches_per_frame():
    for tiles, key_bits, launches in [((120, 68), 45, 11), ((512, 4), 43, 12), ((300, 300), 49, 13)]:
        _, passes, fused = bench.tile_key_plan(*tiles, key_bits)
        assert 10 + passes - fused == launches


def test_list_tiles_read_each_entry_once_per_screen_tile():
    # 2x2 list tiles: each list entry is read by the four screen tiles of its list tile.
    one = bench.frame_bytes(10, 4, 7, 0, 2, 2, 34, 1024)
    four = bench.frame_bytes(10, 4, 7, 0, 1, 1, 32, 1024, readers=4)
    assert four["blend"] - one["blend"] == 3 * 7 * 4
    assert [bench.list_tile_dims(c) for c in (0, 1, 2, 4, 16, 64)] == \
        [(1, 1), (1, 1), (2, 1), (2, 2), (4, 4), (8, 8)]
