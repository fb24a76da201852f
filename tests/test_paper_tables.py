"""The storage arithmetic of Table 2 (Sec. 8), from the per-pixel costs the text gives: a
shadow map holds one FP32 depth per pixel, the accrual map 60 of them (n = 60 slices), and
the inverse accrual map 48 bytes of mapped points per pixel (3 source levels x 2 directions
x 2 coordinates x 4 bytes) plus its 60 accumulation bits, which the printed figures show
held in one 8-byte word (the same uint64 per cell that this library's maps keep)."""
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
MB = float(1 << 20)


def _table2():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table2_memory.txt"))
            if l.strip() and not l.startswith("#")]
    return [(int(r[0]), *map(float, r[1:])) for r in rows]


def _close(got, printed):
    # the table prints 1-4 significant digits; compare at the printed precision
    digits = len(str(printed).rstrip("0").rstrip(".").replace(".", "").lstrip("0")) or 1
    return got == pytest.approx(printed, rel=0.6 * 10 ** (1 - digits))


def test_table2_follows_the_per_pixel_costs():
    rows = _table2()
    assert [r[0] for r in rows] == [512, 800, 1024, 1600, 2048]
    for side, sm, sam, rt, iam in rows:
        px = side * side
        assert _close(px * 4 / MB, sm) and _close(px * 4 / MB, rt), side
        assert _close(px * 60 * 4 / MB, sam), side
        assert 3 * 2 * 2 * 4 == 48
        assert _close(px * (48 + 8) / MB, iam), side
        # 60 bits taken literally (7.5 bytes) would miss the 800 x 800 figure
    assert not _close(800 * 800 * (48 + 7.5) / MB, 34.2)
