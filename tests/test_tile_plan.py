"""Tile plan of the fused per-context kernel: host logic only, checked on the
CPU through tf_plan_tiles (the same planning functions and column cut the
kernel launches use).

The plan must cover every site exactly once with tiles inside the geometry
the kernel was compiled for (at most 32 x 32 sites narrow, 40 x 30 wide),
start every column tile on a 16-byte boundary whenever the rows allow bulk
copies (nx a multiple of 4), and keep a grid that fits one wave of resident
CTAs within that wave.
"""
import ctypes

import pytest

from paper_2511_00445_gb300 import _binding as B
from paper_2511_00445_gb300 import build as Bld

SLOTS = 304          # 152 SMs x 2 CTAs (the narrow kernel's occupancy on GB300)
CAP = 1100


@pytest.fixture(scope="module")
def lib():
    Bld.build()
    return B.load_library()


def plan(lib, nx, ny, batch, slots=SLOTS):
    out = (ctypes.c_int * 3)()
    cs = (ctypes.c_int * CAP)()
    assert lib.tf_plan_tiles(nx, ny, batch, slots, out, cs, CAP) == B.TF_OK
    return bool(out[0]), out[1], out[2], list(cs[:out[1] + 1])


def cdiv(a, b):
    return -(-a // b)


GRIDS = [(256, 256, 4), (256, 256, 1), (64, 64, 1), (64, 48, 1), (1024, 1024, 1), (2048, 2048, 1),
         (1040, 1000, 1), (1030, 1000, 1), (33, 17, 1), (40, 36, 2), (8, 8, 1), (5, 3, 2),
         (2, 7, 1), (1, 1, 1), (128, 128, 16), (512, 512, 16), (4096, 16, 1), (16, 4096, 1),
         (32768, 32, 1), (100, 100, 30), (1000, 1000, 3)]


@pytest.mark.parametrize("nx,ny,batch", GRIDS)
def test_plan_covers_the_grid_within_the_geometry(lib, nx, ny, batch):
    wide, cols, rows, cs = plan(lib, nx, ny, batch)
    txm, tym = (40, 30) if wide else (32, 32)
    # geometry choice: wide exactly when the narrow 32 x 32 tiles exceed one wave
    assert wide == (cdiv(nx, 32) * cdiv(ny, 32) * batch > SLOTS)
    # columns: a partition of [0, nx) into cols tiles of 1 .. txm columns
    assert cols == cdiv(nx, txm)
    assert cs[0] == 0 and cs[-1] == nx
    widths = [b - a for a, b in zip(cs, cs[1:])]
    assert all(1 <= w <= txm for w in widths), widths
    if nx % 4 == 0:
        assert all(c % 4 == 0 for c in cs), cs
    # rows: tile row r = [r ny / rows, (r + 1) ny / rows), every one non-empty
    assert 1 <= rows <= ny
    heights = [(r + 1) * ny // rows - r * ny // rows for r in range(rows)]
    assert sum(heights) == ny and min(heights) >= 1 and max(heights) <= tym
    need = cdiv(ny, tym)
    if cols * need * batch <= SLOTS:
        # one wave: rows cut finer to fill it, never below 8-row tiles
        assert cols * rows * batch <= SLOTS
        assert rows <= max(ny // 8, need)
    else:
        assert rows == need


def test_benchmarked_plans(lib):
    # 4 x 256^2 sweep: narrow, 8 x 9 tiles of 32 x 28-29 per instance (288 CTAs)
    assert plan(lib, 256, 256, 4)[:3] == (False, 8, 9)
    # one 256^2 instance: 32 rows of 8-row tiles (256 CTAs)
    assert plan(lib, 256, 256, 1)[:3] == (False, 8, 32)
    # 1024^2 and 2048^2: wide 40 x 30 tiles over several waves
    assert plan(lib, 1024, 1024, 1)[:3] == (True, 26, 35)
    assert plan(lib, 2048, 2048, 1)[:3] == (True, 52, 69)


def test_plan_argument_errors(lib):
    out = (ctypes.c_int * 3)()
    cs = (ctypes.c_int * 4)()
    for args in ((0, 8, 1, SLOTS), (8, 0, 1, SLOTS), (8, 8, 0, SLOTS), (8, 8, 1, 0),
                 (40000, 8, 1, SLOTS)):
        assert lib.tf_plan_tiles(*args, out, None, 0) == B.TF_ERR_ARG
    # too small a column array: 256 columns narrow need 9 entries
    assert lib.tf_plan_tiles(256, 256, 1, SLOTS, out, cs, 4) == B.TF_ERR_ARG
    assert lib.tf_plan_tiles(256, 256, 1, SLOTS, out, None, 0) == B.TF_OK


def _segments(xs, length, nx):
    """Row segments of a periodic copy of `length` elements from column xs,
    split at the wrap (the kernel's bulk-copy and prefetch row walk)."""
    out, off = [], 0
    while off < length:
        gx = (xs + off) % nx
        n = min(length - off, nx - gx)
        out.append((gx, n))
        off += n
    return out


@pytest.mark.parametrize("nx,ny,batch", GRIDS)
def test_bulk_copy_and_prefetch_segments_are_16_byte_units(lib, nx, ny, batch):
    """The tile loads and the L2 population prefetch move whole 16-byte
    units from 16-byte boundaries (a bulk copy from anywhere else faults).
    Restated host arithmetic of the kernel: a tile row of phi, Q or u is
    loaded from x0 - RH over tw + 2 RH columns (RH = 12 with pending
    sub-steps, 4 without) when nx is a multiple of 4; populations are
    prefetched over x0 - 1 .. x0 + tw widened to whole units of PF elements
    (4 FP32 or 8 16-bit values) when nx is a multiple of PF."""
    wide, cols, rows, cs = plan(lib, nx, ny, batch)
    for k in range(cols):
        x0, tw = cs[k], cs[k + 1] - cs[k]
        if nx % 4 == 0:
            for rh in (12, 4):
                for gx, n in _segments(x0 - rh, tw + 2 * rh, nx):
                    assert gx % 4 == 0 and n % 4 == 0, (x0, tw, rh, gx, n)
        for pf in (4, 8):
            if nx % pf:
                continue
            xs = ((x0 - 1 + pf) // pf - 1) * pf
            xe = (x0 + tw + 1 + pf - 1) // pf * pf
            assert xs <= x0 - 1 and xe >= x0 + tw + 1
            for gx, n in _segments(xs, xe - xs, nx):
                assert gx % pf == 0 and n % pf == 0, (x0, tw, pf, gx, n)
