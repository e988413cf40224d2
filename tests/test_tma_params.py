"""Every TMA-fed column kernel instantiated in csrc/inst_*.cu (CPU only).

A tiled bulk tensor copy must start at an x coordinate whose byte offset is a
multiple of 16; a misaligned x is an illegal instruction on the GPU, and nothing
checks it before the copy runs.  The column kernels start tile t at float
x = 2 * t * W (rows) or, for the odd rows of the row-pair view, at
2 * (S + t * W - 1) with S odd: both are 16-byte aligned exactly when the tile
width W is even.  The same instantiations must also split their tile rows into
a few equal boxes of at most 256 rows, keep at least two ring slots (one in flight while
one is consumed), fit their ring and exchange buffer in 227 KB of shared
memory, and launch at most 1024 threads.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1406_5597_gb300", "csrc")
SMEM_MAX = 227 * 1024


def _instantiations():
    out = []
    for f in sorted(glob.glob(os.path.join(CSRC, "inst_*.cu"))):
        text = open(f).read()
        for m in re.finditer(r"FFT3D_TMA\(\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", text):
            L, E, W, ST, PF, PE, PST, PPF = map(int, m.groups())
            out.append((os.path.basename(f), L, E, W, ST, False))
            out.append((os.path.basename(f), L, PE, W, PST, True))
        for m in re.finditer(r"FFT3D_TMA_NOPAIR\(\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", text):
            L, E, W, ST, PF = map(int, m.groups())
            out.append((os.path.basename(f), L, E, W, ST, False))
    return out


def _xbuf(L, W, ST, pair):
    # the kernel's rule for a dedicated exchange buffer (col_tma_xbuf)
    ring = ST * L * ((W + 2) if pair else W) * 8 + 64
    return ring > 113 * 1024 and ring + L * W * 8 <= SMEM_MAX


def test_tma_instantiations_are_found():
    inst = _instantiations()
    assert len(inst) >= 8
    assert {i[1] for i in inst} >= {256, 512, 1024, 2048}


def test_tma_tiles_start_16_byte_aligned():
    for f, L, E, W, ST, pair in _instantiations():
        assert W % 2 == 0, (f, L, W, pair)
        # bytes of the box's inner extent: 2 W floats (rows) or 2 (W + 2) floats (row pairs)
        assert (8 * (W + 2 if pair else W)) % 16 == 0, (f, L, W, pair)
        for t in range(5):  # first tiles, and for row pairs an odd stride S
            assert (4 * 2 * t * W) % 16 == 0
            if pair:
                for S in (257, 513, 1025):
                    assert (4 * 2 * (S + t * W - 1)) % 16 == 0, (f, L, W, S, t)


def test_tma_boxes_ring_smem_and_threads():
    for f, L, E, W, ST, pair in _instantiations():
        rows = L // 2 if pair else L
        if pair:
            assert L % 2 == 0, (f, L)
        # the kernel's box: the largest divisor of the tile rows that is at most 256
        box = max(b for b in range(1, min(rows, 256) + 1) if rows % b == 0)
        assert rows % box == 0 and box <= 256, (f, L, pair, "tile rows must split into boxes of <= 256 rows")
        assert rows // box <= 8 and (box == rows or box >= 64), (f, L, pair, box, "a few large boxes per tile")
        assert ST >= 2, (f, L, ST)
        ws = W + 2 if pair else W
        smem = ST * L * ws * 8 + (L * W * 8 if _xbuf(L, W, ST, pair) else 0) + 8 * ST
        assert smem <= SMEM_MAX, (f, L, W, ST, pair, smem)
        assert L % E == 0 and (L // E) * W <= 1024, (f, L, E, W)
