"""Row-class tiles of the fused TTMc kernel with short slabs packed SG to a tile, on the CPU.

A model of the addressing in `csrc/ttmc_tc.cu` (rc_load_packed, rc_read_packed, with
rowcls_thread from `csrc/tc_common.cuh`) and of the class maps that `csrc/plan.cpp`
encodes for it (boxes of 32 / SG rows): X is S slabs of K rows of L words (K <= 128 / SG),
placed in a word array at every offset mod 4; each chunk's 4 x SG class boxes are filled
as a tiled tensor-map load fills them (zero outside each map's extent) at their places in
the raw stage; the converter threads read them back.  Checked for every chunk of small
geometries (SG = 2 and 4, ragged slab groups, several l chunks, odd row lengths):
  - every word a box reads lies in a 16-byte granule that holds an element of X;
  - every box starts on a 16-byte multiple along the row, inside the raw stage, and the
    boxes of one stage do not overlap;
  - each converter thread gets X at its (slab, row, l) for rows below K and l below L, and
    elsewhere values of X or zero (finite: they meet zero factor rows).
The GPU parity tests run the kernel itself on these layouts.
"""
import numpy as np
import pytest

BM, BK = 128, 64
PITCH = BK + 4          # words per box row
REGION = BM // 4        # rows of one class's region in the raw stage


def _rowcls_thread(pt):
    w, h = pt >> 5, (pt >> 4) & 1
    return ((((w & 3) + 8 * (w >> 2) + 4 * h) << 4) | (pt & 15))


def _words(row, start, d):
    return row[start:start + 8][d:d + 4]


def _geometry(S, K, L, xoff, seed):
    pad = 8
    n_rows = S * K
    total = n_rows * L
    mem = np.full(total + 2 * pad, np.nan)
    xw = pad + xoff
    X = np.random.default_rng(seed).standard_normal(total)
    mem[xw:xw + total] = X
    lo, hi = (xw // 4) * 4, ((xw + total + 3) // 4) * 4
    maps = []
    for c in range(4):           # the class maps: rows c, c + 4, ... of L words
        start = xw + c * L
        dc = start & 3
        maps.append((start - dc, L + dc, (n_rows - c + 3) // 4, dc))
    return mem, xw, X.reshape(S, K, L), lo, hi, maps


def _load_stage(mem, maps, grp, SG, K, L, kb, lo, hi, xw):
    KP = BM // SG
    rows = KP // 4
    stage = np.full((4 * REGION, PITCH), np.nan)   # NaN: never written by any box
    filled = np.zeros((4 * REGION, PITCH), dtype=int)
    for g in range(SG):
        rowbase = (grp * SG + g) * K
        for c in range(4):
            rc = rowbase + ((c - rowbase) & 3)
            assert (rc - c) % 4 == 0 and rc >= c
            base, ext, nc, dc = maps[c]
            assert dc == (xw + c * L) & 3
            x = dc + kb * BK
            x0 = x & ~3
            assert x0 % 4 == 0                               # a tiled load's x rule
            y = (rc - c) >> 2
            r0 = c * REGION + g * rows                        # the box's first stage row
            assert 0 <= r0 and r0 + rows <= 4 * REGION
            for t in range(rows):
                for e in range(PITCH):
                    xx, yy = x0 + e, y + t
                    v = 0.0
                    if xx < ext and yy < nc:
                        addr = base + yy * 4 * L + xx
                        assert lo <= addr < hi, "a box read outside the granules of X"
                        v = mem[addr]
                    stage[r0 + t, e] = v
                    filled[r0 + t, e] += 1
    assert filled.max() == 1 and filled.min() == 1          # the boxes tile the stage once
    return stage


@pytest.mark.parametrize("S,K,L,SG", [
    (7, 60, 61, 2),     # the paper's short slabs with an odd row length, a partial group
    (5, 64, 66, 2),     # 64-row slabs exactly, two l chunks
    (9, 33, 30, 2),
    (7, 32, 30, 4),     # four 32-row slabs a tile, a partial group
    (6, 20, 150, 4),    # three l chunks
    (5, 3, 9, 4),       # 3-row slabs
])
@pytest.mark.parametrize("xoff", [0, 1, 2, 3])
def test_packed_rowclass_layout(S, K, L, SG, xoff):
    assert K <= BM // SG
    KP, JG = BM // SG, 8 // SG
    mem, xw, X, lo, hi, maps = _geometry(S, K, L, xoff, S * 100 + K * 10 + xoff)
    n_kb = (L + BK - 1) // BK
    groups = (S + SG - 1) // SG
    for grp in range(groups):
        for kb in range(n_kb):
            stage = _load_stage(mem, maps, grp, SG, K, L, kb, lo, hi, xw)
            for pt in range(256):
                t = _rowcls_thread(pt)
                k4, rsub = t & 15, t >> 4
                for g in range(SG):
                    s = grp * SG + g
                    row = s * K + rsub
                    d = (xw + row * L + kb * BK) & 3
                    c = row & 3
                    for jj in range(JG):
                        j = g * JG + jj
                        srow = c * REGION + (rsub >> 2) + 4 * j
                        v = _words(stage[srow], 4 * k4, d)
                        assert len(v) == 4 and np.all(np.isfinite(v)), (grp, kb, pt, j)
                        r = rsub + 16 * j - g * KP                 # the row within slab g
                        assert 0 <= r < KP
                        for e in range(4):
                            k = kb * BK + 4 * k4 + e
                            if s < S and r < K and k < L:
                                assert v[e] == X[s, r, k], (grp, kb, pt, j, e)
