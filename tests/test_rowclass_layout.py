"""Row-class tile layout of the tensor-core MTTKRP (rows not 16-byte aligned), on the CPU.

A model of the addressing in `csrc/mttkrp_tc.cu` (rowcls_load, conv_read_rowcls,
conv_read_rowcls_mn, rowcls_thread) and `csrc/plan.cpp` (encode_x_rowclass_maps): X
lives in a word array at every offset mod 4; the four class boxes of a chunk are filled
as a tiled tensor-map load would fill them (zero outside each map's extent); the
converter threads read them back.  Checked for each chunk of small geometries (wide and
narrow tiles, ragged tails, several outer indices, both cases):
  - every word a box reads lies in a 16-byte granule that holds an element of X;
  - every box starts on a 16-byte multiple along the row (a tiled load's x rule);
  - each converter thread gets the values of X at its (row, k) and zero outside the tile;
  - the thread remap of case 0 is a bijection, and each warp sees one class and offset
    (in case 1 too: a warp holds the k lines of one residue mod 4);
  - the case-1 store of that layout covers the MN-major tile once.
The GPU parity tests run the kernels themselves on these layouts.
"""
import numpy as np
import pytest

BM, BK = 128, 64
P0, R0 = BK + 4, BM // 4      # case 0 box: 32 rows of 68 words
P1, R1 = BM + 4, BK // 4      # case 1 box: 16 lines of 132 words


def _words(a, b, d):
    return np.concatenate([a, b])[d:d + 4]


def _rowcls_thread(pt):
    w, h = pt >> 5, (pt >> 4) & 1
    return ((((w & 3) + 8 * (w >> 2) + 4 * h) << 4) | (pt & 15))


def _maps(xw, length, n):
    out = []
    for c in range(4):
        start = xw + c * length
        dc = start & 3
        out.append((start - dc, length + dc, (n - c + 3) // 4, dc))
    return out


def _fill(mem, maps, c, x0, y, rows, pitch, stride, lo, hi):
    base, ext, nc, _ = maps[c]
    box = np.zeros((rows, pitch))
    for t in range(rows):
        for e in range(pitch):
            xx, yy = x0 + e, y + t
            if xx < ext and yy < nc:
                addr = base + yy * stride + xx
                assert lo <= addr < hi, "a box read outside the granules of X"
                box[t, e] = mem[addr]
    return box


def _x_in_memory(total, xoff, seed):
    pad = 8
    mem = np.full(total + 2 * pad, np.nan)
    xw = pad + xoff
    X = np.random.default_rng(seed).standard_normal(total)
    mem[xw:xw + total] = X
    return mem, xw, X, (xw // 4) * 4, ((xw + total + 3) // 4) * 4


def _case0(P, I, O, K, xoff, gmax=16):
    Q = O * K
    n = P * I
    mem, xw, X, lo, hi = _x_in_memory(n * Q, xoff, P * 1000 + I * 10 + xoff)
    narrow = I < BM
    G = max(1, min(BM // I, gmax, P)) if narrow else 1
    n_cols = 1 if narrow else (I + BM - 1) // BM
    tiles = (P + G - 1) // G if narrow else P
    maps = _maps(xw, Q, n)

    def row_valid(col, rowbase, l):
        return (l < G * I and rowbase + l < n) if narrow else col * BM + l < I

    for col in range(n_cols):
        for t in range(tiles):
            rowbase = t * G * I if narrow else t * I + col * BM
            for o in range(O):
                for kb in range((K + BK - 1) // BK):
                    k0 = kb * BK
                    boxes = []
                    for c in range(4):
                        rc = rowbase + ((c - rowbase) & 3)
                        x = maps[c][3] + o * K + k0
                        assert (x & ~3) % 4 == 0 and rc >= c
                        boxes.append(_fill(mem, maps, c, x & ~3, (rc - c) >> 2, R0, P0, 4 * Q, lo, hi))
                    full = ((G * I == BM and rowbase + BM <= n) if narrow else col * BM + BM <= I) \
                        and k0 + BK <= K
                    seen = {}
                    for pt0 in range(256):
                        pt = _rowcls_thread(pt0)
                        k4, rsub = pt & 15, pt >> 4
                        d = (xw + (rowbase + rsub) * Q + o * K + k0) & 3
                        c = (rowbase + rsub) & 3
                        seen.setdefault(pt0 >> 5, set()).add((c, d))
                        for j in range(8):
                            row = boxes[c][(rsub >> 2) + 4 * j]
                            v = _words(row[4 * k4:4 * k4 + 4], row[4 * k4 + 4:4 * k4 + 8], d)
                            l = rsub + 16 * j
                            for q in range(4):
                                kk = k0 + 4 * k4 + q
                                ok = row_valid(col, rowbase, l) and kk < K
                                if ok:
                                    assert v[q] == X[(rowbase + l) * Q + o * K + kk]
                                else:
                                    assert not full
                    assert all(len(s) == 1 for s in seen.values()), "offset not warp-uniform"


def _case1(O, K, I, xoff):
    n = O * K
    mem, xw, X, lo, hi = _x_in_memory(n * I, xoff, O * 1000 + I * 10 + xoff)
    maps = _maps(xw, I, n)
    for col in range((I + BM - 1) // BM):
        for o in range(O):
            for kb in range((K + BK - 1) // BK):
                k0 = kb * BK
                L0 = o * K + k0
                boxes = []
                for c in range(4):
                    lc = L0 + ((c - L0) & 3)
                    boxes.append(_fill(mem, maps, c, col * BM, (lc - c) >> 2, R1, P1, 4 * I, lo, hi))
                full = k0 + BK <= K and col * BM + BM <= I
                seen = {}
                for pt in range(256):
                    w, lane = pt >> 5, pt & 31
                    r, h = w & 3, w >> 2
                    c = (L0 + r) & 3                                   # one class per warp
                    d = (xw + (L0 + r) * I + col * BM) & 3             # and one offset
                    seen.setdefault(w, set()).add((c, d))
                    for j in range(8):
                        kl = r + 4 * (8 * h + j)
                        assert (L0 + kl) & 3 == c and (xw + (L0 + kl) * I + col * BM) & 3 == d
                        line = boxes[c][8 * h + j]
                        v = _words(line[4 * lane:4 * lane + 4], line[4 * lane + 4:4 * lane + 8], d)
                        for q in range(4):
                            m = col * BM + 4 * lane + q
                            ok = k0 + kl < K and m < I
                            if ok:
                                assert v[q] == X[(o * K + k0 + kl) * I + m]
                            else:
                                assert not full
                assert all(len(s) == 1 for s in seen.values()), "offset not warp-uniform"


def _sw128_mn_offset(m, k):
    """Byte offset of element (m, k) of the MN-major 128-byte-swizzled tile (sm100.cuh)."""
    return ((k >> 3) * 2 + (m >> 6)) * 1024 + (k & 7) * 128 + (((((m & 63) >> 3) ^ (k & 7)) & 7) << 4) + (m & 7) * 2


def test_case1_class_store_covers_the_tile_once():
    """conv_store_mn_cls: thread (warp w, lane) writes rows 4 lane .. + 3 of k line
    kl = w % 4 + 4 (8 (w / 4) + j) at the tile's MN-major offset; every (m, k) once, and
    each 16-lane half of a store fills one 128-byte k-row of one atom."""
    seen = set()
    for j in range(8):
        for w in range(8):
            r, h = w & 3, w >> 2
            rows = {}
            for lane in range(32):
                cl = (lane & 15) >> 1
                kl = r + 4 * (8 * h + j)
                kr = r + 4 * (j & 1)
                off = (lane >> 4) * 1024 + (lane & 1) * 8 + h * 8192 + (j >> 1) * 2048 + kr * 128 + ((cl ^ kr) << 4)
                assert off == _sw128_mn_offset(4 * lane, kl)
                for q in range(4):
                    assert _sw128_mn_offset(4 * lane + q, kl) == off + 2 * q
                    seen.add((4 * lane + q, kl))
                rows.setdefault(lane >> 4, set()).add(off // 128)
            assert all(len(v) == 1 for v in rows.values())
    assert len(seen) == BM * BK


def test_case0_thread_remap_is_a_bijection():
    assert sorted(_rowcls_thread(p) for p in range(256)) == list(range(256))


@pytest.mark.parametrize("P,I,O,K", [(1, 131, 1, 70), (3, 45, 2, 67), (7, 37, 1, 65), (9, 5, 2, 11),
                                     (2, 130, 1, 130), (1, 4, 3, 5)])
def test_case0_rowclass_boxes(P, I, O, K):
    for xoff in range(4):
        _case0(P, I, O, K, xoff)


@pytest.mark.parametrize("O,K,I", [(2, 45, 131), (1, 70, 77), (3, 5, 129), (1, 4, 3)])
def test_case1_rowclass_boxes(O, K, I):
    for xoff in range(4):
        _case1(O, K, I, xoff)
