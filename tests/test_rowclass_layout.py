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
  - the thread remap of case 0 is a bijection, and each warp sees one class and offset.
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
                for pt in range(256):
                    w, lane = pt >> 5, pt & 31
                    for j in range(4):           # lines j and j + 4 share class and offset
                        kl = 8 * w + j
                        c = (L0 + kl) & 3
                        d = (xw + (L0 + 8 * w) * I + col * BM + j * I) & 3
                        assert c == (L0 + kl + 4) & 3 and d == (xw + (L0 + kl + 4) * I + col * BM) & 3
                        for jj, t in ((j, kl >> 2), (j + 4, (kl >> 2) + 1)):
                            line = boxes[c][t]
                            v = _words(line[4 * lane:4 * lane + 4], line[4 * lane + 4:4 * lane + 8], d)
                            for q in range(4):
                                m = col * BM + 4 * lane + q
                                ok = k0 + 8 * w + jj < K and m < I
                                if ok:
                                    assert v[q] == X[(o * K + k0 + 8 * w + jj) * I + m]
                                else:
                                    assert not full


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
