"""Block distribution and redistribution plans (paper Sec. II-C/D, Sec. V), host only.

Pins: Tables I and II of the paper (the running example on P = 8, N_idx = 10);
the per-dimension partitions of Eqs. (20)-(24) and the message matching of
Eq. (25) against the per-element mapping of Eq. (17) (brute force); the send and
receive plans against an element-by-element count (every element of every
y-block received exactly once, from the block's one sending x-replica).
"""
import itertools
import os

import numpy as np
import pytest

import paper_2206_08301_gb300 as dz

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "block_distribution_p8_n10.txt")


def _table():
    rows = []
    with open(GOLDEN) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                v = [int(x) for x in ln.split()]
                rows.append(v)
    return rows


def test_tables_i_and_ii():
    g = dz.Grid([10, 10, 10, 10], [2, 2, 2, 1])        # (i, j, k, a)
    rows = _table()
    assert len(rows) == 8
    for v in rows:
        rank, coords = v[0], tuple(v[1:5])
        assert g.coords(rank) == coords and g.rank(coords) == rank
        lo, hi = g.block_range(rank)
        slices = [(v[5 + 2 * d], v[6 + 2 * d]) for d in range(4)]          # Table I
        assert list(zip(lo, hi)) == slices
        xblock = [(v[13 + 2 * d], v[14 + 2 * d]) for d in range(3)]        # Table II, X[i, j, k]
        assert xblock == slices[:3]
        ablock = [(v[19], v[20]), (v[21], v[22])]                           # Table II, A[j, a]
        assert ablock == [slices[1], slices[3]]


def test_replication_subgrids_of_the_listing():
    # A (j, a) is replicated over the sub-grids keeping i and k (remain = {1, 0, 1, 0}):
    # P_j * P_a = 2 sub-grids of P_i * P_k = 4 ranks, each holding one A-block (Table II)
    g = dz.Grid([10, 10, 10, 10], [2, 2, 2, 1])
    groups = {}
    for r in range(8):
        color, key = g.sub([1, 0, 1, 0], r)
        groups.setdefault(color, []).append((key, r))
    assert sorted(groups) == [0, 1]
    for color, members in groups.items():
        assert sorted(k for k, _ in members) == [0, 1, 2, 3]
        blocks = {tuple(np.array(g.block_range(r)).T[[1, 3]].ravel()) for _, r in members}
        assert len(blocks) == 1                       # one A-block per sub-grid
    # t1 (i, a) partial sums are reduced over the sub-grids keeping j and k: 2 groups of 4
    t1 = {}
    for r in range(8):
        t1.setdefault(g.sub([0, 1, 1, 0], r)[0], []).append(r)
    assert sorted(len(v) for v in t1.values()) == [4, 4]


@pytest.mark.parametrize("seed", range(6))
def test_dim_partitions_match_the_per_element_mapping(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        Bx, By = int(rng.integers(1, 17)), int(rng.integers(1, 17))
        py = int(rng.integers(0, 9))
        parts = dz.redist_dim_partitions(Bx, By, py)
        # Eq. (17) per element: global index i = py By + oy  ->  px = i // Bx, ox = i % Bx
        seen = []
        for px, (oy_lo, oy_hi), (ox_lo, ox_hi) in parts:
            assert oy_hi - oy_lo == ox_hi - ox_lo > 0
            for t, oy in enumerate(range(oy_lo, oy_hi)):
                i = py * By + oy
                assert (i // Bx, i % Bx) == (px, ox_lo + t)
                seen.append(oy)
        assert seen == list(range(By))
        assert len(parts) <= -(-(By - 1) // Bx) + 1          # the bound of Eq. (24)


@pytest.mark.parametrize("seed", range(4))
def test_message_matching_matches_brute_force(seed):
    rng = np.random.default_rng(10 + seed)
    for _ in range(60):
        Bx, By = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        px = int(rng.integers(0, 9))
        lo, hi = dz.redist_match(Bx, By, px)
        xs = set(range(px * Bx, (px + 1) * Bx))
        want = [py for py in range(0, (px + 2) * Bx // By + 2) if xs & set(range(py * By, (py + 1) * By))]
        assert list(range(lo, hi)) == want


def _check_plans(gx, xdims, gy, ydims):
    order = len(xdims)
    ext = [gx.extents[d] for d in xdims]
    # expected: every y-rank receives its whole y-block exactly once
    recv_count = {r: np.zeros(ext, dtype=np.int64) for r in range(gy.size)}
    sent = []
    for r in range(gx.size):
        for peer, lo, hi in dz.redist_plan(gx, xdims, gy, ydims, r, True):
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            recv_count[peer][sl] += 1
            sent.append((r, peer, lo, hi))
            # the box lies inside the sender's x-block and the receiver's y-block
            xlo, xhi = gx.block_range(r)
            ylo, yhi = gy.block_range(peer)
            for t in range(order):
                assert xlo[xdims[t]] <= lo[t] < hi[t] <= xhi[xdims[t]]
                assert ylo[ydims[t]] <= lo[t] < hi[t] <= yhi[ydims[t]]
    for r in range(gy.size):
        ylo, yhi = gy.block_range(r)
        want = np.zeros(ext, dtype=np.int64)
        want[tuple(slice(ylo[d], yhi[d]) for d in ydims)] = 1
        np.testing.assert_array_equal(recv_count[r], want)
    # the receive plans list the same messages
    got = []
    for r in range(gy.size):
        for peer, lo, hi in dz.redist_plan(gx, xdims, gy, ydims, r, False):
            got.append((peer, r, lo, hi))
    assert sorted(got) == sorted(sent)


def test_plans_of_the_running_example():
    # t1 (i, a) from grid0 (i, j, k, a) = (2, 2, 2, 1) to grid1 (i, l, a) = (2, 2, 2)
    _check_plans(dz.Grid([10, 10, 10, 10], [2, 2, 2, 1]), [0, 3], dz.Grid([10, 10, 10], [2, 2, 2]), [0, 2])


def _factor(rng, P, D):
    """P split into D grid extents (random order of its prime factors)."""
    f, n, d = [], P, 2
    while n > 1:
        while n % d == 0:
            f.append(d)
            n //= d
        d += 1
    procs = [1] * D
    for x in f:
        procs[int(rng.integers(0, D))] *= x
    return procs


@pytest.mark.parametrize("seed", range(5))
def test_random_plans(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(8):
        P = int(rng.choice([1, 2, 4, 6, 8, 12]))
        order = int(rng.integers(1, 4))
        ext = [int(rng.integers(1, 12)) for _ in range(order)]

        def grid():
            D = int(rng.integers(order, 5))
            dims = [int(d) for d in rng.permutation(D)[:order]]
            extents = [int(rng.integers(1, 9)) for _ in range(D)]
            for t, d in enumerate(dims):
                extents[d] = ext[t]
            return dz.Grid(extents, _factor(rng, P, D)), dims
        gx, xd = grid()
        gy, yd = grid()
        _check_plans(gx, xd, gy, yd)
