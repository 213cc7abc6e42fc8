"""The running example of Sec. II (ijk,ja,ka,al->il) as the distributed program the
paper generates (Sec. II-C/D and its Python listing), emulated by gloo ranks on the CPU:
block-distributed inputs with replication, local MTTKRP partials, an Allreduce over the
Cartesian sub-grid that shares each t1-block, the redistribution of t1 from the first
grid to the second with the library's send / receive plans (Eqs. 20-25), the local
matrix product and the Allreduce of its partials.  The assembled result must equal the
FP64 oracle.  No GPU is involved (the grids here model the sharding of a multi-GPU run).
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N = {"i": 10, "j": 9, "k": 8, "a": 6, "l": 7}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _groups(grid, remain, world):
    """One process group per sub-grid (every rank creates all of them, in order)."""
    members = {}
    for r in range(world):
        members.setdefault(grid.sub(remain, r)[0], []).append(r)
    mine = None
    for color in sorted(members):
        g = dist.new_group(members[color])
        if dist.get_rank() in members[color]:
            mine = g
    return mine


def _worker(rank, world, port, p0, p1):
    import oracle
    import paper_2206_08301_gb300 as dz
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        rng = np.random.default_rng(5)          # every rank draws the same inputs, keeps its blocks
        X = rng.standard_normal((N["i"], N["j"], N["k"]))
        A = rng.standard_normal((N["j"], N["a"]))
        B = rng.standard_normal((N["k"], N["a"]))
        C = rng.standard_normal((N["a"], N["l"]))
        g0 = dz.Grid([N["i"], N["j"], N["k"], N["a"]], p0)       # (i, j, k, a)
        g1 = dz.Grid([N["i"], N["l"], N["a"]], p1)               # (i, l, a)
        (i0, j0, k0, a0), (i1, j1, k1, a1) = g0.block_range(rank)
        # first group: t1[i, a] = sum_jk X[i, j, k] A[j, a] B[k, a] on this rank's block
        t1 = np.einsum("ijk,ja,ka->ia", X[i0:i1, j0:j1, k0:k1], A[j0:j1, a0:a1], B[k0:k1, a0:a1])
        t1 = torch.from_numpy(np.ascontiguousarray(t1))
        dist.all_reduce(t1, group=_groups(g0, [0, 1, 1, 0], world))   # partials over (j, k)
        # redistribute t1 (modes i, a) from grid 0 (dims 0, 3) to grid 1 (dims 0, 2)
        (yi0, yl0, ya0), (yi1, yl1, ya1) = g1.block_range(rank)
        t2 = torch.zeros(yi1 - yi0, ya1 - ya0, dtype=torch.float64)
        sends = dz.redist_plan(g0, [0, 3], g1, [0, 2], rank, True)
        recvs = dz.redist_plan(g0, [0, 3], g1, [0, 2], rank, False)
        reqs = []
        for peer, lo, hi in sends:
            box = t1[lo[0] - i0:hi[0] - i0, lo[1] - a0:hi[1] - a0].contiguous()
            if peer == rank:
                t2[lo[0] - yi0:hi[0] - yi0, lo[1] - ya0:hi[1] - ya0] = box
            else:
                reqs.append(dist.isend(box, peer))
        for peer, lo, hi in recvs:
            if peer == rank:
                continue
            buf = torch.empty(hi[0] - lo[0], hi[1] - lo[1], dtype=torch.float64)
            dist.recv(buf, src=peer)
            t2[lo[0] - yi0:hi[0] - yi0, lo[1] - ya0:hi[1] - ya0] = buf
        for r in reqs:
            r.wait()
        # second group: out[i, l] = sum_a t2[i, a] C[a, l], partials over a
        out = t2 @ torch.from_numpy(C[ya0:ya1, yl0:yl1])
        dist.all_reduce(out, group=_groups(g1, [0, 0, 1], world))
        # assemble (one replica per out-block contributes) and check against the oracle
        full = torch.zeros(N["i"], N["l"], dtype=torch.float64)
        if g1.coords(rank)[2] == 0:
            full[yi0:yi1, yl0:yl1] = out
        dist.all_reduce(full)
        ref = oracle.mttkrp_mm(X, [None, A, B], 0, C)
        np.testing.assert_allclose(full.numpy(), ref, rtol=1e-12, atol=1e-12)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,p0,p1", [
    (2, [1, 2, 1, 1], [2, 1, 1]),     # j split in the first group, i in the second
    (4, [2, 2, 1, 1], [1, 2, 2]),     # t1 moves from (i) blocks to (a) blocks with replication
    (4, [1, 1, 2, 2], [2, 2, 1]),
])
def test_running_example_distributed(world, p0, p1):
    mp.spawn(_worker, args=(world, _free_port(), p0, p1), nprocs=world, join=True)
