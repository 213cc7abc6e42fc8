"""Failure detection on the device: a bounded wait that runs out.

Every wait inside the tensor-core kernels is bounded.  When one gives up, the
kernel sets its status word, stops every role, lets the bulk copies and MMAs
it issued finish, frees its tensor memory and returns, so the context stays
usable.  These tests make that happen without breaking anything: a wait limit
of 1 ns (deinsum_set_wait_limit_ns) is shorter than the first TMA load from
HBM, so a real execute gives up.  Each test checks that the status reads
DEINSUM_ERR_TIMEOUT (8) and that, with the default limit restored, the next
execute on the same plan (or a new batch) reads DEINSUM_OK and matches the
FP64 oracle within the split-BF16 gate.
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402

TIMEOUT = 8


def _gate(got, ref):
    assert oracle.rel_error(got, ref) <= 1e-5
    assert oracle.max_elem_error(got, ref) <= 1e-4


@pytest.fixture
def short_waits():
    """Sets the 1 ns limit for the test body's launches; always restores the default."""
    yield lambda on: dz.set_wait_limit_ns(1 if on else 0)
    dz.set_wait_limit_ns(0)


@pytest.mark.parametrize("dims,mode,offset", [((300, 200, 136), 0, 0), ((300, 200, 136), 2, 0),
                                              ((255, 130, 131), 1, 1)])
def test_mttkrp_wait_runs_out_then_recovers(short_waits, dims, mode, offset):
    R = 32
    X = inputs.tensor_uniform_f32(51, dims)
    U = [inputs.factor_normal(51, m, d, R).astype(np.float32) for m, d in enumerate(dims)]
    if offset:   # rows not 16-byte aligned: the row-class loads
        buf = torch.empty(X.size + offset, device="cuda")
        Xd = buf[offset:].view(dims)
        Xd.copy_(torch.from_numpy(X))
    else:
        Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    plan = dz.Plan(dz.mttkrp_einsum(3, mode), list(dims) + [R], "float32", "split_bf16")
    ops = [Xd] + [Ud[m] for m in range(3) if m != mode]
    out = torch.empty(dims[mode], R, device="cuda")
    plan(*ops, out=out)               # first execute: workspace, default limit
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    short_waits(True)
    plan(*ops, out=out)
    torch.cuda.synchronize()
    assert plan.last_device_status() == TIMEOUT
    short_waits(False)
    out.fill_(float("nan"))
    plan(*ops, out=out)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    _gate(out.cpu().numpy(), oracle.mttkrp(X, U, mode))


def test_ttmc_wait_runs_out_then_recovers(short_waits):
    dims, keep = (20, 30, 130, 64), 0
    ranks = (None, 8, 24, 32)
    X = inputs.tensor_uniform_f32(52, dims)
    U = [None] + [inputs.factor_normal(52, m, dims[m], ranks[m]).astype(np.float32) for m in (1, 2, 3)]
    Xd = torch.from_numpy(X).cuda()
    Ud = [None] + [torch.from_numpy(u).cuda() for u in U[1:]]
    plan = dz.Plan(dz.ttmc_einsum(4, keep), list(dims) + list(ranks[1:]), "float32", "split_bf16")
    out = torch.empty(dims[0], 8, 24, 32, device="cuda")
    plan(Xd, *Ud[1:], out=out)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    short_waits(True)
    plan(Xd, *Ud[1:], out=out)
    torch.cuda.synchronize()
    assert plan.last_device_status() == TIMEOUT
    short_waits(False)
    plan(Xd, *Ud[1:], out=out)
    torch.cuda.synchronize()
    assert plan.last_device_status() == 0
    _gate(out.cpu().numpy(), oracle.ttmc(X, U, keep))


def test_batched_wait_runs_out_then_recovers(short_waits):
    seed, n = 53, 8
    ext = inputs.draw_int(seed, 0, 40, 150, 3 * n).reshape(n, 3)
    ranks = np.array([8, 16, 32, 64])[inputs.draw_int(seed, 1, 0, 3, n)]
    modes = inputs.draw_int(seed, 2, 0, 2, n)
    einsums, extents, ins, outs, refs = [], [], [], [], []
    for k in range(n):
        dims, R, mode = tuple(int(d) for d in ext[k]), int(ranks[k]), int(modes[k])
        X = inputs.tensor_uniform_f32(seed * 100 + k, dims)
        U = [inputs.factor_normal(seed * 100 + k, m, d, R).astype(np.float32) for m, d in enumerate(dims)]
        einsums.append(dz.mttkrp_einsum(3, mode))
        extents.append(list(dims) + [R])
        ins.append([torch.from_numpy(X).cuda()] + [torch.from_numpy(U[m]).cuda() for m in range(3) if m != mode])
        outs.append(torch.empty(dims[mode], R, device="cuda"))
        refs.append(oracle.mttkrp(X, U, mode))
    short_waits(True)                 # the limit is taken when the batch's graph is captured
    b = dz.Batch(einsums, extents, "split_bf16")
    b(ins, outs)
    torch.cuda.synchronize()
    assert b.status() == TIMEOUT
    short_waits(False)
    b2 = dz.Batch(einsums, extents, "split_bf16")
    b2(ins, outs)
    torch.cuda.synchronize()
    assert b2.status() == 0
    for out, ref in zip(outs, refs):
        _gate(out.cpu().numpy(), ref)
