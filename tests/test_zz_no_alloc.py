"""The allocation-free MTTKRP entry point against the FP64 oracle and the planned one.

deinsum_mttkrp_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they cannot afford cudaMalloc's
implicit synchronisation); its scratch is a fixed array inside the library.
Through the C ABI this file checks that:

* two calls in a row give the FP64 oracle's result within the split-BF16 gate
  (relative Frobenius 1e-5, element-wise 1e-4 of the largest oracle entry) and
  the output of deinsum_plan + deinsum_execute (split-BF16) within 2e-5 --
  orders 2 to 5, and an X that starts one float into its buffer (rows not
  16-byte aligned: the row-class loads);
* deinsum_mttkrp_noalloc_status reads DEINSUM_OK after a normal call, and
  DEINSUM_ERR_TIMEOUT after a call whose bounded waits were given a 1 ns limit,
  after which the next call is correct again;
* calls after the first make no allocation (the library's allocation counter,
  and the device's free memory as a second check), and oversize problems are
  refused.

It is named to be collected last, and passes alone or after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402


def _call(lib, X, U, mode, out):
    order = X.dim()
    R = next(u.shape[1] for m, u in enumerate(U) if m != mode)
    dims = (ctypes.c_int64 * order)(*X.shape)
    fac = (ctypes.c_void_p * order)(*[None if m == mode else U[m].data_ptr() for m in range(order)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.deinsum_mttkrp_noalloc(order, dims, mode, int(R), ctypes.c_void_p(X.data_ptr()), fac,
                                      ctypes.c_void_p(out.data_ptr()), stream)


def _inputs(seed, dims, R, offset=0):
    Xh = inputs.tensor_uniform_f32(seed, dims)
    Uh = [inputs.factor_normal(seed, m, d, R).astype(np.float32) for m, d in enumerate(dims)]
    if offset:
        buf = torch.empty(Xh.size + offset, device="cuda")
        X = buf[offset:].view(dims)
        X.copy_(torch.from_numpy(Xh))
    else:
        X = torch.from_numpy(Xh).cuda()
    return Xh, Uh, X, [torch.from_numpy(u).cuda() for u in Uh]


@pytest.mark.parametrize("dims,R,offset", [((300, 200, 136), 32, 0), ((20, 30, 17, 64), 24, 0),
                                           ((12, 9, 10, 11, 16), 8, 0), ((130, 66, 96), 64, 0),
                                           ((257, 131, 75), 16, 1), ((500, 300), 32, 0)])
def test_noalloc_matches_oracle_and_planned_execute_twice(dims, R, offset):
    lib = dz.load()
    Xh, Uh, X, U = _inputs(31, dims, R, offset)
    for mode in range(len(dims)):
        ref = oracle.mttkrp(Xh, Uh, mode)
        planned = dz.mttkrp(X, U, mode, prec="split_bf16").cpu().numpy().astype(np.float64)
        for _ in range(2):
            out = torch.full((dims[mode], R), float("nan"), device="cuda")
            assert _call(lib, X, U, mode, out) == 0
            torch.cuda.synchronize()
            assert lib.deinsum_mttkrp_noalloc_status() == 0
            got = out.cpu().numpy()
            err = oracle.rel_error(got, ref)
            assert err <= 1e-5, f"mode {mode}: relative error {err:.3e} against the FP64 oracle"
            assert oracle.max_elem_error(got, ref) <= 1e-4
            # the planned path may regroup a short inner mode: both within 1e-5 of the oracle
            assert oracle.rel_error(got, planned) <= 2e-5


def test_noalloc_status_reports_a_wait_that_ran_out():
    lib = dz.load()
    dims, R, mode = (300, 200, 136), 32, 1
    Xh, Uh, X, U = _inputs(33, dims, R)
    out = torch.empty(dims[mode], R, device="cuda")
    try:
        dz.set_wait_limit_ns(1)
        assert _call(lib, X, U, mode, out) == 0      # launched fine; the device gives up
        torch.cuda.synchronize()
        assert lib.deinsum_mttkrp_noalloc_status() == 8
    finally:
        dz.set_wait_limit_ns(0)
    assert _call(lib, X, U, mode, out) == 0
    torch.cuda.synchronize()
    assert lib.deinsum_mttkrp_noalloc_status() == 0
    ref = oracle.mttkrp(Xh, Uh, mode)
    assert oracle.rel_error(out.cpu().numpy(), ref) <= 1e-5
    assert oracle.max_elem_error(out.cpu().numpy(), ref) <= 1e-4


def test_noalloc_allocates_no_device_memory_after_the_first_call():
    lib = dz.load()
    dims, R = (256, 128, 192), 16
    _, _, X, U = _inputs(32, dims, R)
    outs = [torch.empty(dims[m], R, device="cuda") for m in range(3)]
    assert _call(lib, X, U, 0, outs[0]) == 0          # first call: per-device set-up
    torch.cuda.synchronize()
    allocs0 = dz.alloc_count()
    free0 = torch.cuda.mem_get_info()[0]
    for mode in (0, 1, 2, 0, 1, 2):
        assert _call(lib, X, U, mode, outs[mode]) == 0
    torch.cuda.synchronize()
    assert lib.deinsum_mttkrp_noalloc_status() == 0
    assert dz.alloc_count() == allocs0                # the library allocated nothing
    assert torch.cuda.mem_get_info()[0] == free0      # and the device's free memory agrees


def test_noalloc_refuses_oversize_problems():
    lib = dz.load()
    X = torch.zeros(4, device="cuda")
    U = [torch.zeros(4, device="cuda") for _ in range(3)]
    out = torch.zeros(4, device="cuda")
    dims = (ctypes.c_int64 * 3)(16, 16, 16)
    fac = (ctypes.c_void_p * 3)(None, U[1].data_ptr(), U[2].data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # rank above 64
    assert lib.deinsum_mttkrp_noalloc(3, dims, 0, 65, ctypes.c_void_p(X.data_ptr()), fac,
                                      ctypes.c_void_p(out.data_ptr()), st) == 3
    # output mode beyond 256 blocks of 128 rows, and a contracted mode beyond 4096 at rank 64
    big = (ctypes.c_int64 * 3)(40000, 2, 8)
    assert lib.deinsum_mttkrp_noalloc(3, big, 0, 8, ctypes.c_void_p(X.data_ptr()), fac,
                                      ctypes.c_void_p(out.data_ptr()), st) == 3
    long_k = (ctypes.c_int64 * 3)(8, 2, 5000)
    assert lib.deinsum_mttkrp_noalloc(3, long_k, 0, 64, ctypes.c_void_p(X.data_ptr()), fac,
                                      ctypes.c_void_p(out.data_ptr()), st) == 3
