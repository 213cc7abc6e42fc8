"""The allocation-free MTTKRP entry point against the planned one.

deinsum_mttkrp_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they cannot afford cudaMalloc's
implicit synchronisation); its scratch is a fixed array inside the library.
This file checks, through the C ABI, that two calls in a row give the output
of deinsum_plan + deinsum_execute (split-BF16) within the tests' tolerance
(relative Frobenius error 1e-5), that calls after the first leave the free
device memory unchanged, and that oversize problems are refused.  It is named
to be collected last, and passes alone or after the rest of the suite.
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


@pytest.mark.parametrize("dims,R", [((300, 200, 136), 32), ((20, 30, 17, 64), 24), ((12, 9, 10, 11, 16), 8),
                                    ((130, 66, 96), 64)])
def test_noalloc_matches_planned_execute_twice(dims, R):
    lib = dz.load()
    X = torch.from_numpy(inputs.tensor_uniform_f32(31, dims)).cuda()
    U = [torch.from_numpy(inputs.factor_normal(31, m, d, R).astype(np.float32)).cuda() for m, d in enumerate(dims)]
    for mode in range(len(dims)):
        ref = dz.mttkrp(X, U, mode, prec="split_bf16").cpu().numpy().astype(np.float64)
        for _ in range(2):
            out = torch.full((dims[mode], R), float("nan"), device="cuda")
            assert _call(lib, X, U, mode, out) == 0
            torch.cuda.synchronize()
            err = oracle.rel_error(out.cpu().numpy(), ref)
            assert err <= 1e-5, f"mode {mode}: relative error {err:.3e} against the planned path"


def test_noalloc_allocates_no_device_memory_after_the_first_call():
    lib = dz.load()
    dims, R = (256, 128, 192), 16
    X = torch.from_numpy(inputs.tensor_uniform_f32(32, dims)).cuda()
    U = [torch.from_numpy(inputs.factor_normal(32, m, d, R).astype(np.float32)).cuda() for m, d in enumerate(dims)]
    outs = [torch.empty(dims[m], R, device="cuda") for m in range(3)]
    assert _call(lib, X, U, 0, outs[0]) == 0          # first call: per-device set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for mode in (0, 1, 2, 0, 1, 2):
        assert _call(lib, X, U, mode, outs[mode]) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


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
