"""GPU parity at the full benchmark sizes, on sampled outputs.

* MTTKRP order-3, X 1024^3 FP32 uniform[-1,1), factors 1024 x 32 N(0, 1/32),
  modes 0, 1, 2, plain FP32 and split-BF16: 64 output rows per mode chosen
  from the seed.
* MTTKRP order-5, X 64^5 FP32 = rank-24 CP tensor (N(0,1) factors) + 1e-3
  noise, R = 24 (N(0,1) factors), modes 0 and 2: 4 output rows per mode.
* TTMc order-4 ``ijkl,jb,kc,ld->ibcd``, X 256^4 FP32 uniform[-1,1), 256 x 32
  N(0,1) matrices: 2 kept-mode slices.

X is generated on the device by the seeded generator; the oracle's inputs are
the same elements regenerated on the host by index (bit-identical, checked in
test_parity_gpu).  Gate: relative Frobenius error <= 1e-5 over the sample,
every entry within 1e-4 of the sample's largest oracle entry.
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402


def _check(got, ref):
    err = oracle.rel_error(got, ref)
    assert err <= 1e-5, f"relative Frobenius error {err:.3e}"
    worst = oracle.max_elem_error(got, ref)
    assert worst <= 1e-4, f"max element error {worst:.3e}"
    return err


@pytest.fixture(scope="module")
def cube1024():
    seed, n, R = 2024, 1024, 32
    dims = (n, n, n)
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R, sigma=np.sqrt(1.0 / R)).astype(np.float32) for m in range(3)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    refs = {}
    for mode in range(3):
        rows = inputs.sample_rows(seed, n, 64, tag=mode)
        slabs = np.stack([inputs.uniform_slab(seed, dims, mode, int(r)).ravel() for r in rows])
        refs[mode] = (rows, oracle.mttkrp_rows(dims, mode, slabs, Us))
    yield X, Ud, refs
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
def test_mttkrp_1024_cubed_r32_all_modes(cube1024, prec):
    X, Ud, refs = cube1024
    for mode in range(3):
        M = dz.mttkrp(X, Ud, mode, prec=prec)
        torch.cuda.synchronize()
        rows, ref = refs[mode]
        _check(M[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)


@pytest.fixture(scope="module")
def order5_cp():
    seed, n, rc, R = 5055, 64, 24, 24
    dims = (n,) * 5
    A = [inputs.factor_normal(seed, m, n, rc, stream_base=inputs.STREAM_CP) for m in range(5)]
    X = dz.gen_cp(seed, dims, [torch.from_numpy(a).cuda() for a in A], 1e-3)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(5)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    refs = {}
    for mode in (0, 2):
        rows = inputs.sample_rows(seed, n, 4, tag=mode)
        slabs = np.stack([inputs.cp_slab(seed, dims, A, 1e-3, mode, int(r)).ravel() for r in rows])
        refs[mode] = (rows, oracle.mttkrp_rows(dims, mode, slabs, Us))
    yield X, Ud, refs
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
def test_mttkrp_order5_cp_modes_0_2(order5_cp, prec):
    X, Ud, refs = order5_cp
    for mode in (0, 2):
        M = dz.mttkrp(X, Ud, mode, prec=prec)
        torch.cuda.synchronize()
        rows, ref = refs[mode]
        _check(M[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)


def test_ttmc_256_order4_plain():
    seed, n, R = 4096, 256, 32
    dims = (n,) * 4
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(4)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    Y = dz.ttmc(X, Ud, 0)
    torch.cuda.synchronize()
    del X
    rows = inputs.sample_rows(seed, n, 2, tag=7)
    slabs = np.stack([inputs.uniform_slab(seed, dims, 0, int(r)).ravel() for r in rows])
    ref = oracle.ttmc_rows(dims, 0, slabs, Us)
    _check(Y[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)
    torch.cuda.empty_cache()


def test_ttmc_256_order4_split():
    # the benchmark workload: X 256^4 FP32, R = 32, keep mode 0, fused split-BF16 path
    seed, n, R = 4096, 256, 32
    dims = (n,) * 4
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(4)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    Y = dz.ttmc(X, Ud, 0, prec="split_bf16")
    torch.cuda.synchronize()
    del X
    rows = inputs.sample_rows(seed, n, 2, tag=7)
    slabs = np.stack([inputs.uniform_slab(seed, dims, 0, int(r)).ravel() for r in rows])
    ref = oracle.ttmc_rows(dims, 0, slabs, Us)
    _check(Y[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)
    torch.cuda.empty_cache()


def test_ttmc_60_order5_split():
    # TTMc-O5-M0 of the paper's benchmark table: X 60^5, R^n = 24 (fused last two modes + chain)
    seed, n, R = 1301, 60, 24
    dims = (n,) * 5
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(5)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    Y = dz.ttmc(X, Ud, 0, prec="split_bf16")
    torch.cuda.synchronize()
    del X
    rows = inputs.sample_rows(seed, n, 2, tag=3)
    slabs = np.stack([inputs.uniform_slab(seed, dims, 0, int(r)).ravel() for r in rows])
    ref = oracle.ttmc_rows(dims, 0, slabs, Us)
    _check(Y[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)
    torch.cuda.empty_cache()
