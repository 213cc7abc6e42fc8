"""Split-BF16 TTMc (fused last-two-mode tensor-core kernel + plain chain) against the FP64 oracle.

Gate: relative Frobenius error <= 1e-5 and element-wise <= 1e-4 of the largest
oracle entry (the FP32-accurate tolerance of the TTMc contract).  Cases cover
ragged k tiles (I_{N-2} not a multiple of 128), ragged l chunks (I_{N-1} not a
multiple of 64), a k extent below one tile, ranks below the padded 32, orders
3 to 5, every kept mode the fused path takes, short slabs packed two or four to a
tile (partial last groups, every store path of the T2 writer warps), rows of X that
are not 16-byte aligned (the row-class tensor maps, one slab per tile or packed), and
order-5 chains with the kept mode before or
between the two chain modes, ragged trailing extents and ranks that are not multiples
of 8, and order-6 chains (two chain TTMs on the tensor cores, the third in FP32).
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402


def _check(got, ref):
    got = np.asarray(got, dtype=np.float64)
    err = oracle.rel_error(got, ref)
    assert err <= 1e-5, f"relative Frobenius error {err:.3e}"
    worst = oracle.max_elem_error(got, ref)
    assert worst <= 1e-4, f"max element error {worst:.3e}"
    return err


CASES = [
    # (dims, keep, ranks of the contracted modes in mode order)
    ((36, 40, 200, 68), 0, (8, 24, 32)),      # two k tiles (ragged), two l chunks (ragged)
    ((20, 30, 130, 64), 1, (5, 16, 12)),      # keep mode 1: the chain contracts mode 0 afterwards
    ((50, 300, 132), 0, (17, 31)),            # order 3: the fused kernel writes Y directly
    ((70, 40, 100), 0, (32, 20)),             # k extent below one tile (narrow box)
    ((6, 7, 8, 90, 44), 0, (3, 5, 32, 7)),    # order 5, two more chain stages
    ((6, 7, 8, 90, 44), 2, (4, 6, 9, 32)),    # order 5, kept mode in the middle
    # short slabs share a tile: I_{N-2} <= 64 two per tile, <= 32 four per tile; the slab
    # counts leave a partial last group; T2 blocks of up to 8 KB a tile (sizes a multiple
    # of 16 bytes) go out as one bulk store each, other ones from the feed warps
    ((31, 7, 60, 60), 0, (5, 24, 24)),        # two slabs per tile, S = 217
    ((9, 13, 28, 36), 0, (6, 30, 10)),        # four slabs per tile, S = 117
    ((5, 40, 33, 64), 1, (7, 32, 32)),        # two per tile, kept mode 1
    ((70, 64, 20), 0, (32, 13)),              # order 3, I_{N-2} = 64 exactly
    ((3, 5, 32, 8), 0, (2, 3, 4)),            # I_{N-2} = 32 exactly, one 8-wide l chunk
    ((4, 6, 60, 60, 60), 0, (24, 24, 24, 24)),  # the paper's order-5 TTMc shape, fewer slabs
    ((9, 20, 40), 0, (24, 24)),               # four per tile, 9 KB of T2 a tile: the feed warps' own 16-byte stores
    ((7, 50, 44), 0, (5, 7)),                 # two per tile, R_{N-1} = 7: the feed warps' 4-byte stores
    ((7, 50, 44), 0, (5, 6)),                 # bulk stores, the last group's 30 floats copied by words
    # order-5 chains after the fused pair
    ((9, 11, 40, 64, 36), 1, (13, 21, 24, 16)),  # kept mode 1 between the two chain modes
    ((7, 30, 50, 60, 20), 0, (19, 11, 8, 5)),    # ranks 19 / 11, trailing extent 40
    ((6, 50, 9, 64, 20), 0, (40, 7, 16, 8)),     # R_1 = 40
    # chain TTMs on the tensor cores at their edges: a trailing extent of one 128-row column
    # then rank 64 (R_pad 64); a trailing extent of 8 (an 8-row box)
    ((3, 70, 5, 64, 36), 0, (64, 3, 16, 8)),
    ((5, 7, 2, 8, 12), 0, (3, 2, 1, 4)),
    # order 6: three chain stages, the first two on the tensor cores, the last in FP32
    ((5, 6, 7, 8, 60, 36), 0, (4, 5, 6, 24, 16)),
    ((6, 5, 30, 7, 40, 44), 1, (3, 9, 5, 20, 12)),
]


@pytest.mark.parametrize("dims,keep,ranks", CASES)
def test_split_ttmc_matches_oracle(dims, keep, ranks):
    seed = 31 + sum(dims) + keep
    X = inputs.tensor_uniform_f32(seed, dims)
    rk = iter(ranks)
    Us = [None if m == keep else inputs.factor_normal(seed, m, d, next(rk)).astype(np.float32)
          for m, d in enumerate(dims)]
    Xd = torch.from_numpy(X).cuda()
    Ud = [None if u is None else torch.from_numpy(u).cuda() for u in Us]
    Y = dz.ttmc(Xd, Ud, keep, prec="split_bf16")
    torch.cuda.synchronize()
    ref = oracle.ttmc(X, Us, keep)
    assert Y.shape == ref.shape
    _check(Y.cpu().numpy(), ref)
    # against the plain FP32 chain as well
    P = dz.ttmc(Xd, Ud, keep, prec="plain")
    torch.cuda.synchronize()
    y64, p64 = Y.cpu().numpy().astype(np.float64), P.cpu().numpy().astype(np.float64)
    assert oracle.rel_error(y64, p64) <= 1e-5
    assert oracle.max_elem_error(y64, p64) <= 1e-4


def test_split_ttmc_is_bitwise_deterministic():
    dims, keep = (24, 33, 260, 96), 0
    X = torch.from_numpy(inputs.tensor_uniform_f32(5, dims)).cuda()
    U = [None] + [torch.from_numpy(inputs.factor_normal(5, m, dims[m], 32).astype(np.float32)).cuda()
                  for m in (1, 2, 3)]
    a = dz.ttmc(X, U, keep, prec="split_bf16").clone()
    b = dz.ttmc(X, U, keep, prec="split_bf16")
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_split_ttmc_rank1_closed_form():
    # X = a o b o c o d  =>  Y[i, :, :, :] = a_i (U1^T b) o (U2^T c) o (U3^T d)
    n = (40, 50, 150, 72)
    vec = [inputs.factor_normal(77, m, n[m], 1).astype(np.float32)[:, 0] for m in range(4)]
    X = np.einsum("i,j,k,l->ijkl", *[v.astype(np.float64) for v in vec]).astype(np.float32)
    U = [None] + [inputs.factor_normal(77, 10 + m, n[m], r).astype(np.float32) for m, r in ((1, 9), (2, 32), (3, 17))]
    Y = dz.ttmc(torch.from_numpy(X).cuda(), [None if u is None else torch.from_numpy(u).cuda() for u in U], 0,
                prec="split_bf16")
    torch.cuda.synchronize()
    ref = oracle.ttmc(X, U, 0)
    _check(Y.cpu().numpy(), ref)


# Rows of X that are not 16-byte aligned (I_{N-1} not a multiple of 4, or X itself offset):
# the row-class tensor maps, one slab per tile; tensor-core stage 2 (I_{N-2} <= 256) and
# CUDA-core stage 2 (I_{N-2} > 256).
ROWCLASS_CASES = [
    # (dims, keep, ranks, X offset in floats)
    ((8, 9, 130, 66), 0, (5, 16, 12), 0),       # I_{N-1} = 66: rows 8 bytes off, two l chunks
    ((8, 9, 130, 64), 0, (5, 16, 12), 1),       # aligned shape, X one float into its buffer
    ((31, 7, 60, 61), 0, (5, 24, 24), 0),       # short slabs (I_{N-2} = 60) two to a tile
    ((50, 300, 133), 0, (17, 31), 3),           # order 3, I_{N-2} = 300: CUDA-core stage 2
    ((6, 7, 8, 90, 45), 0, (3, 5, 32, 7), 2),   # order 5, two chain stages after the fused pair
    ((4, 6, 60, 60, 61), 0, (24, 24, 24, 24), 0),   # the paper's order-5 shape with an odd last mode
    ((7, 64, 66), 0, (9, 20), 0),               # slabs of exactly 64 rows
    ((3, 65, 70), 0, (9, 20), 1),               # 65-row slabs, X one float into its buffer
    ((5, 3, 5, 9), 0, (2, 3, 7), 2),            # 3-row slabs, 9-word rows
    ((7, 32, 30), 0, (5, 17), 1),               # four 32-row slabs a tile, the last group of three
    ((9, 33, 50), 0, (4, 9), 3),                # two 33-row slabs a tile, the last group of one
    ((5, 20, 150), 0, (3, 20), 2),              # four 20-row slabs a tile, three l chunks
]


@pytest.mark.parametrize("dims,keep,ranks,offset", ROWCLASS_CASES)
def test_split_ttmc_rowclass_matches_oracle(dims, keep, ranks, offset):
    seed = 57 + sum(dims) + keep + offset
    X = inputs.tensor_uniform_f32(seed, dims)
    rk = iter(ranks)
    Us = [None if m == keep else inputs.factor_normal(seed, m, d, next(rk)).astype(np.float32)
          for m, d in enumerate(dims)]
    buf = torch.empty(X.size + offset, device="cuda")
    Xd = buf[offset:].view(dims)
    Xd.copy_(torch.from_numpy(X))
    Ud = [None if u is None else torch.from_numpy(u).cuda() for u in Us]
    Y = dz.ttmc(Xd, Ud, keep, prec="split_bf16")
    torch.cuda.synchronize()
    ref = oracle.ttmc(X, Us, keep)
    _check(Y.cpu().numpy(), ref)
    # the same result as the tensor-map path where one exists (aligned copy of X)
    if dims[-1] % 4 == 0:
        A = dz.ttmc(torch.from_numpy(X).cuda(), Ud, keep, prec="split_bf16")
        torch.cuda.synchronize()
        assert oracle.rel_error(Y.cpu().numpy().astype(np.float64), A.cpu().numpy().astype(np.float64)) <= 1e-5
