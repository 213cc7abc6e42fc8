"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative Frobenius error against the oracle, the gate of the
MTTKRP / TTMc contract): 1e-5 for the FP32-accurate paths (plain FP32 FMA and
split-BF16 on tensor cores), 1e-12 for the plain FP64 path.  Element-wise, no
entry may differ by more than 1e-4 of the largest oracle entry (1e-11 for
FP64).  Inputs are the seeded synthetic tensors of the input module; at full
size the oracle runs on sampled output rows regenerated on the host by index.
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402

TOL = {"plain32": (1e-5, 1e-4), "split_bf16": (1e-5, 1e-4), "plain64": (1e-12, 1e-11)}


def _check(got, ref, kind):
    rel_f, rel_max = TOL[kind]
    got = np.asarray(got, dtype=np.float64)
    err = oracle.rel_error(got, ref)
    assert err <= rel_f, f"{kind}: relative Frobenius error {err:.3e} > {rel_f}"
    worst = oracle.max_elem_error(got, ref)
    assert worst <= rel_max, f"{kind}: max element error {worst:.3e} of max|ref| > {rel_max}"
    return err


def _factors(seed, dims, R, dtype=np.float32, sigma=1.0):
    return [inputs.factor_normal(seed, m, d, R, sigma=sigma).astype(dtype) for m, d in enumerate(dims)]


def _run_mttkrp(Xh, Us, mode, prec, dtype=torch.float32, offset=0):
    if offset:
        buf = torch.empty(Xh.size + offset, dtype=dtype, device="cuda")
        X = buf[offset:].view(Xh.shape)
        X.copy_(torch.from_numpy(Xh))
    else:
        X = torch.from_numpy(Xh).to("cuda")
    U = [torch.from_numpy(u).to("cuda") for u in Us]
    M = dz.mttkrp(X, U, mode, prec=prec)
    torch.cuda.synchronize()
    return M.cpu().numpy()


SMALL_CASES = [
    ((300, 200, 136), 32),     # several tiles, ragged rows and a ragged last chunk
    ((50, 40, 70), 16),        # narrow rows (I < 128) in every mode; K_in % 4 != 0 -> scalar loads
    ((20, 30, 17, 64), 24),    # order 4, rank padded to 32
    ((12, 9, 10, 11, 16), 8),  # order 5, rank 8
    ((500, 300), 64),          # order 2 (a matrix product), rank 64
    ((129, 3, 257), 5),        # odd extents around the tile sizes
    # short output rows with nothing to pack but outer indices (mode 0 with P = 1, and the last
    # mode): the tensor-core path packs G outer indices per tile; aligned (TMA) and not
    ((50, 70, 60), 32),        # mode 0: G = 2 outer indices per tile; mode 2: G = 2 as well
    ((40, 6, 7, 8, 36), 24),   # order 5, mode 0: O = 336 outer indices, G = 3; mode 4: G = 2
    ((1, 50, 70, 60), 16),     # mode 1 with P = 1 and an L row common to the tile
    ((50, 70, 61), 32),        # K_in % 4 != 0 (no TMA, bounds-checked loads) with packing in mode 0
    ((30, 40, 51), 64),        # last mode I = 51 (no TMA in mode 2) with packing; rank 64
    # order 2, last mode shorter than a tile and no outer index to pack: the raw tile is
    # pitch I wide and rows past I read as zero (TMA for I = 100, loads for I = 90)
    ((300, 100), 32),
    ((260, 90), 16),
    # mode 2: 64 < I = 100 < 128 with outer indices (one group per tile, not packed, TMA);
    # mode 0: I = 20 with P = 1 (G = 6 outer indices packed per tile)
    ((20, 30, 100), 16),
    # inner mode of 2100: three fiber groups per (tile, o) on the tensor-core path (16, 16
    # and 1 chunks of 64)
    ((3, 5, 2100), 8),
    # short inner modes merged with their neighbour: the last mode (K = 33 merged with 9,
    # G = 3 outer indices packed), and mode 0 of a view whose merged inner mode (60 x 64)
    # needs four fiber groups per (tile, o)
    ((7, 9, 33, 40), 16),
    ((8, 40, 60, 64), 24),
]


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
@pytest.mark.parametrize("dims,R", SMALL_CASES)
def test_mttkrp_small_all_modes(dims, R, prec):
    seed = 11
    X = inputs.tensor_uniform_f32(seed, dims)
    Us = _factors(seed, dims, R)
    for mode in range(len(dims)):
        ref = oracle.mttkrp(X, Us, mode)
        got = _run_mttkrp(X, Us, mode, prec)
        _check(got, ref, "plain32" if prec == "plain" else prec)


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_mttkrp_misaligned_x(prec, offset):
    """X 4-byte but not 16-byte aligned: no tiled tensor map of the row view; the tensor-core
    path loads through the four row-class maps (every word offset of X)."""
    dims, R = (130, 66, 128), 32
    X = inputs.tensor_uniform_f32(5, dims)
    Us = _factors(5, dims, R)
    for mode in range(3):
        got = _run_mttkrp(X, Us, mode, prec, offset=offset)
        _check(got, oracle.mttkrp(X, Us, mode), "plain32" if prec == "plain" else prec)


# Unaligned rows on the row-class path: several 128-row columns with a ragged last one,
# narrow tiles of G p values (I < 128, P > 1) and a ragged last tile, last modes with odd I
# over several columns, inner ranges with a ragged last chunk, a merged inner mode.
ROWCLASS_CASES = [
    ((131, 45, 263), 32),      # K_in = 263: four offsets along a row; mode 2: I = 263, 3 columns
    ((7, 37, 11, 129), 16),    # mode 1: narrow tiles (I = 37, G = 3), P = 7; mode 3: I = 129
    ((3, 301, 77), 64),        # rank 64; mode 1: I = 301, 3 columns; mode 2: I = 77 > 64 (not packed)
    ((9, 15, 5, 47), 8),       # mode 1: merged inner mode (5 x 47); mode 2: 16 p values per tile
]


@pytest.mark.parametrize("dims,R", ROWCLASS_CASES)
def test_mttkrp_rowclass_path(dims, R):
    X = inputs.tensor_uniform_f32(23, dims)
    Us = _factors(23, dims, R)
    for mode in range(len(dims)):
        for offset in (0, 3):
            _check(_run_mttkrp(X, Us, mode, "split_bf16", offset=offset), oracle.mttkrp(X, Us, mode),
                   "split_bf16")


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
@pytest.mark.parametrize("dims,R", [((1, 1, 1), 1), ((1, 5, 1), 3), ((7, 1, 9), 2), ((1, 1), 1)])
def test_mttkrp_degenerate_extents(dims, R, prec):
    X = inputs.tensor_uniform_f32(3, dims)
    Us = _factors(3, dims, R)
    for mode in range(len(dims)):
        _check(_run_mttkrp(X, Us, mode, prec), oracle.mttkrp(X, Us, mode),
               "plain32" if prec == "plain" else prec)


def test_mttkrp_f64_config_64cubed():
    """MTTKRP order-3, X 64^3 FP64 uniform[-1,1], B, C 64 x 16 N(0,1), mode-0 output 64 x 16 (all modes)."""
    seed = 1
    dims = (64, 64, 64)
    X = inputs.tensor_uniform_f64(seed, dims)
    Us = _factors(seed, dims, 16, dtype=np.float64)
    for mode in range(3):
        got = _run_mttkrp(X, Us, mode, "plain", dtype=torch.float64)
        _check(got, oracle.mttkrp(X, Us, mode), "plain64")


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
def test_mttkrp_bitwise_deterministic(prec):
    dims, R = (256, 190, 300), 32
    X = torch.from_numpy(inputs.tensor_uniform_f32(9, dims)).cuda()
    U = [torch.from_numpy(u).cuda() for u in _factors(9, dims, R)]
    for mode in range(3):
        a = dz.mttkrp(X, U, mode, prec=prec).clone()
        b = dz.mttkrp(X, U, mode, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


@pytest.mark.parametrize("dims,R", [((64, 64, 64, 64), 24), ((48, 40, 96, 64), 32), ((256, 300, 64), 16)])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_tma_and_rowclass_paths_agree_bitwise(dims, R, offset):
    """An aligned X goes through the tensor-map raw-tile ring, an X offset by 1-3 elements
    through the row-class maps (or, with packed outer indices, per-thread loads); the
    split and the MMAs are the same, so the outputs must be identical bit for bit
    (catches a stage reused too early or a row read at the wrong word offset)."""
    X = torch.from_numpy(inputs.tensor_uniform_f32(17, dims)).cuda()
    buf = torch.empty(X.numel() + offset, device="cuda")
    Xu = buf[offset:].view(dims)
    Xu.copy_(X)
    U = [torch.from_numpy(u).cuda() for u in _factors(17, dims, R)]
    for mode in range(len(dims)):
        a = dz.mttkrp(X, U, mode, prec="split_bf16").clone()
        b = dz.mttkrp(Xu, U, mode, prec="split_bf16")
        torch.cuda.synchronize()
        assert torch.equal(a, b), f"mode {mode}"


def test_native_library_is_what_runs():
    before = dz.kernel_launch_count()
    X = torch.ones(64, 64, 64, device="cuda")
    U = [torch.ones(64, 8, device="cuda") for _ in range(3)]
    M = dz.mttkrp(X, U, 0, prec="split_bf16")
    torch.cuda.synchronize()
    assert dz.kernel_launch_count() >= before + 3
    assert torch.allclose(M, torch.full_like(M, 64.0 * 64.0))


# ---------------------------------------------------------------------------
# Seeded generators: device == host bit for bit
# ---------------------------------------------------------------------------

def test_generators_match_host_bitwise():
    n = 1 << 20
    d32 = dz.gen_uniform(77, inputs.STREAM_X, (n,)).cpu().numpy()
    np.testing.assert_array_equal(d32, inputs.uniform_f32(77, inputs.STREAM_X, np.arange(n, dtype=np.uint64)))
    d64 = dz.gen_uniform(78, 5, (n,), dtype=torch.float64).cpu().numpy()
    np.testing.assert_array_equal(d64, inputs.uniform_f64(78, 5, np.arange(n, dtype=np.uint64)))
    dims = (9, 8, 7, 6)
    A = [inputs.factor_normal(4, m, d, 5, stream_base=inputs.STREAM_CP) for m, d in enumerate(dims)]
    dev = dz.gen_cp(4, dims, [torch.from_numpy(a).cuda() for a in A], 1e-2).cpu().numpy()
    np.testing.assert_array_equal(dev, inputs.tensor_cp_f32(4, dims, A, 1e-2))


# ---------------------------------------------------------------------------
# TTMc
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,ranks", [((20, 30, 25, 18), (4, 5, 6, 7)), ((40, 33, 50), (8, 3, 16)),
                                        ((6, 7, 5, 4, 9), (3, 2, 4, 3, 2))])
def test_ttmc_plain_all_keep_modes(dims, ranks):
    X = inputs.tensor_uniform_f32(13, dims)
    Us = [inputs.factor_normal(13, m, d, r).astype(np.float32) for m, (d, r) in enumerate(zip(dims, ranks))]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    for keep in range(len(dims)):
        got = dz.ttmc(Xd, Ud, keep).cpu().numpy()
        _check(got, oracle.ttmc(X, Us, keep), "plain32")


def test_ttmc_identity_returns_x():
    dims = (12, 10, 9)
    X = inputs.tensor_uniform_f32(2, dims)
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.eye(d, device="cuda") for d in dims]
    for keep in range(3):
        np.testing.assert_array_equal(dz.ttmc(Xd, Ud, keep).cpu().numpy(), X)


def test_ttmc_f64():
    dims, ranks = (15, 12, 10, 8), (3, 4, 5, 6)
    X = inputs.tensor_uniform_f64(3, dims)
    Us = [inputs.factor_normal(3, m, d, r) for m, (d, r) in enumerate(zip(dims, ranks))]
    got = dz.ttmc(torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in Us], 0).cpu().numpy()
    _check(got, oracle.ttmc(X, Us, 0), "plain64")


@pytest.mark.parametrize("prec", ["plain", "split_bf16", "plain64"])
@pytest.mark.parametrize("dims,R,L", [((160, 96, 136), 24, 40), ((20, 30, 17, 64), 32, 7), ((50, 70, 60), 16, 64)])
def test_mttkrp_mm_all_modes(dims, R, L, prec):
    """MTTKRP + MM (Sec. II-A running example, product applied in the final reduction)."""
    seed = 23
    dtype = np.float64 if prec == "plain64" else np.float32
    X = inputs.tensor_uniform_f32(seed, dims).astype(dtype)
    Us = _factors(seed, dims, R, dtype=dtype)
    C = inputs.factor_normal(seed, 9, R, L).astype(dtype)
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    Cd = torch.from_numpy(C).cuda()
    for mode in range(len(dims)):
        got = dz.mttkrp_mm(Xd, Ud, mode, Cd, prec="plain" if prec == "plain64" else prec)
        torch.cuda.synchronize()
        assert tuple(got.shape) == (dims[mode], L)
        _check(got.cpu().numpy(), oracle.mttkrp_mm(X, Us, mode, C), "plain32" if prec == "plain" else prec)
