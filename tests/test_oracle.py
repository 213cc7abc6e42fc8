"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formula: each compares it with a different
object -- the Listing-1 brute force, the factored KRP + TDOT form of Sec. II-A,
numpy's einsum (a library routine), closed forms of structured inputs,
invariances, and a hand-worked example (tests/golden).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LETTERS = "ijklmnop"


def _factors(rng, dims, R):
    return [rng.standard_normal((d, R)) for d in dims]


def _mttkrp_spec(order, mode):
    x = LETTERS[:order]
    ins = [x] + [LETTERS[m] + "r" for m in range(order) if m != mode]
    return ",".join(ins) + "->" + LETTERS[mode] + "r"


def _ttmc_spec(order, keep):
    x = LETTERS[:order]
    ranks = "abcdefgh"
    ins = [x] + [LETTERS[m] + ranks[m] for m in range(order) if m != keep]
    out = "".join(LETTERS[m] if m == keep else ranks[m] for m in range(order))
    return ",".join(ins) + "->" + out


def _read_golden(name):
    blocks = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]
    it = iter(lines)
    for header in it:
        parts = header.split()
        shape = tuple(int(p) for p in parts[1:])
        vals = np.array([float(v) for v in next(it).split()])
        blocks[parts[0]] = vals.reshape(shape)
    return blocks


# ---------------------------------------------------------------------------
# MTTKRP
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(3, 4), (3, 4, 2), (2, 3, 2, 3), (2, 2, 3, 2, 2)])
def test_mttkrp_matches_listing1_bruteforce(dims):
    rng = np.random.default_rng(1)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 3)
    for mode in range(len(dims)):
        ops = [X] + [U[m] for m in range(len(dims)) if m != mode]
        ref = oracle.einsum_naive(_mttkrp_spec(len(dims), mode), *ops)
        got = oracle.mttkrp(X, U, mode)
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims", [(3, 4, 2), (2, 3, 2, 3)])
def test_mttkrp_mm_matches_listing1_bruteforce(dims):
    """MTTKRP + MM, the running example of Sec. II-A (``ijk,ja,ka,al->il`` for order 3,
    mode 0), against the brute-force n-ary loop nest of Listing 1, in every mode."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 3)
    C = rng.standard_normal((3, 4))
    for mode in range(len(dims)):
        ops = [X] + [U[m] for m in range(len(dims)) if m != mode] + [C]
        spec = _mttkrp_spec(len(dims), mode)
        lhs, out = spec.split("->")
        ref = oracle.einsum_naive(lhs + ",rz->" + out[0] + "z", *ops)
        np.testing.assert_allclose(oracle.mttkrp_mm(X, U, mode, C), ref, rtol=1e-13, atol=1e-13)
    # a transposed C (square case) must not pass: the product is not symmetric in C
    Cs = rng.standard_normal((3, 3))
    got = oracle.mttkrp_mm(X, U, 0, Cs)
    assert not np.allclose(got, oracle.mttkrp_mm(X, U, 0, Cs.T))


@pytest.mark.parametrize("dims", [(6, 7, 5), (4, 5, 3, 6), (3, 4, 2, 3, 5)])
def test_mttkrp_matches_factored_krp_tdot(dims):
    rng = np.random.default_rng(2)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 5)
    for mode in range(len(dims)):
        np.testing.assert_allclose(oracle.mttkrp(X, U, mode), oracle.mttkrp_krp(X, U, mode),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(9, 8, 7), (5, 6, 4, 3)])
def test_mttkrp_matches_numpy_einsum(dims):
    rng = np.random.default_rng(3)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 4)
    for mode in range(len(dims)):
        ops = [X] + [U[m] for m in range(len(dims)) if m != mode]
        ref = np.einsum(_mttkrp_spec(len(dims), mode), *ops)
        np.testing.assert_allclose(oracle.mttkrp(X, U, mode), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(5, 6, 7), (3, 4, 5, 2, 3)])
def test_mttkrp_rank1_closed_form(dims):
    """X = u0 o u1 o ... gives M_n[i, r] = u_n[i] * prod_{m != n} (u_m . U_m[:, r])."""
    rng = np.random.default_rng(4)
    us = [rng.standard_normal(d) for d in dims]
    X = us[0]
    for u in us[1:]:
        X = np.multiply.outer(X, u)
    U = _factors(rng, dims, 6)
    for mode in range(len(dims)):
        coef = np.ones(6)
        for m in range(len(dims)):
            if m != mode:
                coef = coef * (us[m] @ U[m])
        ref = np.outer(us[mode], coef)
        np.testing.assert_allclose(oracle.mttkrp(X, U, mode), ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("dims,rank", [((6, 5, 4), 3), ((4, 3, 5, 3, 2), 4)])
def test_mttkrp_cp_closed_form(dims, rank):
    """X = sum_s prod_m A_m[:, s] gives M_n = A_n (Hadamard_{m != n} A_m^T U_m)."""
    rng = np.random.default_rng(5)
    A = [rng.standard_normal((d, rank)) for d in dims]
    X = np.zeros(dims)
    for s in range(rank):
        t = A[0][:, s]
        for m in range(1, len(dims)):
            t = np.multiply.outer(t, A[m][:, s])
        X += t
    U = _factors(rng, dims, 5)
    for mode in range(len(dims)):
        H = np.ones((rank, 5))
        for m in range(len(dims)):
            if m != mode:
                H = H * (A[m].T @ U[m])
        np.testing.assert_allclose(oracle.mttkrp(X, U, mode), A[mode] @ H, rtol=1e-11, atol=1e-11)


def test_mttkrp_mode_permutation_invariance():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((5, 6, 7))
    U = _factors(rng, X.shape, 4)
    m1 = oracle.mttkrp(X, U, 1)
    m0 = oracle.mttkrp(X.transpose(1, 0, 2), [U[1], U[0], U[2]], 0)
    np.testing.assert_allclose(m1, m0, rtol=1e-13, atol=1e-13)
    m2 = oracle.mttkrp(X, U, 2)
    m2p = oracle.mttkrp(X.transpose(2, 1, 0), [U[2], U[1], U[0]], 0)
    np.testing.assert_allclose(m2, m2p, rtol=1e-13, atol=1e-13)


def test_mttkrp_linearity():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((4, 5, 6))
    Y = rng.standard_normal((4, 5, 6))
    U = _factors(rng, X.shape, 3)
    for mode in range(3):
        lhs = oracle.mttkrp(2.5 * X - 0.75 * Y, U, mode)
        rhs = 2.5 * oracle.mttkrp(X, U, mode) - 0.75 * oracle.mttkrp(Y, U, mode)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_mttkrp_rows_equal_full_rows():
    rng = np.random.default_rng(8)
    dims = (5, 7, 6, 4)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 3)
    for mode in range(4):
        full = oracle.mttkrp(X, U, mode)
        rows = np.array([0, 2, dims[mode] - 1])
        slabs = np.stack([np.take(X, r, axis=mode).ravel() for r in rows])
        np.testing.assert_array_equal(oracle.mttkrp_rows(dims, mode, slabs, U), full[rows])


def test_golden_hand_worked_example():
    g = _read_golden("mttkrp_o3_2x2x2.txt")
    U = [g["U0"], g["U1"], g["U2"]]
    for mode in range(3):
        np.testing.assert_array_equal(oracle.mttkrp(g["X"], U, mode), g[f"M{mode}"])
    np.testing.assert_array_equal(oracle.ttmc(g["X"], U, 0), g["Y0"])


# ---------------------------------------------------------------------------
# TTMc
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(3, 4, 2), (2, 3, 2, 3)])
def test_ttmc_matches_listing1_bruteforce(dims):
    rng = np.random.default_rng(9)
    X = rng.standard_normal(dims)
    ranks = [2, 3, 2, 3][:len(dims)]
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    for keep in range(len(dims)):
        ops = [X] + [U[m] for m in range(len(dims)) if m != keep]
        ref = oracle.einsum_naive(_ttmc_spec(len(dims), keep), *ops)
        np.testing.assert_allclose(oracle.ttmc(X, U, keep), ref, rtol=1e-13, atol=1e-13)


def test_ttmc_matches_numpy_einsum():
    rng = np.random.default_rng(10)
    dims = (6, 5, 4, 7)
    X = rng.standard_normal(dims)
    U = [rng.standard_normal((d, 3)) for d in dims]
    for keep in range(4):
        ops = [X] + [U[m] for m in range(4) if m != keep]
        np.testing.assert_allclose(oracle.ttmc(X, U, keep),
                                   np.einsum(_ttmc_spec(4, keep), *ops), rtol=1e-12, atol=1e-12)


def test_ttmc_identity_returns_x():
    rng = np.random.default_rng(11)
    dims = (4, 5, 6, 3)
    X = rng.standard_normal(dims)
    U = [np.eye(d) for d in dims]
    for keep in range(4):
        np.testing.assert_array_equal(oracle.ttmc(X, U, keep), X)


def test_ttmc_rank1_closed_form():
    """X = a o b o c o d gives Y[i,b,c,d] = a_i (b^T U1)_b (c^T U2)_c (d^T U3)_d."""
    rng = np.random.default_rng(12)
    dims = (4, 5, 6, 7)
    us = [rng.standard_normal(d) for d in dims]
    X = us[0]
    for u in us[1:]:
        X = np.multiply.outer(X, u)
    U = [rng.standard_normal((d, 3)) for d in dims]
    ref = us[0]
    for m in range(1, 4):
        ref = np.multiply.outer(ref, us[m] @ U[m])
    np.testing.assert_allclose(oracle.ttmc(X, U, 0), ref, rtol=1e-11, atol=1e-12)


def test_mttkrp_is_ttmc_superdiagonal():
    """M_n[i_n, r] = Y_n[r, .., i_n, .., r] when every TTMc matrix is the MTTKRP factor."""
    rng = np.random.default_rng(13)
    dims = (4, 5, 3, 6)
    X = rng.standard_normal(dims)
    U = _factors(rng, dims, 3)
    for keep in range(4):
        Y = oracle.ttmc(X, U, keep)
        M = oracle.mttkrp(X, U, keep)
        for r in range(3):
            idx = tuple(slice(None) if m == keep else r for m in range(4))
            np.testing.assert_allclose(Y[idx], M[:, r], rtol=1e-12, atol=1e-12)


def test_ttmc_rows_equal_full_slices():
    rng = np.random.default_rng(14)
    dims = (5, 4, 6, 3)
    X = rng.standard_normal(dims)
    U = [rng.standard_normal((d, 2)) for d in dims]
    for keep in range(4):
        Y = oracle.ttmc(X, U, keep)
        rows = np.array([1, dims[keep] - 1])
        slabs = np.stack([np.take(X, r, axis=keep).ravel() for r in rows])
        got = oracle.ttmc_rows(dims, keep, slabs, U)
        for s, r in enumerate(rows):
            np.testing.assert_allclose(got[s], np.take(Y, r, axis=keep), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# CP-ALS reference
# ---------------------------------------------------------------------------

def test_cpals_recovers_noise_free_cp_tensor():
    rng = np.random.default_rng(15)
    dims, R = (12, 10, 11), 3
    A = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum("ir,jr,kr->ijk", *A)
    init = [a + 0.05 * rng.standard_normal(a.shape) for a in A]
    factors, lam, fits = oracle.cpals(X, init, 10)
    assert fits[-1] >= 0.9999
    assert all(b >= a - 1e-10 for a, b in zip(fits, fits[1:]))
    Xhat = np.einsum("r,ir,jr,kr->ijk", lam, *factors)
    assert oracle.rel_error(Xhat, X) < 1e-4


def test_cpals_fit_formula_matches_direct_residual():
    rng = np.random.default_rng(16)
    dims, R = (6, 5, 4), 2
    X = rng.standard_normal(dims)
    factors, lam, fits = oracle.cpals(X, [rng.standard_normal((d, R)) for d in dims], 2)
    Xhat = np.einsum("r,ir,jr,kr->ijk", lam, *factors)
    direct = 1.0 - np.linalg.norm(X - Xhat) / np.linalg.norm(X)
    assert abs(fits[-1] - direct) < 1e-10


# ---------------------------------------------------------------------------
# Seeded generator (shared by both sides; holds none of the method)
# ---------------------------------------------------------------------------

def test_generator_uniform_exact_and_deterministic():
    idx = np.arange(100000, dtype=np.uint64)
    a = inputs.uniform_f32(7, inputs.STREAM_X, idx)
    b = inputs.uniform_f32(7, inputs.STREAM_X, idx)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    k = (a.astype(np.float64) + 1.0) * 2.0 ** 23
    np.testing.assert_array_equal(k, np.round(k))
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01
    c = inputs.uniform_f32(8, inputs.STREAM_X, idx)
    assert np.mean(a == c) < 0.01


def test_generator_streams_and_noise_moments():
    z = inputs.noise_z(3, inputs.STREAM_NOISE, np.arange(200000, dtype=np.uint64))
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    n = inputs.normal_f64(3, inputs.STREAM_FACTOR, 200000)
    assert abs(n.mean()) < 0.01 and abs(n.var() - 1.0) < 0.02


def test_cp_values_match_einsum_reconstruction():
    rng_seed = 21
    dims = (5, 6, 7)
    A = [inputs.factor_normal(rng_seed, m, d, 3, stream_base=inputs.STREAM_CP) for m, d in enumerate(dims)]
    X = inputs.tensor_cp_f32(rng_seed, dims, A, 0.0)
    ref = np.einsum("ir,jr,kr->ijk", *A)
    np.testing.assert_allclose(X, ref, rtol=1e-6, atol=1e-6)
    Xn = inputs.tensor_cp_f32(rng_seed, dims, A, 1e-2)
    assert 0.001 < np.abs(Xn - X).mean() < 0.02
    for mode in range(3):
        for row in (0, dims[mode] - 1):
            np.testing.assert_array_equal(inputs.cp_slab(rng_seed, dims, A, 1e-2, mode, row),
                                          np.take(Xn, row, axis=mode))


def test_uniform_slab_matches_whole_tensor():
    dims = (4, 5, 6)
    X = inputs.tensor_uniform_f32(3, dims)
    for mode in range(3):
        np.testing.assert_array_equal(inputs.uniform_slab(3, dims, mode, 2), np.take(X, 2, axis=mode))


def test_cpals_perturbation_hook_is_neutral_and_linear():
    # the hook that the CP-ALS tolerance derivation uses: the identity changes nothing, and
    # a relative perturbation of size eps moves a well-conditioned sweep by O(eps)
    rng = np.random.default_rng(12)
    dims, R = (9, 8, 7), 3
    A = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum("ir,jr,kr->ijk", *A) + 1e-2 * rng.standard_normal(dims)
    init = [a + 0.3 * rng.standard_normal(a.shape) for a in A]
    f0, l0, fit0 = oracle.cpals(X, init, 2)
    f1, l1, fit1 = oracle.cpals(X, init, 2, perturb=lambda M, m, f: M)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    assert np.array_equal(l0, l1) and fit0 == fit1
    f2, l2, fit2 = oracle.cpals(X, init, 2, perturb=lambda M, m, f: M * (1.0 + 1e-7))
    # a uniform scale of M scales the unnormalised update, which the normalisation removes
    # from the factors and moves into lambda
    for a, b in zip(f0, f2):
        assert oracle.rel_error(b, a) <= 1e-12
    assert abs(oracle.rel_error(l2, l0) - 1e-7) <= 1e-9
