"""CP-ALS on the device against the FP64 CP-ALS reference (Kolda & Bader 2009, Sec. 3.4).

* per step: from the GPU's factors before a sweep, one GPU sweep and one oracle
  sweep give the same factors, lambda and fit (1e-5 with the plain FP32 MTTKRP,
  1e-4 with split BF16, relative Frobenius);
* end to end: 10 sweeps from the same start agree in fit (1e-4 absolute) and
  factors (1e-3 relative);
* a noise-free rank-R tensor is recovered (fit >= 0.9999) and the fit never decreases
  beyond rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402


def _problem(seed, dims, rank, sigma, init_scale=None):
    A = [inputs.factor_normal(seed, m, d, rank, stream_base=inputs.STREAM_CP) for m, d in enumerate(dims)]
    X = inputs.tensor_cp_f32(seed, dims, A, sigma)
    if init_scale is None:
        init = [inputs.factor_normal(seed, m, d, rank, stream_base=inputs.STREAM_INIT).astype(np.float32)
                for m, d in enumerate(dims)]
    else:
        init = [(a + init_scale * inputs.factor_normal(seed, m, d, rank, stream_base=inputs.STREAM_INIT))
                .astype(np.float32) for m, (a, d) in enumerate(zip(A, dims))]
    return X, init


@pytest.mark.parametrize("prec,tol", [("plain", 1e-5), ("split_bf16", 1e-4)])
def test_cpals_per_step_parity(prec, tol):
    dims, rank = (40, 50, 30), 6
    X, init = _problem(3, dims, rank, 1e-2)
    Xd = torch.from_numpy(X).cuda()
    F = [torch.from_numpy(u).cuda() for u in init]
    cp = dz.CPALS(dims, rank, prec)
    for sweep in range(4):
        before = [f.cpu().numpy().astype(np.float64) for f in F]
        lam, fits = cp.run(Xd, F, 1)
        torch.cuda.synchronize()
        assert cp.status() == 0
        ref_f, ref_lam, ref_fits = oracle.cpals(X, before, 1)
        for m in range(3):
            err = oracle.rel_error(F[m].cpu().numpy(), ref_f[m])
            assert err <= tol, f"sweep {sweep} factor {m}: {err:.2e}"
        assert oracle.rel_error(lam.cpu().numpy(), ref_lam) <= tol
        assert abs(float(fits[0]) - ref_fits[0]) <= tol


def test_cpals_end_to_end_10_sweeps():
    dims, rank = (64, 48, 56), 8
    X, init = _problem(5, dims, rank, 1e-2)
    Xd = torch.from_numpy(X).cuda()
    F = [torch.from_numpy(u).cuda() for u in init]
    cp = dz.CPALS(dims, rank, "split_bf16")
    lam, fits = cp.run(Xd, F, 10)
    torch.cuda.synchronize()
    ref_f, ref_lam, ref_fits = oracle.cpals(X, [u.astype(np.float64) for u in init], 10)
    assert abs(float(fits[-1]) - ref_fits[-1]) <= 1e-4
    for m in range(3):
        assert oracle.rel_error(F[m].cpu().numpy(), ref_f[m]) <= 1e-3
    assert oracle.rel_error(lam.cpu().numpy(), ref_lam) <= 1e-3


def test_cpals_recovers_noise_free_tensor_and_fit_is_monotone():
    dims, rank = (50, 40, 45), 5
    X, init = _problem(7, dims, rank, 0.0, init_scale=0.1)
    Xd = torch.from_numpy(X).cuda()
    F = [torch.from_numpy(u).cuda() for u in init]
    lam, fits = dz.CPALS(dims, rank, "split_bf16").run(Xd, F, 10)
    f = fits.cpu().numpy()
    # the final fit comes from the residual itself (accurate to ~1e-7 here); the
    # earlier ones from the expansion ||X||^2 + ||Xhat||^2 - 2<X, Xhat>, which near
    # convergence carries the FP32-level MTTKRP error (a few 1e-4 absolute)
    assert f[-1] >= 0.9999
    assert np.all(np.diff(f[:-1]) >= -1e-3)


def test_cpals_order4_and_rank64():
    dims, rank = (20, 24, 18, 22), 16
    X, init = _problem(9, dims, rank, 1e-2)
    F = [torch.from_numpy(u).cuda() for u in init]
    dz.CPALS(dims, rank, "split_bf16").run(torch.from_numpy(X).cuda(), F, 2)
    ref_f, _, _ = oracle.cpals(X, [u.astype(np.float64) for u in init], 2)
    for m in range(4):
        assert oracle.rel_error(F[m].cpu().numpy(), ref_f[m]) <= 1e-3
    dims, rank = (70, 66, 80), 64
    X, init = _problem(10, dims, rank, 1e-2)
    F = [torch.from_numpy(u).cuda() for u in init]
    lam, fits = dz.CPALS(dims, rank, "split_bf16").run(torch.from_numpy(X).cuda(), F, 1)
    ref_f, ref_lam, ref_fits = oracle.cpals(X, [u.astype(np.float64) for u in init], 1)
    assert abs(float(fits[0]) - ref_fits[0]) <= 1e-4


@pytest.mark.parametrize("dims,rank", [((40, 50, 36), 6), ((130, 140, 72), 32), ((90, 30, 200), 17)])
def test_cpals_dimension_tree_per_step_parity(dims, rank):
    """Order 3, rank <= 32: modes 0 and 1 share T = X x_2 U_2 (one tensor-core pass).  Every
    sweep matches the FP64 reference from the same start, with the tree on and off."""
    X, init = _problem(11, dims, rank, 1e-2)
    Xd = torch.from_numpy(X).cuda()
    results = {}
    for tree in (True, False):
        F = [torch.from_numpy(u).cuda() for u in init]
        cp = dz.CPALS(dims, rank, "split_bf16")
        cp.set_dimension_tree(tree)
        assert cp.uses_dimension_tree == tree
        for sweep in range(3):
            before = [f.cpu().numpy().astype(np.float64) for f in F]
            lam, fits = cp.run(Xd, F, 1)
            torch.cuda.synchronize()
            assert cp.status() == 0
            ref_f, ref_lam, ref_fits = oracle.cpals(X, before, 1)
            for m in range(3):
                err = oracle.rel_error(F[m].cpu().numpy(), ref_f[m])
                assert err <= 1e-4, f"tree {tree} sweep {sweep} factor {m}: {err:.2e}"
            assert abs(float(fits[0]) - ref_fits[0]) <= 1e-4
        results[tree] = [f.cpu().numpy().astype(np.float64) for f in F]
    for m in range(3):
        assert oracle.rel_error(results[True][m], results[False][m]) <= 1e-4


def test_cpals_dimension_tree_only_where_it_applies():
    assert dz.CPALS((40, 50, 36), 8, "split_bf16").uses_dimension_tree
    assert not dz.CPALS((40, 50, 30), 8, "split_bf16").uses_dimension_tree     # I_2 % 4 != 0
    assert not dz.CPALS((40, 50, 36), 40, "split_bf16").uses_dimension_tree    # rank > 32
    assert not dz.CPALS((40, 50, 36), 8, "plain").uses_dimension_tree
    assert not dz.CPALS((20, 24, 18, 22), 8, "split_bf16").uses_dimension_tree  # order 4


def test_cpals_final_fit_from_the_expansion_when_the_residual_is_large():
    """With heavy noise the final residual is large, so the final fit comes from the
    expansion rather than a second pass over X; it must still equal the FP64 direct
    residual of the GPU's own final factors within 1e-4."""
    dims, rank = (48, 40, 36), 5
    X, init = _problem(7, dims, rank, 1.0)
    Xd = torch.from_numpy(X).cuda()
    F = [torch.from_numpy(u).cuda() for u in init]
    cp = dz.CPALS(dims, rank, "split_bf16")
    lam, fits = cp.run(Xd, F, 6)
    torch.cuda.synchronize()
    assert cp.status() == 0
    U = [f.cpu().numpy().astype(np.float64) for f in F]
    lamh = lam.cpu().numpy()
    Xhat = np.einsum("r,ir,jr,kr->ijk", lamh, *U)
    x64 = X.astype(np.float64)
    direct = 1.0 - np.linalg.norm(x64 - Xhat) / np.linalg.norm(x64)
    assert direct < 0.9, f"the residual should be large here (fit {direct:.4f})"
    assert abs(float(fits[-1]) - direct) <= 1e-4
