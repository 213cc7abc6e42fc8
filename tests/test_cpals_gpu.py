"""CP-ALS on the device against the FP64 CP-ALS reference (Kolda & Bader 2009, Sec. 3.4).

* per step: from the GPU's factors before a sweep, one GPU sweep and one oracle
  sweep give the same factors, lambda and fit within the sweep's derived
  tolerances (tests/cpals_bounds.py: the sweep's measured sensitivity to MTTKRP
  errors of the MTTKRP's own accuracy, times two; never tighter than 1e-5);
* every sweep of a multi-sweep run -- whose fits come from the expansion, the
  last one from the direct residual -- has the fit of one oracle sweep from the
  GPU's state before it, within the derived fit tolerance;
* end to end: 10 sweeps from the same start agree in fit (1e-4 absolute) and
  factors (1e-3 relative: the two trajectories drift apart by rounding);
* a noise-free rank-R tensor is recovered (fit >= 0.9999).
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs
from cpals_bounds import check_sweep, sweep_with_bounds

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


def _host(F):
    return [f.cpu().numpy().astype(np.float64) for f in F]


@pytest.mark.parametrize("prec", ["plain", "split_bf16"])
def test_cpals_per_step_parity(prec):
    dims, rank = (40, 50, 30), 6
    X, init = _problem(3, dims, rank, 1e-2)
    Xd = torch.from_numpy(X).cuda()
    F = [torch.from_numpy(u).cuda() for u in init]
    cp = dz.CPALS(dims, rank, prec)
    for sweep in range(4):
        before = _host(F)
        lam, fits = cp.run(Xd, F, 1)
        torch.cuda.synchronize()
        assert cp.status() == 0
        ref, tols = sweep_with_bounds(X, before, prec)
        check_sweep(_host(F), lam.cpu().numpy(), float(fits[0]), ref, tols, f"{prec} sweep {sweep}")


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


def test_cpals_recovers_noise_free_tensor_and_every_sweep_fit_matches():
    """The fits of one 10-sweep run (the expansion for sweeps 1-9, which near a perfect fit
    cancels, and the direct residual for the last) each equal the fit of one oracle sweep
    from the GPU's own state before that sweep, within the sweep's derived fit tolerance
    (about sqrt(2 d) near convergence, d the relative error of <X, Xhat>); the state before
    sweep S is the result of a GPU run of S sweeps, which is the same bit for bit."""
    dims, rank = (50, 40, 45), 5
    X, init = _problem(7, dims, rank, 0.0, init_scale=0.1)
    Xd = torch.from_numpy(X).cuda()
    cp = dz.CPALS(dims, rank, "split_bf16")
    F = [torch.from_numpy(u).cuda() for u in init]
    lam, fits = cp.run(Xd, F, 10)
    f = fits.cpu().numpy()
    assert f[-1] >= 0.9999
    for S in range(10):
        G = [torch.from_numpy(u).cuda() for u in init]
        if S:
            cp.run(Xd, G, S)
        torch.cuda.synchronize()
        (_, _, ref_fit), (_, _, tfit) = sweep_with_bounds(X, _host(G), "split_bf16")
        assert abs(f[S] - ref_fit) <= tfit, f"sweep {S}: fit {f[S]:.8f} vs {ref_fit:.8f} (tol {tfit:.2e})"


def test_cpals_order4_and_rank64():
    for seed, dims, rank, sweeps in ((9, (20, 24, 18, 22), 16, 2), (10, (70, 66, 80), 64, 1)):
        X, init = _problem(seed, dims, rank, 1e-2)
        Xd = torch.from_numpy(X).cuda()
        F = [torch.from_numpy(u).cuda() for u in init]
        cp = dz.CPALS(dims, rank, "split_bf16")
        for sweep in range(sweeps):
            before = _host(F)
            lam, fits = cp.run(Xd, F, 1)
            torch.cuda.synchronize()
            assert cp.status() == 0
            ref, tols = sweep_with_bounds(X, before, "split_bf16")
            check_sweep(_host(F), lam.cpu().numpy(), float(fits[0]), ref, tols, f"{dims} R {rank} sweep {sweep}")


@pytest.mark.parametrize("dims,rank", [((40, 50, 36), 6), ((130, 140, 72), 32), ((90, 30, 200), 17)])
def test_cpals_dimension_tree_per_step_parity(dims, rank):
    """Order 3, rank <= 32: modes 0 and 1 share T = X x_2 U_2 (one tensor-core pass).  Every
    sweep matches the FP64 reference from the same start within its derived tolerances,
    with the tree on and off."""
    X, init = _problem(11, dims, rank, 1e-2)
    Xd = torch.from_numpy(X).cuda()
    results = {}
    for tree in (True, False):
        F = [torch.from_numpy(u).cuda() for u in init]
        cp = dz.CPALS(dims, rank, "split_bf16")
        cp.set_dimension_tree(tree)
        assert cp.uses_dimension_tree == tree
        tf_all = 0.0
        for sweep in range(3):
            before = _host(F)
            lam, fits = cp.run(Xd, F, 1)
            torch.cuda.synchronize()
            assert cp.status() == 0
            ref, tols = sweep_with_bounds(X, before, "split_bf16")
            check_sweep(_host(F), lam.cpu().numpy(), float(fits[0]), ref, tols, f"tree {tree} sweep {sweep}")
        results[tree] = _host(F)
    # after three sweeps each run has drifted from the other by at most the sum of the
    # per-sweep tolerances; 1e-3 bounds that sum for these problems
    for m in range(3):
        assert oracle.rel_error(results[True][m], results[False][m]) <= 1e-3


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
