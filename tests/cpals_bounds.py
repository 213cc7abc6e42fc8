"""Derived tolerances of one device CP-ALS sweep against the FP64 reference.

A sweep (Kolda & Bader 2009, Sec. 3.4) carries any error of its MTTKRP results
into the factors and lambda through the Cholesky solve with V, the Hadamard
product of the Grams (amplified by up to about kappa(V)), and into the fit
through the expansion ||X||^2 + ||Xhat||^2 - 2 <X, Xhat>, which cancels as the
residual shrinks (near a perfect fit an error d in <X, Xhat> / ||X||^2 moves the
fit by about sqrt(2 d)).  Rather than a fixed tolerance, the bound of a sweep
from a given state is measured on the FP64 side, under two models of the
device's MTTKRP errors, and the larger effect counts:

* random output errors: every MTTKRP result M becomes M + E, ||E||_F = eps ||M||_F
  (E Gaussian), eps the MTTKRP's gate (1e-5 for split BF16, 1e-6 for the FP32
  CUDA-core kernel: the errors of long FP32 sums);
* split-BF16 input rounding (split precision only): X and every factor are
  multiplied element-wise by 1 + eta, |eta| <= 2^-16 uniform -- the bound on
  |x - hi - lo| for hi = bf16(x), lo = bf16(x - hi), bf16 having an 8-bit
  significand -- before the MTTKRP, plus random output errors of 1e-6 for the
  FP32 accumulation.  These errors lie in the range of the MTTKRP operator, so
  they move the fit more than random directions of the same size do.

Each model is drawn three times; the device sweep must agree with the
unperturbed reference within twice the largest change seen (never tighter than
1e-5 for factors and lambda), the fit within twice the largest fit change plus
1e-6 (the FP32 partial sums of ||X||^2 and <X, Xhat> on the device).
Element-wise, factors must agree within ten times their Frobenius bound,
relative to the largest reference entry.
"""
import numpy as np

import oracle

EPS = {"split_bf16": 1e-5, "plain": 1e-6}
SPLIT_ETA = 2.0 ** -16


def _random_output_errors(rng, eps):
    def perturb(M, mode, factors):
        E = rng.standard_normal(M.shape)
        return M + E * (eps * np.linalg.norm(M) / np.linalg.norm(E))
    return perturb


def _split_input_rounding(rng, X):
    Xp = np.asarray(X, dtype=np.float64) * (1.0 + rng.uniform(-SPLIT_ETA, SPLIT_ETA, np.shape(X)))

    def perturb(M, mode, factors):
        Fp = [f * (1.0 + rng.uniform(-SPLIT_ETA, SPLIT_ETA, f.shape)) for f in factors]
        Mp = oracle.mttkrp(Xp, Fp, mode)
        E = rng.standard_normal(M.shape)
        return Mp + E * (1e-6 * np.linalg.norm(M) / np.linalg.norm(E))
    return perturb


def sweep_with_bounds(X, before, prec, draws=3, seed=0):
    """One FP64 sweep from `before` and its derived tolerances:
    returns (factors, lambda, fit), (tol_factor, tol_lambda, tol_fit)."""
    ref_f, ref_lam, ref_fits = oracle.cpals(X, before, 1)
    rng = np.random.default_rng(seed)
    models = [lambda: _random_output_errors(rng, EPS[prec])]
    if prec == "split_bf16":
        models.append(lambda: _split_input_rounding(rng, X))
    df = dl = dfit = 0.0
    for make in models:
        for _ in range(draws):
            f, lam, fits = oracle.cpals(X, before, 1, perturb=make())
            df = max(df, max(oracle.rel_error(a, b) for a, b in zip(f, ref_f)))
            dl = max(dl, oracle.rel_error(lam, ref_lam))
            dfit = max(dfit, abs(fits[0] - ref_fits[0]))
    tols = (max(1e-5, 2.0 * df), max(1e-5, 2.0 * dl), 2.0 * dfit + 1e-6)
    return (ref_f, ref_lam, ref_fits[0]), tols


def check_sweep(got_factors, got_lam, got_fit, ref, tols, what=""):
    (ref_f, ref_lam, ref_fit), (tf, tl, tfit) = ref, tols
    for m, (g, r) in enumerate(zip(got_factors, ref_f)):
        err = oracle.rel_error(g, r)
        assert err <= tf, f"{what} factor {m}: {err:.2e} > {tf:.2e}"
        worst = oracle.max_elem_error(g, r)
        assert worst <= 10 * tf, f"{what} factor {m} element-wise: {worst:.2e} > {10 * tf:.2e}"
    err = oracle.rel_error(got_lam, ref_lam)
    assert err <= tl, f"{what} lambda: {err:.2e} > {tl:.2e}"
    assert abs(got_fit - ref_fit) <= tfit, f"{what} fit {got_fit:.8f} vs {ref_fit:.8f} (tol {tfit:.2e})"
