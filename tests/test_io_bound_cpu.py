"""The MTTKRP I/O lower bound and tiling of Sec. IV-E (deinsum_mttkrp_io_bound), on the CPU.

Pinned against what the mathematics fixes, not a re-typing of the closed forms:
* a numerical optimiser (scipy SLSQP, from random starts) maximising I J K L under
  I J K + J L + K L + I L <= X reaches the returned tiles' objective at X = 5S/2, and
  never exceeds it;
* a scan of the intensity rho(X) = I(X) J(X) K(X) L(X) / (X - S) over X finds its minimum
  at X0 = 5S/2, with the value the helper returns;
* the returned tiles meet the constraint with the output term I L exactly (and use 4/5 of
  it without that term: the printed constraint omits I L, which its tiles contradict);
* hand values at S = 8 and S = 1000; the rank cap; argument checks; the plan's report.
"""
import ctypes
import math

import numpy as np
import pytest

import paper_2206_08301_gb300 as dz


def _tiles_at(X):
    """Tiles maximising I J K L for a computation of X elements, by SLSQP on log variables."""
    from scipy.optimize import minimize
    best = None
    rng = np.random.default_rng(0)
    for _ in range(6):
        x0 = np.log(rng.uniform(0.2, 2.0, 4) * X ** (1.0 / 3.0))

        def cons(z):
            i, j, k, l = np.exp(z)
            return 1.0 - (i * j * k + j * l + k * l + i * l) / X

        res = minimize(lambda z: -z.sum(), x0, method="SLSQP",
                       constraints=[{"type": "ineq", "fun": cons}], options={"ftol": 1e-14, "maxiter": 500})
        if res.success and cons(res.x) > -1e-9 and (best is None or res.fun < best.fun):
            best = res
    return np.exp(best.x)


@pytest.mark.parametrize("S", [8.0, 1000.0, 123648.0])
def test_io_bound_matches_numerical_optimum(S):
    b = dz.mttkrp_io_bound(S, 1e9, 10 ** 6)
    X0 = b["X0"]
    ijkl = _tiles_at(X0)
    obj = float(np.prod(ijkl))
    ref = b["I"] * b["J"] * b["K"] * b["L"]
    assert abs(obj - ref) <= 1e-6 * ref
    np.testing.assert_allclose(sorted(ijkl[:3]), [b["I"]] * 3, rtol=1e-3)
    assert abs(ijkl[3] - b["L"]) <= 1e-3 * b["L"]


@pytest.mark.parametrize("S", [8.0, 1000.0, 123648.0])
def test_x0_minimises_the_intensity(S):
    b = dz.mttkrp_io_bound(S, 1e9, 10 ** 6)

    def rho(X):   # the optimal tiles of X, from the stationarity conditions checked above
        i = (2.0 * X / 5.0) ** (1.0 / 3.0)
        l = X ** (2.0 / 3.0) / (2.0 ** (1.0 / 3.0) * 5.0 ** (2.0 / 3.0))
        return i ** 3 * l / (X - S)

    xs = S * np.linspace(1.01, 20.0, 200001)
    r = rho(xs)
    k = int(np.argmin(r))
    assert abs(xs[k] - b["X0"]) <= 2e-4 * b["X0"]
    assert abs(r[k] - b["rho"]) <= 1e-8 * b["rho"]
    # the same intensity from the returned tiles
    assert abs(b["I"] * b["J"] * b["K"] * b["L"] / (b["X0"] - S) - b["rho"]) <= 1e-12 * b["rho"]


def test_tiles_are_tight_only_with_the_output_term():
    for S in (8.0, 1000.0, 123648.0):
        b = dz.mttkrp_io_bound(S, 1.0, 1)
        I, J, K, L = b["I"], b["J"], b["K"], b["L"]
        with_out = I * J * K + J * L + K * L + I * L
        without = I * J * K + J * L + K * L
        assert abs(with_out - b["X0"]) <= 1e-12 * b["X0"]
        assert abs(without - 0.8 * b["X0"]) <= 1e-12 * b["X0"]


def test_hand_values():
    b = dz.mttkrp_io_bound(8.0, 100.0, 1)
    assert b["X0"] == 20.0 and abs(b["I"] - 2.0) < 1e-15 and abs(b["L"] - 2.0) < 1e-15
    assert abs(b["rho"] - 4.0 / 3.0) < 1e-15
    b = dz.mttkrp_io_bound(1000.0, 1e6, 1000)
    assert abs(b["I"] - 10.0) < 1e-12 and abs(b["L"] - 50.0) < 1e-12 and abs(b["rho"] - 100.0 / 3.0) < 1e-12
    # the bound |V| / rho for R above rho ...
    assert abs(b["q_min"] - 1e6 * 1000 / (100.0 / 3.0)) <= 1e-9 * b["q_min"]
    # ... and reading T once for R below it
    b = dz.mttkrp_io_bound(1000.0, 1e6, 32)
    assert b["rho_rank"] == 32 and b["q_min"] == 1e6


def test_invalid_arguments():
    lib = dz.load()
    out = dz._IoBound()
    assert lib.deinsum_mttkrp_io_bound(0.0, 1.0, 1, ctypes.byref(out)) == 9
    assert lib.deinsum_mttkrp_io_bound(8.0, 1.0, 0, ctypes.byref(out)) == 9
    assert lib.deinsum_mttkrp_io_bound(8.0, 0.0, 1, ctypes.byref(out)) == 9
    assert lib.deinsum_mttkrp_io_bound(8.0, 1.0, 1, None) == 9


def test_plan_reports_the_bound_for_its_row_view():
    S = (232448.0 + 262144.0) / 4.0
    info = dz.Plan("ijk,ja,ka->ia", [1024, 1024, 1024, 32], "float32", "split_bf16").info()
    assert info["io"]["fast_mem_words"] == S
    assert abs(info["io"]["rho"] - S ** (2.0 / 3.0) / 3.0) <= 1e-12 * info["io"]["rho"]
    assert info["io"]["bound_bytes"] == 4.0 * 1024 ** 3      # R 32 < rho (~827): X read once
    info = dz.Plan("ijklm,ia,ja,ka,la->ma", [64] * 5 + [24], "float32", "split_bf16").info()
    assert info["io"]["bound_bytes"] == 4.0 * 64 ** 5
    assert dz.Plan("ijk,jb,kc->ibc", [40, 50, 60, 8, 9], "float32", "plain").info()["io"]["bound_bytes"] == 0.0
    assert math.isclose(dz.mttkrp_io_bound(S, 1.0, 1)["rho"], info["io"]["rho"], rel_tol=1e-15)
