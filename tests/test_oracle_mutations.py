"""The pins must catch plausible mistakes: plant each one in a copy of the oracle.

Each mutation edits one line of oracle.c (a dropped factor, a transposed
factor index, a wrong output row, a skipped term, a wrong TTM operand index),
compiles the copy with gcc into a temporary directory and checks that at least
one pin (hand-worked example, rank-1 closed form, numpy einsum) now fails.
The error metric that decides every parity test is mutated the same way: the
C norm (no square root, |a| instead of a^2, a skipped element, a wrong
operand) and the Python relative / element-wise errors (no division, the
wrong norm in the denominator, the zero-reference branch returning 0, a sum
instead of a difference, a mean instead of a maximum), each of which must
break a pin of tests/test_oracle_metric.py.
The real oracle is never modified.
"""
import ctypes
import inspect
import os
import subprocess
import textwrap

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)

MUTATIONS = {
    "dropped_factor": ("if (m != mode) term = term * U[m][idx[m] * R + r];",
                       "if (m != mode && m != order - 1) term = term * U[m][idx[m] * R + r];"),
    "transposed_factor": ("if (m != mode) term = term * U[m][idx[m] * R + r];",
                          "if (m != mode) term = term * U[m][(r % dims[m]) * R + idx[m] % R];"),
    "wrong_output_row": ("double *out = M + in * R;", "double *out = M + ((in + 1) % In) * R;"),
    "skipped_term": ("for (int64_t t = 0; t < rest; ++t) {\n            int64_t off = 0;",
                     "for (int64_t t = 1; t < rest; ++t) {\n            int64_t off = 0;"),
    "ttm_operand_index": ("const double u = U[i * Rm + r];", "const double u = U[r * Im + i % Rm];"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    lib.oracle_mttkrp.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int64, _dp,
                                  ctypes.POINTER(_dp), _dp]
    lib.oracle_ttmc.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _i64p, _dp,
                                ctypes.POINTER(_dp), _dp]
    lib.oracle_frobenius.argtypes = [_dp, ctypes.c_int64]
    lib.oracle_frobenius.restype = ctypes.c_double
    return lib


def _mttkrp(lib, X, U, mode):
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = U[(mode + 1) % X.ndim].shape[1]
    Us = [np.ascontiguousarray(u, dtype=np.float64) for u in U]
    arr = (_dp * X.ndim)(*[u.ctypes.data_as(_dp) for u in Us])
    M = np.zeros((X.shape[mode], R))
    dims = np.array(X.shape, dtype=np.int64)
    lib.oracle_mttkrp(X.ndim, dims.ctypes.data_as(_i64p), mode, R, X.ctypes.data_as(_dp), arr,
                      M.ctypes.data_as(_dp))
    return M


def _ttmc(lib, X, U, keep):
    X = np.ascontiguousarray(X, dtype=np.float64)
    Us = [np.ascontiguousarray(u, dtype=np.float64) for u in U]
    arr = (_dp * X.ndim)(*[u.ctypes.data_as(_dp) for u in Us])
    ranks = np.array([X.shape[m] if m == keep else U[m].shape[1] for m in range(X.ndim)], dtype=np.int64)
    Y = np.zeros(tuple(int(r) for r in ranks))
    dims = np.array(X.shape, dtype=np.int64)
    lib.oracle_ttmc(X.ndim, dims.ctypes.data_as(_i64p), keep, ranks.ctypes.data_as(_i64p),
                    X.ctypes.data_as(_dp), arr, Y.ctypes.data_as(_dp))
    return Y


def _pins_pass(lib):
    rng = np.random.default_rng(0)
    dims = (5, 6, 7)
    us = [rng.standard_normal(d) for d in dims]
    X1 = np.multiply.outer(np.multiply.outer(us[0], us[1]), us[2])
    U = [rng.standard_normal((d, 4)) for d in dims]
    for mode in range(3):
        coef = np.ones(4)
        for m in range(3):
            if m != mode:
                coef = coef * (us[m] @ U[m])
        if not np.allclose(_mttkrp(lib, X1, U, mode), np.outer(us[mode], coef), rtol=1e-10, atol=1e-12):
            return False
    X = rng.standard_normal(dims)
    V = [rng.standard_normal((d, 3)) for d in dims]
    if not np.allclose(_ttmc(lib, X, V, 0), np.einsum("ijk,jb,kc->ibc", X, V[1], V[2]), rtol=1e-10):
        return False
    return True


def test_unmutated_copy_passes(tmp_path):
    lib = _build(tmp_path, "identity", "#define ORACLE_MAX_ORDER 8", "#define ORACLE_MAX_ORDER 8")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    lib = _build(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"mutation {name} slipped through the pins"


# ---------------------------------------------------------------------------
# the error metric
# ---------------------------------------------------------------------------

from test_oracle_metric import metric_pins_hold  # noqa: E402

NORM_MUTATIONS = {
    "no_square_root": ("return (double)__builtin_sqrtl(s);", "return (double)s;"),
    "abs_instead_of_square": ("s += (long double)a[i] * (long double)a[i];", "s += (a[i] < 0 ? -a[i] : a[i]);"),
    "skipped_element": ("for (int64_t i = 0; i < n; ++i) s +=", "for (int64_t i = 1; i < n; ++i) s +="),
    "wrong_operand": ("s += (long double)a[i] * (long double)a[i];", "s += (long double)a[i] * (long double)a[0];"),
}

REL_MUTATIONS = {
    "no_division": ("return nd / nr if nr > 0 else nd", "return nd"),
    "wrong_denominator": ("nr = frobenius(ref)", "nr = frobenius(got)"),
    "zero_reference_gives_zero": ("return nd / nr if nr > 0 else nd", "return nd / nr if nr > 0 else 0.0"),
    "sum_not_difference": ("diff = got - ref", "diff = got + ref"),
    "squared_ratio": ("return nd / nr if nr > 0 else nd", "return (nd / nr) ** 2 if nr > 0 else nd"),
}

ELEM_MUTATIONS = {
    "mean_not_max": ("worst = float(np.abs(got - ref).max())", "worst = float(np.abs(got - ref).mean())"),
    "no_scale": ("return worst / scale if scale > 0 else worst", "return worst"),
    "signed_difference": ("worst = float(np.abs(got - ref).max())", "worst = float((got - ref).max())"),
}


def _norm_from(lib):
    def frob(a):
        a = np.ascontiguousarray(np.asarray(a), dtype=np.float64).ravel()
        return float(lib.oracle_frobenius(a.ctypes.data_as(_dp), a.size))
    return frob


def _mutated_python(func, old, new, namespace):
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, (func.__name__, old)
    ns = dict(namespace)
    exec(src.replace(old, new), ns)
    return ns[func.__name__]


def test_unmutated_norm_passes_metric_pins(tmp_path):
    lib = _build(tmp_path, "identity_norm", "#define ORACLE_MAX_ORDER 8", "#define ORACLE_MAX_ORDER 8")
    frob = _norm_from(lib)
    rel = _mutated_python(oracle.rel_error, "diff = got - ref", "diff = got - ref",
                          {"_f64": oracle._f64, "frobenius": frob, "np": np})
    assert metric_pins_hold(frob, rel, oracle.max_elem_error)


@pytest.mark.parametrize("name", sorted(NORM_MUTATIONS))
def test_planted_norm_mistake_is_caught(tmp_path, name):
    old, new = NORM_MUTATIONS[name]
    lib = _build(tmp_path, name, old, new)
    frob = _norm_from(lib)
    rel = _mutated_python(oracle.rel_error, "diff = got - ref", "diff = got - ref",
                          {"_f64": oracle._f64, "frobenius": frob, "np": np})
    assert not metric_pins_hold(frob, rel), f"norm mutation {name} slipped through the pins"


@pytest.mark.parametrize("name", sorted(REL_MUTATIONS))
def test_planted_rel_error_mistake_is_caught(name):
    old, new = REL_MUTATIONS[name]
    rel = _mutated_python(oracle.rel_error, old, new,
                          {"_f64": oracle._f64, "frobenius": oracle.frobenius, "np": np})
    assert not metric_pins_hold(oracle.frobenius, rel), f"rel_error mutation {name} slipped through"


@pytest.mark.parametrize("name", sorted(ELEM_MUTATIONS))
def test_planted_max_elem_error_mistake_is_caught(name):
    old, new = ELEM_MUTATIONS[name]
    elem = _mutated_python(oracle.max_elem_error, old, new, {"_f64": oracle._f64, "np": np})
    assert not metric_pins_hold(oracle.frobenius, oracle.rel_error, elem), \
        f"max_elem_error mutation {name} slipped through"
