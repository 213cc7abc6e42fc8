"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
OpenMP over output rows) through ctypes and adds:

* ``einsum_naive`` -- the n-ary brute-force loop nest of Listing 1 (Sec. II),
  pure Python, for tiny inputs;
* ``mttkrp_mm`` -- the MTTKRP + MM running example of Sec. II-A (the MTTKRP,
  then one library matrix product);
* ``cpals`` -- the CP-ALS reference (Kolda & Bader, SIAM Review 2009, Sec. 3.4),
  plain numpy in float64 (the paper names CP decomposition only as the
  motivation of MTTKRP, Sec. I).

The compiled helper is rebuilt with gcc when it is missing or older than its
source; ``build()`` forces that step.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        for name in ("oracle_mttkrp", "oracle_mttkrp_krp"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int64, _dp,
                          ctypes.POINTER(_dp), _dp]
            f.restype = ctypes.c_int
        lib.oracle_mttkrp_rows.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_int64, _dp, ctypes.POINTER(_dp), _dp]
        lib.oracle_mttkrp_rows.restype = ctypes.c_int
        lib.oracle_ttmc.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _i64p, _dp,
                                    ctypes.POINTER(_dp), _dp]
        lib.oracle_ttmc.restype = ctypes.c_int
        lib.oracle_ttmc_rows.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _i64p, ctypes.c_int64,
                                         _dp, ctypes.POINTER(_dp), _dp]
        lib.oracle_ttmc_rows.restype = ctypes.c_int
        lib.oracle_frobenius.argtypes = [_dp, ctypes.c_int64]
        lib.oracle_frobenius.restype = ctypes.c_double
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _factor_array(factors, order, skip):
    keep = []
    arr = (_dp * order)()
    for m in range(order):
        if m == skip or factors[m] is None:
            arr[m] = ctypes.cast(None, _dp)
        else:
            f = _f64(factors[m])
            keep.append(f)
            arr[m] = _ptr(f)
    return arr, keep


def mttkrp(X, factors, mode: int) -> np.ndarray:
    """Mode-``mode`` MTTKRP of X (any dtype, widened to float64); ``factors[mode]`` is ignored."""
    X = _f64(X)
    order = X.ndim
    R = next(np.asarray(f).shape[1] for m, f in enumerate(factors) if m != mode)
    dims = np.array(X.shape, dtype=np.int64)
    arr, keep = _factor_array(factors, order, mode)
    M = np.zeros((X.shape[mode], R), dtype=np.float64)
    rc = _load().oracle_mttkrp(order, dims.ctypes.data_as(_i64p), mode, R, _ptr(X), arr, _ptr(M))
    if rc:
        raise ValueError(f"oracle_mttkrp failed ({rc})")
    return M


def mttkrp_krp(X, factors, mode: int) -> np.ndarray:
    """Same value by the factored KRP + tensor-dot form (small inputs only)."""
    X = _f64(X)
    order = X.ndim
    R = next(np.asarray(f).shape[1] for m, f in enumerate(factors) if m != mode)
    dims = np.array(X.shape, dtype=np.int64)
    arr, keep = _factor_array(factors, order, mode)
    M = np.zeros((X.shape[mode], R), dtype=np.float64)
    rc = _load().oracle_mttkrp_krp(order, dims.ctypes.data_as(_i64p), mode, R, _ptr(X), arr, _ptr(M))
    if rc:
        raise ValueError(f"oracle_mttkrp_krp failed ({rc})")
    return M


def mttkrp_rows(dims, mode: int, slabs, factors) -> np.ndarray:
    """MTTKRP rows from per-row slabs: ``slabs[s]`` is X with mode ``mode`` fixed to row s."""
    order = len(dims)
    slabs = _f64(slabs)
    n_rows = slabs.shape[0]
    R = next(np.asarray(f).shape[1] for m, f in enumerate(factors) if m != mode)
    d = np.array(dims, dtype=np.int64)
    arr, keep = _factor_array(factors, order, mode)
    out = np.zeros((n_rows, R), dtype=np.float64)
    rc = _load().oracle_mttkrp_rows(order, d.ctypes.data_as(_i64p), mode, R, n_rows,
                                    _ptr(slabs), arr, _ptr(out))
    if rc:
        raise ValueError(f"oracle_mttkrp_rows failed ({rc})")
    return out


def ttmc(X, factors, keep: int) -> np.ndarray:
    """TTMc of X keeping mode ``keep``: every other mode m is contracted with factors[m]."""
    X = _f64(X)
    order = X.ndim
    ranks = np.array([X.shape[m] if m == keep else np.asarray(factors[m]).shape[1]
                      for m in range(order)], dtype=np.int64)
    dims = np.array(X.shape, dtype=np.int64)
    arr, kp = _factor_array(factors, order, keep)
    Y = np.zeros(tuple(int(r) for r in ranks), dtype=np.float64)
    rc = _load().oracle_ttmc(order, dims.ctypes.data_as(_i64p), keep, ranks.ctypes.data_as(_i64p),
                             _ptr(X), arr, _ptr(Y))
    if rc:
        raise ValueError(f"oracle_ttmc failed ({rc})")
    return Y


def ttmc_rows(dims, keep: int, slabs, factors) -> np.ndarray:
    """TTMc keep-mode slices from per-row slabs; result[s] = Y[.., row s, ..] with that mode dropped."""
    order = len(dims)
    slabs = _f64(slabs)
    n_rows = slabs.shape[0]
    ranks = np.array([dims[m] if m == keep else np.asarray(factors[m]).shape[1]
                      for m in range(order)], dtype=np.int64)
    d = np.array(dims, dtype=np.int64)
    arr, kp = _factor_array(factors, order, keep)
    oshape = tuple(int(ranks[m]) for m in range(order) if m != keep)
    out = np.zeros((n_rows,) + oshape, dtype=np.float64)
    rc = _load().oracle_ttmc_rows(order, d.ctypes.data_as(_i64p), keep, ranks.ctypes.data_as(_i64p),
                                  n_rows, _ptr(slabs), arr, _ptr(out))
    if rc:
        raise ValueError(f"oracle_ttmc_rows failed ({rc})")
    return out


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's OpenMP loops (0: leave unchanged); returns the count in force."""
    return int(_load().oracle_set_threads(int(n)))


def frobenius(a) -> float:
    """Frobenius norm sqrt(sum a^2) of an array of any shape (oracle_frobenius, long double sum)."""
    a = _f64(a).ravel()
    return float(_load().oracle_frobenius(_ptr(a), a.size))


def rel_error(got, ref) -> float:
    """Relative Frobenius error ||got - ref|| / ||ref|| (absolute when ||ref|| = 0): the
    parity gate of every floating-point result against this oracle (the paper fixes the
    contraction, Sec. III-B, not a precision; this is the reading of "relative error")."""
    ref = _f64(ref)
    got = _f64(got)
    if got.shape != ref.shape:
        raise ValueError(f"shape mismatch {got.shape} vs {ref.shape}")
    diff = got - ref
    nr = frobenius(ref)
    nd = frobenius(diff)
    return nd / nr if nr > 0 else nd


def max_elem_error(got, ref) -> float:
    """Largest element-wise deviation max |got - ref| relative to the largest oracle entry
    max |ref| (absolute when ref is all zero; 0 for empty arrays): the element-wise backstop
    beside rel_error, so that one wrong entry cannot hide in a large Frobenius norm."""
    ref = _f64(ref)
    got = _f64(got)
    if ref.shape != got.shape:
        raise ValueError(f"shape mismatch {got.shape} vs {ref.shape}")
    if ref.size == 0:
        return 0.0
    worst = float(np.abs(got - ref).max())
    scale = float(np.abs(ref).max())
    return worst / scale if scale > 0 else worst


# ---------------------------------------------------------------------------
# Listing 1 (Sec. II): the n-ary loop nest, one loop per distinct index,
# accumulating the product of every operand into the output.  Pure Python.
# ---------------------------------------------------------------------------

def mttkrp_mm(X, factors, mode: int, C) -> np.ndarray:
    """MTTKRP followed by a matrix product, the running example of Sec. II-A
    (``ijk,ja,ka,al->il``): the mode-``mode`` MTTKRP of X, then times C (R x L),
    in float64; the product is a library matrix multiply of the two factors of
    the binary chain the section writes out (Listing 2: KRP, TDOT, then MM)."""
    return mttkrp(X, factors, mode) @ np.asarray(C, dtype=np.float64)


def einsum_naive(spec: str, *operands) -> np.ndarray:
    """Brute-force einsum ``spec`` ("ab,bc->ac" form, explicit output) over float64 operands."""
    lhs, out = spec.replace(" ", "").split("->")
    terms = lhs.split(",")
    if len(terms) != len(operands):
        raise ValueError("operand count does not match the index string")
    extent = {}
    for t, op in zip(terms, operands):
        op = np.asarray(op)
        if op.ndim != len(t):
            raise ValueError("operand rank does not match its index string")
        for c, n in zip(t, op.shape):
            if extent.setdefault(c, n) != n:
                raise ValueError(f"extent mismatch for index {c}")
    letters = []
    for t in terms + [out]:
        for c in t:
            if c not in letters:
                letters.append(c)
    ops = [np.asarray(o, dtype=np.float64) for o in operands]
    res = np.zeros(tuple(extent[c] for c in out), dtype=np.float64)
    for values in itertools.product(*[range(extent[c]) for c in letters]):
        env = dict(zip(letters, values))
        prod = 1.0
        for t, op in zip(terms, ops):
            prod = prod * float(op[tuple(env[c] for c in t)])
        res[tuple(env[c] for c in out)] += prod
    return res


# ---------------------------------------------------------------------------
# CP-ALS reference (Kolda & Bader 2009, Sec. 3.4, Fig. 3.3), float64 numpy.
# ---------------------------------------------------------------------------

def cpals_step(X, factors, lam, mode: int, perturb=None):
    """One ALS factor update of mode ``mode`` (Gauss-Seidel).

    V = Hadamard product of the Grams U_m^T U_m over m != mode; the update
    solves U_mode V = MTTKRP_mode(X) (V symmetric positive definite, by
    Cholesky), then normalises every column to unit 2-norm, the norms
    becoming lambda (a zero column keeps lambda = 0).
    ``perturb(M, mode, factors)``, if given, replaces the MTTKRP result before the
    solve (the tests use it to measure how errors in M propagate through a sweep).
    Returns the new factor list, lambda and the MTTKRP result used.
    """
    X = _f64(X)
    N = X.ndim
    R = factors[0].shape[1]
    V = np.ones((R, R), dtype=np.float64)
    for m in range(N):
        if m != mode:
            V = V * (factors[m].T @ factors[m])
    Mn = mttkrp(X, factors, mode)
    if perturb is not None:
        Mn = perturb(Mn, mode, factors)
    L = np.linalg.cholesky(V)
    Y = np.linalg.solve(L, Mn.T)
    Un = np.linalg.solve(L.T, Y).T
    lam = np.sqrt((Un * Un).sum(axis=0))
    safe = np.where(lam > 0, lam, 1.0)
    Un = Un / safe
    out = list(factors)
    out[mode] = Un
    return out, lam, Mn


def cp_fit(X, factors, lam, M_last=None, last_mode=None) -> float:
    """fit = 1 - ||X - [[lambda; U]]|| / ||X||, with the residual norm expanded as
    ||X||^2 + ||Xhat||^2 - 2 <X, Xhat> (Kolda & Bader, Sec. 3.4)."""
    X = _f64(X)
    N = X.ndim
    R = factors[0].shape[1]
    normX2 = float((X * X).sum())
    G = np.ones((R, R), dtype=np.float64)
    for m in range(N):
        G = G * (factors[m].T @ factors[m])
    normXhat2 = float(lam @ G @ lam)
    if M_last is None:
        last_mode = N - 1
        M_last = mttkrp(X, factors, last_mode)
    inner = float(((M_last * factors[last_mode]).sum(axis=0) * lam).sum())
    res2 = max(0.0, normX2 + normXhat2 - 2.0 * inner)
    return 1.0 - np.sqrt(res2) / np.sqrt(normX2)


def cpals(X, init_factors, sweeps: int, perturb=None):
    """``sweeps`` full ALS sweeps (modes 0..N-1 each); returns factors, lambda, fit history.
    ``perturb`` as in cpals_step (applied to every MTTKRP result)."""
    factors = [_f64(f).copy() for f in init_factors]
    N = len(factors)
    lam = np.ones(factors[0].shape[1])
    fits = []
    for _ in range(sweeps):
        for n in range(N):
            factors, lam, Mn = cpals_step(X, factors, lam, n, perturb)
        fits.append(cp_fit(X, factors, lam, Mn, N - 1))
    return factors, lam, fits
