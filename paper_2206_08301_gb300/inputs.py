"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle harness.

This module holds no MTTKRP or TTMc arithmetic.  It defines one counter-based
random generator and the synthetic tensors built from it, so that any element
of any input can be regenerated by index on the host (for sampled oracle
checks) and on the device (by the CUDA generator kernels, which implement the
same definitions and are checked bit for bit against this module).

Generator
---------
SplitMix64 (S. Vigna, the ``splitmix64.c`` public-domain generator, also
described by Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state advances by the golden-ratio increment
``GAMMA`` and every output is the 64-bit finaliser ``mix64`` of the state.

* ``state0(seed, stream) = mix64(seed + stream * GAMMA)``            (mod 2^64)
* ``raw(seed, stream, i) = mix64(state0 + (i + 1) * GAMMA)``         (mod 2^64)

i.e. element ``i`` of a stream is the (i+1)-th output of a SplitMix64
generator seeded with ``state0``.

Derived draws (all exact in the stated precision, so host and device agree
bit for bit):

* ``uniform_f32``: ``(raw >> 40) * 2^-23 - 1``  in [-1, 1) (24 random bits).
* ``uniform_f64``: ``(raw >> 11) * 2^-52 - 1``  in [-1, 1) (53 random bits).
* ``noise_z``: ``(sum_{t<4} ((raw >> 16 t) & 0xFFFF) - 2^17) * (sqrt(3) * 2^-16)``,
  an Irwin-Hall sum of the four 16-bit lanes of one draw, scaled to mean 0 and
  variance 1 (a bell-shaped stand-in for N(0, 1)); the integer sum is exact and
  the scale is one fixed float64 constant, so host and device agree.
* ``normal_f64`` (host only): Box-Muller on ``raw(2 i)`` and ``raw(2 i + 1)``.
  It goes through ``log``/``cos``, so it is used only for small operands
  (factor matrices) that are generated on the host and uploaded.

Synthetic CP tensor
-------------------
``X[idx] = sum_s prod_m a_m[i_m, s]  +  f32(sigma) * f32(noise_z(idx))``
evaluated in float32 (a_m = the generating factors rounded to float32) with
every multiply and add rounded to nearest: the product over m = 0..N-1 left
to right, the sum over s = 0..R-1 left to right, no fused multiply-add.
numpy evaluates it with separate float32 multiplies and adds, and the device
kernel uses explicitly rounded float32 operations in the same order.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers: one independent stream per role of a workload.
STREAM_X = 1          # the dense input tensor X
STREAM_NOISE = 2      # additive noise of a CP tensor
STREAM_FACTOR = 16    # factor matrix m uses STREAM_FACTOR + m
STREAM_CP = 64        # CP generating factor m uses STREAM_CP + m
STREAM_INIT = 128     # CP-ALS initial factor m uses STREAM_INIT + m
STREAM_SAMPLE = 250   # choice of sampled output rows
STREAM_DRAW = 251     # workload parameters (extents, ranks, modes)


def mix64(z):
    """SplitMix64 output finaliser (Vigna's constants), on uint64 numpy arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def state0(seed: int, stream: int) -> np.uint64:
    """Initial SplitMix64 state of ``stream`` under ``seed``."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream) * GAMMA
    return np.uint64(mix64(np.array([s], dtype=np.uint64))[0])


def raw(seed: int, stream: int, idx) -> np.ndarray:
    """64-bit draws for element indices ``idx`` (array-like of non-negative ints)."""
    idx = np.asarray(idx, dtype=np.uint64)
    s0 = state0(seed, stream)
    with np.errstate(over="ignore"):
        st = s0 + (idx + np.uint64(1)) * GAMMA
    return mix64(st)


def uniform_f32(seed: int, stream: int, idx) -> np.ndarray:
    """float32 uniform on [-1, 1) for element indices ``idx`` (exact)."""
    u = (raw(seed, stream, idx) >> np.uint64(40)).astype(np.float64)
    return (u * 2.0 ** -23 - 1.0).astype(np.float32)


def uniform_f64(seed: int, stream: int, idx) -> np.ndarray:
    """float64 uniform on [-1, 1) for element indices ``idx`` (exact)."""
    u = (raw(seed, stream, idx) >> np.uint64(11)).astype(np.float64)
    return u * 2.0 ** -52 - 1.0


NOISE_SCALE = float(np.sqrt(3.0) * 2.0 ** -16)


def noise_z(seed: int, stream: int, idx) -> np.ndarray:
    """Approximate N(0,1) draw: Irwin-Hall sum of the four 16-bit lanes of one raw draw.

    The lane sum is an exact integer below 2^18; it is centred and scaled by
    the float64 constant NOISE_SCALE = sqrt(3) * 2^-16 (variance 1).
    """
    r = raw(seed, stream, idx)
    mask = np.uint64(0xFFFF)
    s = (r & mask) + ((r >> np.uint64(16)) & mask) + ((r >> np.uint64(32)) & mask) + (r >> np.uint64(48))
    return (s.astype(np.int64) - (1 << 17)).astype(np.float64) * NOISE_SCALE


def normal_f64(seed: int, stream: int, n: int, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    """Host-only N(mu, sigma^2) draws by Box-Muller (one draw per pair of raws)."""
    i = np.arange(n, dtype=np.uint64)
    r1 = raw(seed, stream, i * np.uint64(2))
    r2 = raw(seed, stream, i * np.uint64(2) + np.uint64(1))
    u1 = ((r1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (r2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return mu + sigma * (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


# ---------------------------------------------------------------------------
# Whole operands
# ---------------------------------------------------------------------------

def tensor_uniform_f32(seed: int, dims, stream: int = STREAM_X) -> np.ndarray:
    """Dense row-major float32 tensor of shape ``dims`` with uniform[-1,1) entries."""
    n = int(np.prod(dims, dtype=np.int64))
    return uniform_f32(seed, stream, np.arange(n, dtype=np.uint64)).reshape(dims)


def tensor_uniform_f64(seed: int, dims, stream: int = STREAM_X) -> np.ndarray:
    n = int(np.prod(dims, dtype=np.int64))
    return uniform_f64(seed, stream, np.arange(n, dtype=np.uint64)).reshape(dims)


def factor_normal(seed: int, m: int, rows: int, cols: int, sigma: float = 1.0,
                  stream_base: int = STREAM_FACTOR) -> np.ndarray:
    """Factor matrix (rows x cols, row-major) with N(0, sigma^2) entries, float64."""
    return normal_f64(seed, stream_base + m, rows * cols, 0.0, sigma).reshape(rows, cols)


def flat_index(dims, coords) -> np.ndarray:
    """Row-major flat index of integer coordinate arrays ``coords`` (one per mode)."""
    flat = np.zeros(np.broadcast(*coords).shape, dtype=np.uint64)
    for d, c in zip(dims, coords):
        flat = flat * np.uint64(d) + np.asarray(c, dtype=np.uint64)
    return flat


def cp_values(dims, cp_factors, sigma: float, seed: int, coords) -> np.ndarray:
    """Entries of the synthetic CP-plus-noise tensor at coordinate arrays ``coords``.

    ``cp_factors[m]`` is the generating factor of mode m (I_m x Rc), rounded to
    float32.  Evaluated exactly as the module docstring states.
    """
    A = [np.asarray(f, dtype=np.float32) for f in cp_factors]
    shape = np.broadcast(*coords).shape
    rc = A[0].shape[1]
    acc = np.zeros(shape, dtype=np.float32)
    for s in range(rc):
        term = A[0][np.asarray(coords[0]), s]
        for m in range(1, len(dims)):
            term = term * A[m][np.asarray(coords[m]), s]
        acc = acc + term
    if sigma != 0.0:
        z = noise_z(seed, STREAM_NOISE, flat_index(dims, coords)).astype(np.float32)
        acc = acc + np.float32(sigma) * z
    return acc.astype(np.float32)


def cp_slab(seed: int, dims, cp_factors, sigma: float, mode: int, row: int) -> np.ndarray:
    """Slab X[.., row, ..] (mode ``mode`` fixed) of the CP-plus-noise tensor, float32.

    Same values, bit for bit, as ``cp_values`` on the slab's coordinates: the
    product over modes is still formed left to right in mode order (the fixed
    index enters as a scalar at its position) and the sum over s left to right.
    """
    A = [np.asarray(f, dtype=np.float32) for f in cp_factors]
    order = len(dims)
    rc = A[0].shape[1]
    shape = tuple(d for m, d in enumerate(dims) if m != mode)
    acc = np.zeros(shape, dtype=np.float32)
    for s in range(rc):
        term = None
        for m in range(order):
            if m == mode:
                v = A[m][row, s]
                term = np.float32(v) if term is None else term * v
            else:
                col = A[m][:, s]
                term = col.copy() if term is None else np.multiply.outer(term, col)
        acc = acc + term
    if sigma != 0.0:
        coords = np.meshgrid(*[np.arange(d) if m != mode else np.array([row]) for m, d in enumerate(dims)],
                             indexing="ij", sparse=True)
        flat = flat_index(dims, coords).reshape(shape)
        acc = acc + np.float32(sigma) * noise_z(seed, STREAM_NOISE, flat).astype(np.float32)
    return acc.astype(np.float32)


def uniform_slab(seed: int, dims, mode: int, row: int, stream: int = STREAM_X) -> np.ndarray:
    """Slab X[.., row, ..] of the uniform float32 tensor, regenerated by index."""
    coords = np.meshgrid(*[np.arange(d) if m != mode else np.array([row]) for m, d in enumerate(dims)],
                         indexing="ij", sparse=True)
    shape = tuple(d for m, d in enumerate(dims) if m != mode)
    return uniform_f32(seed, stream, flat_index(dims, coords).reshape(shape))


def tensor_cp_f32(seed: int, dims, cp_factors, sigma: float) -> np.ndarray:
    """Whole CP-plus-noise tensor (small shapes only: it is built on the host)."""
    coords = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    return cp_values(dims, cp_factors, sigma, seed, coords)


def sample_rows(seed: int, extent: int, count: int, tag: int = 0) -> np.ndarray:
    """``count`` distinct output rows out of ``extent``, chosen from the seed, sorted."""
    count = min(count, extent)
    keys = raw(seed, STREAM_SAMPLE + tag, np.arange(extent, dtype=np.uint64))
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


def draw_int(seed: int, tag: int, lo: int, hi: int, n: int) -> np.ndarray:
    """``n`` integers uniform on [lo, hi] (inclusive), from the workload-parameter stream."""
    r = raw(seed, STREAM_DRAW + tag, np.arange(n, dtype=np.uint64))
    span = np.uint64(hi - lo + 1)
    return (r % span).astype(np.int64) + lo
