"""GB300 (sm_103a) MTTKRP / TTMc library -- Python binding of ``libdeinsum.so``.

A thin ctypes layer over the C ABI declared in ``include/deinsum.h``: it
marshals torch CUDA tensors into device pointers and streams and returns
status codes as exceptions.  Every step of the computation runs in the
library's CUDA kernels; there is no host or PyTorch fallback, and importing a
compute entry point without the built library raises.

Entry points mirror the C names: ``Plan`` (deinsum_plan / deinsum_execute /
deinsum_plan_info / deinsum_workspace_size / deinsum_last_device_status /
deinsum_destroy), ``gen_uniform`` / ``gen_cp`` (the seeded device generators),
``kernel_launch_count`` / ``alloc_count`` / ``set_wait_limit_ns`` and
``mttkrp_noalloc`` / ``mttkrp_noalloc_status``; ``mttkrp`` / ``ttmc`` build the einsum string of
the paper's Table IV pattern for a given tensor and factor list.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["DeinsumError", "Plan", "mttkrp", "ttmc", "mttkrp_einsum", "ttmc_einsum", "mttkrp_mm",
           "mttkrp_mm_einsum",
           "gen_uniform", "gen_cp", "kernel_launch_count", "alloc_count", "set_wait_limit_ns",
           "mttkrp_noalloc", "mttkrp_noalloc_status", "mttkrp_io_bound", "library_path", "load",
           "Grid", "redist_dim_partitions", "redist_match", "redist_plan"]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libdeinsum.so")
_lib = None
_lock = threading.Lock()

STATUS = {0: "ok", 1: "parse", 2: "unsupported", 3: "shape", 4: "dtype", 5: "align", 6: "oom",
          7: "cuda", 8: "timeout", 9: "invalid"}
DTYPES = {"float32": 0, "f32": 0, "float64": 1, "f64": 1}
PRECS = {"plain": 0, "split_bf16": 1}
KINDS = {0: "mttkrp", 1: "ttmc"}


class DeinsumError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS.get(status, str(status))
        msg = _lib.deinsum_status_string(status).decode() if _lib is not None else name
        super().__init__(f"{what}: {name} ({msg})" if what else f"{name} ({msg})")


class _PlanInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order", ctypes.c_int), ("mode", ctypes.c_int),
                ("dtype", ctypes.c_int), ("prec", ctypes.c_int),
                ("dims", ctypes.c_int64 * 8), ("ranks", ctypes.c_int64 * 8),
                ("out_elems", ctypes.c_int64), ("alg_bytes", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("n_units", ctypes.c_int64), ("mm_cols", ctypes.c_int64),
                ("view_merged", ctypes.c_int), ("view_packed", ctypes.c_int), ("view_groups", ctypes.c_int64),
                ("view_aligned_rows", ctypes.c_int), ("view_row_classes", ctypes.c_int),
                ("io_fast_mem_words", ctypes.c_double), ("io_rho", ctypes.c_double),
                ("io_bound_bytes", ctypes.c_double)]


class _IoBound(ctypes.Structure):
    _fields_ = [("X0", ctypes.c_double), ("I", ctypes.c_double), ("J", ctypes.c_double), ("K", ctypes.c_double),
                ("L", ctypes.c_double), ("rho", ctypes.c_double), ("rho_rank", ctypes.c_double),
                ("q_min", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("dims", ctypes.c_int64 * 8), ("rank", ctypes.c_int),
                ("sweeps", ctypes.c_int), ("seed", ctypes.c_uint64), ("cp_rank", ctypes.c_int),
                ("noise", ctypes.c_double), ("cp_factors", ctypes.POINTER(ctypes.c_void_p)),
                ("init_factors", ctypes.POINTER(ctypes.c_void_p)), ("arrival_s", ctypes.c_double),
                ("want_factors", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("arrival_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("gen_ms", ctypes.c_double),
                ("sweeps", ctypes.c_int), ("fit", ctypes.c_double)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load ``libdeinsum.so`` (built in-tree by ``build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is not built; run paper_2206_08301_gb300.build.build() "
                              "(or __graft_entry__.build()) first -- there is no fallback path")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.deinsum_plan.argtypes = [ctypes.c_char_p, ctypes.POINTER(i64), i32, i32, i32, ctypes.POINTER(vp)]
        lib.deinsum_plan.restype = i32
        lib.deinsum_execute.argtypes = [vp, ctypes.POINTER(vp), i32, vp, vp]
        lib.deinsum_execute.restype = i32
        lib.deinsum_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.deinsum_workspace_size.restype = i32
        lib.deinsum_plan_info.argtypes = [vp, ctypes.POINTER(_PlanInfo)]
        lib.deinsum_plan_info.restype = i32
        lib.deinsum_last_device_status.argtypes = [vp]
        lib.deinsum_last_device_status.restype = i32
        lib.deinsum_destroy.argtypes = [vp]
        lib.deinsum_destroy.restype = None
        lib.deinsum_status_string.argtypes = [i32]
        lib.deinsum_status_string.restype = ctypes.c_char_p
        lib.deinsum_kernel_launch_count.argtypes = []
        lib.deinsum_kernel_launch_count.restype = i64
        lib.deinsum_set_kernel_timing.argtypes = [vp, i32]
        lib.deinsum_set_kernel_timing.restype = i32
        lib.deinsum_kernel_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        lib.deinsum_kernel_time.restype = i32
        lib.deinsum_grid_block.restype = i64
        lib.deinsum_grid_rank.restype = i64
        lib.deinsum_grid_coords.restype = i32
        lib.deinsum_grid_block_range.restype = i32
        lib.deinsum_grid_sub.restype = i32
        lib.deinsum_redist_dim_partitions.restype = i32
        lib.deinsum_redist_match.restype = None
        lib.deinsum_redist_plan.restype = i32
        lib.deinsum_cpals_create.argtypes = [i32, ctypes.POINTER(i64), i32, i32, ctypes.POINTER(vp)]
        lib.deinsum_cpals_create.restype = i32
        lib.deinsum_cpals_run.argtypes = [vp, vp, ctypes.POINTER(vp), vp, i32, vp, vp]
        lib.deinsum_cpals_run.restype = i32
        lib.deinsum_cpals_status.argtypes = [vp]
        lib.deinsum_cpals_status.restype = i32
        lib.deinsum_cpals_destroy.argtypes = [vp]
        lib.deinsum_cpals_destroy.restype = None
        lib.deinsum_plan_batched.argtypes = [i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(i32), i32, i32, ctypes.POINTER(vp)]
        lib.deinsum_plan_batched.restype = i32
        lib.deinsum_execute_batched.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(vp), vp]
        lib.deinsum_execute_batched.restype = i32
        lib.deinsum_batched_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(vp), vp,
                                                 ctypes.POINTER(ctypes.c_double)]
        lib.deinsum_batched_autotune.restype = i32
        lib.deinsum_batched_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                             ctypes.POINTER(ctypes.c_double)]
        lib.deinsum_batched_info.restype = i32
        lib.deinsum_batched_status.argtypes = [vp]
        lib.deinsum_batched_status.restype = i32
        lib.deinsum_batched_destroy.argtypes = [vp]
        lib.deinsum_batched_destroy.restype = None
        lib.deinsum_server_clock.argtypes = []
        lib.deinsum_server_clock.restype = ctypes.c_double
        lib.deinsum_server_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)]
        lib.deinsum_server_create.restype = i32
        lib.deinsum_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(i64)]
        lib.deinsum_server_submit.restype = i32
        lib.deinsum_server_poll.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.deinsum_server_poll.restype = i32
        lib.deinsum_server_take.argtypes = [vp, i64, ctypes.POINTER(_Result), vp, vp, vp]
        lib.deinsum_server_take.restype = i32
        lib.deinsum_server_destroy.argtypes = [vp]
        lib.deinsum_server_destroy.restype = None
        lib.deinsum_plan_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.deinsum_plan_workspace_bytes.restype = i32
        lib.deinsum_plan_bind_workspace.argtypes = [vp, vp, ctypes.c_size_t, vp]
        lib.deinsum_plan_bind_workspace.restype = i32
        lib.deinsum_mttkrp_noalloc.argtypes = [i32, ctypes.POINTER(i64), i32, i32, vp, ctypes.POINTER(vp), vp, vp]
        lib.deinsum_mttkrp_noalloc.restype = i32
        lib.deinsum_mttkrp_noalloc_status.argtypes = []
        lib.deinsum_mttkrp_noalloc_status.restype = i32
        lib.deinsum_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
        lib.deinsum_set_wait_limit_ns.restype = None
        lib.deinsum_alloc_count.argtypes = []
        lib.deinsum_alloc_count.restype = i64
        lib.deinsum_mttkrp_io_bound.argtypes = [ctypes.c_double, ctypes.c_double, i64, ctypes.POINTER(_IoBound)]
        lib.deinsum_mttkrp_io_bound.restype = i32
        lib.deinsum_gen_uniform_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i64, vp, vp]
        lib.deinsum_gen_uniform_f32.restype = i32
        lib.deinsum_gen_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i64, vp, vp]
        lib.deinsum_gen_uniform_f64.restype = i32
        lib.deinsum_gen_cp_f32.argtypes = [ctypes.c_uint64, i32, ctypes.POINTER(i64), i32,
                                           ctypes.POINTER(vp), ctypes.c_double, vp, vp]
        lib.deinsum_gen_cp_f32.restype = i32
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != 0:
        raise DeinsumError(status, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch.Tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (dense row-major)")
    return ctypes.c_void_p(t.data_ptr())


def _dev_ptrs(ts, name: str) -> list:
    """Device addresses (ints) of many tensors, checked as in _dev_ptr.  Builds no per-tensor
    ctypes object: a batch call marshals thousands of pointers, and per-element objects made
    the host's garbage collector pause for tens of ms every few dozen calls."""
    import torch
    try:
        ptrs = [t.data_ptr() for t in ts if t.is_cuda and t.is_contiguous()]
    except AttributeError:
        ptrs = []
    if len(ptrs) != len(ts):
        for t in ts:
            _dev_ptr(t, name)   # raises with the reason
        raise TypeError(f"every {name} must be a contiguous CUDA torch.Tensor")
    if not all(isinstance(t, torch.Tensor) for t in ts):
        raise TypeError(f"{name} must be a CUDA torch.Tensor")
    return ptrs


class Plan:
    """A planned MTTKRP / TTMc contraction (``deinsum_plan``).

    ``extents`` maps every einsum letter to its extent (dict), or lists the
    extents in order of first appearance in ``einsum``.
    """

    def __init__(self, einsum: str, extents, dtype: str = "float32", prec: str = "plain"):
        lib = load()
        letters = []
        for c in einsum.replace(" ", ""):
            if c.isalpha() and c not in letters:
                letters.append(c)
        if isinstance(extents, dict):
            ext = [int(extents[c]) for c in letters]
        else:
            ext = [int(e) for e in extents]
        self.einsum = einsum
        self.letters = letters
        self.extents = dict(zip(letters, ext))
        arr = (ctypes.c_int64 * len(ext))(*ext)
        h = ctypes.c_void_p()
        _check(lib.deinsum_plan(einsum.encode(), arr, len(ext), DTYPES[dtype], PRECS[prec], ctypes.byref(h)),
               f"deinsum_plan({einsum!r})")
        self._h = h
        self.dtype = dtype
        self.prec = prec
        info = _PlanInfo()
        _check(lib.deinsum_plan_info(self._h, ctypes.byref(info)), "deinsum_plan_info")
        self.kind = KINDS[info.kind]
        self.order = info.order
        self.mode = info.mode
        out = einsum.replace(" ", "").split("->")[1]
        self.out_shape = tuple(self.extents[c] for c in out)

    def info(self) -> dict:
        info = _PlanInfo()
        _check(load().deinsum_plan_info(self._h, ctypes.byref(info)), "deinsum_plan_info")
        return {"kind": KINDS[info.kind], "order": info.order, "mode": info.mode,
                "dims": list(info.dims[:info.order]), "ranks": list(info.ranks[:info.order]),
                "out_elems": info.out_elems, "alg_bytes": info.alg_bytes, "alg_flops": info.alg_flops,
                "n_units": info.n_units, "mm_cols": info.mm_cols,
                "view": {"merged": bool(info.view_merged), "packed": bool(info.view_packed),
                         "groups": info.view_groups, "aligned_rows": bool(info.view_aligned_rows),
                         "row_classes": bool(info.view_row_classes)},
                "io": {"fast_mem_words": info.io_fast_mem_words, "rho": info.io_rho,
                       "bound_bytes": info.io_bound_bytes}}

    def workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(load().deinsum_workspace_size(self._h, ctypes.byref(n)), "deinsum_workspace_size")
        return int(n.value)

    def set_kernel_timing(self, enable: bool = True):
        _check(load().deinsum_set_kernel_timing(self._h, int(bool(enable))), "deinsum_set_kernel_timing")

    def kernel_time(self):
        """(summed device ms, launches) of the main kernel since the last call (timing enabled)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().deinsum_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)), "deinsum_kernel_time")
        return float(ms.value), int(n.value)

    def last_device_status(self) -> int:
        return int(load().deinsum_last_device_status(self._h))

    def __call__(self, *operands, out=None, stream=None):
        import torch
        lib = load()
        want = torch.float64 if self.dtype in ("float64", "f64") else torch.float32
        ptrs = (ctypes.c_void_p * len(operands))()
        for k, t in enumerate(operands):
            if t.dtype != want:
                raise TypeError(f"operand {k} has dtype {t.dtype}, plan expects {want}")
            ptrs[k] = _dev_ptr(t, f"operand {k}")
        if out is None:
            out = torch.empty(self.out_shape, dtype=want, device=operands[0].device)
        elif tuple(out.shape) != self.out_shape or out.dtype != want:
            raise ValueError("out has the wrong shape or dtype")
        _check(lib.deinsum_execute(self._h, ptrs, len(operands), _dev_ptr(out, "out"), _stream_ptr(stream)),
               "deinsum_execute")
        return out

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.deinsum_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_XL = "abcdefgh"
_RL = "stuvwxyz"


def mttkrp_einsum(order: int, mode: int) -> str:
    """The MTTKRP einsum of Sec. III-B / Table IV for an order-``order`` tensor, mode ``mode``."""
    x = _XL[:order]
    fac = [x[m] + "r" for m in range(order) if m != mode]
    return ",".join([x] + fac) + "->" + x[mode] + "r"


def mttkrp_mm_einsum(order: int, mode: int) -> str:
    """MTTKRP followed by a matrix product, the running example of Sec. II-A
    (``ijk,ja,ka,al->il`` for order 3, mode 0): the MTTKRP operands, then C = "r l"."""
    x = _XL[:order]
    fac = [x[m] + "r" for m in range(order) if m != mode]
    return ",".join([x] + fac + ["rl"]) + "->" + x[mode] + "l"


def mttkrp_mm(X, factors, mode: int, C, prec: str = "plain", out=None, stream=None):
    """``mttkrp(X, factors, mode) @ C`` with the product applied in the final reduction."""
    import torch
    order = X.dim()
    R = next(f.shape[1] for m, f in enumerate(factors) if m != mode)
    spec = mttkrp_mm_einsum(order, mode)
    extents = list(X.shape) + [R, C.shape[1]]
    dtype = "float64" if X.dtype == torch.float64 else "float32"
    plan = _cached_plan(spec, extents, dtype, prec)
    return plan(X, *[factors[m] for m in range(order) if m != mode], C, out=out, stream=stream)


def ttmc_einsum(order: int, keep: int) -> str:
    """The TTMc einsum (Sec. III-B / Table IV) keeping mode ``keep``."""
    x = _XL[:order]
    fac = [x[m] + _RL[m] for m in range(order) if m != keep]
    out = "".join(x[m] if m == keep else _RL[m] for m in range(order))
    return ",".join([x] + fac) + "->" + out


_plan_cache: dict = {}


def _cached_plan(einsum, extents, dtype, prec):
    key = (einsum, tuple(extents), dtype, prec)
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(einsum, list(extents), dtype, prec)
        _plan_cache[key] = p
    return p


def mttkrp(X, factors, mode: int, prec: str = "plain", out=None, stream=None):
    """Mode-``mode`` MTTKRP of X with ``factors`` (``factors[mode]`` is ignored)."""
    import torch
    order = X.dim()
    R = next(f.shape[1] for m, f in enumerate(factors) if m != mode)
    spec = mttkrp_einsum(order, mode)
    extents = list(X.shape) + [R]
    dtype = "float64" if X.dtype == torch.float64 else "float32"
    plan = _cached_plan(spec, extents, dtype, prec)
    return plan(X, *[factors[m] for m in range(order) if m != mode], out=out, stream=stream)


def ttmc(X, factors, keep: int, prec: str = "plain", out=None, stream=None):
    """TTMc of X keeping mode ``keep``; every other mode m is contracted with ``factors[m]``."""
    import torch
    order = X.dim()
    spec = ttmc_einsum(order, keep)
    extents = list(X.shape) + [factors[m].shape[1] for m in range(order) if m != keep]
    dtype = "float64" if X.dtype == torch.float64 else "float32"
    plan = _cached_plan(spec, extents, dtype, prec)
    return plan(X, *[factors[m] for m in range(order) if m != keep], out=out, stream=stream)


class CPALS:
    """CP-ALS on the device (``deinsum_cpals_create`` / ``_run`` / ``_status`` / ``_destroy``)."""

    def __init__(self, dims, rank: int, prec: str = "split_bf16"):
        lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.rank = int(rank)
        d = (ctypes.c_int64 * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        _check(lib.deinsum_cpals_create(len(self.dims), d, self.rank, PRECS[prec], ctypes.byref(h)),
               "deinsum_cpals_create")
        self._h = h

    def run(self, X, factors, sweeps: int, lam=None, fits=None, stream=None):
        """Run ``sweeps`` sweeps; ``factors`` (CUDA float32, I_m x R) are updated in place.
        Returns (lambda, fits) as CUDA float64 tensors."""
        import torch
        lib = load()
        if lam is None:
            lam = torch.zeros(self.rank, dtype=torch.float64, device=X.device)
        if fits is None:
            fits = torch.zeros(sweeps, dtype=torch.float64, device=X.device)
        fp = (ctypes.c_void_p * len(factors))(*[_dev_ptr(f, "factor").value for f in factors])
        _check(lib.deinsum_cpals_run(self._h, _dev_ptr(X, "X"), fp, _dev_ptr(lam, "lambda"), int(sweeps),
                                     _dev_ptr(fits, "fits"), _stream_ptr(stream)), "deinsum_cpals_run")
        return lam, fits

    def status(self) -> int:
        return int(load().deinsum_cpals_status(self._h))

    def set_dimension_tree(self, enable: bool):
        """Share X x_2 U_2 between modes 0 and 1 of each sweep (order 3, rank <= 32; default on)."""
        _check(load().deinsum_cpals_set_dimension_tree(self._h, int(bool(enable))), "deinsum_cpals_set_dimension_tree")

    @property
    def uses_dimension_tree(self) -> bool:
        return bool(load().deinsum_cpals_uses_dimension_tree(self._h))

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.deinsum_cpals_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BoundBatch:
    """A batch bound to fixed operand and output tensors (see ``Batch.bind``)."""

    __slots__ = ("_batch", "_ip", "_op", "_flat", "_refs")

    def __init__(self, batch, ip, op, flat, refs):
        self._batch, self._ip, self._op, self._flat, self._refs = batch, ip, op, flat, refs

    def __call__(self, stream=None):
        _check(load().deinsum_execute_batched(self._batch._h, self._ip, self._op, _stream_ptr(stream)),
               "deinsum_execute_batched")
        return self._refs[1]


class Batch:
    """Batched MTTKRP (``deinsum_plan_batched`` / ``deinsum_execute_batched`` / ...)."""

    def __init__(self, einsums, extents, prec: str = "split_bf16"):
        n = len(einsums)
        self.n = n
        self._enc = [e.encode() for e in einsums]
        es = (ctypes.c_char_p * n)(*self._enc)
        self._ext = [(ctypes.c_int64 * len(x))(*[int(v) for v in x]) for x in extents]
        ex = (ctypes.c_void_p * n)(*[ctypes.cast(x, ctypes.c_void_p).value for x in self._ext])
        ne = (ctypes.c_int * n)(*[len(x) for x in extents])
        h = ctypes.c_void_p()
        _check(load().deinsum_plan_batched(n, es, ex, ne, 0, PRECS[prec], ctypes.byref(h)), "deinsum_plan_batched")
        self._h = h

    def _marshal(self, inputs, outputs):
        # every operand pointer in one flat array; instance i's table starts at its offset
        if len(inputs) != self.n or len(outputs) != self.n:
            raise ValueError(f"expected {self.n} instances")
        flat = [t for ops in inputs for t in ops]
        self._flat = (ctypes.c_void_p * max(1, len(flat)))(*_dev_ptrs(flat, "operand"))
        base, off, starts = ctypes.addressof(self._flat), 0, []
        for ops in inputs:
            starts.append(base + 8 * off)
            off += len(ops)
        ip = (ctypes.c_void_p * self.n)(*starts)
        op = (ctypes.c_void_p * self.n)(*_dev_ptrs(outputs, "output"))
        return ip, op

    def __call__(self, inputs, outputs, stream=None):
        ip, op = self._marshal(inputs, outputs)
        _check(load().deinsum_execute_batched(self._h, ip, op, _stream_ptr(stream)), "deinsum_execute_batched")
        return outputs

    def bind(self, inputs, outputs) -> "BoundBatch":
        """Marshal the operand and output pointers once and return a callable that replays
        the batch on them: ``bound(stream=None)``.  Each replay then costs the host only the
        C entry point (a pointer comparison and a graph launch) instead of re-checking every
        tensor in Python (about 0.8 ms for 512 instances).  The bound object keeps the
        tensors alive; they must not be resized or re-pointed while it is used."""
        ip, op = self._marshal(inputs, outputs)
        return BoundBatch(self, ip, op, self._flat, (list(inputs), list(outputs)))

    def autotune(self, inputs, outputs, stream=None) -> float:
        ip, op = self._marshal(inputs, outputs)
        ms = ctypes.c_double()
        _check(load().deinsum_batched_autotune(self._h, ip, op, _stream_ptr(stream), ctypes.byref(ms)),
               "deinsum_batched_autotune")
        return float(ms.value)

    def info(self) -> dict:
        nu, g, d, b = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(load().deinsum_batched_info(self._h, ctypes.byref(nu), ctypes.byref(g), ctypes.byref(d),
                                           ctypes.byref(b)), "deinsum_batched_info")
        return {"units": nu.value, "grid": g.value, "unit_div": d.value, "alg_bytes": b.value}

    def status(self) -> int:
        return int(load().deinsum_batched_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.deinsum_batched_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """CP-ALS serving loop (``deinsum_server_*``): continuous batching under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, slots: int, prec: str = "split_bf16"):
        h = ctypes.c_void_p()
        _check(load().deinsum_server_create(int(hbm_budget_bytes), int(slots), PRECS[prec], ctypes.byref(h)),
               "deinsum_server_create")
        self._h = h
        self._keep = {}

    @staticmethod
    def clock() -> float:
        return float(load().deinsum_server_clock())

    def submit(self, dims, rank, sweeps, seed, cp_factors, init_factors, noise=0.0, arrival=None,
               want_factors=False) -> int:
        """Queue one request; ``cp_factors`` / ``init_factors`` are host float32 arrays (I_m x rank)."""
        import numpy as np
        order = len(dims)
        cpf = [np.ascontiguousarray(f, dtype=np.float32) for f in cp_factors]
        ini = [np.ascontiguousarray(f, dtype=np.float32) for f in init_factors]
        q = _Request()
        q.order = order
        for m, d in enumerate(dims):
            q.dims[m] = int(d)
        q.rank, q.sweeps, q.seed = int(rank), int(sweeps), int(seed)
        q.cp_rank = int(cpf[0].shape[1])
        q.noise = float(noise)
        cp_arr = (ctypes.c_void_p * order)(*[f.ctypes.data for f in cpf])
        in_arr = (ctypes.c_void_p * order)(*[f.ctypes.data for f in ini])
        q.cp_factors = ctypes.cast(cp_arr, ctypes.POINTER(ctypes.c_void_p))
        q.init_factors = ctypes.cast(in_arr, ctypes.POINTER(ctypes.c_void_p))
        q.arrival_s = self.clock() if arrival is None else float(arrival)
        q.want_factors = int(bool(want_factors))
        rid = ctypes.c_int64()
        _check(load().deinsum_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid)), "deinsum_server_submit")
        self._keep[rid.value] = (tuple(int(d) for d in dims), int(rank), int(sweeps), bool(want_factors))
        return rid.value

    def poll(self):
        a, w = ctypes.c_int(), ctypes.c_int()
        _check(load().deinsum_server_poll(self._h, ctypes.byref(a), ctypes.byref(w)), "deinsum_server_poll")
        return a.value, w.value

    def take(self, rid: int):
        """Result of a finished request as a dict, or None if it has not finished."""
        import numpy as np
        dims, rank, sweeps, want = self._keep[rid]
        res = _Result()
        fits = np.zeros(sweeps)
        lam = np.zeros(rank)
        fac = np.zeros(sum(d * rank for d in dims), dtype=np.float32) if want else None
        st = load().deinsum_server_take(self._h, rid, ctypes.byref(res), fits.ctypes.data, lam.ctypes.data,
                                        fac.ctypes.data if want else None)
        if st != 0:
            return None
        del self._keep[rid]
        out = {"id": res.id, "status": res.status, "arrival": res.arrival_s, "admit": res.admit_s,
               "done": res.done_s, "gen_ms": res.gen_ms, "fit": res.fit, "fits": fits, "lambda": lam}
        if want:
            parts, o = [], 0
            for d in dims:
                parts.append(fac[o:o + d * rank].reshape(d, rank))
                o += d * rank
            out["factors"] = parts
        return out

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.deinsum_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mttkrp_noalloc(X, factors, mode: int, out, stream=None):
    """Split-BF16 MTTKRP through ``deinsum_mttkrp_noalloc``: the library allocates no
    device memory for it (its scratch is a fixed array inside the library); the
    caller provides ``out`` (I_mode x R float32).  Concurrent calls race."""
    order = X.dim()
    R = next(f.shape[1] for m, f in enumerate(factors) if m != mode)
    d = (ctypes.c_int64 * order)(*[int(s) for s in X.shape])
    fp = (ctypes.c_void_p * order)(*[None if m == mode else _dev_ptr(factors[m], "factor").value
                                     for m in range(order)])
    _check(load().deinsum_mttkrp_noalloc(order, d, mode, int(R), _dev_ptr(X, "X"), fp, _dev_ptr(out, "out"),
                                         _stream_ptr(stream)), "deinsum_mttkrp_noalloc")
    return out


def gen_uniform(seed: int, stream_id: int, shape, dtype=None, device="cuda", stream=None):
    """Device tensor of the seeded uniform[-1, 1) stream (float32 or float64)."""
    import torch
    dtype = dtype or torch.float32
    t = torch.empty(tuple(shape), dtype=dtype, device=device)
    lib = load()
    fn = lib.deinsum_gen_uniform_f64 if dtype == torch.float64 else lib.deinsum_gen_uniform_f32
    _check(fn(seed, stream_id, t.numel(), _dev_ptr(t, "out"), _stream_ptr(stream)), "deinsum_gen_uniform")
    return t


def gen_cp(seed: int, dims, cp_factors, sigma: float, device="cuda", stream=None):
    """Device float32 CP-plus-noise tensor; ``cp_factors`` are CUDA tensors (I_m x rank),
    rounded to float32 here if they are not float32 already."""
    import torch
    order = len(dims)
    cp_factors = [f.to(torch.float32).contiguous() for f in cp_factors]
    t = torch.empty(tuple(dims), dtype=torch.float32, device=device)
    d = (ctypes.c_int64 * order)(*[int(x) for x in dims])
    fp = (ctypes.c_void_p * order)(*[_dev_ptr(f, "cp factor").value for f in cp_factors])
    rank = int(cp_factors[0].shape[1])
    _check(load().deinsum_gen_cp_f32(seed, order, d, rank, fp, float(sigma), _dev_ptr(t, "out"),
                                     _stream_ptr(stream)), "deinsum_gen_cp_f32")
    return t


def mttkrp_io_bound(S: float, t_elems: float, R: int) -> dict:
    """The Sec. IV-E MTTKRP I/O lower bound and tiling (``deinsum_mttkrp_io_bound``)."""
    b = _IoBound()
    _check(load().deinsum_mttkrp_io_bound(float(S), float(t_elems), int(R), ctypes.byref(b)),
           "deinsum_mttkrp_io_bound")
    return {f: getattr(b, f) for f, _ in _IoBound._fields_}


def mttkrp_noalloc_status() -> int:
    """Status of the latest ``deinsum_mttkrp_noalloc`` call on the current device
    (``deinsum_mttkrp_noalloc_status``; 0 ok, 8 a bounded wait gave up); synchronise first."""
    return int(load().deinsum_mttkrp_noalloc_status())


def kernel_launch_count() -> int:
    """Kernels the library has launched in this process (all entry points)."""
    return int(load().deinsum_kernel_launch_count())


def alloc_count() -> int:
    """Device and pinned host allocations the library has made in this process (``deinsum_alloc_count``)."""
    return int(load().deinsum_alloc_count())


def set_wait_limit_ns(ns: int) -> None:
    """Limit of the kernels' bounded waits for later launches (``deinsum_set_wait_limit_ns``;
    0 restores the default 2 s)."""
    load().deinsum_set_wait_limit_ns(int(ns))


# ---------------------------------------------------------------------------
# Block distribution and redistribution (``deinsum_grid_*`` / ``deinsum_redist_*``,
# host only; paper Sec. II-C/D and Sec. V)
# ---------------------------------------------------------------------------

class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("extent", ctypes.c_int64 * 8), ("procs", ctypes.c_int * 8)]


class _DimPart(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int64), ("oy_lo", ctypes.c_int64), ("oy_hi", ctypes.c_int64),
                ("ox_lo", ctypes.c_int64), ("ox_hi", ctypes.c_int64)]


class _Msg(ctypes.Structure):
    _fields_ = [("peer", ctypes.c_int64), ("lo", ctypes.c_int64 * 8), ("hi", ctypes.c_int64 * 8)]


class Grid:
    """A Cartesian process grid over an iteration space, block-distributed (one block per process)."""

    def __init__(self, extents, procs):
        if len(extents) != len(procs):
            raise ValueError("one process count per dimension")
        self.extents = [int(e) for e in extents]
        self.procs = [int(p) for p in procs]
        self._g = _Grid(len(extents), (ctypes.c_int64 * 8)(*self.extents), (ctypes.c_int * 8)(*self.procs))

    @property
    def size(self) -> int:
        n = 1
        for p in self.procs:
            n *= p
        return n

    def block(self, j: int) -> int:
        return int(load().deinsum_grid_block(ctypes.byref(self._g), j))

    def coords(self, rank: int):
        c = (ctypes.c_int * 8)()
        _check(load().deinsum_grid_coords(ctypes.byref(self._g), ctypes.c_int64(rank), c), "deinsum_grid_coords")
        return tuple(c[: len(self.procs)])

    def rank(self, coords) -> int:
        c = (ctypes.c_int * 8)(*[int(x) for x in coords])
        return int(load().deinsum_grid_rank(ctypes.byref(self._g), c))

    def block_range(self, rank: int):
        lo, hi = (ctypes.c_int64 * 8)(), (ctypes.c_int64 * 8)()
        _check(load().deinsum_grid_block_range(ctypes.byref(self._g), ctypes.c_int64(rank), lo, hi),
               "deinsum_grid_block_range")
        n = len(self.procs)
        return tuple(lo[:n]), tuple(hi[:n])

    def sub(self, remain, rank: int):
        """(color, key) of ``rank`` in the sub-grid keeping the dimensions with remain[j] true."""
        r = (ctypes.c_int * 8)(*[1 if x else 0 for x in remain])
        color, key = ctypes.c_int64(), ctypes.c_int64()
        _check(load().deinsum_grid_sub(ctypes.byref(self._g), r, ctypes.c_int64(rank), ctypes.byref(color),
                                       ctypes.byref(key)), "deinsum_grid_sub")
        return int(color.value), int(key.value)


def redist_dim_partitions(Bx: int, By: int, py: int):
    """The runs of one dimension of a redistribution (Eqs. 20-24): [(px, (oy_lo, oy_hi), (ox_lo, ox_hi))]."""
    parts = (_DimPart * 64)()
    k = load().deinsum_redist_dim_partitions(ctypes.c_int64(Bx), ctypes.c_int64(By), ctypes.c_int64(py), parts, 64)
    if k < 0:
        raise ValueError("bad block sizes")
    return [(p.px, (p.oy_lo, p.oy_hi), (p.ox_lo, p.ox_hi)) for p in parts[:k]]


def redist_match(Bx: int, By: int, px: int):
    """Message matching (Eq. 25): the half-open range of y-coordinates meeting x-block px."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    load().deinsum_redist_match(ctypes.c_int64(Bx), ctypes.c_int64(By), ctypes.c_int64(px), ctypes.byref(lo),
                                ctypes.byref(hi))
    return int(lo.value), int(hi.value)


def redist_plan(gx: "Grid", xdims, gy: "Grid", ydims, rank: int, sending: bool):
    """Messages of ``rank`` for moving a tensor from its block distribution on ``gx`` (modes on grid
    dimensions ``xdims``) to the one on ``gy``: [(peer, lo, hi)] with boxes in global coordinates."""
    order = len(xdims)
    xd = (ctypes.c_int * 8)(*xdims)
    yd = (ctypes.c_int * 8)(*ydims)
    lib = load()
    n = lib.deinsum_redist_plan(ctypes.byref(gx._g), xd, ctypes.byref(gy._g), yd, order, ctypes.c_int64(rank),
                                int(bool(sending)), None, 0)
    if n < 0:
        raise ValueError("bad redistribution arguments")
    msgs = (_Msg * max(1, n))()
    n2 = lib.deinsum_redist_plan(ctypes.byref(gx._g), xd, ctypes.byref(gy._g), yd, order, ctypes.c_int64(rank),
                                 int(bool(sending)), msgs, n)
    if n2 != n:
        raise RuntimeError("redistribution plan changed between calls")
    return [(int(m.peer), tuple(m.lo[:order]), tuple(m.hi[:order])) for m in msgs[:n]]
