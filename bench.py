#!/usr/bin/env python3
"""Benchmark of the MTTKRP hot path on one GB300 (or N independent replicas).

Workload (one "step"): the mode-0, mode-1 and mode-2 MTTKRP of an order-3
tensor X of 1024 x 1024 x 1024 FP32 entries (uniform[-1,1) from the seeded
generator) with 1024 x 32 factors drawn N(0, 1/32), through the library's C
ABI with the split-BF16 tcgen05 kernel (``--prec plain`` selects the FP32
CUDA-core kernel).  Inputs are resident in HBM when the timed region starts;
X (4.3 GB) is far larger than the 129 MB L2, so no flush is needed.

value   = algorithmic bytes of the three MTTKRPs / time, in GB/s, where the
          algorithmic bytes of one MTTKRP are |X| + factors + output (4 B each).
e2e     = the same metric with X and the factors copied from pinned host memory
          and the three outputs copied back inside the timed region.
roofline: the main contraction kernel, timed with CUDA events that the
          library records around it on the execute stream.
cpu_baseline / --impl reference: the FP64 oracle on the host cores, on a
          bounded sample of output rows of the same workload.

Under torchrun (N > 1) every rank runs its own replica with its own seed; the
timed region is bracketed by barriers and the max over ranks is reported
(weak scaling: there is no data exchange between ranks).
"""
from __future__ import annotations

import argparse
import contextlib
import datetime
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EXT = 1024
RANK_R = 32
MODES = (0, 1, 2)
METRIC = "MTTKRP/TTMc GB/s & % roofline at rel.err≤1e-5; CP-ALS req/s, p50/p99 latency"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _alg_bytes_one_mode():
    x = N_EXT ** 3
    return 4.0 * (x + 2 * N_EXT * RANK_R + N_EXT * RANK_R)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 10 ms.  ``mark_start`` /
    ``mark_stop`` bound the main timed region and ``region(name)`` any number of named ones;
    only the samples whose timestamps fall inside a region are reported for it (with the last
    sample before it when the region is shorter than the sampling interval)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = f"/tmp/deinsum_clocks_{os.getpid()}.csv"
        self.t0 = self.t1 = None
        self.regions = {}
        self.rows = []

    def start(self):
        """Start sampling and return once the first sample has been written (or after 5 s)."""
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 5.0
        while time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def region(self, name):
        sampler = self

        class _Region:
            def __enter__(self):
                self.t0 = time.time()

            def __exit__(self, *exc):
                sampler.regions[name] = (self.t0, time.time())
        return _Region()

    @staticmethod
    def _stamp(text):
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.03)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    self.rows.append((self._stamp(parts[0]), float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        return self.stats(self.t0, self.t1)

    def stats(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self.rows
        inside = [r for r in rows if r[0] is not None and t0 is not None and t0 <= r[0] <= t1]
        if not inside:   # a region shorter than the interval: the sample just before it
            before = [r for r in rows if r[0] is not None and t0 is not None and r[0] < t0]
            inside = before[-1:] if before else rows[:1]
        reasons = set()
        for r in inside:
            for name, val in zip(self.NAMES, r[3]):
                if val.lower() == "active":
                    reasons.add(name)
        sm = [r[1] for r in inside]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "interval_ms": 10, "region_ms": (t1 - t0) * 1e3 if t0 and t1 else None}

    def region_stats(self, name):
        t0, t1 = self.regions.get(name, (None, None))
        return self.stats(t0, t1)


# The sources each main kernel is compiled from (its .cu file and the headers it includes).
KERNEL_SOURCES = {
    "mttkrp_tc.cu": ("mttkrp_tc.cu", "mttkrp_tc.cuh", "tc_common.cuh", "sm100.cuh", "internal.h"),
    "ttmc_tc.cu": ("ttmc_tc.cu", "tc_common.cuh", "sm100.cuh", "internal.h"),
}


def _code_only(text):
    """C/C++ source as the compiler reads it: comments removed (string and character
    literals kept whole), each line stripped, blank lines dropped."""
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch in "\"'":
            j = i + 1
            while j < n and text[j] != ch:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(ch)
            i += 1
    return "\n".join(line.strip() for line in "".join(out).splitlines() if line.strip())


def _kernel_source_hash(source="mttkrp_tc.cu"):
    """Hash of the code (not the comments) of the files a main kernel is compiled from: a
    committed traffic record stays current across edits of comments only."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(source, (source,)):
        with open(os.path.join(ROOT, "paper_2206_08301_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic_per_launch(prec, source="mttkrp_tc.cu"):
    """DRAM bytes per launch of the main kernel from the committed ncu summary, if still current."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
        e = t.get(prec)
        if e and e.get("source_sha") == _kernel_source_hash(source):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def cpu_oracle_sample(seed, budget_s: float, threads: int = 0):
    """Time the FP64 oracle on sampled output rows of the workload until ``budget_s`` is spent,
    on ``threads`` host threads (0: all the oracle's OpenMP runtime offers).

    Returns (GB/s of X covered, seconds, rows, threads used).  Slab generation is not timed.
    """
    import oracle
    from paper_2206_08301_gb300 import inputs
    all_threads = oracle.set_threads(0)
    used = oracle.set_threads(threads if threads > 0 else all_threads)
    dims = (N_EXT,) * 3
    Us = [inputs.factor_normal(seed, m, N_EXT, RANK_R, sigma=np.sqrt(1.0 / RANK_R)).astype(np.float32)
          for m in range(3)]
    rows_all = {m: inputs.sample_rows(seed, N_EXT, 256, tag=m) for m in MODES}
    spent, covered, nrows, k = 0.0, 0.0, 0, 0
    batch = 8
    while spent < budget_s and k * batch < 256:
        for mode in MODES:
            rows = rows_all[mode][k * batch:(k + 1) * batch]
            slabs = np.stack([inputs.uniform_slab(seed, dims, mode, int(r)).ravel() for r in rows])
            t0 = time.perf_counter()
            oracle.mttkrp_rows(dims, mode, slabs, Us)
            spent += time.perf_counter() - t0
            covered += 4.0 * slabs.size
            nrows += len(rows)
        k += 1
    oracle.set_threads(all_threads)
    return covered / spent / 1e9, spent, nrows, used


def run_once(args):
    """One execute per requested mode (for ncu captures of a small case); prints 'ok'.
    With --workload ttmc: one split-BF16 TTMc ijkl,jb,kc,ld->ibcd at X n x n x 256 x 256, R = 32.
    With --workload paper: the order-5 TTMc of the paper's shapes (mode 0 kept, R = 24) at
    X n x 60^4."""
    import torch
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    n = args.n
    if args.workload == "paper":
        dims, R = (n, 60, 60, 60, 60), 24
        X = dz.gen_uniform(1301, inputs.STREAM_X, dims)
        U = [None] + [torch.from_numpy(inputs.factor_normal(1301, m, dims[m], R).astype(np.float32)).cuda()
                      for m in range(1, 5)]
        dz.ttmc(X, U, 0, prec=args.prec)
        torch.cuda.synchronize()
        print("ok")
        return 0
    if args.workload == "ttmc":
        dims = (n, n, 256, 256)
        X = dz.gen_uniform(4096, inputs.STREAM_X, dims)
        U = [None] + [torch.from_numpy(inputs.factor_normal(4096, m, dims[m], 32).astype(np.float32)).cuda()
                      for m in (1, 2, 3)]
        dz.ttmc(X, U, 0, prec=args.prec)
        torch.cuda.synchronize()
        print("ok")
        return 0
    dims = (n, n, n)
    X = dz.gen_uniform(2024, inputs.STREAM_X, dims)
    if args.x_offset:   # X starting args.x_offset floats into its buffer (rows not 16-byte aligned)
        buf = torch.empty(X.numel() + args.x_offset, device="cuda")
        Xo = buf[args.x_offset:].view(dims)
        Xo.copy_(X)
        X = Xo
    U = [torch.from_numpy(inputs.factor_normal(2024, m, n, RANK_R, sigma=np.sqrt(1.0 / RANK_R))
                          .astype(np.float32)).cuda() for m in range(3)]
    for mode in [int(m) for m in args.modes.split(",")]:
        p = dz.Plan(dz.mttkrp_einsum(3, mode), list(dims) + [RANK_R], "float32", args.prec)
        p(X, *[U[m] for m in range(3) if m != mode])
    torch.cuda.synchronize()
    print("ok")
    return 0


def run_unaligned(args):
    """MTTKRP order 3, R = 32, split-BF16, per mode: X 1024^3 aligned (tensor map), X 1024^3
    starting one float into its buffer and X 1023^3 (rows not 16-byte aligned: row-class tensor
    maps).  Main-kernel time from CUDA events around it (average of --steps launches after 3
    warm-up ones); X (4.3 GB) is larger than L2."""
    import torch
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    stream = torch.cuda.Stream()
    peak, peak_kind = _peaks()
    out_cases = []
    for dims, off in [((1024, 1024, 1024), 0), ((1024, 1024, 1024), 1), ((1023, 1023, 1023), 0)]:
        X = dz.gen_uniform(5, inputs.STREAM_X, dims)
        if off:
            buf = torch.empty(X.numel() + off, device="cuda")
            Xo = buf[off:].view(dims)
            Xo.copy_(X)
            del X
            X = Xo
        U = [torch.from_numpy(inputs.factor_normal(5, m, d, RANK_R, sigma=np.sqrt(1.0 / RANK_R))
                              .astype(np.float32)).cuda() for m, d in enumerate(dims)]
        for mode in range(3):
            p = dz.Plan(dz.mttkrp_einsum(3, mode), list(dims) + [RANK_R], "float32", "split_bf16")
            ops = [X] + [U[m] for m in range(3) if m != mode]
            out = torch.empty(dims[mode], RANK_R, device="cuda")
            with torch.cuda.stream(stream):
                for _ in range(3):
                    p(*ops, out=out, stream=stream)
            stream.synchronize()
            p.set_kernel_timing(True)
            p.kernel_time()
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    p(*ops, out=out, stream=stream)
            stream.synchronize()
            kms, kn = p.kernel_time()
            kms /= max(1, kn)
            gbs = 4.0 * float(np.prod(dims)) / kms / 1e6
            out_cases.append({"dims": list(dims), "x_offset_floats": off, "mode": mode,
                              "kernel_ms": round(kms, 4), "GB/s": round(gbs, 1),
                              "frac": round(gbs / peak, 3)})
        del X, U
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "MTTKRP main-kernel GB/s, aligned and unaligned rows", "unit": "GB/s",
                      "peak": peak, "peak_kind": peak_kind, "data": "synthetic", "cases": out_cases}))
    return 0


def _serving_requests(n, seed):
    """Synthetic CP-ALS requests: extents U{64..1024} per mode, R U{8..64}, rank-R CP
    tensor with N(0,1) factors + 1e-2 noise, 10 sweeps, N(0,1) initial factors."""
    from paper_2206_08301_gb300 import inputs
    ext = inputs.draw_int(seed, 0, 64, 1024, 3 * n).reshape(n, 3)
    ranks = inputs.draw_int(seed, 1, 8, 64, n)
    reqs = []
    for k in range(n):
        dims = tuple(int(d) for d in ext[k])
        R = int(ranks[k])
        s = seed * 100003 + k
        cpf = [inputs.factor_normal(s, m, d, R, stream_base=inputs.STREAM_CP).astype(np.float32)
               for m, d in enumerate(dims)]
        ini = [inputs.factor_normal(s, m, d, R, stream_base=inputs.STREAM_INIT).astype(np.float32)
               for m, d in enumerate(dims)]
        reqs.append(dict(dims=dims, rank=R, sweeps=10, seed=s, cp_factors=cpf, init_factors=ini, noise=1e-2))
    return reqs


def _serve_run(reqs, slots, prec, rate, budget, seed):
    """Serve `reqs` with Poisson arrivals at `rate` req/s (None: all at t=0).
    Returns (makespan s, latencies s, gen ms, statuses, fits)."""
    import paper_2206_08301_gb300 as dz
    srv = dz.Server(budget, slots, prec)
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    t0 = srv.clock()
    arrivals = t0 + np.cumsum(gaps)
    ids, out, nxt = [], {}, 0
    while len(out) < len(reqs):
        now = srv.clock()
        while nxt < len(reqs) and arrivals[nxt] <= now:
            ids.append(srv.submit(arrival=float(arrivals[nxt]), **reqs[nxt]))
            nxt += 1
        srv.poll()
        for i in ids:
            if i not in out:
                r = srv.take(i)
                if r is not None:
                    out[i] = r
    srv.close()
    res = [out[i] for i in ids]
    lat = np.array([r["done"] - r["arrival"] for r in res])
    span = max(r["done"] for r in res) - t0
    return span, lat, np.array([r["gen_ms"] for r in res]), [r["status"] for r in res], [r["fit"] for r in res]


def run_serving(args):
    """CP-ALS serving: continuous batching (4 slots, split-BF16) under Poisson arrivals at
    0.5/0.8/1.0/1.2x the measured one-at-a-time split-BF16 service rate, against one-at-a-time
    plain FP32 solves (1 slot) at the same arrival rate."""
    import torch
    budget = 64 << 30
    reqs = _serving_requests(args.requests, 7)
    torch.cuda.synchronize()
    _serve_run(reqs[:8], 1, "split_bf16", None, budget, 1)            # warm-up
    span1, lat1, _, st1, _ = _serve_run(reqs, 1, "split_bf16", None, budget, 1)
    mu = len(reqs) / span1
    rows = []
    for f in (0.5, 0.8, 1.0, 1.2):
        span, lat, gen, st, fits = _serve_run(reqs, 4, "split_bf16", f * mu, budget, 11)
        rows.append({"load": f, "arrival_rate": f * mu, "req_s": len(reqs) / span,
                     "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                     "gen_ms_mean": float(gen.mean()), "ok": int(sum(s == 0 for s in st)),
                     "fit_min": float(min(fits))})
    spanp, latp, _, stp, _ = _serve_run(reqs, 1, "plain", mu, budget, 11)
    line = {"metric": "CP-ALS serving req/s and p50/p99 latency", "unit": "req/s", "n_gpus": 1,
            "requests": len(reqs), "sweeps": 10, "data": "synthetic",
            "config": {"workload": "Poisson CP-ALS requests: extents U{64..1024}, R U{8..64}, rank-R CP N(0,1) "
                                   "+ 1e-2 noise, 10 sweeps, X generated on the device per request",
                       "hbm_budget_gb": budget / 2 ** 30, "slots": 4},
            "one_at_a_time_split": {"req_s": mu, "p50_ms": 1e3 * float(np.percentile(lat1, 50)),
                                    "p99_ms": 1e3 * float(np.percentile(lat1, 99))},
            "continuous_batching_split": rows,
            "one_at_a_time_plain_at_rate_mu": {"req_s": len(reqs) / spanp,
                                               "p50_ms": 1e3 * float(np.percentile(latp, 50)),
                                               "p99_ms": 1e3 * float(np.percentile(latp, 99))}}
    print(json.dumps(line))
    return 0


def run_paper(args):
    """The paper's own benchmark shapes (Table V, single-device sizes; uniform X, factors N(0,1)):
    MTTKRP-O3-M{0,1,2} at 1024^3, R 24; the running example of Sec. II-A (MTTKRP + MM,
    ijk,ja,ka,al->il) at 1024^3, R 24, L 64; MTTKRP-O5-M{0,2,4} at 64^5, R 24 (the order-5 extent
    1024 of the table is read as 64, see the design notes); TTMc-O5-M0 at 60^5, R 24.  One JSON
    line per benchmark: split-BF16 and plain FP32 times, GB/s of algorithmic bytes, the main
    kernel's roofline fraction, and the relative error on sampled output rows."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()

    def timed(plan, ops, out, steps):
        with host_gc_paused(), torch.cuda.stream(stream):
            for _ in range(3):
                plan(*ops, out=out, stream=stream)
            stream.synchronize()
            plan.set_kernel_timing(True)
            plan.kernel_time()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(stream)
            for _ in range(steps):
                plan(*ops, out=out, stream=stream)
            e1.record(stream)
            stream.synchronize()
        kms, kn = plan.kernel_time()
        plan.set_kernel_timing(False)
        return e0.elapsed_time(e1) / steps, kms / max(1, kn)

    cases = [("MTTKRP-O3-M%d" % m, "mttkrp", (1024,) * 3, m) for m in (0, 1, 2)]
    cases += [("MTTKRP+MM-O3-M0", "mm", (1024,) * 3, 0)]   # the running example ijk,ja,ka,al->il, L = 64
    cases += [("MTTKRP-O5-M%d" % m, "mttkrp", (64,) * 5, m) for m in (0, 2, 4)]
    cases += [("TTMc-O5-M0", "ttmc", (60,) * 5, 0)]
    R, seed = 24, 1301
    X, dims_now = None, None
    for name, kind, dims, mode in cases:
        if dims != dims_now:
            X = None
            torch.cuda.empty_cache()
            X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
            Us = [inputs.factor_normal(seed, m, d, R).astype(np.float32) for m, d in enumerate(dims)]
            Ud = [torch.from_numpy(u).cuda() for u in Us]
            dims_now = dims
        N = len(dims)
        if kind == "mttkrp":
            spec, ext = dz.mttkrp_einsum(N, mode), list(dims) + [R]
            out = torch.empty(dims[mode], R, device="cuda")
        elif kind == "mm":
            Cm = inputs.factor_normal(seed, 9, R, 64).astype(np.float32)
            spec, ext = dz.mttkrp_mm_einsum(N, mode), list(dims) + [R, 64]
            out = torch.empty(dims[mode], 64, device="cuda")
        else:
            spec, ext = dz.ttmc_einsum(N, mode), list(dims) + [R] * (N - 1)
            out = torch.empty([dims[m] if m == mode else R for m in range(N)], device="cuda")
        ops = [X] + [Ud[m] for m in range(N) if m != mode]
        if kind == "mm":
            ops.append(torch.from_numpy(Cm).cuda())
        res = {}
        for prec in ("split_bf16", "plain"):
            plan = dz.Plan(spec, ext, "float32", prec)
            ms, kms = timed(plan, ops, out, args.steps if prec == "split_bf16" else max(1, args.steps // 3))
            res[prec] = (ms, kms, plan.info()["alg_bytes"])
            if prec == "split_bf16":
                rows = inputs.sample_rows(seed, dims[mode], 2, tag=mode)
                got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
        slabs = np.stack([inputs.uniform_slab(seed, dims, mode, int(r)).ravel() for r in rows])
        if kind in ("mttkrp", "mm"):
            ref = oracle.mttkrp_rows(dims, mode, slabs, Us)
            if kind == "mm":
                ref = ref @ Cm.astype(np.float64)
            kernel, kbytes = "mttkrp_tc_kernel", 4.0 * float(np.prod(dims))
        else:
            ref = oracle.ttmc_rows(dims, mode, slabs, Us)
            kernel = "ttmc_fused_kernel"
            kbytes = 4.0 * float(np.prod(dims)) * (1.0 + R * R / (dims[-1] * dims[-2]))
        ms, kms, ab = res["split_bf16"]
        achieved = kbytes / (kms * 1e-3) / 1e9
        print(json.dumps({"benchmark": name, "dims": list(dims), "R": R, "mode": mode, "unit": "GB/s",
                          "value": ab / (ms * 1e-3) / 1e9, "ms": ms, "plain_fp32_ms": res["plain"][0],
                          "speedup_vs_plain": res["plain"][0] / ms,
                          "roofline": {"bound": "hbm", "kernel": kernel, "kernel_ms": kms, "achieved": achieved,
                                       "peak": peak, "frac": achieved / peak, "peak_kind": peak_kind},
                          "rel_err_sampled_rows": oracle.rel_error(got, ref)}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Per-configuration measurements (the "workloads" of the benchmark line).  Each
# returns one record: its metric and value, the dominant kernel's time and its
# roofline fraction against the measured peak, the comparison the configuration
# names (plain FP32 CUDA cores, separate launches, one-at-a-time solves), the
# relative error of sampled outputs against the FP64 oracle, and the clocks seen
# during its own timed region.
# ---------------------------------------------------------------------------

FP32_CORE_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


@contextlib.contextmanager
def host_gc_paused():
    """Around a device-timed region and its warm-up: collect the host's garbage first and keep
    the collector off, so that a collection pause of the Python host (tens of ms with large
    heaps) cannot leave the queued GPU work idle inside the region.  The collection runs before
    the warm-up, not between it and the region: after an idle gap of that length the first
    timed launches ran measurably slower.  The e2e region runs without it."""
    was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def _events_ms(stream, fn, reps, warm=3):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with host_gc_paused(), torch.cuda.stream(stream):
        for _ in range(warm):
            fn()
        stream.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
    return e0.elapsed_time(e1) / reps


def _plan_timed(plan, ops, out, stream, reps, warm=3):
    """(ms per execute, average main-kernel ms) of a plan over `reps` executes."""
    import torch
    fn = lambda: plan(*ops, out=out, stream=stream)  # noqa: E731
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with host_gc_paused(), torch_stream(stream):
        for _ in range(warm):
            fn()
        stream.synchronize()
        plan.set_kernel_timing(True)
        plan.kernel_time()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
    kms, kn = plan.kernel_time()
    plan.set_kernel_timing(False)
    return e0.elapsed_time(e1) / reps, kms / max(1, kn)


def torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)


def measure_c0_fp64(clk, reps=200):
    """MTTKRP order 3, X 64^3 FP64 uniform[-1,1), factors 64 x 16 N(0,1), mode 0, plain FP64
    CUDA-core kernel: latency per execute (the configuration fits in L2; no roofline), error
    against the FP64 oracle over the whole output."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    seed, n, R = 64, 64, 16
    dims = (n, n, n)
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims, dtype=torch.float64)
    Us = [inputs.factor_normal(seed, m, n, R) for m in range(3)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    plan = dz.Plan(dz.mttkrp_einsum(3, 0), list(dims) + [R], "float64", "plain")
    out = torch.empty(n, R, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with clk.region("c0"):
        ms, kms = _plan_timed(plan, [X, Ud[1], Ud[2]], out, stream, reps)
    ref = oracle.mttkrp(inputs.tensor_uniform_f64(seed, dims), Us, 0)
    got = out.cpu().numpy()
    ab = plan.info()["alg_bytes"]
    return {"workload": "MTTKRP 64^3 FP64 uniform[-1,1), R 16 N(0,1), mode 0, plain FP64 CUDA cores",
            "metric": "us per execute", "value": ms * 1e3, "unit": "us", "higher_is_better": False,
            "kernel": "mttkrp_plain_kernel<double>", "kernel_us": kms * 1e3, "alg_gb_s": ab / (ms * 1e-3) / 1e9,
            "rel_err": oracle.rel_error(got, ref), "max_elem_err": oracle.max_elem_error(got, ref),
            "gate": "rel_err <= 1e-12", "sample": "whole output", "clocks_region": "c0"}


def measure_c1_plain(clk, X, Ud, Us, seed, peak, reps=5):
    """The benchmark configuration (MTTKRP 1024^3, R 32, modes 0-2) on the plain FP32
    CUDA-core kernel: the arm the split-BF16 tensor-core path must beat."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    dims = (N_EXT,) * 3
    stream = torch.cuda.Stream()
    plans = {m: dz.Plan(dz.mttkrp_einsum(3, m), list(dims) + [RANK_R], "float32", "plain") for m in MODES}
    outs = {m: torch.empty(N_EXT, RANK_R, device="cuda") for m in MODES}
    tot_ms, kern = 0.0, []
    with clk.region("c1_plain"):
        for m in MODES:
            ms, kms = _plan_timed(plans[m], [X] + [Ud[k] for k in range(3) if k != m], outs[m], stream, reps)
            tot_ms += ms
            kern.append(kms)
    errs = []
    for m in MODES:
        rows = inputs.sample_rows(seed, N_EXT, 16, tag=m)
        slabs = np.stack([inputs.uniform_slab(seed, dims, m, int(r)).ravel() for r in rows])
        ref = oracle.mttkrp_rows(dims, m, slabs, Us)
        errs.append(oracle.rel_error(outs[m][torch.from_numpy(rows).cuda()].cpu().numpy(), ref))
    kms = float(np.mean(kern))
    flops = 2.0 * N_EXT ** 3 * RANK_R
    return {"workload": "MTTKRP 1024^3 FP32, R 32, modes 0,1,2 per step, plain FP32 CUDA-core kernel",
            "metric": "GB/s", "value": 3 * _alg_bytes_one_mode() / (tot_ms * 1e-3) / 1e9, "unit": "GB/s",
            "ms_per_step": tot_ms, "kernel": "mttkrp_plain_kernel<float>", "kernel_ms_avg": kms,
            "roofline": {"bound": "alu", "achieved": flops / (kms * 1e-3) / 1e12, "peak": FP32_CORE_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / (kms * 1e-3) / 1e12 / FP32_CORE_TFLOPS,
                         "peak_kind": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2 x 2.07 GHz)",
                         "hbm_frac": 4.0 * N_EXT ** 3 / (kms * 1e-3) / 1e9 / peak},
            "rel_err": max(errs), "sample": "16 output rows per mode", "clocks_region": "c1_plain"}


def measure_c2a_order5(clk, peak, reps=5):
    """MTTKRP order 5, X 64^5 FP32 = rank-24 CP (N(0,1) factors) + 1e-3 noise, R 24 factors
    N(0,1), modes 0 and 2: split-BF16 tensor cores against the plain FP32 kernel."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    seed, n, rc, R = 5055, 64, 24, 24
    dims = (n,) * 5
    A = [inputs.factor_normal(seed, m, n, rc, stream_base=inputs.STREAM_CP) for m in range(5)]
    X = dz.gen_cp(seed, dims, [torch.from_numpy(a).cuda() for a in A], 1e-3)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(5)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    stream = torch.cuda.Stream()
    modes = {}
    xb = 4.0 * n ** 5
    with clk.region("c2a"):
        for mode in (0, 2):
            spec, ext = dz.mttkrp_einsum(5, mode), list(dims) + [R]
            ops = [X] + [Ud[m] for m in range(5) if m != mode]
            res = {}
            for prec in ("split_bf16", "plain"):
                plan = dz.Plan(spec, ext, "float32", prec)
                out = torch.empty(n, R, device="cuda")
                ms, kms = _plan_timed(plan, ops, out, stream, reps if prec == "split_bf16" else 2)
                res[prec] = (ms, kms, plan.info()["alg_bytes"], out)
            modes[mode] = res
    recs = {}
    for mode, res in modes.items():
        rows = inputs.sample_rows(seed, n, 4, tag=mode)
        slabs = np.stack([inputs.cp_slab(seed, dims, A, 1e-3, mode, int(r)).ravel() for r in rows])
        ref = oracle.mttkrp_rows(dims, mode, slabs, Us)
        ms, kms, ab, out = res["split_bf16"]
        recs[f"mode{mode}"] = {
            "value": ab / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms": ms, "plain_fp32_ms": res["plain"][0],
            "speedup_vs_plain": res["plain"][0] / ms,
            "roofline": {"bound": "hbm", "kernel": "mttkrp_tc_kernel", "kernel_ms": kms,
                         "achieved": xb / (kms * 1e-3) / 1e9, "peak": peak,
                         "frac": xb / (kms * 1e-3) / 1e9 / peak},
            "rel_err": oracle.rel_error(out[torch.from_numpy(rows).cuda()].cpu().numpy(), ref)}
    del X
    torch.cuda.empty_cache()
    return {"workload": "MTTKRP 64^5 FP32 = rank-24 CP + 1e-3 noise, R 24, modes 0 and 2, split-BF16 vs plain FP32",
            "metric": "GB/s", "unit": "GB/s", "value": min(r["value"] for r in recs.values()),
            "modes": recs, "rel_err": max(r["rel_err"] for r in recs.values()),
            "sample": "4 output rows per mode", "clocks_region": "c2a"}


def measure_c2b_ttmc(clk, peak, reps=3):
    """TTMc ijkl,jb,kc,ld->ibcd, X 256^4 FP32 uniform[-1,1), U 256 x 32 N(0,1): the fused
    split-BF16 path (modes l and k on the tensor cores, T1 on chip) against the plain FP32
    chain of TTMs."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    seed, n, R = 4096, 256, 32
    dims = (n,) * 4
    spec = dz.ttmc_einsum(4, 0)
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(4)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    out = torch.empty(n, R, R, R, device="cuda")
    stream = torch.cuda.Stream()
    plans = {p: dz.Plan(spec, list(dims) + [R, R, R], "float32", p) for p in ("split_bf16", "plain")}
    with clk.region("c2b"):
        l0 = dz.kernel_launch_count()
        ms, kms = _plan_timed(plans["split_bf16"], [X] + Ud[1:], out, stream, reps)
        launches = (dz.kernel_launch_count() - l0) / (reps + 3)
        status = plans["split_bf16"].last_device_status()
        rows = inputs.sample_rows(seed, n, 2, tag=7)
        got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
        ms_plain, _ = _plan_timed(plans["plain"], [X] + Ud[1:], out, stream, 1, warm=1)
    del X
    torch.cuda.empty_cache()
    slabs = np.stack([inputs.uniform_slab(seed, dims, 0, int(r)).ravel() for r in rows])
    ref = oracle.ttmc_rows(dims, 0, slabs, Us)
    ab = plans["split_bf16"].info()["alg_bytes"]
    kbytes = 4.0 * n ** 4 + 4.0 * n * n * R * R   # X once + T2 written once
    return {"workload": "TTMc ijkl,jb,kc,ld->ibcd, X 256^4 FP32 uniform[-1,1), U 256x32 N(0,1), split-BF16 "
                        "(fused last two modes) vs plain FP32 chain",
            "metric": "GB/s", "value": ab / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "alg_frac": ab / (ms * 1e-3) / 1e9 / peak,
            "roofline": {"bound": "hbm", "kernel": "ttmc_fused_kernel", "kernel_ms": kms,
                         "bytes_per_launch": kbytes, "achieved": kbytes / (kms * 1e-3) / 1e9, "peak": peak,
                         "frac": kbytes / (kms * 1e-3) / 1e9 / peak,
                         "traffic": _traffic_per_launch("ttmc_split_bf16", "ttmc_tc.cu")},
            "plain_chain_ms": ms_plain, "speedup_vs_plain_chain": ms_plain / ms, "launches_per_step": launches,
            "rel_err": oracle.rel_error(got, ref), "max_elem_err": oracle.max_elem_error(got, ref),
            "sample": "2 kept-mode slices (2 x 32^3 outputs)", "device_status": status,
            "clocks_region": "c2b"}


def measure_ttmc_o5(clk, peak, reps=5):
    """The paper's TTMc-O5-M0 (Table V): X 60^5 FP32 uniform[-1,1), U 60 x 24 N(0,1), mode 0
    kept, split-BF16 (fused last two modes, then the chain's two TTMs on the tensor cores)
    against the plain FP32 chain of TTMs."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    seed, n, R, N = 1301, 60, 24, 5
    dims = (n,) * N
    spec = dz.ttmc_einsum(N, 0)
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, n, R).astype(np.float32) for m in range(N)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    out = torch.empty(n, R, R, R, R, device="cuda")
    stream = torch.cuda.Stream()
    plans = {p: dz.Plan(spec, list(dims) + [R] * (N - 1), "float32", p) for p in ("split_bf16", "plain")}
    with clk.region("ttmc_o5"):
        l0 = dz.kernel_launch_count()
        ms, kms = _plan_timed(plans["split_bf16"], [X] + Ud[1:], out, stream, reps)
        launches = (dz.kernel_launch_count() - l0) / (reps + 3)
        status = plans["split_bf16"].last_device_status()
        rows = inputs.sample_rows(seed, n, 2, tag=0)
        got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
        ms_plain, _ = _plan_timed(plans["plain"], [X] + Ud[1:], out, stream, 1, warm=1)
    del X
    torch.cuda.empty_cache()
    slabs = np.stack([inputs.uniform_slab(seed, dims, 0, int(r)).ravel() for r in rows])
    ref = oracle.ttmc_rows(dims, 0, slabs, Us)
    ab = plans["split_bf16"].info()["alg_bytes"]
    kbytes = 4.0 * n ** N + 4.0 * n ** (N - 2) * R * R   # X once + T2 written once
    return {"workload": "TTMc-O5-M0 ijklm,jb,kc,ld,me->ibcde, X 60^5 FP32 uniform[-1,1), U 60x24 N(0,1), "
                        "split-BF16 (fused last two modes, chain TTMs on the tensor cores) vs plain FP32 chain",
            "metric": "GB/s", "value": ab / (ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
            "alg_frac": ab / (ms * 1e-3) / 1e9 / peak,
            "roofline": {"bound": "hbm", "kernel": "ttmc_fused_kernel", "kernel_ms": kms,
                         "bytes_per_launch": kbytes, "achieved": kbytes / (kms * 1e-3) / 1e9, "peak": peak,
                         "frac": kbytes / (kms * 1e-3) / 1e9 / peak,
                         "traffic": _traffic_per_launch("ttmc_split_bf16_packed", "ttmc_tc.cu")},
            "plain_chain_ms": ms_plain, "speedup_vs_plain_chain": ms_plain / ms, "launches_per_step": launches,
            "rel_err": oracle.rel_error(got, ref), "max_elem_err": oracle.max_elem_error(got, ref),
            "sample": "2 kept-mode slices (2 x 24^4 outputs)", "device_status": status,
            "clocks_region": "ttmc_o5"}


def measure_c3_batched(clk, peak, n=512, reps=5):
    """512 uneven order-3 MTTKRP instances (extents U{32..384}, R in {8,16,32,64}, mode
    U{0,1,2}, X uniform[-1,1) float32): the graph-replayed persistent split-BF16 launches
    (autotuned unit size) against 512 separate plain launches and 512 separate split
    executes."""
    import torch
    import oracle
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    seed = 33
    ext = inputs.draw_int(seed, 0, 32, 384, 3 * n).reshape(n, 3)
    ranks = np.array([8, 16, 32, 64])[inputs.draw_int(seed, 1, 0, 3, n)]
    modes = inputs.draw_int(seed, 2, 0, 2, n)
    einsums, extents, ins, outs, facs = [], [], [], [], []
    for k in range(n):
        dims = tuple(int(d) for d in ext[k])
        R, mode = int(ranks[k]), int(modes[k])
        X = dz.gen_uniform(seed * 10000 + k, inputs.STREAM_X, dims)
        U = [torch.from_numpy(inputs.factor_normal(seed * 10000 + k, m, d, R).astype(np.float32)).cuda()
             for m, d in enumerate(dims)]
        einsums.append(dz.mttkrp_einsum(3, mode))
        extents.append(list(dims) + [R])
        ins.append([X] + [U[m] for m in range(3) if m != mode])
        outs.append(torch.empty(dims[mode], R, device="cuda"))
        facs.append(U)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    bsplit = dz.Batch(einsums, extents, "split_bf16")
    with torch.cuda.stream(stream):
        tune_ms = bsplit.autotune(ins, outs, stream=stream)
    replay = bsplit.bind(ins, outs)   # pointers marshalled once: each call is one graph launch
    with clk.region("c3"):
        t_batch = _events_ms(stream, lambda: replay(stream=stream), reps)
    l0 = dz.kernel_launch_count()   # kernels per replay (the graph is captured by now)
    with torch.cuda.stream(stream):
        for _ in range(2):
            replay(stream=stream)
    stream.synchronize()
    launches = (dz.kernel_launch_count() - l0) / 2
    status = bsplit.status()
    info = bsplit.info()
    errs = []
    for k in range(0, n, max(1, n // 16)):
        dims, mode = tuple(int(d) for d in ext[k]), int(modes[k])
        rows = inputs.sample_rows(seed * 10000 + k, dims[mode], 4)
        slabs = np.stack([ins[k][0].select(mode, int(r)).cpu().numpy().ravel() for r in rows])
        ref = oracle.mttkrp_rows(dims, mode, slabs, [f.cpu().numpy() for f in facs[k]])
        errs.append(oracle.rel_error(outs[k][torch.from_numpy(rows).cuda()].cpu().numpy(), ref))
    with clk.region("c3_baselines"):
        bplain = dz.Batch(einsums, extents, "plain")
        t_plain = _events_ms(stream, lambda: bplain(ins, outs, stream=stream), 2, warm=1)
        plans = [dz.Plan(e, x, "float32", "split_bf16") for e, x in zip(einsums, extents)]
        t_sep = _events_ms(stream, lambda: [p(*i, out=o, stream=stream) for p, i, o in zip(plans, ins, outs)], 2,
                           warm=1)
    gb = info["alg_bytes"] / 1e9
    xb = sum(4.0 * float(np.prod(e[:3])) for e in extents)
    del ins, outs, facs, bsplit, bplain, plans
    torch.cuda.empty_cache()
    return {"workload": f"{n} order-3 MTTKRP instances, extents U{{32..384}}, R in {{8,16,32,64}}, mode U{{0,1,2}}, "
                        "X uniform[-1,1) float32, one graph-replayed persistent split-BF16 batch "
                        "(Batch.bind: pointers marshalled once)",
            "metric": "GB/s", "value": gb / (t_batch * 1e-3), "unit": "GB/s", "ms_per_step": t_batch,
            "roofline": {"bound": "hbm", "kernel": "mttkrp_tc_batched_kernel (whole batch)",
                         "achieved": xb / (t_batch * 1e-3) / 1e9, "peak": peak,
                         "frac": xb / (t_batch * 1e-3) / 1e9 / peak, "x_gb": xb / 1e9},
            "separate_plain_launches_ms": t_plain, "separate_split_executes_ms": t_sep,
            "speedup_vs_plain_launches": t_plain / t_batch, "speedup_vs_separate_split": t_sep / t_batch,
            "launches_per_step": launches, "units": info["units"], "unit_div_autotuned": info["unit_div"],
            "autotune_best_ms": tune_ms, "rel_err": max(errs), "sample": "4 rows of every 32nd instance",
            "device_status": status, "clocks_region": "c3"}


def measure_c4_serving(clk, n_req=64):
    """CP-ALS serving: Poisson arrivals of requests (extents U{64..1024}, R U{8..64}, rank-R CP
    N(0,1) + 1e-2 noise, 10 sweeps), continuous batching in 4 slots at the measured
    one-at-a-time split-BF16 service rate, against one-at-a-time plain FP32 solves at the same
    arrival rate."""
    import torch
    budget = 64 << 30
    reqs = _serving_requests(n_req, 7)
    torch.cuda.synchronize()
    _serve_run(reqs[:4], 1, "split_bf16", None, budget, 1)            # warm-up
    with clk.region("c4"):
        span1, lat1, _, st1, _ = _serve_run(reqs, 1, "split_bf16", None, budget, 1)
        mu = len(reqs) / span1
        span, lat, gen, st, fits = _serve_run(reqs, 4, "split_bf16", mu, budget, 11)
    with clk.region("c4_plain"):
        spanp, latp, _, stp, _ = _serve_run(reqs, 1, "plain", mu, budget, 11)
    return {"workload": f"{n_req} Poisson CP-ALS requests: extents U{{64..1024}}, R U{{8..64}}, rank-R CP N(0,1) "
                        "+ 1e-2 noise, 10 sweeps, HBM budget 64 GiB, 4 slots, arrival rate = one-at-a-time rate",
            "metric": "req/s", "value": len(reqs) / span, "unit": "req/s",
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "one_at_a_time_split": {"req_s": mu, "p50_ms": 1e3 * float(np.percentile(lat1, 50)),
                                    "p99_ms": 1e3 * float(np.percentile(lat1, 99))},
            "one_at_a_time_plain_at_same_rate": {"req_s": len(reqs) / spanp,
                                                 "p50_ms": 1e3 * float(np.percentile(latp, 50)),
                                                 "p99_ms": 1e3 * float(np.percentile(latp, 99))},
            "ok": int(sum(x == 0 for x in st)), "fit_min": float(min(fits)),
            "clocks_region": "c4"}


def measure_cpals_sweep(clk, sweeps=4):
    """CP-ALS sweeps on X 1024^3 = rank-32 CP + 1e-2 noise, R 32, split-BF16: steady-state
    ms per sweep with the dimension tree (two X streams) and with three MTTKRPs."""
    import torch
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    n, R, seed = 1024, 32, 77
    dims = (n, n, n)
    A = [torch.from_numpy(inputs.factor_normal(seed, m, n, R, stream_base=inputs.STREAM_CP).astype(np.float32)).cuda()
         for m in range(3)]
    X = dz.gen_cp(seed, dims, A, 1e-2)
    init = [torch.from_numpy(inputs.factor_normal(seed, m, n, R, stream_base=inputs.STREAM_INIT).astype(np.float32))
            .cuda() for m in range(3)]
    stream = torch.cuda.Stream()
    res = {}
    with clk.region("cpals"):
        for tree in (True, False):
            cp = dz.CPALS(dims, R, "split_bf16")
            cp.set_dimension_tree(tree)
            t = {}
            with host_gc_paused(), torch.cuda.stream(stream):
                F = [u.clone() for u in init]
                cp.run(X, F, 1, stream=stream)
                for S in (1, sweeps):
                    F = [u.clone() for u in init]
                    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                    e0.record(stream)
                    lam, fits = cp.run(X, F, S, stream=stream)
                    e1.record(stream)
                    stream.synchronize()
                    t[S] = e0.elapsed_time(e1)
            per = (t[sweeps] - t[1]) / (sweeps - 1)
            res[tree] = (per, float(fits[-1]), cp.status())
    del X
    torch.cuda.empty_cache()
    return {"workload": "CP-ALS on X 1024^3 FP32 = rank-32 CP + 1e-2 noise, R 32, split-BF16 MTTKRPs, FP64 solves",
            "metric": "ms per steady-state sweep", "value": res[True][0], "unit": "ms", "higher_is_better": False,
            "dimension_tree": {"ms_per_sweep": res[True][0], "final_fit": res[True][1], "status": res[True][2]},
            "three_mttkrps": {"ms_per_sweep": res[False][0], "final_fit": res[False][1], "status": res[False][2]},
            "speedup": res[False][0] / res[True][0], "clocks_region": "cpals"}


def _standalone(measure, *a, **kw):
    """Run one per-configuration measurement alone and print its record as a JSON line."""
    import torch
    torch.cuda.set_device(0)
    clk = ClockSampler(0)
    clk.start()
    rec = measure(clk, *a, **kw)
    clk.stop()
    _fill_clocks(clk, rec)
    rec["n_gpus"] = 1
    rec["data"] = "synthetic"
    print(json.dumps(rec))
    return 0


def _fill_clocks(clk, rec):
    if "clocks_region" in rec:
        rec["clocks"] = clk.region_stats(rec.pop("clocks_region"))


def run_batched(args):
    return _standalone(measure_c3_batched, _peaks()[0], n=args.instances, reps=args.steps)


def run_ttmc(args):
    return _standalone(measure_c2b_ttmc, _peaks()[0], reps=args.steps)


def run_cpals(args):
    return _standalone(measure_cpals_sweep, sweeps=max(4, args.steps))


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    steps_v, total_s, total_rows, cores = [], 0.0, 0, 1
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for s in range(args.warmup + args.steps):
        gbs, sec, rows, cores = cpu_oracle_sample(100 + s, per_step)
        if s >= args.warmup:
            steps_v.append(gbs)
            total_s += sec
            total_rows += rows
    value = float(np.mean(steps_v))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "MTTKRP order-3 1024^3 FP32 uniform[-1,1), R=32 N(0,1/32), modes 0,1,2",
                       "sample": "FP64 oracle on sampled output rows"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{total_rows} sampled output rows over modes 0,1,2 "
                                       f"({total_s:.1f} s of oracle time)"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="split_bf16", choices=["split_bf16", "plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="only the benchmark configuration (skip the per-configuration records)")
    ap.add_argument("--once", action="store_true",
                    help="profiling driver: one execute per mode of --modes at extent --n, no timing")
    ap.add_argument("--n", type=int, default=N_EXT, help="extent of each mode (--once only)")
    ap.add_argument("--modes", default="0,1,2", help="modes to run (--once only)")
    ap.add_argument("--x-offset", type=int, default=0,
                    help="--once: X starts this many floats into its buffer (rows not 16-byte aligned)")
    ap.add_argument("--workload", default="mttkrp", choices=["mttkrp", "serving", "batched", "ttmc", "paper", "cpals", "unaligned"],
                    help="mttkrp: the benchmark line; serving / batched / ttmc: the other measurements")
    ap.add_argument("--requests", type=int, default=128, help="requests of the serving workload")
    ap.add_argument("--instances", type=int, default=512, help="instances of the batched workload")
    args = ap.parse_args()
    if args.once:
        return run_once(args)
    if args.workload == "serving" and args.impl == "native":
        return run_serving(args)
    if args.workload == "batched" and args.impl == "native":
        return run_batched(args)
    if args.workload == "unaligned" and args.impl == "native":
        return run_unaligned(args)
    if args.workload == "ttmc" and args.impl == "native":
        return run_ttmc(args)
    if args.workload == "paper" and args.impl == "native":
        return run_paper(args)
    if args.workload == "cpals" and args.impl == "native":
        return run_cpals(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2206_08301_gb300 as dz
    from paper_2206_08301_gb300 import inputs
    import oracle

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    seed = 2024 + rank
    dims = (N_EXT,) * 3
    stream = torch.cuda.Stream()
    X = dz.gen_uniform(seed, inputs.STREAM_X, dims)
    Us = [inputs.factor_normal(seed, m, N_EXT, RANK_R, sigma=np.sqrt(1.0 / RANK_R)).astype(np.float32)
          for m in range(3)]
    Ud = [torch.from_numpy(u).cuda() for u in Us]
    plans, outs = {}, {}
    for mode in MODES:
        spec = dz.mttkrp_einsum(3, mode)
        plans[mode] = dz.Plan(spec, list(dims) + [RANK_R], "float32", args.prec)
        outs[mode] = torch.empty(N_EXT, RANK_R, device="cuda")
    torch.cuda.synchronize()

    def step(strm):
        for mode in MODES:
            plans[mode](X, *[Ud[m] for m in range(3) if m != mode], out=outs[mode], stream=strm)

    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with host_gc_paused(), torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(stream)
        stream.synchronize()
        for p in plans.values():
            p.set_kernel_timing(True)
            p.kernel_time()
        launches0 = dz.kernel_launch_count()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            step(stream)
        ev1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    clocks.mark_stop()
    if dist:
        dist.barrier()
    launches = dz.kernel_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    kern_ms, kern_n = 0.0, 0
    for p in plans.values():
        a, b = p.kernel_time()
        kern_ms += a
        kern_n += b
        p.set_kernel_timing(False)
    status = max(p.last_device_status() for p in plans.values())
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    bytes_step = len(MODES) * _alg_bytes_one_mode()
    value = world * bytes_step * args.steps / (ms * 1e-3) / 1e9

    # accuracy on sampled rows (FP64 oracle, host) -- the metric is valid only at rel.err <= 1e-5
    rel_err = None
    if rank == 0:
        errs = []
        for mode in MODES:
            rows = inputs.sample_rows(seed, N_EXT, 64, tag=mode)
            slabs = np.stack([inputs.uniform_slab(seed, dims, mode, int(r)).ravel() for r in rows])
            ref = oracle.mttkrp_rows(dims, mode, slabs, Us)
            got = outs[mode][torch.from_numpy(rows).cuda()].cpu().numpy()
            errs.append(oracle.rel_error(got, ref))
        rel_err = max(errs)

    peak, peak_kind = _peaks()
    workloads = {}
    run_wl = rank == 0 and world == 1 and not args.no_workloads
    if run_wl:   # the plain FP32 arm of this configuration, while X is resident
        workloads["c1_mttkrp_1024cubed_plain_fp32"] = measure_c1_plain(clocks, X, Ud, Us, seed, peak)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        Xh = torch.empty(dims, dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        Uh = [torch.from_numpy(u).pin_memory() for u in Us]
        Oh = [torch.empty(N_EXT, RANK_R, pin_memory=True) for _ in MODES]
        Xd = torch.empty_like(X)
        Udd = [torch.empty_like(u) for u in Ud]
        del X
        torch.cuda.empty_cache()

        def e2e_step(strm):
            Xd.copy_(Xh, non_blocking=True)
            for d, h in zip(Udd, Uh):
                d.copy_(h, non_blocking=True)
            for mode in MODES:
                plans[mode](Xd, *[Udd[m] for m in range(3) if m != mode], out=outs[mode], stream=strm)
                Oh[mode].copy_(outs[mode], non_blocking=True)

        with torch.cuda.stream(stream):
            for _ in range(2):
                e2e_step(stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                e2e_step(stream)
            e1.record(stream)
        stream.synchronize()
        ems = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ems], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        h2d = Xh.numel() * 4 + sum(u.numel() * 4 for u in Uh)
        d2h = sum(o.numel() * 4 for o in Oh)
        e2e = {"value": world * bytes_step * args.steps / (ems * 1e-3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems / args.steps}

    if run_wl:   # every other configuration, each with its own timed region and clock record
        for key, fn, kw in (("c0_mttkrp_64cubed_fp64", measure_c0_fp64, {}),
                            ("c2a_mttkrp_64pow5_r24_modes_0_2", measure_c2a_order5, {"peak": peak}),
                            ("c2b_ttmc_256pow4_r32", measure_c2b_ttmc, {"peak": peak}),
                            ("ttmc_o5_m0_60pow5_r24", measure_ttmc_o5, {"peak": peak}),
                            ("c3_batched_512_instances", measure_c3_batched, {"peak": peak}),
                            ("c4_cpals_serving", measure_c4_serving, {}),
                            ("cpals_sweep_1024cubed_r32", measure_cpals_sweep, {})):
            try:
                workloads[key] = fn(clocks, **kw)
            except Exception as exc:   # report, never hide, a failed measurement
                workloads[key] = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gbs, sec, rows, cores = cpu_oracle_sample(seed, 15.0)
        gbs1, sec1, rows1, _ = cpu_oracle_sample(seed + 1, 8.0, threads=1)
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle on {rows} sampled output rows over modes 0,1,2 of the same "
                         f"workload ({sec:.1f} s); GB/s of X covered",
               "single_core": {"value": gbs1, "unit": "GB/s", "cores": 1,
                               "sample": f"{rows1} sampled output rows ({sec1:.1f} s)"}}

    clk = clocks.stop()
    for rec in workloads.values():
        _fill_clocks(clocks, rec)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    kern_avg_ms = kern_ms / max(1, kern_n)
    achieved = _alg_bytes_one_mode() / (kern_avg_ms * 1e-3) / 1e9 if kern_n else None
    traffic = _traffic_per_launch(args.prec)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "MTTKRP order-3 X 1024^3 FP32 uniform[-1,1), R=32 factors N(0,1/32), "
                               "modes 0,1,2 per step",
                   "arith": ("split-BF16 hi/lo operands on tcgen05 tensor cores, FP32 accumulation"
                             if args.prec == "split_bf16" else "FP32 FMA on CUDA cores"),
                   "l2": "inputs larger than L2 (X = 4.3 GB)", "rel_err_vs_fp64_oracle": rel_err,
                   "percent_of_roofline_8TBs": 100.0 * value / 8000.0},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "mttkrp_tc_kernel" if args.prec == "split_bf16" else "mttkrp_plain_kernel",
                     "kernel_ms_avg": kern_avg_ms, "peak_kind": peak_kind},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "device_status": status,
    }
    if workloads:
        line["workloads"] = workloads
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
