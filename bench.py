#!/usr/bin/env python
"""Benchmark of sketched ANLS (DSANLS hot path) on one GB300 per rank.

Workload (default ``dense_gaussian``): the dense image-like precision study --
planted M = U0 V0^T + |N(0, 0.01^2)| of 65,536 x 16,384 (U0, V0 ~ U[0,1) with
70% zeros, k = 64), rank 64, Gaussian sketch d = d' = 2048, projected-gradient
step.  A "step" is one outer iteration (U-half + V-half) replayed as a CUDA
graph; the metric is outer iterations per second.  With N ranks each rank runs
its own replica (independent problem, seed = rank): weak scaling, no
collective on the data path.

Also printed on the same JSON line:
  roofline      the dominant kernel (the sketched product A = M S) timed with
                CUDA events on the handle's stream right after the timed region
  cpu_baseline  the FP64 oracle on a bounded row sample, extrapolated
  e2e           the same metric through the public API with host buffers
                (upload of M from pinned memory, one iteration, factors back)
  clocks        nvidia-smi samples taken during the timed region

``--impl reference`` times the FP64 CPU oracle on the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sketched-ANLS outer iters/s and time-to-ε (rel. Frobenius err) vs plain FP32"
UNIT = "outer_iters/s"

WORKLOADS = {
    "dense_gaussian": dict(m=65536, n=16384, k=64, d=2048, d_v=2048, sketch=0, zero_frac=0.7, noise=0.01,
                           desc="dense 65536x16384 planted (k=64, 70% zero factors, |N(0,0.01^2)| noise), "
                                "Gaussian sketch d=d'=2048, PGD"),
    "dense_gaussian_reassoc": dict(m=65536, n=16384, k=64, d=2048, d_v=2048, sketch=0, zero_frac=0.7, noise=0.01,
                                   order=1,
                                   desc="dense 65536x16384 planted (k=64), Gaussian sketch d=d'=2048, PGD, "
                                        "reassociated order R = M (S B^T)"),
    "dense_subsample": dict(m=65536, n=16384, k=64, d=2048, d_v=2048, sketch=1, zero_frac=0.7, noise=0.01,
                            desc="dense 65536x16384 planted (k=64), subsampling sketch d=d'=2048, PGD"),
    "dense_gaussian_8k": dict(m=8192, n=16384, k=64, d=2048, d_v=2048, sketch=0, zero_frac=0.7, noise=0.01,
                              desc="dense 8192x16384 planted (k=64), Gaussian sketch d=d'=2048, PGD "
                                   "(profiling case: M 0.5 GB)"),
    "sparse_text": dict(m=2_000_000, n=500_000, k=100, d=5000, d_v=5000, sketch=1, sparse=True,
                        desc="CSR 2e6 docs x 5e5 terms (lognormal lengths mean 100, Zipf 1.07 ids, "
                             "log(1+Poisson) values, ~1.4e8 nnz), k=100, subsampling d=d'=5000, PGD "
                             "(--precision bf16: bf16 factors)"),
    "sparse_text_small": dict(m=200_000, n=50_000, k=100, d=500, d_v=500, sketch=1, sparse=True,
                              desc="CSR 2e5 x 5e4 text-like (~1.3e7 nnz), k=100, subsampling d=d'=500, PGD"),
    "learned": dict(learned=True, m=65536, n=16384, k=32, d=2048, d_v=2048, sketch=0, eps=0.05, t_max=400,
                    desc="dense 65536x16384 planted (k=32, 70% zero factors), Gaussian d=2048, PGD; network trained "
                         "on ~1e7 triples harvested from seeds 1-20, evaluated on seed 21 to rel. error 0.05"),
    "batched": dict(batched=True, count=1024, m=0, n=0, k=0, d=0, d_v=0, sketch=0,
                    desc="1024 uneven planted instances (m in [128,4096], n in [64,2048], k in {8,16,32}), "
                         "Gaussian d=max(4k,n/8), d'=max(4k,m/8), PGD"),
    "batched_small": dict(batched=True, count=64, m=0, n=0, k=0, d=0, d_v=0, sketch=0,
                          desc="64 uneven planted instances (same recipe)"),
    "dense_identity": dict(m=65536, n=16384, k=64, d=16384, d_v=65536, sketch=2, zero_frac=0.7, noise=0.01,
                           desc="dense 65536x16384 planted (k=64), identity sketch (unsketched subproblem; "
                                "with --solver rcd --alpha 0 --beta 0 this is HALS)"),
    "compare": dict(compare=True, m=65536, n=16384, k=64, d=2048, d_v=2048, sketch=0, zero_frac=0.7, noise=0.01,
                    eps=0.05, t_max=600,
                    desc="dense 65536x16384 planted (k=64, 70% zero factors): iterations and time to rel. error "
                         "0.05 of sketched and unsketched forms on the same kernels"),
    "small": dict(m=1000, n=800, k=10, d=100, d_v=100, sketch=0, zero_frac=0.0, noise=0.01,
                  desc="planted 1000x800, k=10, Gaussian d=100, PGD"),
}

# FP32 CUDA-core peak of a GB300: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2.070 GHz.
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def max_over_ranks(ms, ws, device="cuda"):
    """The job's time: the maximum of the per-rank durations (all ranks)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, steps, ms):
    """Whole-job throughput: outer iterations of every replica per second."""
    return ws * steps / (ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def make_inputs(w, seed):
    """Dense M (float32 ndarray) or a CSR triple (rowptr, col, val)."""
    if w.get("sparse"):
        from synthdata import sparse_text
        return sparse_text(w["m"], w["n"], seed)
    from synthdata import planted_dense
    M, _, _ = planted_dense(w["m"], w["n"], w["k"], seed, zero_frac=w["zero_frac"], noise=w["noise"])
    return M


def _input_bytes(M):
    return int(sum(a.nbytes for a in M)) if isinstance(M, tuple) else int(M.nbytes)


def _set_data(h, M):
    if isinstance(M, tuple):
        h.set_csr(*M)
    else:
        h.set_dense(M)


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(M, w, seed, rows_budget):
    """Time the FP64 oracle on one outer iteration restricted to `rows_budget`
    rows per half and extrapolate linearly in rows (the row-independent part:
    the sketch, B = Y^T S and G are computed in full).  Returns (iters/s, desc)."""
    from oracle import method
    m, n, k = w["m"], w["n"], w["k"]
    U0, V0 = method.default_init(seed, m, n, k)
    U0 = U0.astype(np.float64)
    V0 = V0.astype(np.float64)
    mu = method.mu_t(1.0, 1.0, 0)
    total = 0.0
    for side, K, rows_all, dd in ((0, n, m, w["d"]), (1, m, n, w["d_v"])):
        r = min(rows_all, rows_budget)
        rows = np.arange(r)
        t0 = time.perf_counter()
        S = method.Sketch(w["sketch"], seed, 0, side, K, dd)
        Y = V0 if side == 0 else U0
        if w["sketch"] in method.DENSE_KINDS:
            B = Y.T @ S.dense32.astype(np.float64)
        else:
            B = (Y[S.J, :] * np.float64(S.scale)).T
        G = B @ B.T
        lam = method.lambda_max(G)
        P = S.dense() @ B.T if w.get("order") == 1 else None  # reassociated order: P = S B^T in full
        t1 = time.perf_counter()
        if isinstance(M, tuple):
            import scipy.sparse as sp
            Msp = sp.csr_matrix((M[2].astype(np.float64), M[1], M[0]), shape=(m, n))
            X = Msp[rows] if side == 0 else Msp[:, rows].T.tocsr()
        else:
            X = M[rows].astype(np.float64) if side == 0 else M[:, rows].T.astype(np.float64)
        R = X @ P if P is not None else S.right_multiply(X) @ B.T
        Z = (U0 if side == 0 else V0)[rows]
        method.pgd_update(Z, G, R, 1.0 / (lam + mu))
        t2 = time.perf_counter()
        total += (t1 - t0) + (t2 - t1) * rows_all / r
    desc = "FP64 oracle, one outer iteration on %d rows per half, extrapolated to %dx%d" % (
        min(rows_budget, m), m, n)
    return 1.0 / total, desc


def _cores():
    """Host cores this process may run on (what `nproc` prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _openblas_libs():
    """The OpenBLAS libraries loaded into this process (numpy's and scipy's)."""
    import ctypes
    paths = set()
    try:
        with open("/proc/self/maps") as f:
            for line in f:
                part = line.split()
                if len(part) >= 6 and "openblas" in part[-1].lower() and part[-1].startswith("/"):
                    paths.add(part[-1])
    except OSError:
        pass
    libs = []
    for path in sorted(paths):
        try:
            libs.append(ctypes.CDLL(path))
        except OSError:
            pass
    return libs


_BLAS_PREFIXES = ("scipy_openblas", "openblas")
_BLAS_SUFFIXES = ("64_", "")


def _blas_call(libs, what, *args):
    out = []
    for lib in libs:
        for pre in _BLAS_PREFIXES:
            for suf in _BLAS_SUFFIXES:
                fn = getattr(lib, "%s_%s%s" % (pre, what, suf), None)
                if fn is not None:
                    out.append(fn(*args))
                    break
            else:
                continue
            break
    return out


def _blas_threads():
    n = _blas_call(_openblas_libs(), "get_num_threads")
    return int(max(n)) if n else None


def oracle_single_thread(M, w, seed, rows_budget):
    """The same bounded oracle sample with the BLAS limited to one thread (the
    rest of the oracle is single-threaded already); None when no OpenBLAS is
    loaded to limit."""
    libs = _openblas_libs()
    before = _blas_call(libs, "get_num_threads")
    if not before:
        return None
    _blas_call(libs, "set_num_threads", 1)
    try:
        v, desc = oracle_sample(M, w, seed, rows_budget)
    finally:
        _blas_call(libs, "set_num_threads", int(max(before)))
    return {"value": v, "unit": UNIT, "cores": 1, "sample": desc}


def run_reference(args, w):
    ws, rank, local = _dist()
    if rank != 0:
        return
    M = make_inputs(w, 0)
    rows = 512 if w["m"] > 10000 else w["m"]
    for _ in range(args.warmup):
        oracle_sample(M, w, 0, rows)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc = oracle_sample(M, w, 0, rows)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(statistics.mean(vals))
    single = oracle_single_thread(M, w, 0, min(rows, 128))
    # a step is the timed row sample: ms_per_step is its measured wall time, and
    # value the full iteration's rate extrapolated from it
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "value_source": "extrapolated in rows from the timed sample (ms_per_step is the sample's wall time)",
        "ms_per_full_iteration": 1000.0 / value,
        "config": {"workload": args.workload, "desc": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"],
                   "d": w["d"], "d_v": w["d_v"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "blas_threads": _blas_threads(),
                         "kind": "oracle", "sample": desc, "single_thread": single},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _traffic(kernel_key, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        table = json.load(f)
    ent = table.get(kernel_key, {}).get(workload)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2009_02845_gb300", "csrc", ent["source"])
    if not os.path.exists(src):
        return None
    text = open(src, "rb").read()
    marker = ent.get("source_end_marker")
    if marker:  # only the part of the file that holds the kernel (it ends at the marker)
        cut = text.find(marker.encode())
        if cut < 0:
            return None
        text = text[:cut]
    h = hashlib.sha256(text).hexdigest()[:16]
    return ent["bytes_per_launch"] if h == ent["source_sha"] else None


def time_to_eps(pkg, torch, M, w, T, check_every, stream):
    """Relative error every `check_every` outer iterations for the plain FP32
    path and for the bf16 form with its last 3 iterations in FP32; eps is the
    FP32 path's error after T iterations + 1e-3.  Times are CUDA-event sums of
    the steps alone (error evaluations excluded)."""
    def trajectory(prec_plan, order=0, inner=1):
        h = pkg.DSANLS(w["m"], w["n"], w["k"], w["d"], w["sketch"], seed=0, d_v=w["d_v"], solver=pkg.PGD,
                       precision=prec_plan[0], use_graph=1, order=order, inner_iters=inner)
        h.set_dense(M)
        errs, total_ms = [], 0.0
        for it in range(T):
            prec = prec_plan[1] if it >= T - 3 else prec_plan[0]
            if prec != prec_plan[0] and it == T - 3:
                h.set_options(precision=prec, order=0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(1)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            if (it + 1) % check_every == 0 or it == T - 1:
                errs.append((it + 1, total_ms, h.rel_error()))
        h.close()
        return errs

    fp32 = trajectory((pkg.FP32, pkg.FP32))
    eps = fp32[-1][2] + 1e-3
    forms = {"bf16_closing_fp32": trajectory((pkg.BF16, pkg.FP32)), "fp8_closing_fp32": trajectory((pkg.FP8, pkg.FP32)),
             "bf16_reassociated_closing_fp32": trajectory((pkg.BF16, pkg.FP32), order=1),
             "bf16_reassociated_inner16_closing_fp32": trajectory((pkg.BF16, pkg.FP32), order=1, inner=16),
             "fp8_reassociated_closing_fp32": trajectory((pkg.FP8, pkg.FP32), order=1),
             "fp8_reassociated_inner16_closing_fp32": trajectory((pkg.FP8, pkg.FP32), order=1, inner=16)}

    def first_hit(tr):
        for it, ms, e in tr:
            if e <= eps:
                return {"iters": it, "seconds": ms / 1000.0, "err": e}
        return None

    a = first_hit(fp32)
    out = {"eps": eps, "T": T, "checked_every": check_every,
           "fp32": {"to_eps": a, "final_err": fp32[-1][2], "seconds_T": fp32[-1][1] / 1000.0}}
    for name, tr in forms.items():
        b = first_hit(tr)
        out[name] = {"to_eps": b, "final_err": tr[-1][2], "seconds_T": tr[-1][1] / 1000.0,
                     "speedup_time_to_eps": (a["seconds"] / b["seconds"]) if (a and b) else None}
    # the FP64 oracle's trajectory of the same problem (written offline by
    # tests/golden/make_dense_trajectory.py): the final error of every form against it
    gold = os.path.join(ROOT, "tests", "golden", "dense_%dx%d_k%d_d%d_gaussian_pgd_T%d.json" % (
        w["m"], w["n"], w["k"], w["d"], T))
    if os.path.exists(gold) and w.get("zero_frac") == 0.7 and w["sketch"] == 0 and w["d_v"] == w["d"]:
        ge = json.load(open(gold))["errors"]
        out["oracle_fp64"] = {"final_err": ge[T - 1], "source": os.path.relpath(gold, ROOT)}
        out["fp32"]["max_abs_diff_vs_oracle"] = max(abs(e - ge[it - 1]) for it, _, e in fp32)
        for name in ["fp32"] + list(forms):
            out[name]["final_minus_oracle"] = out[name]["final_err"] - ge[T - 1]
    return out


def time_to_eps_sparse(pkg, torch, M, w, T, check_every, stream):
    """Sparse data (subsampling sketch): the FP32 path against the bf16-factor form
    with its last 3 iterations in FP32, as time_to_eps does for dense data; eps is
    the FP32 path's error after T iterations + 1e-3."""
    def trajectory(prec_plan):
        h = pkg.DSANLS(w["m"], w["n"], w["k"], w["d"], w["sketch"], seed=0, d_v=w["d_v"], solver=pkg.PGD,
                       precision=prec_plan[0], use_graph=1)
        h.set_csr(*M)
        errs, total_ms = [], 0.0
        for it in range(T):
            if prec_plan[1] != prec_plan[0] and it == T - 3:
                h.set_options(precision=prec_plan[1])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(1)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            if (it + 1) % check_every == 0 or it == T - 1:
                errs.append((it + 1, total_ms, h.rel_error()))
        h.close()
        return errs

    fp32 = trajectory((pkg.FP32, pkg.FP32))
    eps = fp32[-1][2] + 1e-3
    bf16 = trajectory((pkg.BF16, pkg.FP32))

    def first_hit(tr):
        for it, ms, e in tr:
            if e <= eps:
                return {"iters": it, "seconds": ms / 1000.0, "err": e}
        return None

    a, b = first_hit(fp32), first_hit(bf16)
    return {"eps": eps, "T": T, "checked_every": check_every,
            "fp32": {"to_eps": a, "final_err": fp32[-1][2], "seconds_T": fp32[-1][1] / 1000.0},
            "bf16_factors_closing_fp32": {"to_eps": b, "final_err": bf16[-1][2], "seconds_T": bf16[-1][1] / 1000.0,
                                          "speedup_time_to_eps": (a["seconds"] / b["seconds"]) if (a and b) else None}}


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    import paper_2009_02845_gb300 as pkg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    prec = {"fp32": pkg.FP32, "bf16": pkg.BF16, "fp8": pkg.FP8}[args.precision]
    if (w.get("sparse") and prec != pkg.BF16) or (w["sketch"] == 1 and not w.get("sparse")) or \
            (w["sketch"] == 2 and prec == pkg.FP8):
        # the tensor-core forms serve dense data with a dense (or, bf16, identity) sketch;
        # sparse data runs in FP32 or with bf16 factors (BF16)
        prec = pkg.FP32
    M = make_inputs(w, rank)
    # all library work and all timing events on one dedicated (non-default) stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    order = w.get("order", 0)
    solver = {"pgd": pkg.PGD, "rcd": pkg.RCD}[args.solver]
    h = pkg.DSANLS(w["m"], w["n"], w["k"], w["d"], w["sketch"], seed=rank, d_v=w["d_v"], solver=solver,
                   precision=prec, use_graph=1, order=order, alpha=args.alpha, beta=args.beta,
                   inner_iters=args.inner_iters, regen_sketch=int(args.regen_sketch))
    _set_data(h, M)

    for _ in range(args.warmup):
        h.step(1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = pkg.kernel_launches()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        h.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = pkg.kernel_launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws)
    value = job_value(ws, args.steps, ms)
    err = h.rel_error()

    # dominant kernel: the sketched product of each half, timed per phase
    phases = [h.profile_half_step(0, reps=2), h.profile_half_step(1, reps=2)]
    peaks, peak_src = _peaks()
    m, n, d, d_v, k = w["m"], w["n"], w["d"], w["d_v"], w["k"]
    dense_sketch = w["sketch"] in (0, 3, 4, 5)  # Gaussian, Rademacher, count, SRHT: S a dense matrix
    if (dense_sketch and order == 1) or (w["sketch"] == 2 and not w.get("sparse")):
        # reassociated order (R = X P) or identity sketch (R = X Y): the streaming
        # product reads X once (bf16 or fp32) and the k x K factor, and writes R
        eb = {pkg.BF16: 2.0, pkg.FP8: 1.0}.get(prec, 4.0)
        bytes_ = [eb * (m * n + k * n) + 4.0 * m * k, eb * (n * m + k * m) + 4.0 * n * k]
        flops = [2.0 * m * n * k, 2.0 * n * m * k]
        prod_ms = [p["rhs"] for p in phases]
        if prec in (pkg.BF16, pkg.FP8):
            achieved = sum(bytes_) / (sum(prod_ms) / 1000.0) / 1e9
            bound, peak, unit = "hbm", peaks["hbm_gbs"], "GB/s"
            kernel_key = "tc_skinny" if prec == pkg.BF16 else "tc_skinny_fp8"
            peak_note = "hbm_gbs of %s" % peak_src
        elif m % 8 == 0 and n % 8 == 0 and dense_sketch:
            # FP32 on tensor cores: the streaming product reads the three bf16 parts of X
            # (6 bytes per entry) and the parts of P^T
            bytes_ = [6.0 * (m * n + k * n) + 4.0 * m * k, 6.0 * (n * m + k * m) + 4.0 * n * k]
            achieved = sum(bytes_) / (sum(prod_ms) / 1000.0) / 1e9
            bound, peak, unit, kernel_key = "hbm", peaks["hbm_gbs"], "GB/s", "tc_skinny_split3"
            peak_note = "hbm_gbs of %s (bytes of the three bf16 parts of X)" % peak_src
        else:
            achieved = sum(flops) / (sum(prod_ms) / 1000.0) / 1e12
            bound, peak, unit, kernel_key = "alu", FP32_SIMT_PEAK_TFLOPS, "TFLOP/s", "sgemm_simt"
            peak_note = "FP32 CUDA-core peak 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz"
    elif dense_sketch:
        flops = [2.0 * m * n * d, 2.0 * n * m * d_v]
        if prec != pkg.FP32:
            flops = [f + 2.0 * m * d * k for f in flops]  # R = A B^T is fused into the same kernel
        prod_ms = [p["product"] for p in phases]
        achieved = sum(flops) / (sum(prod_ms) / 1000.0) / 1e12
        if prec == pkg.BF16:
            # timed alone by profile_half_step right after the timed region: burst conditions
            bound, peak, unit, kernel_key = "tensor", peaks["bf16_tflops"], "TFLOP/s", "tc_sketch_rhs"
            peak_note = "bf16_tflops (burst) of %s: the kernel is timed alone by profile_half_step" % peak_src
        elif prec == pkg.FP8:
            bound, peak, unit, kernel_key = "tensor", 2.0 * peaks["bf16_tflops"], "TFLOP/s", "tc_sketch_rhs_fp8"
            peak_note = ("2 x bf16_tflops (burst) of %s (nominal fp8:bf16 dense ratio 4.5:2.25); the kernel is "
                         "timed alone by profile_half_step" % peak_src)
        elif m % 8 == 0 and n % 8 == 0:
            # binary32 accuracy from six bf16 tensor-core products of three-way splits:
            # the ceiling for the method's FP32 flops is a sixth of the bf16 peak
            bound, peak, unit, kernel_key = "tensor", peaks["bf16_tflops"] / 6.0, "TFLOP/s", "tc_gemm_split3"
            peak_note = ("bf16_tflops (burst) of %s / 6: A = X S as six bf16 products of three-way splits "
                         "(algorithmic FP32 flops 2 rows K d per half)" % peak_src)
        else:
            bound, peak, unit, kernel_key = "alu", FP32_SIMT_PEAK_TFLOPS, "TFLOP/s", "sgemm_simt"
            peak_note = "FP32 CUDA-core peak 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz"
    elif not w.get("sparse"):
        # subsampling: the gathered product reads d columns of M^T per half
        bytes_ = [4.0 * (m * d + d * k) + 4.0 * m * k, 4.0 * (n * d_v + d_v * k) + 4.0 * n * k]
        prod_ms = [p["rhs"] for p in phases]
        achieved = sum(bytes_) / (sum(prod_ms) / 1000.0) / 1e9
        bound, peak, unit, kernel_key = "hbm", peaks["hbm_gbs"], "GB/s", "sgemm_simt_gather"
        peak_note = "hbm_gbs of %s" % peak_src
    else:
        # sparse subsampling: the row update forms the right-hand side of the sampled entries
        # itself -- it reads and writes Z (8 bytes per element; 4 with bf16 factors), the row
        # pointers (8 bytes per row) and sampled entries (8 bytes each; nnz d / K expected) of
        # the sub-CSR and the d sampled rows of the other factor (R only for the few rows of
        # more than 64 entries, not counted)
        zb = 4.0 if prec == pkg.BF16 else 8.0
        es = 2.0 if prec == pkg.BF16 else 4.0
        nnz = float(len(M[1]))
        bytes_ = [zb * m * k + 8.0 * m + 8.0 * nnz * d / n + es * d * k,
                  zb * n * k + 8.0 * n + 8.0 * nnz * d_v / m + es * d_v * k]
        prod_ms = [p["update"] for p in phases]
        achieved = sum(bytes_) / (sum(prod_ms) / 1000.0) / 1e9
        bound, peak, unit, kernel_key = "hbm", peaks["hbm_gbs"], "GB/s", "update"
        peak_note = "hbm_gbs of %s" % peak_src
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": _traffic(kernel_key, args.workload), "kernel": kernel_key, "peak_source": peak_note,
                "launch_ms": [round(x, 4) for x in prod_ms]}

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        Mp = tuple(torch.from_numpy(a).pin_memory() for a in M) if isinstance(M, tuple) else \
            torch.from_numpy(M).pin_memory()
        Uh = torch.empty((m, k), dtype=torch.float32).pin_memory()
        Vh = torch.empty((n, k), dtype=torch.float32).pin_memory()
        he = pkg.DSANLS(m, n, k, d, w["sketch"], seed=rank, d_v=d_v, solver=solver, precision=prec, use_graph=1,
                        order=order, alpha=args.alpha, beta=args.beta, inner_iters=args.inner_iters)

        def e2e_step():
            _set_data(he, Mp)
            he.step(1)
            he.factors()  # synchronising device->host read of U and V
        e2e_step()
        reps = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            e2e_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        he.close()
        e2e = {"value": 1.0 / dt, "unit": UNIT, "h2d_bytes_per_step": _input_bytes(M),
               "d2h_bytes_per_step": int((m + n) * k * 4),
               "note": "per step: set_dense/set_csr from pinned host memory, 1 outer iteration, "
                       "get_factors to host"}
        del Mp

    traj = None
    if rank == 0 and args.trajectory > 0:
        ht = pkg.DSANLS(m, n, k, d, w["sketch"], seed=rank, d_v=d_v, solver=solver, precision=prec, use_graph=1,
                        order=order, alpha=args.alpha, beta=args.beta, inner_iters=args.inner_iters)
        _set_data(ht, M)
        every = max(1, args.trajectory // 10)
        traj = [(0, ht.rel_error())]
        for it in range(1, args.trajectory + 1):
            ht.step(1)
            if it % every == 0 or it == args.trajectory:
                traj.append((it, ht.rel_error()))
        ht.close()

    tte = None
    if rank == 0 and args.time_to_eps > 0 and w["sketch"] == 0:
        tte = time_to_eps(pkg, torch, M, w, args.time_to_eps, 5, stream)
    elif rank == 0 and args.time_to_eps > 0 and w.get("sparse"):
        tte = time_to_eps_sparse(pkg, torch, M, w, args.time_to_eps, 5, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = (20000 if w.get("sparse") else 512) if m > 10000 else m
        v, desc = oracle_sample(M, w, rank, rows)
        cpu = {"value": v, "unit": UNIT, "cores": _cores(), "blas_threads": _blas_threads(), "kind": "oracle",
               "sample": desc, "single_thread": oracle_single_thread(M, w, rank, min(rows, 128))}

    h.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {pkg.FP32: "f32", pkg.BF16: "bf16", pkg.FP8: "e4m3"}[prec],
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n, "k": k, "d": d, "d_v": d_v,
                       "precision": {pkg.FP32: "fp32", pkg.BF16: "bf16", pkg.FP8: "fp8"}[prec], "solver": args.solver, "alpha": args.alpha, "beta": args.beta,
                       "inner_iters": args.inner_iters, "graph": True, "replicas": ws,
                       "sketch_in_gemm": bool(args.regen_sketch),
                       "order": ["paper", "reassociated"][order],
                       "l2": "inputs larger than L2 (M is %.1f GB)" % (_input_bytes(M) / 1e9)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "phases_ms": {"U": {k_: round(v_, 4) for k_, v_ in phases[0].items()},
                          "V": {k_: round(v_, 4) for k_, v_ in phases[1].items()}},
            "rel_error_after": err,
            "rel_error_trajectory": traj,
            "time_to_eps": tte,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dense_gaussian")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default=None,
                    help="arithmetic of the products (default: bf16; fp32 for the batched workloads)")
    ap.add_argument("--sketch", choices=["gaussian", "subsample", "rademacher", "count", "srht"], default=None,
                    help="sketch kind (default: the workload's)")
    ap.add_argument("--order", choices=["paper", "reassociated"], default=None,
                    help="order of R = M S B^T for Gaussian sketches (default: the workload's)")
    ap.add_argument("--solver", choices=["pgd", "rcd"], default="pgd")
    ap.add_argument("--inner-iters", type=int, default=1,
                    help="PGD steps per half-step on the proximal row objective (1: the paper's single step)")
    ap.add_argument("--alpha", type=float, default=1.0, help="mu_t = alpha + beta t")
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--regen-sketch", action="store_true",
                    help="BF16 paper order: draw the Gaussian sketch inside the GEMMs instead of a pre-pass")
    ap.add_argument("--batch-tile", default="",
                    help="batched bf16 paper order: pin the tensor-core tile 'chunk,stages,row_tiles[,pipeline]' "
                         "(e.g. 192,3,2; pipeline 0 cp.async ring, 1 TMA ring, 2 epilogue off the copy path) of both "
                         "halves, or 'U-tile/V-tile', instead of autotuning it")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-steps", type=int, default=6000, help="training steps of the learned workload")
    ap.add_argument("--trajectory", type=int, default=0,
                    help="also run T outer iterations on a fresh handle and report the relative error every "
                         "T/10 iterations (untimed)")
    ap.add_argument("--time-to-eps", type=int, default=100,
                    help="also run T outer iterations of the fp32 and bf16 forms and report time to eps")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.precision is None:
        args.precision = "fp32" if w.get("batched") else "bf16"
    if args.order is not None:
        w["order"] = ["paper", "reassociated"].index(args.order)
    if args.sketch is not None:
        w["sketch"] = {"gaussian": 0, "subsample": 1, "rademacher": 3, "count": 4, "srht": 5}[args.sketch]
    if w.get("learned"):
        run_learned(args, w)
    elif w.get("compare"):
        run_compare(args, w)
    elif w.get("batched"):
        run_batch(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


def run_learned(args, w):
    """Learned warm start on the dense 65536 x 16384, k = 32 planted problem:
    harvest (G, b, x*) triples from training seeds 1..20 (both halves at 15
    iterations spread over the first 300 of a plain bf16 run, 16384 rows per
    half-step, ~1e7 triples), train the network on the GPU, then run the
    held-out seed 21 to relative error eps with: the plain fp32 and bf16 paths
    (one projected-gradient step per half); the learned form (network point +
    PG_ITERS correction steps, fallback to the single plain step); bf16 with
    INNER plain steps per half (the correction without a network: the
    ablation); and the learned form whose fallback is that INNER-step update.
    Times are CUDA-event sums of the steps; errors are checked after every
    outer iteration."""
    import torch
    import paper_2009_02845_gb300 as pkg
    from synthdata import planted_dense_torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m, n, k, d = w["m"], w["n"], w["k"], w["d"]
    hidden, eps, t_max, seeds = 256, w["eps"], w["t_max"], list(range(1, 21))
    PG_ITERS, INNER = 16, 16
    points = [0, 1, 2, 3, 5, 8, 12, 18, 27, 40, 60, 90, 135, 200, 300]
    per_group = 16384
    net = pkg.MLP(k, hidden, max_rows=max(m, n), max_groups=64, seed=0)
    # -- harvest
    t0 = time.perf_counter()
    pool = []
    for seed in seeds:
        M = planted_dense_torch(m, n, k, seed, zero_frac=0.7)
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=seed, precision=pkg.BF16, use_graph=1)
        h.set_dense(M)
        t = 0
        for tp in points:
            if tp > t:
                h.step(tp - t)
            for side in (0, 1):
                G, mu, b, x = h.harvest(side, iters=300)
                sel = torch.randperm(b.shape[0], device="cuda")[:per_group]
                pool.append((G, mu, b[sel].contiguous(), x[sel].contiguous()))
                del b, x
                h.half_step(side)
            t = tp + 1
            h.set_options(t=t)
        h.close()
        del M
    triples = sum(p[2].shape[0] for p in pool)
    harvest_s = time.perf_counter() - t0

    def norm_target(G, mu, b, x):
        # y* = x* s / beta, s = tr(G + mu I) / k, beta = ||b|| / sqrt(k) (1 if zero)
        s_ = (torch.trace(G) + k * mu[0]) / k
        beta = b.norm(dim=1) / math.sqrt(k)
        beta = torch.where(beta > 0, beta, torch.ones_like(beta))
        return x * (s_ / beta)[:, None]

    def val_loss():
        # 1/2 mean ||y - y*||^2 in normalised units on the held-out groups (every 10th),
        # and the fraction of positive network outputs there
        tot, pos, cnt = 0.0, 0.0, 0
        for G, mu, b, x in pool[5::10]:
            bb, xx = b[-512:], x[-512:]
            off1 = torch.tensor([0, bb.shape[0]], dtype=torch.int64, device="cuda")
            pred = net.predict(G[None], mu, off1, bb)
            tot += 0.5 * float(((norm_target(G, mu, bb, pred) - norm_target(G, mu, bb, xx)) ** 2).sum(1).mean())
            pos += float((pred > 0).float().mean())
            cnt += 1
        return tot / cnt, pos / cnt

    ynorm = torch.cat([norm_target(G, mu, b, x).norm(dim=1) for G, mu, b, x in pool[5::10]])
    target_stats = {"p50": float(ynorm.median()), "p99": float(torch.quantile(ynorm.float(), 0.99)),
                    "max": float(ynorm.max()), "zero_loss": float(0.5 * (ynorm ** 2).mean())}
    val_before = val_loss()
    # -- train: 16 groups x 512 rows per step, Adam with a cosine learning rate
    t0 = time.perf_counter()
    g = np.random.default_rng(0)
    losses = []
    steps = args.train_steps
    groups, rows_per = 16, 512
    train_ids = np.array([i for i in range(len(pool)) if i % 10 != 5])
    for step in range(steps):
        pick = g.choice(train_ids, groups, replace=False)
        bs, xs = [], []
        for i in pick:
            r0 = int(g.integers(0, pool[i][2].shape[0] - rows_per + 1))
            bs.append(pool[i][2][r0:r0 + rows_per])
            xs.append(pool[i][3][r0:r0 + rows_per])
        G = torch.stack([pool[i][0] for i in pick])
        mu = torch.cat([pool[i][1] for i in pick])
        off = torch.arange(0, (groups + 1) * rows_per, rows_per, dtype=torch.int64, device="cuda")
        lr = 1e-5 + 0.5 * (1e-3 - 1e-5) * (1.0 + math.cos(math.pi * step / steps))
        losses.append(net.train_step(G, mu, off, torch.cat(bs), torch.cat(xs), lr))
    train_s = time.perf_counter() - t0
    val_after = val_loss()
    del pool
    # -- evaluate on the held-out seed
    from synthdata import planted_dense
    M, _, _ = planted_dense(m, n, k, 21, zero_frac=0.7)

    # a network with all parameters zero proposes x0 = 0: the learned form with it
    # measures what restarting the correction steps from zero gains by itself
    net0 = pkg.MLP(k, hidden, max_rows=max(m, n), max_groups=1, seed=0)
    net0.set_params(np.zeros(net0.n_params, np.float32))

    def run(prec, learned, inner=1, pg_iters=PG_ITERS, network=None):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=21, precision=prec, use_graph=1, inner_iters=inner)
        h.set_dense(M)
        if learned:
            h.set_mlp(network if network is not None else net, pg_iters=pg_iters)
        total, hist, hit = 0.0, [], None
        for it in range(t_max):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(1)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            err = h.rel_error()
            hist.append(err)
            if hit is None and err <= eps:
                hit = {"iters": it + 1, "seconds": total / 1000.0, "err": err}
                break
        kept = h.mlp_kept() if learned else None
        h.close()
        return {"to_eps": hit, "final_err": hist[-1], "iters_run": len(hist), "seconds_run": total / 1000.0,
                "ms_per_iter": total / len(hist), "rows_kept_learned": kept}

    # plain fp32 and bf16 (the paper's single step); bf16 with INNER steps from u
    # (the same correction without a network); the learned form with the network's
    # point corrected by PG_ITERS steps, falling back to the single plain step or
    # to the INNER-step plain update
    res = {"fp32_plain": run(pkg.FP32, False), "bf16": run(pkg.BF16, False),
           "bf16_learned": run(pkg.BF16, True, 1),
           "bf16_inner%d" % INNER: run(pkg.BF16, False, INNER),
           "bf16_learned_inner%d" % INNER: run(pkg.BF16, True, INNER),
           "bf16_zero_network_inner%d" % INNER: run(pkg.BF16, True, INNER, network=net0)}
    net0.close()
    base = res["fp32_plain"]["to_eps"]
    best = res["bf16_learned_inner%d" % INNER]["to_eps"]
    value = (1.0 / best["seconds"]) if best else 0.0
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "1/time_to_eps (1/s)", "n_gpus": ws, "steps": t_max,
        "warmup": 0, "ms_per_step": res["bf16_learned_inner%d" % INNER]["ms_per_iter"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n, "k": k, "d": d, "eps": eps,
                   "train_seeds": "1-20", "eval_seed": 21, "triples": triples, "train_steps": steps,
                   "harvest_iterations": points, "rows_per_step": groups * rows_per, "hidden": hidden,
                   "pg_iters": PG_ITERS, "inner_iters": INNER},
        "harvest_s": harvest_s, "train_s": train_s, "loss_first": float(np.mean(losses[:20])),
        "loss_last": float(np.mean(losses[-20:])), "val_loss_before": val_before[0], "val_loss_after": val_after[0],
        "val_positive_outputs_before": val_before[1], "val_positive_outputs_after": val_after[1],
        "target_norm": target_stats, "results": res,
        "speedup_time_to_eps_vs_fp32": (base["seconds"] / best["seconds"]) if (base and best) else None,
    }), flush=True)
    net.close()


def run_compare(args, w):
    """Sketched and unsketched forms of the method on one dense planted problem
    (the same kernels): outer iterations and CUDA-event time of the steps
    until the relative error (checked after every iteration) reaches eps.
    Gaussian / subsampling sketches with PGD and RCD (Section 3.5), the
    identity sketch with PGD (plain projected gradient ANLS) and with RCD at
    mu = 0 (HALS), bf16 and fp32 where the form allows it."""
    import torch
    import paper_2009_02845_gb300 as pkg
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    m, n, k, d = w["m"], w["n"], w["k"], w["d"]
    M = make_inputs(w, rank)
    G_, S_, I_ = pkg.GAUSSIAN, pkg.SUBSAMPLE, pkg.IDENTITY
    forms = [
        # name, sketch, d, d_v, solver, precision, order, alpha, beta
        ("sanls_gaussian_pgd_bf16", G_, d, d, pkg.PGD, pkg.BF16, 0, 1.0, 1.0),
        ("sanls_gaussian_pgd_bf16_reassociated", G_, d, d, pkg.PGD, pkg.BF16, 1, 1.0, 1.0),
        ("sanls_gaussian_rcd_bf16_reassociated", G_, d, d, pkg.RCD, pkg.BF16, 1, 1.0, 1.0),
        ("sanls_gaussian_pgd16_bf16_reassociated", G_, d, d, pkg.PGD, pkg.BF16, 1, 1.0, 1.0, 16),
        ("sanls_subsample_pgd16_fp32", S_, d, d, pkg.PGD, pkg.FP32, 0, 1.0, 1.0, 16),
        ("sanls_subsample_pgd_fp32", S_, d, d, pkg.PGD, pkg.FP32, 0, 1.0, 1.0),
        ("sanls_subsample_rcd_fp32", S_, d, d, pkg.RCD, pkg.FP32, 0, 1.0, 1.0),
        ("plain_pg_bf16", I_, n, m, pkg.PGD, pkg.BF16, 0, 1.0, 1.0),
        # HALS: mu_t = 1e-6 only guards the division when a column of the fixed factor is zero
        ("hals_bf16", I_, n, m, pkg.RCD, pkg.BF16, 0, 1e-6, 0.0),
        ("hals_fp32", I_, n, m, pkg.RCD, pkg.FP32, 0, 1e-6, 0.0),
    ]
    res = {}
    for name, sk, dd, ddv, solver, prec, order, alpha, beta, *inner in forms:
        h = pkg.DSANLS(m, n, k, dd, sk, seed=0, d_v=ddv, solver=solver, precision=prec, use_graph=1, order=order,
                       alpha=alpha, beta=beta, inner_iters=inner[0] if inner else 1)
        h.set_dense(M)
        total, hit, err = 0.0, None, None
        for it in range(w["t_max"]):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.step(1)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            err = h.rel_error()
            if err <= w["eps"]:
                hit = {"iters": it + 1, "seconds": total / 1000.0, "err": err}
                break
        h.close()
        res[name] = {"to_eps": hit, "iters_run": it + 1, "final_err": err, "ms_per_iter": total / (it + 1)}
        print(json.dumps({"form": name, **res[name]}), file=sys.stderr, flush=True)
    best = min((r["to_eps"]["seconds"] for r in res.values() if r["to_eps"]), default=None)
    print(json.dumps({
        "metric": METRIC, "value": (1.0 / best) if best else 0.0, "unit": "1/time_to_eps (1/s), fastest form",
        "n_gpus": ws, "steps": w["t_max"], "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "m": m, "n": n, "k": k, "d": d, "eps": w["eps"],
                   "t_max": w["t_max"]},
        "results": res,
    }), flush=True)


def parse_batch_tile(spec):
    """--batch-tile: 'chunk,stages,row_tiles[,pipeline]' for both half-steps (side -1),
    or 'U-tile/V-tile' (sides 0 and 1) -> [(side, (chunk, stages, row_tiles[, pipeline]))]."""
    parts = spec.split("/")
    if len(parts) > 2:
        raise ValueError("--batch-tile: at most two tiles (U/V)")
    out = []
    for i, p in enumerate(parts):
        tile = tuple(int(x) for x in p.split(","))
        if len(tile) not in (3, 4):
            raise ValueError("--batch-tile: a tile is chunk,stages,row_tiles[,pipeline]")
        out.append((i if len(parts) == 2 else -1, tile))
    return out


def _batch_inputs(count):
    from synthdata import batch_specs, planted_dense
    specs = batch_specs(count, 0)
    Ms = [planted_dense(s["m"], s["n"], s["k"], s["seed"])[0] for s in specs]
    return specs, Ms


def run_batch(args, w):
    """Batched uneven instances: one step = one outer iteration of every
    instance; value = batch outer iterations/s (x ranks for replicas)."""
    ws, rank, local = _dist()
    specs, Ms = _batch_inputs(w["count"])
    order = w.get("order", 0)
    if order == 1:  # P_i = S_i B_i^T then R_i = X_i P_i, both halves
        flops = sum(2.0 * s["k"] * (s["n"] * s["d"] + s["m"] * s["d_v"]) + 4.0 * s["m"] * s["n"] * s["k"]
                    for s in specs)
    else:
        flops = sum(2.0 * s["m"] * s["n"] * (s["d"] + s["d_v"]) + 2.0 * s["k"] * (s["m"] * s["d"] + s["n"] * s["d_v"])
                    for s in specs)
    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import method
        # bounded sample: one outer iteration of every 64th instance, scaled by problem size
        t0 = time.perf_counter()
        sample = list(range(0, len(specs), 64))
        sf = 0.0
        for i in sample:
            s = specs[i]
            U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
            method.run(Ms[i], U0, V0, s["seed"], 1, method.Options(sketch=0, d=s["d"], d_v=s["d_v"]), log_error=False)
            sf += 2.0 * s["m"] * s["n"] * (s["d"] + s["d_v"])
        dt = (time.perf_counter() - t0) * (flops / sf)
        value = 1.0 / dt
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                          "steps": 1, "warmup": 0, "ms_per_step": 1000 * dt, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": args.workload, "desc": w["desc"], "instances": len(specs)},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                                           "sample": "%d of %d instances, scaled by FLOPs" % (len(sample), len(specs))},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch
    import torch.distributed as dist
    import paper_2009_02845_gb300 as pkg
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = {"fp32": pkg.FP32, "bf16": pkg.BF16}[args.precision]
    b = pkg.Batch(specs, use_graph=1, order=order, precision=prec)
    if args.batch_tile:
        for side, tile in parse_batch_tile(args.batch_tile):
            b.set_tile(*tile, side=side)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    for _ in range(args.warmup):
        b.step(1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = pkg.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws)
    launches = pkg.kernel_launches() - l0
    clk = clocks.stop()
    errs = b.rel_errors()
    prof = b.profile()
    ar_ms = prof["U"]["AR"] + prof["V"]["AR"]
    ar_flops = flops
    achieved = ar_flops / (ar_ms / 1000.0) / 1e12
    tc = prec == pkg.BF16 and order == 0
    if tc:
        # tensor-core product: HBM-bound (about d FLOP per byte of bf16 M, below the ridge):
        # bf16 X_i read once, S_i^T once, R_i written, both halves
        peaks, peak_src = _peaks()
        ar_bytes = sum(2.0 * s["m"] * s["n"] + 2.0 * s["n"] * s["d"] + 4.0 * s["m"] * s["k"] +
                       2.0 * s["n"] * s["m"] + 2.0 * s["m"] * s["d_v"] + 4.0 * s["n"] * s["k"] for s in specs)
        gbs = ar_bytes / (ar_ms / 1000.0) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "kb_ar_tc",
                    "peak_source": "hbm_gbs of %s" % peak_src, "tensor_tflops": achieved,
                    "launch_ms": [prof["U"]["AR"], prof["V"]["AR"]]}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SIMT_PEAK_TFLOPS, "traffic": None, "kernel": "kb_ar",
                    "peak_source": "FP32 CUDA-core peak 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz",
                    "launch_ms": [prof["U"]["AR"], prof["V"]["AR"]]}
    value = job_value(ws, args.steps, ms)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import method
        t0 = time.perf_counter()
        sample = list(range(0, len(specs), 128))
        sf = 0.0
        for i in sample:
            s = specs[i]
            U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
            method.run(Ms[i], U0, V0, s["seed"], 1, method.Options(sketch=0, d=s["d"], d_v=s["d_v"]), log_error=False)
            sf += 2.0 * s["m"] * s["n"] * (s["d"] + s["d_v"])
        dt = (time.perf_counter() - t0) * (flops / sf)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": _cores(), "kind": "oracle",
               "sample": "one outer iteration of %d of %d instances, scaled by FLOPs" % (len(sample), len(specs))}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == pkg.FP32 else "bf16", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "instances": len(specs),
                       "order": ["paper", "reassociated"][order],
                       "graph": True, "persistent_ctas": b.tuned_blocks(), "tc_tile": [b.tuned_tile(0), b.tuned_tile(1)],
                       "l2": "inputs larger than L2 (M_i total %.1f GB)" % (sum(M.nbytes for M in Ms) / 1e9)},
            "instance_iters_per_s": value * len(specs),
            "roofline": roofline,
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clk,
            "phases_ms": prof, "rel_error_median": float(np.median(errs)), "rel_error_max": float(errs.max()),
        }), flush=True)
    b.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
