"""Benchmark: H-matrix build + H-matrix-vector products at N = 2^20 on GB300.

One step = the whole hot path over one synthetic point cloud: hm_build
(Morton codes, radix sort, cluster tree, traversal, batched ACA, near field,
gather lists) followed by 10 products y = H x, then hm_free. Points and x
are resident on the device when the timed region starts (value); the e2e
number repeats the same step through the C-ABI with pinned host buffers
(host->device copies of the points and of every x, device->host copy of
every y inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("H-build s + H-MVP ms at N=2^20 (mixed vs FP64 on GB300, rel err <=1e-5); "
          "% HBM roofline")
WORKLOAD = "mix2d_n1m"
N_MVP = 10
FP32_LANES_PER_SM = 128
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_NOMINAL_TFLOPS = 1.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-multi", action="store_true",
                   help="skip the 16-vector product measured beside the step")
    p.add_argument("--no-otf", action="store_true",
                   help="skip the on-the-fly products measured beside the step")
    p.add_argument("--otf-workloads", default="self,matern3d_n1m",
                   help="comma-separated workloads of the on-the-fly measurement "
                        "(self = the bench workload at its size)")
    p.add_argument("--sweeps", action="store_true",
                   help="instead of the step: the paper's experiments as curves (Sec. 6.4 "
                        "convergence in k, Sec. 6.5 runtime against N), one JSON line")
    p.add_argument("--aca-tune", default="on", choices=["on", "off"],
                   help="time the ACA launch shapes per size class before the timed steps")
    p.add_argument("--batching-study", action="store_true",
                   help="instead of the step: the batching study of Sec. 6.4 (ACA and "
                        "gather time against the batch size), one JSON line")
    p.add_argument("--no-large", action="store_true",
                   help="skip the 2^22-point CG workload and the FP64 on-the-fly 3-D workload")
    p.add_argument("--no-rect", action="store_true",
                   help="skip the context run of A(Y1 x Y2) for two point sets")
    p.add_argument("--no-paper", action="store_true",
                   help="skip the context run in the paper's own setting (N=2^19 Halton, C=2048)")
    p.add_argument("--n", type=int, default=0,
                   help="points of a smaller case of the same workload (profiling only)")
    p.add_argument("--scratch-gb", type=float, default=0.0,
                   help="cap on the ACA scratch of the plain (no rank model) build")
    p.add_argument("--sets", type=int, default=64,
                   help="ragged64 workload: build only the first SETS of the 64 point sets")
    p.add_argument("--batch-mode", default="auto", choices=["auto", "stored", "on-the-fly"],
                   help="ragged64 workload: store the factors and near field, or recompute "
                        "them in every product (hm_build_batch with on_the_fly); auto: "
                        "stored up to 8 sets, on the fly above (all 64 sets stored need "
                        "more than one GPU's memory)")
    p.add_argument("--gather-shape", type=int, default=-1,
                   help="launch shape of the product's gather (hm_set_gather_shape); -1 = tuned")
    p.add_argument("--symmetric", default="near", choices=["near", "on", "off"],
                   help="mixed-precision builds compress only the leaves with tau <= sigma "
                        "and mirror the rest (the kernels are symmetric); near: also store "
                        "each off-diagonal dense leaf once and apply it both ways")
    p.add_argument("--rank-model", default="on", choices=["on", "off"],
                   help="size the ACA factor arena with the learned rank model "
                        "(trained before the timed region on other point sets)")
    return p.parse_args()


# The paper's own GPU numbers for its setting (Sec. 6.7: N = 2^19 Halton
# points in 2-D, exp(-r^2), C_leaf = 2048, eta = 1.5, fixed ACA rank 16,
# FP64, factors stored: "P" mode), on one Tesla P100. Context only.
PAPER_P100 = {"build_s": 1.3, "mvp_s": 1.7, "hardware": "1x Tesla P100 SXM2, CUDA 8.0",
              "precision": "FP64"}
# The same setting without precomputed factors (the paper's NP mode, its
# default): build 0.8 s, product 2.7 s on the P100.
PAPER_P100_NP = {"build_s": 0.8, "mvp_s": 2.7, "hardware": "1x Tesla P100 SXM2, CUDA 8.0",
                 "precision": "FP64"}
PAPER_KERNELS = {0: "exp(-r^2)", 2: "r K_1(r) (Matern, beta - d/2 = 1, phi(0) = 1)"}


def paper_setting(hm, inputs, name="halton2d_n512k_k16", n_mvp=3):
    """Build and multiply in the paper's setting at its size, FP64 and mixed,
    with stored factors (P mode) and recomputed per product (NP mode), CUDA
    events, points and x on the device. Returns a context object."""
    import torch
    w = inputs.WORKLOADS[name]
    pts = torch.from_numpy(inputs.workload_points(name)).cuda()
    x = torch.from_numpy(inputs.normal_vector(w["n"], inputs.X_SEED)).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    out = {"workload": name, "n": w["n"], "d": w["d"], "kernel": PAPER_KERNELS[w["kernel"]],
           "leaf": w["leaf"], "eta": w["eta"], "aca": "fixed rank %d" % w["k_cap"],
           "paper_p100": PAPER_P100, "paper_p100_np": PAPER_P100_NP}

    def run(prec, otf, reps, nm):
        res = []
        for rep in range(reps):         # the first build warms up the tuner
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                           precision=prec, k_cap=w["k_cap"], on_the_fly=otf)
            e[1].record(stream)
            for _ in range(nm):
                H.matvec(x, y)
            e[2].record(stream)
            torch.cuda.synchronize()
            st = H.stats()
            H.free()
            res.append((e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / nm / 1e3, st))
        return res[-1]

    for key, prec in (("fp64", hm.PREC_FP64), ("mixed", hm.PREC_MIXED)):
        b, m, st = run(prec, False, 2, n_mvp)
        out[key] = {"build_s": b, "mvp_s": m,
                    "mvp_hbm_frac": st["mvp_bytes"] / m / 1e9 / peaks()[0],
                    "factor_bytes": st["factor_bytes"], "near_bytes": st["near_bytes"]}
        b, m, st = run(prec, True, 1, 2)
        out[key + "_on_the_fly"] = {"build_s": b, "mvp_s": m,
                                    "aca_passes_per_product": st["aca_passes"]}
    return out


# Algorithmic flops of one kernel evaluation (squared distance in three
# coordinates plus the kernel, as the library counts them for ACA) and the
# multiply-add that takes an evaluated entry into a row sum.
EVAL_FLOPS = {0: 10.0, 1: 13.0, 2: 76.0}


def otf_roofline(so, kernel, peak):
    """ALU rooflines of an on-the-fly product (profiled handle): the ACA
    passes (the library's count of ACA flops for one product) and the dense
    leaves evaluated inside the product (near entries x (evaluation + the
    multiply-add)), each per product against the measured FP32 FMA peak."""
    cnt = max(so["mvp_count"], 1)
    t_aca = so["t_np_aca_ms"] / cnt
    t_low = so["t_np_lowrank_ms"] / cnt
    t_near = so["t_np_near_ms"] / cnt
    near_flops = so["near_entries"] * (EVAL_FLOPS[kernel] + 2.0)
    out = {"bound": "alu", "peak": peak, "unit": "TFLOP/s",
           "peak_source": "measured FP32 FMA peak (hm_alu_peak)",
           "aca": {"ms": t_aca, "flops": so["aca_flops"]},
           "near": {"ms": t_near, "flops": near_flops, "entries": so["near_entries"]},
           "lowrank_ms": t_low}
    for k in ("aca", "near"):
        ms = out[k]["ms"]
        out[k]["achieved"] = out[k]["flops"] / (ms * 1e-3) / 1e12 if ms > 0 else None
        out[k]["frac"] = out[k]["achieved"] / peak if out[k]["achieved"] else None
    return out


def cg_workload(hm, inputs, theta, cg_iters=4, small_logs=(15,)):
    """The 2^22-point solve: 3-D uniform points, Matern-3/2 l = 0.1, CG on
    (A + 1e-2 I) x = b to 1e-6 with the product on the fly (stored, it needs
    more memory than one GPU has), mixed precision, symmetric, the learned
    rank model sizing the ACA passes. At 2^22 the build, one product and a few
    CG iterations are timed (s per iteration); the whole solve is timed at
    smaller N of the same workload, in FP64 (stored) and mixed (on the fly),
    with the true residual of the mixed solution in the FP64 system."""
    import torch
    name = "matern3d_n4m_cg"
    w = inputs.WORKLOADS[name]
    n = w["n"]
    pts = torch.from_numpy(inputs.workload_points(name)).cuda()
    b = inputs.normal_vector(n, inputs.CG_SEED)
    kw = dict(precision=hm.PREC_MIXED, on_the_fly=True, symmetric=True, sigma2=w["sigma2"],
              rank_model_theta=theta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], **kw)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    bd = torch.from_numpy(b).cuda()
    t0 = time.perf_counter()
    H.matvec(bd)
    torch.cuda.synchronize()
    product_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, it, rr = H.cg(b, rtol=w.get("rtol", 1e-6), maxit=cg_iters)
    cg_s = time.perf_counter() - t0
    st = H.stats()
    H.free()
    del pts, bd
    out = {"workload": name, "n": n, "precision": "mixed, on the fly, symmetric, rank model",
           "build_s": build_s, "product_s": product_s, "aca_passes": st["aca_passes"],
           "n_adm": st["n_adm"], "n_dense": st["n_dense"],
           "mispredicted_per_product": st["n_mispredicted"] / (2.0 + it),
           "cg_iterations_timed": it, "cg_relres_after": rr,
           "cg_s_per_iteration": cg_s / (it + 1),   # it iterations + the initial residual
           "solves": []}
    for lg in small_logs:
        ns = 1 << lg
        ps = torch.from_numpy(inputs.workload_points(name, ns)).cuda()
        bs = inputs.normal_vector(ns, inputs.CG_SEED)
        H64 = hm.HMatrix(ps, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                         precision=hm.PREC_FP64, sigma2=w["sigma2"])
        rec = {"n": ns}
        for nm, H in (("fp64_stored", H64),
                      ("mixed_on_the_fly", hm.HMatrix(ps, w["kernel"], w["ell"], w["leaf"], w["eta"],
                                                      w["eps"], **kw))):
            t0 = time.perf_counter()
            x, it, rr = H.cg(bs, rtol=1e-6, maxit=50000)
            dt = time.perf_counter() - t0
            res = bs - H64.matvec(x)
            rec[nm] = {"iterations": it, "relres": rr, "s": dt,
                       "true_relres_fp64_system": float(np.linalg.norm(res) / np.linalg.norm(bs))}
            if H is not H64:
                H.free()
        H64.free()
        out["solves"].append(rec)
    return out


def fp64_on_the_fly(hm, inputs, n_mvp=2):
    """The plain FP64 method on the 3-D Matern-3/2 workload at N = 2^20
    (l = 0.2): its stored form does not fit one GPU (about 525 GB), so every
    product recomputes ACA and the dense leaves; build and n_mvp products."""
    import torch
    name = "matern3d_n1m"
    w = inputs.WORKLOADS[name]
    pts = torch.from_numpy(inputs.workload_points(name)).cuda()
    x = torch.from_numpy(inputs.normal_vector(w["n"], inputs.X_SEED)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                   precision=hm.PREC_FP64, on_the_fly=True, profile=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(n_mvp):
        H.matvec(x)
    torch.cuda.synchronize()
    mvp_s = (time.perf_counter() - t0) / n_mvp
    st = H.stats()
    H.free()
    return {"workload": name, "n": w["n"], "precision": "fp64, on the fly (plain method)",
            "build_s": build_s, "mvp_s": mvp_s, "products_timed": n_mvp,
            "aca_passes": st["aca_passes"], "n_adm": st["n_adm"], "n_dense": st["n_dense"],
            "aca_s_per_product": st["t_np_aca_ms"] / 1e3 / n_mvp,
            "near_s_per_product": st["t_np_near_ms"] / 1e3 / n_mvp,
            "lowrank_s_per_product": st["t_np_lowrank_ms"] / 1e3 / n_mvp}


def rect_context(hm, inputs, w, rows, n_cols=1 << 19, n_mvp=3):
    """A(Y1 x Y2) for two point sets (hm_build_rect): Y1 the step's points,
    Y2 n_cols Halton points in the same unit cube, the step's kernel and
    parameters, mixed precision; build and product time (CUDA events, points
    and x on the device)."""
    import torch
    d = rows.shape[1]
    cols = torch.from_numpy(inputs.halton_points(n_cols, d)).cuda()
    x = torch.from_numpy(inputs.normal_vector(n_cols, inputs.X_SEED)).cuda()
    y = torch.empty(rows.shape[0], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    res = []
    for rep in range(2):                # the first build warms up the tuner
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        H = hm.HMatrix(rows, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], cols=cols,
                       precision=hm.PREC_MIXED)
        e[1].record(stream)
        for _ in range(n_mvp):
            H.matvec(x, y)
        e[2].record(stream)
        torch.cuda.synchronize()
        st = H.stats()
        H.free()
        res.append((e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / n_mvp, st))
    b, m, st = res[-1]
    return {"rows": int(rows.shape[0]), "cols": n_cols, "cols_points": "halton", "d": d,
            "precision": "mixed", "build_s": b, "mvp_ms": m,
            "mvp_hbm_frac": st["mvp_bytes"] / (m / 1e3) / 1e9 / peaks()[0],
            "n_adm": st["n_adm"], "n_dense": st["n_dense"], "max_rank": st["max_rank"]}


def tile_traffic(mvp_tile_bytes):
    """DRAM bytes of one gather launch: the ratio of traffic to algorithmic
    bytes from the committed ncu capture, if the kernel's source is unchanged
    since it was taken (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_tile_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, "paper_1708_09707_gb300", "csrc", "hm_mvp.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if rec.get("source_sha256") != sha:
            return None
        return rec["traffic_per_algorithmic_byte"] * mvp_tile_bytes
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    c = [x.strip() for x in line.split(",")]
                    if len(c) >= 9:
                        rows.append(c)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- oracle leg
def oracle_sample(name: str, budget_s: float = 12.0, seed: int = 0, threads: int = 1):
    """The CPU oracle, as it stands, on a bounded sample of the workload.

    Full-size structure (Morton sort, cluster tree, Alg. 1 traversal) is timed
    as is; ACA is timed on blocks sampled per size class and scaled by the
    class counts; the product is timed on the same workload at N = 2^14 and
    scaled by the number of stored entries. threads > 1 spreads the oracle's
    block loops (ACA, product) over that many host threads (OpenMP). Returns
    seconds per step (build + N_MVP products) and a description of the sample.
    """
    import oracle
    from paper_1708_09707_gb300 import inputs
    oracle.set_threads(threads)
    w = inputs.WORKLOADS[name]
    pts = inputs.workload_points(name)
    t0 = time.perf_counter()
    O = oracle.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                       adm_max=(w["adm"] == "max"), compress=False)
    t_struct = time.perf_counter() - t0
    lo, hi, _, _ = O.tree()
    A = O.adm_leaves()
    m = hi[A[:, 0]] - lo[A[:, 0]]
    n = hi[A[:, 1]] - lo[A[:, 1]]
    size = np.maximum(m, n)
    rng = np.random.default_rng(seed)
    t_aca = 0.0
    spent = 0.0
    nsampled = 0
    classes = np.unique(size)
    per = max(0.5, budget_s / max(len(classes), 1))
    for c in classes:
        idx = np.nonzero(size == c)[0]
        rng.shuffle(idx)
        # grow the sample fourfold until it takes a quarter of the class's time
        k = min(len(idx), max(2 * threads, 4))
        while True:
            ts = time.perf_counter()
            O.compress_ids(idx[:k])
            dt = time.perf_counter() - ts
            spent += dt
            if dt > per / 4 or k >= len(idx):
                break
            k = min(len(idx), 4 * k)
        nsampled += k
        t_aca += dt / k * len(idx)
    # product: full oracle H-matrix at N = 2^14, scaled by stored entries
    ns = 1 << 14
    ps = inputs.workload_points(name, ns)
    Os = oracle.HMatrix(ps, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                        adm_max=(w["adm"] == "max"))
    xs = inputs.normal_vector(ns, 1)
    Os.matvec(xs)
    ts = time.perf_counter()
    reps = 3
    for _ in range(reps):
        Os.matvec(xs)
    t_mv_small = (time.perf_counter() - ts) / reps
    oracle.set_threads(1)

    def entries(H):
        l, h, _, _ = H.tree()
        a, d = H.adm_leaves(), H.dense_leaves()
        return (int((h[d[:, 0]] - l[d[:, 0]]).astype(np.int64) @ (h[d[:, 1]] - l[d[:, 1]]))
                + int((h[a[:, 0]] - l[a[:, 0]] + h[a[:, 1]] - l[a[:, 1]]).sum() * 8))

    t_mv = t_mv_small * entries(O) / max(entries(Os), 1)
    step = t_struct + t_aca + N_MVP * t_mv
    sample = ("full-size structure (%.1f s, one thread); ACA on %d of %d admissible blocks "
              "sampled per size class (%.1f s), scaled by class counts; product timed at "
              "N=2^14 (%.3f s) scaled by stored entries; %d thread%s for ACA and the product" %
              (t_struct, nsampled, len(A), spent, t_mv_small, threads,
               "" if threads == 1 else "s (OpenMP over blocks)"))
    return step, t_struct + t_aca, t_mv, sample


def host_threads() -> int:
    """Host cores this process may use."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1708_09707_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if "n" not in w:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the CPU oracle estimate covers single point-set workloads only"}))
        return
    vals = []
    sample = ""
    cores = host_threads()
    for it in range(args.warmup + args.steps):
        step, tb, tm, sample = oracle_sample(args.workload, budget_s=6.0, seed=it, threads=cores)
        if it >= args.warmup:
            vals.append(step)
    v = float(np.mean(vals))
    unit = "s/step (build + %d H-MVP)" % N_MVP
    line = {"metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "n": w["n"], "d": w["d"],
                       "kernel": "gaussian" if w["kernel"] == 0 else "matern32",
                       "ell": w["ell"], "leaf": w["leaf"], "eta": w["eta"],
                       "aca_eps": w["eps"], "mvp_per_step": N_MVP},
            "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- batch leg
def run_batch(args):
    """The ragged batch of 64 independent point sets (sizes log-uniform in
    [1e4, 2^18], d in {2, 3}): one step builds this rank's sets together
    (hm_build_batch) and multiplies them N_MVP times, with stored factors and
    near field or on the fly (all 64 sets stored need more memory than one
    GPU has; the on-the-fly roofline is the ACA passes' arithmetic). With several ranks the
    sets are sharded (longest first to the least-loaded rank) and no data
    crosses ranks, so the total work is fixed: strong scaling."""
    import torch
    from paper_1708_09707_gb300 import dist as hdist
    from paper_1708_09707_gb300 import build as hbuild
    world, rank, local = hdist.world()
    torch.cuda.set_device(local)
    hdist.init("nccl", torch.device("cuda", local))
    if not os.path.exists(hbuild.LIB):
        hbuild.build()
    from paper_1708_09707_gb300 import hm, inputs
    hm.set_gather_shape(args.gather_shape)
    w = inputs.WORKLOADS["ragged64"]
    sizes, dims = inputs.ragged_batch_sizes(w["count"], w["seed"])
    sizes, dims = sizes[:args.sets], dims[:args.sets]
    mine = hdist.shard_sets(sizes, world, rank)
    sets = [inputs.uniform_points(int(sizes[q]), int(dims[q]), w["seed"] * 10 + q) for q in mine]
    msz, mdim = sizes[mine], dims[mine]
    flat_h = np.concatenate([p.ravel() for p in sets])
    flat = torch.from_numpy(flat_h).cuda()
    n = int(msz.sum())
    x_h = inputs.normal_vector(n, inputs.X_SEED)
    x = torch.from_numpy(x_h).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    otf = args.batch_mode == "on-the-fly" or (args.batch_mode == "auto" and len(sizes) > 8)
    opts = dict(precision=hm.PREC_MIXED, on_the_fly=otf,
                symmetric={"near": 2, "on": 1, "off": 0}[args.symmetric])

    def step(ev=None, profile=False, host=False):
        if ev:
            ev[0].record(stream)
        B = hm.HBatch(None, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                      flat=flat_hp if host else flat, sizes=msz, dims=mdim, profile=profile, **opts)
        if ev:
            ev[1].record(stream)
        for _ in range(N_MVP):
            if host:
                B.matvec(x_hp, y_hp)
            else:
                B.matvec(x, y)
        if ev:
            ev[2].record(stream)
        st = B.stats()
        B.free()
        return st

    flat_hp = torch.from_numpy(flat_h).pin_memory()
    x_hp = torch.from_numpy(x_h).pin_memory()
    y_hp = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    hdist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    l0 = hm.kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_step")
        t0.record(stream)
        stats = [step(evs[k], profile=True) for k in range(args.steps)]
        t1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    clocks = clk.summary()
    launches = (hm.kernel_launches() - l0) / args.steps
    total = t0.elapsed_time(t1) / args.steps
    build_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    mvp_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs])) / N_MVP
    hdist.barrier()
    total, build_ms, mvp_ms = hdist.max_over_ranks([total, build_ms, mvp_ms], "cuda")
    # e2e: host points, x and y through the C-ABI
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(1, min(args.steps, 3))):
        step(host=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / max(1, min(args.steps, 3))
    e2e_ms = hdist.max_over_ranks([e2e_ms], "cuda")[0]
    if rank != 0:
        hdist.finalize()
        return
    st = stats[-1]
    if otf:
        # nothing stored: the products are bound by the ACA passes' arithmetic
        fp32_peak = hm.alu_peak(hm.PREC_MIXED) / 1e12
        o = otf_roofline(st, w["kernel"], fp32_peak)
        roof = {"bound": "alu", "kernel": "batched ACA passes (on the fly)",
                "achieved": o["aca"]["achieved"], "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": o["aca"]["frac"], "traffic": None, "peak_source": o["peak_source"],
                "phases_per_product": o}
    else:
        hbm, peak_src = peaks()
        t_tile = st["t_mvp_tile_ms"] / max(st["mvp_count"], 1)
        roof = {"bound": "hbm", "kernel": "k_tile (gather: U slices + near field)",
                "achieved": st["mvp_tile_bytes"] / (t_tile * 1e-3) / 1e9, "peak": hbm,
                "unit": "GB/s", "traffic": tile_traffic(st["mvp_tile_bytes"]),
                "algorithmic_bytes": st["mvp_tile_bytes"],
                "peak_source": peak_src + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        roof["frac"] = roof["achieved"] / hbm
    unit = "s/step (batched build of %d sets + %d batched H-MVP)" % (len(sizes), N_MVP)
    line = {"metric": METRIC, "value": total / 1e3, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "ragged64", "sets": int(len(sizes)), "of_sets": int(w["count"]),
                       "points": int(sizes.sum()),
                       "sizes": "log-uniform in [1e4, 2^18]", "d": "2 or 3", "kernel": "gaussian",
                       "ell": w["ell"], "leaf": w["leaf"], "eta": w["eta"], "aca_eps": w["eps"],
                       "precision": "mixed", "symmetric": args.symmetric,
                       "mode": "on the fly" if otf else "stored",
                       "mvp_per_step": N_MVP, "parallelism": "sets sharded" if world > 1 else "single"},
            "build_s": build_ms / 1e3, "mvp_ms": mvp_ms,
            "e2e": {"value": e2e_ms / 1e3, "unit": unit,
                    "h2d_bytes_per_step": int(flat_h.nbytes + N_MVP * n * 8),
                    "d2h_bytes_per_step": int(N_MVP * n * 8)},
            "roofline": roof, "gpu_launches": int(round(launches)), "clocks": clocks,
            "cpu_baseline": None,
            "stats": {k: st[k] for k in ("n_adm", "n_dense", "sum_rank", "factor_bytes",
                                         "near_bytes", "mvp_bytes", "t_aca_ms", "t_dense_ms",
                                         "aca_passes", "near_entries")}}
    print(json.dumps(line))
    hdist.finalize()


# ------------------------------------------------------------- sweeps
def _elapsed(fn, stream):
    """CUDA-event time (ms) of fn() on the stream, with a synchronize on both sides."""
    import torch
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    out = fn()
    e[1].record(stream)
    torch.cuda.synchronize()
    return e[0].elapsed_time(e[1]), out


def run_sweeps(args):
    """The paper's experiments on this GPU, FP64 as in the paper, Halton
    points in [0,1]^d, the unscaled kernels, C_leaf, eta and the fixed rank
    of Sec. 6.4 to 6.5; points and x on the device, CUDA events.
      convergence  Sec. 6.4: N = 32768, C_leaf 256, eta 1.5, e_rel of the
                   fixed-rank-k product against the exact product (an eta = 0
                   build: every leaf dense), mean over three x
      structure    Sec. 6.5, first figure: Morton codes + sort (the spatial
                   data structure) and the whole structure (codes, sort, tree,
                   boxes, Alg. 1 traversal) for N up to 2^26, C_leaf 2048;
                   uniform points here (the host makes 2^26 Halton points ten
                   times slower)
      mvp          Sec. 6.5, second figure: product time with stored factors
                   (P) and with factors recomputed per product (NP), C_leaf
                   2048, eta 1.5, k = 16"""
    import torch
    from paper_1708_09707_gb300 import build, hm, inputs
    build.build()
    hm.lib()
    stream = torch.cuda.current_stream()
    out = {"precision": "fp64", "points": "halton", "kernels": {"gaussian": "exp(-r^2)",
           "matern_k1": "r K_1(r), phi(0) = 1"}}
    kernels = (("gaussian", hm.GAUSSIAN), ("matern_k1", hm.MATERN_K1))

    conv = []
    n = 32768
    for d in (2, 3):
        pts = torch.from_numpy(inputs.halton_points(n, d)).cuda()
        xs = [torch.from_numpy(inputs.normal_vector(n, inputs.X_SEED + t)).cuda() for t in range(3)]
        for kname, kern in kernels:
            E = hm.HMatrix(pts, kern, 1.0, 256, 0.0, 1e-6)
            ys = [E.matvec(x) for x in xs]
            E.free()
            errs = []
            for k in (1, 2, 3, 4, 6, 8, 10, 12, 14, 16):
                H = hm.HMatrix(pts, kern, 1.0, 256, 1.5, 0.0, k_cap=k)
                e = [float(torch.linalg.norm(H.matvec(x) - y) / torch.linalg.norm(y))
                     for x, y in zip(xs, ys)]
                H.free()
                errs.append([k, sum(e) / len(e)])
            conv.append({"d": d, "kernel": kname, "n": n, "leaf": 256, "eta": 1.5,
                         "e_rel_by_k": errs})
        del pts, xs
    out["convergence"] = conv

    struct = []
    for d in (2, 3):
        for lg in range(16, 27, 2):
            n = 1 << lg
            pts = torch.from_numpy(inputs.uniform_points(n, d, inputs.POINT_SEED + 20 + d)).cuda()
            codes = torch.empty(n, dtype=torch.int64, device="cuda")
            vals = torch.arange(n, dtype=torch.int32, device="cuda")
            bits = d * min(32, 64 // d)

            def spatial():
                hm.morton_codes(pts, codes)
                hm.radix_sort_pairs(codes, vals, bits)
            spatial()
            t_sp, _ = _elapsed(spatial, stream)
            hm.HMatrix(pts, hm.GAUSSIAN, 1.0, 2048, 1.5, 0.0, k_cap=16, structure_only=True).free()
            t_all, H = _elapsed(lambda: hm.HMatrix(pts, hm.GAUSSIAN, 1.0, 2048, 1.5, 0.0,
                                                   k_cap=16, structure_only=True), stream)
            st = H.stats()
            H.free()
            struct.append({"d": d, "n": n, "morton_sort_ms": t_sp, "structure_ms": t_all,
                           "n_adm": st["n_adm"], "n_dense": st["n_dense"]})
            del pts, codes, vals
    out["structure"] = struct
    out["structure_points"] = "uniform"
    out["structure_paper_p100"] = {"morton_sort_s_at_2^26": "below 0.5",
                                   "tree_and_traversal_s_at_2^26": "below 3"}

    mvp = []
    for d in (2, 3):
        for lg in range(15, 23):
            n = 1 << lg
            pts = torch.from_numpy(inputs.halton_points(n, d)).cuda()
            x = torch.from_numpy(inputs.normal_vector(n, inputs.X_SEED)).cuda()
            y = torch.empty_like(x)
            row = {"d": d, "n": n}
            # stored: the FP64 near field of C_leaf 2048 is 116 GB at 2^19 in 2-D
            stored_max = 19 if d == 2 else 17
            for mode, otf, top in (("P", False, stored_max), ("NP", True, 21 if d == 2 else 20)):
                if lg > top:
                    continue
                try:
                    tb, H = _elapsed(lambda: hm.HMatrix(pts, hm.GAUSSIAN, 1.0, 2048, 1.5, 0.0,
                                                        k_cap=16, on_the_fly=otf), stream)
                    if not otf:
                        H.matvec(x, y)           # the first product tunes the gather
                    reps = 3 if n <= (1 << 18) else 1
                    tm, _ = _elapsed(lambda: [H.matvec(x, y) for _ in range(reps)], stream)
                    H.free()
                    row[mode] = {"build_ms": tb, "mvp_ms": tm / reps}
                except hm.HMError as e:
                    row[mode] = {"error": str(e)}
            mvp.append(row)
            del pts, x, y
    out["mvp"] = mvp
    out["mvp_paper_p100"] = {"np_mvp_at_2^25_d2": "about 6 minutes"}
    print(json.dumps({"sweeps": out}))


def run_batching(args):
    """The batching study of Sec. 6.4 on this GPU: the paper's setting
    (Halton points in [0,1]^2, exp(-r^2), eta 1.5, fixed rank 16, FP64) with
    C_leaf 1024 and 2048, at N = 2^19 (the stored FP64 near field of
    C_leaf 2048 at 2^20 is 232 GB, more than one GPU holds). Batch sizes:
      ACA     reserved factor entries per launch (bs_ACA; 1 = one launch per
              block, 0 = one launch per size class); the build's ACA time
      gather  work items per launch of the product's gather (an item is a
              row tile's near-field blocks and U slices; 1 = one launch per
              item, 0 = one launch); the product's time, mean of 3
    Every batch size gives the same ranks and bit-identical products (checked
    here)."""
    import torch
    from paper_1708_09707_gb300 import build, hm, inputs
    build.build()
    hm.lib()
    stream = torch.cuda.current_stream()
    n = 1 << 19
    pts = torch.from_numpy(inputs.halton_points(n, 2)).cuda()
    x = torch.from_numpy(inputs.normal_vector(n, inputs.X_SEED)).cuda()
    y = torch.empty_like(x)
    out = {"n": n, "d": 2, "kernel": "exp(-r^2)", "eta": 1.5, "aca": "fixed rank 16",
           "precision": "fp64", "points": "halton", "leaves": []}
    hm.set_gather_shape(0)     # one launch shape for every batch size
    try:
        for leaf in (1024, 2048):
            row = {"leaf": leaf, "aca": [], "gather": []}
            ref_y = ref_rank = None
            # one untimed build first: module loading and launch attributes
            hm.HMatrix(pts, hm.GAUSSIAN, 1.0, leaf, 1.5, 0.0, k_cap=16).free()
            for bs in (0, 1 << 27, 1 << 25, 1 << 23, 1 << 21, 1 << 19, 1):
                hm.set_batch_limits(bs, 0)
                H = hm.HMatrix(pts, hm.GAUSSIAN, 1.0, leaf, 1.5, 0.0, k_cap=16)
                st = H.stats()
                yv = H.matvec(x)
                rk = H.structure()["ranks"]
                H.free()
                if ref_y is None:
                    ref_y, ref_rank = yv, rk
                    row["n_adm"], row["n_dense"] = st["n_adm"], st["n_dense"]
                row["aca"].append({"bs_aca": bs, "aca_ms": st["t_aca_ms"],
                                   "same": bool(torch.equal(yv, ref_y)
                                                and (rk == ref_rank).all())})
            hm.set_batch_limits(0, 0)
            H = hm.HMatrix(pts, hm.GAUSSIAN, 1.0, leaf, 1.5, 0.0, k_cap=16)
            H.matvec(x, y)
            ref = y.clone()
            for items in (0, 128, 32, 8, 2, 1):
                hm.set_batch_limits(0, items)
                H.matvec(x, y)
                same = bool(torch.equal(y, ref))
                reps = 5 if items == 0 or items >= 8 else 2
                t, _ = _elapsed(lambda: [H.matvec(x, y) for _ in range(reps)], stream)
                row["gather"].append({"items_per_launch": items, "mvp_ms": t / reps, "same": same})
            row["n_items"] = H.stats()["n_tiles"]
            H.free()
            out["leaves"].append(row)
    finally:
        hm.set_batch_limits(0, 0)
        hm.set_gather_shape(-1)
    print(json.dumps({"batching": out}))


# ---------------------------------------------------------------- GPU leg
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "ragged64":
        run_batch(args)
        return
    if args.sweeps:
        run_sweeps(args)
        return
    if args.batching_study:
        run_batching(args)
        return
    import torch

    from paper_1708_09707_gb300 import dist as hdist
    world, rank, local = hdist.world()
    torch.cuda.set_device(local)
    hdist.init("nccl", torch.device("cuda", local))
    barrier = hdist.barrier

    from paper_1708_09707_gb300 import build as hbuild
    if not os.path.exists(hbuild.LIB):
        hbuild.build()
    from paper_1708_09707_gb300 import hm, inputs
    hm.set_gather_shape(args.gather_shape)
    w = dict(inputs.WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    N, d = w["n"], w["d"]
    pts_np = inputs.workload_points(args.workload, N)
    x_np = inputs.normal_vector(N, inputs.X_SEED)
    pts = torch.from_numpy(pts_np).cuda()
    x = torch.from_numpy(x_np).cuda()
    y = torch.empty_like(x)
    kw = dict(adm_max=(w["adm"] == "max"), scratch_gb=args.scratch_gb)
    stream = torch.cuda.current_stream()

    # learned rank model: trained untimed, on point sets other than the
    # benchmark's (other seeds and sizes), with the library's MLP kernels
    theta = None
    model_info = None
    if args.rank_model == "on":
        from paper_1708_09707_gb300 import rank_model
        t_m = time.time()
        F, T = rank_model.training_data()
        theta, hist = rank_model.train(F, T)
        model_info = {"train_s": time.time() - t_m, "samples": int(F.shape[0]),
                      "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                      "train_sets": [dict(s) for s in rank_model.TRAIN_SETS]}

    # mixed-precision builds use the kernels' symmetry (compress the leaves
    # with tau.lo <= sigma.lo, mirror the rest); the FP64 path stays the
    # paper's plain method
    use_sym = {"near": 2, "on": 1, "off": 0}[args.symmetric]

    def step(prec, ev=None, profile=False, model=True, sym=None):
        if ev:
            ev[0].record(stream)
        mk = dict(kw)
        mk["symmetric"] = (use_sym if sym is None else int(sym)) if prec == hm.PREC_MIXED else 0
        if model and theta is not None:
            mk["rank_model_theta"] = theta
        H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                       precision=prec, profile=profile, **mk)
        if ev:
            ev[1].record(stream)
        for _ in range(N_MVP):
            H.matvec(x, y)
        if ev:
            ev[2].record(stream)
        st = H.stats()
        H.free()
        return st

    def timed(prec, steps, warmup, profile, model=True, sym=None, name="compare"):
        for _ in range(warmup):
            step(prec, model=model, sym=sym)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        l0 = hm.kernel_launches()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        stats = []
        # an NVTX range names the timed launches for a profiler's launch list
        torch.cuda.nvtx.range_push(name)
        t0.record(stream)
        for k in range(steps):
            stats.append(step(prec, evs[k], profile, model, sym))
        t1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches = (hm.kernel_launches() - l0) / steps
        total = t0.elapsed_time(t1) / steps
        build = np.mean([e[0].elapsed_time(e[1]) for e in evs])
        mvp = np.mean([e[1].elapsed_time(e[2]) for e in evs]) / N_MVP
        return total, build, mvp, stats, launches

    # ACA launch shapes tuned on this problem before anything is timed (the
    # gather's shape is tuned by its first product the same way)
    aca_shapes = None
    if args.aca_tune == "on":
        tk = dict(kw)
        tk["symmetric"] = use_sym
        if theta is not None:
            tk["rank_model_theta"] = theta
        t_t = time.time()
        aca_shapes = {"shapes_by_class": hm.tune_aca_shapes(
            pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], reps=2,
            precision=hm.PREC_MIXED, **tk)}
        aca_shapes["tune_s"] = time.time() - t_t

    hbm, peak_src = peaks()
    with ClockSampler(local) as clk:
        total, build_ms, mvp_ms, stats, launches = timed(hm.PREC_MIXED, args.steps,
                                                         args.warmup, True, name="timed_step")
    clocks = clk.summary()
    # max over ranks
    total, build_ms, mvp_ms = hdist.max_over_ranks([total, build_ms, mvp_ms], "cuda")
    st = stats[-1]

    # FP64 reference path on the same GPU (same step, fewer repetitions)
    fp64 = None
    err = None
    if not args.no_fp64:
        t64, b64, m64, s64, _ = timed(hm.PREC_FP64, 1, 1, False, model=False, name="compare_fp64")
        fp64 = {"build_s": b64 / 1e3, "mvp_ms": m64, "ms_per_step": t64,
                "mvp_roofline_frac": s64[-1]["mvp_bytes"] / (m64 * 1e-3) / (hbm * 1e9)}
        # the FP64 product is bound by the FP64 pipe before HBM: one
        # multiply-add (2 flops) per 8-byte entry streamed, so at most
        # 4 B per flop x the measured FP64 FMA throughput
        p64 = hm.alu_peak(hm.PREC_FP64)
        fp64["fp64_pipe_bound"] = {
            "peak_tflops": p64 / 1e12, "bound_gbs": 4.0 * p64 / 1e9,
            "achieved_gbs": s64[-1]["mvp_bytes"] / (m64 * 1e-3) / 1e9,
            "frac": s64[-1]["mvp_bytes"] / (m64 * 1e-3) / (4.0 * p64),
            "peak_source": "measured: FP64 FMA chains on every SM (hm_alu_peak)"}
        H64 = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                         precision=hm.PREC_FP64, **kw)
        y64 = H64.matvec(x).cpu().numpy()
        H64.free()
        mk = dict(kw)
        if theta is not None:
            mk["rank_model_theta"] = theta
        H32 = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                         precision=hm.PREC_MIXED, symmetric=use_sym, **mk)
        y32 = H32.matvec(x).cpu().numpy()
        H32.free()
        err = float(np.linalg.norm(y32 - y64) / np.linalg.norm(y64))

    # per-kernel ACA durations: one more (untimed) build with the size classes
    # run one after another, so each class's time is its own kernels'
    aca_serial = None
    if world == 1:
        mk = dict(kw)
        if theta is not None:
            mk["rank_model_theta"] = theta
        Hs = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                        precision=hm.PREC_MIXED, profile=2, symmetric=use_sym, **mk)
        aca_serial = Hs.stats()["t_aca_class_ms"]
        Hs.free()

    # the same mixed step without the rank model (chunked ACA passes)
    plain = None
    if theta is not None:
        tp, bp, mp, sp, _ = timed(hm.PREC_MIXED, 1, 1, False, model=False,
                                  name="compare_no_rank_model")
        plain = {"build_s": bp / 1e3, "mvp_ms": mp, "ms_per_step": tp,
                 "aca_ms": sp[-1]["t_aca_ms"], "aca_passes": sp[-1]["aca_passes"],
                 "reserved_factor_entries": sp[-1]["reserved_factor_entries"]}

    # the same mixed step without the symmetry (every admissible leaf compressed)
    nonsym = None
    if use_sym:
        tn, bn, mn, sn, _ = timed(hm.PREC_MIXED, 1, 1, False, sym=False,
                                  name="compare_nonsymmetric")
        nonsym = {"build_s": bn / 1e3, "mvp_ms": mn, "ms_per_step": tn,
                  "aca_ms": sn[-1]["t_aca_ms"]}

    # several right-hand sides per call (reported beside the step, not in it):
    # a group of 16 vectors shares one pass over the stored factors and near
    # field, against 16 one-vector products on the same handle
    multi = None
    if world == 1 and not args.no_multi:
        mk = dict(kw)
        if theta is not None:
            mk["rank_model_theta"] = theta
        # (the symmetric near field runs several vectors one at a time, so
        # this leg keeps the mirrored factors only)
        Hm = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                        precision=hm.PREC_MIXED, symmetric=min(use_sym, 1), **mk)
        nr = 16
        Xr = torch.from_numpy(inputs.normal_vector(N, inputs.X_SEED + 1, nrhs=nr)).cuda()
        Yr = torch.empty_like(Xr)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        reps = 3
        for _ in range(2):
            Hm.matvec(Xr, Yr)
        torch.cuda.synchronize()
        ev[0].record(stream)
        torch.cuda.nvtx.range_push("multi_rhs")
        for _ in range(reps):
            Hm.matvec(Xr, Yr)
        torch.cuda.nvtx.range_pop()
        ev[1].record(stream)
        for _ in range(reps):
            for r in range(nr):
                Hm.matvec(Xr[r], Yr[r])
        ev[2].record(stream)
        torch.cuda.synchronize()
        grp_ms = ev[0].elapsed_time(ev[1]) / reps
        one_ms = ev[1].elapsed_time(ev[2]) / reps / nr
        sm = Hm.stats()
        per_vec = N * 24
        grp_bytes = sm["mvp_bytes"] - per_vec + nr * per_vec
        multi = {"nrhs": nr, "ms_per_call": grp_ms, "ms_per_vector": grp_ms / nr,
                 "one_vector_product_ms": one_ms, "speedup_per_vector": one_ms * nr / grp_ms,
                 "algorithmic_bytes": grp_bytes,
                 "achieved_gbs": grp_bytes / (grp_ms * 1e-3) / 1e9,
                 "note": "bytes: stored factors, near field and column indices once, "
                         "x, perm and y per vector"}
        Hm.free()

    # the on-the-fly product (nothing stored: ACA and the dense leaves are
    # recomputed inside every product), reported beside the step: on this
    # workload, and on the 3-D Matern workload at N = 2^20, whose stored
    # H-matrix does not fit one GPU
    otf = None
    fp32_peak = hm.alu_peak(hm.PREC_MIXED) / 1e12
    if world == 1 and not args.no_otf:
        otf = []
        names = [args.workload if q == "self" else q for q in args.otf_workloads.split(",")]
        for wname in names:
            wo = dict(inputs.WORKLOADS[wname])
            if wname == args.workload and args.n:
                wo["n"] = args.n
            po = pts if wname == args.workload else torch.from_numpy(
                inputs.workload_points(wname, wo["n"])).cuda()
            xo = x if wname == args.workload else torch.from_numpy(
                inputs.normal_vector(wo["n"], inputs.X_SEED)).cuda()
            yo = torch.empty_like(xo)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            reps = 2
            torch.cuda.synchronize()
            ev[0].record(stream)
            Ho = hm.HMatrix(po, wo["kernel"], wo["ell"], wo["leaf"], wo["eta"], wo["eps"],
                            precision=hm.PREC_MIXED, on_the_fly=True, profile=True,
                            symmetric=min(use_sym, 1), adm_max=(wo["adm"] == "max"))
            ev[1].record(stream)
            torch.cuda.nvtx.range_push("on_the_fly_" + wname)
            for _ in range(reps):
                Ho.matvec(xo, yo)
            torch.cuda.nvtx.range_pop()
            ev[2].record(stream)
            torch.cuda.synchronize()
            so = Ho.stats()
            otf.append({"workload": wname, "n": wo["n"], "precision": "mixed",
                        "symmetric": use_sym > 0,
                        "build_s": ev[0].elapsed_time(ev[1]) / 1e3,
                        "mvp_ms": ev[1].elapsed_time(ev[2]) / reps,
                        "aca_passes_per_product": so["aca_passes"], "n_adm": so["n_adm"],
                        "n_dense": so["n_dense"],
                        "roofline": otf_roofline(so, wo["kernel"], fp32_peak)})
            Ho.free()
            del po, xo, yo

    # the 2^22-point CG workload and the FP64 3-D Matern workload at 2^20,
    # both on the fly (their stored forms do not fit one GPU)
    cg5 = fp64_otf = None
    if world == 1 and not args.no_large and theta is not None:
        cg5 = cg_workload(hm, inputs, theta)
    if world == 1 and not args.no_large:
        fp64_otf = fp64_on_the_fly(hm, inputs)

    # A(Y1 x Y2): the step's points against 2^19 Halton points
    rect = None
    if world == 1 and not args.no_rect:
        rect = rect_context(hm, inputs, w, pts)

    # e2e: the same step through the C-ABI with pinned host buffers
    pts_h = torch.from_numpy(pts_np).pin_memory()
    xs_h = torch.from_numpy(x_np).pin_memory()
    ys_h = torch.empty(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    mk = dict(kw)
    if theta is not None:
        mk["rank_model_theta"] = theta
    for _ in range(e2e_steps):
        H = hm.HMatrix(pts_h, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                       precision=hm.PREC_MIXED, symmetric=use_sym, **mk)
        for _ in range(N_MVP):
            H.matvec(xs_h, ys_h)
        H.free()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    ysum = float(ys_h.sum())
    assert math.isfinite(ysum)

    if rank != 0:
        hdist.finalize()
        return

    # rooflines from the library's own CUDA events on the launching stream
    mvp_t_tile = st["t_mvp_tile_ms"] / max(st["mvp_count"], 1)
    mvp_t_vtx = st["t_mvp_vtx_ms"] / max(st["mvp_count"], 1)
    mvp_t = st["t_mvp_ms"] / max(st["mvp_count"], 1)
    mvp_t_tail = st["t_mvp_tail_ms"] / max(st["mvp_count"], 1)
    gname = ("k_tile_tma pass A (canonical U slices + symmetric near field, transposed "
             "products)" if use_sym == 2 else "k_tile (gather: U slices + near field)")
    mvp_roof = {"bound": "hbm", "kernel": gname,
                "achieved": st["mvp_tile_bytes"] / (mvp_t_tile * 1e-3) / 1e9, "peak": hbm,
                "unit": "GB/s", "traffic": tile_traffic(st["mvp_tile_bytes"]),
                "algorithmic_bytes": st["mvp_tile_bytes"], "ms": mvp_t_tile,
                "whole_product": {"achieved": st["mvp_bytes"] / (mvp_t * 1e-3) / 1e9,
                                  "ms": mvp_t, "bytes": st["mvp_bytes"]},
                "vtx": {"achieved": st["mvp_vtx_bytes"] / (mvp_t_vtx * 1e-3) / 1e9,
                        "ms": mvp_t_vtx, "bytes": st["mvp_vtx_bytes"]},
                "tail": {"what": ("mirror t (k_tmirror), pass B (mirror slices), finish"
                                  if use_sym == 2 else "finish"),
                         "achieved": st["mvp_tail_bytes"] / (mvp_t_tail * 1e-3) / 1e9
                         if mvp_t_tail > 0 else None,
                         "ms": mvp_t_tail, "bytes": st["mvp_tail_bytes"]}}
    mvp_roof["frac"] = mvp_roof["achieved"] / hbm
    mvp_roof["peak_source"] = peak_src + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    aca_roof = {"bound": "alu", "kernel": "batched ACA (all size classes, concurrent)",
                "achieved": st["aca_flops"] / (st["t_aca_ms"] * 1e-3) / 1e12,
                "peak": fp32_peak, "unit": "TFLOP/s", "traffic": None,
                "peak_source": "measured: FP32 FMA chains on every SM (hm_alu_peak); "
                               "nominal 152 SMs x 128 lanes x 2 x 2070 MHz = %.1f"
                               % (SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12)}
    aca_roof["frac"] = aca_roof["achieved"] / fp32_peak
    # dominant kernel of the step: the gather (N_MVP launches) against the
    # longest ACA size-class kernel, timed alone in the serial-classes build
    aca_roof["class_ms_concurrent"] = list(st["t_aca_class_ms"])
    if aca_serial is not None:
        aca_roof["class_ms_serial"] = list(aca_serial)
    longest_aca = max(aca_serial) if aca_serial is not None else st["t_aca_ms"]
    dominant = aca_roof if longest_aca > N_MVP * mvp_t_tile else mvp_roof

    paper = paper_matern = None
    if not args.no_paper and world == 1:
        paper = paper_setting(hm, inputs)
        paper_matern = paper_setting(hm, inputs, "halton2d_n512k_k16_matern")

    cpu = None
    if not args.no_cpu and world == 1:
        # the oracle on all host cores (OpenMP over blocks), and on one core
        cores = host_threads()
        cstep, cbuild, cmv, sample = oracle_sample(args.workload, budget_s=8.0, threads=cores)
        sstep, sbuild, smv, ssample = oracle_sample(args.workload, budget_s=8.0, threads=1)
        cpu = {"value": cstep, "unit": "s/step (build + %d H-MVP)" % N_MVP, "cores": cores,
               "kind": "oracle", "sample": sample, "build_s": cbuild, "mvp_ms": cmv * 1e3,
               "single_core": {"value": sstep, "build_s": sbuild, "mvp_ms": smv * 1e3,
                               "sample": ssample}}

    value = total / 1e3
    line = {
        "metric": METRIC, "value": value, "unit": "s/step (build + %d H-MVP)" % N_MVP,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": N, "d": d,
                   "points": w["points"], "kernel": "gaussian" if w["kernel"] == 0 else "matern32",
                   "ell": w["ell"], "leaf": w["leaf"], "eta": w["eta"], "aca_eps": w["eps"],
                   "precision": "mixed (FP32 ACA + FP64 stopping test, BF16 hi/lo near field)",
                   "rank_model": args.rank_model, "symmetric": use_sym,
                   "mvp_per_step": N_MVP, "l2": "inputs larger than L2 (product streams "
                   "%.1f GB per call)" % (st["mvp_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "build_s": build_ms / 1e3, "mvp_ms": mvp_ms,
        "fp64": fp64, "mixed_vs_fp64_rel_err": err,
        "mixed_without_rank_model": plain, "mixed_nonsymmetric": nonsym,
        "multi_rhs": multi, "on_the_fly": otf, "rectangular": rect,
        "cg_matern3d_n4m": cg5, "fp64_on_the_fly_matern3d_n1m": fp64_otf,
        "rank_model": model_info,
        "speedup_vs_fp64": (fp64["ms_per_step"] / total) if fp64 else None,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s/step (build + %d H-MVP)" % N_MVP,
                "h2d_bytes_per_step": N * d * 8 + N_MVP * N * 8,
                "d2h_bytes_per_step": N_MVP * N * 8},
        "roofline": dominant, "mvp_roofline": mvp_roof, "aca_roofline": aca_roof,
        "aca_shapes": aca_shapes,
        "gpu_launches": int(round(launches)),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "paper_setting": paper, "paper_setting_matern": paper_matern,
        "stats": {k: st[k] for k in ("n_adm", "n_dense", "sum_rank", "max_rank",
                                     "rank_cap_hits", "n_rejected", "factor_bytes",
                                     "near_bytes", "mvp_bytes", "t_structure_ms",
                                     "t_aca_ms", "t_dense_ms", "aca_passes",
                                     "n_mispredicted", "reserved_factor_entries")},
    }
    print(json.dumps(line))
    hdist.finalize()


if __name__ == "__main__":
    main()
