#!/usr/bin/env python
"""Throughput of the nonlinear FEAST filter library on one GB300 (or N replicas).

Metric: eigenpairs/s at 1e-10 relative residual.  One step = one whole solve
of the workload: node assembly + node LU factorisations (set_contour) and
every iteration of Algorithm 1 until convergence (solve).  An eigenpair counts
when it lies strictly inside the contour, its relative residual is <= 1e-10 and
its eigenvalue is within 1e-10 (relative) of the stored reference eigenvalues.

Default workload (qep_mixed_n4096): T(l) = l^2 M + l C + K, n = 4096, complex128
inputs, 16 Gauss-Legendre nodes on the stored circle holding 64 eigenvalues,
m0 = 96; node LUs and solves in FP32, A_t Q products as exact digit-split BF16
tensor-core GEMMs, everything else FP64 (FP64-accurate results).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one independent replica per GPU (the path has no exchange step):
value = eigenpairs of all ranks / max over ranks of the step time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "eigenpairs/s at 1e-10 rel. residual"
UNIT = "eigenpairs/s"
FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (vector and tensor), nominal
FP32_SIMT_TFLOPS_AT_MAX = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 lanes x FMA x 2.07 GHz
ONE_SM_FP32_TFLOPS_AT_MAX = 128 * 2 * 2.070e9 / 1e12        # one SM
BEYN_NODES = 256                    # trapezoid nodes of the projected delay problem's moments
# DRAM bytes per launch of a phase's kernels (dram__bytes_read.sum +
# dram__bytes_write.sum summed over the phase's launches in one ncu capture of
# the same code, divided by those launches), keyed by (workload, phase); the
# summaries and their commands are under profiles/.  Absent: not captured.
ROOF_TRAFFIC = {
    # node LU of the n = 4096 QEP, 16 nodes: 62.87 GB over 282 launches
    # (profiles/lu_dram_qep_n4096.md)
    ("qep_mixed_n4096", "lu"): 222.9e6,
    # reduced stage (companion order 192): 2.11 MB over the 10 launches of one
    # iteration (profiles/reduced_stage_dram_m96.md)
    ("qep_mixed_n4096", "reduced"): 0.211e6,
}
TF32_OVER_BF16 = 1.1 / 2.25
# arithmetic of the path per node-factor precision
DTYPES = {"fp64": "c128 (FP64 SIMT LU, solves and products) + f64",
          "fp32": "c64 (tf32x3 tensor LU) + f64",
          "fp32_i8": "c64 (tf32x3 tensor LU) + bf16-split f64 products + f64"}


def load_configs():
    """The workloads, one JSON file each under configs/ (generator, n, seed,
    node-factor precision, tolerance, iteration cap; the contour, m0 and the
    reference eigenvalues are in tests/golden/contours.json)."""
    out = {}
    d = os.path.join(ROOT, "configs")
    for f in sorted(os.listdir(d)):
        if f.endswith(".json"):
            with open(os.path.join(d, f)) as fh:
                spec = json.load(fh)
            out[spec["workload"]] = spec
    return out


WORKLOADS = load_configs()


# ---------------------------------------------------------------------------- ranks
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(value, op, device=None):
    """All-reduce one float over the default process group (identity when alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------- inputs
def load_workload(name):
    import workloads
    spec = WORKLOADS[name]
    with open(os.path.join(ROOT, "tests", "golden", "contours.json")) as f:
        c = json.load(f)[name]
    if spec.get("mixed"):
        problems = [getattr(workloads, spec["gen"])(q["n"], q["n"]) for q in c["problems"]]
        gold = [np.array([complex(*x) for x in q["eigs_inside"]]) for q in c["problems"]]
        return spec, c, problems, gold
    problem = getattr(workloads, spec["gen"])(spec["n"], spec["seed"])
    if spec.get("slices"):
        gold = [np.array([complex(*x) for x in e]) for e in c["eigs_inside"]]
    else:
        gold = np.array([complex(*x) for x in c["eigs_inside"]])
    return spec, c, problem, gold


def describe_terms(problem):
    parts = []
    for t in problem["terms"]:
        A = "I" if t["A"] is None else "A"
        f = ("l^%d" % t["p"]) if t["kind"] == "pow" else ("exp(-%g l)" % t["tau"])
        parts.append("%s %s" % (f, A))
    return " + ".join(parts)


def count_good(lam, rr, gold, center, ra, rb, tol=1e-10, acc=None):
    """Kept pairs strictly inside the contour with relres <= tol, matched one-to-one
    to the reference eigenvalues within relative tol.  With `acc` (new_accuracy()),
    every pair inside also records its relative distance to the nearest reference
    eigenvalue not yet matched and its relative residual."""
    used = np.zeros(len(gold), dtype=bool)
    good = 0
    for lv, r in zip(lam, rr):
        d = lv - center
        if (d.real / ra) ** 2 + (d.imag / rb) ** 2 >= 1.0:
            continue
        d = np.abs(gold - lv) / np.abs(gold) if len(gold) else np.array([np.inf])
        if len(gold):
            d[used] = np.inf
        j = int(np.argmin(d))
        if acc is not None:
            acc["err"].append(float(d[j]))
            acc["relres"].append(float(r))
        if r <= tol and d[j] <= tol:
            used[j] = True
            good += 1
    return good


def new_accuracy():
    return {"err": [], "relres": []}


def accuracy_summary(acc):
    """Per-result error against the FP64 oracle's eigenvalues (stored in
    tests/golden/contours.json), over every pair inside the contour of every
    counted step."""
    e, r = np.array(acc["err"]), np.array(acc["relres"])
    if len(e) == 0:
        return {"pairs": 0}
    return {"pairs": int(len(e)), "max_rel_eig_err": float(np.max(e)),
            "median_rel_eig_err": float(np.median(e)), "max_relres": float(np.max(r)),
            "median_relres": float(np.median(r)),
            "reference": "FP64 oracle eigenvalues inside the contour (tests/golden/contours.json)"}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
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
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))
        return out


_LIVE_PEAKS = {}


def probe_peaks(dev):
    """Denominators the driver's peak file does not hold, measured here with the
    vendor library (measurement only, never on the product path): FP64 DGEMM,
    FP32 SGEMM on the FP32 lanes (TF32 off) and TF32 tensor GEMM, each the best
    of five back-to-back calls timed with CUDA events (TFLOP/s, 2 N^3 flops)."""
    if _LIVE_PEAKS:
        return _LIVE_PEAKS
    import torch
    old = torch.backends.cuda.matmul.allow_tf32
    out = {}
    try:
        for key, dt, nn, tf32 in (("fp64_tflops", torch.float64, 4096, False),
                                  ("fp32_simt_tflops", torch.float32, 8192, False),
                                  ("tf32_tflops", torch.float32, 8192, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(nn, nn, dtype=dt, device=dev)
            b = torch.randn(nn, nn, dtype=dt, device=dev)
            c = torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * nn ** 3 / (best / 1e3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    _LIVE_PEAKS.update(out)
    return out


def peaks():
    pk = _peaks_file()
    pk.update({k: v for k, v in _LIVE_PEAKS.items()})
    return pk


def _peaks_file():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)

        def find(keys, default):
            for k in keys:
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
            return default, "fallback"
        hbm, s1 = find(["hbm_gbs", "hbm_GBs", "hbm"], 6800.0)
        bf16, s2 = find(["bf16_tflops", "bf16"], 1900.0)
        bf16s, _ = find(["bf16_tflops_sustained"], bf16)
        return {"hbm_gbs": hbm, "bf16_tflops": bf16, "bf16_tflops_sustained": bf16s,
                "source": s1 if s1 == s2 else "mixed"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


# ---------------------------------------------------------------------------- roofline
DIGIT_SLICES = 7      # FEAST_NL_FP32_I8: digit slices per operand of A_t Q


def phase_work(name, spec, c, iters, nterms_dense, nterms_sliced=None):
    """Flops of one phase over one solve: algorithmic (4M complex counting), except
    the digit-split A_t Q, which counts the BF16 tensor-core flops it executes
    (s(s+1)/2 slice products of the real-embedded n x 2n x 2 m0 GEMM per term),
    and the reduced eigenvalue stage, counted as a dense Hessenberg reduction
    plus an eigenvalues-only complex QR of the k m0 companion matrix:
    (40/3 + 10) N^3 real flops per iteration."""
    n, m0, nc = spec["n"], c["m0"], c["nc"]
    if name == "lu":
        return nc * (8.0 / 3.0) * n ** 3
    if name == "apply":
        if spec["precision"] == "fp32_i8":
            pairs = DIGIT_SLICES * (DIGIT_SLICES + 1) // 2
            # diagonal terms are applied as diagonal scalings, without slices
            ns = nterms_dense if nterms_sliced is None else nterms_sliced
            return iters * ns * pairs * 2.0 * n * (2 * n) * (2 * m0)
        return iters * nterms_dense * 8.0 * n * n * m0
    if name == "solve":
        return (iters - 1) * nc * 8.0 * n * n * m0
    if name == "project":
        return iters * 8.0 * n * m0 * (3 * m0)
    if name == "reduced":
        if spec["gen"] == "delay_problem":
            # contour moments of the projected problem: one m0 x m0 complex LU
            # plus solves against the m0-column probe at each of the 256 nodes
            return iters * BEYN_NODES * (8.0 / 3.0 + 8.0) * m0 ** 3
        N = 2 * m0
        return iters * (40.0 / 3.0 + 10.0) * N ** 3
    return None


def phase_peak(name, precision, pk, sm_mhz, delay=False):
    """Peak of a phase: (TFLOP/s, bound, where the number comes from).  FP64,
    FP32-lane and TF32 rates are the live library probes (probe_peaks) when
    taken, else nominal figures scaled from the driver's BF16 measurement."""
    clk = (sm_mhz or 2070.0) / 2070.0
    if name in ("lu", "solve") and precision in ("fp32", "fp32_i8"):
        # trailing updates / block substitutions: three TF32 products per FP32 product
        if "tf32_tflops" in pk:
            return (pk["tf32_tflops"] / 3.0, "tensor",
                    "TF32 dense, measured (cuBLAS TF32 GEMM 8192^3, live), / 3 for the split products")
        return (pk["bf16_tflops"] * 0.5 / 3.0, "tensor",
                f"TF32 dense = 0.5 x BF16 ({pk['source']}), / 3 for the split products")
    if name == "apply" and precision == "fp32_i8":
        return (pk["bf16_tflops_sustained"], "tensor",
                f"BF16 dense, {pk['source']} (sustained figure: timed inside a long step)")
    if name == "reduced":
        # FP32 arithmetic on the SIMT lanes; the chip-wide rate is the roofline
        # (the one-SM share is reported beside it for the single-CTA kernels)
        if "fp32_simt_tflops" in pk:
            return (pk["fp32_simt_tflops"], "alu",
                    "FP32 lanes of the whole GPU, measured (cuBLAS SGEMM 8192^3 with TF32 off, live)")
        return (FP32_SIMT_TFLOPS_AT_MAX * clk, "alu",
                "FP32 lanes of all 152 SMs, nominal: 152 x 128 x 2 flop x SM clock")
    if "fp64_tflops" in pk:
        return pk["fp64_tflops"], "alu", "FP64, measured (cuBLAS DGEMM 4096^3, live)"
    return FP64_NOMINAL_TFLOPS, "alu", "FP64 nominal 1.25 TFLOP/s"


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1801_09794_gb300 as P
    spec, c, problem, gold = load_workload(args.workload)
    center = complex(*c["center"])
    n, m0 = spec["n"], c["m0"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    # device-resident inputs for the kernel-side value
    pdev = {"n": n, "terms": []}
    for t in problem["terms"]:
        A = t["A"]
        pdev["terms"].append(dict(t, A=None if A is None else torch.from_numpy(A).to(dev)))
    torch.cuda.synchronize()
    s = P.FeastNL(pdev, spec["precision"], stream=stream.cuda_stream)
    nterms_dense = sum(1 for t in problem["terms"] if t["A"] is not None)
    # a dense term with nothing off its diagonal takes the library's diagonal path
    nterms_sliced = sum(1 for t in problem["terms"] if t["A"] is not None
                        and np.count_nonzero(t["A"]) != np.count_nonzero(np.diag(t["A"])))

    def step(h):
        h.set_contour(center, c["ra"], c["rb"], c["nc"], c["rule"])
        st, info = h.solve(m0, tol=spec["tol"], maxit=spec["maxit"], seed=args.seed,
                           allow=(P.FEAST_NL_ENOT_CONVERGED,))
        return info

    for _ in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = P.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    infos = []
    goods = []
    acc = new_accuracy()
    for _ in range(args.steps):
        infos.append(step(s))
        lam, _, rr = s.get_eigpairs(inside_only=True, vectors=False)
        goods.append(count_good(lam, rr, gold, center, c["ra"], c["rb"], acc=acc))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = P.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    # the phase breakdown from one more step with per-phase events (which runs
    # the iteration eagerly: its time is not part of the measured value)
    s.set_profiling(True)
    step(s)
    torch.cuda.synchronize()
    prof = s.get_profile()
    prof_steps = 1
    s.close()
    barrier()
    ms_max = reduce_over_ranks(ms, "max", dev)
    good_total = reduce_over_ranks(min(goods), "sum", dev)
    value = good_total / (ms_max / 1e3)

    # live per-phase roofline (CUDA events on the library's stream)
    iters = infos[-1].iters
    if not args.no_peak_probe:
        probe_peaks(dev)
    pk = peaks()
    phases = {}
    for name, (pms, pl) in prof.items():
        if pms <= 0:
            continue
        w = phase_work(name, spec, c, iters, nterms_dense, nterms_sliced)
        ent = {"ms_per_step": pms / prof_steps, "launches_per_step": pl / prof_steps}
        if w is not None:
            tf = w / (pms / prof_steps / 1e3) / 1e12
            peak, bound, why = phase_peak(name, spec["precision"], pk, clk.get("sm_mhz"), spec["gen"] == "delay_problem")
            ent.update(tflops=tf, peak_tflops=peak, frac=tf / peak, bound=bound)
            if name == "reduced":
                ent["frac_of_one_sm"] = tf / (peak / 152.0)
        phases[name] = ent
    dom = max(phases, key=lambda k: phases[k]["ms_per_step"])
    d = phases[dom]
    if "tflops" in d:
        peak, bound, why = phase_peak(dom, spec["precision"], pk, clk.get("sm_mhz"), spec["gen"] == "delay_problem")
        roof = {"kernel": f"phase '{dom}' (all its launches)", "bound": bound,
                "achieved": d["tflops"], "peak": peak, "unit": "TFLOP/s", "frac": d["frac"],
                "traffic": ROOF_TRAFFIC.get((args.workload, dom)), "peak_source": why,
                "launches_per_step": d["launches_per_step"],
                "avg_launch_ms": d["ms_per_step"] / max(d["launches_per_step"], 1)}
    else:
        roof = {"kernel": f"phase '{dom}'", "bound": "alu", "achieved": None, "peak": None,
                "unit": None, "frac": None, "traffic": None}
    lu = phases.get("lu", {})

    # end to end through the public API with host (pinned) buffers
    e2e = run_e2e(args, P, torch, problem, spec, c, center, gold, dev)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[spec["precision"]],
           "data": "synthetic (seeded generator, no dataset)",
           "config": {"workload": args.workload, "n": n, "T": describe_terms(problem), "nc": c["nc"],
                      "m0": m0, "count_inside": c["count"], "lu_precision": spec["precision"],
                      "tol": spec["tol"], "iterations": iters,
                      "eigenpairs_per_step": min(goods),
                      "l2": "inputs larger than L2 (A_t %.0f MB, node factors %.2f GB)" % (
                          nterms_dense * n * n * 16 / 1e6,
                          c["nc"] * n * n * (16 if spec["precision"] == "fp64" else 8) / 1e9),
                      "parallelism": f"replicas x{ws}"},
           "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                      "reasons": clk["reasons"]},
           "e2e": e2e, "gpu_launches": int(launches),
           "accuracy": accuracy_summary(acc),
           "roofline": roof,
           "node_lu_tflops": lu.get("tflops"),
           "phases": phases,
           "phases_note": "per-phase device time from one extra step with CUDA events around each "
                          "phase (iteration launched eagerly); the timed steps replay the iteration graph",
           "peaks": pk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, problem, spec, c, center, gold)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_e2e(args, P, torch, problem, spec, c, center, gold, dev):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    pinned = {"n": problem["n"], "terms": []}
    h2d = 0
    for t in problem["terms"]:
        A = t["A"]
        if A is not None:
            A = torch.from_numpy(A).pin_memory()
            h2d += A.numel() * 16
        pinned["terms"].append(dict(t, A=A))
    m0 = c["m0"]
    steps = max(1, min(args.steps, 5))
    times = []
    goods = []
    d2h = 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = P.FeastNL(pinned, spec["precision"])
        h.set_contour(center, c["ra"], c["rb"], c["nc"], c["rule"])
        h.solve(m0, tol=spec["tol"], maxit=spec["maxit"], seed=args.seed,
                allow=(P.FEAST_NL_ENOT_CONVERGED,))
        lam, X, rr = h.get_eigpairs(inside_only=True, vectors=True)
        h.close()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if i > 0:                      # first call warms the allocator and module
            times.append(t1 - t0)
            goods.append(count_good(lam, rr, gold, center, c["ra"], c["rb"]))
            d2h = X.nbytes + lam.nbytes + rr.nbytes
    t = reduce_over_ranks(statistics.median(times), "max", dev)
    g = reduce_over_ranks(min(goods), "sum", dev)
    return {"value": g / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "s_per_step": t, "steps": steps}


# ---------------------------------------------------------------------------- CPU oracle
def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_solve(problem, c, center, spec, X0):
    import oracle as O
    t0 = time.perf_counter()
    r = O.nlfeast(problem, {"center": center, "ra": c["ra"], "rb": c["rb"], "nc": c["nc"],
                            "rule": c["rule"]}, c["m0"], X0, tol=spec["tol"], maxit=spec["maxit"])
    return time.perf_counter() - t0, r


def cpu_baseline(args, problem, spec, c, center, gold):
    """The FP64 oracle, as it stands, on the host cores: one whole solve of the
    workload (node LUs + every iteration), started from the same kind of block."""
    from workloads import start_block
    X0 = start_block(problem["n"], c["m0"], args.seed)
    t, r = oracle_solve(problem, c, center, spec, X0)
    good = count_good(r["lam"], r["relres"], gold, center, c["ra"], c["rb"])
    return {"value": good / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"one whole solve of {args.workload} ({r['iters']} iterations, "
                      f"{c['nc']} node LUs) in {t:.1f} s",
            "seconds": t}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    spec, c, problem, gold = load_workload(args.workload)
    center = complex(*c["center"])
    from workloads import start_block
    X0 = start_block(problem["n"], c["m0"], args.seed)
    # each step is one whole oracle solve (~20 s for the default workload), so the
    # arm caps warm-up at 1 and steps at 3 to end within a few minutes
    w, k = min(args.warmup, 1), min(args.steps, 3)
    for _ in range(w):
        oracle_solve(problem, c, center, spec, X0)
    ts, goods, iters = [], [], 0
    for _ in range(k):
        t, r = oracle_solve(problem, c, center, spec, X0)
        ts.append(t)
        goods.append(count_good(r["lam"], r["relres"], gold, center, c["ra"], c["rb"]))
        iters = r["iters"]
    t = statistics.mean(ts)
    v = min(goods) / t
    sample = f"{k} whole oracle solves of {args.workload} ({iters} iterations each)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": k, "warmup": w, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "n": problem["n"], "nc": c["nc"], "m0": c["m0"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------- slicing
def slices_good(sl, centers, r, gold, tol=1e-10, acc=None):
    good = 0
    for d, cen in enumerate(centers):
        lam, _, rr = sl.get_eigpairs(d, inside_only=True, vectors=False)
        good += count_good(lam, rr, gold[d], cen, r, r, tol, acc=acc)
    return good


def run_slices(args):
    """Spectrum slicing (Sec. 1 and Sec. 3): one step = assembly and LU of all
    64 x 8 node matrices in one batch plus every iteration of all 64 contours
    (graph-replayed), on one stream; eigenpairs counted over all discs."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1801_09794_gb300 as P
    spec, c, problem, gold = load_workload(args.workload)
    n, m0, nc = spec["n"], c["m0"], c["nc"]
    centers = np.array([complex(*x) for x in c["centers"]])
    r = c["r"]
    nd = len(centers)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    pdev = {"n": n, "terms": []}
    for t in problem["terms"]:
        A = t["A"]
        pdev["terms"].append(dict(t, A=None if A is None else torch.from_numpy(A).to(dev)))
    torch.cuda.synchronize()
    h = P.FeastNL(pdev, spec["precision"], stream=stream.cuda_stream)
    nterms_dense = sum(1 for t in problem["terms"] if t["A"] is not None)

    def step():
        sl = P.Slices(h, centers, r, r, nc, c["rule"], stream=stream.cuda_stream)
        st, infos = sl.solve(m0, tol=spec["tol"], maxit=spec["maxit"], seed=args.seed,
                             graph=not args.no_graph, allow=(P.FEAST_NL_ENOT_CONVERGED,))
        return sl, infos

    for _ in range(args.warmup):
        sl, _ = step()
        sl.close()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = P.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    goods, fac_ms, it_ms, iters, gl = [], [], [], [], 0
    acc = new_accuracy()
    for _ in range(args.steps):
        sl, infos = step()
        goods.append(slices_good(sl, centers, r, gold, acc=acc))
        fac_ms.append(infos[0].ms_factor)
        it_ms.append(infos[0].ms_iterate)
        iters.append(max(i.iters for i in infos))
        gl = sl.graph_launches()
        sl.close()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = P.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    h.close()
    barrier()
    ms_max = reduce_over_ranks(ms, "max", dev)
    good_total = reduce_over_ranks(min(goods), "sum", dev)
    value = good_total / (ms_max / 1e3)
    if not args.no_peak_probe:
        probe_peaks(dev)
    pk = peaks()
    # dominant kernel group: the batched node LU (assembly + 512 factorisations,
    # CUDA events around it on the set's stream)
    lu_flops = nd * nc * (8.0 / 3.0) * n ** 3
    fms = statistics.median(fac_ms)
    ach = lu_flops / (fms / 1e3) / 1e12
    peak, bound, why = phase_peak("lu", spec["precision"], pk, clk.get("sm_mhz"))
    roof = {"kernel": f"node assembly + batched LU of {nd * nc} nodes (one launch sequence)",
            "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "peak_source": why, "ms_per_launch_sequence": fms}
    e2e = run_slices_e2e(args, P, torch, problem, spec, c, centers, gold, dev)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "c64 (tf32x3 tensor LU) + bf16-split f64 products + f64",
           "data": "synthetic (seeded generator, no dataset)",
           "config": {"workload": args.workload, "n": n, "T": describe_terms(problem),
                      "discs": nd, "nc": nc, "node_lus": nd * nc, "m0": m0,
                      "count_inside": c["count"], "lu_precision": spec["precision"],
                      "tol": spec["tol"], "iterations_max_over_discs": max(iters),
                      "eigenpairs_per_step": min(goods), "graph": not args.no_graph,
                      "graph_kernels_per_iteration": gl,
                      "ms_factor": fms, "ms_iterate": statistics.median(it_ms),
                      "l2": "inputs larger than L2 (A_t %.0f MB, node factors %.1f GB)" % (
                          nterms_dense * n * n * 16 / 1e6, nd * nc * n * n * 8 / 1e9),
                      "parallelism": f"replicas x{ws}"},
           "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                      "reasons": clk["reasons"]},
           "e2e": e2e, "gpu_launches": int(launches), "accuracy": accuracy_summary(acc),
           "roofline": roof, "node_lu_tflops": ach, "peaks": pk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = slices_cpu_sample(args, problem, spec, c, centers, gold, discs=1)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_slices_e2e(args, P, torch, problem, spec, c, centers, gold, dev):
    """Host buffers in, every kept pair (with vectors) out, per step: handle
    creation (H2D of the coefficients), the slicing set, its solve."""
    pinned = {"n": problem["n"], "terms": []}
    h2d = 0
    for t in problem["terms"]:
        A = t["A"]
        if A is not None:
            A = torch.from_numpy(A).pin_memory()
            h2d += A.numel() * 16
        pinned["terms"].append(dict(t, A=A))
    steps = max(1, min(args.steps, 3))
    times, goods, d2h = [], [], 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = P.FeastNL(pinned, spec["precision"])
        sl = P.Slices(h, centers, c["r"], c["r"], c["nc"], c["rule"])
        sl.solve(c["m0"], tol=spec["tol"], maxit=spec["maxit"], seed=args.seed,
                 allow=(P.FEAST_NL_ENOT_CONVERGED,))
        good, nb = 0, 0
        for d, cen in enumerate(centers):
            lam, X, rr = sl.get_eigpairs(d, inside_only=True, vectors=True)
            good += count_good(lam, rr, gold[d], cen, c["r"], c["r"])
            nb += X.nbytes + lam.nbytes + rr.nbytes
        sl.close()
        h.close()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if i > 0:
            times.append(t1 - t0)
            goods.append(good)
            d2h = nb
    t = reduce_over_ranks(statistics.median(times), "max", dev)
    g = reduce_over_ranks(min(goods), "sum", dev)
    return {"value": g / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "s_per_step": t, "steps": steps}


def slices_cpu_sample(args, problem, spec, c, centers, gold, discs=1, first=0):
    """The FP64 oracle on `discs` of the 64 contours (each: its 8 node LUs and
    every iteration), as eigenpairs per second of that sample."""
    from workloads import start_block
    import oracle as O
    t_all, good = 0.0, 0
    iters = []
    for d in range(first, first + discs):
        cen = centers[d]
        X0 = start_block(problem["n"], c["m0"], args.seed + d)
        t0 = time.perf_counter()
        res = O.nlfeast(problem, {"center": cen, "ra": c["r"], "rb": c["r"], "nc": c["nc"],
                                  "rule": c["rule"]}, c["m0"], X0, tol=spec["tol"],
                        maxit=spec["maxit"])
        t_all += time.perf_counter() - t0
        good += count_good(res["lam"], res["relres"], gold[d], cen, c["r"], c["r"])
        iters.append(res["iters"])
    return {"value": good / t_all, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{discs} of the {len(centers)} discs (discs {first}..{first + discs - 1}: "
                      f"{c['nc']} node LUs and {iters} iterations each) in {t_all:.1f} s; "
                      f"{good} eigenpairs",
            "seconds": t_all}


def run_slices_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    spec, c, problem, gold = load_workload(args.workload)
    centers = np.array([complex(*x) for x in c["centers"]])
    w, k = min(args.warmup, 1), min(args.steps, 3)
    for i in range(w):
        slices_cpu_sample(args, problem, spec, c, centers, gold, discs=1, first=i)
    vals, ts, samples = [], [], []
    for i in range(k):
        r = slices_cpu_sample(args, problem, spec, c, centers, gold, discs=1, first=w + i)
        vals.append(r["value"])
        ts.append(r["seconds"])
        samples.append(r["sample"])
    v = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": k, "warmup": w, "ms_per_step": statistics.mean(ts) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": problem["n"], "discs": len(centers),
                   "nc": c["nc"], "m0": c["m0"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": "; ".join(samples)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------- mixed orders
def mixed_step(P, hs, c, spec, seed, gold, stream=None, acc=None):
    """One step: grouped contours + factorisation of all problems, then their
    solves side by side (one host thread and one stream per problem)."""
    import threading
    qs = c["problems"]
    P.set_contour_group(hs, [complex(*q["center"]) for q in qs], [q["r"] for q in qs],
                        [q["r"] for q in qs], c["nc"], c["rule"], stream=stream)
    res = [None] * len(hs)

    def run(i):
        st, info = hs[i].solve(c["m0"], tol=spec["tol"], maxit=spec["maxit"], seed=seed,
                               allow=(P.FEAST_NL_ENOT_CONVERGED,))
        lam, _, rr = hs[i].get_eigpairs(inside_only=True, vectors=False)
        q = qs[i]
        cen = complex(*q["center"])
        res[i] = (count_good(lam, rr, gold[i], cen, q["r"], q["r"], acc=acc), info.iters,
                  info.ms_factor)
    ts = [threading.Thread(target=run, args=(i,)) for i in range(len(hs))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return res


def run_mixed(args):
    """Mixed-order batch: cubics of n = 256 .. 4096, their node matrices
    factored in one grouped launch sequence, their iterations side by side."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1801_09794_gb300 as P
    spec, c, problems, gold = load_workload(args.workload)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    hs = []
    for p in problems:
        pd = {"n": p["n"], "terms": [dict(t, A=None if t["A"] is None else torch.from_numpy(t["A"]).to(dev))
                                    for t in p["terms"]]}
        hs.append(P.FeastNL(pd, spec["precision"]))
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        mixed_step(P, hs, c, spec, args.seed, gold, stream.cuda_stream)
    # the same factorisations one problem at a time, for comparison
    one_by_one = 0.0
    for h, q in zip(hs, c["problems"]):
        h.set_contour(complex(*q["center"]), q["r"], q["r"], c["nc"], c["rule"])
        h.solve(c["m0"], tol=spec["tol"], maxit=1, seed=args.seed, allow=(P.FEAST_NL_ENOT_CONVERGED,))
    for h, q in zip(hs, c["problems"]):
        h.set_contour(complex(*q["center"]), q["r"], q["r"], c["nc"], c["rule"])
        _, info = h.solve(c["m0"], tol=spec["tol"], maxit=1, seed=args.seed,
                          allow=(P.FEAST_NL_ENOT_CONVERGED,))
        one_by_one += info.ms_factor
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = P.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    goods, fac, iters = [], [], []
    acc = new_accuracy()
    for _ in range(args.steps):
        res = mixed_step(P, hs, c, spec, args.seed, gold, stream.cuda_stream, acc=acc)
        goods.append(sum(r[0] for r in res))
        fac.append(res[0][2])
        iters = [r[1] for r in res]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = P.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    for h in hs:
        h.close()
    barrier()
    ms_max = reduce_over_ranks(ms, "max", dev)
    value = reduce_over_ranks(min(goods), "sum", dev) / (ms_max / 1e3)
    ns = [q["n"] for q in c["problems"]]
    lu_flops = c["nc"] * (8.0 / 3.0) * sum(n ** 3 for n in ns)
    fms = statistics.median(fac)
    if not args.no_peak_probe:
        probe_peaks(dev)
    pk = peaks()
    ach = lu_flops / (fms / 1e3) / 1e12
    peak, bound, why = phase_peak("lu", spec["precision"], pk, clk.get("sm_mhz"))
    roof = {"kernel": f"grouped node assembly + LU of {len(ns) * c['nc']} nodes, n = {ns}",
            "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "peak_source": why, "ms_per_launch_sequence": fms}
    e2e = run_mixed_e2e(args, P, torch, problems, spec, c, gold, dev)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "c64 (tf32x3 tensor LU) + bf16-split f64 products + f64",
           "data": "synthetic (seeded generator, no dataset)",
           "config": {"workload": args.workload, "orders": ns, "degree": 3, "nc": c["nc"],
                      "m0": c["m0"], "count_inside": c["count"], "lu_precision": spec["precision"],
                      "tol": spec["tol"], "iterations": iters, "eigenpairs_per_step": min(goods),
                      "ms_factor_grouped": fms, "ms_factor_one_by_one": one_by_one,
                      "l2": "inputs larger than L2 (A_t %.0f MB)" % (4 * sum(n * n for n in ns) * 16 / 1e6),
                      "parallelism": f"replicas x{ws}"},
           "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                      "reasons": clk["reasons"]},
           "e2e": e2e, "gpu_launches": int(launches), "accuracy": accuracy_summary(acc),
           "roofline": roof, "node_lu_tflops": ach, "peaks": pk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = mixed_cpu_sample(args, problems, spec, c, gold, upto=2)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_mixed_e2e(args, P, torch, problems, spec, c, gold, dev):
    h2d = sum(t["A"].nbytes for p in problems for t in p["terms"] if t["A"] is not None)
    steps = max(1, min(args.steps, 3))
    times, goods = [], []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = [P.FeastNL(p, spec["precision"]) for p in problems]
        res = mixed_step(P, hs, c, spec, args.seed, gold)
        for h in hs:
            h.close()
        torch.cuda.synchronize()
        if i > 0:
            times.append(time.perf_counter() - t0)
            goods.append(sum(r[0] for r in res))
    t = reduce_over_ranks(statistics.median(times), "max", dev)
    g = reduce_over_ranks(min(goods), "sum", dev)
    return {"value": g / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(16 * 3 * c["m0"] * len(problems)), "s_per_step": t,
            "steps": steps}


def mixed_cpu_sample(args, problems, spec, c, gold, upto=2):
    """The FP64 oracle on the `upto` smallest problems of the batch (each: its 8
    node LUs and every iteration)."""
    from workloads import start_block
    import oracle as O
    t_all, good, iters = 0.0, 0, []
    for i in range(upto):
        q = c["problems"][i]
        cen = complex(*q["center"])
        X0 = start_block(q["n"], c["m0"], args.seed)
        t0 = time.perf_counter()
        res = O.nlfeast(problems[i], {"center": cen, "ra": q["r"], "rb": q["r"], "nc": c["nc"],
                                      "rule": c["rule"]}, c["m0"], X0, tol=spec["tol"],
                        maxit=spec["maxit"])
        t_all += time.perf_counter() - t0
        good += count_good(res["lam"], res["relres"], gold[i], cen, q["r"], q["r"])
        iters.append(res["iters"])
    return {"value": good / t_all, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"the {upto} smallest problems (n = {[q['n'] for q in c['problems'][:upto]]}, "
                      f"{iters} iterations) in {t_all:.1f} s; {good} eigenpairs",
            "seconds": t_all}


def run_mixed_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    spec, c, problems, gold = load_workload(args.workload)
    w, k = min(args.warmup, 1), min(args.steps, 3)
    for _ in range(w):
        mixed_cpu_sample(args, problems, spec, c, gold, upto=2)
    rs = [mixed_cpu_sample(args, problems, spec, c, gold, upto=2) for _ in range(k)]
    v = statistics.mean(r["value"] for r in rs)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": k, "warmup": w, "ms_per_step": statistics.mean(r["seconds"] for r in rs) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": args.workload, "orders": [q["n"] for q in c["problems"]],
                   "nc": c["nc"], "m0": c["m0"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": rs[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------- serving
SERVING_WARMUP = 8          # requests of the stream used to warm up (not timed)


def serving_stream():
    """The seeded request stream (random PEPs of degree 2-3, n log-uniform in
    [128, 4096], Poisson arrivals at 200/s) with each request's circle and the
    eigenvalues it encloses, as written by tests/golden/make_contours.py from
    the oracle."""
    with open(os.path.join(ROOT, "tests", "golden", "serving_stream.json")) as f:
        d = json.load(f)
    out = []
    for q in d["requests"]:
        out.append(dict(q, center=complex(*q["center"]),
                        ref=np.array([complex(*x) for x in q["eigs_inside"]])))
    return out


def match_count(lam, rr, ref, tol=1e-10):
    """Pairs with relres <= tol whose eigenvalue is within tol (relative) of a
    distinct reference eigenvalue."""
    used = np.zeros(ref.size, dtype=bool)
    good = 0
    for lv, rv in zip(lam, rr):
        if not (rv <= tol) or ref.size == 0:
            continue
        e = np.abs(ref - lv) / np.maximum(np.abs(ref), 1e-300)
        e[used] = np.inf
        j = int(np.argmin(e))
        if e[j] <= tol:
            used[j] = True
            good += 1
    return good


def run_serving(args):
    """Continuous batching on the serving stream: every request is submitted at
    its arrival time (scaled by `rate_scale`) to the library's server, which
    admits it by device-memory footprint and runs up to `max_active` at once.
    Three passes over the same requests: mixed precision at 200 requests/s,
    mixed precision at about half the measured capacity (latency without
    queueing), and the plain FP64 per-node form one request at a time (the
    baseline the served form has to beat at the same accuracy)."""
    import time
    import paper_1801_09794_gb300 as P
    from workloads import random_pep
    stream = serving_stream()
    ntimed = min(len(stream) - SERVING_WARMUP, 24 * args.steps)
    warm, timed = stream[:SERVING_WARMUP], stream[SERVING_WARMUP:SERVING_WARMUP + ntimed]
    t0s = timed[0]["t"]
    probs = {}
    for q in warm + timed:                        # coefficients drawn before any timing
        probs[q["coef_seed"]] = random_pep(q["n"], q["k"], q["coef_seed"])

    def one_pass(reqs, precision, max_active, rate_scale=1.0, paced=True):
        srv = P.Server(max_active=max_active, hbm_budget=100 << 30)
        start = time.perf_counter()
        tickets = []
        for q in reqs:
            if paced:
                dt = (q["t"] - t0s) / rate_scale - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
            tickets.append((srv.submit(probs[q["coef_seed"]], q["center"], q["r"], q["r"], q["nc"],
                                       q["m0"], precision, tol=1e-12, maxit=60, seed=1), q))
        lats, good, iters, unconv = [], 0, [], 0
        for tk, q in tickets:
            st, info, lat = srv.wait(tk, allow=(0, 3, 4))
            lam, _, rr = srv.fetch(tk, inside_only=True, vectors=False)
            lats.append(lat)
            iters.append(info.iters)
            unconv += int(st != 0)
            good += match_count(lam, rr, q["ref"])
        makespan = time.perf_counter() - start
        stats = srv.stats()
        srv.close()
        lats = np.array(lats)
        return {"value": good / makespan, "eigenpairs_found": good, "makespan_s": makespan,
                "requests": len(reqs), "not_converged": unconv,
                "iterations_median": float(np.median(iters)),
                "latency_ms": {"p50": float(np.percentile(lats, 50)), "p99": float(np.percentile(lats, 99)),
                               "max": float(lats.max())},
                "max_concurrent_seen": stats["max_concurrent"], "max_group_seen": stats["max_group"]}

    act = args.max_active
    one_pass(warm, "fp32_i8", act, paced=False)   # library load, kernels, autotuner
    served = one_pass(timed, "fp32_i8", act)
    capacity = len(timed) / served["makespan_s"]             # requests/s the served form sustains
    half = timed[:max(8, len(timed) // 2)]
    scale = 0.5 * capacity / 200.0
    light = one_pass(half, "fp32_i8", act, rate_scale=scale)
    plain = one_pass(timed, "fp64", 1, paced=False)         # plain FP64 per node, one at a time
    want = int(sum(q["count"] for q in timed))
    ns = np.array([q["n"] for q in timed])
    out = {"metric": "eigenpairs/s under Poisson arrivals (serving)", "value": served["value"],
           "unit": "eigenpairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPES["fp32_i8"], "data": "synthetic (seeded request stream)",
           "config": {"workload": "serving", "requests": len(timed), "warmup_requests": len(warm),
                      "arrival_rate_per_s": 200.0, "n_range": [int(ns.min()), int(ns.max())],
                      "n_median": float(np.median(ns)), "degree": [2, 3],
                      "coefficients": "dense complex N(0,1)/sqrt(n)",
                      "count_range": [int(min(q["count"] for q in timed)), int(max(q["count"] for q in timed))],
                      "eigenpairs_wanted": want, "max_active": act, "tol": 1e-12,
                      "check": "relres <= 1e-10 and eigenvalue within 1e-10 of the oracle's"},
           "served": served,
           "sub_saturating": dict(light, arrival_rate_per_s=200.0 * scale,
                                  note="first half of the stream at half the served form's capacity"),
           "plain_fp64_one_at_a_time": plain,
           "served_over_plain_fp64": served["value"] / plain["value"] if plain["value"] > 0 else None}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serving"], default="qep_mixed_n4096")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32_i8"], default=None,
                    help="override the workload's node-factor precision (e.g. fp64: the plain "
                         "complex128 per-node form, for comparison)")
    ap.add_argument("--no-peak-probe", action="store_true",
                    help="skip the library GEMMs that measure the FP64 / FP32 / TF32 peaks after "
                         "the timed region (use for ncu launch lists)")
    ap.add_argument("--max-active", type=int, default=12,
                    help="serving: requests the server runs at once")
    ap.add_argument("--no-graph", action="store_true",
                    help="slicing workloads: launch each iteration's kernels one by one")
    args = ap.parse_args()
    if args.precision and args.workload in WORKLOADS:
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], precision=args.precision)
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving stream is measured "
                              "on the GPU arm only (the oracle has no server)"}))
            return
        run_serving(args)
    elif WORKLOADS[args.workload].get("mixed"):
        if args.impl == "reference":
            run_mixed_reference(args)
        else:
            run_mixed(args)
    elif WORKLOADS[args.workload].get("slices"):
        if args.impl == "reference":
            run_slices_reference(args)
        else:
            run_slices(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
