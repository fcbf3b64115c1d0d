"""Benchmark: QD (4 x binary64, branch-free) GEMM throughput on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 2048] [--impl gb300|reference]

One step = C := A B in QD arithmetic (Algorithms 13/14, Section 3.1) for a
square n x n problem on seeded nonoverlapping inputs (leading component uniform
in [-1, 1), each lower component u * ulp(previous)/2).  `value` is QD ops/s =
2 n^3 / time (one QD multiply and one QD add per multiply-add), whole job over
all ranks (each rank runs its own replica: weak scaling, no collective).

Printed as ONE JSON line on rank 0, with the GEMM kernel's roofline against
the FP64 pipe (the path is bound by FP64 instructions: 209 per QD multiply-add,
Algorithms 13 and 14), the oracle's throughput on the host cores, an end-to-end figure
with host-resident inputs, clocks sampled during the timed region, and (unless
--no-extras) secondary measurements of the other kernels on bounded samples.

--impl reference times the CPU oracle (the method's plain scalar restatement)
on the host cores on a bounded row sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# FP64-pipe instructions per multicomponent operation, counted from Algorithms
# 6/8 (DD), 11/12 (TD), 13/14 (QD); Tables 1 and 2 give the same totals.
INSTR_MUL = {"dd": 9, "ddc": 9, "td": 39, "qd": 106, "ds": 9, "tf": 39, "qf": 106}
INSTR_ADD = {"dd": 20, "ddc": 11, "td": 57, "qd": 103, "ds": 20, "tf": 57, "qf": 103}
FMA_PER_MUL = {"dd": 1, "ddc": 1, "td": 3, "qd": 6, "ds": 1, "tf": 3, "qf": 6}
# TwoSum (Algorithm 2) calls per add and per multiply.  The hybrid engine issues
# one FP64 add for each instead of six and takes the error term from the integer
# pipes, so a hybrid add issues INSTR_ADD - 5 * TWO_SUMS_ADD FP64 instructions.
TWO_SUMS_ADD = {"dd": 2, "ddc": 1, "td": 7, "qd": 11}
TWO_SUMS_MUL = {"dd": 0, "ddc": 0, "td": 2, "qd": 11}
TWO_SUMS = {p: TWO_SUMS_ADD[p] + TWO_SUMS_MUL[p] for p in TWO_SUMS_ADD}


def add_instr(prec, hybrid=True):
    return INSTR_ADD[prec] - (5 * TWO_SUMS_ADD.get(prec, 0) if hybrid else 0)


def mul_instr(prec, hybrid=True):
    return INSTR_MUL[prec] - (5 * TWO_SUMS_MUL.get(prec, 0) if hybrid else 0)
NOMINAL_FP64_TFLOPS = 1.25  # GB300 dense FP64, FMA = 2 flops
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
SM_MAX_MHZ = 2070.0


def mac_instr(prec):
    return INSTR_MUL[prec] + INSTR_ADD[prec]


def mac_instr_hybrid(prec):
    """FP64-pipe instructions of one multiply-add under the hybrid engine."""
    return add_instr(prec) + mul_instr(prec)


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU, replicas only)
# ---------------------------------------------------------------------------

def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl"
        dist.init_process_group(backend=backend)
        return rank, world
    return 0, 1


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over all ranks (the slowest replica sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, work_per_step, max_time):
    """Whole-job throughput: every rank runs `steps` replicas of the step."""
    return world * steps * work_per_step / max_time


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on the host cores (spawned processes, row samples)
# ---------------------------------------------------------------------------

_ORACLE_CACHE = {}


def _oracle_rows(args):
    """Worker: rows r0..r1-1 (mod n) of C = A B with the oracle; inputs are cached
    per process so that only the multiplication is inside the caller's timing."""
    prec, n, seed, r0, r1 = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import mpref
    from paper_2603_14926_gb300 import inputs

    key = (prec, n, seed)
    if key not in _ORACLE_CACHE:
        K, dt = mpref.PRECS[prec]
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[key] = (inputs.mp_uniform(seed, (n, n), K, dt, stream=inputs.STREAM_A),
                              inputs.mp_uniform(seed, (n, n), K, dt, stream=inputs.STREAM_B))
    A, B = _ORACLE_CACHE[key]
    rows = [i % n for i in range(r0, r1)]
    t = time.perf_counter()
    mpref.gemm(prec, np.ascontiguousarray(A[:, rows, :]), B)
    return time.perf_counter() - t


def _oracle_row_rates(_=None):
    """Worker: the oracle, as it stands, on ONE host core over a bounded sample of
    each hot-path row's workload (QD), in the units bench.py reports for the GPU."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import mpref as o
    from paper_2603_14926_gb300 import inputs

    K = 4
    out = {}

    def timed(fn):
        t = time.perf_counter()
        fn()
        return time.perf_counter() - t

    n = 1 << 19
    x = inputs.mp_uniform(1, n, K, stream=inputs.STREAM_X)
    y = inputs.mp_uniform(1, n, K, stream=inputs.STREAM_Y)
    alpha = inputs.mp_uniform(2, 1, K)[:, 0]
    t = timed(lambda: o.axpy("qd", alpha, x, y))
    out["axpy"] = {"elements_per_s": n / t, "sample": f"n = {n}"}
    t = timed(lambda: o.dot("qd", x, y))
    out["dot"] = {"elements_per_s": n / t, "sample": f"n = {n}"}
    m, k = 64, 8192
    A = inputs.mp_uniform(2, (m, k), K)
    xv = inputs.mp_uniform(3, k, K, stream=inputs.STREAM_X)
    t = timed(lambda: o.gemv("qd", A, xv))
    out["gemv"] = {"mac_per_s": m * k / t, "sample": f"{m} rows of 8192 x 8192"}
    deg, npts, npoly = 256, 512, 8
    off = np.arange(0, (npoly + 1) * (deg + 1), deg + 1, dtype=np.int64)
    coef = inputs.mp_uniform(4, npoly * (deg + 1), K, stream=inputs.STREAM_C)
    xs = inputs.mp_uniform(5, npoly * npts, K, stream=inputs.STREAM_X)
    dy = inputs.mp_uniform(6, npoly * npts, K, stream=inputs.STREAM_Y)
    steps = npoly * npts * deg
    t = timed(lambda: o.polyeval("qd", off, coef, npts, xs))
    out["horner_fwd"] = {"steps_per_s": steps / t, "sample": f"{npoly} polynomials x degree {deg} x {npts} points"}
    t = timed(lambda: o.polyeval_estrin("qd", off, coef, npts, xs))
    out["estrin_fwd"] = {"steps_per_s": steps / t, "sample": out["horner_fwd"]["sample"]}
    t = timed(lambda: o.polyeval_backward("qd", off, coef, npts, xs, dy))
    out["horner_bwd"] = {"steps_per_s": steps / t, "sample": out["horner_fwd"]["sample"]}
    nc = 128
    Ar, Ai = inputs.mp_uniform(7, (nc, nc), K), inputs.mp_uniform(8, (nc, nc), K)
    Br, Bi = inputs.mp_uniform(9, (nc, nc), K), inputs.mp_uniform(10, (nc, nc), K)
    t = timed(lambda: o.cgemm("qd", Ar, Ai, Br, Bi))
    out["complex_gemm_3m"] = {"complex_qd_ops_per_s": 8.0 * nc ** 3 / t, "sample": f"n = {nc}"}
    ns = 192
    As, Bs = inputs.mp_uniform(2, (ns, ns), K, stream=inputs.STREAM_A), inputs.mp_uniform(2, (ns, ns), K, stream=inputs.STREAM_B)
    t = timed(lambda: o.gemm_strassen("qd", As, Bs, 32))
    out["gemm_strassen"] = {"classical_equiv_qd_ops_per_s": 2.0 * ns ** 3 / t, "sample": f"n = {ns}, cutoff 32"}
    # Durand-Kerner: a degree-stratified slice of the batched-root workload, 2 sweeps
    prob = inputs.dk_problem(3, 4096, 10, 500)
    sel = np.argsort(prob.degrees, kind="stable")[np.linspace(0, 4095, 8).astype(int)]
    parts = [(prob.rootdata[prob.root_off[b]:prob.root_off[b + 1]], prob.delta[prob.root_off[b]:prob.root_off[b + 1]])
             for b in sel]
    sub = inputs.DKProblem(prob.degrees[sel], np.concatenate([r for r, _ in parts]),
                           np.concatenate([d for _, d in parts]))
    coef = o.poly_from_roots("qd", sub)
    res = {}
    t = timed(lambda: res.update(r=o.roots("qd", sub.coef_off, coef, radius=1.1, max_iter=2)))
    its = res["r"][1]
    out["durand_kerner"] = {"root_sweeps_per_s": float(np.sum(sub.degrees * its)) / t,
                            "sample": f"degrees {sub.degrees.tolist()}, 2 sweeps"}
    # Table 4's standard / BF ratio on one host core (the paper's non-SIMD column):
    # the oracle's GEMM at n = 96, conventional against branch-free
    ng = 96
    ratios = {}
    for bf, nb in (("dd", "ddc"), ("td", "tdc"), ("qd", "qdc")):
        Kb = o.PRECS[bf][0]
        Ag = inputs.mp_uniform(2, (ng, ng), Kb, stream=inputs.STREAM_A)
        Bg = inputs.mp_uniform(2, (ng, ng), Kb, stream=inputs.STREAM_B)
        tb = timed(lambda: o.gemm(bf, Ag, Bg))
        tn = timed(lambda: o.gemm(nb, Ag, Bg))
        ratios[bf.upper()] = {f"{bf}_s": tb, f"{nb}_s": tn, "standard_over_bf": tn / tb}
    out["bf_over_nobf"] = {**ratios, "sample": f"GEMM n = {ng}, one core, the oracle (scalar C, no SIMD)"}
    # Eq. 1 at n = 2049: rows of the classical QD product
    n1, rows = 2049, 4
    s5, s3, tq, ia, ib = inputs.eq1_factors(n1, K)
    r5 = o.mul("qd", np.repeat(s5[:, None], 2 * n1, 1), tq)
    r3 = o.mul("qd", np.repeat(s3[:, None], 2 * n1, 1), tq)
    A1 = np.ascontiguousarray(r5[:, ia[:rows]])
    B1 = np.ascontiguousarray(r3[:, ib])
    t = timed(lambda: o.gemm("qd", A1, B1))
    out["eq1_n2049"] = {"qd_ops_per_s": 2.0 * rows * n1 * n1 / t, "sample": f"{rows} rows of the QD classical product"}
    # the paper's DK problem (Chebyshev, n = 64): one whole solve
    cq = inputs.rational_to_mp(inputs.chebyshev_quadrature(64), K)
    res = {}
    t = timed(lambda: res.update(r=o.roots("qd", np.array([0, 65]), cq)))
    out["chebyshev_dk"] = {"single_solve_s": t, "precision": "qd", "sweeps": int(res["r"][1][0]),
                           "status": int(res["r"][2][0]), "sample": "n = 64, one solve to the end"}
    return out


class OraclePool:
    """Process pool started before the first GPU call (spawn context)."""

    def __init__(self, cores):
        import multiprocessing as mp_

        self.cores = cores
        self.pool = mp_.get_context("spawn").Pool(cores)

    def warm(self, prec, n, seed):
        """Generate the inputs in every worker (outside any timing)."""
        self.pool.map(_oracle_rows, [(prec, n, seed, 0, 0)] * (4 * self.cores), chunksize=1)

    def gemm_rows(self, prec, n, seed, rows_per_core):
        t = time.perf_counter()
        jobs = [(prec, n, seed, c * rows_per_core, (c + 1) * rows_per_core) for c in range(self.cores)]
        list(self.pool.map(_oracle_rows, jobs, chunksize=1))
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_rows(pool, ex):
    """The CPU baseline per hot-path row: the oracle on one host core (bounded
    samples, one spawned worker) beside each GPU row of `ex`, with the GPU's
    throughput over the oracle's (for the Chebyshev solve, the oracle's time over
    the GPU's)."""
    o = pool.pool.apply(_oracle_row_rates)
    def put(key, unit, gpu):
        if key in o and gpu:
            o[key]["gpu_" + unit] = gpu
            o[key]["gpu_over_oracle"] = gpu / o[key][unit]

    if "axpy" in ex:
        put("axpy", "elements_per_s", ex["axpy"]["n"] / (ex["axpy"]["ms"] / 1e3))
    if "dot" in ex:
        put("dot", "elements_per_s", ex["dot"]["n"] / (ex["dot"]["ms"] / 1e3))
    if "gemv" in ex:
        put("gemv", "mac_per_s", ex["gemv"]["m"] * ex["gemv"]["n"] / (ex["gemv"]["ms"] / 1e3))
    if "horner_fwd" in ex:
        h = ex["horner_fwd"]
        steps = h["polys"] * h["points"] * h["degree"]
        put("horner_fwd", "steps_per_s", steps / (h["ms"] / 1e3))
        if "estrin_fwd" in ex:
            put("estrin_fwd", "steps_per_s", steps / (ex["estrin_fwd"]["ms"] / 1e3))
        if "horner_bwd" in ex:
            put("horner_bwd", "steps_per_s", steps / (ex["horner_bwd"]["ms"] / 1e3))
    if "complex_gemm_3m" in ex:
        put("complex_gemm_3m", "complex_qd_ops_per_s", ex["complex_gemm_3m"]["complex_qd_ops_per_s"])
    if ex.get("gemm_strassen"):
        best = max(v["classical_equiv_qd_ops_per_s"] for v in ex["gemm_strassen"].values())
        put("gemm_strassen", "classical_equiv_qd_ops_per_s", best)
    if "durand_kerner" in ex:
        put("durand_kerner", "root_sweeps_per_s", ex["durand_kerner"]["root_sweeps_per_s"])
    if "eq1_n2049" in ex and "qd" in ex["eq1_n2049"]:
        put("eq1_n2049", "qd_ops_per_s", 2.0 * ex["eq1_n2049"]["n"] ** 3 / ex["eq1_n2049"]["qd"]["classical"]["s"])
    if "bf_over_nobf" in ex and "bf_over_nobf" in o:
        for key in ("DD", "TD", "QD"):
            g = ex["bf_over_nobf"].get(key, {})
            gpu = [v["standard_over_bf"] for k, v in g.items() if k.endswith("_fp64")]
            if gpu:
                o["bf_over_nobf"][key]["gpu_standard_over_bf_fp64_engine"] = gpu[-1]
    if "chebyshev_dk" in ex and "chebyshev_dk" in o:
        g, oc = ex["chebyshev_dk"], o["chebyshev_dk"]
        oc["gpu_single_solve_s"] = g["single_solve_gpu_s"]
        oc["gpu_precision"], oc["gpu_sweeps"] = g["precision"], g["sweeps"]
        # a ratio only for the same work: same precision and the same number of sweeps
        same = g["precision"] == oc["precision"] and g["sweeps"] == oc["sweeps"]
        oc["same_work"] = same
        oc["gpu_over_oracle"] = oc["single_solve_s"] / g["single_solve_gpu_s"] if same else None
    return o


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_build():
    from oracle import mpref

    mpref.build()


def cpu_baseline(pool, prec, n, seed, target_s=12.0):
    """Oracle QD GEMM on a row sample sized for ~target_s seconds on all cores."""
    pool.warm(prec, n, seed)
    probe = pool.gemm_rows(prec, n, seed, 1)  # one row per core, also warms up the workers
    rows = max(1, int(target_s / max(probe, 1e-3)))
    t = pool.gemm_rows(prec, n, seed, rows)
    total_rows = rows * pool.cores
    v = 2.0 * total_rows * n * n / t
    return {"value": v, "unit": "QD ops/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"{total_rows} rows of C ({rows} per core) of the {prec.upper()} GEMM n={n}, "
                      f"{t:.1f} s wall on {pool.cores} host cores (spawned processes)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_inputs(prec, n, seed):
    from paper_2603_14926_gb300 import inputs
    import paper_2603_14926_gb300 as mpg

    K = mpg.PRECS[prec][0]
    dt = np.float64 if mpg.PRECS[prec][1] == "float64" else np.float32
    A = inputs.mp_uniform(seed, (n, n), K, dt, stream=inputs.STREAM_A)
    B = inputs.mp_uniform(seed, (n, n), K, dt, stream=inputs.STREAM_B)
    return A, B


def time_region(fn, steps, world, stream):
    import torch

    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    per = []
    for _ in range(steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fn()
        s1.record(stream)
        per.append((s0, s1))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    total = e0.elapsed_time(e1) / 1e3
    launches = [a.elapsed_time(b) / 1e3 for a, b in per]
    return total, launches


def gemm_profile_name(prec, n, hybrid):
    return f"k_gemm_{'hybrid_' if hybrid else ''}{prec}_{n}.md"


def profile_value(name, key, cast=float):
    """A `key: value` line of the ncu summary profiles/<name>, or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", name)):
            if line.startswith(key + ":"):
                return cast(line.split(":", 1)[1].strip())
    except OSError:
        pass
    return None


def gemm_traffic(prec, n, hybrid):
    """DRAM bytes per launch recorded by ncu for this kernel and size, if any."""
    return profile_value(gemm_profile_name(prec, n, hybrid), "traffic_bytes_per_launch", int)


def gemm_pipes(prec, n, hybrid, launch_s, fp64_achieved_g, fp64_nominal_g, fp64_live_g):
    """Both pipes the hybrid GEMM loads: FP64 instructions/s against the FP64
    pipe, and integer instructions/s against the integer ALU pipe and the FMA
    pipe's integer rate (each measured live with the pipe microbenchmark), using
    the per-multiply-add lane-instruction counts of this kernel's ncu summary
    (sm__inst_executed_pipe_alu / _fma x 32 / n^3; they do not depend on n)."""
    name = gemm_profile_name(prec, n, hybrid)
    alu = profile_value(name, "alu_lane_instr_per_mac")
    fma = profile_value(name, "fma_lane_instr_per_mac")
    out = {"fp64": {"instr_per_mac": mac_instr_hybrid(prec) if hybrid else mac_instr(prec),
                    "achieved_G_per_s": fp64_achieved_g, "peak_nominal_G_per_s": fp64_nominal_g,
                    "peak_measured_live_G_per_s": fp64_live_g,
                    "frac_of_nominal": fp64_achieved_g / fp64_nominal_g,
                    "frac_of_measured": fp64_achieved_g / fp64_live_g}}
    if alu is None or fma is None:
        out["integer"] = None
        return out
    live = int_pipe_peaks_live()
    for key, per_mac in (("alu", alu), ("fma", fma)):
        rate = n ** 3 * per_mac / launch_s
        out[key] = {"lane_instr_per_mac": per_mac, "achieved_T_per_s": rate / 1e12,
                    "peak_measured_live_T_per_s": live[key] / 1e12, "frac_of_measured": rate / live[key]}
    out["source"] = (f"per-multiply-add counts: profiles/{name}; peaks: mp_peak_run kinds 0 (DFMA), "
                     "7 (LOP3, integer ALU pipe) and 8 (IMAD, FMA pipe) run in this process")
    out["bound"] = max(("fp64", out["fp64"]["frac_of_measured"]), ("alu", out["alu"]["frac_of_measured"]),
                       ("fma", out["fma"]["frac_of_measured"]), key=lambda kv: kv[1])[0]
    return out


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def fp64_peak_live():
    import paper_2603_14926_gb300 as mpg

    mpg.peak(0, iters=256)
    rate, _ = mpg.peak(0, iters=4096)
    return rate


def int_pipe_peaks_live():
    """Lane instructions/s of the integer ALU pipe (LOP3 chains) and of integer
    work on the FMA pipe (IMAD chains), measured now with the pipe
    microbenchmark (mp_peak_run kinds 7 and 8), best of two launch shapes."""
    import paper_2603_14926_gb300 as mpg

    sms = mpg.lib().mp_sm_count()
    out = {}
    for kind, name in ((7, "alu"), (8, "fma")):
        best = 0.0
        for per_sm, thr in ((4, 256), (8, 256)):
            mpg.peak(kind, iters=1024, blocks=sms * per_sm, threads=thr)
            rate, _ = mpg.peak(kind, iters=65536, blocks=sms * per_sm, threads=thr)
            best = max(best, rate)
        out[name] = best
    return out


def extras(prec="qd", quick=False):
    """Secondary measurements of the other hot-path kernels (bounded samples)."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    out = {}
    K = mpg.PRECS[prec][0]
    # FP64 instructions these kernels issue (hybrid engine for binary64) and the
    # paper's all-FP64 sequence they reproduce bit for bit
    ins, ins_paper = mac_instr_hybrid(prec), mac_instr(prec)
    peak = NOMINAL_FP64_TFLOPS * 1e12 / 2

    def rates(fp64, paper, t):
        return {"fp64_instr_frac": fp64 / t / peak, "paper_sequence_equiv_frac": paper / t / peak}

    def timed(fn, reps=3, warm=True):
        if warm:
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    n = 1 << 24
    x = dev(inputs.mp_uniform(1, n, K, stream=inputs.STREAM_X))
    y = dev(inputs.mp_uniform(1, n, K, stream=inputs.STREAM_Y))
    t = timed(lambda: mpg.axpy(prec, [0.5] + [0.0] * (K - 1), x, y))
    out["axpy"] = {"n": n, "ms": t * 1e3, "GB/s": 3 * K * 8 * n / t / 1e9, **rates(n * ins, n * ins_paper, t)}
    ws = torch.empty(mpg.dot_workspace(prec, n), dtype=torch.uint8, device="cuda")
    r = mpg.empty(prec)
    t = timed(lambda: mpg.dot(prec, x, y, out=r, ws=ws))
    out["dot"] = {"n": n, "ms": t * 1e3, **rates(n * ins, n * ins_paper, t)}
    del x, y
    # binary32 components: AXPY and dot are bound by HBM, not by the FP32 pipe
    hbm = measured_hbm_gbs()
    for p32 in ("ds", "qf"):
        K32 = mpg.PRECS[p32][0]
        n32 = 1 << 26
        x32 = dev(inputs.mp_uniform(1, n32, K32, np.float32, stream=inputs.STREAM_X))
        y32 = dev(inputs.mp_uniform(1, n32, K32, np.float32, stream=inputs.STREAM_Y))
        ta = timed(lambda: mpg.axpy(p32, [0.5] + [0.0] * (K32 - 1), x32, y32))
        ws32 = torch.empty(mpg.dot_workspace(p32, n32), dtype=torch.uint8, device="cuda")
        r32 = mpg.empty(p32)
        td = timed(lambda: mpg.dot(p32, x32, y32, out=r32, ws=ws32))
        ab, db = 3 * K32 * 4 * n32, 2 * K32 * 4 * n32  # AXPY reads x, y and writes y; dot reads x, y
        out[f"axpy_{p32}"] = {"n": n32, "ms": ta * 1e3, "GB/s": ab / ta / 1e9,
                              "hbm_frac_of_measured": ab / ta / 1e9 / hbm if hbm else None}
        out[f"dot_{p32}"] = {"n": n32, "ms": td * 1e3, "GB/s": db / td / 1e9,
                             "hbm_frac_of_measured": db / td / 1e9 / hbm if hbm else None}
        del x32, y32, ws32
    m = 8192
    A = dev(inputs.mp_uniform(2, (m, m), K))
    xv = dev(inputs.mp_uniform(3, m, K, stream=inputs.STREAM_X))
    yv = mpg.empty(prec, m)
    t = timed(lambda: mpg.gemv(prec, A, xv, out=yv))
    out["gemv"] = {"m": m, "n": m, "ms": t * 1e3, **rates(m * m * ins, m * m * ins_paper, t)}
    del A
    # complex GEMM by the 3M method (Eq. 3) vs the real GEMM, n = 1024, Eq. 2 entries
    nc = 512 if quick else 1024
    Ur, Er, Ui, Ei = inputs.complex_eq2(7, (nc, nc), K)
    mk = lambda U, E: mpg.mul(prec, dev(U.reshape(K, -1)),  # noqa: E731
                              dev(inputs.mp_from_double(E.reshape(-1), K))).reshape(K, nc, nc)
    Ar, Ai, Br, Bi = mk(Ur, Er), mk(Ui, Ei), mk(Ur, Ei), mk(Ui, Er)
    Cr, Ci = mpg.empty(prec, nc, nc), mpg.empty(prec, nc, nc)
    tc = timed(lambda: mpg.cgemm(prec, Ar, Ai, Br, Bi, out=(Cr, Ci)), reps=1)
    tr = timed(lambda: mpg.gemm(prec, Ar, Br, out=Cr), reps=1)
    out["complex_gemm_3m"] = {"n": nc, "ms": tc * 1e3, "real_gemm_ms": tr * 1e3, "complex_over_real": tc / tr,
                              "complex_qd_ops_per_s": 8.0 * nc ** 3 / tc,
                              **rates(3 * nc ** 3 * ins, 3 * nc ** 3 * ins_paper, tc)}
    del Ar, Ai, Br, Bi, Cr, Ci
    # Horner forward/backward: 1024 polynomials, degree 256, 4096 real points each
    npoly, deg, npts = (256 if quick else 1024), 256, 4096
    off = torch.arange(0, (npoly + 1) * (deg + 1), deg + 1, dtype=torch.int64, device="cuda")
    coef = dev(inputs.mp_uniform(4, npoly * (deg + 1), K, stream=inputs.STREAM_C))
    xs = dev(inputs.mp_uniform(5, npoly * npts, K, stream=inputs.STREAM_X))
    dy = dev(inputs.mp_uniform(6, npoly * npts, K, stream=inputs.STREAM_Y))
    t = timed(lambda: mpg.polyeval(prec, off, coef, npts, xs), reps=1)
    steps = npoly * npts * deg
    out["horner_fwd"] = {"polys": npoly, "degree": deg, "points": npts, "ms": t * 1e3,
                         **rates(steps * ins, steps * ins_paper, t)}
    # Estrin's scheme (Section 4.1) on the same workload: n multiply-add pairs plus
    # ceil(log2(n+1)) - 1 squarings per point, against Horner's n pairs
    te = timed(lambda: mpg.polyeval(prec, off, coef, npts, xs, scheme="estrin"), reps=1)
    lev = int(np.ceil(np.log2(deg + 1)))
    est_fp64 = npoly * npts * (deg * ins + (lev - 1) * mul_instr(prec))
    est_paper = npoly * npts * (deg * ins_paper + (lev - 1) * INSTR_MUL[prec])
    out["estrin_fwd"] = {"ms": te * 1e3, "vs_horner": te / t, **rates(est_fp64, est_paper, te)}
    # latency case: one polynomial of degree 256 at 64 points (one block)
    off1, c1, x1 = off[:2].contiguous(), coef[:, :deg + 1].contiguous(), xs[:, :64].contiguous()
    th1 = timed(lambda: mpg.polyeval(prec, off1, c1, 64, x1), reps=5)
    te1 = timed(lambda: mpg.polyeval(prec, off1, c1, 64, x1, scheme="estrin"), reps=5)
    out["estrin_latency_one_poly_64_points"] = {"horner_ms": th1 * 1e3, "estrin_ms": te1 * 1e3,
                                                "estrin_over_horner": te1 / th1}
    tb = timed(lambda: mpg.polyeval_backward(prec, off, coef, npts, xs, dy), reps=1)
    # dx: 2 mul + 2 add per step (+1 mul), dcoef: 1 mul + 1 add per (coefficient, point),
    # both on the hybrid engine
    bw = lambda i, mu: steps * 2 * i + npoly * npts * mu + npoly * npts * (deg + 1) * i  # noqa: E731
    out["horner_bwd"] = {"ms": tb * 1e3, "vs_fwd": tb / t,
                         **rates(bw(ins, mul_instr(prec)), bw(ins_paper, INSTR_MUL[prec]), tb)}
    # the plain per-polynomial launch loop for the adjoint: one polyeval_backward
    # call (both kernels) per polynomial, back to back on one stream, on a sample
    # of 8 polynomials spread over the batch; same bits as the batched call
    dcb, dxb = mpg.polyeval_backward(prec, off, coef, npts, xs, dy)
    pick = np.linspace(0, npoly - 1, 8).astype(int)
    off_q = torch.tensor([0, deg + 1], dtype=torch.int64, device="cuda")
    parts = [(coef[:, q * (deg + 1):(q + 1) * (deg + 1)].contiguous(), xs[:, q * npts:(q + 1) * npts].contiguous(),
              dy[:, q * npts:(q + 1) * npts].contiguous()) for q in pick]
    res_q = []
    tq = timed(lambda: res_q.append([mpg.polyeval_backward(prec, off_q, cq, npts, xq, dq) for cq, xq, dq in parts]),
               reps=1)
    same_q = all(torch.equal(dcq.view(torch.int64), dcb[:, q * (deg + 1):(q + 1) * (deg + 1)].view(torch.int64)) and
                 torch.equal(dxq.view(torch.int64), dxb[:, q * npts:(q + 1) * npts].view(torch.int64))
                 for q, (dcq, dxq) in zip(pick, res_q[-1]))
    out["horner_bwd"]["per_poly_loop"] = {
        "form": "one mp_polyeval_backward_P call per polynomial (its dx and dcoef kernels), back to back on one "
                "stream", "polys": len(pick), "ms": tq * 1e3, "identical_bits_to_batched": bool(same_q),
        "batched_over_loop_per_unit_work": (tq / len(pick)) / (tb / npoly)}
    del off, coef, xs, dy, dcb, dxb, parts, res_q
    # GEMM adjoint through torch.autograd.Function: dA = dC B^T, dB = A^T dC
    from paper_2603_14926_gb300.autograd import mp_gemm

    ng = 1024 if quick else 2048
    A = dev(inputs.mp_uniform(11, (ng, ng), K)).requires_grad_(True)
    B = dev(inputs.mp_uniform(12, (ng, ng), K)).requires_grad_(True)
    dC = dev(inputs.mp_uniform(13, (ng, ng), K))
    C = mp_gemm(prec, A, B)
    tf = timed(lambda: mp_gemm(prec, A, B), reps=1)
    tbk = timed(lambda: torch.autograd.grad(C, (A, B), dC, retain_graph=True), reps=1)
    out["gemm_backward"] = {"n": ng, "forward_ms": tf * 1e3, "backward_ms": tbk * 1e3, "backward_over_forward": tbk / tf,
                            "path": "torch.autograd.Function (MPGemm): two transposed-operand GEMMs",
                            **rates(2 * ng ** 3 * ins, 2 * ng ** 3 * ins_paper, tbk)}
    del A, B, dC, C
    # square GEMM across precisions and sizes (built-in configuration; one launch each)
    sizes = (1024,) if quick else (1024, 2048, 4096)
    grid = {}
    for p2 in ("dd", "td", "qd"):
        K2 = mpg.PRECS[p2][0]
        for n2 in sizes:
            A2 = dev(inputs.mp_uniform(2, (n2, n2), K2, stream=inputs.STREAM_A))
            B2 = dev(inputs.mp_uniform(2, (n2, n2), K2, stream=inputs.STREAM_B))
            C2 = mpg.empty(p2, n2, n2)
            # the smallest size warms the precision's kernels; larger ones run once
            t2 = timed(lambda: mpg.gemm(p2, A2, B2, out=C2), reps=1, warm=n2 == sizes[0])
            fp64 = n2 ** 3 * (add_instr(p2) + mul_instr(p2))
            grid[f"{p2}_{n2}"] = {"ms": t2 * 1e3, "mac_per_s": n2 ** 3 / t2,
                                  **rates(fp64, n2 ** 3 * mac_instr(p2), t2)}
            del A2, B2, C2
    fp32_peak = NOMINAL_FP32_TFLOPS * 1e12 / 2
    for p2 in ("tf", "qf"):
        K2 = mpg.PRECS[p2][0]
        n2 = sizes[-1]
        A2 = dev(inputs.mp_uniform(2, (n2, n2), K2, np.float32, stream=inputs.STREAM_A))
        B2 = dev(inputs.mp_uniform(2, (n2, n2), K2, np.float32, stream=inputs.STREAM_B))
        C2 = mpg.empty(p2, n2, n2)
        t2 = timed(lambda: mpg.gemm(p2, A2, B2, out=C2), reps=1)
        grid[f"{p2}_{n2}"] = {"ms": t2 * 1e3, "mac_per_s": n2 ** 3 / t2,
                              "fp32_instr_frac_of_nominal": n2 ** 3 * mac_instr(p2) / t2 / fp32_peak}
        del A2, B2, C2
    out["gemm_sizes"] = grid
    # Strassen's recursion (Section 3.1's scheme) on the QD GEMM: 7^L leaf GEMMs of
    # size n / 2^L plus 18 elementwise sums per node, against the classical fold
    runs = ((1024, 1024),) if quick else ((2048, 2048), (4096, 4096), (4096, 2048))
    strassen = {}
    for i, (n2, cut) in enumerate(runs):
        A2 = dev(inputs.mp_uniform(2, (n2, n2), K, stream=inputs.STREAM_A))
        B2 = dev(inputs.mp_uniform(2, (n2, n2), K, stream=inputs.STREAM_B))
        C2 = mpg.empty(prec, n2, n2)
        ws2 = torch.empty(max(mpg.gemm_strassen_workspace(prec, n2, n2, n2, cut), 1), dtype=torch.uint8,
                          device="cuda")
        t2 = timed(lambda: mpg.gemm_strassen(prec, A2, B2, cut, out=C2, ws=ws2), reps=1, warm=i == 0)
        L, h, sums = 0, n2, 0
        while h >= cut:
            h = (h + 1) // 2
            sums += 7 ** L * 18 * h * h
            L += 1
        macs = 7 ** L * h ** 3
        cls = grid.get(f"{prec}_{n2}", {}).get("ms")
        strassen[f"n{n2}_cutoff{cut}"] = {
            "levels": L, "leaf": h, "ms": t2 * 1e3, "classical_ms": cls,
            "speedup_over_classical": cls / (t2 * 1e3) if cls else None,
            "classical_equiv_qd_ops_per_s": 2.0 * n2 ** 3 / t2,
            **rates(macs * ins + sums * add_instr(prec), macs * ins_paper + sums * INSTR_ADD[prec], t2)}
        del A2, B2, C2, ws2
    out["gemm_strassen"] = strassen
    out["bf_over_nobf"] = bf_over_nobf_extra((1024,) if quick else (1024, 2048))
    out["eq1_n2049"] = eq1_extra(1025 if quick else 2049)
    return out


def bf_over_nobf_extra(sizes):
    """Table 4's standard / BF ratio in its GPU form: the same square GEMM kernel
    and engine with the conventional arithmetic (ddc: Algorithms 4 + 7; tdc:
    Algorithms 9 + 10 with TWRenormalize; qdc: the QD library's quad word with
    QWRenormalize) over the branch-free one (dd, td, qd: Algorithms 6/8, 11/12,
    13/14).  Both engines: the hybrid one (built-in, TwoSum's error term on the
    integer pipes) and the all-FP64 one (configuration 4)."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = {}
    for bf, nb in (("dd", "ddc"), ("td", "tdc"), ("qd", "qdc")):
        K = mpg.PRECS[bf][0]
        row = {}
        for n in sizes:
            A = dev(inputs.mp_uniform(2, (n, n), K, stream=inputs.STREAM_A))
            B = dev(inputs.mp_uniform(2, (n, n), K, stream=inputs.STREAM_B))
            C = mpg.empty(bf, n, n)
            for cfg, eng in ((-1, "hybrid"), (4, "fp64")):
                ms = {}
                for p in (bf, nb):
                    mpg.gemm(p, A, B, out=C, config=cfg)  # warm (module load, first launch)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    mpg.gemm(p, A, B, out=C, config=cfg)
                    e1.record()
                    torch.cuda.synchronize()
                    ms[p] = e0.elapsed_time(e1)
                row[f"n{n}_{eng}"] = {f"{bf}_ms": ms[bf], f"{nb}_ms": ms[nb], "standard_over_bf": ms[nb] / ms[bf]}
            del A, B, C
        out[bf.upper()] = row
    out["paper_table4"] = {"Snapdragon": {"DD": [0.6, 0.7], "TD": [1.2, 1.4], "QD": [2.0, 1.4]},
                           "EPYC": {"DD": [1.0, 0.7], "TD": [1.4, 1.5], "QD": [1.5, 1.9]},
                           "columns": "nonSIMD, SIMD (Strassen GEMM, averaged over n)"}
    return out


def eq1_extra(n):
    """Section 3.1's real GEMM on its own matrices (Eq. 1) at Table 3's n = 2049:
    classical fold and Strassen's recursion (one level: leaves of 1025; two
    levels: leaves of 513), seconds and correct decimal digits against the exact
    product c_ij = sqrt15 * S_i, over every row and the first and last columns."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    from fractions import Fraction

    s15 = inputs.sqrt_fraction(15)
    S = inputs.eq1_row_sums(n)
    out = {"n": n}
    for prec in ("dd", "td", "qd"):
        K = mpg.PRECS[prec][0]
        s5, s3, t, ia, ib = inputs.eq1_factors(n, K)
        r5 = mpg.mul(prec, dev(np.repeat(s5[:, None], 2 * n, 1)), dev(t))
        r3 = mpg.mul(prec, dev(np.repeat(s3[:, None], 2 * n, 1)), dev(t))
        A = r5[:, torch.from_numpy(ia).cuda()].contiguous()
        B = r3[:, torch.from_numpy(ib).cuda()].contiguous()
        del r5, r3
        row = {}
        for name, cut in (("classical", None), ("strassen_1_level", (n + 1) // 2 + 1),
                          ("strassen_2_levels", (n + 3) // 4 + 1)):
            C = mpg.empty(prec, n, n)
            ws = None
            if cut is not None:
                ws = torch.empty(max(mpg.gemm_strassen_workspace(prec, n, n, n, cut), 1), dtype=torch.uint8,
                                 device="cuda")
            run = (lambda: mpg.gemm(prec, A, B, out=C)) if cut is None else \
                (lambda: mpg.gemm_strassen(prec, A, B, cut, out=C, ws=ws))
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            h = C[:, :, [0, n - 1]].cpu().numpy()
            worst = math.inf
            for i in range(n):
                ex = s15 * S[i]
                for c in range(2):
                    got = sum((Fraction(float(v)) for v in h[:, i, c]), Fraction(0))
                    worst = min(worst, -math.log10(float(abs(got - ex) / ex)))
            row[name] = {"s": e0.elapsed_time(e1) / 1e3, "digits": worst,
                         **({"cutoff": cut} if cut is not None else {})}
            del C, ws
        out[prec] = row
        del A, B
    out["paper_section_3_1_digits"] = {"dd": [29.0, 30.4], "td": [45.5, 47.5], "qd": [61.7, 63.5]}
    out["paper_table3_s_n2049"] = {"EPYC 32 threads, block": {"dd": 0.9, "td": 3.4, "qd": 6.2},
                                   "EPYC 1 thread, BF Strassen + AVX2": {"dd": 10.3, "td": 30.4, "qd": 59.9}}
    return out


def dk_instr(prec, degrees, iters, hybrid=False):
    """FP64 instructions of the Durand-Kerner sweeps: per root and sweep, n complex
    Horner steps (4 mul + 3 add) and n - 1 product steps (2 sub + 4 mul + 2 add).
    hybrid=True counts what the hybrid engine issues (TwoSum's error terms on the
    integer pipes), else the paper's all-FP64 sequence."""
    d = degrees.astype(np.float64)
    mu, ad = mul_instr(prec, hybrid), add_instr(prec, hybrid)
    per_root = d * (4 * mu + 3 * ad) + (d - 1) * (4 * mu + 4 * ad)
    return float(np.sum(iters.astype(np.float64) * d * per_root))


def dk_extra(prec="qd", npoly=4096, sweeps=6, loop_polys=16):
    """Batched persistent Durand-Kerner (one CUDA-graph replay: queue reset, degree
    sort, persistent kernel) on the batched-root workload -- 4096 QD polynomials,
    degrees uniform in [10, 500], roots in the unit disk, 1e-30 perturbation, start
    radius 1.1 -- for a fixed number of sweeps, against the per-polynomial launch loop
    on a degree-stratified sample of the same polynomials (same bits)."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    prob = inputs.dk_problem(3, npoly, 10, 500)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    maxdeg = int(prob.degrees.max())
    coef = mpg.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), maxdeg,
                               int(prob.coef_off[-1]))
    off = dev(prob.coef_off)
    g = mpg.RootsGraph(prec, off, coef, maxdeg, radius=1.1, max_iter=sweeps, sort=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r, it, st = g.replay()
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    it, st, r = it.cpu().numpy(), st.cpu().numpy(), r.cpu().numpy()
    instr = dk_instr(prec, prob.degrees, it, hybrid=True)
    instr_paper = dk_instr(prec, prob.degrees, it)
    peak = NOMINAL_FP64_TFLOPS * 1e12 / 2
    res = {"polys": npoly, "degrees": "uniform [10, 500]", "sweeps_cap": sweeps, "batched_graph_s": tb,
           "engine": "hybrid (default)",
           "root_sweeps_per_s": float(np.sum(prob.degrees * it)) / tb,
           "fp64_instr_per_s": instr / tb, "fp64_instr_frac": instr / tb / peak,
           "paper_sequence_equiv_frac": instr_paper / tb / peak,
           "status_counts": np.bincount(st, minlength=5).tolist()}
    # the same replay with every step on the FP64 pipe (opts.engine = 2): same bits
    gh = mpg.RootsGraph(prec, off, coef, maxdeg, radius=1.1, max_iter=sweeps, sort=1, engine=2)
    e0.record()
    rh, ith, _ = gh.replay()
    e1.record()
    torch.cuda.synchronize()
    res["fp64_engine_graph_s"] = e0.elapsed_time(e1) / 1e3
    res["fp64_engine_identical_bits"] = bool(torch.equal(rh.view(torch.int64), g.roots.view(torch.int64)) and
                                               np.array_equal(ith.cpu().numpy(), it))
    del gh
    order = np.argsort(prob.degrees, kind="stable")
    sel = order[np.linspace(0, npoly - 1, loop_polys).astype(int)]
    hc = coef.cpu().numpy()
    so = np.zeros(len(sel) + 1, dtype=np.int64)
    np.cumsum(prob.degrees[sel] + 1, out=so[1:])
    sc = np.concatenate([hc[:, prob.coef_off[b]:prob.coef_off[b + 1]] for b in sel], 1)
    dso, dsc = dev(so), dev(sc)
    md = int(prob.degrees[sel].max())
    mpg.roots(prec, dso, dsc, md, radius=1.1, max_iter=1, mode=1)
    torch.cuda.synchronize()
    e0.record()
    rl, itl, stl = mpg.roots(prec, dso, dsc, md, radius=1.1, max_iter=sweeps, mode=1)
    e1.record()
    torch.cuda.synchronize()
    tl = e0.elapsed_time(e1) / 1e3
    rl = rl.cpu().numpy()
    same = all(np.array_equal(rl[:, so[q] - q:so[q + 1] - q - 1].view(np.uint64),
                              np.ascontiguousarray(r[:, prob.root_off[b]:prob.root_off[b + 1]]).view(np.uint64))
               for q, b in enumerate(sel))
    instr_l = dk_instr(prec, prob.degrees[sel], itl.cpu().numpy(), hybrid=True)
    res["per_poly_loop_sample"] = {
        "polys": len(sel), "degrees": prob.degrees[sel].tolist(), "loop_s": tl,
        "fp64_instr_per_s": instr_l / tl, "identical_bits_to_batched": bool(same),
        "batched_over_loop_throughput": (instr / tb) / (instr_l / tl),
        "loop_s_extrapolated_to_all_polys": tl * instr / instr_l}
    return res


def backward_errors(prec, coef_off, coef, roots, degrees, root_off, coef_off_host):
    """Per polynomial, the largest backward error over its roots,
    |q(z)| / sum_i |c_i| |z|^i: q(z) evaluated by the library's complex Horner
    (K-component arithmetic; its own rounding is at most about (4n + 16) 2^-p of
    the denominator), the denominator in binary64 from leading components."""
    import torch

    import paper_2603_14926_gb300 as mpg

    K = mpg.PRECS[prec][0]
    npoly = len(degrees)
    md = int(degrees.max())
    deg = torch.from_numpy(np.asarray(degrees, dtype=np.int64)).cuda()
    roff = torch.from_numpy(np.asarray(root_off, dtype=np.int64)).cuda()
    j = torch.arange(md, device="cuda")
    valid = j[None, :] < deg[:, None]                                   # (npoly, md)
    src = (roff[:-1, None] + j[None, :]).clamp(max=roots.shape[1] - 1)  # root index per slot
    xr = torch.where(valid[None], roots[:K][:, src], torch.zeros((), dtype=roots.dtype, device="cuda"))
    xi = torch.where(valid[None], roots[K:][:, src], torch.zeros((), dtype=roots.dtype, device="cuda"))
    yr, yi = mpg.polyeval(prec, coef_off, coef, md, xr.reshape(K, -1).contiguous(), xi.reshape(K, -1).contiguous())
    q = torch.hypot(yr[0], yi[0]).reshape(npoly, md)
    az = torch.hypot(xr[0], xi[0])                                      # (npoly, md)
    # sum_i |c_i| |z|^i by Horner on magnitudes, coefficients padded with zeros
    coff = torch.from_numpy(np.asarray(coef_off_host, dtype=np.int64)).cuda()
    den = torch.zeros_like(az)
    for i in range(md, -1, -1):
        idx = (coff[:-1] + i).clamp(max=coef.shape[1] - 1)
        ci = torch.where(deg >= i, coef[0][idx].abs(), torch.zeros((), dtype=coef.dtype, device="cuda"))
        den = den * az + ci[:, None]
    be = torch.where(valid, q / den, torch.zeros((), dtype=q.dtype, device="cuda")).max(dim=1).values
    return be.cpu().numpy()


def roots_full_extra(prec="qd", npoly=4096, max_iter=1000, loop_polys=8, loop_max_sweeps=100, engine=0,
                     eq5_polys=256, eq5_max_degree=200):
    """The batched-root workload solved to the end (4096 QD polynomials, degrees
    uniform in [10, 500], roots in the unit disk, 1e-30 perturbation, start radius
    1.1, at most 1000 sweeps) in one persistent launch: roots/s, statuses, sweeps,
    and each polynomial's backward error against the rounding bound of the
    evaluation; the per-polynomial launch loop (one single-block launch per
    polynomial, each running its whole solve: the same device code, so the same
    bits) on a degree-stratified sample; and a subset solved from Eq. 5's own
    radius beside the radius-1.1 start."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    K = mpg.PRECS[prec][0]
    p_bits = 53 * K
    prob = inputs.dk_problem(3, npoly, 10, 500)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    maxdeg = int(prob.degrees.max())
    coef = mpg.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), maxdeg,
                               int(prob.coef_off[-1]))
    off = dev(prob.coef_off)
    fb0 = mpg.roots_hybrid_fallbacks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    r, it, st = mpg.roots(prec, off, coef, maxdeg, radius=1.1, max_iter=max_iter, sort=1, engine=engine)
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    fallbacks = mpg.roots_hybrid_fallbacks() - fb0
    be = backward_errors(prec, off, coef, r, prob.degrees, prob.root_off, prob.coef_off)
    it, st, rh = it.cpu().numpy(), st.cpu().numpy(), r.cpu().numpy()
    bound = (4.0 * prob.degrees + 16.0) * 2.0 ** -p_bits
    fin = np.isfinite(be)
    lg = lambda v: float(np.log2(v)) if v > 0 else None  # noqa: E731
    roots_total = int(prob.degrees.sum())
    peak = NOMINAL_FP64_TFLOPS * 1e12 / 2
    instr = dk_instr(prec, prob.degrees, it, hybrid=engine != 2)
    out = {"polys": npoly, "degrees": "uniform [10, 500]", "roots": roots_total, "max_sweeps": max_iter,
           "start": "Eq. 5 centre and angles, radius 1.1", "batched_s": tb, "roots_per_s": roots_total / tb,
           "launch": "one persistent launch (queue reset, descending-degree order, persistent kernel)",
           "fp64_instr_frac": instr / tb / peak, "fp64_recomputed_root_updates": int(fallbacks),
           "sweeps_mean": float(it.mean()), "sweeps_max": int(it.max()),
           "status_counts": {"cap": int(np.sum(st == 0)), "converged": int(np.sum(st == 1)),
                             "stagnated": int(np.sum(st == 2)), "breakdown": int(np.sum(st == 4))},
           "backward_error": {
               "definition": "per polynomial, max over its roots of |q(z)| / sum_i |c_i| |z|^i "
                             "(q evaluated in the same K-component arithmetic)",
               "median_log2": lg(np.median(be[fin])) if fin.any() else None,
               "max_log2": lg(be[fin].max()) if fin.any() else None,
               "not_finite": {"polys": int(np.sum(~fin)), "statuses": st[~fin].tolist()[:20]},
               "bound": "(4n + 16) 2^-p, the rounding bound of one K-component Horner evaluation",
               "polys_within_bound": int(np.sum(be <= bound)),
               "by_status": {nm: {"polys": int(np.sum(st == c)),
                                  "median_log2": lg(np.median(be[(st == c) & fin])) if np.any((st == c) & fin)
                                  else None,
                                  "max_log2": lg(be[(st == c) & fin].max()) if np.any((st == c) & fin) else None,
                                  "within_bound": int(np.sum((be <= bound) & (st == c)))}
                             for c, nm in ((0, "cap"), (1, "converged"), (2, "stagnated"))}}}
    # the per-polynomial launch loop on a degree-stratified sample of the polynomials
    # the batched solve finished within loop_max_sweeps sweeps (bounded time)
    cand = np.where(it <= loop_max_sweeps)[0]
    cand = cand[np.argsort(prob.degrees[cand], kind="stable")]
    sel = cand[np.linspace(0, len(cand) - 1, loop_polys).astype(int)]
    hc = coef.cpu().numpy()
    so = np.zeros(len(sel) + 1, dtype=np.int64)
    np.cumsum(prob.degrees[sel] + 1, out=so[1:])
    sc = np.concatenate([hc[:, prob.coef_off[b]:prob.coef_off[b + 1]] for b in sel], 1)
    md = int(prob.degrees[sel].max())
    mpg.roots(prec, dev(so), dev(sc), md, radius=1.1, max_iter=1, mode=1, engine=engine)
    torch.cuda.synchronize()
    e0.record()
    rl, itl, stl = mpg.roots(prec, dev(so), dev(sc), md, radius=1.1, max_iter=max_iter, mode=1, engine=engine)
    e1.record()
    torch.cuda.synchronize()
    tl = e0.elapsed_time(e1) / 1e3
    rl = rl.cpu().numpy()
    same = all(np.array_equal(rl[:, so[q] - q:so[q + 1] - q - 1].view(np.uint64),
                              np.ascontiguousarray(rh[:, prob.root_off[b]:prob.root_off[b + 1]]).view(np.uint64))
               for q, b in enumerate(sel))
    instr_l = dk_instr(prec, prob.degrees[sel], itl.cpu().numpy(), hybrid=engine != 2)
    out["per_poly_loop"] = {
        "form": "one single-block launch per polynomial, each running that polynomial's whole solve "
                "(mp_roots_P mode 1), back to back on one stream",
        "sample": f"{len(sel)} polynomials stratified by degree among the {len(cand)} the batched solve "
                  f"finished within {loop_max_sweeps} sweeps",
        "degrees": prob.degrees[sel].tolist(), "sweeps": itl.cpu().numpy().tolist(), "loop_s": tl,
        "identical_bits_to_batched": bool(same), "roots_per_s": float(prob.degrees[sel].sum()) / tl,
        "batched_over_loop_per_unit_work": (instr / tb) / (instr_l / tl)}
    # the same sample as a host loop of one-sweep launches with a host flag check:
    # per polynomial, launch after launch of one Jacobi sweep (mp_roots_P mode 1,
    # max_iter 1) from the previous launch's iterate, the host reading the status
    # after each; it stops at a converged or broken-down status, or at the sweep
    # count the batched solve took (whose stagnation rule needs the history of
    # delta that one-sweep launches do not keep)
    sweeps_b = it[sel]
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    same_h, launches = True, 0
    for q, b in enumerate(sel):
        n = int(prob.degrees[b])
        oq = dev(np.array([0, n + 1], dtype=np.int64))
        cq = dev(sc[:, so[q]:so[q + 1]])
        z = mpg.roots_init(prec, oq, cq, n, radius=1.1)
        zb = torch.empty_like(z)
        for _ in range(int(sweeps_b[q])):
            zb, _itq, stq = mpg.roots(prec, oq, cq, n, z0=z, max_iter=1, mode=1, engine=engine, out=zb)
            launches += 1
            flag = int(stq.item())  # the host flag check (synchronizes)
            z, zb = zb, z
            if flag in (1, 3):
                break
        same_h &= np.array_equal(z.cpu().numpy().view(np.uint64),
                                 np.ascontiguousarray(rh[:, prob.root_off[b]:prob.root_off[b + 1]]).view(np.uint64))
    th = time.perf_counter() - h0
    out["per_sweep_host_loop"] = {
        "form": "per polynomial, a host loop of one-sweep launches (mp_roots_P mode 1, max_iter 1, z0 = the "
                "previous iterate) with a host read of the status after each, through the Python binding",
        "sample": out["per_poly_loop"]["sample"], "launches": launches, "loop_s": th,
        "identical_bits_to_batched": bool(same_h), "roots_per_s": float(prob.degrees[sel].sum()) / th,
        "batched_over_loop_per_unit_work": (instr / tb) / (instr_l / th)}
    # Eq. 5's own radius against radius 1.1 on a stratified subset of low degree
    small = np.where(prob.degrees <= eq5_max_degree)[0]
    small = small[np.argsort(prob.degrees[small], kind="stable")]
    sub = small[np.linspace(0, len(small) - 1, min(eq5_polys, len(small))).astype(int)]
    so = np.zeros(len(sub) + 1, dtype=np.int64)
    np.cumsum(prob.degrees[sub] + 1, out=so[1:])
    sc = dev(np.concatenate([hc[:, prob.coef_off[b]:prob.coef_off[b + 1]] for b in sub], 1))
    dso = dev(so)
    md = int(prob.degrees[sub].max())
    eq5 = {"polys": len(sub), "degrees": f"stratified over the workload's degrees <= {eq5_max_degree}"}
    for name, rad in (("radius_1.1", 1.1), ("eq5_radius", 0.0)):
        e0.record()
        r5, i5, s5 = mpg.roots(prec, dso, sc, md, radius=rad, max_iter=max_iter, sort=1, engine=engine)
        e1.record()
        torch.cuda.synchronize()
        i5, s5 = i5.cpu().numpy(), s5.cpu().numpy()
        eq5[name] = {"s": e0.elapsed_time(e1) / 1e3, "sweeps_mean": float(i5.mean()), "sweeps_max": int(i5.max()),
                     "status_counts": {"cap": int(np.sum(s5 == 0)), "converged": int(np.sum(s5 == 1)),
                                       "stagnated": int(np.sum(s5 == 2)), "breakdown": int(np.sum(s5 == 4))}}
    out["start_radius_comparison"] = eq5
    return out


def chebyshev_extra(prec="qd", n=64, copies=4096, engine=0):
    """The paper's Durand-Kerner problem (Section 4.2, Eq. 6, n = 64; Table 6): one solve
    on the GPU (latency: one block, and the cluster solve over several SMs;
    `single_solve_gpu_s` is the faster), a batch of `copies` identical problems in
    one persistent launch (throughput); the oracle's single solve is timed in the
    CPU baseline."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    K = mpg.PRECS[prec][0]
    c = inputs.rational_to_mp(inputs.chebyshev_quadrature(n), K)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    off1 = dev(np.array([0, n + 1], dtype=np.int64))
    c1 = dev(c)
    mpg.roots(prec, off1, c1, n)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r, it, st = mpg.roots(prec, off1, c1, n)
    e1.record()
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) / 1e3
    offb = dev(np.arange(0, (n + 1) * (copies + 1), n + 1, dtype=np.int64))
    cb = dev(np.tile(c, copies))
    g = mpg.RootsGraph(prec, offb, cb, n)
    e0.record()
    rb, itb, stb = g.replay()
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    # the cluster solve (mode 2): the same problem over a thread-block cluster of SMs
    mpg.roots(prec, off1, c1, n, mode=2, max_iter=2)
    torch.cuda.synchronize()
    e0.record()
    rc, itc, stc = mpg.roots(prec, off1, c1, n, mode=2)
    e1.record()
    torch.cuda.synchronize()
    tc = e0.elapsed_time(e1) / 1e3
    lanes = 4 if n <= 128 else 2  # lanes per root and CTAs per cluster as the library picks them
    cluster = {"single_solve_gpu_s": tc, "cluster_ctas": max(2, -(-n // (64 // lanes))), "lanes_per_root": lanes,
               "identical_bits": bool(torch.equal(rc.view(torch.int64), r.view(torch.int64)) and
                                      torch.equal(itc, it) and torch.equal(stc, st)),
               "speedup_over_one_block": t1 / tc}
    res = {"n": n, "precision": prec, "sweeps": int(it.cpu()[0]), "status": int(st.cpu()[0]),
           "single_solve_gpu_s": min(t1, tc), "single_solve_one_block_s": t1, "single_solve_cluster": cluster,
           "batch_copies": copies, "batch_s": tb,
           "batch_solves_per_s": copies / tb,
           "batch_fp64_instr_frac": dk_instr(prec, np.full(copies, n), itb.cpu().numpy(), hybrid=engine != 2) /
           tb / (NOMINAL_FP64_TFLOPS * 1e12 / 2),
           "paper_table6_s": {"EPYC BF AVX2": 0.415, "EPYC BF": 0.628, "Snapdragon BF Neon": 0.336,
                              "Snapdragon BF": 0.383}}
    # the other engine on the same problems (same bits)
    other = 2 if engine != 2 else 1
    mpg.roots(prec, off1, c1, n, engine=other)
    torch.cuda.synchronize()
    e0.record()
    r2, _, _ = mpg.roots(prec, off1, c1, n, engine=other)
    e1.record()
    torch.cuda.synchronize()
    t2 = e0.elapsed_time(e1) / 1e3
    g2 = mpg.RootsGraph(prec, offb, cb, n, engine=other)
    e0.record()
    rb2, _, _ = g2.replay()
    e1.record()
    torch.cuda.synchronize()
    res["other_engine"] = {"engine": "FP64 pipe" if other == 2 else "hybrid", "single_solve_gpu_s": t2,
                           "batch_s": e0.elapsed_time(e1) / 1e3,
                           "identical_bits": bool(torch.equal(r2.view(torch.int64), r.view(torch.int64)) and
                                                  torch.equal(rb2.view(torch.int64), rb.view(torch.int64)))}
    return res


def roots_workload(a):
    """The batched-root workload solved to the end: 4096 QD polynomials, degrees
    uniform in [10, 500], roots in the unit disk, 1e-30 perturbation, start radius
    1.1, at most --max-iter sweeps; one CUDA-graph replay (queue reset, descending
    degree order, persistent kernel).  Then the per-polynomial launch loop on a
    degree-stratified sample, to the end as well, with identical bits."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    mpg.load()
    prec = a.prec
    prob = inputs.dk_problem(3, a.npoly, 10, 500)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    maxdeg = int(prob.degrees.max())
    coef = mpg.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), maxdeg,
                               int(prob.coef_off[-1]))
    off = dev(prob.coef_off)
    # constructing the graph runs the solve once outside capture: that run is the warm-up
    g = mpg.RootsGraph(prec, off, coef, maxdeg, radius=1.1, max_iter=a.max_iter, sort=1, engine=a.dk_engine)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record()
        r, it, st = g.replay()
        e1.record()
        torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    it, st, r = it.cpu().numpy(), st.cpu().numpy(), r.cpu().numpy()
    hyb = a.dk_engine != 2
    instr = dk_instr(prec, prob.degrees, it, hybrid=hyb)
    instr_paper = dk_instr(prec, prob.degrees, it)
    order = np.argsort(prob.degrees, kind="stable")
    sel = order[np.linspace(0, a.npoly - 1, a.loop_polys).astype(int)]
    hc = coef.cpu().numpy()
    so = np.zeros(len(sel) + 1, dtype=np.int64)
    np.cumsum(prob.degrees[sel] + 1, out=so[1:])
    sc = np.concatenate([hc[:, prob.coef_off[b]:prob.coef_off[b + 1]] for b in sel], 1)
    md = int(prob.degrees[sel].max())
    e0.record()
    rl, itl, stl = mpg.roots(prec, dev(so), dev(sc), md, radius=1.1, max_iter=a.max_iter, mode=1,
                             engine=a.dk_engine)
    e1.record()
    torch.cuda.synchronize()
    tl = e0.elapsed_time(e1) / 1e3
    rl = rl.cpu().numpy()
    same = all(np.array_equal(rl[:, so[q] - q:so[q + 1] - q - 1].view(np.uint64),
                              np.ascontiguousarray(r[:, prob.root_off[b]:prob.root_off[b + 1]]).view(np.uint64))
               for q, b in enumerate(sel))
    instr_l = dk_instr(prec, prob.degrees[sel], itl.cpu().numpy(), hybrid=hyb)
    roots_total = int(prob.degrees.sum())
    out = {"metric": "batched roots/s", "value": roots_total / tb, "unit": "roots/s",
           "higher_is_better": True, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{a.npoly} {prec.upper()} polynomials, degrees uniform [10, 500], roots "
                                  "in the unit disk, 1e-30 perturbation, start radius 1.1, "
                                  f"<= {a.max_iter} sweeps; one CUDA-graph replay",
                      "engine": "FP64 pipe" if a.dk_engine == 2 else "hybrid (TwoSum error terms on the integer pipes)"},
           "batched_s": tb, "roots": roots_total, "sweeps_mean": float(it.mean()), "sweeps_max": int(it.max()),
           "status_counts": {"cap": int(np.sum(st == 0)), "converged": int(np.sum(st == 1)),
                             "stagnated": int(np.sum(st == 2)), "breakdown": int(np.sum(st == 4))},
           "fp64_instr_per_s": instr / tb, "fp64_instr_frac": instr / tb / (NOMINAL_FP64_TFLOPS * 1e12 / 2),
           "paper_sequence_equiv_frac": instr_paper / tb / (NOMINAL_FP64_TFLOPS * 1e12 / 2),
           "per_poly_loop_sample": {"polys": len(sel), "degrees": prob.degrees[sel].tolist(),
                                    "sweeps": itl.cpu().numpy().tolist(), "loop_s": tl,
                                    "identical_bits_to_batched": bool(same),
                                    "roots_per_s": float(prob.degrees[sel].sum()) / tl,
                                    "batched_over_loop_throughput": (instr / tb) / (instr_l / tl)},
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def profile_one(a):
    """One launch of a kernel family at the given size, for an ncu capture."""
    import torch

    import paper_2603_14926_gb300 as mpg
    from paper_2603_14926_gb300 import inputs

    mpg.load()
    prec = a.prec
    K = mpg.PRECS[prec][0]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    if a.profile == "gemm":
        A, B = make_inputs(prec, a.n, a.seed)
        mpg.gemm(prec, dev(A), dev(B), config=a.gemm_config)
    elif a.profile in ("horner", "estrin", "dcoef"):
        npoly, deg, npts = a.n, 256, 4096
        off = torch.arange(0, (npoly + 1) * (deg + 1), deg + 1, dtype=torch.int64, device="cuda")
        coef = dev(inputs.mp_uniform(4, npoly * (deg + 1), K, stream=inputs.STREAM_C))
        xs = dev(inputs.mp_uniform(5, npoly * npts, K, stream=inputs.STREAM_X))
        if a.profile == "horner":
            mpg.polyeval(prec, off, coef, npts, xs)
        elif a.profile == "estrin":
            mpg.polyeval(prec, off, coef, npts, xs, scheme="estrin")
        else:
            mpg.polyeval_backward(prec, off, coef, npts, xs, xs, want_dx=False)
    elif a.profile == "peak":
        names = {0: "DFMA", 1: "DADD", 2: "DMUL", 3: "FFMA", 4: "FADD", 5: "FFMA2 (f32x2, per lane)",
                 6: "FADD2 (f32x2, per lane)", 7: "LOP3 (integer ALU pipe)", 8: "IMAD (integer, FMA pipe)",
                 9: "IADD3 | LOP3 alternating", 10: "FLO + IADD3 (2 per op)",
                 11: "DFMA, one active lane per warp (= warp instructions)"}
        res = {}
        sms = mpg.lib().mp_sm_count()
        for kind, nm in names.items():
            it = 4096 if kind < 3 or kind == 11 else 131072
            best = 0.0
            for per_sm, thr in ((2, 256), (4, 256), (8, 256), (8, 512)):
                mpg.peak(kind, iters=256, blocks=sms * per_sm, threads=thr)
                rate, _ = mpg.peak(kind, iters=it, blocks=sms * per_sm, threads=thr)
                best = max(best, rate)
            res[nm] = best / 1e9
        per_sm_clk = {k: v * 1e9 / sms / (SM_MAX_MHZ * 1e6) for k, v in res.items()}
        print(json.dumps({"lane_instr_per_s_G": res, "lanes_per_clk_per_sm_at_max_clock": per_sm_clk, "sms": sms}))
        return
    elif a.profile == "dk":
        # mixed degrees 10..500 (the batched-root workload), or one degree for all
        prob = inputs.dk_problem(3, a.n, 10, 500) if a.dk_degree <= 0 else \
            inputs.dk_problem(5, a.n, a.dk_degree, a.dk_degree)
        md = int(prob.degrees.max())
        coef = mpg.poly_from_roots(prec, dev(prob.coef_off), dev(prob.rootdata), dev(prob.delta), md,
                                   int(prob.coef_off[-1]))
        mpg.roots(prec, dev(prob.coef_off), coef, md, radius=1.1, max_iter=2, sort=1, engine=a.dk_engine)
    torch.cuda.synchronize()
    print("ok", a.profile, a.n)


def run_gpu(a, rank, world, pool):
    import torch

    import paper_2603_14926_gb300 as mpg

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    mpg.load()
    prec, n = a.prec, a.n
    A, B = make_inputs(prec, n, a.seed + rank)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = mpg.empty(prec, n, n)
    stream = torch.cuda.current_stream()
    step = lambda: mpg.gemm(prec, dA, dB, out=dC)  # noqa: E731
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        total, per_launch = time_region(step, a.steps, world, stream)
    total = max_over_ranks(total, world)
    ms_step = total / a.steps * 1e3
    value = job_throughput(world, a.steps, 2.0 * n ** 3, total)
    launch_s = statistics.mean(per_launch)
    from paper_2603_14926_gb300.tune import best_gemm_config

    cfg = best_gemm_config(prec, n, n, n)  # -1: the built-in choice, the hybrid engine for binary64
    hybrid = prec in TWO_SUMS and (cfg < 0 or "hybrid" in mpg.gemm_config_name(prec, cfg))
    instr = n ** 3 * (mac_instr_hybrid(prec) if hybrid else mac_instr(prec))
    peak_nominal = NOMINAL_FP64_TFLOPS * 1e12 / 2 / 1e9  # G FP64 instructions/s
    achieved = instr / launch_s / 1e9
    peak_live = fp64_peak_live() / 1e9
    kernel = (f"k_gemm_tma<P_{prec}, HybridEngine<false>, 2, 16, 16, 16, 1, 1> (TMA-staged 16x16 tiles, one output "
              f"per thread; TwoSum error terms on the integer pipes, every other step on the FP64 pipe)" if hybrid else
              f"k_gemm_tma<P_{prec}, NativeEngine<double>, 2, 32, 32, 16, 2, 2> (TMA-staged tiles; FP64 pipe)")
    roofline = {"bound": "alu", "kernel": kernel,
                "achieved": achieved,
                "peak": peak_nominal, "unit": "G FP64 instr/s", "frac": achieved / peak_nominal,
                "peak_source": "nominal 1.25 TFLOP/s FP64 (FMA = 2) -> 625 G FP64 instructions/s "
                               "(152 SMs x 2 lanes/clk x 2.06 GHz)",
                "peak_measured_live": peak_live, "frac_of_measured": achieved / peak_live,
                "fp64_instr_per_mac": mac_instr_hybrid(prec) if hybrid else mac_instr(prec),
                "paper_fp64_instr_per_mac": mac_instr(prec),
                "paper_sequence_equiv_instr_per_s": n ** 3 * mac_instr(prec) / launch_s / 1e9,
                "paper_sequence_equiv_note": "n^3 x the paper's all-FP64 instruction count per multiply-add "
                                             "/ launch time: the rate at which that sequence's results are "
                                             "reproduced; part of it runs on the integer pipes, so this is "
                                             "not a fraction of any one pipe",
                "pipes": gemm_pipes(prec, n, hybrid, launch_s, achieved, peak_nominal, peak_live),
                "algorithmic_instr_per_launch": instr, "launch_ms": launch_s * 1e3,
                "traffic": gemm_traffic(prec, n, hybrid),
                "traffic_source": f"profiles/{gemm_profile_name(prec, n, hybrid)} (ncu dram__bytes_read.sum + "
                                  "dram__bytes_write.sum, one launch of this kernel at this size)",
                "algorithmic_bytes_per_launch": int(3 * A.nbytes)}
    # end to end through the public API with host-resident inputs
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty_like(hA).pin_memory()

    def e2e_step():
        dA.copy_(hA, non_blocking=True)
        dB.copy_(hB, non_blocking=True)
        mpg.gemm(prec, dA, dB, out=dC)
        hC.copy_(dC, non_blocking=True)

    e2e_steps = max(1, min(a.steps, 2))
    e2e_step()
    torch.cuda.synchronize()
    te, _ = time_region(e2e_step, e2e_steps, world, stream)
    te = max_over_ranks(te, world)
    e2e = {"value": job_throughput(world, e2e_steps, 2.0 * n ** 3, te), "unit": "QD ops/s",
           "h2d_bytes_per_step": int(A.nbytes + B.nbytes), "d2h_bytes_per_step": int(A.nbytes),
           "steps": e2e_steps}
    out = {"metric": "QD GEMM ops/s", "value": value, "unit": "QD ops/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded nonoverlapping QD entries)",
           "config": {"workload": f"QD GEMM C := A B, n = {n}, branch-free QD (Algorithms 13/14)",
                      "n": n, "precision": prec, "seed": a.seed,
                      "l2": f"inputs {2 * A.nbytes / 1e6:.0f} MB > 129 MB L2 (no flush needed)",
                      "parallelism": f"replicas x{world}"},
           "roofline": roofline, "e2e": e2e, "gpu_launches": a.steps, "clocks": clk.summary()}
    if rank == 0 and pool is not None:
        out["cpu_baseline"] = cpu_baseline(pool, prec, n, a.seed)
    if rank == 0 and not a.no_extras:
        # each leg on its own: a failing leg is reported and never hides the others
        ex = {}
        legs = (("kernels", lambda: extras(prec, quick=a.quick)),
                ("durand_kerner", lambda: dk_extra(prec, npoly=512 if a.quick else 4096)),
                ("chebyshev_dk", lambda: chebyshev_extra(prec, copies=512 if a.quick else 4096)),
                ("roots_full", lambda: roots_full_extra(prec, npoly=512 if a.quick else 4096)))
        for name, fn in legs:
            try:
                r = fn()
                if name == "kernels":
                    ex.update(r)
                else:
                    ex[name] = r
            except Exception as e:  # noqa: BLE001
                ex[name + "_error"] = repr(e)
        try:
            if pool is not None and "cpu_baseline" in out:
                out["cpu_baseline"]["rows_one_core"] = cpu_baseline_rows(pool, ex)
        except Exception as e:  # noqa: BLE001
            out["cpu_baseline"]["rows_one_core_error"] = repr(e)
        out["extra"] = ex
    return out


def run_reference(a, pool):
    """The CPU oracle on the host cores: each step a row sample of the same GEMM."""
    t0 = time.perf_counter()
    pool.warm(a.prec, a.n, a.seed)
    probe = pool.gemm_rows(a.prec, a.n, a.seed, 1)
    budget = 150.0 / max(1, a.steps + a.warmup)  # whole run within a few minutes
    rows = max(1, int(min(budget, 20.0) / max(probe, 1e-3)))
    for _ in range(a.warmup):
        pool.gemm_rows(a.prec, a.n, a.seed, max(1, rows // 4))
    times = [pool.gemm_rows(a.prec, a.n, a.seed, rows) for _ in range(a.steps)]
    total = sum(times)
    total_rows = rows * pool.cores
    value = a.steps * 2.0 * total_rows * a.n ** 2 / total
    sample = (f"{total_rows} rows of C per step ({rows} per core) of the {a.prec.upper()} GEMM "
              f"n={a.n}, {pool.cores} host cores")
    return {"impl": "reference", "metric": "QD GEMM ops/s", "value": value, "unit": "QD ops/s",
            "n_gpus": 0, "steps": a.steps, "warmup": a.warmup, "ms_per_step": total / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded nonoverlapping QD entries)",
            "config": {"workload": f"QD GEMM C := A B, n = {a.n}, branch-free QD (Algorithms 13/14)",
                       "n": a.n, "precision": a.prec, "seed": a.seed},
            "cpu_baseline": {"value": value, "unit": "QD ops/s", "cores": pool.cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "QD ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--prec", default="qd", choices=["dd", "ddc", "td", "qd", "ds", "tf", "qf"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="smaller extras")
    ap.add_argument("--workload", choices=["gemm", "roots"], default="gemm",
                    help="gemm: the QD GEMM benchmark line (default); roots: the batched-root "
                         "workload solved to the end (a separate, longer measurement)")
    ap.add_argument("--npoly", type=int, default=4096)
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--loop-polys", type=int, default=8)
    ap.add_argument("--gemm-config", type=int, default=None,
                    help="GEMM tile/engine configuration for --profile gemm (default: the built-in choice)")
    ap.add_argument("--dk-engine", type=int, default=0, choices=[0, 1, 2],
                    help="Durand-Kerner engine for --workload roots and --profile dk: 0 automatic (hybrid), "
                         "1 hybrid, 2 FP64 pipe")
    ap.add_argument("--dk-degree", type=int, default=0,
                    help="--profile dk: give every polynomial this degree (0: degrees uniform in [10, 500])")
    ap.add_argument("--profile", choices=["gemm", "horner", "estrin", "dcoef", "dk", "peak"], default=None,
                    help="run one launch of this kernel family at size --n (for ncu) and exit")
    a = ap.parse_args(argv)
    if a.profile:
        profile_one(a)
        return 0
    if a.workload == "roots" and a.impl == "gb300":
        roots_workload(a)
        return 0
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        if rank != 0:
            return 0
        oracle_build()
        pool = OraclePool(cpu_cores())
        try:
            print(json.dumps(run_reference(a, pool)), flush=True)
        finally:
            pool.close()
        return 0
    # the oracle's process pool starts before the first GPU call (spawn)
    pool = None
    if rank == 0 and not a.no_cpu_baseline:
        oracle_build()
        pool = OraclePool(cpu_cores())
    try:
        rank, world = dist_init(a.gpus)
        out = run_gpu(a, rank, world, pool)
        if rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        if pool is not None:
            pool.close()
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
