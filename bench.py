#!/usr/bin/env python
"""Benchmark: seconds for PCG-AMG to reach relative residual 1e-8 on the
256^3 7-point Poisson problem (16.8M rows, 117M nonzeros, FP64 sliced-ELL,
V(1,1) l1-Jacobi, aggregates <= 4, dense Cholesky below 200 rows) on one
GB300, plus the V-cycle's HBM bandwidth.

One step = one pcg_solve from x0 = 0 with the hierarchy resident (the solve
phase the paper times); the hierarchy setup is timed separately (setup_s).
The matrix (1.4 GB) and vectors (134 MB each) exceed the 126 MB L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--side 256] [--precision f64|f32]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Other workloads (--workload): diffusion (256^3, k = exp(g), sigma 2), batch (48
uneven diffusion systems), multi (64 right-hand sides on 128^3 Poisson), and the
paper's own configurations on 200^3 Poisson with b = 1 to 1e-6: paper (VMATCH),
smatch (smoothed prolongators), vbm (Vanek-Mandel-Brezina aggregation).

With N > 1 (torchrun) every rank solves its own replica of the problem: the
path has no exchange step on one node, so there is no collective in it.
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
sys.path.insert(0, ROOT)

METRIC = ("PCG-AMG seconds to 1e-8 rel. residual (256³ Poisson, 1 GB300); "
          "V-cycle HBM GB/s")
SAMPLE_SIDE = 64     # CPU-oracle sample grid
L2_BYTES = 126.5 * 2 ** 20  # GB300 L2 (129 MB)
RHS_SEED = 2
# other workloads (opt-in with --workload): 256^3 diffusion with k = exp(g),
# g a Gaussian field (sigma 2, correlation length 8 cells); 48 diffusion
# systems with sides U{24..96} and sigma U[0.5, 2]
FIELD_ELL = 8.0
DIFF_SIGMA, DIFF_FIELD_SEED, DIFF_RHS_SEED = 2.0, 3, 4
BATCH_SYSTEMS, BATCH_SEED0 = 48, 200
# the paper's own configuration (Sec. 3, VMATCH): 200^3 Poisson (8e6 unknowns),
# b = 1, flexible CG to 1e-6; aggregates <= 8, variable V-cycle from two
# l1-Jacobi sweeps, coarsest level by PCG-l1 (<= 40 iterations); its one-A100
# solve time is the reference number
PAPER_SIDE, PAPER_TOL, PAPER_A100_S = 200, 1e-6, 0.43282
PAPER_OPTS = dict(sweeps=3, smooth_sweeps=2, variable_cycle=1, coarse_solver=1,
                  coarse_maxit=40, coarse_tol=1e-4)
# the paper's SMATCH configuration (Sec. 3): as above with smoothed
# prolongators and four l1-Jacobi sweeps per side on every level (no variable
# cycle); its one-A100 solve time
SMATCH_A100_S = 0.14755
SMATCH_OPTS = dict(sweeps=3, smooth_sweeps=4, variable_cycle=0, coarse_solver=1,
                   coarse_maxit=40, coarse_tol=1e-4, smooth_prolongator=1)
# the paper's VBM configuration (Sec. 3): decoupled Vanek-Mandel-Brezina
# aggregation (strength threshold 0.01; every 7-point coupling is strong),
# smoothed prolongators, V(4,4) l1-Jacobi, PCG-l1 coarsest solve
VBM_A100_S = 0.22308
VBM_OPTS = dict(aggregation=1, vbm_theta=0.01, smooth_sweeps=4, variable_cycle=0,
                coarse_solver=1, coarse_maxit=40, coarse_tol=1e-4, smooth_prolongator=1)
PAPER_LIKE = {"paper": ("vmatch", PAPER_OPTS, PAPER_A100_S, 28),
              "smatch": ("smatch", SMATCH_OPTS, SMATCH_A100_S, 9),
              "vbm": ("vbm", VBM_OPTS, VBM_A100_S, 18)}
METRIC_OF = {
    "diffusion": "PCG-AMG seconds to 1e-8 rel. residual (256³ diffusion, sigma 2, 1 GB300)",
    "batch": "batched PCG-AMG seconds to 1e-8 rel. residual (48 diffusion systems, 1 GB300)",
    "paper": "FCG-AMG (VMATCH) seconds to 1e-6 rel. residual (200³ Poisson, b = 1, 1 GB300)",
    "smatch": "FCG-AMG (SMATCH) seconds to 1e-6 rel. residual (200³ Poisson, b = 1, 1 GB300)",
    "vbm": "FCG-AMG (VBM) seconds to 1e-6 rel. residual (200³ Poisson, b = 1, 1 GB300)",
    "multi": "blocked PCG-AMG seconds to 1e-8 rel. residual for 64 RHS (128³ Poisson, 1 GB300)",
}
MULTI_SIDE, MULTI_RHS, MULTI_SEED0 = 128, 64, 100


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=None, help="grid side (256; 200 for paper)")
    ap.add_argument("--tol", type=float, default=None, help="tolerance (1e-8; 1e-6 for paper)")
    ap.add_argument("--precision", choices=["f64", "f32"], default="f64")
    ap.add_argument("--workload",
                    choices=["poisson", "diffusion", "batch", "paper", "smatch", "vbm", "multi"],
                    default="poisson")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--bf16-from-level", type=int, default=0,
                    help="with --precision f32: BF16 operator values from this level down")
    ap.add_argument("--prolongator-filter", type=float, default=0.0,
                    help="smoothed prolongators: smooth with the filtered matrix (threshold)")
    ap.add_argument("--graph", choices=["loop", "iteration", "none"], default="loop",
                    help="PCG replay: the whole loop as one graph (default), one graph per "
                         "iteration (the host tests after each), or plain launches")
    ap.add_argument("--no-ring", action="store_true",
                    help="per-lane loads instead of the shared-memory ring (stream_ring=0)")
    ap.add_argument("--ring-stages", type=int, default=0,
                    help="stages per warp of the shared-memory ring (2..4; 0: the library's)")
    ap.add_argument("--compress", action="store_true",
                    help="2-byte column offsets in the kernels (compress_columns=1)")
    ap.add_argument("--tail-rows", type=int, default=None,
                    help="levels with at most this many rows run as one persistent launch "
                         "(0 = one launch per step; default: the library's)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32 and FP32+BF16 forms timed beside the FP64 solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    a = ap.parse_args()
    paper = a.workload in PAPER_LIKE
    if a.side is None:
        a.side = PAPER_SIDE if paper else MULTI_SIDE if a.workload == "multi" else 256
    if a.tol is None:
        a.tol = PAPER_TOL if paper else 1e-8
    return a


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks (max-over-ranks timing of replicas):
    an all-reduce of one number on the rank's device (NCCL) or on the host
    (gloo); `value` itself with one rank."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    dev = device if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax = max(smax, float(p[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle

def _oracle_iterations(side):
    path = os.path.join(ROOT, "tests", "golden", "oracle_poisson%d.json" % side)
    try:
        with open(path) as f:
            return json.load(f)["iterations"]
    except Exception:
        return None


def _oracle_full_run(side):
    """The oracle's one measured single-thread run of the full problem (setup
    and solve seconds, host CPU), as recorded with its stored results."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_poisson%d.json" % side)
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    return {"setup_s": d.get("oracle_setup_s"), "solve_s": d.get("oracle_solve_s"),
            "threads": d.get("oracle_threads"), "host": d.get("oracle_host")}


def oracle_sample(min_seconds=10.0, repeats=None, tol=1e-8):
    """Times the CPU oracle's PCG-AMG solve on the SAMPLE_SIDE^3 problem."""
    import oracle
    from synthetic import poisson3d, uniform01

    A = poisson3d(SAMPLE_SIDE)
    b = uniform01(RHS_SEED, SAMPLE_SIDE ** 3)
    H = oracle.Hierarchy(A)
    times, its = [], None
    t_all = time.perf_counter()
    k = 0
    while True:
        t0 = time.perf_counter()
        _, info = oracle.pcg(A, b, tol=tol, hier=H)
        times.append(time.perf_counter() - t0)
        its = info["iterations"]
        k += 1
        if repeats is not None and k >= repeats:
            break
        if repeats is None and time.perf_counter() - t_all >= min_seconds:
            break
    return times, its


def scale_to_full(t_sample, it_sample, side):
    """Per unknown-iteration scaling of a sample solve time to side^3."""
    it_full = _oracle_iterations(side)
    factor = (side / SAMPLE_SIDE) ** 3 * ((it_full / it_sample) if it_full else 1.0)
    return t_sample * factor, it_full


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W, K = a.warmup, a.steps
    times, its = oracle_sample(repeats=W + K, tol=a.tol)
    timed = times[W:]
    per = sum(timed) / len(timed)
    val, it_full = scale_to_full(per, its, a.side)
    sample = ("oracle FP64 PCG-AMG solve of %d^3 Poisson (same generator, RHS seed %d) to %g: "
              "%.3f s, %d iterations; scaled by unknowns x iterations to %d^3 (%s iterations, "
              "the oracle's own count)" % (SAMPLE_SIDE, RHS_SEED, a.tol, per, its, a.side,
                                           it_full))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s",
            "n_gpus": a.gpus, "steps": K, "warmup": W, "ms_per_step": per * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "poisson3d_%d^3_pcg_amg_v11_tol%g" % (a.side, a.tol),
                       "sample_side": SAMPLE_SIDE},
            "cpu_baseline": {"value": val, "unit": "s", "cores": 1, "kind": "oracle",
                             "extrapolated": True,
                             "measured_full_run": _oracle_full_run(a.side),
                             "sample": sample},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def _traffic_from_profiles(kernel_key, workload):
    """traffic_bytes_per_launch recorded from an ncu capture of this kernel."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, fn)) as f:
            for ln in f:
                p = ln.split()
                if len(p) == 4 and p[0] == "traffic_bytes_per_launch" and p[1] == kernel_key \
                        and p[2] == workload:
                    return float(p[3])
    return None


def _oracle_fixture(a):
    """The oracle's stored run of this exact problem, or None."""
    if a.workload != "poisson":
        return None
    path = os.path.join(ROOT, "tests", "golden", "oracle_poisson%d.json" % a.side)
    try:
        with open(path) as f:
            fx = json.load(f)
    except Exception:
        return None
    return fx if fx.get("seed") == RHS_SEED and fx.get("tol") == a.tol else None


def oracle_x_error(a, x):
    """max |x - x_oracle| / max |x_oracle| over the oracle's sampled rows."""
    import torch

    fx = _oracle_fixture(a)
    if fx is None or "x_rows" not in fx:
        return None
    rows = torch.as_tensor(fx["x_rows"], dtype=torch.int64, device=x.device)
    xs = x[rows].double().cpu()
    xo = torch.as_tensor(fx["x_values"], dtype=torch.float64)
    return float((xs - xo).abs().max() / xo.abs().max())


def full_size_parity(a, H, levels, oc, info, x):
    """The FP64 GPU solve against the oracle's stored run of the same problem
    (tests/golden/oracle_poisson<side>.json): levels, entries per level,
    operator complexity, iterations (+-1) and sampled solution entries.
    None when no stored run matches this workload (or another precision)."""
    fx = _oracle_fixture(a)
    if fx is None or a.precision != "f64" or any(
            getattr(H.opts, k, d) != d for k, d in (("sweeps", 2), ("max_coarse", 200))):
        return None
    lv_ok = [tuple(lv) for lv in levels] == [(v["n"], v["nnz"]) for v in fx["levels"]]
    it_ok = abs(info["iterations"] - fx["iterations"]) <= 1
    oc_ok = abs(oc - fx["operator_complexity"]) <= 1e-12
    xerr = oracle_x_error(a, x)
    x_ok = xerr is None or xerr <= 1e-10
    return {"oracle_iterations": fx["iterations"], "iterations": info["iterations"],
            "levels_match": lv_ok, "operator_complexity_match": oc_ok,
            "x_err_vs_oracle": xerr, "ok": bool(lv_ok and it_ok and oc_ok and x_ok),
            "source": "tests/golden/oracle_poisson%d.json" % a.side}


# GB300's FP64 pipe: 1.25 TFLOP/s nominal = 2 FP64 FMA instructions per SM
# per clock (152 SMs at 2.07 GHz); every FP64 add, multiply or FMA takes one
FP64_OPS_PER_SM_CLOCK = 2.0
SM_COUNT, SM_MAX_GHZ = 152, 2.07


def fp64_pipe(H, level, kind, ms, a):
    """FP64 instructions of one pre- or post-smoother launch of an FP64
    hierarchy against the FP64 pipe's peak: one FMA per stored entry; the
    pre-smoother's r = b - (A S) b runs from b_i down by negated FMAs (nothing
    more a row), the post-smoother adds b_i + r_i and ends with
    z = s_i acc + x_c (two a row), and on level 0 forms (r, z) for PCG's beta
    (one FMA a row more).  Those kernels are co-limited by HBM and by GB300's
    reduced-rate FP64 arithmetic."""
    if a.precision != "f64" or kind not in ("pre", "post"):
        return None
    n = H.level_info(level)[0]
    slots = H.level_layout(level, ap=(kind == "post"))["slots"]
    per_row = 0 if kind == "pre" else (3 if level == 0 else 2)
    ops = slots + per_row * n
    peak = FP64_OPS_PER_SM_CLOCK * SM_COUNT * SM_MAX_GHZ * 1e9
    rate = ops / (ms * 1e-3)
    return {"ops_per_launch": ops, "ops_per_s": rate, "peak_ops_per_s": peak,
            "frac": rate / peak,
            "peak_source": "nominal 1.25 TFLOP/s FP64 = 2 FMA per SM per clock at 2.07 GHz"}


def run_ours(a):
    import numpy as np
    import torch

    import paper_2406_19754_gb300 as amg
    from synthetic import poisson3d, uniform01

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    side = a.side
    batch = a.workload == "batch"
    if batch:
        from synthetic import batch_specs, diffusion_problem

        specs = batch_specs(BATCH_SYSTEMS, BATCH_SEED0)
        systems = [diffusion_problem(sd, sg, FIELD_ELL, seed) for sd, sg, seed in specs]
        n = sum(len(S[0]) - 1 for S in systems)
        nnz = sum(int(S[0][-1]) for S in systems)
        b_host = uniform01(RHS_SEED, n)
        Ad = [amg.csr_to_device(S, dev) for S in systems]
        workload = ("batch%d_diffusion_sides%d-%d_pcg_amg_v11_tol%g"
                    % (BATCH_SYSTEMS, min(s[0] for s in specs), max(s[0] for s in specs), a.tol))
        del systems
    else:
        n = side ** 3
        if a.workload == "diffusion":
            from synthetic import diffusion_problem

            A = diffusion_problem(side, DIFF_SIGMA, FIELD_ELL, DIFF_FIELD_SEED)
            b_host = uniform01(DIFF_RHS_SEED, n)
            workload = "diffusion3d_%d^3_sigma%g_ell%g_pcg_amg_v11_tol%g" % (
                side, DIFF_SIGMA, FIELD_ELL, a.tol)
        elif a.workload in PAPER_LIKE:
            A = poisson3d(side)
            b_host = np.ones(n)
            workload = "poisson3d_%d^3_fcg_%s_tol%g" % (side, PAPER_LIKE[a.workload][0], a.tol)
        elif a.workload == "multi":
            A = poisson3d(side)
            b_host = np.ascontiguousarray(np.stack(
                [uniform01(MULTI_SEED0 + c, n) for c in range(MULTI_RHS)], axis=1))
            workload = "poisson3d_%d^3_x%d_rhs_pcg_amg_v11_tol%g" % (side, MULTI_RHS, a.tol)
        else:
            A = poisson3d(side)
            b_host = uniform01(RHS_SEED, n)
            workload = "poisson3d_%d^3_pcg_amg_v11_tol%g" % (side, a.tol)
        nnz = int(A[0][-1])
        Ad = amg.csr_to_device(A, dev)
        del A
    b = torch.as_tensor(b_host, device=dev)
    x = torch.zeros_like(b)

    tail = {} if a.tail_rows is None else {"tail_rows": a.tail_rows}
    if a.compress:
        tail["compress_columns"] = 1
    if a.no_ring:
        tail["stream_ring"] = 0
    elif a.ring_stages:
        tail["stream_ring"] = a.ring_stages
    if a.workload in PAPER_LIKE:
        tail.update(PAPER_LIKE[a.workload][1])
    if a.bf16_from_level:
        tail["bf16_from_level"] = a.bf16_from_level
    if a.prolongator_filter:
        tail["prolongator_filter"] = a.prolongator_filter
    beta = "flexible" if a.workload in PAPER_LIKE else "auto"

    def make_hierarchy():
        if batch:
            return amg.BatchHierarchy(Ad, precision=a.precision, autotune=int(a.autotune),
                                      **tail)
        return amg.Hierarchy(*Ad, precision=a.precision, autotune=int(a.autotune), **tail)

    multi = a.workload == "multi"

    def solve(bv, xv, hier=None):
        H_ = hier if hier is not None else H
        if multi:
            _, stats = H_.pcg_multi(bv, xv, tol=a.tol)
            worst = min(s["status"] for s in stats) if any(s["status"] < 0 for s in stats) \
                else max(s["status"] for s in stats)
            return dict(iterations=max(s["iterations"] for s in stats), status=worst,
                        per_rhs=[s["iterations"] for s in stats])
        if batch:
            _, stats = H_.pcg(bv, xv, tol=a.tol, use_graph=GRAPH_MODE[a.graph])
            worst = min(s["status"] for s in stats) if any(s["status"] < 0 for s in stats) \
                else max(s["status"] for s in stats)
            return dict(iterations=max(s["iterations"] for s in stats), status=worst,
                        per_system=[s["iterations"] for s in stats])
        return H_.pcg(bv, xv, tol=a.tol, beta_form=beta, use_graph=GRAPH_MODE[a.graph])[1]

    # warm the module on a small problem, then time the setup of the real one
    amg.Hierarchy(*amg.csr_to_device(poisson3d(16), dev), precision=a.precision).close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = make_hierarchy()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    nl = H.levels
    levels = [H.level_info(l) for l in range(nl)]
    oc = H.operator_complexity()

    for _ in range(a.warmup):
        x.zero_()
        info = solve(b, x)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    iters = []
    for _ in range(a.steps):
        x.zero_()
        info = solve(b, x)
        iters.append(info["iterations"])
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dev)
    per_solve = elapsed / a.steps
    it = iters[-1]
    assert info["status"] == 0, info
    x_ref = x.clone() if not (batch or multi) else None
    parity = full_size_parity(a, H, levels, oc, info, x_ref) if not (batch or multi) else None

    # the blocked V-cycle of all right-hand sides against one column at a time
    mvc = None
    if multi:
        b = b.contiguous()
        Zm = torch.empty_like(b)
        for _ in range(3):
            H.vcycle_multi(b, Zm)
        e0m, e1m = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0m.record()
        for _ in range(5):
            H.vcycle_multi(b, Zm)
        e1m.record()
        torch.cuda.synchronize()
        mvc = e0m.elapsed_time(e1m) / 5
        b_multi, b = b, b[:, 0].contiguous()

    # per-kernel V-cycle timing (CUDA events on the launching stream)
    agg = {}
    for _ in range(3):
        H.vcycle_profile(b)
    reps = 5
    _, recs = H.vcycle_profile(b)

    # our kernel launches per solve (see pcg.cu, batch.cu, vcycle.cu, tail.cu):
    # one per V-cycle profile record, plus the second phase of a coarse solve
    # over a block larger than 1024 rows, the level-0 dot kernel of a
    # one-level hierarchy, and the separate dot kernel of V-cycles with
    # several sweeps or smoothed prolongators
    V = len(recs)
    if any(r_["kind"] == "coarse" for r_ in recs) and H.level_info(nl - 1)[0] > 1024:
        V += 1
    if nl == 1 or (not batch and (H.opts.smooth_sweeps > 1 or H.opts.smooth_prolongator)):
        V += 1
    if batch:
        launches = (2 + (V + 5) + (it - 1) * (V + 6) + 2) * a.steps
    elif multi:
        launches = None  # the blocked kernels (multi.cu) are not counted here
    else:
        # initial residual, first iteration (V-cycle, SpMV, update), the others
        # (+ p update), the owed x update, and the loop graph's stopping tests
        ctl = it if a.graph == "loop" else 0
        launches = (1 + (V + 2) + (it - 1) * (V + 3) + 1 + ctl) * a.steps
    nlaunch = {}  # launches per V-cycle of each (level, kind)
    for _ in range(reps):
        _, recs = H.vcycle_profile(b)
        for r_ in recs:
            key = (r_["level"], r_["kind"])
            e = agg.setdefault(key, [0.0, 0.0])
            e[0] += r_["ms"] / reps
            e[1] += r_["bytes"] / reps
    for r_ in recs:
        key = (r_["level"], r_["kind"])
        nlaunch[key] = nlaunch.get(key, 0) + 1
    vc_ms = sum(v[0] for v in agg.values())
    vc_bytes = sum(v[1] for v in agg.values())
    vcycle_gbs = vc_bytes / (vc_ms * 1e-3) / 1e9
    # the dominant kernel: most V-cycle time among the kernels whose bytes per
    # launch exceed the L2 (the HBM roofline means nothing for levels that live
    # in L2: those are latency bound); all kernels when none is that large
    big = {k: v for k, v in agg.items() if v[1] / nlaunch[k] > L2_BYTES}
    (dl, dk), (dms, dbytes) = max((big or agg).items(), key=lambda kv: kv[1][0])
    dms, dbytes = dms / nlaunch[(dl, dk)], dbytes / nlaunch[(dl, dk)]  # per launch
    peak, peak_src = _peaks()
    dom_name = "vcycle_%s_level%d" % (dk, dl)
    wl_key = "%s%d_%s" % (a.workload, side, a.precision)
    roof = {"bound": "hbm", "kernel": dom_name, "achieved": dbytes / (dms * 1e-3) / 1e9,
            "peak": peak, "unit": "GB/s", "frac": dbytes / (dms * 1e-3) / 1e9 / peak,
            "peak_source": peak_src,
            "traffic": _traffic_from_profiles(dom_name, wl_key),
            "bytes_per_launch": dbytes, "ms_per_launch": dms,
            "selection": "most V-cycle time among kernels moving more than the L2 "
                         "(%.0f MB) per launch" % (L2_BYTES / 1e6)}
    if multi:
        roof["scope"] = "the single-column V-cycle of the same hierarchy"
    fp64 = fp64_pipe(H, dl, dk, dms, a)
    if fp64:
        roof["fp64_pipe"] = fp64

    # SpMV (PCG operator) timed alone
    y = torch.empty_like(b)
    for _ in range(3):
        H.spmv(b, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        H.spmv(b, y)
    e1.record(stream)
    torch.cuda.synchronize()
    spmv_ms = e0.elapsed_time(e1) / 10
    lay = H.level_layout(0)
    idx_bytes = 2.0 + 4.0 / lay["slice_height"] if lay["compressed"] else 4.0
    spmv_gbs = ((8.0 + idx_bytes) * nnz + 16.0 * n) / (spmv_ms * 1e-3) / 1e9

    # end to end through the public API from pinned host memory
    e2e = None
    if not a.no_e2e:
        bfull = b_multi if multi else b
        bh = torch.from_numpy(b_host).pin_memory()
        xh = torch.empty(tuple(bfull.shape), dtype=torch.float64).pin_memory()
        bd = torch.empty_like(bfull)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            bd.copy_(bh, non_blocking=True)
            x.zero_()
            solve(bd, x)
            xh.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_s = e0.elapsed_time(e1) / 1e3 / a.steps
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * bfull.numel(),
               "d2h_bytes_per_step": 8 * bfull.numel()}
        assert np.allclose(xh[:8].numpy(), x[:8].cpu().numpy())

    # the mixed-precision forms of the same solve (FP64 outer PCG): time to
    # tolerance, iterations, true residual and distance to the FP64 solution
    forms = None
    if not a.no_forms and a.workload in ("poisson", "diffusion") and a.precision == "f64":
        forms = {"f64": {"time_to_tol_s": per_solve, "iterations": it,
                         "true_relres": info["true_relres"], "setup_s": setup_s}}
        if parity and parity.get("x_err_vs_oracle") is not None:
            forms["f64"]["x_err_vs_oracle"] = parity["x_err_vs_oracle"]
        for name, kw in (("f32", {}), ("f32_bf16_from_level2", {"bf16_from_level": 2})):
            opts = dict(tail)
            opts.update(kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Hf = amg.Hierarchy(*Ad, precision="f32", autotune=int(a.autotune), **opts)
            torch.cuda.synchronize()
            fsetup = time.perf_counter() - t0
            for _ in range(a.warmup):
                x.zero_()
                finfo = solve(b, x, Hf)
            ev0.record(stream)
            for _ in range(a.steps):
                x.zero_()
                finfo = solve(b, x, Hf)
            ev1.record(stream)
            torch.cuda.synchronize()
            fper = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dev) / a.steps
            assert finfo["status"] == 0, (name, finfo)
            d = {"time_to_tol_s": fper, "iterations": finfo["iterations"],
                 "true_relres": finfo["true_relres"], "setup_s": fsetup,
                 "x_err_vs_f64": float(torch.linalg.vector_norm(x - x_ref)
                                       / torch.linalg.vector_norm(x_ref)),
                 "time_cut_vs_f64": 1.0 - fper / per_solve}
            ox = oracle_x_error(a, x)
            if ox is not None:
                d["x_err_vs_oracle"] = ox
            forms[name] = d
            Hf.close()

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline and a.workload == "poisson":
        times, its_s = oracle_sample(min_seconds=10.0, tol=a.tol)
        per = sum(times) / len(times)
        val, it_full = scale_to_full(per, its_s, side)
        cpu = {"value": val, "unit": "s", "cores": 1, "kind": "oracle",
               "extrapolated": True, "measured_full_run": _oracle_full_run(side),
               "sample": ("oracle FP64 PCG-AMG solve of %d^3 Poisson (same generator, RHS seed "
                          "%d) to %g, %d runs of %.3f s, %d iterations; scaled by unknowns x "
                          "iterations to %d^3 (%s iterations, the oracle's own count)"
                          % (SAMPLE_SIDE, RHS_SEED, a.tol, len(times), per, its_s, side,
                             it_full))}

    if rank == 0:
        line = {
            "metric": METRIC_OF.get(a.workload, METRIC), "value": per_solve, "unit": "s",
            "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "f64"
            else "f64 outer / f32 V-cycle", "data": "synthetic",
            "config": {"workload": workload, "n": n, "nnz": nnz, "levels": nl,
                       "level_rows": [lv[0] for lv in levels],
                       "operator_complexity": round(oc, 4), "iterations": it,
                       "precision": a.precision, "autotune": bool(a.autotune),
                       "bf16_from_level": a.bf16_from_level,
                       "prolongator_filter": a.prolongator_filter,
                       "tail_rows": int(H.opts.tail_rows),
                       "level0_layout": lay,
                       "level_layouts": [[H.level_layout(l)["slice_height"],
                                          H.level_layout(l)["threads_per_row"]]
                                         for l in range(nl)],
                       "pcg_graph": a.graph,
                       "stream_ring": int(H.opts.stream_ring),
                       "level0_ap_layout": H.level_layout(0, ap=True) if nl > 1 else None,
                       "rhs": "uniform[0,1) seed %d" % RHS_SEED,
                       "l2": "inputs larger than L2 (matrix %.2f GB)" % (12.0 * nnz / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "setup_s": setup_s, "iterations": it, "vcycle_gbs": vcycle_gbs,
            "vcycle_ms": vc_ms, "spmv_gbs": spmv_gbs, "spmv_ms": spmv_ms,
            "ms_per_iteration": per_solve * 1e3 / max(it, 1),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "parity": parity, "precision_forms": forms,
            "clocks": clk,
            "vcycle_kernels": [{"level": k[0], "kind": k[1], "launches": nlaunch[k],
                                "ms": round(v[0], 5),
                                "gbs": round(v[1] / (v[0] * 1e-3) / 1e9, 1)}
                               for k, v in sorted(agg.items())],
        }
        if ws > 1:
            line["solves_per_s"] = ws * a.steps / elapsed
        if batch:
            line["systems_per_s"] = ws * BATCH_SYSTEMS * a.steps / elapsed
            line["config"]["per_system_iterations"] = info["per_system"]
            line["config"]["rhs"] = "uniform[0,1) seed %d, concatenated" % RHS_SEED
        if a.workload == "diffusion":
            line["config"]["rhs"] = "uniform[0,1) seed %d" % DIFF_RHS_SEED
        if multi:
            line["config"]["rhs"] = ("%d columns uniform[0,1) seeds %d..%d, row-major"
                                     % (MULTI_RHS, MULTI_SEED0, MULTI_SEED0 + MULTI_RHS - 1))
            line["config"]["per_rhs_iterations"] = info["per_rhs"]
            # one V-cycle of all columns (blocked SpMM kernels) against the
            # single-vector V-cycle times the number of columns
            line["multi"] = {"vcycle_all_rhs_ms": mvc, "vcycle_one_rhs_ms": vc_ms,
                             "blocked_speedup_per_rhs": vc_ms * MULTI_RHS / mvc,
                             "rhs_iterations_per_s": sum(info["per_rhs"]) / per_solve}
        if a.workload == "paper":
            line["config"]["rhs"] = "b = 1"
            line["config"]["cycle"] = ("aggregates <= 8 (3 matching sweeps), variable V-cycle "
                                       "(2 l1-Jacobi sweeps on level 0, doubled per level), "
                                       "coarsest: PCG-l1 <= 40 iterations to 1e-4, FCG")
            if side == PAPER_SIDE and a.tol == PAPER_TOL and ws == 1:
                # the paper's VMATCH solve time on one A100 (8e6 unknowns, 1e-6)
                line["vs_baseline"] = per_solve / PAPER_A100_S
                line["baseline"] = {"value": PAPER_A100_S, "unit": "s", "hardware": "1 A100",
                                    "iterations": 28}
        if a.workload in ("smatch", "vbm"):
            line["config"]["rhs"] = "b = 1"
            line["config"]["cycle"] = (
                ("aggregates <= 8 (3 matching sweeps)" if a.workload == "smatch" else
                 "decoupled Vanek-Mandel-Brezina aggregation, theta 0.01") +
                ", smoothed prolongators, V(4,4) l1-Jacobi on every level, "
                "coarsest: PCG-l1 <= 40 iterations to 1e-4, FCG")
            if side == PAPER_SIDE and a.tol == PAPER_TOL and ws == 1:
                # the paper's solve time for this configuration on one A100
                _, _, ref_s, ref_it = PAPER_LIKE[a.workload]
                line["vs_baseline"] = per_solve / ref_s
                line["baseline"] = {"value": ref_s, "unit": "s", "hardware": "1 A100",
                                    "iterations": ref_it}
        print(json.dumps(line), flush=True)
    H.close()
    if parity is not None and not parity["ok"]:
        print("bench: the solve does not match the oracle's run of this problem: %s"
              % json.dumps(parity), file=sys.stderr, flush=True)
        sys.exit(1)
    if ws > 1:
        torch.distributed.destroy_process_group()


GRAPH_MODE = {"loop": 1, "iteration": 2, "none": 0}


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
