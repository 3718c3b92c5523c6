#!/usr/bin/env python
"""Benchmark of the image-plane chi^2 path on one GB300 (or N, one process each).

Workload (one step = one chi^2 evaluation of one lens-parameter sample):
  100 PIEMD potentials (centres in a 200" square, e U[0,0.5], r_core
  0.05-1", r_cut 50-200", sigma_v log-U[50,1200] km/s), 2000^2 image-plane
  grid over 200", 20 multiple-image systems (72 observed images, stored in
  tests/golden/obs_c2.json), mixed precision; the FP64 form is timed beside it.

Metric: chi^2 evaluations/s (whole job) and node x potential deflections/s.
Each rank evaluates its own proposals (independent MCMC chains, Sect. 2.2.1):
weak scaling, no collective on the data path.  The batched workload (1024
samples on uneven grids) is sharded over the ranks by work, and its per-sample
chi^2 values are gathered to every rank in sample order afterwards.

Besides the headline line's keys, the line carries the other workloads: the
single-SIS latency case, the 1024-sample batch, the gradient case, the large
case as its full 64-sample batch with chi^2 and gradients, the paper's own
deflection benchmark, the FP64 form against the FP64 pipe, and the oracle's
CPU time for every workload (full or on a stated subset).

--impl reference runs the FP64 CPU oracle on the host cores instead (rank 0),
on a bounded band of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chi² evals/s & node·potential deflections/s, mixed vs FP64 on one GB300"
UNIT = "chi2_evals/s"
WORKLOAD = ("c2: 100 PIEMD, 2000^2 grid over 200\", 20 systems / 72 observed images, "
            "one lens sample per chi^2 evaluation")
SM_PER_GPU_FALLBACK = 152
# Algorithmic work of one PIEMD node x potential evaluation (difference form,
# counted from its formulas on the common path where both special functions
# are their polynomials; the range reductions of a minority of node x
# potentials are not counted): 46 FP32 pipe operations (translate 2, rotate 4,
# squares 2, q^2 x^2 + y^2 1, psi_a^2 and psi_s^2 2, psi_a 1, psi_a + psi_s 1,
# d_x and d_y 2, the two denominators' factors 6 and sums 2, t_x and t_y 4,
# their squares 2, the two polynomials 6 + 4, g 2, rotation back and
# accumulation 4, the bound term P / psi_a 1) and 5 MUFU operations (rsqrt for
# psi_a, sqrt for psi_s, three reciprocals).  At 128 FP32 lanes and 16 MUFU
# lanes per SM per clock the FP32 pipe allows 128 / 46 = 2.78 and the MUFU pipe
# 3.2 node x potential per SM-clock: the FP32 pipe bounds the kernel.
PIEMD_FP32_OPS = 46
PIEMD_MUFU_OPS = 5
FP32_LANES_PER_SM_CLK = 128.0
MUFU_LANES_PER_SM_CLK = 16.0
PIEMD_NODE_POT_PER_SM_CLK = min(FP32_LANES_PER_SM_CLK / PIEMD_FP32_OPS,
                                MUFU_LANES_PER_SM_CLK / PIEMD_MUFU_OPS)
# The plain FP64 form: GB300 runs FP64 at 1/64 of the FP32 rate, 2 FP64
# lanes per SM per clock.  FP64 pipe operations per PIEMD node x potential,
# counted from the formula (52 add/mul/sub, 6 sqrt, 8 div, 2 atan, 2 atanh)
# with each library function's FP64 pipe operations as executed (ncu).
FP64_LANES_PER_SM_CLK = 2.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--clock-warmup", type=float, default=2.0,
                    help="seconds of untimed steps before the warm-up steps")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the HFF deflection and batched measurements")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_obs():
    with open(os.path.join(ROOT, "tests", "golden", "obs_c2.json")) as f:
        return json.load(f)


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts only once the sampler is producing rows
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _code_only(name: str, text: str) -> str:
    """The code of a source file without its comments and blank lines, so that
    an edit to a comment does not change the key of a kernel's profile."""
    if name.endswith(".py"):
        text = re.sub(r"#[^\n]*", "", text)
    else:
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
    lines = (" ".join(ln.split()) for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def source_sha(files) -> str:
    """sha256 over the code of the kernel sources (csrc/ file names)."""
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_1902_03252_gb300", "csrc", name)) as f:
            h.update(_code_only(name, f.read()).encode())
    return h.hexdigest()


# the kernel sources and the build flags (-ftz etc.) they are compiled with
DEFLECT32_SOURCES = ("lt_deflect32.cu", "lt_fp32.cuh", "lt_internal.cuh", "../_build.py")


def traffic_for(kernel: str, files):
    """DRAM traffic per launch recorded in profiles/<kernel>_*.md, if the kernel
    sources have not changed since the capture (else None)."""
    sha = source_sha(files)
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for name in sorted(os.listdir(pdir)):
        if not (name.startswith(kernel) and name.endswith(".md")):
            continue
        with open(os.path.join(pdir, name)) as f:
            txt = f.read()
        for section in txt.split("\n### "):
            m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", section)
            m2 = re.search(r"source_sha256:\s*([0-9a-f]{64})", section)
            if m1 and m2 and m2.group(1) == sha:
                return float(m1.group(1))
    return None


def load_golden(cfg):
    with open(os.path.join(ROOT, "tests", "golden", f"obs_{cfg}.json")) as f:
        return json.load(f)


# ------------------------------------------------------------- CPU baseline
def _oracle_eval_s(oracle, params, grid, obs, threads, rows=None):
    """Seconds of one oracle chi^2 evaluation (deflection on all cores,
    barycentres, triangle search over cell rows on all cores, matching), on
    the whole grid or on its first ``rows`` cell rows."""
    g = grid if rows is None else (grid[0], grid[1], grid[2], grid[3], grid[4], rows + 1)
    t0 = time.perf_counter()
    oracle.chi2(params, g, obs, n_threads=threads, capacity=1 << 18)
    return time.perf_counter() - t0


def cpu_baselines(W):
    """The oracle as it stands, on the host's cores: every workload's chi^2
    evaluations/s, whole evaluations where they take seconds (c1, c2, c4) and
    stated subsets scaled to whole evaluations otherwise (c3: two samples of
    the batch, each in full; c5: a band of cell rows of one sample)."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    out = {}

    def whole(name, w, o):
        dt = _oracle_eval_s(oracle, w.params[0], w.grids[0].as_tuple(), o, threads)
        out[name] = {"value": 1.0 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                     "seconds_per_chi2": dt,
                     "node_pot_per_s": w.grids[0].nodes * w.n_pot / dt,
                     "sample": "one full chi^2 evaluation"}

    whole("c1", W.c1(), load_golden("c1"))
    whole("c2", W.c2(), load_golden("c2"))
    whole("c4", W.c4(), load_golden("c4"))
    w3, o3 = W.c3(), load_golden("c3")
    picks = [0, 1]
    t3 = sum(_oracle_eval_s(oracle, w3.params[b], w3.grids[b].as_tuple(), o3, threads)
             for b in picks)
    nodes3 = sum(w3.grids[b].nodes for b in picks)
    per_node = t3 / nodes3
    batch_s = per_node * sum(g.nodes for g in w3.grids)
    out["c3"] = {"value": w3.batch / batch_s, "unit": UNIT, "cores": threads, "kind": "oracle",
                 "seconds_per_batch": batch_s,
                 "sample": f"samples {picks} of the 1024 in full ({t3:.1f} s), scaled to the "
                           "batch by its node count"}
    w5, o5 = W.c5(batch=1), load_golden("c5")
    g5 = w5.grids[0].as_tuple()
    rows = 60
    t5 = _oracle_eval_s(oracle, w5.params[0], g5, o5, threads, rows=rows)
    full5 = t5 * (g5[5] - 1) / rows
    out["c5"] = {"value": 1.0 / full5, "unit": UNIT, "cores": threads, "kind": "oracle",
                 "seconds_per_chi2": full5,
                 "sample": f"{rows} of {g5[5] - 1} cell rows of one sample ({t5:.1f} s: "
                           "deflection, barycentres and search of that band), scaled to "
                           "the whole grid"}
    return out


# --------------------------------------------------------------- reference
def run_reference(a, rank, world):
    """The FP64 oracle on the host cores, each step a band of grid rows."""
    if rank != 0:
        return
    import oracle
    from paper_1902_03252_gb300 import workloads as W
    oracle.build()
    w = W.c2()
    o = load_obs()
    p = w.params[0]
    g = w.grids[0]
    threads = os.cpu_count() or 1
    bary, _ = oracle.barycentres(p, o)

    def band(rows):
        sub = (g.x0, g.y0, g.dx, g.dy, g.nx, rows + 1)
        t0 = time.perf_counter()
        oracle.find_images(p, sub, bary, o["dls_ds"], n_threads=threads, capacity=1 << 16)
        return time.perf_counter() - t0

    # size the band so that warm-up + steps take about two minutes
    probe_rows = 20
    t_probe = band(probe_rows)
    per_row = t_probe / probe_rows
    budget = 120.0 / max(1, a.steps + a.warmup)
    rows = int(min(g.ny - 1, max(10, budget / per_row)))
    for _ in range(a.warmup):
        band(rows)
    times = [band(rows) for _ in range(a.steps)]
    frac = rows / (g.ny - 1)
    t = statistics.mean(times)
    value = frac / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_of(a, precision="fp64 (oracle)", shape=None),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{rows} of {g.ny - 1} cell rows per step (deflection and "
                                   "triangle search of that band), scaled to whole evaluations"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(a, precision, shape):
    """The workload description shared by both arms' lines."""
    return {"workload": WORKLOAD, "precision": precision,
            "l2": "flushed between timed steps (256 MB write outside the step events)",
            "step": "parameter preparation from device-resident parameters + chi^2",
            "clock_warmup_s": a.clock_warmup, "deflect_shape": shape}


# --------------------------------------------------------------------- ours
def pick_shape(m, lt, torch, grid, obs, dev_params, out, steps=30):
    """The deflection's launch shape, chosen by timing whole evaluations (the
    step the benchmark times) with each shape of the library's table: the
    kernel-only autotuner does not see the barycentre kernels that share the
    SMs at the start of a step.  Untimed setup, before the timed region."""
    best, best_ms = 0, float("inf")
    for v in range(m.num_shapes()):
        m.set_shape(v)
        for _ in range(3):
            m.set_params(dev_params)
            m.chi2(grid, obs, precision=lt.MIXED, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            m.set_params(dev_params)
            m.chi2(grid, obs, precision=lt.MIXED, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if ms < best_ms * 0.997:  # a later shape must be clearly faster
            best, best_ms = v, ms
    m.set_shape(best)
    return best


def run_ours(a, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1902_03252_gb300 import _build, lt, workloads as W

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    w = W.c2()
    params = W.c2_proposal(rank)  # every rank evaluates its own proposal
    o = load_obs()
    grid = [w.grids[0].as_tuple()]
    nodes = w.grids[0].nodes
    node_pot = nodes * w.n_pot
    m = lt.Model(w.n_pot, 1)
    m.set_params(params)
    obs = lt.Observations.from_dict(o, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    dev_params = torch.as_tensor(np.ascontiguousarray(params), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    shape = None if a.no_autotune else pick_shape(m, lt, torch, grid, obs, dev_params, out)

    # correctness of the timed configuration
    m.chi2(grid, obs, precision=lt.MIXED, out=out)
    st, stats = m.sync()
    if st != lt.LT_OK:
        raise RuntimeError(f"lt status {st}")

    def timed(precision, steps, warmup, stages):
        """Device time of each step (CUDA events on the launching stream);
        the library also brackets the given kernel stages with events (each
        pair adds a little time to a step: the throughput steps time only
        the deflection, the kernel of the roofline)."""
        for _ in range(warmup):
            m.set_params(dev_params)
            m.chi2(grid, obs, precision=precision, out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        m.profile(True, stages=stages)
        m.profile_read(reset=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record()
            # one step = the whole path for one proposal: parameter preparation
            # from the device-resident parameters, then the chi^2 evaluation
            m.set_params(dev_params)
            m.chi2(grid, obs, precision=precision, out=out)
            ev[k][1].record()
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        prof = m.profile_read(reset=True)
        m.profile(False)
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        return statistics.mean(ms), ms, prof, wall

    # An idle GPU raises its SM clock over the first seconds of load (measured:
    # a first run at a median 1995 MHz, the next ones at 2070 MHz): untimed
    # steps for a.clock_warmup seconds before the W warm-up steps and the
    # timed region, so that the timed steps see the clock a long run sees.
    t_w = time.perf_counter()
    while time.perf_counter() - t_w < a.clock_warmup:
        for _ in range(20):
            m.set_params(dev_params)
            m.chi2(grid, obs, precision=lt.MIXED, out=out)
        torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms_mixed, ms_list, prof_defl, wall = timed(lt.MIXED, a.steps, a.warmup, ("deflect",))
    clk = clocks.stop()
    st, stats = m.sync()
    ms_mixed = max_over_ranks(ms_mixed)
    value = world * 1000.0 / ms_mixed

    # stage breakdown: stages 0-3 run one after another on the stream, so
    # with k_prep and the counter reset they make up the step; the
    # barycentres run on a side stream under the deflection
    prof_steps = max(1, min(a.steps, 50))
    ms_prof, _, prof, _ = timed(lt.MIXED, prof_steps, 1, lt.PROFILE_KINDS)
    stage_ms = {k: prof[k]["ms"] / prof_steps for k in prof}
    seq = sum(stage_ms[k] for k in ("deflect", "search", "resolve", "chi2"))
    breakdown = {"deflect": stage_ms["deflect"], "search": stage_ms["search"],
                 "fp64_resolve": stage_ms["resolve"], "match_chi2": stage_ms["chi2"],
                 "prep_reset_and_gaps": ms_prof - seq, "step": ms_prof,
                 "barycentres_side_stream_latency": stage_ms["bary"],
                 "note": "the first five add up to the step (the profiled steps carry one "
                         "event pair per stage); the barycentre kernels are issued on a side "
                         "stream at the start of the step and run as the persistent "
                         "deflection's blocks drain, before the search needs them: their "
                         "latency is not part of the step's sum"}
    ms64, _, prof64, _ = timed(lt.FP64, max(1, min(a.steps, a.fp64_steps)), 1, ("deflect",))
    ms64 = max_over_ranks(ms64)
    value64 = world * 1000.0 / ms64

    # end to end through the public API with host buffers: params from pinned
    # host memory in, chi^2 back to pinned host memory, every step; the
    # evaluation is replayed from a CUDA graph (lt_chi2_graph), the call an
    # MCMC loop makes while its grids and observations stay fixed.  Each step
    # is bracketed by CUDA events from the upload to the download, the host
    # waits for the result, and L2 is flushed between steps (outside the
    # brackets), as for the device-timed steps.
    host_params = torch.from_numpy(np.ascontiguousarray(params)).pin_memory()
    host_out = torch.empty(1, dtype=torch.float64).pin_memory()
    for _ in range(a.warmup):
        m.set_params(host_params.numpy())
        m.chi2(grid, obs, precision=lt.MIXED, out=out, graph=True)
        host_out.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]
    for k in range(a.steps):
        flush.zero_()
        ev2[k][0].record()
        m.set_params(host_params.numpy())
        m.chi2(grid, obs, precision=lt.MIXED, out=out, graph=True)
        host_out.copy_(out, non_blocking=True)
        ev2[k][1].record()
        torch.cuda.current_stream().synchronize()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(statistics.mean(b0.elapsed_time(b1) for b0, b1 in ev2))
    st2, _ = m.sync()

    # roofline of the dominant kernel (FP32 deflection): CUDA events around
    # every deflection launch of the timed region
    d = prof_defl["deflect"]
    defl_ms = d["ms"] / max(1, d["launches"])
    achieved = node_pot / (defl_ms * 1e-3) / 1e9  # G node.pot / s
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = sm_count * f_max * PIEMD_NODE_POT_PER_SM_CLK / 1e9
    traffic = traffic_for("k_deflect32", DEFLECT32_SOURCES)
    d64 = prof64["deflect"]
    defl64_ms = d64["ms"] / max(1, d64["launches"])
    fp64_ops = fp64_ops_per_node_pot()
    fp64_roof = None
    if fp64_ops:
        ach64 = node_pot / (defl64_ms * 1e-3) * fp64_ops  # FP64 pipe operations / s
        pk64 = sm_count * f_max * FP64_LANES_PER_SM_CLK
        fp64_roof = {"bound": "fp64", "kernel": "k_deflect64", "kernel_ms": defl64_ms,
                     "fp64_ops_per_node_pot": fp64_ops,
                     "achieved": ach64 / 1e9, "peak": pk64 / 1e9, "unit": "G FP64 ops/s",
                     "frac": ach64 / pk64,
                     "peak_basis": f"{sm_count} SMs x {f_max / 1e6:.0f} MHz x 2 FP64 lanes "
                                   "per SM-clock (1/64 of the FP32 rate)"}
    launches_per_step = sum(prof[k]["launches"] for k in prof) / prof_steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 predicate fallback, f64 chi2)",
        "data": "synthetic",
        "config": config_of(a, precision="mixed", shape=shape),
        "node_pot_per_s": value * node_pot,
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64,
                 "node_pot_per_s": value64 * node_pot,
                 "deflect_kernel_ms": defl64_ms, "roofline": fp64_roof},
        "mixed_over_fp64": value / value64,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gnode_pot/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per "
                                       "launch from the committed ncu capture in profiles/ "
                                       "(used only while the kernel's source hash matches; "
                                       "null otherwise)",
                     "kernel": "k_deflect32", "kernel_ms": defl_ms,
                     "peak_basis": f"{sm_count} SMs x {f_max / 1e6:.0f} MHz (max SM clock) x "
                                   f"{PIEMD_NODE_POT_PER_SM_CLK:.3f} PIEMD node.pot per SM-clock "
                                   f"(FP32 pipe: 128 lanes / {PIEMD_FP32_OPS} ops; the MUFU "
                                   f"pipe allows 16 lanes / {PIEMD_MUFU_OPS} ops)"},
        "kernel_ms_per_step": breakdown,
        "stats": stats,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT,
                "h2d_bytes_per_step": int(host_params.numel() * 8),
                "d2h_bytes_per_step": int(host_out.numel() * 8), "ms_per_step": e2e_ms},
        "clocks": clk,
        # kernels of the chi^2 stages (counted by the library) + k_prep and
        # the counter reset (k_zero64) per step
        "gpu_launches": int(round((launches_per_step + 2) * a.steps)),
        "wall_s_timed_region": wall,
        "deflect32_source_sha256": source_sha(DEFLECT32_SOURCES),
    }
    m.close()
    del flush
    if not a.no_extras:
        # the batch is sharded over the ranks; the other workloads run on rank 0
        line["batched_c3"] = extra_batched(lt, W, torch, dev, peak * 1e9, rank, world,
                                           max_over_ranks, barrier)
        if rank == 0:
            line["latency_c1"] = extra_latency(lt, W, torch, dev)
            line["gradient_c4"] = extra_gradient(lt, W, torch, dev)
            line["large_c5"] = extra_large(lt, W, torch, dev, peak * 1e9)
            line["hff_deflection"] = extra_hff(lt, W, torch, dev)
        barrier()
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baselines(W)
        line["cpu_baseline"] = dict(cb["c2"], sample="one full chi^2 evaluation of the "
                                    "workload (deflection and triangle search on all cores)")
        line["cpu_baseline_all"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def fp64_ops_per_node_pot():
    """FP64 pipe operations of one PIEMD node x potential in the FP64
    deflection, as recorded in the committed ncu capture of k_deflect64
    (profiles/k_deflect64_*.md), or None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for name in sorted(os.listdir(pdir)):
        if name.startswith("k_deflect64") and name.endswith(".md"):
            with open(os.path.join(pdir, name)) as f:
                mm = re.search(r"fp64_ops_per_node_pot:\s*([0-9.eE+]+)", f.read())
            if mm:
                return float(mm.group(1))
    return None


def _time(fn, torch, steps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps / 1e3


def _deflect_rate(m, call, torch, npot):
    """node x potential / s of the FP32 deflection kernel alone inside one
    profiled call (CUDA events around each deflection launch, untimed run)."""
    m.profile(True, stages=["deflect"])
    m.profile_read(reset=True)
    call()
    torch.cuda.synchronize()
    d = m.profile_read(reset=True)["deflect"]
    m.profile(False)
    return npot / (d["ms"] * 1e-3) if d["ms"] > 0 else None


def extra_latency(lt, W, torch, dev, steps=200):
    """The single-SIS case (256^2 nodes): time per chi^2, device-timed and as
    the host sees it (parameters in, chi^2 back, waiting for each result)."""
    w = W.c1()
    o = load_golden("c1")
    grid = [w.grids[0].as_tuple()]
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    obs = lt.Observations.from_dict(o, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    host_out = torch.empty(1, dtype=torch.float64).pin_memory()
    t_dev = _time(lambda: m.chi2(grid, obs, precision=lt.MIXED, out=out), torch, steps)
    t_graph = _time(lambda: m.chi2(grid, obs, precision=lt.MIXED, out=out, graph=True), torch,
                    steps)
    for _ in range(5):
        m.set_params(w.params)
        m.chi2(grid, obs, precision=lt.MIXED, out=out, graph=True)
        host_out.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        m.set_params(w.params)
        m.chi2(grid, obs, precision=lt.MIXED, out=out, graph=True)
        host_out.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    t_host = (time.perf_counter() - t0) / steps
    st, _ = m.sync()
    m.close()
    return {"workload": "c1: one SIS, 256^2 grid over 100\", one system", "status": int(st),
            "ms_per_chi2_device": t_dev * 1e3, "ms_per_chi2_graph": t_graph * 1e3,
            "ms_per_chi2_host_roundtrip": t_host * 1e3,
            "note": "device: back-to-back eager calls; graph: lt_chi2_graph replays; host "
                    "roundtrip: host parameters in, chi^2 out, the host waiting for every "
                    "result (wall clock)"}


def extra_hff(lt, W, torch, dev, steps=3):
    """The paper's benchmark (Sect. 4): deflection of 6730^2 pixels at 0.03"
    by 2 cluster + 700 galaxy SIE, FP32 (with its running bound) and FP64."""
    w = W.hff()
    grid = w.grids[0].as_tuple()
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    shape = m.autotune(grid)
    t32 = _time(lambda: m.deflect_grid(grid, precision=lt.MIXED), torch, steps)
    t_paper = _time(lambda: m.deflect_grid(grid, precision=lt.PAPER), torch, steps)
    st, stats = m.sync()
    t64 = _time(lambda: m.deflect_grid(grid, precision=lt.FP64), torch, 1)
    m.close()
    npot = w.grids[0].nodes * w.n_pot
    return {"workload": "6730^2 pixels at 0.03\", 2 cluster + 700 galaxy SIE (Sect. 4)",
            "node_pot": npot, "fp32_s": t32, "fp64_s": t64, "paper_mixed_s": t_paper,
            "paper_mixed_fp64_nodes": stats["fp64_nodes"], "deflect_shape": shape,
            "fp32_node_pot_per_s": npot / t32, "fp64_node_pot_per_s": npot / t64,
            "paper_s": {"V100": {"dp": 0.46, "mixed": 0.39}, "P100": {"dp": 0.71, "mixed": 0.58},
                        "GTX1080Ti": {"dp": 6.8, "mixed": 1.58}, "Xeon12c": {"dp": 8.1, "mixed": 7.40}},
            "note": "deflection grid only, as timed in the paper; fp32 is the grid with its "
                    "per-node error bound; paper_mixed is the paper's rule (FP32, then FP64 in "
                    "halo patches and where the distortion criteria fire)"}


def extra_batched(lt, W, torch, dev, peak, rank, world, max_over_ranks, barrier, steps=3):
    """1024 perturbed 50-PIEMD samples on grids of 500^2..2000^2, 10 systems,
    one chi^2 per sample, each rank's shard per call through the CUDA-graph
    path; the deflection's launch shape from the library's autotuner on the
    shard's median grid; the per-sample chi^2 gathered in sample order."""
    from paper_1902_03252_gb300 import sharding
    w = W.c3()
    o = load_golden("c3")
    work = [g.nodes * w.n_pot for g in w.grids]
    mine = sharding.shard_for(work, rank, world)
    grids = [w.grids[b].as_tuple() for b in mine]
    m = lt.Model(w.n_pot, len(mine))
    m.set_params(w.params[mine])
    med = sorted(grids, key=lambda g: g[4] * g[5])[len(grids) // 2]
    shape = m.autotune(med)
    obs = lt.Observations.from_dict(o, device=dev)
    out = torch.empty(len(mine), dtype=torch.float64, device=dev)
    m.chi2(grids, obs, precision=lt.MIXED, out=out, graph=True)
    st, stats = m.sync()
    torch.cuda.synchronize()
    barrier()
    t = _time(lambda: m.chi2(grids, obs, precision=lt.MIXED, out=out, graph=True), torch, steps)
    t = max_over_ranks(t)
    chi2 = sharding.gather_in_order(out.cpu().tolist(), mine, w.batch)
    npot = w.node_pot()
    npot_mine = sum(w.grids[b].nodes for b in mine) * w.n_pot
    krate = _deflect_rate(m, lambda: m.chi2(grids, obs, precision=lt.MIXED, out=out), torch,
                          npot_mine)
    m.close()
    return {"workload": "c3: 1024 samples x 50 PIEMD, grids 500^2..2000^2, 10 systems",
            "ranks": world, "samples_per_rank": [len(s) for s in
                                                  sharding.balanced_shards(work, world)],
            "deflect_shape": shape, "s_per_batch": t, "chi2_evals_per_s": w.batch / t,
            "node_pot_per_s": npot / t,
            # the whole batch (search, FP64 resolution, matching included)
            # against the deflection's roofline (per GPU)
            "frac_of_deflection_roofline": npot / t / (peak * world),
            # the deflection kernel alone inside the batch (rank 0's shard), and
            # the whole batch's rate over it: what the other stages cost
            "deflect_kernel_node_pot_per_s": krate,
            "batch_over_deflect_kernel": (npot_mine / (t * 1.0)) / krate if krate else None,
            "chi2_gathered": len(chi2), "chi2_sum": float(sum(chi2)),
            "status": int(st), "stats": stats}


def extra_gradient(lt, W, torch, dev, steps=5):
    """chi^2 with d chi^2/d(x, y, e, phi, r_core, sigma_v) of 100 PIEMD on the
    1000^2 grid with 20 systems, against chi^2 alone, mixed precision."""
    w = W.c4()
    o = load_golden("c4")
    grid = [w.grids[0].as_tuple()]
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    obs = lt.Observations.from_dict(o, device=dev)
    t_val = _time(lambda: m.chi2(grid, obs, precision=lt.MIXED), torch, steps)
    t_grad = _time(lambda: m.chi2_grad(grid, obs, precision=lt.MIXED), torch, steps)
    st, _ = m.sync()
    m.close()
    return {"workload": "c4: 100 PIEMD x 6 parameters, 1000^2 grid, 20 systems",
            "chi2_ms": t_val * 1e3, "chi2_grad_ms": t_grad * 1e3,
            "gradient_overhead": t_grad / t_val - 1.0, "status": int(st)}


def extra_large(lt, W, torch, dev, peak, steps=2):
    """The large workload as stated: a batch of 64 samples of 1000 PIEMD on
    4000^2 grids with 100 systems, chi^2 and gradients in one call (chunked
    by the model's workspace budget), mixed precision."""
    w = W.c5()
    o = load_golden("c5")
    grids = [g.as_tuple() for g in w.grids]
    m = lt.Model(w.n_pot, w.batch, hit_capacity=1 << 16)
    m.set_params(w.params)
    shape = m.autotune(grids[0])
    obs = lt.Observations.from_dict(o, device=dev)
    t_val = _time(lambda: m.chi2(grids, obs, precision=lt.MIXED), torch, steps)
    t_grad = _time(lambda: m.chi2_grad(grids, obs, precision=lt.MIXED), torch, steps)
    st, stats = m.sync()
    npot = w.node_pot()
    krate = _deflect_rate(m, lambda: m.chi2(grids, obs, precision=lt.MIXED), torch, npot)
    m.close()
    return {"workload": "c5: 64 samples x 1000 PIEMD, 4000^2 grids, 100 systems, chi^2 and "
                        "gradients per call", "batch": w.batch,
            "chi2_s_per_batch": t_val, "chi2_grad_s_per_batch": t_grad,
            "chi2_evals_per_s": w.batch / t_val, "chi2_grad_evals_per_s": w.batch / t_grad,
            "deflect_shape": shape, "node_pot_per_s": npot / t_val,
            "frac_of_deflection_roofline": npot / t_val / peak,
            "deflect_kernel_node_pot_per_s": krate,
            "batch_over_deflect_kernel": (npot / t_val) / krate if krate else None,
            "status": int(st), "stats": stats}


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_ours(a, rank, world, local)


if __name__ == "__main__":
    main()
