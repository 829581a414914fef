"""Benchmark of the sliced big-head contraction on one GB300 (or N, one process
per GPU under torchrun).

Default workload: the 53-qubit Sycamore-shaped lattice (6 x 9 rotated grid,
one site removed), 14 cycles, 16 open qubits, the other 37 fixed to a seeded
bitstring, intermediates capped at 2^30 elements by slicing, contracted with
the stored tree of paper_2103_03074_gb300/trees/syc53_m14.json (256
hierarchical-bipartition trials of seed 5, ranked by roofline time: the
fastest of eight searched trees on the GPU; it needs no slicing under the
cap).  One step = every slice of that tree contracted and summed into the
FP64 amplitude tensor (the whole 2^16-entry tensor), then the FP64
probability / XEB reduction.  The
error of every form is measured on the FP64 oracle's sampled entries of the
same tensor (tests/golden/cfg4_amplitudes_sampled.txt).  The line also
carries a short measurement of the 20-cycle, 21-open-qubit workload (cap
2^31): the split form against plain FP32 on the same slices.

Metric: slices/s (and complex TFLOP/s = 8 x complex MACs / s).
  value     device time (CUDA events on the launching stream), L2 flushed
            between steps outside the timed events; the fastest form that
            keeps 22+ significant bits per operand (FP32, TF32x3, FP16X3) and
            measures within 1e-5 of the oracle.
  e2e       the same through tn_contract_slices_host with host buffers: every
            step copies the leaf values in, contracts, reduces the
            probabilities and copies the amplitudes out (pinned memory).
  roofline  of the dominant kernel class, from the step-timing recorder's
            CUDA events in a separate pass of the same step.
  cpu_baseline  the CPU FP64 oracle on a bounded sample of the same
            workload, on all host cores and on one.

--impl reference times the CPU FP64 oracle as the reference arm (no product
code is loaded: the slice count comes from the stored tree's JSON file).
--workload gemm times one batched complex GEMM step of a given shape (the
tensor-core kernel in isolation, e.g. for ncu).
Multi-GPU (torchrun): each rank contracts its own seeded instance (weak
scaling, no collective on the data path); time = max over ranks.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TREES = os.path.join(ROOT, "paper_2103_03074_gb300", "trees")
SMS = 152
FP32_LANES_PER_SM = 128
METRIC = "slices/s & complex TFLOP/s per GB300 at <=1e-5 amp err, split-TC vs plain FP32"
DEFAULT_WORKLOAD = "syc53_m14"

# DRAM traffic per tensor-core GEMM launch of the default step, by form, from
# the one-pass ncu capture summarised in profiles/launches_syc53_m14_fp16x3.md
# (dram__bytes_read.sum + dram__bytes_write.sum averaged over the step's 6
# GEMM launches, 10 executions of the step); a form is absent until such a
# capture exists for the current kernel and tree
GEMM_TRAFFIC_PER_LAUNCH = {"fp16x3": 7.572e9}


def peaks():
    if os.path.exists(MEASURED_PEAKS):
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return dict(hbm_gbs=p["hbm_gbs"], bf16_tflops=p["bf16_tflops"],
                    bf16_tflops_sustained=p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                    sm_max_mhz=p.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
                source="fallback")


def fp32_alu_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# tensor-core flops the split forms issue per complex MAC: 4 real products x
# 3 piece products x 2 (FP16S: 4 x 1 x 2); the TF32 peak is half the bf16
# peak (nominal dense ratio 1.1 : 2.25)
TC_FLOPS_PER_MAC = {"bf16x3": 24.0, "tf32x3": 24.0, "fp16x3": 24.0, "fp16s": 8.0,
                    # Gauss's 3M product: 3 real products x 3 piece products x 2
                    "bf16x3_3m": 18.0, "tf32x3_3m": 18.0, "fp16x3_3m": 18.0}
TC_PEAK_RATIO = {"bf16x3": 1.0, "tf32x3": 0.5, "fp16x3": 1.0, "fp16s": 1.0,
                 "bf16x3_3m": 1.0, "tf32x3_3m": 0.5, "fp16x3_3m": 1.0}
FORM_CHOICES = ["fp32", "bf16x3", "tf32x3", "fp16x3", "fp16s", "bf16x3_3m", "tf32x3_3m", "fp16x3_3m"]


# plan options every bench plan takes, and whether plans autotune their
# tensor-core GEMMs before use (set from the command line)
PLAN_DEFAULTS = {}
AUTOTUNE = []


def make_plan(tn, L, T, O, sliced, tree, name, **opts):
    """A plan for a bench form name: the library form, with Gauss's 3M
    product on the tensor cores for the *_3m names (tc_products 3)."""
    form, _, m3 = name.partition("_")
    o = dict(PLAN_DEFAULTS, **opts)
    plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(tc_products=3 if m3 else 0, **o))
    if AUTOTUNE:
        plan.autotune()
    return plan


def roofline_ms(row, form, pk):
    """Roofline time of one launch of a profiled step: its algorithmic bytes
    over the measured HBM bandwidth, or its flops over the peak of the unit
    that runs it, whichever is larger."""
    kind = row["kind"]
    t_mem = row["bytes"] / (pk["hbm_gbs"] * 1e9)
    if kind in ("small", "tasks") or (kind == "gemm" and form == "fp32"):
        t_math = 8.0 * row["macs"] / (fp32_alu_peak_tflops(pk["sm_max_mhz"]) * 1e12)
    elif kind == "gemm":
        t_math = TC_FLOPS_PER_MAC[form] * row["macs"] / (pk["bf16_tflops"] * TC_PEAK_RATIO[form] * 1e12)
    else:
        t_math = 0.0
    return 1e3 * max(t_mem, t_math)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device=None):
    """Max of a float over ranks (identity at world 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def instance_seed_offset(rank):
    """Rank r contracts its own seeded instance (weak scaling)."""
    return 1000 * rank


class Clocks:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tn_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Workloads.  "tree" names the stored tree (paper_2103_03074_gb300/trees/)
# used unless --search-method asks for a fresh search; "search" is that
# fresh search's options.  "step_slices": slices per timed step (None: all).
WORKLOADS = {
    "rect3x4": dict(cfg=1, search=dict(trials=256, n_sliced=0), tree=None, step_slices=None, golden=None,
                    forms=["fp32", "tf32x3", "fp16x3", "bf16x3", "fp16s"],
                    desc="rect3x4_m8_allopen: 12 qubits, 8 cycles, all 12 open, no slicing "
                         "(one contraction per step: a latency-bound circuit)"),
    "rect5x6": dict(cfg=2, search=dict(trials=16384, n_sliced=8), tree="rect5x6", step_slices=None,
                    golden="cfg2_amplitudes.txt",
                    forms=["fp32", "tf32x3", "tf32x3_3m", "fp16x3", "fp16x3_3m", "bf16x3", "fp16s"],
                    desc="rect5x6_m12_open8_sliced8: 30 qubits, 12 cycles, 8 open, 22 fixed, "
                         "2^8 slices over 8 searched bonds"),
    "syc53_m14": dict(cfg=4, search=dict(trials=1024, log2_cap=30), tree="syc53_m14", step_slices=None,
                      golden="cfg4_amplitudes_sampled.txt",
                      forms=["fp16x3", "fp16x3_3m", "tf32x3", "tf32x3_3m", "fp32", "bf16x3", "fp16s"],
                      desc="rotated6x9m1_m14_open16_cap30: 53 qubits, 14 cycles, 16 open, 37 fixed, "
                           "intermediates <= 2^30, every slice of the stored tree's slice set (the whole "
                           "2^16-amplitude tensor per step)"),
    "syc53_m20": dict(cfg=5, search=dict(trials=1024, log2_cap=31), tree="syc53_m20", step_slices=64, golden=None,
                      forms=["fp16x3", "tf32x3"],
                      desc="rotated6x9m1_m20_open21_cap31: 53 qubits, 20 cycles, 21 open, 32 fixed, "
                           "intermediates <= 2^31, a fixed 64-slice subset (ids 0..63) of the stored tree's "
                           "slice set per step"),
}
# the batched workload: 256 independent seeded circuits of uneven size
# (16-30 qubits, 8-14 cycles, 6-10 open, 2^0-2^6 slices each) in one
# multi-stream CUDA graph (tn_batch_*); its parity is checked circuit by
# circuit in the GPU tests
BATCH_DESC = ("batch256: 256 seeded circuits on rectangular grids of 16-30 qubits, 8-14 cycles, 6-10 open qubits, "
              "2^0-2^6 slices each, one multi-stream CUDA graph")

# forms that meet the 1e-5 bound by construction (22+ significant bits per
# operand); only these can be the headline (BF16x3 keeps 16 bits, FP16S 11)
ACCURATE_FORMS = ("fp32", "tf32x3", "fp16x3", "tf32x3_3m", "fp16x3_3m")
DTYPE = {"fp32": "f32", "bf16x3": "bf16x3 (fp32 accumulate)", "tf32x3": "tf32x3 (fp32 accumulate)",
         "fp16x3": "fp16x3 (scaled, fp32 accumulate)", "fp16s": "f16 (scaled)",
         "bf16x3_3m": "bf16x3, 3M product (fp32 accumulate)", "tf32x3_3m": "tf32x3, 3M product (fp32 accumulate)",
         "fp16x3_3m": "fp16x3, 3M product (scaled, fp32 accumulate)"}


def workload(name, seed_offset=0):
    from tn_inputs.configs import make_config, CONFIGS
    import tn_inputs
    w = WORKLOADS[name]
    cfg = make_config(w["cfg"])
    if seed_offset:
        c = CONFIGS[w["cfg"]]
        cfg["circuit"] = tn_inputs.sycamore_circuit(c["layout"], c["rows"], c["cols"], c["cycles"],
                                                    c["seed"] + seed_offset)
    return cfg


def stored_tree_json(name):
    """The stored tree file's contents (plain JSON; loads no product code)."""
    if not name:
        return None
    p = os.path.join(TREES, f"{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def step_roofline(tn, L, O, sliced, tree, form, slices_per_batch, n_slices, measured_ms):
    """One timed step against its compiled plan's roofline time: the plan's
    ops priced on the host by tn_estimate_tree_ms (nominal peaks: 7 TB/s HBM,
    80 TFLOP/s FP32, 2.25 PFLOP/s tensor, 1.125 for TF32x3, + 2 us a launch)
    at the plan's own block width, the prologue once and the body once per
    block of the step.  Never raises: an error becomes the entry."""
    try:
        nb = int(round(math.log2(slices_per_batch)))
        e = tn.estimate_tree_ms(L, O, sliced, tree, form=form, batch_log2=nb)
        est = e.prologue_ms + (n_slices / float(1 << e.batch_log2)) * e.block_ms
        return {"estimate_ms": est, "measured_ms": measured_ms, "frac": est / measured_ms,
                "peaks": "nominal (7 TB/s, 80 / 2250 / 1125 TFLOP/s) + 2 us per launch"}
    except Exception as exc:  # the bench line must not depend on this extra key
        return {"error": str(exc)}


# ---------------------------------------------------------------- CPU oracle
class OracleSampler:
    """The CPU FP64 oracle on bounded samples of a workload, in slices/s.

    Small workloads (30 qubits and below): the oracle contracts whole slices
    (its own one-tensor-per-gate network, the sliced bonds fixed), one after
    another.  53-qubit workloads: one slice of the open network is out of the
    oracle's reach (its greedy order needs ~2^54 MACs), so it contracts a
    closed amplitude (the open qubits set to a sampled bitstring: the route
    of the stored oracle values) pair by pair, and the rate is extrapolated
    by MACs: slices/s = (MACs done / s) x n_slices / (2^n_open x MACs of one
    closed amplitude).  One pairwise step of that contraction can take tens
    of seconds, so samples end between steps: after a time budget, a MAC
    budget or a number of steps."""

    def __init__(self, workload_name, sliced, n_slices):
        from oracle import network as onet, contract as oc
        self.onet, self.oc = onet, oc
        self.cfg = workload(workload_name)
        self.k = len(self.cfg["open_qubits"])
        self.small = self.cfg["circuit"].n_qubits <= 30
        self.sliced, self.n_slices = list(sliced), n_slices
        self.it, self.idx, self.amp_macs = None, 0, None
        self.macs, self.secs, self.units, self.steps, self.finished = 0.0, 0.0, 0, 0, 0
        if self.small:
            self.net = onet.circuit_network(self.cfg["circuit"], self.cfg["fixed_bits"], self.cfg["open_qubits"])

    def _next_amplitude(self):
        bits = list(self.cfg["fixed_bits"])
        b = (0x9E3779B1 * (self.idx + 1)) % (1 << self.k)
        for j, q in enumerate(self.cfg["open_qubits"]):
            bits[q] = (b >> (self.k - 1 - j)) & 1
        self.idx += 1
        L, T, O = self.onet.circuit_network(self.cfg["circuit"], bits, [])
        self.it = self.oc.contract_iter(L, T, O)

    def run(self, budget_s=None, macs=None, steps=None):
        """Oracle work until budget_s seconds, `macs` MACs or `steps` pairwise
        steps (whole slices for the small workloads) have been done, checked
        between steps; returns the seconds spent."""
        t0 = time.perf_counter()
        m0, s0, u0 = self.macs, self.steps, self.units
        while True:
            if budget_s is not None and time.perf_counter() - t0 >= budget_s:
                break
            if macs is not None and self.macs - m0 >= macs:
                break
            if steps is not None and self.steps - s0 >= steps:
                break
            if self.small:
                L, T, O = self.net
                self.oc.slice_partial(L, T, O, self.sliced, self.units % (1 << len(self.sliced)))
                self.units += 1
                self.steps += 1
                continue
            if self.it is None:
                self._next_amplitude()
            try:
                t, step_macs = next(self.it)
                self.macs += step_macs[t]
                self.amp_macs = float(sum(step_macs))
                self.step_macs = step_macs
                self.steps += 1
            except StopIteration:
                self.it = None
                self.finished += 1
        dt = time.perf_counter() - t0
        self.secs += dt
        return dt

    def rate(self, macs=None, secs=None, units=None):
        """slices/s over every sample so far (or over the given totals)."""
        macs = self.macs if macs is None else macs
        secs = self.secs if secs is None else secs
        units = self.units if units is None else units
        if self.small:
            return units / secs
        return macs / secs * self.n_slices / ((1 << self.k) * self.amp_macs)

    def describe(self):
        if self.small:
            return (f"{self.units} whole-slice contractions of the 2^{len(self.sliced)}-slice workload by the FP64 "
                    f"oracle (numpy), {self.secs:.1f} s")
        return (f"closed-amplitude contraction of the FP64 oracle (numpy, greedy order, "
                f"2^{math.log2(self.amp_macs):.1f} complex MACs per amplitude): {self.steps} pairwise steps, "
                f"{self.macs:.3g} MACs in {self.secs:.1f} s; slices/s = MAC rate x {self.n_slices} slices / "
                f"(2^{self.k} amplitudes x MACs per amplitude)")


def cpu_baseline(workload_name, sliced, n_slices, budget_s=15.0):
    """The oracle timed on all host cores, then on one core (a subprocess with
    one BLAS/OpenMP thread) over the first pairwise steps (or slices) that the
    all-core sample finished in its first third; every number says what its
    sample was."""
    smp = OracleSampler(workload_name, sliced, n_slices)
    smp.run(budget_s=budget_s / 6)
    prefix = max(smp.steps, 1)
    smp.run(budget_s=budget_s * 5 / 6)
    out = {"value": smp.rate(), "unit": "slices/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": smp.describe()}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", workload_name,
           "--oracle-steps", str(prefix), "--oracle-sliced", json.dumps(list(sliced)),
           "--oracle-n-slices", str(n_slices)]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": one["value"], "unit": "slices/s", "cores": 1, "sample": one["sample"]}
    except Exception as exc:
        out["one_core"] = {"error": str(exc)[:200]}
    return out


def run_reference(args):
    """The reference arm: the CPU FP64 oracle as it stands, on this host's
    cores, on the bench's workload; each step a bounded sample (about 4 s of
    oracle work).  Loads no product code."""
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return 0
    name = args.workload
    w = WORKLOADS[name]
    st = stored_tree_json(w["tree"])
    sliced = st["sliced"] if st else []
    n_slices = (1 << len(sliced)) if st else 1
    if w["step_slices"]:
        n_slices = min(n_slices, w["step_slices"])
    smp = OracleSampler(name, sliced, n_slices)
    if smp.small:
        # one whole slice per step
        for _ in range(args.warmup):
            smp.run(steps=1)
        how = "one whole slice per step"
    else:
        # one closed amplitude in all, its pairwise steps cut into warm-up +
        # timed chunks at fixed step indices where the cumulative MACs cross
        # j / (W + K) of the total (a chunk holding no boundary-crossing step
        # is empty; one holding a large step is long)
        smp.run(steps=1)
        n_chunks = args.warmup + args.steps
        cum, ends = 0.0, []
        for i, m in enumerate(smp.step_macs):
            cum += m
            while len(ends) < n_chunks and cum >= (len(ends) + 1) * smp.amp_macs / n_chunks * (1 - 1e-12):
                ends.append(i + 1)
        ends += [len(smp.step_macs)] * (n_chunks - len(ends))
        done = 1
        for j in range(args.warmup):
            smp.run(steps=max(ends[j] - done, 0))
            done = max(done, ends[j])
        how = f"the pairwise steps of one closed amplitude cut into {n_chunks} chunks of about equal MACs"
    macs0, secs0, units0 = smp.macs, smp.secs, smp.units
    t0 = time.perf_counter()
    for j in range(args.warmup, args.warmup + args.steps):
        if smp.small:
            smp.run(steps=1)
        else:
            smp.run(steps=max(ends[j] - done, 0))
            done = max(done, ends[j])
    dt = time.perf_counter() - t0
    v = smp.rate(smp.macs - macs0, smp.secs - secs0, smp.units - units0)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "slices/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Sycamore-style circuit)",
            "config": {"workload": w["desc"], "step": "a bounded sample of CPU FP64 oracle work: " + how,
                       "slices_per_gpu_step": n_slices},
            "cpu_baseline": {"value": v, "unit": "slices/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} timed steps ({how}) after {args.warmup} warm-up steps; "
                                       f"in all: " + smp.describe()},
            "e2e": {"value": v, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_oracle_sample(args):
    """Subprocess leg of cpu_baseline (one core): the given number of
    pairwise steps (or slices)."""
    smp = OracleSampler(args.oracle_sample, json.loads(args.oracle_sliced), args.oracle_n_slices)
    smp.run(steps=args.oracle_steps)
    print(json.dumps({"value": smp.rate(), "sample": smp.describe()}))
    return 0


# ---------------------------------------------------------------- GPU arm
def load_golden_amplitudes(name):
    """(indices, amplitudes) of the stored FP64 oracle output, if present."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    idx, vals = [], []
    for line in open(path):
        if line.startswith("#"):
            continue
        i, re, im = line.split()
        idx.append(int(i))
        vals.append(complex(float(re), float(im)))
    return np.array(idx), np.array(vals)


def l2_flush_buffer(torch):
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")


def time_steps(torch, plan, ranges, amp, steps, warmup, stream, flush, n_open, n_qubits, d_out):
    """Per-step device times (ms); step k contracts ranges[k % len(ranges)];
    L2 flushed before each step, untimed."""
    import paper_2103_03074_gb300 as tn

    def one(k):
        b, e = ranges[k % len(ranges)]
        amp.zero_()
        plan.contract(b, e, amp, stream)
        tn.probabilities_xeb(amp, n_open, n_qubits, d_out=d_out, stream=stream, sync=False)

    with torch.cuda.stream(stream):
        for k in range(warmup):
            one(k)
        stream.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            one(k)
            evs[k][1].record(stream)
        stream.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def profile_roofline(tn, torch, L, T, O, sliced, tree, form, rng, amp, stream, pk, steps, dump=None, tag=""):
    """Per-op CUDA events (step-timing recorder) over `steps` steps: the
    dominant kernel class's roofline entry and every class's share."""
    pplan = make_plan(tn, L, T, O, sliced, tree, form, profile=1)
    with torch.cuda.stream(stream):
        pplan.contract(rng[0], rng[1], amp, stream)
        pplan.profile(reset=True)
        for _ in range(steps):
            pplan.contract(rng[0], rng[1], amp, stream)
    rows = pplan.profile()
    pplan.close()
    if dump:
        with open(f"{dump}.{tag}{form}.json", "w") as f:
            json.dump({"steps": steps, "rows": rows}, f)
    return summarise_profile(rows, form, pk, steps)


def summarise_profile(rows, form, pk, steps):
    """(roofline entry of the kernel class with the largest share, share of
    every class) from step-timing rows (kind, ms, launches, macs and bytes
    per launch) recorded over `steps` steps."""
    by_kind = {}
    for r in rows:
        d = by_kind.setdefault(r["kind"], {"ms": 0.0, "launches": 0, "macs": 0.0, "bytes": 0.0, "t_roof": 0.0})
        d["ms"] += r["ms"]
        d["launches"] += r["launches"]
        d["macs"] += r["macs"] * r["launches"]
        d["bytes"] += r["bytes"] * r["launches"]
        d["t_roof"] += r["launches"] * roofline_ms(r, form, pk)
    total_ms = sum(d["ms"] for d in by_kind.values())
    top = max(by_kind, key=lambda k: by_kind[k]["ms"])
    d = by_kind[top]
    avg_ms = d["ms"] / max(d["launches"], 1)
    if top == "gemm" and form == "fp32":
        peak = fp32_alu_peak_tflops(pk["sm_max_mhz"])
        achieved = 8 * d["macs"] / d["launches"] / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "gemm_f32_kernel (complex FP32 FMA)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock (derived)"}
    elif top == "gemm":
        peak = pk["bf16_tflops"] * TC_PEAK_RATIO[form]
        achieved = TC_FLOPS_PER_MAC[form] * d["macs"] / d["launches"] / (avg_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": GEMM_TRAFFIC_PER_LAUNCH.get(form), "kernel": "tc_gemm_kernel (tcgen05 split form)",
                "peak_source": pk["source"] + (" (bf16 burst x 0.5 for TF32)" if form == "tf32x3" else " (bf16 burst)")}
    else:
        achieved = d["bytes"] / d["launches"] / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": top, "peak_source": pk["source"]}
    roof["algorithmic_per_launch"] = {"flops": (TC_FLOPS_PER_MAC.get(form, 8.0) if top == "gemm" else 8.0) *
                                      d["macs"] / d["launches"], "bytes": d["bytes"] / d["launches"]}
    roof["share_of_step"] = d["ms"] / total_ms if total_ms else None
    roof["launches_per_step"] = d["launches"] / steps
    # per-launch roofline time (bytes over HBM bandwidth or flops over the
    # unit's peak, whichever is larger) summed over the class's launches,
    # over their measured time: the class mixes tensor-bound and HBM-bound
    # launches, so this is its meaningful fraction
    roof["roofline_time_frac"] = d["t_roof"] / d["ms"] if d["ms"] else None
    # the same over every launch of the step (measured peaks), the step's
    # kernel time against its per-launch roofline time
    roof["step_roofline_time_frac"] = (sum(v["t_roof"] for v in by_kind.values()) / total_ms) if total_ms else None
    share = {k: v["ms"] / total_ms for k, v in by_kind.items()}
    return roof, share


def plan_inputs(tn, args, wl, cfg):
    """(L, T, O, tree, sliced, stats, how): the stored tree unless a fresh
    search is asked for."""
    if args.choose_open:
        # the paper's choice: the open qubits behind a small first cut
        cfg["open_qubits"] = tn.choose_open_qubits(
            cfg["circuit"], len(cfg["open_qubits"]),
            tn.search_opts(**dict(wl["search"], trials=64), method="bipartition"))[0]
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    stored = None
    if args.search_method is None and wl["tree"]:
        from paper_2103_03074_gb300.trees import make_trees
        stored = make_trees.load(wl["tree"], L, O)
    if stored is not None:
        tree, sliced, st = stored
        how = f"stored tree paper_2103_03074_gb300/trees/{wl['tree']}.json"
    else:
        method = args.search_method or "greedy"
        search = dict(wl["search"], seed=args.seed) if args.seed is not None else dict(wl["search"])
        tree, sliced, st = tn.find_order(L, O, tn.search_opts(**search, method=method, objective=args.objective,
                                                              rank_form="fp16x3" if args.form == "all"
                                                              else args.form))
        how = f"fresh search ({method}, {args.objective})"
    if args.branch_merge:
        tree, _ = tn.merge_branches(L, O, sliced, tree)
    return L, T, O, tree, sliced, st, how


def cfg5_sample(tn, torch, stream, pk, n_slices=4):
    """The 20-cycle, 21-open-qubit workload on its stored tree: FP16X3 against
    plain FP32 on the same slices [0, n_slices) (one block), device time of
    one contraction after one warm-up; no oracle value exists at this size,
    so the split form is compared with FP32.  Returns a dict (or an error)."""
    import numpy as np
    try:
        cfg = workload("syc53_m20")
        wl = WORKLOADS["syc53_m20"]
        L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
        from paper_2103_03074_gb300.trees import make_trees
        stored = make_trees.load(wl["tree"], L, O)
        if stored is None:
            return {"error": "no stored tree"}
        tree, sliced, st = stored
        n_total = 1 << len(sliced)
        out = {"workload": wl["desc"].split(",")[0] + f", slices 0..{n_slices - 1} of {n_total} (stored tree)",
               "log2_macs_per_slice": st["log2_slice"]}
        amps = {}
        for form in ("fp16x3", "fp32"):
            plan = tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(use_graph=1))
            stats = plan.stats()
            amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
            with Clocks(torch.cuda.current_device()) as clk:
                ms = time_steps(torch, plan, [(0, n_slices)], amp, 1, 1, stream, l2_flush_buffer(torch), len(O),
                                cfg["circuit"].n_qubits, torch.zeros(3, dtype=torch.float64, device="cuda"))[0]
            macs = stats["macs_batch"] * (n_slices / stats["slices_per_batch"]) + stats["macs_prologue"]
            amps[form] = amp.cpu().numpy()
            out[form] = {"ms": ms, "slices_per_s": n_slices / (ms / 1e3),
                         "complex_tflops": 8 * macs / (ms / 1e3) / 1e12,
                         "extrapolated_full_s": n_total * ms / 1e3 / n_slices, "clocks": clk.summary()}
            plan.close()
            del amp
            torch.cuda.empty_cache()
        a, b = amps["fp16x3"], amps["fp32"]
        out["fp16x3_vs_fp32_rel_l2"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out["speedup_fp16x3_over_fp32"] = out["fp32"]["ms"] / out["fp16x3"]["ms"]
        return out
    except Exception as exc:
        return {"error": str(exc)[:300]}


def run_native(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build_library()
    if world > 1:
        torch.distributed.barrier()
    import paper_2103_03074_gb300 as tn

    pk = peaks()
    wl = WORKLOADS[args.workload]
    big = args.workload in ("syc53_m14", "syc53_m20")
    cfg = workload(args.workload, instance_seed_offset(rank))
    n_qubits = cfg["circuit"].n_qubits
    n_open = len(cfg["open_qubits"])
    L, T, O, tree, sliced, st, how = plan_inputs(tn, args, wl, cfg)
    n_total = 1 << len(sliced)
    n_slices = min(n_total, wl["step_slices"] or n_total)
    ranges = [(0, n_slices)]
    forms = [args.form] if args.form != "all" else wl["forms"]
    golden = None
    if wl["golden"] and instance_seed_offset(rank) == 0 and not args.choose_open:
        golden = load_golden_amplitudes(wl["golden"])
    stream = torch.cuda.Stream()
    flush = l2_flush_buffer(torch)
    amp = torch.zeros(2 << n_open, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(3, dtype=torch.float64, device="cuda")
    results = {}
    plans = {}
    for form in forms:
        try:
            plan = make_plan(tn, L, T, O, sliced, tree, form, use_graph=1)
        except tn.TNError as e:
            results[form] = {"error": str(e)}
            continue
        stats = plan.stats()
        macs_step = stats["macs_batch"] * (n_slices / stats["slices_per_batch"]) + stats["macs_prologue"]
        # FP32 (CUDA cores) is several times slower: on the 53-qubit steps it
        # gets 3 timed steps, the split forms the full count
        steps = args.steps if (form != "fp32" or not big) else min(args.steps, 3)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            times = time_steps(torch, plan, ranges, amp, steps, args.warmup if steps == args.steps else 1, stream,
                               flush, n_open, n_qubits, d_out)
        ms = max_over_ranks(sum(times), world, device="cuda")
        per_step = ms / steps
        err = None
        if golden is not None:
            a = amp.cpu().numpy()
            got = (a[0::2] + 1j * a[1::2])[golden[0]]
            err = float(np.linalg.norm(got - golden[1]) / np.linalg.norm(golden[1]))
        res = {"ms_per_step": per_step, "steps": steps, "slices_per_s": world * n_slices / (per_step / 1e3),
               "rel_l2_err": err, "complex_tflops": world * 8 * macs_step / (per_step / 1e3) / 1e12,
               "clocks": clk.summary(), "plan": stats, "macs_per_step": macs_step,
               "launches_per_step": stats["launches_prologue"] + stats["launches_batch"] *
               (n_slices / stats["slices_per_batch"]) + 2}
        res["roofline"], res["kernel_time_share"] = profile_roofline(
            tn, torch, L, T, O, sliced, tree, form, ranges[0], amp, stream, pk, 1 if big else min(steps, 5),
            dump=args.dump_profile)
        res["step_roofline"] = step_roofline(tn, L, O, sliced, tree, form, stats["slices_per_batch"], n_slices,
                                             per_step)
        results[form] = res
        if big:
            plan.close()  # the 53-qubit arenas are tens of GB each
            torch.cuda.empty_cache()
        else:
            plans[form] = plan
    ok = [f for f in forms if "error" not in results[f]]
    if not ok:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": {f: results[f]["error"] for f in forms}}))
        return 1
    # headline: the fastest form that meets the 1e-5 bound by construction
    # (22+ significant bits per operand) and, where an oracle value exists,
    # by measurement; BF16x3 (16 bits) and FP16S never
    within = [f for f in ok if f in ACCURATE_FORMS and
              (results[f]["rel_l2_err"] is None or results[f]["rel_l2_err"] <= 1e-5)]
    best = max(within or ok, key=lambda f: results[f]["slices_per_s"])
    r = results[best]
    # end to end through the C-ABI with host buffers (tn_contract_slices_host)
    plan = plans.get(best) or make_plan(tn, L, T, O, sliced, tree, best, use_graph=1)
    data = np.concatenate([np.stack([np.asarray(t, np.complex64).reshape(-1).real,
                                     np.asarray(t, np.complex64).reshape(-1).imag], 1).reshape(-1)
                           for t in T]).astype(np.float32)
    h_in = torch.from_numpy(data).pin_memory()
    h_amp = torch.empty(2 << n_open, dtype=torch.float64).pin_memory()
    h_stats = torch.empty(3, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        plan.contract_host(0, n_slices, h_in, n_qubits, h_amp, h_stats, stream)
    e2e_steps = r["steps"]
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.contract_host(0, n_slices, h_in, n_qubits, h_amp, h_stats, stream)
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), world, device="cuda") / e2e_steps
    e2e = {"value": world * n_slices / (e2e_ms / 1e3), "unit": "slices/s", "form": best,
           "h2d_bytes_per_step": int(data.nbytes), "d2h_bytes_per_step": int(h_amp.numel() * 8 + 24),
           "api": "tn_contract_slices_host (leaf values in, amplitudes and P(s1)/XEB/max p out, host buffers)"}
    for p in plans.values():
        p.close()
    if best not in plans:
        plan.close()
    torch.cuda.empty_cache()
    cfg5 = None
    if args.workload == "syc53_m14" and not args.no_cfg5 and world == 1:
        cfg5 = cfg5_sample(tn, torch, stream, pk)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, sliced, n_slices)
    split = [f for f in ok if f != "fp32" and f in ACCURATE_FORMS]  # split-precision tensor-core forms
    line = {
        "metric": METRIC, "value": r["slices_per_s"], "unit": "slices/s", "n_gpus": world, "steps": r["steps"],
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[best],
        "data": "synthetic (seeded Sycamore-style circuit, random bitstring)",
        "config": {"workload": wl["desc"], "form": best,
                   "step": f"{n_slices} of {n_total} slices summed in FP64 + probabilities/XEB",
                   "amplitudes_per_step": f"2^{n_open}" + (" (the whole tensor)" if n_slices == n_total else
                                                           f" ({n_slices} of {n_total} slices)"),
                   "full_slice_count": n_total, "tree": how,
                   "executor": "CUDA-graph replay of the prologue and per-block body",
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events); the "
                         "53-qubit intermediates are far larger than L2",
                   "complex_macs_per_step": r["macs_per_step"], "log2_macs_per_slice": st["log2_slice"],
                   "log2_width_per_slice": st["log2_width"], "slices_per_batch": r["plan"]["slices_per_batch"],
                   "arena_bytes": r["plan"]["arena_bytes"],
                   "open_qubits": cfg["open_qubits"] if args.choose_open else "fixed (the workload's)",
                   "branch_merge": bool(args.branch_merge)},
        "complex_tflops": r["complex_tflops"],
        "rel_l2_err_vs_fp64_oracle": r["rel_l2_err"],
        "split_vs_fp32": ({"split_form": max(split, key=lambda f: results[f]["slices_per_s"]),
                           "speedup": max(results[f]["slices_per_s"] for f in split) /
                           results["fp32"]["slices_per_s"]} if split and "fp32" in ok else None),
        "forms": {f: ({"slices_per_s": results[f]["slices_per_s"], "complex_tflops": results[f]["complex_tflops"],
                       "rel_l2_err_vs_fp64_oracle": results[f]["rel_l2_err"], "steps": results[f]["steps"],
                       "ms_per_step": results[f]["ms_per_step"], "roofline": results[f]["roofline"],
                       "kernel_time_share": results[f]["kernel_time_share"],
                       "step_roofline": results[f].get("step_roofline")}
                      if "error" not in results[f] else results[f]) for f in forms},
        "roofline": r["roofline"],
        "step_roofline": r.get("step_roofline"),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": r["clocks"],
        "gpu_launches": int(r["launches_per_step"] * r["steps"]),
        "syc53_m20": cfg5,
    }
    if n_slices < n_total:
        line["extrapolated_full_s"] = n_total / r["slices_per_s"]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """The batched workload: every circuit's slices in one tn_batch_run."""
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    from tn_inputs.configs import batch_recipes, make_batch_member
    torch.cuda.set_device(0)
    members = [make_batch_member(r) for r in batch_recipes()]
    nets = []
    for m in members:
        L, T, O = tn.circuit_network(m["circuit"], m["fixed_bits"], m["open_qubits"])
        tree, sliced, st = tn.find_order(L, O, tn.search_opts(trials=32, n_sliced=m["n_sliced"],
                                                              method=args.search_method or "greedy"))
        nets.append((L, T, O, tree, sliced, st))
    n_slices = sum(1 << len(x[4]) for x in nets)
    macs = sum((1 << len(x[4])) * 2.0 ** x[5]["log2_slice"] for x in nets)
    forms = [args.form] if args.form != "all" else ["fp32", "tf32x3", "fp16x3"]
    stream = torch.cuda.Stream()
    flush = l2_flush_buffer(torch)
    results = {}
    for form in forms:
        plans, amps = [], []
        for L, T, O, tree, sliced, st in nets:
            plans.append(tn.Plan(L, T, O, sliced, tree, form=form, opts=tn.plan_opts(**dict(PLAN_DEFAULTS, batch_log2=3))))
            amps.append(torch.zeros(2 << len(O), dtype=torch.float64, device="cuda"))
        batch = tn.Batch(plans, amps, n_streams=8)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                batch.run(stream)
            stream.synchronize()
            with Clocks(0) as clk:
                tot = 0.0
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    batch.run(stream)
                    e1.record(stream)
                    stream.synchronize()
                    tot += e0.elapsed_time(e1)
        ms = tot / args.steps
        results[form] = {"ms_per_step": ms, "slices_per_s": n_slices / (ms / 1e3),
                         "complex_tflops": 8 * macs / (ms / 1e3) / 1e12, "clocks": clk.summary()}
        batch.close()
        for p in plans:
            p.close()
    best = max([f for f in forms if f in ACCURATE_FORMS] or forms, key=lambda f: results[f]["slices_per_s"])
    r = results[best]
    line = {"metric": METRIC, "value": r["slices_per_s"], "unit": "slices/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[best],
            "data": "synthetic (seeded Sycamore-style circuits, random bitstrings)",
            "config": {"workload": BATCH_DESC, "form": best, "circuits": len(members), "slices_per_step": n_slices,
                       "complex_macs_per_step": macs,
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "order_search": args.search_method or "greedy"},
            "complex_tflops": r["complex_tflops"], "forms": results, "clocks": r["clocks"],
            "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line))
    return 0


def run_gemm(args):
    """One batched complex GEMM step C[h,m,n] = sum_k A[h,m,k] B[h,k,n] of log2
    shape --gemm H,M,K,N through a two-tensor plan (the h labels sliced and
    kept as batch labels): mean device time per contraction and its complex
    and tensor-core flop rates."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    h, m, k, n = (int(x) for x in args.gemm.split(","))
    name = "fp16x3" if args.form == "all" else args.form
    form = name.partition("_")[0]
    rng = np.random.default_rng(0)
    hl, ml, kl, nl = (list(range(b, b + c)) for b, c in ((300, h), (0, m), (100, k), (200, n)))
    A = (rng.standard_normal(2 ** (h + m + k)) + 1j * rng.standard_normal(2 ** (h + m + k))).astype(np.complex64)
    B = (rng.standard_normal(2 ** (h + k + n)) + 1j * rng.standard_normal(2 ** (h + k + n))).astype(np.complex64)
    labels = [hl + ml + kl, hl + kl + nl]
    tensors = [A.reshape((2,) * (h + m + k)), B.reshape((2,) * (h + k + n))]
    out_l, tree = ml + nl, [(0, 1)]
    if args.gemm_next:
        # a second GEMM C[h,m,n] D[.., p] (D of more values than a small step
        # takes) makes the first GEMM write its output as the second one's
        # split planes (the planar epilogue).  D contracts all n labels, or
        # with --gemm-next-low L the lowest L m labels and the lowest L n
        # labels, so that the first GEMM's half tile is one contiguous run of
        # the planes (as in the 53-qubit step's largest GEMM)
        p, low = args.gemm_next, args.gemm_next_low
        pl = list(range(400, 400 + p))
        dl = (ml[m - low:] + nl[n - low:] + pl) if low else (nl + pl)
        D = (rng.standard_normal(2 ** len(dl)) + 1j * rng.standard_normal(2 ** len(dl))).astype(np.complex64)
        labels.append(dl)
        tensors.append(D.reshape((2,) * len(dl)))
        out_l = (ml[:m - low] + nl[:n - low] + pl) if low else (ml + pl)
        tree = [(0, 1), (3, 2)]
    plan = make_plan(tn, labels, tensors, out_l, hl, tree, name, use_graph=1, tc_chunk_bytes=args.tc_chunk,
                     tc_flush_bytes=args.tc_flush)
    amp = torch.zeros(2 << len(out_l), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.contract(0, 1 << h, amp, stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.contract(0, 1 << h, amp, stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    macs = 2.0 ** (h + m + k + n)
    desc = plan.describe()
    plan.close()
    # per-op device times (step-timing recorder, CUDA events around each op)
    pplan = make_plan(tn, labels, tensors, out_l, hl, tree, name, profile=1, tc_chunk_bytes=args.tc_chunk,
                      tc_flush_bytes=args.tc_flush)
    with torch.cuda.stream(stream):
        pplan.contract(0, 1 << h, amp, stream)
        pplan.profile(reset=True)
        for _ in range(args.steps):
            pplan.contract(0, 1 << h, amp, stream)
    ops = [{"kind": r["kind"], "shape": r["shape"], "ms": r["ms"] / max(r["launches"], 1)}
           for r in pplan.profile() if r["launches"]]
    pplan.close()
    print(json.dumps({"gemm": {"log2_hmkn": [h, m, k, n], "form": name}, "ms_per_contraction": ms,
                      "complex_tflops": 8 * macs / (ms / 1e3) / 1e12,
                      "tensor_tflops": TC_FLOPS_PER_MAC.get(name, 8.0) * macs / (ms / 1e3) / 1e12,
                      "ops": ops, "plan": desc}))
    return 0


def run_rank53(args):
    """Tree ranking on the 53-qubit 14-cycle workload: candidate trees from
    bipartition searches with different seeds, each timed (FP16X3, CUDA
    graph, median of 3 steps) and profiled step by step; the learned cost
    model ranks each half of the candidates after training on the other
    half's per-step timings (cross-fitting), against the roofline-time
    (tn_estimate_tree_ms) and MAC rankings.  One JSON line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_03074_gb300 as tn
    torch.cuda.set_device(0)
    cfg = workload("syc53_m14")
    L, T, O = tn.circuit_network(cfg["circuit"], cfg["fixed_bits"], cfg["open_qubits"])
    cands = []
    for seed in range(1, 1 + args.rank_seeds):
        tree, sl, st = tn.find_order(L, O, tn.search_opts(trials=256, log2_cap=30, method="bipartition",
                                                          objective="roofline", rank_form="fp16x3", seed=seed))
        if all(tree != c["tree"] for c in cands):
            cands.append({"seed": seed, "tree": tree, "sliced": sl, "log2_macs": st["log2_total"],
                          "roofline_ms": tn.estimate_tree_ms(L, O, sl, tree, form="fp16x3").ms})
    stream = torch.cuda.Stream()
    amp = torch.zeros(2 << len(O), dtype=torch.float64, device="cuda")
    for c in cands:
        n = 1 << len(c["sliced"])
        plan = tn.Plan(L, T, O, c["sliced"], c["tree"], form="fp16x3", opts=tn.plan_opts(use_graph=1))
        ms = time_steps(torch, plan, [(0, n)], amp, 3, 1, stream, l2_flush_buffer(torch), len(O),
                        cfg["circuit"].n_qubits, torch.zeros(3, dtype=torch.float64, device="cuda"))
        c["measured_ms"] = float(np.median(ms))
        plan.close()
        pplan = tn.Plan(L, T, O, c["sliced"], c["tree"], form="fp16x3", opts=tn.plan_opts(profile=1))
        with torch.cuda.stream(stream):
            pplan.contract(0, n, amp, stream)
            pplan.profile(reset=True)
            pplan.contract(0, n, amp, stream)
        rows = [r for r in pplan.profile() if r["kind"] not in ("extract", "accumulate")]
        c["X"] = pplan.op_features()
        c["y"] = np.log2(np.maximum([r["ms"] / max(r["launches"], 1) for r in rows], 1e-4)).astype(np.float32)
        pplan.close()
        torch.cuda.empty_cache()
    # cross-fitting: the model that ranks a candidate never saw its steps
    halves = [cands[0::2], cands[1::2]]
    for i in (0, 1):
        train, test = halves[1 - i], halves[i]
        if not train or not test:
            continue
        X = np.concatenate([c["X"] for c in train])
        y = np.concatenate([c["y"] for c in train])
        cm = tn.CostModel(seed=11 + i)
        cm.train(torch.from_numpy(X).cuda(), torch.from_numpy((y - 16.0 * X[:, 14]).astype(np.float32)).cuda(),
                 epochs=3000, lr=3e-3)
        for c in test:
            d = torch.zeros(len(c["X"]), dtype=torch.float32, device="cuda")
            cm.predict(torch.from_numpy(c["X"]).cuda(), d)
            torch.cuda.synchronize()
            c["model_ms"] = float(np.sum(2.0 ** (16.0 * c["X"][:, 14] + d.cpu().numpy())))
        cm.close()
    pick = lambda key: min(cands, key=lambda c: c.get(key, float("inf")))
    out = {"workload": WORKLOADS["syc53_m14"]["desc"].split(",")[0] + ", FP16X3, the whole tensor per step",
           "candidates": [{k: c[k] for k in ("seed", "log2_macs", "roofline_ms", "measured_ms", "model_ms") if k in c}
                          for c in cands],
           "best_ms": min(c["measured_ms"] for c in cands),
           "mac_pick_ms": pick("log2_macs")["measured_ms"], "roofline_pick_ms": pick("roofline_ms")["measured_ms"],
           "model_pick_ms": pick("model_ms")["measured_ms"]}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--form", default="all", choices=FORM_CHOICES + ["all"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batch256", "gemm", "rank53"])
    ap.add_argument("--rank-seeds", type=int, default=8, help="--workload rank53: search seeds (candidate trees)")
    ap.add_argument("--gemm", default="0,15,11,9", help="--workload gemm: log2 H,M,K,N")
    ap.add_argument("--gemm-next", type=int, default=0,
                    help="--workload gemm: follow the GEMM by a second one of log2 N = this, so that the first "
                         "writes the second one's split planes from its epilogue")
    ap.add_argument("--gemm-next-low", type=int, default=0,
                    help="--workload gemm with --gemm-next: the second GEMM contracts the lowest L m and n labels")
    ap.add_argument("--tc-chunk", type=int, default=0, help="tensor-core K chunk bytes (plan option tc_chunk_bytes)")
    ap.add_argument("--tc-flush", type=int, default=0,
                    help="K bytes between accumulator read-outs (plan option tc_flush_bytes)")
    ap.add_argument("--search-method", default=None, choices=["greedy", "bipartition", "mixed"],
                    help="search a fresh tree (randomised greedy, hierarchical bipartition, or both) instead of "
                         "the workload's stored tree")
    ap.add_argument("--objective", default="macs", choices=["macs", "roofline"],
                    help="with --search-method: rank the search's trees by total MACs (default) or by the roofline "
                         "time of their compiled plan (tn_estimate_tree_ms) for --form (fp16x3 with --form all)")
    ap.add_argument("--seed", type=int, default=None, help="order-search seed (default: the library's)")
    ap.add_argument("--choose-open", action="store_true",
                    help="take the open qubits behind a small first cut (tn_choose_open_qubits) instead of the "
                         "workload's fixed set; the stored oracle amplitudes then do not apply (no error reported)")
    ap.add_argument("--branch-merge", action="store_true",
                    help="rewrite ((X a) b) into (X (a b)) where the step-time estimate drops (tn_merge_branches)")
    ap.add_argument("--small-tasks", type=int, default=0,
                    help="plan option small_tasks: 0 tiny small steps as tasks of one launch, -1 one launch each")
    ap.add_argument("--small-tc-bits", type=int, default=0,
                    help="plan option small_tc_bits: small steps with K + N of at least this many bits on the tensor cores")
    ap.add_argument("--tc-tma-store", type=int, default=0,
                    help="plan option tc_tma_store: 0 (default) staged planar GEMM outputs stored by TMA where "
                         "their layout allows, -1 from the epilogue warps")
    ap.add_argument("--autotune", action="store_true",
                    help="time each tensor-core GEMM's (chunk, read-out) candidates before use (tn_plan_autotune)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cfg5", action="store_true", help="skip the 20-cycle sample of the default line")
    ap.add_argument("--dump-profile", default="", help="write per-op step timings to PATH.<form>.json")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-steps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-sliced", default="[]", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-n-slices", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        return run_oracle_sample(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.choose_open and args.search_method is None:
        args.search_method = "bipartition"
    if args.small_tasks:
        PLAN_DEFAULTS["small_tasks"] = args.small_tasks
    if args.small_tc_bits:
        PLAN_DEFAULTS["small_tc_bits"] = args.small_tc_bits
    if args.tc_chunk:
        PLAN_DEFAULTS["tc_chunk_bytes"] = args.tc_chunk
    if args.tc_flush:
        PLAN_DEFAULTS["tc_flush_bytes"] = args.tc_flush
    if args.tc_tma_store:
        PLAN_DEFAULTS["tc_tma_store"] = args.tc_tma_store
    if args.autotune:
        AUTOTUNE.append(True)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        return run_batch(args)
    if args.workload == "gemm":
        return run_gemm(args)
    if args.workload == "rank53":
        return run_rank53(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
