#!/usr/bin/env python
"""Benchmark of libk2svd on GB300: FP64 2x2 SVDs/s on the wide-range workload, as a
fraction of the FP64-pipe roofline, plus the FP32 variant and the end-to-end rate
through the Python API with host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs the same per-GPU workload on its own GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.

Workload (one step, per GPU): 2^27 general matrices through k2svd_dgesvd2 plus 2^27
upper-triangular matrices through k2svd_dtrsvd2, entries with exponents uniform over
the normal range and 2% subnormal or near-overflow entries (paper_2407_13116_gb300/inputs.py).
Inputs (7.5 GB) are larger than L2, so no L2 flush is needed between steps.
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

SEED = 0x240713116
N_HALF_D = 1 << 27
N_HALF_S = 1 << 28
E2E_HALF = 1 << 27
N_DIFF = 1 << 24
N_KOG = 8192
N_COMPLEX = 1 << 26
N_RECT = 2048
E2E_CHUNK = 1 << 22
METRIC = "FP64 2×2 SVDs/s & % of roofline; fwd+bwd/s; batched Kogbetliantz speedup"
BYTES_GE = {"d": 112, "s": 56}          # in 4 T + out (4 U + 4 V + 2 S) T
BYTES_TR = {"d": 104, "s": 52}          # in 3 T + out 10 T


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp32", action="store_true")
    p.add_argument("--no-fwd-bwd", action="store_true")
    p.add_argument("--no-kog", action="store_true")
    p.add_argument("--no-phases", action="store_true")
    p.add_argument("--no-complex", action="store_true")
    p.add_argument("--no-rect", action="store_true")
    p.add_argument("--no-ncr", action="store_true")
    p.add_argument("--no-kog-grad", action="store_true")
    p.add_argument("--no-narrow", action="store_true")
    p.add_argument("--summarize-ncu", default=None, help="print per-pipe counts per unit from an ncu --csv log")
    p.add_argument("--units", default="", help="with --summarize-ncu: substring=units per launch, ...")
    p.add_argument("--profile-case", choices=["d", "s", "dn", "sn", "kog", "kog128", "z", "misc"], default=None,
                   help="run a small case of the 2x2 kernels (d, s; dn, sn: the variant with the hypot "
                        "that is not correctly rounded), of the complex kernel (z) or of the persistent "
                        "Kogbetliantz kernel (kog), for ncu captures, and exit")
    p.add_argument("--profile-n", type=int, default=1 << 22)
    return p.parse_args()


# ----------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU; barrier and max-over-ranks timing only)
# ----------------------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


def shard_offset(n_per_rank, rank):
    """First global matrix index of a rank's contiguous slice: rank r takes matrices
    [r n, (r+1) n) of one global batch.  The generators are counter-based, so each rank
    builds exactly its slice and no data moves between ranks."""
    return rank * n_per_rank


def shard_seed(seed, rank):
    """Seed of a rank's independent batch for the workloads generated per batch (the
    differentiation and Kogbetliantz sets): distinct per rank, equal to `seed` on rank 0."""
    return seed + 1000003 * rank


# ----------------------------------------------------------------------------------------
# clock sampling during the timed region
# ----------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------
# roofline bookkeeping
# ----------------------------------------------------------------------------------------
# ----------------------------------------------------------------------------------------
# Per-pipe instruction ceilings.  A kernel cannot finish faster than its busiest pipe can
# issue the warp instructions it executes, so for each pipe P the time
#     t_P = (warp instructions on P per unit) x units / (peak rate of P per SM per clock x SMs x clock)
# is a lower bound on the kernel's duration, and the kernel's ceiling is the largest t_P.
# The counts per unit come from one ncu capture of each kernel on a small case of the same
# workload (bench.py --profile-case ..., summarised by --summarize-ncu into the tables of
# profiles/pipe_ceilings.md); the clock is the median SM clock sampled during the timed
# region.  A count table is valid only for the kernel sources whose hash it was taken at;
# after any change to them the ceiling is reported as null until a new capture is taken.
# ----------------------------------------------------------------------------------------
PIPE_METRIC = {"issue": "sm__inst_executed", "fp64": "sm__inst_executed_pipe_fp64",
               "alu": "sm__inst_executed_pipe_alu", "fmaheavy": "sm__inst_executed_pipe_fmaheavy",
               "fmalite": "sm__inst_executed_pipe_fmalite", "fma": "sm__inst_executed_pipe_fma",
               "lsu": "sm__inst_executed_pipe_lsu", "xu": "sm__inst_executed_pipe_xu",
               "cbu": "sm__inst_executed_pipe_cbu", "adu": "sm__inst_executed_pipe_adu",
               "uniform": "sm__inst_executed_pipe_uniform"}
# warp instructions per clock per SM (ncu `<metric>.sum.peak_sustained` on a GB300 / 152 SMs)
PIPE_PEAK = {"issue": 4.0, "fp64": 1.0 / 16, "alu": 2.0, "fmaheavy": 2.0, "fmalite": 2.0, "fma": 4.0,
             "lsu": 1.0, "xu": 1.0, "cbu": 4.0, "adu": 0.5, "uniform": 2.0}
SRC_2X2 = ("k2_fp.cuh", "k2_svd2.cuh", "k2_svd2_kernel.cuh", "k2_gesvd2.cu")
SRC_GROUPS = {"2x2": SRC_2X2, "complex": SRC_2X2 + ("k2_complex.cu",), "bwd": ("k2_fp.cuh", "k2_bwd.cu"),
              "kog": SRC_2X2 + ("k2_kog.cu", "k2_kog_dev.cuh")}
# The source hashes at which the count tables below were taken (profiles/pipe_ceilings.md).
PIPE_COUNTS_HASH = {"2x2": "66c5311866092db6", "complex": "863ca888f717e75a", "bwd": "411a7ed9f6c0a0b6",
                    "kog": "5203ec2c0f0f9d40"}


def _pc(group, unit, counts, dram):
    return (group, unit, dict(zip(("issue", "fp64", "alu", "fmaheavy", "fmalite", "fma", "lsu", "xu", "cbu",
                                   "adu", "uniform"), counts)), dram)


# kernel -> (source group, unit, {pipe: warp instructions per unit}, DRAM bytes per unit under
# ncu, caches flushed before each launch); 2^22-matrix captures of the benchmark workloads
PIPE_COUNTS = {
    "svd2a_kernel<double>": _pc("2x2", "matrix", (81.284, 1.3574, 43.682, 15.843, 1.5647, 17.407, 2.4248, 1.1828, 6.5887, 0.30869, 0), 101.4),
    "svd2b_kernel<double>": _pc("2x2", "matrix", (116.39, 1.3503, 54.034, 27.184, 2.7579, 29.942, 8.5144, 1.7869, 11.121, 0.60196, 0.125), 135.55),
    "svd2_kernel<double,tri>": _pc("2x2", "matrix", (100.61, 1.4394, 47.036, 25.429, 2.2595, 27.688, 3.1595, 1.4839, 10.404, 0.43565, 0.12732), 100.64),
    "svd2_kernel<float,general>": _pc("2x2", "matrix", (83.694, 0.53125, 35.634, 18.224, 7.0246, 25.249, 1.2257, 2.1746, 9.0441, 0.55958, 0.12732), 46.024),
    "svd2_kernel<float,tri>": _pc("2x2", "matrix", (50.633, 0, 22.662, 10.339, 4.3216, 14.661, 0.69446, 1.2046, 6.087, 0.2887, 0.12732), 39.138),
    "lasv2_kernel<double>": _pc("2x2", "matrix", (98.237, 1.4707, 47.182, 23.393, 2.2597, 25.653, 2.7323, 1.4839, 10.529, 0.43565, 0.0023193), 74.048),
    "csvd2_kernel<double>": _pc("complex", "matrix", (265.53, 4.2253, 116.98, 68.34, 6.1931, 74.533, 11.673, 3.9658, 25.641, 1.2871, 0.085815), 654.65),
    "bwd_kernel<double>": _pc("bwd", "matrix", (16.355, 1.2188, 5.5112, 2.6453, 0.21848, 2.8638, 0.75116, 0.125, 1.0449, 0.034611, 0.12616), 188.62),
    # the three instantiations of the 608-matrix run (orders <= 32 with U and V in shared
    # memory, 33..64 with 64 registers, above 64) summed: one unit mix, a slightly lower bound
    "kog_persistent<double>": _pc("kog", "rotation FP64 operation", (0.60907, 0.035216, 0.16407, 0.15840, 0.0038365,
                                                                     0.16223, 0.061835, 0.0093784, 0.032953,
                                                                     0.0040808, 0.0051653), 0.0010475),
}


def src_hash(group):
    """Hash of the code of a group of kernel sources, comments and blank space removed (a
    comment edit does not invalidate a count table)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in SRC_GROUPS[group]:
        with open(os.path.join(ROOT, "paper_2407_13116_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        code = " ".join(code.split())
        h.update(hashlib.sha256(code.encode()).hexdigest().encode() + b"  " + f.encode() + b"\n")
    return h.hexdigest()[:16]


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def ceiling(kernels, units, clock_mhz):
    """Lower bound (seconds) on the summed duration of `kernels` processing `units` units
    each, from their per-pipe instruction counts; None when a count table is missing or was
    taken at other kernel sources.  Returns (seconds, {kernel: binding pipe}, DRAM bytes)."""
    sms, f = sm_count(), clock_mhz * 1e6
    total, pipes, dram = 0.0, {}, 0.0
    for k in kernels:
        if k not in PIPE_COUNTS:
            return None
        group, _, per, dbytes = PIPE_COUNTS[k]
        if PIPE_COUNTS_HASH.get(group) != src_hash(group):
            return None
        t = {p: c * units / (PIPE_PEAK[p] * sms * f) for p, c in per.items()}
        b = max(t, key=t.get)
        total += t[b]
        pipes[k] = b
        dram += dbytes * units
    return total, pipes, dram


def roofline_entry(kernels, units, unit_name, measured_s, clock_mhz, algorithmic_bytes, fp64_model=None):
    """The bench line's roofline object for kernels timed together (CUDA events): achieved
    units/s against the per-pipe instruction ceiling at the sampled clock."""
    c = ceiling(kernels, units, clock_mhz)
    hbm, hbm_src = hbm_peak_gbs()
    out = {"bound": "alu", "unit": unit_name + "/s", "achieved": units / measured_s, "kernels": list(kernels),
           "kernel_ms": measured_s * 1e3, "algorithmic_bytes": algorithmic_bytes,
           "hbm_frac": (algorithmic_bytes / measured_s / (hbm * 1e9)) if algorithmic_bytes else None,
           "clock_mhz": clock_mhz}
    if c is None:
        out.update({"peak": None, "frac": None, "traffic": None,
                    "note": "no per-pipe count table for the current kernel sources"})
    else:
        t, pipes, dram = c
        out.update({"peak": units / t, "frac": t / measured_s, "traffic": dram, "binding_pipe": pipes,
                    "ceiling_ms": t * 1e3,
                    "peak_source": "per-pipe warp-instruction counts (ncu, profiles/pipe_ceilings.md) at the pipes' "
                                   "issue rates (ncu peak_sustained) x %d SMs x the median SM clock %.0f MHz sampled "
                                   "during the timed region" % (sm_count(), clock_mhz)})
    if fp64_model is not None:
        out["fp64_model_frac"] = fp64_model
    return out


def summarize_ncu(path, units_spec):
    """Per-kernel per-pipe warp instructions per unit from an ncu --csv metrics log (the
    metrics of profiles/pipe_ceilings.md); units_spec: 'substring=units,...' (units per
    launch of the kernels whose name contains substring, or 'total:' + units for all
    launches of the kernel together).  Prints a markdown table and the count literals."""
    import collections
    import csv
    rows = [r for r in csv.reader(open(path)) if len(r) > 14 and r[0] != "ID"]
    launches = collections.OrderedDict()
    for r in rows:
        try:
            v = float(r[14].replace(",", ""))
        except ValueError:
            continue
        launches.setdefault(r[0], {"name": r[4]})[r[12]] = v
    spec = [kv.split("=") for kv in units_spec.split(",")] if units_spec else []
    agg = collections.OrderedDict()
    for d in launches.values():
        a = agg.setdefault(d["name"], collections.defaultdict(float))
        a["launches"] += 1
        a["cycles"] += d.get("sm__cycles_elapsed.max", 0.0)
        a["ms"] += d.get("gpu__time_duration.sum", 0.0) / 1e6
        a["dram"] += d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
        for p, m in PIPE_METRIC.items():
            a[p] += d.get(m + ".sum", 0.0)
        for k in ("smsp__thread_inst_executed_per_inst_executed.ratio", "launch__registers_per_thread",
                  "sm__cycles_elapsed.avg.per_second"):
            a[k] = d.get(k, 0.0)
    print("| kernel | launches | units | ms | clock MHz | lanes | " + " | ".join(PIPE_METRIC) +
          " | busiest pipe, fraction of elapsed | DRAM B/unit |")
    print("|" + "---|" * (len(PIPE_METRIC) + 8))
    lits = {}
    for nm, a in agg.items():
        units = None
        for sub, u in spec:
            if sub in nm:
                units = float(u[6:]) if u.startswith("total:") else float(u) * a["launches"]
        if not units:
            continue
        per = {p: a[p] / units for p in PIPE_METRIC}
        frac = {p: a[p] / (PIPE_PEAK[p] * 152) / a["cycles"] for p in PIPE_METRIC}
        b = max(frac, key=frac.get)
        print("| %s | %d | %.6g | %.3f | %.0f | %.1f | %s | %s %.3f | %.1f |" % (
            nm, a["launches"], units, a["ms"], a["sm__cycles_elapsed.avg.per_second"] / 1e6,
            a["smsp__thread_inst_executed_per_inst_executed.ratio"],
            " | ".join("%.4g" % per[p] for p in PIPE_METRIC), b, frac[b], a["dram"] / units))
        lits[nm] = {p: float("%.5g" % per[p]) for p in PIPE_METRIC}, float("%.5g" % (a["dram"] / units))
    print()
    for nm, (per, d) in lits.items():
        print(repr(nm), per, d)


def fp64_peak(clock_mhz):
    """Nominal FP64 fma rate: 152 SMs x 2 DFMA per clock per SM (the sm_103 pipe rate
    ncu reports as sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained) x clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 2.0 * clock_mhz * 1e6


def hbm_peak_gbs():
    """The measured HBM copy bandwidth of this GPU model (MEASURED_PEAKS.json), else the
    earlier measurement on a GB300 (6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


# FP64 operations of the 2x2 adjoint per matrix (k2svd_dgesvd2_bwd): J12 - J21 and K12 - K21
# (2 fma, 2 mul, 1 add each), the gap and F12 (2 add, 2 mul, 1 division), the two
# off-diagonal entries of M (fma, mul, mul each), W = U M and dG = W V^T (8 each).
BWD_OPS = {"arith": 36, "div": 1}


def load_opcounts():
    with open(os.path.join(ROOT, "tests", "golden", "opcounts.json")) as f:
        return json.load(f)["workloads"]


def slot_costs(c, rates, prec):
    """FP64-pipe and FP32-pipe issue slots per matrix for the method's operations.

    A division and a square root cost rate(fma)/rate(div) and rate(fma)/rate(sqrt) fma
    slots of their pipe (measured); a correctly rounded hypot costs one multiplication,
    one fma and one square root; eq. (EXT) is integer work for double (0 FP slots) and a
    double multiplication, fma and division for float; the square roots of the variant's
    hypot cost one square root each."""
    sq = c.get("sqrt", 0.0)
    if prec == "d":
        wd, ws = rates["dfma"] / rates["ddiv"], rates["dfma"] / rates["dsqrt"]
        fp64 = c["add"] + c["mul"] + c["fma"] + c["div"] * wd + c["hypot"] * (2 + ws) + sq * ws
        return {"fp64": fp64, "fp32": 0.0}
    wd, ws = rates["ffma"] / rates["fdiv"], rates["ffma"] / rates["fsqrt"]
    fp32 = c["add"] + c["mul"] + c["fma"] + c["div"] * wd + c["hypot"] * (2 + ws) + sq * ws
    fp64 = c["ext"] * (2 + rates["dfma"] / rates["ddiv"])
    return {"fp64": fp64, "fp32": fp32}


def probe_rates(L):
    import ctypes as C
    L.k2probe_rate.argtypes = [C.c_int, C.c_void_p]
    L.k2probe_rate.restype = C.c_int
    out = {}
    for op, nm in enumerate(("dfma", "ddiv", "dsqrt", "ffma", "fdiv", "fsqrt")):
        v = C.c_double(0)
        rc = L.k2probe_rate(op, C.byref(v))
        if rc != 0:
            raise RuntimeError("k2probe_rate(%d) returned %d" % (op, rc))
        out[nm] = v.value
    return out


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def leg(prec, n_half, steps, warmup, dev, D, clocks_index=None, ncr=False):
    """Time `steps` steps of gesvd2(n_half general) + trsvd2(n_half triangular) (ncr: the
    variant with the hypot that is not correctly rounded)."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    dt = torch.float64 if prec == "d" else torch.float32
    i0 = shard_offset(n_half, D.rank)          # this rank's slice of the global batch
    G = I.general(n_half, SEED + 2, prec, "wide", i0=i0, xp="torch", device=dev)
    T3 = I.triangular(n_half, SEED + 3, prec, "wide", i0=i0, xp="torch", device=dev)
    F, Gu, H = T3[0], T3[1], T3[2]
    Ug = torch.empty((4, n_half), dtype=dt, device=dev); Vg = torch.empty_like(Ug)
    Sg = torch.empty((2, n_half), dtype=dt, device=dev)
    Ut = torch.empty_like(Ug); Vt = torch.empty_like(Ug); St = torch.empty_like(Sg)
    torch.cuda.synchronize()

    def step():
        k2svd.gesvd2(G, U=Ug, V=Vg, S=Sg, want_info=False, ncr=ncr)
        k2svd.trsvd2(F, Gu, H, U=Ut, V=Vt, S=St, want_info=False, ncr=ncr)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(clocks_index) if clocks_index is not None else None
    if clk:
        clk.start()
    D.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        k2svd.gesvd2(G, U=Ug, V=Vg, S=Sg, want_info=False, ncr=ncr)
        ev[k][1].record(stream)
        k2svd.trsvd2(F, Gu, H, U=Ut, V=Vt, S=St, want_info=False, ncr=ncr)
        ev[k][2].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    D.barrier()
    clocks = clk.stop() if clk else None
    ms = t0.elapsed_time(t1) / steps
    ge_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    tr_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    del G, T3, F, Gu, H, Ug, Vg, Sg, Ut, Vt, St
    torch.cuda.empty_cache()
    # kernels per step: the FP64 general batch of 65536 or more runs as two launches (phases
    # 1-2, phase 3), everything else as one; the triangular batch as one
    per_step = (3 if prec == "d" and not ncr and n_half >= (1 << 16) else 2)
    return {"ms": ms, "ge_ms": ge_ms, "tr_ms": tr_ms, "clocks": clocks, "launches": per_step * steps}


def ncr_leg(steps, warmup, dev, D, rates, clk_mhz, oc, value_cr, fp32_cr):
    """The variant with the hypot that is not correctly rounded (Alg. 1's branch for it) on
    the headline workloads: 2^27 + 2^27 FP64 and 2^28 + 2^28 FP32 wide-range matrices."""
    out = {}
    for prec, n_half, cr in (("d", N_HALF_D, value_cr), ("s", N_HALF_S, (fp32_cr or {}).get("value"))):
        r = leg(prec, n_half, steps, warmup, dev, D, ncr=True)
        ms = D.max(r["ms"])
        v = D.world * 2 * n_half / (ms / 1e3)
        c_ge = slot_costs(oc["wide_%s_gesvd2_ncr" % prec], rates, prec)
        c_tr = slot_costs(oc["wide_%s_trsvd2_ncr" % prec], rates, prec)
        o = {"value": v, "unit": "SVDs/s", "ms_per_step": ms, "gesvd2_ms": r["ge_ms"], "trsvd2_ms": r["tr_ms"],
             "matrices_per_gpu_per_step": 2 * n_half,
             "vs_correctly_rounded": (v / cr) if cr else None}
        if prec == "d":
            peak = fp64_peak(clk_mhz)
            ach = n_half * c_ge["fp64"] / (r["ge_ms"] / 1e3)
            o["roofline"] = {"bound": "alu", "achieved": ach / 1e9, "peak": peak / 1e9, "unit": "G FP64-pipe op/s",
                             "frac": ach / peak, "kernel": "svd2_kernel<double,false,true> (k2svd_dgesvd2_ncr)",
                             "ops_per_matrix": c_ge["fp64"]}
        else:
            roof32 = 2 / ((c_ge["fp32"] + c_tr["fp32"]) / rates["ffma"])
            roof64 = 2 / ((c_ge["fp64"] + c_tr["fp64"]) / rates["dfma"])
            o["frac_of_min_roofline"] = v / D.world / min(roof32, roof64)
        out[prec] = o
    out["workload"] = "the headline wide-range workloads through k2svd_{d,s}gesvd2_ncr / k2svd_{d,s}trsvd2_ncr"
    return out


def fwd_bwd_leg(steps, warmup, dev, D, rates, clk_mhz):
    """The differentiation workload: 2^24 FP64 matrices R(theta) diag(s1, s2) R(phi)^T; one step
    is the forward (k2svd_dgesvd2) and the backward (k2svd_dgesvd2_bwd) with upstream
    gradients dS, dU, dV ~ N(0,1)."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    n = N_DIFF
    G = torch.from_numpy(I.rotated(n, shard_seed(SEED + 3, D.rank))[0]).to(dev)
    gen = torch.Generator(device=dev).manual_seed(SEED + 3)
    dS = torch.randn((2, n), dtype=torch.float64, device=dev, generator=gen)
    dU = torch.randn((4, n), dtype=torch.float64, device=dev, generator=gen)
    dV = torch.randn((4, n), dtype=torch.float64, device=dev, generator=gen)
    U = torch.empty((4, n), dtype=torch.float64, device=dev); V = torch.empty_like(U)
    S = torch.empty((2, n), dtype=torch.float64, device=dev); dG = torch.empty_like(U)
    torch.cuda.synchronize()

    def step(ev=None):
        if ev:
            ev[0].record()
        k2svd.gesvd2(G, U=U, V=V, S=S, want_info=False)
        if ev:
            ev[1].record()
        k2svd.gesvd2_bwd(U, S, V, dS, dU, dV, dG=dG)
        if ev:
            ev[2].record()

    for _ in range(warmup):
        step()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(steps)]
    D.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        step(evs[k])
    torch.cuda.synchronize()
    D.barrier()
    fwd = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    bwd = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    ms = D.max(fwd + bwd)
    bwd_bytes = 192 * n
    del G, dS, dU, dV, U, V, S, dG
    torch.cuda.empty_cache()
    hbm, hbm_src = hbm_peak_gbs()
    ops = BWD_OPS["arith"] + BWD_OPS["div"] * rates["dfma"] / rates["ddiv"]
    peak = fp64_peak(clk_mhz)
    t_fp64, t_hbm = n * ops / peak, bwd_bytes / (hbm * 1e9)
    return {"value": D.world * n / (ms / 1e3), "unit": "fwd+bwd/s", "matrices_per_gpu_per_step": n,
            "fwd_ms": fwd, "bwd_ms": bwd, "bwd_over_fwd": bwd / fwd,
            "bwd_roofline": roofline_entry(["bwd_kernel<double>"], n, "matrix", bwd / 1e3, clk_mhz, bwd_bytes,
                                           fp64_model=(n * ops / (bwd / 1e3)) / peak),
            "workload": "2^24 FP64 R(theta) diag(s1,s2) R(phi)^T, 10% near-equal singular values, upstream N(0,1)"}


KOG_BUCKETS = ((8, 32), (33, 64), (65, 96), (97, 128))


def kog_leg(steps, warmup, dev, D, rates):
    """Batched Kogbetliantz: 8192 FP64 matrices of order uniform in {8..128} (Q1 diag(sigma)
    Q2^T, sigma log-uniform in [1e-12, 1]) to off-norm < n eps ||G||_F.  The persistent form
    (one graph launch of per-bucket persistent kernels) is timed over `steps` runs with the
    SM clock sampled; the per-step form (three launches per step, a host read-back per sweep)
    after one warm-up run, median of three.  Beside them: each order range alone, the
    rotation floor (the 8 n^3 FP64 operations per sweep of the row, column, U and V
    rotations at the FP64 pipe's rate) and the per-pipe instruction ceiling."""
    import numpy as np
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    orders = I.kog_orders(N_KOG, 8, 128, shard_seed(SEED + 4, D.rank))
    flat, _ = I.kog_batch(orders, shard_seed(SEED + 4, D.rank))
    A = torch.from_numpy(flat).to(dev)
    n, offs, soffs, tot, stot = k2svd.kog_layout(orders)
    U = torch.empty(tot, dtype=torch.float64, device=dev); V = torch.empty_like(U)
    S = torch.empty(stot, dtype=torch.float64, device=dev)
    sw = torch.empty(len(n), dtype=torch.int32, device=dev); info = torch.empty_like(sw)
    ws = k2svd.kogbet_workspace(orders, torch.float64, k2svd.KOG_GRAPH, dev)
    run = lambda fl, w: k2svd.kogbet(A, orders, flags=fl, workspace=w, U=U, V=V, S=S, sweeps=sw, info=info)
    for _ in range(warmup + 1):                 # the first call tunes the block sizes
        run(k2svd.KOG_GRAPH, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(D.local)
    clk.start()
    D.barrier()
    e0.record()
    for _ in range(steps):
        run(k2svd.KOG_GRAPH, ws)
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    pers_ms = D.max(e0.elapsed_time(e1) / steps)
    clk_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    sweeps = sw.cpu().numpy().astype(np.int64)
    conv = int((info.cpu().numpy() == 0).sum())
    Sp = S.clone()
    wsp = k2svd.kogbet_workspace(orders, torch.float64, k2svd.KOG_PLAIN, dev)
    run(k2svd.KOG_PLAIN, wsp)                   # warm-up of the per-step form
    torch.cuda.synchronize()
    plain = []
    for _ in range(3):
        t = time.perf_counter()
        run(k2svd.KOG_PLAIN, wsp)
        torch.cuda.synchronize()
        plain.append((time.perf_counter() - t) * 1e3)
    plain_ms = D.max(statistics.median(plain))
    same = bool(torch.equal(Sp, S))
    del wsp
    nn = orders.astype(np.int64)
    rot = sweeps * 8 * nn ** 3                  # FP64 operations of the rotations, per matrix
    sms = sm_count()
    nominal = sms * 2.0 * clk_mhz * 1e6         # 2 DFMA per clock per SM
    floor_ms = float(rot.sum()) / nominal * 1e3
    floor_probe_ms = float(rot.sum()) / rates["dfma"] * 1e3
    # each order range alone (same matrices, same form)
    buckets = {}
    for lo, hi in KOG_BUCKETS:
        sel = np.flatnonzero((orders >= lo) & (orders <= hi))
        if len(sel) == 0:
            continue
        ob = orders[sel]
        Ab = torch.from_numpy(np.concatenate([flat[offs[i]:offs[i] + orders[i] ** 2] for i in sel])).to(dev)
        nb_, ob_offs, ob_soffs, tb, sb = k2svd.kog_layout(ob)
        Ub = torch.empty(tb, dtype=torch.float64, device=dev); Vb = torch.empty_like(Ub)
        Sb = torch.empty(sb, dtype=torch.float64, device=dev)
        wsb = k2svd.kogbet_workspace(ob, torch.float64, k2svd.KOG_GRAPH, dev)
        runb = lambda: k2svd.kogbet(Ab, ob, flags=k2svd.KOG_GRAPH, workspace=wsb, U=Ub, V=Vb, S=Sb)
        runb()
        torch.cuda.synchronize()
        tb_ms = []
        for _ in range(3):
            e0.record(); runb(); e1.record(); torch.cuda.synchronize()
            tb_ms.append(e0.elapsed_time(e1))
        bf = float(rot[sel].sum()) / nominal * 1e3
        buckets["%d..%d" % (lo, hi)] = {"matrices": int(len(sel)), "ms": statistics.median(tb_ms),
                                        "rotation_floor_ms": bf, "over_floor": statistics.median(tb_ms) / bf}
        del Ab, Ub, Vb, Sb, wsb
    # the dynamic pivot ordering (persistent graph form), same matrices and stopping rule
    wsd = k2svd.kogbet_workspace(orders, torch.float64, k2svd.KOG_GRAPH | k2svd.KOG_DYNAMIC, dev)
    for _ in range(warmup + 1):
        run(k2svd.KOG_GRAPH | k2svd.KOG_DYNAMIC, wsd)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        run(k2svd.KOG_GRAPH | k2svd.KOG_DYNAMIC, wsd)
    e1.record()
    torch.cuda.synchronize()
    dyn_ms = D.max(e0.elapsed_time(e1) / steps)
    dyn_sweeps = sw.cpu().numpy().astype(np.int64)
    dyn_conv = int((info.cpu().numpy() == 0).sum())
    del wsd
    # BASELINE's FP64 model: per sweep n(n-1)/2 pivots at 239 FP64 slots and 16 n FP64
    # operations per pivot for the rotations
    ops = float((sweeps * (nn * (nn - 1) // 2) * (16 * nn + 239)).sum())
    roof = roofline_entry(["kog_persistent<double>"], float(rot.sum()), "rotation FP64 op", pers_ms / 1e3, clk_mhz, None,
                          fp64_model=ops / (pers_ms / 1e3) / nominal)
    roof["unit_note"] = ("units are the rotations' FP64 operations (8 n^3 per sweep); the ceiling scales the "
                         "instructions counted per such operation on a 608-matrix sample of the same order mix")
    del A, U, V, S, ws
    torch.cuda.empty_cache()
    return {"speedup_vs_per_step": plain_ms / pers_ms, "persistent_ms": pers_ms, "per_step_ms": plain_ms,
            "per_step_runs_ms": plain, "matrices_per_gpu": N_KOG, "converged": conv,
            "mean_sweeps": float(sweeps.mean()), "max_sweeps": int(sweeps.max()), "forms_bitwise_equal": same,
            "rotation_floor_ms": floor_ms, "rotation_floor_probe_ms": floor_probe_ms,
            "over_rotation_floor": pers_ms / floor_ms,
            "max_speedup_at_floor": plain_ms / floor_ms,
            "buckets": buckets, "clocks": clocks, "roofline": roof,
            "dynamic_ordering": {"persistent_ms": dyn_ms, "speedup_vs_per_step": plain_ms / dyn_ms,
                                 "vs_modulus_persistent": pers_ms / dyn_ms, "mean_sweeps": float(dyn_sweeps.mean()),
                                 "max_sweeps": int(dyn_sweeps.max()), "converged": dyn_conv},
            "workload": "8192 FP64 Q1 diag(sigma) Q2^T, n uniform in {8..128}, sigma log-uniform [1e-12,1], "
                        "modulus strategy (and the dynamic ordering beside it), off < n eps ||G||_F"}


def kog_grad_leg(steps, warmup, dev, D):
    """Batched Kogbetliantz with gradients: 2048 FP64 matrices of order uniform in {32..256}
    and 4096 FP32 matrices of order uniform in {8..128}, built as the batched workload.  A step
    is, for each batch, the forward (persistent graph form) and the gradient of sum(dS * S)
    with respect to A (dA = U diag(dS) V^T) through the autograd Function, dS ~ N(0,1)."""
    import numpy as np
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    from paper_2407_13116_gb300.autograd import kogbet_sigma
    seed = shard_seed(SEED + 5, D.rank)
    parts = []
    for count, lo, hi, dt, sd in ((2048, 32, 256, np.float64, seed), (4096, 8, 128, np.float32, seed + 1)):
        o = I.kog_orders(count, lo, hi, sd)
        f, _ = I.kog_batch(o, sd, dtype=dt)
        A = torch.from_numpy(f).to(dev).requires_grad_(True)
        stot = int(k2svd.kog_layout(o)[4])
        gen = torch.Generator(device=dev).manual_seed(sd)
        dS = torch.randn(stot, dtype=A.dtype, device=dev, generator=gen)
        parts.append((o, A, dS))

    def one(o, A, dS):
        U, S, V, sw, info = kogbet_sigma(A, o, flags=k2svd.KOG_GRAPH)
        (dA,) = torch.autograd.grad(S, A, dS)
        return sw, info

    for _ in range(warmup + 1):                 # the first call tunes the block sizes
        for p_ in parts:
            one(*p_)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    D.barrier()
    for k in range(steps):
        ev[k][0].record()
        sw64, info64 = one(*parts[0])
        ev[k][1].record()
        sw32, info32 = one(*parts[1])
        ev[k][2].record()
    torch.cuda.synchronize()
    ms64 = statistics.median(e[0].elapsed_time(e[1]) for e in ev)
    ms32 = statistics.median(e[1].elapsed_time(e[2]) for e in ev)
    ms = D.max(ms64 + ms32)
    out = {"value": D.world * (2048 + 4096) / (ms / 1e3), "unit": "matrices/s (forward + sigma gradient)",
           "ms_per_step": ms, "fp64_ms": ms64, "fp32_ms": ms32,
           "fp64_mean_sweeps": float(sw64.double().mean()), "fp32_mean_sweeps": float(sw32.double().mean()),
           "converged": int((info64 == 0).sum()) + int((info32 == 0).sum()),
           "workload": "2048 FP64 of order uniform in {32..256} + 4096 FP32 of order uniform in {8..128}, "
                       "Q1 diag(sigma) Q2^T; forward and dA = U diag(dS) V^T through the autograd Function"}
    del parts
    torch.cuda.empty_cache()
    return out


def narrow_leg(steps, warmup, dev, D):
    """The plain forward on 2^20 FP64 narrow-range matrices (exponents in [-20, 20], 25% upper
    triangular, 5% with a zero row or column) through k2svd_dgesvd2.  The 112 MB of inputs and
    outputs fit in L2, so a 512 MB buffer is written between timed calls (outside the events)."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    n = 1 << 20
    G = I.general(n, SEED + 1, "d", "narrow", i0=shard_offset(n, D.rank), xp="torch", device=dev)
    U = torch.empty((4, n), dtype=torch.float64, device=dev); V = torch.empty_like(U)
    S = torch.empty((2, n), dtype=torch.float64, device=dev)
    flush = torch.empty(1 << 26, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        k2svd.gesvd2(G, U=U, V=V, S=S, want_info=False)
    ts = []
    D.barrier()
    for _ in range(max(steps, 10)):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        k2svd.gesvd2(G, U=U, V=V, S=S, want_info=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = D.max(statistics.median(ts))
    del G, U, V, S, flush
    torch.cuda.empty_cache()
    return {"value": D.world * n / (ms / 1e3), "unit": "SVDs/s", "ms": ms, "l2": "flushed between calls",
            "workload": "2^20 FP64 narrow-range general matrices (25% triangular, 5% with a zero row or column)"}


def phases_leg(steps, warmup, dev, D, rates, clk_mhz, oc):
    """The standalone phase 1 (k2svd_dprescale2, extra = 1, on 2^27 general matrices) and the
    xLASV2 argument shape (k2svd_dlasv2 on 2^27 triangular matrices) of the wide workload."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    n = N_HALF_D
    i0 = shard_offset(n, D.rank)
    G = I.general(n, SEED + 2, "d", "wide", i0=i0, xp="torch", device=dev)
    Gs = torch.empty_like(G)
    res = {}

    def timed(fn):
        for _ in range(warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        D.barrier()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return D.max(e0.elapsed_time(e1) / steps)

    ms = timed(lambda: k2svd.prescale2(G, extra=1, Gs=Gs))
    hbm, hbm_src = hbm_peak_gbs()
    nbytes = 72 * n
    res["prescale2"] = {"value": D.world * n / (ms / 1e3), "unit": "matrices/s", "ms": ms,
                        "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm,
                                     "unit": "GB/s", "frac": nbytes / (ms / 1e3) / (hbm * 1e9),
                                     "algorithmic_bytes": nbytes, "peak_source": hbm_src},
                        "workload": "2^27 wide-range FP64 general matrices, extra = 1 (G in 32 B, Gs out 32 B, s, types)"}
    del G, Gs
    T3 = I.triangular(n, SEED + 3, "d", "wide", i0=i0, xp="torch", device=dev)
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(6)]
    L = k2svd.lib()
    ptrs = [o.data_ptr() for o in outs]
    st = torch.cuda.current_stream().cuda_stream
    ms = timed(lambda: L.k2svd_dlasv2(n, T3[0].data_ptr(), T3[1].data_ptr(), T3[2].data_ptr(), *ptrs, st))
    cost = slot_costs(oc["wide_d_trsvd2"], rates, "d")["fp64"]
    peak = fp64_peak(clk_mhz)
    res["lasv2"] = {"value": D.world * n / (ms / 1e3), "unit": "SVDs/s", "ms": ms,
                    "roofline": roofline_entry(["lasv2_kernel<double>"], n, "SVD", ms / 1e3, clk_mhz, 72 * n,
                                               fp64_model=n * cost / (ms / 1e3) / peak),
                    "workload": "2^27 wide-range FP64 upper-triangular matrices (F, G, H in, 6 planes out)"}
    del T3, outs
    torch.cuda.empty_cache()
    return res


def complex_leg(steps, warmup, dev, D, rates, clk_mhz, oc):
    """The complex 2x2 SVD (k2svd_zgesvd2, Sect. 3.4) on 2^26 double complex matrices whose
    real and imaginary planes are two wide-range streams."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    n = N_COMPLEX
    i0 = shard_offset(n, D.rank)
    G = torch.empty((8, n), dtype=torch.float64, device=dev)
    G[0::2] = I.general(n, SEED + 6, "d", "wide", i0=i0, xp="torch", device=dev)
    G[1::2] = I.general(n, SEED + 7, "d", "wide", i0=i0, xp="torch", device=dev)
    U = torch.empty((8, n), dtype=torch.float64, device=dev); V = torch.empty_like(U)
    S = torch.empty((2, n), dtype=torch.float64, device=dev)
    fn = lambda: k2svd.cgesvd2(G, U=U, V=V, S=S, want_info=False)
    for _ in range(warmup):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = D.max(e0.elapsed_time(e1) / steps)
    cost = slot_costs(oc["wide_d_cgesvd2"], rates, "d")["fp64"]
    peak = fp64_peak(clk_mhz)
    hbm, _ = hbm_peak_gbs()
    nbytes = (64 + 64 + 64 + 16) * n
    del G, U, V, S
    torch.cuda.empty_cache()
    return {"value": D.world * n / (ms / 1e3), "unit": "SVDs/s", "ms": ms,
            "roofline": roofline_entry(["csvd2_kernel<double>"], n, "SVD", ms / 1e3, clk_mhz, nbytes,
                                       fp64_model=n * cost / (ms / 1e3) / peak),
            "workload": "2^26 double complex 2x2 matrices, real and imaginary parts wide-range (exponents "
                        "uniform in [-1021,1021], 2% subnormal or near-overflow); 208 B per matrix"}


def rect_leg(steps, warmup, dev, D, rates, clk_mhz):
    """Rectangular matrices (k2svd_dgesvdr: QR with column pivoting to square, the n x n
    Kogbetliantz driver, U = Q U_R): 2048 FP64 matrices with n uniform in {8..128} and m
    uniform in {n..3n}, N(0,1) entries."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    seed = shard_seed(SEED + 8, D.rank)
    n = I.kog_orders(N_RECT, 8, 128, seed)
    m = (n + np.floor(I.uniform01(N_RECT, seed, 9) * (2 * n + 1))).astype(np.int32)
    shapes = np.stack([m, n], 1)
    mm, nn, ao, uo, vo, so, (na, nu, nv, ns) = k2svd.rect_layout(shapes)
    A = torch.from_numpy(I.normal(na, seed, 10)).to(dev)
    U = torch.empty(nu, dtype=torch.float64, device=dev); V = torch.empty(nv, dtype=torch.float64, device=dev)
    S = torch.empty(ns, dtype=torch.float64, device=dev)
    sw = torch.empty(N_RECT, dtype=torch.int32, device=dev); info = torch.empty_like(sw)
    L = k2svd.lib()
    wsb = C.c_size_t(0)
    assert L.k2svd_dgesvdr_ws(N_RECT, mm.ctypes.data, nn.ctypes.data, 0, C.byref(wsb)) == 0
    ws = torch.empty(wsb.value + 256, dtype=torch.uint8, device=dev)
    wp = C.c_void_p((ws.data_ptr() + 255) // 256 * 256)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (N_RECT, mm.ctypes.data, nn.ctypes.data, ao.ctypes.data, uo.ctypes.data, vo.ctypes.data, so.ctypes.data,
            A.data_ptr(), U.data_ptr(), V.data_ptr(), S.data_ptr(), sw.data_ptr(), info.data_ptr(), 40, 1.0, 0,
            wp, wsb.value, st)
    fn = lambda: L.k2svd_dgesvdr(*args)
    for _ in range(max(warmup, 1)):
        assert fn() == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = D.max(e0.elapsed_time(e1) / steps)
    sweeps = sw.cpu().numpy().astype(np.float64)
    p_, q_ = np.maximum(m, n).astype(np.float64), np.minimum(m, n).astype(np.float64)
    wd = rates["dfma"] / rates["ddiv"]
    ops = 0.0
    for p1, q1, s1 in zip(p_, q_, sweeps):
        j = np.arange(q1)
        ops += float(((q1 - j) * (p1 - j)).sum())                              # column norms
        ops += float(((q1 - j - 1) * (2 * (p1 - j) + wd)).sum())               # reflector applications
        ops += float((q1 * (2 * (p1 - j) + wd)).sum())                         # Q
        ops += s1 * (q1 * (q1 - 1) / 2) * (16 * q1 + 239)                      # Kogbetliantz sweeps
        ops += p1 * q1 * q1                                                     # Q U_R
    peak = fp64_peak(clk_mhz)
    conv = int((info.cpu().numpy() == 0).sum())
    del A, U, V, S, ws
    torch.cuda.empty_cache()
    return {"value": D.world * N_RECT / (ms / 1e3), "unit": "matrices/s", "ms": ms, "converged": conv,
            "mean_sweeps": float(sweeps.mean()),
            "roofline": {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e9, "peak": peak / 1e9,
                         "unit": "G FP64-pipe op/s", "frac": ops / (ms / 1e3) / peak, "ops": ops},
            "workload": "2048 FP64 m x n matrices, n uniform in {8..128}, m uniform in {n..3n}, N(0,1) entries; "
                        "QR with column pivoting, the n x n Kogbetliantz driver, U = Q U_R"}


def host_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def e2e_leg(steps, warmup, dev, D):
    """End to end through the public API on the headline batch: the inputs (2^27 general and
    2^27 triangular matrices) sit in pinned host memory, k2svd.svd2_host streams them through
    the device in 2^22-matrix chunks (host-to-device copy, k2svd_dgesvd2 / k2svd_dtrsvd2,
    device-to-host copy of U, V and S, on three streams), and a step ends when every output
    is back in host memory."""
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    torch.cuda.empty_cache()          # the earlier legs' cached blocks go back to the driver
    n, c = E2E_HALF, E2E_CHUNK
    # pinned host memory for inputs and outputs: 27 doubles per general + triangular pair
    while n > c and host_bytes() and 2 * n * 27 * 8 > 0.5 * host_bytes():
        n //= 2
    nc = n // c
    dt = torch.float64
    i0 = shard_offset(n, D.rank)
    Gh = torch.empty((nc, 4, c), dtype=dt, pin_memory=True)
    Th = torch.empty((nc, 3, c), dtype=dt, pin_memory=True)
    for q in range(nc):              # generated on the device chunk by chunk, kept in host memory
        Gh[q].copy_(I.general(c, SEED + 2, "d", "wide", i0=i0 + q * c, xp="torch", device=dev))
        Th[q].copy_(I.triangular(c, SEED + 3, "d", "wide", i0=i0 + q * c, xp="torch", device=dev))
    Og = torch.empty((nc, 10, c), dtype=dt, pin_memory=True)
    Ot = torch.empty((nc, 10, c), dtype=dt, pin_memory=True)
    jobs = [(Gh, Og, False), (Th, Ot, True)]
    for _ in range(warmup):
        k2svd.svd2_host(jobs, device=dev)
    D.barrier()
    per = []
    t = time.perf_counter()
    for _ in range(steps):
        t1 = time.perf_counter()
        k2svd.svd2_host(jobs, device=dev)
        per.append(time.perf_counter() - t1)
    el = D.max((time.perf_counter() - t) / steps)
    # two more steps outside the timed region with every copy and kernel bracketed by events:
    # where the time of a step goes (the device-to-host stream's busy time against the span)
    traces = []
    for _ in range(2):
        tr = []
        k2svd.svd2_host(jobs, device=dev, trace=tr)
        traces.append(tr)
    tr = max(traces, key=lambda x: x[-1]["end_ms"])
    span = max(r["end_ms"] for r in tr)
    trace_summary = {"span_ms": span, "d2h_busy_ms": sum(r["d2h_ms"] for r in tr),
                     "h2d_busy_ms": sum(r["h2d_ms"] for r in tr), "kernel_busy_ms": sum(r["kernel_ms"] for r in tr),
                     "max_d2h_ms": max(r["d2h_ms"] for r in tr), "max_h2d_ms": max(r["h2d_ms"] for r in tr),
                     "max_kernel_ms": max(r["kernel_ms"] for r in tr)}
    h2d = (4 + 3) * 8 * n
    d2h = 2 * (4 + 4 + 2) * 8 * n
    # the host link's own copy rates on this machine (one pinned 2 GiB copy each way, then both
    # at once), for reading the end-to-end number
    link = {}
    x = Og.view(-1)[: 1 << 28]
    y = torch.empty(x.numel(), dtype=dt, device=dev)
    sa, sb = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(ops):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for st, fn in ops:
            with torch.cuda.stream(st):
                fn()
        torch.cuda.synchronize()
        return x.numel() * 8 / (time.perf_counter() - t0) / 1e9
    up, down = (sa, lambda: y.copy_(x, non_blocking=True)), (sb, lambda: x.copy_(y, non_blocking=True))
    timed([up, down])
    link["h2d_gbs"], link["d2h_gbs"], link["both_gbs_each"] = timed([up]), timed([down]), timed([up, down])
    del Gh, Th, Og, Ot, x, y
    torch.cuda.empty_cache()
    med = statistics.median(per)
    return {"value": D.world * 2 * n / el, "unit": "SVDs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "batch": 2 * n, "ms_per_step": el * 1e3, "chunk": c, "api": "k2svd.svd2_host", "link": link,
            "copy_bound_ms": max(h2d / link["h2d_gbs"], d2h / link["d2h_gbs"]) / 1e6,
            "step_ms_min_max": [min(per) * 1e3, max(per) * 1e3], "step_ms_median": med * 1e3,
            "step_ms": [round(x * 1e3, 2) for x in per],
            "mean_over_median": el / med, "traced_step": trace_summary,
            "note": "inputs and outputs in pinned host memory; every copy is inside the timed region"}


def cpu_baseline(seconds=10.0):
    """The oracle (plain C, all host cores) on a bounded sample of the same workload."""
    import oracle
    from paper_2407_13116_gb300 import inputs as I
    cores = os.cpu_count() or 1
    probe = 1 << 14
    Gs = I.general(probe, SEED + 2, "d", "wide")
    Ts = I.triangular(probe, SEED + 3, "d", "wide")
    t = time.perf_counter()
    oracle.gesvd2(Gs, "d", nthreads=cores)
    oracle.trsvd2(Ts[0], Ts[1], Ts[2], "d", nthreads=cores)
    rate = 2 * probe / (time.perf_counter() - t)
    m = int(min(max(rate * seconds / 2, probe), 1 << 23))
    Gs = I.general(m, SEED + 2, "d", "wide")
    Ts = I.triangular(m, SEED + 3, "d", "wide")
    t = time.perf_counter()
    oracle.gesvd2(Gs, "d", nthreads=cores)
    oracle.trsvd2(Ts[0], Ts[1], Ts[2], "d", nthreads=cores)
    el = time.perf_counter() - t
    # one thread on a smaller sample (about 2 s), beside the all-core rate
    m1 = int(min(max(rate / cores * 2.0 / 2, 1 << 12), 1 << 20))
    t = time.perf_counter()
    oracle.gesvd2(Gs[:, :m1], "d", nthreads=1)
    oracle.trsvd2(Ts[0, :m1], Ts[1, :m1], Ts[2, :m1], "d", nthreads=1)
    el1 = time.perf_counter() - t
    return {"value": 2 * m / el, "unit": "SVDs/s", "cores": cores, "kind": "oracle",
            "sample": "first %d general + %d triangular matrices of the wide-range FP64 workload, "
                      "OpenMP over matrices on %d host threads, %.1f s" % (m, m, cores, el),
            "single_thread": {"value": 2 * m1 / el1, "unit": "SVDs/s",
                              "sample": "first %d + %d of the same matrices on one thread, %.1f s" % (m1, m1, el1)}}


def headline_config():
    """The headline workload, shared by both arms (the reference arm times a sample of it)."""
    return {"workload": "wide-range FP64 2x2 SVD: 2^27 general (k2svd_dgesvd2) + 2^27 upper-triangular "
                        "(k2svd_dtrsvd2) per GPU, exponents uniform in [-1021,1021], 2% subnormal or "
                        "near-overflow entries, SoA planes",
            "matrices_per_gpu_per_step": 2 * N_HALF_D, "l2": "inputs (7.5 GB) larger than L2",
            "parallelism": "one slice of the global batch per rank (weak scaling, no collective)"}


def run_ours(a):
    import torch
    D = Dist()
    dev = torch.device("cuda", D.local)
    torch.cuda.set_device(dev)
    from paper_2407_13116_gb300 import build as B
    B.build()
    from paper_2407_13116_gb300 import k2svd
    k2svd.lib()
    rates = probe_rates(k2svd.probe_lib())
    oc = load_opcounts()
    res = leg("d", N_HALF_D, a.steps, a.warmup, dev, D, clocks_index=D.local)
    ms = D.max(res["ms"])
    value = D.world * 2 * N_HALF_D / (ms / 1e3)
    clk_mhz = (res["clocks"] or {}).get("sm_mhz") or 2070.0
    # BASELINE's FP64-pipe model of the method's counted operations, kept beside the ceiling
    cost_ge = slot_costs(oc["wide_d_gesvd2"], rates, "d")["fp64"]
    cost_tr = slot_costs(oc["wide_d_trsvd2"], rates, "d")["fp64"]
    peak64 = fp64_peak(clk_mhz)
    model_ge = N_HALF_D * cost_ge / (res["ge_ms"] / 1e3) / peak64
    model_step = 2 * N_HALF_D / (ms / 1e3) / D.world / (2 * N_HALF_D / ((N_HALF_D * (cost_ge + cost_tr)) / peak64))
    roofline = roofline_entry(["svd2a_kernel<double>", "svd2b_kernel<double>"], N_HALF_D, "SVD",
                              res["ge_ms"] / 1e3, clk_mhz, BYTES_GE["d"] * N_HALF_D, fp64_model=model_ge)
    roofline["entry"] = "k2svd_dgesvd2 (phases 1-2, then phase 3)"
    tri = roofline_entry(["svd2_kernel<double,tri>"], N_HALF_D, "SVD", res["tr_ms"] / 1e3, clk_mhz,
                         BYTES_TR["d"] * N_HALF_D)
    c_step = ceiling(["svd2a_kernel<double>", "svd2b_kernel<double>", "svd2_kernel<double,tri>"], N_HALF_D, clk_mhz)
    roofline["step"] = {"frac": (c_step[0] / (ms / 1e3)) if c_step else None, "fp64_model_frac": model_step,
                        "trsvd2": tri}
    out = {"metric": METRIC, "value": value, "unit": "SVDs/s", "n_gpus": D.world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": headline_config(),
           "clocks": res["clocks"], "gpu_launches": res["launches"], "roofline": roofline,
           "pipe_rates": rates}
    if D.world == 1 and not a.no_e2e:
        out["e2e"] = e2e_leg(max(8, a.steps), 1, dev, D)
    if not a.no_fp32:
        rs = leg("s", N_HALF_S, a.steps, a.warmup, dev, D, clocks_index=D.local)
        mss = D.max(rs["ms"])
        clk_s = (rs["clocks"] or {}).get("sm_mhz") or clk_mhz
        cs_ge = slot_costs(oc["wide_s_gesvd2"], rates, "s")
        cs_tr = slot_costs(oc["wide_s_trsvd2"], rates, "s")
        roof32 = 2 / ((cs_ge["fp32"] + cs_tr["fp32"]) / rates["ffma"])
        roof64 = 2 / ((cs_ge["fp64"] + cs_tr["fp64"]) / rates["dfma"])
        roofhbm = 2 / ((BYTES_GE["s"] + BYTES_TR["s"]) / (hbm_peak_gbs()[0] * 1e9))
        vs = D.world * 2 * N_HALF_S / (mss / 1e3)
        out["fp32"] = {"value": vs, "unit": "SVDs/s", "ms_per_step": mss, "matrices_per_gpu_per_step": 2 * N_HALF_S,
                       "gesvd2_ms": rs["ge_ms"], "trsvd2_ms": rs["tr_ms"], "clocks": rs["clocks"],
                       "roofline": roofline_entry(["svd2_kernel<float,general>"], N_HALF_S, "SVD", rs["ge_ms"] / 1e3,
                                                  clk_s, BYTES_GE["s"] * N_HALF_S),
                       "roofline_trsvd2": roofline_entry(["svd2_kernel<float,tri>"], N_HALF_S, "SVD",
                                                         rs["tr_ms"] / 1e3, clk_s, BYTES_TR["s"] * N_HALF_S),
                       "fp32_model_frac": vs / D.world / min(roof32, roof64, roofhbm),
                       "fp32_model_svds_per_s": {"fp32_pipe": roof32, "fp64_pipe": roof64, "hbm": roofhbm}}
    if not a.no_ncr:
        out["ncr"] = ncr_leg(a.steps, a.warmup, dev, D, rates, clk_mhz, oc, value, out.get("fp32"))
    if not a.no_fwd_bwd:
        out["fwd_bwd"] = fwd_bwd_leg(a.steps, a.warmup, dev, D, rates, clk_mhz)
    if not a.no_phases:
        out["phases"] = phases_leg(a.steps, a.warmup, dev, D, rates, clk_mhz, oc)
    if not a.no_complex:
        out["complex"] = complex_leg(a.steps, a.warmup, dev, D, rates, clk_mhz, oc)
    # the n x n legs: the batched Kogbetliantz workload first, so that the driver's block
    # sizes (tuned on a device's first call, per order bucket) are picked on its matrices
    if not a.no_kog:
        out["kogbet"] = kog_leg(max(2, a.steps // 3), 1, dev, D, rates)
    if not a.no_kog_grad:
        out["kogbet_grad"] = kog_grad_leg(max(2, a.steps // 5), 1, dev, D)
    if not a.no_rect:
        out["rect"] = rect_leg(max(1, a.steps // 5), 1, dev, D, rates, clk_mhz)
    if not a.no_narrow:
        out["narrow"] = narrow_leg(a.steps, a.warmup, dev, D)
    if D.rank == 0 and D.world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    D.close()
    if D.rank == 0:
        print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------------
# reference arm: the oracle (the paper has no code; its CPU restatement is the reference)
# ----------------------------------------------------------------------------------------
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    from paper_2407_13116_gb300 import inputs as I
    cores = os.cpu_count() or 1
    m = 1 << 17
    Gs = I.general(m, SEED + 2, "d", "wide")
    Ts = I.triangular(m, SEED + 3, "d", "wide")

    def step():
        oracle.gesvd2(Gs, "d", nthreads=cores)
        oracle.trsvd2(Ts[0], Ts[1], Ts[2], "d", nthreads=cores)

    for _ in range(a.warmup):
        step()
    ts = []
    for _ in range(a.steps):
        t = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t)
    el = statistics.mean(ts)
    value = 2 * m / el
    sample = ("first %d general + %d triangular matrices of the wide-range FP64 workload per step, by the "
              "oracle (plain C, OpenMP over matrices on the host cores)" % (m, m))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "SVDs/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": el * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": headline_config(),
           "cpu_baseline": {"value": value, "unit": "SVDs/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "SVDs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def profile_case(a):
    """A few launches of each kernel on a small case of its benchmark workload, for ncu
    captures: the 2x2 kernels on 2^22 wide-range matrices (d, s; dn, sn: the variant with the
    hypot that is not correctly rounded; 470 MB of inputs and outputs in double, above L2),
    the complex kernel (z), lasv2 and the adjoint (misc: 2^22 matrices each), or one
    persistent Kogbetliantz run over 608 FP64 matrices of the batched workload's order mix
    (kog: one launch per order bucket; prints the rotation operations 8 n^3 per sweep, the
    unit of its ceiling)."""
    import numpy as np
    import torch
    from paper_2407_13116_gb300 import inputs as I
    from paper_2407_13116_gb300 import k2svd
    dev = torch.device("cuda", 0)
    n = a.profile_n
    if a.profile_case == "z":
        G = torch.empty((8, n), dtype=torch.float64, device=dev)
        G[0::2] = I.general(n, SEED + 6, "d", "wide", xp="torch", device=dev)
        G[1::2] = I.general(n, SEED + 7, "d", "wide", xp="torch", device=dev)
        torch.cuda.synchronize()
        for _ in range(3):
            k2svd.cgesvd2(G, want_info=False)
        torch.cuda.synchronize()
        print("profile case z n=%d done" % n)
        return
    if a.profile_case == "misc":
        T3 = I.triangular(n, SEED + 3, "d", "wide", xp="torch", device=dev)
        R, _, _ = I.rotated(n, SEED + 3)
        G = torch.from_numpy(R).to(dev)
        U, V, S, _, _, _ = k2svd.gesvd2(G, want_info=False)
        gen = torch.Generator(device=dev).manual_seed(SEED + 3)
        dS = torch.randn((2, n), dtype=torch.float64, device=dev, generator=gen)
        dU = torch.randn((4, n), dtype=torch.float64, device=dev, generator=gen)
        dV = torch.randn((4, n), dtype=torch.float64, device=dev, generator=gen)
        torch.cuda.synchronize()
        for _ in range(3):
            k2svd.lasv2(T3[0], T3[1], T3[2])
            k2svd.gesvd2_bwd(U, S, V, dS, dU, dV)
        torch.cuda.synchronize()
        print("profile case misc n=%d done" % n)
        return
    if a.profile_case in ("kog", "kog128"):
        orders = I.kog_orders(608, 8, 128, SEED + 4) if a.profile_case == "kog" else np.full(304, 128, np.int32)
        flat, _ = I.kog_batch(orders, SEED + 4)
        A = torch.from_numpy(flat).to(dev)
        U, S, V, sw, info = k2svd.kogbet(A, orders, flags=k2svd.KOG_NOTUNE)
        torch.cuda.synchronize()
        swn = sw.cpu().numpy().astype(np.int64)
        rot = float((swn * 8 * orders.astype(np.int64) ** 3).sum())
        print("profile case kog: %d matrices, mean sweeps %.2f, converged %d, rotation operations %.6g" %
              (len(orders), swn.mean(), int((info == 0).sum().item()), rot))
        return
    prec, ncr = a.profile_case[0], a.profile_case.endswith("n")
    G = I.general(n, SEED + 2, prec, "wide", xp="torch", device=dev)
    T3 = I.triangular(n, SEED + 3, prec, "wide", xp="torch", device=dev)
    torch.cuda.synchronize()
    for _ in range(3):
        k2svd.gesvd2(G, want_info=False, ncr=ncr)
        k2svd.trsvd2(T3[0], T3[1], T3[2], want_info=False, ncr=ncr)
    torch.cuda.synchronize()
    print("profile case %s n=%d done" % (a.profile_case, n))


def main():
    a = parse()
    if a.summarize_ncu:
        summarize_ncu(a.summarize_ncu, a.units)
        return
    if a.profile_case:
        profile_case(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
