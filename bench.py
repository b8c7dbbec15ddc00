"""Benchmark of the circuit-cutting hot path on one GB300 (or N replicas).

One step = one pass over every stage of the path for one synthetic circuit:
  T_pre    host preprocessing (Algorithm 1) + upload of the plan tables
  T_sub    subcircuit simulation of all 2^{c_i} variants (Algorithm 2)
  T_merge  full-state reconstruction of the 2^q vector (Algorithm 3)
  T_orig   uncut simulation of the same circuit (pass planning + HBM passes)
  verify   FP64 device reductions between the cut and uncut states
The reported value is T_cut = T_pre + T_sub + T_merge in seconds (Eq. 3),
the workload q = 30 random U3+CZ brickwork, depth 16, two 15-qubit segments,
c_total = 6 cuts, complex64.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch under torch.distributed.run; each rank runs an independent
replica (its own seed) and the slowest rank's time is reported.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "q=30 cut-sim wall s (per stage) & merge GB/s vs HBM peak; cut vs uncut, 1 GB300"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--q", type=int, default=30)
    p.add_argument("--depth", type=int, default=16)
    p.add_argument("--n", type=int, default=2)
    p.add_argument("--ctotal", type=int, default=6)
    p.add_argument("--prec", choices=["c64", "c128"], default="c64")
    p.add_argument("--decomp", choices=["projector", "s_sdg"], default="projector")
    p.add_argument("--merge-form", default="auto", choices=["auto", "fma", "tf32x3", "bf16x3", "f16x3", "ozaki"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--sweep", choices=["boundary", "batch", "paper", "planner"], default=None,
                   help="run a measurement sweep instead of the single-line benchmark")
    p.add_argument("--planner-instances", type=int, default=4000,
                   help="timed instances of the planner sweep")
    p.add_argument("--sweep-cmax", type=int, default=20,
                   help="largest c_total of the boundary sweep (capped by the depth)")
    p.add_argument("--sweep-both", action="store_true",
                   help="sweep complex64 and complex128")
    p.add_argument("--oracle-timing", default=None, help=argparse.SUPPRESS)
    return p.parse_args(argv)


def workload_config(a):
    import workload as w

    segs = w.equal_partition(a.q, a.n)
    cpb = w.split_cuts(a.ctotal, a.n)
    return segs, cpb, {
        "workload": (f"random U3+CZ brickwork q={a.q} depth={a.depth}, n={a.n} equal segments "
                     f"{'/'.join(map(str, segs))}, c_total={a.ctotal}, {a.prec}, {a.decomp} split"),
        "q": a.q, "depth": a.depth, "n_seg": a.n, "seg_qubits": segs, "c_total": a.ctotal,
        "cuts_per_boundary": cpb, "precision": a.prec, "decomp": a.decomp,
        "merge_form": a.merge_form, "seed": a.seed,
    }


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", FALLBACK_BF16_TFLOPS)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"


def fp32_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2603_01443_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (no measured figure; nominal)

# FP32-pipe instructions per amplitude for each operation the pass kernels
# execute on every amplitude of the vector, by gate arithmetic: a dense 2x2
# (one complex row: a product and three multiply-adds per real), a
# tangent-form rotation (one multiply-add per real) and a complex product (a
# phase block's or a table term's factor: two products, two multiply-adds).
# Double-float: y + t x costs 15 FP32 instructions (TwoProduct 2, TwoSum 6,
# cross terms and low sums 4, Fast2Sum 3), a product 7, so a rotation costs
# 2 x 15, a complex product 2 x 15 + 2 x 7, a dense row 2 x (3 x 15 + 7).
PASS_INST = {"f32": {"dense": 8, "rot": 2, "cmul": 4},
             "dfl": {"dense": 2 * (3 * 15 + 7), "rot": 2 * 15, "cmul": 2 * 15 + 2 * 7}}
# the same operations in flops of their own precision (a multiply-add counts 2)
PASS_FLOPS = {"dense": 14, "rot": 4, "cmul": 6}


def program_ops(words):
    """Per-amplitude operation counts of a gate program (its image as
    cc_program_image lays it out): every op of every stage of every pass is
    applied once to each of the program's 2^nq amplitudes."""
    wd = [int(x) for x in words]
    nq, n_pass, n_stage, n_op = wd[1], wd[3], wd[4], wd[5]
    i = 9 + 74 * n_pass + 10 * n_stage  # header, passes, stages
    c = {"dense": 0, "rot": 0, "cmul": 0, "nq": nq}
    for _ in range(n_op):
        typ, n_phase, n_table = wd[i], wd[i + 4], wd[i + 5]
        i += 8
        if typ == 0:
            c["dense"] += 1
        elif typ in (2, 3):
            c["rot"] += 1
        elif typ == 4:  # packed rotations: one per register bit of the mask
            c["rot"] += bin(wd[i - 7] & 0xFF).count("1")
        c["cmul"] += (1 if n_phase else 0) + n_table
    return c


def executed_work(counts, arith):
    """(FP32-pipe instructions, flops) of a program over its whole vector."""
    n = float(1 << counts["nq"])
    inst = sum(PASS_INST[arith][k] * counts[k] for k in PASS_FLOPS) * n
    flops = sum(PASS_FLOPS[k] * counts[k] for k in PASS_FLOPS) * n
    return inst, flops


def gate_arith(prec):
    """The gate-pass arithmetic the library picks for a precision."""
    if prec == "c64":
        return "f32"
    return "f64" if os.environ.get("CUTSIM_C128_GATES") == "fp64" else "dfl"


def fp32_inst_rate(sm_mhz=2070.0, sms=152):
    """FP32 instructions per second: SMs x 128 lanes x clock."""
    return sms * 128 * sm_mhz * 1e6


def traffic_key(kernel, a):
    return f"{kernel}@q{a.q}_d{a.depth}_n{a.n}_c{a.ctotal}_{a.prec}"


def recorded_traffic(kernel, a):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source and this workload (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)[traffic_key(kernel, a)]
    except Exception:
        return None
    try:
        if d.get("source_hash") != kernel_source_hash(d["sources"]):
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.summarize(out)

    @staticmethod
    def summarize(out):
        """Median SM clock, the maximum clock and every throttle reason seen
        Active, from nvidia-smi's CSV lines in FIELDS order (None if none)."""
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "samples": len(mhz),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU oracle
# The FP64 oracle timed on the host cores, in a separate interpreter that
# never touches the GPU, over a pool of spawned worker processes (one per
# usable core, numpy single-threaded in each):
#   Algorithm 1 in full (sequential, as written);
#   Algorithm 2 in full: every subcircuit, spread over the pool, its state
#     written into one shared-memory block;
#   Algorithm 3 on a sample of contiguous slabs of the output, each slab one
#     full row of the lowest segment (2^{q_0} amplitudes, the oracle's
#     per-amplitude form of the sum), the slabs spread evenly over the 2^q
#     output and over the pool; every slab is the same work, so the wall time
#     scales to the whole output by the number of slabs.  The estimate is
#     taken at S and at 2S slabs to show that it has converged.
# The pool also evaluates the oracle's amplitudes at the 4096 seeded indices
# of the GPU parity check (outside every timed region).

_OW = {}


def _ow_init(root, spec, shm_name, offsets, shapes):
    import sys as _sys

    if root not in _sys.path:
        _sys.path.insert(0, root)
    import numpy as np
    from multiprocessing import shared_memory

    import workload as w
    from oracle import cutting as ct

    segs = w.equal_partition(spec["q"], spec["n"])
    gates = w.brickwork_cut(spec["q"], spec["depth"], spec["seed"], segs,
                            w.split_cuts(spec["ctotal"], spec["n"]))
    _OW["pre"] = ct.preprocess(spec["q"], gates, segs, spec["decomp"])
    shm = shared_memory.SharedMemory(name=shm_name)
    _OW["shm"] = shm
    buf = np.ndarray((sum(int(np.prod(s)) for s in shapes),), dtype=np.complex128, buffer=shm.buf)
    _OW["states"] = [[buf[o:o + shapes[i][1]] for o in offs] for i, offs in enumerate(offsets)]


def _ow_ping(_):
    return os.getpid()


def _ow_sub(job):
    from oracle import statevector as sv

    i, r = job
    pre = _OW["pre"]
    _OW["states"][i][r][:] = sv.simulate_ops(pre.seg_sizes[i], pre.subcircuits[i][r])
    return job


def _ow_slab(x0):
    import numpy as np

    from oracle import cutting as ct

    pre = _OW["pre"]
    L = 1 << pre.seg_sizes[0]
    ct.amplitudes(pre, _OW["states"], np.arange(x0, x0 + L, dtype=np.int64))
    return x0


def _ow_sample(xs):
    from oracle import cutting as ct

    out = ct.amplitudes(_OW["pre"], _OW["states"], xs)
    return [[float(v.real), float(v.imag)] for v in out]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_timing_main(spec):
    """Entry of the CPU oracle timing interpreter (see above); prints one JSON line."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np

    import workload as w
    from oracle import cutting as ct

    q, n = spec["q"], spec["n"]
    segs = w.equal_partition(q, n)
    gates = w.brickwork_cut(q, spec["depth"], spec["seed"], segs, w.split_cuts(spec["ctotal"], n))
    t0 = time.perf_counter()
    pre = ct.preprocess(q, gates, segs, spec["decomp"])
    t_pre = time.perf_counter() - t0

    shapes = [(len(pre.subcircuits[i]), 1 << segs[i]) for i in range(n)]
    offsets, off = [], 0
    for nv, size in shapes:
        offsets.append([off + r * size for r in range(nv)])
        off += nv * size
    shm = shared_memory.SharedMemory(create=True, size=max(16, off * 16))
    cores = spec.get("cores") or host_cores()
    ctx = mp.get_context("spawn")
    res = {}
    try:
        with ctx.Pool(cores, initializer=_ow_init,
                      initargs=(ROOT, spec, shm.name, offsets, shapes)) as pool:
            pool.map(_ow_ping, range(4 * cores), chunksize=1)  # every worker up before timing
            jobs = [(i, r) for i in range(n) for r in range(shapes[i][0])]
            t0 = time.perf_counter()
            pool.map(_ow_sub, jobs, chunksize=1)
            t_sub = time.perf_counter() - t0
            L = 1 << segs[0]
            n_slabs_total = (1 << q) // L
            # an untimed pass first maps every worker's view of the shared
            # subcircuit vectors; chunks of a few slabs keep the tail of each
            # pass (workers idle while the last chunks finish) short
            pool.map(_ow_slab, [j * L for j in range(min(n_slabs_total, 4 * cores))], chunksize=1)
            # each sample is timed in `reps` passes over different slabs
            # (every pass and sample at its own offset inside the stride), the
            # passes of the samples interleaved so that all samples see the
            # same load on a shared host, and the median pass taken: one pass
            # of a second or so varies by 10-20 % from one second to the next
            reps = int(spec.get("reps", 3))
            sizes = [min(S, n_slabs_total) for S in spec["slabs"]]
            n_pass = reps * len(sizes)
            passes = [[] for _ in sizes]
            for r in range(reps):
                for si, S in enumerate(sizes):
                    stride = n_slabs_total // S
                    shift = (stride * (si * reps + r)) // n_pass
                    x0s = [(j * stride + shift) * L for j in range(S)]
                    t0 = time.perf_counter()
                    pool.map(_ow_slab, x0s, chunksize=max(1, S // (16 * cores)))
                    passes[si].append(time.perf_counter() - t0)
            est = []
            for S, ps in zip(sizes, passes):
                t_s = statistics.median(ps)
                est.append({"slabs": S, "slab_amplitudes": L, "seconds": t_s, "passes_s": ps,
                            "t_merge": t_s * n_slabs_total / S})
            if spec.get("sample_seed") is not None:
                xs = w.sample_indices(q, 4096, spec["sample_seed"])
                chunks = [xs[k:k + 256] for k in range(0, len(xs), 256)]
                amps = [v for part in pool.map(_ow_sample, chunks) for v in part]
                res["sample_amplitudes"] = amps
                res["sample_seed"] = spec["sample_seed"]
    finally:
        shm.close()
        shm.unlink()
    res.update({"t_pre": t_pre, "t_sub": t_sub, "merge_estimates": est, "cores": cores,
                "n_sub": sum(s[0] for s in shapes)})
    print(json.dumps(res))
    return 0


def run_oracle_timing(a, slabs, sample_seed=None, timeout=900):
    """The CPU oracle timing interpreter for workload a; its JSON result or {"error": ...}."""
    spec = {"q": a.q, "depth": a.depth, "n": a.n, "ctotal": a.ctotal, "seed": a.seed,
            "decomp": a.decomp, "slabs": list(slabs), "sample_seed": sample_seed}
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-timing",
                        json.dumps(spec)], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        tail = r.stderr.strip().splitlines()
        return {"error": tail[-1] if tail else "failed"}
    return json.loads(r.stdout.strip().splitlines()[-1])


# Slabs of the Algorithm 3 sample: the estimate from BASE_SLABS is the value;
# the cpu_baseline leg also measures 2 x BASE_SLABS as the convergence check.
BASE_SLABS = 1024


def cpu_value(d, a, which=0):
    t_merge = d["merge_estimates"][which]["t_merge"]
    return d["t_pre"] + d["t_sub"] + t_merge


def cpu_record(d, a):
    e0 = d["merge_estimates"][0]
    rec = {
        "value": cpu_value(d, a, 0), "unit": "s", "cores": d["cores"], "kind": "oracle",
        "sample": (f"Algorithm 1 in full; Algorithm 2 in full ({d['n_sub']} subcircuits over "
                   f"{d['cores']} worker processes); the Algorithm 3 sum (per-amplitude form) on "
                   f"{e0['slabs']} contiguous slabs of {e0['slab_amplitudes']} amplitudes spread "
                   f"evenly over the 2^{a.q} output, scaled by the slab count (median of "
                   f"{len(e0.get('passes_s', [0]))} passes over different slabs)"),
        "sample_seconds": d["t_pre"] + d["t_sub"] + e0["seconds"],
        "stages": {"pre_s": d["t_pre"], "sub_s": d["t_sub"], "merge_s": e0["t_merge"]},
    }
    if len(d["merge_estimates"]) > 1:
        e1 = d["merge_estimates"][1]
        rec["convergence"] = {"slabs": [e0["slabs"], e1["slabs"]],
                              "t_merge_s": [e0["t_merge"], e1["t_merge"]],
                              "ratio": e1["t_merge"] / e0["t_merge"]}
    return rec


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings across the process group (the
    slowest replica sets the job's time); identity for a single process."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    segs, cpb, cfg = workload_config(a)
    vals, secs = [], []
    last = None
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        d = run_oracle_timing(a, [BASE_SLABS])
        if "error" in d:
            print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + d["error"]}))
            return 0
        if i >= a.warmup:
            vals.append(cpu_value(d, a))
            secs.append(time.perf_counter() - t0)
            last = d
    value = statistics.mean(vals)
    cpu = cpu_record(last, a)
    cpu["value"] = value
    out = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * statistics.mean(secs), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg, "impl": "reference", "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def sweep_boundary(a):
    """Speedup-boundary sweep (the paper's Sec. V.B experiment on this GPU):
    q in {16, 20, 24}, depth in {8, 16, 32}, n = 2 equal segments, c_total
    from 0 to min(--sweep-cmax, depth), stopping two points after the cut form
    stops winning; per point the stage times and
    Delta = (T_cut - T_orig) / T_orig.  One JSON line per point, then a
    summary with the largest c_total that still gives Delta < 0 per (q, depth)
    next to Eq. 13's c_total < q / 2."""
    import torch

    import workload as w
    from paper_2603_01443_gb300 import api, capi

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    summary = {}
    precs = ["c64", "c128"] if a.prec == "c64" and a.sweep_both else [a.prec]
    for prec in precs:
        for q in (16, 20, 24):
            for depth in (8, 16, 32):
                best = None
                above = 0
                for c in range(0, min(a.sweep_cmax, depth) + 1):
                    if above >= 2:  # past the crossover: the merge only grows from here
                        break
                    if q - q // 2 + c > 28:  # keep each segment block within 2^28 amplitudes
                        break
                    gates = w.brickwork_cut(q, depth, a.seed, [q // 2, q - q // 2], c)
                    packed = capi.GateArray(gates)
                    probe = api.CutPlan(packed, q, [q // 2, q - q // 2], a.decomp, prec)
                    seg, psi, ws = probe.alloc_seg_buf(), probe.alloc_psi(), probe.alloc_workspace()
                    probe.close()
                    psi_u = torch.empty_like(psi)
                    rec = []
                    for rep in range(1 + 3):
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        plan = api.CutPlan(packed, q, [q // 2, q - q // 2], a.decomp, prec)
                        t_pre = time.perf_counter() - t0
                        ev[0].record(stream)
                        plan.simulate_segments(seg, stream)
                        ev[1].record(stream)
                        plan.merge(seg, psi, ws, "auto", stream)
                        ev[2].record(stream)
                        ev[2].synchronize()  # keep the merge out of the uncut plan's time
                        t1 = time.perf_counter()
                        up = api.UncutPlan(packed, q, prec)
                        t_up = time.perf_counter() - t1
                        ev[3].record(stream)
                        up.simulate(psi_u, stream)
                        end = torch.cuda.Event(enable_timing=True)
                        end.record(stream)
                        end.synchronize()
                        if rep:
                            rec.append((t_pre, ev[0].elapsed_time(ev[1]) / 1e3,
                                        ev[1].elapsed_time(ev[2]) / 1e3,
                                        t_up + ev[3].elapsed_time(end) / 1e3))
                        plan.close()
                        up.close()
                    pre, sub, mer, orig = (statistics.mean(x) for x in zip(*rec))
                    cut = pre + sub + mer
                    delta = (cut - orig) / orig
                    print(json.dumps({"sweep": "boundary", "precision": prec, "q": q,
                                      "depth": depth, "c_total": c, "pre_s": pre, "sub_s": sub,
                                      "merge_s": mer, "cut_s": cut, "orig_s": orig,
                                      "delta": delta}), flush=True)
                    if delta < 0:
                        best = c
                        above = 0
                    else:
                        above += 1
                    del seg, psi, ws, psi_u
                summary.setdefault(prec, {}).setdefault(str(q), {})[str(depth)] = best
    print(json.dumps({"sweep": "boundary", "largest_c_total_with_speedup": summary,
                      "eq13_threshold": {str(q): q / 2 for q in (16, 20, 24)}}))
    return 0


def measure_point(gates, q, segs, prec, decomp, reps=3, warmup=True, form="auto", tile_bits=None):
    """Mean (T_pre, T_sub, T_merge, T_orig) of one circuit over `reps` runs
    after one warm-up (unless warmup=False); buffers allocated outside the
    timing."""
    import torch

    from paper_2603_01443_gb300 import api, capi

    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    packed = capi.GateArray(gates)
    saved_tile = os.environ.get("CUTSIM_SEG_TILE_BITS")
    if tile_bits is not None:  # the library reads the segment tile width per plan
        os.environ["CUTSIM_SEG_TILE_BITS"] = str(tile_bits)
    probe = api.CutPlan(packed, q, segs, decomp, prec)
    seg, psi, ws = probe.alloc_seg_buf(), probe.alloc_psi(), probe.alloc_workspace()
    probe.close()
    psi_u = torch.empty_like(psi)
    rec = []
    first = 1 if warmup else 0
    for rep in range(first + reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = api.CutPlan(packed, q, segs, decomp, prec)
        t_pre = time.perf_counter() - t0
        ev[0].record(stream)
        plan.simulate_segments(seg, stream)
        ev[1].record(stream)
        plan.merge(seg, psi, ws, form, stream)
        ev[2].record(stream)
        ev[2].synchronize()
        t1 = time.perf_counter()
        up = api.UncutPlan(packed, q, prec)
        t_up = time.perf_counter() - t1
        ev[3].record(stream)
        up.simulate(psi_u, stream)
        ev[4].record(stream)
        ev[4].synchronize()
        if rep >= first:
            rec.append((t_pre, ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3,
                        t_up + ev[3].elapsed_time(ev[4]) / 1e3))
        plan.close()
        up.close()
    capi.check(capi.lib().cc_sync(stream.cuda_stream), "cc_sync")
    if tile_bits is not None:
        if saved_tile is None:
            os.environ.pop("CUTSIM_SEG_TILE_BITS", None)
        else:
            os.environ["CUTSIM_SEG_TILE_BITS"] = saved_tile
    return tuple(statistics.mean(x) for x in zip(*rec))


def fit_boundary(points, iters=4000, lr=0.05):
    """Linear boundary c = slope * q + intercept between the speedup (Delta < 0)
    and slowdown points of a (q, c_total) grid: a class-balanced linear
    soft-margin SVM (hinge loss, L2 penalty) fitted by subgradient descent on
    standardised features, as the paper fits its measured boundary with a
    weighted SVM.  Only the q that have points of both classes take part: a
    q where no c_total gives a speedup (on this GPU the smallest circuits,
    whose every stage is a few launch-bound microseconds) has no boundary
    to fit.  And at each q only the c_total from its smallest speedup point
    up: the staircase's uncut time grows with its c_total gate blocks, so
    the fewest cuts can lose too, and a line cannot separate that band's
    lower edge together with the upper one the method's threshold is about.
    Returns None when one class is empty."""
    import numpy as np

    lo = {}
    for q, c, d in points:
        if d <= 0:
            lo[q] = min(lo.get(q, c), c)
    both = set(lo) & {p[0] for p in points if p[2] > 0}
    points = [p for p in points if p[0] in both and p[1] >= lo[p[0]]]
    if not points:
        return None
    X = np.array([[p[0], p[1]] for p in points], dtype=float)
    y = np.array([1.0 if p[2] > 0 else -1.0 for p in points])
    if (y > 0).all() or (y < 0).all():
        return None
    mu, sd = X.mean(0), X.std(0) + 1e-12
    Z = (X - mu) / sd
    wts = np.where(y > 0, 0.5 / (y > 0).mean(), 0.5 / (y < 0).mean())
    w = np.zeros(2)
    b = 0.0
    lam = 1e-3
    for t in range(iters):
        m = y * (Z @ w + b)
        act = m < 1
        gw = lam * w - (wts[act, None] * y[act, None] * Z[act]).sum(0) / len(y)
        gb = -(wts[act] * y[act]).sum() / len(y)
        step = lr / (1 + t / 500)
        w -= step * gw
        b -= step * gb
    # back to (q, c): w0 (q - mu0)/sd0 + w1 (c - mu1)/sd1 + b = 0
    a0, a1 = w[0] / sd[0], w[1] / sd[1]
    c0 = b - a0 * mu[0] - a1 * mu[1]
    if abs(a1) < 1e-12:
        return None
    return {"slope": float(-a0 / a1), "intercept": float(-c0 / a1)}


def sweep_paper(a):
    """The paper's own workload on this GPU (Sec. V.B, V.C): the H/T/CX
    staircase (Fig. 1; c_total = blocks x (n - 1)), equal partitions, the
    Delta grids of Fig. 4 -- n = 2: q = 2..24 step 2 (extended to 28),
    c_total = 1..10; n = 3: q = 3..24 step 3 (extended to 27), c_total =
    2..14 step 2 -- each q continued past the grid's last c_total while
    cutting still wins (up to c_total 18 / 24 and 32 GiB of segment
    buffers), so the boundary lies inside the measured points; then a fitted
    linear boundary next to the paper's fits (0.70 q - 7.30, 1.00 q - 11.50)
    and Eqs. 13-14, and the largest c_total with a speedup per q; then the depth sweep
    (10^p T/X layers on the edge qubits, p = 0, 2, 3, 4) at n = 2."""
    import math

    import torch

    import workload as w

    torch.cuda.set_device(0)
    prec = a.prec
    fits = {}
    grids = {2: ([*range(2, 25, 2), 26, 28], list(range(1, 11))),
             3: ([*range(3, 25, 3), 27], list(range(2, 15, 2)))}
    cap_c = {2: 18, 3: 24}
    amp_bytes = 16 if prec == "c128" else 8
    largest = {}
    for n, (qs, cs) in grids.items():
        pts = []
        step = cs[1] - cs[0]
        largest[f"n{n}"] = {}
        for q in qs:
            segs = w.equal_partition(q, n)
            c, last = cs[0], None
            while True:
                if c > cs[-1]:  # past the grid: only while cutting still wins
                    seg_amps = sum(1 << (s + c // (n - 1) * (2 if 0 < i < n - 1 else 1))
                                   for i, s in enumerate(segs))
                    if last is None or last >= 0 or c > cap_c[n] or \
                            seg_amps * amp_bytes > 32 << 30:
                        break
                blocks = c // (n - 1)
                gates = w.staircase(q, blocks)
                pre, sub, mer, orig = measure_point(gates, q, segs, prec, a.decomp)
                cut = pre + sub + mer
                delta = (cut - orig) / orig
                pts.append((q, c, delta))
                if delta < 0:
                    largest[f"n{n}"][q] = c
                print(json.dumps({"sweep": "paper", "family": "staircase", "precision": prec,
                                  "n": n, "q": q, "c_total": c, "pre_s": pre, "sub_s": sub,
                                  "merge_s": mer, "cut_s": cut, "orig_s": orig, "delta": delta}),
                      flush=True)
                last = delta
                c += step
        fits[f"n{n}"] = fit_boundary(pts)
    depth = {}
    for pexp in (0, 2, 3, 4):
        pts = []
        for q in range(4, 25, 4):
            for c in range(1, 11):
                gates = w.staircase_depth(q, c, pexp)
                pre, sub, mer, orig = measure_point(gates, q, w.equal_partition(q, 2), prec,
                                                    a.decomp, reps=2)
                cut = pre + sub + mer
                delta = (cut - orig) / orig
                pts.append((q, c, delta))
                print(json.dumps({"sweep": "paper", "family": "staircase_depth", "p": pexp,
                                  "precision": prec, "n": 2, "q": q, "c_total": c,
                                  "n_gates": len(gates), "pre_s": pre, "sub_s": sub,
                                  "merge_s": mer, "cut_s": cut, "orig_s": orig,
                                  "delta": delta}), flush=True)
        depth[f"p{pexp}"] = fit_boundary(pts)
    print(json.dumps({"sweep": "paper", "precision": prec, "fit": fits, "depth_fit": depth,
                      "largest_c_total_with_speedup": largest,
                      "paper_fit": {"n2": {"slope": 0.70, "intercept": -7.30},
                                    "n3": {"slope": 1.00, "intercept": -11.50}},
                      "theory": {"n2": {"slope": 0.5, "intercept": 0.0},
                                 "n3": {"slope": 2.0 / 3.0, "intercept": math.log2(3)}}}))
    return 0


def planner_instance_features(q, depth, segs, cpb, gates, tile_bits=13, form="fma"):
    from paper_2603_01443_gb300 import planner as pl

    n = len(segs)
    seg_c = [(cpb[i - 1] if i > 0 else 0) + (cpb[i] if i < n - 1 else 0) for i in range(n)]
    n_sub = sum(1 << c for c in seg_c)
    max_seg_bits = max(s + c for s, c in zip(segs, seg_c))
    dense = sum(1 for g in gates if g.kind in ("U3", "H", "X"))
    two = sum(1 for g in gates if g.q1 >= 0)
    return pl.features(q, depth, n, sum(cpb), n_sub, max_seg_bits, dense, two, tile_bits,
                       form), seg_c


def merge_forms(prec):
    """The merge forms a plan of this precision can run (AUTO aside)."""
    return ("fma", "tf32x3", "f16x3", "bf16x3") if prec == "c64" else ("fma", "ozaki")


def resolved_form(form, prec, k_last, qa, qb):
    """The form a merge request runs: a tensor-core form needs both factors
    of >= 2^7 amplitudes (the library then merges on CUDA cores)."""
    if form in ("tf32x3", "f16x3", "bf16x3", "ozaki") and (qa < 7 or qb < 7):
        return "fma"
    return form


def sweep_planner(a, n_inst=4000):
    """Learned planner: time n_inst random brickwork instances (q 14..30,
    depth 4..64, n in {2, 3, 4} equal segments, c_total 0..16, each with a
    random segment tile width of 2^11..2^13 amplitudes and a random merge form
    the plan can run) stage by stage on this GPU, train an ensemble of FP32
    networks (3 hidden layers of 64, hand-written CUDA kernels) on an 80/20
    split to predict log10 stage seconds, and report the prediction error on
    the held-out 20 %, the cut/no-cut decisions of the model, of the
    closed-form threshold and of the model with its fallback (held-out error
    near the query above 20 %), the choice of n, merge form and tile width on
    separate circuit families against the measured best, and the largest q
    that fits a 10-minute budget with and without cutting.  Instances whose
    segment buffers would exceed 2^31 amplitudes or whose merge would exceed
    2^39 amplitude-terms are redrawn (their cost is out of proportion to what
    they teach)."""
    import numpy as np

    import torch

    import workload as w
    from paper_2603_01443_gb300 import planner as pl

    torch.cuda.set_device(0)
    rng = np.random.default_rng(a.seed + 4242)
    forms = merge_forms(a.prec)
    tiles = (11, 12, 13)
    measure_point(w.brickwork_cut(16, 4, 0, [8, 8], 1), 16, [8, 8], a.prec, a.decomp, reps=1)
    X, Y, meta = [], [], []
    t0 = time.perf_counter()
    while len(X) < n_inst:
        q = int(rng.integers(14, 31))
        depth = int(rng.integers(4, 65))
        n = int(rng.integers(2, 5))
        c = int(rng.integers(0, min(16, depth * (n - 1)) + 1))
        segs = w.equal_partition(q, n)
        cpb = w.split_cuts(c, n)
        seg_c = [(cpb[i - 1] if i > 0 else 0) + (cpb[i] if i < n - 1 else 0) for i in range(n)]
        if sum(1 << (s_ + c_) for s_, c_ in zip(segs, seg_c)) > (1 << 31) or q + max(cpb) > 39:
            continue
        gates = w.brickwork_cut(q, depth, int(rng.integers(1 << 30)), segs, cpb)
        form = resolved_form(str(rng.choice(forms)), a.prec, 1 << cpb[-1], q - segs[-1], segs[-1])
        tile = int(rng.choice(tiles))
        pre, sub, mer, orig = measure_point(gates, q, segs, a.prec, a.decomp, reps=1,
                                            warmup=False, form=form, tile_bits=tile)
        f, _ = planner_instance_features(q, depth, segs, cpb, gates, tile, form)
        X.append(f)
        Y.append([pre, sub, mer, orig])
        meta.append((q, depth, n, c, pl.depth_ratio(gates, segs)))
    t_data = time.perf_counter() - t0
    X, Y = np.array(X), np.array(Y)
    perm = rng.permutation(len(X))
    n_tr = int(0.8 * len(X))
    tr, te = perm[:n_tr], perm[n_tr:]
    t1 = time.perf_counter()
    P = pl.StagePlanner(n_models=4, seed=a.seed)
    curves = P.fit(X[tr], Y[tr], epochs=3000, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    pr = P.predict(X[te])
    err = {}
    for i, s_ in enumerate(pl.STAGES):
        rel = np.abs(pr[s_] - Y[te, i]) / Y[te, i]
        err[s_] = {"median": float(np.median(rel)), "p90": float(np.percentile(rel, 90))}
    t_cut_meas = Y[te, 0] + Y[te, 1] + Y[te, 2]
    rel = np.abs(pr["cut"] - t_cut_meas) / t_cut_meas
    err["cut"] = {"median": float(np.median(rel)), "p90": float(np.percentile(rel, 90))}
    # fallback trigger: held-out error near each query, estimated without the
    # query itself (leave-one-out over the held-out set)
    half = len(te) // 2
    te_a, te_b = te[:half], te[half:]
    P.set_holdout(X[te_a], Y[te_a])
    exp_b = P.expected_error(X[te_b])
    truth = t_cut_meas[half:] < Y[te_b, 3]
    model = pr["cut"][half:] < pr["orig"][half:]
    closed = np.array([meta[k][3] < pl.threshold(meta[k][0], meta[k][2]) for k in te_b])
    closed15 = np.array([meta[k][3] < pl.nonuniform_threshold(meta[k][0], meta[k][2], meta[k][4])
                         for k in te_b])
    fb = exp_b > P.fallback_error
    combined = np.where(fb, closed15, model)
    decisions = {"test_instances": int(len(te_b)), "cut_wins_measured": float(truth.mean()),
                 "accuracy_model": float((model == truth).mean()),
                 "accuracy_closed_form_eq13_14": float((closed == truth).mean()),
                 "accuracy_closed_form_eq15": float((closed15 == truth).mean()),
                 "accuracy_model_with_fallback": float((combined == truth).mean()),
                 "fallback_rate": float(fb.mean()),
                 "fallback_trigger": "held-out T_cut/T_orig error of the 8 nearest held-out "
                                     "instances > 20 %"}
    print(json.dumps({"sweep": "planner", "part": "data", "instances": int(len(X)),
                      "data_s": t_data, "train_s": t_train, "precision": a.prec,
                      "forms": list(forms), "tile_bits": list(tiles),
                      "final_train_loss": [float(c_[-1]) for c_ in curves],
                      "features": list(pl.FEATURES), "stages": list(pl.STAGES)}), flush=True)
    print(json.dumps({"sweep": "planner", "part": "prediction_error_test", "error": err,
                      "decisions": decisions}), flush=True)
    P.set_holdout(X[te], Y[te])

    # choice of n, merge form and tile width on separate circuit families:
    # every option measured, the planner's choice against the measured best
    fam_rng = np.random.default_rng(a.seed + 77)
    n_fam = 32
    tols = [2e-6, 5e-5] if a.prec == "c64" else [1e-12]
    stats = {str(t): {"agree_n": 0, "agree_all": 0, "fallback": 0, "regret": []} for t in tols}
    rows = []
    for k in range(n_fam):
        q = int(fam_rng.integers(18, 31))
        depth = int(fam_rng.choice([8, 16, 32, 64]))
        cpb1 = int(fam_rng.integers(1, 6))
        seed = int(fam_rng.integers(1 << 30))
        opts, times = [], {}
        t_orig = None
        ratio = None
        for n in (2, 3, 4):
            segs = w.equal_partition(q, n)
            cpb = [cpb1] * (n - 1)
            gates = w.brickwork_cut(q, depth, seed, segs, cpb)
            ratio = pl.depth_ratio(gates, segs) if ratio is None else ratio
            done = set()
            for form in forms:
                rf = resolved_form(form, a.prec, 1 << cpb1, q - segs[-1], segs[-1])
                for tile in (12, 13):
                    if (rf, tile) in done:
                        continue
                    done.add((rf, tile))
                    pre, sub, mer, orig = measure_point(gates, q, segs, a.prec, a.decomp, reps=1,
                                                        form=rf, tile_bits=tile)
                    times[(n, rf, tile)] = pre + sub + mer
                    t_orig = orig if t_orig is None else min(t_orig, orig)
                    f, seg_c = planner_instance_features(q, depth, segs, cpb, gates, tile, rf)
                    opts.append({"n": n, "form": rf, "seg_tile_bits": tile, "features": f,
                                 "cut_bits": sum(cpb), "n_sub": sum(1 << c_ for c_ in seg_c)})
        row = {"q": q, "depth": depth, "c_per_boundary": cpb1, "uncut_s": t_orig,
               "measured_s": {f"{n}/{fm}/{tb}": t for (n, fm, tb), t in times.items()}}
        for tol in tols:
            adm = {key: t for key, t in times.items() if pl.FORM_TOL[key[1]] <= tol}
            best_key = min(adm, key=adm.get)
            best = (0, None, None) if t_orig < adm[best_key] else best_key
            best_t = min(t_orig, adm[best_key])
            d = P.decide(q, opts, tol=tol, dseg_over_d=ratio)
            if d["choice"] == 0:
                got_t = t_orig
            elif d["form"] in (None, "auto"):  # fallback: the library's AUTO form, default tile
                cands = [t for (n, fm, tb), t in adm.items() if n == d["choice"] and tb == 13]
                got_t = min(cands) if cands else t_orig
            else:
                got_t = times[(d["choice"], d["form"], d["seg_tile_bits"])]
            st_ = stats[str(tol)]
            st_["agree_n"] += int(d["choice"] == best[0])
            st_["agree_all"] += int((d["choice"], d["form"], d["seg_tile_bits"]) == best)
            st_["fallback"] += int(d["fallback"])
            st_["regret"].append(got_t / best_t - 1.0)
            row[f"tol {tol:g}"] = {"choice": [d["choice"], d["form"], d["seg_tile_bits"]],
                                   "best": list(best), "fallback": d["fallback"]}
        rows.append(row)
    summary = {t: {"agreement_n": v["agree_n"] / n_fam, "agreement_n_form_tile": v["agree_all"] / n_fam,
                   "fallback_rate": v["fallback"] / n_fam, "mean_regret": float(np.mean(v["regret"])),
                   "max_regret": float(np.max(v["regret"]))} for t, v in stats.items()}
    print(json.dumps({"sweep": "planner", "part": "choose_n_form_tile", "families": n_fam,
                      "options": "n in {2,3,4} x merge forms within the tolerance x tile 2^12, 2^13",
                      "summary_by_tolerance": summary, "rows": rows}), flush=True)

    # largest q within a 10-minute budget (brickwork depth 16, n = 2, c_total = 6)
    def predict(q, which):
        qq = min(q, 30)
        segs = w.equal_partition(qq, 2)
        gates = w.brickwork_cut(qq, 16, 0, segs, [6])
        form = "f16x3" if a.prec == "c64" else "ozaki"
        f, _ = planner_instance_features(qq, 16, segs, [6], gates, 13, form)
        p = P.predict(np.array([f]))
        t = float(p["cut"][0] if which == "cut" else p["orig"][0])
        return t * 2.0 ** (q - qq)  # state-vector work doubles per qubit beyond the data
    hbm = torch.cuda.get_device_properties(0).total_memory
    amp = 8 if a.prec == "c64" else 16
    q_mem = int(math.floor(math.log2(hbm * 0.9 / amp)))  # one 2^q vector (+ small segment buffers)
    res = {w_: pl.max_feasible_q(lambda q: predict(q, w_), 600.0, q_mem, 14) for w_ in ("cut", "orig")}
    print(json.dumps({"sweep": "planner", "part": "max_feasible_q", "budget_s": 600.0,
                      "workload": "brickwork depth 16, n = 2, c_total = 6",
                      "memory_cap_q": q_mem, "cut": res["cut"], "uncut": res["orig"],
                      "pred_s_at_cap": {"cut": predict(q_mem, "cut"),
                                        "uncut": predict(q_mem, "orig")}}), flush=True)
    return 0


def sweep_batch(a, n_circ=64):
    """Batched uneven workload: n_circ independent random brickwork circuits
    (q uniform in 16..26, depth in {8, 16, 32}, n in {2, 3} unequal segments,
    c_total 2..6).  All segment passes of all circuits run in one persistent
    launch and the merges in one launch per chain level, replayed from a CUDA
    graph after the autotuner picked the segment tile width and merge tile
    height.  Reported next to the plain form: the same circuits one after
    another through the one-circuit API (plans made beforehand, AUTO merge).
    Latency of circuit i in the batch = completion of its merge minus the
    start of the persistent launch (device %globaltimer)."""
    import numpy as np
    import torch

    import workload as w
    from paper_2603_01443_gb300 import api, capi

    torch.cuda.set_device(0)
    items = w.uneven_batch(n_circ, a.seed)
    circ = [(capi.GateArray(it.gates), it.q, it.seg_sizes) for it in items]
    t0 = time.perf_counter()
    b = api.Batch(circ, a.decomp, a.prec)
    t_plan = time.perf_counter() - t0
    seg, psi, ws = b.alloc_buffers()
    stamps = b.alloc_stamps()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, stream, reps):
        for _ in range(max(1, a.warmup)):
            fn()
        stream.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    cur = torch.cuda.current_stream()
    default_info = dict(b.info)
    t_default = timed(lambda: b.run(seg, psi, ws, None, cur), cur, a.steps)
    table = b.autotune(seg, psi, ws, cur)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    b.capture(seg, psi, ws, None, stream=s)
    t_batch = timed(lambda: b.launch(s), s, a.steps)
    # completion times: a replay of a second graph that stamps every circuit
    b.capture(seg, psi, ws, stamps, stream=s)
    b.launch(s)
    b.launch(s)
    s.synchronize()
    capi.check(capi.lib().cc_sync(s.cuda_stream), "cc_sync")
    st = stamps.cpu().numpy().view(np.uint64).astype(np.float64)
    lat = (st[1:] - st[0]) / 1e9

    # the plain form: one circuit at a time through the one-circuit API
    plans = [api.CutPlan(g, q, segs, a.decomp, a.prec) for g, q, segs in circ]
    bufs = [(p.alloc_seg_buf(), p.alloc_psi(), p.alloc_workspace()) for p in plans]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_circ + 1)]

    def sequential():
        evs[0].record(cur)
        for i, (p, (sg, ps, wk)) in enumerate(zip(plans, bufs)):
            p.simulate_segments(sg, cur)
            p.merge(sg, ps, wk, "auto", cur)
            evs[i + 1].record(cur)

    for _ in range(max(1, a.warmup)):
        sequential()
    torch.cuda.synchronize()
    seq_tot, seq_dur, seq_done = [], [], []
    for _ in range(a.steps):
        sequential()
        evs[-1].synchronize()
        seq_tot.append(evs[0].elapsed_time(evs[-1]) / 1e3)
        seq_dur.append([evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(n_circ)])
        seq_done.append([evs[0].elapsed_time(evs[i + 1]) / 1e3 for i in range(n_circ)])
    dur = np.mean(np.array(seq_dur), axis=0)
    done = np.mean(np.array(seq_done), axis=0)
    worst = 0.0
    for i, (_, (_, ps, _)) in enumerate(zip(plans, bufs)):
        r = api.compare(b.psi_view(psi, i), ps, a.prec)
        worst = max(worst, r["max_abs_diff"] / r["max_abs_b"])
    n_amp = sum(1 << it.q for it in items)
    t_seq = statistics.mean(seq_tot)
    print(json.dumps({
        "sweep": "batch", "n_circ": n_circ, "precision": a.prec, "decomp": a.decomp,
        "workload": "uneven_batch(64): q 16..26, depth {8,16,32}, n {2,3} unequal, c_total 2..6",
        "n_sub": b.info["n_sub"], "amplitudes": n_amp, "plan_s": t_plan,
        "default": {"tile_bits": default_info["tile_bits"], "merge_rows": default_info["merge_rows"],
                    "batch_s": t_default},
        "autotune": table, "chosen": {"tile_bits": b.info["tile_bits"],
                                      "merge_rows": b.info["merge_rows"]},
        "persistent_launch": {"grid": b.info["grid"], "block": b.info["block"],
                              "jobs": b.info["n_jobs"], "tiles": b.info["n_items"]},
        "batch_s": t_batch, "circuits_per_s": n_circ / t_batch,
        "output_gbs": n_amp * api.AMP_BYTES[a.prec] / t_batch / 1e9,
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "sequential": {"total_s": t_seq, "circuits_per_s": n_circ / t_seq,
                       "duration_p50_s": float(np.percentile(dur, 50)),
                       "duration_p99_s": float(np.percentile(dur, 99)),
                       "completion_p50_s": float(np.percentile(done, 50)),
                       "completion_p99_s": float(np.percentile(done, 99))},
        "speedup_vs_sequential": t_seq / t_batch,
        "max_rel_diff_vs_sequential": worst,
    }), flush=True)
    return 0


def main(argv=None):
    a = parse_args(argv)
    if a.oracle_timing is not None:
        return oracle_timing_main(json.loads(a.oracle_timing))
    if a.impl == "reference":
        return reference_arm(a)
    if a.sweep == "boundary":
        return sweep_boundary(a)
    if a.sweep == "batch":
        return sweep_batch(a)
    if a.sweep == "paper":
        return sweep_paper(a)
    if a.sweep == "planner":
        return sweep_planner(a, a.planner_instances)

    import torch
    import torch.distributed as dist

    import workload as w
    from paper_2603_01443_gb300 import api, capi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    segs, cpb, cfg = workload_config(a)
    seed = a.seed + rank
    gates = w.brickwork_cut(a.q, a.depth, seed, segs, cpb)
    stream = torch.cuda.current_stream()
    packed = capi.GateArray(gates)  # the circuit as the C ABI takes it, packed once

    probe = api.CutPlan(gates, a.q, segs, a.decomp, a.prec)
    assert probe.info["c_total"] == a.ctotal
    seg = probe.alloc_seg_buf(dev)
    psi = probe.alloc_psi(dev)
    ws = probe.alloc_workspace(dev)
    up_probe = api.UncutPlan(gates, a.q, a.prec)
    psi_u = up_probe.alloc_psi(dev)
    info = dict(probe.info)
    uinfo = dict(up_probe.info)
    probe.close()
    up_probe.close()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    rec = {"pre": [], "sub": [], "merge": [], "orig": [], "orig_host": [], "verify": [], "cmp": []}

    def step(record):
        t0 = time.perf_counter()
        plan = api.CutPlan(packed, a.q, segs, a.decomp, a.prec)
        t_pre = time.perf_counter() - t0
        ev[0].record(stream)
        plan.simulate_segments(seg, stream)
        ev[1].record(stream)
        plan.merge(seg, psi, ws, a.merge_form, stream)
        ev[2].record(stream)
        ev[2].synchronize()  # the uncut plan's table upload must not wait on the merge
        t1 = time.perf_counter()
        up = api.UncutPlan(packed, a.q, a.prec)
        t_uplan = time.perf_counter() - t1
        ev[3].record(stream)
        up.simulate(psi_u, stream)
        ev[4].record(stream)
        cmp = api.compare(psi, psi_u, a.prec, stream)  # synchronizes
        ev[5].record(stream)
        ev[5].synchronize()
        t_verify_end = time.perf_counter()
        if record:
            rec["verify"].append(ev[4].elapsed_time(ev[5]) / 1e3)
            rec["pre"].append(t_pre)
            rec["sub"].append(ev[0].elapsed_time(ev[1]) / 1e3)
            rec["merge"].append(ev[1].elapsed_time(ev[2]) / 1e3)
            rec["orig_host"].append(t_uplan)
            rec["orig"].append(t_uplan + ev[3].elapsed_time(ev[4]) / 1e3)
            rec["cmp"].append(cmp)
        plan.close()
        up.close()
        return t_verify_end

    for _ in range(a.warmup):
        step(False)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    for _ in range(a.steps):
        step(True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = time.perf_counter() - t_start
    clk = clocks.stop()

    mean = {k: statistics.mean(v) for k, v in rec.items() if k != "cmp"}
    t_cut = mean["pre"] + mean["sub"] + mean["merge"]
    elapsed, t_cut = max_over_ranks([elapsed, t_cut], world, dev)

    # e2e: host circuit in, host state out (pinned), copies inside the timed region
    e2e = None
    if not a.no_e2e:
        host_psi = torch.empty(psi.numel(), dtype=psi.dtype, pin_memory=True)
        times = []
        h2d = 0
        for i in range(a.warmup + a.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan = api.CutPlan(packed, a.q, segs, a.decomp, a.prec)
            plan.simulate_segments(seg, stream)
            plan.merge(seg, psi, ws, a.merge_form, stream)
            api.copy_to_host(psi, host_psi, stream)
            torch.cuda.synchronize()
            if i >= a.warmup:
                times.append(time.perf_counter() - t0)
            h2d = plan.info["table_bytes"]
            plan.close()
        (e2e_v,) = max_over_ranks([statistics.mean(times)], world, dev)
        e2e = {"value": e2e_v, "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(info["psi_bytes"])}
        del host_psi

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    hbm, bf16, peak_src = measured_peaks()
    amp = 8 if a.prec == "c64" else 16
    n_amp = 1 << a.q
    K = 1 << a.ctotal
    # merge: the output written once plus the factors read once
    merge_bytes = amp * n_amp + amp * sum(
        (1 << (info["seg_cuts"][i] + info["seg_qubits"][i])) for i in range(info["n_seg"]))
    merge_gbs = merge_bytes / mean["merge"] / 1e9
    # uncut passes: the first only writes the vector, every later one reads and writes it
    n_pass = uinfo["n_passes"]
    orig_dev = mean["orig"] - mean["orig_host"]
    pass_bytes = amp * n_amp * (2 * n_pass - 1) / n_pass
    pass_s = orig_dev / n_pass
    pass_gbs = pass_bytes / pass_s / 1e9
    merge_rf = {"bound": "hbm", "achieved": merge_gbs, "peak": hbm, "unit": "GB/s",
                "frac": merge_gbs / hbm, "traffic": None,
                "kernel": "cut_merge", "bytes_per_launch": merge_bytes,
                "launch_s": mean["merge"], "peak_source": peak_src}
    # Algorithmic work of the uncut passes: a complex 2x2 per amplitude (8 FMA,
    # 16 flops) for every dense one-qubit gate of the circuit (U3, H, X; a CX
    # is H CZ H on its target) and nothing for the diagonal ones.  The rotation
    # engine executes fewer (2 FMA per rotation plus its phase blocks), so a
    # fraction near or above 1 would not mean the FP32 pipes are saturated.
    n_dense = sum(1 for g in gates if g.kind in ("U3", "H", "X")) + \
        2 * sum(1 for g in gates if g.kind == "CX")
    uncut_flops = 16.0 * n_dense * n_amp
    if a.prec == "c64":
        alu_peak, alu_src = fp32_peak_tflops(), "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"
    else:  # complex128 in native FP64 (CUTSIM_C128_GATES=fp64) runs on the FP64 pipes
        alu_peak, alu_src = FP64_NOMINAL_TFLOPS, "nominal GB300 FP64 (no measured FP64 peak)"
    arith = gate_arith(a.prec)
    inst_rate = fp32_inst_rate()

    def executed(inst, flops, secs):
        # FP32-pipe instructions the program's arithmetic needs at least,
        # against the pipes' instruction rate over the measured time
        return {"fp32_inst_per_launch": inst, "flops_per_launch": flops,
                "achieved_tflops": flops / secs / 1e12, "inst_per_s": inst / secs,
                "inst_peak_per_s": inst_rate, "frac": inst / secs / inst_rate,
                "arith": arith}

    pass_tf = uncut_flops / n_pass / pass_s / 1e12
    pass_rf = {"bound": "alu", "achieved": pass_tf, "peak": alu_peak, "unit": "TFLOP/s",
               "frac": pass_tf / alu_peak, "traffic": recorded_traffic("uncut_pass", a),
               "kernel": "stage_kernel (uncut passes)", "flops_per_launch": uncut_flops / n_pass,
               "launch_s": pass_s, "hbm_gbs": pass_gbs, "hbm_bytes_per_launch": pass_bytes,
               "peak_source": alu_src}
    if arith != "f64":
        ui, uf = executed_work(program_ops(api.program_image(gates, a.q, a.prec)[0]), arith)
        pass_rf["executed"] = executed(ui / n_pass, uf / n_pass, pass_s)
    if arith == "dfl":
        # double-float: the FP32 pipes run the complex128 arithmetic; its
        # peak is the flops of this op mix at the full FP32 instruction rate
        ex = pass_rf["executed"]
        pass_rf.update({"achieved": ex["achieved_tflops"], "frac": ex["frac"],
                        "peak": ex["flops_per_launch"] / ex["fp32_inst_per_launch"] * inst_rate / 1e12,
                        "flops_per_launch": ex["flops_per_launch"],
                        "peak_source": "double-float on the FP32 pipes: 152 SMs x 128 lanes x "
                                       "2070 MHz instructions, at this program's instructions "
                                       "per flop"})
    # AUTO's rule (the library's kAutoTcMinTerms): 3xTF32 from K = 8 terms on
    # AUTO's rule (the library's kAutoTcMinTerms / kAutoOzakiMinTerms): 3xTF32
    # from K = 8 terms on for complex64, the Ozaki form from K = 2 on for complex128
    k_last = 1 << cpb[-1]
    tc_form = a.merge_form if a.merge_form != "auto" else (
        ("f16x3" if k_last >= 8 else "fma") if a.prec == "c64" else
        ("ozaki" if k_last >= 2 else "fma"))
    merge_rf["traffic"] = recorded_traffic("merge_" + tc_form, a)
    if tc_form == "fma":
        # complex FMA merge: 8 flops per term per output amplitude on the ALU
        # pipes, for the last (2^q-sized) stage's K_last terms
        fma_flops = 8.0 * (1 << cpb[-1]) * n_amp
        merge_rf["alu"] = {"achieved": fma_flops / mean["merge"] / 1e12, "peak": alu_peak,
                           "unit": "TFLOP/s",
                           "frac": fma_flops / mean["merge"] / 1e12 / alu_peak,
                           "peak_source": alu_src}
    if tc_form in ("tf32x3", "bf16x3", "f16x3"):
        # three split products of the real GEMM of the last (2^q-sized) merge
        # stage: 3 x 8 K_last flops per output amplitude, K_last = 2^(cuts on
        # the last boundary) (all of c_total for n = 2)
        k_last = 1 << cpb[-1]
        tc_flops = 3.0 * 8 * k_last * n_amp
        tc_peak = bf16 * (0.5 if tc_form == "tf32x3" else 1.0)  # nominal TF32:BF16 = 1:2
        merge_rf["tensor"] = {"achieved": tc_flops / mean["merge"] / 1e12, "peak": tc_peak,
                              "unit": "TFLOP/s", "form": tc_form,
                              "frac": tc_flops / mean["merge"] / 1e12 / tc_peak,
                              "peak_source": peak_src + " bf16 burst" +
                              (" x 0.5 (nominal TF32/BF16)" if tc_form == "tf32x3" else "")}
    if tc_form == "ozaki":
        # 21 bf16 slice products of the real GEMM of the last merge stage, each
        # 4 KR flops per output amplitude (KR = 2 K_last rounded up to 32)
        kr = ((2 * k_last + 31) // 32) * 32
        tc_flops = 21.0 * 4 * kr * n_amp
        merge_rf["tensor"] = {"achieved": tc_flops / mean["merge"] / 1e12, "peak": bf16,
                              "unit": "TFLOP/s", "form": "ozaki",
                              "frac": tc_flops / mean["merge"] / 1e12 / bf16,
                              "peak_source": peak_src + " bf16 burst",
                              "method_flops": 8.0 * k_last * n_amp}
    # verification: both 2^q vectors read once (complex64: FP32 exact products
    # in double-float, HBM-bound; complex128: FP64 arithmetic bounds it)
    verify_bytes = 2.0 * amp * n_amp
    verify_rf = {"bound": "hbm", "achieved": verify_bytes / mean["verify"] / 1e9, "peak": hbm,
                 "unit": "GB/s", "frac": verify_bytes / mean["verify"] / 1e9 / hbm,
                 "traffic": None, "kernel": "compare_partial", "bytes_per_launch": verify_bytes,
                 "launch_s": mean["verify"], "peak_source": peak_src}
    dominant = pass_rf if orig_dev > mean["merge"] else merge_rf
    # per step: one persistent launch for every segment pass, the earlier
    # chain stages (FMA), the last stage (split + tensor-core kernel, or FMA),
    # the uncut passes, and the two verification kernels
    merge_launches = {"fma": 1, "f16x3": 3}.get(tc_form, 2)  # f16x3: maxima, split, merge
    launches = 1 + (info["n_seg"] - 2) + merge_launches + n_pass + 2
    # subcircuit stage (Algorithm 2): N_sub variants of 2^{q_i} amplitudes, 16
    # flops per amplitude per dense one-qubit gate of the segment, 6 per
    # diagonal factor (CZ inside the segment, the cut terms on its side)
    seg_flops = 0.0
    for i in range(info["n_seg"]):
        lo, hi = info["seg_start"][i], info["seg_start"][i] + info["seg_qubits"][i]
        inside = lambda x: lo <= x < hi
        g_nd = g_diag = 0
        for g in gates:
            if g.q1 < 0:
                if inside(g.q0):
                    if g.kind in ("U3", "H", "X"):
                        g_nd += 1
                    else:
                        g_diag += 1
            elif inside(g.q0) and inside(g.q1):
                g_nd += 2 if g.kind == "CX" else 0
                g_diag += 1
            elif inside(g.q0) or inside(g.q1):  # a cut: its term on this side
                g_nd += 2 if (g.kind == "CX" and inside(g.q1)) else 0
                g_diag += 1
        seg_flops += (1 << (info["seg_cuts"][i] + info["seg_qubits"][i])) * (16.0 * g_nd + 6.0 * g_diag)
    seg_tf = seg_flops / mean["sub"] / 1e12
    seg_rf = {"bound": "alu", "achieved": seg_tf, "peak": alu_peak, "unit": "TFLOP/s",
              "frac": seg_tf / alu_peak, "traffic": recorded_traffic("segments", a),
              "kernel": "batch_kernel (all passes of all segments, one persistent launch)",
              "flops_per_launch": seg_flops, "launch_s": mean["sub"],
              "bytes_written": float(info["seg_buf_bytes"]), "peak_source": alu_src}
    if arith != "f64":
        si = sf = 0.0
        for i in range(info["n_seg"]):
            words, _ = api.plan_program_image(gates, a.q, segs, i, a.decomp, a.prec)
            x, y = executed_work(program_ops(words), arith)
            si, sf = si + x, sf + y
        seg_rf["executed"] = executed(si, sf, mean["sub"])
        if arith == "dfl":
            ex = seg_rf["executed"]
            seg_rf.update({"achieved": ex["achieved_tflops"], "frac": ex["frac"],
                           "peak": sf / si * inst_rate / 1e12, "flops_per_launch": sf,
                           "peak_source": pass_rf["peak_source"]})
    cmp = rec["cmp"][-1]
    orc = None
    if not a.no_cpu_baseline:
        orc = run_oracle_timing(a, [BASE_SLABS, 2 * BASE_SLABS], sample_seed=2024)
    cpu = None
    oracle_parity = None
    if orc is not None and "error" in orc:
        cpu = {"error": orc["error"]}
    elif orc is not None:
        cpu = cpu_record(orc, a)
        import numpy as np

        xs = w.sample_indices(a.q, 4096, orc["sample_seed"])
        got = api.gather(psi, xs, a.prec).astype(np.complex128)
        ref = np.array([complex(re, im) for re, im in orc["sample_amplitudes"]])
        scale = api.compare(psi, psi, a.prec)["max_abs_b"]  # max |psi| of the whole cut state
        dot = np.vdot(ref, got)
        oracle_parity = {
            "samples": len(xs), "seed": orc["sample_seed"],
            "max_abs_diff_over_max": float(np.max(np.abs(got - ref)) / scale),
            "fidelity_sampled": float(abs(dot) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)),
            "tolerance": {"c64": 2e-6, "c128": 1e-12}[a.prec] if a.merge_form != "bf16x3" else 5e-5,
        }
    out = {
        "metric": METRIC,
        "value": t_cut,
        "unit": "s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": 1000.0 * elapsed / a.steps,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "dfl": "f32x2 (double-float)", "f64": "f64"}[arith],
        "data": "synthetic",
        "config": dict(cfg, l2=("not flushed explicitly: every step writes the 2^q uncut vector "
                                "and reads both 2^q vectors (>> 129 MB L2) between merges")),
        "stages": {"pre_s": mean["pre"], "sub_s": mean["sub"], "merge_s": mean["merge"],
                   "cut_s": t_cut, "orig_s": mean["orig"], "orig_plan_s": mean["orig_host"],
                   "verify_s": mean["verify"],
                   "delta": (t_cut - mean["orig"]) / mean["orig"]},
        "merge_gbs": merge_gbs,
        "gate_pass_gbs": pass_gbs,
        "uncut_passes": n_pass,
        "seg_passes": info["seg_passes"],
        "merge_terms": K,
        "threshold_n2": a.q / 2 if a.n == 2 else None,
        "parity": {"vs_uncut_gpu": {"max_abs_diff_over_max": cmp["max_abs_diff"] / cmp["max_abs_b"],
                                    "fidelity": cmp["fidelity"], "norm2_cut": cmp["norm2_a"],
                                    "norm2_uncut": cmp["norm2_b"]},
                   "vs_oracle_sampled": oracle_parity},
        "roofline": dominant,
        "rooflines": {"merge": merge_rf, "uncut_pass": pass_rf, "segments": seg_rf,
                      "verify": verify_rf},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches * a.steps,
        "clocks": clk,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
