#!/usr/bin/env python
"""Benchmark of the multirate DG shallow-water hot path on GB300.

Metric: DOF-updates/s per RHS stage = (sum over finest substeps of active
elements x Np x 3) / wall time. One benchmark "step" is one MRAB macro step
(2^{L-1} finest substeps, every level advanced once or more) of the tsunami-like
workload: 500,000 triangles graded 8:1 toward a tanh beach, N = 4, 4 levels,
positivity + TVB limiting, FP32, replayed as one CUDA graph. The state and the
Adams-Bashforth history (~0.56 GB) exceed L2, so no flush is needed between steps.

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the
scenarios do not exchange data); value sums all ranks' DOF-updates over the max time.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (there is no reference implementation to install: the paper ships no code).

--oracle-configs times the oracle (no GPU) on bounded samples of every
configuration, with all host threads and with one, and prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RHS stage"
UNIT = "DOF-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1000)
    ap.add_argument("--ny", type=int, default=250)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--precision", default="fp32tc", choices=["fp32tc", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-regroup", action="store_true")
    ap.add_argument("--no-colloc", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-scenarios", type=int, default=64)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--oracle-configs", action="store_true")
    ap.add_argument("--oracle-configs-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-sample-child", nargs=3, metavar=("NX", "NY", "SCHEME"), help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(args, nx=None, ny=None):
    from workloads import scenarios as sc
    return sc.tsunami(nx=nx or args.nx, ny=ny or args.ny, N=args.order, nlevels=4)


def workload_config(args, K, extra=None):
    cfg = {"workload": f"tsunami_{2 * args.nx * args.ny}_N{args.order}_L4",
           "mesh": f"{args.nx}x{args.ny}x2 triangles, x-graded 8:1, jitter 0.15, seed 3",
           "triangles": K, "N": args.order, "levels_max": 4, "limiters": "PP+TVB",
           "scheme": "MRAB3 (Algorithm 2)", "precision": args.precision,
           "step": "one macro step = 2^(L-1) finest substeps (CUDA graph)",
           "l2": "no flush: state + AB history > L2 (129 MB)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline bookkeeping

def stage_bytes_per_element(N, ts):
    """Algorithmic HBM bytes one element moves in the stage kernel: read Q (3Np),
    B (Np), two older R slots (6Np), geometry (4) and connectivity (4 words);
    write R (3Np), Q (3Np), means (3), the P1 vertex values the TVB limiter reads
    (9) and the dry byte. Neighbour traces are counted as L2 hits; the half-step
    records of elements with a finer neighbour are not counted."""
    Np = (N + 1) * (N + 2) // 2
    return (16 * Np + 4 + 3 + 9) * ts + 4 * 4 + 1


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


STAGE_KERNEL_SOURCES = ("kernel_types.hpp", "kernels.cuh", "kernels_tc.cuh", "kernels_order.inc")


def kernel_source_hash():
    """Hash of the sources that define the stage kernels (a recorded ncu traffic
    figure is used only while they are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1403_1661_gb300", "csrc")
    for f in STAGE_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(N, precision):
    """DRAM bytes per element of the stage kernel from a committed ncu summary, if
    it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"traffic_stage_{precision}_n{N}.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_element")


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample

def oracle_sample(args, nsteps=1, nx=200, ny=50, scheme="cubature"):
    from oracle import problem
    scn = workload(args, nx=nx, ny=ny)
    om, ref, model, integ = problem.build(scn)
    if scheme == "collocation":
        from oracle.colloc import CollocModel
        from oracle.mrab import MRAB
        B, h, hu, hv = problem.nodal_inputs(scn, om, ref)
        integ = MRAB(CollocModel(om, ref, model.B, scn.g, scn.h0), h, hu, hv, integ.level, integ.dt_min,
                     limiter_mask=scn.limiter_mask, tvb_M=scn.tvb_M, tvb_nu=scn.tvb_nu, dry_mode=scn.dry_mode)
    period = 2 ** (integ.L - 1)
    t = time.perf_counter()
    d0 = integ.dof_updates
    for _ in range(nsteps * period):
        integ.substep()
    dt = time.perf_counter() - t
    return (integ.dof_updates - d0) / dt, dt, om.K, period


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def oracle_sample_single_thread(args, nx, ny, scheme="cubature"):
    """oracle_sample (one macro step) in a fresh interpreter whose numerical
    libraries are limited to one thread, so that the reported core count is the one
    the oracle used. Returns (DOF-updates/s, seconds, triangles)."""
    env = dict(os.environ, **SINGLE_THREAD_ENV)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--order", str(args.order),
                        "--oracle-sample-child", str(nx), str(ny), scheme],
                       capture_output=True, text=True, env=env, check=True)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["value"], d["seconds"], d["triangles"]


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count(), model


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nx, ny = 100, 25
    for _ in range(args.warmup):
        oracle_sample(args, 1, nx, ny)
    vals, secs = [], []
    dofs_total, t_total = 0.0, 0.0
    for _ in range(args.steps):
        v, dt, K, period = oracle_sample(args, 1, nx, ny)
        dofs_total += v * dt
        t_total += dt
    value = dofs_total / t_total
    _, model = cpu_info()
    # one thread when this process set the limit before numpy was imported (main)
    cores = 1 if os.environ.get("OPENBLAS_NUM_THREADS") == "1" else os.cpu_count()
    sample = (f"same scenario at {nx}x{ny}x2 = {2 * nx * ny} triangles (N={args.order}, 4 levels, PP+TVB), "
              f"one macro step per bench step, FP64 numpy oracle, {cores} thread(s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, 2 * args.nx * args.ny),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm

def combine_ranks(ms, dofs, dist=None, device="cuda"):
    """Whole-job numbers of independent replicas: the slowest rank's time and the
    DOF updates of all ranks (one collective each, outside the timed region)."""
    if dist is None:
        return ms, float(dofs)
    import torch
    tmax = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(dofs)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    from paper_1403_1661_gb300 import build as _build
    _build.build()
    import paper_1403_1661_gb300 as P

    scn = workload(args)
    s = P.solver_from_scenario(scn, precision=args.precision)
    L, counts, dt_min = s.level_info()
    period = 2 ** (L - 1)
    stream = s.stream

    # warm-up (also captures the graph)
    s.step(args.warmup)
    torch.cuda.synchronize()
    d0 = s.stats()["dof_updates"]
    launches0 = s.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    st = s.stats()
    dofs = st["dof_updates"] - d0
    launches = s.kernel_launches() - launches0
    ms_all, dofs_all = combine_ranks(ms, dofs, dist, "cuda")
    value = dofs_all / (ms_all / 1e3)

    # per-kernel timing of one more macro step (events around every launch)
    prof = s.profile_substeps(2 * period)
    ts = 8 if args.precision == "fp64" else 4
    bpe = stage_bytes_per_element(args.order, ts)
    stage_bytes = prof["stage_elements"] * bpe
    achieved = stage_bytes / (prof["stage_ms"] / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    per_launch_elems = prof["stage_elements"] / max(1, prof["stage_launches"])
    traffic_pe = recorded_traffic(args.order, args.precision)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (traffic_pe * per_launch_elems) if traffic_pe else None,
                "kernel": (f"k_stage_tc<{args.order}>" if args.precision == "fp32tc"
                           else f"k_stage<{'float' if ts == 4 else 'double'},{args.order}>"),
                "algorithmic_bytes_per_launch": bpe * per_launch_elems,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "stage_share_of_step": prof["stage_ms"] / max(1e-9, prof["stage_ms"] + prof["tvb_ms"] + prof["other_ms"]),
                "tvb_ms_per_step": prof["tvb_ms"] / 2, "stage_ms_per_step": prof["stage_ms"] / 2}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32" if ts == 4 else "f64",
              "data": "synthetic", "gpu_launches": int(launches),
              "config": workload_config(args, s.K, {"levels": int(L), "elements_per_level": counts.tolist(),
                                                   "parallelism": f"replicas x{world}"}),
              "roofline": roofline, "clocks": clk}

    # end to end through the public API with page-locked host buffers: the state in
    # (swe_set_state), one macro step (swe_step), the state out (swe_get_state)
    if not args.no_e2e:
        B, h, hu, hv = P.scenario_inputs(scn, s.mesh)

        def pinned(a=None):
            buf = torch.empty((s.K, s.Np), dtype=torch.float64, pin_memory=True).numpy()
            if a is not None:
                buf[...] = np.asarray(a).reshape(s.K, s.Np)
            return buf
        hin, huin, hvin = pinned(h), pinned(hu), pinned(hv)
        outs = (pinned(), pinned(), pinned())
        ne = 5
        s.set_state(hin, huin, hvin)            # warm-up of the whole loop
        s.step(1)
        s.get_state(out=outs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne):
            s.set_state(hin, huin, hvin)
            s.step(1)
            s.get_state(out=outs)
        te = (time.perf_counter() - t0) / ne
        de = s.stats()["dof_updates"]            # set_state restarts the count: one macro step's
        nbytes = 3 * s.K * s.Np * 8
        result["e2e"] = {"value": de / te, "unit": UNIT, "ms_per_step": te * 1e3,
                         "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 4,
                         "note": "swe_set_state + swe_step(1) + swe_get_state per step, FP64 (h, hu, hv) "
                                 "arrays in page-locked host memory, caller layout"}

    # the plain FP64 GPU form on the same workload (fewer steps: ~60x slower)
    if not args.no_fp64 and rank == 0:
        s64 = P.solver_from_scenario(scn, precision="fp64")
        s64.step(1)
        torch.cuda.synchronize()
        d0 = s64.stats()["dof_updates"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n64 = 2
        e0.record(s64.stream)
        s64.step(n64)
        e1.record(s64.stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        d64 = s64.stats()["dof_updates"] - d0
        result["fp64_gpu"] = {"value": d64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64 / n64,
                              "fp32_speedup": value / (d64 / (ms64 / 1e3))}
        s64.close()
        del s64

    # the same tier with the compensated state update (swe_params.compensated)
    if rank == 0 and args.precision != "fp64":
        sc_ = P.solver_from_scenario(scn, precision=args.precision, compensated=True)
        sc_.step(2)
        torch.cuda.synchronize()
        d0 = sc_.stats()["dof_updates"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        nc = 10
        e0.record(sc_.stream)
        sc_.step(nc)
        e1.record(sc_.stream)
        torch.cuda.synchronize()
        msc = e0.elapsed_time(e1)
        dc = sc_.stats()["dof_updates"] - d0
        result["compensated"] = {"value": dc / (msc / 1e3), "unit": UNIT, "ms_per_step": msc / nc,
                                 "vs_plain": (dc / (msc / 1e3)) / value,
                                 "note": "same workload and tier, state updated with a compensated sum (mass "
                                         "kept to rounding, FP64's accuracy over long runs)"}
        sc_.close()
        del sc_

    # the nodal-collocation scheme on the same workload (FP32 SIMT kernels)
    if rank == 0 and not args.no_colloc:
        result["collocation"] = run_collocation(args, scn, P)

    # the rules of integration order 2N (Fig. 2's caption) on the same workload
    if rank == 0 and not args.no_colloc:
        v, ms2, prof2, ach2 = _colloc_run(args, scn, P, "fp32tc", 10, scheme="cubature_2n")
        peak2, _ = measured_peaks()
        result["cubature_2n"] = {"value": v, "unit": UNIT, "ms_per_step": ms2, "steps": 10,
                                 "precision": "fp32tc", "kernel": f"k_stage_tc<{32 + args.order}>",
                                 "stage_ms_per_step": prof2["stage_ms"] / 2, "stage_hbm_frac": ach2 / peak2,
                                 "note": "volume rule of degree 2N ((N+1)^2 points), N+1 Gauss points per "
                                         "face, pre-balanced form; same workload, levels and limiters"}

    # kernel-structure ablation (Section 7): one R evaluation of the whole mesh by the
    # fused kernels and by the paper's three-kernel split with stored face traces
    if rank == 0 and not args.no_ablation:
        result["kernel_structure"] = run_ablation(s, P)

    # level regrouping without restart (Section 4): one CFL regroup of the full mesh
    if rank == 0 and not args.no_regroup:
        result["regroup"] = run_regroup(s)

    # batched ensemble: uneven scenarios advanced by one graph launch per macro step
    if rank == 0 and not args.no_batch:
        result["batched"] = run_batched(args)
    # served stream: Poisson arrivals, continuous batching under an HBM budget
    if rank == 0 and not args.no_serve:
        result["served"] = run_served(args)

    if rank == 0 and not args.no_cpu_baseline:
        v, dt, Ks = oracle_sample_single_thread(args, 400, 100)
        _, model = cpu_info()
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"same scenario at 400x100x2 = {Ks} triangles (N={args.order}, 4 levels, "
                                            f"PP+TVB), one macro step, FP64 numpy oracle ({dt:.1f} s), one thread "
                                            f"(BLAS and OpenMP limited to one)",
                                  "cpu": model}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def _colloc_run(args, scn, P, precision, steps, scheme="collocation"):
    import torch
    s = P.solver_from_scenario(scn, precision=precision, scheme=scheme)
    s.step(3)
    torch.cuda.synchronize()
    d0 = s.stats()["dof_updates"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dofs = s.stats()["dof_updates"] - d0
    L = s.level_info()[0]
    prof = s.profile_substeps(2 * 2 ** (L - 1))
    bpe = stage_bytes_per_element(args.order, 4)
    achieved = prof["stage_elements"] * bpe / (prof["stage_ms"] / 1e3) / 1e9
    return dofs / (ms / 1e3), ms / steps, prof, achieved


def run_collocation(args, scn, P, steps=10):
    """The nodal-collocation scheme (fluxes at the nodes and face nodes) on the same
    workload and levels, tensor-core and SIMT FP32 tiers: DOF-updates/s, and the
    tensor-core stage kernel against HBM."""
    value, ms_step, prof, achieved = _colloc_run(args, scn, P, "fp32tc", steps)
    v_simt, ms_simt, _, ach_simt = _colloc_run(args, scn, P, "fp32", steps)
    peak, kind = measured_peaks()
    out_cpu = None
    if not args.no_cpu_baseline:
        v, dt, Ks = oracle_sample_single_thread(args, 400, 100, scheme="collocation")
        out_cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle (oracle/colloc.py)",
                   "sample": f"same scenario at 400x100x2 = {Ks} triangles, one macro step ({dt:.1f} s), one thread"}
    return {"value": value, "unit": UNIT, "ms_per_step": ms_step, "steps": steps,
            "cpu_oracle": out_cpu,
            "precision": "fp32tc", "kernel": f"k_stage_tc<{16 + args.order}> (collocation code)",
            "stage_ms_per_step": prof["stage_ms"] / 2, "tvb_ms_per_step": prof["tvb_ms"] / 2,
            "stage_hbm_frac": achieved / peak, "stage_achieved_gbs": achieved,
            "simt_fp32": {"value": v_simt, "ms_per_step": ms_simt, "stage_hbm_frac": ach_simt / peak,
                          "kernel": f"k_stage<float,{16 + args.order}>"},
            "note": "same workload, levels and limiters; R from nodal fluxes (Ncub = Np, face nodes)"}


def run_ablation(s, P, reps=10):
    """ms per R evaluation (all elements, level-synchronous state) of each kernel
    structure; L2 flushed (256 MB written) before every timed launch."""
    import torch
    from paper_1403_1661_gb300 import _native as nat
    variants = [("fused_tc" if s.precision == nat.SWE_FP32_TC else "fused", nat.SWE_RHS_FUSED),
                ("fused_simt_ops_in_smem", nat.SWE_RHS_FUSED_SIMT),
                ("fused_simt_ops_in_global", nat.SWE_RHS_GLOBAL_OPS),
                ("split_3_kernels_stored_traces", nat.SWE_RHS_SPLIT)]
    if s.precision != nat.SWE_FP32_TC:
        variants.pop(1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=s.device)
    dofs = 3 * s.K * s.Np
    out = {"unit": "ms per R evaluation", "elements": s.K, "reps": reps, "l2": "flushed before each launch"}
    base = None
    for name, v in variants:
        nbytes = s.rhs_scratch_bytes(v)
        scratch = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=s.device) if nbytes else None
        for _ in range(3):
            s.rhs_variant(v, scratch)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            with torch.cuda.stream(s.stream):
                flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.rhs_variant(v, scratch)
            e1.record(s.stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / reps
        base = base or ms
        out[name] = {"ms": ms, "dof_per_s": dofs / (ms / 1e3), "vs_first": ms / base,
                     "scratch_mb": nbytes / 1e6}
        del scratch
    return out


def run_regroup(s):
    """Wall time of one swe_regroup by the CFL rule after three macro steps, and of
    the next macro step (graph re-capture included)."""
    import numpy as np
    import torch
    s.step(3)
    torch.cuda.synchronize()
    old = s.level.copy()
    t0 = time.perf_counter()
    lev, margin = s.regroup(None)
    t1 = time.perf_counter()
    s.step(1)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"ms": (t1 - t0) * 1e3, "next_macro_step_ms": (t2 - t1) * 1e3, "elements": int(lev.size),
            "changed": int((lev != old).sum()), "levels": np.bincount(lev)[1:].tolist(), "cfl_margin": margin,
            "where": "device: CFL steps, history re-interpolation, gather of every per-element array; "
                     "host: level rule and new order from K steps"}


def run_batched(args, steps=5):
    import torch
    import paper_1403_1661_gb300 as P
    from workloads import scenarios as sc
    scns = sc.ensemble(n=args.batch_scenarios)
    tuned = {N: P.tune(N, args.precision) for N in sorted({s.N for s in scns})}
    solvers = []
    for s in scns:
        so = P.solver_from_scenario(s, precision=args.precision)
        so.set_launch_config(tuned[s.N])
        solvers.append(so)
    b = P.Batch(solvers, max_macro=1)
    b.step(1)
    torch.cuda.synchronize()
    d0 = sum(so.stats()["dof_updates"] for so in solvers)
    l0 = b.launches()
    # every batch step reads its per-scenario statuses back (a synchronisation), so
    # the step is timed as a whole: CUDA events around the replays on the batch stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(steps):
        b.step(1)
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dofs = sum(so.stats()["dof_updates"] for so in solvers) - d0
    # element-stages of one macro step per scenario (active levels per substep)
    d_step = {}
    for so in solvers:
        L, counts, _ = so.level_info()
        per_macro = 0
        for j in range(2 ** (L - 1)):
            m = 1
            while j and m < L and j % (2 ** m) == 0:
                m += 1
            per_macro += int(sum(counts[:(L if j == 0 else m)]))
        d_step[so] = per_macro
    # the same solvers stepped one by one, each replaying its own graph on its own
    # stream (enqueued back to back, so their kernels overlap on the GPU): the
    # schedule the persistent kernel replaces
    torch.cuda.synchronize()
    d1 = sum(so.stats()["dof_updates"] for so in solvers)
    t0 = time.perf_counter()
    for _ in range(steps):
        for so in solvers:
            so.step(1)
    torch.cuda.synchronize()
    ms_alone = (time.perf_counter() - t0) * 1e3
    dofs_alone = sum(so.stats()["dof_updates"] for so in solvers) - d1
    bpe = {N: stage_bytes_per_element(N, 4 if args.precision != "fp64" else 8) for N in {s.N for s in scns}}
    byts = sum(d_step[so] * bpe[s_.N] for s_, so in zip(scns, solvers))
    peak, peak_kind = measured_peaks()
    ach = byts / (ms / steps / 1e3) / 1e9
    out = {"value": dofs / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "scenarios": len(scns),
           "triangles": int(sum(so.K for so in solvers)), "orders": sorted({s.N for s in scns}),
           "autotuned": {str(k): v for k, v in tuned.items()},
           "gpu_launches_per_step": (b.launches() - l0) / steps,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "kernel": "k_batch (persistent; stage + TVB tickets)",
                        "algorithmic_bytes_per_step": byts,
                        "basis": "stage-kernel algorithmic bytes of every element-stage of the step over the "
                                 "whole step time (the TVB work inside the same kernels is not counted)",
                        "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"},
           "step": "one graph replay = one macro step of every scenario: per (tier, order) group one "
                   "persistent kernel over a device ticket queue",
           "per_solver_streams": {"value": dofs_alone / (ms_alone / 1e3), "unit": UNIT,
                                  "ms_per_step": ms_alone / steps,
                                  "note": "same solvers and steps, each solver's own captured graph on its own "
                                          "stream, host wall clock"}}
    b.close()
    # the same batch at the default shape (as many CTAs as fit, four warps per
    # tensor-core CTA): what the tuning buys
    default = {"ctas_per_sm": 0, "tc_warps": 4 if args.precision == "fp32tc" else None}
    for so in solvers:
        so.set_launch_config(default)
    b = P.Batch(solvers, max_macro=1)
    b.step(1)
    torch.cuda.synchronize()
    d2 = sum(so.stats()["dof_updates"] for so in solvers)
    e0.record(b.stream)
    for _ in range(steps):
        b.step(1)
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms_u = e0.elapsed_time(e1)
    out["untuned"] = {"value": (sum(so.stats()["dof_updates"] for so in solvers) - d2) / (ms_u / 1e3),
                      "unit": UNIT, "ms_per_step": ms_u / steps, "shape": default}
    b.close()
    for so in solvers:
        so.close()
    return out


def run_served(args):
    import torch
    from paper_1403_1661_gb300.serve import GpuFactory, Server, requests_from_stream
    from workloads import scenarios as sc
    import paper_1403_1661_gb300 as P
    stream = sc.served_stream(duration=args.serve_seconds)
    reqs = requests_from_stream(stream, substeps=500)
    tuned = {N: P.tune(N, args.precision) for N in sorted({r.scenario.N for r in reqs})}
    srv = Server(budget_bytes=150e9, max_slots=64, macro_per_round=4, prep_workers=8, start_workers=8,
                 factory=GpuFactory(args.precision, tuned=tuned))
    out = srv.run(reqs)
    torch.cuda.synchronize()
    # stage-kernel algorithmic bytes of every element-stage served, over the wall time
    ts = 4 if args.precision != "fp64" else 8
    byts = 0.0
    for r in out["done"]:
        N = r.scenario.N
        # a DOF-update is one field (eta, hu, hv) at one node: 3 Np per element-stage
        byts += r.dof_updates / (3 * (N + 1) * (N + 2) // 2) * stage_bytes_per_element(N, ts)
    peak, peak_kind = measured_peaks()
    ach = byts / out["wall_s"] / 1e9
    offered = sum(r.dof_updates for r in out["done"]) / args.serve_seconds
    return {"requests": out["requests"], "p50_s": out["p50_s"], "p99_s": out["p99_s"], "mean_s": out["mean_s"],
            "offered_dof_per_s": offered,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "basis": "stage-kernel algorithmic bytes of every element-stage of the served requests "
                                  "over the wall time (TVB and host work not counted)",
                         "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"},
            "aggregate_dof_per_s": out["aggregate_dof_per_s"], "wall_s": out["wall_s"],
            "peak_running": out["peak_running"], "peak_gb": out["peak_bytes"] / 1e9,
            "autotuned": {str(k): v for k, v in tuned.items()},
            "rejected": out["rejected"], "failed": out["failed"],
            "arrivals": f"Poisson 50/s for {args.serve_seconds:.0f} s, K log-uniform 2k-1M, N in {{2,3,4}}, "
                        f"500 MRAB substeps each, HBM budget 150 GB; 8 preparation and 8 creation threads"}


def _oracle_rate(scn, substeps):
    """DOF-updates/s of the oracle over ``substeps`` finest substeps of ``scn``
    (set-up not timed)."""
    from oracle import problem
    om, ref, model, integ = problem.build(scn)
    d0, t = integ.dof_updates, time.perf_counter()
    for _ in range(substeps):
        integ.substep()
    dt = time.perf_counter() - t
    return (integ.dof_updates - d0) / dt, dt, om.K


def oracle_configs_child():
    """One line of oracle rates on bounded samples of configurations 1-4."""
    import numpy as np
    from workloads import scenarios as sc
    out = {}
    v, dt, K = _oracle_rate(sc.hump_square(), 100)
    out["1_hump_512_N2"] = {"value": v, "seconds": dt, "sample": f"full run: {K} triangles, 100 AB3 steps"}
    v, dt, K = _oracle_rate(sc.dam_break(), 20)
    out["2_dam_break_20480_N3"] = {"value": v, "seconds": dt,
                                   "sample": f"{K} triangles, first 20 of 2000 steps (PP + TVB)"}
    scn = sc.tsunami(nx=400, ny=100)
    v, dt, K = _oracle_rate(scn, 8)
    out["3_tsunami_N4_L4"] = {"value": v, "seconds": dt,
                              "sample": f"same beach at 400x100x2 = {K} triangles, one macro step (8 substeps)"}
    ens = sc.ensemble()
    pick = np.random.Generator(np.random.PCG64(9)).choice(len(ens), size=8, replace=False)
    dofs, secs, ks = 0.0, 0.0, []
    for i in sorted(pick):
        v, dt, K = _oracle_rate(ens[i], 1)
        dofs, secs = dofs + v * dt, secs + dt
        ks.append(f"{K}/N{ens[i].N}")
    out["4_ensemble"] = {"value": dofs / secs, "seconds": secs,
                         "sample": "8 seeded scenarios of the 64, first finest substep each (all levels active): "
                                   + ", ".join(ks)}
    print(json.dumps(out), flush=True)


def oracle_configs():
    """The oracle on every configuration, all host threads and one thread (a fresh
    interpreter with the BLAS/OpenMP thread counts set to 1)."""
    cores, model = cpu_info()
    line = {"kind": "oracle (FP64 numpy)", "unit": UNIT, "cores": cores, "cpu": model}
    one = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for name, extra in (("all_threads", {}), ("one_thread", one)):
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-configs-child"],
                           env=dict(os.environ, **extra), capture_output=True, text=True, check=True)
        line[name] = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_sample_child:
        nx, ny, scheme = args.oracle_sample_child
        v, dt, K, _ = oracle_sample(args, 1, int(nx), int(ny), scheme=scheme)
        print(json.dumps({"value": v, "seconds": dt, "triangles": K}), flush=True)
        return
    if args.impl == "reference" and "numpy" not in sys.modules:
        # the oracle runs in this process: its numerical libraries get one thread,
        # set before numpy is first imported, so that "cores" is what it used
        os.environ.update(SINGLE_THREAD_ENV)
    if args.oracle_configs_child:
        oracle_configs_child()
        return
    if args.oracle_configs:
        oracle_configs()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
