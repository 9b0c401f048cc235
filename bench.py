#!/usr/bin/env python
"""Throughput of the reconstructed-DG convection-diffusion solve on GB300.

One bench step = one full solve of the single-GPU workload: N = 4 (Np = 15) nodal DG on a
256 x 256 x 2 jittered periodic mesh (131072 triangles, seed 1), v = (1, 0.5), D = 1 inside
the circle r < 0.25 about (0.5, 0.5) and 1e-4 outside, Gaussian pulse of width 0.05,
500 SSP-RK3 steps (1500 right-hand sides) at 0.5 x the stability bound, FP32 arithmetic.
The metric is GDOF/s = K Np x (right-hand sides) / time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank runs an independent replica (weak scaling, no collective on the
data path); rank 0 prints one JSON line.  --impl reference times the FP64 NumPy oracle on
the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "recDG diffusion RHS GDOF/s, FP32 vs FP64 at stated L2 err; serve p50/p99"
UNIT = "GDOF/s"
N_ORDER = 4
RK_STEPS = 500


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=256, help="mesh side (cells)")
    p.add_argument("--rk-steps", type=int, default=RK_STEPS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--precision", default="fp32", choices=["fp32", "tf32"],
                   help="fp32: stored per-edge operators; tf32: GEMM form on the tensor cores (split 3xTF32)")
    p.add_argument("--serve", action="store_true", help="run the request-stream server instead")
    p.add_argument("--serve-requests", type=int, default=200)
    p.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second of the request stream")
    p.add_argument("--serve-slots", type=int, default=32)
    p.add_argument("--serve-setup-workers", type=int, default=6)
    p.add_argument("--batch", action="store_true", help="run the batched uneven workload instead")
    p.add_argument("--paper-problems", action="store_true",
                   help="the paper's Gaussian diffusion / advection-diffusion convergence series instead")
    p.add_argument("--sweep", action="store_true", help="the N=3 manufactured-solution precision sweep instead")
    p.add_argument("--batch-chunk", type=int, default=25)
    p.add_argument("--orders", action="store_true",
                   help="the circle pulse stage at every order N = 1..6, FP32 and FP64, instead")
    p.add_argument("--orders-list", default="1,2,3,4,5,6")
    p.add_argument("--orders-precisions", default="fp32,fp64")
    p.add_argument("--hbm-read", action="store_true",
                   help="plain streaming-read time and bandwidth at a few sizes (the size-matched HBM bound)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(t_ms_local, units_local, dist=None, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's time (max over ranks)
    and the units of all ranks.  Returns (t_ms_max, units_total, units_total / t_max)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t_ms_local, units_local, units_local / (t_ms_local / 1e3)
    t = torch.tensor([float(t_ms_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t), float(n), float(n) / (float(t) / 1e3)


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


TRAFFIC_CSV = os.path.join(ROOT, "profiles", "stage_kernels_circle_pulse_N4_m256_fp32_dram.csv")
STAGE_SOURCES = ("rhs_kernels.cuh", "rhs_order.cu")     # the stage and element kernels' code


def stage_source_hash():
    """sha256 (first 16 hex digits) of the stage kernels' sources, to tell whether a stored
    ncu capture still describes the kernels being timed."""
    import hashlib
    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_1912_06221_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(args, kernel="edge_flux_kernel<float, 4, 1>"):
    """DRAM bytes (read + write) per launch of `kernel`, averaged over the launches of the
    committed ncu capture of this workload (steady state: no cache flush between launches),
    or None for another workload or when the kernels' sources changed after the capture
    (the capture records the source hash on its first line)."""
    if args.m != 256 or args.rk_steps <= 0 or args.precision != "fp32" or not os.path.exists(TRAFFIC_CSV):
        return None, "no capture for this workload"
    import csv
    with open(TRAFFIC_CSV) as fh:
        first = fh.readline()
        if ("source_sha16=" + stage_source_hash()) not in first:
            return None, "stage kernel sources changed since the capture"
        rows = [r for r in csv.DictReader(line for line in fh if not line.startswith("=="))]
    per = {}
    for r in rows:
        if r.get("Kernel Name", "").replace("void ", "").startswith(kernel):
            if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                per.setdefault(r["ID"], 0.0)
                per[r["ID"]] += float(r["Metric Value"].replace(",", ""))
    if not per:
        return None, "kernel not in the capture"
    return float(np.mean(list(per.values()))), "%s (ncu, %d launches, no cache flush)" % (
        os.path.relpath(TRAFFIC_CSV, ROOT), len(per))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alg_bytes_per_element(N, esz):
    """Algorithmic HBM bytes per element per right-hand-side stage of the stored-operator
    form: read the stage input and step start and write the output (3 Np values), the Nfp x
    2Np operator of 1.5 edges, and 56 bytes (FP32; 88 in FP64) of element coefficients and
    edge/element ids.  Intermediates (face fluxes, volume term) are not counted."""
    Np, Nfp = (N + 1) * (N + 2) // 2, N + 1
    return esz * (3 * Np + 3 * Nfp * Np) + (56 if esz == 4 else 88)


# ---------------------------------------------------------------------------------------
# The oracle leg.  Only this leg (and --impl reference) runs the FP64 NumPy oracle: on
# sampled elements of the full-size workload, through patches of their neighbourhoods
# (oracle/patch.py), so the right-hand side and one SSP-RK3 step on those elements are the
# oracle's exact values for the full 131072-triangle mesh.

def oracle_sample(w, seed=0, n_random=512):
    """Sampled elements: random ones, the first and the last (ragged) element tiles, elements
    on the periodic boundary and on the D jump."""
    K = w.K
    rng = np.random.default_rng(seed)
    from synth import centroids
    c = centroids(w.xy, w.tri)
    h = 1.0 / w.m
    r = np.hypot(c[:, 0] - 0.5, c[:, 1] - 0.5)
    on_jump = np.flatnonzero(np.abs(r - 0.25) < h)
    on_edge = np.flatnonzero((c[:, 0] < h) | (c[:, 0] > 1 - h) | (c[:, 1] < h) | (c[:, 1] > 1 - h))
    picks = [rng.choice(K, n_random, replace=False), np.arange(32), np.arange(K - 32, K),
             rng.choice(on_jump, min(64, on_jump.size), replace=False),
             rng.choice(on_edge, min(64, on_edge.size), replace=False)]
    return np.unique(np.concatenate(picks))


def oracle_leg(w, iface, rhs_sample, step_sample, u_rhs, t_rhs, u_step, dt, seconds_budget=10.0):
    """Oracle values on the sampled elements (right-hand side of u_rhs at t_rhs; one SSP-RK3
    step of u_step from t = 0 with dt) and the oracle's own throughput on the right-hand-side
    patch, timed on the host cores (setup excluded)."""
    from oracle.patch import PatchProblem, face_neighbours
    nbr = face_neighbours(w.xy, w.tri)
    t0 = time.perf_counter()
    p1 = PatchProblem(w.xy, w.tri, w.N, w.D_elem, rhs_sample, v=w.v, rings=1, interface=iface, nbr=nbr)
    p3 = PatchProblem(w.xy, w.tri, w.N, w.D_elem, step_sample, v=w.v, rings=3, interface=iface, nbr=nbr)
    t_setup = time.perf_counter() - t0
    rhs = {k: p1.rhs(u, t_rhs) for k, u in u_rhs.items()}
    step = {k: p3.rk3_step(u, 0.0, dt) for k, u in u_step.items()}
    u0 = next(iter(u_rhs.values()))
    n = 0
    t0 = time.perf_counter()
    while True:
        p1.rhs(u0, t_rhs)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds_budget or n >= 2000:
            break
    Np = (w.N + 1) * (w.N + 2) // 2
    gd = p1.patch_elements * Np * n / el / 1e9
    meta = {"kind": "oracle", "cores": 1, "nproc": os.cpu_count(),
            "blas_threads": os.environ.get("OMP_NUM_THREADS"),
            "sample": "FP64 NumPy oracle (Algorithm %s) on a %d-element patch of the full %d-triangle mesh (the "
                      "%d sampled elements and their face neighbours), %d right-hand sides in %.1f s, setup (%.1f s, "
                      "both patches) excluded, BLAS pinned to 1 thread"
                      % ("1" if iface == "alg1" else "2", p1.patch_elements, w.K, len(rhs_sample), n, el, t_setup)}
    return gd, meta, rhs, step


def compare_rows(got, want):
    """Element-wise and normwise relative errors of sampled rows."""
    got = np.asarray(got, float)
    want = np.asarray(want, float)
    d = got - want
    return {"max_abs_over_max_ref": float(np.abs(d).max() / np.abs(want).max()),
            "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(want)),
            "elements": int(want.shape[0])}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import circle_pulse
    from oracle.patch import PatchProblem
    w = circle_pulse(m=args.m, N=N_ORDER)
    sample = oracle_sample(w)
    pp = PatchProblem(w.xy, w.tri, w.N, w.D_elem, sample, v=w.v, rings=1, interface="alg1")
    u = w.u0(pp.mesh.x, pp.mesh.y)
    per_step = 40          # right-hand sides of the patch in one bench step
    for i in range(args.warmup):
        for j in range(per_step):
            pp.problem.rhs(u, 0.0)
    t0 = time.perf_counter()
    for i in range(args.steps):
        for j in range(per_step):
            pp.problem.rhs(u, 0.0)
    el = time.perf_counter() - t0
    val = pp.patch_elements * pp.mesh.ops.Np * per_step * args.steps / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": val, "unit": UNIT, "kind": "oracle", "cores": 1, "nproc": os.cpu_count(),
                             "sample": "FP64 NumPy oracle (Algorithm 1) on a %d-element patch of the full %d-triangle "
                                       "mesh (%d sampled elements and their face neighbours), %d right-hand sides "
                                       "per bench step, setup excluded, BLAS pinned to 1 thread"
                                       % (pp.patch_elements, w.K, len(sample), per_step)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "circle_pulse N=4 (Np=15), %dx%dx2=%d jittered periodic triangles (seed 1), v=(1,0.5), "
                        "D=1 in r<0.25 else 1e-4 (Algorithm 1 interface rule), Gaussian w=0.05, %d SSP-RK3 steps "
                        "at 0.5x stability bound" % (args.m, args.m, 2 * args.m * args.m, args.rk_steps),
            "N": N_ORDER, "triangles": 2 * args.m * args.m, "rk_steps_per_bench_step": args.rk_steps,
            "rhs_per_bench_step": 3 * args.rk_steps,
            "precision": "fp32" if args.precision == "fp32" else "fp32 state, edge flux as split-3xTF32 tensor-core GEMM",
            "l2_flush": "256 MB buffer written between timed steps (outside the events)",
            "parallelism": "replicas" if args.gpus > 1 else "single"}


# ---------------------------------------------------------------------------------------
def spectral_radius(s, torch, iters=50, seed=0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((s.K, s.Np), generator=g, device="cuda", dtype=s.dtype)
    y = torch.empty_like(x)
    rho = 0.0
    for _ in range(iters):
        x /= torch.linalg.vector_norm(x)
        s.rhs_eval(x, y, 0.0)
        rho = float(torch.linalg.vector_norm(y))
        x, y = y, x
    return rho


def run_ours(args):
    import torch
    import __graft_entry__
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_1912_06221_gb300 as rdg
    rdg.load()
    from synth import circle_pulse
    w = circle_pulse(m=args.m, N=N_ORDER)
    gemm = args.precision == "tf32"
    # The paper's Algorithm 1 for the element-wise D: on this 1e4 jump Algorithm 2's operator
    # has eigenvalues with positive real part and the solve grows without bound (reported
    # below as a labelled extra); the kernels and bytes are the same for both rules.
    iface = rdg.IFACE_HARMONIC if gemm else rdg.IFACE_ALG1
    s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=rdg.FP32_3XTF32 if gemm else rdg.FP32,
                   device=local, interface=iface)
    stream = torch.cuda.current_stream()
    xyn = s.node_coords()
    u0_host = w.u0(xyn[..., 0], xyn[..., 1]).astype(np.float32)
    u0 = torch.tensor(u0_host, device="cuda")
    rho = spectral_radius(s, torch)
    dt = 0.5 * 2.5127 / rho
    nrk = args.rk_steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        s.set_state(u0)
        s.solve_to_time(0.0, dt, nrk)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.set_state(u0)
        s.solve_to_time(0.0, dt, nrk)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t_local = sum(a.elapsed_time(b) for a, b in evs)
    t_ms, dofs, rate = aggregate(t_local, s.K * s.Np * 3 * nrk * args.steps, dist, device="cuda")
    value = rate / 1e9
    u_fp32 = s.get_state_host().astype(np.float64)

    # per-kernel times (event-bracketed launches of one more solve)
    s.profile(True)
    s.set_state(u0)
    s.solve_to_time(0.0, dt, 100)
    st = s.kernel_stats()
    s.profile(False)
    edge_n, edge_ms = st["edge"]
    elem_n, elem_ms = st["elem"]
    E, K, Np, Nfp = s.E, s.K, s.Np, s.Nfp
    # the algorithmic bytes of one stage (stored operators, state in and out,
    # coefficients and ids); the stage kernel is the dominant launch
    stage_alg = alg_bytes_per_element(N_ORDER, 4) * K
    # the two kernels' own bytes, intermediates (volume term, face fluxes) included
    edge_bytes = E * ((Nfp * (2 * Np - 1) + 1) * 4 + 8 + Nfp * 4) + K * Np * 4 + K * Np * 4 + K * 5 * 4
    if gemm:   # parameter records (16-byte words) instead of operators, plus the face-pair word
        edge_bytes = E * (((2 * Np + Nfp + 3 + 3) // 4) * 16 + 12 + Nfp * 4) + K * Np * 4 + K * Np * 4 + K * 5 * 4
    elem_bytes = int(K * ((3 + 2.0 / 3.0) * Np * 4 + 12 + 4) + E * Nfp * 4)
    peak, peak_kind = measured_peaks()
    edge_avg = edge_ms / edge_n
    elem_avg = elem_ms / elem_n
    ach = stage_alg / (edge_avg / 1e3) / 1e9
    traffic, traffic_src = (None, "GEMM form: no capture") if gemm else profiled_traffic(args)
    kname = "edge_gemm_pipe_kernel<4>" if gemm else "edge_flux_kernel<float,4,VOL=1>"
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind, "traffic": traffic,
            "traffic_source": traffic_src,
            "alg_bytes_per_launch": stage_alg,
            "alg_bytes_rule": "%d B per element per stage (stored operators, state in/out, coefficients, ids) x K"
                              % alg_bytes_per_element(N_ORDER, 4),
            "avg_launch_us": edge_avg * 1e3,
            "share_of_kernel_time": edge_ms / (edge_ms + elem_ms),
            "kernel_own_bytes": {"edge_and_volume_blocks": edge_bytes, "element_updates": elem_bytes,
                                 "note": "reads and writes of the stage's two parts, volume-term and face-flux "
                                         "round trips included (they mostly hit L2 in steady state)"},
            "elem_kernel": {"name": "elem_lite_kernel<float,4,MODE>", "avg_launch_us": elem_avg * 1e3}}
    # the whole stage inside the replayed graph (programmatic dependent launch): the same
    # algorithmic bytes over the timed solve's time per stage
    t_stage_s = t_ms / args.steps / (3 * nrk) / 1e3
    roof["whole_stage_in_graph"] = {"alg_bytes": stage_alg, "us": t_stage_s * 1e6,
                                    "achieved_gbs": stage_alg / t_stage_s / 1e9,
                                    "frac": stage_alg / t_stage_s / 1e9 / peak}

    # the compute side: measured FMA rates (in-process, this GPU at its current clocks) and
    # the flops per element per stage, 8 Np^2 + 12 Np Nfp + 12 Np
    p32, p64 = rdg.peak_fma(local, rdg.FP32), rdg.peak_fma(local, rdg.FP64)
    flops_stage = (8 * Np * Np + 12 * Np * Nfp + 12 * Np) * K
    roof["rhs_roofline"] = {"t_bytes_us": stage_alg / (peak * 1e9) * 1e6, "t_flops_us": flops_stage / p32 * 1e6,
                            "bound": "hbm" if stage_alg / (peak * 1e9) >= flops_stage / p32 else "fp32",
                            "frac": max(stage_alg / (peak * 1e9), flops_stage / p32) / t_stage_s,
                            "flops_per_stage": flops_stage}
    compute_peaks = {"fp32_tflops": p32 / 1e12, "fp64_tflops": p64 / 1e12,
                     "how": "rdg_peak_fma: independent FMA chains on every SM, CUDA events, best of 4"}
    # the size-matched bound: a plain streaming read of the stage's algorithmic bytes and of
    # the operators alone, each a standalone launch (rdg_stream_read)
    w_bytes = ((E + 31) // 32) * ((Nfp * (2 * Np - 1) + 1 + 3) // 4) * 32 * 16
    t_rd_stage = rdg.stream_read_seconds(local, stage_alg)
    t_rd_w = rdg.stream_read_seconds(local, w_bytes)
    roof["size_matched_read"] = {"stage_alg_bytes": stage_alg, "read_us": t_rd_stage * 1e6,
                                 "read_gbs": stage_alg / t_rd_stage / 1e9,
                                 "operator_bytes": w_bytes, "operator_read_us": t_rd_w * 1e6,
                                 "stage_us_in_graph": t_stage_s * 1e6,
                                 "stage_time_over_read_time": t_stage_s / t_rd_stage,
                                 "how": "rdg_stream_read: float4 evict-first grid-stride read, L2 flushed, "
                                        "median of 8 standalone launches"}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_t = []
    in_pinned = torch.from_numpy(u0_host).pin_memory()       # inputs in pinned host memory
    out_pinned = torch.empty_like(in_pinned).pin_memory()
    for i in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_state(in_pinned)                  # host -> device copy of the step's input
        s.solve_to_time(0.0, dt, nrk)
        s.get_state(out_pinned)                 # device -> host copy of the result (waits for it)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = s.K * s.Np * 3 * nrk * world / (float(np.mean(e2e_t))) / 1e9

    fp64 = None
    s64_head = None
    if not args.no_fp64:
        # the same solve in FP64 on the GPU for each interface rule: FP32-vs-FP64 differences
        # at t_final and the size of the solution (Algorithm 2 grows on this jump)
        fp64 = {}
        u64s = {}
        rules = ((rdg.IFACE_ALG1, "algorithm1"), (rdg.IFACE_ALG2, "algorithm2"), (rdg.IFACE_HARMONIC, "harmonic"))
        for rule, name in rules:
            if rule == iface:
                u32 = u_fp32
            else:
                s32 = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=rdg.FP32, device=local, interface=rule)
                s32.set_state(u0)
                s32.solve_to_time(0.0, dt, nrk)
                u32 = s32.get_state_host().astype(np.float64)
                s32.close()
            s64 = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=rdg.FP64, device=local, interface=rule)
            u064 = torch.tensor(w.u0(xyn[..., 0], xyn[..., 1]), device="cuda")
            s64.set_state(u064)
            s64.solve_to_time(0.0, dt, 16)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s64.set_state(u064)
            a.record(stream)
            s64.solve_to_time(0.0, dt, nrk)
            b.record(stream)
            torch.cuda.synchronize()
            t64 = a.elapsed_time(b)
            u64 = s64.get_state_host()
            u64s[name] = u64
            fp64[name] = {"fp64_value": s.K * s.Np * 3 * nrk / (t64 / 1e3) / 1e9, "unit": UNIT,
                          "fp32_rel_l2_vs_fp64": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
                          "fp32_rel_linf_vs_fp64": float(np.abs(u32 - u64).max() / np.abs(u64).max()),
                          "max_abs_u_t_final": float(np.abs(u64).max()), "t_final": nrk * dt,
                          "roofline_fp64": {"t_bytes_us": alg_bytes_per_element(N_ORDER, 8) * K / (peak * 1e9) * 1e6,
                                            "t_flops_us": flops_stage / p64 * 1e6,
                                            "stage_us": t64 / 1e3 / (3 * nrk) * 1e6,
                                            "frac": max(alg_bytes_per_element(N_ORDER, 8) * K / (peak * 1e9),
                                                        flops_stage / p64) / (t64 / 1e3 / (3 * nrk))},
                          "role": ("headline" if rule == iface else
                                   "extra: grows without bound on this jump" if rule == rdg.IFACE_ALG2 else "extra")}
            if name == "algorithm1":
                s64_head = s64
            else:
                s64.close()

    # the same solve with the GEMM form of the edge flux (tcgen05, split 3xTF32)
    tf32 = None
    if fp64 and not gemm:
        # harmonic interface rule (the GEMM form folds a single edge coefficient)
        st_ = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=rdg.FP32_3XTF32, device=local,
                         interface=rdg.IFACE_HARMONIC)
        st_.set_state(u0)
        st_.solve_to_time(0.0, dt, nrk)
        torch.cuda.synchronize()
        tt = []
        for _ in range(max(2, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st_.set_state(u0)
            st_.solve_to_time(0.0, dt, nrk)
            b.record(stream)
            torch.cuda.synchronize()
            tt.append(a.elapsed_time(b))
        ut = st_.get_state_host().astype(np.float64)
        st_.synchronize()
        st_.close()
        u64 = u64s["harmonic"]
        # its own roofline: per element per stage the state (3 Np values), 1.5 parameter
        # records (16-byte words) and the coefficients and ids; the split products on the
        # tensor cores (2 sides x NPAD x KP x 2 flop x 3 products per edge); TF32 peak = the
        # measured bf16 burst rate x the nominal TF32/BF16 ratio 1.1/2.25
        pw4 = (2 * Np + Nfp + 3 + 3) // 4
        npad, kp = (Np * Nfp + 15) // 16 * 16, (2 * Np + 7) // 8 * 8
        g_bytes = K * (4 * 3 * Np + 56) + E * pw4 * 16
        g_flops = E * 2 * npad * kp * 2 * 3
        bf16 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] * 1e12 \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1.9e15
        p_tf32 = bf16 * 1.1 / 2.25
        t_g = float(np.median(tt)) / 1e3 / (3 * nrk)
        t_roof_g = max(g_bytes / (peak * 1e9), g_flops / p_tf32)
        tf32 = {"value": s.K * s.Np * 3 * nrk / (float(np.median(tt)) / 1e3) / 1e9, "unit": UNIT,
                "roofline": {"alg_bytes_per_stage": g_bytes, "tensor_flops_per_stage": g_flops,
                             "t_bytes_us": g_bytes / (peak * 1e9) * 1e6, "t_tensor_us": g_flops / p_tf32 * 1e6,
                             "tf32_peak_tflops": p_tf32 / 1e12, "stage_us": t_g * 1e6, "frac": t_roof_g / t_g},
                "kernel": "edge_gemm_pipe_kernel<4> (warp-specialised, tcgen05.mma kind::tf32, split 3xTF32) + elem_lite_kernel",
                "rel_l2_vs_fp64": float(np.linalg.norm(ut - u64) / np.linalg.norm(u64)),
                "rel_linf_vs_fp64": float(np.abs(ut - u64).max() / np.abs(u64).max()),
                "interface": "harmonic"}

    # the oracle leg (rank 0 of a single-GPU run): the FP64 oracle on sampled elements of the
    # full mesh, element by element against the GPU's right-hand side and one SSP-RK3 step,
    # FP32 and FP64, and the oracle's own throughput as the CPU baseline
    cpu = None
    vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not gemm:
        samp = oracle_sample(w)
        samp3 = oracle_sample(w, seed=1, n_random=64)[::2]
        ur = np.random.default_rng(5).standard_normal((s.K, s.Np))
        ins = {"pulse": w.u0(xyn[..., 0], xyn[..., 1]), "random": ur}
        gpu = {}
        solvers = [("fp32", s, np.float32)] + ([("fp64", s64_head, np.float64)] if s64_head is not None else [])
        for pname, sv, npt in solvers:
            for iname, uin in ins.items():
                ud = torch.tensor(uin.astype(npt), device="cuda")
                rd = torch.empty_like(ud)
                sv.rhs_eval(ud, rd, 0.0)
                sv.synchronize()
                gpu[(pname, "rhs", iname)] = rd.cpu().numpy()[samp]
            sv.set_state(torch.tensor(ins["pulse"].astype(npt), device="cuda"))
            sv.rk_step(0.0, dt)
            gpu[(pname, "step", "pulse")] = sv.get_state_host()[samp3]
        # the oracle sees the values the GPU saw (FP32 inputs rounded as the FP32 path reads them)
        u_rhs = {iname: uin for iname, uin in ins.items()}
        u_rhs32 = {iname: uin.astype(np.float32).astype(np.float64) for iname, uin in ins.items()}
        gd, meta, o_rhs, o_step = oracle_leg(w, "alg1", samp, samp3, {**{k + "64": v for k, v in u_rhs.items()},
                                                                       **{k + "32": v for k, v in u_rhs32.items()}},
                                             0.0, {"pulse64": ins["pulse"],
                                                   "pulse32": ins["pulse"].astype(np.float32).astype(np.float64)}, dt)
        cpu = dict(value=gd, unit=UNIT, **meta)
        vs_oracle = {"interface": "algorithm1", "sampled_elements_rhs": int(len(samp)),
                     "sampled_elements_step": int(len(samp3)),
                     "tolerance": {"fp32": 1e-5, "fp64": 1e-12}}
        for pname, _, _ in solvers:
            tag = "32" if pname == "fp32" else "64"
            vs_oracle[pname] = {
                "rhs_pulse": compare_rows(gpu[(pname, "rhs", "pulse")], o_rhs["pulse" + tag]),
                "rhs_random": compare_rows(gpu[(pname, "rhs", "random")], o_rhs["random" + tag]),
                "rk3_step_pulse": compare_rows(gpu[(pname, "step", "pulse")], o_step["pulse" + tag])}
    if s64_head is not None:
        s64_head.close()

    per_solve = (1 + (nrk // 16) * (16 * 6 + 1) if nrk >= 16 else 0) + (nrk % 16) * 6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args), "dt": dt, "rho": rho,
            "clocks": clk, "roofline": roof, "cpu_baseline": cpu, "fp32_vs_oracle_full_mesh": vs_oracle,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(u0_host.nbytes),
                    "d2h_bytes_per_step": int(out_pinned.numel() * out_pinned.element_size())},
            "gpu_launches": per_solve * args.steps, "compute_peaks": compute_peaks,
            "fp64_gpu": fp64, "fp32_3xtf32": tf32}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_serve(args):
    """Poisson stream of solve requests (rate 200/s unless --serve-rate, seed 3): jittered periodic meshes of
    log-uniform size 1e3..1e6 triangles, N in 2..6, element-wise D with a log-uniform contrast
    in [1, 1e4] across a random circle, v in [-1,1]^2, 50..500 SSP-RK3 steps, FP32, 120 GB
    admission budget; FP64 spot check of the requests the stream marks (1%).  Prints one
    JSON line with p50/p99 latency and the aggregate GDOF/s."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    from paper_1912_06221_gb300.serve import Server, SolveRequest, latency_stats, solve_alone
    from synth import serve_stream
    stream = serve_stream(seed=3, nreq=args.serve_requests, rate=args.serve_rate, build_mesh=False)
    reqs = []
    for r in stream:
        w = r.workload
        reqs.append(SolveRequest(r.rid, r.arrival, None, None, w.N, None, w.v, w.u0, w.steps,
                                 build=w.meta["build"], n_triangles=w.meta["triangles"]))
    srv = Server(budget_bytes=120 * 10 ** 9, max_slots=args.serve_slots, chunk=16,
                 setup_workers=args.serve_setup_workers)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    st = latency_stats(res)
    by_id = {r.rid: r for r in res}
    # the requests the stream marks for an FP64 check (1%), topped up in arrival order to at
    # least 1% of the requests served
    marked = [r.rid for r in stream if r.fp64_check]
    for r in stream:
        if len(marked) >= math.ceil(0.01 * len(stream)):
            break
        if r.rid not in marked:
            marked.append(r.rid)
    checks = []
    for r in stream:
        if r.rid in marked:
            got = by_id[r.rid]
            ref = solve_alone(reqs[r.rid], got.dt, precision=rdg.FP64)
            checks.append({"rid": r.rid, "triangles": got.K, "N": reqs[r.rid].N,
                           "fp32_rel_l2_vs_fp64": float(np.linalg.norm(got.state - ref) / np.linalg.norm(ref))})
    line = {"metric": "serve p50/p99 latency and aggregate GDOF/s", "value": st["gdof_per_s"], "unit": "GDOF/s",
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"], "n_requests": st["n"],
            "makespan_s": st["makespan_s"], "wall_s": wall, "peak_admitted_bytes": srv.peak_in_use,
            "max_resident": srv.max_concurrent, "budget_bytes": srv.budget, "fp64_spot_checks": checks,
            "setup_seconds_summed": srv.setup_summary(), "setup_workers": args.serve_setup_workers,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Poisson stream, rate %g/s, seed 3, %d requests, K log-uniform 1e3..1e6, "
                                   "N 2..6, D contrast log-uniform 1..1e4 across a random circle, 50..500 steps"
                                   % (args.serve_rate, args.serve_requests)}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 independent periodic heat problems (seed 2): mesh side uniform in 8..256 cells
    (2 triangles per cell, 10% jitter), N uniform in 1..6, D log-uniform in [1e-3, 1], random
    low-mode Fourier u0, 100 SSP-RK3 steps each at 0.5 x its stability bound, FP32, all
    members stepped together by the library's batch: one persistent launch per chunk of steps
    walking a (member, phase, tile) work list, replayed from a CUDA graph, with the tile
    mapping per order and the chunk chosen by the autotuner (or the branch graph, if the tuner
    measures it faster).  One bench step = the 100 steps of all 64 problems.  Beside it: the same problems solved one after another (each with its own
    graph), and every member's FP32 state against its FP64 GPU solve."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    from synth import batched_heat
    torch.cuda.set_device(0)
    from paper_1912_06221_gb300 import autotune
    probs = batched_heat(seed=2)
    steps = probs[0].steps
    solvers, dts, u0s = [], [], []
    t_tune = time.perf_counter()
    choices = [autotune.choose_precision(w.xy, w.tri, w.N, w.D_elem, v=w.v) for w in probs]
    t_tune = time.perf_counter() - t_tune
    t_setup = time.perf_counter()
    for w, ch in zip(probs, choices):
        s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=ch["precision"])
        xyn = s.node_coords()
        u0 = np.ascontiguousarray(w.u0(xyn[..., 0], xyn[..., 1]))
        rho = spectral_radius(s, torch, iters=30)
        dts.append(w.dt_factor * 2.5127 / rho)
        u0s.append(torch.tensor(u0, dtype=torch.float32, device="cuda"))
        solvers.append(s)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    units = sum(s.K * s.Np * 3 * steps for s in solvers)
    stream = torch.cuda.current_stream()
    bt = rdg.Batch(chunk=args.batch_chunk)
    for s, dt in zip(solvers, dts):
        bt.add(s, dt)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(batched):
        for s, u in zip(solvers, u0s):
            s.set_state(u)
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if batched:
            # the heat members have no time-dependent forcing: the time the batch carries
            # on from does not enter their results
            bt.step(steps)
        else:
            for s, dt in zip(solvers, dts):
                s.solve_to_time(0.0, dt, steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    chunk_tune = autotune.choose_chunk(bt, solvers, u0s, steps, candidates=(5, 10, 25, 50, 100))
    tile_tune = autotune.choose_tiles(bt, solvers, u0s, steps)
    for _ in range(args.warmup):
        one(True)
        one(False)
    clk = ClockSampler(0)
    clk.start()
    tb = [one(True) for _ in range(args.steps)]
    clocks = clk.stop()
    ts = [one(False) for _ in range(args.steps)]
    bt.synchronize()
    ms_b, ms_s = float(np.median(tb)), float(np.median(ts))
    # FP32 batch result against each member's FP64 solve on the GPU
    one(True)
    errs = []
    for w, s, dt, u in zip(probs, solvers, dts, u0s):
        s64 = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, v=w.v, precision=rdg.FP64)
        s64.set_state(u.double())
        # (FP32 members are stepped by whichever FP32-accurate form the tuner picked)
        s64.solve_to_time(0.0, dt, steps)
        a64 = s64.get_state_host()
        s64.close()
        a32 = s.get_state_host().astype(np.float64)
        errs.append(float(np.linalg.norm(a32 - a64) / np.linalg.norm(a64)))
    line = {"metric": "batched uneven solves, aggregate GDOF/s", "value": units / (ms_b / 1e3) / 1e9,
            "batch_form": "one persistent launch per chunk of steps (work list over members, phases, tiles)"
                          if bt.mode == rdg.BATCH_PERSISTENT else "CUDA graph of per-member branches",
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 periodic heat problems (seed 2), side 8..256, N 1..6, D log-uniform "
                                   "[1e-3,1], Fourier u0, 100 SSP-RK3 steps each, FP32",
                       "triangles_total": int(sum(s.K for s in solvers)),
                       "dof_total": int(sum(s.K * s.Np for s in solvers)),
                       "orders": [int(w.N) for w in probs], "graph_chunk": chunk_tune["chunk"],
                       "l2_flush": "256 MB buffer written before each timed step (outside the events)"},
            "sequential": {"value": units / (ms_s / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms_s,
                           "note": "the same 64 solves one after another, each replaying its own graph"},
            "fp32_rel_l2_vs_fp64": {"max": max(errs), "median": float(np.median(errs))},
            "setup_s": t_setup, "clocks": clocks,
            "autotune": {"seconds": t_tune,
                         "precision_by_order_and_size_class": sorted(
                             {(int(w.N), autotune.size_class(w.K), "fp32" if c["precision"] == rdg.FP32 else "fp32_3xtf32",
                               json.dumps(c["ms"])) for w, c in zip(probs, choices)}),
                         "graph_chunk_ms": chunk_tune["ms"],
                         "batch_form": tile_tune["mode"],
                         "edges_per_thread_tiles_per_item_by_order": tile_tune["edges_per_thread_tiles_per_item"],
                         "tile_and_form_ms": tile_tune["ms"]}}
    print(json.dumps(line), flush=True)
    bt.close()
    for s in solvers:
        s.close()


def _gpu_rho(s, torch, iters=40):
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((s.K, s.Np), generator=g, device="cuda", dtype=s.dtype)
    y = torch.empty_like(x)
    for _ in range(iters):
        x /= torch.linalg.vector_norm(x)
        s.rhs_eval(x, y, 0.0)
        x, y = y, x
    return float(torch.linalg.vector_norm(x))


def run_paper_problems(args):
    """The paper's verification problems (Sec. 5.1 Gaussian diffusion, Sec. 5.2 Gaussian
    advection-diffusion; D = 1, D0 = 2, t = 0.5) on stand-ins for its grid-a series (32 ..
    8192 triangles, every triangle pair a parallelogram, periodic 10 x 10 square with the
    image-sum exact solution), FP64 on the GPU with the paper's five-stage fourth-order
    Runge-Kutta scheme at a time step fixed by the finest mesh.  Reports L2 / L_inf errors
    (Eqs. L2_norm_cellUnit, Linf_norm_cellUnit, in FP64 on the GPU), two-mesh orders, and the paper's Tables
    purediff_ooa / adv_diff_ooa (grid a) beside them."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    from synth import paper_gaussian
    tables = {False: {1: 2.015, 2: 2.828, 3: 4.005}, True: {1: 1.690, 2: 2.629, 3: 3.970}}
    ms = (4, 8, 16, 32, 64)
    out = {}
    t_start = time.perf_counter()
    for adv in (False, True):
        for N in (1, 2, 3):
            wf = paper_gaussian(ms[-1], N, advection=adv)
            s = rdg.Solver(wf.xy, wf.tri, N, wf.D_elem, v=wf.v, period=(10.0, 10.0), precision=rdg.FP64)
            n = int(math.ceil(0.5 / (0.5 * 2.5127 / _gpu_rho(s, torch))))
            s.close()
            dt = 0.5 / n
            l2, li = [], []
            for m in ms:
                w = paper_gaussian(m, N, advection=adv)
                s = rdg.Solver(w.xy, w.tri, N, w.D_elem, v=w.v, period=(10.0, 10.0), precision=rdg.FP64)
                s.set_integrator(rdg.LSRK54)
                xyn = s.node_coords()
                s.set_state(w.exact(xyn[..., 0], xyn[..., 1], 0.0))
                s.solve_to_time(0.0, dt, n)
                q = s.error_quadrature()
                e2, ei = s.error_norms(w.exact(q[..., 0], q[..., 1], 0.5))     # FP64 on the GPU
                s.synchronize()
                s.close()
                l2.append(e2)
                li.append(ei)
            key = "%s_P%d" % ("advection_diffusion" if adv else "diffusion", N)
            out[key] = {"triangles": [2 * m * m for m in ms], "steps": n, "dt": dt, "l2": l2, "linf": li,
                        "l2_orders": [math.log2(l2[i] / l2[i + 1]) for i in range(len(ms) - 1)],
                        "linf_orders": [math.log2(li[i] / li[i + 1]) for i in range(len(ms) - 1)],
                        "paper_table_l2_grid_a": tables[adv][N]}
    line = {"metric": "observed order of accuracy, paper verification problems", "unit": "order",
            "value": out["diffusion_P3"]["l2_orders"][-1], "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "integrator": "LSRK5(4)", "seconds": time.perf_counter() - t_start,
            "config": {"workload": "Gaussian diffusion and advection-diffusion (D=1, D0=2, a=(6,6)), t=0.5, "
                                   "grid-a series 32..8192 triangles, periodic 10x10"},
            "results": out}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """N = 3 manufactured solution u = sin(pi x) sin(pi y) cos t (Dirichlet, D = 1) in FP64, FP32
    and FP32 with the split-3xTF32 GEMM form.  Meshes 32^2..128^2 x 2 run to T = 2^-10 (L2 error
    against the exact solution, orders); 256^2..1024^2 x 2 (up to 2.1M triangles) run 30 steps
    at 0.5 x the stability bound (difference to the FP64 GPU state and throughput), since the
    full T takes ~1e5..1e6 steps there."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    from synth import manufactured_dirichlet
    modes = (("fp64", rdg.FP64), ("fp32", rdg.FP32), ("fp32_3xtf32", rdg.FP32_3XTF32))
    rows = []
    for m in (32, 64, 128, 256, 512, 1024):
        w = manufactured_dirichlet(m, N=3)
        full = m <= 128
        row = {"m": m, "triangles": 2 * m * m}
        states = {}
        for name, prec in modes:
            s = rdg.Solver(w.xy, w.tri, w.N, w.D_elem, bc=rdg.BC_DIRICHLET, period=None, precision=prec)
            xyn = s.node_coords()
            gxy = s.ghost_coords()
            s.set_forcing([(f(xyn[..., 0], xyn[..., 1]), k, o) for f, k, o in
                           zip(w.source.funcs, w.source.kinds, w.source.omegas)],
                          [(f(gxy[..., 0], gxy[..., 1]), k, o) for f, k, o in
                           zip(w.ghost.funcs, w.ghost.kinds, w.ghost.omegas)])
            if "dt" not in row:
                rho = _gpu_rho(s, torch)
                dt = 0.5 * 2.5127 / rho
                T = w.meta["T"]
                n = int(math.ceil(T / dt)) if full else 30
                row["dt"] = T / n if full else dt
                row["steps"] = n
            u0 = np.ascontiguousarray(w.exact(xyn[..., 0], xyn[..., 1], 0.0), dtype=s.np_dtype)
            s.set_state(u0)
            s.solve_to_time(0.0, row["dt"], min(row["steps"], 16))
            torch.cuda.synchronize()
            s.set_state(u0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s.solve_to_time(0.0, row["dt"], row["steps"])
            b.record()
            torch.cuda.synchronize()
            ms_ = a.elapsed_time(b)
            u = s.get_state_host().astype(np.float64)
            s.synchronize()
            row[name + "_gdof_per_s"] = s.K * s.Np * 3 * row["steps"] / (ms_ / 1e3) / 1e9
            states[name] = u
            if full:
                q = s.error_quadrature()
                e2, ei = s.error_norms(w.exact(q[..., 0], q[..., 1], row["dt"] * row["steps"]))   # FP64 on the GPU
                row[name + "_l2_err"] = e2
                row[name + "_linf_err"] = ei
            s.close()
        for name in ("fp32", "fp32_3xtf32"):
            d = states[name] - states["fp64"]
            row[name + "_rel_l2_vs_fp64"] = float(np.linalg.norm(d) / np.linalg.norm(states["fp64"]))
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    for name, _ in modes:
        e = [r[name + "_l2_err"] for r in rows if name + "_l2_err" in r]
        for i, r in enumerate([r for r in rows if name + "_l2_err" in r][1:]):
            r[name + "_l2_order"] = math.log2(e[i] / e[i + 1])
    line = {"metric": "precision sweep, N=3 manufactured solution", "unit": "rel L2 / order / GDOF/s",
            "value": rows[-1]["fp32_gdof_per_s"], "higher_is_better": True, "dtype": "f64/f32/3xtf32",
            "data": "synthetic", "config": {"workload": "u = sin(pi x) sin(pi y) cos t, Dirichlet, D = 1, N = 3, "
                                                        "meshes 32^2..1024^2 x 2, seed 10"}, "rows": rows}
    print(json.dumps(line), flush=True)


def run_orders(args):
    """Graph-replayed SSP-RK3 stage of the circle pulse workload (m x m x 2 triangles) at each
    order, FP32 and FP64: microseconds per stage (the default kernel form, and both forms:
    stage kernel + element kernel, or the one-kernel stage), GDOF/s and the stage's
    algorithmic HBM bytes (stored operators, state in and out, coefficients and ids) per
    second."""
    import torch
    import paper_1912_06221_gb300 as rdg
    from synth import circle_pulse
    orders = [int(x) for x in args.orders_list.split(",") if x]
    rows = []
    clk = ClockSampler(0)
    clk.start()
    for N in orders:
        w = circle_pulse(m=args.m, N=N)
        for prec, esz, name in ((rdg.FP32, 4, "fp32"), (rdg.FP64, 8, "fp64")):
            if name not in args.orders_precisions.split(","):
                continue
            s = rdg.Solver(w.xy, w.tri, N, w.D_elem, v=w.v, precision=prec)
            u = torch.zeros((s.K, s.Np), dtype=s.dtype, device="cuda")
            dt = 1e-9
            per = 32 * 3                          # stages per timed replay (32 steps)
            forms = {}
            for fname, form in (("two_kernels", rdg.STAGE_TWO_KERNELS), ("one_kernel", rdg.STAGE_ONE_KERNEL),
                                ("default", rdg.STAGE_AUTO)):
                s.set_stage_form(form)
                s.set_state(u)
                for _ in range(max(args.warmup, 1)):
                    s.solve_to_time(0.0, dt, 32)
                torch.cuda.synchronize()
                ts = []
                for _ in range(max(args.steps, 1)):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(s.stream)
                    s.solve_to_time(0.0, dt, 32)
                    b.record(s.stream)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b) * 1e3 / per)
                forms[fname] = float(np.median(ts))
            us = forms["default"]
            default_form = "one_kernel" if s.stage_form == rdg.STAGE_ONE_KERNEL else "two_kernels"
            E, K, Np, Nfp = s.E, s.K, s.Np, N + 1
            w_bytes = E * (Nfp * (2 * Np - 1) + 1) * esz
            # the algorithmic bytes per element (stored operators, state in and out,
            # coefficients, ids); beside them the two kernels' own bytes at this order and
            # precision: edge pass (operators, edge ids, face fluxes, stage input, volume term,
            # element coefficients) and element pass (volume term, stage input, step start in
            # two of three stages, output, ids, 1/J, face fluxes)
            alg = alg_bytes_per_element(N, esz) * K
            own = (E * ((Nfp * (2 * Np - 1) + 1) * esz + 8 + Nfp * esz) + 2 * K * Np * esz + K * 5 * esz
                   + int(K * ((3 + 2.0 / 3.0) * Np * esz + 12 + esz) + E * Nfp * esz))
            rows.append({"N": N, "precision": name, "stage_us": us, "stage_form": default_form,
                         "stage_us_two_kernels": forms["two_kernels"], "stage_us_one_kernel": forms["one_kernel"],
                         "gdofs": s.K * Np / (us * 1e-6) / 1e9,
                         "operator_mb": w_bytes / 1e6, "alg_mb": alg / 1e6, "alg_gbs": alg / (us * 1e-6) / 1e9,
                         "kernels_own_mb": own / 1e6})
            s.synchronize()
            s.close()
    clocks = clk.stop()
    peak, src = measured_peaks()
    for r in rows:
        r["frac_of_%s_hbm" % src] = r["alg_gbs"] / peak
    line = {"metric": "stage time per order", "value": None, "unit": "us", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": "circle_pulse %dx%dx2=%d jittered periodic triangles (seed 1), v=(1,0.5), "
                                   "D=1 in r<0.25 else 1e-4, zero state, 32 SSP-RK3 steps per timed graph replay"
                                   % (args.m, args.m, 2 * args.m * args.m),
                       "l2_flush": "none: operators above 129 MB (FP32 N >= 5, FP64 N >= 4) stream from HBM; "
                                   "smaller orders partly hit L2 across replays"},
            "orders": rows, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_hbm_read(args):
    """Plain streaming reads (rdg_stream_read) of 115 MiB, 150 MiB and 1 GiB, event-timed: how
    the reachable read bandwidth of one standalone launch depends on its size."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06221_gb300 as rdg
    rows = []
    for mib in (115, 150, 1024):
        t = rdg.stream_read_seconds(0, mib << 20)
        rows.append({"bytes": mib << 20, "us": t * 1e6, "gbs": (mib << 20) / t / 1e9})
    (b1, t1), (b2, t2) = [(r["bytes"], r["us"]) for r in rows[1:]]
    slope = (t2 - t1) / (b2 - b1)
    line = {"metric": "streaming read time by size", "unit": "us", "rows": rows,
            "asymptotic_gbs": 1e-3 / slope, "fixed_us": t1 - slope * b1, "data": "synthetic"}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve:
        run_serve(a)
    elif a.batch:
        run_batch(a)
    elif a.paper_problems:
        run_paper_problems(a)
    elif a.sweep:
        run_sweep(a)
    elif a.orders:
        run_orders(a)
    elif a.hbm_read:
        run_hbm_read(a)
    else:
        run_ours(a)
