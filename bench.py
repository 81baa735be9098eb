"""Benchmark of the KIFMM Kelvin matvec on GB300 (one JSON line on rank 0).

Workload: 1,000,000 source = target points sampled area-uniformly on the surface of a
2 x 1 x 1 box with 20 spherical voids (radius 0.05-0.15), FP32 positions, unit normals out
of the material, N(0,1) single- and double-layer 3-vector densities, multipole order p = 6
(152-point equivalent surfaces), leaf cap 64, G = 1, nu = 0.3.  One step = one pass of the
hot path: octree build (Morton keys, radix sort, split, U/V/W/X lists) + one FMM evaluation
of the single + double layer sum (S2M, M2M, M2L, P2L, L2L, L2P, M2P, P2P).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (weak scaling, no collective on the data path);
value = all ranks' targets / the slowest rank's time.  --impl reference times the FP64 CPU
oracle (direct summation) on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec targets/sec (Kelvin SL+DL, 3-vec) & BEM solves/sec at 1e-6 residual; P2P % FP32 peak"
WORKLOAD = "KIFMM matvec, 1e6 surface points (2x1x1 box + 20 spherical voids), Kelvin SL+DL, p=6, leaf cap 64"
N_POINTS = 1_000_000
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# algorithmic FP32 operations per pair (counted from the kernel formulas, FMA = 2)
FLOPS_SLDL = 61   # single + double layer displacement
FLOPS_SL = 30     # single layer only (equivalent densities: L2P, M2P)
L2_FLUSH_BYTES = 512 << 20


def fp32_peak_tflops(mhz):
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(n):
    """Seeded inputs, rounded to FP32 once so the GPU and the FP64 oracle sum the same data."""
    import workloads as W
    pts, nrm = W.box_with_voids_points(n, n_voids=20)
    sl, dl = W.densities(n)
    return tuple(np.asarray(a, np.float32).astype(np.float64) for a in (pts, nrm, sl, dl))


def cpu_oracle_sample(pts, nrm, sl, dl, k):
    """FP64 oracle direct sum at k sampled targets; returns (idx, values, seconds)."""
    import oracle as O
    import workloads as W
    idx = W.subsample(len(pts), k)
    t = time.perf_counter()
    ref = O.direct_disp(pts[idx], pts, nrm, sl, dl, 1.0, 0.3)
    return idx, ref, time.perf_counter() - t


def host_threads():
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env else os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    pts, nrm, sl, dl = workload(N_POINTS)
    k = args.ref_sample
    times = []
    for s in range(args.warmup + args.steps):
        _, _, dt = cpu_oracle_sample(pts, nrm, sl, dl, k)
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = k / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle, all-pairs direct sum",
                       "sample": f"{k} targets x {N_POINTS} sources per step"},
            "cpu_baseline": {"value": value, "unit": "targets/s", "cores": host_threads(), "kind": "oracle",
                             "sample": f"{k} of {N_POINTS} targets, all {N_POINTS} sources, per step"},
            "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--cpu-sample", type=int, default=2000)
    ap.add_argument("--ref-sample", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1612_04082_gb300 as K

    dev = torch.device("cuda", local)
    pts, nrm, sl, dl = workload(args.n)
    x = torch.tensor(pts, dtype=torch.float32, device=dev)
    nn = torch.tensor(nrm, dtype=torch.float32, device=dev)
    s = torch.tensor(sl, dtype=torch.float32, device=dev)
    d = torch.tensor(dl, dtype=torch.float32, device=dev)
    out = torch.empty(args.n, 3, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    f = K.Kfmm(p=6, leaf_cap=64, device=local)
    f.set_material(K.material_K(1.0, 0.3), 1.0)
    f.set_stream(stream)

    def step():
        f.build(x, nn, x)
        f.eval(s, d, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = f.stats()

    # ---- timed region: K steps, per-step CUDA events on the launching stream
    f.set_profiling(True)
    f.phase_times(reset=True)
    launches0 = f.stats()["kernel_launches"]
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    launches = (f.stats()["kernel_launches"] - launches0) // max(1, args.steps)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    phases = f.phase_times(reset=True)
    f.set_profiling(False)
    ms = float(np.mean(step_ms))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.n / (ms / 1e3)
    ph_ms = {k: v[0] / max(1, args.steps) for k, v in phases.items()}
    eval_ms = sum(v for k, v in ph_ms.items() if k != "tree")

    # ---- end to end through the C-ABI with host buffers (H2D and D2H inside the timing)
    hx = torch.tensor(pts, dtype=torch.float32).pin_memory()
    hn = torch.tensor(nrm, dtype=torch.float32).pin_memory()
    hs = torch.tensor(sl, dtype=torch.float32).pin_memory()
    hd = torch.tensor(dl, dtype=torch.float32).pin_memory()
    ho = torch.empty(args.n, 3, dtype=torch.float32).pin_memory()
    e2e_t = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f.build(hx, hn, hx)
        f.eval(hs, hd, ho)
        torch.cuda.synchronize(dev)
        if k >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    h2d = 4 * 3 * args.n * 4  # points (as sources and targets), normals, two densities
    d2h = 4 * 3 * args.n

    # ---- roofline of the dominant phase (FP32 ALU bound: pair evaluations / GEMM flops)
    dom = max((k for k in ph_ms if k != "tree"), key=lambda k: ph_ms[k])
    r = st["m2l_rank"]
    m = 3 * st["n_surf"]
    flops = {
        "eval": st["p2p_interactions"] * FLOPS_SLDL + st["l2p_interactions"] * FLOPS_SL,
        "m2l": st["n_v_pairs"] * 2 * r * r + st["n_boxes"] * 2 * r * m,
        "s2m": args.n * st["n_surf"] * FLOPS_SLDL,
        "up_pinv": st["n_leaves"] * 2 * m * m,
        "m2m": (st["n_boxes"] - 1) * 2 * m * m,
        "down": st["n_boxes"] * 2 * m * r + (st["n_boxes"] - 1) * 2 * m * m,
        "p2l": st["p2l_interactions"] * FLOPS_SLDL,
    }
    peak = fp32_peak_tflops(SM_MAX_MHZ)
    ach = flops.get(dom, 0) / (ph_ms[dom] / 1e3) / 1e12 if ph_ms[dom] > 0 else 0.0
    roof = {"bound": "alu", "kernel_phase": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None,
            "peak_note": "FP32 FMA peak derived: 152 SMs x 128 lanes x 2 flop x 2070 MHz",
            "frac_at_sampled_clock": (ach / fp32_peak_tflops(clocks["sm_mhz"])) if clocks.get("sm_mhz") else None}
    p2p_ach = flops["eval"] / (ph_ms["eval"] / 1e3) / 1e12 if ph_ms["eval"] > 0 else 0.0

    line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_points": args.n, "p": 6, "leaf_cap": 64, "G": 1.0, "nu": 0.3,
                       "step": "tree build + one SL+DL FMM evaluation", "l2": "flushed (512 MB write) between steps",
                       "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
            "clocks": clocks,
            "e2e": {"value": world * args.n / (e2e_ms / 1e3), "unit": "targets/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "roofline": roof,
            "eval_only_targets_per_s": world * args.n / (eval_ms / 1e3),
            "p2p_eval_fp32_frac": p2p_ach / peak,
            "phases_ms": ph_ms,
            "tree": {k: st[k] for k in ("n_boxes", "n_leaves", "n_levels", "m2l_rank", "n_v_pairs",
                                        "n_w_pairs", "n_x_pairs", "p2p_interactions")}}

    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the host cores over a bounded sample; its values also check the
        # GPU result at full size
        idx, ref, dt = cpu_oracle_sample(pts, nrm, sl, dl, args.cpu_sample)
        f.eval(s, d, out)
        got = out.cpu().numpy().astype(np.float64)[idx]
        line["cpu_baseline"] = {"value": args.cpu_sample / dt, "unit": "targets/s", "cores": host_threads(),
                                "kind": "oracle",
                                "sample": f"{args.cpu_sample} of {args.n} targets x all {args.n} sources, FP64"}
        line["rel_l2_error_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
