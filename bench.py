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

The line also carries the BEM half of the metric:
 - "bem": the 2x1x1 cantilever at voxel size 0.01 (400,000 triangles, 1.2M unknowns), clamped
   at x = 0, unit downward traction on the 0.1 x 0.1 patch at x = 2, solved to a 1e-6
   relative residual by mixed-precision GMRES with iterative refinement (FP32 FMM corrections,
   FP64-grade compensated direct residuals); then stress, topological derivative and energy
   density at the 256 x 128 x 128 cell centres (4,194,304 points); the oracle checks sampled
   rows of the residual and sampled grid points;
 - "bem_small": the same cantilever at 5760 triangles, GMRES-IR beside plain FP64 GMRES on the
   same GPU at the same 1e-6 residual;
and the homogenisation leg ("homogenisation"): the six unit-macro-strain load cases of a
periodic cell with ellipsoidal voids (~209k triangles, 18 density columns) in one solve with
the periodic FMM, beside one case at a time, and the homogenised stiffness (its bulk modulus
against the Hashin-Shtrikman bound); and the batch leg ("batch"): 32 independent surfaces of uneven
size in one build and evaluation, beside the same surfaces one by one; and the periodic leg
("periodic"): the periodic KIFMM on 1e6 points of a periodic unit cell, beside the same points
as a free-space sum.  Per-phase times come from separate
profiled steps (phases serialised); "eval_only_ms" is the evaluation alone on the last tree.
The FP32 peak of the "alu" rooflines is measured by the library's FMA-chain kernel.
--no-bem, --no-batch (also the periodic leg) and --no-cpu-baseline leave those legs out.
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
FP32_LANES_PER_SM = 128
# algorithmic FP32 operations per pair (counted from the kernel formulas, FMA = 2)
FLOPS_SLDL = 61   # single + double layer displacement
FLOPS_SL = 30     # single layer only (equivalent densities: L2P, M2P)
L2_FLUSH_BYTES = 512 << 20
BEM_N = 12          # small cantilever: cells per unit length, 40 n^2 = 5760 triangles
BEM3_N = 100        # the 400,000-triangle cantilever (voxel size 0.01)
BEM3_PATCH = 0.05   # half-side of its loaded patch (0.1 x 0.1)
TD_GRID = (256, 128, 128)
BEM3_TOL_HI = 2e-7  # GMRES-IR tolerance in the compensated residual (true residual <= 1e-6)
HOMOG_N = 175       # periodic cell voxels per side: ~200k void-surface triangles
# DRAM bytes per launch of the dominant kernel at this workload, from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` (profiles/); None when the
# kernel has changed since the counters were taken
TRAFFIC_BYTES = {"m2l": 350924032 + 114690304,            # the one tc_m2l_kernel launch
                 "down": 334326272 + 117628672}           # the phase's ten tc_box_gemm_kernel launches
TRAFFIC_NOTE = {"m2l": "DRAM bytes of the phase's tc_m2l_kernel launch (ncu, one pass, profiles/)",
                "down": "DRAM bytes of the phase's ten tc_box_gemm_kernel launches, summed like the flops "
                        "(ncu, one pass, profiles/)"}


def max_over_ranks(x, world, device):
    """The slowest rank's value (every rank calls this; world == 1 returns x).  Runs on any
    torch.distributed backend: NCCL on the GPUs, gloo in the CPU tests."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, slowest_seconds):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's
    time (weak scaling)."""
    return world * units_per_rank / slowest_seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp32_nominal_tflops(n_sms, mhz):
    return n_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_one_core_rate(k=100):
    """Targets/s of the oracle's direct sum on one host core: a fresh interpreter with
    OMP_NUM_THREADS=1 (this process has a CUDA context, so nothing is forked from it)."""
    code = ("import sys, time; sys.path.insert(0, %r); import bench as B; "
            "p, n, s, d = B.workload(B.N_POINTS); _, _, dt = B.cpu_oracle_sample(p, n, s, d, %d); print(dt)") % (ROOT, k)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        return k / float(r.stdout.strip().splitlines()[-1])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


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


def bem_small_leg(K, local, world):
    """Cantilever (40 n^2 triangles, clamped at x = 0, unit traction patch at x = 2) solved to a
    1e-6 relative residual: mixed-precision GMRES-IR on the FMM with compensated FP64-grade
    residuals (timed over 3 solves after a warm-up) and plain FP64 GMRES with the FP64 direct
    operator, both on the GPU."""
    import torch
    import workloads as W
    V, T, mask, vals = W.cantilever(BEM_N)
    nt = len(T)
    u, t = np.zeros((nt, 3)), np.zeros((nt, 3))
    out = {"workload": f"cantilever 2x1x1, {nt} triangles ({3 * nt} unknowns), mixed BC, patch 0.5x0.5, G=1, nu=0.3",
           "tol": 1e-6, "residual": "FP64-grade compensated direct discrete operator"}
    with K.Bem(V, T, K.BEM_FMM, device=local) as b:
        b.set_material(K.material_K(1.0, 0.3), 1.0)
        b.set_bc(mask, vals)
        kw = dict(tol=1e-6, restart=100, maxit=3000, refine=1, inner_tol=1e-3)
        b.solve(u, t, **kw)
        times, st = [], None
        for _ in range(3):
            torch.cuda.synchronize()
            st = b.solve(u, t, **kw)
            times.append(st["seconds"])
    sec = max_over_ranks(float(np.mean(times)), world, f"cuda:{local}")
    out.update({"solves_per_s": aggregate_rate(1, world, sec), "ms_per_solve": 1e3 * sec, "inner_iters": st["iters"],
                "outer": st["outer"], "fmm_matvecs": st["matvecs"], "hi_matvecs": st["matvecs_hi"],
                "relres": st["relres"], "method": "GMRES-IR: FP32 FMM corrections (p=6), compensated direct residuals"})
    with K.Bem(V, T, K.BEM_DIRECT_FP64, device=local) as b:
        b.set_material(K.material_K(1.0, 0.3), 1.0)
        b.set_bc(mask, vals)
        st = b.solve(u, t, tol=1e-6, restart=100, maxit=3000)
    out["fp64_gmres"] = {"ms_per_solve": 1e3 * st["seconds"], "iters": st["iters"], "relres": st["relres"],
                         "method": "plain GMRES, FP64 direct operator on the GPU"}
    out["speedup_vs_fp64_gmres"] = st["seconds"] / sec
    return out


def td_grid(shape=TD_GRID, box=(2.0, 1.0, 1.0)):
    """Cell centres of a regular grid over the box, [nx*ny*nz, 3] float32."""
    axes = [(np.arange(n) + 0.5) * (L / n) for n, L in zip(shape, box)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(g, dtype=np.float32)


def oracle_rows(V, T, u, t, idx):
    """The oracle's M(u, t) = 1/2 u + P^D u - U^D t (Eq. num) at the collocation points idx:
    direct sum over all quadrature sources, the element's own terms replaced by its analytic
    singular blocks."""
    import oracle as O
    nrm, area, cen = O.tri_geometry(V, T)
    q, w = O.tri_quadrature(V, T)
    q[12::16] = cen  # the centre sub-triangle's centroid is the collocation point
    qn = np.repeat(nrm, 16, axis=0)
    sl = -np.repeat(t, 16, axis=0) * w[:, None]
    dl = np.repeat(u, 16, axis=0) * w[:, None]
    m = O.direct_disp(cen[idx], q, qn, sl, dl, 1.0, 0.3)
    for r, l in enumerate(idx):
        own = slice(16 * l, 16 * l + 16)
        m[r] -= O.direct_disp(cen[l:l + 1], q[own], qn[own], sl[own], dl[own], 1.0, 0.3)[0]
        Us, Ts = O.self_integrals(*V[T[l]], 1.0, 0.3)
        m[r] += 0.5 * u[l] + Ts @ u[l] - Us @ t[l]
    return m


def bem_config3_leg(K, local, world, rank, check=True):
    """The 400,000-triangle cantilever (voxel size 0.01): GMRES-IR to a 1e-6 relative residual,
    then stress, topological derivative and energy density at the 256 x 128 x 128 cell
    centres.  One solve after a warm-up call (set-up, tree build, tuning); the grid
    evaluation once after a warm-up.  rank 0 checks sampled residual rows and grid points
    against the oracle."""
    import torch
    import workloads as W
    dev = torch.device("cuda", local)
    V, T, mask, vals = W.cantilever(BEM3_N, BEM3_PATCH)
    nt = len(T)
    u, t = np.zeros((nt, 3)), np.zeros((nt, 3))
    pts = torch.tensor(td_grid(), device=dev)
    npt = pts.shape[0]
    td = torch.empty(npt, dtype=torch.float32, device=dev)
    en = torch.empty_like(td)
    sig = torch.empty(npt, 6, dtype=torch.float32, device=dev)
    out = {"workload": f"cantilever 2x1x1, voxel 0.01, {nt} triangles ({3 * nt} unknowns, {16 * nt} quadrature "
                       f"sources), clamped x=0, traction (0,0,-1) on the 0.1x0.1 patch at x=2 ({int((np.abs(vals).sum(1) > 0).sum())} "
                       f"triangles); TD grid {TD_GRID[0]}x{TD_GRID[1]}x{TD_GRID[2]} ({npt} points)",
           "tol": 1e-6, "tol_compensated": BEM3_TOL_HI,
           "residual": "true residual of the exact discrete operator <= 1e-6: the solve runs to "
                       f"{BEM3_TOL_HI:g} in the compensated operator's residual, whose distance from the exact "
                       "operator is below 8e-7 of ||b|| (tests); the oracle checks sampled rows"}
    with K.Bem(V, T, K.BEM_FMM, device=local) as b:
        b.set_material(K.material_K(1.0, 0.3), 1.0)
        b.set_bc(mask, vals)
        rhs = np.zeros((nt, 3))
        b.rhs(rhs)  # warm-up: quadrature set-up, FMM tree of the 6.4M sources, tuning
        torch.cuda.synchronize(dev)
        st = b.solve(u, t, tol=BEM3_TOL_HI, restart=200, maxit=8000, refine=1, inner_tol=1e-3)
        sec = max_over_ranks(st["seconds"], world, dev)
        out.update({"solves_per_s": aggregate_rate(1, world, sec), "ms_per_solve": 1e3 * sec,
                    "inner_iters": st["iters"], "outer": st["outer"], "fmm_matvecs": st["matvecs"],
                    "hi_matvecs": st["matvecs_hi"], "relres": st["relres"], "converged": bool(st["converged"]),
                    "method": "GMRES-IR: FP32 FMM corrections (p=6, restart 200, inner tol 1e-3), compensated "
                              "FP64-grade direct residuals"})
        b.topo_derivative(pts, td, en, sig)  # warm-up: the interior tree of sources and grid points
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        e0.record(stream)
        b.topo_derivative(pts, td, en, sig)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        td_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        out["td"] = {"ms": td_ms, "points_per_s": aggregate_rate(npt, world, td_ms / 1e3),
                     "step": "interior FMM build (6.4M sources, 4.2M targets) + STRESS evaluation + Eq. deriv",
                     "p": 8}
        if check and rank == 0:
            import oracle as O
            # residual at sampled rows: the oracle's M(u, t) relative to ||b|| on the same rows
            idx = np.asarray(__import__("workloads").subsample(nt, 200))
            t0 = time.perf_counter()
            m_or = oracle_rows(V, T, u, t, idx)
            bn_rows = np.sqrt(len(idx) / nt) * np.linalg.norm(rhs)
            out["oracle_residual_sampled"] = float(np.linalg.norm(m_or) / bn_rows)
            out["oracle_residual_rows"] = int(len(idx))
            # stress at sampled grid points against the oracle's Somigliana sum (Eq. stress_1)
            gi = np.asarray(W.subsample(npt, 200))
            p64 = pts[gi].double().cpu().numpy()
            _, s_ref = O.bem_interior(p64, V, T, u, t, 1.0, 0.3, disp=False, stress=True)
            td_ref, _ = O.topo_derivative(s_ref, 1.0, 0.3)
            s_got = sig[gi].double().cpu().numpy()
            out["stress_rel_l2_vs_oracle"] = float(np.linalg.norm(s_got - s_ref) / np.linalg.norm(s_ref))
            out["td_rel_l2_vs_oracle"] = float(np.linalg.norm(td[gi].double().cpu().numpy() - td_ref)
                                               / np.linalg.norm(td_ref))
            # split by the distance to the nearest face of the 2x1x1 box: within two elements
            # (the discrete sum is near-singular there) and beyond
            dist = np.minimum(np.minimum(p64, np.array([2.0, 1.0, 1.0]) - p64).min(axis=1), 1.0)
            for name, sel in (("near_surface", dist < 2.0 / BEM3_N), ("interior", dist >= 2.0 / BEM3_N)):
                if sel.any():
                    out[f"stress_rel_l2_vs_oracle_{name}"] = float(np.linalg.norm(s_got[sel] - s_ref[sel])
                                                                   / np.linalg.norm(s_ref[sel]))
                    out[f"oracle_grid_points_{name}"] = int(sel.sum())
            out["oracle_check_s"] = time.perf_counter() - t0
            out["oracle_grid_points"] = int(len(gi))
    return out


def unit_strain_tractions(V, T, G, nu):
    """t = -sigma^h n on the void surfaces for the six unit macro strains (xx, yy, zz, yz, xz,
    xy; shear as eps_ij = eps_ji = 1/2), sigma^h = lambda tr(eps) I + 2 G eps: [nt, 18]."""
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1)[:, None]
    lam = 2 * G * nu / (1 - 2 * nu)
    cols = []
    for i, j in [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]:
        eps = np.zeros((3, 3))
        eps[i, j] = eps[j, i] = 1.0 if i == j else 0.5
        cols.append(-n @ (lam * np.trace(eps) * np.eye(3) + 2 * G * eps).T)
    return np.ascontiguousarray(np.concatenate(cols, axis=1))


def effective_stiffness(V, T, u, G, nu):
    """Homogenised stiffness [6, 6] (Voigt, engineering shear) of a unit periodic cell from the
    fluctuation displacements u [nt, 18] of the six unit macro strains: <sigma> = C : [(1 - phi)
    eps + int sym(u n) dS] (n out of the material, the void volume fraction phi from the mesh)."""
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / (2 * area[:, None])
    phi = -np.sum(np.einsum("ij,ij->i", (a + b + c) / 3, n) * area) / 3
    lam = 2 * G * nu / (1 - 2 * nu)
    vo = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    C = np.zeros((6, 6))
    for col, (i, j) in enumerate(vo):
        eps = np.zeros((3, 3))
        eps[i, j] = eps[j, i] = 1.0 if i == j else 0.5
        S = np.einsum("ki,kj,k->ij", u[:, 3 * col:3 * col + 3], n, area)
        e = (1 - phi) * eps + 0.5 * (S + S.T)
        sig = lam * np.trace(e) * np.eye(3) + 2 * G * e
        C[:, col] = [sig[p, q] for p, q in vo]
    return C, phi


def homogenisation_leg(K, local, world, tol=1e-5):
    """The six unit-macro-strain load cases of a periodic cell with voids (the periodic traction
    problem, t = -sigma^h n on the voids, 18 density columns) in one BEM solve, GMRES on the
    periodic FMM operator, beside the same six solved one at a time; the homogenised stiffness
    and its bulk modulus against the Hashin-Shtrikman upper bound."""
    import torch
    import workloads as W
    V, T = W.periodic_cell_voids(HOMOG_N)
    nt = len(T)
    vals = unit_strain_tractions(V, T, 1.0, 0.3)
    mask = np.zeros((nt, 3), np.uint8)
    out = {"workload": f"periodic unit cell, {nt} void-surface triangles (ellipsoidal voids voxelised at "
                       f"h = 1/{HOMOG_N}), 6 unit macro strains = 18 density columns, periodic traction problem, "
                       "G=1, nu=0.3",
           "tol": tol, "residual": "the periodic FMM operator's (FP32, p = 6)"}
    with K.Bem(V, T, K.BEM_FMM, device=local) as b:
        b.set_material(K.material_K(1.0, 0.3), 1.0)
        b.set_periodic((0.0, 0.0, 0.0), 1.0)
        b.set_bc(mask, vals)
        rhs = np.zeros((nt, 18))
        b.rhs(rhs)  # warm-up: set-up, tree, tuning
        u = np.zeros((nt, 18))
        torch.cuda.synchronize()
        st = b.solve(u, None, tol=tol, restart=100, maxit=3000)
        sec = max_over_ranks(st["seconds"], world, f"cuda:{local}")
        one = 0.0
        its = []
        for c in range(6):
            b.set_bc(mask, np.ascontiguousarray(vals[:, 3 * c:3 * c + 3]))
            u1 = np.zeros((nt, 3))
            s1 = b.solve(u1, None, tol=tol, restart=100, maxit=3000)
            one += s1["seconds"]
            its.append(s1["iters"])
            if c == 0:
                out["column0_rel_diff"] = float(np.linalg.norm(u1 - u[:, 0:3]) / np.linalg.norm(u1))
        one = max_over_ranks(one, world, f"cuda:{local}")
    C, phi = effective_stiffness(V, T, u, 1.0, 0.3)
    kb = 2 * 1.0 * 1.3 / (3 * (1 - 0.6))
    k_eff = C[:3, :3].sum() / 9
    k_hs = kb * (1 - phi * (3 * kb + 4.0) / (4.0 + 3 * kb * phi))
    out.update({"void_fraction": phi, "bulk_modulus_over_matrix": k_eff / kb, "bulk_modulus_over_hs_bound": k_eff / k_hs,
                "stiffness_asymmetry": float(np.abs(C - C.T).max() / np.abs(C).max()),
                "stiffness_voigt": np.round(C, 5).tolist()})
    out.update({"load_cases_per_s": aggregate_rate(6, world, sec), "ms_per_6_case_solve": 1e3 * sec,
                "iters": st["iters"], "relres": st["relres"], "fmm_matvecs": st["matvecs"],
                "one_case_at_a_time_ms": 1e3 * one, "one_case_iters": its, "speedup_vs_one_at_a_time": one / sec})
    return out


def batch_leg(K, local, world, flush, steps=3, warmup=1):
    """32 independent box-with-voids surfaces of uneven size, 5k-250k triangles each
    (log-uniform) as their 16 quadrature points per triangle (80k-4M points), in one tree and
    one set of launches (kfmm_build_sets + one SL+DL evaluation), against the same surfaces
    built and evaluated one by one on the same context."""
    import torch
    import workloads as W
    dev = torch.device("cuda", local)
    pts, nrm, off = W.surface_batch(32, 16 * 5000, 16 * 250000)
    sl, dl = W.densities(len(pts))
    x = torch.tensor(pts, dtype=torch.float32, device=dev)
    nn = torch.tensor(nrm, dtype=torch.float32, device=dev)
    s = torch.tensor(sl, dtype=torch.float32, device=dev)
    d = torch.tensor(dl, dtype=torch.float32, device=dev)
    out = torch.empty(len(pts), 3, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    n_sets = len(off) - 1
    f = K.Kfmm(p=6, leaf_cap=64, device=local)
    f.set_material(K.material_K(1.0, 0.3), 1.0)
    f.set_stream(stream)

    def batched():
        f.build_sets(off, x, nn, off, x)
        f.eval(s, d, out)

    def one_by_one():
        for k in range(n_sets):
            a, b = int(off[k]), int(off[k + 1])
            f.build(x[a:b], nn[a:b], x[a:b])
            f.eval(s[a:b], d[a:b], out[a:b])

    def timed(fn):
        for _ in range(warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)

    ms_b = timed(batched)
    ms_s = timed(one_by_one)
    f.close()
    return {"workload": f"{n_sets} box-with-voids surfaces of 5k-250k triangles as 16 quadrature points each: "
                        f"{int(np.diff(off).min())}-{int(np.diff(off).max())} points per surface, {len(pts)} in all; "
                        "tree build + one SL+DL evaluation per step, p=6",
            "ms_per_step": ms_b, "targets_per_s": aggregate_rate(len(pts), world, ms_b / 1e3),
            "one_by_one_ms_per_step": ms_s, "speedup_vs_one_by_one": ms_s / ms_b}


def periodic_leg(K, local, world, flush, n=1000000, steps=10, warmup=3):
    """The periodic KIFMM on the surfaces of 12 spherical voids of a periodic unit cell (points
    wrapped across the cell's faces): tree build + one SL+DL evaluation per step, against the
    same points summed as a free-space problem on the same context."""
    import torch
    import workloads as W
    dev = torch.device("cuda", local)
    pts, nrm = W.periodic_cell_points(n)
    sl, dl = W.densities(n)
    x = torch.tensor(pts, dtype=torch.float32, device=dev)
    nn = torch.tensor(nrm, dtype=torch.float32, device=dev)
    s = torch.tensor(sl, dtype=torch.float32, device=dev)
    d = torch.tensor(dl, dtype=torch.float32, device=dev)
    out = torch.empty(n, 3, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    f = K.Kfmm(p=6, leaf_cap=64, device=local)
    f.set_material(K.material_K(1.0, 0.3), 1.0)
    f.set_stream(stream)

    def step():
        f.build(x, nn, x)
        f.eval(s, d, out)

    def timed():
        for _ in range(warmup):
            step()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)

    f.set_periodic((0.0, 0.0, 0.0), 1.0)
    t0 = time.perf_counter()
    step()  # the lattice operator (host FP64, once per operator set) and the launch-shape tuning
    torch.cuda.synchronize(dev)
    first_s = time.perf_counter() - t0
    ms_p = timed()
    st = f.stats()
    f.set_periodic(None)
    ms_f = timed()
    f.close()
    return {"workload": f"{n} points on the surfaces of 12 spherical voids of a periodic unit cell, wrapped "
                        "across its faces; tree build + one SL+DL evaluation per step, p=6, leaf cap 64",
            "ms_per_step": ms_p, "targets_per_s": aggregate_rate(n, world, ms_p / 1e3),
            "free_space_ms_per_step": ms_f, "periodic_over_free_space": ms_p / ms_f,
            "first_step_s": first_s, "n_v_pairs": st["n_v_pairs"], "n_levels": st["n_levels"]}


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
    ap.add_argument("--no-bem", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
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
    fp32_meas = f.measure_fp32_peak()

    def step():
        f.build(x, nn, x)
        f.eval(s, d, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = f.stats()

    # ---- timed region: K steps, per-step CUDA events on the launching stream
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
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)
    value = aggregate_rate(args.n, world, ms / 1e3)

    # ---- per-phase CUDA-event times, after the timed region: profiling serialises the phases
    #      that otherwise overlap on the library's second stream
    n_prof = max(1, min(args.steps, 10))
    f.set_profiling(True)
    f.phase_times(reset=True)
    for _ in range(n_prof):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    phases = f.phase_times(reset=True)
    f.set_profiling(False)
    ph_ms = {k: v[0] / n_prof for k, v in phases.items()}

    # ---- evaluation alone on the last tree (repeated arguments: graph replay, as in a solve)
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_prof)]
    for k in range(args.warmup + n_prof):
        flush.zero_()
        if k >= args.warmup:
            eev[k - args.warmup][0].record(stream)
        f.eval(s, d, out)
        if k >= args.warmup:
            eev[k - args.warmup][1].record(stream)
    torch.cuda.synchronize(dev)
    eval_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in eev])), world, dev)

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
    e2e_ms = max_over_ranks(1e3 * float(np.mean(e2e_t)), world, dev)
    h2d = 4 * 3 * args.n * 4  # points (as sources and targets), normals, two densities
    d2h = 4 * 3 * args.n

    # ---- rooflines per phase (CUDA-event time per step); the dominant one goes in "roofline"
    r = st["m2l_rank"]
    m = 3 * st["n_surf"]
    ku, kd = st["up_rank"], st["down_rank"]
    peaks, peak_src = load_peaks()
    fp32_peak = fp32_meas["tflops"]
    bf16_peak = peaks["bf16_tflops_sustained"]
    # (bound, executed operations per step, peak, note)
    work = {
        "eval": ("alu", st["p2p_interactions"] * FLOPS_SLDL + st["l2p_interactions"] * FLOPS_SL, fp32_peak,
                 "FP32 pair evaluations (61 flop SL+DL P2P, 30 flop SL L2P/M2P)"),
        "s2m": ("alu", st["s2m_interactions"] * FLOPS_SLDL, fp32_peak, "FP32 pair evaluations"),
        "p2l": ("alu", st["p2l_interactions"] * FLOPS_SLDL, fp32_peak, "FP32 pair evaluations"),
        "m2l": ("tensor", 3 * 2 * r * r * st["n_v_pairs"], bf16_peak,
                "BF16 MMA flops: 3 split-pair products per FP32-grade product, 2 r^2 per V pair"),
        "m2l_basis": ("tensor", 6 * 2 * r * ku * st["n_boxes"], bf16_peak,
                      "BF16 MMA flops: 6 three-term products per FP32-grade product"),
        "up_pinv": ("tensor", 6 * 2 * ku * m * st["n_leaves"], bf16_peak, "BF16 MMA flops, three-term splits"),
        "m2m": ("tensor", 6 * 2 * ku * ku * (st["n_boxes"] - 1), bf16_peak, "BF16 MMA flops, three-term splits"),
        "down": ("tensor", 6 * 2 * (kd * r * st["n_boxes"] + kd * m * st["n_xboxes"] + kd * kd * (st["n_boxes"] - 1)
                                    + m * kd * st["n_leaves"] + m * ku * st["n_wboxes"]), bf16_peak,
                 "BF16 MMA flops, three-term splits"),
    }

    def roofline_of(k):
        bound, ops, peak, note = work[k]
        t = ph_ms[k] / 1e3
        ach = ops / t / 1e12 if t > 0 else 0.0
        return {"bound": bound, "kernel_phase": k, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": TRAFFIC_BYTES.get(k), "traffic_note": TRAFFIC_NOTE.get(k),
                "peak_note": (f"FP32 FMA peak measured by kfmm_measure_fp32_peak on this GPU ({fp32_meas['n_sms']} SMs, "
                              f"FMA chains, fastest of 5 launches)" if bound == "alu"
                              else f"BF16 dense tensor peak, sustained, of {peak_src} (MEASURED_PEAKS.json)"),
                "ops_note": note}

    dom = max((k for k in work if k in ph_ms), key=lambda k: ph_ms[k])
    roof = roofline_of(dom)
    if clocks.get("sm_mhz") and roof["bound"] == "alu":
        roof["frac_of_nominal_at_sampled_clock"] = roof["achieved"] / fp32_nominal_tflops(fp32_meas["n_sms"],
                                                                                           clocks["sm_mhz"])
    kernels = {k: {"ms": ph_ms[k], "frac": roofline_of(k)["frac"], "bound": work[k][0]} for k in work if k in ph_ms}
    p2p_ach = work["eval"][1] / (ph_ms["eval"] / 1e3) / 1e12 if ph_ms["eval"] > 0 else 0.0

    # ---- BEM leg: mixed-precision refinement vs plain FP64 GMRES at a 1e-6 FP64 residual
    def leg(fn, *a, **kw):
        # a side leg that fails (e.g. a solve that does not converge) is reported in its own
        # key; the headline line is still printed
        try:
            return fn(*a, **kw)
        except Exception as exc:  # noqa: BLE001
            return {"error": f"{type(exc).__name__}: {exc}"}

    bem = leg(bem_config3_leg, K, local, world, rank, check=not args.no_cpu_baseline) if not args.no_bem else None
    bem_small = leg(bem_small_leg, K, local, world) if not args.no_bem else None
    homog = leg(homogenisation_leg, K, local, world) if not args.no_bem else None
    batch = leg(batch_leg, K, local, world, flush) if not args.no_batch else None
    periodic = leg(periodic_leg, K, local, world, flush) if not args.no_batch else None

    line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_points": args.n, "p": 6, "leaf_cap": 64, "G": 1.0, "nu": 0.3,
                       "step": "tree build + one SL+DL FMM evaluation", "l2": "flushed (512 MB write) between steps",
                       "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
            "clocks": clocks,
            "e2e": {"value": aggregate_rate(args.n, world, e2e_ms / 1e3), "unit": "targets/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "roofline": roof,
            "eval_only_targets_per_s": world * args.n / (eval_ms / 1e3),
            "p2p_eval_fp32_frac": p2p_ach / fp32_peak,
            "eval_only_ms": eval_ms,
            "phases_ms": ph_ms,
            "phases_note": "CUDA-event time per phase over separate profiled steps, phases serialised on one "
                           "stream; the timed steps run P2L and the leaf-to-leaf P2P on a second stream, "
                           "overlapped with the upward pass and M2L",
            "kernels": kernels,
            "bem": bem,
            "bem_small": bem_small,
            "homogenisation": homog,
            "batch": batch,
            "periodic": periodic,
            "fp32_peak": {"tflops": fp32_meas["tflops"], "n_sms": fp32_meas["n_sms"], "source": "measured",
                          "nominal_at_max_clock": fp32_nominal_tflops(fp32_meas["n_sms"], 2070.0)},
            "tree": {k: st[k] for k in ("n_boxes", "n_leaves", "n_levels", "m2l_rank", "n_v_pairs",
                                        "n_w_pairs", "n_x_pairs", "p2p_interactions")}}

    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the host cores over a bounded sample; its values also check the
        # GPU result at full size
        idx, ref, dt = cpu_oracle_sample(pts, nrm, sl, dl, args.cpu_sample)
        f.eval(s, d, out)
        got = out.cpu().numpy().astype(np.float64)[idx]
        line["cpu_baseline"] = {"value": args.cpu_sample / dt, "unit": "targets/s", "cores": host_threads(),
                                "kind": "oracle", "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                                "one_core_value": oracle_one_core_rate(),
                                "sample": f"{args.cpu_sample} of {args.n} targets x all {args.n} sources, FP64 "
                                          "(one_core_value: 100 targets, OMP_NUM_THREADS=1)"}
        line["rel_l2_error_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
