#!/usr/bin/env python
"""Throughput of the Lippmann-Schwinger corrector solve on GB300.

Metric: voxel-CG-iterations per second of the mixed-precision batched solver
against the plain FP64 solver, at C* agreeing to 1e-8.  The default workload
is the batched one: 64 seeded two-phase elastic sphere microstructures whose
grids are drawn from {32, 48, 64, 96, 128}^3 (volume fractions U(0.1, 0.4),
radius N/16 voxels, contrast 10), 6 Mandel loads each (384 systems), one batch
handle per grid with all of that grid's microstructures x loads in the same
launches; one step computes all 64 effective tensors C* to relative residual
1e-10.  `value` counts N^3 x the CG iterations the plain FP64 solver needs for
the same systems, divided by the mixed solver's device time (an accuracy-fair
count; the raw inner-iteration rate and the FP64 solver's own rate are
reported beside it).

Also reported: an end-to-end number through the public API with the phase
maps in pinned host memory (host->device copies and the C* readback inside
the timed region), the C* error of the mixed solver against the FP64 one, the
roofline of the dominant FP32 pass (per-pass CUDA events recorded live on the
solve stream), the GPU clocks sampled during the timed region, and the FP64
CPU oracle timed on a bounded sample of the same workload.

Other workloads (--workload): spheres128 (one 128^3 packing, filtered and
truncated operators), contrast256, gradient128, convergence, cufft.
--impl reference times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun): every rank solves its own copy of the workload
(independent replicas, no data-path collective); value = all voxel-iterations
/ the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-CG-iterations/s of LS solve, mixed+batched vs FP64 plain at 1e-8 C* error"
UNIT = "voxel-iterations/s"
N = 128
TOL = 1e-10


def k_mu(E, nu):
    return E / (3.0 * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def workload():
    from paper_1411_0330_gb300 import microstructures as ms
    ph, cen, r = ms.sphere_microstructure(N, 8.0, 0.3, seed=1411)
    mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    return ph, mods, len(cen)


def config(nspheres, frac):
    return {"workload": f"{N}^3 isotropic elasticity, {nspheres} RSA spheres r=8 vox, f={frac:.4f}, seed 1411, "
                        f"E 1/10 nu 0.3/0.2, mu0=mu_min/2 nu0=0.3, CG rel.res {TOL:g}, 6 Mandel loads, "
                        f"filtered + truncated Gamma (12 solves per step)",
            "grid": [N, N, N], "components": 6, "loads_per_step": 12, "tol": TOL,
            "l2": "working set 686 MB per handle > 129 MB L2 (no flush needed)"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
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
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- roofline bookkeeping
def pass_traffic(kind, V, c, nx, nxh, ncoef, b):
    """Algorithmic bytes of one launch of a pass over the whole field (b = bytes per real)."""
    cV = c * V
    half = nxh / nx  # complex half-spectrum elements per real element
    if kind == "x_forward":      # read x, r, p; write x, p; write the half spectrum
        return cV * (5 * b + 2 * b * half)
    if kind in ("y_forward", "y_inverse"):
        return cV * 4 * b * half
    if kind == "z_gamma":        # spectrum in and out + the symmetric Gamma table
        return cV * 4 * b * half + V * ncoef * b * half
    if kind == "x_inverse_local":  # spectrum, p in; q out; phase byte per element
        return cV * (2 * b * half + 2 * b + 1)
    if kind == "cg_update":      # r, q in; r out
        return cV * 3 * b
    raise KeyError(kind)


def pass_flops(kind, V, c, nx, ny, nz, nxh):
    """Conventional FFT flop count 5 n log2 n per complex length-n transform, plus the
    arithmetic of the fused epilogues."""
    lg = lambda n: np.log2(n) if n > 1 else 0.0
    if kind == "x_forward":
        return c * nz * ny / 2 * 5 * nx * lg(nx) + c * V * 4 + c * nz * ny / 2 * nxh * 8
    if kind in ("y_forward", "y_inverse"):
        return c * nz * nxh * 5 * ny * lg(ny)
    if kind == "z_gamma":
        return 2 * c * ny * nxh * 5 * nz * lg(nz) + ny * nz * nxh * (2 * c * c - 2 * c + 2 * c) * 2
    if kind == "x_inverse_local":
        return c * nz * ny / 2 * 5 * nx * lg(nx) + c * V * 6
    if kind == "cg_update":
        return c * V * 4
    raise KeyError(kind)


PROF_EVERY = 8  # per-pass events in one CG chunk of this many

# DRAM bytes (read + write) of one launch of each FP32 pass (plane schedule)
# over the 6 load systems of the 128^3 workload, from the ncu captures in the
# plane-pass summary under profiles/ (filtered operator); to be retaken
# whenever one of these kernels changes (None: not captured for the current
# kernel).
NCU_TRAFFIC_FP32 = {"x_forward": 1774.9e6, "y_forward": None, "z_gamma": 724.2e6, "y_inverse": None,
                    "x_inverse_local": 909.1e6, "cg_update": 861.8e6}
NCU_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch over 6 systems at 128^3 "
                      "(filtered), scaled to the batch's average launch by its algorithmic bytes")


def ncu_traffic_per_launch(kind, alg_bytes_per_launch):
    """DRAM traffic of an average batch launch of `kind`: the 128^3 capture's ratio of DRAM
    to algorithmic bytes times the batch launch's algorithmic bytes (None without a capture)."""
    t = NCU_TRAFFIC_FP32.get(kind)
    if t is None:
        return None
    alg = 6 * pass_traffic(kind, N ** 3, 6, N, N // 2 + 1, 0, 4) + batch_pass_bytes(kind, N)[1]
    return t / alg * alg_bytes_per_launch


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6780.0), "source": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


# ----------------------------------------------------------------- CPU oracle sample
def oracle_sample(ph, mods, iters=2):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the 128^3
    workload: `iters` CG iterations of one filtered solve (shear load)."""
    import oracle
    oracle.build()
    P = oracle.Problem(ph, mods, physics=oracle.ELASTIC, green=oracle.FILTERED)
    load = np.zeros(6)
    load[5] = 1.0
    t0 = time.perf_counter()
    try:
        oracle.solve(P, load, tol=1e-30, maxit=iters, solver=oracle.SOLVER_CG)
    except oracle.OracleError as e:
        if e.code != 5:  # not converged is expected for a bounded sample
            raise
    dt = time.perf_counter() - t0
    return {"value": ph.size * iters / dt, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
            "sample": f"{iters} CG iterations of one {N}^3 filtered solve (shear load), {dt:.1f} s"}


def oracle_cores():
    """Threads the oracle's OpenMP loops use."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def batch_sample(phases, meta):
    """One microstructure of each grid of the batch (the first one drawn)."""
    picks = {}
    for ph, m in zip(phases, meta):
        picks.setdefault(m["n"], ph)
    return [picks[n] for n in sorted(picks)]


def oracle_batch_sample(sample, mods, iters):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the batched
    workload: `iters` CG iterations of one filtered solve (shear load) of one
    microstructure per grid size.  Returns (voxel-iterations, seconds)."""
    import oracle
    oracle.build()
    load = np.zeros(6)
    load[5] = 1.0
    units, t0 = 0, time.perf_counter()
    for ph in sample:
        P = oracle.Problem(ph, mods, physics=oracle.ELASTIC, green=oracle.FILTERED)
        try:
            oracle.solve(P, load, tol=1e-30, maxit=iters, solver=oracle.SOLVER_CG)
        except oracle.OracleError as e:
            if e.code != 5:  # not converged is expected for a bounded sample
                raise
        units += ph.size * iters
    return units, time.perf_counter() - t0


def batch_sample_text(sample, iters):
    grids = "/".join(str(p.shape[0]) for p in sample)
    return f"{iters} CG iterations of one filtered solve (shear load) of one microstructure per grid ({grids})^3"


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle on the batched workload's sample: each step is one CG
    iteration of one microstructure per grid size; W such steps first, untimed."""
    if rank != 0:
        return 0
    phases, meta = batch64_inputs()
    mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    sample = batch_sample(phases, meta)
    for _ in range(args.warmup):
        oracle_batch_sample(sample, mods, 1)
    units, secs = 0, 0.0
    for _ in range(args.steps):
        u, dt = oracle_batch_sample(sample, mods, 1)
        units += u
        secs += dt
    v = units / secs
    cb = {"value": v, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
          "sample": batch_sample_text(sample, 1) + f" per step, {args.steps} steps"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": batch_config(meta), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ncu case
def profile_case(kind):
    """4 CG iterations of the 6 load systems of one microstructure in one wave, as the
    bench runs them: the small case the ncu captures run on (a few GB on the device).
    fp64 / mixed: the 128^3 packing, filtered operator (spectrum 306 MB FP32 / 612 MB
    FP64, larger than L2); mixed96: a 96^3 packing of the batched recipe (seed 1411 + 1,
    f = 0.25, r = 6 voxels).  The mixed handles run the FP32 plane passes with the z
    variant the autotuner picks at both sizes, set by hand so that the launch sequence
    is fixed."""
    import torch
    from paper_1411_0330_gb300 import lsh
    from paper_1411_0330_gb300 import microstructures as ms
    if kind == "mixed96":
        ph, _, _ = ms.sphere_microstructure(96, 6.0, 0.25, seed=1412)
        mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    else:
        ph, mods, _ = workload()
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED,
                   precision=lsh.FP64 if kind == "fp64" else lsh.MIXED)
    if kind in ("mixed", "mixed96"):
        h.set_variants(0, 0, 2, 11)  # plane passes, fused TMA z pass (the tuned choice at 96^3 and 128^3)
    _, infos = h.effective(tol=1e-30, maxit=4, raise_on_fail=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": kind, "info": infos[0]}))
    return 0


# ----------------------------------------------------------------- replicas
def slowest_rank_ms(ms, world, device):
    """The timed region's duration on the slowest rank (every rank solves its own
    copy of the workload; no data-path collective)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def replica_rate(units_per_rank, world, ms_slowest):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms_slowest / 1e3)


# ----------------------------------------------------------------- other workloads
def _wall(fn):
    """Wall time of a synchronous call that may use several streams."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def _cstar_err(A, B):
    """max_ij |A_ij - B_ij| / max_kl |B_kl|, and the largest true relative error
    over the entries with |B_ij| >= 1e-3 max |B|."""
    A, B = np.asarray(A), np.asarray(B)
    m = np.abs(B).max()
    big = np.abs(B) >= 1e-3 * m
    return float(np.abs(A - B).max() / m), float((np.abs(A - B)[big] / np.abs(B)[big]).max())


def batch64_inputs(count=64, grids=(32, 48, 64, 96, 128), seed0=1411):
    """64 two-phase sphere microstructures: microstructure i draws its grid
    uniformly from `grids` and its volume fraction from U(0.1, 0.4) with seed
    seed0 + i; spheres of radius N/16 voxels (the same physical radius 1/16
    as the 128^3 workload), random sequential addition or hard-sphere Monte
    Carlo above f = 0.3."""
    from paper_1411_0330_gb300 import microstructures as ms
    phases, meta = [], []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.choice(grids))
        f = float(rng.uniform(0.1, 0.4))
        ph, _, _ = ms.sphere_microstructure(n, n / 16.0, f, seed=seed0 + i)
        phases.append(ph)
        meta.append({"n": n, "f_target": f, "f": float(ph.mean())})
    return phases, meta


def batch_config(meta):
    counts = {}
    for m in meta:
        counts[str(m["n"])] = counts.get(str(m["n"]), 0) + 1
    vox = sum(m["n"] ** 3 for m in meta)
    # FP32 CG state per grid handle: all its microstructures x 6 loads x 6 components, 4 fields
    smallest = min(counts[str(n)] * 6 * 6 * n ** 3 * 4 * 4 for n in (int(k) for k in counts))
    return {"workload": "64 two-phase elastic sphere microstructures, grids U{32,48,64,96,128}^3, "
                        "f ~ U(0.1,0.4), r = N/16 vox, seeds 1411+i, E 1/10 nu 0.3/0.2, mu0=mu_min/2 nu0=0.3, "
                        "filtered Gamma, 6 Mandel loads each (384 systems), CG rel.res 1e-10; mixed precision "
                        "(FP32 inner CG, double-float / FP64 refinement residual) vs plain FP64",
            "grids": counts, "voxel_systems": int(vox * 6), "components": 6, "tol": TOL,
            "l2": f"inputs larger than L2: the smallest grid handle's FP32 CG fields are {smallest / 1e6:.0f} MB "
                  "(> 129 MB), no flush needed"}


def batch_pass_bytes(k, n, filtered=True):
    """Algorithmic FP32 bytes of pass k per live system-iteration on an n^3 grid (6
    components), and the Gamma-table bytes read once per launch (filtered operator)."""
    V, nxh = n ** 3, n // 2 + 1
    per_sys = pass_traffic(k, V, 6, n, nxh, 0, 4)
    table = V * 21 * 4 * nxh / n if (k == "z_gamma" and filtered) else 0.0
    return per_sys, table


def run_batch(args, rank, world, local):
    """The default arm: the 64-microstructure batch, mixed precision against plain FP64."""
    import torch
    import torch.distributed as dist
    from paper_1411_0330_gb300 import lsh
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)  # every grid handle issues its work here: events see all of it
    phases, meta = batch64_inputs()
    mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    gmx = lsh.GridBatch(phases, mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED, device=dev,
                        stream=stream, tune=True)
    g64 = lsh.GridBatch(phases, mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.FP64, device=dev,
                        stream=stream, tune=False)
    for _ in range(args.warmup):
        gmx.effective(tol=TOL)
    g64.effective(tol=TOL)

    def timed(gb, steps, profile, name):
        for h in gb.handles:
            h.profile_read(reset=True)
            h.profile_enable(bool(profile), every=max(int(profile), 1))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(name)  # lets a profiler select the timed region
        e0.record(stream)
        out = None
        for _ in range(steps):
            out = gb.effective(tol=TOL)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = slowest_rank_ms(e0.elapsed_time(e1), world, dev)
        profs = [h.profile_read(reset=True) for h in gb.handles]
        for h in gb.handles:
            h.profile_enable(False)
        return ms / steps, out, profs, clocks

    # headline: the mixed solver; per-pass events in one CG chunk of PROF_EVERY
    ms_mx, (A_mx, I_mx), prof_mx, clocks = timed(gmx, args.steps, PROF_EVERY, "timed_mixed")
    # comparison: the plain FP64 solver on the same systems (one step: its iteration counts and time)
    ms_64, (A_64, I_64), _, clocks64 = timed(g64, 1, 0, "timed_fp64")
    vox = np.array([m["n"] ** 3 for m in meta], dtype=np.float64)
    it64 = np.array([sum(i["iters"] for i in inf) for inf in I_64], dtype=np.float64)
    itmx = np.array([sum(i["iters"] for i in inf) for inf in I_mx], dtype=np.float64)
    errs = [_cstar_err(a, b) for a, b in zip(A_mx, A_64)]
    value = replica_rate(float((vox * it64).sum()), world, ms_mx)  # FP64-equivalent
    value_raw = replica_rate(float((vox * itmx).sum()), world, ms_mx)
    value_64 = replica_rate(float((vox * it64).sum()), world, ms_64)
    launches = sum(p["launches"] for p in prof_mx) // args.steps

    # roofline of the dominant FP32 pass over all grid handles, from the live per-pass events:
    # algorithmic bytes of the live system-iterations inside the timed chunks / their event time
    peaks = load_peaks()
    grid_of = [h.shape[0] for h in gmx.handles]
    tot_ms = {k: sum(p["pass_ms"][k] for p in prof_mx) for k in lsh.PASS_NAMES}
    tot_n = {k: sum(p["pass_launches"][k] for p in prof_mx) for k in lsh.PASS_NAMES}

    def bytes_of(p, n, k):
        """Algorithmic bytes of pass k in the timed chunks of one grid handle (none when the
        pass did not run: the plane passes do the y transforms inside the x passes)."""
        if not p["pass_launches"][k]:
            return 0.0
        per_sys, table = batch_pass_bytes(k, n)
        return per_sys * p["timed_sys_iters"] + table * p["pass_launches"][k]

    tot_b = {k: sum(bytes_of(p, n, k) for p, n in zip(prof_mx, grid_of)) for k in lsh.PASS_NAMES}
    dom = max(tot_ms, key=tot_ms.get)
    achieved = tot_b[dom] / (tot_ms[dom] / 1e3) / 1e9
    sh_sum = max(sum(tot_ms.values()), 1e-30)
    per_grid_pass = {}
    for p, n in zip(prof_mx, grid_of):
        per_grid_pass[str(n)] = {k: {"ms_per_launch": p["pass_ms"][k] / p["pass_launches"][k],
                                     "gbs": bytes_of(p, n, k) / (p["pass_ms"][k] / 1e3) / 1e9,
                                     "frac": bytes_of(p, n, k) / (p["pass_ms"][k] / 1e3) / 1e9 / peaks["hbm_gbs"]}
                                 for k in lsh.PASS_NAMES if p["pass_launches"][k]}
        per_grid_pass[str(n)]["live_system_iterations_timed"] = p["timed_sys_iters"]
    iter_b = sum(tot_b.values())
    # the step's time split: FP32 inner CG passes (sampled events scaled by all live
    # system-iterations / the sampled ones, per grid) and the rest (refinement residuals,
    # precision conversions, host-side convergence checks, graph launch gaps)
    cg_ms = 0.0
    for p, hh in zip(prof_mx, gmx.handles):
        live = sum(sum(i["iters"] for i in I_mx[k]) for k in range(len(I_mx)) if meta[k]["n"] == hh.shape[0])
        if p["timed_sys_iters"]:
            cg_ms += sum(p["pass_ms"].values()) * live * args.steps / p["timed_sys_iters"]
    step_split = {"inner_cg_ms_est": cg_ms / args.steps, "other_ms_est": ms_mx - cg_ms / args.steps}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic_per_launch(dom, tot_b[dom] / tot_n[dom]),
                "traffic_source": NCU_TRAFFIC_SOURCE,
                "kernel": f"{dom} (FP32, all grids)", "avg_launch_ms": tot_ms[dom] / tot_n[dom],
                "algorithmic_bytes_per_launch": tot_b[dom] / tot_n[dom],
                "peak_source": peaks["source"] + " hbm_gbs (copy)",
                "pass_share_fp32": {k: tot_ms[k] / sh_sum for k in lsh.PASS_NAMES},
                "pass_frac_fp32": {k: tot_b[k] / (tot_ms[k] / 1e3) / 1e9 / peaks["hbm_gbs"]
                                   for k in lsh.PASS_NAMES if tot_n[k]},
                "whole_iteration_frac": iter_b / (sh_sum / 1e3) / 1e9 / peaks["hbm_gbs"],
                "step_split": step_split,
                "per_grid": per_grid_pass}

    # end to end through the public API: phase maps from pinned host memory in, C* out, every step
    pinned = [torch.from_numpy(st).pin_memory() for st in gmx.grid_stacks(phases)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gmx.set_microstructures(pinned)  # host -> device inside the call
        gmx.effective(tol=TOL)  # C* back on the host
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    dt = slowest_rank_ms(dt * 1e3, world, dev) / 1e3
    e2e = {"value": replica_rate(float((vox * it64).sum()), world, dt * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(t.numel() for t in pinned)), "d2h_bytes_per_step": 64 * 36 * 8,
           "s_per_step": dt}

    cpu = None
    if rank == 0 and not args.no_cpu:
        sample = batch_sample(phases, meta)
        u, secs = oracle_batch_sample(sample, mods, 4)  # about 20 s on 16 host cores
        cpu = {"value": u / secs, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
               "sample": batch_sample_text(sample, 4) + f", {secs:.1f} s"}

    per_grid = {}
    for m, e, a, b in zip(meta, errs, itmx, it64):
        g = per_grid.setdefault(str(m["n"]), {"count": 0, "inner_iters": 0, "fp64_iters": 0, "max_err": 0.0})
        g["count"] += 1
        g["inner_iters"] += int(a)
        g["fp64_iters"] += int(b)
        g["max_err"] = max(g["max_err"], e[0])
    if rank == 0:
        cfg = batch_config(meta)
        cfg["timing"] = "CUDA events on the one stream all grid handles use, around the steps"
        cfg["value_counting"] = ("sum over systems of N^3 x the plain FP64 solver's CG iterations, divided by the "
                                 "mixed solver's time (accuracy-fair); raw inner-iteration rate in mixed")
        cfg["autotune"] = {str(n): h.tune_report for n, h in zip(grid_of, gmx.handles)}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_mx, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": cfg,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks,
                "mixed": {"value_raw": value_raw, "inner_iterations_per_step": int(itmx.sum()),
                          "pass_events": f"one CG chunk in {PROF_EVERY}",
                          "c_star_max_err_vs_fp64": max(e[0] for e in errs),
                          "c_star_max_true_rel_err_vs_fp64": max(e[1] for e in errs),
                          "speedup_vs_fp64": ms_64 / ms_mx,
                          "outer_steps_per_step": int(sum(i["outer"] for inf in I_mx for i in inf)),
                          "residual_applies_per_step": int(sum(i["applies64"] for inf in I_mx for i in inf))},
                "fp64_plain": {"value": value_64, "ms_per_step": ms_64, "iterations_per_step": int(it64.sum()),
                               "clocks": clocks64},
                "per_grid": per_grid}
        print(json.dumps(line), flush=True)
    gmx.close()
    g64.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_contrast256(args):
    """The 128^3 sphere packing's centres at 256^3 (radius 16 voxels), inclusion
    stiffness 10, 100 and 1000 x the matrix: C* of the mixed-precision solver
    against the plain FP64 solver entry by entry, with both solvers' rates."""
    import torch
    from paper_1411_0330_gb300 import lsh
    from paper_1411_0330_gb300 import microstructures as ms
    torch.cuda.set_device(0)
    n = 256
    _, cen, r = ms.sphere_microstructure(N, 8.0, 0.3, seed=1411)
    ph = ms.voxelize_spheres(n, cen, r)
    ph_dev = torch.from_numpy(ph).cuda()
    V = float(ph.size)
    out = []
    for contrast in (10.0, 100.0, 1000.0):
        mods = np.array([k_mu(1.0, 0.3), k_mu(contrast, 0.2)])
        row = {"contrast": contrast}
        res = {}
        for name, prec in (("mixed", lsh.MIXED), ("fp64", lsh.FP64)):
            h = lsh.Handle(ph_dev, mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=prec,
                           tune=prec == lsh.MIXED)
            h.profile_read(reset=True)
            h.profile_enable(True, every=PROF_EVERY)
            dt, (A, infos) = _wall(lambda: h.effective(tol=TOL, maxit=40000))
            pf = h.profile_read(reset=True)
            h.profile_enable(False)
            its = sum(i["iters"] for i in infos)
            res[name] = (A, its, dt)
            row[name] = {"s": dt, "iterations": its, "voxel_it_per_s": its * V / dt,
                         "launches": pf["launches"],
                         "max_relres": max(i["relres"] for i in infos),
                         "outer": sum(i["outer"] for i in infos)}
            if prec == lsh.MIXED:
                # per-pass events of the FP32 inner CG (one chunk in PROF_EVERY), algorithmic
                # bytes of the live system-iterations over their event time
                passes = {}
                for k in lsh.PASS_NAMES:
                    if not pf["pass_launches"][k]:
                        continue
                    per_sys, table = batch_pass_bytes(k, n)
                    byts = per_sys * pf["timed_sys_iters"] + table * pf["pass_launches"][k]
                    gbs = byts / (pf["pass_ms"][k] / 1e3) / 1e9
                    passes[k] = {"ms_per_launch": pf["pass_ms"][k] / pf["pass_launches"][k], "gbs": gbs,
                                 "frac_of_copy_peak": gbs / load_peaks()["hbm_gbs"]}
                row[name]["fp32_passes"] = passes
                row[name]["autotune"] = h.tune_report
            h.close()
            del h
            torch.cuda.empty_cache()
        A_mx, A_64 = res["mixed"][0], res["fp64"][0]
        m = np.abs(A_64).max()
        row["c_star_fp64_mandel"] = A_64.tolist()
        row["c_star_abs_err_over_max"] = (np.abs(A_mx - A_64) / m).tolist()
        e_max, e_true = _cstar_err(A_mx, A_64)
        row["c_star_max_err"] = e_max
        row["c_star_max_true_rel_err_entries_ge_1e-3max"] = e_true
        row["fp64_equivalent_voxel_it_per_s"] = res["fp64"][1] * V / res["mixed"][2]
        row["speedup_mixed_vs_fp64"] = res["fp64"][2] / res["mixed"][2]
        out.append(row)
        print(json.dumps({"contrast": contrast, "err": e_max, "mixed_s": res["mixed"][2],
                          "fp64_s": res["fp64"][2]}), file=sys.stderr, flush=True)
    line = {"metric": METRIC, "value": out[0]["fp64_equivalent_voxel_it_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"256^3 isotropic elasticity, the {len(cen)} sphere centres of the 128^3 packing "
                                   f"at radius 16 vox (f={ph.mean():.4f}), E_i/E_m in 10/100/1000, nu 0.3/0.2, "
                                   "filtered Gamma, 6 Mandel loads, CG rel.res 1e-10, mixed vs FP64",
                       "value": "FP64-equivalent rate of the mixed solver at contrast 10",
                       "timing": "wall clock around the synchronous lsh_effective call, one solve each "
                                 "(first call: includes the CUDA-graph captures)"},
            "sweep": out}
    print(json.dumps(line), flush=True)
    return 0


def run_gradient128(args, nfd=32, hfd=1e-6):
    """dObj/ds for Obj = C*_1111 + C*_1212 with a per-voxel stiffness scale s ~
    U(0.5, 2) on the 128^3 packing: the adjoint gradient (torch.autograd through
    the library), timed, then checked by central differences of the variational
    estimate of Obj on nfd random voxels (FP64 solves at rel.res 1e-13 warm-started
    from the unperturbed polarisations)."""
    import torch
    from paper_1411_0330_gb300 import lsh, autograd
    from paper_1411_0330_gb300 import microstructures as ms
    torch.cuda.set_device(0)
    ph, mods, nsph = workload()
    s = ms.scale_field(ph.shape, seed=1412)
    V = ph.size
    # reference medium: the usual rule (mu0 = half the smallest shear modulus, nu0 = 0.3)
    # over the scaled moduli, whose smallest scale is 0.5
    mu0 = 0.5 * 0.5 * float(mods[:, 1].min())
    ref = np.array([mu0 * 2.0 * 1.3 / (3.0 * 0.4), mu0])
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                   scale=torch.from_numpy(s).cuda())
    # Obj = C*_1111 + C*_1212 = A[0,0] + A[5,5] / 2 in Mandel components
    W = np.zeros((6, 6))
    W[0, 0], W[5, 5] = 1.0, 0.5

    def grad_once():
        st = torch.from_numpy(s).cuda().requires_grad_(True)
        A = autograd.effective_tensor(st, h, tol=1e-12)
        obj = (A * torch.from_numpy(W).to(A)).sum()
        obj.backward()
        return float(obj), st.grad

    grad_once()
    dt, (obj, g) = _wall(grad_once)
    g = g.double().cpu().numpy()

    def obj_var(hv, phase_np, taus):
        """Variational estimate sum_p W_pp (p.A0 p + h^d (2 b_p.tau_p - tau_p.K tau_p)) on the
        handle hv with the phase map phase_np, returned as per-voxel terms so that differences
        are taken voxel by voxel."""
        hv.set_microstructure(phase_np, s)
        terms = []
        for j, tau0 in zip((0, 5), taus):
            load = np.zeros(6)
            load[j] = 1.0
            tau, info = hv.solve(load, tau=tau0.clone(), tol=1e-13, warm_start=True, maxit=20000)
            Kt = hv.apply(tau)
            t_np, k_np = tau.cpu().numpy(), Kt.cpu().numpy()
            # b = p on I0 and tau = 0 off I0, so b.tau = p.tau summed over all voxels
            terms.append(W[j, j] * (2.0 * t_np[j] - (t_np * k_np).sum(axis=0)))
        return terms[0] + terms[1]

    rng = np.random.default_rng(1413)
    vox = rng.choice(V, size=nfd, replace=False)
    base = []
    h.set_microstructure(ph, s)
    for j in (0, 5):
        load = np.zeros(6)
        load[j] = 1.0
        tau, _ = h.solve(load, tol=1e-13)
        base.append(tau)
    h.close()
    torch.cuda.empty_cache()
    fd, ad = [], []
    t0 = time.perf_counter()
    ph_flat, s_flat = ph.reshape(-1), s.reshape(-1)
    for v in vox:
        # the perturbation s_v -> s_v +- h in FP64: voxel v moves to an extra phase whose
        # moduli are (1 +- h / s_v) A_phase(v), so that s_v A stays the stored FP32 s_v
        # times an FP64 factor (the scale field itself is FP32)
        sv, pv = float(s_flat[v]), int(ph_flat[v])
        m4 = np.vstack([mods, (1.0 + hfd / sv) * mods[pv], (1.0 - hfd / sv) * mods[pv]])
        hv = lsh.Handle(torch.from_numpy(ph).cuda(), m4, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                        scale=torch.from_numpy(s).cuda(), max_systems=1)
        pp, pm = ph_flat.copy(), ph_flat.copy()
        pp[v], pm[v] = 2, 3
        dp = obj_var(hv, pp.reshape(ph.shape), base)
        dm = obj_var(hv, pm.reshape(ph.shape), base)
        fd.append(float((dp - dm).sum()) / V / (2.0 * hfd))
        ad.append(float(g.reshape(-1)[v]))
        hv.close()
        del hv
        torch.cuda.empty_cache()
    t_fd = time.perf_counter() - t0
    fd, ad = np.array(fd), np.array(ad)
    relerr = np.abs(fd - ad) / np.abs(ad).max()
    line = {"metric": "adjoint gradient dObj/ds of C*_1111 + C*_1212 (128^3, FP64 solves)", "value": dt,
            "unit": "s per gradient (6 solves + adjoint contraction)", "n_gpus": 1, "higher_is_better": False,
            "dtype": "f64 (scale field f32)", "data": "synthetic",
            "config": {"workload": f"128^3 sphere packing (seed 1411, {nsph} spheres), per-voxel scale "
                                   "s ~ U(0.5,2) (seed 1412) on the phase moduli, filtered Gamma, tol 1e-12",
                       "fd": f"central differences of the variational estimate on {nfd} voxels (seed 1413), "
                             f"h={hfd:g} applied in FP64 (an extra phase with moduli (1 +- h/s_v) A_phase at "
                             "the perturbed voxel), FP64 solves at 1e-13 warm-started"},
            "objective": obj, "fd_vs_adjoint_max_err_over_max_grad": float(relerr.max()),
            "fd_vs_adjoint_median_err_over_max_grad": float(np.median(relerr)),
            "grad_abs_max": float(np.abs(g).max()), "fd_seconds": t_fd,
            "samples": [{"voxel": int(v), "adjoint": a, "fd": f} for v, a, f in zip(vox[:8], ad[:8], fd[:8])]}
    print(json.dumps(line), flush=True)
    return 0


def run_convergence(args, grids=(16, 32, 64, 128, 256), fine=512):
    """Grid convergence of C* (the Table 2 / Fig. 2-3 kind of study) on a synthetic
    500-sphere hard-sphere packing at f = 0.4 (Monte Carlo, seed 1411): each grid
    N solved with the centre rule (one phase per voxel) and with the sub-voxel
    averaged local operator of Eq. (def_ah) (volume fractions from a 512^3
    lattice); mixed-precision solver, filtered Gamma, contrast 10, tol 1e-9.
    Reports C*_1111, C*_1212 against N and the observed rate of the differences
    between successive grids."""
    import torch
    from paper_1411_0330_gb300 import lsh
    from paper_1411_0330_gb300 import microstructures as ms
    torch.cuda.set_device(0)
    nsph, f = 500, 0.4
    r = (f * 3.0 / (4.0 * np.pi * nsph)) ** (1.0 / 3.0)
    cen = ms.hard_sphere_mc(r, nsph, seed=1411)
    fine_ph = ms.voxelize_spheres(fine, cen, r)
    mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    rows = []
    for n in grids:
        k = fine // n
        frac = fine_ph.reshape(n, k, n, k, n, k).mean(axis=(1, 3, 5), dtype=np.float64).astype(np.float32)
        centre = ms.voxelize_spheres(n, cen, r)
        row = {"n": n}
        for name, kw in (("centre", {}), ("averaged", {"fraction": torch.from_numpy(frac).cuda()})):
            ph = centre if name == "centre" else np.zeros_like(centre)
            h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED,
                           precision=lsh.MIXED, **kw)
            dt, (A, infos) = _wall(lambda: h.effective(tol=1e-9))
            row[name] = {"C1111": float(A[0, 0]), "C1212": float(A[5, 5] / 2.0), "s": dt,
                         "iterations": sum(i["iters"] for i in infos),
                         "f": float(ph.mean()) if name == "centre" else float(frac.mean())}
            h.close()
            del h
            torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    rates = {}
    for name in ("centre", "averaged"):
        for comp in ("C1111", "C1212"):
            v = [row[name][comp] for row in rows]
            d = [abs(v[i + 1] - v[i]) for i in range(len(v) - 1)]
            rates[f"{name}_{comp}"] = [float(np.log2(d[i] / d[i + 1])) if d[i + 1] > 0 else None
                                       for i in range(len(d) - 1)]
    line = {"metric": "grid convergence of C* (centre rule vs sub-voxel averaged local operator)",
            "value": rows[-1]["averaged"]["C1111"], "unit": "C*_1111 at the finest grid", "n_gpus": 1,
            "data": "synthetic",
            "config": {"workload": f"{nsph} hard spheres (MC, seed 1411), f={f}, r={r:.4f}, E 1/10 nu 0.3/0.2, "
                                   f"filtered Gamma, mixed solver tol 1e-9, fractions from a {fine}^3 lattice",
                       "grids": list(grids)},
            "rows": rows, "observed_rates_log2": rates}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- main arm
def run_cufft(args, reps=20):
    """Timed comparison with the vendor FFT: cuFFT (through torch.fft) forward R2C
    and inverse C2R of the 6 load systems x 6 components of the 128^3 FP32 field
    (the transforms alone: no Gamma^h, local term, projection or CG vector work),
    against this library's five FP32 operator passes at the same size, which do
    all of that, as the inner CG of the mixed solver runs them."""
    import torch
    from paper_1411_0330_gb300 import lsh
    torch.cuda.set_device(0)
    ph, mods, _ = workload()
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    tune = h.autotune()
    h.effective(tol=1e-30, maxit=8, raise_on_fail=False)  # warm-up, graph capture
    h.profile_read(reset=True)
    h.profile_enable(True)
    h.effective(tol=1e-30, maxit=40, raise_on_fail=False)
    pf = h.profile_read(reset=True)
    h.profile_enable(False)
    ours = {k: pf["pass_ms"][k] / max(pf["pass_launches"][k], 1) for k in lsh.PASS_NAMES}
    h.close()
    del h
    torch.cuda.empty_cache()
    x = torch.randn(6, 6, N, N, N, device="cuda", dtype=torch.float32)
    dims = (-3, -2, -1)
    X = torch.fft.rfftn(x, dim=dims)
    y = torch.fft.irfftn(X, s=(N, N, N), dim=dims)
    err = float((y - x).abs().max() / x.abs().max())
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(3):
        torch.fft.rfftn(x, dim=dims, out=X)
        torch.fft.irfftn(X, s=(N, N, N), dim=dims, out=y)
    torch.cuda.synchronize()
    fwd = inv = 0.0
    for _ in range(reps):  # 302 MB field and 307 MB spectrum: larger than L2
        e[0].record()
        torch.fft.rfftn(x, dim=dims, out=X)
        e[1].record()
        torch.fft.irfftn(X, s=(N, N, N), dim=dims, out=y)
        e[2].record()
        torch.cuda.synchronize()
        fwd += e[0].elapsed_time(e[1])
        inv += e[1].elapsed_time(e[2])
    fwd /= reps
    inv /= reps
    fft_passes = ["x_forward", "y_forward", "z_gamma", "y_inverse", "x_inverse_local"]
    ours_fft = sum(ours[k] for k in fft_passes)
    line = {"workload": "cufft_comparison",
            "config": {"grid": [N, N, N], "fields": "6 load systems x 6 components, FP32",
                       "variants": {k: tune[k] for k in ("xf_variant", "x_variant", "y_variant", "z_variant")}},
            "cufft_ms": {"rfftn": fwd, "irfftn": inv, "sum": fwd + inv, "round_trip_max_rel_err": err},
            "lsh_ms": {"passes": ours, "five_operator_passes": ours_fft,
                       "with_cg_update": ours_fft + ours["cg_update"]},
            "ratio_cufft_over_lsh_operator": (fwd + inv) / ours_fft}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lsh", choices=["lsh", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--concurrent", action="store_true",
                    help="solve the filtered and truncated handles together, one stream each")
    ap.add_argument("--workload", default="batch64",
                    choices=["spheres128", "batch64", "contrast256", "gradient128", "convergence", "cufft"],
                    help="batch64: 64 microstructures of uneven grids, mixed+batched vs FP64 (default); "
                         "spheres128: the 128^3 sphere packing, filtered and truncated; contrast256: 256^3 mixed vs FP64 at contrasts "
                         "10/100/1000; gradient128: adjoint gradient of C* and its finite-difference check; "
                         "convergence: C* against the grid, centre rule vs sub-voxel averaging; cufft: "
                         "the FP32 operator passes against cuFFT R2C + C2R alone at 128^3")
    ap.add_argument("--profile-case", choices=["fp64", "mixed", "mixed96"], default=None,
                    help="small case for ncu: 4 CG iterations of one 128^3 (96^3) filtered solve, then exit")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.workload == "batch64":
        return run_batch(args, rank, world, local)
    if args.workload == "spheres128":
        return run_spheres128(args, rank, world, local)
    if args.workload == "contrast256":
        return run_contrast256(args)
    if args.workload == "gradient128":
        return run_gradient128(args)
    if args.workload == "convergence":
        return run_convergence(args)
    if args.workload == "cufft":
        return run_cufft(args)
    return 0


def run_spheres128(args, rank, world, local):
    """One 128^3 packing (the 3D elasticity configuration), filtered and truncated
    operators, 6 loads each: mixed precision against plain FP64."""
    import torch
    import torch.distributed as dist
    from paper_1411_0330_gb300 import lsh

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ph, mods, nsph = workload()
    ph_dev = torch.from_numpy(ph).to(dev)
    V = ph.size
    greens = (lsh.FILTERED, lsh.TRUNCATED)
    # with --concurrent each handle has its own stream and the two operators'
    # solves run together (lsh_effective_batch: one host thread per handle)
    streams = [torch.cuda.Stream(dev) if args.concurrent else None for _ in range(4)]
    h64 = [lsh.Handle(ph_dev, mods, physics=lsh.ELASTIC, green=g, stream=streams[i]) for i, g in enumerate(greens)]
    hmx = [lsh.Handle(ph_dev, mods, physics=lsh.ELASTIC, green=g, precision=lsh.MIXED, tune=True,
                      stream=streams[2 + i]) for i, g in enumerate(greens)]

    def step(handles):
        its, res = 0, []
        if args.concurrent:
            As, Is = lsh.effective_batch(handles, tol=TOL)
            for A, infos in zip(As, Is):
                its += sum(i["iters"] for i in infos)
                res.append((A, infos))
            return its, res
        for h in handles:
            A, infos = h.effective(tol=TOL)
            its += sum(i["iters"] for i in infos)
            res.append((A, infos))
        return its, res

    def timed(handles, profile, name, steps=None):
        steps = steps or args.steps
        for h in handles:
            h.profile_read(reset=True)
            h.profile_enable(bool(profile), every=int(profile))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(name)  # lets a profiler select the timed region
        e0.record(stream)
        tot_its, last = 0, None
        for _ in range(steps):
            its, last = step(handles)
            tot_its += its
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        ms = slowest_rank_ms(ms, world, dev)
        profs = [h.profile_read(reset=True) for h in handles]
        for h in handles:
            h.profile_enable(False)
        return ms, tot_its, last, profs, clocks

    for _ in range(args.warmup):
        step(hmx)
        step(h64)
    # headline: the mixed-precision solver, all 6 loads of a handle batched in one launch sequence.
    # Per-pass CUDA events are recorded in one CG chunk of PROF_EVERY (event nodes in every
    # graph would add gaps between the kernels: 3.4% on the step)
    ms_mx, its_mx, last_mx, prof_mx, clocks = timed(hmx, PROF_EVERY, "timed_mixed")
    # comparison: the plain FP64 solver on the same workload
    ms_64, its_64, last_64, prof_64, clocks64 = timed(h64, PROF_EVERY, "timed_fp64")
    nrep = world
    value_64 = replica_rate(its_64 * V, nrep, ms_64)
    value_raw = replica_rate(its_mx * V, nrep, ms_mx)
    value = replica_rate(its_64 * V, nrep, ms_mx)  # FP64-equivalent: the FP64 solver's iterations, mixed time
    cerr = max(float(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()) for a, b in zip(last_mx, last_64))
    launches = sum(p["launches"] for p in prof_mx)

    # roofline of the dominant FP32 pass of the inner CG (largest share of the
    # timed region over both handles), from the live per-pass events
    peaks = load_peaks()
    nxh = N // 2 + 1

    def pass_bytes(k, filtered):
        """Algorithmic bytes of one launch over the 6 load systems; the Gamma table
        (filtered operator only; the truncated one is computed in the kernel) counts once."""
        b = 6 * pass_traffic(k, V, 6, N, nxh, 21 if filtered else 0, 4)
        if k == "z_gamma" and filtered:
            b -= 5 * V * 21 * 4 * nxh / N
        return b

    tot_ms = {k: sum(p["pass_ms"][k] for p in prof_mx) for k in lsh.PASS_NAMES}
    tot_n = {k: sum(p["pass_launches"][k] for p in prof_mx) for k in lsh.PASS_NAMES}
    dom = max(tot_ms, key=tot_ms.get)
    dom_bytes = sum(pass_bytes(dom, i == 0) * prof_mx[i]["pass_launches"][dom] for i in range(len(prof_mx)))
    avg_ms = tot_ms[dom] / max(tot_n[dom], 1)
    byts = dom_bytes / max(tot_n[dom], 1)
    achieved = dom_bytes / (tot_ms[dom] / 1e3) / 1e9
    sh_sum = max(sum(tot_ms.values()), 1e-30)
    pf = prof_mx[0]

    def gbs(p, filtered):
        return {k: pass_bytes(k, filtered) / (p["pass_ms"][k] / p["pass_launches"][k] / 1e3) / 1e9
                for k in lsh.PASS_NAMES if p["pass_launches"][k]}

    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC_FP32.get(dom),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch (filtered)",
                "kernel": f"{dom} (FP32, both operators)", "avg_launch_ms": avg_ms,
                "algorithmic_bytes_per_launch": byts, "peak_source": peaks["source"] + " hbm_gbs (copy)",
                "pass_avg_ms_fp32": {k: pf["pass_ms"][k] / max(pf["pass_launches"][k], 1) for k in lsh.PASS_NAMES},
                "pass_share_fp32": {k: tot_ms[k] / sh_sum for k in lsh.PASS_NAMES},
                "pass_gbs_fp32": gbs(pf, True),
                "pass_gbs_fp32_truncated": gbs(prof_mx[1], False) if len(prof_mx) > 1 else None,
                "pass_frac_fp32": {k: v / peaks["hbm_gbs"] for k, v in gbs(pf, True).items()}}
    p64 = prof_64[0]
    fp64_alu = {k: 6 * pass_flops(k, V, 6, N, N, N, nxh) / (p64["pass_ms"][k] / max(p64["pass_launches"][k], 1) / 1e3)
                / 1e9 for k in lsh.PASS_NAMES if p64["pass_launches"][k]}

    # end to end through the C ABI: host phase map in, C* out, every step (mixed solver)
    ph_pinned = torch.from_numpy(ph).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for h in hmx:
            h.set_microstructure(ph_pinned)  # host -> device inside the call
            h.effective(tol=TOL)  # C* back on the host
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    e2e = {"value": its_64 * V * nrep / dt, "unit": UNIT, "h2d_bytes_per_step": 2 * V,
           "d2h_bytes_per_step": 2 * 36 * 8}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_sample(ph, mods, iters=20)  # about 10 s on 16 host cores

    if rank == 0:
        cfg = config(nsph, float(ph.mean()))
        cfg["solver"] = ("mixed precision (FP32 FFT/Gamma/CG vectors, FP64 inner-product accumulation, "
                         "iterative-refinement residual to FP64 accuracy in double-float arithmetic on the "
                         "FP32 pipes), 6 loads batched per launch")
        cfg["value_counting"] = ("N^3 x CG iterations of the plain FP64 solver on the same 12 solves, divided by "
                                 "the mixed solver's time (accuracy-fair); raw inner-iteration rate in mixed")
        cfg["autotune"] = {"filtered": hmx[0].tune_report, "truncated": hmx[1].tune_report}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_mx / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks,
                "mixed": {"value_raw": value_raw, "inner_iterations_per_step": its_mx / args.steps,
                          "pass_events": f"one CG chunk in {PROF_EVERY}",
                          "c_star_max_rel_err_vs_fp64": cerr,
                          "speedup_vs_fp64": ms_64 / ms_mx,
                          "outer_steps_per_step": sum(i["outer"] for r in last_mx for i in r[1]),
                          "residual_applies_per_step": sum(i["applies64"] for r in last_mx for i in r[1]),
                          "residual_arithmetic": "double-float" if os.environ.get("LSH_NO_DF") != "1" else "fp64"},
                "fp64_plain": {"value": value_64, "ms_per_step": ms_64 / args.steps,
                               "iterations_per_step": its_64 / args.steps, "clocks": clocks64,
                               "pass_avg_ms": {k: p64["pass_ms"][k] / max(p64["pass_launches"][k], 1)
                                               for k in lsh.PASS_NAMES},
                               "fp64_gflops_conventional": fp64_alu,
                               "c_star_filtered_1111_1212": [float(last_64[0][0][0, 0]),
                                                             float(last_64[0][0][5, 5] / 2)]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
