#!/usr/bin/env python3
"""Throughput of the coupled model-H step (fluctuating LB + stochastic psi step).

Default workload: the D3Q19 512^3 spinodal quench (A -0.0625, B 0.0625, K 0.04,
M 0.1, kT 1e-5, psi0 uniform in [-0.01, 0.01], u0 = 0), FP32 population
deviations, finite-volume psi scheme, Heun integrator, structure factor
|k_a| <= 8 accumulated every 10 steps.  One "step" advances every lattice site
once in both equations.  Metric: coupled lattice-site updates per second
(MLUPS), whole job.  Replicas only: with N GPUs every rank advances its own
512^3 box (weak scaling, no data-path collective).

--impl reference times the FP64 CPU checker on a bounded sample of the same
workload (a 48^3 box with the same parameters) on the host cores.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALG_BYTES_SITE = {0: 160, 1: 84}          # populations in+out + psi in+out, FP32 / FP16 deviations
LB_ALG_BYTES_SITE = {0: 152, 1: 76}       # populations in+out (the LB kernel's share)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=512, help="edge of the cubic box")
    ap.add_argument("--storage", choices=["f32", "f16"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default psi tile depth (64 planes)")
    ap.add_argument("--variant-size", type=int, default=512,
                    help="edge of the cubic box of the path variants (2D variant: 8x this edge)")
    ap.add_argument("--variants", default="",
                    help="comma-separated variant names to run (default: all)")
    ap.add_argument("--variant-steps", type=int, default=10,
                    help="steps timed for each variant of the path (FD scheme, FP16 storage, D2Q9); 0 skips them")
    ap.add_argument("--ensemble-steps", type=int, default=40,
                    help="steps of the 256-replica ensemble timed batched vs plain (0: skip)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The step time of the job: the slowest rank's (an all-reduce MAX of one
    float; NCCL on the GPUs, any backend the process group has)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_sites: int, steps: int, world: int, ms: float) -> float:
    """Whole-job MLUPS: every rank advances its own n_sites replica `steps`
    times (weak scaling), over the slowest rank's time in ms."""
    return n_sites * steps * world / (ms / 1e3) / 1e6


def replica_seeds(base_seed: int, rank: int):
    """(Philox seed, psi0 seed) of this rank's replica: independent per rank."""
    return base_seed + rank, 11 + rank


def workload(size: int, storage: int):
    from paper_1104_0078_gb300 import inputs as I
    d = dict(I.WORKLOADS["quench"])
    d.update(nx=size, ny=size, nz=size)
    name = f"D3Q19 {size}^3 spinodal quench, {'FP32' if storage == 0 else 'FP16'} deviations, FV, Heun"
    return d, name


def oracle_mlups(d: dict, box: int, budget_s: float, nsteps=None):
    """Time the FP64 checker on a box^3 sample with the workload's parameters."""
    import oracle as O
    from paper_1104_0078_gb300 import inputs as I
    p = O.Params(dim=3, q=19, nx=box, ny=box, nz=box, tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"],
                 M=d["M"], scheme=1, integrator=2, coupling=3, seed=d["seed"])
    st = O.State.rest(p, psi=I.uniform_field(p.n, -0.01, 0.01, 11))
    t0 = time.perf_counter()
    st.advance(1)
    t1 = time.perf_counter() - t0
    n = nsteps if nsteps is not None else max(1, int(budget_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    st.advance(n)
    dt = time.perf_counter() - t0
    return p.n * n / dt / 1e6, n, dt, O.threads()


def cpu_baselines(d: dict) -> dict:
    """The FP64 checker on the host cores, bounded to about half a minute: on all
    cores and on one thread, on samples of the quench workload (64^3 and 32^3
    boxes, same parameters), and the 2D bulk workload (D2Q9 64^2, FD, Heun) as a
    full 2000-step run on all cores."""
    import oracle as O
    from paper_1104_0078_gb300 import inputs as I
    mlups, n, dt, cores = oracle_mlups(d, 64, 15.0)
    out = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{n} coupled steps of a 64^3 box with the workload's parameters, FP64, all host cores",
           "build": "gcc -O3 -fopenmp -ffp-contract=off (no -march=native: host code builds alike on both machines)"}
    O.set_threads(1)
    try:
        m1, n1, _, _ = oracle_mlups(d, 32, 8.0)
    finally:
        O.set_threads(cores)
    out["single_thread"] = {"value": m1, "unit": "MLUPS", "cores": 1,
                            "sample": f"{n1} coupled steps of a 32^3 box with the workload's parameters"}
    b = dict(I.WORKLOADS["bulk_2d"])
    p = O.Params(dim=2, q=9, nx=b["nx"], ny=b["ny"], nz=1, tau=b["tau"], kT=b["kT"], A=b["A"], B=b["B"], K=b["K"],
                 M=b["M"], scheme=0, integrator=2, coupling=3, seed=1)
    st = O.State.rest(p)
    t0 = time.perf_counter()
    st.advance(2000)
    dt2 = time.perf_counter() - t0
    out["bulk_2d_full_run"] = {"value": p.n * 2000 / dt2 / 1e6, "unit": "MLUPS", "cores": cores,
                               "sample": "D2Q9 64^2, FD, Heun, 2000 steps (the whole run)", "seconds": dt2}
    return out


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 - 0.15 <= t <= t1 + 0.15] or [l for (_, l) in self.lines[-3:]]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in rows:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_sm_max_mhz() -> float:
    """Maximum SM clock recorded beside the measured peaks (2070 MHz if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return 2070.0


LB_SOURCES = ("flb_lb3d.cu", "flb_site3d.cuh", "flb_internal.cuh", "flb_lane.cuh")


def lb_source_sha():
    """sha256 over the sources the collide-stream kernel is compiled from."""
    h = hashlib.sha256()
    for name in LB_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1104_0078_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def lb_record(storage: int):
    """The committed ncu record of the LB kernel, if it was taken on the current
    kernel sources and storage, else None."""
    path = os.path.join(ROOT, "profiles", "lb_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != lb_source_sha() or rec.get("storage") != storage:
        return None
    return rec


def lb_traffic(storage: int, n_sites: int):
    """DRAM bytes per LB launch from the committed ncu record, scaled by sites
    when the capture was smaller."""
    rec = lb_record(storage)
    try:
        return rec["dram_bytes_per_launch"] * n_sites / rec["sites"] if rec else None
    except KeyError:
        return None


def lb_issue_roofline(storage: int, n_sites: int, lb_ms: float, n_sm: int, sm_max_mhz: float):
    """Secondary (ALU) roofline of the LB kernel: its executed instructions per
    launch (ncu record, scaled by sites; every lane of every warp is active) over
    its live launch time, against the issue peak of one warp-instruction per
    scheduler and cycle: SMs x 4 schedulers x 32 lanes x the maximum SM clock."""
    rec = lb_record(storage)
    if not rec or "warp_inst_per_launch" not in rec or not lb_ms:
        return None
    warp_inst = rec["warp_inst_per_launch"] * n_sites / rec["sites"]
    achieved = 32 * warp_inst / (lb_ms / 1e3) / 1e12
    peak = n_sm * 4 * 32 * sm_max_mhz * 1e6 / 1e12
    return {"bound": "alu", "kernel": "LB collide-stream", "achieved": achieved, "peak": peak,
            "unit": "T thread-instructions/s", "frac": achieved / peak,
            "inst_per_site": 32 * warp_inst / n_sites,
            "peak_from": f"{n_sm} SMs x 4 schedulers x 1 warp-instruction/cycle x 32 lanes x {sm_max_mhz:.0f} MHz"}


def ensemble_batched_vs_plain(F, I, steps, local, rank, autotune=True):
    """256 uneven D3Q19 replicas (64 each of 16^3, 24^3, 32^3, 48^3, kT_r in
    [1e-5, 1e-4], seed 1 + r): aggregate MLUPS of the plain per-replica launch
    sequence, of the batched mode (one launch per phase for all replicas,
    CUDA-graph replay) and of the persistent mode (one cooperative launch for
    all replicas and all steps), same state, same number of steps."""
    import torch
    reps = I.ensemble()
    ps = [F.flb_params_default(nx=d["nx"], ny=d["ny"], nz=d["nz"], tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"],
                               K=d["K"], M=d["M"], psi_scheme=F.FLB_FV, integrator=F.FLB_HEUN, seed=d["seed"] + 1000 * rank)
          for d in reps]
    sites = sum(p.nx * p.ny * p.nz for p in ps)
    out = {"workload": "256 D3Q19 replicas (64 each of 16^3, 24^3, 32^3, 48^3), FV, Heun", "sites": sites,
           "steps": steps}
    for mode, key in ((F.FLB_MODE_PLAIN, "plain"), (F.FLB_MODE_BATCHED, "batched"),
                      (F.FLB_MODE_PERSISTENT, "persistent")):
        s = F.Solver(ps, device=f"cuda:{local}")
        s.set_mode(mode)
        if autotune:
            out[key + "_psi_zchunk"] = sorted(set(s.autotune()))
        s.step(3)
        s.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[key + "_mlups"] = sites * steps / (ms / 1e3) / 1e6
        out[key + "_ms_per_step"] = ms / steps
        del s
        torch.cuda.empty_cache()
    out["ratio"] = out["batched_mlups"] / out["plain_mlups"]
    out["persistent_vs_plain"] = out["persistent_mlups"] / out["plain_mlups"]
    return out


def ensemble_d3q15(F, I, steps, local, rank, autotune=True):
    """25 replicas of the paper's own fluctuation run on its lattice (Sec. VI:
    D3Q15 32^3, tau 1.1, kT 1/3000, A 0.625, B = K = 0, M 0.095; seeds 1..25),
    with the FV psi scheme (the batched modes run the FV stage): aggregate MLUPS
    of the plain per-replica launches, the batched graph and the persistent
    launch, same state, same number of steps."""
    import torch
    d = dict(I.WORKLOADS["fluct_d3q15"])
    ps = [F.flb_params_default(q=15, nx=d["nx"], ny=d["ny"], nz=d["nz"], tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"],
                               K=d["K"], M=d["M"], psi_scheme=F.FLB_FV, integrator=F.FLB_HEUN, seed=1 + r + 1000 * rank)
          for r in range(25)]
    sites = sum(p.nx * p.ny * p.nz for p in ps)
    out = {"workload": "25 D3Q15 32^3 replicas, the paper's fluctuation run (tau 1.1, kT 1/3000, A 0.625, "
                       "M 0.095), FV, Heun", "sites": sites, "steps": steps}
    for mode, key in ((F.FLB_MODE_PLAIN, "plain"), (F.FLB_MODE_BATCHED, "batched"),
                      (F.FLB_MODE_PERSISTENT, "persistent")):
        s = F.Solver(ps, device=f"cuda:{local}")
        s.set_mode(mode)
        if autotune:
            out[key + "_psi_zchunk"] = sorted(set(s.autotune()))
        s.step(3)
        s.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[key + "_mlups"] = sites * steps / (ms / 1e3) / 1e6
        out[key + "_ms_per_step"] = ms / steps
        del s
        torch.cuda.empty_cache()
    out["ratio"] = out["batched_mlups"] / out["plain_mlups"]
    out["persistent_vs_plain"] = out["persistent_mlups"] / out["plain_mlups"]
    return out


def path_variants(F, I, local, steps, peak, n=512, only=(), autotune=True):
    """Throughput of the other forms of the path, each on its own handle after 3
    warm-up steps, inputs larger than L2 at the default n = 512: the FD psi
    scheme, the FP16 storage variant, the RK4 integrator, the stress-form force
    and the D3Q15 lattice (FD) on the n^3 quench; the quench with S(q) and the
    dynamic S(q, tau) (8 lags) sampled every 10 steps; the per-site general
    path of the paper's stencil studies: FD with the PK Laplacian, the naive
    contrast scheme with the CD Laplacian, FV on D3Q15; the single-pass Heun
    step (both stages in one launch) of the FV and FD schemes; and the D2Q9 path on an
    (8n)^2 quench (same free energy, FD as in the 2D workload).  MLUPS and the
    fraction of the HBM roofline on the algorithmic bytes of that form."""
    import torch
    d = dict(I.WORKLOADS["quench"])
    cube = dict(nx=n, ny=n, nz=n)
    forms = [
        (f"fd_{n}", dict(cube, psi_scheme=F.FLB_FD), 160),
        (f"fp16_{n}", dict(cube, psi_scheme=F.FLB_FV, storage=F.FLB_F16_DEV), 84),
        (f"rk4_{n}", dict(cube, psi_scheme=F.FLB_FV, integrator=F.FLB_RK4), 160),
        (f"stress_force_{n}", dict(cube, psi_scheme=F.FLB_FV, force_grad=F.FLB_FORCE_STRESS), 160),
        (f"d3q15_fd_{n}", dict(cube, q=15, psi_scheme=F.FLB_FD), 128),
        (f"sq_dynamic_{n}", dict(cube, psi_scheme=F.FLB_FV, sq_kmax=8, sq_lags=8), 160, (10, 1 | 4)),
        (f"pk_laplacian_fd_{n}", dict(cube, psi_scheme=F.FLB_FD, laplacian=F.FLB_LAP_PK), 160),
        (f"naive_cd_{n}", dict(cube, psi_scheme=F.FLB_NAIVE, laplacian=F.FLB_LAP_CD), 160),
        (f"d3q15_fv_{n}", dict(cube, q=15, psi_scheme=F.FLB_FV), 128),
        (f"heun_fused_{n}", dict(cube, psi_scheme=F.FLB_FV), 160, None, True),
        (f"heun_fused_fd_{n}", dict(cube, psi_scheme=F.FLB_FD), 160, None, True),
        (f"d2q9_{8 * n}", dict(dim=2, q=9, nx=8 * n, ny=8 * n, nz=1, psi_scheme=F.FLB_FD), 80),
    ]
    if only:
        forms = [f for f in forms if f[0].rsplit("_", 1)[0] in only]
    out = {}
    for key, kw, alg, *extra in forms:
        sampling = extra[:1] if extra and extra[0] is not None else []
        fused = len(extra) > 1 and extra[1]
        kw = {"integrator": F.FLB_HEUN, **kw}
        p = F.flb_params_default(tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"], K=d["K"], M=d["M"],
                                 seed=d["seed"], **kw)
        N = p.nx * p.ny * p.nz
        s = F.Solver(p, device=f"cuda:{local}")
        s.set_fields(psi=I.uniform_field(N, -0.01, 0.01, 11))
        if fused:   # both Heun stages of psi in one launch (halo recompute); tuned as such
            s.set_psi_fused(True)
        if p.dim == 3 and autotune:
            s.autotune()
        if sampling:
            s.set_sampling(*sampling[0])
        s.step(3)
        s.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        mlups = N / (ms / 1e3) / 1e6
        out[key] = {"mlups": mlups, "ms_per_step": ms, "alg_bytes_per_site": alg,
                    "step_frac_of_peak": alg * N / (ms / 1e3) / 1e9 / peak}
        del s
        torch.cuda.empty_cache()
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    storage = 0 if args.storage == "f32" else 1
    d, name = workload(args.size, storage)
    box = 48
    # each step: one checker step on a 48^3 sample of the workload
    for _ in range(max(args.warmup, 0)):
        oracle_mlups(d, box, 0, nsteps=1)
    mlups, n, dt, cores = oracle_mlups(d, box, 0, nsteps=args.steps)
    line = {
        "impl": "reference", "metric": "coupled lattice-site updates/s", "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / n * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "sample": f"{box}^3 box, same parameters"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{n} steps of a {box}^3 box"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1104_0078_gb300 as F
    from paper_1104_0078_gb300 import inputs as I

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    storage = F.FLB_F32_DEV if args.storage == "f32" else F.FLB_F16_DEV
    d, name = workload(args.size, storage)
    p = F.flb_params_default(nx=d["nx"], ny=d["ny"], nz=d["nz"], tau=d["tau"], kT=d["kT"], A=d["A"], B=d["B"],
                             K=d["K"], M=d["M"], psi_scheme=F.FLB_FV, integrator=F.FLB_HEUN, storage=storage,
                             seed=replica_seeds(d["seed"], rank)[0], sq_kmax=8)
    N = p.nx * p.ny * p.nz
    s = F.Solver(p, device=f"cuda:{local}")
    psi0 = I.uniform_field(N, -0.01, 0.01, replica_seeds(d["seed"], rank)[1])
    s.set_fields(psi=psi0)
    zchunk = s.autotune()[0] if not args.no_autotune else s.get_tuning(0)
    s.set_sampling(10, 1)
    s.step(args.warmup)
    s.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    l0 = s.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.perf_counter()
    ev0.record(s.stream)
    s.step(args.steps)
    ev1.record(s.stream)
    ev1.synchronize()
    tw1 = time.perf_counter()
    barrier()
    launches = s.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    sampler.stop()
    clocks = sampler.summary(tw0, tw1)
    ms = max_over_ranks(ms, dist, f"cuda:{local}")
    value = job_value(N, args.steps, ws, ms)

    # live per-kernel timing on the library's stream (CUDA events around each launch)
    s.set_profiling(True)
    kp = min(args.steps, 20)
    s.step(kp)
    kms, kcnt = s.kernel_times()
    s.set_profiling(False)
    lb_ms = kms["lb"] / max(kcnt["lb"], 1)
    peak, peak_kind = measured_peak()
    lb_bytes = LB_ALG_BYTES_SITE[storage] * N
    achieved = lb_bytes / (lb_ms / 1e3) / 1e9
    step_ms = ms / args.steps
    step_gbs = ALG_BYTES_SITE[storage] * N / (step_ms / 1e3) / 1e9
    sm_max = (clocks or {}).get("sm_max_mhz") or measured_sm_max_mhz()
    issue = lb_issue_roofline(storage, N, lb_ms, torch.cuda.get_device_properties(local).multi_processor_count, sm_max)

    # end to end through the public API: upload the initial field, step, read the
    # totals and the final psi field back
    e2e = None
    if not args.no_e2e:
        s2 = s  # reuse the handle and workspace; set_fields re-initialises the state
        barrier()
        t0 = time.perf_counter()
        s2.set_fields(psi=psi0)
        s2.step(args.steps)
        tot, u2, rc = s2.moments()
        psi_end = s2.get_psi()
        t1 = time.perf_counter()
        assert psi_end.shape == (N,)
        e2e_ms = max_over_ranks((t1 - t0) * 1e3, dist, f"cuda:{local}")
        h2d = 4 * N  # psi0 as interior FP32 values (padded on the device; u0 = 0 is a device memset)
        d2h = 72 + 4 * N  # the totals, and psi as interior FP32 values (gathered on the device)
        e2e = {"value": job_value(N, args.steps, ws, e2e_ms), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}
    ens = None
    if args.ensemble_steps > 0:
        del s
        torch.cuda.empty_cache()
        ens = ensemble_batched_vs_plain(F, I, args.ensemble_steps, local, rank, autotune=not args.no_autotune)
        ens["d3q15_paper_ensemble"] = ensemble_d3q15(F, I, args.ensemble_steps, local, rank,
                                                     autotune=not args.no_autotune)
    variants = None
    if args.variant_steps > 0 and rank == 0:
        only = tuple(v for v in args.variants.split(",") if v)
        variants = path_variants(F, I, local, args.variant_steps, peak, n=args.variant_size, only=only,
                                 autotune=not args.no_autotune)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(d)
    if rank == 0:
        line = {
            "metric": "coupled lattice-site updates/s", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if storage == 0 else "f16-storage/f32",
            "data": "synthetic",
            "config": {"workload": name, "box": [p.nx, p.ny, p.nz], "lattice": "D3Q19", "psi_scheme": "FV",
                       "integrator": "Heun", "sampling": "S(q) |k_a|<=8 every 10 steps",
                       "l2": "inputs larger than L2 (populations %.1f GB)" % (2 * 19 * N * (4 if storage == 0 else 2) / 1e9),
                       "parallelism": f"replicas x{ws}", "psi_zchunk": zchunk},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": lb_traffic(storage, N),
                         "kernel": "LB collide-stream", "peak_kind": peak_kind,
                         "alg_bytes_per_site": LB_ALG_BYTES_SITE[storage], "kernel_ms": lb_ms},
            "issue_roofline": issue,
            "step_roofline": {"alg_bytes_per_site": ALG_BYTES_SITE[storage], "achieved_gbs": step_gbs,
                              "frac": step_gbs / peak, "kernel_ms_per_step": {k: v / kp for k, v in kms.items()}},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "batched_vs_plain": ens, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
