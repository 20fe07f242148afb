#!/usr/bin/env python3
"""Throughput of the SIPF-PIC step (Algorithm 4) on GB300.

Workload: the ring-shaped data at scale -- P = 1e7 particles from a Gaussian
torus (major radius 0.25 L, minor sigma 0.03 L) plus 5% uniform background,
H = 128, L = 1, M0 = 300, chi = 1, mu = 0.5, eps = k = 1, tau = 5e-5, FP32.
One step = one full pass of Algorithm 4 (F_H of the deposit, implicit update
with the filtered gradient, three inverse transforms, the particle move fused
with the deposit of the new positions).  Inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload (the method has no data-parallel exchange in this build), so
`value` is the sum over ranks and the scaling is weak.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec at P=1e7,H=128 (FP32 vs FP64 plain) + % HBM roofline; adjoint ms/step"
UNIT = "particle-steps/s"
P_FULL, H_FULL = 10_000_000, 128
# algorithmic bytes of the particle kernel per particle-step (FP32): read X (12 B) + write X (12 B)
BYTES_PER_PARTICLE = 24
# DRAM traffic (read + write bytes) of the particle phase, move + re-bin
# (299.6 MB) and deposit (133.6 MB) launches of one step, from ncu captures of
# the torus workload, keyed by the SHA-256 of the kernel sources they were
# taken on (a changed kernel reports null until it is captured again).
MOVE_TRAFFIC = {"4dcf580b08ec301d09cbd40561b51f6355c651130cf8c66b76a9069438413064": 433.24e6}
FALLBACK_HBM_GBS = 6800.0
# Warp-instructions of one move + re-bin launch (136.76 M) and one deposit
# launch (114.26 M) at P = 1e7, H = 128, FP32, from the same ncu captures,
# keyed like the traffic: the particle kernels against the SMs' issue rate.
PARTICLE_WARP_INSTR = {"4dcf580b08ec301d09cbd40561b51f6355c651130cf8c66b76a9069438413064": 251.03e6}
# FP64 form: FP64-pipe thread instructions (DFMA + DADD + DMUL) of one FP64 step
# at P = 1e7, H = 128 (move 2.580e9, deposit 0.823e9, forward plane 0.112e9,
# x pass 0.279e9, inverse plane 0.334e9), from an ncu capture of the bench's
# FP64 leg, keyed by the SHA-256 of the kernel sources it was taken on.
FP64_PIPE_INSTR = {"abbf5d2a7846741ad101791e36e02233e61004fe83b7c3ba7dfb38f2462ff404": 4.12745e9}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "measured"
    except Exception:
        return 2070.0, "nominal"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(names=("particle_kernels.cu", "sipf_device.cuh")):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2512_03452_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# ----------------------------------------------------------------- clocks
_CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(dev_index):
    path = tempfile.mktemp(prefix="sipf_clocks_", suffix=".csv")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={_CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                              "-i", str(dev_index), "-lms", "50"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f, path
    except Exception:
        return None, None, path


def clocks_stop(handle):
    p, f, path = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(path)
    except Exception:
        pass
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- oracle baseline
def oracle_rate(X_sample, w, steps):
    """Oracle (FP64 numpy, as it stands) particle-steps/s on a sample of the workload."""
    from oracle import sipf_oracle as O
    p = O.Params.from_workload(w, P=X_sample.shape[0])
    s = O.init_state(X_sample, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        s = O.step(s, p)
    dt = time.perf_counter() - t0
    return X_sample.shape[0] * steps / dt, dt


# ----------------------------------------------------------------- oracle on all host cores
# The oracle's particle loops (Algorithm 2's deposit and the particle move)
# split over a process pool by particle slices, the grid work (F_H, the
# gradient grids of alpha^(n-1), the update of alpha) on the calling process,
# in the order of the oracle's own step.  Workers are started with `spawn` and
# share X, the gradient grids and their partial deposits through shared memory.
_PW = {}


def _pw_init(names, P, H, nparts, pdict):
    from multiprocessing import shared_memory

    import numpy as np

    from oracle import sipf_oracle as O
    shm = [shared_memory.SharedMemory(name=n) for n in names]
    _PW.update(shm=shm, O=O, p=O.Params(**pdict),
               X=np.ndarray((P, 3), dtype=np.float64, buffer=shm[0].buf),
               grads=np.ndarray((3, H, H, H), dtype=np.float64, buffer=shm[1].buf),
               parts=np.ndarray((nparts, H ** 3), dtype=np.float64, buffer=shm[2].buf))


def _pw_deposit(task):
    k, a, b = task
    O, p = _PW["O"], _PW["p"]
    _PW["parts"][k] = O.deposit(_PW["X"][a:b], p.mass / p.P, p.H, p.L, p.p2g_order).ravel()


def _pw_move(task):
    a, b, n = task
    O, p = _PW["O"], _PW["p"]
    _PW["X"][a:b] = O.move(_PW["X"][a:b], _PW["grads"], p, n, first=a)


class ParallelOracle:
    """Steps of the FP64 oracle with its particle loops on `workers` processes."""

    def __init__(self, X0, p, workers):
        import dataclasses
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        from oracle import sipf_oracle as O
        self.O, self.p = O, p
        P, H = X0.shape[0], p.H
        self.workers = max(1, int(workers))
        self.nparts = min(self.workers * 2, max(1, P // 1000))
        sizes = [P * 3 * 8, 3 * H ** 3 * 8, self.nparts * H ** 3 * 8]
        self.shm = [shared_memory.SharedMemory(create=True, size=sz) for sz in sizes]
        self.X = np.ndarray((P, 3), dtype=np.float64, buffer=self.shm[0].buf)
        self.grads = np.ndarray((3, H, H, H), dtype=np.float64, buffer=self.shm[1].buf)
        self.parts = np.ndarray((self.nparts, H ** 3), dtype=np.float64, buffer=self.shm[2].buf)
        self.X[:] = X0
        self.alpha = np.zeros((H, H, H // 2 + 1), dtype=np.complex128)
        self.n = 0
        edges = np.linspace(0, P, self.nparts + 1).astype(np.int64)
        self.slices = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]
        self.pool = mp.get_context("spawn").Pool(
            self.workers, initializer=_pw_init,
            initargs=([m.name for m in self.shm], P, H, self.nparts, dataclasses.asdict(p)))
        self.t_particles = self.t_grid = 0.0

    def step(self):
        O, p = self.O, self.p
        n = self.n + 1
        t0 = time.perf_counter()
        self.pool.map(_pw_deposit, [(k, a, b) for k, (a, b) in enumerate(self.slices)])
        t1 = time.perf_counter()
        phi = self.parts.sum(axis=0).reshape(p.H, p.H, p.H)
        beta = O.forward_ft(phi, p.L)
        self.grads[:] = O.gradient_grids(self.alpha, p)           # grad c^(n-1) from alpha^(n-1)
        if p.propagator == "exp":
            self.alpha = O.update_alpha_exp(self.alpha, beta, p)
        else:
            self.alpha = O.update_alpha(self.alpha, beta, p)
        t2 = time.perf_counter()
        self.pool.map(_pw_move, [(a, b, n) for a, b in self.slices])
        t3 = time.perf_counter()
        self.t_particles += (t1 - t0) + (t3 - t2)
        self.t_grid += t2 - t1
        self.n = n

    def close(self):
        self.pool.close()
        self.pool.join()
        del self.X, self.grads, self.parts
        for m in self.shm:
            m.close()
            m.unlink()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def oracle_rate_parallel(X_sample, w, steps, workers=None, warmup=1):
    """All-core oracle particle-steps/s on a sample of the workload; also the
    share of the step spent in the grid work (F_H, gradient grids, update)."""
    from oracle import sipf_oracle as O
    workers = workers or os.cpu_count() or 1
    p = O.Params.from_workload(w, P=X_sample.shape[0])
    with ParallelOracle(X_sample, p, workers) as po:
        for _ in range(warmup):
            po.step()
        po.t_particles = po.t_grid = 0.0
        t0 = time.perf_counter()
        for _ in range(steps):
            po.step()
        dt = time.perf_counter() - t0
        grid_share = po.t_grid / max(po.t_particles + po.t_grid, 1e-30)
    return X_sample.shape[0] * steps / dt, dt, grid_share, workers


def cpu_baselines(X0, w):
    """The oracle on this host: the benchmark workload on all cores (particle
    loops over a process pool) and a sample on one core, plus the other
    workloads (the oracle-sized blob in full, the blow-up blob for 20 steps)."""
    import numpy as np

    from paper_2512_03452_gb300 import workloads
    cores = os.cpu_count() or 1
    rate, dt, share, _ = oracle_rate_parallel(np.asarray(X0, dtype=np.float64), w, 3, workers=cores)
    ns = 200_000
    r1, dt1 = oracle_rate(np.asarray(X0[:ns], dtype=np.float64), w, 2)
    wb = workloads.small_blob()
    rc1, dtc1 = oracle_rate(workloads.sample_positions(wb), wb, wb.steps)
    wc2 = workloads.blowup_blob()
    rc2, dtc2, sh2, _ = oracle_rate_parallel(workloads.sample_positions(wc2), wc2, 20, workers=cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the full benchmark workload ({w.P} particles, H={w.H}), 3 steps after 1 warm-up step "
                      f"({dt:.1f} s, numpy FP64, particle loops over {cores} processes)",
            "grid_share": share,
            "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                            "sample": f"first {ns} particles of the same sample, H={w.H}, 2 steps ({dt1:.1f} s)"},
            "configs": {
                wb.name: {"value": rc1, "unit": UNIT, "cores": 1, "s_per_step": dtc1 / wb.steps,
                          "sample": f"all {wb.P} particles, all {wb.steps} steps"},
                wc2.name: {"value": rc2, "unit": UNIT, "cores": cores, "s_per_step": dtc2 / 20, "grid_share": sh2,
                           "sample": f"all {wc2.P} particles, 20 steps after 1 warm-up step"}}}


# ----------------------------------------------------------------- distributed
def dist_init(args):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def dist_max(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ----------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2512_03452_gb300 import Simulation, _abi, build, params_from_workload, workloads

    build.build()
    _abi.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads.torus_ring(H=H_FULL, P=P_FULL)
    X0 = workloads.sample_positions(w, seed=w.seed + rank)
    stream = torch.cuda.Stream(device=dev)
    K, W = args.steps, args.warmup

    sim = Simulation(params_from_workload(w, precision=32), X0, stream=stream.cuda_stream)
    sim.step(W)
    sim.sync()
    dist_barrier(world, dev)
    torch.cuda.synchronize()
    clk = clocks_start(local)
    time.sleep(0.2)
    # the headline steps run without the per-stage events (7 event records
    # and an overflow counter per step); launches counted by the library
    l0 = _abi.sipf_kernel_launches(sim.ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
    e1.synchronize()
    dist_barrier(world, dev)
    torch.cuda.synchronize()
    clocks = clocks_stop(clk)
    ms = e0.elapsed_time(e1)
    launches = _abi.sipf_kernel_launches(sim.ctx) - l0
    sim.sync()
    # the stage breakdown from a separate pass with the per-stage events on
    _abi.sipf_timing_enable(sim.ctx, 1)
    sim.step(max(1, min(K, 100)))
    tim = _abi.sipf_timing_read(sim.ctx)
    _abi.sipf_timing_enable(sim.ctx, 0)
    sim.sync()
    diag = sim.diagnostics()
    ms_max = dist_max(ms, world, dev)
    value = world * P_FULL * K / (ms_max * 1e-3)

    # roofline of the dominant work: the particle phase (move + re-bin kernel and
    # deposit kernel), against the algorithmic 24 B per particle-step
    peak, peak_kind = measured_peaks()
    move_ms = tim.move_ms / max(tim.steps, 1)
    dep_ms = tim.deposit_ms / max(tim.steps, 1)
    part_ms = move_ms + dep_ms
    achieved = BYTES_PER_PARTICLE * P_FULL / (part_ms * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    traffic = MOVE_TRAFFIC.get(src_hash)
    # figures captured on other kernel sources are reported, marked stale,
    # but never used as this build's traffic
    stale = None
    if traffic is None or PARTICLE_WARP_INSTR.get(src_hash) is None:
        stale = {"traffic": list(MOVE_TRAFFIC.values())[-1] if MOVE_TRAFFIC else None,
                 "warp_instructions": list(PARTICLE_WARP_INSTR.values())[-1] if PARTICLE_WARP_INSTR else None,
                 "note": "ncu counters of an earlier build of the particle kernels (sources changed since); "
                         "not this build's figures"}
    # the same kernels against the SMs' instruction issue rate (4 warp-
    # instructions per clock per SM), the bound they actually meet
    n_issue = PARTICLE_WARP_INSTR.get(src_hash)
    issue = None
    if n_issue is not None:
        mhz, mhz_kind = sm_max_mhz()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        pk = 4.0 * sms * mhz * 1e6
        ach = n_issue / (part_ms * 1e-3)
        issue = {"bound": "issue", "unit": "warp-instructions/s", "achieved": ach, "peak": pk, "frac": ach / pk,
                 "instructions_per_step": n_issue,
                 "peak_source": f"4 per clock x {sms} SMs x {mhz:.0f} MHz ({mhz_kind} maximum SM clock)"}
    stages = {k: getattr(tim, k) / max(tim.steps, 1) for k in
              ("forward_ms", "spectral_ms", "inverse_ms", "move_ms", "bookkeeping_ms", "deposit_ms")}

    # FP64 plain path on the same workload
    K64, W64 = max(1, min(K, 20)), min(W, 3)
    sim64 = Simulation(params_from_workload(w, precision=64), X0, stream=stream.cuda_stream)
    sim64.step(W64)
    sim64.sync()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        f0.record(stream)
        sim64.step(K64)
        f1.record(stream)
    f1.synchronize()
    ms64 = dist_max(f0.elapsed_time(f1), world, dev)
    sim64.sync()
    sim64.close()
    # the FP64 form is bound by the FP64 pipe: its instruction rate against
    # this GPU's measured FP64 FMA issue rate
    fma_gflops = _abi.sipf_measure_fp64_fma(stream.cuda_stream)
    n64 = FP64_PIPE_INSTR.get(kernel_source_hash(("particle_kernels.cu", "sipf_device.cuh", "fft_kernels.cu")))
    fp64_alu = None
    if n64 is not None:
        ach = n64 / (ms64 / K64 * 1e-3)
        pk = fma_gflops * 1e9 / 2.0
        fp64_alu = {"bound": "alu", "unit": "FP64 instructions/s", "achieved": ach, "peak": pk, "frac": ach / pk,
                    "instructions_per_step": n64,
                    "peak_source": "measured: sipf_measure_fp64_fma (dependent-chain FP64 FMAs over all SMs)"}

    # end to end through the C ABI with host buffers: every step uploads the
    # positions from pinned host memory, steps, and reads them back.  The host
    # copy starts from the context's own positions, so the loop continues its
    # trajectory (re-sending X0 would hand the bins, sized for the evolved
    # distribution, particles they no longer fit until the next capacity
    # rebuild)
    Ke = max(1, min(K, 20))
    hx = [torch.empty(P_FULL, dtype=torch.float32).pin_memory() for _ in range(3)]
    ptrs = [t.data_ptr() for t in hx]
    _abi.sipf_download_soa(sim.ctx, *ptrs)
    sim.sync()
    for _ in range(2):
        _abi.sipf_upload_soa(sim.ctx, *ptrs)
        sim.step(1)
        _abi.sipf_download_soa(sim.ctx, *ptrs)
    sim.sync()
    dist_barrier(world, dev)
    t0 = time.perf_counter()
    for _ in range(Ke):
        _abi.sipf_upload_soa(sim.ctx, *ptrs)
        sim.step(1)
        _abi.sipf_download_soa(sim.ctx, *ptrs)
        sim.sync()
    te = time.perf_counter() - t0
    te_max = dist_max(te, world, dev)
    sim.close()
    e2e = {"value": world * P_FULL * Ke / te_max, "unit": UNIT, "h2d_bytes_per_step": 12 * P_FULL,
           "d2h_bytes_per_step": 12 * P_FULL, "steps": Ke,
           "path": "sipf_upload_soa + sipf_step + sipf_download_soa, pinned host SoA float32"}

    extra = None if args.no_extra else run_extra_legs(world, dev, stream, X0)
    batch = None if args.no_batch else run_batch_leg(world, dev, stream)
    adjoint = None if args.no_adjoint else run_adjoint_leg(world, dev, stream)
    convergence = None if args.no_convergence else run_convergence_leg(full=args.study)
    two_d = None if args.no_2d else run_2d_leg(world, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(X0, w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "P": P_FULL, "H": H_FULL, "L": w.L, "M0": w.mass, "chi": w.chi,
                       "mu": w.mu, "eps": w.eps, "k": w.k, "tau": w.dt, "precision": "fp32",
                       "l2": "inputs larger than L2 (per step 2 x 16 B x 1e7 particle traffic + 76 MB of grids)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": "particle phase: k_move (move + re-bin) and k_binned (deposit)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_source": peak_kind, "bytes_per_particle": BYTES_PER_PARTICLE,
                         "kernel_ms": part_ms, "overflow_per_step": tim.overflow / max(tim.steps, 1),
                         "issue": issue, "stale_counters": stale},
            "stages_ms_per_step": stages,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "fp64": {"value": world * P_FULL * K64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / K64,
                     "steps": K64, "fma_gflops": fma_gflops, "roofline": fp64_alu},
            "diagnostics": {k: diag[k] for k in ("mass", "peak", "m2", "ring_radius", "step")},
            "batch": batch,
            "adjoint": adjoint,
            "convergence": convergence,
            "two_d": two_d,
            "sweep": extra,
        }
        print(json.dumps(line), flush=True)


def run_extra_legs(world, dev, stream, X0_128, steps=50, warmup=5):
    """The ring workload at H = 64 and 256 (same particles), the deterministic
    deposit at H = 128, cuFFT (torch.fft) doing the field solve's transforms
    at H = 128 for comparison, and this GPU's FP64 FMA rate (the FP64 form's
    arithmetic bound)."""
    import torch

    from paper_2512_03452_gb300 import Simulation, _abi, params_from_workload, workloads

    out = {}

    def timed_sim(w, steps, **kw):
        sim = Simulation(params_from_workload(w, **kw), X0_128, stream=stream.cuda_stream)
        sim.step(warmup)
        sim.sync()
        _abi.sipf_timing_enable(sim.ctx, 1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            sim.step(steps)
            b.record(stream)
        b.synchronize()
        ms = dist_max(a.elapsed_time(b), world, dev)
        t = _abi.sipf_timing_read(sim.ctx)
        sim.close()
        stages = {k: getattr(t, k) / max(t.steps, 1) for k in
                  ("forward_ms", "spectral_ms", "inverse_ms", "move_ms", "bookkeeping_ms", "deposit_ms")}
        return {"value": world * w.P * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                "steps": steps, "stages_ms_per_step": stages}

    for H in (64, 256):
        out[f"H{H}"] = timed_sim(workloads.torus_ring(H=H, P=P_FULL), steps, precision=32)
    out["H128_deterministic_deposit"] = timed_sim(workloads.torus_ring(H=H_FULL, P=P_FULL), steps, precision=32,
                                                  deposit_mode=1)
    # cuFFT via torch.fft: r2c of the deposit, and three c2r of gradient spectra
    H = H_FULL
    g = torch.randn((H, H, H), device=dev, dtype=torch.float32)
    G = torch.fft.rfftn(g)
    G3 = torch.stack([G, G, G])
    for _ in range(3):
        torch.fft.rfftn(g)
        torch.fft.irfftn(G3, s=(H, H, H))
    reps = 50
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        torch.fft.rfftn(g)
        torch.fft.irfftn(G3, s=(H, H, H))
    b.record()
    b.synchronize()
    out["cufft_H128_ms"] = {"forward_plus_3_inverse": a.elapsed_time(b) / reps,
                            "note": "torch.fft (cuFFT): rfftn of one H^3 grid + irfftn of three spectra, "
                                    "transforms only (no spectral update, no filter, no interleaved output)"}
    out["fp64_fma_gflops"] = _abi.sipf_measure_fp64_fma(stream.cuda_stream)
    return out


def run_batch_leg(world, dev, stream, n_runs=256, steps=64, warmup=32):
    """The batched form on an ensemble of uneven runs (P log-uniform in
    [1e4, 1e6], H in {32, 64}, FP32): replayed 32-step graphs, the same steps
    issued directly, and the same runs as separate single-run contexts stepped
    one after another."""
    import numpy as np
    import torch

    from paper_2512_03452_gb300 import Batch, Simulation, _abi, params_from_workload, workloads

    ws = workloads.ensemble(n_runs)
    params = [params_from_workload(w, precision=32) for w in ws]
    X0s = [workloads.sample_positions(w) for w in ws]
    total_p = sum(w.P for w in ws)

    def timed(fn, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            fn(k)
            b.record(stream)
        b.synchronize()
        return dist_max(a.elapsed_time(b), world, dev)

    out = {"workload": f"ensemble of {n_runs} runs, P log-uniform 1e4..1e6, H in {{32, 64}}, FP32",
           "runs": n_runs, "particles": total_p, "steps": steps, "unit": UNIT}
    with Batch(params, X0s, stream=stream.cuda_stream) as b:
        b.step(warmup)
        b.sync()
        out["autotune"] = b.autotune(3)
        k0 = _abi.sipf_batch_kernel_launches(b.handle)
        ms = timed(b.step, steps)
        out["gpu_launches_per_step"] = (_abi.sipf_batch_kernel_launches(b.handle) - k0) / steps
        b.use_graph(False)
        ms_direct = timed(b.step, steps)
        b.sync()
    out["value"] = world * total_p * steps / (ms * 1e-3)
    out["ms_per_step"] = ms / steps
    out["direct_issue_ms_per_step"] = ms_direct / steps
    sims = [Simulation(p, X, stream=stream.cuda_stream) for p, X in zip(params, X0s)]
    try:
        def seq(k):
            for _ in range(k):
                for sim in sims:
                    sim.step(1)
        seq(2)
        torch.cuda.synchronize()
        ms_seq = timed(seq, steps // 4)
    finally:
        for sim in sims:
            sim.close()
    out["sequential_single_runs_ms_per_step"] = ms_seq / (steps // 4)
    out["speedup_vs_sequential"] = out["sequential_single_runs_ms_per_step"] / out["ms_per_step"]
    return out


def run_adjoint_leg(world, dev, stream, nsteps=200, checkpoint=20, reps=2):
    """The adjoint form on its workload: P = 1e6, H = 64, FP32 forward, N = 200
    steps, checkpoints every 20; loss J = sum_j (rho_j(T) - rho*_j)^2 in FP64
    with rho* from a chi = 1.3 run with the same X0 and noise.  Device time of
    the forward (with checkpoints) and of the reverse sweep (segment
    recomputation included), per step."""
    import numpy as np

    from paper_2512_03452_gb300 import _abi, params_from_workload, workloads
    from paper_2512_03452_gb300.adjoint import Adjoint

    w = workloads.adjoint_case()
    X0 = workloads.sample_positions(w)
    p = params_from_workload(w, precision=32)
    with Adjoint(p, X0, nsteps, checkpoint, stream=stream.cuda_stream) as eng:
        rho_star = eng.forward(1.3, w.mu)
        fwd, bwd = [], []
        for _ in range(reps + 1):
            rho = eng.forward(w.chi, w.mu)
            gc, gm, gX = eng.backward(2.0 * (rho - rho_star))
            f, b = eng.timing()
            fwd.append(f)
            bwd.append(b)
        launches = _abi.sipf_adjoint_kernel_launches(eng.handle)
    f, b = dist_max(min(fwd[1:]), world, dev), dist_max(min(bwd[1:]), world, dev)
    J = float(np.sum((rho - rho_star) ** 2))
    return {"workload": f"{w.name}, N={nsteps}, checkpoint every {checkpoint}, FP32 forward, FP64 loss",
            "adjoint_ms_per_step": (f + b) / nsteps, "forward_ms_per_step": f / nsteps,
            "backward_ms_per_step": b / nsteps, "backward_over_forward": b / f,
            "loss": J, "dJ_dchi": gc, "dJ_dmu": gm, "dJ_dX0_max": float(np.max(np.abs(gX))),
            "gpu_launches_total": launches}


def run_convergence_leg(full=False):
    """The Sec. 5.1 convergence study on this GPU: the uniform-ball set-up
    (FP32, 2000 steps to T = 0.02) against the stored radial finite-volume
    reference (tests/golden/sec51_reference_quantiles.json, written from the
    oracle); E = the truncated quantile W1 averaged over seeds; slopes of
    log2 E against log2 P (H fixed) and log2 H (P fixed), beside the paper's.
    Default: 8 seeds, P = 2^11..2^19 at H = 128 and H = 16..128 at P = 2^19;
    full: the paper's sweep, 30 seeds, P = 2^11..2^20 at H = 256 and
    H = 8..256 at P = 2^20."""
    import numpy as np

    from paper_2512_03452_gb300 import convergence as C

    with open(os.path.join(ROOT, "tests", "golden", "sec51_reference_quantiles.json")) as f:
        gold = json.load(f)
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")) as f:
        paper = json.load(f)["convergence_slopes"]
    levels, q_ref = np.array(gold["levels"]), np.array(gold["quantiles"])
    if full:
        seeds, Hfix, Pfix = range(30), 256, 2 ** 20
        Ps, Hs = [2 ** e for e in range(11, 21)], [8, 16, 32, 64, 128, 256]
    else:
        seeds, Hfix, Pfix = range(8), 128, 2 ** 19
        Ps, Hs = [2 ** e for e in range(11, 20, 2)], [16, 32, 64, 128]
    cells, t0, psteps = {}, time.perf_counter(), 0

    def cell(P, H):
        nonlocal psteps
        if (P, H) not in cells:
            errs = [float(np.mean(np.abs(C.radial_quantiles(r, levels) - q_ref))) for r in C.final_radii(P, H, seeds)]
            cells[(P, H)] = {"P": P, "H": H, "E_mean": float(np.mean(errs)), "E_std": float(np.std(errs)),
                             "runs_below_2x_mean": float(np.mean(np.array(errs) < 2 * np.mean(errs)))}
            psteps += P * 2000 * len(seeds)
        return cells[(P, H)]["E_mean"]

    EP = [cell(P, Hfix) for P in Ps]
    EH = [cell(Pfix, H) for H in Hs]
    dt = time.perf_counter() - t0
    return {"workload": "Sec. 5.1 uniform ball (M0 = 80, L = 8, eps = 1e-4, k = 0.1, tau = 1e-5, 2000 steps), FP32",
            "seeds": len(seeds), "slope_P": C.fitted_slope(Ps, EP), "slope_P_at_H": Hfix,
            "slope_H": C.fitted_slope(Hs, EH), "slope_H_at_P": Pfix, "paper_slopes": {"P": paper["P"], "H": paper["H"]},
            "cells": list(cells.values()), "seconds": dt, "particle_steps_per_s": psteps / dt}


def run_2d_leg(world, dev, stream):
    """The 2D parabolic-elliptic variant (Sec. 5.2) on this GPU: device time of
    the step at P = 2^20, H = 256, L = 10 (FP32, unit disk, M0 = 25), and the
    second-moment experiment -- unit disk, (k, eps, mu, chi) = (0, 0, 1, 1),
    tau = 5e-4 to T = 2 (4000 steps), P = 2^20, H = 256 -- at masses around
    8 pi and box sides 10 and 20, beside the whole-plane value
    m2(2) = 17/2 - M0/pi."""
    import numpy as np
    import torch

    from paper_2512_03452_gb300 import Simulation2D, make_params

    def disk(P, seed):
        rng = np.random.default_rng(seed)
        r = np.sqrt(rng.uniform(size=P))
        th = rng.uniform(0, 2 * math.pi, size=P)
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)

    P = 2 ** 20
    X0 = disk(P, 0)

    def params(L, M0):
        return make_params(P=P, H=256, L=L, mass=M0, chi=1.0, mu=1.0, eps=0.0, k=0.0, dt=5e-4, seed=1, precision=32)

    out = {"workload": "2D parabolic-elliptic (Sec. 5.2): unit disk, P = 2^20, H = 256, tau = 5e-4, FP32"}
    with Simulation2D(params(10.0, 25.0), X0, stream=stream.cuda_stream) as sim:
        sim.step(20)
        sim.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            sim.step(200)
            b.record(stream)
        b.synchronize()
        ms = dist_max(a.elapsed_time(b), world, dev) / 200
    out["ms_per_step"] = ms
    out["value"] = world * P / (ms * 1e-3)
    out["unit"] = UNIT
    rows = []
    for L in (10.0, 20.0):
        for M0 in (24.6, 25.0, 25.6):
            with Simulation2D(params(L, M0), X0, stream=stream.cuda_stream) as sim:
                sim.step(4000)
                d = sim.diagnostics()
            rows.append({"L": L, "h": L / 256, "M0": M0, "m2_T2": d["m2"], "closed_form": 8.5 - M0 / math.pi,
                         "peak": d["peak"], "hf_frac": d["hf_frac"]})
    out["second_moment"] = rows
    return out


# ----------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    from oracle import sipf_oracle as O
    from paper_2512_03452_gb300 import workloads

    w = workloads.torus_ring(H=H_FULL, P=P_FULL)
    ns = 1_000_000
    X = workloads.sample_positions(w)[:ns]
    p = O.Params.from_workload(w, P=ns)
    cores = os.cpu_count() or 1
    with ParallelOracle(X, p, cores) as po:
        for _ in range(args.warmup):
            po.step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            po.step()
        dt = time.perf_counter() - t0
    value = ns * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "P": P_FULL, "H": H_FULL, "precision": "fp64 oracle",
                       "parallelism": "host"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the first {ns} particles of the torus workload per step, H=128 "
                                       f"(numpy FP64, particle loops over {cores} processes)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch_case(args):
    """A small batch for kernel captures: 128 runs at H = 64 with 1e4 particles
    each (Gaussian blobs), `warmup` directly issued steps, then `steps` timed
    ones; prints the device ms per step.  Not a benchmark line."""
    import torch

    from paper_2512_03452_gb300 import Batch, _abi, build, params_from_workload, workloads

    build.build()
    _abi.load()
    ws = [workloads.Workload(f"r{i}", P=10_000, H=64, L=1.0, mass=50.0, chi=1.0, dt=1e-4, steps=100, seed=i,
                             sigma=0.1) for i in range(128)]
    params = [params_from_workload(w, precision=32) for w in ws]
    X0s = [workloads.sample_positions(w) for w in ws]
    stream = torch.cuda.Stream()
    with Batch(params, X0s, stream=stream.cuda_stream) as b:
        b.use_graph(False)
        b.step(args.warmup)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        print(json.dumps({"case": "batch of 128 runs, H=64, P=1e4 each, FP32",
                          "ms_per_step": e0.elapsed_time(e1) / max(args.steps, 1)}), flush=True)


def run_field_case(args):
    """One grid size's field solve for kernel captures: the ring workload with
    1e6 particles at H = args.field_case (the field kernels do not depend on
    P), `warmup` steps, then `steps` steps with the per-stage events; prints
    the stage times.  Not a benchmark line."""
    import torch

    from paper_2512_03452_gb300 import Simulation, _abi, build, params_from_workload, workloads

    build.build()
    _abi.load()
    w = workloads.torus_ring(H=args.field_case, P=1_000_000)
    stream = torch.cuda.Stream()
    with Simulation(params_from_workload(w, precision=32), workloads.sample_positions(w),
                    stream=stream.cuda_stream) as sim:
        sim.step(args.warmup)
        sim.sync()
        _abi.sipf_timing_enable(sim.ctx, 1)
        sim.step(args.steps)
        t = _abi.sipf_timing_read(sim.ctx)
    n = max(t.steps, 1)
    print(json.dumps({"case": f"field solve, ring workload, H={args.field_case}, P=1e6, FP32",
                      **{k: getattr(t, k) / n for k in ("forward_ms", "spectral_ms", "inverse_ms")}}), flush=True)


def run_adjoint_case():
    """Only the adjoint leg (for kernel captures); prints its JSON object."""
    import torch

    from paper_2512_03452_gb300 import _abi, build

    build.build()
    _abi.load()
    dev = torch.device("cuda", 0)
    print(json.dumps(run_adjoint_leg(1, dev, torch.cuda.Stream(device=dev))), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--no-convergence", action="store_true", help="skip the Sec. 5.1 convergence-study leg")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2D parabolic-elliptic leg (Sec. 5.2)")
    ap.add_argument("--study", action="store_true",
                    help="run the convergence leg over the paper's full sweep (30 seeds, P up to 2^20, H up to 256)")
    ap.add_argument("--no-extra", action="store_true", help="skip the H sweep, deterministic, cuFFT and FP64 legs")
    ap.add_argument("--batch-case", action="store_true",
                    help="only run a small 128-run H = 64 batch (for kernel captures) and print its ms per step")
    ap.add_argument("--adjoint-case", action="store_true", help="only run the adjoint leg (for kernel captures)")
    ap.add_argument("--field-case", type=int, choices=[32, 64, 128, 256], default=0,
                    help="only run a few steps at this H with stage timing (field-solve kernel captures)")
    args = ap.parse_args()
    if args.field_case:
        run_field_case(args)
        return
    if args.batch_case:
        run_batch_case(args)
        return
    if args.adjoint_case:
        run_adjoint_case()
        return
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
