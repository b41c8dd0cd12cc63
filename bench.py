#!/usr/bin/env python3
"""Benchmark: Fock(J+K) builds/s of the closed-shell HF two-electron hot path.

Workload: the 40-atom s+p lattice molecule (seed 1; nbf 220; hydrogen 2 s
shells, C/O 3 s + 2 p shells, 3 primitives, exponents log-uniform in
[0.05, 50]; charges from {1, 6, 8}), at its converged RHF density, Schwarz
tau = 1e-12, plain FP64.  One step = one hf_fock_jk call (all ERI classes
with the fused J/K digestion, then the symmetrisation), with the density
resident in HBM.  L2 is flushed (256 MiB write) between timed steps; each
step is timed with CUDA events on the library's stream.

--impl reference times the CPU oracle (plain C, McMurchie-Davidson) on a
bounded random sample of the same unique surviving shell quartets per step
and scales to builds/s.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(natom=40, seed=1, rules="sp", tau=1e-12)
METRIC = "Fock(J+K) builds/s"
UNIT = "builds/s"


def workload_desc(nbf):
    return {"workload": f"40-atom s+p lattice molecule (seed 1), nbf {nbf}, converged RHF density, "
                        f"Schwarz tau 1e-12, FP64 hf_fock_jk",
            "natom": WORKLOAD["natom"], "nbf": nbf, "basis_rules": "H 2s; C/O 3s2p; K=3; exp logU[0.05,50]",
            "schwarz_tau": WORKLOAD["tau"], "precision": "fp64",
            "l2": "flushed between timed steps (256 MiB write)"}


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock / throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- peaks
def fp64_alu_peak(sm_count: int, clock_mhz: float):
    """Nominal FP64 CUDA-core peak of GB300: 2 FP64 FMA per SM per clock."""
    return sm_count * 4 * clock_mhz * 1e6 / 1e12   # TFLOP/s


def kernel_hash():
    h = hashlib.sha256()
    for f in ("eri.cuh", "eri_classes.cuh", "hf_device.h"):
        with open(os.path.join(ROOT, "paper_1303_4916_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name: str):
    """DRAM bytes per launch of the named kernel from the committed ncu summary,
    when it was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "eri_jk_c2_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for ln in open(p):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_hash") != kernel_hash() or kv.get("class") != kernel_name:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- oracle sample
def oracle_sample_rate(mol, tau, seconds_target=15.0, seed=0):
    """Oracle time per unique surviving quartet on a random sample; returns
    (builds_per_s, n_sample, n_total, seconds)."""
    import oracle
    ob = oracle.Basis(mol)
    Q = ob.schwarz()
    ns = mol.nshell
    n_total = ob.count_quartets(tau)
    rng = np.random.default_rng(seed)
    pairs = np.array([(a, b) for a in range(ns) for b in range(a + 1)], dtype=np.int64)
    D = np.eye(ob.nbf) * 0.1

    def draw(n):
        out = []
        while len(out) < n:
            i, j = rng.integers(0, len(pairs), size=2)
            if j > i:
                i, j = j, i
            (a, b), (c, d) = pairs[i], pairs[j]
            if Q[a, b] * Q[c, d] < tau:
                continue
            out.append((a, b, c, d))
        return np.array(out, dtype=np.int32)

    # calibrate on a small batch, then size the sample for ~seconds_target
    q = draw(200)
    t0 = time.perf_counter()
    ob.jk_quartets(D, q)
    per = (time.perf_counter() - t0) / len(q)
    n = int(max(200, min(2_000_000, seconds_target / max(per, 1e-9))))
    q = draw(n)
    t0 = time.perf_counter()
    ob.jk_quartets(D, q)
    dt = time.perf_counter() - t0
    per = dt / n
    return 1.0 / (per * n_total), n, n_total, dt


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from synth import lattice_molecule
    import oracle
    mol = lattice_molecule(WORKLOAD["natom"], WORKLOAD["seed"], WORKLOAD["rules"])
    per_step = max(1.0, 30.0 / max(1, args.steps + args.warmup))
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        v, n, tot, dt = oracle_sample_rate(mol, WORKLOAD["tau"], seconds_target=per_step, seed=k)
        if k >= args.warmup:
            vals.append(v)
            info = (n, tot, dt)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(mol.nbf),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{info[0]} random unique surviving shell quartets of {info[1]} per step "
                                       f"({info[2]:.1f} s), scaled to one full build"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, world, local = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_1303_4916_gb300 as hf
    from synth import lattice_molecule

    mol = lattice_molecule(WORKLOAD["natom"], WORKLOAD["seed"], WORKLOAD["rules"])
    ctx = hf.Context(local)
    basis = hf.Basis(ctx, mol)
    n = basis.nbf
    stream = torch.cuda.current_stream(local)
    dev = torch.device("cuda", local)

    # converged density (setup, untimed); its wall time is the single-molecule SCF latency
    t0 = time.perf_counter()
    scf = basis.scf(max_iter=128, e_tol=1e-8, diis_size=8, schwarz_tau=WORKLOAD["tau"])
    scf_latency = time.perf_counter() - t0
    D = scf.tensors["D"].contiguous()
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    opts = hf.jk_opts(schwarz_tau=WORKLOAD["tau"])
    stats = basis.class_stats(opts)
    nq_total = sum(s.quartets_fp64 + s.quartets_fp32 for s in stats)
    launches_per_step = sum((s.quartets_fp64 > 0) + (s.quartets_fp32 > 0) for s in stats) + 1
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        basis.fock_jk(D, J, K, opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        basis.fock_jk(D, J, K, opts)
        ends[k].record(stream)
    torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1000.0
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
        dist.barrier()

    # per-class kernel durations (CUDA events on the library stream), averaged
    prof = []
    for k in range(max(3, min(args.steps, 10))):
        flush.zero_()
        prof.append(basis.fock_jk_profiled(D, J, K, opts))
    clk = clocks.stop()
    prof = np.mean(np.array(prof), axis=0)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Dh = D.cpu().pin_memory()
    Jh = torch.empty_like(Dh).pin_memory()
    Kh = torch.empty_like(Dh).pin_memory()
    hopts = hf.jk_opts(schwarz_tau=WORKLOAD["tau"], host=True)
    for _ in range(2):
        basis.fock_jk_host(Dh.data_ptr(), Jh.data_ptr(), Kh.data_ptr(), hopts)
    e2e_t = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        basis.fock_jk_host(Dh.data_ptr(), Jh.data_ptr(), Kh.data_ptr(), hopts)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = world * len(e2e_t) / sum(e2e_t)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline: the dominant class kernel
    flops = []
    for c, s in enumerate(stats):
        f64 = s.prim_quartets_fp64 * s.prim_flops + s.quartets_fp64 * (s.hrr_flops + s.digest_flops)
        flops.append(f64)
    dom = int(np.argmax(prof[:, 0]))
    s = stats[dom]
    dom_ms = float(prof[dom, 0])
    achieved = flops[dom] / (dom_ms * 1e-3) / 1e12
    sm_count = ctx.num_sms
    peak = fp64_alu_peak(sm_count, 2070.0)
    cls_name = f"({'spd'[s.la]}{'spd'[s.lb]}|{'spd'[s.lc]}{'spd'[s.ld]})"
    traffic = ncu_traffic(cls_name)
    all_ms = float(prof[:, 0].sum() + prof[:, 1].sum())
    all_flops = sum(flops)

    value = world * args.steps / total_s
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, nsmp, ntot, dt = oracle_sample_rate(mol, WORKLOAD["tau"], seconds_target=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nsmp} random unique surviving shell quartets of {ntot} ({dt:.1f} s single-thread), "
                         f"scaled to one full build"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(n), parallelism=("replicas" if world > 1 else "single-gpu")),
        "eri_quartets_per_s": value * nq_total,
        "quartets_per_build": nq_total,
        "scf": {"latency_s": scf_latency, "iterations": scf.iterations, "converged": scf.converged,
                "energy": scf.energy, "fock_builds": scf.fock_builds},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"eri_jk_kernel {cls_name} fp64",
                     "kernel_ms": dom_ms, "kernel_flops": flops[dom],
                     "peak_note": "FP64 CUDA-core nominal: 152 SM x 2 DFMA/clk x 2.07 GHz",
                     "all_classes_tflops": all_flops / (all_ms * 1e-3) / 1e12},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * n * 8,
                "d2h_bytes_per_step": 2 * n * n * 8},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
