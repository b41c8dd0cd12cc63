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
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, max clock, max power and the throttle reasons seen
        Active in nvidia-smi CSV lines (the query order of Q, no header)."""
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
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


def fp32_alu_peak(sm_count: int, clock_mhz: float):
    """Nominal FP32 lane-operation rate of GB300: 128 FP32 lanes per SM, one
    FADD / FMUL / FFMA each per clock (T operations/s)."""
    return sm_count * 128 * clock_mhz * 1e6 / 1e12


# FP32 operations of one double-float operation, counted in df64.cuh:
# sum 11 (two-sum + renormalisation), product 7, product by a float 6,
# fused multiply-add 15, 1/sqrt 25 (estimate + one Newton step)
DF_ADD, DF_MUL, DF_FMA, DF_RSQRT = 11, 7, 15, 25


def df64_ops_per_prim_quartet(la, lb, lc, ld, vrr_flops):
    """FP32 operations per primitive quartet of the df64 thread-per-quartet
    kernel of class (la lb|lc ld): set-up (p+q, 1/sqrt, 1/(p+q), rho/zeta and
    rho/eta where used, PQ, WP and WQ where used, T, prefactor, scaling of the
    L+1 B_m), the df64 Boys evaluation (row index and x 13; Horner of F_L 79;
    for L >= 1 the exp series 79, its product 7, 2T 2 and L downward steps of
    25) and the VRR, whose generated multiply-adds run as fused df64 steps
    (15 FP32 operations per two counted flops)."""
    L = la + lb + lc + ld
    bra, ket = la + lb > 0, lc + ld > 0
    setup = (DF_ADD                    # p + q
             + DF_RSQRT + DF_MUL       # (p+q)^-1/2 and its square
             + DF_MUL + DF_MUL * ket   # rho/zeta (T needs it), rho/eta
             + 3 * DF_ADD              # PQ
             + 3 * DF_MUL * bra + 3 * DF_MUL * ket   # WP, WQ
             + 5 * DF_MUL + 2 * DF_ADD   # T = zeta (rho/zeta) |PQ|^2
             + 2 * DF_MUL              # prefactor
             + DF_MUL * (L + 1))       # B_m = prefactor F_m
    boys = 13 + 79 + ((79 + DF_MUL + 2 + 25 * L) if L >= 1 else 0)
    return setup + boys + vrr_flops * DF_FMA / 2.0


def kernel_hash():
    """Hash of the source the dominant kernel, eri_jk_kernel<C_ps_ss, double>,
    is compiled from, with // comments removed: eri.cuh without the
    cooperative (L >= 5) kernel's section and the launcher macros, the
    generated C_ps_ss class and hf_device.h."""
    import re
    csrc = os.path.join(ROOT, "paper_1303_4916_gb300", "csrc")

    def code(text):
        lines = re.sub(r"//[^\n]*", "", text).splitlines()
        return "\n".join(ln.rstrip() for ln in lines if ln.strip())
    with open(os.path.join(csrc, "eri.cuh")) as fh:
        src = fh.read()
    a = src.find("// ------------------------------------------------------------- cooperative kernel")
    b = src.find("// ------------------------------------------------------------- ERI tensor kernel")
    c = src.find("// Instantiate the launchers of one class")
    part = src[:a] + src[b:c] if 0 <= a < b < c else src
    with open(os.path.join(csrc, "eri_classes.cuh")) as fh:
        gen = fh.read()
    i = gen.find("struct C_ps_ss {")
    with open(os.path.join(csrc, "hf_device.h")) as fh:
        dev = fh.read()
    h = hashlib.sha256()
    for t in (part, gen[i:gen.find("\n};\n", i)], dev):
        h.update(code(t).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name: str, tier: str = "fp64"):
    """DRAM bytes per launch of the named kernel from the committed ncu summary
    (profiles/eri_jk_c2_traffic.txt for FP64, eri_jk_c2_traffic_df64.txt for
    the df64 tier), when it was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "eri_jk_c2_traffic.txt" if tier == "fp64" else "eri_jk_c2_traffic_df64.txt")
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


def _oracle_slice(args):
    """Worker of the all-core oracle timing: the oracle's own jk_quartets on
    one slice of the sampled quartets; returns its elapsed seconds."""
    mol, q = args
    import oracle
    ob = oracle.Basis(mol)
    D = np.eye(ob.nbf) * 0.1
    t0 = time.perf_counter()
    ob.jk_quartets(D, q)
    return time.perf_counter() - t0


def oracle_sample_rate_all_cores(mol, tau, n_sample, seed=1, cores=None):
    """The same oracle, unchanged, on all host cores: the sample of unique
    surviving quartets is split into one slice per core and the slices run
    in parallel in spawned worker processes (started with 'spawn', so no
    CUDA state is forked).  Returns (builds_per_s, cores, n_sample, seconds):
    the sample's quartets over the slowest worker's time, scaled to a build."""
    import multiprocessing as mp
    import oracle
    cores = cores or os.cpu_count() or 1
    ob = oracle.Basis(mol)
    Q = ob.schwarz()
    ns = mol.nshell
    n_total = ob.count_quartets(tau)
    rng = np.random.default_rng(seed)
    pairs = np.array([(a, b) for a in range(ns) for b in range(a + 1)], dtype=np.int64)
    out = []
    while len(out) < n_sample:
        i, j = rng.integers(0, len(pairs), size=2)
        if j > i:
            i, j = j, i
        (a, b), (c, d) = pairs[i], pairs[j]
        if Q[a, b] * Q[c, d] >= tau:
            out.append((a, b, c, d))
    q = np.array(out, dtype=np.int32)
    slices = [(mol, q[k::cores]) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        secs = pool.map(_oracle_slice, slices, chunksize=1)
    t = max(secs)
    return n_sample / t / n_total, cores, n_sample, t


def cpu_description():
    """Host CPU model, architecture and core count, as lscpu or /proc report them."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    arch = platform.machine()
    note = ("the oracle's Boys series runs in long double: 80-bit hardware on x86-64, "
            "128-bit software quad precision on aarch64") if arch in ("aarch64", "arm64", "x86_64") else ""
    return {"cpu_model": model or platform.processor() or "unknown", "arch": arch,
            "cores_all": os.cpu_count(), "long_double_note": note}


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


# ---------------------------------------------------------------- multi-rank
def max_over_ranks(seconds: float, dist=None, device="cpu") -> float:
    """The job's time is the slowest rank's (replicas, no data-path collective)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps_per_rank: int, seconds_max: float, world: int) -> float:
    """Whole-job builds/s: the builds of all ranks over the slowest rank's time."""
    return world * steps_per_rank / seconds_max


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
        total_s = max_over_ranks(total_s, dist, dev)
        dist.barrier()

    # per-class kernel durations (CUDA events on the library stream), averaged
    prof = []
    for k in range(max(3, min(args.steps, 10))):
        flush.zero_()
        prof.append(basis.fock_jk_profiled(D, J, K, opts))
    clk = clocks.stop()
    prof = np.mean(np.array(prof), axis=0)

    # production precision modes on the same workload, each timed the same way
    # and compared with the FP64 build: F = 2J - K
    F64 = 2.0 * J - K
    modes = {}
    for name, o in (("df64", hf.jk_opts(schwarz_tau=WORKLOAD["tau"], df64=True)),
                    ("fp32_split", hf.jk_opts(schwarz_tau=WORKLOAD["tau"], fp32_bound=1e-5)),
                    ("fp32_split_df64", hf.jk_opts(schwarz_tau=WORKLOAD["tau"], fp32_bound=1e-5, df64=True)),
                    ("fp32_split_df64_fp32boys", hf.jk_opts(schwarz_tau=WORKLOAD["tau"], fp32_bound=1e-5,
                                                            df64=True, fp32_boys=True))):
        Jm = torch.empty_like(D)
        Km = torch.empty_like(D)
        basis.fock_jk(D, Jm, Km, o)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            basis.fock_jk(D, Jm, Km, o)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        modes[name] = {"builds_per_s": 1000.0 / ms, "ms_per_build": ms,
                       "max_abs_dF_vs_fp64": float((2.0 * Jm - Km - F64).abs().max())}

    # df64 tier: per-class kernel durations of the same build, for its roofline
    odf = hf.jk_opts(schwarz_tau=WORKLOAD["tau"], df64=True)
    Jd = torch.empty_like(D)
    Kd = torch.empty_like(D)
    basis.fock_jk_profiled(D, Jd, Kd, odf)
    prof_df = []
    for k in range(max(3, min(args.steps, 10))):
        flush.zero_()
        prof_df.append(basis.fock_jk_profiled(D, Jd, Kd, odf))
    prof_df = np.mean(np.array(prof_df), axis=0)

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
    cls_name = f"({'spdfg'[s.la]}{'spdfg'[s.lb]}|{'spdfg'[s.lc]}{'spdfg'[s.ld]})"
    traffic = ncu_traffic(cls_name)
    all_ms = float(prof[:, 0].sum() + prof[:, 1].sum())
    all_flops = sum(flops)

    # df64 roofline: the dominant df64 class kernel, counted FP32 operations
    # per primitive quartet against the FP32 lane-operation rate
    ddom = int(np.argmax(prof_df[:, 0]))
    sd = stats[ddom]
    ops_pq = df64_ops_per_prim_quartet(sd.la, sd.lb, sd.lc, sd.ld, sd.vrr_flops)
    d_ms = float(prof_df[ddom, 0])
    d_ach = ops_pq * sd.prim_quartets_fp64 / (d_ms * 1e-3) / 1e12
    d_peak = fp32_alu_peak(sm_count, 2070.0)
    d_name = f"({'spdfg'[sd.la]}{'spdfg'[sd.lb]}|{'spdfg'[sd.lc]}{'spdfg'[sd.ld]})"
    roofline_df64 = {"bound": "alu", "achieved": d_ach, "peak": d_peak, "unit": "T FP32-op/s",
                     "frac": d_ach / d_peak, "traffic": ncu_traffic(d_name, "df64"),
                     "kernel": f"eri_jk_kernel {d_name} df64", "kernel_ms": d_ms,
                     "fp32_ops_per_prim_quartet": ops_pq, "prim_quartets": sd.prim_quartets_fp64,
                     "peak_note": "FP32 nominal: 152 SM x 128 lanes x 2.07 GHz (FADD/FMUL/FFMA one per lane per clock)"}

    value = job_value(args.steps, total_s, world)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, nsmp, ntot, dt = oracle_sample_rate(mol, WORKLOAD["tau"], seconds_target=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nsmp} random unique surviving shell quartets of {ntot} ({dt:.1f} s single-thread), "
                         f"scaled to one full build"}
        desc = cpu_description()
        cpu.update(desc)
        try:
            # all cores: a sample sized for about cpu_seconds of work per core
            n_all = int(nsmp * max(1, desc["cores_all"] or 1) * min(1.0, 6.0 / max(dt, 1e-9)))
            va, cores, n2, t2 = oracle_sample_rate_all_cores(mol, WORKLOAD["tau"], max(n_all, 1000))
            cpu.update({"value_all_cores": va, "cores_all": cores,
                        "sample_all_cores": f"{n2} random unique surviving shell quartets split over {cores} "
                                            f"spawned processes ({t2:.1f} s slowest), scaled to one full build"})
        except Exception as e:  # the single-thread figure stands on its own
            cpu["value_all_cores"] = None
            cpu["all_cores_error"] = f"{type(e).__name__}: {e}"
    # the rest of the metric, measured in the same run: p99 SCF latency of the
    # served stream (df64 and df64 + FP32 split against a FIFO loop of plain
    # FP64 solves, energies against FP64 and the oracle) and the 150-atom
    # molecule's builds per precision mode; each guarded so that a failure is
    # recorded instead of losing the line
    extras = {}
    if world == 1 and not args.no_extras:
        t_ex = time.perf_counter()
        pending = []
        try:
            extras["serving"] = measure_serve(args.nreq, args.atoms_max, args.max_active, args.e_tol,
                                              args.oracle_budget, oracle_background=pending)
        except Exception as e:
            extras["serving"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            extras["rys_water_qz"] = rys_water_qz(cluster=4)
        except Exception as e:
            extras["rys_water_qz"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            extras["mp2_40_atom"] = measure_mp2(mol)
        except Exception as e:
            extras["mp2_40_atom"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            left = args.extras_budget - (time.perf_counter() - t_ex)
            extras["c3_150_atom"] = measure_c3(budget_s=max(0.0, left), modes=("fp32_split_df64", "fp64"))
        except Exception as e:
            extras["c3_150_atom"] = {"error": f"{type(e).__name__}: {e}"}
        for check, served_e, fifo_e, into in pending:   # the oracle ran meanwhile on the host cores
            into["vs_oracle"] = check.collect(served_e, fifo_e, timeout_s=5.0)
        extras["extras_wall_s"] = time.perf_counter() - t_ex
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(n), parallelism=("replicas" if world > 1 else "single-gpu")),
        "eri_quartets_per_s": value * nq_total,
        "quartets_per_build": nq_total,
        # beside the quartet rate: unique Cartesian integrals and primitive
        # quartets per second, and the counted FP64 work of a whole build
        "cartesian_integrals_per_s": value * sum(
            (s_.quartets_fp64 + s_.quartets_fp32) * ((s_.la + 1) * (s_.la + 2) // 2) * ((s_.lb + 1) * (s_.lb + 2) // 2)
            * ((s_.lc + 1) * (s_.lc + 2) // 2) * ((s_.ld + 1) * (s_.ld + 2) // 2) for s_ in stats),
        "prim_quartets_per_s": value * sum(s_.prim_quartets_fp64 + s_.prim_quartets_fp32 for s_ in stats),
        "build_tflops_fp64": all_flops * value / 1e12,
        "scf": {"latency_s": scf_latency, "iterations": scf.iterations, "converged": scf.converged,
                "energy": scf.energy, "fock_builds": scf.fock_builds},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"eri_jk_kernel {cls_name} fp64",
                     "kernel_ms": dom_ms, "kernel_flops": flops[dom],
                     "peak_note": "FP64 CUDA-core nominal: 152 SM x 2 DFMA/clk x 2.07 GHz",
                     "all_classes_tflops": all_flops / (all_ms * 1e-3) / 1e12},
        "roofline_df64": roofline_df64,
        "precision_modes": modes,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * n * 8,
                "d2h_bytes_per_step": 2 * n * n * 8},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other workloads
# Secondary measurements (not the driver's default line): each prints one
# JSON line of its own.

def _ctx_basis(mol, hf):
    ctx = hf.Context(0)
    return ctx, hf.Basis(ctx, mol)


def run_c1(args):
    """8-atom H chain (seed 0): RHF, DIIS off, direct and stored-tensor J/K."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import h_line
    mol = h_line()
    ctx, basis = _ctx_basis(mol, hf)
    out = {"workload": "8-atom H chain (seed 0), nbf 8, RHF DIIS off, max 30 iterations"}
    for stored in (False, True):
        basis.scf(max_iter=30, e_tol=1e-8, diis_size=0, schwarz_tau=0.0, stored_eri=stored)
        t0 = time.perf_counter()
        r = basis.scf(max_iter=30, e_tol=1e-8, diis_size=0, schwarz_tau=0.0, stored_eri=stored)
        out["stored" if stored else "direct"] = {"scf_latency_s": time.perf_counter() - t0,
                                                 "iterations": r.iterations, "energy": r.energy}
    D = r.tensors["D"]
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    opts = hf.jk_opts(schwarz_tau=0.0)
    for _ in range(5):
        basis.fock_jk(D, J, K, opts)
    torch.cuda.synchronize()
    n = 200
    t0 = time.perf_counter()
    for _ in range(n):
        basis.fock_jk(D, J, K, opts)
    torch.cuda.synchronize()
    out["direct_builds_per_s"] = n / (time.perf_counter() - t0)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": out["direct_builds_per_s"], "dtype": "f64",
                      "data": "synthetic", "config": out}), flush=True)


def run_c3(args):
    """150-atom s+p+d lattice (seed 2): FP64 J/K build versus the precision
    split (Schwarz bound < 1e-5 in FP32), at the density of iteration 1."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import lattice_molecule
    mol = lattice_molecule(150, 2, "spd")
    t0 = time.perf_counter()
    ctx, basis = _ctx_basis(mol, hf)
    setup_s = time.perf_counter() - t0
    mixed = hf.jk_opts(schwarz_tau=1e-12, fp32_bound=1e-5)
    plain = hf.jk_opts(schwarz_tau=1e-12)
    nq, nf = basis.count_quartets(mixed)

    def est_seconds(o, tflops64=0.6, tflops32=20.0):
        t = 0.0
        for st in basis.class_stats(o):
            t += (st.prim_quartets_fp64 * st.prim_flops + st.quartets_fp64 * (st.hrr_flops + st.digest_flops)) / (tflops64 * 1e12)
            t += (st.prim_quartets_fp32 * st.prim_flops + st.quartets_fp32 * (st.hrr_flops + st.digest_flops)) / (tflops32 * 1e12)
        return t
    est = {"fp64": est_seconds(plain), "mixed": est_seconds(mixed)}
    print(json.dumps({"c3_estimate_s_per_build": est, "quartets": nq, "quartets_fp32": nf, "nbf": basis.nbf}),
          flush=True)
    if max(est.values()) > args.c3_max_seconds:
        print(json.dumps({"skipped": f"estimated build time above --c3-max-seconds {args.c3_max_seconds}"}))
        return 0
    r = basis.scf(max_iter=1, e_tol=1e-8, diis_size=0, fp32_bound=1e-5)   # D_1 from diagonalising H
    D = r.tensors["D"]
    res = {}
    for name, o in (("mixed", mixed), ("fp64", plain)):
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        basis.fock_jk(D, J, K, o)
        torch.cuda.synchronize()
        steps = max(1, args.steps if name == "mixed" else 1)
        t0 = time.perf_counter()
        for _ in range(steps):
            basis.fock_jk(D, J, K, o)
        torch.cuda.synchronize()
        res[name] = {"builds_per_s": steps / (time.perf_counter() - t0), "F": 2 * J - K}
    dF = float((res["mixed"]["F"] - res["fp64"]["F"]).abs().max())
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": res["mixed"]["builds_per_s"], "dtype": "f64+f32",
                      "data": "synthetic",
                      "config": {"workload": f"150-atom s+p+d lattice (seed 2), nbf {basis.nbf}, density of RHF "
                                             f"iteration 1, Schwarz 1e-12, FP32 below bound 1e-5",
                                 "quartets": nq, "quartets_fp32": nf, "setup_s": setup_s},
                      "fp64_builds_per_s": res["fp64"]["builds_per_s"],
                      "speedup_mixed_vs_fp64": res["mixed"]["builds_per_s"] / res["fp64"]["builds_per_s"],
                      "max_abs_dF_mixed_vs_fp64": dF}), flush=True)


def measure_c3(budget_s=900.0, modes=("fp32_split_df64", "df64", "fp64")):
    """150-atom s+p+d lattice (seed 2; nbf 1366), full size: one J/K build
    per precision mode at a density supported on six shells, timed with CUDA
    events, compared with the FP64 build and with the stored J/K rows of the
    CPU oracle (tests/golden/c3_rows.npz, written by
    tests/golden/make_c3_rows.py).  Modes run cheapest first; a mode is
    skipped when the time spent plus its estimate (from the first mode's
    time and the modes' quartet work) would pass budget_s."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import lattice_molecule, shell_supported_density
    t_start = time.perf_counter()
    mol = lattice_molecule(150, 2, "spd")
    ctx, basis = _ctx_basis(mol, hf)
    setup_s = time.perf_counter() - t_start
    Dn, shells, rows = shell_supported_density(mol, seed=11)
    gold = np.load(os.path.join(ROOT, "tests", "golden", "c3_rows.npz"))
    if gold["rows"].tolist() != rows.tolist() or gold["shells"].tolist() != list(shells):
        raise RuntimeError("stored 150-atom oracle rows were made for another density")
    D = torch.tensor(Dn, device="cuda:0")
    opts = {"fp64": hf.jk_opts(schwarz_tau=1e-12),
            "df64": hf.jk_opts(schwarz_tau=1e-12, df64=True),
            "fp32_split_df64": hf.jk_opts(schwarz_tau=1e-12, fp32_bound=1e-5, df64=True)}
    # relative cost of a mode, measured on this molecule (fp64 411 s, df64 173 s, split+df64 143 s)
    rel = {"fp32_split_df64": 1.0, "df64": 1.2, "fp64": 2.9}
    stream = torch.cuda.current_stream()
    out, res, skipped = {}, {}, {}
    first_s = None
    first_mode = None
    for name in modes:
        spent = time.perf_counter() - t_start
        if first_s is not None:
            est = first_s * rel[name] / rel[first_mode]
            if spent + est > budget_s:
                skipped[name] = f"estimated {est:.0f} s would pass the {budget_s:.0f} s budget ({spent:.0f} s spent)"
                continue
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        basis.fock_jk(D, J, K, opts[name])
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1000.0
        if first_s is None:
            first_s, first_mode = sec, name
        nq, nf = basis.count_quartets(opts[name])
        out[name] = (J.cpu().numpy(), K.cpu().numpy())
        res[name] = {"seconds_per_build": sec, "builds_per_s": 1.0 / sec, "quartets": nq, "quartets_fp32": nf,
                     "quartets_per_s": nq / sec,
                     "max_abs_dJ_rows_vs_oracle": float(np.abs(out[name][0][rows] - gold["J"]).max()),
                     "max_abs_dK_rows_vs_oracle": float(np.abs(out[name][1][rows] - gold["K"]).max())}
    if "fp64" in out:
        F64 = 2 * out["fp64"][0] - out["fp64"][1]
        for name in out:
            if name != "fp64":
                res[name]["max_abs_dF_vs_fp64"] = float(np.abs(2 * out[name][0] - out[name][1] - F64).max())
    return {"workload": f"150-atom s+p+d lattice (seed 2), nbf {basis.nbf}, density on shells {list(shells)}, "
                        f"Schwarz 1e-12, one J/K build per mode",
            "setup_s": setup_s, "rows": rows.tolist(), "modes": res, "skipped": skipped,
            "wall_s": time.perf_counter() - t_start}


def run_c3check(args):
    """150-atom s+p+d lattice: the measure_c3 modes, without a time budget."""
    r = measure_c3(budget_s=1e9)
    m = r["modes"]
    best = m.get("fp32_split_df64") or next(iter(m.values()))
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": best["builds_per_s"], "dtype": "f64/df64+f32",
                      "data": "synthetic", "config": {"workload": r["workload"], "setup_s": r["setup_s"],
                                                      "rows": r["rows"]},
                      "modes": m}), flush=True)


def run_batch(args):
    """Batched SCF of the first --nmol molecules of the 512-molecule stream
    (atoms U[4,60], s+p rules, seeds 1000+i) versus a loop of single-molecule
    FP64 solves; the autotuner's per-class launch choices come from the
    context's JSON log; the cheapest members are checked against the CPU
    oracle's RHF in a background process while the GPU runs."""
    import tempfile
    import paper_1303_4916_gb300 as hf
    from synth import batch_molecules
    mols = batch_molecules(512)[: args.nmol]
    check = OracleCheck(mols, args.e_tol, args.oracle_budget) if args.oracle_budget > 0 else None
    ctx = hf.Context(0)
    logf = tempfile.NamedTemporaryFile(suffix=".jsonl", delete=False).name
    ctx.set_log(logf)
    bases = [hf.Basis(ctx, m) for m in mols]
    t0 = time.perf_counter()
    plain = [b.scf(max_iter=128, e_tol=args.e_tol, diis_size=8, outputs=False) for b in bases]
    t_plain = time.perf_counter() - t0
    out = {}
    for name, fb, dfm in (("batch_fp64", 0.0, False), ("batch_df64", 0.0, True), ("batch_df64_fp32split", 1e-5, True)):
        t0 = time.perf_counter()
        res, st = hf.scf_solve_batch(bases, max_iter=128, e_tol=args.e_tol, diis_size=8, fp32_bound=fb, df64=dfm)
        dt = time.perf_counter() - t0
        builds = sum(r.fock_builds for r in res)
        both = [(r, p) for r, p in zip(res, plain) if r.converged and p.converged]
        out[name] = {"seconds": dt, "mol_fock_builds_per_s": builds / dt, "scf_per_s": len(res) / dt,
                     "speedup_vs_plain_loop": t_plain / dt,
                     "converged": int(sum(r.converged for r in res)),
                     "max_abs_dE_vs_plain_both_converged": max(abs(r.energy - p.energy) for r, p in both),
                     "n_both_converged": len(both),
                     "n_dE_above_1e-8": int(sum(abs(r.energy - p.energy) > 1e-8 for r, p in both))}
        out[name]["energies"] = [float(r.energy) for r in res]
    ctx.set_log(None)
    tune = [json.loads(x) for x in open(logf) if '"autotune"' in x]
    os.unlink(logf)
    pb = sum(p.fock_builds for p in plain)
    line = {"metric": "molecule Fock builds/s", "unit": "builds/s", "value": out["batch_df64"]["mol_fock_builds_per_s"],
            "dtype": "df64", "data": "synthetic",
            "config": {"workload": f"first {len(mols)} of 512 molecules, atoms U[4,60], s+p, seeds 1000+i",
                       "e_tol": args.e_tol, "nbf_total": int(sum(b.nbf for b in bases)),
                       "atoms": [int(m.natom) for m in mols]},
            "plain_loop_fp64": {"seconds": t_plain, "mol_fock_builds_per_s": pb / t_plain,
                                "scf_per_s": len(mols) / t_plain, "converged": int(sum(p.converged for p in plain))},
            "autotune": tune}
    if check is not None:
        line["vs_oracle"] = check.collect({k: v["energies"] for k, v in out.items()},
                                          [float(p.energy) for p in plain], timeout_s=5.0)
    for v in out.values():
        v.pop("energies")
    line.update(out)
    print(json.dumps(line), flush=True)


def _oracle_cost(mol):
    """Rough cost of the oracle's RHF on a molecule: (functions x mean primitives)^4."""
    return (float(mol.nbf) * float(np.mean(mol.shell_nprim))) ** 4


def _oracle_rhf_energy(args):
    """Background worker: the oracle's RHF of one molecule, or None once the
    deadline has passed; returns (index, energy, converged, seconds)."""
    mol, i, e_tol, deadline, threads = args
    if time.time() > deadline:
        return None
    import oracle
    t0 = time.time()
    r = oracle.rhf(mol, max_iter=128, e_tol=e_tol, diis_size=8, tau=1e-12, nthreads=threads)
    return (int(i), float(r.energy), bool(r.converged), time.time() - t0)


def mp_timeout():
    import multiprocessing as mp
    return mp.TimeoutError


class OracleCheck:
    """The CPU oracle's RHF on the cheapest members of the served stream, run
    in one spawned process while the GPU measurements go on (the host cores
    are otherwise idle then), collected at the end."""

    def __init__(self, mols, e_tol, budget_s, threads=None):
        import multiprocessing as mp
        self.mols = mols
        order = sorted(range(len(mols)), key=lambda i: _oracle_cost(mols[i]))
        threads = threads or max(1, (os.cpu_count() or 2) // 2)
        self.t0 = time.time()
        self.pool = mp.get_context("spawn").Pool(1)
        tasks = [(mols[i], i, e_tol, self.t0 + budget_s, threads) for i in order]
        self.it = self.pool.imap(_oracle_rhf_energy, tasks)
        self.n = len(tasks)
        self.threads = threads

    def collect(self, served, fifo, timeout_s=60.0):
        got, err = [], None
        t_end = time.time() + timeout_s
        for _ in range(self.n):   # whatever has finished by now; a member still running is dropped
            try:
                r = self.it.next(timeout=max(0.01, t_end - time.time()))
            except StopIteration:
                break
            except Exception as e:
                err = f"{type(e).__name__}: {e}" if not isinstance(e, mp_timeout()) else None
                break
            if r is None:
                break
            got.append(r)
        self.pool.terminate()
        self.pool.join()
        checked = []
        for i, e, conv, sec in got:
            if not conv:
                continue
            checked.append({"request": i, "natom": int(self.mols[i].natom), "nbf": int(self.mols[i].nbf),
                            "oracle_s": sec, **{f"dE_{k}": abs(v[i] - e) for k, v in served.items()},
                            "dE_fifo_fp64": abs(fifo[i] - e)})
        keys = [f"dE_{k}" for k in served] + ["dE_fifo_fp64"]
        return {"n_checked": len(checked), "host_threads": self.threads, "wall_s": time.time() - self.t0,
                "error": err, **{f"max_abs_{k}": max((c[k] for c in checked), default=None) for k in keys},
                "members": checked}


def measure_serve(nreq=24, atoms_max=16, max_active=32, e_tol=1e-8, oracle_budget_s=90.0, timeout_s=1800.0,
                  oracle_background=None):
    """Open-loop replay of the first nreq requests of the Poisson stream
    (mean 200/s, seed 7; atoms log-uniform [4, atoms_max], s+p+d rules,
    molecule seeds 10000+i), through the continuous-batching server in the
    df64 tier and in the df64 tier with the FP32 split (bound 1e-5), and
    through a FIFO loop of single-molecule plain FP64 solves on the same
    arrival times.  Latency = done - arrival.  Every served energy is
    compared with the FIFO FP64 one; the cheapest members (by an oracle cost
    estimate) are compared with the CPU oracle's RHF, computed in a
    background process for oracle_budget_s seconds (or, when
    oracle_background is a list, the OracleCheck is appended to it and
    collected by the caller after its other GPU measurements)."""
    import threading as th
    import paper_1303_4916_gb300 as hf
    import oracle
    from synth import lattice_molecule, serve_stream
    t_arr, sizes, seeds = serve_stream(nreq, atoms=(4, atoms_max))
    mols = [lattice_molecule(int(n), int(sd), "spd") for n, sd in zip(sizes, seeds)]
    ctx = hf.Context(0)
    q = lambda v, p: float(np.percentile(np.array(v), p))
    check = OracleCheck(mols, e_tol, oracle_budget_s) if oracle_budget_s > 0 else None

    def served(fp32_bound):
        srv = hf.Server(ctx, max_active=max_active, fp32_bound=fp32_bound, df64=True, e_tol=e_tol)
        tickets = [None] * len(mols)
        t_start = time.perf_counter()

        def feeder():
            for i, m in enumerate(mols):
                d = t_arr[i] - (time.perf_counter() - t_start)
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(m)
        f = th.Thread(target=feeder)
        f.start()
        f.join()
        srv.drain(timeout_s)
        wall = time.perf_counter() - t_start
        rs = [srv.poll(t) for t in tickets]
        srv.close()
        lat = [r.t_done - r.t_submit for r in rs]
        return rs, {"p50_s": q(lat, 50), "p99_s": q(lat, 99), "solves_per_s": len(mols) / wall,
                    "fock_builds_per_s": sum(r.fock_builds for r in rs) / wall,
                    "achieved_per_s": len(mols) / wall, "n_converged": int(sum(r.converged for r in rs))}

    out = {"workload": f"first {nreq} requests of the Poisson stream (200/s, seed 7), atoms logU[4,{atoms_max}], "
                       f"s+p+d rules, e_tol {e_tol:g}, DIIS 8",
           "offered_per_s": len(mols) / max(float(t_arr[-1]), 1e-9), "max_active": max_active}
    res_df, out["served_df64"] = served(0.0)
    res_mx, out["served_df64_fp32split"] = served(1e-5)
    # FIFO loop of plain FP64 single-molecule solves on the same arrivals
    end = 0.0
    lat, e_plain, conv_plain = [], [], []
    t0all = time.perf_counter()
    for i, m in enumerate(mols):
        t0 = time.perf_counter()   # basis set-up included, as in the served latency (admission)
        b = hf.Basis(ctx, m)
        r = b.scf(max_iter=128, e_tol=e_tol, diis_size=8, outputs=False)
        dt = time.perf_counter() - t0
        start = max(float(t_arr[i]), end)
        end = start + dt
        lat.append(end - float(t_arr[i]))
        e_plain.append(r.energy)
        conv_plain.append(bool(r.converged))
        b.close()
    out["fifo_fp64"] = {"p50_s": q(lat, 50), "p99_s": q(lat, 99), "solves_per_s": len(mols) / end,
                        "achieved_per_s": len(mols) / end, "n_converged": int(sum(conv_plain)),
                        "gpu_busy_s": time.perf_counter() - t0all}
    e_plain = np.array(e_plain)
    for key, rs in (("served_df64", res_df), ("served_df64_fp32split", res_mx)):
        both = np.array([r.converged for r in rs]) & np.array(conv_plain)
        dE = np.abs(np.array([r.energy for r in rs]) - e_plain)
        out[key]["max_abs_dE_vs_fifo_fp64"] = float(dE[both].max()) if both.any() else None
        out[key]["n_dE_above_1e-8"] = int((dE[both] > 1e-8).sum())
        out[key]["n_both_converged"] = int(both.sum())
    # the CPU oracle on the cheapest members (background process)
    served_e = {"served_df64": [r.energy for r in res_df], "served_df64_fp32split": [r.energy for r in res_mx]}
    if check is not None:
        if oracle_background is not None:
            oracle_background.append((check, served_e, [float(x) for x in e_plain], out))
        else:
            out["vs_oracle"] = check.collect(served_e, [float(x) for x in e_plain],
                                             timeout_s=max(1.0, oracle_budget_s - (time.time() - check.t0)) + 120)
    out["per_request"] = [{"natom": int(m.natom), "nbf": int(m.nbf), "arrival_s": float(t),
                           "lat_df64_s": r1.t_done - r1.t_submit, "lat_df64_split_s": r2.t_done - r2.t_submit,
                           "lat_fifo_fp64_s": lf, "it": int(r1.iterations)}
                          for m, t, r1, r2, lf in zip(mols, t_arr, res_df, res_mx, lat)]
    return out


def run_serve(args):
    """measure_serve on --nreq requests with atoms up to --atoms-max."""
    r = measure_serve(args.nreq, args.atoms_max, args.max_active, args.e_tol, args.oracle_budget)
    print(json.dumps({"metric": "p99 SCF latency", "unit": "s", "value": r["served_df64"]["p99_s"],
                      "higher_is_better": False, "dtype": "df64", "data": "synthetic",
                      "config": {"workload": r["workload"]}, **r}), flush=True)


def rys_water_qz(steps=10, warmup=3, cluster=8):
    """H2O in the synthetic quadruple-zeta-shaped basis (synth.water_qz(0):
    O 5s4p3d2f1g, H 4s3p2d1f; nbf 140), the shape of the paper's HF timing
    benchmark: every quartet with an f or g shell runs on the Rys-quadrature
    kernel.  Returns the RHF solve (time, iterations, |dE| against the
    stored oracle energy), FP64 J/K builds/s at the converged density
    (Schwarz tau 1e-12, L2 flushed between timed builds, CUDA events on the
    library stream) and the Rys kernels' FP64 roofline: counted operations
    per primitive quartet (recurrences, transfers, products; an FMA counts
    2) over the class kernels timed one by one."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import water_qz
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "water_qz.json")))
    ctx = hf.Context(0)
    mol = water_qz(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    basis = hf.Basis(ctx, mol)
    r = basis.scf(max_iter=100, e_tol=1e-10, diis_size=8, schwarz_tau=0.0)
    torch.cuda.synchronize()
    scf_s = time.perf_counter() - t0
    D = r.tensors["D"]
    o = hf.jk_opts()
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=D.device)
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        basis.fock_jk(D, J, K, o)
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        basis.fock_jk(D, J, K, o)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    # analytic RHF gradient (forces) at the converged density; the first call
    # builds the derivative lists, the second is timed
    basis.gradient(r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad = basis.gradient(r)
    torch.cuda.synchronize()
    grad_s = time.perf_counter() - t0
    prof = basis.fock_jk_profiled(D, J, K, o)
    stats = basis.class_stats(o)
    rys_ms = rys_flops = 0.0
    dom = (0.0, None, 0.0)
    for c, sc in enumerate(stats):
        if max(sc.la, sc.lb, sc.lc, sc.ld) < 3:
            continue
        t = float(prof[c, 0] + prof[c, 1])
        f = (sc.prim_quartets_fp64 + sc.prim_quartets_fp32) * sc.prim_flops + \
            (sc.quartets_fp64 + sc.quartets_fp32) * (sc.hrr_flops + sc.digest_flops)
        rys_ms += t
        rys_flops += f
        if t > dom[0]:
            dom = (t, sc, f)
    peak = fp64_alu_peak(ctx.num_sms, 2070.0)
    ach = rys_flops / (rys_ms * 1e-3) / 1e12 if rys_ms > 0 else 0.0
    out = {"workload": "H2O, synthetic quadruple-zeta-shaped basis (synth.water_qz(0); O 5s4p3d2f1g, H 4s3p2d1f, "
                       "contracted s/p, single-primitive polarisation shells), nbf 140",
           "nbf": int(basis.nbf), "scf_s": scf_s, "scf_iterations": int(r.iterations),
           "energy": r.energy, "abs_dE_vs_oracle": abs(r.energy - ref["energy"]),
           "jk_ms": statistics.median(ms), "builds_per_s": 1000.0 / statistics.median(ms),
           "gradient_s": grad_s, "gradient_max_abs": float(np.abs(grad).max()),
           "gradient_sum_abs": float(np.abs(grad.sum(axis=0)).max()),
           "class_ms_serial_total": float(prof.sum()), "rys_class_ms_serial": rys_ms,
           "rys_share_serial": rys_ms / float(prof.sum()) if prof.sum() > 0 else 0.0,
           "roofline_rys": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                            "scope": "all f/g class kernels, each timed alone",
                            "peak_note": "FP64 nominal: 152 SM x 2 DFMA x 2 x 2.07 GHz"}}
    if dom[1] is not None:
        sc = dom[1]
        name = f"({'spdfg'[sc.la]}{'spdfg'[sc.lb]}|{'spdfg'[sc.lc]}{'spdfg'[sc.ld]})"
        out["rys_dominant"] = {"class": name, "ms": dom[0], "prim_quartets": int(sc.prim_quartets_fp64),
                               "flops_per_prim_quartet": int(sc.prim_flops),
                               "tflops": dom[2] / (dom[0] * 1e-3) / 1e12}
    basis.close()
    if cluster > 0:
        out["cluster"] = rys_cluster(ctx, cluster, steps=max(2, steps // 3))
    return out


def measure_mp2(mol):
    """MP2 correlation energy of the converged RHF state of mol: the AO
    tensor (nbf^4 doubles) built and held in HBM, four one-index transforms
    (cuBLAS DGEMM) and the energy sum; wall time of hf_mp2_energy."""
    import torch
    import paper_1303_4916_gb300 as hf
    ctx = hf.Context(0)
    basis = hf.Basis(ctx, mol)
    r = basis.scf(max_iter=128, e_tol=1e-10, diis_size=8)
    no = mol.n_electrons // 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = basis.mp2_energy(r.tensors["C"], r.tensors["eps"], no)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n = basis.nbf
    out = {"workload": f"{mol.natom}-atom s+p molecule, nbf {n}, n_occ {no}", "e_mp2": e2, "seconds": dt,
           "ao_tensor_gb": n ** 4 * 8 / 1e9,
           "transform_tflops_fp64": 2.0 * (n ** 4 * no + n ** 3 * no * (n - no) + n ** 2 * no * no * (n - no)
                                           + n * no * no * (n - no) ** 2) / dt / 1e12}
    basis.close()
    return out


def rys_class_roofline(basis, D, o, peak):
    """FP64 roofline of the f/g (Rys) class kernels of one J/K build: counted
    operations over the class kernels timed one by one."""
    import torch
    prof = basis.fock_jk_profiled(D, torch.empty_like(D), torch.empty_like(D), o)
    stats = basis.class_stats(o)
    ms = fl = 0.0
    for c, sc in enumerate(stats):
        if max(sc.la, sc.lb, sc.lc, sc.ld) < 3:
            continue
        ms += float(prof[c, 0] + prof[c, 1])
        fl += (sc.prim_quartets_fp64 + sc.prim_quartets_fp32) * sc.prim_flops + \
            (sc.quartets_fp64 + sc.quartets_fp32) * (sc.hrr_flops + sc.digest_flops)
    ach = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "rys_class_ms_serial": ms, "class_ms_serial_total": float(prof.sum()),
            "scope": "all f/g class kernels, each timed alone"}


def rys_cluster(ctx, n, steps=3):
    """n QZ-shaped waters (synth.water_cluster_qz; nbf 140 n): FP64 J/K
    builds/s for a seeded density C C^T (C: nbf x 5n Gaussian / sqrt(nbf);
    the work, set by Schwarz screening, does not depend on D) and the Rys
    kernels' roofline."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import water_cluster_qz
    mol = water_cluster_qz(n, 0)
    basis = hf.Basis(ctx, mol)
    nb = basis.nbf
    rng = np.random.default_rng(5)
    Cm = rng.normal(size=(nb, 5 * n)) / np.sqrt(nb)
    D = torch.tensor(Cm @ Cm.T, dtype=torch.float64, device="cuda:0")
    o = hf.jk_opts()
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    basis.fock_jk(D, J, K, o)
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        basis.fock_jk(D, J, K, o)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    nq, _ = basis.count_quartets(o)
    out = {"workload": f"{n} QZ-shaped waters on a 5.7-bohr cubic lattice (synth.water_cluster_qz({n}, 0)), "
                       f"nbf {nb}, seeded density, Schwarz tau 1e-12",
           "nbf": int(nb), "quartets": int(nq), "jk_ms": statistics.median(ms),
           "builds_per_s": 1000.0 / statistics.median(ms),
           "roofline_rys": rys_class_roofline(basis, D, o, fp64_alu_peak(ctx.num_sms, 2070.0))}
    basis.close()
    return out


def run_rys(args):
    """--workload rys: one JSON line for the quadruple-zeta-shaped water."""
    r = rys_water_qz(args.steps, args.warmup, cluster=args.nwater)
    print(json.dumps({"metric": "Fock(J+K) builds/s (H2O, QZ-shaped basis s..g)", "unit": "builds/s",
                      "value": r["builds_per_s"], "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": r["workload"], "l2": "flushed between timed steps"}, **r}), flush=True)


def run_setup(args):
    """Basis set-up (pair records, Schwarz factors, work lists) of the first
    --nreq molecules of the serving stream (atoms log-uniform [4, --atoms-max],
    s+p+d): the per-request admission cost of the server."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import lattice_molecule, serve_stream
    t_arr, sizes, seeds = serve_stream(args.nreq, atoms=(4, args.atoms_max))
    mols = [lattice_molecule(int(n), int(sd), "spd") for n, sd in zip(sizes, seeds)]
    ctx = hf.Context(0)
    hf.Basis(ctx, mols[0]).close()
    torch.cuda.synchronize()
    per = []
    for m in mols:
        t0 = time.perf_counter()
        b = hf.Basis(ctx, m)
        b.count_quartets(hf.jk_opts())
        torch.cuda.synchronize()
        per.append({"natom": int(m.natom), "nbf": int(b.nbf), "seconds": time.perf_counter() - t0})
        b.close()
    tot = sum(p["seconds"] for p in per)
    print(json.dumps({"metric": "basis set-up", "unit": "s", "value": tot / len(per), "higher_is_better": False,
                      "config": {"workload": f"first {len(mols)} requests of the serving stream, atoms "
                                             f"logU[4,{args.atoms_max}], s+p+d"},
                      "total_s": tot, "per_request": per}), flush=True)


def run_classes(args):
    """Per-class kernel time and achieved FP64 rate on an s+p+d lattice
    molecule (--natom atoms, seed 3), one J/K build at a seeded density."""
    import torch
    import paper_1303_4916_gb300 as hf
    from synth import lattice_molecule
    mol = lattice_molecule(args.natom, 3, "spd")
    ctx, basis = _ctx_basis(mol, hf)
    n = basis.nbf
    rng = np.random.default_rng(0)
    C = rng.normal(size=(n, max(1, mol.n_electrons // 2))) / np.sqrt(n)
    D = torch.tensor(C @ C.T, device="cuda:0")
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    o = hf.jk_opts(schwarz_tau=1e-12, fp32_bound=args.fp32_bound, df64=args.df64)
    basis.fock_jk_profiled(D, J, K, o)
    ms = np.mean([basis.fock_jk_profiled(D, J, K, o) for _ in range(3)], axis=0)
    rows = []
    for c, st in enumerate(basis.class_stats(o)):
        name = f"({'spd'[st.la]}{'spd'[st.lb]}|{'spd'[st.lc]}{'spd'[st.ld]})"
        for r, (q, pq) in enumerate(((st.quartets_fp64, st.prim_quartets_fp64), (st.quartets_fp32, st.prim_quartets_fp32))):
            if q == 0:
                continue
            fl = pq * st.prim_flops + q * (st.hrr_flops + st.digest_flops)
            hi = "df64" if args.df64 else "fp64"
            rows.append({"class": name, "precision": "fp32" if r else hi, "quartets": q, "prim_quartets": pq,
                         "ms": float(ms[c, r]), "tflops": fl / (ms[c, r] * 1e-3) / 1e12 if ms[c, r] > 0 else None})
    print(json.dumps({"workload": f"{args.natom}-atom s+p+d lattice (seed 3), nbf {n}", "fp32_bound": args.fp32_bound,
                      "df64": bool(args.df64),
                      "total_ms": float(ms.sum()), "classes": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c1", "c3", "c3check", "batch", "serve", "classes", "setup", "rys"],
                    help="c2 (default) is the benchmark line; the others print secondary measurements")
    ap.add_argument("--nmol", type=int, default=64)
    ap.add_argument("--nreq", type=int, default=24)
    ap.add_argument("--atoms-max", type=int, default=16)
    ap.add_argument("--max-active", type=int, default=32)
    ap.add_argument("--serve-timeout", type=float, default=1800.0)
    ap.add_argument("--oracle-budget", type=float, default=600.0,
                    help="seconds the background oracle check of served members may run")
    ap.add_argument("--extras-budget", type=float, default=900.0,
                    help="default run: seconds for the serving stream and the 150-atom builds")
    ap.add_argument("--no-extras", action="store_true",
                    help="default run: skip the serving stream and the 150-atom builds")
    ap.add_argument("--c3-max-seconds", type=float, default=120.0)
    ap.add_argument("--natom", type=int, default=12)
    ap.add_argument("--nwater", type=int, default=8, help="rys: waters in the throughput cluster (0 = none)")
    ap.add_argument("--fp32-bound", type=float, default=0.0)
    ap.add_argument("--e-tol", type=float, default=1e-8)
    ap.add_argument("--df64", action="store_true", help="serve, batch, classes: df64 tier above the FP32 bound")
    ap.add_argument("--no-fp32-split", action="store_true", help="serve: no FP32 quartets")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        return {"c1": run_c1, "c3": run_c3, "c3check": run_c3check, "batch": run_batch, "serve": run_serve,
                "classes": run_classes, "setup": run_setup, "rys": run_rys}[args.workload](args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
