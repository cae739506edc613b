"""Throughput benchmark of the fused D2Q9 KBC stream-collide step.

Workload (default): KBC D2Q9, model B, FP32 deviation storage, 16384^2 doubly
periodic grid (A-B population buffers of 19.3 GB, far larger than the 129 MB
L2), seeded random turbulent initial field (E(k) ~ k^4 exp(-2 (k/16)^2),
u_rms = 0.03, Re = 1e5).  One step = one pull-stream + collide update of
every node.  Metric: million lattice-node updates per second (MLUPS).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead, on a bounded sample of the same workload.
Multi-GPU runs (torchrun, one rank per GPU) are independent replicas: each
rank advances its own grid, with no collective on the data path.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline (FP64/FP32/FP16-store) at stated error vs FP64 oracle"
UNIT = "MLUPS"
def workload(n: int) -> str:
    return (f"KBC D2Q9 {'throughput stress: ' if n == 16384 else ''}{n}^2 doubly periodic, "
            "seeded random turbulent initial field (E(k)~k^4 exp(-2(k/16)^2), u_rms=0.03, Re=1e5)")
DTYPE_BYTES = {"f64": 8, "f32": 4, "f16": 2}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--dtype", default="f32", choices=["f64", "f32", "f16"])
    p.add_argument("--variant", default="B", choices=["lbgk", "A", "B", "C", "D"])
    p.add_argument("--kernel", default="auto", choices=["auto", "rows", "bulk", "nodes"],
                   help="step kernel of the headline run (auto: the library's choice)")
    p.add_argument("--extras", type=int, default=1, help="also time f64/f16/LBGK (0: skip)")
    p.add_argument("--extra-steps", type=int, default=100)
    p.add_argument("--e2e", type=int, default=1)
    p.add_argument("--cpu-baseline", type=int, default=1)
    p.add_argument("--seed", type=int, default=2024)
    p.add_argument("--adjoint-steps", type=int, default=0,
                   help="> 0: time only kbc_adjoint (KBC --variant, --dtype, n^2, this many "
                        "steps, checkpoints every --ckpt) and print its JSON line")
    p.add_argument("--ckpt", type=int, default=100)
    p.add_argument("--diag-only", type=int, default=0,
                   help="1: time only kbc_diagnostics and kbc_diagnostics_ext on n^2")
    return p.parse_args()


# ---------------------------------------------------------------- helpers

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def step_kernel_name(args) -> str:
    """The step kernel the headline run launches; "auto" resolves as the
    library does: the bulk-copy kernel for FP16 KBC, the vector rows
    otherwise (every bench width is a multiple of the row vector)."""
    k = args.kernel
    if k == "auto":
        k = "bulk" if args.dtype == "f16" and args.variant != "lbgk" else "rows"
    return {"rows": "step_rows", "bulk": "step_tma", "nodes": "step_nodes"}[k]


def kernel_source_hash() -> str:
    """Hash of the code that defines the vector-row step kernel: the lattice,
    lane and collision headers, the kernel's own section of kbc_kernels.cuh
    and its launch width."""
    csrc = os.path.join(ROOT, "paper_1507_02509_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("kbc_lattice.cuh", "kbc_lanes.cuh", "kbc_collide.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(csrc, "kbc_kernels.cuh")) as f:
        text = f.read()
    a = text.index("// ---------------------------------------------------------------- step, rows")
    b = text.index("// ---------------------------------------------------------------- step, nodes")
    h.update(text[a:b].encode())
    with open(os.path.join(csrc, "kbc_launch.cuh")) as f:
        h.update("".join(l for l in f if "kRowBlock" in l).encode())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str, dtype: str, n: int):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, scaled to n^2 nodes; None if missing, taken on another kernel
    (name, variant, storage) or on other sources."""
    path = os.path.join(ROOT, "profiles", f"kbc_step_rows_{dtype}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    try:
        if vals.get("kernel_source_hash") != kernel_source_hash() or vals.get("kernel") != kernel:
            return None
        return float(vals["dram_bytes_per_node"]) * n * n
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class Ranks:
    """Replica bookkeeping for torchrun launches: one rank per GPU, each rank
    advancing its own grid; timing is the maximum over ranks after a
    barrier, and the job's value is the units of all ranks over that time."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None

    def init(self, backend: str):
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float, device) -> float:
        if self.dist is None:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def job_mlups(world: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' node updates over the slowest rank's time."""
    return world * nodes * steps / seconds / 1e6


def reynolds_viscosity(n: int, urms: float = 0.03, re: float = 1e5):
    from paper_1507_02509_gb300 import viscosity_for_reynolds

    return viscosity_for_reynolds(n, 0.5 * urms * urms, re)


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(steps: int, n: int = 1024, seed: int = 2024, max_seconds: float = 20.0):
    """MLUPS of the FP64 oracle on all host cores on an n^2 field of the same
    workload family; runs at most `steps` steps or about max_seconds."""
    import oracle
    from paper_1507_02509_gb300 import beta_from_viscosity, flows

    cores = os.cpu_count() or 1
    nu = reynolds_viscosity(n)
    beta = beta_from_viscosity(nu)
    rho, ux, uy = flows.turbulence(n, k0=16, urms=0.03, seed=seed)
    g = oracle.init_feq(rho, ux, uy)
    # one probe step to size the run
    t0 = time.perf_counter()
    g = oracle.step(g, oracle.B, beta, 1, nthreads=cores)
    per = time.perf_counter() - t0
    k = max(1, min(steps, int(max_seconds / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.step(g, oracle.B, beta, k, nthreads=cores)
    dt = time.perf_counter() - t0
    return n * n * k / dt / 1e6, cores, k, n


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_oracle_table(seed: int = 2024, per_run_seconds: float = 0.6):
    """The oracle's MLUPS per collision model on one core and on all cores
    (1024^2 samples of the workload's field, steps bounded by time), and for
    KBC B on a 4096^2 sample on all cores: the CPU-baseline matrix, kept to a
    few seconds in all."""
    import oracle
    from paper_1507_02509_gb300 import beta_from_viscosity, flows

    cores = os.cpu_count() or 1
    out = {}
    for n, models, threads in ((1024, ("lbgk", "A", "B", "C", "D"), (1, cores)),
                               (4096, ("B",), (cores,))):
        beta = beta_from_viscosity(reynolds_viscosity(n))
        rho, ux, uy = flows.turbulence(n, k0=16, urms=0.03, seed=seed)
        g = oracle.init_feq(rho, ux, uy)
        del rho, ux, uy
        for m in models:
            for th in threads:
                v = oracle.VARIANTS[m]
                t0 = time.perf_counter()
                oracle.step(g, v, beta, 1, nthreads=th)
                per = time.perf_counter() - t0
                k = max(1, min(5, int(per_run_seconds / max(per, 1e-6))))
                t0 = time.perf_counter()
                oracle.step(g, v, beta, k, nthreads=th)
                dt = time.perf_counter() - t0
                out[f"{m}_{n}_{'1t' if th == 1 else 'all'}"] = round(n * n * k / dt / 1e6, 3)
        del g
    return out


# ---------------------------------------------------------------- GPU arm

def time_steps(lat, steps, stream):
    import torch

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    lat.step(steps)
    end.record(stream)
    end.synchronize()
    lat.sync()
    return start.elapsed_time(end) / 1e3


def run_ours(args):
    import torch

    from paper_1507_02509_gb300 import Lattice, beta_from_viscosity, capi, flows

    ranks = Ranks()
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    ranks.init("nccl")
    stream = torch.cuda.current_stream()
    capi.load()

    n = args.n
    nu = reynolds_viscosity(n)
    beta = beta_from_viscosity(nu)
    rho, ux, uy = flows.turbulence(n, k0=16, urms=0.03, seed=args.seed + rank,
                                   backend="torch", device=f"cuda:{local}")

    barrier = ranks.barrier

    def max_over_ranks(x: float) -> float:
        return ranks.max(x, "cuda")

    # ---- headline: default workload
    lat = Lattice(n, n, variant=args.variant, beta=beta, dtype=args.dtype)
    lat.set_kernel(args.kernel)
    lat.init(rho, ux, uy)
    lat.step(args.warmup)
    lat.sync()
    guard_nodes = lat.guard_count() if args.dtype != "f64" and args.variant != "lbgk" else 0
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t = time_steps(lat, args.steps, stream)
    barrier()
    torch.cuda.synchronize()
    t = max_over_ranks(t)
    guard_on = args.dtype != "f64" and args.variant != "lbgk"
    launches_per_step = 2 if guard_on else 1
    value = job_mlups(world, n * n, args.steps, t)

    # ---- roofline: the step kernel alone (guard pass off), same launch shape
    bpu = DTYPE_BYTES[args.dtype] * 18
    k_roof = min(args.steps, 200)
    if guard_on:
        lat.set_guard(0.0)
    t_roof = time_steps(lat, k_roof, stream)
    if guard_on:
        lat.set_guard(1e-16)
    kernel_s = t_roof / k_roof
    peak, peak_kind = load_peaks()
    achieved = bpu * n * n / kernel_s / 1e9
    kname = f"{step_kernel_name(args)}<{args.variant},{args.dtype}>"
    traffic = traffic_from_profile(kname, args.dtype, n)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes": bpu * n * n, "peak_kind": peak_kind,
                "kernel": kname,
                "kernel_ms": round(kernel_s * 1e3, 4)}

    # ---- e2e through the C ABI with pinned host buffers
    e2e = None
    if args.e2e:
        h_rho = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        h_u = torch.empty((2, n, n), dtype=torch.float64, pin_memory=True)
        h_rho.copy_(rho)
        h_u[0].copy_(ux)
        h_u[1].copy_(uy)
        o_rho = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        o_u = torch.empty((2, n, n), dtype=torch.float64, pin_memory=True)
        # untimed warm-up of the same sequence: the library's first host
        # transfer allocates its staging buffer and copy stream
        capi.kbc_init(lat.h, h_rho, h_u)
        capi.kbc_step(lat.h, 1)
        capi.kbc_moments(lat.h, o_rho, o_u)
        lat.sync()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        capi.kbc_init(lat.h, h_rho, h_u)
        capi.kbc_step(lat.h, args.steps)
        capi.kbc_moments(lat.h, o_rho, o_u)
        lat.sync()
        te = max_over_ranks(time.perf_counter() - t0)
        barrier()
        hb = h_rho.numel() * 8 + h_u.numel() * 8
        db = o_rho.numel() * 8 + o_u.numel() * 8
        e2e = {"value": round(job_mlups(world, n * n, args.steps, te), 1), "unit": UNIT,
               "h2d_bytes_per_step": hb // args.steps, "d2h_bytes_per_step": db // args.steps,
               "what": ("kbc_init from pinned host rho,u + kbc_step(K) + kbc_moments to pinned "
                        "host; copies amortised over the K steps")}
        del h_rho, h_u, o_rho, o_u
    lat.close()
    del lat
    torch.cuda.empty_cache()

    # ---- extras: other storage / LBGK on the same field
    extras = {}
    if args.extras:
        for tag, dt, var in (("f64", "f64", args.variant), ("f16", "f16", args.variant),
                             ("lbgk_f32", "f32", "lbgk"), ("lbgk_f64", "f64", "lbgk"),
                             ("A_f32", "f32", "A"), ("C_f32", "f32", "C"), ("D_f32", "f32", "D")):
            if dt == args.dtype and var == args.variant:
                continue
            lx = Lattice(n, n, variant=var, beta=beta, dtype=dt)
            lx.init(rho, ux, uy)
            lx.step(3)
            lx.sync()
            te = time_steps(lx, args.extra_steps, stream)
            g_on = dt != "f64" and var != "lbgk" and dt == "f32"
            if g_on:
                lx.set_guard(0.0)
                tk = time_steps(lx, args.extra_steps, stream) / args.extra_steps
            else:
                tk = te / args.extra_steps
            b = DTYPE_BYTES[dt] * 18
            extras[tag] = {"mlups": round(n * n * args.extra_steps / te / 1e6, 1),
                           "kernel_gbs": round(b * n * n / tk / 1e9, 1),
                           "frac": round(b * n * n / tk / 1e9 / peak, 4),
                           "steps": args.extra_steps}
            lx.close()
            del lx
            torch.cuda.empty_cache()

    # ---- the other rows of the path: diagnostics reduction and the adjoint
    if args.extras:
        import numpy as np

        lx = Lattice(n, n, variant=args.variant, beta=beta, dtype=args.dtype)
        lx.init(rho, ux, uy)
        lx.sync()
        out = np.zeros(capi.KBC_DIAG_N)
        t0 = time.perf_counter()
        for _ in range(3):
            capi.kbc_diagnostics(lx.h, out)
        td = (time.perf_counter() - t0) / 3
        extras["diagnostics"] = {"ms": round(td * 1e3, 3),
                                 "mlups": round(n * n / td / 1e6, 1),
                                 "what": "kbc_diagnostics (FP64 reductions incl. gamma) + host read"}
        lx.close()
        del lx
        torch.cuda.empty_cache()
        extras["adjoint"] = adjoint_extras(args, local)
        torch.cuda.empty_cache()
        extras["next_rows"] = next_rows_extras(args, rho, ux, uy, beta, peak, stream)
        torch.cuda.empty_cache()
        # the FP64 storage path is bound by the FP64 pipe: its ceiling is the
        # measured DFMA issue rate, its use the FP64 thread-instructions per
        # node (ncu, profiles/) at the measured update rate
        rate = capi.kbc_fp64_fma_rate(ctypes.c_void_p(stream.cuda_stream))
        ops = fp64_ops_from_profile("step_rows<B,f64>") if args.variant == "B" else None
        if "f64" in extras:
            extras["f64"]["fp64_dfma_per_s"] = rate
            extras["f64"]["fp64_inst_per_node"] = ops
            extras["f64"]["fp64_frac"] = (round(ops * extras["f64"]["mlups"] * 1e6 / rate, 4)
                                          if ops else None)

    cpu = None
    if args.cpu_baseline and rank == 0:
        rate, cores, k, nc = cpu_oracle_rate(args.steps)
        cpu = {"value": round(rate, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 C oracle, {nc}^2 field of the same generator, KBC B, {k} steps",
               "cpu_model": cpu_model(),
               "by_model": cpu_oracle_table(args.seed)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": workload(n), "n": n, "variant": args.variant,
                       "storage": args.dtype, "beta": beta, "nu": nu,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (A-B buffers "
                             f"{2 * 9 * n * n * DTYPE_BYTES[args.dtype] / 1e9:.1f} GB vs 129 MB)",
                       "guard_nodes_last_step": guard_nodes},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk.summary(), "extras": extras,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


def adjoint_extras(args, local):
    """The adjoint configuration (512^2, k0 = 8, u_rms = 0.03, Re = 5000 on N,
    KBC B, checkpoints every 100): seconds of kbc_adjoint for 2000 and for
    100 steps in FP32 and FP64, and where its gradient means something: the
    FP32 and FP64 dJ/du0 agree (max norm, relative) to about 1e-3 for the
    first ~100 steps; beyond that the exact linearisation amplifies rounding
    where gamma* is poorly determined (<dh|dh> tiny), and at 2000 steps both
    precisions return rounding-dominated gradients.  valid_steps is the
    largest step count up to which every count tried agrees within 1e-3."""
    import torch

    from paper_1507_02509_gb300 import Lattice, beta_from_viscosity, capi, flows

    na, ka = 512, 100
    ra, xa, ya = flows.turbulence(na, k0=8, urms=0.03, seed=args.seed, backend="torch",
                                  device=f"cuda:{local}")
    beta_a = beta_from_viscosity(na * 0.03 / 5000.0)
    ua = torch.stack((xa, ya)).contiguous()
    counts = (50, 100, 150, 200, 400, 1000, 2000)
    res = {"n": na, "ckpt_every": ka, "seconds": {}, "finite": {}}
    grads = {}
    for dt in ("f32", "f64"):
        la = Lattice(na, na, variant="B", beta=beta_a, dtype=dt)
        g = torch.empty_like(ua)
        capi.kbc_adjoint(la.h, ra, ua, 20, 10, 0, None, g)  # warm-up
        for st in counts:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            finite = True
            try:
                capi.kbc_adjoint(la.h, ra, ua, st, ka, 0, None, g)
            except capi.KBCError as e:
                if e.status != capi.KBC_ERR_NONFINITE:
                    raise
                finite = False
            ta = time.perf_counter() - t0
            if st in (100, 2000):
                res["seconds"][f"{dt}_{st}"] = round(ta, 4)
                res["finite"][f"{dt}_{st}"] = finite
            grads[(dt, st)] = g.clone() if finite else None
        la.close()
    agree, valid, ok = {}, 0, True
    for st in counts:
        a, b = grads[("f32", st)], grads[("f64", st)]
        d = (float((a - b).abs().max() / b.abs().max()) if a is not None and b is not None
             else float("inf"))
        agree[str(st)] = float(f"{d:.3g}")
        ok = ok and d <= 1e-3
        if ok:
            valid = st
    res["fp32_vs_fp64_grad_max_rel"] = agree
    res["valid_steps"] = valid
    res["what"] = ("kbc_adjoint: forward with checkpoints + reverse sweep with segment recompute; "
                   "2000 steps timed as the configuration asks, but its gradient is "
                   "rounding-dominated beyond valid_steps")
    return res


def next_rows_extras(args, rho, ux, uy, beta, peak, stream):
    """The further rows of the path on the bench field (F32 storage, KBC B):
    Grad initialisation against the equilibrium one, the regularised
    stabiliser gamma = 1/beta (the step kernel of gamma*), the exact
    stabiliser (the per-node all-double kernel with the Newton root), the
    extended diagnostics, the spectra, and the y-slab split of the grid into
    four slabs on this GPU (halo exchange before every step).  Times from
    CUDA events on the bound stream (host-returning calls: wall clock around
    the call)."""
    import numpy as np
    import torch

    from paper_1507_02509_gb300 import Lattice, capi, slabs, spectra

    n = args.n
    nodes = n * n
    res = {}

    def events(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()  # warm-up
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    u = torch.stack((ux, uy)).contiguous()
    lat = Lattice(n, n, variant="B", beta=beta, dtype="f32")
    for name, fn in (("init_feq", lambda: capi.kbc_init(lat.h, rho, u)),
                     ("init_grad", lambda: capi.kbc_init_grad(lat.h, rho, u))):
        t = events(fn, 3)
        gbs = 60.0 * nodes / t / 1e9  # rho, u in (FP64), nine FP32 populations out
        res[name] = {"ms": round(t * 1e3, 3), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                     "algorithmic_bytes_per_node": 60}
    lat.init(rho, ux, uy)
    lat.set_gamma(1.0 / beta)
    t = events(lambda: lat.step(100), 1) / 100
    res["regularised_gamma"] = {"mlups": round(nodes / t / 1e6, 1),
                                "frac": round(72.0 * nodes / t / 1e9 / peak, 4),
                                "what": "gamma fixed at 1/beta, F32, the vector-row step kernel"}
    lat.close()
    ne = min(n, 4096)
    le = Lattice(ne, ne, variant="B", beta=beta, dtype="f32")
    le.init(rho[:ne, :ne].contiguous(), ux[:ne, :ne].contiguous(), uy[:ne, :ne].contiguous())
    le.set_gamma("exact")
    t = events(lambda: le.step(5), 1) / 5
    res["exact_gamma"] = {"n": ne, "mlups": round(ne * ne / t / 1e6, 1),
                          "frac_hbm": round(72.0 * ne * ne / t / 1e9 / peak, 4),
                          "what": "root of the exact entropic condition by Newton in FP64 per node "
                                  "(F32 storage): bound by the FP64 pipe and the per-node kernel"}
    le.close()
    lat = Lattice(n, n, variant="B", beta=beta, dtype="f32")
    lat.init(rho, ux, uy)
    lat.sync()
    out = np.zeros(capi.KBC_DIAG_EXT_N)
    capi.kbc_diagnostics_ext(lat.h, out)
    t0 = time.perf_counter()
    for _ in range(2):
        capi.kbc_diagnostics_ext(lat.h, out)
    res["diagnostics_ext_ms"] = round((time.perf_counter() - t0) / 2 * 1e3, 3)
    _, vx, vy = lat.moments()
    lat.close()
    spectra.energy_spectrum(vx, vy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    spectra.energy_spectrum(vx, vy)
    torch.cuda.synchronize()
    res["spectrum_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    del vx, vy
    torch.cuda.empty_cache()
    grp = slabs.SlabGroup(n, n, 4, variant="B", beta=beta, dtype="f32")
    grp.init(rho, ux, uy)
    t = events(lambda: grp.step(20), 1) / 20
    grp.close()
    res["slabs_4_on_one_gpu"] = {"mlups": round(nodes / t / 1e6, 1),
                                 "frac": round(72.0 * nodes / t / 1e9 / peak, 4),
                                 "what": "the grid as four y-slabs with a halo exchange (two "
                                         "device copies per slab) before every step"}
    return res


def fp64_ops_from_profile(kernel: str):
    """FP64 thread-instructions per node of the FP64 step kernel from the
    committed ncu summary, or None when missing, taken on another kernel or
    on other sources."""
    path = os.path.join(ROOT, "profiles", "kbc_step_rows_f64_ops.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    try:
        if vals.get("kernel_source_hash") != kernel_source_hash() or vals.get("kernel") != kernel:
            return None
        return float(vals["fp64_inst_per_node"])
    except (KeyError, ValueError):
        return None


def run_reference(args):
    """The oracle on the host cores: each step is one oracle step of a
    1024^2 periodic field of the same workload family."""
    ranks = Ranks()
    world, rank = ranks.world, ranks.rank
    if rank != 0:
        return
    import oracle
    from paper_1507_02509_gb300 import beta_from_viscosity, flows

    n = 1024
    cores = os.cpu_count() or 1
    beta = beta_from_viscosity(reynolds_viscosity(n))
    rho, ux, uy = flows.turbulence(n, k0=16, urms=0.03, seed=args.seed)
    g = oracle.init_feq(rho, ux, uy)
    g = oracle.step(g, oracle.B, beta, args.warmup, nthreads=cores)
    t0 = time.perf_counter()
    oracle.step(g, oracle.B, beta, args.steps, nthreads=cores)
    dt = time.perf_counter() - t0
    v = n * n * args.steps / dt / 1e6
    line = {
        "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": workload(args.n), "n": args.n, "variant": "B", "storage": "f64",
                   "sample": f"{n}^2 periodic field of the same generator per step"},
        "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"FP64 C oracle, {n}^2 field, {args.steps} steps"},
        "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """kbc_adjoint alone: forward sweep with checkpoints, J, reverse sweep
    with segment recompute; seeded turbulent field (k0 = n/64, u_rms = 0.03,
    Re = 5000 on N), gradient of the final kinetic energy.  One warm-up call,
    then min(--steps, 10) timed calls (wall clock around each synchronous
    call; the median is reported)."""
    import numpy as np
    import torch

    from paper_1507_02509_gb300 import Lattice, beta_from_viscosity, capi, flows

    n = args.n
    rho, ux, uy = flows.turbulence(n, k0=max(1.0, n / 64), urms=0.03, seed=args.seed,
                                   backend="torch", device="cuda")
    lat = Lattice(n, n, variant=args.variant, beta=beta_from_viscosity(n * 0.03 / 5000.0),
                  dtype=args.dtype)
    u = torch.stack((ux, uy)).contiguous()
    g = torch.empty_like(u)
    times, finite = [], True
    for k in range(1 + max(1, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            capi.kbc_adjoint(lat.h, rho, u, args.adjoint_steps, args.ckpt, 0, None, g)
        except capi.KBCError as e:
            if e.status != capi.KBC_ERR_NONFINITE:
                raise
            finite = False
        if k:
            times.append(time.perf_counter() - t0)
    lat.close()
    t = float(np.median(times))
    print(json.dumps({"metric": "kbc_adjoint seconds", "value": round(t, 4), "unit": "s",
                      "higher_is_better": False, "n": n, "variant": args.variant,
                      "dtype": args.dtype, "steps": args.adjoint_steps, "ckpt_every": args.ckpt,
                      "gradients_finite": finite, "data": "synthetic"}))


def run_diagnostics(args):
    """kbc_diagnostics and kbc_diagnostics_ext alone on the seeded turbulent
    field (--variant, --dtype, n^2): one warm-up call each, then the median of
    min(--steps, 10) timed calls (each returns its values on the host)."""
    import numpy as np
    import torch

    from paper_1507_02509_gb300 import Lattice, beta_from_viscosity, capi, flows

    n = args.n
    rho, ux, uy = flows.turbulence(n, k0=16, urms=0.03, seed=args.seed, backend="torch",
                                   device="cuda")
    lat = Lattice(n, n, variant=args.variant, beta=beta_from_viscosity(n * 0.03 / 1e5),
                  dtype=args.dtype)
    lat.init(rho, ux, uy)
    lat.sync()
    res = {}
    for name, fn, k in (("diagnostics", capi.kbc_diagnostics, capi.KBC_DIAG_N),
                        ("diagnostics_ext", capi.kbc_diagnostics_ext, capi.KBC_DIAG_EXT_N)):
        out = np.zeros(k)
        times = []
        for r in range(1 + max(1, min(args.steps, 10))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn(lat.h, out)
            if r:
                times.append(time.perf_counter() - t0)
        res[name] = round(float(np.median(times)) * 1e3, 3)
    lat.close()
    print(json.dumps({"metric": "diagnostics ms per call", "value": res["diagnostics"], "unit": "ms",
                      "higher_is_better": False, "diagnostics_ext_ms": res["diagnostics_ext"],
                      "n": n, "variant": args.variant, "dtype": args.dtype, "data": "synthetic"}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.adjoint_steps > 0:
        run_adjoint(args)
    elif args.diag_only:
        run_diagnostics(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
