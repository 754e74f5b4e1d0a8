"""Benchmark of the fused stream-and-collide sweep (GLUPS, HBM GB/s).

Workload: 3D periodic 256^3 grid, D3Q111 velocity set with the N=5
equilibrium, source = 64 periodic Gaussians (sigma 2 cells, centres from
SplitMix64 seed 0, charges alternating +-1, mean removed), tau_lb from Kn =
0.2.  Populations are stored as 64-bit fixed point with one power-of-two scale
per array (PKR_FX64: the density an exact integer sum, the equilibrium and
source terms in binary64; every stored value resolved to 2^-51 of the
largest, parity with the binary64 oracle <= 1e-12 at full size), 1784 bytes
per site update like binary64 storage.  On this GPU the binary64 storage
sweep is bound by the FP64 pipe (one FMA per velocity and site); its own
rate and roofline fraction ride on the same line (``other_storage``).  One
benchmark step = 32 sweeps followed by the binary64 relative-L2 residual
check (one pass of the whole hot path: pull, density, BGK relaxation, source,
store, residual).  The populations (2 x 14.9 GB) are far larger than L2, so
no flush is needed between steps.

``e2e``: the same metric for a complete solve to rel. residual 1e-10 through
``pkr_solve`` with host buffers (H2D of rho and D2H of Phi inside the timed
region).  ``cpu_baseline``: the oracle (serial C) on a 16-plane slab of the same
source; ``cpu_baseline_openmp``: the same source built with OpenMP on every host
core; ``cpu_full_solve``: the oracle's whole 2D 64^2 D2Q169 solve (serial and
OpenMP) beside the GPU's.  ``--impl reference`` times the serial oracle alone on
the same slab, as the reference arm.

Two more of the reference's metrics ride on the same line (single GPU only,
after the timed region; the headline value is the sweep's):
``time_to_1e8``: the exact fixed point by the FFT comparator, then the plain
binary64 solve (the e2e solve above) against the MIXED and MIXED_FX64 ladders,
each to rel. residual 1e-10, with each result's rel. L2 distance to the fixed
point (all ~7e-9); ``serving``: the serving trace (Poisson arrivals of 3D
solves, edges 32-256, tolerances 1e-6/1e-8/1e-10) at 200/s and at a
sub-capacity rate, with solves/s and p50/p99 latency.

Multi-GPU: the path does not shard (one grid per GPU, no collectives), so N
ranks run N independent replicas; value = all ranks' site updates / the
slowest rank's time.
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

SHAPE = (256, 256, 256)
LATTICE, ORDER, KN = "D3Q111", 5, 0.2
PRECISION = "fx64"   # 64-bit fixed-point storage, binary64-accurate (parity 1e-12)
TAU = 0.0            # > 0: tau_lb directly instead of the Knudsen number
SWEEPS_PER_STEP = 32
SLAB = 16            # planes of the CPU-baseline sample (the reference arm's step too)
METRIC = "GLUPS (site updates/s, 1e9) of the fused sweep"
WORKLOAD = "poisson3d_256cube_d3q111_n5_fx64_64gauss_sigma2_seed0_kn0.2"


def dist_env():
    from paper_1504_05869_gb300 import replicas
    return replicas.env()


def source():
    from paper_1504_05869_gb300.workloads import stiff_source
    rho, _ = stiff_source(SHAPE, count=64, sigma=2.0, seed=0)
    return rho


def configure(args):
    """Smaller or different cases (profiling, sweeps of sizes); the default is
    the headline workload."""
    global SHAPE, LATTICE, ORDER, PRECISION, WORKLOAD, TAU
    if args.size:
        SHAPE = (args.size,) * 3
    LATTICE, ORDER, PRECISION = args.lattice, args.order, args.precision
    if PRECISION in ("mixed", "mixed_fx64"):
        raise SystemExit("--precision mixed* applies to the batch and serve workloads")
    TAU = args.tau
    if (SHAPE, LATTICE, ORDER, PRECISION, TAU) != ((256, 256, 256), "D3Q111", 5, "fx64", 0.0):
        n = SHAPE[0]
        WORKLOAD = (f"poisson3d_{n}cube_{LATTICE.lower()}_n{ORDER}_{PRECISION}"
                    f"_64gauss_sigma2_seed0_" + (f"tau{TAU:g}" if TAU > 0 else "kn0.2"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources of the plan sweep kernels (the recorded traffic is void once they change)
KERNEL_SOURCES = ("pkr_sweep.cuh", "pkr_sweep_pair.cuh", "pkr_sweep_ws.cuh", "pkr_lattices.h",
                  "sweep_d3q111.cu")


def kernel_label(pk, variant):
    """Name of the sweep kernel a plan variant launches."""
    T = {"fp64": "double", "fx64": "long long"}.get(PRECISION, "float")
    if PRECISION == "fp16":
        return ("sweep_h16p_kernel" if variant == 1 else "sweep_h16_kernel") + f"<{LATTICE}>"
    nb = pk._pkr.pkr_batch_variant_count(pk.LATTICES[LATTICE])   # staged geometries
    nv = pk._pkr.pkr_variant_count(pk.LATTICES[LATTICE])
    if variant < nb:
        return f"sweep_staged_kernel<{LATTICE},{T}>"
    if nv - variant <= 2 and nv - nb == 3:
        form = "early refill" if variant == nv - 1 else "refill after the pair"
        return f"sweep_pair_kernel<{LATTICE},{T},G=2> ({form})"
    return f"sweep_ws_kernel<{LATTICE},{T}>"


def kernel_code_hash(texts):
    """sha256[:16] of the sweep sources with C/C++ comments and trailing
    blanks removed: a capture stays valid through comment edits and is void
    once any code changes."""
    import hashlib
    h = hashlib.sha256()
    for t in texts:
        out, i, n = [], 0, len(t)
        while i < n:
            c = t[i]
            if c in "\"'":                      # string or character literal
                j = i + 1
                while j < n and t[j] != c:
                    j += 2 if t[j] == "\\" else 1
                out.append(t[i:j + 1])
                i = j + 1
            elif t.startswith("//", i):
                j = t.find("\n", i)
                i = n if j < 0 else j
            elif t.startswith("/*", i):
                j = t.find("*/", i + 2)
                i = n if j < 0 else j + 2
            else:
                out.append(c)
                i += 1
        code = "\n".join(line.rstrip() for line in "".join(out).splitlines())
        h.update(code.encode())
    return h.hexdigest()[:16]


def recorded_traffic(variant):
    """DRAM bytes per sweep launch of the headline workload from the committed
    ncu summary, or None if the kernel code changed since it was taken or
    the run launched another variant than the one captured."""
    if (SHAPE, LATTICE, ORDER) != ((256, 256, 256), "D3Q111", 5) or \
            PRECISION not in ("fp64", "fx64"):
        return None
    csrc = os.path.join(ROOT, "paper_1504_05869_gb300", "csrc")
    code = kernel_code_hash(open(os.path.join(csrc, f), encoding="utf-8").read()
                            for f in KERNEL_SOURCES)
    try:
        txt = open(os.path.join(ROOT, "profiles",
                                f"sweep_d3q111_{PRECISION}_128cube_traffic.md")).read()
    except OSError:
        return None
    vals = dict(line.split(": ", 1) for line in txt.splitlines()
                if line.startswith(("traffic_bytes_per_launch_256cube", "code_sha256_16",
                                    "kernel_variant")))
    if vals.get("code_sha256_16", "").strip() != code:
        return None
    if vals.get("kernel_variant", "").strip() != str(variant):
        return None
    return float(vals["traffic_bytes_per_launch_256cube"])


def cpu_baseline(rho, tau):
    """The oracle (serial C, one core) on a 64-plane slab of the source."""
    import oracle
    slab = np.ascontiguousarray(rho[:SLAB])
    t0 = time.perf_counter()
    oracle.solve(slab, LATTICE, ORDER, tau_lb=tau, max_steps=1)
    dt = time.perf_counter() - t0
    return {"value": slab.size / dt / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
            "sample": f"1 step (source prep + collide/stream + density) on a "
                      f"{SLAB}x256x256 slab of the same source, serial C, {dt:.1f} s"}


def cpu_baseline_openmp(rho, tau):
    """The same oracle source built with OpenMP (the site loop of a step
    shared by z-plane; bitwise the serial result), on every host core, on
    the same slab: a second reported baseline."""
    import oracle
    try:
        cores = oracle.threads(len(os.sched_getaffinity(0)))
    except Exception as e:              # no OpenMP-capable compiler on this host
        return {"unavailable": f"OpenMP oracle build failed: {e}"[:200]}
    slab = np.ascontiguousarray(rho[:SLAB])
    oracle.solve(slab[:4], LATTICE, ORDER, tau_lb=tau, max_steps=1, openmp=True)   # warm-up
    t0 = time.perf_counter()
    oracle.solve(slab, LATTICE, ORDER, tau_lb=tau, max_steps=1, openmp=True)
    dt = time.perf_counter() - t0
    return {"value": slab.size / dt / 1e9, "unit": "GLUPS", "cores": cores,
            "kind": "oracle (OpenMP build)",
            "sample": f"1 step on the same {SLAB}x256x256 slab, {cores} threads, {dt:.2f} s"}


def cpu_full_solve(pk, torch):
    """A whole solve on the host's cores: the 2D 64^2 problem (D2Q169 N=7,
    rho = sin(2 pi x/64) sin(2 pi y/64), Kn 0.1, stop at max|dPhi| < 1e-12),
    serial and with the OpenMP build, beside the same solve on the GPU.  A
    reported baseline only."""
    import oracle
    from paper_1504_05869_gb300.workloads import sinusoid
    rho = sinusoid((64, 64))
    out = {"problem": "64^2 D2Q169 N=7, Kn 0.1, max|dPhi| < 1e-12 (every step)"}
    t0 = time.perf_counter()
    ref = oracle.solve(rho, "D2Q169", 7, knudsen=0.1, tol=1e-12, tol_kind=0, check_every=1,
                       max_steps=100000)
    out["serial"] = {"seconds": time.perf_counter() - t0, "steps": ref.steps, "cores": 1}
    try:
        cores = oracle.threads(len(os.sched_getaffinity(0)))
        t0 = time.perf_counter()
        ro = oracle.solve(rho, "D2Q169", 7, knudsen=0.1, tol=1e-12, tol_kind=0, check_every=1,
                          max_steps=100000, openmp=True)
        out["openmp"] = {"seconds": time.perf_counter() - t0, "steps": ro.steps, "cores": cores}
    except Exception as e:              # no OpenMP-capable compiler on this host
        out["openmp"] = {"unavailable": f"{e}"[:200]}
    r = torch.from_numpy(rho).cuda()
    phi = torch.empty_like(r)
    prob = pk.problem("D2Q169", (64, 64), 7, knudsen=0.1, tol=1e-12, tol_kind="max_abs",
                      check_every=1, max_sweeps=100000)
    pk.solve(r, phi, prob)               # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, st = pk.solve(r, phi, prob)
    torch.cuda.synchronize()
    out["gpu"] = {"seconds": time.perf_counter() - t0, "steps": st["sweeps"], "status": rc}
    return out


def time_to_1e8(pk, torch, r, stream, e2e_solve, e2e_phi):
    """Time to a solution within ~1e-8 (rel. L2) of the scheme's exact
    binary64 fixed point at 256^3: the FFT comparator gives the fixed point
    itself; plain binary64 storage, 64-bit fixed point (the e2e solve, host
    buffers) and the MIXED / MIXED_FX64 ladders (binary32 steps, then
    binary64 or 64-bit fixed point from the converted state) each run to rel.
    residual 1e-10 on device buffers."""
    ref = torch.empty_like(r)
    prob = pk.problem(LATTICE, SHAPE, ORDER, knudsen=KN)
    pk.fixed_point_fft(r, ref, prob)                 # warm-up (cuFFT plans)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pk.fixed_point_fft(r, ref, prob)
    torch.cuda.synchronize()
    out = {"fixed_point_fft_s": time.perf_counter() - t0}
    nref = torch.linalg.norm(ref).item()
    for prec in ("fp64", "mixed", "mixed_fx64"):
        phi = torch.empty_like(r)
        p = pk.problem(LATTICE, SHAPE, ORDER, knudsen=KN, tol=1e-10, tol_kind="rel_l2",
                       check_every=SWEEPS_PER_STEP, max_sweeps=200000, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, st = pk.solve(r, phi, p, stream=stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[prec] = {"seconds": dt, "sweeps": st["sweeps"], "status": rc,
                     "rel_l2_vs_fixed_point": torch.linalg.norm(phi - ref).item() / nref}
        del phi
    if PRECISION != "fp64":
        out[PRECISION] = {"seconds": e2e_solve["seconds"], "sweeps": e2e_solve["sweeps"],
                          "status": e2e_solve["status"], "host_buffers": True,
                          "rel_l2_vs_fixed_point":
                              torch.linalg.norm(e2e_phi - ref).item() / nref}
    t64 = out["fp64"]["seconds"]
    for k in list(out):
        if isinstance(out[k], dict) and k != "fp64":
            out[k]["speedup_vs_fp64"] = t64 / out[k]["seconds"]
    del ref
    torch.cuda.empty_cache()
    out["note"] = ("each run to rel. residual 1e-10 (device buffers; the "
                   f"{PRECISION} entry is the e2e solve, host copies included)")
    return out


def sweep_rate(pk, torch, r, precision, steps, stream, hbm_peak):
    """Autotuned sweep throughput of another storage mode on the same input
    (reported beside the headline): GLUPS, HBM GB/s and fraction of peak."""
    prob = pk.problem(LATTICE, SHAPE, ORDER, knudsen=KN, tol=0.0, check_every=SWEEPS_PER_STEP,
                      max_sweeps=10 ** 9, precision=precision)
    with torch.cuda.stream(stream):
        plan = pk.Plan(prob, stream=stream)
        plan.load_source(r)
    variant, _ = plan.autotune(2)
    plan.run(SWEEPS_PER_STEP)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.run(SWEEPS_PER_STEP)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.close()
    launch_ms = e0.elapsed_time(e1) / (steps * SWEEPS_PER_STEP)
    V = r.numel()
    es = {"fp64": 8, "fx64": 8, "fp32": 4, "fp16": 2}[precision]
    bs = 2 * 111 * es + (8 if precision in ("fp64", "fx64") else 4)
    gbs = V * bs / (launch_ms * 1e-3) / 1e9
    return {"glups": V / (launch_ms * 1e-3) / 1e9, "hbm_gbs": gbs, "frac": gbs / hbm_peak,
            "ms_per_sweep": launch_ms, "bytes_per_site": bs, "kernel_variant": variant,
            "steps": steps, "sweeps_per_step": SWEEPS_PER_STEP}


def run_reference(args):
    """Reference arm: the oracle timed on the host, each step one oracle step
    on the 16-plane slab of the benchmark's source that the GPU line's
    cpu_baseline times."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    rho = source()
    lat = oracle.lattice(LATTICE, ORDER)
    tau = oracle.tau_from_knudsen(KN, SHAPE[::-1], lat.cs2)
    slab = np.ascontiguousarray(rho[:SLAB])
    for _ in range(args.warmup):
        oracle.solve(slab, LATTICE, ORDER, tau_lb=tau, max_steps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(slab, LATTICE, ORDER, tau_lb=tau, max_steps=1)
    dt = time.perf_counter() - t0
    val = slab.size * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{SLAB}x256x256 slab, 1 step"},
            "cpu_baseline": {"value": val, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"one oracle step on a {SLAB}x256x256 slab per "
                                       "benchmark step (the slab of the GPU line's "
                                       "cpu_baseline)"},
            "e2e": {"value": val, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk

    rho = source()
    V = rho.size
    stream = torch.cuda.Stream()
    prob = pk.problem(LATTICE, SHAPE, ORDER, knudsen=KN, tau_lb=TAU, tol=0.0,
                      check_every=SWEEPS_PER_STEP, max_sweeps=10 ** 9, precision=PRECISION,
                      variant=args.variant)
    # tau_lb = 1 in binary64 runs the scalar stencil (Phi-only state)
    stencil = TAU == 1.0 and PRECISION == "fp64"
    r_dev = torch.from_numpy(rho).cuda()
    with torch.cuda.stream(stream):
        plan = pk.Plan(prob, stream=stream)
        plan.load_source(r_dev)
    Q = {"D3Q111": 111, "D3Q19": 19}[LATTICE]
    esize = {"fp64": 8, "fx64": 8, "fp32": 4, "fp16": 2}[PRECISION]
    tau = None

    def step():
        rc, st = plan.run(SWEEPS_PER_STEP)
        return st

    if args.variant >= 0:        # a fixed geometry (profiling); default: autotuned
        variant = args.variant
    else:
        variant, tuned_ms = plan.autotune(2)
    for _ in range(args.warmup):
        st = step()
    tau = st["tau_lb"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    dev_ms = ev0.elapsed_time(ev1)
    sweeps = args.steps * SWEEPS_PER_STEP
    from paper_1504_05869_gb300 import replicas
    dev_ms, total_updates = replicas.aggregate(dev_ms, float(V) * sweeps, device="cuda")
    if dist:
        dist.barrier()
    glups = total_updates / (dev_ms * 1e-3) / 1e9
    bytes_site = 2 * Q * esize + (8 if PRECISION in ("fp64", "fx64") else 4)
    if stencil:
        bytes_site = 24      # read Phi and the summed source, write Phi
    # kernels per timed step: each sweep, the array-exponent update that
    # follows every fixed-point and binary16 sweep, and one residual reduction
    # per check (one check per step)
    per_sweep = 2 if PRECISION in ("fx64", "fp16") and not stencil else 1
    launches_per_step = SWEEPS_PER_STEP * per_sweep + 1
    # per-launch: plain sweeps move 2*Q*8 + 8 bytes per site
    launch_ms = dev_ms / sweeps
    achieved = V * bytes_site / (launch_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    plan.close()

    # end to end: full solve to 1e-10 through pkr_solve with host buffers
    e2e = None
    if not args.no_e2e:
        rho_h = torch.from_numpy(rho).pin_memory()
        phi_h = torch.empty_like(rho_h).pin_memory()
        eprob = pk.problem(LATTICE, SHAPE, ORDER, knudsen=KN, tau_lb=TAU, tol=1e-10,
                           tol_kind="rel_l2",
                           check_every=SWEEPS_PER_STEP, max_sweeps=200000,
                           precision=PRECISION)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, est = pk.solve(rho_h.numpy(), phi_h.numpy(), eprob, stream=stream)
        torch.cuda.synchronize()
        e_s = time.perf_counter() - t0
        from paper_1504_05869_gb300 import replicas
        e_s, e_updates = replicas.aggregate(e_s, float(V) * est["launches"], device="cuda")
        e2e = {"value": e_updates / e_s / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": V * 8, "d2h_bytes_per_step": V * 8,
               "solve": {"sweeps": est["sweeps"], "residual": est["residual"],
                         "status": rc, "seconds": e_s, "tol": 1e-10}}

    # the reference's other two metrics, on one GPU, after the timed region
    t2e8 = serving = other = None
    if world == 1 and not args.no_extras and e2e is not None and TAU == 0.0 and \
            PRECISION in ("fp64", "fx64") and (LATTICE, ORDER, SHAPE) == ("D3Q111", 5, (256,) * 3):
        other_prec = "fp64" if PRECISION == "fx64" else "fx64"
        other = {other_prec: sweep_rate(pk, torch, r_dev, other_prec, 4, stream, hbm_peak)}
        t2e8 = time_to_1e8(pk, torch, r_dev, stream, e2e["solve"], phi_h.cuda())
        serving = {"overloaded": serve_trace(pk, args.serve_requests, 200.0, "mixed", 150.0),
                   "sub_capacity": serve_trace(pk, args.serve_sub_requests,
                                               args.serve_sub_rate, "mixed", 150.0)}

    cpu = cpu_omp = cpu_full = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(rho, tau)
        cpu_omp = cpu_baseline_openmp(rho, tau)
        cpu_full = cpu_full_solve(pk, torch)

    if stencil:
        # binary64 FMA bound: Q FMAs per site; peak from the GB300's nominal
        # FP64 rate (1.25 TFLOP/s = 625 G FMA/s)
        fma_s = V * Q / (launch_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": fma_s, "peak": 625.0, "unit": "GFMA/s",
                    "frac": fma_s / 625.0, "traffic": None, "peak_source": "nominal FP64",
                    "kernel": f"stencil_kernel<{LATTICE}>", "hbm_gbs": achieved,
                    "algorithmic_bytes_per_launch": V * bytes_site}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                    "unit": "GB/s", "frac": achieved / hbm_peak,
                    "traffic": recorded_traffic(variant), "peak_source": peak_src,
                    "kernel": kernel_label(pk, variant),
                    "algorithmic_bytes_per_launch": V * bytes_site}
    if rank == 0:
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fx64": "int64 (fixed point)", "fp32": "f32",
                      "fp16": "f16"}[PRECISION], "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(SHAPE), "lattice": LATTICE,
                       "order": ORDER, "knudsen": None if TAU > 0 else KN, "tau_lb": tau,
                       "sweeps_per_step": SWEEPS_PER_STEP, "residual_check": "rel_l2 fp64",
                       "kernel_variant": variant,
                       "l2": (f"inputs larger than L2 (2 x {Q * V * esize / 1e9:.2f} GB populations)"
                              if Q * V * esize > 129e6 else
                              f"populations ({2 * Q * V * esize / 1e6:.0f} MB) fit in L2"),
                       "parallelism": f"replicas x{world}"},
            "hbm_gbs": V * bytes_site * sweeps * world / (dev_ms * 1e-3) / 1e9,
            "roofline": roofline,
            "cpu_baseline": cpu, "cpu_baseline_openmp": cpu_omp, "cpu_full_solve": cpu_full,
            "other_storage": other, "e2e": e2e, "time_to_1e8": t2e8, "serving": serving,
            "clocks": clocks, "gpu_launches": args.steps * launches_per_step,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Other workloads (one JSON line each; the default run is the sweep above)
# ---------------------------------------------------------------------------
def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def run_batch(args):
    """256 independent periodic 3D grids, edges log-uniform in [32, 128]
    (seed 2), 1-16 Gaussians (sigma 1-4), D3Q111 N=5, Kn 0.2 per grid, all
    advanced by the batch engine (one persistent launch per step, K-step
    graphs, geometry from the autotuner) until each retires."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    from paper_1504_05869_gb300.workloads import batch_jobs
    jobs = batch_jobs(args.batch_count, seed=2)
    tol = args.tol if args.tol > 0 else (1e-7 if args.precision == "fp32" else 1e-8)
    rhos = [torch.from_numpy(j.rho()).cuda() for j in jobs]
    phis = [torch.zeros_like(r) for r in rhos]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    ctx = pk.Context("D3Q111", 5, precision=args.precision, check_every=SWEEPS_PER_STEP,
                     hbm_budget_bytes=int(args.budget_gb * 1e9), variant=-2, probe_edge=64,
                     stream=stream)
    t0 = time.perf_counter()
    tickets = [ctx.submit(r, p, knudsen=KN, tol=tol, tol_kind="rel_l2", max_sweeps=50000)
               for r, p in zip(rhos, phis)]
    ctx.run()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    info = ctx.info()
    stats = [ctx.poll(t) for t in tickets]
    ctx.close()
    ok = sum(1 for rc, _ in stats if rc == 0)
    sweeps = [st["sweeps"] for rc, st in stats if st]
    sites = sum(r.numel() for r in rhos)
    # distance of the first grids' results to their exact fixed points (FFT comparator)
    errs = []
    for j, r, p in list(zip(jobs, rhos, phis))[:16]:
        fx = torch.empty_like(r)
        pk.fixed_point_fft(r, fx, pk.problem("D3Q111", r.shape, 5, knudsen=KN))
        errs.append(torch.linalg.norm(p - fx).item() / torch.linalg.norm(fx).item())
    line = {"metric": "batched solves: GLUPS over all grids and solves/s", "workload": "batch",
            "value": info["site_updates"] / dt / 1e9, "unit": "GLUPS",
            "solves_per_s": ok / dt, "solves": len(jobs), "converged": ok, "seconds": dt,
            "sites_total": sites, "site_updates": info["site_updates"],
            "sweeps_min_median_max": [min(sweeps), _pct(sweeps, 50), max(sweeps)],
            "precision": args.precision, "tol_rel_l2": tol, "kernel_variant": info["variant"],
            "rel_l2_vs_fixed_point_first16": {"median": _pct(errs, 50), "max": max(errs)},
            "windows": info["windows"], "check_every": SWEEPS_PER_STEP,
            "hbm_budget_gb": args.budget_gb, "data": "synthetic",
            "config": {"grids": len(jobs), "edges": "log-uniform [32,128], seed 2",
                       "lattice": "D3Q111", "order": 5, "knudsen": KN}}
    print(json.dumps(line), flush=True)
    return 0


def serve_trace(pk, count, rate, precision, budget_gb):
    """Serve the first `count` requests of the seed-3 arrival trace at `rate`
    per second through a threaded context (continuous batching under an HBM
    budget; requests are submitted at their arrival times, host-side inputs
    prepared beforehand).  Latency = completion - submission."""
    import threading as th
    import torch
    from paper_1504_05869_gb300.workloads import serving_trace
    trace = serving_trace(count, rate_hz=rate, seed=3)
    rhos = [torch.from_numpy(rq.rho()).cuda() for rq in trace]
    phis = [torch.zeros_like(r) for r in rhos]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    ctx = pk.Context("D3Q111", 5, precision=precision, check_every=SWEEPS_PER_STEP,
                     hbm_budget_bytes=int(budget_gb * 1e9), variant=-1, threaded=True,
                     stream=stream)
    tickets = [None] * len(trace)
    t0 = time.perf_counter()

    def feeder():
        for k, rq in enumerate(trace):
            delay = rq.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = ctx.submit(rhos[k], phis[k], knudsen=KN, tol=rq.tol,
                                    tol_kind="rel_l2", max_sweeps=50000)

    f = th.Thread(target=feeder)
    f.start()
    f.join()
    lat, sw, rcs = [], [], []
    for t in tickets:
        rc, st = ctx.wait(t)
        rcs.append(rc)
        lat.append(st["wall_ms"] / 1e3)
        sw.append(st["sweeps"])
        ctx.release(t)
    dt = time.perf_counter() - t0
    info = ctx.info()
    ctx.close()
    del rhos, phis
    torch.cuda.empty_cache()
    offered = len(trace) / max(trace[-1].arrival_s, 1e-9)
    return {"solves_per_s": len(trace) / dt, "p50_latency_s": _pct(lat, 50),
            "p99_latency_s": _pct(lat, 99), "max_latency_s": max(lat),
            "offered_rate_hz": offered, "requests": len(trace), "seconds": dt,
            "ok": sum(1 for r in rcs if r == 0), "statuses": sorted(set(rcs)),
            "glups": info["site_updates"] / dt / 1e9, "precision": precision,
            "sweeps_median": _pct(sw, 50), "hbm_budget_gb": budget_gb,
            "trace": f"first {len(trace)} arrivals of the seed-3 Poisson trace at {rate:g}/s"}


def run_serve(args):
    """Poisson arrivals (seed 3) of periodic 3D solves, edges log-uniform in
    [32, 256], tolerances from {1e-6, 1e-8, 1e-10}, smooth/stiff mix,
    continuous batching under an HBM budget; latency = completion - arrival."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    r = serve_trace(pk, args.requests, args.rate, args.precision, args.budget_gb)
    line = {"metric": "served solves/s with p50/p99 latency", "workload": "serve",
            "value": r["solves_per_s"], "unit": "solves/s", **r,
            "check_every": SWEEPS_PER_STEP, "data": "synthetic",
            "config": {"arrivals": f"Poisson {args.rate}/s, seed 3", "edges": "[32,256]",
                       "tols": [1e-6, 1e-8, 1e-10], "lattice": "D3Q111", "knudsen": KN}}
    print(json.dumps(line), flush=True)
    return 0


def run_poisson2d(args):
    """64x64 periodic, rho = sin(2 pi x/64) sin(2 pi y/64), D2Q169 N=7, Kn 0.1,
    stop at max |dPhi| < 1e-12; also at the paper's tau_lb = 1."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    from paper_1504_05869_gb300.workloads import sinusoid
    rho = sinusoid((64, 64))
    k = 2 * np.pi / 64
    exact = rho / (2 * k * k)
    out = {}
    for label, kw in (("kn0.1", {"knudsen": 0.1}), ("tau1", {"tau_lb": 1.0})):
        r = torch.from_numpy(rho).cuda()
        phi = torch.empty_like(r)
        prob = pk.problem("D2Q169", (64, 64), 7, tol=1e-12, tol_kind="max_abs", check_every=1,
                          max_sweeps=100000, **kw)
        pk.solve(r, phi, prob)   # warm-up (module load, first launches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = pk.solve(r, phi, prob)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        got = phi.cpu().numpy()
        fx = torch.empty_like(r)
        pk.fixed_point_fft(r, fx, prob)
        fx = fx.cpu().numpy()
        out[label] = {"status": rc, "sweeps": st["sweeps"], "seconds": dt,
                      "glups": 4096 * st["launches"] / dt / 1e9, "tau_lb": st["tau_lb"],
                      "rel_l2_vs_analytic": float(np.linalg.norm(got - exact) /
                                                  np.linalg.norm(exact)),
                      "rel_l2_vs_scheme_fixed_point": float(np.linalg.norm(got - fx) /
                                                            np.linalg.norm(fx)),
                      "fixed_point_vs_analytic": float(np.linalg.norm(fx - exact) /
                                                       np.linalg.norm(exact))}
    cpu = None
    if not args.no_cpu:
        # the oracle's full solve of the same problem (Kn 0.1), serial C, one core
        import oracle
        t0 = time.perf_counter()
        ref = oracle.solve(rho, "D2Q169", 7, knudsen=0.1, tol=1e-12, tol_kind=0,
                           check_every=1, max_steps=100000)
        dt = time.perf_counter() - t0
        cpu = {"value": dt, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"the whole Kn 0.1 solve ({ref.steps} steps), serial C",
               "same_steps_as_gpu": ref.steps == out["kn0.1"]["sweeps"]}
    line = {"metric": "time to max|dPhi| < 1e-12, 2D 64^2 D2Q169 N=7", "workload": "poisson2d",
            "value": out["kn0.1"]["seconds"], "unit": "s", "higher_is_better": False,
            "runs": out, "cpu_baseline": cpu, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Storage precision: (1) sweep throughput of binary64 and binary32
    storage at 512^3 (256 Gaussians, sigma 1.5, seed 1); (2) time to a
    solution within 1e-8 (rel L2) of the binary64 fixed point at 256^3
    (64 Gaussians, sigma 2, seed 0, Kn 0.2): plain binary64 vs the mixed
    ladder (binary32 steps, then binary64 from the converted state) vs
    binary32 alone, each result's error against the exact fixed point from
    the FFT comparator (whose own time is reported as the direct solve)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    from paper_1504_05869_gb300.workloads import stiff_source
    out = {"throughput_512": {}, "time_to_1e-8_256": {}}
    if not args.no_512:
        rho, _ = stiff_source((512, 512, 512), count=256, sigma=1.5, seed=1)
        r = torch.from_numpy(rho).cuda()
        del rho
        for prec in ("fp16", "fp32", "fp64", "fx64"):
            stream = torch.cuda.Stream()
            prob = pk.problem("D3Q111", r.shape, 5, knudsen=KN, max_sweeps=10 ** 6,
                              precision=prec)
            with pk.Plan(prob, stream=stream) as P:
                P.load_source(r)
                P.sweeps(2)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.sweeps(8)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 8
            es = {"fp64": 8, "fx64": 8, "fp32": 4, "fp16": 2}[prec]
            ss = 8 if prec in ("fp64", "fx64") else 4
            out["throughput_512"][prec] = {"ms_per_sweep": ms, "glups": r.numel() / ms / 1e6,
                                           "gbs": r.numel() * (2 * 111 * es + ss) / ms / 1e6,
                                           "bytes_per_site": 2 * 111 * es + ss}
            torch.cuda.empty_cache()
        if args.solve_512:
            # each storage solved to its tolerance at 512^3, against the exact
            # binary64 fixed point; the ladders hand their state on with one
            # spare array at a time (peak 238 GB, the binary64 tail's two arrays)
            ref = torch.empty_like(r)
            prob = pk.problem("D3Q111", r.shape, 5, knudsen=KN)
            fst = pk.fixed_point_fft(r, ref, prob)
            nref = torch.linalg.norm(ref).item()
            out["solve_512"] = {"fixed_point_seconds": fst["wall_ms"] / 1e3}
            for prec, tol in (("fp16", 1e-3), ("fp32", 1e-7), ("fp64", 1e-10),
                              ("fx64", 1e-10), ("mixed", 1e-10), ("mixed_fx64", 1e-10)):
                phi = torch.empty_like(r)
                prob = pk.problem("D3Q111", r.shape, 5, knudsen=KN, tol=tol, tol_kind="rel_l2",
                                  check_every=SWEEPS_PER_STEP, max_sweeps=200000,
                                  precision=prec)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, st = pk.solve(r, phi, prob)
                torch.cuda.synchronize()
                out["solve_512"][prec] = {
                    "seconds": time.perf_counter() - t0, "sweeps": st["sweeps"], "status": rc,
                    "tol": tol, "rel_l2_vs_fp64_fixed_point":
                        torch.linalg.norm(phi - ref).item() / nref}
                del phi
                torch.cuda.empty_cache()
            del ref
        del r
        torch.cuda.empty_cache()
    rho, _ = stiff_source(SHAPE, count=64, sigma=2.0, seed=0)
    r = torch.from_numpy(rho).cuda()

    def solve(prec, tol):
        phi = torch.empty_like(r)
        prob = pk.problem("D3Q111", SHAPE, 5, knudsen=KN, tol=tol, tol_kind="rel_l2",
                          check_every=SWEEPS_PER_STEP, max_sweeps=200000, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = pk.solve(r, phi, prob)
        torch.cuda.synchronize()
        return phi, rc, st, time.perf_counter() - t0

    # the exact binary64 fixed point, by the FFT comparator (direct solver)
    ref = torch.empty_like(r)
    prob = pk.problem("D3Q111", SHAPE, 5, knudsen=KN)
    pk.fixed_point_fft(r, ref, prob)                 # warm-up (loads cuFFT kernels)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = pk.fixed_point_fft(r, ref, prob)
    torch.cuda.synchronize()
    out["reference"] = {"method": "pkr_fixed_point_fft (exact fixed point, binary64)",
                        "seconds": time.perf_counter() - t0, "library_wall_ms": st["wall_ms"]}
    nref = torch.linalg.norm(ref).item()
    for label, prec, tol in (("fp64", "fp64", args.target_tol), ("mixed", "mixed", args.target_tol),
                             ("mixed16", "mixed16", args.target_tol),
                             ("mixed_fx64", "mixed_fx64", args.target_tol),
                             ("fx64", "fx64", args.target_tol), ("fp32", "fp32", 1e-7),
                             ("fp16", "fp16", 1e-3)):
        phi, rc, st, dt = solve(prec, tol)
        err = (torch.linalg.norm(phi - ref).item() / nref)
        out["time_to_1e-8_256"][label] = {"seconds": dt, "sweeps": st["sweeps"],
                                          "launches": st["launches"], "status": rc,
                                          "tol": tol, "rel_l2_vs_fp64_fixed_point": err}
    t64 = out["time_to_1e-8_256"]["fp64"]["seconds"]
    tmx = min(out["time_to_1e-8_256"][m]["seconds"] for m in ("mixed", "mixed16", "mixed_fx64"))
    line = {"metric": "time to rel L2 1e-8 of the binary64 fixed point, mixed vs plain binary64",
            "workload": "precision", "value": tmx, "unit": "s", "higher_is_better": False,
            "plain_fp64_s": t64, "speedup_vs_plain_fp64": t64 / tmx, **out,
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_knudsen(args):
    """The 256^3 stiff-source problem (64 Gaussians, sigma 2, seed 0) solved
    in binary64 to rel. L2 residual 1e-10 at Kn 0.05, 0.2 and 0.5, with the
    N=5 3D set and with standard first-order LB (D3Q19, N=1).  Each run
    reports its sweeps, wall time and GLUPS, its distance to the scheme's
    exact fixed point (FFT comparator) and that fixed point's distance to
    the continuum periodic Poisson solution (spectral, reported only)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    rho = source()
    r = torch.from_numpy(rho).cuda()
    # continuum: Phi(k) = rho(k) / |k|^2 (eps = 1), Phi(0) = 0
    ks = [2 * np.pi * torch.fft.fftfreq(n, device="cuda", dtype=torch.float64) for n in SHAPE]
    k2 = ks[0][:, None, None] ** 2 + ks[1][None, :, None] ** 2 + ks[2][None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    rk = torch.fft.fftn(r - r.mean()) / k2
    rk[0, 0, 0] = 0.0
    cont = torch.fft.ifftn(rk).real
    del rk, k2
    ncont = torch.linalg.norm(cont).item()
    out = {}
    for lattice, order in (() if args.skip_kn else (("D3Q111", 5), ("D3Q19", 1))):
        stream = torch.cuda.Stream()
        with pk.Plan(pk.problem(lattice, SHAPE, order, knudsen=0.2, max_sweeps=10 ** 6),
                     stream=stream) as P:
            P.load_source(r)
            variant, _ = P.autotune(4)
        torch.cuda.empty_cache()
        for kn in (0.05, 0.2, 0.5):
            prob = pk.problem(lattice, SHAPE, order, knudsen=kn, tol=1e-10, tol_kind="rel_l2",
                              check_every=SWEEPS_PER_STEP, max_sweeps=200000, variant=variant)
            phi = torch.empty_like(r)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = pk.solve(r, phi, prob)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            fx = torch.empty_like(r)
            fst = pk.fixed_point_fft(r, fx, prob)
            nfx = torch.linalg.norm(fx).item()
            out[f"{lattice}_kn{kn}"] = {
                "status": rc, "tau_lb": st["tau_lb"], "sweeps": st["sweeps"], "seconds": dt,
                "glups": r.numel() * st["launches"] / dt / 1e9, "variant": variant,
                "rel_l2_vs_scheme_fixed_point": torch.linalg.norm(phi - fx).item() / nfx,
                "fixed_point_seconds": fst["wall_ms"] / 1e3,
                "fixed_point_vs_continuum": torch.linalg.norm(fx - cont).item() / ncont}
            del phi, fx
            torch.cuda.empty_cache()
    # The paper's own setting, tau_lb = 1 (both sets run the scalar stencil):
    # time for the iterate to come within eps (rel. L2) of the continuum
    # solution, for a ladder of eps, next to the fixed point's own distance.
    targets = (1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5)
    tau1 = {}
    buf = torch.empty_like(r)
    for lattice, order in (("D3Q111", 5), ("D3Q19", 1)):
        prob = pk.problem(lattice, SHAPE, order, tau_lb=1.0, max_sweeps=10 ** 9)
        fx = torch.empty_like(r)
        pk.fixed_point_fft(r, fx, prob)
        fp_err = torch.linalg.norm(fx - cont).item() / ncont
        del fx
        hits, steps, secs, err = {}, 0, 0.0, None
        stream = torch.cuda.Stream()
        with pk.Plan(prob, stream=stream) as P:
            P.load_source(r)
            chunk = 256
            while secs < args.tau1_budget_s:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P.run(chunk)
                torch.cuda.synchronize()
                secs += time.perf_counter() - t0
                steps += chunk
                P.phi(buf)
                err = torch.linalg.norm(buf - cont).item() / ncont
                for eps in targets:
                    if eps not in hits and err <= eps:
                        hits[eps] = {"sweeps": steps, "seconds": secs}
                # stop once every target the fixed point allows has been met
                if all(e in hits for e in targets if e > 1.05 * fp_err):
                    break
        tau1[f"{lattice}_tau1"] = {"fixed_point_vs_continuum": fp_err,
                                   "time_to_eps_vs_continuum": {f"{e:g}": v for e, v in hits.items()},
                                   "sweeps_run": steps, "seconds_run": secs,
                                   "final_vs_continuum": err,
                                   "glups": r.numel() * steps / secs / 1e9}
    out.update(tau1)
    line = {"metric": "binary64 solve to rel. L2 residual 1e-10 at 256^3, Kn 0.05/0.2/0.5",
            "workload": "knudsen", "value": out.get("D3Q111_kn0.2", {}).get("seconds"), "unit": "s",
            "higher_is_better": False, "runs": out, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_paper1d(args):
    """The paper's 1D experiments on the GPU (Sec. "Computational
    performance", Table 2): rho = sin(2 pi x / L), tau_lb = 1, converged to a
    rel. residual of 1e-14 (checked every step, on the device); per-node error
    against the analytic solution next to the printed Table 2 values, the
    orders of convergence, and the L = 100 step counts next to the paper's."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk

    def rows(name):
        out = []
        for line in open(os.path.join(ROOT, "tests", "golden", name)):
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
        return out

    lat_for = {1: "D1Q5", 3: "D1Q5", 5: "D1Q9", 7: "D1Q13"}

    def solve(N, L, tol, l=1):
        x = np.arange(L)
        k = 2 * np.pi * l / L
        rho = np.sin(k * x)
        prob = pk.problem(lat_for[N], (L,), N, tau_lb=1.0, tol=tol, tol_kind="rel_l2",
                          check_every=1, max_sweeps=10 ** 6)
        r = torch.from_numpy(rho).cuda()
        phi = torch.empty_like(r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = pk.solve(r, phi, prob)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        exact = rho / k ** 2
        err = float(np.abs(phi.cpu().numpy() - exact).max() / np.abs(exact).max())
        return err, st["sweeps"], dt, rc

    table = []
    for L, N, printed in rows("table2_per_node_error.txt"):
        err, sw, dt, rc = solve(int(N), int(L), 1e-14)
        table.append({"L": int(L), "N": int(N), "error": err, "paper": float(printed),
                      "sweeps": sw, "seconds": dt, "status": rc})
    orders = {}
    for N in (3, 5, 7):
        e32 = solve(N, 32, 1e-14)[0]
        e64 = solve(N, 64, 1e-14)[0]
        orders[N] = float(np.log2(e32 / e64))
    # Fig. 5: error and steps against L for every N, with the fits
    # error = a_N L^-alpha_N and steps = b_N L^2 (least squares in log space)
    fig5 = {}
    for N in (1, 3, 5, 7):
        Ls = [8, 16, 32, 64, 128]
        res = [solve(N, L, 1e-14) for L in Ls]
        lL = np.log(np.array(Ls, dtype=float))
        alpha, loga = np.polyfit(lL, np.log([r[0] for r in res]), 1)
        b = float(np.exp(np.mean(np.log([r[1] for r in res]) - 2 * lL)))
        fig5[N] = {"L": Ls, "error": [r[0] for r in res], "sweeps": [r[1] for r in res],
                   "alpha": float(-alpha), "a": float(np.exp(loga)), "b_steps_per_L2": b}
    # Figs. 1-4: the l = 1 and l = 4 sources at L = 128, 32 and 8
    figs = {}
    for l, L in ((1, 128), (4, 128), (4, 32), (1, 8)):
        figs[f"l{l}_L{L}"] = {N: solve(N, L, 1e-14, l)[0] for N in (1, 3, 5, 7)}
    steps = {}
    paper_steps = {int(r[0]): int(r[2]) for r in rows("steps_L100.txt")}
    for N in (1, 3, 5, 7):
        err, sw, dt, rc = solve(N, 100, 1e-13)
        steps[N] = {"sweeps": sw, "paper": paper_steps[N], "seconds": dt, "error": err}
    line = {"metric": "the paper's 1D experiments on the GPU (Table 2, orders, L=100 steps)",
            "workload": "paper1d", "value": sum(r["seconds"] for r in table), "unit": "s",
            "higher_is_better": False, "table2": table, "orders_L32_L64": orders,
            "fig5": fig5, "figs_1_to_4_error": figs,
            "steps_L100_rel_residual_1e-13": steps, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_tau1(args):
    """The paper's setting tau_lb = 1 (D3Q111 N=5): the scalar-stencil path
    against the population sweep, per step at 256^3 (64 Gaussians) and for a
    whole solve to relative residual 1e-10 at 64^3 (same source statistics;
    at tau_lb = 1 the slowest mode needs ~L^2 steps, 67k at 256^3)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    from paper_1504_05869_gb300.workloads import stiff_source
    rho = source()
    r = torch.from_numpy(rho).cuda()
    r64 = torch.from_numpy(stiff_source((64, 64, 64), count=16, sigma=2.0, seed=0)[0]).cuda()
    out = {}
    for label, var in (("stencil", -1), ("population", 2)):
        stream = torch.cuda.Stream()
        prob = pk.problem("D3Q111", SHAPE, 5, tau_lb=1.0, max_sweeps=10 ** 6, variant=var)
        with pk.Plan(prob, stream=stream) as P:
            P.load_source(r)
            P.sweeps(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.sweeps(20)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
        phi = torch.empty_like(r64)
        prob = pk.problem("D3Q111", r64.shape, 5, tau_lb=1.0, tol=1e-10, tol_kind="rel_l2",
                          check_every=SWEEPS_PER_STEP, max_sweeps=10 ** 6, variant=var)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, st = pk.solve(r64, phi, prob, stream=stream)
        torch.cuda.synchronize()
        out[label] = {"ms_per_step": ms, "glups": r.numel() / ms / 1e6,
                      "solve_seconds": time.perf_counter() - t0, "sweeps": st["sweeps"],
                      "status": rc, "phi": phi}
    d = (torch.linalg.norm(out["stencil"]["phi"] - out["population"]["phi"]) /
         torch.linalg.norm(out["population"]["phi"])).item()
    for v in out.values():
        v.pop("phi")
    line = {"metric": "tau_lb = 1 solve time, scalar stencil vs population sweep",
            "workload": "tau1", "value": out["stencil"]["solve_seconds"], "unit": "s",
            "higher_is_better": False, "runs": out, "rel_l2_between_paths": d,
            "stencil_bytes_per_site": 24, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_pull_ceiling(args):
    """Memory ceiling of the sweep's access pattern at 256^3 (pkr_pull_copy_
    ceiling): the bytes of one D3Q111 sweep moved with no arithmetic, through
    the staged sweep's staging with the pull offsets kept per axis, through
    aligned x pairs, and through the x-pairs sweep's own staging, for 8- and
    4-byte populations; beside D3Q19's."""
    import ctypes
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
    n = (ctypes.c_int64 * 3)(*SHAPE)
    out = {}
    for lattice in ("D3Q111", "D3Q19"):
        for elem in (8, 4):
            for axes, label in ((0, "none"), (2, "yz"), (1, "x"), (3, "xyz"),
                                (7, "xyz_aligned_pairs"), (8, "xyz_pair_sweep_staging")):
                g = ctypes.c_double()
                rc = pk._pkr.pkr_pull_copy_ceiling(pk.LATTICES[lattice], n, elem, axes, 5,
                                                   ctypes.byref(g), None)
                out[f"{lattice}_{elem}B_shift_{label}"] = (
                    {"gbs": g.value, "frac_of_copy_peak": g.value / peak} if rc == 0
                    else {"status": rc})
    torch.cuda.synchronize()
    line = {"metric": "GB/s of the sweep's access pattern without arithmetic",
            "workload": "pull-ceiling", "value": out["D3Q111_8B_shift_xyz"].get("gbs"),
            "unit": "GB/s", "copy_peak_gbs": peak, "runs": out,
            "config": {"grid": list(SHAPE), "staging": "per-lane cp.async, 32-site tiles, "
                       "2 velocity groups x 2 tiles per block"}, "data": "synthetic (zeros)"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pkr", choices=["pkr", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-1e-8 and serving objects of the default line")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="default line: arrivals of the 200/s serving trace")
    ap.add_argument("--serve-sub-requests", type=int, default=100)
    ap.add_argument("--serve-sub-rate", type=float, default=2.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--size", type=int, default=0, help="cube edge (default 256)")
    ap.add_argument("--lattice", default="D3Q111", choices=["D3Q111", "D3Q19"])
    ap.add_argument("--order", type=int, default=5)
    ap.add_argument("--precision", default="fx64",
                    choices=["fp64", "fp32", "fp16", "fx64", "mixed", "mixed_fx64"],
                    help="sweep workload: fp64/fp32/fp16/fx64; batch/serve: "
                         "fp64/fp32/fx64/mixed/mixed_fx64")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "batch", "serve", "poisson2d", "precision", "tau1",
                             "knudsen", "paper1d", "pull-ceiling"])
    ap.add_argument("--no-512", action="store_true")
    ap.add_argument("--solve-512", action="store_true",
                    help="precision workload: also solve at 512^3 against the FFT fixed point")
    ap.add_argument("--target-tol", type=float, default=1e-10)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--variant", type=int, default=-1,
                    help="sweep workload: a fixed kernel geometry instead of the autotuned one")
    ap.add_argument("--tau1-budget-s", type=float, default=90.0,
                    help="knudsen workload: GPU seconds per lattice for the tau_lb = 1 runs")
    ap.add_argument("--skip-kn", action="store_true",
                    help="knudsen workload: only the tau_lb = 1 runs")
    ap.add_argument("--tau", type=float, default=0.0,
                    help="sweep workload: tau_lb instead of Kn 0.2 (1.0 in fp64: the stencil)")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "poisson2d":
        return run_poisson2d(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "tau1":
        return run_tau1(args)
    if args.workload == "knudsen":
        return run_knudsen(args)
    if args.workload == "paper1d":
        return run_paper1d(args)
    if args.workload == "pull-ceiling":
        return run_pull_ceiling(args)
    configure(args)
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
