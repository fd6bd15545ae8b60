#!/usr/bin/env python3
"""Throughput of the 25-point acoustic leapfrog on one GB300.

Workload (default): Algorithm 1 on a 512^3 interior (halo 4), FP32,
radius-4 8th-order star Laplacian, layered velocity 1500-4500 m/s with 16
seeded Gaussian perturbations, h = 10 m, dt at CFL 0.4, 15 Hz Ricker source
at depth 20.  One benchmark "step" = one propagation call of 100 leapfrog
steps over the whole grid.  Fields (3 x 562 MB) are larger than L2, so no
flush is needed between steps.

The default path is wave_propagate_tb: pairs of steps fused in one launch
(2-step temporal blocking, 20 algorithmic bytes per point per pair);
--path single times wave_propagate (one launch per step, 16 bytes per point
update).  Both compute the same fields (to FP32 rounding).

Prints ONE JSON line (rank 0) with Gpoint-updates/s for the whole job, the
roofline of the dominant kernel (HBM bound), an end-to-end number through
host buffers, the FP64 oracle timed on the host cores, SM clocks sampled
during the timed region, and the number of kernel launches.  The
single-step path is reported beside it (forms.single_step).  Extra forms
(--forms) measure the other rows: 16-bit storage, the radius sweep, errors
against the FP64 oracle, the 1024^3 precision grid, the absorbing layer,
batches of shots, the adjoint gradient and the Table 4 suite.  The oracle
runs only where a number is measured against it: the cpu_baseline objects
(the headline's, the batched form's and the adjoint form's: the oracle timed
on the host cores on a bounded sample), the accuracy forms (errors against
the FP64 oracle) and --impl reference, which times the FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gpoint-updates/s & % HBM roofline, 25-pt 512^3; BF16/batched vs plain FP32"
UNIT = "Gpoint-updates/s"
BYTES_PER_POINT = 16          # read u, u_prev, vel; write u_next (FP32)
BYTES_PER_POINT_PAIR = 20     # two fused steps: read u^t, u^{t-1}, vel; write u^{t+1}, u^{t+2}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0      # GB300 HBM3e nominal bandwidth (context; the measured copy peak is the basis)
CSRC = os.path.join(ROOT, "paper_2309_04671_gb300", "csrc")
# committed ncu DRAM counts per launch, valid while the kernel sources hash the same
TRAFFIC = {
    "single": (os.path.join(ROOT, "profiles", "k_tma_wave_512_traffic.json"),
               [os.path.join(CSRC, f) for f in ("k_tma.cu", "gbs_internal.cuh")]),
    "tb": (os.path.join(ROOT, "profiles", "k_wf_pair_512_traffic.json"),
           [os.path.join(CSRC, f) for f in ("k_wf.cu", "gbs_wf.cuh", "gbs_internal.cuh")]),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="interior side")
    ap.add_argument("--nz", type=int, default=0, help="interior z extent (default: n; smaller for profiling runs)")
    ap.add_argument("--nsteps", type=int, default=100, help="leapfrog steps per benchmark step")
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--path", choices=["tb", "single"], default="tb",
                    help="FP32 propagation: fused pairs of steps (tb) or one launch per step (single)")
    ap.add_argument("--time-block", type=int, choices=[2, 3], default=2,
                    help="tb path: steps fused per launch (3 needs 64 x 16 tiles to fit the SMs)")
    ap.add_argument("--graph", action="store_true", help="replay the step loop as a CUDA graph")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32",
                    help="wave-field storage of the main timed path (arithmetic is FP32 in all)")
    ap.add_argument("--forms", default="single,storage,radius,errors,precision,absorb,pml,batched,adjoint,suite,tblock",
                    help="comma list of extra forms to measure after the main line, or 'none'")
    ap.add_argument("--no-forms", action="store_true", help="same as --forms none")
    ap.add_argument("--adj-n", type=int, default=256, help="adjoint form: interior side")
    ap.add_argument("--adj-steps", type=int, default=1000, help="adjoint form: time steps")
    ap.add_argument("--adj-shots", type=int, default=8, help="adjoint form: shots")
    ap.add_argument("--adj-no-fused", action="store_true",
                    help="adjoint form: skip timing the one-launch backward step (for profiling runs)")
    ap.add_argument("--batch-shots", type=int, default=64, help="batched form: shots")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--ref-leapfrog", type=int, default=16, help="oracle leapfrog steps per reference step")
    return ap.parse_args()


def workload_desc(n, nsteps, nz=None):
    size = f"{n}^3" if nz in (None, n) else f"{n}x{n}x{nz}"
    return (f"wave_propagate {size} interior + halo 4, FP32, 25-pt radius-4 8th-order Laplacian, "
            f"{nsteps} leapfrog steps per step, layered 1500-4500 m/s + 16 Gaussians, h=10 m, CFL 0.4, "
            f"15 Hz Ricker at depth 20")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        self.windows = []

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        lo = min(w[0] for w in self.windows) - 1.0 if self.windows else -1e18
        hi = max(w[1] for w in self.windows) + 1.0 if self.windows else 1e18
        sel = [r for r in rows if lo <= r[0] <= hi] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in sel for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
                "reasons": reasons, "samples": len(sel)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_sha(path="single"):
    h = hashlib.sha256()
    for p in TRAFFIC[path][1]:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(n, path="single"):
    """DRAM bytes per launch from the committed ncu summary, if it matches
    the current kernel source and workload size."""
    try:
        with open(TRAFFIC[path][0]) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_sha") != kernel_sha(path) or int(t.get("n", -1)) != n:
        return None
    return float(t["dram_bytes_per_launch"])


def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(points_per_rank, world, elapsed_ms):
    """Whole-job throughput (Gpoint-updates/s): the points every rank
    processed over the slowest rank's timed region."""
    return points_per_rank * world / (elapsed_ms * 1e-3) / 1e9


def cpu_oracle_rate(prob, target_s):
    """FP64 oracle (C, OpenMP over z) on the host cores: leapfrog steps of the
    same grid, timed; returns (Gpt/s, steps, seconds, threads)."""
    import oracle
    oracle.build()
    n, halo = prob.nx, prob.halo
    z = np.zeros(W_padded(prob), np.float64)
    vel = prob.vel.astype(np.float64)
    # calibration: 1 step, then 4 steps (the difference removes the per-call buffer copies)
    t0 = time.perf_counter()
    a, b, _ = oracle.wave_propagate(z, z, vel, prob.dt, prob.h, halo, 1,
                                    src_idx=prob.src_idx, src_amp=prob.src_amp)
    t1 = time.perf_counter()
    a, b, _ = oracle.wave_propagate(a, b, vel, prob.dt, prob.h, halo, 4, t0=1,
                                    src_idx=prob.src_idx, src_amp=prob.src_amp)
    t2 = time.perf_counter()
    per_step = max(1e-4, ((t2 - t1) - (t1 - t0)) / 3.0)
    steps = max(1, min(400, int(target_s / per_step)))
    t0 = time.perf_counter()
    oracle.wave_propagate(a, b, vel, prob.dt, prob.h, halo, steps, t0=5,
                          src_idx=prob.src_idx, src_amp=prob.src_amp)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return prob.npoints * steps / dt / 1e9, steps, dt, threads


def time_calls(fn, k, stream):
    """Run fn() k times between CUDA events on `stream`; returns (ms per call,
    step-kernel ms per launch, launches) with the library's event profiler."""
    import torch
    import paper_2309_04671_gb300 as gbs
    torch.cuda.synchronize()
    gbs.profile_enable(True)
    gbs.profile_take()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    kms, kl = gbs.profile_take()
    gbs.profile_enable(False)
    return e0.elapsed_time(e1) / k, (kms / kl if kl else None), kl


def storage_forms(prob, args, stream, hbm):
    """BF16 and FP16 storage on the same workload: whole-call throughput and
    the step kernel's roofline at 10 algorithmic bytes per point."""
    import torch
    import paper_2309_04671_gb300 as gbs
    dev = torch.device("cuda", torch.cuda.current_device())
    shape = W_padded(prob)
    vel = torch.from_numpy(prob.vel).to(dev)
    si, sa = torch.from_numpy(prob.src_idx).to(dev), torch.from_numpy(prob.src_amp).to(dev)
    out = {}
    for fmt in ("bf16", "f16"):
        a, b = torch.zeros(shape, device=dev), torch.zeros(shape, device=dev)
        work = gbs.lp_workspace(a, prob.halo)
        st = {"a": a, "b": b}

        def run():
            st["a"], st["b"] = gbs.wave_propagate_lp(st["a"], st["b"], vel, prob.dt, prob.h, prob.halo, prob.nsteps,
                                                     storage=fmt, work=work, src_idx=si, src_amp=sa)
        for _ in range(2):
            run()
        k = max(3, args.steps // 4)
        ms, kms, kl = time_calls(run, k, stream)
        gbs.device_status()
        ach = 10 * prob.npoints / (kms * 1e-3) / 1e9
        out[fmt] = {"value": prob.npoints * prob.nsteps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
                    "calls": k, "bytes_per_point": 10,
                    "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                 "kernel_ms_per_launch": kms, "kernel_launches": kl}}
        del a, b, work, st
    torch.cuda.empty_cache()
    return out


def precision_form(args, stream, hbm, n=1024, nsteps=500):
    """The precision configuration: n^3 layered model, nsteps steps per call,
    wave fields stored in FP32, BF16 and FP16 (FP32 arithmetic in all).  One
    untimed call, then one timed call each; kernel roofline at 16 / 10 B/pt.
    (The FP64-oracle errors of the same setup are taken at 256^3.)"""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    halo, h = 4, 10.0
    vel = W.layered_velocity_torch(n, n, n, halo, W.SEED_BASE + 3, dev)
    dt = W.dt_for_cfl(0.4, h, float(vel.max()))
    si = torch.tensor([W.linear_index(n // 2, n // 2, 20, n, n)], dtype=torch.int64, device=dev)
    sa = torch.from_numpy(W.ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)).to(dev)
    out = {"workload": f"{n}^3 interior + halo 4, {nsteps} leapfrog steps per call, layered 1500-4500 m/s + 16 "
                       f"Gaussians, CFL 0.4, 15 Hz Ricker at depth 20"}
    a, b = torch.zeros_like(vel), torch.zeros_like(vel)
    work = None
    for fmt in ("f32", "bf16", "f16"):
        if fmt != "f32" and work is None:
            work = gbs.lp_workspace(a, halo)

        def run():
            a.zero_()
            b.zero_()
            if fmt == "f32":
                gbs.wave_propagate(a, b, vel, dt, h, halo, nsteps, src_idx=si, src_amp=sa)
            else:
                gbs.wave_propagate_lp(a, b, vel, dt, h, halo, nsteps, storage=fmt, work=work, src_idx=si,
                                      src_amp=sa)
        run()
        ms, kms, kl = time_calls(run, 1, stream)
        gbs.device_status()
        bpp = 16 if fmt == "f32" else 10
        ach = bpp * n ** 3 / (kms * 1e-3) / 1e9
        out[fmt] = {"value": n ** 3 * nsteps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_call": ms,
                    "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                 "bytes_per_point": bpp, "kernel_ms_per_launch": kms, "kernel_launches": kl}}
    for fmt in ("bf16", "f16"):
        out[fmt]["speedup_vs_f32"] = out["f32"]["ms_per_call"] / out[fmt]["ms_per_call"]
    del a, b, work, vel
    torch.cuda.empty_cache()
    return out


def absorb_form(prob, args, stream, hbm, width=20):
    """The headline workload inside an absorbing layer of `width` cells on
    every face (damped wave equation, eta_max for a 1e-3 reflection target):
    whole-call throughput and the step kernel's roofline at 16 B/pt."""
    import torch
    import paper_2309_04671_gb300 as gbs
    dev = torch.device("cuda", torch.cuda.current_device())
    vel = torch.from_numpy(prob.vel).to(dev)
    si, sa = torch.from_numpy(prob.src_idx).to(dev), torch.from_numpy(prob.src_amp).to(dev)
    vmax = float(prob.meta.get("vmax", vel.max().item()))
    eta_max = 3 * vmax * np.log(1e3) / (2 * width * prob.h)
    st = {"a": torch.zeros_like(vel), "b": torch.zeros_like(vel)}

    def run():
        st["a"], st["b"] = gbs.wave_propagate(st["a"], st["b"], vel, prob.dt, prob.h, prob.halo, prob.nsteps,
                                              src_idx=si, src_amp=sa, absorb=(width, eta_max))
    for _ in range(2):
        run()
    k = max(3, args.steps // 4)
    ms, kms, kl = time_calls(run, k, stream)
    gbs.device_status()
    ach = 16 * prob.npoints / (kms * 1e-3) / 1e9
    out = {"width": width, "eta_max": eta_max, "value": prob.npoints * prob.nsteps / (ms * 1e-3) / 1e9,
           "unit": UNIT, "ms_per_step": ms, "calls": k,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "kernel_ms_per_launch": kms, "kernel_launches": kl}}
    # the same through fused pairs of steps (20 algorithmic bytes per point per pair)
    if gbs.tb_supported(prob.nx, prob.ny, prob.nz, prob.halo)[0]:
        work = gbs.tb_workspace(vel, prob.halo)

        def run_tb():
            st["a"], st["b"] = gbs.wave_propagate_tb(st["a"], st["b"], vel, prob.dt, prob.h, prob.halo,
                                                     prob.nsteps, src_idx=si, src_amp=sa, absorb=(width, eta_max),
                                                     work=work)
        for _ in range(2):
            run_tb()
        ms2, kms2, kl2 = time_calls(run_tb, k, stream)
        gbs.device_status()
        ach2 = 20 * prob.npoints / (kms2 * 1e-3) / 1e9
        out["fused_pairs"] = {"value": prob.npoints * prob.nsteps / (ms2 * 1e-3) / 1e9, "unit": UNIT,
                              "ms_per_step": ms2, "speedup_vs_single_steps": ms / ms2,
                              "roofline": {"bound": "hbm", "achieved": ach2, "peak": hbm, "unit": "GB/s",
                                           "frac": ach2 / hbm, "kernel_ms_per_launch": kms2,
                                           "kernel_launches": kl2, "alg_bytes_per_point_per_launch": 20}}
        del work
    del st
    torch.cuda.empty_cache()
    return out


FP32_FMA_LANES_PER_SM = 128      # FP32 FMA lanes per SM (4 partitions x 32)


def fp32_peak_tflops(sm_mhz=2070.0):
    """FP32 peak from unit counts and clock: SMs x 128 lanes x 2 FLOP x clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP32_FMA_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def suite_form(args, stream, hbm):
    """The 20 kernels of the paper's numerical-accuracy suite (Table 4) on
    uniform[0,1) fields with seeded weights: 3D kernels on 512^3 (256^3 for
    box3d3r / box3d4r), 2D kernels on one 8192^2 plane.  Star and j* kernels
    are HBM-bound (8 B/pt); the box kernels of order >= 2 are bound by FP32
    FMA throughput (2 FLOP per footprint point)."""
    import torch
    import paper_2309_04671_gb300 as gbs
    dev = torch.device("cuda", torch.cuda.current_device())
    H = 4
    peak_f = fp32_peak_tflops()
    out = {"fp32_peak_tflops": peak_f, "fp32_peak_basis": "SMs x 128 FMA lanes x 2 FLOP x 2070 MHz"}
    g = torch.Generator(device=dev).manual_seed(11)
    for name, (shape, dims, r, div) in gbs.SUITE.items():
        n = 512 if dims == 3 else 8192
        if shape == "box" and dims == 3 and r >= 3:
            n = 256
        nz, hz = (n, H) if dims == 3 else (1, 0)
        x = torch.rand((nz + 2 * hz, n + 2 * H, n + 2 * H), device=dev, generator=g)
        y = torch.zeros_like(x)
        npts = gbs.suite_points(dims, shape, r)
        w = np.random.default_rng(npts).uniform(-1, 1, npts)

        def run():
            gbs.stencil_suite(x, y, dims=dims, shape=shape, radius=r, weights=w, halo=H,
                              divisor=7.0 if div else 1.0)
        for _ in range(3):
            run()
        ms, _, _ = time_calls(run, 10, stream)
        gbs.device_status()
        pts = n * n * nz
        flops = 2 * npts - 1 + (1 if div else 0)
        gbs_s = 8 * pts / (ms * 1e-3) / 1e9
        tf = flops * pts / (ms * 1e-3) / 1e12
        compute = shape == "box" and r >= 2
        out[name] = {"grid": [n, n, nz], "value": pts / (ms * 1e-3) / 1e9, "unit": UNIT, "us_per_call": ms * 1e3,
                     "flops_per_point": flops,
                     "roofline": ({"bound": "alu", "achieved": tf, "peak": peak_f, "unit": "TFLOP/s",
                                   "frac": tf / peak_f} if compute else
                                  {"bound": "hbm", "achieved": gbs_s, "peak": hbm, "unit": "GB/s",
                                   "frac": gbs_s / hbm})}
        del x, y
    torch.cuda.empty_cache()
    return out


def radius_sweep(args, stream, hbm):
    """stencil_apply R = 1..4 (7/13/19/25 points) on a uniform[-1,1] n^3 field."""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    n, halo = args.n, 4
    x = torch.from_numpy(W.uniform_field(n, n, n, halo, W.SEED_BASE + 22)).to(dev)
    y = torch.empty_like(x)
    out = {}
    for R in (1, 2, 3, 4):
        c = gbs.fd2_coeffs(R)

        def run():
            gbs.stencil_apply(x, y, radius=R, cx=c, cy=c, cz=c, halo=halo)
        for _ in range(3):
            run()
        ms, kms, kl = time_calls(run, 20, stream)
        ach = 8 * n ** 3 / (kms * 1e-3) / 1e9
        out[f"R{R}"] = {"points": 6 * R + 1, "value": n ** 3 / (ms * 1e-3) / 1e9, "unit": UNIT,
                        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                     "kernel_ms_per_launch": kms}}
    del x, y
    torch.cuda.empty_cache()
    return out


def precision_errors(stream, n=256, nsteps=500):
    """Error of FP32 / BF16 / FP16 storage against the FP64 oracle on an n^3
    copy of the layered workload (same generator), after nsteps steps."""
    import torch
    import oracle
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    prob = W.layered_problem(n=n, nsteps=nsteps, seed_offset=3)
    z = np.zeros(W_padded(prob), np.float32)
    vel = torch.from_numpy(prob.vel).to(dev)
    si, sa = torch.from_numpy(prob.src_idx).to(dev), torch.from_numpy(prob.src_amp).to(dev)
    t0 = time.perf_counter()
    _, ref, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, nsteps, src_idx=prob.src_idx,
                                      src_amp=prob.src_amp)
    t_oracle = time.perf_counter() - t0
    out = {"grid": [n, n, n], "steps": nsteps, "oracle_seconds": t_oracle}
    for fmt in ("f32", "f32_tb", "bf16", "f16"):
        a, b = torch.zeros_like(vel), torch.zeros_like(vel)
        if fmt == "f32":
            _, cur = gbs.wave_propagate(a, b, vel, prob.dt, prob.h, prob.halo, nsteps, src_idx=si, src_amp=sa)
        elif fmt == "f32_tb":
            # the headline path: fused pairs of steps (falls back to single steps where no fused shape fits)
            out["f32_tb_fused"] = bool(gbs.tb_supported(n, n, n, prob.halo)[0])
            _, cur = gbs.wave_propagate_tb(a, b, vel, prob.dt, prob.h, prob.halo, nsteps, src_idx=si, src_amp=sa)
        else:
            _, cur = gbs.wave_propagate_lp(a, b, vel, prob.dt, prob.h, prob.halo, nsteps, storage=fmt, src_idx=si,
                                           src_amp=sa)
        gbs.device_status()
        e = oracle.err_norms(cur.cpu().numpy(), ref)
        out[fmt] = {k: e[k] for k in ("norm_max_rel", "l2_rel", "max_abs", "rmsd")}
    return out


def batched_forms(args, stream, hbm, nshots=64, nsteps=200):
    """Many shots of uneven size (sides uniform in 96-320 per axis, own
    layered velocity and Ricker source each, 200 steps): one batch plan (one
    launch per step for all shots, autotuned tiling, graph-captured loop) in
    FP32 and BF16 storage, against the same shots advanced one after the
    other by the single-shot entry points."""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    specs = W.batch_specs(nshots)
    shots = []
    for s in specs:
        vel = W.layered_velocity_torch(s.nx, s.ny, s.nz, 4, s.vel_seed, dev)
        dt = W.dt_for_cfl(s.cfl, s.h, float(vel.max()))
        idx = torch.tensor([W.linear_index(*s.src, s.nx, s.ny)], dtype=torch.int64, device=dev)
        amp = torch.from_numpy(W.ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)).to(dev)
        z = torch.zeros_like(vel)
        shots.append(gbs.Shot(z, z.clone(), vel, dt, s.h, 4, idx, amp))
    pts = sum(s.nx * s.ny * s.nz for s in specs)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    out = {"workload": f"{nshots} shots, sides uniform in 96-320 per axis (seeded), halo 4, own layered velocity "
                       f"and 15 Hz Ricker source each, CFL 0.4, {nsteps} leapfrog steps per step",
           "points_per_step_leapfrog": pts, "leapfrog_steps": nsteps}
    k = 3
    for fmt in ("f32", "bf16"):
        for sh in shots:
            sh.u.zero_(), sh.u_prev.zero_()
        t0 = time.perf_counter()
        plan = gbs.BatchPlan(shots, storage=fmt, stream=side)
        t_plan = time.perf_counter() - t0
        info = plan.info()
        with torch.cuda.stream(side):
            plan.run(nsteps, use_graph=True)        # warm-up; builds the cached graph
            ms, _, _ = time_calls(lambda: plan.run(nsteps, use_graph=True), k, side)
            # kernel time per launch: the same run without the graph (the profiler skips captured launches)
            _, kms, kl = time_calls(lambda: plan.run(nsteps), 1, side)
        side.synchronize()
        gbs.device_status()
        bpp = 16 if fmt == "f32" else 10
        ach = bpp * pts / (kms * 1e-3) / 1e9
        out[fmt] = {"value": pts * nsteps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "calls": k,
                    "plan_create_s": t_plan, "autotuned": info,
                    "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                 "bytes_per_point": bpp, "kernel_ms_per_launch": kms, "kernel_launches": kl}}
        plan.close()

        def seq():
            for sh in shots:
                if fmt == "f32":
                    gbs.wave_propagate(sh.u_prev, sh.u, sh.vel, sh.dt, sh.h, 4, nsteps, src_idx=sh.src_idx,
                                       src_amp=sh.src_amp)
                else:
                    gbs.wave_propagate_lp(sh.u_prev, sh.u, sh.vel, sh.dt, sh.h, 4, nsteps, storage=fmt,
                                          src_idx=sh.src_idx, src_amp=sh.src_amp)
        seq()
        ms_seq, _, _ = time_calls(seq, 1, stream)
        gbs.device_status()
        out[fmt]["sequential_single_shot"] = {"value": pts * nsteps / (ms_seq * 1e-3) / 1e9, "unit": UNIT,
                                              "ms_per_step": ms_seq}
        out[fmt]["speedup_vs_sequential"] = ms_seq / ms
    # the FP64 oracle on the host cores: 4 of the shots, a bounded number of steps
    import oracle
    oracle.build()
    sample, ost = shots[:4], 50
    hostv = [(sh.vel.cpu().numpy(), sh.src_idx.cpu().numpy(), sh.src_amp.cpu().numpy()) for sh in sample]
    t0 = time.perf_counter()
    for (v, si, sa), sh in zip(hostv, sample):
        z = np.zeros_like(v)
        oracle.wave_propagate(z, z, v, sh.dt, sh.h, 4, ost, src_idx=si, src_amp=sa)
    t_o = time.perf_counter() - t0
    ipts = sum((v.shape[0] - 8) * (v.shape[1] - 8) * (v.shape[2] - 8) for v, _, _ in hostv)
    out["cpu_baseline"] = {"value": ipts * ost / t_o / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                           "sample": f"{ost} FP64 leapfrog steps of the first 4 shots ({t_o:.1f} s)"}
    del shots
    torch.cuda.empty_cache()
    return out


def _plain_gradient(vel, dt, h, nsteps, src, amp, rec, resid, ckpt):
    """The same gradient assembled from the library's single-step calls
    (gbs_wave_step for the forward, recomputation and adjoint steps,
    gbs_stencil_apply for L u^m) with the imaging product in torch FP64: the
    unfused way to compute it.  Same sqrt(N) checkpoints."""
    import torch
    import paper_2309_04671_gb300 as gbs
    halo = 4
    c = [w / (h * h) for w in gbs.fd2_coeffs(4)]
    a, b = torch.zeros_like(vel), torch.zeros_like(vel)
    cks = []
    for m in range(nsteps):
        if m % ckpt == 0:
            cks.append((a.clone(), b.clone()))
        gbs.wave_step(a, b, a, vel, dt, h, halo, src_idx=src, src_amp=amp, step=m)
        a, b = b, a
    g = torch.zeros(vel.shape, dtype=torch.float64, device=vel.device)
    v64 = vel.double()
    na, nb = torch.zeros_like(vel), torch.zeros_like(vel)
    lap = torch.zeros_like(vel)
    flat = src.clone()
    nx = vel.shape[2] - 2 * halo
    ny = vel.shape[1] - 2 * halo
    pidx = (flat % nx + halo) + vel.shape[2] * ((flat // nx) % ny + halo + vel.shape[1] * (flat // (nx * ny) + halo))
    for s in range(len(cks) - 1, -1, -1):
        m0, m1 = s * ckpt, min(s * ckpt + ckpt, nsteps)
        states = [cks[s][0], cks[s][1]]
        for m in range(m0 + 1, m1):
            nxt = torch.zeros_like(vel)
            gbs.wave_step(states[-2], states[-1], nxt, vel, dt, h, halo, src_idx=src, src_amp=amp, step=m - 1)
            states.append(nxt)
        for m in range(m1 - 1, m0 - 1, -1):
            gbs.wave_step(na, nb, na, vel, dt, h, halo, src_idx=rec, src_amp=resid, step=m)
            gbs.stencil_apply(states[m - m0 + 1], lap, radius=4, cx=c, cy=c, cz=c, halo=halo)
            g += 2.0 * na.double() * lap.double() / v64
            if m < amp.shape[0]:
                g.view(-1).index_add_(0, pidx, 2.0 * na.view(-1)[pidx].double() * amp[m].double() / v64.view(-1)[pidx])
            na, nb = nb, na
    g[:halo] = 0
    g[-halo:] = 0
    g[:, :halo] = 0
    g[:, -halo:] = 0
    g[:, :, :halo] = 0
    g[:, :, -halo:] = 0
    return g


def adjoint_form(args, stream, hbm, n=256, nsteps=1000, nshots=8):
    """Velocity gradient of the L2 trace misfit: n^3 layered + Gaussian model,
    nshots sources at seeded surface positions (depth 2), receivers on the
    full n x n plane at depth 8, data from a model with a +5% Gaussian
    anomaly, nsteps FP32 steps, sqrt(N) checkpoints, FP64 accumulation."""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    halo, h = 4, 10.0
    vel = W.layered_velocity_torch(n, n, n, halo, W.SEED_BASE + 5, dev)
    zz, yy, xx = torch.meshgrid(*(torch.arange(n + 2 * halo, device=dev, dtype=torch.float32) - halo - n / 2
                                  for _ in range(3)), indexing="ij")
    vtrue = vel * (1.0 + 0.05 * torch.exp(-(xx * xx + yy * yy + zz * zz) / (2 * (n / 8) ** 2)))
    del zz, yy, xx
    dt = W.dt_for_cfl(0.4, h, float(vtrue.max()))
    rng = np.random.default_rng(W.SEED_BASE + 5)
    pos = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(nshots)]
    rec = torch.tensor([W.linear_index(i, j, 8, n, n) for j in range(n) for i in range(n)], dtype=torch.int64,
                       device=dev)
    amp = torch.from_numpy(W.ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)).to(dev)
    srcs = [torch.tensor([W.linear_index(i, j, 2, n, n)], dtype=torch.int64, device=dev) for i, j in pos]
    d_obs = []
    for si in srcs:
        tr = torch.zeros((nsteps, rec.numel()), device=dev)
        gbs.wave_propagate(torch.zeros_like(vel), torch.zeros_like(vel), vtrue, dt, h, halo, nsteps, src_idx=si,
                           src_amp=amp, rec_idx=rec, rec_trace=tr)
        d_obs.append(tr)
    work = gbs.adjoint_workspace(vel, halo, nsteps)
    grad = torch.zeros(vel.shape, dtype=torch.float64, device=dev)
    misfit = torch.zeros(1, dtype=torch.float64, device=dev)

    def gradient(fused=False, tile_y=0):
        grad.zero_()
        misfit.zero_()
        for si, d in zip(srcs, d_obs):
            gbs.fwi_gradient(vel, dt, h, halo, nsteps, d, src_idx=si, src_amp=amp, rec_idx=rec, work=work,
                             grad=grad, misfit=misfit, fused=fused, tile_y=tile_y)

    def forward_only():
        tr = torch.empty((nsteps, rec.numel()), device=dev)
        for si in srcs:
            gbs.wave_propagate(torch.zeros_like(vel), torch.zeros_like(vel), vel, dt, h, halo, nsteps, src_idx=si,
                               src_amp=amp, rec_idx=rec, rec_trace=tr)
    fused_ms = {}
    for ty in (() if args.adj_no_fused else (0, 16, 28)):
        gradient(fused=True, tile_y=ty)
        fused_ms[str(ty) if ty else "auto"], _, _ = time_calls(lambda: gradient(fused=True, tile_y=ty), 1, stream)
    gradient()
    ms_g, kms, kl = time_calls(gradient, 1, stream)
    gbs.device_status()
    forward_only()
    ms_f, _, _ = time_calls(forward_only, 1, stream)
    k = int(np.ceil(np.sqrt(nsteps)))
    pts = n ** 3
    # algorithmic bytes per point per step: forward 16, recomputation 16 (K-1)/K,
    # adjoint step 16, imaging 20 (u^m, nu, w, FP32 partial read + write) and
    # the FP64 fold every 32 steps (FP32 read + write, FP64 read + write: 24/32)
    bpp = 16 + 16 * (k - 1) / k + 16 + 20 + 24 / 32
    alg = pts * nshots * nsteps * bpp
    kernel_ms = kms * kl            # summed duration of the step and imaging launches
    ach = alg / (kernel_ms * 1e-3) / 1e9
    out = {"workload": f"{n}^3 layered+16 Gaussians, {nshots} shots (depth 2, seeded x/y), {n}x{n} receivers at "
                       f"depth 8, {nsteps} steps FP32, CFL 0.4, data from a +5% Gaussian anomaly, checkpoints every "
                       f"{k} steps, FP64 gradient",
           "value": pts * nsteps * nshots / (ms_g * 1e-3) / 1e9, "unit": "gradient point-steps/s (x1e9)",
           "ms_per_gradient": ms_g, "shots": nshots, "forward_only_ms": ms_f, "gradient_over_forward": ms_g / ms_f,
           "fused_backward": {"ms_per_gradient_by_tile_y": fused_ms,
                              "note": "each backward step as one launch of the adjoint step and the imaging "
                                      "condition (k_adjimg; 28 B per point-step instead of 36)"},
           "misfit": float(misfit.cpu()[0]),
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "bytes_per_point_step": bpp, "kernel_ms": kernel_ms,
                        "kernel_launches": kl}}
    # the unfused composition of single-step calls, one shot
    g_fused = torch.zeros_like(grad)
    m1 = torch.zeros_like(misfit)
    _, _, _, resid = gbs.fwi_gradient(vel, dt, h, halo, nsteps, d_obs[0], src_idx=srcs[0], src_amp=amp,
                                      rec_idx=rec, work=work, grad=g_fused, misfit=m1)
    torch.cuda.synchronize()
    del work
    torch.cuda.empty_cache()
    # every state kept in HBM (K = 1: no recomputation), one shot, if it fits
    need = gbs.adjoint_workspace_bytes(n, n, n, nsteps, 1)
    free, _ = torch.cuda.mem_get_info()
    if need < 0.8 * free:
        work1 = gbs.adjoint_workspace(vel, halo, nsteps, ckpt_every=1)
        g1 = torch.zeros_like(grad)

        def store_all():
            g1.zero_()
            gbs.fwi_gradient(vel, dt, h, halo, nsteps, d_obs[0], src_idx=srcs[0], src_amp=amp, rec_idx=rec,
                             work=work1, grad=g1, ckpt_every=1)
        store_all()
        ms1, _, _ = time_calls(store_all, 1, stream)
        gbs.device_status()
        out["store_all_states"] = {"workspace_gb": need / 1e9, "ms_one_shot": ms1,
                                   "checkpointed_ms_one_shot": ms_g / nshots,
                                   "gradient_over_forward": ms1 / (ms_f / nshots),
                                   "bit_identical_to_checkpointed": bool(torch.equal(g1, g_fused))}
        del work1, g1
        torch.cuda.empty_cache()
    res = {}

    def plain():
        res["g"] = _plain_gradient(vel, dt, h, nsteps, srcs[0], amp, rec, resid, k)
    ms_p, _, _ = time_calls(plain, 1, stream)
    gbs.device_status()
    diff = float((res["g"] - g_fused).abs().max() / g_fused.abs().max())
    out["unfused_single_step_calls"] = {"ms_one_shot": ms_p, "fused_ms_one_shot": ms_g / nshots,
                                        "speedup_fused": ms_p / (ms_g / nshots), "grad_norm_max_rel_diff": diff}
    del res, d_obs
    torch.cuda.empty_cache()
    out["cpu_baseline"], out["vs_oracle_64"] = _adjoint_oracle_64(nsteps, stream)
    return out


def _adjoint_oracle_64(nsteps, stream, m=64):
    """The gradient recipe on an m^3 copy (one shot, every step): the FP64
    oracle on the host cores, timed (the form's CPU baseline), and the GPU
    path against it (time and error)."""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    import oracle
    oracle.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    halo, h = 4, 10.0
    vel = W.layered_velocity(m, m, m, halo, W.SEED_BASE + 5)
    c = np.arange(m + 2 * halo, dtype=np.float64) - halo - m / 2
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    vtrue = (vel * (1.0 + 0.05 * np.exp(-(xx * xx + yy * yy + zz * zz) / (2 * (m / 8) ** 2)))).astype(np.float32)
    vtrue = W.zero_halo(vtrue, halo)
    dt = W.dt_for_cfl(0.4, h, float(vtrue.max()))
    src = np.array([W.linear_index(m // 3, m // 2, 2, m, m)], np.int64)
    rec = np.array([W.linear_index(i, j, 8, m, m) for j in range(m) for i in range(m)], np.int64)
    amp = W.ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)
    _, d_obs = oracle.forward_states(vtrue, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    d_obs = d_obs.astype(np.float32)
    t0 = time.perf_counter()
    j_o, g_o = oracle.fwi_gradient(vel, dt, h, halo, nsteps, d_obs, src_idx=src, src_amp=amp, rec_idx=rec)
    t_o = time.perf_counter() - t0
    args = (torch.from_numpy(vel).to(dev), dt, h, halo, nsteps, torch.from_numpy(d_obs).to(dev))
    kw = dict(src_idx=torch.from_numpy(src).to(dev), src_amp=torch.from_numpy(amp).to(dev),
              rec_idx=torch.from_numpy(rec).to(dev))
    res = {}

    def run():
        res["r"] = gbs.fwi_gradient(*args, **kw)
    run()
    ms, _, _ = time_calls(run, 1, stream)
    gbs.device_status()
    misfit, grad = res["r"][0], res["r"][1]
    e = oracle.err_norms(grad.cpu().numpy(), g_o)
    base = {"value": m ** 3 * nsteps / t_o / 1e9, "unit": "gradient point-steps/s (x1e9)", "cores": os.cpu_count(),
            "kind": "oracle", "sample": f"one {m}^3 gradient, {nsteps} forward + {nsteps} adjoint steps ({t_o:.1f} s)"}
    return base, {"grid": [m, m, m], "steps": nsteps, "oracle_seconds": t_o, "gpu_ms": ms,
                  "gpu_vs_oracle": t_o * 1e3 / ms, "grad_norm_max_rel_err": e["norm_max_rel"],
                  "grad_l2_rel_err": e["l2_rel"], "misfit_rel_err": abs(float(misfit.cpu()[0]) - j_o) / j_o}


def W_padded(prob):
    import workloads as W
    return W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo)


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    prob = W.layered_problem(n=args.n, nsteps=args.nsteps)
    z = np.zeros(W_padded(prob), np.float64)
    vel = prob.vel.astype(np.float64)
    a, b = z, z.copy()
    t = 0
    per = max(1, args.ref_leapfrog)
    for _ in range(max(0, args.warmup)):
        a, b, _ = oracle.wave_propagate(a, b, vel, prob.dt, prob.h, prob.halo, per, t0=t,
                                        src_idx=prob.src_idx, src_amp=prob.src_amp)
        t += per
    t0 = time.perf_counter()
    for _ in range(args.steps):
        a, b, _ = oracle.wave_propagate(a, b, vel, prob.dt, prob.h, prob.halo, per, t0=t,
                                        src_idx=prob.src_idx, src_amp=prob.src_amp)
        t += per
    el = time.perf_counter() - t0
    value = prob.npoints * per * args.steps / el / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.n, args.nsteps),
                   "reference_step": f"{per} FP64 leapfrog steps of the full grid per step (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} x {per} FP64 leapfrog steps of the {args.n}^3 grid"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def single_step_form(prob, args, stream, hbm, vel, si, sa):
    """The same workload with one launch per step (wave_propagate): the
    single-step kernel against its own 16-byte roofline."""
    import torch
    import paper_2309_04671_gb300 as gbs
    halo, ns = prob.halo, prob.nsteps
    shape = W_padded(prob)
    a = torch.zeros(shape, device=vel.device)
    b = torch.zeros(shape, device=vel.device)
    st = {"a": a, "b": b}

    def run():
        st["a"], st["b"] = gbs.wave_propagate(st["a"], st["b"], vel, prob.dt, prob.h, halo, ns, src_idx=si,
                                              src_amp=sa)
    for _ in range(3):
        run()
    gbs.device_status()
    k = max(3, min(10, args.steps))
    ms, kms, kl = time_calls(run, k, stream)
    gbs.device_status()
    ach = BYTES_PER_POINT * prob.npoints / (kms * 1e-3) / 1e9 if kms else None
    return {"value": prob.npoints * ns / ms / 1e6, "unit": UNIT, "ms_per_call": ms, "calls": k,
            "kernel": "k_tma<R=4,wave,16,float>", "kernel_us": kms * 1e3 if kms else None,
            "achieved_gbs": ach, "frac": ach / hbm if ach else None,
            "traffic": traffic_per_launch(prob.nx, "single"), "alg_bytes_per_point": BYTES_PER_POINT}


def tblock_form(args, stream, hbm, sizes=(256, 384, 512), nsteps=96):
    """Temporal blocking against the number of steps fused per launch (1, 2,
    3) on the layered workload at several sizes: whole-call throughput, the
    fused kernel's time per launch, and DRAM bytes per update at the
    algorithmic minimum (16, 10, 8).  Nothing is recomputed across tiles; a
    z-chunked shape adds (steps-1) R planes either side of a chunk to the
    earlier stages (reported as the fraction of extra plane updates)."""
    import torch
    import paper_2309_04671_gb300 as gbs
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"leapfrog_steps_per_call": nsteps,
           "alg_bytes_per_update": {"1": 16, "2": 10, "3": 8}}
    for n in sizes:
        halo = 4
        vel = W.layered_velocity_torch(n, n, n, halo, W.SEED_BASE + 2, dev)
        dt = W.dt_for_cfl(0.4, 10.0, float(vel.max()))
        src = torch.tensor([W.linear_index(n // 2, n // 2, 20, n, n)], dtype=torch.int64, device=dev)
        amp = torch.from_numpy(W.ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)).to(dev)
        pts = n * n * n
        row = {}
        for tb in (1, 2, 3):
            if tb > 1:
                ok, ty, ctas = gbs.tbn_supported(n, n, n, halo, tb)
                if not ok:
                    row[str(tb)] = {"fused": False}
                    continue
                work = gbs.tbn_workspace(vel, halo, tb)
            a, b = torch.zeros_like(vel), torch.zeros_like(vel)
            st = {"a": a, "b": b}

            def run():
                if tb == 1:
                    st["a"], st["b"] = gbs.wave_propagate(st["a"], st["b"], vel, dt, 10.0, halo, nsteps, src_idx=src,
                                                          src_amp=amp)
                else:
                    st["a"], st["b"] = gbs.wave_propagate_tbn(st["a"], st["b"], vel, dt, 10.0, halo, nsteps, tb,
                                                              src_idx=src, src_amp=amp, work=work)
            for _ in range(2):
                run()
            gbs.device_status()
            ms, kms, kl = time_calls(run, 4, stream)
            gbs.device_status()
            alg = {1: 16, 2: 20, 3: 24}[tb]
            ach = alg * pts / (kms * 1e-3) / 1e9 if kms else None
            r = {"value": pts * nsteps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_call": ms,
                 "kernel_us_per_launch": kms * 1e3 if kms else None, "launches_per_call": kl / 4 if kl else None,
                 "kernel_us_per_step": kms * 1e3 / tb if kms else None,
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                              "frac": ach / hbm if ach else None, "alg_bytes_per_point_per_launch": alg}}
            if tb > 1:
                nt = ((n + 63) // 64) * ((n + ty - 1) // ty)
                chunks = ctas // nt
                zc = -(-n // chunks)
                extra = sum(min(n, zc * (c + 1) + (tb - 1 - s) * 4) - max(0, zc * c - (tb - 1 - s) * 4)
                            for c in range(chunks) for s in range(tb)) / (tb * n) - 1.0
                r.update({"fused": True, "tile_y": ty, "ctas": ctas, "zchunks": chunks,
                          "extra_plane_updates": extra})
            row[str(tb)] = r
            del a, b, st
        out[f"{n}^3"] = row
        del vel
        torch.cuda.empty_cache()
    return out


def pml_form(prob, args, stream, hbm, width=20):
    """The headline workload inside a PML of `width` cells (Grote & Sim
    equations; the inner box on the TMA kernel, six slabs on the slab kernel
    with their auxiliary fields), against the plain loop and the damping
    layer of the same width.  Algorithmic bytes per step: 16 per inner point,
    48 per slab point (u, u_prev, vel, u_next; phi x3 and psi read and
    written)."""
    import torch
    import paper_2309_04671_gb300 as gbs
    dev = torch.device("cuda", torch.cuda.current_device())
    n, halo, ns = prob.nx, prob.halo, prob.nsteps
    vel = torch.from_numpy(prob.vel).to(dev)
    si, sa = torch.from_numpy(prob.src_idx).to(dev), torch.from_numpy(prob.src_amp).to(dev)
    vmax = float(prob.meta["vmax"])
    zmax = 3 * vmax * np.log(1e3) / (2 * (width - 1) * prob.h)
    state = gbs.pml_state(vel, halo, width)
    a, b = torch.zeros_like(vel), torch.zeros_like(vel)
    st = {"a": a, "b": b}

    def run():
        st["a"], st["b"] = gbs.wave_propagate_pml(st["a"], st["b"], vel, prob.dt, prob.h, halo, ns, width, zmax,
                                                  state=state, state_init=True, src_idx=si, src_amp=sa)
    for _ in range(2):
        run()
    gbs.device_status()
    k = 3
    ms, kms, kl = time_calls(run, k, stream)
    gbs.device_status()
    inner = (n - 2 * width) ** 3
    slab = n ** 3 - inner
    kernel_ms_per_step = kms * kl / (k * ns) if kms else None
    alg = 16 * inner + 48 * slab
    ach = alg / (kernel_ms_per_step * 1e-3) / 1e9 if kernel_ms_per_step else None
    out = {"workload": f"{n}^3 layered workload, PML of {width} cells on every face, zeta_max "
                       f"{zmax:.1f} 1/s (3 v_max ln(1e3) / (2 (W-1) h)), {ns} steps per call",
           "value": prob.npoints * ns / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_call": ms, "calls": k,
           "slab_points": slab, "inner_points": inner,
           "state_bytes": int(state.numel()),
           "kernel_ms_per_step": kernel_ms_per_step,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm if ach else None, "alg_bytes_per_step": alg}}
    del a, b, st, state
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    import paper_2309_04671_gb300 as gbs
    import workloads as W

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbs.load()

    prob = W.layered_problem(n=args.n, nsteps=args.nsteps, nz=args.nz or None)
    n, halo, ns = prob.nx, prob.halo, prob.nsteps
    shape = W_padded(prob)
    a = torch.zeros(shape, device=dev)
    b = torch.zeros(shape, device=dev)
    vel = torch.from_numpy(prob.vel).to(dev)
    si = torch.from_numpy(prob.src_idx).to(dev)
    sa = torch.from_numpy(prob.src_amp).to(dev)
    stream = torch.cuda.current_stream()
    tb = args.storage == "f32" and args.path == "tb"
    tblk = args.time_block
    if tb:
        kw = dict(src_idx=si, src_amp=sa, kernel=args.kernel, use_graph=args.graph,
                  work=gbs.tbn_workspace(a, halo, tblk))

        def propagate(u_prev, u, vel_, dt_, h_, halo_, n_, **k):
            return gbs.wave_propagate_tbn(u_prev, u, vel_, dt_, h_, halo_, n_, tblk, **k)
    elif args.storage == "f32":
        kw = dict(src_idx=si, src_amp=sa, kernel=args.kernel, tile_y=args.tile_y, zchunk=args.zchunk,
                  use_graph=args.graph)
        propagate = gbs.wave_propagate
    else:
        kw = dict(src_idx=si, src_amp=sa, tile_y=args.tile_y, zchunk=args.zchunk, use_graph=args.graph,
                  storage=args.storage, work=gbs.lp_workspace(a, halo))
        propagate = gbs.wave_propagate_lp
    # algorithmic bytes per point of one launch of the dominant kernel
    bytes_per_point = (BYTES_PER_POINT_PAIR if tblk == 2 else 24) if tb else \
        (BYTES_PER_POINT if args.storage == "f32" else 10)
    tb_shape = gbs.tbn_supported(prob.nx, prob.ny, prob.nz, halo, tblk) if tb else None

    # warm-up (also builds the wavefield)
    for _ in range(max(3, args.warmup)):
        a, b = propagate(a, b, vel, prob.dt, prob.h, halo, ns, **kw)
    gbs.device_status()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    gbs.profile_enable(True)
    gbs.profile_take()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        a, b = propagate(a, b, vel, prob.dt, prob.h, halo, ns, **kw)
    ev1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    barrier(world)
    clocks.mark(w0, w1)
    kernel_ms, kernel_launches = gbs.profile_take()
    gbs.profile_enable(False)
    gbs.device_status()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    clk = clocks.stop()

    value = job_value(prob.npoints * ns * args.steps, world, elapsed_ms)
    hbm, peak_kind = peaks()
    per_launch_ms = kernel_ms / max(1, kernel_launches)
    alg_bytes = bytes_per_point * prob.npoints
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9 if kernel_launches else None
    traffic = (traffic_per_launch(n, "tb" if tb else "single")
               if args.storage == "f32" and prob.nz == n and not (tb and tblk != 2) else None)
    # sources are added inside the step kernels (at most 16); the fused path
    # also zeroes its workspace halo with one kernel per call
    inject_launches = args.steps if tb else 0

    # end to end through host buffers (pinned): every step copies its inputs
    # to the device and its two result fields back.  Headline: two
    # independent problems in a pipeline (gbs_pipeline_*), so the copies of
    # one overlap the steps of the other; beside it, one host-buffer call at
    # a time (gbs_wave_propagate_host), whose copies cannot overlap its steps.
    e2e = None
    if not args.no_e2e and args.storage == "f32":
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hv = pin(prob.vel)
        hsi, hsa = pin(prob.src_idx), pin(prob.src_amp)
        fields = [(torch.zeros(shape, dtype=torch.float32).pin_memory(),
                   torch.zeros(shape, dtype=torch.float32).pin_memory()) for _ in range(2)]
        fb = prob.vel.nbytes
        h2d_bytes, d2h_bytes = 3 * fb + prob.src_idx.nbytes + prob.src_amp.nbytes, 2 * fb
        pipe = gbs.Pipeline(n, n, n, halo, depth=2, time_block=2 if tb else 0, nsrc_max=prob.src_idx.size,
                            src_nt_max=prob.src_amp.shape[0], kernel=args.kernel,
                            tile_y=0 if tb else args.tile_y, zchunk=0 if tb else args.zchunk, use_graph=args.graph)
        for a, b in fields:                                  # warm-up: both workspaces once
            pipe.submit(a, b, hv, prob.dt, prob.h, ns, src_idx=hsi, src_amp=hsa)
        pipe.wait()
        e2e_steps = max(2, args.steps)                      # the same K steps as the device-timed region
        barrier(world)
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            a, b = fields[k % 2]
            pipe.submit(a, b, hv, prob.dt, prob.h, ns, src_idx=hsi, src_amp=hsa)
        pipe.wait()
        el = max_over_ranks(time.perf_counter() - t0, world)
        gbs.device_status()
        pipe.close()
        # one host-buffer call at a time
        hp, hu = fields[0]
        if tb:
            hkw = dict(src_idx=hsi, src_amp=hsa, kernel=args.kernel, use_graph=args.graph, work=kw["work"])
            hcall = gbs.wave_propagate_tb
        else:
            hkw = dict(src_idx=hsi, src_amp=hsa, kernel=args.kernel, tile_y=args.tile_y, zchunk=args.zchunk,
                       use_graph=args.graph)
            hcall = gbs.wave_propagate
        one_steps = max(1, min(3, args.steps))
        hcall(hp, hu, hv, prob.dt, prob.h, halo, ns, **hkw)   # warm-up (workspace allocation)
        barrier(world)
        t1 = time.perf_counter()
        for _ in range(one_steps):
            hcall(hp, hu, hv, prob.dt, prob.h, halo, ns, **hkw)
        el1 = max_over_ranks(time.perf_counter() - t1, world)
        e2e = {"value": prob.npoints * ns * e2e_steps * world / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes, "steps": e2e_steps,
               "mode": "gbs_pipeline: two independent problems in flight from pinned host memory, each step's "
                       "copies overlapping the other problem's steps",
               "one_call_at_a_time": {"value": prob.npoints * ns * one_steps * world / el1 / 1e9, "unit": UNIT,
                                      "steps": one_steps, "call": "gbs_wave_propagate_host"}}
        del fields, hv

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, steps, secs, threads = cpu_oracle_rate(prob, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{steps} FP64 leapfrog steps of the full {n}^3 grid ({secs:.1f} s), after 1 untimed step"}

    forms = None
    wanted = set() if args.no_forms or args.forms == "none" else set(args.forms.split(","))
    if rank == 0 and wanted:
        forms = {}
        if "single" in wanted and tb:
            forms["single_step"] = single_step_form(prob, args, stream, hbm, vel, si, sa)
        if "storage" in wanted:
            forms["storage"] = storage_forms(prob, args, stream, hbm)
        if "radius" in wanted:
            forms["radius_sweep"] = radius_sweep(args, stream, hbm)
        if "errors" in wanted:
            forms["error_vs_fp64_oracle"] = precision_errors(stream)
        if "precision" in wanted:
            forms["precision_1024"] = precision_form(args, stream, hbm)
        if "batched" in wanted:
            forms["batched"] = batched_forms(args, stream, hbm, nshots=args.batch_shots)
        if "absorb" in wanted:
            forms["absorbing_layer"] = absorb_form(prob, args, stream, hbm)
        if "suite" in wanted:
            forms["suite"] = suite_form(args, stream, hbm)
        if "pml" in wanted:
            forms["pml"] = pml_form(prob, args, stream, hbm)
        if "tblock" in wanted:
            forms["temporal_blocking"] = tblock_form(args, stream, hbm)
        if "adjoint" in wanted:
            forms["adjoint"] = adjoint_form(args, stream, hbm, n=args.adj_n, nsteps=args.adj_steps,
                                            nshots=args.adj_shots)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(n, ns, prob.nz), "grid": [prob.nx, prob.ny, prob.nz], "halo": halo,
                       "leapfrog_steps_per_step": ns, "dt": prob.dt, "h": prob.h,
                       "l2": f"no flush: each of the 3 fields ({4 * int(np.prod(shape)) / 1e6:.0f} MB) exceeds "
                             "the 129 MB L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "kernel": (f"k_wf<TY={tb_shape[1]}>: {tblk} fused leapfrog steps per launch "
                                  f"({tblk}-step temporal blocking, {tb_shape[2]} cooperative CTAs)" if tb else
                                  ("k_tma<R=4,wave>" if args.kernel != 2 else "k_generic<R=4,wave>"))
                       if args.storage == "f32" else f"k_tma<R=4,wave,{args.storage} storage>",
                       "path": ("fused pairs of steps" if tblk == 2 else "three fused steps per launch") if tb
                       else "one launch per step",
                       "storage": args.storage,
                       "tile_y": (tb_shape[1] if tb else args.tile_y or 16), "zchunk": args.zchunk or "auto",
                       "graph": args.graph},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "frac_of_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "nominal_peak": NOMINAL_HBM_GBS, "alg_bytes_per_launch": alg_bytes,
                         "alg_bytes_per_point_per_launch": bytes_per_point,
                         "point_updates_per_launch": prob.npoints * (tblk if tb else 1),
                         "kernel_ms_per_launch": per_launch_ms, "kernel_launches": kernel_launches,
                         # the throughput against the single-step minimum of 16 B per update (can exceed 1)
                         "single_step_basis_frac": (value * BYTES_PER_POINT / hbm) if args.storage == "f32"
                         else None},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": kernel_launches + inject_launches,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
