"""Throughput of the J.v + projection hot path on the 256^3 tanh-stretched cube at Gr = 2e8.

One step = one Chebyshev-filter step of the Arnoldi iteration on a 256^3 FP32 Krylov vector:
    y_next = alpha (P (J(q) y - sigma y) + sigma y) + beta y + gamma y_prev      (J.v, divergence,
             fast-diagonalisation pressure solve, gradient correction with the recurrence fused)
followed by its FP64 inner product <y_next, y_next> (read back to the host).  The metric counts one
J.v + projection per step.  Inputs (base state q, Krylov vectors) are seeded synthetic fields of the
paper's workload shape; every buffer (268 MB per FP32 vector) is larger than the 129 MB L2.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead (the reference
arm: there is no reference code, only the paper).  The one-GPU run also measures the time to the leading
eigenpairs at 64^3, Gr = 4e7, mixed against plain FP64 (about ten minutes of the run, most of it the FP64
form; --no-eigen skips it), a batched leg and the CPU baseline.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "J.v+projection/s at 256^3 (HBM %); time-to-leading-eigenpair vs plain FP64 @1e-6"
UNIT = "J.v+projection/s"
NX = NY = NZ = 256
STRETCH, GR, PR = 1.5, 2.0e8, 0.71
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=256)
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-eigen", action="store_true", help="skip the high-Gr time-to-eigenpair leg")
    p.add_argument("--eigen-grid", type=int, default=64, help="cells per axis of the time-to-eigenpair leg")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison leg")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    p.add_argument("--no-batch", action="store_true", help="skip the batched (block of 16 vectors) leg")
    p.add_argument("--cpu-sample-only", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


# ----------------------------------------------------------------------------- distributed (replicas)
def dist_setup(n):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def max_over_ranks(ws, x, device):
    """Slowest rank's time (a scalar, not a data-path collective)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as td
    t = torch.tensor([x], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, steps_per_rank, ms_max):
    """Whole-job value: every rank's steps over the slowest rank's time (replicas, weak scaling)."""
    return ws * steps_per_rank / (ms_max / 1e3)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- inputs
def make_inputs(n, device):
    """Base state q = conduction + N(0, 50^2) seeded perturbation, projected by the library (FP64);
    Krylov vectors y0, y1: seeded N(0,1).  Host generation (SplitMix64 + Box-Muller), then upload."""
    import numpy as np
    import torch
    from paper_2210_08816_gb300 import fv, seeded
    g = fv.Grid(n, n, n, stretch=STRETCH, Pr=PR)
    shape = (n, n, n)

    def to_dev(fields, dtype):
        return torch.from_numpy(np.stack(fields)).to(device=device, dtype=dtype).contiguous().view(-1)

    q = to_dev(seeded.normal_fields(100, shape, 50.0), torch.float64)
    fv.fv_project(g, fv.FV_FP64, q)          # divergence-free perturbation (wall slots zeroed inside)
    xf = np.array(g_faces(n))
    xc = 0.5 * (xf[:-1] + xf[1:])
    T = q.view(4, n, n, n)[3]
    T += torch.from_numpy(1.0 - xc).to(device)[None, None, :]
    y0 = to_dev(seeded.normal_fields(101, shape), torch.float64)
    y1 = to_dev(seeded.normal_fields(102, shape), torch.float64)
    fv.fv_project(g, fv.FV_FP64, y0)
    fv.fv_project(g, fv.FV_FP64, y1)
    return g, q, y0, y1


def g_faces(n):
    import math
    f = [0.5 * (1.0 + math.tanh(STRETCH * (2.0 * i / n - 1.0)) / math.tanh(STRETCH)) for i in range(n + 1)]
    for k in range(n // 2 + 1):
        f[n - k] = 1.0 - f[k]
    if n % 2 == 0:
        f[n // 2] = 0.5
    f[0], f[n] = 0.0, 1.0
    return f


# ----------------------------------------------------------------------------- GPU arm
def run_steps(fv, g, prec, q, ya, yb, K, stream, sigma, profile=False):
    """K recurrence steps y_{j+1} = 2 t (A - d) y_j - c2 t t' y_{j-1} (fixed coefficients of a
    degree-K Chebyshev filter on [-2|sigma|, 0]), each with its FP64 norm summed in the correction pass
    and stored on the device (stream-ordered); the norms are read back every 16 steps for the overflow
    guard, as the library's own filter does; returns (ms, last norm)."""
    import torch
    d, c2 = sigma, sigma * sigma * 0.9
    s = 10.0 - d
    tau = 1.0 / s
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    if profile:
        fv.fv_profile(g, True)
    norms = torch.zeros(K, dtype=torch.float64, device=ya.device)
    start.record(stream)
    nrm = 0.0
    for i in range(K):
        tn = 1.0 / (2.0 * s - c2 * tau)
        # yb <- 2 tn (A - d) ya - c2 tau tn yb   (A = P(J - sigma) + sigma)
        fv.fv_jvp_project_lincomb_dev(g, prec, GR, sigma, q, ya, yb, 2.0 * tn, -2.0 * tn * d, -c2 * tau * tn, yb,
                                      norm2=norms[i:i + 1])
        if i % 16 == 15 or i == K - 1:
            nrm = float(norms[i].item())
            if nrm > 1e30 or (0.0 < nrm < 1e-30):
                sc = 1.0 / nrm ** 0.5
                fv.fv_axpby(g, prec, 0.0, yb, sc, yb)
                fv.fv_axpby(g, prec, 0.0, ya, sc, ya)
        ya, yb = yb, ya
        tau = tn
    stop.record(stream)
    stop.synchronize()
    prof = fv.fv_profile_read(g) if profile else None
    if profile:
        fv.fv_profile(g, False)
    return start.elapsed_time(stop), nrm, prof, ya, yb


def gpu_arm(args, ws, rank, local):
    import torch
    from paper_2210_08816_gb300 import build, fv
    build.build()
    fv.lib()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream()
    n = args.grid
    g, q64, y0_64, y1_64 = make_inputs(n, device)
    sigma = -0.5 * (1.0 / PR) * 3 * 4.0 / (min(b - a for a, b in zip(g_faces(n)[:-1], g_faces(n)[1:])) ** 2)
    # FP32 copies (the mixed form's Krylov vectors and base state)
    q = q64.float()
    ya, yb = y0_64.float(), y1_64.float()
    N = n * n * n
    W, K = max(3, args.warmup), args.steps
    run_steps(fv, g, fv.FV_FP32, q, ya, yb, W, stream, sigma)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, nrm, prof, ya, yb = run_steps(fv, g, fv.FV_FP32, q, ya, yb, K, stream, sigma, profile=True)
    torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(ws, ms, device)
    ms_step = ms / K
    value = job_throughput(ws, K, ms)
    launches = sum(c for _, c in prof.values())

    # roofline of the dominant kernel class
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    per_launch_ms = dom_ms / max(dom_n, 1)
    clocks = clk.summary()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    if dom == "transform_tc":
        # One pass reads the N-cell field and writes it with the contracted axis rotated: 2 N FP32 values of
        # HBM traffic, which bounds it.  Its tensor work: the grid is mirror-symmetric, so a pass contracts
        # the sums and differences of mirrored inputs with two n/2 x n/2 matrices, N n flops (half of the
        # dense 2 N n), executed three times as 3 x TF32.
        traffic_bytes = 2 * N * 4
        achieved = traffic_bytes / (per_launch_ms * 1e-3) / 1e9
        flops = 1.0 * N * n
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        tf32_peak = bf16 * (1.1 / 2.25)   # TF32 dense = bf16 dense x nominal ratio 1.1 / 2.25 PFLOP/s
        executed = 3.0 * flops / (per_launch_ms * 1e-3) / 1e12
        roof = {"kernel": "k_transform_tcp (tcgen05 fast-diagonalisation pass, 3 x TF32 split)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "peak_source": hbm_src,
                "tensor": {"executed_tflops": round(executed, 2), "peak": round(tf32_peak, 1),
                           "frac": round(executed / tf32_peak, 4), "flops_per_pass": 3 * flops,
                           "peak_source": ("measured bf16 burst x 1.1/2.25 (TF32)" if "bf16_tflops" in peaks
                                           else "fallback 1.9 PF bf16 x 1.1/2.25")}}
    elif dom == "transform":
        flops = 2.0 * N * n
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"kernel": "k_transform (SIMT fast-diagonalisation pass)", "bound": "alu",
                "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "peak_source": "FP32 FMA lanes x 2 x 152 SMs x 2070 MHz (unit counts and max clock)"}
        traffic_bytes = 2 * N * 4
    else:
        bytes_per = {"stencil": 12 * N * 4, "correct": 17 * N * 4, "divergence": 4 * N * 4}.get(dom, 2 * 4 * N * 4)
        achieved = bytes_per / (per_launch_ms * 1e-3) / 1e9
        names = {"stencil": stencil_name(n), "correct": "k_correct4", "divergence": "k_divergence4"}
        roof = {"kernel": names.get(dom, dom), "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "peak_source": hbm_src}
        traffic_bytes = bytes_per
    roof["traffic"] = measured_traffic(dom, n)
    roof["algorithmic_bytes"] = traffic_bytes
    roof["launch_ms"] = round(per_launch_ms, 4)
    st_ms, st_n = prof["stencil"]
    st_gbs = 12 * N * 4 / (st_ms / st_n * 1e-3) / 1e9
    hbm_stencil = {"kernel": stencil_name(n), "achieved": round(st_gbs, 1), "peak": hbm_peak,
                   "unit": "GB/s", "frac": round(st_gbs / hbm_peak, 4), "algorithmic_bytes": 12 * N * 4,
                   "launch_ms": round(st_ms / st_n, 4), "traffic": measured_traffic("stencil", n)}
    # algorithmic bytes of one step: stencil 12 N, divergence 4 N, six passes 2 N each, correction 17 N
    # (the norm is summed inside the correction pass)
    step_bytes = (12 + 4 + 12 + 17) * N * 4
    breakdown = {k: {"ms_per_step": round(v[0] / K, 4), "launches_per_step": v[1] / K} for k, v in prof.items()}
    # the pressure solve's share of the step: the most that any replacement of the direct solve (a learned
    # Poisson surrogate included) could remove, since the direct solve needs one pass (I_p = 1)
    poisson_ms = (prof["transform_tc"][0] + prof["transform"][0]) / K
    breakdown["poisson_solve_share"] = round(poisson_ms / ms_step, 4) if ms_step > 0 else None

    # e2e through the C-ABI with host buffers: H2D of the step's input vector, the step, D2H of the result
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(fv, g, q, ya, yb, sigma, K, ws, device, stream)
    fp64 = None
    if not args.no_fp64:
        fp64 = fp64_leg(fv, g, q64, y0_64, y1_64, sigma, K, ws, device, stream)
    return finish(args, ws, rank, n, value, K, W, ms_step, e2e, launches, roof, hbm_stencil, step_bytes, breakdown,
                  fp64, clocks, g, device)


def e2e_leg(fv, g, q, ya, yb, sigma, K, ws, device, stream):
    """The step through the C-ABI with host buffers, as a streaming caller runs it: every step copies its
    input vector from pinned host memory to the device, runs the fused step (norm left on the device) and
    copies its result back to pinned host memory.  Three streams and two device buffer pairs let the
    upload of step i+1 and the download of step i-1 overlap the compute of step i (events order them)."""
    import torch
    nb = ya.numel()
    host_in = [ya.cpu().pin_memory() for _ in range(2)]
    host_out = [torch.empty(nb, dtype=ya.dtype).pin_memory() for _ in range(2)]
    d_in = [torch.empty_like(ya) for _ in range(2)]
    d_out = [torch.empty_like(yb) for _ in range(2)]
    norms = torch.zeros(2, dtype=torch.float64, device=ya.device)
    s_up, s_down = torch.cuda.Stream(device), torch.cuda.Stream(device)
    Ke = max(3, K)

    def run(nsteps):
        up = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        down = [torch.cuda.Event() for _ in range(2)]
        used = [False, False]
        for i in range(nsteps):
            b = i % 2
            with torch.cuda.stream(s_up):
                if used[b]:
                    s_up.wait_event(done[b])          # step i-2 has consumed d_in[b]
                d_in[b].copy_(host_in[b], non_blocking=True)
                up[b].record(s_up)
            stream.wait_event(up[b])
            if used[b]:
                stream.wait_event(down[b])            # step i-2's result has left d_out[b]
            fv.fv_jvp_project_lincomb_dev(g, fv.FV_FP32, GR, sigma, q, d_in[b], None, 1.0, 0.0, 0.0, d_out[b],
                                          norm2=norms[b:b + 1])
            done[b].record(stream)
            with torch.cuda.stream(s_down):
                s_down.wait_event(done[b])
                host_out[b].copy_(d_out[b], non_blocking=True)
                down[b].record(s_down)
            used[b] = True
        for st in (s_up, s_down):
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)

    run(4)
    torch.cuda.synchronize()
    link = host_link(host_in[0], d_in[0], host_out[0], d_out[0], stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    e0.record(stream)
    s_up.wait_event(e0)
    s_down.wait_event(e0)
    run(Ke)
    e1.record(stream)
    e1.synchronize()
    e_ms = max_over_ranks(ws, e0.elapsed_time(e1), device)
    e2e = {"value": round(ws * Ke / (e_ms / 1e3), 3), "unit": UNIT, "h2d_bytes_per_step": nb * ya.element_size(),
           "d2h_bytes_per_step": nb * yb.element_size(), "steps": Ke,
           "pipeline": "upload of step i+1 and download of step i-1 overlap step i (3 streams, 2 buffer pairs)",
           "host_link": link}
    del host_in, host_out, d_in, d_out
    return e2e


def host_link(h_in, d_in, h_out, d_out, stream, reps=3):
    """Bandwidth of the host link on this machine for the e2e leg's buffers: one pinned H2D and one pinned D2H copy
    of a step's vector, each timed alone with CUDA events (best of `reps`), so that the e2e figure can be
    read against what the link allows."""
    import torch
    best = {"h2d": 1e30, "d2h": 1e30}
    for _ in range(reps):
        for k, (dst, src) in (("h2d", (d_in, h_in)), ("d2h", (h_out, d_out))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            best[k] = min(best[k], e0.elapsed_time(e1))
    nbytes = h_in.numel() * h_in.element_size()
    return {"pinned": bool(h_in.is_pinned() and h_out.is_pinned()), "bytes": nbytes,
            "h2d_gbs": round(nbytes / (best["h2d"] * 1e-3) / 1e9, 1),
            "d2h_gbs": round(nbytes / (best["d2h"] * 1e-3) / 1e9, 1),
            "step_bound_per_s": round(1.0 / max(best["h2d"], best["d2h"]) * 1e3, 1)}


def fp64_leg(fv, g, q64, y0_64, y1_64, sigma, K, ws, device, stream):
    """Plain FP64 form on the same GPU (same step, FP64 everywhere)."""
    za, zb = y0_64.clone(), y1_64.clone()
    run_steps(fv, g, fv.FV_FP64, q64, za, zb, 2, stream, sigma)
    K64 = max(3, min(K, 5))
    ms64, _, _, _, _ = run_steps(fv, g, fv.FV_FP64, q64, za, zb, K64, stream, sigma)
    ms64 = max_over_ranks(ws, ms64, device)
    fp64 = {"value": round(ws * K64 / (ms64 / 1e3), 3), "ms_per_step": round(ms64 / K64, 3), "steps": K64}
    del za, zb
    return fp64


def finish(args, ws, rank, n, value, K, W, ms_step, e2e, launches, roof, hbm_stencil, step_bytes, breakdown, fp64,
           clocks, g, device):
    import torch
    from paper_2210_08816_gb300 import fv
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(n, ws), "precision": "mixed (FP32 vectors, FP64 reductions)",
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "hbm_stencil": hbm_stencil,
        "step_algorithmic_bytes": step_bytes, "kernel_breakdown": breakdown, "fp64_plain": fp64,
        "clocks": clocks,
    }
    g.close()
    torch.cuda.empty_cache()
    # single-GPU legs: rank 0 of the one-GPU run only (the scaling runs time the step alone)
    if rank == 0 and ws == 1 and not args.no_eigen:
        result["time_to_eigenpair"] = eigen_leg(fv, device, n=args.eigen_grid)
    if rank == 0 and ws == 1 and not args.no_batch:
        result["batched"] = batch_leg(fv, device)
    if rank == 0 and ws == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(n)
    return result


def stencil_name(n):
    """The FP32 J.v kernel the library picks for an n^3 grid (two cells per thread when n % 64 == 0)."""
    return "k_stencil_pair (J.v, two cells per thread)" if n % 64 == 0 else "k_stencil_z<float,1> (J.v)"


def measured_traffic(kind, n):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kind)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2210_08816_gb300", "csrc", rec["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != rec.get("sha") or rec.get("grid") != n:
        return None
    return rec.get("bytes_per_launch")


BATCH_POINTS = ((64, 3.0e7), (64, 4.06e7), (64, 5.50e7), (64, 7.44e7), (100, 1.01e8), (100, 1.36e8),
                (128, 1.85e8), (128, 2.5e8))


def batch_leg(fv, device, reps=10, nvec=16):
    """The batched workload: 8 continuation points, Gr log-spaced 3e7 .. 2.5e8, on stretched grids 4 x 64^3,
    2 x 100^3, 2 x 128^3, each applying a block of 16 seeded FP32 N(0,1) vectors (projected) through
    J.v + projection.  Base state per grid: conduction plus a seeded projected perturbation.
    Per grid size (first point of that size): 16 single-vector fv_jvp_project calls ("loop") against the
    block path eager and graph-replayed (z-chunk autotuned).  Then all 8 problems in ONE captured graph
    with concurrent branches (fv_batch_plan): 128 J.v + projections per replay."""
    import torch
    out = {"workload": "8 continuation points (Gr 3e7..2.5e8 log-spaced; 4 x 64^3, 2 x 100^3, 2 x 128^3 stretched), "
                       "blocks of 16 FP32 N(0,1) vectors, J.v+projection each", "unit": "J.v+projection/s"}

    def timed(fn, count):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return round(reps * count / (e0.elapsed_time(e1) / 1e3), 1)

    probs, seen = [], set()
    for k, (n, gr) in enumerate(BATCH_POINTS):
        g, q64, _, _ = make_inputs(n, device)
        q = q64.float()
        del q64
        gen = torch.Generator(device=device).manual_seed(100 + k)
        V = torch.randn(nvec * g.n, generator=gen, device=device, dtype=torch.float32)
        for i in range(nvec):
            fv.fv_project(g, fv.FV_FP32, V[i * g.n:(i + 1) * g.n])
        W = torch.empty_like(V)
        sig = -0.5 * (1.0 / PR) * 3 * 4.0 / (min(b - a for a, b in zip(g_faces(n)[:-1], g_faces(n)[1:])) ** 2)
        probs.append((g, gr, sig, q, V, W, nvec))
        if n in seen:
            continue
        seen.add(n)

        def loop():
            for i in range(nvec):
                fv.fv_jvp_project(g, fv.FV_FP32, gr, sig, q, V[i * g.n:(i + 1) * g.n], W[i * g.n:(i + 1) * g.n])

        row = {"loop": timed(loop, nvec)}
        for name, graph in (("block_eager", False), ("block_graph", True)):
            row[name] = timed(lambda: fv.fv_jvp_project_batch(g, fv.FV_FP32, gr, sig, q, V, W, nvec,
                                                              use_graph=graph, autotune=True), nvec)
        row["zchunk"] = fv.fv_get_tuning(g)[0]
        row["block_graph_vs_loop"] = round(row["block_graph"] / row["loop"], 3)
        out[f"{n}^3 Gr={gr:g}"] = row
    plan = fv.BatchPlan(probs, fv.FV_FP32, autotune=True)
    stream = torch.cuda.current_stream().cuda_stream
    total = sum(p[6] for p in probs)
    out["one_graph_8_points"] = {"value": timed(lambda: plan.launch(stream), total), "products_per_replay": total}
    plan.close()
    for p in probs:
        p[0].close()
    del probs
    torch.cuda.empty_cache()
    return out


def eigen_leg(fv, device, n=64, Gr=4.0e7):
    """Time to the leading eigenpairs at high Gr: n^3 tanh-stretched (s = 1.5), Pr = 0.71, Gr = 4e7 (below
    the first bifurcation, Section 4.1), k = 4, tol 1e-6.  Base state: pseudo-transient Newton (mixed) from
    conduction along a x4 Gr ladder from 1e5, timed.  Eigen-solver: shift-invert Arnoldi (implicit-Euler
    transform, dt = 1e-2, m = 30, GMRES(150) shifted solves), plain FP64 against the mixed form (FP32 phase,
    then FP64 cycles with refined solves) on the same GPU and state."""
    import torch
    g = fv.Grid(n, n, n, stretch=STRETCH, Pr=PR)
    xf = g_faces(n)
    xc = [0.5 * (a + b) for a, b in zip(xf[:-1], xf[1:])]
    q = torch.zeros(4, n, n, n, dtype=torch.float64, device=device)
    q[3] = (1.0 - torch.tensor(xc, dtype=torch.float64, device=device))[None, None, :]
    q = q.view(-1).contiguous()
    o = fv.fv_newton_default_opts()
    o.precision = fv.FV_FP32
    o.ptc_dt0 = 1e-3
    o.gr_start, o.gr_ratio = 1e5, 4.0
    o.max_newton = 60
    torch.cuda.synchronize()
    t0 = time.time()
    st, rep = fv.newton_steady(g, Gr, q, o)
    torch.cuda.synchronize()
    out = {"workload": f"{n}^3 tanh-stretched (s=1.5), Gr={Gr:g}, Pr=0.71, k=4, tol 1e-6, shift-invert "
                       "(euler_dt 1e-2, m 30, GMRES(150))",
           "newton_s": round(time.time() - t0, 2), "newton_status": st, "newton_matvecs": rep.matvecs,
           "newton_residual": rep.residual}
    lam = {}
    for name, prec in (("mixed", fv.FV_FP32), ("fp64", fv.FV_FP64)):
        a = fv.fv_arnoldi_default_opts()
        a.precision, a.tol, a.euler_dt, a.m = prec, 1e-6, 1e-2, 30
        a.inner_m, a.inner_max, a.max_restarts, a.low_max_restarts = 150, 4000, 8, 8
        torch.cuda.synchronize()
        t0 = time.time()
        st, l, r = fv.arnoldi_leading(g, 4, Gr, q, a)
        torch.cuda.synchronize()
        out[name] = {"seconds": round(time.time() - t0, 2), "status": st, "matvecs": r.matvecs,
                     "matvecs_fp64": r.matvecs_fp64, "cycles": r.restarts, "solves": r.solves,
                     "max_residual": max(r.residual[i] for i in range(r.nconv)) if r.nconv else None,
                     "lambda": [[z.real, z.imag] for z in l]}
        lam[name] = l[0] if l else None
    if lam.get("fp64") is not None and lam.get("mixed") is not None:
        out["lambda1_rel_diff"] = abs(lam["mixed"] - lam["fp64"]) / abs(lam["fp64"])
        out["speedup_mixed_vs_fp64"] = round(out["fp64"]["seconds"] / max(out["mixed"]["seconds"], 1e-9), 3)
    g.close()
    return out


# ----------------------------------------------------------------------------- CPU oracle
def workload_config(n, ws):
    """The bench's workload, the same for both arms."""
    return {"workload": f"{n}^3 tanh-stretched (s=1.5) cube, Gr=2e8, Pr=0.71: one Chebyshev-filter step "
                        "(J.v + projection + recurrence) + FP64 norm",
            "grid": [n, n, n], "stretch": STRETCH, "Gr": GR, "Pr": PR,
            "poisson": "direct fast diagonalisation (I_p = 1)",
            "l2": (f"inputs larger than L2 ({4 * n ** 3 * 4 / 1e6:.0f} MB per FP32 vector vs 129 MB L2)"
                   if 4 * n ** 3 * 4 > 129e6 else "inputs fit in the 129 MB L2 (no flush between steps)"),
            "parallelism": f"replicas x{ws}"}


def oracle_step_seconds(n, reps=1):
    """Time `reps` oracle steps (FP64 numpy) of the bench's workload: one step of the Chebyshev recurrence
    y_b <- 2 t (A - d) y_a - c2 t t' y_b with A = P(J - sigma) + sigma, and its norm; seconds per step."""
    import numpy as np
    import oracle.discretisation as D
    from oracle.projection import Projector
    from paper_2210_08816_gb300 import seeded
    og = D.Grid(n, n, n, stretch=STRETCH, Pr=PR)
    P = Projector(og)
    q = D.from_api(og, seeded.normal_fields(100, og.shape, 50.0))
    q[3] = q[3] + (1.0 - og.axes[0].xc)[None, None, :]
    ya = D.from_api(og, seeded.normal_fields(101, og.shape))
    yb = D.from_api(og, seeded.normal_fields(102, og.shape))
    hmin = min(float(np.min(a.dx)) for a in og.axes)
    sigma = -0.5 * (1.0 / PR) * 3 * 4.0 / hmin ** 2
    d, c2 = sigma, sigma * sigma * 0.9
    s = 10.0 - d
    tau = 1.0 / s
    tn = 1.0 / (2.0 * s - c2 * tau)
    t0 = time.time()
    for _ in range(reps):
        J = D.jvp_full(og, GR, q, ya)
        Ay = P.full([J[c] - sigma * ya[c] for c in range(4)])
        out = [2.0 * tn * (Ay[c] + (sigma - d) * ya[c]) - c2 * tau * tn * yb[c] for c in range(4)]
        nrm = sum(float(np.sum(o * o)) for o in out)
    dt = (time.time() - t0) / reps
    del out, nrm
    return dt


def cpu_baseline(n):
    """The oracle timed on this host: one full n^3 step of the workload in a single-threaded subprocess."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-only", "--grid", str(n)],
                           env=env, capture_output=True, text=True, timeout=900)
        sec = float(json.loads(r.stdout.strip().splitlines()[-1])["seconds"])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(e)[:200]}
    return {"value": round(1.0 / sec, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full {n}^3 step: J.v + projection + recurrence + norm (FP64 numpy oracle, "
                      f"fast-diagonalisation solve), {sec:.1f} s, single thread (BLAS threads = 1)",
            "cpu": cpu_model()}


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


def reference_arm(args, ws, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores, same workload and metric."""
    if rank != 0:
        return None
    n = args.grid
    W, K = max(1, min(args.warmup, 1)), args.steps
    oracle_step_seconds(n, W)
    t0 = time.time()
    for _ in range(K):
        oracle_step_seconds(n, 1)
    sec = (time.time() - t0) / K
    value = 1.0 / sec
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    cb = {"value": round(value, 5), "unit": UNIT, "cores": int(threads) if threads.isdigit() else os.cpu_count(),
          "kind": "oracle", "sample": f"{K} full {n}^3 steps (FP64 numpy oracle)", "cpu": cpu_model()}
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n, ws), "precision": "FP64 (numpy oracle)",
            "cpu_baseline": cb, "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.cpu_sample_only:
        print(json.dumps({"seconds": oracle_step_seconds(args.grid, 1)}))
        return
    ws, rank, local = (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                       int(os.environ.get("LOCAL_RANK", "0")))
    if args.impl == "reference":
        res = reference_arm(args, ws, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    ws, rank, local = dist_setup(args.gpus)
    res = gpu_arm(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
