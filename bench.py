"""Benchmark of the explicit P_N transport step on one or more B300 GPUs.

Workload (default): 128^3 grid, dx 0.25 mm, P_7 (64 complex moments), a
12-cell perfectly matched layer, background (mu_a 0.01, mu_s 10, g 0.9) with
8 seeded spheres, a pulsed l = 0 point source and 16 detector voxels, FP32
state, dt = 0.5 dt*. A step is one explicit step of Eq. 11 (forward/inverse
transforms, k-space coupling, pointwise stage, source, readouts).

Metric: moment-voxel updates/s = M V steps / time, summed over replicas.
Under torchrun every rank runs its own replica of the workload (the path has
no data exchange between problems), timed between barriers; the maximum time
over ranks is used.

--impl reference times the FP64 CPU oracle (the only other implementation
there is) on the same workload and metric.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "P_N moment-voxel updates/s"
UNIT = "updates/s"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def workload_config(wl, precision, dt, K, real=False):
    nz, ny, nx = wl.shape
    return {
        "workload": f"{nx}x{ny}x{nz} P_{wl.N} time-domain step: dx {wl.dx} mm, PML {wl.pml_width} cells "
                    f"(mu_b {wl.pml_mu0}->{wl.pml_mu1}/mm), background (0.01, 10, 0.9) + 8 spheres, "
                    f"pulsed l=0 source (FWHM 10 ps), {len(wl.det_voxel)} detectors",
        "grid": list(wl.shape), "N": wl.N, "moments": wl.M, "voxels": wl.V,
        "precision": precision, "dt_ps": dt, "timed_steps": K,
        "layout": "real radiance: m >= 0 moments stored, m < 0 from psi_l^-m = (-1)^m conj(psi_l^m)"
                  if real else "all (N+1)^2 moments stored",
        "l2": f"inputs larger than L2: state {wl.M * wl.V * 8 / 1e9:.2f} GB (FP32) per buffer vs 126 MB L2",
        "parallelism": "replicas (one independent problem per GPU)",
    }


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed regions: NVML
    every 5 ms in a background thread (nvidia-smi every 50 ms if the NVML
    binding is missing)."""
    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index, period_s=0.005):
        import threading
        self.period = period_s
        self.samples = []          # (sm_mhz, max_mhz, reason bits)
        self.proc = None
        self.thread = None
        self.stop_ev = threading.Event()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            if not uuid.startswith("GPU-"):
                uuid = "GPU-" + uuid
        except Exception:
            pass
        try:
            import pynvml
            pynvml.nvmlInit()
            try:
                h = pynvml.nvmlDeviceGetHandleByUUID(uuid) if uuid else pynvml.nvmlDeviceGetHandleByIndex(device_index)
            except Exception:
                h = pynvml.nvmlDeviceGetHandleByIndex(device_index)
            reasons = getattr(pynvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(pynvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
            mx = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)

            def poll():
                while not self.stop_ev.is_set():
                    try:
                        self.samples.append((pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM), mx, int(reasons(h))))
                    except Exception:
                        pass
                    self.stop_ev.wait(self.period)
            self.thread = threading.Thread(target=poll, daemon=True)
            self.source = "nvml every 5 ms"
        except Exception:
            self.source = "nvidia-smi every 50 ms"
            sel = ["-i", uuid] if uuid else ["-i", str(device_index)]
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.sel = sel

    def start(self):
        if self.thread is not None:
            self.thread.start()
            return
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", *self.sel, "--query-gpu=clocks.sm,clocks.max.sm,"
                                          "clocks_event_reasons.active", "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join(timeout=5)
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                except (ValueError, IndexError):
                    continue
            os.unlink(self.path)
        if not self.samples:
            return None
        bits = 0
        for _, _, r in self.samples:
            bits |= r
        return {"sm_mhz": float(np.median([x[0] for x in self.samples])),
                "sm_max_mhz": float(max(x[1] for x in self.samples)),
                "samples": len(self.samples), "source": self.source,
                "reasons": sorted(v for k, v in self.REASONS.items() if bits & k)}


KERNEL_SOURCES = ["rte_plane.cuh", "rte_kernels.cuh", "rte_fft.cuh", "rte_types.h", "rte_plan.cu"]


def sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1801_06364_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload_key):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, when it
    was measured on this workload with the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(path) if ":" in line)
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if kv.get("sources_sha256") != sources_sha256() or kv.get("workload_key") != workload_key:
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def reduce_over_ranks(dist, device, max_vals=(), sum_vals=()):
    """Job-wide view of per-rank measurements: maxima of the timings (the job
    ends when the slowest replica does) and sums of the counts. With dist None
    (one process) the values pass through."""
    import torch
    mx = [float(v) for v in max_vals]
    sm = [float(v) for v in sum_vals]
    if dist is not None:
        if mx:
            t = torch.tensor(mx, dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mx = t.tolist()
        if sm:
            t = torch.tensor(sm, dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            sm = t.tolist()
    return mx, sm


def job_value(units_per_rank, world, t_max_ms):
    """Whole-job throughput: units all replicas processed / slowest replica's time."""
    return units_per_rank * world / (t_max_ms / 1e3)


def kernel_bytes(name, M, V, b, r, L):
    """Algorithmic HBM bytes of one launch of each step kernel; M = stored
    moments, L = N + 1 damping planes."""
    n = M * V * b
    return {
        "k_zderiv": 2 * n,                         # read psi~, write Dz
        "k_zderiv(fixed)": 2 * n,
        "k_zstream": 2 * n,                        # read psi~ (every operand tile once), write w
        "k_ypass(inverse)": 2 * n,                 # read psi~, write T1
        "k_xpass(pointwise)": 2 * n + V * 4 * r,   # read/write T1, read media once
        "k_ypass(forward+coupling)": 4 * n,        # read T1, psi~, Dz; write psi~'
        "k_ypass_fixed(inverse)": 2 * n,
        "k_xpass_fixed(pointwise)": 2 * n + V * 4 * r,
        "k_ypass_fixed(forward+coupling)": 4 * n,
        "k_plane": 3 * n + V * L * r,              # read psi~, Dz, D_l once; write psi~'
    }.get(name)


def run_ours(args):
    import torch
    import paper_1801_06364_b300 as rte

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = synth.c2(N=args.N) if args.nz == 128 else synth.c2(shape=(args.nz, 128, 128), N=args.N)
    prec = args.precision
    stream = torch.cuda.current_stream()
    real = args.layout == "real"
    plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                    wl.pml_mu1, prec, stream=stream.cuda_stream, real_radiance=real)
    Ms = (wl.N + 1) * (wl.N + 2) // 2 if real else wl.M
    dt = 0.5 * plan.stability_limit()
    plan.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
    plan.set_detectors(wl.det_voxel)
    K, W = args.steps, args.warmup
    plan.step(dt, W)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(nsteps, p=plan):
        e0.record(stream)
        p.step(dt, nsteps)             # readouts to the host every call: part of the step
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # clocks sampled over the sustained blocks and the headline K steps, which
    # run back to back under load
    sampler = ClockSampler(local)
    sampler.start()
    blocks = [timed(args.block_steps) for _ in range(args.blocks)]
    barrier()
    l0 = rte.kernel_launches()
    t_ms = timed(K)                    # the headline: exactly K steps, replayed from step graphs
    launches = rte.kernel_launches() - l0
    clocks = sampler.stop()
    barrier()
    (t_ms, tb_med), (launches,) = reduce_over_ranks(dist, "cuda", [t_ms, float(np.median(blocks))], [launches])
    launches = int(launches)
    updates = wl.M * wl.V * K * world
    value = job_value(wl.M * wl.V * K, world, t_ms)

    # per-kernel CUDA events in a separate pass (they turn the step graphs off)
    plan.profile(True)
    plan.step(dt, K)
    prof = plan.profile_read()
    plan.profile(False)

    b = 16 if prec == "fp64" else 8
    r = b // 2
    peak, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, ms) = dom
    alg = kernel_bytes(name, Ms, wl.V, b, r, wl.N + 1)
    per_launch_s = ms / cnt / 1e3
    achieved = alg / per_launch_s / 1e9 if alg else None
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms / cnt,
                "traffic": args.traffic if args.traffic is not None else
                measured_traffic(name, f"N={wl.N} layout={args.layout} precision={prec}")}
    tot = sum(x[1] for x in prof.values())
    kernels = {k: {"launches": c, "total_ms": round(m, 3), "share": round(m / tot, 4),
                   "GBs": (kernel_bytes(k, Ms, wl.V, b, r, wl.N + 1) or 0) / (m / c / 1e3) / 1e9 or None}
               for k, (c, m) in prof.items()}
    fused = "k_plane" in prof
    # bytes per step over the stored moments: the lower bound 4b + 16/M per
    # update (read and write the state, write and read one intermediate, the
    # media once), and what this schedule moves
    lower = (4 * b * Ms + 16) * wl.V
    sched = ((5 * b * Ms + (wl.N + 1) * r) if fused else (10 * b * Ms + 4 * r)) * wl.V
    step_s = t_ms / K / 1e3
    step_roof = {"schedule": ("z streaming + fused plane (5 sweeps)" if fused else "Z, Y^-1, X, Y+ (10 sweeps)")
                 + (f", real-radiance layout ({Ms} of {wl.M} moments stored)" if real else ", all moments stored"),
                 "bytes_per_step_lower_bound": lower, "bytes_per_step_this_schedule": sched,
                 "frac_of_lower_bound_roofline": lower / step_s / (peak * 1e9),
                 "frac_this_schedule": sched / step_s / (peak * 1e9),
                 "achieved_GBs_this_schedule": sched / step_s / 1e9,
                 "full_layout_equivalent_frac": value / world * (4 * b + 16.0 / wl.M) / (peak * 1e9),
                 "note": "frac_of_lower_bound_roofline counts the bytes of the stored moments; "
                         "full_layout_equivalent_frac applies 4b + 16/M per update to all (N+1)^2 moments, "
                         "bytes the real layout never moves"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 (f32)" if prec == "fp32" else "c128 (f64)", "data": "synthetic",
            "config": workload_config(wl, prec, dt, K, real), "gpu_launches": launches, "roofline": roofline,
            "step_roofline": step_roof, "kernels": kernels, "clocks": clocks,
            "sustained": {"value": job_value(wl.M * wl.V * args.block_steps, world, tb_med), "unit": UNIT,
                          "ms_per_step": tb_med / args.block_steps, "blocks": args.blocks,
                          "steps_per_block": args.block_steps,
                          "note": "median of the blocks, each timed with CUDA events, step graphs, readouts "
                                  "to the host per block"}}

    if real and args.full_steps > 0:
        # the same step with every moment stored, for comparison
        plan.close()
        torch.cuda.empty_cache()
        pf = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                      wl.pml_mu1, prec, stream=stream.cuda_stream, real_radiance=False)
        pf.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
        pf.set_detectors(wl.det_voxel)
        pf.step(dt, 4)
        barrier()
        tf = timed(args.full_steps, pf)
        line["full_layout"] = {"value": wl.M * wl.V * args.full_steps / (tf / 1e3) * world, "unit": UNIT,
                               "steps": args.full_steps, "ms_per_step": tf / args.full_steps}
        pf.close()
        torch.cuda.empty_cache()
        plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                        wl.pml_mu1, prec, stream=stream.cuda_stream, real_radiance=real)
        plan.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
        plan.set_detectors(wl.det_voxel)
        plan.step(dt, 4)

    # end to end through the C ABI with host buffers: state in from pinned
    # memory, K steps with detector readouts to the host, state out to pinned memory
    host = torch.zeros(plan.field_shape, dtype=torch.complex64 if prec == "fp32" else torch.complex128).pin_memory()
    hout = torch.empty_like(host).pin_memory()
    barrier()
    t0 = time.perf_counter()
    plan.set_state(host)
    plan.set_time(0.0)
    plan.step(dt, K)
    plan.get_state(hout)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    (te,), _ = reduce_over_ranks(dist, "cuda", [te])
    # in: the stored moments only (a real-layout plan gathers its m >= 0
    # moments from the host field); out: the whole field (the m < 0 moments
    # are rebuilt on the device and copied too)
    sb_in = host.numel() * host.element_size() * Ms // wl.M
    sb_out = host.numel() * host.element_size()
    ns = len(wl.src_voxel)
    t_copy = max(te - step_s * K, 0.0)
    line["e2e"] = {"value": updates / te, "unit": UNIT,
                   "h2d_bytes_per_step": (sb_in + K * ns * r) / K,
                   "d2h_bytes_per_step": (sb_out + K * len(wl.det_voxel) * 8) / K,
                   "note": f"state uploaded and read back once per {K}-step solve (format conversion included), "
                           f"source amplitudes in and detector readouts out every step; the once-per-solve part "
                           f"took {t_copy * 1e3:.1f} ms, equal to {t_copy / step_s:.0f} steps, so a solve of K steps "
                           f"spends t_copy / (t_copy + K step) on it (half at K = {t_copy / step_s:.0f}, "
                           f"{100 * t_copy / (t_copy + 2000 * step_s):.1f}% at the 2000-step workload)"}
    plan.close()
    del host, hout
    torch.cuda.empty_cache()

    if not args.no_cufft:
        line["cufft_comparison"] = cufft_comparison(Ms, wl.shape, prec, t_ms / K)

    if not args.no_fp64 and prec == "fp32":
        dfma = rte.fma_peak("fp64")
        line["fp64"] = {"dfma_peak_tflops": dfma / 1e12, "note": "plain FP64 path, the same kernels in double "
                        "precision; FP64-pipe bound on B300. dfma_peak_tflops: the library's own FMA-chain kernel "
                        "(rte_fma_peak), 2 flops per FMA"}
        for lay in ("full", "real"):
            p64 = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0,
                           wl.pml_mu1, "fp64", stream=stream.cuda_stream, real_radiance=lay == "real")
            p64.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
            p64.set_detectors(wl.det_voxel)
            K64 = max(4, min(K, args.fp64_steps))
            p64.step(dt, 4)
            barrier()
            t64 = timed(K64, p64)
            v64 = wl.M * wl.V * K64 / (t64 / 1e3)
            M64 = Ms if lay == "real" else wl.M
            line["fp64"][lay] = {"value": v64 * world, "unit": UNIT, "steps": K64, "ms_per_step": t64 / K64,
                                 "frac_hbm_this_schedule": (M64 * 16 * 10 + 4 * 8) * wl.V / (t64 / K64 / 1e3)
                                 / (peak * 1e9),
                                 "flops_per_update_conventional": FP64_FLOPS_PER_UPDATE,
                                 "frac_dfma_peak_conventional": v64 * M64 / wl.M * FP64_FLOPS_PER_UPDATE / dfma}
            p64.close()
            torch.cuda.empty_cache()

    if not args.no_e2:
        # steady state by time integration against the Krylov solve (the
        # paper's E2 run); rank-local work, no part of the timed step
        line["e2_steady_state"] = e2_steady_costs(stream, 1e-6)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, dt)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def cufft_comparison(Ms, shape, prec, step_ms, reps=10):
    """A timed comparison only (cuFFT is not in the product): torch.fft's
    forward and inverse 3-D transforms (cuFFT) of every stored moment, the
    transforms alone that a step keeping the state in k-space needs, before any
    coupling or pointwise work, against this library's whole step."""
    import torch
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(1801063640)
    x = torch.randn((Ms, *shape), dtype=dt, device="cuda", generator=g)
    for _ in range(2):                                    # plans and workspace
        y = torch.fft.ifftn(torch.fft.fftn(x, dim=(1, 2, 3)), dim=(1, 2, 3))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    for _ in range(reps):
        y = torch.fft.ifftn(torch.fft.fftn(x, dim=(1, 2, 3)), dim=(1, 2, 3))
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    err = float((y - x).abs().max() / x.abs().max())
    del x, y
    torch.cuda.empty_cache()
    return {"what": f"torch.fft.fftn + ifftn over (z, y, x) of {Ms} moments of {shape[0]}x{shape[1]}x{shape[2]} "
                    f"({'complex64' if prec == 'fp32' else 'complex128'}, cuFFT), CUDA events, mean of {reps}",
            "ms": ms, "this_library_step_ms": step_ms, "cufft_transforms_over_step": ms / step_ms,
            "roundtrip_max_rel_err": err}


# Conventional FP64 flop count per stored moment-voxel update at 128^3: two
# xy transforms and one z-derivative pair (5 log2 n flops per point per
# transform), the coupling (about 48) and the pointwise stage (about 8).
FP64_FLOPS_PER_UPDATE = 2 * 5 * 21 + 48 + 8


def cpu_baseline(wl, dt, nsteps=1):
    """The FP64 oracle on the host cores: `nsteps` full-size explicit steps."""
    import oracle
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1)
    src = oracle.Sources(wl.src_voxel, np.zeros(len(wl.src_voxel), np.int32), wl.src_amp, wl.src_t0, wl.src_fwhm)
    psi = np.zeros((p.M,) + p.shape, complex)
    t0 = time.perf_counter()
    oracle.run(p, psi, dt, nsteps, sources=src, det_voxels=wl.det_voxel)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": wl.M * wl.V * nsteps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": el,
            "sample": f"{nsteps} explicit step(s) of the full 128^3 P_7 workload ({wl.M * wl.V * nsteps} "
                      f"moment-voxel updates), FP64 C oracle with OpenMP"}


def run_steady(args):
    """Steady-state solve of the 256^3 P_5 layered workload (C3): FP32 GMRES
    corrections refined with FP64 residuals to |q - T psi| / |q| <= 1e-6."""
    import torch
    import paper_1801_06364_b300 as rte
    wl = synth.c3()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                    args.precision, stream=stream.cuda_stream, real_radiance=args.layout == "real")
    plan.set_sources(wl.src_voxel, [0], wl.src_amp, wl.src_t0, wl.src_fwhm)
    setup = time.perf_counter() - t0
    torch.cuda.synchronize()
    l0 = rte.kernel_launches()
    t0 = time.perf_counter()
    it, rel, conv = plan.solve_steady(rtol=args.rtol, restart=args.restart, max_iter=args.max_iter)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    line = {"metric": "steady-state solve time (C3)", "value": el, "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "c64 (f32) + f64 residuals" if args.precision == "fp32" else "c128 (f64)",
            "data": "synthetic", "converged": conv, "arnoldi_steps": it, "rel_residual": rel,
            "rtol": args.rtol, "restart": args.restart, "gpu_launches": rte.kernel_launches() - l0,
            "plan_setup_s": setup,
            "config": {"workload": "256^3 P_5, dx 0.2 mm, PML 16, three z-slabs (mu_a 0.02/0.01/0.05, "
                                   "mu_s 8/12/6, g 0.8) with log-normal mu_s, CW l=0 source",
                       "layout": args.layout, "precision": args.precision}}
    print(json.dumps(line))


def run_adjoint(args):
    """Gradient of L = sum_d y_d^2 for the 128^3 P_5 random-field workload (C5):
    1500 FP32 steps forward with a checkpoint every 50, then the adjoint sweep."""
    import torch
    import paper_1801_06364_b300 as rte
    wl = synth.c5()
    stream = torch.cuda.current_stream()
    plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                    args.precision, stream=stream.cuda_stream, real_radiance=args.layout == "real")
    plan.set_sources(wl.src_voxel, np.zeros(len(wl.src_voxel)), wl.src_amp, wl.src_t0, wl.src_fwhm)
    plan.set_detectors(wl.det_voxel)
    dt = 0.5 * plan.stability_limit()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    y = plan.forward(dt, wl.nsteps, 50, wl.det_gate)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    ga, gs = plan.adjoint(2 * y)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    line = {"metric": "adjoint gradient time (C5)", "value": tf + tb, "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "c64 (f32)" if args.precision == "fp32" else "c128 (f64)", "data": "synthetic",
            "forward_s": tf, "adjoint_s": tb, "steps": wl.nsteps, "ckpt_every": 50,
            "loss": float(np.sum(y * y)), "grad_mua_norm": float(torch.linalg.norm(ga)),
            "grad_mus_norm": float(torch.linalg.norm(gs)),
            "forward_updates_per_s": wl.M * wl.V * wl.nsteps / tf,
            "config": {"workload": "128^3 P_5, dx 0.25 mm, PML 12, Gaussian-random-field mu_a, mu_s "
                                   "(correlation 3 mm), 4 pulsed sources, 32 gated detectors",
                       "layout": args.layout, "precision": args.precision, "dt_ps": dt}}
    print(json.dumps(line))


def fifo_latencies(arrivals, service):
    """Latencies of a single FIFO server (one request at a time) with the
    given arrival and service times: start_i = max(arrival_i, end_{i-1})."""
    end, out = 0.0, []
    for a, s in zip(arrivals, service):
        end = max(a, end) + s
        out.append(end - a)
    return np.array(out), end


def run_serve(args):
    """Serving workload (C4): --requests forward solves drawn from the recipe
    (grids 64-160^3 at dx 0.25, N 3-9, 500-3000 steps, PML 12, 1-6 spheres,
    16 detectors), FP32 real layout, each shape's schedule pinned by the
    autotuner, same-shape requests grouped into one launch per step pass:
    (a) as a seeded Poisson stream at 0.8 / (mean one-at-a-time FP32 service
    time), (b) as a burst at t = 0, (c) the burst without grouping; against
    one-at-a-time FP32 (every request, measured) and one-at-a-time FP64 (full
    layout, measured in full on a seeded sample of --fp64-sample requests)."""
    import dataclasses
    import torch
    import paper_1801_06364_b300 as rte
    from paper_1801_06364_b300.autotune import Autotuner, key_of
    from paper_1801_06364_b300.serving import Request, Server, poisson_arrivals, run_request, summarize
    real = args.layout == "real"
    reqs = [Request.from_workload(i, synth.c4_request(i)) for i in range(args.requests)]
    stream = torch.cuda.current_stream()
    # warm-up: first launches of every kernel family and the module's load
    for w in (synth.c4_request(0, grids=(64,), orders=(3,), steps_range=(20, 20)),
              synth.c4_request(1, grids=(96,), orders=(3,), steps_range=(20, 20))):
        run_request(Request.from_workload(-1, w), "fp32", real, stream.cuda_stream)
    torch.cuda.synchronize()
    # autotune every shape of the stream once (pinned for all later runs)
    tuner = Autotuner(steps=32, repeats=3)
    t0 = time.perf_counter()
    for r in reqs:
        tuner.choice(r.shape, r.N, "fp32", real, r.dx, r.c, r.pml_cells, r.pml_mu0, r.pml_mu1,
                     stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    l0 = rte.kernel_launches()
    one = Server(slots=1, precision="fp32", real_radiance=real, tuner=tuner)
    r1 = one.run(reqs)
    svc = np.array([r.end - r.admitted for r in r1])
    rate = 0.8 / float(svc.mean())
    arr = poisson_arrivals(len(reqs), rate, synth.BASE_SEED + 44)
    preqs = [dataclasses.replace(r, arrival=float(a)) for r, a in zip(reqs, arr)]
    clocks = ClockSampler(torch.cuda.current_device(), period_s=0.05)
    clocks.start()
    srv = Server(slots=args.slots, precision="fp32", real_radiance=real, grouping=True, tuner=tuner)
    r2 = srv.run(preqs)
    ck = clocks.stop()
    s2 = summarize(r2, preqs, srv.stats["makespan_s"])
    burst = Server(slots=args.slots, precision="fp32", real_radiance=real, grouping=True, tuner=tuner)
    r3 = burst.run(reqs)
    s3 = summarize(r3, reqs, burst.stats["makespan_s"])
    plain = Server(slots=args.slots, precision="fp32", real_radiance=real, grouping=False, tuner=tuner)
    r4 = plain.run(reqs)
    s4 = summarize(r4, reqs, plain.stats["makespan_s"])
    launches = rte.kernel_launches() - l0
    same = sum(int(a.ok and b.ok and np.array_equal(a.readouts, b.readouts)) for rr in (r2, r3, r4)
               for a, b in zip(r1, rr))
    # one-at-a-time FP64, full layout, every step run, on a seeded sample
    rng = np.random.default_rng(synth.BASE_SEED + 64)
    sample = sorted(rng.choice(len(reqs), min(args.fp64_sample, len(reqs)), replace=False).tolist())
    sreqs = [reqs[i] for i in sample]
    r64 = Server(slots=1, precision="fp64", real_radiance=False).run(sreqs)
    svc64 = np.array([r.end - r.admitted for r in r64])
    agree = [float(np.linalg.norm(a.readouts - r1[i].readouts) / max(np.linalg.norm(a.readouts), 1e-300))
             for a, i in zip(r64, sample) if a.ok and r1[i].ok]
    ups = sum(q.updates for q in reqs)
    ups64 = sum(q.updates for q in sreqs)
    rate64 = ups64 / float(svc64.sum())             # measured FP64 updates/s on the sample
    est64 = np.array([q.updates / rate64 for q in reqs])
    lat1p, end1p = fifo_latencies(arr, svc)
    lat64p, end64p = fifo_latencies(arr, est64)
    lat64b, end64b = fifo_latencies(np.zeros(len(reqs)), est64)

    def pct(x):
        return {"p50_latency_s": float(np.percentile(x, 50)), "p99_latency_s": float(np.percentile(x, 99))}
    line = {"metric": "served P_N moment-voxel updates/s (C4), p50/p99 latency", "value": s2["updates_per_s"],
            "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": "c64 (f32)", "data": "synthetic",
            "requests": len(reqs), "slots": args.slots, "arrival_rate_per_s": rate,
            "served_poisson_grouped": s2, "served_burst_grouped": s3, "served_burst_ungrouped": s4,
            "peak_group": [srv.stats.get("peak_group"), burst.stats.get("peak_group")],
            "completed": [s2["completed"], s3["completed"], s4["completed"]],
            "errors": sorted({r.error for r in list(r1) + list(r2) + list(r3) + list(r4) if not r.ok})[:4],
            "identical_to_alone": f"{same}/{3 * len(reqs)}",
            "peak_concurrent": [srv.stats["peak_active"], burst.stats["peak_active"], plain.stats["peak_active"]],
            "autotuner": {"seconds": tune_s, "choices": {k: {"schedule": v["schedule"], "graph_steps": v["graph_steps"],
                                                              "ms_per_step": v["ms_per_step"]}
                                                          for k, v in tuner.cache.items()}},
            "one_at_a_time_fp32": {"measured_service_s_mean": float(svc.mean()),
                                   "updates_per_s": ups / float(svc.sum()),
                                   "poisson": pct(lat1p), "burst": pct(np.cumsum(svc))},
            "one_at_a_time_fp64": {"kind": f"full layout, every step run, one at a time, on {len(sample)} seeded "
                                           f"requests {sample}; latencies of the whole stream from a FIFO queue of "
                                           f"each request's updates at the sample's measured rate",
                                   "sample_service_s": [float(x) for x in svc64],
                                   "updates_per_s": rate64,
                                   "fp32_vs_fp64_readouts_rel_l2_max": max(agree) if agree else None,
                                   "poisson": pct(lat64p), "burst": pct(lat64b)},
            "gpu_launches": launches, "clocks": ck,
            "config": {"workload": f"{len(reqs)} requests of the serving recipe: grid 64/96/128/160^3 dx 0.25, "
                                   "N 3/5/7/9, 500-3000 steps, PML 12, 1-6 spheres, 16 detectors",
                       "layout": args.layout, "precision": "fp32"}}
    print(json.dumps(line))


def e2_steady_costs(stream, rtol, kinds=("none",)):
    """The paper's E2 steady state two ways (Sec. II.A; Sec. IV runs it by
    time integration): 25 000 explicit FP32 steps (real layout) from zero
    with the constant source, then the steady-state residual |q - T psi| / |q|
    of the integrated state ((2l+1)-weighted); and restarted GMRES(60) on
    T psi = q to `rtol` (FP32 refined with FP64 residuals), for each
    preconditioner kind. Seconds of each, on `stream`."""
    import torch
    import paper_1801_06364_b300 as rte
    wl = synth.e2()
    res = {}
    plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                    "fp32", stream=stream.cuda_stream, real_radiance=True)
    plan.set_sources(wl.src_voxel, [0], wl.src_amp, wl.src_t0, wl.src_fwhm)
    dt = 0.5 * plan.stability_limit()
    plan.step(dt, 4, readouts=False)
    plan.set_state(np.zeros((wl.M,) + wl.shape, dtype=np.complex64))
    plan.set_time(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.step(dt, wl.nsteps, readouts=False)
    torch.cuda.synchronize()
    res["integrate_s"] = time.perf_counter() - t0
    res["integrate_steps"] = wl.nsteps
    res["physical_time_ps"] = dt * wl.nsteps
    psi = torch.from_numpy(plan.get_state()).cuda()
    tpsi = plan.apply_transport(psi)
    q = torch.zeros_like(psi)
    q.view(wl.M, -1)[0, int(wl.src_voxel[0])] = 1.0 / wl.dx ** 3
    wlv = torch.tensor([2 * l + 1 for l in range(wl.N + 1) for _ in range(2 * l + 1)], device="cuda",
                       dtype=torch.float64)

    def wn(u):
        return float(torch.sqrt((wlv[:, None] * (u.reshape(wl.M, -1).abs().double() ** 2)).sum()))
    res["integrated_residual"] = wn(q - tpsi) / wn(q)
    del psi, tpsi, q
    plan.close()
    torch.cuda.empty_cache()
    for kind in kinds:
        plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                        "fp32", stream=stream.cuda_stream, real_radiance=True)
        plan.set_sources(wl.src_voxel, [0], wl.src_amp, wl.src_t0, wl.src_fwhm)
        plan.set_preconditioner(kind)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rel, conv = plan.solve_steady(rtol=rtol, restart=60, max_iter=20000)
        torch.cuda.synchronize()
        res[f"gmres60_{kind}"] = {"s": time.perf_counter() - t0, "arnoldi_steps": it, "rel_residual": rel,
                                  "converged": conv}
        plan.close()
        torch.cuda.empty_cache()
    res["rtol"] = rtol
    res["workload"] = ("E2: 64^3 P_7, 35.5 mm cube of mu_a 0.01, mu_s 10, g 0.95 in a 50 mm box, 9-cell "
                       "half-cosine layer 0.01 -> 1 /mm, constant point source")
    return res


def run_paper(args):
    """Synthetic replays of the paper's two runs (Sec. IV) at the paper's step
    counts, timed on this GPU, next to the paper's own times on a Tesla K40
    (context: a different machine, and the paper's time steps, 0.1 and
    0.04 ps, are chosen by inspection, while here dt = 0.5 of this explicit
    scheme's stability limit). E1: 64^3 P_21, 400 steps (paper: 70 s). E2:
    64^3 P_7 with the layer, 25 000 steps towards the steady state (paper:
    223 s); E2's steady state is also solved directly by preconditioned
    GMRES, and the steady-state residual of the 25 000-step state is
    reported beside it."""
    import torch
    import paper_1801_06364_b300 as rte
    st = torch.cuda.Stream()
    out = {}

    def timed(plan, dt, n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.step(dt, n, readouts=False)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # E1: initial isotropic Gaussian, 1/e diameter 1.5 mm, in psi_00
    wl = synth.e1()
    pulse = synth.gaussian_pulse_state(0, wl.shape, wl.dx, sigma=0.75 / np.sqrt(2.0))[0]
    for prec, real, steps in (("fp32", True, 400), ("fp64", False, args.fp64_steps)):
        cd = torch.complex64 if prec == "fp32" else torch.complex128
        plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, 0, 0.0, 0.0, prec,
                        stream=st.cuda_stream, real_radiance=real)
        psi0 = torch.zeros((wl.M,) + wl.shape, dtype=cd, device="cuda")
        psi0[0] = torch.from_numpy(pulse).to(cd).cuda()
        dt = 0.5 * plan.stability_limit()
        plan.set_state(psi0)
        plan.step(dt, 4, readouts=False)   # first launches, graph capture
        plan.set_state(psi0)
        el = timed(plan, dt, steps)
        out[f"E1_{prec}"] = {"steps_timed": steps, "s_per_400_steps": el / steps * 400, "ms_per_step": 1e3 * el / steps,
                             "updates_per_s": wl.M * wl.V * steps / el, "dt_ps": dt,
                             "layout": "real" if real else "full", "paper_s_400_steps_K40": 70.0}
        plan.close()
        del psi0
        torch.cuda.empty_cache()
    # E2: constant source, towards the steady state
    wl = synth.e2()
    for prec, real, steps in (("fp32", True, wl.nsteps), ("fp64", False, args.fp64_steps * 10)):
        plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1,
                        prec, stream=st.cuda_stream, real_radiance=real)
        plan.set_sources(wl.src_voxel, [0], wl.src_amp, wl.src_t0, wl.src_fwhm)
        dt = 0.5 * plan.stability_limit()
        plan.step(dt, 4, readouts=False)
        plan.set_state(np.zeros((wl.M,) + wl.shape, dtype=np.complex64 if prec == "fp32" else np.complex128))
        plan.set_time(0.0)
        el = timed(plan, dt, steps)
        out[f"E2_{prec}"] = {"steps_timed": steps, "s_per_25000_steps": el / steps * 25000,
                             "ms_per_step": 1e3 * el / steps, "updates_per_s": wl.M * wl.V * steps / el, "dt_ps": dt,
                             "layout": "real" if real else "full", "paper_s_25000_steps_K40": 223.0}
        plan.close()
        torch.cuda.empty_cache()
    # the layer fills 63% of E2's grid and absorbs weakly without scattering,
    # where the mean-medium preconditioner does not fit: time both settings
    res = e2_steady_costs(st, args.rtol, ("none", "low"))
    out["E2_steady"] = res
    line = {"metric": "paper runs replayed (s per paper step count)", "value": out["E1_fp32"]["s_per_400_steps"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "runs": out,
            "config": {"workload": "E1: 64^3 P_21 50 mm cube, mu_s 1 / 5 /mm, g 0.9, 400 steps; "
                                   "E2: 64^3 P_7, mu_s 10, g 0.95, half-cosine layer 0.01 -> 1 /mm, CW source, "
                                   "25 000 steps, and its steady state by GMRES",
                       "note": "value is E1 FP32 (real layout) seconds for 400 steps; the paper's K40 times are "
                               "context (other machine, other dt)"}}
    print(json.dumps(line))


def run_c1(args):
    """The small periodic workload (C1): 32^3 P_3, dx 0.5 mm, homogeneous
    (0.01, 1, 0.5), isotropic Gaussian pulse (sigma 1 mm) in psi_00, 200
    steps at 0.5 dt*, the integral of psi_00 read every step. FP64 as
    configured, FP32 beside it. The state (4 MB) lives in L2: this measures
    launch and latency cost, which the step graphs address."""
    import torch
    import paper_1801_06364_b300 as rte
    wl = synth.c1()
    st = torch.cuda.Stream()
    out = {}
    for prec in ("fp64", "fp32"):
        plan = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, 0, 0.0, 0.0, prec, stream=st.cuda_stream)
        psi0 = synth.gaussian_pulse_state(wl.N, wl.shape, wl.dx, sigma=1.0)
        dt = 0.5 * plan.stability_limit()
        plan.set_state(psi0)
        plan.step(dt, 10, readouts=False, integral=True)
        best = None
        for _ in range(5):
            plan.set_state(psi0)
            plan.set_time(0.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, integ = plan.step(dt, wl.nsteps, readouts=False, integral=True)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            best = el if best is None else min(best, el)
        out[prec] = {"s_per_200_steps": best, "us_per_step": 1e6 * best / wl.nsteps,
                     "updates_per_s": wl.M * wl.V * wl.nsteps / best, "dt_ps": dt,
                     "integral_last": [float(integ[-1].real), float(integ[-1].imag)]}
        plan.close()
    line = {"metric": "C1 200-step run time", "value": out["fp64"]["s_per_200_steps"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "c128 (f64)", "data": "synthetic", "runs": out,
            "config": {"workload": "32^3 P_3 periodic, dx 0.5 mm, mu_a 0.01, mu_s 1, g 0.5, Gaussian pulse, "
                                   "200 steps, integral of psi_00 each step (host call per run: upload, "
                                   "200 steps, readback)", "note": "best of 5 runs, host wall clock"}}
    print(json.dumps(line))


def run_expo(args):
    """Exponential step for homogeneous media (the paper's arbitrary-step
    scheme for homogeneous media) on the C1 medium: one exponential step over
    the C1 run's 200 explicit steps, both against the oracle's exact
    per-wavevector solution at that time; then the cost at 128^3."""
    import torch
    import oracle
    import paper_1801_06364_b300 as rte
    wl = synth.c1()
    psi0 = synth.gaussian_pulse_state(wl.N, wl.shape, wl.dx, sigma=1.0)
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g)
    out = {}
    for prec in ("fp64", "fp32"):
        g = rte.Plan(wl.shape, wl.dx, wl.N, wl.c, wl.mua, wl.mus, wl.g, precision=prec)
        dt = 0.5 * g.stability_limit()
        T = wl.nsteps * dt
        exact = oracle.exp_step(p, psi0, T, 1) if prec == "fp64" else exact
        g.set_state(psi0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(dt, wl.nsteps, readouts=False)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        err_e = float(np.linalg.norm(g.get_state() - exact) / np.linalg.norm(exact))
        g.set_state(psi0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step_exponential(T, 1)
        torch.cuda.synchronize()
        tx = time.perf_counter() - t0
        err_x = float(np.linalg.norm(g.get_state() - exact) / np.linalg.norm(exact))
        out[f"C1_{prec}"] = {"time_ps": T, "explicit_steps": wl.nsteps, "explicit_s": te, "explicit_rel_err": err_e,
                             "exponential_s_with_setup": tx, "exponential_rel_err": err_x}
        g.close()
    # cost at 128^3 P_3 in the C1 medium (dx 0.5): setup once, then per step
    n = 128
    g = rte.Plan((n, n, n), wl.dx, wl.N, wl.c, float(wl.mua.flat[0]), float(wl.mus.flat[0]), float(wl.g.flat[0]),
                 precision="fp32")
    g.set_state(torch.zeros(g.field_shape, dtype=torch.complex64, device="cuda"))
    dts = 0.5 * g.stability_limit()
    Tb = 50 * dts
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step_exponential(Tb, 1)                 # builds E_k
    torch.cuda.synchronize()
    tsetup = time.perf_counter() - t0
    t0 = time.perf_counter()
    g.step_exponential(Tb, 10)
    torch.cuda.synchronize()
    tstep = (time.perf_counter() - t0) / 10
    t0 = time.perf_counter()
    g.step(dts, 100, readouts=False)
    torch.cuda.synchronize()
    texp = (time.perf_counter() - t0) / 100
    out["128cubed_P3_fp32"] = {"exponential_step_s": tstep, "first_step_with_E_build_s": tsetup,
                               "explicit_step_s": texp, "explicit_steps_per_exponential_step": 50,
                               "speedup_at_equal_time": 50 * texp / tstep}
    line = {"metric": "exponential step vs explicit steps (homogeneous medium)", "value": out["C1_fp64"]["exponential_rel_err"],
            "unit": "relative L2 error at the C1 end time", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "runs": out, "config": {"workload": "C1 medium (32^3 P_3, dx 0.5, mu_a 0.01, mu_s 1, g 0.5, periodic, "
                                                "Gaussian pulse), 200 explicit steps at 0.5 dt* vs one exponential "
                                                "step; 128^3 P_3 in the same medium for cost"}}
    print(json.dumps(line))


def run_reference(args):
    """FP64 CPU oracle on the same workload and metric, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    wl = synth.c2()
    p = oracle.Problem(wl.N, wl.shape, wl.dx, wl.c, wl.mua, wl.mus, wl.g, wl.pml_width, wl.pml_mu0, wl.pml_mu1)
    dt = 0.5 * oracle.stability_limit(p)
    src = oracle.Sources(wl.src_voxel, np.zeros(len(wl.src_voxel), np.int32), wl.src_amp, wl.src_t0, wl.src_fwhm)
    psi = np.zeros((p.M,) + p.shape, complex)
    K = max(1, min(args.steps, args.ref_steps))
    # untimed warm-up steps (at most 3: a full-size oracle step takes seconds),
    # then the timed sample continues from the warmed-up state
    W = max(0, min(args.warmup, 3))
    if W:
        psi, _, _ = oracle.run(p, psi, dt, W, sources=src, det_voxels=wl.det_voxel)
    t0 = time.perf_counter()
    oracle.run(p, psi, dt, K, t_start=W * dt, sources=src, det_voxels=wl.det_voxel)
    el = time.perf_counter() - t0
    value = wl.M * wl.V * K / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{K} explicit step(s) of the full 128^3 P_7 workload after {W} untimed ones, FP64 C oracle, "
              f"OpenMP; requested {args.steps} steps and {args.warmup} warm-up steps, capped at "
              f"{args.ref_steps} and 3 to bound the run")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128 (f64)", "data": "synthetic", "impl": "reference",
            "config": workload_config(wl, "fp64", dt, K),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="step", choices=["step", "steady", "adjoint", "serve", "paper", "c1", "expo"],
                    help="step: the benchmark time step (default); steady: C3 GMRES; adjoint: C5 gradient; "
                         "serve: C4 request stream; paper: replays of the paper's two runs; c1: the 32^3 run; "
                         "expo: exponential step for homogeneous media")
    ap.add_argument("--requests", type=int, default=256, help="serve: requests drawn from the recipe")
    ap.add_argument("--fp64-sample", type=int, default=6, help="serve: requests run one at a time in FP64")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent requests")
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--blocks", type=int, default=10, help="step: sustained-rate blocks (median reported)")
    ap.add_argument("--block-steps", type=int, default=100, help="step: steps per sustained-rate block")
    ap.add_argument("--N", type=int, default=7, help="P_N order (7 is the benchmark workload)")
    ap.add_argument("--nz", type=int, default=128,
                    help="step: z planes of the grid (128 is the benchmark workload; fewer for profiling captures)")
    ap.add_argument("--layout", default="real", choices=["real", "full"],
                    help="real: store m >= 0 moments (exact for real radiance); full: all (N+1)^2")
    ap.add_argument("--full-steps", type=int, default=50, help="steps of the extra full-layout timing")
    ap.add_argument("--ref-steps", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2", action="store_true", help="step: skip the E2 steady-state comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="step: skip the timed cuFFT comparison")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured for the current kernel sources")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # not started by torchrun: start one replica rank per GPU the same way
        import socket
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "steady":
        run_steady(args)
    elif args.mode == "adjoint":
        run_adjoint(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "paper":
        run_paper(args)
    elif args.mode == "c1":
        run_c1(args)
    elif args.mode == "expo":
        run_expo(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
