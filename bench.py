#!/usr/bin/env python3
"""Benchmark of the transpose-free 3D r2c + c2r FFT on GB300.

Workload (one step): forward r2c then inverse c2r of a 512 x 512 x 512 FP32
spectrum-shaped field (random-phase, divergence-free velocity component,
E(k) ~ k^4 exp(-2 (k/4)^2) below k = 8, k^-5/3 above, 2/3-truncated; seed
1408), on the plain FP32 transpose-free path, inputs resident in HBM.

Metric: effective HBM throughput = the two-pass minimum bytes of r2c + c2r,
2 * (4N + 24M) with N = n^3 reals and M = n*n*(n/2+1) complex values, divided
by the step time; ms per step alongside.  The same bytes/time is reported for
the end-to-end call with host buffers (``e2e``) and for the FP64 CPU oracle
(``cpu_baseline``; ``--impl reference`` times only the oracle).

Multi-GPU: the transform is one volume per GPU (replicas only, no exchange):
each rank transforms its own field; value = all ranks' bytes / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D r2c+c2r ms & HBM GB/s vs 8 TB/s; split-BF16 TC vs FP32 at stated rel-L2 error"
UNIT = "GB/s"
FALLBACK_HBM_GBS = 6800.0


def two_pass_bytes(n0, n1, n2):
    N = n0 * n1 * n2
    M = n0 * n1 * (n2 // 2 + 1)
    return 2 * (4 * N + 24 * M), N, M


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def workload_config(n, args):
    n0, n1, n2 = args.shape
    field = ("spectrum-shaped velocity component (seed 1408)" if args.field == "spectrum"
             else "seeded uniform[-1,1) field (seed 1408)")
    return {
        "workload": f"{n0}x{n1}x{n2} FP32 r2c+c2r, transpose-free, {field}",
        "n0": n0, "n1": n1, "n2": n2, "batch": 1,
        "bytes_per_step": two_pass_bytes(n0, n1, n2)[0],
        "bytes_definition": "2*(4N+24M): one read + one write per pass of the 2-pass minimum, r2c and c2r",
        "l2": "inputs larger than L2 (0.54 GB real + 0.54 GB complex per field), no flush",
        "parallelism": f"replicas x{args.gpus}",
    }


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources the row and column kernels of the 2^k lengths are built from
KERNEL_SOURCES = ("args.h", "inst.cuh", "inst_256_512.cu", "inst_1024_2048.cu", "kernels.cuh", "radix.cuh",
                  "stockham.cuh", "tma.cuh", "tma_host.h")


def kernel_source_hash():
    """Hash of the row / column kernels' device-code sources."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1406_5597_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in KERNEL_SOURCES:
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(pass_name, shape):
    """dram bytes per launch of a pass at this shape ("n0xn1xn2"), from the
    committed ncu summary, if it was taken on the current kernel sources
    (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("pass") == pass_name and kv.get("shape") == shape and kv.get("src") == src:
            return float(kv["bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"fft3d_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


SLOWDOWN_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def max_over_ranks(values, device):
    """Element-wise maximum of a list of numbers over all ranks of the process
    group (the job's time is that of its slowest rank); every rank gets it."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def clocks_rejected(clocks, world=1, device=None):
    """A timed region whose clock record shows a hardware or thermal slowdown,
    or SM clocks well below their maximum with no reason given (a clock lock
    left by someone else), is not a valid measurement.  Under torchrun every
    rank must take the same decision, so the verdict is max-reduced."""
    bad = bool(clocks) and (any(r in clocks["reasons"] for r in SLOWDOWN_REASONS)
                            or (not clocks["reasons"] and clocks["sm_mhz"] < 0.9 * clocks["sm_max_mhz"]))
    if world > 1:
        bad = max_over_ranks([1.0 if bad else 0.0], device)[0] > 0.0
    return bad


def make_field_shape(n0, n1, n2):
    import numpy as np

    import synth
    S = synth.spectral_velocity(n0, n1, n2, seed=synth.seed_for_config(2), components=(0,))[0]
    return S.astype(np.complex64)


def run_reference(args):
    """FP64 CPU oracle on the host cores, same workload (shape and field),
    metric and unit; W warm-up steps and K timed ones, both capped so that the
    run stays within a few minutes."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth
    n0, n1, n2 = args.shape
    if args.field == "spectrum":
        x = oracle.c2r3d(make_field_shape(n0, n1, n2).astype(np.complex128), n2)  # setup, not timed
    else:
        x = synth.uniform_field((n0, n1, n2), 1408)
    nbytes, _, _ = two_pass_bytes(n0, n1, n2)
    cores = oracle.threads()

    def step():
        X = oracle.r2c3d(x)
        oracle.c2r3d(X, n2)

    t0 = time.perf_counter()
    step()
    t_first = time.perf_counter() - t0
    warmup = 1 + max(0, min(args.warmup - 1, int(30.0 / max(t_first, 1e-3))))
    for _ in range(warmup - 1):
        step()
    steps = max(1, min(args.steps, int(150.0 / max(t_first, 1e-3))))
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = nbytes / (ms * 1e-3) / 1e9
    sample = (f"full {n0}x{n1}x{n2} r2c+c2r in FP64 per step; {steps} timed step(s) after {warmup} warm-up "
              f"step(s) (both capped so the run stays within a few minutes)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(n0, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(fn, stream, steps):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fft3d", choices=["fft3d", "reference"])
    ap.add_argument("--n", type=int, default=512, help="cubic size (default workload 512^3)")
    ap.add_argument("--shape", type=str, default=None, help="n0,n1,n2 (overrides --n)")
    ap.add_argument("--field", default="spectrum", choices=["spectrum", "uniform"],
                    help="input field; uniform skips the host-side spectrum generator (large sizes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--tc", action="store_true", help="time the tensor-core forms even with --no-variants")
    ap.add_argument("--no-autotune", action="store_true", help="keep the compiled kernel shapes")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (args.n, args.n, args.n)
    if args.field == "spectrum" and args.shape[2] % 2:
        args.field = "uniform"  # the spectrum-shaped field is defined for even n2 only

    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1406_5597_gb300 as fft3d

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    fft3d.load()
    n = args.n
    n0, n1, n2 = args.shape
    nbytes, N, M = two_pass_bytes(n0, n1, n2)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    plan = fft3d.Plan(n0, n1, n2)
    x = torch.empty((n0, n1, n2), dtype=torch.float32, device=dev)
    S = None
    if args.field == "spectrum":
        S = make_field_shape(n0, n1, n2)
        Sd = torch.from_numpy(S).to(dev)
        plan.c2r(Sd.data_ptr(), x.data_ptr(), sptr)  # the real field (setup)
        del Sd
    else:
        gen = torch.Generator(device=dev)
        gen.manual_seed(1408)
        x.uniform_(-1.0, 1.0, generator=gen)
    X = torch.empty((n0, n1, n2 // 2 + 1), dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    if not args.no_autotune:  # the library's autotuner picks the kernel shapes (untimed set-up)
        yf = y.view(-1)
        st = fft3d.fft3d_autotune(plan.handle, yf.data_ptr(), X.data_ptr(), 3, sptr)
        if st != fft3d.FFT3D_OK:
            raise fft3d.Fft3dError(st, "fft3d_autotune")

    def step():
        plan.r2c(x.data_ptr(), X.data_ptr(), sptr)
        plan.c2r(X.data_ptr(), y.data_ptr(), sptr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    def timed_region():
        sampler = ClockSampler(local_rank)
        sampler.start()
        time.sleep(1.0)
        fft3d.fft3d_set_profiling(plan.handle, True)
        ms_total = time_steps(step, stream, args.steps)
        fft3d.fft3d_set_profiling(plan.handle, False)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        prof = fft3d.fft3d_profile_read(plan.handle)
        if world > 1:
            ms_total = max_over_ranks([ms_total], dev)[0]
            dist.barrier()
        return ms_total, clocks, prof

    ms_total, clocks, prof = timed_region()
    first = None
    if clocks_rejected(clocks, world, dev):  # a slowed-down or clock-locked GPU: measure once more
        first = {"ms_per_step": ms_total / args.steps, "clocks": clocks}
        ms_total, clocks, prof = timed_region()
    ms = ms_total / args.steps
    value = world * nbytes / (ms * 1e-3) / 1e9
    launches = args.steps * (fft3d.fft3d_launches_per_call(plan.handle, -1) + fft3d.fft3d_launches_per_call(plan.handle, 1))

    # dominant kernel (pass) and its roofline
    names = fft3d.pass_names()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(1, prof[dom][1])
    dom_bytes = fft3d.fft3d_pass_bytes(plan.handle, names.index(dom))
    peak, peak_kind = measured_peak_hbm()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(dom, f"{n0}x{n1}x{n2}"), "kernel": dom, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms}
    passes = {k: {"avg_ms": v[0] / v[1], "launches": v[1],
                  "gbs": fft3d.fft3d_pass_bytes(plan.handle, names.index(k)) / (v[0] / v[1] * 1e-3) / 1e9}
              for k, v in prof.items() if v[1]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(n, args),
        "frac_of_8tbs": value / world / 8000.0, "frac_of_measured_copy": value / world / peak,
        "roofline": roofline, "passes": passes, "gpu_launches": launches, "clocks": clocks,
        "plan": plan.describe(), "choices": fft3d.fft3d_get_choices(plan.handle),
        "autotuned": not args.no_autotune,
    }
    if first is not None:
        line["remeasured"] = {"reason": "clock record of the first timed region rejected", "first": first}

    # comparator: the explicit-transpose variant (+1 pass), and with transpose-back (+2)
    if not args.no_variants:
        variants = {}
        for name, flags in (("explicit_transpose", fft3d.FFT3D_FLAG_EXPLICIT_TRANSPOSE),
                            ("explicit_transpose_back", fft3d.FFT3D_FLAG_EXPLICIT_TRANSPOSE
                             | fft3d.FFT3D_FLAG_TRANSPOSE_BACK),
                            ("fused_plane", fft3d.FFT3D_FLAG_FUSED_PLANE),
                            ("cluster_plane", fft3d.FFT3D_FLAG_CLUSTER_PLANE)):
            vp = fft3d.Plan(n0, n1, n2, flags=flags)

            def vstep(vp=vp):
                vp.r2c(x.data_ptr(), X.data_ptr(), sptr)
                vp.c2r(X.data_ptr(), y.data_ptr(), sptr)

            for _ in range(3):
                vstep()
            vms = time_steps(vstep, stream, max(5, args.steps // 2)) / max(5, args.steps // 2)
            variants[name] = {"ms_per_step": vms, "gbs_effective": nbytes / (vms * 1e-3) / 1e9,
                              "slowdown_vs_transpose_free": vms / ms, "plan": vp.describe()}
            vp.close()
        # FFTW's padded real layout, transformed in place (one 0.54 GB buffer
        # instead of two); the unnormalised round trips scale the values by N
        # per step, which does not change the work
        H = n2 // 2 + 1
        vp = fft3d.Plan(n0, n1, n2, flags=fft3d.FFT3D_FLAG_PADDED_REAL)
        buf = torch.zeros((n0, n1, 2 * H), dtype=torch.float32, device=dev)
        buf[..., :n2] = x

        def istep(vp=vp):
            vp.r2c(buf.data_ptr(), buf.data_ptr(), sptr)
            vp.c2r(buf.data_ptr(), buf.data_ptr(), sptr)

        for _ in range(3):
            istep()
        vms = time_steps(istep, stream, max(5, args.steps // 2)) / max(5, args.steps // 2)
        variants["in_place_padded"] = {"ms_per_step": vms, "gbs_effective": nbytes / (vms * 1e-3) / 1e9,
                                       "slowdown_vs_transpose_free": vms / ms, "plan": vp.describe()}
        vp.close()
        del buf
        # c2r that leaves its input intact (first column pass into workspace)
        vp = fft3d.Plan(n0, n1, n2, flags=fft3d.FFT3D_FLAG_PRESERVE_INPUT)

        def pstep(vp=vp):
            vp.r2c(x.data_ptr(), X.data_ptr(), sptr)
            vp.c2r(X.data_ptr(), y.data_ptr(), sptr)

        for _ in range(3):
            pstep()
        vms = time_steps(pstep, stream, max(5, args.steps // 2)) / max(5, args.steps // 2)
        variants["preserve_input"] = {"ms_per_step": vms, "gbs_effective": nbytes / (vms * 1e-3) / 1e9,
                                      "slowdown_vs_transpose_free": vms / ms, "plan": vp.describe()}
        vp.close()
        # the FP64 path (FFT3D_F64: double data, runtime-length kernels); its
        # minimum bytes are twice the FP32 step's
        vp = fft3d.Plan(n0, n1, n2, dtype=fft3d.FFT3D_F64)
        x64 = x.double()
        X64 = torch.empty((n0, n1, H), dtype=torch.complex128, device=dev)
        y64 = torch.empty_like(x64)

        def dstep(vp=vp):
            vp.r2c(x64.data_ptr(), X64.data_ptr(), sptr)
            vp.c2r(X64.data_ptr(), y64.data_ptr(), sptr)

        for _ in range(3):
            dstep()
        vms = time_steps(dstep, stream, max(5, args.steps // 2)) / max(5, args.steps // 2)
        vp.r2c(x64.data_ptr(), X64.data_ptr(), sptr)
        vp.c2r(X64.data_ptr(), y64.data_ptr(), sptr)
        torch.cuda.synchronize(dev)
        rt = float((y64 / (n0 * n1 * n2) - x64).norm() / x64.norm())
        variants["fp64"] = {"ms_per_step": vms, "gbs_effective": 2 * nbytes / (vms * 1e-3) / 1e9,
                            "slowdown_vs_transpose_free": vms / ms, "round_trip_rel_l2": rt,
                            "plan": vp.describe()}
        vp.close()
        del x64, X64, y64
        line["variants"] = variants

    # tensor-core radix-16 forms (split-BF16 x3, FP16) of the same step, with
    # their accuracy against the exact spectrum N*S of the field (x = c2r(S)),
    # or (uniform field) against the FP32 path's spectrum
    if not args.no_variants or args.tc:
        Nn = float(n0 * n1 * n2)
        if S is not None:
            Sref = Nn * torch.from_numpy(S).to(dev)  # complex64 copy; differences in FP64 per chunk
        else:
            plan.r2c(x.data_ptr(), X.data_ptr(), sptr)
            Sref = X.clone()

        def rel_vs_exact(Xc):
            num = 0.0
            den = 0.0
            step = max(1, (1 << 26) // (n1 * (n2 // 2 + 1)))  # about 512 MB of complex128 per chunk
            for a0 in range(0, n0, step):
                r = Sref[a0:a0 + step].to(torch.complex128)
                d = Xc[a0:a0 + step].to(torch.complex128) - r
                num += float(torch.sum(d.real ** 2 + d.imag ** 2))
                den += float(torch.sum(r.real ** 2 + r.imag ** 2))
            return (num / den) ** 0.5

        plan.r2c(x.data_ptr(), X.data_ptr(), sptr)
        tc = {"fp32": {"ms_per_step": ms, "rel_l2_r2c_vs_exact": rel_vs_exact(X)}}
        for name, dt in (("tc_bf16x3", fft3d.FFT3D_F32_TC_BF16X3), ("tc_f16", fft3d.FFT3D_F32_TC_F16)):
            tp = fft3d.Plan(n0, n1, n2, dtype=dt)
            tp.r2c(x.data_ptr(), X.data_ptr(), sptr)
            err = rel_vs_exact(X)

            def tstep(tp=tp):
                tp.r2c(x.data_ptr(), X.data_ptr(), sptr)
                tp.c2r(X.data_ptr(), y.data_ptr(), sptr)

            for _ in range(3):
                tstep()
            tms = time_steps(tstep, stream, max(5, args.steps // 2)) / max(5, args.steps // 2)
            tc[name] = {"ms_per_step": tms, "gbs_effective": nbytes / (tms * 1e-3) / 1e9,
                        "rel_l2_r2c_vs_exact": err, "speed_vs_fp32": ms / tms, "plan": tp.describe()}
            tp.close()
        tc["reference"] = "exact spectrum N*S" if S is not None else "FP32 path spectrum"
        line["tensor_core_forms"] = tc
        del Sref

    # pseudo-spectral nonlinear term at 256^3 (3 velocity spectra in, 6 dealiased
    # product spectra out), replayed as one CUDA graph
    if not args.no_variants:
        m = 256
        nl = fft3d.NonlinearTerm(m, m, m)
        import synth
        U = torch.from_numpy(synth.spectral_velocity(m, m, m, seed=synth.seed_for_config(4)).astype(np.complex64)).to(dev)
        out = torch.empty((6, m, m, m // 2 + 1), dtype=torch.complex64, device=dev)
        Mc = m * m * (m // 2 + 1)
        ns = torch.cuda.Stream(dev)
        ns.wait_stream(stream)
        with torch.cuda.stream(ns):
            for _ in range(3):
                nl(U, out=out, stream=ns)
            reps = 50
            nms = time_steps(lambda: nl(U, out=out, stream=ns), ns, reps) / reps
        run_bytes = 360 * Mc        # bytes of the five passes as run (3+3 inverse, 6+6 forward, fused rows)
        line["nonlinear_256"] = {"ms_per_application": nms, "gbs_passes_run": run_bytes / (nms * 1e-3) / 1e9,
                                 "passes_run_bytes": run_bytes, "launches": fft3d.fft3d_nonlinear_launches(nl.handle),
                                 "graph": True}
        nl.close()
        del U, out

    # one Heun step of the pseudo-spectral Navier-Stokes equations at 256^3
    # (nonlinear term twice + two fused stage kernels), replayed as one graph
    if not args.no_variants:
        m = 256
        ns = fft3d.NavierStokes(m, m, m)
        import synth
        U = torch.from_numpy(synth.spectral_velocity(m, m, m, seed=synth.seed_for_config(4)).astype(np.complex64)).to(dev)
        Mc = m * m * (m // 2 + 1)
        nss = torch.cuda.Stream(dev)
        nss.wait_stream(stream)
        with torch.cuda.stream(nss):
            for _ in range(3):
                ns.step(U, 0.01, 1e-3, stream=nss)
            reps = 20
            sms = time_steps(lambda: ns.step(U, 0.01, 1e-3, stream=nss), nss, reps) / reps
        # two nonlinear terms as run, and the two stage passes: u (3 fields) in,
        # the six products read only inside the 2/3 rule (fraction f of the bins),
        # u* and the accumulator out (stage 1); u*, products, accumulator in, u out (stage 2)
        kept = (2 * ((m - 1) // 3) + 1) ** 2 * ((m - 1) // 3 + 1)
        f = kept / Mc
        run_bytes = int(2 * 360 * Mc + 8 * Mc * ((3 + 6 * f + 6) + (3 + 6 * f + 3 + 3)))
        line["navier_stokes_256"] = {"ms_per_step": sms, "gbs_passes_run": run_bytes / (sms * 1e-3) / 1e9,
                                     "passes_run_bytes": run_bytes, "launches": fft3d.fft3d_ns_launches(ns.handle),
                                     "graph": True, "scheme": "Heun RK2, nu = 0.01, dt = 1e-3"}
        ns.close()
        del U

    # grouped uneven batch: 64^3, 96^3, 128^3, 192^3, 160^3 x 4 fields, r2c + c2r,
    # each direction one graph launch, shapes autotuned
    if not args.no_variants:
        gdims = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 192, 192), (160, 160, 160)]
        grp = fft3d.Group(gdims, [4] * len(gdims))
        gin, gmid, gout = [], [], []
        for (a0, a1, a2) in gdims:
            gin.append(torch.randn((4, a0, a1, a2), device=dev))
            gmid.append(torch.empty((4, a0, a1, a2 // 2 + 1), dtype=torch.complex64, device=dev))
            gout.append(torch.empty((4, a0, a1, a2), device=dev))
        for i in range(len(gdims)):
            fft3d.fft3d_autotune(fft3d.fft3d_group_plan_at(grp.handle, i), gin[i].data_ptr(), gmid[i].data_ptr(), 3,
                                 sptr)
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            def gstep():
                grp.r2c(gin, gmid, stream=gs.cuda_stream)
                grp.c2r(gmid, gout, stream=gs.cuda_stream)
            for _ in range(3):
                gstep()
            reps = 50
            gms = time_steps(gstep, gs, reps) / reps
        gbytes = sum(2 * 4 * (4 * a0 * a1 * a2 + 40 * a0 * a1 * (a2 // 2 + 1)) for (a0, a1, a2) in gdims)
        line["grouped_uneven"] = {"us_per_r2c_c2r": gms * 1e3, "gbs_passes_run": gbytes / (gms * 1e-3) / 1e9,
                                  "sizes": [f"{a}^3" for (a, _, _) in gdims], "fields_per_size": 4,
                                  "launches": fft3d.fft3d_group_launches(grp.handle, -1)
                                  + fft3d.fft3d_group_launches(grp.handle, 1), "graphs_per_step": 2}
        grp.close()
        del gin, gmid, gout

    # end to end through the C ABI with host buffers: every step copies its
    # input field host -> device (pinned), runs r2c + c2r, and copies the result
    # back.  Reported two ways: a stream of steps, double-buffered so that the
    # copies of one step overlap the other direction's copies and the compute
    # of its neighbours (copy streams in and out, events between them), and a
    # single isolated step (copy in, compute, copy out, one after the other).
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        sets = [(x, X, y), (torch.empty_like(x), torch.empty_like(X), torch.empty_like(y))]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "comp", "out")}
        for k in ev:
            for e_ in ev[k]:
                e_.record(stream)

        def pstep(i):
            xb, Xb, yb = sets[i % 2]
            s_in.wait_event(ev["comp"][i % 2])  # x of this set is free once its last r2c ran
            with torch.cuda.stream(s_in):
                xb.copy_(xh, non_blocking=True)
            ev["in"][i % 2].record(s_in)
            stream.wait_event(ev["in"][i % 2])
            stream.wait_event(ev["out"][i % 2])  # y of this set has been copied out
            plan.r2c(xb.data_ptr(), Xb.data_ptr(), sptr)
            plan.c2r(Xb.data_ptr(), yb.data_ptr(), sptr)
            ev["comp"][i % 2].record(stream)
            s_out.wait_event(ev["comp"][i % 2])
            with torch.cuda.stream(s_out):
                yh.copy_(yb, non_blocking=True)
            ev["out"][i % 2].record(s_out)

        for i in range(4):
            pstep(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        esteps = max(6, args.steps // 4)
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for i in range(esteps):
            pstep(i)
        stream.wait_stream(s_out)
        b_.record(stream)
        b_.synchronize()
        ems = a_.elapsed_time(b_) / esteps

        def estep():
            x.copy_(xh, non_blocking=True)
            plan.r2c(x.data_ptr(), X.data_ptr(), sptr)
            plan.c2r(X.data_ptr(), y.data_ptr(), sptr)
            yh.copy_(y, non_blocking=True)

        for _ in range(3):
            estep()
        torch.cuda.synchronize()
        sms_ = time_steps(estep, stream, max(5, args.steps // 4)) / max(5, args.steps // 4)
        if world > 1:
            ems, sms_ = max_over_ranks([ems, sms_], dev)
        line["e2e"] = {"value": world * nbytes / (ems * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ems,
                       "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
                       "mode": "stream of steps, double-buffered: copies in / out on their own streams",
                       "single_step_ms": sms_,
                       "single_step_value": world * nbytes / (sms_ * 1e-3) / 1e9}
        del sets

    # FP64 CPU oracle on the host cores (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        xs = x.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        Xo = oracle.r2c3d(xs)
        oracle.c2r3d(Xo, n2)
        t_cpu = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nbytes / t_cpu / 1e9, "unit": UNIT, "cores": oracle.threads(),
                                "kind": "oracle", "ms_per_step": 1e3 * t_cpu,
                                "sample": f"one full {n0}x{n1}x{n2} r2c+c2r of the same field in FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
