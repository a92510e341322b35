"""Benchmark: MLUPS of the fractional-ADE lattice Boltzmann time step on GB300.

One benchmark step = one full run of the workload: reset to the initial
condition (untimed), then all of its lattice time steps (timed), each time step
being the whole hot path: fractional terms along every axis, equilibrium,
collision, streaming, Dirichlet walls and new concentration.  L2 is flushed
(a 512 MiB write) before every benchmark step; within a run the state stays
resident, as in any real run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload mrt_aniso_512] [--precision P]

N > 1 runs under torchrun, one independent replica per GPU (the workload does
not shard), timing is the max over ranks and ``value`` counts every rank's
lattice updates.  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
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

METRIC = "MLUPS per GB300 (full step incl. fractional operator)"
UNIT = "MLUPS"

WORKLOADS = {
    "mrt_aniso_512": dict(
        desc="2-D anisotropic fractional ADE, D2Q5 MRT, 512x512, alpha=(1.5,1.8), p=(0.3,0.7), g=(1,1), "
             "D=diag(2e-3,5e-4), u=(0.05,0.02) lattice units, free rates U[0.8,1.9] seed 2, "
             "Dirichlet C=0, 5x5 unit-mass pulse, 5000 steps",
        default_precision="bf16split"),
    "fp64_bgk_64": dict(desc="2-D D2Q5 BGK 64x64 FP64, alpha=1.7, 200 steps", default_precision="fp64"),
    "batch64": dict(desc="64 independent 2-D D2Q5 MRT problems, sides U{128,256,384,512,768,1024} (seed 4), "
                         "alpha~U[1.2,2], p~U[0,1], D~U[1e-4,3e-3] diagonal, |u|<=0.08, Gaussian pulses sigma~U[2,6], "
                         "free rates U[0.8,1.9], 1000 steps each, grouped launches",
                    default_precision="bf16split"),
    "inverse_256": dict(desc="inverse problem: 2-D D2Q5 MRT 256x256, alpha=(1.45,1.75), p=(0.35,0.65), "
                             "D=diag(1.5e-3,7e-4), u=(0.04,-0.01); loss over 10 snapshots of 3000 steps + N(0,1e-4) noise; "
                             "one bench step = one loss+gradient evaluation (forward, checkpointed recompute, adjoint; "
                             "checkpoint every 100); value counts forward lattice updates",
                        default_precision="fp32"),
    "mrt3d_128": dict(desc="3-D D3Q7 MRT 128^3 with the 256^3 workload's parameters (profiling captures only)",
                      default_precision="tf32split"),
    "mrt3d_256": dict(desc="3-D fractional ADE, D3Q7 MRT, 256^3, alpha=(1.6,1.6,1.9), p=(0.5,0.2,0.8), g=(1,1,1), "
                           "D=diag(1e-3,1e-3,4e-4), u=(0.03,0,0) lattice units, free rates U[0.8,1.9] seed 3, "
                           "Dirichlet C=0, unit-mass Gaussian sigma=3, 2000 steps",
                      default_precision="tf32split"),
}

# measured peaks (driver-written), with the profiling recipe's fallback
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
SMS = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 rate


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def cublas_tflops(kind: str) -> float:
    """Dense cuBLAS GEMM throughput on this GPU for `kind` ("tf32" or "fp64"): context
    for the split-tf32 and FP64 operator fractions (the roofline peak itself stays the
    measured bf16 figure times the nominal ratio)."""
    import torch
    n = 8192 if kind == "tf32" else 4096
    dt = torch.float32 if kind == "tf32" else torch.float64
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = kind == "tf32"
    try:
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        for _ in range(2):
            a @ b
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10 if kind == "tf32" else 3
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            a @ b
        e1.record()
        torch.cuda.synchronize()
        return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old


def make_workload(name):
    """(problems, initial fields, lattice steps) of a named workload."""
    from paper_1706_09161_gb300 import workloads as W
    if name == "batch64":
        return W.batch64()
    if name == "inverse_256":
        pb, C0, snaps = W.inverse_256()
        return [pb], [C0], snaps[-1]
    pb, C0, n = W.mrt3d_256(128) if name == "mrt3d_128" else getattr(W, name)()
    return [pb], [C0], n


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle legs

def oracle_sample(pb, C0, nsteps):
    """Run the FP64 CPU oracle for nsteps; returns (seconds, C, threads)."""
    import torch
    from oracle import lbm_oracle as O
    ops = O.Operators(pb)
    f = O.init_populations(ops, torch.tensor(C0))
    t0 = time.perf_counter()
    for _ in range(nsteps):
        f = O.step(ops, f)
    dt = time.perf_counter() - t0
    return dt, O.concentration(f).numpy(), torch.get_num_threads()


# --------------------------------------------------------------------------- main

def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    probs, fields, nlbm = make_workload(args.workload)
    nodes = sum(pb.nodes for pb in probs)
    sample = max(1, min(nlbm, args.ref_sample, int(2e7 // nodes) or 1))
    for _ in range(args.warmup):
        for pb, C0 in zip(probs, fields):
            oracle_sample(pb, C0, 1)
    times = []
    threads = 1
    for _ in range(args.steps):
        dt = 0.0
        for pb, C0 in zip(probs, fields):
            t, _, threads = oracle_sample(pb, C0, sample)
            dt += t
        times.append(dt)
    total = sum(times)
    mlups = nodes * sample * args.steps / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                       "lbm_steps_per_bench_step": sample, "note": "bounded sample of the workload's run"},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} lattice steps of {args.workload} per bench step"},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def job_value(local_ms, units_per_rank, world, dist=None, device=None):
    """Whole-job throughput in MLUPS: every rank's lattice updates over the slowest rank's
    time (max over ranks through an all-reduce), and that time in ms."""
    t = float(local_ms)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_rank / (t * 1e-3) / 1e6, t


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(workload, kernel, precision):
    """DRAM bytes per launch from the committed ncu summary of this workload and precision
    form, or None if there is none or the kernel changed since."""
    kernel_key = f"{workload}:{kernel}"
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(kernel_key)
    if not rec or rec.get("precision") != precision:
        return None
    if rec.get("source_sha") != source_sha(rec["sources"]):
        return None
    return rec.get("bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="mrt_aniso_512", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None)
    ap.add_argument("--ref-sample", type=int, default=40, help="lattice steps per reference-arm bench step")
    ap.add_argument("--cpu-sample", type=int, default=800, help="lattice steps of the cpu_baseline leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch configuration")
    ap.add_argument("--lattice-steps", type=int, default=None,
                    help="override the workload's lattice steps per bench step (profiling runs only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1706_09161_gb300 import build as _build
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()
    from paper_1706_09161_gb300 import lbm

    probs, fields, nlbm = make_workload(args.workload)
    if args.lattice_steps:
        nlbm = args.lattice_steps
    precision = args.precision or WORKLOADS[args.workload]["default_precision"]
    batched = len(probs) > 1
    nodes = sum(pb.nodes for pb in probs)
    lat = lbm.Batch(probs, fields, precision) if batched else lbm.Lattice(probs[0], fields[0], precision)
    # launch configuration chosen by the library's autotuner on this workload (untimed
    # setup; the populations are restored afterwards)
    tuned = None if args.no_autotune else lat.autotune(64)
    stream = torch.cuda.ExternalStream(lat.stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    inverse = args.workload == "inverse_256"
    if inverse:
        from paper_1706_09161_gb300 import workloads as W
        _, _, snaps = W.inverse_256()
        # synthetic observations: the GPU forward run itself plus N(0, (1e-4)^2) noise
        obs = []
        lat.reset()
        t = 0
        for ts in snaps:
            lat.step(ts - t)
            t = ts
            obs.append(lat.C())
        obs = np.stack(obs) + W.observation_noise((len(snaps),) + probs[0].shape)

    def one_run():
        lat.reset()
        flush.add_(1.0)  # L2 flush on torch's stream
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        if inverse:
            lat.grad(snaps, obs, 100)
        else:
            lat.step(nlbm)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    for _ in range(args.warmup):
        one_run()
    warm_status = lbm.lbm_sync(lat.h)  # a latched instability does not change the work timed
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_ms = []
    for _ in range(args.steps):
        t_ms.append(one_run())
    torch.cuda.synchronize()
    clk = clocks.stop()
    rc = lbm.lbm_sync(lat.h)
    value, total_ms = job_value(sum(t_ms), nodes * nlbm * args.steps, world, dist, "cuda")
    lps = lat.launches_per_step
    # 0: the fused step, one cooperative launch per lbm_step call of up to 4096 steps
    gpu_launches = args.steps * (nlbm * lps if lps > 0 else -(-nlbm // 4096))
    if inverse:
        d0 = probs[0].d
        # forward + checkpointed recompute (d+1 each) and adjoint (step, d transposes, d G sums, combine)
        gpu_launches = args.steps * nlbm * (2 * (d0 + 1) + 2 + 2 * d0)

    # ---- end to end through the C ABI with pinned host buffers
    pins = [torch.from_numpy(np.ascontiguousarray(C0)).pin_memory() for C0 in fields]
    outs = [torch.empty(p.shape, dtype=torch.float64).pin_memory() for p in pins]
    e2e_s = []
    if inverse:
        obs_pin = torch.from_numpy(np.ascontiguousarray(obs)).pin_memory()
    for k in range(args.steps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, p in enumerate(pins):
            if batched:
                lat.set_C(i, p.numpy())
            else:
                lat.set_C(p.numpy())
        if inverse:  # observations go host -> device inside lbm_grad; loss and gradient come back
            lat.grad(snaps, obs_pin.numpy(), 100)
            e2e_s.append(time.perf_counter() - t0)
            continue
        lat.step(nlbm)
        for i, o in enumerate(outs):
            # data is copied; a latched instability is only reported
            rc_e2e = (lbm._lib.lbm_batch_read_C(lat.h, i, lbm._dptr(o.numpy())) if batched
                      else lbm._lib.lbm_read_C(lat.h, lbm._dptr(o.numpy())))
            if rc_e2e not in (lbm.LBM_OK, lbm.LBM_ERR_UNSTABLE):
                raise lbm.LBMError(rc_e2e, "read C")
        e2e_s.append(time.perf_counter() - t0)
    e2e_val, _ = job_value(1e3 * sum(e2e_s), nodes * nlbm * args.steps, world, dist, "cuda")
    io_bytes = int(sum(C0.size for C0 in fields) * 8)
    h2d_bytes, d2h_bytes = io_bytes, io_bytes
    if inverse:
        h2d_bytes = io_bytes + int(obs.size * 8)
        d2h_bytes = 8 * (1 + 4 * probs[0].d)

    # ---- dominant kernel, timed live with events on the library stream
    nprof = min(nlbm, 200)
    lat.reset()
    ms_frac, ms_cs = lat.profile(nprof)
    d = probs[0].d
    Q = 2 * d + 1
    peaks, peak_src = load_peaks()
    elem = 8 if precision == "fp64" else 4
    flops = float(sum(2.0 * pb.nodes * sum(pb.grid) for pb in probs))  # 2 side flops per node per axis
    dur = ms_frac / nprof * 1e-3
    achieved = flops / dur / 1e12
    split_products = {"bf16split": 3, "tf32split": 3, "bf16x5split": 5}
    if precision in split_products:
        bound = "tensor"
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        if precision == "tf32split":
            peak = peak / 2.0  # nominal tf32/bf16 ratio
    else:
        bound = "alu"
        if precision == "fp32":
            # FP32 FMA lanes x 2 flops x max SM clock
            peak = SMS * FP32_LANES_PER_SM * 2.0 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        else:
            peak = FP64_NOMINAL_TFLOPS
    roof_op = {"kernel": "fractional_operator", "bound": bound, "achieved": achieved, "peak": peak,
               "unit": "TFLOP/s", "frac": achieved / peak,
               "traffic": traffic_for(args.workload, "fractional_operator", precision),
               "algorithmic_per_launch": flops, "launch_ms": dur * 1e3, "peak_source": peak_src}
    if precision in split_products:
        # the split forms issue three (hi*hi, hi*lo, lo*hi) or five products per
        # algorithmic one: the tensor pipe's own load
        npr = split_products[precision]
        roof_op["executed_per_launch"] = npr * flops
        roof_op["executed_frac"] = npr * achieved / peak
    if precision in ("tf32split", "fp64"):
        kind = "tf32" if precision == "tf32split" else "fp64"
        roof_op[f"cublas_{kind}_tflops_measured"] = cublas_tflops(kind)
    bytes_ = float(nodes) * (2 * Q * elem + d * elem + elem)
    dur = ms_cs / nprof * 1e-3
    achieved = bytes_ / dur / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    roof_cs = {"kernel": "collide_stream", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": achieved / peak, "traffic": traffic_for(args.workload, "collide_stream", precision),
               "algorithmic_per_launch": bytes_, "launch_ms": dur * 1e3, "peak_source": peak_src}
    if precision in split_products:
        # the kernel also writes the operator's operands of the new C: its hi/lo split
        # (x contiguous) and, for tf32 on the TMA-fed marches (one operator and one
        # collide-stream launch per step), the copies regrouped along y (and z)
        per_node = 8 if precision == "tf32split" else 4
        if precision == "tf32split" and lat.launches_per_step == 2:
            per_node += 8 * (d - 1)
        ex = bytes_ + float(nodes) * per_node
        roof_cs["executed_per_launch"] = ex
        roof_cs["executed_frac"] = ex / dur / 1e9 / peak
    # the dominant kernel is the roofline; the other one is reported beside it
    roof, roof_other = (roof_op, roof_cs) if ms_frac >= ms_cs else (roof_cs, roof_op)
    roof["other_kernel_ms"] = {"fractional_operator": ms_frac / nprof, "collide_stream": ms_cs / nprof}

    # ---- CPU baseline (oracle) and accuracy against it, rank 0 at N = 1 only
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = max(2, min(nlbm, args.cpu_sample, int(1e8 // nodes)))
        dt, refs, threads = 0.0, [], 1
        for pb, C0 in zip(probs, fields):
            t, C_ref, threads = oracle_sample(pb, C0, ns)
            dt += t
            refs.append(C_ref)
        cpu = {"value": nodes * ns / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {ns} of {nlbm} lattice steps of {args.workload} (FP64, torch CPU)"}
        lat.reset()
        lat.step(ns)
        got = [lat.C(i) for i in range(len(probs))] if batched else [lat.C()]
        num = sum(float(np.sum((g - r) ** 2)) for g, r in zip(got, refs))
        den = sum(float(np.sum(r ** 2)) for r in refs)
        accuracy = {"rel_l2_vs_fp64_oracle": float(np.sqrt(num / den)), "lattice_steps": ns}

    lat.close()

    # the same workload in the five-product bf16 form, the split form that meets the 1e-5
    # error target: timed the same way (library stream, L2 flushed per bench step) and
    # checked against the same oracle sample
    at_target = None
    if accuracy is not None and precision == "bf16split" and not batched and not inverse:
        alt = "bf16x5split"
        with lbm.Lattice(probs[0], fields[0], alt) as l5:
            tuned5 = None if args.no_autotune else l5.autotune(64)
            s5 = torch.cuda.ExternalStream(l5.stream)

            def run5():
                l5.reset()
                flush.add_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s5)
                l5.step(nlbm)
                e1.record(s5)
                e1.synchronize()
                return e0.elapsed_time(e1)

            for _ in range(args.warmup):
                run5()
            ms5 = sum(run5() for _ in range(args.steps)) / args.steps
            st5 = lbm.lbm_sync(l5.h)
            l5.reset()
            l5.step(accuracy["lattice_steps"])
            C5 = l5.C()
        err5 = float(np.sqrt(np.sum((C5 - refs[0]) ** 2) / np.sum(refs[0] ** 2)))
        at_target = {"precision": alt, "dtype": "f32+bf16x5", "value": nodes * nlbm / (ms5 * 1e-3) / 1e6,
                     "unit": UNIT, "ms_per_step": ms5, "launch_config": tuned5 if tuned5 is not None else "built-in",
                     "accuracy": {"rel_l2_vs_fp64_oracle": err5, "lattice_steps": accuracy["lattice_steps"]},
                     "status": lbm.lbm_strerror(st5)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16split": "f32+bf16x3", "tf32split": "f32+tf32x3",
                          "bf16x5split": "f32+bf16x5"}[precision],
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                           "precision": precision, "lattice_steps_per_bench_step": nlbm,
                           "nodes": nodes, "problems": len(probs), "parallelism": f"replicas x{world}",
                           "l2": "flushed (512 MiB write) before every bench step; state L2-resident within a run",
                           "launch_config": tuned if tuned is not None else "built-in"},
                "roofline": roof, "roofline_other": roof_other, "cpu_baseline": cpu, "accuracy": accuracy,
                "at_error_target": at_target,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                        "d2h_bytes_per_step": d2h_bytes},
                "gpu_launches": gpu_launches, "clocks": clk,
                "status": lbm.lbm_strerror(rc if rc else warm_status)}
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
