#!/usr/bin/env python3
"""Throughput of the LB + raspberry-coupling step on the GB300.

One step = one pass of the whole hot path over the lattice: bodies half-kick
and drift, virtual sites, bead coupling (interpolate, drag, spread, reduce),
fused collide-and-stream with bounce-back, bodies second half-kick.

Default workload: 256^3 periodic D3Q19 box, MRT (nu = 0.016) with thermal
fluctuations (kT = 1e-4, Philox noise), populations stored in FP32 as
deviations from w_i rho0, 64 prolate ellipsoidal raspberries (aspect 2-4,
semi-axes 2-8, 1 bead per unit area, ~23k beads) at seeded positions and
orientations. Inputs are synthetic and seeded; the state (1.27 GB of
populations) is far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
WORKLOAD = "ellipsoids64_256^3_mrt_kT_fp32"
METRIC = "MLUPS incl. coupling (D3Q19 MRT + fluctuations + raspberry coupling)"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d and d[k]:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def copy_ceiling(torch, stream, nbytes=2 << 30, reps=10):
    """Live device-copy bandwidth (read + write bytes per second) of a plain
    torch copy between two buffers far larger than L2, timed with events on
    the given stream: a second denominator beside the roofline peak."""
    n = nbytes // 4
    with torch.cuda.stream(stream):
        src = torch.ones(n, dtype=torch.float32, device="cuda")
        dst = torch.empty_like(src)
        for _ in range(3):
            dst.copy_(src)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            dst.copy_(src)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del src, dst
    torch.cuda.empty_cache()
    return 2.0 * n * 4 / (ms * 1e-3) / 1e9


def kernel_source_hash():
    """Hash of what the collide-and-stream kernels are compiled from: the
    collision and device headers, the fluid-kernel part of lb_fluid.cu and
    the parameter structs (CollParams, FluidArgs) of the shared header, so
    that unrelated edits keep committed counters valid."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_01829_gb300", "csrc")
    for f in ("lb_collide.cuh", "lb_device.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    # the fluid-kernel part of lb_fluid.cu (pore wall masks, collide and stream)
    src = open(os.path.join(csrc, "lb_fluid.cu"), "rb").read()
    h.update(src[:src.index(b"// ------------------------------------------------------------ population I/O")])
    hdr = open(os.path.join(csrc, "lb_internal.h"), "rb").read()
    start = hdr.index(b"struct CollParams")
    end = hdr.index(b"};", hdr.index(b"struct FluidArgs")) + 2
    h.update(hdr[start:end])
    return h.hexdigest()[:16]


def ncu_entry(key):
    """An entry of the committed ncu summary, or None if there is none or the
    kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "collide_stream_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        e = json.load(open(p)).get(key)
        if not e or e.get("kernel_source_hash") != kernel_source_hash():
            return None
        return e
    except Exception:
        return None


def ncu_traffic(workload_key):
    """DRAM bytes per launch of the collide kernel from the committed ncu
    summary, or None if none exists or the kernel changed since."""
    e = ncu_entry(workload_key)
    return None if e is None else float(e["dram_bytes_per_launch"])


# FP64 pipe of GB300: the nominal 1.25 TFLOP/s FP64 over 152 SMs at 2.07 GHz
# is 2 FMA lanes per SM per clock, i.e. this many FP64 thread-instructions/s
FP64_PIPE_INSTR_PER_S = 152 * 2 * 2.07e9
FP64_NOMINAL_TFLOPS = 1.25


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


ARGS = None


def make_reducer(dist, device):
    """max over ranks of a host float (identity without a process group)."""
    def barrier_max(v):
        if dist is None:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return barrier_max


def whole_job_mlups(nodes_per_rank, steps, world_size, max_ms):
    """Weak scaling: every rank advances its own replica of `nodes_per_rank`
    nodes; the job's throughput is all ranks' node updates over the slowest
    rank's time."""
    return nodes_per_rank * steps * world_size / (max_ms * 1e-3) / 1e6


def build_workload(precision):
    from paper_1604_01829_gb300 import workloads as W
    L = ARGS.lattice if ARGS else 256
    nb = ARGS.bodies if ARGS else 64
    return W.ellipsoids_256(n_bodies=nb, L=L, precision=precision)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_1604_01829_gb300 import build, lb

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    barrier_max = make_reducer(dist, "cuda")

    def measure(precision, steps, warmup, with_clocks):
        w = build_workload(precision)
        stream = torch.cuda.Stream()
        L = lb.from_workload(w, stream=stream.cuda_stream)
        N = w.nodes
        L.lb_step(warmup)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local) if with_clocks else None
        if clocks:
            clocks.start()
        L.lb_set_timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lb_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, klaunch = L.lb_kernel_time()
        L.lb_set_timing(False)
        clk = clocks.stop() if clocks else None
        if dist is not None:
            dist.barrier()
        ms_max = barrier_max(ms)
        m, p = L.lb_conservation()   # raises on non-finite state
        res = dict(ms=ms_max, kernel_ms=kms / max(klaunch, 1), launches=klaunch, nodes=N,
                   nbeads=w.nbeads, nbodies=len(w.bodies), clocks=clk, L=L, w=w)
        return res

    main = measure(32, args.steps, args.warmup, True)
    N = main["nodes"]
    K = args.steps
    value = whole_job_mlups(N, K, ws, main["ms"])
    peak, peak_kind = measured_peak()
    bytes_per_node = 2 * 19 * 4
    achieved = bytes_per_node * N / (main["kernel_ms"] * 1e-3) / 1e9
    default_size = (args.lattice, args.bodies) == (256, 64)
    # the committed DRAM counters are for the 256^3 / 64-body workload
    traffic = ncu_traffic(WORKLOAD) if default_size else None
    copy_gbs = copy_ceiling(torch, torch.cuda.Stream())

    # end to end through the C ABI with host buffers: per step the host sets
    # the external forces of every body (H2D) and reads every body's force
    # and torque back (D2H), in one library call (lb_step_io)
    L, w = main["L"], main["w"]
    nb = len(w.bodies)
    # page-locked host buffers (torch pins them; numpy views share the memory)
    pinned = [torch.zeros(3 * nb, dtype=torch.float64).pin_memory() for _ in range(4)]
    Fext, Text, Fout, Tout = (t.numpy() for t in pinned)
    e2e_steps = 0 if args.no_e2e else max(10, min(K, 200))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.lb_step_io(Fext, Text, Fout, Tout)
    t1 = time.perf_counter()
    e2e_ms = barrier_max((t1 - t0) * 1e3 / max(e2e_steps, 1))
    e2e_value = N * ws / (e2e_ms * 1e-3) / 1e6 if e2e_steps else None
    main["L"].close()
    del main["L"]

    # FP64 populations on the same workload (the metric compares FP32 and FP64)
    fp64_line = None
    if not args.skip_fp64:
        k64 = max(3, K // 4)
        fp64 = measure(64, k64, 3, False)
        fp64_value = fp64["nodes"] * k64 * ws / (fp64["ms"] * 1e-3) / 1e6
        fp64_ach = 2 * 19 * 8 * fp64["nodes"] / (fp64["kernel_ms"] * 1e-3) / 1e9
        fp64["L"].close()
        fp64_line = {"value": round(fp64_value, 1), "unit": "MLUPS", "steps": k64,
                     "ms_per_step": round(fp64["ms"] / k64, 4),
                     "kernel_ms": round(fp64["kernel_ms"], 4),
                     "kernel_achieved_gbs": round(fp64_ach, 1),
                     "hbm_frac": round(fp64_ach / peak, 4), "bytes_per_node": 2 * 19 * 8}
        # the FP64 step is bound by the FP64 pipe: instruction counts per node
        # from the committed ncu capture of the same kernel
        ops = ncu_entry(WORKLOAD.replace("_fp32", "_fp64_ops")) if default_size else None
        if ops is not None:
            rate = fp64["nodes"] / (fp64["kernel_ms"] * 1e-3)
            pipe = ops["fp64_thread_inst_per_node"]["fp64_pipe"] * rate
            flops = ops["flops_per_node"] * rate / 1e12
            fp64_line["roofline"] = {
                "bound": "alu", "unit": "G FP64-pipe thread-instr/s",
                "achieved": round(pipe / 1e9, 1), "peak": round(FP64_PIPE_INSTR_PER_S / 1e9, 1),
                "frac": round(pipe / FP64_PIPE_INSTR_PER_S, 4),
                "peak_kind": "derived from nominal FP64 rate, SM count and clock",
                "fp64_pipe_instr_per_node": ops["fp64_thread_inst_per_node"]["fp64_pipe"],
                "achieved_tflops": round(flops, 3), "nominal_tflops": FP64_NOMINAL_TFLOPS}

    batched = None if args.skip_batched else measure_batched(args, torch, lb, barrier_max, ws)
    pore = None if args.skip_pore else measure_pore(torch, lb)
    sphere32 = None if args.skip_pore else measure_sphere32(torch, lb)
    adjoint = None if args.skip_adjoint else measure_adjoint(args, torch, lb)
    construction = None if args.skip_construction else measure_construction(args, torch, lb)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 1),
            "unit": "MLUPS",
            "n_gpus": ws,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": round(main["ms"] / K, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded ellipsoidal raspberries, Philox thermal noise)",
            "config": {"workload": WORKLOAD if (args.lattice, args.bodies) == (256, 64)
                       else f"ellipsoids{args.bodies}_{args.lattice}^3_mrt_kT_fp32",
                       "lattice": [args.lattice] * 3, "collision": "MRT",
                       "kT": 1e-4, "nu": 0.016, "bodies": main["nbodies"], "beads": main["nbeads"],
                       "storage": "fp32 deviation f - w rho0",
                       "l2": f"state {N * 76 / 1e9:.2f} GB " + ("> L2, no flush" if N * 76 > 129e6 else "fits in L2"),
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "kernel": "k_collide_stream<float,MRT,noise>",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "bytes_per_node": bytes_per_node,
                         "kernel_ms": round(main["kernel_ms"], 5),
                         "traffic": traffic,
                         "copy_ceiling_gbs": round(copy_gbs, 1),
                         "frac_of_copy_ceiling": round(achieved / copy_gbs, 4)},
            "e2e": {"value": None if e2e_value is None else round(e2e_value, 1), "unit": "MLUPS", "steps": e2e_steps,
                    "h2d_bytes_per_step": 2 * 3 * 8 * nb, "d2h_bytes_per_step": 2 * 3 * 8 * nb},
            # per step the body prologue, the coupling and the fused collide-stream
            # kernel; one finishing launch (last half kick, counter advance) per call
            "gpu_launches": 3 * K + 1,
            "fp64": fp64_line,
            "batched": batched,
            "pore": pore,
            "sphere32": sphere32,
            "adjoint": adjoint,
            "construction": construction,
            "clocks": main["clocks"],
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def measure_batched(args, torch, lb, barrier_max, ws):
    """256 independent instances of uneven size (cubic 24-64 periodic boxes and
    cylindrical pores R 8-28, each with one raspberry), FP32 MRT, advanced
    together: autotuned schedule, two-step CUDA graph. Compared with the same
    instances stepped one handle after another."""
    from paper_1604_01829_gb300 import workloads as W
    ws_list = W.batched_instances(args.batch_instances)
    stream = torch.cuda.Stream()
    B = lb.batch_from_workloads(ws_list, stream=stream.cuda_stream)
    if args.batch_schedule:
        chosen = [int(v) for v in args.batch_schedule.split(",")]
        B.lb_batch_set_schedule(*chosen)
    else:
        chosen, _ = B.lb_batch_autotune(10)
    nodes = B.lb_batch_info()["total_nodes"]
    K = args.batch_steps
    B.lb_batch_step(4)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.lb_batch_step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = barrier_max(e0.elapsed_time(e1))
    # fluid kernel alone (eager launches with events) for the roofline
    B.lb_batch_set_timing(True)
    B.lb_batch_step(20)
    kms, kn = B.lb_batch_kernel_time()
    B.lb_batch_set_timing(False)
    # the same steps with the trajectory recorder on (every 10 steps, all
    # bodies), then the GPU MSD analysis of trajectories of the analysis scale
    B.lb_batch_record_bodies(10, 1024)
    B.lb_batch_step(4)
    torch.cuda.synchronize()
    e0.record(stream)
    B.lb_batch_step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_rec = barrier_max(e0.elapsed_time(e1))
    nrec = len(B.lb_batch_get_trajectory(0, 0)[0])
    traj = measure_msd(torch, lb)
    traj.update({"record_every": 10, "records_per_body": nrec,
                 "ms_per_step_recording": round(ms_rec / K, 4),
                 "recording_overhead_pct": round(100.0 * (ms_rec - ms) / ms, 2)})
    fluid = 0
    for w in ws_list:
        if w.pore is None:
            fluid += w.nodes
        else:
            R, ax = w.pore
            n2 = [w.nx, w.ny, w.nz]
            a1, a2 = [d for d in range(3) if d != ax]
            c = 0
            for i in range(n2[a1]):
                for j in range(n2[a2]):
                    if (2 * i + 1 - n2[a1]) ** 2 + (2 * j + 1 - n2[a2]) ** 2 < math.ceil(4 * R * R):
                        c += 1
            fluid += c * n2[ax]
    B.close()
    # the same instances one handle after another (eager launches)
    K1 = max(2, K // 10)
    handles = [lb.from_workload(w, stream=stream.cuda_stream) for w in ws_list]
    for L in handles:
        L.lb_step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for L in handles:
        L.lb_step(K1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = barrier_max(e0.elapsed_time(e1))
    for L in handles:
        L.close()
    peak, kind = measured_peak()
    ach = 152.0 * fluid / (kms / max(kn, 1) * 1e-3) / 1e9
    return {"workload": f"{len(ws_list)} instances (cubic 24-64 periodic, pores R 8-28), one raspberry each, "
                        f"FP32 MRT, kT=0", "instances": len(ws_list), "nodes": nodes, "fluid_nodes": fluid,
            "steps": K, "ms_per_step": round(ms / K, 4),
            "value": round(nodes * ws * K / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "fluid_mlups": round(fluid * ws * K / (ms * 1e-3) / 1e6, 1),
            "one_by_one": {"steps": K1, "ms_per_step": round(ms1 / K1, 4),
                           "value": round(nodes * ws * K1 / (ms1 * 1e-3) / 1e6, 1)},
            "speedup_vs_one_by_one": round((ms1 / K1) / (ms / K), 2),
            "schedule": {"tile_nodes": chosen[0], "blocks_per_sm": chosen[1], "order": chosen[2]},
            "fluid_kernel": {"ms": round(kms / max(kn, 1), 4), "achieved_gbs": round(ach, 1),
                             "frac": round(ach / peak, 4), "peak_kind": kind},
            "trajectory": traj}


def measure_pore(torch, lb, steps=5000):
    """The confinement workload as configured: 48x48x96 pore R = 20 along z,
    sphere R = 4 at radial offsets 0, 0.2, 0.4, 0.6 R, MRT with fluctuations,
    repulsive wall beads (5 apart, r_p = 6.25, r_r = 0.5, epsilon = kT, all in
    lattice units = nm), centre recorded every 200 steps; 5000 steps each in
    FP32 (deviation storage) and FP64. Then the deterministic drag
    enhancement S = xi_pore / xi_0 at the same offsets in FP32 and FP64
    (paper_1604_01829_gb300.drag), and the binned pore-frame MSD of a
    trajectory of 1.2e6 records (20 radial bins, 25 lags)."""
    import numpy as np
    from paper_1604_01829_gb300 import drag as D
    from paper_1604_01829_gb300 import workloads as W
    stream = torch.cuda.Stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    betas = [0.0, 0.2, 0.4, 0.6]
    timed = {32: [], 64: []}
    rec = None
    for precision in (32, 64):
        for beta in betas:
            w = W.pore_48(offset_frac=beta, precision=precision)
            L = lb.from_workload(w, stream=stream.cuda_stream)
            L.lb_set_pore_beads(5.0, 6.25, 0.5, w.params["kT"])
            L.lb_record_bodies(200, 64)
            L.lb_step(10)
            torch.cuda.synchronize()
            e0.record(stream)
            L.lb_step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            timed[precision].append(e0.elapsed_time(e1))
            if precision == 32 and rec is None:
                rec = len(L.lb_get_trajectory(0)[0])
            L.close()
    nodes = w.nodes

    def leg(ms_list):
        ms = float(np.mean(ms_list))
        return {"steps": steps, "ms_per_step": round(ms / steps, 4),
                "value": round(nodes * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                "ms_per_step_by_offset": [round(m / steps, 4) for m in ms_list]}

    # deterministic drag enhancement (Stokes flow: BGK tau = 1, kT = 0)
    beads = W.sphere_raspberry(4.0)
    mass = 4.0 / 3.0 * math.pi * 64.0
    eta = 1.0 / 6.0
    R_h = D.pore_flux_radius(48, 96, 20.0, eta)
    Ls = [32, 48, 64, 80]
    xi0 = D.unbounded([D.pulled_drag(Lb, beads, mass, 0) for Lb in Ls], Ls, eta)
    lam = xi0 / (6 * math.pi * eta) / R_h
    S = {p: [D.pore_drag(48, 96, 20.0, beads, mass, offset=b * 20.0, precision=p) / xi0 for b in betas]
         for p in (64, 32)}
    Sx = {p: [D.pore_radial_drag(48, 96, 20.0, beads, mass, offset=b * 20.0, precision=p) / xi0 for b in betas]
          for p in (64, 32)}
    rng = np.random.default_rng(1611)
    n = 1_200_000
    X = np.empty((n, 3))
    X[:, 2] = np.cumsum(rng.normal(scale=0.3, size=n)) + 48.0
    ang = np.cumsum(rng.normal(scale=0.02, size=n))
    rad = 8.0 + 4.0 * np.sin(np.cumsum(rng.normal(scale=0.01, size=n)))
    X[:, 0] = 24.0 + rad * np.cos(ang)
    X[:, 1] = 24.0 + rad * np.sin(ang)
    lb.lb_pore_msd(X[:1000], (48, 48, 96), 2, 20.0, 20, 25)          # warm-up
    t0 = time.perf_counter()
    lb.lb_pore_msd(X, (48, 48, 96), 2, 20.0, 20, 25)
    sec = time.perf_counter() - t0
    f32 = leg(timed[32])
    return {"workload": "pore_48x48x96_R20, sphere R 4 at offsets 0, 0.2, 0.4, 0.6 R; MRT nu=0.016 kT=1e-4, "
                        "WCA wall beads 5 apart (r_p 6.25, r_r 0.5, eps kT), record every 200 steps",
            "offsets": betas, "nodes": nodes, "steps": steps, "ms_per_step": f32["ms_per_step"],
            "value": f32["value"], "unit": "MLUPS", "l2": "state 34 MB fits in L2: MLUPS only", "records": rec,
            "fp32": f32, "fp64": leg(timed[64]),
            "enhancement": {
                "protocol": "deterministic (kT = 0, BGK tau = 1, bead friction 0.3); axial: sphere moving along "
                            "the pore through fluid at rest far away (zero-flux superposition of a pulled and a "
                            "carried sphere); radial: sphere pulled towards the wall; S = xi_pore / xi_0, xi_0 "
                            "from periodic boxes L = 32-80 by Hasimoto's law",
                "xi0": round(xi0, 5), "R_h": round(R_h, 4), "lambda": round(lam, 5),
                "bohlin_centreline": round(D.bohlin(lam), 5),
                "S_axial_fp64": [round(v, 5) for v in S[64]], "S_axial_fp32": [round(v, 5) for v in S[32]],
                "S_radial_fp64": [round(v, 5) for v in Sx[64]], "S_radial_fp32": [round(v, 5) for v in Sx[32]],
                "fp32_vs_fp64_max_rel": float(max(np.max(np.abs(np.array(S[32]) / np.array(S[64]) - 1)),
                                                  np.max(np.abs(np.array(Sx[32]) / np.array(Sx[64]) - 1)))),
                "off_axis_reference": "Happel-Brenner / Higdon-Muldowney off-axis values not available: unpinned"},
            "pore_msd": {"records": n, "bins": 20, "lags": 25, "ms": round(sec * 1e3, 2)}}


def measure_sphere32(torch, lb, steps=200):
    """The small validation case: 32^3 periodic FP64 BGK tau = 1, one filled
    sphere R = 3 (224 beads) pulled by a constant force, the drive compensated
    on the fluid; 200 steps; L2-resident (MLUPS only). Also the conservation
    check the case is for: total mass and momentum (fluid + body) after the
    run."""
    from paper_1604_01829_gb300 import workloads as W
    w = W.sphere_32()
    stream = torch.cuda.Stream()
    L = lb.from_workload(w, stream=stream.cuda_stream)
    L.lb_step(10)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.lb_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m, p = L.lb_conservation()
    L.close()
    return {"workload": w.name + ", sphere R = 3 (224 beads), F_ext 1e-4 compensated on the fluid",
            "nodes": w.nodes, "steps": steps, "ms_per_step": round(ms / steps, 4),
            "value": round(w.nodes * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "l2": "state 10 MB fits in L2: MLUPS only", "mass_rel_error": abs(m / w.nodes - 1.0)}


def measure_msd(torch, lb, nbodies=256, nrec=4000, max_lag=400, seed=1610):
    """GPU MSD analysis (lab- and body-frame translation and rotation) of
    seeded random-walk trajectories: 256 bodies x 4000 records x 400 lags,
    host arrays in and out (copies included)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    X = np.cumsum(rng.normal(scale=0.2, size=(nbodies, nrec, 3)), axis=1)
    d = np.concatenate([np.ones((nbodies, nrec, 1)), rng.normal(scale=0.05, size=(nbodies, nrec, 3))], axis=2)
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    q = np.empty_like(d)                    # random walk of orientations: q_k = q_{k-1} (x) d_k
    q[:, 0] = d[:, 0]
    for k in range(1, nrec):
        a, b = q[:, k - 1], d[:, k]
        q[:, k, 0] = a[:, 0] * b[:, 0] - (a[:, 1:] * b[:, 1:]).sum(1)
        q[:, k, 1:] = a[:, :1] * b[:, 1:] + b[:, :1] * a[:, 1:] + np.cross(a[:, 1:], b[:, 1:])
    lb.lb_msd_trajectory(X[:2, :100], q[:2, :100], 10)          # warm-up
    t0 = time.perf_counter()
    lb.lb_msd_trajectory(X, q, max_lag)
    sec = time.perf_counter() - t0
    pairs = nbodies * sum(nrec - l for l in range(1, max_lag + 1))
    return {"msd_bodies": nbodies, "msd_records": nrec, "msd_lags": max_lag, "msd_ms": round(sec * 1e3, 2),
            "msd_pairs_per_s": round(pairs / sec, 1)}


def measure_construction(args, torch, lb):
    """Raspberry construction (Sec. 2.1, SI construction section) for the 64
    ellipsoids of the headline workload: every shell of every raspberry
    (outer, inner at -0.5, fill shells every unit; one bead per unit area)
    relaxed together in one launch, FP32, the paper's damping and time step
    (eta dt = 1, dt = 0.001), from seeded evenly spread starts."""
    import numpy as np
    from paper_1604_01829_gb300 import workloads as W
    specs = [b.axes for b in build_workload(32).bodies]
    axes, starts = [], []
    for r, (a, b, c) in enumerate(specs):
        for s, (ax, n) in enumerate(W.raspberry_shells(a, b, c)):
            axes.append(ax)
            starts.append(W.spread_shell_start(*ax, n, seed=r * 1000003 + s))
    counts = np.array([len(x) for x in starts], dtype=np.float64)
    steps = args.construction_steps
    lb.lb_relax_shells(axes, starts, 20, precision=32)        # warm-up (module load, attribute set-up)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = lb.lb_relax_shells(axes, starts, steps, precision=32)
    wall = time.perf_counter() - t0
    ax_arr = np.array(axes)
    on_surface = max(float(np.abs(((x / a) ** 2).sum(1) - 1).max()) for x, a in zip(out, ax_arr))
    pairs = float((counts * counts).sum())
    return {"workload": f"{len(specs)} ellipsoidal raspberries of the headline workload: {len(axes)} shells, "
                        f"{int(counts.sum())} beads, largest shell {int(counts.max())}; FP32, dt 0.001, eta 1000, "
                        f"k 1000, WCA sigma 1.4 eps 0.1",
            "shells": len(axes), "beads": int(counts.sum()), "steps": steps,
            "ms_per_step": round(wall * 1e3 / steps, 4),
            "bead_steps_per_s": round(counts.sum() * steps / wall, 1),
            "pair_tests_per_s": round(pairs * steps / wall, 1),
            "max_surface_residual": on_surface,
            "timing": "host wall clock around one synchronous C-ABI call (copies included)"}


def measure_adjoint(args, torch, lb):
    """Hand-written adjoint on the 96^3 deterministic box with one prolate
    ellipsoid (a = 15, b = c = 5) pulled along its long axis: J = terminal
    velocity over the last steps, dJ/dgamma, dJ/ds for every bead, FP32
    storage. For each checkpointing schedule (two-level with sqrt(T) slots,
    binomial with 16 and 8 kept states) the split of device time from the
    library's own CUDA events (first forward sweep, recomputation, reverse
    kernels) on a second call that reuses the workspace, and the allocation
    time of the first. Compared with the FP32 and FP64 forward steps on the
    same workload; the FP32 drag is compared with the FP64 drag."""
    import numpy as np
    from paper_1604_01829_gb300 import workloads as W
    w32 = W.ellipsoid_adjoint_96(precision=32)
    T, Wn = args.adjoint_steps, max(1, args.adjoint_steps // 15)
    stream = torch.cuda.Stream()

    # FP32 forward alone (same steps) and FP64 forward on the same workload
    def forward(precision, steps):
        Lf = lb.from_workload(W.ellipsoid_adjoint_96(precision=precision), stream=stream.cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        Lf.lb_step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        Lf.lb_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        v = Lf.lb_get_body(0)["V"][0]
        Lf.close()
        return e0.elapsed_time(e1) / steps, v
    f32_ms, _ = forward(32, min(T, 500))
    f64_ms, _ = forward(64, 50)

    schedules = {}
    J32 = dg = ds = None
    for name, sched, snaps in (("two_level", lb.LB_ADJ_TWO_LEVEL, 0), ("binomial_16", lb.LB_ADJ_BINOMIAL, 16),
                               ("binomial_8", lb.LB_ADJ_BINOMIAL, 8)):
        L = lb.from_workload(w32, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        J, g, d, st1 = L.lb_adjoint_drag_ex(T, Wn, body=0, axis=0, schedule=sched, snapshots=snaps,
                                            with_stats=True)
        if J32 is None:
            J32, dg, ds = J, g, d
        t0 = time.perf_counter()
        _, _, _, st = L.lb_adjoint_drag_ex(T, Wn, body=0, axis=0, schedule=sched, snapshots=snaps,
                                           with_stats=True)
        wall = time.perf_counter() - t0
        L.close()
        total = st["forward_ms"] + st["recompute_ms"] + st["reverse_ms"]
        schedules[name] = {
            "snapshots": snaps if snaps else math.ceil(math.sqrt(T)),
            "alloc_ms_first_call": round(st1["alloc_ms"], 1),
            "forward_ms_per_step": round(st["forward_ms"] / T, 4),
            "recompute_ms_per_step": round(st["recompute_ms"] / T, 4),
            "reverse_ms_per_step": round(st["reverse_ms"] / T, 4),
            "total_ms_per_step": round(total / T, 4),
            "host_wall_ms_per_step": round(1e3 * wall / T, 4),
            "recompute_steps_per_step": round(st["recompute_steps"] / T, 3),
            "reverse_over_fp32_forward_step": round(st["reverse_ms"] / T / f32_ms, 3),
            "total_over_fp32_forward_step": round(total / T / f32_ms, 3),
            "total_over_fp64_forward_step": round(total / T / f64_ms, 3),
            "workspace_gb": round(st["workspace_bytes"] / 1e9, 3)}
    # drag of the FP64 reference run over the same steps and window
    L64 = lb.from_workload(W.ellipsoid_adjoint_96(precision=64), stream=stream.cuda_stream)
    vs = []
    for n in range(T):
        L64.lb_step(1)
        if n >= T - Wn:
            vs.append(L64.lb_get_body(0)["V"][0])
    L64.close()
    J64 = float(np.mean(vs))
    F = w32.bodies[0].F_ext[0]
    tl = schedules["two_level"]
    return {"workload": f"96^3 periodic, MRT nu=0.016, kT=0, FP32; prolate ellipsoid 15x5x5 "
                        f"({w32.nbeads} beads) pulled along its axis, {T} steps, J over the last {Wn}",
            "timing": "device time from CUDA events inside lb_adjoint_drag_ex, second call (workspace reused)",
            "adjoint_ms_per_step": tl["total_ms_per_step"],
            "fp32_forward_ms_per_step": round(f32_ms, 4), "fp64_forward_ms_per_step": round(f64_ms, 4),
            "adjoint_step_over_fp32_forward_step": tl["total_over_fp32_forward_step"],
            "adjoint_step_over_fp64_forward_step": tl["total_over_fp64_forward_step"],
            "reverse_step_over_fp32_forward_step": tl["reverse_over_fp32_forward_step"],
            "schedules": schedules,
            "drag_fp32": F / J32, "drag_fp64": F / J64,
            "drag_rel_error_fp32_vs_fp64": abs(J64 / J32 - 1.0),
            "dJ_dgamma": dg, "dxi_dgamma": -F / J32 ** 2 * dg,
            "dJ_ds_norm": float(np.linalg.norm(ds))}


def _oracle_box():
    """The oracle's bounded sample of the workload: a 64^3 periodic box (1/64
    of the lattice) with the same physics, holding the first ellipsoid of the
    workload (about the full box's nodes-per-bead ratio)."""
    from oracle import oracle as O
    from paper_1604_01829_gb300 import workloads as W
    w = W.ellipsoids_256(n_bodies=1, L=64, precision=64)
    p = w.params
    o = O.OracleLB(64, 64, 64, **{k: p[k] for k in ("collision", "gamma_shear", "gamma_bulk", "gamma_odd",
                                                      "gamma_even", "rho0", "kT", "gamma_bead", "seed")})
    b = w.bodies[0]
    o.add_raspberry(b.beads, b.X, b.q, b.mass, b.inertia)
    return o, w


def _oracle_worker(job):
    """One host core's share of the all-cores timing: its own sample box,
    `warmup` untimed steps, then `steps` steps from the common start time;
    returns (node updates, start, end) in wall-clock seconds."""
    warmup, steps, start_at = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    o, w = _oracle_box()
    o.step(warmup)
    delay = start_at - time.time()
    if delay > 0:
        time.sleep(delay)
    t0 = time.time()
    o.step(steps)
    t1 = time.time()
    return w.nodes * steps, t0, t1


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_all_cores(ncores, warmup, steps):
    """The oracle, unchanged, on every host core at once: one independent
    sample box per core in its own process (spawned, so no process is forked
    after the CUDA context exists), started together; aggregate node updates
    over the span from the first start to the last end."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    start_at = time.time() + 8.0 + 0.5 * warmup
    with ctx.Pool(ncores) as pool:
        res = pool.map(_oracle_worker, [(warmup, steps, start_at)] * ncores)
    work = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return work / span / 1e6, span


def oracle_sample(seconds):
    """The FP64 CPU oracle, as it stands, on the bounded sample box: single
    thread for ~`seconds`, then one sample box per host core for about the
    same time."""
    o, w = _oracle_box()
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(1, int(seconds / per) - 1)
    o.step(n)
    t2 = time.perf_counter()
    steps = n + 1
    mlups1 = w.nodes * steps / (t2 - t0) / 1e6
    ncores = host_cores()
    # with every core busy each box is slower (shared memory bandwidth):
    # half the single-thread steps keeps the run near `seconds`
    steps_all = max(2, steps // 2)
    mlups_all, span = oracle_all_cores(ncores, 1, steps_all)
    return {"value": round(mlups_all, 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle",
            "sample": f"64^3 periodic box, MRT + fluctuations, 1 ellipsoid ({w.nbeads} beads): one box per host "
                      f"core in its own process, {steps_all} steps each, {span:.1f} s",
            "single_thread": {"value": round(mlups1, 4), "unit": "MLUPS", "cores": 1,
                              "sample": f"the same box, {steps} steps, {t2 - t0:.1f} s"}}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle on the bounded sample box, one box
    per host core (independent processes started together), K timed steps
    after W untimed ones."""
    if rank != 0:
        return
    ncores = host_cores()
    v, span = oracle_all_cores(ncores, args.warmup, args.steps)
    sample = (f"64^3 periodic box (1/64 of the 256^3 lattice), MRT + fluctuations, 1 ellipsoid; one box per "
              f"host core ({ncores}) in its own process, {args.steps} steps each, {span:.1f} s")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(span * 1e3 / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the FP64-population leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--lattice", type=int, default=256, help="cubic lattice edge (profiling cases)")
    ap.add_argument("--bodies", type=int, default=64, help="number of ellipsoids (profiling cases)")
    ap.add_argument("--skip-batched", action="store_true", help="skip the batched-instances leg")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--batch-schedule", default=None,
                    help="tile_nodes,blocks_per_sm,order for the batched leg instead of the autotuner")
    ap.add_argument("--skip-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--skip-pore", action="store_true", help="skip the confinement leg")
    ap.add_argument("--adjoint-steps", type=int, default=3000)
    ap.add_argument("--skip-construction", action="store_true", help="skip the raspberry-construction leg")
    ap.add_argument("--construction-steps", type=int, default=2000)
    args = ap.parse_args()
    global ARGS
    ARGS = args
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
