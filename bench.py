"""Throughput benchmark of the thermal lattice Boltzmann step on GB300.

Workload: side-heated cubic cell, 257^3 nodes, Ra = 1e7, Pr = 0.71, hot wall
x = 0 (T = +1/2), cold wall x = H (T = -1/2), four adiabatic walls, all walls
no-slip; free-fall scaling with U = 0.1.  One benchmark step is one chunk of
100 lattice Boltzmann time steps (D3Q19 + D3Q7 stream-and-collide of every
node) with the global diagnostics (Nu, Re, dissipation) sampled once, i.e. a
pass over every row of the hot path.  The state (1.77 GB in FP32, 0.88 GB in
FP16) is far larger than the 129 MB L2, so no flush is needed between steps.

Metric: GLUPS = lattice-node updates of both distributions per second
(nodes x time steps / s), whole job.  The line also carries the HBM roofline
fraction of the step kernel, the FP16/BF16-storage variants, the end-to-end
figure through the C ABI with host buffers, and the FP64 CPU oracle timed on
this machine's host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EDGE = 257
RA, PR, U = 1e7, 0.71, 0.1
CHUNK = 100                  # LB time steps per benchmark step
BYTES_PER_NODE = {"fp32": 208, "fp16s": 104, "bf16s": 104, "fp16m": 132}  # 26 populations read + written
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0
METRIC = "GLUPS (D3Q19+D3Q7) and % HBM roofline at 257^3, FP32 vs FP16 storage"
# sources of each storage's step kernels: FP32 runs the register kernels, the
# 2-byte storages the staged kernels (plus the register face kernel)
STEP_KERNEL_SRC = {
    "fp32": ("lbm_kernels.cu", "lbm_device.cuh"),
    "staged": ("lbm_kernels.cu", "lbm_staged.cu", "lbm_device.cuh"),
}
# kernels of one LB time step with the library's default kernels per storage
STEP_KERNELS = {
    "fp32": "k_aa_even2 (even steps); k_aa_odd_rows + k_aa_odd_face on the y/z-face nodes (odd steps)",
    "staged": "k_aa_staged<even> (even steps); k_aa_staged<odd> + k_aa_odd_face on the face nodes (odd steps)",
}


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _kernel_hash(storage):
    """Hash of a storage's step kernels' code: sources with comments and
    whitespace removed, so that only a change of the code invalidates stored
    counters."""
    h = hashlib.sha256()
    for f in STEP_KERNEL_SRC["fp32" if storage == "fp32" else "staged"]:
        with open(os.path.join(ROOT, "paper_1903_08882_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def _profiled_traffic(storage):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_dram_traffic.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(rf"kernel_source_sha256_16_{storage}:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != _kernel_hash(storage):
        return None
    m = re.search(rf"traffic_per_launch_{storage}_257:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        return dist, int(os.environ["RANK"]), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _max_over_ranks(dist, x, device="cuda"):
    """The largest of the ranks' values (the slowest rank's time)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist, cuda=True):
    """All ranks' GPU work done and all ranks at this point."""
    import torch

    if cuda:
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
        if cuda:
            torch.cuda.synchronize()


def aggregate_rate(units_per_rank, world_size, seconds):
    """Whole-job rate of independent replicas: the units every rank processed
    divided by the slowest rank's time (weak scaling)."""
    return units_per_rank * world_size / seconds


def _cpu_oracle_rate(max_seconds=15.0, min_steps=2):
    """FP64 oracle (the test reference, as it stands) on a bounded sample of
    the workload: a 257 x 257 x 8 slab of the side-heated 257^3 cell with the
    same walls, stepped until about max_seconds have passed."""
    import oracle

    oracle.build()
    nz = 8
    p = oracle.cell((N_EDGE, N_EDGE, nz), RA, PR, oracle.side_heated_walls(), H=N_EDGE)
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = oracle.run(p, f, g, 1)  # warm the pages
    steps, t0 = 0, time.perf_counter()
    while True:
        f, g = oracle.run(p, f, g, 1)
        steps += 1
        el = time.perf_counter() - t0
        if steps >= min_steps and el >= max_seconds:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nodes = N_EDGE * N_EDGE * nz
    return nodes * steps / el / 1e9, threads, f"{N_EDGE}x{N_EDGE}x{nz} slab of the 257^3 side-heated cell, " \
                                               f"{steps} FP64 oracle steps in {el:.1f} s"


def run_reference(args):
    """The reference arm: the FP64 oracle (the test reference, as it stands)
    on the host cores.  Each benchmark step is a bounded sample of the
    workload: `lb` oracle LB steps of a 257 x 257 x 8 slab of the 257^3
    side-heated cell (same walls and parameters), lb chosen once so that a
    step takes about 2 s.  ms_per_step is the time those steps took."""
    # the oracle runs on the host: rank 0 alone times it, the other ranks of a
    # multi-rank launch exit without work (no process group is needed)
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle

    oracle.build()
    nz = 8
    p = oracle.cell((N_EDGE, N_EDGE, nz), RA, PR, oracle.side_heated_walls(), H=N_EDGE)
    f, g = oracle.init_equilibrium(p, 1.0, np.zeros(3), 0.0)
    f, g = oracle.run(p, f, g, 1)  # warms the pages
    t0 = time.perf_counter()
    f, g = oracle.run(p, f, g, 2)
    lb = max(1, int(round(2.0 / max((time.perf_counter() - t0) / 2, 1e-3))))
    for _ in range(args.warmup):
        f, g = oracle.run(p, f, g, lb)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, g = oracle.run(p, f, g, lb)
    el = time.perf_counter() - t0
    nodes = N_EDGE * N_EDGE * nz
    value = nodes * lb * args.steps / el / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    workload = (f"{N_EDGE}x{N_EDGE}x{nz} slab of the side-heated 257^3 cell (Ra=1e7, Pr=0.71, U=0.1), "
                f"{lb} FP64 oracle LB steps per benchmark step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "lb_steps_per_step": lb, "nodes": nodes},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{workload}; {args.steps} timed steps, {el:.1f} s"},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_chunks(lat, k, stream):
    import torch

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(k):
        lat.step(CHUNK)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def _step_kernel_seconds(lat, stream, launches=98):
    """Average duration of one LB time step's kernels: `launches` consecutive
    plain steps (no diagnostic sample falls among them), each bracketed by
    events on the library's stream; also the median even and odd step."""
    import torch

    c = lat.diagnostics(raise_on_diverged=False)["step"]
    lat.step((-c) % CHUNK + 1)  # now one past a sampling step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(launches + 1)]
    for k in range(launches):
        ev[k].record(stream)
        lat.step(1)
    ev[launches].record(stream)
    ev[launches].synchronize()
    t = [ev[k].elapsed_time(ev[k + 1]) / 1e3 for k in range(launches)]
    first_even = lat.diagnostics(raise_on_diverged=False)["step"] - launches
    even = sorted(t[(first_even % 2)::2])
    odd = sorted(t[1 - (first_even % 2)::2])
    return ev[0].elapsed_time(ev[launches]) / 1e3 / launches, even[len(even) // 2], odd[len(odd) // 2]


def _event_ms(fn, stream, reps=10):
    """Mean duration of fn() over reps calls, CUDA events on `stream`."""
    import torch

    fn()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        fn()
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / reps


def bench_diagnostics(lbm, lat, stream, peak):
    """Timing of the diagnostics of one state of the benchmark cell (Secs. 3-4):
    the reduction kernel alone (k_diag + its one-block finish, run through
    lbm_reduce_noalloc on the moment arrays of the state), a whole sample
    (moments of the state, then the reduction), the dissipation-rate PDFs and
    the Nusselt profile with the mid-line wall values."""
    import torch

    N = N_EDGE
    n = N ** 3
    stride = (n + 127) // 128 * 128
    rho, u3, T = lat.moments()
    fields = torch.zeros((11, stride), dtype=torch.float32)
    fields[0, :n] = torch.from_numpy((rho - 1.0).ravel().astype(np.float32))
    for a in range(3):
        fields[1 + a, :n] = torch.from_numpy(u3[a].ravel().astype(np.float32))
    fields[4, :n] = torch.from_numpy(T.ravel().astype(np.float32))
    fields = fields.cuda()
    sums = torch.zeros(24, dtype=torch.float64, device="cuda")
    walls, a_T = lbm.walls_side_heated(), lat.constants["a_T"]
    red = _event_ms(lambda: lbm.lbm_reduce_noalloc(fields.data_ptr(), stride, N, N, N, walls, a_T,
                                                   sums.data_ptr(), stream=stream), stream)
    in_bytes = 5 * 4 * n  # rho - rho0, u, v, w, T once each (neighbours from cache)
    ach = in_bytes / (red * 1e-3) / 1e9
    sample = _event_ms(lat.sample, stream)
    t0 = time.perf_counter()
    for _ in range(3):
        lat.dissipation_pdf(nbins=200, xmax=20.0)
    pdf = (time.perf_counter() - t0) / 3 * 1e3
    t0 = time.perf_counter()
    for _ in range(3):
        lat.nusselt_profile(axis=0)
    prof = (time.perf_counter() - t0) / 3 * 1e3
    del fields, sums
    return {"reduction": {"kernel": "k_diag + k_diag_finish", "ms": round(red, 4), "input_bytes": in_bytes,
                          "achieved_gbs": round(ach, 1), "frac_of_peak": round(ach / peak, 4)},
            "sample_ms": round(sample, 4),
            "sample_what": "moments of the state (k_moments) then the reduction",
            "dissipation_pdf_ms": round(pdf, 3), "nusselt_profile_ms": round(prof, 3),
            "host_synchronous": "dissipation_pdf and nusselt_profile include their host read-back"}


def bench_storage(lbm, storage, args, stream, dist, with_e2e):
    import torch

    N = N_EDGE
    nodes = N ** 3
    lat = lbm.Lattice(N, N, N, lbm.walls_side_heated(), Ra=RA, Pr=PR, U=U, storage=storage,
                      diag_every=CHUNK, stream=stream, nodes_per_thread=args.npt)
    res = {}
    try:
        for _ in range(args.warmup):
            lat.step(CHUNK)
        _barrier(dist)
        with ClockSampler(torch.cuda.current_device()) as cs:
            dt = _time_chunks(lat, args.steps, stream)
        _barrier(dist)
        dt = _max_over_ranks(dist, dt)
        res["seconds"] = dt
        res["glups"] = aggregate_rate(nodes * CHUNK * args.steps, dist.get_world_size() if dist else 1, dt) / 1e9
        res["clocks"] = cs.summary()
        tk, te, to = _step_kernel_seconds(lat, stream)
        res["kernel_seconds"] = tk
        res["kernel_even_seconds"], res["kernel_odd_seconds"] = te, to
        d = lat.diagnostics(raise_on_diverged=False)
        res["Nu_hot"] = float(d["Nu_face"][0])
        res["diverged"] = bool(d["diverged"])
        if with_e2e:
            res["diagnostics"] = bench_diagnostics(lbm, lat, stream, _peak_hbm()[0])
            res["e2e"] = _e2e(lbm, lat, args, stream, dist)
    finally:
        lat.close()
    return res


def _e2e(lbm, lat, args, stream, dist):
    """Same metric through the public API with host buffers: every step
    uploads its input fields (rho, u, T) from pinned host memory, advances one
    chunk from them and reads the diagnostics back to the host.  The uploads
    go through lbm_upload_fields on the context's copy stream, step k + 1's
    beside step k's chunk, and lbm_apply_fields builds each step's state from
    them; every upload is inside the timed region.  `set_fields_value` is the
    same loop with the synchronous lbm_set_fields (copy, then chunk)."""
    import torch

    N = N_EDGE
    sh = (N, N, N)
    rho = torch.ones(sh, dtype=torch.float64).pin_memory().numpy()
    u3 = torch.zeros((3,) + sh, dtype=torch.float64).pin_memory().numpy()
    T = torch.zeros(sh, dtype=torch.float64).pin_memory().numpy()

    def serial(steps):
        for _ in range(steps):
            lat.set_fields(rho, u3, T)
            lat.step(CHUNK)
            lat.diagnostics(raise_on_diverged=False)

    def pipelined(steps):
        lat.upload_fields(rho, u3, T)
        for k in range(steps):
            lat.apply_fields()
            lat.step(CHUNK)
            if k + 1 < steps:
                lat.upload_fields(rho, u3, T)  # the next step's inputs, beside this chunk
            lat.diagnostics(raise_on_diverged=False)

    rates = {}
    for name, run in (("set_fields", serial), ("pipelined", pipelined)):
        run(max(1, args.warmup // 2))
        _barrier(dist)
        t0 = time.perf_counter()
        run(args.steps)
        torch.cuda.synchronize()
        dt = _max_over_ranks(dist, time.perf_counter() - t0)
        ws = dist.get_world_size() if dist else 1
        rates[name] = aggregate_rate(N ** 3 * CHUNK * args.steps, ws, dt) / 1e9
    return {"value": rates["pipelined"], "unit": "GLUPS", "set_fields_value": rates["set_fields"],
            "h2d_bytes_per_step": int(rho.nbytes + u3.nbytes + T.nbytes), "d2h_bytes_per_step": 8 * (2 * 24 + 1)}


def bench_batched(lbm, args, stream):
    """Batched sweep: 64 cells (edges 33-97, Ra 1e4-1e7, Pr 0.71/7, half side-
    heated, half Rayleigh-Benard) advanced by one persistent launch per run of
    steps, replayed as 1000-step CUDA graphs with an autotuned schedule, against
    the same cells advanced one launch (pair) per cell per step."""
    import torch

    from paper_1903_08882_gb300 import drivers

    lats, draws = drivers.sweep_cells(lbm, stream=stream)
    nodes = sum(d["edge"] ** 3 for d in draws)
    chunk = 1000
    res = {"cells": len(lats), "nodes": nodes, "edges": sorted({d["edge"] for d in draws})}
    try:
        with lbm.Batch(lats, stream=stream) as b:
            best = b.autotune(trial_steps=20)
            b.set_schedule(steps_per_launch=100, graph_chunk=chunk)
            b.step(chunk)  # capture + warm-up
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = max(1, args.steps // 3)
            ev0.record(stream)
            b.step(k * chunk)
            ev1.record(stream)
            ev1.synchronize()
            t_b = ev0.elapsed_time(ev1) / 1e3
            res["schedule"] = b.schedule
        ev0.record(stream)
        for lat in lats:
            lat.step(chunk)
        ev1.record(stream)
        ev1.synchronize()
        t_s = ev0.elapsed_time(ev1) / 1e3
        res["glups_batched"] = round(nodes * chunk * k / t_b / 1e9, 3)
        res["glups_one_launch_per_cell"] = round(nodes * chunk / t_s / 1e9, 3)
        res["speedup"] = round(res["glups_batched"] / res["glups_one_launch_per_cell"], 3)
        res["graph_chunk_steps"] = chunk
        res["autotuned"] = best
    finally:
        for lat in lats:
            lat.close()
    return res


def bench_warmstart_network(stream, edge=129, reps=5):
    """Forward and backward of the warm-start U-Net (one sample, 129^3 fine
    lattice, random weights and inputs), on its own kernels: the whole
    network's times and the convolutions' algorithmic FLOP rate (2 x voxels
    x Cin x Cout x 27 per convolution; the backward pass does the data and
    the weight gradient, twice that), against the measured BF16 dense rate
    of the tensor cores (the convolutions multiply BF16 weights with FP32
    operands carried as two BF16 terms, so their MMAs do 2-3x these FLOPs)."""
    import torch

    from paper_1903_08882_gb300 import unet

    size = (edge, edge, edge)
    net = unet.UNet(size, seed=1)
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.rand((7,) + size, device="cuda", generator=g) - 0.5
    t = torch.rand((5,) + size, device="cuda", generator=g) - 0.5
    flops = 0.0
    for name, cin, cout in unet.layer_shapes():
        lvl = 0 if name == "head" else int(name[1])
        v = net.sizes[lvl][0] * net.sizes[lvl][1] * net.sizes[lvl][2]
        flops += 2.0 * v * cin * cout * 27
    with torch.cuda.stream(stream):
        for _ in range(2):
            net.zero_grad()
            net.forward(x)
            net.backward(x, t)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        fw = bw = 0.0
        for _ in range(reps):
            net.zero_grad()
            e0.record(stream)
            net.forward(x)
            e1.record(stream)
            net.backward(x, t)
            e2.record(stream)
            e2.synchronize()
            fw += e0.elapsed_time(e1)
            bw += e1.elapsed_time(e2)
    fw, bw = fw / reps, bw / reps
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    ach_f, ach_b = flops / (fw * 1e-3) / 1e12, 2 * flops / (bw * 1e-3) / 1e12
    del net
    return {"size": list(size), "forward_ms": round(fw, 3), "backward_ms": round(bw, 3),
            "conv_gflop_forward": round(flops / 1e9, 2),
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "peak": peak, "peak_kind": kind,
                         "achieved_forward": round(ach_f, 2), "achieved_backward": round(ach_b, 2),
                         "frac_forward": round(ach_f / peak, 4), "frac_backward": round(ach_b / peak, 4)},
            "kernels": "k_conv_fwd_tc (forward and data gradient), k_conv_bww_tc (weight gradient): mma.sync "
                       "m16n8k16 BF16 -> FP32"}


def run_gpu(args):
    import torch

    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    from paper_1903_08882_gb300 import _build, lbm

    if not _build.up_to_date():
        _build.build()
    stream = torch.cuda.Stream()
    peak, peak_kind = _peak_hbm()
    if args.unet_only:  # profiling run of the warm-start network alone
        if rank == 0:
            print(json.dumps({"warmstart_network": bench_warmstart_network(stream)}), flush=True)
        return
    storages = ["fp32"] if args.fp32_only else ["fp32", "fp16s", "bf16s", "fp16m"]
    if args.only:
        storages = [args.only]
    results = {}
    with torch.cuda.stream(stream):
        for st in storages:
            results[st] = bench_storage(lbm, st, args, stream, dist, with_e2e=(st == "fp32"))
    if rank != 0:
        return
    if "fp32" not in results:  # profiling run of one storage form
        for st, r in results.items():
            print(json.dumps({"storage": st, "glups": r["glups"], "kernel_ms": r["kernel_seconds"] * 1e3,
                              "even_ms": r["kernel_even_seconds"] * 1e3, "odd_ms": r["kernel_odd_seconds"] * 1e3}))
        return
    main = results["fp32"]
    nodes = N_EDGE ** 3

    def roof(r, st):
        ach = BYTES_PER_NODE[st] * nodes / r["kernel_seconds"] / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_kind": peak_kind,
                "frac_of_nominal_8000": round(ach / NOMINAL_HBM_GBS, 4),
                "algorithmic_bytes_per_launch": BYTES_PER_NODE[st] * nodes,
                "traffic": _profiled_traffic(st) if N_EDGE == 257 else None,
                "kernel": f"one AA LB time step, {st} storage: " + STEP_KERNELS["fp32" if st == "fp32" else "staged"],
                "kernel_ms": round(r["kernel_seconds"] * 1e3, 4),
                "kernel_even_ms": round(r["kernel_even_seconds"] * 1e3, 4),
                "kernel_odd_ms": round(r["kernel_odd_seconds"] * 1e3, 4),
                "kernel_glups": round(nodes / r["kernel_seconds"] / 1e9, 3)}

    batched = None
    if not args.no_batch and ws == 1:
        with torch.cuda.stream(stream):
            batched = bench_batched(lbm, args, stream)
    network = bench_warmstart_network(stream) if ws == 1 and not args.no_batch else None
    cpu_rate, threads, sample = _cpu_oracle_rate() if not args.no_cpu else (None, None, None)
    line = {
        "metric": METRIC, "value": round(main["glups"], 3), "unit": "GLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(main["seconds"] / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "side-heated cube 257^3, Ra=1e7, Pr=0.71, U=0.1, FP32 storage, AA streaming",
                   "lb_steps_per_step": CHUNK, "diag_every": CHUNK, "nodes": nodes,
                   "l2": f"state ({N_EDGE ** 3 * 104 / 1e9:.2f} GB FP32) larger than L2, no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": roof(main, "fp32"),
        "clocks": main["clocks"],
        "e2e": main.get("e2e"),
        # per chunk: CHUNK/2 even steps (one kernel), CHUNK/2 odd steps (row or
        # staged kernel + face kernel), one diagnostic sample (two kernels)
        "gpu_launches": (CHUNK // 2 * 3 + 2) * args.steps,
        "cpu_baseline": ({"value": cpu_rate, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                          "sample": sample} if cpu_rate else None),
        "storage_variants": {st: {"value": round(r["glups"], 3), "unit": "GLUPS",
                                  "ms_per_step": round(r["seconds"] / args.steps * 1e3, 3),
                                  "roofline": roof(r, st), "clocks": r["clocks"],
                                  "speedup_vs_fp32": round(r["glups"] / main["glups"], 3)}
                             for st, r in results.items() if st != "fp32"},
        "diagnostics": main.get("diagnostics"),
        "Nu_hot_after_run": main["Nu_hot"],
        "batched_sweep": batched,
        "warmstart_network": network,
    }
    print(json.dumps(line), flush=True)


def main():
    global N_EDGE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp32-only", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-cell batched sweep")
    ap.add_argument("--edge", type=int, default=N_EDGE, help="cube edge; other than 257 only for profiling")
    ap.add_argument("--only", default=None, choices=["fp32", "fp16s", "bf16s", "fp16m"],
                    help="time one storage form only (profiling)")
    ap.add_argument("--npt", type=int, default=0, help="nodes per thread of the AA kernels (0: library default)")
    ap.add_argument("--unet-only", action="store_true", help="time the warm-start network alone (profiling)")
    args = ap.parse_args()
    N_EDGE = args.edge
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
