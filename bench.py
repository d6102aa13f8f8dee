"""Benchmark of the D2Q9 pseudopotential MRT lattice update (one step = one
lattice update of the whole channel: streaming with boundaries, density,
pseudopotential, forces, velocity, MRT collision and the RK4 temperature update).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun every rank advances its own
replica of the channel (weak scaling, no data-path collective); the timed region
is bracketed by a barrier and a device synchronize and the elapsed time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_01756_gb300 import inputs  # noqa: E402

# Algorithmic bytes per cell-update (FP32 storage): populations 9 x 4 read + 9 x 4
# written, temperature 4 read + 4 written.
BYTES_PER_CELL_UPDATE = 80
# Per-kernel algorithmic bytes per cell for the split path (unique bytes each
# launch must move): density/psi reads f and T and writes rho, psi; collide reads
# f and psi and writes f and u; energy reads T, rho, u and writes T.
SPLIT_KERNEL_BYTES = {"k_density_psi": 36 + 4 + 8, "k_collide": 36 + 4 + 36 + 8,
                      "k_energy": 4 + 4 + 8 + 4, "k_fused_step": 80}
# The two-pass path: k_stream_collide reads and writes the populations, reads T and writes
# rho and u (FP32 populations: 36 + 36 + 4 + 12); k_energy_rk4 reads T, rho and u and
# writes T.  The update as a whole is still measured against the 80 B of the fused update.
TWOPASS_RK4_BYTES = 4 + 4 + 8 + 4


def twopass_sc_bytes(pop_bytes: int) -> int:
    """Algorithmic bytes per cell of one k_stream_collide launch with pop_bytes-byte
    populations."""
    return 2 * 9 * pop_bytes + 4 + 12


L2_BYTES = 129e6
# updates per CUDA-graph chunk of lbm_step on the fused path
GRAPH_CHUNK = 16
# maximum SM clock of the GB300 (nvidia-smi clocks.max.sm)
SM_MAX_MHZ = 2070
# ncu counters of one k_fused_step launch on the 4096 x 512 channel with FP32 storage:
# DRAM bytes read + written (dram__bytes_read.sum + dram__bytes_write.sum) and warp
# instructions executed (smsp__inst_executed.sum; with the live launch time they give the
# kernel's issue rate against the SMs' issue limit of 4 schedulers x 1 warp instruction per
# cycle).  They hold for the kernel sources whose hash is FUSED_COUNTERS_SOURCE (the
# profiles/ summary of the capture records the same hash); when the built sources hash
# differently the counters are stale and the bench reports them as null.
FUSED_F32_4096x512_DRAM_BYTES = 103.403264e6 + 39.863040e6
FUSED_F32_4096x512_WARP_INSTR = 43732808
FUSED_COUNTERS_SOURCE = "9219133cdaaedea1"
# the files that determine the fused kernel's machine code
FUSED_SOURCES = ["paper_1803_01756_gb300/csrc/lbm_common.cuh",
                 "paper_1803_01756_gb300/csrc/lbm_internal.h",
                 "paper_1803_01756_gb300/csrc/lbm_fused_tile.cuh",
                 "paper_1803_01756_gb300/csrc/lbm_fused_step.cuh",
                 "paper_1803_01756_gb300/csrc/lbm_fused.cu",
                 "paper_1803_01756_gb300/build.py"]


def fused_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the fused kernel's source files."""
    import hashlib
    h = hashlib.sha256()
    for rel in FUSED_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# --physics: which parts of the update run (the energy equation of Eqs. 16-18 and the
# pseudopotential forces of Eqs. 9-14 are separate switches of the library)
PHYSICS = {"full": {}, "no-thermal": {"thermal": 0}, "no-multiphase": {"multiphase": 0},
           "plain": {"thermal": 0, "multiphase": 0}}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, name in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def setup_distributed():
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def max_over_ranks(value: float, dist) -> float:
    """Largest value over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_oracle(w: dict, nx: int, ny: int, steps: int):
    """FP64 oracle (single thread) on an nx x ny cut of workload w; returns MLUPS."""
    import oracle
    rho0 = inputs.noisy_density(nx, ny, inputs.RHO_V_086, w["noise"], w["seed"])
    o = oracle.Oracle(nx, ny, w["params"])
    o.set_fields(rho0)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, dt


def _oracle_cut(job):
    """One oracle process of the all-cores CPU figure: `steps` updates of an nx x ny cut of
    the workload; returns (node-updates, seconds)."""
    name, nx, ny, steps = job
    w = inputs.workload(name)
    mlups, dt = time_oracle(w, nx, ny, steps)
    return nx * ny * steps, dt


def oracle_all_cores(name: str, nx: int, ny: int, steps: int):
    """The unmodified oracle run as one process per host core, each on its own nx x ny cut
    (spawned before any GPU work): aggregate MLUPS over the wall time of the slowest."""
    from multiprocessing import get_context
    n = os.cpu_count() or 1
    t0 = time.perf_counter()
    with get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_cut, [(name, nx, ny, steps)] * n)
    wall = time.perf_counter() - t0
    cell = sum(r[0] for r in res)
    return {"value": cell / max(r[1] for r in res) / 1e6, "unit": "MLUPS", "cores": n,
            "sample": f"{n} oracle processes, each {steps} updates of a {nx}x{ny} cut "
                      f"({wall:.1f} s wall including start-up)"}


def reference_arm(args, world, rank):
    """The FP64 oracle as the reference arm: each step is one update of a bounded
    cut of the channel, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    w = inputs.workload(args.workload)
    # size the cut so that warmup + steps take about two minutes at ~1.5 MLUPS
    budget_cells = max(2048, int(180e6 / max(1, args.steps + args.warmup)))
    ny = min(w["ny"], 64)
    nx = max(32, min(w["nx"], budget_cells // ny))
    import oracle
    rho0 = inputs.noisy_density(nx, ny, inputs.RHO_V_086, w["noise"], w["seed"])
    o = oracle.Oracle(nx, ny, w["params"])
    o.set_fields(rho0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = nx * ny * args.steps / dt / 1e6
    sample = f"{nx}x{ny} cut of {args.workload}, {args.steps} updates per run, FP64 oracle"
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nx": nx, "ny": ny, "sample_of": [w["nx"], w["ny"]]},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": sample, "host_nproc": os.cpu_count()},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


METRIC = "lattice updates per second (MLUPS), D2Q9 pseudopotential MRT + RK4 energy update"


def our_arm(args, world, rank, local, dist):
    import torch
    from paper_1803_01756_gb300 import lattice as L

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    w = inputs.workload(args.workload)
    # parts of the update switched off (to see what each part costs); the default is all
    w["params"] = dict(w["params"], **PHYSICS[args.physics])
    nx, ny = w["nx"], w["ny"]
    kernel = {"auto": L.KERNEL_AUTO, "split": L.KERNEL_SPLIT, "fused": L.KERNEL_FUSED,
              "fused1": L.KERNEL_FUSED_1COL, "fused2": L.KERNEL_FUSED_2COL,
              "twopass": L.KERNEL_TWOPASS}[args.kernel]
    storage = {"f32": 0, "bf16": 1, "f16": 2}[args.storage]
    # algorithmic bytes per cell-update: populations read and written once, T read and written
    bytes_cell = 2 * 9 * (4 if args.storage == "f32" else 2) + 8

    # CPU baseline first (rank 0, N = 1): the oracle on the host cores, before any
    # GPU work so that nothing forks after CUDA initialisation
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        steps = args.cpu_steps
        mlups, dt = time_oracle(w, nx, ny, steps)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{steps} updates of the full {nx}x{ny} channel ({dt:.1f} s, 1 thread)",
               "host_nproc": os.cpu_count(),
               "note": "the oracle is a sequential program and runs on one of the host's cores"}
        if not args.no_cpu_all_cores:
            cpu["all_cores"] = oracle_all_cores(args.workload, nx, min(ny, 64), args.cpu_steps * 4)

    stream = torch.cuda.current_stream()
    lat = L.Lattice(nx, ny, w["params"], kernel=kernel, storage=storage)
    info = lat.info()
    rho0 = inputs.initial_density(w)
    lat.write_fields(rho0)
    lat.step(args.warmup, stream=stream)
    # 16 more untimed updates: the first full chunk at the timed region's buffer parity
    # captures the CUDA graph that the timed region replays
    lat.step(GRAPH_CHUNK, stream=stream)
    torch.cuda.synchronize()

    # ---- timed region: K updates, device time from CUDA events on the stream, with a
    # device synchronize on both sides; repeated (K updates each time) until the repeats
    # add up to --min-timed-s, so that the clock sampler sees the GPU under load, and the
    # median repeat is reported (the fused path replays 16-update CUDA graphs here) ----
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    repeats = []
    while True:
        torch.cuda.synchronize()
        ev0.record(stream)
        lat.step(args.steps, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        repeats.append(ev0.elapsed_time(ev1))
        if sum(repeats) >= 1e3 * args.min_timed_s or len(repeats) >= 100000:
            break
    if dist:
        dist.barrier()
    elapsed_ms = statistics.median(repeats)
    # ---- per-kernel launch durations: a second pass of K updates with CUDA events
    # recorded around every launch on the stream (one launch per kernel and update) ----
    lat.timing_enable(True)
    lat.timing_get(stream=stream)  # reset per-kernel totals
    lat.step(args.steps, stream=stream)
    per_kernel = lat.timing_get(stream=stream)
    lat.timing_enable(False)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, dist)
    status = lat.status()

    cells = nx * ny
    value = world * cells * args.steps / (elapsed_ms / 1e3) / 1e6
    # kernels per update are the same in both passes (a graph replays one kernel node
    # per update)
    launches = sum(n for _, n in per_kernel.values())

    # dominant kernel roofline.  Its average launch duration is its share of the timed
    # region (CUDA events on the launching stream around the K updates) per launch, the
    # shares taken from the per-launch events of the second pass.  On the fused path (one
    # kernel per update) that is the timed region over K, inter-kernel gaps and the
    # boundary-scalar copies included.
    peak, peak_kind = measured_peaks()
    total_ms = sum(v[0] for v in per_kernel.values())
    shares = {k: v[0] / total_ms for k, v in per_kernel.items()}
    top_name = max(shares, key=shares.get)
    top_ms, top_n = per_kernel[top_name]
    if top_name == "k_fused_step":
        per_cell = bytes_cell
    elif top_name == "k_stream_collide":
        per_cell = twopass_sc_bytes(4 if args.storage == "f32" else 2)
    elif top_name == "k_energy_rk4":
        per_cell = TWOPASS_RK4_BYTES
    else:
        per_cell = SPLIT_KERNEL_BYTES[top_name]
    traffic = args.traffic
    src_hash = fused_source_hash()
    counters_current = src_hash == FUSED_COUNTERS_SOURCE
    if (traffic is None and top_name == "k_fused_step" and args.storage == "f32"
            and args.workload == "channel_4096x512" and args.physics == "full"
            and info["cols_per_thread"] == 1 and counters_current):
        traffic = FUSED_F32_4096x512_DRAM_BYTES
    bytes_per_launch = per_cell * cells
    avg_us = elapsed_ms * shares[top_name] / top_n * 1e3
    achieved = bytes_per_launch / (avg_us / 1e6) / 1e9
    roofline = {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_us,
                "launch_timing": ("kernel's share of the timed region per launch; shares from "
                                  f"CUDA events around each launch in a second pass of "
                                  f"{args.steps} updates"),
                "event_bracketed_launch_us": top_ms / top_n * 1e3,
                "kernel_share": shares, "kernel_source_sha": src_hash,
                "counters_source_sha": FUSED_COUNTERS_SOURCE}
    if traffic is not None and args.traffic is None:
        # the same kernel, workload and storage as the ncu counts: its issue roofline
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or SM_MAX_MHZ
        issue_peak = sms * 4 * mhz * 1e6
        issue = FUSED_F32_4096x512_WARP_INSTR / (avg_us / 1e6)
        roofline["issue"] = {
            "achieved": issue / 1e9, "peak": issue_peak / 1e9, "unit": "G warp-instr/s",
            "frac": issue / issue_peak,
            "instr_per_cell_update": FUSED_F32_4096x512_WARP_INSTR * 32 / cells,
            "peak_source": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        inner = args.e2e_inner
        reps = args.e2e_reps
        rho_h = torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
        rho_h[:] = rho0
        outs = [torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
                for _ in range(4)]
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        lib = L.load_library()
        sp = stream.cuda_stream
        # one untimed job first
        lib.lbm_write_fields(lat._h, dptr(rho_h), None, sp)
        lib.lbm_step(lat._h, inner, sp)
        lib.lbm_read_fields(lat._h, *[dptr(o) for o in outs], sp)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            rc = lib.lbm_write_fields(lat._h, dptr(rho_h), None, sp)
            rc |= lib.lbm_step(lat._h, inner, sp)
            rc |= lib.lbm_read_fields(lat._h, *[dptr(o) for o in outs], sp)
            assert rc == 0, rc
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist)
        # host rho in per job, plus the boundary scalars (12 B per update) that the
        # fused path copies to the device in chunks of 16 updates
        sc_bytes = 12 if info["kernel"] in (L.KERNEL_FUSED, L.KERNEL_TWOPASS) else 0
        e2e = {"value": world * cells * inner * reps / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * cells / inner + sc_bytes,
               "d2h_bytes_per_step": 4 * 8 * cells / inner,
               "job": f"write_fields (host rho) + {inner} updates + read_fields (host rho,u,T)"}
    lat.close()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "nx": nx, "ny": ny, "storage": args.storage,
                   "physics": args.physics,
                   "timing": (f"median of {len(repeats)} timed regions of {args.steps} updates "
                              f"each ({sum(repeats) / 1e3:.2f} s in all; min "
                              f"{min(repeats) / args.steps * 1e3:.2f}, max "
                              f"{max(repeats) / args.steps * 1e3:.2f} us per update)"),
                   "kernel": {1: "split", 2: "fused", 5: "twopass"}[info["kernel"]],
                   "tile": [info["tile_cols"], info["tile_rows"]],
                   "cols_per_thread": info["cols_per_thread"],
                   "launch": ("16-update CUDA graphs"
                              if info["kernel"] in (L.KERNEL_FUSED, L.KERNEL_TWOPASS)
                              else "one launch per kernel"),
                   "untimed_updates_before": args.warmup + GRAPH_CHUNK,
                   "parallelism": f"replicas x{world}",
                   "l2": (f"state {info['device_bytes'] / 1e6:.0f} MB > L2 129 MB; no flush"
                          if info["device_bytes"] > L2_BYTES else
                          f"state {info['device_bytes'] / 1e6:.1f} MB fits in L2 (129 MB): an "
                          "L2-resident rate, no flush; not an HBM measurement"),
                   "bytes_per_cell_update": bytes_cell},
        "hbm_frac_step": value * 1e6 / world * bytes_cell / 1e9 / peak,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "status_bits": status,
    }
    print(json.dumps(line), flush=True)


def batch_channels(n: int = 96, seed: int = 3):
    """Seeded batch mix: n channels with length U[256, 2048], width U[32, 256], contact
    angle U[45, 135] degrees (the wall strength from the oracle's G_w -> angle table at
    0.86 Tc) and inlet period U[2000, 20000] (15.8 M nodes for n = 96)."""
    u = inputs.uniform01(4 * n, seed).reshape(n, 4)
    out = []
    for k in range(n):
        nx, ny = int(256 + u[k, 0] * 1792), int(32 + u[k, 1] * 224)
        p = inputs.base_params(Gw=inputs.wall_strength_for_angle(45.0 + 90.0 * u[k, 2]),
                               u_amp=0.02, u_period=float(2000 + int(18000 * u[k, 3])))
        out.append((nx, ny, p, inputs.noisy_density(nx, ny, inputs.RHO_V_086, 0.01, nx)))
    return out


def batch_arm(args):
    """MLUPS of one persistent launch per update over the batch mix, against the same
    lattices advanced one after another with lbm_step."""
    import torch
    from paper_1803_01756_gb300 import lattice as L
    torch.cuda.set_device(0)
    specs = batch_channels()
    lats = []
    for nx, ny, p, rho0 in specs:
        lat = L.Lattice(nx, ny, p, kernel=L.KERNEL_FUSED)
        lat.write_fields(rho0)
        lats.append(lat)
    cells = sum(nx * ny for nx, ny, _, _ in specs)
    stream = torch.cuda.current_stream()
    b = L.Batch(lats)
    info = b.info()
    b.step(args.warmup, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b.close()
    seq_steps = max(1, min(args.steps, 200))
    for lat in lats:
        lat.step(2, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.step(seq_steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    status = 0
    for lat in lats:
        status |= lat.status()
        lat.close()
    # the same, each lattice on the library's own kernel choice (the two-pass path for
    # lattices of at most 2^18 nodes)
    auto = []
    for nx, ny, p, rho0 in specs:
        lat = L.Lattice(nx, ny, p)
        lat.write_fields(rho0)
        lat.step(2, stream)
        auto.append(lat)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in auto:
        lat.step(seq_steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    auto_ms = e0.elapsed_time(e1)
    for lat in auto:
        status |= lat.status()
        lat.close()
    line = {
        "metric": "lattice updates per second (MLUPS), batched channels", "value":
        cells * args.steps / ms / 1e3, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {len(specs)} channels 256-2048 x 32-256, {cells} nodes",
                   "tiles": info["tiles"], "tile_rows": info["tile_rows"], "grid": info["grid"]},
        "sequential_mlups": cells * seq_steps / seq_ms / 1e3,
        "sequential_library_choice_mlups": cells * seq_steps / auto_ms / 1e3,
        "gpu_launches": args.steps,
        "status_bits": status,
    }
    print(json.dumps(line), flush=True)


def serving_jobs(n: int, steps: int, seed: int = 4):
    """Seeded job stream: 90 % channels with length U[256, 2048], width U[32, 256],
    contact angle U[45, 135] degrees (wall strength from the oracle's table), inlet period
    U[2000, 20000]; 10 % 4096 x 512 channels.  Poisson arrivals at 20 jobs/s."""
    u = inputs.uniform01(6 * n, seed).reshape(n, 6)
    jobs, t = [], 0.0
    for k in range(n):
        t += -np.log(1.0 - u[k, 5]) / 20.0
        if u[k, 0] < 0.1:
            nx, ny = 4096, 512
        else:
            nx, ny = int(256 + u[k, 1] * 1792), int(32 + u[k, 2] * 224)
        p = inputs.base_params(Gw=inputs.wall_strength_for_angle(45.0 + 90.0 * u[k, 3]),
                               u_period=float(2000 + int(18000 * u[k, 4])))
        jobs.append(dict(t=t, nx=nx, ny=ny, p=p, steps=steps, seed=1000 + k))
    return jobs


def run_server(args, L, jobs, rho0, storage):
    """Serve the job stream with the given population storage: Poisson arrivals from a
    client thread, continuous batching in the library's worker.  Returns (wall seconds,
    per-job latencies, peak device bytes)."""
    import threading
    import torch
    free, _ = torch.cuda.mem_get_info()
    srv = L.Server(hbm_budget=int(0.5 * free), max_active=args.max_active,
                   chunk_steps=args.chunk_steps)
    ids = [None] * len(jobs)
    t0 = time.perf_counter()

    def client():
        for k, j in enumerate(jobs):
            delay = t0 + j["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[k] = srv.submit(j["nx"], j["ny"], j["p"], j["steps"], rho0[k], storage=storage)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    lat = []
    for jid in ids:
        assert srv.wait(jid, 3600) == L.JOB_DONE
        lat.append(srv.poll(jid)[2])
    wall = time.perf_counter() - t0
    peak = srv.stats()["peak_bytes"]
    srv.close()
    return wall, lat, peak


def serving_arm(args):
    """jobs/hour and latency of the continuous-batching server, with BF16 population
    storage (the headline) and with FP32 storage (the batching gain alone), against the
    same arrivals solved one at a time in FP32 (first come, first served) on the library's
    kernel choice for each job (the two-pass path for jobs of at most 2^18 nodes, the fused
    kernel for larger ones)."""
    import torch
    from paper_1803_01756_gb300 import lattice as L
    torch.cuda.set_device(0)
    jobs = serving_jobs(args.jobs, args.job_steps)
    rho0 = [inputs.noisy_density(j["nx"], j["ny"], inputs.RHO_V_086, 0.01, j["seed"]) for j in jobs]
    cells = sum(j["nx"] * j["ny"] * j["steps"] for j in jobs)
    served = {}
    for name, storage in (("bf16", 1), ("f32", 0)):
        wall, lat, peak = run_server(args, L, jobs, rho0, storage)
        served[name] = {"jobs_per_hour": len(jobs) / wall * 3600, "wall_s": wall,
                        "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                        "mlups": cells / wall / 1e6, "peak_device_bytes": peak}
    # sequential FP32 solves of the same stream, one at a time
    service = []
    for k, j in enumerate(jobs):
        torch.cuda.synchronize()
        a = time.perf_counter()
        lt = L.Lattice(j["nx"], j["ny"], j["p"])
        lt.write_fields(rho0[k])
        lt.step(j["steps"])
        lt.read_fields()
        lt.close()
        service.append(time.perf_counter() - a)
    finish, seq_lat = 0.0, []
    for j, sv in zip(jobs, service):
        start = max(finish, j["t"])
        finish = start + sv
        seq_lat.append(finish - j["t"])
    head = served["bf16"]
    line = {
        "metric": "jobs/hour (continuous-batching server)", "value": head["jobs_per_hour"],
        "unit": "jobs/h", "n_gpus": 1, "steps": len(jobs), "warmup": 0,
        "ms_per_step": head["wall_s"] / len(jobs) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "serving: Poisson 20 jobs/s, 90 % 256-2048 x 32-256 channels, "
                               "10 % 4096x512", "jobs": len(jobs), "steps_per_job": args.job_steps,
                   "storage": "bf16", "arithmetic": "f32", "chunk_steps": args.chunk_steps,
                   "max_active": args.max_active, "peak_device_bytes": head["peak_device_bytes"]},
        "latency_s": {"p50": head["p50"], "p99": head["p99"]},
        "mlups": head["mlups"],
        "server_fp32": served["f32"],
        "sequential_fp32": {"jobs_per_hour": len(jobs) / finish * 3600,
                            "p50": float(np.percentile(seq_lat, 50)),
                            "p99": float(np.percentile(seq_lat, 99)),
                            "mlups": cells / sum(service) / 1e6},
    }
    print(json.dumps(line), flush=True)


def condensation_arm(args):
    """The 1024 x 128 channel (and its walls-at-0.65-Tc variant) on the GPU: droplet
    statistics of the density field at intervals, and the update rate of the run."""
    import torch
    from paper_1803_01756_gb300 import lattice as L
    torch.cuda.set_device(0)
    thr = 0.5 * (inputs.RHO_L_086 + inputs.RHO_V_086)
    report = {}
    for name, every in (("channel_1024x128", 10000), ("cold_1024x128", 5000)):
        w = inputs.workload(name)
        lat = L.Lattice(w["nx"], w["ny"], w["params"])
        lat.write_fields(inputs.initial_density(w))
        rows, ms = {}, 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while lat.t < w["steps"]:
            e0.record()
            lat.step(every)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            rho = lat.read_fields(check=False)[0]
            st = L.droplet_stats(rho, thr, inputs.RHO_V_086)
            st["status_bits"] = lat.status()
            rows[lat.t] = st
        lat.close()
        report[name] = {"mlups": w["nx"] * w["ny"] * w["steps"] / ms / 1e3, "stats": rows}
    line = {"metric": "droplet count / spacing / condensed mass, 1024 x 128 channel",
            "value": report["channel_1024x128"]["mlups"], "unit": "MLUPS", "n_gpus": 1,
            "steps": inputs.workload("channel_1024x128")["steps"], "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "channel_1024x128 and cold_1024x128"},
            "condensation": report}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="channel_4096x512", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--kernel", default="auto",
                    choices=["auto", "split", "fused", "fused1", "fused2", "twopass"],
                    help="fused1 / fused2: the fused kernel with one / two lattice columns per thread")
    ap.add_argument("--physics", default="full", choices=sorted(PHYSICS),
                    help="full update, or without the energy equation / the pseudopotential")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="population storage (FP32 arithmetic in every case)")
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--min-timed-s", type=float, default=2.0,
                    help="repeat the K-update timed region until the repeats add up to this")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true",
                    help="skip the oracle's all-cores figure (one process per host core)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-inner", type=int, default=100)
    ap.add_argument("--e2e-reps", type=int, default=5)
    ap.add_argument("--mode", default="lattice",
                    choices=["lattice", "batch", "serve", "condensation"],
                    help="lattice: MLUPS of one channel; batch: one launch per update over 96 "
                         "channels; serve: the job server")
    ap.add_argument("--jobs", type=int, default=160)
    ap.add_argument("--job-steps", type=int, default=10000)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--chunk-steps", type=int, default=250)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    world, rank, local, dist = setup_distributed()
    try:
        if args.impl == "reference":
            reference_arm(args, world, rank)
        elif args.mode == "batch":
            if rank == 0:
                batch_arm(args)
        elif args.mode == "serve":
            if rank == 0:
                serving_arm(args)
        elif args.mode == "condensation":
            if rank == 0:
                condensation_arm(args)
        else:
            our_arm(args, world, rank, local, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
