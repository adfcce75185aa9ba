"""Benchmark of the fused D2Q9 ADE-LBM step on the 4096 x 4096 reactive
porous workload.

One benchmark step is one lattice time step of the whole hot path: pull
streaming with bounce-back, max-entropy Dirichlet inlet / Neumann outlet,
moments, BGK collision with the surface reaction sink, and the dissolution
pass (mineral update and exact mask flips).

Workload (synthetic, seeded): 4096 x 4096 nodes, random overlapping disks
(radius 8-24) at porosity 0.6, 16-mode stream-function velocity with
|v|max = 0.05, tau = 0.7, first-order surface reaction k = 1e-3 with unit
mineral per solid node, Dirichlet c = 1 on the west side, zero-flux Neumann
on the east side, periodic in y, c0 = 0.  The populations (2 x 604 MB) are
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
instead, on a crop of the same workload sized to finish in about a minute.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LBM-ADE GLUPS & % HBM roofline (FP32 vs FP64); adjoint/forward time ratio"
# Algorithmic bytes of the fused step per node and launch: a fluid node reads
# and writes 9 populations, reads 2 velocity components and one byte of solid
# flag; a solid node costs its flag byte.  (The library stores the flag in a
# 4-byte word that also encodes the neighbourhood; the algorithmic count keeps
# the information content.)
BYTES_FLUID = {32: 9 * 4 * 2 + 2 * 4 + 1, 64: 9 * 8 * 2 + 2 * 8 + 1}
BYTES_SOLID = 1
# FP64 arithmetic of the fused step per fluid node (an FMA counts 2): 8 adds
# for u, 14 for the factors shared by all directions (v.v, 1 - omega, the
# rest population's (1 - k) u, the e.v of the diagonals), 15 per opposite
# pair (4 pairs).  The counters of the FP64 kernel show about 109 executed,
# the rest being boundary code and idle lanes in blocks on a side.
FLOPS_FLUID_FP64 = 82
FP64_PEAK_GFLOPS = 1250.0  # nominal dense FP64 of one GB300


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def shard_instances(sizes, rank, world):
    """Indices of the batch instances rank `rank` of `world` runs: largest
    first, each to the rank with the least work so far (ties: lowest rank).
    Every rank computes the same assignment; the instances are independent,
    so the ranks exchange nothing but the final timing."""
    load = [0] * world
    owner = {}
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def reduce_max(value, dist=None, device="cpu"):
    """Max of a float over all ranks (the value itself without a process
    group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


_FP64_FMA_SRC = r"""
// FP64 FMA rate of this GPU: independent FMA chains per thread, no memory.
#include <cstdio>
#include <cuda_runtime.h>
__global__ void chains(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains live
}
int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  double* out = nullptr;
  cudaMalloc(&out, 8 * 1024 * sizeof(double));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  chains<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) chains<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double flops = 5.0 * blocks * threads * (double)iters * 8 * 2;
  printf("%.3f\n", flops / (ms * 1e-3) / 1e9);
  return cudaGetLastError() != cudaSuccess;
}
"""


def measured_fp64_peak_gflops():
    """FP64 FMA throughput of this GPU from a small microbenchmark (compiled
    with nvcc for sm_103a on the spot), else the part's nominal rate."""
    import shutil
    import subprocess
    import tempfile
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    try:
        with tempfile.TemporaryDirectory() as d:
            src, exe = os.path.join(d, "fma.cu"), os.path.join(d, "fma")
            with open(src, "w") as fh:
                fh.write(_FP64_FMA_SRC)
            subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                            src], check=True, capture_output=True, timeout=120)
            out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60)
            return float(out.stdout.strip()), "measured (FP64 FMA chains)"
    except (OSError, ValueError, subprocess.SubprocessError):
        return FP64_PEAK_GFLOPS, "nominal FP64 rate of the part"


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons of the benchmark's GPU,
    sampled during the timed region.  Reads NVML through ctypes every
    millisecond on a thread (so even a few-millisecond region gets samples);
    without NVML it falls back to nvidia-smi every 200 ms.  Reads only: no
    setting of the GPU is changed."""

    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.samples = []  # (sm_mhz, reason bits)
        self.sm_max = None
        self.proc = None
        self.source = None

    def _uuid(self):
        try:
            import torch
            u = torch.cuda.get_device_properties(self.cuda_index).uuid
            return "GPU-" + str(u)
        except Exception:
            return None

    def _start_nvml(self):
        import ctypes
        import threading
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        uuid = self._uuid()
        if uuid is None or nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
            nv.nvmlShutdown()
            return False
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
            self.sm_max = float(mx.value)
        reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        self._stop = threading.Event()

        def loop():
            mhz, bits = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self._stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and \
                        reasons_fn(h, ctypes.byref(bits)) == 0:
                    self.samples.append((float(mhz.value), int(bits.value)))
                self._stop.wait(0.001)

        self._nv = nv
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        self.source = "nvml, 1 ms"
        return True

    def __enter__(self):
        try:
            if self._start_nvml():
                return self
        except (OSError, AttributeError):
            pass
        try:
            ident = self._uuid() or str(self.cuda_index)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={ident}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 200 ms"
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.source and self.source.startswith("nvml"):
            self._stop.set()
            self._thread.join(timeout=2)
            self._nv.nvmlShutdown()
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                     "sw_power_cap"]
            bits = {v: k for k, v in self.REASONS.items()}
            for ln in out.splitlines():
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    mhz = float(parts[1])
                    self.sm_max = float(parts[2])
                except ValueError:
                    continue
                r = 0
                for name, val in zip(names, parts[5:9]):
                    if val.lower() in ("active", "1"):
                        r |= bits[name]
                self.samples.append((mhz, r))

    def summary(self):
        sm = [m for m, _ in self.samples]
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.sm_max,
                "reasons": sorted(reasons), "samples": len(sm), "source": self.source}


def workload(n):
    from paper_1601_02708_gb300 import inputs
    case = inputs.porous_case(n, n, seed=2)
    return case


def lattice_kwargs(case):
    return {k: case[k] for k in ("edges", "solid", "vel", "u0", "react_mode", "k",
                                 "dissolution", "mineral")}


def cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate_one_thread(steps, crop):
    """Oracle node-steps per second on one thread: a child process with
    OMP_NUM_THREADS=1 (the in-process oracle keeps the threads it started
    with).  Returns (seconds, nodes)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "from paper_1601_02708_gb300 import inputs; "
            "c = inputs.porous_case(64, 64, seed=2); c['tau'] = 0.7; "
            "dt, n, _ = bench.run_oracle(c, %d, crop=%d); print(json.dumps([dt, n]))"
            % (ROOT, steps, crop))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=600)
    dt, n = json.loads(r.stdout.strip().splitlines()[-1])
    return dt, n


def run_oracle(case, steps, crop=None):
    """Time `steps` oracle steps (FP64 CPU) on the workload or a crop of it.
    Returns (seconds, nodes, threads)."""
    import oracle
    oracle.build()
    kw = lattice_kwargs(case)
    nx, ny = case["nx"], case["ny"]
    ud, q = case["u_dir"], case["q_neu"]
    if crop is not None:
        from paper_1601_02708_gb300 import inputs
        c = inputs.porous_case(crop, crop, seed=2)
        kw, nx, ny, ud, q = lattice_kwargs(c), crop, crop, c["u_dir"], c["q_neu"]
    ref = oracle.LBMOracle(nx, ny, case["tau"], **kw)
    t0 = time.perf_counter()
    ref.substeps(steps, 1, ud, ud, q)
    dt = time.perf_counter() - t0
    threads = _env_int("OMP_NUM_THREADS", os.cpu_count() or 1)
    return dt, nx * ny, threads


def reference_arm(args):
    """The FP64 CPU oracle timed as it stands, each step a time step of a
    crop of the workload sized so that all steps end in about a minute."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    case = workload(64)  # parameters only; the crop is regenerated
    case["tau"] = 0.7
    cal_t, cal_nodes, _ = run_oracle(case, 2, crop=256)
    rate = 2 * cal_nodes / max(cal_t, 1e-9)               # node-steps per second
    total = max(1, args.steps + args.warmup)
    side = int(math.sqrt(60.0 * rate / total) // 64 * 64)
    side = max(64, min(args.size, side))
    if args.warmup:
        run_oracle(case, args.warmup, crop=side)
    dt, nodes, threads = run_oracle(case, args.steps, crop=side)
    glups = nodes * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"reactive porous D2Q9 ADE-LBM, {side}x{side} crop of "
                               "the 4096x4096 generator (porosity 0.6, tau 0.7, k 1e-3, "
                               "dissolution)", "nx": side, "ny": side},
        "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} steps of a {side}x{side} crop"},
        "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--fp64-steps", type=int, default=300)
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel-steps", type=int, default=1000)
    ap.add_argument("--bimolecular-steps", type=int, default=300,
                    help="steps of the two-invariant leg (instantaneous A + 2B -> C; 0: skip)")
    ap.add_argument("--walls-steps", type=int, default=500,
                    help="steps of the leg with maximum-entropy pore walls (0: skip)")
    ap.add_argument("--adjoint-steps", type=int, default=5000)
    ap.add_argument("--hybrid-coarse", type=int, default=200)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--kernel", default="auto", choices=["auto", "generic", "tma"],
                    help="FP32 step kernel of the headline lattice (auto: the library's choice)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    if args.impl == "reference":
        reference_arm(args)
        return

    import torch

    from paper_1601_02708_gb300 import LBM

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return reduce_max(v, dist, "cuda")

    n = args.size
    case = workload(n)
    kw = lattice_kwargs(case)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ud, q = dev(case["u_dir"]), dev(case["q_neu"])
    nodes = n * n
    stream = torch.cuda.current_stream()

    # ---- FP32 fused step: the headline ------------------------------------
    # one GPU: the 4096 x 4096 lattice; N GPUs: one lattice of 4096 x 4096N
    # nodes split into row slabs, one 4096 x 4096 slab per rank, the one-row
    # halo moved by NCCL point-to-point operations between the two halves of
    # every step (weak scaling: the work per GPU stays fixed)
    if world > 1:
        from paper_1601_02708_gb300 import inputs as _inputs
        from paper_1601_02708_gb300.partition import SlabLattice
        whole = _inputs.porous_case(n, n * world, seed=2)
        lat = SlabLattice(n, n * world, whole["tau"], rank=rank, world=world, precision=32,
                          **lattice_kwargs(whole))
        ud_w, q_w = dev(whole["u_dir"]), dev(whole["q_neu"])
        if args.kernel != "auto":
            for sl in lat.slabs:
                sl.set_kernel(args.kernel)
        lat.substeps(args.warmup, 1, ud_w, ud_w, q_w)
        ud, q = ud_w, q_w
        timed = lat.slabs[0]
    else:
        lat = LBM(n, n, case["tau"], precision=32, **kw)
        if args.kernel != "auto":
            lat.set_kernel(args.kernel)
        lat.substeps(args.warmup, 1, ud, ud, q)
        timed = lat
    variant = timed.kernel()
    kernel_name = {"tma": "lbm_step_tma<false>", "generic": "lbm_step<float, false>"}[variant]
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        ev0.record(stream)
        lat.substeps(args.steps, 1, ud, ud, q)
        ev1.record(stream)
        ev1.synchronize()
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    launches = 2 * args.steps  # one step and one dissolution launch per step
    # per-kernel durations from CUDA events around every launch, on a
    # separate stretch of steps (the events add small gaps between launches)
    timed.kernel_timing(True)
    lat.substeps(args.kernel_steps, 1, ud, ud, q)
    step_ms, step_n, diss_ms, diss_n = timed.kernel_times()
    timed.kernel_timing(False)
    diag = timed.diagnostics()  # this rank's lattice (or slab): n x n nodes
    n_solid = diag["n_solid"]
    n_fluid = nodes - n_solid
    lat.close()
    del lat, timed
    torch.cuda.empty_cache()
    ud, q = dev(case["u_dir"]), dev(case["q_neu"])

    value = world * nodes * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peak_gbs()
    bytes_step = BYTES_FLUID[32] * n_fluid + BYTES_SOLID * n_solid
    per_launch_ms = step_ms / max(step_n, 1)
    achieved = bytes_step / (per_launch_ms / 1e3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", {"tma": "lbm_step_traffic.json",
                                            "generic": "lbm_step_generic_traffic.json"}[variant])
    try:
        from paper_1601_02708_gb300 import build as _b
        import hashlib
        rec = json.load(open(tpath))
        h = hashlib.sha256()
        for name in rec["source_files"]:  # the files that define the step kernel
            h.update(open(os.path.join(_b.CSRC, name), "rb").read())
        if rec.get("source_sha256") == h.hexdigest():
            traffic = rec["dram_bytes_per_launch_full_size"]
    except (OSError, ValueError, KeyError):
        traffic = None

    # ---- FP64 mode of the same kernels ---------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        lat64 = LBM(n, n, case["tau"], precision=64, **kw)
        lat64.substeps(3, 1, ud, ud, q)
        barrier()
        lat64.kernel_timing(True)
        ev0.record(stream)
        lat64.substeps(args.fp64_steps, 1, ud, ud, q)
        ev1.record(stream)
        ev1.synchronize()
        ms64 = max_over_ranks(ev0.elapsed_time(ev1))
        s64_ms, s64_n, _, _ = lat64.kernel_times()
        d64 = lat64.diagnostics()
        lat64.close()
        del lat64
        torch.cuda.empty_cache()
        b64 = BYTES_FLUID[64] * (nodes - d64["n_solid"]) + BYTES_SOLID * d64["n_solid"]
        a64 = b64 / (s64_ms / max(s64_n, 1) / 1e3) / 1e9
        f64_gflops = FLOPS_FLUID_FP64 * (nodes - d64["n_solid"]) / (s64_ms / max(s64_n, 1) / 1e3) / 1e9
        fp64_peak, fp64_kind = measured_fp64_peak_gflops()
        fp64 = {"value": world * nodes * args.fp64_steps / (ms64 / 1e3) / 1e9,
                "unit": "GLUPS", "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps,
                "roofline": {"bound": "hbm", "achieved": a64, "peak": peak,
                             "unit": "GB/s", "frac": a64 / peak},
                # GB300 runs FP64 at 1/64 of FP32: the FP64 lattice is bound by
                # its FP64 arithmetic (moments, equilibrium and collision with
                # the sink), against the FP64 FMA rate measured on the spot
                "alu_roofline": {"bound": "alu", "achieved": f64_gflops, "peak": fp64_peak,
                                 "unit": "GFLOP/s", "frac": f64_gflops / fp64_peak,
                                 "peak_kind": fp64_kind,
                                 "flops_per_fluid_node": FLOPS_FLUID_FP64}}

    # ---- the same workload with maximum-entropy pore walls ---------------------
    # both precisions of the wall solve: the Lagrange multiplier by Newton's
    # method in FP64 ("maxent") and in FP32 ("maxent_lattice")
    walls = None
    if args.walls_steps > 0:
        walls = {}
        for mode in ("maxent", "maxent_lattice"):
            latw = LBM(n, n, case["tau"], precision=32, walls=mode, **kw)
            latw.substeps(3, 1, ud, ud, q)
            barrier()
            ev0.record(stream)
            latw.substeps(args.walls_steps, 1, ud, ud, q)
            ev1.record(stream)
            ev1.synchronize()
            msw = max_over_ranks(ev0.elapsed_time(ev1))
            latw.kernel_timing(True)
            latw.substeps(min(args.kernel_steps, args.walls_steps), 1, ud, ud, q)
            sw_ms, sw_n, _, _ = latw.kernel_times()
            dw = latw.diagnostics()
            latw.close()
            del latw
            torch.cuda.empty_cache()
            bw = BYTES_FLUID[32] * (nodes - dw["n_solid"]) + BYTES_SOLID * dw["n_solid"]
            aw = bw / (sw_ms / max(sw_n, 1) / 1e3) / 1e9
            walls[mode] = {
                "value": world * nodes * args.walls_steps / (msw / 1e3) / 1e9,
                "unit": "GLUPS", "steps": args.walls_steps,
                "newton_precision": "f64" if mode == "maxent" else "f32",
                "ms_per_step": msw / args.walls_steps,
                "kernel_ms_per_launch": sw_ms / max(sw_n, 1),
                "bc_infeasible": dw["bc_infeasible"], "newton_fail": dw["newton_fail"],
                "roofline": {"bound": "hbm", "achieved": aw, "peak": peak, "unit": "GB/s",
                             "frac": aw / peak}}

    # ---- instantaneous bimolecular reaction: two invariants, then species ------
    bimol = None
    if args.bimolecular_steps > 0:
        from paper_1601_02708_gb300 import Bimolecular, species_from_invariants
        fluid = kw["solid"] == 0
        uA0 = np.zeros((n, n))
        uB0 = np.where(fluid, 0.5, 0.0)  # B resident; A enters at the inlet
        coeffs = (1.0, 2.0, 1.0)
        a_in = ud  # alpha = u_A + u_C at the inlet: the inlet value of A
        b_in = torch.zeros_like(ud)
        probe = Bimolecular(n, n, case["tau"], coeffs, uA0, uB0, precision=32,
                            edges=kw["edges"], solid=kw["solid"], vel=kw["vel"])
        default_pair = probe.pair is not None  # the library's default for this size
        probe.close()
        del probe
        msb = {}
        for fused in (False, True):  # two lattices a substep, then the fused pair kernel
            if fused:
                bm.close()
                del bm
                torch.cuda.empty_cache()
            bm = Bimolecular(n, n, case["tau"], coeffs, uA0, uB0, precision=32, fused=fused,
                             edges=kw["edges"], solid=kw["solid"], vel=kw["vel"])
            bm.substeps(3, 1, (a_in, a_in), (b_in, b_in))
            barrier()
            ev0.record(stream)
            bm.substeps(args.bimolecular_steps, 1, (a_in, a_in), (b_in, b_in))
            ev1.record(stream)
            ev1.synchronize()
            msb[fused] = max_over_ranks(ev0.elapsed_time(ev1))
        al = torch.empty((n, n), dtype=torch.float64, device="cuda")
        be = torch.empty_like(al)
        bm.alpha.concentration(out=al)
        bm.beta.concentration(out=be)
        spc = tuple(torch.empty_like(al) for _ in range(3))
        species_from_invariants(al, be, coeffs, out=spc)  # warm
        torch.cuda.synchronize()
        reps = 20  # back to back, so the host's share of each call overlaps the GPU's
        ev0.record(stream)
        for _ in range(reps):
            species_from_invariants(al, be, coeffs, out=spc)
        ev1.record(stream)
        ev1.synchronize()
        epi_ms = ev0.elapsed_time(ev1) / reps
        uA, uB, uC = spc
        produced = float(uC.sum())
        bm.close()
        del bm, al, be, uA, uB, uC
        torch.cuda.empty_cache()
        ms_f = msb[True] / args.bimolecular_steps
        ms_u = msb[False] / args.bimolecular_steps
        default_fused = bool(default_pair)  # what Bimolecular(fused=None) chose
        ms_d = ms_f if default_fused else ms_u
        n_sol = int((kw["solid"] != 0).sum())
        # two fields' populations and one velocity and mask read per node (the
        # fused pair's algorithmic bytes; two separate lattices move these too
        # plus a second velocity and mask)
        bp = (2 * 9 * 4 * 2 + 2 * 4 + 1) * (nodes - n_sol) + BYTES_SOLID * n_sol
        ap_ = bp / (ms_d / 1e3) / 1e9
        bimol = {"value": world * 2 * nodes / (ms_d / 1e3) / 1e9,
                 "unit": "GLUPS (both invariants)", "steps": args.bimolecular_steps,
                 "default": "fused pair" if default_fused else "two lattices",
                 "ms_per_step": ms_d, "fused_ms_per_step": ms_f, "unfused_ms_per_step": ms_u,
                 "roofline": {"bound": "hbm", "achieved": ap_, "peak": peak, "unit": "GB/s",
                              "frac": ap_ / peak, "bytes_per_fluid_node": 2 * 9 * 4 * 2 + 2 * 4 + 1,
                              "timing": "whole substep calls (launch gaps included)"},
                 "species_ms": epi_ms, "species_gbs": 5 * 8 * nodes / (epi_ms / 1e3) / 1e9,
                 "sum_uC": produced,
                 "reaction": "A + 2B -> C, instantaneous; A enters at the inlet, B resident"}

    # ---- end to end through the public API with host buffers -----------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_solid = pin(kw["solid"].astype(np.uint8))
        h_vel, h_min, h_u0 = pin(kw["vel"]), pin(kw["mineral"]), pin(kw["u0"])
        h_ud, h_q = pin(case["u_dir"]), pin(case["q_neu"])
        h_out = torch.empty((n, n), dtype=torch.float32).pin_memory()
        kwh = dict(kw, solid=h_solid, vel=h_vel, mineral=h_min, u0=h_u0)
        barrier()
        t0 = time.perf_counter()
        lat2 = LBM(n, n, case["tau"], precision=32, **kwh)
        lat2.substeps(args.steps, 1, h_ud, h_ud, h_q)
        lat2.concentration(h_out, precision=32)
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        lat2.close()
        bi = sum(t.numel() * t.element_size() for t in (h_solid, h_vel, h_min, h_u0)) + \
            3 * h_ud.numel() * 8
        bo = h_out.numel() * h_out.element_size()
        e2e = {"value": world * nodes * args.steps / t_e2e / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": bi / args.steps, "d2h_bytes_per_step": bo / args.steps,
               "seconds": t_e2e}

    # ---- batched ragged instances (one persistent launch per step) -------------
    batched = None
    if not args.no_batch and args.batch_steps > 0:
        from paper_1601_02708_gb300 import LBMBatch, inputs
        all_cases = inputs.batch_cases(n_inst=args.batch_instances)
        sizes = [c["nx"] * c["ny"] for c in all_cases]
        cases = [all_cases[i] for i in shard_instances(sizes, rank, world)]
        bstream = torch.cuda.Stream()
        members = [LBM(c["nx"], c["ny"], c["tau"], precision=32, stream=bstream.cuda_stream,
                       **lattice_kwargs(c)) for c in cases]
        batch = LBMBatch(members)
        bud = [dev(c["u_dir"]) for c in cases]
        bq = [dev(c["q_neu"]) for c in cases]
        batch.substeps(1, 1, bud, bud, bq)  # loads the edge data into every member
        tune = {} if args.no_autotune else batch.autotune(trial_steps=20, repeats=2)
        batch.substeps(args.warmup, 1, bud, bud, bq)
        batch.time_steps(args.batch_steps)  # records the graph of the timed length
        barrier()
        bms = max_over_ranks(batch.time_steps(args.batch_steps))
        bnodes = sum(sizes)  # every rank's instances together
        bglups = bnodes * args.batch_steps / (bms / 1e3) / 1e9
        batched = {"value": bglups, "unit": "GLUPS", "instances": len(all_cases),
                   "instances_per_rank": len(cases), "nodes": bnodes,
                   "steps": args.batch_steps,
                   "scaling": "strong (instances sharded across ranks)" if world > 1 else None,
                   "ms_per_step": bms / args.batch_steps,
                   "ratio_to_single_lattice": bglups / value,
                   "tile_shape": LBMBatch.shapes()[batch.shape],
                   "autotune_ms": {str(LBMBatch.shapes()[k]): v for k, v in tune.items()},
                   "workload": f"{len(all_cases)} instances, side log-uniform 64-1024, porosity "
                               "U[0.4,0.8], tau U[0.6,1.2], k 1e-3 with dissolution"}
        batch.close()
        for m in members:
            m.close()
        del members, batch
        torch.cuda.empty_cache()

    # ---- adjoint: gradient of the outlet breakthrough (512^2 workload) -------
    adjoint = None
    if args.adjoint_steps > 0:
        from paper_1601_02708_gb300 import inputs
        c4 = inputs.adjoint_case()
        kw4 = {k: c4[k] for k in ("edges", "solid", "vel", "u0", "react_mode", "k_field")}
        lat4 = LBM(c4["nx"], c4["ny"], c4["tau"], precision=32, **kw4)
        ud4, q4 = dev(c4["u_dir"]), dev(c4["q_neu"])
        start = lat4.save()
        na = args.adjoint_steps
        # two warm-up calls of each path: the first sizes the checkpoint
        # buffers, the second records its launch sequence into a CUDA graph,
        # so the timed calls replay recorded graphs (forward and adjoint alike)
        for _ in range(2):
            lat4.adjoint(na, 1, ud4, ud4, q4, stride=na)
            lat4.restore(start)
            lat4.substeps(na, 1, ud4, ud4, q4)
            lat4.restore(start)
        barrier()
        ev0.record(stream)
        lat4.substeps(na, 1, ud4, ud4, q4)
        ev1.record(stream)
        ev1.synchronize()
        fwd_ms = max_over_ranks(ev0.elapsed_time(ev1))
        lat4.restore(start)
        barrier()
        ev0.record(stream)
        r4 = lat4.adjoint(na, 1, ud4, ud4, q4, stride=na)
        ev1.record(stream)
        ev1.synchronize()
        adj_ms = max_over_ranks(ev0.elapsed_time(ev1))
        # the same gradient with sqrt(n) checkpoints and one recompute
        sq = int(math.ceil(math.sqrt(na)))
        for _ in range(2):
            lat4.restore(start)
            lat4.adjoint(na, 1, ud4, ud4, q4, stride=sq)
        lat4.restore(start)
        barrier()
        ev0.record(stream)
        lat4.adjoint(na, 1, ud4, ud4, q4, stride=sq)
        ev1.record(stream)
        ev1.synchronize()
        ck_ms = max_over_ranks(ev0.elapsed_time(ev1))
        lat4.close()
        del lat4
        torch.cuda.empty_cache()
        adjoint = {"ratio": adj_ms / fwd_ms, "forward_ms": fwd_ms, "adjoint_ms": adj_ms,
                   "forward_us_per_step_graph_replay": fwd_ms * 1e3 / na,
                   "reverse_only_ratio": (adj_ms - fwd_ms) / fwd_ms, "steps": na,
                   "stride": na, "history": "whole (u and Neumann branches of every step "
                                            "stored by the forward run; no recompute)",
                   "checkpointed": {"stride": sq, "adjoint_ms": ck_ms, "ratio": ck_ms / fwd_ms},
                   "J": r4["J"], "dtype": "f32",
                   "workload": "512x512 porous (porosity 0.6, disks r 8-24, stream function "
                               "|v|max 0.05 plus mean flow 0.15 along x), bulk rate field "
                               "1e-3 (1 +- 0.2 U), tau 0.7, Dirichlet 1 west, zero-flux "
                               "east, periodic y; J = outlet breakthrough; gradients "
                               "w.r.t. every node's rate and the inlet value",
                   "graph_replay": True,
                   "note": "adjoint_ms is one lbm_adjoint call: forward recording the "
                           "history, reverse sweep, gradients copied to the host; the "
                           "checkpointed call adds the recompute of every segment; all "
                           "timed calls replay recorded CUDA graphs"}

    # ---- hybrid runs (Algorithm 1): Q1 continuum + lattice, Schwarz ---------
    hybrid = None
    if args.hybrid_coarse > 0:
        from paper_1601_02708_gb300 import inputs
        from paper_1601_02708_gb300.hybrid import Hybrid
        hybrid = {}
        for name, layout, ncoarse in (
                ("plain", inputs.hybrid_plain_layout(), 100),
                ("pore_block", inputs.hybrid_block_layout(), args.hybrid_coarse),
                ("many_blocks", inputs.hybrid_multiblock_layout(), 50)):
            run = Hybrid(layout, precision=32)
            run.run(1)  # warm-up: allocations, first solves
            barrier()
            ev0.record(stream)
            t0 = time.perf_counter()
            run.run(ncoarse)
            ev1.record(stream)
            ev1.synchronize()
            wall = time.perf_counter() - t0
            hms = max_over_ranks(ev0.elapsed_time(ev1))
            lats = layout["lbms"] if "lbms" in layout else [layout["lbm"]]
            node_steps = sum(a["nx"] * a["ny"] for a in lats) * layout["eta"] * \
                layout["max_iter"] * ncoarse
            its = run.solver_iters[-ncoarse * layout["max_iter"]:]
            hybrid[name] = {
                "coarse_steps": ncoarse, "ms_per_coarse_step": hms / ncoarse,
                "lattices": [[a["nx"], a["ny"]] for a in lats],
                "fem_elements": [layout["fem"]["nex"], layout["fem"]["ney"]],
                "substeps": layout["eta"], "schwarz_iterations": layout["max_iter"],
                "lattice_glups": world * node_steps / (hms / 1e3) / 1e9,
                "fem_solver_iterations_mean": float(np.mean(its)),
                "wall_s": wall}
            if name == "plain":
                # the lattice's eta substeps alone, replayed from their recorded
                # graph: the small lattice is launch-bound, so time per substep
                lat, eta = run.lbm, layout["eta"]
                snap = lat.save()
                for _ in range(3):
                    lat.substeps(eta, eta, run.ua[0], run.ub[0], run.q)
                reps = 200
                ev0.record(stream)
                for _ in range(reps):
                    lat.substeps(eta, eta, run.ua[0], run.ub[0], run.q)
                ev1.record(stream)
                ev1.synchronize()
                hybrid[name]["lattice_us_per_substep_graph_replay"] = \
                    ev0.elapsed_time(ev1) * 1e3 / (reps * eta)
                lat.restore(snap)
            run.close()
            del run
            torch.cuda.empty_cache()

    # ---- CPU oracle on a bounded sample --------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_steps > 0:
        dt, cn, threads = run_oracle(case, args.cpu_steps)
        cpu = {"value": cn * args.cpu_steps / dt / 1e9, "unit": "GLUPS", "cores": threads,
               "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"{args.cpu_steps} steps of the full {n}x{n} lattice, FP64, "
                         f"{dt:.1f} s"}
        try:  # the same oracle on one thread, 2 steps of a 2048 x 2048 crop
            dt1, n1 = oracle_rate_one_thread(2, 2048)
            cpu["one_thread"] = {"value": n1 * 2 / dt1 / 1e9, "unit": "GLUPS", "cores": 1,
                                 "sample": f"2 steps of a 2048x2048 crop, FP64, {dt1:.1f} s"}
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            cpu["one_thread"] = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"reactive porous D2Q9 ADE-LBM {n}x{n}, disks r 8-24 at "
                                   "porosity 0.6, 16-mode stream function |v|max 0.05, "
                                   "tau 0.7, surface k 1e-3 with dissolution, Dirichlet "
                                   "inlet / Neumann outlet, periodic y",
                       "nx": n, "ny": n, "fluid_nodes": n_fluid,
                       "parallelism": (f"one {n}x{n * world} lattice split in {world} row "
                                       f"slabs of {n}x{n}, halo over NCCL")
                                      if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (2 x 604 MB populations), no flush"},
            "fluid_glups": world * n_fluid * args.steps / (ms / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "kernel": kernel_name,
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": bytes_step,
                         "kernel_ms_per_launch": per_launch_ms,
                         "kernel_timing_steps": args.kernel_steps,
                         "dissolve_ms_per_launch": diss_ms / max(diss_n, 1)},
            "fp64": fp64, "maxent_walls": walls, "bimolecular": bimol, "batched": batched, "adjoint": adjoint, "hybrid": hybrid,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
