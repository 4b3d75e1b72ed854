#!/usr/bin/env python
"""Benchmark of the body-free vortex-in-cell step on GB300.

Workload: 1024 x 1024 nodes on [-1, 1]^2 (2048^2 padded FFT), 1e6 point
vortices uniform in the central 80 %, strengths N(0, 1e-4), seed 1001.  One
step = regularize (R_v), unbounded Poisson solve with the LGF (L^{-1}),
spectral node velocity (curl) and interpolation to the vortices (E_v), i.e.
one call of pf_vic_velocity.  Inputs are device resident; L2 is flushed
(256 MB write) between timed steps, outside the timed events.

`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload per step, extrapolated to a full step.

Under torchrun every rank runs an independent replica (the path does not
shard); the reported value is the whole-job aggregate.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# 32 hardware work queues (read when CUDA starts, so before torch is imported):
# the batched and served workloads run one stream per instance
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "VIC steps/s (R+L^-1+Schur+E) at <=1e-5 rel err vs FP64; p50/p99 latency"
UNIT = "steps/s"
WORKLOAD = ("vic_1024: 1024x1024 nodes, dx=2/1023, 2048^2 padded LGF FFT, 1e6 vortices uniform in the "
            "central 80%, Gamma~N(0,1e-4), seed 1001; body-free step R_v + L^-1 + curl + E_v")
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, world, device="cuda"):
    """The largest x over the ranks of the process group (x itself on one rank):
    every timing of a multi-GPU run is the slowest rank's."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle timing
ORACLE_SAMPLE = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs
nsub, nodes, reps, worker = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4])
wl = inputs.vic_1024()
g = wl["grid"]; og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
X, Y, G = wl["X"], wl["Y"], wl["G"]
nv = len(X)
t0 = time.perf_counter(); tab = lgf_table(g.nx + 1, g.ny + 1); t_tab = time.perf_counter() - t0
w_full = OV.regularize(og, X, Y, G)          # source field of the sampled direct sums
f = np.zeros((g.ny, g.nx))
rng = np.random.default_rng(100 + worker)
sys.stdout.write("ready\n"); sys.stdout.flush()
sys.stdin.readline()                          # all workers start the timed part together
out = []
for r in range(reps):
    sel = rng.integers(0, nv, nsub)
    t0 = time.perf_counter(); OV.regularize(og, X[sel], Y[sel], G[sel]); t_reg = (time.perf_counter() - t0) / nsub
    ti = rng.integers(0, g.nx, nodes); tj = rng.integers(0, g.ny, nodes)
    t0 = time.perf_counter(); OV.inv_laplacian_at(og, w_full, ti, tj, tab); t_node = (time.perf_counter() - t0) / nodes
    t0 = time.perf_counter(); OV.interpolate(og, f, X[sel], Y[sel]); t_int = 2 * (time.perf_counter() - t0) / nsub
    out.append(dict(t_reg=t_reg, t_node=t_node, t_int=t_int))
print(json.dumps(dict(reps=out, t_table=t_tab)))
"""


def run_oracle_sample(nsub, nodes, reps, cores=None):
    """Time the oracle on `cores` host cores (default: all): one worker process
    per core, each a single thread running its share of the sample, all timed
    while running together.  Returns per-repetition step times extrapolated to
    the full step divided over the cores."""
    cores = cores or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ORACLE_SAMPLE.format(root=ROOT)
    ns, nn = max(1000, nsub // cores), max(1, nodes // cores)
    procs = [subprocess.Popen([sys.executable, "-c", code, str(ns), str(nn), str(reps), str(i)], stdin=subprocess.PIPE,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env) for i in range(cores)]
    for p in procs:
        if p.stdout.readline().strip() != "ready":
            raise RuntimeError("oracle worker failed: " + p.stderr.read()[-2000:])
    for p in procs:
        p.stdin.write("go\n")
        p.stdin.flush()
    res = []
    for p in procs:
        o, e = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError("oracle worker failed: " + e[-2000:])
        res.append(json.loads(o.strip().splitlines()[-1]))
    nv, M = 1_000_000, 1026 * 1026
    steps = []
    for r in range(reps):
        t_reg = statistics.mean(w["reps"][r]["t_reg"] for w in res)
        t_node = statistics.mean(w["reps"][r]["t_node"] for w in res)
        t_int = statistics.mean(w["reps"][r]["t_int"] for w in res)
        steps.append((t_reg * nv + t_node * M + t_int * nv) / cores)
    return {"steps": steps, "cores": cores, "nsub": ns, "nodes": nn, "t_table": res[0]["t_table"]}


def oracle_line_fields(res):
    mean = statistics.mean(res["steps"])
    sample = ("per step and core: R_v of %d random vortices, the direct-sum L^-1 at %d random nodes, E_v (u and v) of "
              "the same vortices, each worker a single thread, %d workers running together; per-unit times "
              "extrapolated to 1e6 vortices and all 1026^2 nodes the step needs (O(M^2) direct sum) and divided "
              "over the %d cores; LGF table by quadrature excluded (%.2f s, once per grid)") % (
                  res["nsub"], res["nodes"], res["cores"], res["cores"], res["t_table"])
    return mean, sample


# ------------------------------------------------------------------ clocks
class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (ctypes, the driver's
    libnvidia-ml) every millisecond in a thread, so that even a timed loop of a
    few milliseconds has its own record.  Reading only; nothing is set."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes
        import threading
        self.ok = False
        self.samples, self.reasons, self.maxmhz = [], 0, 0
        self._stop = threading.Event()
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            if self.lib.nvmlDeviceGetMaxClockInfo(self.h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
                self.maxmhz = mx.value
            self.reason_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.ok = True
        except Exception:
            self.ok = False

    def _run(self):
        import ctypes
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, ctypes.c_int(1), ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if self.reason_fn(self.h, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value
            time.sleep(0.001)

    def start(self):
        import threading
        if self.ok:
            self.th = threading.Thread(target=self._run, daemon=True)
            self.th.start()

    def stop(self):
        if not self.ok:
            return None
        self._stop.set()
        self.th.join()
        if not self.samples:
            return None
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.maxmhz,
                "reasons": sorted(v for k, v in self.REASONS.items() if self.reasons & k),
                "samples": len(self.samples), "source": "nvml, 1 ms"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index
        self.nvml = NvmlSampler(index)

    def start(self):
        self.nvml.start()
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=None):
        gpu_index = self.index if gpu_index is None else gpu_index
        nv = self.nvml.stop()
        smi = None
        if self.proc is not None:
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
                    if int(parts[0]) != gpu_index:
                        continue
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
            if sm:
                smi = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                       "samples": len(sm), "source": "nvidia-smi, 50 ms"}
        return nv or smi


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(vis) if vis.isdigit() else local


def kernel_bytes(name, nx, ny, nv, esz):
    """Algorithmic bytes of a launch in the step model (36 B/vortex + 28 B/node
    for the FP32 path): R_v reads a 16-byte cell record per vortex and writes w;
    the three FFT passes read w and the kernel spectrum quadrant and write the
    node velocity; E_v reads 12 bytes of position per vortex and the node
    velocity and writes (u, v).  Binning, record copies and FFT intermediates
    are implementation traffic (None here; reported from ncu)."""
    M = nx * ny
    return {
        "regularize": 16 * nv + esz * M,
        "fft_rows_fwd": esz * M,
        "fft_cols_conv": esz * M,
        "fft_rows_inv": 2 * esz * M,
        "interpolate": 12 * nv + 2 * esz * nv + 2 * esz * M,
        "vic_advect": 12 * nv + 2 * esz * nv + 2 * esz * M,
    }.get(name)


def step_traffic():
    """Per-step DRAM bytes of the step kernels from the committed ncu summary,
    if it was taken from the current sources."""
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(tpath):
        return None
    tj = json.load(open(tpath))
    if tj.get("csrc_sha") != csrc_sha():
        return None
    return tj


# the sources the body-free step's kernels and their launches are built from
STEP_SOURCES = ("common.cuh", "transfer.cuh", "transfer.cu", "fft.cu", "fft.cuh", "fft_reg.cuh", "dfloat.cuh",
                "lgf.cu", "api.cu", "tune.cu")


def csrc_sha():
    """Short hash of the step kernels' CUDA sources (ties an ncu record to the
    build it measured)."""
    import hashlib
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(ROOT, "paper_2102_11910_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def time_events(step, K, stream, flush):
    """K steps bracketed by CUDA events on `stream`, L2 flushed before each
    (outside the events); returns the per-step times in ms."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(k & 255)
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]


def kernel_table(rep, nsteps, g, nv, esz, hbm_peak):
    """Per-kernel event times of the timing pass with each kernel's algorithmic
    bytes (scope model) and the bandwidth they represent."""
    kern = {}
    total = sum(v[1] for v in rep.values())
    for name, (n, ms) in rep.items():
        b = kernel_bytes(name, g.nx, g.ny, nv, esz)
        avg = ms / n
        kern[name] = {"launches_per_step": n / nsteps, "avg_ms": avg, "share": ms / total, "alg_bytes": b,
                      "gbs": (b / (avg / 1e3) / 1e9) if b else None,
                      "frac": (b / (avg / 1e3) / 1e9 / hbm_peak) if b else None}
    return kern


# FP32 FMA lanes: 152 SMs x 128 lanes x 2 flops at the 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def fft_flop_roofline(kern, nx, ny, P, Q):
    """The three FFT passes of the velocity solve against the FP32 ALU peak,
    with the radix-2 count 5 n log2 n flops per complex transform of length n:
    ny/2 forward row transforms (two real rows each) of length P, P/2 + 1
    columns of one forward and two inverse length-Q transforms plus the two
    spectral products, ny inverse row transforms (u + i v) of length P."""
    names = ("fft_rows_fwd", "fft_cols_conv", "fft_rows_inv")
    if not all(n in kern for n in names):
        return None
    lp, lq = math.log2(P), math.log2(Q)
    flops = (ny / 2) * 5 * P * lp + (P / 2 + 1) * (3 * 5 * Q * lq + 2 * 6 * Q) + ny * 5 * P * lp
    us = 1e3 * sum(kern[n]["avg_ms"] for n in names)
    achieved = flops / (us * 1e-6) / 1e12
    return {"bound": "alu", "flops": flops, "us": us, "achieved": achieved, "unit": "TFLOP/s",
            "peak": FP32_PEAK_TFLOPS, "frac": achieved / FP32_PEAK_TFLOPS,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.070 GHz"}


def roofline_of(kern, hbm_peak, peak_note, traffic_rec):
    """The dominant kernel (most time among those with algorithmic bytes)."""
    dom = max((k for k in kern if kern[k]["gbs"]), key=lambda k: kern[k]["avg_ms"] * kern[k]["launches_per_step"])
    traffic = None
    if traffic_rec and dom in traffic_rec.get("kernels", {}):
        traffic = traffic_rec["kernels"][dom].get("dram_bytes")
    return {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": kern[dom]["gbs"] / hbm_peak, "traffic": traffic, "peak_source": peak_note,
            "alg_bytes_per_launch": kern[dom]["alg_bytes"]}


# ------------------------------------------------------------------ our arm
def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2102_11910_gb300 as pf
    from paper_2102_11910_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    wl = inputs.vic_1024()
    g = wl["grid"]
    X, Y, G = (torch.from_numpy(a).cuda() for a in (wl["X"], wl["Y"], wl["G"]))
    nv = X.numel()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=stream)
        # launch configuration picked by the library's autotuner for this grid
        # and vortex count (before the warm-up; not part of any timed step)
        t0 = time.perf_counter()
        tuned_cfg, tuned_us = pf.pf_autotune(plan, nv, None, reps=15)
        tune_s = time.perf_counter() - t0
        uq = torch.empty(nv, dtype=torch.float32, device="cuda")
        vq = torch.empty(nv, dtype=torch.float32, device="cuda")

        def step():
            pf.pf_vic_velocity(plan, X, Y, G, 0.0, 0.0, uq, vq)

        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        pf.pf_sync(plan)
        K = args.steps
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        clk = ClockSampler(gpu_index(local))
        clk.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for k in range(K):
            flush.fill_(k & 255)
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        if world > 1:
            dist.barrier()
        clocks = clk.stop()
        pf.pf_sync(plan)
        per = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        total_ms = max_over_ranks(sum(per), world)
        value = world * K / (total_ms / 1e3)
        ms_per_step = total_ms / K
        srt = sorted(per)
        p50 = srt[len(srt) // 2]
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]

        # per-kernel CUDA-event timing pass (same stream, same flushes)
        KT = min(K, 200)
        pf.pf_timing_enable(plan, True)
        for k in range(KT):
            flush.fill_(k & 255)
            step()
        rep = pf.pf_timing_report(plan)
        pf.pf_timing_enable(plan, False)
        launches_per_step = sum(n for n, _ in rep.values()) / KT
    # kernel roofline
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_note = "measured" if peaks else "fallback"
    kern = kernel_table(rep, KT, g, nv, 4, hbm_peak)
    traffic_rec = step_traffic()
    roof = roofline_of(kern, hbm_peak, peak_note, traffic_rec)
    step_bytes = 36 * nv + 28 * g.nx * g.ny
    step_roof = {"alg_bytes": step_bytes, "model": "36 B/vortex + 28 B/node (FP32)",
                 "achieved_gbs": step_bytes / (ms_per_step / 1e3) / 1e9,
                 "frac": step_bytes / (ms_per_step / 1e3) / 1e9 / hbm_peak, "peak": hbm_peak,
                 "dram_bytes_measured": (traffic_rec or {}).get("step_dram_bytes", {}).get("pf_vic_velocity")}
    fft_roof = fft_flop_roofline(kern, g.nx, g.ny, plan.P, plan.Q)

    # the same workload as a tile-ordered vortex state, stepped in time (forward
    # Euler): deposit, node velocity, E_v with the move, incremental re-bin
    with torch.cuda.stream(stream):
        vstate = pf.VicState(plan, nv)
        pf.pf_vic_state_set(vstate, X, Y, G)
        umax = float(torch.sqrt(uq.double() ** 2 + vq.double() ** 2).max())
        dt = 0.25 * g.dx / max(umax, 1e-30)       # a quarter cell per step at the fastest vortex

        def vstep():
            pf.pf_vic_step(vstate, dt, 0.0, 0.0)
        for _ in range(args.warmup):
            flush.fill_(1)
            vstep()
        pf.pf_sync(plan)
        KV = min(K, 400)
        per_v = time_events(vstep, KV, stream, flush)
        pf.pf_sync(plan)
        pf.pf_timing_enable(plan, True)
        for k in range(min(KV, 100)):
            flush.fill_(k & 255)
            vstep()
        rep_v = pf.pf_timing_report(plan)
        pf.pf_timing_enable(plan, False)
        _, _, _, nv_left, _ = pf.pf_vic_state_get(vstate)
        vstate.close()
    ms_v = max_over_ranks(sum(per_v), world) / KV
    kern_v = kernel_table(rep_v, min(KV, 100), g, nv, 4, hbm_peak)
    vic_state = {"value": world / (ms_v / 1e3), "unit": UNIT, "ms_per_step": ms_v, "steps": KV,
                 "dt": dt, "vortices_after": nv_left,
                 "step_roofline": {"alg_bytes": step_bytes, "achieved_gbs": step_bytes / (ms_v / 1e3) / 1e9,
                                   "frac": step_bytes / (ms_v / 1e3) / 1e9 / hbm_peak},
                 "roofline": roofline_of(kern_v, hbm_peak, peak_note, traffic_rec), "kernels": kern_v,
                 "desc": "same 1e6 vortices as a tile-ordered pf_vic_state: one forward-Euler time step per "
                         "call (R_v from the binned records, spectral node velocity, E_v with the move, "
                         "incremental re-bin), dt = a quarter cell at the fastest vortex, L2 flushed between steps"}

    # end to end through the host-buffer entry points (page-locked host memory),
    # every step copying its inputs in and its velocities out:
    #  - synchronous: one pf_vic_velocity_host call per step;
    #  - pipelined (the reported value): pf_vic_velocity_host_async on a ring of
    #    four plans, so that the copies of one step overlap the kernels of
    #    others; a plan is synchronised before it takes its next step (three
    #    plans: 6.9e3 steps/s, four: 7.26e3, five: 7.3e3 on a GB300).
    import torch as _t
    hX, hY, hG = (_t.from_numpy(a).pin_memory() for a in (wl["X"], wl["Y"], wl["G"]))
    NPIPE = 4
    hout = [(_t.empty(nv, dtype=_t.float32).pin_memory(), _t.empty(nv, dtype=_t.float32).pin_memory())
            for _ in range(NPIPE)]
    KE = max(3, min(K, 100))
    with _t.cuda.stream(stream):
        pf.pf_vic_velocity_host(plan, hX, hY, hG, 0.0, 0.0, *hout[0])
        lat_e = []
        t0 = time.perf_counter()
        for _ in range(KE):
            t1 = time.perf_counter()
            pf.pf_vic_velocity_host(plan, hX, hY, hG, 0.0, 0.0, *hout[0])
            lat_e.append(time.perf_counter() - t1)
        te = time.perf_counter() - t0
    lat_e.sort()
    plans = [plan]
    for _ in range(NPIPE - 1):
        sk = torch.cuda.Stream()
        with torch.cuda.stream(sk):
            plans.append(pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=sk))
            pf.pf_launch_config_set(plans[-1], **tuned_cfg)
    for k in range(NPIPE):
        pf.pf_vic_velocity_host_async(plans[k], hX, hY, hG, 0.0, 0.0, *hout[k])
    for pl in plans:
        pf.pf_sync(pl)
    KP = max(3 * NPIPE, min(2 * K, 60))
    t0 = time.perf_counter()
    for k in range(KP):
        pl = plans[k % NPIPE]
        if k >= NPIPE:
            pf.pf_sync(pl)          # its step k - NPIPE has finished: outputs complete
        pf.pf_vic_velocity_host_async(pl, hX, hY, hG, 0.0, 0.0, *hout[k % NPIPE])
    for pl in plans:
        pf.pf_sync(pl)
    tp = time.perf_counter() - t0
    te, tp = max_over_ranks(te, world), max_over_ranks(tp, world)
    e2e = {"value": world * KP / tp, "unit": UNIT, "h2d_bytes_per_step": 24 * nv, "d2h_bytes_per_step": 8 * nv,
           "mode": "pf_vic_velocity_host_async on a ring of %d plans (pipelined), %d steps" % (NPIPE, KP),
           "sync_value": world * KE / te, "sync_mode": "pf_vic_velocity_host, one synchronous call per step",
           "sync_latency_ms": {"p50": 1e3 * lat_e[len(lat_e) // 2],
                               "p99": 1e3 * lat_e[min(len(lat_e) - 1, int(math.ceil(0.99 * len(lat_e))) - 1)],
                               "calls": KE, "what": "host wall time of one call: inputs in, the step, velocities "
                                                   "out, synchronised"}}

    extras = {}
    if not args.no_extras:
        # impulse diagnostics (Sec. 2.6.2) of the step's vorticity: node reduction time
        with torch.cuda.stream(stream):
            w = pf.pf_regularize(plan, X, Y, G)
            pf.pf_impulse(plan, w)
            pf.pf_timing_enable(plan, True)
            for _ in range(20):
                flush.fill_(3)
                pf.pf_impulse(plan, w)
            rimp = pf.pf_timing_report(plan)
            pf.pf_timing_enable(plan, False)
        n_i, ms_i = rimp["impulse"]
        us_i = 1e3 * ms_i / n_i
        gbs_i = g.nx * g.ny * 4 / (us_i * 1e-6) / 1e9
        extras["impulse"] = {"kernel_us": us_i, "alg_bytes": g.nx * g.ny * 4, "gbs": gbs_i, "frac": gbs_i / hbm_peak,
                             "final_us": 1e3 * rimp["impulse_final"][1] / rimp["impulse_final"][0],
                             "value": [float(v) for v in pf.pf_impulse(plan, w)]}
        # all-FP64 GPU path on the same workload, and the mixed path's error against it
        with torch.cuda.stream(stream):
            p64 = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_FP64, stream=stream)
            u64 = torch.empty(nv, dtype=torch.float64, device="cuda")
            v64 = torch.empty(nv, dtype=torch.float64, device="cuda")
            pf.pf_vic_velocity(p64, X, Y, G, 0.0, 0.0, u64, v64)
            pf.pf_sync(p64)
            K64 = max(3, min(K, 20))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(K64):
                pf.pf_vic_velocity(p64, X, Y, G, 0.0, 0.0, u64, v64)
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1) / K64
            pf.pf_vic_velocity(plan, X, Y, G, 0.0, 0.0, uq, vq)
            pf.pf_sync(plan)
            num = torch.sqrt(torch.sum((uq.double() - u64) ** 2) + torch.sum((vq.double() - v64) ** 2))
            den = torch.sqrt(torch.sum(u64 ** 2) + torch.sum(v64 ** 2))
            extras["fp64_path"] = {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64}
            extras["mixed_rel_err_vs_fp64_gpu"] = float(num / den)
            p64.close()
        # the FFT convolution next to cuFFT (torch.fft; a timed comparison, not a product path):
        # the same zero-padded P x Q real-to-complex transform of w, products with two spectra
        # (u and v) and two complex-to-real inverses, FP32, L2 flushed between repetitions
        with torch.cuda.stream(stream):
            Pp, Qp = plan.P, plan.Q
            gen = torch.Generator(device="cuda").manual_seed(5)
            wpad = torch.zeros((Qp, Pp), dtype=torch.float32, device="cuda")
            wpad[:g.ny, :g.nx] = torch.randn(g.ny, g.nx, device="cuda", generator=gen)
            H1 = torch.randn(Qp, Pp // 2 + 1, dtype=torch.complex64, device="cuda", generator=gen)
            H2 = torch.randn(Qp, Pp // 2 + 1, dtype=torch.complex64, device="cuda", generator=gen)

            def cufft_conv():
                Wh = torch.fft.rfft2(wpad)
                return (torch.fft.irfft2(Wh * H1, s=(Qp, Pp))[:g.ny, :g.nx],
                        torch.fft.irfft2(Wh * H2, s=(Qp, Pp))[:g.ny, :g.nx])
            for _ in range(3):
                cufft_conv()
            tot = 0.0
            for k in range(20):
                flush.fill_(k & 255)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cufft_conv()
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            ours = sum(1e3 * kern[k]["avg_ms"] for k in ("fft_rows_fwd", "fft_cols_conv", "fft_rows_inv") if k in kern)
            extras["fft_vs_cufft"] = {"ours_us": ours, "cufft_us": 1e3 * tot / 20, "grid": [Pp, Qp],
                                      "desc": "u and v of the padded convolution: our three fused passes (sum of "
                                              "their per-kernel event averages) against torch.fft rfft2, two "
                                              "spectral products and two irfft2 (cuFFT)"}
            del wpad, H1, H2
        if world == 1:
            try:
                extras["workloads"] = bench_workloads(pf, inputs, torch, stream)
            except Exception as e:          # reported, never fatal for the main line
                extras["workloads"] = {"error": "%s: %s" % (type(e).__name__, e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        res = run_oracle_sample(nsub=400000, nodes=1200, reps=1)
        mean, sample = oracle_line_fields(res)
        cpu = {"value": 1.0 / mean, "unit": UNIT, "cores": res["cores"], "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed (FP32 grid path, FP64 positions and LGF setup)",
                       "l2": "flushed between timed steps (256 MB write, outside the timed events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch_config": dict(tuned_cfg, source="pf_autotune (%.2f s, best %.1f us on its synthetic "
                                             "vortices, L2 flushed before each timed call)" % (tune_s, tuned_us))},
            "latency_ms": {"p50": p50, "p99": p99},
            "roofline": roof, "step_roofline": step_roof, "fft_flop_roofline": fft_roof,
            "kernels": kern, "gpu_launches": int(round(launches_per_step * K)),
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "wall_s_timed_loop": t_wall,
            "vic_state_step": vic_state,
        }
        line.update(extras)
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ other workloads
def _steps_per_s(pf, plan, fn, n):
    pf.pf_sync(plan)
    t0 = time.perf_counter()
    for _ in range(n):
        fn()
    pf.pf_sync(plan)
    return n / (time.perf_counter() - t0)


def bench_workloads(pf, inputs, torch, stream, n_batch=256, n_requests=256):
    """Body workloads: single-step plate, pitching plate, uneven batch, request server."""
    import numpy as np
    out = {}
    with torch.cuda.stream(stream):
        # plate, 128^2, 64 points, 256 vortices, Euler with two-edge release
        wl = inputs.plate_vortices_128()
        g = wl["grid"]
        res = {}
        for prec, name in ((pf.PF_MIXED, "mixed"), (pf.PF_FP64, "fp64")):
            plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec, stream=stream)
            state = pf.State(plan, 256 + 2 * 64)
            pf.pf_state_set(state, wl["X"], wl["Y"], wl["G"])
            body = pf.plate_kinematics(64, 1.0, wl["alpha"], Uinf=1.0)
            pf.pf_step(plan, state, 0.002, body)             # includes the one-off factorisation
            res[name] = _steps_per_s(pf, plan, lambda: pf.pf_step(plan, state, 0.002, body), 20)
            # the same step captured once and replayed as a graph (pf_batch of one)
            gs = torch.cuda.Stream()
            gplan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec, stream=gs)
            gstate = pf.State(gplan, 256 + 2 * 64)
            pf.pf_state_set(gstate, wl["X"], wl["Y"], wl["G"])
            batch = pf.Batch([gplan], [gstate], [body], [0.002])
            batch.step(1)
            res[name + "_graph"] = _steps_per_s(pf, gplan, lambda: batch.step(1), 20)
            batch.close()
        # the same with the generalized edge condition at the leading edge (Sec. 2.5)
        plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=stream)
        state = pf.State(plan, 256 + 2 * 64)
        pf.pf_state_set(state, wl["X"], wl["Y"], wl["G"])
        xi = -1.0 + (2.0 * np.arange(1, 65) - 1.0) / 64
        body = pf.BodyKinematics(0.5 * xi, np.zeros(64), np.full(64, 1.0 / 64), (0, 63), wl["alpha"], Uinf=1.0,
                                 edge_bounds=((-0.5, 0.5), (0.0, 0.0)))
        pf.pf_step(plan, state, 0.002, body)
        res["mixed_edge_bounded"] = _steps_per_s(pf, plan, lambda: pf.pf_step(plan, state, 0.002, body), 20)
        out["plate_128"] = {"unit": "steps/s", "desc": "128^2, plate 20 deg, Ns 64, 256 vortices, Euler, dt 0.002, "
                            "two-edge release every step (factor reused), one pf_step per step or (_graph) one "
                            "launch of the captured step; edge_bounded: leading edge under |ftilde| <= 0.5 "
                            "(generalized edge condition), trailing edge Kutta", **res}
        print("workload done: %s" % 'plate_128', file=sys.stderr, flush=True)
        # pitching plate, 768 x 512, RK2, S refactored at every stage.  With the
        # configured Ns = 256 (dS/dx = 0.39, below the paper's 1-4) the released
        # strengths diverge and vortices leave the grid after ~20-50 steps (the
        # FP64 oracle too, at the same dS/dx on a smaller grid): timed over its
        # first 16 steps.  The 2000-step run, wake growing to 4000 vortices, uses
        # Ns = 64 (dS/dx = 1.56) and is timed whole.
        pw = inputs.pitching_plate_512x768()
        g = pw["grid"]
        omega = 2.0 * pw["k"] * pw["Uinf"] / pw["chord"]
        res = {}
        for ns, nsteps, name in ((pw["ns"], 16, "ns256_first_16_steps"), (64, 2000, "ns64_2000_steps")):
            plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=stream)
            state = pf.State(plan, 2 * nsteps + 64)
            pf.pf_state_set(state, np.zeros(0), np.zeros(0), np.zeros(0))
            body = pf.plate_kinematics(ns, pw["chord"], pw["alpha0"], pw["amp"], omega, pw["Uinf"])
            res[name] = _steps_per_s(pf, plan, lambda: pf.pf_step(plan, state, pw["dt"], body, scheme=1), nsteps)
            _, _, G, _ = pf.pf_state_get(state)
            res[name + "_vortices"] = len(G)
            res[name + "_max_abs_gamma"] = float(np.abs(G).max())
            state.close()
            plan.close()
        out["pitching_plate_768x512"] = {"unit": "steps/s", "desc": "768x512, dx 0.01, 30+10 sin(t) deg, k 0.5, "
                                         "RK2, dt 0.0025, two releases per step, mixed; Ns 256 (dS/dx 0.39) diverges "
                                         "after ~20 steps, so its first 16 are timed; Ns 64 (dS/dx 1.56) runs the "
                                         "configured 2000 steps (0 -> 4000 vortices), timed whole", **res}
        # two plates (Sec. 2.7, as the paper's two-plate example): chord 1 at 60 deg, c/2 apart
        # vertically, dx = c/100, dS/dx = 2 (50 points each), dt U/c = 0.01, four releases per step
        gtp = inputs.GridSpec(384, 256, 0.01, -1.0, -0.5 * 255 * 0.01)
        plan = pf.Plan(gtp.nx, gtp.ny, gtp.dx, gtp.x0, gtp.y0, pf.PF_MIXED, stream=stream)
        state = pf.State(plan, 4 * 40)
        pf.pf_state_set(state, np.zeros(0), np.zeros(0), np.zeros(0))
        tp = [inputs.plate(50, 1.0, math.radians(60.0), 0.0, yc) for yc in (0.25, -0.25)]
        tpk = [pf.BodyKinematics(b.x, b.y, b.ds, b.edges, 0.0, Uinf=1.0) for b in tp]
        for _ in range(5):
            pf.pf_step_multi(plan, state, 0.01, tpk)
        out["two_plates_384x256"] = {"unit": "steps/s", "desc": "two plates, chord 1 at 60 deg, c/2 apart, 384x256, "
                                     "dx 0.01, Ns 2x50, Euler, dt 0.01, four vortices released per step "
                                     "(Kutta at every edge, Kelvin per body; factor reused)",
                                     "mixed": _steps_per_s(pf, plan, lambda: pf.pf_step_multi(plan, state, 0.01, tpk),
                                                           20)}
        print("workload done: %s" % 'two_plates_384x256', file=sys.stderr, flush=True)
        # surface pressure (Sec. 2.6.1) of the 128^2 plate at dS/dx = 1: the jump operator's setup
        # once, then per step the potential jump of the sheet and the pressure jump
        gsp = inputs.centred_grid(128, 128, 0.02)
        plan = pf.Plan(gsp.nx, gsp.ny, gsp.dx, gsp.x0, gsp.y0, pf.PF_MIXED, stream=stream)
        pb = inputs.plate(50, 1.0, math.radians(20.0))
        schur = pf.pf_schur_factor(plan, pb.x, pb.y, pb.ds)
        t0 = time.perf_counter()
        pf.pf_pressure_setup(plan, schur, np.full(50, math.sin(math.radians(20.0))),
                             np.full(50, math.cos(math.radians(20.0))))
        setup_ms = 1e3 * (time.perf_counter() - t0)
        wsp = plan.field()
        wsp.zero_()
        fsp, _, _ = pf.pf_sheet_solve(plan, schur, wsp, (0.0, 0.0, 0.0, 1.0, 0.0), pf.PF_SHEET_KUTTA_STEADY, 0.0,
                                      [pb.edges[1]])
        pf.pf_sheet_regularize(plan, schur, fsp, wsp)
        psi_sp = pf.pf_poisson_solve(plan, wsp)
        prev = pf.pf_potential_jump(plan, schur, fsp)

        def pressure_step():
            d = pf.pf_potential_jump(plan, schur, fsp)
            dd = (d - prev) / 0.01
            pf.pf_pressure_field(plan, psi_sp, wsp, (0.0, 0.0, 0.0, 1.0, 0.0), schur, fsp, dd)
            return pf.pf_pressure_jump(plan, schur, psi_sp, (0.0, 0.0, 0.0, 1.0, 0.0), fsp, dd)
        for _ in range(3):
            pressure_step()
        out["pressure_plate_128"] = {"unit": "calls/s", "setup_ms": setup_ms,
                                     "desc": "plate 128^2, Ns 50 (dS/dx 1): potential jump, cell-centre pressure "
                                             "field and surface pressure jump per call (steady Kutta sheet, psi of "
                                             "the sheet); setup = jump operator build and inverse, once per "
                                             "geometry",
                                     "mixed": _steps_per_s(pf, plan, pressure_step, 50)}
        print("workload done: %s" % 'pressure_plate_128', file=sys.stderr, flush=True)
        out["uneven_batch"] = bench_uneven_batch(pf, inputs, torch, stream, n_batch)
        print("workload done: %s" % 'uneven_batch', file=sys.stderr, flush=True)
    out["serving"] = bench_serving(pf, inputs, n_requests, (0.3, 0.7, 1.0))
    return out


def bench_body_profile(pf, inputs, torch, which, K, W):
    """CUDA-event shares of the body step's phases (Schur factor, R_v with the
    circulation sum, sheet solve with release, velocity = R_v + sheet
    deposit + L^-1 + E_v, position update) and of the kernels timed inside
    them, for the 128^2 plate (Euler, factor reused) and the 768x512 pitching
    plate (Ns 64, RK2, refactored at every stage) and the 1024^2 plate with
    1e5 vortices of the served mix (Ns 256, Euler).  W steps untimed, then K
    steps each bracketed by events on the plan stream."""
    import numpy as np
    stream = torch.cuda.Stream()
    out = {}
    cases = []
    if which in ("all", "plate"):
        wl = inputs.plate_vortices_128()
        g = wl["grid"]
        # the free stream carries the outer vortices off the 128^2 grid after ~40
        # steps: the state is reloaded every 20 steps (outside the events)
        cases.append(("plate_128", g, wl["X"], wl["Y"], wl["G"], pf.plate_kinematics(64, 1.0, wl["alpha"], Uinf=1.0),
                      0.002, 0, 256 + 2 * 21, 20))
    if which in ("all", "pitching"):
        pw = inputs.pitching_plate_512x768()
        g = pw["grid"]
        omega = 2.0 * pw["k"] * pw["Uinf"] / pw["chord"]
        cases.append(("pitching_plate_768x512_ns64", g, np.zeros(0), np.zeros(0), np.zeros(0),
                      pf.plate_kinematics(64, pw["chord"], pw["alpha0"], pw["amp"], omega, pw["Uinf"]), pw["dt"], 1,
                      2 * (K + W + 1), None))
    if which in ("all", "big"):
        bw = inputs.plate_vortices_1024()
        b = bw["body"]
        cases.append(("plate_1024_1e5", bw["grid"], bw["X"], bw["Y"], bw["G"],
                      pf.BodyKinematics(b["xb"], b["yb"], b["ds"], b["edges"], b["alpha0"], Uinf=bw["Uinf"]),
                      bw["dt"], 0, len(bw["X"]) + 2 * (K + W + 1), None))
    with torch.cuda.stream(stream):
        for name, g, X, Y, G, body, dt, scheme, cap, reload in cases:
            plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=stream)
            state = pf.State(plan, cap)
            pf.pf_state_set(state, X, Y, G)
            for _ in range(W):
                pf.pf_step(plan, state, dt, body, scheme=scheme)
            pf.pf_sync(plan)
            pf.pf_timing_enable(plan, True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for k, (a, b) in enumerate(ev):
                if reload and k % reload == 0:
                    pf.pf_state_set(state, X, Y, G)
                a.record(stream)
                pf.pf_step(plan, state, dt, body, scheme=scheme)
                b.record(stream)
            pf.pf_sync(plan)
            rep = pf.pf_timing_report(plan)
            pf.pf_timing_enable(plan, False)
            step_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
            phases = {k: v for k, v in rep.items() if k.startswith("phase_")}
            tot = sum(v[1] for v in phases.values())
            _, _, Gs, _ = pf.pf_state_get(state)
            out[name] = {
                "steps": K, "warmup": W, "scheme": "RK2" if scheme else "Euler", "vortices_at_end": len(Gs),
                "step_ms": step_ms, "phase_ms_per_step": {k: v[1] / K for k, v in phases.items()},
                "phase_share": {k: v[1] / tot for k, v in phases.items()},
                "phase_sum_over_step": tot / K / step_ms,
                "kernels_ms_per_step": {k: v[1] / K for k, v in rep.items() if not k.startswith("phase_")},
                "kernel_launches_per_step": {k: v[0] / K for k, v in rep.items() if not k.startswith("phase_")},
            }
            state.close()
            plan.close()
    return out


def bench_uneven_batch(pf, inputs, torch, stream, n_batch=256):
    """The uneven batch (256 independent instances), one step each per call."""
    with torch.cuda.stream(stream):
        # uneven batch: independent instances, one step each per call, in the
        # same precision three ways: one CUDA graph of every instance's step
        # (pf_batch), one stream per instance enqueued per call (pf_step_batch),
        # and one instance at a time (pf_step, synchronised)
        inst = inputs.batched_instances(n=n_batch)
        dts = [r["dt"] for r in inst]
        res = {}
        for prec, pname in ((pf.PF_MIXED, "mixed"), (pf.PF_FP64, "fp64")):
            for mode in ("graph", "streams", "unbatched"):
                bases, plans, states, bodies = {}, [], [], []
                for r in inst:
                    gg = r["grid"]
                    key = (gg.nx, gg.ny)
                    if key not in bases:
                        bases[key] = pf.Plan(gg.nx, gg.ny, gg.dx, gg.x0, gg.y0, prec, stream=stream)
                    p = pf.pf_plan_clone(bases[key], prec, torch.cuda.Stream())
                    st = pf.State(p, len(r["X"]) + 64)
                    pf.pf_state_set(st, r["X"], r["Y"], r["G"])
                    b = r["body"]
                    plans.append(p)
                    states.append(st)
                    bodies.append(pf.BodyKinematics(b["xb"], b["yb"], b["ds"], b["edges"], b["alpha0"],
                                                    Uinf=r["Uinf"]))
                torch.cuda.synchronize()
                if mode == "graph":
                    t0 = time.perf_counter()
                    batch = pf.Batch(plans, states, bodies, dts)       # factorisations and the capture
                    torch.cuda.synchronize()
                    res["graph_create_s_" + pname] = time.perf_counter() - t0
                    batch.step(1)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(3):
                        batch.step(1)
                    torch.cuda.synchronize()
                    res["graph_" + pname] = 3 * len(inst) / (time.perf_counter() - t0)
                    batch.close()
                elif mode == "streams":
                    pf.pf_step_batch(plans, states, bodies, dts)          # factorisations
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(3):
                        pf.pf_step_batch(plans, states, bodies, dts)
                    torch.cuda.synchronize()
                    res["streams_" + pname] = 3 * len(inst) / (time.perf_counter() - t0)
                else:
                    for p, st, b, dt in zip(plans, states, bodies, dts):
                        pf.pf_step(p, st, dt, b)
                        pf.pf_sync(p)
                    t0 = time.perf_counter()
                    for p, st, b, dt in zip(plans, states, bodies, dts):
                        pf.pf_step(p, st, dt, b)
                        pf.pf_sync(p)
                    res["unbatched_" + pname] = len(inst) / (time.perf_counter() - t0)
                for p in plans:
                    pf.pf_sync(p)
                del plans, states, bases
        return {"unit": "instance-steps/s", "instances": len(inst),
                "desc": "grids 128^2..512^2, plate or ellipse, Ns 32-256, 100-20000 vortices "
                        "N(0,1e-3), a CFL step each; per precision: graph = one CUDA graph launch "
                        "steps every instance (pf_batch, captured once), streams = one stream per "
                        "instance enqueued every call (pf_step_batch), unbatched = one instance at "
                        "a time, synchronised", **res}


def bench_serving(pf, inputs, n_requests, fractions):
    """The request server under load: a burst (every request at time 0) gives the
    saturation throughput; then Poisson arrivals at the given fractions of it,
    with p50/p99 latency (submission to completion) at each rate."""
    import numpy as np
    reqs = inputs.serving_requests(n=n_requests)

    def run(rate):
        server = pf.Server(max_slots=32, hbm_budget_bytes=32 << 30, precision=pf.PF_MIXED)
        rng = np.random.default_rng(7)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs))) if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        pending, lats, i, steps, failed = set(), [], 0, 0, 0
        last_done = time.perf_counter()
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            if pending and time.perf_counter() - last_done > 120.0:
                q, a, u = pf.pf_server_stats(server)
                raise RuntimeError("serving stalled: no request finished for 120 s (queued %d, running %d, "
                                   "%d bytes resident)" % (q, a, u))
            while i < len(reqs) and arrivals[i] <= now:
                r = reqs[i]
                b = r["body"]
                body = pf.BodyKinematics(b["xb"], b["yb"], b["ds"], b["edges"], b["alpha0"], Uinf=r["Uinf"])
                gg = r["grid"]
                pending.add(pf.pf_server_submit(server, (gg.nx, gg.ny, gg.dx, gg.x0, gg.y0), r["X"], r["Y"], r["G"],
                                                r["nsteps"], r["dt"], body))
                steps += r["nsteps"]
                i += 1
            for t in pf.pf_server_progress(server):
                last_done = time.perf_counter()
                pending.discard(t)
                try:
                    lats.append(pf.pf_server_result(server, t, 200000)[3])
                except pf.GridPfError:
                    failed += 1
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        server.close()
        lats = sorted(lats) or [float("nan")]
        return {"requests": len(reqs), "failed": failed, "steps": steps, "wall_s": wall, "steps_per_s": steps / wall,
                "requests_per_s": len(reqs) / wall, "offered_requests_per_s": rate,
                "p50_ms": 1e3 * lats[len(lats) // 2], "p99_ms": 1e3 * lats[min(len(lats) - 1, int(0.99 * len(lats)))]}
    burst = run(None)
    out = {"desc": "%d requests: instances of the uneven batch (strengths N(0,1e-3), a CFL step each) plus 10%% at "
                   "1024^2 with 1e5 vortices, 1-50 steps each, mixed precision, 32 slots; burst = all at t=0 "
                   "(saturation), then Poisson arrivals at fractions of the burst throughput" % len(reqs),
           "burst": burst}
    for f in fractions:
        out["poisson_at_%gx" % f] = run(f * burst["requests_per_s"])
        print("serving rate %gx done" % f, file=sys.stderr, flush=True)
    return out


# ------------------------------------------------------------------ reference arm
def bench_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    # per-step sample sized so that K + W steps take about two minutes on the host cores
    cores = os.cpu_count() or 1
    per = 120.0 / max(1, K + W) * cores
    nodes = max(cores, int(per / 3 / 0.012))
    nsub = max(1000 * cores, min(200000 * cores, int(per / 3 / 1.5e-6)))
    res = run_oracle_sample(nsub=nsub, nodes=nodes, reps=K + W, cores=cores)
    res["steps"] = res["steps"][W:]
    mean, sample = oracle_line_fields(res)
    value = 1.0 / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 leg and the CPU baseline")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="only the request server: 4096 requests, Poisson arrivals from 0.1x to 1.2x of saturation")
    ap.add_argument("--body-profile", choices=["all", "plate", "pitching", "big"],
                    help="only the body steps' phase shares (CUDA events): --warmup steps untimed, --steps timed")
    ap.add_argument("--vic", type=int, nargs=2, metavar=("N", "NV"),
                    help="only the body-free step on N^2 nodes with NV vortices (the benchmark recipe scaled; "
                         "--warmup untimed, --steps timed), for profiling smaller cases")
    ap.add_argument("--serving", type=int, default=0, metavar="N",
                    help="only the request server: N requests at once (the burst), no Poisson rates")
    ap.add_argument("--uneven-batch", action="store_true",
                    help="only the uneven batch of 256 instances (graph, streams, unbatched; mixed and FP64)")
    args = ap.parse_args()
    if args.vic:
        import torch
        import paper_2102_11910_gb300 as pf
        from paper_2102_11910_gb300 import inputs
        torch.cuda.set_device(dist_env()[2])
        n, nvv = args.vic
        wl = inputs.vic_1024(nv=nvv, n=n)
        g = wl["grid"]
        stream = torch.cuda.Stream()
        X, Y, G = (torch.from_numpy(a).cuda() for a in (wl["X"], wl["Y"], wl["G"]))
        with torch.cuda.stream(stream):
            plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, stream=stream)
            uq = torch.empty(nvv, dtype=torch.float32, device="cuda")
            vq = torch.empty_like(uq)
            flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

            def step():
                pf.pf_vic_velocity(plan, X, Y, G, 0.0, 0.0, uq, vq)
            for _ in range(args.warmup):
                step()
            pf.pf_sync(plan)
            per = time_events(step, args.steps, stream, flush)
            pf.pf_sync(plan)
        print(json.dumps({"vic": {"n": n, "nv": nvv, "ms_per_step": statistics.mean(per), "steps": args.steps}}))
        return
    if args.serving:
        import torch
        import paper_2102_11910_gb300 as pf
        from paper_2102_11910_gb300 import inputs
        torch.cuda.set_device(dist_env()[2])
        print(json.dumps({"serving": bench_serving(pf, inputs, args.serving, ())}))
        return
    if args.uneven_batch:
        import torch
        import paper_2102_11910_gb300 as pf
        from paper_2102_11910_gb300 import inputs
        torch.cuda.set_device(dist_env()[2])
        print(json.dumps({"uneven_batch": bench_uneven_batch(pf, inputs, torch, torch.cuda.Stream())}))
        return
    if args.body_profile:
        import torch
        import paper_2102_11910_gb300 as pf
        from paper_2102_11910_gb300 import inputs
        torch.cuda.set_device(dist_env()[2])
        print(json.dumps({"body_profile": bench_body_profile(pf, inputs, torch, args.body_profile, args.steps,
                                                             args.warmup)}))
        return
    if args.serving_sweep:
        import torch
        import paper_2102_11910_gb300 as pf
        from paper_2102_11910_gb300 import inputs
        torch.cuda.set_device(dist_env()[2])
        res = bench_serving(pf, inputs, 4096, (0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.2))
        print(json.dumps({"serving_sweep": res}))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
