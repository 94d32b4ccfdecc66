#!/usr/bin/env python3
"""Throughput benchmark of the multilevel Chebyshev-Hutchinson engine on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat20_triangles|logdet64|estrada_rmat22]

One step is one pass of the whole hot path over one batch of synthetic input:

  rmat20_triangles (default): exact int64 triangle moments of an R-MAT graph
      (scale 20, edge factor 16, a=0.57, b=c=0.19, seed 0; symmetric, no
      self-loops or duplicates) for 1024 Rademacher probes in blocks of 128,
      plus the control-variate estimate.  Units: probe-matvecs (2 per probe).
  logdet64: multilevel log-det of the 64x64 Dirichlet Laplacian + 0.1 I,
      levels {8, 32, 128} with {256, 64, 16} probes, FP64.  Units: probe-matvecs
      with the doubling evaluation (3072 per step).
  estrada_rmat22: FP32 Chebyshev moments of the scale-22 R-MAT adjacency
      scaled to spectral radius <= 10 (interval [-10, 10]), 256 probes to
      degree 128.  Units: probe-matvecs (64 per probe).

Under torchrun every rank runs its own probes (disjoint probe ids): weak
scaling with no collective on the data path; the timing is the max over ranks.
`--impl reference` times the CPU oracle (the plain C/numpy restatement of the
method) on a bounded sample of the same workload on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def step_bytes(d, nnz, entry_bytes, sv, probe_matvecs, launches_per_step):
    """Average algorithmic bytes per launch of the fused recurrence step: the
    matrix once per launch (rowptr and entry_bytes per stored entry), and per
    live probe its row of V_k and V_{k-1} read and V_{k+1} written (sv bytes
    each).  Live probes summed over a step's launches are its probe-matvecs,
    since probes retire by degree and wide blocks run as several groups."""
    n = launches_per_step.get("cheb_step")
    if not n:
        return {}
    return {"cheb_step": nnz * entry_bytes + 8 * (d + 1) + 3 * d * sv * probe_matvecs / n}


class Triangles:
    name = "rmat20_triangles"
    unit = "probe-matvecs/s"
    dtype = "int64"
    NPROBES = 1024
    BLOCK = 128

    def __init__(self):
        from paper_2103_10516_gb300 import synth
        self.csr = synth.rmat_adjacency(20, 16, seed=0)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz

    def units(self):
        return 2 * self.NPROBES

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale 20, edge factor 16, a=0.57 b=c=0.19, seed 0",
                "d": self.d, "nnz": self.nnz, "probes": self.NPROBES, "block": self.BLOCK,
                "control_variates": True,
                "l2": "inputs larger than L2 (col 4*nnz = %.0f MB + rowptr %.0f MB + y 128 B/row = %.0f MB)"
                      % (4e-6 * self.nnz, 8e-6 * self.d, 128e-6 * self.d)}

    def kernel_bytes(self, launches_per_step):
        """Algorithmic bytes per launch (one 128-probe block) of each kernel:
        every array touched once, gathered rows assumed cached.  y of a row
        takes 128 B (degree <= 127, int8), 256 B (<= 32767, int16) or 512 B
        (int32).  Pass 1 reads rowptr, col and the sign bits and writes y;
        pass 2 reads the out-list pointers, columns (nnz/2), small-section
        lengths and slots, and y of every row with an edge once."""
        d, nnz = self.d, self.nnz
        deg = np.diff(self.csr.rowptr)
        ybytes = int(128 * np.sum((deg > 0) & (deg <= 127)) + 256 * np.sum((deg > 127) & (deg <= 32767))
                     + 512 * np.sum(deg > 32767))
        return {
            "tri_zbits": 16 * d,
            "tri_pass1": 8 * (d + 1) + 4 * nnz + 16 * d + ybytes,
            "tri_pass2": 8 * (d + 1) + 4 * (nnz // 2) + 8 * d + ybytes,
        }

    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    # from an ncu capture of this workload, per kernel; empty until the
    # current kernels have been captured
    TRAFFIC = {}

    # ours
    def setup(self, mlt, torch, rank):
        self.M = mlt.Matrix(self.csr)
        self.x = torch.empty((self.NPROBES, 3), dtype=torch.int64, device="cuda")
        self.base = rank * (1 << 24)

    def step(self, mlt, stream, i):
        return mlt.mlt_triangle_trace(self.M.handle, 0, self.base + (i % 4096) * self.NPROBES,
                                      self.NPROBES, self.BLOCK, True, self.x, stream)

    def e2e_setup(self, torch):
        self.h_rowptr = torch.from_numpy(self.csr.rowptr).pin_memory()
        self.h_col = torch.from_numpy(self.csr.col).pin_memory()
        self.h_x = torch.empty((self.NPROBES, 3), dtype=torch.int64).pin_memory()
        return (self.h_rowptr.numel() * 8 + self.h_col.numel() * 4, self.h_x.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h_rowptr, self.h_col, None,
                               stream=stream)
        try:
            mlt.mlt_triangle_trace(h, 0, self.base + i * self.NPROBES, self.NPROBES, self.BLOCK,
                                   True, self.h_x, stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        x = oracle.triangle_moments(self.csr, 0, offset, nprobes)
        oracle.triangle_estimate(x, self.nnz, True)
        return 2 * nprobes


class LogDet64:
    name = "logdet64"
    unit = "probe-matvecs/s"
    dtype = "f64"

    def __init__(self):
        from paper_2103_10516_gb300 import synth
        self.csr = synth.grid_laplacian_2d(64, shift=0.1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.levels, self.m = [8, 32, 128], [256, 64, 16]

    def units(self):
        return sum(mk * ((l + 1) // 2) for l, mk in zip(self.levels, self.m))

    def config(self):
        return {"workload": self.name, "matrix": "64x64 Dirichlet Laplacian + 0.1 I", "d": self.d,
                "nnz": self.nnz, "f": "log", "interval": [0.1, 8.1], "n": 128,
                "levels": self.levels, "m": self.m,
                "l2": "L2-resident working set (11 MB); flushed between steps by a 256 MB write"}

    def kernel_bytes(self, launches_per_step):
        return step_bytes(self.d, self.nnz, 12, 8, self.units(), launches_per_step)

    def setup(self, mlt, torch, rank):
        self.M = mlt.Matrix(self.csr)
        self.flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
        self.base = rank

    def step(self, mlt, stream, i):
        self.flush.fill_(float(i))
        return self.M.mlmc("log", 0.1, 8.1, 128, seed=self.base * 100003 + i, levels=self.levels,
                           m=self.m, stream=stream)

    def e2e_setup(self, torch):
        self.h_rowptr = torch.from_numpy(self.csr.rowptr).pin_memory()
        self.h_col = torch.from_numpy(self.csr.col).pin_memory()
        self.h_val = torch.from_numpy(self.csr.val).pin_memory()
        return (self.h_rowptr.numel() * 8 + self.h_col.numel() * 4 + self.h_val.numel() * 8,
                sum(self.m) * 129 * 8)

    def e2e_step(self, mlt, stream, i):
        from paper_2103_10516_gb300.mlt import Matrix  # noqa: F401
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h_rowptr, self.h_col, self.h_val,
                               stream=stream)
        try:
            P = mlt.mlt_mlmc_default_params()
            P.fn, P.a, P.b, P.n, P.seed = 0, 0.1, 8.1, 128, i
            P.nlevels = 3
            for k in range(3):
                P.levels[k] = self.levels[k]
                P.m[k] = self.m[k]
            P.stream = stream
            mlt.mlt_mlmc_estimate(h, P)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        deg = np.array(([8] * 16 + [32] * 4 + [128]) * max(1, nprobes // 21), dtype=np.int32)
        oracle.moments(self.csr, 0.1, 8.1, offset, 0, deg)
        return int(np.sum((deg + 1) // 2))


class EstradaRmat22:
    name = "estrada_rmat22"
    unit = "probe-matvecs/s"
    dtype = "f32"
    NPROBES = 256
    DEG = 128

    def __init__(self):
        from paper_2103_10516_gb300 import synth
        self.csr = synth.rmat_adjacency(22, 16, seed=1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.scale = None

    def units(self):
        return self.NPROBES * ((self.DEG + 1) // 2)

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale 22, edge factor 16, seed 1",
                "d": self.d, "nnz": self.nnz, "probes": self.NPROBES, "degree": self.DEG,
                "precision": "fp32 vectors, fp64 dots", "interval": [-10.0, 10.0],
                "group_width": getattr(self, "group_width", None),
                "l2": "inputs larger than L2 (V 2 x %.0f MB)" % (self.d * self.NPROBES * 4e-6)}

    def kernel_bytes(self, launches_per_step):
        return step_bytes(self.d, self.nnz, 4, 4, self.units(), launches_per_step)

    def setup(self, mlt, torch, rank):
        from paper_2103_10516_gb300 import mlt as _m  # noqa: F401
        # scale so that the Gershgorin radius is 10: spectrum inside [-10, 10]
        self.M0 = mlt.Matrix(self.csr)
        _, b = self.M0.bounds()
        self.M0.close()
        self.scale = 10.0 / b
        self.M = mlt.Matrix(self.csr, scale=self.scale)
        # probe-group width by the library's autotuner (untimed setup)
        self.group_width = mlt.mlt_autotune(self.M.handle, "fp32", 4)
        self.out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64, device="cuda")
        self.deg = np.full(self.NPROBES, self.DEG, dtype=np.int32)
        self.base = rank * (1 << 24)

    def step(self, mlt, stream, i):
        return mlt.mlt_moments(self.M.handle, -10.0, 10.0, 0, self.base + (i % 1024) * self.NPROBES,
                               self.deg, precision="fp32", out=self.out, stream=stream)

    def e2e_setup(self, torch):
        self.h_rowptr = torch.from_numpy(self.csr.rowptr).pin_memory()
        self.h_col = torch.from_numpy(self.csr.col).pin_memory()
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (self.h_rowptr.numel() * 8 + self.h_col.numel() * 4, self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h_rowptr, self.h_col, None,
                               scale=self.scale, stream=stream)
        try:
            mlt.mlt_moments(h, -10.0, 10.0, 0, self.base + i * self.NPROBES, self.deg,
                            precision="fp32", out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if self.scale is None:
            self.scale = 10.0 / oracle.gershgorin(self.csr)[1]
        deg = np.full(nprobes, 16, dtype=np.int32)
        oracle.moments(self.csr, -10.0, 10.0, 0, offset, deg, scale=self.scale)
        return nprobes * 16      # the oracle runs direct: one matvec per degree

WORKLOADS = {c.name: c for c in (Triangles, LogDet64, EstradaRmat22)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------

def cpu_oracle_rate(wl, budget_s=12.0):
    import oracle
    oracle.lib()
    cores = os.cpu_count() or 1
    n = max(1, min(cores, 16))
    t0 = time.perf_counter()
    units = wl.cpu_sample(oracle, n, 1 << 30)
    dt = time.perf_counter() - t0
    # grow the sample to about budget_s of wall time
    if dt < budget_s / 4:
        reps = max(1, int(budget_s / max(dt, 1e-3)) - 1)
        n2 = n * reps
        t0 = time.perf_counter()
        units = wl.cpu_sample(oracle, n2, (1 << 30) + n)
        dt = time.perf_counter() - t0
        n = n2
    return {"value": units / dt, "unit": wl.unit, "cores": cores, "kind": "oracle",
            "sample": "%d probes of the same workload (%.1f s wall, OpenMP over probes)" % (n, dt)}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_ours(args, dist):
    import torch
    from paper_2103_10516_gb300 import mlt

    torch.cuda.set_device(dist.local)
    mlt.lib()
    wl = WORKLOADS[args.workload]()
    wl.setup(mlt, torch, dist.rank)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    for i in range(args.warmup):
        wl.step(mlt, sptr, i)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if dist.rank == 0:
        clocks.start()
    mlt.mlt_profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        wl.step(mlt, sptr, args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    stats = mlt.mlt_profile_stop()
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop() if dist.rank == 0 else None
    ms = e0.elapsed_time(e1) / args.steps
    ms = dist.max(ms)
    value = wl.units() * dist.world / (ms / 1e3)

    # roofline of the dominant kernel
    peaks, src = load_peaks()
    kb = wl.kernel_bytes({k: v[0] / args.steps for k, v in stats.items()})
    top = max(stats.items(), key=lambda kv: kv[1][1]) if stats else None
    roof = None
    if top:
        name, (n, tot) = top
        # rows longer than a work chunk of the fused step are finished by a
        # companion launch; its time belongs to the same algorithmic bytes
        companion = {"cheb_step": "cheb_step_long"}.get(name)
        if companion in stats:
            tot = tot + stats[companion][1]
        avg_ms = tot / n
        byt = kb.get(name)
        if byt is not None:
            ach = byt / (avg_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1),
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                    "peak_source": src, "avg_launch_ms": round(avg_ms, 4),
                    "algorithmic_bytes_per_launch": int(byt),
                    "includes": companion if companion in stats else None,
                    "traffic": getattr(wl, "TRAFFIC", {}).get(name),
                    "share_of_step": round(tot / (ms * args.steps), 4)}
    launches = int(sum(v[0] for v in stats.values()))

    # end to end through the C ABI with pinned host buffers
    ke = max(1, min(args.steps, args.e2e_steps))
    h2d, d2h = wl.e2e_setup(torch)
    wl.e2e_step(mlt, sptr, 0)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for i in range(ke):
        wl.e2e_step(mlt, sptr, 1 + i)
    torch.cuda.synchronize()
    te = dist.max((time.perf_counter() - t0) / ke)
    e2e = {"value": wl.units() * dist.world / te, "unit": wl.unit, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": round(te * 1e3, 3), "steps": ke}

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(wl)

    if dist.rank == 0:
        line = {"metric": "probe-matvecs/s", "value": value, "unit": wl.unit, "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": wl.dtype, "data": "synthetic (seeded generator, shapes of the paper's workloads)",
                "config": wl.config(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk,
                "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 4)} for k, v in stats.items()}}
        print(json.dumps(line))


def run_reference(args, dist):
    if dist.rank != 0:
        return
    import oracle
    oracle.lib()
    wl = WORKLOADS[args.workload]()
    cores = os.cpu_count() or 1
    n = max(1, min(cores, 16))
    for i in range(args.warmup):
        wl.cpu_sample(oracle, n, (1 << 30) + i * n)
    t0 = time.perf_counter()
    units = 0
    for i in range(args.steps):
        units += wl.cpu_sample(oracle, n, (1 << 31) + i * n)
    dt = time.perf_counter() - t0
    v = units / dt
    line = {"impl": "reference", "metric": "probe-matvecs/s", "value": v, "unit": wl.unit,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype,
            "data": "synthetic (seeded generator, shapes of the paper's workloads)",
            "config": wl.config(),
            "cpu_baseline": {"value": v, "unit": wl.unit, "cores": cores, "kind": "oracle",
                             "sample": "%d probes per step of the same workload" % n},
            "e2e": {"value": v, "unit": wl.unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat20_triangles", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
