#!/usr/bin/env python3
"""Throughput benchmark of the multilevel Chebyshev-Hutchinson engine on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload estrada_rmat22|rmat20_triangles|logdet64|diffusion64_batched|
                                nuclear_gram|nuclear_explicit|stencil3d|estrada_learned|level_study|
                                estrada_hutchpp]
                    [--precision df64|fp64|fp32|mixed] [--scale S] [--no-comparison]

One step is one pass of the whole hot path over one batch of synthetic input:

  estrada_rmat22 (default): Chebyshev moments of the Estrada-index workload,
      the scale-22 R-MAT adjacency (edge factor 16, seed 1) scaled to spectral
      radius 10 (a Lanczos bound; interval [-10, 10]), 128 probes to degree
      128, in double-float pairs (FP64-class; --precision fp64 or fp32 also),
      on the handle relabelled by degree.  Units: probe-matvecs (64 per probe).
      Setup also compares, untimed, the learned level (FP32 moments, network
      trained on 2^14 probes) with plain FP64 MLMC at equal standard error and
      reports the variance-per-GPU-second gain in config["comparison"].
  rmat20_triangles: exact int64 triangle moments of an R-MAT graph
      (scale 20, edge factor 16, a=0.57, b=c=0.19, seed 0; symmetric, no
      self-loops or duplicates) for 1024 Rademacher probes in blocks of 128,
      two blocks per launch,
      plus the control-variate estimate.  Units: probe-matvecs (2 per probe).
  logdet64: multilevel log-det of the 64x64 Dirichlet Laplacian + 0.1 I,
      levels {8, 32, 128} with {256, 64, 16} probes, FP64.  Units: probe-matvecs
      with the doubling evaluation (3072 per step).
  diffusion64_batched: FP64 log-det level moments of 64 3D diffusion
      operators (10^3 .. 100^3 grids) in one CUDA-graph launch.  Units:
      probe-matvecs summed over the matrices.
  nuclear_gram: moments of X^T X (X 2^18 x 2^16, density 1e-4) for the
      nuclear norm, 512 probes to degree 512, in the --precision given.
      Units: probe-matvecs (X then X^T).
  nuclear_explicit: the same with A = X^T X formed once on the host and
      applied as one SpMM per step (the bandwidth ablation).
  stencil3d: moments of the 7-point 3D diffusion operator on a 100^3 grid,
      128 probes to degree 128, in the --precision given (fp32 default): the
      streaming case of the fused step.
  level_study: the automated-level experiments of Section 5 (level counts,
      budget split, degree sweep against single-level) on a synthetic stand-in
      for the paper's FA graph; the study is in config.
  estrada_learned: the learned coarse level (BF16 network, FP32 moments)
      against plain FP64 MLMC at equal standard error on the Estrada index of
      an R-MAT graph (scale 22 unless --scale); the comparison is in config.
  estrada_hutchpp: Hutch++ (64 sketch + 64 remainder probes, FP64) on the
      configuration-5 Estrada problem, with plain FP64 Hutchinson at the same
      16,384 operator applications run once afterwards; both standard errors
      are in config.  Units: operator applications (probe-matvecs).

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
# FP64 (non-tensor) rate of a GB300, nominal: the denominator of FP64
# recurrence steps (bound by FP64 arithmetic on this part, not by HBM) when the
# measured rate (mlt_fp64_rate, an FMA loop timed on the device) is unavailable
FP64_TFLOPS_NOMINAL = 1.25


# Each rank draws its probes from ids probe_base(rank) .. probe_base(rank) +
# PROBE_SPAN of its workload: disjoint ranges, so the ranks' samples are
# independent (and 8 ranks stay below the 2^32 probe ids of the library).
PROBE_BASE_SHIFT = 28


def probe_base(rank):
    return int(rank) << PROBE_BASE_SHIFT


def estrada_scale(mlt, csr, radius=10.0):
    """Scale that brings the adjacency's spectral radius to `radius`: the
    Lanczos interval (60 steps, Ritz values widened by their residuals and 1%)
    bounds the spectrum, so [-radius, radius] holds the scaled spectrum."""
    M0 = mlt.Matrix(csr)
    try:
        lo, hi = mlt.mlt_spectrum_bounds(M0.handle, mlt.MLT_BOUNDS_LANCZOS, 60, 0)
    finally:
        M0.close()
    return radius / max(abs(lo), abs(hi))


def step_flops(d, nnz, probe_matvecs):
    """Algorithmic FP64 flops of a step's recurrence: 2 per stored entry (one
    FMA) and 8 per vector entry (the update and both dot products) per
    probe-matvec."""
    return probe_matvecs * (2 * nnz + 8 * d)


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
    BLOCK = 256
    PROBE_SPAN = (4096 + 64) * 1024     # timed steps cycle through 4096 blocks; e2e steps follow

    def __init__(self):
        from paper_2103_10516_gb300 import synth
        self.csr = synth.rmat_adjacency(20, 16, seed=0)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz

    def units(self):
        return 2 * self.NPROBES

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale 20, edge factor 16, a=0.57 b=c=0.19, seed 0",
                "d": self.d, "nnz": self.nnz, "probes": self.NPROBES, "block": 128,
                "blocks_per_launch": self.BLOCK // 128,
                "control_variates": True, "control_variate_forms": getattr(self, "cv", None),
                "l2": "inputs larger than L2 (col 4*nnz = %.0f MB + rowptr %.0f MB + y rows %.0f MB)"
                      % (4e-6 * self.nnz, 8e-6 * self.d, 1e-6 * self._ybytes())}

    def _ybytes(self):
        """Bytes of y for one block: 256 per int8 row (degree <= 127), 512 per
        int16 row (<= 32767), 1024 per int32 row; isolated rows have none."""
        deg = np.diff(self.csr.rowptr)
        return int(256 * np.sum((deg > 0) & (deg <= 127)) + 512 * np.sum((deg > 127) & (deg <= 32767))
                   + 1024 * np.sum(deg > 32767))

    def kernel_bytes(self, launches_per_step):
        """Algorithmic bytes per launch (one 256-probe block) of each kernel:
        every array touched once, gathered rows assumed cached.  y of a row
        takes 256 B (degree <= 127, int8), 512 B (<= 32767, int16) or 1 KB
        (int32); the sign bits 32 B.  Pass 1 reads rowptr, col and the sign
        bits and writes y; pass 2 reads the out-list pointers, columns
        (nnz/2), small-section lengths and slots, and y of every row with an
        edge once."""
        d, nnz = self.d, self.nnz
        ybytes = self._ybytes()
        return {
            "tri_zbits": 32 * d,
            "tri_pass1": 8 * (d + 1) + 4 * nnz + 32 * d + ybytes,
            "tri_pass2": 8 * (d + 1) + 4 * (nnz // 2) + 8 * d + ybytes,
        }

    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    # from an ncu capture of this workload, per kernel; to be re-taken
    # whenever the kernel changes
    TRAFFIC = {"tri_pass1": 329.22e6, "tri_pass2": 332.15e6}

    # ours
    def setup(self, mlt, torch, rank):
        self.M = mlt.Matrix(self.csr)
        self.x = torch.empty((self.NPROBES, 3), dtype=torch.int64, device="cuda")
        self.base = probe_base(rank)
        # spectral radius bound for the a-priori control variates (untimed)
        lo, hi = mlt.mlt_spectrum_bounds(self.M.handle, mlt.MLT_BOUNDS_LANCZOS, 60, 0)
        self.rho = max(abs(lo), abs(hi))
        self.cv = None

    def finish(self, ms_per_step):
        """After the timed steps: the estimate of the last step's 1024 probes
        with each control-variate form of Section 5.4 (none; least-squares
        slopes; a priori from the Chebyshev expansion of x^3 on [-r, r] for the
        Gershgorin radius (largest degree) and for the Lanczos bound)."""
        from paper_2103_10516_gb300 import mlt
        x = self.x.cpu().numpy()
        dmax = float(np.max(np.diff(self.csr.rowptr)))
        self.cv = {"probes": int(x.shape[0])}
        for key, cv, r in (("none", "none", 1.0), ("fit", "fit", 1.0), ("cheb_gershgorin", "cheb", dmax),
                           ("cheb_lanczos", "cheb", self.rho)):
            e, se, a1, a2 = mlt.mlt_triangle_estimate(x, self.nnz, cv, -r, r)
            self.cv[key] = {"estimate": e, "stderr": se, "a1": a1, "a2": a2}
            if cv == "cheb":
                self.cv[key]["radius"] = r

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
            mlt.mlt_triangle_trace(h, 0, self.base + (4096 + i) * self.NPROBES, self.NPROBES, self.BLOCK,
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
    PROBE_SPAN = 0     # probes ids restart per seed; each rank and step has its own seed

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

    def kernel_flops(self, launches_per_step):
        n = launches_per_step.get("cheb_step")
        return {"cheb_step": step_flops(self.d, self.nnz, self.units()) / n} if n else {}

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


def learned_comparison(mlt, torch, M, sp, base, ntrain, budget, precision="fp32", epochs=40, batch=2048):
    """The learned coarse level against the plain FP64 multilevel estimator at
    equal standard error, on the handle M (Estrada index: exp on [-10, 10],
    n = 128, levels S, P_64 - S, P_128 - P_64 for the learned form).

      1. plain FP64 MLMC, levels and sample counts from a 10-probe pilot under
         a `budget`-matvec budget: estimate, standard error s_p, GPU time t_p
         (and the same in FP32, to separate precision from the network);
      2. the BF16 network trained on `ntrain` probes ((mu_0..mu_15)/d -> P_64/d);
      3. a pilot of the learned estimator gives its level variances V_k; sample
         counts m_k = sqrt(V_k / C_k) sum_j sqrt(V_j C_j) / s_p^2 (C = 8, 32, 64
         recurrence steps) target the standard error s_p.
    Returns (comparison dict, surrogate, m); the caller times learned estimates
    with m and calls finish_comparison."""
    def timed(fn):
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        out = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3
    N, L1, COST = 128, 64, (8, 32, 64)
    plain, t_p = timed(lambda: M.mlmc("exp", -10.0, 10.0, N, seed=3, m_pilot=10, mode="budget", target=budget,
                                      precision="fp64", stream=sp))
    plain32, t_p32 = timed(lambda: M.mlmc("exp", -10.0, 10.0, N, seed=3, m_pilot=10, mode="budget", target=budget,
                                          precision="fp32", stream=sp))
    S = mlt.Surrogate(5)
    P = mlt.learned_params("exp", -10.0, 10.0, N, L1, 1, 1, 1, seed=7, probe_offset=base, precision=precision,
                           stream=sp)
    loss, t_train = timed(lambda: mlt.mlt_learned_train(M.handle, S.handle, P, ntrain, base, epochs, batch, 2e-3))
    pil = mlt.learned_params("exp", -10.0, 10.0, N, L1, 512, 128, 32, seed=11, probe_offset=base + (1 << 22),
                             precision=precision, stream=sp)
    pilot, t_pil = timed(lambda: mlt.mlt_learned_estimate(M.handle, S.handle, pil))
    V = [max(v, 1e-300) for v in pilot["level_var"]]
    s2 = plain["stderr"] ** 2
    tot = sum(np.sqrt(v * c) for v, c in zip(V, COST))
    m = [max(2, int(np.ceil(np.sqrt(v / c) * tot / s2))) for v, c in zip(V, COST)]
    cmp = {"plain_fp64": {"estimate": plain["estimate"], "stderr": plain["stderr"], "gpu_s": round(t_p, 4),
                          "levels": plain["levels"], "m": plain["m"], "level_var": plain["level_var"],
                          "budget_matvecs": budget},
           "plain_fp32": {"estimate": plain32["estimate"], "stderr": plain32["stderr"], "gpu_s": round(t_p32, 4),
                          "levels": plain32["levels"], "m": plain32["m"]},
           "learned": {"precision": precision, "train_probes": ntrain, "train_gpu_s": round(t_train, 3),
                       "train_loss": loss, "pilot_level_var": V, "pilot_gpu_s": round(t_pil, 4)}}
    return cmp, S, m


def finish_comparison(cmp, results, gpu_s, m):
    """(s^2 t)_plain / (s^2 t)_learned from the learned estimates' standard
    errors (results: (estimate, stderr) pairs) and their mean GPU time."""
    if not results:
        return
    se = float(np.sqrt(np.mean([e[1] ** 2 for e in results])))
    lp = cmp["learned"]
    lp.update({"estimate_first": results[0][0], "stderr": se, "gpu_s": round(gpu_s, 4), "m": m,
               "estimates": len(results)})
    pl = cmp["plain_fp64"]
    cmp["variance_time_gain"] = round((pl["stderr"] ** 2 * pl["gpu_s"]) / (se ** 2 * gpu_s), 3)
    p32 = cmp["plain_fp32"]
    cmp["variance_time_gain_vs_plain_fp32"] = round((p32["stderr"] ** 2 * p32["gpu_s"]) / (se ** 2 * gpu_s), 3)
    cmp["estimates_to_amortise_training"] = round(
        lp["train_gpu_s"] / max(pl["gpu_s"] * (pl["stderr"] ** 2 / se ** 2) - gpu_s, 1e-9), 1)


class EstradaRmat22:
    """The Estrada-index configuration (R-MAT scale 22, edge factor 16, seed 1,
    adjacency scaled to spectral radius 10 by a Lanczos bound, exp on [-10, 10],
    degree 128): Chebyshev moments of 128 probes to degree 128 per step, in
    double-float pairs by default (FP64-class moments on the FP32 pipes; fp64
    and fp32 selectable), on the handle relabelled by degree (MLT_REORDER).
    Setup also runs, untimed, the learned level against plain FP64 MLMC
    (learned_comparison, network trained on 2^14 probes) and reports the
    variance-per-GPU-second gain in config["comparison"]."""
    name = "estrada_rmat22"
    unit = "probe-matvecs/s"
    NPROBES = 128
    DEG = 128
    PROBE_SPAN = 1 << 28     # timed (2^20 ids), e2e (2^20) and comparison (from 2^24) ranges

    def __init__(self, precision=None, compare=True, train_probes=1 << 14, scale=None):
        from paper_2103_10516_gb300 import synth
        self.precision = precision or "df64"
        self.dtype = {"df64": "df64", "fp64": "f64", "fp32": "f32"}[self.precision]
        self.scale_log2 = scale or 22
        self.csr = synth.rmat_adjacency(self.scale_log2, 16, seed=1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.scale = None
        self.compare = compare
        self.train_probes = train_probes
        self.cmp = None

    def units(self):
        return self.NPROBES * ((self.DEG + 1) // 2)

    def config(self):
        prec = {"df64": "double-float vectors and per-thread dots (FP64-class), fp64 after",
                "fp64": "fp64 throughout",
                "fp32": "fp32 vectors, compensated fp32 dots per thread, fp64 after"}[self.precision]
        return {"workload": self.name, "graph": "R-MAT scale %d, edge factor 16, a=0.57 b=c=0.19, seed 1"
                % self.scale_log2,
                "d": self.d, "nnz": self.nnz, "probes": self.NPROBES, "degree": self.DEG, "f": "exp",
                "precision": prec, "interval": [-10.0, 10.0], "scale": self.scale, "relabelled_by_degree": True,
                "group_width": getattr(self, "group_width", None), "comparison": self.cmp,
                "l2": "inputs larger than L2 (V blocks 2 x %.0f MB)" % (self.d * self.NPROBES * self._sv() * 1e-6)}

    def _sv(self):
        return 4 if self.precision == "fp32" else 8

    def kernel_bytes(self, launches_per_step):
        return step_bytes(self.d, self.nnz, 4, self._sv(), self.units(), launches_per_step)

    def kernel_flops(self, launches_per_step):
        n = launches_per_step.get("cheb_step")
        return {"cheb_step": step_flops(self.d, self.nnz, self.units()) / n} if n else {}

    @property
    def TRAFFIC(self):
        """DRAM bytes per cheb_step launch (dram__bytes_read.sum + dram__bytes_write.sum)
        from an ncu capture of the default configuration (scale 22, double-float,
        width 64, relabelled): the mean of three launches; re-taken whenever
        the kernel changes.  Other configurations have no capture."""
        if self.precision == "df64" and self.scale_log2 == 22:
            return {"cheb_step": 29.01e9}
        return {}

    def gather_bytes(self, launches_per_step):
        """Bytes of gathered V_k rows per launch (every stored entry reads its
        column's row slice of the live probes): nnz x s_v per probe-matvec."""
        n = launches_per_step.get("cheb_step")
        return self.nnz * self._sv() * self.units() / n if n else None

    def setup(self, mlt, torch, rank):
        sp = torch.cuda.current_stream().cuda_stream
        self.scale = estrada_scale(mlt, self.csr)       # spectral radius 10: spectrum in [-10, 10]
        self.M = mlt.Matrix(self.csr, scale=self.scale, reorder=True)
        # probe-group width by the library's autotuner (untimed setup)
        self.group_width = mlt.mlt_autotune(self.M.handle, self.precision, 4)
        self.out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64, device="cuda")
        self.deg = np.full(self.NPROBES, self.DEG, dtype=np.int32)
        self.base = probe_base(rank)
        if self.compare:
            cbase = self.base + (1 << 24)
            self.cmp, S, m = learned_comparison(mlt, torch, self.M, sp, cbase, self.train_probes, 16384)
            res, t = [], 0.0
            for i in range(3):
                P = mlt.learned_params("exp", -10.0, 10.0, 128, 64, *m, seed=13,
                                       probe_offset=cbase + (1 << 23) + i * sum(m), precision="fp32", stream=sp)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
                r = mlt.mlt_learned_estimate(self.M.handle, S.handle, P)
                e1.record(torch.cuda.current_stream())
                torch.cuda.synchronize()
                t += e0.elapsed_time(e1) / 1e3
                res.append((r["estimate"], r["stderr"]))
            finish_comparison(self.cmp, res, t / len(res), m)
            S.close()

    def step(self, mlt, stream, i):
        return mlt.mlt_moments(self.M.handle, -10.0, 10.0, 0, self.base + (i % 8192) * self.NPROBES,
                               self.deg, precision=self.precision, out=self.out, stream=stream)

    def e2e_setup(self, torch):
        self.h_rowptr = torch.from_numpy(self.csr.rowptr).pin_memory()
        self.h_col = torch.from_numpy(self.csr.col).pin_memory()
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (self.h_rowptr.numel() * 8 + self.h_col.numel() * 4, self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h_rowptr, self.h_col, None,
                               scale=self.scale, flags=mlt.MLT_REORDER, stream=stream)
        try:
            mlt.mlt_moments(h, -10.0, 10.0, 0, self.base + (8192 + i) * self.NPROBES, self.deg,
                            precision=self.precision, out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if self.scale is None:
            self.scale = 10.0 / gershgorin_upper(self.csr)
        # degree 4: 128M entries a matvec, and the oracle's long-double sums are
        # software quad precision on aarch64 hosts (the rate per matvec is the same)
        deg = np.full(nprobes, 4, dtype=np.int32)
        oracle.moments(self.csr, -10.0, 10.0, 0, offset, deg, scale=self.scale)
        return nprobes * 4       # the oracle runs direct: one matvec per degree


class EstradaHutchpp:
    """Hutch++ (Section 5.3's proposal for the Estrada index) against plain
    Hutchinson at the same operator applications, on configuration 5's matrix:
    R-MAT scale 22 (seed 1) scaled to spectral radius 10, exp on [-10, 10],
    degree 128, FP64.  A step is one Hutch++ estimate with S = 64 sketch and
    G = 64 remainder probes, 64*128 + 128*64 = 16,384 operator applications:
    the cost of 256 doubling probes, configuration 5's step.  After the timed
    steps, one Hutch++ estimate and plain FP64 Hutchinson with 256 probes run
    on fresh probe ids, and the line's config carries both standard errors."""
    name = "estrada_hutchpp"
    unit = "probe-matvecs/s"
    S, G, DEG = 64, 64, 128
    PROBE_SPAN = 1088 * 128 + 128 + 256   # timed, e2e, then the comparison's two runs

    def __init__(self, precision="df64"):
        # fp32: FP32 sketch, the rest FP64; fp64: all FP64; df64: FP32 sketch and
        # double-float moments (FP64-class accuracy on the FP32 pipes)
        self.precision = precision
        self.dtype = "df64" if precision == "df64" else "f64"
        from paper_2103_10516_gb300 import synth
        self.csr = synth.rmat_adjacency(22, 16, seed=1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.scale = None
        self.cmp = None

    def units(self):
        return self.S * self.DEG + (self.S + self.G) * ((self.DEG + 1) // 2)

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale 22, edge factor 16, seed 1",
                "d": self.d, "nnz": self.nnz, "f": "exp", "interval": [-10.0, 10.0], "degree": self.DEG,
                "scale": self.scale, "sketch_probes": self.S, "remainder_probes": self.G,
                "precision": {"fp32": "fp32 sketch, all else fp64", "fp64": "all fp64",
                              "df64": "fp32 sketch, double-float moments, all else fp64"}[self.precision],
                "comparison": self.cmp,
                "l2": "inputs larger than L2 (four 64-column FP64 blocks of %.0f MB)" % (self.d * 64 * 8e-6)}

    def kernel_bytes(self, launches_per_step):
        """Per launch: the matrix (4-byte columns, pattern values) and rowptr, plus per
        column 8-byte rows of V_k, V_{k-1} (and the Clenshaw addend) read and the
        output written."""
        out = {}
        mat = 4 * self.nnz + 8 * (self.d + 1)
        if launches_per_step.get("clenshaw_step"):
            out["clenshaw_step"] = mat + 4 * 8 * self.d * self.S
        n = launches_per_step.get("cheb_step")
        if n:
            out["cheb_step"] = mat + 3 * 8 * self.d * (self.S + self.G) * ((self.DEG + 1) // 2) / n
        return out

    def kernel_flops(self, launches_per_step):
        if self.precision == "df64":
            return {}   # double-float steps are rated against HBM, not the FP64 rate
        out = {}
        if launches_per_step.get("clenshaw_step"):
            out["clenshaw_step"] = self.S * (2 * self.nnz + 8 * self.d)
        n = launches_per_step.get("cheb_step")
        if n:
            out["cheb_step"] = step_flops(self.d, self.nnz, (self.S + self.G) * ((self.DEG + 1) // 2)) / n
        return out

    def setup(self, mlt, torch, rank):
        self.mlt = mlt
        self.scale = estrada_scale(mlt, self.csr)
        self.M = mlt.Matrix(self.csr, scale=self.scale)
        self.c = mlt.mlt_cheb_coeffs("exp", -10.0, 10.0, self.DEG)
        self.base = probe_base(rank)

    def step(self, mlt, stream, i):
        return mlt.mlt_hutchpp_estimate(self.M.handle, -10.0, 10.0, self.c, 0,
                                        self.base + (i % 1024) * (self.S + self.G), self.S, self.G,
                                        precision=self.precision, stream=stream)

    def finish(self, ms):
        mlt = self.mlt
        off = self.base + 1088 * 128
        r = mlt.mlt_hutchpp_estimate(self.M.handle, -10.0, 10.0, self.c, 0, off, self.S, self.G,
                                     precision=self.precision)
        nplain = (self.units() + (self.DEG + 1) // 2 - 1) // ((self.DEG + 1) // 2)
        mu = mlt.mlt_moments(self.M.handle, -10.0, 10.0, 0, off + self.S + self.G, [self.DEG] * nplain,
                             precision="fp64")
        q = mu @ self.c
        se = float(np.std(q, ddof=1) / np.sqrt(nplain))
        self.cmp = {"hutchpp": {"estimate": r.estimate, "stderr": r.std_error, "t_sketch": r.t_sketch,
                                "rank": r.rank, "matvecs": r.matvecs},
                    "hutchinson": {"estimate": float(np.mean(q)), "stderr": se, "probes": nplain,
                                   "matvecs": nplain * ((self.DEG + 1) // 2)},
                    "variance_ratio": (se / r.std_error) ** 2 if r.std_error > 0 else None}

    def e2e_setup(self, torch):
        self.h_rowptr = torch.from_numpy(self.csr.rowptr).pin_memory()
        self.h_col = torch.from_numpy(self.csr.col).pin_memory()
        self.h_samples = np.zeros(self.G)
        return (self.h_rowptr.numel() * 8 + self.h_col.numel() * 4, 8 * self.G + 48)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h_rowptr, self.h_col, None,
                               scale=self.scale, stream=stream)
        try:
            mlt.mlt_hutchpp_estimate(h, -10.0, 10.0, self.c, 0, self.base + (1024 + i) * (self.S + self.G),
                                     self.S, self.G, precision=self.precision, samples=self.h_samples,
                                     stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        """The oracle's Hutch++ at degree 2 with s = g = nprobes / 16 (direct
        recurrences: n operator applications per vector and per moment run)."""
        if self.scale is None:
            self.scale = 10.0 / gershgorin_upper(self.csr)
        n = 2
        c = oracle.cheb_coeffs("exp", -10.0, 10.0, n)
        s = g = max(1, nprobes // 16)
        oracle.hutchpp(self.csr, -10.0, 10.0, c, 0, offset, s, g, scale=self.scale)
        return s * n + (s + g) * n


def gershgorin_upper(c):
    """max_i (a_ii + sum_{j != i} |a_ij|): an upper bound on the spectrum of a
    symmetric CSR (the CPU arms' interval; the GPU arm asks the library)."""
    rows = np.repeat(np.arange(c.nrows), np.diff(c.rowptr))
    v = np.ones(c.nnz) if c.val is None else np.asarray(c.val, dtype=np.float64)
    diag = rows == c.col
    r = np.bincount(rows, weights=np.where(diag, v, np.abs(v)), minlength=c.nrows)
    return float(r.max())


def gram_upper(x):
    """||X||_1 ||X||_inf >= ||X^T X||_2."""
    v = np.abs(np.asarray(x.val, dtype=np.float64))
    rows = np.repeat(np.arange(x.nrows), np.diff(x.rowptr))
    return float(np.bincount(rows, weights=v, minlength=x.nrows).max() *
                 np.bincount(x.col, weights=v, minlength=x.ncols).max())


class Diffusion64Batched:
    """64 log-det moment jobs as one persistent CUDA graph (mlt_batch_create
    once in setup, mlt_batch_run per step with the probe ids shifted).

    Matrix i is the 7-point 3D diffusion operator on an s_i^3 grid, s_i =
    round(10 * 10^(i/63)) (10 .. 100), lognormal cell coefficients (seed i)
    and a diagonal shift drawn from U[0.01, 1]; interval [shift, Gershgorin
    upper bound]; f = log.  Even i: levels {16, 64, 256} with {64, 16, 4}
    probes; odd i: {16, 48, 128, 256} with {64, 32, 8, 4}.  FP64, or
    double-float pairs with --precision df64."""
    name = "diffusion64_batched"
    unit = "probe-matvecs/s"
    NMAT = 64
    PROBE_SPAN = (4096 + 64 + 2) * 128   # every matrix draws from the same id range (its own seed stream)

    def __init__(self, precision="fp64"):
        self.precision = precision
        self.dtype = "df64" if precision == "df64" else "f64"
        from paper_2103_10516_gb300 import synth
        self.mats, self.shift, self.deg = [], [], []
        for i in range(self.NMAT):
            side = int(round(10 * 10 ** (i / 63)))
            sh = float(np.random.default_rng(1000 + i).uniform(0.01, 1.0))
            self.mats.append(synth.diffusion_3d(side, sigma=1.0, shift=sh, seed=i))
            self.shift.append(sh)
            lv, m = ([16, 64, 256], [64, 16, 4]) if i % 2 == 0 else ([16, 48, 128, 256], [64, 32, 8, 4])
            self.deg.append(np.repeat(np.array(lv, dtype=np.int32), m))
        self.d = sum(c.nrows for c in self.mats)
        self.nnz = sum(c.nnz for c in self.mats)
        self.widths = [0] * self.NMAT
        self.seq_ms = None

    def units(self):
        return int(sum(int(np.sum((dg + 1) // 2)) for dg in self.deg))

    def config(self):
        return {"workload": self.name, "matrices": self.NMAT,
                "grid_sides": [self.mats[0].nrows and round(self.mats[0].nrows ** (1 / 3)),
                               round(self.mats[-1].nrows ** (1 / 3))],
                "sum_d": self.d, "sum_nnz": self.nnz, "f": "log",
                "probes_per_matrix": [int(self.deg[0].size), int(self.deg[1].size)],
                "group_widths": sorted(set(self.widths)),
                "sequential_ms_per_step": self.seq_ms, "precision": self.precision,
                "batch_create_ms": getattr(self, "create_ms", None),
                "launch": "one persistent graph (mlt_batch_create once, mlt_batch_run per step)",
                "l2": "inputs larger than L2 (sum of matrices %.0f MB)" % ((12 * self.nnz + 8 * self.d) * 1e-6)}

    def _launches(self, dg, width):
        """Recurrence launches of one job: probes sorted by degree, cut into
        equal groups of at most `width`, each running to its top degree."""
        dg = np.sort(dg)[::-1]
        ng = -(-dg.size // width)
        gs = -(-dg.size // ng)
        return int(sum((int(dg[g0]) + 1) // 2 for g0 in range(0, dg.size, gs)))

    def kernel_bytes(self, launches_per_step):
        return {}

    def graph_step(self):
        """(algorithmic bytes, kernel launches) of one step's graph: per job,
        the recurrence launches stream the matrix once each and every live
        probe's V rows (3 x 8 B); per probe group there is also one probe
        initialisation, one finalisation and a reduction every 16 steps."""
        byt, launches = 0, 0
        for c, dg, w in zip(self.mats, self.deg, self.widths):
            L = self._launches(dg, w if w > 0 else 1024)
            byt += L * (12 * c.nnz + 8 * (c.nrows + 1)) + 24 * c.nrows * int(np.sum((dg + 1) // 2))
            d = np.sort(dg)[::-1]
            width = w if w > 0 else 1024
            ng = -(-d.size // width)
            gs = -(-d.size // ng)
            for g0 in range(0, d.size, gs):
                K = (int(d[g0]) + 1) // 2
                launches += K + 2 + -(-K // 16)
        return byt, launches

    def graph_flops(self):
        return sum(step_flops(c.nrows, c.nnz, int(np.sum((dg + 1) // 2))) for c, dg in zip(self.mats, self.deg))

    def _jobs(self, handles, outs, off):
        return [{"matrix": h.handle, "a": self.shift[k], "b": self.b[k], "seed": 7, "probe_offset": off,
                 "degrees": self.deg[k], "out": outs[k], "group_width": self.widths[k]}
                for k, h in enumerate(handles)]

    def setup(self, mlt, torch, rank):
        self.M = [mlt.Matrix(c) for c in self.mats]
        self.b = [M.bounds()[1] for M in self.M]
        self.widths = [mlt.mlt_autotune(M.handle, self.precision, 4) for M in self.M]
        self.out = [torch.empty((dg.size, 257), dtype=torch.float64, device="cuda") for dg in self.deg]
        self.base = probe_base(rank)
        # the same 64 jobs as separate calls, for comparison (untimed setup)
        stream = torch.cuda.current_stream()
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k, M in enumerate(self.M):
                mlt.mlt_moments(M.handle, self.shift[k], self.b[k], 7, self.base + (4160 + rep) * 128, self.deg[k],
                                precision=self.precision, out=self.out[k], stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            self.seq_ms = round(e0.elapsed_time(e1), 3)
        # the persistent batch: prepared, captured and instantiated once (untimed)
        t0 = time.perf_counter()
        self.batch = mlt.Batch(self._jobs(self.M, self.out, self.base), self.precision,
                               stream=stream.cuda_stream)
        torch.cuda.synchronize()
        self.create_ms = round((time.perf_counter() - t0) * 1e3, 3)

    def step(self, mlt, stream, i):
        # one graph replay; the probe ids move on by 128 a step
        self.batch.run((i % 4096) * 128, stream=stream)

    def e2e_setup(self, torch):
        self.h = [(torch.from_numpy(c.rowptr).pin_memory(), torch.from_numpy(c.col).pin_memory(),
                   torch.from_numpy(c.val).pin_memory()) for c in self.mats]
        self.h_out = [torch.empty((dg.size, 257), dtype=torch.float64).pin_memory() for dg in self.deg]
        h2d = sum(r.numel() * 8 + c.numel() * 4 + v.numel() * 8 for r, c, v in self.h)
        return h2d, sum(o.numel() * 8 for o in self.h_out)

    def e2e_step(self, mlt, stream, i):
        hs = [mlt.mlt_create_csr(c.nrows, c.nrows, c.nnz, r, col, v, stream=stream)
              for c, (r, col, v) in zip(self.mats, self.h)]
        try:
            jobs = [{"matrix": h, "a": self.shift[k], "b": self.b[k], "seed": 7,
                     "probe_offset": self.base + (4096 + i) * 128,
                     "degrees": self.deg[k], "out": self.h_out[k], "group_width": self.widths[k]}
                    for k, h in enumerate(hs)]
            with mlt.Batch(jobs, self.precision, stream=stream) as b:
                b.run(0, stream=stream)
        finally:
            for h in hs:
                mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        # every matrix, nprobes probes to degree 8 each (the oracle runs the
        # direct recurrence: one matvec per degree)
        if not hasattr(self, "b_cpu"):
            self.b_cpu = [gershgorin_upper(c) for c in self.mats]
        deg = np.full(nprobes, 8, dtype=np.int32)
        for c, sh, b in zip(self.mats, self.shift, self.b_cpu):
            oracle.moments(c, sh, b, 7, offset, deg)
        return self.NMAT * int(np.sum(deg))


class NuclearGram:
    """Chebyshev moments of A = X^T X for the nuclear norm (f = sqrt):
    X has 2^18 rows and 2^16 columns, each entry nonzero with probability
    1e-4, N(0,1) values (seed 0); the interval comes from 50 Lanczos steps on
    X^T X; 512 probes to degree 512.  A probe-matvec applies X and then X^T.
    Precision: fp32 (vectors FP32, dots FP64; default), fp64, or mixed
    (FP32 for the first 128 steps, then FP64)."""
    name = "nuclear_gram"
    unit = "probe-matvecs/s"
    NPROBES = 512
    DEG = 512
    PROBE_SPAN = (1024 + 64) * 512

    def __init__(self, precision=None):
        from paper_2103_10516_gb300 import synth
        self.X = synth.sparse_gaussian(1 << 18, 1 << 16, 1e-4, seed=0)
        self.d = self.X.ncols
        self.nnz = self.X.nnz
        self.precision = precision or "fp32"
        self.dtype = {"fp32": "f32", "fp64": "f64", "df64": "df64", "mixed": "f32+f64"}[self.precision]
        self.drift = None

    def _prec(self, mlt):
        return mlt.mixed_at(128) if self.precision == "mixed" else self.precision

    def units(self):
        return self.NPROBES * ((self.DEG + 1) // 2)

    def config(self):
        return {"workload": self.name, "X": "2^18 x 2^16, density 1e-4, N(0,1) values, seed 0",
                "nnz": self.nnz, "operator": "X^T X (two SpMMs per step)", "f": "sqrt",
                "probes": self.NPROBES, "degree": self.DEG, "precision": self.precision,
                "interval": getattr(self, "ab", None), "group_width": getattr(self, "group_width", None),
                "max_abs_dmu_vs_fp64_over_d": self.drift,
                "l2": "inputs larger than L2 per step (V blocks 2 x %.0f MB, X and X^T %.0f MB)"
                      % (self.d * self.NPROBES * (8 if self.precision in ("fp64", "df64") else 4) * 1e-6,
                         2 * 12 * self.nnz * 1e-6)}

    def kernel_bytes(self, launches_per_step):
        """Per launch of each SpMM: its matrix once, and per live probe the
        gathered vector read once and the output written (X V -> W: V read, W
        written; X^T W -> V_{k+1}: W, V_k and V_{k-1} read, V_{k+1} written)."""
        sv = 8 if self.precision in ("fp64", "df64") else 4
        m, n, nnz = self.X.nrows, self.X.ncols, self.nnz
        out = {}
        pm = self.units()
        if launches_per_step.get("gram_spmm"):
            L = launches_per_step["gram_spmm"]
            out["gram_spmm"] = (12 * nnz + 8 * (m + 1)) + (n + m) * sv * pm / L
        if launches_per_step.get("cheb_step"):
            L = launches_per_step["cheb_step"]
            out["cheb_step"] = (12 * nnz + 8 * (n + 1)) + (m + 3 * n) * sv * pm / L
        return out

    def setup(self, mlt, torch, rank):
        self.M = mlt.Matrix(self.X, gram=True)
        self.ab = [round(v, 6) for v in mlt.mlt_spectrum_bounds(self.M.handle, mlt.MLT_BOUNDS_LANCZOS, 50, 0)]
        self.group_width = mlt.mlt_autotune(self.M.handle, "fp32" if self.precision == "mixed" else self.precision, 4)
        self.out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64, device="cuda")
        self.deg = np.full(self.NPROBES, self.DEG, dtype=np.int32)
        self.base = probe_base(rank)
        if self.precision != "fp64":
            # drift of this precision against FP64 on 32 probes (untimed)
            deg = self.deg[:32]
            lo = mlt.mlt_moments(self.M.handle, *self.ab, 0, 0, deg, precision=self._prec(mlt))
            hi = mlt.mlt_moments(self.M.handle, *self.ab, 0, 0, deg, precision="fp64")
            self.drift = float(np.max(np.abs(lo - hi)) / self.d)

    def step(self, mlt, stream, i):
        return mlt.mlt_moments(self.M.handle, self.ab[0], self.ab[1], 0, self.base + (i % 1024) * self.NPROBES,
                               self.deg, precision=self._prec(mlt), out=self.out, stream=stream)

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.X.rowptr).pin_memory(), torch.from_numpy(self.X.col).pin_memory(),
                  torch.from_numpy(self.X.val).pin_memory())
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (sum(t.numel() * t.element_size() for t in self.h), self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        r, c, v = self.h
        h = mlt.mlt_create_csr(self.X.nrows, self.X.ncols, self.nnz, r, c, v, flags=mlt.MLT_GRAM, stream=stream)
        try:
            mlt.mlt_moments(h, self.ab[0], self.ab[1], 0, self.base + (1024 + i) * self.NPROBES, self.deg,
                            precision=self._prec(mlt), out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if not hasattr(self, "ab"):
            self.ab = [0.0, gram_upper(self.X)]
        deg = np.full(nprobes, 16, dtype=np.int32)
        oracle.moments(self.X, self.ab[0], self.ab[1], 0, offset, deg, gram=True)
        return int(np.sum(deg))                  # direct recurrence: one probe-matvec per degree


class NuclearExplicit(NuclearGram):
    """The nuclear-norm workload with A = X^T X formed explicitly (a sparse
    product on the host, about 11M entries) and run through the plain
    recurrence: the bandwidth ablation of the two-SpMM Gram operator.  Same
    probes, degree, precision and Lanczos interval (taken from the Gram
    handle)."""
    name = "nuclear_explicit"

    def __init__(self, precision=None):
        super().__init__(precision)
        import scipy.sparse as sp
        from paper_2103_10516_gb300 import synth
        X = sp.csr_matrix((self.X.val, self.X.col, self.X.rowptr), shape=(self.X.nrows, self.X.ncols))
        A = (X.T @ X).tocsr()
        A.sort_indices()
        self.A = synth.CSR(A.shape[0], A.shape[1], A.indptr.astype(np.int64), A.indices.astype(np.int32),
                           A.data.astype(np.float64))
        self.nnz_a = int(A.nnz)

    def config(self):
        c = super().config()
        c.update({"workload": self.name, "operator": "A = X^T X formed explicitly (one SpMM per step)",
                  "nnz_A": self.nnz_a})
        return c

    def kernel_bytes(self, launches_per_step):
        sv = 8 if self.precision in ("fp64", "df64") else 4
        return step_bytes(self.d, self.nnz_a, 4 + sv, sv, self.units(), launches_per_step)

    def setup(self, mlt, torch, rank):
        G = mlt.Matrix(self.X, gram=True)
        self.ab = [round(v, 6) for v in mlt.mlt_spectrum_bounds(G.handle, mlt.MLT_BOUNDS_LANCZOS, 50, 0)]
        G.close()
        self.M = mlt.Matrix(self.A)
        self.group_width = mlt.mlt_autotune(self.M.handle, "fp32" if self.precision == "mixed" else self.precision, 4)
        self.out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64, device="cuda")
        self.deg = np.full(self.NPROBES, self.DEG, dtype=np.int32)
        self.base = probe_base(rank)

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.A.rowptr).pin_memory(), torch.from_numpy(self.A.col).pin_memory(),
                  torch.from_numpy(self.A.val).pin_memory())
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (sum(t.numel() * t.element_size() for t in self.h), self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        r, c, v = self.h
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz_a, r, c, v, stream=stream)
        try:
            mlt.mlt_moments(h, self.ab[0], self.ab[1], 0, self.base + (1024 + i) * self.NPROBES, self.deg,
                            precision=self._prec(mlt), out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if not hasattr(self, "ab"):
            self.ab = [0.0, gram_upper(self.X)]
        deg = np.full(nprobes, 16, dtype=np.int32)
        oracle.moments(self.A, self.ab[0], self.ab[1], 0, offset, deg)
        return int(np.sum(deg))


class Stencil3D:
    """Chebyshev moments of one large 3D diffusion operator: the 7-point
    operator on a 100^3 grid (d = 10^6, lognormal coefficients, seed 0, shift
    0.1), 128 probes to degree 128, interval [0.1, Gershgorin bound], in the
    --precision given (fp32 by default).  A streaming case for the fused step:
    V rows of neighbouring grid cells are near each other, so the step's cost
    is the matrix and the three V blocks it streams."""
    name = "stencil3d"
    unit = "probe-matvecs/s"
    NPROBES = 128
    DEG = 128
    PROBE_SPAN = (1024 + 64) * 128

    def __init__(self, precision=None):
        from paper_2103_10516_gb300 import synth
        self.csr = synth.diffusion_3d(100, sigma=1.0, shift=0.1, seed=0)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.precision = precision or "fp32"
        # DRAM bytes per launch (128 live probes) from an ncu capture of the
        # FP32 step kernel as built (dram__bytes_read.sum + dram__bytes_write.sum)
        self.TRAFFIC = {"fp32": {"cheb_step": 1.632e9}}.get(self.precision, {})
        self.dtype = {"fp32": "f32", "fp64": "f64", "df64": "df64", "mixed": "f32+f64"}[self.precision]

    def _prec(self, mlt):
        return mlt.mixed_at(32) if self.precision == "mixed" else self.precision

    def units(self):
        return self.NPROBES * ((self.DEG + 1) // 2)

    def config(self):
        return {"workload": self.name, "matrix": "7-point 3D diffusion, 100^3 grid, lognormal kappa, shift 0.1",
                "d": self.d, "nnz": self.nnz, "probes": self.NPROBES, "degree": self.DEG,
                "precision": self.precision, "interval": getattr(self, "ab", None),
                "group_width": getattr(self, "group_width", None),
                "l2": "inputs larger than L2 (V blocks 2 x %.0f MB)"
                      % (self.d * self.NPROBES * (8 if self.precision in ("fp64", "df64") else 4) * 1e-6)}

    def kernel_bytes(self, launches_per_step):
        sv = 8 if self.precision in ("fp64", "df64") else 4
        return step_bytes(self.d, self.nnz, 4 + sv, sv, self.units(), launches_per_step)

    def kernel_flops(self, launches_per_step):
        n = launches_per_step.get("cheb_step")
        return {"cheb_step": step_flops(self.d, self.nnz, self.units()) / n} if n else {}

    def setup(self, mlt, torch, rank):
        self.M = mlt.Matrix(self.csr)
        self.ab = [0.1, self.M.bounds()[1]]
        self.group_width = mlt.mlt_autotune(self.M.handle, "fp32" if self.precision == "mixed" else self.precision, 4)
        self.out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64, device="cuda")
        self.deg = np.full(self.NPROBES, self.DEG, dtype=np.int32)
        self.base = probe_base(rank)

    def step(self, mlt, stream, i):
        return mlt.mlt_moments(self.M.handle, self.ab[0], self.ab[1], 0, self.base + (i % 1024) * self.NPROBES,
                               self.deg, precision=self._prec(mlt), out=self.out, stream=stream)

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.csr.rowptr).pin_memory(), torch.from_numpy(self.csr.col).pin_memory(),
                  torch.from_numpy(self.csr.val).pin_memory())
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (sum(t.numel() * t.element_size() for t in self.h), self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        r, c, v = self.h
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, r, c, v, stream=stream)
        try:
            mlt.mlt_moments(h, self.ab[0], self.ab[1], 0, self.base + (1024 + i) * self.NPROBES, self.deg,
                            precision=self._prec(mlt), out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if not hasattr(self, "ab"):
            self.ab = [0.1, gershgorin_upper(self.csr)]
        deg = np.full(nprobes, 8, dtype=np.int32)
        oracle.moments(self.csr, self.ab[0], self.ab[1], 0, offset, deg)
        return int(np.sum(deg))                  # direct recurrence: one probe-matvec per degree


class EstradaLearned:
    """The learned coarse level against the plain FP64 multilevel estimator,
    at equal standard error, on the Estrada index tr exp(A): R-MAT adjacency
    (edge factor 16, seed 1) scaled to spectral radius 10 (a Lanczos bound),
    interval [-10, 10], n = 128.

    Setup (untimed, reported in config["comparison"]):
      1. plain FP64 MLMC with levels and sample counts from a 10-probe pilot
         under a fixed matvec budget: estimate, standard error s_p, GPU time t_p;
      2. the BF16 network trained on 2^16 probes ((mu_0..mu_15)/d ->
         P_64/d), GPU time of training;
      3. a small pilot of the learned estimator gives the variances V_k of its
         levels (S, P_64 - S, P_128 - P_64); sample counts m_k follow the
         optimal allocation m_k = sqrt(V_k / C_k) sum_j sqrt(V_j C_j) / s_p^2
         (C = 8, 32, 64 recurrence steps) so that its standard error matches s_p.
    Step (timed): one learned estimate with those m_k, its moments in the
    --precision given (fp32 by default, or fp64).  The reported ratio is
    (s^2 t)_plain / (s^2 t)_learned, the variance-per-GPU-second gain."""
    name = "estrada_learned"
    unit = "probe-matvecs/s"
    L1, N = 64, 128
    COST = (8, 32, 64)
    PROBE_SPAN = 1 << 28       # training, pilot, timed and e2e ranges below, all inside it

    def __init__(self, scale=None, precision=None):
        from paper_2103_10516_gb300 import synth
        self.scale_log2 = scale or 22
        self.precision = precision or "fp32"
        self.dtype = "f32+bf16" if self.precision == "fp32" else "f64+bf16"
        self.csr = synth.rmat_adjacency(self.scale_log2, 16, seed=1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.ntrain = 1 << 16
        self.budget = 16384
        self.cmp = None
        self.m = None
        self.scale = None

    def units(self):
        return int(sum(mk * c for mk, c in zip(self.m, self.COST)))

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale %d, edge factor 16, seed 1" % self.scale_log2,
                "d": self.d, "nnz": self.nnz, "f": "exp", "interval": [-10.0, 10.0], "scale": self.scale,
                "n": self.N,
                "l1": self.L1, "train_probes": self.ntrain, "precision": self.precision, "m": self.m,
                "comparison": self.cmp,
                "l2": "inputs larger than L2 (V blocks of 4 B x d per probe)"}

    def kernel_bytes(self, launches_per_step):
        sv = 8 if self.precision in ("fp64", "df64") else 4
        return step_bytes(self.d, self.nnz, 4, sv, self.units(), launches_per_step)

    def setup(self, mlt, torch, rank):
        sp = torch.cuda.current_stream().cuda_stream
        self.scale = estrada_scale(mlt, self.csr)       # spectral radius 10: spectrum in [-10, 10]
        self.M = mlt.Matrix(self.csr, scale=self.scale, reorder=True)
        self.group_width = mlt.mlt_autotune(self.M.handle, self.precision, 4)
        base = probe_base(rank)
        self.cmp, self.S, self.m = learned_comparison(mlt, torch, self.M, sp, base, self.ntrain, self.budget,
                                                      precision=self.precision)
        self.base = base + (1 << 23)
        self.results = []

    def step(self, mlt, stream, i):
        P = mlt.learned_params("exp", -10.0, 10.0, self.N, self.L1, *self.m, seed=13,
                               probe_offset=self.base + i * sum(self.m), precision=self.precision, stream=stream)
        r = mlt.mlt_learned_estimate(self.M.handle, self.S.handle, P)
        self.results.append((r["estimate"], r["stderr"]))
        return r

    def finish(self, ms_per_step):
        """Called after the timed steps: the comparison at the measured time."""
        finish_comparison(self.cmp, self.results, ms_per_step / 1e3, self.m)

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.csr.rowptr).pin_memory(), torch.from_numpy(self.csr.col).pin_memory(),
                  torch.from_numpy(self.csr.val).pin_memory())
        self.h_out = torch.empty((self.NPROBES, self.DEG + 1), dtype=torch.float64).pin_memory()
        return (sum(t.numel() * t.element_size() for t in self.h), self.h_out.numel() * 8)

    def e2e_step(self, mlt, stream, i):
        r, c, v = self.h
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, r, c, v, stream=stream)
        try:
            mlt.mlt_moments(h, self.ab[0], self.ab[1], 0, self.base + (1024 + i) * self.NPROBES, self.deg,
                            precision=self._prec(mlt), out=self.h_out, stream=stream)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if not hasattr(self, "ab"):
            self.ab = [0.1, gershgorin_upper(self.csr)]
        deg = np.full(nprobes, 8, dtype=np.int32)
        oracle.moments(self.csr, self.ab[0], self.ab[1], 0, offset, deg)
        return int(np.sum(deg))                  # direct recurrence: one probe-matvec per degree


class EstradaLearned:
    """The learned coarse level against the plain FP64 multilevel estimator,
    at equal standard error, on the Estrada index tr exp(A): R-MAT adjacency
    (edge factor 16, seed 1) scaled to spectral radius 10 (a Lanczos bound),
    interval [-10, 10], n = 128.

    Setup (untimed, reported in config["comparison"]):
      1. plain FP64 MLMC with levels and sample counts from a 10-probe pilot
         under a fixed matvec budget: estimate, standard error s_p, GPU time t_p;
      2. the BF16 network trained on 2^16 probes ((mu_0..mu_15)/d ->
         P_64/d), GPU time of training;
      3. a small pilot of the learned estimator gives the variances V_k of its
         levels (S, P_64 - S, P_128 - P_64); sample counts m_k follow the
         optimal allocation m_k = sqrt(V_k / C_k) sum_j sqrt(V_j C_j) / s_p^2
         (C = 8, 32, 64 recurrence steps) so that its standard error matches s_p.
    Step (timed): one learned estimate with those m_k, its moments in the
    --precision given (fp32 by default, or fp64).  The reported ratio is
    (s^2 t)_plain / (s^2 t)_learned, the variance-per-GPU-second gain."""
    name = "estrada_learned"
    unit = "probe-matvecs/s"
    L1, N = 64, 128
    COST = (8, 32, 64)
    PROBE_SPAN = 1 << 28       # training, pilot, timed and e2e ranges below, all inside it

    def __init__(self, scale=None, precision=None):
        from paper_2103_10516_gb300 import synth
        self.scale_log2 = scale or 22
        self.precision = precision or "fp32"
        self.dtype = "f32+bf16" if self.precision == "fp32" else "f64+bf16"
        self.csr = synth.rmat_adjacency(self.scale_log2, 16, seed=1)
        self.d = self.csr.nrows
        self.nnz = self.csr.nnz
        self.ntrain = 1 << 16
        self.budget = 16384
        self.cmp = None
        self.m = None
        self.scale = None

    def units(self):
        return int(sum(mk * c for mk, c in zip(self.m, self.COST)))

    def config(self):
        return {"workload": self.name, "graph": "R-MAT scale %d, edge factor 16, seed 1" % self.scale_log2,
                "d": self.d, "nnz": self.nnz, "f": "exp", "interval": [-10.0, 10.0], "scale": self.scale,
                "n": self.N,
                "l1": self.L1, "train_probes": self.ntrain, "precision": self.precision, "m": self.m,
                "comparison": self.cmp,
                "l2": "inputs larger than L2 (V blocks of 4 B x d per probe)"}

    def kernel_bytes(self, launches_per_step):
        sv = 8 if self.precision in ("fp64", "df64") else 4
        return step_bytes(self.d, self.nnz, 4, sv, self.units(), launches_per_step)

    def _timed(self, torch, fn):
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        out = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    def setup(self, mlt, torch, rank):
        sp = torch.cuda.current_stream().cuda_stream
        self.scale = estrada_scale(mlt, self.csr)       # spectral radius 10: spectrum in [-10, 10]
        self.M = mlt.Matrix(self.csr, scale=self.scale)
        self.group_width = mlt.mlt_autotune(self.M.handle, self.precision, 4)
        base = probe_base(rank)
        plain, t_p = self._timed(torch, lambda: self.M.mlmc(
            "exp", -10.0, 10.0, self.N, seed=3, m_pilot=10, mode="budget", target=self.budget,
            precision="fp64", stream=sp))
        # the same plain estimator with FP32 moments, to separate the precision
        # from the learned level in the comparison
        plain32, t_p32 = self._timed(torch, lambda: self.M.mlmc(
            "exp", -10.0, 10.0, self.N, seed=3, m_pilot=10, mode="budget", target=self.budget,
            precision="fp32", stream=sp))
        self.S = mlt.Surrogate(5)
        P = mlt.learned_params("exp", -10.0, 10.0, self.N, self.L1, 1, 1, 1, seed=7, probe_offset=base,
                               precision=self.precision, stream=sp)
        loss, t_train = self._timed(torch, lambda: mlt.mlt_learned_train(
            self.M.handle, self.S.handle, P, self.ntrain, base, 40, 2048, 2e-3))
        pil = mlt.learned_params("exp", -10.0, 10.0, self.N, self.L1, 512, 128, 32, seed=11,
                                 probe_offset=base + (1 << 22), precision=self.precision, stream=sp)
        pilot, t_pil = self._timed(torch, lambda: mlt.mlt_learned_estimate(self.M.handle, self.S.handle, pil))
        V = [max(v, 1e-300) for v in pilot["level_var"]]
        s2 = plain["stderr"] ** 2
        tot = sum(np.sqrt(v * c) for v, c in zip(V, self.COST))
        self.m = [max(2, int(np.ceil(np.sqrt(v / c) * tot / s2))) for v, c in zip(V, self.COST)]
        self.base = base + (1 << 23)
        self.cmp = {"plain_fp64": {"estimate": plain["estimate"], "stderr": plain["stderr"],
                                   "gpu_s": round(t_p, 4), "levels": plain["levels"], "m": plain["m"],
                                   "level_var": plain["level_var"], "budget_matvecs": self.budget},
                    "plain_fp32": {"estimate": plain32["estimate"], "stderr": plain32["stderr"],
                                   "gpu_s": round(t_p32, 4), "levels": plain32["levels"], "m": plain32["m"]},
                    "learned": {"precision": self.precision, "train_gpu_s": round(t_train, 3), "train_loss": loss,
                                "pilot_level_var": V, "pilot_gpu_s": round(t_pil, 4)}}
        self.results = []

    def step(self, mlt, stream, i):
        P = mlt.learned_params("exp", -10.0, 10.0, self.N, self.L1, *self.m, seed=13,
                               probe_offset=self.base + i * sum(self.m), precision=self.precision, stream=stream)
        r = mlt.mlt_learned_estimate(self.M.handle, self.S.handle, P)
        self.results.append((r["estimate"], r["stderr"]))
        return r

    def finish(self, ms_per_step):
        """Called after the timed steps: the comparison at the measured time."""
        if not self.results:
            return
        se = float(np.sqrt(np.mean([e[1] ** 2 for e in self.results])))
        lp = self.cmp["learned"]
        lp.update({"estimate_first": self.results[0][0], "stderr": se, "gpu_s": round(ms_per_step / 1e3, 4),
                   "m": self.m})
        pl = self.cmp["plain_fp64"]
        gain = (pl["stderr"] ** 2 * pl["gpu_s"]) / (se ** 2 * lp["gpu_s"])
        self.cmp["variance_time_gain"] = round(gain, 3)
        p32 = self.cmp["plain_fp32"]
        self.cmp["variance_time_gain_vs_plain_fp32"] = round(
            (p32["stderr"] ** 2 * p32["gpu_s"]) / (se ** 2 * lp["gpu_s"]), 3)
        n_runs_to_amortise = lp["train_gpu_s"] / max(pl["gpu_s"] * (pl["stderr"] ** 2 / se ** 2) - lp["gpu_s"], 1e-9)
        self.cmp["estimates_to_amortise_training"] = round(n_runs_to_amortise, 1)

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.csr.rowptr).pin_memory(), torch.from_numpy(self.csr.col).pin_memory())
        return (self.h[0].numel() * 8 + self.h[1].numel() * 4, 8 * 3 * 4)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.d, self.d, self.nnz, self.h[0], self.h[1], None, scale=self.scale,
                               flags=mlt.MLT_REORDER, stream=stream)
        try:
            P = mlt.learned_params("exp", -10.0, 10.0, self.N, self.L1, *self.m, seed=17,
                                   probe_offset=base_e2e(self.base) + i * sum(self.m), precision=self.precision,
                                   stream=stream)
            mlt.mlt_learned_estimate(h, self.S.handle, P)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if self.scale is None:
            self.scale = 10.0 / gershgorin_upper(self.csr)
        deg = np.full(nprobes, 4, dtype=np.int32)     # as for estrada_rmat22
        oracle.moments(self.csr, -10.0, 10.0, 0, offset, deg, scale=self.scale)
        return nprobes * 4


class LevelStudy:
    """The automated-level experiments of Section 5 replayed on a synthetic
    stand-in for the paper's directed graph FA (10,617 nodes, 72,176 edges):
    a directed R-MAT graph (scale 14, a=0.57, b=c=0.19, seed 4) restricted to
    its first 10,617 vertices, the first 72,176 distinct edges in generation
    order, no self-loops.  f = sqrt of A^T A (the nuclear norm of A), interval
    [0, b] with b from 50 Lanczos steps on A^T A, FP64.

    Setup (untimed, reported in config["study"]):
      level selection: TRIALS automatic estimates at n = 300 with a budget of
        15,000 (steps of A^T A, ceil(l/2) per probe of degree l) and a 10-probe
        pilot: level counts, the share of the budget spent at degree <= 50,
        the degree of the second most expensive level, standard errors;
      degree sweep: for n in SWEEP, single-level estimates (50 probes at
        degree n) against automatic multilevel ones at the same cost
        (budget 50 ceil(n/2)): median standard errors and median |errors|
        against the exact nuclear norm, beside |tr p_n - tr f| from the exact
        spectrum (a dense eigendecomposition of A^T A, for reference only).
    Step (timed): one automatic estimate at n = 300, budget 15,000."""
    name = "level_study"
    unit = "probe-matvecs/s"
    dtype = "f64"
    D, E = 10617, 72176
    N, BUDGET, PILOT = 300, 15000, 10
    TRIALS = 100
    SWEEP = (25, 50, 100, 150, 200, 250, 300, 350)
    SWEEP_TRIALS = 30
    PROBE_SPAN = 0     # probes ids restart per seed; each trial and rank has its own seed

    def __init__(self):
        from paper_2103_10516_gb300 import synth
        r, c = synth.rmat_edges(14, 8, seed=4)
        keep = (r < self.D) & (c < self.D) & (r != c)
        key = r[keep] * self.D + c[keep]
        _, first = np.unique(key, return_index=True)
        key = key[np.sort(first)][: self.E]
        self.X = synth._from_coo(self.D, self.D, key // self.D, key % self.D, None)
        self.study = None
        self.done = []

    def units(self):
        return float(np.mean(self.done)) if self.done else 1.0

    def config(self):
        return {"workload": self.name, "graph": "directed R-MAT stand-in for FA: %d nodes, %d edges" % (self.D, self.E),
                "operator": "A^T A (two SpMMs per step)", "f": "sqrt", "n": self.N, "budget": self.BUDGET,
                "m_pilot": self.PILOT, "interval": getattr(self, "ab", None), "study": self.study,
                "l2": "L2-resident (A: %d entries); flushed between steps by a 256 MB write" % self.X.nnz}

    def kernel_bytes(self, launches_per_step):
        return {}

    def kernel_flops(self, launches_per_step):
        out = {}
        fl = self.units() * (2 * self.X.nnz + 4 * self.D)     # one X or X^T product per launch
        for k in ("cheb_step", "gram_spmm"):
            if launches_per_step.get(k):
                out[k] = fl / launches_per_step[k]
        return out

    def _trial(self, seed, n, stream, budget=None, single=None):
        if single is not None:
            return self.M.mlmc("sqrt", self.ab[0], self.ab[1], n, seed=seed, levels=[n], m=[single], stream=stream)
        return self.M.mlmc("sqrt", self.ab[0], self.ab[1], n, seed=seed, m_pilot=self.PILOT, mode="budget",
                           target=float(budget), stream=stream)

    def setup(self, mlt, torch, rank):
        sp = torch.cuda.current_stream().cuda_stream
        self.M = mlt.Matrix(self.X, gram=True)
        _, hi = mlt.mlt_spectrum_bounds(self.M.handle, mlt.MLT_BOUNDS_LANCZOS, 50, 0)
        self.ab = [0.0, hi]
        self.flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
        self.seed0 = (rank + 1) << 20
        # exact spectrum of A^T A, for the error columns only
        Xd = torch.zeros((self.D, self.D), dtype=torch.float64, device="cuda")
        rows = np.repeat(np.arange(self.D), np.diff(self.X.rowptr))
        Xd[torch.from_numpy(rows).cuda(), torch.from_numpy(self.X.col.astype(np.int64)).cuda()] = 1.0
        lam = torch.linalg.eigvalsh(Xd.T @ Xd).clamp_min(0.0).cpu().numpy()
        del Xd
        tr_f = float(np.sum(np.sqrt(lam)))
        x = np.clip((2 * lam - (self.ab[0] + self.ab[1])) / (self.ab[1] - self.ab[0]), -1.0, 1.0)
        th = np.arccos(x)

        def tr_p(n):
            c = mlt.mlt_cheb_coeffs("sqrt", self.ab[0], self.ab[1], n)
            return float(sum(c[j] * np.sum(np.cos(j * th)) for j in range(n + 1)))

        # level selection at n = 300
        nlev, share50, second, se = [], [], [], []
        for t in range(self.TRIALS):
            r = self._trial(self.seed0 + t, self.N, sp, budget=self.BUDGET)
            cost = [mk * ((l + 1) // 2) for l, mk in zip(r["levels"], r["m"])]
            nlev.append(len(r["levels"]))
            share50.append(sum(cst for l, cst in zip(r["levels"], cost) if l <= 50) / sum(cost))
            order = np.argsort(cost)[::-1]
            second.append(int(r["levels"][order[1]]) if len(order) > 1 else int(r["levels"][0]))
            se.append(r["stderr"])
        sel = {"trials": self.TRIALS, "levels_median": float(np.median(nlev)), "levels_min": int(min(nlev)),
               "levels_max": int(max(nlev)), "budget_share_deg_le_50_median": round(float(np.median(share50)), 3),
               "second_costliest_degree_median": float(np.median(second)),
               "second_costliest_degree_max": int(max(second)),
               # a level drawn once has no sample variance: its trial's standard error is NaN
               "stderr_median_finite": float(np.nanmedian(se)) if np.isfinite(se).any() else None,
               "trials_with_a_single_sample_level": int(np.sum(~np.isfinite(se))),
               "exact_nuclear_norm": tr_f}
        # degree sweep at equal cost
        sweep = []
        for n in self.SWEEP:
            s1, e1, s2, e2 = [], [], [], []
            for t in range(self.SWEEP_TRIALS):
                a = self._trial(self.seed0 + 10000 + t, n, sp, single=50)
                b = self._trial(self.seed0 + 20000 + t, n, sp, budget=50 * ((n + 1) // 2))
                s1.append(a["stderr"])
                e1.append(abs(a["estimate"] - tr_f))
                s2.append(b["stderr"])
                e2.append(abs(b["estimate"] - tr_f))
            sweep.append({"n": n, "poly_error": abs(tr_p(n) - tr_f), "single_stderr_median": float(np.median(s1)),
                          "single_abs_error_median": float(np.median(e1)),
                          "multi_stderr_median_finite": float(np.nanmedian(s2)) if np.isfinite(s2).any() else None,
                          "multi_trials_with_a_single_sample_level": int(np.sum(~np.isfinite(s2))),
                          "multi_abs_error_median": float(np.median(e2))})
        self.study = {"level_selection": sel, "degree_sweep": sweep, "sweep_trials": self.SWEEP_TRIALS}

    def step(self, mlt, stream, i):
        self.flush.fill_(float(i))
        r = self._trial(self.seed0 + 100000 + i, self.N, stream, budget=self.BUDGET)
        self.done.append(r["matvecs"])
        return r

    def e2e_setup(self, torch):
        self.h = (torch.from_numpy(self.X.rowptr).pin_memory(), torch.from_numpy(self.X.col).pin_memory())
        return (self.h[0].numel() * 8 + self.h[1].numel() * 4, 8 * 2)

    def e2e_step(self, mlt, stream, i):
        h = mlt.mlt_create_csr(self.D, self.D, self.X.nnz, self.h[0], self.h[1], None, flags=mlt.MLT_GRAM,
                               stream=stream)
        try:
            P = mlt.mlt_mlmc_default_params()
            P.fn, P.a, P.b, P.n, P.seed = 1, self.ab[0], self.ab[1], self.N, self.seed0 + 200000 + i
            P.m_pilot, P.target = self.PILOT, float(self.BUDGET)
            P.stream = stream
            mlt.mlt_mlmc_estimate(h, P)
        finally:
            mlt.mlt_destroy(h)

    def cpu_sample(self, oracle, nprobes, offset):
        if not hasattr(self, "ab"):
            self.ab = [0.0, gram_upper(self.X)]
        deg = np.full(nprobes, 64, dtype=np.int32)
        oracle.moments(self.X, self.ab[0], self.ab[1], 0, offset, deg, gram=True)
        return int(np.sum(deg))


def base_e2e(timed_base):
    """Probe ids of the learned workload's end-to-end steps: past its timed ones."""
    return timed_base + (1 << 26)


WORKLOADS = {c.name: c for c in (Triangles, LogDet64, EstradaRmat22, Diffusion64Batched, NuclearGram,
                                            NuclearExplicit, Stencil3D, EstradaLearned, LevelStudy,
                                            EstradaHutchpp)}


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
    wl = make_workload(args)
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
    if hasattr(wl, "finish"):
        wl.finish(ms)
    value = wl.units() * dist.world / (ms / 1e3)

    # roofline of the dominant kernel
    peaks, src = load_peaks()
    fp64_peak, fp64_src = FP64_TFLOPS_NOMINAL, "nominal FP64 rate of GB300"
    if wl.dtype == "f64":
        try:
            fp64_peak = max(mlt.mlt_fp64_rate(1 << 16) for _ in range(3))
            fp64_src = "measured: register-resident FP64 FMA loop (mlt_fp64_rate), best of 3"
        except Exception:
            pass
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
        kf = wl.kernel_flops({k: v[0] / args.steps for k, v in stats.items()}) \
            if wl.dtype == "f64" and hasattr(wl, "kernel_flops") else {}
        if kf.get(name) is not None:
            ach = kf[name] / (avg_ms / 1e3) / 1e12
            roof = {"bound": "alu", "kernel": name, "achieved": round(ach, 4), "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                    "peak_source": fp64_src, "avg_launch_ms": round(avg_ms, 4),
                    "algorithmic_flops_per_launch": int(kf[name]),
                    "hbm_gbs_on_algorithmic_bytes": round(byt / (avg_ms / 1e3) / 1e9, 1) if byt else None,
                    "includes": companion if companion in stats else None,
                    "traffic": getattr(wl, "TRAFFIC", {}).get(name), "share_of_step": round(tot / (ms * args.steps), 4)}
        elif byt is not None:
            ach = byt / (avg_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1),
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                    "peak_source": src, "avg_launch_ms": round(avg_ms, 4),
                    "algorithmic_bytes_per_launch": int(byt),
                    "includes": companion if companion in stats else None,
                    "traffic": getattr(wl, "TRAFFIC", {}).get(name),
                    "share_of_step": round(tot / (ms * args.steps), 4)}
            gb = wl.gather_bytes({k: v[0] / args.steps for k, v in stats.items()}) \
                if hasattr(wl, "gather_bytes") and name == "cheb_step" else None
            if gb:
                # the gathered rows, beside the algorithmic bytes: a row of V_k
                # is read once per stored entry, mostly from L2
                roof["gathered_bytes_per_launch"] = int(gb)
                roof["gather_tbs"] = round(gb / (avg_ms / 1e3) / 1e12, 3)
    launches = int(sum(v[0] for v in stats.values()))
    if not stats and hasattr(wl, "graph_step"):
        # the step is one CUDA graph: its kernels are not timed one by one, so
        # the roofline covers the whole step
        byt, nl = wl.graph_step()
        fl = wl.graph_flops()
        ach = fl / (ms / 1e3) / 1e12
        if wl.dtype == "df64":   # double-float pairs: rated against HBM, not the FP64 rate
            ach = byt / (ms / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": "moments_graph (whole step)", "achieved": round(ach, 1),
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                    "peak_source": src, "avg_launch_ms": round(ms, 4), "algorithmic_bytes_per_launch": int(byt),
                    "includes": "every kernel of the graph", "traffic": None, "share_of_step": 1.0}
        else:
            roof = {"bound": "alu", "kernel": "moments_graph (whole step)", "achieved": round(ach, 4),
                    "peak": round(fp64_peak, 4), "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                    "peak_source": fp64_src, "avg_launch_ms": round(ms, 4),
                    "algorithmic_flops_per_launch": int(fl),
                    "hbm_gbs_on_algorithmic_bytes": round(byt / (ms / 1e3) / 1e9, 1),
                    "includes": "every kernel of the graph", "traffic": None, "share_of_step": 1.0}
        launches = nl * args.steps

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
    wl = make_workload(args)
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


def make_workload(args):
    cls = WORKLOADS[args.workload]
    kw = {}
    if args.scale is not None:
        if cls not in (EstradaLearned, EstradaRmat22):
            raise SystemExit("--scale applies to the estrada_learned and estrada_rmat22 workloads only")
        kw["scale"] = args.scale
    if args.precision is not None:
        if cls not in (NuclearGram, NuclearExplicit, Stencil3D, EstradaLearned, EstradaHutchpp, Diffusion64Batched,
                       EstradaRmat22):
            raise SystemExit("--precision applies to estrada_rmat22, nuclear_gram, stencil3d, estrada_learned, "
                             "estrada_hutchpp and diffusion64_batched only")
        if cls is EstradaRmat22 and args.precision not in ("df64", "fp64", "fp32"):
            raise SystemExit("estrada_rmat22 takes df64, fp64 or fp32")
        if cls is Diffusion64Batched and args.precision not in ("fp64", "df64"):
            raise SystemExit("diffusion64_batched takes fp64 or df64")
        if cls is EstradaHutchpp and args.precision not in ("fp32", "fp64", "df64"):
            raise SystemExit("estrada_hutchpp takes fp32 (the sketch), fp64 (all) or df64 (fp32 sketch, "
                             "double-float moments)")
        if cls is EstradaLearned and args.precision not in ("fp32", "fp64"):
            raise SystemExit("estrada_learned takes fp32 or fp64")
        kw["precision"] = args.precision
    if cls is EstradaRmat22 and getattr(args, "no_comparison", False):
        kw["compare"] = False
    return cls(**kw)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="estrada_rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "df64", "mixed"])
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale of estrada_learned / estrada_rmat22")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparison", action="store_true",
                    help="estrada_rmat22: skip the learned-vs-plain comparison in setup")
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
