"""The reference arm of bench.py (the oracle timed on the host cores) keeps its
JSON contract, alone and under torchrun with two gloo ranks, where rank 0
alone runs and prints.  CPU only: the reference arm touches no GPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "logdet64", "--steps", "3", "--warmup", "3"]


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_line(d, n):
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "ms_per_step", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["n_gpus"] == n and d["steps"] == 3 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["config"]["workload"] == "logdet64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py"] + ARGS, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2"] + ARGS
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1          # rank 0 alone prints
    _check_line(lines[0], 2)


def test_roofline_byte_and_flop_models():
    # the per-launch algorithmic bytes of the recurrence step (survey 8(d)):
    # the matrix once (4 bytes a stored entry for a pattern, 8 (d + 1) of row
    # pointers) and, per live probe, V_k and V_{k-1} read and V_{k+1} written.
    # The default Estrada step (R-MAT scale 22, 128 probes to degree 128 in
    # double-float, two 64-probe groups of 64 launches) gives the 6.99 GB the
    # bench line reports; an FP64 step costs 2 flops a stored entry and 8 a
    # vector entry per probe-matvec.
    sys.path.insert(0, ROOT)
    import bench
    d, nnz = 1 << 22, 128_307_214
    got = bench.step_bytes(d, nnz, 4, 8, 128 * 64, {"cheb_step": 128})["cheb_step"]
    assert got == 4 * nnz + 8 * (d + 1) + 3 * d * 8 * 64 == 6_989_234_240
    # probes that retire early lower the average live width per launch
    got2 = bench.step_bytes(1000, 7000, 8, 8, 10 * 3 + 2 * 5, {"cheb_step": 5})["cheb_step"]
    assert got2 == 7000 * 8 + 8 * 1001 + 3 * 1000 * 8 * (40 / 5)
    assert bench.step_bytes(d, nnz, 4, 8, 10, {}) == {}
    assert bench.step_flops(4096, 20_224, 3) == 3 * (2 * 20_224 + 8 * 4096)


def test_learned_comparison_figure_of_merit():
    # the metric's comparison: at equal standard error the GPU time an
    # estimator needs scales with its variance, so the figure of merit is
    # (s^2 t)_plain / (s^2 t)_learned.  Hand example: plain FP64 s = 6, t = 5 s;
    # plain FP32 s = 6, t = 1 s; learned estimates with s = 3 and 5 (pooled
    # s^2 = 17) in 2 s each.  Training 9 s is repaid after 9 / (5 * 36/17 - 2)
    # estimates.
    sys.path.insert(0, ROOT)
    import bench
    cmp = {"plain_fp64": {"stderr": 6.0, "gpu_s": 5.0}, "plain_fp32": {"stderr": 6.0, "gpu_s": 1.0},
           "learned": {"train_gpu_s": 9.0}}
    bench.finish_comparison(cmp, [(10.0, 3.0), (11.0, 5.0)], 2.0, [7, 2])
    assert abs(cmp["learned"]["stderr"] ** 2 - 17.0) < 1e-12
    assert cmp["variance_time_gain"] == round(36 * 5 / (17 * 2), 3)
    assert cmp["variance_time_gain_vs_plain_fp32"] == round(36 * 1 / (17 * 2), 3)
    assert cmp["estimates_to_amortise_training"] == round(9 / (5 * 36 / 17 - 2), 1)
    assert cmp["learned"]["estimate_first"] == 10.0 and cmp["learned"]["estimates"] == 2
