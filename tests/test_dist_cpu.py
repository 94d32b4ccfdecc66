"""The multi-rank path of bench.py on CPU: two gloo ranks run the same
barrier and max-over-ranks that time a weak-scaling run, and every
workload's per-rank probe ranges are disjoint (the ranks' samples are
independent) and inside the library's 2^32 probe ids for eight ranks.
Probes are independent samples (Section 4, Eq. multiEstimator), so the data
path has no collective; only the timing is reduced."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    d = bench.Dist()
    try:
        d.barrier()
        m = d.max(1.5 + rank)        # e.g. per-rank step times
        d.barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%d %d %r %d\n" % (d.rank, d.world, m, bench.probe_base(rank)))
    finally:
        d.close()


def test_two_gloo_ranks_barrier_and_max(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("the CPU path is what this covers")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = {}
    for r in range(2):
        rank, world, m, base = (tmp_path / ("rank%d.txt" % r)).read_text().split()
        got[int(rank)] = (int(world), float(m), int(base))
    assert got[0][0] == got[1][0] == 2
    assert got[0][1] == got[1][1] == 2.5           # both ranks see the slowest rank's time
    assert got[0][2] != got[1][2]


def test_probe_ranges_disjoint_for_eight_ranks():
    import bench
    for name, cls in bench.WORKLOADS.items():
        span = cls.PROBE_SPAN
        assert 0 <= span <= 1 << bench.PROBE_BASE_SHIFT, name
        ranges = [(bench.probe_base(r), bench.probe_base(r) + span) for r in range(8)]
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 <= b0, name
        assert ranges[-1][1] <= 1 << 32, name


# ---- the sharded multilevel estimator (paper_2103_10516_gb300.shard) ---------

def _grid():
    from paper_2103_10516_gb300 import synth
    return synth.grid_laplacian_2d(12, shift=0.1)


def _oracle_moments(g):
    import oracle
    return lambda off, deg: oracle.moments(g, 0.1, 8.1, 7, off, deg)


AUTO = dict(m_pilot=6, mode="budget", target=700.0)
FIXED = dict(levels=[6, 20, 40], m=[23, 9, 4])


def _shard_main(rank, world, port, out_dir):
    import json
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2103_10516_gb300 import shard
        g = _grid()
        res = {"auto": shard.mlmc_sharded(_oracle_moments(g), "log", 0.1, 8.1, 40, **AUTO),
               "fixed": shard.mlmc_sharded(_oracle_moments(g), "log", 0.1, 8.1, 40, **FIXED)}
        with open(os.path.join(out_dir, "shard%d.json" % rank), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_mlmc_equals_one_process(tmp_path, world, O):
    """Multilevel estimates split over gloo ranks, with the oracle standing in
    for each rank's moment kernels: rank 0's pilot and level selection are
    broadcast, every rank takes a contiguous part of the fresh probe ids and the
    band samples are gathered in id order.  Every rank must report exactly the
    one-process estimate, standard error, levels and counts (same probes, same
    samples, same order), and that estimate must agree with the oracle's own
    multilevel estimator on the same probe ids."""
    import json
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_2103_10516_gb300 import build, shard
    build.build()
    g = _grid()
    one = {"auto": shard.mlmc_sharded(_oracle_moments(g), "log", 0.1, 8.1, 40, **AUTO),
           "fixed": shard.mlmc_sharded(_oracle_moments(g), "log", 0.1, 8.1, 40, **FIXED)}
    port = _free_port()
    mp.start_processes(_shard_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        got = json.loads((tmp_path / ("shard%d.json" % r)).read_text())
        for key in ("auto", "fixed"):
            for f in ("estimate", "stderr", "levels", "m", "level_mean", "level_var", "probes", "matvecs"):
                np.testing.assert_array_equal(np.asarray(got[key][f]), np.asarray(one[key][f]),
                                              err_msg="%d %s %s" % (r, key, f))   # NaN == NaN
            assert got[key]["ranks"] == world
    ref = O.mlmc_auto(g, "log", 0.1, 8.1, 40, seed=7, **AUTO)
    tol = 1e-12 * sum(abs(v) for v in ref["coeffs"]) * g.nrows
    assert one["auto"]["levels"] == ref["levels"] and one["auto"]["m"] == ref["m"]
    assert abs(one["auto"]["estimate"] - ref["estimate"]) <= tol
    assert abs(one["auto"]["stderr"] - ref["stderr"]) <= 1e-9 * ref["stderr"]
    reff = O.mlmc_fixed(g, "log", 0.1, 8.1, 40, FIXED["levels"], FIXED["m"], seed=7)
    assert abs(one["fixed"]["estimate"] - reff["estimate"]) <= tol


def test_split_range_covers_every_item():
    from paper_2103_10516_gb300.shard import split_range
    for count in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            parts = [split_range(count, r, world) for r in range(world)]
            assert parts[0][0] == 0
            for (s0, n0), (s1, _) in zip(parts, parts[1:]):
                assert s0 + n0 == s1
            assert sum(n for _, n in parts) == count
            assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
