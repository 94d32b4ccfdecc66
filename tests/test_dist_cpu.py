"""The multi-rank path of bench.py on CPU: two gloo ranks run the same
barrier and max-over-ranks that time a weak-scaling run, and every
workload's per-rank probe ranges are disjoint (the ranks' samples are
independent) and inside the library's 2^32 probe ids for eight ranks.
Probes are independent samples (Section 4, Eq. multiEstimator), so the data
path has no collective; only the timing is reduced."""
import os
import socket
import sys

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
