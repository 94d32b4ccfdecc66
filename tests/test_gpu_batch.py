"""The persistent batch (mlt_batch_create / mlt_batch_run): one CUDA graph
built once for a set of moment jobs on matrices of uneven sizes with ragged
degrees, replayed with shifted probe ids.  Every replay must give the oracle's
moments of the shifted probes (FP64 tolerance 1e-10 d), for host and device
outputs; while the batch lives its handles refuse other calls, and after it is
destroyed they work again."""
import numpy as np
import pytest

from paper_2103_10516_gb300 import synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-10


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


def _jobs(O):
    rng = np.random.default_rng(1)
    g = synth.rmat_adjacency(9, 8, seed=2)
    cases = [(synth.grid_laplacian_2d(6, shift=0.1), 1.0), (synth.grid_laplacian_2d(13, shift=0.1), 1.0),
             (synth.random_symmetric(200, 0.05, seed=3, diag_shift=3.0), 1.0), (g, 0.05),
             (synth.diffusion_3d(12, sigma=1.0, shift=0.2, seed=4), 1.0)]
    out = []
    for k, (m, sc) in enumerate(cases):
        a, b = O.interval(m, scale=sc)
        deg = rng.integers(0, 60, size=20 + 13 * k).astype(np.int32)
        out.append((m, sc, a, b, 11 + k, 100 * k, deg))
    return out


def test_batch_replays_match_oracle(L, O):
    import torch
    cases = _jobs(O)
    mats = [L.Matrix(m, scale=sc) for m, sc, *_ in cases]
    outs = []
    for k, (m, sc, a, b, seed, off, deg) in enumerate(cases):
        shape = (deg.size, int(deg.max()) + 1)
        outs.append(np.zeros(shape) if k % 2 == 0 else torch.zeros(shape, dtype=torch.float64, device="cuda"))
    jobs = [{"matrix": M.handle, "a": a, "b": b, "seed": seed, "probe_offset": off, "degrees": deg, "out": o}
            for M, (m, sc, a, b, seed, off, deg), o in zip(mats, cases, outs)]
    try:
        with L.Batch(jobs) as B:
            for shift in (0, 5000, 0, 777):
                B.run(shift)
                torch.cuda.synchronize()
                for (m, sc, a, b, seed, off, deg), o in zip(cases, outs):
                    got = o if isinstance(o, np.ndarray) else o.cpu().numpy()
                    ref = O.moments(m, a, b, seed, off + shift, deg, scale=sc)
                    assert np.max(np.abs(got - ref)) <= TOL64 * m.nrows, (shift, m.nrows)
            # the handles belong to the batch: other calls are refused
            with pytest.raises(L.MLTError) as e:
                mats[0].moments(cases[0][2], cases[0][3], 1, 0, [4])
            assert e.value.code == L.MLT_EINVAL
            with pytest.raises(L.MLTError):
                L.mlt_autotune(mats[1].handle, "fp64", 2)
            with pytest.raises(L.MLTError):
                B.run(1 << 32)                     # probe ids beyond 2^32
        # released: the handles work again
        m, sc, a, b, seed, off, deg = cases[0]
        got = mats[0].moments(a, b, seed, off, deg)
        assert np.max(np.abs(got - O.moments(m, a, b, seed, off, deg, scale=sc))) <= TOL64 * m.nrows
    finally:
        for M in mats:
            M.close()


def test_batch_rejects_bad_jobs(L, O):
    m = synth.grid_laplacian_2d(5, shift=0.1)
    with L.Matrix(m) as M:
        out = np.zeros((3, 5))
        job = {"matrix": M.handle, "a": 0.1, "b": 8.1, "degrees": [4, 4, 4], "out": out}
        with pytest.raises(L.MLTError):
            L.Batch([job, dict(job)])              # the same handle twice
        with pytest.raises(L.MLTError):
            L.Batch([dict(job, a=9.0)])            # a >= b
        # a failed create leaves the handle free
        assert M.moments(0.1, 8.1, 0, 0, [4]).shape == (1, 5)
