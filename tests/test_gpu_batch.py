"""Batched persistent launch: many cells of different sizes, walls and
parameters in one cooperative launch per run of steps (and CUDA-graph
replays of such runs) give the same populations, bit for bit, as the same
cells stepped one launch at a time; the schedule autotuner keeps that; a
grid-barrier wait that runs out of its budget is reported, not hung on."""
import numpy as np
import pytest

from paper_1903_08882_gb300 import inputs

pytestmark = pytest.mark.gpu

CELLS = [  # (nx, ny, nz, walls, Ra, Pr)
    ((9, 7, 8), "side", 1e4, 0.71),
    ((33, 33, 33), "rb", 1e5, 7.0),
    ((17, 21, 19), "side", 1e5, 0.71),
    ((5, 5, 40), "rb", 1e4, 0.71),
    ((49, 31, 27), "side", 1e6, 7.0),
]


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_08882_gb300 import _build
    from paper_1903_08882_gb300 import lbm as L

    _build.build()
    return L


def _make(lbm, storage="fp32"):
    lats = []
    for k, (n, kind, Ra, Pr) in enumerate(CELLS):
        walls = lbm.walls_side_heated() if kind == "side" else lbm.walls_rayleigh_benard()
        # the batched kernel runs the register kernels' tile code: step the
        # single-cell references with those kernels for a bitwise comparison
        lat = lbm.Lattice(*n, walls, Ra=Ra, Pr=Pr, storage=storage, pipeline="register")
        sh = (n[2], n[1], n[0])
        rho, u, T = inputs.random_fields(sh, 100 + k, du=0.02)
        lat.set_fields(rho, u, T)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("span", [1, 3])
@pytest.mark.parametrize("storage", ["fp32", "fp16s", "fp16m"])
def test_batch_matches_single_cells(lbm, storage, span):
    import torch

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ref = _make(lbm, storage)
        bat = _make(lbm, storage)
        for lat in ref:
            lat.step(37)
        with lbm.Batch(bat, stream=stream) as b:
            b.set_schedule(block_size=128, blocks_per_sm=2, steps_per_launch=5, graph_chunk=10, tile_span=span)
            b.step(37)  # three graph replays and seven steps launched directly
        for r, x in zip(ref, bat):
            fr, gr = r.populations()
            fx, gx = x.populations()
            assert np.array_equal(fr, fx) and np.array_equal(gr, gx)
            assert r.diagnostics()["step"] == x.diagnostics()["step"] == 37
        for lat in ref + bat:
            lat.close()


def test_batch_autotune_and_timeout(lbm):
    import torch

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bat = _make(lbm)
        ref = _make(lbm)
        with lbm.Batch(bat, stream=stream) as b:
            best = b.autotune(trial_steps=6)
            assert best["block_size"] in (128, 256) and best["blocks_per_sm"] >= 1
            assert b.schedule == best
            done = bat[0].diagnostics()["step"]
            for lat in ref:
                lat.step(done)
            b.step(20)
            for lat in ref:
                lat.step(20)
            for r, x in zip(ref, bat):
                assert np.array_equal(r.populations()[0], x.populations()[0])
            # a barrier budget of zero cycles: waits give up at once, the call reports it
            b.set_barrier_budget(0)
            with pytest.raises(lbm.LbmError) as ei:
                b.step(4)
            assert ei.value.status == lbm.LBM_ERR_TIMEOUT
            # the context is still usable: reset the states and step again
            b.set_barrier_budget(1 << 31)
            for k, lat in enumerate(bat):
                n = CELLS[k][0]
                lat.set_fields(1.0, np.zeros(3), 0.0)
            b.step(6)
            for lat in bat:
                lat.sample()
                assert not lat.diagnostics()["diverged"]
            # cells at different parities are refused
            bat[0].step(1)
            with pytest.raises(lbm.LbmError) as ei:
                b.step(2)
            assert ei.value.status == lbm.LBM_ERR_STATE
        for lat in ref + bat:
            lat.close()
