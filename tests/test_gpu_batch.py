"""Batched stepping (lbm_batch_*): many boxes of uneven size in one persistent
launch per step, relabel periods replayed as CUDA graphs. Each box must end
bitwise where it ends when stepped alone."""
import numpy as np
import pytest

import inputs
from paper_1708_01613_gb300 import Batch, LbmError, Simulation, make_config

pytestmark = pytest.mark.gpu

RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
# the last two: rows the staged kernel cannot copy (nx % 16 != 0); the batch
# steps them with the plain-load kernel in the same sequence
SIZES = [(256, 256), (320, 192), (528, 64), (1024, 96), (80, 48), (250, 100), (131, 77)]


def make_box(nx, ny, storage, barrier, K, seed):
    bub = inputs.poisson_disk_bubbles(nx, ny, 3, 6.0, min(14.0, 0.2 * min(nx, ny)), 2.0, seed=seed)
    sim = Simulation(make_config(nx, ny, storage=storage, barrier=barrier, relabel_every=K, rho_ref=RL))
    sim.init_bubbles(bub, RL, RG, 4.0)
    return sim


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_boxes_alone_bitwise(storage, graph):
    K, steps = 3, 11
    alone = [make_box(nx, ny, storage, True, K, 100 + i) for i, (nx, ny) in enumerate(SIZES)]
    for s in alone:
        s.step(steps)
    boxes = [make_box(nx, ny, storage, True, K, 100 + i) for i, (nx, ny) in enumerate(SIZES)]
    b = Batch(boxes)
    b.use_graph(graph)
    b.step(4)
    b.step(steps - 4)
    b.sync()
    assert b.steps_done == steps and b.kernel_launches > 0
    b.close()
    for s, a in zip(boxes, alone):
        assert s.steps_done == steps
        got = s.read("pops", "mask")
        ref = a.read("pops", "mask")
        assert np.array_equal(got["pops"], ref["pops"]), (s.nx, s.ny)
        assert np.array_equal(got["mask"], ref["mask"])


def test_batch_tiles_tune_and_activity():
    storage = "f16"
    boxes = [make_box(nx, ny, storage, True, 2, 200 + i) for i, (nx, ny) in enumerate(SIZES)]
    ref = [make_box(nx, ny, storage, True, 2, 200 + i) for i, (nx, ny) in enumerate(SIZES)]
    b = Batch(boxes)
    ms = b.tune(trial_steps=1)
    strip, rows = b.tiles
    assert ms > 0 and strip in (256, 512) and rows % 8 == 0
    tuned = b.steps_done
    assert tuned == 20  # ten candidates x (1 + 1) steps
    for s in ref:
        s.step(tuned)
    # box 1 sits out 5 steps; the others advance
    b.set_active(1, False)
    b.step(5)
    b.sync()
    for i, (s, r) in enumerate(zip(boxes, ref)):
        if i != 1:
            r.step(5)
    for s, r in zip(boxes, ref):
        assert np.array_equal(s.read("pops")["pops"], r.read("pops")["pops"])
    # box 1 rejoins 5 steps behind the others: each box keeps its own
    # relabel phase, and all stay bitwise equal to their lone runs
    b.set_active(1, True)
    for strip, rows in ((256, 16), (512, 40)):
        b.set_tiles(strip, rows)
        b.step(7)
    b.sync()
    for r in ref:
        r.step(14)
    for s, r in zip(boxes, ref):
        assert np.array_equal(s.read("pops", "mask")["pops"], r.read("pops")["pops"])
    with pytest.raises(LbmError):
        b.set_tiles(384, 16)
    b.close()


def test_batch_rules():
    a = make_box(256, 64, "f32", True, 1, 1)
    c = make_box(256, 64, "f16", True, 1, 2)
    with pytest.raises(LbmError):
        Batch([a, c])  # mixed storage
    d = Simulation(make_config(100, 64))
    d.init_density(np.full((64, 100), 0.7))
    alone = Simulation(make_config(100, 64))
    alone.init_density(np.full((64, 100), 0.7))
    bd = Batch([d])  # rows the staged kernel cannot copy: stepped by the plain kernel
    bd.step(3)
    bd.sync()
    bd.close()
    alone.step(3)
    assert np.array_equal(d.read("pops")["pops"], alone.read("pops")["pops"])
    b = Batch([a])
    with pytest.raises(LbmError):
        a.step(1)  # a batched box is stepped through its batch
    b.close()
    a.step(1)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_step_each_multi_rate_bitwise(storage):
    """Boxes advancing different step counts in one call (prefix launches,
    per-box relabel phases), mixed with common steps and a switched-off box,
    end bitwise where the lone runs end."""
    K = 3
    boxes = [make_box(nx, ny, storage, True, K, 300 + i) for i, (nx, ny) in enumerate(SIZES)]
    ref = [make_box(nx, ny, storage, True, K, 300 + i) for i, (nx, ny) in enumerate(SIZES)]
    b = Batch(boxes)
    plan = [[7, 0, 3, 12, 1, 5, 2], [2, 5, 5, 0, 9, 1, 6]]
    b.step_each(plan[0])
    b.step(4)
    b.set_active(3, False)
    b.step_each(plan[1])
    with pytest.raises(LbmError):
        b.step_each([1] * len(SIZES))  # box 3 is switched off
    b.sync()
    total = [p0 + 4 + p1 for p0, p1 in zip(*plan)]
    assert b.steps_done == 12 + 4 + 9
    for s, r, n in zip(boxes, ref, total):
        r.step(n)
        assert s.steps_done == n
        assert np.array_equal(s.read("pops")["pops"], r.read("pops")["pops"]), (s.nx, s.ny)
        assert np.array_equal(s.read("mask")["mask"], r.read("mask")["mask"])
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_step_one_between_batch_steps_bitwise(storage):
    """A box advanced alone inside its batch (lbm_batch_step_one: the
    single-box path) between multi-rate and graph-replayed batch steps ends
    bitwise where its lone run ends, and so do the boxes around it."""
    K = 3
    boxes = [make_box(nx, ny, storage, True, K, 500 + i) for i, (nx, ny) in enumerate(SIZES)]
    ref = [make_box(nx, ny, storage, True, K, 500 + i) for i, (nx, ny) in enumerate(SIZES)]
    b = Batch(boxes)
    plan = [[4, 0, 3, 7, 1, 5, 2], [2, 5, 5, 1, 3, 1, 6]]
    extra = {2: 5, 5: 4, 6: 1}
    b.step_each(plan[0])
    for i, n in extra.items():
        b.step_one(i, n)
    b.step(4)
    b.step_one(0, 2)
    b.step_each(plan[1])
    with pytest.raises(LbmError):
        b.step_one(len(SIZES), 1)
    b.sync()
    for i, (s, r) in enumerate(zip(boxes, ref)):
        n = plan[0][i] + extra.get(i, 0) + 4 + (2 if i == 0 else 0) + plan[1][i]
        r.step(n)
        assert s.steps_done == n
        assert np.array_equal(s.read("pops")["pops"], r.read("pops")["pops"]), (s.nx, s.ny)
        assert np.array_equal(s.read("mask")["mask"], r.read("mask")["mask"])
    b.close()


ORACLE_SIZES = [(160, 80), (256, 128), (192, 96), (96, 64), (150, 90)]


@pytest.mark.parametrize("storage,K,steps", [("f32", 3, 30), ("f16", 10, 50)])
def test_batch_matches_oracle(storage, K, steps):
    """A batch of four boxes of mixed size (barrier on, bubbles 2 cells
    apart, so walls and rupture are active) against one FP64 oracle run per
    box: FP32 populations within 1e-5, FP16 deviation storage within 2e-3 on
    rho; blocked-edge masks equal for FP32."""
    import oracle as O

    boxes, refs = [], []
    for i, (nx, ny) in enumerate(ORACLE_SIZES):
        R = 0.2 * ny
        bub = [[nx / 2 - R - 1.0, ny / 2, R], [nx / 2 + R + 1.0, ny / 2, R]]
        P = O.make_params(nx, ny, barrier=True, relabel_every=K)
        rho0 = O.init_bubbles(P, bub, RL, RG, 4.0)
        ref = O.OracleSim(P)
        ref.init_density(rho0)
        refs.append(ref)
        sim = Simulation(make_config(nx, ny, storage=storage, barrier=True, relabel_every=K,
                                     rho_ref=float(np.mean(rho0))))
        sim.init_density(rho0)
        boxes.append(sim)
    b = Batch(boxes)
    b.step(steps)
    b.sync()
    b.close()
    for s, ref in zip(boxes, refs):
        ref.step(steps)
        if storage == "f32":
            got = s.read("pops", "mask")
            err = float(np.max(np.abs(got["pops"] - ref.f)) / np.max(np.abs(ref.f)))
            assert np.array_equal(got["mask"], ref.mask) and ref.opened_total >= 0
            tol = 1e-5
        else:
            rho = ref.fields()["rho"]
            err = float(np.max(np.abs(s.read("rho")["rho"] - rho)) / np.max(np.abs(rho)))
            tol = 2e-3
        print(f"batch {storage} K={K} {s.nx}x{s.ny} step {steps}: rel err {err:.3e}, "
              f"blocked edges {int(np.count_nonzero(ref.mask))}")
        assert err < tol, (s.nx, s.ny, err)
    assert any(np.count_nonzero(r.mask) for r in refs)
