"""Nucleation and growth (Sec. 2.1.3) on the GPU against the FP64 oracle:
nuclei bit-exact, the growth source within the storage tolerance, the
released total exactly, and mass = initial + released."""
import numpy as np
import pytest

import inputs
import oracle as O
from paper_1708_01613_gb300 import Batch, LbmError, Simulation, make_config

pytestmark = pytest.mark.gpu

RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
TOL = {"f32": 1e-5, "f16": 2e-3}


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def pair(nx, ny, rho, *, storage="f32", barrier=True, K=4, rate=0.0, budget=0.0):
    sim = Simulation(make_config(nx, ny, storage=storage, barrier=barrier, relabel_every=K,
                                 rho_ref=float(np.mean(rho)), growth=True))
    sim.init_density(rho)
    if rate > 0 or budget > 0:
        sim.set_growth(rate, budget)
    orc = O.OracleSim(O.make_params(nx, ny, barrier=barrier, relabel_every=K, growth_rate=rate,
                                    growth_budget=budget))
    orc.init_density(rho)
    return sim, orc


def test_nucleation_bit_exact():
    nx, ny = 96, 64
    rho = np.full((ny, nx), RL)
    sim, orc = pair(nx, ny, rho, barrier=False)
    nuclei = [[0.5, 0.0, 3.0], [50.25, 31.5, 6.0], [95.0, 63.0, 2.0], [20.0, 40.0, 0.0]]
    sim.nucleate(nuclei, RG)
    orc.nucleate(nuclei, RG)
    got = sim.read("pops")["pops"]
    assert np.array_equal(got, orc.f.astype(np.float32))
    assert (orc.f[0] == O.lattice()[2][0] * RG).sum() > 100


@pytest.mark.parametrize("storage,barrier", [("f32", True), ("f32", False)])
def test_growth_matches_oracle(storage, barrier):
    """Two bubbles of radius 20 with a 6-cell film (the stable hand case),
    fed by the blowing agent until the budget is spent."""
    nx, ny, R, gap = 160, 80, 20, 6.0
    b = [[nx / 2 - R - gap / 2, ny / 2, R], [nx / 2 + R + gap / 2, ny / 2, R]]
    rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    sim, orc = pair(nx, ny, rho, storage=storage, barrier=barrier, rate=0.05, budget=3.75)
    m0 = sim.mass()
    for n in (1, 9, 90):
        sim.step(n)
        orc.step(n)
        assert sim.growth_released == orc.injected  # same FP64 sequence of releases
        if storage == "f32":
            err = rel_inf(sim.read("pops")["pops"], orc.f)
        else:  # 16-bit storage: the density error (its tolerance is stated on rho)
            err = rel_inf(sim.read("rho")["rho"], orc.fields()["rho"])
        print(f"{storage} barrier={barrier} step {sim.steps_done}: rel err {err:.3e}")
        assert err < TOL[storage]
    assert orc.injected == pytest.approx(3.75, abs=1e-12)  # 75 releases of 0.05
    if storage == "f32":
        assert abs(sim.mass() - (m0 + sim.growth_released)) < 1e-5 * m0


def test_nucleation_schedule_with_growth():
    """Random nuclei appear at their steps while the blowing agent releases
    gas; GPU and oracle follow the same schedule."""
    nx, ny = 128, 96
    rho = np.full((ny, nx), RL)
    sim, orc = pair(nx, ny, rho, barrier=True, K=5, rate=0.3, budget=40.0)
    sched = inputs.nucleation_schedule(nx, ny, 6, 120, 6.0, 10.0, seed=3)
    t = 0
    for step, cx, cy, r in list(sched) + [(200.0, 0.0, 0.0, 0.0)]:
        sim.step(int(step) - t)
        orc.step(int(step) - t)
        t = int(step)
        if t < 200:
            sim.nucleate([[cx, cy, r]], RG)
            orc.nucleate([[cx, cy, r]], RG)
    assert sim.steps_done == 200
    err = rel_inf(sim.read("pops")["pops"], orc.f)
    assert err < 1e-4, err  # nuclei's sharp fronts amplify rounding over 200 steps
    assert sim.growth_released == orc.injected > 0


def test_growth_waits_for_a_census_and_rules():
    nx, ny = 64, 32
    b = [[32.0, 16.0, 8.0]]
    rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    sim, _ = pair(nx, ny, rho, K=4)
    sim.step(3)
    sim.set_growth(0.25, 10.0)
    assert sim.growth_released == 0.0
    sim.step(1)  # step 3: no census since the call
    assert sim.growth_released == 0.0
    sim.step(1)  # step 4: census, then a release
    assert sim.growth_released == 0.25
    sim.step(3)
    assert sim.growth_released == 1.0
    with pytest.raises(LbmError):
        sim.set_growth(-1.0, 1.0)
    plain = Simulation(make_config(nx, ny, barrier=True, relabel_every=4))
    plain.init_density(rho)
    with pytest.raises(LbmError):
        plain.set_growth(0.1, 1.0)  # created without room for the source
    g = Simulation(make_config(64, 32, storage="f16", barrier=True, relabel_every=4, growth=True))
    g.init_density(rho)
    with pytest.raises(LbmError) as e:
        Batch([g])
    assert e.value.code == 6
    with pytest.raises(LbmError):
        sim.nucleate([[1.0, 1.0, -2.0]], RG)
    with pytest.raises(LbmError) as e:
        g.set_growth(0.1, 1.0)  # 16-bit deviations cannot hold the per-step increments
    assert e.value.code == 6


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_nucleation_16bit(storage):
    """Nuclei in 16-bit deviation storage: the density matches the oracle
    within the storage tolerance right after nucleation and 10 steps on."""
    nx, ny = 96, 64
    rho = np.full((ny, nx), RL)
    sim, orc = pair(nx, ny, rho, storage=storage, barrier=True)
    nuclei = [[30.0, 30.0, 9.0], [70.0, 20.0, 7.0]]
    sim.nucleate(nuclei, RG)
    orc.nucleate(nuclei, RG)
    tol = 2e-3 if storage == "f16" else 2e-2
    assert rel_inf(sim.read("rho")["rho"], orc.fields()["rho"]) < tol
    sim.step(10)
    orc.step(10)
    assert rel_inf(sim.read("rho")["rho"], orc.fields()["rho"]) < tol
