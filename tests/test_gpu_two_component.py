"""Two-component variant (melt and gas lattices, Sec. 2.1.5) on the GPU
against the FP64 oracle: populations within the FP32 tolerance, barrier
state bit-exact, fields, conservation, and the rules of the mode."""
import numpy as np
import pytest

import inputs
import oracle as O
from paper_1708_01613_gb300 import Batch, LbmError, Simulation, make_config

pytestmark = pytest.mark.gpu

RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def pair(nx, ny, rm, rg, **kw):
    gpu_kw = dict(tau=kw.get("tau_m", 1.0), tau_g=kw.get("tau_g", 1.0), G=kw.get("G_mm", -5.5),
                  G_mg=kw.get("G_mg", 0.0), G_gg=kw.get("G_gg", 0.0), barrier=kw.get("barrier", False),
                  relabel_every=kw.get("relabel_every", 1), rupture_eps=kw.get("rupture_eps", 1e-6))
    sim = Simulation(make_config(nx, ny, components=2, **gpu_kw))
    sim.init_density(rm, rg)
    orc = O.OracleSim2(O.make_params2(nx, ny, **kw))
    orc.init_density(rm, rg)
    return sim, orc


def both(orc):
    return np.concatenate([orc.fm, orc.fg])


@pytest.mark.parametrize("nx,ny", [(96, 64), (300, 70), (37, 9), (320, 64), (784, 24)])
@pytest.mark.parametrize("taus", [(1.0, 0.8), (1.0, 1.0)])
def test_mixture_parity(nx, ny, taus):
    """Demixing mixture (melt cohesion, melt-gas repulsion): plain-load
    kernel (96, 300, 37 columns) and staged kernel (320, 784: full strips
    and a ragged one), unequal and unit relaxation times."""
    a = inputs.noise_density(nx, ny, seed=11, rho_mean=0.7)
    b = inputs.noise_density(nx, ny, seed=12, rho_mean=0.6)
    sim, orc = pair(nx, ny, a, b, tau_m=taus[0], tau_g=taus[1], G_mm=-1.0, G_mg=2.5, G_gg=-0.3)
    for n in (1, 9, 40):
        sim.step(n)
        orc.step(n)
        err = rel_inf(sim.read("pops")["pops"], both(orc))
        print(f"{nx}x{ny} step {sim.steps_done}: rel err {err:.3e}")
        assert err < 1e-5


@pytest.mark.parametrize("nx,ny,last", [(160, 80, 90), (352, 80, 90), (170, 77, 40)])
def test_two_bubbles_with_barrier_parity(nx, ny, last):
    """Plain (160 columns) and staged (352) kernels with the barrier mask; a
    box with ragged relabel tiles (170 x 77, whose film ruptures within 10
    steps, after which rounding differences grow faster: checked to step
    50)."""
    R, gap = 12, 3.0
    b = [[nx / 2 - R - gap / 2, ny / 2, R], [nx / 2 + R + gap / 2, ny / 2, R]]
    rm = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    rg = 0.005 + 0.3 * (RL - rm) / (RL - RG)
    sim, orc = pair(nx, ny, rm, rg, G_mm=-5.5, G_mg=1.0, barrier=True, relabel_every=1)
    walls = 0
    for n in (1, 9, last):
        sim.step(n)
        orc.step(n)
        got = sim.read("pops", "mask", "owner")
        err = rel_inf(got["pops"], both(orc))
        print(f"two bubbles step {sim.steps_done}: rel err {err:.3e}, blocked cells {int(np.count_nonzero(orc.mask))}")
        assert err < 1e-5
        assert np.array_equal(got["mask"], orc.mask) and np.array_equal(got["owner"], orc.owner)
        walls += int(np.count_nonzero(orc.mask))
    assert walls > 0  # a wall stood at one of the checked steps at least
    f = orc.fields()
    g = sim.read("rho", "rho_gas", "ux", "uy", "p")
    assert rel_inf(g["rho"], f["rho_m"]) < 1e-5 and rel_inf(g["rho_gas"], f["rho_g"]) < 1e-5
    assert rel_inf(g["p"], f["p"]) < 1e-5
    umax = max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max())
    assert np.abs(g["ux"] - f["ux"]).max() < 1e-4 * umax + 1e-7
    assert np.abs(g["uy"] - f["uy"]).max() < 1e-4 * umax + 1e-7


def test_empty_gas_lattice_matches_one_component_box():
    nx, ny, R, gap = 160, 80, 20, 6.0
    b = [[nx / 2 - R - gap / 2, ny / 2, R], [nx / 2 + R + gap / 2, ny / 2, R]]
    rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    two = Simulation(make_config(nx, ny, components=2, barrier=True, relabel_every=5, G_mg=1.0))
    two.init_density(rho, np.zeros_like(rho))
    one = Simulation(make_config(nx, ny, barrier=True, relabel_every=5))
    one.init_density(rho)
    two.step(100)
    one.step(100)
    p2 = two.read("pops")["pops"]
    assert not p2[9:].any()
    assert rel_inf(p2[:9], one.read("pops")["pops"]) < 1e-5
    assert np.array_equal(two.read("mask")["mask"], one.read("mask")["mask"])


def test_mass_conservation_and_rules():
    n = 128
    a = inputs.noise_density(n, n, seed=21, rho_mean=0.7)
    b = inputs.noise_density(n, n, seed=22, rho_mean=0.7)
    sim = Simulation(make_config(n, n, components=2, G=0.0, G_mg=3.0))
    sim.init_density(a, b)
    m0 = sim.mass()
    assert m0 == pytest.approx(a.sum() + b.sum(), rel=1e-6)
    sim.step(500)
    assert abs(sim.mass() - m0) < 2e-5 * m0
    with pytest.raises(LbmError):
        Simulation(make_config(n, n, components=2, storage="f16"))
    with pytest.raises(LbmError):
        Simulation(make_config(100, 64, components=2, barrier=True, zone_radius=17))  # tiled relabel: R_z <= 16
    with pytest.raises(LbmError) as e:
        sim.init_bubbles([[10.0, 10.0, 5.0]], RL, RG, 4.0)
    assert e.value.code == 6
    with pytest.raises(LbmError) as e:
        Batch([sim])
    assert e.value.code == 6
    with pytest.raises(LbmError):
        sim.init_density(a)  # the gas density is required
