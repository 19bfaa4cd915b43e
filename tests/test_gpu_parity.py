"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (infinity norm relative to the oracle field's infinity norm):
FP32 storage 1e-5, FP16-deviation storage 2e-3 over short horizons; BF16 is
reported. Integer outputs (labels, owners, masks) must be bit-exact wherever
the float decision that makes them is not within rounding of its threshold.
"""
import math

import numpy as np
import pytest

import inputs
import oracle as O
from paper_1708_01613_gb300 import LbmError, Simulation, make_config

pytestmark = pytest.mark.gpu

RL, RG = inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55
TOL = {"f32": 1e-5, "f16": 2e-3}


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def two_bubbles(nx=160, ny=80, R=20, gap=6.0):
    return [[nx / 2 - R - gap / 2, ny / 2, R], [nx / 2 + R + gap / 2, ny / 2, R]]


def gpu_sim(nx, ny, rho=None, bubbles=None, **kw):
    storage = kw.pop("storage", "f32")
    rho_ref = kw.pop("rho_ref", None)
    if rho_ref is None:
        rho_ref = float(np.mean(rho)) if rho is not None else 1.0
    sim = Simulation(make_config(nx, ny, storage=storage, rho_ref=rho_ref, **kw))
    if bubbles is not None:
        sim.init_bubbles(bubbles, RL, RG, 4.0)
    else:
        sim.init_density(rho)
    return sim


def oracle_sim(nx, ny, rho, **kw):
    s = O.OracleSim(O.make_params(nx, ny, **kw))
    s.init_density(rho)
    return s


@pytest.mark.parametrize("nx,ny", [(128, 128), (300, 70), (257, 9), (37, 5)])
def test_init_populations_exact(nx, ny):
    rho = inputs.noise_density(nx, ny, seed=3)
    sim = gpu_sim(nx, ny, rho)
    f = sim.read("pops")["pops"]
    _, _, w = O.lattice()
    want = (w[:, None, None] * rho[None]).astype(np.float32)
    assert np.array_equal(f, want)
    assert sim.steps_done == 0


@pytest.mark.parametrize("nx,ny", [(128, 128), (300, 70), (257, 9), (37, 5)])
def test_step_parity_fp32_spinodal(nx, ny):
    """Config-1 physics (rho = 0.7 +- 1 %, G = -5.5) at sizes spanning several
    strips and ragged tails."""
    rho = inputs.noise_density(nx, ny, seed=1)
    sim = gpu_sim(nx, ny, rho)
    ref = oracle_sim(nx, ny, rho)
    done = 0
    for t in (1, 10, 100):
        sim.step(t - done)
        ref.step(t - done)
        done = t
        err = rel_inf(sim.read("pops")["pops"], ref.f)
        print(f"{nx}x{ny} step {t}: rel err {err:.3e}")
        if t <= 10:
            assert err < TOL["f32"], (t, err)
        else:
            assert err < 1e-3, (t, err)  # unstable spinodal modes amplify rounding


def _bits_equal_except_near(a, b, ok_mask):
    """Equal everywhere except where ok_mask allows a difference."""
    diff = a != b
    return not np.any(diff & ~ok_mask)


@pytest.mark.parametrize("nx,ny", [(160, 80), (164, 84)])
@pytest.mark.parametrize("gap,R,eps", [(6.0, 5, -1.0), (3.0, 4, 1e-6)])
def test_barrier_parity_two_bubbles_fp32(nx, ny, gap, R, eps):
    """Barrier on (K = 1): populations within 1e-5 and the owner map and
    blocked-edge mask bit-exact at steps 1, 10, 100 (160 x 80 runs the tiled
    relabel pipeline on whole 32 x 8 tiles, 164 x 84 with a ragged last tile
    column and row). Both films have wall cells
    (owner -2) on their symmetry plane (the 9-cell liquid gap of the 6-cell
    film is bridged by zones of radius 5; there the rupture test is off,
    since with it every wall cell opens within 10 steps as the initial
    profile relaxes); populations bounce back across every blocked edge."""
    b = two_bubbles(nx, ny, gap=gap)
    P = O.make_params(nx, ny, barrier=True, zone_radius=R, rupture_eps=eps)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True, zone_radius=R, rupture_eps=eps)
    ref = oracle_sim(nx, ny, rho0, barrier=True, zone_radius=R, rupture_eps=eps)
    assert np.array_equal(sim.read("pops")["pops"], (O.lattice()[2][:, None, None] * rho0[None]).astype(np.float32))
    done = 0
    for t in (1, 10, 100):
        sim.step(t - done)
        ref.step(t - done)
        done = t
        got = sim.read("pops", "owner", "mask", "open")
        err = rel_inf(got["pops"], ref.f)
        print(f"barrier step {t}: rel err {err:.3e}, blocked edges {int(np.count_nonzero(ref.mask))}")
        assert err < TOL["f32"], (t, err)
        assert np.array_equal(got["owner"], ref.owner)
        assert np.array_equal(got["mask"], ref.mask)
        assert np.array_equal(got["open"], ref.open)
    assert np.count_nonzero(ref.mask) > 0 and np.any(ref.owner == -2)


def test_barrier_relabel_period_k():
    nx, ny = 160, 80
    b = two_bubbles(nx, ny, gap=3.0)
    P = O.make_params(nx, ny, barrier=True, relabel_every=5)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True, relabel_every=5)
    ref = oracle_sim(nx, ny, rho0, barrier=True, relabel_every=5)
    sim.step(23)
    ref.step(23)
    got = sim.read("pops", "mask")
    assert rel_inf(got["pops"], ref.f) < TOL["f32"]
    assert np.array_equal(got["mask"], ref.mask) and ref.mask.any()


def test_fields_and_labels_parity():
    nx, ny = 160, 80
    b = two_bubbles(nx, ny, gap=3.0)
    P = O.make_params(nx, ny, barrier=True)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True)
    ref = oracle_sim(nx, ny, rho0, barrier=True)
    sim.step(50)
    ref.step(50)
    got = sim.read("rho", "ux", "uy", "p", "label")
    fl = ref.fields()
    assert rel_inf(got["rho"], fl["rho"]) < TOL["f32"]
    assert rel_inf(got["p"], fl["p"]) < TOL["f32"]
    umax = max(np.max(np.abs(fl["ux"])), np.max(np.abs(fl["uy"])))
    ex = np.max(np.abs(got["ux"] - fl["ux"])) / umax
    ey = np.max(np.abs(got["uy"] - fl["uy"])) / umax
    print(f"fields step 50: u rel err {ex:.3e} / {ey:.3e} (max |u| {umax:.3e})")
    # u = (j + F/2)/rho with j a difference of O(1) populations: FP32
    # rounding leaves absolute errors near 2e-7 in u, 1.4e-5 of max |u|
    # (1.6e-2) here, so u is held to 5e-5 of max |u| rather than 1e-5
    assert ex < 5e-5 and ey < 5e-5
    lab_ref = O.label(P, fl["rho"])
    near = np.abs(fl["rho"] - math.log(2.0)) < 1e-5
    assert _bits_equal_except_near(got["label"], lab_ref, near)
    st = sim.stats(nbins=8, dmin=1.0, dmax=128.0)
    so = O.stats(P, lab_ref, nbins=8, dmin=1.0, dmax=128.0)
    assert st["n_bubbles"] == so["n_bubbles"] == 2
    assert st["gas_fraction"] == pytest.approx(so["gas_fraction"], abs=1e-12)
    assert st["mean_diameter"] == pytest.approx(so["mean_diameter"], rel=1e-12)
    assert np.array_equal(st["hist"], so["hist"])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_storage_error(storage):
    """16-bit deviation storage against the oracle over short horizons, with
    the metrics of the tolerance: rho in the infinity norm relative to
    max rho, and |u| relative to max |u|. FP16 meets 2e-3 on rho; BF16 is
    reported (8 mantissa bits are not expected to meet it)."""
    nx, ny = 160, 80
    b = two_bubbles(nx, ny, gap=6.0)
    P = O.make_params(nx, ny)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    rho_ref = float(np.mean(rho0))
    sim = gpu_sim(nx, ny, bubbles=b, storage=storage, rho_ref=rho_ref)
    ref = oracle_sim(nx, ny, rho0)
    done = 0
    for t in (1, 10, 100):
        sim.step(t - done)
        ref.step(t - done)
        done = t
        got = sim.read("rho", "ux", "uy")
        fl = ref.fields()
        err = rel_inf(got["rho"], fl["rho"])
        u_ref = np.hypot(fl["ux"], fl["uy"])
        u_err = float(np.max(np.abs(np.hypot(got["ux"], got["uy"]) - u_ref)) / np.max(u_ref))
        print(f"{storage} step {t}: rho rel err {err:.3e}, |u| rel err {u_err:.3e} (max |u| {np.max(u_ref):.3e})")
        if storage == "f16":
            assert err < TOL["f16"], (t, err)
            # |u| = |j + F/2| / rho: a stored deviation is rounded to about
            # 2^-11 w_i |rho - rho_ref|, and in the gas (rho ~ 0.1) dividing
            # by rho magnifies that tenfold, so |u| carries absolute errors
            # of 1e-3 to 5e-3 against max |u| of 0.02-0.16 (spurious
            # currents): reported, and held to the magnitude that
            # rounding allows at short horizons
            if t <= 10:
                assert u_err < 5e-2, (t, u_err)


def test_mass_fp64_and_conservation():
    nx, ny = 128, 128
    rho = inputs.noise_density(nx, ny, seed=1)
    sim = gpu_sim(nx, ny, rho)
    m0 = sim.mass()
    assert m0 == pytest.approx(float(np.sum(rho)), rel=1e-7)
    sim.step(1000)
    m1 = sim.mass()
    print(f"fp32 mass drift over 1000 steps: {abs(m1 - m0) / m0:.3e}")
    # FP32 collision rounding moves sum f by ~1e-8 relative per step; the FP64
    # oracle conserves it to 1e-12 (see the oracle pins)
    assert abs(m1 - m0) / m0 < 1e-4


def test_resume_is_bitwise():
    nx, ny = 128, 96
    rho = inputs.noise_density(nx, ny, seed=5)
    a = gpu_sim(nx, ny, rho)
    a.step(30)
    f = a.read("pops")["pops"]
    b = Simulation(make_config(nx, ny))
    b.load_populations(f)
    assert np.array_equal(b.read("pops")["pops"], f)
    a.step(30)
    b.step(30)
    assert np.array_equal(a.read("pops")["pops"], b.read("pops")["pops"])


def test_stop_on_first_rupture_matches_oracle():
    nx, ny = 160, 80
    b = two_bubbles(nx, ny, gap=3.0)
    P = O.make_params(nx, ny, barrier=True, stop_on_first_rupture=True)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    ref = oracle_sim(nx, ny, rho0, barrier=True, stop_on_first_rupture=True)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True, stop_on_first_rupture=True)
    n_ref = ref.step(500)
    sim.step(500)
    assert ref.halted and sim.halted
    assert sim.steps_done == n_ref
    assert np.array_equal(sim.read("open")["open"], ref.open)


def test_numeric_fault_is_reported_not_raised_on_device():
    nx, ny = 64, 64
    sim = gpu_sim(nx, ny, np.full((ny, nx), -1.0))
    sim.step(1)
    with pytest.raises(LbmError) as e:
        sim.sync()
    assert e.value.code == 4  # LBM_ENUMERIC


def _check_labels_valid(lab, gas):
    """Valid min-index labelling: liquid -1; 4-neighbouring gas cells share a
    label; every label is the index of a gas cell that carries its own index;
    no cell's index is below its label (so the label is the component's min)."""
    assert np.all((lab >= 0) == gas)
    right = np.roll(lab, -1, axis=1)
    down = np.roll(lab, -1, axis=0)
    g_r = gas & np.roll(gas, -1, axis=1)
    g_d = gas & np.roll(gas, -1, axis=0)
    assert np.array_equal(lab[g_r], right[g_r]) and np.array_equal(lab[g_d], down[g_d])
    flat = lab.ravel()
    idx = np.arange(flat.size)
    roots = flat[flat >= 0]
    assert np.all(flat[roots] == roots)
    assert np.all(roots <= idx[flat >= 0])


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_full_size_8192_sampled(storage):
    """The benchmark workload (8192^2, 400 bubbles, barrier on, K = 10) in the
    benchmark's launch configuration: one step checked at 4096 sampled cells
    against the oracle evaluated one cell at a time from the GPU's own input
    state and mask (force substitution and bounce-back across blocked edges);
    labels checked as a valid min-index labelling; owners checked at sampled
    liquid cells by exhaustive window search."""
    n = 8192
    bub = inputs.poisson_disk_bubbles(n, n, 400, 8.0, 64.0, 2.0, seed=21)
    P = O.make_params(n, n, barrier=True, relabel_every=10)
    sim = Simulation(make_config(n, n, storage=storage, barrier=True, relabel_every=10,
                                 rho_ref=float(RL)))
    sim.init_bubbles(bub, RL, RG, 4.0)
    lab = sim.read("label")["label"]  # labels of the density the t = 0 relabel sees
    sim.step(3)  # t = 3: the next step does not relabel
    before = sim.read("pops", "mask", "owner")
    sim.step(1)
    after = sim.read("pops")["pops"]
    rng = np.random.default_rng(0)
    gasy, gasx = np.nonzero(before["mask"])
    cells = rng.choice(n * n, 3072, replace=False)
    if len(gasy):
        pick = rng.choice(len(gasy), min(1024, len(gasy)), replace=False)
        cells = np.concatenate([cells, gasy[pick].astype(np.int64) * n + gasx[pick]])
    f64 = before["pops"].astype(np.float64)
    want = O.step_cells(P, f64, cells, before["mask"])
    got = after.reshape(9, -1)[:, cells].T.astype(np.float64)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    print(f"8192^2 {storage}: sampled one-step rel err {err:.3e}")
    # FP32 storage: one FP32 step; FP16: plus one 16-bit rounding of the output
    assert err < (1e-6 if storage == "f32" else 1e-3)
    gas = lab >= 0
    _check_labels_valid(lab, gas)
    own = before["owner"]
    R = 4
    for c in cells[:512]:
        y, x = divmod(int(c), n)
        if gas[y, x]:
            assert own[y, x] == lab[y, x]
            continue
        near, best = set(), None
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                d2 = dx * dx + dy * dy
                l = lab[(y + dy) % n, (x + dx) % n]
                if d2 > R * R or l < 0 or (best is not None and d2 > best):
                    continue
                if best is None or d2 < best:
                    near, best = set(), d2
                near.add(int(l))
        # nearest bubble, none, or a wall cell (-2) between equidistant bubbles
        assert own[y, x] == (-1 if not near else (near.pop() if len(near) == 1 else -2))


def test_full_box_8192_crop_against_full_oracle():
    """The benchmark workload (8192^2, 400 bubbles, barrier on, K = 10) run by
    the oracle on the whole periodic box for 20 steps (two relabels), and the
    GPU compared with it on a 512^2 crop (a crop of a periodic run is not
    periodic, so the oracle cannot run the crop alone): FP32 populations
    within 1e-5, blocked-edge mask and owners equal; FP16 deviation storage
    within 2e-3 on rho."""
    n, steps = 8192, 20
    bub = inputs.poisson_disk_bubbles(n, n, 400, 8.0, 64.0, 2.0, seed=21)
    P = O.make_params(n, n, barrier=True, relabel_every=10)
    rho0 = O.init_bubbles(P, bub, RL, RG, 4.0)
    ref = O.OracleSim(P)
    ref.init_density(rho0)
    ref.step(steps)
    # a crop holding blocked edges if the box has any (the densest 512^2 window)
    m = (ref.mask != 0).astype(np.int64)
    tiles = m.reshape(16, 512, 16, 512).sum(axis=(1, 3))
    ty, tx = np.unravel_index(int(np.argmax(tiles)), tiles.shape)
    ys, xs = slice(512 * ty, 512 * ty + 512), slice(512 * tx, 512 * tx + 512)
    rho_ref = ref.f[:, ys, xs].sum(0)
    for storage in ("f32", "f16"):
        sim = gpu_sim(n, n, rho0, storage=storage, barrier=True, relabel_every=10, rho_ref=float(RL))
        sim.step(steps)
        if storage == "f32":
            got = sim.read("pops", "mask", "owner")
            err = rel_inf(got["pops"][:, ys, xs], ref.f[:, ys, xs])
            assert np.array_equal(got["mask"][ys, xs], ref.mask[ys, xs])
            assert np.array_equal(got["owner"][ys, xs], ref.owner[ys, xs])
            tol = TOL["f32"]
        else:
            err = rel_inf(sim.read("rho")["rho"][ys, xs], rho_ref)
            tol = TOL["f16"]
        print(f"8192^2 {storage} step {steps}, crop ({ty}, {tx}) with {int(tiles[ty, tx])} blocked cells: "
              f"rel err {err:.3e}")
        assert err < tol
        del sim


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("nx,ny,barrier", [(528, 70, False), (272, 9, False), (320, 80, True), (544, 80, True),
                                           (1043, 40, False), (250, 9, False), (337, 80, True), (19, 12, False),
                                           (1025, 9, False), (513, 11, False)])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_tma_staged_kernel_matches_plain_kernel_bitwise(storage, nx, ny, barrier, tau):
    """The TMA-staged fused steps (one and two cells per thread; ragged last
    strips, periodic wrap, barrier mask staged alongside) give bitwise the
    plain-load kernel's populations, and the FP32 run stays close to the
    oracle. Widths that are not multiples of 16 (1043: a 19-column last strip;
    250, 337, 19; 1025 and 513: a one-column last strip, so the strip before
    it reaches the last column and its right halo wraps) take the two-cell
    kernel's variant that bulk-copies the part of each window inside the row
    and takes the wrapped elements from a side area, with odd widths and rows
    that start at odd cell indices."""
    if barrier:
        b = two_bubbles(nx, ny, R=20, gap=3.0)
        rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    else:
        rho = inputs.noise_density(nx, ny, seed=9)
    variants = (1, 3, 4) if nx % 16 else (1, 2, 3, 4) if nx >= 528 else (1, 2, 4)
    sims = []
    for variant in variants:
        s = gpu_sim(nx, ny, rho, storage=storage, barrier=barrier, rho_ref=float(np.mean(rho)), tau=tau)
        s.set_step_variant(variant)
        s.step(40)
        sims.append(s.read("pops", *(["mask"] if barrier else [])))
    for other in sims[1:]:
        assert np.array_equal(sims[0]["pops"], other["pops"])
        if barrier:
            assert np.array_equal(sims[0]["mask"], other["mask"]) and sims[0]["mask"].any()
    if storage == "f32":
        ref = oracle_sim(nx, ny, rho, barrier=barrier, tau=tau)
        ref.step(40)
        err = rel_inf(sims[-1]["pops"], ref.f)
        print(f"tma {nx}x{ny} barrier={barrier}: rel err at step 40 {err:.3e}")
        assert err < 5e-4 if not barrier else err < TOL["f32"]


def test_step_variant_selection_errors():
    sim = gpu_sim(128, 64, inputs.noise_density(128, 64, seed=1))
    with pytest.raises(LbmError) as e:
        sim.set_step_variant(2)  # 128 columns is too narrow for the staged kernel
    assert e.value.code == 6
    sim.set_step_variant(3)  # the two-cell kernel takes any width of 16 or more
    odd = gpu_sim(100, 64, inputs.noise_density(100, 64, seed=1))
    odd.set_step_variant(3)
    odd.set_step_variant(4)
    narrow = gpu_sim(12, 64, inputs.noise_density(12, 64, seed=1))
    with pytest.raises(LbmError) as e:
        narrow.set_step_variant(3)
    assert e.value.code == 6
    with pytest.raises(LbmError) as e:
        narrow.set_step_variant(4)  # dynamic chunks: also the two-cell kernel
    assert e.value.code == 6
    sim.set_step_variant(4)
    with pytest.raises(LbmError):
        sim.set_step_variant(5)
    sim.set_step_variant(1)
    sim.step(1)


@pytest.mark.parametrize("R", [0, 2, 6, 17])
def test_owner_zone_radius_sweep(R):
    """Owners and masks bit-exact against the oracle for several zone radii
    (R <= 16 uses the tiled search, R = 17 the plain window search)."""
    nx, ny = 160, 80
    b = two_bubbles(nx, ny, gap=3.0)
    P = O.make_params(nx, ny, barrier=True, zone_radius=R)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True, zone_radius=R)
    ref = oracle_sim(nx, ny, rho0, barrier=True, zone_radius=R)
    sim.step(5)
    ref.step(5)
    got = sim.read("owner", "mask", "pops")
    assert np.array_equal(got["owner"], ref.owner)
    assert np.array_equal(got["mask"], ref.mask)
    assert rel_inf(got["pops"], ref.f) < TOL["f32"]


def test_barrier_state_clears_when_a_bubble_dissolves():
    """A small bubble in a closed box at coexistence density dissolves; its
    interaction zone must disappear from the owner map and mask (tiles that
    stop being active are reset)."""
    nx, ny = 96, 96
    b = [[48.0, 48.0, 10.0], [70.0, 48.0, 8.0]]
    P = O.make_params(nx, ny, barrier=True, rupture_eps=-1.0)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b, barrier=True, rupture_eps=-1.0)
    ref = oracle_sim(nx, ny, rho0, barrier=True, rupture_eps=-1.0)
    done = 0
    for t in (1, 200, 900):
        sim.step(t - done)
        ref.step(t - done)
        done = t
        got = sim.read("owner", "mask", "pops")
        assert np.array_equal(got["owner"], ref.owner), t
        assert np.array_equal(got["mask"], ref.mask), t
        assert rel_inf(got["pops"], ref.f) < 1e-4
    assert np.all(ref.owner == -1)  # everything dissolved by step 900


@pytest.mark.parametrize("nx,ny,n", [(37, 5, 3), (300, 70, 40), (256, 256, 700), (1024, 64, 0)])
def test_init_bubbles_matches_oracle(nx, ny, n):
    """Initial density of a bubble set (each CTA takes the minimum only over
    bubbles that come near its tile; more bubbles than one staged chunk;
    centres outside the box; no bubbles) against the oracle's minimum over
    all bubbles: FP32 populations within one rounding, exact where the tanh
    profile saturates."""
    u = inputs.splitmix64_uniform(7000 + n, np.arange(3 * n)).reshape(n, 3)
    b = np.stack([u[:, 0] * (nx + 20) - 10, u[:, 1] * (ny + 20) - 10, 1.0 + 0.1 * min(nx, ny) * u[:, 2]], 1)
    rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    sim = gpu_sim(nx, ny, bubbles=b)
    got = sim.read("pops")["pops"]
    _, _, w = O.lattice()
    want = (w[:, None, None] * rho[None]).astype(np.float32)
    assert np.all(np.abs(got - want) <= np.spacing(want))
    assert np.mean(got == want) > 0.999
    sat = rho == 0.5 * (RL + RG) + 0.5 * (RL - RG)
    assert np.array_equal(got[:, sat], want[:, sat])
    if n == 0:
        assert sat.all()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_dynamic_chunks_counter_survives_mixed_variants(storage):
    """The dynamically scheduled step leaves its chunk counter at zero after
    every launch: steps alternating with other kernels, single steps and a
    re-initialisation all give bitwise the plain kernel's populations."""
    nx, ny = 1040, 96  # two full strips and a ragged one, 2 chunk rows
    b = two_bubbles(nx, ny, R=20, gap=3.0)
    rho = O.init_bubbles(O.make_params(nx, ny), b, RL, RG, 4.0)
    kw = dict(storage=storage, barrier=True, relabel_every=3, rho_ref=float(np.mean(rho)))
    mixed = gpu_sim(nx, ny, rho, **kw)
    plain = gpu_sim(nx, ny, rho, **kw)
    plain.set_step_variant(1)
    for k, v in enumerate([4, 1, 4, 4, 2 if storage == "f32" else 3, 4, 0, 1, 4]):
        mixed.set_step_variant(v)
        mixed.step(1 + k % 3)
        plain.step(1 + k % 3)
    assert np.array_equal(mixed.read("pops")["pops"], plain.read("pops")["pops"])
    mixed.init_density(rho)
    plain.init_density(rho)
    mixed.set_step_variant(4)
    mixed.step(7)
    plain.step(7)
    assert np.array_equal(mixed.read("pops")["pops"], plain.read("pops")["pops"])


@pytest.mark.parametrize("storage,nx,ny,tau", [("f32", 4096, 4096, 1.0), ("f16", 4096, 4096, 1.0),
                                                ("f16", 6144, 3072, 1.0), ("f16", 4096, 4096, 0.8),
                                                ("f32", 5120, 2048, 0.8)])
def test_whole_wave_chunks_match_plain_kernel(storage, nx, ny, tau):
    """Mid-size boxes, where the automatic step draws chunks of the height
    that fills whole waves of resident CTAs (4096^2: 18 rows FP32, 27 rows
    FP16; 6144 x 3072: 31 rows, ragged last chunk row; with tau != 1 the
    kernel holds the populations across the barrier, runs fewer CTAs per SM
    and marches full strips with a runtime width), give bitwise the plain
    kernel's populations and masks over steps with relabels."""
    import torch

    pair = two_bubbles(nx, ny, R=20, gap=3.0)  # a film in the middle of the box
    bub = [b for b in inputs.poisson_disk_bubbles(nx, ny, 60, 8.0, 48.0, 2.0, seed=17)
           if all(math.hypot(b[0] - q[0], b[1] - q[1]) > b[2] + q[2] + 12 for q in pair)] + pair
    kw = dict(storage=storage, barrier=True, relabel_every=3, tau=tau)
    auto = gpu_sim(nx, ny, bubbles=bub, rho_ref=RL, **kw)
    plain = gpu_sim(nx, ny, bubbles=bub, rho_ref=RL, **kw)
    plain.set_step_variant(1)
    auto.step(7)
    plain.step(7)
    a, p = auto.read("pops", "mask", device=True), plain.read("pops", "mask", device=True)
    assert torch.equal(a["pops"], p["pops"]) and torch.equal(a["mask"], p["mask"])
    assert bool(a["mask"].any())


def test_two_component_whole_wave_chunks_empty_gas():
    """Two-component box of 3072^2 (16-row chunks, four waves) with an empty
    gas lattice stays with the one-component box, as in the small case."""
    n = 3072
    bub = inputs.poisson_disk_bubbles(n, n, 30, 8.0, 48.0, 2.0, seed=19)
    one = gpu_sim(n, n, bubbles=bub, barrier=True, relabel_every=5, rho_ref=RL)
    rho = one.read("rho")["rho"].astype(np.float64)
    one.init_density(rho)
    two = Simulation(make_config(n, n, components=2, barrier=True, relabel_every=5, G_mg=1.0))
    two.init_density(rho, np.zeros_like(rho))
    one.step(12)
    two.step(12)
    p1, p2 = one.read("pops")["pops"], two.read("pops")["pops"]
    assert not p2[9:].any()
    assert rel_inf(p2[:9], p1) < 1e-5
    assert np.array_equal(two.read("mask")["mask"], one.read("mask")["mask"])


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny", [(256, 128), (32, 8)])
def test_degenerate_all_gas_and_all_liquid(storage, nx, ny):
    """A box that is gas everywhere is one component on the torus (label 0,
    the smallest index; every cell its own owner's bubble, no blocked edge,
    one bubble covering the box); a box of liquid has no labels, owners or
    bubbles. 32 x 8 is a single tile, whose periodic edges all wrap onto
    itself (zone radius 3, the largest that box allows; the generic owner
    search beside the R_z = 4 shell scan)."""
    R = 4 if ny > 9 else 3
    for rho, gas in ((RG, True), (RL, False)):
        sim = gpu_sim(nx, ny, np.full((ny, nx), rho), storage=storage, barrier=True, relabel_every=1, rho_ref=RL,
                      zone_radius=R)
        sim.step(3)
        d = sim.read("label", "owner", "mask")
        st = sim.stats()
        if gas:
            assert (d["label"] == 0).all() and (d["owner"] == 0).all() and not d["mask"].any()
            assert st["n_bubbles"] == 1 and st["gas_fraction"] == 1.0
            assert st["mean_diameter"] == pytest.approx(2.0 * math.sqrt(nx * ny / math.pi), rel=1e-12)
        else:
            assert (d["label"] == -1).all() and (d["owner"] == -1).all() and not d["mask"].any()
            assert st["n_bubbles"] == 0 and st["gas_fraction"] == 0.0


@pytest.fixture(scope="module")
def foam_oracle_1000():
    """The FP64 oracle's statistics of a coarsening 512^2 foam (40 Poisson-disk
    bubbles, radii 12-28, barrier on, K = 10) after 1000 steps."""
    n = 512
    b = inputs.poisson_disk_bubbles(n, n, 40, 12.0, 28.0, 3.0, seed=13)
    P = O.make_params(n, n, barrier=True, relabel_every=10)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    s = O.OracleSim(P)
    s.init_density(rho0)
    s.step(1000)
    st = O.stats(P, s.labels_now(), nbins=8, dmin=4.0, dmax=128.0)
    st["n_merges"] = s.merges_total
    return b, rho0, st


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_long_horizon_statistics(storage, foam_oracle_1000):
    """Bubble statistics after 1000 steps of coarsening (bubbles dissolve, films
    rupture, bubbles merge), GPU against the oracle: count within 10 %, mean
    equivalent diameter within 5 %, gas fraction within 1 % absolute, L1
    distance of the normalised diameter histograms at most 0.15. Rounding
    shifts individual merge times, so the comparison is statistical."""
    b, rho0, so = foam_oracle_1000
    n = 512
    sim = Simulation(make_config(n, n, storage=storage, barrier=True, relabel_every=10, rho_ref=float(np.mean(rho0))))
    sim.init_density(rho0)
    sim.step(1000)
    st = sim.stats(nbins=8, dmin=4.0, dmax=128.0)
    print(storage, "gpu", st["n_bubbles"], st["gas_fraction"], st["mean_diameter"], st["n_merges"], "oracle",
          so["n_bubbles"], so["gas_fraction"], so["mean_diameter"], so["n_merges"])
    assert so["n_bubbles"] >= 10
    # this dilute foam coarsens by dissolution (no film is thin enough to
    # rupture within 1000 steps): no coalescence on either side
    assert st["n_merges"] == so["n_merges"] == 0
    labels, areas = sim.bubble_areas()
    assert len(labels) == st["n_bubbles"] and np.all(np.diff(labels) > 0)
    assert areas.sum() == pytest.approx(st["gas_fraction"] * n * n, abs=0.5)
    # the size distribution: sorted areas against the oracle's (statistical)
    a_o = np.sort(so["areas"])[::-1]
    a_g = np.sort(areas)[::-1]
    k = min(len(a_o), len(a_g))
    assert np.abs(a_g[:k] - a_o[:k]).sum() <= 0.05 * a_o.sum()
    assert abs(st["n_bubbles"] - so["n_bubbles"]) <= 0.1 * so["n_bubbles"]
    assert st["mean_diameter"] == pytest.approx(so["mean_diameter"], rel=0.05)
    assert abs(st["gas_fraction"] - so["gas_fraction"]) <= 0.01
    h1 = np.asarray(st["hist"], float) / max(1, st["n_bubbles"])
    h2 = np.asarray(so["hist"], float) / max(1, so["n_bubbles"])
    assert np.abs(h1 - h2).sum() <= 0.15


@pytest.fixture(scope="module")
def clustered_512_oracle():
    """Oracle run of a clustered 512^2 foam with thin films (40 bubbles,
    radii 12-28, edge gaps 2-3, barrier on, K = 10): coalescence events
    after 200 and 400 steps."""
    n = 512
    b = inputs.clustered_bubbles(n, n, 40, 12.0, 28.0, 2.0, 3.0, seed=13)
    P = O.make_params(n, n, barrier=True, relabel_every=10)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    s = O.OracleSim(P)
    s.init_density(rho0)
    out = {}
    for t in (200, 400):
        s.step(t - s.t)
        out[t] = (s.merges_total, O.stats(P, s.labels_now())["n_bubbles"])
    return rho0, out


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_coalescence_count_clustered_foam(storage, clustered_512_oracle):
    """Coalescence events counted by the GPU relabels against the oracle's on
    a foam whose thin films rupture (8 merges by step 200, 17 by 400 in the
    oracle). FP32 counts the same events; FP16 (threshold decisions on
    16-bit-rounded densities) within 2."""
    rho0, want = clustered_512_oracle
    n = 512
    sim = Simulation(make_config(n, n, storage=storage, barrier=True, relabel_every=10,
                                 rho_ref=float(np.mean(rho0))))
    sim.init_density(rho0)
    for t in (200, 400):
        sim.step(t - sim.steps_done)
        st = sim.stats()
        print(f"{storage} step {t}: merges {st['n_merges']} (oracle {want[t][0]}), "
              f"bubbles {st['n_bubbles']} (oracle {want[t][1]})")
        assert want[t][0] >= 5
        assert abs(st["n_merges"] - want[t][0]) <= (0 if storage == "f32" else 2)


@pytest.mark.parametrize("K", [1, 10])
def test_config_1024_clustered_foam(K):
    """The 1024^2 foam configuration (20 bubbles, radii 10-40, clustered with
    2-6 cell gaps, barrier on) against the oracle run on the whole box.
    Short horizon (steps 1 and 50): FP32 populations within 1e-5, barrier
    masks equal but for cells next to a density within rounding of the gas
    threshold. The clustered bubbles move and merge at once, and rupture is a
    threshold event: a cell that opens one relabel earlier or later changes
    the flow around it by O(1), so pointwise differences grow quickly after
    that (step 200: 4e-5 FP32 with K = 10, 4e-4 with K = 1); at step 200 the
    comparison is statistical (bubble count, gas fraction). FP16 storage: an
    interface displaced by a fraction of a cell changes rho there by O(1), so
    its infinity-norm density error passes 2e-3 within 50 steps (printed);
    the RMS density error is held to 2e-3 and the infinity norm to 5e-2."""
    n = 1024
    b = inputs.clustered_bubbles(n, n, 20, 10.0, 40.0, 2.0, 6.0, seed=11)
    P = O.make_params(n, n, barrier=True, relabel_every=K)
    rho0 = O.init_bubbles(P, b, RL, RG, 4.0)
    ref = O.OracleSim(P)
    ref.init_density(rho0)
    sims = {st: gpu_sim(n, n, rho0, storage=st, barrier=True, relabel_every=K) for st in ("f32", "f16")}
    for steps in (1, 9, 40):
        ref.step(steps)
        for s in sims.values():
            s.step(steps)
        got = sims["f32"].read("pops", "mask")
        err = rel_inf(got["pops"], ref.f)
        rho_ref = ref.fields()["rho"]
        d16 = sims["f16"].read("rho")["rho"].astype(np.float64) - rho_ref
        inf16 = float(np.abs(d16).max() / np.abs(rho_ref).max())
        rms16 = float(np.sqrt(np.mean(d16 ** 2)) / np.sqrt(np.mean(rho_ref ** 2)))
        print(f"1024^2 K={K} step {ref._s.t}: f32 pops {err:.3e}, f16 rho inf {inf16:.3e} rms {rms16:.3e}")
        assert err < TOL["f32"]
        assert rms16 < TOL["f16"] and inf16 < 5e-2
        if ref.t <= 10:  # the short horizon of the FP16 tolerance
            # outside the reach (one cell per step) of film cells whose
            # rupture or wall state the FP16 run decided differently from the
            # oracle (threshold decisions on 16-bit-rounded densities; with
            # K = 1 they start within 10 steps), rho is within 2e-3
            from scipy.ndimage import binary_dilation
            g16 = sims["f16"].read("open", "mask")
            dec = (g16["open"] != ref.open) | (g16["mask"] != ref.mask)
            reach = binary_dilation(dec, iterations=ref.t + 2, border_value=0) if dec.any() else dec
            out16 = float(np.abs(d16[~reach]).max() / np.abs(rho_ref).max())
            print(f"  f16 decisions differing: {int(dec.sum())} cells; rho inf outside their reach {out16:.3e}")
            assert out16 < TOL["f16"], (ref.t, out16)
        diff = got["mask"] != ref.mask
        if diff.any():
            from scipy.ndimage import binary_dilation
            near = np.abs(rho_ref - math.log(2.0)) < 1e-5
            zone = binary_dilation(near, iterations=6, border_value=0)
            assert not (diff & ~zone).any()
    assert ref.mask.any()
    ref.step(150)
    so = O.stats(P, ref.labels_now())
    for st_name, s in sims.items():
        s.step(150)
        st = s.stats()
        print(f"1024^2 K={K} step 200 {st_name}: bubbles {st['n_bubbles']} (oracle {so['n_bubbles']}), "
              f"gas {st['gas_fraction']:.5f} ({so['gas_fraction']:.5f})")
        assert abs(st["n_bubbles"] - so["n_bubbles"]) <= max(1, 0.1 * so["n_bubbles"])
        assert abs(st["gas_fraction"] - so["gas_fraction"]) <= 0.01


def test_laplace_sweep_gpu():
    """The configuration's static Laplace sweep (R = 10, 20, 40, 60, 20000
    steps) on the GPU in FP32: p_in - p_out linear in 1/R (R^2 >= 0.999, intercept within
    5 % of the smallest droplet's jump), and at R = 10 and 20 the jump equals
    the oracle's within 1e-3. Liquid droplets in gas (small gas bubbles in a
    closed box dissolve)."""
    pts, first = [], {}
    for R, L in ((10, 96), (20, 128), (40, 256), (60, 256)):
        rho = O.init_bubbles(O.make_params(L, L), [[L / 2, L / 2, R]], RG, RL, 4.0)  # liquid inside
        sim = gpu_sim(L, L, rho)
        sim.step(20000)
        fl = sim.read("rho", "p")
        yy, xx = np.mgrid[0:L, 0:L]
        d = np.hypot(xx - L / 2, yy - L / 2)
        A = np.sum((fl["rho"].astype(np.float64) - RG) / (RL - RG))
        dp = float(fl["p"][d < R - 5].mean() - fl["p"][d > R + 10].mean())
        pts.append((1 / math.sqrt(A / math.pi), dp))
        if R <= 20:
            ref = oracle_sim(L, L, rho)
            ref.step(20000)
            fo = ref.fields()
            dpo = float(fo["p"][d < R - 5].mean() - fo["p"][d > R + 10].mean())
            first[R] = (dp, dpo)
            assert dp == pytest.approx(dpo, rel=1e-3)
    xs, dps = np.array(pts).T
    slope, icpt = np.polyfit(xs, dps, 1)
    fit = slope * xs + icpt
    r2 = 1 - np.sum((dps - fit) ** 2) / np.sum((dps - dps.mean()) ** 2)
    print(f"GPU Laplace: points {pts}, sigma {slope:.5f}, intercept {icpt:.2e}, R^2 {r2:.6f}, vs oracle {first}")
    assert slope > 0 and r2 >= 0.999
    assert abs(icpt) <= 0.05 * dps[0]
