"""Batched engine: many cavities in one persistent launch.

Every slot of a batch must give exactly what a single-instance handle running
the same (general) kernel gives, retire at the same step on its own residual,
be unaffected by the other slots of the mix, and survive a diverging
neighbour; slots can be added and removed between launches.
"""
import numpy as np
import pytest

from oracle import stepper as S
from paper_2208_03562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2208_03562_gb300.lbm")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L.load()


MIX = [
    # nx, ny, r, gamma, nu, u_lid, bc, drho, fx
    (70, 19, 2.0, 0.1, 0.01, 0.02, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
    (130, 64, 0.5, 0.3, 0.01, 0.03, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
    (33, 40, 1.0, 1.0, 0.02, 0.05, L.BC_CHANNEL, L.DRHO_OFF, 1e-5),
    (96, 32, 0.25, 0.6, 0.002, 0.01, L.BC_PERIODIC, L.DRHO_CURRENT, 2e-6),
    (5, 7, 1.6, 0.2, 0.005, 0.01, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
]


def params(case, dtype):
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    return L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype, bc=bc, drho=drho, fx=fx)


def start_state(case, seed):
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
    return w[:, None, None] + I.noise(seed, (9, ny, nx), 1e-3)


def single(case, dtype, f0):
    h = L.Lbm(params(case, dtype))
    h.variant = -1  # the general kernel, as in the batch
    h.set_populations(f0)
    return h


@pytest.mark.parametrize("dtype", [L.F32, L.F64, L.F16])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_single_instances(dtype, use_graph):
    b = L.Batch(8, dtype)
    slots, refs = [], []
    for k, case in enumerate(MIX):
        f0 = start_state(case, 100 + k)
        s = b.add(params(case, dtype), 0.0, 10 ** 6)
        b.set_populations(s, f0)
        slots.append(s)
        refs.append(single(case, dtype, f0))
    for n in (7, 40):
        b.launch(n, use_graph)
        assert b.wait() == len(MIX)
        for s, h in zip(slots, refs):
            h.step(n)
            info, st = b.query(s)
            assert st == L.SLOT_ACTIVE and info.step == h.info().step
            assert np.array_equal(b.populations(s), h.populations())
            if info.residual_step:
                assert info.residual == h.residual() and info.mass == h.info().mass


def test_each_slot_retires_on_its_own_residual():
    cav = [I.Cavity(48, 24, 0.5, 0.5, 20.0, 0.02, "f32"), I.Cavity(40, 40, 1.0, 1.0, 50.0, 0.05, "f32"),
           I.Cavity(30, 60, 2.0, 0.25, 20.0, 0.02, "f32")]
    tols = [1e-6, 1e-5, 1e-7]
    b = L.Batch(4, L.F32)
    b.set_body(L.BATCH_BODY_GENERAL)
    slots = [b.add(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32), t, 500000)
             for c, t in zip(cav, tols)]
    active = len(slots)
    while active:
        active = b.run(5000)
    for c, t, s in zip(cav, tols, slots):
        info, st = b.query(s)
        assert st == L.SLOT_CONVERGED and info.residual < t
        h = L.Lbm(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32))
        h.variant = -1
        status, steps = h.run(t, 500000)
        assert status == L.OK and steps == info.step
        assert np.array_equal(b.populations(s), h.populations())


def test_alone_equals_in_mix():
    """The same request alone and inside a mix of 40 uneven cavities."""
    req = I.Cavity(77, 45, 0.5, 0.3, 100.0, 0.03, "f32", 1e-6)
    mk = lambda c: L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32)
    alone = L.Batch(1, L.F32)
    sa = alone.add(mk(req), req.tol, 40000)
    while alone.run(2000):
        pass
    mix = L.Batch(64, L.F32)
    others = I.batched_sweep(seed=3, n=40)
    for c in others[:20]:
        mix.add(mk(I.Cavity(min(c.nx, 200), min(c.ny, 100), c.r, max(c.gamma, 0.3), c.re, c.u_lid, "f32")),
                1e-30, 3000)
    sm = mix.add(mk(req), req.tol, 40000)
    for c in others[20:]:
        mix.add(mk(I.Cavity(min(c.nx, 150), min(c.ny, 90), c.r, max(c.gamma, 0.3), c.re, c.u_lid, "f32")),
                1e-30, 7000)
    while mix.run(2000):
        pass
    ia, sta = alone.query(sa)
    im, stm = mix.query(sm)
    assert sta == stm and ia.step == im.step and ia.residual == im.residual
    assert np.array_equal(alone.populations(sa), mix.populations(sm))


def test_diverging_slot_does_not_disturb_the_others():
    bad = I.deep_cavity_128_as_stated(0.1)
    good = I.Cavity(64, 32, 0.5, 0.5, 100.0, 0.03, "f32")
    mk = lambda c: L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32)
    b = L.Batch(4, L.F32)
    b.set_body(L.BATCH_BODY_GENERAL)
    sb = b.add(mk(bad), 1e-7, 4000)
    sg = b.add(mk(good), 1e-30, 1000)
    b.run(4000)
    assert b.query(sb)[1] == L.SLOT_DIVERGED
    info, st = b.query(sg)
    assert st == L.SLOT_MAXSTEPS and info.step == 1000
    h = L.Lbm(mk(good))
    h.variant = -1
    h.step(1000)
    assert np.array_equal(b.populations(sg), h.populations())


def test_add_and_remove_between_launches():
    mk = lambda nx, ny: L.lbm_params_init(nx, ny, 1.0, 0.5, 0.02, 0.03, L.F32)
    b = L.Batch(3, L.F32)
    b.set_body(L.BATCH_BODY_GENERAL)
    s0 = b.add(mk(40, 30), 1e-30, 10 ** 6)
    s1 = b.add(mk(50, 20), 1e-30, 10 ** 6)
    b.run(30)
    b.remove(s0)
    s2 = b.add(mk(64, 64), 1e-30, 10 ** 6)
    assert s2 == s0  # the freed slot is reused
    b.run(30)
    assert b.query(s1)[0].step == 60 and b.query(s2)[0].step == 30
    h = L.Lbm(mk(64, 64))
    h.variant = -1
    h.step(30)
    assert np.array_equal(b.populations(s2), h.populations())
    s3 = b.add(mk(20, 20), 1e-30, 10 ** 6)
    with pytest.raises(L.LbmError) as e:
        b.add(mk(20, 20), 1e-30, 10 ** 6)
    assert e.value.status == L.ENOMEM
    b.remove(s3)


@pytest.mark.parametrize("body", [L.BATCH_BODY_AUTO, L.BATCH_BODY_GENERAL])
def test_grid_barrier_wait_runs_out_and_reports_timeout(body):
    """Failure detection without a fault: the first CTA withholds its arrival
    at the first grid barrier (a flag that nothing clears), every other CTA's
    bounded wait runs out (limit about 1 ms), the launch ends with
    LBM_ETIMEOUT, no slot's state has moved, and the device and the batch
    stay usable: the next launch steps as if the failed one had not been.
    Both tile bodies (TMA-staged and general) share the barrier."""
    mk = lambda nx, ny: L.lbm_params_init(nx, ny, 0.5, 0.3, 0.01, 0.03, L.F32)
    b = L.Batch(2, L.F32)
    b.set_body(body)
    s0 = b.add(mk(64, 32), 1e-30, 10 ** 6)
    s1 = b.add(mk(200, 90), 1e-30, 10 ** 6)
    assert b.tma_body == (body == L.BATCH_BODY_AUTO)
    f0 = [b.populations(s) for s in (s0, s1)]
    b.set_wait_limit(2_000_000, hold=True)
    with pytest.raises(L.LbmError) as e:
        b.run(50)
    assert e.value.status == L.ETIMEOUT
    for s, f in zip((s0, s1), f0):
        info, st = b.query(s)
        assert st == L.SLOT_ACTIVE and info.step == 0
        assert np.array_equal(b.populations(s), f)
    assert b.run(40) == 2  # the default limit again, one launch only
    for s, (nx, ny) in zip((s0, s1), ((64, 32), (200, 90))):
        h = L.Lbm(mk(nx, ny))
        h.variant = 0 if body == L.BATCH_BODY_AUTO else L.VARIANT_GENERAL
        h.step(40)
        info, st = b.query(s)
        assert info.step == 40 and np.array_equal(b.populations(s), h.populations())
        h.close()


def test_wait_limit_rejects_negative_cycles():
    b = L.Batch(1, L.F32)
    with pytest.raises(L.LbmError) as e:
        b.set_wait_limit(-1)
    assert e.value.status == L.EINVAL


@pytest.mark.parametrize("dtype", [L.F32, L.F64])
def test_launch_shape_leaves_results_and_autotune_restores_state(dtype):
    """The persistent grid size changes how tiles are shared among CTAs, not
    what any slot computes; lbm_batch_autotune puts every slot back."""
    def make(cps):
        b = L.Batch(8, dtype)
        slots = []
        for k, case in enumerate(MIX):
            s = b.add(params(case, dtype), 0.0, 10 ** 6)
            b.set_populations(s, start_state(case, 400 + k))
            slots.append(s)
        if cps:
            b.ctas_per_sm = cps
        return b, slots
    a, sa = make(0)
    one, s1 = make(1)
    assert a.ctas_per_sm == a.max_ctas_per_sm >= 1 and one.ctas_per_sm == 1
    a.run(33)
    one.run(33)
    for x, y in zip(sa, s1):
        assert np.array_equal(a.populations(x), one.populations(y))
    before = [(a.populations(x), a.query(x)[0].step) for x in sa]
    best, ms = a.autotune(10)
    assert 1 <= best <= a.max_ctas_per_sm and a.ctas_per_sm == best
    assert len(ms) == a.max_ctas_per_sm and all(m > 0 for m in ms)
    for x, (p, step) in zip(sa, before):
        info, st = a.query(x)
        assert st == L.SLOT_ACTIVE and info.step == step
        assert np.array_equal(a.populations(x), p)
    a.run(27)
    one.run(27)
    for x, y in zip(sa, s1):
        assert np.array_equal(a.populations(x), one.populations(y))
        assert a.query(x)[0].step == one.query(y)[0].step == 60


def test_launch_shape_rejects_out_of_range():
    b = L.Batch(2, L.F32)
    m = b.max_ctas_per_sm
    for bad in (-1, m + 1):
        with pytest.raises(L.LbmError) as e:
            b.ctas_per_sm = bad
        assert e.value.status == L.EINVAL
    b.ctas_per_sm = 1
    b.ctas_per_sm = 0  # back to the default: the maximum
    assert b.ctas_per_sm == m
    best, ms = b.autotune(5)  # no active slot: nothing is timed
    assert best == m and all(v == -1.0 for v in ms)


@pytest.mark.parametrize("dtype", [L.F32, L.F16])
def test_specialised_kernel_equals_single_instances(dtype):
    """A mix with the density-gradient terms, no force and the central scheme
    everywhere runs the form of the batch kernel with the tile body fixed at
    compile time.  Grids of several tiles in both directions, one with a
    ragged last row and column of tiles and one smaller than a tile, must
    give exactly what single handles on the general kernel give."""
    cases = [  # nx, ny, r, gamma, nu, u_lid
        (300, 100, 0.5, 0.3, 0.01, 0.03),
        (200, 90, 2.0, 0.1, 0.01, 0.02),
        (134, 26, 1.0, 0.6, 0.02, 0.05),
        (70, 19, 1.0, 1.0, 0.02, 0.05),
        (517, 211, 0.25, 0.2, 0.005, 0.02),
    ]
    b = L.Batch(len(cases), dtype)
    b.set_body(L.BATCH_BODY_GENERAL)
    slots, refs = [], []
    for k, (nx, ny, r, gamma, nu, u) in enumerate(cases):
        p = L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype)
        w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
        f0 = w[:, None, None] + I.noise(700 + k, (9, ny, nx), 1e-3)
        s = b.add(p, 0.0, 10 ** 6)
        b.set_populations(s, f0)
        h = L.Lbm(p)
        h.variant = -1
        h.set_populations(f0)
        slots.append(s)
        refs.append(h)
    assert not b.tma_body
    for n in (1, 18, 41):  # crossing residual steps
        b.run(n)
        for s, h in zip(slots, refs):
            h.step(n)
            info, st = b.query(s)
            assert st == L.SLOT_ACTIVE and info.step == h.info().step
            assert np.array_equal(b.populations(s), h.populations())
            if info.residual_step:
                assert info.residual == h.residual() and info.mass == h.info().mass
    for h in refs:
        h.close()


# nx, ny, r, gamma, nu, u_lid: grids whose single-handle interior kernel has
# several interior tiles both ways with a shifted last tile column and row
# (300 x 100, 200 x 90, 517 x 211), a single interior tile row or column
# (134 x 26, 72 x 12 and 70 x 19 in FP32; the last two have none in FP16, whose
# tile origins align to 8 nodes), or none (33 x 40); in the batch body they
# cover tiles clear of the walls, wall tiles on every side and corner, odd
# widths (517, 33) and last rows and columns reaching past the grid
TMA_CASES = [
    (300, 100, 0.5, 0.3, 0.01, 0.03),
    (200, 90, 2.0, 0.1, 0.01, 0.02),
    (134, 26, 1.0, 0.6, 0.02, 0.05),
    (70, 19, 1.0, 1.0, 0.02, 0.05),
    (517, 211, 0.25, 0.2, 0.005, 0.02),
    (72, 12, 0.5, 0.5, 0.01, 0.02),
    (33, 40, 1.6, 0.4, 0.01, 0.02),
]


def batch_tile_variant(dtype):
    """The interior-kernel variant with the batch body's tile: 64 x 8 nodes,
    256 threads."""
    for v in range(L.lbm_variant_count(dtype)):
        if L.lbm_variant_info(dtype, v)[:3] == (64, 8, 256):
            return v
    raise AssertionError("no 64 x 8 interior-kernel variant")


@pytest.mark.parametrize("dtype", [L.F32, L.F16])
@pytest.mark.parametrize("use_graph", [True, False])
def test_tma_body_equals_single_instances_on_the_interior_kernel(dtype, use_graph):
    """The TMA-staged batch body runs, per node, what a single handle runs on
    the interior kernel with the same 64 x 8 tile: the staged pulls, the
    density ring, the gradients and the packed collision in tiles clear of
    the walls, and in tiles at a wall the wall-aware pulls from the taller
    staged windows, ring densities inside the grid and clamped gradients,
    where the handle takes the general tile body on its edge strips (and on
    the whole of a grid without interior tiles).  Every slot's populations
    must equal that handle's bitwise, with the step counts; the residual and
    mass sum the same node terms grouped by tile instead of by CTA, so they
    agree to FP64 round-off."""
    b = L.Batch(len(TMA_CASES), dtype)
    slots, refs = [], []
    for k, (nx, ny, r, gamma, nu, u) in enumerate(TMA_CASES):
        p = L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype)
        w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
        f0 = w[:, None, None] + I.noise(1700 + k, (9, ny, nx), 1e-3)
        s = b.add(p, 0.0, 10 ** 6)
        b.set_populations(s, f0)
        h = L.Lbm(p)
        h.variant = batch_tile_variant(dtype)
        h.set_populations(f0)
        slots.append(s)
        refs.append(h)
    assert b.tma_body
    for n in (1, 18, 41, 60):  # crossing residual steps
        b.launch(n, use_graph)
        assert b.wait() == len(TMA_CASES)
        for s, h in zip(slots, refs):
            h.step(n)
            info, st = b.query(s)
            assert st == L.SLOT_ACTIVE and info.step == h.info().step
            assert np.array_equal(b.populations(s), h.populations()), (b.shapes[s], info.step)
            if info.residual_step:
                hi = h.info()
                assert abs(info.residual - hi.residual) <= 1e-9 * hi.residual
                assert abs(info.mass - hi.mass) <= 1e-12 * hi.mass
    for h in refs:
        h.close()


# nx, ny, r, gamma, nu, u_lid: grids no larger than a tile or two, where every
# tile of the TMA-staged batch body is a wall tile: the smallest grid, a tile
# row shorter than the 8-row tile, odd widths, one exact tile, one node past it
TINY_CASES = [
    (3, 3, 1.0, 0.5, 0.02, 0.03),
    (5, 7, 1.6, 0.2, 0.005, 0.01),
    (9, 4, 0.5, 1.0, 0.01, 0.02),
    (64, 8, 0.25, 0.3, 0.01, 0.02),
    (65, 9, 2.0, 0.6, 0.02, 0.05),
    (130, 17, 1.0, 0.1, 0.01, 0.02),
]


@pytest.mark.parametrize("dtype", [L.F32, L.F16])
def test_tma_body_on_grids_of_a_tile_or_less(dtype):
    """Wall tiles on every side of one tile at once (ghost cells of all four
    walls and their corners in one window, rows and columns past the grid):
    each slot of the TMA-staged body equals a single handle bitwise."""
    b = L.Batch(len(TINY_CASES), dtype)
    slots, refs = [], []
    for k, (nx, ny, r, gamma, nu, u) in enumerate(TINY_CASES):
        p = L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype)
        w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
        f0 = w[:, None, None] + I.noise(3700 + k, (9, ny, nx), 1e-3)
        s = b.add(p, 0.0, 10 ** 6)
        b.set_populations(s, f0)
        h = L.Lbm(p)
        h.variant = batch_tile_variant(dtype)
        h.set_populations(f0)
        slots.append(s)
        refs.append(h)
    assert b.tma_body
    for n in (1, 19, 40):  # crossing residual steps
        b.run(n)
        for s, h in zip(slots, refs):
            h.step(n)
            info, st = b.query(s)
            assert st == L.SLOT_ACTIVE and info.step == h.info().step
            assert np.array_equal(b.populations(s), h.populations()), (b.shapes[s], info.step)
    for h in refs:
        h.close()


def test_tma_body_retires_where_single_handles_stop():
    """Retirement on the residual with the TMA-staged body: each slot stops at
    the step where a single handle on the interior kernel stops, with the
    same populations."""
    cav = [I.Cavity(150, 60, 0.5, 0.5, 50.0, 0.03, "f32"), I.Cavity(100, 100, 1.0, 1.0, 100.0, 0.05, "f32"),
           I.Cavity(90, 130, 2.0, 0.25, 60.0, 0.02, "f32")]
    tols = [1e-5, 1e-5, 2e-6]
    b = L.Batch(4, L.F32)
    slots = [b.add(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32), t, 500000)
             for c, t in zip(cav, tols)]
    assert b.tma_body
    while b.run(5000):
        pass
    for c, t, s in zip(cav, tols, slots):
        info, st = b.query(s)
        assert st == L.SLOT_CONVERGED and info.residual < t
        h = L.Lbm(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32))
        h.variant = 0
        status, steps = h.run(t, 500000)
        assert status == L.OK and steps == info.step
        assert np.array_equal(b.populations(s), h.populations())
        h.close()


def test_tma_body_and_general_body_agree():
    """The two tile bodies of the batch engine take the same steps up to FP32
    round-off (different tile shapes, the same node arithmetic)."""
    out = []
    for body in (L.BATCH_BODY_AUTO, L.BATCH_BODY_GENERAL):
        b = L.Batch(len(TMA_CASES), L.F32)
        b.set_body(body)
        slots = []
        for k, (nx, ny, r, gamma, nu, u) in enumerate(TMA_CASES):
            p = L.lbm_params_init(nx, ny, r, gamma, nu, u, L.F32)
            w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
            s = b.add(p, 0.0, 10 ** 6)
            b.set_populations(s, w[:, None, None] + I.noise(2700 + k, (9, ny, nx), 1e-3))
            slots.append(s)
        assert b.tma_body == (body == L.BATCH_BODY_AUTO)
        b.run(45)
        out.append([b.populations(s) for s in slots])
    for a, g in zip(*out):
        assert np.max(np.abs(a - g)) < 1e-7


def test_autotune_restores_state_when_a_wait_runs_out():
    """A grid-barrier timeout during the timing launches ends lbm_batch_autotune
    with LBM_ETIMEOUT after the slots' state is put back; the batch stays
    usable and its launch shape unchanged."""
    cases = [(64, 32, 1.0, 0.5, 0.02, 0.05), (200, 90, 2.0, 0.1, 0.01, 0.02)]
    b = L.Batch(2, L.F32)
    slots = []
    for k, (nx, ny, r, gamma, nu, u) in enumerate(cases):
        s = b.add(L.lbm_params_init(nx, ny, r, gamma, nu, u, L.F32), 0.0, 10 ** 6)
        w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
        b.set_populations(s, w[:, None, None] + I.noise(900 + k, (9, ny, nx), 1e-3))
        slots.append(s)
    b.run(13)
    before = [(b.populations(s), b.query(s)[0].step) for s in slots]
    shape = b.ctas_per_sm
    b.set_wait_limit(2_000_000, hold=True)  # the first timing launch's waits run out
    with pytest.raises(L.LbmError) as e:
        b.autotune(10)
    assert e.value.status == L.ETIMEOUT
    assert b.ctas_per_sm == shape
    for s, (p, step) in zip(slots, before):
        info, st = b.query(s)
        assert st == L.SLOT_ACTIVE and info.step == step
        assert np.array_equal(b.populations(s), p)
    assert b.run(7) == 2
    for s, (_, step) in zip(slots, before):
        assert b.query(s)[0].step == step + 7
