"""The D2Q9 path (Table I) on the GPU against the D2Q9 FP64 oracle on identical
seeded inputs and noise, and its statistics and hydrodynamics.

Tolerances as for D3Q19: FP64 1e-12, FP32 1e-5, FP16 / BF16 deviation storage
(steps + 1) ulp of the format at the largest |n - rho0 a_i|.
"""
import math

import numpy as np
import pytest

from paper_0707_1581_gb300 import flb
from paper_0707_1581_gb300.inputs import relative_perturbation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


@pytest.fixture(scope="module")
def D():
    from oracle import d2q9
    return d2q9


@pytest.fixture(scope="module")
def a9(D):
    return D.lattice()[1]


def state(a9, nx, ny, seed, amp=0.02):
    return a9[:, None, None] * relative_perturbation((ny, nx), seed=seed, amp=amp, ncomp=9)


def cfg2(nx, ny, kT, gs, gb, gg, seed, **kw):
    return flb.config(nx, ny, 1, 1.0, kT, gs, gb, gg, seed, lattice="d2q9", **kw)


def run2(n0, nx, ny, kT, gs, gb, gg, seed, steps, **kw):
    with flb.flb_create_ex(cfg2(nx, ny, kT, gs, gb, gg, seed, **kw)) as ctx:
        if n0 is not None:
            ctx.flb_set_populations(n0)
        ctx.flb_step(steps)
        return ctx.flb_get_populations()


def oparams(D, nx, ny, kT, gs, gb, gg, seed, **kw):
    return D.make_params(nx, ny, rho0=1.0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=seed, **kw)


def test_nz_must_be_one_and_lattices_do_not_mix():
    with pytest.raises(flb.FlbError) as e:
        flb.flb_create_ex(flb.config(8, 8, 2, lattice="d2q9"))
    assert e.value.code == flb.FLB_EINVAL
    with pytest.raises(flb.FlbError):
        flb.flb_create_batch([flb.config(8, 8, 1, lattice="d2q9"), flb.config(8, 8, 8)])


@pytest.mark.parametrize("shape", [(1, 1), (3, 2), (37, 23), (130, 5)])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_f64_parity_ragged(D, a9, shape, pattern):
    nx, ny = shape
    n0 = state(a9, nx, ny, seed=nx * 10 + ny)
    steps = 7
    got = run2(n0, nx, ny, 1e-3, 0.35, -0.2, 0.15, 42, steps, store="f64", pattern=pattern)
    ref = D.run(oparams(D, nx, ny, 1e-3, 0.35, -0.2, 0.15, 42), n0, 0, steps)
    assert np.abs(got - ref).max() <= 1e-12


def test_f64_from_rest_force_and_launch_shapes(D):
    nx, ny, steps = 48, 40, 60
    ref = D.run(oparams(D, nx, ny, 1e-4, 0.2, 0.1, 0.0, 3, force_amp=1e-4), D.rest_state(nx, ny), 0, steps)
    for bx, by in ((32, 8), (64, 1), (128, 2)):
        got = run2(None, nx, ny, 1e-4, 0.2, 0.1, 0.0, 3, steps, store="f64", pattern="aa", force_amp=1e-4,
                   block_x=bx, block_y=by)
        assert np.abs(got - ref).max() <= 1e-12, (bx, by)
    assert np.abs(ref - D.rest_state(nx, ny)).max() > 1e-3


def test_stress_only_and_local_density_variants(D, a9):
    nx, ny = 24, 20
    n0 = state(a9, nx, ny, seed=5, amp=0.05)
    for kw in ({"noise_ghosts": False}, {"noise_rho_local": True}):
        got = run2(n0, nx, ny, 1e-3, 0.3, 0.2, 0.1, 7, 5, store="f64", **kw)
        ref = D.run(oparams(D, nx, ny, 1e-3, 0.3, 0.2, 0.1, 7, **kw), n0, 0, 5)
        assert np.abs(got - ref).max() <= 1e-12, kw


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_f32_parity(D, a9, pattern):
    nx, ny, steps = 200, 70, 20
    n0 = state(a9, nx, ny, seed=8)
    got = run2(n0, nx, ny, 1e-4, 0.5, 0.2, 0.0, 11, steps, store="f32", pattern=pattern, force_amp=1e-5)
    ref = D.run(oparams(D, nx, ny, 1e-4, 0.5, 0.2, 0.0, 11, force_amp=1e-5), n0, 0, steps)
    assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("store,ostore,mant", [("f16dev", 2, 11), ("bf16dev", 3, 8), ("bf16sr", 4, 8)])
def test_deviation_storage(D, a9, store, ostore, mant):
    nx, ny, steps = 64, 16, 4
    n0 = state(a9, nx, ny, seed=20)
    ref = D.run(oparams(D, nx, ny, 1e-4, 0.3, 0.2, 0.0, 5, store=ostore), n0, 0, steps)
    got = run2(n0, nx, ny, 1e-4, 0.3, 0.2, 0.0, 5, steps, store=store)
    dev = np.abs(ref - a9[:, None, None]).max()
    ulp = 2.0 ** (np.floor(np.log2(dev)) - (mant - 1))
    assert np.abs(got - ref).max() <= (steps + 1) * ulp
    assert np.mean(got == ref) > 0.8


def test_batch_graphs_and_checkpoint(D, a9, tmp_path):
    shapes = [(32, 8), (17, 9), (64, 4)]
    cfgs = [cfg2(nx, ny, 1e-4, 0.2 + 0.2 * r, 0.1, 0.0, 4, replica=r, store="f32", pattern="aa", graph_steps=4)
            for r, (nx, ny) in enumerate(shapes)]
    starts = [state(a9, nx, ny, seed=40 + b) for b, (nx, ny) in enumerate(shapes)]
    path = str(tmp_path / "d2.flb")
    with flb.flb_create_batch(cfgs) as ctx:
        for b, n0 in enumerate(starts):
            ctx.flb_set_populations(n0, box=b)
        ctx.flb_step(6)
        ctx.flb_save(path)
        ctx.flb_step(5)
        got = [ctx.flb_get_populations(box=b) for b in range(3)]
    for b, (nx, ny) in enumerate(shapes):
        ref = D.run(oparams(D, nx, ny, 1e-4, 0.2 + 0.2 * b, 0.1, 0.0, 4, replica=b), starts[b], 0, 11)
        assert np.abs(got[b] - ref).max() <= 1e-5, b
    with flb.flb_create_batch(cfgs) as ctx:
        ctx.flb_load(path)
        assert ctx.flb_get_step() == 6
        ctx.flb_step(5)
        for b in range(3):
            assert np.array_equal(ctx.flb_get_populations(box=b), got[b])
    # a D3Q19 context of the same sizes refuses the D2Q9 checkpoint
    with flb.flb_create_batch([flb.config(nx, ny, 1, store="f32", pattern="aa") for nx, ny in shapes]) as ctx:
        with pytest.raises(flb.FlbError):
            ctx.flb_load(path)


def test_moments_profile_and_init_velocity(D):
    nx, ny = 24, 16
    y, x = np.mgrid[0:ny, 0:nx]
    u = np.stack([0.01 * np.sin(2 * np.pi * y / ny), 0.005 * np.cos(2 * np.pi * x / nx)])
    ref = D.equilibrium_field(np.ones((ny, nx)), u)
    with flb.flb_create_ex(cfg2(nx, ny, 0.0, 0.3, 0.2, 0.0, 1, store="f64")) as ctx:
        ctx.flb_init_velocity(u)
        n = ctx.flb_get_populations()
        rho, j, Pi = ctx.flb_moments()
        prho, pj = ctx.flb_z_profile()
        sites = ctx.flb_get_sites([0, 5, nx * ny - 1])
    assert np.abs(n - ref).max() <= 1e-15
    c = D.lattice()[0].astype(float)
    assert np.abs(rho - ref.sum(0)).max() <= 1e-14
    assert np.abs(j - np.tensordot(c.T, ref, axes=(1, 0))).max() <= 1e-14
    pis = [c[:, 0] ** 2, c[:, 1] ** 2, c[:, 0] * c[:, 1]]
    assert np.abs(Pi - np.stack([np.tensordot(p, ref, axes=(0, 0)) for p in pis])).max() <= 1e-14
    assert np.allclose(prho, rho.mean(1), atol=1e-14)
    assert np.allclose(pj[0], j[0].mean(1), atol=1e-14) and np.allclose(pj[1], j[1].mean(1), atol=1e-14)
    assert np.all(pj[2] == 0)
    assert np.array_equal(sites, n.reshape(9, -1)[:, [0, 5, nx * ny - 1]].T)   # the same gather, site by site


@pytest.mark.parametrize("store", ["f32", "f16dev"])
def test_equipartition_and_structure_factor(store):
    """64^2, k_BT = 1e-4: every mode variance within 1 % of mu rho0 w_k (Table I
    norms), <u_a^2> rho0 / k_BT and S(q) / (mu rho0) within 2 %."""
    L, kT = 64, 1e-4
    with flb.flb_create_ex(cfg2(L, L, kT, 0.5, 0.2, 0.0, 9, store=store)) as ctx:
        ctx.flb_enable_structure_factor()
        ctx.flb_step(300)
        ctx.flb_stats_reset()
        for _ in range(3000):
            ctx.flb_step(5)
            ctx.flb_stats_sample()
        st = ctx.flb_mode_stats()
        S, cnt = ctx.flb_structure_factor(48)
    r = st["mode_ratio"][:9]
    assert np.all(st["mode_ratio"][9:] == 0) and st["nonfinite"] == 0
    assert np.max(np.abs(r[3:] - 1)) < 0.01, r
    assert np.max(np.abs(r[:3] - 1)) < 0.03, r
    assert np.max(np.abs(st["u2_ratio"][:2] - 1)) < 0.02 and st["u2_ratio"][2] == 0
    sel = cnt > 0
    assert abs(np.sum(S[sel] * cnt[sel]) / cnt[sel].sum() / (3 * kT) - 1) < 0.02


def test_shear_viscosity_from_decay():
    """k_BT = 0, u_x = u0 sin(2 pi y / L): decay rate nu q^2 with Eq. shearviscosity
    (the same nu as D3Q19) to the O(q^2) lattice correction, < 0.5 % at L = 128."""
    L, gs, u0 = 128, 0.5, 1e-4
    nu = (1 + gs) / (6 * (1 - gs))
    q = 2 * np.pi / L
    y = np.arange(L)
    u = np.zeros((2, L, 4))
    u[0] = u0 * np.sin(q * y)[:, None]
    with flb.flb_create_ex(cfg2(4, L, 0.0, gs, 0.2, 0.0, 0, store="f64")) as ctx:
        ctx.flb_init_velocity(u)
        amps = []
        for t in range(0, 401, 100):
            rho, j = ctx.flb_z_profile()
            amps.append((2.0 / L) * np.sum(j[0] / rho * np.sin(q * y)))
            ctx.flb_step(100)
    rate = -np.polyfit(np.arange(0, 401, 100)[1:], np.log(amps[1:]), 1)[0]
    assert rate / (nu * q * q) == pytest.approx(1.0, abs=0.005)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("store,shape,V,bx,by,tol", [
    ("f32", (8, 5), 4, 32, 1, 1e-5),       # two groups per row: a warp spans 16 rows
    ("f32", (4, 7), 4, 32, 2, 1e-5),       # one group per row: every lane is a row start and end
    ("f32", (12, 9), 4, 64, 4, 1e-5),      # three groups per row, ragged last block
    ("f32", (1024, 3), 4, 128, 2, 1e-5),   # rows span several warps
    ("f64", (6, 5), 2, 32, 1, 1e-12),      # FP64: 2 sites per thread
    ("f64", (200, 3), 2, 64, 1, 1e-12),
])
def test_vector_kernel_against_oracle(D, a9, pattern, store, shape, V, bx, by, tol):
    nx, ny = shape
    n0 = state(a9, nx, ny, seed=nx + ny)
    cfg = cfg2(nx, ny, 1e-3, 0.3, -0.1, 0.2, 17, store=store, pattern=pattern, sites_per_thread=V, block_x=bx,
               block_y=by, force_amp=1e-4)
    with flb.flb_create_ex(cfg) as ctx:
        assert ctx.flb_get_launch() == (V, bx, by)
        ctx.flb_set_populations(n0)
        ctx.flb_step(5)
        got = ctx.flb_get_populations()
    ref = D.run(oparams(D, nx, ny, 1e-3, 0.3, -0.1, 0.2, 17, force_amp=1e-4), n0, 0, 5)
    assert np.abs(got - ref).max() <= tol


def test_scalar_and_vector_kernels_agree():
    """The same D2Q9 box with one and four sites per thread: identical noise, FP32
    rounding of the same arithmetic (within 1e-6)."""
    runs = []
    for V in (1, 4):
        with flb.flb_create_ex(cfg2(256, 16, 1e-4, 0.3, 0.2, 0.0, 2, store="f32", pattern="aa",
                                    sites_per_thread=V)) as ctx:
            assert ctx.flb_get_launch()[0] == V
            ctx.flb_step(9)
            runs.append(ctx.flb_get_populations())
    assert np.abs(runs[0] - runs[1]).max() <= 1e-6


def test_sound_wave_speed_and_attenuation():
    """k_BT = 0, a standing density wave along y on a 4 x 64 D2Q9 box,
    gamma_s = 0.2, gamma_b = -0.3: speed c_s = sqrt(1/3) and attenuation
    (nu + zeta/rho) q^2 / 2 with Eq. bulkviscosity at d = 2 (in 2-D the
    longitudinal viscosity is zeta + (2 - 2/d) eta = zeta + eta), within 1 %
    (the lattice's own O(q^2) dispersion is a few 0.1 %)."""
    from scipy.optimize import least_squares
    L, cross, gs, gb, drho = 64, 4, 0.2, -0.3, 1e-4
    q = 2 * math.pi / L
    nu = (1 + gs) / (6 * (1 - gs))
    zeta = (1 + gb) / (6 * (1 - gb))          # c_s^2 / d (1 + gb) / (1 - gb), d = 2
    a = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    y = np.arange(L)
    n = a[:, None, None] * (1.0 + drho * np.cos(q * y))[None, :, None] * np.ones((9, L, cross))
    ts, amps = [], []
    with flb.flb_create_ex(cfg2(cross, L, 0.0, gs, gb, 0.0, 0, store="f64")) as ctx:
        ctx.flb_set_populations(n)
        for t in range(0, 601, 2):
            rho, _ = ctx.flb_z_profile()
            amps.append(2.0 / L * np.sum((rho - 1.0) * np.cos(q * y)))
            ts.append(t)
            ctx.flb_step(2)
    ts, amps = np.array(ts, float), np.array(amps)
    G0, w0 = (nu + zeta) * q * q / 2, q / math.sqrt(3)
    fit = least_squares(lambda p: p[0] * np.exp(-p[1] * ts) * np.cos(p[2] * ts + p[3]) - amps, [drho, G0, w0, 0.0],
                        x_scale=[drho, G0, w0, 1.0])
    _, G, w, _ = fit.x
    assert w / w0 == pytest.approx(1.0, abs=0.003)
    assert G / G0 == pytest.approx(1.0, abs=0.01)


def test_kolmogorov_flow_amplitude():
    """F_x(y) = F0 sin(2 pi y / L) on a 4 x 128 D2Q9 box from rest, 4000 steps:
    the amplitude of u_x(y) follows F0 / (rho0 nu k^2) (1 - exp(-nu k^2 t)) within 1 %."""
    L, cross, gs, F0, T = 128, 4, 0.3, 1e-5, 4000
    nu = (1 + gs) / (6 * (1 - gs))
    k = 2 * math.pi / L
    with flb.flb_create_ex(cfg2(cross, L, 0.0, gs, 0.2, 0.0, 0, store="f32", pattern="aa", force_amp=F0)) as ctx:
        ctx.flb_step(T)
        rho, j = ctx.flb_z_profile()
    y = np.arange(L)
    amp = 2.0 / L * np.sum(j[0] / rho * np.sin(k * y))
    expect = F0 / (nu * k * k) * (1 - math.exp(-nu * k * k * T))
    assert amp / expect == pytest.approx(1.0, abs=0.01)


@pytest.mark.parametrize("pattern,steps,nx", [("ab", 30, 16), ("aa", 30, 16), ("aa", 31, 16), ("ab", 31, 14)])
@pytest.mark.parametrize("store", ["f64", "f32"])
def test_mode_stats_match_the_oracle_on_the_same_state(D, store, pattern, steps, nx):
    """One statistics sample of the device state against the oracle's
    observables of the same (gathered) populations: every streaming layout,
    rows of whole four-site groups and ragged rows."""
    ny = 12
    with flb.flb_create_ex(cfg2(nx, ny, 1e-4, 0.2, 0.2, 0.0, 1, store=store, pattern=pattern)) as ctx:
        ctx.flb_step(steps)
        ctx.flb_stats_reset()
        ctx.flb_stats_sample()
        st = ctx.flb_mode_stats()
        n = ctx.flb_get_populations()
    tol = 1e-12 if store == "f64" else 1e-5
    assert st["nsamples"] == 1
    assert np.allclose(st["mode_m2"][:9], D.mode_second_moments(n, 1.0), rtol=tol * 10, atol=1e-20)
    c = D.lattice()[0].astype(float)
    rho = n.sum(axis=0)
    j = np.tensordot(c.T, n, axes=(1, 0))
    assert np.allclose(st["u2"][:2], ((j / rho) ** 2).reshape(2, -1).mean(1), rtol=1e-5)
    assert st["mass_last"] == pytest.approx(rho.sum(), rel=1e-12 if store == "f64" else 1e-9)


def test_finite_time_mode_variances_from_rest_follow_the_linear_recursion(D):
    """64 D2Q9 replicas of 16 x 12 in one batch, FP32, from rest: every mode
    variance of the first 20 steps within 5 standard errors of the exact
    covariance recursion of the linearised chain."""
    from tests.test_oracle_d2q9 import mode_variance_recursion_2d
    c, a, e, w = D.lattice()
    nx, ny, kT, rho0, gs, gb, gg, T, nrep = 16, 12, 1e-4, 1.0, 0.2, 0.1, 0.0, 20, 64
    pred = mode_variance_recursion_2d(c.astype(float), a, e, w, (nx, ny), kT, rho0, gs, gb, gg, T)
    cfgs = [cfg2(nx, ny, kT, gs, gb, gg, 1, replica=r, store="f32") for r in range(nrep)]
    obs = np.zeros((nrep, T, 9))
    with flb.flb_create_batch(cfgs) as ctx:
        for t in range(T):
            ctx.flb_step(1)
            ctx.flb_stats_reset()
            ctx.flb_stats_sample()
            for b in range(nrep):
                obs[b, t] = ctx.flb_mode_stats(box=b)["mode_ratio"][:9]
    mean = obs.mean(0)
    se = obs.std(0, ddof=1) / np.sqrt(nrep)
    assert np.all(np.abs(mean - pred) < 5 * se + 2e-3), np.abs(mean - pred) / (se + 1e-12)


def test_bench_box_sampled_sites(D):
    """The benchmark's D2Q9 variant as it is timed: 8192^2 FP32, AB, F_x(y) =
    1e-5 sin(2 pi y / ny), k_BT = 1e-4, seed 3, the library's default launch
    (the vector kernel).  Two steps from rest; 300 sampled sites and the four
    corners are recomputed by the oracle one collision at a time."""
    import bench
    from paper_0707_1581_gb300.inputs import sample_sites
    E = bench.D2Q9_EDGE
    w = {**bench.workload_config("f32", E, "d2q9"), "pattern": "ab"}
    cfg = flb.config(**w)
    N = E * E
    sites = np.unique(np.concatenate([np.array([0, E - 1, N - E, N - 1], dtype=np.int64),
                                      sample_sites(N, 300, seed=9)]))
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(2)
        got = ctx.flb_get_sites(sites)
    c, a = D.lattice()[0], D.lattice()[1]
    p = D.make_params(E, E, rho0=w["rho0"], kT=w["kT"], gamma_shear=w["gamma_shear"], gamma_bulk=w["gamma_bulk"],
                      gamma_ghost=w["gamma_ghost"], seed=w["seed"], force_amp=w["force_amp"])
    F0 = w["force_amp"]
    memo = {}

    def n_at(x, y, t):
        key = (x % E, y % E, t)
        if key in memo:
            return memo[key]
        x, y = key[:2]
        if t == 0:
            val = a.copy()
        else:
            val = np.empty(9)
            for i in range(9):
                xs, ys = (x - c[i, 0]) % E, (y - c[i, 1]) % E
                Fx = F0 * np.sin(2 * np.pi * ys / E)
                val[i] = D.collide_site(p, n_at(xs, ys, t - 1), site=int(xs + E * ys), step=t - 1, force=[Fx, 0])[i]
        memo[key] = val
        return val

    worst = max(np.abs(got[k] - n_at(s % E, s // E, 2)).max() for k, s in enumerate(sites))
    assert worst <= 1e-5
    assert np.abs(got - a).max() > 1e-4          # the noise moved the state off rest
