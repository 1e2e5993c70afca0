"""CUDA path versus the FP64 oracle on identical seeded inputs and noise.

Tolerances (max |n_gpu - n_oracle| over every population, rho0 = 1):
  FP64 storage and collide          1e-12   (rounding-order differences only)
  FP32 storage and collide          1e-5    (FP32 rounding ~1e-7 per step, the
                                             hardware log2/sin of the normals
                                             ~1e-6 of sigma_k in rare draws)
  FP16 / BF16 deviation storage     (steps + 1) ulp of the format at the largest
                                    |n - rho0 a_i|: the oracle rounds its FP64
                                    result, the kernel its FP32 result, and the two
                                    roundings may fall on different sides of a tie.
"""
import numpy as np
import pytest

from paper_0707_1581_gb300 import flb
from paper_0707_1581_gb300.inputs import relative_perturbation, sample_sites, smooth_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


@pytest.fixture(scope="module")
def weights(ora):
    return ora.lattice()[1]


def oracle_params(ora, nx, ny, nz, kT, gs, gb, gg, seed, replica=0, force=0.0, store=0, noise_ghosts=True):
    return ora.make_params(nx, ny, nz, rho0=1.0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=seed,
                           replica=replica, force_amp=force, store=store, noise_ghosts=noise_ghosts)


def random_state(weights, shape, seed, amp=0.02):
    return weights[:, None, None, None] * relative_perturbation(shape, seed=seed, amp=amp)


def run_gpu(n0, nx, ny, nz, kT, gs, gb, gg, seed, steps, **kw):
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, kT, gs, gb, gg, seed, **kw)) as ctx:
        if n0 is not None:
            ctx.flb_set_populations(n0)
        ctx.flb_step(steps)
        assert ctx.flb_get_step() == steps
        return ctx.flb_get_populations()


# --- FP64: parity at 1e-12 -------------------------------------------------

def test_f64_config1_from_rest_200_steps(ora):
    """16^3, k_BT = 1e-4, gamma_s = gamma_b = 0.2, gamma_ghost = 0, seed 1, 200 steps."""
    L = 16
    got = run_gpu(None, L, L, L, 1e-4, 0.2, 0.2, 0.0, 1, 200, store="f64")
    ref = ora.run(oracle_params(ora, L, L, L, 1e-4, 0.2, 0.2, 0.0, 1), ora.rest_state(L, L, L), 0, 200)
    assert np.abs(got - ref).max() <= 1e-12
    # the state has really moved away from rest
    assert np.abs(ref - ora.rest_state(L, L, L)).max() > 1e-3


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (3, 4, 5), (7, 5, 3), (33, 2, 3)])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_f64_ragged_boxes(ora, weights, shape, pattern):
    nx, ny, nz = shape
    n0 = random_state(weights, (nz, ny, nx), seed=nx * 100 + ny * 10 + nz)
    steps = 7                     # odd: ends on an AA odd-step layout
    got = run_gpu(n0, nx, ny, nz, 1e-3, 0.35, -0.2, 0.15, 42, steps, store="f64", pattern=pattern)
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-3, 0.35, -0.2, 0.15, 42), n0, 0, steps)
    assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("nx,V,bx,by", [(40, 1, 32, 4), (40, 2, 64, 2), (40, 4, 32, 1), (40, 1, 256, 1),
                                        (32, 2, 16, 4)])
def test_f64_launch_shapes_agree(ora, weights, nx, V, bx, by):
    ny, nz = 9, 6
    n0 = random_state(weights, (nz, ny, nx), seed=9)
    got = run_gpu(n0, nx, ny, nz, 1e-4, 0.5, 0.1, 0.0, 3, 5, store="f64", sites_per_thread=V, block_x=bx, block_y=by)
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-4, 0.5, 0.1, 0.0, 3), n0, 0, 5)
    assert np.abs(got - ref).max() <= 1e-12


def test_f64_force_and_zero_temperature(ora, weights):
    nx, ny, nz = 6, 5, 16
    n0 = random_state(weights, (nz, ny, nx), seed=4)
    for kT in (0.0, 1e-4):
        got = run_gpu(n0, nx, ny, nz, kT, 0.3, 0.2, 0.0, 8, 9, store="f64", force_amp=1e-3)
        ref = ora.run(oracle_params(ora, nx, ny, nz, kT, 0.3, 0.2, 0.0, 8, force=1e-3), n0, 0, 9)
        assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("store,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_local_density_noise_variant(ora, weights, store, tol):
    """noise variance mu rho(r) w_k with the local density (Sec. III, before the
    low-velocity limit is taken at the mean density)."""
    nx, ny, nz = 12, 6, 5
    n0 = random_state(weights, (nz, ny, nx), seed=13, amp=0.05)
    got = run_gpu(n0, nx, ny, nz, 1e-3, 0.3, 0.1, 0.2, 4, 5, store=store, noise_rho_local=True)
    p = ora.make_params(nx, ny, nz, rho0=1.0, kT=1e-3, gamma_shear=0.3, gamma_bulk=0.1, gamma_ghost=0.2, seed=4,
                        noise_rho_local=True)
    ref = ora.run(p, n0, 0, 5)
    assert np.abs(got - ref).max() <= tol
    plain = ora.run(oracle_params(ora, nx, ny, nz, 1e-3, 0.3, 0.1, 0.2, 4), n0, 0, 5)
    assert np.abs(plain - ref).max() > 10 * tol       # the variant really differs


def test_f64_stress_only_thermalisation_variant(ora, weights):
    nx, ny, nz = 8, 4, 4
    n0 = random_state(weights, (nz, ny, nx), seed=6)
    got = run_gpu(n0, nx, ny, nz, 1e-3, 0.2, 0.2, 0.0, 2, 4, store="f64", noise_ghosts=False)
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-3, 0.2, 0.2, 0.0, 2, noise_ghosts=False), n0, 0, 4)
    assert np.abs(got - ref).max() <= 1e-12


# --- FP32: parity at 1e-5 --------------------------------------------------

@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_f32_64cube(ora, weights, pattern):
    """64^3, k_BT = 1e-4, gamma_s = 0.5, gamma_b = 0.2, gamma_ghost = 0, seed 7."""
    L, steps = 64, 12
    n0 = random_state(weights, (L, L, L), seed=70, amp=0.01)
    got = run_gpu(n0, L, L, L, 1e-4, 0.5, 0.2, 0.0, 7, steps, store="f32", pattern=pattern)
    ref = ora.run(oracle_params(ora, L, L, L, 1e-4, 0.5, 0.2, 0.0, 7), n0, 0, steps)
    assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("shape,V,bx,by", [
    ((13, 6, 5), 1, 32, 4),      # ragged row: scalar path
    ((12, 6, 5), 2, 32, 4),      # one warp spans several rows
    ((12, 6, 5), 4, 4, 8),       # one inactive thread per block row, a warp spans 8 rows
    ((12, 6, 5), 4, 32, 1),      # most lanes inactive
    ((24, 5, 3), 2, 4, 8),       # block row covers 8 of 24 sites
    ((256, 3, 3), 2, 32, 2),     # warp edges in the middle of a row
    ((512, 2, 2), 4, 128, 1),    # the benchmark's launch shape (row-exchange variant)
    ((128, 3, 5), 4, 32, 2),     # in-warp rows: one warp per row, its own periodic neighbour
    ((256, 5, 3), 4, 64, 2),     # row exchange: two warps per row, two rows per block, ragged y
    ((64, 5, 3), 4, 16, 4),      # in-warp rows: two rows per warp, ragged y
    ((8, 7, 3), 4, 2, 16),       # in-warp rows: sixteen rows per warp
    ((4, 9, 2), 4, 1, 32),       # in-warp rows of one lane (its own periodic neighbour)
    ((32, 6, 4), 2, 16, 2),      # in-warp rows with 2 sites per thread
])
def test_f32_vector_paths_and_edges(ora, weights, pattern, shape, V, bx, by):
    nx, ny, nz = shape
    n0 = random_state(weights, (nz, ny, nx), seed=V * 7 + bx)
    steps = 5
    cfg = dict(store="f32", pattern=pattern, sites_per_thread=V, block_x=bx, block_y=by)
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, 1e-3, -0.3, 0.4, 0.2, 11, **cfg)) as ctx:
        assert ctx.flb_get_launch() == (V, bx, by)
        ctx.flb_set_populations(n0)
        ctx.flb_step(steps)
        got = ctx.flb_get_populations()
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-3, -0.3, 0.4, 0.2, 11), n0, 0, steps)
    assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("store,ostore,mant", [("f16dev", 2, 11), ("bf16dev", 3, 8), ("bf16sr", 4, 8)])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_deviation_storage_row_exchange(ora, weights, store, ostore, mant, pattern):
    nx, ny, nz, steps = 256, 3, 4, 3
    n0 = random_state(weights, (nz, ny, nx), seed=21, amp=0.02)
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 5, store=ostore), n0, 0, steps)
    got = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 5, steps, store=store, pattern=pattern,
                  sites_per_thread=4, block_x=64, block_y=2)
    dev = np.abs(ref - weights[:, None, None, None]).max()
    ulp = 2.0 ** (np.floor(np.log2(dev)) - (mant - 1))
    assert np.abs(got - ref).max() <= (steps + 1) * ulp


def test_sites_per_thread_falls_back_when_nx_is_not_divisible():
    with flb.flb_create_ex(flb.config(16, 4, 4, store="f32", sites_per_thread=4, block_x=4, block_y=4)) as ctx:
        assert ctx.flb_get_launch()[0] == 1          # 16-thread blocks: no full warps
    with flb.flb_create_ex(flb.config(13, 4, 4, store="f32", sites_per_thread=4)) as ctx:
        assert ctx.flb_get_launch()[0] == 1
    with flb.flb_create_ex(flb.config(14, 4, 4, store="f32", sites_per_thread=4)) as ctx:
        assert ctx.flb_get_launch()[0] == 2
    with flb.flb_create_ex(flb.config(16, 4, 4, store="f64", sites_per_thread=4)) as ctx:
        assert ctx.flb_get_launch()[0] == 2


def test_f32_kolmogorov_force(ora, weights):
    nx, ny, nz = 8, 8, 32
    n0 = random_state(weights, (nz, ny, nx), seed=12, amp=0.005)
    got = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 3, 10, store="f32", pattern="aa", force_amp=1e-5)
    ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 3, force=1e-5), n0, 0, 10)
    assert np.abs(got - ref).max() <= 1e-5


# --- 16-bit deviation storage -------------------------------------------------

@pytest.mark.parametrize("launch", [{}, dict(sites_per_thread=4, block_x=4, block_y=32)])   # default; in-warp rows
@pytest.mark.parametrize("store,ostore,mant", [("f16dev", 2, 11), ("bf16dev", 3, 8), ("bf16sr", 4, 8)])
def test_deviation_storage(ora, weights, store, ostore, mant, launch):
    nx, ny, nz, steps = 16, 8, 8, 4
    n0 = random_state(weights, (nz, ny, nx), seed=20, amp=0.02)
    p = oracle_params(ora, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 5, store=ostore)
    ref = ora.run(p, n0, 0, steps)
    got = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 5, steps, store=store, **launch)
    dev = np.abs(ref - weights[:, None, None, None]).max()
    ulp = 2.0 ** (np.floor(np.log2(dev)) - (mant - 1))
    assert np.abs(got - ref).max() <= (steps + 1) * ulp
    # most populations agree exactly
    assert np.mean(got == ref) > 0.8


# --- kT = 0, batches, graphs, checkpoints ------------------------------------

def test_zero_temperature_ignores_seed_bitwise(weights):
    nx, ny, nz = 20, 6, 4
    n0 = random_state(weights, (nz, ny, nx), seed=30)
    a = run_gpu(n0, nx, ny, nz, 0.0, 0.4, 0.1, 0.0, 1, 6, store="f32")
    b = run_gpu(n0, nx, ny, nz, 0.0, 0.4, 0.1, 0.0, 999, 6, store="f32")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shapes,pattern,V", [
    ([(8, 8, 8), (12, 6, 5), (16, 16, 4), (5, 3, 7)], "ab", 0),      # ragged: scalar batch path
    ([(8, 8, 8), (12, 6, 5), (32, 16, 4), (64, 3, 7)], "aa", 4),     # nx % 4 == 0: vector batch path
    ([(8, 8, 8), (12, 6, 5), (32, 16, 4), (64, 3, 7)], "ab", 2),
])
def test_batch_matches_single_boxes(ora, weights, shapes, pattern, V):
    gammas = [0.0, 0.3, 0.6, 0.8]
    cfgs = [flb.config(nx, ny, nz, 1.0, 1e-4, g, 0.2, 0.0, 4, replica=r, store="f32", pattern=pattern,
                       sites_per_thread=V)
            for r, ((nx, ny, nz), g) in enumerate(zip(shapes, gammas))]
    steps = 5
    with flb.flb_create_batch(cfgs) as ctx:
        assert ctx.flb_num_boxes() == len(shapes)
        assert V == 0 or ctx.flb_get_launch()[0] == V
        starts = []
        for b, (nx, ny, nz) in enumerate(shapes):
            n0 = random_state(weights, (nz, ny, nx), seed=40 + b)
            ctx.flb_set_populations(n0, box=b)
            starts.append(n0)
        ctx.flb_step(steps)
        for b, ((nx, ny, nz), g) in enumerate(zip(shapes, gammas)):
            got = ctx.flb_get_populations(box=b)
            ref = ora.run(oracle_params(ora, nx, ny, nz, 1e-4, g, 0.2, 0.0, 4, replica=b), starts[b], 0, steps)
            assert np.abs(got - ref).max() <= 1e-5, b


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_cuda_graph_replay_is_bitwise_identical(weights, pattern):
    nx, ny, nz = 32, 8, 8
    n0 = random_state(weights, (nz, ny, nx), seed=50)
    a = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 6, 11, store="f32", pattern=pattern)
    b = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 6, 11, store="f32", pattern=pattern, graph_steps=4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_checkpoint_resume_is_bitwise(tmp_path, weights, pattern):
    nx, ny, nz = 16, 8, 8
    n0 = random_state(weights, (nz, ny, nx), seed=60)
    full = run_gpu(n0, nx, ny, nz, 1e-4, 0.3, 0.2, 0.0, 9, 10, store="f32", pattern=pattern)
    path = str(tmp_path / "ck.flb")
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 9, store="f32", pattern=pattern)
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_step(5)
        ctx.flb_save(path)
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_load(path)
        assert ctx.flb_get_step() == 5
        ctx.flb_step(5)
        resumed = ctx.flb_get_populations()
    assert np.array_equal(full, resumed)


# --- moments, initial states, statistics ---------------------------------------

def test_moments_and_init_velocity(ora):
    nx, ny, nz = 12, 10, 8
    u = smooth_velocity((nz, ny, nx), seed=1, amp=0.02)
    ref_n = ora.equilibrium_field(np.ones((nz, ny, nx)), u)
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, 0.0, 0.3, 0.2, 0.0, 1, store="f64")) as ctx:
        ctx.flb_init_velocity(u)
        got_n = ctx.flb_get_populations()
        rho, j, Pi = ctx.flb_moments()
    assert np.abs(got_n - ref_n).max() <= 1e-15
    r_rho, r_j, r_Pi = ora.moments(ref_n)
    assert np.abs(rho - r_rho).max() <= 1e-14
    assert np.abs(j - r_j).max() <= 1e-14
    assert np.abs(Pi - r_Pi).max() <= 1e-14


@pytest.mark.parametrize("pattern,steps,nx", [("ab", 30, 16), ("aa", 30, 16), ("aa", 31, 16), ("ab", 31, 14)])
@pytest.mark.parametrize("store,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16dev", 1e-5)])
def test_mode_stats_and_structure_factor_match_oracle_on_same_state(ora, weights, store, tol, pattern, steps, nx):
    """Every streaming layout (AB; AA after an even and after an odd step), rows
    of whole four-site groups (vector loads) and ragged rows (scalar loads)."""
    ny, nz = 12, 8
    kT = 1e-4
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, kT, 0.2, 0.2, 0.0, 1, store=store, pattern=pattern)) as ctx:
        ctx.flb_enable_structure_factor()
        ctx.flb_step(steps)
        ctx.flb_stats_reset()
        ctx.flb_stats_sample()
        st = ctx.flb_mode_stats()
        S, cnt = ctx.flb_structure_factor(16)
        S0 = np.zeros(16)                             # the box-0 entry point gives the same means
        assert flb.lib().flb_structure_factor(ctx.h, S0.ctypes.data, 16) == flb.FLB_OK
        assert np.array_equal(S0, S)
        n = ctx.flb_get_populations()
    m2 = ora.mode_second_moments(n, 1.0)
    assert st["nsamples"] == 1
    assert np.allclose(st["mode_m2"], m2, rtol=max(tol, 1e-6) * 10, atol=1e-20)
    rho, j, _ = ora.moments(n)
    assert np.allclose(st["u2"], ((j / rho) ** 2).reshape(3, -1).mean(1), rtol=1e-5)
    # per-site sums in the compute type, accumulated in FP64
    assert st["mass_last"] == pytest.approx(rho.sum(), rel=1e-12 if store == "f64" else 1e-9)
    # S(q) shells from numpy's FFT of the same state
    Sq = ora.structure_factor(n)
    nmax = max(nx, ny, nz)

    def freq(n):   # signed wave number / n, as the shell definition in flb.h states it
        k = np.arange(n)
        return np.where(k <= n // 2, k, k - n) / n

    fz, fy, fx = freq(nz)[:, None, None], freq(ny)[None, :, None], freq(nx)[None, None, :]
    shell = np.floor(nmax * np.sqrt(fx ** 2 + fy ** 2 + fz ** 2)).astype(int)
    for s in range(16):
        sel = shell == s
        sel[0, 0, 0] = False
        if sel.sum() == 0:
            assert cnt[s] == 0
            continue
        assert cnt[s] == sel.sum()
        assert S[s] == pytest.approx(Sq[sel].mean(), rel=1e-6)


def test_full_size_512cube_structure_factor(ora):
    """S(q) of the benchmark's 512^3 FP32 box (AA, Kolmogorov force, k_BT =
    1e-4) after 200 thermal steps from rest, every shell s = 0..443: the
    library's sample (density in the stats pass, half-spectrum FFT with the
    radix-8 passes and the persistent z pass, fixed-point shell sums) against
    numpy's FP64 FFT of the same density field, taken plane by plane of the
    half spectrum.  Bound: 2e-6 of the shell's own value (FP32 rounding of the
    density and of the butterflies, ~1e-7 measured) plus 30 eps32 sqrt(S <S>),
    the part of the transform's rounding that does not scale with a shell's
    own power (an error of ~eps sqrt(log2 N) of the field's rms amplitude on
    every X(q)); it matters for shells with little power (measured 9e-14 on
    the lowest shell after 4 steps, when it holds 7e-7 of the mean power)."""
    import bench
    L, nsh = 512, 444
    cfg = flb.config(**bench.workload_config("f32", L))
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_enable_structure_factor()
        ctx.flb_step(200)
        ctx.flb_stats_sample()
        S, cnt = ctx.flb_structure_factor(nsh)
        st = ctx.flb_mode_stats()
        rho = np.empty((L, L, L))
        assert flb.lib().flb_box_moments(ctx.h, 0, rho.ctypes.data, None, None) == flb.FLB_OK
    # the same sample's FP64 mass equals the sum of the density field
    assert st["nonfinite"] == 0 and st["nsamples"] == 1
    assert st["mass_last"] == pytest.approx(rho.sum(), rel=1e-9)
    F = np.fft.rfftn(rho - rho.mean())          # [kz][ky][kx], kx = 0 .. L/2
    N = float(L) ** 3
    k = np.arange(L)
    f = np.where(k <= L // 2, k, k - L) / L
    fx = np.arange(L // 2 + 1) / L
    wx = np.where((np.arange(L // 2 + 1) == 0) | (np.arange(L // 2 + 1) == L // 2), 1.0, 2.0)   # mirrored columns
    sums, counts = np.zeros(nsh + 1), np.zeros(nsh + 1)
    for kz in range(L):
        P = (F[kz].real ** 2 + F[kz].imag ** 2) / N
        sh = np.floor(L * np.sqrt(f[kz] ** 2 + f[:, None] ** 2 + fx[None, :] ** 2)).astype(np.int64)
        w = np.broadcast_to(wx, sh.shape).copy()
        if kz == 0:
            w[0, 0] = 0.0                            # q = 0 is no shell
        sh = np.minimum(sh, nsh)
        sums += np.bincount(sh.ravel(), weights=(P * w).ravel(), minlength=nsh + 1)
        counts += np.bincount(sh.ravel(), weights=w.ravel(), minlength=nsh + 1)
    want = sums[:nsh] / np.maximum(counts[:nsh], 1)
    assert np.array_equal(cnt, counts[:nsh].astype(np.int64))
    sel = counts[:nsh] > 0
    assert sel.sum() > 400
    bound = 2e-6 * want[sel] + 30 * 2.0 ** -24 * np.sqrt(want[sel] * want[sel].mean())
    assert np.all(np.abs(S[sel] - want[sel]) <= bound), np.abs(S[sel] / want[sel] - 1).max()


def _shells_of_state(ora, n, nshells):
    """Shell means of |FFT(rho - <rho>)|^2 / N of a canonical state (numpy's FFT),
    with the shell definition of flb.h, and the wave vectors per shell."""
    Sq = ora.structure_factor(n)
    nz, ny, nx = Sq.shape
    nmax = max(nx, ny, nz)

    def freq(m):
        k = np.arange(m)
        return np.where(k <= m // 2, k, k - m) / m

    fz, fy, fx = freq(nz)[:, None, None], freq(ny)[None, :, None], freq(nx)[None, None, :]
    shell = np.floor(nmax * np.sqrt(fx ** 2 + fy ** 2 + fz ** 2)).astype(int)
    shell[0, 0, 0] = -1
    sums = np.array([Sq[shell == s].sum() for s in range(nshells)])
    cnt = np.array([(shell == s).sum() for s in range(nshells)])
    return np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0), cnt


@pytest.mark.parametrize("shape", [(15, 12, 7), (40, 48, 56), (22, 13, 1), (9, 1, 1), (1, 6, 10), (33, 2, 3),
                                   (512, 6, 4), (6, 512, 3), (4, 6, 512)])
@pytest.mark.parametrize("store,rel", [("f64", 1e-10), ("f32", 1e-6)])
def test_structure_factor_on_odd_and_mixed_radix_edges(ora, shape, store, rel):
    """S(q) shells of odd edges (the half spectrum's mirrored columns), edges
    with factors 3, 5, 7, 11, 13 (the mixed-radix stages; 40 .. 56 are edges of
    the ensemble's cubes), degenerate edges of 1 and 2, and one edge of 512 in
    each direction (the fixed 512-point passes of the FP32 transform beside the
    general ones), after a thermal run: the mean of two samples equals the mean
    of numpy's FFT of the two states."""
    nx, ny, nz = shape
    nsh = 24
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.1, 3, store=store, pattern="aa")) as ctx:
        ctx.flb_enable_structure_factor()
        ctx.flb_step(5)
        ctx.flb_stats_sample()
        n1 = ctx.flb_get_populations()
        ctx.flb_step(3)
        ctx.flb_stats_sample()
        n2 = ctx.flb_get_populations()
        S, cnt = ctx.flb_structure_factor(nsh)
        ctx.flb_stats_reset()
        S0, _ = ctx.flb_structure_factor(nsh)
    a1, c1 = _shells_of_state(ora, n1, nsh)
    a2, _ = _shells_of_state(ora, n2, nsh)
    assert np.array_equal(cnt, c1)
    want = 0.5 * (a1 + a2)
    sel = c1 > 0
    # relative bound, plus the part of the rounding of the transform that does
    # not scale with a shell's own power: the rounding adds to every X(q) an
    # error of ~eps sqrt(log2 N) times the field's rms amplitude, which moves
    # |X|^2 by ~2 |X| times that, i.e. S by ~2 eps sqrt(log2 N) sqrt(S <S>)
    # (it matters for shells holding ~1e-6 of the power, here the long
    # direction of a 512-long box a few steps after a thermal start)
    eps = 2.0 ** -24 if store == "f32" else 2.0 ** -53
    floor = 30 * eps * np.sqrt(want[sel] * want[sel].mean())
    assert np.all(np.abs(S[sel] - want[sel]) <= rel * np.abs(want[sel]) + floor), (S[sel], want[sel])
    assert np.all(S[~sel] == 0) and np.all(S0 == 0)


@pytest.mark.parametrize("store,tol", [("f32", 1e-5), ("f16dev", 4 * 2.0 ** -16)])
def test_full_size_ensemble_sampled_sites(ora, tmp_path, store, tol):
    """The batched ensemble as the benchmark runs it: 64 replicas of 64^3 and 16
    cubes of 32..128 in one batch (28.26 M sites), gamma_shear ~ U[0, 0.8] per
    box, k_BT = 1e-4, seed 4, launch shape and streaming pattern chosen by the
    autotuner, steps replayed from CUDA graphs.  Two steps from rest; 10 sampled
    sites in each of six boxes are recomputed by the oracle one collision at a
    time with the box's own gamma_shear and replica number."""
    import bench
    from paper_0707_1581_gb300 import tuning
    edges, gammas = bench.ensemble_boxes()
    e = bench.ENSEMBLE
    cfgs = [flb.config(L, L, L, 1.0, e["kT"], g, e["gamma_bulk"], e["gamma_ghost"], e["seed"], replica=r,
                       store=store, pattern="aa", graph_steps=2)
            for r, (L, g) in enumerate(zip(edges, gammas))]
    boxes = [0, 37, 63, 64, 71, 79]
    picks = {b: sample_sites(edges[b] ** 3, 10, seed=100 + b) for b in boxes}
    with flb.flb_create_batch(cfgs) as ctx:
        choice = tuning.autotune_cached(ctx, str(tmp_path / "tuning.json"), trials=6, pattern=True)
        ctx.flb_step(2)
        got = {b: ctx.flb_get_sites(picks[b], box=b) for b in boxes}
    c, a, _, _ = ora.lattice()
    worst = 0.0
    for b in boxes:
        L = edges[b]
        p = ora.make_params(L, L, L, rho0=1.0, kT=e["kT"], gamma_shear=gammas[b], gamma_bulk=e["gamma_bulk"],
                            gamma_ghost=e["gamma_ghost"], seed=e["seed"], replica=b, store=0)
        memo = {}

        def n_at(x, y, z, t):
            key = (x % L, y % L, z % L, t)
            if key in memo:
                return memo[key]
            x, y, z = key[:3]
            if t == 0:
                val = a.copy()   # rest: n = rho0 a_i
            else:
                val = np.empty(19)
                for i in range(19):
                    xs, ys, zs = x - c[i, 0], y - c[i, 1], z - c[i, 2]
                    site = (xs % L) + L * ((ys % L) + L * (zs % L))
                    val[i] = ora.collide_site(p, n_at(xs, ys, zs, t - 1), site=site, step=t - 1)[i]
                if store == "f16dev":
                    val = a + np.array([ora.round_f16(v) for v in (val - a)])
            memo[key] = val
            return val

        for k, site in enumerate(picks[b]):
            x, y, z = site % L, (site // L) % L, site // (L * L)
            worst = max(worst, np.abs(got[b][k] - n_at(x, y, z, 2)).max())
    assert worst <= tol, (worst, choice)
    assert max(np.abs(got[b] - a).max() for b in boxes) > 1e-4     # the noise moved the state off rest


def test_nonfinite_populations_are_counted(weights):
    nx, ny, nz = 8, 8, 8
    n0 = random_state(weights, (nz, ny, nx), seed=70)
    n0[3, 2, 1, 0] = np.nan
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, 0.0, 0.3, 0.2, 0.0, 1, store="f32")) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_stats_sample()
        assert ctx.flb_mode_stats()["nonfinite"] == 1


# --- full size: the launch configuration the benchmark times -----------------

@pytest.mark.parametrize("store,tol", [("f32", 1e-5), ("f16dev", 4 * 2.0 ** -16)])
def test_full_size_512cube_sampled_sites(ora, store, tol):
    """512^3 AA, Kolmogorov force 1e-5, k_BT = 1e-4, gamma_s = 0.3, seed 3: two
    steps from n_eq(rho0, u(r)); 600 sampled sites are recomputed by the oracle
    one collision at a time (site r at step 2 pulls n*_i(r - c_i, 1), which
    pulls from step 0)."""
    L = 512
    kT, gs, gb, gg, seed, F0 = 1e-4, 0.3, 0.2, 0.0, 3, 1e-5
    u = smooth_velocity((L, L, L), seed=5, amp=0.01)
    cfg = flb.config(L, L, L, 1.0, kT, gs, gb, gg, seed, store=store, pattern="aa", force_amp=F0)
    sites = sample_sites(L ** 3, 600, seed=8)
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_init_velocity(u)
        ctx.flb_step(2)
        got = ctx.flb_get_sites(sites)
    c, a, _, _ = ora.lattice()
    p = ora.make_params(L, L, L, rho0=1.0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=seed,
                        force_amp=F0, store=0)
    memo = {}

    def n_at(x, y, z, t):
        """pre-collision populations at (x,y,z) and step t from the initial equilibrium"""
        key = (x % L, y % L, z % L, t)
        if key in memo:
            return memo[key]
        x, y, z = key[:3]
        if t == 0:
            val = ora.equilibrium_field(np.ones((1, 1, 1)), u[:, z, y, x].reshape(3, 1, 1, 1)).reshape(19)
            if store == "f16dev":
                val = a + np.array([ora.round_f16(v) for v in (val - a)])
        else:
            val = np.empty(19)
            for i in range(19):
                xs, ys, zs = x - c[i, 0], y - c[i, 1], z - c[i, 2]
                prev = n_at(xs, ys, zs, t - 1)
                Fx = F0 * np.sin(2 * np.pi * (zs % L) / L)
                site = (xs % L) + L * ((ys % L) + L * (zs % L))
                val[i] = ora.collide_site(p, prev, site=site, step=t - 1, force=[Fx, 0, 0])[i]
            if store == "f16dev":
                val = a + np.array([ora.round_f16(v) for v in (val - a)])
        memo[key] = val
        return val

    worst = 0.0
    for s_idx, site in enumerate(sites[:60] if store == "f16dev" else sites):
        x, y, z = site % L, (site // L) % L, site // (L * L)
        worst = max(worst, np.abs(got[s_idx] - n_at(x, y, z, 2)).max())
    assert worst <= tol
