"""Pins of the stochastic bfloat16 rounding of the oracle (store format 4).

The paper has no storage format; stochastic rounding is the storage option
whose rounding error has zero mean.  Pinned by what the definition fixes:
values already in bfloat16 are kept, the mean over all 2^16 random values is
the binary32 input exactly, the round-up probability is (low 16 bits) / 2^16,
non-finite values pass through, the random values are the documented words
of Philox blocks 2..4, and one oracle step averaged over seeds matches the
unrounded FP64 step to the sampling error while nearest rounding keeps a
fixed error.
"""
import numpy as np
import pytest


def f32_bits(x):
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def from_bits(b):
    return float(np.array([b], dtype=np.uint32).view(np.float32)[0])


def test_representable_values_are_kept(ora):
    rng = np.random.default_rng(0)
    for _ in range(200):
        x = from_bits(f32_bits(rng.standard_normal() * 10.0 ** rng.integers(-8, 3)) & 0xFFFF0000)
        for r in (0, 1, 0x7FFF, 0xFFFF, int(rng.integers(0, 65536))):
            assert ora.sr_bf16(x, r) == x


@pytest.mark.parametrize("x", [1.0 + 2 ** -12, -3.7e-3, 1.234567e-5, -0.4999, 6.1e-39])
def test_mean_over_all_random_values_is_exact(ora, x):
    xf = float(np.float32(x))
    vals = np.array([ora.sr_bf16(xf, r) for r in range(65536)])
    lo, hi = vals.min(), vals.max()
    up = (f32_bits(xf) & 0xFFFF)
    assert np.sum(vals == (hi if xf > 0 else lo)) == up            # away from zero with probability low16 / 2^16
    assert np.sum(vals) / 65536 == pytest.approx(xf, rel=0, abs=abs(xf) * 1e-15 + 1e-300)
    assert len(np.unique(vals)) <= 2


def test_non_finite_values_pass_through(ora):
    assert ora.sr_bf16(np.inf, 0xFFFF) == np.inf
    assert ora.sr_bf16(-np.inf, 1) == -np.inf
    assert np.isnan(ora.sr_bf16(np.nan, 5))


def test_random_values_are_philox_blocks_two_to_four(ora):
    seed, site, step, rep = 0x1234_5678_9ABC, 77, 12, 3
    r = ora.sr_bits(seed, site, step, rep)
    for p in range(24):
        w = ora.philox([[site, step, rep, 2 + p // 8]], [[seed & 0xFFFFFFFF, seed >> 32]])[0][(p % 8) // 2]
        assert r[p] == (int(w) >> (16 * (p % 2))) & 0xFFFF


def test_one_step_is_unbiased_over_seeds(ora):
    """k_BT = 0 (the seed only keys the rounding): the mean over 96 seeds of one
    stochastically rounded step equals the FP64 step to the sampling error,
    while nearest rounding keeps its deterministic error."""
    nx = ny = nz = 4
    c, a, _, _ = ora.lattice()
    rng = np.random.default_rng(1)
    n0 = a[:, None, None, None] * (1 + 0.03 * rng.standard_normal((19, nz, ny, nx)))
    n0 = ora.quantize(ora.make_params(nx, ny, nz, store=ora.STORE_BF16DEV), n0)   # start on the bf16 grid
    exact = ora.run(ora.make_params(nx, ny, nz, kT=0.0, gamma_shear=0.3, gamma_bulk=0.1), n0, 0, 1)
    rne = ora.run(ora.make_params(nx, ny, nz, kT=0.0, gamma_shear=0.3, gamma_bulk=0.1, store=ora.STORE_BF16DEV),
                  n0, 0, 1)
    runs = np.stack([ora.run(ora.make_params(nx, ny, nz, kT=0.0, gamma_shear=0.3, gamma_bulk=0.1, seed=s,
                                             store=ora.STORE_BF16SR), n0, 0, 1) for s in range(96)])
    dev = np.abs(exact - a[:, None, None, None])
    ulp = 2.0 ** (np.floor(np.log2(np.maximum(dev, 1e-30))) - 7)
    err_sr = (runs.mean(0) - exact) / ulp
    err_rne = (rne - exact) / ulp
    # per value the SR mean has standard deviation <= 0.5 ulp / sqrt(96)
    assert np.abs(err_sr).max() < 6 * 0.5 / np.sqrt(96)
    assert np.abs(err_sr.mean()) < 0.01
    assert np.abs(err_rne).mean() > 0.2          # nearest rounding: a fixed error of ~1/4 ulp on average
    # every stochastic result is one of the two bfloat16 neighbours of the exact value
    assert np.all(np.abs(runs - exact) <= ulp * 1.0000001)


def test_slow_shear_wave_freezes_with_nearest_and_decays_with_stochastic_rounding(ora):
    """A shear wave u_x = 1e-3 sin(2 pi z / 256) at k_BT = 0 changes each
    bfloat16 deviation by ~0.05 ulp per step: nearest rounding returns every
    value to where it was and the wave never decays, while stochastic rounding
    follows the FP64 decay exp(-nu q^2 t) (Eq. shearviscosity)."""
    L, u0, gs = 256, 1e-3, 0.5
    nu, q = (1 + gs) / (6 * (1 - gs)), 2 * np.pi / L
    z = np.arange(L)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = u0 * np.sin(q * z)
    n0 = ora.quantize(ora.make_params(1, 1, L, store=ora.STORE_BF16DEV), ora.equilibrium_field(np.ones((L, 1, 1)), u))
    c = ora.lattice()[0].astype(float)

    def amp(n):
        return (2 / L) * np.sum((np.tensordot(c[:, 0], n, axes=(0, 0)) / n.sum(0))[:, 0, 0] * np.sin(q * z))

    out = {}
    for store in (0, ora.STORE_BF16DEV, ora.STORE_BF16SR):
        p = ora.make_params(1, 1, L, kT=0.0, gamma_shear=gs, gamma_bulk=0.2, store=store, seed=5)
        out[store] = amp(ora.run(p, n0, 0, 2000)) / amp(n0)
    expect = np.exp(-nu * q * q * 2000)
    assert out[0] == pytest.approx(expect, rel=2e-3)
    assert out[ora.STORE_BF16DEV] > 0.99
    assert out[ora.STORE_BF16SR] == pytest.approx(out[0], rel=0.01)
