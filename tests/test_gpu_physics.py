"""Statistical and hydrodynamic acceptance on the GPU (reduced sizes of the
validation workloads): what the paper fixes for the stationary state and the
hydrodynamic limit, for every storage format."""
import numpy as np
import pytest

from paper_0707_1581_gb300 import validate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


@pytest.mark.parametrize("store", ["f64", "f32", "f16dev", "bf16dev", "bf16sr"])
def test_equipartition_every_mode_within_one_percent(store):
    """32^3, k_BT = 1e-4: every non-conserved mode variance within 1 % of
    mu rho0 w_k (Eq. modeprob), <u^2> rho0 / k_BT and S(q)/(mu rho0) within 2 %."""
    r = validate.equipartition(32, store=store, kT=1e-4, gamma_shear=0.5, steps=3000, burn=300, every=10)
    ratios = np.array(r["mode_ratio"])
    assert r["nonfinite"] == 0
    assert np.max(np.abs(ratios[4:] - 1)) < 0.01, ratios
    assert np.max(np.abs(ratios[:4] - 1)) < 0.03, ratios       # slow hydrodynamic modes: fewer independent samples
    assert np.max(np.abs(np.array(r["u2_ratio"]) - 1)) < 0.03
    assert abs(r["S_ratio_mean"] - 1) < 0.02
    # each step rounds every stored deviation n - rho0 a_i: the total mass random-walks
    bound = {"f64": 1e-12, "f32": 1e-8, "f16dev": 1e-4, "bf16dev": 1e-3, "bf16sr": 1e-3}[store]
    assert abs(r["mass_drift_rel"]) < bound


def test_shear_viscosity_from_decay():
    """k_BT = 0, L = 64, gamma_s = 0.5: nu_eff within 0.5 % of Eq. shearviscosity
    (the lattice correction is O(q^2) ~ 0.3 % here)."""
    r = validate.shear_wave(64, store="f32", kT=0.0, gamma_shear=0.5)
    assert abs(r["rel_err"]) < 0.005, r["rel_err"]


@pytest.mark.parametrize("store", ["f32", "f16dev"])
def test_kolmogorov_flow_amplitude(store):
    """F_x = F0 sin(k z), 32 x 32 x 128, 4000 steps, k_BT = 1e-4: the amplitude
    of u_x(z) within 2 % of the Navier-Stokes solution (thermal noise of the
    projected amplitude ~0.3 %, lattice correction O(k^2) ~ 0.1 %)."""
    r = validate.kolmogorov(128, store=store, steps=4000, cross=32, F0=1e-5)
    assert abs(r["rel_err"]) < 0.02, r


def test_ensemble_batch_equipartition():
    r = validate.ensemble(n_replicas=4, L=32, n_mixed=4, steps=1200, burn=200, every=10, graph_steps=10)
    assert r["boxes"] == 8
    assert r["mode_ratio_max_abs_dev_from_1"] < 0.02
    assert r["mlups_stepping"] > 0


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_sound_wave_speed_and_attenuation(store):
    """A standing density wave (k_BT = 0, L = 64, gamma_s = gamma_b = 0.2):
    speed c_s = sqrt(1/3) (Sec. II) and attenuation (4/3 nu + zeta/rho) q^2 / 2
    with Eqs. shearviscosity and bulkviscosity; the lattice's own correction at
    this q is +0.18 % (exact eigenvalue of the linear one-step operator)."""
    r = validate.sound_wave(64, store=store, drho=1e-4)
    assert abs(r["cs_rel_err"]) < 0.002, r
    assert abs(r["Gamma_rel_err"]) < 0.01, r


def test_stress_only_thermalisation_fails_at_short_scales():
    """Sec. IV: thermalizing every non-conserved mode gives equipartition on all
    scales; noise on the stress modes only leaves the kinetic modes cold, and the
    density fluctuations S(q) fall below mu rho0 at large q while the longest
    waves stay thermalized."""
    r = validate.thermalization_variants(32, steps=2000, burn=300, every=10)
    full, old = r["all_modes"], r["stress_only"]
    assert np.max(np.abs(np.array(full["mode_ratio"][4:]) - 1)) < 0.01
    S_full = np.array(full["S_ratio_shells"])
    assert np.max(np.abs(S_full[:-1] - 1)) < 0.05        # the corner shell has few wave vectors
    S_old = np.array(old["S_ratio_shells"])
    assert abs(S_old[0] - 1) < 0.1                        # longest wavelengths
    assert np.max(S_old[-8:]) < 0.5                       # shortest wavelengths under-thermalized
    assert np.max(np.array(old["mode_ratio"][10:])) < 0.6  # kinetic modes far below equipartition


def _sound_eigenvalue(ora, q, gs, gb, gg):
    """Sound pair of the linearised one-step operator at wave vector (0, 0, q):
    the eigenvalue with the largest density overlap, as (Omega, Gamma) with
    lambda = exp(-Gamma +- i Omega)."""
    from tests.test_oracle_box import one_step_linear_operator
    c, a = ora.lattice()[:2]
    lam, V = np.linalg.eig(one_step_linear_operator(c.astype(float), a, np.array([0.0, 0.0, q]), gs, gb, gg))
    overlap = np.abs(V.sum(0)) / np.linalg.norm(V, axis=0)
    k = np.argmax(overlap * (np.abs(lam) > 0.5))
    return abs(np.angle(lam[k])), -np.log(abs(lam[k]))


def test_dynamic_structure_factor_brillouin_peaks(ora):
    """Sec. V (Eqs. ce11-ce12, mpeos): at k_BT = 1e-4 the density autocorrelation
    at q = 2 pi n / 64 (n = 2, 3) is a damped sound mode whose frequency and
    damping are the exact sound eigenvalue of the linearised lattice operator,
    and whose equal-time value is S(q) = mu rho0.  2^16 samples every 4 steps:
    the estimator's spread (Monte Carlo of the same fit on a synthetic damped
    oscillator) is 0.3 % in Omega, 3 % / 2 % in Gamma and 2 % / 0.6 % in S."""
    gs = gb = 0.2
    r = validate.dynamic_structure_factor(L=64, cross=8, kT=1e-4, gamma_shear=gs, gamma_bulk=gb, samples=1 << 16,
                                          every=4, nq=3)
    for m, tol_G in zip(r["modes"][1:], (0.15, 0.10)):
        W, G = _sound_eigenvalue(ora, m["q"], gs, gb, 0.0)
        assert abs(m["Omega_fit"] / W - 1) < 0.015, (m, W)
        assert abs(m["Gamma_fit"] / G - 1) < tol_G, (m, G)
        assert abs(m["S_static_ratio"] - 1) < 0.08, m
        assert abs(m["S_fit_ratio"] - 1) < 0.08, m


def test_stochastic_rounding_keeps_a_slow_shear_wave_decaying():
    """k_BT = 0, u_x = 1e-3 sin(2 pi z / 256), 2000 steps: with bfloat16 nearest
    rounding the wave freezes (each step's change is ~0.05 ulp); with
    stochastic rounding it decays as exp(-nu q^2 t) (Eq. shearviscosity) like
    the FP64 kernel."""
    r = validate.rounding_shear_wave(256, steps=2000, stores=("f64", "bf16dev", "bf16sr"))
    assert abs(r["f64"]["rel_err"]) < 0.003, r
    assert r["bf16dev"]["amplitude_ratio"] > 0.99, r
    assert r["bf16sr"]["amplitude_ratio"] == pytest.approx(r["f64"]["amplitude_ratio"], rel=0.01), r


def test_batched_fp16_ensemble_beats_the_single_box_fp32_kernel():
    """The ensemble workload (64 replicas of 64^3 and 16 cubes of 32..128,
    28.3 M sites) in FP16 deviations, batched and autotuned, steps more sites
    per second than one 512^3 FP32 box, and keeps every mode ratio of every
    box within 1 % of 1."""
    import time
    import torch
    from paper_0707_1581_gb300 import flb
    r = validate.ensemble(steps=600, burn=100, every=50, store="f16dev")
    assert r["mode_ratio_max_abs_dev_from_1"] < 0.01, r
    s = torch.cuda.Stream()
    with flb.flb_create_ex(flb.config(512, 512, 512, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, store="f32", pattern="aa",
                                      force_amp=1e-5, stream=s)) as ctx:
        ctx.flb_step(6)
        ctx.flb_sync()
        t0 = time.perf_counter()
        ctx.flb_step(40)
        ctx.flb_sync()
        single = 512 ** 3 * 40 / (time.perf_counter() - t0) / 1e6
    assert r["mlups_stepping"] > 1.05 * single, (r["mlups_stepping"], single)


def test_thermal_shear_wave_decay_over_replicas():
    """Config 2 at k_BT = 1e-4: the shear wave u0 = 1e-3 sin(2 pi z / 64) averaged
    over 128 replicas (independent noise) decays with Eq. shearviscosity to
    within 2 % (sampling error ~0.7 %, lattice O(q^2) term 0.3 %)."""
    r = validate.shear_wave(64, kT=1e-4, cross=64, t_fit=(20, 300), replicas=128)
    assert abs(r["rel_err"]) < 0.02, r["rel_err"]


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_finite_time_mode_variances_from_rest_follow_the_linear_recursion(ora, store):
    """From rest, every mode variance of the device chain follows, step by step,
    the exact covariance recursion of the linearised chain per Fourier mode
    (collision projectors, noise covariance of Eq. FDT, push streaming): 64
    replicas of 16 x 12 x 10 in one batch, config 1 parameters, 24 steps,
    within 5 standard errors over the replicas."""
    from paper_0707_1581_gb300 import flb
    from tests.test_oracle_box import mode_variance_recursion
    c, a, e, w = ora.lattice()
    nx, ny, nz = 16, 12, 10
    kT, rho0, gs, gb, gg, T, nrep = 1e-4, 1.0, 0.2, 0.2, 0.0, 24, 64
    pred = mode_variance_recursion(c.astype(float), a, e, w, (nx, ny, nz), kT, rho0, gs, gb, gg, T)
    cfgs = [flb.config(nx, ny, nz, rho0, kT, gs, gb, gg, 1, replica=r, store=store) for r in range(nrep)]
    obs = np.zeros((nrep, T, 19))
    with flb.flb_create_batch(cfgs) as ctx:
        for t in range(T):
            ctx.flb_step(1)
            ctx.flb_stats_reset()
            ctx.flb_stats_sample()
            for b in range(nrep):
                obs[b, t] = ctx.flb_mode_stats(box=b)["mode_ratio"]
    mean = obs.mean(0)
    se = obs.std(0, ddof=1) / np.sqrt(nrep)
    assert np.all(np.abs(mean - pred) < 5 * se + 2e-3), np.abs(mean - pred) / (se + 1e-12)
