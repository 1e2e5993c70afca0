"""Host-side analysis of the validation workloads, on synthetic series with a
known answer (no GPU): the density-autocorrelation estimator and fit behind
S(q, omega), and the Brillouin line shape."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_0707_1581_gb300 import validate


def damped_oscillator_series(rng, T, every, S, ws, G):
    """Exact sampling, every `every` time units, of the stationary Gaussian
    process dx = v dt, dv = (-ws^2 x - 2 G v) dt + noise with <x^2> = S: its
    autocorrelation is S exp(-G t)(cos(W t) + (G / W) sin(W t)), W^2 = ws^2 - G^2.
    Real and imaginary parts are independent copies, each of variance S / 2."""
    A = np.array([[0.0, 1.0], [-ws * ws, -2 * G]])
    M = expm(A * every)
    Sig = np.diag([S / 2, S * ws * ws / 2])
    Lq = np.linalg.cholesky(Sig - M @ Sig @ M.T)
    out = np.zeros(T, complex)
    for part in (1.0, 1j):
        z = np.linalg.cholesky(Sig) @ rng.standard_normal(2)
        xi = rng.standard_normal((T, 2)) @ Lq.T
        x = np.empty(T)
        for t in range(T):
            x[t] = z[0]
            z = M @ z + xi[t]
        out += part * x
    return out


def test_acf_is_unbiased_on_white_noise():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4096) + 1j * rng.standard_normal(4096)
    C = validate.density_acf(x, 5)
    assert C[0] == pytest.approx(np.mean(np.abs(x) ** 2), rel=1e-12)
    assert C[3] == pytest.approx(np.mean((x[3:] * np.conj(x[:-3])).real), rel=1e-12)
    assert np.all(np.abs(C[1:]) < 5 * math.sqrt(2 / 4096) * 2)


def test_damped_sound_fit_recovers_known_parameters():
    """q = 2 pi 3 / 64, Gamma = q^2 / 4, c_s^2 = 1/3: the same fit as the S(q, omega)
    workload recovers Omega within 1 %, Gamma within 10 % and S within 4 %
    (about four standard deviations of the estimator at 2^14 samples)."""
    q = 2 * math.pi * 3 / 64
    G, ws, every = 0.25 * q * q, q / math.sqrt(3), 4
    x = damped_oscillator_series(np.random.default_rng(3), 1 << 14, every, 2.0, ws, G)
    max_lag = int(4.0 / (G * every))
    C = validate.density_acf(x, max_lag)
    S, W, Gf, b = validate.fit_damped_sound(every * np.arange(max_lag + 1.0), C, math.sqrt(ws * ws - G * G), G)
    assert W == pytest.approx(math.sqrt(ws * ws - G * G), rel=0.01)
    assert Gf == pytest.approx(G, rel=0.10)
    assert S == pytest.approx(2.0, rel=0.04)


def test_brillouin_spectrum_sum_rule_and_peak():
    """The spectrum integrates to S over d omega / 2 pi and peaks at
    sqrt(Omega^2 - Gamma^2); it is the transform of the fitted correlation."""
    S, W, G = 1.7, 0.11, 0.01
    w = np.linspace(-40, 40, 2_000_001)
    Sw = validate.brillouin_spectrum(w, S, W, G)
    assert np.trapezoid(Sw, w) / (2 * math.pi) == pytest.approx(S, rel=1e-3)
    pos = w[w > 0][np.argmax(Sw[w > 0])]
    assert pos == pytest.approx(math.sqrt(W * W - G * G), abs=1e-4)
    t = np.arange(0, 3000.0)
    C = S * np.exp(-G * t) * (np.cos(W * t) + G / W * np.sin(W * t))
    direct = C[0] + 2 * np.sum(C[1:] * np.cos(0.09 * t[1:]))
    assert validate.brillouin_spectrum(np.array([0.09]), S, W, G)[0] == pytest.approx(direct, rel=2e-2)
