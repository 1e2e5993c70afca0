"""Physical-unit helpers of Sec. VI (host only, no GPU): they invert the
transport coefficients of Eqs. shearviscosity and bulkviscosity and give the
noise level mu = k_B T h^2 / (c_hat_s^2 b^5)."""

import pytest

from paper_0707_1581_gb300 import flb


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


@pytest.mark.parametrize("gs,gb", [(0.0, 0.0), (0.5, 0.2), (-0.7, 0.9), (0.99, -0.5)])
def test_gammas_invert_the_viscosity_formulas(gs, gb):
    b, h, rho = 2e-9, 3e-12, 1000.0
    cs2 = b * b / (3 * h * h)                         # c_s = c_hat_s b / h
    eta = h * rho * cs2 / 2 * (1 + gs) / (1 - gs)     # Eq. shearviscosity
    zeta = h * rho * cs2 / 3 * (1 + gb) / (1 - gb)    # Eq. bulkviscosity, d = 3
    got_s, got_b = flb.flb_gammas_from_viscosities(eta, zeta, rho, b, h)
    assert got_s == pytest.approx(gs, abs=1e-12)
    assert got_b == pytest.approx(gb, abs=1e-12)


def test_small_time_steps_give_over_relaxation():
    """Sec. VI: small h means eta_hat < 1/2, i.e. gamma < 0."""
    gs, gb = flb.flb_gammas_from_viscosities(1e-3, 1e-3, 1000.0, 1e-6, 1e-10)
    assert gs < 0 and gb < 0


def test_lattice_kT_matches_mu():
    kT, rho, b, h = 4.1e-21, 1000.0, 1e-8, 1e-11
    mu_phys = kT * h * h / ((1 / 3) * b ** 5)          # mass per volume, Sec. VI
    kT_lat = flb.flb_lattice_kT(kT, rho, b, h, rho0=1.0)
    # in lattice units mu = 3 kT_lattice (rho0 = 1 stands for rho)
    assert 3 * kT_lat == pytest.approx(mu_phys / rho, rel=1e-12)
    assert flb.flb_lattice_kT(kT, rho, b, h, rho0=2.0) == pytest.approx(2 * kT_lat, rel=1e-12)


def test_bad_inputs_are_rejected():
    with pytest.raises(flb.FlbError):
        flb.flb_gammas_from_viscosities(-1, 1, 1, 1, 1)
    with pytest.raises(flb.FlbError):
        flb.flb_lattice_kT(1, 1, 0, 1)
    with pytest.raises(flb.FlbError):
        flb.flb_lattice_kT(float("inf"), 1, 1, 1)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("gs,gb", [(0.0, 0.0), (0.5, 0.2), (-0.7, 0.9)])
def test_lattice_params_in_two_and_three_dimensions(d, gs, gb):
    """Eq. bulkviscosity carries 1/d: zeta = h rho c_s^2 / d (1 + gb) / (1 - gb);
    mu = k_B T h^2 / (c_hat_s^2 b^(d+2)) per unit density (Sec. VI)."""
    b, h, rho, kT = 2e-9, 3e-12, 1000.0, 4.1e-21
    cs2 = b * b / (3 * h * h)
    eta = h * rho * cs2 / 2 * (1 + gs) / (1 - gs)
    zeta = h * rho * cs2 / d * (1 + gb) / (1 - gb)
    got_s, got_b, kt = flb.flb_lattice_params(d, eta, zeta, kT, rho, b, h)
    assert got_s == pytest.approx(gs, abs=1e-12)
    assert got_b == pytest.approx(gb, abs=1e-12)
    assert 3 * kt == pytest.approx(kT * h * h / ((1 / 3) * b ** (d + 2)) / rho, rel=1e-12)
    if d == 3:
        assert (got_s, got_b) == pytest.approx(flb.flb_gammas_from_viscosities(eta, zeta, rho, b, h), abs=1e-15)
        assert kt == pytest.approx(flb.flb_lattice_kT(kT, rho, b, h), rel=1e-15)
    assert flb.flb_lattice_params(d, eta, zeta, 0.0, rho, b, h)[2] == 0.0
    with pytest.raises(flb.FlbError):
        flb.flb_lattice_params(4, eta, zeta, kT, rho, b, h)
