"""Pins of the oracle's lattice tables against what the paper fixes.

Weights and sound speed: Sec. II (Eqs. wi0-wi4, equilcond2-equilcond3, D3Q19
example).  Basis: Table II (w_k column) and the model-independent hydrodynamic
vectors of Sec. III.  Stress identities: Sec. IV (Pi_xy and Pi_yy - Pi_zz in
terms of the scaled modes 7 and 6).
"""
import itertools

import numpy as np
import pytest

from tests.golden.fixtures import read_table


@pytest.fixture(scope="module")
def lat(ora):
    c, a, e, w = ora.lattice()
    return c.astype(float), a, e, w


def test_velocity_set_is_d3q19(lat):
    c, _, _, _ = lat
    c2 = (c ** 2).sum(1)
    assert sorted(c2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert len({tuple(v) for v in c.astype(int).tolist()}) == 19
    # every velocity has its opposite in the set
    s = {tuple(v) for v in c.astype(int).tolist()}
    assert all(tuple(-x for x in v) in s for v in s)


def test_weights_match_paper(lat):
    c, a, _, _ = lat
    ref = read_table("d3q19_weights.txt")
    c2 = (c ** 2).sum(1).astype(int)
    for i in range(19):
        assert a[i] == pytest.approx(ref[f"c2={c2[i]}"], abs=1e-16)


def test_weight_moment_conditions(lat):
    """Eqs. wi0-wi4 with sigma_2 = c_s^2, sigma_4 = sigma_2^2, kappa_4 = 0."""
    c, a, _, _ = lat
    cs2 = read_table("d3q19_weights.txt")["cs2"]
    assert a.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(a @ c).max() < 1e-16
    M2 = np.einsum("i,ia,ib->ab", a, c, c)
    assert np.allclose(M2, cs2 * np.eye(3), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ig->abg", a, c, c, c)
    assert np.abs(M3).max() < 1e-15
    M4 = np.einsum("i,ia,ib,ig,id->abgd", a, c, c, c, c)
    d = np.eye(3)
    iso = np.einsum("ab,gd->abgd", d, d) + np.einsum("ag,bd->abgd", d, d) + np.einsum("ad,bg->abgd", d, d)
    # kappa_4 = 0 and sigma_4 = sigma_2^2
    assert np.allclose(M4, cs2 ** 2 * iso, atol=1e-15)


def test_table2_norms_match_paper(lat):
    _, _, _, w = lat
    ref = read_table("d3q19_table2_wk.txt")
    for k in range(19):
        assert w[k] == pytest.approx(ref[str(k)], abs=1e-15), k


def test_table2_orthogonality(lat):
    """sum_i a_i e_ki e_li = w_k delta_kl, i.e. Eq. orthogonality for the
    scaled vectors e^_ki = sqrt(a_i / w_k) e_ki (Eq. evectors_orthonormal)."""
    _, a, e, w = lat
    G = (e * a) @ e.T
    assert np.allclose(G, np.diag(w), atol=1e-15)
    ehat = np.sqrt(a)[None, :] * e / np.sqrt(w)[:, None]
    assert np.allclose(ehat @ ehat.T, np.eye(19), atol=1e-14)
    assert np.allclose(ehat.T @ ehat, np.eye(19), atol=1e-14)


def test_model_independent_hydrodynamic_vectors(lat):
    """The general-d expressions of Sec. III for the mass, momentum, bulk,
    diagonal-shear and off-diagonal-shear vectors (d = 3) equal rows 0..9 of
    the scaled Table II basis."""
    c, a, e, w = lat
    cs2 = 1.0 / 3.0
    d = 3
    ehat = np.sqrt(a)[None, :] * e / np.sqrt(w)[:, None]
    sa = np.sqrt(a)
    c2 = (c ** 2).sum(1)
    assert np.allclose(ehat[0], sa, atol=1e-15)
    for al in range(3):
        assert np.allclose(ehat[1 + al], np.sqrt(a / cs2) * c[:, al], atol=1e-15)
    bulk = (1 / cs2) * np.sqrt(a / (2 * d)) * (c2 - d * cs2)
    assert np.allclose(ehat[4], bulk, atol=1e-15)
    shear_x = (1 / cs2) * np.sqrt(a / (2 * d * (d - 1))) * (d * c[:, 0] ** 2 - c2)
    assert np.allclose(ehat[5], shear_x, atol=1e-15)
    shear_yz = sa / (2 * cs2) * (c[:, 1] ** 2 - c[:, 2] ** 2)
    assert np.allclose(ehat[6], shear_yz, atol=1e-15)
    for k, (p, q) in zip((7, 8, 9), ((0, 1), (1, 2), (2, 0))):
        assert np.allclose(ehat[k], sa / cs2 * c[:, p] * c[:, q], atol=1e-15)


def test_ghost_rows_orthogonal_to_quadratic_polynomials(lat):
    """Kinetic modes (k >= 10) are orthogonal, with weights a_i, to every
    polynomial of degree <= 2 in c_i, so any equilibrium of the form of
    Eq. derived_equil_distrib has no projection on them (Sec. V)."""
    c, a, e, _ = lat
    polys = [np.ones(19)] + [c[:, k] for k in range(3)] + \
        [c[:, p] * c[:, q] for p, q in itertools.combinations_with_replacement(range(3), 2)]
    for k in range(10, 19):
        for P in polys:
            assert abs(np.sum(a * e[k] * P)) < 1e-15


def test_stress_modes_give_stress_tensor(lat):
    """Sec. IV: Pi_xy = sqrt(mu rho) c_s^2 m^_7 and Pi_yy - Pi_zz =
    2 sqrt(mu rho) c_s^2 m^_6 for the scaled modes m^_k = sum_i e^_ki x_i."""
    c, a, e, w = lat
    rng = np.random.default_rng(3)
    mu, rho, cs2 = 3e-4, 1.1, 1.0 / 3.0
    x = rng.standard_normal(19)
    nneq = np.sqrt(mu * rho * a) * x                       # Eq. xdef
    ehat = np.sqrt(a)[None, :] * e / np.sqrt(w)[:, None]
    mhat = ehat @ x                                        # Eq. modes
    Pi = np.einsum("i,ia,ib->ab", nneq, c, c)
    assert Pi[0, 1] == pytest.approx(np.sqrt(mu * rho) * cs2 * mhat[7], rel=1e-13)
    assert Pi[1, 1] - Pi[2, 2] == pytest.approx(2 * np.sqrt(mu * rho) * cs2 * mhat[6], rel=1e-13)


def test_inverse_transform_is_identity(lat):
    """n_i = a_i sum_k e_ki m_k / w_k inverts m_k = sum_i e_ki n_i (Eq. x_s with
    Eq. evectors_orthonormal)."""
    _, a, e, w = lat
    rng = np.random.default_rng(1)
    n = rng.random(19)
    m = e @ n
    back = a * (e.T @ (m / w))
    assert np.allclose(back, n, atol=1e-15)
