"""Pins of the oracle's stochastic collision (Sec. IV) against what the paper
and the mathematics fix, each independent of the Table II matrices that the
oracle uses internally:

* mass and momentum conservation (Eq. conservationlaws);
* at k_B T = 0 with one eigenvalue for every mode, the textbook BGK rule
  n* = n^eq + gamma (n - n^eq) with n^eq of Eq. derived_equil_distrib;
* at k_B T = 0, the stress update rules Eqs. stress_updaterule1-2 (R = 0), and
  the kinetic-mode part relaxing by gamma_ghost, with every subspace built
  by a weighted projection onto polynomials in c_i (no Table II);
* one collision from rest equilibrium gives the random-stress covariance of
  Eq. stressfluctuations_microscopic;
* on a 1x1x1 periodic box (streaming is the identity) the chain is linear,
  and its stationary law is x_i = n^neq_i / sqrt(mu rho0 a_i) with
  covariance I - (projection on the conserved modes) (Eqs. probdistfluct2,
  modeprob, detailedbalance); lag-1 stress correlations equal gamma (Eq. langevin);
* the two thermalisation variants: with the local-density switch one
  collision from rest has noise covariance proportional to the local rho
  (Sec. III, the population variance mu rho a_i), without it to rho0; with
  stress-only noise (Sec. IV) the kinetic modes carry no noise, decay as
  gamma_ghost^t on a 1x1x1 box, and the stationary covariance is the
  stress and bulk block alone.
"""
import numpy as np
import pytest

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def lat(ora):
    c, a, e, w = ora.lattice()
    return c.astype(float), a, e, w


def neq_paper(rho, u, c, a):
    """Eq. derived_equil_distrib written out with sigma_2 = 1/3."""
    cu = c @ u
    return rho * a * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))


def random_state(rng, c, a, rho0=1.0, amp=0.05):
    n = rho0 * a * (1 + amp * rng.standard_normal(19))
    return n


def subspace_projectors(c, a):
    """Projectors in population space, orthogonal in <n, n'> = sum n_i n'_i / a_i,
    onto: conserved {a, a c_alpha}, bulk {a (c^2 - 3 c_s^2)}, traceless shear
    {a (c_a c_b - delta_ab c^2/3)}, and the remaining kinetic part."""
    W = np.diag(1 / a)

    def proj(cols):
        H = np.stack(cols, 1)
        return H @ np.linalg.solve(H.T @ W @ H, H.T @ W)

    c2 = (c ** 2).sum(1)
    cons = [a] + [a * c[:, k] for k in range(3)]
    bulk = [a * (c2 - 3 * CS2)]
    shear = [a * (c[:, 0] ** 2 - c[:, 1] ** 2), a * (c[:, 1] ** 2 - c[:, 2] ** 2),
             a * c[:, 0] * c[:, 1], a * c[:, 1] * c[:, 2], a * c[:, 2] * c[:, 0]]
    Pc, Pb, Ps = proj(cons), proj(bulk), proj(shear)
    Pall = proj(cons + bulk + shear)
    Pg = np.eye(19) - Pall
    return Pc, Pb, Ps, Pg


def test_conservation_per_collision(ora, lat):
    c, a, _, _ = lat
    rng = np.random.default_rng(0)
    for trial in range(50):
        p = ora.make_params(1, 1, 1, rho0=1.0, kT=1e-3, gamma_shear=rng.uniform(-1, 1),
                            gamma_bulk=rng.uniform(-1, 1), gamma_ghost=rng.uniform(-1, 1), seed=trial)
        n = random_state(rng, c, a)
        ns = ora.collide_site(p, n, site=trial, step=3)
        assert ns.sum() == pytest.approx(n.sum(), abs=1e-14)
        assert np.allclose(ns @ c, n @ c, atol=1e-15)
        assert not np.allclose(ns, n)


def test_bgk_reduction_at_zero_temperature(ora, lat):
    c, a, _, _ = lat
    rng = np.random.default_rng(1)
    for gam in (-0.7, 0.0, 0.2, 0.5, 0.95):
        p = ora.make_params(1, 1, 1, kT=0.0, gamma=np.r_[np.ones(4), np.full(15, gam)])
        for _ in range(10):
            n = random_state(rng, c, a, rho0=rng.uniform(0.5, 2.0), amp=0.1)
            rho = n.sum()
            u = (n @ c) / rho
            neq = neq_paper(rho, u, c, a)
            expect = neq + gam * (n - neq)
            assert np.allclose(ora.collide_site(p, n), expect, rtol=0, atol=1e-15)


def test_stress_and_kinetic_relaxation_at_zero_temperature(ora, lat):
    """Eqs. stress_updaterule1-2 with R = 0: traceless Pi^neq scales by gamma_s,
    its trace by gamma_b; the kinetic part scales by gamma_ghost."""
    c, a, _, _ = lat
    _, _, _, Pg = subspace_projectors(c, a)
    rng = np.random.default_rng(2)
    gs, gb, gg = 0.3, -0.4, 0.65
    p = ora.make_params(1, 1, 1, kT=0.0, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg)
    for _ in range(20):
        n = random_state(rng, c, a, amp=0.1)
        ns = ora.collide_site(p, n)
        rho = n.sum()
        u = (n @ c) / rho
        Peq = rho * CS2 * np.eye(3) + rho * np.outer(u, u)          # Euler stress, Sec. II
        Pneq = np.einsum("i,ia,ib->ab", n, c, c) - Peq
        Pneq_s = np.einsum("i,ia,ib->ab", ns, c, c) - Peq
        tr, tr_s = np.trace(Pneq), np.trace(Pneq_s)
        bar = Pneq - tr / 3 * np.eye(3)
        bar_s = Pneq_s - tr_s / 3 * np.eye(3)
        assert np.allclose(bar_s, gs * bar, atol=1e-15)
        assert tr_s == pytest.approx(gb * tr, abs=1e-15)
        assert np.allclose(Pg @ ns, gg * (Pg @ n), atol=1e-15)


def test_random_stress_covariance_single_collision(ora, lat):
    """Eq. stressfluctuations_microscopic: from a site at rest equilibrium one
    collision gives Pi*^neq = R with <R_ab R_cd> / (mu rho c_s^4) =
    (1 - gs^2)(d_ac d_bd + d_ad d_bc) + (2/3)(gs^2 - gb^2) d_ab d_cd."""
    c, a, _, _ = lat
    nx = ny = nz = 64
    N = nx * ny * nz
    kT, gs, gb, rho0 = 1e-4, 0.35, -0.2, 1.0
    mu = 3 * kT
    p = ora.make_params(nx, ny, nz, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=0.1, seed=21)
    n = ora.rest_state(nx, ny, nz, rho0)
    ns = ora.collide_field(p, n, step=4).reshape(19, N)
    Pi = np.einsum("in,ia,ib->abn", ns, c, c) - (rho0 * CS2 * np.eye(3))[:, :, None]
    R = Pi.reshape(9, N)
    C = R @ R.T / N
    d = np.eye(3)
    expect = (1 - gs ** 2) * (np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) \
        + (2 / 3) * (gs ** 2 - gb ** 2) * np.einsum("ab,cd->abcd", d, d)
    expect = expect.reshape(9, 9) * mu * rho0 * CS2 ** 2
    # standard error of a sample second moment of a Gaussian pair: sqrt((s_aa s_bb + s_ab^2) / N)
    diag = np.diag(expect)
    se = np.sqrt((np.outer(diag, diag) + expect ** 2) / N)
    assert np.all(np.abs(C - expect) < 5 * se + 1e-30)


def test_single_site_stationary_covariance_and_ar1(ora, lat):
    """1x1x1 box: the collision is exactly linear (rho, j fixed), so the
    stationary covariance of n is mu rho0 sqrt(a_i a_j) (delta_ij -
    sqrt(a_i a_j)(1 + c_i.c_j / c_s^2)), and Pi_xy, trace Pi and the
    kinetic part are AR(1) with coefficients gamma_s, gamma_b, gamma_ghost."""
    c, a, _, _ = lat
    kT, gs, gb, gg, rho0 = 1e-4, 0.4, 0.1, -0.3, 1.0
    mu = 3 * kT
    nrep, nsteps, burn = 16, 12000, 50
    samples = []
    for rep in range(nrep):
        p = ora.make_params(1, 1, 1, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg,
                            seed=77, replica=rep)
        tr = ora.run_trace(p, ora.rest_state(1, 1, 1, rho0), 0, nsteps).reshape(nsteps, 19)
        samples.append(tr[burn:])
    X = np.stack(samples)                      # [rep, t, 19]
    D = X - rho0 * a
    flat = D.reshape(-1, 19)
    Ns = flat.shape[0]
    C = flat.T @ flat / Ns
    sa = np.sqrt(a)
    expect = mu * rho0 * np.outer(sa, sa) * (np.eye(19) - np.outer(sa, sa) * (1 + (c @ c.T) / CS2))
    # samples are nearly independent (|gamma| <= 0.4); bound by 6 standard errors
    dg = np.diag(expect)
    se = np.sqrt((np.outer(dg, dg) + expect ** 2) / Ns)
    assert np.all(np.abs(C - expect) < 6 * se + 1e-18)
    # conserved quantities drift only by rounding: at most ~1e-15 per step
    assert np.abs(D.sum(-1)).max() < 1e-15 * nsteps
    assert np.abs(D @ c).max() < 1e-15 * nsteps

    def lag1(s):
        s0, s1 = s[:, :-1].reshape(-1), s[:, 1:].reshape(-1)
        return np.mean(s0 * s1) / np.mean(s0 * s0)

    Pxy = np.einsum("rti,i->rt", D, c[:, 0] * c[:, 1])
    trP = np.einsum("rti,i->rt", D, (c ** 2).sum(1))
    assert lag1(Pxy) == pytest.approx(gs, abs=0.03)
    assert lag1(trP) == pytest.approx(gb, abs=0.03)
    _, _, _, Pg = subspace_projectors(c, a)
    G = np.einsum("ij,rtj->rti", Pg, D)
    num = np.sum(G[:, 1:] * (G[:, :-1] / a), axis=(0, 1, 2))
    den = np.sum(G[:, :-1] * (G[:, :-1] / a), axis=(0, 1, 2))
    assert num / den == pytest.approx(gg, abs=0.03)


def test_deterministic_limit_has_no_noise(ora, lat):
    """phi_k = 0 for every mode at k_B T = 0 (end of Sec. IV): two different
    seeds give the identical post-collision state."""
    c, a, _, _ = lat
    rng = np.random.default_rng(4)
    n = random_state(rng, c, a)
    p1 = ora.make_params(1, 1, 1, kT=0.0, gamma_shear=0.3, gamma_bulk=0.2, seed=1)
    p2 = ora.make_params(1, 1, 1, kT=0.0, gamma_shear=0.3, gamma_bulk=0.2, seed=2)
    assert np.array_equal(ora.collide_site(p1, n, 5, 9), ora.collide_site(p2, n, 5, 9))


def test_gamma_plus_minus_one_gives_no_noise(ora, lat):
    """phi = (1 - gamma^2)^(1/2) = 0 at |gamma| = 1 (Eq. FDT)."""
    c, a, _, _ = lat
    n = a.copy()
    p = ora.make_params(1, 1, 1, kT=1e-3, gamma=np.r_[np.ones(4), np.ones(6), -np.ones(9)], seed=3)
    ns = ora.collide_site(p, n, 0, 0)
    assert np.allclose(ns, n, atol=1e-16)


def _one_collision_covariance(ora, p, rho_field):
    """Collides every site of a rest state n_i = rho(r) a_i once and returns
    the post-collision deviations n* - rho a_i as [19, N]."""
    c, a, _, _ = ora.lattice()
    nz, ny, nx = rho_field.shape
    n = ora.equilibrium_field(rho_field, np.zeros((3, nz, ny, nx)))
    ns = ora.collide_field(p, n, step=2)
    return (ns - n).reshape(19, -1)


def _within_se(C, expect, N, k):
    dg = np.clip(np.diag(expect), 0.0, None)
    se = np.sqrt((np.outer(dg, dg) + expect ** 2) / N)
    return np.abs(C - expect) < k * se + 1e-30


def test_local_density_noise_variance_scales_with_the_local_density(ora, lat):
    """Sec. III: the variance of a population, mu rho a_i at low velocity, is
    taken at the local density when the switch is set.  From a site at rest
    with density rho (n_i = rho a_i, u = 0) the equilibrium is unchanged by
    the collision, so n* - rho a is pure noise with covariance
    mu rho_var sum_s (1 - gamma_s^2) P_s diag(a) over the bulk, shear and
    kinetic subspaces (weighted projections onto polynomials in c_i, no
    Table II), rho_var = rho(r) for the local switch and rho0 without it.
    Two half-boxes of density 0.7 rho0 and 1.3 rho0 are checked separately,
    so a variance linear in rho0 but not in rho, or one growing like rho^2
    (a misplaced square root), fails by many standard errors."""
    c, a, _, _ = lat
    _, Pb, Ps, Pg = subspace_projectors(c, a)
    nx = ny = nz = 48
    kT, rho0, gs, gb, gg = 1e-4, 1.0, 0.3, -0.25, 0.15
    mu = 3 * kT
    rho = np.full((nz, ny, nx), 0.7 * rho0)
    rho[nz // 2:] = 1.3 * rho0
    half = nx * ny * (nz // 2)
    shape = ((1 - gs ** 2) * Ps + (1 - gb ** 2) * Pb + (1 - gg ** 2) * Pg) @ np.diag(a)
    for local in (True, False):
        p = ora.make_params(nx, ny, nz, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg,
                            seed=31, noise_rho_local=local)
        D = _one_collision_covariance(ora, p, rho)
        # mass and momentum untouched at every site
        assert np.abs(D.sum(0)).max() < 1e-15
        assert np.abs(c.T @ D).max() < 1e-15
        for sl, r in ((slice(0, half), 0.7 * rho0), (slice(half, 2 * half), 1.3 * rho0)):
            X = D[:, sl]
            C = X @ X.T / X.shape[1]
            expect = mu * (r if local else rho0) * shape
            assert np.all(_within_se(C, expect, X.shape[1], 5)), (local, r)
            wrong = mu * (rho0 if local else r) * shape
            assert not np.all(_within_se(C, wrong, X.shape[1], 5)), (local, r)


def test_stress_only_thermalisation_leaves_the_kinetic_modes_cold(ora, lat):
    """Sec. IV, stress-only noise (the kinetic modes relax without noise):
    (i) one collision from rest gives n* - rho0 a with covariance
    mu rho0 ((1 - gamma_s^2) P_s + (1 - gamma_b^2) P_b) diag(a), and no
    kinetic content at all; (ii) on a 1x1x1 periodic box (streaming is the
    identity) a kinetic perturbation decays as gamma_ghost^t to zero while the
    stress and bulk modes reach their equipartition value: the stationary
    covariance is mu rho0 (P_s + P_b) diag(a), against mu rho0 (I - P_c) diag(a)
    when every mode is thermalised."""
    c, a, _, _ = lat
    Pc, Pb, Ps, Pg = subspace_projectors(c, a)
    kT, rho0, gs, gb, gg = 1e-4, 1.0, 0.35, 0.1, 0.5
    mu = 3 * kT
    nx = ny = nz = 48
    p = ora.make_params(nx, ny, nz, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg,
                        seed=41, noise_ghosts=False)
    D = _one_collision_covariance(ora, p, np.full((nz, ny, nx), rho0))
    assert np.abs(Pg @ D).max() < 1e-16
    C = D @ D.T / D.shape[1]
    expect = mu * rho0 * ((1 - gs ** 2) * Ps + (1 - gb ** 2) * Pb) @ np.diag(a)
    assert np.all(_within_se(C, expect, D.shape[1], 5))

    # (ii) the single-site chain, started with a kinetic perturbation
    rng = np.random.default_rng(12)
    kick = Pg @ (a * 0.05 * rng.standard_normal(19))
    nrep, nsteps, burn = 12, 8000, 60
    samples, first = [], []
    for rep in range(nrep):
        p1 = ora.make_params(1, 1, 1, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg,
                             seed=43, replica=rep, noise_ghosts=False)
        n0 = ora.rest_state(1, 1, 1, rho0).reshape(19) + kick
        tr = ora.run_trace(p1, n0.reshape(19, 1, 1, 1), 0, nsteps).reshape(nsteps, 19)
        first.append(tr[:8] - rho0 * a)
        samples.append(tr[burn:] - rho0 * a)
    # the kinetic part is deterministic: exactly gamma_ghost^t times the kick
    for t in range(8):
        for f in first:
            assert np.allclose(Pg @ f[t], gg ** (t + 1) * kick, rtol=0, atol=1e-16)
    X = np.concatenate(samples).T
    assert np.abs(Pg @ X).max() < 1e-16 + 0.05 * gg ** burn
    C = X @ X.T / X.shape[1]
    stationary = mu * rho0 * (Ps + Pb) @ np.diag(a)
    assert np.all(_within_se(C, stationary, X.shape[1], 6))
    all_modes = mu * rho0 * (np.eye(19) - Pc) @ np.diag(a)
    assert not np.all(_within_se(C, all_modes, X.shape[1], 6))
