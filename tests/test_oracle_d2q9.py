"""Pins of the D2Q9 oracle (Table I) against what the paper and the
mathematics fix, independent of the oracle's own Table I matrices:

* the weights are the unique solution of Eqs. wi0-wi4 on speeds 0, 1, sqrt 2
  with sigma_2 = c_s^2 = 1/3 (Sec. VI: c_s^2 = 1/3 for D2Q9) and an isotropic
  fourth moment; the w_k column of Table I;
* mass and momentum conservation; the BGK limit and Guo forcing at equal
  eigenvalues; Eqs. stress_updaterule1-2 at k_B T = 0;
* Eq. stressfluctuations_microscopic with d = 2 for one collision from rest;
* the linear invariant measure (equipartition, <u^2> = k_B T / rho0, flat S(k));
* shear and sound eigenvalues of the linearised one-step operator, with
  Eq. shearviscosity and Eq. bulkviscosity at d = 2.
"""
import numpy as np
import pytest

from tests.golden.fixtures import read_table

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def D():
    from oracle import d2q9
    return d2q9


@pytest.fixture(scope="module")
def lat(D):
    c, a, e, w = D.lattice()
    return c.astype(float), a, e, w


def neq2(rho, u, c, a):
    cu = c @ u
    return rho * a * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))


def test_velocity_set_and_opposites(lat):
    c, _, _, _ = lat
    assert sorted((c ** 2).sum(1).tolist()) == [0] + [1] * 4 + [2] * 4
    ci = c.astype(int)
    assert len({tuple(v) for v in ci.tolist()}) == 9
    for i in range(1, 9, 2):
        assert np.array_equal(ci[i], -ci[i + 1])


def test_weights_are_the_unique_solution_of_the_moment_conditions(lat):
    """sum a = 1, sum a c_x^2 = c_s^2, sum a c_x^4 = 3 c_s^4, sum a c_x^2 c_y^2 = c_s^4
    for speed classes 0, 1, sqrt 2: three unknowns, determined uniquely."""
    c, a, _, _ = lat
    sp = (c ** 2).sum(1)
    classes = [sp == 0, sp == 1, sp == 2]
    M = np.array([[cl.sum() for cl in classes],
                  [(c[cl, 0] ** 2).sum() for cl in classes],
                  [(c[cl, 0] ** 2 * c[cl, 1] ** 2).sum() for cl in classes]])
    sol = np.linalg.solve(M, [1.0, CS2, CS2 ** 2])
    for k, cl in enumerate(classes):
        assert np.allclose(a[cl], sol[k], atol=1e-16)
    assert (a * c[:, 0] ** 4).sum() == pytest.approx(3 * CS2 ** 2, abs=1e-16)
    assert np.abs(np.einsum("i,ia,ib,ig->abg", a, c, c, c)).max() < 1e-16


def test_table1_norms_and_orthogonality(lat):
    _, a, e, w = lat
    ref = read_table("d2q9_table1_wk.txt")
    for k in range(9):
        assert w[k] == pytest.approx(ref[str(k)], rel=1e-15)
    G = (e * a) @ e.T
    assert np.allclose(G, np.diag([ref[str(k)] for k in range(9)]), rtol=1e-15, atol=1e-15)


def test_conservation_per_collision(D, lat):
    c, a, _, _ = lat
    rng = np.random.default_rng(0)
    for trial in range(40):
        p = D.make_params(1, 1, kT=1e-3, gamma_shear=rng.uniform(-1, 1), gamma_bulk=rng.uniform(-1, 1),
                          gamma_ghost=rng.uniform(-1, 1), seed=trial)
        n = a * (1 + 0.05 * rng.standard_normal(9))
        ns = D.collide_site(p, n, site=trial, step=2)
        assert ns.sum() == pytest.approx(n.sum(), abs=1e-15)
        assert np.allclose(ns @ c, n @ c, atol=1e-16)
        assert not np.allclose(ns, n)


def test_bgk_and_guo_forcing_at_equal_eigenvalues(D, lat):
    c, a, _, _ = lat
    rng = np.random.default_rng(1)
    for gam in (-0.6, 0.0, 0.4, 0.9):
        p = D.make_params(1, 1, kT=0.0, gamma=np.r_[np.ones(3), np.full(6, gam)])
        for _ in range(10):
            n = a * rng.uniform(0.5, 2.0) * (1 + 0.1 * rng.standard_normal(9))
            rho = n.sum()
            neq = neq2(rho, (n @ c) / rho, c, a)
            assert np.allclose(D.collide_site(p, n), neq + gam * (n - neq), rtol=0, atol=1e-15)
            # Guo, Zheng, Shi (2002): u = (j + F/2)/rho, source (1 + gam)/2 a_i [(c - u).F / c_s^2 + (c.u)(c.F) / c_s^4]
            F = 1e-2 * rng.standard_normal(2)
            u = (n @ c + 0.5 * F) / rho
            neqF = neq2(rho, u, c, a)
            G = a * (((c - u) @ F) / CS2 + (c @ u) * (c @ F) / CS2 ** 2)
            got = D.collide_site(p, n, force=F)
            assert np.allclose(got, neqF + gam * (n - neqF) + 0.5 * (1 + gam) * G, rtol=0, atol=1e-15)
            assert np.allclose(got @ c, n @ c + F, atol=1e-16)


def test_stress_relaxation_at_zero_temperature(D, lat):
    """Eqs. stress_updaterule1-2 with R = 0 in d = 2: traceless Pi^neq scales by
    gamma_s and the trace by gamma_b."""
    c, a, _, _ = lat
    rng = np.random.default_rng(2)
    gs, gb = 0.3, -0.45
    p = D.make_params(1, 1, kT=0.0, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=0.7)
    for _ in range(20):
        n = a * (1 + 0.1 * rng.standard_normal(9))
        ns = D.collide_site(p, n)
        rho = n.sum()
        u = (n @ c) / rho
        Peq = rho * CS2 * np.eye(2) + rho * np.outer(u, u)
        P0 = np.einsum("i,ia,ib->ab", n, c, c) - Peq
        P1 = np.einsum("i,ia,ib->ab", ns, c, c) - Peq
        assert np.allclose(P1 - np.trace(P1) / 2 * np.eye(2), gs * (P0 - np.trace(P0) / 2 * np.eye(2)), atol=1e-15)
        assert np.trace(P1) == pytest.approx(gb * np.trace(P0), abs=1e-15)


def test_random_stress_covariance_in_two_dimensions(D, lat):
    """Eq. stressfluctuations_microscopic with d = 2:
    <R_ab R_cd> / (mu rho c_s^4) = (1 - gs^2)(d_ac d_bd + d_ad d_bc) + (2/2)(gs^2 - gb^2) d_ab d_cd."""
    c, a, _, _ = lat
    nx = ny = 512
    N = nx * ny
    kT, gs, gb, rho0 = 1e-4, 0.35, -0.2, 1.0
    mu = 3 * kT
    p = D.make_params(nx, ny, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=0.1, seed=21)
    ns = D.collide_field(p, D.rest_state(nx, ny, rho0), step=4).reshape(9, N)
    R = (np.einsum("in,ia,ib->abn", ns, c, c) - (rho0 * CS2 * np.eye(2))[:, :, None]).reshape(4, N)
    C = R @ R.T / N
    d = np.eye(2)
    expect = (1 - gs ** 2) * (np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) \
        + (2 / 2) * (gs ** 2 - gb ** 2) * np.einsum("ab,cd->abcd", d, d)
    expect = expect.reshape(4, 4) * mu * rho0 * CS2 ** 2
    dg = np.diag(expect)
    se = np.sqrt((np.outer(dg, dg) + expect ** 2) / N)
    assert np.all(np.abs(C - expect) < 5 * se + 1e-30)


def test_equipartition_velocity_variance_and_structure_factor(D, lat):
    """64^2, k_B T = 1e-4: every mode variance mu rho0 w_k, <u_a^2> = k_B T / rho0
    and S(k) = mu rho0 (the linear invariant measure; O(mu) bias 3e-4)."""
    c, a, e, w = lat
    L, kT, rho0 = 64, 1e-4, 1.0
    mu = 3 * kT
    p = D.make_params(L, L, rho0=rho0, kT=kT, gamma_shear=0.2, gamma_bulk=0.1, gamma_ghost=0.0, seed=5)
    n = D.run(p, D.rest_state(L, L, rho0), 0, 200)
    t, r, u2, S, ns = 200, np.zeros(9), np.zeros(2), np.zeros((L, L)), 0
    while t < 1400:
        n = D.run(p, n, t, 6)
        t += 6
        r += D.mode_second_moments(n, rho0)
        rho = n.sum(0)
        j = np.tensordot(c.T, n, axes=(1, 0))
        u2 += ((j / rho) ** 2).reshape(2, -1).mean(1)
        F = np.fft.fft2(rho - rho.mean())
        S += np.abs(F) ** 2 / rho.size
        ns += 1
    r = r / ns / (mu * rho0 * w)
    expect = np.ones(9)
    expect[:3] -= 1.0 / L ** 2
    assert np.allclose(r, expect, atol=0.02), r
    assert np.allclose(u2 / ns * rho0 / kT, 1.0, atol=0.02)
    Sk = S / ns / (mu * rho0)
    assert abs(Sk.reshape(-1)[1:].mean() - 1.0) < 0.01


def one_step_operator_2d(c, a, q, gs, gb, gg):
    """Linearised collision about rest with weighted projectors onto conserved,
    bulk (c^2 - 2 c_s^2), traceless shear and kinetic subspaces (no Table I),
    followed by push streaming of the Fourier mode q."""
    W = np.diag(1 / a)

    def proj(cols):
        H = np.stack(cols, 1)
        return H @ np.linalg.solve(H.T @ W @ H, H.T @ W)

    c2 = (c ** 2).sum(1)
    cons = [a, a * c[:, 0], a * c[:, 1]]
    bulk = [a * (c2 - 2 * CS2)]
    shear = [a * (c[:, 0] ** 2 - c[:, 1] ** 2), a * c[:, 0] * c[:, 1]]
    Pc, Pb, Ps = proj(cons), proj(bulk), proj(shear)
    Pg = np.eye(9) - proj(cons + bulk + shear)
    return np.diag(np.exp(-1j * (c @ q))) @ (Pc + gs * Ps + gb * Pb + gg * Pg)


def test_linear_operator_matches_the_oracle(D, lat):
    """One deterministic oracle step of a small-amplitude plane wave equals the
    linear operator (to O(amplitude^2))."""
    c, a, _, _ = lat
    L, gs, gb, gg = 16, 0.3, -0.2, 0.5
    q = np.array([2 * np.pi * 3 / L, 2 * np.pi / L])
    A = one_step_operator_2d(c, a, q, gs, gb, gg)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    y, x = np.mgrid[0:L, 0:L]
    ph = np.exp(1j * (q[0] * x + q[1] * y))
    eps = 1e-7
    n = a[:, None, None] + eps * (v[:, None, None] * ph).real
    p = D.make_params(L, L, kT=0.0, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg)
    out = D.run(p, n, 0, 1)
    expect = a[:, None, None] + eps * ((A @ v)[:, None, None] * ph).real
    assert np.abs(out - expect).max() < 1e-12


def test_shear_and_sound_eigenvalues_give_the_viscosities(lat):
    """Eq. shearviscosity (nu = c_s^2 (1 + gs) / (2 (1 - gs))) and Eq. bulkviscosity
    with d = 2 (zeta / rho = c_s^2 (1 + gb) / (2 (1 - gb))): the shear eigenvalue decays
    by nu q^2, the sound pair by (nu + zeta/rho) q^2 / 2 and oscillates at c_s q, each
    to O(q^2) (checked by convergence from L = 256 to 1024)."""
    c, a, _, _ = lat
    gs, gb = 0.4, -0.3
    nu = CS2 * (1 + gs) / (2 * (1 - gs))
    zeta = CS2 * (1 + gb) / (2 * (1 - gb))
    errs = []
    for L in (256, 1024):
        qv = 2 * np.pi / L
        lam, V = np.linalg.eig(one_step_operator_2d(c, a, np.array([0.0, qv]), gs, gb, 0.0))
        jx = np.abs(c[:, 0] @ V) / np.linalg.norm(V, axis=0)
        rho = np.abs(V.sum(0)) / np.linalg.norm(V, axis=0)
        ls = lam[np.argmax(jx * (np.abs(lam) > 0.5))]
        lsound = lam[np.argmax(rho * (np.abs(lam) > 0.5))]
        e1 = -np.log(abs(ls)) / qv ** 2 / nu - 1
        e2 = -np.log(abs(lsound)) / qv ** 2 / ((nu + zeta) / 2) - 1
        e3 = abs(np.angle(lsound)) / qv / np.sqrt(CS2) - 1
        errs.append(np.abs([e1, e2, e3]))
    assert np.all(errs[1] < 1e-3)
    assert np.all(errs[1] < errs[0] / 8 + 1e-9)


def test_pure_streaming_is_periodic_shift(D, lat):
    c, _, _, _ = lat
    nx, ny = 5, 4
    n = np.random.default_rng(8).random((9, ny, nx))
    out = D.run(D.make_params(nx, ny, kT=1e-3, gamma=np.ones(9), seed=1), n, 0, 1)
    ci = c.astype(int)
    for i in range(9):
        assert np.allclose(out[i], np.roll(n[i], shift=(ci[i, 1], ci[i, 0]), axis=(0, 1)), rtol=0, atol=1e-14)


def test_stress_only_noise_leaves_ghosts_cold(D, lat):
    """Sec. IV: with noise on the stress modes only, the kinetic modes 6..8 of
    a site collided from rest carry no fluctuation at gamma_ghost = 0."""
    c, a, e, w = lat
    p = D.make_params(64, 64, kT=1e-4, gamma_shear=0.2, gamma_bulk=0.2, gamma_ghost=0.0, seed=9,
                      noise_ghosts=False)
    ns = D.collide_field(p, D.rest_state(64, 64), step=0).reshape(9, -1)
    m = e @ (ns - a[:, None])
    assert np.abs(m[6:]).max() < 1e-15          # rounding of the transforms only
    assert np.all(m[3:6].std(1) > 0.5 * np.sqrt(3e-4 * w[3:6]))


def mode_variance_recursion_2d(c, a, e, w, shape, kT, rho0, gs, gb, gg, T):
    """r_k(t), t = 1..T, of the linearised D2Q9 chain started from rest on an
    nx x ny box: per Fourier mode C(t+1) = L C(t) L^H + S Sigma S^H, L the
    projector collision and push streaming of one_step_operator_2d and Sigma =
    mu rho0 sum_s (1 - gamma_s^2) P_s diag(a) the noise covariance of one
    collision (Eq. FDT; no Table I in the prediction); the site average of
    m_k^2 is the mean over q of (e C e^T)_kk."""
    nx, ny = shape
    mu = 3 * kT
    Wi = np.diag(1 / a)

    def proj(cols):
        H = np.stack(cols, 1)
        return H @ np.linalg.solve(H.T @ Wi @ H, H.T @ Wi)

    c2 = (c ** 2).sum(1)
    cons = [a, a * c[:, 0], a * c[:, 1]]
    bulk = [a * (c2 - 2 * CS2)]
    shear = [a * (c[:, 0] ** 2 - c[:, 1] ** 2), a * c[:, 0] * c[:, 1]]
    Pb, Ps = proj(bulk), proj(shear)
    Pg = np.eye(9) - proj(cons + bulk + shear)
    Sig = mu * rho0 * ((1 - gs ** 2) * Ps + (1 - gb ** 2) * Pb + (1 - gg ** 2) * Pg) @ np.diag(a)
    kx, ky = np.meshgrid(np.fft.fftfreq(nx), np.fft.fftfreq(ny), indexing="ij")
    qs = 2 * np.pi * np.stack([kx.ravel(), ky.ravel()], 1)
    Lq = np.stack([one_step_operator_2d(c, a, q, gs, gb, gg) for q in qs])
    ph = np.exp(-1j * (qs @ c.T))
    Nq = ph[:, :, None] * Sig[None] * ph.conj()[:, None, :]
    Ct = np.zeros_like(Nq)
    pred = []
    for _ in range(T):
        Ct = Lq @ Ct @ Lq.conj().transpose(0, 2, 1) + Nq
        pred.append(np.einsum("ki,qij,kj->k", e, Ct, e).real / len(qs))
    return np.array(pred) / (mu * rho0 * w)


def test_finite_time_mode_variances_follow_the_linear_covariance_recursion(D, lat):
    """From rest, the oracle's site-averaged variance of every mode follows,
    step by step, mode_variance_recursion_2d: 64 seeds on a 16 x 12 box, 20
    steps, within 5 standard errors."""
    c, a, e, w = lat
    nx, ny, kT, rho0, gs, gb, gg, T, nseeds = 16, 12, 1e-4, 1.0, 0.2, 0.1, 0.0, 20, 64
    mu = 3 * kT
    pred = mode_variance_recursion_2d(c, a, e, w, (nx, ny), kT, rho0, gs, gb, gg, T)
    obs = np.zeros((nseeds, T, 9))
    for s in range(nseeds):
        p = D.make_params(nx, ny, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=500 + s)
        n = D.rest_state(nx, ny, rho0)
        for t in range(T):
            n = D.run(p, n, t, 1)
            obs[s, t] = D.mode_second_moments(n, rho0) / (mu * rho0 * w)
    mean = obs.mean(0)
    se = obs.std(0, ddof=1) / np.sqrt(nseeds)
    assert np.ptp(pred[:, :3], axis=0).min() > 0.1          # the transient is resolved
    assert np.all(np.abs(mean - pred) < 5 * se + 2e-3), np.abs(mean - pred) / (se + 1e-12)
