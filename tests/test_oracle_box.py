"""Box-level pins of the oracle (streaming, equipartition, viscosity, forcing,
storage rounding), each against something other than the oracle itself:

* pure streaming (all gamma = 1) is a periodic shift by c_i (Eq. LBE);
* equipartition: every mode variance mu rho0 w_k (Eq. modeprob with the
  unscaled basis), velocity variance k_B T / rho0 per component and a flat
  S(k) = mu rho0 = rho0 k_B T / c_s^2 (Sec. V, Eq. mpeos);
* from rest, the site-averaged variance of every mode follows, step by step,
  the exact covariance recursion of the linearised chain per Fourier mode
  (collision projectors, noise covariance of Eq. FDT, push streaming);
* the decay of a shear wave at k_B T = 0 equals, step by step, the power of
  the shear eigenvalue of the linearised one-step operator built from weighted
  polynomial projections (no Table II), and gives the shear viscosity of
  Eq. shearviscosity up to O(q^2);
* the body force (absent from the paper; second-order moment-space forcing)
  equals the population-space forcing of Guo, Zheng and Shi (PRE 65, 046308,
  2002) when every eigenvalue is the same, and the Kolmogorov flow reaches the
  exact linear steady state and the Navier-Stokes amplitude F0 / (rho0 nu q^2);
* the storage rounding to binary16 and bfloat16 matches numpy's float16 cast and
  a bit-level bfloat16 rounding of binary32.
"""
import numpy as np
import pytest

from tests.test_oracle_collision import CS2, subspace_projectors


@pytest.fixture(scope="module")
def lat(ora):
    c, a, e, w = ora.lattice()
    return c.astype(float), a, e, w


def test_pure_streaming_is_periodic_shift(ora, lat):
    c, a, _, _ = lat
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(8)
    n = rng.random((19, nz, ny, nx))
    p = ora.make_params(nx, ny, nz, kT=1e-3, gamma=np.ones(19), seed=1)
    out = ora.run(p, n, 0, 1)
    ci = c.astype(int)
    for i in range(19):
        expect = np.roll(n[i], shift=(ci[i, 2], ci[i, 1], ci[i, 0]), axis=(0, 1, 2))
        # the collision still runs the forward and inverse transform: equal to rounding
        assert np.allclose(out[i], expect, rtol=0, atol=1e-14)


def test_equipartition_velocity_variance_and_structure_factor(ora, lat):
    """16^3, rho0 = 1, k_B T = 1e-4, gamma_s = gamma_b = 0.2, gamma_ghost = 0,
    seed 1, from rest equilibrium; samples every 4 steps from t = 100 to 400."""
    c, a, e, w = lat
    L, kT, rho0 = 16, 1e-4, 1.0
    mu = 3 * kT
    p = ora.make_params(L, L, L, rho0=rho0, kT=kT, gamma_shear=0.2, gamma_bulk=0.2, gamma_ghost=0.0, seed=1)
    n = ora.rest_state(L, L, L, rho0)
    n = ora.run(p, n, 0, 100)
    t = 100
    r_acc = np.zeros(19)
    u2 = np.zeros(3)
    S = np.zeros((L, L, L))
    ns = 0
    while t < 400:
        n = ora.run(p, n, t, 4)
        t += 4
        r_acc += ora.mode_second_moments(n, rho0)
        rho, j, _ = ora.moments(n)
        u2 += ((j / rho) ** 2).reshape(3, -1).mean(1)
        S += ora.structure_factor(n)
        ns += 1
    r = r_acc / ns / (mu * rho0 * w)
    N = L ** 3
    # mass and momentum are globally conserved: the k = 0..3 site variances lack 1/N
    expect = np.ones(19)
    expect[:4] -= 1.0 / N
    # 75 samples x 4096 sites; statistical error ~0.3%, nonlinear bias O(mu) = 3e-4
    assert np.allclose(r, expect, atol=0.02), r
    assert np.abs(r - expect).mean() < 0.01
    v = u2 / ns * rho0 / kT
    assert np.allclose(v, 1.0, atol=0.02), v
    Sk = S / ns / (mu * rho0)
    mask = np.ones_like(Sk, dtype=bool)
    mask[0, 0, 0] = False
    assert abs(Sk[mask].mean() - 1.0) < 0.02, Sk[mask].mean()
    # flat: the shells are all at 1 within their sampling error
    q = np.fft.fftfreq(L) * L
    Q2 = q[:, None, None] ** 2 + q[None, :, None] ** 2 + q[None, None, :] ** 2
    for lo, hi in ((1, 4), (4, 16), (16, 64), (64, 200)):
        sel = mask & (Q2 >= lo) & (Q2 < hi)
        assert abs(Sk[sel].mean() - 1.0) < 0.1, (lo, hi, Sk[sel].mean())


def one_step_linear_operator(c, a, q, gs, gb, gg):
    """Linearised collision about rest, C = P_cons + gs P_shear + gb P_bulk +
    gg P_kinetic, followed by push streaming of a Fourier mode q:
    n^(q, t+1) = diag(exp(-i q.c_i)) C n^(q, t)."""
    Pc, Pb, Ps, Pg = subspace_projectors(c, a)
    C = Pc + gs * Ps + gb * Pb + gg * Pg
    return np.diag(np.exp(-1j * (c @ q))) @ C


def test_shear_wave_decay_matches_linear_operator(ora, lat):
    c, a, _, _ = lat
    L, gs, gb, gg, u0 = 64, 0.5, 0.2, 0.0, 1e-5
    qz = 2 * np.pi / L
    A = one_step_linear_operator(c, a, np.array([0.0, 0.0, qz]), gs, gb, gg)
    lam, V = np.linalg.eig(A)
    jx = np.abs(c[:, 0] @ V) / np.linalg.norm(V, axis=0)
    k = np.argmax(jx * (np.abs(lam) > 0.9))
    lam_s = lam[k]
    assert abs(lam_s.imag) < 1e-12
    lam_s = lam_s.real
    z = np.arange(L)
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = u0 * np.sin(qz * z)
    n = ora.equilibrium_field(np.ones((L, 1, 1)), u)
    p = ora.make_params(1, 1, L, kT=0.0, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg)
    tr = ora.run_trace(p, n, 0, 400)
    rho = tr.sum(axis=1)
    ux = np.einsum("tizyx,i->tzyx", tr, c[:, 0]) / rho
    amp = (2.0 / L) * (ux[:, :, 0, 0] * np.sin(qz * z)).sum(1)
    t0 = 40
    ratio = amp[t0:] / amp[t0 - 1]
    expect = lam_s ** np.arange(1, len(ratio) + 1)
    assert np.allclose(ratio, expect, rtol=0, atol=1e-9)
    # Eq. shearviscosity: nu = c_s^2 (1 + gs) / (2 (1 - gs)), decay exp(-nu q^2) per step
    nu = CS2 * (1 + gs) / (2 * (1 - gs))
    nu_eff = -np.log(lam_s) / qz ** 2
    assert nu_eff == pytest.approx(nu, rel=0.01)


def mode_variance_recursion(c, a, e, w, shape, kT, rho0, gs, gb, gg, T):
    """r_k(t) = <m_k^2>(t) / (mu rho0 w_k), t = 1..T, of the linearised chain
    started from rest on a periodic box of `shape` (nx, ny, nz).  Per Fourier
    mode q the covariance obeys C(t+1) = L C(t) L^H + S Sigma S^H with
    L = S(q) (P_cons + gs P_shear + gb P_bulk + gg P_kinetic), S(q) =
    diag(exp(-i q.c_i)) the push streaming and Sigma = mu rho0 sum_s
    (1 - gamma_s^2) P_s diag(a) the population-space covariance of the noise
    of one collision (variance mu rho0 w_k (1 - gamma_k^2) per non-conserved
    mode, Eq. FDT; projectors from polynomials, no Table II); the site average
    of m_k^2 is the mean over q of (e C e^T)_kk."""
    nx, ny, nz = shape
    mu = 3 * kT
    Pc, Pb, Ps, Pg = subspace_projectors(c, a)
    Ccol = Pc + gs * Ps + gb * Pb + gg * Pg
    Sig = mu * rho0 * ((1 - gs ** 2) * Ps + (1 - gb ** 2) * Pb + (1 - gg ** 2) * Pg) @ np.diag(a)
    assert np.allclose(Sig, Sig.T, atol=1e-18)
    kx, ky, kz = np.meshgrid(np.fft.fftfreq(nx), np.fft.fftfreq(ny), np.fft.fftfreq(nz), indexing="ij")
    q = 2 * np.pi * np.stack([kx.ravel(), ky.ravel(), kz.ravel()], 1)
    ph = np.exp(-1j * (q @ c.T))                             # [N, 19]
    Lq = ph[:, :, None] * Ccol[None]
    Nq = ph[:, :, None] * Sig[None] * ph.conj()[:, None, :]
    Ct = np.zeros_like(Nq)
    pred = []
    for _ in range(T):
        Ct = Lq @ Ct @ Lq.conj().transpose(0, 2, 1) + Nq
        pred.append(np.einsum("ki,qij,kj->k", e, Ct, e).real / len(q))
    return np.array(pred) / (mu * rho0 * w)                  # [T, 19]


def test_finite_time_mode_variances_follow_the_linear_covariance_recursion(ora, lat):
    """From rest (no fluctuations at t = 0) the oracle, averaged over 64 seeds
    on a 16 x 12 x 10 box (config 1 parameters), follows the exact covariance
    recursion of the linearised chain (mode_variance_recursion) for every mode
    through the transient, conserved modes included (they gain variance only
    through streaming)."""
    c, a, e, w = lat
    nx, ny, nz = 16, 12, 10
    kT, rho0, gs, gb, gg, T, nseeds = 1e-4, 1.0, 0.2, 0.2, 0.0, 24, 64
    mu = 3 * kT
    pred = mode_variance_recursion(c, a, e, w, (nx, ny, nz), kT, rho0, gs, gb, gg, T)
    obs = np.zeros((nseeds, T, 19))
    n0 = ora.rest_state(nx, ny, nz, rho0)
    for s in range(nseeds):
        p = ora.make_params(nx, ny, nz, rho0=rho0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg,
                            seed=1000 + s)
        tr = ora.run_trace(p, n0, 0, T)
        for t in range(T):
            obs[s, t] = ora.mode_second_moments(tr[t], rho0) / (mu * rho0 * w)
    mean = obs.mean(0)
    se = obs.std(0, ddof=1) / np.sqrt(nseeds)
    # the recursion is far from equilibrium early on: the test resolves the transient
    assert np.ptp(pred[:, :4], axis=0).min() > 0.1
    assert np.all(np.abs(mean - pred) < 5 * se + 2e-3), np.abs(mean - pred) / (se + 1e-12)


def test_viscosity_of_shear_mode_at_several_gammas(ora, lat):
    """nu_eff from the linear operator converges to Eq. shearviscosity as q -> 0."""
    c, a, _, _ = lat
    for gs in (-0.5, 0.0, 0.3, 0.8):
        nu = CS2 * (1 + gs) / (2 * (1 - gs))
        errs = []
        for L in (256, 1024):
            qz = 2 * np.pi / L
            A = one_step_linear_operator(c, a, np.array([0.0, 0.0, qz]), gs, 0.2, 0.0)
            lam, V = np.linalg.eig(A)
            jx = np.abs(c[:, 0] @ V) / np.linalg.norm(V, axis=0)
            lam_s = lam[np.argmax(jx * (np.abs(lam) > 0.5))].real
            errs.append(abs(-np.log(lam_s) / qz ** 2 / nu - 1))
        assert errs[1] < errs[0] / 10 or errs[1] < 1e-6
        assert errs[1] < 1e-3


def guo_bgk_forcing(n, F, gam, c, a):
    """Guo, Zheng, Shi (2002) population-space forcing with one relaxation
    factor gam = 1 - 1/tau: u = (j + F/2) / rho and
    n*_i = n^eq_i(u) + gam (n_i - n^eq_i(u)) + (1 + gam)/2 a_i [(c_i - u).F / c_s^2
    + (c_i.u)(c_i.F) / c_s^4]."""
    rho = n.sum()
    u = (n @ c + 0.5 * F) / rho
    cu = c @ u
    neq = rho * a * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
    G = a * (((c - u) @ F) / CS2 + cu * (c @ F) / CS2 ** 2)
    return neq + gam * (n - neq) + 0.5 * (1 + gam) * G


def test_forcing_equals_guo_bgk_for_equal_eigenvalues(ora, lat):
    c, a, _, _ = lat
    rng = np.random.default_rng(12)
    for gam in (-0.5, 0.0, 0.3, 0.9):
        p = ora.make_params(1, 1, 1, kT=0.0, gamma=np.r_[np.ones(4), np.full(15, gam)])
        for _ in range(10):
            n = a * (1 + 0.1 * rng.standard_normal(19))
            F = 1e-2 * rng.standard_normal(3)
            got = ora.collide_site(p, n, force=F)
            assert np.allclose(got, guo_bgk_forcing(n, F, gam, c, a), rtol=0, atol=1e-15)
            assert got.sum() == pytest.approx(n.sum(), abs=1e-15)
            assert np.allclose(got @ c, n @ c + F, atol=1e-15)


def test_kolmogorov_steady_state(ora, lat):
    """F_x(z) = F0 sin(q z): the oracle's steady state equals the steady state of
    the exact linear one-step map (19 L x 19 L real system), and the velocity
    amplitude (j + F/2)/rho matches F0 / (rho0 nu q^2) of the Navier-Stokes
    solution (Eq. shearviscosity) to O(q^2)."""
    c, a, _, _ = lat
    L, gs, gb, gg, F0 = 64, 0.3, 0.2, 0.0, 1e-7
    q = 2 * np.pi / L
    nu = CS2 * (1 + gs) / (2 * (1 - gs))
    p = ora.make_params(1, 1, L, kT=0.0, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, force_amp=F0)
    n = ora.rest_state(1, 1, L)
    n = ora.run(p, n, 0, 12000)     # ~36 viscous times 1 / (nu q^2)
    rho, j, _ = ora.moments(n)
    z = np.arange(L)
    F = F0 * np.sin(q * z)
    ux = (j[0, :, 0, 0] + 0.5 * F) / rho[:, 0, 0]
    # exact linear steady state of n(t+1) = S (C n(t) + f), f_i = a_i c_ix F(z) / c_s^2
    Pc, Pb, Ps, Pg = subspace_projectors(c, a)
    C = Pc + gs * Ps + gb * Pb + gg * Pg
    ci = c.astype(int)
    N = 19 * L
    S = np.zeros((N, N))
    for i in range(19):
        for zz in range(L):
            S[i * L + (zz + ci[i, 2]) % L, i * L + zz] = 1.0
    Cbig = np.kron(C, np.eye(L))
    f = np.kron(a * c[:, 0] / CS2, F)
    dn = np.linalg.lstsq(np.eye(N) - S @ Cbig, S @ f, rcond=None)[0].reshape(19, L)
    # uniform mass and momentum are fixed points of the map; the run starts at
    # rest and sum_z F = 0, so remove any uniform component a_i (drho + c_i.dj / c_s^2)
    drho = dn.sum() / L
    dj = (c.T @ dn).sum(1) / L
    dn -= (a * (drho + (c @ dj) / CS2))[:, None]
    n_lin = np.kron(a, np.ones(L)).reshape(19, L) + dn
    j_lin = c[:, 0] @ n_lin
    ux_lin = (j_lin + 0.5 * F) / n_lin.sum(0)
    assert np.allclose(ux, ux_lin, rtol=0, atol=1e-6 * np.abs(ux_lin).max())
    amp = (2.0 / L) * (ux * np.sin(q * z)).sum()
    assert amp == pytest.approx(F0 / (nu * q * q), rel=0.01)


def test_storage_rounding_formats(ora):
    rng = np.random.default_rng(6)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-9, 4, 2000),
                         [0.0, 6e-8, -3e-8, 65504.0, 65519.0, 65520.0, 1e-5, 2 ** -14, 2 ** -24]])
    with np.errstate(over="ignore"):          # 65520 rounds to infinity, as intended
        for x in xs:
            assert ora.round_f16(x) == float(np.float16(x)), x
    # bfloat16 = binary32 rounded to its top 16 bits, ties to even
    for x in xs:
        f = np.float32(x)
        if float(f) != x:
            continue                   # compare only where binary32 holds x exactly
        b = np.array([f], dtype=np.float32).view(np.uint32)[0]
        lsb = (b >> 16) & 1
        rb = np.uint32((int(b) + 0x7FFF + int(lsb)) & 0xFFFF0000)
        ref = float(np.array([rb], dtype=np.uint32).view(np.float32)[0])
        assert ora.round_bf16(x) == ref, x
