"""Physics validation of the fluctuating D3Q19 library on the GPU.

Each function runs one workload through the C ABI and returns a dict of
measured observables next to the values the paper fixes:

* ``equipartition``  every mode variance <m_k^2> = mu rho0 w_k (Sec. III,
  Eq. modeprob with the unscaled basis), velocity variance k_BT / rho0 per
  component and a flat S(q) = mu rho0 = rho0 k_BT / c_s^2 (Sec. V, Eq. mpeos);
* ``shear_wave``     decay rate of u_x = u0 sin(2 pi z / L) against the shear
  viscosity nu = c_s^2 (1 + gamma_s) / (2 (1 - gamma_s)) (Eq. shearviscosity);
* ``kolmogorov``     u_x(z, t) under F_x = F0 sin(k z) against the Navier-Stokes
  solution F0 / (rho0 nu k^2) (1 - exp(-nu k^2 t)) sin(k z);
* ``precision_table`` the above statistics for FP32, FP16- and BF16-deviation
  storage against the FP64 kernel (itself equal to the FP64 oracle to 1e-12);
* ``ensemble``        a batch of independent replicas and mixed-size boxes in
  one launch per step, replayed as CUDA graphs, with per-box equipartition;
* ``sound_wave``, ``dynamic_structure_factor``  the sound branch: speed c_s and
  attenuation (4/3 nu + zeta/rho) q^2/2 with Eq. bulkviscosity, deterministic
  and from the Brillouin peaks of S(q, omega);
* ``rounding_shear_wave`` a slow shear wave per storage format: nearest
  rounding to bfloat16 freezes it, stochastic rounding follows the decay;
* ``thermalization_variants``  all modes versus stress modes only (Sec. IV).

Run ``python -m paper_0707_1581_gb300.validate --help``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import flb
from .inputs import mixed_edges, shear_wave as shear_wave_field, uniform_draws

CS2 = 1.0 / 3.0
W_K = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9, 2 / 3, 2 / 3, 2 / 3, 2 / 9, 2 / 9, 2 / 9,
                2, 4 / 3, 4 / 9])


def shear_viscosity(gamma_shear: float) -> float:
    """Eq. shearviscosity divided by rho (h = 1)."""
    return CS2 * (1 + gamma_shear) / (2 * (1 - gamma_shear))


def _sync_time(ctx):
    ctx.flb_sync()
    return time.perf_counter()


def equipartition(L=64, store="f32", kT=1e-4, gamma_shear=0.5, gamma_bulk=0.2, gamma_ghost=0.0, seed=7, steps=20000,
                  burn=500, every=20, pattern="aa", nshells=None, shape=None):
    """From rest equilibrium: run `burn` steps, then sample every `every` steps
    until `steps`.  Returns the 19 ratios <m_k^2>/(mu rho0 w_k), <u_a^2> rho0/kT,
    S(q)/(mu rho0) per shell and the total-mass drift."""
    nx, ny, nz = shape or (L, L, L)
    cfg = flb.config(nx, ny, nz, 1.0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed, store=store, pattern=pattern)
    nshells = nshells or int(math.ceil(math.sqrt(3) * max(nx, ny, nz) / 2)) + 2
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_enable_structure_factor()
        ctx.flb_step(burn)
        ctx.flb_stats_reset()
        t0 = _sync_time(ctx)
        t = burn
        while t + every <= steps:
            ctx.flb_step(every)
            t += every
            ctx.flb_stats_sample()
        t1 = _sync_time(ctx)
        st = ctx.flb_mode_stats()
        S, cnt = ctx.flb_structure_factor(nshells)
    mu = 3 * kT
    sel = cnt > 0
    return {
        "box": [nx, ny, nz], "store": store, "kT": kT, "gamma_shear": gamma_shear, "samples": int(st["nsamples"]),
        "mode_ratio": st["mode_ratio"].tolist(),
        "u2_ratio": st["u2_ratio"].tolist(),
        "S_ratio_shells": (S[sel] / (mu * 1.0)).tolist(),
        "S_ratio_mean": float(np.sum(S[sel] * cnt[sel]) / np.sum(cnt[sel]) / mu),
        "mass_drift_rel": (st["mass_last"] - st["mass_first"]) / st["mass_first"],
        "nonfinite": int(st["nonfinite"]),
        "seconds": t1 - t0,
    }


def shear_wave(L=64, store="f32", kT=0.0, gamma_shear=0.5, gamma_bulk=0.2, gamma_ghost=0.0, seed=7, u0=1e-3,
               steps=400, every=10, t_fit=(50, 400), cross=8, replicas=1):
    """Decay of u_x = u0 sin(2 pi z / L) on an (cross x cross x L) periodic box:
    the amplitude A(t) = (2/L) sum_z <u_x>(z) sin(2 pi z / L), averaged over
    `replicas` boxes with independent noise (Philox replica ids, one batched
    context), is fitted by A0 exp(-nu_eff q^2 t) over t_fit; returns nu_eff
    against Eq. shearviscosity."""
    q = 2 * math.pi / L
    cfgs = [flb.config(cross, cross, L, 1.0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed, replica=r, store=store)
            for r in range(replicas)]
    ts, amps = [], []
    zs = np.arange(L)
    with flb.flb_create_batch(cfgs) as ctx:
        for b in range(replicas):
            ctx.flb_init_velocity(shear_wave_field((L, cross, cross), u0), box=b)
        t = 0
        while t <= steps:
            a = 0.0
            for b in range(replicas):
                rho, j = ctx.flb_z_profile(box=b)
                a += 2.0 / L * np.sum(j[0] / rho * np.sin(q * zs))
            amps.append(a / replicas)
            ts.append(t)
            ctx.flb_step(every)
            t += every
    ts, amps = np.array(ts, float), np.array(amps)
    m = (ts >= t_fit[0]) & (ts <= t_fit[1]) & (amps > 0)
    slope = np.polyfit(ts[m], np.log(amps[m]), 1)[0]
    nu_eff = -slope / q ** 2
    nu = shear_viscosity(gamma_shear)
    return {"L": L, "store": store, "kT": kT, "gamma_shear": gamma_shear, "replicas": replicas, "nu_eff": nu_eff,
            "nu_paper": nu, "rel_err": nu_eff / nu - 1.0, "amplitude": amps.tolist()[:: max(1, len(amps) // 20)]}


def bulk_viscosity(gamma_bulk: float) -> float:
    """Eq. bulkviscosity divided by rho (h = 1, d = 3)."""
    return CS2 / 3 * (1 + gamma_bulk) / (1 - gamma_bulk)


def sound_wave(L=64, store="f32", gamma_shear=0.2, gamma_bulk=0.2, gamma_ghost=0.0, drho=1e-4, steps=600,
               cross=4, every=2):
    """A standing density wave rho = rho0 + drho cos(q z) at rest (k_BT = 0).
    Linearised hydrodynamics (Sec. V, Eqs. ce11-ce12) gives
    drho(t) ~ cos(omega t) exp(-Gamma t) with omega = c_s q and
    Gamma = (4/3 nu + zeta/rho) q^2 / 2; returns the fitted c_s and Gamma."""
    q = 2 * math.pi / L
    cfg = flb.config(cross, cross, L, 1.0, 0.0, gamma_shear, gamma_bulk, gamma_ghost, 0, store=store)
    zs = np.arange(L)
    # at rest with a density modulation: n_i = rho(z) a_i, weights of Sec. II
    a = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rho_z = 1.0 + drho * np.cos(q * zs)
    n = a[:, None, None, None] * rho_z[None, :, None, None] * np.ones((19, L, cross, cross))
    ts, amps = [], []
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_set_populations(n)
        t = 0
        while t <= steps:
            rho, _ = ctx.flb_z_profile()
            amps.append(2.0 / L * np.sum((rho - 1.0) * np.cos(q * zs)))
            ts.append(t)
            ctx.flb_step(every)
            t += every
    ts, amps = np.array(ts, float), np.array(amps)
    # fit A exp(-G t) cos(w t + phi) by nonlinear least squares from the linear-theory guess
    from scipy.optimize import least_squares
    G0 = (4 / 3 * shear_viscosity(gamma_shear) + bulk_viscosity(gamma_bulk)) * q * q / 2
    w0 = math.sqrt(CS2) * q

    def resid(p):
        A, G, w, phi = p
        return A * np.exp(-G * ts) * np.cos(w * ts + phi) - amps

    fit = least_squares(resid, [drho, G0, w0, 0.0], x_scale=[drho, G0, w0, 1.0])
    _, G, w, _ = fit.x
    G_theory = (4 / 3 * shear_viscosity(gamma_shear) + bulk_viscosity(gamma_bulk)) * q * q / 2
    return {"L": L, "store": store, "cs_fit": w / q, "cs_paper": math.sqrt(CS2), "Gamma_fit": G,
            "Gamma_paper": G_theory, "cs_rel_err": w / q / math.sqrt(CS2) - 1, "Gamma_rel_err": G / G_theory - 1}


def density_acf(series: np.ndarray, max_lag: int) -> np.ndarray:
    """Re <x(t + tau) x*(t)> for tau = 0..max_lag, averaged over every time
    origin of one complex series (zero-padded FFT, unbiased 1/(T - tau))."""
    T = len(series)
    n = 1 << int(math.ceil(math.log2(2 * T)))
    F = np.fft.fft(series, n)
    c = np.fft.ifft(F * np.conj(F))[: max_lag + 1]
    return c.real / (T - np.arange(max_lag + 1))


def fit_damped_sound(lags: np.ndarray, C: np.ndarray, omega0: float, Gamma0: float):
    """Least-squares fit of C(t) = S exp(-Gamma t) (cos(Omega t) + b sin(Omega t)),
    the density autocorrelation of linearised fluctuating hydrodynamics
    (Eqs. ce11-ce12 at one wave vector: a damped sound mode; b = Gamma / Omega
    in the continuum).  Returns (S, Omega, Gamma, b)."""
    from scipy.optimize import least_squares

    def model(p):
        S, W, G, b = p
        return S * np.exp(-G * lags) * (np.cos(W * lags) + b * np.sin(W * lags))

    p0 = [C[0], omega0, Gamma0, Gamma0 / omega0]
    fit = least_squares(lambda p: (model(p) - C) / C[0], p0, x_scale=[abs(C[0]), omega0, Gamma0, 0.1])
    S, W, G, b = fit.x
    return float(S), float(abs(W)), float(G), float(b)


def brillouin_spectrum(omega: np.ndarray, S: float, Omega: float, Gamma: float) -> np.ndarray:
    """Fourier transform of S exp(-Gamma|t|)(cos(Omega t) + (Gamma/Omega) sin(Omega|t|)):
    S(q, w) = 4 S Gamma w_s^2 / ((w^2 - w_s^2)^2 + 4 Gamma^2 w^2), w_s^2 = Omega^2 + Gamma^2,
    the Brillouin doublet of an isothermal fluid (no Rayleigh line)."""
    ws2 = Omega * Omega + Gamma * Gamma
    return 4 * S * Gamma * ws2 / ((omega ** 2 - ws2) ** 2 + 4 * Gamma ** 2 * omega ** 2)


def dynamic_structure_factor(L=64, cross=8, kT=1e-4, gamma_shear=0.2, gamma_bulk=0.2, gamma_ghost=0.0, seed=21,
                             samples=1 << 16, every=4, burn=1000, nq=3, store="f32", decay_lengths=4.0):
    """Density fluctuations rho^(q, t) = sum_r drho(r) e^{-i q z} for q = 2 pi n / L
    (n = 1..nq along z, q_x = q_y = 0; the plane averages give them exactly),
    sampled every `every` steps after `burn`.  Linearised fluctuating
    hydrodynamics (Sec. V, Eqs. ce11-ce12) makes each one a damped sound mode:
    oscillation Omega with c_s^2 q^2 = Omega^2 + Gamma^2, Gamma = (4/3 nu +
    zeta/rho) q^2 / 2 (Eqs. shearviscosity, bulkviscosity), and the static
    S(q) = mu rho0 (Eq. mpeos).  The autocorrelation over all time origins is
    fitted up to `decay_lengths` / Gamma; S(q, omega) is its Fourier transform,
    a pair of Brillouin peaks near +-c_s q of half width Gamma."""
    A = cross * cross
    cfg = flb.config(cross, cross, L, 1.0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed, store=store)
    zs = np.arange(L)
    qs = 2 * math.pi * np.arange(1, nq + 1) / L
    phase = np.exp(-1j * np.outer(qs, zs))          # [nq, L]
    series = np.zeros((nq, samples), complex)
    t0 = time.perf_counter()
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(burn)
        for s in range(samples):
            rho, _ = ctx.flb_z_profile()
            series[:, s] = phase @ (rho - 1.0)
            ctx.flb_step(every)
    seconds = time.perf_counter() - t0
    mu = 3 * kT
    nu, zeta = shear_viscosity(gamma_shear), bulk_viscosity(gamma_bulk)
    out = []
    for n, q in enumerate(qs):
        G0 = (4 / 3 * nu + zeta) * q * q / 2
        w0 = math.sqrt(CS2) * q
        max_lag = max(8, int(decay_lengths / (G0 * every)))
        C = density_acf(series[n], max_lag) * A / L          # S(q) normalisation: |rho^|^2 / N
        lags = every * np.arange(max_lag + 1, dtype=float)
        S, W, G, b = fit_damped_sound(lags, C, math.sqrt(max(w0 * w0 - G0 * G0, 0.0)), G0)
        cs_fit = math.sqrt(W * W + G * G) / q
        wpk = math.sqrt(max(W * W - G * G, 0.0))           # maximum of brillouin_spectrum
        out.append({"n": n + 1, "q": q, "samples": samples, "every": every, "max_lag_steps": int(lags[-1]),
                    "Omega_fit": W, "Gamma_fit": G, "b_fit": b, "S_fit_ratio": S / mu,
                    "S_static_ratio": float(np.mean(np.abs(series[n]) ** 2) * A / L / mu),
                    "cs_fit": cs_fit, "cs_rel_err": cs_fit / math.sqrt(CS2) - 1,
                    "Gamma_theory": G0, "Gamma_rel_err": G / G0 - 1,
                    "peak_omega": wpk, "peak_halfwidth": G})
    return {"L": L, "cross": cross, "kT": kT, "store": store, "gamma_shear": gamma_shear, "gamma_bulk": gamma_bulk,
            "seconds": seconds, "modes": out}


def thermalization_variants(L=32, kT=1e-4, gamma_shear=0.5, gamma_bulk=0.2, gamma_ghost=0.0, seed=5, steps=3000,
                            burn=300, every=10, store="f32"):
    """All non-conserved modes thermalized (the detailed-balance rule of Sec. IV)
    against stress modes only (the earlier rule the paper discusses in Sec. IV):
    mode variance ratios and S(q) per shell for both."""
    out = {}
    for name, ghosts in (("all_modes", True), ("stress_only", False)):
        nx = ny = nz = L
        cfg = flb.config(nx, ny, nz, 1.0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed, store=store,
                         noise_ghosts=ghosts)
        nshells = int(math.ceil(math.sqrt(3) * L / 2)) + 2
        with flb.flb_create_ex(cfg) as ctx:
            ctx.flb_enable_structure_factor()
            ctx.flb_step(burn)
            ctx.flb_stats_reset()
            t = burn
            while t + every <= steps:
                ctx.flb_step(every)
                t += every
                ctx.flb_stats_sample()
            st = ctx.flb_mode_stats()
            S, cnt = ctx.flb_structure_factor(nshells)
        sel = cnt > 0
        out[name] = {"mode_ratio": st["mode_ratio"].tolist(), "u2_ratio": st["u2_ratio"].tolist(),
                     "S_ratio_shells": (S[sel] / (3 * kT)).tolist()}
    return out


def kolmogorov(L=512, store="f32", kT=1e-4, gamma_shear=0.3, gamma_bulk=0.2, gamma_ghost=0.0, seed=3, F0=1e-5,
               steps=5000, pattern="aa", cross=None):
    """u_x(z, t) under F_x = F0 sin(2 pi z / L) from rest, against the
    Navier-Stokes solution F0 / (rho0 nu k^2) (1 - exp(-nu k^2 t)) sin(k z)."""
    cross = cross or L
    k = 2 * math.pi / L
    nu = shear_viscosity(gamma_shear)
    cfg = flb.config(cross, cross, L, 1.0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed, store=store,
                     pattern=pattern, force_amp=F0)
    with flb.flb_create_ex(cfg) as ctx:
        t0 = _sync_time(ctx)
        ctx.flb_step(steps)
        t1 = _sync_time(ctx)
        rho, j = ctx.flb_z_profile()
    zs = np.arange(L)
    ux = j[0] / rho
    amp = 2.0 / L * np.sum(ux * np.sin(k * zs))
    expect = F0 / (1.0 * nu * k * k) * (1 - math.exp(-nu * k * k * steps))
    return {"L": L, "cross": cross, "store": store, "steps": steps, "amplitude": amp, "navier_stokes": expect,
            "rel_err": amp / expect - 1.0, "mach": abs(amp) / math.sqrt(CS2), "seconds": t1 - t0,
            "mlups": cross * cross * L * steps / (t1 - t0) / 1e6}


def precision_table(L=256, kTs=(1e-5, 1e-4, 1e-3), stores=("f32", "f16dev", "bf16dev", "bf16sr"), steps=1000, burn=200,
                    every=10, gamma_shear=0.0, seed=11):
    """Statistics of each storage format against the FP64 kernel on the same
    workload (same seed: the same noise), per k_BT."""
    rows = []
    for kT in kTs:
        ref = equipartition(L, "f64", kT, gamma_shear, 0.2, 0.0, seed, steps, burn, every)
        for store in stores:
            r = equipartition(L, store, kT, gamma_shear, 0.2, 0.0, seed, steps, burn, every)
            rows.append({
                "store": store, "kT": kT,
                "mode_ratio_max_abs_err_vs_f64": float(np.max(np.abs(np.array(r["mode_ratio"]) - ref["mode_ratio"]))),
                "mode_ratio_max_abs_dev_from_1": float(np.max(np.abs(np.array(r["mode_ratio"][4:]) - 1))),
                "u2_ratio_err_vs_f64": float(np.max(np.abs(np.array(r["u2_ratio"]) - ref["u2_ratio"]))),
                "S_mean_err_vs_f64": r["S_ratio_mean"] - ref["S_ratio_mean"],
                "mass_drift_rel": r["mass_drift_rel"], "mass_drift_rel_f64": ref["mass_drift_rel"],
                "f64_mode_ratio_max_abs_dev_from_1": float(np.max(np.abs(np.array(ref["mode_ratio"][4:]) - 1))),
            })
    return rows


def rounding_shear_wave(L=256, u0=1e-3, gamma_shear=0.5, steps=2000, cross=4,
                        stores=("f64", "f32", "f16dev", "bf16dev", "bf16sr"), seed=5):
    """A slow shear wave u_x = u0 sin(2 pi z / L) at k_BT = 0: each step changes
    a 16-bit deviation by a small fraction of its ulp.  Returns, per storage
    format, the amplitude after `steps` relative to the start and to the
    viscous decay exp(-nu q^2 t) of Eq. shearviscosity."""
    q = 2 * math.pi / L
    expect = math.exp(-shear_viscosity(gamma_shear) * q * q * steps)
    zs = np.arange(L)
    u = np.zeros((3, L, cross, cross))
    u[0] = u0 * np.sin(q * zs)[:, None, None]
    out = {}
    for store in stores:
        cfg = flb.config(cross, cross, L, 1.0, 0.0, gamma_shear, 0.2, 0.0, seed, store=store, pattern="aa")
        with flb.flb_create_ex(cfg) as ctx:
            ctx.flb_init_velocity(u)

            def amp():
                rho, j = ctx.flb_z_profile()
                return (2.0 / L) * float(np.sum(j[0] / rho * np.sin(q * zs)))

            a0 = amp()
            ctx.flb_step(steps)
            ratio = amp() / a0
        out[store] = {"amplitude_ratio": ratio, "viscous_decay": expect, "rel_err": ratio / expect - 1}
    return out


def ensemble(n_replicas=64, L=64, n_mixed=16, kT=1e-4, steps=2000, burn=200, every=20, seed=4, store="f32",
             graph_steps=20, autotune=True, unbatched=False):
    """n_replicas boxes of L^3 plus n_mixed cubes of edges 32..128, each with its
    own gamma_shear ~ U[0, 0.8] and Philox replica id, advanced together.  With
    `unbatched`, also the same boxes as one context each (one kernel per box
    and step, each context replaying its own CUDA graph) for comparison."""
    edges = [L] * n_replicas + mixed_edges(n_mixed)
    gammas = uniform_draws(len(edges), seed, 0.0, 0.8)
    cfgs = [flb.config(e, e, e, 1.0, kT, float(g), 0.2, 0.0, seed, replica=r, store=store, pattern="aa",
                       graph_steps=graph_steps) for r, (e, g) in enumerate(zip(edges, gammas))]
    sites = sum(e ** 3 for e in edges)
    with flb.flb_create_batch(cfgs) as ctx:
        if autotune:
            ctx.flb_autotune(2, pattern=True)
        ctx.flb_step(burn)
        ctx.flb_stats_reset()
        t0 = _sync_time(ctx)
        t = burn
        while t + every <= steps:
            ctx.flb_step(every)
            t += every
            ctx.flb_stats_sample()
        t1 = _sync_time(ctx)
        # timing of the plain stepping, without statistics
        ctx.flb_sync()
        t2 = _sync_time(ctx)
        ctx.flb_step(200)
        t3 = _sync_time(ctx)
        ratios = np.array([ctx.flb_mode_stats(box=b)["mode_ratio"] for b in range(len(cfgs))])
        u2 = np.array([ctx.flb_mode_stats(box=b)["u2_ratio"] for b in range(len(cfgs))])
        launch = ctx.flb_get_launch()
        pattern = ctx.flb_get_pattern()
    extra = {}
    if unbatched:
        import torch
        stream = torch.cuda.Stream()
        ctxs = [flb.flb_create_ex(flb.config(e, e, e, 1.0, kT, float(g), 0.2, 0.0, seed, replica=r, store=store,
                                             pattern="aa", graph_steps=graph_steps, stream=stream))
                for r, (e, g) in enumerate(zip(edges, gammas))]
        try:
            for c in ctxs:
                c.flb_step(2 * graph_steps)
            torch.cuda.synchronize()
            t4 = time.perf_counter()
            for _ in range(200 // graph_steps):
                for c in ctxs:
                    c.flb_step(graph_steps)
            torch.cuda.synchronize()
            t5 = time.perf_counter()
        finally:
            for c in ctxs:
                c.close()
        extra["mlups_unbatched"] = sites * (200 // graph_steps) * graph_steps / (t5 - t4) / 1e6
    return {"boxes": len(cfgs), "sites": sites, "launch": launch, "pattern": pattern, **extra,
            "mlups_stepping": sites * 200 / (t3 - t2) / 1e6,
            "mlups_with_stats": sites * (t - burn) / (t1 - t0) / 1e6,
            "mode_ratio_max_abs_dev_from_1": float(np.max(np.abs(ratios[:, 4:] - 1))),
            "mode_ratio_mean_per_mode": ratios.mean(0).tolist(),
            "u2_ratio_max_abs_dev_from_1": float(np.max(np.abs(u2 - 1)))}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("what", choices=["equipartition", "shear", "sound", "skw", "kolmogorov", "precision", "ensemble",
                                     "variants", "rounding", "all"])
    ap.add_argument("--quick", action="store_true", help="smaller boxes and fewer steps")
    ap.add_argument("--out", default=None, help="write the JSON report here")
    args = ap.parse_args()
    q = args.quick
    report = {}
    if args.what in ("equipartition", "all"):
        report["equipartition_64"] = equipartition(32 if q else 64, steps=2000 if q else 20000)
    if args.what in ("shear", "all"):
        report["shear_wave_kT0"] = shear_wave(64, kT=0.0)
        report["shear_wave_kT1e-4"] = shear_wave(64, kT=1e-4, cross=64 if not q else 16, t_fit=(20, 300),
                                                 replicas=256 if not q else 4)
    if args.what in ("sound", "all"):
        report["sound_wave"] = sound_wave(64)
    if args.what in ("skw", "all"):
        report["dynamic_structure_factor"] = dynamic_structure_factor(samples=1 << 14 if q else 1 << 18)
    if args.what in ("variants", "all"):
        report["thermalization_variants"] = thermalization_variants(32 if q else 64)
    if args.what in ("kolmogorov", "all"):
        for store in ("f32", "f16dev"):
            report[f"kolmogorov_{store}"] = kolmogorov(128 if q else 512, store=store, steps=1000 if q else 5000)
    if args.what in ("precision", "all"):
        report["precision"] = precision_table(64 if q else 256, steps=400 if q else 1000)
    if args.what in ("rounding", "all"):
        report["rounding_shear_wave"] = rounding_shear_wave()
    if args.what in ("ensemble", "all"):
        report["ensemble"] = ensemble(n_replicas=8 if q else 64, steps=400 if q else 2000, unbatched=True)
    text = json.dumps(report, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
