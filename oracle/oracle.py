"""Python access to the FP64 CPU oracle (``flb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, obviously correct reference of the
fluctuating lattice Boltzmann update of Duenweg, Schiller and Ladd
(arXiv:0707.1581) that the CUDA library is checked against.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It imports nothing from the CUDA package and the CUDA package imports
nothing from here.

The C file holds the per-site update (Table II transform, Eq. updaterule with
Eq. FDT, Eq. LBE streaming).  This module adds ctypes marshalling and the
plain observables used by the statistical pins, each written from its
definition in the paper:

* ``moments``            rho, j, Pi        (Sec. I, Eqs. defrho, defj, defstress)
* ``mode_second_moments`` <m_k^2> of n - rho0 a_i over sites (Sec. III, Eq. modeprob)
* ``structure_factor``   S(k) = <|sum_r drho(r) e^{-ik.r}|^2> / N via an FFT
                         (isothermal ideal gas, Sec. V, Eq. mpeos)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flb_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "flb_oracle_d2q9.c")]
_LIB = os.path.join(_HERE, "_build", "libflb_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile the oracle (D3Q19 and D2Q9 files) with gcc (-O2, OpenMP over z-planes; results do not
    depend on the thread count because every site is updated independently)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Mirror of ``ora_params`` in flb_oracle.c."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("rho0", ctypes.c_double), ("kT", ctypes.c_double),
        ("gamma", ctypes.c_double * Q),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
        ("noise_ghosts", ctypes.c_int), ("noise_rho_local", ctypes.c_int),
        ("force_amp", ctypes.c_double), ("store", ctypes.c_int),
    ]


STORE_F64, STORE_F16DEV, STORE_BF16DEV, STORE_BF16SR = 0, 2, 3, 4


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, u32, u64, i64 = ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            vp = ctypes.c_void_p
            lib.ora_lattice.argtypes = [vp, vp, vp, vp]
            lib.ora_philox4x32_10.argtypes = [vp, vp, vp]
            lib.ora_philox_many.argtypes = [vp, vp, i64, vp]
            lib.ora_uniform16.argtypes = [u32]
            lib.ora_uniform16.restype = d
            lib.ora_gaussians.argtypes = [u64, u32, u32, u32, vp]
            lib.ora_gaussians_many.argtypes = [u64, u32, u32, i64, vp]
            lib.ora_equilibrium_field.argtypes = [i64, vp, vp, vp]
            lib.ora_collide_site.argtypes = [P(Params), vp, u32, u32, vp, vp, vp]
            lib.ora_run.argtypes = [P(Params), vp, u32, u32]
            lib.ora_run.restype = ctypes.c_int
            lib.ora_quantize.argtypes = [P(Params), vp]
            lib.ora_collide_field.argtypes = [P(Params), vp, u32, vp]
            lib.ora_run_trace.argtypes = [P(Params), vp, u32, u32, vp]
            lib.ora_run_trace.restype = ctypes.c_int
            lib.ora_round_f16.argtypes = [d]
            lib.ora_round_f16.restype = d
            lib.ora_round_bf16.argtypes = [d]
            lib.ora_round_bf16.restype = d
            lib.ora_sr_bf16.argtypes = [d, u32]
            lib.ora_sr_bf16.restype = d
            lib.ora_sr_bits.argtypes = [u64, u32, u32, u32, vp]
            lib.ora_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lattice():
    """(c[19,3] int, a[19], e[19,19] with e[k,i], w[19]) as the oracle builds them."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    a = np.zeros(Q)
    e = np.zeros((Q, Q))
    w = np.zeros(Q)
    lib.ora_lattice(_ptr(c), _ptr(a), _ptr(e), _ptr(w))
    return c, a, e, w


def gamma_vector(gamma_shear: float, gamma_bulk: float, gamma_ghost: float) -> np.ndarray:
    """Eigenvalue assignment of Sec. IV: conserved modes 1, bulk mode 4 gamma_b,
    the five shear modes 5..9 gamma_s, the nine kinetic modes 10..18 gamma_ghost."""
    g = np.empty(Q)
    g[:4] = 1.0
    g[4] = gamma_bulk
    g[5:10] = gamma_shear
    g[10:] = gamma_ghost
    return g


def make_params(nx, ny, nz, rho0=1.0, kT=0.0, gamma_shear=0.0, gamma_bulk=0.0, gamma_ghost=0.0,
                seed=0, replica=0, noise_ghosts=True, noise_rho_local=False, force_amp=0.0,
                store=STORE_F64, gamma=None) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.rho0, p.kT = float(rho0), float(kT)
    gv = gamma_vector(gamma_shear, gamma_bulk, gamma_ghost) if gamma is None else np.asarray(gamma, float)
    for k in range(Q):
        p.gamma[k] = float(gv[k])
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.replica = int(replica)
    p.noise_ghosts = 1 if noise_ghosts else 0
    p.noise_rho_local = 1 if noise_rho_local else 0
    p.force_amp = float(force_amp)
    p.store = int(store)
    return p


def philox(ctr, key) -> np.ndarray:
    """Philox-4x32-10 of an array of counters [n,4] and keys [n,2] (uint32)."""
    lib = _load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(ctr)
    lib.ora_philox_many(_ptr(ctr), _ptr(key), ctr.shape[0], _ptr(out))
    return out


def uniform16(h: int) -> float:
    """(h + 1/2) 2^-16 for a 16-bit value h."""
    return _load().ora_uniform16(int(h) & 0xFFFF)


def gaussians(seed, site, step, replica=0) -> np.ndarray:
    g = np.zeros(16)
    _load().ora_gaussians(int(seed), int(site), int(step), int(replica), _ptr(g))
    return g


def gaussians_many(seed, step, replica, nsites) -> np.ndarray:
    g = np.zeros((int(nsites), 16))
    _load().ora_gaussians_many(int(seed), int(step), int(replica), int(nsites), _ptr(g))
    return g


def equilibrium_field(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """n_eq(rho(r), u(r)) of Eq. derived_equil_distrib; rho[...] and u[3,...]
    over the same site shape; returns [19, *shape]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    shape = rho.shape
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3, -1))
    n = np.zeros((Q, rho.size))
    _load().ora_equilibrium_field(rho.size, _ptr(rho.reshape(-1)), _ptr(u), _ptr(n))
    return n.reshape((Q,) + shape)


def rest_state(nx, ny, nz, rho0=1.0) -> np.ndarray:
    return equilibrium_field(np.full((nz, ny, nx), float(rho0)), np.zeros((3, nz, ny, nx)))


def collide_site(params: Params, n, site=0, step=0, force=None, g=None) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros(Q)
    F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    G = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    _load().ora_collide_site(ctypes.byref(params), _ptr(n), int(site), int(step),
                             None if F is None else _ptr(F), None if G is None else _ptr(G), _ptr(out))
    return out


def run(params: Params, n: np.ndarray, t0: int, nsteps: int) -> np.ndarray:
    """Advance pre-collision populations n[19,nz,ny,nx] from step t0 by nsteps;
    returns a new array (the input is not modified)."""
    out = np.array(n, dtype=np.float64, order="C", copy=True)
    assert out.shape == (Q, params.nz, params.ny, params.nx), out.shape
    rc = _load().ora_run(ctypes.byref(params), _ptr(out), int(t0), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"ora_run failed ({rc})")
    return out


def collide_field(params: Params, n: np.ndarray, step: int) -> np.ndarray:
    """Collision only (no streaming) at every site of n[19,nz,ny,nx]."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    _load().ora_collide_field(ctypes.byref(params), _ptr(n), int(step), _ptr(out))
    return out


def run_trace(params: Params, n: np.ndarray, t0: int, nsteps: int) -> np.ndarray:
    """States after each of nsteps steps: [nsteps, 19, nz, ny, nx]."""
    cur = np.array(n, dtype=np.float64, order="C", copy=True)
    trace = np.zeros((int(nsteps),) + cur.shape)
    rc = _load().ora_run_trace(ctypes.byref(params), _ptr(cur), int(t0), int(nsteps), _ptr(trace))
    if rc != 0:
        raise RuntimeError(f"ora_run_trace failed ({rc})")
    return trace


def quantize(params: Params, n: np.ndarray) -> np.ndarray:
    out = np.array(n, dtype=np.float64, order="C", copy=True)
    _load().ora_quantize(ctypes.byref(params), _ptr(out))
    return out


def round_f16(x: float) -> float:
    return _load().ora_round_f16(float(x))


def round_bf16(x: float) -> float:
    return _load().ora_round_bf16(float(x))


def sr_bf16(x: float, r: int) -> float:
    """Stochastic rounding of x to bfloat16 with the 16 random bits r."""
    return _load().ora_sr_bf16(float(x), int(r) & 0xFFFF)


def sr_bits(seed, site, step, replica=0) -> np.ndarray:
    """The 24 16-bit rounding values of (site, step, replica) (Philox blocks 2..4)."""
    r = np.zeros(24, dtype=np.uint32)
    _load().ora_sr_bits(int(seed), int(site), int(step), int(replica), _ptr(r))
    return r


def threads() -> int:
    return int(_load().ora_threads())


# --------------------------------------------------------------------------
# Observables, each from its definition in the paper.
# --------------------------------------------------------------------------

def moments(n: np.ndarray):
    """rho = sum_i n_i, j = sum_i n_i c_i (Eqs. defrho, defj) and the full second
    moment Pi_ab = sum_i n_i c_ia c_ib (Eq. equilibriumstress), as
    (rho[...], j[3,...], Pi[6,...]) with Pi components xx, yy, zz, xy, yz, zx."""
    c, _, _, _ = lattice()
    c = c.astype(np.float64)
    rho = n.sum(axis=0)
    j = np.tensordot(c.T, n, axes=(1, 0))
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]
    Pi = np.stack([np.tensordot(c[:, a] * c[:, b], n, axes=(0, 0)) for a, b in pairs])
    return rho, j, Pi


def modes(n: np.ndarray) -> np.ndarray:
    """m_k = sum_i e_ki n_i over every site (Table II basis)."""
    _, _, e, _ = lattice()
    return np.tensordot(e, n, axes=(1, 0))


def mode_second_moments(n: np.ndarray, rho0: float) -> np.ndarray:
    """Site average of (sum_i e_ki (n_i - rho0 a_i))^2 for k = 0..18."""
    _, a, e, _ = lattice()
    dn = n - rho0 * a.reshape((Q,) + (1,) * (n.ndim - 1))
    m = np.tensordot(e, dn, axes=(1, 0)).reshape(Q, -1)
    return (m * m).mean(axis=1)


def structure_factor(n: np.ndarray) -> np.ndarray:
    """|FFT(rho - <rho>)|^2 / N over all wave vectors of the box; [nz,ny,nx]."""
    rho = n.sum(axis=0)
    drho = rho - rho.mean()
    F = np.fft.fftn(drho)
    return (F.real ** 2 + F.imag ** 2) / drho.size
