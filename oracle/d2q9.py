"""Python access to the D2Q9 FP64 CPU oracle (``flb_oracle_d2q9.c``, Table I).

TEST INFRASTRUCTURE ONLY, under the same rule as ``oracle.py``: only the tests
and ``__graft_entry__.smoke()`` may use it.  Populations are n[9, ny, nx]
with velocity order rest; +x, -x, +y, -y; (1,1), (-1,-1), (1,-1), (-1,1).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import oracle as _o

Q = 9
STORE_F64, STORE_F16DEV, STORE_BF16DEV, STORE_BF16SR = _o.STORE_F64, _o.STORE_F16DEV, _o.STORE_BF16DEV, _o.STORE_BF16SR


class Params(ctypes.Structure):
    """Mirror of ``ora2_params`` in flb_oracle_d2q9.c."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("rho0", ctypes.c_double), ("kT", ctypes.c_double),
        ("gamma", ctypes.c_double * Q),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
        ("noise_ghosts", ctypes.c_int), ("noise_rho_local", ctypes.c_int),
        ("force_amp", ctypes.c_double), ("store", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = _o._load()
        P, vp, u32, i64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int64
        lib.ora2_lattice.argtypes = [vp, vp, vp, vp]
        lib.ora2_equilibrium_field.argtypes = [i64, vp, vp, vp]
        lib.ora2_collide_site.argtypes = [P(Params), vp, u32, u32, vp, vp, vp]
        lib.ora2_run.argtypes = [P(Params), vp, u32, u32]
        lib.ora2_run.restype = ctypes.c_int
        lib.ora2_quantize.argtypes = [P(Params), vp]
        lib.ora2_collide_field.argtypes = [P(Params), vp, u32, vp]
        _lib = lib
    return _lib


_ptr = _o._ptr


def lattice():
    """(c[9,2] int, a[9], e[9,9] with e[k,i], w[9]) as the oracle builds them."""
    c = np.zeros((Q, 2), dtype=np.int32)
    a, e, w = np.zeros(Q), np.zeros((Q, Q)), np.zeros(Q)
    _load().ora2_lattice(_ptr(c), _ptr(a), _ptr(e), _ptr(w))
    return c, a, e, w


def gamma_vector(gamma_shear: float, gamma_bulk: float, gamma_ghost: float) -> np.ndarray:
    """Conserved modes 0..2 -> 1, bulk mode 3 -> gamma_b, shear modes 4, 5 ->
    gamma_s, kinetic modes 6..8 -> gamma_ghost."""
    g = np.empty(Q)
    g[:3] = 1.0
    g[3] = gamma_bulk
    g[4:6] = gamma_shear
    g[6:] = gamma_ghost
    return g


def make_params(nx, ny, rho0=1.0, kT=0.0, gamma_shear=0.0, gamma_bulk=0.0, gamma_ghost=0.0, seed=0, replica=0,
                noise_ghosts=True, noise_rho_local=False, force_amp=0.0, store=STORE_F64, gamma=None) -> Params:
    p = Params()
    p.nx, p.ny = int(nx), int(ny)
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


def equilibrium_field(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """n_eq(rho(r), u(r)) (Eq. derived_equil_distrib, d = 2); u[2, ...]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    shape = rho.shape
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(2, -1))
    n = np.zeros((Q, rho.size))
    _load().ora2_equilibrium_field(rho.size, _ptr(rho.reshape(-1)), _ptr(u), _ptr(n))
    return n.reshape((Q,) + shape)


def rest_state(nx, ny, rho0=1.0) -> np.ndarray:
    return equilibrium_field(np.full((ny, nx), float(rho0)), np.zeros((2, ny, nx)))


def collide_site(params: Params, n, site=0, step=0, force=None, g=None) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros(Q)
    F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    G = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    _load().ora2_collide_site(ctypes.byref(params), _ptr(n), int(site), int(step),
                              None if F is None else _ptr(F), None if G is None else _ptr(G), _ptr(out))
    return out


def run(params: Params, n: np.ndarray, t0: int, nsteps: int) -> np.ndarray:
    """Advance n[9, ny, nx] from step t0 by nsteps (returns a new array)."""
    out = np.array(n, dtype=np.float64, order="C", copy=True)
    assert out.shape == (Q, params.ny, params.nx), out.shape
    rc = _load().ora2_run(ctypes.byref(params), _ptr(out), int(t0), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"ora2_run failed ({rc})")
    return out


def collide_field(params: Params, n: np.ndarray, step: int) -> np.ndarray:
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    _load().ora2_collide_field(ctypes.byref(params), _ptr(n), int(step), _ptr(out))
    return out


def quantize(params: Params, n: np.ndarray) -> np.ndarray:
    out = np.array(n, dtype=np.float64, order="C", copy=True)
    _load().ora2_quantize(ctypes.byref(params), _ptr(out))
    return out


def modes(n: np.ndarray) -> np.ndarray:
    """m_k = sum_i e_ki n_i over every site (Table I basis)."""
    _, _, e, _ = lattice()
    return np.tensordot(e, n, axes=(1, 0))


def mode_second_moments(n: np.ndarray, rho0: float) -> np.ndarray:
    """Site average of (sum_i e_ki (n_i - rho0 a_i))^2, k = 0..8."""
    _, a, e, _ = lattice()
    dn = n - rho0 * a.reshape((Q,) + (1,) * (n.ndim - 1))
    m = np.tensordot(e, dn, axes=(1, 0)).reshape(Q, -1)
    return (m * m).mean(axis=1)
