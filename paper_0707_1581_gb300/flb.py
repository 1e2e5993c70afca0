"""Thin ctypes binding of the C ABI in include/flb.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA kernels of libflb.so.
Host arrays are numpy arrays; PyTorch is used only to hand the library a CUDA
stream (``flb_config.stream``) when the caller wants one.  If the library has
not been built, ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FLB_LIBRARY=check selects the bounds-checked build (libflb_check.so), for debugging
LIB_PATH = (os.path.join(HERE, "_build_check", "libflb_check.so") if os.environ.get("FLB_LIBRARY") == "check"
            else os.path.join(HERE, "_build", "libflb.so"))
Q = 19

FLB_OK = 0
FLB_EINVAL, FLB_ENOMEM, FLB_ECUDA, FLB_ETIMEOUT, FLB_ENONFINITE, FLB_ERANGE, FLB_EIO = -1, -2, -3, -4, -5, -6, -7
STORE_F64, STORE_F32, STORE_F16DEV, STORE_BF16DEV, STORE_BF16SR = 0, 1, 2, 3, 4
PATTERN_AB, PATTERN_AA = 0, 1
LATTICE_D3Q19, LATTICE_D2Q9 = 0, 1
TUNE_PATTERN = 1
LATTICE_NAMES = {"d3q19": LATTICE_D3Q19, "d2q9": LATTICE_D2Q9}
STORE_NAMES = {"f64": STORE_F64, "f32": STORE_F32, "f16dev": STORE_F16DEV, "bf16dev": STORE_BF16DEV,
               "bf16sr": STORE_BF16SR}
STORE_BYTES = {STORE_F64: 8, STORE_F32: 4, STORE_F16DEV: 2, STORE_BF16DEV: 2, STORE_BF16SR: 2}

# Every symbol declared in include/flb.h.
EXPORTS = [
    "flb_config_init", "flb_create", "flb_create_ex", "flb_create_batch", "flb_destroy", "flb_num_boxes",
    "flb_step", "flb_sync", "flb_get_step", "flb_box_get_populations", "flb_get_populations", "flb_box_get_sites",
    "flb_box_set_populations", "flb_set_populations", "flb_box_init_velocity", "flb_init_velocity",
    "flb_box_moments", "flb_moments", "flb_box_z_profile", "flb_stats_reset", "flb_stats_sample", "flb_box_mode_stats",
    "flb_mode_stats", "flb_box_enable_structure_factor", "flb_box_structure_factor", "flb_box_state_bytes",
    "flb_box_state_download", "flb_box_state_upload", "flb_save", "flb_load", "flb_get_launch", "flb_autotune",
    "flb_last_error", "flb_create_error", "flb_version", "flb_mode_sums_noalloc", "flb_gammas_from_viscosities",
    "flb_lattice_kT", "flb_lattice_params", "flb_box_step_host", "flb_autotune_ex", "flb_get_pattern",
    "flb_set_pattern", "flb_box_check_finite", "flb_philox4x32_10", "flb_normals", "flb_set_launch",
    "flb_host_alloc", "flb_host_free", "flb_set_device_allocator", "flb_enable_structure_factor",
    "flb_structure_factor", "flb_bounds_violations", "flb_bounds_selftest",
]


class flb_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("rho0", ctypes.c_double), ("kT", ctypes.c_double),
        ("gamma_shear", ctypes.c_double), ("gamma_bulk", ctypes.c_double), ("gamma_ghost", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32),
        ("store", ctypes.c_int), ("pattern", ctypes.c_int),
        ("noise_ghosts", ctypes.c_int), ("noise_rho_local", ctypes.c_int),
        ("force_amp", ctypes.c_double),
        ("sites_per_thread", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
        ("graph_steps", ctypes.c_int), ("lattice", ctypes.c_int), ("stats_every", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class flb_mode_stats_t(ctypes.Structure):
    _fields_ = [
        ("nsamples", ctypes.c_uint64), ("nsites", ctypes.c_uint64),
        ("mode_m2", ctypes.c_double * Q), ("mode_ratio", ctypes.c_double * Q),
        ("u2", ctypes.c_double * 3), ("u2_ratio", ctypes.c_double * 3),
        ("mass_first", ctypes.c_double), ("mass_last", ctypes.c_double),
        ("momentum_first", ctypes.c_double * 3), ("momentum_last", ctypes.c_double * 3),
        ("nonfinite", ctypes.c_uint64),
    ]


class FlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"flb error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded libflb.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               "g.build()'` (needs nvcc); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, vp = ctypes.POINTER, ctypes.c_void_p
        i, d, i64, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "flb_config_init": (None, [P(flb_config)]),
            "flb_create": (i, [i, i, i, d, d, d, d, d, u64, P(vp)]),
            "flb_create_ex": (i, [P(flb_config), P(vp)]),
            "flb_create_batch": (i, [P(flb_config), i, P(vp)]),
            "flb_destroy": (None, [vp]),
            "flb_num_boxes": (i, [vp]),
            "flb_step": (i, [vp, i64]),
            "flb_sync": (i, [vp]),
            "flb_get_step": (i, [vp, P(u64)]),
            "flb_box_get_populations": (i, [vp, i, vp]),
            "flb_get_populations": (i, [vp, vp]),
            "flb_box_get_sites": (i, [vp, i, vp, i64, vp]),
            "flb_box_set_populations": (i, [vp, i, vp]),
            "flb_set_populations": (i, [vp, vp]),
            "flb_box_init_velocity": (i, [vp, i, vp]),
            "flb_init_velocity": (i, [vp, vp]),
            "flb_box_moments": (i, [vp, i, vp, vp, vp]),
            "flb_moments": (i, [vp, vp, vp, vp]),
            "flb_box_z_profile": (i, [vp, i, vp, vp]),
            "flb_stats_reset": (i, [vp]),
            "flb_stats_sample": (i, [vp]),
            "flb_box_mode_stats": (i, [vp, i, P(flb_mode_stats_t)]),
            "flb_mode_stats": (i, [vp, P(flb_mode_stats_t)]),
            "flb_box_enable_structure_factor": (i, [vp, i]),
            "flb_box_structure_factor": (i, [vp, i, vp, vp, i]),
            "flb_enable_structure_factor": (i, [vp]),
            "flb_structure_factor": (i, [vp, vp, i]),
            "flb_box_state_bytes": (i, [vp, i, P(ctypes.c_size_t)]),
            "flb_box_state_download": (i, [vp, i, vp]),
            "flb_box_state_upload": (i, [vp, i, vp]),
            "flb_box_step_host": (i, [vp, i, vp, i64]),
            "flb_host_alloc": (i, [ctypes.c_size_t, P(vp)]),
            "flb_host_free": (i, [vp]),
            "flb_set_device_allocator": (i, [vp, vp, vp]),
            "flb_bounds_violations": (i, [vp, P(u64)]),
            "flb_bounds_selftest": (i, [vp]),
            "flb_save": (i, [vp, ctypes.c_char_p]),
            "flb_load": (i, [vp, ctypes.c_char_p]),
            "flb_get_launch": (i, [vp, P(i), P(i), P(i)]),
            "flb_set_launch": (i, [vp, i, i, i]),
            "flb_autotune": (i, [vp, i]),
            "flb_autotune_ex": (i, [vp, i, i]),
            "flb_get_pattern": (i, [vp, P(i)]),
            "flb_set_pattern": (i, [vp, i]),
            "flb_box_check_finite": (i, [vp, i, P(u64)]),
            "flb_philox4x32_10": (i, [vp, vp, i64, vp]),
            "flb_normals": (i, [u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, i64, i, vp]),
            "flb_last_error": (ctypes.c_char_p, [vp]),
            "flb_create_error": (ctypes.c_char_p, []),
            "flb_version": (i, [ctypes.c_char_p, i]),
            "flb_mode_sums_noalloc": (i, [vp, i, i64, i, i, i, d, vp, vp]),
            "flb_gammas_from_viscosities": (i, [d, d, d, d, d, P(d), P(d)]),
            "flb_lattice_kT": (i, [d, d, d, d, d, P(d)]),
            "flb_lattice_params": (i, [i, d, d, d, d, d, d, d, P(d), P(d), P(d)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def config(nx=32, ny=32, nz=32, rho0=1.0, kT=0.0, gamma_shear=0.0, gamma_bulk=0.0, gamma_ghost=0.0, seed=0,
           replica=0, store=STORE_F32, pattern=PATTERN_AB, noise_ghosts=True, noise_rho_local=False, force_amp=0.0,
           sites_per_thread=0, block_x=0, block_y=0, graph_steps=0, stream=None, lattice="d3q19",
           stats_every=0) -> flb_config:
    """An flb_config from keyword arguments (defaults of flb_config_init).
    lattice "d2q9" makes an nx x ny box (nz must be 1)."""
    c = flb_config()
    lib().flb_config_init(ctypes.byref(c))
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.rho0, c.kT = float(rho0), float(kT)
    c.gamma_shear, c.gamma_bulk, c.gamma_ghost = float(gamma_shear), float(gamma_bulk), float(gamma_ghost)
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    c.replica = int(replica)
    c.store = STORE_NAMES[store] if isinstance(store, str) else int(store)
    c.pattern = {"ab": PATTERN_AB, "aa": PATTERN_AA}[pattern.lower()] if isinstance(pattern, str) else int(pattern)
    c.noise_ghosts = 1 if noise_ghosts else 0
    c.noise_rho_local = 1 if noise_rho_local else 0
    c.force_amp = float(force_amp)
    c.sites_per_thread, c.block_x, c.block_y = int(sites_per_thread), int(block_x), int(block_y)
    c.graph_steps = int(graph_steps)
    c.lattice = LATTICE_NAMES[lattice.lower()] if isinstance(lattice, str) else int(lattice)
    c.stats_every = int(stats_every)
    if stream is not None:
        # a torch.cuda.Stream, or a raw cudaStream_t as an int
        c.stream = int(getattr(stream, "cuda_stream", stream))
    return c


_live_contexts = weakref.WeakSet()


class Context:
    """Owner of one flb_ctx handle (one box, or a batch of boxes)."""

    def __init__(self, handle: ctypes.c_void_p, cfgs: list[flb_config]):
        self.h = handle
        self.cfgs = cfgs
        _live_contexts.add(self)

    # -- lifetime --------------------------------------------------------
    def close(self):
        if self.h:
            lib().flb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int):
        if rc != FLB_OK:
            raise FlbError(rc, lib().flb_last_error(self.h).decode())

    def shape(self, box=0):
        """Site shape of host fields: (nz, ny, nx), or (ny, nx) for D2Q9."""
        c = self.cfgs[box]
        return (c.ny, c.nx) if c.lattice == LATTICE_D2Q9 else (c.nz, c.ny, c.nx)

    def q(self, box=0) -> int:
        """Populations per site (19 or 9)."""
        return 9 if self.cfgs[box].lattice == LATTICE_D2Q9 else Q

    def dims(self, box=0) -> int:
        return 2 if self.cfgs[box].lattice == LATTICE_D2Q9 else 3

    # -- C ABI, one method per entry point --------------------------------
    def flb_step(self, nsteps: int):
        self._check(lib().flb_step(self.h, int(nsteps)))

    def flb_sync(self):
        self._check(lib().flb_sync(self.h))

    def flb_get_step(self) -> int:
        v = ctypes.c_uint64()
        self._check(lib().flb_get_step(self.h, ctypes.byref(v)))
        return v.value

    def flb_num_boxes(self) -> int:
        return lib().flb_num_boxes(self.h)

    def flb_get_populations(self, box=0) -> np.ndarray:
        out = np.empty((self.q(box),) + self.shape(box))
        self._check(lib().flb_box_get_populations(self.h, int(box), _ptr(out)))
        return out

    def flb_get_sites(self, sites, box=0) -> np.ndarray:
        idx = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((idx.size, self.q(box)))
        self._check(lib().flb_box_get_sites(self.h, int(box), _ptr(idx), idx.size, _ptr(out)))
        return out

    def flb_set_populations(self, n: np.ndarray, box=0):
        a = np.ascontiguousarray(n, dtype=np.float64)
        assert a.shape == (self.q(box),) + self.shape(box), a.shape
        self._check(lib().flb_box_set_populations(self.h, int(box), _ptr(a)))

    def flb_init_velocity(self, u: np.ndarray | None = None, box=0):
        a = None
        if u is not None:
            a = np.ascontiguousarray(u, dtype=np.float64)
            assert a.shape == (self.dims(box),) + self.shape(box), a.shape
        self._check(lib().flb_box_init_velocity(self.h, int(box), _ptr(a)))

    def flb_moments(self, box=0):
        shp = self.shape(box)
        d = self.dims(box)
        rho, j, Pi = np.empty(shp), np.empty((d,) + shp), np.empty((d * (d + 1) // 2,) + shp)
        self._check(lib().flb_box_moments(self.h, int(box), _ptr(rho), _ptr(j), _ptr(Pi)))
        return rho, j, Pi

    def flb_z_profile(self, box=0):
        """Plane averages along z (row averages along y for D2Q9): rho[n], j[3][n]."""
        c = self.cfgs[box]
        nz = c.ny if c.lattice == LATTICE_D2Q9 else c.nz
        rho, j = np.empty(nz), np.empty((3, nz))
        self._check(lib().flb_box_z_profile(self.h, int(box), _ptr(rho), _ptr(j)))
        return rho, j

    def flb_stats_reset(self):
        self._check(lib().flb_stats_reset(self.h))

    def flb_stats_sample(self):
        self._check(lib().flb_stats_sample(self.h))

    def flb_mode_stats(self, box=0) -> dict:
        s = flb_mode_stats_t()
        self._check(lib().flb_box_mode_stats(self.h, int(box), ctypes.byref(s)))
        return {
            "nsamples": s.nsamples, "nsites": s.nsites,
            "mode_m2": np.array(s.mode_m2[:]), "mode_ratio": np.array(s.mode_ratio[:]),
            "u2": np.array(s.u2[:]), "u2_ratio": np.array(s.u2_ratio[:]),
            "mass_first": s.mass_first, "mass_last": s.mass_last,
            "momentum_first": np.array(s.momentum_first[:]), "momentum_last": np.array(s.momentum_last[:]),
            "nonfinite": s.nonfinite,
        }

    def flb_enable_structure_factor(self, box=0):
        self._check(lib().flb_box_enable_structure_factor(self.h, int(box)))

    def flb_structure_factor(self, nshells: int, box=0):
        S = np.zeros(int(nshells))
        cnt = np.zeros(int(nshells), dtype=np.int64)
        self._check(lib().flb_box_structure_factor(self.h, int(box), _ptr(S), _ptr(cnt), int(nshells)))
        return S, cnt

    def flb_state_bytes(self, box=0) -> int:
        v = ctypes.c_size_t()
        self._check(lib().flb_box_state_bytes(self.h, int(box), ctypes.byref(v)))
        return v.value

    def flb_state_download(self, host: np.ndarray, box=0):
        assert host.nbytes >= self.flb_state_bytes(box)
        self._check(lib().flb_box_state_download(self.h, int(box), _ptr(host)))

    def flb_state_upload(self, host: np.ndarray, box=0):
        assert host.nbytes >= self.flb_state_bytes(box)
        self._check(lib().flb_box_state_upload(self.h, int(box), _ptr(host)))

    def flb_step_host(self, host: np.ndarray, nsteps: int = 1, box=0):
        """Upload the raw state in `host`, advance nsteps, download it back (overlapped)."""
        assert host.nbytes >= self.flb_state_bytes(box)
        self._check(lib().flb_box_step_host(self.h, int(box), _ptr(host), int(nsteps)))

    def flb_save(self, path: str):
        self._check(lib().flb_save(self.h, path.encode()))

    def flb_load(self, path: str):
        self._check(lib().flb_load(self.h, path.encode()))

    def flb_bounds_violations(self) -> int:
        """Out-of-range accesses the kernels caught (checking build only)."""
        n = ctypes.c_uint64()
        self._check(lib().flb_bounds_violations(self.h, ctypes.byref(n)))
        return n.value

    def flb_bounds_selftest(self):
        self._check(lib().flb_bounds_selftest(self.h))

    def flb_get_launch(self):
        V, bx, by = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().flb_get_launch(self.h, ctypes.byref(V), ctypes.byref(bx), ctypes.byref(by)))
        return V.value, bx.value, by.value

    def flb_set_launch(self, V: int, bx: int, by: int):
        self._check(lib().flb_set_launch(self.h, int(V), int(bx), int(by)))

    def flb_autotune(self, trials: int = 3, pattern: bool = False):
        """Time the launch shapes (and with pattern=True also the other streaming pattern)."""
        if pattern:
            self._check(lib().flb_autotune_ex(self.h, int(trials), TUNE_PATTERN))
        else:
            self._check(lib().flb_autotune(self.h, int(trials)))

    def flb_check_finite(self, box=0) -> int:
        """Number of non-finite stored populations (0 when the state is healthy)."""
        v = ctypes.c_uint64()
        rc = lib().flb_box_check_finite(self.h, int(box), ctypes.byref(v))
        if rc not in (FLB_OK, FLB_ENONFINITE):
            self._check(rc)
        return v.value

    def flb_get_pattern(self) -> str:
        v = ctypes.c_int()
        self._check(lib().flb_get_pattern(self.h, ctypes.byref(v)))
        return "ab" if v.value == PATTERN_AB else "aa"

    def flb_set_pattern(self, pattern: str):
        self._check(lib().flb_set_pattern(self.h, {"ab": PATTERN_AB, "aa": PATTERN_AA}[pattern.lower()]))


def _created(rc: int, h: ctypes.c_void_p, cfgs) -> Context:
    if rc != FLB_OK:
        raise FlbError(rc, lib().flb_create_error().decode())
    return Context(h, list(cfgs))


def flb_create(nx, ny, nz, rho0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed) -> Context:
    h = ctypes.c_void_p()
    rc = lib().flb_create(int(nx), int(ny), int(nz), float(rho0), float(kT), float(gamma_shear), float(gamma_bulk),
                          float(gamma_ghost), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(h))
    cfg = config(nx, ny, nz, rho0, kT, gamma_shear, gamma_bulk, gamma_ghost, seed)
    return _created(rc, h, [cfg])


def flb_create_ex(cfg: flb_config) -> Context:
    h = ctypes.c_void_p()
    rc = lib().flb_create_ex(ctypes.byref(cfg), ctypes.byref(h))
    return _created(rc, h, [cfg])


def flb_create_batch(cfgs: list[flb_config]) -> Context:
    arr = (flb_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    rc = lib().flb_create_batch(arr, len(cfgs), ctypes.byref(h))
    return _created(rc, h, cfgs)


DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_keep = []   # every installed hook stays alive: contexts made under it free through it


def flb_set_device_allocator(alloc=None, free=None):
    """Device allocator of the contexts created from now on: alloc(nbytes,
    stream) -> device pointer as an int (0 or None on failure) and free(ptr,
    stream), stream being the context's cudaStream_t as an int; both None
    restores cudaMalloc / cudaFree."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        rc = lib().flb_set_device_allocator(None, None, None)
    else:
        def a(nbytes, stream, user):
            try:
                return alloc(int(nbytes), int(stream or 0)) or None
            except Exception:
                return None

        def f(ptr, stream, user):
            try:
                free(int(ptr), int(stream or 0))
            except Exception:
                pass

        cb = (DEV_ALLOC_FN(a), DEV_FREE_FN(f))
        _allocator_keep.append(cb)
        rc = lib().flb_set_device_allocator(ctypes.cast(cb[0], ctypes.c_void_p), ctypes.cast(cb[1], ctypes.c_void_p),
                                            None)
    if rc != FLB_OK:
        raise FlbError(rc, "flb_set_device_allocator failed")


def use_torch_allocator(enable: bool = True):
    """torch's caching allocator (on the context's stream) for the device memory
    of the contexts created from now on; False restores cudaMalloc / cudaFree."""
    if not enable:
        flb_set_device_allocator(None, None)
        return
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    flb_set_device_allocator(alloc, free)


@atexit.register
def _close_live_contexts():
    # before interpreter teardown, while the allocator callbacks can still run
    for ctx in list(_live_contexts):
        try:
            ctx.close()
        except Exception:
            pass


def flb_mode_sums_noalloc(populations_ptr: int, store: int, plane: int, nx: int, ny: int, nz: int, rho0: float,
                          sums_ptr: int, stream: int | None = None) -> int:
    """Raw call of the allocation-free statistics entry point (device pointers as ints)."""
    return lib().flb_mode_sums_noalloc(ctypes.c_void_p(populations_ptr), int(store), int(plane), int(nx), int(ny),
                                       int(nz), float(rho0), ctypes.c_void_p(sums_ptr),
                                       None if stream is None else ctypes.c_void_p(int(stream)))


def flb_gammas_from_viscosities(eta, zeta, rho, b, h):
    gs, gb = ctypes.c_double(), ctypes.c_double()
    rc = lib().flb_gammas_from_viscosities(float(eta), float(zeta), float(rho), float(b), float(h), ctypes.byref(gs),
                                           ctypes.byref(gb))
    if rc != FLB_OK:
        raise FlbError(rc, "viscosities, density, b and h must be positive and finite")
    return gs.value, gb.value


def flb_lattice_kT(kT, rho, b, h, rho0=1.0):
    out = ctypes.c_double()
    rc = lib().flb_lattice_kT(float(kT), float(rho), float(b), float(h), float(rho0), ctypes.byref(out))
    if rc != FLB_OK:
        raise FlbError(rc, "kT, rho, b, h and rho0 must be positive and finite")
    return out.value


def flb_lattice_params(d, eta, zeta, kT, rho, b, h, rho0=1.0):
    """(gamma_shear, gamma_bulk, kT_lattice) for a d-dimensional lattice (d = 2 or 3)."""
    gs, gb, kt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().flb_lattice_params(int(d), float(eta), float(zeta), float(kT), float(rho), float(b), float(h),
                                  float(rho0), ctypes.byref(gs), ctypes.byref(gb), ctypes.byref(kt))
    if rc != FLB_OK:
        raise FlbError(rc, "d must be 2 or 3, kT >= 0, the other inputs positive and finite")
    return gs.value, gb.value, kt.value


def flb_philox4x32_10(ctr, key) -> np.ndarray:
    """The device Philox-4x32-10 of counters ctr[n, 4] under keys key[n, 2]."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(c)
    rc = lib().flb_philox4x32_10(_ptr(c), _ptr(k), c.shape[0], _ptr(out))
    if rc != FLB_OK:
        raise FlbError(rc, "device Philox failed")
    return out


def flb_normals(seed, step, replica, site0, nsites, fp64=True) -> np.ndarray:
    """The sixteen normals per site that the FP64 (or FP32) kernels draw: [nsites, 16]."""
    out = np.zeros((int(nsites), 16))
    rc = lib().flb_normals(int(seed) & 0xFFFFFFFFFFFFFFFF, int(step), int(replica), int(site0), int(nsites),
                           1 if fp64 else 0, _ptr(out))
    if rc != FLB_OK:
        raise FlbError(rc, "device normals failed")
    return out


class HostBuffer:
    """Page-locked host memory from flb_host_alloc (huge pages where offered,
    registered with the driver); `array` is a uint8 numpy view of it.  Free it
    with close() (or a with-block); the view must not be used afterwards."""

    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        rc = lib().flb_host_alloc(int(nbytes), ctypes.byref(p))
        if rc != FLB_OK:
            raise FlbError(rc, f"flb_host_alloc({nbytes}) failed")
        self.ptr, self.nbytes = p.value, int(nbytes)
        self.array = np.ctypeslib.as_array((ctypes.c_uint8 * self.nbytes).from_address(self.ptr))

    def close(self):
        if self.ptr:
            self.array = None
            ptr, self.ptr = self.ptr, None
            rc = lib().flb_host_free(ptr)
            if rc != FLB_OK:
                raise FlbError(rc, "flb_host_free failed")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flb_version() -> str:
    buf = ctypes.create_string_buffer(256)
    lib().flb_version(buf, 256)
    return buf.value.decode()
