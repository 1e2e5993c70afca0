"""The C-ABI library loads and exports every symbol include/flb.h declares;
host-side parameter checks answer without a GPU."""
import ctypes
import os
import re

import pytest

from paper_0707_1581_gb300 import flb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_0707_1581_gb300 import build as B
    B.build()
    return flb.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "flb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flb_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("flb_create", "flb_step", "flb_moments", "flb_mode_stats", "flb_create_batch",
                 "flb_get_populations", "flb_set_populations", "flb_box_structure_factor"):
        assert name in syms


def test_library_exports_every_declared_symbol(L):
    syms = declared_symbols()
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(flb.EXPORTS) == syms


def test_version_string(L):
    v = flb.flb_version()
    assert "sm_103a" in v


def _create_rc(**kw):
    cfg = flb.config(**kw)
    h = ctypes.c_void_p()
    rc = flb.lib().flb_create_ex(ctypes.byref(cfg), ctypes.byref(h))
    return rc, flb.lib().flb_create_error().decode(), h


@pytest.mark.parametrize("kw,word", [
    (dict(gamma_shear=1.5), "gamma_shear"),
    (dict(gamma_bulk=-1.01), "gamma_bulk"),
    (dict(gamma_ghost=float("nan")), "gamma_ghost"),
    (dict(kT=-1e-4), "kT"),
    (dict(rho0=0.0), "rho0"),
    (dict(nx=0), "edges"),
    (dict(nx=2048, ny=2048, nz=1024), "2^31"),
    (dict(store=7), "store"),
    (dict(pattern=3), "pattern"),
    (dict(sites_per_thread=3), "sites_per_thread"),
    (dict(block_x=512, block_y=1), "block"),
    (dict(lattice=7), "lattice"),
    (dict(nz=2, lattice="d2q9"), "nz = 1"),
    (dict(graph_steps=-1), "graph_steps"),
    (dict(stats_every=-5), "stats_every"),
    (dict(force_amp=float("inf")), "force_amp"),
])
def test_invalid_parameters_are_rejected_on_the_host(L, kw, word):
    rc, msg, h = _create_rc(**kw)
    assert rc == flb.FLB_EINVAL
    assert word in msg
    assert not h.value


def test_batch_reports_the_bad_box(L):
    cfgs = [flb.config(nx=8, ny=8, nz=8), flb.config(nx=8, ny=8, nz=8, gamma_shear=2.0)]
    arr = (flb.flb_config * 2)(*cfgs)
    h = ctypes.c_void_p()
    rc = flb.lib().flb_create_batch(arr, 2, ctypes.byref(h))
    assert rc == flb.FLB_EINVAL
    assert "box 1" in flb.lib().flb_create_error().decode()


def test_null_handles_are_rejected(L):
    assert L.flb_bounds_violations(None, None) == flb.FLB_EINVAL
    assert L.flb_bounds_selftest(None) == flb.FLB_EINVAL
    assert L.flb_step(None, 1) == flb.FLB_EINVAL
    assert L.flb_sync(None) == flb.FLB_EINVAL
    assert L.flb_num_boxes(None) == 0
    L.flb_destroy(None)


def test_host_alloc_rejects_bad_arguments_on_the_host(L):
    out = ctypes.c_void_p()
    assert L.flb_host_alloc(0, ctypes.byref(out)) == flb.FLB_EINVAL
    assert L.flb_host_alloc(4096, None) == flb.FLB_EINVAL
    assert L.flb_host_free(None) == flb.FLB_OK
    buf = ctypes.create_string_buffer(64)            # not from flb_host_alloc
    assert L.flb_host_free(ctypes.addressof(buf)) == flb.FLB_EINVAL


def test_device_allocator_hook_takes_both_functions_or_neither(L):
    fn = flb.DEV_FREE_FN(lambda p, s, u: None)
    assert L.flb_set_device_allocator(None, ctypes.cast(fn, ctypes.c_void_p), None) == flb.FLB_EINVAL
    assert L.flb_set_device_allocator(None, None, None) == flb.FLB_OK


def test_no_gpu_fails_loudly_not_silently(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, msg, h = _create_rc(nx=8, ny=8, nz=8)
    assert rc == flb.FLB_ECUDA
    assert not h.value


def test_config_struct_layout_matches_the_library(L):
    """flb_config_init clears sizeof(flb_config) bytes: exactly the binding's
    struct (nothing beyond it, the last field included)."""
    n = ctypes.sizeof(flb.flb_config)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    L.flb_config_init(ctypes.cast(buf, ctypes.POINTER(flb.flb_config)))
    assert all(b == 0xAB for b in buf[n:])
    c = ctypes.cast(buf, ctypes.POINTER(flb.flb_config)).contents
    assert c.stream is None and c.stats_every == 0 and c.lattice == 0 and c.nx == 32


def test_config_defaults(L):
    c = flb.flb_config()
    L.flb_config_init(ctypes.byref(c))
    assert (c.nx, c.ny, c.nz) == (32, 32, 32)
    assert c.rho0 == 1.0 and c.kT == 0.0
    assert c.store == flb.STORE_F32 and c.pattern == flb.PATTERN_AB
    assert c.noise_ghosts == 1
