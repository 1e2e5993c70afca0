"""The largest boxes the library accepts (nx ny nz < 2^31 sites): 32-bit site
indices and 64-bit plane offsets at their limits.  Two thermal, forced steps
from rest on one GPU; sampled sites (the corners and the last site among them)
are recomputed by the oracle one collision at a time, as in the full-size
parity test of the benchmark box."""
import numpy as np
import pytest

from paper_0707_1581_gb300 import flb
from paper_0707_1581_gb300.inputs import sample_sites

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


def _need(nbytes):
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes * 1.05:
        pytest.skip(f"needs {nbytes / 1e9:.0f} GB of free device memory")


def _sites(shape, count, seed):
    N = int(np.prod(shape))
    corners = [0, N - 1, shape[0] - 1, N - shape[0]]
    return np.unique(np.concatenate([np.array(corners, dtype=np.int64), sample_sites(N, count, seed=seed)]))


def test_d3q19_largest_box_sampled_sites(ora):
    nx, ny, nz = 2048, 1024, 1023                  # 2,145,386,496 sites, 163 GB of FP32 state
    N = nx * ny * nz
    assert N < 2 ** 31 and N > 2 ** 31 - 2 ** 22
    _need(19 * N * 4)
    kT, gs, gb, gg, seed, F0 = 1e-4, 0.3, 0.2, 0.0, 3, 1e-5
    cfg = flb.config(nx, ny, nz, 1.0, kT, gs, gb, gg, seed, store="f32", pattern="aa", force_amp=F0)
    sites = _sites((nx, ny, nz), 60, seed=2)
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(2)
        got = ctx.flb_get_sites(sites)
    c, a, _, _ = ora.lattice()
    p = ora.make_params(nx, ny, nz, rho0=1.0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=seed,
                        force_amp=F0)
    memo = {}

    def n_at(x, y, z, t):
        key = (x % nx, y % ny, z % nz, t)
        if key in memo:
            return memo[key]
        x, y, z = key[:3]
        if t == 0:
            val = a.copy()                         # rest
        else:
            val = np.empty(19)
            for i in range(19):
                xs, ys, zs = (x - c[i, 0]) % nx, (y - c[i, 1]) % ny, (z - c[i, 2]) % nz
                prev = n_at(xs, ys, zs, t - 1)
                Fx = F0 * np.sin(2 * np.pi * zs / nz)
                val[i] = ora.collide_site(p, prev, site=int(xs + nx * (ys + ny * zs)), step=t - 1,
                                          force=[Fx, 0, 0])[i]
        memo[key] = val
        return val

    worst = 0.0
    for k, s in enumerate(sites):
        x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
        worst = max(worst, np.abs(got[k] - n_at(x, y, z, 2)).max())
    assert worst <= 1e-5


def test_d2q9_largest_box_sampled_sites():
    from oracle import d2q9 as D
    nx = ny = 46340                                # 2,147,395,600 sites, 77 GB of FP32 state
    N = nx * ny
    assert N < 2 ** 31 and N > 2 ** 31 - 2 ** 18
    _need(9 * N * 4)
    kT, gs, gb, gg, seed, F0 = 1e-4, 0.3, 0.2, 0.0, 3, 1e-5
    cfg = flb.config(nx, ny, 1, 1.0, kT, gs, gb, gg, seed, store="f32", pattern="aa", force_amp=F0, lattice="d2q9")
    sites = _sites((nx, ny), 60, seed=3)
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(2)
        got = ctx.flb_get_sites(sites)
    c, a = D.lattice()[0], D.lattice()[1]
    p = D.make_params(nx, ny, rho0=1.0, kT=kT, gamma_shear=gs, gamma_bulk=gb, gamma_ghost=gg, seed=seed,
                      force_amp=F0)
    memo = {}

    def n_at(x, y, t):
        key = (x % nx, y % ny, t)
        if key in memo:
            return memo[key]
        x, y = key[:2]
        if t == 0:
            val = a.copy()
        else:
            val = np.empty(9)
            for i in range(9):
                xs, ys = (x - c[i, 0]) % nx, (y - c[i, 1]) % ny
                prev = n_at(xs, ys, t - 1)
                Fx = F0 * np.sin(2 * np.pi * ys / ny)
                val[i] = D.collide_site(p, prev, site=int(xs + nx * ys), step=t - 1, force=[Fx, 0])[i]
        memo[key] = val
        return val

    worst = 0.0
    for k, s in enumerate(sites):
        worst = max(worst, np.abs(got[k] - n_at(s % nx, s // nx, 2)).max())
    assert worst <= 1e-5
