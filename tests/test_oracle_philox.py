"""Pins of the oracle's random numbers.

The paper only asks for Gaussian numbers of zero mean and unit variance
(Sec. IV, Eq. updaterule).  The oracle uses Philox-4x32-10 (Salmon et al.,
SC'11), two 16-bit uniforms per 32-bit word and the Box-Muller transform.  Philox is pinned against two independent
library implementations that are called, not read: cuRAND's host-side
generator (counter words 0..2) and the header-only engine shipped with
PyTorch (all four counter words, through its subsequence argument).
"""
import ctypes
import ctypes.util
import os
import subprocess

import numpy as np
import pytest


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    path = "/usr/local/cuda/lib64/libcurand.so"
    if os.path.exists(path):
        return ctypes.CDLL(path)
    return None


def _curand_host_words(lib, seed, nwords, offset=0):
    gen = ctypes.c_void_p()
    PHILOX4_32_10 = 161
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 7, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(ora, seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    # cuRAND's host generator emits block B with counter
    # (lo32(B >> 16), hi32(B >> 16), B & 0xffff, 0) and key (lo32(seed), hi32(seed)).
    for offset_blocks in (0, 3 * 65536 + 11, (1 << 48) + 5):
        nb = 70000 if offset_blocks == 0 else 4096
        words = _curand_host_words(lib, seed, 4 * nb, 4 * offset_blocks).reshape(nb, 4)
        B = np.arange(nb, dtype=np.uint64) + np.uint64(offset_blocks)
        hi = B >> np.uint64(16)
        ctr = np.zeros((nb, 4), dtype=np.uint32)
        ctr[:, 0] = (hi & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        ctr[:, 1] = (hi >> np.uint64(32)).astype(np.uint32)
        ctr[:, 2] = (B & np.uint64(0xFFFF)).astype(np.uint32)
        key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (nb, 1))
        assert np.array_equal(ora.philox(ctr, key), words)


_ATEN_DRIVER = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::Philox4_32 e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def test_philox_matches_torch_header_engine(ora, tmp_path):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("torch Philox header not shipped")
    src = tmp_path / "drv.cpp"
    src.write_text(_ATEN_DRIVER)
    exe = tmp_path / "drv"
    try:
        subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}", str(src), "-o", str(exe)],
                       check=True, capture_output=True)
    except (OSError, subprocess.CalledProcessError) as err:
        pytest.skip(f"cannot build the torch Philox driver: {err}")
    rng = np.random.default_rng(2024)
    n = 3000
    seeds = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    subs = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    offs = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    inp = "\n".join(f"{int(a)} {int(b)} {int(c)}" for a, b, c in zip(seeds, subs, offs))
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(v) for v in line.split()] for line in out.strip().splitlines()], dtype=np.uint32)
    ctr = np.stack([offs & 0xFFFFFFFF, offs >> np.uint64(32), subs & 0xFFFFFFFF, subs >> np.uint64(32)], 1)
    key = np.stack([seeds & 0xFFFFFFFF, seeds >> np.uint64(32)], 1)
    got = ora.philox(ctr.astype(np.uint32), key.astype(np.uint32))
    assert np.array_equal(got, ref)


def test_uniform_mapping_is_exact_and_open(ora):
    assert ora.uniform16(0) == 2.0 ** -17
    assert ora.uniform16(0xFFFF) == 1.0 - 2.0 ** -17
    for h in range(0, 65536, 97):
        u = ora.uniform16(h)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # exact in binary32
        assert u == (h + 0.5) / 2 ** 16


def test_box_muller_identities(ora):
    """Word p of the two Philox blocks gives pair (g[2p], g[2p+1]) with
    radius^2 = -2 ln u(low 16 bits) and angle 2 pi u(high 16 bits)."""
    seed, site, step, rep = 99, 1234, 56, 7
    g = ora.gaussians(seed, site, step, rep)
    for b in range(2):
        w = ora.philox([[site, step, rep, b]], [[seed & 0xFFFFFFFF, seed >> 32]])[0]
        for j in range(4):
            p = 4 * b + j
            g0, g1 = g[2 * p], g[2 * p + 1]
            u1, u2 = ora.uniform16(int(w[j]) & 0xFFFF), ora.uniform16(int(w[j]) >> 16)
            assert g0 * g0 + g1 * g1 == pytest.approx(-2 * np.log(u1), rel=1e-13)
            ang = np.arctan2(g1, g0) / (2 * np.pi) % 1.0
            assert ang == pytest.approx(u2, abs=1e-12)


def test_sixteen_bit_normals_exact_moments():
    """Over all 2^16 radius and angle values the discrete Box-Muller normals
    have variance 1 - 5.3e-6, kurtosis 2.9998 and a cut at 4.855 sigma."""
    h = np.arange(65536, dtype=np.float64)
    u = (h + 0.5) / 65536
    r2 = -2 * np.log(u)
    assert abs(r2.mean() / 2 - 1) < 1e-5
    assert abs(3 * (r2 ** 2).mean() / 8 / (r2.mean() / 2) ** 2 - 3) < 1e-3
    assert np.sqrt(r2.max()) == pytest.approx(4.8546, abs=1e-4)


def test_normals_moments(ora):
    """Mean 0, variance 1, kurtosis 3 and no correlation between the 16 normals
    of a site, over 2^18 sites x 16 = 4.2M draws (5 sigma bounds)."""
    g = ora.gaussians_many(11, 3, 0, 1 << 18)
    x = g.reshape(-1)
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / n)
    kurt = np.mean(x ** 4) / np.mean(x ** 2) ** 2
    assert abs(kurt - 3) < 5 * np.sqrt(24 / n)
    C = np.corrcoef(g.T)
    off = C[~np.eye(16, dtype=bool)]
    assert np.abs(off).max() < 5 / np.sqrt(g.shape[0])
