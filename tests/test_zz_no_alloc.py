"""The allocation-free statistics entry point, for callers that must not
allocate device memory (cudaMalloc stalls the whole device and may fail; some
hosts hand a library only the buffers it works on).  Its sums must equal the
ordinary statistics path on the same state, on two calls in a row (the
static scratch array keeps the previous call's contents, which must not leak
into the next result)."""
import numpy as np
import pytest

from paper_0707_1581_gb300 import flb

pytestmark = pytest.mark.gpu


# format -> (store code, element bytes, relative tolerance of the sums): FP64
# states are summed in FP64 on both paths; the other formats collect per-lane
# FP32 partials, which the two paths group differently
FORMATS = {
    "f64": (flb.STORE_F64, 8, 1e-12),
    "f32": (flb.STORE_F32, 4, 1e-5),
    "f16dev": (flb.STORE_F16DEV, 2, 1e-5),
    "bf16dev": (flb.STORE_BF16DEV, 2, 1e-5),
    "bf16sr": (flb.STORE_BF16SR, 2, 1e-5),
}


@pytest.mark.parametrize("store", list(FORMATS))
def test_noalloc_sums_equal_the_allocating_path_twice(store):
    torch = pytest.importorskip("torch")
    from paper_0707_1581_gb300 import build as B
    B.build()
    code, elt, rtol = FORMATS[store]
    nx, ny, nz = 24, 20, 16
    N = nx * ny * nz
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 5, store=store, pattern="aa")
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(6)     # even step: the AA buffer holds the populations in natural order
        ctx.flb_stats_reset()
        ctx.flb_stats_sample()
        ref = ctx.flb_mode_stats()
        nbytes = ctx.flb_state_bytes()
        host = np.empty(nbytes, dtype=np.uint8)
        ctx.flb_state_download(host)
    plane = nbytes // (19 * elt)
    pop = torch.from_numpy(host).cuda()          # caller-owned device input
    sums = torch.empty(27, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        sums.fill_(-7.0)
        rc = flb.flb_mode_sums_noalloc(pop.data_ptr(), code, plane, nx, ny, nz, 1.0, sums.data_ptr())
        assert rc == flb.FLB_OK
        torch.cuda.synchronize()
        s = sums.cpu().numpy()
        np.testing.assert_allclose(s[:19] / N, ref["mode_m2"], rtol=rtol)
        np.testing.assert_allclose(s[19:22] / N, ref["u2"], rtol=rtol)
        assert s[22] == pytest.approx(ref["mass_last"], rel=1e-9)
        np.testing.assert_allclose(s[23:26], ref["momentum_last"], rtol=0, atol=1e-6)
        assert s[26] == ref["nonfinite"] == 0


def test_noalloc_rejects_boxes_over_the_limit():
    torch = pytest.importorskip("torch")
    x = torch.zeros(16, device="cuda")
    rc = flb.flb_mode_sums_noalloc(x.data_ptr(), flb.STORE_F32, 1 << 25, 512, 512, 65, 1.0, x.data_ptr())
    assert rc == flb.FLB_ERANGE


@pytest.mark.parametrize("plane_pad,offset", [(3, 0), (64, 1), (5, 2)])
def test_noalloc_accepts_any_plane_stride_and_element_offset(plane_pad, offset):
    """A caller's populations need not be laid out like the library's: a plane
    stride that is not a multiple of 4 elements, or a base pointer one or two
    elements past an aligned address, take the scalar loads and give the same
    sums as the packed, aligned layout (up to the grouping of the FP32 partials)."""
    torch = pytest.importorskip("torch")
    from paper_0707_1581_gb300 import build as B
    B.build()
    nx, ny, nz = 24, 20, 16
    N = nx * ny * nz
    rng = np.random.default_rng(plane_pad)
    a = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=np.float32)
    dev = (0.01 * a[:, None] * rng.standard_normal((19, N))).astype(np.float32)   # deviations n_i - rho0 a_i
    packed = torch.from_numpy(dev.copy()).cuda()
    plane = N + plane_pad
    flat = torch.zeros(offset + 19 * plane, dtype=torch.float32, device="cuda")
    flat[offset:].view(19, plane)[:, :N] = packed
    out = []
    for ptr, pl in ((packed.data_ptr(), N), (flat.data_ptr() + 4 * offset, plane)):
        sums = torch.empty(27, dtype=torch.float64, device="cuda")
        assert flb.flb_mode_sums_noalloc(ptr, flb.STORE_F32, pl, nx, ny, nz, 1.0, sums.data_ptr()) == flb.FLB_OK
        torch.cuda.synchronize()
        out.append(sums.cpu().numpy())
    np.testing.assert_allclose(out[1][:22], out[0][:22], rtol=1e-5)
    assert out[1][22] == pytest.approx(out[0][22], rel=1e-9)      # rho0 N plus FP32-grouped deviations
    np.testing.assert_allclose(out[1][23:26], out[0][23:26], rtol=0, atol=1e-5)
