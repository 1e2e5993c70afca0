"""Runtime features of the library on the GPU: autotuner, checkpoint errors,
step-counter range, batched graphs, error reporting."""
import numpy as np
import pytest

from paper_0707_1581_gb300 import flb
from paper_0707_1581_gb300.inputs import relative_perturbation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0707_1581_gb300 import build as B
    B.build()


def state_of(weights, shape, seed):
    return weights[:, None, None, None] * relative_perturbation(shape, seed=seed, amp=0.02)


@pytest.fixture(scope="module")
def weights(ora):
    return ora.lattice()[1]


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_autotune_restores_state_and_keeps_results(weights, pattern):
    nx, ny, nz = 64, 16, 8
    n0 = state_of(weights, (nz, ny, nx), 1)
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 2, store="f32", pattern=pattern)
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(3)
        before = ref.flb_get_populations()
        ref.flb_step(4)
        want = ref.flb_get_populations()
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_step(3)
        ctx.flb_autotune(2)
        assert ctx.flb_get_step() == 3
        assert np.array_equal(ctx.flb_get_populations(), before)
        V, bx, by = ctx.flb_get_launch()
        assert V in (1, 2, 4) and bx * by <= 256 and nx % V == 0
        ctx.flb_step(4)
        # the noise is keyed by site and step, not by launch shape; only the
        # rounding of the arithmetic may differ between kernel variants
        assert np.abs(ctx.flb_get_populations() - want).max() <= 1e-6


def test_batch_with_graphs_and_autotune(weights):
    shapes = [(32, 8, 8), (64, 4, 4), (16, 16, 16)]
    cfgs = [flb.config(nx, ny, nz, 1.0, 1e-4, 0.2 + 0.1 * r, 0.2, 0.0, 9, replica=r, store="f32", pattern="aa",
                       graph_steps=4) for r, (nx, ny, nz) in enumerate(shapes)]
    plain = [flb.config(nx, ny, nz, 1.0, 1e-4, 0.2 + 0.1 * r, 0.2, 0.0, 9, replica=r, store="f32", pattern="aa")
             for r, (nx, ny, nz) in enumerate(shapes)]
    starts = [state_of(weights, (nz, ny, nx), 10 + b) for b, (nx, ny, nz) in enumerate(shapes)]
    results = []
    for cs, tune in ((cfgs, True), (plain, False)):
        with flb.flb_create_batch(cs) as ctx:
            for b, n0 in enumerate(starts):
                ctx.flb_set_populations(n0, box=b)
            if tune:
                ctx.flb_autotune(1)
            ctx.flb_step(10)
            results.append([ctx.flb_get_populations(box=b) for b in range(len(shapes))])
    for a, b in zip(*results):
        assert np.abs(a - b).max() <= 1e-6


def test_checkpoint_errors(tmp_path, weights):
    cfg = flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store="f32")
    path = str(tmp_path / "ck.flb")
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(2)
        ctx.flb_save(path)
        with pytest.raises(flb.FlbError) as e:
            ctx.flb_load(str(tmp_path / "missing.flb"))
        assert e.value.code == flb.FLB_EIO
    data = open(path, "rb").read()
    open(str(tmp_path / "short.flb"), "wb").write(data[: len(data) // 2])
    open(str(tmp_path / "bad.flb"), "wb").write(b"XXXXXXXX" + data[8:])
    with flb.flb_create_ex(cfg) as ctx:
        for name in ("short.flb", "bad.flb"):
            with pytest.raises(flb.FlbError) as e:
                ctx.flb_load(str(tmp_path / name))
            assert e.value.code == flb.FLB_EIO
    other = flb.config(16, 8, 4, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store="f32")
    with flb.flb_create_ex(other) as ctx:
        with pytest.raises(flb.FlbError) as e:
            ctx.flb_load(path)
        assert e.value.code == flb.FLB_EIO
    f16 = flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store="f16dev")
    with flb.flb_create_ex(f16) as ctx:
        with pytest.raises(flb.FlbError):
            ctx.flb_load(path)
    # another seed, kT or eigenvalue would continue a different noise stream or dynamics
    for other in (flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 2, store="f32"),
                  flb.config(16, 8, 8, 1.0, 2e-4, 0.3, 0.2, 0.0, 1, store="f32"),
                  flb.config(16, 8, 8, 1.0, 1e-4, 0.4, 0.2, 0.0, 1, store="f32")):
        with flb.flb_create_ex(other) as ctx:
            with pytest.raises(flb.FlbError) as e:
                ctx.flb_load(path)
            assert e.value.code == flb.FLB_EIO
    # a corrupt header: the buffer index (int32 after magic, version, nboxes,
    # store, pattern) outside {0, 1}, or a step counter past 2^32 - 1
    cur_at, step_at = 8 + 4 + 4 + 4 + 4, 8 + 4 + 4 + 4 + 4 + 4 + 4
    bad_cur = bytearray(data)
    bad_cur[cur_at:cur_at + 4] = (7).to_bytes(4, "little", signed=True)
    bad_step = bytearray(data)
    bad_step[step_at:step_at + 8] = (1 << 33).to_bytes(8, "little")
    open(str(tmp_path / "cur.flb"), "wb").write(bytes(bad_cur))
    open(str(tmp_path / "step.flb"), "wb").write(bytes(bad_step))
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(3)
        before = ctx.flb_get_populations()
        for name in ("cur.flb", "step.flb", "short.flb"):
            with pytest.raises(flb.FlbError) as e:
                ctx.flb_load(str(tmp_path / name))
            assert e.value.code == flb.FLB_EIO
        # nothing was uploaded: the context still holds its own state and step
        assert ctx.flb_get_step() == 3
        assert np.array_equal(ctx.flb_get_populations(), before)


def test_step_counter_range_and_bad_arguments():
    with flb.flb_create_ex(flb.config(8, 8, 8, store="f32")) as ctx:
        with pytest.raises(flb.FlbError) as e:
            ctx.flb_step(-1)
        assert e.value.code == flb.FLB_EINVAL
        with pytest.raises(flb.FlbError) as e:
            ctx.flb_step(1 << 32)
        assert e.value.code == flb.FLB_ERANGE
        assert ctx.flb_get_step() == 0
        with pytest.raises(flb.FlbError) as e:
            ctx.flb_get_sites([8 ** 3])
        assert e.value.code == flb.FLB_EINVAL
        with pytest.raises(flb.FlbError):
            ctx.flb_structure_factor(4)        # not enabled
        out = np.empty(19 * 8 ** 3)
        assert flb.lib().flb_box_get_populations(ctx.h, 1, out.ctypes.data) == flb.FLB_EINVAL   # no such box


def test_torch_stream_is_used(weights):
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    n0 = state_of(weights, (8, 8, 16), 3)
    with flb.flb_create_ex(flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store="f32", stream=s)) as a, \
            flb.flb_create_ex(flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store="f32")) as b:
        for c in (a, b):
            c.flb_set_populations(n0)
            c.flb_step(5)
        assert np.array_equal(a.flb_get_populations(), b.flb_get_populations())


@pytest.mark.parametrize("store,pattern,shape,start,nsteps", [
    ("f32", "aa", (64, 16, 40), 0, 1),     # AA even step: chunks are independent
    ("f32", "aa", (64, 16, 40), 1, 1),     # AA odd step: chunks need their neighbours
    ("f32", "ab", (64, 16, 40), 0, 1),
    ("f32", "ab", (64, 16, 40), 1, 1),
    ("f16dev", "aa", (32, 8, 17), 1, 1),
    ("bf16sr", "aa", (32, 8, 17), 0, 1),
    ("f32", "aa", (16, 8, 2), 1, 1),       # two chunks of one plane
    ("f32", "aa", (16, 8, 1), 1, 1),       # one chunk
    ("f64", "aa", (24, 8, 20), 1, 3),      # several steps: only the first is chunked
])
def test_host_resident_stepping_matches_device_stepping(weights, store, pattern, shape, start, nsteps):
    nx, ny, nz = shape
    n0 = state_of(weights, (nz, ny, nx), 5)
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, store=store, pattern=pattern, force_amp=1e-5)
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(start)
        host = np.zeros(ref.flb_state_bytes(), np.uint8)
        ref.flb_state_download(host)
        ref.flb_step(nsteps)
        want_raw = np.zeros_like(host)
        ref.flb_state_download(want_raw)
        want = ref.flb_get_populations()
        ref.flb_step(2)
        later = ref.flb_get_populations()
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_step(start)
        ctx.flb_init_velocity(None)            # a different device state: the upload must replace it
        ctx.flb_step_host(host, nsteps)
        assert ctx.flb_get_step() == start + nsteps
        assert np.array_equal(host, want_raw)
        assert np.array_equal(ctx.flb_get_populations(), want)
        ctx.flb_step(2)                        # the device state and orientation carry on
        assert np.array_equal(ctx.flb_get_populations(), later)


@pytest.mark.parametrize("start", [0, 1])
def test_host_resident_stepping_from_the_library_host_buffer(weights, start):
    nx, ny, nz = 64, 32, 48
    n0 = state_of(weights, (nz, ny, nx), 6)
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, store="f32", pattern="aa", force_amp=1e-5)
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(start + 2)
        want = np.zeros(ref.flb_state_bytes(), np.uint8)
        ref.flb_state_download(want)
    with flb.flb_create_ex(cfg) as ctx, flb.HostBuffer(ctx.flb_state_bytes()) as buf:
        assert buf.ptr % 64 == 0 and not buf.array.any()    # zeroed
        ctx.flb_set_populations(n0)
        ctx.flb_step(start)
        ctx.flb_state_download(buf.array)
        ctx.flb_step_host(buf.array, 1)
        ctx.flb_step_host(buf.array, 1)
        assert np.array_equal(buf.array, want)


def test_host_resident_stepping_of_one_batch_box(weights):
    shapes = [(16, 8, 8), (32, 8, 12)]
    cfgs = [flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 4, replica=r, store="f32", pattern="aa")
            for r, (nx, ny, nz) in enumerate(shapes)]
    n1 = state_of(weights, (12, 8, 32), 8)
    with flb.flb_create_ex(cfgs[1]) as one:
        one.flb_set_populations(n1)
        one.flb_step(1)
        want = one.flb_get_populations()
    with flb.flb_create_batch(cfgs) as ctx:
        ctx.flb_set_populations(n1, box=1)
        host = np.zeros(ctx.flb_state_bytes(box=1), np.uint8)
        ctx.flb_state_download(host, box=1)
        ctx.flb_step_host(host, 1, box=1)
        assert np.array_equal(ctx.flb_get_populations(box=1), want)
    with pytest.raises(flb.FlbError):
        with flb.flb_create_ex(flb.config(8, 8, 1, lattice="d2q9")) as d2:
            d2.flb_step_host(np.zeros(d2.flb_state_bytes(), np.uint8), 1)


@pytest.mark.parametrize("store,lattice", [("f32", "d3q19"), ("f64", "d3q19"), ("f16dev", "d3q19"), ("f32", "d2q9")])
@pytest.mark.parametrize("start", [2, 3])
def test_pattern_conversion_keeps_the_state_bitwise(store, lattice, start):
    rng = np.random.default_rng(start)
    if lattice == "d2q9":
        nx, ny, nz = 64, 24, 1
        a = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
        shape = (ny, nx)
    else:
        nx, ny, nz = 32, 8, 6
        a = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
        shape = (nz, ny, nx)
    n0 = a.reshape((-1,) + (1,) * len(shape)) * (1 + 0.02 * rng.standard_normal((len(a),) + shape))
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 7, store=store, pattern="aa", lattice=lattice)
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(start + 3)
        want = ref.flb_get_populations()
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_step(start)
        before = ctx.flb_get_populations()
        ctx.flb_set_pattern("ab")
        assert ctx.flb_get_pattern() == "ab"
        assert np.array_equal(ctx.flb_get_populations(), before)
        ctx.flb_step(2)
        ctx.flb_set_pattern("aa")
        assert ctx.flb_get_pattern() == "aa"
        ctx.flb_step(1)
        # the same arithmetic per site in both patterns: only where values are read and written differs
        assert np.abs(ctx.flb_get_populations() - want).max() <= (0 if store == "f64" else 1e-6)


def test_autotune_with_pattern_choice_restores_the_state(weights):
    nx, ny, nz = 64, 16, 8
    n0 = state_of(weights, (nz, ny, nx), 11)
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 2, store="f32", pattern="aa")
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(3)
        before = ref.flb_get_populations()
        ref.flb_step(4)
        want = ref.flb_get_populations()
    with flb.flb_create_ex(cfg) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_step(3)
        ctx.flb_autotune(2, pattern=True)
        assert ctx.flb_get_step() == 3
        assert ctx.flb_get_pattern() in ("ab", "aa")
        assert np.array_equal(ctx.flb_get_populations(), before)
        ctx.flb_step(4)
        assert np.abs(ctx.flb_get_populations() - want).max() <= 1e-6


def test_batched_statistics_equal_single_box_statistics(weights):
    """The two-launch statistics of a batch give every box bitwise the sums a
    context of that box alone gives (same blocks, same fixed reduction order);
    S(q) of an enabled box is unchanged by the batching (to the rounding of its
    atomic shell sums)."""
    shapes = [(16, 8, 8), (32, 12, 6), (64, 4, 4)]
    cfgs = [flb.config(nx, ny, nz, 1.0, 1e-4, 0.2 + 0.1 * r, 0.2, 0.0, 5, replica=r, store="f32", pattern="aa")
            for r, (nx, ny, nz) in enumerate(shapes)]
    with flb.flb_create_batch(cfgs) as ctx:
        ctx.flb_enable_structure_factor(box=1)
        ctx.flb_step(7)
        ctx.flb_stats_sample()
        ctx.flb_step(2)
        ctx.flb_stats_sample()
        got = [ctx.flb_mode_stats(box=b) for b in range(3)]
        S, cnt = ctx.flb_structure_factor(20, box=1)
    for b, cfg in enumerate(cfgs):
        with flb.flb_create_ex(cfg) as one:
            if b == 1:
                one.flb_enable_structure_factor()
            one.flb_step(7)
            one.flb_stats_sample()
            one.flb_step(2)
            one.flb_stats_sample()
            want = one.flb_mode_stats()
            for key in ("mode_m2", "u2", "momentum_last"):
                assert np.array_equal(got[b][key], want[key]), (b, key)
            assert got[b]["mass_last"] == want["mass_last"] and got[b]["nsamples"] == 2
            if b == 1:
                S1, cnt1 = one.flb_structure_factor(20)
                # the shell sums use atomic adds: equal up to the order of the additions
                assert np.allclose(S, S1, rtol=1e-12, atol=0) and np.array_equal(cnt, cnt1)


@pytest.mark.parametrize("store", ["f64", "f32", "f16dev", "bf16dev", "bf16sr"])
@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
def test_check_finite_counts_bad_populations(store, lattice):
    nx, ny, nz = (16, 8, 4) if lattice == "d3q19" else (16, 8, 1)
    q = 19 if lattice == "d3q19" else 9
    with flb.flb_create_ex(flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 1, store=store, lattice=lattice)) as ctx:
        ctx.flb_step(3)
        assert ctx.flb_check_finite() == 0
        n = ctx.flb_get_populations()
        n.reshape(q, -1)[5, 17] = np.nan
        n.reshape(q, -1)[q - 1, 3] = np.inf
        ctx.flb_set_populations(n)
        assert ctx.flb_check_finite() == 2
        with pytest.raises(flb.FlbError) as e:
            flb.lib().flb_box_check_finite(ctx.h, 0, None) and ctx._check(flb.lib().flb_box_check_finite(ctx.h, 0, None))
        assert e.value.code == flb.FLB_ENONFINITE


def test_tuning_cache_and_set_launch(tmp_path, weights):
    from paper_0707_1581_gb300 import tuning
    cfg = flb.config(64, 32, 16, 1.0, 1e-4, 0.3, 0.2, 0.0, 2, store="f32", pattern="aa")
    path = str(tmp_path / "tune.json")
    with flb.flb_create_ex(cfg) as a:
        r1 = tuning.autotune_cached(a, path, trials=1, pattern=True)
        assert not r1["cached"]
    with flb.flb_create_ex(cfg) as b:
        r2 = tuning.autotune_cached(b, path, trials=1, pattern=True)
        assert r2["cached"] and r2["launch"] == r1["launch"] and r2["pattern"] == r1["pattern"]
        assert list(b.flb_get_launch()) == r1["launch"] and b.flb_get_pattern() == r1["pattern"]
        with pytest.raises(flb.FlbError):
            b.flb_set_launch(4, 7, 1)            # not whole warps for 4 sites per thread
        b.flb_set_launch(1, 64, 4)
        assert b.flb_get_launch() == (1, 64, 4)
        n0 = state_of(weights, (16, 32, 64), 3)
        b.flb_set_populations(n0)
        b.flb_step(3)
        assert b.flb_check_finite() == 0


class _CountingTorchAllocator:
    """torch's caching allocator, recording every block the library takes."""

    def __init__(self, fail_after=None):
        import torch
        self.torch = torch
        self.live, self.allocs, self.frees, self.fail_after = {}, 0, 0, fail_after

    def alloc(self, nbytes, stream):
        if self.fail_after is not None and self.allocs >= self.fail_after:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(nbytes, self.torch.cuda.current_device(), stream)
        assert p % 256 == 0
        self.live[p] = nbytes
        self.allocs += 1
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "freed a block the allocator did not hand out"
        del self.live[ptr]
        self.frees += 1
        self.torch.cuda.caching_allocator_delete(ptr)


@pytest.fixture
def restore_allocator():
    yield
    flb.flb_set_device_allocator(None, None)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_device_allocator_hook_owns_every_context_buffer(weights, restore_allocator, pattern):
    import torch
    nx, ny, nz = 32, 16, 12
    n0 = state_of(weights, (nz, ny, nx), 9)
    cfg = flb.config(nx, ny, nz, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, store="f32", pattern=pattern)
    with flb.flb_create_ex(cfg) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(7)
        want = ref.flb_get_populations()
    A = _CountingTorchAllocator()
    flb.flb_set_device_allocator(A.alloc, A.free)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with flb.flb_create_ex(cfg) as ctx:
        assert torch.cuda.memory_allocated() - before >= ctx.flb_state_bytes()
        ctx.flb_set_populations(n0)                  # staging buffer
        ctx.flb_enable_structure_factor()            # FFT workspace
        launch = ctx.flb_get_launch()
        ctx.flb_autotune(1)                          # state copies, returned at the end
        ctx.flb_set_launch(*launch)                  # the reference's launch shape, for a bitwise comparison
        ctx.flb_step(3)
        ctx.flb_set_pattern("aa" if pattern == "ab" else "ab")   # second buffer taken or returned
        ctx.flb_step(4)
        assert np.array_equal(ctx.flb_get_populations(), want)
        assert A.allocs > 5 and A.live
    assert not A.live and A.frees == A.allocs
    flb.flb_set_device_allocator(None, None)
    with flb.flb_create_ex(cfg) as ctx:                  # back on cudaMalloc: the hook sees nothing
        ctx.flb_step(1)
    assert A.allocs == A.frees


def test_device_allocator_failure_is_reported_and_cleaned_up(restore_allocator):
    cfgs = [flb.config(16, 8, 8, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, replica=r, store="f32") for r in range(3)]
    for k in range(0, 9, 2):
        A = _CountingTorchAllocator(fail_after=k)
        flb.flb_set_device_allocator(A.alloc, A.free)
        with pytest.raises(flb.FlbError) as e:
            flb.flb_create_batch(cfgs)
        assert e.value.code == flb.FLB_ENOMEM
        assert not A.live and A.frees == A.allocs == k


@pytest.mark.parametrize("graph_steps", [0, 4, 10])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_automatic_statistics_samples_equal_manual_ones(weights, graph_steps, pattern):
    """stats_every = 6: flb_step samples after the steps that reach 6, 12, 18,
    ... whatever the graph length and however the calls split the steps; the
    accumulators equal manual samples at the same steps."""
    nx, ny, nz = 32, 8, 6
    n0 = state_of(weights, (nz, ny, nx), 4)
    base = dict(nx=nx, ny=ny, nz=nz, rho0=1.0, kT=1e-4, gamma_shear=0.3, gamma_bulk=0.2, gamma_ghost=0.0, seed=5,
                store="f32", pattern=pattern, graph_steps=graph_steps)
    with flb.flb_create_ex(flb.config(**base)) as ref:
        ref.flb_set_populations(n0)
        ref.flb_step(3)
        ref.flb_stats_reset()
        for t in range(3, 40):
            ref.flb_step(1)
            if (t + 1) % 6 == 0:
                ref.flb_stats_sample()
        want = ref.flb_mode_stats()
    with flb.flb_create_ex(flb.config(**base, stats_every=6)) as ctx:
        ctx.flb_set_populations(n0)
        ctx.flb_step(3)
        ctx.flb_stats_reset()
        for n in (5, 1, 13, 2, 13):       # 3 + 34 = 37 ... then 3 more
            ctx.flb_step(n)
        ctx.flb_step(3)
        assert ctx.flb_get_step() == 40
        got = ctx.flb_mode_stats()
    assert got["nsamples"] == want["nsamples"] == 6       # steps 6, 12, ..., 36
    assert np.array_equal(got["mode_m2"], want["mode_m2"])
    assert np.array_equal(got["u2"], want["u2"])
    assert got["mass_last"] == want["mass_last"]
