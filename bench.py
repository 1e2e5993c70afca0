"""Benchmark of the thermalized D3Q19 stream-collide (one JSON line on stdout).

Workload (default): a 512^3 periodic box, rho0 = 1, k_BT = 1e-4,
gamma_shear = 0.3, gamma_bulk = 0.2, gamma_ghost = 0, Kolmogorov force
F_x = 1e-5 sin(2 pi z / 512), Philox seed 3, AA in-place streaming, FP32
populations; the FP16-deviation storage of the same workload is measured
beside it.  One step = one time step of the whole box (one kernel launch).
The state (10.2 GB in FP32) is far larger than the 129 MB L2, so no flush is
needed between steps.

  value      MLUPS = sites * steps / device time of the K timed steps (CUDA
             events on the library's stream), max over ranks, summed over ranks
  e2e        the same metric through the C ABI with host buffers: every step
             uploads the state from pinned host memory, steps, and downloads it
  roofline   algorithmic bytes per launch (19 loads + 19 stores of the storage
             type per site) / mean launch time, against the measured HBM copy
             bandwidth; `traffic` is DRAM read+write per launch from ncu
  cpu_baseline  the FP64 oracle on this host's cores, on a 128^3 sample of
             the same workload
  variants   the same box in FP16 deviations; D2Q9 on 8192^2; the batched
             ensemble (64 replicas of 64^3 + 16 cubes of 32..128, CUDA graphs,
             autotuned) in FP32 and FP16 deviations, each with its own CUDA-event
             MLUPS, HBM roofline, clocks, and for the ensemble the worst
             equipartition ratio over every box from a sampled run outside the
             timed steps
  statistics one statistics sample of the 512^3 state (mode sums), and the same
             sample with the static structure factor S(q) added, timed alone

--impl reference times the oracle itself as the reference arm.
Multi-GPU (torchrun): each rank runs an independent replica box (weak
scaling; replicas only, no data exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "thermalized D3Q19 MLUPS at 1 GB300 and % of HBM roofline; FP32 vs FP16-deviation"
WORKLOAD = dict(L=512, rho0=1.0, kT=1e-4, gamma_shear=0.3, gamma_bulk=0.2, gamma_ghost=0.0, seed=3, force=1e-5)
STORE_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2, "bf16sr": 2}
D2Q9_EDGE = 8192          # the D2Q9 variant: an 8192^2 periodic box (67 M sites, 2.4 GB of FP32 state)
KERNEL_SOURCES = ["paper_0707_1581_gb300/csrc/d3q19.cuh", "paper_0707_1581_gb300/csrc/kernels.cuh",
                  "paper_0707_1581_gb300/csrc/step_impl.cuh"]


D2Q9_SOURCES = KERNEL_SOURCES[:1] + ["paper_0707_1581_gb300/csrc/d2q9.cuh"]


def kernel_hash(sources=None) -> str:
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def issue_peak(torch, sm_mhz: float | None) -> tuple[float, str]:
    """Issue-rate peak of the 16-bit formats' bound: the device's SM count x 4
    schedulers x 32 lanes x the median SM clock sampled while the kernel ran
    (one warp instruction per scheduler and cycle); without a clock sample, the
    maximum SM clock of MEASURED_PEAKS.json."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    src = "median SM clock sampled during the timed steps"
    if not sm_mhz:
        src = "maximum SM clock"
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                sm_mhz = float(json.load(f)["sm_max_mhz"])
        except (OSError, KeyError, ValueError):
            sm_mhz, src = 2070.0, "nominal maximum SM clock"
    return sms * 4 * 32 * sm_mhz * 1e6, f"{sms} SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz ({src})"


def ncu_record(store: str) -> dict | None:
    """The committed ncu record of the stream-collide kernel for a storage
    format ("d2q9_f32": the D2Q9 kernel), if it was taken on the current
    kernel sources."""
    path = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(store)
    except (OSError, ValueError):
        return None
    want = kernel_hash(D2Q9_SOURCES if store.startswith("d2q9") else None)
    if not rec or rec.get("kernel_hash") != want:
        return None
    return rec


def ensemble_traffic(store: str, pattern: str) -> float | None:
    """DRAM bytes per step of the batched ensemble (both launches of a step)
    from the committed capture, if it was taken on the current kernel sources
    with the same streaming pattern."""
    rec = ncu_record(f"ensemble_{store}")
    if rec is None or rec.get("pattern") != pattern:
        return None
    return rec["dram_bytes_per_step"]


def ncu_traffic(store: str) -> float | None:
    """DRAM bytes per launch at the benchmark's box size (per-site bytes of the
    256^3 capture times the sites of one launch)."""
    rec = ncu_record(store)
    if rec is None:
        return None
    per_site = rec["dram_bytes_per_launch"] / rec["sites"]
    return per_site * WORKLOAD["L"] ** 3


def d2_traffic(edge: int) -> float | None:
    rec = ncu_record("d2q9_f32")
    return None if rec is None else rec["dram_bytes_per_launch"] / rec["sites"] * edge * edge


def ncu_instr_per_site(store: str) -> float | None:
    rec = ncu_record(store)
    return None if rec is None else rec.get("lane_instr_per_site")


class NvmlReader:
    """Read-only NVML queries of one GPU through the driver's libnvidia-ml:
    SM clock, maximum SM clock and the clock-event reason bits.  open()
    returns None where NVML is missing."""

    CLOCK_SM = 1

    def __init__(self, lib, handle):
        self.lib, self.handle = lib, handle
        self._reasons = (getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
                         or getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None))

    @classmethod
    def open(cls, index: int, props=None):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            handle = ctypes.c_void_p()
            rc = 1
            if props is not None and hasattr(props, "pci_bus_id"):
                bus = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                            getattr(props, "pci_device_id", 0))
                rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(handle))
            if rc != 0:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(handle))
            return cls(lib, handle) if rc == 0 else None
        except (OSError, AttributeError):
            return None

    def _clock(self, fn) -> float | None:
        import ctypes
        v = ctypes.c_uint()
        return float(v.value) if fn(self.handle, self.CLOCK_SM, ctypes.byref(v)) == 0 else None

    def sm_mhz(self) -> float | None:
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def max_sm_mhz(self) -> float | None:
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self) -> int | None:
        import ctypes
        v = ctypes.c_ulonglong()
        if self._reasons is None or self._reasons(self.handle, ctypes.byref(v)) != 0:
            return None
        return int(v.value)


# NVML clock-event reason bits that the timing rules name
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                0x80: "hw_power_brake_slowdown"}


class ClockSampler:
    """SM clock and clock-event reasons of the timed GPU during the timed
    region: NVML read every 2 ms on a host thread (read-only queries), else
    nvidia-smi samples every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.002

    def __init__(self, index: int, reader=None, props=None):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.reader = reader if reader is not None else NvmlReader.open(index, props)
        self.samples: list[tuple[float, int]] = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None

    def _poll(self):
        while True:
            mhz, bits = self.reader.sm_mhz(), self.reader.reasons()
            if mhz is not None:
                self.samples.append((mhz, bits or 0))
            if self._stop.wait(self.PERIOD_S):
                break

    def __enter__(self):
        if self.reader is not None:
            self.max_mhz = self.reader.max_sm_mhz()
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.smi_reader = threading.Thread(target=self._read, daemon=True)
            self.smi_reader.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.smi_reader.join(timeout=2)

    def summary(self) -> dict:
        if self.reader is not None:
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": "nvml"}
            bits = 0
            for _, b in self.samples:
                bits |= b
            return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(name for bit, name in NVML_REASONS.items() if bits & bit),
                    "samples": len(self.samples), "source": "nvml"}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": "nvidia-smi"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


def clock_sampler(torch) -> ClockSampler:
    dev = torch.cuda.current_device()
    return ClockSampler(dev, props=torch.cuda.get_device_properties(dev))


def workload_config(store: str, L: int, lattice: str = "d3q19") -> dict:
    w = WORKLOAD
    nz = 1 if lattice == "d2q9" else L
    return dict(nx=L, ny=L, nz=nz, rho0=w["rho0"], kT=w["kT"], gamma_shear=w["gamma_shear"],
                gamma_bulk=w["gamma_bulk"], gamma_ghost=w["gamma_ghost"], seed=w["seed"], store=store,
                pattern="aa", force_amp=w["force"], lattice=lattice)


ENSEMBLE = dict(replicas=64, L=64, mixed=16, kT=1e-4, gamma_bulk=0.2, gamma_ghost=0.0, seed=4, graph_steps=20)


def ensemble_boxes() -> tuple[list[int], list[float]]:
    """The batched-ensemble workload: 64 replicas of 64^3 and 16 cubes of edges
    32 + 8 round(12 j / 15), j = 0..15 (28.26 M sites), each with its own
    gamma_shear ~ U[0, 0.8] drawn with seed 4."""
    from paper_0707_1581_gb300.inputs import mixed_edges, uniform_draws
    e = ENSEMBLE
    edges = [e["L"]] * e["replicas"] + mixed_edges(e["mixed"])
    return edges, [float(g) for g in uniform_draws(len(edges), e["seed"], 0.0, 0.8)]


def time_ensemble(store: str, steps: int, warmup: int, rank: int, torch, dist, cache: str) -> dict:
    """The ensemble as one batch (one kernel per step, graph_steps steps per
    CUDA graph), launch shape and streaming pattern from the autotuner's JSON
    cache (tuned and recorded on a miss).  Device time of `steps` steps by CUDA
    events on the library's stream; then, outside the timed region, 300 more
    steps and 30 statistics samples 10 steps apart give every box's mode and
    velocity ratios."""
    from paper_0707_1581_gb300 import flb, tuning
    e = ENSEMBLE
    edges, gammas = ensemble_boxes()
    stream = torch.cuda.Stream()
    nb = len(edges)
    cfgs = [flb.config(L, L, L, 1.0, e["kT"], g, e["gamma_bulk"], e["gamma_ghost"], e["seed"],
                       replica=rank * nb + r, store=store, pattern="aa", graph_steps=e["graph_steps"], stream=stream)
            for r, (L, g) in enumerate(zip(edges, gammas))]
    sites = sum(L ** 3 for L in edges)
    ctx = flb.flb_create_batch(cfgs)
    try:
        t0 = time.perf_counter()
        choice = tuning.autotune_cached(ctx, cache, trials=6, pattern=True)
        tune_s = time.perf_counter() - t0
        ctx.flb_step(max(warmup, e["graph_steps"]))
        ctx.flb_sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with clock_sampler(torch) as clocks:
            ev0.record(stream)
            ctx.flb_step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        total_ms = ev0.elapsed_time(ev1)
        # equipartition, outside the timed region
        ctx.flb_step(300)
        ctx.flb_stats_reset()
        for _ in range(30):
            ctx.flb_step(10)
            ctx.flb_stats_sample()
        worst_mode, worst_u2, nonfinite = 0.0, 0.0, 0
        for b, L in enumerate(edges):
            st = ctx.flb_mode_stats(box=b)
            # mass and momentum are conserved exactly: their site variance is short by 1/N
            expect = [1.0 - 1.0 / L ** 3] * 4 + [1.0] * 15
            worst_mode = max(worst_mode, max(abs(st["mode_ratio"][k] - expect[k]) for k in range(19)))
            worst_u2 = max(worst_u2, max(abs(st["u2_ratio"][a] - (1.0 - 1.0 / L ** 3)) for a in range(3)))
            nonfinite += st["nonfinite"]
        launch = ctx.flb_get_launch()
        pattern = ctx.flb_get_pattern()
    finally:
        ctx.close()
    return {"total_ms": total_ms, "sites": sites, "boxes": nb, "clocks": clocks.summary(), "launch": launch,
            "pattern": pattern, "tuning_cached": choice["cached"], "tuning_s": tune_s,
            "worst_mode_ratio_dev": worst_mode, "worst_u2_ratio_dev": worst_u2, "nonfinite": nonfinite}


def time_device(store: str, L: int, steps: int, warmup: int, replica: int, torch, dist, lattice="d3q19",
                pattern="aa", sk: bool = False, launch=None) -> dict:
    """Device-timed steps on resident inputs; per-launch CUDA events on the library's stream."""
    from paper_0707_1581_gb300 import flb
    stream = torch.cuda.Stream()
    cfg = flb.config(**{**workload_config(store, L, lattice), "pattern": pattern}, replica=replica, stream=stream)
    ctx = flb.flb_create_ex(cfg)
    try:
        if launch:
            ctx.flb_set_launch(*launch)
        ctx.flb_step(warmup)
        ctx.flb_sync()
        events = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with clock_sampler(torch) as clocks:
            events[0].record(stream)
            for k in range(steps):
                ctx.flb_step(1)
                events[k + 1].record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        per = [events[k].elapsed_time(events[k + 1]) for k in range(steps)]
        total_ms = events[0].elapsed_time(events[-1])
        launch = ctx.flb_get_launch()
        st = None
        stats_ms = sk_ms = None
        if replica == 0:
            # one statistics sample (outside the timed steps), timed on its own
            ctx.flb_stats_sample()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.flb_stats_sample()
            e1.record(stream)
            torch.cuda.synchronize()
            stats_ms = e0.elapsed_time(e1)
            st = ctx.flb_mode_stats()
            if sk:
                # the same sample with the static structure factor (density, 3-D
                # FFT, shell sums) added to it
                ctx.flb_enable_structure_factor()
                ctx.flb_stats_sample()
                e0.record(stream)
                ctx.flb_stats_sample()
                e1.record(stream)
                torch.cuda.synchronize()
                sk_ms = e0.elapsed_time(e1)
    finally:
        ctx.close()
    return {"total_ms": total_ms, "per_launch_ms": per, "clocks": clocks.summary(), "launch": launch,
            "stats_ms": stats_ms, "sk_ms": sk_ms,
            "nonfinite": None if st is None else st["nonfinite"]}


def f16_roofline(issued, ips, gbs, peak, ipeak, ipeak_source) -> dict:
    alu = {"bound": "alu", "achieved": None if issued is None else issued / 1e12, "peak": ipeak / 1e12,
           "unit": "T lane-instructions/s", "frac": None if issued is None else issued / ipeak,
           "lane_instr_per_site": ips, "peak_source": ipeak_source}
    hbm = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "traffic": ncu_traffic("f16dev"), "bytes_per_site": 76}
    near, far = (hbm, alu) if alu["frac"] is None or hbm["frac"] >= alu["frac"] else (alu, hbm)
    return {**near, "other": far}


def time_e2e(store: str, L: int, steps: int, warmup: int, replica: int, torch, dist) -> dict:
    """Through the C ABI with host buffers: every step, flb_box_step_host uploads
    the state from page-locked host memory (flb_host_alloc), advances one step
    and downloads it back (the copies of the two directions overlap each other
    and the kernel)."""
    from paper_0707_1581_gb300 import flb
    stream = torch.cuda.Stream()
    cfg = flb.config(**workload_config(store, L), replica=replica, stream=stream)
    ctx = flb.flb_create_ex(cfg)
    try:
        nbytes = ctx.flb_state_bytes()
        # page-locked huge-page memory; if the host cannot give it (many ranks on
        # one host), torch's pinned memory, else plain pageable memory: every
        # rank reaches the barriers below whatever it got
        kind = "flb_host_alloc"
        try:
            host = flb.HostBuffer(nbytes)
            ptr = host.ptr
        except flb.FlbError:
            try:
                host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
                kind = "torch pinned"
            except RuntimeError:
                host = torch.empty(nbytes, dtype=torch.uint8)
                kind = "pageable"
            ptr = host.data_ptr()
        lib = flb.lib()
        lib.flb_box_state_download(ctx.h, 0, ptr)
        for _ in range(warmup):
            ctx._check(lib.flb_box_step_host(ctx.h, 0, ptr, 1))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx._check(lib.flb_box_step_host(ctx.h, 0, ptr, 1))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            dist.barrier()
        if kind == "flb_host_alloc":
            host.close()
        del host
    finally:
        ctx.close()
    return {"seconds": dt, "bytes": 19 * L ** 3 * flb.STORE_BYTES[flb.STORE_NAMES[store]], "host_memory": kind}


def cpu_baseline(target_seconds: float = 12.0, L: int = 128) -> dict:
    """The oracle as it stands, on a periodic L^3 sample of the workload, enough
    steps for ~target_seconds of CPU work."""
    from oracle import oracle as O
    w = WORKLOAD
    p = O.make_params(L, L, L, rho0=w["rho0"], kT=w["kT"], gamma_shear=w["gamma_shear"],
                      gamma_bulk=w["gamma_bulk"], gamma_ghost=w["gamma_ghost"], seed=w["seed"],
                      force_amp=w["force"])
    n = O.rest_state(L, L, L)
    t0 = time.perf_counter()
    n = O.run(p, n, 0, 1)
    one = time.perf_counter() - t0
    steps = max(1, int(target_seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    O.run(p, n, 1, steps)
    dt = time.perf_counter() - t0
    return {"value": L ** 3 * steps / dt / 1e6, "unit": "MLUPS", "cores": O.threads(), "kind": "oracle",
            "sample": f"{L}^3 periodic box of the same parameters, {steps} steps after 1 untimed step, FP64"}


def arm_config(store: str, L: int, world: int) -> dict:
    """The workload both arms report (the reference arm times a sample of it)."""
    return {
        "workload": f"D3Q19 fluctuating LB, {L}^3 periodic, {store} populations, AA in-place, "
                    f"Kolmogorov force 1e-5, k_BT=1e-4, gamma_s=0.3, gamma_b=0.2, gamma_ghost=0, seed 3",
        "sites": L ** 3, "storage": store, "pattern": "AA",
        "l2": "state larger than L2 (no flush needed)",
        "parallelism": f"replicas x{world}",
    }


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    w = WORKLOAD
    L = 128
    p = O.make_params(L, L, L, rho0=w["rho0"], kT=w["kT"], gamma_shear=w["gamma_shear"],
                      gamma_bulk=w["gamma_bulk"], gamma_ghost=w["gamma_ghost"], seed=w["seed"],
                      force_amp=w["force"])
    n = O.rest_state(L, L, L)
    n = O.run(p, n, 0, args.warmup)
    t0 = time.perf_counter()
    n = O.run(p, n, args.warmup, args.steps)
    dt = time.perf_counter() - t0
    value = L ** 3 * args.steps / dt / 1e6
    sample = f"{L}^3 periodic sample of the {w['L']}^3 workload, FP64, one oracle step per bench step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**arm_config(args.store, args.size, args.gpus), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": O.threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="flb", choices=["flb", "reference"])
    ap.add_argument("--store", default="f32", choices=["f32", "f16dev", "bf16dev", "bf16sr", "f64"])
    ap.add_argument("--size", type=int, default=WORKLOAD["L"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--launch", default=None,
                    help="sites_per_thread,block_x,block_y of the main run (default: the library's choice)")
    ap.add_argument("--no-sk", action="store_true", help="skip the timing of the S(q) statistics sample")
    ap.add_argument("--tuning-cache", default=os.path.join(ROOT, "paper_0707_1581_gb300", "_build", "tuning.json"),
                    help="JSON cache of the autotuner's choices for the ensemble")
    ap.add_argument("--d2q9-edge", type=int, default=D2Q9_EDGE, help="edge of the D2Q9 variant's square box")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_0707_1581_gb300 import replicas
    dist = None
    info = replicas.rank_info()
    rank, world = info.rank, info.world
    torch.cuda.set_device(info.local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_0707_1581_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_0707_1581_gb300 import flb
    flb.use_torch_allocator()   # device memory of every context from torch's caching allocator
    L = args.size
    sites = L ** 3
    replica = replicas.replica_id(rank)

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, dist, device="cuda")

    launch = tuple(int(v) for v in args.launch.split(",")) if args.launch else None
    main_run = time_device(args.store, L, args.steps, args.warmup, replica, torch, dist, sk=not args.no_sk,
                           launch=launch)
    total_ms = max_over_ranks(main_run["total_ms"])
    value = replicas.aggregate_mlups(sites, args.steps, world, total_ms * 1e-3)
    mean_launch_ms = statistics.mean(main_run["per_launch_ms"])
    peak, peak_kind = measured_peaks()
    alg_bytes = 2 * 19 * STORE_BYTES[args.store] * sites
    achieved = alg_bytes / (mean_launch_ms * 1e-3) / 1e9
    traffic = ncu_traffic(args.store)

    variants = {}
    if not args.no_variants and args.store == "f32":
        v = time_device("f16dev", L, args.steps, args.warmup, replica, torch, dist)
        v_ms = max_over_ranks(v["total_ms"])
        v_mean = statistics.mean(v["per_launch_ms"])
        v_bytes = 2 * 19 * 2 * sites
        ips = ncu_instr_per_site("f16dev")
        issued = None if ips is None else ips * sites / (v_mean * 1e-3)
        variants["f16dev"] = {
            "value": replicas.aggregate_mlups(sites, args.steps, world, v_ms * 1e-3), "unit": "MLUPS",
            "storage": "FP16 deviation n - rho0 a_i, FP32 collide",
            # the 16-bit kernel sits between two rooflines, instruction issue and
            # HBM: the nearer one is reported as the bound, the other beside it
            "roofline": f16_roofline(issued, ips, v_bytes / (v_mean * 1e-3) / 1e9, peak,
                                     *issue_peak(torch, v["clocks"].get("sm_mhz"))),
            "clocks": v["clocks"],
        }
        # the D2Q9 lattice (Table I): 9 populations, 72 bytes per FP32 site update
        E = args.d2q9_edge
        v = time_device("f32", E, args.steps, args.warmup, replica, torch, dist, lattice="d2q9", pattern="ab")
        v_ms = max_over_ranks(v["total_ms"])
        v_mean = statistics.mean(v["per_launch_ms"])
        v_bytes = 2 * 9 * 4 * E * E
        variants["d2q9_f32"] = {
            "value": replicas.aggregate_mlups(E * E, args.steps, world, v_ms * 1e-3), "unit": "MLUPS",
            "workload": f"D2Q9 fluctuating LB, {E}^2 periodic, f32 populations, AB (two buffers), force F_x(y) 1e-5, "
                        "k_BT=1e-4, gamma_s=0.3, gamma_b=0.2, gamma_ghost=0, seed 3",
            "launch": {"block": list(v["launch"][1:])},
            "roofline": {"bound": "hbm", "achieved": v_bytes / (v_mean * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": v_bytes / (v_mean * 1e-3) / 1e9 / peak,
                         "traffic": d2_traffic(E), "bytes_per_site": 72, "kernel": "d2::k_stream_collide_vec"},
            "clocks": v["clocks"],
        }

    if not args.no_variants and not args.no_ensemble and args.store == "f32":
        # the batched ensemble (replicas and mixed boxes in one batch), FP32 and FP16 deviations
        for est in ("f32", "f16dev"):
            r = time_ensemble(est, args.steps, args.warmup, rank, torch, dist, args.tuning_cache)
            r_ms = max_over_ranks(r["total_ms"])
            per_step = r_ms / args.steps
            bps = 2 * 19 * STORE_BYTES[est]
            gbs = bps * r["sites"] / (per_step * 1e-3) / 1e9
            variants[f"ensemble_{est}"] = {
                "value": replicas.aggregate_mlups(r["sites"], args.steps, world, r_ms * 1e-3), "unit": "MLUPS",
                "workload": f"{r['boxes']} boxes in one batch: {ENSEMBLE['replicas']} replicas of "
                            f"{ENSEMBLE['L']}^3 + {ENSEMBLE['mixed']} cubes of 32..128, {r['sites']} sites, "
                            f"{est} populations, k_BT=1e-4, gamma_s ~ U[0,0.8] (seed 4), gamma_b=0.2, "
                            f"gamma_ghost=0, CUDA graphs of {ENSEMBLE['graph_steps']} steps",
                "ms_per_step": per_step,
                "launch": {"sites_per_thread": r["launch"][0], "block": list(r["launch"][1:]),
                           "pattern": r["pattern"], "from_tuning_cache": r["tuning_cached"],
                           "tuning_s": r["tuning_s"]},
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                             "traffic": ensemble_traffic(est, r["pattern"]), "bytes_per_site": bps,
                             "kernel": "k_stream_collide_batch",
                             "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"},
                "equipartition": {"worst_mode_ratio_abs_dev": r["worst_mode_ratio_dev"],
                                  "worst_u2_ratio_abs_dev": r["worst_u2_ratio_dev"], "nonfinite": r["nonfinite"],
                                  "how": "every box, all 19 modes (1 - 1/N expected for the conserved ones) and "
                                         "3 velocity components; 30 samples 10 steps apart after 300 more steps, "
                                         "outside the timed region"},
                "clocks": r["clocks"],
            }

    e2e = None
    if not args.no_e2e:
        r = time_e2e(args.store, L, args.e2e_steps, 3, replica, torch, dist)   # the first two calls set up copies
        secs = max_over_ranks(r["seconds"])
        e2e = {"value": replicas.aggregate_mlups(sites, args.e2e_steps, world, secs), "unit": "MLUPS",
               "h2d_bytes_per_step": r["bytes"], "d2h_bytes_per_step": r["bytes"],
               "steps": args.e2e_steps, "host_memory": r["host_memory"],
               "what": "per step: flb_box_step_host(1): the state uploaded from host memory (host_memory "
                       "says which kind), one step, downloaded back, the copies overlapped chunk by chunk"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    V, bx, by = main_run["launch"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.store != "f64" else "f64",
        "data": "synthetic",
        "config": {**arm_config(args.store, L, world), "launch": {"sites_per_thread": V, "block": [bx, by]}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                     "bytes_per_site": 2 * 19 * STORE_BYTES[args.store],
                     "mean_launch_ms": mean_launch_ms, "kernel": "k_stream_collide"},
        "clocks": main_run["clocks"],
        "gpu_launches": args.steps,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "variants": variants,
        "nonfinite": main_run["nonfinite"],
        # A10: one sample of the on-device statistics (mode sums, <u^2>, mass and
        # momentum in FP64 accumulators), outside the timed steps
        "statistics": None if main_run["stats_ms"] is None else {
            "sample_ms": main_run["stats_ms"],
            "read_GBs": 19 * STORE_BYTES[args.store] * sites / (main_run["stats_ms"] * 1e-3) / 1e9,
            # the same sample with S(q) (Sec. V) enabled; sk_sample_ms is the difference
            "with_sk_sample_ms": main_run["sk_ms"],
            "sk_sample_ms": None if main_run["sk_ms"] is None else main_run["sk_ms"] - main_run["stats_ms"]},
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
