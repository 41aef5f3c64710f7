#!/usr/bin/env python3
"""Benchmark of the all-sky seedless-clustering scorer on one B300.

One step = one pass of the whole hot path over one batch: draw T templates,
rasterise, gather, phase-rotate, sum, normalise (Eq. 7) and select the k
loudest.  Workload: the realistic single map (500 time columns x 1600
frequency bins of 0.5 Hz from 40 Hz, per-frequency power-law sigma, one
injected chirp), T = 5e6 templates, tau uniform in +-10 ms, k = 1024.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the reference arm of this project) on a bounded sample of the same workload.
Under torchrun each rank scores its own 5e6-template range of the same map
(weak scaling, no data-path collective); rank 0 merges the k-records.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "track-pixels/s and tracks/s per ft-map on 1 B300; batched/FP16 vs plain FP32; % roofline"
WORKLOAD = "realistic"
BYTES_PER_TRACK_PIXEL = 8     # one complex FP32 pixel (the per-frequency weight table is not counted)
SMEM_BYTES_PER_CLK_PER_SM = 128


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU model (GB/s) from MEASURED_PEAKS.json beside
    this script, else None."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP16 and batched variant measurements")
    ap.add_argument("--batch-maps", type=int, default=256, help="maps in the batched variant (0: skip it)")
    ap.add_argument("--batch-tracks", type=int, default=1_000_000, help="templates per map in the batched variant")
    ap.add_argument("--tracks", type=int, default=0,
                    help="profiling aid: templates per GPU other than the workload's 5e6 (reported in config)")
    ap.add_argument("--cpu-sample", type=int, default=400000,
                    help="templates per oracle chunk (CPU baseline: chunks until ~10 s; reference arm: one per step)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class _NvmlCtypes:
    """The few read-only NVML calls the sampler needs, through the driver's
    libnvidia-ml.so.1, for hosts without the pynvml module."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        self._ok(self.lib.nvmlInit_v2())

    def _ok(self, rc):
        if rc != 0:
            raise RuntimeError(f"NVML error {rc}")

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        h = self.C.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), self.C.byref(h)))
        return h

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.C.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.C.c_uint(i), self.C.byref(h)))
        return h

    def _clock(self, fn, h, kind):
        v = self.C.c_uint()
        self._ok(fn(h, self.C.c_int(kind), self.C.byref(v)))
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h, kind)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h, kind)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.C.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.C.byref(v)))
        return v.value


class ClockSampler:
    """SM clock and throttle-reason samples (NVML reads, every ~2 ms) while the
    timed region runs.  Read-only: no clock or power setting is touched."""

    REASONS = [("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap")]

    def __init__(self, torch_device):
        self.dev = torch_device
        self.samples = []
        self.max_mhz = None
        self.err = None
        self._stop = threading.Event()

    def _handle(self, nv):
        import torch
        p = torch.cuda.get_device_properties(self.dev)
        bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        try:
            return nv.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            return nv.nvmlDeviceGetHandleByIndex(0)

    def __enter__(self):
        try:
            try:
                import pynvml as nv
                nv.nvmlInit()
            except ImportError:
                nv = _NvmlCtypes()
            self.nv = nv
            self.h = self._handle(nv)
            self.max_mhz = nv.nvmlDeviceGetMaxClockInfo(self.h, nv.NVML_CLOCK_SM)
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        except Exception as e:  # no NVML: report no samples
            self.err = repr(e)
            self.nv = None
        return self

    def _run(self):
        nv = self.nv
        while not self._stop.is_set():
            try:
                mhz = nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM)
                rs = nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                self.samples.append((mhz, rs))
            except Exception as e:
                self.err = repr(e)
                return
            time.sleep(0.002)

    def __exit__(self, *a):
        self._stop.set()
        if self.nv:
            self.t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "error": self.err}
        reasons = set()
        for _, rs in self.samples:
            for name, attr in self.REASONS:
                if rs & getattr(self.nv, attr):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "sm_min_mhz": min(m for m, _ in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "NVML, every ~2 ms during the timed region"}


def kernel_source_hash():
    """Hash of the sources that define the slab scoring kernel."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1401_8060_b300", "csrc")
    for f in ("stk_internal.cuh", "stk_pixel.cuh", "stk_score.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the scoring kernel from the committed ncu summary,
    or None when the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "score_staged_realistic_traffic.txt")
    if not os.path.exists(p):
        return None, None
    kv = {}
    for line in open(p):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = (t.strip() for t in line.split("=", 1))
            kv[k] = v
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return None, kv.get("kernel_source_hash")
    return int(kv["dram_bytes_per_launch"]), kv.get("kernel_source_hash")


def cpu_baseline(fm, w, chunk, seconds=10.0, check=None):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    consecutive chunks of templates from index 0 until about `seconds` of
    wall time have passed (or the workload is exhausted).

    check: optional {"n": n, "hits": {name: hits}}; after the timed part (not in
    the rate), the oracle also scores templates 0 .. n - 1 with each one's
    comparison scale sum_j |z_j| / sqrt(W), and the templates of each hit list,
    so the GPU's SNRs can be stated against it.  Returns (baseline, oracle SNRs
    or None)."""
    import oracle
    om = oracle.OracleMap.from_ftmap(fm)
    cores = os.cpu_count() or 1
    done = 0
    t0 = time.perf_counter()
    while done < w["n_tracks"] and time.perf_counter() - t0 < seconds:
        n = min(chunk, w["n_tracks"] - done)
        om.score_range(w["seed"], done, n, w["tau_max"], nthreads=cores)
        done += n
    dt = time.perf_counter() - t0
    px = done * fm.n_t
    base = {"value": px / dt, "unit": "track-pixels/s", "tracks_per_s": done / dt, "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"templates 0..{done - 1} of the {w['n_tracks']}-template realistic workload "
                      f"({px:.3g} track-pixels; chunks of {chunk} until ~{seconds:g} s), FP64, all host threads"}
    if not check:
        return base, None
    snr, sc = om.score_range_scale(w["seed"], 0, check["n"], w["tau_max"], nthreads=cores)
    top = {name: om.score_explicit(np.array([list(v) for v in h["f"]], np.uint32), h["tau"])
           for name, h in check["hits"].items()}
    return base, {"snr": snr, "scale": sc, "top": top}


def oracle_errors(gpu_sample, hits, orc, name):
    """SNR error of the GPU against the FP64 oracle: over the sample, |dSNR| in units
    of the template's scale sum_j |z_j| / sqrt(W) (the parity bound is 1e-5 of it);
    over the k hits, plain relative error."""
    d = np.abs(np.asarray(gpu_sample, np.float64) - orc["snr"]) / orc["scale"]
    t = np.abs(hits["snr"] - orc["top"][name]) / np.abs(orc["top"][name])
    return {"sample_templates": int(d.size), "sample_max_over_scale": float(d.max()),
            "sample_rms_over_scale": float(np.sqrt(np.mean(d * d))),
            "topk_max_rel": float(t.max()), "topk_rms_rel": float(np.sqrt(np.mean(t * t))),
            "scale": "sum_j |z_j| / sqrt(W) per template; top-k: |SNR_gpu - SNR_oracle| / |SNR_oracle|"}


def data_path_roofline(bytes_per_unit, units, ms, peak, kernel, note):
    """Algorithmic bytes over the shared-memory / L1 data path (128 B/clk/SM)."""
    achieved = bytes_per_unit * units / (ms / 1e3) / 1e9
    return {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel, "kernel_ms": ms, "bytes_per_unit": bytes_per_unit, "units": units,
            "note": note}


WORKLOAD_TEXT = ("realistic 500x1600 map (0.5 Hz bins from 40 Hz), per-frequency power-law sigma, "
                 "one injected chirp; 5e6 Philox templates per GPU, tau in +-10 ms, k=1024")


def workload_config(fm, n_tracks, k, world, profiling_tracks=False):
    """The config object both arms print (the driver compares the arms on it)."""
    return {"workload": WORKLOAD_TEXT, "n_t": fm.n_t, "n_f": fm.n_f, "n_tracks_per_gpu": n_tracks, "k": k,
            "reduced_for_profiling": bool(profiling_tracks), "l2": "flushed between steps (256 MB write)",
            "parallelism": f"template ranges x{world}"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_1401_8060_b300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    fm = synth.realistic_map()
    import oracle
    om = oracle.OracleMap.from_ftmap(fm)
    cores = os.cpu_count() or 1
    n = args.cpu_sample
    for _ in range(args.warmup):
        om.score_range(w["seed"], 0, min(n, 2000), w["tau_max"], nthreads=cores)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        om.score_range(w["seed"], s * n, n, w["tau_max"], nthreads=cores)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    value = n * fm.n_t / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "track-pixels/s",
            "tracks_per_s": n / dt, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(fm, w["n_tracks"], w["k"], world),
            "cpu_baseline": {"value": value, "unit": "track-pixels/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} templates per step of the realistic workload (consecutive "
                                       "ranges), FP64 oracle; the L2 flush does not apply on the host"},
            "e2e": {"value": value, "unit": "track-pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1401_8060_b300 as stk
    from paper_1401_8060_b300 import _lib, build, search, synth

    torch.cuda.set_device(local)             # before the process group: NCCL binds the current device
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    build.build()

    w = synth.WORKLOADS[WORKLOAD]
    fm = synth.realistic_map()
    T, K = (args.tracks or w["n_tracks"]), w["k"]
    stream = torch.cuda.current_stream()
    ctx = stk.Context(local, stream)
    y_dev, s_dev = torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda()
    m = ctx.load_map(y_dev, s_dev, fm.f_min, fm.df)
    # map pack (row a1, once per map, outside the track-pixel rate): stk_update_map from device
    # buffers is the pack kernel alone (y and sigma read, packed records and weights written)
    for _ in range(3):
        ctx.update_map(m, y_dev, s_dev)
    torch.cuda.synchronize()
    pk0, pk1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pk0.record(stream)
    for _ in range(20):                     # back to back: the GPU time per pack unless enqueueing is slower
        ctx.update_map(m, y_dev, s_dev)
    pk1.record(stream)
    torch.cuda.synchronize()
    pack_ms = pk0.elapsed_time(pk1) / 20
    pack_bytes = fm.y.nbytes + fm.sigma.nbytes + fm.n_t * fm.n_f * 8 + fm.n_f * 4
    offset = rank * T                       # each rank: its own T templates
    ctx.set_tracks(T, w["seed"], offset, w["tau_max"])
    out = torch.zeros(K * 40, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 126 MB L2

    ctx.set_profiling(True)
    for _ in range(max(args.warmup, 3)):
        ctx.score(m, K, out=out)
    ctx.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    score_ms, select_ms, order_ms, launches = [], [], [], 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.zero_()                    # evict the map from L2 between steps
            ev[s][0].record(stream)
            ctx.score(m, K, out=out)
            ev[s][1].record(stream)
            t = ctx.last_timings()           # library events around its kernels (same stream)
            score_ms.append(t["score_ms"])
            select_ms.append(t["select_ms"])
            order_ms.append(t["order_ms"])
            launches += t["launches"]
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    hits = out.cpu().numpy().view(stk.HIT_DTYPE)
    plan = ctx.last_plan()

    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 2032.0
    peak = SMEM_BYTES_PER_CLK_PER_SM * n_sm * sm_mhz * 1e6 / 1e9
    ACC_N = 100_000                          # templates whose SNRs are checked against the oracle
    acc_gpu = {}

    # the same workload scored in template-index order (no coherent-order pre-pass)
    variants = {}
    if not args.no_variants:
        ctx.set_option(_lib.STK_OPT_ORDER, 0)
        outi = torch.zeros(K * 40, dtype=torch.uint8, device="cuda")
        for _ in range(max(args.warmup, 3)):
            ctx.score(m, K, out=outi)
        evi = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        ki = []
        torch.cuda.synchronize()
        for s_ in range(5):
            flush.zero_()
            evi[s_][0].record(stream)
            ctx.score(m, K, out=outi)
            evi[s_][1].record(stream)
            ki.append(ctx.last_timings()["score_ms"])
        torch.cuda.synchronize()
        ctx.set_option(_lib.STK_OPT_ORDER, 1)
        msi = sum(a.elapsed_time(b_) for a, b_ in evi) / 5
        hi = outi.cpu().numpy().view(stk.HIT_DTYPE)
        variants["index_order"] = {
            "ms_per_step": msi, "kernel_ms": sum(ki) / len(ki), "speedup_of_coherent_order": msi / ms,
            "topk_identical": bool(np.array_equal(hi["index"], hits["index"]) and
                                   np.array_equal(hi["snr"], hits["snr"])),
            "roofline": data_path_roofline(BYTES_PER_TRACK_PIXEL, T * fm.n_t, sum(ki) / len(ki), peak,
                                           "score_staged_kernel", "8 B per track-pixel, template-index order")}

    # FP16 pixel storage on the same workload (4-byte records), same timing rules
    if not args.no_variants:
        ctx.set_profiling(True)
        m16 = ctx.load_map(torch.from_numpy(fm.y).cuda(), torch.from_numpy(fm.sigma).cuda(), fm.f_min, fm.df,
                           fp16=True)
        out16 = torch.zeros(K * 40, dtype=torch.uint8, device="cuda")
        for _ in range(max(args.warmup, 3)):
            ctx.score(m16, K, out=out16)
        ev16 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        k16 = []
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()
            ev16[s][0].record(stream)
            ctx.score(m16, K, out=out16)
            ev16[s][1].record(stream)
            k16.append(ctx.last_timings()["score_ms"])
        torch.cuda.synchronize()
        ms16 = sum(a.elapsed_time(b) for a, b in ev16) / args.steps
        h16 = out16.cpu().numpy().view(stk.HIT_DTYPE)
        common = np.intersect1d(h16["index"], hits["index"])
        s32 = dict(zip(hits["index"].tolist(), hits["snr"].tolist()))
        s16 = dict(zip(h16["index"].tolist(), h16["snr"].tolist()))
        rel = [abs(s16[i] - s32[i]) / abs(s32[i]) for i in common.tolist()]
        variants["fp16"] = {
            "value": T * fm.n_t / (ms16 / 1e3), "unit": "track-pixels/s", "ms_per_step": ms16,
            "kernel_ms": sum(k16) / len(k16), "speedup_vs_fp32": ms / ms16,
            "topk_overlap_with_fp32": len(common) / K,
            "max_rel_snr_diff_vs_fp32_on_common_topk": max(rel) if rel else None,
            "storage": "4 B/pixel: FP16 |y|/sigma (per-frequency scaling) + Q0.16 phase; FP32 sums",
            "roofline": data_path_roofline(4, T * fm.n_t, sum(k16) / len(k16), peak, "score_staged_kernel",
                                           "4 B per track-pixel (the FP16 record)")}
        # SNRs of templates 0 .. ACC_N - 1 in both precisions (checked against the oracle below)
        ctx.set_profiling(False)
        ctx.set_tracks(ACC_N, w["seed"], 0, w["tau_max"])
        acc_gpu["fp32"] = ctx.score_all(m).cpu().numpy()
        acc_gpu["fp16"] = ctx.score_all(m16).cpu().numpy()
        acc_gpu["hits16"] = h16
        ctx.set_tracks(T, w["seed"], offset, w["tau_max"])
        ctx.set_profiling(True)
        m16.close()

    # general templates (random start / middle / end times, duration >= 25 columns = 100 s)
    if not args.no_variants:
        Tg, tmin_g = 1_000_000, 25
        ctx.set_template_shape(True, tmin_g)
        ctx.set_tracks(Tg, w["seed"], 0, w["tau_max"])
        outg = torch.zeros(K * 40, dtype=torch.uint8, device="cuda")
        for _ in range(max(args.warmup, 3)):
            ctx.score(m, K, out=outg)
        ctx.sync()
        evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        kg = []
        for s_ in range(3):
            flush.zero_()
            evg[s_][0].record(stream)
            ctx.score(m, K, out=outg)
            evg[s_][1].record(stream)
            kg.append(ctx.last_timings()["score_ms"])
        torch.cuda.synchronize()
        msg = sum(a.elapsed_time(b_) for a, b_ in evg) / 3
        M_ = fm.n_t - 1
        pxg = Tg * ((tmin_g + M_) / 2 + 1)            # expected pixels: duration uniform on [t_min, M]
        variants["general_templates"] = {
            "value": pxg / (msg / 1e3), "unit": "track-pixels/s (expected pixels)", "ms_per_step": msg,
            "kernel_ms": sum(kg) / len(kg), "templates": Tg, "t_min_columns": tmin_g,
            "rasteriser": "FP32 estimate of the curve's frequency, exact integer test within a proven error "
                          "margin of a rounding boundary; one thread per template, L2 gathers",
            "roofline": data_path_roofline(BYTES_PER_TRACK_PIXEL, pxg, sum(kg) / len(kg), peak,
                                           "score_general_kernel", "8 B per expected track-pixel; the gathers "
                                           "come from L2 through the L1 data path")}
        ctx.set_template_shape(False)
        ctx.set_tracks(T, w["seed"], offset, w["tau_max"])

    # refinement of the k loudest: 50 gradient-ascent steps on the interpolated statistic
    if not args.no_variants:
        ctx.set_profiling(False)
        f3r = torch.tensor(np.array([list(v) for v in hits["f"]]), dtype=torch.float32, device="cuda")
        taur = torch.tensor(hits["tau"], dtype=torch.float32, device="cuda")
        stk.refine(ctx, m, f3r, taur, w["tau_max"], steps=2)          # warm-up
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        f_new, tau_new, hist = stk.refine(ctx, m, f3r, taur, w["tau_max"], steps=50)
        r1.record(stream)
        torch.cuda.synchronize()
        d_after = ctx.score_explicit(m, torch.round(f_new).to(torch.int32), tau_new.to(torch.float64)).cpu().numpy()
        # discrete follow-up: climb the discrete statistic from the start and from the
        # rounded refined templates; the scorer's SNR picks, so no template loses
        f_start = np.array([list(v) for v in hits["f"]], dtype=np.int64)
        ctx.polish(m, f_start, hits["tau"], w["tau_max"], alt_f3=f_new, alt_tau=tau_new, moves=8)   # warm-up
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        _, _, snr_p, which_p = ctx.polish(m, f_start, hits["tau"], w["tau_max"], alt_f3=f_new, alt_tau=tau_new,
                                          moves=8)
        p1.record(stream)
        torch.cuda.synchronize()
        snr_p, which_p = snr_p.cpu().numpy(), which_p.cpu().numpy()
        gain = snr_p - hits["snr"]
        variants["refine"] = {
            "templates": int(K), "steps": 50, "ms": r0.elapsed_time(r1),
            "interp_snr_mean_before": float(hist[0].mean()), "interp_snr_mean_after": float(hist[-1].mean()),
            "frac_improved": float((hist[-1] > hist[0]).float().mean()),
            "discrete_snr_mean_before": float(np.mean(hits["snr"])),
            "discrete_snr_mean_after_rounding": float(np.mean(d_after)),
            "kernels": "stk_refine: one launch runs all 50 steps, each the interpolated SNR, its gradient and the "
                       "Adam step (32-128 threads per template, chosen by count; position and phase in fixed point)",
            "roofline": data_path_roofline(16, float(K) * fm.n_t * 50, r0.elapsed_time(r1), peak, "refine_kernel",
                                           "16 B per template-column per step (the two FP32 records that "
                                           "interpolation reads); gathers from L2 through the L1 data path"),
            "polish": {
                "ms": p0.elapsed_time(p1), "moves": 8,
                "discrete_snr_mean_after": float(np.mean(snr_p)),
                "discrete_gain_mean": float(np.mean(gain)), "discrete_gain_min": float(np.min(gain)),
                "frac_improved": float(np.mean(gain > 0)),
                "kept": {"start": int(np.sum(which_p == 0)), "polished_start": int(np.sum(which_p == 1)),
                         "polished_refined": int(np.sum(which_p == 2))},
                "kernel": "stk_polish: one block per template, six warps climbing the discrete statistic from the "
                          "start and six from the refined template (Newton on the delay at fixed pixels; the six "
                          "+-1 bin moves of a round one per warp); the scorer's own SNR picks among start, "
                          "polished start and polished refined template"}}
        ctx.set_profiling(True)

    # 256 ragged maps in one persistent launch vs 256 sequential single-map launches
    if not args.no_variants and args.batch_maps > 0:
        bmaps = synth.batched_maps(args.batch_maps)
        ctx.set_profiling(False)
        dm = [ctx.load_map(torch.from_numpy(f.y).cuda(), torch.from_numpy(f.sigma).cuda(), f.f_min, f.df)
              for f in bmaps]
        nb, Tb, kb = len(dm), args.batch_tracks, 16
        seeds = [1000 + i for i in range(nb)]
        batch = stk.Batch(ctx, dm, [Tb] * nb, seeds, [0] * nb, w["tau_max"])
        t0 = time.perf_counter()
        cfg = batch.tune(kb)
        tune_s = time.perf_counter() - t0
        outb = torch.zeros(nb * kb * 40, dtype=torch.uint8, device="cuda")
        for _ in range(max(args.warmup, 3)):
            batch.score(kb, out=outb)
        ctx.sync()
        steps_b = max(1, min(args.steps, 5))
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps_b)]
        for s_ in range(steps_b):
            flush.zero_()
            evb[s_][0].record(stream)
            batch.score(kb, out=outb)
            evb[s_][1].record(stream)
        torch.cuda.synchronize()
        ctx.sync()
        msb = sum(a.elapsed_time(b_) for a, b_ in evb) / steps_b
        # the same work as nb separate single-map scoring calls
        outs = torch.zeros(kb * 40, dtype=torch.uint8, device="cuda")
        seq_ms = []
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            for i, m_ in enumerate(dm):
                ctx.set_tracks(Tb, seeds[i], 0, w["tau_max"])
                ctx.score(m_, kb, out=outs)
            e1.record(stream)
            torch.cuda.synchronize()
            seq_ms.append(e0.elapsed_time(e1))
        ctx.sync()
        pxb = float(sum(f.n_t for f in bmaps)) * Tb
        hb = outb.cpu().numpy().view(stk.HIT_DTYPE).reshape(nb, kb)
        inj = [i for i, f in enumerate(bmaps) if f.injections]
        variants["batched"] = {
            "value": pxb / (msb / 1e3), "unit": "track-pixels/s", "ms_per_step": msb,
            "maps": nb, "templates_per_map": Tb, "k": kb, "track_pixels": pxb,
            "sequential_ms": min(seq_ms), "speedup_vs_sequential": min(seq_ms) / msb,
            "tuned": cfg, "tune_s": tune_s, "launch": "one persistent kernel + merge, CUDA graph replay",
            "loudest_snr_injected_maps_median": float(np.median(hb[inj, 0]["snr"])) if inj else None,
            "loudest_snr_noise_maps_median": float(np.median(np.delete(hb[:, 0]["snr"], inj))),
            "config": "n_t ~ U{100..1000}, n_f ~ U{200..2000}, 0.5 Hz from 40 Hz, sigma0 ~ U(0.5, 2), "
                      "10% injected (SNR 10-30)",
            "roofline": data_path_roofline(BYTES_PER_TRACK_PIXEL, pxb, msb, peak, "score_batch_kernel",
                                           "8 B per track-pixel; time of the whole graph (order pass, "
                                           "persistent scoring kernel, merge)")}
        batch.close()
        # the same maps with little work per map (2e4 templates): launch overheads and
        # per-map fill dominate the sequential calls; one batched launch avoids them
        Ts = 20_000
        bsm = stk.Batch(ctx, dm, [Ts] * nb, seeds, [0] * nb, w["tau_max"])
        bsm.tune(kb)
        for _ in range(3):
            bsm.score(kb, out=outb)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        bsm.score(kb, out=outb)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_small = e0.elapsed_time(e1)
        bsm.close()
        seq_small = []
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            for i, m_ in enumerate(dm):
                ctx.set_tracks(Ts, seeds[i], 0, w["tau_max"])
                ctx.score(m_, kb, out=outs)
            e1.record(stream)
            torch.cuda.synchronize()
            seq_small.append(e0.elapsed_time(e1))
        ctx.sync()
        variants["batched"]["small_work"] = {
            "templates_per_map": Ts, "ms_per_step": ms_small, "sequential_ms": min(seq_small),
            "speedup_vs_sequential": min(seq_small) / ms_small,
            "value": float(sum(f.n_t for f in bmaps)) * Ts / (ms_small / 1e3), "unit": "track-pixels/s"}
        for m_ in dm:
            m_.close()
        ctx.set_tracks(T, w["seed"], offset, w["tau_max"])

    # end to end through the public API with host buffers (pinned), copies timed.
    # Pipelined: two maps alternate, so step i's host -> device copy and pack (copy
    # stream) overlap step i-1's scoring (compute stream); every step still copies
    # its map in and its k records out inside the timed region.  The serial form
    # (waiting for each step's records) is reported beside it.
    e2e = None
    if not args.no_e2e:
        y_pin = torch.from_numpy(fm.y).pin_memory()
        s_pin = torch.from_numpy(fm.sigma).pin_memory()
        ctx.set_profiling(False)
        mm = ctx.load_map(y_pin, s_pin, fm.f_min, fm.df)
        for _ in range(2):
            ctx.update_map(mm, y_pin, s_pin)
            ctx.score(mm, K)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.update_map(mm, y_pin, s_pin)   # this step's map: host -> device copy + pack
            h = ctx.score(mm, K)               # host output: waits for the result
        dt_serial = (time.perf_counter() - t0) / args.steps
        if world > 1:                          # the slowest rank's time, as for the device-timed value
            tt = torch.tensor([dt_serial], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt_serial = float(tt.item())
        mm.close()
        assert np.array_equal(h["index"], hits["index"]) or world > 1

        # two maps alternate: map j's next data is copied in (and packed) on a copy
        # stream once its previous scoring has finished, while the other map scores
        copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
        ectx = stk.Context(local)              # follows the current torch stream
        ectx.set_tracks(T, w["seed"], offset, w["tau_max"])
        pm = [ectx.load_map(y_pin, s_pin, fm.f_min, fm.df) for _ in range(2)]
        out_dev = [torch.zeros(K * 40, dtype=torch.uint8, device="cuda") for _ in range(2)]
        out_host = [torch.zeros(K * 40, dtype=torch.uint8).pin_memory() for _ in range(2)]

        def pipelined(n):
            scored = [None, None]
            for i in range(n):
                j = i % 2
                if scored[j] is not None:
                    scored[j].synchronize()        # map j and its records buffer are free again
                with torch.cuda.stream(copy_s):
                    ectx.update_map(pm[j], y_pin, s_pin)
                    copied = torch.cuda.Event()
                    copied.record(copy_s)
                with torch.cuda.stream(comp_s):
                    comp_s.wait_event(copied)
                    ectx.score(pm[j], K, out=out_dev[j])
                    out_host[j].copy_(out_dev[j], non_blocking=True)
                    scored[j] = torch.cuda.Event()
                    scored[j].record(comp_s)
            torch.cuda.synchronize()

        pipelined(4)
        if world > 1:
            dist.barrier()
        e2e_steps = max(args.steps, 30)       # a longer run: the pipeline's fill and drain amortised
        t0 = time.perf_counter()
        pipelined(e2e_steps)
        dt = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            tt = torch.tensor([dt], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt = float(tt.item())
        ectx.sync()
        hp = out_host[(e2e_steps - 1) % 2].numpy().view(stk.HIT_DTYPE)
        assert np.array_equal(hp["index"], hits["index"]) or world > 1
        ectx.close()
        e2e = {"value": world * T * fm.n_t / dt, "unit": "track-pixels/s", "ms_per_step": dt * 1e3,
               "steps": e2e_steps,
               "h2d_bytes_per_step": int(fm.y.nbytes + fm.sigma.nbytes), "d2h_bytes_per_step": int(K * 40),
               "api": "per step: stk_update_map(STK_HOST_PTR, pinned; copy stream) + stk_score(device out; "
                      "compute stream) + copy of the k records to pinned host memory; two maps alternate, so "
                      "step i's copy-in overlaps step i-1's scoring",
               "serial": {"value": world * T * fm.n_t / dt_serial, "ms_per_step": dt_serial * 1e3,
                          "api": "stk_update_map(STK_HOST_PTR) + stk_score(STK_OUT_HOST), waiting every step"}}

    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, hits.tobytes())
        if rank == 0:
            hits = search.merge_hits([np.frombuffer(b, dtype=stk.HIT_DTYPE) for b in gathered], K)

    if rank == 0:
        px = world * T * fm.n_t
        value = px / (ms / 1e3)
        score_avg = sum(score_ms) / len(score_ms)
        achieved = T * fm.n_t * BYTES_PER_TRACK_PIXEL / (score_avg / 1e3) / 1e9
        traffic, src_hash = profiled_traffic()
        line = {
            "metric": METRIC, "value": value, "unit": "track-pixels/s",
            "tracks_per_s": world * T / (ms / 1e3),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "dtype_notes": "FP32 pixel records (|z| and the angle of z), FP32 sums; the normalisation S / sqrt(W) "
                           "in FP32 with the square root and the division rounded to nearest (within 2^-23 of the "
                           "quotient of the FP32 sums); SNRs widened to FP64 in the hits; FP64 only in each "
                           "template's delay and its exact fixed-point phase constants",
            "notes": "synthetic maps shaped like the paper's searches stand in for its LIGO data",
            "config": workload_config(fm, T, K, world, args.tracks),
            "roofline": {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "score_staged_kernel", "kernel_ms": score_avg,
                         "bytes_per_track_pixel": BYTES_PER_TRACK_PIXEL,
                         "peak_source": f"derived: {SMEM_BYTES_PER_CLK_PER_SM} B/clk/SM x {n_sm} SMs x "
                                        f"{sm_mhz:.0f} MHz (median SM clock sampled in the timed region)"},
            "select_ms": sum(select_ms) / len(select_ms), "order_ms": sum(order_ms) / len(order_ms),
            "map_pack": {"ms": pack_ms, "bytes": pack_bytes, "GB_per_s": pack_bytes / pack_ms / 1e6,
                         "frac_of_hbm": pack_bytes / pack_ms / 1e6 / hbm_peak_gbs() if hbm_peak_gbs() else None,
                         "api": "stk_update_map from device buffers (a weight-table clear and the pack kernel: "
                                "y, sigma in; FP32 records and the weight table out), 20 back to back, per call; "
                                "not in the track-pixel rate"},
            "clocks": clocks,
            "gpu_launches": launches,
            "wall_s_timed_region": wall,
            "plan": plan,
            "top1": {"snr": float(hits["snr"][0]), "index": int(hits["index"][0]),
                     "f": [int(v) for v in hits["f"][0]], "tau": float(hits["tau"][0])},
        }
        if e2e:
            line["e2e"] = e2e
        if variants:
            line["variants"] = variants
        if world == 1 and not args.no_cpu_baseline:
            check = None
            if "fp32" in acc_gpu:
                check = {"n": ACC_N, "hits": {"fp32": hits, "fp16": acc_gpu["hits16"]}}
            line["cpu_baseline"], orc = cpu_baseline(fm, w, args.cpu_sample, check=check)
            if orc is not None:
                line["accuracy_vs_oracle"] = oracle_errors(acc_gpu["fp32"], hits, orc, "fp32")
                variants["fp16"]["err_vs_oracle"] = oracle_errors(acc_gpu["fp16"], acc_gpu["hits16"], orc, "fp16")
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
