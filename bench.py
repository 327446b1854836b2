#!/usr/bin/env python
"""Benchmark of exact all-pairs Kendall tau-b on one GB300 (and N GPUs as independent shards).

One step = the whole hot path over one gene-expression-shaped matrix (m=16384 variables x
n=128 samples, float32, synthetic): rank transform of every variable (K-a) + every one of the
134,209,536 pairs counted exactly (Knight merge path K-b or sign contraction K-c, chosen by the
library) + FP64 tau-b, stored as the packed FP32 triangle plus int32 S and n_3.

Prints ONE JSON line (rank 0). `value` is pairs/s with the input resident in HBM; `e2e` is the
same metric through the C ABI with host buffers (input H2D and every output D2H inside the timed
region). `--impl reference` times the CPU oracle (Knight, all host cores) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N = 16384, 128
METRIC = "tau-b pairs/s (m=16384,n=128) batched vs plain launch; query p50/p99 latency"
WORKLOAD = "gene-expression all-pairs tau-b, m=16384 x n=128 float32 (log-normal, 256 latent " \
           "factors, 10% quantised ties), packed FP32 tau + int32 S and n_3"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="auto", choices=["auto", "merge", "signgemm"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-query", action="store_true")
    ap.add_argument("--query-batches", type=int, default=2000,
                    help="batches per offered load in the serving measurement")
    ap.add_argument("--no-merge", action="store_true",
                    help="skip the merge-path (Knight) measurement")
    ap.add_argument("--no-perm", action="store_true",
                    help="skip the permutation-test measurement")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: every rank takes its static share of one matrix's pair "
                         "range (Sec. 4.4) instead of a matrix of its own")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout: float):
        t0 = time.monotonic()
        while self.proc is not None and not self.lines and time.monotonic() - t0 < timeout:
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlSampler:
    """SM clock and clock-event reasons read in-process through NVML (libnvidia-ml, public C API)
    every `period` seconds while the timed region runs: the region lasts milliseconds, shorter
    than the interval at which nvidia-smi prints, so this gives the samples under load."""

    # nvmlClocksEventReasons bits (nvml.h)
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown"}

    def __init__(self, dev, period: float = 0.002):
        import ctypes

        self.period = period
        self.sm, self.reasons, self.smax = [], set(), None
        self.stop_evt = threading.Event()
        self.t = None
        self.lib = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            import torch

            props = torch.cuda.get_device_properties(dev)
            bus = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0),
                                          getattr(props, "pci_bus_id", 0),
                                          getattr(props, "pci_device_id", 0))
            h, count = ctypes.c_void_p(), ctypes.c_uint()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                # one visible GPU: NVML's index 0 is that GPU
                if lib.nvmlDeviceGetCount_v2(ctypes.byref(count)) != 0 or count.value != 1 or \
                        lib.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    return
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.smax = float(mx.value)
            self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.h, self.lib, self.ct = h, lib, ctypes
        except (OSError, AttributeError, RuntimeError):
            self.lib = None

    def _run(self):
        ct, lib, h = self.ct, self.lib, self.h
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_evt.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ct.byref(mhz)) == 0:
                self.sm.append(float(mhz.value))
            if self.reason_fn(h, ct.byref(rs)) == 0:
                for bit, name in self.BITS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            self.stop_evt.wait(self.period)

    def start(self):
        if self.lib is not None:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()

    def stop(self) -> dict | None:
        if self.t is None:
            return None
        self.stop_evt.set()
        self.t.join(timeout=2)
        return {"sm_mhz": statistics.median(self.sm) if self.sm else None,
                "sm_max_mhz": self.smax, "reasons": sorted(self.reasons),
                "samples": len(self.sm)}


def _traffic(kernel: str):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu capture, or None
    when the kernel's source has changed since that capture (its SHA-256 is recorded beside the
    figure)."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))[kernel]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha256(src).hexdigest() != rec["sha256"]:
        return None
    return rec["dram_bytes_per_launch"]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


def _gemm_peak(f, n: int) -> float:
    """Best of 10 launches of f (an n^3 GEMM) in TFLOP/s (2 n^3 flops each)."""
    import torch

    for _ in range(3):
        f()
    best = float("inf")
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def tensor_peaks(dev) -> dict:
    """Dense low-precision tensor rates of this GPU, measured as MEASURED_PEAKS.json measures BF16:
    cuBLAS GEMMs (torch._scaled_mm, BF16 output) of 8192^3, best of 10 launches. FP8: e4m3 with
    unit tensor scales. FP4: e2m1 with one e4m3 scale per 16 elements (the FP4 tensor format that
    torch exposes; the contraction uses e2m1 with one power-of-two scale per 32 elements, the same
    FP4 MMA rate class). Taken before the timed region."""
    import torch

    n = 8192
    out = {"how": "torch._scaled_mm, 8192^3, best of 10 (burst), BF16 output"}
    a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
    one = torch.tensor(1.0, device=dev)
    out["fp8_tflops"] = _gemm_peak(
        lambda: torch._scaled_mm(a, b, one, one, out_dtype=torch.bfloat16), n)
    del a, b
    try:
        a4 = torch.randint(0, 256, (n, n // 2), device=dev, dtype=torch.uint8).view(
            torch.float4_e2m1fn_x2)
        b4 = torch.randint(0, 256, (n, n // 2), device=dev, dtype=torch.uint8).view(
            torch.float4_e2m1fn_x2)
        sa = torch.ones((n, n // 16), device=dev).to(torch.float8_e4m3fn)
        sb = torch.ones((n, n // 16), device=dev).to(torch.float8_e4m3fn)
        out["fp4_tflops"] = _gemm_peak(
            lambda: torch._scaled_mm(a4, b4.t(), sa, sb, out_dtype=torch.bfloat16), n)
        del a4, b4, sa, sb
    except (RuntimeError, AttributeError, TypeError) as e:  # FP4 GEMM not exposed by this torch
        out["fp4_error"] = str(e).splitlines()[0][:200]
    torch.cuda.empty_cache()
    return out


def _timed_oracle(Xd, threads: int, p_end: int):
    """Wall and process CPU seconds of one oracle run over the first p_end pairs."""
    import oracle

    c0, t0 = time.process_time(), time.perf_counter()
    oracle.allpairs(Xd, method="knight", threads=threads, p_begin=0, p_end=p_end)
    return time.perf_counter() - t0, time.process_time() - c0


def cpu_baseline(X, seconds: float):
    """The oracle as it stands (Knight per pair, Sec. 3.2; the requested pair range cut into
    equal contiguous slices, one per host core, Sec. 4.2-4.3) on the first pairs of the same
    matrix; returns pairs/s with the measured CPU time / wall time (cores actually busy)."""
    import numpy as np

    threads = os.cpu_count() or 1
    Xd = np.asarray(X, dtype=np.float64)
    probe = 20000
    dt, _ = _timed_oracle(Xd, threads, probe)
    P = M * (M - 1) // 2
    sample = int(min(P, max(probe, probe * seconds / max(dt, 1e-6))))
    dt, cpu = _timed_oracle(Xd, threads, sample)
    # the same oracle on one core, on a sample a quarter as long in time
    one = max(2000, int(sample / threads / 4))
    dt1, cpu1 = _timed_oracle(Xd, 1, one)
    return {"value": sample / dt, "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "cpu_time_over_wall": cpu / dt,
            "sample": f"first {sample} packed pairs (rows 0..) of the same m=16384 x n=128 matrix, "
                      f"Knight counting, {threads} threads, {dt:.1f} s wall, {cpu:.1f} s CPU",
            "single_core": {"value": one / dt1, "unit": "pairs/s", "cores": 1,
                            "cpu_time_over_wall": cpu1 / dt1,
                            "sample": f"first {one} packed pairs, {dt1:.1f} s"},
            "speedup_over_single_core": (sample / dt) / (one / dt1)}


def bench_batched(ktau, steps: int, warmup: int, fp4_tflops: float | None = None) -> dict:
    """Batched form on 1000 uneven datasets: one graph launch per step vs the plain launch
    (rank + all-pairs per dataset, one after another). The roofline of its contraction: the
    algorithmic 2 n_0 flops of every contraction pair over the summed contraction kernel time of
    one traced (serialised) run, against the FP4 tensor rate."""
    import torch

    from paper_1704_03767_gb300 import autotune
    from synthetic import batched_uneven

    mats = batched_uneven(1000, seed0=0)
    table = autotune.load()
    plans = autotune.batch_plans(table, mats) if table else [{"path": 0, "mapping": 0}] * len(mats)
    paths = [pl["path"] for pl in plans]
    dev = torch.device("cuda")
    descs, keep, outs = [], [], []
    for X, pl in zip(mats, plans):
        Xd = torch.from_numpy(X).to(dev)
        m = X.shape[0]
        P = m * (m - 1) // 2
        o = (torch.empty(P, dtype=torch.float32, device=dev),
             torch.empty(P, dtype=torch.int32, device=dev),
             torch.empty(P, dtype=torch.int32, device=dev))
        descs.append(ktau.batch_desc(Xd, None, o[0], o[1], o[2], 32, pl["path"], pl["mapping"]))
        keep.append(Xd)
        outs.append(o)
    B = ktau.Batch(descs, keepalive=keep)
    pairs = B.pairs()
    n_merge, n_sg = B.paths()
    st = torch.cuda.Stream()
    for _ in range(max(1, warmup)):
        B.graph_launch(st)
    B.check(st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        B.graph_launch(st)
    e1.record(st)
    st.synchronize()
    B.check(st)
    ms = e0.elapsed_time(e1) / steps
    # One traced run of the same work through the workspace form (ktau_allpairs_batched), whose
    # groups all run on the caller's stream one after another, so each launch's events time that
    # kernel alone (the plan's eight lanes would overlap them): the per-kernel split and the
    # contraction's time for its roofline.
    ws = torch.empty(ktau.ktau_workspace_size(descs), dtype=torch.uint8, device=dev)
    ktau.ktau_allpairs_batched(descs, ws, stream=st)  # warm-up of the one-stream form
    st.synchronize()
    ktau.ktau_trace_collect()
    ktau.ktau_trace_filter(None)
    ktau.ktau_trace_enable(True)
    ktau.ktau_allpairs_batched(descs, ws, stream=st)
    st.synchronize()
    ktau.ktau_trace_enable(False)
    tr = ktau.ktau_trace_collect()
    B.check(st)
    del ws
    per_kernel = {}
    for name, t in tr:
        per_kernel[name] = per_kernel.get(name, 0.0) + t
    serial_ms = sum(per_kernel.values())
    flops = 0.0
    for X, pth in zip(mats, paths):
        if pth == 2 or (pth == 0 and X.shape[1] <= 2048):
            m, n = X.shape
            flops += 2.0 * (m * (m - 1) // 2) * (n * (n - 1) // 2)
    c_ms = per_kernel.get("contract_kernel", 0.0)
    roof = None
    if c_ms > 0 and fp4_tflops:
        ach = flops / (c_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": fp4_tflops, "unit": "TFLOP/s",
                "frac": ach / fp4_tflops, "contraction_ms_serialised": c_ms,
                "peak_source": "of measured: the FP4 GEMM rate of the main line's roofline"}
    # plain launch of the same work, dataset by dataset, with the same per-dataset paths
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    p0.record(cur)
    for Xd, o, pl in zip(keep, outs, plans):
        R = ktau.ktau_rank_prepare(Xd)
        ktau.ktau_allpairs(R, 0, R.pairs, None, o[0], o[1], o[2], 32,
                           {"path": pl["path"], "mapping": pl["mapping"]})
        R.free_on(cur)
    p1.record(cur)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    B.free()
    return {"workload": "1000 matrices, m log-uniform [16,1024], n log-uniform [20,2000], "
                        "5% duplicated entries; FP32 tau + int32 S, n_3",
            "datasets": len(mats), "pairs": pairs, "paths": {"merge": n_merge, "signgemm": n_sg},
            "autotuned": bool(table), "ms_per_step": ms, "value": pairs / (ms / 1e3),
            "unit": "pairs/s", "plain_launch": {"ms": plain_ms, "value": pairs / (plain_ms / 1e3)},
            "speedup_vs_plain": plain_ms / ms, "roofline": roof,
            "kernels_serialised_ms": per_kernel, "kernels_serialised_total_ms": serial_ms}


def bench_merge(ktau, clocks_mhz: float | None) -> dict:
    """The Knight merge path (K-b) on its own: the long heavy-tie profiles it is the path for
    (2048 x 4096 int32, values 0..63, int64 counts + FP64 tau) and the bench matrix, each timed
    by the library's per-kernel CUDA events. Roof: one compare-and-count merge step per int32
    lane per clock (152 SMs x 128 lanes at the sampled SM clock)."""
    import torch

    from synthetic import gene_expression, heavy_ties_ordinal

    dev = torch.device("cuda")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f = (clocks_mhz or 2070.0) * 1e6
    peak = sms * 128 * f / 1e9
    out = {}
    cases = (("heavy_ties_2048x4096_int32", heavy_ties_ordinal(2048, 4096, seed=0), 64),
             ("gene_expression_16384x128", gene_expression(M, N, seed=0), 32))
    for name, X, bits in cases:
        m, n = X.shape
        P = m * (m - 1) // 2
        Xd = torch.from_numpy(X).to(dev)
        R = ktau.ktau_rank_prepare(Xd)
        cdt = torch.int64 if bits == 64 else torch.int32
        S = torch.empty(P, dtype=cdt, device=dev)
        n3 = torch.empty(P, dtype=cdt, device=dev)
        t64 = torch.empty(P, dtype=torch.float64, device=dev) if bits == 64 else None
        t32 = None if bits == 64 else torch.empty(P, dtype=torch.float32, device=dev)
        opts = {"path": 1}
        ktau.ktau_allpairs(R, 0, P, t64, t32, S, n3, bits, opts)  # warm-up
        torch.cuda.synchronize()
        reps = 2
        ktau.ktau_trace_collect()
        ktau.ktau_trace_enable(True)
        for _ in range(reps):
            ktau.ktau_allpairs(R, 0, P, t64, t32, S, n3, bits, opts)
        torch.cuda.synchronize()
        ktau.ktau_trace_enable(False)
        tr = ktau.ktau_trace_collect()
        ktau.ktau_device_status()
        ms = sum(t for k, t in tr if k.startswith("merge")) / reps
        lg = max(1, (n - 1).bit_length())
        steps = n * lg  # Step 3 compare-and-count steps per pair
        ach = P * steps / (ms / 1e3) / 1e9
        out[name] = {"m": m, "n": n, "pairs": P, "count_bits": bits, "kernel_ms": ms,
                     "pairs_per_s": P / (ms / 1e3), "ns_per_pair": ms * 1e6 / P,
                     "sample_comparisons_per_s": P * (n * (n - 1) // 2) / (ms / 1e3),
                     "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                                  "unit": "G merge-steps/s vs int32 lane-ops/s", "frac": ach / peak,
                                  "steps_per_pair": steps}}
        if bits == 64:
            # the same outputs on the library's default path (for these rows: the sign
            # contraction, n_3 from the contraction of the magnitudes)
            path = ktau.ktau_allpairs_path(R)
            ktau.ktau_allpairs(R, 0, P, t64, t32, S, n3, bits, None)  # builds the operands
            torch.cuda.synchronize()
            ktau.ktau_trace_collect()
            ktau.ktau_trace_enable(True)
            ktau.ktau_allpairs(R, 0, P, t64, t32, S, n3, bits, None)
            torch.cuda.synchronize()
            ktau.ktau_trace_enable(False)
            dms = sum(t for _, t in ktau.ktau_trace_collect())
            ktau.ktau_device_status()
            out[name]["default_path"] = {"path": {1: "merge", 2: "signgemm"}.get(path, path),
                                         "kernel_ms": dms, "ns_per_pair": dms * 1e6 / P,
                                         "pairs_per_s": P / (dms / 1e3)}
        R.free()
        del Xd, S, n3, t64, t32
        torch.cuda.empty_cache()
    return out


def bench_bits(ktau) -> dict:
    """The bit-parallel dominance count (KTAU_PATH_BITS) on the bench matrix: its pair kernel's
    time from the library's CUDA events (masks built by the first, untimed call)."""
    import torch

    from synthetic import gene_expression

    X = gene_expression(M, N, seed=0)
    P = M * (M - 1) // 2
    Xd = torch.from_numpy(X).cuda()
    R = ktau.ktau_rank_prepare(Xd)
    S = torch.empty(P, dtype=torch.int32, device="cuda")
    n3 = torch.empty(P, dtype=torch.int32, device="cuda")
    t32 = torch.empty(P, dtype=torch.float32, device="cuda")
    opts = {"path": ktau.KTAU_PATH_BITS}
    ktau.ktau_allpairs(R, 0, P, None, t32, S, n3, 32, opts)
    torch.cuda.synchronize()
    ktau.ktau_trace_collect()
    ktau.ktau_trace_filter("bits_pairs_kernel")
    ktau.ktau_trace_enable(True)
    for _ in range(2):
        ktau.ktau_allpairs(R, 0, P, None, t32, S, n3, 32, opts)
    torch.cuda.synchronize()
    ktau.ktau_trace_enable(False)
    ktau.ktau_trace_filter(None)
    ms = sum(t for _, t in ktau.ktau_trace_collect()) / 2
    R.free()
    return {"workload": "gene-expression 16384 x 128", "kernel_ms": ms, "ns_per_pair": ms * 1e6 / P,
            "pairs_per_s": P / (ms / 1e3)}


def bench_permutation(ktau, Xd, P: int, B: int = 8) -> dict:
    """Permutation test on the bench matrix: B relabellings, each a full pass over the
    134,209,536 pairs (relabelled ranks, their sign expansion, pair contraction counting
    exceedances)."""
    import torch

    from synthetic import permutations

    R = ktau.ktau_rank_prepare(Xd)
    S = torch.empty(P, dtype=torch.int32, device=Xd.device)
    ktau.ktau_allpairs(R, 0, P, None, None, S, None, 32)
    exc = torch.zeros(P, dtype=torch.uint32, device=Xd.device)
    perms = torch.from_numpy(permutations(B, N, seed=5)).to(Xd.device)
    ktau.ktau_permutation_exceed(R, perms[:1], S, exc)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ktau.ktau_permutation_exceed(R, perms, S, exc)  # returns when finished
    dt = time.perf_counter() - t0
    R.free()
    return {"permutations": B, "seconds": dt, "ms_per_permutation": dt * 1e3 / B,
            "pair_permutations_per_s": P * B / dt}


def bench_query(ktau, batches_per_load: int) -> dict:
    """Serving: resident 65536 x 256 database, batches of 1..512 profiles (log-uniform),
    exact tau-b against every row + top-100; closed-loop capacity, then Poisson streams at 0.3,
    0.6 and 0.9 of it with p50 / p99 latency, and at 0.1 (a batch nearly always finds the server
    idle: the server's own overhead over the plain launch)."""
    import time

    from paper_1704_03767_gb300.serving import QueryServer, percentile, run_open_loop
    from synthetic import gene_expression, query_batch_sizes

    D = gene_expression(65536, 256, seed=0)
    sizes = query_batch_sizes(batches_per_load, max_batch=512, seed=2)
    pool = gene_expression(512, 256, seed=1)
    batches = [pool[:b] for b in sizes]
    srv = QueryServer(D, k=100, slots=4)
    for q in batches[:8]:  # warm-up
        srv.submit(q).done.wait()
    # Like a latency-bound service after start-up: the objects made so far (this process has
    # built the other measurements' inputs) move to the collector's permanent generation, so that
    # no full collection pass over them stalls the server threads in the middle of a measurement.
    import gc

    gc.collect()
    gc.freeze()
    t0 = time.perf_counter()
    reqs = [srv.submit(q) for q in batches]
    for r in reqs:
        r.done.wait()
    dt = time.perf_counter() - t0
    profiles = sum(sizes)
    cap_batches = len(batches) / dt
    out = {"workload": "resident DB 65536 x 256 (gene-expression recipe), batches of "
                       "round(exp(U[0, ln 512])) profiles, top-100 by |tau|",
           "closed_loop": {"batches_per_s": cap_batches, "queries_per_s": profiles / dt,
                           "pairs_per_s": profiles * 65536 / dt},
           "open_loop": []}
    # Plain launch of the same batches, one after another on one stream (no continuous
    # batching): H2D, rank, query + top-k, D2H, synchronise.
    import numpy as np
    import torch

    import paper_1704_03767_gb300 as kb

    lat_plain = []
    tq = time.perf_counter()
    for q in batches:
        ts = time.perf_counter()
        qd = torch.from_numpy(q).cuda()
        Rq = kb.ktau_rank_prepare(qd)
        b = q.shape[0]
        Sq = torch.empty((b, 65536), dtype=torch.int32, device="cuda")
        idx = torch.empty((b, 100), dtype=torch.int32, device="cuda")
        tk = torch.empty((b, 100), dtype=torch.float64, device="cuda")
        kb.ktau_query(srv.db, Rq, None, Sq, None, 32, 100, idx, tk)
        idx.cpu(), tk.cpu()
        Rq.free()
        lat_plain.append((time.perf_counter() - ts) * 1e3)
    dtp = time.perf_counter() - tq
    out["plain_launch"] = {"batches_per_s": len(batches) / dtp, "queries_per_s": profiles / dtp,
                           "p50_ms": percentile(lat_plain, 50), "p99_ms": percentile(lat_plain, 99)}
    out["speedup_vs_plain"] = (profiles / dt) / (profiles / dtp)
    for load in (0.1, 0.3, 0.6, 0.9):
        t1 = time.perf_counter()
        rs = run_open_loop(srv, batches, rate_per_s=load * cap_batches)
        wall = time.perf_counter() - t1
        lat = [r.latency * 1e3 for r in rs if r.error is None]
        out["open_loop"].append({"offered_load": load, "batches": len(rs),
                                 "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                                 "queries_per_s": sum(r.queries.shape[0] for r in rs) / wall,
                                 "errors": sum(r.error is not None for r in rs)})
    srv.stop()
    gc.unfreeze()
    return out


def run_reference(args):
    """Reference arm: the CPU oracle (Knight, Sec. 3.2) as it stands, on every host core, over a
    bounded sample of the bench matrix per step (about 4 s of wall time each)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    from synthetic import gene_expression

    X = gene_expression(M, N, seed=0).astype(np.float64)
    threads = os.cpu_count() or 1
    probe = 20000
    dt, _ = _timed_oracle(X, threads, probe)
    sample = int(max(probe, 4.0 * probe / max(dt, 1e-9)))
    for _ in range(args.warmup):
        _timed_oracle(X, threads, sample)
    wall = cpu = 0.0
    for _ in range(args.steps):
        w, c = _timed_oracle(X, threads, sample)
        wall, cpu = wall + w, cpu + c
    value = sample * args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_pairs_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                         "cpu_time_over_wall": cpu / wall,
                         "sample": f"first {sample} packed pairs per step, Knight counting, "
                                   f"{threads} threads"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1704_03767_gb300 as ktau
    from synthetic import gene_expression

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    path = {"auto": 0, "merge": 1, "signgemm": 2}[args.path]
    opts = {"path": path}

    # Weak scaling (default): every rank runs its own independent matrix (seed = rank). Strong
    # scaling (--shard): one matrix, every rank its static contiguous share of the pair range
    # (Sec. 4.4). No collective on the data path either way.
    from paper_1704_03767_gb300.sharding import shard_range

    X = gene_expression(M, N, seed=0 if args.shard else rank)
    P = M * (M - 1) // 2
    lo, hi = shard_range(P, world, rank) if args.shard else (0, P)
    Xd = torch.from_numpy(X).to(dev)
    tau32 = torch.empty(hi - lo, dtype=torch.float32, device=dev)
    S = torch.empty(hi - lo, dtype=torch.int32, device=dev)
    n3 = torch.empty(hi - lo, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    tpeaks = tensor_peaks(dev)
    R0 = ktau.ktau_rank_prepare(Xd, stream)
    path_id = ktau.ktau_allpairs_path(R0, opts)
    R0.free()
    path_used = {1: "merge", 2: "signgemm"}[path_id]

    def step():
        # The statistics (NaN flag, tie counts) are read by ktau_allpairs, so the sign expansion
        # is enqueued while the rank transform finishes.
        R = ktau.ktau_rank_prepare_async(Xd, stream)
        if path_id == 2:
            ktau.ktau_prepare_signs(R, stream)  # sign expansion + tie lists (part of the step)
        ktau.ktau_allpairs(R, lo, hi, None, tau32, S, n3, 32, opts, stream)
        return R

    for _ in range(args.warmup):
        step().free()
    torch.cuda.synchronize()
    ktau.ktau_device_status(stream)

    sampler = ClockSampler(local)
    nvml = NvmlSampler(dev)
    sampler.start()
    sampler.wait_first(5.0)  # nvidia-smi is printing before the timed region starts
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    nvml.start()
    total_ms = 0.0
    ktau.ktau_trace_collect()
    # CUDA events on the launching stream around the dominant kernel only: every traced launch
    # adds two event records to the step, so the full per-kernel breakdown is taken from extra
    # steps after the timed region.
    dominant = "contract_kernel" if path_id == 2 else "merge_pairs_kernel"
    ktau.ktau_trace_filter(dominant)
    ktau.ktau_trace_enable(True)
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between steps (256 MB write), outside the timed events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R = step()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        R.free()
    nv = nvml.stop()
    clocks = sampler.stop()
    if nv is not None and nv["samples"]:
        # In-process samples inside the timed region; nvidia-smi's around it (reasons merged).
        clocks = {"sm_mhz": nv["sm_mhz"], "sm_max_mhz": nv["sm_max_mhz"] or clocks["sm_max_mhz"],
                  "reasons": sorted(set(nv["reasons"]) | set(clocks["reasons"])),
                  "samples": nv["samples"], "source": "NVML every 2 ms inside the timed region",
                  "nvidia_smi": clocks}
    ktau.ktau_trace_enable(False)
    dom = [ms for name, ms in ktau.ktau_trace_collect() if name == dominant]
    ktau.ktau_device_status(stream)
    # per-kernel breakdown: three more steps with every launch traced (not part of the timing)
    ktau.ktau_trace_filter(None)
    ktau.ktau_trace_enable(True)
    for _ in range(3):
        flush.zero_()
        step().free()
    torch.cuda.synchronize()
    ktau.ktau_trace_enable(False)
    trace = ktau.ktau_trace_collect()
    per_kernel = {}
    for name, ms in trace:
        c, t = per_kernel.get(name, (0, 0.0))
        per_kernel[name] = (c + 1, t + ms)
    kernels = {k: {"launches": c, "avg_ms": t / c, "share": t / max(1e-9, sum(
        x[1] for x in per_kernel.values()))} for k, (c, t) in per_kernel.items()}
    dominant_ms = sum(dom) / max(1, len(dom))  # inside the timed region
    if dist:
        from paper_1704_03767_gb300.sharding import max_over_ranks

        total_ms = max_over_ranks(total_ms, device=dev)  # whole-job time = slowest rank
        dist.barrier()
    ms_per_step = total_ms / args.steps
    # whole-job pairs per second: every rank's own matrix (weak) or the one shared matrix (strong)
    value = (P if args.shard else P * world) * args.steps / (total_ms / 1e3)

    # Roofline of the dominant kernel (the pair kernel).
    peaks = _peaks()
    roof = None
    if path_used == "merge":
        # Algorithmic work: n * ceil(log2 n) compare-and-count merge steps per pair (Step 3).
        steps_per_pair = N * 7
        kern_avg_ms = dominant_ms
        achieved = (hi - lo) * steps_per_pair / (kern_avg_ms / 1e3) / 1e9
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        f = (clocks.get("sm_mhz") or 1455.0) * 1e6
        peak = sms * 128 * f / 1e9  # int32 lane-ops per second at the sampled clock
        roof = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Gop/s (merge steps vs int32 lane-ops)", "frac": achieved / peak,
                "traffic": None, "kernel": "merge_pairs_kernel",
                "kernel_ms": kern_avg_ms}
    else:
        # Algorithmic work of the contraction: n_0 multiply-adds (2 flops) per pair. Its
        # operands are FP4 e2m1 (block-scaled MMA), so the tensor roof is the FP4 GEMM rate
        # measured on this GPU (the FP8 rate x 3, the nominal FP4/FP8 ratio, when torch exposes
        # no FP4 GEMM). The HBM view: the
        # stored outputs (12 bytes per pair) and the operands read once.
        flops = 2.0 * (hi - lo) * (N * (N - 1) // 2)
        kern_avg_ms = dominant_ms
        achieved = flops / (kern_avg_ms / 1e3) / 1e12
        bf16 = (peaks or {}).get("bf16_tflops", 1899.7)
        if "fp4_tflops" in tpeaks:
            peak, src = tpeaks["fp4_tflops"], "FP4 e2m1 cuBLAS GEMM on this GPU (" + tpeaks["how"] + ")"
        else:
            peak, src = 3.0 * tpeaks["fp8_tflops"], "FP8 cuBLAS GEMM on this GPU x 3 (nominal ratio)"
        alg_bytes = 12.0 * (hi - lo) + M * ((N * (N - 1) // 2 + 255) // 256 * 128)
        hbm = (peaks or {}).get("hbm_gbs", 6779.7)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": _traffic("contract2_kernel"),
                "peak_source": "of measured: " + src + "; the kernel's operands are FP4 e2m1",
                "frac_vs_fp8": achieved / tpeaks["fp8_tflops"],
                "fp8_tflops": tpeaks["fp8_tflops"],
                "hbm_view": {"algorithmic_bytes": alg_bytes,
                             "achieved_gbs": alg_bytes / (kern_avg_ms / 1e3) / 1e9, "peak_gbs": hbm,
                             "frac": alg_bytes / (kern_avg_ms / 1e3) / 1e9 / hbm},
                "kernel": "contract2_kernel<1, MX, 0> (2-CTA tcgen05 kind::mxf4 pair)",
                "kernel_ms": kern_avg_ms}

    # tau-a (Sec. 2, no tie correction) on the same workload: the whole step without n_3.
    taua = None
    if world == 1:
        opts_a = dict(opts, statistic=1)
        for _ in range(2):
            R = ktau.ktau_rank_prepare(Xd, stream)
            ktau.ktau_allpairs(R, 0, P, None, tau32, S, None, 32, opts_a, stream)
            R.free()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a0.record(stream)
            R = ktau.ktau_rank_prepare_async(Xd, stream)
            if path_id == 2:
                ktau.ktau_prepare_signs(R, stream)
            ktau.ktau_allpairs(R, 0, P, None, tau32, S, None, 32, opts_a, stream)
            a1.record(stream)
            torch.cuda.synchronize()
            a_ms += a0.elapsed_time(a1)
            R.free()
        ktau.ktau_device_status(stream)
        taua = {"outputs": "FP32 tau-a + int32 S (no n_3)", "ms_per_step": a_ms / args.steps,
                "pairs_per_s": P * args.steps / (a_ms / 1e3)}

    e2e = None
    if not args.no_e2e:
        # End to end through the C ABI with host buffers: the input goes host -> device, and the
        # outputs come back in passes whose copies overlap the next pass (ktau_allpairs_host).
        Xh = torch.from_numpy(X).pin_memory()
        out_h = [torch.empty(hi - lo, dtype=t.dtype).pin_memory() for t in (tau32, S, n3)]
        h2d = Xh.numel() * 4
        d2h = sum(t.numel() * t.element_size() for t in out_h)

        def e2e_step():
            R = ktau.ktau_rank_prepare_host(Xh, stream)  # H2D copy inside the library call
            ktau.ktau_allpairs_host(R, lo, hi, None, out_h[0], out_h[1], out_h[2], 32, opts, 0,
                                    stream)
            R.free()

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if dist:
            from paper_1704_03767_gb300.sharding import max_over_ranks

            e2e_s = max_over_ranks(e2e_s, device=dev)
        e2e = {"value": (P if args.shard else P * world) * args.steps / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "ktau_rank_prepare_host (pinned host input) + ktau_allpairs_host (pinned "
                      "host outputs, passes with overlapped D2H)"}

    batched = None
    if not args.no_batched and world == 1:
        batched = bench_batched(ktau, max(3, args.steps // 2), args.warmup,
                                tpeaks.get("fp4_tflops", 3.0 * tpeaks["fp8_tflops"]))
    query = None
    if not args.no_query and world == 1:
        query = bench_query(ktau, args.query_batches)
    perm = None
    if not args.no_perm and world == 1 and path_id == 2:
        perm = bench_permutation(ktau, Xd, P)
    merge = None
    if not args.no_merge and world == 1:
        merge = bench_merge(ktau, clocks.get("sm_mhz"))
        merge["bits_path"] = bench_bits(ktau)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(X, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "pairs": P, "path": path_used,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": (f"{world} static shards of one matrix's pair range"
                                   if args.shard else
                                   f"{world} independent shards (one matrix per GPU)")},
        "gpu_launches": round(len(trace) / 3 * args.steps),  # library kernels per step x steps
        "kernels": kernels,
        "kernels_source": "CUDA events around every library launch in 3 steps after the timed "
                          "region; the roofline's kernel time is from events around that kernel "
                          "inside the timed region",
        "clocks": clocks, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "sample_comparisons_per_s": value * (N * (N - 1) // 2),
        "batched": batched, "query": query, "merge_path": merge, "tau_a": taua,
        "permutation_test": perm,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
