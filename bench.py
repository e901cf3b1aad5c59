#!/usr/bin/env python3
"""CMIF benchmark: shift*angle evaluations per second at 1024^2, K = 16.

One step = one full CMIF map of the 1024 x 1024, K_A = K_B = 16 workload
(synthetic Voronoi labels, all-ones masks, planted shift; the paper's image
datasets are not available): the level-set transforms of A and B, the 256
pair correlations, the rounding + entropy epilogue and the gamma-gated peak of
Alg. 1.  One evaluation = the MI at one displacement of the full linear range
(2047 x 2047 = 4,190,209 per map, one angle).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one replica per GPU (the path has no exchange step;
each rank computes its own map) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CMIF shift·angle evaluations/sec at 1024², K=16 (1 GB300); % HBM roofline"
UNIT = "shift·angle evals/s"
WORKLOAD = "single-1024x1024-K16"
GAMMA = 0.5
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

# DRAM bytes per launch of the pair kernels, from ncu captures of the same
# kernel instantiations on smaller cases (1024 x 256 and 256 x 1024 pairs) scaled
# by the units processed (2047/511 output rows; 1025/257 kx columns).  Set to
# None when a kernel changes after its capture.
NCU_TRAFFIC = {
    "pair_rows_f32": 4.36e9,  # (1.076 GB read + 0.013 GB written) at 511 rows x 2047/511
    "pair_cols_f32": 5.03e9,  # 0.202 GB read x 1025/257 + 1.067 GB written x 1028/260
}


def algorithmic_bytes(name, g):
    """Bytes one launch of a kernel must move at minimum (its inputs once, its outputs once)."""
    HA, WA, HB, WB, KA, KB = g
    R, C = HA + HB - 1, WA + WB - 1
    P = 1 << max(4, math.ceil(math.log2(R)))
    Q = 1 << max(4, math.ceil(math.log2(C)))
    Qh = Q // 2 + 1
    cs = 8  # FP32 complex
    y = KA * KB * R * Qh * cs                 # column-inverted products, output rows only
    spectra = (KA + KB) * Qh * P * cs
    if name.startswith("pair_rows"):
        return y + R * C * (8 + 4)            # Y in, MI (f64) + N (i32) out
    if name.startswith("pair_cols"):
        return spectra + y                    # spectra in, Y out
    if name.startswith("fwd_cols_A"):
        return KA * HA * Qh * cs + KA * Qh * P * cs
    if name.startswith("fwd_cols_B"):
        return KB * HB * Qh * cs + KB * Qh * P * cs
    if name.startswith("fwd_rows_A"):
        return HA * WA * 5 + KA * HA * Qh * cs
    if name.startswith("fwd_rows_B"):
        return HB * WB * 5 + KB * HB * Qh * cs
    return 0


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class _Nvml:
    """The few read-only NVML calls the clock sampler needs, through ctypes (no
    Python NVML package on the GPU hosts).  Raises OSError when NVML is absent."""

    SM = 1  # NVML_CLOCK_SM
    # clock event reason bits of nvml.h
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        n = ctypes.c_uint()
        if self.lib.nvmlDeviceGetCount_v2(ctypes.byref(n)) != 0 or n.value == 0:
            raise OSError("no NVML device")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(min(index, n.value - 1), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reason_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.max_sm = self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def _clock(self, fn):
        v = self.c.c_uint()
        if fn(self.h, self.SM, self.c.byref(v)) != 0:
            raise OSError("clock query failed")
        return float(v.value)

    def sample(self):
        r = self.c.c_ulonglong()
        if self.reason_fn(self.h, self.c.byref(r)) != 0:
            raise OSError("reason query failed")
        return self._clock(self.lib.nvmlDeviceGetClockInfo), self.max_sm, \
            sorted(nm for bit, nm in self.REASONS.items() if r.value & bit)


class ClockSampler:
    """SM clock and clock event reasons sampled during the timed region: every
    2 ms from NVML in a background thread, or, without NVML, every 10 ms from
    nvidia-smi.  stop() returns the median SM clock, the maximum, the reasons
    seen and the number of samples."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.thread = None
        self.samples = []

    def start(self):
        import threading
        try:
            nv = _Nvml(self.idx)
            nv.sample()
        except Exception:
            nv = None
        if nv is not None:
            self.stop_evt = threading.Event()

            def run():
                while not self.stop_evt.is_set():
                    try:
                        self.samples.append(nv.sample())
                    except Exception:
                        pass
                    time.sleep(0.002)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # nvidia-smi's start-up, so that the region is covered
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_evt.set()
            self.thread.join(timeout=5)
            if not self.samples:
                return None
            sm = [x[0] for x in self.samples]
            reasons = sorted({r for x in self.samples for r in x[2]})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(x[1] for x in self.samples),
                    "reasons": reasons, "samples": len(sm), "source": "nvml, 2 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_csv(f)
        os.unlink(self.path)
        if out:
            out["source"] = "nvidia-smi, 10 ms"
        return out


def parse_clock_csv(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen, from the
    lines nvidia-smi writes for ClockSampler.Q (csv, no header, no units); None
    when no line holds a sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


REJECT_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "hw_power_brake_slowdown")


def clocks_rejected(clocks, floor=0.85):
    """True when a timed region must be taken again: it saw a hardware or thermal
    slowdown, or its median SM clock sat below floor x the maximum with no reason
    active (a clock lock left by someone else).  sw_power_cap alone is kept."""
    if not clocks:
        return False
    if any(r in REJECT_REASONS for r in clocks["reasons"]):
        return True
    return not clocks["reasons"] and clocks["sm_mhz"] < floor * clocks["sm_max_mhz"]


def cpu_oracle_rate(cfg, budget_s, rng_seed=7):
    """Direct-method oracle on a bounded random sample of shifts of the same map.
    Returns (shifts per second, shifts, seconds, threads)."""
    import oracle
    A, B = cfg["A"], cfg["B"]
    HA, WA = A.shape
    HB, WB = B.shape
    rng = np.random.default_rng(rng_seed)

    def sample(n):
        return (rng.integers(-(HA - 1), HB, n).astype(np.int32), rng.integers(-(WA - 1), WB, n).astype(np.int32))

    threads = oracle.max_threads()
    n = max(8, threads)
    while True:  # calibrate on growing samples until one takes >= 1 s (or a tenth of the budget)
        dy, dx = sample(n)
        t0 = time.perf_counter()
        oracle.cmif_at(A, cfg["M_A"], B, cfg["M_B"], cfg["K_A"], cfg["K_B"], dy, dx)
        el = time.perf_counter() - t0
        if el >= min(1.0, budget_s / 10) or n > 10_000_000:
            break
        n *= 4
    n = max(threads, int(n * budget_s / max(el, 1e-9)))
    dy, dx = sample(n)
    t0 = time.perf_counter()
    oracle.cmif_at(A, cfg["M_A"], B, cfg["M_B"], cfg["K_A"], cfg["K_B"], dy, dx)
    secs = time.perf_counter() - t0
    return n / secs, n, secs, threads


def cpu_oracle_rate_units(units, budget_s, rng_seed=11):
    """The oracle on a bounded random sample of a workload made of several maps.

    units: list of (A, M_A, B, M_B, K_A, K_B), one per map (B already warped
    for a rotation).  Shifts are drawn uniformly over all the maps' shifts (a
    map is drawn with probability proportional to its shift count), so the
    rate reflects the workload's mix.  Returns (shifts per second, shifts,
    seconds, threads)."""
    import oracle
    rng = np.random.default_rng(rng_seed)
    sizes = np.array([(u[0].shape[0] + u[2].shape[0] - 1) * (u[0].shape[1] + u[2].shape[1] - 1) for u in units],
                     np.float64)
    prob = sizes / sizes.sum()
    threads = oracle.max_threads()

    def run(n):
        which = rng.choice(len(units), size=n, p=prob)
        t0 = time.perf_counter()
        for k in np.unique(which):
            A, MA, B, MB, KA, KB = units[k]
            m = int((which == k).sum())
            dy = rng.integers(-(A.shape[0] - 1), B.shape[0], m).astype(np.int32)
            dx = rng.integers(-(A.shape[1] - 1), B.shape[1], m).astype(np.int32)
            oracle.cmif_at(A, MA, B, MB, KA, KB, dy, dx)
        return time.perf_counter() - t0

    n = max(64, threads)
    while True:
        el = run(n)
        if el >= min(1.0, budget_s / 10) or n > 10_000_000:
            break
        n *= 4
    n = max(threads, int(n * budget_s / max(el, 1e-9)))
    secs = run(n)
    return n / secs, n, secs, threads


def run_reference(args, rank, world):
    """The oracle (the direct method of Sec. 2.2) as the reference arm, on the host cores.

    A full 1024^2 map takes the direct method about two minutes on 16 cores, so
    each step is a bounded random sample of the map's shifts (a few seconds);
    ms_per_step is the measured time of one such step and units_per_step its
    shifts, so that value = units / time of what actually ran."""
    if rank != 0:
        return
    import synth
    cfg = synth.make_workload(WORKLOAD)
    HA, WA = cfg["A"].shape
    HB, WB = cfg["B"].shape
    per_step = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    n_tot, s_tot, thr, ms_steps = 0, 0.0, 1, []
    for i in range(args.warmup + args.steps):
        rate, n, secs, thr = cpu_oracle_rate(cfg, per_step, rng_seed=100 + i)
        if i >= args.warmup:
            n_tot += n
            s_tot += secs
            ms_steps.append(1000.0 * secs)
    value = n_tot / s_tot
    shifts = (HA + HB - 1) * (WA + WB - 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms_steps) / len(ms_steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": HA, "W": WA, "K_A": cfg["K_A"], "K_B": cfg["K_B"],
                   "shifts_per_map": shifts, "angles": 1, "precision": "FP64 direct method (oracle)",
                   "gamma": GAMMA, "units_per_step": n_tot // max(1, args.steps),
                   "step": "a bounded random sample of the map's shifts",
                   "ms_per_map_at_this_rate": 1000.0 * shifts / value,
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{n_tot} random shifts of the 1024^2 K=16 map over {args.steps} steps "
                                   f"of ~{per_step:.0f} s (direct method, FP64 entropies)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_shape(args):
    """Device step loop only, on a smaller planted pair (inputs and workspace of a few GB at most)."""
    import torch
    import paper_2106_14699_gb300 as cm
    import synth
    H, W = (int(v) for v in args.profile_shape.lower().split("x"))
    rng = np.random.default_rng(5)
    A_np, B_np = synth.planted_pair(rng, H, W, max(40, H * W // 500), 16, 16, (3, -5), 0.1, same_labels=True)
    dev = torch.device("cuda", 0)
    A, B = torch.from_numpy(A_np).to(dev), torch.from_numpy(B_np).to(dev)
    R, C = 2 * H - 1, 2 * W - 1
    mi = torch.empty((R, C), dtype=torch.float64, device=dev)
    n = torch.empty((R, C), dtype=torch.int32, device=dev)
    peak = torch.empty(24, dtype=torch.uint8, device=dev)
    plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32)
    for _ in range(args.warmup + args.steps):
        plan.compute(A, None, B, None, mi, n, None, GAMMA, peak)
    torch.cuda.synchronize()
    print(json.dumps({"profile_shape": [H, W], "status": plan.status(),
                      "workspace_gb": plan.workspace_bytes() / 1e9}), flush=True)


class TorchFFTPlain:
    """Comparison baseline, not this library: the plain frequency-domain form of
    the same CMIF map with cuFFT through torch.fft and torch elementwise ops (the
    paper's own PyTorch approach): one-hot level sets, rfft2, per-pair product
    conj(F_a) F_b, irfft2, rounding, c log2 c sums (FP64 accumulation), MI.
    ``dtype`` float64 gives the plain FP64 form (cuFFT Z2D/D2Z): the accuracy of
    this library's FP32 path with its guard, without the guard."""

    def __init__(self, torch, A, MA, B, MB, KA, KB, dev, dtype=None):
        self.t = torch
        self.dt = torch.float32 if dtype is None else dtype
        HA, WA = A.shape
        HB, WB = B.shape
        self.R, self.C = HA + HB - 1, WA + WB - 1
        self.P = 1 << max(4, math.ceil(math.log2(self.R)))
        self.Q = 1 << max(4, math.ceil(math.log2(self.C)))
        self.HA, self.WA, self.KA, self.KB = HA, WA, KA, KB

        def planes(X, MX, K):
            x = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
            m = torch.ones_like(x, dtype=torch.bool) if MX is None else torch.from_numpy(MX).to(dev).bool()
            out = torch.zeros((K, self.P, self.Q), dtype=self.dt, device=dev)
            for k in range(K):
                out[k, :x.shape[0], :x.shape[1]] = ((x == k) & m).to(self.dt)
            return out
        self.la, self.lb = planes(A, MA, KA), planes(B, MB, KB)

    def __call__(self):
        t = self.t
        FA = t.fft.rfft2(self.la)
        FB = t.fft.rfft2(self.lb)
        S = t.zeros((self.P, self.Q), dtype=t.float64, device=FA.device)
        N = t.zeros_like(S)
        CB = t.zeros((self.KB, self.P, self.Q), dtype=self.dt, device=FA.device)
        for a in range(self.KA):
            c = t.round(t.fft.irfft2(t.conj(FA[a])[None] * FB, s=(self.P, self.Q)))  # c[s] = sum_x a(x) b(x + s)
            ca = c.sum(0)
            S += (c * t.log2(c.clamp_min(1.0))).sum(0, dtype=t.float64)
            S -= (ca * t.log2(ca.clamp_min(1.0))).double()
            CB += c
            N += ca.double()
        S -= (CB * t.log2(CB.clamp_min(1.0))).sum(0, dtype=t.float64)
        mi = t.where(N > 0, (S + N * t.log2(N.clamp_min(1.0))) / N.clamp_min(1.0), t.zeros_like(S))
        # circular shift index -> map row / column (chi + H_A - 1, chi + W_A - 1)
        self.out = t.roll(mi, shifts=(self.HA - 1, self.WA - 1), dims=(0, 1))[:self.R, :self.C]
        return self.out

    def status(self):
        return ("OK", None, 0)


def run_secondary(args):
    """The other configurations as bench lines of the same metric (device-timed, graph replay)."""
    import torch
    import paper_2106_14699_gb300 as cm
    import synth
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    d = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    if args.workload == "volume":
        rng = np.random.default_rng(33)
        D = H = W = 64
        Av = rng.integers(0, 8, (D, H, W)).astype(np.int32)
        Av[:, : H // 2, : W // 3] = 3                      # some structure, then a planted 3-D shift
        Bv = np.roll(Av, (3, -5, 7), axis=(0, 1, 2))
        Bv[rng.random(Bv.shape) < 0.1] = 0
        plan = cm.VolumePlan(D, H, W, D, H, W, 8, 8, cm.FP32, graph=True)
        mi = torch.empty((plan.R, plan.C), dtype=torch.float64, device=dev)
        n = torch.empty((plan.R, plan.C), dtype=torch.int32, device=dev)
        pk = torch.empty(24, dtype=torch.uint8, device=dev)
        A, B = d(Av), d(Bv)
        step = lambda: plan.compute(A, None, B, None, mi, n, None, 0.5, pk)
        units, name = plan.R * plan.C, "volume-64^3-K8 FP32"
    elif args.workload in ("torchfft", "torchfft64"):
        cfg = synth.make_workload("single-1024x1024-K16")
        H, W = cfg["A"].shape
        f64 = args.workload == "torchfft64"
        plan = TorchFFTPlain(torch, cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], 16, 16, dev,
                             torch.float64 if f64 else torch.float32)
        step = plan
        units, name = (2 * H - 1) * (2 * W - 1), cfg["name"] + " torch.fft (cuFFT) plain form " + ("FP64" if f64 else "FP32")
        # sanity: the same map as this library's, at a few shifts
        ref = cm.cmif(d(cfg["A"]), d(cfg["M_A"]), d(cfg["B"]), d(cfg["M_B"]), 16, 16, precision=cm.FP32)["mi"]
        got = plan()
        torch.cuda.synchronize()
        print(json.dumps({"torchfft_vs_library_max_abs_mi_diff": float((got - ref).abs().max())}), flush=True)
    elif args.workload == "swmi":
        cfg = synth.make_workload("single-256x256-K16")
        H, W = cfg["A"].shape
        plan = cm.Plan(H, W, H, W, 16, 16, cm.FP64, graph=True, weighted=True)
        R, C = 2 * H - 1, 2 * W - 1
        rng = np.random.default_rng(12)
        wa = d(rng.random((H, W)) * cfg["M_A"])
        wb = d(rng.random((H, W)) * cfg["M_B"])
        mi = torch.empty((R, C), dtype=torch.float64, device=dev)
        nw = torch.empty((R, C), dtype=torch.float64, device=dev)
        pk = torch.empty(24, dtype=torch.uint8, device=dev)
        A, B = d(cfg["A"]), d(cfg["B"])
        step = lambda: plan.compute_weighted(A, wa, B, wb, mi, nw, 0.5, pk)
        units, name = R * C, cfg["name"] + " SWMI FP64"
    elif args.workload == "nmi":
        cfg = synth.make_workload("single-1024x1024-K16")
        H, W = cfg["A"].shape
        plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, graph=True, nmi=True)
        R, C = 2 * H - 1, 2 * W - 1
        mi = torch.empty((R, C), dtype=torch.float64, device=dev)
        n = torch.empty((R, C), dtype=torch.int32, device=dev)
        pk = torch.empty(24, dtype=torch.uint8, device=dev)
        ins = [d(cfg[k]) for k in ("A", "M_A", "B", "M_B")]
        step = lambda: plan.compute(ins[0], ins[1], ins[2], ins[3], mi, n, None, 0.5, pk)
        units, name = R * C, cfg["name"] + " NMI FP32"
    elif args.workload in ("single256", "plain64"):
        small = args.workload == "single256"
        cfg = synth.make_workload("single-256x256-K16" if small else "plain-64x64-K8")
        H, W = cfg["A"].shape
        K = cfg["K_A"]
        prec = cm.FP32 if small else cm.FP64
        plan = cm.Plan(H, W, H, W, K, K, prec, graph=True)
        R, C = 2 * H - 1, 2 * W - 1
        mi = torch.empty((R, C), dtype=torch.float64, device=dev)
        n = torch.empty((R, C), dtype=torch.int32, device=dev)
        pk = torch.empty(24, dtype=torch.uint8, device=dev)
        ins = [d(cfg[k]) for k in ("A", "M_A", "B", "M_B")]
        step = lambda: plan.compute(ins[0], ins[1], ins[2], ins[3], mi, n, None, 0.5, pk)
        units, name = R * C, cfg["name"] + (" FP32" if prec == cm.FP32 else " FP64")
    elif args.workload in ("rotation", "rotation-window"):
        cfg = synth.make_workload("rotation-512x512-K16-64angles")
        H, W = cfg["A"].shape
        win = args.workload == "rotation-window"
        plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, graph=True, window=win, batch_angles=True, autotune=True)
        top = torch.empty(24 * 5, dtype=torch.uint8, device=dev)
        A, B = d(cfg["A"]), d(cfg["B"])
        step = lambda: plan.align_rotations(A, None, B, None, cfg["angles"], 0.5, 5, top)
        if win:  # X_S of the padded search: |chi_i| <= ceil(size_i (1 - gamma)) (equal sizes)
            py, px = math.ceil(H * 0.5), math.ceil(W * 0.5)
            units = (2 * min(py, H - 1) + 1) * (2 * min(px, W - 1) + 1) * len(cfg["angles"])
            name = cfg["name"] + " padded-window FP32"
        else:
            units, name = (2 * H - 1) * (2 * W - 1) * len(cfg["angles"]), cfg["name"] + " FP32"
    elif args.workload == "two-stage":
        cfg = synth.make_workload("rotation-512x512-K16-64angles")
        H, W = cfg["A"].shape
        # no graph: the two stages have different angle lists (one cached graph would be re-captured each call)
        plan = cm.Plan(H, W, H, W, 16, 16, cm.FP32, graph=False, window=True)
        A, B = d(cfg["A"]), d(cfg["B"])
        u = [(i + 0.5) / 16 for i in range(16)]
        step = lambda: plan.align_two_stage(A, None, B, None, 64, u, 0.5)
        py, px = math.ceil(H * 0.5), math.ceil(W * 0.5)
        units = (2 * min(py, H - 1) + 1) * (2 * min(px, W - 1) + 1) * (64 + len(u))
        name = cfg["name"] + " two-stage 64+16 padded-window FP32"
    else:
        cfg = synth.make_workload("uneven-batch-128pairs")
        pairs = [dict(A=d(p["A"]), M_A=d(p["M_A"]), B=d(p["B"]), M_B=d(p["M_B"]), K_A=p["K_A"], K_B=p["K_B"],
                      angles=p["angles"], gamma=0.5) for p in cfg["pairs"]]
        plan = cm.Batch(pairs, cm.FP32, graph=True, batch_angles=True, autotune=True)
        res = torch.empty(24 * len(pairs), dtype=torch.uint8, device=dev)
        stat = torch.empty(len(pairs), dtype=torch.int32, device=dev)
        step = lambda: plan.run(res, stat)
        units = sum((p["A"].shape[0] + p["B"].shape[0] - 1) * (p["A"].shape[1] + p["B"].shape[1] - 1) * len(p["angles"])
                    for p in cfg["pairs"])
        name = cfg["name"] + " FP32"
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clk = ClockSampler(0)
    clk.start()
    stream = torch.cuda.current_stream()
    for i in range(steps):
        flush.zero_()
        e0[i].record(stream)
        step()
        e1[i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / steps
    st = plan.status()
    cpu = None
    if not args.no_cpu_baseline and args.workload in ("plain64", "single256", "rotation", "batch"):
        # the oracle on a bounded sample of the same workload (host cores, after the timed region)
        import oracle
        if args.workload == "batch":
            ou = [(p["A"], p["M_A"]) + oracle.warp_nn(p["B"], p["M_B"], th) + (p["K_A"], p["K_B"])
                  for p in cfg["pairs"] for th in p["angles"]]
            what = "random shifts over the 128 pairs x 4 angles (B warped by the oracle's NN warp)"
        elif args.workload == "rotation":
            ou = [(cfg["A"], cfg["M_A"]) + oracle.warp_nn(cfg["B"], cfg["M_B"], th) + (cfg["K_A"], cfg["K_B"])
                  for th in cfg["angles"][::8]]
            what = "random shifts of 8 of the 64 angles' maps (B warped by the oracle's NN warp)"
        else:
            ou = [(cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], cfg["K_A"], cfg["K_B"])]
            what = "random shifts of the map"
        rate, n_s, secs, thr = cpu_oracle_rate_units(ou, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{n_s} {what} ({secs:.1f} s, direct method, FP64)"}
    print(json.dumps({"metric": METRIC.replace("at 1024², K=16", "on " + name), "value": units / (ms * 1e-3),
                      "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32" if "FP32" in name else "f64",
                      "data": "synthetic", "config": {"workload": name, "units_per_step": units,
                                                       "l2": "flushed between steps (256 MB write)"},
                      "clocks": clocks, "cpu_baseline": cpu,
                      "device_status": {"status": st[0], "max_residual": st[1], "escalations": st[2]},
                      **({"impl": "torch.fft (cuFFT) plain form: comparison baseline, not this library"}
                         if args.workload.startswith("torchfft") else {})}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="single1024",
                    choices=["single1024", "rotation", "rotation-window", "two-stage", "batch", "single256",
                             "plain64", "nmi", "swmi", "torchfft", "torchfft64", "volume"],
                    help="single1024 (default, the headline): 1024^2, K=16; rotation: 512^2, K=16, 64 angles; "
                         "batch: 128 uneven pairs x 4 angles; single256 / plain64: 256^2, K=16 / 64^2, K=8")
    ap.add_argument("--profile-shape", default=None,
                    help="HxW: run only the device step loop on a planted pair of this size (for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_shape:
        run_profile_shape(args)
        return
    if args.workload != "single1024":
        run_secondary(args)
        return

    import torch
    import paper_2106_14699_gb300 as cm
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cfg = synth.make_workload(WORKLOAD)
    A_np, B_np, MA_np, MB_np = cfg["A"], cfg["B"], cfg["M_A"], cfg["M_B"]
    HA, WA = A_np.shape
    HB, WB = B_np.shape
    KA, KB = cfg["K_A"], cfg["K_B"]
    R, C = HA + HB - 1, WA + WB - 1
    shifts = R * C

    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    MA = torch.from_numpy(MA_np).to(dev)
    MB = torch.from_numpy(MB_np).to(dev)
    mi = torch.empty((R, C), dtype=torch.float64, device=dev)
    n = torch.empty((R, C), dtype=torch.int32, device=dev)
    peak = torch.empty(24, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    plan = cm.Plan(HA, WA, HB, WB, KA, KB, cm.FP32)
    stream = torch.cuda.current_stream()

    def step():
        plan.compute(A, MA, B, MB, mi, n, None, GAMMA, peak, stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    st = plan.status()
    if st[0] != "OK":
        raise SystemExit(f"device status after warm-up: {st}")

    def timed_region():
        plan.set_profiling(True)
        clk = ClockSampler(local)
        clk.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stage = {}
        launches = 0
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the step's events)
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
            for name, ms in plan.stage_times():  # synchronises; between steps
                stage.setdefault(name, []).append(ms)
                launches += 2 if name in ("peak", "finalize") else 1  # peak: partial + final; finalize: + merge
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = clk.stop()
        plan.set_profiling(False)
        ms_steps = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        ms_per_step = sum(ms_steps) / len(ms_steps)
        if dist:
            t = torch.tensor([ms_per_step], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_per_step = float(t.item())
        return ms_per_step, stage, launches, clocks

    ms_per_step, stage, launches, clocks = timed_region()
    retake = clocks_rejected(clocks)
    if dist:  # every rank takes the same decision (the retake has barriers)
        t = torch.tensor([1.0 if retake else 0.0], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        retake = bool(t.item() > 0)
    if retake:
        first = clocks
        ms_per_step, stage, launches, clocks = timed_region()
        clocks = dict(clocks or {}, rejected_first_run=first)
    st = plan.status()

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A_np).pin_memory()
        hB = torch.from_numpy(B_np).pin_memory()
        hMA = torch.from_numpy(MA_np).pin_memory()
        hMB = torch.from_numpy(MB_np).pin_memory()
        hmi = torch.empty((R, C), dtype=torch.float64).pin_memory()
        hpk = cm.Peak()
        for _ in range(2):
            plan.compute_host(hA, hMA, hB, hMB, hmi, None, GAMMA, hpk, stream)
        if dist:
            dist.barrier()
        ts = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.compute_host(hA, hMA, hB, hMB, hmi, None, GAMMA, hpk, stream)
            ts.append(time.perf_counter() - t0)
        e2e_s = sum(ts) / len(ts)
        if dist:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = A_np.nbytes + B_np.nbytes + MA_np.nbytes + MB_np.nbytes
        d2h = R * C * 8 + 24
        e2e = {"value": shifts * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (largest mean launch time)
    g = (HA, WA, HB, WB, KA, KB)
    mean_ms = {k: sum(v) / len(v) for k, v in stage.items()}
    dom = max(mean_ms, key=mean_ms.get)
    peak_gbs, peak_kind = measured_peak_gbs()
    alg = algorithmic_bytes(dom, g)
    achieved = alg / (mean_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "traffic": NCU_TRAFFIC.get(dom), "kernel": dom,
                "kernel_ms": mean_ms[dom], "algorithmic_bytes": alg, "peak_source": peak_kind}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, n_s, secs, thr = cpu_oracle_rate(cfg, 15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{n_s} random shifts of the 1024^2 K=16 map ({secs:.1f} s, direct method, FP64)"}

    line = {
        "metric": METRIC, "value": shifts * world / (ms_per_step * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": HA, "W": WA, "K_A": KA, "K_B": KB,
                   "shifts_per_map": shifts, "angles": 1, "precision": "FP32 transforms, fixed-point entropy",
                   "gamma": GAMMA, "l2": "flushed between steps (256 MB write), per-step CUDA events",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "stage_ms": {k: round(v, 4) for k, v in mean_ms.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "device_status": {"status": st[0], "max_residual": st[1], "escalations": st[2]},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
