#!/usr/bin/env python
"""Benchmark of the fused overlap-and-save convolution on GB300.

One step = one ``ols_convolve`` call over the whole workload: the filter bank
(Ns = 2^23 complex64 samples, F = 32 filters of M = 257 taps, Hann-windowed,
segment length N = 2048), inputs resident in HBM.  Metric: output samples per
second, F * (Ns - M + 1) / time.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank convolves its own independent signal of the
same size (weak scaling, no collective on the data path); timing is the max
over ranks.  ``--impl reference`` times the FP64 CPU oracle instead (rank 0
only), on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "output samples/s (F*(Ns-M+1))"
UNIT = "samples/s"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1910_01972_gb300/csrc/ols_forward.cu", "paper_1910_01972_gb300/csrc/ols_segment.cuh",
                  "paper_1910_01972_gb300/csrc/ols_fft_passes.cuh", "paper_1910_01972_gb300/csrc/fft_regs.cuh",
                  "paper_1910_01972_gb300/csrc/tmem.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_forward_bank_Ns8388608_F32_M257_N2048.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--ns", type=int, default=0, help="override the signal length (profiling a smaller case)")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads (batched, adjoint, tensor-core)")
    ap.add_argument("--only", choices=["plain_1x1", "diff", "batched", "tensor_core", "r2r", "post", "cufft"], default=None,
                    help="run just this other workload (with --ns: its signal length) and print its numbers")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def tc_flops(N, F, nseg):
    """Tensor-core operations of one split-precision call: every radix-16 pass
    (log2 N // 4 of them per FFT, one forward per segment and one inverse per
    segment and filter) is, per row of 16 points (N/16 rows per segment), six
    MMAs of N = 32, K = 16 (three split products of a 32 x 32 real DFT-16 matrix
    in two K halves): 6 x 2 x 32 x 16 operations per row."""
    lg = N.bit_length() - 1
    return nseg * (lg // 4) * (F + 1) * (N // 16) * 6 * 2 * 32 * 16


def tc_peak():
    """Dense 16-bit tensor peak in TFLOP/s: the measured bf16 burst figure (FP16
    and BF16 run at the same kind::f16 rate), or the nominal 2250."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured bf16 burst"
    except Exception:
        return 2250.0, "nominal"


def fp32_flops(N, F, nseg):
    """FP32 operations of one call by the conventional count: 5 N log2 N per
    complex N-point FFT (one forward per segment, one inverse per segment and
    filter) and 6 per complex product of a spectrum point."""
    lg = N.bit_length() - 1
    return nseg * (F + 1) * 5 * N * lg + nseg * F * 6 * N


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since that capture."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m_t or not m_h or m_h.group(1) != kernel_source_hash():
        return None
    return float(m_t.group(1))


class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons."""
    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[4], parts[6:10]))
            except (ValueError, IndexError):
                continue
        inwin = [r for r in rows if any(a - 0.05 <= r[0] <= b + 0.05 for a, b in self.windows)]
        used = inwin if len(inwin) >= 3 else rows
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in used for i in range(4) if r[4][i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in used), "sm_max_mhz": max(r[2] for r in used),
                "reasons": reasons, "samples": len(used),
                "window": "timed region" if used is inwin else "whole run (timed region too short)"}


# ------------------------------------------------------------------ oracle legs
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_single_core_rate(s, h, seconds):
    """Oracle outputs/s on one thread, over a prefix sized to ~seconds."""
    import oracle
    n = oracle.threads()
    oracle.set_threads(1)
    try:
        rate, _, desc, _, _ = oracle_rate(s, h, seconds)
    finally:
        oracle.set_threads(n)
    return rate, desc


def oracle_rate(s, h, seconds, max_outputs=None):
    """Time the FP64 oracle on a prefix of the workload sized to ~seconds of
    CPU work.  Returns (outputs/s, threads, sample description, prefix Ns, y_ref)."""
    import oracle
    F, M = h.shape
    cal_ns = min(len(s), M - 1 + 2048)
    t0 = time.perf_counter()
    oracle.conv(s[:cal_ns], h)
    t_cal = max(time.perf_counter() - t0, 1e-6)
    per_out = t_cal / (F * (cal_ns - M + 1))
    n_out = int(seconds / per_out / F)
    if max_outputs:
        n_out = min(n_out, max_outputs)
    n_out = max(1, min(n_out, len(s) - M + 1))
    ns = n_out + M - 1
    t0 = time.perf_counter()
    y_ref = oracle.conv(s[:ns], h)
    dt = time.perf_counter() - t0
    desc = "first %d samples of the signal (all %d filters, %d outputs per filter)" % (ns, F, n_out)
    return F * n_out / dt, oracle.threads(), desc, ns, y_ref


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import synth
    cfg = synth.PLAIN_BANK
    s, h = synth.plain_inputs(cfg)
    budget = 150.0
    per_step = max(0.5, min(5.0, budget / max(1, args.steps + args.warmup)))
    # size each step's sample once, then run W untimed + K timed steps
    rate0, threads, desc, ns, _ = oracle_rate(s, h, per_step)
    import oracle
    for _ in range(args.warmup):
        oracle.conv(s[:ns], h)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.conv(s[:ns], h)
    dt = time.perf_counter() - t0
    outputs = cfg.F * (ns - cfg.M + 1)
    value = outputs * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg.name, "Ns": cfg.Ns, "F": cfg.F, "M": cfg.M, "N": cfg.N,
                   "note": "FP64 direct convolution (Eq. 1) on host cores; each step is a bounded sample"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc + " per step", "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ other workloads
def _time_events(fn, reps, flush=None):
    """Mean device time (ms) of fn() over reps calls, each bracketed by events
    on the current stream; an optional L2 flush runs between calls, outside
    the events."""
    import torch
    st = torch.cuda.current_stream()
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def measure_others(peak, only=None, ns=0):
    """Throughput of the other workloads on this GPU (outputs and samples for
    oracle checks are returned separately; the oracle runs in the CPU leg).
    `only` restricts the run to one workload (for profiling); `ns` then
    overrides the differentiable, real-to-real or tensor-core workload's signal length."""
    import torch
    res, samples = {}, {}
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")       # 256 MB > L2

    def want(name):
        return only is None or only == name

    # one signal, one filter (65,536 samples, M = 64, N = 512): fits in L2, so flush between calls
    if want("plain_1x1"):
        _plain_1x1(res, flush)
    if want("diff"):
        _diff(res, samples, peak, ns)
    if want("batched"):
        _batched(res, samples, peak)
    if want("tensor_core"):
        _tensor_core(res, samples, peak, ns)
    if want("r2r"):
        _r2r(res, samples, peak, ns)
    if want("post"):
        _post(res, samples, peak)
    if want("cufft"):
        _cufft_ols(res, samples, peak)
    torch.cuda.empty_cache()
    return res, samples


def _plain_1x1(res, flush):
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan
    cfg = synth.PLAIN_1x1
    s_np, h_np = synth.plain_inputs(cfg)
    p = Plan(cfg.M, cfg.F, cfg.N)
    p.set_filters(torch.from_numpy(h_np).cuda())
    s = torch.from_numpy(s_np).cuda()
    y = p.convolve(s)
    ms = _time_events(lambda: p.convolve(s, out=y), 50, flush)
    nout = cfg.Ns - cfg.M + 1
    res["plain_1x1"] = {"workload": cfg.name, "value": nout / (ms * 1e-3), "unit": UNIT, "ms": ms,
                        "note": "L2 flushed between calls; launch-latency bound (146 segments)"}
    p.close()


def _diff(res, samples, peak, ns):
    """Differentiable shape: forward + adjoint (ds and dh)."""
    import dataclasses
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan, _native
    cfg = synth.DIFF
    if ns:
        cfg = dataclasses.replace(cfg, Ns=ns, name=cfg.name.replace("Ns4194304", "Ns%d" % ns))
    s_np, h_np, w_np = synth.diff_inputs(cfg)
    p = Plan(cfg.M, cfg.F, cfg.N)
    p.set_filters(torch.from_numpy(h_np).cuda())
    s = torch.from_numpy(s_np).cuda()
    y = p.convolve(s)
    gy = (2.0 * torch.from_numpy(w_np).cuda()[None, :] * y).contiguous()
    nout = cfg.Ns - cfg.M + 1
    ms_f = _time_events(lambda: p.convolve(s, out=y), 10)
    nb = p.backward_workspace(cfg.Ns)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) & ~255
    ds = torch.empty(cfg.Ns, dtype=torch.complex64, device="cuda")
    dh = torch.empty((cfg.F, cfg.M), dtype=torch.complex64, device="cuda")
    stp = torch.cuda.current_stream().cuda_stream

    def bwd():
        _native.check(_native.ols_convolve_backward(p.handle, s.data_ptr(), cfg.Ns, gy.data_ptr(), ds.data_ptr(),
                                                    dh.data_ptr(), wp, nb, stp), "ols_convolve_backward")
    bwd()
    ms_b = _time_events(bwd, 10)
    b_bytes = 8 * cfg.Ns + 8 * cfg.F * nout + 8 * cfg.Ns + 8 * cfg.F * cfg.M
    res["diff"] = {"workload": cfg.name, "forward": {"value": cfg.F * nout / (ms_f * 1e-3), "unit": UNIT, "ms": ms_f},
                   "backward": {"value": cfg.F * nout / (ms_b * 1e-3), "unit": "gradient samples/s (F*(Ns-M+1))",
                                "ms": ms_b, "hbm_frac": b_bytes / (ms_b * 1e-3) / 1e9 / peak,
                                "algorithmic_bytes": b_bytes}}
    samples["diff"] = None
    p.close()
    del y, gy, ds, dh, ws


def _batched(res, samples, peak):
    """Uneven batch: one graph replay of the batched launches vs 64 per-signal plain launches."""
    import numpy as np
    import torch
    import synth
    from paper_1910_01972_gb300 import BatchPlan, Plan
    spec = synth.batch_spec()
    ss, hs = synth.batch_inputs(spec)
    bp = BatchPlan(spec.Ns, spec.M, spec.F)
    bp.set_filters([torch.from_numpy(h).cuda() for h in hs])
    sd = [torch.from_numpy(x).cuda() for x in ss]
    ys = bp.outputs()
    st_t, yt_t = bp.pointer_table(sd), bp.pointer_table(ys)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        bp.launch(st_t, yt_t)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            bp.launch(st_t, yt_t)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    outs = sum(f * n for f, n in zip(spec.F, bp.Nout))
    ms_g = _time_events(graph.replay, 5)
    # the tile schedule: tuned runs of tiles per item against one tile per item
    ms_tuned = _time_events(lambda: bp.launch(st_t, yt_t), 5)
    b1 = BatchPlan(spec.Ns, spec.M, spec.F, N=bp.N, tiles=[1] * bp.B)
    b1.set_filters([torch.from_numpy(h).cuda() for h in hs])
    b1.launch(st_t, yt_t)
    ms_one = _time_events(lambda: b1.launch(st_t, yt_t), 5)
    items_one = sum(b1.items)
    b1.close()
    hist = {}
    for r in bp.tiles:
        hist[str(r)] = hist.get(str(r), 0) + 1
    tile_schedule = {"tiles_per_item_histogram": hist, "items": sum(bp.items), "ms_tuned": ms_tuned,
                     "one_tile_per_item": {"items": items_one, "ms": ms_one},
                     "note": "direct launches (no graph); runs tuned per (M, F, N) by ols_autotune_tiles"}
    # the same batch as one persistent launch per segment length
    bq = BatchPlan(spec.Ns, spec.M, spec.F, N=bp.N, per_n=True)
    bq.set_filters([torch.from_numpy(h).cuda() for h in hs])
    bq.launch(st_t, yt_t)
    ms_n = _time_events(lambda: bq.launch(st_t, yt_t), 5)
    n_launches = bq.ngroups
    bq.close()
    plans = []
    for b in range(bp.B):
        q = Plan(spec.M[b], spec.F[b], bp.N[b])
        q.set_filters(torch.from_numpy(hs[b]).cuda())
        plans.append(q)

    def per_signal():
        for b in range(bp.B):
            plans[b].convolve(sd[b], out=ys[b])
    per_signal()
    ms_p = _time_events(per_signal, 5)
    in_bytes = 8 * sum(spec.Ns)
    bb = in_bytes + 8 * outs
    res["batched"] = {"workload": "batch_B64_Ns2^16..2^22_F8..128_M33..1025_autotuned",
                      "value": outs / (ms_g * 1e-3), "unit": UNIT, "ms": ms_g, "hbm_frac": bb / (ms_g * 1e-3) / 1e9 / peak,
                      "launches": bp.ngroups, "segment_lengths": sorted(set(bp.N)),
                      "per_segment_length": {"value": outs / (ms_n * 1e-3), "ms": ms_n, "launches": n_launches,
                                             "note": "one persistent launch per distinct N, no graph"},
                      "per_signal": {"value": outs / (ms_p * 1e-3), "ms": ms_p, "launches": bp.B},
                      "speedup_vs_per_signal": ms_p / ms_g, "total_outputs": outs, "tile_schedule": tile_schedule}
    graph.replay()
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(5))
    picks = []
    for b in range(0, bp.B, 8):
        fi = g.integers(0, spec.F[b], 32)
        ji = g.integers(0, bp.Nout[b], 32)
        got = ys[b][torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()
        picks.append((ss[b], hs[b], fi, ji, got))
    samples["batched"] = picks
    for q in plans:
        q.close()
    bp.close()
    del ys, sd, graph


def _tensor_core(res, samples, peak, ns=0):
    """Tensor-core split precision vs FP32 on the same inputs (`ns` overrides
    the signal length)."""
    import dataclasses
    import numpy as np
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan, _native
    cfg = synth.TC_SPLIT
    if ns:
        cfg = dataclasses.replace(cfg, Ns=ns, name=cfg.name.replace("Ns16777216", "Ns%d" % ns))
    s_np, h_np = synth.plain_inputs(cfg)
    s = torch.from_numpy(s_np).cuda()
    h = torch.from_numpy(h_np).cuda()
    nout = cfg.Ns - cfg.M + 1
    y = torch.empty((cfg.F, nout), dtype=torch.complex64, device="cuda")
    tcres = {}
    g = np.random.Generator(np.random.PCG64(6))
    fi = g.integers(0, cfg.F, 4000)
    ji = g.integers(0, nout, 4000)
    samples["tc"] = {"s": s_np, "h": h_np, "fi": fi, "ji": ji}
    for flag, name in ((0, "fp32"), (_native.OLS_FLAG_TC_FP16SPLIT, "fp16split"), (_native.OLS_FLAG_TC_BF16SPLIT,
                                                                                     "bf16split")):
        q = Plan(cfg.M, cfg.F, cfg.N, flags=flag)
        q.set_filters(h)
        q.convolve(s, out=y)
        ms = _time_events(lambda: q.convolve(s, out=y), 5)
        tb = 8 * cfg.Ns + 8 * cfg.F * nout
        tcres[name] = {"value": cfg.F * nout / (ms * 1e-3), "unit": UNIT, "ms": ms,
                       "hbm_frac": tb / (ms * 1e-3) / 1e9 / peak, "status": q.status()}
        if flag:
            nseg = q.query(cfg.Ns)["nseg"]
            fl = tc_flops(cfg.N, cfg.F, nseg)
            tp, tk = tc_peak()
            tcres[name].update({"tensor_tflops": fl / (ms * 1e-3) / 1e12, "tensor_frac": fl / (ms * 1e-3) / 1e12 / tp,
                                "tensor_flops_per_launch": fl, "tensor_peak": tp, "tensor_peak_kind": tk})
            # the workload's stored form: the signal as 16-bit hi / lo planes
            # (8 bytes per sample, the same bytes as FP32)
            hi, lo = q.split_signal(s)
            q.convolve_split(hi, lo, out=y)
            ms_sp = _time_events(lambda: q.convolve_split(hi, lo, out=y), 5)
            tcres[name]["split_input"] = {"value": cfg.F * nout / (ms_sp * 1e-3), "unit": UNIT, "ms": ms_sp,
                                          "hbm_frac": tb / (ms_sp * 1e-3) / 1e9 / peak,
                                          "note": "ols_convolve_split on planes from ols_split_signal"}
            del hi, lo
        torch.cuda.synchronize()
        samples["tc"][name] = y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()
        q.close()
    res["tensor_core"] = {"workload": cfg.name, **tcres}
    del y, s, h


def _r2r(res, samples, peak, ns=0):
    """Real-to-real form (Sec. 3.4's R2R variant) on the filter-bank shape
    (`ns` overrides the signal length)."""
    import dataclasses
    import numpy as np
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan, _native
    cfg = synth.R2R_BANK
    if ns:
        cfg = dataclasses.replace(cfg, Ns=ns, name=cfg.name.replace("Ns8388608", "Ns%d" % ns))
    s_np, h_np = synth.real_inputs(cfg)
    p = Plan(cfg.M, cfg.F, cfg.N, flags=_native.OLS_FLAG_R2R)
    p.set_filters_real(torch.from_numpy(h_np).cuda())
    s = torch.from_numpy(s_np).cuda()
    y = p.convolve_real(s)
    ms = _time_events(lambda: p.convolve_real(s, out=y), 20)
    nout = cfg.Ns - cfg.M + 1
    fc = (cfg.F + 1) // 2
    rb = 4 * cfg.Ns + 8 * fc * cfg.N + 4 * cfg.F * nout
    res["r2r"] = {"workload": cfg.name, "value": cfg.F * nout / (ms * 1e-3), "unit": "real " + UNIT, "ms": ms,
                  "hbm_frac": rb / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes": rb,
                  "note": "real signal and filters; filters paired into one complex inverse FFT each"}
    g = np.random.Generator(np.random.PCG64(9))
    fi = g.integers(0, cfg.F, 4000)
    ji = g.integers(0, nout, 4000)
    samples["r2r"] = {"s": s_np, "h": h_np, "fi": fi, "ji": ji,
                      "got": y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()}
    p.close()
    del y, s


def _post(res, samples, peak):
    """Post-processing fused into the convolution (Sec. 4.3, 4.4) on the
    filter-bank shape: power |y|^2, threshold detection, peak finding,
    derivative of y."""
    import numpy as np
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan
    cfg = synth.PLAIN_BANK
    s_np, h_np = synth.plain_inputs(cfg)
    p = Plan(cfg.M, cfg.F, cfg.N)
    p.set_filters(torch.from_numpy(h_np).cuda())
    s = torch.from_numpy(s_np).cuda()
    nout = cfg.Ns - cfg.M + 1
    outs = cfg.F * nout
    base = 8 * cfg.Ns + 8 * cfg.F * cfg.N
    pw = p.convolve_power(s)
    ms_p = _time_events(lambda: p.convolve_power(s, out=pw), 20)
    g = np.random.Generator(np.random.PCG64(10))
    fi = g.integers(0, cfg.F, 3000)
    ji = g.integers(0, nout, 3000)
    fit, jit = torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()
    samples["post"] = {"s": s_np, "h": h_np, "fi": fi, "ji": ji, "p": pw[fit, jit].cpu().numpy()}
    thr = float(torch.quantile(pw.flatten()[: 1 << 22], 0.9999).item())
    del pw
    cap = 1 << 20
    rec, cnt = p.convolve_detect(s, thr, cap)
    ms_d = _time_events(lambda: p.convolve_detect(s, thr, cap), 20)
    torch.cuda.synchronize()
    found = int(cnt.item())
    del rec, cnt
    rec, cnt = p.convolve_peaks(s, thr, cap)
    ms_k = _time_events(lambda: p.convolve_peaks(s, thr, cap), 20)
    torch.cuda.synchronize()
    n_peaks = int(cnt.item())
    from paper_1910_01972_gb300 import decode_candidates
    kf, kj, kp = decode_candidates(rec, min(n_peaks, 2000))
    samples["post"]["peaks"] = (kf, kj, kp)
    del rec, cnt
    d = p.convolve_derivative(s)
    ms_v = _time_events(lambda: p.convolve_derivative(s, out=d), 20)
    samples["post"]["d"] = d[fit, jit].cpu().numpy()
    del d
    b_p = base + 4 * outs
    b_d = base + 16 * min(found, cap)
    b_v = base + 8 * outs
    b_k = base + 16 * min(n_peaks, cap)
    res["post"] = {"workload": cfg.name,
                   "power": {"value": outs / (ms_p * 1e-3), "unit": UNIT, "ms": ms_p,
                             "hbm_frac": b_p / (ms_p * 1e-3) / 1e9 / peak, "algorithmic_bytes": b_p},
                   "detect": {"value": outs / (ms_d * 1e-3), "unit": UNIT, "ms": ms_d, "threshold": thr,
                              "candidates": found, "hbm_frac": b_d / (ms_d * 1e-3) / 1e9 / peak,
                              "algorithmic_bytes": b_d},
                   "peaks": {"value": outs / (ms_k * 1e-3), "unit": UNIT, "ms": ms_k, "threshold": thr,
                             "candidates": n_peaks, "hbm_frac": b_k / (ms_k * 1e-3) / 1e9 / peak,
                             "algorithmic_bytes": b_k,
                             "note": "local maxima of the power at or above the threshold; segments laid out "
                                     "like the derivative's"},
                   "derivative": {"value": outs / (ms_v * 1e-3), "unit": UNIT, "ms": ms_v,
                                  "hbm_frac": b_v / (ms_v * 1e-3) / 1e9 / peak, "algorithmic_bytes": b_v,
                                  "note": "segments advance by L-2 (1790 of 2048 points) so each output's "
                                          "neighbours are in its own segment"}}
    p.close()
    del s


def _cufft_ols(res, samples, peak):
    """Library comparison, not the product path: the unfused overlap-and-save of
    Sec. 3.3 with cuFFT through torch.fft (segment separation, batched forward
    FFT, product with every filter's spectrum, batched inverse FFT, discard of
    the M-1 aliased samples), each step a separate kernel with its result in
    HBM.  The paper's cuFFT-OLS uses load/store callbacks for the product and
    the discard; torch.fft has none, so this is the callback-free form."""
    import numpy as np
    import torch
    import synth
    cfg = synth.PLAIN_BANK
    s_np, h_np = synth.plain_inputs(cfg)
    N, M, F = cfg.N, cfg.M, cfg.F
    L = N - M + 1
    nout = cfg.Ns - M + 1
    nseg = (nout + L - 1) // L
    s = torch.from_numpy(s_np).cuda()
    H = torch.fft.fft(torch.from_numpy(h_np).cuda(), n=N, dim=1)                 # [F][N]
    s_pad = torch.zeros((nseg - 1) * L + N, dtype=torch.complex64, device="cuda")
    y = torch.empty((F, nseg * L), dtype=torch.complex64, device="cuda")

    def step():
        s_pad[: cfg.Ns].copy_(s)
        seg = s_pad.unfold(0, N, L)                                               # [nseg][N] view
        S = torch.fft.fft(seg, dim=1)                                             # forward FFTs
        Yf = torch.fft.ifft(S[None, :, :] * H[:, None, :], dim=2)                 # [F][nseg][N]
        y.view(F, nseg, L).copy_(Yf[:, :, M - 1:])                                # discard, merge
    step()
    ms = _time_events(step, 5)
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(11))
    fi = g.integers(0, F, 3000)
    ji = g.integers(0, nout, 3000)
    samples["cufft"] = {"s": s_np, "h": h_np, "fi": fi, "ji": ji,
                        "got": y[torch.from_numpy(fi).cuda(), torch.from_numpy(ji).cuda()].cpu().numpy()}
    res["cufft_ols_comparison"] = {
        "workload": cfg.name, "value": F * nout / (ms * 1e-3), "unit": UNIT, "ms": ms,
        "note": "library comparison (not the product path): unfused overlap-and-save with cuFFT via torch.fft, "
                "no callbacks; intermediate [F][nseg][N] complex in HBM"}
    del y, s_pad, H, s
    torch.cuda.empty_cache()


def others_errors(samples):
    """Relative L2 errors of the other workloads' sampled outputs against the oracle."""
    import numpy as np
    import oracle
    out = {}
    if samples.get("batched"):
        num = den = 0.0
        for s, h, fi, ji, got in samples["batched"]:
            ref = oracle.conv_at(s, h, fi, ji)
            num += float(np.sum(np.abs(got - ref) ** 2))
            den += float(np.sum(np.abs(ref) ** 2))
        out["batched"] = (num / den) ** 0.5
    if samples.get("post"):
        d = samples["post"]
        ref_p = oracle.power_at(d["s"], d["h"], d["fi"], d["ji"])
        out["post_power"] = float(np.linalg.norm(d["p"].astype(np.float64) - ref_p) / np.linalg.norm(ref_p))
        ref_d = oracle.derivative_at(d["s"], d["h"], d["fi"], d["ji"])
        ref_y = oracle.conv_at(d["s"], d["h"], d["fi"], d["ji"])
        out["post_derivative_vs_y_norm"] = float(np.linalg.norm(d["d"] - ref_d) / np.linalg.norm(ref_y))
        if "peaks" in d:
            # reported peaks: their powers against the oracle's (the peak test itself is in the GPU tests)
            kf, kj, kp = d["peaks"]
            ref_k = oracle.power_at(d["s"], d["h"], kf, kj)
            out["post_peaks_power"] = float(np.linalg.norm(kp.astype(np.float64) - ref_k) / np.linalg.norm(ref_k))
    if samples.get("cufft"):
        d = samples["cufft"]
        ref = oracle.conv_at(d["s"], d["h"], d["fi"], d["ji"])
        out["cufft_ols_comparison"] = float(np.linalg.norm(d["got"] - ref) / np.linalg.norm(ref))
    if samples.get("r2r"):
        d = samples["r2r"]
        ref = oracle.conv_real_at(d["s"], d["h"], d["fi"], d["ji"])
        out["r2r"] = float(np.linalg.norm(d["got"].astype(np.float64) - ref) / np.linalg.norm(ref))
    if samples.get("tc"):
        d = samples["tc"]
        ref = oracle.conv_at(d["s"], d["h"], d["fi"], d["ji"])
        for name in ("fp32", "fp16split", "bf16split"):
            out["tc_" + name] = float(np.linalg.norm(d[name] - ref) / np.linalg.norm(ref))
    return out


# ------------------------------------------------------------------ our leg
def run_ours(args):
    import numpy as np
    import torch
    import synth
    from paper_1910_01972_gb300 import Plan, _native
    from paper_1910_01972_gb300 import build as _build

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    _native.lib()
    if args.only:
        # one other workload alone (profiling aid): its numbers, no headline line
        if rank == 0:
            peak, _ = measured_peaks()
            res, _ = measure_others(peak, only=args.only, ns=args.ns)
            print(json.dumps({"only": args.only, "others": res}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    cfg = synth.PLAIN_BANK
    if args.ns:
        import dataclasses
        cfg = dataclasses.replace(cfg, Ns=args.ns, name=cfg.name.replace("Ns8388608", "Ns%d" % args.ns))
    s_np, h_np = synth.plain_inputs(cfg)
    if rank:
        # every rank convolves its own independent signal of the same size
        s_np = synth.signal(synth.rng(cfg.index, salt=100 + rank), cfg.Ns)
    plan = Plan(cfg.M, cfg.F, cfg.N)
    q = plan.query(cfg.Ns)
    Nout, L, nseg = q["Nout"], q["L"], q["nseg"]
    s = torch.from_numpy(s_np).cuda()
    h = torch.from_numpy(h_np).cuda()
    plan.set_filters(h)
    y = torch.empty((cfg.F, Nout), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream()
    if not args.no_e2e:
        # the end-to-end leg's pinned host buffers, allocated and first used now, well before
        # that leg's timed loop (a fresh 2 GB pinned allocation can leave the host busy for a while)
        s_host = torch.from_numpy(s_np).pin_memory()
        y_host = torch.empty((cfg.F, Nout), dtype=torch.complex64, pin_memory=True)
        plan.convolve_host(s_host, y_host)
        torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()

    for _ in range(max(3, args.warmup)):
        plan.convolve(s, out=y)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    e0.record(st)
    for _ in range(args.steps):
        plan.convolve(s, out=y)
    e1.record(st)
    torch.cuda.synchronize()
    t_host1 = time.time()
    if dist is not None:
        dist.barrier()
    clocks.mark(t_host0, t_host1)
    ms_total = e0.elapsed_time(e1)
    launches = plan.last_launch_count() * args.steps
    if dist is not None:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    outputs = cfg.F * Nout
    value = world * outputs / (ms_step * 1e-3)

    # roofline of the (only) kernel: algorithmic bytes per launch / average launch time
    alg_bytes = 8 * cfg.Ns + 8 * cfg.F * cfg.N + 8 * cfg.F * Nout
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms_step * 1e-3) / 1e9
    traffic = ncu_traffic()

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        plan.convolve_host(s_host, y_host)
        torch.cuda.synchronize()

        def d2h_probe(n=3):
            # one whole-output copy device -> host, individually timed
            r = []
            for _ in range(n):
                e0.record(st)
                y_host.copy_(y, non_blocking=True)
                e1.record(st)
                torch.cuda.synchronize()
                r.append(round(e0.elapsed_time(e1), 3))
            return r

        probe_before = d2h_probe()
        if dist is not None:
            dist.barrier()
        per_call = []
        t0 = time.time()
        e0.record(st)
        for _ in range(args.e2e_steps):
            tc = time.perf_counter()
            plan.convolve_host(s_host, y_host)      # returns after y_host is complete
            per_call.append((time.perf_counter() - tc) * 1e3)
        e1.record(st)
        torch.cuda.synchronize()
        t1 = time.time()
        clocks.mark(t0, t1)
        ms_e2e = (t1 - t0) * 1e3 / args.e2e_steps
        probe_after = d2h_probe()
        # one more call (outside the timed region) with the library's per-stage events
        plan.host_timing(True)
        plan.convolve_host(s_host, y_host)
        stages = {k: (round(v, 3) if k != "chunks" else v) for k, v in plan.host_stage_ms().items()}
        plan.host_timing(False)
        if dist is not None:
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        cseg_chunks = plan.last_launch_count()
        h2d = 8 * (cfg.Ns + (cseg_chunks - 1) * (cfg.M - 1))
        # the host link on this machine, same run: one whole-array copy each way
        # (pinned), the floor of any pipelined host-buffer convolution
        # (the best of three individually timed copies: one copy of 2 GB is
        # itself noisy from call to call)
        link = {}
        for name, dst, src in (("h2d", s, s_host), ("d2h", y_host, y)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            times = []
            for _ in range(3):
                e0.record(st)
                dst.copy_(src, non_blocking=True)
                e1.record(st)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = min(times)
            link[name + "_GBps"] = src.numel() * 8 / (ms * 1e-3) / 1e9
            link[name + "_ms"] = ms
        link["floor_ms"] = max(link["h2d_ms"], link["d2h_ms"])
        e2e = {"value": world * outputs / (ms_e2e * 1e-3), "unit": UNIT, "ms_per_step": ms_e2e,
               "steps": args.e2e_steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * cfg.F * Nout,
               "path": "ols_convolve_host: pinned host buffers, chunked H2D / kernel / D2H on two streams",
               "link": link, "frac_of_link_floor": link["floor_ms"] / ms_e2e,
               "per_call_ms": {"min": round(min(per_call), 3), "median": round(statistics.median(per_call), 3),
                               "max": round(max(per_call), 3), "all": [round(x, 2) for x in per_call]},
               "d2h_probe_ms": {"before": probe_before, "after": probe_after},
               "stages_one_call": stages}
        del y_host, s_host
    others, samples = (None, None)
    if rank == 0 and world == 1 and not args.no_others and not args.ns:
        others, samples = measure_others(peak)
    clk = clocks.stop()

    # FP32 roofline (context beside the HBM one): the conventional operation
    # count against the peak of the FP32 units (SMs x 128 lanes x 2 operations
    # per FMA x the SM clock measured under load, else the maximum clock)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    flops = fp32_flops(cfg.N, cfg.F, nseg)
    fp32_achieved = flops / (ms_step * 1e-3) / 1e12
    roof_fp32 = {"bound": "fp32", "achieved": fp32_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                 "frac": fp32_achieved / fp32_peak, "flops_per_launch": flops,
                 "count": "5 N log2 N per complex FFT + 6 per complex product",
                 "peak_basis": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (sms, mhz)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, desc, ns, y_ref = oracle_rate(s_np, h_np, args.cpu_seconds)
        got = y[:, : ns - cfg.M + 1].cpu().numpy()
        err = max(float(np.linalg.norm(got[f] - y_ref[f]) / np.linalg.norm(y_ref[f])) for f in range(cfg.F))
        rate1, desc1 = oracle_single_core_rate(s_np, h_np, min(4.0, args.cpu_seconds / 3))
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "cpu_model": cpu_model(), "single_core": {"value": rate1, "unit": UNIT, "sample": desc1},
               "gpu_rel_l2_on_sample": err}
        if samples:
            cpu["other_workloads_rel_l2_on_samples"] = others_errors(samples)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "Ns": cfg.Ns, "F": cfg.F, "M": cfg.M, "N": cfg.N, "L": L, "nseg": nseg,
                   "filters": "complex Gaussian x Hann, unit L2", "signal": "uniform[-1,1] re/im, seeded",
                   "l2": "working set %.2f GB > 129 MB L2: each step streams %.2f GB of output through L2, "
                         "evicting the previous step's data (no separate flush)" % (
                             (8 * cfg.Ns + 8 * cfg.F * Nout) / 1e9, 8 * cfg.F * Nout / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes},
        "roofline_fp32": roof_fp32,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "others": others,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
