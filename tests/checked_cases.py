"""Parity cases run against the bounds-checked build of the library (built
with OLS_CHECK=1 and selected through OLS_LIBRARY): every global access of
the forward, real-to-real, post-processing, tensor-core, adjoint and batched
kernels is checked against its buffer, and a failed check sets bit 2 of the
plan's status word instead of accessing memory.  Run as ``python -m tests.checked_cases`` by
tests/test_checked_gpu.py; prints one JSON line."""
import json
import os

import numpy as np
import torch

import oracle
import synth
from paper_1910_01972_gb300 import BatchPlan, Plan, _native, decode_candidates

FWD = [  # (N, M, F, Ns): every segment length, ragged tails, the degenerate sizes
    (256, 33, 3, 20_001), (512, 64, 2, 65_536), (1024, 129, 4, 30_000), (2048, 257, 3, 60_001),
    (4096, 512, 2, 100_000), (8192, 1025, 2, 90_000), (1024, 129, 2, 129), (1024, 100, 2, 900),
    (512, 1, 2, 3_000), (4096, 4096, 1, 9_000), (512, 257, 3, 7_000)]
TC = [(4096, 512, 3, 60_000), (256, 33, 2, 20_001), (2048, 257, 3, 9_001)]
BWD = [(1024, 129, 4, 30_000), (256, 33, 3, 5_000), (2048, 257, 2, 20_001), (1024, 129, 3, 129)]
R2R = [(2048, 257, 5, 40_000), (256, 256, 2, 2_000), (512, 1, 1, 5_000), (8192, 1025, 3, 30_000),
       (1024, 100, 7, 1_000), (2048, 257, 2, 257)]
POST = [(256, 254, 2, 3_000), (2048, 257, 3, 40_001), (512, 1, 2, 5_000), (8192, 1025, 2, 30_000),
        (1024, 100, 3, 1_000), (2048, 257, 2, 258)]
BATCH = {"Ns": [20_001, 3_000, 65_536, 258, 9_000], "M": [33, 257, 64, 257, 1025],
         "F": [3, 2, 1, 5, 2], "N": [256, 2048, 512, 1024, 4096]}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def main():
    out = {"library": os.path.basename(_native.LIB_PATH), "cases": 0, "status": 0, "worst": {}, "at": {}}
    worst = {"fwd": 0.0, "tc": 0.0, "ds": 0.0, "dh": 0.0}

    def note(key, value, case):
        if value > worst.get(key, 0.0):
            worst[key] = value
            out["at"][key] = list(case)
    for N, M, F, Ns in FWD:
        g = np.random.Generator(np.random.PCG64(N + M + F))
        s, h = synth.signal(g, Ns), synth.filters(g, F, M)
        p = Plan(M, F, N)
        p.set_filters(dev(h))
        y = p.convolve(dev(s)).cpu().numpy()
        out["status"] |= p.status()
        note("fwd", oracle.max_stream_rel_l2(y, oracle.conv(s, h), oracle.stream_scale(s, h, y.shape[1])), (N, M, F, Ns))
        out["cases"] += 1
        p.close()
    for N, M, F, Ns in TC:
        g = np.random.Generator(np.random.PCG64(7 * N + M))
        s, h = synth.signal(g, Ns), synth.filters(g, F, M)
        p = Plan(M, F, N, flags=_native.OLS_FLAG_TC_FP16SPLIT)
        p.set_filters(dev(h))
        sd = dev(s)
        y = p.convolve(sd)
        hi, lo = p.split_signal(sd)
        y2 = p.convolve_split(hi, lo)
        torch.cuda.synchronize()
        out["status"] |= p.status()
        note("tc", oracle.max_stream_rel_l2(y.cpu().numpy(), oracle.conv(s, h), oracle.stream_scale(s, h, y.shape[1])),
             (N, M, F, Ns))
        out.setdefault("tc_split_equal", True)
        out["tc_split_equal"] = out["tc_split_equal"] and bool(torch.equal(y, y2))
        out["cases"] += 1
        p.close()
    for N, M, F, Ns in BWD:
        g = np.random.Generator(np.random.PCG64(11 * N + M))
        s, h = synth.signal(g, Ns), synth.filters(g, F, M)
        gy = (g.normal(size=(F, Ns - M + 1)) + 1j * g.normal(size=(F, Ns - M + 1))).astype(np.complex64)
        p = Plan(M, F, N)
        p.set_filters(dev(h))
        ds, dh = p.convolve_backward(dev(s), dev(gy))
        torch.cuda.synchronize()
        out["status"] |= p.status()
        ds_ref, dh_ref = oracle.adjoint(s, h, gy)
        note("ds", oracle.rel_l2(ds.cpu().numpy(), ds_ref), (N, M, F, Ns))
        note("dh", oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref), (N, M, F, Ns))
        out["cases"] += 1
        p.close()
    worst.update({"r2r": 0.0, "power": 0.0, "deriv": 0.0, "detect": 0.0, "peaks": 0.0, "batch": 0.0})
    for N, M, F, Ns in R2R:
        g = np.random.Generator(np.random.PCG64(13 * N + M + F))
        s, h = synth.real_signal(g, Ns), synth.real_filters(g, F, M)
        p = Plan(M, F, N, flags=_native.OLS_FLAG_R2R)
        p.set_filters_real(dev(h))
        y = p.convolve_real(dev(s)).cpu().numpy()
        out["status"] |= p.status()
        note("r2r", oracle.max_stream_rel_l2(y, oracle.conv_real(s, h), oracle.stream_scale(s, h, y.shape[1])),
             (N, M, F, Ns))
        out["cases"] += 1
        p.close()
    for N, M, F, Ns in POST:
        g = np.random.Generator(np.random.PCG64(17 * N + M + F))
        s, h = synth.signal(g, Ns), synth.filters(g, F, M)
        p = Plan(M, F, N)
        p.set_filters(dev(h))
        sd = dev(s)
        pw = p.convolve_power(sd).cpu().numpy()
        d = p.convolve_derivative(sd).cpu().numpy()
        p_ref, y_ref = oracle.power(s, h), oracle.conv(s, h)
        thr = float(np.quantile(p_ref, 0.99))
        rec, cnt = p.convolve_detect(sd, thr, capacity=64)   # overflows: the cap check is exercised
        torch.cuda.synchronize()
        out["status"] |= p.status()
        count = int(cnt.item())
        fi, ji, pj = decode_candidates(rec, count)
        note("power", oracle.max_stream_rel_l2(pw, p_ref), (N, M, F, Ns))
        d_ref = oracle.derivative(s, h)
        note("deriv", max(np.linalg.norm(d[f] - d_ref[f]) / np.linalg.norm(y_ref[f]) for f in range(F)),
             (N, M, F, Ns))
        band = 1e-5 * thr
        ok = int(np.sum(p_ref >= thr + band)) <= count <= int(np.sum(p_ref >= thr - band))
        ok = ok and bool(np.all(p_ref[fi, ji] >= thr - band))
        note("detect", 0.0 if ok else 1.0, (N, M, F, Ns))
        if N - M + 1 >= 3:                                   # peaks: the L-2 layout
            rec, cnt = p.convolve_peaks(sd, thr, capacity=64)
            torch.cuda.synchronize()
            out["status"] |= p.status()
            count = int(cnt.item())
            fi, ji, _ = decode_candidates(rec, count)
            left = np.pad(p_ref[:, :-1], ((0, 0), (1, 0)), constant_values=-np.inf)
            right = np.pad(p_ref[:, 1:], ((0, 0), (0, 1)), constant_values=-np.inf)
            may = (p_ref >= thr * (1 - 2e-5)) & (p_ref >= left * (1 - 2e-5)) & (p_ref >= right * (1 - 2e-5))
            must = (p_ref >= thr * (1 + 2e-5)) & (p_ref > left * (1 + 2e-5)) & (p_ref >= right * (1 + 2e-5))
            ok = int(must.sum()) <= count <= int(may.sum()) and bool(np.all(may[fi, ji]))
            note("peaks", 0.0 if ok else 1.0, (N, M, F, Ns))
        out["cases"] += 1
        p.close()
    g = np.random.Generator(np.random.PCG64(19))
    ss = [synth.signal(g, n) for n in BATCH["Ns"]]
    hs = [synth.filters(g, f, m) for f, m in zip(BATCH["F"], BATCH["M"])]
    for per_n in (False, True):
        bp = BatchPlan(BATCH["Ns"], BATCH["M"], BATCH["F"], BATCH["N"], per_n=per_n)
        bp.set_filters([dev(h) for h in hs])
        ys = bp.convolve([dev(s) for s in ss])
        torch.cuda.synchronize()
        out["status"] |= bp.status()
        for b in range(bp.B):
            note("batch", oracle.max_stream_rel_l2(ys[b].cpu().numpy(), oracle.conv(ss[b], hs[b]),
                                                   oracle.stream_scale(ss[b], hs[b], bp.Nout[b])), (per_n, b))
        out["cases"] += 1
        bp.close()
    out["worst"] = worst
    print(json.dumps(out))


if __name__ == "__main__":
    main()
