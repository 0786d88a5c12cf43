"""Parity cases run against the bounds-checked build of the library (built
with OLS_CHECK=1 and selected through OLS_LIBRARY): every global access of
the forward, tensor-core and adjoint kernels is checked against its buffer,
and a failed check sets bit 2 of the plan's status word instead of
accessing memory.  Run as ``python -m tests.checked_cases`` by
tests/test_checked_gpu.py; prints one JSON line."""
import json
import os

import numpy as np
import torch

import oracle
import synth
from paper_1910_01972_gb300 import Plan, _native

FWD = [  # (N, M, F, Ns): every segment length, ragged tails, the degenerate sizes
    (256, 33, 3, 20_001), (512, 64, 2, 65_536), (1024, 129, 4, 30_000), (2048, 257, 3, 60_001),
    (4096, 512, 2, 100_000), (8192, 1025, 2, 90_000), (1024, 129, 2, 129), (1024, 100, 2, 900),
    (512, 1, 2, 3_000), (4096, 4096, 1, 9_000), (512, 257, 3, 7_000)]
TC = [(4096, 512, 3, 60_000), (256, 33, 2, 20_001), (2048, 257, 3, 9_001)]
BWD = [(1024, 129, 4, 30_000), (256, 33, 3, 5_000), (2048, 257, 2, 20_001), (1024, 129, 3, 129)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def main():
    out = {"library": os.path.basename(_native.LIB_PATH), "cases": 0, "status": 0, "worst": {}}
    worst = {"fwd": 0.0, "tc": 0.0, "ds": 0.0, "dh": 0.0}
    for N, M, F, Ns in FWD:
        g = np.random.Generator(np.random.PCG64(N + M + F))
        s, h = synth.signal(g, Ns), synth.filters(g, F, M)
        p = Plan(M, F, N)
        p.set_filters(dev(h))
        y = p.convolve(dev(s)).cpu().numpy()
        out["status"] |= p.status()
        worst["fwd"] = max(worst["fwd"], oracle.max_stream_rel_l2(y, oracle.conv(s, h)))
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
        worst["tc"] = max(worst["tc"], oracle.max_stream_rel_l2(y.cpu().numpy(), oracle.conv(s, h)))
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
        worst["ds"] = max(worst["ds"], oracle.rel_l2(ds.cpu().numpy(), ds_ref))
        worst["dh"] = max(worst["dh"], oracle.max_stream_rel_l2(dh.cpu().numpy(), dh_ref))
        out["cases"] += 1
        p.close()
    out["worst"] = worst
    print(json.dumps(out))


if __name__ == "__main__":
    main()
