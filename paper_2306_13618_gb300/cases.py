"""Named single-kernel workloads of the library, timed with CUDA events:

    python -m paper_2306_13618_gb300.cases <case> [--n N] [--reps K]

cases
  direct    Gaussian kernel sum, direct FP32 form, on the 5-component mixture
            (d = 3, eps = 0.02), n = m = N
  nfft      the same with the NFFT fast summation (grid 128^3)
  nfft_reg  Laplace kernel sum (ell = 1/2), regularised NFFT (grid 256^3, p = 4),
            points and weights uniform on [0, 1] (d = 3), n = m = N
  tc        Gaussian kernel sum, d = 64, tensor-core BF16x3 form, n = m = N

Each run does one untimed call, then K timed calls; prints one JSON line with the
milliseconds of each.  Used to time and profile one kernel at a chosen size.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import build, inputs, uotk


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["direct", "nfft", "nfft_reg", "tc"])
    p.add_argument("--n", type=int, default=1 << 17)
    p.add_argument("--reps", type=int, default=2)
    return p.parse_args()


def main():
    a = _args()
    build.build()
    dev = torch.device("cuda", 0)
    if a.case in ("direct", "nfft"):
        W = inputs.gmm3(seed=2000, n=a.n, m=a.n)
        src, w, tgt = (torch.from_numpy(v).to(dev) for v in (W.y, W.b, W.x))
        call = lambda: uotk.kernel_sum(src, w, tgt, W.eps, method=a.case)  # noqa: E731
    elif a.case == "nfft_reg":
        g = inputs.rng(741)
        src, tgt = (torch.from_numpy(g.uniform(0, 1, (a.n, 3)).astype(np.float32)).to(dev)
                    for _ in range(2))
        w = torch.from_numpy(g.uniform(0, 1, a.n).astype(np.float32)).to(dev)
        call = lambda: uotk.kernel_sum(src, w, tgt, 0.5, method="nfft",  # noqa: E731
                                       kernel="laplace")
    else:
        W = inputs.gauss64(n=a.n, m=a.n)
        src, w, tgt = (torch.from_numpy(v).to(dev) for v in (W.y, W.b, W.x))
        call = lambda: uotk.kernel_sum(src, w, tgt, W.eps, method="direct_bf16x3")  # noqa: E731
    call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"case": a.case, "n": a.n, "ms": ms}))


if __name__ == "__main__":
    main()
