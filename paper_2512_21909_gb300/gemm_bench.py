"""Microbenchmark of the contraction kernels through cdcc_dgemm.

    python -m paper_2512_21909_gb300.gemm_bench M N K [ta tb] [modes]

modes: comma list of cdcc_dgemm modes (0 FP64 DFMA, 1-3 split BF16 slices,
12-14 exact slices); default 0,2,14.  Prints wall time and algorithmic
TFLOP/s (2MNK / time) per mode, operands slicing included.
"""
from __future__ import annotations

import sys
import time

import torch

from . import cdcc


def run(M, N, K, ta=0, tb=1, modes=(0, 2, 14), reps=2):
    cdcc.load()
    A = torch.randn((K, M) if ta else (M, K), dtype=torch.float64,
                    device="cuda")
    B = torch.randn((N, K) if tb else (K, N), dtype=torch.float64,
                    device="cuda")
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    out = {}
    for mode in modes:
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cdcc.cdcc_dgemm(ta, tb, M, N, K, 1.0, A, A.shape[1], B,
                            B.shape[1], 0.0, C, N, mode=mode)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        out[mode] = best
        print(f"M{M} N{N} K{K} ta{ta} tb{tb} mode{mode}: {best * 1e3:.2f} ms "
              f"{2.0 * M * N * K / best / 1e12:.2f} TFLOP/s", flush=True)
    return out


if __name__ == "__main__":
    a = sys.argv[1:]
    M, N, K = int(a[0]), int(a[1]), int(a[2])
    ta = int(a[3]) if len(a) > 3 else 0
    tb = int(a[4]) if len(a) > 4 else 1
    modes = tuple(int(x) for x in a[5].split(",")) if len(a) > 5 else \
        (0, 2, 14)
    run(M, N, K, ta, tb, modes)
