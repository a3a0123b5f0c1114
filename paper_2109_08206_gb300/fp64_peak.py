"""Measured float64 arithmetic rate of the GPU: the denominator for kernels
bound by float64 arithmetic (the FP64 solver, the float64 pair decision and
assembly).

Times a square float64 matrix product (cuBLAS DGEMM through torch.matmul,
2 N^3 flops) as a burst (best of 10 after warm-up) with CUDA events and
prints one JSON line.  Usage: ``python -m paper_2109_08206_gb300.fp64_peak``.
"""
from __future__ import annotations

import json


def measure(n: int = 8192, reps: int = 10) -> dict:
    import torch
    dev = torch.device("cuda")
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = torch.empty(n, n, dtype=torch.float64, device=dev)
    for _ in range(3):
        torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return {"fp64_tflops": 2.0 * n ** 3 / best / 1e12, "n": n, "seconds": best,
            "how": "torch.matmul float64 (cuBLAS DGEMM), 2 N^3 flops, best of "
                   f"{reps} after 3 warm-ups, CUDA events",
            "gpu": torch.cuda.get_device_name(dev), "torch": torch.__version__}


if __name__ == "__main__":
    print(json.dumps(measure()))
