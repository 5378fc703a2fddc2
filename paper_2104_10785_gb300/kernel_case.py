"""Run one product kernel family on a seeded dense operator, for profiling with ncu.

    python -m paper_2104_10785_gb300.kernel_case --dtype bf16 --m 40000 --n 20000 --reps 3

Builds A (m x n, N(0,1) values drawn by torch's CUDA generator, stored in the given
dtype) and calls gk_matvec(A, x) and gk_matvec(A, y, trans=True) `reps` times each,
through the C ABI.  Nothing is timed here: ncu does the measuring.
"""
import argparse

import torch

from . import gk


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f16", "f32", "f64"])
    ap.add_argument("--m", type=int, default=40000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args()
    dt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32, "f64": torch.float64}[a.dtype]
    g = torch.Generator(device="cuda").manual_seed(a.seed)
    A = torch.randn(a.m, a.n, generator=g, device="cuda", dtype=torch.float32).to(dt)
    x = torch.randn(a.n, generator=g, device="cuda", dtype=torch.float64)
    y = torch.randn(a.m, generator=g, device="cuda", dtype=torch.float64)
    for _ in range(a.reps):
        gk.gk_matvec(A, x)
        gk.gk_matvec(A, y, trans=True)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
