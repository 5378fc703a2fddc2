"""Run one kernel family on seeded inputs, for profiling with ncu.

    python -m paper_2104_10785_gb300.kernel_case --dtype bf16 --m 40000 --n 20000 --reps 3
    python -m paper_2104_10785_gb300.kernel_case --batched 64 --reps 1

Products: builds A (m x n, N(0,1) values drawn by torch's CUDA generator, stored in the
given dtype) and calls gk_matvec(A, x) and gk_matvec(A, y, trans=True) `reps` times each.
Batched (--batched COUNT): the first COUNT problems of the 512-problem batched recipe
(uneven f32 products of rank 5..64 + 1e-6 noise); runs the learned pipeline's sketch
(gk_sketch_batched) and its batched partial SVD with the committed network's (rank, K)
`reps` times and prints the operator bytes the last solve streamed (products x m x n x 4).
Everything goes through the C ABI; nothing is timed here.
"""
import argparse

import torch

from . import gk


def products(a):
    dt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32, "f64": torch.float64}[a.dtype]
    g = torch.Generator(device="cuda").manual_seed(a.seed)
    A = torch.randn(a.m, a.n, generator=g, device="cuda", dtype=torch.float32).to(dt)
    x = torch.randn(a.n, generator=g, device="cuda", dtype=torch.float64)
    y = torch.randn(a.m, generator=g, device="cuda", dtype=torch.float64)
    for _ in range(a.reps):
        gk.gk_matvec(A, x)
        gk.gk_matvec(A, y, trans=True)


def batched(a):
    import synth

    from . import predictor

    w = synth.WORKLOADS["batched_f32_512_rank5to64"]
    shapes = synth.batched_shapes(512, w["seed"])[: a.batched]
    mats = synth.torch_batched_products(shapes, 1e-6, w["seed"])
    params = predictor.load()
    if params is None:
        raise SystemExit("trained predictor weights are missing")
    for _ in range(a.reps):
        pred = predictor.predict(mats, params)
        out, _, _ = gk.gk_psvd_batched([dict(A=A, k=r, krylov_dim=K, tol=w["tol"], rank_cut=w["eps"])
                                        for A, (r, K) in zip(mats, pred)])
    # the operator bytes the last launch had to stream: every product reads its A once
    alg = sum(o[3]["matvecs"] * A.shape[0] * A.shape[1] * 4 for o, A in zip(out, mats))
    print("algorithmic_bytes_per_launch", alg)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "f16", "f32", "f64"])
    ap.add_argument("--m", type=int, default=40000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--batched", type=int, default=0)
    a = ap.parse_args()
    if a.batched:
        batched(a)
    else:
        products(a)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
