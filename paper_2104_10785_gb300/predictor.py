"""Learned rank / Krylov-dimension predictor: training orchestration and thin wrappers.

The inference pipelines (the sketch, the network, the margins, the judge and the plain
fallback) run inside libgk.so behind the C ABI (gk_predictor_load, opts->predictor in gk_psvd
and gk_psvd_batched); this module trains the weights with the library's own kernels
(forward/backward/Adam) and wraps those calls.

Targets, measured by the plain method itself on each training matrix:
  r  = the rank gk_numrank_batched (Algorithm 3) returns at eps;
  K* = the smallest Krylov dimension in r + {2, 4, 6, 8, 12, 16, 24, 32} (then 2r + 16)
       at which gk_psvd_batched(k = r, K) converges in ONE cycle at tol (found by a
       per-problem binary search over that grid; the largest entry if none does).
The network maps the 35 sketch features to (log r, log K*).

Pipelines on a batch of dense device operators:
  plain:   gk_numrank_batched -> r; gk_psvd_batched(k = r, default K).
  learned: sketch + network -> (r^, K^), r^ rounded up with a safety margin;
           gk_psvd_batched(k = r^, K = K^, rank_cut = eps), the restart loop covering a
           Krylov dimension that was too small.  The solver's own spectrum judges r^: the
           triplets below eps * sigma_1 are left out of the convergence test and dropped,
           so an over-estimate costs a little work; if no Ritz value of the last projected
           matrix fell below the cut (every theta_i, i <= r^ + 1, above eps * sigma_1) the
           rank was under-estimated and that problem is re-solved by the plain pipeline.
"""
from __future__ import annotations

import math
import os

import numpy as np
import torch

from . import gk

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS_FILE = os.path.join(HERE, "predictor_params.f32")
KRYLOV_PARAMS_FILE = os.path.join(HERE, "predictor_krylov_params.f32")
SKETCH_SEED = 0x5E7C4
K_OFFSETS = (2, 4, 6, 8, 12, 16, 24, 32)
RANK_MARGIN = (1.05, 1)  # r^ = ceil(1.05 * exp(prediction)) + 1: an under-estimate costs a re-solve
K_MARGIN = 2  # added to the predicted Krylov dimension
K_LIMIT = 500


def k_grid(r, mn):
    g = [min(r + o, mn) for o in K_OFFSETS] + [min(2 * r + 16, mn)]
    out = []
    for v in g:
        if v > r and v not in out:
            out.append(v)
    return out or [mn]


def targets(mats, eps=1e-5, tol=1e-8, seed=None):
    """(rank, K*) per operator, measured with the batched solvers."""
    res, st, _ = gk.gk_numrank_batched([dict(A=A, eps=eps, kmax=min(min(A.shape), 160)) for A in mats], seed=seed)
    ranks = [max(1, r[0]) for r in res]
    grids = [k_grid(r, min(A.shape)) for r, A in zip(ranks, mats)]
    lo = [0] * len(mats)
    hi = [len(g) - 1 for g in grids]
    while any(l < h for l, h in zip(lo, hi)):
        idx = [i for i in range(len(mats)) if lo[i] < hi[i]]
        probs = []
        for i in idx:
            mid = (lo[i] + hi[i]) // 2
            probs.append(dict(A=mats[i], k=ranks[i], krylov_dim=grids[i][mid], tol=tol))
        out, _, _ = gk.gk_psvd_batched(probs, max_restarts=0, seed=seed, check=False)
        for i, o in zip(idx, out):
            mid = (lo[i] + hi[i]) // 2
            if o[3]["status"] == gk.GK_OK:
                hi[i] = mid
            else:
                lo[i] = mid + 1
    kstar = [g[h] for g, h in zip(grids, hi)]
    return ranks, kstar


def dataset(n_total, seed, batch=512, eps=1e-5, tol=1e-8, log=None):
    """Features and targets of n_total seeded training operators (recipe of the batched workload)."""
    import synth

    X, Y = [], []
    done = 0
    b = 0
    while done < n_total:
        cnt = min(batch, n_total - done)
        shapes = synth.batched_shapes(cnt, seed + b)
        mats = synth.torch_batched_products(shapes, 1e-6, seed + b, fast=True)
        feats = gk.gk_sketch_batched(mats, SKETCH_SEED)
        r, k = targets(mats, eps, tol, seed=seed + b)
        X.append(feats)
        Y.append(torch.tensor(np.log(np.stack([r, k], axis=1)), dtype=torch.float32, device=feats.device))
        done += cnt
        b += 1
        del mats
        if log:
            log(f"dataset {done}/{n_total}")
    return torch.cat(X), torch.cat(Y)


def init_params(X, Y, seed=0):
    """Seeded initial parameters (scaled normal weights, zero biases) plus the
    standardization statistics of the training features and targets."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    F, H = gk.GK_FEATURES, 256

    def w(o, i):
        return torch.randn(o, i, generator=g) * math.sqrt(2.0 / i)

    parts = [w(H, F).ravel(), torch.zeros(H), w(H, H).ravel(), torch.zeros(H), w(2, H).ravel() * 0.5, torch.zeros(2)]
    xmu = X.mean(0).cpu()
    xsd = X.std(0).cpu().clamp_min(1e-3)
    ymu = Y.mean(0).cpu()
    ysd = Y.std(0).cpu().clamp_min(1e-3)
    p = torch.cat(parts + [xmu, xsd, ymu, ysd]).to(torch.float32)
    assert p.numel() == gk.GK_MLP_PARAMS
    return p.to(X.device)


def train(X, Y, epochs=200, batch=256, lr=1e-3, seed=0):
    params = init_params(X, Y, seed)
    m = torch.zeros(gk.GK_MLP_TRAINABLE, dtype=torch.float32, device=X.device)
    v = torch.zeros_like(m)
    losses = gk.gk_mlp_train(params, m, v, 0, X, Y, batch=batch, epochs=epochs, lr=lr, seed=seed)
    return params, losses


def save(params, path=PARAMS_FILE):
    params.detach().cpu().numpy().astype(np.float32).tofile(path)


def load(device="cuda", path=PARAMS_FILE):
    if not os.path.exists(path):
        return None
    a = np.fromfile(path, dtype=np.float32)
    if a.size != gk.GK_MLP_PARAMS:
        return None
    return torch.from_numpy(a).to(device)


def handle(params):
    """The library-side predictor (gk.Predictor, gk_predictor_load) for a parameter tensor, kept on
    the tensor itself and reloaded when the tensor has been modified in place since (its version
    counter moved); a Predictor is returned as is."""
    if isinstance(params, gk.Predictor):
        return params
    cached = getattr(params, "_gk_predictor", None)
    if cached is not None and cached[0] == params._version:
        return cached[1]
    h = gk.Predictor(params)
    params._gk_predictor = (params._version, h)
    return h


def predict_raw(mats, params, bf16=True):
    """The network's de-standardized outputs (log r, log K) per operator (host array): the
    library's sketch and bf16-weight forward pass (gk_predictor_predict)."""
    if bf16:
        return handle(params).predict(mats)
    feats = gk.gk_sketch_batched(mats, SKETCH_SEED)
    return gk.gk_mlp_forward(params, feats, bf16_weights=False).cpu().numpy()


def margins(rf, kf, mn, cap=None):
    """(r^, K^) from the network's rank and Krylov estimates (rf, kf) for an operator with
    min(m, n) = mn -- the rule the library's learned pipeline applies (gk_psvd_batched with a
    predictor): r^ = ceil(1.05 rf) + 1 and K^ = ceil(kf) + 2 shifted by the same margin, clamped
    to 1 <= r^ <= min(cap, K^) and K^ <= min(mn, K_LIMIT) with K^ >= r^ + 2 where there is room;
    a non-finite estimate asks for the whole range."""
    lim = min(mn, K_LIMIT)
    if not math.isfinite(rf):
        rf = float(lim)
    if not math.isfinite(kf):
        kf = float(lim)
    ri = int(min(max(1, math.ceil(RANK_MARGIN[0] * rf) + RANK_MARGIN[1]), max(1, lim - 1)))
    if cap is not None:
        ri = min(ri, cap)
    Ki = int(math.ceil(kf)) + K_MARGIN + (ri - int(round(rf)))
    Ki = int(min(max(Ki, ri + 2), lim))
    return ri, max(Ki, ri)


def predict(mats, params, bf16=True):
    """(r^, K^) per operator: the rank rounded up with the safety margin, K^ >= r^ + 2."""
    out = predict_raw(mats, params, bf16)
    with np.errstate(over="ignore", invalid="ignore"):
        rc = np.exp(np.clip(out[:, 0], -20.0, 20.0))
        kc = np.exp(np.clip(out[:, 1], -20.0, 20.0))
    return [margins(float(rf), float(kf), min(A.shape)) for A, rf, kf in zip(mats, rc, kc)]


def plain_batched(mats, eps=1e-5, tol=1e-8, autotune=True):
    """Algorithm 3 for the rank, then the top-r partial SVD with the default Krylov dimension
    (cluster sizes autotuned per batch signature)."""
    res, st1, info1 = gk.gk_numrank_batched([dict(A=A, eps=eps, kmax=min(min(A.shape), 160)) for A in mats],
                                            autotune=autotune)
    ranks = [max(1, r[0]) for r in res]
    out, st, info2 = gk.gk_psvd_batched([dict(A=A, k=r, tol=tol) for A, r in zip(mats, ranks)], autotune=autotune)
    per = [a[2]["matvecs"] + b[3]["matvecs"] for a, b in zip(res, out)]
    return ranks, out, dict(matvecs=info1["matvecs"] + info2["matvecs"], status=min(st1, st) if min(st1, st) < 0
                            else max(st1, st), matvecs_per_problem=per)


def learned_batched(mats, params, eps=1e-5, tol=1e-8, max_restarts=200, autotune=True, capacity=80):
    """The library's learned pipeline (gk_psvd_batched with a predictor): predicted (rank, K), one
    batched partial SVD with the rank cut, each problem judged by its own spectrum, the rejected ones
    re-solved by the plain pipeline.  `capacity` = output columns per problem."""
    h = handle(params)
    probs = [dict(A=A, k=min(capacity, min(A.shape)), tol=tol, rank_cut=eps) for A in mats]
    out, st, info = gk.gk_psvd_batched(probs, max_restarts=max_restarts, autotune=autotune, predictor=h)
    ranks = [max(1, rr["rank"]) for (_, _, _, rr) in out]
    final = [(U[:, :r], S[:r], V[:, :r], rr) for (U, S, V, rr), r in zip(out, ranks)]
    # every problem's triplets sit in the call's three output buffers (each problem's capacity
    # columns back to back): a caller can move them to the host in three copies
    return ranks, final, dict(matvecs=info["matvecs"], fallbacks=info["fallbacks"], status=st,
                              matvecs_per_problem=[rr["matvecs"] for (_, _, _, rr) in out],
                              outputs=info["outputs"])


def main(argv=None):
    """Regenerate the committed weights: seeded training operators (the batched workload's recipe),
    targets measured by the batched solvers, Adam training through the library's kernels."""
    import argparse
    import time

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=20480)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=PARAMS_FILE)
    a = ap.parse_args(argv)
    t0 = time.time()
    X, Y = dataset(a.count, a.seed, log=lambda s: print(s, flush=True))
    t1 = time.time()
    params, losses = train(X, Y, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    losses = losses.cpu().numpy()
    save(params, a.out)
    print(f"dataset {t1 - t0:.1f} s, training {time.time() - t1:.1f} s, loss {losses[0]:.3g} -> {losses[-1]:.3g}")




# ---------------------------------------------------------------------------
# Krylov dimension of a single large partial SVD (the bf16 precision form)
# ---------------------------------------------------------------------------
# The same network, trained on another family: dense operators A = U diag(i^-e) V^T stored
# in bf16, e ~ U[1.1, 2.0], sizes between 4000 x 2000 and 20000 x 8000, top k = 100 at tol
# 1e-8.  Targets: (log k, log K*) with K* the smallest Krylov dimension in k + {10, 20, ...,
# 140} at which the partial SVD converges in one cycle (binary search over one-cycle solves).
# For this family K* depends on the decay of the spectrum, not on the sizes, so the sketch
# features carry it; the plain restart loop covers a dimension that is too small.
KRYLOV_K = 100
KRYLOV_TOL = 1e-8
KRYLOV_GRID = tuple(KRYLOV_K + d for d in range(10, 150, 10))


def krylov_targets(A, k=KRYLOV_K, tol=KRYLOV_TOL):
    lo, hi = 0, len(KRYLOV_GRID) - 1
    while lo < hi:
        mid = (lo + hi) // 2
        st = gk.gk_psvd(A, k, tol, krylov_dim=KRYLOV_GRID[mid], max_restarts=0, check=False)[3]
        if st == gk.GK_OK:
            hi = mid
        else:
            lo = mid + 1
    return KRYLOV_GRID[hi]


def krylov_dataset(count, seed, log=None):
    """Features and targets of `count` seeded operators of the bf16 power-law family."""
    import synth

    g = np.random.default_rng(seed)
    X, Y = [], []
    for i in range(count):
        e = float(g.uniform(1.1, 2.0))
        m = int(np.exp(g.uniform(np.log(4000), np.log(20000))))
        n = int(np.exp(g.uniform(np.log(2000), np.log(min(m, 8000)))))
        sig = synth.sigma_power(n, e)
        A32, _, _ = synth.torch_prescribed_spectrum(m, n, sig, seed * 1000 + i)
        A = A32.to(torch.bfloat16)
        del A32
        feats = gk.gk_sketch_batched([A], SKETCH_SEED)
        ks = krylov_targets(A)
        X.append(feats)
        Y.append(torch.tensor([[math.log(KRYLOV_K), math.log(ks)]], dtype=torch.float32, device=feats.device))
        del A
        torch.cuda.empty_cache()
        if log:
            log(f"krylov dataset {i + 1}/{count}: e={e:.2f} {m}x{n} K*={ks}")
    return torch.cat(X), torch.cat(Y)


def predict_krylov(A, params, k=KRYLOV_K, margin=2, bf16=True):
    """Krylov dimension for the top-k partial SVD of A from its sketch features (the rule gk_psvd
    applies with a predictor: ceil(exp(out_K)) + 2 within [k + 2, min(m, n, 500)])."""
    out = predict_raw([A], params, bf16)[0]
    K = int(math.ceil(math.exp(min(max(float(out[1]), 0.0), 20.0)))) + margin
    return int(min(max(K, k + 2), min(A.shape), K_LIMIT))


def learned_psvd(A, params, k=KRYLOV_K, tol=KRYLOV_TOL, out=None, **kw):
    """gk_psvd with the predictor's Krylov dimension, through the C ABI (the library sketches the
    operator; a host operator is staged by the library itself).  `out`: host tensors (U k x m, S k,
    V k x n) for a host operator's results."""
    U, S, V, st, info = gk.gk_psvd(A, k, tol, predictor=handle(params), out=out, **kw)
    info["krylov_dim"] = info["kprime"]
    return U, S, V, st, info


def main_krylov(argv=None):
    import argparse
    import time

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=240)
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--out", default=KRYLOV_PARAMS_FILE)
    a = ap.parse_args(argv)
    t0 = time.time()
    X, Y = krylov_dataset(a.count, a.seed, log=lambda s: print(s, flush=True))
    t1 = time.time()
    params, losses = train(X, Y, epochs=a.epochs, batch=32, lr=1e-3, seed=a.seed)
    losses = losses.cpu().numpy()
    save(params, a.out)
    print(f"dataset {t1 - t0:.1f} s, training {time.time() - t1:.1f} s, loss {losses[0]:.3g} -> {losses[-1]:.3g}")


if __name__ == "__main__":
    import sys

    if len(sys.argv) > 1 and sys.argv[1] == "krylov":
        main_krylov(sys.argv[2:])
    else:
        main()
