"""Host logic of the learned predictor (no GPU): how the network's estimates become the
(rank, Krylov dimension) a batched solve gets, and the Krylov grid of the training targets."""
import math

import numpy as np
import torch

from paper_2104_10785_gb300 import predictor as P


def test_margins_round_the_rank_up_and_keep_room_above_it():
    r, K = P.margins(40.2, 90.7, 784)
    assert r == math.ceil(1.05 * 40.2) + 1 == 44
    assert K == math.ceil(90.7) + 2 + (44 - 40) == 97  # the Krylov estimate moves with the rank margin
    r, K = P.margins(40.0, 30.0, 784)
    assert K == r + 2  # never fewer than two columns beyond the rank


def test_margins_clamp_to_the_operator_and_the_limit():
    assert P.margins(5000.0, 9000.0, 4096) == (P.K_LIMIT - 1, P.K_LIMIT)
    assert P.margins(300.0, 400.0, 256) == (255, 256)
    assert P.margins(0.01, 0.01, 500) == (2, 5)  # K = 1 + 2 + (2 - 0)
    # degenerate shapes still give a valid request: 1 <= r <= K <= min(m, n)
    assert P.margins(5.0, 20.0, 1) == (1, 1)
    assert P.margins(5.0, 20.0, 2) == (1, 2)
    for mn in (1, 2, 3, 7, 128):
        for rf, kf in ((0.0, 0.0), (1e6, 1e6), (3.0, 1.0)):
            r, K = P.margins(rf, kf, mn)
            assert 1 <= r <= K <= min(mn, P.K_LIMIT)


def test_margins_of_a_non_finite_estimate_ask_for_the_whole_range():
    assert P.margins(float("nan"), 20.0, 300) == (299, 300)
    assert P.margins(10.0, float("inf"), 300)[1] == 300


def test_predict_applies_the_margins_per_operator(monkeypatch):
    mats = [torch.empty(784, 256), torch.empty(300, 2000), torch.empty(1, 50)]
    raw = np.array([[math.log(20.0), math.log(40.0)], [math.log(7.5), math.log(30.0)], [0.0, 0.0]], np.float32)
    monkeypatch.setattr(P, "predict_raw", lambda m, p, bf16=True: raw)
    got = P.predict(mats, params=None)
    want = [P.margins(float(np.exp(a)), float(np.exp(b)), min(A.shape)) for A, (a, b) in zip(mats, raw)]
    assert got == want and got[2] == (1, 1)


def test_k_grid_offsets_then_the_fallback():
    """r + 2, 4, 6, 8, 12, 16, 24, 32 (increasing), then 2 r + 16, each capped at min(m, n) and
    kept only if above r and new; the binary search over it takes the last entry when no other
    converges in one cycle."""
    assert P.k_grid(10, 1000) == [12, 14, 16, 18, 22, 26, 34, 42, 36]
    assert P.k_grid(60, 4096) == [62, 64, 66, 68, 72, 76, 84, 92, 136]
    assert P.k_grid(100, 110) == [102, 104, 106, 108, 110]
    assert P.k_grid(3, 4) == [4]
    for r, mn in ((5, 784), (60, 4096), (100, 110), (3, 4), (1, 1)):
        g = P.k_grid(r, mn)
        assert len(set(g)) == len(g) and all(K <= mn for K in g)
        assert all(r < K for K in g) or g == [mn]


def test_learned_batched_judges_each_prediction_and_re_solves_the_short_ones(monkeypatch):
    """A solve is accepted when its spectrum shows a value below the cut (reported rank < k, or
    sigma_{k+1} <= eps sigma_1); otherwise the problem goes to the plain pipeline."""
    mats = [torch.empty(40, 30) for _ in range(3)]
    monkeypatch.setattr(P, "predict", lambda m, p: [(3, 8)] * len(m))

    def fake_psvd_batched(probs, **kw):
        assert all(p["rank_cut"] == 1e-5 and p["k"] == 3 and p["krylov_dim"] == 8 for p in probs)
        rr = [dict(status=0, rank=2, sigma_next=0.5, matvecs=17),    # a value below the cut: rank 2
              dict(status=0, rank=3, sigma_next=1e-9, matvecs=17),   # sigma_4 <= eps sigma_1: rank 3
              dict(status=0, rank=3, sigma_next=1.0, matvecs=17)]    # nothing below: r^ too small
        out = [(torch.ones(40, 3), torch.tensor([10.0, 5.0, 1.0]), torch.ones(30, 3), r) for r in rr]
        info = dict(matvecs=51, sigma_1=torch.tensor([10.0, 10.0, 10.0]), outputs=("U", "S", "V"))
        return out, 0, info

    def fake_plain(ms, eps, tol, autotune=False):
        assert len(ms) == 1
        o = (torch.ones(40, 4), torch.tensor([10.0, 5.0, 1.0, 0.5]), torch.ones(30, 4), dict(status=0))
        return [4], [o], dict(matvecs=40, status=0, matvecs_per_problem=[40])

    monkeypatch.setattr(P.gk, "gk_psvd_batched", fake_psvd_batched)
    monkeypatch.setattr(P, "plain_batched", fake_plain)
    ranks, final, info = P.learned_batched(mats, params=None)
    assert ranks == [2, 3, 4]
    assert [f[1].numel() for f in final] == [2, 3, 4] and final[0][0].shape == (40, 2)
    assert info["fallbacks"] == 1 and info["matvecs"] == 51 + 40
    assert info["matvecs_per_problem"] == [18, 18, 58]  # + one sketch pass each, + the plain re-solve
    assert info["outputs"] is None  # a re-solved problem's triplets are not in the solve's buffers
