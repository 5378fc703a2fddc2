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


def test_library_margins_follow_the_stated_rule():
    """The library's (r^, K^) rule (gk_predictor_margins, host-only): hand-worked cases and the
    module's restatement on a grid, including the capacity clamp and non-finite estimates."""
    import ctypes as C

    from paper_2104_10785_gb300 import gk

    def lib_margins(rf, kf, mn, cap):
        r, K = C.c_int(), C.c_int()
        assert gk.lib().gk_predictor_margins(rf, kf, mn, cap, C.byref(r), C.byref(K)) == 0
        return r.value, K.value

    # rf = 20: r^ = ceil(21) + 1 = 22; kf = 40.3: K^ = 41 + 2 + (22 - 20) = 45
    assert lib_margins(20.0, 40.3, 1000, 80) == (22, 45)
    # capacity 10 clamps r^, and K^ follows it: 41 + 2 + (10 - 20) = 33
    assert lib_margins(20.0, 40.3, 1000, 10) == (10, 33)
    # K^ at least r^ + 2; a small operator caps both (min(m, n) = 12: r^ <= 11, K^ <= 12)
    assert lib_margins(30.0, 5.0, 12, 80) == (11, 12)
    # non-finite estimates ask for the whole range min(mn, 500)
    assert lib_margins(float("inf"), float("nan"), 2000, 600) == (499, 500)
    for rf in (0.3, 1.0, 4.7, 17.2, 63.9, 120.0):
        for kf in (2.0, 20.4, 77.7, 140.2, 700.0):
            for mn, cap in ((256, 80), (3000, 80), (64, 30), (5000, 600)):
                assert lib_margins(rf, kf, mn, cap) == P.margins(rf, kf, mn, cap), (rf, kf, mn, cap)
