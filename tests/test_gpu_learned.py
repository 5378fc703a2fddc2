"""The learned predictor's kernels against the oracle (sketch features, MLP forward,
gradients), training through the library's Adam kernel, and what the trained network
gains over the plain batched pipeline on the same batch."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
import synth

pytestmark = pytest.mark.gpu


def gk():
    import paper_2104_10785_gb300 as m

    return m


def _params(seed=0, scale=0.1):
    g = np.random.default_rng(seed)
    p = g.standard_normal(mlp.N_PARAMS) * scale
    p[mlp.N_TRAINABLE:mlp.N_TRAINABLE + 35] = g.standard_normal(35) * 0.5
    p[mlp.N_TRAINABLE + 35:mlp.N_TRAINABLE + 70] = 1.0 + 0.2 * np.abs(g.standard_normal(35))
    p[mlp.N_TRAINABLE + 70:mlp.N_TRAINABLE + 72] = [2.0, 3.0]
    p[mlp.N_TRAINABLE + 72:] = [0.7, 0.4]
    return p.astype(np.float32)


def test_sketch_features_bf16_tensor_path_match_oracle():
    """bf16 operators take the tensor-pipe sketch (mma.sync bf16 fragments, f32 accumulation) with
    Omega rounded to bf16; the oracle forms the same features in f64 from the same rounded Omega.
    Shapes: ragged row chunks, widths not multiples of 8 or 64 (rows padded to 16-byte strides),
    one wider than a tile row of 64 many times.  Bound as the f32 path's: the f32 sums perturb Y by
    a few 1e-6 of sigma_1."""
    mats, As = [], []
    g = synth.rng(45)
    for i, (m, n) in enumerate([(1000, 300), (129, 61), (700, 8), (300, 1025), (4000, 200)]):
        r = int(g.integers(2, 30))
        A32 = synth.gaussian_product(m, n, r, 1e-3, seed=100 + i, dtype=np.float32)
        bits = synth.to_bf16_bits(A32)
        ldp = (n + 7) // 8 * 8
        T = torch.zeros((m, ldp), dtype=torch.int16)
        T[:, :n] = torch.from_numpy(bits.view(np.int16))
        mats.append(T.cuda().view(torch.bfloat16)[:, :n])
        As.append(synth.bf16_bits_to_f32(bits).astype(np.float64))
    f = gk().gk_sketch_batched(mats, seed=92).cpu().numpy()
    for i, A in enumerate(As):
        fo = mlp.sketch_features(A, 92, omega_bf16=True)
        sg, so = np.exp(f[i, :32].astype(np.float64)), np.exp(fo[:32])
        assert np.all(np.abs(sg - so) <= 2e-5 * so[0] + 1e-5 * so), (i, np.abs(sg - so).max() / so[0])
        np.testing.assert_allclose(f[i, 32:], fo[32:], rtol=1e-6, atol=1e-6)


def test_sketch_features_match_oracle():
    mats, As = [], []
    g = synth.rng(44)
    for i in range(12):
        m = int(g.integers(40, 700))
        n = int(g.integers(20, 300))
        r = int(g.integers(2, 40))
        A = synth.gaussian_product(m, n, r, 1e-3, seed=i, dtype=np.float32)
        As.append(A)
        mats.append(torch.from_numpy(A).cuda())
    f = gk().gk_sketch_batched(mats, seed=91).cpu().numpy()
    for i, A in enumerate(As):
        fo = mlp.sketch_features(A.astype(np.float64), 91)
        # sigma_i(Y): the f32 products perturb Y by ~2^-24 sqrt(n) ||A|| ||Omega||, i.e. an absolute
        # error of a few 1e-6 sigma_1 (Weyl), on top of f32 rounding of each feature
        sg, so = np.exp(f[i, :32].astype(np.float64)), np.exp(fo[:32])
        assert np.all(np.abs(sg - so) <= 2e-5 * so[0] + 1e-5 * so), (i, np.abs(sg - so).max() / so[0])
        np.testing.assert_allclose(f[i, 32:], fo[32:], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("B", [1, 7, 256, 300])
def test_mlp_forward_matches_oracle(B):
    p = _params(1)
    X = np.random.default_rng(B).standard_normal((B, 35)).astype(np.float32)
    out = gk().gk_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-4)
    outb = gk().gk_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), bf16_weights=True)
    np.testing.assert_allclose(outb.cpu().numpy(), ref, rtol=0.05, atol=0.05)  # bf16 weights: 2^-9 relative each


def test_mlp_gradient_matches_oracle():
    p = _params(2)
    g = np.random.default_rng(9)
    X = g.standard_normal((64, 35)).astype(np.float32)
    Y = (g.standard_normal((64, 2)) * 0.5 + [2.0, 3.0]).astype(np.float32)
    grad, loss = gk().gk_mlp_grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    lo, go = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    grad = grad.cpu().numpy()
    scale = np.abs(go).max()
    assert np.abs(grad - go).max() <= 1e-4 * scale


def test_adam_step_matches_oracle():
    """One step of gk_mlp_train (epochs = 1 over one full minibatch: a single Adam update at
    t = t0 + 1) against the oracle's Adam step fed the oracle's own full-batch gradient, with
    nonzero starting moments and t0 = 3 so that both bias corrections and both beta powers
    matter.  Tolerance: the gradients agree to 1e-4 max|g| (the gradient parity bound), and an
    update moves by at most |d update / d g| times that, plus f32 rounding."""
    p = _params(4)
    g = np.random.default_rng(12)
    B = 96
    X = g.standard_normal((B, 35)).astype(np.float32)
    Y = (g.standard_normal((B, 2)) * 0.5 + [2.0, 3.0]).astype(np.float32)
    _, go = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    rms = float(np.sqrt(np.mean(go * go)))
    nt = mlp.N_TRAINABLE
    m0 = (g.standard_normal(nt) * rms).astype(np.float32)
    v0 = (rms * rms * g.uniform(0.5, 2.0, nt)).astype(np.float32)
    t0, lr, b1, b2, eps = 3, 1e-3, 0.9, 0.999, 1e-8
    pd = torch.from_numpy(p.copy()).cuda()
    md = torch.from_numpy(m0.copy()).cuda()
    vd = torch.from_numpy(v0.copy()).cuda()
    gk().gk_mlp_train(pd, md, vd, t0, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), batch=B, epochs=1,
                      lr=lr, seed=5)
    pn, mn, vn = pd.cpu().numpy().astype(np.float64), md.cpu().numpy(), vd.cpu().numpy()
    po, mo, vo = mlp.adam_step(p[:nt].astype(np.float64), m0, v0, go, t0 + 1, lr)
    # the non-trainable tail (standardization) is left alone
    assert np.array_equal(pn[nt:], p[nt:].astype(np.float64))
    t = t0 + 1
    c1, c2 = 1 - b1 ** t, 1 - b2 ** t
    dg = 1e-4 * np.abs(go).max()
    sv = np.sqrt(vo / c2)
    du_dg = lr * np.abs((1 - b1) / c1 / (sv + eps) - (mo / c1) * (1 - b2) * go / (c2 * np.maximum(sv, 1e-30) *
                                                                                 (sv + eps) ** 2))
    upd = p[:nt].astype(np.float64) - po
    assert np.all(np.abs(pn[:nt] - po) <= 1.5 * du_dg * dg + 1e-6 * np.abs(upd) + 2.0**-23 * np.abs(po) + 1e-12)
    assert np.all(np.abs(mn - mo) <= (1 - b1) * dg * 1.01 + 2.0**-23 * np.abs(mo))
    assert np.all(np.abs(vn - vo) <= (1 - b2) * (2 * np.abs(go) * dg + dg * dg) * 1.01 + 2.0**-23 * np.abs(vo))
    # the update itself is far above the tolerance: the test sees the rule, not noise
    assert np.median(np.abs(upd)) > 50 * np.median(1.5 * du_dg * dg)


def test_training_reduces_the_loss():
    g = np.random.default_rng(3)
    X = g.standard_normal((2048, 35)).astype(np.float32)
    W = g.standard_normal((35, 2)) * 0.3
    Y = (np.tanh(X @ W) + [2.0, 3.0]).astype(np.float32)
    from paper_2104_10785_gb300 import predictor

    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    params, losses = predictor.train(Xd, Yd, epochs=30, batch=128, lr=1e-3, seed=1)
    losses = losses.cpu().numpy()
    assert losses[-1] < 0.2 * losses[0], losses
    # the trained network agrees with the oracle's forward pass on its own parameters
    out = gk().gk_mlp_forward(params, Xd[:50]).cpu().numpy()
    ref, _ = mlp.forward(params.cpu().numpy().astype(np.float64), X[:50].astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-4)


def test_batched_rank_cut_returns_the_numerical_rank():
    """k above the rank with rank_cut = eps: the triplets below eps * sigma_1 leave the convergence
    test, `rank` counts the rest, and those equal the oracle's top-r triplets."""
    probs, cases = [], []
    for i in range(16):
        g = synth.rng(300 + i)
        m = int(g.integers(80, 600))
        n = int(g.integers(40, m + 1))
        r = int(g.integers(3, 25))
        A = synth.gaussian_product(m, n, r, 1e-9, seed=400 + i, dtype=np.float64)
        k = min(r + int(g.integers(1, 6)), min(m, n) - 2)
        q1 = synth.start_vector(m, i)
        probs.append(dict(A=torch.from_numpy(A).cuda(), k=k, krylov_dim=min(k + 8, min(m, n)), tol=1e-10,
                          rank_cut=1e-6, start=torch.from_numpy(q1).cuda()))
        cases.append((A, r, q1))
    res, st, info = gk().gk_psvd_batched(probs, max_restarts=100)
    assert st == 0, [x[3] for x in res]
    for (U, S, V, rr), (A, r, q1) in zip(res, cases):
        assert rr["rank"] == r
        op = oracle.Operator.dense(A)
        Uo, So, Vo, io = oracle.psvd(op, r, min(r + 12, min(A.shape)), q1, tol=1e-12, max_restarts=500)
        np.testing.assert_allclose(S.cpu().numpy()[:r], So, rtol=1e-9)
        r1, r2 = oracle.residuals(op, U.cpu().numpy()[:, :r], S.cpu().numpy()[:r], V.cpu().numpy()[:, :r])
        assert max(r1.max(), r2.max()) <= 1.01e-10 * So[0]


def _held_out(count, seed):
    shapes = synth.batched_shapes(count, seed)
    return shapes, synth.torch_batched_products(shapes, 1e-6, seed)


def _check_against_plain(ranks, out, ranks_p, out_p, shapes, mats):
    assert ranks == ranks_p == [s[2] for s in shapes]
    M = gk()
    for (U, S, V, _), (Up, Sp, Vp, _), A in zip(out, out_p, mats):
        np.testing.assert_allclose(S.cpu().numpy(), Sp.cpu().numpy(), rtol=1e-7)
        r1, r2 = M.gk_residuals(A, U, S, V)
        r1p, r2p = M.gk_residuals(A, Up, Sp, Vp)
        # both at the f32-product floor or below the tolerance
        lim = max(2.0 * float(max(r1p.max(), r2p.max())), 1e-8 * float(Sp[0]))
        assert float(max(r1.max(), r2.max())) <= lim


def test_wrong_predictions_cost_only_work():
    """A network with random weights: every wrong rank is caught by the solver's own spectrum and
    re-solved by the plain pipeline, so the results equal the plain ones."""
    from paper_2104_10785_gb300 import predictor

    shapes, mats = _held_out(48, 4242)
    p = torch.from_numpy(_params(5, scale=0.05)).cuda()
    rl, outl, il = predictor.learned_batched(mats, p)
    rp, outp, ip = predictor.plain_batched(mats)
    _check_against_plain(rl, outl, rp, outp, shapes, mats)


def test_trained_predictor_gains_over_plain():
    """The committed network on a held-out batch (a seed outside the training range): the same ranks
    and triplets as the plain pipeline, with fewer products with A and less time."""
    import time

    from paper_2104_10785_gb300 import predictor

    params = predictor.load()
    assert params is not None, "trained weights missing"
    shapes, mats = _held_out(256, 777)
    runs = {}
    for name, fn in (("plain", lambda: predictor.plain_batched(mats)),
                     ("learned", lambda: predictor.learned_batched(mats, params))):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        runs[name] = (time.perf_counter() - t, out)
    tp, (rp, outp, ip) = runs["plain"]
    tl, (rl, outl, il) = runs["learned"]
    _check_against_plain(rl, outl, rp, outp, shapes, mats)
    assert il["fallbacks"] <= 0.05 * len(mats)
    assert il["matvecs"] < 0.75 * ip["matvecs"], (il["matvecs"], ip["matvecs"])
    assert tl < tp, (tl, tp)


def test_krylov_predictor_on_a_held_out_operator():
    """The committed Krylov-dimension network on an operator of its family that it was not trained
    on (sigma_i = i^-1.4, 9000 x 3500, bf16, its own seed): the predicted K is at least the
    measured one-cycle K* and at most 30 above it, and the learned solve converges to the
    tolerance with fewer products than K = 2k."""
    from paper_2104_10785_gb300 import predictor

    params = predictor.load(path=predictor.KRYLOV_PARAMS_FILE)
    assert params is not None, "trained Krylov-dimension weights missing"
    sig = synth.sigma_power(3500, 1.4)
    A32, _, _ = synth.torch_prescribed_spectrum(9000, 3500, sig, 4242)
    A = A32.to(torch.bfloat16)
    kstar = predictor.krylov_targets(A)
    K = predictor.predict_krylov(A, params)
    assert kstar <= K <= kstar + 30, (K, kstar)
    U, S, V, st, info = predictor.learned_psvd(A, params)
    assert st == 0 and info["resid_est_max"] <= predictor.KRYLOV_TOL and info["restarts"] == 0
    U2, S2, V2, st2, info2 = gk().gk_psvd(A, predictor.KRYLOV_K, predictor.KRYLOV_TOL,
                                          krylov_dim=2 * predictor.KRYLOV_K)
    assert info["matvecs"] < info2["matvecs"]
    np.testing.assert_allclose(S.cpu().numpy(), S2.cpu().numpy(), rtol=1e-6)
