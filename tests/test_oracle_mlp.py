"""Pins of the oracle's learned light-subspace proposal (oracle/or_mlp.c).

Each check comes from the mathematics, not from the code under test:
bf16 rounding against IEEE round-to-nearest-even, the backward pass against
central finite differences of the forward pass, the forward pass against a
permutation network whose outputs are known, the sampler against the
probabilities it reports (the property the unbiasedness of the connection
estimate rests on), the cross-entropy gradient at its closed-form stationary
point, and Adam's first step in closed form.
"""

import math

import numpy as np
import pytest

import oracle as O

K, KT = 12, 5
NP = O.mlp_nparams(K, KT)
OFF_W2, OFF_B2, OFF_W3 = 1024, 1024 + 4096, 1024 + 4096 + 64
OFF_B3 = OFF_W3 + 64 * K
OFF_E = OFF_B3 + K


def test_bf16_round_to_nearest_even():
    # bf16 keeps 8 significant bits: the spacing above 1 is 2^-7
    assert O.bf16(1.0) == 1.0
    assert O.bf16(1 + 2 ** -8) == 1.0                    # tie -> even (1.0)
    assert O.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6        # tie between 1+2^-7 (odd) and 1+2^-6 (even)
    assert O.bf16(1 + 3 * 2 ** -9) == 1 + 2 ** -7        # above the midpoint
    assert O.bf16(-(1 + 2 ** -9)) == -1.0
    assert O.bf16(65504.0) == 65536.0                   # 0x477FE000: low half above the midpoint
    assert O.bf16(2.0 ** -130) == 2.0 ** -130            # subnormal exactly representable


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    raw = rng.uniform(-1, 1, (n, 10))
    T = rng.integers(0, KT, n).astype(np.int32)
    S = rng.integers(0, K, n).astype(np.int32)
    wt = rng.uniform(0.1, 3.0, n)
    return raw, T, S, wt


def test_backward_matches_central_differences():
    w = O.mlp_init(K, KT, seed=3)
    w[OFF_B2:OFF_B2 + 64] = np.random.default_rng(4).uniform(-0.2, 0.2, 64)
    w[OFF_B3:OFF_B3 + K] = np.random.default_rng(5).uniform(-0.5, 0.5, K)
    raw, T, S, wt = _batch(7, 6)
    loss, g = O.mlp_loss_grad(w, K, KT, raw, T, S, wt)
    h = 1e-6
    num = np.zeros(NP)
    for i in range(NP):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num[i] = (O.mlp_loss_grad(wp, K, KT, raw, T, S, wt)[0] - O.mlp_loss_grad(wm, K, KT, raw, T, S, wt)[0]) / (2 * h)
    # every block of parameters receives gradient, and all agree
    for lo, hi in ((0, OFF_W2), (OFF_W2, OFF_B2), (OFF_B2, OFF_W3), (OFF_W3, OFF_B3), (OFF_B3, OFF_E), (OFF_E, NP)):
        assert np.abs(g[lo:hi]).max() > 0
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_forward_of_a_permutation_network():
    """W1 selects input pi1(i), W2 permutes hidden units by pi2, W3 reads hidden
    unit pi3(k): with inputs >= 0 every ReLU passes and z_k is a known input
    plus b3_k. A transposed weight matrix would read the wrong inputs."""
    rng = np.random.default_rng(7)
    pi1, pi2, pi3 = rng.permutation(10), rng.permutation(10), rng.permutation(10)
    w = np.zeros(NP)
    for i in range(10):
        w[i * 16 + pi1[i]] = 1.0
        w[OFF_W2 + i * 64 + pi2[i]] = 1.0
    for k in range(10):
        w[OFF_W3 + k * 64 + pi3[k]] = 1.0
    w[OFF_B3:OFF_B3 + K] = 0.01 * np.arange(K)
    raw = rng.uniform(0, 1, (3, 10))
    T = np.zeros(3, np.int32)
    z = O.mlp_logits(w, K, KT, raw, T)
    for k in range(10):
        np.testing.assert_allclose(z[:, k], raw[:, pi1[pi2[pi3[k]]]] + 0.01 * k, rtol=0, atol=1e-15)
    np.testing.assert_allclose(z[:, 10:], 0.01 * np.arange(10, K) + 0 * z[:, 10:], atol=1e-15)
    # the embedding and the bias input reach the first layer through x[10..14]
    w2 = w.copy()
    w2[0 * 16 + pi1[0]] = 0.0
    w2[0 * 16 + 10] = 1.0          # hidden 0 <- E[T][0]
    w2[1 * 16 + pi1[1]] = 0.0
    w2[1 * 16 + 14] = 0.25         # hidden 1 <- bias input 1
    w2[OFF_E + 4 * 2 + 0] = 0.375  # E[2][0]
    z2 = O.mlp_logits(w2, K, KT, raw, np.full(3, 2, np.int32))
    k0 = int(np.where(pi2[pi3] == 0)[0][0])
    k1 = int(np.where(pi2[pi3] == 1)[0][0])
    np.testing.assert_allclose(z2[:, k0], 0.375 + 0.01 * k0, atol=1e-15)
    np.testing.assert_allclose(z2[:, k1], 0.25 + 0.01 * k1, atol=1e-15)


def _select_all(w, raw, T, g, start, n):
    """stratified uniforms over [0,1): counts per subspace and reported Q"""
    counts = np.zeros(K)
    Qs = {}
    for i in range(n):
        S, Q = O.mlp_select(w, K, raw, T, g, start, (i + 0.5) / n)
        counts[S] += 1
        Qs.setdefault(S, Q)
        assert abs(Qs[S] - Q) < 1e-15
    return counts / n, Qs


def test_sampler_frequencies_equal_reported_probabilities():
    """For any weights, the subspace drawn with a uniform u has probability
    equal to the Q(S) returned with it, Q sums to one over the occupied
    subspaces, and Q >= eps * gamma (the table's defensive share)."""
    w = O.mlp_init(K, KT, seed=11)
    w[OFF_W3:OFF_B3] *= 40.0   # a peaked softmax
    rng = np.random.default_rng(12)
    g = rng.uniform(0.05, 1.0, K).astype(np.float32)
    counts = np.array([3, 0, 1, 5, 0, 2, 2, 0, 1, 4, 1, 1])   # subspaces 1, 4, 7 empty
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    raw = rng.uniform(-1, 1, 10)
    n = 40000
    freq, Qs = _select_all(w, raw, 3, g, start, n)
    occ = counts > 0
    assert freq[~occ].sum() == 0
    Q = np.array([Qs.get(k, 0.0) for k in range(K)])
    assert abs(Q[occ].sum() - 1.0) < 1e-12
    np.testing.assert_allclose(freq[occ], Q[occ], atol=2.5 / n)
    gam = g[occ] / g[occ].sum()
    assert np.all(Q[occ] >= 0.1 * gam - 1e-12)


def test_softmax_part_reduces_to_the_table_when_logits_are_log_gamma():
    """W3 = 0 and b3 = log gamma make the network's softmax equal the table
    row over the occupied subspaces, so Q(S) = gamma(S) / Z exactly."""
    w = O.mlp_init(K, KT, seed=2)
    g = np.random.default_rng(3).uniform(0.1, 1.0, K).astype(np.float32)
    w[OFF_W3:OFF_B3] = 0.0
    w[OFF_B3:OFF_B3 + K] = np.log(g.astype(np.float64))
    counts = np.array([1, 2, 0, 1, 1, 0, 3, 1, 1, 0, 2, 1])
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    occ = counts > 0
    for u in (0.01, 0.05, 0.2, 0.5, 0.77, 0.999):
        S, Q = O.mlp_select(w, K, np.zeros(10), 0, g, start, u)
        assert occ[S]
        assert abs(Q - g[S] / g[occ].sum()) < 1e-7   # g is float32; the bf16 b3 rounding is below that here
    # and the sampled S follows the table's CDF in the softmax branch
    cdf = np.cumsum(np.where(occ, g, 0)) / g[occ].sum()
    for u in (0.2, 0.5, 0.77):
        S, _ = O.mlp_select(w, K, np.zeros(10), 0, g, start, u)
        v = (u - 0.1) / 0.9
        assert S == int(np.searchsorted(cdf, v, side="right"))


def test_cross_entropy_gradient_vanishes_at_the_weighted_target():
    """With W3 = 0 the logits are b3 for every row; the loss is minimal where
    softmax(b3) equals the w-weighted frequencies of the targets S_b, and the
    b3 gradient there is zero; elsewhere it is (sum w / n) (p - target)."""
    w = O.mlp_init(K, KT, seed=5)
    w[OFF_W3:OFF_B3] = 0.0
    raw, T, S, wt = _batch(50, 9)
    tgt = np.bincount(S, weights=wt, minlength=K) / wt.sum()
    assert np.all(tgt > 0)
    w[OFF_B3:OFF_B3 + K] = np.log(tgt)
    _, g = O.mlp_loss_grad(w, K, KT, raw, T, S, wt)
    np.testing.assert_allclose(g[OFF_B3:OFF_B3 + K], 0.0, atol=1e-13)
    b3 = np.random.default_rng(1).normal(0, 1, K)
    w[OFF_B3:OFF_B3 + K] = b3
    _, g = O.mlp_loss_grad(w, K, KT, raw, T, S, wt)
    p = np.exp(b3 - b3.max())
    p /= p.sum()
    np.testing.assert_allclose(g[OFF_B3:OFF_B3 + K], wt.sum() / len(wt) * (p - tgt), atol=1e-13)


def test_adam_first_step_is_sign_like():
    """From zero moments the bias-corrected ratio m/sqrt(v) is g/|g|: the
    first step moves each weight by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    w0 = rng.normal(0, 1, 100)
    g = rng.normal(0, 1e-3, 100)
    w1, m1, m2 = O.mlp_adam(w0, g, np.zeros(100), np.zeros(100), 1, lr=0.01)
    np.testing.assert_allclose(w1, w0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(m2, 0.001 * g * g, rtol=1e-12)
