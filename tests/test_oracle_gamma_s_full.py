"""Oracle pins for reading A of the gamma_s update (ORC_FLAG_GAMMA_S_FULL).

Under reading A the sparse-code sweep also draws every inactive weight from
its prior, s_ik ~ N(0, 1/gamma_s), and gamma_s ~ Ga(c + N K / 2,
d + sum_all s^2 / 2).  Under the default reading B inactive weights are
integrated out.  Both are valid samplers of the same posterior over (z,
active s, gamma_s).  The pins:

* for the same counters, z and the active s are identical under A and B,
  and the inactive s are exactly zero under B;
* the inactive s under A follow N(0, 1/gamma_s) (Kolmogorov-Smirnov);
* the gamma_s draws under A follow Ga(c + N K / 2, d + sum_all s^2 / 2) for
  a fixed state (Kolmogorov-Smirnov);
* full Gibbs chains (codes, pi, gamma_s, gamma_eps; the dictionary fixed)
  under A and under B on one small patch give the same posterior means of
  gamma_s and of z, within batch-means errors.
"""
import numpy as np
from scipy import stats

import oracle as O

FULL = O.FLAG_GAMMA_S_FULL


def _frame_problem(K, seed, flags):
    rng = np.random.default_rng(seed)
    M, B, S = (2, 90), (2, 3), (2, 3)
    prm = O.params(M, B, S, K, seed=seed, flags=flags)
    N, P = O.num_patches(prm), O.patch_size(prm)
    mask = (rng.random(M) < 0.7).astype(np.uint8)
    D = rng.standard_normal((K, P)) / np.sqrt(P)
    x = (rng.standard_normal(M) * 0.5).astype(np.float32)
    return prm, x, mask, D


def test_full_reading_keeps_z_and_active_s():
    K = 4
    outs = {}
    for flags in (0, FULL):
        prm, x, mask, D = _frame_problem(K, 5, flags)
        st = O.State(prm, D=D, pi=[0.4] * K, gamma_s=2.0, gamma_eps=3.0, t=7)
        for t in range(7, 10):   # a few sweeps, so that codes change on both sides
            st.t = t
            O.zs_sweep(st, x, mask)
        outs[flags] = st
    a, b = outs[FULL], outs[0]
    np.testing.assert_array_equal(a.Z, b.Z)
    on = a.Z.astype(bool)
    np.testing.assert_array_equal(a.S[on], b.S[on])
    assert (b.S[~on] == 0).all()
    assert (a.S[~on] != 0).all()
    assert 0 < on.sum() < on.size


def test_inactive_s_follow_the_prior():
    K, gs = 6, 4.0
    prm, x, mask, D = _frame_problem(K, 9, FULL)
    draws = []
    for t in range(40):
        st = O.State(prm, D=D, pi=[1e-9] * K, gamma_s=gs, gamma_eps=3.0, t=t)
        O.zs_sweep(st, x, mask)
        draws.append(st.S[st.Z == 0])
    v = np.concatenate(draws)
    assert v.size > 5000
    assert stats.kstest(v, stats.norm(scale=1 / np.sqrt(gs)).cdf).pvalue > 1e-3


def test_gamma_s_full_conditional():
    K = 3
    prm, x, mask, D = _frame_problem(K, 33, FULL)
    N = O.num_patches(prm)
    rng = np.random.default_rng(33)
    Z = (rng.random((N, K)) < 0.5).astype(np.uint8)
    Sv = rng.standard_normal((N, K))          # every entry carries an s under reading A
    T = 20000
    gss = np.zeros(T)
    for t in range(T):
        st = O.State(prm, D=D, Z=Z, S=Sv, gamma_eps=1.0, t=t)
        O.hyper(st, x, mask)
        gss[t] = st.gamma_s
    law = stats.gamma(prm.c + 0.5 * N * K, scale=1 / (prm.d + 0.5 * np.sum(Sv ** 2)))
    assert stats.kstest(gss, law.cdf).pvalue > 1e-3
    # reading B on the same state ignores the inactive s
    prm_b = O.params((2, 90), (2, 3), (2, 3), K, seed=33)
    st = O.State(prm_b, D=D, Z=Z, S=Sv * Z, gamma_eps=1.0, t=0)
    s_b = O.hyper(st, x, mask)
    assert np.isclose(s_b[1], np.sum((Sv * Z) ** 2), rtol=1e-13, atol=0)


def _chain_means(flags, T=24000, burn=1000, batches=40):
    M, B, S, K = (3, 3), (3, 3), (1, 1), 2
    prm = O.params(M, B, S, K, a=2.0, b=2.0, c=2.0, d=2.0, e=2.0, f=0.5, seed=17, flags=flags)
    rng = np.random.default_rng(17)
    x = rng.standard_normal(M).astype(np.float32)
    mask = np.ones(M, np.uint8)
    D = rng.standard_normal((K, 9)) / 3.0
    st = O.State(prm, D=D, gamma_s=1.0, gamma_eps=1.0)
    gs, z = [], []
    for t in range(T):
        st.t = t
        O.zs_sweep(st, x, mask)
        O.hyper(st, x, mask)
        if t >= burn:
            gs.append(st.gamma_s)
            z.append(st.Z[0].astype(float))
    gs, z = np.array(gs), np.array(z)

    def mean_se(v):
        bm = v[: len(v) // batches * batches].reshape(batches, -1).mean(axis=1)
        return v.mean(), bm.std(ddof=1) / np.sqrt(batches)

    return mean_se(gs), [mean_se(z[:, k]) for k in range(K)]


def test_readings_sample_the_same_posterior():
    (ga, sa), za = _chain_means(FULL)
    (gb, sb), zb = _chain_means(0)
    assert abs(ga - gb) < 5 * np.hypot(sa, sb), (ga, gb, sa, sb)
    for (ma, ea), (mb, eb) in zip(za, zb):
        assert abs(ma - mb) < 5 * np.hypot(ea, eb) + 1e-3, (ma, mb, ea, eb)
