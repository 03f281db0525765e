"""Pins for the oracle's Gibbs conditionals, each against an independent route.

* z_ik with s_ik integrated out, and s_ik | z_ik = 1: numerical quadrature of
  the joint density (scipy.integrate.quad) on a single patch with one atom.
* The whole sparse-code sweep: the z-vector frequencies of a long chain equal
  the exact posterior enumerated over all 2^K states, with s integrated out in
  closed form as x_Omega | z ~ N(0, D_z D_z^T / gamma_s + I / gamma_eps)
  (scipy.stats.multivariate_normal).
* d_kp in atom order: the draws, standardised by the ridge least-squares
  posterior (numpy.linalg.lstsq / inv on the prior-augmented system) given the
  other atom's current value, are standard normal.
* pi_k, gamma_s, gamma_eps: the draws follow the conjugate Beta / Gamma laws
  (scipy.stats) whose parameters come from sufficient statistics computed by
  dense numpy algebra.
"""
import itertools

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O


def _single_patch_problem(K, seed, P_side=3, frac_obs=0.67):
    rng = np.random.default_rng(seed)
    M = (P_side, P_side)
    prm = O.params(M, M, (1, 1), K, seed=seed)
    P = P_side * P_side
    mask = np.zeros(M, np.uint8)
    obs = rng.permutation(P)[: int(round(frac_obs * P))]
    mask.reshape(-1)[obs] = 1
    D = rng.standard_normal((K, P)) / np.sqrt(P) * 2.0
    x = (D.T @ (rng.standard_normal(K) * (rng.random(K) < 0.5))).astype(np.float32).reshape(M)
    x += (0.2 * rng.standard_normal(M)).astype(np.float32)
    return prm, x.astype(np.float32), mask, D


def test_z_and_s_conditionals_match_quadrature():
    prm, x, mask, D = _single_patch_problem(1, seed=6)
    pi0, gs, ge = 0.3, 2.0, 6.0
    om = mask.reshape(-1).astype(bool)
    xo = x.reshape(-1)[om].astype(np.float64)
    do = D[0][om]

    def loglik(s):
        r = xo - do * s
        return -0.5 * ge * np.dot(r, r)

    base = loglik(0.0)

    def f1(s):  # joint density of (z = 1, s) up to the factor shared with z = 0
        return np.exp(loglik(s) - base) * stats.norm(0, 1 / np.sqrt(gs)).pdf(s)

    lim = 30.0
    A1 = pi0 * integrate.quad(f1, -lim, lim, limit=200)[0]
    A0 = 1 - pi0
    p1 = A1 / (A1 + A0)
    m1 = integrate.quad(lambda s: s * f1(s), -lim, lim, limit=200)[0] / (A1 / pi0)
    v1 = integrate.quad(lambda s: (s - m1) ** 2 * f1(s), -lim, lim, limit=200)[0] / (A1 / pi0)
    assert 0.15 < p1 < 0.85

    st = O.State(prm, D=D, pi=[pi0], gamma_s=gs, gamma_eps=ge)
    T = 40000
    zs, ss = np.zeros(T), np.zeros(T)
    for t in range(T):
        st.t = t
        O.zs_sweep(st, x, mask)
        zs[t], ss[t] = st.Z[0, 0], st.S[0, 0]
    assert abs(zs.mean() - p1) < 5 * np.sqrt(p1 * (1 - p1) / T)
    act = ss[zs == 1]
    assert abs(act.mean() - m1) < 5 * np.sqrt(v1 / len(act))
    assert abs(act.var() / v1 - 1) < 5 * np.sqrt(2.0 / len(act))
    assert np.all(ss[zs == 0] == 0)


def test_sweep_chain_matches_exact_z_posterior():
    K = 3
    prm, x, mask, D = _single_patch_problem(K, seed=11)
    pi = np.array([0.35, 0.5, 0.2])
    gs, ge = 1.5, 8.0
    om = mask.reshape(-1).astype(bool)
    xo = x.reshape(-1)[om].astype(np.float64)
    Do = D[:, om]
    states = list(itertools.product([0, 1], repeat=K))
    logp = []
    for z in states:
        zz = np.array(z, bool)
        cov = Do[zz].T @ Do[zz] / gs + np.eye(om.sum()) / ge
        prior = np.sum(np.where(zz, np.log(pi), np.log1p(-pi)))
        logp.append(prior + stats.multivariate_normal(np.zeros(om.sum()), cov).logpdf(xo))
    logp = np.array(logp)
    p = np.exp(logp - logp.max())
    p /= p.sum()

    st = O.State(prm, D=D, pi=pi, gamma_s=gs, gamma_eps=ge)
    T, burn = 60000, 200
    counts = np.zeros(len(states))
    for t in range(T + burn):
        st.t = t
        O.zs_sweep(st, x, mask)
        if t >= burn:
            counts[int("".join(str(int(v)) for v in st.Z[0]), 2)] += 1
    freq = counts / T
    # autocorrelated chain: allow a variance inflation of 10 on each state
    tol = 6 * np.sqrt(10 * p * (1 - p) / T) + 1e-3
    assert np.all(np.abs(freq - p) < tol), (freq, p)
    assert 0.5 * np.abs(freq - p).sum() < 0.02


def _small_frame_problem(K, seed):
    rng = np.random.default_rng(seed)
    M, B, S = (2, 90), (2, 3), (2, 3)
    prm = O.params(M, B, S, K, seed=seed)
    N, P = O.num_patches(prm), O.patch_size(prm)
    mask = (rng.random(M) < 0.7).astype(np.uint8)
    D = rng.standard_normal((K, P)) / np.sqrt(P)
    Z = (rng.random((N, K)) < 0.6).astype(np.uint8)
    Sv = rng.standard_normal((N, K)) * Z
    x = (rng.standard_normal(M) * 0.5).astype(np.float32)
    return prm, x, mask, D, Z, Sv


def _ridge(w, y, ge, P):
    """Posterior mean and variance of a scalar coefficient by least squares on
    the prior-augmented system [sqrt(ge) w; sqrt(P)] d = [sqrt(ge) y; 0]."""
    A = np.concatenate([np.sqrt(ge) * w, [np.sqrt(P)]])[:, None]
    b = np.concatenate([np.sqrt(ge) * y, [0.0]])
    mean = np.linalg.lstsq(A, b, rcond=None)[0][0]
    var = np.linalg.inv(A.T @ A)[0, 0]
    return mean, var


def test_dictionary_conditionals_in_atom_order():
    K, ge = 2, 5.0
    prm, x, mask, D0, Z, Sv = _small_frame_problem(K, seed=21)
    N, P = Z.shape[0], D0.shape[1]
    idx = O.patch_origins(prm)[:, None] + O.pixel_offsets(prm)[None, :]
    X = x.reshape(-1)[idx].astype(np.float64)
    Om = mask.reshape(-1)[idx].astype(bool)
    W = Z * Sv
    T = 3000
    z0, z1 = [], []
    for t in range(T):
        st = O.State(prm, D=D0, Z=Z, S=Sv, gamma_eps=ge, t=t)
        O.d_sweep(st, x, mask)
        for p in range(P):
            o = Om[:, p]
            m0, v0 = _ridge(W[o, 0], X[o, p] - D0[1, p] * W[o, 1], ge, P)
            z0.append((st.D[0, p] - m0) / np.sqrt(v0))
            m1, v1 = _ridge(W[o, 1], X[o, p] - st.D[0, p] * W[o, 0], ge, P)
            z1.append((st.D[1, p] - m1) / np.sqrt(v1))
    for zz in (np.array(z0), np.array(z1)):
        assert stats.kstest(zz, "norm").pvalue > 1e-3
        assert abs(zz.mean()) < 5 / np.sqrt(len(zz))
        assert abs(zz.var() - 1) < 5 * np.sqrt(2.0 / len(zz))


def test_pi_and_precision_conditionals():
    K = 3
    prm, x, mask, D, Z, Sv = _small_frame_problem(K, seed=33)
    N, P = Z.shape[0], D.shape[1]
    idx = O.patch_origins(prm)[:, None] + O.pixel_offsets(prm)[None, :]
    X = x.reshape(-1)[idx].astype(np.float64)
    Om = mask.reshape(-1)[idx].astype(bool)
    W = Z * Sv
    R = (X - W @ D) * Om
    m = Z.sum(0).astype(np.float64)
    a_, b_ = prm.a / K, prm.b * (K - 1) / K
    T = 20000
    pis, gss, ges = np.zeros((T, K)), np.zeros(T), np.zeros(T)
    for t in range(T):
        st = O.State(prm, D=D, Z=Z, S=Sv, gamma_eps=1.0, t=t)
        O.hyper(st, x, mask)
        pis[t], gss[t], ges[t] = st.pi, st.gamma_s, st.gamma_eps
    for k in range(K):
        assert stats.kstest(pis[:, k], stats.beta(a_ + m[k], b_ + N - m[k]).cdf).pvalue > 1e-3
    gs_law = stats.gamma(prm.c + 0.5 * Z.sum(), scale=1 / (prm.d + 0.5 * np.sum(W ** 2)))
    ge_law = stats.gamma(prm.e + 0.5 * Om.sum(), scale=1 / (prm.f + 0.5 * np.sum(R ** 2)))
    assert stats.kstest(gss, gs_law.cdf).pvalue > 1e-3
    assert stats.kstest(ges, ge_law.cdf).pvalue > 1e-3


def test_consecutive_code_draws_are_independent():
    """With two atoms orthogonal on the observed pixels and both (almost)
    always active, s_0 and s_1 are independent with the single-atom
    posteriors N(ge d_k.x / lam_k, 1 / lam_k), lam_k = gs + ge |d_k|^2: their
    correlation must vanish (random words shared between the two draws would
    correlate them) and each must have its posterior moments."""
    M, B, S, K = (3, 3), (3, 3), (1, 1), 2
    prm = O.params(M, B, S, K, seed=21)
    rng = np.random.default_rng(21)
    x = rng.standard_normal(M).astype(np.float32)
    mask = np.ones(M, np.uint8)
    D = np.zeros((K, 9))
    D[0, :3] = 1.0 / np.sqrt(3.0)
    D[1, 3], D[1, 4] = 1.0 / np.sqrt(2.0), -1.0 / np.sqrt(2.0)
    gs, ge = 2.0, 3.0
    st = O.State(prm, D=D, pi=[0.999999, 0.999999], gamma_s=gs, gamma_eps=ge)
    T = 30000
    s = np.zeros((T, K))
    for t in range(T):
        st.t = t
        O.zs_sweep(st, x, mask)
        s[t] = st.S[0]
    assert np.all(st.Z[0] == 1)
    xo = x.reshape(-1).astype(np.float64)
    for k in range(K):
        lam = gs + ge * np.dot(D[k], D[k])
        mean, var = ge * np.dot(D[k], xo) / lam, 1.0 / lam
        assert abs(s[:, k].mean() - mean) < 5 * np.sqrt(var / T)
        assert abs(s[:, k].var() / var - 1) < 5 * np.sqrt(2.0 / T)
    assert abs(np.corrcoef(s[:, 0], s[:, 1])[0, 1]) < 5 / np.sqrt(T)
