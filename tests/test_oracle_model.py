"""Pins for the oracle's model arithmetic against what the mathematics fixes:

- pure death (upsilon = 0): I_T ~ Binomial(I_0, exp(-gamma T));
- frozen phi (alpha = beta = epsilon = 0): every animal is an independent
  two-state chain, so I_T is a sum of two binomials (per age class for SISe3);
- a 10-animal SIS node with phi evolving between days: the exact law of I_T by
  enumerating daily paths with matrix exponentials of the 11-state generator
  (chi-square on 1e6 samples);
- phi at constant counts: the closed form of the linear recursion (Eq. numstep5
  with Eq. siminfpressure), constant and seasonal beta;
- scheduled events: per-class bookkeeping when nothing is clamped, S/I
  conservation under aging and transfers, clamping and the ERROR policy, and the
  exact (multivariate) hypergeometric law of the sampled animals.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy import stats

import oracle
from paper_1502_02908_gb300 import workloads as W


def _chisq_pvalue(observed, expected_prob, min_expected=5.0):
    n = observed.sum()
    exp = expected_prob * n
    obs_b, exp_b = [], []
    o_acc = e_acc = 0.0
    for o, e in zip(observed, exp):
        o_acc += o; e_acc += e
        if e_acc >= min_expected:
            obs_b.append(o_acc); exp_b.append(e_acc); o_acc = e_acc = 0.0
    if e_acc > 0:
        obs_b[-1] += o_acc; exp_b[-1] += e_acc
    obs_b = np.array(obs_b); exp_b = np.array(exp_b)
    exp_b *= obs_b.sum() / exp_b.sum()
    return stats.chisquare(obs_b, exp_b).pvalue


def _copies(model, u0_node, copies, T, params, phi0=0.0, seed=11):
    w = W.tiny_node(model=model, herd=1, infected=0, copies=copies, T=T, params=params,
                    phi0=phi0, seed=seed)
    w.u0 = np.repeat(np.asarray(u0_node, np.int32)[:, None], copies, axis=1)
    return w


def test_pure_death_binomial():
    I0, gamma, T, n = 50, 0.1, 5, 20_000
    w = _copies(W.SISE, [0, I0], n, T, dict(upsilon=0.0, gamma=gamma, alpha=0.0, beta=0.0, epsilon=0.0))
    r = oracle.run(w)
    I_T = r.counts[0, 1]
    assert (r.counts[0].sum(0) == I0).all()           # recovered animals become S
    p = math.exp(-gamma * T)
    pmf = stats.binom.pmf(np.arange(I0 + 1), I0, p)
    assert _chisq_pvalue(np.bincount(I_T, minlength=I0 + 1), pmf) > 1e-4
    se = math.sqrt(I0 * p * (1 - p) / n)
    assert abs(I_T.mean() - I0 * p) < 4 * se


def _two_state_pmf(S0, I0, c, g, T):
    lam = c + g
    p_si = c / lam * (1 - math.exp(-lam * T))
    p_ii = c / lam + g / lam * math.exp(-lam * T)
    a = stats.binom.pmf(np.arange(S0 + 1), S0, p_si)
    b = stats.binom.pmf(np.arange(I0 + 1), I0, p_ii)
    return np.convolve(a, b)


def test_frozen_phi_two_state_law_sise():
    S0, I0, ups, phi0, gam, T, n = 30, 10, 0.05, 2.0, 0.2, 3, 20_000
    w = _copies(W.SISE, [S0, I0], n, T, dict(upsilon=ups, gamma=gam, alpha=0.0, beta=0.0, epsilon=0.0),
                phi0=phi0)
    r = oracle.run(w)
    assert np.all(r.phi == phi0)                     # alpha = beta = eps = 0 keeps phi
    I_T = r.counts[0, 1]
    pmf = _two_state_pmf(S0, I0, ups * phi0, gam, T)
    assert _chisq_pvalue(np.bincount(I_T, minlength=S0 + I0 + 1), pmf) > 1e-4


def test_frozen_phi_two_state_law_sise3_per_class():
    # classes evolve independently while phi is frozen; each marginal is exact
    u0 = [20, 5, 12, 12, 30, 2]
    ups = [0.05, 0.02, 0.1]; gam = [0.2, 0.3, 0.05]; phi0 = 2.0; T = 2; n = 20_000
    w = _copies(W.SISE3, u0, n, T, dict(upsilon=ups, gamma=gam, alpha=0.0, beta=0.0, epsilon=0.0),
                phi0=phi0)
    r = oracle.run(w)
    for j in range(3):
        S0, I0 = u0[2 * j], u0[2 * j + 1]
        I_T = r.counts[0, 2 * j + 1]
        assert (r.counts[0, 2 * j] + I_T == S0 + I0).all()
        pmf = _two_state_pmf(S0, I0, ups[j] * phi0, gam[j], T)
        assert _chisq_pvalue(np.bincount(I_T, minlength=S0 + I0 + 1), pmf) > 1e-4, j


def sis_exact_law(N, I0, ups, gam, alpha, beta, eps, phi0, T):
    """Law of I_T for one SISe node without events: day by day, I_{d+1} ~ row
    I_d of expm(Q(phi_d)) and phi_{d+1} = phi_d (1 - beta) + alpha I_{d+1} / N + eps."""
    def P(phi):
        Q = np.zeros((N + 1, N + 1))
        for i in range(N + 1):
            if i < N:
                Q[i, i + 1] = ups * phi * (N - i)
            if i > 0:
                Q[i, i - 1] = gam * i
            Q[i, i] = -Q[i].sum()
        return scipy.linalg.expm(Q)
    law = {(I0, phi0): 1.0}
    for _ in range(T):
        nxt = {}
        for (i, phi), pr in law.items():
            row = P(phi)[i]
            for k in range(N + 1):
                key = (k, phi * (1 - beta) + alpha * k / N + eps)
                nxt[key] = nxt.get(key, 0.0) + pr * row[k]
        law = nxt
    out = np.zeros(N + 1)
    for (i, _), pr in law.items():
        out[i] += pr
    return out


def test_ten_animal_sis_matches_matrix_exponential_paths():
    N, I0, ups, gam, alpha, beta, eps, phi0, T = 10, 2, 0.3, 0.4, 1.0, 0.2, 0.01, 0.5, 3
    exact = sis_exact_law(N, I0, ups, gam, alpha, beta, eps, phi0, T)
    assert abs(exact.sum() - 1) < 1e-12
    n = 1_000_000
    w = _copies(W.SISE, [N - I0, I0], n, T, dict(upsilon=ups, gamma=gam, alpha=alpha, beta=beta, epsilon=eps),
                phi0=phi0)
    r = oracle.run(w)
    I_T = r.counts[0, 1]
    assert _chisq_pvalue(np.bincount(I_T, minlength=N + 1), exact) > 1e-4
    # a one-day horizon reduces to the frozen-phi binomial law
    assert np.allclose(sis_exact_law(N, I0, ups, gam, alpha, beta, eps, phi0, 1),
                       _two_state_pmf(N - I0, I0, ups * phi0, gam, 1), atol=1e-12)


def test_phi_closed_form_constant_beta():
    S, I, alpha, beta, eps, phi0, T = 7, 3, 0.7, 0.05, 1e-3, 0.25, 200
    w = _copies(W.SISE, [S, I], 1, T, dict(upsilon=0.0, gamma=0.0, alpha=alpha, beta=beta, epsilon=eps),
                phi0=phi0)
    r = oracle.run(w)
    a = 1 - beta
    q = alpha * I / (S + I) + eps
    closed = a ** T * phi0 + q * (1 - a ** T) / beta
    assert abs(r.phi[0, 0] - closed) <= 1e-13 * closed


def test_phi_closed_form_seasonal_beta_and_empty_node():
    alpha, eps, phi0, T = 1.0, 1e-6, 0.1, 730
    betas = W.vtec_beta()
    w = _copies(W.SISE3, [10, 2, 0, 0, 5, 3], 2, T,
                dict(upsilon=0.0, gamma=0.0, alpha=alpha, beta=betas, epsilon=eps), phi0=phi0)
    w.u0[:, 1] = 0                                   # node 1 holds no animals
    r = oracle.run(w)
    # closed form per season block: phi_end = a^L phi + q (1 - a^L) / beta
    def blocks(T):
        d = 0
        while d < T:
            dm = d % 365
            s = 0 if dm <= 91 else 1 if dm <= 182 else 2 if dm <= 273 else 3
            end = d
            while end < T and ((end % 365 <= 91 and s == 0) or (91 < end % 365 <= 182 and s == 1)
                               or (182 < end % 365 <= 273 and s == 2) or (end % 365 > 273 and s == 3)):
                end += 1
            yield s, end - d
            d = end
    for v, q in ((0, alpha * 5 / 20 + eps), (1, eps)):
        phi = phi0
        for s, L in blocks(T):
            a = 1 - betas[s]
            phi = a ** L * phi + q * (1 - a ** L) / betas[s]
        assert abs(r.phi[0, v] - phi) <= 1e-13 * phi, v


def _event_workload(model, u0, events, T, seed=5, R=1):
    w = W.tiny_node(model=model, herd=1, infected=0, copies=u0.shape[1], T=T, R=R,
                    params=dict(upsilon=0.0, gamma=0.0, alpha=0.0, beta=0.0, epsilon=0.0), seed=seed)
    w.u0 = np.ascontiguousarray(u0, np.int32)
    w.events = events
    return w


def test_events_bookkeeping_without_clamping():
    rng = np.random.default_rng(7)
    N, T, n_ev = 50, 20, 3000
    u0 = rng.integers(400, 600, size=(6, N)).astype(np.int32)
    kind = rng.integers(0, 4, size=n_ev)
    node = rng.integers(0, N, size=n_ev)
    dest = (node + rng.integers(1, N, size=n_ev)) % N
    cls = np.where(kind == W.INTERNAL, rng.integers(0, 2, size=n_ev), rng.integers(0, 3, size=n_ev))
    ev = W.Events(rng.integers(0, T, size=n_ev).astype(np.int32), kind.astype(np.int32),
                  node.astype(np.int32), np.where(kind == W.EXTERNAL, dest, -1).astype(np.int32),
                  rng.integers(1, 6, size=n_ev).astype(np.int32), cls.astype(np.int32))
    w = _event_workload(W.SISE3, u0, ev, T)
    r = oracle.run(w)
    assert r.counters[0, 2] == 0 and r.counters[0, 1] == n_ev
    # per node and class, S + I follows the event arithmetic exactly
    tot = (u0[0::2] + u0[1::2]).astype(np.int64)            # [3, N]
    for k, v, d_, n, c in zip(ev.kind, ev.node, ev.dest, ev.count, ev.cls):
        if k == W.EXIT: tot[c, v] -= n
        elif k == W.ENTER: tot[c, v] += n
        elif k == W.INTERNAL: tot[c, v] -= n; tot[c + 1, v] += n
        else: tot[c, v] -= n; tot[c, d_] += n
    got = r.counts[0, 0::2].astype(np.int64) + r.counts[0, 1::2]
    assert np.array_equal(got, tot)
    assert (r.counts >= 0).all()
    # without exits and enters, S and I totals (summed over classes) are conserved
    keep = (ev.kind == W.INTERNAL) | (ev.kind == W.EXTERNAL)
    r2 = oracle.run(w, events=ev.select(keep))
    assert r2.counts[0, 0::2].sum() == u0[0::2].sum()
    assert r2.counts[0, 1::2].sum() == u0[1::2].sum()
    assert r2.prev_i[0, -1] == u0[1::2].sum()


def test_events_clamp_and_error_policy():
    u0 = np.array([[2], [1]], np.int32)
    ev = W.Events(*(np.array([x], np.int32) for x in (0, W.EXIT, 0, -1, 5, -1)))
    w = _event_workload(W.SISE, u0, ev, 1)
    r = oracle.run(w)
    assert r.counts[0].sum() == 0 and r.counters[0, 2] == 1
    r = oracle.run(w, underflow_error=True)
    assert (r.counts[0] == u0).all() and r.counters[0, 3] == 1 and r.counters[0, 1] == 0


def test_exit_sample_is_hypergeometric():
    S, I, n_take, N = 12, 8, 6, 30_000
    u0 = np.repeat(np.array([[S], [I]], np.int32), N, axis=1)
    z = np.zeros(N, np.int32)
    ev = W.Events(z, z + W.EXIT, np.arange(N, dtype=np.int32), z - 1, z + n_take, z - 1)
    r = oracle.run(_event_workload(W.SISE, u0, ev, 1))
    removed_I = I - r.counts[0, 1]
    assert (r.counts[0].sum(0) == S + I - n_take).all()
    pmf = stats.hypergeom.pmf(np.arange(n_take + 1), S + I, I, n_take)
    assert _chisq_pvalue(np.bincount(removed_I, minlength=n_take + 1), pmf) > 1e-4


def test_transfer_all_classes_is_multivariate_hypergeometric():
    comp = np.array([5, 3, 7, 2, 4, 9], np.int32)
    n_take, N = 10, 20_000
    u0 = np.zeros((6, 2 * N), np.int32)
    u0[:, :N] = comp[:, None]
    z = np.zeros(N, np.int32)
    src = np.arange(N, dtype=np.int32)
    ev = W.Events(z, z + W.EXTERNAL, src, src + N, z + n_take, z - 1)
    r = oracle.run(_event_workload(W.SISE3, u0, ev, 1))
    moved = r.counts[0][:, N:]
    assert np.array_equal(moved + r.counts[0][:, :N], np.repeat(comp[:, None], N, axis=1))
    assert (moved.sum(0) == n_take).all()
    total = comp.sum()
    for c in range(6):
        pmf = stats.hypergeom.pmf(np.arange(n_take + 1), total, comp[c], n_take)
        assert _chisq_pvalue(np.bincount(moved[c], minlength=n_take + 1), pmf) > 1e-4, c
    # joint law of (S1, I1) taken: multivariate hypergeometric cell probabilities
    cells = moved[0] * (n_take + 1) + moved[1]
    prob = np.zeros((n_take + 1) ** 2)
    rest = total - comp[0] - comp[1]
    for a in range(n_take + 1):
        for b in range(n_take + 1 - a):
            if a <= comp[0] and b <= comp[1] and n_take - a - b <= rest:
                prob[a * (n_take + 1) + b] = (math.comb(int(comp[0]), a) * math.comb(int(comp[1]), b)
                                              * math.comb(int(rest), n_take - a - b)) / math.comb(int(total), n_take)
    assert _chisq_pvalue(np.bincount(cells, minlength=prob.size), prob) > 1e-4


def test_synthetic_benchmark_instance_law():
    # The Sec. 4.2 benchmark as generated: unit rates both ways, phi held at 1.
    # Without transfers every node is an independent two-state population, so I_T
    # follows the two-binomial law with c = gamma = 1.
    S0 = I0 = 20
    w = W.synthetic_sis(N=20_000, T=2, S0=S0, I0=I0, rho=0.0)
    assert len(w.events) == 0
    r = oracle.run(w)
    assert np.all(r.phi == 1.0)
    I_T = r.counts[0, 1]
    pmf = _two_state_pmf(S0, I0, 1.0, 1.0, w.T)
    assert _chisq_pvalue(np.bincount(I_T, minlength=S0 + I0 + 1), pmf) > 1e-4
    # with transfers (one animal each, between different sub-domains) totals move
    # only by the transfers
    w = W.synthetic_sis(N=64, T=5, S0=S0, I0=I0, rho=1.0, k=8)
    r = oracle.run(w)
    tot = r.counts[0].sum(0)
    ev = w.events
    delta = np.zeros(w.N, np.int64)
    np.add.at(delta, np.asarray(ev.node), -np.asarray(ev.count))
    np.add.at(delta, np.asarray(ev.dest), np.asarray(ev.count))
    assert np.array_equal(tot, S0 + I0 + delta)
    dom = (np.arange(w.N) * 8) // w.N
    assert np.all(dom[np.asarray(ev.node)] != dom[np.asarray(ev.dest)])
