"""Pins for the oracle's score-function terms (likelihood-ratio gradient).

For a trajectory, log p(path) = sum over fired transitions of log(rate) minus the
integral of a0 (from the direct method's sampling law, Eqs. sampling and
sampling2), with phi carried through Eq. numstep5.  The score identity
E[f s] = d E[f] / d theta is checked against exact derivatives:

- independent animals (alpha = 0, so phi is deterministic): E[I_T] from products of
  per-day 2x2 matrix exponentials, derivatives by central differences;
- a 3-animal SIS node with phi depending on the path (alpha > 0): exact law by
  enumerating daily paths (matrix exponentials), derivatives by central
  differences, for all of (upsilon, gamma, beta, alpha).
"""
import math

import numpy as np
import scipy.linalg

import oracle
from paper_1502_02908_gb300 import workloads as W

UPS, GAM, BETA, ALPHA = 0, 3, 6, 7


def _copies(model, u0_node, copies, T, params, phi0, seed=21):
    w = W.tiny_node(model=model, herd=1, infected=0, copies=copies, T=T, params=params,
                    phi0=phi0, seed=seed)
    w.u0 = np.repeat(np.asarray(u0_node, np.int32)[:, None], copies, axis=1)
    return w


def _score_check(f, s, exact, k=4.0):
    """Covariance form of the score estimator, within k standard errors."""
    fc = f - f.mean()
    prod = fc * s
    est = prod.mean()
    se = prod.std(ddof=1) / math.sqrt(f.size)
    assert abs(est - exact) < k * se + 1e-12, (est, exact, se)
    assert abs(s.mean()) < k * s.std(ddof=1) / math.sqrt(s.size)
    return est, se


def _indep_mean_I(S0, I0, ups, gam, beta, eps, phi0, T):
    phi = phi0
    M = np.eye(2)
    for _ in range(T):
        c = ups * phi
        Q = np.array([[-c, c], [gam, -gam]])
        M = M @ scipy.linalg.expm(Q)
        phi = phi * (1 - beta) + eps
    return S0 * M[0, 1] + I0 * M[1, 1]


def test_score_identity_independent_animals():
    S0, I0, ups, gam, beta, eps, phi0, T = 6, 4, 0.08, 0.3, 0.1, 0.05, 1.5, 4
    n = 400_000
    w = _copies(W.SISE, [S0, I0], n, T, dict(upsilon=ups, gamma=gam, alpha=0.0, beta=beta, epsilon=eps), phi0)
    r = oracle.run(w, score=True)
    f = r.counts[0, 1].astype(np.float64)
    sc = r.score[0]
    base = dict(S0=S0, I0=I0, ups=ups, gam=gam, beta=beta, eps=eps, phi0=phi0, T=T)

    def d(name, h):
        lo = dict(base); hi = dict(base)
        lo[name] -= h; hi[name] += h
        return (_indep_mean_I(**hi) - _indep_mean_I(**lo)) / (2 * h)

    _score_check(f, sc[UPS], d("ups", 1e-6))
    _score_check(f, sc[GAM], d("gam", 1e-6))
    _score_check(f, sc[BETA], d("beta", 1e-6))


def _sis_law(N, I0, ups, gam, alpha, beta, eps, phi0, T):
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


def test_score_identity_path_dependent_phi():
    N, I0, ups, gam, alpha, beta, eps, phi0, T = 3, 1, 0.6, 0.5, 1.2, 0.3, 0.02, 0.4, 3
    n = 1_000_000
    w = _copies(W.SISE, [N - I0, I0], n, T,
                dict(upsilon=ups, gamma=gam, alpha=alpha, beta=beta, epsilon=eps), phi0)
    r = oracle.run(w, score=True)
    I_T = r.counts[0, 1]
    sc = r.score[0]
    base = dict(N=N, I0=I0, ups=ups, gam=gam, alpha=alpha, beta=beta, eps=eps, phi0=phi0, T=T)
    fs = {"mean_I": lambda law: float(np.dot(np.arange(N + 1), law)),
          "extinct": lambda law: float(law[0])}
    vals = {"mean_I": I_T.astype(np.float64), "extinct": (I_T == 0).astype(np.float64)}
    for fname, fn in fs.items():
        for pname, k in (("ups", UPS), ("gam", GAM), ("beta", BETA), ("alpha", ALPHA)):
            h = 1e-6 * base[pname]
            lo = dict(base); hi = dict(base)
            lo[pname] -= h; hi[pname] += h
            exact = (fn(_sis_law(**hi)) - fn(_sis_law(**lo))) / (2 * h)
            _score_check(vals[fname], sc[k], exact)


def test_score_identity_sise3_classes():
    u0 = [8, 2, 5, 5, 9, 1]
    ups = [0.05, 0.1, 0.02]; gam = [0.3, 0.2, 0.4]; phi0 = 2.0; T = 2; n = 300_000
    w = _copies(W.SISE3, u0, n, T, dict(upsilon=ups, gamma=gam, alpha=0.0, beta=0.0, epsilon=0.0), phi0)
    r = oracle.run(w, score=True)
    sc = r.score[0]
    for j in range(3):
        f = r.counts[0, 2 * j + 1].astype(np.float64)

        def m(u, g):
            return _indep_mean_I(u0[2 * j], u0[2 * j + 1], u, g, 0.0, 0.0, phi0, T)
        h = 1e-6
        _score_check(f, sc[UPS + j], (m(ups[j] + h, gam[j]) - m(ups[j] - h, gam[j])) / (2 * h))
        _score_check(f, sc[GAM + j], (m(ups[j], gam[j] + h) - m(ups[j], gam[j] - h)) / (2 * h))
        # a class's count does not depend on another class's parameters
        other = (j + 1) % 3
        _score_check(f, sc[UPS + other], 0.0)
