"""Pins for the general-model oracle (oracle/general.c) against what fixes it from
outside:

- SISe written in the general form is the SISe oracle's model: counts, phi and
  counters equal bit for bit (post- and pre-event phi, events, two replicates);
- SISe3 in the general form with the stochastic step switched off: the event
  masks, the aging offset and the phi update equal the SISe3 oracle bit for bit;
- SIR with beta = 0: I_T ~ Binomial(I_0, exp(-gamma T));
- SIR on 10-animal nodes (frequency-dependent and mass-action infection): the
  law of (S_T, I_T) from the matrix exponential of the generator (chi-square);
- the chain E -> I -> R: the closed-form occupation probabilities of a
  two-step linear chain (means within 4 standard errors);
- the continuous update at constant counts: the closed form of the linear
  recursion, with and without a denominator;
- the three update sources on a hand-computed one-node example (post-event,
  post-SSA, and the midpoint of Eq. numstep2);
- event bookkeeping by hand for one-compartment masks and offsets, clamping and
  the ERROR policy; the multivariate hypergeometric law of a draw from a
  non-contiguous mask.
The last test plants plausible mistakes in a copy of general.c and checks that a
pin catches each.
"""
import math
import pathlib

import numpy as np
import pytest
import scipy.linalg
from scipy import stats

import oracle
from paper_1502_02908_gb300 import workloads as W
from tests.test_oracle_model import _chisq_pvalue

G = W.GeneralWorkload


def _copies(model, u0_node, copies, T, rates, var_params=None, y0_node=None, events=None, seed=7,
            underflow_error=False):
    u0 = np.repeat(np.asarray(u0_node, np.int32)[:, None], copies, axis=1)
    ny = model.ny
    y0 = np.zeros((ny, copies)) if y0_node is None else np.repeat(np.asarray(y0_node, float)[:, None], copies, 1)
    vp = np.zeros((1, ny, 6)) if var_params is None else np.asarray(var_params, float).reshape(1, ny, 6)
    ev = W.GeneralEvents.empty() if events is None else events
    return G("copies", model, copies, T, 1, u0, y0, np.asarray(rates, float).reshape(1, -1), vp, ev, seed,
             underflow_error)


def _ev(rows):
    cols = list(zip(*rows))
    return W.GeneralEvents(*(np.array(c, np.int32) for c in cols))


def _sir(freq=True):
    return W.sir_general(N=2, T=1, n_events=0, freq=freq).model


# ------------------------------------------------------------ against the SISe oracle
@pytest.mark.parametrize("pre_event", [False, True])
def test_sise_general_equals_sise_oracle(pre_event):
    w = W.sise_plain(N=300, T=40, n_events=3000, R=2, seed=5)
    w.params.upsilon[1, 0] *= 1.3
    w.params.gamma[1, 0] *= 0.8
    w.phi0 = np.random.default_rng(3).uniform(0.0, 0.2, size=w.N)
    g = W.as_general(w, W.Y_PRE_EVENT if pre_event else W.Y_POST_EVENT)
    a = oracle.run(w, phi_pre_event=pre_event)
    b = oracle.run_general(g)
    assert np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.phi, b.y[:, 0, :])
    assert np.array_equal(a.counters, b.counters)
    assert a.counters[:, 0].min() > 1000 and a.counters[:, 2].sum() > 0


def test_sise_general_error_policy_equals_sise_oracle():
    w = W.sise_plain(N=60, T=30, n_events=2000, seed=9)
    w.events.count[:] = w.events.count * 20
    g = W.as_general(w)
    g.underflow_error = True
    a = oracle.run(w, underflow_error=True)
    b = oracle.run_general(g)
    assert np.array_equal(a.counts, b.counts) and np.array_equal(a.counters, b.counters)
    assert a.counters[0, 3] > 0


def test_sise3_events_and_phi_equal_sise3_oracle_with_ssa_off():
    w = W.sise3_national(N=800, T=30, n_events=20_000)
    w.params.upsilon[:] = 0.0
    w.params.gamma[:] = 0.0
    w.phi0 = np.random.default_rng(4).uniform(0.0, 0.1, size=w.N)
    a = oracle.run(w)
    b = oracle.run_general(W.as_general(w))
    assert np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.phi, b.y[:, 0, :])
    assert np.array_equal(a.counters, b.counters)
    assert a.counters[0, 1] > 5000


# ------------------------------------------------------------------- closed forms
def test_sir_pure_recovery_binomial():
    I0, gamma, T, n = 40, 0.15, 4, 20_000
    w = _copies(_sir(), [30, I0, 0], n, T, [0.0, gamma])
    r = oracle.run_general(w)
    S, I, R = r.counts[0]
    assert (S == 30).all() and (I + R == I0).all()
    p = math.exp(-gamma * T)
    pmf = stats.binom.pmf(np.arange(I0 + 1), I0, p)
    assert _chisq_pvalue(np.bincount(I, minlength=I0 + 1), pmf) > 1e-4
    assert abs(I.mean() - I0 * p) < 4 * math.sqrt(I0 * p * (1 - p) / n)


def _sir_law(S0, I0, Ntot, beta, gamma, T, freq):
    states = [(s, i) for s in range(Ntot + 1) for i in range(Ntot + 1 - s)]
    idx = {st: k for k, st in enumerate(states)}
    Q = np.zeros((len(states), len(states)))
    for (s, i), k in idx.items():
        inf = beta * s * i / (Ntot if freq else 1.0)
        rec = gamma * i
        if inf > 0:
            Q[k, idx[(s - 1, i + 1)]] += inf
        if rec > 0:
            Q[k, idx[(s, i - 1)]] += rec
        Q[k, k] = -(inf + rec)
    p0 = np.zeros(len(states)); p0[idx[(S0, I0)]] = 1.0
    return states, p0 @ scipy.linalg.expm(Q * T)


@pytest.mark.parametrize("freq,beta", [(True, 1.2), (False, 0.12)])
def test_sir_ten_animals_matches_generator(freq, beta):
    S0, I0, gamma, T, n = 7, 3, 0.4, 2, 60_000
    w = _copies(_sir(freq), [S0, I0, 0], n, T, [beta, gamma])
    r = oracle.run_general(w)
    S, I, R = r.counts[0]
    assert ((S + I + R) == 10).all()
    states, law = _sir_law(S0, I0, 10, beta, gamma, T, freq)
    code = {st: k for k, st in enumerate(states)}
    obs = np.bincount([code[(s, i)] for s, i in zip(S.tolist(), I.tolist())], minlength=len(states))
    assert _chisq_pvalue(obs, law) > 1e-4


def test_linear_chain_means():
    # SEIRS with only E -> I (sigma) and I -> R (gamma): each exposed animal is
    # an independent two-step chain
    sigma, gamma, T, E0, n = 0.3, 0.1, 3, 6, 40_000
    w0 = W.seirs_env(N=2, T=1, n_events=0, R=1)
    rates = [0.0, 0.0, sigma, gamma, 0.0, 0.0]
    w = _copies(w0.model, [5, E0, 0, 0], n, T, rates, var_params=np.zeros((2, 6)), y0_node=[0.0, 0.0])
    r = oracle.run_general(w)
    S, E, I, R = r.counts[0]
    assert (S == 5).all() and ((E + I + R) == E0).all()
    pE = math.exp(-sigma * T)
    pI = sigma / (gamma - sigma) * (math.exp(-sigma * T) - math.exp(-gamma * T))
    for got, p in ((E, pE), (I, pI)):
        se = math.sqrt(E0 * p * (1 - p) / n)
        assert abs(got.mean() - E0 * p) < 4 * se


def test_continuous_update_closed_form():
    # all rates 0, no events: y_n = (1-b)^n y_0 + c (1 - (1-b)^n) / b with
    # c = alpha U / D + eps (first variable) and alpha U + eps (second, no denominator)
    w0 = W.seirs_env(N=2, T=1, n_events=0, R=1)
    b0, b1, a0, a1, e0, e1 = 0.05, 0.2, 0.7, 0.3, 1e-3, 2e-4
    vp = np.array([[a0, b0, b0, b0, b0, e0], [a1, b1, b1, b1, b1, e1]])
    u = [20, 4, 6, 10]                     # I / N = 6 / 40, E = 4
    T = 60
    w = _copies(w0.model, u, 3, T, np.zeros(6), var_params=vp, y0_node=[0.4, 0.0])
    r = oracle.run_general(w)
    for q, (y0, b, c) in enumerate(((0.4, b0, a0 * 6 / 40 + e0), (0.0, b1, a1 * 4 + e1))):
        want = (1 - b) ** T * y0 + c * (1 - (1 - b) ** T) / b
        np.testing.assert_allclose(r.y[0, q], want, rtol=1e-13)
    assert (r.counts[0] == np.asarray(u)[:, None]).all()


@pytest.mark.parametrize("source,want", [(W.Y_POST_EVENT, 1 / 7), (W.Y_PRE_EVENT, 2 / 4), (W.Y_MIDPOINT, 3 / 11)])
def test_midpoint_hand_example(source, want):
    # one node (S, I) = (2, 2), no transitions; day 0 brings 4 susceptibles and
    # removes 1 infected: X_0 = (2, 2), X_1 = (6, 1).  alpha = 1, beta = eps = 0,
    # y_0 = 0: post-event I/N = 1/7, post-SSA 2/4, midpoint
    # ((2 + 1) / 2) / ((4 + 7) / 2) = 3/11
    m = W.general_model(("S", "I"), [], variables=[(("I",), ("S", "I"))], selects=[("S",), ("I",)],
                        y_source=source)
    ev = _ev([(0, W.ENTER, 0, -1, 4, 0, -1), (0, W.EXIT, 0, -1, 1, 1, -1)])
    w = _copies(m, [2, 2], 1, 1, [], var_params=[1.0, 0, 0, 0, 0, 0.0], y0_node=[0.0], events=ev)
    r = oracle.run_general(w)
    assert r.y[0, 0, 0] == want
    assert r.counts[0, :, 0].tolist() == [6, 1]


def test_event_bookkeeping_by_hand():
    # compartments S, E, I, R; masks: 0 all, 1 {S}, 2 {S, E}; offset row 0: S -> R (+3)
    m = W.seirs_env(N=2, T=1, n_events=0).model
    u = [[10, 5], [4, 0], [3, 1], [0, 2]]
    # (day, kind, node, dest, count, select, shift)
    ev = _ev([(0, W.ENTER, 0, -1, 3, 1, 0),      # 3 animals into S + 3 = R of node 0
              (0, W.INTERNAL, 0, -1, 4, 1, 0),   # 4 S -> R at node 0
              (0, W.EXTERNAL, 1, 0, 5, 1, -1),   # all 5 S of node 1 to node 0
              (1, W.EXIT, 1, -1, 9, 1, -1),      # node 1 has no S left: clamped to 0
              (1, W.EXIT, 0, -1, 2, 1, -1)])     # 2 S leave node 0
    w = _copies(m, [0, 0, 0, 0], 2, 2, np.zeros(6), var_params=np.zeros((2, 6)), y0_node=[0, 0], events=ev)
    w.u0 = np.array(u, np.int32)
    r = oracle.run_general(w)
    assert r.counts[0].tolist() == [[10 - 4 + 5 - 2, 0], [4, 0], [3, 1], [0 + 3 + 4, 2]]
    assert r.counters[0, 1:].tolist() == [5, 1, 0]
    w.underflow_error = True
    r = oracle.run_general(w)
    assert r.counts[0].tolist() == [[10 - 4 + 5 - 2, 0], [4, 0], [3, 1], [7, 2]]
    assert r.counters[0, 1:].tolist() == [4, 0, 1]


def test_exit_draw_from_noncontiguous_mask_is_hypergeometric():
    # mask {S, I, R} of (S, E, I, R) = (3, 4, 2, 5): an exit of 4 removes a
    # multivariate hypergeometric composition and never touches E
    m = W.seirs_env(N=2, T=1, n_events=0).model
    m.select = np.array([0b1101], np.uint32)
    n = 30_000
    ev = W.GeneralEvents(np.zeros(n, np.int32), np.full(n, W.EXIT, np.int32), np.arange(n, dtype=np.int32),
                         np.full(n, -1, np.int32), np.full(n, 4, np.int32), np.zeros(n, np.int32),
                         np.full(n, -1, np.int32))
    w = _copies(m, [3, 4, 2, 5], n, 1, np.zeros(6), var_params=np.zeros((2, 6)), y0_node=[0, 0], events=ev)
    r = oracle.run_general(w)
    S, E, I, R = r.counts[0]
    assert (E == 4).all()
    took = np.stack([3 - S, 2 - I, 5 - R], 1)
    assert (took.sum(1) == 4).all()
    assert (took >= 0).all() and (took <= np.array([3, 2, 5])).all()
    combos = [(a, b, 4 - a - b) for a in range(4) for b in range(3) if 0 <= 4 - a - b <= 5]
    pmf = np.array([math.comb(3, a) * math.comb(2, b) * math.comb(5, c) for a, b, c in combos], float)
    pmf /= math.comb(10, 4)
    code = {cmb: k for k, cmb in enumerate(combos)}
    obs = np.bincount([code[tuple(t)] for t in took.tolist()], minlength=len(combos))
    assert _chisq_pvalue(obs, pmf) > 1e-4


# --------------------------------------------------------------- planted mistakes
SRC = (pathlib.Path(oracle.__file__).parent / "general.c").read_text()

MUTATIONS = [
    ("rate drops the population division",
     "a = P > 0 ? a / (double)P : 0.0;", "a = P > 0 ? a : 0.0;",
     [lambda: test_sir_ten_animals_matches_generator(True, 1.2)]),
    ("rate drops its second factor",
     "if (m->fb[j] >= 0) a = a * (double)GX(m->fb[j], v);", "",
     [lambda: test_sir_ten_animals_matches_generator(False, 0.12)]),
    ("selection takes the last threshold reached",
     "if (r <= P) { chosen = j; break; }", "if (r <= P) { chosen = j; }",
     [lambda: test_sir_ten_animals_matches_generator(True, 1.2)]),
    ("stoichiometry applied with the wrong sign",
     "GX(c, v) += m->stoich[c * nt + chosen];", "GX(c, v) -= m->stoich[c * nt + chosen];",
     [test_sir_pure_recovery_binomial]),
    ("rate ignores its continuous variable",
     "if (m->fy[j] >= 0) a = a * yv[m->fy[j]];", "",
     [lambda: test_sise_general_equals_sise_oracle(False)]),
    ("continuous update drops epsilon",
     "return ((y * omb) + mid) + g->epsilon[q];", "return ((y * omb) + mid);",
     [test_continuous_update_closed_form]),
    ("variable without denominator divides anyway",
     "if (m->den[q] == 0) mid = g->alpha[q] * U;", "if (0) mid = g->alpha[q] * U;",
     [test_continuous_update_closed_form]),
    ("midpoint uses the end-of-day state only",
     "U = 0.5 * (U0[(int64_t)q * N + v] + U);", "U = U;",
     [lambda: test_midpoint_hand_example(W.Y_MIDPOINT, 3 / 11)]),
    ("entry ignores the offset",
     "GX(c0 + off[c0], node) += n;", "GX(c0, node) += n;", [test_event_bookkeeping_by_hand]),
    ("internal move ignores the offset",
     "if (kind == GO_INTERNAL) GX(got + off[got], node) += 1;", "if (kind == GO_INTERNAL) GX(got, node) += 1;",
     [test_event_bookkeeping_by_hand, test_sise3_events_and_phi_equal_sise3_oracle_with_ssa_off]),
    ("sampling slot off by one",
     "if (slot < have) got = c; else slot -= have;", "if (slot <= have) got = c; else slot -= have;",
     [test_exit_draw_from_noncontiguous_mask_is_hypergeometric]),
    ("midpoint denominator uses the end-of-day state only",
     "D = 0.5 * (D0[(int64_t)q * N + v] + D);", "D = D;",
     [lambda: test_midpoint_hand_example(W.Y_MIDPOINT, 3 / 11)]),
    ("a0 is the last rate, not the sum",
     "for (int j = 0; j < nt; ++j) a0 = a0 + a[j];", "for (int j = 0; j < nt; ++j) a0 = a[j];",
     [lambda: test_sir_ten_animals_matches_generator(True, 1.2)]),
    ("stopping rule ignores elapsed time",
     "if (t + tau >= 1.0) break;", "if (tau >= 1.0) break;", [test_sir_pure_recovery_binomial]),
    ("transfer lands in the source node",
     "else if (kind == GO_EXTERNAL) GX(got + off[got], dest) += 1;",
     "else if (kind == GO_EXTERNAL) GX(got + off[got], node) += 1;", [test_event_bookkeeping_by_hand]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, pins, tmp_path, monkeypatch):
    assert SRC.count(old) == 1, name
    L = oracle.compile_variant(SRC.replace(old, new), tmp_path / "libmut.so", which="general.c")
    monkeypatch.setattr(oracle, "_LIB", L)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin()
