"""Parameter fitting as in Sec. 4.3 of the paper.

N trajectories of the model with parameters k are compared with a reference
trajectory X(t; k*) through region totals (the paper aggregates nodes into the 21
Swedish counties; here a seeded assignment of nodes to regions stands in):

  G(k)^2  = sum over days, regions, compartments of (mean over trajectories of the
            region total - the reference's region total)^2          (Eq. (goal))
  VG(k)^2 = sum of the trajectories' sample variances of the region totals
                                                      (Eqs. (goalvariance), (goalsigma))

with the paper's time integral taken over the daily observations.  The statistics
and both sums run on the GPU (sim_set_regions, sim_goal); this module holds the
host-side driver: the super-parameters k_j = upsilon_j delta_j (Eq.
(superparameters), delta_j = 1 / gamma_j held fixed), the relative residual
(Eq. (residuall)), and the Hooke-Jeeves pattern search the paper uses (Hooke and
Jeeves, J. ACM 8 (1961) 212-229).  Every evaluation of G reuses one simulation
handle (new parameters, same events, same random streams: common random numbers,
so G is a deterministic function of k).

A gradient-based variant (PrevalenceGoal, gradient_descent) fits the daily
national prevalence curve with the library's score-function gradient instead.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import binding as B
from . import workloads as W


def county_regions(N, n_regions=21, seed=21):
    """A seeded assignment of N nodes to n_regions regions (uniform)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n_regions, size=N).astype(np.int32)


def superparameters(upsilon, gamma):
    """k_j = upsilon_j * delta_j with delta_j = 1 / gamma_j (Eq. (superparameters))."""
    return np.asarray(upsilon, np.float64) / np.asarray(gamma, np.float64)


def with_upsilon(params: W.Params, upsilon):
    """params with every replicate's upsilon replaced."""
    ups = np.array(params.upsilon, copy=True)
    ups[:, :len(upsilon)] = np.asarray(upsilon, np.float64)
    return W.Params(ups, params.gamma.copy(), params.alpha.copy(), params.beta.copy(), params.epsilon.copy())


def reference_totals(w: W.Workload, regions, n_regions, upsilon, days=None, replicate_base=1 << 20):
    """Region totals [days, n_regions, Nc] (int64) of one reference trajectory with
    the given upsilon (its own random stream: replicate word replicate_base)."""
    days = w.T if days is None else days
    p = with_upsilon(w.params.replicate(0), upsilon)
    sim = B.Sim(w.model, w.u0, w.phi0, p, w.T, seed=w.seed, replicate_base=replicate_base)
    try:
        sim.load_events(w.events)
        sim.set_regions(regions, n_regions)
        sim.run(days)
        s1, _ = sim.region_moments()
    finally:
        sim.close()
    return s1[:days].astype(np.int64)


class Goal:
    """G(k)^2 and VG(k)^2 of N trajectories against reference region totals."""

    def __init__(self, w: W.Workload, regions, n_regions, ref, trajectories, days=None, launch="graph"):
        self.w = w
        self.days = w.T if days is None else days
        self.ref = np.ascontiguousarray(ref[:self.days], np.int64)
        self.gamma = np.asarray(w.params.gamma[0], np.float64)
        base = W.Params.broadcast(trajectories, w.params.upsilon[0], w.params.gamma[0], w.params.alpha[0],
                                  w.params.beta[0], w.params.epsilon[0])
        self.base = base
        self.sim = B.Sim(w.model, w.u0, w.phi0, base, w.T, seed=w.seed)
        self.sim.load_events(w.events)
        self.sim.set_regions(regions, n_regions)
        self.sim.set_launch(launch)
        self.u0 = np.repeat(w.u0[None], trajectories, 0)
        self.phi0 = np.repeat(w.phi0[None], trajectories, 0)
        self.evaluations = 0

    def __call__(self, k):
        """(G^2, VG^2) at super-parameters k (upsilon_j = k_j / delta_j = k_j gamma_j)."""
        ups = np.asarray(k, np.float64) * self.gamma[:len(k)]
        self.sim.set_params(with_upsilon(self.base, ups))
        self.sim.set_state(self.u0, self.phi0, 0)
        self.sim.run(self.days)
        self.evaluations += 1
        return self.sim.goal(self.ref, 0, self.days)

    def close(self):
        self.sim.close()


def relative_residual(g, g_star):
    """R(k) = |G(k) - G(k*)| / |G(k*)| (Eq. (residuall))."""
    return abs(g - g_star) / abs(g_star)


@dataclasses.dataclass
class SearchResult:
    x: np.ndarray
    f: float
    iterations: int
    evaluations: int
    history: list


def hooke_jeeves(f, x0, step, iterations=20, shrink=0.5, min_step=0.0):
    """Hooke-Jeeves pattern search minimising f (a float-valued function of a
    vector).  Each iteration explores around the base point, one coordinate at a
    time (+step, else -step, kept when f decreases); on success it makes pattern
    moves (jump by the last displacement, explore again) while they keep
    improving, otherwise it multiplies the steps by `shrink`.  Stops after
    `iterations` iterations or when every step is below min_step."""
    cache = {}

    def fx(x):
        key = tuple(np.round(x, 15))
        if key not in cache:
            cache[key] = float(f(np.array(x)))
        return cache[key]

    def explore(x, fxv, s):
        x = np.array(x, np.float64)
        for i in range(len(x)):
            for d in (s[i], -s[i]):
                y = x.copy()
                y[i] += d
                fy = fx(y)
                if fy < fxv:
                    x, fxv = y, fy
                    break
        return x, fxv

    base = np.array(x0, np.float64)
    fb = fx(base)
    s = np.array(step, np.float64) * np.ones_like(base)
    history = [(0, base.copy(), fb)]
    it = 0
    for it in range(1, iterations + 1):
        x, fxv = explore(base, fb, s)
        if fxv < fb:
            while True:                              # pattern moves
                prev = base
                base, fb = x, fxv
                trial = base + (base - prev)
                x, fxv = explore(trial, fx(trial), s)
                if not fxv < fb:
                    break
        else:
            s = s * shrink
        history.append((it, base.copy(), fb))
        if np.all(s < min_step):
            break
    return SearchResult(base, fb, it, len(cache), history)


# ------------------------------------------------------------- gradient-based variant
# The goal above compares region totals of a few trajectories and is searched
# without derivatives.  The score-function gradient of the library (d E[f] /
# d theta = E[f s], s = d log p(path) / d theta, see gradient.py) gives a
# gradient-based variant on the daily national prevalence f_d = I_d / N_d:
#   G_f(x)^2 = sum_d (E[f_d](theta(x)) - f*_d)^2,  theta(x) = (upsilon e^{x_0},
# gamma e^{x_1}) with the age-class ratios kept, searched in log scale.


def scaled_params(params: W.Params, x):
    """params with upsilon scaled by e^{x_0} and gamma by e^{x_1} (every class)."""
    x = np.asarray(x, np.float64)
    return W.Params(params.upsilon * np.exp(x[0]), params.gamma * np.exp(x[1]), params.alpha.copy(),
                    params.beta.copy(), params.epsilon.copy())


def prevalence_curve(w: W.Workload, days, x=(0.0, 0.0), seed_offset=0):
    """E[f_d] over w.R replicates at log scales x (replicate streams of seed w.seed + seed_offset)."""
    from . import gradient as GR
    wx = dataclasses.replace(w, params=scaled_params(w.params, x), seed=w.seed + seed_offset)
    spec = GR.GradientSpec(wx, np.asarray(days, np.int32))
    m, R, _ = GR.run_moments(spec)
    return GR.estimate(m, R, spec.class_ratios())[0]


class PrevalenceGoal:
    """G_f(x)^2 and its score-function gradient in x (log scales of upsilon and
    gamma) for the workload's R replicates against a target curve f*."""

    def __init__(self, w: W.Workload, days, target, chunk=1024):
        self.w, self.days, self.target, self.chunk = w, np.asarray(days, np.int32), np.asarray(target), chunk
        self.evaluations = 0

    def __call__(self, x):
        """(G_f^2, gradient [2], standard error of the gradient [2])."""
        from . import gradient as GR
        wx = dataclasses.replace(self.w, params=scaled_params(self.w.params, x))
        spec = GR.GradientSpec(wx, self.days, self.chunk)
        m, R, (f, s) = GR.run_moments(spec, per_replicate=True)
        mean_f, grad, _ = GR.estimate(m, R, spec.class_ratios())    # d E[f_d] / d (upsilon_1, gamma_1, ...)
        self.evaluations += 1
        diff = mean_f - self.target
        th = spec.theta()
        # d theta_i / d x_i = theta_i for theta = theta_0 e^{x}
        dth = np.array([th[0], th[1]])
        g = 2.0 * (diff @ grad[:, :2]) * dth
        # standard error of g from the replicates' centred contributions
        ru, rg = spec.class_ratios()
        na = ru.size
        s_up = s[:, :na] @ ru                                      # score of upsilon_1 with ratios kept
        s_ga = s[:, 3:3 + na] @ rg
        fc = (f - f.mean(0)) @ diff                                # [R]
        contrib = 2.0 * np.stack([fc * (s_up - s_up.mean()), fc * (s_ga - s_ga.mean())], 1) * dth
        g_se = contrib.std(0, ddof=1) / np.sqrt(R)
        return float(diff @ diff), g, g_se


def gradient_descent(fg, x0, step, iterations=20, shrink=0.5, grow=1.5, min_step=0.0):
    """Normalised gradient descent with an acceptance test, for a goal whose
    gradient is an estimate: from x try x - step g / |g|; keep it when the goal
    decreases (and lengthen the step by `grow`), otherwise shorten the step by
    `shrink`.  fg(x) returns (value, gradient, ...).  Stops after `iterations`
    trials or when the step falls below min_step."""
    x = np.array(x0, np.float64)
    fx, gx = fg(x)[:2]
    s = float(step)
    history = [(0, x.copy(), fx)]
    evaluations = 1
    it = 0
    for it in range(1, iterations + 1):
        n = float(np.linalg.norm(gx))
        if n == 0.0:
            break
        y = x - s * gx / n
        fy, gy = fg(y)[:2]
        evaluations += 1
        if fy < fx:
            x, fx, gx = y, fy, gy
            s *= grow
        else:
            s *= shrink
        history.append((it, x.copy(), fx))
        if s < min_step:
            break
    return SearchResult(x, fx, it, evaluations, history)
