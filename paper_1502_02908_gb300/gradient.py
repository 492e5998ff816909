"""Score-function (likelihood-ratio) gradients of expected prevalence.

For a trajectory, log p(path) is the sum over fired transitions of log(rate)
minus the integral of the total rate a0 (the direct method's sampling law), with
phi's dependence on (beta, alpha) carried through the daily recursion.  Then
d E[f] / d theta = E[f * d log p / d theta], estimated by the covariance of f and
the score over replicates.  The simulation, the per-node score terms, the reverse
sweep of the phi recursion and the moment sums all run in libepisim's kernels,
and the covariance estimate and its standard error in the library's
sim_gradient_estimate; this module chooses replicate chunks, passes their moment
sums on and exposes the estimate as a ``torch.autograd.Function``.

theta = (upsilon, gamma, beta, alpha).  upsilon and gamma scale every age class
(SISe3: the class ratios of the workload are kept), beta is one value for the
four seasons, alpha the shedding rate.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import binding as B
from . import workloads as W

N_MOMENTS = B.N_MOMENTS


@dataclasses.dataclass
class GradientSpec:
    """What to differentiate: workload ``w`` (its replicate count R), the days whose
    prevalence is f, and how many replicates one handle holds at a time."""
    w: W.Workload
    days: np.ndarray
    chunk: int = 1024

    def with_theta(self, theta):
        th = np.asarray(theta, np.float64)
        p = self.w.params
        u0 = p.upsilon[:, :1].copy(); u0[u0 == 0] = 1.0
        g0 = p.gamma[:, :1].copy(); g0[g0 == 0] = 1.0
        params = W.Params(p.upsilon / u0 * th[0], p.gamma / g0 * th[1], np.full_like(p.alpha, th[3]),
                          np.full_like(p.beta, th[2]), p.epsilon.copy())
        w = dataclasses.replace(self.w, params=params)
        return GradientSpec(w, self.days, self.chunk)

    def theta(self):
        p = self.w.params
        return np.array([p.upsilon[0, 0], p.gamma[0, 0], p.beta[0, 0], p.alpha[0]])

    def class_ratios(self):
        p = self.w.params
        nage = 3 if self.w.model == W.SISE3 else 1
        u = p.upsilon[0, :nage] / (p.upsilon[0, 0] if p.upsilon[0, 0] else 1.0)
        g = p.gamma[0, :nage] / (p.gamma[0, 0] if p.gamma[0, 0] else 1.0)
        return u, g


def _slice_params(p: W.Params, r0, r1):
    return W.Params(p.upsilon[r0:r1].copy(), p.gamma[r0:r1].copy(), p.alpha[r0:r1].copy(),
                    p.beta[r0:r1].copy(), p.epsilon[r0:r1].copy())


def run_moments(spec: GradientSpec, per_replicate=False, rank=0, world=1):
    """Runs every replicate (in chunks), returns (moment sums [n_chunks, F, 42], one
    row per chunk in replicate order, R, optional per-replicate (f [R, F], score
    [R, 8])).  With world > 1 (torch.distributed initialised, one GPU per rank)
    each rank runs its contiguous replicate range and the ranks' chunk rows are
    gathered in rank order, so every rank holds the single-process rows."""
    from . import replicas
    w = spec.w
    days = np.ascontiguousarray(spec.days, np.int32)
    rows = []
    fs, ss = [], []
    lo, hi = replicas.shard(w.R, world, rank)
    for r0 in range(lo, hi, spec.chunk):
        r1 = min(hi, r0 + spec.chunk)
        s = B.Sim(w.model, w.u0, w.phi0, _slice_params(w.params, r0, r1), w.T, seed=w.seed,
                  score_reverse=True, replicate_base=r0)
        try:
            if len(w.events):
                s.load_events(w.events)
            s.run(w.T)
            s.score_backward()
            m, per = s.gradient_moments(days)
            rows.append(m)
            if per_replicate:
                pi, pn, _ = s.stats()
                fs.append(pi[:, days] / np.maximum(pn[:, days], 1))
                ss.append(per)
        finally:
            s.close()
    chunks = np.stack(rows) if rows else np.zeros((0, days.size, N_MOMENTS))
    if world > 1:
        chunks = replicas.allgather_rows(chunks)
    extra = (np.concatenate(fs), np.concatenate(ss)) if per_replicate and fs else None
    return chunks, w.R, extra


def jacobian(ratios):
    """d theta_k / d (upsilon, gamma, beta, alpha) for the 8 score terms: upsilon
    and gamma scale every age class with the given class ratios."""
    ru, rg = ratios
    na = ru.size
    J = np.zeros((8, 4))
    J[0:na, 0] = ru
    J[3:3 + na, 1] = rg
    J[6, 2] = 1.0
    J[7, 3] = 1.0
    return J


def estimate(moments, R, ratios):
    """E[f], the gradient with respect to theta and its standard error, computed by
    the library (sim_gradient_estimate) from the moment sums of run_moments
    ([n_chunks, F, 42] or [F, 42]).  Returns mean_f [F], grad [F, 4], se [F, 4]."""
    return B.gradient_estimate(moments, R, jacobian(ratios))


def score_gradient(spec: GradientSpec):
    m, R, _ = run_moments(spec)
    return estimate(m, R, spec.class_ratios())


def fd_gradient(spec: GradientSpec, rel_h=1e-3):
    """Central finite differences with common random numbers (same seeds at
    theta +- h).  Returns grad [F, 4] and its standard error from the paired
    per-replicate differences."""
    th = spec.theta()
    F = len(spec.days)
    grad = np.zeros((F, 4)); se = np.zeros((F, 4))
    for k in range(4):
        h = rel_h * abs(th[k]) if th[k] != 0 else rel_h
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        fp = _per_replicate_f(spec.with_theta(tp))
        fm = _per_replicate_f(spec.with_theta(tm))
        d = (fp - fm) / (2 * h)                                  # [R, F]
        grad[:, k] = d.mean(0)
        se[:, k] = d.std(0, ddof=1) / math.sqrt(d.shape[0])
    return grad, se


def _per_replicate_f(spec: GradientSpec):
    w = spec.w
    out = []
    for r0 in range(0, w.R, spec.chunk):
        r1 = min(w.R, r0 + spec.chunk)
        s = B.Sim(w.model, w.u0, w.phi0, _slice_params(w.params, r0, r1), w.T, seed=w.seed, replicate_base=r0)
        try:
            if len(w.events):
                s.load_events(w.events)
            s.run(w.T)
            pi, pn, _ = s.stats()
            out.append(pi[:, spec.days] / np.maximum(pn[:, spec.days], 1))
        finally:
            s.close()
    return np.concatenate(out)


def _autograd():
    import torch

    class ScoreFn(torch.autograd.Function):
        """E[f](theta) with a score-function backward: forward runs the replicates
        and returns the mean prevalence at the spec's days; backward multiplies the
        incoming gradient by the estimated Jacobian d E[f] / d theta."""

        @staticmethod
        def forward(ctx, theta, spec):
            th = theta.detach().cpu().double().numpy()
            mean_f, grad, _ = score_gradient(spec.with_theta(th))
            ctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(mean_f, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (J,) = ctx.saved_tensors
            return grad_out @ J, None

    return ScoreFn


_SCOREFN = None


def score_fn():
    global _SCOREFN
    if _SCOREFN is None:
        _SCOREFN = _autograd()
    return _SCOREFN
