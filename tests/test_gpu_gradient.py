"""Score-function gradients on the GPU: against central finite differences with
common random numbers (the SISe workload at reduced size), and against the exact
gradient of a one-node, 10-animal SIS law computed by enumerating daily paths
with matrix exponentials."""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import gradient as G
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def test_score_gradient_agrees_with_central_differences():
    w = W.sise_plain(N=200, T=60, n_events=20 * 200 * 60 // 365, R=4096, upsilon=0.012, beta=0.05)
    spec = G.GradientSpec(w, np.array([29, 59]), chunk=2048)
    mean_f, g, se = G.score_gradient(spec)
    fd, fd_se = G.fd_gradient(spec, rel_h=1e-3)
    z = np.abs(g - fd) / np.sqrt(se ** 2 + fd_se ** 2)
    assert np.all(z < 3.0), (g, fd, se, fd_se)


def test_score_gradient_agrees_with_central_differences_at_gradient_workload_size():
    # the 10,000-node, 365-day gradient workload on 1,024 replicates: the final
    # prevalence and the 52 week-end prevalences, all four parameters (212
    # comparisons: none 4 standard errors apart, at most 3 beyond 3, where the
    # normal law expects 0.57); final and week 26 each within 3
    days = np.array([364] + [7 * k - 1 for k in range(1, 53)], np.int32)
    w = W.sise_gradient(R=1024)
    spec = G.GradientSpec(w, days, chunk=1024)
    _, g, se = G.score_gradient(spec)
    fd, fd_se = G.fd_gradient(spec, rel_h=1e-3)
    z = np.abs(g - fd) / np.sqrt(se ** 2 + fd_se ** 2)
    assert z.max() < 4.0 and (z >= 3.0).sum() <= 3, (z.max(), (z >= 3.0).sum())
    assert np.all(z[[0, 26]] < 3.0), (g[[0, 26]], fd[[0, 26]])


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


def test_ten_animal_node_gradient_matches_matrix_exponential():
    N, I0, ups, gam, alpha, beta, eps, phi0, T = 10, 2, 0.3, 0.4, 1.0, 0.2, 0.01, 0.5, 3
    R = 1 << 17
    w = W.tiny_node(model=W.SISE, herd=N, infected=I0, R=R, T=T, phi0=phi0,
                    params=dict(upsilon=ups, gamma=gam, alpha=alpha, beta=beta, epsilon=eps))
    spec = G.GradientSpec(w, np.array([T - 1]), chunk=R)
    mean_f, g, se = G.score_gradient(spec)
    base = dict(N=N, I0=I0, ups=ups, gam=gam, alpha=alpha, beta=beta, eps=eps, phi0=phi0, T=T)
    law = _sis_law(**base)
    assert abs(mean_f[0] - np.dot(np.arange(N + 1), law) / N) < 4 * math.sqrt(0.25 / R)
    for k, name in enumerate(("ups", "gam", "beta", "alpha")):
        h = 1e-6 * base[name]
        hi = dict(base); lo = dict(base)
        hi[name] += h; lo[name] -= h
        exact = (np.dot(np.arange(N + 1), _sis_law(**hi)) - np.dot(np.arange(N + 1), _sis_law(**lo))) / (2 * h) / N
        assert abs(g[0, k] - exact) < 4 * se[0, k], (name, g[0, k], exact, se[0, k])


def test_autograd_function_backward_is_the_estimated_jacobian():
    import torch
    w = W.sise_plain(N=100, T=30, n_events=500, R=512)
    spec = G.GradientSpec(w, np.array([29]), chunk=512)
    theta = torch.tensor(spec.theta(), dtype=torch.float64, requires_grad=True)
    f = G.score_fn().apply(theta, spec)
    f.sum().backward()
    _, g, _ = G.score_gradient(spec)
    assert np.allclose(theta.grad.numpy(), g.sum(0), rtol=1e-12, atol=0)
