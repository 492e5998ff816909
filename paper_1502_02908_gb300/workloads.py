"""Seeded synthetic inputs for the SISe / SISe3 event-based simulation.

This module only draws inputs (herds, initial counts, per-replicate parameters
and scheduled-event lists).  It holds none of the simulation arithmetic, so both
the CUDA library and the CPU oracle can be fed from it.

The paper's workloads (Sec. 4.1: the VTEC O157 model on 37,221 Swedish herds with
register events; Sec. 4.2: a synthetic SIS benchmark) use data that is not
available here.  The generators below draw inputs with the same shape: heavy
tailed herd sizes, many more single-node (E1) than two-node (E2) events per day,
power-law sources and preferential-attachment destinations.  Every array comes
from ``numpy.random.Generator(PCG64(seed))``.

Compartment order inside one node is class-major: SISe ``[S, I]``; SISe3
``[S1, I1, S2, I2, S3, I3]`` (calves, young stock, adults).
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

SISE = 1
SISE3 = 3

EXIT, ENTER, INTERNAL, EXTERNAL = 0, 1, 2, 3


@dataclasses.dataclass
class Params:
    """Per-replicate model constants, arrays with a leading replicate axis.

    upsilon, gamma: [R, 3] (SISe uses column 0); alpha, epsilon: [R];
    beta: [R, 4] seasonal decay values for day-of-year bins
    [0, 91], (91, 182], (182, 273], (273, 364] (Sec. 4.1, seasonal beta).
    """
    upsilon: np.ndarray
    gamma: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    epsilon: np.ndarray

    @staticmethod
    def broadcast(R, upsilon, gamma, alpha, beta, epsilon):
        ups = np.zeros((R, 3)); gam = np.zeros((R, 3))
        u = np.atleast_1d(np.asarray(upsilon, dtype=np.float64))
        g = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
        ups[:, :u.size] = u; gam[:, :g.size] = g
        b = np.atleast_1d(np.asarray(beta, dtype=np.float64))
        bet = np.empty((R, 4)); bet[:] = b if b.size == 4 else b[0]
        return Params(ups, gam, np.full(R, float(alpha)), bet, np.full(R, float(epsilon)))

    def replicate(self, r):
        return Params(self.upsilon[r:r + 1].copy(), self.gamma[r:r + 1].copy(),
                      self.alpha[r:r + 1].copy(), self.beta[r:r + 1].copy(),
                      self.epsilon[r:r + 1].copy())


@dataclasses.dataclass
class Events:
    """Scheduled events as int32 structure-of-arrays (Sec. 3.2, E1/E2 records).

    kind: EXIT / ENTER / INTERNAL (aging, class cls -> cls+1) / EXTERNAL
    (node -> dest).  cls = -1 selects every class where sampling is involved.
    dest = -1 for single-node events.
    """
    day: np.ndarray
    kind: np.ndarray
    node: np.ndarray
    dest: np.ndarray
    count: np.ndarray
    cls: np.ndarray

    def __len__(self):
        return int(self.day.size)

    @staticmethod
    def empty():
        z = np.zeros(0, np.int32)
        return Events(z, z.copy(), z.copy(), z.copy(), z.copy(), z.copy())

    def select(self, mask):
        return Events(*(np.ascontiguousarray(getattr(self, f.name)[mask])
                        for f in dataclasses.fields(self)))

    def stable_by_day(self):
        order = np.argsort(self.day, kind="stable")
        return self.select(order)


@dataclasses.dataclass
class Workload:
    name: str
    model: int
    N: int
    T: int
    R: int
    u0: np.ndarray          # [Nc, N] int32
    phi0: np.ndarray        # [N] float64
    params: Params
    events: Events
    seed: int               # Philox key

    @property
    def nc(self):
        return 2 * (1 if self.model == SISE else 3)


def _round_half_even(x):
    return np.rint(x).astype(np.int64)


def _split_classes(herd, frac=(0.2, 0.2, 0.6)):
    """Largest-remainder split of each herd into three age classes."""
    herd = np.asarray(herd, np.int64)
    exact = herd[:, None] * np.asarray(frac)[None, :]
    base = np.floor(exact).astype(np.int64)
    rem = herd - base.sum(1)
    frac_part = exact - base
    # ties broken by class order (lower class first)
    order = np.argsort(-frac_part, axis=1, kind="stable")
    for k in range(3):
        give = rem > k
        rows = np.nonzero(give)[0]
        base[rows, order[rows, k]] += 1
    return base


def _initial_counts(model, herd, prevalence=0.05):
    if model == SISE:
        i0 = _round_half_even(prevalence * herd)
        return np.stack([herd - i0, i0]).astype(np.int32)
    cls = _split_classes(herd)
    out = np.zeros((6, herd.size), np.int32)
    for j in range(3):
        i0 = _round_half_even(prevalence * cls[:, j])
        out[2 * j] = cls[:, j] - i0
        out[2 * j + 1] = i0
    return out


def _uniform_events(rng, N, T, n_events, mix, max_count=5, aging=False):
    """Events with uniform day and node, destination uniform != node."""
    kinds = rng.choice(len(mix), size=n_events, p=np.asarray(mix, float))
    day = rng.integers(0, T, size=n_events)
    node = rng.integers(0, N, size=n_events)
    dest = rng.integers(0, N - 1, size=n_events)
    dest = dest + (dest >= node)                     # uniform over nodes != node
    count = rng.integers(1, max_count + 1, size=n_events)
    kind_map = np.array([EXIT, ENTER, EXTERNAL] if not aging else [EXIT, ENTER, INTERNAL, EXTERNAL])
    kind = kind_map[kinds]
    cls = np.where(kind == ENTER, 0, -1)
    dest = np.where(kind == EXTERNAL, dest, -1)
    ev = Events(day.astype(np.int32), kind.astype(np.int32), node.astype(np.int32),
                dest.astype(np.int32), count.astype(np.int32), cls.astype(np.int32))
    return ev.stable_by_day()


def sise_plain(N=1000, T=365, n_events=20_000, seed=1, R=1, herd_lo=20, herd_hi=200,
               upsilon=0.0357, gamma=0.1, alpha=1.0, beta=0.005, epsilon=1e-6, gen_seed=1):
    """SISe on N nodes, herds U{20..200}, 5% initial prevalence, phi0 = 0; events
    exit/enter/external 50/30/20 %, uniform day and node, 1-5 animals."""
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    herd = rng.integers(herd_lo, herd_hi + 1, size=N)
    u0 = _initial_counts(SISE, herd)
    ev = _uniform_events(rng, N, T, n_events, (0.5, 0.3, 0.2)) if n_events else Events.empty()
    params = Params.broadcast(R, upsilon, gamma, alpha, beta, epsilon)
    return Workload("sise_plain", SISE, N, T, R, u0, np.zeros(N), params, ev, seed)


def synthetic_sis(N=1000, T=1000, S0=1000, I0=1000, rho=0.1, k=16, count=1, seed=1, R=1, gen_seed=26):
    """The synthetic benchmark of Sec. 4.2: two compartments S and I on N nodes with
    S -> I and I -> S both at unit rate per animal, S = I = 1000 per node at the
    start, T daily windows.  As an SISe instance: upsilon = gamma = 1 and phi held
    at 1 (phi0 = 1, alpha = beta = epsilon = 0, so the update returns phi
    unchanged).  The nodes form k contiguous sub-domains; at the end of every day
    round(rho k (k-1) / 2) external transfers of `count` animals each connect a
    random node of one sub-domain to a random node of another (both drawn
    uniformly, the two sub-domains distinct).  The paper leaves the transfer size
    open; one animal by default."""
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    u0 = np.zeros((2, N), np.int32)
    u0[0] = S0
    u0[1] = I0
    m = int(round(rho * k * (k - 1) / 2))
    dom = (np.arange(N) * k) // N
    members = [np.nonzero(dom == d)[0] for d in range(k)]
    n_ev = m * T
    day = np.repeat(np.arange(T), m)
    a = rng.integers(0, k, size=n_ev)
    b = rng.integers(0, k - 1, size=n_ev)
    b = b + (b >= a)                                  # a different sub-domain
    src = np.array([members[x][rng.integers(0, members[x].size)] for x in a], dtype=np.int64)
    dst = np.array([members[x][rng.integers(0, members[x].size)] for x in b], dtype=np.int64)
    ev = Events(day.astype(np.int32), np.full(n_ev, EXTERNAL, np.int32), src.astype(np.int32),
                dst.astype(np.int32), np.full(n_ev, count, np.int32), np.full(n_ev, -1, np.int32))
    params = Params.broadcast(R, 1.0, 1.0, 0.0, 0.0, 0.0)
    return Workload("synthetic_sis", SISE, N, T, R, u0, np.ones(N), params, ev, seed)


VTEC_UPSILON = (8e-3, 7e-3, 1e-3)          # Sec. 4.1, per age class
VTEC_DELTA = (28.0, 25.0, 22.0)           # mean infectious period, days
VTEC_BETA_DIV = (14.0, 26.0, 20.0, 12.0)  # beta = log(2)/k per season


def vtec_beta():
    return np.array([math.log(2.0) / k for k in VTEC_BETA_DIV])


def _national_events(rng, N, T, n_events, herd, mix=(0.4, 0.3, 0.2, 0.1), max_count=5,
                     power=2.2, e1_source="herd"):
    """Register-shaped events.  Single-node events (exit, enter, aging) happen at
    nodes drawn in proportion to herd size (births, deaths and aging scale with the
    number of animals); external transfers leave nodes drawn with power-law weights
    (out-degree exponent 2.2) and arrive at destinations chosen by preferential
    attachment over the events in day order (P(j) ~ in-degree so far + 1,
    j != source).  e1_source="powerlaw" draws the single-node events with the
    power-law weights as well (a stress case: one small herd then carries a long
    chain of events every day)."""
    weights = rng.zipf(power, size=N).astype(np.float64)
    weights = np.minimum(weights, N)
    p_out = weights / weights.sum()
    hw = np.asarray(herd, np.float64)
    p_e1 = hw / hw.sum() if e1_source == "herd" else p_out
    kinds = rng.choice(4, size=n_events, p=np.asarray(mix, float))
    kind = np.array([EXIT, ENTER, INTERNAL, EXTERNAL])[kinds]
    day = rng.integers(0, T, size=n_events)
    node = rng.choice(N, size=n_events, p=p_e1)
    is_ext = kind == EXTERNAL
    node[is_ext] = rng.choice(N, size=int(is_ext.sum()), p=p_out)
    count = rng.integers(1, max_count + 1, size=n_events)
    cls = np.full(n_events, -1, np.int64)
    cls[kind == ENTER] = 0
    aging = kind == INTERNAL
    cls[aging] = rng.integers(0, 2, size=int(aging.sum()))
    order = np.argsort(day, kind="stable")
    day, kind, node, count, cls = day[order], kind[order], node[order], count[order], cls[order]
    dest = np.full(n_events, -1, np.int64)
    ext = np.nonzero(kind == EXTERNAL)[0]
    # urn holding each node (in-degree + 1) times; uniform picks from it are
    # preferential attachment
    urn = np.empty(N + ext.size, np.int64)
    urn[:N] = np.arange(N)
    size = N
    picks = rng.random(size=4 * ext.size + 16)
    pi = 0
    for e in ext:
        src = node[e]
        while True:
            if pi >= picks.size:
                picks = rng.random(size=picks.size)
                pi = 0
            j = urn[int(picks[pi] * size)]
            pi += 1
            if j != src:
                break
        dest[e] = j
        urn[size] = j
        size += 1
    return Events(day.astype(np.int32), kind.astype(np.int32), node.astype(np.int32),
                  dest.astype(np.int32), count.astype(np.int32), cls.astype(np.int32))


def sise3_national(N=37_000, T=1460, n_events=3_000_000, seed=1, R=1, gen_seed=2, e1_source="herd"):
    """SISe3 with VTEC O157 constants (Sec. 4.1) on a national-scale synthetic
    network: herds lognormal (median 50, sigma 1, capped at 5000) split 20/20/60
    into calves/young/adults, 5% infected per class; seasonal beta."""
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    herd = np.minimum(5000, np.maximum(1, _round_half_even(rng.lognormal(math.log(50.0), 1.0, size=N))))
    u0 = _initial_counts(SISE3, herd)
    ev = _national_events(rng, N, T, n_events, herd, e1_source=e1_source) if n_events else Events.empty()
    gam = [1.0 / d for d in VTEC_DELTA]
    params = Params.broadcast(R, VTEC_UPSILON, gam, 1.0, vtec_beta(), 1e-6)
    return Workload("sise3_national", SISE3, N, T, R, u0, np.zeros(N), params, ev, seed)


def sise3_batched(R=256, T=365, seed=1, base=None):
    """The national SISe3 network and its events for days [0, T), R replicates,
    each with its own (upsilon, gamma) log-uniform over +/-50% of the SISe
    values 0.0357 and 0.1, shared by the three age classes."""
    w = base if base is not None else sise3_national()
    ev = w.events.select(w.events.day < T)
    rng = np.random.Generator(np.random.PCG64(3))
    ups = np.exp(rng.uniform(math.log(0.5 * 0.0357), math.log(1.5 * 0.0357), size=R))
    gam = np.exp(rng.uniform(math.log(0.05), math.log(0.15), size=R))
    params = Params(np.repeat(ups[:, None], 3, 1), np.repeat(gam[:, None], 3, 1),
                    np.ones(R), np.repeat(vtec_beta()[None, :], R, 0), np.full(R, 1e-6))
    return Workload("sise3_batched", SISE3, w.N, T, R, w.u0.copy(), w.phi0.copy(), params, ev, seed)


def sise_gradient(N=10_000, R=4096, T=365, seed=4):
    """SISe, config-1 style herds and events at 20 events per node-year."""
    w = sise_plain(N=N, T=T, n_events=20 * N * T // 365, seed=seed, R=R, gen_seed=4)
    w.name = "sise_gradient"
    return w


def tiny_node(model=SISE, herd=10, infected=1, R=1, copies=1, **kw):
    """One herd (optionally repeated as independent nodes) with no events."""
    if model == SISE:
        u0 = np.array([[herd - infected], [infected]], np.int32)
    else:
        u0 = np.zeros((6, 1), np.int32)
        u0[0, 0] = herd - infected
        u0[1, 0] = infected
    u0 = np.repeat(u0, copies, axis=1)
    p = dict(upsilon=0.0, gamma=0.1, alpha=0.0, beta=0.0, epsilon=0.0)
    p.update(kw.pop("params", {}))
    params = Params.broadcast(R, **p)
    phi0 = np.full(copies, float(kw.pop("phi0", 0.0)))
    return Workload("tiny", model, copies, kw.pop("T", 1), R, u0, phi0, params,
                    Events.empty(), kw.pop("seed", 1))


def latin_hypercube(rng, n, lo, hi):
    """n points, one per stratum in every dimension, uniform within strata."""
    lo = np.asarray(lo, float); hi = np.asarray(hi, float)
    d = lo.size
    u = (np.stack([rng.permutation(n) for _ in range(d)], 1) + rng.random((n, d))) / n
    return lo + u * (hi - lo)


def _uniform_events_by_day(rng, N, T, n_events, mix, max_count=5):
    """The law of _uniform_events without its sort: i.i.d. events with uniform day
    and node (destination uniform != node) listed stably by day.  Sorting i.i.d.
    records by day leaves the other fields i.i.d. and independent of the days, and
    the number of events on each day multinomial, so the days are drawn as
    multinomial counts and every other field in list order."""
    per_day = rng.multinomial(n_events, np.full(T, 1.0 / T))
    day = np.repeat(np.arange(T, dtype=np.int32), per_day)
    kinds = np.searchsorted(np.cumsum(mix)[:-1], rng.random(n_events), side="right")
    node = rng.integers(0, N, size=n_events, dtype=np.int32)
    dest = rng.integers(0, N - 1, size=n_events, dtype=np.int32)
    dest += (dest >= node)
    count = rng.integers(1, max_count + 1, size=n_events, dtype=np.int32)
    kind = np.array([EXIT, ENTER, EXTERNAL], np.int32)[kinds]
    cls = np.where(kind == ENTER, 0, -1).astype(np.int32)
    dest = np.where(kind == EXTERNAL, dest, -1).astype(np.int32)
    return Events(day, kind, node, dest, count, cls)


def uneven_batch(n_inst=512, N_lo=100, N_hi=50_000, T_lo=90, T_hi=1460, events_per_node_year=80,
                 seed=5, R=1, threads=None):
    """Instances mixing SISe and SISe3 (probability 1/2 each), node counts
    log-uniform in [N_lo, N_hi], horizons uniform in [T_lo, T_hi], events at
    `events_per_node_year` with the plain SISe type mix (exit/enter/external
    50/30/20 %, no aging), and parameters from an n_inst-point Latin hypercube over
    log(upsilon, gamma, beta, alpha) in [0.5, 1.5] x (0.0357, 0.1, 0.005, 1.0).
    SISe3 instances use one (upsilon, gamma) for the three age classes.  Herds are
    U{20..200}, 5% infected (SISe3: split 20/20/60 by age).  The instance
    scalars come from one stream; each instance's arrays from a child stream of
    its own (numpy SeedSequence.spawn), so instances are generated in parallel
    (`threads`, default all cores) with the same result."""
    import concurrent.futures as cf
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.log([0.0357, 0.1, 0.005, 1.0])
    lhs = np.exp(latin_hypercube(rng, n_inst, base + np.log(0.5), base + np.log(1.5)))
    model = np.where(rng.random(n_inst) < 0.5, SISE, SISE3)
    Ns = np.rint(np.exp(rng.uniform(math.log(N_lo), math.log(N_hi), size=n_inst))).astype(np.int64)
    Ts = rng.integers(T_lo, T_hi + 1, size=n_inst)
    children = np.random.SeedSequence(seed).spawn(n_inst)

    def make(i):
        crng = np.random.Generator(np.random.PCG64(children[i]))
        m, N, T = int(model[i]), int(Ns[i]), int(Ts[i])
        herd = crng.integers(20, 201, size=N)
        u0 = _initial_counts(m, herd)
        n_ev = int(round(events_per_node_year * N * T / 365))
        ev = _uniform_events_by_day(crng, N, T, n_ev, (0.5, 0.3, 0.2)) if n_ev else Events.empty()
        ups, gam, bet, alp = lhs[i]
        na = 3 if m == SISE3 else 1
        params = Params.broadcast(R, [ups] * na, [gam] * na, alp, bet, 1e-6)
        return Workload(f"uneven_{i}", m, N, T, R, u0, np.zeros(N), params, ev, seed=1000 + i)

    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        return list(ex.map(make, range(n_inst)))


# ------------------------------------------------------------------ general model
# Inputs of the general compartment model (include/episim_general.h): a model
# descriptor (stoichiometry, propensity factors, continuous variables, event
# compartment masks and offsets), initial state, per-replicate constants and
# events.  Descriptors are data; the arithmetic they describe lives in the
# library and the oracle.

Y_POST_EVENT, Y_PRE_EVENT, Y_MIDPOINT = 0, 1, 2


@dataclasses.dataclass
class GeneralModel:
    """stoich [Nc, Nt] int32; per transition factor_a, factor_b (compartment or
    -1), cont (continuous variable or -1), pop_mask (uint32, 0: no division);
    per variable num_mask, den_mask; select [n_select] compartment masks;
    shift [n_shift, Nc] compartment offsets; y_source Y_*."""
    comps: tuple
    stoich: np.ndarray
    factor_a: np.ndarray
    factor_b: np.ndarray
    cont: np.ndarray
    pop_mask: np.ndarray
    num_mask: np.ndarray
    den_mask: np.ndarray
    select: np.ndarray
    shift: np.ndarray
    y_source: int = Y_POST_EVENT

    @property
    def nc(self):
        return int(self.stoich.shape[0])

    @property
    def nt(self):
        return int(self.stoich.shape[1])

    @property
    def ny(self):
        return int(self.num_mask.size)


def general_model(comps, transitions, variables=(), selects=(), shifts=(), y_source=Y_POST_EVENT):
    """Builds a GeneralModel from names.  transitions: dicts with "change"
    {compartment: delta}, optional "a", "b" (compartment names), "cont" (variable
    index) and "pop" (compartment names).  variables: (numerator names,
    denominator names).  selects: tuples of names.  shifts: {name: offset}."""
    idx = {c: i for i, c in enumerate(comps)}
    nc, nt = len(comps), len(transitions)

    def mask(names):
        m = 0
        for n in names:
            m |= 1 << idx[n]
        return m

    stoich = np.zeros((nc, nt), np.int32)
    fa = np.full(nt, -1, np.int32); fb = np.full(nt, -1, np.int32); fy = np.full(nt, -1, np.int32)
    pop = np.zeros(nt, np.uint32)
    for j, t in enumerate(transitions):
        for c, d in t["change"].items():
            stoich[idx[c], j] = d
        if "a" in t: fa[j] = idx[t["a"]]
        if "b" in t: fb[j] = idx[t["b"]]
        if "cont" in t: fy[j] = t["cont"]
        if "pop" in t: pop[j] = mask(t["pop"])
    num = np.array([mask(v[0]) for v in variables], np.uint32)
    den = np.array([mask(v[1]) for v in variables], np.uint32)
    sel = np.array([mask(s) for s in selects], np.uint32)
    sh = np.zeros((len(shifts), nc), np.int32)
    for s, offs in enumerate(shifts):
        for c, o in offs.items():
            sh[s, idx[c]] = o
    return GeneralModel(tuple(comps), stoich, fa, fb, fy, pop, num, den, sel, sh, y_source)


@dataclasses.dataclass
class GeneralEvents:
    """int32 structure of arrays: day, kind (EXIT/ENTER/INTERNAL/EXTERNAL), node,
    dest (-1 unless EXTERNAL), count, select (mask index), shift (-1: none)."""
    day: np.ndarray
    kind: np.ndarray
    node: np.ndarray
    dest: np.ndarray
    count: np.ndarray
    select: np.ndarray
    shift: np.ndarray

    def __len__(self):
        return int(self.day.size)

    @staticmethod
    def empty():
        z = np.zeros(0, np.int32)
        return GeneralEvents(*(z.copy() for _ in range(7)))

    def take(self, mask):
        return GeneralEvents(*(np.ascontiguousarray(getattr(self, f.name)[mask])
                               for f in dataclasses.fields(self)))


@dataclasses.dataclass
class GeneralWorkload:
    name: str
    model: GeneralModel
    N: int
    T: int
    R: int
    u0: np.ndarray           # [Nc, N] int32
    y0: np.ndarray           # [Ny, N] float64
    rates: np.ndarray        # [R, Nt] float64
    var_params: np.ndarray   # [R, Ny, 6]: alpha, beta[4], epsilon
    events: GeneralEvents
    seed: int
    underflow_error: bool = False


def _var_params(R, ny, alpha, beta, epsilon):
    vp = np.zeros((R, ny, 6))
    for q in range(ny):
        b = np.atleast_1d(np.asarray(beta[q], float))
        vp[:, q, 0] = alpha[q]
        vp[:, q, 1:5] = b if b.size == 4 else b[0]
        vp[:, q, 5] = epsilon[q]
    return vp


def _general_events(rng, N, T, n_events, spec):
    """spec: list of (probability, kind, select choices, shift choices); day and
    node uniform, dest uniform != node for EXTERNAL, 1-5 animals (stable by day)."""
    p = np.array([s[0] for s in spec], float)
    which = rng.choice(len(spec), size=n_events, p=p / p.sum())
    day = rng.integers(0, T, size=n_events)
    node = rng.integers(0, N, size=n_events)
    dest = rng.integers(0, N - 1, size=n_events)
    dest = dest + (dest >= node)
    count = rng.integers(1, 6, size=n_events)
    kind = np.array([s[1] for s in spec])[which]
    sel = np.empty(n_events, np.int64); sh = np.empty(n_events, np.int64)
    for i, (_, _, sels, shs) in enumerate(spec):
        rows = np.nonzero(which == i)[0]
        sel[rows] = np.asarray(sels)[rng.integers(0, len(sels), size=rows.size)]
        sh[rows] = np.asarray(shs)[rng.integers(0, len(shs), size=rows.size)]
    dest = np.where(kind == EXTERNAL, dest, -1)
    order = np.argsort(day, kind="stable")
    return GeneralEvents(*(a[order].astype(np.int32) for a in (day, kind, node, dest, count, sel, sh)))


def sir_general(N=2000, T=60, n_events=10_000, R=1, freq=True, beta=0.4, gamma=0.1, seed=1, gen_seed=11,
                herd_lo=20, herd_hi=200):
    """The SIR example of Eq. (SIRstoich): S + I -> 2I at beta S I (divided by the
    node's population when freq), I -> R at gamma I.  Events: exits of any
    animal, entries of susceptibles, vaccination S -> R (an internal move by
    offset +2), transfers of any animal."""
    m = general_model(("S", "I", "R"),
                      [dict(change={"S": -1, "I": 1}, a="S", b="I", **({"pop": ("S", "I", "R")} if freq else {})),
                       dict(change={"I": -1, "R": 1}, a="I")],
                      selects=[("S", "I", "R"), ("S",)], shifts=[{"S": 2}])
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    herd = rng.integers(herd_lo, herd_hi + 1, size=N)
    i0 = _round_half_even(0.05 * herd)
    u0 = np.stack([herd - i0, i0, np.zeros(N, np.int64)]).astype(np.int32)
    spec = [(0.4, EXIT, [0], [-1]), (0.3, ENTER, [1], [-1]), (0.1, INTERNAL, [1], [0]), (0.2, EXTERNAL, [0], [-1])]
    ev = _general_events(rng, N, T, n_events, spec) if n_events else GeneralEvents.empty()
    rates = np.tile(np.array([beta, gamma]), (R, 1))
    return GeneralWorkload("sir", m, N, T, R, u0, np.zeros((0, N)), rates, np.zeros((R, 0, 6)), ev, seed)


def seirs_env(N=3000, T=90, n_events=30_000, R=2, y_source=Y_POST_EVENT, seed=1, gen_seed=13):
    """SEIRS with two continuous variables: y0 an environmental load fed by the
    prevalence I/N (as phi in Eq. siminfpressure), y1 an exposure pressure fed by
    the count E with no division.  Transitions: S -> E at k0 y0 S, at k1 S I / N
    and at k5 y1 S; E -> I at k2 E; I -> R at k3 I; R -> S at k4 R.  Events:
    exits (any animal), entries (susceptibles), vaccination S -> R (offset +3),
    transfers (any animal, or only S and E)."""
    comps = ("S", "E", "I", "R")
    allc = comps
    m = general_model(comps,
                      [dict(change={"S": -1, "E": 1}, a="S", cont=0),
                       dict(change={"S": -1, "E": 1}, a="S", b="I", pop=allc),
                       dict(change={"E": -1, "I": 1}, a="E"),
                       dict(change={"I": -1, "R": 1}, a="I"),
                       dict(change={"R": -1, "S": 1}, a="R"),
                       dict(change={"S": -1, "E": 1}, a="S", cont=1)],
                      variables=[(("I",), allc), (("E",), ())],
                      selects=[allc, ("S",), ("S", "E")], shifts=[{"S": 3}], y_source=y_source)
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    herd = np.minimum(2000, np.maximum(1, _round_half_even(rng.lognormal(math.log(60.0), 1.0, size=N))))
    e0 = _round_half_even(0.02 * herd); i0 = _round_half_even(0.03 * herd)
    u0 = np.stack([herd - e0 - i0, e0, i0, np.zeros(N, np.int64)]).astype(np.int32)
    y0 = np.stack([rng.uniform(0.0, 0.05, size=N), np.zeros(N)])
    spec = [(0.35, EXIT, [0], [-1]), (0.3, ENTER, [1], [-1]), (0.1, INTERNAL, [1], [0]),
            (0.25, EXTERNAL, [0, 2], [-1])]
    ev = _general_events(rng, N, T, n_events, spec) if n_events else GeneralEvents.empty()
    base = np.array([0.02, 0.3, 0.2, 0.1, 0.01, 1e-4])
    rates = base[None, :] * np.exp(rng.uniform(-0.3, 0.3, size=(R, base.size)))
    vp = _var_params(R, 2, alpha=(1.0, 0.5), beta=(vtec_beta(), 0.2), epsilon=(1e-6, 0.0))
    return GeneralWorkload("seirs_env", m, N, T, R, u0, y0, rates, vp, ev, seed)


def erlang_sis(N=1500, T=40, n_events=8_000, stages=8, R=1, seed=1, gen_seed=17):
    """SIS-like model with an Erlang-distributed infectious period: S, I1..Ik, R.
    Infection S -> I1 at k0 y0 S (y0 the prevalence-fed environment) and at
    k1 S I1 / N; progression I_i -> I_(i+1) and Ik -> R at k2 per animal; loss
    of immunity R -> S at k3 R.  k + 3 transitions (11 for k = 8)."""
    comps = ("S",) + tuple(f"I{i + 1}" for i in range(stages)) + ("R",)
    inf = comps[1:-1]
    tr = [dict(change={"S": -1, "I1": 1}, a="S", cont=0),
          dict(change={"S": -1, "I1": 1}, a="S", b="I1", pop=comps)]
    for i in range(stages):
        nxt = comps[i + 2]
        tr.append(dict(change={comps[i + 1]: -1, nxt: 1}, a=comps[i + 1]))
    tr.append(dict(change={"R": -1, "S": 1}, a="R"))
    m = general_model(comps, tr, variables=[(inf, comps)], selects=[comps, ("S",)])
    rng = np.random.Generator(np.random.PCG64(gen_seed))
    herd = rng.integers(20, 400, size=N)
    u0 = np.zeros((len(comps), N), np.int32)
    i1 = _round_half_even(0.05 * herd)
    u0[0] = herd - i1; u0[1] = i1
    spec = [(0.4, EXIT, [0], [-1]), (0.3, ENTER, [1], [-1]), (0.3, EXTERNAL, [0], [-1])]
    ev = _general_events(rng, N, T, n_events, spec) if n_events else GeneralEvents.empty()
    rates = np.tile(np.array([0.05, 0.2] + [float(stages) / 10.0] * stages + [0.02]), (R, 1))
    vp = _var_params(R, 1, alpha=(1.0,), beta=(0.1,), epsilon=(1e-6,))
    return GeneralWorkload("erlang_sis", m, N, T, R, u0, np.zeros((1, N)), rates, vp, ev, seed)


def sise_model(y_source=Y_POST_EVENT, n_age=1):
    """SISe (n_age 1) or SISe3 (n_age 3) in the general form: per class j,
    S_j -> I_j at upsilon_j phi S_j and I_j -> S_j at gamma_j I_j, transitions in
    the order inf_1, rec_1, inf_2, ...; phi fed by sum I / sum (S + I).  Event
    masks: 0 every compartment, 1 + j class j, 1 + n_age + j the S of class j;
    offset row 0 moves a class up by one (aging)."""
    comps = tuple(c for j in range(n_age) for c in (f"S{j + 1}", f"I{j + 1}"))
    tr = []
    for j in range(n_age):
        s, i = f"S{j + 1}", f"I{j + 1}"
        tr.append(dict(change={s: -1, i: 1}, a=s, cont=0))
        tr.append(dict(change={i: -1, s: 1}, a=i))
    sel = [comps] + [(f"S{j + 1}", f"I{j + 1}") for j in range(n_age)] + [(f"S{j + 1}",) for j in range(n_age)]
    shifts = [{c: 2 for c in comps}] if n_age > 1 else []
    infected = tuple(f"I{j + 1}" for j in range(n_age))
    return general_model(comps, tr, variables=[(infected, comps)], selects=sel, shifts=shifts, y_source=y_source)


def as_general(w, y_source=Y_POST_EVENT):
    """An SISe / SISe3 workload in the general form (same counts, phi, constants
    and events).  Event cls maps to the class mask (cls = -1: every compartment),
    enter to the S of its class, aging to the class mask with offset row 0."""
    na = 1 if w.model == SISE else 3
    m = sise_model(y_source, na)
    ev = w.events
    cls = ev.cls.astype(np.int64)
    sel = np.where(cls < 0, 0, 1 + cls)
    sel = np.where(ev.kind == ENTER, 1 + na + np.maximum(cls, 0), sel)
    sh = np.where(ev.kind == INTERNAL, 0, -1)
    gev = GeneralEvents(ev.day.copy(), ev.kind.copy(), ev.node.copy(), ev.dest.copy(), ev.count.copy(),
                        sel.astype(np.int32), sh.astype(np.int32))
    rates = np.zeros((w.R, 2 * na))
    for j in range(na):
        rates[:, 2 * j] = w.params.upsilon[:, j]
        rates[:, 2 * j + 1] = w.params.gamma[:, j]
    vp = np.zeros((w.R, 1, 6))
    vp[:, 0, 0] = w.params.alpha
    vp[:, 0, 1:5] = w.params.beta
    vp[:, 0, 5] = w.params.epsilon
    return GeneralWorkload(w.name + "_general", m, w.N, w.T, w.R, w.u0.copy(), w.phi0[None, :].copy(), rates, vp,
                           gev, w.seed)
