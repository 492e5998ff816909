"""CPU oracle for the event-based SISe / SISe3 simulation (arXiv:1502.02908).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  The arithmetic
lives in ``oracle.c`` (plain C, single-threaded, no FMA contraction); this module
compiles it with gcc and wraps it with ctypes.

Functions with no independent pin: none.  Every routine is checked by
``tests/test_oracle_*.py`` (closed forms, a matrix-exponential law, invariants,
published Philox answers, 300-bit logarithms, brute-force sampling laws).
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess
import threading

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_SOURCES = [_HERE / "oracle.c", _HERE / "general.c"]
_HEADERS = [_HERE / "oracle_rng.h"]
_BUILD = _HERE / "_build"
_LIB = None
_LOCK = threading.Lock()


class OrcCfg(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("replicate", ctypes.c_int32), ("phi_pre_event", ctypes.c_int32),
                ("underflow_error", ctypes.c_int32), ("score", ctypes.c_int32),
                ("seed", ctypes.c_uint64),
                ("upsilon", ctypes.c_double * 3), ("gamma", ctypes.c_double * 3),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double * 4),
                ("epsilon", ctypes.c_double)]


class OrcCounters(ctypes.Structure):
    _fields_ = [("transitions", ctypes.c_int64), ("events_applied", ctypes.c_int64),
                ("events_clamped", ctypes.c_int64), ("events_skipped", ctypes.c_int64)]


GO_MAX_COMP, GO_MAX_TRANS, GO_MAX_CONT, GO_MAX_SELECT, GO_MAX_SHIFT = 16, 32, 4, 32, 32


class GoModel(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int32), ("n_trans", ctypes.c_int32), ("n_cont", ctypes.c_int32),
                ("n_select", ctypes.c_int32), ("n_shift", ctypes.c_int32), ("y_source", ctypes.c_int32),
                ("stoich", ctypes.c_int32 * (GO_MAX_COMP * GO_MAX_TRANS)),
                ("fa", ctypes.c_int32 * GO_MAX_TRANS), ("fb", ctypes.c_int32 * GO_MAX_TRANS),
                ("fy", ctypes.c_int32 * GO_MAX_TRANS), ("pop", ctypes.c_uint32 * GO_MAX_TRANS),
                ("num", ctypes.c_uint32 * GO_MAX_CONT), ("den", ctypes.c_uint32 * GO_MAX_CONT),
                ("select", ctypes.c_uint32 * GO_MAX_SELECT),
                ("shift", ctypes.c_int32 * (GO_MAX_SHIFT * GO_MAX_COMP))]


class GoCfg(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("replicate", ctypes.c_int32),
                ("underflow_error", ctypes.c_int32), ("pad", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("rate", ctypes.c_double * GO_MAX_TRANS), ("alpha", ctypes.c_double * GO_MAX_CONT),
                ("beta", (ctypes.c_double * 4) * GO_MAX_CONT), ("epsilon", ctypes.c_double * GO_MAX_CONT)]


def build(force: bool = False) -> pathlib.Path:
    """Compiles oracle.c into _build/liboracle.so (gcc -O2, no FP contraction)."""
    _BUILD.mkdir(exist_ok=True)
    out = _BUILD / "liboracle.so"
    newest = max(p.stat().st_mtime for p in _SOURCES + _HEADERS)
    if force or not out.exists() or out.stat().st_mtime < newest:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-I", str(_HERE),
                        "-o", str(tmp)] + [str(p) for p in _SOURCES] + ["-lm"], check=True)
        os.replace(tmp, out)
    return out


def load(path):
    """Loads a compiled oracle library and declares its C signatures."""
    L = ctypes.CDLL(str(path))
    P = ctypes.POINTER
    L.orc_run.restype = ctypes.c_int
    L.orc_run.argtypes = [P(OrcCfg), P(ctypes.c_int32), P(ctypes.c_double),
                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int64] + \
                         [P(ctypes.c_int32)] * 6 + \
                         [P(ctypes.c_int64), P(ctypes.c_int64), P(OrcCounters),
                          P(ctypes.c_double), P(ctypes.c_double)]
    L.orc_apply_events.restype = ctypes.c_int
    L.orc_apply_events.argtypes = [P(OrcCfg), P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_int64)] + \
                                  [P(ctypes.c_int32)] * 6 + [P(OrcCounters)]
    L.orc_ssa_nodes.restype = ctypes.c_int
    L.orc_ssa_nodes.argtypes = [P(OrcCfg), P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32, P(OrcCounters)]
    L.orc_phi_nodes.restype = ctypes.c_int
    L.orc_phi_nodes.argtypes = [P(OrcCfg), P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32]
    L.go_run.restype = ctypes.c_int
    L.go_run.argtypes = [P(GoModel), P(GoCfg), P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int32,
                         ctypes.c_int32, ctypes.c_int64] + [P(ctypes.c_int32)] * 7 + [P(OrcCounters)]
    L.orc_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
    L.orc_uniform.restype = ctypes.c_double
    L.orc_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.orc_neglog.restype = ctypes.c_double
    L.orc_neglog.argtypes = [ctypes.c_uint64]
    L.orc_neglog_q58.restype = ctypes.c_uint64
    L.orc_neglog_q58.argtypes = [ctypes.c_uint64]
    L.orc_logr_q62.restype = ctypes.c_int64
    L.orc_logr_q62.argtypes = [ctypes.c_int]
    L.orc_recip.restype = ctypes.c_int64
    L.orc_recip.argtypes = [ctypes.c_int]
    L.orc_ln2_q62.restype = ctypes.c_uint64
    L.orc_lemire_draw.restype = ctypes.c_uint32
    L.orc_lemire_draw.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32]
    return L


def compile_variant(source_text, out_path, which="oracle.c"):
    """Compiles the oracle with a modified copy of one of its sources (used by
    the tests that plant mistakes in the oracle to show that its pins catch them)."""
    src = pathlib.Path(out_path).with_suffix(".c")
    src.write_text(source_text)
    others = [str(p) for p in _SOURCES if p.name != which]
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-I", str(_HERE),
                    "-o", str(out_path), str(src)] + others + ["-lm"], check=True)
    return load(out_path)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = load(build())
    return _LIB


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def philox(ctr, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (two words)."""
    c = np.asarray(ctr, np.uint32); k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def neglog(j):
    return lib().orc_neglog(int(j))


def uniform(lo, hi):
    return lib().orc_uniform(int(lo), int(hi))


def make_cfg(model, N, params, r, seed, phi_pre_event=False, underflow_error=False, score=False):
    c = OrcCfg()
    c.model = model; c.n_nodes = N; c.replicate = r; c.seed = seed
    c.phi_pre_event = int(bool(phi_pre_event)); c.underflow_error = int(bool(underflow_error))
    c.score = int(bool(score))
    for j in range(3):
        c.upsilon[j] = float(params.upsilon[r, j]); c.gamma[j] = float(params.gamma[r, j])
    for s in range(4):
        c.beta[s] = float(params.beta[r, s])
    c.alpha = float(params.alpha[r]); c.epsilon = float(params.epsilon[r])
    return c


class Result:
    """Per-replicate results: counts [R, Nc, N], phi [R, N], prev_i / prev_n
    [R, ndays], counters [R, 4], per-node score terms [R, 8, N] (or None)."""

    def __init__(self, counts, phi, prev_i, prev_n, counters, score):
        self.counts, self.phi, self.prev_i, self.prev_n = counts, phi, prev_i, prev_n
        self.counters, self.score = counters, score


def run(w, ndays=None, d0=0, replicates=None, counts=None, phi=None, phi_pre_event=False,
        underflow_error=False, score=False, events=None, lib_handle=None):
    """Runs the oracle for the workload ``w`` (see paper_1502_02908_gb300.workloads).

    ``counts`` [R', Nc, N] / ``phi`` [R', N] override the initial state (default: u0 and
    phi0 for every replicate); ``replicates`` selects which replicate indices run.
    """
    ndays = w.T if ndays is None else ndays
    reps = list(range(w.R)) if replicates is None else list(replicates)
    ev = w.events if events is None else events
    nc = w.nc
    out_c = np.empty((len(reps), nc, w.N), np.int32)
    out_p = np.empty((len(reps), w.N), np.float64)
    pi = np.zeros((len(reps), ndays), np.int64)
    pn = np.zeros((len(reps), ndays), np.int64)
    ctrs = np.zeros((len(reps), 4), np.int64)
    sc = np.zeros((len(reps), 8, w.N), np.float64) if score else None
    evs = [np.ascontiguousarray(a, dtype=np.int32) for a in (ev.day, ev.kind, ev.node, ev.dest, ev.count, ev.cls)]
    L = lib_handle if lib_handle is not None else lib()
    for i, r in enumerate(reps):
        c = np.ascontiguousarray(w.u0 if counts is None else counts[i], dtype=np.int32).copy()
        p = np.ascontiguousarray(w.phi0 if phi is None else phi[i], dtype=np.float64).copy()
        cfg = make_cfg(w.model, w.N, w.params, r, w.seed, phi_pre_event, underflow_error, score)
        ctr = OrcCounters()
        s = np.zeros(8 * w.N, np.float64) if score else None
        tang = np.zeros(2 * w.N, np.float64) if score else None
        rc = L.orc_run(ctypes.byref(cfg), _ptr(c, ctypes.c_int32), _ptr(p, ctypes.c_double),
                       d0, ndays, len(ev), *[_ptr(a, ctypes.c_int32) for a in evs],
                       _ptr(pi[i], ctypes.c_int64), _ptr(pn[i], ctypes.c_int64), ctypes.byref(ctr),
                       _ptr(s, ctypes.c_double), _ptr(tang, ctypes.c_double))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        out_c[i] = c; out_p[i] = p
        ctrs[i] = (ctr.transitions, ctr.events_applied, ctr.events_clamped, ctr.events_skipped)
        if score:
            sc[i] = s.reshape(8, w.N)
    return Result(out_c, out_p, pi, pn, ctrs, sc)


def apply_events(w, counts, pos, events, replicate=0, underflow_error=False):
    """Applies ``events`` (already in the wanted order) to ``counts`` [Nc, N] in place,
    event k with Philox position pos[k]; returns the counters."""
    L = lib()
    cfg = make_cfg(w.model, w.N, w.params, replicate, w.seed, underflow_error=underflow_error)
    ctr = OrcCounters()
    pos = np.ascontiguousarray(pos, np.int64)
    arr = [np.ascontiguousarray(a, np.int32) for a in (events.day, events.kind, events.node, events.dest,
                                                       events.count, events.cls)]
    L.orc_apply_events(ctypes.byref(cfg), _ptr(counts, ctypes.c_int32), len(pos), _ptr(pos, ctypes.c_int64),
                       *[_ptr(a, ctypes.c_int32) for a in arr], ctypes.byref(ctr))
    return (ctr.transitions, ctr.events_applied, ctr.events_clamped, ctr.events_skipped)


def ssa_nodes(w, counts, phi, day, v0, v1, replicate=0):
    """The stochastic step of day ``day`` for nodes [v0, v1) of ``counts`` [Nc, N]
    (in place) with phi [N] frozen; returns the transitions fired."""
    L = lib()
    cfg = make_cfg(w.model, w.N, w.params, replicate, w.seed)
    ctr = OrcCounters()
    if L.orc_ssa_nodes(ctypes.byref(cfg), _ptr(counts, ctypes.c_int32), _ptr(phi, ctypes.c_double), int(day),
                       int(v0), int(v1), ctypes.byref(ctr)) != 0:
        raise ValueError("oracle rejected its arguments")
    return ctr.transitions


def phi_nodes(w, counts, phi, day, v0, v1, replicate=0):
    """The continuous-state update after day ``day`` for nodes [v0, v1) of phi [N]
    (in place) from ``counts`` [Nc, N]."""
    L = lib()
    cfg = make_cfg(w.model, w.N, w.params, replicate, w.seed)
    if L.orc_phi_nodes(ctypes.byref(cfg), _ptr(counts, ctypes.c_int32), _ptr(phi, ctypes.c_double), int(day),
                       int(v0), int(v1)) != 0:
        raise ValueError("oracle rejected its arguments")


def _go_model(m):
    g = GoModel()
    g.n_comp, g.n_trans, g.n_cont = m.nc, m.nt, m.ny
    g.n_select, g.n_shift, g.y_source = int(m.select.size), int(m.shift.shape[0]), int(m.y_source)
    for c in range(m.nc):
        for j in range(m.nt):
            g.stoich[c * m.nt + j] = int(m.stoich[c, j])
    for j in range(m.nt):
        g.fa[j], g.fb[j], g.fy[j], g.pop[j] = int(m.factor_a[j]), int(m.factor_b[j]), int(m.cont[j]), int(m.pop_mask[j])
    for q in range(m.ny):
        g.num[q], g.den[q] = int(m.num_mask[q]), int(m.den_mask[q])
    for s in range(m.select.size):
        g.select[s] = int(m.select[s])
    for s in range(m.shift.shape[0]):
        for c in range(m.nc):
            g.shift[s * GO_MAX_COMP + c] = int(m.shift[s, c])
    return g


class GeneralResult:
    """Per-replicate results: counts [R, Nc, N], y [R, Ny, N], counters [R, 4]."""

    def __init__(self, counts, y, counters):
        self.counts, self.y, self.counters = counts, y, counters


def run_general(w, ndays=None, d0=0, replicates=None, counts=None, y=None, events=None, model=None,
                lib_handle=None):
    """Runs the general-model oracle for the workload ``w``
    (paper_1502_02908_gb300.workloads.GeneralWorkload); ``counts`` [R', Nc, N] and
    ``y`` [R', Ny, N] override the initial state, ``model`` the descriptor."""
    m = w.model if model is None else model
    ndays = w.T if ndays is None else ndays
    reps = list(range(w.R)) if replicates is None else list(replicates)
    ev = w.events if events is None else events
    gm = _go_model(m)
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (ev.day, ev.kind, ev.node, ev.dest, ev.count,
                                                                ev.select, ev.shift)]
    out_c = np.empty((len(reps), m.nc, w.N), np.int32)
    out_y = np.empty((len(reps), m.ny, w.N), np.float64)
    ctrs = np.zeros((len(reps), 4), np.int64)
    L = lib_handle if lib_handle is not None else lib()
    for i, r in enumerate(reps):
        c = np.ascontiguousarray(w.u0 if counts is None else counts[i], dtype=np.int32).copy()
        yy = np.ascontiguousarray(w.y0 if y is None else y[i], dtype=np.float64).reshape(m.ny, w.N).copy()
        g = GoCfg()
        g.n_nodes, g.replicate, g.underflow_error, g.seed = w.N, r, int(bool(w.underflow_error)), w.seed
        for j in range(m.nt):
            g.rate[j] = float(w.rates[r, j])
        for q in range(m.ny):
            g.alpha[q] = float(w.var_params[r, q, 0])
            for s in range(4):
                g.beta[q][s] = float(w.var_params[r, q, 1 + s])
            g.epsilon[q] = float(w.var_params[r, q, 5])
        ctr = OrcCounters()
        rc = L.go_run(ctypes.byref(gm), ctypes.byref(g), _ptr(c, ctypes.c_int32),
                      _ptr(yy if m.ny else np.zeros(1), ctypes.c_double), d0, ndays, len(ev),
                      *[_ptr(a, ctypes.c_int32) for a in arrs], ctypes.byref(ctr))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        out_c[i] = c
        out_y[i] = yy
        ctrs[i] = (ctr.transitions, ctr.events_applied, ctr.events_clamped, ctr.events_skipped)
    return GeneralResult(out_c, out_y, ctrs)
