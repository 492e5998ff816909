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


def build(force: bool = False) -> pathlib.Path:
    """Compiles oracle.c into _build/liboracle.so (gcc -O2, no FP contraction)."""
    _BUILD.mkdir(exist_ok=True)
    out = _BUILD / "liboracle.so"
    if force or not out.exists() or out.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", str(tmp), str(_SRC), "-lm"], check=True)
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


def compile_variant(source_text, out_path):
    """Compiles a modified copy of oracle.c (used by the tests that plant
    mistakes in the oracle to show that its pins catch them)."""
    src = pathlib.Path(out_path).with_suffix(".c")
    src.write_text(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", str(out_path), str(src), "-lm"], check=True)
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
