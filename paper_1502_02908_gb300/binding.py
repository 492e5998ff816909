"""ctypes binding of libepisim (include/episim.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing or no CUDA
device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import pathlib
import threading

import numpy as np

from . import workloads as W

_LIB = None
_LOCK = threading.Lock()
HEADER = pathlib.Path(__file__).resolve().parent.parent / "include" / "episim.h"

SIM_OK, SIM_E_INVALID_ARG, SIM_E_OOM, SIM_E_CUDA, SIM_E_UNDERFLOW, SIM_E_TIMEOUT, SIM_E_STATE = range(7)
# moment sums per day written by sim_gradient_moments (see include/episim.h)
N_MOMENTS = 42
SIM_HOST, SIM_DEVICE = 0, 1
FLAG_PHI_PRE_EVENT, FLAG_SCORE, FLAG_SCORE_REVERSE = 1, 2, 4
STATUS_NAMES = {0: "SIM_OK", 1: "SIM_E_INVALID_ARG", 2: "SIM_E_OOM", 3: "SIM_E_CUDA",
                4: "SIM_E_UNDERFLOW", 5: "SIM_E_TIMEOUT", 6: "SIM_E_STATE"}


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SimConfig(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("n_replicates", ctypes.c_int32), ("max_days", ctypes.c_int32),
                ("underflow_policy", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("replicate_base", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SimParams(ctypes.Structure):
    _fields_ = [("upsilon", ctypes.POINTER(ctypes.c_double)), ("gamma", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("epsilon", ctypes.POINTER(ctypes.c_double))]


class GenModel(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int32), ("n_trans", ctypes.c_int32), ("n_cont", ctypes.c_int32),
                ("n_select", ctypes.c_int32), ("n_shift", ctypes.c_int32), ("y_source", ctypes.c_int32),
                ("stoich", ctypes.POINTER(ctypes.c_int32)), ("trans", ctypes.POINTER(ctypes.c_int32)),
                ("vars", ctypes.POINTER(ctypes.c_uint32)), ("select", ctypes.POINTER(ctypes.c_uint32)),
                ("shift", ctypes.POINTER(ctypes.c_int32))]


class GenConfig(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_replicates", ctypes.c_int32), ("max_days", ctypes.c_int32),
                ("underflow_policy", ctypes.c_int32), ("seed", ctypes.c_uint64), ("replicate_base", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


GEN_OPT_LAUNCH, GEN_OPT_WARP_THRESHOLD, GEN_OPT_GROUP_THRESHOLD, GEN_OPT_CLOCK_MARGIN = 1, 2, 3, 4


def library_path() -> pathlib.Path:
    from .build import LIB
    return LIB


def load_library(build_if_missing: bool = True):
    """Loads libepisim.so (building it first when missing)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = library_path()
        if not path.exists():
            if not build_if_missing:
                raise FileNotFoundError(f"{path} not built")
            from .build import build
            build()
        L = ctypes.CDLL(str(path))
        P, i32, i64, vp = ctypes.POINTER, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        pi32, pi64, pd = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_double)
        sigs = {
            "sim_create": [P(SimConfig), pi32, pd, P(SimParams), P(vp)],
            "sim_create_on": [P(SimConfig), pi32, pd, P(SimParams), vp, vp, vp, P(vp)],
            "sim_load_events": [vp, i64, pi32, pi32, pi32, pi32, pi32, pi32],
            "sim_run_days": [vp, i32, vp],
            "sim_sync": [vp, vp],
            "sim_state": [vp, vp, vp, pi32, i32, vp],
            "sim_set_state": [vp, vp, vp, i32, i32, vp],
            "sim_stats": [vp, pi64, pi64, pi64, vp],
            "sim_score": [vp, pd, vp],
            "sim_reset": [vp, i32],
            "sim_schedule_events": [i32, i32, i32, i64, pi32, pi32, pi32, pi32, pi32, pi32, pi64, pi32, pi64],
            "sim_debug_neglog": [vp, vp, i64],
            "sim_debug_neglog_f32": [vp, vp, i64],
            "sim_debug_div": [vp, vp, vp, vp, i64, i32],
            "sim_debug_schedule": [vp, pi64, pi32],
            "sim_profile": [vp, i32],
            "sim_debug_event_variant": [vp, i32],
            "sim_tune": [vp, i32],
            "sim_score_backward": [vp, vp],
            "sim_gradient_moments": [vp, pi32, i32, pd, pd, vp],
            "sim_gradient_moments_noalloc": [vp, pi32, i32, pd, pd, vp],
            "sim_gradient_estimate": [pd, i32, i32, i64, pd, i32, pd, pd, pd],
            "sim_fp64_peak": [i32, i64, pd, pd],
            "sim_shard": [vp, i32, i32],
            "sim_run_day_stochastic": [vp, vp],
            "sim_run_day_events": [vp, vp],
            "sim_touched_nodes": [vp, i32, pi32],
            "sim_pack_touched": [vp, vp, vp],
            "sim_unpack_touched": [vp, vp, i32, pi32, vp],
            "sim_run_batch": [P(vp), i32, pi32, vp],
            "sim_batch_shape": [i32, i32],
            "sim_set_option": [vp, i32, i64],
            "sim_set_regions": [vp, pi32, i32],
            "sim_set_params": [vp, vp],
            "sim_region_moments": [vp, vp, vp],
            "sim_goal": [vp, pi64, i32, i32, pd, pd],
            "sim_debug_batch_spin_limit": [i64],
            "sim_debug_batch_stall": [vp, i32, i64],
            "sim_debug_flow_stall": [vp, i32, i64],
            "sim_profile_read": [vp, pd, pi64],
            "gen_model_check": [P(GenModel), P(ctypes.c_uint32)],
            "gen_create": [P(GenModel), P(GenConfig), pi32, pd, pd, pd, P(vp)],
            "gen_load_events": [vp, i64, pi32, pi32, pi32, pi32, pi32, pi32, pi32],
            "gen_run_days": [vp, i32, vp],
            "gen_state": [vp, vp, vp, pi32, i32, vp],
            "gen_set_state": [vp, vp, vp, i32, i32, vp],
            "gen_counters": [vp, pi64],
            "gen_set_option": [vp, i32, i64],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sim_destroy.argtypes = [vp]
        L.sim_destroy.restype = None
        L.sim_last_error.argtypes = [vp]
        L.sim_last_error.restype = ctypes.c_char_p
        L.gen_destroy.argtypes = [vp]
        L.gen_destroy.restype = None
        L.gen_last_error.argtypes = [vp]
        L.gen_last_error.restype = ctypes.c_char_p
        L.gen_warp_nodes.argtypes = [vp]
        L.gen_warp_nodes.restype = ctypes.c_int32
        L.gen_group_nodes.argtypes = [vp]
        L.gen_group_nodes.restype = ctypes.c_int32
        L.sim_warp_nodes.argtypes = [vp]
        L.sim_warp_nodes.restype = ctypes.c_int32
        L.sim_touched_count.argtypes = [vp, i32]
        L.sim_touched_count.restype = ctypes.c_int32
        L.sim_debug_schedule_size.argtypes = [vp]
        L.sim_debug_schedule_size.restype = ctypes.c_int64
        _LIB = L
        return L


def header_symbols():
    """Names of the functions the headers under include/ declare."""
    import re
    names = set()
    for hdr in sorted(HEADER.parent.glob("*.h")):
        names |= set(re.findall(r"^\s*(?:sim_status|void|const char\*|int64_t|int32_t)\s+((?:sim|gen)_\w+)\s*\(",
                                hdr.read_text(), re.M))
    return sorted(names)


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _check(L, h, status):
    if status != SIM_OK:
        msg = L.sim_last_error(h)
        raise SimError(status, msg.decode() if msg else "")


def gradient_estimate(chunks, R: int, jac):
    """The score-function estimate from moment sums (sim_gradient_estimate):
    chunks [n_chunks, F, 42] (each a sim_gradient_moments result, added in chunk
    order), R replicates in all, jac [8, P].  Returns mean_f [F], grad [F, P],
    se [F, P]."""
    L = load_library()
    m = np.ascontiguousarray(chunks, np.float64)
    if m.ndim == 2:
        m = m[None]
    J = np.ascontiguousarray(jac, np.float64)
    F, P = m.shape[1], J.shape[1]
    mean_f = np.zeros(F)
    grad = np.zeros((F, P))
    se = np.zeros((F, P))
    st = L.sim_gradient_estimate(_p(m, ctypes.c_double), m.shape[0], F, int(R), _p(J, ctypes.c_double), P,
                                 _p(mean_f, ctypes.c_double), _p(grad, ctypes.c_double), _p(se, ctypes.c_double))
    if st != SIM_OK:
        raise SimError(st, "sim_gradient_estimate: invalid arguments")
    return mean_f, grad, se


def fp64_peak(kind: int = 0, iters: int = 1 << 16):
    """Measured FP64 instruction-lane throughput of the current device (lane-ops/s)
    and the best launch's time in ms (sim_fp64_peak; kind 0 = FMA, 1 = add)."""
    L = load_library()
    v = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    st = L.sim_fp64_peak(int(kind), int(iters), ctypes.byref(v), ctypes.byref(ms))
    if st != SIM_OK:
        raise SimError(st, "sim_fp64_peak failed")
    return v.value, ms.value


def current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def schedule_events(events: W.Events, n_nodes: int, model: int, max_days: int):
    """Host-only event preprocessing: (order, level) in execution order."""
    L = load_library()
    n = len(events)
    order = np.zeros(max(n, 1), np.int64)
    level = np.zeros(max(n, 1), np.int32)
    ns = ctypes.c_int64(0)
    arr = [np.ascontiguousarray(a, np.int32) for a in (events.day, events.kind, events.node, events.dest,
                                                       events.count, events.cls)]
    st = L.sim_schedule_events(n_nodes, model, max_days, n, *[_p(a, ctypes.c_int32) for a in arr],
                               _p(order, ctypes.c_int64), _p(level, ctypes.c_int32), ctypes.byref(ns))
    _check(L, None, st)
    return order[:ns.value].copy(), level[:ns.value].copy()


class Sim:
    """One simulation handle: R replicates of one model on N nodes.  With
    ``state=(counts, phi)`` (device tensors int32 [R, Nc, N] and float64 [R, N],
    contiguous) the live state is those tensors' storage (sim_create_on)."""

    def __init__(self, model, u0, phi0, params: W.Params, max_days, seed=1,
                 underflow_error=False, phi_pre_event=False, score=False, replicate_base=0,
                 score_reverse=False, state=None):
        self.L = load_library()
        u0 = np.ascontiguousarray(u0, np.int32)
        self.nc, self.N = u0.shape
        self.model = model
        self.R = params.upsilon.shape[0]
        self.max_days = max_days
        cfg = SimConfig(model, self.N, self.R, max_days, 1 if underflow_error else 0,
                        (FLAG_PHI_PRE_EVENT if phi_pre_event else 0) | (FLAG_SCORE if score else 0)
                        | (FLAG_SCORE_REVERSE if score_reverse else 0), seed,
                        int(replicate_base), 0)
        self._keep = [np.ascontiguousarray(x, np.float64) for x in
                      (params.upsilon, params.gamma, params.alpha, params.beta, params.epsilon)]
        sp = SimParams(*[_p(a, ctypes.c_double) for a in self._keep])
        h = ctypes.c_void_p()
        phi0 = np.ascontiguousarray(phi0, np.float64)
        if state is None:
            _check(self.L, None, self.L.sim_create(ctypes.byref(cfg), _p(u0, ctypes.c_int32),
                                                   _p(phi0, ctypes.c_double), ctypes.byref(sp), ctypes.byref(h)))
        else:
            counts_t, phi_t = state
            if tuple(counts_t.shape) != (self.R, self.nc, self.N) or tuple(phi_t.shape) != (self.R, self.N) or \
                    not counts_t.is_contiguous() or not phi_t.is_contiguous():
                raise ValueError("state tensors must be contiguous [R, Nc, N] int32 and [R, N] float64")
            import torch
            if counts_t.dtype != torch.int32 or phi_t.dtype != torch.float64:
                raise ValueError("state tensors must be int32 and float64")
            self._state = state                      # keep the storage alive with the handle
            _check(self.L, None, self.L.sim_create_on(ctypes.byref(cfg), _p(u0, ctypes.c_int32),
                                                      _p(phi0, ctypes.c_double), ctypes.byref(sp),
                                                      ctypes.c_void_p(counts_t.data_ptr()),
                                                      ctypes.c_void_p(phi_t.data_ptr()), current_stream(),
                                                      ctypes.byref(h)))
        self.h = h

    @classmethod
    def from_workload(cls, w: W.Workload, events=True, max_days=None, global_events=False, event_variant=None, **kw):
        s = cls(w.model, w.u0, w.phi0, w.params, w.T if max_days is None else max_days, seed=w.seed, **kw)
        if global_events:
            _check(s.L, s.h, s.L.sim_debug_event_variant(s.h, 1))
        if event_variant is not None:
            _check(s.L, s.h, s.L.sim_debug_event_variant(s.h, int(event_variant)))
        if events and len(w.events):
            s.load_events(w.events)
        return s

    def _stream(self, stream):
        if stream is None:
            return current_stream()
        return ctypes.c_void_p(stream)

    def load_events(self, ev: W.Events):
        arr = [np.ascontiguousarray(a, np.int32) for a in (ev.day, ev.kind, ev.node, ev.dest, ev.count, ev.cls)]
        _check(self.L, self.h, self.L.sim_load_events(self.h, len(ev), *[_p(a, ctypes.c_int32) for a in arr]))

    def run(self, days, stream=None):
        _check(self.L, self.h, self.L.sim_run_days(self.h, int(days), self._stream(stream)))

    def sync(self, stream=None):
        _check(self.L, self.h, self.L.sim_sync(self.h, self._stream(stream)))

    def state(self, stream=None):
        counts = np.empty((self.R, self.nc, self.N), np.int32)
        phi = np.empty((self.R, self.N), np.float64)
        day = ctypes.c_int32(0)
        _check(self.L, self.h, self.L.sim_state(self.h, _p(counts, ctypes.c_int32), _p(phi, ctypes.c_double),
                                                ctypes.byref(day), SIM_HOST, self._stream(stream)))
        return counts, phi, day.value

    def state_device(self, counts_t, phi_t, stream=None):
        """Copies the state into torch CUDA tensors (int32 [R,Nc,N], float64 [R,N])."""
        day = ctypes.c_int32(0)
        _check(self.L, self.h, self.L.sim_state(self.h, ctypes.c_void_p(counts_t.data_ptr()),
                                                ctypes.c_void_p(phi_t.data_ptr()), ctypes.byref(day),
                                                SIM_DEVICE, self._stream(stream)))
        return day.value

    def set_state(self, counts, phi, day, stream=None):
        counts = np.ascontiguousarray(counts, np.int32)
        phi = np.ascontiguousarray(phi, np.float64)
        _check(self.L, self.h, self.L.sim_set_state(self.h, counts.ctypes.data_as(ctypes.c_void_p),
                                                    phi.ctypes.data_as(ctypes.c_void_p), int(day), SIM_HOST,
                                                    self._stream(stream)))

    def stats(self, stream=None):
        pi = np.zeros((self.R, self.max_days), np.int64)
        pn = np.zeros((self.R, self.max_days), np.int64)
        ctr = np.zeros((self.R, 4), np.int64)
        _check(self.L, self.h, self.L.sim_stats(self.h, _p(pi, ctypes.c_int64), _p(pn, ctypes.c_int64),
                                                _p(ctr, ctypes.c_int64), self._stream(stream)))
        return pi, pn, ctr

    def score(self, stream=None):
        out = np.zeros((self.R, 8, self.N), np.float64)
        _check(self.L, self.h, self.L.sim_score(self.h, _p(out, ctypes.c_double), self._stream(stream)))
        return out

    def score_backward(self, stream=None):
        _check(self.L, self.h, self.L.sim_score_backward(self.h, self._stream(stream)))

    def gradient_moments(self, days, stream=None):
        """Returns (moments [n_days, 42], per-replicate scores [R, 8])."""
        d = np.ascontiguousarray(days, np.int32)
        out = np.zeros((d.size, N_MOMENTS), np.float64)
        per = np.zeros((self.R, 8), np.float64)
        _check(self.L, self.h, self.L.sim_gradient_moments(self.h, _p(d, ctypes.c_int32), d.size,
                                                           _p(per, ctypes.c_double), _p(out, ctypes.c_double),
                                                           self._stream(stream)))
        return out, per

    def reset(self, clear_events=False):
        _check(self.L, self.h, self.L.sim_reset(self.h, 1 if clear_events else 0))

    def schedule(self):
        n = self.L.sim_debug_schedule_size(self.h)
        order = np.zeros(max(n, 1), np.int64)
        level = np.zeros(max(n, 1), np.int32)
        _check(self.L, self.h, self.L.sim_debug_schedule(self.h, _p(order, ctypes.c_int64), _p(level, ctypes.c_int32)))
        return order[:n], level[:n]

    def tune(self, warp_herd_threshold=-1):
        _check(self.L, self.h, self.L.sim_tune(self.h, int(warp_herd_threshold)))
        return self.L.sim_warp_nodes(self.h)

    LAUNCH = {"stream": 0, "graph": 1, "persistent": 2, "flow": 3}

    def set_launch(self, mode):
        _check(self.L, self.h, self.L.sim_set_option(self.h, 2, self.LAUNCH[mode]))

    def set_overlap(self, on):
        """Programmatic dependent launch between the day's kernels (results unchanged)."""
        _check(self.L, self.h, self.L.sim_set_option(self.h, 4, 1 if on else 0))

    def set_group_threshold(self, herd):
        """Herd size from which a node gets an 8-lane group (-1 automatic; results unchanged)."""
        _check(self.L, self.h, self.L.sim_set_option(self.h, 6, int(herd)))

    def set_params(self, params: W.Params):
        """Replaces every replicate's parameters (state, events and statistics stay)."""
        if params.upsilon.shape[0] != self.R:
            raise ValueError("parameters for a different replicate count")
        keep = [np.ascontiguousarray(x, np.float64) for x in
                (params.upsilon, params.gamma, params.alpha, params.beta, params.epsilon)]
        sp = SimParams(*[_p(a, ctypes.c_double) for a in keep])
        _check(self.L, self.h, self.L.sim_set_params(self.h, ctypes.byref(sp)))
        self._keep = keep

    def set_regions(self, region_of_node, n_regions):
        """Region statistics of the fitting goal (region_of_node [N], values < n_regions)."""
        arr = np.ascontiguousarray(region_of_node, np.int32)
        self.n_regions = int(n_regions)
        _check(self.L, self.h, self.L.sim_set_regions(self.h, _p(arr, ctypes.c_int32), int(n_regions)))

    def region_moments(self):
        """(s1, s2) uint64 [max_days, n_regions, Nc]: sums over replicates of the
        daily region totals and of their squares."""
        shape = (self.max_days, self.n_regions, self.nc)
        s1 = np.zeros(shape, np.uint64)
        s2 = np.zeros(shape, np.uint64)
        _check(self.L, self.h, self.L.sim_region_moments(self.h, ctypes.c_void_p(s1.ctypes.data),
                                                         ctypes.c_void_p(s2.ctypes.data)))
        return s1, s2

    def goal(self, ref, day0, ndays):
        """(G^2, VG^2) over days [day0, day0 + ndays) against ref [ndays, n_regions, Nc]."""
        r = np.ascontiguousarray(ref, np.int64)
        g2 = ctypes.c_double(0.0)
        vg2 = ctypes.c_double(0.0)
        _check(self.L, self.h, self.L.sim_goal(self.h, _p(r, ctypes.c_int64), int(day0), int(ndays),
                                               ctypes.byref(g2), ctypes.byref(vg2)))
        return g2.value, vg2.value

    def set_split(self, on):
        """Untouched herds' stochastic step alongside the previous day's events (results unchanged)."""
        _check(self.L, self.h, self.L.sim_set_option(self.h, 5, 1 if on else 0))

    def set_clock_margin(self, k):
        """Speculative clock margin 2^-k, k in [0, 17] (0: exact clock only)."""
        _check(self.L, self.h, self.L.sim_set_option(self.h, 3, int(k)))

    def shard(self, node_lo, node_hi):
        """Restricts the stochastic step, phi update and statistics to nodes
        [node_lo, node_hi) (sim_shard); events still apply to every node."""
        _check(self.L, self.h, self.L.sim_shard(self.h, int(node_lo), int(node_hi)))

    def run_day_stochastic(self, stream=None):
        _check(self.L, self.h, self.L.sim_run_day_stochastic(self.h, self._stream(stream)))

    def run_day_events(self, stream=None):
        _check(self.L, self.h, self.L.sim_run_day_events(self.h, self._stream(stream)))

    def touched_count(self, day):
        return int(self.L.sim_touched_count(self.h, int(day)))

    def touched_nodes(self, day):
        out = np.zeros(max(self.touched_count(day), 0), np.int32)
        _check(self.L, self.h, self.L.sim_touched_nodes(self.h, int(day), _p(out, ctypes.c_int32)))
        return out

    def pack_touched(self, dev_out, stream=None):
        """Counts of the current day's touched herds, int32 [R][Nc][n], into the
        device buffer at address dev_out."""
        _check(self.L, self.h, self.L.sim_pack_touched(self.h, ctypes.c_void_p(dev_out), self._stream(stream)))

    def unpack_touched(self, dev_in, bounds, stream=None):
        """Every touched herd's counts from its owner's pack: dev_in = the ranks'
        packs back to back in rank order; bounds [world + 1] the ranks' node ranges."""
        b = np.ascontiguousarray(bounds, np.int32)
        _check(self.L, self.h, self.L.sim_unpack_touched(self.h, ctypes.c_void_p(dev_in), b.size - 1,
                                                         _p(b, ctypes.c_int32), self._stream(stream)))

    def profile(self, enable=True):
        _check(self.L, self.h, self.L.sim_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        ms = np.zeros(3, np.float64)
        n = np.zeros(3, np.int64)
        _check(self.L, self.h, self.L.sim_profile_read(self.h, _p(ms, ctypes.c_double), _p(n, ctypes.c_int64)))
        return {"ssa": (float(ms[0]), int(n[0])), "events": (float(ms[1]), int(n[1])),
                "finalize": (float(ms[2]), int(n[2]))}

    def close(self):
        if getattr(self, "h", None):
            self.L.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batch(sims, until=None, stream=None):
    """Advances several Sim handles together in one persistent kernel launch."""
    L = load_library()
    arr = (ctypes.c_void_p * len(sims))(*[s.h for s in sims])
    u = None if until is None else np.ascontiguousarray(until, np.int32)
    st = current_stream() if stream is None else ctypes.c_void_p(stream)
    status = L.sim_run_batch(arr, len(sims), _p(u, ctypes.c_int32), st)
    _check(L, None, status)


BATCH_SHAPES = ((256, 2), (256, 1), (128, 4))   # the first is the library's default


def batch_shape(threads: int, blocks_per_sm: int):
    """Block shape (threads a block, resident blocks an SM) of run_batch's
    persistent kernel, process-wide; one of BATCH_SHAPES."""
    L = load_library()
    _check(L, None, L.sim_batch_shape(int(threads), int(blocks_per_sm)))


def debug_div(x, y, out, ref, n, device):
    """x, y, out, ref: pointers (ints) to n doubles, host or device."""
    L = load_library()
    st = L.sim_debug_div(ctypes.c_void_p(x), ctypes.c_void_p(y), ctypes.c_void_p(out), ctypes.c_void_p(ref),
                         int(n), SIM_DEVICE if device else SIM_HOST)
    _check(L, None, st)


def debug_neglog(j_dev_ptr, out_dev_ptr, n):
    L = load_library()
    st = L.sim_debug_neglog(ctypes.c_void_p(j_dev_ptr), ctypes.c_void_p(out_dev_ptr), int(n))
    _check(L, None, st)


def debug_neglog_f32(j_dev_ptr, out_dev_ptr, n):
    L = load_library()
    st = L.sim_debug_neglog_f32(ctypes.c_void_p(j_dev_ptr), ctypes.c_void_p(out_dev_ptr), int(n))
    _check(L, None, st)


def _gen_model(m: W.GeneralModel):
    """The gen_model struct of a GeneralModel, with the arrays it points to."""
    stoich = np.ascontiguousarray(m.stoich, np.int32)
    trans = np.zeros((max(m.nt, 1), 4), np.int32)
    trans[:m.nt, 0], trans[:m.nt, 1], trans[:m.nt, 2] = m.factor_a, m.factor_b, m.cont
    trans[:m.nt, 3] = m.pop_mask.astype(np.uint32).view(np.int32)
    vars_ = np.zeros((max(m.ny, 1), 2), np.uint32)
    vars_[:m.ny, 0], vars_[:m.ny, 1] = m.num_mask, m.den_mask
    select = np.ascontiguousarray(m.select, np.uint32)
    shift = np.ascontiguousarray(m.shift, np.int32)
    keep = (stoich, trans, vars_, select, shift)
    gm = GenModel(m.nc, m.nt, m.ny, int(select.size), int(shift.shape[0]), int(m.y_source),
                  _p(stoich, ctypes.c_int32), _p(trans, ctypes.c_int32), _p(vars_, ctypes.c_uint32),
                  _p(select if select.size else np.zeros(1, np.uint32), ctypes.c_uint32),
                  _p(shift if shift.size else np.zeros(1, np.int32), ctypes.c_int32))
    return gm, keep


def gen_dependency(m: W.GeneralModel):
    """Validates the model (host only) and returns its dependency graph: dep[n]
    bit j set when firing transition n can change rate j."""
    L = load_library()
    gm, keep = _gen_model(m)
    dep = np.zeros(max(m.nt, 1), np.uint32)
    st = L.gen_model_check(ctypes.byref(gm), _p(dep, ctypes.c_uint32))
    if st != SIM_OK:
        msg = L.gen_last_error(None)
        raise SimError(st, msg.decode() if msg else "")
    return dep[:m.nt].copy()


class GenSim:
    """One handle of the general compartment model: R replicates on N nodes."""

    def __init__(self, model: W.GeneralModel, u0, y0, rates, var_params, max_days, seed=1,
                 underflow_error=False, replicate_base=0):
        self.L = load_library()
        u0 = np.ascontiguousarray(u0, np.int32)
        self.nc, self.N = u0.shape
        self.ny = model.ny
        rates = np.ascontiguousarray(rates, np.float64)
        self.R = rates.shape[0]
        self.max_days = max_days
        gm, keep = _gen_model(model)
        cfg = GenConfig(self.N, self.R, max_days, 1 if underflow_error else 0, seed, int(replicate_base), 0)
        y0 = np.ascontiguousarray(y0, np.float64).reshape(self.ny, self.N)
        vp = np.ascontiguousarray(var_params, np.float64)
        h = ctypes.c_void_p()
        st = self.L.gen_create(ctypes.byref(gm), ctypes.byref(cfg), _p(u0, ctypes.c_int32),
                               _p(y0 if y0.size else np.zeros(1), ctypes.c_double),
                               _p(rates if rates.size else np.zeros(1), ctypes.c_double),
                               _p(vp if vp.size else np.zeros(1), ctypes.c_double), ctypes.byref(h))
        del keep
        self._check(None, st)
        self.h = h

    def _check(self, h, st):
        if st != SIM_OK:
            msg = self.L.gen_last_error(h)
            raise SimError(st, msg.decode() if msg else "")

    @classmethod
    def from_workload(cls, w: W.GeneralWorkload, events=True, max_days=None, **kw):
        s = cls(w.model, w.u0, w.y0, w.rates, w.var_params, w.T if max_days is None else max_days, seed=w.seed,
                underflow_error=w.underflow_error, **kw)
        if events and len(w.events):
            s.load_events(w.events)
        return s

    def load_events(self, ev: W.GeneralEvents):
        arr = [np.ascontiguousarray(a, np.int32) for a in (ev.day, ev.kind, ev.node, ev.dest, ev.count, ev.select,
                                                           ev.shift)]
        self._check(self.h, self.L.gen_load_events(self.h, len(ev), *[_p(a, ctypes.c_int32) for a in arr]))

    def set_launch(self, mode):
        self._check(self.h, self.L.gen_set_option(self.h, GEN_OPT_LAUNCH, {"stream": 0, "graph": 1}[mode]))

    def set_clock_margin(self, k):
        """Binary32 clock margin 2^-k of the one-per-thread nodes, k in [0, 16] (0: exact only)."""
        self._check(self.h, self.L.gen_set_option(self.h, GEN_OPT_CLOCK_MARGIN, int(k)))

    def set_warp_threshold(self, population):
        """Nodes with at least this initial population run one per warp (-1: automatic)."""
        self._check(self.h, self.L.gen_set_option(self.h, GEN_OPT_WARP_THRESHOLD, int(population)))
        return self.L.gen_warp_nodes(self.h)

    def set_group_threshold(self, population):
        """Nodes below the warp threshold with at least this initial population run
        four per warp (-1: automatic); returns how many."""
        self._check(self.h, self.L.gen_set_option(self.h, GEN_OPT_GROUP_THRESHOLD, int(population)))
        return self.L.gen_group_nodes(self.h)

    def run(self, days, stream=None):
        st = current_stream() if stream is None else ctypes.c_void_p(stream)
        self._check(self.h, self.L.gen_run_days(self.h, int(days), st))

    def state(self, stream=None):
        counts = np.empty((self.R, self.nc, self.N), np.int32)
        y = np.empty((self.R, self.ny, self.N), np.float64)
        day = ctypes.c_int32()
        st = current_stream() if stream is None else ctypes.c_void_p(stream)
        self._check(self.h, self.L.gen_state(self.h, counts.ctypes.data_as(ctypes.c_void_p),
                                             y.ctypes.data_as(ctypes.c_void_p) if y.size else None,
                                             ctypes.byref(day), SIM_HOST, st))
        return counts, y, day.value

    def set_state(self, counts, y, day, stream=None):
        counts = np.ascontiguousarray(counts, np.int32)
        y = np.ascontiguousarray(y, np.float64)
        st = current_stream() if stream is None else ctypes.c_void_p(stream)
        self._check(self.h, self.L.gen_set_state(self.h, counts.ctypes.data_as(ctypes.c_void_p),
                                                 y.ctypes.data_as(ctypes.c_void_p) if y.size else None,
                                                 int(day), SIM_HOST, st))

    def counters(self):
        out = np.zeros((self.R, 4), np.int64)
        self._check(self.h, self.L.gen_counters(self.h, _p(out, ctypes.c_int64)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.L.gen_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
