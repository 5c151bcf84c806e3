"""Thin Python binding of libcfr.so (the C ABI in include/cfr.h).

Argument marshalling only: every step of a CFR+ iteration runs in the
library's sm_103a kernels. PyTorch provides the device arena and streams.
There is no CPU fallback: if ``libcfr.so`` is missing or fails to load, the
import of this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcfr.so")

CFR_OK = 0
ERRORS = {
    -1: "CFR_ERR_ARG", -2: "CFR_ERR_INVALID_SPEC", -3: "CFR_ERR_NOT_BOUND", -4: "CFR_ERR_REBOUND",
    -5: "CFR_ERR_ARENA_SMALL", -6: "CFR_ERR_TIMEOUT", -7: "CFR_ERR_DEVICE", -8: "CFR_ERR_HOST_MEMORY",
    -9: "CFR_ERR_UNSUPPORTED",
}
CFR_ERR_ARG, CFR_ERR_INVALID_SPEC, CFR_ERR_NOT_BOUND, CFR_ERR_REBOUND = -1, -2, -3, -4
CFR_ERR_ARENA_SMALL, CFR_ERR_TIMEOUT, CFR_ERR_DEVICE, CFR_ERR_HOST_MEMORY, CFR_ERR_UNSUPPORTED = -5, -6, -7, -8, -9
P64, P32 = 0, 1
EXEC_AUTO, EXEC_LEVELS, EXEC_GRAPH, EXEC_PERSISTENT = 0, 1, 2, 3
RULE_CFR_PLUS, RULE_CFR, RULE_PCFR_PLUS = 0, 1, 2
ORDER_SIMULTANEOUS, ORDER_ALTERNATING = 0, 1
REACH_MEMBERS, REACH_BFS, REACH_SLOTS = 0, 1, 2
TILES_AUTO, TILES_OFF, TILES_ON = 0, 1, 2
OVERLAP_AUTO, OVERLAP_OFF, OVERLAP_ON = 0, 1, 2
DEBUG_BARRIER_MISSING_ARRIVALS = 1
DEBUG_FAIL_GRAPH_CAPTURE = 2
DEBUG_STREAM_STALL = 3
EXPORT = {"child_begin": 0, "node_slot": 1, "level_begin": 2, "iset_slot": 3, "iset_mem": 4, "mem_node": 5,
          "chance_list": 6, "level_chance": 7, "level_iset": 8, "new_of_spec": 9, "tmpl": 10,
          "spec_slot_of": 11, "level_lanes": 12, "int_slot": 13, "int_mask": 14, "int_cirank": 15,
          "big_irank": 16, "mem_irank": 17, "level_int": 18, "vslot": 19, "iset_vb": 20, "mem_vs": 21,
          "ch_vb": 22, "ch_nch": 23, "ch_vs": 24, "wide_vb": 25, "wide_nch": 26, "wide_vs": 27, "tmpl_vs": 28,
          "int_edge": 29, "iset_rank": 30, "level_tiled": 31, "set_info": 32, "stream_chunks": 33, "stream_c0": 34,
          "stream_ok": 35, "pull_grid": 36}
STREAM_LANES = 512  # lanes_per_set code of the streaming FP32 backward


class CfrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (ERRORS.get(code, str(code)), msg))
        self.code = code


class GameSpecC(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int64), ("n_infosets", ctypes.c_int64),
        ("kind", ctypes.c_void_p), ("infoset", ctypes.c_void_p), ("child_begin", ctypes.c_void_p),
        ("child", ctypes.c_void_p), ("chance_prob", ctypes.c_void_p), ("payoff", ctypes.c_void_p),
        ("iset_player", ctypes.c_void_p), ("iset_nact", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("exec_form", ctypes.c_int), ("rule", ctypes.c_int),
        ("lanes_per_set", ctypes.c_int), ("persistent_ctas", ctypes.c_int),
        ("barrier_spin_limit", ctypes.c_int64), ("order", ctypes.c_int), ("reach_order", ctypes.c_int),
        ("member_tiles", ctypes.c_int), ("launch_overlap", ctypes.c_int), ("graph_iters", ctypes.c_int),
    ]


class Counts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "n_edges", "n_infosets", "n_slots", "n_internal", "n_decision", "n_chance", "n_terminal",
        "depth_blocks", "max_actions", "algo_bytes_per_iter", "upload_bytes", "iteration")] + [
        ("exec_form", ctypes.c_int), ("lanes_per_set", ctypes.c_int), ("graph_kernels", ctypes.c_int64),
        ("graph_k_kernels", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcfr.so is not built (run __graft_entry__.build() or "
                          "python -m paper_2609_11923_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    sig = {
        "cfr_compile": [ctypes.POINTER(GameSpecC), ctypes.POINTER(Options), ctypes.POINTER(H)],
        "cfr_get_counts": [H, ctypes.POINTER(Counts)],
        "cfr_plan": [H, ctypes.POINTER(ctypes.c_size_t)],
        "cfr_bind": [H, vp, ctypes.c_size_t, vp],
        "cfr_iterate": [H, i64, vp],
        "cfr_synchronize": [H, vp],
        "cfr_avg_strategy": [H, vp, ctypes.c_int, vp],
        "cfr_current_strategy": [H, vp, ctypes.c_int, vp],
        "cfr_exploitability": [H, dp, dp, vp],
        "cfr_reset": [H, vp],
        "cfr_set_payoffs": [H, dp, vp],
        "cfr_get_state": [H, dp, dp, ctypes.POINTER(i64), vp],
        "cfr_set_state": [H, dp, dp, i64, vp],
        "cfr_export_array": [H, ctypes.c_int, vp, i64, ctypes.POINTER(i64)],
        "cfr_debug_set": [H, ctypes.c_int, i64],
        "cfr_level_bytes": [H, ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "cfr_profile_iteration": [H, dp, dp, vp],
        "cfr_iterate_noalloc": [H, i64, vp],
        "cfr_autotune": [H, ctypes.c_int, vp],
        "cfr_launch_floor": [H, i64, vp, dp, dp],
        "cfr_pin_host": [H, ctypes.c_int],
        "cfr_set_chance_sums": [H, dp, dp, dp],
        "cfr_set_root_chance": [H, dp, i64, vp],
        "cfr_batch_iterate": [ctypes.POINTER(H), ctypes.c_int, ctypes.POINTER(i64), i64, vp, ctypes.c_size_t,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, vp],
        "cfr_batch_exploitability": [ctypes.POINTER(H), ctypes.c_int, dp, vp, ctypes.c_size_t, ctypes.c_int,
                                     ctypes.c_int, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.cfr_last_error.restype = ctypes.c_char_p
    lib.cfr_last_error.argtypes = []
    lib.cfr_destroy.restype = None
    lib.cfr_destroy.argtypes = [H]
    lib.cfr_batch_table_bytes.restype = ctypes.c_size_t
    lib.cfr_batch_table_bytes.argtypes = [ctypes.c_int]
    return lib


_lib = _load()
EXPORTED = ["cfr_compile", "cfr_get_counts", "cfr_plan", "cfr_bind", "cfr_iterate", "cfr_synchronize",
            "cfr_avg_strategy", "cfr_current_strategy", "cfr_exploitability", "cfr_reset", "cfr_set_payoffs",
            "cfr_get_state", "cfr_set_state", "cfr_export_array", "cfr_debug_set", "cfr_last_error",
            "cfr_destroy", "cfr_level_bytes", "cfr_profile_iteration", "cfr_iterate_noalloc", "cfr_autotune",
            "cfr_batch_table_bytes", "cfr_batch_iterate", "cfr_batch_exploitability", "cfr_launch_floor",
            "cfr_set_root_chance", "cfr_pin_host", "cfr_set_chance_sums"]


def _check(rc: int) -> None:
    if rc != CFR_OK:
        raise CfrError(rc, (_lib.cfr_last_error() or b"").decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def spec_struct(spec) -> Tuple[GameSpecC, list]:
    """ctypes view of a GameSpec (gamegen.GameSpec or any object with the
    same arrays); the returned list keeps the converted arrays alive."""
    arrs = [
        np.ascontiguousarray(spec.kind, dtype=np.int8),
        np.ascontiguousarray(spec.infoset, dtype=np.int32),
        np.ascontiguousarray(spec.child_begin, dtype=np.int64),
        np.ascontiguousarray(spec.child, dtype=np.int32),
        np.ascontiguousarray(spec.chance_prob, dtype=np.float64),
        np.ascontiguousarray(spec.payoff, dtype=np.float64),
        np.ascontiguousarray(spec.iset_player, dtype=np.int8),
        np.ascontiguousarray(spec.iset_nact, dtype=np.int32),
    ]
    s = GameSpecC()
    s.n_nodes = int(arrs[0].shape[0])
    s.n_infosets = int(arrs[6].shape[0])
    (s.kind, s.infoset, s.child_begin, s.child, s.chance_prob, s.payoff, s.iset_player,
     s.iset_nact) = [a.ctypes.data if a.size else None for a in arrs]
    return s, arrs


def make_options(precision=P32, exec_form=EXEC_AUTO, rule=RULE_CFR_PLUS, lanes_per_set=0, persistent_ctas=0,
                 barrier_spin_limit=0, order=ORDER_SIMULTANEOUS, reach_order=REACH_MEMBERS,
                 member_tiles=TILES_AUTO, launch_overlap=OVERLAP_AUTO, graph_iters=0) -> Options:
    o = Options()
    o.precision, o.exec_form, o.rule = precision, exec_form, rule
    o.lanes_per_set, o.persistent_ctas, o.barrier_spin_limit = lanes_per_set, persistent_ctas, barrier_spin_limit
    o.order = order
    o.reach_order = reach_order
    o.member_tiles = member_tiles
    o.launch_overlap = launch_overlap
    o.graph_iters = graph_iters
    return o


# ---------------------------------------------------------------- C-ABI mirror
def cfr_compile(spec, options: Optional[Options] = None) -> int:
    s, keep = spec_struct(spec)
    h = ctypes.c_void_p()
    _check(_lib.cfr_compile(ctypes.byref(s), ctypes.byref(options) if options is not None else None,
                            ctypes.byref(h)))
    del keep
    return h.value


def cfr_get_counts(h: int) -> dict:
    c = Counts()
    _check(_lib.cfr_get_counts(h, ctypes.byref(c)))
    return c.as_dict()


def cfr_plan(h: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib.cfr_plan(h, ctypes.byref(n)))
    return n.value


def cfr_bind(h: int, arena_ptr: int, nbytes: int, stream: int = 0) -> None:
    _check(_lib.cfr_bind(h, arena_ptr, nbytes, stream))


def cfr_iterate(h: int, n: int, stream: int = 0) -> None:
    _check(_lib.cfr_iterate(h, n, stream))


def cfr_iterate_noalloc(h: int, n: int, stream: int = 0) -> None:
    """n iterations with the scratch in the library's static device array
    (no allocation during the call; synchronises the stream)."""
    _check(_lib.cfr_iterate_noalloc(h, n, stream))


def cfr_autotune(h: int, reps: int = 5, stream: int = 0) -> None:
    """Pick lanes per information set for every depth by timing (resets the state)."""
    _check(_lib.cfr_autotune(h, reps, stream))


def cfr_synchronize(h: int, stream: int = 0) -> None:
    _check(_lib.cfr_synchronize(h, stream))


def cfr_avg_strategy(h: int, out, on_device: bool, stream: int = 0) -> None:
    """out: a host float64 numpy array, or a device pointer (int) if on_device."""
    ptr = out if on_device else out.ctypes.data
    _check(_lib.cfr_avg_strategy(h, ptr, 1 if on_device else 0, stream))


def cfr_current_strategy(h: int, out, on_device: bool, stream: int = 0) -> None:
    ptr = out if on_device else out.ctypes.data
    _check(_lib.cfr_current_strategy(h, ptr, 1 if on_device else 0, stream))


def cfr_exploitability(h: int, stream: int = 0) -> Tuple[float, float, float, float]:
    """(exploitability, br1, br2, u(avg)) in player-1 units."""
    e = ctypes.c_double()
    br = (ctypes.c_double * 3)()
    _check(_lib.cfr_exploitability(h, ctypes.byref(e), br, stream))
    return e.value, br[0], br[1], br[2]


def cfr_reset(h: int, stream: int = 0) -> None:
    _check(_lib.cfr_reset(h, stream))


def cfr_set_payoffs(h: int, payoff: np.ndarray, stream: int = 0) -> None:
    p = np.ascontiguousarray(payoff, dtype=np.float64)
    _check(_lib.cfr_set_payoffs(h, _dp(p), stream))


def cfr_get_state(h: int, n_slots: int, stream: int = 0):
    R = np.empty(n_slots)
    avg = np.empty(n_slots)
    t = ctypes.c_int64()
    _check(_lib.cfr_get_state(h, _dp(R), _dp(avg), ctypes.byref(t), stream))
    return R, avg, t.value


def cfr_set_state(h: int, R: np.ndarray, avg: np.ndarray, t: int, stream: int = 0) -> None:
    R = np.ascontiguousarray(R, dtype=np.float64)
    avg = np.ascontiguousarray(avg, dtype=np.float64)
    _check(_lib.cfr_set_state(h, _dp(R), _dp(avg), t, stream))


def cfr_export_array(h: int, name: str) -> np.ndarray:
    which = EXPORT[name]
    n = ctypes.c_int64()
    _check(_lib.cfr_export_array(h, which, None, 0, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.float64 if name in ("tmpl", "tmpl_vs") else np.int32)
    _check(_lib.cfr_export_array(h, which, out.ctypes.data if n.value else None, n.value, ctypes.byref(n)))
    return out


def cfr_debug_set(h: int, key: int, value: int) -> None:
    _check(_lib.cfr_debug_set(h, key, value))


def cfr_level_bytes(h: int, level: int) -> Tuple[int, int]:
    f, b = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.cfr_level_bytes(h, level, ctypes.byref(f), ctypes.byref(b)))
    return f.value, b.value


def cfr_set_root_chance(h: int, prob, stream: int = 0) -> None:
    p = np.ascontiguousarray(prob, dtype=np.float64)
    _check(_lib.cfr_set_root_chance(h, _dp(p), len(p), stream))


def cfr_set_chance_sums(h: int, n_sets: int, root_w=None):
    """(mass[I], wsum[I] or None) in spec set order: per set the sum of its
    members' chance products, and of those times root_w[root outcome]."""
    mass = np.zeros(n_sets)
    wsum = np.zeros(n_sets) if root_w is not None else None
    rw = np.ascontiguousarray(root_w, dtype=np.float64) if root_w is not None else None
    _check(_lib.cfr_set_chance_sums(h, _dp(rw) if rw is not None else None, _dp(mass),
                                    _dp(wsum) if wsum is not None else None))
    return mass, wsum


def cfr_pin_host(h: int, pin: bool = True) -> None:
    """Page-lock (or release) the handle's host arrays that cfr_bind uploads."""
    _check(_lib.cfr_pin_host(h, 1 if pin else 0))


def cfr_launch_floor(h: int, n: int, stream: int = 0) -> Tuple[float, float]:
    """Per-iteration ms of the launch structure alone: (graph of empty kernels, empty persistent kernel)."""
    g, p = ctypes.c_double(), ctypes.c_double()
    _check(_lib.cfr_launch_floor(h, n, stream, ctypes.byref(g), ctypes.byref(p)))
    return g.value, p.value


def cfr_profile_iteration(h: int, depth_blocks: int, stream: int = 0):
    """Per-launch device times (ms) of one iteration: (fwd[D], bwd[D])."""
    f = np.zeros(max(depth_blocks, 1))
    b = np.zeros(max(depth_blocks, 1))
    _check(_lib.cfr_profile_iteration(h, _dp(f), _dp(b), stream))
    return f[:depth_blocks], b[:depth_blocks]


def cfr_batch_table_bytes(n: int) -> int:
    return int(_lib.cfr_batch_table_bytes(n))


def _handles(hs):
    arr = (ctypes.c_void_p * len(hs))()
    for i, h in enumerate(hs):
        arr[i] = h
    return arr


def cfr_batch_iterate(hs, n_iter, table_ptr: int, table_bytes: int, threads: int = 0, lanes: int = 0,
                      stream: int = 0, iters=None, cluster: int = 1) -> None:
    """n_iter iterations of every handle in one launch (or iters[i] each);
    cluster > 1 gives every instance a thread-block cluster of that many CTAs."""
    it = None
    if iters is not None:
        it = (ctypes.c_int64 * len(hs))(*[int(x) for x in iters])
    _check(_lib.cfr_batch_iterate(_handles(hs), len(hs), it, n_iter, table_ptr, table_bytes, threads, lanes,
                                  cluster, stream))


def cfr_batch_exploitability(hs, table_ptr: int, table_bytes: int, threads: int = 0, lanes: int = 0,
                             stream: int = 0) -> np.ndarray:
    """[n, 4]: (exploitability, br1, br2, u) of every handle's average strategy."""
    out = np.zeros(4 * len(hs))
    _check(_lib.cfr_batch_exploitability(_handles(hs), len(hs), _dp(out), table_ptr, table_bytes, threads, lanes,
                                         stream))
    return out.reshape(len(hs), 4)


def cfr_last_error() -> str:
    return (_lib.cfr_last_error() or b"").decode()


def cfr_destroy(h: int) -> None:
    _lib.cfr_destroy(h)


# ------------------------------------------------------------ convenience
class Solver:
    """A compiled game bound to a PyTorch-allocated device arena."""

    def __init__(self, spec, precision: int = P32, exec_form: int = EXEC_AUTO, rule: int = RULE_CFR_PLUS,
                 lanes_per_set: int = 0, persistent_ctas: int = 0, barrier_spin_limit: int = 0,
                 device: str = "cuda", stream=None, order: int = ORDER_SIMULTANEOUS,
                 reach_order: int = REACH_MEMBERS, member_tiles: int = TILES_AUTO,
                 launch_overlap: int = OVERLAP_AUTO, graph_iters: int = 0):
        import torch

        self.torch = torch
        self.opts = make_options(precision, exec_form, rule, lanes_per_set, persistent_ctas, barrier_spin_limit,
                                 order, reach_order, member_tiles, launch_overlap, graph_iters)
        self.h = cfr_compile(spec, self.opts)
        self.counts = cfr_get_counts(self.h)
        self.n_slots = self.counts["n_slots"]
        self.pot = float(getattr(spec, "pot", 1.0))
        nbytes = cfr_plan(self.h)
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        self.arena_ptr = (self.arena.data_ptr() + 255) & ~255
        self.arena_bytes = nbytes
        self.stream = stream
        cfr_bind(self.h, self.arena_ptr, nbytes, self._s())

    def _s(self) -> int:
        if self.stream is not None:
            return int(self.stream.cuda_stream)
        return int(self.torch.cuda.current_stream().cuda_stream)

    def iterate(self, n: int) -> None:
        cfr_iterate(self.h, n, self._s())

    def autotune(self, reps: int = 5) -> list:
        cfr_autotune(self.h, reps, self._s())
        return list(cfr_export_array(self.h, "level_lanes"))

    def synchronize(self) -> None:
        cfr_synchronize(self.h, self._s())

    def avg_strategy(self) -> np.ndarray:
        out = np.empty(self.n_slots)
        cfr_avg_strategy(self.h, out, False, self._s())
        return out

    def avg_strategy_device(self):
        out = self.torch.empty(self.n_slots, dtype=self.torch.float64, device=self.arena.device)
        cfr_avg_strategy(self.h, out.data_ptr(), True, self._s())
        return out

    def current_strategy(self) -> np.ndarray:
        out = np.empty(self.n_slots)
        cfr_current_strategy(self.h, out, False, self._s())
        return out

    def exploitability(self) -> float:
        return cfr_exploitability(self.h, self._s())[0]

    def best_response(self):
        return cfr_exploitability(self.h, self._s())[1:]

    def reset(self) -> None:
        cfr_reset(self.h, self._s())

    def set_payoffs(self, payoff) -> None:
        cfr_set_payoffs(self.h, payoff, self._s())

    def pin_host(self, pin: bool = True) -> None:
        cfr_pin_host(self.h, pin)

    def set_root_chance(self, prob) -> None:
        cfr_set_root_chance(self.h, prob, self._s())

    def get_state(self):
        return cfr_get_state(self.h, self.n_slots, self._s())

    def set_state(self, R, avg, t) -> None:
        cfr_set_state(self.h, R, avg, t, self._s())

    def counts_now(self) -> dict:
        return cfr_get_counts(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            cfr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
