"""FP64 CPU oracle for CFR+ — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It never imports the CUDA package and the CUDA
package never imports it; the two meet only through the seeded game specs of
``gamegen``.

``oracle.c`` is the plain recursive CFR+ / best response / brute force in C
(``-ffp-contract=off``); ``lp.py`` solves the sequence-form LP for the game
value with SciPy's HiGHS. See the header of ``oracle.c`` for the paper
passages each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
CFR_PLUS, CFR, PCFR_PLUS = 0, 1, 2
SIMULTANEOUS, ALTERNATING = 0, 1


class _Game(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int64),
        ("n_infosets", ctypes.c_int64),
        ("kind", ctypes.c_void_p),
        ("infoset", ctypes.c_void_p),
        ("child_begin", ctypes.c_void_p),
        ("child", ctypes.c_void_p),
        ("chance_prob", ctypes.c_void_p),
        ("payoff", ctypes.c_void_p),
        ("iset_player", ctypes.c_void_p),
        ("iset_nact", ctypes.c_void_p),
    ]


def build(verbose: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc -O2 -ffp-contract=off)."""
    src = os.path.join(_HERE, "oracle.c")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(
        os.path.join(_HERE, "oracle.c")
    ):
        build()
    lib = ctypes.CDLL(_LIB_PATH)
    G = ctypes.POINTER(_Game)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.or_cfr_run.argtypes = [G, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    lib.or_cfr_run.restype = ctypes.c_int
    lib.or_avg_strategy.argtypes = [G, dp, dp]
    lib.or_avg_strategy.restype = None
    lib.or_current_strategy.argtypes = [G, dp, dp, dp]
    lib.or_current_strategy.restype = None
    lib.or_expected_value.argtypes = [G, dp]
    lib.or_expected_value.restype = ctypes.c_double
    lib.or_best_response.argtypes = [G, dp, dp, dp, dp]
    lib.or_best_response.restype = ctypes.c_int
    lib.or_exploitability.argtypes = [G, dp]
    lib.or_exploitability.restype = ctypes.c_double
    lib.or_bruteforce_br.argtypes = [G, dp, ctypes.c_int, ctypes.c_int64, dp]
    lib.or_bruteforce_br.restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """FP64 CFR solver state over one game spec (plain recursive tree walk)."""

    def __init__(self, spec, rule: int = CFR_PLUS, order: int = SIMULTANEOUS):
        self.spec = spec
        self.rule, self.order = rule, order
        # keep contiguous arrays of the exact dtypes alive for the C side
        self._arrs = [
            np.ascontiguousarray(spec.kind, dtype=np.int8),
            np.ascontiguousarray(spec.infoset, dtype=np.int32),
            np.ascontiguousarray(spec.child_begin, dtype=np.int64),
            np.ascontiguousarray(spec.child, dtype=np.int32),
            np.ascontiguousarray(spec.chance_prob, dtype=np.float64),
            np.ascontiguousarray(spec.payoff, dtype=np.float64),
            np.ascontiguousarray(spec.iset_player, dtype=np.int8),
            np.ascontiguousarray(spec.iset_nact, dtype=np.int32),
        ]
        g = _Game()
        g.n_nodes = spec.n_nodes
        g.n_infosets = spec.n_infosets
        (g.kind, g.infoset, g.child_begin, g.child, g.chance_prob, g.payoff, g.iset_player,
         g.iset_nact) = [a.ctypes.data for a in self._arrs]
        self._g = g
        self.A = int(spec.iset_nact.sum())
        self.R = np.zeros(self.A)
        self.sbar = np.zeros(self.A)
        self.pred = np.zeros(self.A)  # PCFR+ prediction: each slot's last instantaneous regret
        self.t = 0
        self.root_value = 0.0

    def iterate(self, n: int) -> None:
        rv = ctypes.c_double(0.0)
        rc = _load().or_cfr_run(ctypes.byref(self._g), self.t, n, self.rule, self.order,
                                _dp(self.R), _dp(self.sbar), _dp(self.pred), ctypes.byref(rv))
        if rc != 0:
            raise RuntimeError("oracle: or_cfr_run failed (%d)" % rc)
        self.t += n
        self.root_value = rv.value

    def avg_strategy(self) -> np.ndarray:
        out = np.empty(self.A)
        _load().or_avg_strategy(ctypes.byref(self._g), _dp(self.sbar), _dp(out))
        return out

    def current_strategy(self) -> np.ndarray:
        out = np.empty(self.A)
        pred = _dp(self.pred) if self.rule == PCFR_PLUS else None
        _load().or_current_strategy(ctypes.byref(self._g), _dp(self.R), pred, _dp(out))
        return out

    # evaluation helpers (also usable on arbitrary strategies)
    def expected_value(self, sigma: np.ndarray) -> float:
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        return float(_load().or_expected_value(ctypes.byref(self._g), _dp(sigma)))

    def best_response(self, sigma: np.ndarray):
        """(br1, br2, u(sigma)) in player-1 units."""
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        b1, b2, v = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = _load().or_best_response(ctypes.byref(self._g), _dp(sigma), ctypes.byref(b1),
                                      ctypes.byref(b2), ctypes.byref(v))
        if rc != 0:
            raise RuntimeError("oracle: best response failed (%d)" % rc)
        return b1.value, b2.value, v.value

    def exploitability(self, sigma: np.ndarray | None = None) -> float:
        if sigma is None:
            sigma = self.avg_strategy()
        b1, b2, _ = self.best_response(sigma)
        return 0.5 * (b1 - b2)

    def bruteforce_br(self, sigma: np.ndarray, player: int, max_strategies: int = 10 ** 7) -> float:
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        out = ctypes.c_double()
        rc = _load().or_bruteforce_br(ctypes.byref(self._g), _dp(sigma), player, max_strategies,
                                      ctypes.byref(out))
        if rc != 0:
            raise RuntimeError("oracle: brute force refused or failed (%d)" % rc)
        return out.value


def solve(spec, iters: int, rule: int = CFR_PLUS, order: int = SIMULTANEOUS) -> Oracle:
    o = Oracle(spec, rule, order)
    o.iterate(iters)
    return o
