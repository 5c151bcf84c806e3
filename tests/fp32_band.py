"""How far FP32 rounding alone can move a case's exploitability (test helper).

The FP32 mode stores the chance-weighted terminal values, reach, values and
strategy in FP32, so every solve it runs is the oracle's solve of a slightly
perturbed game, perturbed at FP32's unit roundoff (2^-24 relative). Under
regret matching+ some cases amplify such perturbations without bound (near
zero regrets change sign, the strategy changes support; the paper reports
run-to-run spreads of this kind from reduction order alone). On those cases
no FP32 implementation can pin the oracle's exploitability to 1e-4 of the
pot. fp32_band measures it: the oracle's exploitability, and its largest
change over k seeded games whose payoffs are each scaled by (1 + 2^-24 u),
u ~ U[-1, 1], evaluated on the unperturbed game. A parity test then holds
the FP32 mode to max(1e-4 pot, 2 x that change): the strict bar wherever the
case is well conditioned.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

EPS32 = 2.0 ** -24


def fp32_band(make, iters, rule=oracle.CFR_PLUS, order=oracle.SIMULTANEOUS, k=3):
    """(exploitability of the oracle after iters, largest change under k
    FP32-sized payoff perturbations). make() builds a fresh copy of the game."""
    def run(j):
        g = make()
        if j > 0:
            u = np.random.default_rng(7919 * j).uniform(-1.0, 1.0, g.n_nodes)
            g.payoff[:] = g.payoff * (1.0 + EPS32 * u)
        o = oracle.solve(g, iters, rule=rule, order=order)
        return o.avg_strategy()

    with ThreadPoolExecutor(max_workers=k + 1) as ex:  # the oracle's C routine releases the interpreter lock
        sig = list(ex.map(run, range(k + 1)))
    ref = oracle.Oracle(make())
    e = [ref.exploitability(s) for s in sig]
    return e[0], max(abs(x - e[0]) for x in e[1:])


def fp32_bar(pot, delta):
    """The FP32 parity bar: 1e-4 of the pot, widened only where FP32-sized
    perturbations alone move the oracle further."""
    return max(1e-4 * pot, 2.0 * delta)
