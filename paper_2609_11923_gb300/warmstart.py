"""Learned warm start for the endgame family (no counterpart in the paper).

Pipeline: solve many training games with the batched CFR+ kernels, take
their average strategies as targets, train the MLP (mlp.py) on per-
information-set features, then seed new solves with R0(I, a) = kappa * pot *
sigma_hat(I, a) (so the first iterate plays the network's strategy) and let
plain CFR+ continue. Cold-start CFR+ on the same games is the yardstick.

Features of an information set (172 values, padded to 176): the two private
cards (two-hot over 32 cards), the public card (one-hot), the three-card hand
category (trips / pair / high) and its normalised showdown value, acting
player, betting round, number of actions (one-hot), the betting history
(8 positions x 11 action codes, one-hot), both contributions and the amount
to call, the set's chance mass relative to the sets with the same public
state (the weight of this private hand in the range), and the hand's
equity against the opponent's range: the chance-weighted share of the set's
deals that the acting player wins at the check-down showdown (value and a
10-bucket one-hot).
"""
from __future__ import annotations

import os
import time
from concurrent.futures import ThreadPoolExecutor
from typing import List, Optional

import numpy as np

from . import cfr, serve
from .mlp import MLP, N_OUT

F_RAW = 183
F_IN = 192
N_CARDS, N_SUITS = 32, 4


def _rank3(r0, r1, r2):
    a, b, c = sorted((r0, r1, r2), reverse=True)
    if a == c:
        return 2, 2 * 4096 + a
    if a == b:
        return 1, 4096 + a * 64 + c
    if b == c:
        return 1, 4096 + b * 64 + a
    return 0, a * 256 + b * 16 + c


def _rank3_vec(r0, r1, r2):
    """Vectorised _rank3: (category, value) arrays."""
    r = np.sort(np.stack([r0, r1, r2], axis=1), axis=1)[:, ::-1]
    a, b, c = r[:, 0].astype(np.int64), r[:, 1].astype(np.int64), r[:, 2].astype(np.int64)
    trips = a == c
    pair_hi = (a == b) & ~trips
    pair_lo = (b == c) & ~trips
    cat = np.where(trips, 2, np.where(pair_hi | pair_lo, 1, 0))
    val = np.where(trips, 2 * 4096 + a,
                   np.where(pair_hi, 4096 + a * 64 + c, np.where(pair_lo, 4096 + b * 64 + a, a * 256 + b * 16 + c)))
    return cat, val


def checkdown_value(spec) -> np.ndarray:
    """Player-1 payoff of the line that takes action 0 everywhere below each
    root outcome (check-check to the showdown in the card games)."""
    root = spec.child[spec.child_begin[0]:spec.child_begin[1]].astype(np.int64)
    cur = root.copy()
    for _ in range(64):
        term = spec.kind[cur] == 0
        if term.all():
            break
        cur = np.where(term, cur, spec.child[spec.child_begin[cur]].astype(np.int64))
    return spec.payoff[cur]


def features(spec, return_mass: bool = False, handle: Optional[int] = None) -> tuple:
    """(X [I, F_IN] float32, nact [I] int32) for every information set
    (and the sets' chance masses when return_mass). The chance sums behind
    the range weight and the equity come from the compiled game (the
    library's cfr_set_chance_sums over the chance products the compiler
    folded); handle: an already compiled handle of spec (else one is
    compiled here and released)."""
    f = spec.iset_feat
    if f is None:
        raise ValueError("features need the card-game metadata of the generator")
    I = spec.n_infosets
    X = np.zeros((I, F_IN), dtype=np.float32)
    rows = np.arange(I)
    X[rows, f[:, 1]] = 1.0
    X[rows, f[:, 2]] = 1.0
    has_board = f[:, 3] >= 0
    X[rows[has_board], 32 + f[has_board, 3]] = 1.0
    if has_board.any():
        cat, val = _rank3_vec(f[has_board, 1] // N_SUITS, f[has_board, 2] // N_SUITS, f[has_board, 3] // N_SUITS)
        X[rows[has_board], 64 + cat] = 1.0
        X[rows[has_board], 67] = val / 8199.0
    X[rows, 68 + f[:, 0]] = 1.0
    X[rows, 70 + np.clip(f[:, 4], 0, 1)] = 1.0
    X[rows, 72 + np.clip(f[:, 5] - 1, 0, 7)] = 1.0
    for pos in range(8):
        code = f[:, 6 + pos]
        ok = code >= 0
        X[rows[ok], 80 + pos * 11 + np.clip(code[ok], 0, 10)] = 1.0
    c1, c2 = f[:, 14] / 2.0, f[:, 15] / 2.0
    X[:, 168] = c1 / 10.0
    X[:, 169] = c2 / 10.0
    me, op = np.where(f[:, 0] == 0, c1, c2), np.where(f[:, 0] == 0, c2, c1)
    X[:, 170] = (op - me) / 10.0
    # relative range weight: chance mass of the set over the mean of its
    # public state; equity against the opponent's range at the check-down
    # showdown: the chance-weighted share of the set's deals player 1 wins
    sd = checkdown_value(spec)
    win1 = (1.0 + np.sign(sd)) / 2.0
    own = handle is None
    h = cfr.cfr_compile(spec, cfr.make_options(precision=cfr.P32)) if own else handle
    try:
        mass, wsum = cfr.cfr_set_chance_sums(h, I, win1)
    finally:
        if own:
            cfr.cfr_destroy(h)
    eq1 = wsum / np.maximum(mass, 1e-300)
    eq = np.where(f[:, 0] == 0, eq1, 1.0 - eq1)
    X[:, 172] = eq
    X[rows, 173 + np.clip((eq * 10).astype(np.int64), 0, 9)] = 1.0
    # the public state: acting player, board card, round, betting history
    # (small integers, each shifted to be >= 0), packed into one int64 key
    key = np.zeros(I, dtype=np.int64)
    for col, width in ((0, 3), (3, 33), (4, 3)) + tuple((6 + p, 12) for p in range(8)):
        v = f[:, col].astype(np.int64) + 1
        if I and (v.min() < 0 or v.max() >= width):  # the packing is one-to-one only within these ranges
            raise ValueError("set feature %d outside the range the public-state key packs" % col)
        key = key * width + v
    _, grp = np.unique(key, return_inverse=True)
    grp = grp.reshape(-1)
    gmean = np.bincount(grp, weights=mass) / np.maximum(np.bincount(grp), 1)
    rel = mass / np.maximum(gmean[grp], 1e-300)
    X[:, 171] = np.clip(np.log(np.maximum(rel, 1e-12)), -5.0, 5.0) / 5.0
    nact = spec.iset_nact.astype(np.int32)
    if nact.max(initial=0) > N_OUT:
        raise ValueError("information sets with more than %d actions" % N_OUT)
    return (X, nact, mass) if return_mass else (X, nact)


def _pad_slots(spec, vec) -> np.ndarray:
    """Slot vector (spec order) -> [I, N_OUT] rows padded with zeros."""
    off = spec.slot_offsets()
    out = np.zeros((spec.n_infosets, N_OUT), dtype=np.float32)
    na = spec.iset_nact
    for a in range(N_OUT):
        ok = na > a
        out[ok, a] = vec[off[:-1][ok] + a]
    return out


def solve_batch(specs, iters: int, precision=cfr.P32, threads=1024, lanes=8, chunk=256, init=None,
                with_features: bool = False):
    """Average strategies of `specs` after `iters` CFR+ iterations (batched);
    with_features also returns every game's (X, nact), computed from the
    same compiled handles."""
    import torch

    out, feats = [], []
    s = int(torch.cuda.current_stream().cuda_stream)
    opts = cfr.make_options(precision=precision)
    for c0 in range(0, len(specs), chunk):
        part = specs[c0:c0 + chunk]
        hs = compile_many(part, opts)
        if with_features:
            workers = min(16, os.cpu_count() or 1)
            with ThreadPoolExecutor(workers) as ex:
                feats += list(ex.map(lambda a: features(a[0], handle=a[1]), zip(part, hs)))
        sizes = [cfr.cfr_plan(h) for h in hs]
        pool = serve.DevicePool(sum(n + serve.ALIGN for n in sizes) + serve.ALIGN)
        for j, (h, n) in enumerate(zip(hs, sizes)):
            cfr.cfr_bind(h, pool.ptr(pool.alloc(n)), n, s)
            if init is not None and init[c0 + j] is not None:
                A = cfr.cfr_get_counts(h)["n_slots"]
                cfr.cfr_set_state(h, init[c0 + j], np.zeros(A), 0, s)
        tb = cfr.cfr_batch_table_bytes(len(hs))
        table = torch.empty(tb + 16, dtype=torch.uint8, device="cuda")
        cfr.cfr_batch_iterate(hs, iters, (table.data_ptr() + 15) & ~15, tb, threads, lanes, s)
        for h in hs:
            v = np.empty(cfr.cfr_get_counts(h)["n_slots"])
            cfr.cfr_avg_strategy(h, v, False, s)
            out.append(v)
            cfr.cfr_destroy(h)
    return (out, feats) if with_features else out


def make_dataset(specs, iters: int = 1000, max_sets_per_game: int = 256, seed: int = 0):
    """Features and target strategies of (a sample of) every game's sets."""
    rng = np.random.default_rng(seed)
    strat, feats = solve_batch(specs, iters, with_features=True)
    Xs, Ns, Ts = [], [], []
    for sp, st, (X, na) in zip(specs, strat, feats):
        T = _pad_slots(sp, st)
        idx = np.arange(sp.n_infosets)
        if len(idx) > max_sets_per_game:
            idx = rng.choice(idx, size=max_sets_per_game, replace=False)
        Xs.append(X[idx]); Ns.append(na[idx]); Ts.append(T[idx])
    return np.concatenate(Xs), np.concatenate(Ns), np.concatenate(Ts)


def train(X, nact, T, epochs: int = 3, batch: int = 4096, lr: float = 2e-3, seed: int = 0, log=None) -> MLP:
    import torch

    net = MLP(F_IN, seed=seed)
    dev = net.dev
    Xd = torch.tensor(X, device=dev)
    Nd = torch.tensor(nact, device=dev)
    Td = torch.tensor(T, device=dev)
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n), device=dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            loss = net.loss_and_grad(Xd[idx].contiguous(), Nd[idx].contiguous(), Td[idx].contiguous())
            net.adam_step(lr * (0.5 ** ep))
            tot += loss
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    net.history = hist
    return net


def _regrets_from(spec, prob: np.ndarray, mass: np.ndarray, kappa: float) -> np.ndarray:
    off = spec.slot_offsets()
    R0 = np.zeros(int(off[-1]))
    for a in range(N_OUT):
        ok = spec.iset_nact > a
        R0[off[:-1][ok] + a] = prob[ok, a] * mass[ok]
    return kappa * spec.pot * R0


def warm_regrets(net: MLP, spec, kappa: float) -> np.ndarray:
    """R0 in spec slot order: kappa * pot * mass(I) * sigma_hat(I, a), i.e.
    about kappa iterations' worth of regret pointing at the network's
    strategy (mass(I) = chance probability of reaching I, the scale of one
    iteration's regret increment at I)."""
    return warm_regrets_many(net, [spec], kappa, workers=1)[0]


def warm_regrets_many(net: MLP, specs, kappa: float, workers: Optional[int] = None,
                      handles: Optional[list] = None, timings: Optional[dict] = None) -> List[np.ndarray]:
    """warm_regrets for many games: their features computed on a thread pool
    (the library and NumPy's array loops release the interpreter lock), from
    the games' compiled handles when given, then one network pass over every
    game's sets. timings (optional) receives the seconds of each part."""
    import torch

    t0 = time.perf_counter()
    workers = workers or min(16, os.cpu_count() or 1)
    hs = handles if handles is not None else [None] * len(specs)
    if workers > 1 and len(specs) > 1:
        with ThreadPoolExecutor(workers) as ex:
            feats = list(ex.map(lambda a: features(a[0], return_mass=True, handle=a[1]), zip(specs, hs)))
    else:
        feats = [features(sp, return_mass=True, handle=h) for sp, h in zip(specs, hs)]
    t1 = time.perf_counter()
    X = np.concatenate([f[0] for f in feats])
    na = np.concatenate([f[1] for f in feats])
    prob = net.predict(torch.tensor(X, device=net.dev), torch.tensor(na, device=net.dev)).cpu().numpy()
    t2 = time.perf_counter()
    out, row = [], 0
    for sp, (_, nag, mass) in zip(specs, feats):
        out.append(_regrets_from(sp, prob[row:row + len(nag)], mass, kappa))
        row += len(nag)
    if timings is not None:
        timings.update(features_s=t1 - t0, inference_s=t2 - t1, regrets_s=time.perf_counter() - t2,
                       sets=int(X.shape[0]))
    return out


def compile_many(specs, opts, workers: Optional[int] = None):
    """cfr_compile of every spec on a thread pool (the compiler releases the
    interpreter lock)."""
    workers = workers or min(16, os.cpu_count() or 1)
    if workers > 1 and len(specs) > 1:
        with ThreadPoolExecutor(workers) as ex:
            return list(ex.map(lambda sp: cfr.cfr_compile(sp, opts), specs))
    return [cfr.cfr_compile(sp, opts) for sp in specs]


def iterations_to_target(specs, init=None, target=1e-3, check_every=50, max_iters=5000, threads=1024, lanes=8,
                         net: Optional[MLP] = None, kappa: float = 8.0, timings: Optional[dict] = None):
    """Iterations each game needs to reach target * pot (checked every
    `check_every`), all games in one batch, and the wall time (compile,
    then for a warm start the features of the compiled games and one
    network pass, then the solves). init: initial regrets per game (spec
    slot order); or net: the warm start computed here from the handles."""
    import torch

    s = int(torch.cuda.current_stream().cuda_stream)
    opts = cfr.make_options(precision=cfr.P32)
    t0 = time.perf_counter()
    hs = compile_many(specs, opts)
    tc = time.perf_counter()
    tw = {}
    if net is not None:
        init = warm_regrets_many(net, specs, kappa, handles=hs, timings=tw)
    t_warm = time.perf_counter()
    sizes = [cfr.cfr_plan(h) for h in hs]
    pool = serve.DevicePool(sum(n + serve.ALIGN for n in sizes) + serve.ALIGN)
    for j, (h, n) in enumerate(zip(hs, sizes)):
        cfr.cfr_bind(h, pool.ptr(pool.alloc(n)), n, s)
        if init is not None:
            cfr.cfr_set_state(h, init[j], np.zeros(len(init[j])), 0, s)
    tb = cfr.cfr_batch_table_bytes(len(hs))
    table = torch.empty(tb + 16, dtype=torch.uint8, device="cuda")
    tp = (table.data_ptr() + 15) & ~15
    t_bind = time.perf_counter()
    done = np.zeros(len(hs), dtype=np.int64)
    finished = np.zeros(len(hs), dtype=bool)
    active = list(range(len(hs)))
    while active:
        sub = [hs[i] for i in active]
        cfr.cfr_batch_iterate(sub, check_every, tp, tb, threads, lanes, s)
        ex = cfr.cfr_batch_exploitability(sub, tp, tb, threads, lanes, s)
        keep = []
        for i, row in zip(active, ex):
            done[i] += check_every
            if row[0] <= target * specs[i].pot:
                finished[i] = True
            elif done[i] < max_iters:
                keep.append(i)
        active = keep
    t_end = time.perf_counter()
    wall = t_end - t0
    if timings is not None:
        timings.update(compile_s=tc - t0, warm_start_s=t_warm - tc, bind_s=t_bind - t_warm, solve_s=t_end - t_bind, **tw)
    for h in hs:
        cfr.cfr_destroy(h)
    return done, finished, wall


def time_to_target_alone(spec, net: Optional[MLP] = None, kappa: float = 8.0, target: float = 1e-3,
                         check_every: int = 50, max_iters: int = 5000):
    """One game solved on its own, the way a single real-time re-solve runs:
    compile, bind, (warm start: features from the compiled game, one
    network pass, the initial regrets), then CFR+ in the single-game form
    chosen by size (cfr EXEC_AUTO) with the exploitability checked every
    `check_every` iterations. Returns (iterations, seconds, reached)."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = cfr.Solver(spec, precision=cfr.P32, exec_form=cfr.EXEC_AUTO)
    if net is not None:
        R0 = warm_regrets_many(net, [spec], kappa, workers=1, handles=[s.h])[0]
        s.set_state(R0, np.zeros(len(R0)), 0)
    done, reached = 0, False
    pot = float(getattr(spec, "pot", 1.0))
    while done < max_iters:
        n = min(check_every, max_iters - done)
        s.iterate(n)
        done += n
        if s.exploitability() <= target * pot:
            reached = True
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return done, dt, reached


def iter_endgame_family(seeds, lo: float = 1e3, hi: float = 1e6):
    """Endgames with edge targets log-uniform in [lo, hi] (seeded per list),
    generated one at a time."""
    import gamegen as gg

    seeds = list(seeds)
    rng = np.random.default_rng(int(seeds[0]) if len(seeds) else 0)
    for s in seeds:
        yield gg.endgame(int(s), int(np.exp(rng.uniform(np.log(lo), np.log(hi)))))


def endgame_family(seeds, lo: float = 1e3, hi: float = 1e6):
    """Endgames with edge targets log-uniform in [lo, hi] (seeded per list)."""
    return list(iter_endgame_family(seeds, lo, hi))


def choose_kappa(net: MLP, specs, kappas=(4.0, 8.0, 16.0), max_iters: int = 3000):
    """The kappa with the fewest mean iterations to 1e-3 pot on `specs`."""
    best, best_it, table = None, float("inf"), {}
    for k in kappas:
        done, fin, _ = iterations_to_target(specs, net=net, kappa=k, max_iters=max_iters)
        table[k] = float(np.mean(done))
        if table[k] < best_it:
            best, best_it = k, table[k]
    return best, table
