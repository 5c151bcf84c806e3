#!/usr/bin/env python3
"""Writes the oracle's exploitability of the two-round card game after T
iterations of CFR+ (simultaneous updates, linear averaging) into
``card_oracle.json`` beside this file.

Calls only ``oracle/`` (plain recursive FP64 CFR+ and exact best response)
on specs from ``gamegen``; nothing here touches the CUDA path. Each entry is
keyed by ``gamegen.spec_digest`` of the game, so a test that reads it checks
first that it generated the same game. The full game (264,306,001 nodes)
takes about half an hour of one core for 1,000 iterations; the stack-1
variant (68,395,921 nodes) about ten minutes.

  python tests/golden/make_card_oracle.py --game stack1|full [--iters 1000]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gamegen as gg  # noqa: E402
import oracle  # noqa: E402

GAMES = {
    # name: (generator arguments of gamegen.large_card, description)
    "stack1": ((8, 4, 1, 3), "two-round card game, 8 ranks x 4 suits, stack 1 ante, cap 3 bets per round"),
    "full": ((8, 4, 2, 3), "two-round card game, 8 ranks x 4 suits, stack 2 antes, cap 3 bets per round"),
}
OUT = os.path.join(HERE, "card_oracle.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--game", choices=sorted(GAMES), required=True)
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--checkpoints", default="100", help="extra iteration counts to record, comma separated")
    a = ap.parse_args()
    args, desc = GAMES[a.game]
    t0 = time.time()
    g = gg.large_card(*args)
    digest = gg.spec_digest(g)
    print("%s: %d nodes, digest %s (%.0f s)" % (a.game, g.n_nodes, digest, time.time() - t0), flush=True)
    o = oracle.Oracle(g)
    marks = sorted({int(x) for x in a.checkpoints.split(",") if x} | {a.iters})
    rec = {}
    for m in marks:
        o.iterate(m - o.t)
        b1, b2, u = o.best_response(o.avg_strategy())
        rec[str(m)] = {"exploitability": 0.5 * (b1 - b2), "br1": b1, "br2": b2, "u": u}
        print("T=%d expl %.9e (%.0f s)" % (m, 0.5 * (b1 - b2), time.time() - t0), flush=True)
    entry = {
        "cite": "oracle/ (recursive FP64 CFR+, simultaneous updates, linear averaging w_t = t; exact best "
                "response, eq. (exploitability)), written by tests/golden/make_card_oracle.py",
        "generator": "gamegen.large_card%r" % (args,), "description": desc, "spec_digest": digest,
        "n_nodes": g.n_nodes, "pot": g.pot, "by_iterations": rec,
        "oracle_seconds": round(time.time() - t0, 1),
    }
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[a.game] = entry
    tmp = OUT + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=2, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, OUT)


if __name__ == "__main__":
    main()
