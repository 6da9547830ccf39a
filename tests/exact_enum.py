"""Exact burn probabilities of the automaton on tiny grids (test helper).

Enumerates every reachable (per-cell state) configuration of the synchronous
automaton of Sec. 2.1 with the exact per-trial success probability T / 2^32
taken from the oracle's threshold table.  A target cell with burning
neighbours in directions D ignites with probability 1 - prod_{d in D}
(1 - T_d / 2^32), independently of every other target cell in the same step;
burning cells burn out after one step.  Used to check the oracle's Monte
Carlo frequencies on grids of at most nine cells.
"""
from itertools import product

import numpy as np

DIRS = ((-1, 0), (-1, 1), (0, 1), (1, 1), (1, 0), (1, -1), (0, -1), (-1, -1))
UNBURNT, BURNING, BURNT, BLOCKED = 0, 1, 2, 3


def exact_burn_probability(burnable, T, ignition):
    """P(cell ever burns) for every cell; T is uint64 (8, H, W)."""
    H, W = burnable.shape
    n = H * W
    start = [UNBURNT if burnable.flat[i] else BLOCKED for i in range(n)]
    ign = ignition[0] * W + ignition[1]
    start[ign] = BURNING
    frontier = {tuple(start): 1.0}
    p_burn = np.zeros(n)
    p_burn[ign] = 1.0
    q = T.astype(np.float64) / 2.0 ** 32
    while frontier:
        nxt = {}
        for state, pr in frontier.items():
            cands, probs = [], []
            for i in range(n):
                if state[i] != UNBURNT:
                    continue
                r, c = divmod(i, W)
                miss = 1.0
                hit = False
                for d, (dr, dc) in enumerate(DIRS):
                    sr, sc = r - dr, c - dc
                    if 0 <= sr < H and 0 <= sc < W and \
                            state[sr * W + sc] == BURNING:
                        hit = True
                        miss *= 1.0 - q[d, r, c]
                if hit:
                    cands.append(i)
                    probs.append(1.0 - miss)
            base = [BURNT if s == BURNING else s for s in state]
            if not cands:
                continue  # extinct: absorbing
            for pick in product((0, 1), repeat=len(cands)):
                w = pr
                s = list(base)
                for i, p, k in zip(cands, probs, pick):
                    w *= p if k else (1.0 - p)
                    if k:
                        s[i] = BURNING
                if w == 0.0:
                    continue
                for i, k in zip(cands, pick):
                    if k:
                        p_burn[i] += w
                key = tuple(s)
                nxt[key] = nxt.get(key, 0.0) + w
        frontier = nxt
    return p_burn.reshape(H, W)
