"""Pins for the oracle's genetic algorithm (Appendix B: elitism, tournament
of two, one-point crossover, mutation decaying over the generations).

The checks use properties fixed by those operators: the elites are the two
best individuals; a two-way tournament with replacement puts the winner in
the better half with probability exactly 3/4; a crossover child is a prefix
of one parent followed by a suffix of the other, with the cut uniform on
1..G-1; the mutation frequency matches 0.2 (1 - g/NG) + 0.01 within a
binomial bound and mutated genes stay in bounds.
"""
import math

import numpy as np
import pytest


def _bound(p, n, k=5.0):
    return k * math.sqrt(p * (1 - p) / n) + 1.0 / n


def test_elites_are_the_two_best_with_nan_worst_and_ties_to_lower_index(
        oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(50):
        P, G = int(rng.integers(2, 40)), int(rng.integers(1, 8))
        genes = rng.normal(0, 5, (P, G))
        f = rng.integers(0, 6, P).astype(float)   # many ties
        f[rng.random(P) < 0.2] = np.nan
        out = oracle_mod.ga_step(genes, f, 3, 10, int(rng.integers(1 << 40)),
                                 [-100] * G, [100] * G)
        order = sorted(range(P), key=lambda i: (math.isnan(f[i]),
                                                0 if math.isnan(f[i]) else f[i],
                                                i))
        assert np.array_equal(out[0], genes[order[0]])
        assert np.array_equal(out[1], genes[order[1]])


def test_single_individual_is_kept():
    import oracle

    out = oracle.ga_step([[1.0, 2.0]], [0.5], 0, 5, 1, [-9, -9], [9, 9])
    assert np.array_equal(out, [[1.0, 2.0]])


def test_tournament_winner_in_better_half_three_quarters(oracle_mod):
    """G = 1 (no crossover), gene = individual index: an unmutated child's
    gene names its parent."""
    P = 8192
    genes = np.arange(P, dtype=float).reshape(P, 1)
    f = np.random.default_rng(1).permutation(P).astype(float)
    rank = np.argsort(np.argsort(f))
    hits = n = 0
    for seed in range(4):
        out = oracle_mod.ga_step(genes, f, 99, 100, seed, [-1e9], [1e9])
        child = out[2:, 0]
        clean = child == np.round(child)      # unmutated genes stay integral
        par = child[clean].astype(int)
        hits += int((rank[par] < P // 2).sum())
        n += par.size
    assert abs(hits / n - 0.75) <= _bound(0.75, n)


def test_crossover_children_are_prefix_suffix_swaps(oracle_mod):
    P, G = 2050, 6
    base = np.arange(P, dtype=float)[:, None] * 100.0
    genes = base + np.arange(G)[None, :]
    f = np.random.default_rng(2).random(P)
    cuts = []
    for seed in range(3):
        out = oracle_mod.ga_step(genes, f, 99, 100, 10 + seed, [-1e9] * G,
                                 [1e9] * G)
        for j in range(2, P - 1, 2):
            a, b = out[j], out[j + 1]
            ida = (a - np.arange(G)) / 100.0
            idb = (b - np.arange(G)) / 100.0
            ok = (ida == np.round(ida)) & (idb == np.round(idb))
            if not ok.all():
                continue                      # a gene mutated: skip the pair
            pa0, pb0 = ida[0], idb[0]
            c = next((k for k in range(1, G) if ida[k] != pa0), G)
            assert c < G or (ida == pa0).all()
            if c == G:
                continue                      # both parents were the same one
            # after the cut the two children have exchanged parents
            assert (ida[:c] == pa0).all() and (idb[:c] == pb0).all()
            assert (ida[c:] == pb0).all() and (idb[c:] == pa0).all()
            cuts.append(c)
    hist = np.bincount(cuts, minlength=G)[1:G]
    exp = len(cuts) / (G - 1)
    assert (((hist - exp) ** 2) / exp).sum() < 4 + 6 * math.sqrt(8)


@pytest.mark.parametrize("g,NG", [(0, 50), (25, 50), (49, 50)])
def test_mutation_rate_and_bounds(oracle_mod, g, NG):
    P, G = 4000, 5
    lo, hi = np.full(G, -30.0), np.full(G, 30.0)
    genes = np.random.default_rng(3).uniform(-29, 29, (P, G))
    f = np.zeros(P)                       # all ties: parents by index order
    out = oracle_mod.ga_step(genes, f, g, NG, 77, lo, hi)
    s = 1 - g / NG
    pm = 0.2 * s + 0.01
    scale = 0.1 * 60.0 * s
    # With identical fitness each tournament returns the lower contestant;
    # a gene mutated iff it is not one of the population's gene values.
    pool = set(genes.ravel().tolist())
    mut = np.array([[v not in pool for v in row] for row in out[2:]])
    n = mut.size
    assert abs(mut.mean() - pm) <= _bound(pm, n)
    assert np.all(out >= lo) and np.all(out <= hi)
    # a mutated gene moved by at most the step scale from some parent value
    vals = np.sort(genes.ravel())
    for v in out[2:][mut][:300]:
        k = np.searchsorted(vals, v)
        d = min(abs(v - vals[max(k - 1, 0)]), abs(v - vals[min(k, vals.size - 1)]))
        assert d <= scale + 1e-12 or v in (-30.0, 30.0)


def test_ga_is_deterministic_and_seed_dependent(oracle_mod):
    rng = np.random.default_rng(4)
    genes, f = rng.normal(0, 5, (64, 5)), rng.random(64)
    a = oracle_mod.ga_step(genes, f, 1, 10, 5, [-30] * 5, [30] * 5)
    b = oracle_mod.ga_step(genes, f, 1, 10, 5, [-30] * 5, [30] * 5)
    c = oracle_mod.ga_step(genes, f, 1, 10, 6, [-30] * 5, [30] * 5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_group_mean_against_exact_sum(oracle_mod):
    rng = np.random.default_rng(5)
    v = rng.normal(0, 1e3, 16 * 37)
    got = oracle_mod.group_mean(v, 16)
    want = [math.fsum(v[i * 16:(i + 1) * 16]) / 16 for i in range(37)]
    assert np.allclose(got, want, rtol=1e-13, atol=0)
