"""Pins of the CPU oracle (Algorithm 2 in oracle/alg2.c) to things other than
itself: the paper's printed worked examples, closed forms, exhaustive search
from the definition, the literal Algorithm 1, and invariants."""
import itertools
import os

import numpy as np
import pytest

import graphgen
import oracle
from oracle import checks

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def fig2():
    """Figure 2 graph: edges as (a, b) ids with a=0 ... l=11, and its classes."""
    classes = {}
    for parts in _read_fixture("fig2_example2.txt"):
        k = int(parts[0])
        for p in parts[1:]:
            a, b = ord(p[0]) - ord("a"), ord(p[1]) - ord("a")
            classes[(min(a, b), max(a, b))] = k
    return classes


def run(edges, n=None):
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    if n is None:
        n = int(max(src.max(), dst.max())) + 1 if len(edges) else 1
    r = oracle.truss(n, src, dst)
    sup = {e: int(s) for e, s in zip(edges, r.support)}
    phi = {e: int(t) for e, t in zip(edges, r.truss)}
    return sup, phi, r


def clique(vs):
    return [(a, b) for a, b in itertools.combinations(sorted(vs), 2)]


# ------------------------------------------------------------ worked example
def test_fig2_classes_as_printed():
    classes = fig2()
    edges = sorted(classes)
    assert len(edges) == 26
    sup, phi, r = run(edges)
    assert phi == classes
    assert r.kmax == 5
    assert r.m == 26


def test_fig2_example4_support_and_psi():
    vals = {k: int(v) for k, v in _read_fixture("fig2_example4.txt")}
    classes = fig2()
    edges = sorted(classes)
    sup, phi, _ = run(edges)
    d, g = 3, 6
    assert sup[(d, g)] == vals["sup_dg"]
    nb = checks.adjacency(edges)
    key = lambda a, b: (min(a, b), max(a, b))
    x_d = checks.h_index([sup[key(d, z)] for z in nb[d] if z != g])
    x_g = checks.h_index([sup[key(g, z)] for z in nb[g] if z != d])
    assert x_d == vals["x_d"] and x_g == vals["x_g"]
    psi = checks.psi_upper(edges, sup)
    assert psi[(d, g)] == vals["psi_dg"]
    assert all(psi[e] == vals["psi_class5"] for e in edges if classes[e] == 5)


def test_fig2_example5_top2():
    rows = {p[0]: p[1:] for p in _read_fixture("fig2_example5.txt")}
    classes = fig2()
    edges = sorted(classes)
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    sup, ps = oracle.psi(12, src, dst)
    assert int(ps.max()) == int(rows["first_k"][0])
    t = int(rows["t"][0])
    top, kmax = oracle.top(12, src, dst, t)
    key = lambda p: (min(ord(p[0]) - 97, ord(p[1]) - 97), max(ord(p[0]) - 97, ord(p[1]) - 97))
    want4 = sorted(key(p) for p in rows["class4"])
    got4 = sorted(e for e, v in zip(edges, top) if v == 4)
    assert got4 == want4
    assert sorted(e for e, v in zip(edges, top) if v == 5) == sorted(
        e for e in edges if classes[e] == 5)
    assert all(v in (0, 4, 5) for v in top) and kmax == 5


@pytest.mark.parametrize("seed", range(12))
def test_psi_counting_equals_definition(seed):
    """oracle.psi (counting h-index in C) against checks.psi_upper (sorted
    lists in Python), and Lemma 2 (phi <= psi) with the oracle's phi."""
    n = 20 + 7 * seed
    src, dst = graphgen.er(n, 3 * n, seed=seed)
    perm = graphgen.permutation(n, seed=seed, stream=1)
    src, dst = graphgen.add_cliques(src, dst, perm[:10], [4, 6])
    edges = checks.canonical_edges(src, dst)
    s = np.array([a for a, _ in edges], np.int32)
    d = np.array([b for _, b in edges], np.int32)
    sup, ps = oracle.psi(n, s, d)
    sd = {e: int(x) for e, x in zip(edges, sup)}
    want = checks.psi_upper(edges, sd)
    assert [int(x) for x in ps] == [want[e] for e in edges]
    r = oracle.truss(n, s, d)
    assert (r.truss <= ps).all()


def test_top_t_is_the_full_decomposition_restricted():
    src, dst = graphgen.rmat_raw(9, 16 << 9, seed=4)
    r = oracle.truss(1 << 9, src, dst)
    for t in (1, 2, 5, 1000):
        top, kmax = oracle.top(1 << 9, src, dst, t)
        thr = max(kmax - t + 1, 2)
        keep = r.truss >= thr
        assert (top[keep] == r.truss[keep]).all()
        assert (top[(r.truss >= 0) & ~keep] == 0).all()
        assert (top[r.truss < 0] == -1).all()
        assert kmax == r.kmax


def test_fig2_support_matches_definition():
    edges = sorted(fig2())
    sup, _, r = run(edges)
    assert sup == checks.support_triples(edges)
    assert sum(sup.values()) == 3 * checks.triangle_count_trace(12, edges)
    assert r.triangles * 3 == sum(sup.values())


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", range(2, 13))
def test_complete_graph(n):
    sup, phi, r = run(clique(range(n)))
    assert set(sup.values()) == {n - 2}
    assert set(phi.values()) == {n}
    assert r.kmax == n


@pytest.mark.parametrize("n", range(4, 11))
def test_complete_minus_edge(n):
    edges = [e for e in clique(range(n)) if e != (0, 1)]
    _, phi, _ = run(edges)
    assert set(phi.values()) == {n - 1}


@pytest.mark.parametrize("rim", range(4, 12))
def test_wheel(rim):
    edges = [(0, i) for i in range(1, rim + 1)]
    edges += [(min(i, i % rim + 1), max(i, i % rim + 1)) for i in range(1, rim + 1)]
    sup, phi, _ = run(sorted(set(edges)))
    assert set(phi.values()) == {3}
    assert all(sup[(0, i)] == 2 for i in range(1, rim + 1))


@pytest.mark.parametrize("pages", [1, 2, 5, 17])
def test_book(pages):
    edges = [(0, 1)] + [(0, 2 + i) for i in range(pages)] + [(1, 2 + i) for i in range(pages)]
    sup, phi, _ = run(edges)
    assert set(phi.values()) == {3}
    assert sup[(0, 1)] == pages


def test_triangle_free_graphs():
    path = [(i, i + 1) for i in range(20)]
    cycle = [(i, (i + 1) % 9) for i in range(9)]
    cycle = [(min(a, b), max(a, b)) for a, b in cycle]
    kab = [(a, 5 + b) for a in range(5) for b in range(7)]
    star = [(0, i) for i in range(1, 30)]
    for edges in (path, cycle, kab, star):
        sup, phi, _ = run(edges)
        assert set(sup.values()) == {0}
        assert set(phi.values()) == {2}


def test_disjoint_union_is_componentwise():
    parts = [clique(range(5)), [(a + 5, b + 5) for a, b in clique(range(7))],
             [(12 + i, 12 + (i + 1) % 6) for i in range(5)] + [(12, 17)],
             [(a + 18, b + 18) for a, b in sorted(fig2())]]
    union = sorted(set(itertools.chain(*parts)))
    _, phi_u, _ = run(union)
    for p in parts:
        _, phi_p, _ = run(sorted(p), n=40)
        assert all(phi_u[e] == phi_p[e] for e in p)


def test_empty_and_degenerate():
    r = oracle.truss(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert r.m == 0 and len(r.support) == 0 and r.kmax == 0
    # only self-loops
    r = oracle.truss(3, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32))
    assert list(r.support) == [-1, -1, -1] and list(r.truss) == [-1, -1, -1]
    # a single edge
    r = oracle.truss(2, np.array([1], np.int32), np.array([0], np.int32))
    assert list(r.support) == [0] and list(r.truss) == [2] and r.kmax == 2
    with pytest.raises(ValueError):
        oracle.truss(3, np.array([0], np.int32), np.array([3], np.int32))


# ------------------------------------------------------------ brute force
def _random_small(seed, n, m):
    src, dst = graphgen.er(n, m, seed=seed, stream=7)
    return sorted({(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist())})


@pytest.mark.parametrize("seed", range(60))
def test_bruteforce_from_definition(seed):
    n = 5 + seed % 4
    m = min(n * (n - 1) // 2, 8 + seed % 6)
    edges = _random_small(seed, n, m)
    sup, phi, _ = run(edges, n=n)
    assert phi == checks.truss_bruteforce(edges)
    assert sup == checks.support_triples(edges)


@pytest.mark.parametrize("seed", range(12))
def test_alg1_literal(seed):
    n = 40 + 10 * seed
    m = 3 * n + 40 * seed
    src, dst = graphgen.er(n, m, seed=1000 + seed, stream=0)
    perm = graphgen.permutation(n, seed=1000 + seed, stream=1)
    s = 4 + seed % 9
    src, dst = graphgen.add_cliques(src, dst, perm[:s], [s])
    edges = checks.canonical_edges(src, dst)
    sup, phi, r = run(edges, n=n)
    assert phi == checks.truss_alg1(edges)
    assert sup == checks.support_triples(edges)
    assert all(phi[e] >= s for e in clique(perm[:s].tolist()))


@pytest.mark.parametrize("seed", range(4))
def test_alg1_rmat(seed):
    src, dst = graphgen.rmat_distinct(8, 1200, seed=77 + seed)
    edges = checks.canonical_edges(src, dst)
    sup, phi, _ = run(edges, n=256)
    assert phi == checks.truss_alg1(edges)
    assert sup == checks.support_triples(edges)


@pytest.mark.parametrize("seed", range(6))
def test_invariants(seed):
    n = 60 + 20 * seed
    src, dst = graphgen.er(n, 5 * n, seed=500 + seed)
    perm = graphgen.permutation(n, seed=500 + seed, stream=1)
    src, dst = graphgen.add_cliques(src, dst, perm[:16], [7, 9])
    edges = checks.canonical_edges(src, dst)
    sup, phi, r = run(edges, n=n)
    assert checks.invariants(edges, sup, phi) == []
    assert r.triangles == checks.triangle_count_trace(n, edges)


def test_support_sum_is_three_times_triangles():
    for seed in range(5):
        src, dst = graphgen.rmat_distinct(8, 1500, seed=seed)
        edges = checks.canonical_edges(src, dst)
        sup, _, r = run(edges, n=256)
        assert sum(sup.values()) == 3 * checks.triangle_count_trace(256, edges)


# ------------------------------------------------------------ metamorphic
def test_metamorphic_relabel_permute_duplicate():
    n, src, dst = 300, *graphgen.er(300, 1500, seed=9)
    perm = graphgen.permutation(n, seed=9, stream=1)
    src, dst = graphgen.add_cliques(src, dst, perm[:10], [10])
    base = oracle.truss(n, src, dst)
    # reversed rows
    r = oracle.truss(n, dst, src)
    assert (r.support == base.support).all() and (r.truss == base.truss).all()
    # vertex relabelling
    relab = graphgen.permutation(n, seed=10, stream=0)
    r = oracle.truss(n, relab[src], relab[dst])
    assert (r.support == base.support).all() and (r.truss == base.truss).all()
    # row permutation
    order = graphgen.permutation(len(src), seed=11, stream=0)
    r = oracle.truss(n, src[order], dst[order])
    assert (r.truss == base.truss[order]).all() and (r.support == base.support[order]).all()
    # duplicated rows and self-loops appended
    s2 = np.concatenate([src, dst[:50], np.arange(7, dtype=np.int32)])
    d2 = np.concatenate([dst, src[:50], np.arange(7, dtype=np.int32)])
    r = oracle.truss(n, s2, d2)
    L = len(src)
    assert (r.truss[:L] == base.truss).all()
    assert (r.truss[L:L + 50] == base.truss[:50]).all()
    assert (r.truss[L + 50:] == -1).all() and (r.support[L + 50:] == -1).all()


# ------------------------------------------------------------ C checker
def test_c_validity_checker_accepts_oracle_and_rejects_mistakes():
    n, src, dst = graphgen.tiny()
    r = oracle.truss(n, src, dst)
    assert oracle.check_valid(n, src, dst, r.truss, r.support) == 0
    # planted mistakes in the oracle's output must be caught
    t = r.truss.copy()
    i = int(np.argmax(t))
    t[i] += 1
    assert oracle.check_valid(n, src, dst, t, r.support) > 0
    s = r.support.copy()
    j = int(np.nonzero(r.truss == 2)[0][0])
    s[j] += 1
    assert oracle.check_valid(n, src, dst, r.truss, s) > 0


def test_tiny_config_planted_cliques():
    n, src, dst = graphgen.tiny()
    r = oracle.truss(n, src, dst)
    perm = graphgen.permutation(n, seed=0, stream=1)
    base = 0
    key = {}
    eu, ev, r2e = oracle.edges(n, src, dst)
    phi_e = np.empty(len(eu), np.int32)
    phi_e[r2e] = r.truss
    for i, (a, b) in enumerate(zip(eu.tolist(), ev.tolist())):
        key[(a, b)] = phi_e[i]
    for s in graphgen.TINY_CLIQUES:
        vs = sorted(perm[base:base + s].tolist())
        base += s
        assert all(key[e] >= s for e in clique(vs))
    assert r.kmax == 32


def test_sampled_checker_accepts_oracle_and_rejects_mistakes():
    n, (src, dst) = 2 ** 12, graphgen.rmat_raw(12, 16 * 2 ** 12, seed=21)
    r = oracle.truss(n, src, dst)
    sample = np.arange(0, len(src), 7, dtype=np.int64)
    bad, sup = oracle.check_sample(n, src, dst, r.truss, r.support, sample)
    assert bad == 0 and np.array_equal(sup, r.support[sample])
    t = r.truss.copy()
    i = int(np.argmax(t))
    t[i] += 1  # too high a truss number is not locally valid
    bad, _ = oracle.check_sample(n, src, dst, t, r.support, np.array([i], np.int64))
    assert bad == 1
    s = r.support.copy()
    s[sample[3]] += 1
    bad, _ = oracle.check_sample(n, src, dst, r.truss, s, sample)
    assert bad == 1


# ------------------------------------------------------------ core numbers
@pytest.mark.parametrize("seed", range(8))
def test_core_bins_equal_min_degree_deletion(seed):
    """oracle.core (bin-sorted degree array, C) against checks.core_numbers
    (repeated min-degree deletion, Python)."""
    n = 40 + 9 * seed
    src, dst = graphgen.er(n, 4 * n, seed=seed)
    perm = graphgen.permutation(n, seed=seed, stream=1)
    src, dst = graphgen.add_cliques(src, dst, perm[:12], [5, 7])
    edges = checks.canonical_edges(src, dst)
    core, kmax = oracle.core(n, src, dst)
    want = checks.core_numbers(edges)
    assert [int(c) for c in core] == [want.get(v, 0) for v in range(n)]
    assert kmax == max(want.values())


def test_core_closed_forms():
    def core_of(n, edges):
        s = np.array([a for a, _ in edges], np.int32)
        d = np.array([b for _, b in edges], np.int32)
        return [int(x) for x in oracle.core(n, s, d)[0]]
    assert core_of(7, clique(range(7))) == [6] * 7                       # K_n: n - 1
    assert core_of(6, [(i, (i + 1) % 6) for i in range(6)]) == [2] * 6   # cycle: 2
    assert core_of(5, [(i, i + 1) for i in range(4)]) == [1] * 5         # path: 1
    assert core_of(6, [(0, i) for i in range(1, 6)]) == [1] * 6          # star: 1
    assert core_of(4, [(0, 1)]) == [1, 1, 0, 0]                          # isolated: 0
    kab = [(a, b) for a in range(3) for b in range(3, 8)]                # K_{3,5}: 3
    assert core_of(8, kab) == [3] * 8


def test_truss_lies_in_the_core():
    """Every edge of the k-truss has both endpoints in the (k-1)-core."""
    n, src, dst = graphgen.tiny()
    core, _ = oracle.core(n, src, dst)
    r = oracle.truss(n, src, dst)
    ok = r.truss > 0
    assert (core[src[ok]] >= r.truss[ok] - 1).all()
    assert (core[dst[ok]] >= r.truss[ok] - 1).all()


# ------------------------------------------- bottom-up under a budget (Sec. 5)
@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("budget", [8, 40, 150])
def test_bottom_up_equals_algorithm2(seed, budget):
    """Algorithms 3 and 4 (plain Python, local truss numbers by the literal
    Algorithm 1) against Algorithm 2 on the whole graph."""
    n = 30 + 6 * seed
    src, dst = graphgen.er(n, 4 * n, seed=seed)
    perm = graphgen.permutation(n, seed=seed, stream=1)
    src, dst = graphgen.add_cliques(src, dst, perm[:13], [5, 8])
    edges = checks.canonical_edges(src, dst)
    _, phi, _ = run(edges, n)
    assert checks.bottom_up(n, edges, budget) == phi


def test_bottom_up_step8_reading():
    """A triangle {0, 1, 2} beside a path 3-...-9, budget 4: the first pass
    splits the triangle as {0, 1} | {2, 3} and moves (0, 1) to G_new; in the
    next pass (0, 2) and (1, 2) have support 0 in what is left of G although
    they lie in a triangle.  Testing the lower bound (3, set in the first
    pass) keeps them out of Phi_2; testing the support in H would not."""
    edges = [(0, 1), (0, 2), (1, 2)] + [(i, i + 1) for i in range(3, 9)]
    _, phi, _ = run(edges, 10)
    assert checks.bottom_up(10, edges, 4) == phi
    literal = checks.bottom_up(10, edges, 4, literal_phi2=True)
    assert phi[(0, 2)] == 3 and literal[(0, 2)] == 2 and literal[(1, 2)] == 2
