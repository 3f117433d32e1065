"""Independent checkers written from the paper's definitions -- TEST
INFRASTRUCTURE ONLY (pure Python, small inputs).

Each function restates one definition or algorithm of Wang & Cheng, "Truss
Decomposition in Massive Networks", without sharing code with ``alg2.c``:

* :func:`support_triples`   -- Definition 1 (Section 2): count common
  neighbours of each edge's endpoints.
* :func:`truss_bruteforce`  -- Definition 2 (Section 2) by exhaustive search
  over edge subsets (m <= 16): T_k is the union of all subgraphs whose edges
  each have >= k-2 triangles inside them.
* :func:`truss_alg1`        -- Algorithm 1 (Section 3.1), the existing
  in-memory algorithm, literally: for k = 3, 4, ..., remove any edge with
  support < k-2, recomputing common neighbourhoods on the current graph.
* :func:`core_numbers`      -- k-core numbers (Section 1 relates the k-truss to
  the (k-1)-core).
* :func:`psi_upper`         -- the upper bound psi(e) = min{sup(e), x_u, x_v}+2
  of Procedure 6 (Section 6.2) with the whole graph as H.
* :func:`bottom_up`         -- Algorithm 3 (LowerBounding) and Algorithm 4 with
  Procedure 5 (Section 5) under an edge budget, with the local truss numbers
  taken from :func:`truss_alg1`; ``literal_phi2`` selects the reading of
  Algorithm 3 step 8 (see the function).
* :func:`invariants`        -- the checks a correct decomposition must pass.
"""
from __future__ import annotations

from collections import defaultdict


def canonical_edges(src, dst):
    """Distinct undirected non-loop pairs (a, b), a < b, sorted."""
    es = set()
    for a, b in zip(map(int, src), map(int, dst)):
        if a == b:
            continue
        es.add((a, b) if a < b else (b, a))
    return sorted(es)


def adjacency(edges):
    nb = defaultdict(set)
    for a, b in edges:
        nb[a].add(b)
        nb[b].add(a)
    return nb


def support_triples(edges):
    """Definition 1: sup(e) = |{w : (u,w) and (v,w) are edges}| for e = (u,v)."""
    nb = adjacency(edges)
    return {e: len(nb[e[0]] & nb[e[1]]) for e in edges}


def triangle_count_trace(n, edges):
    """Number of triangles as trace(A^3) / 6 (a closed form, numpy)."""
    import numpy as np
    A = np.zeros((n, n), dtype=np.int64)
    for a, b in edges:
        A[a, b] = A[b, a] = 1
    return int(np.trace(A @ A @ A)) // 6


def truss_bruteforce(edges):
    """Definition 2 by exhaustive search (m <= 16).

    For every edge subset S, s(S) = min over e in S of the triangles of e
    inside S.  T_k is the union of the subsets with s(S) >= k-2 (the largest
    such subgraph: the property is closed under union).  phi(e) is the largest
    k with e in T_k."""
    m = len(edges)
    assert m <= 16, "exhaustive search is for tiny graphs"
    idx = {e: i for i, e in enumerate(edges)}
    nb = adjacency(edges)
    tri_pairs = [[] for _ in range(m)]  # for edge i: list of (j, l) masks
    for i, (u, v) in enumerate(edges):
        for w in nb[u] & nb[v]:
            j = idx[(min(u, w), max(u, w))]
            l = idx[(min(v, w), max(v, w))]
            tri_pairs[i].append((1 << j) | (1 << l))
    best = [2] * m  # T_2 = G
    for S in range(1, 1 << m):
        smin = None
        for i in range(m):
            if S >> i & 1:
                c = sum(1 for pm in tri_pairs[i] if S & pm == pm)
                smin = c if smin is None or c < smin else smin
        k = smin + 2
        for i in range(m):
            if S >> i & 1 and best[i] < k:
                best[i] = k
    return {e: best[i] for i, e in enumerate(edges)}


def truss_alg1(edges):
    """Algorithm 1 (Section 3.1), literally, on the current graph.

    k starts at 3; while some remaining edge has support < k-2 it is removed
    and its triangles' other edges lose one support each.  What remains is
    T_k; edges removed during the pass for k have truss number k-1."""
    nb = adjacency(edges)
    sup = {e: len(nb[e[0]] & nb[e[1]]) for e in edges}
    alive = set(edges)
    phi = {}
    k = 3
    while alive:
        queue = [e for e in sorted(alive) if sup[e] < k - 2]
        while queue:
            e = queue.pop()
            if e not in alive or sup[e] >= k - 2:
                continue
            u, v = e
            for w in nb[u] & nb[v]:
                for x in ((min(u, w), max(u, w)), (min(v, w), max(v, w))):
                    sup[x] -= 1
                    if sup[x] < k - 2:
                        queue.append(x)
            nb[u].discard(v)
            nb[v].discard(u)
            alive.discard(e)
            phi[e] = k - 1
        k += 1
    return phi


def core_numbers(edges):
    """Core number of every vertex: repeatedly delete a minimum-degree vertex;
    a vertex's core number is the largest minimum degree seen up to its
    deletion."""
    nb = adjacency(edges)
    deg = {v: len(s) for v, s in nb.items()}
    core = {}
    cur = 0
    live = set(nb)
    while live:
        v = min(live, key=lambda x: (deg[x], x))
        cur = max(cur, deg[v])
        core[v] = cur
        live.discard(v)
        for w in nb[v]:
            if w in live:
                deg[w] -= 1
    return core


def h_index(values):
    vals = sorted(values, reverse=True)
    h = 0
    for i, x in enumerate(vals):
        if x >= i + 1:
            h = i + 1
        else:
            break
    return h


def psi_upper(edges, sup):
    """Procedure 6 (Section 6.2) with H = G: x_w is the largest x such that w
    has x incident edges other than e with support >= x;
    psi(e) = min{sup(e), x_u, x_v} + 2."""
    nb = adjacency(edges)

    def key(a, b):
        return (a, b) if a < b else (b, a)

    psi = {}
    for e in edges:
        u, v = e
        xs = []
        for w, other in ((u, v), (v, u)):
            xs.append(h_index([sup[key(w, z)] for z in nb[w] if z != other]))
        psi[e] = min(sup[e], xs[0], xs[1]) + 2
    return psi


def invariants(edges, sup, phi):
    """Return a list of violated properties (empty = all hold).

    1. phi = 2 <=> sup = 0;  2 <= phi <= sup + 2;  phi <= psi (Lemma 2).
    2. Validity: each edge of T_k = {phi >= k} has >= k-2 triangles in T_k.
    3. Maximality: peeling T_k at threshold k-1 leaves exactly T_{k+1}.
    4. Both endpoints of every edge of T_k have core number >= k-1."""
    bad = []
    psi = psi_upper(edges, sup)
    for e in edges:
        if (phi[e] == 2) != (sup[e] == 0):
            bad.append(("phi2-sup0", e))
        if not (2 <= phi[e] <= sup[e] + 2):
            bad.append(("range", e))
        if phi[e] > psi[e]:
            bad.append(("psi", e))
    kmax = max(phi.values()) if phi else 2
    core = core_numbers(edges)
    for k in range(2, kmax + 2):
        Tk = {e for e in edges if phi[e] >= k}
        Tk1 = {e for e in edges if phi[e] >= k + 1}
        nb = adjacency(Tk)

        def s_in(e, nbx):
            return len(nbx[e[0]] & nbx[e[1]])

        for e in Tk:
            if s_in(e, nb) < k - 2:
                bad.append(("valid", k, e))
            if core[e[0]] < k - 1 or core[e[1]] < k - 1:
                bad.append(("core", k, e))
        # maximality: peel Tk at threshold k-1
        S = set(Tk)
        nbs = adjacency(S)
        changed = True
        while changed:
            changed = False
            for e in sorted(S):
                if e in S and s_in(e, nbs) < k - 1:
                    S.discard(e)
                    nbs[e[0]].discard(e[1])
                    nbs[e[1]].discard(e[0])
                    changed = True
        if S != Tk1:
            bad.append(("maximal", k))
    return bad


def _peel_at(edges, pinned, k):
    """Procedure 5 steps 1-6 on H = edges: repeatedly remove a non-pinned
    edge with support <= k-2 in what is left; returns the removed edges."""
    nb = adjacency(edges)
    key = lambda a, b: (a, b) if a < b else (b, a)  # noqa: E731
    sup = {e: len(nb[e[0]] & nb[e[1]]) for e in edges}
    alive = set(edges)
    removed = set()
    changed = True
    while changed:
        changed = False
        for e in sorted(alive):
            if e in pinned or sup[e] > k - 2:
                continue
            alive.discard(e)
            removed.add(e)
            changed = True
            u, v = e
            for w in nb[u] & nb[v]:
                a, b = key(u, w), key(v, w)
                if a in alive and b in alive:
                    sup[a] -= 1
                    sup[b] -= 1
            nb[u].discard(v)
            nb[v].discard(u)
    return removed


def bottom_up(n, edges, budget, literal_phi2=False):
    """Section 5 under an edge budget.  Algorithm 3: split the vertices into
    id ranges whose degrees in the current G sum to at most `budget` (one
    range once G fits; the budget doubles after a pass that removed
    nothing); for each range's neighbourhood subgraph H every edge keeps
    max(lower bound, truss number in H) (Lemma 1), and every internal edge
    leaves G for Phi_2 or G_new.  Step 8's test: with ``literal_phi2`` an
    internal edge goes to Phi_2 when its support in H is 0; otherwise when
    its lower bound is still 2.  Algorithm 4: for k = 3, 4, ... (jumping to
    the smallest bound left), U_k = endpoints of G_new edges with bound <= k,
    H = NS(U_k) in G_new, and the internal edges Procedure 5 removes at
    threshold k are Phi_k.  Returns {edge: phi}."""
    state = {e: 0 for e in edges}
    lower = {e: 0 for e in edges}
    phi = {}
    part_budget, last = budget, -1
    while True:
        G = [e for e in edges if state[e] == 0]
        if not G:
            break
        if len(G) == last:
            part_budget *= 2
        last = len(G)
        deg = [0] * n
        for u, v in G:
            deg[u] += 1
            deg[v] += 1
        if len(G) <= part_budget:
            parts = [(0, n)]
        else:
            parts, acc, a = [], 0, 0
            for v in range(n):
                if acc > 0 and acc + deg[v] > part_budget:
                    parts.append((a, v))
                    a, acc = v, 0
                acc += deg[v]
            parts.append((a, n))
        for a, b in parts:
            H = [e for e in G if a <= e[0] < b or a <= e[1] < b]
            if not H:
                continue
            t = truss_alg1(H)
            nbH = adjacency(H)
            for e in H:
                lower[e] = max(lower[e], t[e])
                if a <= e[0] < b and a <= e[1] < b:
                    zero = (len(nbH[e[0]] & nbH[e[1]]) == 0) if literal_phi2 else lower[e] <= 2
                    if zero:
                        phi[e] = 2
                        state[e] = 2
                    else:
                        state[e] = 1
    k = 3
    while True:
        Gn = [e for e in edges if state[e] == 1]
        if not Gn:
            break
        k = max(k, min(lower[e] for e in Gn))
        U = {x for e in Gn if lower[e] <= k for x in e}
        H = [e for e in Gn if e[0] in U or e[1] in U]
        pinned = {e for e in H if not (e[0] in U and e[1] in U)}
        for e in _peel_at(H, pinned, k):
            phi[e] = k
            state[e] = 2
        k += 1
    return phi
