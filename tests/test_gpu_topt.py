"""GPU parity of the upper bound psi (Procedure 6) and the top-t classes
(Algorithm 7) against the oracle, bit-exact, through the C ABI."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).to("cuda:0")


def gpu_psi(ctx, n, src, dst):
    s, d = _dev(src), _dev(dst)
    sup, ps = torch.empty_like(s), torch.empty_like(s)
    ctx.upper_bound(n, s, d, sup, ps)
    torch.cuda.synchronize()
    return sup.cpu().numpy(), ps.cpu().numpy()


def gpu_top(ctx, n, src, dst, t):
    s, d = _dev(src), _dev(dst)
    out = torch.empty_like(s)
    kmax = ctx.top(n, s, d, t, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), kmax


def fig2_rows():
    from test_oracle import fig2
    classes = fig2()
    edges = sorted(classes)
    return (edges, np.array([a for a, _ in edges], np.int32),
            np.array([b for _, b in edges], np.int32), classes)


def test_fig2_psi_example4(ctx):
    edges, src, dst, classes = fig2_rows()
    sup, ps = gpu_psi(ctx, 12, src, dst)
    osup, ops = oracle.psi(12, src, dst)
    assert np.array_equal(sup, osup) and np.array_equal(ps, ops)
    i = edges.index((3, 6))  # (d, g)
    assert ps[i] == 4
    assert all(p == 5 for e, p in zip(edges, ps) if classes[e] == 5)


def test_fig2_top2_example5(ctx):
    edges, src, dst, classes = fig2_rows()
    top, kmax = gpu_top(ctx, 12, src, dst, 2)
    want, wk = oracle.top(12, src, dst, 2)
    assert np.array_equal(top, want) and kmax == wk == 5
    clique = [(5, 7), (5, 8), (5, 9), (7, 8), (7, 9), (8, 9)]  # f, h, i, j
    assert sorted(e for e, v in zip(edges, top) if v == 4) == clique


def _cases():
    yield "tiny", graphgen.tiny()
    for sc, seed in ((12, 3), (14, 5)):
        s, d = graphgen.rmat_raw(sc, 16 << sc, seed=seed)
        yield f"rmat{sc}", (1 << sc, s, d)
    n = 3000
    s, d = graphgen.er(n, 12000, seed=9)
    perm = graphgen.permutation(n, seed=9, stream=1)
    s, d = graphgen.add_cliques(s, d, perm[:60], [5, 9, 13, 17])
    yield "er+cliques", (n, s, d)


CASES = list(_cases())
_ORACLE = {}


def oracle_top(name, n, src, dst, t):
    """oracle.top, with the full decomposition computed once per case."""
    if name not in _ORACLE:
        _ORACLE[name] = oracle.truss(n, src, dst)
    r = _ORACLE[name]
    thr = max(r.kmax - t + 1, 2)
    out = np.where(r.truss >= thr, r.truss, 0).astype(np.int32)
    out[r.truss < 0] = -1
    return out, r.kmax


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_psi_parity(ctx, name, case):
    n, src, dst = case
    sup, ps = gpu_psi(ctx, n, src, dst)
    osup, ops = oracle.psi(n, src, dst)
    assert np.array_equal(sup, osup)
    bad = np.nonzero(ps != ops)[0]
    assert len(bad) == 0, f"psi differs on {len(bad)} rows, first {bad[:5]}"
    r = oracle.truss(n, src, dst)
    assert (r.truss <= ps).all()  # Lemma 2


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("t", [1, 3, 10, 100000])
def test_top_parity(ctx, name, case, t):
    n, src, dst = case
    top, kmax = gpu_top(ctx, n, src, dst, t)
    want, wk = oracle_top(name, n, src, dst, t)
    assert kmax == wk
    bad = np.nonzero(top != want)[0]
    assert len(bad) == 0, f"top-{t} differs on {len(bad)} rows, first {bad[:5]}"
    st = ctx.stats()
    assert st["rounds"] >= 1 and 0 < st["candidates"] <= st["m"]


def test_top_edge_cases(ctx):
    from paper_1205_6693_gb300 import truss as T
    # no rows
    e = np.zeros(0, np.int32)
    out = np.zeros(0, np.int32)
    assert ctx.top(5, e, e, 3, out) == 0
    # triangle-free graph (a path) with a self-loop row: every edge is in Phi_2
    src = np.array([0, 1, 2, 3, 3], np.int32)
    dst = np.array([1, 2, 3, 4, 3], np.int32)
    top, kmax = gpu_top(ctx, 5, src, dst, 1)
    assert kmax == 2 and list(top) == [2, 2, 2, 2, -1]
    # a single clique: top-1 is every edge
    a, b = np.triu_indices(9, 1)
    top, kmax = gpu_top(ctx, 9, a, b, 1)
    assert kmax == 9 and (top == 9).all()
    with pytest.raises(T.TrussError):
        gpu_top(ctx, 9, a, b, 0)


def test_top_mid_against_stored_oracle(ctx):
    """Full-size mid graph: the stored oracle digest gives the class sizes
    and sampled rows' truss numbers."""
    dg = json.load(open(os.path.join(GOLDEN, "digests.json")))["mid"]
    n, src, dst = graphgen.mid()
    t = 10
    top, kmax = gpu_top(ctx, n, src, dst, t)
    assert kmax == dg["kmax"]
    thr = kmax - t + 1
    rows = np.array(dg["sample_rows"], np.int64)
    want = np.array(dg["sample_truss"], np.int32)
    want = np.where(want >= thr, want, np.where(want < 0, -1, 0))
    assert np.array_equal(top[rows], want)
    eu, ev, r2e = oracle.edges(n, src, dst)
    per_edge = np.zeros(len(eu), np.int32)
    ok = r2e >= 0
    per_edge[r2e[ok]] = top[ok]
    got = {int(k): int(c) for k, c in zip(*np.unique(per_edge[per_edge > 0],
                                                     return_counts=True))}
    want_cls = {int(k): int(c) for k, c in dg["classes"].items() if int(k) >= thr}
    assert got == want_cls
    st = ctx.stats()
    assert st["candidates"] < st["m"] // 4  # the candidate subgraph is a small part


def test_upper_bound_and_top_with_host_buffers(ctx):
    """Host (numpy) inputs and outputs go through the same entry points."""
    n, src, dst = graphgen.tiny()
    sup = np.empty(len(src), np.int32)
    ps = np.empty(len(src), np.int32)
    ctx.upper_bound(n, src, dst, sup, ps)
    osup, ops = oracle.psi(n, src, dst)
    assert np.array_equal(sup, osup) and np.array_equal(ps, ops)
    out = np.empty(len(src), np.int32)
    k = ctx.top(n, src, dst, 4, out)
    want, wk = oracle.top(n, src, dst, 4)
    assert k == wk and np.array_equal(out, want)


def test_top_rejects_bad_ids(ctx):
    from paper_1205_6693_gb300 import truss as T
    src = np.array([0, 1, 7], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    out = np.empty(3, np.int32)
    with pytest.raises(T.TrussError) as ei:
        ctx.top(5, src, dst, 1, out)
    assert ei.value.code == T.TRUSS_EINVAL
