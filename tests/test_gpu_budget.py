"""GPU parity of the budgeted bottom-up decomposition (Section 5: Algorithm 3,
Algorithm 4, Procedure 5; truss_decompose_budget) against the oracle,
bit-exact, with budgets small enough to force many neighbourhood
subgraphs."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0)
    yield c
    c.close()


def gpu_budget(ctx, n, src, dst, budget):
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to("cuda:0")
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to("cuda:0")
    sup, tr = torch.empty_like(s), torch.empty_like(s)
    k = ctx.decompose_budget(n, s, d, budget, sup, tr)
    torch.cuda.synchronize()
    return sup.cpu().numpy(), tr.cpu().numpy(), k, ctx.stats()


def _cases():
    from test_oracle import fig2
    cl = fig2()
    edges = sorted(cl)
    yield "fig2", (12, np.array([a for a, _ in edges], np.int32),
                   np.array([b for _, b in edges], np.int32)), (4, 8, 26)
    yield "tiny", graphgen.tiny(), (2000, 9000, 40000)
    s, d = graphgen.rmat_raw(12, 16 << 12, seed=3)
    yield "rmat12", (1 << 12, s, d), (3000, 20000)
    n = 3000
    s, d = graphgen.er(n, 12000, seed=9)
    perm = graphgen.permutation(n, seed=9, stream=1)
    s, d = graphgen.add_cliques(s, d, perm[:60], [5, 9, 13, 17])
    yield "er+cliques", (n, s, d), (1500, 6000)


CASES = [(name, case, b) for name, case, bs in _cases() for b in bs]


@pytest.mark.parametrize("name,case,budget", CASES,
                         ids=[f"{c[0]}-b{c[2]}" for c in CASES])
def test_budget_parity(ctx, name, case, budget):
    n, src, dst = case
    sup, tr, k, st = gpu_budget(ctx, n, src, dst, budget)
    ref = oracle.truss(n, src, dst)
    assert np.array_equal(sup, ref.support)
    bad = np.nonzero(tr != ref.truss)[0]
    assert len(bad) == 0, f"truss differs on {len(bad)} rows, first {bad[:5]}"
    assert k == ref.kmax
    if budget < ref.m:
        assert st["rounds"] > 1  # several neighbourhood subgraphs


def test_budget_edge_cases(ctx):
    from paper_1205_6693_gb300 import truss as T
    e = np.zeros(0, np.int32)
    out = np.zeros(0, np.int32)
    assert ctx.decompose_budget(4, e, e, 10, out, out) == 0
    src = np.array([0, 1, 2, 3, 2], np.int32)  # a path plus a self-loop row
    dst = np.array([1, 2, 3, 4, 2], np.int32)
    sup, tr, k, _ = gpu_budget(ctx, 5, src, dst, 2)
    assert list(tr) == [2, 2, 2, 2, -1] and list(sup) == [0, 0, 0, 0, -1] and k == 2
    with pytest.raises(T.TrussError):
        gpu_budget(ctx, 5, src, dst, 0)


def test_budget_with_host_buffers_and_duplicates(ctx):
    n, src, dst = graphgen.tiny()
    src = np.concatenate([src, dst[:500], np.arange(20, dtype=np.int32)])
    dst = np.concatenate([dst, src[:500], np.arange(20, dtype=np.int32)])
    sup = np.empty(len(src), np.int32)
    tr = np.empty(len(src), np.int32)
    k = ctx.decompose_budget(n, src, dst, 5000, sup, tr)
    ref = oracle.truss(n, src, dst)
    assert np.array_equal(sup, ref.support) and np.array_equal(tr, ref.truss)
    assert k == ref.kmax


@pytest.mark.parametrize("name,case,budget", CASES[::2],
                         ids=[f"{c[0]}-b{c[2]}" for c in CASES[::2]])
def test_budget_parity_own_parts_in_place(name, case, budget):
    """The neighbourhood subgraphs' lists with each edge's own part left in
    the records (truss_opts.lists_in_place)."""
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0, lists_in_place=1)
    try:
        n, src, dst = case
        sup, tr, k, st = gpu_budget(c, n, src, dst, budget)
        ref = oracle.truss(n, src, dst)
        assert np.array_equal(sup, ref.support) and np.array_equal(tr, ref.truss)
        assert k == ref.kmax
    finally:
        c.close()
