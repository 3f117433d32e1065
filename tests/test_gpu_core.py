"""GPU parity of the vertex core numbers (truss_core) against the oracle's
bin-sorted degree array, bit-exact, through the C ABI."""
import itertools

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


def gpu_core(ctx, n, src, dst):
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to("cuda:0")
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to("cuda:0")
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda:0")
    k = ctx.core(n, s, d, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:n], k


def rows_of(edges):
    return (np.array([a for a, _ in edges], np.int32), np.array([b for _, b in edges], np.int32))


def test_closed_forms(ctx):
    cases = [
        (7, list(itertools.combinations(range(7), 2)), [6] * 7),
        (6, [(i, (i + 1) % 6) for i in range(6)], [2] * 6),
        (5, [(i, i + 1) for i in range(4)], [1] * 5),
        (6, [(0, i) for i in range(1, 6)], [1] * 6),
        (4, [(0, 1)], [1, 1, 0, 0]),
        (8, [(a, b) for a in range(3) for b in range(3, 8)], [3] * 8),
    ]
    for n, edges, want in cases:
        core, k = gpu_core(ctx, n, *rows_of(edges))
        assert list(core) == want and k == max(want)


def _cases():
    yield "tiny", graphgen.tiny()
    for sc, seed in ((12, 3), (16, 7)):
        s, d = graphgen.rmat_raw(sc, 16 << sc, seed=seed)
        yield f"rmat{sc}", (1 << sc, s, d)
    n = 5000
    s, d = graphgen.er(n, 20000, seed=11)
    perm = graphgen.permutation(n, seed=11, stream=1)
    s, d = graphgen.add_cliques(s, d, perm[:80], [10, 30, 40])
    yield "er+cliques", (n, s, d)
    yield "mid", graphgen.mid()


CASES = list(_cases())


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_core_parity(ctx, name, case):
    n, src, dst = case
    core, k = gpu_core(ctx, n, src, dst)
    want, wk = oracle.core(n, src, dst)
    bad = np.nonzero(core != want)[0]
    assert len(bad) == 0, f"core differs on {len(bad)} vertices, first {bad[:5]}"
    assert k == wk


def test_core_with_self_loops_duplicates_and_host_buffers(ctx):
    n, src, dst = graphgen.tiny()
    src = np.concatenate([src, dst[:100], np.arange(50, dtype=np.int32)])
    dst = np.concatenate([dst, src[:100], np.arange(50, dtype=np.int32)])
    out = np.empty(n, np.int32)
    k = ctx.core(n, src, dst, out)
    want, wk = oracle.core(n, src, dst)
    assert np.array_equal(out, want) and k == wk


def test_truss_inside_core_on_gpu(ctx):
    """phi(e) <= min(core(u), core(v)) + 1: a k-truss lies in the (k-1)-core."""
    s, d = graphgen.rmat_raw(14, 16 << 14, seed=2)
    n = 1 << 14
    core, _ = gpu_core(ctx, n, s, d)
    st, dt = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    sup, tr = torch.empty_like(st), torch.empty_like(st)
    ctx.decompose(n, st, dt, sup, tr)
    tr = tr.cpu().numpy()
    ok = tr > 0
    assert (tr[ok] <= np.minimum(core[s[ok]], core[d[ok]]) + 1).all()


def test_core_empty_and_invalid(ctx):
    from paper_1205_6693_gb300 import truss as T
    e = np.zeros(0, np.int32)
    out = np.full(6, -7, np.int32)
    assert ctx.core(6, e, e, out) == 0
    assert (out == 0).all()  # every vertex without edges has core number 0
    with pytest.raises(T.TrussError) as ei:
        ctx.core(3, np.array([0, 5], np.int32), np.array([1, 2], np.int32),
                 np.empty(3, np.int32))
    assert ei.value.code == T.TRUSS_EINVAL
