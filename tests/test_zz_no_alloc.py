"""The allocation-free support entry point (truss_support_noalloc) against the
context-based truss_support and against the CPU oracle, through the C ABI.
Collected last on purpose: it must also pass after every other test has run
in the same process."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _graph(seed):
    # ER plus two planted cliques, with a few duplicated, reversed and
    # self-loop rows appended
    n = 3000 + 500 * seed
    src, dst = graphgen.er(n, 8 * n, seed=seed, stream=4)
    perm = graphgen.permutation(n, seed=seed, stream=5)
    src, dst = graphgen.add_cliques(src, dst, perm[:40], [15, 25])
    extra = np.arange(50, dtype=np.int32)
    src = np.concatenate([src, dst[:200], extra])
    dst = np.concatenate([dst, src[:200], extra])
    return n, src, dst


def test_noalloc_matches_truss_support_on_two_calls_in_a_row():
    from paper_1205_6693_gb300 import truss as T
    dev = torch.device("cuda:0")
    ctx = T.Context(0)
    try:
        for seed in (1, 2):
            n, src, dst = _graph(seed)
            assert len(src) <= 65536
            s = torch.from_numpy(src).to(dev)
            d = torch.from_numpy(dst).to(dev)
            ref = torch.empty_like(s)
            ctx.support(n, s, d, ref)
            out = torch.full_like(s, -7)
            T.truss_support_noalloc(n, s, d, out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), f"graph {seed}: {int((out != ref).sum())} rows differ"
    finally:
        ctx.close()


def test_noalloc_rejects_oversize_and_bad_ids():
    from paper_1205_6693_gb300 import truss as T
    dev = torch.device("cuda:0")
    big = torch.zeros(65537, dtype=torch.int32, device=dev)
    with pytest.raises(T.TrussError) as ei:
        T.truss_support_noalloc(10, big, big, big)
    assert ei.value.code == T.TRUSS_EINVAL
    s = torch.tensor([0, 1, 9], dtype=torch.int32, device=dev)
    d = torch.tensor([1, 2, 2], dtype=torch.int32, device=dev)
    out = torch.empty_like(s)
    with pytest.raises(T.TrussError) as ei:
        T.truss_support_noalloc(5, s, d, out)  # id 9 >= n
    assert ei.value.code == T.TRUSS_EINVAL


MAX_ROWS = 65536
MAX_N = 65536


def _at_limits():
    """n = 65,536 and exactly 65,536 rows: a clique K_362 (65,341 edges, the
    hash table at its design load) on vertices spread over [0, n) including
    0 and n - 1, then reversed duplicates and self-loops up to the row
    limit."""
    n = MAX_N
    perm = graphgen.permutation(n, seed=11, stream=2)
    verts = np.concatenate([[0, n - 1], perm[~np.isin(perm, [0, n - 1])][:360]]).astype(np.int32)
    iu, ju = np.triu_indices(len(verts), k=1)
    src, dst = verts[iu], verts[ju]
    assert len(src) == 65341
    extra = MAX_ROWS - len(src)
    loops = np.arange(extra // 2, dtype=np.int32) * 300
    k = extra - len(loops)
    src, dst = (np.concatenate([src, dst[:k], loops]).astype(np.int32),
                np.concatenate([dst, src[:k], loops]).astype(np.int32))
    assert len(src) == MAX_ROWS
    return n, src, dst


def _hub_heavy():
    """One hub joined to 20,000 vertices, ER edges among those, 65,536 rows."""
    n = MAX_N
    leaves = graphgen.permutation(n - 1, seed=12, stream=2)[:20000].astype(np.int32) + 1
    s1 = np.zeros(len(leaves), np.int32)
    es, ed = graphgen.er(20000, MAX_ROWS - len(leaves), seed=12, stream=3)
    src = np.concatenate([s1, leaves[es]]).astype(np.int32)
    dst = np.concatenate([leaves, leaves[ed]]).astype(np.int32)
    assert len(src) == MAX_ROWS
    return n, src, dst


@pytest.mark.parametrize("case", [_at_limits, _hub_heavy])
def test_noalloc_matches_the_oracle_at_the_size_limits(case):
    from paper_1205_6693_gb300 import truss as T
    n, src, dst = case()
    ref = oracle.truss(n, src, dst, with_truss=False).support
    dev = torch.device("cuda:0")
    s = torch.from_numpy(src).to(dev)
    d = torch.from_numpy(dst).to(dev)
    for _ in range(2):
        out = torch.full_like(s, -7)
        T.truss_support_noalloc(n, s, d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), f"{int((got != ref).sum())} rows differ from the oracle"


def test_noalloc_rejects_sizes_one_past_the_limits():
    from paper_1205_6693_gb300 import truss as T
    dev = torch.device("cuda:0")
    s = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    d = torch.tensor([1, 2], dtype=torch.int32, device=dev)
    out = torch.empty_like(s)
    with pytest.raises(T.TrussError) as ei:
        T.truss_support_noalloc(MAX_N + 1, s, d, out)
    assert ei.value.code == T.TRUSS_EINVAL
    big = torch.zeros(MAX_ROWS + 1, dtype=torch.int32, device=dev)
    with pytest.raises(T.TrussError) as ei:
        T.truss_support_noalloc(10, big, big, big)
    assert ei.value.code == T.TRUSS_EINVAL


def test_noalloc_refuses_pageable_host_buffers_before_any_launch():
    from paper_1205_6693_gb300 import truss as T
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    out = np.full(3, -7, np.int32)
    with pytest.raises(T.TrussError) as ei:
        T.truss_support_noalloc(3, src, dst, out)
    assert ei.value.code == T.TRUSS_EINVAL
    assert (out == -7).all()
