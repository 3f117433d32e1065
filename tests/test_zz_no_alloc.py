"""The allocation-free support entry point (truss_support_noalloc) against the
context-based truss_support, through the C ABI.  Collected last on purpose:
it must also pass after every other test has run in the same process."""
import numpy as np
import pytest

import graphgen

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
