"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle,
element by element and bit-exact (all outputs are integers)."""
import hashlib
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


def gpu_run(ctx, n, src, dst, host=False, support_only=False):
    if host:
        s, d = np.ascontiguousarray(src, np.int32), np.ascontiguousarray(dst, np.int32)
        sup = np.empty(len(s), np.int32)
        tr = np.empty(len(s), np.int32)
    else:
        dev = torch.device("cuda:0")
        s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to(dev)
        d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to(dev)
        sup = torch.empty_like(s)
        tr = torch.empty_like(s)
    if support_only:
        ctx.support(n, s, d, sup)
        kmax = None
    else:
        kmax = ctx.decompose(n, s, d, sup, tr)
    torch.cuda.synchronize()
    if host:
        return sup, tr, kmax
    return sup.cpu().numpy(), tr.cpu().numpy(), kmax


def assert_same(ctx, n, src, dst, **kw):
    ref = oracle.truss(n, src, dst)
    sup, tr, kmax = gpu_run(ctx, n, src, dst, **kw)
    bad_s = np.nonzero(sup != ref.support)[0]
    bad_t = np.nonzero(tr != ref.truss)[0]
    assert len(bad_s) == 0, f"support differs on {len(bad_s)} rows, first {bad_s[:5]}"
    assert len(bad_t) == 0, f"truss differs on {len(bad_t)} rows, first {bad_t[:5]}"
    assert kmax == ref.kmax
    st = ctx.stats()
    assert st["m"] == ref.m and st["triangles"] == ref.triangles
    return ref


# ------------------------------------------------------------- fixtures ---
def test_fig2_example(ctx):
    from test_oracle import fig2
    classes = fig2()
    edges = sorted(classes)
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    _, tr, kmax = gpu_run(ctx, 12, src, dst)
    assert [int(t) for t in tr] == [classes[e] for e in edges]
    assert kmax == 5


@pytest.mark.parametrize("n", [3, 4, 7, 12, 33, 64])
def test_complete_graphs(ctx, n):
    a, b = np.triu_indices(n, 1)
    sup, tr, kmax = gpu_run(ctx, n, a.astype(np.int32), b.astype(np.int32))
    assert (sup == n - 2).all() and (tr == n).all() and kmax == n


# ---------------------------------------------------- seeded random graphs ---
@pytest.mark.parametrize("seed", range(8))
def test_er_with_cliques(ctx, seed):
    n = 200 + 700 * seed
    src, dst = graphgen.er(n, 6 * n, seed=seed)
    perm = graphgen.permutation(n, seed=seed, stream=1)
    sizes = [5 + seed, 9 + 2 * seed, 30]
    src, dst = graphgen.add_cliques(src, dst, perm[: sum(sizes)], sizes)
    assert_same(ctx, n, src, dst)


@pytest.mark.parametrize("scale,ef", [(8, 8), (10, 16), (12, 16), (14, 8), (15, 16)])
def test_rmat_raw_rows(ctx, scale, ef):
    # raw R-MAT rows keep duplicates, reversed pairs and self-loops
    n, (src, dst) = 2 ** scale, graphgen.rmat_raw(scale, ef * 2 ** scale, seed=scale)
    assert_same(ctx, n, src, dst)


@pytest.mark.parametrize("seed", range(3))
def test_chung_lu_small(ctx, seed):
    n = 20000
    src, dst = graphgen.chung_lu(n, 200000, 20.0, 2000.0, 2.1, seed=seed)
    assert_same(ctx, n, src, dst)


def test_tiny_config(ctx):
    n, src, dst = graphgen.tiny()
    ref = assert_same(ctx, n, src, dst)
    assert ref.kmax == 32


def test_host_pointers_match_device(ctx):
    n, src, dst = graphgen.tiny()
    ref = oracle.truss(n, src, dst)
    sup, tr, kmax = gpu_run(ctx, n, src, dst, host=True)
    assert np.array_equal(sup, ref.support) and np.array_equal(tr, ref.truss)
    assert kmax == ref.kmax


def test_pinned_host_buffers_match_oracle(ctx):
    # pinned (page-locked) rows and outputs are read and written in place by
    # the kernels; pageable ones go through staged copies; mixing the kinds
    # in one call must not matter
    n, (src, dst) = 2 ** 13, graphgen.rmat_raw(13, 16 * 2 ** 13, seed=7)
    ref = oracle.truss(n, src, dst)
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).pin_memory()
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).pin_memory()
    sup = torch.full_like(s, -7).pin_memory()
    tr = torch.full_like(s, -7).pin_memory()
    kmax = ctx.decompose(n, s, d, sup, tr)
    assert np.array_equal(sup.numpy(), ref.support) and np.array_equal(tr.numpy(), ref.truss)
    assert kmax == ref.kmax
    dev = torch.device("cuda:0")
    sup2 = np.full(len(src), -7, np.int32)  # pageable output
    tr2 = torch.full((len(src),), -7, dtype=torch.int32, device=dev)  # device output
    ctx.decompose(n, s, np.ascontiguousarray(dst, np.int32), sup2, tr2)
    assert np.array_equal(sup2, ref.support)
    assert np.array_equal(tr2.cpu().numpy(), ref.truss)
    sup3 = torch.full_like(s, -7).pin_memory()
    ctx.support(n, s, d, sup3)
    assert np.array_equal(sup3.numpy(), ref.support)


def test_support_only(ctx):
    n, (src, dst) = 4096, graphgen.rmat_raw(12, 16 * 4096, seed=5)
    ref = oracle.truss(n, src, dst, with_truss=False)
    sup, _, _ = gpu_run(ctx, n, src, dst, support_only=True)
    assert np.array_equal(sup, ref.support)


def test_deterministic(ctx):
    n, (src, dst) = 2 ** 13, graphgen.rmat_raw(13, 16 * 2 ** 13, seed=3)
    a = gpu_run(ctx, n, src, dst)
    b = gpu_run(ctx, n, src, dst)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ------------------------------------------------------------ edge cases ---
def test_empty_graph(ctx):
    e = np.zeros(0, np.int32)
    sup, tr, kmax = gpu_run(ctx, 10, e, e)
    assert len(sup) == 0 and kmax == 0


def test_only_self_loops(ctx):
    x = np.arange(5, dtype=np.int32)
    sup, tr, kmax = gpu_run(ctx, 5, x, x)
    assert (sup == -1).all() and (tr == -1).all() and kmax == 0


def test_single_edge_and_duplicates(ctx):
    src = np.array([0, 1, 0, 2, 2], np.int32)
    dst = np.array([1, 0, 1, 2, 0], np.int32)
    assert_same(ctx, 3, src, dst)


def test_isolated_vertices_and_large_n(ctx):
    n = 5_000_000
    src = np.array([4_999_999, 17, 17, 123456], np.int32)
    dst = np.array([17, 123456, 4_999_999, 4_999_999], np.int32)
    ref = assert_same(ctx, n, src, dst)
    assert ref.kmax == 3  # the three distinct edges form one triangle


def test_invalid_ids_rejected(ctx):
    from paper_1205_6693_gb300.truss import TRUSS_EINVAL, TrussError
    for bad in ([0, 5], [-1, 2]):
        src = np.array([0, bad[0]], np.int32)
        dst = np.array([1, bad[1]], np.int32)
        with pytest.raises(TrussError) as ei:
            gpu_run(ctx, 5, src, dst)
        assert ei.value.code == TRUSS_EINVAL
    # the context stays usable
    assert_same(ctx, 3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32))


# ------------------------------------------------------------------ batch ---
def test_batch_matches_oracle_per_graph(ctx):
    G = 300
    ns, off, src, dst = graphgen.batch(G)
    dev = torch.device("cuda:0")
    s = torch.from_numpy(src).to(dev)
    d = torch.from_numpy(dst).to(dev)
    sup = torch.empty_like(s)
    tr = torch.empty_like(s)
    kmax = torch.empty(G, dtype=torch.int32, device=dev)
    ctx.decompose_batch(ns, off, s, d, sup, tr, kmax)
    torch.cuda.synchronize()
    sup, tr, kmax = sup.cpu().numpy(), tr.cpu().numpy(), kmax.cpu().numpy()
    for g in range(G):
        a, b = off[g], off[g + 1]
        ref = oracle.truss(int(ns[g]), src[a:b], dst[a:b])
        assert np.array_equal(sup[a:b], ref.support), g
        assert np.array_equal(tr[a:b], ref.truss), g
        assert kmax[g] == ref.kmax, g


# ------------------------------------------------------------- full size ---
def _digest(name):
    with open(os.path.join(GOLDEN, "digests.json")) as f:
        return json.load(f)[name]


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def _check_full(ctx, name, gen):
    exp = _digest(name)
    n, src, dst = gen()
    sup, tr, kmax = gpu_run(ctx, n, src, dst)
    idx = np.array(exp["sample_rows"], np.int64)
    assert np.array_equal(sup[idx], np.array(exp["sample_support"], np.int32))
    assert np.array_equal(tr[idx], np.array(exp["sample_truss"], np.int32))
    st = ctx.stats()
    assert st["m"] == exp["m"] and st["triangles"] == exp["triangles"]
    assert kmax == exp["kmax"]
    assert _sha(sup) == exp["sha256_support"]
    assert _sha(tr) == exp["sha256_truss"]


def test_mid_full_size(ctx):
    _check_full(ctx, "mid", graphgen.mid)


def test_large_full_size(ctx):
    # 167.8M distinct edges, 3.5G triangles.  The oracle checks sampled rows
    # one by one (exact support by neighbour-list intersection and local
    # validity of the truss number); the stored oracle digest, when present,
    # fixes every output.
    n, src, dst = graphgen.large()
    sup, tr, kmax = gpu_run(ctx, n, src, dst)
    st = ctx.stats()
    assert st["m"] == len(src)  # distinct rows, no self-loops
    assert int(sup.astype(np.int64).sum()) == 3 * st["triangles"]
    assert kmax == int(tr.max())
    rows = len(src)
    sample = np.unique(np.array([graphgen.draw(77, 5, i) % rows for i in range(4096)], np.int64))
    bad, exact = oracle.check_sample(n, src, dst, tr, sup, sample)
    assert np.array_equal(exact, sup[sample])
    assert bad == 0
    with open(os.path.join(GOLDEN, "digests.json")) as f:
        dig = json.load(f)
    if "large" in dig:
        exp = dig["large"]
        assert st["triangles"] == exp["triangles"] and kmax == exp["kmax"]
        assert _sha(sup) == exp["sha256_support"]
        assert _sha(tr) == exp["sha256_truss"]


def test_gpu_generator_matches_cpu_generator():
    s_cpu, d_cpu = graphgen.rmat_raw(16, 1 << 20, seed=11, stream=2)
    s_gpu, d_gpu = graphgen.rmat_raw_cuda(16, 1 << 20, seed=11, stream=2)
    torch.cuda.synchronize()
    assert np.array_equal(s_gpu.cpu().numpy(), s_cpu)
    assert np.array_equal(d_gpu.cpu().numpy(), d_cpu)


def test_bounded_wait_reports_timeout_and_context_survives():
    # A 1 ns limit on the peel kernel's grid barrier makes waiting blocks give
    # up at once: the kernel must return TRUSS_ETIMEOUT, not hang, and both
    # this context and a fresh one must still work afterwards.
    from paper_1205_6693_gb300 import truss as T
    n, (src, dst) = 2 ** 12, graphgen.rmat_raw(12, 16 * 2 ** 12, seed=9)
    c = T.Context(0, wait_limit_ns=1)
    try:
        with pytest.raises(T.TrussError) as ei:
            gpu_run(c, n, src, dst)
        assert ei.value.code == T.TRUSS_ETIMEOUT
        # support does not use the grid barrier and still works on this context
        ref = oracle.truss(n, src, dst)
        sup, _, _ = gpu_run(c, n, src, dst, support_only=True)
        assert np.array_equal(sup, ref.support)
    finally:
        c.close()
    c2 = T.Context(0)
    try:
        assert_same(c2, n, src, dst)
    finally:
        c2.close()


def test_lists_by_second_walk():
    """The list builder taken when the triangle records do not fit (a second,
    owner-centric walk), forced through truss_opts.lists_by_walk."""
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0, lists_by_walk=1)
    try:
        for n, src, dst in (graphgen.tiny(),
                            (1 << 13, *graphgen.rmat_raw(13, 16 << 13, seed=4))):
            assert_same(c, n, src, dst)
    finally:
        c.close()


def _in_place_cases():
    yield "tiny", graphgen.tiny()
    for sc, seed in ((12, 3), (15, 8)):
        s, d = graphgen.rmat_raw(sc, 16 << sc, seed=seed)
        yield f"rmat{sc}", (1 << sc, s, d)
    n = 4000
    s, d = graphgen.er(n, 16000, seed=23)
    perm = graphgen.permutation(n, seed=23, stream=1)
    s, d = graphgen.add_cliques(s, d, perm[:120], [4, 17, 18, 33, 47])
    yield "er+cliques", (n, s, d)


IN_PLACE_CASES = list(_in_place_cases())


@pytest.mark.parametrize("variant", [0, 1, 3])
@pytest.mark.parametrize("name,case", IN_PLACE_CASES, ids=[c[0] for c in IN_PLACE_CASES])
def test_lists_own_parts_in_place(name, case, variant):
    """Lists that leave each edge's own triangles in the support walk's
    records (truss_opts.lists_in_place): the peel reads every list in two
    stretches, and a work item may span both.  Clique sizes 17, 18, 33 and 47
    give supports on both sides of the 16-entry item size."""
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0, lists_in_place=1, peel_variant=variant)
    try:
        n, src, dst = case
        assert_same(c, n, src, dst)
        assert c.stats()["lists_layout"] == 3
    finally:
        c.close()


def test_lists_layout_reported():
    """truss_last_stats names the list layout each call used."""
    from paper_1205_6693_gb300 import truss as T
    n, src, dst = graphgen.tiny()
    for kw, want in (({}, 2), ({"lists_by_walk": 1}, 1), ({"lists_in_place": 1}, 3),
                     ({"lists_in_place": 1, "peel_variant": 4}, 2)):
        c = T.Context(0, **kw)
        try:
            assert_same(c, n, src, dst)
            assert c.stats()["lists_layout"] == want, kw
            s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to("cuda:0")
            d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to("cuda:0")
            c.support(n, s, d, torch.empty_like(s))
            assert c.stats()["lists_layout"] == 0
        finally:
            c.close()


def test_peel_tag_rewrite(monkeypatch):
    """The peel's 16-bit edge tags repeat every 65,534 sub-rounds, so the
    kernel rewrites stale ones periodically; forced every 1 and every 3
    sub-rounds (TRUSS_PEEL_RETAG), the results stay bit-exact."""
    from paper_1205_6693_gb300 import truss as T
    cases = [graphgen.tiny(), (1 << 13, *graphgen.rmat_raw(13, 16 << 13, seed=4)),
             IN_PLACE_CASES[-1][1]]
    for period in ("1", "3"):
        monkeypatch.setenv("TRUSS_PEEL_RETAG", period)
        c = T.Context(0)
        try:
            for n, src, dst in cases:
                assert_same(c, n, src, dst)
        finally:
            c.close()


@pytest.fixture(scope="module")
def ctx_async():
    from paper_1205_6693_gb300 import truss as T
    c = T.Context(0, peel_variant=4)
    yield c
    c.close()


def _async_cases():
    yield "tiny", graphgen.tiny()
    for sc, seed in ((10, 2), (13, 4), (15, 6)):
        s, d = graphgen.rmat_raw(sc, 16 << sc, seed=seed)
        yield f"rmat{sc}", (1 << sc, s, d)
    n = 4000
    s, d = graphgen.er(n, 16000, seed=21)
    perm = graphgen.permutation(n, seed=21, stream=1)
    s, d = graphgen.add_cliques(s, d, perm[:100], [6, 11, 17, 23, 40])
    yield "er+cliques", (n, s, d)


ASYNC_CASES = list(_async_cases())


@pytest.mark.parametrize("name,case", ASYNC_CASES, ids=[c[0] for c in ASYNC_CASES])
def test_barrier_free_peel(ctx_async, name, case):
    """Peel variant 4 (triangle destroyed-bits, work queue per level) against
    the oracle, bit-exact."""
    n, src, dst = case
    assert_same(ctx_async, n, src, dst)


def test_barrier_free_peel_fig2_and_cliques(ctx_async):
    from test_oracle import fig2
    classes = fig2()
    edges = sorted(classes)
    src = np.array([a for a, _ in edges], np.int32)
    dst = np.array([b for _, b in edges], np.int32)
    _, tr, kmax = gpu_run(ctx_async, 12, src, dst)
    assert [int(t) for t in tr] == [classes[e] for e in edges] and kmax == 5
    for n in (3, 9, 40):
        a, b = np.triu_indices(n, 1)
        _, tr, kmax = gpu_run(ctx_async, n, a.astype(np.int32), b.astype(np.int32))
        assert (tr == n).all() and kmax == n


def test_barrier_free_peel_mid_full_size(ctx_async):
    _check_full(ctx_async, "mid", graphgen.mid)


def test_barrier_free_peel_bounded_wait():
    from paper_1205_6693_gb300 import truss as T
    n, (src, dst) = 2 ** 12, graphgen.rmat_raw(12, 16 * 2 ** 12, seed=9)
    c = T.Context(0, wait_limit_ns=1, peel_variant=4)
    try:
        with pytest.raises(T.TrussError) as ei:
            gpu_run(c, n, src, dst)
        assert ei.value.code == T.TRUSS_ETIMEOUT
    finally:
        c.close()
    c2 = T.Context(0, peel_variant=4)
    try:
        assert_same(c2, n, src, dst)
    finally:
        c2.close()


def test_workspace_settles_after_calls_of_another_order():
    """The context's workspace is one chunk of the peak size once a call has
    needed several, so calls of the same shape reuse it without allocating,
    also after a host-buffer call (which stages its inputs first)."""
    from paper_1205_6693_gb300 import truss as T
    n, src, dst = 1 << 14, *graphgen.rmat_raw(14, 16 << 14, seed=9)
    dev = torch.device("cuda:0")
    s, d = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    sup, tr = torch.empty_like(s), torch.empty_like(s)
    c = T.Context(0)
    try:
        seen = []
        for host in (False, False, False, True, True, True, False, False):
            if host:
                hs, ht = np.empty(len(src), np.int32), np.empty(len(src), np.int32)
                c.decompose(n, src, dst, hs, ht)
            else:
                c.decompose(n, s, d, sup, tr)
            st = c.stats()
            assert 0 < st["workspace_peak"] <= st["workspace_bytes"]
            seen.append(st["workspace_bytes"])
        # steady within each run of same-shaped calls: no growth after the first two
        assert seen[1] == seen[2] and seen[4] == seen[5] and seen[6] == seen[7], seen
        ref = oracle.truss(n, src, dst)
        assert np.array_equal(tr.cpu().numpy(), ref.truss)
    finally:
        c.close()
