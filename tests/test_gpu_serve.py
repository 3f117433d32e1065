"""GPU tests of the request server (truss_serve_*): every result in a mix of
concurrent requests equals the oracle's result for that request alone."""
import threading

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_1205_6693_gb300 import truss as T
    return T


def _requests(count, seed=0):
    """Mixed sizes: batch-sized graphs plus a few larger R-MAT graphs."""
    out = []
    for j in range(count):
        if j % 7 == 6:
            scale = 12 + (j % 3)
            n, (s, d) = 2 ** scale, graphgen.rmat_raw(scale, 16 * 2 ** scale, seed=seed + j)
        else:
            n, s, d = graphgen.batch_graph(seed * 1000 + j)
        out.append((n, np.ascontiguousarray(s), np.ascontiguousarray(d)))
    return out


def _serve_opts(T, **kw):
    o = T.truss_serve_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_mix_equals_alone(T):
    ctx = T.truss_ctx_create(0)
    srv = T.truss_serve_start(ctx, _serve_opts(T, streams=3, batch_rows=20000, max_batch=64))
    T.truss_ctx_destroy(ctx)
    reqs = _requests(60, seed=1)
    # half the requests from host memory, half from device memory
    dev = torch.device("cuda:0")
    keep = []
    tickets = [None] * len(reqs)

    def client(idx):
        for j in idx:
            n, s, d = reqs[j]
            if j % 2:
                s, d = torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev)
                torch.cuda.synchronize()
            keep.append((s, d))
            tickets[j] = T.truss_serve_submit(srv, n, s, d)

    ths = [threading.Thread(target=client, args=(range(i, len(reqs), 2),)) for i in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    batched = 0
    for j, (n, s, d) in enumerate(reqs):
        sup = np.empty(len(s), np.int32)
        tr = np.empty(len(s), np.int32)
        st = T.truss_serve_wait(srv, tickets[j], -1, sup, tr)
        ref = oracle.truss(n, s, d)
        assert np.array_equal(sup, ref.support), j
        assert np.array_equal(tr, ref.truss), j
        assert st["kmax"] == ref.kmax and st["m"] == ref.m and st["triangles"] == ref.triangles
        batched += st["batched"] > 1
    stats = T.truss_serve_stop(srv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["launches"] < len(reqs)  # small requests shared launches
    assert batched > 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_admission_rejects_over_budget_and_serialises(T):
    ctx = T.truss_ctx_create(0)
    n, (s, d) = 4096, graphgen.rmat_raw(12, 16 * 4096, seed=3)
    fp = T.truss_serve_footprint(n, len(s))
    # budget fits exactly one such request at a time
    srv = T.truss_serve_start(ctx, _serve_opts(T, streams=2, hbm_budget_bytes=fp + fp // 2))
    T.truss_ctx_destroy(ctx)
    big_n, (bs, bd) = 2 ** 14, graphgen.rmat_raw(14, 16 * 2 ** 14, seed=4)
    with pytest.raises(T.TrussError) as ei:
        T.truss_serve_submit(srv, big_n, bs, bd)
    assert ei.value.code == T.TRUSS_EBUSY
    ref = oracle.truss(n, s, d)
    tickets = [T.truss_serve_submit(srv, n, s, d) for _ in range(5)]
    for t in tickets:
        tr = np.empty(len(s), np.int32)
        T.truss_serve_wait(srv, t, -1, None, tr)
        assert np.array_equal(tr, ref.truss)
    stats = T.truss_serve_stop(srv)
    assert stats["rejected"] == 1 and stats["completed"] == 5


def test_poll_and_stop_drains_queue(T):
    ctx = T.truss_ctx_create(0)
    srv = T.truss_serve_start(ctx, _serve_opts(T, streams=1, batch_rows=1))
    T.truss_ctx_destroy(ctx)
    reqs = _requests(8, seed=5)
    tickets = [T.truss_serve_submit(srv, n, s, d) for n, s, d in reqs]
    # an unknown ticket is an argument error
    with pytest.raises(T.TrussError):
        T.truss_serve_poll(srv, 10 ** 9)
    # wait for the first request by polling
    n, s, d = reqs[0]
    tr = np.empty(len(s), np.int32)
    for _ in range(200000):
        st = T.truss_serve_poll(srv, tickets[0], None, tr)
        if st is not None:
            break
    assert st is not None
    assert np.array_equal(tr, oracle.truss(n, s, d).truss)
    # stop with the rest queued or running: they are finished before the join
    stats = T.truss_serve_stop(srv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0


def _clique(k, n=None):
    iu, ju = np.triu_indices(k, k=1)
    return (n or k), iu.astype(np.int32), ju.astype(np.int32)


def test_dense_request_completes_or_fails_alone(T):
    """Requests far denser in triangles than the admission projection assumes
    (cliques K_300 and K_400: 4.5x and 6x their projected footprint) mixed
    into concurrent small requests under a small budget.  Each dense request
    either completes bit-exact or fails alone with TRUSS_ENOMEM; every other
    request completes and matches the oracle."""
    ctx = T.truss_ctx_create(0)
    budget = 256 << 20
    srv = T.truss_serve_start(ctx, _serve_opts(T, streams=3, hbm_budget_bytes=budget,
                                                batch_rows=20000, max_batch=32))
    T.truss_ctx_destroy(ctx)
    small = _requests(30, seed=7)
    er_n = 3000
    es, ed = graphgen.er(er_n, 12000, seed=8)
    perm = graphgen.permutation(er_n, seed=8, stream=1)
    es, ed = graphgen.add_cliques(es, ed, perm[:60], [60])
    reqs = small[:10] + [_clique(300)] + small[10:20] + [(er_n, es, ed)] + [_clique(400)] \
        + small[20:]
    dense = {10, 22}
    for j in dense:
        n, s, _ = reqs[j]
        assert T.truss_serve_footprint(n, len(s)) < budget  # admitted on its projection
    tickets = [None] * len(reqs)

    def client():
        for j, (n, s, d) in enumerate(reqs):
            tickets[j] = T.truss_serve_submit(srv, n, s, d)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    outcomes = {}
    for j, (n, s, d) in enumerate(reqs):
        sup = np.empty(len(s), np.int32)
        tr = np.empty(len(s), np.int32)
        try:
            T.truss_serve_wait(srv, tickets[j], -1, sup, tr)
        except T.TrussError as e:
            assert j in dense and e.code == T.TRUSS_ENOMEM, (j, e)
            outcomes[j] = "ENOMEM"
            continue
        ref = oracle.truss(n, s, d)
        assert np.array_equal(sup, ref.support), j
        assert np.array_equal(tr, ref.truss), j
        outcomes[j] = "ok"
    stats = T.truss_serve_stop(srv)
    failed = sum(v == "ENOMEM" for v in outcomes.values())
    assert stats["completed"] == len(reqs) - failed and stats["failed"] == failed
    assert all(outcomes[j] == "ok" for j in range(len(reqs)) if j not in dense)
    # K_300 exceeds twice its projection: its first run fails and it is run
    # again alone with the whole budget, which it fits
    assert outcomes[10] == "ok" and stats["retried"] >= 1
