"""Autotuner on the GPU: every candidate schedule gives bit-identical outputs
(the search itself raises otherwise), the tuned schedule matches the oracle,
and the winner lands in the JSON cache under this GPU's key."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _device_inputs(src, dst):
    dev = torch.device("cuda:0")
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to(dev)
    return s, d, torch.empty_like(s), torch.empty_like(s)


def test_tuned_single_graph_schedule_is_exact(tmp_path, monkeypatch):
    from paper_1205_6693_gb300 import autotune as A
    from paper_1205_6693_gb300 import truss as T
    monkeypatch.setenv("TRUSS_TUNE_CACHE", str(tmp_path / "s.json"))
    src, dst = graphgen.rmat_raw(14, 16 << 14, seed=5)
    n = 1 << 14
    s, d, sup, tr = _device_inputs(src, dst)
    space = {"support_range_work": (0, 1024, 65536), "support_stage_max": (0, 32),
             "support_pair_cost": (0, 64), "peel_variant": (0, 1, 3)}
    ent = A.tune_call(0, lambda c: (c.decompose(n, s, d, sup, tr), (sup, tr))[1],
                      len(src), space=space, reps=1)
    key = A.gpu_key(0)
    assert A.lookup(key, len(src), nearest=False) == ent["opts"]
    ctx = T.Context(0, **ent["opts"])
    kmax = ctx.decompose(n, s, d, sup, tr)
    torch.cuda.synchronize()
    ctx.close()
    ref = oracle.truss(n, src, dst)
    assert np.array_equal(sup.cpu().numpy(), ref.support)
    assert np.array_equal(tr.cpu().numpy(), ref.truss)
    assert kmax == ref.kmax


@pytest.mark.parametrize("opts", [
    {"support_stage_max": 1},            # nothing staged: every out-list from global memory
    {"support_range_work": 1},           # one oriented edge per range
    {"support_pair_cost": 100000},       # cost dominated by the edge count
    {"peel_variant": 1}, {"peel_variant": 3},
])
def test_extreme_schedules_are_exact(opts):
    from paper_1205_6693_gb300 import truss as T
    n, src, dst = graphgen.tiny()
    s, d, sup, tr = _device_inputs(src, dst)
    ctx = T.Context(0, **opts)
    kmax = ctx.decompose(n, s, d, sup, tr)
    torch.cuda.synchronize()
    ctx.close()
    ref = oracle.truss(n, src, dst)
    assert np.array_equal(sup.cpu().numpy(), ref.support)
    assert np.array_equal(tr.cpu().numpy(), ref.truss)
    assert kmax == ref.kmax


def test_tuned_batch_schedule_is_exact(tmp_path, monkeypatch):
    from paper_1205_6693_gb300 import autotune as A
    monkeypatch.setenv("TRUSS_TUNE_CACHE", str(tmp_path / "s.json"))
    ns, off, src, dst = graphgen.batch(64)
    G = len(ns)
    s, d, sup, tr = _device_inputs(src, dst)
    kmax = torch.empty(G, dtype=torch.int32, device="cuda:0")
    space = {"support_range_work": (0, 4096), "peel_variant": (0, 1)}
    ent = A.tune_call(0, lambda c: (c.decompose_batch(ns, off, s, d, sup, tr, kmax),
                                    (sup, tr, kmax))[1],
                      int(off[-1]), G, space=space, reps=1)
    assert A.lookup(A.gpu_key(0), int(off[-1]), G, nearest=False) == ent["opts"]
    sup_h, tr_h = sup.cpu().numpy(), tr.cpu().numpy()
    for g in range(0, G, 7):
        a, b = int(off[g]), int(off[g + 1])
        ref = oracle.truss(int(ns[g]), src[a:b], dst[a:b])
        assert np.array_equal(sup_h[a:b], ref.support)
        assert np.array_equal(tr_h[a:b], ref.truss)
