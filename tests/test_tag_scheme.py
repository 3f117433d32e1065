"""Model check of the peel's 16-bit edge tags (CPU, no GPU).

The peel kernel keeps one 16-bit tag per edge instead of the sub-round
number at which the edge joined a frontier: 0 = alive, tag(s) = 1 + (s-1)
mod 65534 = in the frontier of sub-round s, any other value = removed, and at
least every P <= 32768 sub-rounds a pass rewrites every tag except the
current frontier's to a dead value.  This test replays many random push times
over more than two wraps of the tag space and checks that, at every
sub-round, the tag classification (alive / in the frontier / removed) equals
the one computed from unbounded sub-round numbers.  It models the scheme
only; the kernel itself is checked by the GPU parity tests, which also force
the rewrite every 1 and 3 sub-rounds."""
import numpy as np
import pytest

MOD = 65534
DEAD = 0xFFFF


def tag(s):
    return 1 + (s - 1) % MOD


def classify_exact(st, s):
    # st: sub-round of the edge's frontier (0 = never pushed yet)
    alive = (st == 0) | (st > s)
    front = st == s
    return alive, front


def classify_tags(tg, s):
    ts, tn = tag(s), tag(s + 1)
    alive = (tg == 0) | (tg == tn)
    front = tg == ts
    return alive, front


@pytest.mark.parametrize("period", [32768, 20000, 7])
def test_tags_classify_like_unbounded_sub_rounds(period):
    rng = np.random.default_rng(period)
    S = 2 * MOD + 5000          # more than two wraps of the tag space
    M = 1500
    push_at = rng.integers(1, S + 1, M)   # sub-round whose frontier the edge joins
    push_at[:50] = rng.integers(1, 40, 50)        # some removed very early
    push_at[50:100] = S + 10                       # some never removed
    order = np.argsort(push_at, kind="stable")
    tg = np.zeros(M, np.int64)
    st = np.zeros(M, np.int64)  # exact frontier sub-round once pushed
    nxt = 0
    last = 0
    checks = 0
    for s in range(1, S + 1):
        # edges of frontier s were tagged during s-1 (or by the level scan)
        while nxt < M and push_at[order[nxt]] == s:
            e = order[nxt]
            tg[e] = tag(s)
            st[e] = s
            nxt += 1
        # the periodic rewrite at the start of the phase
        if s - last >= period:
            last = s
            keep = tag(s)
            tg[(tg != 0) & (tg != keep)] = DEAD
        # every edge's classification while sub-round s decides; edges pushed
        # during s (tag(s+1)) read as alive either way
        if s % 97 == 0 or s < 300 or abs(s - MOD) < 300 or abs(s - 2 * MOD) < 300:
            a1, f1 = classify_exact(st, s)
            a2, f2 = classify_tags(tg, s)
            assert np.array_equal(a1, a2) and np.array_equal(f1, f2), s
            pushed_now = push_at == s + 1
            tn = np.where(pushed_now, tag(s + 1), tg)
            a3, f3 = classify_tags(tn, s)
            assert np.array_equal(a1, a3) and np.array_equal(f1, f3), s
            checks += 1
    assert checks > 1000


def test_without_rewrite_a_wrapped_tag_is_misread():
    """The rewrite is needed: an edge removed at sub-round 1 carries tag 1,
    which is tag(MOD + 1), so without a rewrite it would read as in the
    frontier of sub-round MOD + 1."""
    s = MOD + 1
    alive, front = classify_tags(np.array([tag(1)]), s)
    assert front[0]
    exact_alive, exact_front = classify_exact(np.array([1]), s)
    assert not exact_front[0] and not exact_alive[0]
