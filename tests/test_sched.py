"""Triple-group scheduler (Sec. 3.5, Table 4) driven through its simulated
stream/event backend: no GPU. Checks the compatibility matrix on random
multi-stream programs and that compatible groups really overlap."""
import ctypes

import numpy as np
import pytest

from paper_2603_17168_gb300 import build as B

R, U, I = 0, 1, 2


@pytest.fixture(scope="module")
def sim():
    L = ctypes.CDLL(B.build_sim())
    f = L.hkv_sched_sim
    P = np.ctypeslib.ndpointer
    f.argtypes = [ctypes.c_int, P(np.int32), P(np.int32), P(np.float64), P(np.float64),
                  ctypes.c_int, P(np.float64), P(np.float64)]
    f.restype = ctypes.c_int

    def run(groups, streams, issue=None, dur=None, n_streams=None):
        g = np.asarray(groups, np.int32)
        s = np.asarray(streams, np.int32)
        n = g.size
        iss = np.zeros(n) if issue is None else np.asarray(issue, np.float64)
        d = np.ones(n) if dur is None else np.asarray(dur, np.float64)
        st, en = np.zeros(n), np.zeros(n)
        assert f(n, g, s, iss, d, int(n_streams or s.max() + 1), st, en) == 0
        return st, en
    return run


def compatible(a, b):
    return a == b and a != I


def test_readers_overlap_and_inserter_serialises(sim):
    st, en = sim([R, R, R, I, R, R], [0, 1, 2, 0, 1, 2])
    assert st[:3].tolist() == [0, 0, 0]          # R || R || R
    assert st[3] == 1                            # I after all readers
    assert st[4] == st[5] == 2                   # readers after I, together


def test_updaters_overlap_but_not_with_readers(sim):
    st, en = sim([U, U, R, R, U], [0, 1, 2, 3, 0])
    assert st[0] == st[1] == 0
    assert st[2] == st[3] == 1
    assert st[4] == 2


def test_inserters_never_overlap_each_other(sim):
    st, en = sim([I, I, I], [0, 1, 2])
    assert st.tolist() == [0, 1, 2]


@pytest.mark.parametrize("seed", range(20))
def test_random_programs_respect_table4(sim, seed):
    rng = np.random.default_rng(seed)
    n, ns = 200, 4
    g = rng.integers(0, 3, n)
    s = rng.integers(0, ns, n)
    issue = np.cumsum(rng.random(n) * 0.3)
    dur = 0.1 + rng.random(n)
    st, en = sim(g, s, issue, dur, ns)
    assert np.all(st >= issue - 1e-12)
    for i in range(n):
        for j in range(i + 1, n):
            if s[i] == s[j] or not compatible(g[i], g[j]):
                # issue order is preserved between incompatible ops
                assert en[i] <= st[j] + 1e-12, (i, j, g[i], g[j])
    # and compatible ops on different streams are not needlessly serialised:
    # a reader never waits for another reader
    for j in range(n):
        if g[j] == R:
            blockers = [en[i] for i in range(j) if (s[i] == s[j] or g[i] != R)]
            assert st[j] == pytest.approx(max(blockers + [issue[j]]))


@pytest.fixture(scope="module")
def sim_rw():
    L = ctypes.CDLL(B.build_sim())
    f = L.hkv_sched_sim_mode
    P = np.ctypeslib.ndpointer
    f.argtypes = [ctypes.c_int, P(np.int32), P(np.int32), P(np.float64), P(np.float64),
                  ctypes.c_int, ctypes.c_int, P(np.float64), P(np.float64)]
    f.restype = ctypes.c_int

    def run(groups, streams, rw, issue=None, dur=None, n_streams=None):
        g = np.asarray(groups, np.int32)
        s = np.asarray(streams, np.int32)
        n = g.size
        iss = np.zeros(n) if issue is None else np.asarray(issue, np.float64)
        d = np.ones(n) if dur is None else np.asarray(dur, np.float64)
        st, en = np.zeros(n), np.zeros(n)
        assert f(n, g, s, iss, d, int(n_streams or s.max() + 1), int(rw), st, en) == 0
        return st, en
    return run


def test_rw_lock_serialises_updaters_triple_group_overlaps_them(sim_rw):
    """The Exp 3e ablation in miniature: ten updaters on ten streams finish
    in one unit of time under the triple-group rule and in ten under a
    reader/writer lock; readers still overlap under both."""
    st, en = sim_rw([U] * 10, list(range(10)), False)
    assert en.max() == 1
    st, en = sim_rw([U] * 10, list(range(10)), True)
    assert sorted(st.tolist()) == list(range(10))
    st, en = sim_rw([R] * 6, list(range(6)), True)
    assert en.max() == 1


@pytest.mark.parametrize("seed", range(10))
def test_rw_lock_programs_respect_rw_compatibility(sim_rw, seed):
    rng = np.random.default_rng(100 + seed)
    n, ns = 150, 4
    g = rng.integers(0, 3, n)
    s = rng.integers(0, ns, n)
    issue = np.cumsum(rng.random(n) * 0.3)
    dur = 0.1 + rng.random(n)
    st, en = sim_rw(g, s, True, issue, dur, ns)
    for i in range(n):
        for j in range(i + 1, n):
            if s[i] == s[j] or not (g[i] == g[j] == R):
                assert en[i] <= st[j] + 1e-12, (i, j, g[i], g[j])


@pytest.fixture(scope="module")
def sim_threads():
    L = ctypes.CDLL(B.build_sim(force=True))
    f = L.hkv_sched_sim_threads
    P = np.ctypeslib.ndpointer
    f.argtypes = [ctypes.c_int, ctypes.c_int, P(np.int32), P(np.float64), ctypes.c_int,
                  ctypes.c_int, P(np.float64), P(np.float64)]
    f.restype = ctypes.c_int

    def run(groups, dur, rw_lock=0, launch_us=20):
        g = np.ascontiguousarray(groups, np.int32)
        n_threads, per = g.shape
        st, en = np.zeros(g.size), np.zeros(g.size)
        assert f(n_threads, per, g.ravel(), np.ascontiguousarray(dur, np.float64).ravel(),
                 rw_lock, launch_us, st, en) == 0
        return st.reshape(g.shape), en.reshape(g.shape)
    return run


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("rw_lock", [0, 1])
def test_threads_launching_concurrently_keep_table4(sim_threads, seed, rw_lock):
    """Host threads take roles and launch at the same time (the scheduler's
    mutex is not held while a call launches): no two incompatible ops
    overlap on the virtual clock, and the run ends (no deadlock)."""
    rng = np.random.default_rng(seed)
    n_threads, per = 6, 120
    # mostly one group at a time, with runs of each, so epochs of several
    # concurrent members form and are then broken by other groups
    runs = rng.integers(0, 3, size=(n_threads, per // 10))
    groups = np.repeat(runs, 10, axis=1)
    flip = rng.random(groups.shape) < 0.1
    groups[flip] = rng.integers(0, 3, size=flip.sum())
    dur = rng.uniform(0.5, 2.0, size=groups.shape)
    st, en = sim_threads(groups, dur, rw_lock=rw_lock, launch_us=30)
    g, s, e = groups.ravel(), st.ravel(), en.ravel()
    owner = np.repeat(np.arange(n_threads), per)
    ok_pair = (g[:, None] == g[None, :]) & (g[:, None] != I)
    if rw_lock:
        ok_pair &= g[:, None] == R
    overlap = (s[:, None] < e[None, :]) & (s[None, :] < e[:, None])
    bad = overlap & ~ok_pair & (owner[:, None] != owner[None, :])
    assert not bad.any(), np.argwhere(bad)[:5]
    if not rw_lock:
        # compatible groups did run side by side somewhere
        both = overlap & ok_pair & (owner[:, None] != owner[None, :])
        assert both.any()
