"""Pins of the oracle's score policies (Sec. 3.3 "Scoring policies"; the
formulas are our readings, fixed here by closed-form sequences)."""
import numpy as np

import oracle

Z = lambda n, d=1: np.zeros((n, d), np.float32)  # noqa: E731


def scores_of(t, keys):
    _, found, s = t.find(np.asarray(keys, np.uint64))
    assert found.all()
    return s.tolist()


def test_lru_step_per_call_and_set_step():
    t = oracle.OracleTable(4, 1, oracle.LRU)
    t.insert_or_assign(np.array([1, 2], np.uint64), Z(2))
    t.insert_or_assign(np.array([2, 3, 3], np.uint64), Z(3))
    assert scores_of(t, [1, 2, 3]) == [1, 2, 2]
    t.set_step(100)
    t.assign(np.array([1, 99], np.uint64), Z(2))         # assign writes the step too
    assert scores_of(t, [1, 2, 3]) == [101, 2, 2]
    assert t.step == 101


def test_lfu_counts_and_saturation():
    t = oracle.OracleTable(4, 1, oracle.LFU)
    t.insert_or_assign(np.array([7] * 5 + [8], np.uint64), Z(6))
    t.insert_or_assign(np.array([7, 7, 9], np.uint64), Z(3))
    assert scores_of(t, [7, 8, 9]) == [7, 1, 1]
    big = 2**64 - 3
    u = oracle.OracleTable(4, 1, oracle.LFU)
    b1, _, _ = oracle.map_keys(4, False, np.array([5], np.uint64))
    u.load(np.array([5], np.uint64), np.array([big], np.uint64), Z(1), b1)
    u.insert_or_assign(np.array([5] * 10, np.uint64), Z(10))
    assert scores_of(u, [5]) == [2**64 - 1]


def test_epoch_policies():
    t = oracle.OracleTable(4, 1, oracle.EPOCH_LRU)
    t.set_epoch(3)
    t.set_step((1 << 32) + 6)                             # low 32 bits of the step
    t.insert_or_assign(np.array([1], np.uint64), Z(1))
    assert scores_of(t, [1]) == [(3 << 32) | 7]
    f = oracle.OracleTable(4, 1, oracle.EPOCH_LFU)
    f.set_epoch(2)
    f.insert_or_assign(np.array([1, 1, 2], np.uint64), Z(3))
    f.set_epoch(5)
    f.insert_or_assign(np.array([1], np.uint64), Z(1))
    assert scores_of(f, [1, 2]) == [(5 << 32) | 3, (2 << 32) | 1]


def test_custom_and_ts_freq():
    t = oracle.OracleTable(4, 1, oracle.CUSTOM)
    t.insert_or_assign(np.array([1, 2, 1], np.uint64), Z(3), np.array([10, 20, 30], np.uint64))
    assert scores_of(t, [1, 2]) == [30, 20]
    t.assign(np.array([1], np.uint64), Z(1))              # no scores: keep
    t.assign(np.array([2], np.uint64), Z(1), np.array([5], np.uint64))
    assert scores_of(t, [1, 2]) == [30, 5]
    g = oracle.OracleTable(4, 1, oracle.CUSTOM_TS_FREQ)
    g.set_epoch(9)
    g.insert_or_assign(np.array([1, 1, 1], np.uint64), Z(3))
    g.set_epoch(11)
    g.insert_or_assign(np.array([1, 2], np.uint64), Z(2))
    assert scores_of(g, [1, 2]) == [(11 << 16) | 4, (11 << 16) | 1]
    h = oracle.OracleTable(4, 1, oracle.CUSTOM_TS_FREQ)
    h.insert_or_assign(np.array([3] * 70000, np.uint64), Z(70000))
    assert scores_of(h, [3]) == [0xFFFF]


def test_custom_requires_scores():
    t = oracle.OracleTable(4, 1, oracle.CUSTOM)
    try:
        t.insert_or_assign(np.array([1], np.uint64), Z(1))
    except oracle.OracleError as e:
        assert e.code == oracle.ERR_INVALID_ARG
    else:
        raise AssertionError("custom policy accepted an upsert without scores")
