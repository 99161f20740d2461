"""Pins of the oracle's hash-map semantics (Sec. 5: guaranteed find / insert / erase with unique
keys) against a brute-force dictionary model, on random operation sequences chosen to contain
heavy duplication, insert+erase of one key inside one batch, misses and invalid keys."""
import numpy as np
import pytest

from oracle import (OracleMap, OP_FIND, OP_INSERT, OP_ERASE, ST_FOUND, ST_NOT_FOUND,
                    ST_INSERTED, ST_EXISTS, ST_ERASED, ST_INVALID, NONE)


def brute_force_batch(state: dict, ops, keys, vals):
    """Phased reading: finds see the pre-batch state, then inserts, then erases, each in batch
    order.  Written as three independent loops over a Python dict."""
    n = len(ops)
    res = [None] * n
    st = [None] * n
    pre = dict(state)
    ok = [o in (0, 1, 2) and all(-(1 << 20) <= c < (1 << 20) for c in k) for o, k in zip(ops, keys)]
    for i in range(n):
        if not ok[i]:
            res[i], st[i] = NONE, ST_INVALID
        elif ops[i] == OP_FIND:
            if keys[i] in pre:
                res[i], st[i] = pre[keys[i]], ST_FOUND
            else:
                res[i], st[i] = NONE, ST_NOT_FOUND
    for i in range(n):
        if ok[i] and ops[i] == OP_INSERT:
            if keys[i] in state:
                st[i] = ST_EXISTS
            else:
                state[keys[i]] = vals[i]
                st[i] = ST_INSERTED
    for i in range(n):
        if ok[i] and ops[i] == OP_INSERT:
            res[i] = state[keys[i]]
    for i in range(n):
        if ok[i] and ops[i] == OP_ERASE:
            if keys[i] in state:
                res[i], st[i] = state.pop(keys[i]), ST_ERASED
            else:
                res[i], st[i] = NONE, ST_NOT_FOUND
    return np.array(res, np.uint32), np.array(st, np.uint8)


@pytest.mark.parametrize("universe,n_batches,batch", [(8, 40, 16), (64, 30, 100), (5000, 10, 2000)])
def test_random_sequences_match_brute_force(universe, n_batches, batch):
    rng = np.random.default_rng(universe)
    pool = rng.integers(-(1 << 20), 1 << 20, size=(universe, 3))
    m = OracleMap()
    model = {}
    for _ in range(n_batches):
        ops = rng.choice([OP_FIND, OP_INSERT, OP_ERASE], size=batch, p=[0.5, 0.3, 0.2]).astype(np.uint8)
        ki = rng.integers(0, universe, size=batch)
        keys = pool[ki].astype(np.int32)
        vals = rng.integers(0, 1 << 31, size=batch).astype(np.uint32)
        res, st = m.batch(ops, keys, vals)
        eres, est = brute_force_batch(model, ops.tolist(), [tuple(k) for k in keys.tolist()],
                                      vals.tolist())
        np.testing.assert_array_equal(st, est)
        np.testing.assert_array_equal(res, eres)
        assert len(m) == len(model)
    k, v = m.dump()
    assert len({tuple(x) for x in k.tolist()}) == k.shape[0]   # uniqueness
    assert dict(zip(map(tuple, k.tolist()), v.tolist())) == model


def test_insert_then_erase_same_batch_and_duplicates():
    m = OracleMap()
    key = np.array([[1, 2, 3]] * 4, np.int32)
    ops = np.array([OP_INSERT, OP_INSERT, OP_ERASE, OP_FIND], np.uint8)
    res, st = m.batch(ops, key, np.array([7, 9, 0, 0], np.uint32))
    # the find sees the pre-batch (empty) state; first insert wins; erase removes it afterwards
    assert st.tolist() == [ST_INSERTED, ST_EXISTS, ST_ERASED, ST_NOT_FOUND]
    assert res.tolist() == [7, 7, 7, NONE]
    assert len(m) == 0


def test_invalid_keys_and_ops():
    m = OracleMap()
    keys = np.array([[1 << 20, 0, 0], [0, -(1 << 20) - 1, 0], [0, 0, 0], [0, 0, 0]], np.int32)
    ops = np.array([OP_INSERT, OP_INSERT, 9, OP_INSERT], np.uint8)
    res, st = m.batch(ops, keys, np.arange(4, dtype=np.uint32))
    assert st.tolist() == [ST_INVALID, ST_INVALID, ST_INVALID, ST_INSERTED]
    assert len(m) == 1


def test_extreme_valid_keys():
    m = OracleMap()
    lo, hi = -(1 << 20), (1 << 20) - 1
    keys = np.array([[lo, lo, lo], [hi, hi, hi], [lo, hi, 0], [hi, lo, -1]], np.int32)
    m.batch(np.full(4, OP_INSERT, np.uint8), keys, np.arange(4, dtype=np.uint32))
    res, st = m.batch(np.full(4, OP_FIND, np.uint8), keys)
    assert st.tolist() == [ST_FOUND] * 4 and res.tolist() == [0, 1, 2, 3]
