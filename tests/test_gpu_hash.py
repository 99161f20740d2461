"""GPU parity of the hash batch (Sec. 5 find / insert / erase, phased reading) against the CPU
oracle, through the C ABI.  Bit-exact: per-op statuses and results (finds exactly; duplicate
inserts / erases of one key compared as a multiset per key, since which duplicate wins is not
fixed), and the final key -> value contents."""
import numpy as np
import pytest
import torch

from oracle import OracleMap
from paper_1805_03709_b300 import synth
from paper_1805_03709_b300 import vbh as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def HashMap(*a, **k):
    from paper_1805_03709_b300.volume import HashMap as H
    return H(*a, **k)


def key_value(keys):
    k = keys.astype(np.int64)
    return ((k[:, 0] * 73 + k[:, 1] * 977 + k[:, 2] * 10007) & 0x7FFFFFFF).astype(np.uint32)


def gpu_batch(hm, ops, keys, vals):
    o = torch.from_numpy(ops).cuda()
    k = torch.from_numpy(np.ascontiguousarray(keys, np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda() if vals is not None else None
    res, st = hm.batch(o, k, v)
    return res.cpu().numpy().view(np.uint32), st.cpu().numpy()


def assert_same(ops, keys, res_g, st_g, res_o, st_o):
    """Finds and invalid ops exactly; inserts and erases as per-key multisets."""
    exact = (ops == V.VBH_OP_FIND) | (st_o == V.VBH_ST_INVALID)
    np.testing.assert_array_equal(st_g[exact], st_o[exact])
    np.testing.assert_array_equal(res_g[exact], res_o[exact])
    for op in (V.VBH_OP_INSERT, V.VBH_OP_ERASE):
        sel = (ops == op) & (st_o != V.VBH_ST_INVALID)
        if not sel.any():
            continue
        def rows(res, st):
            k = keys[sel].astype(np.int64)
            a = np.stack([k[:, 0], k[:, 1], k[:, 2], st[sel].astype(np.int64),
                          res[sel].astype(np.int64)], 1)
            return a[np.lexsort(a.T[::-1])]
        np.testing.assert_array_equal(rows(res_g, st_g), rows(res_o, st_o))


def check_contents(hm, om):
    kg, vg = hm.dump()
    ko, vo = om.dump()
    order = np.lexsort(kg.T[::-1])
    np.testing.assert_array_equal(kg[order], ko)
    np.testing.assert_array_equal(vg[order], vo)
    c = hm.counters()
    assert c.live == len(om)
    assert c.live + c.tombstones + c.empty == hm.cfg.n_buckets * 4


def mixed_ops(rng, n, pool, present, p=(0.5, 0.3, 0.2)):
    ops = rng.choice([0, 1, 2], size=n, p=p).astype(np.uint8)
    idx = rng.integers(0, len(pool), size=n)
    return ops, pool[idx]


@pytest.mark.parametrize("hash_fn", [V.VBH_HASH_MIX, V.VBH_HASH_PRIMES])
@pytest.mark.parametrize("universe,batch,n_batches", [(16, 37, 30), (3000, 1000, 12), (200000, 65537, 4)])
def test_random_batches(hash_fn, universe, batch, n_batches):
    rng = np.random.default_rng(universe + hash_fn)
    pool = synth.random_hash_keys(universe, seed=universe)
    hm = HashMap(n_buckets=max(16, 1 << int(np.ceil(np.log2(universe / 2)))), hash_fn=hash_fn)
    om = OracleMap()
    for _ in range(n_batches):
        ops, keys = mixed_ops(rng, batch, pool, None)
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
    check_contents(hm, om)


def test_small_and_phased_batches_interleaved():
    """A plain map runs batches of at most 2^17 ops as one launch with one thread per op and
    larger ones as phased launches over compacted op lists; interleaved on one map (each kind
    of batch leaves the other's list counts ready), both give the oracle's results."""
    rng = np.random.default_rng(17)
    pool = synth.random_hash_keys(300000, seed=17)
    hm = HashMap(n_buckets=1 << 17, max_batch=1 << 18)
    om = OracleMap()
    for n in (1000, (1 << 17) + 3, 37, 150001, 1 << 17, 5000, 140000):
        ops, keys = mixed_ops(rng, n, pool, None, p=(0.4, 0.4, 0.2))
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
        c = hm.counters()
        assert c.live == len(om) and c.error_flags == 0
    check_contents(hm, om)


def test_zipf_clustered_keys_heavy_duplication():
    rng = np.random.default_rng(7)
    hm = HashMap(n_buckets=1 << 14)
    om = OracleMap()
    for b in range(6):
        keys = synth.zipf_cluster_keys(50000, seed=b, hot_side=32)
        ops = rng.choice([0, 1, 2], size=len(keys), p=[0.5, 0.3, 0.2]).astype(np.uint8)
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
    check_contents(hm, om)


def test_values_at_the_top_of_the_range():
    """A plain map stores any uint32 value, the library's internal markers included; the
    duplicate inserts of a batch report the winner's value."""
    hm = HashMap(n_buckets=64)
    keys = np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3], [7, 8, 9], [4, 5, 6]], np.int32)
    vals = np.array([0xFFFFFFFE, 0xFFFFFFFF, 0xFFFFFFFE, 0x80000000, 0xFFFFFFFF], np.uint32)
    rg, sg = gpu_batch(hm, np.ones(5, np.uint8), keys, vals)
    assert sorted(sg.tolist()) == [V.VBH_ST_INSERTED] * 3 + [V.VBH_ST_EXISTS] * 2
    np.testing.assert_array_equal(rg, vals)
    rg, sg = gpu_batch(hm, np.zeros(5, np.uint8), keys, None)
    assert np.all(sg == V.VBH_ST_FOUND)
    np.testing.assert_array_equal(rg, vals)
    assert hm.counters().live == 3 and hm.counters().error_flags == 0


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 9, 31, 33, 255, 257])
def test_ragged_sizes_and_invalid(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(-40, 40, size=(n, 3)).astype(np.int32)
    keys[::5, 1] = 1 << 20          # out of range
    ops = rng.integers(0, 4, size=n).astype(np.uint8)   # 3 = unknown op
    hm = HashMap(n_buckets=64)
    om = OracleMap()
    for _ in range(3):
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
        ops = np.roll(ops, 1)
    check_contents(hm, om)


def test_single_kind_batches_in_sequence():
    """Batches of one op kind each, an all-invalid batch and an empty one, back to back: the
    other two op lists of each batch are empty, and consecutive batches use alternate sets of
    list lengths (each batch's first pass zeroes the next batch's set)."""
    rng = np.random.default_rng(11)
    pool = synth.random_hash_keys(3000, seed=11, lo=-200, hi=200)
    hm = HashMap(n_buckets=1024)   # 4096 slots: every key of the pool fits
    om = OracleMap()
    bad = pool[:500].copy()
    bad[:, 2] = -(1 << 21)   # out of range
    plan = [(V.VBH_OP_INSERT, pool[:1500]), (V.VBH_OP_FIND, pool[rng.integers(0, 3000, 2000)]),
            (V.VBH_OP_ERASE, pool[rng.integers(0, 1500, 900)]), (None, None),
            (V.VBH_OP_FIND, pool[:3000]), (V.VBH_OP_INSERT, pool[rng.integers(0, 3000, 2500)]),
            (V.VBH_OP_INSERT, bad), (V.VBH_OP_ERASE, pool[1000:2000]),
            (V.VBH_OP_FIND, pool[rng.integers(0, 3000, 777)])]
    for op, keys in plan:
        if op is None:
            e = torch.zeros(0, dtype=torch.uint8, device="cuda")
            hm.batch(e, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
            continue
        ops = np.full(len(keys), op, np.uint8)
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
    check_contents(hm, om)


def test_empty_batch():
    hm = HashMap(n_buckets=16)
    e = torch.zeros(0, dtype=torch.uint8, device="cuda")
    res, st = hm.batch(e, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    assert res.numel() == 0 and hm.counters().live == 0


def test_full_table_reports_capacity_and_recovers():
    hm = HashMap(n_buckets=4)      # 16 slots
    keys = np.array([[i, 2 * i, -i] for i in range(20)], np.int32)
    ops = np.full(20, V.VBH_OP_INSERT, np.uint8)
    rg, sg = gpu_batch(hm, ops, keys, key_value(keys))
    assert (sg == V.VBH_ST_INSERTED).sum() == 16 and (sg == V.VBH_ST_CAPACITY).sum() == 4
    assert np.all(rg[sg == V.VBH_ST_CAPACITY] == V.VBH_NONE)
    assert hm.counters().error_flags & 2
    ins = keys[sg == V.VBH_ST_INSERTED]
    lost = keys[sg == V.VBH_ST_CAPACITY]
    # erase two, then the lost keys can go in (tombstones are reused)
    gpu_batch(hm, np.full(2, V.VBH_OP_ERASE, np.uint8), ins[:2], None)
    c = hm.counters()
    assert (c.live, c.tombstones, c.empty) == (14, 2, 0)   # full buckets: tombstones
    rg, sg = gpu_batch(hm, np.full(2, V.VBH_OP_INSERT, np.uint8), lost[:2], key_value(lost[:2]))
    assert np.all(sg == V.VBH_ST_INSERTED)
    back = np.concatenate([ins[2:], lost[:2]])
    rg, sg = gpu_batch(hm, np.zeros(len(back), np.uint8), back, None)
    assert len(back) == 16 and np.all(sg == V.VBH_ST_FOUND)
    np.testing.assert_array_equal(rg, key_value(back))
    # more ops than keys is refused before any launch (the kernels read one key per op)
    with pytest.raises(ValueError):
        hm.batch(torch.zeros(18, dtype=torch.uint8, device="cuda"),
                 torch.from_numpy(np.ascontiguousarray(back)).cuda())


def test_erase_beside_an_empty_slot_leaves_no_tombstone():
    """An erased slot whose bucket still holds a never-used slot becomes never-used itself (no
    find's probe sequence changes); keys that overflowed into later buckets stay findable."""
    hm = HashMap(n_buckets=1 << 10)
    om = OracleMap()
    keys = synth.random_hash_keys(200, seed=11)
    vals = key_value(keys)
    gpu_batch(hm, np.ones(200, np.uint8), keys, vals)
    om.batch(np.ones(200, np.uint8), keys, vals)
    rg, sg = gpu_batch(hm, np.full(100, 2, np.uint8), keys[::2], None)
    om.batch(np.full(100, 2, np.uint8), keys[::2], None)
    assert np.all(sg == V.VBH_ST_ERASED)
    c = hm.counters()
    assert c.live == 100 and c.tombstones == 0 and c.empty == 4096 - 100
    check_contents(hm, om)
    # a crowded small table: overflow chains, erases both ways, finds stay exact
    hm2 = HashMap(n_buckets=16)
    om2 = OracleMap()
    rng = np.random.default_rng(5)
    pool = synth.random_hash_keys(56, seed=12)
    gpu_batch(hm2, np.ones(56, np.uint8), pool, key_value(pool))
    om2.batch(np.ones(56, np.uint8), pool, key_value(pool))
    for _ in range(20):
        ops = rng.choice([0, 1, 2], size=40, p=[0.4, 0.3, 0.3]).astype(np.uint8)
        k = pool[rng.integers(0, 56, size=40)]
        rg, sg = gpu_batch(hm2, ops, k, key_value(k))
        ro, so = om2.batch(ops, k, key_value(k))
        assert_same(ops, k, rg, sg, ro, so)
    check_contents(hm2, om2)


def test_small_batch_keys_at_the_top_of_the_coordinate_range():
    """Keys at both ends of the coordinate range: the two largest keys pack to 2^63 - 1 and
    2^63 - 2, one bit below the free-slot markers (all ones, all ones minus one).  Mixed small
    batches of those keys, their neighbours and ordinary keys (duplicate inserts, insert and
    erase of one key in a batch, finds of keys inserted in the same batch) give the oracle's
    results."""
    top = (1 << 20) - 1
    special = np.array([[top, top, top], [top - 1, top, top]], np.int32)
    near = np.array([[top, top - 1, top], [top - 2, top, top], [top, top, top - 1],
                     [-(1 << 20), -(1 << 20), -(1 << 20)]], np.int32)
    pool = np.concatenate([special, near, synth.random_hash_keys(20, seed=23)])
    rng = np.random.default_rng(29)
    for n_buckets in (8, 64):   # a crowded table (32 slots for 26 keys) and a roomy one
        hm = HashMap(n_buckets=n_buckets)
        om = OracleMap()
        for b in range(40):
            n = int(rng.integers(1, 48))
            ops = rng.choice([0, 1, 2], size=n, p=[0.35, 0.4, 0.25]).astype(np.uint8)
            keys = pool[rng.integers(0, len(pool) if b % 2 else len(special), size=n)]
            vals = key_value(keys)
            rg, sg = gpu_batch(hm, ops, keys, vals)
            ro, so = om.batch(ops, keys, vals)
            assert_same(ops, keys, rg, sg, ro, so)
            c = hm.counters()
            assert c.live == len(om) and c.error_flags == 0
        check_contents(hm, om)


@pytest.mark.parametrize("lf", [0.5, 0.7, 0.84, 0.9])
def test_load_factor_mixed_and_rebuild(lf):
    """Mixed batches on a small table prefilled to load factor lf (long probe chains at the
    higher loads), a rebuild in the middle."""
    rng = np.random.default_rng(int(lf * 10))
    n_buckets = 1 << 12
    cap = n_buckets * 4
    pool = synth.random_hash_keys(int(cap * 1.5), seed=3)
    hm = HashMap(n_buckets=n_buckets)
    om = OracleMap()
    pre = pool[:int(cap * lf)]
    for ch in np.array_split(np.arange(len(pre)), 4):
        k = pre[ch]
        gpu_batch(hm, np.full(len(k), 1, np.uint8), k, key_value(k))
        om.batch(np.full(len(k), 1, np.uint8), k, key_value(k))
    check_contents(hm, om)
    for b in range(6):
        ops = rng.choice([0, 1, 2], size=4000, p=[0.5, 0.25, 0.25]).astype(np.uint8)
        keys = pool[rng.integers(0, len(pool), size=4000)]
        vals = key_value(keys)
        rg, sg = gpu_batch(hm, ops, keys, vals)
        ro, so = om.batch(ops, keys, vals)
        assert_same(ops, keys, rg, sg, ro, so)
        if b == 3:
            hm.rebuild()
            assert hm.counters().tombstones == 0
            check_contents(hm, om)
    check_contents(hm, om)


def test_voxel_block_map_pool_indices():
    hm = HashMap(n_buckets=256, max_blocks=100)
    keys = np.array([[i, -i, 3] for i in range(120)], np.int32)
    ops = np.full(120, V.VBH_OP_INSERT, np.uint8)
    rg, sg = gpu_batch(hm, ops, keys, None)
    ok = sg == V.VBH_ST_INSERTED
    assert ok.sum() == 100 and (sg == V.VBH_ST_CAPACITY).sum() == 20
    assert sorted(rg[ok].tolist()) == list(range(100))       # each pool entry once
    assert hm.counters().free_blocks == 0 and hm.counters().live == 100
    # duplicates of one key share its pool index (which 100 keys won the pool is not fixed)
    won, lost = keys[ok], keys[~ok]
    dup = np.repeat(won[:3], 4, axis=0)
    rg2, sg2 = gpu_batch(hm, np.full(12, V.VBH_OP_INSERT, np.uint8), dup, None)
    assert np.all(sg2 == V.VBH_ST_EXISTS)
    np.testing.assert_array_equal(rg2, np.repeat(rg[ok][:3], 4))
    # erase returns entries to the pool; re-insert reuses them
    rg3, sg3 = gpu_batch(hm, np.full(10, V.VBH_OP_ERASE, np.uint8), won[:10], None)
    assert np.all(sg3 == V.VBH_ST_ERASED) and hm.counters().free_blocks == 10
    rg4, sg4 = gpu_batch(hm, np.full(10, V.VBH_OP_INSERT, np.uint8), lost[:10], None)
    assert np.all(sg4 == V.VBH_ST_INSERTED)
    assert sorted(rg4.tolist()) == sorted(rg3.tolist())


@pytest.mark.parametrize("lf", [0.7, 0.9])
def test_full_size_table_batch_2e20(lf):
    """2^22 buckets x 4 slots, prefilled to load factor lf with uniform keys in [-2^20, 2^20)^3,
    then a 2^20-op batch (50 % find half hits, 30 % insert of absent keys, 20 % erase), then
    2^16-, 2^12- and 2^16-op batches of the same mix."""
    n_buckets = 1 << 22
    cap = n_buckets * 4
    n_pre = int(lf * cap)
    rng = np.random.default_rng(1805)
    pool = synth.random_hash_keys(n_pre + (1 << 20), seed=1805)
    pre, fresh = pool[:n_pre], pool[n_pre:]
    hm = HashMap(n_buckets=n_buckets)
    om = OracleMap()
    for ch in np.array_split(np.arange(n_pre), 4):
        k = pre[ch]
        gpu_batch(hm, np.full(len(k), 1, np.uint8), k, key_value(k))
        om.batch(np.full(len(k), 1, np.uint8), k, key_value(k))
    n = 1 << 20
    nf, ni = n // 2, int(0.3 * n)
    ne = n - nf - ni
    keys = np.concatenate([pre[rng.integers(0, n_pre, nf // 2)], fresh[rng.integers(0, len(fresh), nf - nf // 2)],
                           fresh[:ni], pre[rng.integers(0, n_pre, ne)]])
    ops = np.concatenate([np.zeros(nf), np.ones(ni), np.full(ne, 2)]).astype(np.uint8)
    perm = rng.permutation(n)
    keys, ops = keys[perm], ops[perm]
    vals = key_value(keys)
    rg, sg = gpu_batch(hm, ops, keys, vals)
    ro, so = om.batch(ops, keys, vals)
    assert_same(ops, keys, rg, sg, ro, so)
    c = hm.counters()
    assert c.live == len(om)
    # then batches of 2^16 and 2^12 ops (one cooperative launch each, one thread per op), the
    # sizes the small-batch measurement times, on the same full-size table
    for m in (1 << 16, 1 << 12, 1 << 16):
        mf, mi = m // 2, int(0.3 * m)
        me = m - mf - mi
        k2 = np.concatenate([pre[rng.integers(0, n_pre, mf // 2)],
                             fresh[rng.integers(0, len(fresh), mf - mf // 2)],
                             synth.random_hash_keys(mi, seed=int(rng.integers(1 << 30))),
                             pre[rng.integers(0, n_pre, me)]])
        o2 = np.concatenate([np.zeros(mf), np.ones(mi), np.full(me, 2)]).astype(np.uint8)
        p2 = rng.permutation(m)
        k2, o2 = k2[p2], o2[p2]
        v2 = key_value(k2)
        rg, sg = gpu_batch(hm, o2, k2, v2)
        ro, so = om.batch(o2, k2, v2)
        assert_same(o2, k2, rg, sg, ro, so)
        assert hm.counters().live == len(om)


def test_full_size_table_batch_2e22():
    """The largest batch the benchmark times: 2^22 ops of the same mix on the 2^22 x 4 table at
    load factor 0.7; the prefill's inserts (batches of ~2.9 M ops) are compared too, and the
    table's contents at the end."""
    n_buckets = 1 << 22
    n_pre = int(0.7 * n_buckets * 4)
    n = 1 << 22
    rng = np.random.default_rng(22)
    pool = synth.distinct_keys(n_pre + n, seed=22)
    pre, fresh = pool[:n_pre], pool[n_pre:]
    hm = HashMap(n_buckets=n_buckets, max_batch=1 << 23)
    om = OracleMap()
    for ch in np.array_split(np.arange(n_pre), 4):
        k = pre[ch]
        o = np.full(len(k), 1, np.uint8)
        rg, sg = gpu_batch(hm, o, k, key_value(k))
        ro, so = om.batch(o, k, key_value(k))
        assert_same(o, k, rg, sg, ro, so)
    nf, ni = n // 2, int(0.3 * n)
    ne = n - nf - ni
    keys = np.concatenate([pre[rng.integers(0, n_pre, nf // 2)],
                           fresh[rng.integers(0, len(fresh), nf - nf // 2)],
                           fresh[:ni], pre[rng.integers(0, n_pre, ne)]])
    ops = np.concatenate([np.zeros(nf), np.ones(ni), np.full(ne, 2)]).astype(np.uint8)
    perm = rng.permutation(n)
    keys, ops = keys[perm], ops[perm]
    vals = key_value(keys)
    rg, sg = gpu_batch(hm, ops, keys, vals)
    ro, so = om.batch(ops, keys, vals)
    assert_same(ops, keys, rg, sg, ro, so)
    assert hm.counters().error_flags == 0
    check_contents(hm, om)
