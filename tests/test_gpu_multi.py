"""GPU parity of multi-table batches (hive_multi_*) against per-table oracles.

Every segment's per-op statuses and find values must equal the oracle
dictionary of its table applied to that segment; after each batch every
table's size, contents and invariants are checked, and resizable tables must
follow the oracle's capacity model call by call.
"""
import numpy as np
import pytest

import oracle
from paper_2510_15095_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
S = 32


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def _batch(rng, live, ctr, seed, n_ins, n_er, n_fd):
    new, ctr = W.take_keys(seed, ctr, n_ins)
    absent, ctr = W.take_keys(seed, ctr, max(n_fd // 4, 1))
    n_er = min(n_er, live.size)
    ops, keys, vals = W.mixed_batch(rng, live, new, n_ins, n_er, n_fd - n_fd // 4, seed=seed)
    # add finds of absent keys
    ops = np.concatenate([ops, np.full(absent.size, W.OP_FIND, np.uint8)])
    keys = np.concatenate([keys, absent]).astype(np.uint32)
    vals = np.concatenate([vals, np.zeros(absent.size, np.uint32)]).astype(np.uint32)
    perm = rng.permutation(ops.size)
    return ops[perm], keys[perm], vals[perm], ctr


def _run(H, tables, dicts, policies, batches, use_graph, rng, seed0, skip_prob=0.2, host=False):
    m = H.HiveMulti(tables, max_segments=2 * len(tables), max_ops=1 << 22, use_graph=use_graph)
    ctrs = [1_000_000 * (i + 1) for i in range(len(tables))]
    for b, (n_ins, n_er, n_fd) in enumerate(batches):
        segs, exp = [], []
        order = rng.permutation(len(tables))
        for t in order:
            if rng.random() < skip_prob:
                continue
            live, _ = dicts[t].dump()
            ni = int(rng.integers(0, n_ins + 1))
            ops, keys, vals, ctrs[t] = _batch(rng, live, ctrs[t], seed0 + t, ni,
                                             int(rng.integers(0, n_er + 1)), int(rng.integers(1, n_fd + 1)))
            if host:  # payload in pinned host memory, used in place by the kernels
                g = {"table": int(t), "ops": torch.from_numpy(ops).pin_memory(),
                     "keys": torch.from_numpy(keys.view(np.int32)).pin_memory(),
                     "vals": torch.from_numpy(vals.view(np.int32)).pin_memory(),
                     "vals_out": torch.empty(keys.size, dtype=torch.int32, pin_memory=True),
                     "status": torch.empty(keys.size, dtype=torch.uint8, pin_memory=True)}
            else:
                g = {"table": int(t), "ops": torch.from_numpy(ops).cuda(),
                     "keys": H.to_device_u32(keys), "vals": H.to_device_u32(vals),
                     "vals_out": torch.empty(keys.size, dtype=torch.int32, device="cuda"),
                     "status": torch.empty(keys.size, dtype=torch.uint8, device="cuda")}
            g["n_insert"] = int((ops == W.OP_INSERT).sum())
            if policies[t] is not None:
                policies[t].grow(len(dicts[t]), g["n_insert"])
            ev, est = dicts[t].execute(ops, keys, vals)
            segs.append(g)
            exp.append((t, ev, est))
        segs.append({"table": 0, "ops": torch.empty(0, dtype=torch.uint8, device="cuda"),
                     "keys": torch.empty(0, dtype=torch.int32, device="cuda")})  # empty segment
        m.execute(segs)
        torch.cuda.synchronize()
        for g, (t, ev, est) in zip(segs, exp):
            got_st = g["status"].cpu().numpy()
            got_v = H.to_host_u32(g["vals_out"])
            assert np.array_equal(got_st, est), (b, t, np.flatnonzero(got_st != est)[:5])
            assert np.array_equal(got_v, ev), (b, t)
        for t, tb in enumerate(tables):
            if policies[t] is not None:
                policies[t].shrink(len(dicts[t]))
                assert tb.capacity() == policies[t].s.S * policies[t].state[0], (b, t, tb.capacity(), policies[t].state)
            img = tb.dump()
            code, where = oracle.check_image(img, img["S"], dicts[t], policies[t])
            assert code == 0, (b, t, code, where)
            assert tb.check() == 0
    m.close()


@pytest.mark.parametrize("use_graph,bs", [(False, 32), (True, 32), (True, 16)])
def test_multi_fixed_tables(H, use_graph, bs):
    rng = np.random.default_rng(3 if use_graph else 4)
    sizes = [1 << int(x) for x in rng.integers(10, 17, 24)]
    tables = [H.HiveTable(sz, bucket_slots=bs) for sz in sizes]
    dicts = [oracle.Dict() for _ in tables]
    for i, (tb, d) in enumerate(zip(tables, dicts)):  # preload to about half
        k, _ = W.take_keys(500 + i, 0, sizes[i] // 2)
        v = W.values_for(k, 500 + i)
        tb.insert(H.to_device_u32(k), H.to_device_u32(v))
        d.insert(k, v)
    _run(H, tables, dicts, [None] * len(tables), [(200, 150, 400)] * 5, use_graph, rng, 500)
    for tb in tables:
        tb.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_multi_resizable_grow_and_shrink(H, use_graph):
    rng = np.random.default_rng(11 if use_graph else 12)
    n = 16
    init = [1 << int(x) for x in rng.integers(10, 14, n)]
    K = 32
    tables = [H.HiveTable(sz, max_slots=1 << 22, resizable=True, resize_batch=K) for sz in init]
    pols = [oracle.Policy(sz // S, (1 << 22) // S, K=K) for sz in init]
    dicts = [oracle.Dict() for _ in tables]
    grow = [(20_000, 2_000, 3_000)] * 4
    shrink = [(500, 20_000, 3_000)] * 4
    _run(H, tables, dicts, pols, grow + shrink, use_graph, rng, 900, skip_prob=0.1)
    for tb in tables:
        tb.close()


def test_multi_mixed_fixed_and_resizable_with_single_calls(H):
    rng = np.random.default_rng(21)
    tables = [H.HiveTable(1 << 12), H.HiveTable(1 << 11, max_slots=1 << 18, resizable=True, resize_batch=16),
              H.HiveTable(1 << 14), H.HiveTable(1 << 10, max_slots=1 << 18, resizable=True, resize_batch=64)]
    pols = [None, oracle.Policy(64, 1 << 13, K=16), None, oracle.Policy(32, 1 << 13, K=64)]
    dicts = [oracle.Dict() for _ in tables]
    _run(H, tables, dicts, pols, [(800, 200, 500)] * 3, True, rng, 1300, skip_prob=0.0)
    # single-table calls between batches keep working on the same tables
    k, _ = W.take_keys(77, 5_000_000, 500)
    v = W.values_for(k, 77)
    pols[1].grow(len(dicts[1]), 500)
    st = tables[1].insert(H.to_device_u32(k), H.to_device_u32(v)).cpu().numpy()
    assert np.array_equal(st, dicts[1].insert(k, v))
    pols[1].shrink(len(dicts[1]))
    assert tables[1].capacity() == S * pols[1].state[0]
    _run(H, tables, dicts, pols, [(800, 200, 500)] * 2, True, rng, 1400, skip_prob=0.0)
    for tb in tables:
        tb.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_multi_host_payload_segments(H, use_graph):
    """Segments whose arrays are pinned host tensors: the kernels read the ops
    and write the results in place across the CPU-GPU link; results, sizes,
    capacities and contents equal the oracles', as with device arrays."""
    rng = np.random.default_rng(31 if use_graph else 32)
    n = 8
    init = [1 << int(x) for x in rng.integers(10, 13, n)]
    K = 32
    tables = [H.HiveTable(sz, max_slots=1 << 20, resizable=True, resize_batch=K, bucket_slots=16)
              for sz in init]
    pols = [oracle.Policy(sz // 16, (1 << 20) // 16, K=K, S=16) for sz in init]
    dicts = [oracle.Dict() for _ in tables]
    _run(H, tables, dicts, pols, [(5_000, 500, 2_000)] * 3 + [(200, 6_000, 2_000)] * 2,
         use_graph, rng, 1700, skip_prob=0.1, host=True)
    for tb in tables:
        tb.close()
