"""HIVE_DEBUG on the GPU: a table created with HIVE_DEBUG set checks the batch
contract of every update call on the host before it queues anything
(hive_check_batch).  A batch that breaks it (a key updated twice, or updated
and searched in one mixed batch) returns INVALID_ARG and leaves the table as
it was; a batch that keeps it runs as usual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15095_gb300 import hive
    hive.load_library()
    return hive


def i32(a, device="cuda"):
    return torch.tensor(np.asarray(a, dtype=np.uint32).view(np.int32), device=device)


def u8(a, device="cuda"):
    return torch.tensor(np.asarray(a, dtype=np.uint8), device=device)


def rejected(H, fn, *args, **kw):
    with pytest.raises(H.HiveError) as e:
        fn(*args, **kw)
    assert e.value.code == 1 and "batch contract" in str(e.value)


@pytest.mark.parametrize("resizable", [False, True])
def test_debug_table_rejects_broken_batches(H, monkeypatch, resizable):
    monkeypatch.setenv("HIVE_DEBUG", "1")
    t = H.HiveTable(1 << 12, max_slots=1 << 14, resizable=resizable)
    rejected(H, t.insert, i32([1, 2, 1]), i32([10, 20, 30]))
    assert t.size() == 0
    st = t.insert(i32([1, 2, 3]), i32([10, 20, 30]))
    assert st.cpu().tolist() == [H.INSERTED] * 3
    rejected(H, t.erase, i32([2, 2]))
    rejected(H, t.execute, u8([H.OP_FIND, H.OP_ERASE]), i32([3, 3]))
    rejected(H, t.execute, u8([H.OP_INSERT, H.OP_FIND]), i32([4, 4]), i32([1, 1]), fused=True)
    rejected(H, t.insert_host, i32([7, 8, 7], "cpu"), i32([1, 2, 3], "cpu"))
    if not resizable:
        rejected(H, t.insert_noalloc, i32([5, 5]), i32([1, 2]))
    assert t.size() == 3
    # repeated finds are allowed
    vo, st = t.execute(u8([H.OP_FIND, H.OP_FIND, H.OP_ERASE, H.OP_INSERT]), i32([1, 1, 2, 4]),
                       i32([0, 0, 0, 44]))
    assert st.cpu().tolist() == [H.FOUND, H.FOUND, H.ERASED, H.INSERTED]
    assert H.to_host_u32(vo).tolist() == [10, 10, 0, 0]
    vo, fo = t.find(i32([1, 2, 3, 4]))
    assert H.to_host_u32(vo).tolist() == [10, 0, 30, 44]
    assert fo.cpu().tolist() == [1, 0, 1, 1]
    assert t.size() == 3
    t.close()


def test_debug_hive32_rejects_broken_batches(H, monkeypatch):
    monkeypatch.setenv("HIVE_DEBUG", "1")
    t = H.Hive32Table(1 << 12, H.KEY16_VAL16)
    rejected(H, t.insert, i32([9, 9]), i32([1, 2]))
    st = t.insert(i32([9, 10]), i32([1, 2]))
    assert st.cpu().tolist() == [H.INSERTED] * 2
    rejected(H, t.execute, u8([H.OP_ERASE, H.OP_FIND]), i32([10, 10]))
    assert t.size() == 2
    t.close()
    s = H.Hive32Table(1 << 12, H.KEY_ONLY)
    rejected(H, s.insert, i32([70000, 70000]))
    rejected(H, s.erase, i32([3, 3]))
    assert s.insert(i32([70000, 70001])).cpu().tolist() == [H.INSERTED] * 2
    assert s.size() == 2
    s.close()


def test_debug_multi_table_batch(H, monkeypatch):
    """The contract holds per table over all of its segments of a batch; one
    key in two different tables is fine."""
    monkeypatch.setenv("HIVE_DEBUG", "1")
    ta, tb = H.HiveTable(1 << 12), H.HiveTable(1 << 12)
    m = H.HiveMulti([ta, tb], max_segments=4, max_ops=1 << 10, use_graph=False)

    def seg(t, ops, keys, vals):
        n = len(keys)
        return {"table": t, "ops": u8(ops), "keys": i32(keys), "vals": i32(vals),
                "vals_out": torch.empty(n, dtype=torch.int32, device="cuda"),
                "status": torch.empty(n, dtype=torch.uint8, device="cuda")}

    with pytest.raises(H.HiveError) as e:
        m.execute([seg(0, [H.OP_INSERT], [5], [1]), seg(1, [H.OP_INSERT], [5], [2]),
                   seg(0, [H.OP_FIND], [5], [0])])
    assert e.value.code == 1 and "table 0" in str(e.value)
    assert ta.size() == 0 and tb.size() == 0
    g = [seg(0, [H.OP_INSERT], [5], [1]), seg(1, [H.OP_INSERT, H.OP_FIND], [5, 6], [2, 0])]
    m.execute(g)
    torch.cuda.synchronize()
    assert g[0]["status"].cpu().tolist() == [H.INSERTED]
    assert g[1]["status"].cpu().tolist() == [H.INSERTED, H.NOT_FOUND]
    assert ta.size() == 1 and tb.size() == 1
    m.close()
    ta.close()
    tb.close()
