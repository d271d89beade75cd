"""Host-side scheduling of the continuous-batching server, on CPU: batch
formation (one request per table per batch, per-table arrival order, op and
request caps) and HBM-budget admission with the growth rule of the resize
policy.  The kernels are not involved."""
from collections import deque

import pytest

torch = pytest.importorskip("torch")

from paper_2510_15095_gb300 import serving as SV  # noqa: E402


def server(n_tables, cap_slots, size_ub, budget, max_ops=1 << 20, max_reqs=64, slack=0):
    s = SV.HiveServer.__new__(SV.HiveServer)  # scheduler state only, no tables
    s.budget = float(budget)
    s.max_ops = max_ops
    s.max_reqs = max_reqs
    s.grow = (9, 10)
    s.size_ub = list(size_ub)
    s.cap_slots = list(cap_slots)
    s.slack = [slack] * n_tables
    return s


def req(rid, table, n, n_insert):
    k = torch.zeros(n, dtype=torch.int32)
    return SV.Request(rid=rid, table=table, arrival=0.0, ops=None, keys=k, vals=None,
                      n_insert=n_insert)


def test_needed_slots_follow_the_growth_rule():
    s = server(1, [1000], [800], budget=1e12, slack=64)
    # 800 + 50 live keys stay under 0.9 of 1000 slots: no growth
    assert s._needed_slots(0, 50) == 1000
    # 800 + 100 reach 0.9 exactly: the table must grow past 1000 * 10 / 9,
    # and the admission reserves one K-step of slack on top
    assert s._needed_slots(0, 100) == (900 * 10) // 9 + 1 + 64
    assert s._needed_slots(0, 200) == (1000 * 10) // 9 + 1 + 64


def test_one_request_per_table_in_arrival_order():
    s = server(3, [4096] * 3, [0] * 3, budget=1e12)
    reqs = [req(0, 0, 10, 5), req(1, 1, 10, 5), req(2, 0, 10, 5), req(3, 2, 10, 5),
            req(4, 1, 10, 5)]
    pending = deque(range(5))
    assert s._form_batch(pending, reqs) == [0, 1, 3]
    assert list(pending) == [2, 4]  # the later requests of tables 0 and 1 wait, in order
    assert s._form_batch(pending, reqs) == [2, 4]
    assert not pending


def test_op_and_request_caps():
    s = server(4, [4096] * 4, [0] * 4, budget=1e12, max_ops=25, max_reqs=2)
    reqs = [req(i, i, 10, 0) for i in range(4)]
    pending = deque(range(4))
    assert s._form_batch(pending, reqs) == [0, 1]  # two requests per batch
    s.max_reqs, s.max_ops = 8, 15
    assert s._form_batch(pending, reqs) == [2]  # 10 + 10 ops would pass the cap of 15
    assert list(pending) == [3]
    assert s._form_batch(pending, reqs) == [3]


def test_hbm_budget_blocks_a_growing_table_and_its_later_requests():
    slot = SV.SLOT_BYTES
    # table 0 would have to grow past the budget; table 1 fits
    s = server(2, [1024, 1024], [900, 100], budget=2100 * slot)
    reqs = [req(0, 0, 500, 500), req(1, 1, 50, 50), req(2, 0, 10, 0)]
    pending = deque(range(3))
    assert s._form_batch(pending, reqs) == [1]
    assert list(pending) == [0, 2]  # table 0 keeps its FIFO order behind the blocked request


class _FlatGroup:
    """Stands in for the library's multi-table group: erases balance the
    inserts, so every table's live size stays where it started."""

    def __init__(self, sizes):
        self.sizes = list(sizes)

    def bounds(self):
        return list(self.sizes)


class _Table:
    def __init__(self, slots):
        self.slots = slots

    def capacity(self):
        return self.slots


def test_flat_live_size_is_never_rejected():
    """40/20/40-style traffic whose erases keep the live size flat: the
    admission bound is refreshed from the library before each batch, so a
    long run of inserting requests never outgrows a budget that the live size
    fits in (counting inserts alone would pass it after a few batches)."""
    slot = SV.SLOT_BYTES
    s = server(1, [1024], [880], budget=1200 * slot, slack=64)
    s.multi = _FlatGroup([880])
    s.tables = [_Table(1024)]
    reqs = [req(i, 0, 40, 40) for i in range(50)]
    pending = deque(range(50))
    launched = []
    while pending:
        s._sync_bounds()
        chosen = s._form_batch(pending, reqs)
        assert chosen, f"request {pending[0]} would be rejected"
        s._note_launch(chosen, reqs)
        launched += chosen
    assert launched == list(range(50))
    # without the refresh the insert count alone exhausts the budget
    s = server(1, [1024], [880], budget=1200 * slot, slack=64)
    pending = deque(range(50))
    blocked = False
    while pending:
        chosen = s._form_batch(pending, reqs)
        if not chosen:
            blocked = True
            break
        s._note_launch(chosen, reqs)
    assert blocked
