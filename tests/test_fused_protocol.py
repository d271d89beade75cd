"""Model check, on CPU, of the bucket-version protocol that makes lookups of
the single-kernel batch safe against eviction chains in flight (the design
of k_fused; the CUDA kernel is covered by tests/test_gpu_fused.py).

A chain moves key K out of one candidate bucket and into the other; a lookup
of K probes both candidates.  Under sequential consistency (the fences of
the protocol order exactly these accesses), every interleaving of the
chain's steps with the lookup's steps is enumerated, and a lookup that ends
in a miss it accepts would be a lost key.  Without the version marks the same
enumeration finds such interleavings, so the check is not vacuous."""
import itertools

T = 1 << 16  # transit unit of a version word


def chain_steps(moves, marks=True):
    """Steps of one chain that moves K along `moves` = [(src, dst), ...]."""
    steps = []
    for src, dst in moves:
        if marks:
            steps.append(("mark", src))
        steps.append(("out", src))
        steps.append(("in", dst))
        if marks:
            steps.append(("unmark", src))
    return steps


READER = [("v0",), ("probe", 0), ("probe", 1), ("v1",)]


def run(order, writer, start):
    """Execute one interleaving; returns the lookup's verdict."""
    where = {start}
    ver = [0, 0]
    wi = ri = 0
    found = False
    v_before = v_after = None
    for who in order:
        if who == "w":
            op, b = writer[wi]
            wi += 1
            if op == "mark":
                ver[b] += T
            elif op == "unmark":
                ver[b] += 1 - T
            elif op == "out":
                where.discard(b)
            else:
                where.add(b)
        else:
            step = READER[ri]
            ri += 1
            if step[0] == "v0":
                v_before = tuple(ver)
            elif step[0] == "probe":
                found |= step[1] in where
            else:
                v_after = tuple(ver)
    if found:
        return "hit"
    quiet = all(v < T for v in v_before) and v_before == v_after
    return "miss" if quiet else "retry"


def verdicts(writer, start):
    n_w, n_r = len(writer), len(READER)
    out = set()
    for pos in itertools.combinations(range(n_w + n_r), n_r):
        order = ["w"] * (n_w + n_r)
        for p in pos:
            order[p] = "r"
        out.add(run(order, writer, start))
    return out


def test_one_move_never_loses_the_key():
    # K moves from bucket 0 to bucket 1 while the lookup runs
    assert "miss" not in verdicts(chain_steps([(0, 1)]), start=0)


def test_two_moves_never_lose_the_key():
    # K moves 0 -> 1 and later back 1 -> 0 (two steps of chains)
    assert "miss" not in verdicts(chain_steps([(0, 1), (1, 0)]), start=0)


def test_reverse_probe_order_is_also_safe():
    global READER
    saved = READER
    try:
        READER = [("v0",), ("probe", 1), ("probe", 0), ("v1",)]
        assert "miss" not in verdicts(chain_steps([(0, 1), (1, 0)]), start=0)
    finally:
        READER = saved


def test_without_marks_a_key_can_be_lost():
    assert "miss" in verdicts(chain_steps([(0, 1)], marks=False), start=0)


def test_a_quiet_table_gives_hits():
    assert verdicts([], start=0) == {"hit"}
