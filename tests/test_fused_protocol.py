"""Model check, on CPU, of the bucket-version protocol that makes lookups of
the single-kernel batch safe against eviction chains in flight (the design
of k_fused; the CUDA kernel is covered by tests/test_gpu_fused.py).

A chain moves key K out of one candidate bucket and into the other (or into
the stash); a lookup of K probes both candidates and the stash.  The chain
marks the version word of K's BitHash1 bucket (bucket 0 here) while K is in
transit, whichever bucket K leaves, so the lookup reads that one version
word before and after probing.  Under sequential consistency (the fences of
the protocol order exactly these accesses), every interleaving of the
chain's steps with the lookup's steps is enumerated, and a lookup that ends
in a miss it accepts would be a lost key.  Without the marks, or with marks
on the bucket K leaves while the lookup reads only bucket 0's version, the
same enumeration finds such interleavings, so the check is not vacuous."""
import itertools

# A version word: bits 0..15 count words in transit, bits 16..31 count
# finished moves (modulo 2^16: the carry leaves the 32-bit word).
MOVE = 1 << 16
TRANSIT = MOVE - 1
WORD = (1 << 32) - 1


STASH = 2  # the stash, as a third place K can be


def chain_steps(moves, marks="key"):
    """Steps of one chain that moves K along `moves` = [(src, dst), ...].
    marks: "key" marks K's BitHash1 bucket (0), "src" the bucket K leaves,
    None leaves the versions alone."""
    steps = []
    for src, dst in moves:
        m = 0 if marks == "key" else src
        if marks:
            steps.append(("mark", m))
        steps.append(("out", src))
        steps.append(("in", dst))
        if marks:
            steps.append(("unmark", m))
    return steps


READER = [("v0",), ("probe", 0), ("probe", 1), ("probe", STASH), ("v1",)]


def run(order, writer, start, ver0=0):
    """Execute one interleaving; returns the lookup's verdict."""
    where = {start}
    ver = [ver0, 0, 0]
    wi = ri = 0
    found = False
    v_before = v_after = None
    for who in order:
        if who == "w":
            op, b = writer[wi]
            wi += 1
            if op == "mark":
                ver[b] = (ver[b] + 1) & WORD
            elif op == "unmark":
                ver[b] = (ver[b] + MOVE - 1) & WORD
            elif op == "out":
                where.discard(b)
            else:
                where.add(b)
        else:
            step = READER[ri]
            ri += 1
            if step[0] == "v0":
                v_before = ver[0]
            elif step[0] == "probe":
                found |= step[1] in where
            else:
                v_after = ver[0]
    if found:
        return "hit"
    quiet = (v_before & TRANSIT) == 0 and v_before == v_after
    return "miss" if quiet else "retry"


def verdicts(writer, start, ver0=0):
    n_w, n_r = len(writer), len(READER)
    out = set()
    for pos in itertools.combinations(range(n_w + n_r), n_r):
        order = ["w"] * (n_w + n_r)
        for p in pos:
            order[p] = "r"
        out.add(run(order, writer, start, ver0))
    return out


def test_one_move_never_loses_the_key():
    # K moves from bucket 0 to bucket 1 while the lookup runs
    assert "miss" not in verdicts(chain_steps([(0, 1)]), start=0)


def test_two_moves_never_lose_the_key():
    # K moves 0 -> 1 and later back 1 -> 0 (two steps of chains)
    assert "miss" not in verdicts(chain_steps([(0, 1), (1, 0)]), start=0)


def test_moves_from_the_other_bucket_never_lose_the_key():
    # K starts in its BitHash2 bucket and moves 1 -> 0 -> 1
    assert "miss" not in verdicts(chain_steps([(1, 0), (0, 1)]), start=1)


def test_a_move_into_the_stash_never_loses_the_key():
    # a chain that gives up puts the word it holds in the stash
    assert "miss" not in verdicts(chain_steps([(0, 1), (1, STASH)]), start=0)
    assert "miss" not in verdicts(chain_steps([(1, STASH)]), start=1)


def test_every_probe_order_is_also_safe():
    global READER
    saved = READER
    try:
        for probes in itertools.permutations([0, 1, STASH]):
            READER = [("v0",)] + [("probe", b) for b in probes] + [("v1",)]
            for start, moves in ((0, [(0, 1), (1, 0)]), (1, [(1, 0), (0, STASH)])):
                assert "miss" not in verdicts(chain_steps(moves), start=start), probes
    finally:
        READER = saved


def test_without_marks_a_key_can_be_lost():
    assert "miss" in verdicts(chain_steps([(0, 1)], marks=None), start=0)


def test_marks_on_the_left_bucket_miss_with_one_version_read():
    # marking the bucket K leaves is not enough when the lookup reads only
    # bucket 0's version: a move out of bucket 1 goes unseen
    assert "miss" in verdicts(chain_steps([(1, 0), (0, 1)], marks="src"), start=1)


def test_a_quiet_table_gives_hits():
    assert verdicts([], start=0) == {"hit"}


def test_the_move_counter_wraps_without_touching_the_transit_count():
    # a version whose move counter is about to wrap: a move during the
    # lookup is still caught, and once the move is over a lookup of an absent
    # key settles (a carry into the transit count would make every later
    # lookup retry for ever)
    near = (MOVE - 1) * MOVE
    assert "miss" not in verdicts(chain_steps([(0, 1), (1, 0)]), start=0, ver0=near)
    # another key's move, sharing version word 0, finishes before a lookup of
    # an absent key (kept at a place no lookup probes)
    other = [("mark", 0), ("unmark", 0)]
    done_first = run(["w"] * len(other) + ["r"] * len(READER), other, start=99, ver0=near)
    assert done_first == "miss"
    # after 2^16 finished moves on one word the transit count is still 0
    v = 0
    for _ in range(MOVE + 3):
        v = (v + 1) & WORD
        v = (v + MOVE - 1) & WORD
    assert v & TRANSIT == 0
