"""Model check, on CPU, of slot ownership in the single-kernel batch: why a
claim may publish its word with a plain store while erases and eviction
chains run beside it.

One bucket slot holds word X; its free bit is clear.  Three actors run at
once (each step below is one atomic action):

* an eraser of X: CAS(slot, X -> EMPTY), and if that succeeded, set the free
  bit (Algorithm 4);
* a claimer of a new word N: fetch_and the free bit, and if the bit was set,
  store N (Algorithm 2 with a plain publishing store);
* an eviction chain carrying word Y: read the slot, and if it held a word w
  (not EMPTY), swap Y in with CAS(slot, w -> Y), taking w in hand.

Every interleaving is enumerated.  At the end, every word must be exactly
once in the slot, in the chain's hand, or erased (X only); the claimer's N
must be in the slot or the chain's hand if the claim succeeded.  With the
chain's swap as an unconditional exchange instead of a CAS on the word it
read, the same enumeration finds a lost word, so the check is not vacuous.
"""
import itertools

EMPTY = "EMPTY"


def actors(swap):
    eraser = [("e_cas",), ("e_setbit",)]
    claimer = [("c_take",), ("c_store",)]
    chain = [("h_read",), (swap,)]
    return {"e": eraser, "c": claimer, "h": chain}


def run(order, acts):
    st = {"slot": "X", "bit": 0, "erased": False, "e_ok": False, "c_ok": False,
          "h_seen": None, "hand": None, "h_swapped": False}
    pos = {k: 0 for k in acts}
    for who in order:
        step = acts[who][pos[who]][0]
        pos[who] += 1
        if step == "e_cas":
            if st["slot"] == "X":
                st["slot"] = EMPTY
                st["e_ok"] = st["erased"] = True
        elif step == "e_setbit":
            if st["e_ok"]:
                st["bit"] = 1
        elif step == "c_take":
            if st["bit"]:
                st["bit"] = 0
                st["c_ok"] = True
        elif step == "c_store":
            if st["c_ok"]:
                st["slot"] = "N"  # plain store
        elif step == "h_read":
            st["h_seen"] = st["slot"]
        elif step == "h_cas":
            w = st["h_seen"]
            if w != EMPTY and st["slot"] == w:
                st["slot"] = "Y"
                st["hand"] = w
                st["h_swapped"] = True
        elif step == "h_exch":
            if st["h_seen"] != EMPTY:  # the chain saw an occupied slot
                st["hand"] = st["slot"]
                st["slot"] = "Y"
                st["h_swapped"] = True
    return st


def lost_words(st):
    """Words that are nowhere they should be."""
    have = [st["slot"], st["hand"]]
    lost = []
    if not st["erased"] and "X" not in have:
        lost.append("X")
    if st["c_ok"] and "N" not in have:
        lost.append("N")
    if st["h_swapped"] and "Y" not in have:
        lost.append("Y")
    if st["hand"] == EMPTY:
        lost.append("EMPTY in hand")
    if have.count("X") > 1 or have.count("N") > 1 or have.count("Y") > 1:
        lost.append("duplicate")
    return lost


def interleavings(acts):
    names = sorted(acts)
    seq = [n for n in names for _ in acts[n]]
    seen = set()
    for order in itertools.permutations(seq):
        if order in seen:
            continue
        seen.add(order)
        yield order


def outcomes(swap):
    acts = actors(swap)
    return [(o, run(o, acts)) for o in interleavings(acts)]


def test_cas_swap_and_plain_store_claims_lose_no_word():
    res = outcomes("h_cas")
    assert len(res) == 90  # 6! / (2! 2! 2!) interleavings
    for order, st in res:
        assert not lost_words(st), (order, st)


def test_the_claim_only_stores_into_an_empty_slot():
    for order, st in outcomes("h_cas"):
        acts = actors("h_cas")
        # replay up to the claimer's store and look at the slot it overwrites
        pos = {k: 0 for k in acts}
        s = {"slot": "X", "bit": 0, "erased": False, "e_ok": False, "c_ok": False,
             "h_seen": None, "hand": None, "h_swapped": False}
        prefix = []
        for who in order:
            step = acts[who][pos[who]][0]
            pos[who] += 1
            if step == "c_store" and s["c_ok"]:
                assert s["slot"] == EMPTY, (prefix, s)
            prefix.append(who)
            s = run(prefix, acts)


def test_an_exchanging_chain_can_lose_a_word():
    # the phased eviction kernel swaps with an exchange; that is safe only
    # where no erase runs beside it
    assert any(lost_words(st) for _, st in outcomes("h_exch"))
