"""Writes the regression fixtures of tests/golden/ from the CPU oracle only.

  bithash.txt   BitHash1 / BitHash2 (Section III-C, Listing 1, without the
                final reduction) and the linear-hashing address (Section
                IV-C) of 64 fixed keys at three (M, p) states.
  ops.txt       a fixed op stream of 96 inserts / finds / erases (Section
                III-D) applied in order to the oracle dictionary: per-op
                status and value.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
KEYS = [0, 1, 2, 3, 7, 8, 15, 16, 31, 32, 63, 64, 255, 256, 1023, 1024, 65535, 65536,
        0x7FFFFFFF, 0x80000000, 0xDEADBEEF, 0xCAFEBABE, 0x12345678, 0x9E3779B9,
        0xFFFFFFFD] + [(i * 2654435761) & 0xFFFFFFFF for i in range(1, 40)]
STATES = [(1023, 0), (1023, 511), (32767, 100)]  # (M, p)


def ops_stream():
    """Inserts of 40 keys, a re-insert of 8 with new values, finds of 24
    (16 present, 8 absent), erases of 16 (12 present, 4 absent), all in one
    fixed order; keys are distinct across updates except the re-inserts,
    which run as separate ops of the same stream (the oracle applies ops in
    order)."""
    keys = [(i * 40503 + 17) & 0xFFFFFFFF for i in range(1, 49)]
    ops = []
    for i in range(40):
        ops.append((0, keys[i], (i * 7919) & 0xFFFFFFFF))
    for i in range(8):
        ops.append((0, keys[i * 3], 1000 + i))
    for i in range(16):
        ops.append((1, keys[i * 2], 0))
    for i in range(8):
        ops.append((1, keys[40 + i], 0))
    for i in range(12):
        ops.append((2, keys[i * 3 + 1], 0))
    for i in range(4):
        ops.append((2, keys[44 + i], 0))
    for i in range(8):  # finds after the erases
        ops.append((1, keys[i * 3 + 1], 0))
    return ops


def main():
    with open(os.path.join(HERE, "bithash.txt"), "w") as f:
        f.write("# key bithash1 bithash2 then lh_address of each hash at (M,p) = "
                + " ".join(f"({M},{p})" for M, p in STATES) + "\n")
        f.write("# written by tests/golden/make_golden.py from oracle/ (Listing 1; Section IV-C)\n")
        for k in KEYS:
            h1, h2 = oracle.bithash1(k), oracle.bithash2(k)
            addr = [oracle.lh_address(h, M, p) for M, p in STATES for h in (h1, h2)]
            f.write(" ".join(str(x) for x in [k, h1, h2] + addr) + "\n")
    ops = ops_stream()
    d = oracle.Dict()
    o = np.array([x[0] for x in ops], np.uint8)
    k = np.array([x[1] for x in ops], np.uint32)
    v = np.array([x[2] for x in ops], np.uint32)
    ev, est = d.execute(o, k, v)
    with open(os.path.join(HERE, "ops.txt"), "w") as f:
        f.write("# op key value -> status value_out (ops 0 insert, 1 find, 2 erase; Section III-D)\n")
        f.write("# written by tests/golden/make_golden.py from oracle/ (the dictionary applied in order)\n")
        for i in range(len(ops)):
            f.write(f"{o[i]} {k[i]} {v[i]} {est[i]} {ev[i]}\n")


if __name__ == "__main__":
    main()
