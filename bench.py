#!/usr/bin/env python
"""Benchmark of the Hive hash table on GB300: Gops/s for bulk insert, find and
mixed batches at 95% load on one fixed 2^26-slot table.

One step = clear the table, bulk-insert 63,753,421 unique uniform keys (95% of
2^26 slots), run 2^26 finds at a 50% hit rate, then a mixed batch of 2^24 ops
(insert:find:erase = 1:2:1, new keys / live keys / live keys) that holds the load
at 95%.  Value = all ops of the step / step time.  Inputs and the 512 MiB table
are larger than L2, so nothing is flushed between steps.

Multi-GPU: one process per GPU, each holding its own shard (an independent
table with its own seeded keys); no data-path collective ("scaling": "weak").

``--impl reference`` runs the CPU oracle (a plain single-threaded dictionary)
on a bounded sample of the same workload, as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gops/s insert/find/mixed at 95% load"
SLOTS = 1 << 26
LOAD = (19, 20)
N_FIND = 1 << 26
N_MIXED = 1 << 24
SEED = 2
L2_BYTES = 129 * 10**6  # GB300 L2
# configurations the benchmark's tuner chooses among (fixed table, 95% load)
BENCH_SPACE = {"bucket_slots": [16, 32], "placement": [0], "max_evictions": [16],
               "block_threads": [128, 256, 512], "l2_persist": [0, 1]}
KERNEL_SRC = os.path.join(ROOT, "paper_2510_15095_gb300", "csrc", "hive_kernels.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--slots", type=int, default=SLOTS)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE,
                    help="inserts (and as many finds) in the CPU oracle sample")
    ap.add_argument("--no-tables", action="store_true", help="skip the multi-table leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-resize", action="store_true", help="skip the resize-stream leg")
    ap.add_argument("--bucket-slots", type=int, choices=[16, 32], default=0,
                    help="fix the bucket width instead of autotuning it (profiling runs)")
    ap.add_argument("--l2-persist", type=int, choices=[-1, 0, 1], default=-1,
                    help="fix the persisting L2 window of the free masks (-1: autotuned)")
    ap.add_argument("--block-threads", type=int, choices=[0, 128, 256, 512], default=0,
                    help="fix the bulk kernels' block shape (0: autotuned)")
    ap.add_argument("--no-cpu-parallel", action="store_true",
                    help="skip the parallel CPU baseline (whole step on all host cores)")
    ap.add_argument("--no-breakdown", action="store_true",
                    help="skip the insertion-step breakdown against load factor")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the load-factor sweep and the L2-resident small-table leg")
    ap.add_argument("--resize-batches", type=int, default=32)
    ap.add_argument("--resize-full", action="store_true",
                    help="the whole resize trajectory: 159 growth + 159 shrink batches of 2^22 "
                         "ops, 2^20 -> about 2^27 live keys and back (several minutes)")
    ap.add_argument("--tables-n", type=int, default=1024)
    ap.add_argument("--tables-steps", type=int, default=8)
    ap.add_argument("--serving-requests", type=int, default=3000)
    ap.add_argument("--serving-preload-log2", type=int, default=22,
                    help="keys preloaded into each of the 64 served tables (log2)")
    ap.add_argument("--serving-max-log2", type=int, default=25,
                    help="growth limit of each served table in slots (log2)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(seed: int, slots: int):
    from paper_2510_15095_gb300 import workload as W
    w = W.fill_and_query(seed=seed, slots=slots, load_num=LOAD[0], load_den=LOAD[1],
                         n_find=N_FIND if slots == SLOTS else slots)
    n_mixed = N_MIXED if slots == SLOTS else max(slots // 4, 64)
    rng = np.random.default_rng(seed + 77)
    n_ins = n_mixed // 4
    n_er = n_mixed // 4
    n_fd = n_mixed - n_ins - n_er
    # new keys: counters beyond the insert keys and the absent query keys
    new, _ = W.take_keys(seed, 1 << 31, n_ins)
    ops, keys, vals = W.mixed_batch(rng, w["insert_keys"], new, n_ins, n_er, n_fd, seed=seed)
    w.update({"mix_ops": ops, "mix_keys": keys, "mix_vals": vals})
    return w


def workload_config(w, slots):
    n_ins = int(w["insert_keys"].size)
    return {
        "workload": (f"fixed table of {slots} slots; bulk insert {n_ins} unique "
                     f"uniform u32 keys (95% load), {w['find_keys'].size} finds at 50% hit "
                     f"(uniform), mixed batch of {w['mix_ops'].size} ops insert:find:erase 1:2:1 "
                     "at 95% load"),
        "slots": slots, "load": LOAD[0] / LOAD[1], "n_insert": n_ins,
        "n_find": int(w["find_keys"].size), "n_mixed": int(w["mix_ops"].size),
        "key_dist": "uniform u32 in [1, 2^32-3], unique per batch", "seed": SEED,
        "l2": l2_note(slots * 8),
    }


def l2_note(table_bytes: int) -> str:
    """How the timed steps relate to the 129 MB L2 (nothing is flushed)."""
    mib = table_bytes / (1 << 20)
    if table_bytes > L2_BYTES:
        return f"no flush: {mib:g} MiB table and inputs exceed the 129 MB L2"
    return f"no flush: the {mib:g} MiB table fits in the 129 MB L2 (an L2-resident case)"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,temperature.gpu")

    def __init__(self, gpu_id: str):
        self.path = tempfile.mktemp(prefix="clk_", suffix=".csv")
        self.f = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, temp, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
            if len(parts) > 7:
                try:
                    temp.append(float(parts[7]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
               "reasons": sorted(reasons)}
        if temp:
            out["temp_c_max"] = max(temp)
        return out


def gpu_select(torch, dev) -> str:
    """nvidia-smi -i argument for this process's GPU (UUID when available)."""
    import re
    u = str(getattr(torch.cuda.get_device_properties(dev), "uuid", ""))
    m = re.search(r"[0-9a-fA-F]{8}-[0-9a-fA-F]{4}-[0-9a-fA-F]{4}-[0-9a-fA-F]{4}-[0-9a-fA-F]{12}", u)
    if m:
        return "GPU-" + m.group(0)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        return vis.split(",")[dev.index].strip()
    return str(dev.index)


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    try:
        sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
        for line in open(TRAFFIC_FILE):
            if line.startswith("#") or "=" not in line:
                continue
            kv = dict(tok.split("=", 1) for tok in line.split())
            if kv.get("kernel") == kernel and kv.get("source_sha") == sha:
                return float(kv["bytes_per_launch"]), kv
    except Exception:
        pass
    return None, None


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

CPU_SAMPLE = 1 << 21  # inserts per oracle sample (and as many finds, a quarter as many mixed ops)


def host_info() -> dict:
    """The host the oracle runs on: logical CPUs and the CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"cpus": os.cpu_count(), "model": model or platform.machine()}


def cpu_parallel_leg(w):
    """A parallel CPU baseline, labelled apart from the oracle: the whole bench
    step (every insert, find and mixed op of the workload) on all host cores,
    the dictionary sharded by key over one std::unordered_map per thread
    (oracle.sharded_step).  Its insert statuses and find flags are checked
    against the workload's own expectations."""
    import oracle
    threads = os.cpu_count() or 1
    sec, ist, fv, ff, mvo, mst = oracle.sharded_step(
        threads, w["insert_keys"], w["insert_vals"], w["find_keys"], w["mix_ops"], w["mix_keys"],
        w["mix_vals"])
    ops = ist.size + ff.size + mst.size
    ok = bool((ist == oracle.INSERTED).all() and np.array_equal(ff.astype(bool), w["is_hit"]))
    return {"value": ops / sec / 1e9, "unit": "Gops/s", "threads": threads,
            "kind": "sharded std::unordered_map (a CPU baseline, not the oracle)",
            "sample": f"the whole step: {ist.size} inserts, {ff.size} finds, {mst.size} mixed ops",
            "seconds": sec, "results_as_expected": ok, "host": host_info()}


def oracle_sample(w, n_sample: int):
    """Time the oracle on a prefix sample: n inserts, n finds, n/4 mixed ops."""
    import oracle
    d = oracle.Dict()
    ins_k = w["insert_keys"][:n_sample]
    ins_v = w["insert_vals"][:n_sample]
    fk = w["find_keys"][:n_sample]
    nm = min(n_sample // 4, w["mix_ops"].size)
    t0 = time.perf_counter()
    d.insert(ins_k, ins_v)
    d.find(fk)
    d.execute(w["mix_ops"][:nm], w["mix_keys"][:nm], w["mix_vals"][:nm])
    dt = time.perf_counter() - t0
    ops = ins_k.size + fk.size + nm
    return ops, dt


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# multi-rank bookkeeping: independent shards, slowest rank's time
# ---------------------------------------------------------------------------

def shard_seed(rank: int) -> int:
    """Each rank owns an independent shard: its own seeded keys and table."""
    return SEED + rank


def max_over_ranks(torch, dist, x: float, world: int, device) -> float:
    """The slowest rank's time (no data-path collective: timing only)."""
    if world <= 1:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gops(ops_per_rank_step: int, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput: the ops all ranks processed over the slowest
    rank's time (weak scaling: the per-rank work is fixed)."""
    return ops_per_rank_step * steps * world / (ms / 1e3) / 1e9


def run_reference(args, rank):
    if rank != 0:
        return
    w = make_workload(SEED, args.slots)
    # each step times the same prefix sample as the own arm's cpu_baseline
    # (about a second of single-threaded work per step)
    n = min(args.cpu_sample, w["insert_keys"].size)
    for _ in range(args.warmup):
        oracle_sample(w, n)
    times, ops = [], 0
    for _ in range(args.steps):
        ops, dt = oracle_sample(w, n)
        times.append(dt)
    v = ops * len(times) / sum(times) / 1e9
    sample = (f"prefix sample per step: {n} inserts, {n} finds, {n // 4} mixed ops "
              f"of the {args.slots}-slot workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gops/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(w, args.slots),
            "cpu_baseline": {"value": v, "unit": "Gops/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": v, "unit": "Gops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# multi-table leg: many independent tables, one batched launch per step
# ---------------------------------------------------------------------------

def tables_leg(torch, H, dev, n_tables=1024, steps=8, seed=40):
    """1024 resizable tables with initial capacities log-uniform in
    [2^10, 2^22] slots, preloaded to half load; per step every table gets a
    mixed batch of log-uniform [2^6, 2^20] ops (insert:find:erase 2:1:1).
    The same steps run once as one multi-table batch per step (CUDA graph
    replay) and once as one hive_execute per table per step, on two equal sets
    of tables; outputs must be identical.  The same two arms also run on
    fixed-capacity tables sized for every insert of the run: a fixed table's
    hive_execute never waits for the GPU, so that plain arm measures launch
    cost without the resizable arm's per-call size read-back."""
    from paper_2510_15095_gb300 import autotune as AT
    from paper_2510_15095_gb300 import workload as W
    rng = np.random.default_rng(seed)
    caps = (np.exp(rng.uniform(10, 22, n_tables) * np.log(2)).astype(np.int64) // 32 + 1) * 32
    nops = np.exp(rng.uniform(6, 20, (steps, n_tables)) * np.log(2)).astype(np.int64)
    # knobs from the autotuner for this class: resizable tables of up to 2^22
    # slots served in multi-table batches, 2:1:1
    tuned = AT.tune(1 << 22, 90, (2, 1, 1), True, multi=True)
    K = int(tuned.get("resize_batch", 1024))
    knobs = {"max_evictions": int(tuned.get("max_evictions", 16)),
             "placement": int(tuned.get("placement", 0)),
             "bucket_slots": int(tuned.get("bucket_slots", 32))}
    ins_total = nops.sum(axis=0) // 2
    max_slots = caps + (ins_total * 10 // 9) + caps // 2 + 64 * K
    sets = []
    for arm in range(4):  # resizable batched, resizable plain, fixed batched, fixed plain
        tabs = []
        for t in range(n_tables):
            if arm < 2:
                tb = H.HiveTable(int(caps[t]), max_slots=int(max_slots[t]), resizable=True,
                                 resize_batch=K, **knobs)
            else:
                tb = H.HiveTable(int(max_slots[t]), **knobs)
            k, v = W.preload_t(torch, 7000 + t, int(caps[t]) // 2, dev)
            tb.insert(k, v, status=False)
            tabs.append(tb)
        sets.append(tabs)
    counts = [int(c) // 2 for c in caps]
    work = []
    for st in range(steps):
        row = []
        for t in range(n_tables):
            ops, keys, vals, counts[t], n_ins = W.mixed_step_t(torch, 7000 + t, counts[t],
                                                                int(nops[st, t]), dev, salt=st)
            row.append((ops, keys, vals, n_ins))
        work.append(row)
    outs = [[(torch.empty(w[1].numel(), dtype=torch.int32, device=dev),
              torch.empty(w[1].numel(), dtype=torch.uint8, device=dev)) for w in row] for row in work]
    max_ops = int(nops.sum(axis=1).max()) + 1

    def batched(tabs, out):
        multi = H.HiveMulti(tabs, max_segments=n_tables, max_ops=max_ops, use_graph=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for st in range(steps):
            multi.execute([{"table": t, "ops": w[0], "keys": w[1], "vals": w[2], "n_insert": w[3],
                            "vals_out": out[st][t][0], "status": out[st][t][1]}
                           for t, w in enumerate(work[st])])
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        multi.close()
        return dt

    def plain(tabs):
        res = []
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for st in range(steps):
            for t, w in enumerate(work[st]):
                res.append(tabs[t].execute(w[0], w[1], w[2]))
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, res

    p0 = sum(tb.stats()["probes"] for tb in sets[0])
    c0 = sum(tb.stats()["claimed_fast"] + tb.stats()["claimed_slow"] for tb in sets[0])
    t_multi = batched(sets[0], outs)
    probes = sum(tb.stats()["probes"] for tb in sets[0]) - p0
    claims = sum(tb.stats()["claimed_fast"] + tb.stats()["claimed_slow"] for tb in sets[0]) - c0
    t_plain, plain_out = plain(sets[1])
    outs_fixed = [[(torch.empty_like(o[0]), torch.empty_like(o[1])) for o in row] for row in outs]
    t_multi_fixed = batched(sets[2], outs_fixed)
    t_plain_fixed, plain_fixed_out = plain(sets[3])

    def same_as(res):
        return all(torch.equal(outs[st][t][0], res[st * n_tables + t][0]) and
                   torch.equal(outs[st][t][1], res[st * n_tables + t][1])
                   for st in range(steps) for t in range(n_tables))
    same = same_as(plain_out) and same_as(plain_fixed_out) and all(
        torch.equal(outs[st][t][i], outs_fixed[st][t][i])
        for st in range(steps) for t in range(n_tables) for i in range(2))
    caps_same = all(a.capacity() == b.capacity() for a, b in zip(sets[0], sets[1]))
    ops_total = int(nops.sum())
    # step-level algorithmic bytes of the batched resizable arm (op I/O, every
    # probed bucket, a written sector per claimed slot) over its wall time
    S = knobs["bucket_slots"]
    byts = 14 * ops_total + 8 * S * probes + 32 * claims
    peak_gbs, peak_kind = measured_peak()
    for tabs in sets:
        for tb in tabs:
            tb.close()
    return {"workload": (f"{n_tables} resizable tables, capacities log-uniform 2^10-2^22 slots "
                         f"(half full), {steps} steps of log-uniform 2^6-2^20 ops per table "
                         "(insert:find:erase 2:1:1)"),
            "ops": ops_total, "batched_gops": ops_total / t_multi / 1e9,
            "plain_gops": ops_total / t_plain / 1e9, "speedup": t_plain / t_multi,
            "batched_s": t_multi, "plain_s": t_plain,
            "fixed_tables": {"batched_gops": ops_total / t_multi_fixed / 1e9,
                             "plain_gops": ops_total / t_plain_fixed / 1e9,
                             "speedup": t_plain_fixed / t_multi_fixed},
            "roofline": {"bound": "hbm", "algorithmic_bytes": byts,
                         "achieved": byts / t_multi / 1e9, "peak": peak_gbs, "unit": "GB/s",
                         "frac": byts / t_multi / 1e9 / peak_gbs, "peak_source": peak_kind,
                         "probes_per_op": probes / ops_total,
                         "note": "batched resizable arm, whole steps by host wall clock; most "
                                 "of the 1024 tables fit in L2"},
            "identical_results": bool(same),
            "identical_capacity": bool(caps_same), "graph": True,
            "tuned": {"resize_batch": K, **knobs}}


# ---------------------------------------------------------------------------
# single-kernel mixed batches against the phased launches
# ---------------------------------------------------------------------------

def fused_leg(torch, H, dev, t, ik, iv, mo, mk, mv, reps=3, small=4096, n_small=256):
    """The bench's mixed batch at 95% load run as one concurrent kernel
    (hive_execute_fused) and as the phased launches (hive_execute): whole
    batch, and as `n_small` consecutive slices of `small` ops (latency-bound
    small batches).  Results must be identical."""
    stream = torch.cuda.current_stream(dev)

    def restore():
        t.clear()
        t.insert(ik, iv, status=False)

    out = {"workload": (f"mixed batch of {mo.numel()} ops (insert:find:erase 1:2:1) at 95% load, "
                        f"whole and as {n_small} slices of {small} ops")}
    res = {}
    for name, fused in (("phased", False), ("fused", True)):
        restore()
        res[name] = t.execute(mo, mk, mv, fused=fused)
        ms = _median_ms(torch, stream, dev, lambda: t.execute(mo, mk, mv, fused=fused), reps,
                        setup=restore)
        out[f"{name}_gops"] = mo.numel() / ms / 1e6
        out[f"{name}_ms"] = ms
        m = min(n_small * small, mo.numel())

        def slices():
            for j in range(0, m, small):
                t.execute(mo[j:j + small], mk[j:j + small], mv[j:j + small], fused=fused)
        ms_s = _median_ms(torch, stream, dev, slices, reps, setup=restore)
        out[f"{name}_small_batch_us"] = ms_s * 1e3 / (m // small)
        out[f"{name}_small_gops"] = m / ms_s / 1e6
    out["identical_results"] = bool(torch.equal(res["phased"][0], res["fused"][0]) and
                                    torch.equal(res["phased"][1], res["fused"][1]))
    assert out["identical_results"], "fused and phased mixed batches disagree"
    restore()
    before = t.stats()["fused_retries"]
    t.execute(mo, mk, mv, fused=True)
    out["lookup_retries"] = t.stats()["fused_retries"] - before
    return out


# ---------------------------------------------------------------------------
# 32-bit entries: a key-only set with 128-byte buckets
# ---------------------------------------------------------------------------

def hive32_leg(torch, H, dev, slots=SLOTS, n_find=N_FIND, seed=90, reps=3):
    """The load-factor-sweep table with 32-bit entries (a set of 32-bit keys,
    32 slots per 128-byte bucket): bulk insert to 95% load, n_find finds at 50%
    hit, and a mixed batch of slots / 4 ops (insert:find:erase 1:2:1)."""
    from paper_2510_15095_gb300 import workload as W
    stream = torch.cuda.current_stream(dev)
    n = (slots * 19 * 2 + 20) // 40
    k32 = _i32(torch, _valid_keys_t(torch, W, seed, 0, n, dev))
    a32 = _i32(torch, _valid_keys_t(torch, W, seed, 1 << 31, n_find, dev))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hit = torch.rand(n_find, generator=g, device=dev) < 0.5
    q = torch.where(hit, k32[torch.randint(0, n, (n_find,), generator=g, device=dev)],
                    a32[torch.randint(0, n_find, (n_find,), generator=g, device=dev)])
    n_mix = slots // 4
    perm = torch.randperm(n, generator=g, device=dev)
    new = _i32(torch, _valid_keys_t(torch, W, seed, 1 << 30, n_mix // 4, dev))
    keys_m = torch.cat([new, k32[perm[: n_mix // 4]], k32[perm[n_mix // 4: n_mix // 4 + n_mix // 2]]])
    ops_m = torch.cat([torch.zeros(n_mix // 4, dtype=torch.uint8, device=dev),
                       torch.full((n_mix // 4,), 2, dtype=torch.uint8, device=dev),
                       torch.ones(n_mix // 2, dtype=torch.uint8, device=dev)])
    order = torch.randperm(keys_m.numel(), generator=g, device=dev)
    keys_m, ops_m = keys_m[order].contiguous(), ops_m[order].contiguous()
    t = H.Hive32Table(slots, H.KEY_ONLY)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    fv = torch.empty(n_find, dtype=torch.int32, device=dev)
    ff = torch.empty(n_find, dtype=torch.uint8, device=dev)
    ins_ms = _median_ms(torch, stream, dev, lambda: t.insert(k32, status=st), reps, setup=t.clear)
    assert bool((st == H.INSERTED).all()) and t.check() == 0
    s0 = t.stats()["probes"]
    t.find(q, vals_out=fv, found=ff)
    probes = (t.stats()["probes"] - s0) / n_find
    f_ms = _median_ms(torch, stream, dev, lambda: t.find(q, vals_out=fv, found=ff), reps)
    assert bool(((ff == 1) == hit).all())

    def restore():
        t.clear()
        t.insert(k32, status=False)
    m_ms = _median_ms(torch, stream, dev, lambda: t.execute(ops_m, keys_m), reps, setup=restore)
    assert t.check() == 0
    t.close()
    return {"workload": (f"fixed table of {slots} slots with 32-bit entries (key-only set, 128-byte "
                         f"buckets): insert {n} keys (95% load), {n_find} finds at 50% hit, mixed "
                         f"batch of {n_mix} ops 1:2:1"),
            "insert_gops": n / ins_ms / 1e6, "find_gops": n_find / f_ms / 1e6,
            "mixed_gops": n_mix / m_ms / 1e6, "probes_per_find": probes,
            # key in, value + flag out, 128 bytes per probed bucket
            "find_algorithmic_gbs": n_find * (9 + 128 * probes) / f_ms / 1e6,
            "insert_algorithmic_gbs": n * (4 + 1 + 2 * 128 + 32) / ins_ms / 1e6,
            "ms": {"insert": ins_ms, "find": f_ms, "mixed": m_ms}}


# ---------------------------------------------------------------------------
# load-factor sweep and the L2-resident small table
# ---------------------------------------------------------------------------

def _valid_keys_t(torch, W, seed, pos0, n, dev):
    """The first n keys of stream `seed` from position pos0 on that are not
    reserved (0, 0xFFFFFFFE, 0xFFFFFFFF), as int64 tensors in [1, 2^32 - 3]."""
    pos = torch.arange(pos0, pos0 + n + 64, device=dev, dtype=torch.int64)
    k = W.feistel_bits_t(pos, seed, 32)
    k = k[(k >= 1) & (k <= 0xFFFFFFFD)][:n]
    assert k.numel() == n
    return k


def _i32(torch, t):
    return (t - ((t >> 31) << 32)).to(torch.int32)


def _median_ms(torch, stream, dev, fn, reps, setup=None):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        if setup is not None:
            setup()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out.append(e0.elapsed_time(e1))
    return float(np.median(out))


def sweep_leg(torch, H, dev, table_kw, slots=SLOTS, n_find=N_FIND, seed=70, reps=3):
    """Load-factor sweep on a fixed table of `slots` slots (the paper's
    insert/find experiment over load factors): fresh bulk fills to 50/80/90/95%
    load, the incremental fill from 90% to 95%, and n_find finds at 50% hit at
    each load, with hits and misses drawn uniformly or Zipf(0.99) over ranks."""
    from paper_2510_15095_gb300 import workload as W
    stream = torch.cuda.current_stream(dev)
    loads = (50, 80, 90, 95)
    n_at = {L: (slots * L * 2 + 100) // 200 for L in loads}
    k = _valid_keys_t(torch, W, seed, 0, n_at[95], dev)
    v = W.splitmix32_t(k ^ seed)
    a = _valid_keys_t(torch, W, seed, 1 << 31, n_find, dev)  # never inserted
    k32, v32, a32 = _i32(torch, k), _i32(torch, v), _i32(torch, a)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hit = torch.rand(n_find, generator=g, device=dev) < 0.5
    st = torch.empty(n_at[95], dtype=torch.uint8, device=dev)
    fv = torch.empty(n_find, dtype=torch.int32, device=dev)
    ff = torch.empty(n_find, dtype=torch.uint8, device=dev)
    t = H.HiveTable(slots, **table_kw)
    S = int(table_kw.get("bucket_slots", 32))
    out = {"workload": (f"fixed table of {slots} slots; fresh fills to 50/80/90/95% load and the "
                        f"90->95% fill; {n_find} finds at 50% hit, uniform and Zipf(0.99) over ranks"),
           "table": dict(table_kw), "loads": {}}
    for L in loads:
        n = n_at[L]
        ins_ms = _median_ms(torch, stream, dev, lambda: t.insert(k32[:n], v32[:n], status=st[:n]),
                            reps, setup=t.clear)
        assert bool((st[:n] == H.INSERTED).all()) and t.check() == 0
        row = {"n_insert": n, "insert_gops": n / ins_ms / 1e6, "insert_ms": ins_ms}
        for dist_name in ("uniform", "zipf"):
            if dist_name == "uniform":
                hi = torch.randint(0, n, (n_find,), generator=g, device=dev)
                mi = torch.randint(0, n_find, (n_find,), generator=g, device=dev)
            else:
                hi = W.zipf_ranks_t(torch, n, 0.99, n_find, g, dev) - 1
                mi = W.zipf_ranks_t(torch, min(n, n_find), 0.99, n_find, g, dev) - 1
            q = torch.where(hit, k32[hi], a32[mi])
            before = t.stats()["probes"]
            t.find(q, vals_out=fv, found=ff)
            probes = (t.stats()["probes"] - before) / n_find
            f_ms = _median_ms(torch, stream, dev, lambda: t.find(q, vals_out=fv, found=ff), reps)
            assert bool(((ff == 1) == hit).all())
            assert bool((fv[hit] == v32[hi[hit]]).all())
            row[f"find_{dist_name}_gops"] = n_find / f_ms / 1e6
            row[f"find_{dist_name}_probes"] = probes
            row[f"find_{dist_name}_algorithmic_gbs"] = n_find * (9 + 8 * S * probes) / f_ms / 1e6
        out["loads"][str(L)] = row
    n90, n95 = n_at[90], n_at[95]
    inc_ms = _median_ms(torch, stream, dev,
                        lambda: t.insert(k32[n90:n95], v32[n90:n95], status=st[n90:n95]), reps,
                        setup=lambda: (t.clear(), t.insert(k32[:n90], v32[:n90], status=False)))
    assert bool((st[n90:n95] == H.INSERTED).all()) and t.check() == 0
    out["incremental_90_95"] = {"n_insert": n95 - n90, "insert_gops": (n95 - n90) / inc_ms / 1e6,
                                "insert_ms": inc_ms}
    t.close()
    return out


BREAKDOWN_LOADS = (55, 65, 75, 85, 90, 93, 95, 97)
STEP_STATS = ("replaced", "claimed_fast", "overflowed", "claimed_slow", "evict_rounds",
              "lock_acquired", "lock_timeouts", "stashed", "pending", "stash_reinserted")


def breakdown_leg(torch, H, dev, table_kw, slots=SLOTS, seed=75, reps=3):
    """Insertion-step breakdown against load factor (the paper's Section V-D
    analysis, over loads 0.55-0.97).  For each load, a fresh bulk fill of an
    empty fixed table to that load ("fill") and the last 5% of the fill alone
    ("window", from load - 5% on), each timed per kernel with the profiling
    hook's CUDA events and counted per step with the table's counters:

    - steps 1-2 (replace, claim) run in the bulk kernel;
    - step 3 (bounded eviction) is the eviction kernel, which also appends
      the words of chains that gave up to the stash (one atomic each);
    - step 4 (stash) is that append plus the maintenance kernel.

    The phased design runs each step as its own kernel, so the shares are
    kernel times, where the paper sums per-step clock counts inside one
    kernel."""
    from paper_2510_15095_gb300 import workload as W
    stream = torch.cuda.current_stream(dev)
    n_max = (slots * BREAKDOWN_LOADS[-1] + 50) // 100
    k = _valid_keys_t(torch, W, seed, 0, n_max, dev)
    v = W.splitmix32_t(k ^ seed)
    k32, v32 = _i32(torch, k), _i32(torch, v)
    st = torch.empty(n_max, dtype=torch.uint8, device=dev)
    t = H.HiveTable(slots, **table_kw)
    out = {"workload": (f"fixed table of {slots} slots; fresh bulk fills to each load and the "
                        f"last 5% of each fill alone; uniform unique u32 keys"),
           "table": dict(table_kw), "loads": {}}
    kinds = {"steps_1_2": ("insert",), "step_3": ("evict",), "step_4": ("maint",)}

    def one(lo, hi):
        def setup():
            t.clear()
            if lo:
                t.insert(k32[:lo], v32[:lo], status=False)
        runs = []
        for _ in range(reps):
            setup()
            torch.cuda.synchronize(dev)
            before = t.stats()
            t.profile(True)
            t.profile_read()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.insert(k32[lo:hi], v32[lo:hi], status=st[lo:hi])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            prof = t.profile_read()
            t.profile(False)
            after = t.stats()
            runs.append((e0.elapsed_time(e1), prof, {f: after[f] - before[f] for f in STEP_STATS}))
        runs.sort(key=lambda r: r[0])
        ms, prof, cnt = runs[len(runs) // 2]
        n = hi - lo
        steps = {name: sum(prof.get(kk, (0.0, 0))[0] for kk in ks) for name, ks in kinds.items()}
        tot = sum(steps.values()) or 1.0
        inserted = int((st[lo:hi] == H.INSERTED).sum().item())
        code = t.check()
        return {"n_insert": n, "ms": ms, "gops": n / ms / 1e6,
                "kernel_ms": {kk: round(vv, 4) for kk, vv in steps.items()},
                "share": {kk: round(vv / tot, 5) for kk, vv in steps.items()},
                "counts": cnt, "lock_fraction": cnt["lock_acquired"] / n,
                "inserted": inserted, "check": code}

    for L in BREAKDOWN_LOADS:
        hi = (slots * L + 50) // 100
        lo = (slots * (L - 5) + 50) // 100
        out["loads"][str(L)] = {"fill": one(0, hi), "window": one(lo, hi)}
    t.close()
    return out


def plain_leg(torch, H, dev, seed=80, reps=5):
    """The small plain table (2^20 slots, 8 MiB, resident in the 129 MB L2):
    insert 838,861 keys (80%), 1,677,722 finds (half absent), erase a seeded
    half of the keys, the same finds again.  Throughput here is bounded by L2
    and launch latency, not HBM."""
    from paper_2510_15095_gb300 import workload as W
    stream = torch.cuda.current_stream(dev)
    slots, n_ins, n_find = 1 << 20, 838861, 1677722
    k = _valid_keys_t(torch, W, seed, 0, n_ins, dev)
    v = W.splitmix32_t(k ^ seed)
    a = _valid_keys_t(torch, W, seed, 1 << 31, n_find, dev)
    k32, v32, a32 = _i32(torch, k), _i32(torch, v), _i32(torch, a)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hit = torch.rand(n_find, generator=g, device=dev) < 0.5
    q = torch.where(hit, k32[torch.randint(0, n_ins, (n_find,), generator=g, device=dev)],
                    a32[torch.randint(0, n_find, (n_find,), generator=g, device=dev)])
    er = k32[torch.randperm(n_ins, generator=g, device=dev)[: n_ins // 2]]
    t = H.HiveTable(slots)
    S = int(t.config.bucket_slots)
    st = torch.empty(n_ins, dtype=torch.uint8, device=dev)
    fv = torch.empty(n_find, dtype=torch.int32, device=dev)
    ff = torch.empty(n_find, dtype=torch.uint8, device=dev)
    es = torch.empty(n_ins // 2, dtype=torch.uint8, device=dev)
    ins_ms = _median_ms(torch, stream, dev, lambda: t.insert(k32, v32, status=st), reps, setup=t.clear)
    p0 = t.stats()["probes"]
    t.find(q, vals_out=fv, found=ff)
    find_probes = t.stats()["probes"] - p0
    f1_ms = _median_ms(torch, stream, dev, lambda: t.find(q, vals_out=fv, found=ff), reps)
    assert bool(((ff == 1) == hit).all())

    def restore():
        t.clear()
        t.insert(k32, v32, status=False)
    er_ms = _median_ms(torch, stream, dev, lambda: t.erase(er, status=es), reps, setup=restore)
    assert bool((es == H.ERASED).all())
    f2_ms = _median_ms(torch, stream, dev, lambda: t.find(q, vals_out=fv, found=ff), reps)
    assert t.size() == n_ins - n_ins // 2 and t.check() == 0
    t.close()
    return {"workload": ("fixed table of 2^20 slots (L2-resident): insert 838,861, find 1,677,722 "
                         "(half absent), erase 419,430, find again"),
            "insert_gops": n_ins / ins_ms / 1e6, "find_gops": n_find / f1_ms / 1e6,
            "erase_gops": (n_ins // 2) / er_ms / 1e6, "find_after_erase_gops": n_find / f2_ms / 1e6,
            "ms": {"insert": ins_ms, "find": f1_ms, "erase": er_ms, "find_after_erase": f2_ms},
            # bytes served from L2: each insert probes both buckets, each find
            # the buckets it reads (counted by the kernel), plus the op I/O
            "achieved_l2_gbs": {"insert": (9 + 2 * 8 * S + 32) * n_ins / ins_ms / 1e6,
                                "find": (9 * n_find + 8 * S * find_probes) / f1_ms / 1e6},
            "find_probes_per_op": find_probes / n_find}


# ---------------------------------------------------------------------------
# resize-stream leg: one table grows and shrinks through linear hashing
# ---------------------------------------------------------------------------

def resize_leg(torch, H, dev, batches=32, n_batch=1 << 22, seed=60):
    """One resizable table starting with 2^20 live keys; `batches` growth
    batches of 2^22 ops (insert:erase:find 40/20/40) then as many shrink
    batches (20/40/40), finds Zipf(0.99) over live keys, thresholds 0.9/0.4,
    K = 1024.  159 + 159 batches is the whole trajectory to 2^27 live keys
    and back.  The op-weighted roofline counts each op's probed buckets and
    I/O and each split or merge's bucket reads and writes.  At the end a
    sample of live keys must be found with their values and a sample of
    erased ones must not.  Also times single split and merge launches of
    32,768 bucket pairs (the size the paper reports resize throughput on)."""
    from paper_2510_15095_gb300 import workload as W
    start = 1 << 20
    peak_est = start + batches * (n_batch // 5)
    max_slots = 1 << max(27, int(peak_est * 10 // 9 + 1).bit_length())
    t = H.HiveTable(1 << 21, max_slots=max_slots, resizable=True, resize_batch=1024, shrink=(2, 5))
    S = int(t.config.bucket_slots)
    k, v = W.preload_t(torch, seed, start, dev)
    t.insert(k, v, status=False)
    live = torch.arange(start, dtype=torch.int64, device=dev)
    ctr = start
    work = {"grow": [], "shrink": []}
    for phase, fr in (("grow", ((2, 5), (1, 5))), ("shrink", ((1, 5), (2, 5)))):
        for b in range(batches):
            ops, keys, vals, live, ctr = W.stream_step_t(torch, seed, live, ctr, n_batch, dev,
                                                         fr[0], fr[1], 0.99, salt=b)
            work[phase].append((ops, keys, vals))
        if phase == "grow":
            peak = int(live.numel())
    out = {}
    t.profile(True)
    t.profile_read()
    s0 = t.stats()
    t_total = 0.0
    for phase in ("grow", "shrink"):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for w in work[phase]:
            t.execute(*w)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        t_total += dt
        out[f"{phase}_gops"] = batches * n_batch / dt / 1e9
        out[f"{phase}_capacity_slots"] = t.capacity()
    prof = t.profile_read()
    t.profile(False)
    st = t.stats()
    size_end = t.size()
    # op-weighted algorithmic bytes: op I/O (op code, key, value in; value,
    # status out), every probed bucket, a written sector per claimed slot,
    # and per split or merge pair one bucket read and two written
    n_ops = 2 * batches * n_batch
    probes = st["probes"] - s0["probes"]
    claims = (st["claimed_fast"] - s0["claimed_fast"]) + (st["claimed_slow"] - s0["claimed_slow"])
    pairs = (st["splits"] - s0["splits"]) + (st["merges"] - s0["merges"])
    byts = 14 * n_ops + 8 * S * probes + 32 * claims + 3 * 8 * S * pairs
    peak_gbs, peak_kind = measured_peak()
    ach = byts / t_total / 1e9
    out["roofline"] = {"bound": "hbm", "algorithmic_bytes": byts, "achieved": ach,
                       "peak": peak_gbs, "unit": "GB/s", "frac": ach / peak_gbs,
                       "peak_source": peak_kind, "probes_per_op": probes / n_ops,
                       "note": "whole stream by host wall clock, resize launches included"}
    # properties at the end: live keys found with their values, erased keys not
    g = torch.Generator(device=dev)
    g.manual_seed(seed + 5)
    dead = torch.ones(ctr, dtype=torch.bool, device=dev)
    dead[live] = False
    dead_pos = torch.nonzero(dead).flatten()
    nsamp = min(1 << 20, int(live.numel()), int(dead_pos.numel()))
    lp = live[torch.randint(0, live.numel(), (nsamp,), generator=g, device=dev)]
    dp = dead_pos[torch.randint(0, dead_pos.numel(), (nsamp,), generator=g, device=dev)]
    to32 = lambda x: (x - ((x >> 31) << 32)).to(torch.int32)  # noqa: E731
    lk = W.feistel_bits_t(lp, seed, 32)
    lk = lk[lk < 0xFFFFFFFE]  # a reserved key is never stored
    fv, ff = t.find(to32(lk))
    ok_live = bool((ff == 1).all()) and bool(torch.equal(fv, to32(W.splitmix32_t(lk ^ seed))))
    _, fd = t.find(to32(W.feistel_bits_t(dp, seed, 32)))
    ok_dead = bool((fd == 0).all())
    n_live = int((W.feistel_bits_t(live, seed, 32) < 0xFFFFFFFE).sum())
    assert ok_live and ok_dead and size_end == n_live, "resize stream lost keys"
    out["sample_check"] = {"live_found": ok_live, "erased_absent": ok_dead, "sample": nsamp,
                           "size_matches_generator": size_end == n_live}
    t.close()
    # split / merge launches of 32,768 pairs on a table of 32,768 buckets
    m = H.HiveTable(1 << 20, max_slots=1 << 22, resizable=True, resize_batch=32768, shrink=(2, 5))
    k, v = W.preload_t(torch, seed + 1, (1 << 20) * 85 // 100, dev)
    m.insert(k, v, status=False)
    m.profile(True)
    m.profile_read()
    m.reserve(1 << 21)
    sp = m.profile_read()
    m.erase(k[: k.numel() * 45 // 100], status=False)
    mg = m.profile_read()
    m.profile(False)
    m.close()
    split_ms = sp.get("split", (float("nan"), 0))[0]
    merge_ms = mg.get("merge", (float("nan"), 0))[0]
    out.update({
        "workload": (f"one resizable table from 2^20 live keys, {batches} growth + {batches} shrink "
                     "batches of 2^22 ops (40/20/40 then 20/40/40 insert:erase:find, Zipf 0.99 "
                     f"finds), thresholds 0.9 / 0.4, K = 1024, growth limit {max_slots} slots"),
        "peak_live_keys": peak, "end_live_keys": size_end,
        "splits": st["splits"], "merges": st["merges"],
        "kernel_ms": {kk: vv[0] for kk, vv in prof.items()},
        "split_32768_pairs_ms": split_ms, "merge_32768_pairs_ms": merge_ms,
        "split_gbuckets_per_s": 32768 / (split_ms / 1e3) / 1e9,
        # a split reads the source bucket and writes both buckets of the pair
        "split_algorithmic_gbs": 32768 * 3 * 256 / (split_ms / 1e3) / 1e9,
        "merge_gbuckets_per_s": 32768 / (merge_ms / 1e3) / 1e9,
        "split_entries_per_s": (1 << 20) * 0.85 / (split_ms / 1e3),
    })
    return out


# ---------------------------------------------------------------------------
# serving leg: continuous batching vs one launch per request
# ---------------------------------------------------------------------------

SERVING_RATES = (0.25, 0.5, 0.75, 0.9, 1.0, 1.2)  # x the batched server's saturation rate
FIFO_RATES = (0.25, 0.5, 0.75, 0.9)               # x the FIFO reference's own saturation rate


def serving_leg(torch, H, dev, n_tables=64, n_requests=3000, seed=50, preload_log2=22,
                max_slots_log2=25):
    """64 resizable tables preloaded with 2^preload_log2 keys each; requests of
    log-uniform [1, 2^20] ops (insert:erase:find 40/20/40) on uniform random
    tables.  Both servers first run closed-loop (every request available at
    once) for their saturation throughput; then Poisson arrivals sweep the
    batched server over SERVING_RATES x its saturation request rate, and the
    FIFO reference over FIFO_RATES x its own (above its saturation its queue
    only grows).  Every run must give every request the same results."""
    from paper_2510_15095_gb300 import serving as SV
    from paper_2510_15095_gb300 import workload as W
    pre = 1 << preload_log2

    from paper_2510_15095_gb300 import autotune as AT
    tuned = AT.tune(1 << 22, 90, (2, 1, 1), True, multi=True)  # the multi-table leg's class
    knobs = {"bucket_slots": int(tuned.get("bucket_slots", 32)),
             "max_evictions": int(tuned.get("max_evictions", 16)),
             "placement": int(tuned.get("placement", 0))}
    init_slots = 1 << (preload_log2 + 1)

    def fresh():
        tabs = []
        for t in range(n_tables):
            tb = H.HiveTable(init_slots, max_slots=1 << max_slots_log2, resizable=True,
                             resize_batch=int(tuned.get("resize_batch", 1024)), **knobs)
            k, v = W.preload_t(torch, 1000 + t, pre, dev)
            tb.insert(k, v, status=False)
            tabs.append(tb)
        return tabs

    counts = [pre] * n_tables
    base = SV.make_trace(torch, n_tables, n_requests, rate_per_s=1.0, seed=seed, counts=counts,
                         max_log2_ops=20, device=dev)

    def with_arrivals(arr):
        return [SV.Request(r.rid, r.table, float(a), r.ops, r.keys, r.vals, r.n_insert)
                for r, a in zip(base, arr)]

    sizes = {}

    def serve(reqs, fifo):
        tabs = fresh()
        torch.cuda.synchronize(dev)
        if fifo:
            out = SV.run_fifo(tabs, reqs)
        else:
            srv = SV.HiveServer(tabs, hbm_budget_bytes=64e9, max_batch_ops=1 << 23,
                                max_batch_reqs=256, depth=2)
            out = srv.run(reqs)
            srv.close()
        sizes["live"] = [tb.size() for tb in tabs]
        sizes["slots"] = [tb.capacity() for tb in tabs]
        for tb in tabs:
            tb.close()
        return out

    ref, same = [], [True]

    def check(reqs):
        if not ref:
            ref.extend((r.status.clone(), r.vals_out.clone()) for r in reqs)
        else:
            same[0] = same[0] and all(torch.equal(a, r.status) and torch.equal(b, r.vals_out)
                                      for (a, b), r in zip(ref, reqs))
        for r in reqs:
            r.status = r.vals_out = None

    def poisson(rate, salt):
        gaps = np.random.default_rng(seed + salt).exponential(1.0 / rate, n_requests)
        return np.cumsum(gaps) - gaps[0]

    zeros = np.zeros(n_requests)
    reqs = with_arrivals(zeros)
    sat_b = serve(reqs, False)
    check(reqs)
    end_live, end_slots = sizes["live"], sizes["slots"]
    host_payload = host_payload_run(torch, SV, H, base, serve, ref)
    reqs = with_arrivals(zeros)
    sat_f = serve(reqs, True)
    check(reqs)
    keep = ("p50_ms", "p99_ms", "mean_ms", "gops", "batches", "mean_batch_requests", "rejected")
    sat_rate_b = n_requests / sat_b["makespan_s"]
    sat_rate_f = n_requests / sat_f["makespan_s"]
    rates = []
    for i, f in enumerate(SERVING_RATES):
        reqs = with_arrivals(poisson(f * sat_rate_b, 1 + i))
        out = serve(reqs, False)
        check(reqs)
        rates.append({"server": "batched", "rate_x_saturation": f, "req_per_s": f * sat_rate_b,
                      **{k: out[k] for k in keep}})
    for i, f in enumerate(FIFO_RATES):
        reqs = with_arrivals(poisson(f * sat_rate_f, 11 + i))
        out = serve(reqs, True)
        check(reqs)
        rates.append({"server": "fifo", "rate_x_saturation": f, "req_per_s": f * sat_rate_f,
                      **{k: out[k] for k in keep}})
    return {"workload": (f"{n_tables} resizable tables preloaded with 2^{preload_log2} keys "
                         f"(growth limit 2^{max_slots_log2} slots each), {n_requests} requests of "
                         "log-uniform 1-2^20 ops (insert:erase:find 40/20/40), HBM budget 64 GB"),
            "ops": int(sat_b["ops"]),
            "saturation": {"batched_gops": sat_b["gops"], "fifo_gops": sat_f["gops"],
                           "speedup": sat_b["gops"] / sat_f["gops"],
                           "batched_req_per_s": sat_rate_b, "fifo_req_per_s": sat_rate_f},
            "rates": rates,
            "tables_at_end": {"live_keys_min": int(min(end_live)),
                              "live_keys_max": int(max(end_live)),
                              "slots_max": int(max(end_slots)),
                              "committed_gb": float(sum(end_slots) * SV.SLOT_BYTES / 1e9)},
            "host_payload": host_payload,
            "identical_results": bool(same[0]), "tuned": tuned}


def host_payload_run(torch, SV, H, base, serve, ref):
    """The serving leg's closed-loop batched run with every request's payload
    (ops, keys, values in; values and statuses out) in pinned host memory,
    which the multi-table kernels read and write in place across the CPU-GPU
    link.  The arrays are views of one pinned buffer per field, filled before
    the run; results must equal the device-payload run's."""
    def pinned(ts, dtype, fill):
        flat = torch.empty(sum(int(t.numel()) for t in ts), dtype=dtype, pin_memory=True)
        out, off = [], 0
        for t in ts:
            n = int(t.numel())
            v = flat[off:off + n]
            if fill:
                v.copy_(t)
            out.append(v)
            off += n
        return out
    ops = pinned([r.ops for r in base], torch.uint8, True)
    keys = pinned([r.keys for r in base], torch.int32, True)
    vals = pinned([r.vals for r in base], torch.int32, True)
    vout = pinned([r.keys for r in base], torch.int32, False)
    stat = pinned([r.ops for r in base], torch.uint8, False)
    reqs = [SV.Request(r.rid, r.table, 0.0, o, k, v, r.n_insert, vo, st)
            for r, o, k, v, vo, st in zip(base, ops, keys, vals, vout, stat)]
    out = serve(reqs, False)
    same = all(torch.equal(a.cpu(), r.status) and torch.equal(b.cpu(), r.vals_out)
               for (a, b), r in zip(ref, reqs))
    return {"batched_gops": out["gops"], "p50_ms": out["p50_ms"], "p99_ms": out["p99_ms"],
            "identical_results": bool(same), "direct_access": H.host_direct_access(),
            "h2d_bytes": int(sum(9 * int(r.keys.numel()) for r in base)),
            "d2h_bytes": int(sum(5 * int(r.keys.numel()) for r in base))}


# ---------------------------------------------------------------------------
# own arm
# ---------------------------------------------------------------------------

def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2510_15095_gb300 import hive as H

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    seed = shard_seed(rank)
    w = make_workload(seed, args.slots)
    cfg = workload_config(w, args.slots)
    up = lambda a: H.to_device_u32(a, dev)  # noqa: E731
    ik, iv, fk = up(w["insert_keys"]), up(w["insert_vals"]), up(w["find_keys"])
    mo = torch.from_numpy(w["mix_ops"]).to(dev)
    mk, mv = up(w["mix_keys"]), up(w["mix_vals"])
    n_ins, n_find, n_mix = ik.numel(), fk.numel(), mk.numel()
    ins_st = torch.empty(n_ins, dtype=torch.uint8, device=dev)
    f_val = torch.empty(n_find, dtype=torch.int32, device=dev)
    f_fnd = torch.empty(n_find, dtype=torch.uint8, device=dev)
    # bucket width and knobs from the autotuner for this workload class (the
    # paper's default S = 32 is measured too, below)
    from paper_2510_15095_gb300 import autotune as AT
    if args.bucket_slots:
        tuned = {"bucket_slots": args.bucket_slots, "max_evictions": 16, "placement": 0}
    else:
        tuned = AT.tune(args.slots, 95, (1, 2, 1), False, space=BENCH_SPACE)
    if args.l2_persist >= 0:
        tuned["l2_persist"] = args.l2_persist
    if args.block_threads:
        tuned["block_threads"] = args.block_threads
    cfg["table"] = dict(tuned)
    t = H.HiveTable(args.slots, **tuned)
    stream = torch.cuda.current_stream(dev)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step(times=None):
        t.clear()
        if times is not None:
            ev[0].record(stream)
        t.insert(ik, iv, status=ins_st)
        if times is not None:
            ev[1].record(stream)
        t.find(fk, vals_out=f_val, found=f_fnd)
        if times is not None:
            ev[2].record(stream)
        mvo, mst = t.execute(mo, mk, mv)
        if times is not None:
            ev[3].record(stream)
            torch.cuda.synchronize(dev)
            times.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                          ev[2].elapsed_time(ev[3])))
        return mvo, mst

    # warm-up, then a correctness gate on the last warm-up step
    for _ in range(max(args.warmup, 1)):
        mvo, mst = step()
    torch.cuda.synchronize(dev)
    assert bool((ins_st == H.INSERTED).all()), "bulk insert did not insert every key"
    hits = torch.from_numpy(w["is_hit"]).to(dev)
    assert bool(((f_fnd == 1) == hits).all()), "find flags disagree with the workload"
    assert t.check() == 0

    # per-phase breakdown and bucket probes (outside the timed region)
    phase_ms = []
    for _ in range(3):
        step(phase_ms)
    t.clear()
    t.insert(ik, iv, status=ins_st)
    s_ins = t.stats()
    t.find(fk, vals_out=f_val, found=f_fnd)
    s_find = t.stats()
    t.execute(mo, mk, mv)
    s_mix = t.stats()
    probes_ins = s_ins["probes"]
    probes_find = s_find["probes"] - s_ins["probes"]
    probes_mix = s_mix["probes"] - s_find["probes"]
    claimed_mix = s_mix["claimed_fast"] - s_find["claimed_fast"]
    overflowed_mix = s_mix["overflowed"] - s_find["overflowed"]
    overflowed = s_ins["overflowed"]
    stashed = s_ins["stashed"]

    # timed region
    gpu_id = gpu_select(torch, dev)
    barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.2)
    t.profile(True)
    t.profile_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    prof = t.profile_read()
    t.profile(False)
    ms = max_over_ranks(torch, dist, e0.elapsed_time(e1), world, dev)
    ops_step = n_ins + n_find + n_mix
    value = job_gops(ops_step, args.steps, world, ms)
    gpu_launches = sum(c for _, c in prof.values())

    # roofline of the dominant kernel (algorithmic bytes per op x ops per launch)
    peak, peak_kind = measured_peak()
    ins_ms = prof.get("insert", (0.0, 1))
    find_ms = prof.get("find", (0.0, 1))
    mix_ms = prof.get("mixed", (0.0, 1))
    claim_ms = prof.get("claim", (0.0, 1))
    # mixed I/O: op, key, value in; value, status out.  A batch of 2^18 ops or
    # more claims its new keys in the claim kernel, whose bytes are its own:
    # a 12-byte list entry and a status byte per new key, a written sector
    # per claim (the free masks it reads are served by L2)
    bb = 8 * int(tuned.get("bucket_slots", 32))  # bytes per bucket probe
    deferred = claim_ms[1] > 0
    bytes_mix = 14 * n_mix + bb * probes_mix + (0 if deferred else 32 * claimed_mix)
    bytes_claim = 13 * (claimed_mix + overflowed_mix) + 32 * claimed_mix
    bytes_find = 9 * n_find + bb * probes_find  # key in, value + flag out, probed buckets
    bytes_ins = 9 * n_ins + bb * probes_ins + 32 * (n_ins - overflowed)  # + one written sector
    rl = {}
    sw = int(tuned.get("bucket_slots", 32))
    for name, (tot, cnt), byts, kname in (("insert", ins_ms, bytes_ins, f"k_ops<insert,S={sw}>"),
                                            ("find", find_ms, bytes_find, f"k_ops<find,S={sw}>"),
                                            ("mixed", mix_ms, bytes_mix, f"k_ops<mixed,S={sw}>"),
                                            ("claim", claim_ms, bytes_claim, f"k_claim<S={sw}>")):
        if name == "claim" and not deferred:
            continue
        avg = tot / max(cnt, 1)
        ach = byts / (avg / 1e3) / 1e9 if avg > 0 else 0.0
        traffic, _ = recorded_traffic(kname)
        rl[name] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": traffic, "algorithmic_bytes": byts,
                    "avg_ms": avg, "kernel": kname, "peak_source": peak_kind}
    dom = max(("insert", ins_ms[0]), ("find", find_ms[0]), ("mixed", mix_ms[0]), key=lambda x: x[1])[0]
    roofline = dict(rl[dom])
    roofline["others"] = {k: v for k, v in rl.items() if k != dom}

    # the paper's default bucket width, for reference (same steps, untimed region)
    default_s32 = None
    if tuned.get("bucket_slots", 32) != 32:
        t32 = H.HiveTable(args.slots)
        ev4 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        rows = []
        for r in range(4):
            t32.clear()
            ev4[0].record(stream)
            t32.insert(ik, iv, status=ins_st)
            ev4[1].record(stream)
            t32.find(fk, vals_out=f_val, found=f_fnd)
            ev4[2].record(stream)
            t32.execute(mo, mk, mv)
            ev4[3].record(stream)
            torch.cuda.synchronize(dev)
            if r:
                rows.append([ev4[0].elapsed_time(ev4[1]), ev4[1].elapsed_time(ev4[2]),
                             ev4[2].elapsed_time(ev4[3])])
        a = np.array(rows).mean(axis=0)
        default_s32 = {"insert_gops": n_ins / a[0] / 1e6, "find_gops": n_find / a[1] / 1e6,
                       "mixed_gops": n_mix / a[2] / 1e6,
                       "step_gops": ops_step / (a.sum() + 0.0) / 1e6}
        t32.close()

    fused = fused_leg(torch, H, dev, t, ik, iv, mo, mk, mv)

    ph = np.array(phase_ms)
    phases = {"insert_gops": n_ins / (ph[:, 0].mean() / 1e3) / 1e9,
              "find_gops": n_find / (ph[:, 1].mean() / 1e3) / 1e9,
              "mixed_gops": n_mix / (ph[:, 2].mean() / 1e3) / 1e9,
              "insert_ms": float(ph[:, 0].mean()), "find_ms": float(ph[:, 1].mean()),
              "mixed_ms": float(ph[:, 2].mean()),
              "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
              "probes_per_find": probes_find / n_find, "probes_per_insert": probes_ins / n_ins,
              "probes_per_mixed": probes_mix / n_mix,
              "insert_overflowed": overflowed, "insert_stashed": stashed,
              "paper_default_s32": default_s32, "fused_mixed": fused}

    # end to end through the public API with host buffers, every transfer
    # inside the timed region.  On a GPU with coherent host access (GB300's
    # NVLink-C2C) the host-buffer calls run the kernels on the pinned arrays
    # in place: inputs are read and results written across the link.
    # Elsewhere, and for the "staged" figure, they stream the arrays through
    # device staging with copies overlapped with the kernels.
    h_ik = torch.from_numpy(w["insert_keys"].view(np.int32)).pin_memory()
    h_iv = torch.from_numpy(w["insert_vals"].view(np.int32)).pin_memory()
    h_fk = torch.from_numpy(w["find_keys"].view(np.int32)).pin_memory()
    h_mo = torch.from_numpy(w["mix_ops"]).pin_memory()
    h_mk = torch.from_numpy(w["mix_keys"].view(np.int32)).pin_memory()
    h_mv = torch.from_numpy(w["mix_vals"].view(np.int32)).pin_memory()
    o_st = torch.empty(n_ins, dtype=torch.uint8).pin_memory()
    o_fv = torch.empty(n_find, dtype=torch.int32).pin_memory()
    o_ff = torch.empty(n_find, dtype=torch.uint8).pin_memory()
    o_mv = torch.empty(n_mix, dtype=torch.int32).pin_memory()
    o_ms = torch.empty(n_mix, dtype=torch.uint8).pin_memory()

    def e2e_step():
        t.clear()
        t.insert_host(h_ik, h_iv, o_st)
        t.find_host(h_fk, o_fv, o_ff)
        t.execute_host(h_mo, h_mk, h_mv, o_mv, o_ms)

    def e2e_run():
        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        w0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
        ms = max_over_ranks(torch, dist, max(e0.elapsed_time(e1), 0.0), world, dev)
        assert bool((o_st.numpy() == H.INSERTED).all()), "e2e insert statuses disagree"
        assert bool((o_ff.numpy() == w["is_hit"]).all()), "e2e find flags disagree"
        return ms, wall

    direct = H.host_direct_access()
    e2e_ms, wall = e2e_run()
    prev = os.environ.get("HIVE_HOSTIO_STAGED")
    os.environ["HIVE_HOSTIO_STAGED"] = "1"
    try:
        staged_ms, _ = e2e_run()
    finally:
        if prev is None:
            os.environ.pop("HIVE_HOSTIO_STAGED")
        else:
            os.environ["HIVE_HOSTIO_STAGED"] = prev
    h2d = 4 * (2 * n_ins + n_find + 2 * n_mix) + n_mix
    d2h = n_ins + 5 * n_find + 5 * n_mix
    e2e = {"value": job_gops(ops_step, args.e2e_steps, world, e2e_ms), "unit": "Gops/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
           "api": "hive_insert_host / hive_find_host / hive_execute_host (pinned host buffers)",
           "transfer": ("kernels read and write the pinned host arrays in place over the "
                        "coherent CPU-GPU link" if direct else
                        "chunked copies through device staging, overlapped with the kernels"),
           "host_wall_gops": ops_step * args.e2e_steps / wall / 1e9,
           "staged_gops": job_gops(ops_step, args.e2e_steps, world, staged_ms)}

    extra = {}
    if not args.no_tables:
        extra["multi_table"] = tables_leg(torch, H, dev, n_tables=args.tables_n,
                                          steps=args.tables_steps)
    if not args.no_serving:
        extra["serving"] = serving_leg(torch, H, dev, n_requests=args.serving_requests,
                                       preload_log2=args.serving_preload_log2,
                                       max_slots_log2=args.serving_max_log2)
    if not args.no_resize:
        extra["resize_stream"] = resize_leg(torch, H, dev,
                                           batches=159 if args.resize_full else args.resize_batches)
    if not args.no_breakdown:
        extra["insert_breakdown"] = {
            "tuned": breakdown_leg(torch, H, dev, tuned, slots=args.slots),
            "paper_s32": breakdown_leg(torch, H, dev, dict(tuned, bucket_slots=32),
                                       slots=args.slots)}
    if not args.no_sweep:
        extra["load_sweep"] = sweep_leg(torch, H, dev, tuned, slots=args.slots,
                                        n_find=N_FIND if args.slots == SLOTS else args.slots)
        extra["plain_2e20"] = plain_leg(torch, H, dev)
        extra["hive32_key_only"] = hive32_leg(torch, H, dev, slots=args.slots,
                                              n_find=N_FIND if args.slots == SLOTS else args.slots)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n = min(args.cpu_sample, n_ins)
        ops, dt = oracle_sample(w, n)
        cpu = {"value": ops / dt / 1e9, "unit": "Gops/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} inserts + {n} finds + {n // 4} mixed ops (prefix of the workload), "
                         f"{dt:.1f} s single-threaded std::unordered_map",
               "host": host_info()}
        if not args.no_cpu_parallel:
            extra["cpu_parallel"] = cpu_parallel_leg(w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gops/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32/u64", "data": "synthetic", "config": cfg, "phases": phases,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": gpu_launches, **extra}
        print(json.dumps(line), flush=True)
    t.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
