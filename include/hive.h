/*
 * hive.h -- C ABI of the Hive hash table on one GB300 GPU (sm_103a).
 *
 * The table is the one of "Hive Hash Table: A Warp-Cooperative, Dynamically
 * Resizable Hash Table for GPUs" (arXiv 2510.15095): 32-bit keys and 32-bit
 * values packed into 64-bit words (Section III-A), buckets of S slots with a
 * per-bucket free mask and lock plus an overflow stash (Section III-B), two
 * candidate buckets per key from BitHash1/BitHash2 (Section III-C), insert by
 * replace -> claim-then-commit -> bounded cuckoo eviction -> stash
 * (Section IV-A, Algorithms 1-3), lookup and delete by warp match-and-elect
 * (Section IV-B, Algorithm 4), and linear-hashing growth and shrinkage in
 * batches of K bucket pairs (Section IV-C).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Op arrays (keys, values, op codes, outputs) are DEVICE pointers owned by
 *    the caller (any memory the GPU can address).  They must stay valid until
 *    the work queued on `stream` has completed.  `stream` is a cudaStream_t
 *    passed as void*; NULL means the legacy default stream.
 *  - Calls are stream-ordered and asynchronous unless stated otherwise.  A
 *    fixed-capacity table never synchronises inside insert/find/erase/execute.
 *    A resizable table reads a few counters back to the host after each
 *    mutating call (to apply the load-factor policy), so those calls return
 *    after the work on `stream` has completed.
 *  - n == 0 is a no-op that returns HIVE_OK.  A NULL table, a NULL required
 *    array with n > 0, or n >= 2^32 returns HIVE_ERR_INVALID_ARG and queues
 *    nothing.
 *  - Keys 0xFFFFFFFE and 0xFFFFFFFF are reserved (0xFFFFFFFF'FFFFFFFF is the
 *    empty-slot word).  An op on a reserved key is skipped, reports
 *    HIVE_ST_RESERVED_KEY, and raises the table's sticky error word, which
 *    hive_check() returns.  Values are unrestricted.
 *  - Batch contract: within one call no key may appear in more than one update
 *    (insert or erase), and in hive_execute no key may be both updated and
 *    searched.  Repeated finds of one key are allowed.  Under this contract
 *    every result is unique and equals applying the ops one by one to a
 *    dictionary.  Outside it the outcome is some serialisation of the batch.
 *  - A table is driven by one host thread at a time.  No C++ exception
 *    crosses this interface.  hive_last_error() describes the last failure of
 *    the calling thread.
 */
#ifndef HIVE_H_
#define HIVE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hive_table hive_table; /* opaque; the library owns all table memory */

typedef enum {
  HIVE_OK = 0,
  HIVE_ERR_INVALID_ARG = 1,  /* bad pointer, size or configuration */
  HIVE_ERR_RESERVED_KEY = 2, /* sticky: an op used a reserved key */
  HIVE_ERR_OOM = 3,          /* device allocation failed; table unchanged */
  HIVE_ERR_FULL = 4,         /* sticky: fixed table had no room for some insert */
  HIVE_ERR_TIMEOUT = 5,      /* sticky: a bounded wait gave up (bucket lock) */
  HIVE_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  HIVE_ERR_CONTRACT = 7      /* sticky: batch contract violated (concurrent update of one key) */
} hive_status;

/* Per-op result codes (one byte per op). */
enum {
  HIVE_ST_INSERTED = 0,     /* insert of an absent key */
  HIVE_ST_REPLACED = 1,     /* insert of a present key: value overwritten */
  HIVE_ST_ERASED = 2,       /* erase of a present key */
  HIVE_ST_NOT_FOUND = 3,    /* erase or find of an absent key */
  HIVE_ST_FOUND = 4,        /* find of a present key (hive_execute only) */
  HIVE_ST_FULL = 5,         /* insert dropped: fixed table and stash full */
  HIVE_ST_RESERVED_KEY = 6  /* op on a reserved key, skipped */
};

/* Op codes for hive_execute (one byte per op). */
enum { HIVE_OP_INSERT = 0, HIVE_OP_FIND = 1, HIVE_OP_ERASE = 2 };

/* Placement of a new key among its two candidate buckets (Section V: "bucketed
 * two-choice placement").  BALANCED picks the bucket with more free slots
 * (ties go to the BitHash1 bucket); FIRST picks the BitHash1 bucket whenever it
 * has room. */
enum { HIVE_PLACE_BALANCED = 0, HIVE_PLACE_FIRST = 1 };

typedef struct {
  uint64_t initial_slots;   /* capacity at creation; rounded up to whole buckets */
  uint64_t max_slots;       /* resizable: growth limit (memory reserved up front);
                               ignored for fixed tables */
  uint32_t bucket_slots;    /* S, slots per bucket: 32 (Section III-A) */
  uint32_t max_evictions;   /* cuckoo displacement bound (Section III-B), >= 1 */
  uint32_t resize_batch;    /* K, bucket pairs per split/merge launch (Section IV-C) */
  uint32_t stash_permille;  /* stash capacity as a fraction of slots, in 1/1000
                               (Section IV-A step 4: "typically 1-2%") */
  uint32_t grow_num, grow_den;     /* expand while load > grow_num/grow_den (0.9) */
  uint32_t shrink_num, shrink_den; /* contract while load < shrink_num/shrink_den */
  uint32_t resizable;       /* 0: fixed capacity; 1: linear-hashing resize */
  uint32_t placement;       /* HIVE_PLACE_* */
  uint32_t lock_spin_limit; /* tries before a bucket-lock wait gives up */
  uint32_t blocks_per_sm;   /* resident 256-thread blocks per SM of the bulk kernel's
                               persistent grid; 0 = as many as fit (a tuning knob) */
  uint32_t map_on_demand;   /* resizable tables: 1 = reserve the address range of
                               max_slots and map bucket memory as the table grows
                               (CUDA virtual memory; committed HBM follows the
                               capacity, see hive_memory); 0 = allocate max_slots
                               of buckets up front (default; faster on the
                               multi-table path) */
  uint32_t l2_persist;      /* 1 = the kernels that claim slots (bulk insert,
                               mixed batch, claims, eviction) keep the free masks
                               in a persisting L2 access-policy window, so that
                               the claim atomics hit L2 while the bucket reads
                               stream past; the first such table of the process
                               sets the CUDA context's persisting-L2 limit (a
                               per-process setting, gone when the process exits).
                               0 = off (default; a tuning knob) */
  uint32_t stage_wait_limit;/* tries before a wait for staged bucket copies
                               gives up (TIMEOUT) and the round is redone with
                               direct loads; 0 = 2^22 (default).  Only the
                               256-byte-bucket (S = 32) copies wait on an
                               mbarrier; a small value exercises the fallback */
  uint32_t block_threads;   /* block shape of the bulk kernels: 128, 256 or 512
                               threads (one op per lane); 0 = 256 (default; a
                               tuning knob) */
} hive_config;

/* Per-table counters, accumulated since creation or the last hive_clear.
 * Steps follow Section IV-A: step 1 replace, step 2 claim-then-commit,
 * step 3 bounded cuckoo eviction, step 4 overflow stash. */
typedef struct {
  uint64_t replaced;         /* inserts finished in step 1 */
  uint64_t claimed_fast;     /* inserts finished in step 2 by the bulk kernel
                                (mixed batches: by the claim kernel that follows it) */
  uint64_t overflowed;       /* inserts handed to the eviction kernel */
  uint64_t claimed_slow;     /* of those, placed by a lock-free claim */
  uint64_t evict_rounds;     /* displacement rounds executed (step 3) */
  uint64_t lock_acquired;    /* bucket locks taken */
  uint64_t lock_timeouts;    /* bounded lock waits that gave up */
  uint64_t stashed;          /* words appended to the stash (step 4) */
  uint64_t pending;          /* inserts that found no room (FULL or re-run after growth) */
  uint64_t stash_reinserted; /* stash words moved back into buckets by maintenance */
  uint64_t splits;           /* bucket pairs split */
  uint64_t merges;           /* bucket pairs merged */
  uint64_t probes;           /* 256-byte bucket reads by the bulk kernel (Section IV-B:
                                one per candidate bucket examined) */
  uint64_t stash_lookups;    /* binary searches of the stash by the bulk kernel */
  uint64_t fused_retries;    /* single-kernel batches: lookups repeated because a
                                candidate bucket had a word in transit */
} hive_stats_t;

/* Kernel kinds timed by the profiling hook. */
enum {
  HIVE_K_FIND = 0,     /* bulk kernel, find batch */
  HIVE_K_INSERT = 1,   /* bulk kernel, insert batch (steps 1-2) */
  HIVE_K_ERASE = 2,    /* bulk kernel, erase batch */
  HIVE_K_MIXED = 3,    /* bulk kernel, mixed batch */
  HIVE_K_EVICT = 4,    /* eviction + stash kernel (steps 3-4) */
  HIVE_K_MAINT = 5,    /* stash maintenance */
  HIVE_K_SPLIT = 6,    /* linear-hashing split */
  HIVE_K_MERGE = 7,    /* linear-hashing merge and its pre-check */
  HIVE_K_COUNT = 8,    /* insert counting for a resizable mixed batch */
  HIVE_K_FUSED = 9,    /* single-kernel mixed batch (hive_execute_fused) */
  HIVE_K_CLAIM = 10,   /* claims of a mixed batch's new keys (step 2) */
  HIVE_K_KINDS = 16
};

/* Per-kind device time of the kernels launched while profiling was on. */
typedef struct {
  double ms[HIVE_K_KINDS];         /* summed kernel time, milliseconds */
  uint64_t launches[HIVE_K_KINDS]; /* kernels launched */
} hive_profile_t;

/* Host image of a quiescent table, for tests and checkpoints (hive_dump). */
typedef struct {
  uint64_t nb;          /* buckets in use = M + 1 + p */
  uint32_t S;           /* slots per bucket */
  uint32_t M;           /* linear-hashing index mask 2^m - 1 */
  uint32_t p;           /* split pointer */
  uint32_t reserved0;
  uint64_t stash_n;     /* stash words in use */
  uint64_t stash_cap;   /* stash capacity */
  uint64_t size;        /* live-entry counter */
  uint64_t pending;     /* words waiting for room (0 at quiescence) */
  uint64_t* buckets;    /* [nb * S] packed words, or NULL to query sizes only */
  uint32_t* masks;      /* [nb] free masks, bit i set = slot i free */
  uint32_t* locks;      /* [nb] lock words */
  uint64_t* stash;      /* [stash_n] packed words */
} hive_image;

/* Fills *cfg with defaults: 2^20 slots, S = 32, max_evictions 16, K = 1024,
 * stash 1%, thresholds 9/10 and 2/5, fixed capacity, balanced placement. */
void hive_config_default(hive_config* cfg);

/* Creates a table (Section III-B: buckets, freeMask, lock, metadata, stash).
 * All device memory is allocated here, on the current CUDA device; a resizable
 * table reserves max_slots up front.  The table is empty on return, and its
 * initialisation is ordered on `stream`.  Errors: INVALID_ARG (bad config),
 * OOM (nothing leaked), CUDA. */
hive_status hive_create(const hive_config* cfg, void* stream, hive_table** out);

/* Frees every allocation of the table.  Synchronises the device first. */
hive_status hive_destroy(hive_table* t);

/* Insert/Replace (Section III-D; Section IV-A, Algorithms 1-3 and step 4).
 * keys[n], vals[n]: inputs.  status[n] (nullable): per-op
 * INSERTED / REPLACED / FULL / RESERVED_KEY. */
hive_status hive_insert(hive_table* t, const uint32_t* keys, const uint32_t* vals,
                        uint64_t n, uint8_t* status, void* stream);

/* Search (Section III-D; Section IV-B, WCME).  vals_out[n]: the value, or 0 when
 * absent.  found[n] (nullable): 1 when present, else 0.  Never mutates. */
hive_status hive_find(hive_table* t, const uint32_t* keys, uint64_t n, uint32_t* vals_out,
                      uint8_t* found, void* stream);

/* Delete (Section III-D; Section IV-B, Algorithm 4).  status[n] (nullable):
 * ERASED / NOT_FOUND / RESERVED_KEY. */
hive_status hive_erase(hive_table* t, const uint32_t* keys, uint64_t n, uint8_t* status,
                       void* stream);

/* Mixed batch (Section V-C2, imbalanced workloads).  ops[n] holds HIVE_OP_*.
 * vals[n] supplies insert values; it may be NULL, and the batch's inserts
 * then store value 0 (the kernels never read a NULL vals).
 * vals_out[n] (nullable): find results, 0 otherwise.  status[n] (nullable):
 * per-op code (finds report FOUND / NOT_FOUND). */
hive_status hive_execute(hive_table* t, const uint8_t* ops, const uint32_t* keys,
                         const uint32_t* vals, uint64_t n, uint32_t* vals_out,
                         uint8_t* status, void* stream);

/* The same mixed batch in one kernel, the paper's single-kernel mode
 * (Section III-D: all operation types of a batch run concurrently in one
 * launch).  Finds, erases, replaces, claims, cuckoo eviction chains
 * (Algorithm 3) and stash appends of the batch all run at once.  A lookup
 * that misses while a chain is moving a word out of one of its candidate
 * buckets is repeated: each bucket carries a version word that a chain
 * raises and lowers around the move of any word whose BitHash1 bucket it
 * is, and a miss counts only if the version of the key's BitHash1 bucket was
 * quiet and unchanged across the probe.  Arguments, per-op results, the batch
 * contract and the errors are exactly those of hive_execute(), and so are
 * the results.  A resizable table grows before the kernel as in
 * hive_execute(); inserts that still find no room (stash full) are placed
 * after further growth by the eviction kernel, before the call returns.
 * Stash maintenance follows as a second, usually empty, launch. */
hive_status hive_execute_fused(hive_table* t, const uint8_t* ops, const uint32_t* keys,
                               const uint32_t* vals, uint64_t n, uint32_t* vals_out,
                               uint8_t* status, void* stream);

/* Live entries (buckets + stash).  Synchronises `stream`. */
hive_status hive_size(hive_table* t, uint64_t* out, void* stream);

/* Grows a resizable table until it has at least `slots` slots (or reaches
 * max_slots), by linear-hashing splits in launches of K bucket pairs
 * (Section IV-C1), so that later batches need not grow.  A fixed table only
 * checks that it already has `slots` slots (else INVALID_ARG).  Stream-ordered;
 * no synchronisation. */
hive_status hive_reserve(hive_table* t, uint64_t slots, void* stream);

/* Device memory of the table in bytes: `committed` is backed by physical
 * memory now, `reserved` is the most it can grow to.  A resizable table keeps
 * its buckets on CUDA virtual memory: it reserves the address range of
 * max_slots at creation, maps physical memory as splits add buckets and
 * returns it after merges, so committed memory follows the capacity (the
 * other arrays are allocated at their maximum).  Host-side, no sync. */
hive_status hive_memory(hive_table* t, uint64_t* committed, uint64_t* reserved);

/* The two hash mixes of Section III-C on the device: h1_out[i] = BitHash1(keys[i])
 * and h2_out[i] = BitHash2(keys[i]), the full 32-bit mixes before any bucket
 * reduction (the tables address buckets with the linear-hashing rule of
 * Section IV-C on these values).  Device arrays of n entries owned by the
 * caller; either output may be NULL.  Stream-ordered, no synchronisation.
 * For callers that place or shard keys the way the tables do, and for tests
 * of the mixes.  INVALID_ARG for NULL keys or two NULL outputs with n > 0. */
hive_status hive_hash(const uint32_t* keys, uint64_t n, uint32_t* h1_out, uint32_t* h2_out,
                      void* stream);

/* Current slot capacity S * nBuckets (host-side state, no synchronisation). */
hive_status hive_capacity(hive_table* t, uint64_t* slots_out);

/* Empties the table and returns it to its initial capacity (stream-ordered). */
hive_status hive_clear(hive_table* t, void* stream);

/* Reads the sticky device error word, clears it, and returns the first
 * condition seen (RESERVED_KEY, FULL, TIMEOUT, CONTRACT) or HIVE_OK.
 * Synchronises `stream`. */
hive_status hive_check(hive_table* t, void* stream);

/* Copies the counters to *out.  Synchronises `stream`. */
hive_status hive_stats(hive_table* t, hive_stats_t* out, void* stream);

/* Copies the table into caller-owned host arrays.  With img->buckets == NULL
 * only the scalar fields are filled (to size the arrays).  Synchronises. */
hive_status hive_dump(hive_table* t, hive_image* img, void* stream);

/* Turns per-kernel timing on (enable != 0) or off.  While on, every kernel
 * the table launches is bracketed by two CUDA events recorded on the launch
 * stream.  Host-side only; no synchronisation. */
hive_status hive_profile_enable(hive_table* t, int enable);

/* Accumulates the recorded kernel times into *out (adding to what it holds)
 * and forgets them.  Synchronises on the recorded events. */
hive_status hive_profile_read(hive_table* t, hive_profile_t* out);

/* ---- Host-buffer calls ----
 * Same operations with the op arrays in HOST memory.  The call returns when
 * every output is in host memory; results equal the device-pointer calls.
 * Two ways through, picked per call:
 *  - direct: when the current device reaches host memory coherently through
 *    the CPU-GPU link (hive_host_direct_access reports 1; GB300's NVLink-C2C)
 *    and every array is pinned or registered host memory (cudaMallocHost,
 *    cudaHostRegister) or device memory, the kernels read the inputs and write
 *    the results in place, with no staging copies;
 *  - staged: otherwise (pageable arrays, other GPUs, or HIVE_HOSTIO_STAGED=1
 *    in the environment) the batch streams through device staging in chunks
 *    of 2^22 ops, two at a time, so that the host-to-device copy of one
 *    chunk, the kernels of the previous one and the copy back of the one
 *    before overlap (fully when the host buffers are pinned).  Chunking does
 *    not change results under the batch contract.  The staging (about 120 MB)
 *    is allocated on the first staged call of a table and freed by
 *    hive_destroy. */
hive_status hive_insert_host(hive_table* t, const uint32_t* h_keys, const uint32_t* h_vals,
                             uint64_t n, uint8_t* h_status, void* stream);
hive_status hive_find_host(hive_table* t, const uint32_t* h_keys, uint64_t n,
                           uint32_t* h_vals_out, uint8_t* h_found, void* stream);
hive_status hive_execute_host(hive_table* t, const uint8_t* h_ops, const uint32_t* h_keys,
                              const uint32_t* h_vals, uint64_t n, uint32_t* h_vals_out,
                              uint8_t* h_status, void* stream);

/* *out = 1 when the current device reaches host memory coherently through the
 * CPU-GPU link (cudaDevAttrPageableMemoryAccessUsesHostPageTables), so that
 * host-buffer calls on pinned or registered arrays take the direct way; else
 * 0.  INVALID_ARG for NULL out; CUDA when the device cannot be queried. */
hive_status hive_host_direct_access(int* out);

/* ---- Multi-table batches (many independent tables, one launch per phase) ----
 * Not in the paper: the tables are the paper's, the batching is a library
 * layer for services that hold many tables.  A batch is a list of segments;
 * each segment is a mixed op range (HIVE_OP_* codes, as in hive_execute) on one
 * table.  Per table, the ops of all its segments in one call obey the batch
 * contract of hive_execute, and the results equal running those segments
 * through hive_execute on that table.  Differences from hive_execute:
 *  - a resizable table grows before the batch for n_insert new keys of its
 *    segments (give the exact insert count, or n); an insert that still finds
 *    no room (stash full) reports FULL instead of growing mid-batch;
 *  - find statuses are FOUND / NOT_FOUND like hive_execute; there is no
 *    separate found-flag array. */
typedef struct hive_multi hive_multi;

typedef struct {
  uint32_t table;         /* index into the tables given to hive_multi_create */
  uint32_t reserved0;     /* must be 0 */
  uint64_t n;             /* ops in this segment, < 2^32 */
  uint64_t n_insert;      /* upper bound of HIVE_OP_INSERT ops among them */
  const uint8_t* ops;     /* [n] HIVE_OP_* (device) */
  const uint32_t* keys;   /* [n] (device) */
  const uint32_t* vals;   /* [n] insert values (device, nullable without inserts) */
  uint32_t* vals_out;     /* [n] find results, 0 otherwise (device, nullable) */
  uint8_t* status;        /* [n] per-op status (device, nullable) */
} hive_segment;
/* "device" above: any address the kernels can use, which includes pinned or
 * registered host memory (cudaMallocHost, cudaHostRegister): the kernels then
 * read the inputs and write the results across the CPU-GPU link, at near
 * device speed where hive_host_direct_access() reports 1.  The caller keeps
 * such host arrays untouched until the batch has completed. */

/* Flags of hive_multi_create. */
enum {
  HIVE_MULTI_GRAPH = 1, /* capture the fixed kernel sequence into a CUDA graph on the
                           first batch and replay it afterwards */
  HIVE_MULTI_ASYNC = 2  /* never wait for a batch: resizable tables grow for an upper
                           bound of their size (last gathered size + inserts queued
                           since) and are not contracted; two batches may be in flight */
};

/* Groups tables (created by hive_create on the current device) for batched
 * calls.  max_segments and max_ops bound one batch.  The tables stay owned by
 * the caller and must outlive the group.  Without HIVE_MULTI_ASYNC they may
 * still be used one by one between batches (same stream); with it, drive them
 * only through the group. */
hive_status hive_multi_create(hive_table* const* tables, uint32_t n_tables,
                              uint32_t max_segments, uint64_t max_ops, int flags,
                              void* stream, hive_multi** out);

/* Runs one batch on `stream`.  Consecutive batches of one group go on one
 * stream.  Without HIVE_MULTI_ASYNC, a group holding resizable tables waits
 * once for the batch (exact sizes, contraction policy applied to its tables);
 * otherwise the call returns after queueing, waiting only for the batch
 * queued two calls earlier.  Errors: INVALID_ARG (bad segment, too many ops,
 * segments or split launches), CUDA. */
hive_status hive_multi_execute(hive_multi* m, const hive_segment* segs, uint32_t n_segs,
                               void* stream);

/* Frees the group (not its tables).  Synchronises the device first. */
hive_status hive_multi_destroy(hive_multi* m);

/* Upper bounds of the live sizes of the group's first n_tables tables, into
 * out[n_tables]: the size gathered after the newest completed batch of each
 * table plus the inserts of its batches queued since (HIVE_MULTI_ASYNC), or
 * the exact sizes (synchronous groups).  A scheduler that admits work by
 * memory uses these, and hive_capacity() of each table, instead of counting
 * inserts itself: erases make the bounds fall again.  Host-side; it queries
 * the batches' events and never waits.  INVALID_ARG for NULL pointers or
 * n_tables above the group's. */
hive_status hive_multi_bounds(hive_multi* m, uint64_t* out, uint32_t n_tables);

/* Insert into a FIXED-capacity table without allocating anything.  The paper
 * has no counterpart; this is a library convenience.  Same inputs, outputs and
 * results as hive_insert, for callers that must not call cudaMalloc: a process
 * whose device memory is all pre-reserved by another allocator, or a
 * latency-bound loop that cannot stall behind the device synchronisation that
 * precedes hive_insert's on-demand growth of its scratch list.  The list of
 * inserts handed to the eviction kernel lives instead in one file-scope device
 * array of 2^18 entries (3 MiB per GPU, held until exit).
 *  - n must be <= 2^18 (262,144) per call, else HIVE_ERR_INVALID_ARG and nothing
 *    is queued; a resizable table also gives HIVE_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept with the id of the CUDA
 *    context it belongs to and looked up again when the current context
 *    differs (after cudaDeviceReset the array may move); where the driver
 *    gives no context ids, every call looks it up.
 *  - All calls share the array: calls whose work overlaps on the GPU (e.g. on
 *    two streams at once) race and must not be issued. */
hive_status hive_insert_noalloc(hive_table* t, const uint32_t* keys, const uint32_t* vals,
                                uint64_t n, uint8_t* status, void* stream);

/* ---- Tables with 32-bit entries ----
 * Section III-B: with 32-bit entries (a key-only set, or a 16-bit key and a
 * 16-bit value) a bucket of 32 slots fits one 128-byte cache line, half the
 * bytes of a probe of the 64-bit table.  Same algorithm (replace, claim,
 * bounded cuckoo eviction, stash; match-and-elect lookups), fixed capacity,
 * 32 slots per bucket, BitHash1/BitHash2 of the (16- or 32-bit) key.  Same
 * conventions as the calls above: device op arrays owned by the caller,
 * stream-ordered, the batch contract, per-op status codes, sticky errors.
 *  - HIVE32_KEY16_VAL16: entry = value << 16 | key.  Keys must be below
 *    0xFFFE and values below 2^16; an op whose key (or, for an insert, value)
 *    is out of range reports HIVE_ST_RESERVED_KEY and raises
 *    HIVE_ERR_RESERVED_KEY.  Finds return the 16-bit value.
 *  - HIVE32_KEY_ONLY: entry = key, a set of 32-bit keys (0xFFFFFFFE and
 *    0xFFFFFFFF reserved).  vals may be NULL and is ignored; an insert of a
 *    present key reports HIVE_ST_REPLACED; finds return value 0 and the
 *    found flag. */
enum { HIVE32_KEY16_VAL16 = 0, HIVE32_KEY_ONLY = 1 };

typedef struct hive32_table hive32_table; /* opaque */

typedef struct {
  uint64_t slots;           /* capacity in slots, rounded up to a multiple of 32 (>= 32) */
  uint32_t layout;          /* HIVE32_KEY16_VAL16 or HIVE32_KEY_ONLY */
  uint32_t max_evictions;   /* cuckoo displacement bound per insert (1..64, default 16) */
  uint32_t stash_permille;  /* stash capacity in 1/1000 of the slots (default 10, at most 1000; at least 1024 entries) */
  uint32_t lock_spin_limit; /* bounded bucket-lock wait, in tries (default 1 << 16) */
} hive32_config;

/* A host image of a quiescent 32-bit table (hive32_dump). */
typedef struct {
  uint64_t nb;          /* buckets = M + 1 + p */
  uint32_t M, p;        /* linear-hashing address state (p > 0 when nb is not a power of two) */
  uint32_t layout;
  uint32_t* buckets;    /* [nb * 32] entries, 0xFFFFFFFF = empty (caller-allocated) */
  uint32_t* masks;      /* [nb] free masks */
  uint32_t* locks;      /* [nb] */
  uint32_t* stash;      /* [stash_cap] sorted live prefix of stash_n entries */
  uint64_t stash_n, stash_cap, size, pending;
} hive32_image;

void hive32_config_default(hive32_config* cfg);
/* Allocates the table (buckets, masks, locks, stash) on the current device.
 * Errors: INVALID_ARG for a bad layout, size, max_evictions, stash_permille
 * or lock_spin_limit; OOM. */
hive_status hive32_create(const hive32_config* cfg, void* stream, hive32_table** out);
hive_status hive32_destroy(hive32_table* t);
/* Insert/Replace (vals may be NULL for HIVE32_KEY_ONLY); status nullable:
 * INSERTED / REPLACED / FULL / RESERVED_KEY. */
hive_status hive32_insert(hive32_table* t, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                          uint8_t* status, void* stream);
/* Search: vals_out (nullable) gets the value or 0, found (nullable) 1 or 0. */
hive_status hive32_find(hive32_table* t, const uint32_t* keys, uint64_t n, uint32_t* vals_out,
                        uint8_t* found, void* stream);
/* Delete: status nullable, ERASED / NOT_FOUND / RESERVED_KEY. */
hive_status hive32_erase(hive32_table* t, const uint32_t* keys, uint64_t n, uint8_t* status,
                         void* stream);
/* Mixed batch of HIVE_OP_* codes, as hive_execute (a NULL vals makes the
 * batch's inserts store value 0). */
hive_status hive32_execute(hive32_table* t, const uint8_t* ops, const uint32_t* keys,
                           const uint32_t* vals, uint64_t n, uint32_t* vals_out, uint8_t* status,
                           void* stream);
/* Live entries; synchronises `stream`. */
hive_status hive32_size(hive32_table* t, uint64_t* out, void* stream);
/* Empties the table (stream-ordered; no synchronisation). */
hive_status hive32_clear(hive32_table* t, void* stream);
/* Returns and clears the sticky error word, as hive_check; synchronises. */
hive_status hive32_check(hive32_table* t, void* stream);
/* Counters (the fields of hive_stats_t that apply); synchronises. */
hive_status hive32_stats(hive32_table* t, hive_stats_t* out, void* stream);
/* Host image; with img->buckets == NULL only the scalar fields are filled. */
hive_status hive32_dump(hive32_table* t, hive32_image* img, void* stream);

/* ---- Batch-contract check (a debugging aid; the paper has none) ----
 * Section III-D runs the ops of a batch concurrently, so a batch has one
 * result only under the batch contract above.  This checks it on HOST
 * arrays: h_keys[n], and h_ops[n] (HIVE_OP_* codes) for a mixed batch.  With
 * h_ops NULL every op is `op`: HIVE_OP_INSERT or HIVE_OP_ERASE for an
 * insert or erase batch, HIVE_OP_FIND for a find batch (which always
 * passes).  Ops whose key is >= key_limit touch nothing and are ignored: pass
 * 0xFFFFFFFE for 32-bit keys, 0xFFFE for HIVE32_KEY16_VAL16.  Unknown op
 * codes count as finds, as in the kernels.  Returns HIVE_OK, or
 * HIVE_ERR_INVALID_ARG with *first_bad (nullable; n when the batch passes)
 * = the smallest i such that ops [0, i] already break the contract, and an
 * error text naming the key.  Cost: a two-pass radix sort of the keys.
 *
 * With the environment variable HIVE_DEBUG set (to anything but "0") when a
 * table is created, every update call on it (insert, erase, execute, their
 * 32-bit, allocation-free and host-buffer forms) first copies its key and
 * op arrays to the host on `stream`, waits, and runs this check; a batch
 * that fails returns HIVE_ERR_INVALID_ARG and queues nothing.  In a
 * multi-table batch (hive_multi_execute) each such table is checked over
 * all of its segments of the batch, in segment order, and the error text
 * names the table.  The check waits on `stream`, so a debug table makes
 * every update call synchronous. */
hive_status hive_check_batch(const uint8_t* h_ops, uint32_t op, const uint32_t* h_keys, uint64_t n,
                             uint32_t key_limit, uint64_t* first_bad);

/* ---- Fault injection for tests (host side; the paper has none) ----
 * The library's failure paths -- a bounded wait that gives up, a device
 * allocation that fails -- are made to run by these calls from the host.
 * Neither makes the GPU fault or hang.
 *
 * hive_debug_fail_alloc: the n-th device allocation the library makes from
 * now on (counted over every table of the process, n >= 1) fails as if the
 * device were out of memory; n = 0 cancels a pending failure.  The call that
 * made the allocation returns HIVE_ERR_OOM and leaves its table as it was
 * (hive_create frees what it had allocated; an op call queues nothing and
 * the table's data is untouched).  Always returns HIVE_OK.
 *
 * hive_debug_hold_lock: sets the bucket lock of `bucket` (Algorithm 3) to held
 * (held != 0) or free (held == 0), stream-ordered on `stream`; bucket =
 * UINT64_MAX sets every bucket in use.  An eviction round that needs a held
 * lock gives up after lock_spin_limit tries: the chain puts the word it holds
 * in the stash, the table's sticky error gets HIVE_ERR_TIMEOUT (hive_check)
 * and hive_stats counts lock_timeouts.  Every result stays what the dictionary
 * semantics give.  Free every held lock before the table is used without this
 * hook again.  Returns INVALID_ARG for a bucket not in use, CUDA on a failed
 * memset.
 *
 * hive_debug_set_versions: sets the bucket version word of every bucket (the
 * single-kernel batch's eviction-safe lookups) to `value`, stream-ordered on
 * `stream`: bits 16..31 are the count of finished moves, which a test sets
 * next to its wrap; bits 0..15, the words in transit, must be 0 (a
 * quiescent table).  Results are unaffected.  Returns INVALID_ARG for a
 * non-zero transit count, CUDA on a failed launch. */
hive_status hive_debug_fail_alloc(uint32_t n);
hive_status hive_debug_hold_lock(hive_table* t, uint64_t bucket, int held, void* stream);
hive_status hive_debug_set_versions(hive_table* t, uint32_t value, void* stream);

/* Text of the calling thread's last error (never NULL). */
const char* hive_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HIVE_H_ */
