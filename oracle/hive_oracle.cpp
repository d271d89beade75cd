// Hive hash table -- CPU ORACLE.  TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
//
// Only the test suite, the smoke check of the graft entry point and the CPU
// baseline leg of the benchmark may load this library.  The CUDA path shares
// no code with it: nothing here is included by, or includes, the GPU sources.
//
// What it computes (each item cites the passage it follows):
//
//  1. The dictionary the table implements (Section III-D, "Supported
//     Concurrent Operations"): Insert adds <k,v>, Replace overwrites the value
//     of a present key, Delete removes a key, Search returns the value or
//     "not found".  Ops are applied one by one in array order to a plain
//     std::unordered_map.  Under the batch contract of the library (no key in
//     more than one update per batch, no key both updated and searched in one
//     mixed batch) every serialisation of a batch gives this same result, so
//     per-op results and the final map are unique and compared bit-exactly.
//
//  2. BitHash1 and BitHash2 (Section III-C, Listing 1) as 32-bit mixes, without
//     the final reduction: they only enter the layout checks below.
//
//  3. The linear-hashing address and the load-factor resize policy
//     (Section IV-C): nBuckets = 2^m + p, index_mask M = 2^m - 1, split pointer
//     p; expansion past load factor 0.9, contraction below the lower threshold
//     (0.25 in the text, 0.4 in the resize-stream workload), in batches of K
//     bucket pairs.
//
//  4. A checker of the table's structural invariants over a host copy of the
//     device layout (Section III-A/B: packed words, freeMask, lock, stash).
//
//  5. A parallel CPU baseline for the benchmark (not part of the oracle's
//     definition): the same dictionary sharded by key over host threads.
//
// Parity notes: items 1 and 3 are pinned by tests against a brute-force map,
// closed forms and textbook linear-hashing properties; item 2 is pinned by
// inverting each published mixing step and by Theorem 1's collision count;
// item 4 is pinned by planted corruptions.  The concrete slot each key lands in
// is not unique under concurrency ("parity unpinned" for layout); only the
// invariants apply to it.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

// Per-op result codes (documented interface; the GPU library defines the same
// numbers in its own header).
enum : uint8_t {
  ORC_INSERTED = 0,
  ORC_REPLACED = 1,
  ORC_ERASED = 2,
  ORC_NOT_FOUND = 3,
  ORC_FOUND = 4,
  ORC_FULL = 5,
  ORC_RESERVED = 6,
};
enum : uint8_t { ORC_OP_INSERT = 0, ORC_OP_FIND = 1, ORC_OP_ERASE = 2 };

// The two largest keys are reserved: an all-ones word marks an empty slot
// (key 0xFFFFFFFF) and 0xFFFFFFFE is held back as a second sentinel.
inline bool reserved_key(uint32_t k) { return k >= 0xFFFFFFFEu; }
constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;

struct Dict {
  std::unordered_map<uint32_t, uint32_t> m;
};

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// 1. Dictionary (Section III-D)
// ---------------------------------------------------------------------------
void* orc_new(void) { return new Dict(); }
void orc_free(void* d) { delete static_cast<Dict*>(d); }
uint64_t orc_size(void* d) { return static_cast<Dict*>(d)->m.size(); }
void orc_clear(void* d) { static_cast<Dict*>(d)->m.clear(); }

// Insert/Replace: S <- (S - <k,*>) u <k,v>.
void orc_insert(void* dp, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                uint8_t* status) {
  auto& m = static_cast<Dict*>(dp)->m;
  for (uint64_t i = 0; i < n; ++i) {
    uint8_t st;
    if (reserved_key(keys[i])) {
      st = ORC_RESERVED;
    } else {
      auto it = m.find(keys[i]);
      if (it == m.end()) {
        m.emplace(keys[i], vals[i]);
        st = ORC_INSERTED;
      } else {
        it->second = vals[i];
        st = ORC_REPLACED;
      }
    }
    if (status) status[i] = st;
  }
}

// Search: the value of k, or "not found" (value 0, flag 0).
void orc_find(void* dp, const uint32_t* keys, uint64_t n, uint32_t* vals_out,
              uint8_t* found) {
  auto& m = static_cast<Dict*>(dp)->m;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t v = 0;
    uint8_t f = 0;
    if (!reserved_key(keys[i])) {
      auto it = m.find(keys[i]);
      if (it != m.end()) {
        v = it->second;
        f = 1;
      }
    }
    if (vals_out) vals_out[i] = v;
    if (found) found[i] = f;
  }
}

// Delete: S <- S - <k,*>.
void orc_erase(void* dp, const uint32_t* keys, uint64_t n, uint8_t* status) {
  auto& m = static_cast<Dict*>(dp)->m;
  for (uint64_t i = 0; i < n; ++i) {
    uint8_t st;
    if (reserved_key(keys[i]))
      st = ORC_RESERVED;
    else
      st = m.erase(keys[i]) ? ORC_ERASED : ORC_NOT_FOUND;
    if (status) status[i] = st;
  }
}

// A mixed batch: op i is applied after op i-1.  Finds report FOUND/NOT_FOUND
// in the status and the value (0 on a miss) in vals_out.
void orc_execute(void* dp, const uint8_t* ops, const uint32_t* keys, const uint32_t* vals,
                 uint64_t n, uint32_t* vals_out, uint8_t* status) {
  for (uint64_t i = 0; i < n; ++i) {
    uint8_t st = ORC_RESERVED;
    uint32_t out = 0;
    if (ops[i] == ORC_OP_INSERT) {
      orc_insert(dp, keys + i, vals + i, 1, &st);
    } else if (ops[i] == ORC_OP_ERASE) {
      orc_erase(dp, keys + i, 1, &st);
    } else {
      uint8_t f = 0;
      orc_find(dp, keys + i, 1, &out, &f);
      st = reserved_key(keys[i]) ? ORC_RESERVED : (f ? ORC_FOUND : ORC_NOT_FOUND);
    }
    if (vals_out) vals_out[i] = out;
    if (status) status[i] = st;
  }
}

// The whole map, sorted by key.
void orc_dump(void* dp, uint32_t* keys_out, uint32_t* vals_out) {
  auto& m = static_cast<Dict*>(dp)->m;
  std::vector<std::pair<uint32_t, uint32_t>> v(m.begin(), m.end());
  std::sort(v.begin(), v.end());
  for (size_t i = 0; i < v.size(); ++i) {
    keys_out[i] = v[i].first;
    vals_out[i] = v[i].second;
  }
}

// ---------------------------------------------------------------------------
// 2. Hash functions (Section III-C, Listing 1), as 32-bit mixes.
//    BitHash1 is Thomas Wang's shift-and-multiply hash ending in a *2057 step;
//    BitHash2 is Bob Jenkins' six-step add/xor/shift integer hash.  Each
//    shift-and-add of the listing is written as the multiplication it equals
//    modulo 2^32.
// ---------------------------------------------------------------------------
uint32_t orc_bithash1(uint32_t x) {
  x = x * 32767u - 1u;  // (2^15 - 1) * x - 1  ==  ~x + x * 2^15
  x ^= x >> 12;
  x = x * 5u;  // x + 4x
  x ^= x >> 4;
  x = x * 2057u;
  x ^= x >> 16;
  return x;
}

uint32_t orc_bithash2(uint32_t x) {
  x = x * 4097u + 0x7ed55d16u;  // x + 2^12 x + c
  x = (x ^ 0xc761c23cu) ^ (x >> 19);
  x = x * 33u + 0x165667b1u;  // x + 2^5 x + c
  x = (x + 0xd3a2646cu) ^ (x << 9);
  x = x * 9u + 0xfd7046c5u;  // x + 2^3 x + c
  x = (x ^ 0xb55a4f09u) ^ (x >> 16);
  return x;
}

// Array forms for tests: which = 1 or 2 selects the mix.
void orc_bithash_many(int which, const uint32_t* in, uint32_t* out, uint64_t n) {
  for (uint64_t i = 0; i < n; ++i) out[i] = which == 1 ? orc_bithash1(in[i]) : orc_bithash2(in[i]);
}

// A position-weighted sum of both mixes over every key of [lo, hi) (keys are
// the 32-bit values lo..hi-1, hi <= 2^32), modulo 2^64:
//   sum_k (BitHash1(k) + 2^32 BitHash2(k)) * (2k + 1).
// Every weight is odd, so one wrong output anywhere changes the sum; a test
// compares it with the same sum over the GPU's outputs to check both mixes on
// all 2^32 keys without moving the outputs to the host.
uint64_t orc_bithash_checksum(uint64_t lo, uint64_t hi) {
  uint64_t acc = 0;
  for (uint64_t k = lo; k < hi; ++k) {
    const uint32_t x = static_cast<uint32_t>(k);
    const uint64_t w = static_cast<uint64_t>(orc_bithash1(x)) |
                       (static_cast<uint64_t>(orc_bithash2(x)) << 32);
    acc += w * (2 * k + 1);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// 3. Linear hashing (Section IV-C).  Buckets below the split pointer p have
//    already been split in this round and are addressed with one more hash bit.
// ---------------------------------------------------------------------------
uint32_t orc_lh_address(uint32_t h, uint32_t M, uint32_t p) {
  uint32_t low = h & M;
  if (low < p) return h & (2u * M + 1u);
  return low;
}

void orc_lh_address_many(const uint32_t* h, uint32_t* out, uint64_t n, uint32_t M, uint32_t p) {
  for (uint64_t i = 0; i < n; ++i) out[i] = orc_lh_address(h[i], M, p);
}

struct orc_lh {
  uint64_t nb;       // number of buckets = M + 1 + p
  uint64_t nb_init;  // never contract below this
  uint64_t nb_max;   // never expand above this
  uint32_t M;        // index_mask = 2^m - 1
  uint32_t p;        // split pointer, 0 <= p <= M
  uint32_t S;        // slots per bucket
  uint32_t K;        // bucket pairs per split/merge launch
  uint32_t grow_num, grow_den;      // expand while size / C > grow_num / grow_den
  uint32_t shrink_num, shrink_den;  // contract while size / C < shrink_num / shrink_den
};

void orc_lh_init(orc_lh* s, uint64_t nb_init, uint64_t nb_max, uint32_t S, uint32_t K,
                 uint32_t grow_num, uint32_t grow_den, uint32_t shrink_num,
                 uint32_t shrink_den) {
  s->nb = nb_init;
  s->nb_init = nb_init;
  s->nb_max = nb_max < nb_init ? nb_init : nb_max;
  uint64_t pow2 = 1;
  while (pow2 * 2 <= nb_init) pow2 *= 2;
  s->M = static_cast<uint32_t>(pow2 - 1);
  s->p = static_cast<uint32_t>(nb_init - pow2);
  s->S = S;
  s->K = K;
  s->grow_num = grow_num;
  s->grow_den = grow_den;
  s->shrink_num = shrink_num;
  s->shrink_den = shrink_den;
}

// One split launch: pairs (p+i, p+i+2^m) for i < min(K, 2^m - p); the round
// advances when every low bucket of the round has been split.
uint32_t orc_lh_split_step(orc_lh* s) {
  uint64_t room = static_cast<uint64_t>(s->M) + 1 - s->p;
  uint64_t step = std::min<uint64_t>(s->K, room);
  step = std::min<uint64_t>(step, s->nb_max - s->nb);
  if (step == 0) return 0;
  s->p += static_cast<uint32_t>(step);
  s->nb += step;
  if (s->p == s->M + 1u) {
    s->M = 2u * s->M + 1u;
    s->p = 0;
  }
  return static_cast<uint32_t>(step);
}

// One merge launch (the inverse of a split): when p == 0 the round first
// regresses (M >>= 1, p = M + 1), then pairs (p-j, p-j+2^m), j = 1..step merge.
uint32_t orc_lh_merge_step(orc_lh* s, uint32_t max_step) {
  uint32_t M = s->M, p = s->p;
  if (p == 0) {
    if (M == 0) return 0;
    M >>= 1;
    p = M + 1u;
  }
  uint64_t step = std::min<uint64_t>(std::min<uint32_t>(s->K, max_step), p);
  step = std::min<uint64_t>(step, s->nb - s->nb_init);
  if (step == 0) return 0;
  s->M = M;
  s->p = p - static_cast<uint32_t>(step);
  s->nb -= step;
  return static_cast<uint32_t>(step);
}

static bool over_grow(const orc_lh* s, uint64_t live, uint64_t nb) {
  // live / (S * nb) > grow_num / grow_den, by cross-multiplication
  return static_cast<unsigned __int128>(live) * s->grow_den >
         static_cast<unsigned __int128>(s->S) * nb * s->grow_num;
}
static bool under_shrink(const orc_lh* s, uint64_t live, uint64_t nb) {
  return static_cast<unsigned __int128>(live) * s->shrink_den <
         static_cast<unsigned __int128>(s->S) * nb * s->shrink_num;
}

// Before a batch with up to n_ins new keys: split until the worst case stays at
// or under the upper threshold, or nb_max is reached.  Returns launches made.
uint32_t orc_lh_grow(orc_lh* s, uint64_t size, uint64_t n_ins) {
  uint32_t launches = 0;
  while (over_grow(s, size + n_ins, s->nb) && s->nb < s->nb_max) {
    if (orc_lh_split_step(s) == 0) break;
    ++launches;
  }
  return launches;
}

// After a batch: merge while the load factor is under the lower threshold, the
// table is above its initial size, and the merged table stays at or under the
// upper threshold.  Returns launches made.
uint32_t orc_lh_shrink(orc_lh* s, uint64_t size) {
  uint32_t launches = 0;
  while (s->nb > s->nb_init && under_shrink(s, size, s->nb)) {
    orc_lh trial = *s;
    if (orc_lh_merge_step(&trial, s->K) == 0) break;
    if (over_grow(s, size, trial.nb)) break;
    *s = trial;
    ++launches;
  }
  return launches;
}

// ---------------------------------------------------------------------------
// 4. Structural invariants of a quiescent table image (Section III-A/B).
//    Returns 0 when all hold, else the number of the first failed invariant,
//    with the offending bucket/slot/stash index in *where:
//      1  freeMask bit i of bucket b is set  <=>  slot (b,i) holds EMPTY;
//         bits >= S are clear
//      2  every occupied slot of bucket b holds a key whose LH address under
//         BitHash1 or BitHash2 is b
//      3  no key occurs twice over all slots and the stash
//      4  live entries == size counter, and (if a dictionary is given) the
//         multiset of <k,v> equals it
//      5  nb == M + 1 + p with p <= M; every lock is 0; pending == 0;
//         stash_n <= stash_cap
//      6  the stash holds no EMPTY word in [0, stash_n) and is sorted by key
//         (the library's reading: the stash is compacted and sorted between
//         calls so that lookups can binary-search it)
//      7  resizable tables: load factor within the policy's thresholds
//         (upper always; lower unless nb == nb_init)
// ---------------------------------------------------------------------------
int orc_check_image(const uint64_t* buckets, const uint32_t* masks, const uint32_t* locks,
                    uint64_t nb, uint32_t S, uint32_t M, uint32_t p, const uint64_t* stash,
                    uint64_t stash_n, uint64_t stash_cap, uint64_t size_counter,
                    uint64_t pending, void* dict, const orc_lh* policy, uint64_t* where) {
  *where = 0;
  if (nb != static_cast<uint64_t>(M) + 1 + p || p > M) return 5;
  if (stash_n > stash_cap || pending != 0) return 5;
  for (uint64_t b = 0; b < nb; ++b)
    if (locks[b] != 0) {
      *where = b;
      return 5;
    }
  const uint32_t valid = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u);
  std::unordered_map<uint32_t, uint32_t> seen;
  uint64_t live = 0;
  for (uint64_t b = 0; b < nb; ++b) {
    if (masks[b] & ~valid) {
      *where = b;
      return 1;
    }
    for (uint32_t i = 0; i < S; ++i) {
      uint64_t w = buckets[b * S + i];
      uint32_t k = static_cast<uint32_t>(w & 0xFFFFFFFFu);
      bool empty = (w == ~0ull);
      bool free_bit = (masks[b] >> i) & 1u;
      if (empty != free_bit || (!empty && k == EMPTY_KEY)) {
        *where = b * S + i;
        return 1;
      }
      if (empty) continue;
      uint32_t a1 = orc_lh_address(orc_bithash1(k), M, p);
      uint32_t a2 = orc_lh_address(orc_bithash2(k), M, p);
      if (a1 != b && a2 != b) {
        *where = b * S + i;
        return 2;
      }
      if (!seen.emplace(k, static_cast<uint32_t>(w >> 32)).second) {
        *where = b * S + i;
        return 3;
      }
      ++live;
    }
  }
  for (uint64_t j = 0; j < stash_n; ++j) {
    uint64_t w = stash[j];
    uint32_t k = static_cast<uint32_t>(w & 0xFFFFFFFFu);
    if (k == EMPTY_KEY) {
      *where = j;
      return 6;
    }
    if (j > 0 && static_cast<uint32_t>(stash[j - 1] & 0xFFFFFFFFu) >= k) {
      // equal keys are duplicates (3); a descent breaks the order (6)
      *where = j;
      return static_cast<uint32_t>(stash[j - 1] & 0xFFFFFFFFu) == k ? 3 : 6;
    }
    if (!seen.emplace(k, static_cast<uint32_t>(w >> 32)).second) {
      *where = j;
      return 3;
    }
    ++live;
  }
  if (live != size_counter) {
    *where = live;
    return 4;
  }
  if (dict) {
    auto& m = static_cast<Dict*>(dict)->m;
    if (m.size() != seen.size()) {
      *where = m.size();
      return 4;
    }
    for (auto& kv : m) {
      auto it = seen.find(kv.first);
      if (it == seen.end() || it->second != kv.second) {
        *where = kv.first;
        return 4;
      }
    }
  }
  if (policy) {
    if (over_grow(policy, live, nb)) return 7;
    if (nb != policy->nb_init && under_shrink(policy, live, nb)) return 7;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// 5. A parallel CPU baseline (not part of the oracle's definition): the bench
//    step's three phases -- n_ins inserts, n_find finds, n_mix mixed ops --
//    on T threads.  Each key belongs to one of T shards (the high bits of
//    k * 0x9E3779B1, a multiplicative hash), and each shard is a
//    std::unordered_map that one thread updates in array order.  Keys of
//    different shards never interact, so every per-op result equals the
//    single map's.  Per phase: the threads first sort the op indices of
//    their slice of the array by shard (order kept), then each thread runs
//    its shard's ops slice by slice.  Returns the seconds the three phases
//    took, thread start-up included.
// ---------------------------------------------------------------------------
double orc_sharded_step(int T, const uint32_t* ik, const uint32_t* iv, uint64_t n_ins,
                        uint8_t* ist, const uint32_t* fk, uint64_t n_find, uint32_t* fv,
                        uint8_t* ff, const uint8_t* mo, const uint32_t* mk, const uint32_t* mv,
                        uint64_t n_mix, uint32_t* mvo, uint8_t* mst) {
  if (T < 1) T = 1;
  std::vector<Dict> shard(T);
  auto owner = [T](uint32_t k) {
    return static_cast<int>((static_cast<uint64_t>(k * 0x9E3779B1u) * static_cast<uint64_t>(T)) >> 32);
  };
  // idx[slice][shard]: the slice's op indices of that shard, in order
  std::vector<std::vector<std::vector<uint32_t>>> idx(T, std::vector<std::vector<uint32_t>>(T));
  auto phase = [&](const uint32_t* keys, uint64_t n, auto&& apply) {
    std::vector<std::thread> th;
    for (int s = 0; s < T; ++s)
      th.emplace_back([&, s] {
        const uint64_t a = n * s / T, b = n * (s + 1) / T;
        for (auto& v : idx[s]) v.clear();
        for (uint64_t i = a; i < b; ++i) idx[s][owner(keys[i])].push_back(static_cast<uint32_t>(i));
      });
    for (auto& t : th) t.join();
    th.clear();
    for (int h = 0; h < T; ++h)
      th.emplace_back([&, h] {
        for (int s = 0; s < T; ++s)
          for (uint32_t i : idx[s][h]) apply(&shard[h], i);
      });
    for (auto& t : th) t.join();
  };
  const auto t0 = std::chrono::steady_clock::now();
  phase(ik, n_ins, [&](Dict* d, uint32_t i) { orc_insert(d, ik + i, iv + i, 1, ist ? ist + i : nullptr); });
  phase(fk, n_find, [&](Dict* d, uint32_t i) {
    orc_find(d, fk + i, 1, fv ? fv + i : nullptr, ff ? ff + i : nullptr);
  });
  phase(mk, n_mix, [&](Dict* d, uint32_t i) {
    orc_execute(d, mo + i, mk + i, mv + i, 1, mvo ? mvo + i : nullptr, mst ? mst + i : nullptr);
  });
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // extern "C"
