// GPU hash map of packed int3 block keys: bucketed (4 x 16 B slots per 64 B bucket), double
// hashing over buckets (probe_step), one thread per operation reading whole buckets.
//
// Guarantees (Sec. 5: concurrent retrieval, insertion and removal succeed and keys stay unique,
// which the paper obtains with per-entry locks and an excess list; here with CAS claims):
//   * A launch changes the table in one way only: finds (read-only), inserts (slots only go
//     free -> key), or erases (slots only go key -> tombstone, or key -> EMPTY in a bucket that
//     already holds an EMPTY slot; the pending insert values that a plain map's erase launch
//     reads first are value fields, which no erase writes).  The host orders the phases of a
//     batch.  A batch's first pass (which
//     writes no slot) runs the finds and sorts the other ops into an insert and an erase list,
//     so each later phase launch covers only its own ops.
//   * A live key never moves (the paper's invariant that entry positions are preserved), so a
//     find needs no lock: it walks the buckets from the key's home bucket until it meets the
//     key or a bucket with a never-used (EMPTY) slot.  Any fixed probe sequence per key keeps
//     these arguments; double hashing keeps it short at high loads.  Tombstones keep chains intact, and an
//     erase makes a slot EMPTY only where a find would stop anyway.
//   * A plain map's batch: the winner of an insert writes its value and final result at once;
//     inserts that met their key take the value in a follow-up launch (skipped when none did),
//     the erase launch (k_finish_erase) for a batch of op lists.
//   * Insert: pass 1 walks the chain to its end; if the key is absent it remembers the first
//     free slot (tombstone or EMPTY).  Pass 2 claims free slots in probe order from there with
//     a 64-bit CAS, re-reading a bucket after a lost CAS.  Because no slot becomes free during
//     an insert launch, two inserters of one key always meet at the same first free slot, so
//     exactly one CAS succeeds and the other sees the key (uniqueness).
//   * The winner writes the value after the claim; duplicates record only the slot and read the
//     value in the follow-up launch, so nobody reads a half-written entry.
#include "vbh_internal.cuh"

namespace vbh {

namespace {

constexpr int kThreads = 256;

// outcome codes of thread_insert
constexpr int kInserted = 1, kExists = 2, kFull = 3;

// An insert in two passes.  Pass 1 (insert_walk, reads only) walks the whole chain to be sure
// the key is absent and notes the first free slot (tombstone or EMPTY) and the bucket it ended
// on; pass 2 (insert_claim) claims free slots in probe order from there with a 64-bit CAS.  A
// launch that writes nothing between the two passes may run them on either side of a barrier.
struct InsertWalk {
  unsigned int first_free, held;
  ulonglong2 s[4];   // the bucket pass 1 ended on
};

// Pass 1: kExists (the key is in the table: *pos_out, *val_out), kFull (no free slot on its
// sequence) or 0 (absent; claim next).
template <int W = 1>
__device__ int insert_walk(const TableView& t, unsigned long long key, unsigned int* pos_out,
                           unsigned int* val_out, InsertWalk& wk) {
  const unsigned int b0 = home_bucket(key, t.bmask, t.hash_fn);
  const unsigned int step = probe_step(key);
  unsigned int first_free = kNone, held = kNone;
  ulonglong2 (&s)[4] = wk.s;   // the bucket pass 1 ended on
  // pass 1: the whole chain, to be sure the key is absent
  if constexpr (W == 1) {
    unsigned int b = b0;
    for (unsigned int probe = 0; probe <= t.bmask; ++probe) {
      load_bucket<false>(&t.slots[4u * b], s);
      held = b;
      bool empty = false;
      int hit = -1, f = -1;   // f: the bucket's first free slot
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        if (s[q].x == key) hit = q;
        if (s[q].x >= kTomb) f = q;
        empty |= s[q].x == kEmpty;
      }
      if (hit >= 0) {
        *pos_out = 4u * b + hit;
        *val_out = (unsigned)bucket_slot(s, hit).y;
        return kExists;
      }
      if (first_free == kNone && f >= 0) first_free = 4u * b + f;
      if (empty) break;
      b = (b + step) & t.bmask;
    }
  } else {
  // W buckets of the chain per round trip, examined in sequence order
  for (unsigned int probe = 0; probe <= t.bmask; probe += W) {
    ulonglong2 g[W][4];
    unsigned int bb[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      bb[w] = (b0 + (probe + w) * step) & t.bmask;
      load_bucket<false>(&t.slots[4u * bb[w]], g[w]);
    }
    bool stop = false;
    unsigned int hit_pos = kNone, hit_val = kNone;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      bool empty = false;
      int hit = -1, f = -1;   // f: the bucket's first free slot
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        if (g[w][q].x == key) hit = q;
        if (g[w][q].x >= kTomb) f = q;
        empty |= g[w][q].x == kEmpty;
      }
      const bool live = !stop && (W == 1 || probe + w <= t.bmask);   // every bucket once
      if (live) {
        if (hit >= 0) {
          hit_pos = 4u * bb[w] + hit;
          hit_val = (unsigned)bucket_slot(g[w], hit).y;
        } else {
          if (first_free == kNone && f >= 0) first_free = 4u * bb[w] + f;
          if (empty) {
            held = bb[w];
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = g[w][q];
          }
        }
        stop = hit >= 0 || empty;
      }
    }
    if (hit_pos != kNone) {
      *pos_out = hit_pos;
      *val_out = hit_val;
      return kExists;
    }
    if (stop) break;
  }
  }
  wk.first_free = first_free;
  wk.held = held;
  return first_free == kNone ? kFull : 0;
}

// Pass 2: kInserted (*pos_out, *observed_out: the slot's previous content), kExists (another
// insert of the key claimed first: *pos_out) or kFull.
__device__ int insert_claim(const TableView& t, unsigned long long key, InsertWalk& wk,
                            unsigned int* pos_out, unsigned long long* observed_out) {
  // pass 2: claim in probe order starting at the first free slot.  The bucket pass 1 ended on
  // is reused for the first attempt: a stale copy only costs a failed CAS and a re-read.
  const unsigned int step = probe_step(key);
  ulonglong2 (&s)[4] = wk.s;
  unsigned int b = wk.first_free >> 2;
  bool have = b == wk.held;
  for (unsigned int steps = 0; steps <= t.bmask;) {
    if (!have) load_bucket<false>(&t.slots[4u * b], s);
    have = false;
    int hit = -1, l = -1;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      if (s[q].x == key) hit = q;
      if (s[q].x >= kTomb) l = q;
    }
    if (hit >= 0) {
      *pos_out = 4u * b + hit;
      return kExists;
    }
    if (l < 0) {
      b = (b + step) & t.bmask;
      ++steps;
      continue;
    }
    const unsigned long long obs = bucket_slot(s, l).x;
    const unsigned long long old = atomicCAS(&t.slots[4u * b + l].key, obs, key);
    if (old == obs) {
      *pos_out = 4u * b + l;
      *observed_out = obs;
      return kInserted;
    }
    if (old == key) {
      *pos_out = 4u * b + l;
      return kExists;
    }
    // another key took the slot: look at the same bucket again
  }
  return kFull;
}

template <int W = 1>
__device__ int thread_insert(const TableView& t, unsigned long long key, unsigned int* pos_out,
                             unsigned long long* observed_out) {
  InsertWalk wk;
  unsigned int val;
  const int r = insert_walk<W>(t, key, pos_out, &val, wk);
  return r ? r : insert_claim(t, key, wk, pos_out, observed_out);
}

// ---------------------------------------------------------------------------- batch compaction
// Every op of a batch is read once: invalid ops get their status; valid inserts and erases go to
// two lists of (op index, packed key), and valid finds run in place.  A CTA takes kPrepOps x
// kThreads ops, each thread kPrepOps of them a CTA width apart (coalesced loads, all in flight at
// once); one warp scan of the packed counts and one reservation per list per CTA place them.
constexpr int kPrepOps = 4;

// Each phase of a batch is a device function that its own kernel launches.  The first pass
// also runs the batch's finds (nothing writes the table before the insert launch), so finds
// need neither a list nor a launch of their own; at 8 CTAs per SM (32 registers, a few bytes
// spilled) a 2^20-op batch is one round of the grid.
#ifndef VBH_PREP_MIN_CTAS
#define VBH_PREP_MIN_CTAS 8
#endif
__device__ __forceinline__ void prep_phase(const TableView& t, DevCounters* cnt,
                                           const unsigned char* ops,
                                           const int* keys3, unsigned int* res,
                                           unsigned char* st, unsigned int n, BatchLists lists,
                                           unsigned int* s_warp, unsigned int* s_base) {
  if (blockIdx.x == 0 && threadIdx.x < 3u) {
    lists.n_next[threadIdx.x] = 0u;   // the previous batch, which used them, has finished
    if (threadIdx.x == 0) cnt->n_exists = 0;   // the batch's insert phase follows
  }
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int span = gridDim.x * blockDim.x * kPrepOps;
  for (unsigned int base = blockIdx.x * blockDim.x * kPrepOps; base < n; base += span) {
    int kind[kPrepOps];   // 0 find, 1 insert, 2 erase, -1 none
    unsigned long long key[kPrepOps];
    unsigned int packed = 0;   // per-kind counts of this thread's ops, 10 bits each
#pragma unroll
    for (int j = 0; j < kPrepOps; ++j) {
      const unsigned int i = base + j * kThreads + threadIdx.x;
      kind[j] = -1;
      key[j] = 0;
      if (i < n) {
        const unsigned char op = ops[i];
        const int x = keys3[3u * i], y = keys3[3u * i + 1], z = keys3[3u * i + 2];
        if (op > kOpErase || !key_ok(x, y, z)) {
          res[i] = kNone;
          st[i] = kStInvalid;
        } else {
          key[j] = pack_key(x, y, z);
          kind[j] = op == kOpFind ? 0 : op == kOpInsert ? 1 : 2;
          if (kind[j] != 0) packed += 1u << (10 * kind[j]);   // finds are not listed
        }
      }
    }
    unsigned int incl = packed;   // inclusive warp scan of the packed counts (a field <= 128)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (unsigned int)d) incl += v;
    }
    if (lane == 31u) s_warp[warp] = incl;
    __syncthreads();
    if (threadIdx.x < 3u) {
      const unsigned int q = threadIdx.x, sh = 10u * q;
      unsigned int* const counter = lists.n + q;
      unsigned int run = 0;
      for (int w = 0; w < kThreads / 32; ++w) run += (s_warp[w] >> sh) & 1023u;
      s_base[q] = run ? atomicAdd(counter, run) : 0u;
    }
    __syncthreads();
    unsigned int pos[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      unsigned int before = 0;   // ops of kind q in the CTA's earlier warps
      for (unsigned int w = 0; w < warp; ++w) before += (s_warp[w] >> (10 * q)) & 1023u;
      pos[q] = s_base[q] + before + (((incl - packed) >> (10 * q)) & 1023u);
    }
#pragma unroll
    for (int j = 0; j < kPrepOps; ++j) {
      const int q = kind[j];
      if (q <= 0) continue;
      const unsigned int k = q == 1 ? pos[1]++ : pos[2]++;
      unsigned int* const idx = q == 1 ? lists.ins_idx : lists.era_idx;
      unsigned long long* const ko = q == 1 ? lists.ins_key : lists.era_key;
      idx[k] = base + j * kThreads + threadIdx.x;
      ko[k] = key[j];
    }
    // the finds: nothing writes the table before the batch's insert launch, so they see it as
    // the batch found it (read-only walks through the non-coherent path)
#pragma unroll
    for (int j = 0; j < kPrepOps; ++j) {
      if (kind[j] != 0) continue;
      const unsigned int i = base + j * kThreads + threadIdx.x;
      unsigned int val;
      const bool hit = thread_find<true>(t, key[j], &val) != kNone;
      res[i] = hit ? val : kNone;
      st[i] = hit ? kStFound : kStNotFound;
    }
    __syncthreads();   // s_warp and s_base are rewritten next round
  }
}

__global__ void __launch_bounds__(kThreads, VBH_PREP_MIN_CTAS)
    k_batch_prep(TableView t, DevCounters* cnt, const unsigned char* ops, const int* keys3,
                 unsigned int* res, unsigned char* st, unsigned int n, BatchLists lists) {
  __shared__ unsigned int s_warp[kThreads / 32], s_base[3];
  prep_phase(t, cnt, ops, keys3, res, st, n, lists, s_warp, s_base);
}

// ------------------------------------------------------------------------------- insert phase
// A list of packed keys, all inserts (a batch's insert list, or a frame's candidate blocks),
// *count_dev entries capped at n_cap (n_cap itself without count_dev); idx (optional) maps list
// entry i to the op whose value, result and status it carries.
__device__ __forceinline__ void insert_phase(const TableView& t, const PoolView& pool,
                                             DevCounters* cnt, const unsigned long long* pkeys,
                                             const unsigned int* count_dev,
                                             const unsigned int* vals, unsigned int* res,
                                             unsigned char* st, unsigned int n_cap,
                                             const unsigned int* idx, unsigned int* sh) {
  unsigned int& s_live = sh[0];
  unsigned int& s_from_empty = sh[1];
  unsigned int& s_from_tomb = sh[2];
  unsigned int& s_err = sh[3];
  if (threadIdx.x == 0) { s_live = 0; s_from_empty = 0; s_from_tomb = 0; s_err = 0; }
  __syncthreads();
  const unsigned int n = count_dev ? min(__ldcg(count_dev), n_cap) : n_cap;
  const unsigned int free_top = pool.max_blocks ? (unsigned)max(cnt->free_top, 0) : 0u;
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int stride = gridDim.x * blockDim.x;
  // whole warps iterate together (warp-aggregated pool pops and counters)
  for (unsigned int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n;
       base += stride) {
    const unsigned int i = base + lane;
    unsigned long long key = 0;
    bool doit = false;
    unsigned int oi = i;   // the op's index in the batch (results, statuses, values)
    if (i < n) {
      key = __ldcg(pkeys + i);
      if (idx) oi = __ldcg(idx + i);
      doit = true;
    }
    int outcome = 0;
    unsigned int pos = kNone;
    unsigned long long observed = 0;
    if (doit) outcome = thread_insert(t, key, &pos, &observed);
    const bool won = outcome == kInserted;
    if (pool.max_blocks) {
      unsigned int k = warp_append(&cnt->n_popped, won, 0xFFFFFFFFu);
      if (won) {
        if (k < free_top) {
          unsigned int p = pool.stack[free_top - 1u - k];
          t.slots[pos].val = p;
          pool.pkeys[p] = key;
          pool.state[p] = kFresh;
          uint4* m = reinterpret_cast<uint4*>(pool.masks + 32u * p);
#pragma unroll
          for (int q = 0; q < 8; ++q) m[q] = make_uint4(0u, 0u, 0u, 0u);
        } else {
          t.slots[pos].val = kPoolFail;
        }
      }
    } else if (won) {
      const unsigned int v = vals ? vals[oi] : 0u;
      t.slots[pos].val = v;
      pos = v;   // a plain map's winner knows its value: the result is final
    }
    const unsigned int n_won = __popc(__ballot_sync(0xFFFFFFFFu, won));
    const unsigned int n_empty = __popc(__ballot_sync(0xFFFFFFFFu, won && observed == kEmpty));
    const unsigned int n_ex = __popc(__ballot_sync(0xFFFFFFFFu, outcome == kExists));
    if (lane == 0 && n_won) {
      atomicAdd(&s_live, n_won);
      if (n_empty) atomicAdd(&s_from_empty, n_empty);
      if (n_won > n_empty) atomicAdd(&s_from_tomb, n_won - n_empty);
    }
    if (lane == 0 && n_ex && !pool.max_blocks) atomicAdd(&cnt->n_exists, n_ex);
    if (doit) {
      res[oi] = pos;
      st[oi] = outcome == kInserted ? kStInserted : outcome == kExists ? kStExists : kStCapacity;
      if (outcome == kFull) atomicOr(&s_err, kErrTable);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_live) atomicAdd(&cnt->n_live, s_live);
    if (s_from_empty) atomicSub(&cnt->n_empty, s_from_empty);
    if (s_from_tomb) atomicSub(&cnt->n_tomb, s_from_tomb);
    if (s_err) atomicOr(&cnt->err, s_err);
  }
}

__global__ void __launch_bounds__(kThreads) k_insert(TableView t, PoolView pool,
                                                     DevCounters* cnt,
                                                     const unsigned long long* pkeys,
                                                     const unsigned int* count_dev,
                                                     const unsigned int* vals, unsigned int* res,
                                                     unsigned char* st, unsigned int n_cap,
                                                     const unsigned int* idx) {
  __shared__ unsigned int sh[4];
  insert_phase(t, pool, cnt, pkeys, count_dev, vals, res, st, n_cap, idx, sh);
}

// Resolve every insert's value once all claims are visible (the inserts are the first
// *count_dev ops, capped at n_cap, or the ops idx lists); undo claims whose pool pop failed;
// optionally append each distinct pool index to a frame's touched list (epoch de-duplication).
__device__ __forceinline__ void finish_phase(const TableView& t, const PoolView& pool,
                                             DevCounters* cnt, const unsigned int* count_dev,
                                             unsigned int* res, unsigned char* st,
                                             unsigned int n_cap, unsigned int* touched,
                                             unsigned long long* tkey, float2* tdepth,
                                             unsigned int* n_touched, const FrameCtl* ctl,
                                             const unsigned int* idx, unsigned int* sh) {
  // A plain map's winners wrote their final results; only inserts that met their key (whose
  // value another thread may still have been writing) are left, and usually there are none.
  // (Every thread of the grid reads the same count, so a CTA leaves as a whole.)
  const bool plain = pool.max_blocks == 0;
  if (plain && !touched && *reinterpret_cast<volatile unsigned int*>(&cnt->n_exists) == 0) return;
  unsigned int& s_undo = sh[0];
  unsigned int& s_new = sh[1];
  unsigned int& s_err = sh[2];
  if (threadIdx.x == 0) { s_undo = 0; s_new = 0; s_err = 0; }
  __syncthreads();
  const unsigned int n = count_dev ? min(__ldcg(count_dev), n_cap) : n_cap;
  const unsigned int epoch = ctl ? ctl->epoch_touch : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0 && pool.max_blocks) {
    int popped = (int)cnt->n_popped;
    cnt->free_top = max(cnt->free_top - popped, 0);
    cnt->n_popped = 0;
  }
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (n + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int j = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int p = kNone;
    bool fresh_win = false;
    if (j < n) {
      const unsigned int i = idx ? __ldcg(idx + j) : j;   // the insert's index in the batch
      unsigned char s = __ldcg(st + i);
      if (s == kStExists || (s == kStInserted && !plain)) {
        unsigned int pos = __ldcg(res + i);
        unsigned int v = __ldcg(&t.slots[pos].val);
        if (!plain && v == kPoolFail) {
          if (s == kStInserted) {
            t.slots[pos].key = kTomb;
            atomicAdd(&s_undo, 1u);
          }
          st[i] = kStCapacity;
          res[i] = kNone;
          atomicOr(&s_err, kErrPool);
        } else {
          res[i] = v;
          p = v;
          fresh_win = s == kStInserted;
        }
      } else if (s == kStCapacity) {
        res[i] = kNone;
      }
    }
    if (touched) {
      bool first = false;
      if (p != kNone) first = atomicExch(&pool.mark[p], epoch) != epoch;
      unsigned int k = warp_append(n_touched, first, 0xFFFFFFFFu);
      if (first) {
        // the record the fusion kernel reads: index + fresh bit, key, origin camera depth
        const unsigned long long key = pool.pkeys[p];
        touched[k] = p | ((pool.state[p] & kFresh) ? kTouchedFresh : 0u);
        if (tkey) tkey[k] = key;
        if (tdepth) tdepth[k] = block_depth(ctl->fp, unpack_key(key));
      }
      if (fresh_win) atomicAdd(&s_new, 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_undo) {
      atomicSub(&cnt->n_live, s_undo);
      atomicAdd(&cnt->n_tomb, s_undo);
    }
    if (s_new) {
      atomicAdd(&cnt->n_new, s_new);
      atomicAdd(&cnt->tot_new, (unsigned long long)s_new);
    }
    if (s_err) atomicOr(&cnt->err, s_err);
  }
}

__global__ void __launch_bounds__(kThreads) k_insert_finish(TableView t, PoolView pool,
                                                            DevCounters* cnt,
                                                            const unsigned int* count_dev,
                                                            unsigned int* res, unsigned char* st,
                                                            unsigned int n_cap,
                                                            unsigned int* touched,
                                                            unsigned long long* tkey,
                                                            float2* tdepth,
                                                            unsigned int* n_touched,
                                                            const FrameCtl* ctl,
                                                            const unsigned int* idx) {
  __shared__ unsigned int sh[3];
  finish_phase(t, pool, cnt, count_dev, res, st, n_cap, touched, tkey, tdepth, n_touched, ctl,
               idx, sh);
}

// -------------------------------------------------------------------------------- erase phase
// The batch's erase list (packed keys ekeys and op indices eidx from k_batch_prep, *count_dev
// entries, capped at n_cap).
__device__ __forceinline__ void erase_phase(const TableView& t, const PoolView& pool,
                                            DevCounters* cnt, const unsigned long long* ekeys,
                                            const unsigned int* eidx,
                                            const unsigned int* count_dev, unsigned int* res,
                                            unsigned char* st, unsigned int n_cap,
                                            unsigned int* sh) {
  unsigned int& s_erased = sh[0];
  unsigned int& s_emptied = sh[1];
  if (threadIdx.x == 0) { s_erased = 0; s_emptied = 0; }
  __syncthreads();
  const unsigned int n = min(__ldcg(count_dev), n_cap);
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n;
       base += stride) {
    const unsigned int i = base + lane;
    unsigned long long key = 0;
    unsigned int oi = 0;   // the op's index in the batch
    const bool doit = i < n;
    if (doit) {
      key = __ldcg(ekeys + i);
      oi = __ldcg(eidx + i);
    }
    int how = 0;
    unsigned int val = kNone;
    if (doit) {
      bool bucket_empty = false;
      const unsigned int pos = thread_find(t, key, &val, &bucket_empty);
      if (pos != kNone) how = erase_found(t, pos, key, bucket_empty);
    }
    const bool erased = how != 0;
    const bool push = erased && pool.max_blocks;
    unsigned int k = warp_append(reinterpret_cast<unsigned int*>(&cnt->free_top), push,
                                 0xFFFFFFFFu);
    if (push) {
      pool.stack[k] = val;
      pool.pkeys[val] = kEmpty;
      pool.state[val] = 0u;
      pool.seq[val] = 0u;
    }
    if (doit) {
      res[oi] = erased ? val : kNone;
      st[oi] = erased ? kStErased : kStNotFound;
    }
    const unsigned int n_er = __popc(__ballot_sync(0xFFFFFFFFu, erased));
    const unsigned int n_em = __popc(__ballot_sync(0xFFFFFFFFu, how == 1));
    if (lane == 0 && n_er) {
      atomicAdd(&s_erased, n_er);
      if (n_em) atomicAdd(&s_emptied, n_em);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_erased) {
    atomicSub(&cnt->n_live, s_erased);
    if (s_emptied) atomicAdd(&cnt->n_empty, s_emptied);
    if (s_erased > s_emptied) atomicAdd(&cnt->n_tomb, s_erased - s_emptied);
  }
}

__global__ void __launch_bounds__(kThreads) k_erase(TableView t, PoolView pool, DevCounters* cnt,
                                                    const unsigned long long* ekeys,
                                                    const unsigned int* eidx,
                                                    const unsigned int* count_dev,
                                                    unsigned int* res, unsigned char* st,
                                                    unsigned int n_cap) {
  __shared__ unsigned int sh[2];
  erase_phase(t, pool, cnt, ekeys, eidx, count_dev, res, st, n_cap, sh);
}

// A plain map's last two phases in one launch: the inserts that met their key read its value
// (usually none did), then the erases run.  They touch disjoint fields -- the pending inserts
// read value fields, which an erase never writes -- so they need no barrier between them; a
// pool-backed map keeps the separate launches (its finish phase settles the free stack the
// erases push to).
__global__ void __launch_bounds__(kThreads) k_finish_erase(TableView t, PoolView pool,
                                                           DevCounters* cnt,
                                                           const unsigned int* ins_count,
                                                           const unsigned int* ins_idx,
                                                           const unsigned long long* ekeys,
                                                           const unsigned int* eidx,
                                                           const unsigned int* era_count,
                                                           unsigned int* res, unsigned char* st,
                                                           unsigned int n_cap) {
  __shared__ unsigned int sh_f[3], sh_e[2];
  finish_phase(t, pool, cnt, ins_count, res, st, n_cap, nullptr, nullptr, nullptr, nullptr,
               nullptr, ins_idx, sh_f);
  erase_phase(t, pool, cnt, ekeys, eidx, era_count, res, st, n_cap, sh_e);
}

// ------------------------------------------------------------------------- small batch
// A small batch of a plain map is bound by the latency of its phases, not by bandwidth.
// k_batch_small runs it in one cooperative launch (every CTA resident) with one thread per op
// that keeps its op and key in registers, so there are no op lists, and three phases separated
// by two grid barriers:
//   1. every op is read and checked; the finds run (nothing writes the table yet, so they see
//      it as the batch found it), so do the inserts' read-only walks (a key already in the
//      table gets its final result here), and the erases prefetch the first buckets of their
//      probe sequences to L2;
//   2. the inserts of absent keys claim their slots from where their walks ended; a winner
//      writes its value and its final result;
//   3. the inserts that met their key read its value (every winner wrote its value before the
//      barrier, and an erase leaves the value field alone), and the erases run.
// Results, statuses and counters are those of the phased launches.  A barrier waits at most
// ~1 s (GPU global timer); one that gives up raises the sticky timeout flag and lets its CTA go.
// Grid barrier on a counter that only grows: every CTA adds one on arrival (no reply waited
// for) and waits until the counter reaches `target` (the count before this launch, which the
// host keeps, plus the CTAs x the barriers so far), so the last arrival releases the others
// without a second round trip.
__device__ __forceinline__ void grid_barrier(DevCounters* cnt, unsigned int target) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();   // the CTA's writes before its arrival
    atomicAdd(&cnt->gbar_arrive, 1u);
    volatile unsigned int* c = &cnt->gbar_arrive;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while ((int)(*c - target) < 0) {
      __nanosleep(20);
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) {
        atomicOr(&cnt->err, kErrTimeout);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

#ifndef VBH_SMALL_BATCH_PROBES
#define VBH_SMALL_BATCH_PROBES 2
#endif
// Buckets of a probe sequence loaded per round trip in a small batch, whose phases last as long
// as their longest walk (at load 0.7 a miss reads ~1.7 buckets on average, the longest of 2^16
// walks ten or more); phased batches of many ops are bound by bandwidth and load one at a time.
constexpr int kSmallProbes = VBH_SMALL_BATCH_PROBES;
#ifndef VBH_SMALL_PDL
#define VBH_SMALL_PDL 1   // launch small batches with programmatic stream serialisation
#endif

__global__ void __launch_bounds__(kThreads) k_batch_small(TableView t, DevCounters* cnt,
                                                          const unsigned char* ops,
                                                          const int* keys3,
                                                          const unsigned int* vals,
                                                          unsigned int* res, unsigned char* st,
                                                          unsigned int n,
                                                          unsigned int* lists_next,
                                                          unsigned int bar_base) {
#if VBH_SMALL_PDL
  // launched with programmatic serialisation: everything the previous grid in the stream wrote
  // is visible after this wait; the next batch's launch may start now (it waits likewise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
  // inserts won, won from EMPTY, won from a tombstone, error bits; erased, erased to EMPTY
  __shared__ unsigned int sh[6];
  const unsigned int i = blockIdx.x * kThreads + threadIdx.x;
  const unsigned int lane = threadIdx.x & 31u;
  // the list counts a following phased batch uses start at zero (its predecessor zeroes them)
  if (blockIdx.x == 0 && threadIdx.x < 3u) lists_next[threadIdx.x] = 0u;
  if (threadIdx.x < 6u) sh[threadIdx.x] = 0u;
  int kind = -1;   // kOpFind, kOpInsert or kOpErase
  unsigned long long key = 0;
  if (i < n) {
    const unsigned char op = ops[i];
    const int x = keys3[3u * i], y = keys3[3u * i + 1], z = keys3[3u * i + 2];
    if (op > kOpErase || !key_ok(x, y, z)) {
      res[i] = kNone;
      st[i] = kStInvalid;
    } else {
      key = pack_key(x, y, z);
      kind = op;
    }
  }
  // an insert's walk reads only, so it runs here beside the finds; the table does not change
  // before its claim in the next phase
  InsertWalk wk;
  int outcome = 0;
  unsigned int pos = kNone;
  if (kind == kOpFind) {
    unsigned int val;
    const bool hit = thread_find<false, kSmallProbes>(t, key, &val) != kNone;
    res[i] = hit ? val : kNone;
    st[i] = hit ? kStFound : kStNotFound;
  } else if (kind == kOpInsert) {
    unsigned int val = kNone;
    outcome = insert_walk<kSmallProbes>(t, key, &pos, &val, wk);
    if (outcome == kExists) {   // in the table before the batch: its value is final
      res[i] = val;
      st[i] = kStExists;
    } else if (outcome == kFull) {
      res[i] = kNone;
      st[i] = kStCapacity;
      atomicOr(&sh[3], kErrTable);
    }
  } else if (kind == kOpErase) {
    const unsigned int b0 = home_bucket(key, t.bmask, t.hash_fn), step = probe_step(key);
#pragma unroll
    for (int w = 0; w < kSmallProbes; ++w) {
      const Slot* b = &t.slots[4u * ((b0 + w * step) & t.bmask)];
      asm volatile("prefetch.global.L2 [%0];" ::"l"(b));
    }
  }
  grid_barrier(cnt, bar_base + gridDim.x);

  unsigned long long observed = 0;
  bool pending = false;   // met its key claimed by another insert of this batch: value next phase
  if (kind == kOpInsert && outcome == 0) {
    outcome = insert_claim(t, key, wk, &pos, &observed);
    pending = outcome == kExists;
    if (outcome == kInserted) {
      const unsigned int v = vals ? vals[i] : 0u;
      t.slots[pos].val = v;
      res[i] = v;
      st[i] = kStInserted;
    } else if (outcome == kFull) {
      res[i] = kNone;
      st[i] = kStCapacity;
      atomicOr(&sh[3], kErrTable);
    }
  }
  const bool won = outcome == kInserted;
  const unsigned int n_won = __popc(__ballot_sync(0xFFFFFFFFu, won));
  const unsigned int n_emp = __popc(__ballot_sync(0xFFFFFFFFu, won && observed == kEmpty));
  if (lane == 0 && n_won) {
    atomicAdd(&sh[0], n_won);
    if (n_emp) atomicAdd(&sh[1], n_emp);
    if (n_won > n_emp) atomicAdd(&sh[2], n_won - n_emp);
  }
  grid_barrier(cnt, bar_base + 2u * gridDim.x);

  if (pending) {
    res[i] = __ldcg(&t.slots[pos].val);
    st[i] = kStExists;
  }
  int how = 0;
  if (kind == kOpErase) {
    bool bucket_empty = false;
    unsigned int val = kNone;
    const unsigned int p = thread_find<false, kSmallProbes>(t, key, &val, &bucket_empty);
    if (p != kNone) how = erase_found(t, p, key, bucket_empty);
    res[i] = how ? val : kNone;
    st[i] = how ? kStErased : kStNotFound;
  }
  const unsigned int n_er = __popc(__ballot_sync(0xFFFFFFFFu, how != 0));
  const unsigned int n_em = __popc(__ballot_sync(0xFFFFFFFFu, how == 1));
  if (lane == 0 && n_er) {
    atomicAdd(&sh[4], n_er);
    if (n_em) atomicAdd(&sh[5], n_em);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ins = sh[0], ins_e = sh[1], ins_t = sh[2], er = sh[4], er_e = sh[5];
    if (ins != er) atomicAdd(&cnt->n_live, ins - er);   // modulo 2^32: a net change
    if (er_e != ins_e) atomicAdd(&cnt->n_empty, er_e - ins_e);
    if (er - er_e != ins_t) atomicAdd(&cnt->n_tomb, (er - er_e) - ins_t);
    if (sh[3]) atomicOr(&cnt->err, sh[3]);
  }
}

// ------------------------------------------------------------------------------------ rebuild
// The table has been filled with EMPTY; re-insert every live entry of the shadow copy.  Keys are
// unique, so each one simply claims the first EMPTY slot along its probe sequence.
__global__ void __launch_bounds__(kThreads) k_rebuild(TableView t, const Slot* shadow,
                                                      unsigned int n_slots, DevCounters* cnt) {
  __shared__ unsigned int s_live;
  if (threadIdx.x == 0) s_live = 0;
  __syncthreads();
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += stride) {
    ulonglong2 s = __ldg(reinterpret_cast<const ulonglong2*>(&shadow[i]));
    if (s.x >= kTomb) continue;
    unsigned int b = home_bucket(s.x, t.bmask, t.hash_fn);
    const unsigned int step = probe_step(s.x);
    bool done = false;
    for (unsigned int probe = 0; probe <= t.bmask && !done; ++probe, b = (b + step) & t.bmask) {
      for (unsigned int l = 0; l < 4u && !done; ++l) {
        Slot* dst = &t.slots[4u * b + l];
        if (__ldcg(&dst->key) != kEmpty) continue;
        if (atomicCAS(&dst->key, kEmpty, s.x) == kEmpty) {
          dst->val = (unsigned int)s.y;
          done = true;
        }
      }
    }
    atomicAdd(&s_live, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_live) atomicAdd(&cnt->rebuild_n, s_live);
}

__global__ void k_rebuild_counters(DevCounters* cnt, unsigned int n_slots) {
  cnt->n_live = cnt->rebuild_n;
  cnt->n_tomb = 0;
  cnt->n_empty = n_slots - cnt->rebuild_n;
  cnt->rebuild_n = 0;
}

// --------------------------------------------------------------------- dump / load utilities
__global__ void k_dump_table(TableView t, unsigned int n_slots, unsigned long long* out_keys,
                             unsigned int* out_vals, unsigned int cap, unsigned int* out_n) {
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (n_slots + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    ulonglong2 s = make_ulonglong2(kEmpty, 0ull);
    if (i < n_slots) s = __ldg(reinterpret_cast<const ulonglong2*>(&t.slots[i]));
    bool live = i < n_slots && s.x < kTomb;
    unsigned int k = warp_append(out_n, live, 0xFFFFFFFFu);
    if (live && k < cap) {
      out_keys[k] = s.x;
      out_vals[k] = (unsigned int)s.y;
    }
  }
}

__global__ void k_gather_blocks(PoolView pool, const unsigned int* idx, unsigned int n,
                                float* tsdf, float* w) {
  for (unsigned int b = blockIdx.x; b < n; b += gridDim.x) {
    unsigned int p = idx[b];
    bool fresh = pool.state[p] & kFresh;
    for (unsigned int v = threadIdx.x; v < 512u; v += blockDim.x) {
      float2 x = fresh ? make_float2(0.f, 0.f) : pool.vox[512ull * p + v];
      if (tsdf) tsdf[512ull * b + v] = x.x;
      if (w) w[512ull * b + v] = x.y;
    }
  }
}

__global__ void k_scatter_blocks(PoolView pool, const unsigned int* idx, unsigned int n,
                                 const float* tsdf, const float* w) {
  for (unsigned int b = blockIdx.x; b < n; b += gridDim.x) {
    unsigned int p = idx[b];
    if (p >= pool.max_blocks) continue;
    for (unsigned int v = threadIdx.x; v < 512u; v += blockDim.x)
      pool.vox[512ull * p + v] = make_float2(tsdf[512ull * b + v], w[512ull * b + v]);
    __syncthreads();
    if (threadIdx.x == 0) pool.state[p] &= ~kFresh;
  }
}

// Sign / weight bit masks of whole blocks from their voxel data (after an upload).
__global__ void k_block_masks(PoolView pool, const unsigned int* idx, unsigned int n) {
  const unsigned int warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  for (unsigned int b = blockIdx.x; b < n; b += gridDim.x) {
    unsigned int p = idx[b];
    if (p >= pool.max_blocks) continue;
    for (unsigned int w = warp; w < 16u; w += blockDim.x >> 5) {
      float2 x = pool.vox[512ull * p + 32u * w + lane];
      unsigned int neg = __ballot_sync(0xFFFFFFFFu, x.x < 0.f);
      unsigned int val = __ballot_sync(0xFFFFFFFFu, x.y > 0.f);
      if (lane == 0) {
        pool.masks[32u * p + w] = neg;
        pool.masks[32u * p + 16u + w] = val;
      }
    }
  }
}

__global__ void k_pack_keys(const int* keys3, unsigned int n, unsigned long long* out) {
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = pack_key(keys3[3u * i], keys3[3u * i + 1], keys3[3u * i + 2]);
}

}  // namespace

#define VBH_GRID(kernel, threads)                                  \
  static const int grid_##kernel = persistent_grid(kernel, threads, L.sms)

// A batch of n ops needs no more CTAs than it has ops per CTA-wide round (small batches would
// otherwise launch the whole persistent grid for a handful of ops).
inline unsigned int fit_grid(int persistent, unsigned int n) {
  const unsigned int need = (n + kThreads - 1u) / kThreads;
  return need < 1u ? 1u : (need < (unsigned int)persistent ? need : (unsigned int)persistent);
}

void launch_hash_find(const Launch& L, TableView t, DevCounters* cnt, const unsigned char* ops,
                      const int* keys3, unsigned int* res, unsigned char* st, unsigned int n,
                      BatchLists lists) {
  VBH_GRID(k_batch_prep, kThreads);
  k_batch_prep<<<fit_grid(grid_k_batch_prep, (n + kPrepOps - 1u) / kPrepOps), kThreads, 0,
                 L.stream>>>(t, cnt, ops, keys3, res, st, n, lists);
}
void launch_hash_insert(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                        const unsigned long long* pkeys, const unsigned int* count_dev,
                        const unsigned int* vals, unsigned int* res, unsigned char* st,
                        unsigned int n, const unsigned int* idx) {
  VBH_GRID(k_insert, kThreads);
  k_insert<<<fit_grid(grid_k_insert, n), kThreads, 0, L.stream>>>(t, pool, cnt, pkeys, count_dev,
                                                                    vals, res, st, n, idx);
}
void launch_hash_insert_finish(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                               const unsigned int* count_dev, unsigned int* res,
                               unsigned char* st, unsigned int n, unsigned int* touched,
                               unsigned long long* tkey, float2* tdepth,
                               unsigned int* n_touched, const FrameCtl* ctl,
                               const unsigned int* idx) {
  VBH_GRID(k_insert_finish, kThreads);
  k_insert_finish<<<fit_grid(grid_k_insert_finish, n), kThreads, 0, L.stream>>>(
      t, pool, cnt, count_dev, res, st, n, touched, tkey, tdepth, n_touched, ctl, idx);
}
void launch_hash_finish_erase(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                              unsigned int* res, unsigned char* st, unsigned int n,
                              BatchLists lists) {
  VBH_GRID(k_finish_erase, kThreads);
  k_finish_erase<<<fit_grid(grid_k_finish_erase, n), kThreads, 0, L.stream>>>(
      t, pool, cnt, lists.n + 1, lists.ins_idx, lists.era_key, lists.era_idx, lists.n + 2, res,
      st, n);
}
void launch_hash_erase(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       unsigned int* res, unsigned char* st, unsigned int n, BatchLists lists) {
  VBH_GRID(k_erase, kThreads);
  k_erase<<<fit_grid(grid_k_erase, n), kThreads, 0, L.stream>>>(
      t, pool, cnt, lists.era_key, lists.era_idx, lists.n + 2, res, st, n);
}
int small_batch_grid(const Launch& L) {
  static const int grid = persistent_grid(k_batch_small, kThreads, L.sms);
  return grid;
}
bool small_batch_fits(const Launch& L, unsigned int n) {
  return n > 0 && (n + kThreads - 1u) / kThreads <= (unsigned int)small_batch_grid(L);
}
cudaError_t launch_hash_batch_small(const Launch& L, TableView t, DevCounters* cnt,
                                    const unsigned char* ops, const int* keys3,
                                    const unsigned int* vals, unsigned int* res,
                                    unsigned char* st, unsigned int n, unsigned int* lists_next,
                                    unsigned int* bar_base) {
  if (!small_batch_fits(L, n)) return cudaErrorInvalidValue;
  const unsigned int grid = (n + kThreads - 1u) / kThreads;   // one thread per op
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = VBH_SMALL_PDL ? 2 : 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch_small, t, cnt, ops, keys3, vals, res,
                                           st, n, lists_next, *bar_base);
  if (e == cudaSuccess) *bar_base += 2u * grid;   // the counter after the launch's two barriers
  return e;
}
void launch_rebuild(const Launch& L, TableView t, const Slot* shadow, unsigned int n_slots,
                    DevCounters* cnt) {
  VBH_GRID(k_rebuild, kThreads);
  k_rebuild<<<grid_k_rebuild, kThreads, 0, L.stream>>>(t, shadow, n_slots, cnt);
  k_rebuild_counters<<<1, 1, 0, L.stream>>>(cnt, n_slots);
}
void launch_dump_table(const Launch& L, TableView t, unsigned int n_slots,
                       unsigned long long* out_keys, unsigned int* out_vals, unsigned int cap,
                       unsigned int* out_n) {
  VBH_GRID(k_dump_table, kThreads);
  k_dump_table<<<grid_k_dump_table, kThreads, 0, L.stream>>>(t, n_slots, out_keys, out_vals,
                                                              cap, out_n);
}
void launch_gather_blocks(const Launch& L, PoolView pool, const unsigned int* idx,
                          unsigned int n, float* tsdf, float* w) {
  VBH_GRID(k_gather_blocks, 128);
  if (n) k_gather_blocks<<<grid_k_gather_blocks, 128, 0, L.stream>>>(pool, idx, n, tsdf, w);
}
void launch_scatter_blocks(const Launch& L, PoolView pool, const unsigned int* idx,
                           unsigned int n, const float* tsdf, const float* w) {
  VBH_GRID(k_scatter_blocks, 128);
  if (n) k_scatter_blocks<<<grid_k_scatter_blocks, 128, 0, L.stream>>>(pool, idx, n, tsdf, w);
}
void launch_block_masks(const Launch& L, PoolView pool, const unsigned int* idx, unsigned int n) {
  VBH_GRID(k_block_masks, 128);
  if (n) k_block_masks<<<grid_k_block_masks, 128, 0, L.stream>>>(pool, idx, n);
}
void launch_pack_keys(const Launch& L, const int* keys3, unsigned int n,
                      unsigned long long* out) {
  VBH_GRID(k_pack_keys, kThreads);
  if (n) k_pack_keys<<<grid_k_pack_keys, kThreads, 0, L.stream>>>(keys3, n, out);
}

}  // namespace vbh
