// Device-resident request loop for multi-client delta streaming (the server side of Sec. 4.2:
// clients ask for the MC blocks changed since their last update).  The requests, results and
// versions are those of serve.cu (a client is one change sequence number v on the device; a
// request admitted at snapshot sigma returns the blocks whose newest refresh is in (v, sigma],
// or the whole model for v = 0), but admission, batching and completion run on the GPU:
//
//   host  --(mapped ring: id, client)-->  scheduler warp  --(chunk ring, tickets)-->  workers
//   host  <--(mapped ring: completions)--  worker that finishes a request's last tile
//
// One persistent kernel, launched cooperatively (every CTA resident at once) on a non-blocking
// stream of its own, runs beside the frames on the volume's stream.  Warp 0 of CTA 0 is the
// scheduler: it reads new requests from the mapped request ring into a device pending queue,
// admits them in arrival order (one request per client at a time, a free slot, and room for
// the request's worst case in the stream buffer, taken from a ring allocator), cuts the
// admitted ranges into chunks and publishes chunks of all active requests in rounds, smallest
// remainder first, whenever the workers' backlog runs low.  Every other warp is a worker: it
// takes the next tile (32 change records, 64 for a request with many left) by ticket (one
// atomic), waits until that tile has been published, finds its chunk, and serves the tile.
// The worker that finishes a request's last tile moves the client to its new version and
// writes the completion to mapped host memory.
//
// Concurrency with frames.  Fusion and MC extraction keep running on the volume's stream, so
// a block can be refreshed again while a worker copies its indices.  The MC extraction (mc.cu)
// stores a refresh's sequence number before its indices when a loop runs; a worker reads the
// sequence number, copies the 512 B, fences, and reads it again: a block whose number changed
// is dropped from this result (its newer refresh is after sigma, so the client's next request
// carries it).  Table rebuilds are deferred while the loop runs (entries never move under a
// find).  All state shared with concurrent kernels is read through L2 (ld.cg / volatile).
//
// Bounded waits.  The scheduler stops the loop with VBH_ERR_TIMEOUT once the host has been
// silent (no loop call) for the configured time, measured on the GPU's global timer; a worker
// waiting for work stops when the scheduler's heartbeat has not moved for twice that time.
#include <time.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace vbh {

namespace {

// One CTA per SM of 8 warps, each copying 16 blocks at a time (64 KB of staging per CTA).  The
// frames' kernels must find room beside the loop: with the smallest shared-memory configuration
// that holds a larger loop CTA, a frame kernel's CTA did not fit and the frames waited for the
// loop to end (12 warps x 8 blocks looked faster only because the frames were kept out).
#ifndef VBH_LOOP_THREADS
#define VBH_LOOP_THREADS 256
#endif
constexpr int kLoopThreads = VBH_LOOP_THREADS;
#ifndef VBH_LOOP_CARVEOUT
#define VBH_LOOP_CARVEOUT -1
#endif
constexpr int kLoopCarveout = VBH_LOOP_CARVEOUT;   // % of the SM's shared memory (-1: driver's choice)
constexpr int kLoopWarps = kLoopThreads / 32;
constexpr unsigned int kLoopMaxSlots = 64u;
constexpr unsigned int kChunkRing = 1024u;    // chunks published and not yet finished
constexpr unsigned int kRegionRing = 8192u;   // stream-buffer regions not yet released
constexpr unsigned int kRecHdr = 16u, kRecPay = 512u, kRecAll = 528u;
constexpr unsigned int kErrOverrun = 2u, kErrCap = 4u;   // as kServeErr* (serve.cu)
#ifndef VBH_LOOP_MAX_NAP
#define VBH_LOOP_MAX_NAP 2048u   // longest sleep (ns) between a waiting worker's polls
#endif
#ifndef VBH_LOOP_STAGE_BLOCKS
#define VBH_LOOP_STAGE_BLOCKS 16
#endif
constexpr unsigned int kStageBlocks = VBH_LOOP_STAGE_BLOCKS;   // blocks a worker copies at once
#ifndef VBH_LOOP_TILE_RECS
#define VBH_LOOP_TILE_RECS 32
#endif
constexpr unsigned int kTileRecs = VBH_LOOP_TILE_RECS;   // change records per tile
#ifndef VBH_LOOP_BIG_TILE_RECS
#define VBH_LOOP_BIG_TILE_RECS 64
#endif
#ifndef VBH_LOOP_BIG_REMAIN
#define VBH_LOOP_BIG_REMAIN 4096u   // remaining records from which a chunk has long tiles
#endif
constexpr unsigned int kBigTileRecs = VBH_LOOP_BIG_TILE_RECS;
constexpr unsigned int kBigRemain = VBH_LOOP_BIG_REMAIN;
static_assert(kTileRecs >= 1u && (kTileRecs <= 32u || kTileRecs % 32u == 0u) &&
                  kBigTileRecs >= 1u && (kBigTileRecs <= 32u || kBigTileRecs % 32u == 0u),
              "a tile is served 32 records (one per lane) at a time");

// Host -> device (mapped host memory).
struct LoopReq {
  unsigned int id, client;
};
// A request slot of the host -> device ring: one 64-bit word, the request's tag (its id) in
// the high half and its client in the low half, written by the host in one store.  Tags run
// 1, 2, .., 0x7FFFFFFF, 1, ..: the slot of the next request holds the next tag once it is
// written, so one read both finds and fetches it (no separate tail to read first).
__host__ __device__ __forceinline__ unsigned int next_tag(unsigned int t) {
  return t == 0x7FFFFFFFu ? 1u : t + 1u;
}
// Device -> host (mapped host memory); tok = completion number + 1, written last.
struct LoopDone {
  unsigned int id, client, n_records, flags;
  unsigned int v0, v1, region, cap;
  unsigned long long off;
  unsigned int tok;
  unsigned int dev_ns;   // GPU timer from admission to publication (saturating)
};
// Words the host writes.
struct LoopHostIn {
  unsigned int req_tail;    // requests written (for inspection; the loop reads the slots)
  unsigned int rel_tail;    // releases written
  unsigned int done_read;   // completions consumed
  unsigned int beat;        // changes on every host call (sign of life)
  unsigned int stop;        // 1: stop the loop
  unsigned int pad[11];
};
// Words the device writes.
struct LoopHostOut {
  unsigned int req_head;    // requests taken off the ring
  unsigned int rel_head;    // releases taken off the ring
  unsigned int status;      // 0, or the vbh_status the loop stopped with
  unsigned int exited;      // 1 once the scheduler has left its loop
  unsigned int pad[12];
};

struct ReqSlot {            // a request in flight (its bit clear in free_mask)
  unsigned int id, client, scan;
  unsigned int sigma, cap, v0, v1, flags;
  unsigned int region, chunks_total;
  unsigned int chunks_done;    // atomic (workers)
  unsigned int rec_count;      // atomic (workers)
  unsigned int err;            // atomic (workers)
  unsigned long long off;      // byte offset of its region in the stream buffer
  unsigned long long t_adm;    // GPU timer at admission
};

struct Chunk {
  unsigned long long start_tile;   // first ticket of the chunk
  unsigned int idx;                // absolute chunk number (ring position check)
  unsigned int tiles, slot, lo, hi;
  unsigned int finished;           // atomic: tiles served
  unsigned int recs;               // change records per tile
};

struct Region {
  unsigned long long start, bytes;   // monotonic allocator positions
  unsigned int freed, pad;
};

struct LoopDev {
  // shared between the scheduler and the workers
  unsigned long long next_ticket;   // atomic: tiles handed out
  unsigned long long end_tile;      // tiles published
  unsigned long long free_mask;     // bit i: slot i free (workers set, the scheduler clears)
  unsigned int chunk_tail;          // chunks published
  unsigned int stop;                // workers leave
  unsigned int sched_beat;          // scheduler heartbeat
  unsigned int done_count;          // completions published (atomic)
  unsigned int worker_err;          // a worker gave up waiting
  unsigned int max_active;
  // statistics (written by the scheduler every 64 rounds and at the end)
  unsigned long long records_served, scanned, chunks, rounds, deferred, bytes_peak, a_in_use;
};

struct LoopArgs {
  LoopDev* d;
  ReqSlot* slots;
  Chunk* chunks;
  Region* regions;
  LoopReq* pend;                    // device pending queue (ring entries)
  unsigned int* client_busy;
  // mapped host memory (device pointers)
  const unsigned long long* req_ring;
  const unsigned int* rel_ring;
  LoopDone* done_ring;
  const LoopHostIn* hin;
  LoopHostOut* hout;
  // the volume and its server
  TableView t;
  PoolView pool;
  const ServeLog* sl;
  unsigned int* client_v;
  unsigned char* arena;
  unsigned long long budget;
  unsigned int ring_mask;           // request / completion / pending rings
  unsigned int n_slots, chunk_records, bypass_rounds, max_blocks, log_cap, n_workers, n_clients;
  unsigned long long timeout_ns;
};

// ---- memory helpers: system-scope accesses to mapped host memory, L2 accesses to device state
__device__ __forceinline__ unsigned int ld_acq_sys(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_sys(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_sys64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys(unsigned int* p, unsigned int v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Acquire-release fence at GPU scope (orders the copies before the second look at a refresh
// number, and the scheduler's descriptor writes before their publication).
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
template <typename T>
__device__ __forceinline__ T vload(const T* p) {
  return *reinterpret_cast<const volatile T*>(p);
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, T v) {
  *reinterpret_cast<volatile T*>(p) = v;
}

__device__ __forceinline__ unsigned int rem_latest_cg(const ServeLog& S, unsigned long long key) {
  unsigned int b = hash_mix(key) & S.rem_mask;
  for (unsigned int probe = 0; probe <= S.rem_mask; ++probe, b = (b + 1u) & S.rem_mask) {
    const unsigned long long k = __ldcg(S.rem_keys + b);
    if (k == key) return __ldcg(S.rem_seq + b);
    if (k == kEmpty) break;
  }
  return 0u;
}

// Find through L2 (the table changes under the loop; a live entry never moves while it runs).
__device__ __forceinline__ bool live_cg(const TableView& t, unsigned long long key) {
  unsigned int b = home_bucket(key, t.bmask, t.hash_fn);
  const unsigned int step = probe_step(key);
  for (unsigned int probe = 0; probe <= t.bmask; ++probe, b = (b + step) & t.bmask) {
    bool empty = false;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const unsigned long long k = __ldcg(&t.slots[4u * b + l].key);
      if (k == key) return true;
      empty = empty || k == kEmpty;
    }
    if (empty) return false;
  }
  return false;
}

// One completion into the mapped ring: fields, a system fence, then the token.
__device__ void publish_done(const LoopArgs& A, unsigned int id, unsigned int client,
                             unsigned int n, unsigned int flags, unsigned int v0,
                             unsigned int v1, unsigned int region, unsigned int cap,
                             unsigned long long off, unsigned int dev_ns = 0u) {
  const unsigned int d = atomicAdd(&A.d->done_count, 1u);
  LoopDone* D = A.done_ring + (d & A.ring_mask);
  volatile unsigned int* w = reinterpret_cast<volatile unsigned int*>(D);
  w[0] = id;
  w[1] = client;
  w[2] = n;
  w[3] = flags;
  w[4] = v0;
  w[5] = v1;
  w[6] = region;
  w[7] = cap;
  w[8] = (unsigned int)off;
  w[9] = (unsigned int)(off >> 32);
  w[11] = dev_ns;
  __threadfence_system();
  st_rel_sys(&D->tok, d + 1u);
}

// The request of slot `si` has all its tiles served: move the client, publish, free the slot.
__device__ void complete_request(const LoopArgs& A, unsigned int si) {
  ReqSlot* R = A.slots + si;
  __threadfence();
  const unsigned int nr = atomicExch(&R->rec_count, 0u);
  const unsigned int ef = atomicExch(&R->err, 0u);
  const unsigned int id = vload(&R->id), client = vload(&R->client);
  const unsigned int v0 = vload(&R->v0), v1 = vload(&R->v1), region = vload(&R->region);
  const unsigned int cap = vload(&R->cap);
  unsigned int flags = vload(&R->flags);
  const unsigned long long off = vload(&R->off);
  if (ef & kErrOverrun) flags |= VBH_SERVE_ERR_OVERRUN;
  if (ef & kErrCap) flags |= VBH_SERVE_ERR_CAPACITY;
  vstore(&A.client_v[client], v1);
  atomicAdd(&A.d->records_served, (unsigned long long)nr);
  const unsigned long long dt = globaltimer() - vload(&R->t_adm);
  publish_done(A, id, client, nr, flags, v0, v1, region, cap, off,
               dt < 0xFFFFFFFFull ? (unsigned int)dt : 0xFFFFFFFFu);
  __threadfence();
  vstore(&A.client_busy[client], 0u);   // the client and the slot are free for the scheduler
  atomicOr(&A.d->free_mask, 1ull << si);
}

// Serve up to 32 records of a tile (one warp, a lane per record): test each record for being
// current; copy every current block's 512 B of indices into the warp's staging area in shared
// memory with asynchronous 16 B copies (all of the tile's copies in flight at once), fence, and
// read each block's refresh number again -- a block whose number changed meanwhile is dropped;
// reserve the tile's output with one atomic, write the headers, and the payloads from the
// staging area.  Records rec0 + 1 .. rec_end of the log (scan: pool entries rec0 .. rec_end - 1).
__device__ void serve_tile(const LoopArgs& A, const ServeLog& S, uint4* stage, unsigned int si,
                           bool scan, unsigned int sigma, unsigned int cap,
                           unsigned long long off, unsigned int rec0, unsigned int rec_end) {
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int lt = (1u << lane) - 1u;
  ReqSlot* R = A.slots + si;
  bool cur = false;
  unsigned long long key = 0ull;
  unsigned int info = 0u, p = kNone, e_ref = 0u, err = 0u;
  if (scan) {
    const unsigned int j = rec0 + lane;
    if (j < rec_end) {
      const unsigned long long k = __ldcg(A.pool.pkeys + j);
      const unsigned int sq = __ldcg(A.pool.seq + j);
      if (k != kEmpty && sq != 0u && sq <= sigma) {
        cur = true;
        key = k;
        p = j;
        e_ref = sq;
        info = __ldcg(A.pool.version + j) & 0x7FFFFFFFu;
      }
    }
  } else {
    const unsigned int e = rec0 + 1u + lane;
    if (e <= rec_end) {
      const ulonglong2 raw = __ldcg(reinterpret_cast<const ulonglong2*>(S.log + (e & S.log_mask)));
      const unsigned int aux = (unsigned int)raw.y, seq = (unsigned int)(raw.y >> 32);
      if (seq != e) {
        err |= kErrOverrun;
      } else if (raw.x & kLogRemoved) {
        const unsigned long long k = raw.x & ~kLogRemoved;
        if (rem_latest_cg(S, k) == e && !live_cg(A.t, k)) {
          cur = true;
          key = k;
          info = 0x80000000u | aux;
        }
      } else if (aux < A.max_blocks && __ldcg(A.pool.seq + aux) == e &&
                 __ldcg(A.pool.pkeys + aux) == raw.x) {
        cur = true;
        key = raw.x;
        p = aux;
        e_ref = e;
        info = __ldcg(A.pool.version + aux) & 0x7FFFFFFFu;
      }
    }
  }
  unsigned char* region = A.arena + off;
  int4* hdr = reinterpret_cast<int4*>(region);
  uint4* pay = reinterpret_cast<uint4*>(region + (size_t)cap * kRecHdr);
  // removal records: a header only
  const unsigned int rm = __ballot_sync(0xFFFFFFFFu, cur && p == kNone);
  if (rm) {
    unsigned int base = 0u;
    if (lane == 0u) base = atomicAdd(&R->rec_count, (unsigned int)__popc(rm));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((unsigned long long)base + __popc(rm) > cap) {
      err |= kErrCap;
    } else if (cur && p == kNone) {
      const int3 k3 = unpack_key(key);
      hdr[base + __popc(rm & lt)] = make_int4(k3.x, k3.y, k3.z, (int)info);
    }
  }
  // current blocks, kStageBlocks at a time: block i of the group at stage + 32 i (lane L
  // copies word L of each), all copies of the group in flight at once
  unsigned int rest = __ballot_sync(0xFFFFFFFFu, cur && p != kNone);
  while (rest) {
    unsigned int grp = 0u;
    for (unsigned int i = 0; i < kStageBlocks && rest; ++i) {
      const int src = __ffs(rest) - 1;
      rest &= rest - 1u;
      grp |= 1u << src;
      const unsigned int q = __shfl_sync(0xFFFFFFFFu, p, src);
      const unsigned int dst = (unsigned int)__cvta_generic_to_shared(stage + 32u * i + lane);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                   "l"(S.store + 32u * q + lane)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_all;" ::: "memory");
    fence_acq_rel_gpu();
    // a block refreshed again while it was copied is dropped (its newer refresh is after sigma)
    const bool mine = (grp >> lane) & 1u;
    const bool ok = mine && __ldcg(A.pool.seq + p) == e_ref && __ldcg(A.pool.pkeys + p) == key;
    const unsigned int okm = __ballot_sync(0xFFFFFFFFu, ok);
    const unsigned int n = __popc(okm);
    if (n) {
      unsigned int base = 0u;
      if (lane == 0u) base = atomicAdd(&R->rec_count, n);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if ((unsigned long long)base + n > cap) {
        err |= kErrCap;
      } else {
        if (ok) {
          const int3 k3 = unpack_key(key);
          hdr[base + __popc(okm & lt)] = make_int4(k3.x, k3.y, k3.z, (int)info);
        }
        unsigned int g = grp;
        for (unsigned int i = 0; g; ++i) {
          const int src = __ffs(g) - 1;
          g &= g - 1u;
          if ((okm >> src) & 1u)
            pay[(size_t)(base + __popc(okm & ((1u << src) - 1u))) * 32u + lane] =
                stage[32u * i + lane];
        }
      }
    }
    __syncwarp();   // the group's staging area is read before the next group's copies land
  }
  __syncwarp();   // the staging area is free for the warp's next tile
  err = __reduce_or_sync(0xFFFFFFFFu, err);
  if (err && lane == 0u) atomicOr(&R->err, err);
}

// Ring allocator over the stream buffer (scheduler-private): regions are handed out in order
// and released in any order; the tail passes released regions in order.  A region never wraps
// (the rest of the buffer before the wrap becomes a released filler region).
struct Arena {
  unsigned long long head, tail;   // monotonic byte positions
  unsigned int r_head, r_tail;     // region FIFO
};

__device__ bool arena_alloc(const LoopArgs& A, Arena& a, unsigned long long bytes,
                            unsigned long long* start, unsigned int* idx) {
  if (a.head == a.tail) {   // nothing in use: start at the beginning of the buffer
    a.head = (a.head + A.budget - 1ull) / A.budget * A.budget;
    a.tail = a.head;
  }
  const unsigned long long pos = a.head % A.budget;
  const unsigned long long pad = pos + bytes > A.budget ? A.budget - pos : 0ull;
  if (a.r_head - a.r_tail + (pad ? 2u : 1u) > kRegionRing) return false;
  if (a.head + pad + bytes - a.tail > A.budget) return false;
  if (pad) {
    Region& f = A.regions[a.r_head % kRegionRing];
    f.start = a.head;
    f.bytes = pad;
    f.freed = 1u;
    a.r_head += 1u;
    a.head += pad;
  }
  Region& g = A.regions[a.r_head % kRegionRing];
  g.start = a.head;
  g.bytes = bytes;
  g.freed = 0u;
  *idx = a.r_head;
  *start = a.head;
  a.r_head += 1u;
  a.head += bytes;
  return true;
}

// The scheduler (one thread).  Its own state lives in registers and in the shared memory of
// its warp (per-slot chunk cursors); device memory shared with the workers is touched only to
// read client state, take a slot and publish chunks, and mapped host memory once per round
// (the request ring's tail), every 4th round (the release ring) and every 16th round (the
// host's sign of life): each of those reads crosses PCIe.
__device__ void scheduler(const LoopArgs& A, unsigned int* sm) {
  LoopDev* d = A.d;
  const ServeLog* sl = A.sl;
  unsigned int* s_next = sm;                   // next change record to chunk, per slot
  unsigned int* s_hi = sm + kLoopMaxSlots;     // end of the slot's range
  unsigned int req_head = 0u, rel_head = 0u, pend_head = 0u, pend_tail = 0u;
  unsigned int tag = 1u;         // tag of the next request
  unsigned int done_read = 0u;   // completions the host has consumed, as last read
  unsigned int chunk_low = 0u, chunk_tail = 0u, head_blocked = 0u, max_active = 0u;
  unsigned long long end_tile = 0ull, work = 0ull;   // work: slots with chunks left
  unsigned long long scanned = 0ull, chunks = 0ull, rounds = 0ull, deferred = 0ull, peak = 0ull;
  Arena a{0ull, 0ull, 0u, 0u};
  unsigned int last_beat = ld_sys(&A.hin->beat);
  unsigned long long t_host = globaltimer();
  unsigned int status = 0u;
  const unsigned long long low_water = (unsigned long long)A.n_workers + 64ull;
  const unsigned long long all_slots =
      A.n_slots >= 64u ? ~0ull : ((1ull << A.n_slots) - 1ull);
  for (unsigned int round = 1;; ++round) {
    vstore(&d->sched_beat, round);
    bool busy = false;
    if ((round & 15u) == 1u) {
      const unsigned long long now = globaltimer();
      const unsigned int hb = ld_sys(&A.hin->beat);
      if (hb != last_beat) {
        last_beat = hb;
        t_host = now;
      }
      if (ld_acq_sys(&A.hin->stop)) break;
      if (now - t_host > A.timeout_ns) {
        status = VBH_ERR_TIMEOUT;
        break;
      }
    }
    // releases, then the allocator's tail over released regions
    if ((round & 3u) == 1u) {
      const unsigned int rt = ld_acq_sys(&A.hin->rel_tail);
      while (rel_head != rt) {
        const unsigned int r = ld_sys(A.rel_ring + (rel_head & A.ring_mask));
        A.regions[r % kRegionRing].freed = 1u;
        rel_head += 1u;
        busy = true;
      }
      st_rel_sys(&A.hout->rel_head, rel_head);
      while (a.r_tail != a.r_head && A.regions[a.r_tail % kRegionRing].freed) {
        const Region& g = A.regions[a.r_tail % kRegionRing];
        a.tail = g.start + g.bytes;
        a.r_tail += 1u;
      }
    }
    // new requests into the pending queue (arrival order): the next two slots are read at once
    // (one round trip over the host link when requests come one at a time or in pairs)
    for (bool more = true; more && pend_tail - pend_head + 2u <= A.ring_mask + 1u;) {
      const unsigned long long v0 = ld_sys64(A.req_ring + (req_head & A.ring_mask));
      const unsigned long long v1 = ld_sys64(A.req_ring + ((req_head + 1u) & A.ring_mask));
      more = false;
      if ((unsigned int)(v0 >> 32) == tag) {
        A.pend[pend_tail & A.ring_mask] = LoopReq{tag, (unsigned int)v0};
        pend_tail += 1u;
        req_head += 1u;
        tag = next_tag(tag);
        busy = true;
        if ((unsigned int)(v1 >> 32) == tag) {
          A.pend[pend_tail & A.ring_mask] = LoopReq{tag, (unsigned int)v1};
          pend_tail += 1u;
          req_head += 1u;
          tag = next_tag(tag);
          more = true;
        }
      }
    }
    if (busy) st_rel_sys(&A.hout->req_head, req_head);
    // admission in arrival order at the newest published snapshot
    if (pend_head != pend_tail) {
      const unsigned int sigma = vload(&sl->seq_next) - 1u;
      fence_acq_rel_gpu();
      unsigned long long free = vload(&d->free_mask) & all_slots;
      unsigned int w = pend_head;
      bool head = true, stop_adm = false, admitted = false;
      for (unsigned int r = pend_head; r != pend_tail; ++r) {
        const LoopReq q = A.pend[r & A.ring_mask];
        bool keep = true;
        if (!stop_adm) {
          const unsigned int active = A.n_slots - __popcll(free);
          unsigned int outstanding = vload(&d->done_count) - done_read;
          if (outstanding + active + 1u > A.ring_mask + 1u) {   // read the host's count again
            done_read = ld_sys(&A.hin->done_read);
            outstanding = vload(&d->done_count) - done_read;
          }
          if (outstanding + active + 1u > A.ring_mask + 1u) {
            stop_adm = true;   // no completion-ring room for one more
          } else if (q.client >= A.n_clients) {   // never written by the library's host side
            publish_done(A, q.id, q.client, 0u, VBH_SERVE_ERR_VERSION, 0u, 0u, 0xFFFFFFFFu, 0u,
                         0ull);
            keep = false;
          } else if (vload(&A.client_busy[q.client])) {
            head = false;   // one request per client at a time, in arrival order
          } else if (!free) {
            stop_adm = true;   // no free slot
          } else {
            const unsigned int v = vload(&A.client_v[q.client]);
            const unsigned int margin = A.log_cap / 2u;   // records appended while one runs
            const unsigned int floor = sigma > margin ? sigma - margin : 0u;
            const bool scan = v == 0u || v < floor;
            if (!scan && sigma <= v) {   // nothing changed since v: complete without work
              publish_done(A, q.id, q.client, 0u, 0u, v, v, 0xFFFFFFFFu, 0u, 0ull);
              keep = false;
            } else {
              unsigned long long count = scan ? A.max_blocks : (unsigned long long)(sigma - v);
              unsigned int flags = scan ? VBH_SERVE_RESET : 0u;
              const unsigned long long max_recs = A.budget / kRecAll;
              if (count > max_recs) {
                count = max_recs;
                flags |= VBH_SERVE_PARTIAL;
              }
              const unsigned long long bytes = (count * kRecAll + 255ull) & ~255ull;
              unsigned long long start;
              unsigned int region;
              if (!arena_alloc(A, a, bytes, &start, &region)) {
                deferred += 1ull;
                if (head && ++head_blocked > A.bypass_rounds) stop_adm = true;
                head = false;
              } else {
                if (head) head_blocked = 0u;
                if (a.head - a.tail > peak) peak = a.head - a.tail;
                const unsigned int si = (unsigned int)(__ffsll((long long)free) - 1);
                free &= ~(1ull << si);
                atomicAnd(&d->free_mask, ~(1ull << si));
                ReqSlot& R = A.slots[si];
                R.id = q.id;
                R.client = q.client;
                R.scan = scan ? 1u : 0u;
                R.sigma = sigma;
                R.cap = (unsigned int)count;
                R.v0 = v;
                R.v1 = scan ? sigma : v + (unsigned int)count;
                R.flags = flags;
                R.region = region;
                R.off = start % A.budget;
                R.chunks_total =
                    (unsigned int)((count + A.chunk_records - 1ull) / A.chunk_records);
                R.chunks_done = 0u;
                R.rec_count = 0u;
                R.err = 0u;
                R.t_adm = globaltimer();
                s_next[si] = scan ? 0u : v;
                s_hi[si] = scan ? A.max_blocks : v + (unsigned int)count;
                work |= 1ull << si;
                vstore(&A.client_busy[q.client], 1u);
                keep = false;
                admitted = true;
                const unsigned int now_active = active + 1u;
                if (now_active > max_active) max_active = now_active;
              }
            }
          }
        }
        if (keep) A.pend[(w++) & A.ring_mask] = q;
      }
      pend_tail = w;
      if (admitted) busy = true;
    }
    // chunks: keep the workers' backlog of published tiles above the low-water mark, each
    // chunk to the active request with the smallest remainder; one publication per round
    const unsigned long long nt = vload(&d->next_ticket);
    unsigned long long backlog = end_tile > nt ? end_tile - nt : 0ull;
    if (work && backlog < low_water) {
      if (chunk_tail - chunk_low + 32u > kChunkRing) {
        while (chunk_low != chunk_tail) {
          const Chunk& c = A.chunks[chunk_low % kChunkRing];
          if (vload(&c.finished) < c.tiles) break;
          chunk_low += 1u;
        }
      }
      unsigned int published = 0u;
      while (work && backlog < low_water && chunk_tail - chunk_low < kChunkRing) {
        unsigned int best = 0u, best_rem = 0xFFFFFFFFu;
        for (unsigned long long m = work; m; m &= m - 1ull) {
          const unsigned int i = (unsigned int)(__ffsll((long long)m) - 1);
          const unsigned int rem = s_hi[i] - s_next[i];
          if (rem < best_rem) {
            best_rem = rem;
            best = i;
          }
        }
        const unsigned int take = best_rem < A.chunk_records ? best_rem : A.chunk_records;
        Chunk& c = A.chunks[chunk_tail % kChunkRing];
        c.start_tile = end_tile;
        c.idx = chunk_tail;
        // a request with at least kBigRemain records left gets longer tiles (fewer tickets,
        // chunk look-ups and reservations per record: its tail latency falls); a shorter
        // remainder keeps short tiles (a request's latency is then about one tile's)
        const unsigned int recs = best_rem >= kBigRemain ? kBigTileRecs : kTileRecs;
        c.recs = recs;
        c.tiles = (take + recs - 1u) / recs;
        c.slot = best;
        c.lo = s_next[best];
        c.hi = s_next[best] + take;
        c.finished = 0u;
        s_next[best] += take;
        if (s_next[best] == s_hi[best]) work &= ~(1ull << best);
        scanned += take;
        chunks += 1ull;
        chunk_tail += 1u;
        end_tile += c.tiles;
        backlog += c.tiles;
        published += 1u;
      }
      if (published) {
        fence_acq_rel_gpu();   // descriptors (and the slots they name) before their tickets
        vstore(&d->chunk_tail, chunk_tail);
        fence_acq_rel_gpu();
        vstore(&d->end_tile, end_tile);
        busy = true;
      }
    }
    if (busy) rounds += 1ull;
    if ((round & 63u) == 0u) {   // statistics for vbh_serve_loop_stats_read
      d->scanned = scanned;
      d->chunks = chunks;
      d->rounds = rounds;
      d->deferred = deferred;
      d->bytes_peak = peak;
      d->max_active = max_active;
      d->a_in_use = a.head - a.tail;
    }
    if (!busy) __nanosleep(100);
  }
  d->scanned = scanned;
  d->chunks = chunks;
  d->rounds = rounds;
  d->deferred = deferred;
  d->bytes_peak = peak;
  d->max_active = max_active;
  d->a_in_use = a.head - a.tail;
  __threadfence();
  vstore(&d->stop, 1u);
  __threadfence_system();
  st_rel_sys(&A.hout->status, status);
  st_rel_sys(&A.hout->exited, 1u);
}

// A worker warp: take a ticket, wait (bounded) until its tile is published, find the tile's
// chunk, serve it, and close the chunk / request when it was the last tile.
__device__ void worker(const LoopArgs& A, uint4* stage) {
  LoopDev* d = A.d;
  const unsigned int lane = threadIdx.x & 31u;
  const ServeLog S = *A.sl;   // its pointers and masks do not change while a server is attached
  const unsigned long long stall_ns = 2ull * A.timeout_ns;
  unsigned int hint = 0u;     // the chunk of this warp's previous tile (tickets only grow)
  for (;;) {
    unsigned long long t = 0ull;
    if (lane == 0u) t = atomicAdd(&d->next_ticket, 1ull);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    int state = 0;   // 0 tile published, 1 stop, 2 the scheduler stopped beating
    if (lane == 0u) {
      unsigned int beat = vload(&d->sched_beat);
      unsigned long long t_beat = globaltimer();
      unsigned int nap = 32u;
      for (;;) {
        if (vload(&d->end_tile) > t) break;
        if (vload(&d->stop)) {
          state = 1;
          break;
        }
        const unsigned int b = vload(&d->sched_beat);
        const unsigned long long now = globaltimer();
        if (b != beat) {
          beat = b;
          t_beat = now;
        } else if (now - t_beat > stall_ns) {
          state = 2;
          break;
        }
        __nanosleep(nap);
        if (nap < VBH_LOOP_MAX_NAP) nap *= 2u;
      }
    }
    state = __shfl_sync(0xFFFFFFFFu, state, 0);
    if (state == 2 && lane == 0u) atomicOr(&d->worker_err, 1u);
    if (state) return;
    fence_acq_rel_gpu();
    // the chunk holding ticket t: the last published chunk whose first ticket is <= t (ring
    // positions reused by newer chunks belong to chunks older than every unfinished one);
    // chunk c qualifies when its position holds an older chunk or it starts at or before t
    auto qualifies = [&](unsigned int x) {
      const Chunk& m = A.chunks[x % kChunkRing];
      return vload(&m.idx) != x || vload(&m.start_tile) <= t;
    };
    unsigned int hi = 0u;
    if (lane == 0u) hi = vload(&d->chunk_tail);
    hi = __shfl_sync(0xFFFFFFFFu, hi, 0);
    unsigned int lo = hi > kChunkRing ? hi - kChunkRing : 0u;
    if (hint > lo) lo = hint;
    // the 32 newest candidates at once, one per lane (a waiting worker's tile was published in
    // the last rounds): the newest qualifying one; else a binary search below them
    const bool cand = lane < hi - lo;
    const unsigned int found = __ballot_sync(0xFFFFFFFFu, cand && qualifies(hi - 1u - lane));
    unsigned int c = 0u;
    if (found) {
      c = hi - 1u - (unsigned int)(__ffs(found) - 1);
    } else if (lane == 0u) {   // only when more than 32 chunks lie above the hint
      unsigned int top = hi - 32u;
      while (top - lo > 1u) {   // invariant: chunk lo qualifies, chunk top does not
        const unsigned int mid = lo + (top - lo) / 2u;
        if (qualifies(mid)) lo = mid;
        else top = mid;
      }
      c = lo;
    }
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    hint = c;
    Chunk* ch = A.chunks + (c % kChunkRing);
    const unsigned int k = (unsigned int)(t - vload(&ch->start_tile));
    const unsigned int tiles = vload(&ch->tiles), si = vload(&ch->slot);
    const unsigned int clo = vload(&ch->lo), chi = vload(&ch->hi);
    ReqSlot* R = A.slots + si;
    const bool scan = vload(&R->scan) != 0u;
    const unsigned int recs = vload(&ch->recs);
    const unsigned int rec0 = clo + recs * k;
    const unsigned int rec_end = rec0 + recs < chi ? rec0 + recs : chi;
    {   // the tile's records, 32 (one per lane) at a time
      const unsigned int sig = vload(&R->sigma), cap = vload(&R->cap);
      const unsigned long long off = vload(&R->off);
      for (unsigned int r0 = rec0; r0 < rec_end; r0 += 32u)
        serve_tile(A, S, stage, si, scan, sig, cap, off, r0,
                   r0 + 32u < rec_end ? r0 + 32u : rec_end);
    }
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0u && atomicAdd(&ch->finished, 1u) == tiles - 1u) {
      if (atomicAdd(&R->chunks_done, 1u) == vload(&R->chunks_total) - 1u) complete_request(A, si);
    }
    __syncwarp();
  }
}

// Dynamic shared memory: each warp's staging area (kStageBlocks blocks x 512 B).
constexpr unsigned int kStageBytes = kLoopWarps * kStageBlocks * kRecPay;

__global__ void __launch_bounds__(kLoopThreads) k_serve_loop(const LoopArgs A) {
  extern __shared__ __align__(16) uint4 s_stage[];
  if (blockIdx.x == 0 && threadIdx.x < 32) {   // warp 0's staging area holds scheduler state
    if (threadIdx.x == 0) scheduler(A, reinterpret_cast<unsigned int*>(s_stage));
    return;
  }
  worker(A, s_stage + (threadIdx.x >> 5) * kStageBlocks * (kRecPay / 16u));
}

uint64_t loop_now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace
}  // namespace vbh

using namespace vbh;

struct vbh_serve_loop {
  vbh_serve* s = nullptr;
  vbh_handle* h = nullptr;
  ServeShared X{};
  vbh_serve_loop_config cfg{};
  cudaStream_t stream = nullptr;   // the loop kernel (non-blocking: never waits for others)
  cudaStream_t aux = nullptr;      // statistics copies while the loop runs
  // device state
  LoopDev* d = nullptr;
  ReqSlot* slots = nullptr;
  Chunk* chunks = nullptr;
  Region* regions = nullptr;
  LoopReq* pend = nullptr;
  unsigned int* client_busy = nullptr;
  // mapped host memory
  unsigned long long* req_ring = nullptr;
  unsigned int* rel_ring = nullptr;
  LoopDone* done_ring = nullptr;
  LoopHostIn* hin = nullptr;
  LoopHostOut* hout = nullptr;
  uint32_t ring = 0, req_tail = 0, rel_tail = 0, done_read = 0, beat = 0, next_id = 1;
  bool launched = false;
  struct Info {
    uint32_t client = 0;
    uint64_t t_arrival = 0;
    bool done = false;
    LoopDone rec{};
  };
  std::unordered_map<uint32_t, Info> reqs;
  std::vector<vbh_serve_done> ready;   // completions read by drain, handed out by poll
  uint64_t submitted = 0, completed = 0;

  void alive() {   // sign of life for the scheduler's liveness check
    reinterpret_cast<volatile unsigned int*>(&hin->beat)[0] = ++beat;
  }
  bool exited() const { return reinterpret_cast<volatile unsigned int*>(&hout->exited)[0] != 0u; }
  unsigned int dev_status() const {
    return reinterpret_cast<volatile unsigned int*>(&hout->status)[0];
  }
  // Move published completions from the ring into `ready` (in publication order).
  void collect() {
    const volatile LoopDone* ring_v = done_ring;
    for (;;) {
      const volatile LoopDone& D = ring_v[done_read & (ring - 1u)];
      if (D.tok != done_read + 1u) break;
      std::atomic_thread_fence(std::memory_order_acquire);
      LoopDone r;
      r.id = D.id;
      r.client = D.client;
      r.n_records = D.n_records;
      r.flags = D.flags;
      r.v0 = D.v0;
      r.v1 = D.v1;
      r.dev_ns = D.dev_ns;
      r.region = D.region;
      r.cap = D.cap;
      r.off = D.off;
      done_read += 1u;
      auto it = reqs.find(r.id);
      vbh_serve_done o{};
      o.id = r.id;
      o.client = r.client;
      o.v_before = r.v0;
      o.v_after = r.v1;
      o.n_records = r.n_records;
      o.flags = r.flags;
      o.t_done_ns = loop_now_ns();
      // admission in the host's clock: completion seen minus the GPU's time from admission
      // to publication (the two clocks are not compared)
      o.t_admit_ns = o.t_done_ns - r.dev_ns;
      o.bytes_reserved = r.region == 0xFFFFFFFFu ? 0ull
                                                 : (((uint64_t)r.cap * kRecAll + 255u) & ~255ull);
      if (it != reqs.end()) {
        o.t_arrival_ns = it->second.t_arrival;
        if (o.t_admit_ns < o.t_arrival_ns) o.t_admit_ns = o.t_arrival_ns;
        it->second.done = true;
        it->second.rec = r;
      }
      ready.push_back(o);
      completed += 1;
    }
    std::atomic_thread_fence(std::memory_order_release);
    reinterpret_cast<volatile unsigned int*>(&hin->done_read)[0] = done_read;
  }
  vbh_status stopped_status() const {
    const unsigned int st = dev_status();
    if (st == VBH_ERR_TIMEOUT)
      return fail(VBH_ERR_TIMEOUT, "serving loop stopped: no sign of life from the host in time");
    return fail(st ? (vbh_status)st : VBH_ERR_TIMEOUT, "serving loop has stopped");
  }
};

namespace {

void loop_free(vbh_serve_loop* L) {
  void* dev[] = {L->d, L->slots, L->chunks, L->regions, L->pend, L->client_busy};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {L->req_ring, L->rel_ring, L->done_ring, L->hin, L->hout};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  if (L->stream) cudaStreamDestroy(L->stream);
  if (L->aux) cudaStreamDestroy(L->aux);
  delete L;
}

template <typename T>
cudaError_t host_mapped(T** host, size_t n) {
  cudaError_t e = cudaHostAlloc((void**)host, sizeof(T) * n, cudaHostAllocMapped);
  if (e == cudaSuccess) std::memset((void*)*host, 0, sizeof(T) * n);
  return e;
}

template <typename T>
T* dev_alias(T* host) {
  T* d = nullptr;
  return cudaHostGetDevicePointer((void**)&d, (void*)host, 0) == cudaSuccess ? d : nullptr;
}

}  // namespace

extern "C" {

vbh_status vbh_serve_loop_start(vbh_serve* s, const vbh_serve_loop_config* cfg_in,
                                vbh_serve_loop** out) {
  if (!s || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (serve_loop_of(s)) return fail(VBH_ERR_INVALID_ARG, "a serving loop is already running");
  if (!serve_idle(s)) return fail(VBH_ERR_INVALID_ARG, "server has requests in flight");
  vbh_serve_loop_config c = cfg_in ? *cfg_in : vbh_serve_loop_config{};
  const ServeShared X = serve_shared(s);
  vbh_handle* h = X.h;
  if (c.max_slots == 0) c.max_slots = kLoopMaxSlots;
  if (c.chunk_records == 0) c.chunk_records = 4096u;
  if (c.ring == 0) c.ring = 4096u;
  if (c.idle_timeout_us == 0) c.idle_timeout_us = 1000000u;
  if (c.ctas == 0) c.ctas = (uint32_t)h->L.sms;
  if (c.max_slots > kLoopMaxSlots) return fail(VBH_ERR_INVALID_ARG, "max_slots must be 1..64");
  if (c.ring < 64u || c.ring > (1u << 20) || (c.ring & (c.ring - 1u)))
    return fail(VBH_ERR_INVALID_ARG, "ring must be a power of two in [64, 2^20]");
  if (c.chunk_records > (1u << 24)) return fail(VBH_ERR_INVALID_ARG, "chunk_records too large");
  int occ = 0;
  VBH_CUDA(cudaFuncSetAttribute(k_serve_loop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kStageBytes));
  // a preferred shared-memory share for the SMs the loop occupies (default: the driver's choice)
  if (kLoopCarveout >= 0)
    VBH_CUDA(cudaFuncSetAttribute(k_serve_loop, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  kLoopCarveout));
  VBH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve_loop, kLoopThreads,
                                                         kStageBytes));
  if (c.ctas > (uint32_t)(occ * h->L.sms))
    return fail(VBH_ERR_INVALID_ARG, "ctas above what can be resident at once");
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  vbh_serve_loop* L = new vbh_serve_loop();
  L->s = s;
  L->h = h;
  L->X = X;
  L->cfg = c;
  L->ring = c.ring;
  auto bail = [&](const char* what, cudaError_t e) {
    loop_free(L);
    return fail(VBH_ERR_CUDA, std::string("vbh_serve_loop_start: ") + what + ": " +
                                  cudaGetErrorString(e));
  };
#define LOOP_CUDA(call)                  \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) return bail(#call, e_); \
  } while (0)
  LOOP_CUDA(cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking));
  LOOP_CUDA(cudaStreamCreateWithFlags(&L->aux, cudaStreamNonBlocking));
  LOOP_CUDA(cudaMalloc(&L->d, sizeof(LoopDev)));
  LOOP_CUDA(cudaMalloc(&L->slots, sizeof(ReqSlot) * kLoopMaxSlots));
  LOOP_CUDA(cudaMalloc(&L->chunks, sizeof(Chunk) * kChunkRing));
  LOOP_CUDA(cudaMalloc(&L->regions, sizeof(Region) * kRegionRing));
  LOOP_CUDA(cudaMalloc(&L->pend, sizeof(LoopReq) * c.ring));
  LOOP_CUDA(cudaMalloc(&L->client_busy, sizeof(unsigned int) * X.n_clients));
  LOOP_CUDA(host_mapped(&L->req_ring, c.ring));
  LOOP_CUDA(host_mapped(&L->rel_ring, c.ring));
  LOOP_CUDA(host_mapped(&L->done_ring, c.ring));
  LOOP_CUDA(host_mapped(&L->hin, 1));
  LOOP_CUDA(host_mapped(&L->hout, 1));
  LoopDev init{};
  init.free_mask = c.max_slots >= 64u ? ~0ull : ((1ull << c.max_slots) - 1ull);
  LOOP_CUDA(cudaMemcpyAsync(L->d, &init, sizeof init, cudaMemcpyHostToDevice, L->stream));
  LOOP_CUDA(cudaMemsetAsync(L->slots, 0, sizeof(ReqSlot) * kLoopMaxSlots, L->stream));
  LOOP_CUDA(cudaMemsetAsync(L->chunks, 0xFF, sizeof(Chunk) * kChunkRing, L->stream));
  LOOP_CUDA(cudaMemsetAsync(L->regions, 0, sizeof(Region) * kRegionRing, L->stream));
  LOOP_CUDA(cudaMemsetAsync(L->client_busy, 0, sizeof(unsigned int) * X.n_clients, L->stream));
  LoopArgs A{};
  A.d = L->d;
  A.slots = L->slots;
  A.chunks = L->chunks;
  A.regions = L->regions;
  A.pend = L->pend;
  A.client_busy = L->client_busy;
  A.req_ring = dev_alias(L->req_ring);
  A.rel_ring = dev_alias(L->rel_ring);
  A.done_ring = dev_alias(L->done_ring);
  A.hin = dev_alias(L->hin);
  A.hout = dev_alias(L->hout);
  if (!A.req_ring || !A.rel_ring || !A.done_ring || !A.hin || !A.hout)
    return bail("cudaHostGetDevicePointer", cudaErrorInvalidValue);
  A.t = h->table();
  A.pool = h->pool();
  A.sl = X.sl;
  A.client_v = X.client_v;
  A.arena = X.arena;
  A.budget = X.budget;
  A.ring_mask = c.ring - 1u;
  A.n_slots = c.max_slots;
  A.chunk_records = c.chunk_records;
  A.bypass_rounds = c.bypass_rounds;
  A.max_blocks = h->cfg.max_blocks;
  A.log_cap = X.log_cap;
  A.n_workers = c.ctas * kLoopWarps - 1u;
  A.n_clients = X.n_clients;
  A.timeout_ns = (unsigned long long)c.idle_timeout_us * 1000ull;
  LOOP_CUDA(cudaStreamSynchronize(L->stream));
  L->alive();
  void* args[] = {&A};
  LOOP_CUDA(cudaLaunchCooperativeKernel((const void*)k_serve_loop, dim3(c.ctas),
                                        dim3(kLoopThreads), args, kStageBytes, L->stream));
#undef LOOP_CUDA
  L->launched = true;
  h->launches += 1;
  h->serve_loop_active = true;
  serve_set_loop(s, L);
  *out = L;
  return VBH_OK;
}

vbh_status vbh_serve_loop_submit(vbh_serve_loop* L, uint32_t client, uint64_t t_arrival_ns,
                                 uint32_t* id) {
  if (!L) return fail(VBH_ERR_INVALID_ARG, "null loop");
  if (client >= L->X.n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
  L->alive();
  if (L->exited()) return L->stopped_status();
  const uint32_t head = reinterpret_cast<volatile unsigned int*>(&L->hout->req_head)[0];
  if (L->req_tail - head >= L->ring) return fail(VBH_ERR_CAPACITY, "request ring full");
  const uint32_t rid = L->next_id;
  L->next_id = next_tag(L->next_id);
  auto& inf = L->reqs[rid];
  inf.client = client;
  inf.t_arrival = t_arrival_ns ? t_arrival_ns : loop_now_ns();
  // the whole request in one aligned 64-bit store: the loop reads it in one load
  reinterpret_cast<volatile unsigned long long*>(L->req_ring)[L->req_tail & (L->ring - 1u)] =
      (unsigned long long)rid << 32 | client;
  std::atomic_thread_fence(std::memory_order_release);
  L->req_tail += 1u;
  reinterpret_cast<volatile unsigned int*>(&L->hin->req_tail)[0] = L->req_tail;
  L->submitted += 1;
  if (id) *id = rid;
  return VBH_OK;
}

vbh_status vbh_serve_loop_poll(vbh_serve_loop* L, vbh_serve_done* out, uint32_t cap,
                               uint32_t* n) {
  if (!L || !n || (cap && !out)) return fail(VBH_ERR_INVALID_ARG, "null argument");
  L->alive();
  L->collect();
  const uint32_t k = (uint32_t)std::min<size_t>(cap, L->ready.size());
  for (uint32_t i = 0; i < k; ++i) out[i] = L->ready[i];
  L->ready.erase(L->ready.begin(), L->ready.begin() + k);
  *n = k;
  return VBH_OK;
}

vbh_status vbh_serve_loop_result(vbh_serve_loop* L, uint32_t id, vbh_serve_view* out) {
  if (!L || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  auto it = L->reqs.find(id);
  if (it == L->reqs.end() || !it->second.done)
    return fail(VBH_ERR_INVALID_ARG, "no completed request with this id");
  const LoopDone& r = it->second.rec;
  out->n_records = r.n_records;
  out->flags = r.flags;
  if (r.region != 0xFFFFFFFFu) {
    out->recs_dev = reinterpret_cast<const int32_t*>(L->X.arena + r.off);
    out->indices_dev = L->X.arena + r.off + (size_t)r.cap * kRecHdr;
  } else {
    out->recs_dev = nullptr;
    out->indices_dev = nullptr;
  }
  return VBH_OK;
}

vbh_status vbh_serve_loop_release(vbh_serve_loop* L, uint32_t id) {
  if (!L) return fail(VBH_ERR_INVALID_ARG, "null loop");
  auto it = L->reqs.find(id);
  if (it == L->reqs.end() || !it->second.done)
    return fail(VBH_ERR_INVALID_ARG, "no completed request with this id");
  L->alive();
  const uint32_t region = it->second.rec.region;
  if (region != 0xFFFFFFFFu) {
    const uint32_t head = reinterpret_cast<volatile unsigned int*>(&L->hout->rel_head)[0];
    if (L->rel_tail - head >= L->ring) {
      if (L->exited()) return L->stopped_status();
      return fail(VBH_ERR_CAPACITY, "release ring full");
    }
    reinterpret_cast<volatile unsigned int*>(L->rel_ring)[L->rel_tail & (L->ring - 1u)] = region;
    std::atomic_thread_fence(std::memory_order_release);
    L->rel_tail += 1u;
    reinterpret_cast<volatile unsigned int*>(&L->hin->rel_tail)[0] = L->rel_tail;
  }
  L->reqs.erase(it);
  return VBH_OK;
}

vbh_status vbh_serve_loop_drain(vbh_serve_loop* L, uint64_t timeout_ns) {
  if (!L) return fail(VBH_ERR_INVALID_ARG, "null loop");
  const uint64_t t0 = loop_now_ns();
  for (;;) {
    L->alive();
    L->collect();
    if (L->completed >= L->submitted) return VBH_OK;
    if (L->exited()) return L->stopped_status();
    if (loop_now_ns() - t0 > timeout_ns)
      return fail(VBH_ERR_TIMEOUT, "serving loop drain: requests still in flight");
    usleep(2);
  }
}

vbh_status vbh_serve_loop_run(vbh_serve_loop* L, const vbh_serve_script* sc, vbh_serve_done* out,
                              uint32_t cap, uint32_t* n_out) {
  if (!L || !sc || !n_out || (sc->n_events && (!sc->t_ns || !sc->client)))
    return fail(VBH_ERR_INVALID_ARG, "null argument");
  *n_out = 0;
  uint32_t n_frames = 0;
  for (uint32_t i = 0; i < sc->n_events; ++i) {
    if (sc->client[i] < 0) ++n_frames;
    else if ((uint32_t)sc->client[i] >= L->X.n_clients)
      return fail(VBH_ERR_INVALID_ARG, "client out of range");
    if (i && sc->t_ns[i] < sc->t_ns[i - 1]) return fail(VBH_ERR_INVALID_ARG, "events not sorted");
  }
  if (n_frames && (!sc->depth_dev || !sc->T_wc || !sc->frame_id || !sc->frame_out))
    return fail(VBH_ERR_INVALID_ARG, "frame events need depth, poses, ids and an output");
  const uint64_t t0 = loop_now_ns();
  uint32_t ev = 0, fr = 0, k = 0;
  std::vector<vbh_serve_done> buf(256);
  for (;;) {
    const uint64_t t = loop_now_ns() - t0;
    while (ev < sc->n_events && sc->t_ns[ev] <= t) {
      vbh_status st;
      if (sc->client[ev] < 0) {
        st = vbh_process_frame(L->h, sc->depth_dev[fr], sc->T_wc + 12u * fr, sc->frame_id[fr],
                               sc->erase_radius, sc->frame_out);
        ++fr;
      } else {
        st = vbh_serve_loop_submit(L, (uint32_t)sc->client[ev], t0 + sc->t_ns[ev], nullptr);
      }
      if (st != VBH_OK) return st;
      ++ev;
    }
    uint32_t got = 0;
    vbh_status st = vbh_serve_loop_poll(L, buf.data(), (uint32_t)buf.size(), &got);
    if (st != VBH_OK) return st;
    for (uint32_t i = 0; i < got; ++i) {
      if (k < cap && out) out[k] = buf[i];
      ++k;
      st = vbh_serve_loop_release(L, buf[i].id);
      if (st != VBH_OK) return st;
    }
    if (ev == sc->n_events && L->completed >= L->submitted && L->ready.empty()) break;
    if (L->exited()) return L->stopped_status();
  }
  *n_out = std::min(k, cap);
  return VBH_OK;
}

vbh_status vbh_serve_loop_stats_read(vbh_serve_loop* L, vbh_serve_loop_stats* out) {
  if (!L || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  L->alive();
  LoopDev D;
  VBH_CUDA(cudaMemcpyAsync(&D, L->d, sizeof D, cudaMemcpyDeviceToHost, L->aux));
  VBH_CUDA(cudaStreamSynchronize(L->aux));
  std::memset(out, 0, sizeof *out);
  out->requests_done = L->completed;
  out->records_served = D.records_served;
  out->change_records_scanned = D.scanned;
  out->chunks = D.chunks;
  out->rounds = D.rounds;
  out->deferred_memory = D.deferred;
  out->bytes_in_use = D.a_in_use;
  out->bytes_peak = D.bytes_peak;
  out->max_active = D.max_active;
  out->status = L->exited() ? L->dev_status() : 0u;
  if (D.worker_err && !out->status) out->status = VBH_ERR_TIMEOUT;
  out->launches = L->launched ? 1u : 0u;
  return VBH_OK;
}

vbh_status vbh_serve_loop_stop(vbh_serve_loop* L) {
  if (!L) return fail(VBH_ERR_INVALID_ARG, "null loop");
  const bool by_itself = L->exited();
  reinterpret_cast<volatile unsigned int*>(&L->hin->stop)[0] = 1u;
  L->alive();
  // the scheduler sees the stop within a round and the workers leave after their current tile
  const uint64_t limit = std::max<uint64_t>(5000000000ull,
                                            4000ull * (uint64_t)L->cfg.idle_timeout_us);
  const uint64_t t0 = loop_now_ns();
  cudaError_t q = cudaErrorNotReady;
  while ((q = cudaStreamQuery(L->stream)) == cudaErrorNotReady) {
    if (loop_now_ns() - t0 > limit) break;
    usleep(20);
  }
  vbh_status st = VBH_OK;
  if (q == cudaErrorNotReady) {
    // cannot happen while the GPU runs the loop (every wait in it is bounded); keep the
    // server refused rather than free memory the kernel may still use
    return fail(VBH_ERR_TIMEOUT, "serving loop kernel did not stop");
  }
  if (q != cudaSuccess) st = fail(VBH_ERR_CUDA, std::string("serving loop: ") +
                                                    cudaGetErrorString(q));
  LoopDev D;
  if (st == VBH_OK && cudaMemcpy(&D, L->d, sizeof D, cudaMemcpyDeviceToHost) == cudaSuccess) {
    const unsigned int ds = L->dev_status();
    if (by_itself || ds) st = ds ? L->stopped_status() : VBH_OK;
    if (st == VBH_OK && D.worker_err)
      st = fail(VBH_ERR_TIMEOUT, "serving loop: a worker stopped waiting for the scheduler");
  }
  L->h->serve_loop_active = false;
  serve_set_loop(L->s, nullptr);
  vbh_status rv = serve_reload_versions(L->s);
  loop_free(L);
  return st != VBH_OK ? st : rv;
}

}  // extern "C"
