// Internal device-side definitions of libvbh (not part of the C ABI).
//
// Data layout in HBM (one handle):
//   table   : n_buckets x 4 slots x 16 B.  Slot = {u64 key, u32 value, u32 pad}; a bucket is one
//             64 B line, read whole by one thread (four 16 B loads); a key's buckets follow its
//             probe sequence (home bucket, then steps of probe_step).  Keys are the
//             int3 block coordinate packed as three 21-bit fields (x + 2^20 | y + 2^20 << 21 |
//             z + 2^20 << 42); bit 63 is never set in a key, so EMPTY (all ones) and TOMB
//             (all ones but bit 0) cannot collide with one.
//   pool    : max_blocks x 512 float2 (TSDF, weight), 4 KiB per block, voxel lx + 8 ly + 64 lz.
//   masks   : max_blocks x 32 u32: words 0-15 hold "TSDF < 0" bits, words 16-31 "weight > 0"
//             bits of the 512 voxels (voxel i -> word i / 32, bit i % 32).  Written by every
//             fusion of the block; the Marching Cubes pass reads only these 128 B per block.
//   pkeys   : max_blocks u64, the packed key owning each pool entry (EMPTY when free).
//   state   : max_blocks u32, bit 0 = fresh (allocated, voxel data not yet written: reads as 0).
//   mark    : max_blocks u32 epoch stamps used to de-duplicate per-frame block lists.
//   version : max_blocks u32, frame version of the block's last MC refresh.
//   stack   : max_blocks u32 free pool indices, `free_top` of them valid.
//   seq     : max_blocks u32, change sequence number of the block's last MC refresh while a
//             server is attached (0 = none since allocation; reset when the block is erased).
// Serving state (allocated when a server attaches, see serve.cu):
//   log     : 2^L x 16 B ring of change records indexed by sequence number (LogEnt).
//   store   : max_blocks x 512 B dense MC cube indices of each live block at its last refresh.
//   lastrem : 2^R open-addressed (key u64, seq u32) pairs: sequence number of each key's last
//             removal, so that only the newest removal record of a key is served.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vbh {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kTomb = ~0ull - 1ull;
constexpr unsigned int kNone = 0xFFFFFFFFu;
constexpr unsigned int kPoolFail = 0xFFFFFFFEu;   // value of a slot whose pool pop failed
constexpr int kKeyBits = 21;
constexpr int kKeyOffset = 1 << 20;
constexpr unsigned int kFresh = 1u;

// sticky error flags (vbh_counters.error_flags)
constexpr unsigned int kErrPool = 1u, kErrTable = 2u, kErrStream = 4u, kErrTimeout = 8u,
                       kErrStreamOut = 16u;

// op codes and per-op statuses (same numbers as the C ABI)
constexpr unsigned char kOpFind = 0, kOpInsert = 1, kOpErase = 2;
constexpr unsigned char kStFound = 1, kStNotFound = 2, kStInserted = 3, kStExists = 4,
                        kStErased = 5, kStCapacity = 6, kStInvalid = 7;

struct __align__(16) Slot {
  unsigned long long key;
  unsigned int val;
  unsigned int pad;
};

// Device counters (one instance per handle, in device memory).
struct DevCounters {
  int free_top;                 // valid entries of the free stack
  unsigned int n_popped;        // pops in the current insert launch
  unsigned int n_exists;        // plain-map batch: inserts that met their key (value pending)
  // a hash batch's find / insert / erase list lengths, one set per batch parity: each batch's
  // first pass zeroes the other set for the next batch (no memset between batches)
  unsigned int op_lists[2][3];
  unsigned int n_live, n_tomb, n_empty;
  unsigned int n_cand, n_touched, n_new;
  unsigned int n_mset, n_tombrec, n_removed;
  unsigned int n_erased;
  unsigned int err;
  unsigned int mc_blocks, mc_entries;
  unsigned int rebuild_n;       // live entries copied by the last rebuild
  unsigned long long vox_updated;   // voxels written by the last frame (fused or zeroed)
  unsigned long long tot_touched;   // running totals over all fused frames (never reset)
  unsigned long long tot_new;
  unsigned long long tot_written;
  unsigned long long tot_frames;
  unsigned int gbar_arrive;   // arrivals at the small-batch kernel's grid barriers (only grows)
};

struct TableView {
  Slot* slots;
  unsigned int bmask;     // n_buckets - 1
  unsigned int hash_fn;   // 0 primes, 1 mix
};

struct PoolView {
  float2* vox;
  unsigned int* masks;
  unsigned long long* pkeys;
  unsigned int* state;
  unsigned int* mark;
  unsigned int* version;
  unsigned int* stack;
  unsigned int* seq;
  unsigned int max_blocks;  // 0 for a plain map
};

// Change record of the serving log.  key: packed block key, bit 63 set for a removal record;
// aux: pool index of a refreshed block, frame version of a removal; seq: its sequence number
// (a record whose seq differs from the index it is read at has been overwritten by the ring).
struct __align__(16) LogEnt {
  unsigned long long key;
  unsigned int aux;
  unsigned int seq;
};
constexpr unsigned long long kLogRemoved = 1ull << 63;

// Device-resident state shared by the per-frame MC extraction (which appends change records)
// and the serving kernels (which read them).
struct ServeLog {
  LogEnt* log;
  uint4* store;                    // 32 x 16 B per pool entry
  unsigned long long* rem_keys;    // lastrem table (kEmpty = free)
  unsigned int* rem_seq;
  unsigned int* sigma_host;        // mapped host word: last assigned sequence number
  unsigned int log_mask, rem_mask;
  unsigned int seq_next;           // next sequence number (starts at 1)
  unsigned int mc_done;            // CTAs of the running extraction that have finished
  unsigned int err;                // kServeErr* bits
};
constexpr unsigned int kServeErrRemFull = 1u, kServeErrOverrun = 2u, kServeErrCap = 4u;

// Stream-out (blocks leaving the active model move to host memory).  The erase kernels record
// each erased block's pool index and key at its erase number; the gather kernel copies them into
// the device transfer ring.
struct StreamList {
  unsigned int* p;           // nullptr: stream-out off
  unsigned long long* k;
};
struct StreamRing {
  float2* data;                        // cap x 512 (TSDF, weight)
  unsigned long long* keys;            // cap packed keys
  unsigned long long* head_host;       // mapped host word: slots ever filled
  unsigned long long head;             // slots ever filled (device copy)
  unsigned long long lost;             // blocks that found no room
  unsigned long long cap;              // slots
  unsigned int done;                   // CTAs of the running gather that finished
};

// Touched-list entry: pool index in bits 0-30, bit 31 set when the block is fresh (allocated by
// this frame, voxel data not yet written).
constexpr unsigned int kTouchedFresh = 0x80000000u;

// ------------------------------------------------------------------------------ keys, hashing
__host__ __device__ __forceinline__ bool key_ok(int x, int y, int z) {
  return x >= -kKeyOffset && x < kKeyOffset && y >= -kKeyOffset && y < kKeyOffset &&
         z >= -kKeyOffset && z < kKeyOffset;
}
__host__ __device__ __forceinline__ unsigned long long pack_key(int x, int y, int z) {
  return (unsigned long long)(unsigned)(x + kKeyOffset) |
         ((unsigned long long)(unsigned)(y + kKeyOffset) << kKeyBits) |
         ((unsigned long long)(unsigned)(z + kKeyOffset) << (2 * kKeyBits));
}
__host__ __device__ __forceinline__ int3 unpack_key(unsigned long long k) {
  const unsigned long long m = (1ull << kKeyBits) - 1ull;
  return make_int3((int)(k & m) - kKeyOffset, (int)((k >> kKeyBits) & m) - kKeyOffset,
                   (int)((k >> (2 * kKeyBits)) & m) - kKeyOffset);
}

// Sec. 5 "Retrieval": b = (x p1 XOR y p2 XOR z p3) mod n with p1 = 73856093, p2 = 19349669,
// p3 = 83492791, evaluated in uint32 wrap-around arithmetic; n is a power of two (mask).
__host__ __device__ __forceinline__ unsigned int hash_primes(unsigned long long packed) {
  int3 k = unpack_key(packed);
  return ((unsigned)k.x * 73856093u) ^ ((unsigned)k.y * 19349669u) ^ ((unsigned)k.z * 83492791u);
}
// SplitMix64 finaliser (Steele, Lea and Flood, 2014) of the packed key: neighbouring
// coordinates land in unrelated buckets.
__host__ __device__ __forceinline__ unsigned int hash_mix(unsigned long long z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (unsigned int)(z ^ (z >> 32));
}
__host__ __device__ __forceinline__ unsigned int home_bucket(unsigned long long packed,
                                                             unsigned int bmask, unsigned int fn) {
  return (fn == 0 ? hash_primes(packed) : hash_mix(packed)) & bmask;
}
// Probe sequence of a key (double hashing over buckets): its i-th bucket is (home + i * step)
// mod n_buckets with an odd step from a second, independent hash of the key, so the sequence
// visits every bucket once (n_buckets is a power of two) and keys that share a home bucket
// part after it: no primary clustering, and a walk that ends at the first bucket with an EMPTY
// slot stays short at high loads (at load 0.9 a miss reads ~4 buckets against ~13 when the
// sequence is the next bucket each time).
__host__ __device__ __forceinline__ unsigned int probe_step(unsigned long long packed) {
  return hash_mix(~packed) | 1u;
}

#ifdef __CUDACC__
// ------------------------------------------------------------------------ thread-per-op probe
// One thread reads a whole bucket (four 16 B loads from one 64 B line), so a warp keeps 32
// independent bucket reads in flight.  kReadOnly selects the non-coherent path for launches
// that do not modify the table; otherwise the loads go to L2, where the table's atomics land.
template <bool kReadOnly>
__device__ __forceinline__ void load_bucket(const Slot* b, ulonglong2 (&s)[4]) {
  const ulonglong2* p = reinterpret_cast<const ulonglong2*>(b);
  if constexpr (kReadOnly) {
    s[0] = __ldg(p); s[1] = __ldg(p + 1); s[2] = __ldg(p + 2); s[3] = __ldg(p + 3);
  } else {
    s[0] = __ldcg(p); s[1] = __ldcg(p + 1); s[2] = __ldcg(p + 2); s[3] = __ldcg(p + 3);
  }
}

// Slot q of a loaded bucket by a select chain (keeps the bucket in registers).
__device__ __forceinline__ ulonglong2 bucket_slot(const ulonglong2 (&s)[4], int q) {
  return q == 0 ? s[0] : q == 1 ? s[1] : q == 2 ? s[2] : s[3];
}

// Find by one thread: walk the key's probe sequence until the key or a bucket with an EMPTY
// slot.  Returns the slot index or kNone; *val receives the value and, if given,
// *bucket_empty whether the key's bucket held an EMPTY slot when it was read.  W buckets of the
// sequence are loaded per round trip (their addresses are known in advance); they are examined
// in sequence order, so the result is that of the one-bucket walk.
template <bool kReadOnly = false, int W = 1>
__device__ __forceinline__ unsigned int thread_find(const TableView& t, unsigned long long key,
                                                    unsigned int* val,
                                                    bool* bucket_empty = nullptr) {
  const unsigned int b0 = home_bucket(key, t.bmask, t.hash_fn);
  const unsigned int step = probe_step(key);
  for (unsigned int probe = 0; probe <= t.bmask; probe += W) {
    ulonglong2 s[W][4];
    unsigned int bb[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      bb[w] = (b0 + (probe + w) * step) & t.bmask;
      load_bucket<kReadOnly>(&t.slots[4u * bb[w]], s[w]);
    }
    // the first of the W buckets (in sequence order) that holds the key or an EMPTY slot
    bool stop = false;
    unsigned int pos = kNone, v = kNone;
    bool emp = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      int hit = -1;
      bool empty = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (s[w][q].x == key) hit = q;
        empty |= s[w][q].x == kEmpty;
      }
      const bool live = !stop && (W == 1 || probe + w <= t.bmask);   // every bucket once
      if (live && hit >= 0) {
        pos = 4u * bb[w] + hit;
        v = (unsigned)bucket_slot(s[w], hit).y;
        emp = empty;
      }
      stop |= live && (hit >= 0 || empty);
    }
    if (stop) {
      *val = v;
      if (pos != kNone && bucket_empty) *bucket_empty = emp;
      return pos;
    }
  }
  *val = kNone;
  return kNone;
}

// Erase phase: remove `key` from the slot thread_find returned.  The slot becomes EMPTY when its
// bucket already held an EMPTY slot: every find that reaches the bucket stops there anyway, so
// no probe sequence changes (no live key has a bucket with an EMPTY slot between its home
// bucket and its own, and such buckets only gain EMPTY slots this way), and the slot ends the
// chains of later inserts as a never-used slot would.  Otherwise it becomes a tombstone.
// Returns 0 (another erase got there first), 1 (now EMPTY) or 2 (now a tombstone).
__device__ __forceinline__ int erase_found(const TableView& t, unsigned int pos,
                                           unsigned long long key, bool bucket_empty) {
  const unsigned long long to = bucket_empty ? kEmpty : kTomb;
  if (atomicCAS(&t.slots[pos].key, key, to) != key) return 0;
  return bucket_empty ? 1 : 2;
}

// Warp-aggregated append: every lane with `pred` gets a distinct index from *counter.
__device__ __forceinline__ unsigned int warp_append(unsigned int* counter, bool pred,
                                                    unsigned int active_mask) {
  unsigned int bal = __ballot_sync(active_mask, pred);
  if (!bal) return kNone;
  unsigned int lane = threadIdx.x & 31u;
  unsigned int leader = __ffs(bal) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(bal));
  base = __shfl_sync(active_mask, base, (int)leader);
  return pred ? base + (unsigned)__popc(bal & ((1u << lane) - 1u)) : kNone;
}
// Error-free transformations: s + e == a + b exactly (Knuth's TwoSum); p + e == a * b exactly
// (TwoProduct with a fused multiply-add; Ogita, Rump and Oishi 2005).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}

// CTAs of `kernel` that fit on the GPU at once (resident CTAs per SM x SMs).  Launchers keep it
// in a function-local `static const` (computed by the first launch, thread-safe).
template <class K>
inline int persistent_grid(K kernel, int threads, int sms) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0);
  return (occ < 1 ? 1 : occ) * sms;
}
#endif  // __CUDACC__

// ------------------------------------------------------------------------ per-frame constants
// Canonical binary32 decision arithmetic: the kernels evaluate every discrete decision with
// explicitly rounded intrinsics (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn, __frcp_rn, floorf)
// in the order the host documentation fixes, so that no compiler contraction changes a result.
struct FrameParams {
  float R[9];          // row-major R of T_wc
  float t[3];
  float s, mu, inv_mu, wmax, ds, zmax;
  float fx, fy, cxh, cyh;   // cxh = fl(cx + 0.5f)
  float cx, cy;
  float inv_bs;        // fl(1 / fl(8 s))
  float fw, fh;        // (float)width, (float)height
  int width, height;
  int J;               // band steps: samples j = 0..J
  unsigned int raw_max;   // raw depth r is valid iff 1 <= r <= raw_max (fl(r ds) <= zmax)
  unsigned int wait_limit;   // polls of a bounded device wait before it gives up
  const unsigned short* depth;
};

// Per-call control block in device memory.  Every entry point first launches one setup kernel
// whose only by-value argument is this struct; the setup kernel stores it and zeroes the
// per-call counters, and the work kernels read their per-call inputs (pose, depth pointer,
// epochs, output pointers) from it.  A whole frame captured as a CUDA graph can therefore be
// re-launched with new inputs by updating the argument of one kernel node.
constexpr unsigned int kResetFrame = 1u, kResetErase = 2u, kResetMset = 4u;
struct FrameCtl {
  FrameParams fp;
  float erase_c[3];
  float erase_r2;               // fl(R * R)
  unsigned int do_erase;        // 0 none, 1 radius (erase_c, erase_r2), 2 frustum (fp pose)
  float erase_zfar;             // frustum erase: far limit (0 = none)
  unsigned int visible;         // fusion set = touched blocks + every live block in view
  unsigned int epoch_touch, epoch_mset, version;
  unsigned int clear_removed;   // the extraction consumes the removal list
  unsigned int reset;           // kReset* bits: counters the setup kernel zeroes
  int* rec_keys3;               // MC output stream (caller buffers)
  unsigned int* rec_info;
  unsigned int* rec_off;
  unsigned int* rec_cnt;
  unsigned short* ent_local;
  unsigned char* ent_idx;
  unsigned int* n_blocks_dev;
  unsigned int* n_entries_dev;
  unsigned int cap_blocks, cap_entries;
  ServeLog* slog;               // attached server (nullptr: none)
  unsigned long long so_tail;   // stream-out ring slots the host has consumed
  unsigned int serve_mark;      // this extraction refreshes the store and appends to the log
  unsigned int store_only;      // no MC stream output (populating the store)
};

#ifdef __CUDACC__
// Copy the per-call frame parameters into shared memory (one word per thread).
__device__ __forceinline__ void load_frame_params(FrameParams& dst, const FrameCtl* ctl) {
  constexpr int kWords = sizeof(FrameParams) / 4;
  static_assert(kWords <= 128, "FrameParams larger than one CTA's copy");
  if (threadIdx.x < kWords)
    reinterpret_cast<int*>(&dst)[threadIdx.x] = reinterpret_cast<const int*>(&ctl->fp)[threadIdx.x];
  __syncthreads();
}
#endif  // __CUDACC__

#ifdef __CUDACC__
// Block k in view of the frame's pose (its bounding sphere, centre (8k + 3.5) s and radius
// fl(7 s), is not outside the frustum): camera coordinates of the centre by the voxel
// projection chain, the four side planes fx p_x + cxh p_z >= 0, (W - cxh) p_z - fx p_x >= 0
// (and in y) with the margin rho G, G = max(fx, fy) + max(cxh, W - cxh, cyh, H - cyh) (no
// smaller than any plane normal's norm, so every block with a voxel in view passes), near
// p_z >= -rho and, when zfar > 0, far p_z <= zfar + rho.  Binary32, rounding explicit.
__device__ __forceinline__ bool block_in_view(const FrameParams& fp, int3 k, float zfar) {
  const float c0 = __fmul_rn(__fadd_rn((float)(8 * k.x), 3.5f), fp.s);
  const float c1 = __fmul_rn(__fadd_rn((float)(8 * k.y), 3.5f), fp.s);
  const float c2 = __fmul_rn(__fadd_rn((float)(8 * k.z), 3.5f), fp.s);
  const float d0 = __fsub_rn(c0, fp.t[0]), d1 = __fsub_rn(c1, fp.t[1]), d2 = __fsub_rn(c2, fp.t[2]);
  const float px = __fmaf_rn(fp.R[6], d2, __fmaf_rn(fp.R[3], d1, __fmul_rn(fp.R[0], d0)));
  const float py = __fmaf_rn(fp.R[7], d2, __fmaf_rn(fp.R[4], d1, __fmul_rn(fp.R[1], d0)));
  const float pz = __fmaf_rn(fp.R[8], d2, __fmaf_rn(fp.R[5], d1, __fmul_rn(fp.R[2], d0)));
  const float rho = __fmul_rn(7.0f, fp.s);
  const float rx = __fsub_rn(fp.fw, fp.cxh), ry = __fsub_rn(fp.fh, fp.cyh);
  const float G = __fadd_rn(fmaxf(fp.fx, fp.fy), fmaxf(fmaxf(fp.cxh, rx), fmaxf(fp.cyh, ry)));
  const float m = -__fmul_rn(rho, G);
  const float a = __fmul_rn(fp.fx, px), b = __fmul_rn(fp.fy, py);
  if (!(pz >= -rho)) return false;
  if (zfar > 0.0f && !(pz <= __fadd_rn(zfar, rho))) return false;
  return __fmaf_rn(fp.cxh, pz, a) >= m && __fmaf_rn(rx, pz, -a) >= m &&
         __fmaf_rn(fp.cyh, pz, b) >= m && __fmaf_rn(ry, pz, -b) >= m;
}

// Camera depth of a block's origin, sum_i R_i2 (8 k_i s - t_i), as an unevaluated hi + lo sum
// of floats (exact up to ~1e-13 m); feeds the value path of the fusion, never a decision.
__device__ __forceinline__ float2 block_depth(const FrameParams& fp, int3 k) {
  const int kk[3] = {k.x, k.y, k.z};
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 P = two_prod((float)(8 * kk[i]), fp.s);     // 8 k s, exact
    const float2 S = two_sum(P.x, -fp.t[i]);                 // (8 k s)_hi - t, exact
    const float al = __fadd_rn(S.y, P.y);                    // a = S.x + al
    const float r = fp.R[3 * i + 2];
    const float2 Q = two_prod(r, S.x);
    const float ql = __fmaf_rn(r, al, Q.y);
    const float2 T = two_sum(hi, Q.x);
    hi = T.x;
    lo = __fadd_rn(lo, __fadd_rn(T.y, ql));
  }
  return two_sum(hi, lo);
}
#endif

// ------------------------------------------------------------------------------- host launchers
struct Launch {
  cudaStream_t stream;
  int sms;            // persistent grids are (resident CTAs per SM) x sms
};

// A hash batch's valid inserts and erases, compacted by its first pass (which runs the finds
// itself): op index + packed key.
struct BatchLists {
  unsigned int* ins_idx = nullptr;
  unsigned long long* ins_key = nullptr;
  unsigned int* era_idx = nullptr;
  unsigned long long* era_key = nullptr;
  unsigned int* n = nullptr;        // this batch's list lengths: [1] inserts, [2] erases
                                    // ([0] stays 0); zero when it starts
  unsigned int* n_next = nullptr;   // the next batch's, zeroed by this batch's first pass
};

// hash.cu
// The batch's first pass: statuses of invalid ops, the finds, the insert and erase lists.
void launch_hash_find(const Launch& L, TableView t, DevCounters* cnt, const unsigned char* ops,
                      const int* keys3, unsigned int* res, unsigned char* st, unsigned int n,
                      BatchLists lists);
// keys: ops + keys3 (a batch), or pkeys + *count_dev (a key list; with idx, the list's op
// indices in the batch, for values, results and statuses)
void launch_hash_insert(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                        const unsigned long long* pkeys, const unsigned int* count_dev,
                        const unsigned int* vals, unsigned int* res, unsigned char* st,
                        unsigned int n, const unsigned int* idx = nullptr);
void launch_hash_insert_finish(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                               const unsigned int* count_dev, unsigned int* res,
                               unsigned char* st, unsigned int n, unsigned int* touched,
                               unsigned long long* tkey, float2* tdepth,
                               unsigned int* n_touched, const FrameCtl* ctl,
                               const unsigned int* idx = nullptr);
// The batch's erases, from the erase list its first pass compacted.
void launch_hash_erase(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       unsigned int* res, unsigned char* st, unsigned int n, BatchLists lists);
// A plain map's batch: the pending inserts' values and the erases in one launch.
void launch_hash_finish_erase(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                              unsigned int* res, unsigned char* st, unsigned int n,
                              BatchLists lists);
// A plain map's small batch in one cooperative launch, one thread per op (finds; inserts;
// insert values and erases, separated by grid barriers).  lists_next: the three list counts
// of the next phased batch, zeroed.  Returns cudaErrorInvalidValue when n ops need more CTAs
// than can be resident at once.
int small_batch_grid(const Launch& L);
bool small_batch_fits(const Launch& L, unsigned int n);   // n ops fit one resident grid
cudaError_t launch_hash_batch_small(const Launch& L, TableView t, DevCounters* cnt,
                                    const unsigned char* ops, const int* keys3,
                                    const unsigned int* vals, unsigned int* res,
                                    unsigned char* st, unsigned int n, unsigned int* lists_next,
                                    unsigned int* bar_base);
void launch_rebuild(const Launch& L, TableView t, const Slot* shadow, unsigned int n_slots,
                    DevCounters* cnt);
void launch_dump_table(const Launch& L, TableView t, unsigned int n_slots,
                       unsigned long long* out_keys, unsigned int* out_vals, unsigned int cap,
                       unsigned int* out_n);
void launch_gather_blocks(const Launch& L, PoolView pool, const unsigned int* idx,
                          unsigned int n, float* tsdf, float* w);
void launch_scatter_blocks(const Launch& L, PoolView pool, const unsigned int* idx,
                           unsigned int n, const float* tsdf, const float* w);
void launch_pack_keys(const Launch& L, const int* keys3, unsigned int n,
                      unsigned long long* out);
void launch_block_masks(const Launch& L, PoolView pool, const unsigned int* idx, unsigned int n);

// frame.cu
void launch_alloc_keys(const Launch& L, const FrameCtl* ctl, int width, int height,
                       unsigned long long* cand, unsigned int cap, DevCounters* cnt,
                       float* dimg);
void launch_integrate(const Launch& L, const FrameParams& fp, const float* dimg, PoolView pool,
                      const unsigned int* touched, const unsigned long long* tkey,
                      const float2* tdepth, const unsigned int* n_touched, DevCounters* cnt);
// The fusion kernel's entry (to find its node in a captured frame graph).
const void* integrate_kernel();
// Visible-set integration: append every live block in view that this frame did not touch.
void launch_visible(const Launch& L, const FrameCtl* ctl, PoolView pool, unsigned int* touched,
                    unsigned long long* tkey, float2* tdepth, unsigned int* n_touched);

// erase.cu
void launch_erase_radius(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                         const FrameCtl* ctl, unsigned long long* removed,
                         unsigned int removed_cap, int* out_keys3, unsigned int* out_n,
                         StreamList so);
void launch_erase_keys(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       const int* keys3, unsigned int n, unsigned long long* removed,
                       unsigned int removed_cap, int* out_keys3, unsigned int* out_n,
                       StreamList so);
void launch_stream_gather(const Launch& L, StreamRing* ring, const FrameCtl* ctl, PoolView pool,
                          DevCounters* cnt, StreamList so);

// mc.cu
void launch_mset_touched(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                         const FrameCtl* ctl, const unsigned int* touched,
                         const unsigned int* n_touched, const unsigned long long* removed,
                         const unsigned int* n_removed, unsigned int removed_cap,
                         unsigned int* mset, unsigned long long* tombrec);
void launch_mset_keys(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                      const FrameCtl* ctl, const int* keys3, unsigned int n, unsigned int* mset);
void launch_mset_scan(const Launch& L, PoolView pool, DevCounters* cnt, unsigned int* mset,
                      int since_mode, unsigned int since_version);
void launch_mc_extract(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       const FrameCtl* ctl, const unsigned int* mset,
                       const unsigned long long* tombrec);

}  // namespace vbh
