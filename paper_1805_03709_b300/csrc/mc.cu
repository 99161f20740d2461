// Marching Cubes index extraction (Sec. 4.2): per-voxel 8-bit cube indices of a set of blocks,
// with indices 0 and 255 (the set S^c) written as 0 and left out of the compacted stream.
//
// Block set.  After a fusion step the set is the touched blocks together with their seven
// neighbours in negative direction (k - o, o in {0,1}^3 \ 0): the cube at a voxel reads the
// corners g + {0,1}^3, so a change in block k alters cubes stored in those neighbours.  Blocks
// erased since the last extraction are reported as removal records, and their live negative
// neighbours are refreshed too (their cubes lose corners).  Lists are de-duplicated with epoch
// stamps on the pool entries.
//
// Cube index.  Corner i of the cube at voxel g is g + c_i with c = (000, 100, 110, 010, 001,
// 101, 111, 011) (x fastest); bit i is set iff TSDF(g + c_i) < 0; a cube with a corner in a
// missing block or with weight 0 is invalid and gets 0.  The kernel never reads TSDF values:
// fusion keeps a 128 B sign/weight bit mask per block, and one warp per block assembles the
// 9 x 9 x 9 corner lattice from the masks of the block and its 7 positive neighbours, then
// classifies a whole 8-voxel row at once: which cubes are emitted comes from 32-bit logic on
// the lattice's bit rows, the 8 index bytes from one 8 x 8 bit transpose.
//
// Serving.  While a server is attached, an extraction that refreshes blocks (the per-frame one)
// also stores each block's 512 dense cube indices, gives every record the next change sequence
// number e (refreshed blocks first, then removals), stamps seq[p] = e and writes the change
// record to log[e mod 2^L]; the last CTA to finish advances the sequence counter and publishes
// the last number to host memory.
#include "vbh_internal.cuh"

namespace vbh {

namespace {

constexpr int kThreads = 256;
constexpr int kMcThreads = 128;   // 4 warps, one block each
#ifndef VBH_MC_STAGE
#define VBH_MC_STAGE 512   // a smaller stage leaves the SM more L1 (19.3 -> 18.7 us per frame)
#endif
constexpr unsigned int kStage = VBH_MC_STAGE;   // MC entries staged per warp (>= 512, one block)
static_assert(kStage >= 512u, "a block's entries must fit the stage");
#ifndef VBH_MC_STAGE_BLOCKS
#define VBH_MC_STAGE_BLOCKS 16
#endif
constexpr unsigned int kStageBlocks = VBH_MC_STAGE_BLOCKS;   // blocks staged per warp (<= 32)

__device__ __forceinline__ void add_to_set(PoolView& pool, unsigned int q, unsigned int epoch,
                                           bool pred, unsigned int* mset, unsigned int* n_mset,
                                           int stamp_version, unsigned int version) {
  bool first = false;
  if (pred) first = atomicExch(&pool.mark[q], epoch) != epoch;
  unsigned int k = warp_append(n_mset, first, 0xFFFFFFFFu);
  if (first) {
    mset[k] = q;
    if (stamp_version) pool.version[q] = version;
  }
}

// touched blocks x 8 offsets, then removed keys x 8 offsets
__global__ void __launch_bounds__(kThreads) k_mset_touched(TableView t, PoolView pool,
                                                           DevCounters* cnt, const FrameCtl* ctl,
                                                           const unsigned int* touched,
                                                           const unsigned int* n_touched,
                                                           const unsigned long long* removed,
                                                           const unsigned int* n_removed,
                                                           unsigned int removed_cap,
                                                           unsigned int* mset,
                                                           unsigned long long* tombrec) {
  const unsigned int epoch = ctl->epoch_mset, version = ctl->version;
  const unsigned int nt = n_touched ? *n_touched : 0u;
  const unsigned int nr = min(*n_removed, removed_cap);
  const unsigned int items = 8u * (nt + nr);
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (items + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int e = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int q = kNone;
    bool tomb = false;
    unsigned long long tkey = 0;
    if (e < items) {
      const unsigned int o = e & 7u, b = e >> 3;
      unsigned long long key;
      bool is_removed = b >= nt;
      if (!is_removed) {
        const unsigned int p = touched[b] & ~kTouchedFresh;
        key = pool.pkeys[p];
        if (o == 0) q = key == kEmpty ? kNone : p;
      } else {
        key = removed[b - nt];
      }
      if (key != kEmpty && (o != 0 || is_removed)) {
        int3 k = unpack_key(key);
        k.x -= (int)(o & 1u);
        k.y -= (int)((o >> 1) & 1u);
        k.z -= (int)((o >> 2) & 1u);
        if (key_ok(k.x, k.y, k.z)) {
          unsigned int val;
          const unsigned long long nk = pack_key(k.x, k.y, k.z);
          unsigned int pos = thread_find(t, nk, &val);
          if (o == 0) {   // a removed key itself: a removal record unless it is live again
            tomb = pos == kNone;
            tkey = nk;
          } else if (pos != kNone) {
            q = val;
          }
        }
      }
    }
    add_to_set(pool, q, epoch, q != kNone, mset, &cnt->n_mset, 1, version);
    unsigned int k = warp_append(&cnt->n_tombrec, tomb, 0xFFFFFFFFu);
    if (tomb) tombrec[k] = tkey;
  }
}

// explicit keys x 8 offsets (o = 0 is the key itself)
__global__ void __launch_bounds__(kThreads) k_mset_keys(TableView t, PoolView pool,
                                                        DevCounters* cnt, const FrameCtl* ctl,
                                                        const int* keys3, unsigned int n,
                                                        unsigned int* mset) {
  const unsigned int epoch = ctl->epoch_mset;
  const unsigned int items = 8u * n;
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (items + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int e = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int q = kNone;
    if (e < items) {
      const unsigned int o = e & 7u, b = e >> 3;
      int x = keys3[3u * b] - (int)(o & 1u);
      int y = keys3[3u * b + 1] - (int)((o >> 1) & 1u);
      int z = keys3[3u * b + 2] - (int)((o >> 2) & 1u);
      if (key_ok(x, y, z)) {
        unsigned int val;
        if (thread_find(t, pack_key(x, y, z), &val) != kNone) q = val;
      }
    }
    add_to_set(pool, q, epoch, q != kNone, mset, &cnt->n_mset, 0, 0u);
  }
}

// every live pool entry (since_mode: only those with version > since)
__global__ void __launch_bounds__(kThreads) k_mset_scan(PoolView pool, DevCounters* cnt,
                                                        unsigned int* mset, int since_mode,
                                                        unsigned int since) {
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (pool.max_blocks + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int p = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    if (p < pool.max_blocks && pool.pkeys[p] != kEmpty)
      take = !since_mode || pool.version[p] > since;
    unsigned int k = warp_append(&cnt->n_mset, take, 0xFFFFFFFFu);
    if (take) mset[k] = p;
  }
}

// Sequence number e of the newest removal of `key` (lastrem table, linear probing; the table
// only grows, so a claimed key never moves).
__device__ __forceinline__ void note_removal(ServeLog* sl, unsigned long long key, unsigned int e) {
  unsigned int b = hash_mix(key) & sl->rem_mask;
  for (unsigned int probe = 0; probe <= sl->rem_mask; ++probe, b = (b + 1u) & sl->rem_mask) {
    const unsigned long long cur = atomicCAS(&sl->rem_keys[b], kEmpty, key);
    if (cur == kEmpty || cur == key) {
      atomicMax(&sl->rem_seq[b], e);
      return;
    }
  }
  atomicOr(&sl->err, kServeErrRemFull);
}

// 8 x 8 bit-matrix transpose of the 64-bit word hi:lo (row i = byte i, column j = bit j), by
// the three delta swaps of Hacker's Delight (Sec. 7-3): 2 x 2, 4 x 4 and 8 x 8 sub-blocks.  The
// first two swap within each 32-bit half; the third moves bits 4..7 of lo's bytes to bits 0..3
// of hi's and back.
__device__ __forceinline__ void transpose8x8(unsigned int& lo, unsigned int& hi) {
  unsigned int t;
  t = (lo ^ (lo >> 7)) & 0x00AA00AAu;
  lo ^= t ^ (t << 7);
  t = (hi ^ (hi >> 7)) & 0x00AA00AAu;
  hi ^= t ^ (t << 7);
  t = (lo ^ (lo >> 14)) & 0x0000CCCCu;
  lo ^= t ^ (t << 14);
  t = (hi ^ (hi >> 14)) & 0x0000CCCCu;
  hi ^= t ^ (t << 14);
  t = (lo ^ (hi << 4)) & 0xF0F0F0F0u;
  lo ^= t;
  hi ^= t >> 4;
}

// Bit i of an 8-bit value moved to bit 8 i (three masked shift steps: nibbles to 32-bit halves,
// pairs to 16-bit quarters, bits to bytes); times 0xFF it is the byte mask of the set bits.
__device__ __forceinline__ unsigned long long spread8(unsigned int b) {
  unsigned long long m = b;
  m = (m | (m << 28)) & 0x0000000F0000000Full;
  m = (m | (m << 14)) & 0x0003000300030003ull;
  m = (m | (m << 7)) & 0x0101010101010101ull;
  return m;
}

// The lattice of a block and its 7 positive neighbours (n = ox + 2 oy + 4 oz) in shared memory:
// L[n][w] = (sign word w, weight word w) of neighbour n, w = (ly >> 2) + 2 lz, byte ly & 3 of a
// word holding the 8 voxels x = 0..7 of row (ly, lz).  A 9-bit lattice row (x = 0..8) at
// (Y, Z), Y, Z in 0..8, is byte (Y & 3) of L[n][w] with bit 0 of the same byte of L[n + 1][w]
// (the +x neighbour) above it: one byte permute per kind builds it from two 8-byte loads.
struct LatticeRow {
  unsigned int off;   // n * 16 + w
  unsigned int sel;   // byte-permute selector: byte k of the first word, byte k of the second
};
__device__ __forceinline__ LatticeRow lattice_row(int Y, int Z) {
  const int n = 2 * (Y >> 3) + 4 * (Z >> 3);
  const int ly = Y & 7, lz = Z & 7;
  const unsigned int k = (unsigned int)(ly & 3);
  return LatticeRow{(unsigned int)(16 * n + (ly >> 2) + 2 * lz), k | ((4u + k) << 4)};
}

// 9 CTAs (36 warps) per SM at 56 registers, no spill: a room frame's ~14k-block set is at most
// three blocks per warp of the persistent grid.
#ifndef VBH_MC_MIN_CTAS
#define VBH_MC_MIN_CTAS 9
#endif
__global__ void __launch_bounds__(kMcThreads, VBH_MC_MIN_CTAS) k_mc_extract(TableView t, PoolView pool,
                                                          DevCounters* cnt, const FrameCtl* ctl,
                                                          const unsigned int* mset,
                                                          const unsigned long long* tombrec) {
  __shared__ __align__(16) uint2 msk[kMcThreads / 32][8 * 16];   // the lattice, per warp
  __shared__ unsigned short stage_loc[kMcThreads / 32][kStage];
  __shared__ unsigned char stage_idx[kMcThreads / 32][kStage];
  __shared__ unsigned int stage_r[kMcThreads / 32][kStageBlocks];
  __shared__ unsigned int stage_off[kMcThreads / 32][kStageBlocks];
  int* const rec_keys3 = ctl->rec_keys3;
  unsigned int* const rec_info = ctl->rec_info;
  unsigned int* const rec_off = ctl->rec_off;
  unsigned int* const rec_cnt = ctl->rec_cnt;
  unsigned short* const ent_local = ctl->ent_local;
  unsigned char* const ent_idx = ctl->ent_idx;
  unsigned int* const n_blocks_dev = ctl->n_blocks_dev;
  unsigned int* const n_entries_dev = ctl->n_entries_dev;
  const unsigned int cap_blocks = ctl->cap_blocks, cap_entries = ctl->cap_entries;
  const unsigned int tomb_version = ctl->version;
  ServeLog* const sl = ctl->serve_mark ? ctl->slog : nullptr;
  const bool emit = !ctl->store_only;
  __shared__ unsigned int s_seq0;
  if (threadIdx.x == 0) s_seq0 = sl ? sl->seq_next : 0u;   // every CTA reads it before the
  __syncthreads();                                        // last one advances it
  const unsigned int seq0 = s_seq0;
  const unsigned int n_m = cnt->n_mset, n_t = cnt->n_tombrec, total = n_m + n_t;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (emit) *n_blocks_dev = total;
    cnt->mc_blocks = total;
    if (ctl->clear_removed) cnt->n_removed = 0;   // the set kernel that read it has finished
  }
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int nwarps = gridDim.x * (kMcThreads / 32);
  uint2* const lat = msk[warp];
  // this lane's 2 x 4 lattice rows: rows y = lane & 7, z = (lane >> 3) + 4 h of the block,
  // each with its +y, +z, +y+z rows
  LatticeRow lr[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      lr[h][c] = lattice_row((int)(lane & 7u) + (c & 1), (int)(lane >> 3) + 4 * h + (c >> 1));
  bool overflow = false;
  // Entries are staged per warp in shared memory and leave with one reservation per flush
  // (atomics on one address serialise in L2: one per block would bound the kernel).
  unsigned short* const st_loc = stage_loc[warp];
  unsigned char* const st_idx = stage_idx[warp];
  unsigned int* const st_r = stage_r[warp];
  unsigned int* const st_off = stage_off[warp];
  unsigned int fill = 0u, nblk = 0u;   // warp-uniform
  auto flush = [&]() {
    __syncwarp();
    unsigned int base = 0u;
    if (lane == 0 && fill) base = atomicAdd(n_entries_dev, fill);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((unsigned long long)base + fill <= cap_entries) {
      for (unsigned int i = lane; i < fill; i += 32u) {
        ent_local[base + i] = st_loc[i];
        ent_idx[base + i] = st_idx[i];
      }
    } else {
      overflow = true;
    }
    if (lane < nblk && st_r[lane] < cap_blocks) rec_off[st_r[lane]] = base + st_off[lane];
    __syncwarp();
    fill = 0u;
    nblk = 0u;
  };
  // Refreshed blocks, software-pipelined over the warp's blocks: the next block's list entry,
  // key and first neighbour probe are loaded while the current block is classified.
  unsigned int r = blockIdx.x * (kMcThreads / 32) + warp;
  unsigned int q = 0u, nb = kNone;
  unsigned long long key = kEmpty;
  if (r < n_m) {
    q = mset[r];
    key = pool.pkeys[q];
    if (lane == 0) {
      nb = q;
    } else if (lane < 8) {
      const int3 k0 = unpack_key(key);
      const int x = k0.x + (int)(lane & 1u), y = k0.y + (int)((lane >> 1) & 1u),
                z = k0.z + (int)((lane >> 2) & 1u);
      unsigned int val;
      if (key_ok(x, y, z) && thread_find(t, pack_key(x, y, z), &val) != kNone) nb = val;
    }
  }
  for (; r < n_m; r += nwarps) {
    // lane L: neighbour L >> 2 (0 = the block itself), its sign words 4c .. 4c + 3 and weight
    // words 4c .. 4c + 3, c = L & 3 (two 16 B loads of its 128 B of masks)
    uint4 ms = make_uint4(0u, 0u, 0u, 0u), mwt = ms;
    {
      const unsigned int qn = __shfl_sync(0xFFFFFFFFu, nb, (int)(lane >> 2));
      if (qn != kNone) {
        const uint4* mp = reinterpret_cast<const uint4*>(pool.masks + 32u * qn);
        ms = __ldcg(mp + (lane & 3u));
        mwt = __ldcg(mp + 4u + (lane & 3u));
      }
    }
    const unsigned int rn = r + nwarps;
    unsigned int q_next = 0u;
    unsigned long long key_next = kEmpty, nkey = kEmpty;
    ulonglong2 pb0 = make_ulonglong2(0ull, 0ull), pb1 = pb0, pb2 = pb0, pb3 = pb0;
    if (rn < n_m) {
      q_next = mset[rn];
      key_next = pool.pkeys[q_next];
      if (lane >= 1u && lane < 8u) {
        const int3 kn = unpack_key(key_next);
        const int x = kn.x + (int)(lane & 1u), y = kn.y + (int)((lane >> 1) & 1u),
                  z = kn.z + (int)((lane >> 2) & 1u);
        if (key_ok(x, y, z)) {
          nkey = pack_key(x, y, z);
          const ulonglong2* bp = reinterpret_cast<const ulonglong2*>(
              &t.slots[4u * home_bucket(nkey, t.bmask, t.hash_fn)]);
          pb0 = __ldcg(bp);
          pb1 = __ldcg(bp + 1);
          pb2 = __ldcg(bp + 2);
          pb3 = __ldcg(bp + 3);
        }
      }
    }
    {   // lattice entries 16 n + 4 c .. + 3 (sign word, weight word) as two 16 B stores
      uint4* dst = reinterpret_cast<uint4*>(lat) + 8u * (lane >> 2) + 2u * (lane & 3u);
      dst[0] = make_uint4(ms.x, mwt.x, ms.y, mwt.y);
      dst[1] = make_uint4(ms.z, mwt.z, ms.w, mwt.w);
    }
    __syncwarp();
    const int3 k = unpack_key(key);
    // per row h: the 8 cube indices (byte x of hi:lo) and which of them are emitted (bit x of
    // e8: all 8 corners weighted, at least one corner negative, not all 8 negative)
    unsigned int idx_lo[2], idx_hi[2], e8[2];
    unsigned int mine = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // sign rows (Y, Z), (Y+1, Z), (Y, Z+1), (Y+1, Z+1) in bits 0..8 (bits above 8 are not
      // read) and the AND of their weight rows
      unsigned int sg[4], va = 0xFFFFFFFFu;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint2 a = lat[lr[h][c].off], b = lat[lr[h][c].off + 16u];
        sg[c] = __byte_perm(a.x, b.x, lr[h][c].sel);
        va &= __byte_perm(a.y, b.y, lr[h][c].sel);
      }
      const unsigned int n00 = sg[0], n10 = sg[1], n01 = sg[2], n11 = sg[3];
      // corner i's signs over x as byte i of hi:lo (corners 000 100 110 010 | 001 101 111 011),
      // then the 8 x 8 bit transpose: byte x = the cube index at x
      unsigned int lo = __byte_perm(__byte_perm(n00, n00 >> 1, 0x0040u),
                                    __byte_perm(n10 >> 1, n10, 0x0040u), 0x5410u);
      unsigned int hi = __byte_perm(__byte_perm(n01, n01 >> 1, 0x0040u),
                                    __byte_perm(n11 >> 1, n11, 0x0040u), 0x5410u);
      transpose8x8(lo, hi);
      const unsigned int any4 = n00 | n10 | n01 | n11, all4 = n00 & n10 & n01 & n11;
      e8[h] = va & (va >> 1) & (any4 | (any4 >> 1)) & ~(all4 & (all4 >> 1)) & 0xFFu;
      idx_lo[h] = lo;
      idx_hi[h] = hi;
      mine += __popc(e8[h]);
    }
    if (sl) {   // dense indices of voxel x + 8 row: row lane in word lane, row lane + 32 next
      // the refresh's number goes out before its indices: a serving loop that copies the store
      // concurrently reads the number before and after its copy and drops a changed block
      if (lane == 0) pool.seq[q] = seq0 + r;
      __syncwarp();
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      unsigned long long* st = reinterpret_cast<unsigned long long*>(sl->store + 32u * q);
#pragma unroll
      for (int h = 0; h < 2; ++h)   // cubes that are not emitted are stored as 0
        st[32u * h + lane] = (((unsigned long long)idx_hi[h] << 32) | idx_lo[h]) &
                             (spread8(e8[h]) * 0xFFull);
      if (lane == 0) {
        const unsigned int e = seq0 + r;
        LogEnt le;
        le.key = key;
        le.aux = q;
        le.seq = e;
        sl->log[e & sl->log_mask] = le;
      }
    }
    if (emit) {
      const unsigned int tot = __reduce_add_sync(0xFFFFFFFFu, mine);
      if (fill + tot > kStage || nblk == kStageBlocks) flush();
      if (tot) {   // warp-uniform: about a third of the blocks have no nonzero index
        unsigned int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
          if ((int)lane >= d) incl += v;
        }
        unsigned int o = fill + incl - mine;
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // the row's nonzero cubes, in x order, no divergence
          const unsigned int base_loc = 8u * (lane + 32u * h);
#pragma unroll
          for (int x = 0; x < 8; ++x) {
            if ((e8[h] >> x) & 1u) {
              st_loc[o] = (unsigned short)(base_loc + x);
              st_idx[o] = (unsigned char)((x < 4 ? idx_lo[h] : idx_hi[h]) >> (8 * (x & 3)));
              ++o;
            }
          }
        }
      }
      if (lane == 0) {
        st_r[nblk] = r;
        st_off[nblk] = fill;
        if (r < cap_blocks) {
          rec_keys3[3u * r] = k.x;
          rec_keys3[3u * r + 1] = k.y;
          rec_keys3[3u * r + 2] = k.z;
          rec_info[r] = pool.version[q] & 0x7FFFFFFFu;
          rec_cnt[r] = tot;
        }
      }
      fill += tot;
      nblk += 1u;
    }
    __syncwarp();   // the lattice in shared memory is refilled for the next block
    // the next block's neighbours: almost always settled by the prefetched home bucket
    unsigned int nb_next = kNone;
    if (lane == 0) {
      nb_next = q_next;
    } else if (nkey != kEmpty) {
      if (pb0.x == nkey) nb_next = (unsigned int)pb0.y;
      else if (pb1.x == nkey) nb_next = (unsigned int)pb1.y;
      else if (pb2.x == nkey) nb_next = (unsigned int)pb2.y;
      else if (pb3.x == nkey) nb_next = (unsigned int)pb3.y;
      else if (pb0.x != kEmpty && pb1.x != kEmpty && pb2.x != kEmpty && pb3.x != kEmpty) {
        unsigned int val;   // full home bucket: continue the probe sequence
        if (thread_find(t, nkey, &val) != kNone) nb_next = val;
      }
    }
    q = q_next;
    key = key_next;
    nb = nb_next;
  }
  if (emit) flush();
  for (; r < total; r += nwarps) {   // removal records
    if (lane == 0) {
      const unsigned long long tk = tombrec[r - n_m];
      if (emit && r < cap_blocks) {
        const int3 kk = unpack_key(tk);
        rec_keys3[3u * r] = kk.x;
        rec_keys3[3u * r + 1] = kk.y;
        rec_keys3[3u * r + 2] = kk.z;
        rec_info[r] = 0x80000000u | tomb_version;
        rec_off[r] = 0u;
        rec_cnt[r] = 0u;
      }
      if (sl) {
        const unsigned int e = seq0 + r;
        LogEnt le;
        le.key = tk | kLogRemoved;
        le.aux = tomb_version;
        le.seq = e;
        sl->log[e & sl->log_mask] = le;
        note_removal(sl, tk, e);
      }
    }
  }
  if (emit && (overflow || (total > cap_blocks && blockIdx.x == 0)) && lane == 0)
    atomicOr(&cnt->err, kErrStream);
  if (sl) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(&sl->mc_done, 1u) == gridDim.x - 1u) {
        sl->mc_done = 0u;
        sl->seq_next = seq0 + total;
        __threadfence_system();
        *reinterpret_cast<volatile unsigned int*>(sl->sigma_host) = seq0 + total - 1u;
      }
    }
  }
}

}  // namespace

void launch_mset_touched(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                         const FrameCtl* ctl, const unsigned int* touched,
                         const unsigned int* n_touched, const unsigned long long* removed,
                         const unsigned int* n_removed, unsigned int removed_cap,
                         unsigned int* mset, unsigned long long* tombrec) {
  static const int grid = persistent_grid(k_mset_touched, kThreads, L.sms);
  k_mset_touched<<<grid, kThreads, 0, L.stream>>>(t, pool, cnt, ctl, touched, n_touched, removed,
                                                  n_removed, removed_cap, mset, tombrec);
}

void launch_mset_keys(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                      const FrameCtl* ctl, const int* keys3, unsigned int n, unsigned int* mset) {
  static const int grid = persistent_grid(k_mset_keys, kThreads, L.sms);
  if (n) k_mset_keys<<<grid, kThreads, 0, L.stream>>>(t, pool, cnt, ctl, keys3, n, mset);
}

void launch_mset_scan(const Launch& L, PoolView pool, DevCounters* cnt, unsigned int* mset,
                      int since_mode, unsigned int since_version) {
  static const int grid = persistent_grid(k_mset_scan, kThreads, L.sms);
  k_mset_scan<<<grid, kThreads, 0, L.stream>>>(pool, cnt, mset, since_mode, since_version);
}

void launch_mc_extract(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       const FrameCtl* ctl, const unsigned int* mset,
                       const unsigned long long* tombrec) {
  static const int grid = persistent_grid(k_mc_extract, kMcThreads, L.sms);
  k_mc_extract<<<grid, kMcThreads, 0, L.stream>>>(t, pool, cnt, ctl, mset, tombrec);
}

}  // namespace vbh
