// Removal of voxel blocks that leave the active region (Sec. 4.1: blocks that are no longer in
// the sensor's view leave the GPU model).  An erase launch only turns keys into tombstones and
// returns pool entries to the free stack; each pool entry is owned by exactly one key, so the
// radius scan needs no de-duplication.
//
// Frustum erase (the scene reset of Sec. 4.1) removes every block in view of a pose by the
// block_in_view test.
// Canonical binary32 distance test of block k against point c and radius R:
//   centre_i = fl(fl((float)(8 k_i) + 3.5) * s); e_i = fl(centre_i - c_i)
//   d2 = fma(e_2, e_2, fma(e_1, e_1, fl(e_0 * e_0)));   erased iff d2 > fl(R * R)
#include "vbh_internal.cuh"

namespace vbh {

namespace {

constexpr int kThreads = 256;

// Remove one block: tombstone its key, free its pool entry, record it.
__device__ __forceinline__ void finish_removal(bool erased, unsigned int p, unsigned long long key,
                                               PoolView& pool, DevCounters* cnt,
                                               unsigned long long* removed,
                                               unsigned int removed_cap, int* out_keys3,
                                               const StreamList& so, unsigned int* s_erased,
                                               unsigned int* s_err) {
  unsigned int k = warp_append(reinterpret_cast<unsigned int*>(&cnt->free_top), erased,
                               0xFFFFFFFFu);
  if (erased) {
    pool.stack[k] = p;
    pool.pkeys[p] = kEmpty;
    pool.state[p] = 0u;
    pool.seq[p] = 0u;   // change records of the erased block are no longer current
  }
  unsigned int r = warp_append(&cnt->n_removed, erased, 0xFFFFFFFFu);
  if (erased) {
    if (r < removed_cap) removed[r] = key;
    else atomicOr(s_err, kErrStream);
  }
  unsigned int o = warp_append(&cnt->n_erased, erased, 0xFFFFFFFFu);
  if (erased) {
    atomicAdd(s_erased, 1u);
    if (so.p) {   // stream-out: the gather after this launch copies the block's voxels away
      so.p[o] = p;
      so.k[o] = key;
    }
    if (out_keys3) {
      int3 kk = unpack_key(key);
      out_keys3[3u * o] = kk.x;
      out_keys3[3u * o + 1] = kk.y;
      out_keys3[3u * o + 2] = kk.z;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_erase_radius(TableView t, PoolView pool,
                                                           DevCounters* cnt, const FrameCtl* ctl,
                                                           unsigned long long* removed,
                                                           unsigned int removed_cap,
                                                           int* out_keys3, StreamList so) {
  __shared__ unsigned int s_erased, s_err, s_emptied;
  if (threadIdx.x == 0) { s_erased = 0; s_err = 0; s_emptied = 0; }
  __syncthreads();
  const unsigned int mode = ctl->do_erase;
  if (!mode) return;   // uniform across the grid
  const float cx = ctl->erase_c[0], cy = ctl->erase_c[1], cz = ctl->erase_c[2];
  const float R2 = ctl->erase_r2, s = ctl->fp.s, zfar = ctl->erase_zfar;
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (pool.max_blocks + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int p = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kEmpty;
    if (p < pool.max_blocks) key = pool.pkeys[p];
    bool erased = false;
    if (key != kEmpty) {
      const int3 k = unpack_key(key);
      bool out;
      if (mode == 2u) {   // scene reset: every block in view of the given pose
        out = block_in_view(ctl->fp, k, zfar);
      } else {
        const float e0 = __fsub_rn(__fmul_rn(__fadd_rn((float)(8 * k.x), 3.5f), s), cx);
        const float e1 = __fsub_rn(__fmul_rn(__fadd_rn((float)(8 * k.y), 3.5f), s), cy);
        const float e2 = __fsub_rn(__fmul_rn(__fadd_rn((float)(8 * k.z), 3.5f), s), cz);
        const float d2 = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
        out = d2 > R2;
      }
      if (out) {
        unsigned int val;
        bool bucket_empty = false;
        const unsigned int pos = thread_find(t, key, &val, &bucket_empty);
        if (pos != kNone) {
          const int how = erase_found(t, pos, key, bucket_empty);
          erased = how != 0;
          if (how == 1) atomicAdd(&s_emptied, 1u);
        }
      }
    }
    finish_removal(erased, p, key, pool, cnt, removed, removed_cap, out_keys3, so, &s_erased,
                   &s_err);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_erased) {
      atomicSub(&cnt->n_live, s_erased);
      if (s_emptied) atomicAdd(&cnt->n_empty, s_emptied);
      if (s_erased > s_emptied) atomicAdd(&cnt->n_tomb, s_erased - s_emptied);
    }
    if (s_err) atomicOr(&cnt->err, s_err);
  }
}

__global__ void __launch_bounds__(kThreads) k_erase_keys(TableView t, PoolView pool,
                                                         DevCounters* cnt, const int* keys3,
                                                         unsigned int n,
                                                         unsigned long long* removed,
                                                         unsigned int removed_cap,
                                                         int* out_keys3, StreamList so) {
  __shared__ unsigned int s_erased, s_err, s_emptied;
  if (threadIdx.x == 0) { s_erased = 0; s_err = 0; s_emptied = 0; }
  __syncthreads();
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (n + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kEmpty;
    bool erased = false;
    unsigned int val = kNone;
    if (i < n) {
      const int x = keys3[3u * i], y = keys3[3u * i + 1], z = keys3[3u * i + 2];
      if (key_ok(x, y, z)) {
        key = pack_key(x, y, z);
        bool bucket_empty = false;
        const unsigned int pos = thread_find(t, key, &val, &bucket_empty);
        if (pos != kNone) {
          const int how = erase_found(t, pos, key, bucket_empty);
          erased = how != 0;
          if (how == 1) atomicAdd(&s_emptied, 1u);
        }
      }
    }
    finish_removal(erased, val, key, pool, cnt, removed, removed_cap, out_keys3, so, &s_erased,
                   &s_err);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_erased) {
      atomicSub(&cnt->n_live, s_erased);
      if (s_emptied) atomicAdd(&cnt->n_empty, s_emptied);
      if (s_erased > s_emptied) atomicAdd(&cnt->n_tomb, s_erased - s_emptied);
    }
    if (s_err) atomicOr(&cnt->err, s_err);
  }
}

// Stream-out gather: the voxels and keys of the blocks the preceding erase launch removed are
// copied into the next slots of the device transfer ring (before an allocation can reuse the
// pool entries).  The host copies filled slots to pinned memory and folds them into its map;
// the control block carries how far it has consumed, so the ring is never overwritten: blocks
// that do not fit are counted as lost and flagged, never dropped silently.  The last CTA to
// finish publishes the new head to host memory.
constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads) k_stream_gather(StreamRing* ring,
                                                                  const FrameCtl* ctl,
                                                                  PoolView pool,
                                                                  DevCounters* cnt,
                                                                  StreamList so) {
  __shared__ unsigned long long s_head;
  __shared__ unsigned int s_take, s_n;
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    const unsigned long long head = ring->head;
    const unsigned long long used = head - ctl->so_tail;   // <= capacity
    const unsigned long long room = ring->cap > used ? ring->cap - used : 0ull;
    const unsigned int n = cnt->n_erased;
    s_head = head;
    s_n = n;
    s_take = (unsigned int)(n < room ? n : room);
  }
  __syncthreads();
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int nwarps = gridDim.x * (kGatherThreads / 32);
  for (unsigned int o = blockIdx.x * (kGatherThreads / 32) + (threadIdx.x >> 5); o < s_take;
       o += nwarps) {
    const unsigned long long slot = (s_head + o) % ring->cap;
    const uint4* src = reinterpret_cast<const uint4*>(pool.vox + 512ull * so.p[o]);
    uint4* dst = reinterpret_cast<uint4*>(ring->data + 512ull * slot);
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[lane + 32 * i] = __ldcs(src + lane + 32 * i);
    if (lane == 0) ring->keys[slot] = so.k[o];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ring->done, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    ring->done = 0u;
    ring->head = s_head + s_take;
    if (s_take < s_n) {
      ring->lost += s_n - s_take;
      atomicOr(&cnt->err, kErrStreamOut);
    }
    __threadfence_system();
    *reinterpret_cast<volatile unsigned long long*>(ring->head_host) = s_head + s_take;
  }
}

}  // namespace

void launch_erase_radius(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                         const FrameCtl* ctl, unsigned long long* removed,
                         unsigned int removed_cap, int* out_keys3, unsigned int* out_n,
                         StreamList so) {
  static const int grid = persistent_grid(k_erase_radius, kThreads, L.sms);
  k_erase_radius<<<grid, kThreads, 0, L.stream>>>(t, pool, cnt, ctl, removed, removed_cap,
                                                  out_keys3, so);
  if (out_n)
    cudaMemcpyAsync(out_n, &cnt->n_erased, sizeof(unsigned int), cudaMemcpyDeviceToDevice,
                    L.stream);
}

void launch_erase_keys(const Launch& L, TableView t, PoolView pool, DevCounters* cnt,
                       const int* keys3, unsigned int n, unsigned long long* removed,
                       unsigned int removed_cap, int* out_keys3, unsigned int* out_n,
                       StreamList so) {
  static const int grid = persistent_grid(k_erase_keys, kThreads, L.sms);
  if (n)
    k_erase_keys<<<grid, kThreads, 0, L.stream>>>(t, pool, cnt, keys3, n, removed, removed_cap,
                                                  out_keys3, so);
  if (out_n)
    cudaMemcpyAsync(out_n, &cnt->n_erased, sizeof(unsigned int), cudaMemcpyDeviceToDevice,
                    L.stream);
}

void launch_stream_gather(const Launch& L, StreamRing* ring, const FrameCtl* ctl, PoolView pool,
                          DevCounters* cnt, StreamList so) {
  k_stream_gather<<<L.sms, kGatherThreads, 0, L.stream>>>(ring, ctl, pool, cnt, so);
}

}  // namespace vbh
