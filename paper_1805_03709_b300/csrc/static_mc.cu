// vbh_mc_from_tsdf_static: Marching Cubes indices of a caller's TSDF blocks without any device
// allocation (declared in include/vbh.h).
//
// Who needs it: callers that must not call cudaMalloc at all -- code running inside another
// framework's memory pool or allocator (where a stray cudaMalloc fragments or bypasses the
// pool), real-time threads that cannot risk the device-wide synchronisation an allocation can
// cause, and hosts that pre-reserve all memory at start-up.  Such a caller cannot create a
// vbh_handle (that allocates the table and pool), so this entry point works on buffers the
// caller already owns and keeps its scratch in a fixed array below.
//
// Scratch: one file-scope __device__ array of kScratchBytes (8 MiB + 256 B), present on every
// GPU that loads this library until the process exits.  Its first part is a key -> block-index
// hash table (2^16 buckets x 4 slots x 16 B), its second part the per-block sign/weight bit
// masks (2^15 blocks x 128 B), its last part an error word (bit0 key out of range, bit1 repeated
// key, bit2 stream capacity exceeded).  Every call re-initialises what it
// reads (the table is reset to EMPTY, the error word to 0, the masks of every input block are
// rewritten), so what a previous call left behind does not matter -- but all calls share the
// one array: calls whose work overlaps on the GPU (on different streams, or from different host
// threads) race and must be serialised by the caller.
#include <mutex>

#include "handle.cuh"

namespace vbh {

namespace {

constexpr unsigned int kStaticMaxBlocks = 1u << 15;
constexpr unsigned int kStaticBuckets = 1u << 16;
constexpr size_t kTableBytes = (size_t)kStaticBuckets * 4 * sizeof(Slot);
constexpr size_t kMaskBytes = (size_t)kStaticMaxBlocks * 32 * sizeof(unsigned int);
constexpr size_t kFlagBytes = 256;   // error word (+ padding)
constexpr size_t kScratchBytes = kTableBytes + kMaskBytes + kFlagBytes;
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the device symbol: its
// device address comes from cudaGetSymbolAddress (see scratch_address()).
static __device__ __align__(256) unsigned char g_mc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

constexpr unsigned long long kLo7 = 0x7F7F7F7F7F7F7F7Full;
constexpr unsigned long long kHi1 = 0x8080808080808080ull;

__device__ __forceinline__ unsigned long long zero_bytes_s(unsigned long long v) {
  unsigned long long y = (v & kLo7) + kLo7;
  return ~(y | v | kLo7);
}

__device__ __forceinline__ unsigned int row9_s(const unsigned int (*m)[32], int kind, int Y, int Z) {
  const int nb = 2 * (Y >> 3) + 4 * (Z >> 3);
  const int ly = Y & 7, lz = Z & 7;
  const int word = 16 * kind + (ly >> 2) + 2 * lz;
  const int sh = (ly & 3) * 8;
  return ((m[nb][word] >> sh) & 0xFFu) | (((m[nb + 1][word] >> sh) & 1u) << 8);
}

// One CTA per input block: enter its key into the scratch table (value = block index) and write
// its sign / weight masks.  A repeated key keeps the first entry that claimed a slot.
__global__ void __launch_bounds__(128) k_static_prepare(Slot* table, unsigned int* masks,
                                                        const int* keys3, const float* tsdf,
                                                        const float* weight, unsigned int n,
                                                        unsigned int* err) {
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int bmask = kStaticBuckets - 1u;
  for (unsigned int b = blockIdx.x; b < n; b += gridDim.x) {
    if (threadIdx.x == 0) {
      const int x = keys3[3u * b], y = keys3[3u * b + 1], z = keys3[3u * b + 2];
      if (!key_ok(x, y, z)) {
        atomicOr(err, 1u);
      } else {
        const unsigned long long key = pack_key(x, y, z);
        unsigned int h = hash_mix(key) & bmask;
        bool done = false;
        for (unsigned int probe = 0; probe <= bmask && !done; ++probe, h = (h + 1u) & bmask) {
          for (unsigned int l = 0; l < 4u && !done; ++l) {
            const unsigned long long old = atomicCAS(&table[4u * h + l].key, kEmpty, key);
            if (old == kEmpty) {
              table[4u * h + l].val = b;
              done = true;
            } else if (old == key) {
              atomicOr(err, 2u);   // duplicate key
              done = true;
            }
          }
        }
      }
    }
    for (unsigned int w = warp; w < 16u; w += blockDim.x >> 5) {
      const size_t v = 512ull * b + 32u * w + lane;
      const float f = tsdf[v], wt = weight[v];
      const unsigned int neg = __ballot_sync(0xFFFFFFFFu, f < 0.f);
      const unsigned int val = __ballot_sync(0xFFFFFFFFu, wt > 0.f);
      if (lane == 0) {
        masks[32u * b + w] = neg;
        masks[32u * b + 16u + w] = val;
      }
    }
  }
}

// One warp per input block: assemble the 9^3 corner lattice from the masks of the block and its
// seven positive neighbours (found in the scratch table), classify, compact into the stream.
__global__ void __launch_bounds__(128) k_static_mc(const Slot* table, const unsigned int* masks,
                                                   const int* keys3, unsigned int n,
                                                   int* rec_keys3, unsigned int* rec_info,
                                                   unsigned int* rec_off, unsigned int* rec_cnt,
                                                   unsigned short* ent_local,
                                                   unsigned char* ent_idx,
                                                   unsigned int cap_blocks,
                                                   unsigned int cap_entries,
                                                   unsigned int* n_blocks_dev,
                                                   unsigned int* n_entries_dev,
                                                   unsigned int* err) {
  __shared__ unsigned long long spread[256];
  __shared__ unsigned int msk[4][8][32];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) {
    unsigned long long v = 0;
    for (int i = 0; i < 8; ++i) v |= (unsigned long long)((b >> i) & 1) << (8 * i);
    spread[b] = v;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_blocks_dev = n;
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int nwarps = gridDim.x * 4u;
  const unsigned int bmask = kStaticBuckets - 1u;
  unsigned int(*m)[32] = msk[warp];
  for (unsigned int r = blockIdx.x * 4u + warp; r < n; r += nwarps) {
    const int kx = keys3[3u * r], ky = keys3[3u * r + 1], kz = keys3[3u * r + 2];
    unsigned int nb = kNone;
    if (lane == 0) {
      nb = r;
    } else if (lane < 8) {
      const int x = kx + (int)(lane & 1u), y = ky + (int)((lane >> 1) & 1u),
                z = kz + (int)((lane >> 2) & 1u);
      if (key_ok(x, y, z)) {
        const unsigned long long key = pack_key(x, y, z);
        unsigned int h = hash_mix(key) & bmask;
        for (unsigned int probe = 0; probe <= bmask; ++probe, h = (h + 1u) & bmask) {
          bool empty = false, hit = false;
          for (unsigned int l = 0; l < 4u; ++l) {
            const unsigned long long k = table[4u * h + l].key;
            if (k == key) { nb = table[4u * h + l].val; hit = true; break; }
            empty = empty || k == kEmpty;
          }
          if (hit || empty) break;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned int qn = __shfl_sync(0xFFFFFFFFu, nb, q);
      m[q][lane] = qn != kNone ? masks[32u * qn + lane] : 0u;
    }
    __syncwarp();
    unsigned long long idx8[2], nz[2];
    unsigned int mine = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = (int)lane + 32 * h, y = row & 7, z = row >> 3;
      const unsigned int n00 = row9_s(m, 0, y, z), n10 = row9_s(m, 0, y + 1, z);
      const unsigned int n01 = row9_s(m, 0, y, z + 1), n11 = row9_s(m, 0, y + 1, z + 1);
      const unsigned int va = row9_s(m, 1, y, z) & row9_s(m, 1, y + 1, z) &
                              row9_s(m, 1, y, z + 1) & row9_s(m, 1, y + 1, z + 1);
      unsigned long long c = spread[n00 & 0xFFu] | (spread[(n00 >> 1) & 0xFFu] << 1) |
                             (spread[(n10 >> 1) & 0xFFu] << 2) | (spread[n10 & 0xFFu] << 3) |
                             (spread[n01 & 0xFFu] << 4) | (spread[(n01 >> 1) & 0xFFu] << 5) |
                             (spread[(n11 >> 1) & 0xFFu] << 6) | (spread[n11 & 0xFFu] << 7);
      c &= spread[(va & (va >> 1)) & 0xFFu] * 0xFFull;
      c &= ~((zero_bytes_s(~c) >> 7) * 0xFFull);
      nz[h] = ~zero_bytes_s(c) & kHi1;
      idx8[h] = c;
      mine += __popcll(nz[h]);
    }
    unsigned int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if ((int)lane >= d) incl += v;
    }
    const unsigned int tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned int base = 0;
    if (lane == 0 && tot) base = atomicAdd(n_entries_dev, tot);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const bool fits = (unsigned long long)base + tot <= cap_entries;
    if (lane == 0 && (!fits || r >= cap_blocks)) atomicOr(err, 4u);   // stream overflow
    if (fits) {
      unsigned int o = base + incl - mine;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = (int)lane + 32 * h;
        unsigned long long bits = nz[h];
        while (bits) {
          const int x = (__ffsll((long long)bits) - 1) >> 3;
          ent_local[o] = (unsigned short)(x + 8 * row);
          ent_idx[o] = (unsigned char)(idx8[h] >> (8 * x));
          ++o;
          bits &= bits - 1ull;
        }
      }
    }
    if (lane == 0 && r < cap_blocks) {
      rec_keys3[3u * r] = kx;
      rec_keys3[3u * r + 1] = ky;
      rec_keys3[3u * r + 2] = kz;
      rec_info[r] = 0u;
      rec_off[r] = base;
      rec_cnt[r] = tot;
    }
    __syncwarp();
  }
}

// Device address of the scratch array on the current device; looked up once per device with
// that device current and kept for the life of the process (a cudaDeviceReset reloads the
// module, after which the kept address is stale: the entry point is not for processes that
// reset a device they have used it on).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace vbh

extern "C" vbh_status vbh_mc_from_tsdf_static(const int32_t* keys3_dev, const float* tsdf_dev,
                                              const float* weight_dev, uint32_t n_blocks,
                                              const vbh_mc_stream* out, void* cuda_stream,
                                              uint32_t* error_flags_dev) {
  using namespace vbh;
  if (!out || !out->n_blocks_dev || !out->n_entries_dev)
    return fail(VBH_ERR_INVALID_ARG, "vbh_mc_from_tsdf_static: null output stream or totals");
  if (n_blocks > kStaticMaxBlocks)   // the scratch holds 2^15 blocks
    return fail(VBH_ERR_INVALID_ARG,
                "vbh_mc_from_tsdf_static: n_blocks above the fixed scratch limit of 32768");
  if (n_blocks && (!keys3_dev || !tsdf_dev || !weight_dev))
    return fail(VBH_ERR_INVALID_ARG, "vbh_mc_from_tsdf_static: null input pointer");
  if ((out->cap_blocks && (!out->keys3 || !out->info || !out->offsets || !out->counts)) ||
      (out->cap_entries && (!out->local || !out->index)))
    return fail(VBH_ERR_INVALID_ARG, "vbh_mc_from_tsdf_static: incomplete output stream");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  VBH_CUDA(scratch_address(&base));
  unsigned char* b8 = static_cast<unsigned char*>(base);
  Slot* table = reinterpret_cast<Slot*>(b8);
  unsigned int* masks = reinterpret_cast<unsigned int*>(b8 + kTableBytes);
  unsigned int* err = reinterpret_cast<unsigned int*>(b8 + kTableBytes + kMaskBytes);
  VBH_CUDA(cudaMemsetAsync(out->n_entries_dev, 0, sizeof(uint32_t), stream));
  VBH_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), stream));
  if (n_blocks == 0) {
    VBH_CUDA(cudaMemsetAsync(out->n_blocks_dev, 0, sizeof(uint32_t), stream));
  } else {
    VBH_CUDA(cudaMemsetAsync(table, 0xFF, kTableBytes, stream));
    int sms = 0, dev = 0;
    VBH_CUDA(cudaGetDevice(&dev));
    VBH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned int cap = (unsigned)sms * 16u;
    const int grid_p = (int)(n_blocks < cap ? n_blocks : cap);
    k_static_prepare<<<grid_p, 128, 0, stream>>>(table, masks, keys3_dev, tsdf_dev, weight_dev,
                                                 n_blocks, err);
    const unsigned int warps = (n_blocks + 3u) / 4u;
    const int grid_m = (int)(warps < cap ? warps : cap);
    k_static_mc<<<grid_m, 128, 0, stream>>>(table, masks, keys3_dev, n_blocks, out->keys3,
                                            out->info, out->offsets, out->counts, out->local,
                                            out->index, out->cap_blocks, out->cap_entries,
                                            out->n_blocks_dev, out->n_entries_dev, err);
    VBH_CUDA(cudaGetLastError());
  }
  if (error_flags_dev)
    VBH_CUDA(cudaMemcpyAsync(error_flags_dev, err, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                             stream));
  return VBH_OK;
}
