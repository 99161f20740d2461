// Band allocation of voxel block hashing (Sec. 4.1): every valid pixel's truncation band is
// sampled, each sample's block key goes into a per-tile set in shared memory, and the tile's
// distinct keys are appended to the candidate list (the global de-duplication is the hash
// insert that follows).  The canonical binary32 decisions (depth, samples, ray, world point,
// block) are those listed at the top of frame.cu.
#include "vbh_internal.cuh"

namespace vbh {

namespace {

#ifndef VBH_ALLOC_TILE_X
#define VBH_ALLOC_TILE_X 16
#endif
#ifndef VBH_ALLOC_TILE_Y
#define VBH_ALLOC_TILE_Y 16
#endif
constexpr int kTileX = VBH_ALLOC_TILE_X;   // pixel tiles of kTileX x kTileY, one thread per pixel
constexpr int kTileY = VBH_ALLOC_TILE_Y;
constexpr int kTileThreads = kTileX * kTileY;
constexpr int kTileSet = 4 * kTileThreads;   // shared-memory key set per tile (power of two)
static_assert((kTileSet & (kTileSet - 1)) == 0 && kTileThreads % 32 == 0, "tile shape");
// Band allocation: every valid pixel's samples -> block keys -> per-tile distinct set in shared
// memory -> appended to the candidate list (the global de-duplication is the hash insert).
// Every pixel's metric depth fl(raw ds) also goes to `dimg` for the fusion kernel, with invalid
// pixels (raw 0, or beyond zmax) as -inf: there the band test fl(d - p_z) >= -mu fails, so
// fusion needs no validity test, conversion or scaling of its own.
__global__ void __launch_bounds__(kTileThreads) k_alloc_keys(const FrameCtl* ctl,
                                                             unsigned long long* cand,
                                                             unsigned int cap,
                                                             DevCounters* cnt, float* dimg) {
  __shared__ unsigned long long set[kTileSet];
  __shared__ FrameParams fp;
  __shared__ unsigned int s_warp[kTileThreads / 32];
  __shared__ unsigned int s_base;
  const unsigned int lane = threadIdx.x & 31u;
  load_frame_params(fp, ctl);
  for (int i = threadIdx.x; i < kTileSet; i += kTileThreads) set[i] = kEmpty;
  __syncthreads();
  const int tiles_x = (fp.width + kTileX - 1) / kTileX;
  const int tiles_y = (fp.height + kTileY - 1) / kTileY;
  const int n_tiles = tiles_x * tiles_y;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int pu = (tile % tiles_x) * kTileX + (threadIdx.x % kTileX);
    const int pv = (tile / tiles_x) * kTileY + (threadIdx.x / kTileX);
    if (pu < fp.width && pv < fp.height) {
      const unsigned short raw = __ldg(fp.depth + (size_t)pv * fp.width + pu);
      const float d = __fmul_rn((float)raw, fp.ds);
      const bool valid = raw != 0 && !(fp.zmax > 0.0f && d > fp.zmax);
      dimg[(size_t)pv * fp.width + pu] = valid ? d : -INFINITY;
      if (valid) {
        const float au = __fdiv_rn(__fsub_rn((float)pu, fp.cx), fp.fx);
        const float av = __fdiv_rn(__fsub_rn((float)pv, fp.cy), fp.fy);
        const float z0 = __fsub_rn(d, fp.mu);
        float pq0 = 0.0f, pq1 = 0.0f, pq2 = 0.0f;   // the previous sample's block
        bool have_prev = false;
        // one sample's block: consecutive samples usually share a block, so it is compared with
        // the previous one before anything else is done with it (a repeated block had the same
        // range test and set insertion already)
        auto visit = [&](float q0, float q1, float q2) {
          if (have_prev && q0 == pq0 && q1 == pq1 && q2 == pq2) return;
          have_prev = true;
          pq0 = q0;
          pq1 = q1;
          pq2 = q2;
          if (!(q0 >= -1048576.0f && q0 < 1048576.0f && q1 >= -1048576.0f && q1 < 1048576.0f &&
                q2 >= -1048576.0f && q2 < 1048576.0f))
            return;
          const int kx = (int)q0, ky = (int)q1, kz = (int)q2;
          const unsigned long long key = pack_key(kx, ky, kz);
          // slot in the tile's set: a 32-bit mix of the coordinates (the set is small and local)
          unsigned int h = ((unsigned int)kx * 73856093u ^ (unsigned int)ky * 19349669u ^
                            (unsigned int)kz * 83492791u) & (kTileSet - 1);
          bool placed = false;
          for (int probe = 0; probe < 64; ++probe) {
            const unsigned long long seen = set[h];   // most keys are already in the set
            if (seen == key) { placed = true; break; }
            if (seen == kEmpty) {
              const unsigned long long old = atomicCAS(&set[h], kEmpty, key);
              if (old == kEmpty || old == key) { placed = true; break; }
            }
            h = (h + 1) & (kTileSet - 1);
          }
          if (!placed) {   // tile set saturated: hand the key straight to the global list
            unsigned int k = atomicAdd(&cnt->n_cand, 1u);
            if (k < cap) cand[k] = key;
          }
        };
        for (int j = 0; j <= fp.J; ++j) {
          const float z = __fmaf_rn((float)j, fp.s, z0);
          if (!(z > 0.0f)) continue;
          const float px = __fmul_rn(au, z);
          const float py = __fmul_rn(av, z);
          float q[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            float x = __fmaf_rn(fp.R[3 * i + 0], px, fp.t[i]);
            x = __fmaf_rn(fp.R[3 * i + 1], py, x);
            x = __fmaf_rn(fp.R[3 * i + 2], z, x);
            q[i] = floorf(__fmul_rn(x, fp.inv_bs));
          }
          visit(q[0], q[1], q[2]);
        }
      }
    }
    __syncthreads();
    // the tile's distinct keys go out with one reservation per CTA (atomics on one address
    // serialise in L2; one per warp would bound the kernel)
    constexpr int kPer = kTileSet / kTileThreads;
    unsigned long long mine[kPer];
    unsigned int nmine = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      mine[j] = set[threadIdx.x * kPer + j];
      nmine += mine[j] != kEmpty;
    }
    unsigned int incl = nmine;   // inclusive scan over the warp, then over the warps
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if ((int)lane >= d) incl += v;
    }
    if (lane == 31u) s_warp[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int run = 0;
      for (int w = 0; w < kTileThreads / 32; ++w) {
        const unsigned int c = s_warp[w];
        s_warp[w] = run;
        run += c;
      }
      s_base = run ? atomicAdd(&cnt->n_cand, run) : 0u;
    }
    __syncthreads();
    unsigned int o = s_base + s_warp[threadIdx.x >> 5] + incl - nmine;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (mine[j] != kEmpty) {
        if (o < cap) cand[o] = mine[j];
        ++o;
        set[threadIdx.x * kPer + j] = kEmpty;
      }
    }
    __syncthreads();
  }
}

}  // namespace

void launch_alloc_keys(const Launch& L, const FrameCtl* ctl, int width, int height,
                       unsigned long long* cand, unsigned int cap, DevCounters* cnt,
                       float* dimg) {
  static const int grid = persistent_grid(k_alloc_keys, kTileThreads, L.sms);
  const int tiles = ((width + kTileX - 1) / kTileX) * ((height + kTileY - 1) / kTileY);
  k_alloc_keys<<<tiles < grid ? tiles : grid, kTileThreads, 0, L.stream>>>(ctl, cand, cap, cnt,
                                                                          dimg);
}

}  // namespace vbh
