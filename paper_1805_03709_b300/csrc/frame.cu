// Per-frame voxel block hashing kernels (Sec. 4.1): band allocation and projective TSDF fusion.
//
// Canonical binary32 decisions.  Which block a depth sample falls in, which pixel a voxel
// projects to, and whether a voxel lies inside the truncation band are discontinuous functions
// of the inputs.  They are defined as the following sequences of correctly rounded binary32
// operations, written with rounding-explicit intrinsics so that nothing is contracted:
//   depth     d   = fl(raw * ds);  raw == 0 or (zmax > 0 and d > zmax) -> invalid pixel
//   sample j  z_j = fma(j, s, fl(d - mu)), j = 0..J, J = ceil(2 mu / s - 1e-6); z_j <= 0 skipped
//   ray       a_u = fl(fl(u - cx) / fx), a_v likewise; P = (fl(a_u z), fl(a_v z), z)
//   world     X_i = fma(R_i2, z, fma(R_i1, P_y, fma(R_i0, P_x, t_i)))
//   block     k_i = floor(fl(X_i * inv_bs)), inv_bs = fl(1 / (8 s)); outside [-2^20, 2^20) skipped
//   voxel     dX_i = fma(g_i, s, -t_i); p_j = fma(R_2j, dX_2, fma(R_1j, dX_1, fl(R_0j dX_0)))
//   pixel     p_z > 0; r = fl(1 / p_z); u = floor(fma(fl(fx p_x), r, fl(cx + 0.5))), v likewise;
//             valid iff 0 <= u < width and 0 <= v < height (compared as floats)
//   band      fl(d - p_z) >= -mu
// Values (the SDF fed into the running average) are computed more accurately than binary32:
// the camera depth of each block's origin is formed once per touched block (block_depth, in the
// kernel that builds the touched list) as an unevaluated sum of two floats with error-free
// transformations, so the per-voxel SDF error stays near 1e-8 m without any FP64 instruction.
#include "vbh_internal.cuh"

namespace vbh {

namespace {

constexpr int kTile = 16;            // 16 x 16 pixel tiles, one thread per pixel
constexpr int kTileThreads = kTile * kTile;
constexpr int kTileSet = 1024;       // shared-memory key set per tile (power of two)
constexpr int kIntThreads = 128;     // fusion: 4 voxels per thread, one block per CTA step

// Copy the per-call frame parameters into shared memory (one word per thread).
__device__ __forceinline__ void load_frame_params(FrameParams& dst, const FrameCtl* ctl) {
  constexpr int kWords = sizeof(FrameParams) / 4;
  static_assert(kWords <= 128, "FrameParams larger than one CTA's copy");
  if (threadIdx.x < kWords)
    reinterpret_cast<int*>(&dst)[threadIdx.x] = reinterpret_cast<const int*>(&ctl->fp)[threadIdx.x];
  __syncthreads();
}

// Band allocation: every valid pixel's samples -> block keys -> per-tile distinct set in shared
// memory -> appended to the candidate list (the global de-duplication is the hash insert).
__global__ void __launch_bounds__(kTileThreads) k_alloc_keys(const FrameCtl* ctl,
                                                             unsigned long long* cand,
                                                             unsigned int cap,
                                                             DevCounters* cnt) {
  __shared__ unsigned long long set[kTileSet];
  __shared__ FrameParams fp;
  load_frame_params(fp, ctl);
  for (int i = threadIdx.x; i < kTileSet; i += kTileThreads) set[i] = kEmpty;
  __syncthreads();
  const int tiles_x = (fp.width + kTile - 1) / kTile;
  const int tiles_y = (fp.height + kTile - 1) / kTile;
  const int n_tiles = tiles_x * tiles_y;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int pu = (tile % tiles_x) * kTile + (threadIdx.x % kTile);
    const int pv = (tile / tiles_x) * kTile + (threadIdx.x / kTile);
    if (pu < fp.width && pv < fp.height) {
      const unsigned short raw = __ldg(fp.depth + (size_t)pv * fp.width + pu);
      const float d = __fmul_rn((float)raw, fp.ds);
      if (raw != 0 && !(fp.zmax > 0.0f && d > fp.zmax)) {
        const float au = __fdiv_rn(__fsub_rn((float)pu, fp.cx), fp.fx);
        const float av = __fdiv_rn(__fsub_rn((float)pv, fp.cy), fp.fy);
        const float z0 = __fsub_rn(d, fp.mu);
        unsigned long long prev = kEmpty;
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
          bool ok = true;
#pragma unroll
          for (int i = 0; i < 3; ++i) ok = ok && q[i] >= -1048576.0f && q[i] < 1048576.0f;
          if (!ok) continue;
          const unsigned long long key = pack_key((int)q[0], (int)q[1], (int)q[2]);
          if (key == prev) continue;   // consecutive samples usually share a block
          prev = key;
          unsigned int h = hash_mix(key) & (kTileSet - 1);
          bool placed = false;
          for (int probe = 0; probe < 64; ++probe) {
            unsigned long long old = atomicCAS(&set[h], kEmpty, key);
            if (old == kEmpty || old == key) { placed = true; break; }
            h = (h + 1) & (kTileSet - 1);
          }
          if (!placed) {   // tile set saturated: hand the key straight to the global list
            unsigned int k = atomicAdd(&cnt->n_cand, 1u);
            if (k < cap) cand[k] = key;
          }
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTileSet; i += kTileThreads) {
      const unsigned long long key = set[i];
      const bool has = key != kEmpty;
      const unsigned int k = warp_append(&cnt->n_cand, has, 0xFFFFFFFFu);
      if (has) {
        if (k < cap) cand[k] = key;
        set[i] = kEmpty;
      }
    }
    __syncthreads();
  }
}

// Interleave two 16-bit masks: bit i of `even` -> bit 2i, bit i of `odd` -> bit 2i + 1.
__device__ __forceinline__ unsigned int interleave16(unsigned int even, unsigned int odd) {
  unsigned int x = even & 0xFFFFu, y = odd & 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  y = (y | (y << 8)) & 0x00FF00FFu;
  y = (y | (y << 4)) & 0x0F0F0F0Fu;
  y = (y | (y << 2)) & 0x33333333u;
  y = (y | (y << 1)) & 0x55555555u;
  return x | (y << 1);
}

// Projective TSDF fusion of every voxel of every touched block; also rewrites the block's
// sign / weight bit masks.  Thread t owns the voxel pairs q = t and t + 128 (voxels 2q, 2q + 1),
// moved with one 16-byte access each, so a warp access covers 512 contiguous bytes.  The depth
// fetch of all four voxels is issued unconditionally (clamped index, predicated use) so the
// loads overlap.
__global__ void __launch_bounds__(kIntThreads) k_integrate(const FrameCtl* ctl, PoolView pool,
                                                           const unsigned int* touched,
                                                           const float2* tdepth,
                                                           const unsigned int* n_touched,
                                                           DevCounters* cnt) {
  __shared__ unsigned int s_upd;
  __shared__ unsigned int s_fresh;
  __shared__ FrameParams fp;
  if (threadIdx.x == 0) s_upd = 0;
  load_frame_params(fp, ctl);
  const unsigned int n = *n_touched;
  const int t = threadIdx.x;
  const unsigned int lane = t & 31, warp = t >> 5;
  const int lx0 = 2 * (t & 3), ly = (t >> 2) & 7, lz0 = t >> 5;   // voxel (lx0 + e, ly, lz0 + 4j)
  // per-voxel part of the camera depth, s * (R_02 lx + R_12 ly + R_22 lz) (value path only)
  float tau[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e)
      tau[j][e] = fp.s * fmaf(fp.R[8], (float)(lz0 + 4 * j),
                              fmaf(fp.R[5], (float)ly, fp.R[2] * (float)(lx0 + e)));
  // frame constants in registers (the shared copy would be re-read after every barrier)
  const float R0 = fp.R[0], R1 = fp.R[1], R2 = fp.R[2], R3 = fp.R[3], R4 = fp.R[4],
              R5 = fp.R[5], R6 = fp.R[6], R7 = fp.R[7], R8 = fp.R[8];
  const float s = fp.s, t0 = fp.t[0], t1 = fp.t[1], t2 = fp.t[2];
  const float fx = fp.fx, fy = fp.fy, cxh = fp.cxh, cyh = fp.cyh, fw = fp.fw, fh = fp.fh;
  const float ds = fp.ds, zmax = fp.zmax, mu = fp.mu, inv_mu = fp.inv_mu, wmax = fp.wmax;
  const int width = fp.width;
  const unsigned short* __restrict__ depth = fp.depth;
  unsigned int my_upd = 0;
  for (unsigned int b = blockIdx.x; b < n; b += gridDim.x) {
    const unsigned int p = touched[b];
    const int3 k = unpack_key(pool.pkeys[p]);
    if (t == 0) s_fresh = pool.state[p] & kFresh;
    __syncthreads();
    const bool fresh = s_fresh != 0;
    float4* vox = reinterpret_cast<float4*>(pool.vox + 512ull * p);
    float4 v[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) v[j] = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : vox[t + 128 * j];
    const float2 bd = tdepth[b];
    const float dY = __fmaf_rn((float)(8 * k.y + ly), s, -t1);
    float ix[2], iy[2], iz[2];   // R_0j dX + R_1j dY, per voxel column e
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float dX = __fmaf_rn((float)(8 * k.x + lx0 + e), s, -t0);
      ix[e] = __fmaf_rn(R3, dY, __fmul_rn(R0, dX));
      iy[e] = __fmaf_rn(R4, dY, __fmul_rn(R1, dX));
      iz[e] = __fmaf_rn(R5, dY, __fmul_rn(R2, dX));
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float dZ = __fmaf_rn((float)(8 * k.z + lz0 + 4 * j), s, -t2);
      bool ok[2];
      float dm[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float px = __fmaf_rn(R6, dZ, ix[e]);
        const float py = __fmaf_rn(R7, dZ, iy[e]);
        const float pz = __fmaf_rn(R8, dZ, iz[e]);
        const float r = __frcp_rn(pz);
        const float uf = floorf(__fmaf_rn(__fmul_rn(fx, px), r, cxh));
        const float vf = floorf(__fmaf_rn(__fmul_rn(fy, py), r, cyh));
        const bool in = pz > 0.0f && uf >= 0.0f && uf < fw && vf >= 0.0f && vf < fh;
        const int idx = in ? (int)vf * width + (int)uf : 0;
        const unsigned short raw = __ldg(depth + idx);
        const float d = __fmul_rn((float)raw, ds);
        ok[e] = in && raw != 0 && !(zmax > 0.0f && d > zmax) && !(__fsub_rn(d, pz) < -mu);
        dm[e] = d;
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (!ok[e]) continue;
        const float sdf = ((dm[e] - bd.x) - bd.y) - tau[j][e];
        const float f = fminf(1.0f, fmaxf(-1.0f, sdf * inv_mu));
        float& F = e ? v[j].z : v[j].x;
        float& W = e ? v[j].w : v[j].y;
        F = F + __fdividef(f - F, W + 1.0f);
        W = fminf(W + 1.0f, wmax);
      }
      const bool wr = fresh || ok[0] || ok[1];
      if (wr) vox[t + 128 * j] = v[j];
      my_upd += wr ? 2u : 0u;
      const unsigned int ne = __ballot_sync(0xFFFFFFFFu, v[j].x < 0.0f);
      const unsigned int no = __ballot_sync(0xFFFFFFFFu, v[j].z < 0.0f);
      const unsigned int ve = __ballot_sync(0xFFFFFFFFu, v[j].y > 0.0f);
      const unsigned int vo = __ballot_sync(0xFFFFFFFFu, v[j].w > 0.0f);
      if (lane < 2) {   // lane 0: voxels of lanes 0-15, lane 1: lanes 16-31
        const unsigned int sh = 16u * lane;
        const unsigned int word = 2u * warp + 8u * j + lane;   // first voxel 64 warp + 256 j
        pool.masks[32u * p + word] = interleave16(ne >> sh, no >> sh);
        pool.masks[32u * p + 16u + word] = interleave16(ve >> sh, vo >> sh);
      }
    }
    __syncthreads();
    if (t == 0 && fresh) pool.state[p] = 0u;
  }
  atomicAdd(&s_upd, my_upd);
  __syncthreads();
  if (threadIdx.x == 0 && s_upd) {
    atomicAdd(&cnt->vox_updated, (unsigned long long)s_upd);
    atomicAdd(&cnt->tot_written, (unsigned long long)s_upd);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&cnt->tot_touched, (unsigned long long)n);
    atomicAdd(&cnt->tot_frames, 1ull);
  }
}

}  // namespace

void launch_alloc_keys(const Launch& L, const FrameCtl* ctl, int width, int height,
                       unsigned long long* cand, unsigned int cap, DevCounters* cnt) {
  static int grid = 0;
  if (!grid) grid = persistent_grid(k_alloc_keys, kTileThreads, L.sms);
  const int tiles = ((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
  k_alloc_keys<<<tiles < grid ? tiles : grid, kTileThreads, 0, L.stream>>>(ctl, cand, cap, cnt);
}

void launch_integrate(const Launch& L, const FrameCtl* ctl, PoolView pool,
                      const unsigned int* touched, const float2* tdepth,
                      const unsigned int* n_touched, DevCounters* cnt) {
  static int grid = 0;
  if (!grid) grid = persistent_grid(k_integrate, kIntThreads, L.sms);
  k_integrate<<<grid, kIntThreads, 0, L.stream>>>(ctl, pool, touched, tdepth, n_touched, cnt);
}

}  // namespace vbh
