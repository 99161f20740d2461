// Per-frame voxel block hashing kernels (Sec. 4.1): projective TSDF fusion and the visible set.
// (Band allocation is in alloc.cu; both follow the canonical decisions listed here.)
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

constexpr int kIntThreads = 128;     // fusion: 4 warps per CTA, one work unit per warp at a time

// ---- asynchronous bulk copies into shared memory (completion counted on an mbarrier)
__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arm the barrier for `bytes` and start one bulk copy global -> shared that completes them.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned int bytes,
                                          unsigned long long* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Approximate reciprocal (the hardware's rcp.approx, ~1 ulp) for the value path only.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Bounded wait: false (and the sticky timeout flag) if the copy has not landed within `limit`
// polls (limit 0 gives up at once: the handle's fault-injection setting).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity,
                                          unsigned int limit, DevCounters* cnt) {
  for (unsigned int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(&cnt->err, kErrTimeout);
  return false;
}

// Projective TSDF fusion of every voxel of every touched block; also rewrites the block's
// sign / weight bit masks.  A warp owns one work unit at a time -- kSlices of the block's 16
// voxel sets (a half block by default, so that the last round of units leaves fewer warps
// idle) -- with no barriers between warps: the unit's (TSDF, weight) pairs arrive in shared
// memory by one bulk asynchronous copy, started when the warp's previous unit is done with the
// buffer and waited for only after the projections and the first depth fetches of the unit.
// Lane L fuses voxels L + 32 m: shared-memory reads are conflict-free, global writes cover 256
// contiguous bytes, and the ballot over voxel set m is mask word m (collected in shared memory,
// stored by the lanes that own the words).  The touched list carries the pool index with the
// block's "fresh" bit, its key and its origin's camera depth.
#ifndef VBH_FUSE_GROUP
#define VBH_FUSE_GROUP 4
#endif
#ifndef VBH_FUSE_MIN_CTAS
#define VBH_FUSE_MIN_CTAS 1
#endif
#ifndef VBH_FUSE_SLICES
#define VBH_FUSE_SLICES 8
#endif
#ifndef VBH_FUSE_PACKED
#define VBH_FUSE_PACKED 1    // 1: the voxels of rows ly0 and ly0 + 4 share FP32x2 instructions
#endif
constexpr int kWarps = kIntThreads / 32;
constexpr int kGroup = VBH_FUSE_GROUP;     // voxels per lane whose depth fetches overlap
constexpr int kSlices = VBH_FUSE_SLICES;   // voxel sets (32 voxels each) per work unit
constexpr unsigned int kUnits = 16u / kSlices;   // work units per block
constexpr unsigned int kUnitVox = 32u * kSlices;
static_assert(kSlices % kGroup == 0 && 16 % kSlices == 0, "unit / group sizes");
static_assert(kGroup % 2 == 0 || !VBH_FUSE_PACKED, "packed pairs need an even group");

// The frame parameters arrive by value (the frame graph patches this node's argument every
// frame), so the compiler takes them as constant-bank operands instead of holding ~25 of them
// in registers, which leaves room for more resident warps to hide the depth-gather latency.
__global__ void __launch_bounds__(kIntThreads, VBH_FUSE_MIN_CTAS)
    k_integrate(const FrameParams fp, const float* __restrict__ dimg, PoolView pool,
                const unsigned int* touched, const unsigned long long* tkey,
                const float2* tdepth, const unsigned int* n_touched, DevCounters* cnt) {
  __shared__ __align__(128) float2 sbuf[kWarps][kUnitVox];
  __shared__ __align__(8) unsigned long long sbar[kWarps];
  __shared__ unsigned int smask[kWarps][32];
  __shared__ unsigned int s_upd;
  if (threadIdx.x == 0) s_upd = 0;
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    mbar_init(&sbar[warp]);
    mbar_fence_init();
  }
  __syncthreads();
  const unsigned int n_units = *n_touched * kUnits;
  const int lx = lane & 7, ly0 = lane >> 3;      // voxel (lx, ly0 + 4 (m & 1), m >> 1)
  const float R0 = fp.R[0], R1 = fp.R[1], R2 = fp.R[2], R3 = fp.R[3], R4 = fp.R[4],
              R5 = fp.R[5], R6 = fp.R[6], R7 = fp.R[7], R8 = fp.R[8];
  const float s = fp.s, t0 = fp.t[0], t1 = fp.t[1], t2 = fp.t[2];
  const float fx = fp.fx, fy = fp.fy, cxh = fp.cxh, cyh = fp.cyh;
  const float mu = fp.mu, inv_mu = fp.inv_mu, wmax = fp.wmax;
  const int width = fp.width, height = fp.height;
  // per-voxel part of the camera depth: tau(h, lz) = s (R_02 lx + R_12 ly + R_22 lz)
  //                                              = base[h] + lz * s R_22   (value path only)
  const float sR22 = s * R8;
  float tbase[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) tbase[h] = s * fmaf(R5, (float)(ly0 + 4 * h), R2 * (float)lx);
  unsigned int my_upd = 0;
  unsigned int parity = 0u;
  const unsigned int stride = gridDim.x * kWarps;
  unsigned int u = blockIdx.x * kWarps + warp;
  unsigned int rec = 0;
  if (u < n_units) {
    rec = touched[u / kUnits];
    if (lane == 0 && !(rec & kTouchedFresh))
      bulk_load(sbuf[warp], pool.vox + 512ull * (rec & ~kTouchedFresh) + kUnitVox * (u % kUnits),
                kUnitVox * 8u, &sbar[warp]);
  }
  bool alive = true;
  while (u < n_units && alive) {
    const unsigned int un = u + stride;
    const unsigned int rec_next = un < n_units ? touched[un / kUnits] : 0u;
    const unsigned int b = u / kUnits, part = u % kUnits;
    const unsigned int p = rec & ~kTouchedFresh;
    const bool fresh = (rec & kTouchedFresh) != 0;
    const int3 k = unpack_key(tkey[b]);
    const float2 bd = tdepth[b];
    const float2* vin = sbuf[warp];
    float2* vout = pool.vox + 512ull * p + kUnitVox * part;
    if (fresh) {   // a new block starts from zero: no copy was started for this unit
      float4* z = reinterpret_cast<float4*>(sbuf[warp]);
#pragma unroll
      for (unsigned int q = lane; q < kUnitVox / 2u; q += 32u) z[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncwarp();
    }
    const int z0 = 8 * k.z + (kSlices / 2) * (int)part;   // voxel z of the unit's first set
    const float dX = __fmaf_rn((float)(8 * k.x + lx), s, -t0);
    float ix[2], iy[2], iz[2];   // R_0j dX + R_1j dY for the rows ly0 and ly0 + 4
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float dY = __fmaf_rn((float)(8 * k.y + ly0 + 4 * h), s, -t1);
      ix[h] = __fmaf_rn(R3, dY, __fmul_rn(R0, dX));
      iy[h] = __fmaf_rn(R4, dY, __fmul_rn(R1, dX));
      iz[h] = __fmaf_rn(R5, dY, __fmul_rn(R2, dX));
    }
    // low-order part of the block depth folded into the per-voxel offsets (value path)
    const float lz0 = (float)((kSlices / 2) * (int)part);
    const float tb0 = fmaf(lz0, sR22, tbase[0] + bd.y), tb1 = fmaf(lz0, sR22, tbase[1] + bd.y);
#pragma unroll
    for (int g = 0; g < kSlices; g += kGroup) {
      bool ok[kGroup];
      float dm[kGroup];
#if VBH_FUSE_PACKED
      // voxels j (row ly0) and j + 1 (row ly0 + 4) share their z: every binary32 operation of
      // their decision chains runs as one FP32x2 instruction, which rounds each component
      // exactly as the scalar operation does
#pragma unroll
      for (int i = 0; i < kGroup; i += 2) {
        const int j = g + i;
        const float dZ = __fmaf_rn((float)(z0 + (j >> 1)), s, -t2);
        const float2 dZ2 = make_float2(dZ, dZ);
        const float2 px = __ffma2_rn(make_float2(R6, R6), dZ2, make_float2(ix[0], ix[1]));
        const float2 py = __ffma2_rn(make_float2(R7, R7), dZ2, make_float2(iy[0], iy[1]));
        const float2 pz = __ffma2_rn(make_float2(R8, R8), dZ2, make_float2(iz[0], iz[1]));
        const float2 r = make_float2(__frcp_rn(pz.x), __frcp_rn(pz.y));
        const float2 au = __ffma2_rn(__fmul2_rn(make_float2(fx, fx), px), r, make_float2(cxh, cxh));
        const float2 av = __ffma2_rn(__fmul2_rn(make_float2(fy, fy), py), r, make_float2(cyh, cyh));
        float2 d2;
        bool in2[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float auc = c ? au.y : au.x, avc = c ? av.y : av.x, pzc = c ? pz.y : pz.x;
          const int iu = __float2int_rd(auc), iv = __float2int_rd(avc);
          in2[c] = pzc > 0.0f && auc == auc && avc == avc &&
                   (unsigned int)iu < (unsigned int)width && (unsigned int)iv < (unsigned int)height;
          const int idx = in2[c] ? iv * width + iu : 0;
          (c ? d2.y : d2.x) = __ldg(dimg + idx);   // fl(raw ds), or -inf for an invalid pixel
        }
        // band test fl(d - p_z) >= -mu (d + (-p_z) rounds as d - p_z)
        const float2 band = __fadd2_rn(d2, make_float2(-pz.x, -pz.y));
        ok[i] = in2[0] && !(band.x < -mu);
        ok[i + 1] = in2[1] && !(band.y < -mu);
        dm[i] = d2.x;
        dm[i + 1] = d2.y;
      }
#else
#pragma unroll
      for (int i = 0; i < kGroup; ++i) {
        const int j = g + i, h = j & 1;
        const float dZ = __fmaf_rn((float)(z0 + (j >> 1)), s, -t2);
        const float px = __fmaf_rn(R6, dZ, ix[h]);
        const float py = __fmaf_rn(R7, dZ, iy[h]);
        const float pz = __fmaf_rn(R8, dZ, iz[h]);
        const float r = __frcp_rn(pz);
        const float au = __fmaf_rn(__fmul_rn(fx, px), r, cxh);
        const float av = __fmaf_rn(__fmul_rn(fy, py), r, cyh);
        // pixel = (floor au, floor av) inside the image: a conversion rounding down saturates
        // out-of-range values, so 0 <= floor(au) < width is an unsigned compare of it; NaN
        // (which that conversion would map to 0) is excluded explicitly
        const int iu = __float2int_rd(au), iv = __float2int_rd(av);
        const bool in = pz > 0.0f && au == au && av == av && (unsigned int)iu < (unsigned int)width &&
                        (unsigned int)iv < (unsigned int)height;
        const int idx = in ? iv * width + iu : 0;
        const float d = __ldg(dimg + idx);   // fl(raw ds), or -inf for an invalid pixel
        ok[i] = in && !(__fsub_rn(d, pz) < -mu);
        dm[i] = d;
      }
#endif
      if (g == 0 && !fresh) {
        // the unit's voxels are needed from here on: their copy has been in flight during
        // the projections and the first group's depth fetches
        alive = __all_sync(0xFFFFFFFFu, mbar_wait(&sbar[warp], parity, fp.wait_limit, cnt));
        if (!alive) break;   // a copy that never landed (flag raised): stop this warp
        parity ^= 1u;
      }
#if VBH_FUSE_PACKED
      float2 vv[kGroup];
#pragma unroll
      for (int i = 0; i < kGroup; i += 2) {   // the pair's running means in FP32x2 as well
        const int j = g + i;
        const float2 va = vin[lane + 32 * j], vb = vin[lane + 32 * (j + 1)];
        const float tz = (float)(j >> 1);
        const float2 tau = __ffma2_rn(make_float2(tz, tz), make_float2(sR22, sR22),
                                      make_float2(tb0, tb1));
        const float2 sdf = __fadd2_rn(__fadd2_rn(make_float2(dm[i], dm[i + 1]),
                                                 make_float2(-bd.x, -bd.x)),
                                      make_float2(-tau.x, -tau.y));
        const float2 q = __fmul2_rn(sdf, make_float2(inv_mu, inv_mu));
        const float2 f = make_float2(fminf(1.0f, fmaxf(-1.0f, q.x)), fminf(1.0f, fmaxf(-1.0f, q.y)));
        const float2 w1 = __fadd2_rn(make_float2(va.y, vb.y), make_float2(1.0f, 1.0f));
        const float2 rc = make_float2(rcp_approx(w1.x), rcp_approx(w1.y));
        // running weighted mean, weight 1 per frame
        const float2 nx = __ffma2_rn(__fadd2_rn(f, make_float2(-va.x, -vb.x)), rc,
                                     make_float2(va.x, vb.x));
        vv[i] = ok[i] ? make_float2(nx.x, fminf(w1.x, wmax)) : va;
        vv[i + 1] = ok[i + 1] ? make_float2(nx.y, fminf(w1.y, wmax)) : vb;
      }
#endif
#pragma unroll
      for (int i = 0; i < kGroup; ++i) {
        const int j = g + i;
#if VBH_FUSE_PACKED
        const float2 v = vv[i];
#else
        const int h = j & 1;
        float2 v = vin[lane + 32 * j];
        if (ok[i]) {
          const float tau = fmaf((float)(j >> 1), sR22, h ? tb1 : tb0);
          const float sdf = (dm[i] - bd.x) - tau;
          const float f = fminf(1.0f, fmaxf(-1.0f, sdf * inv_mu));
          const float w1 = v.y + 1.0f;
          v.x = fmaf(f - v.x, rcp_approx(w1), v.x);   // running weighted mean, weight 1 per frame
          v.y = fminf(w1, wmax);
        }
#endif
        const bool wr = ok[i] || fresh;
        if (wr) vout[lane + 32 * j] = v;
        const unsigned int negm = __ballot_sync(0xFFFFFFFFu, v.x < 0.0f);
        const unsigned int valm = __ballot_sync(0xFFFFFFFFu, v.y > 0.0f);
        if (lane == 0) {
          smask[warp][j] = negm;
          smask[warp][16 + j] = valm;
        }
        my_upd += wr ? 1u : 0u;
      }
    }
    if (!alive) break;
    __syncwarp();   // the mask words are in shared memory; every lane is done with the buffer
    if (un < n_units && lane == 0 && !(rec_next & kTouchedFresh))
      bulk_load(sbuf[warp],
                pool.vox + 512ull * (rec_next & ~kTouchedFresh) + kUnitVox * (un % kUnits),
                kUnitVox * 8u, &sbar[warp]);
    // sign words kSlices part .. + kSlices - 1, weight words 16 + the same
    const unsigned int q = lane & 15u;
    if (q < (unsigned)kSlices)
      pool.masks[32u * p + (lane & 16u) + kSlices * part + q] = smask[warp][(lane & 16u) + q];
    if (lane == 0 && fresh && part == kUnits - 1u) pool.state[p] = 0u;
    __syncwarp();   // mask words read before the next unit overwrites them
    rec = rec_next;
    u = un;
  }
  if (!alive) {
    // wait (bounded) for this warp's copy still in flight before the CTA may exit
    for (unsigned int i = 0; i < (1u << 20) && !mbar_try_wait(&sbar[warp], parity); ++i) {
    }
  }
  atomicAdd(&s_upd, my_upd);
  __syncthreads();
  if (threadIdx.x == 0 && s_upd) {
    atomicAdd(&cnt->vox_updated, (unsigned long long)s_upd);
    atomicAdd(&cnt->tot_written, (unsigned long long)s_upd);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&cnt->tot_touched, (unsigned long long)*n_touched);
    atomicAdd(&cnt->tot_frames, 1ull);
  }
}

// Visible-set integration (the fusion set is the touched blocks plus every live block in view,
// so voxels of blocks the truncation band does not reach are still updated where they see free
// space): a scan of the pool appends each live block in view that this frame has not touched
// (its epoch mark) to the touched list, with its key and origin depth.  One reservation per CTA
// and round.
__global__ void __launch_bounds__(256) k_visible(const FrameCtl* ctl, PoolView pool,
                                                 unsigned int* touched,
                                                 unsigned long long* tkey, float2* tdepth,
                                                 unsigned int* n_touched) {
  __shared__ FrameParams fp;
  __shared__ unsigned int s_warp[8], s_base;
  load_frame_params(fp, ctl);
  if (!ctl->visible) return;   // uniform
  const unsigned int epoch = ctl->epoch_touch;
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int stride = gridDim.x * blockDim.x;
  const unsigned int rounds = (pool.max_blocks + stride - 1u) / stride;
  for (unsigned int r = 0; r < rounds; ++r) {
    const unsigned int p = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kEmpty;
    bool take = false;
    if (p < pool.max_blocks) {
      key = pool.pkeys[p];
      take = key != kEmpty && pool.mark[p] != epoch && block_in_view(fp, unpack_key(key), fp.zmax);
    }
    const unsigned int bal = __ballot_sync(0xFFFFFFFFu, take);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int run = 0;
      for (int w = 0; w < 8; ++w) {
        const unsigned int c = s_warp[w];
        s_warp[w] = run;
        run += c;
      }
      s_base = run ? atomicAdd(n_touched, run) : 0u;
    }
    __syncthreads();
    if (take) {
      const unsigned int k = s_base + s_warp[warp] + __popc(bal & ((1u << lane) - 1u));
      pool.mark[p] = epoch;
      touched[k] = p;   // live, so never fresh
      tkey[k] = key;
      tdepth[k] = block_depth(fp, unpack_key(key));
    }
    __syncthreads();
  }
}

}  // namespace

void launch_visible(const Launch& L, const FrameCtl* ctl, PoolView pool, unsigned int* touched,
                    unsigned long long* tkey, float2* tdepth, unsigned int* n_touched) {
  static const int grid = persistent_grid(k_visible, 256, L.sms);
  k_visible<<<grid, 256, 0, L.stream>>>(ctl, pool, touched, tkey, tdepth, n_touched);
}

void launch_integrate(const Launch& L, const FrameParams& fp, const float* dimg, PoolView pool,
                      const unsigned int* touched, const unsigned long long* tkey,
                      const float2* tdepth, const unsigned int* n_touched, DevCounters* cnt) {
  static const int grid = persistent_grid(k_integrate, kIntThreads, L.sms);
  k_integrate<<<grid, kIntThreads, 0, L.stream>>>(fp, dimg, pool, touched, tkey, tdepth,
                                                  n_touched, cnt);
}

const void* integrate_kernel() { return reinterpret_cast<const void*>(&k_integrate); }

}  // namespace vbh
