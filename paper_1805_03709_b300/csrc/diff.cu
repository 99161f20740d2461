// Differentiable window fusion: forward and hand-written backward of TSDF fusion with respect to
// per-pixel depth and per-frame se(3) pose (an extension of the fusion step of Sec. 4.1; the
// paper has no backward pass).
//
// Definition (shared with the C ABI documentation):
//   * a window of n_f frames of float32 metric depth is fused at fixed sample voxels g (world
//     position g s); F(g) = mean over valid frames of f = clamp(sdf / mu, -1, 1), with
//     sdf = D(u, v) - p_z, D bilinear in the frame's depth; L = sum_samples F^2;
//   * pose f is exp(xi_f), xi = (rho, omega): R = I + A [w]x + B [w]x^2, t = V rho,
//     V = I + B [w]x + C [w]x^2 (Rodrigues and the left Jacobian);
//   * validity and the bilinear cell of every (sample, frame) are fixed at nominal float32 poses
//     T0 by canonical binary32 arithmetic (p = R0^T (g s - t0) with the fusion's fma chain,
//     u = fma(fl(fx p_x), fl(1/p_z), cx), cell = floor(u, v), valid iff p_z > 0, the 2 x 2 cell
//     is inside the image, its four depths are > 0 and span at most mu -- no interpolation
//     across a depth discontinuity -- and the canonical bilinear sdf0 >= -mu), and
//     so is the side of the clamp (live, f = sdf / mu, iff sdf0 < mu; otherwise f = 1); at
//     other poses the same cell and side are kept, so L is smooth.
// The backward pass recomputes every projection instead of storing it; depth gradients are
// scattered with atomics.  With p = R^T (x - t) and g = dL/dp, the pose gradient of one sample
// is g . (R^T dR_k R p) - (R g) . dt_k; R^T dR_k is skew (R is a rotation), [k_k]x, so the
// first term is k_k . (g x p) and every frame needs only two sums, G = sum g and C = sum g x p
// (camera frame), contracted once per frame in FP64:
//   dL/dxi_k = k_k . C - (R G) . dt_k,   k_k = vee(R^T dR/dxi_k).
// G and C are summed in float within a thread's samples and over the warp, then in double per
// warp and per CTA; the per-CTA partials are reduced in a fixed order, so the pose gradient is
// deterministic.
#include "handle.cuh"

namespace vbh {

struct DiffPose {          // per frame, derived from xi on the device
  float R[9];
  float t[3];
  double Rd[9];
  double dR[6][9];
  double dt[6][3];
};

namespace {

constexpr int kDiffThreads = 256;
constexpr int kMaxDiffFrames = 256;

struct DiffParams {
  float s, mu, inv_mu, fx, fy, cx, cy;
  int W, H, nf, words;
};

__device__ void skew3(const double w[3], double S[9]) {
  S[0] = 0; S[1] = -w[2]; S[2] = w[1];
  S[3] = w[2]; S[4] = 0; S[5] = -w[0];
  S[6] = -w[1]; S[7] = w[0]; S[8] = 0;
}
__device__ void mul3(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// One thread per frame: exponential map and its derivatives, in FP64 (a few hundred operations
// per frame).  A, B, C and their theta-derivatives over theta use series below theta = 1e-3.
__global__ void k_diff_poses(const float* xi_f, int nf, DiffPose* out, float* T_out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double rho[3], w[3];
  for (int i = 0; i < 3; ++i) {
    rho[i] = xi_f[6 * f + i];
    w[i] = xi_f[6 * f + 3 + i];
  }
  const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]), t2 = th * th;
  double A, B, C, Ap, Bp, Cp;   // Ap = A'(th) / th etc.
  if (th < 1e-3) {
    A = 1 - t2 / 6 + t2 * t2 / 120;
    B = 0.5 - t2 / 24 + t2 * t2 / 720;
    C = 1.0 / 6 - t2 / 120 + t2 * t2 / 5040;
    Ap = -1.0 / 3 + t2 / 30 - t2 * t2 / 840;
    Bp = -1.0 / 12 + t2 / 180 - t2 * t2 / 6720;
    Cp = -1.0 / 60 + t2 / 1260 - t2 * t2 / 60480;
  } else {
    const double s = sin(th), c = cos(th);
    A = s / th;
    B = (1 - c) / t2;
    C = (th - s) / (t2 * th);
    Ap = (th * c - s) / (t2 * th);
    Bp = (th * s - 2 * (1 - c)) / (t2 * t2);
    Cp = (1 - c) / (t2 * t2) - 3 * (th - s) / (t2 * t2 * th);
  }
  double W[9], W2[9], V[9];
  skew3(w, W);
  mul3(W, W, W2);
  DiffPose P;
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    P.Rd[i] = I + A * W[i] + B * W2[i];
    V[i] = I + B * W[i] + C * W2[i];
    P.R[i] = (float)P.Rd[i];
  }
  double t[3];
  for (int i = 0; i < 3; ++i) {
    t[i] = V[3 * i] * rho[0] + V[3 * i + 1] * rho[1] + V[3 * i + 2] * rho[2];
    P.t[i] = (float)t[i];
  }
  for (int k = 0; k < 3; ++k) {
    for (int i = 0; i < 9; ++i) P.dR[k][i] = 0;
    for (int i = 0; i < 3; ++i) P.dt[k][i] = V[3 * i + k];
  }
  for (int k = 0; k < 3; ++k) {
    double e[3] = {0, 0, 0};
    e[k] = 1;
    double E[9], EW[9], WE[9], dV[9];
    skew3(e, E);
    mul3(E, W, EW);
    mul3(W, E, WE);
    for (int i = 0; i < 9; ++i) {
      P.dR[3 + k][i] = Ap * w[k] * W[i] + A * E[i] + Bp * w[k] * W2[i] + B * (EW[i] + WE[i]);
      dV[i] = Bp * w[k] * W[i] + B * E[i] + Cp * w[k] * W2[i] + C * (EW[i] + WE[i]);
    }
    for (int i = 0; i < 3; ++i)
      P.dt[3 + k][i] = dV[3 * i] * rho[0] + dV[3 * i + 1] * rho[1] + dV[3 * i + 2] * rho[2];
  }
  out[f] = P;
  if (T_out) {
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) T_out[12 * f + 4 * i + j] = P.R[3 * i + j];
      T_out[12 * f + 4 * i + 3] = P.t[i];
    }
  }
}

// Canonical binary32 cell and validity of sample g in frame f at the nominal pose T0.
__device__ __forceinline__ bool diff_cell(const DiffParams& c, int gx, int gy, int gz,
                                          const float* T0, const float* D, int* iu, int* iv,
                                          bool* live) {
  const float dX = __fmaf_rn((float)gx, c.s, -T0[3]);
  const float dY = __fmaf_rn((float)gy, c.s, -T0[7]);
  const float dZ = __fmaf_rn((float)gz, c.s, -T0[11]);
  const float px = __fmaf_rn(T0[8], dZ, __fmaf_rn(T0[4], dY, __fmul_rn(T0[0], dX)));
  const float py = __fmaf_rn(T0[9], dZ, __fmaf_rn(T0[5], dY, __fmul_rn(T0[1], dX)));
  const float pz = __fmaf_rn(T0[10], dZ, __fmaf_rn(T0[6], dY, __fmul_rn(T0[2], dX)));
  if (!(pz > 0.0f)) return false;
  const float r = __frcp_rn(pz);
  const float u = __fmaf_rn(__fmul_rn(c.fx, px), r, c.cx);
  const float v = __fmaf_rn(__fmul_rn(c.fy, py), r, c.cy);
  const float uf = floorf(u), vf = floorf(v);
  if (!(uf >= 0.0f && uf <= (float)(c.W - 2) && vf >= 0.0f && vf <= (float)(c.H - 2)))
    return false;
  const int a = (int)uf, b = (int)vf;
  const float d00 = D[b * c.W + a], d10 = D[b * c.W + a + 1];
  const float d01 = D[(b + 1) * c.W + a], d11 = D[(b + 1) * c.W + a + 1];
  if (!(d00 > 0.0f && d10 > 0.0f && d01 > 0.0f && d11 > 0.0f)) return false;
  const float dmax = fmaxf(fmaxf(d00, d10), fmaxf(d01, d11));
  const float dmin = fminf(fminf(d00, d10), fminf(d01, d11));
  if (__fsub_rn(dmax, dmin) > c.mu) return false;
  const float fa = __fsub_rn(u, uf), fb = __fsub_rn(v, vf);
  const float wa = __fsub_rn(1.0f, fa), wb = __fsub_rn(1.0f, fb);
  float Dv = __fmul_rn(__fmul_rn(wa, wb), d00);
  Dv = __fmaf_rn(__fmul_rn(fa, wb), d10, Dv);
  Dv = __fmaf_rn(__fmul_rn(wa, fb), d01, Dv);
  Dv = __fmaf_rn(__fmul_rn(fa, fb), d11, Dv);
  const float sdf0 = __fsub_rn(Dv, pz);
  if (sdf0 < -c.mu) return false;
  *iu = a;
  *iv = b;
  *live = sdf0 < c.mu;
  return true;
}

struct DiffTerm {
  float f;        // clamped observation
  float gs;       // d f / d sdf (1/mu inside the clamp, 0 outside)
  float w[4];     // bilinear weights of the cell's four depths
  float dDdu, dDdv;
  float p[3], y[3];
  int idx;        // depth index of the cell's (u0, v0)
};

// Value of sample g in frame f at pose (R, t), on the fixed cell (iu, iv).
__device__ __forceinline__ DiffTerm diff_term(const DiffParams& c, int gx, int gy, int gz,
                                              const float* R, const float* t, const float* D,
                                              int iu, int iv, bool live) {
  DiffTerm T;
  T.y[0] = (float)gx * c.s - t[0];
  T.y[1] = (float)gy * c.s - t[1];
  T.y[2] = (float)gz * c.s - t[2];
#pragma unroll
  for (int j = 0; j < 3; ++j) T.p[j] = R[j] * T.y[0] + R[3 + j] * T.y[1] + R[6 + j] * T.y[2];
  const float iz = 1.0f / T.p[2];
  const float u = c.fx * T.p[0] * iz + c.cx, v = c.fy * T.p[1] * iz + c.cy;
  const float a = u - (float)iu, b = v - (float)iv;
  T.idx = iv * c.W + iu;
  const float d00 = D[T.idx], d10 = D[T.idx + 1], d01 = D[T.idx + c.W], d11 = D[T.idx + c.W + 1];
  T.w[0] = (1.f - a) * (1.f - b);
  T.w[1] = a * (1.f - b);
  T.w[2] = (1.f - a) * b;
  T.w[3] = a * b;
  const float Dv = T.w[0] * d00 + T.w[1] * d10 + T.w[2] * d01 + T.w[3] * d11;
  const float q = (Dv - T.p[2]) * c.inv_mu;
  T.f = live ? q : 1.0f;
  T.gs = live ? c.inv_mu : 0.0f;
  T.dDdu = (1.f - b) * (d10 - d00) + b * (d11 - d01);
  T.dDdv = (1.f - a) * (d01 - d00) + a * (d11 - d10);
  return T;
}

__global__ void __launch_bounds__(kDiffThreads) k_diff_masks(DiffParams c, const int* samples,
                                                             unsigned int n, const float* depth,
                                                             const float* T0,
                                                             unsigned int* masks) {
  __shared__ float sT0[kMaxDiffFrames * 12];
  for (int i = threadIdx.x; i < c.nf * 12; i += blockDim.x) sT0[i] = T0[i];
  __syncthreads();
  for (unsigned int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int gx = samples[3u * s], gy = samples[3u * s + 1], gz = samples[3u * s + 2];
    for (int w = 0; w < c.words; ++w) {
      unsigned int bits = 0;
      for (int f = 32 * w; f < min(c.nf, 32 * w + 32); ++f) {
        int iu, iv;
        bool live;
        if (diff_cell(c, gx, gy, gz, sT0 + 12 * f, depth + (size_t)f * c.W * c.H, &iu, &iv,
                      &live))
          bits |= 1u << (f - 32 * w);
      }
      masks[(size_t)s * c.words + w] = bits;
    }
  }
}

__global__ void __launch_bounds__(kDiffThreads) k_diff_forward(DiffParams c, const int* samples,
                                                               unsigned int n, const float* depth,
                                                               const float* T0,
                                                               const DiffPose* poses,
                                                               const unsigned int* masks,
                                                               float* F, double* loss) {
  __shared__ float sT0[kMaxDiffFrames * 12];
  __shared__ float sRt[kMaxDiffFrames * 12];
  __shared__ double s_red[kDiffThreads / 32];
  for (int i = threadIdx.x; i < c.nf * 12; i += blockDim.x) {
    sT0[i] = T0[i];
    const int f = i / 12, e = i % 12;
    sRt[i] = e < 9 ? poses[f].R[e] : poses[f].t[e - 9];
  }
  __syncthreads();
  double acc = 0.0;
  for (unsigned int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int gx = samples[3u * s], gy = samples[3u * s + 1], gz = samples[3u * s + 2];
    float sum = 0.f;
    int cnt = 0;
    for (int w = 0; w < c.words; ++w) {
      unsigned int bits = masks[(size_t)s * c.words + w];
      while (bits) {
        const int f = 32 * w + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float* D = depth + (size_t)f * c.W * c.H;
        int iu = 0, iv = 0;
        bool live = false;
        diff_cell(c, gx, gy, gz, sT0 + 12 * f, D, &iu, &iv, &live);
        sum += diff_term(c, gx, gy, gz, sRt + 12 * f, sRt + 12 * f + 9, D, iu, iv, live).f;
        ++cnt;
      }
    }
    const float Fs = cnt ? sum / (float)cnt : 0.f;
    F[s] = Fs;
    acc += (double)Fs * (double)Fs;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kDiffThreads / 32; ++i) t += s_red[i];
    atomicAdd(loss, t);
  }
}

// Sum of 8 per-lane values over the warp in 9 shuffles (each step halves the values a lane
// carries); on return lane L holds the total of value L >> 2 (lanes with L & 3 == 0 hold them).
__device__ __forceinline__ float warp_sum8(const float v[8], unsigned int lane) {
  float w[4], x[2];
  const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b4 ? v[i + 4] : v[i], send = b4 ? v[i] : v[i + 4];
    w[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b3 ? w[i + 2] : w[i], send = b3 ? w[i] : w[i + 2];
    x[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
  }
  float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xFFFFFFFFu, b2 ? x[0] : x[1], 4);
  y += __shfl_xor_sync(0xFFFFFFFFu, y, 2);
  y += __shfl_xor_sync(0xFFFFFFFFu, y, 1);
  return y;
}

constexpr int kDiffChunk = 4;   // samples a thread holds while it walks the frames

// Per sample: dL/dF = 2F, spread over its valid frames; the depth gradient is scattered with
// atomics; per frame, G = sum g and C = sum g x p are summed over the thread's chunk of samples
// and the warp, accumulated in double per warp in shared memory, and written per CTA to
// part[cta][frame][6].  Dynamic shared memory: T0 and (R, t) as floats (2 x 12 nf) and the
// per-warp sums (warps x 6 nf doubles).
__global__ void __launch_bounds__(kDiffThreads) k_diff_backward(DiffParams c, const int* samples,
                                                                unsigned int n,
                                                                const float* depth,
                                                                const float* T0,
                                                                const DiffPose* poses,
                                                                const unsigned int* masks,
                                                                const float* F, float* gdepth,
                                                                double* part) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* sW = reinterpret_cast<double*>(dsm);                      // [warps][nf * 6]
  float* sT0 = reinterpret_cast<float*>(sW + (kDiffThreads / 32) * c.nf * 6);
  float* sRt = sT0 + c.nf * 12;
  for (int i = threadIdx.x; i < c.nf * 12; i += blockDim.x) {
    sT0[i] = T0[i];
    const int f = i / 12, e = i % 12;
    sRt[i] = e < 9 ? poses[f].R[e] : poses[f].t[e - 9];
  }
  for (int i = threadIdx.x; i < (kDiffThreads / 32) * c.nf * 6; i += blockDim.x) sW[i] = 0.0;
  __syncthreads();
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* myW = sW + warp * c.nf * 6;
  const unsigned int nthreads = gridDim.x * blockDim.x;
  const unsigned int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t npx = (size_t)c.W * c.H;
  for (size_t base = 0; base < n; base += (size_t)kDiffChunk * nthreads) {
    int gx[kDiffChunk], gy[kDiffChunk], gz[kDiffChunk];
    float gF[kDiffChunk];
    unsigned int sid[kDiffChunk], word[kDiffChunk];
#pragma unroll
    for (int j = 0; j < kDiffChunk; ++j) {
      const size_t s = base + (size_t)j * nthreads + tid;
      sid[j] = s < n ? (unsigned int)s : 0xFFFFFFFFu;
      gx[j] = gy[j] = gz[j] = 0;
      gF[j] = 0.f;
      word[j] = 0u;
      if (s < n) {
        gx[j] = samples[3 * s];
        gy[j] = samples[3 * s + 1];
        gz[j] = samples[3 * s + 2];
        int cnt = 0;
        for (int w = 0; w < c.words; ++w) cnt += __popc(masks[s * c.words + w]);
        gF[j] = cnt ? 2.0f * F[s] / (float)cnt : 0.f;
      }
    }
    for (int f = 0; f < c.nf; ++f) {   // frames in lockstep over the warp for the reductions
      if ((f & 31) == 0) {
#pragma unroll
        for (int j = 0; j < kDiffChunk; ++j)
          word[j] = (sid[j] != 0xFFFFFFFFu && gF[j] != 0.f)
                        ? masks[(size_t)sid[j] * c.words + (f >> 5)] : 0u;
      }
      const unsigned int bit = 1u << (f & 31);
      bool mine = false;
#pragma unroll
      for (int j = 0; j < kDiffChunk; ++j) mine |= (word[j] & bit) != 0u;
      if (!__any_sync(0xFFFFFFFFu, mine)) continue;
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float* D = depth + (size_t)f * npx;
      float* GD = gdepth + (size_t)f * npx;
#pragma unroll
      for (int j = 0; j < kDiffChunk; ++j) {
        if (!(word[j] & bit)) continue;
        int iu = 0, iv = 0;
        bool live = false;
        diff_cell(c, gx[j], gy[j], gz[j], sT0 + 12 * f, D, &iu, &iv, &live);
        if (!live) continue;   // saturated: f = 1, no gradient
        const DiffTerm T =
            diff_term(c, gx[j], gy[j], gz[j], sRt + 12 * f, sRt + 12 * f + 9, D, iu, iv, live);
        const float g = gF[j] * T.gs;   // dL / dsdf
        atomicAdd(GD + T.idx, g * T.w[0]);
        atomicAdd(GD + T.idx + 1, g * T.w[1]);
        atomicAdd(GD + T.idx + c.W, g * T.w[2]);
        atomicAdd(GD + T.idx + c.W + 1, g * T.w[3]);
        const float iz = 1.0f / T.p[2];
        const float gp0 = g * T.dDdu * c.fx * iz;
        const float gp1 = g * T.dDdv * c.fy * iz;
        const float gp2 = -(gp0 * T.p[0] + gp1 * T.p[1]) * iz - g;
        acc[0] += gp0;
        acc[1] += gp1;
        acc[2] += gp2;
        acc[3] += gp1 * T.p[2] - gp2 * T.p[1];
        acc[4] += gp2 * T.p[0] - gp0 * T.p[2];
        acc[5] += gp0 * T.p[1] - gp1 * T.p[0];
      }
      const float tot = warp_sum8(acc, lane);
      const unsigned int e = lane >> 2;
      if ((lane & 3u) == 0 && e < 6) myW[6 * f + e] += (double)tot;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c.nf * 6; i += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kDiffThreads / 32; ++w) t += sW[w * c.nf * 6 + i];
    part[(size_t)blockIdx.x * c.nf * 6 + i] = t;
  }
}

// dL/dxi per frame: one CTA of 6 warps per frame; warp e sums component e of (G, C) over the
// per-CTA partials in a fixed order, then thread 0 contracts with the exponential map's
// derivatives.
__global__ void k_diff_pose_grad(const DiffPose* poses, const double* part, int n_parts, int nf,
                                 float* gxi) {
  __shared__ double sGC[6];
  const int f = blockIdx.x, e = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double t = 0.0;
  for (int b = lane; b < n_parts; b += 32) t += part[((size_t)b * nf + f) * 6 + e];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
  if (lane == 0) sGC[e] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const DiffPose& P = poses[f];
  const double* G = sGC;
  const double* C = sGC + 3;
  double RG[3];
  for (int i = 0; i < 3; ++i)
    RG[i] = P.Rd[3 * i] * G[0] + P.Rd[3 * i + 1] * G[1] + P.Rd[3 * i + 2] * G[2];
  for (int k = 0; k < 6; ++k) {
    double K[9];   // R^T dR_k, skew
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        K[3 * i + j] = P.Rd[i] * P.dR[k][j] + P.Rd[3 + i] * P.dR[k][3 + j] +
                       P.Rd[6 + i] * P.dR[k][6 + j];
    const double kv[3] = {0.5 * (K[7] - K[5]), 0.5 * (K[2] - K[6]), 0.5 * (K[3] - K[1])};
    double acc = kv[0] * C[0] + kv[1] * C[1] + kv[2] * C[2];
    for (int i = 0; i < 3; ++i) acc -= RG[i] * P.dt[k][i];
    gxi[6 * f + k] = (float)acc;
  }
}

}  // namespace
}  // namespace vbh

// ------------------------------------------------------------------------------------ C ABI
struct vbh_diff {
  vbh_diff_config cfg;
  cudaStream_t stream;
  int sms;
  vbh::DiffPose* poses;
  double* part;        // per-CTA (G, C) partials of the backward pass: bwd_grid x nf x 6
  double* loss;        // device scalar used when the caller passes none
  int bwd_grid;        // resident CTAs of k_diff_backward (occupancy x SMs)
  size_t bwd_smem;     // its dynamic shared memory
};

namespace {
vbh::DiffParams diff_params(const vbh_diff* d) {
  vbh::DiffParams c;
  c.s = d->cfg.voxel_size;
  c.mu = d->cfg.trunc;
  c.inv_mu = 1.0f / d->cfg.trunc;
  c.fx = d->cfg.fx;
  c.fy = d->cfg.fy;
  c.cx = d->cfg.cx;
  c.cy = d->cfg.cy;
  c.W = d->cfg.width;
  c.H = d->cfg.height;
  c.nf = (int)d->cfg.n_frames;
  c.words = (c.nf + 31) / 32;
  return c;
}
// The status of the launches just enqueued, with the CUDA error as the last-error message.
vbh_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return VBH_OK;
  return vbh::fail(VBH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
int diff_grid(const vbh_diff* d, unsigned int n) {
  const unsigned int blocks = (n + vbh::kDiffThreads - 1) / vbh::kDiffThreads;
  const unsigned int cap = (unsigned)d->sms * 8u;
  return (int)(blocks < cap ? (blocks ? blocks : 1u) : cap);
}
}  // namespace

extern "C" {

vbh_status vbh_diff_create(const vbh_diff_config* cfg, void* cuda_stream, vbh_diff** out) {
  if (!cfg || !out) return vbh::fail(VBH_ERR_INVALID_ARG, "vbh_diff_create: null argument");
  *out = nullptr;
  if (!(cfg->voxel_size > 0.f) || !(cfg->trunc > 0.f) || cfg->width < 2 || cfg->height < 2 ||
      !(cfg->fx > 0.f) || !(cfg->fy > 0.f) || cfg->n_frames == 0 ||
      cfg->n_frames > (uint32_t)vbh::kMaxDiffFrames)
    return vbh::fail(VBH_ERR_INVALID_ARG,
                     "vbh_diff_create: voxel_size, trunc, fx, fy must be > 0, width and height "
                     ">= 2, n_frames in [1, " + std::to_string(vbh::kMaxDiffFrames) + "]");
  vbh_diff* d = new vbh_diff();
  d->cfg = *cfg;
  d->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMalloc(&d->poses, sizeof(vbh::DiffPose) * cfg->n_frames) != cudaSuccess ||
      cudaMalloc(&d->loss, sizeof(double)) != cudaSuccess) {
    vbh_diff_destroy(d);
    return vbh::fail(VBH_ERR_CUDA, "vbh_diff_create: device query or pose buffers failed");
  }
  d->bwd_smem = sizeof(double) * (vbh::kDiffThreads / 32) * 6 * cfg->n_frames +
                sizeof(float) * 24 * cfg->n_frames;
  int occ = 0;
  if (cudaFuncSetAttribute(vbh::k_diff_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)d->bwd_smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vbh::k_diff_backward,
                                                    vbh::kDiffThreads, d->bwd_smem) !=
          cudaSuccess ||
      occ < 1) {
    vbh_diff_destroy(d);
    return vbh::fail(VBH_ERR_CUDA,
                     "vbh_diff_create: the backward kernel does not fit with n_frames' shared "
                     "memory");
  }
  d->bwd_grid = occ * d->sms;
  if (cudaMalloc(&d->part, sizeof(double) * 6 * cfg->n_frames * (size_t)d->bwd_grid) !=
      cudaSuccess) {
    vbh_diff_destroy(d);
    return vbh::fail(VBH_ERR_CUDA, "vbh_diff_create: device memory for the pose partials");
  }
  *out = d;
  return VBH_OK;
}

vbh_status vbh_diff_destroy(vbh_diff* d) {
  if (!d) return VBH_OK;
  cudaStreamSynchronize(d->stream);
  if (d->poses) cudaFree(d->poses);
  if (d->part) cudaFree(d->part);
  if (d->loss) cudaFree(d->loss);
  delete d;
  return VBH_OK;
}

vbh_status vbh_diff_poses(vbh_diff* d, const float* xi_dev, float* T_dev) {
  if (!d || !xi_dev) return vbh::fail(VBH_ERR_INVALID_ARG, "vbh_diff_poses: null argument");
  const int nf = (int)d->cfg.n_frames;
  vbh::k_diff_poses<<<(nf + 63) / 64, 64, 0, d->stream>>>(xi_dev, nf, d->poses, T_dev);
  return launched("vbh_diff_poses");
}

vbh_status vbh_diff_masks(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                          const float* depth_dev, const float* T0_dev, uint32_t* masks_dev) {
  if (!d || (n && (!samples_dev || !depth_dev || !T0_dev || !masks_dev)))
    return vbh::fail(VBH_ERR_INVALID_ARG, "vbh_diff_masks: null argument");
  if (!n) return VBH_OK;
  vbh::k_diff_masks<<<diff_grid(d, n), vbh::kDiffThreads, 0, d->stream>>>(
      diff_params(d), samples_dev, n, depth_dev, T0_dev, masks_dev);
  return launched("vbh_diff_masks");
}

vbh_status vbh_diff_forward(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                            const float* depth_dev, const float* T0_dev, const float* xi_dev,
                            const uint32_t* masks_dev, float* F_dev, double* loss_dev) {
  if (!d || !xi_dev || !F_dev || (n && (!samples_dev || !depth_dev || !T0_dev || !masks_dev)))
    return vbh::fail(VBH_ERR_INVALID_ARG, "vbh_diff_forward: null argument");
  double* loss = loss_dev ? loss_dev : d->loss;
  VBH_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), d->stream));
  vbh_status st = vbh_diff_poses(d, xi_dev, nullptr);
  if (st != VBH_OK || !n) return st;
  vbh::k_diff_forward<<<diff_grid(d, n), vbh::kDiffThreads, 0, d->stream>>>(
      diff_params(d), samples_dev, n, depth_dev, T0_dev, d->poses, masks_dev, F_dev, loss);
  return launched("vbh_diff_forward");
}

vbh_status vbh_diff_backward(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                             const float* depth_dev, const float* T0_dev, const float* xi_dev,
                             const uint32_t* masks_dev, const float* F_dev, float* gdepth_dev,
                             float* gxi_dev) {
  if (!d || !xi_dev || !gdepth_dev || !gxi_dev ||
      (n && (!samples_dev || !depth_dev || !T0_dev || !masks_dev || !F_dev)))
    return vbh::fail(VBH_ERR_INVALID_ARG, "vbh_diff_backward: null argument");
  const size_t npx = (size_t)d->cfg.n_frames * d->cfg.width * d->cfg.height;
  VBH_CUDA(cudaMemsetAsync(gdepth_dev, 0, npx * sizeof(float), d->stream));
  vbh_status st = vbh_diff_poses(d, xi_dev, nullptr);
  if (st != VBH_OK) return st;
  const int nf = (int)d->cfg.n_frames;
  int parts = 0;
  if (n) {
    const unsigned int per = vbh::kDiffThreads * vbh::kDiffChunk;
    const unsigned int want = (n + per - 1) / per;
    parts = (int)(want < (unsigned)d->bwd_grid ? want : (unsigned)d->bwd_grid);
    vbh::k_diff_backward<<<parts, vbh::kDiffThreads, d->bwd_smem, d->stream>>>(
        diff_params(d), samples_dev, n, depth_dev, T0_dev, d->poses, masks_dev, F_dev,
        gdepth_dev, d->part);
  }
  vbh::k_diff_pose_grad<<<nf, 192, 0, d->stream>>>(d->poses, d->part, parts, nf, gxi_dev);
  return launched("vbh_diff_backward");
}

}  // extern "C"
