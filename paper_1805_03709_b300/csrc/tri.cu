// Marching Cubes triangulation of an MC stream (Sec. 4.3: the exploration client builds its
// mesh from the transmitted indices, with vertices at edge midpoints -- no interpolation).
//
// The triangle table is derived here from the cube cases, at first use, not stored:
//   * corner i of a cube is c_i = (000, 100, 110, 010, 001, 101, 111, 011)[i] (x fastest), bit i
//     of the index set means the corner is inside (TSDF < 0); edges 0-11 join the corner pairs
//     (0,1) (1,2) (2,3) (3,0) (4,5) (5,6) (6,7) (7,4) (0,4) (1,5) (2,6) (3,7);
//   * each face is walked counter-clockwise as seen from outside the cube; a crossing from an
//     inside corner to an outside one (exit) is joined to the crossing into the inside that
//     precedes it (entry), so an ambiguous face keeps its inside corners apart, and both cubes
//     sharing the face join its crossings alike;
//   * the directed joins exit -> entry close into loops; a loop starts at its smallest edge and
//     is cut by ear clipping at the first position whose new diagonal joins two edges on no
//     common face (a diagonal lying on a face would be shared with the neighbouring cube), each
//     triangle in the reversed loop order so that normals point to positive TSDF.
// The kernel: the CTA's warps count the triangles of their next records (one per warp and
// round, up to 4 rounds), chunk by chunk of 32 entries; one reservation per round places the
// records' output; then the warps take the CTA's chunks in turn (a record of 500 entries is
// spread over all of them) and write each chunk's triangles (9 floats each, metres) in order,
// through a per-warp stage in shared memory, one lane per vertex.
#include <cstring>
#include <mutex>
#include <vector>

#include "handle.cuh"

namespace vbh {

namespace {

// The tables in device memory; every CTA of the kernel copies them to shared memory, where the
// lanes' different cube cases are read without the serialisation of divergent constant reads.
__device__ __align__(4) unsigned char g_tri_n[256];
__device__ __align__(4) unsigned char g_tri_e[256 * 15];
// 2 x edge midpoint (0, 1 or 2 per axis), padded to whole words
__device__ __align__(4) unsigned char g_mid2[12 * 3 + 4];

constexpr int kCube[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                             {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
constexpr int kEdges[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                               {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

struct Tables {
  unsigned char n[256];
  unsigned char e[256][15];
  unsigned char mid2[12][3];
};

int find_edge(int p, int q) {
  for (int j = 0; j < 12; ++j)
    if ((kEdges[j][0] == p && kEdges[j][1] == q) || (kEdges[j][0] == q && kEdges[j][1] == p))
      return j;
  return -1;
}

bool on_one_face(int e1, int e2) {
  const int v[4] = {kEdges[e1][0], kEdges[e1][1], kEdges[e2][0], kEdges[e2][1]};
  for (int ax = 0; ax < 3; ++ax)
    if (kCube[v[0]][ax] == kCube[v[1]][ax] && kCube[v[0]][ax] == kCube[v[2]][ax] &&
        kCube[v[0]][ax] == kCube[v[3]][ax])
      return true;
  return false;
}

Tables derive_tables() {
  Tables T{};
  for (int j = 0; j < 12; ++j)
    for (int ax = 0; ax < 3; ++ax)
      T.mid2[j][ax] = (unsigned char)(kCube[kEdges[j][0]][ax] + kCube[kEdges[j][1]][ax]);
  // faces: corners with coordinate `ax` equal to `side`, in a cycle along cube edges, turned
  // counter-clockwise about the outward normal
  int face[6][4];
  int nf = 0;
  for (int ax = 0; ax < 3; ++ax)
    for (int side = 0; side <= 1; ++side) {
      int cyc[4], k = 0;
      bool taken[8] = {false};
      for (int c = 0; c < 8 && k == 0; ++c)
        if (kCube[c][ax] == side) { cyc[k++] = c; taken[c] = true; }
      while (k < 4)
        for (int c = 0; c < 8; ++c)
          if (!taken[c] && kCube[c][ax] == side && find_edge(cyc[k - 1], c) >= 0) {
            cyc[k++] = c;
            taken[c] = true;
            break;
          }
      int u[3], w[3];
      for (int i = 0; i < 3; ++i) {
        u[i] = kCube[cyc[1]][i] - kCube[cyc[0]][i];
        w[i] = kCube[cyc[2]][i] - kCube[cyc[1]][i];
      }
      const int cross_ax = u[(ax + 1) % 3] * w[(ax + 2) % 3] - u[(ax + 2) % 3] * w[(ax + 1) % 3];
      if ((side == 1 && cross_ax < 0) || (side == 0 && cross_ax > 0)) {
        const int t = cyc[1];
        cyc[1] = cyc[3];
        cyc[3] = t;
      }
      for (int i = 0; i < 4; ++i) face[nf][i] = cyc[i];
      ++nf;
    }
  for (int idx = 0; idx < 256; ++idx) {
    int join[12];
    for (int j = 0; j < 12; ++j) join[j] = -1;
    for (int f = 0; f < 6; ++f) {
      int edge_at[4], kind[4], m = 0;   // kind: 1 entry, 0 exit
      for (int i = 0; i < 4; ++i) {
        const int p = face[f][i], q = face[f][(i + 1) % 4];
        const int ip = (idx >> p) & 1, iq = (idx >> q) & 1;
        if (ip == iq) continue;
        edge_at[m] = find_edge(p, q);
        kind[m] = iq;
        ++m;
      }
      for (int i = 0; i < m; ++i)
        if (kind[i] == 0) join[edge_at[i]] = edge_at[(i + m - 1) % m];
    }
    int count = 0;
    bool done[12] = {false};
    for (int start = 0; start < 12; ++start) {
      if (join[start] < 0 || done[start]) continue;
      std::vector<int> poly;
      for (int e = start; !done[e]; e = join[e]) {
        done[e] = true;
        poly.push_back(e);
      }
      while (poly.size() > 3) {
        const size_t n = poly.size();
        size_t at = 0;
        for (size_t i = 0; i < n; ++i)
          if (!on_one_face(poly[(i + n - 1) % n], poly[(i + 1) % n])) {
            at = i;
            break;
          }
        const int a = poly[(at + n - 1) % n], b = poly[at], c = poly[(at + 1) % n];
        T.e[idx][3 * count] = (unsigned char)a;
        T.e[idx][3 * count + 1] = (unsigned char)c;
        T.e[idx][3 * count + 2] = (unsigned char)b;
        ++count;
        poly.erase(poly.begin() + (long)at);
      }
      T.e[idx][3 * count] = (unsigned char)poly[0];
      T.e[idx][3 * count + 1] = (unsigned char)poly[2];
      T.e[idx][3 * count + 2] = (unsigned char)poly[1];
      ++count;
    }
    T.n[idx] = (unsigned char)count;
  }
  return T;
}

std::mutex g_tri_mutex;
std::vector<int> g_tri_ready;   // per device

vbh_status upload_tables() {
  int dev = 0;
  VBH_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(g_tri_mutex);
  if ((int)g_tri_ready.size() <= dev) g_tri_ready.resize(dev + 1, 0);
  if (g_tri_ready[dev]) return VBH_OK;
  static const Tables T = derive_tables();
  static_assert(sizeof T.n == 256 && sizeof T.e == 256 * 15 && sizeof T.mid2 == 36, "tables");
  VBH_CUDA(cudaMemcpyToSymbol(g_tri_n, T.n, sizeof T.n));
  VBH_CUDA(cudaMemcpyToSymbol(g_tri_e, T.e, sizeof T.e));
  VBH_CUDA(cudaMemcpyToSymbol(g_mid2, T.mid2, sizeof T.mid2));
  g_tri_ready[dev] = 1;
  return VBH_OK;
}

constexpr int kTriThreads = 256;
constexpr int kTriWarps = kTriThreads / 32;
constexpr unsigned int kTriGroup = 4;   // rounds of records counted before they are written
constexpr unsigned int kTriSlots = kTriGroup * kTriWarps;   // records of a CTA per group
constexpr unsigned int kTriMaxChunks = 16;   // 32-entry chunks of a record (one per voxel)

__global__ void __launch_bounds__(kTriThreads) k_mc_triangulate(
    const int* keys3, const unsigned int* offsets, const unsigned int* counts,
    const unsigned short* local, const unsigned char* index, const unsigned int* n_blocks_dev,
    unsigned int cap_blocks, unsigned int cap_entries, float half_s, float* tris,
    unsigned int cap_tris, unsigned int* n_tris) {
  __shared__ __align__(4) unsigned char s_n[256], s_e[256 * 15], s_mid[12 * 3 + 4];
  __shared__ unsigned int s_mid4[12];   // the edge midpoints (x2) as one word per edge
  // the group's records (slot j * kTriWarps + w: round j of warp w): entries, key, triangles
  __shared__ unsigned int s_roff[kTriSlots], s_rcnt[kTriSlots], s_rtris[kTriSlots];
  __shared__ int s_rkey[kTriSlots][3];
  __shared__ unsigned char s_ccnt[kTriSlots][kTriMaxChunks];   // triangles of each chunk
  // the group's chunks: slot | chunk << 5, and the chunk's first triangle
  __shared__ unsigned int s_chunk[kTriSlots * kTriMaxChunks], s_choff[kTriSlots * kTriMaxChunks];
  __shared__ unsigned int s_nchunks;
  __shared__ unsigned int s_stage[kTriWarps][32 * 5];   // <= 5 triangles per cube
  for (unsigned int i = threadIdx.x; i < 64u; i += kTriThreads)
    reinterpret_cast<unsigned int*>(s_n)[i] = reinterpret_cast<const unsigned int*>(g_tri_n)[i];
  for (unsigned int i = threadIdx.x; i < 960u; i += kTriThreads)
    reinterpret_cast<unsigned int*>(s_e)[i] = reinterpret_cast<const unsigned int*>(g_tri_e)[i];
  for (unsigned int i = threadIdx.x; i < 10u; i += kTriThreads)
    reinterpret_cast<unsigned int*>(s_mid)[i] = reinterpret_cast<const unsigned int*>(g_mid2)[i];
  __syncthreads();
  if (threadIdx.x < 12u)
    s_mid4[threadIdx.x] = s_mid[3u * threadIdx.x] | (unsigned int)s_mid[3u * threadIdx.x + 1] << 8 |
                          (unsigned int)s_mid[3u * threadIdx.x + 2] << 16;
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int nb = min(*n_blocks_dev, cap_blocks);
  const unsigned int per_round = gridDim.x * kTriWarps;
  const unsigned int rounds = (nb + per_round - 1u) / per_round;
  for (unsigned int r0 = 0; r0 < rounds; r0 += kTriGroup) {
    const unsigned int nr = min(kTriGroup, rounds - r0);
    // 1. each warp counts the triangles of its next nr records, chunk by chunk
    for (unsigned int j = 0; j < nr; ++j) {
      const unsigned int slot = j * kTriWarps + warp;
      const unsigned int r = (r0 + j) * per_round + blockIdx.x * kTriWarps + warp;
      unsigned int off = 0, cnt = 0;
      if (r < nb) {
        off = offsets[r];
        cnt = counts[r];
        // an overflowed stream, or more entries than voxels: nothing of the record is read
        if ((unsigned long long)off + cnt > cap_entries || cnt > 32u * kTriMaxChunks) cnt = 0;
      }
      unsigned int tot = 0;
      for (unsigned int c = 0; 32u * c < cnt; ++c) {
        const unsigned int e = 32u * c + lane;
        const unsigned int k = __reduce_add_sync(0xFFFFFFFFu, e < cnt ? s_n[index[off + e]] : 0u);
        if (lane == 0) s_ccnt[slot][c] = (unsigned char)k;
        tot += k;
      }
      if (lane == 0) {
        s_roff[slot] = off;
        s_rcnt[slot] = cnt;
        s_rtris[slot] = tot;
      }
      if (lane < 3u) s_rkey[slot][lane] = r < nb ? keys3[3u * r + lane] : 0;
    }
    __syncthreads();
    // 2. warp 0: one output reservation per round, then the list of the group's chunks with
    //    each chunk's first triangle
    if (warp == 0) {
      if (lane < nr) {
        unsigned int run = 0;
        for (int w = 0; w < kTriWarps; ++w) {
          const unsigned int c = s_rtris[lane * kTriWarps + w];
          s_rtris[lane * kTriWarps + w] = run;
          run += c;
        }
        const unsigned int base = run ? atomicAdd(n_tris, run) : 0u;
        for (int w = 0; w < kTriWarps; ++w) s_rtris[lane * kTriWarps + w] += base;
      }
      __syncwarp();
      static_assert(kTriSlots <= 32, "one lane per slot");
      const unsigned int slot = lane;
      const unsigned int nch = slot < nr * kTriWarps ? (s_rcnt[slot] + 31u) / 32u : 0u;
      unsigned int at = nch;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, at, d);
        if ((int)lane >= d) at += v;
      }
      if (lane == 31u) s_nchunks = at;
      at -= nch;
      unsigned int o = nch ? s_rtris[slot] : 0u;
      for (unsigned int c = 0; c < nch; ++c) {
        s_chunk[at + c] = slot | c << 5;
        s_choff[at + c] = o;
        o += s_ccnt[slot][c];
      }
    }
    __syncthreads();
    // 3. the warps take the group's chunks in turn (records differ widely in size): each lane
    //    packs its entry's triangles (voxel index, three edges) into the warp's stage, then
    //    each lane writes whole vertices of the chunk's triangles, in order
    const unsigned int nchunks = s_nchunks;
    unsigned int* stage = s_stage[warp];
    for (unsigned int k = warp; k < nchunks; k += kTriWarps) {
      const unsigned int slot = s_chunk[k] & 31u, c = s_chunk[k] >> 5;
      const unsigned int off = s_roff[slot] + 32u * c;
      const unsigned int cnt = min(32u, s_rcnt[slot] - 32u * c);
      const int gx = 16 * s_rkey[slot][0], gy = 16 * s_rkey[slot][1], gz = 16 * s_rkey[slot][2];
      const unsigned int o = s_choff[k];
      unsigned int nt = 0, ci = 0, l = 0;
      if (lane < cnt) {
        ci = index[off + lane];
        l = local[off + lane];
        nt = s_n[ci];
      }
      unsigned int at = nt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned int v = __shfl_up_sync(0xFFFFFFFFu, at, d);
        if ((int)lane >= d) at += v;
      }
      const unsigned int tot = __shfl_sync(0xFFFFFFFFu, at, 31);
      at -= nt;
      for (unsigned int t = 0; t < nt; ++t) {
        const unsigned char* ed = &s_e[15u * ci + 3u * t];
        stage[at + t] = l | ((unsigned int)ed[0] << 9) | ((unsigned int)ed[1] << 13) |
                        ((unsigned int)ed[2] << 17);
      }
      __syncwarp();
      for (unsigned int q = lane; q < 3u * tot; q += 32u) {
        const unsigned int tr = q / 3u, v = q - 3u * tr;
        if (o + tr >= cap_tris) continue;
        const unsigned int w = stage[tr];
        const unsigned int m = s_mid4[(w >> (9u + 4u * v)) & 15u];
        // 2 x the vertex, (2 (8 key + l) + edge midpoint x 2), then x voxel_size / 2
        const int x2 = gx + 2 * (int)(w & 7u) + (int)(m & 0xFFu);
        const int y2 = gy + 2 * (int)((w >> 3) & 7u) + (int)((m >> 8) & 0xFFu);
        const int z2 = gz + 2 * (int)((w >> 6) & 7u) + (int)(m >> 16);
        float* dst = tris + 9ull * o + 3u * q;
        dst[0] = __fmul_rn((float)x2, half_s);
        dst[1] = __fmul_rn((float)y2, half_s);
        dst[2] = __fmul_rn((float)z2, half_s);
      }
      __syncwarp();
    }
    __syncthreads();   // the group's shared arrays are refilled next
  }
}

}  // namespace
}  // namespace vbh

using namespace vbh;

extern "C" {

vbh_status vbh_mc_tri_table(uint8_t* n_host, uint8_t* edges_host) {
  if (!n_host || !edges_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  static const Tables T = derive_tables();
  std::memcpy(n_host, T.n, sizeof T.n);
  std::memcpy(edges_host, T.e, sizeof T.e);
  return VBH_OK;
}

vbh_status vbh_mc_triangulate(const vbh_mc_stream* in, float voxel_size, float* tris_dev,
                              uint32_t cap_tris, uint32_t* n_tris_dev, void* cuda_stream) {
  if (!in || !n_tris_dev || (cap_tris && !tris_dev)) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (!in->n_blocks_dev || (in->cap_blocks && (!in->keys3 || !in->offsets || !in->counts)) ||
      (in->cap_entries && (!in->local || !in->index)))
    return fail(VBH_ERR_INVALID_ARG, "incomplete input stream");
  if (!(voxel_size > 0.f)) return fail(VBH_ERR_INVALID_ARG, "voxel_size must be positive");
  vbh_status st = upload_tables();
  if (st != VBH_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  VBH_CUDA(cudaMemsetAsync(n_tris_dev, 0, sizeof(uint32_t), s));
  int dev = 0, sms = 0;
  VBH_CUDA(cudaGetDevice(&dev));
  VBH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  k_mc_triangulate<<<sms * 8, kTriThreads, 0, s>>>(
      in->keys3, in->offsets, in->counts, in->local, in->index, in->n_blocks_dev, in->cap_blocks,
      in->cap_entries, 0.5f * voxel_size, tris_dev, cap_tris, n_tris_dev);
  VBH_CUDA(cudaGetLastError());
  return VBH_OK;
}

}  // extern "C"
