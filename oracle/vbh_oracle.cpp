// CPU ORACLE for the voxel-block-hashing hot path -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow and deliberately obvious: a std::unordered_map key store, FP64 projective TSDF
// values, sequential allocation / integration / erase / Marching-Cubes classification (a timing
// mode runs the allocation's rows and the fusion's and classification's independent blocks on
// OpenMP threads, with identical results; hash operations always run serially).  Only the
// tests, the smoke check and the benchmark's CPU-baseline leg load this library; the product
// path never does.  It shares no code, header, table or constant with the CUDA library.
//
// What it follows (SLAMCast, Stotko et al.):
//   * Sec. 5 "Retrieval / Insertion / Removal": a map of unique keys with guaranteed find,
//     insert (no overwrite; succeeds once the key is present) and erase.
//   * Sec. 4.1 (reconstruction client): voxel block hashing -- allocation of the blocks around
//     each depth sample and projective TSDF fusion (inherited from Niessner et al. / InfiniTAM,
//     the paper gives no formula; the standard running average is written out below).
//   * Sec. 4.2 (server): the per-voxel 8-bit Marching Cubes index, with indices 0 and 255 (the
//     set S^c of the S^c equation) written as 0, recomputed for each updated block and its seven
//     neighbours in negative direction.
//
// Readings of what the paper leaves open (each stated where it is used):
//   R-batch  A batch of hash operations runs all finds on the pre-batch state, then all inserts,
//            then all erases.  Among duplicate inserts (erases) of one key, the first in batch
//            order reports INSERTED (ERASED); the rest report EXISTS (NOT_FOUND).
//   R-canon  Every discrete decision (which pixel a voxel projects to, band membership, which
//            block a depth sample falls in, the erase distance test) is defined as a fixed
//            sequence of IEEE-754 binary32 operations, each rounded to nearest even: + - * /,
//            fmaf (one rounding), floorf and exact int->float conversion.  This file is built
//            with -ffp-contract=off so that the compiler fuses nothing on its own.
//   R-value  TSDF values and weights are carried in FP64.
//   R1 voxel g sits at world position g*s (corner convention).
//   R2 depth in metres d = fl32(raw * depth_scale); raw == 0 is invalid; pixels with
//      d > zmax are ignored when zmax > 0.
//   R3 allocation samples z_j = fmaf(j, s, fl32(d - mu)), j = 0..J, J = ceil(2 mu / s) taken in
//      double from the float inputs with a 1e-6 guard; every sample's block is allocated.
//   R4 the integration set of a frame is the set of blocks its allocation touched.
//   R5 projective SDF sdf = d(pixel) - p_z, observation f = clamp(sdf / mu, -1, 1), skipped when
//      the canonical sdf32 < -mu; running average with weight 1 per observation, capped at Wmax:
//      F <- (w F + f) / (w + 1), W <- min(w + 1, Wmax) with w = W.
//   R6 a block is erased when its centre (8k + 3.5) s is farther than R from a given point.
//   R7 a block is in view of pose T when its bounding sphere (centre c = (8k + 3.5) s, radius
//      rho = fl(7 s)) is not outside the camera frustum, tested on camera coordinates of the
//      centre p (the voxel projection chain of R5 applied to c) against the four side planes
//      fx p_x + cxh p_z >= 0, (W - cxh) p_z - fx p_x >= 0 (and likewise in y) with the margin
//      rho G, G = fl(max(fx, fy) + max(cxh, W - cxh, cyh, H - cyh)) >= every plane normal's
//      norm (so the test keeps every block that has a voxel in view), and p_z >= -rho, plus
//      p_z <= zfar + rho when a far limit zfar > 0 is given.
//   R8 (visible integration) the integration set of a frame is the touched set of R4 together
//      with every live block in view (R7, far limit zmax): blocks that are not reached by the
//      frame's truncation band are still updated where their voxels see free space (f = 1).
//   R9 (scene reset, Sec. 4.1) a frustum erase removes every live block in view (R7).
//   R10 (triangulation, Sec. 4.3: vertices at edge midpoints, no interpolation) the triangles of
//      a cube index come from a cube-case analysis: on every face, walked counter-clockwise as
//      seen from outside the cube, each crossing from an inside corner (bit set) to an outside
//      one (an exit) is joined to the crossing into the inside that precedes it (an entry), so
//      an ambiguous face keeps its inside corners apart; the directed joins exit -> entry close
//      into loops over the cube's faces (each started at its smallest edge number); a loop is
//      cut by ear clipping, always at the first position (in loop order) whose new diagonal
//      joins two edges on no common face (else at the first position), each triangle in the
//      reversed loop order so that normals point to the outside (positive TSDF).  Edge j joins
//      corners kEdge[j].
//   R-mc corner i of the cube at voxel g is g + c_i with the classic numbering
//      c = (000,100,110,010,001,101,111,011) (x fastest); bit i is set iff F(corner) < 0; a cube
//      with any corner in a missing block or with W == 0 is invalid and gets index 0.

#include <array>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <omp.h>
#include <set>
#include <unordered_map>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Keys: an int3 block coordinate.  The oracle keeps its own 64-bit packing only as a hash key
// for std::unordered_map; it is never exposed.
struct K3 {
  int32_t x, y, z;
  bool operator==(const K3& o) const { return x == o.x && y == o.y && z == o.z; }
  bool operator<(const K3& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};
struct K3Hash {
  size_t operator()(const K3& k) const {
    uint64_t h = (uint64_t)(uint32_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k.y + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k.z + 0x85157AF5ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

const int kOpFind = 0, kOpInsert = 1, kOpErase = 2;
const uint8_t kStFound = 1, kStNotFound = 2, kStInserted = 3, kStExists = 4, kStErased = 5,
              kStInvalid = 7;
const uint32_t kNone = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------------
// Sec. 5: a map of unique keys to 32-bit values.
struct OracleMap {
  std::unordered_map<K3, uint32_t, K3Hash> m;
};

// Block of 8^3 voxels, FP64 values (R-value).
struct Block {
  double F[512];
  double W[512];
};

struct Volume {
  float s, mu, wmax, ds, zmax, fx, fy, cx, cy;
  int width, height;
  std::unordered_map<K3, Block, K3Hash> blocks;
  std::set<K3> touched;   // blocks allocated/updated by the last integrated frame (R4)
  std::set<K3> removed;   // blocks erased since the last touched-set extraction
  // Passive host map of the blocks streamed out of the active model (Sec. 4.1, blocks that
  // left the active region move to CPU memory): the block's values at its last erase.
  std::unordered_map<K3, Block, K3Hash> host;
};

inline int floordiv8(int g) { return g >= 0 ? g / 8 : -((-g + 7) / 8); }
inline int mod8(int g) { return g - 8 * floordiv8(g); }

bool key_in_range(float fq) { return fq >= -1048576.0f && fq < 1048576.0f; }

// R3: number of sample steps J along the band [d - mu, d + mu].
int band_steps(float mu, float s) {
  return (int)std::ceil(2.0 * (double)mu / (double)s - 1e-6);
}

// Timing mode: 1 = the single-threaded reference; n > 1 = OpenMP over image rows (allocation)
// and over blocks (fusion, MC classification).  Blocks are independent in both steps and a set
// union does not depend on the order of its inserts, so every mode gives the same results.
int g_threads = 1;

// R-canon, allocation: collect the block of every band sample of every valid pixel of rows
// [pv0, pv1).
void allocate_rows(const Volume& v, const uint16_t* depth, const float* T, int pv0, int pv1,
                   std::set<K3>& out) {
  const float inv_bs = 1.0f / (8.0f * v.s);
  const int J = band_steps(v.mu, v.s);
  for (int pv = pv0; pv < pv1; ++pv) {
    for (int pu = 0; pu < v.width; ++pu) {
      uint16_t raw = depth[(size_t)pv * v.width + pu];
      if (raw == 0) continue;
      float d = (float)raw * v.ds;
      if (v.zmax > 0.0f && d > v.zmax) continue;
      float du = (float)pu - v.cx;
      float au = du / v.fx;
      float dv = (float)pv - v.cy;
      float av = dv / v.fy;
      float z0 = d - v.mu;
      for (int j = 0; j <= J; ++j) {
        float z = std::fma((float)j, v.s, z0);
        if (!(z > 0.0f)) continue;
        float px = au * z;
        float py = av * z;
        float X[3];
        for (int i = 0; i < 3; ++i) {
          float acc = std::fma(T[4 * i + 0], px, T[4 * i + 3]);
          acc = std::fma(T[4 * i + 1], py, acc);
          X[i] = std::fma(T[4 * i + 2], z, acc);
        }
        float q[3];
        bool ok = true;
        for (int i = 0; i < 3; ++i) {
          q[i] = std::floor(X[i] * inv_bs);
          ok = ok && key_in_range(q[i]);
        }
        if (!ok) continue;
        out.insert(K3{(int)q[0], (int)q[1], (int)q[2]});
      }
    }
  }
}

// The allocation of a whole frame: the union over all rows.
void allocate_blocks(const Volume& v, const uint16_t* depth, const float* T, std::set<K3>& out) {
  if (g_threads <= 1) {
    allocate_rows(v, depth, T, 0, v.height, out);
    return;
  }
  std::vector<std::set<K3>> part(g_threads);
#pragma omp parallel num_threads(g_threads)
  {
    const int i = omp_get_thread_num(), n = omp_get_num_threads();
    allocate_rows(v, depth, T, (int)((long)v.height * i / n), (int)((long)v.height * (i + 1) / n),
                  part[i]);
  }
  for (auto& p : part) out.insert(p.begin(), p.end());
}

// R-canon + R5 + R-value: fuse one frame into one block.
void integrate_block(const Volume& v, const K3& k, Block& b, const uint16_t* depth, const float* T) {
  const float cxh = v.cx + 0.5f;
  const float cyh = v.cy + 0.5f;
  const float fw = (float)v.width, fh = (float)v.height;
  for (int lz = 0; lz < 8; ++lz)
    for (int ly = 0; ly < 8; ++ly)
      for (int lx = 0; lx < 8; ++lx) {
        const int g[3] = {8 * k.x + lx, 8 * k.y + ly, 8 * k.z + lz};
        // decision path, binary32
        float dX[3];
        for (int i = 0; i < 3; ++i) dX[i] = std::fma((float)g[i], v.s, -T[4 * i + 3]);
        float p[3];
        for (int j = 0; j < 3; ++j) {   // p = R^T (X - t)
          float acc = T[0 * 4 + j] * dX[0];
          acc = std::fma(T[1 * 4 + j], dX[1], acc);
          p[j] = std::fma(T[2 * 4 + j], dX[2], acc);
        }
        if (!(p[2] > 0.0f)) continue;
        float r = 1.0f / p[2];
        float uf = std::floor(std::fma(v.fx * p[0], r, cxh));
        float vf = std::floor(std::fma(v.fy * p[1], r, cyh));
        if (!(uf >= 0.0f && uf < fw && vf >= 0.0f && vf < fh)) continue;
        uint16_t raw = depth[(size_t)(int)vf * v.width + (int)uf];
        if (raw == 0) continue;
        float d = (float)raw * v.ds;
        if (v.zmax > 0.0f && d > v.zmax) continue;
        float sdf32 = d - p[2];
        if (sdf32 < -v.mu) continue;
        // value path, binary64
        double pz = 0.0;
        for (int i = 0; i < 3; ++i)
          pz += (double)T[4 * i + 2] * ((double)g[i] * (double)v.s - (double)T[4 * i + 3]);
        double sdf = (double)d - pz;
        double f = sdf / (double)v.mu;
        f = std::min(1.0, std::max(-1.0, f));
        const int idx = lx + 8 * ly + 64 * lz;
        double w = b.W[idx];
        b.F[idx] = (w * b.F[idx] + f) / (w + 1.0);
        b.W[idx] = std::min(w + 1.0, (double)v.wmax);
      }
}

// R6: canonical squared distance of the block centre from a point.
bool erase_test(const Volume& v, const K3& k, const float* c, float R) {
  const int kk[3] = {k.x, k.y, k.z};
  float dc[3];
  for (int i = 0; i < 3; ++i) {
    float centre = ((float)(8 * kk[i]) + 3.5f) * v.s;
    dc[i] = centre - c[i];
  }
  float d2 = dc[0] * dc[0];
  d2 = std::fma(dc[1], dc[1], d2);
  d2 = std::fma(dc[2], dc[2], d2);
  return d2 > R * R;
}

// R7: the bounding sphere of block k against the frustum of pose T (binary32 decisions).
bool in_view(const Volume& v, const K3& k, const float* T, float zfar) {
  const int kk[3] = {k.x, k.y, k.z};
  float dX[3];
  for (int i = 0; i < 3; ++i) {
    const float c = ((float)(8 * kk[i]) + 3.5f) * v.s;
    dX[i] = c - T[4 * i + 3];
  }
  float p[3];
  for (int j = 0; j < 3; ++j) {
    float acc = T[0 * 4 + j] * dX[0];
    acc = std::fma(T[1 * 4 + j], dX[1], acc);
    p[j] = std::fma(T[2 * 4 + j], dX[2], acc);
  }
  const float rho = 7.0f * v.s;
  const float cxh = v.cx + 0.5f, cyh = v.cy + 0.5f;
  const float rx = (float)v.width - cxh, ry = (float)v.height - cyh;
  const float G = std::max(v.fx, v.fy) + std::max(std::max(cxh, rx), std::max(cyh, ry));
  const float m = -(rho * G);
  const float a = v.fx * p[0], b = v.fy * p[1];
  if (!(p[2] >= -rho)) return false;
  if (zfar > 0.0f && !(p[2] <= zfar + rho)) return false;
  return std::fma(cxh, p[2], a) >= m && std::fma(rx, p[2], -a) >= m &&
         std::fma(cyh, p[2], b) >= m && std::fma(ry, p[2], -b) >= m;
}

// R-mc corner offsets, classic numbering.
const int kCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                           {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

// R10: the triangle table, derived from the cube cases (no stored table).
const int kEdge[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                          {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

int edge_of(int a, int b) {
  for (int j = 0; j < 12; ++j)
    if ((kEdge[j][0] == a && kEdge[j][1] == b) || (kEdge[j][0] == b && kEdge[j][1] == a)) return j;
  return -1;
}

// two cube edges lie on a common face when their four corners agree in one coordinate
bool share_face(int e1, int e2) {
  const int cs[4] = {kEdge[e1][0], kEdge[e1][1], kEdge[e2][0], kEdge[e2][1]};
  for (int axis = 0; axis < 3; ++axis) {
    bool same = true;
    for (int i = 1; i < 4; ++i) same = same && kCorner[cs[i]][axis] == kCorner[cs[0]][axis];
    if (same) return true;
  }
  return false;
}

struct TriTable {
  std::vector<std::array<int, 3>> tris[256];
  TriTable() {
    // the six faces as corner cycles, counter-clockwise seen from outside (checked by the
    // cross product against the outward normal)
    std::vector<std::array<int, 4>> faces;
    for (int axis = 0; axis < 3; ++axis)
      for (int side = 0; side < 2; ++side) {
        std::vector<int> cs;
        for (int c = 0; c < 8; ++c)
          if (kCorner[c][axis] == side) cs.push_back(c);
        // order the 4 corners around the face: start at cs[0], then walk along cube edges
        std::array<int, 4> cyc{cs[0], -1, -1, -1};
        std::vector<bool> used(8, false);
        used[cs[0]] = true;
        for (int k = 1; k < 4; ++k)
          for (int c : cs)
            if (!used[c] && edge_of(cyc[k - 1], c) >= 0) {
              cyc[k] = c;
              used[c] = true;
              break;
            }
        double a[3], b[3], n[3];
        for (int i = 0; i < 3; ++i) {
          a[i] = kCorner[cyc[1]][i] - kCorner[cyc[0]][i];
          b[i] = kCorner[cyc[2]][i] - kCorner[cyc[1]][i];
        }
        n[0] = a[1] * b[2] - a[2] * b[1];
        n[1] = a[2] * b[0] - a[0] * b[2];
        n[2] = a[0] * b[1] - a[1] * b[0];
        const double outward = side ? 1.0 : -1.0;
        if (n[axis] * outward < 0) std::swap(cyc[1], cyc[3]);
        faces.push_back(cyc);
      }
    for (int c = 0; c < 256; ++c) {
      int next[12];
      for (int j = 0; j < 12; ++j) next[j] = -1;
      for (const auto& f : faces) {
        // crossing events along the cycle: +1 entry, -1 exit, at the edge of (f[k], f[k+1])
        int ev_edge[4], ev_type[4], m = 0;
        for (int k = 0; k < 4; ++k) {
          const bool in0 = (c >> f[k]) & 1, in1 = (c >> f[(k + 1) % 4]) & 1;
          if (in0 != in1) {
            ev_edge[m] = edge_of(f[k], f[(k + 1) % 4]);
            ev_type[m] = in1 ? +1 : -1;
            ++m;
          }
        }
        for (int i = 0; i < m; ++i)
          if (ev_type[i] == -1) {   // the entry before this exit (events alternate)
            const int e = ev_edge[(i + m - 1) % m];
            next[ev_edge[i]] = e;
          }
      }
      bool seen[12] = {false};
      for (int s0 = 0; s0 < 12; ++s0) {
        if (next[s0] < 0 || seen[s0]) continue;
        std::vector<int> loop;
        for (int e = s0; !seen[e]; e = next[e]) {
          seen[e] = true;
          loop.push_back(e);
        }
        // ear clipping: the first ear (in loop order) whose new diagonal joins two edges on no
        // common face (a diagonal on a face would be shared with the neighbouring cube)
        while (loop.size() > 3) {
          size_t pick = 0;
          bool found = false;
          for (size_t i = 0; i < loop.size() && !found; ++i) {
            const int a = loop[(i + loop.size() - 1) % loop.size()], b = loop[(i + 1) % loop.size()];
            if (!share_face(a, b)) {
              pick = i;
              found = true;
            }
          }
          const size_t n = loop.size();
          const int a = loop[(pick + n - 1) % n], m = loop[pick], b = loop[(pick + 1) % n];
          tris[c].push_back({a, b, m});   // reversed loop order: normals to the outside
          loop.erase(loop.begin() + (long)pick);
        }
        tris[c].push_back({loop[0], loop[2], loop[1]});
      }
    }
  }
};

const TriTable& tri_table() {
  static TriTable t;
  return t;
}

// Sec. 4.2: the MC index of the cube at voxel g, with S^c (0 and 255) written as 0.
// `margin` receives min |F| over the 8 corners (+inf for an invalid cube).
uint8_t mc_index(const Volume& v, const int g[3], double* margin) {
  int idx = 0;
  double mn = INFINITY;
  for (int i = 0; i < 8; ++i) {
    int gc[3] = {g[0] + kCorner[i][0], g[1] + kCorner[i][1], g[2] + kCorner[i][2]};
    K3 kc{floordiv8(gc[0]), floordiv8(gc[1]), floordiv8(gc[2])};
    auto it = v.blocks.find(kc);
    if (it == v.blocks.end()) { *margin = INFINITY; return 0; }
    int li = mod8(gc[0]) + 8 * mod8(gc[1]) + 64 * mod8(gc[2]);
    if (it->second.W[li] == 0.0) { *margin = INFINITY; return 0; }
    double F = it->second.F[li];
    mn = std::min(mn, std::fabs(F));
    if (F < 0.0) idx |= 1 << i;
  }
  *margin = mn;
  if (idx == 255) idx = 0;   // S^c
  return (uint8_t)idx;
}

void fill_keys(const std::vector<K3>& ks, int32_t* out, uint32_t cap) {
  for (size_t i = 0; i < ks.size() && i < cap; ++i) {
    out[3 * i + 0] = ks[i].x;
    out[3 * i + 1] = ks[i].y;
    out[3 * i + 2] = ks[i].z;
  }
}

}  // namespace

extern "C" {

// ----------------------------------------------------------------------------------- hash map
void* orc_map_create() { return new OracleMap(); }
void orc_map_destroy(void* h) { delete (OracleMap*)h; }
uint32_t orc_map_size(void* h) { return (uint32_t)((OracleMap*)h)->m.size(); }

// Sec. 5 + R-batch.  vals may be null (then inserted values are 0).  results[i] is the value
// found / kept / erased, or 0xFFFFFFFF.  Keys outside [-2^20, 2^20) and unknown ops are
// reported INVALID and change nothing.
void orc_map_batch(void* h, uint32_t n, const uint8_t* ops, const int32_t* keys3,
                   const uint32_t* vals, uint32_t* results, uint8_t* status) {
  auto& m = ((OracleMap*)h)->m;
  auto valid = [&](uint32_t i) {
    for (int a = 0; a < 3; ++a)
      if (keys3[3 * i + a] < -1048576 || keys3[3 * i + a] >= 1048576) return false;
    return ops[i] <= 2;
  };
  for (uint32_t i = 0; i < n; ++i) {   // phase 1: finds against the pre-batch state
    if (!valid(i)) { status[i] = kStInvalid; results[i] = kNone; continue; }
    if (ops[i] != kOpFind) continue;
    auto it = m.find(K3{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]});
    if (it == m.end()) { status[i] = kStNotFound; results[i] = kNone; }
    else { status[i] = kStFound; results[i] = it->second; }
  }
  for (uint32_t i = 0; i < n; ++i) {   // phase 2: inserts, batch order
    if (!valid(i) || ops[i] != kOpInsert) continue;
    K3 k{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]};
    auto it = m.find(k);
    if (it != m.end()) { status[i] = kStExists; continue; }
    m[k] = vals ? vals[i] : 0u;
    status[i] = kStInserted;
  }
  for (uint32_t i = 0; i < n; ++i) {   // inserts report the value the key ended up with
    if (!valid(i) || ops[i] != kOpInsert) continue;
    results[i] = m[K3{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]}];
  }
  for (uint32_t i = 0; i < n; ++i) {   // phase 3: erases, batch order
    if (!valid(i) || ops[i] != kOpErase) continue;
    K3 k{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]};
    auto it = m.find(k);
    if (it == m.end()) { status[i] = kStNotFound; results[i] = kNone; continue; }
    results[i] = it->second;
    status[i] = kStErased;
    m.erase(it);
  }
}

// Dump in ascending key order.
uint32_t orc_map_dump(void* h, int32_t* keys3, uint32_t* vals, uint32_t cap) {
  auto& m = ((OracleMap*)h)->m;
  std::vector<std::pair<K3, uint32_t>> all(m.begin(), m.end());
  std::sort(all.begin(), all.end(), [](auto& a, auto& b) { return a.first < b.first; });
  for (size_t i = 0; i < all.size() && i < cap; ++i) {
    keys3[3 * i] = all[i].first.x;
    keys3[3 * i + 1] = all[i].first.y;
    keys3[3 * i + 2] = all[i].first.z;
    vals[i] = all[i].second;
  }
  return (uint32_t)all.size();
}

// -------------------------------------------------------------------------------------- volume
// params: s, mu, wmax, depth_scale, zmax, fx, fy, cx, cy
void* orc_vol_create(const float* params, int width, int height) {
  Volume* v = new Volume();
  v->s = params[0]; v->mu = params[1]; v->wmax = params[2]; v->ds = params[3];
  v->zmax = params[4]; v->fx = params[5]; v->fy = params[6]; v->cx = params[7];
  v->cy = params[8]; v->width = width; v->height = height;
  return v;
}
void orc_vol_destroy(void* h) { delete (Volume*)h; }
uint32_t orc_vol_size(void* h) { return (uint32_t)((Volume*)h)->blocks.size(); }

// Allocation only (R3): the set of blocks one frame touches, sorted; nothing is modified.
uint32_t orc_alloc_keys(void* h, const uint16_t* depth, const float* T, int32_t* out, uint32_t cap) {
  std::set<K3> s;
  allocate_blocks(*(Volume*)h, depth, T, s);
  std::vector<K3> ks(s.begin(), s.end());
  fill_keys(ks, out, cap);
  return (uint32_t)ks.size();
}

// One frame: allocation (R3, new blocks start at F = 0, W = 0) then fusion of the touched set
// (R4, R5), or with `visible` of the touched set and every live block in view (R8).  Returns
// the number of blocks fused.
uint32_t orc_vol_integrate_mode(void* h, const uint16_t* depth, const float* T, int visible) {
  Volume& v = *(Volume*)h;
  std::set<K3> s;
  allocate_blocks(v, depth, T, s);
  for (const K3& k : s) {
    auto it = v.blocks.find(k);
    if (it == v.blocks.end()) {
      Block& b = v.blocks[k];
      std::fill(b.F, b.F + 512, 0.0);
      std::fill(b.W, b.W + 512, 0.0);
    }
  }
  if (visible)
    for (auto& kv : v.blocks)
      if (in_view(v, kv.first, T, v.zmax)) s.insert(kv.first);
  std::vector<std::pair<K3, Block*>> work;
  for (const K3& k : s) work.emplace_back(k, &v.blocks[k]);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 64) if (g_threads > 1)
  for (long i = 0; i < (long)work.size(); ++i)
    integrate_block(v, work[i].first, *work[i].second, depth, T);
  v.touched = s;
  return (uint32_t)s.size();
}

uint32_t orc_vol_integrate(void* h, const uint16_t* depth, const float* T) {
  return orc_vol_integrate_mode(h, depth, T, 0);
}

// R7 for a list of keys (flags out[i] = 1 when in view).
void orc_in_view(void* h, const int32_t* keys3, uint32_t n, const float* T, float zfar,
                 uint8_t* out) {
  const Volume& v = *(const Volume*)h;
  for (uint32_t i = 0; i < n; ++i)
    out[i] = in_view(v, K3{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]}, T, zfar) ? 1 : 0;
}

// R9: erase every live block in view of T (far limit zfar > 0, or none); erased keys sorted.
uint32_t orc_vol_erase_frustum(void* h, const float* T, float zfar, int32_t* out, uint32_t cap) {
  Volume& v = *(Volume*)h;
  std::vector<K3> gone;
  for (auto& kv : v.blocks)
    if (in_view(v, kv.first, T, zfar)) gone.push_back(kv.first);
  std::sort(gone.begin(), gone.end());
  for (const K3& k : gone) {
    v.host[k] = v.blocks[k];
    v.blocks.erase(k);
    v.removed.insert(k);
  }
  if (out) fill_keys(gone, out, cap);
  return (uint32_t)gone.size();
}

uint32_t orc_vol_touched(void* h, int32_t* out, uint32_t cap) {
  Volume& v = *(Volume*)h;
  std::vector<K3> ks(v.touched.begin(), v.touched.end());
  fill_keys(ks, out, cap);
  return (uint32_t)ks.size();
}

// R6: erase every block whose centre is farther than R from `centre`; erased keys sorted.
uint32_t orc_vol_erase_radius(void* h, const float* centre, float R, int32_t* out, uint32_t cap) {
  Volume& v = *(Volume*)h;
  std::vector<K3> gone;
  for (auto& kv : v.blocks)
    if (erase_test(v, kv.first, centre, R)) gone.push_back(kv.first);
  std::sort(gone.begin(), gone.end());
  for (const K3& k : gone) {
    v.host[k] = v.blocks[k];   // stream-out: the erased block's values go to the host map
    v.blocks.erase(k);
    v.removed.insert(k);
  }
  if (out) fill_keys(gone, out, cap);
  return (uint32_t)gone.size();
}

// Erase an explicit key list (absent keys are ignored); returns the number erased.
uint32_t orc_vol_erase_keys(void* h, const int32_t* keys3, uint32_t n) {
  Volume& v = *(Volume*)h;
  uint32_t c = 0;
  for (uint32_t i = 0; i < n; ++i) {
    K3 k{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]};
    auto it = v.blocks.find(k);
    if (it != v.blocks.end()) {
      v.host[k] = it->second;   // stream-out
      v.blocks.erase(it);
      v.removed.insert(k);
      ++c;
    }
  }
  return c;
}

// R10: triangles of cube index c as edge triples (out: up to cap triangles); returns count.
uint32_t orc_tri_case(int c, int32_t* edges, uint32_t cap) {
  const auto& t = tri_table().tris[c & 255];
  for (size_t i = 0; i < t.size() && i < cap; ++i)
    for (int j = 0; j < 3; ++j) edges[3 * i + j] = t[i][j];
  return (uint32_t)t.size();
}

// R10 on the model: every triangle of the cubes at the voxels of the given blocks (their MC
// indices by Sec. 4.2), vertices at edge midpoints in metres, 9 doubles per triangle, in block
// order then voxel order lx + 8 ly + 64 lz then table order; returns the count.
uint32_t orc_vol_triangles(void* h, const int32_t* keys3, uint32_t n, double* out, uint32_t cap) {
  const Volume& v = *(const Volume*)h;
  uint32_t m = 0;
  for (uint32_t b = 0; b < n; ++b)
    for (int l = 0; l < 512; ++l) {
      const int g[3] = {8 * keys3[3 * b] + (l & 7), 8 * keys3[3 * b + 1] + ((l >> 3) & 7),
                        8 * keys3[3 * b + 2] + (l >> 6)};
      double margin;
      const int c = mc_index(v, g, &margin);
      for (const auto& tri : tri_table().tris[c]) {
        if (m < cap && out)
          for (int k = 0; k < 3; ++k) {
            const int* e = kEdge[tri[k]];
            for (int i = 0; i < 3; ++i)
              out[9 * m + 3 * k + i] =
                  (g[i] + 0.5 * (kCorner[e[0]][i] + kCorner[e[1]][i])) * (double)v.s;
          }
        ++m;
      }
    }
  return m;
}

// The host map of streamed-out blocks, keys sorted (like orc_vol_dump).
uint32_t orc_vol_host_dump(void* h, int32_t* keys3, double* F, double* W, uint32_t cap) {
  Volume& v = *(Volume*)h;
  std::vector<K3> ks;
  for (auto& kv : v.host) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  for (size_t i = 0; i < ks.size() && i < cap; ++i) {
    keys3[3 * i] = ks[i].x; keys3[3 * i + 1] = ks[i].y; keys3[3 * i + 2] = ks[i].z;
    const Block& b = v.host[ks[i]];
    if (F) std::memcpy(F + 512 * i, b.F, sizeof b.F);
    if (W) std::memcpy(W + 512 * i, b.W, sizeof b.W);
  }
  return (uint32_t)ks.size();
}

// Stream-in: every listed key that is in the host map and not live moves back into the model
// with its stored values (a live block is newer and stays; its host copy stays too).
uint32_t orc_vol_stream_in(void* h, const int32_t* keys3, uint32_t n) {
  Volume& v = *(Volume*)h;
  uint32_t c = 0;
  for (uint32_t i = 0; i < n; ++i) {
    K3 k{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]};
    auto it = v.host.find(k);
    if (it == v.host.end() || v.blocks.count(k)) continue;
    v.blocks[k] = it->second;
    v.host.erase(it);
    ++c;
  }
  return c;
}

// Dump in ascending key order; F and W are 512 doubles per block (x fastest).
uint32_t orc_vol_dump(void* h, int32_t* keys3, double* F, double* W, uint32_t cap) {
  Volume& v = *(Volume*)h;
  std::vector<K3> ks;
  for (auto& kv : v.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  for (size_t i = 0; i < ks.size() && i < cap; ++i) {
    keys3[3 * i] = ks[i].x; keys3[3 * i + 1] = ks[i].y; keys3[3 * i + 2] = ks[i].z;
    const Block& b = v.blocks[ks[i]];
    if (F) std::memcpy(F + 512 * i, b.F, sizeof b.F);
    if (W) std::memcpy(W + 512 * i, b.W, sizeof b.W);
  }
  return (uint32_t)ks.size();
}

// Replace / add blocks (test upload).
void orc_vol_load(void* h, const int32_t* keys3, const double* F, const double* W, uint32_t n) {
  Volume& v = *(Volume*)h;
  for (uint32_t i = 0; i < n; ++i) {
    Block& b = v.blocks[K3{keys3[3 * i], keys3[3 * i + 1], keys3[3 * i + 2]}];
    std::memcpy(b.F, F + 512 * i, sizeof b.F);
    std::memcpy(b.W, W + 512 * i, sizeof b.W);
  }
}

// The MC block set of Sec. 4.2.  mode 0: every block the last frame touched together with its
// seven neighbours in negative direction (k - o, o in {0,1}^3), live ones only; the erased
// blocks since the last mode-0 call are returned separately as removals (only those not live
// again).  mode 1: every live block.  Returns |M|; keys sorted; clears the removal list in
// mode 0.
uint32_t orc_vol_mc_set(void* h, int mode, int32_t* keys3, uint32_t cap, int32_t* removed3,
                        uint32_t rcap, uint32_t* n_removed) {
  Volume& v = *(Volume*)h;
  std::set<K3> M;
  std::vector<K3> rem;
  if (mode == 0) {
    for (const K3& k : v.touched)
      for (int o = 0; o < 8; ++o) {
        K3 n{k.x - (o & 1), k.y - ((o >> 1) & 1), k.z - ((o >> 2) & 1)};
        if (v.blocks.count(n)) M.insert(n);
      }
    for (const K3& k : v.removed)
      if (!v.blocks.count(k)) {
        rem.push_back(k);
        for (int o = 1; o < 8; ++o) {
          K3 n{k.x - (o & 1), k.y - ((o >> 1) & 1), k.z - ((o >> 2) & 1)};
          if (v.blocks.count(n)) M.insert(n);
        }
      }
    v.removed.clear();
  } else {
    for (auto& kv : v.blocks) M.insert(kv.first);
  }
  std::vector<K3> ks(M.begin(), M.end());
  fill_keys(ks, keys3, cap);
  if (removed3) fill_keys(rem, removed3, rcap);
  if (n_removed) *n_removed = (uint32_t)rem.size();
  return (uint32_t)ks.size();
}

// Dense MC indices (512 per block, x fastest) and the per-cube margin min|F| for given blocks.
void orc_vol_mc_dense(void* h, const int32_t* keys3, uint32_t n, uint8_t* idx, float* margin) {
  Volume& v = *(Volume*)h;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 64) if (g_threads > 1)
  for (long b = 0; b < (long)n; ++b)
    for (int lz = 0; lz < 8; ++lz)
      for (int ly = 0; ly < 8; ++ly)
        for (int lx = 0; lx < 8; ++lx) {
          int g[3] = {8 * keys3[3 * b] + lx, 8 * keys3[3 * b + 1] + ly, 8 * keys3[3 * b + 2] + lz};
          double m;
          uint8_t c = mc_index(v, g, &m);
          size_t o = (size_t)b * 512 + lx + 8 * ly + 64 * lz;
          idx[o] = c;
          if (margin) margin[o] = (float)m;
        }
}

// The version of the oracle library (for the tests' build check).
int orc_abi_version() { return 1; }

// Timing mode (see g_threads): n <= 1 the single-threaded reference, else n OpenMP threads.
void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads() { return g_threads; }

}  // extern "C"

// =============================================================================================
// Differentiable window fusion (the backward-pass extension of the fusion step; not in the
// paper).  Readings:
//   R-diff-1 a window of n_f frames of float32 metric depth (0 = invalid) is fused at a fixed
//            set of sample voxels g (world position g s); the value of a sample is the plain
//            mean F = sum_f m_f f_f / sum_f m_f over the frames where it is valid (the weight cap
//            never binds: n_f <= Wmax), with f_f = clamp(sdf_f / mu, -1, 1) and
//            sdf_f = D_f(u, v) - p_z, D_f bilinear in the depth image; L = sum_samples F^2.
//   R-diff-2 poses are absolute se(3) vectors xi = (rho, omega): R = exp([omega]x) (Rodrigues),
//            t = V(omega) rho with V = I + B [omega]x + C [omega]x^2.
//   R-diff-3 the validity m_f, the bilinear cell (iu, iv) and the side of the truncation clamp of
//            every sample and frame are fixed at nominal float32 poses T0 with canonical binary32
//            arithmetic: p = R0^T (g s - t0) (fma chain as in fusion),
//            u = fma(fl(fx p_x), fl(1/p_z), cx), iu = floor(u) (same for v); valid iff p_z > 0,
//            the 2 x 2 cell is inside the image, its four depths are > 0 and span at most mu
//            (max - min <= mu: no interpolation across a depth discontinuity) and the canonical
//            bilinear sdf0 at T0 is >= -mu; the term is live (f = sdf / mu) iff sdf0 < mu, else
//            it is saturated (f = 1).  At other poses the same cell is interpolated (linearly
//            extended) and the same side is kept, which makes L smooth in (xi, depth).
namespace {

struct Pose64 {
  double R[9], t[3];
  double dR[6][9];   // dR / dxi_k (zero for the rho components)
  double dt[6][3];   // dt / dxi_k
};

void skew(const double w[3], double S[9]) {
  S[0] = 0; S[1] = -w[2]; S[2] = w[1];
  S[3] = w[2]; S[4] = 0; S[5] = -w[0];
  S[6] = -w[1]; S[7] = w[0]; S[8] = 0;
}
void matmul3(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

// Coefficients A = sin t / t, B = (1 - cos t) / t^2, C = (t - sin t) / t^3 of the exponential map
// and their derivatives divided by t (A'/t, B'/t, C'/t), with Taylor series for small t.
void exp_coeffs(double th, double* A, double* B, double* C, double* Ap, double* Bp, double* Cp) {
  const double t2 = th * th;
  if (th < 1e-3) {
    *A = 1 - t2 / 6 + t2 * t2 / 120;
    *B = 0.5 - t2 / 24 + t2 * t2 / 720;
    *C = 1.0 / 6 - t2 / 120 + t2 * t2 / 5040;
    *Ap = -1.0 / 3 + t2 / 30 - t2 * t2 / 840;
    *Bp = -1.0 / 12 + t2 / 180 - t2 * t2 / 6720;
    *Cp = -1.0 / 60 + t2 / 1260 - t2 * t2 / 60480;
    return;
  }
  const double s = std::sin(th), c = std::cos(th);
  *A = s / th;
  *B = (1 - c) / t2;
  *C = (th - s) / (t2 * th);
  *Ap = (th * c - s) / (t2 * th);
  *Bp = (th * s - 2 * (1 - c)) / (t2 * t2);
  *Cp = (1 - c) / (t2 * t2) - 3 * (th - s) / (t2 * t2 * th);
}

void se3_exp(const double xi[6], Pose64& P) {
  const double* rho = xi;
  const double* w = xi + 3;
  const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double A, B, C, Ap, Bp, Cp;
  exp_coeffs(th, &A, &B, &C, &Ap, &Bp, &Cp);
  double W[9], W2[9];
  skew(w, W);
  matmul3(W, W, W2);
  double V[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    P.R[i] = I + A * W[i] + B * W2[i];
    V[i] = I + B * W[i] + C * W2[i];
  }
  for (int i = 0; i < 3; ++i) P.t[i] = V[3 * i] * rho[0] + V[3 * i + 1] * rho[1] + V[3 * i + 2] * rho[2];
  for (int k = 0; k < 3; ++k) {   // rho components
    for (int i = 0; i < 9; ++i) P.dR[k][i] = 0;
    for (int i = 0; i < 3; ++i) P.dt[k][i] = V[3 * i + k];
  }
  for (int k = 0; k < 3; ++k) {   // omega components
    double e[3] = {0, 0, 0};
    e[k] = 1;
    double E[9], EW[9], WE[9];
    skew(e, E);
    matmul3(E, W, EW);
    matmul3(W, E, WE);
    double dV[9];
    for (int i = 0; i < 9; ++i) {
      P.dR[3 + k][i] = Ap * w[k] * W[i] + A * E[i] + Bp * w[k] * W2[i] + B * (EW[i] + WE[i]);
      dV[i] = Bp * w[k] * W[i] + B * E[i] + Cp * w[k] * W2[i] + C * (EW[i] + WE[i]);
    }
    for (int i = 0; i < 3; ++i)
      P.dt[3 + k][i] = dV[3 * i] * rho[0] + dV[3 * i + 1] * rho[1] + dV[3 * i + 2] * rho[2];
  }
}

struct DiffCfg {
  float s, mu, fx, fy, cx, cy;
  int W, H, nf;
};

// R-diff-3: canonical binary32 cell and validity at the nominal pose.
bool diff_cell(const DiffCfg& c, const int* g, const float* T0, const float* D, int* iu, int* iv,
               bool* live) {
  float dX[3];
  for (int i = 0; i < 3; ++i) dX[i] = std::fma((float)g[i], c.s, -T0[4 * i + 3]);
  float p[3];
  for (int j = 0; j < 3; ++j) {
    float acc = T0[j] * dX[0];
    acc = std::fma(T0[4 + j], dX[1], acc);
    p[j] = std::fma(T0[8 + j], dX[2], acc);
  }
  if (!(p[2] > 0.0f)) return false;
  const float r = 1.0f / p[2];
  const float u = std::fma(c.fx * p[0], r, c.cx);
  const float v = std::fma(c.fy * p[1], r, c.cy);
  const float uf = std::floor(u), vf = std::floor(v);
  if (!(uf >= 0.0f && uf <= (float)(c.W - 2) && vf >= 0.0f && vf <= (float)(c.H - 2))) return false;
  const int a = (int)uf, b = (int)vf;
  const float d00 = D[b * c.W + a], d10 = D[b * c.W + a + 1];
  const float d01 = D[(b + 1) * c.W + a], d11 = D[(b + 1) * c.W + a + 1];
  if (!(d00 > 0.0f && d10 > 0.0f && d01 > 0.0f && d11 > 0.0f)) return false;
  const float dmax = std::max(std::max(d00, d10), std::max(d01, d11));
  const float dmin = std::min(std::min(d00, d10), std::min(d01, d11));
  if (dmax - dmin > c.mu) return false;
  const float fa = u - uf, fb = v - vf;
  const float wa = 1.0f - fa, wb = 1.0f - fb;
  const float w00 = wa * wb, w10 = fa * wb, w01 = wa * fb, w11 = fa * fb;
  float Dv = w00 * d00;
  Dv = std::fma(w10, d10, Dv);
  Dv = std::fma(w01, d01, Dv);
  Dv = std::fma(w11, d11, Dv);
  const float sdf = Dv - p[2];
  if (sdf < -c.mu) return false;
  *iu = a;
  *iv = b;
  *live = sdf < c.mu;
  return true;
}

// One sample and frame at pose P (FP64): f, and (if grad) the derivatives of f wrt the four
// cell depths, and wrt p; y = X - t.
struct Term {
  double f, dfdD[4], dfdp[3], y[3];
  int idx[4];
  bool live;   // |sdf / mu| < 1 (inside the clamp)
};

Term diff_term(const DiffCfg& c, const int* g, const Pose64& P, const float* D, int iu, int iv,
               bool live) {
  Term T;
  double p[3];
  for (int i = 0; i < 3; ++i) T.y[i] = (double)g[i] * (double)c.s - P.t[i];
  for (int j = 0; j < 3; ++j) p[j] = P.R[j] * T.y[0] + P.R[3 + j] * T.y[1] + P.R[6 + j] * T.y[2];
  const double u = (double)c.fx * p[0] / p[2] + (double)c.cx;
  const double v = (double)c.fy * p[1] / p[2] + (double)c.cy;
  const double a = u - iu, b = v - iv;
  T.idx[0] = iv * c.W + iu;
  T.idx[1] = iv * c.W + iu + 1;
  T.idx[2] = (iv + 1) * c.W + iu;
  T.idx[3] = (iv + 1) * c.W + iu + 1;
  const double d00 = D[T.idx[0]], d10 = D[T.idx[1]], d01 = D[T.idx[2]], d11 = D[T.idx[3]];
  const double w[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
  const double Dv = w[0] * d00 + w[1] * d10 + w[2] * d01 + w[3] * d11;
  const double sdf = Dv - p[2];
  const double q = sdf / (double)c.mu;
  T.live = live;
  T.f = live ? q : 1.0;
  const double k = T.live ? 1.0 / (double)c.mu : 0.0;
  for (int i = 0; i < 4; ++i) T.dfdD[i] = k * w[i];
  const double dDdu = (1 - b) * (d10 - d00) + b * (d11 - d01);
  const double dDdv = (1 - a) * (d01 - d00) + a * (d11 - d10);
  const double iz = 1.0 / p[2];
  T.dfdp[0] = k * dDdu * c.fx * iz;
  T.dfdp[1] = k * dDdv * c.fy * iz;
  T.dfdp[2] = k * (-dDdu * c.fx * p[0] * iz * iz - dDdv * c.fy * p[1] * iz * iz - 1.0);
  return T;
}

DiffCfg diff_cfg(const float* params, int W, int H, int nf) {
  DiffCfg c;
  c.s = params[0]; c.mu = params[1]; c.fx = params[2]; c.fy = params[3]; c.cx = params[4];
  c.cy = params[5]; c.W = W; c.H = H; c.nf = nf;
  return c;
}

}  // namespace

extern "C" {

// Exponential map with derivatives (for tests).  R[9], t[3], dR[6*9], dt[6*3] (row-major).
void orc_se3_exp(const double* xi, double* R, double* t, double* dR, double* dt) {
  Pose64 P;
  se3_exp(xi, P);
  std::memcpy(R, P.R, sizeof P.R);
  std::memcpy(t, P.t, sizeof P.t);
  if (dR) std::memcpy(dR, P.dR, sizeof P.dR);
  if (dt) std::memcpy(dt, P.dt, sizeof P.dt);
}

// params: s, mu, fx, fy, cx, cy.  depth: nf * H * W float32; T0: nf * 12 float32;
// masks: n * ceil(nf / 32) uint32 (bit f of sample i: frame f valid).
void orc_diff_masks(const float* params, int W, int H, int nf, const int32_t* samples, uint32_t n,
                    const float* depth, const float* T0, uint32_t* masks) {
  const DiffCfg c = diff_cfg(params, W, H, nf);
  const int words = (nf + 31) / 32;
  for (uint32_t i = 0; i < n; ++i) {
    for (int w = 0; w < words; ++w) masks[(size_t)i * words + w] = 0;
    for (int f = 0; f < nf; ++f) {
      int iu, iv;
      bool live;
      if (diff_cell(c, samples + 3 * i, T0 + 12 * f, depth + (size_t)f * W * H, &iu, &iv, &live))
        masks[(size_t)i * words + f / 32] |= 1u << (f % 32);
    }
  }
}

// Forward (FP64): F per sample (may be null); returns L.  xi: nf * 6 doubles.
double orc_diff_forward(const float* params, int W, int H, int nf, const int32_t* samples,
                        uint32_t n, const float* depth, const float* T0, const double* xi,
                        const uint32_t* masks, double* F) {
  const DiffCfg c = diff_cfg(params, W, H, nf);
  const int words = (nf + 31) / 32;
  std::vector<Pose64> P(nf);
  for (int f = 0; f < nf; ++f) se3_exp(xi + 6 * f, P[f]);
  double L = 0;
  for (uint32_t i = 0; i < n; ++i) {
    double sum = 0;
    int cnt = 0;
    for (int f = 0; f < nf; ++f) {
      if (!(masks[(size_t)i * words + f / 32] >> (f % 32) & 1u)) continue;
      int iu, iv;
      bool live;
      diff_cell(c, samples + 3 * i, T0 + 12 * f, depth + (size_t)f * W * H, &iu, &iv, &live);
      sum += diff_term(c, samples + 3 * i, P[f], depth + (size_t)f * W * H, iu, iv, live).f;
      ++cnt;
    }
    const double Fi = cnt ? sum / cnt : 0.0;
    if (F) F[i] = Fi;
    L += Fi * Fi;
  }
  return L;
}

// Backward (FP64): dL/d depth (nf * H * W doubles, overwritten) and dL/d xi (nf * 6 doubles).
void orc_diff_backward(const float* params, int W, int H, int nf, const int32_t* samples,
                       uint32_t n, const float* depth, const float* T0, const double* xi,
                       const uint32_t* masks, double* gdepth, double* gxi) {
  const DiffCfg c = diff_cfg(params, W, H, nf);
  const int words = (nf + 31) / 32;
  std::vector<Pose64> P(nf);
  for (int f = 0; f < nf; ++f) se3_exp(xi + 6 * f, P[f]);
  std::fill(gdepth, gdepth + (size_t)nf * W * H, 0.0);
  std::fill(gxi, gxi + 6 * nf, 0.0);
  std::vector<double> M(9 * nf, 0.0), G(3 * nf, 0.0);
  for (uint32_t i = 0; i < n; ++i) {
    std::vector<Term> terms;
    std::vector<int> fr;
    for (int f = 0; f < nf; ++f) {
      if (!(masks[(size_t)i * words + f / 32] >> (f % 32) & 1u)) continue;
      int iu, iv;
      bool live;
      diff_cell(c, samples + 3 * i, T0 + 12 * f, depth + (size_t)f * W * H, &iu, &iv, &live);
      terms.push_back(diff_term(c, samples + 3 * i, P[f], depth + (size_t)f * W * H, iu, iv, live));
      fr.push_back(f);
    }
    if (terms.empty()) continue;
    double sum = 0;
    for (const Term& T : terms) sum += T.f;
    const double Fi = sum / terms.size();
    const double gf = 2.0 * Fi / terms.size();   // dL / df_f
    for (size_t q = 0; q < terms.size(); ++q) {
      const Term& T = terms[q];
      const int f = fr[q];
      for (int k = 0; k < 4; ++k) gdepth[(size_t)f * W * H + T.idx[k]] += gf * T.dfdD[k];
      for (int a = 0; a < 3; ++a) {
        const double gp = gf * T.dfdp[a];
        G[3 * f + a] += gp;
        for (int b = 0; b < 3; ++b) M[9 * f + 3 * b + a] += T.y[b] * gp;   // M = sum y g^T
      }
    }
  }
  for (int f = 0; f < nf; ++f) {
    double RG[3];
    for (int i = 0; i < 3; ++i)
      RG[i] = P[f].R[3 * i] * G[3 * f] + P[f].R[3 * i + 1] * G[3 * f + 1] + P[f].R[3 * i + 2] * G[3 * f + 2];
    for (int k = 0; k < 6; ++k) {
      double acc = 0;
      for (int e = 0; e < 9; ++e) acc += P[f].dR[k][e] * M[9 * f + e];
      for (int i = 0; i < 3; ++i) acc -= RG[i] * P[f].dt[k][i];
      gxi[6 * f + k] = acc;
    }
  }
}

}  // extern "C"
