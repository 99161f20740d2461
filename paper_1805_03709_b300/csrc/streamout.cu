// Stream-out of blocks that leave the active model (Sec. 4.1: blocks no longer in the sensor's
// view move to CPU memory) and explicit stream-in.
//
// Device side (erase.cu): every erase launch records the pool index and key of each block it
// removes, and the gather kernel that follows copies their 4 KiB of (TSDF, weight) and keys into
// the next slots of a device transfer ring before an allocation can reuse the pool entries.  It
// publishes the ring head to pinned host memory.
// Host side (here): a poll -- at the start of every frame or erase call, or explicitly -- copies
// the newly filled slots to a pinned host ring with asynchronous copies on a side stream, and
// once a copy has landed folds its blocks into the host map (the block's values at its last
// erase) and advances the tail that the next control block tells the gather.  A ring that
// would overflow loses nothing silently: the gather counts what found no room and raises a
// sticky flag; the poll keeps the ring at most half full by waiting for copies first.
#include <algorithm>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace vbh {

struct StreamOutHost {
  unsigned long long cap = 0;
  float2* h_data = nullptr;                 // pinned host ring, cap x 512
  unsigned long long* h_keys = nullptr;     // pinned host ring, cap
  unsigned long long* head_mapped = nullptr;   // mapped: slots the device has filled
  unsigned long long issued = 0;            // slots whose copy has been started
  unsigned long long tail = 0;              // slots folded into the map (free again)
  cudaStream_t side = nullptr;
  struct Copy {
    cudaEvent_t ev;
    unsigned long long b, e;
  };
  std::deque<Copy> copies;
  std::vector<cudaEvent_t> ev_free;
  std::unordered_map<unsigned long long, unsigned int> index;   // key -> store slot
  std::vector<float2> store;                                    // slots x 512
  std::vector<unsigned int> free_slots;
  unsigned long long streamed = 0;          // blocks folded in so far
};

namespace {

unsigned long long published_head(const StreamOutHost* so) {
  return *reinterpret_cast<volatile unsigned long long*>(so->head_mapped);
}

void fold(StreamOutHost* so, unsigned long long b, unsigned long long e) {
  for (unsigned long long i = b; i < e; ++i) {
    const unsigned long long slot = i % so->cap;
    const unsigned long long key = so->h_keys[slot];
    unsigned int at;
    auto it = so->index.find(key);
    if (it != so->index.end()) {
      at = it->second;
    } else if (!so->free_slots.empty()) {
      at = so->free_slots.back();
      so->free_slots.pop_back();
      so->index.emplace(key, at);
    } else {
      at = (unsigned int)(so->store.size() / 512);
      so->store.resize(so->store.size() + 512);
      so->index.emplace(key, at);
    }
    std::memcpy(so->store.data() + 512ull * at, so->h_data + 512ull * slot, 512 * sizeof(float2));
  }
  so->streamed += e - b;
}

// Start copies of [b, e) (split at the ring's end) on the side stream.
vbh_status issue(vbh_handle* h, StreamOutHost* so, unsigned long long b, unsigned long long e) {
  while (b < e) {
    const unsigned long long s0 = b % so->cap;
    const unsigned long long n = std::min(e - b, so->cap - s0);
    VBH_CUDA(cudaMemcpyAsync(so->h_data + 512ull * s0, h->so_data_dev + 512ull * s0,
                             n * 512 * sizeof(float2), cudaMemcpyDeviceToHost, so->side));
    VBH_CUDA(cudaMemcpyAsync(so->h_keys + s0, h->so_keys_dev + s0,
                             n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, so->side));
    b += n;
  }
  return VBH_OK;
}

}  // namespace

unsigned long long stream_out_tail(const vbh_handle* h) { return h->so ? h->so->tail : 0ull; }

vbh_status stream_out_poll(vbh_handle* h, bool wait) {
  StreamOutHost* so = h->so;
  if (!so) return VBH_OK;
  if (wait) VBH_CUDA(cudaStreamSynchronize(h->stream));
  for (int round = 0; round < 2; ++round) {
    const unsigned long long head = published_head(so);
    if (head > so->issued) {
      vbh_status st = issue(h, so, so->issued, head);
      if (st != VBH_OK) return st;
      cudaEvent_t ev;
      if (!so->ev_free.empty()) {
        ev = so->ev_free.back();
        so->ev_free.pop_back();
      } else {
        VBH_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      }
      VBH_CUDA(cudaEventRecord(ev, so->side));
      so->copies.push_back(StreamOutHost::Copy{ev, so->issued, head});
      so->issued = head;
    }
    // fold landed copies; keep the ring at most half full (a frame may erase many blocks)
    while (!so->copies.empty()) {
      StreamOutHost::Copy& c = so->copies.front();
      const bool must = wait || (published_head(so) - so->tail) * 2 > so->cap;
      if (must) {
        VBH_CUDA(cudaEventSynchronize(c.ev));
      } else {
        const cudaError_t q = cudaEventQuery(c.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return fail(VBH_ERR_CUDA, cudaGetErrorString(q));
      }
      fold(so, c.b, c.e);
      so->tail = c.e;
      so->ev_free.push_back(c.ev);
      so->copies.pop_front();
    }
    if (!wait) break;
  }
  return VBH_OK;
}

void stream_out_release(vbh_handle* h) {
  StreamOutHost* so = h->so;
  if (!so) return;
  if (so->side) cudaStreamSynchronize(so->side);
  for (auto& c : so->copies) cudaEventDestroy(c.ev);
  for (auto e : so->ev_free) cudaEventDestroy(e);
  if (so->side) cudaStreamDestroy(so->side);
  if (so->h_data) cudaFreeHost(so->h_data);
  if (so->h_keys) cudaFreeHost(so->h_keys);
  if (so->head_mapped) cudaFreeHost(so->head_mapped);
  if (h->so_data_dev) cudaFree(h->so_data_dev);
  if (h->so_keys_dev) cudaFree(h->so_keys_dev);
  if (h->so_ring) cudaFree(h->so_ring);
  if (h->so_p) cudaFree(h->so_p);
  if (h->so_k) cudaFree(h->so_k);
  delete so;
  h->so = nullptr;
  h->so_ring = nullptr;
  h->so_p = nullptr;
  h->so_k = nullptr;
  h->so_data_dev = nullptr;
  h->so_keys_dev = nullptr;
}

}  // namespace vbh

using namespace vbh;

extern "C" {

vbh_status vbh_stream_out_enable(vbh_handle* h, uint32_t ring_blocks) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (h->so) return VBH_OK;
  if (ring_blocks == 0) ring_blocks = h->cfg.max_blocks;
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  StreamOutHost* so = new StreamOutHost();
  so->cap = ring_blocks;
  h->so = so;
  const unsigned int nb = h->cfg.max_blocks;
  auto bail = [&](const char* what, cudaError_t e) {
    stream_out_release(h);
    return fail(VBH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMalloc(&h->so_p, sizeof(unsigned int) * nb)) != cudaSuccess ||
      (e = cudaMalloc(&h->so_k, sizeof(unsigned long long) * nb)) != cudaSuccess ||
      (e = cudaMalloc(&h->so_data_dev, 512ull * sizeof(float2) * ring_blocks)) !=
          cudaSuccess ||
      (e = cudaMalloc(&h->so_keys_dev, sizeof(unsigned long long) * ring_blocks)) !=
          cudaSuccess ||
      (e = cudaMalloc(&h->so_ring, sizeof(StreamRing))) != cudaSuccess)
    return bail("stream-out device memory", e);
  if ((e = cudaHostAlloc(&so->h_data, 512ull * sizeof(float2) * ring_blocks,
                         cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(&so->h_keys, sizeof(unsigned long long) * ring_blocks,
                         cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(&so->head_mapped, sizeof(unsigned long long), cudaHostAllocMapped)) !=
          cudaSuccess)
    return bail("stream-out pinned memory", e);
  *so->head_mapped = 0ull;
  unsigned long long* head_dev = nullptr;
  if ((e = cudaHostGetDevicePointer((void**)&head_dev, so->head_mapped, 0)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&so->side, cudaStreamNonBlocking)) != cudaSuccess)
    return bail("stream-out stream", e);
  StreamRing r{};
  r.data = h->so_data_dev;
  r.keys = h->so_keys_dev;
  r.head_host = head_dev;
  r.cap = ring_blocks;
  if ((e = cudaMemcpy(h->so_ring, &r, sizeof r, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail("stream-out ring", e);
  // the frame graph is captured again with the gather node
  if (h->frame_exec) cudaGraphExecDestroy(h->frame_exec);
  if (h->frame_graph) cudaGraphDestroy(h->frame_graph);
  h->frame_exec = nullptr;
  h->frame_graph = nullptr;
  return VBH_OK;
}

vbh_status vbh_stream_out_poll(vbh_handle* h, uint64_t* streamed_host) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (!h->so) return fail(VBH_ERR_UNSUPPORTED, "stream-out is not enabled");
  vbh_status st = stream_out_poll(h, false);
  if (streamed_host) *streamed_host = h->so->streamed;
  return st;
}

vbh_status vbh_stream_out_flush(vbh_handle* h) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (!h->so) return fail(VBH_ERR_UNSUPPORTED, "stream-out is not enabled");
  return stream_out_poll(h, true);
}

vbh_status vbh_stream_out_stats(vbh_handle* h, uint64_t* streamed_host, uint64_t* lost_host,
                                uint32_t* host_blocks_host) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (!h->so) return fail(VBH_ERR_UNSUPPORTED, "stream-out is not enabled");
  vbh_status st = stream_out_poll(h, true);
  if (st != VBH_OK) return st;
  StreamRing r{};
  VBH_CUDA(cudaMemcpy(&r, h->so_ring, sizeof r, cudaMemcpyDeviceToHost));
  if (streamed_host) *streamed_host = h->so->streamed;
  if (lost_host) *lost_host = r.lost;
  if (host_blocks_host) *host_blocks_host = (uint32_t)h->so->index.size();
  return VBH_OK;
}

vbh_status vbh_host_map_dump(vbh_handle* h, int32_t* keys3, float* tsdf, float* weight,
                             uint32_t cap, uint32_t* n_host) {
  if (!h || !n_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (!h->so) return fail(VBH_ERR_UNSUPPORTED, "stream-out is not enabled");
  if (cap && !keys3) return fail(VBH_ERR_INVALID_ARG, "null key buffer");
  vbh_status st = stream_out_poll(h, true);
  if (st != VBH_OK) return st;
  const StreamOutHost* so = h->so;
  uint32_t i = 0;
  for (const auto& kv : so->index) {
    if (i >= cap) break;
    const int3 k = unpack_key(kv.first);
    keys3[3 * i] = k.x;
    keys3[3 * i + 1] = k.y;
    keys3[3 * i + 2] = k.z;
    const float2* b = so->store.data() + 512ull * kv.second;
    for (int v = 0; v < 512; ++v) {
      if (tsdf) tsdf[512ull * i + v] = b[v].x;
      if (weight) weight[512ull * i + v] = b[v].y;
    }
    ++i;
  }
  *n_host = (uint32_t)so->index.size();
  return VBH_OK;
}

vbh_status vbh_stream_in(vbh_handle* h, const int32_t* keys3_host, uint32_t n,
                         uint32_t* n_loaded_host) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (!h->so) return fail(VBH_ERR_UNSUPPORTED, "stream-out is not enabled");
  if (n && !keys3_host) return fail(VBH_ERR_INVALID_ARG, "null key list");
  if (n_loaded_host) *n_loaded_host = 0;
  vbh_status st = stream_out_poll(h, true);
  if (st != VBH_OK || n == 0) return st;
  StreamOutHost* so = h->so;
  // candidates: listed keys that are in the host map (in range, each once)
  std::vector<int32_t> cand;
  std::vector<unsigned int> at;
  std::unordered_map<unsigned long long, int> seen;
  for (uint32_t i = 0; i < n; ++i) {
    const int x = keys3_host[3 * i], y = keys3_host[3 * i + 1], z = keys3_host[3 * i + 2];
    if (!key_ok(x, y, z)) continue;
    const unsigned long long key = pack_key(x, y, z);
    auto it = so->index.find(key);
    if (it == so->index.end() || !seen.emplace(key, 1).second) continue;
    cand.insert(cand.end(), {x, y, z});
    at.push_back(it->second);
  }
  const uint32_t m = (uint32_t)at.size();
  if (!m) return VBH_OK;
  if (m > h->cfg.max_batch) return fail(VBH_ERR_INVALID_ARG, "more blocks than max_batch");
  // which of them are live now (a live block is newer: it stays and so does its host copy)
  int* dk = nullptr;
  unsigned char *dops = nullptr, *dst = nullptr;
  unsigned int* dres = nullptr;
  std::vector<unsigned char> ops(m, (unsigned char)VBH_OP_FIND), hst(m);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&dk, (size_t)m * 12)) == cudaSuccess &&
      (e = cudaMalloc(&dops, m)) == cudaSuccess && (e = cudaMalloc(&dst, m)) == cudaSuccess &&
      (e = cudaMalloc(&dres, (size_t)m * 4)) == cudaSuccess) {
    cudaMemcpyAsync(dk, cand.data(), (size_t)m * 12, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dops, ops.data(), m, cudaMemcpyHostToDevice, h->stream);
    st = vbh_hash_batch(h, dops, dk, nullptr, dres, dst, m);
    if (st == VBH_OK) {
      cudaMemcpyAsync(hst.data(), dst, m, cudaMemcpyDeviceToHost, h->stream);
      e = cudaStreamSynchronize(h->stream);
    }
  }
  for (void* p : {(void*)dk, (void*)dops, (void*)dst, (void*)dres})
    if (p) cudaFree(p);
  if (e != cudaSuccess) return fail(VBH_ERR_CUDA, std::string("vbh_stream_in: ") + cudaGetErrorString(e));
  if (st != VBH_OK) return st;
  std::vector<int32_t> keys;
  std::vector<float> F, W;
  std::vector<unsigned long long> moved;
  for (uint32_t i = 0; i < m; ++i) {
    if (hst[i] != VBH_ST_NOT_FOUND) continue;
    keys.insert(keys.end(), {cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]});
    const float2* b = so->store.data() + 512ull * at[i];
    for (int v = 0; v < 512; ++v) {
      F.push_back(b[v].x);
      W.push_back(b[v].y);
    }
    moved.push_back(pack_key(cand[3 * i], cand[3 * i + 1], cand[3 * i + 2]));
  }
  const uint32_t k = (uint32_t)moved.size();
  if (k) {
    st = vbh_load(h, keys.data(), F.data(), W.data(), k);
    if (st != VBH_OK) return st;
    for (unsigned long long key : moved) {
      auto it = so->index.find(key);
      so->free_slots.push_back(it->second);
      so->index.erase(it);
    }
  }
  if (n_loaded_host) *n_loaded_host = k;
  return VBH_OK;
}

}  // extern "C"
