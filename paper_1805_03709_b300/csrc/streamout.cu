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
// sticky flag; the poll waits for copies once the ring is three quarters full.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace vbh {

// Flat open-addressing map from packed block keys to a location (linear probing, power-of-two
// capacity kept at most half full; erase by backward shift).  A location is a ring sequence
// number (the block's latest copy still sits in the pinned ring) or, with kInStore set, a slot
// of the long-term store.
class KeyIndex {
 public:
  static constexpr unsigned long long kFree = ~0ull;
  KeyIndex() { rehash(1u << 16); }
  unsigned long long* find(unsigned long long key) {
    for (size_t i = slot(key);; i = (i + 1) & mask_) {
      if (keys_[i] == key) return &vals_[i];
      if (keys_[i] == kFree) return nullptr;
    }
  }
  // inserts or overwrites; returns the previous value or kFree
  unsigned long long put(unsigned long long key, unsigned long long val) {
    if ((size_ + 1) * 2 > keys_.size()) rehash(keys_.size() * 2);
    for (size_t i = slot(key);; i = (i + 1) & mask_) {
      if (keys_[i] == key) {
        const unsigned long long old = vals_[i];
        vals_[i] = val;
        return old;
      }
      if (keys_[i] == kFree) {
        keys_[i] = key;
        vals_[i] = val;
        ++size_;
        return kFree;
      }
    }
  }
  void erase(unsigned long long key) {
    size_t i = slot(key);
    for (;; i = (i + 1) & mask_) {
      if (keys_[i] == kFree) return;
      if (keys_[i] == key) break;
    }
    for (size_t j = (i + 1) & mask_; keys_[j] != kFree; j = (j + 1) & mask_) {
      const size_t home = slot(keys_[j]);
      // move j back to the hole i unless its home lies cyclically in (i, j]
      if (((j - home) & mask_) >= ((j - i) & mask_)) {
        keys_[i] = keys_[j];
        vals_[i] = vals_[j];
        i = j;
      }
    }
    keys_[i] = kFree;
    --size_;
  }
  size_t size() const { return size_; }
  template <class F>
  void each(F f) const {
    for (size_t i = 0; i < keys_.size(); ++i)
      if (keys_[i] != kFree) f(keys_[i], vals_[i]);
  }

 private:
  size_t slot(unsigned long long key) const { return hash_mix(key) & mask_; }
  void rehash(size_t cap) {
    std::vector<unsigned long long> k(cap, kFree), v(cap);
    keys_.swap(k);
    vals_.swap(v);
    mask_ = cap - 1;
    size_ = 0;
    for (size_t i = 0; i < k.size(); ++i)
      if (k[i] != kFree) put(k[i], v[i]);
  }
  std::vector<unsigned long long> keys_, vals_;
  size_t mask_ = 0, size_ = 0;
};

constexpr unsigned long long kInStore = 1ull << 63;

// A few persistent host threads for the eviction copies (one thread copies ~14 GB/s).
class CopyPool {
 public:
  explicit CopyPool(unsigned int n) {
    for (unsigned int i = 0; i < n; ++i) threads_.emplace_back([this, i] { run(i); });
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  // copies jobs[i].second -> jobs[i].first (4 KiB each) on the pool, returns when done
  void copy(const std::vector<std::pair<float2*, const float2*>>& jobs) {
    if (jobs.size() < 64 || threads_.empty()) {
      for (const auto& j : jobs) std::memcpy(j.first, j.second, 512 * sizeof(float2));
      return;
    }
    {
      std::lock_guard<std::mutex> g(m_);
      jobs_ = &jobs;
      pending_ = (unsigned int)threads_.size();
      ++gen_;
    }
    cv_.notify_all();
    std::unique_lock<std::mutex> l(m_);
    done_.wait(l, [this] { return pending_ == 0; });
    jobs_ = nullptr;
  }

 private:
  void run(unsigned int me) {
    unsigned long long seen = 0;
    for (;;) {
      const std::vector<std::pair<float2*, const float2*>>* jobs;
      {
        std::unique_lock<std::mutex> l(m_);
        cv_.wait(l, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
        jobs = jobs_;
      }
      const size_t n = jobs->size(), k = threads_.size();
      for (size_t i = me * n / k; i < (me + 1) * n / k; ++i)
        std::memcpy((*jobs)[i].first, (*jobs)[i].second, 512 * sizeof(float2));
      {
        std::lock_guard<std::mutex> g(m_);
        if (--pending_ == 0) done_.notify_one();
      }
    }
  }
  std::vector<std::thread> threads_;
  std::mutex m_;
  std::condition_variable cv_, done_;
  const std::vector<std::pair<float2*, const float2*>>* jobs_ = nullptr;
  unsigned long long gen_ = 0;
  unsigned int pending_ = 0;
  bool stop_ = false;
};

constexpr unsigned int kChunkBlocks = 4096;   // long-term store chunk: 16 MiB

struct StreamOutHost {
  unsigned long long cap = 0;
  float2* h_data = nullptr;                 // pinned host ring, cap x 512
  unsigned long long* h_keys = nullptr;     // pinned host ring, cap
  unsigned long long* head_mapped = nullptr;   // mapped: slots the device has filled
  unsigned long long issued = 0;            // slots whose copy has been started
  unsigned long long landed = 0;            // slots whose copy has landed (indexed)
  unsigned long long tail = 0;              // slots released to the device again
  cudaStream_t side = nullptr;
  struct Copy {
    cudaEvent_t ev;
    unsigned long long b, e;
  };
  std::deque<Copy> copies;
  std::vector<cudaEvent_t> ev_free;
  KeyIndex index;                           // key -> ring sequence number or store slot
  std::vector<std::unique_ptr<float2[]>> chunks;   // long-term store: blocks never move
  unsigned int n_slots = 0;
  std::vector<unsigned int> free_slots;
  unsigned long long streamed = 0;          // blocks folded in so far
  CopyPool pool{8};
  std::vector<std::pair<float2*, const float2*>> jobs;
  float2* slot_ptr(unsigned int at) {
    return chunks[at / kChunkBlocks].get() + 512ull * (at % kChunkBlocks);
  }
  const float2* data_of(unsigned long long loc) const {
    if (loc & kInStore) {
      const unsigned int at = (unsigned int)(loc & ~kInStore);
      return chunks[at / kChunkBlocks].get() + 512ull * (at % kChunkBlocks);
    }
    return h_data + 512ull * (loc % cap);
  }
  unsigned int new_slot() {
    if (!free_slots.empty()) {
      const unsigned int at = free_slots.back();
      free_slots.pop_back();
      return at;
    }
    if (n_slots % kChunkBlocks == 0) chunks.emplace_back(new float2[512ull * kChunkBlocks]);
    return n_slots++;
  }
};

namespace {

unsigned long long published_head(const StreamOutHost* so) {
  return *reinterpret_cast<volatile unsigned long long*>(so->head_mapped);
}

// Landed copies only update the index: a block's data stays in its ring slot until the slot is
// needed again (a block erased again meanwhile -- the common case at the edge of the active
// region -- never costs a host copy).
void fold(StreamOutHost* so, unsigned long long b, unsigned long long e) {
  for (unsigned long long i = b; i < e; ++i) {
    const unsigned long long old = so->index.put(so->h_keys[i % so->cap], i);
    if (old != KeyIndex::kFree && (old & kInStore)) so->free_slots.push_back((unsigned int)(old & ~kInStore));
  }
  so->streamed += e - b;
  so->landed = e;
}

// Release ring slots [tail, upto): blocks whose latest copy is still there move to the store
// (the copies run on the pool).
void evict(StreamOutHost* so, unsigned long long upto) {
  so->jobs.clear();
  for (unsigned long long i = so->tail; i < upto; ++i) {
    const unsigned long long key = so->h_keys[i % so->cap];
    unsigned long long* loc = so->index.find(key);
    if (!loc || *loc != i) continue;   // superseded or streamed back in
    const unsigned int at = so->new_slot();
    so->jobs.emplace_back(so->slot_ptr(at), so->h_data + 512ull * (i % so->cap));
    *loc = kInStore | at;
  }
  so->pool.copy(so->jobs);
  so->tail = upto;
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
    // index landed copies; the newest half of the ring stays indexed in place, older slots are
    // released (their current blocks move to the store); past three quarters, wait for copies
    while (!so->copies.empty()) {
      StreamOutHost::Copy& c = so->copies.front();
      const bool must = wait || (published_head(so) - so->tail) * 4 > so->cap * 3;
      if (must) {
        VBH_CUDA(cudaEventSynchronize(c.ev));
      } else {
        const cudaError_t q = cudaEventQuery(c.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return fail(VBH_ERR_CUDA, cudaGetErrorString(q));
      }
      fold(so, c.b, c.e);
      so->ev_free.push_back(c.ev);
      so->copies.pop_front();
    }
    const unsigned long long keep = so->cap / 2;   // recent slots stay in the ring
    if (so->landed - so->tail > keep) evict(so, so->landed - keep);
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
  so->index.each([&](unsigned long long key, unsigned long long loc) {
    if (i >= cap) return;
    const int3 k = unpack_key(key);
    keys3[3 * i] = k.x;
    keys3[3 * i + 1] = k.y;
    keys3[3 * i + 2] = k.z;
    const float2* b = so->data_of(loc);
    for (int v = 0; v < 512; ++v) {
      if (tsdf) tsdf[512ull * i + v] = b[v].x;
      if (weight) weight[512ull * i + v] = b[v].y;
    }
    ++i;
  });
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
  std::vector<unsigned long long> at;
  std::unordered_map<unsigned long long, int> seen;
  for (uint32_t i = 0; i < n; ++i) {
    const int x = keys3_host[3 * i], y = keys3_host[3 * i + 1], z = keys3_host[3 * i + 2];
    if (!key_ok(x, y, z)) continue;
    const unsigned long long key = pack_key(x, y, z);
    const unsigned long long* loc = so->index.find(key);
    if (!loc || !seen.emplace(key, 1).second) continue;
    cand.insert(cand.end(), {x, y, z});
    at.push_back(*loc);
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
    const float2* b = so->data_of(at[i]);
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
      const unsigned long long loc = *so->index.find(key);
      if (loc & kInStore) so->free_slots.push_back((unsigned int)(loc & ~kInStore));
      so->index.erase(key);
    }
  }
  if (n_loaded_host) *n_loaded_host = k;
  return VBH_OK;
}

}  // extern "C"
