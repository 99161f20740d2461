// Multi-client delta streaming with continuous batching (the server side of Sec. 4.2, where each
// client requests the MC blocks that changed since its last update).  The paper keeps one hash
// set of changed block ids per client; here every MC refresh of a block, and every removal
// record, takes the next number of one change sequence (written by the per-frame extraction in
// mc.cu to a ring log, with the block's dense cube indices kept in a store), and a client is a
// single sequence number v kept on the device: its request is the range (v, sigma] of the log.
//
// A change record e is current when it is the newest word on its key at the time it is read:
//   refresh of pool entry p: seq[p] == e (seq is reset when the block is erased) and the
//   entry still holds the record's key;
//   removal of key k: lastrem[k] == e and k is not live.
// One batch of requests is one launch of k_serve_extract: every request contributes a chunk
// (a range of log records, or of pool entries for a reset), the chunks -- smallest first -- are
// cut into tiles of 32 records, and the persistent grid's warps take tiles in turn.  A warp
// tests its 32 records, reserves output records with one atomic on the request's counter and
// copies each current block's 512 B of cube indices (one 16 B word per lane).  The warp that
// finishes the last tile of a request's final chunk moves the client to its new version and
// publishes the record count with the request's id as a token in mapped host memory, so a
// small request completes as soon as its own tiles are done, not when the whole batch is.
//
// The host side (a scheduler, a first-fit arena for the stream buffer, the real-time loop of
// vbh_serve_run) decides admission and chunking; the batch table travels as the kernel's
// parameter block, so a launch needs no host-to-device copy.
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace vbh {

namespace {

constexpr int kServeThreads = 256;
constexpr int kServeWarps = kServeThreads / 32;
constexpr int kServeMaxBatch = 64;
constexpr unsigned int kRecHeader = 16u, kRecPayload = 512u, kRecBytes = 528u;
constexpr unsigned int kItemScan = 1u, kItemFinal = 2u, kItemFirst = 4u;

struct ServeItem {
  unsigned int slot, client;
  unsigned int lo, hi;        // log: records lo+1 .. hi; scan: pool entries lo .. hi-1
  unsigned int sigma;         // snapshot of the request
  unsigned int flags;
  unsigned int cap;           // output records of the request's region
  unsigned int v0, v1;        // client version before / after the request
  unsigned int id;            // request id (completion token)
  unsigned long long out;     // byte offset of the region in the arena
};

struct ServeBatch {
  unsigned int n, pad;
  unsigned int tiles[kServeMaxBatch + 1];   // prefix sums of 32-record tiles
  ServeItem it[kServeMaxBatch];
};
static_assert(sizeof(ServeBatch) + 128 <= 4096, "batch table must fit the kernel parameters");

struct ServeCtx {
  TableView t;
  PoolView pool;
  const ServeLog* sl;
  unsigned char* arena;
  unsigned int* rec_count;    // per slot, zero while the slot is free
  unsigned int* slot_err;     // per slot
  unsigned int* client_v;     // per client
  unsigned int* tiles_done;   // per slot: tiles of the current chunk finished
  uint4* done_host;           // mapped: per slot (records, error bits, token = request id)
};

__device__ __forceinline__ unsigned int rem_latest(const ServeLog& S, unsigned long long key) {
  unsigned int b = hash_mix(key) & S.rem_mask;
  for (unsigned int probe = 0; probe <= S.rem_mask; ++probe, b = (b + 1u) & S.rem_mask) {
    const unsigned long long k = __ldcg(S.rem_keys + b);
    if (k == key) return __ldcg(S.rem_seq + b);
    if (k == kEmpty) break;
  }
  return 0u;
}

__global__ void __launch_bounds__(kServeThreads) k_serve_extract(const ServeBatch B,
                                                                 const ServeCtx X) {
  __shared__ unsigned int s_tiles[kServeMaxBatch + 1];
  __shared__ ServeItem s_it[kServeMaxBatch];
  const unsigned int nb = B.n;
  for (unsigned int i = threadIdx.x; i <= nb; i += blockDim.x) s_tiles[i] = B.tiles[i];
  for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) s_it[i] = B.it[i];
  __syncthreads();
  const ServeLog S = *X.sl;
  const unsigned int total = s_tiles[nb];
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned int nwarps = gridDim.x * kServeWarps;
  const unsigned int lt_mask = (1u << lane) - 1u;
  for (unsigned int tile = blockIdx.x * kServeWarps + warp; tile < total; tile += nwarps) {
    unsigned int a = 0, b = nb;   // s_tiles[a] <= tile < s_tiles[b]
    while (b - a > 1u) {
      const unsigned int m = (a + b) >> 1;
      if (s_tiles[m] <= tile) a = m;
      else b = m;
    }
    const ServeItem& it = s_it[a];
    const unsigned int t = tile - s_tiles[a];
    bool cur = false;
    unsigned long long key = 0ull;
    unsigned int info = 0u, p = kNone, err = 0u;
    if (it.flags & kItemScan) {
      const unsigned int j = it.lo + 32u * t + lane;
      if (j < it.hi) {
        const unsigned long long k = X.pool.pkeys[j];
        const unsigned int sq = X.pool.seq[j];
        if (k != kEmpty && sq != 0u && sq <= it.sigma) {
          cur = true;
          key = k;
          p = j;
          info = X.pool.version[j] & 0x7FFFFFFFu;
        }
      }
    } else {
      const unsigned int e = it.lo + 1u + 32u * t + lane;
      if (e <= it.hi) {
        const LogEnt le = S.log[e & S.log_mask];
        if (le.seq != e) {
          err |= kServeErrOverrun;
        } else if (le.key & kLogRemoved) {
          const unsigned long long k = le.key & ~kLogRemoved;
          unsigned int v;
          if (rem_latest(S, k) == e && thread_find(X.t, k, &v) == kNone) {
            cur = true;
            key = k;
            info = 0x80000000u | le.aux;
          }
        } else {
          const unsigned int q = le.aux;
          if (X.pool.seq[q] == e && X.pool.pkeys[q] == le.key) {
            cur = true;
            key = le.key;
            p = q;
            info = X.pool.version[q] & 0x7FFFFFFFu;
          }
        }
      }
    }
    if ((it.flags & kItemFirst) && t == 0u && lane == 0u && X.client_v[it.client] != it.v0)
      err |= 16u;   // the device version disagrees with the planned one
    const unsigned int bal = __ballot_sync(0xFFFFFFFFu, cur);
    const unsigned int n = __popc(bal);
    unsigned int base = 0u;
    if (n) {
      if (lane == 0u) base = atomicAdd(&X.rec_count[it.slot], n);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
    }
    if (n && (unsigned long long)base + n > it.cap) {
      err |= kServeErrCap;
    } else if (n) {
      unsigned char* region = X.arena + it.out;
      int4* hdr = reinterpret_cast<int4*>(region);
      uint4* pay = reinterpret_cast<uint4*>(region + (size_t)it.cap * kRecHeader);
      if (cur) {
        const int3 k3 = unpack_key(key);
        hdr[base + __popc(bal & lt_mask)] = make_int4(k3.x, k3.y, k3.z, (int)info);
      }
      unsigned int live = __ballot_sync(0xFFFFFFFFu, cur && p != kNone);
      while (live) {   // four 512 B copies in flight per round
        uint4 v[4];
        unsigned int dst[4];
        int m = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!live) break;
          const int src = __ffs(live) - 1;
          live &= live - 1u;
          const unsigned int q = __shfl_sync(0xFFFFFFFFu, p, src);
          dst[i] = base + __popc(bal & ((1u << src) - 1u));
          v[i] = S.store[32u * q + lane];
          m = i + 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < m) pay[(size_t)dst[i] * 32u + lane] = v[i];
      }
    }
    if (err) atomicOr(&X.slot_err[it.slot], err);
    // the warp that finishes the chunk's last tile closes it; after a final chunk it publishes
    // the request (every lane fences its writes before the warp's tile is counted)
    __threadfence();
    __syncwarp();
    if (lane == 0u) {
      const unsigned int chunk_tiles = s_tiles[a + 1] - s_tiles[a];
      if (atomicAdd(&X.tiles_done[it.slot], 1u) == chunk_tiles - 1u) {
        X.tiles_done[it.slot] = 0u;
        if (it.flags & kItemFinal) {
          __threadfence();
          const unsigned int nr = atomicExch(&X.rec_count[it.slot], 0u);
          const unsigned int ef = atomicExch(&X.slot_err[it.slot], 0u);
          X.client_v[it.client] = it.v1;
          volatile unsigned int* d = reinterpret_cast<volatile unsigned int*>(X.done_host + it.slot);
          d[0] = nr;
          d[1] = ef;
          __threadfence_system();
          d[2] = it.id;
        }
      }
    }
  }
}

__global__ void k_live_seq(const unsigned long long* pkeys, const unsigned int* seq, unsigned int n,
                           unsigned int* out, unsigned int* n_out) {
  for (unsigned int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const bool take = pkeys[p] != kEmpty && seq[p] != 0u;
    const unsigned int k = warp_append(n_out, take, __activemask());
    if (take) out[k] = seq[p];
  }
}

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, size) with coalescing frees (offsets aligned to 256 B).
class Arena {
 public:
  explicit Arena(uint64_t size) : size_(size) { free_[0] = size; }
  bool alloc(uint64_t bytes, uint64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes;
      const uint64_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }

 private:
  uint64_t size_;
  uint64_t used_ = 0, peak_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

enum ReqState { kPending = 0, kActive = 1, kDone = 2 };

struct Req {
  vbh_serve_done d{};
  ReqState state = kPending;
  bool scan = false;
  int slot = -1;
  unsigned int start = 0, next = 0, end = 0, sigma = 0, cap = 0;
  uint64_t off = 0, bytes = 0;
};

struct Iter {
  cudaEvent_t ev;
  std::vector<uint32_t> finishing;
};

}  // namespace
}  // namespace vbh

using namespace vbh;

struct vbh_serve {
  vbh_handle* h = nullptr;
  vbh_serve_config cfg{};
  unsigned int log_cap = 0;
  // device state
  ServeLog* sl_dev = nullptr;
  LogEnt* log = nullptr;
  uint4* store = nullptr;
  unsigned long long* rem_keys = nullptr;
  unsigned int* rem_seq = nullptr;
  unsigned int* client_v = nullptr;
  unsigned int* rec_count = nullptr;
  unsigned int* slot_err = nullptr;
  unsigned int* tiles_done = nullptr;
  unsigned int* scratch = nullptr;   // two words for the store-only refresh
  unsigned char* arena = nullptr;
  // mapped host words
  unsigned int* sigma_host = nullptr;
  unsigned int* sigma_dev = nullptr;
  uint4* done_host = nullptr;
  uint4* done_dev = nullptr;
  int grid = 0;
  // host scheduler
  Arena* heap = nullptr;
  std::vector<unsigned int> v_mirror;
  std::vector<char> client_busy;
  std::vector<int> slot_req;
  std::unordered_map<uint32_t, Req> reqs;
  std::deque<uint32_t> pending;
  std::vector<int> active;           // slots with chunks left, oldest first
  std::deque<Iter> inflight;
  std::deque<uint32_t> completed;
  std::vector<cudaEvent_t> ev_free;
  uint32_t next_id = 1;
  uint32_t head_blocked = 0;         // iterations the head request has been memory-blocked
  vbh_serve_loop* loop = nullptr;    // a device-resident request loop owns the server
  vbh_serve_stats st{};

  unsigned int sigma() const { return *reinterpret_cast<volatile unsigned int*>(sigma_host); }
  cudaEvent_t get_event() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }
  int free_slot() const {
    for (int i = 0; i < (int)cfg.max_batch; ++i)
      if (slot_req[i] < 0) return i;
    return -1;
  }
  void finish(Req& r, uint64_t t) {
    r.state = kDone;
    r.d.t_done_ns = t;
    completed.push_back(r.d.id);
    st.requests_done += 1;
    st.records_served += r.d.n_records;
  }
  vbh_status reap();
  void admit();
  vbh_status launch();
};

namespace {

vbh_status check_policy(const vbh_serve_config& c) {
  if (c.max_batch < 1 || c.max_batch > (uint32_t)kServeMaxBatch)
    return fail(VBH_ERR_INVALID_ARG, "max_batch must be in 1..64");
  return VBH_OK;
}

}  // namespace

// Complete the requests whose token the device has published; retire finished iterations.
vbh_status vbh_serve::reap() {
  auto try_complete = [&](uint32_t& id) {
    if (!id) return true;
    Req& r = reqs[id];
    const volatile unsigned int* dw = reinterpret_cast<volatile unsigned int*>(done_host + r.slot);
    if (dw[2] != id) return false;
    std::atomic_thread_fence(std::memory_order_acquire);
    const unsigned int n = dw[0], e = dw[1];
    r.d.n_records = n;
    if (e & kServeErrOverrun) r.d.flags |= VBH_SERVE_ERR_OVERRUN;
    if (e & kServeErrCap) r.d.flags |= VBH_SERVE_ERR_CAPACITY;
    if (e & 16u) r.d.flags |= VBH_SERVE_ERR_VERSION;
    slot_req[r.slot] = -1;
    client_busy[r.d.client] = 0;
    v_mirror[r.d.client] = r.d.v_after;
    finish(r, now_ns());
    id = 0;
    return true;
  };
  for (Iter& I : inflight)
    for (uint32_t& id : I.finishing) try_complete(id);
  while (!inflight.empty()) {
    const cudaError_t q = cudaEventQuery(inflight.front().ev);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return fail(VBH_ERR_CUDA, std::string("serve: ") + cudaGetErrorString(q));
    for (uint32_t& id : inflight.front().finishing)
      if (!try_complete(id))
        return fail(VBH_ERR_CUDA, "serve: a batch finished without completing a request");
    ev_free.push_back(inflight.front().ev);
    inflight.pop_front();
  }
  return VBH_OK;
}

// Admit pending requests in arrival order while a slot is free and their worst case fits.
void vbh_serve::admit() {
  const unsigned int sig = sigma();
  const unsigned int margin = log_cap / 2u;   // records that may be appended while one runs
  const unsigned int floor = sig > margin ? sig - margin : 0u;
  const uint64_t max_recs = (cfg.budget_bytes & ~255ull) / kRecBytes;
  bool head = true;
  for (auto it = pending.begin(); it != pending.end();) {
    const int slot = free_slot();
    if (slot < 0) break;
    Req& r = reqs[*it];
    const uint32_t c = r.d.client;
    if (client_busy[c]) {   // one request per client at a time, in arrival order
      ++it;
      head = false;
      continue;
    }
    const unsigned int v = v_mirror[c];
    r.scan = v == 0u || v < floor;
    r.sigma = sig;
    r.d.v_before = v;
    r.d.flags = r.scan ? VBH_SERVE_RESET : 0u;
    uint64_t count;
    if (r.scan) {
      r.start = 0u;
      r.end = h->cfg.max_blocks;
      r.d.v_after = sig;
      count = h->cfg.max_blocks;
    } else {
      if (sig <= v) {   // nothing changed since v: complete without device work
        r.d.v_after = v;
        r.d.n_records = 0u;
        r.d.t_admit_ns = now_ns();
        finish(r, r.d.t_admit_ns);
        it = pending.erase(it);
        continue;
      }
      count = sig - v;
      if (count > max_recs) {
        count = max_recs;
        r.d.flags |= VBH_SERVE_PARTIAL;
      }
      r.start = v;
      r.end = v + (unsigned int)count;
      r.d.v_after = r.end;
    }
    r.cap = (unsigned int)count;
    r.bytes = (count * kRecBytes + 255u) & ~255ull;
    if (!heap->alloc(r.bytes, &r.off)) {
      st.deferred_memory += 1;
      if (head && ++head_blocked > cfg.bypass_iters) break;   // stop passing the head
      head = false;
      ++it;
      continue;
    }
    if (head) head_blocked = 0;
    r.d.bytes_reserved = r.bytes;
    r.d.t_admit_ns = now_ns();
    r.state = kActive;
    r.slot = slot;
    r.next = r.start;
    slot_req[slot] = (int)r.d.id;
    client_busy[c] = 1;
    active.push_back(slot);
    it = pending.erase(it);
  }
  st.bytes_in_use = heap->used();
  st.bytes_peak = heap->peak();
}

// One batch: a chunk of every active request (oldest first), one launch, one event.
vbh_status vbh_serve::launch() {
  if (active.empty()) return VBH_OK;
  ServeBatch B;
  std::memset(&B, 0, sizeof B);
  Iter I;
  uint64_t total = 0;
  std::vector<int> keep;
  for (size_t a = 0; a < active.size(); ++a) {
    Req& r = reqs[(uint32_t)slot_req[active[a]]];
    uint64_t take = r.end - r.next;
    if (cfg.chunk_records) take = std::min<uint64_t>(take, cfg.chunk_records);
    if (cfg.iter_records && B.n > 0) {
      if (total >= cfg.iter_records) take = 0;
      else take = std::min<uint64_t>(take, cfg.iter_records - total);
    }
    if (take == 0) {
      keep.push_back(active[a]);
      continue;
    }
    ServeItem& it = B.it[B.n];
    it.slot = (unsigned int)r.slot;
    it.client = r.d.client;
    it.lo = r.next;
    it.hi = r.next + (unsigned int)take;
    it.sigma = r.sigma;
    it.cap = r.cap;
    it.v0 = r.d.v_before;
    it.v1 = r.d.v_after;
    it.out = r.off;
    it.id = r.d.id;
    it.flags = (r.scan ? kItemScan : 0u) | (r.next == r.start ? kItemFirst : 0u);
    r.next += (unsigned int)take;
    if (r.next == r.end) {
      it.flags |= kItemFinal;
      I.finishing.push_back(r.d.id);
    } else {
      keep.push_back(active[a]);
    }
    total += take;
    B.n += 1;
  }
  active.swap(keep);
  if (B.n == 0) return VBH_OK;
  // smallest chunks first: their tiles go to the first wave of warps
  std::sort(B.it, B.it + B.n, [](const ServeItem& x, const ServeItem& y) {
    return x.hi - x.lo < y.hi - y.lo;
  });
  for (unsigned int i = 0; i < B.n; ++i)
    B.tiles[i + 1] = B.tiles[i] + (B.it[i].hi - B.it[i].lo + 31u) / 32u;
  ServeCtx X;
  X.t = h->table();
  X.pool = h->pool();
  X.sl = sl_dev;
  X.arena = arena;
  X.rec_count = rec_count;
  X.slot_err = slot_err;
  X.client_v = client_v;
  X.tiles_done = tiles_done;
  X.done_host = done_dev;
  const unsigned int tiles = B.tiles[B.n];
  const unsigned int want = (tiles + kServeWarps - 1u) / kServeWarps;
  const int grid_n = (int)std::min<unsigned int>(want ? want : 1u, (unsigned int)grid);
  k_serve_extract<<<grid_n, kServeThreads, 0, h->stream>>>(B, X);
  VBH_CUDA(cudaGetLastError());
  I.ev = get_event();
  VBH_CUDA(cudaEventRecord(I.ev, h->stream));
  inflight.push_back(std::move(I));
  h->launches += 1;
  st.iterations += 1;
  st.changes_scanned += total;
  return VBH_OK;
}

namespace vbh {
vbh_handle* serve_handle(vbh_serve* s) { return s->h; }
const ServeLog* serve_log(vbh_serve* s) { return s->sl_dev; }
ServeShared serve_shared(vbh_serve* s) {
  ServeShared x;
  x.h = s->h;
  x.sl = s->sl_dev;
  x.client_v = s->client_v;
  x.arena = s->arena;
  x.budget = s->cfg.budget_bytes & ~255ull;
  x.n_clients = s->cfg.n_clients;
  x.log_cap = s->log_cap;
  return x;
}
bool serve_idle(vbh_serve* s) {
  return s->pending.empty() && s->inflight.empty() && s->active.empty() &&
         std::none_of(s->slot_req.begin(), s->slot_req.end(), [](int r) { return r >= 0; });
}
vbh_serve_loop* serve_loop_of(vbh_serve* s) { return s->loop; }
void serve_set_loop(vbh_serve* s, vbh_serve_loop* L) { s->loop = L; }
// The host mirror of the client versions after a device loop has moved them.
vbh_status serve_reload_versions(vbh_serve* s) {
  VBH_CUDA(cudaMemcpy(s->v_mirror.data(), s->client_v, sizeof(unsigned int) * s->cfg.n_clients,
                      cudaMemcpyDeviceToHost));
  return VBH_OK;
}
}  // namespace vbh

namespace {
// While a device-resident loop owns the server, its host scheduler is not used.
bool loop_owned(vbh_serve* s) {
  if (s && s->loop) {
    fail(VBH_ERR_UNSUPPORTED, "a device-resident serving loop is running on this server");
    return true;
  }
  return false;
}
}  // namespace

extern "C" {

uint64_t vbh_serve_now_ns(void) { return now_ns(); }

vbh_status vbh_serve_create(vbh_handle* h, const vbh_serve_config* cfg, vbh_serve** out) {
  if (!h || !cfg || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (h->server) return fail(VBH_ERR_INVALID_ARG, "a server is already attached");
  vbh_serve_config c = *cfg;
  if (c.n_clients == 0 || c.n_clients > (1u << 20))
    return fail(VBH_ERR_INVALID_ARG, "n_clients must be in 1..2^20");
  vbh_status pst = check_policy(c);
  if (pst != VBH_OK) return pst;
  if (c.max_inflight == 0) c.max_inflight = 2;
  if (c.log_bits == 0) c.log_bits = 22;
  if (c.rem_bits == 0) c.rem_bits = 22;
  if (c.log_bits > 28 || c.rem_bits > 28 || (1ull << c.log_bits) < 4ull * h->cfg.max_blocks)
    return fail(VBH_ERR_INVALID_ARG, "log_bits must give >= 4 x max_blocks records (<= 2^28)");
  if ((c.budget_bytes & ~255ull) < (((uint64_t)kRecBytes * h->cfg.max_blocks + 255u) & ~255ull))
    return fail(VBH_ERR_INVALID_ARG, "budget_bytes must hold a full model (528 B x max_blocks)");
  vbh_serve* s = new vbh_serve();
  s->h = h;
  s->cfg = c;
  s->log_cap = 1u << c.log_bits;
  auto bail = [&](vbh_status e) {
    vbh_serve_destroy(s);
    return e;
  };
#define SERVE_CUDA(call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      fail(VBH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return bail(VBH_ERR_CUDA);                                                      \
    }                                                                                 \
  } while (0)
  const unsigned int nb = h->cfg.max_blocks;
  const size_t rem_n = (size_t)1 << c.rem_bits;
  SERVE_CUDA(cudaMalloc(&s->log, sizeof(LogEnt) * (size_t)s->log_cap));
  SERVE_CUDA(cudaMalloc(&s->store, (size_t)nb * kRecPayload));
  SERVE_CUDA(cudaMalloc(&s->rem_keys, sizeof(unsigned long long) * rem_n));
  SERVE_CUDA(cudaMalloc(&s->rem_seq, sizeof(unsigned int) * rem_n));
  SERVE_CUDA(cudaMalloc(&s->client_v, sizeof(unsigned int) * c.n_clients));
  SERVE_CUDA(cudaMalloc(&s->rec_count, sizeof(unsigned int) * kServeMaxBatch));
  SERVE_CUDA(cudaMalloc(&s->slot_err, sizeof(unsigned int) * kServeMaxBatch));
  SERVE_CUDA(cudaMalloc(&s->tiles_done, sizeof(unsigned int) * kServeMaxBatch));
  SERVE_CUDA(cudaMalloc(&s->scratch, 2 * sizeof(unsigned int)));
  SERVE_CUDA(cudaMalloc(&s->sl_dev, sizeof(ServeLog)));
  SERVE_CUDA(cudaMalloc(&s->arena, c.budget_bytes));
  SERVE_CUDA(cudaHostAlloc(&s->sigma_host, sizeof(unsigned int), cudaHostAllocMapped));
  SERVE_CUDA(cudaHostGetDevicePointer((void**)&s->sigma_dev, s->sigma_host, 0));
  SERVE_CUDA(cudaHostAlloc(&s->done_host, sizeof(uint4) * kServeMaxBatch, cudaHostAllocMapped));
  SERVE_CUDA(cudaHostGetDevicePointer((void**)&s->done_dev, s->done_host, 0));
  *s->sigma_host = 0u;
  std::memset(s->done_host, 0, sizeof(uint4) * kServeMaxBatch);
  cudaStream_t st = h->stream;
  SERVE_CUDA(cudaMemsetAsync(s->log, 0, sizeof(LogEnt) * (size_t)s->log_cap, st));
  SERVE_CUDA(cudaMemsetAsync(s->rem_keys, 0xFF, sizeof(unsigned long long) * rem_n, st));
  SERVE_CUDA(cudaMemsetAsync(s->rem_seq, 0, sizeof(unsigned int) * rem_n, st));
  SERVE_CUDA(cudaMemsetAsync(s->client_v, 0, sizeof(unsigned int) * c.n_clients, st));
  SERVE_CUDA(cudaMemsetAsync(s->rec_count, 0, sizeof(unsigned int) * kServeMaxBatch, st));
  SERVE_CUDA(cudaMemsetAsync(s->slot_err, 0, sizeof(unsigned int) * kServeMaxBatch, st));
  SERVE_CUDA(cudaMemsetAsync(s->tiles_done, 0, sizeof(unsigned int) * kServeMaxBatch, st));
  SERVE_CUDA(cudaMemsetAsync(h->seq, 0, sizeof(unsigned int) * nb, st));
  ServeLog L{};
  L.log = s->log;
  L.store = s->store;
  L.rem_keys = s->rem_keys;
  L.rem_seq = s->rem_seq;
  L.sigma_host = s->sigma_dev;
  L.log_mask = s->log_cap - 1u;
  L.rem_mask = (unsigned int)(rem_n - 1u);
  L.seq_next = 1u;
  SERVE_CUDA(cudaMemcpyAsync(s->sl_dev, &L, sizeof L, cudaMemcpyHostToDevice, st));
  int occ = 0;
  SERVE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve_extract, kServeThreads, 0));
  s->grid = std::max(1, occ) * h->L.sms;
  s->heap = new Arena(c.budget_bytes);
  s->v_mirror.assign(c.n_clients, 0u);
  s->client_busy.assign(c.n_clients, 0);
  s->slot_req.assign(kServeMaxBatch, -1);
  h->slog = s->sl_dev;
  h->server = s;
  vbh_status rst = refresh_all_blocks(h, s->scratch);
  if (rst != VBH_OK) return bail(rst);
  SERVE_CUDA(cudaStreamSynchronize(st));
#undef SERVE_CUDA
  *out = s;
  return VBH_OK;
}

vbh_status vbh_serve_destroy(vbh_serve* s) {
  if (!s) return VBH_OK;
  if (s->loop) vbh_serve_loop_stop(s->loop);
  if (s->h) {
    cudaStreamSynchronize(s->h->stream);
    if (s->h->server == s) {
      s->h->server = nullptr;
      s->h->slog = nullptr;
    }
  }
  for (auto& I : s->inflight) cudaEventDestroy(I.ev);
  for (auto e : s->ev_free) cudaEventDestroy(e);
  void* ptrs[] = {s->log, s->store, s->rem_keys, s->rem_seq, s->client_v, s->rec_count,
                  s->slot_err, s->tiles_done, s->scratch, s->sl_dev, s->arena};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->sigma_host) cudaFreeHost(s->sigma_host);
  if (s->done_host) cudaFreeHost(s->done_host);
  delete s->heap;
  delete s;
  return VBH_OK;
}

vbh_status vbh_serve_set_policy(vbh_serve* s, const vbh_serve_config* cfg) {
  if (!s || !cfg) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  VBH_CUDA(cudaStreamSynchronize(s->h->stream));   // retire launches whose requests are done
  vbh_status rs = s->reap();
  if (rs != VBH_OK) return rs;
  if (!s->pending.empty() || !s->inflight.empty() ||
      std::any_of(s->slot_req.begin(), s->slot_req.end(), [](int r) { return r >= 0; }))
    return fail(VBH_ERR_INVALID_ARG, "server is not idle");
  vbh_status st = check_policy(*cfg);
  if (st != VBH_OK) return st;
  s->cfg.max_batch = cfg->max_batch;
  s->cfg.chunk_records = cfg->chunk_records;
  s->cfg.iter_records = cfg->iter_records;
  s->cfg.max_inflight = cfg->max_inflight ? cfg->max_inflight : 2;
  s->cfg.bypass_iters = cfg->bypass_iters;
  return VBH_OK;
}

vbh_status vbh_serve_set_versions(vbh_serve* s, const uint32_t* clients, const uint32_t* versions,
                                  uint32_t n) {
  if (!s || (n && (!clients || !versions))) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  for (uint32_t i = 0; i < n; ++i) {
    if (clients[i] >= s->cfg.n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
    if (s->client_busy[clients[i]]) return fail(VBH_ERR_INVALID_ARG, "client has a request");
  }
  for (uint32_t i = 0; i < n; ++i) s->v_mirror[clients[i]] = versions[i];
  VBH_CUDA(cudaStreamSynchronize(s->h->stream));
  VBH_CUDA(cudaMemcpy(s->client_v, s->v_mirror.data(), sizeof(unsigned int) * s->cfg.n_clients,
                      cudaMemcpyHostToDevice));
  return VBH_OK;
}

vbh_status vbh_serve_get_versions(vbh_serve* s, uint32_t* versions) {
  if (!s || !versions) return fail(VBH_ERR_INVALID_ARG, "null argument");
  VBH_CUDA(cudaStreamSynchronize(s->h->stream));
  VBH_CUDA(cudaMemcpy(versions, s->client_v, sizeof(unsigned int) * s->cfg.n_clients,
                      cudaMemcpyDeviceToHost));
  return VBH_OK;
}

vbh_status vbh_serve_versions_for_backlog(vbh_serve* s, const uint32_t* backlog, uint32_t n,
                                          uint32_t* versions) {
  if (!s || (n && (!backlog || !versions))) return fail(VBH_ERR_INVALID_ARG, "null argument");
  vbh_handle* h = s->h;
  const unsigned int nb = h->cfg.max_blocks;
  unsigned int* d = nullptr;
  VBH_CUDA(cudaMalloc(&d, sizeof(unsigned int) * (nb + 1u)));
  cudaMemsetAsync(d + nb, 0, sizeof(unsigned int), h->stream);
  k_live_seq<<<h->L.sms * 4, 256, 0, h->stream>>>(h->pkeys, h->seq, nb, d, d + nb);
  std::vector<unsigned int> seqs(nb + 1u);
  cudaError_t e = cudaMemcpyAsync(seqs.data(), d, sizeof(unsigned int) * (nb + 1u),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(VBH_ERR_CUDA, cudaGetErrorString(e));
  const unsigned int m = seqs[nb];
  seqs.resize(m);
  std::sort(seqs.begin(), seqs.end(), std::greater<unsigned int>());
  for (uint32_t i = 0; i < n; ++i)
    versions[i] = backlog[i] < m ? seqs[backlog[i]] : 0u;
  return VBH_OK;
}

vbh_status vbh_serve_submit(vbh_serve* s, uint32_t client, uint64_t t_arrival_ns, uint32_t* id) {
  if (!s) return fail(VBH_ERR_INVALID_ARG, "null server");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  if (client >= s->cfg.n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
  Req r;
  r.d.id = s->next_id++;
  if (s->next_id == 0) s->next_id = 1;
  r.d.client = client;
  r.d.t_arrival_ns = t_arrival_ns ? t_arrival_ns : now_ns();
  s->pending.push_back(r.d.id);
  s->reqs.emplace(r.d.id, r);
  if (id) *id = r.d.id;
  return VBH_OK;
}

vbh_status vbh_serve_step(vbh_serve* s, uint32_t* launched) {
  if (!s) return fail(VBH_ERR_INVALID_ARG, "null server");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  if (launched) *launched = 0;
  vbh_status st = s->reap();
  if (st != VBH_OK) return st;
  if (s->inflight.size() >= s->cfg.max_inflight) return VBH_OK;
  s->admit();
  const uint64_t it0 = s->st.iterations;
  st = s->launch();
  if (launched) *launched = (uint32_t)(s->st.iterations - it0);
  return st;
}

vbh_status vbh_serve_poll(vbh_serve* s, vbh_serve_done* out, uint32_t cap, uint32_t* n) {
  if (!s || !n || (cap && !out)) return fail(VBH_ERR_INVALID_ARG, "null argument");
  uint32_t k = 0;
  while (k < cap && !s->completed.empty()) {
    out[k++] = s->reqs[s->completed.front()].d;
    s->completed.pop_front();
  }
  *n = k;
  return VBH_OK;
}

vbh_status vbh_serve_result(vbh_serve* s, uint32_t id, vbh_serve_view* out) {
  if (!s || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != kDone)
    return fail(VBH_ERR_INVALID_ARG, "no completed request with this id");
  const Req& r = it->second;
  out->n_records = r.d.n_records;
  out->flags = r.d.flags;
  if (r.bytes) {
    out->recs_dev = reinterpret_cast<const int32_t*>(s->arena + r.off);
    out->indices_dev = s->arena + r.off + (size_t)r.cap * kRecHeader;
  } else {
    out->recs_dev = nullptr;
    out->indices_dev = nullptr;
  }
  return VBH_OK;
}

vbh_status vbh_serve_release(vbh_serve* s, uint32_t id) {
  if (!s) return fail(VBH_ERR_INVALID_ARG, "null server");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != kDone)
    return fail(VBH_ERR_INVALID_ARG, "no completed request with this id");
  if (it->second.bytes) s->heap->release(it->second.off, it->second.bytes);
  s->st.bytes_in_use = s->heap->used();
  s->reqs.erase(it);
  return VBH_OK;
}

vbh_status vbh_serve_drain(vbh_serve* s) {
  if (!s) return fail(VBH_ERR_INVALID_ARG, "null server");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  for (uint64_t guard = 0;; ++guard) {
    const bool busy = !s->pending.empty() || !s->inflight.empty() || !s->active.empty();
    if (!busy) break;
    if (guard > (1ull << 26)) return fail(VBH_ERR_TIMEOUT, "serve drain made no progress");
    const size_t pend = s->pending.size();
    const uint64_t it0 = s->st.iterations;
    vbh_status st = vbh_serve_step(s, nullptr);
    if (st != VBH_OK) return st;
    if (s->st.iterations == it0 && !s->inflight.empty()) {
      VBH_CUDA(cudaEventSynchronize(s->inflight.front().ev));
    } else if (s->st.iterations == it0 && s->inflight.empty() && s->active.empty() &&
               s->pending.size() == pend && pend) {
      return fail(VBH_ERR_CAPACITY, "pending requests cannot be admitted (budget held)");
    }
  }
  return VBH_OK;
}

vbh_status vbh_serve_stats_read(vbh_serve* s, vbh_serve_stats* out) {
  if (!s || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  ServeLog L;
  VBH_CUDA(cudaStreamSynchronize(s->h->stream));
  VBH_CUDA(cudaMemcpy(&L, s->sl_dev, sizeof L, cudaMemcpyDeviceToHost));
  s->st.err_flags = L.err;
  s->st.sigma = s->sigma();
  *out = s->st;
  return VBH_OK;
}

vbh_status vbh_serve_run(vbh_serve* s, const vbh_serve_script* sc, vbh_serve_done* out,
                         uint32_t cap, uint32_t* n_out) {
  if (!s || !sc || !n_out || (sc->n_events && (!sc->t_ns || !sc->client)))
    return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (loop_owned(s)) return VBH_ERR_UNSUPPORTED;
  *n_out = 0;
  uint32_t n_frames = 0;
  for (uint32_t i = 0; i < sc->n_events; ++i) {
    if (sc->client[i] < 0) ++n_frames;
    else if ((uint32_t)sc->client[i] >= s->cfg.n_clients)
      return fail(VBH_ERR_INVALID_ARG, "client out of range");
    if (i && sc->t_ns[i] < sc->t_ns[i - 1]) return fail(VBH_ERR_INVALID_ARG, "events not sorted");
  }
  if (n_frames && (!sc->depth_dev || !sc->T_wc || !sc->frame_id || !sc->frame_out))
    return fail(VBH_ERR_INVALID_ARG, "frame events need depth, poses, ids and an output");
  const uint64_t t0 = now_ns();
  uint32_t ev = 0, fr = 0, k = 0;
  std::vector<vbh_serve_done> buf(64);
  for (;;) {
    const uint64_t t = now_ns() - t0;
    while (ev < sc->n_events && sc->t_ns[ev] <= t) {
      vbh_status st;
      if (sc->client[ev] < 0) {
        st = vbh_process_frame(s->h, sc->depth_dev[fr], sc->T_wc + 12u * fr, sc->frame_id[fr],
                               sc->erase_radius, sc->frame_out);
        ++fr;
      } else {
        st = vbh_serve_submit(s, (uint32_t)sc->client[ev], t0 + sc->t_ns[ev], nullptr);
      }
      if (st != VBH_OK) return st;
      ++ev;
    }
    vbh_status st = vbh_serve_step(s, nullptr);
    if (st != VBH_OK) return st;
    uint32_t got = 0;
    do {
      st = vbh_serve_poll(s, buf.data(), (uint32_t)buf.size(), &got);
      if (st != VBH_OK) return st;
      for (uint32_t i = 0; i < got; ++i) {
        if (k < cap && out) out[k] = buf[i];
        ++k;
        st = vbh_serve_release(s, buf[i].id);
        if (st != VBH_OK) return st;
      }
    } while (got == buf.size());
    if (ev == sc->n_events && s->pending.empty() && s->inflight.empty() && s->active.empty())
      break;
  }
  *n_out = std::min(k, cap);
  return VBH_OK;
}

}  // extern "C"
