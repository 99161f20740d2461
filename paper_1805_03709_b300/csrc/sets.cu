// Per-client stream sets -- the paper's own serving design (Sec. 4.2), built beside the
// version-based server for comparison: every exploration client has a hash set of the MC blocks
// queued for it; the blocks a frame refreshes (and the keys it removes) are inserted into every
// client's set; a (re)connecting client's set is filled with every live block; a request takes a
// random subset of at most its size limit out of its set by concurrent removal, and the blocks'
// MC indices (or removal records) are copied out.
//
// Layout: one open-addressed table of packed block keys per client (capacity S, a power of
// two; EMPTY / TOMB sentinels as in the block table), linear probing from hash_mix(key).
// Inserts and removals run in separate launches.  An insert item (client, key) scans the probe
// sequence to the first EMPTY (the key already queued: nothing to do) and claims the first
// TOMB or that EMPTY with a CAS (a lost CAS retries; keys are distinct within one launch, so a
// key is never inserted twice).  A fetch is one CTA per request: 8 consecutive slots per
// thread and round from a random start, each queued key takes a ticket and the first `limit` tickets remove their key
// (CAS to TOMB) into a shared list; the keys are then looked up in the block table and each
// block's 512 B of dense indices is copied from the serving store (one warp per block).
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.cuh"

namespace vbh {

namespace {

constexpr int kSetThreads = 256;
constexpr unsigned int kMaxLimit = 1024;   // largest request (the paper's packages: 128-1024)

struct SetView {
  unsigned long long* keys;   // n_clients x cap
  unsigned int* count;        // queued keys per client
  unsigned int* tombs;        // tombstones per client
  unsigned int cap;           // slots per client (power of two)
  unsigned int* err;          // bit0: a set was full
};

// Item i: client client0 + i / n, key j = i % n of the source -- the last extraction's
// refreshed pool entries then its removal keys, or (all_live) every pool entry, or (list) keys.
__global__ void __launch_bounds__(kSetThreads) k_sets_insert(SetView S, PoolView pool,
                                                             const unsigned int* mset,
                                                             const unsigned int* n_mset,
                                                             const unsigned long long* tombrec,
                                                             const unsigned int* n_tombrec,
                                                             const unsigned long long* list,
                                                             const unsigned int* n_list,
                                                             unsigned int client0,
                                                             unsigned int n_clients,
                                                             int all_live) {
  const unsigned int nm = list ? *n_list : (all_live ? pool.max_blocks : *n_mset);
  const unsigned int nt = (list || all_live) ? 0u : *n_tombrec;
  const unsigned long long n = (unsigned long long)nm + nt;
  const unsigned long long total = n * n_clients;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned int mask = S.cap - 1u;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       i < total; i += stride) {
    const unsigned int c = client0 + (unsigned int)(i / n);
    const unsigned int j = (unsigned int)(i % n);
    unsigned long long key;
    if (list) key = list[j];
    else if (all_live) key = pool.pkeys[j];
    else key = j < nm ? pool.pkeys[mset[j]] : tombrec[j - nm];
    if (key == kEmpty) continue;
    unsigned long long* T = S.keys + (size_t)c * S.cap;
    bool done = false;
    for (int attempt = 0; attempt < 16 && !done; ++attempt) {
      unsigned int h = hash_mix(key) & mask, free_at = kNone;
      unsigned long long free_was = kEmpty;
      bool present = false;
      for (unsigned int probe = 0; probe <= mask; ++probe, h = (h + 1u) & mask) {
        const unsigned long long v = __ldcg(T + h);
        if (v == key) { present = true; break; }
        if (v == kTomb && free_at == kNone) { free_at = h; free_was = kTomb; }
        if (v == kEmpty) {
          if (free_at == kNone) { free_at = h; free_was = kEmpty; }
          break;
        }
      }
      if (present || free_at == kNone) {   // queued already, or the set is full
        if (!present) atomicOr(S.err, 1u);
        done = true;
      } else if (atomicCAS(T + free_at, free_was, key) == free_was) {
        atomicAdd(S.count + c, 1u);
        if (free_was == kTomb) atomicSub(S.tombs + c, 1u);
        done = true;
      }
    }
    if (!done) atomicOr(S.err, 1u);
  }
}

struct FetchReq {
  unsigned int client, limit, start, pad;
  unsigned long long out;     // first record of this request in the output
};

__global__ void __launch_bounds__(kSetThreads) k_sets_fetch(SetView S, TableView t,
                                                            PoolView pool, const ServeLog* sl,
                                                            const FetchReq* reqs,
                                                            int4* out_hdr, uint4* out_pay,
                                                            unsigned int* out_n) {
  __shared__ unsigned int s_tickets, s_taken;
  __shared__ unsigned long long s_keys[kMaxLimit];
  __shared__ unsigned int s_q[kMaxLimit];
  const FetchReq R = reqs[blockIdx.x];
  const unsigned int limit = min(R.limit, kMaxLimit);
  if (threadIdx.x == 0) {
    s_tickets = 0;
    s_taken = 0;
  }
  __syncthreads();
  unsigned long long* T = S.keys + (size_t)R.client * S.cap;
  const unsigned int mask = S.cap - 1u;
  // selection: concurrent removal of up to `limit` queued keys, scanning from a random start
  // (a multiple of 8); a thread takes 8 consecutive slots (four 16 B loads) per round
  constexpr unsigned int kRound = 8u * kSetThreads;
  const unsigned int start = R.start & ~7u;
  for (unsigned int base = 0; base < S.cap; base += kRound) {
    const unsigned int h0 = (start + base + 8u * threadIdx.x) & mask;
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(T + h0);
    ulonglong2 w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = __ldcg(src + i);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const unsigned long long v = (i & 1) ? w[i >> 1].y : w[i >> 1].x;
      if (v != kEmpty && v != kTomb) {
        const unsigned int ticket = atomicAdd(&s_tickets, 1u);
        if (ticket < limit && atomicCAS(T + h0 + i, v, kTomb) == v) {
          const unsigned int r = atomicAdd(&s_taken, 1u);
          s_keys[r] = v;
        }
      }
    }
    __syncthreads();
    if (s_tickets >= limit) break;   // uniform: every thread reads it after the barrier
    __syncthreads();
  }
  __syncthreads();
  const unsigned int n = s_taken;
  // headers: the block's frame version if live, else a removal record
  for (unsigned int r = threadIdx.x; r < n; r += blockDim.x) {
    const unsigned long long key = s_keys[r];
    unsigned int val;
    const unsigned int pos = thread_find(t, key, &val);
    const unsigned int q = pos != kNone ? val : kNone;
    s_q[r] = q;
    const int3 k = unpack_key(key);
    const unsigned int info = q != kNone ? (pool.version[q] & 0x7FFFFFFFu) : 0x80000000u;
    out_hdr[R.out + r] = make_int4(k.x, k.y, k.z, (int)info);
  }
  __syncthreads();
  const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (unsigned int r = warp; r < n; r += kSetThreads / 32) {
    const unsigned int q = s_q[r];
    if (q != kNone) out_pay[(R.out + r) * 32ull + lane] = sl->store[32ull * q + lane];
  }
  if (threadIdx.x == 0) {
    if (n) {
      atomicSub(S.count + R.client, n);
      atomicAdd(S.tombs + R.client, n);
    }
    out_n[blockIdx.x] = n;
  }
}

// live keys of one client's set into a list (for a rebuild without tombstones)
__global__ void k_sets_collect(SetView S, unsigned int c, unsigned long long* list,
                               unsigned int* n_list) {
  const unsigned long long* T = S.keys + (size_t)c * S.cap;
  for (unsigned int h = blockIdx.x * blockDim.x + threadIdx.x; h < S.cap;
       h += gridDim.x * blockDim.x) {
    const unsigned long long v = T[h];
    const bool take = v != kEmpty && v != kTomb;
    const unsigned int k = warp_append(n_list, take, __activemask());
    if (take) list[k] = v;
  }
}

}  // namespace
}  // namespace vbh

using namespace vbh;

struct vbh_sets {
  vbh_serve* server = nullptr;
  vbh_handle* h = nullptr;
  SetView S{};
  unsigned int n_clients = 0;
  FetchReq* reqs_dev = nullptr;
  unsigned long long* list = nullptr;   // rebuild scratch (cap keys)
  unsigned int* n_list = nullptr;
  int grid = 0;
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  uint64_t next() {   // SplitMix64 steps for the random start of each fetch
    rng += 0x9E3779B97F4A7C15ull;
    uint64_t z = rng;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

extern "C" {

vbh_status vbh_sets_create(vbh_serve* s, uint32_t n_clients, uint32_t cap_log2, vbh_sets** out) {
  if (!s || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n_clients == 0 || n_clients > 4096 || cap_log2 < 11 || cap_log2 > 26)
    return fail(VBH_ERR_INVALID_ARG, "n_clients in 1..4096 and cap_log2 in 11..26");
  vbh_sets* q = new vbh_sets();
  q->server = s;
  q->h = serve_handle(s);
  q->n_clients = n_clients;
  q->S.cap = 1u << cap_log2;
  const size_t slots = (size_t)n_clients << cap_log2;
  cudaError_t e;
  if ((e = cudaMalloc(&q->S.keys, slots * 8)) != cudaSuccess ||
      (e = cudaMalloc(&q->S.count, 4ull * n_clients)) != cudaSuccess ||
      (e = cudaMalloc(&q->S.tombs, 4ull * n_clients)) != cudaSuccess ||
      (e = cudaMalloc(&q->S.err, 4)) != cudaSuccess ||
      (e = cudaMalloc(&q->reqs_dev, sizeof(FetchReq) * 4096)) != cudaSuccess ||
      (e = cudaMalloc(&q->list, 8ull * q->S.cap)) != cudaSuccess ||
      (e = cudaMalloc(&q->n_list, 4)) != cudaSuccess) {
    vbh_sets_destroy(q);
    return fail(VBH_ERR_CUDA, std::string("vbh_sets_create: ") + cudaGetErrorString(e));
  }
  cudaStream_t st = q->h->stream;
  cudaMemsetAsync(q->S.keys, 0xFF, slots * 8, st);
  cudaMemsetAsync(q->S.count, 0, 4ull * n_clients, st);
  cudaMemsetAsync(q->S.tombs, 0, 4ull * n_clients, st);
  cudaMemsetAsync(q->S.err, 0, 4, st);
  q->grid = q->h->L.sms * 8;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
    vbh_sets_destroy(q);
    return fail(VBH_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = q;
  return VBH_OK;
}

vbh_status vbh_sets_destroy(vbh_sets* q) {
  if (!q) return VBH_OK;
  if (q->h) cudaStreamSynchronize(q->h->stream);
  for (void* p : {(void*)q->S.keys, (void*)q->S.count, (void*)q->S.tombs, (void*)q->S.err,
                  (void*)q->reqs_dev, (void*)q->list, (void*)q->n_list})
    if (p) cudaFree(p);
  delete q;
  return VBH_OK;
}

vbh_status vbh_sets_insert_last(vbh_sets* q) {
  if (!q) return fail(VBH_ERR_INVALID_ARG, "null sets");
  vbh_handle* h = q->h;
  k_sets_insert<<<q->grid, kSetThreads, 0, h->stream>>>(q->S, h->pool(), h->mset, &h->cnt->n_mset,
                                                        h->tombrec, &h->cnt->n_tombrec, nullptr,
                                                        nullptr, 0u, q->n_clients, 0);
  h->launches += 1;
  VBH_CUDA(cudaGetLastError());
  return VBH_OK;
}

vbh_status vbh_sets_fill(vbh_sets* q, uint32_t client) {
  if (!q) return fail(VBH_ERR_INVALID_ARG, "null sets");
  if (client >= q->n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
  vbh_handle* h = q->h;
  k_sets_insert<<<q->grid, kSetThreads, 0, h->stream>>>(q->S, h->pool(), nullptr, nullptr,
                                                        nullptr, nullptr, nullptr, nullptr,
                                                        client, 1u, 1);
  h->launches += 1;
  VBH_CUDA(cudaGetLastError());
  return VBH_OK;
}

vbh_status vbh_sets_fetch(vbh_sets* q, const uint32_t* clients_host, const uint32_t* limits_host,
                          uint32_t n_req, int32_t* recs_dev, uint8_t* indices_dev,
                          uint32_t* n_out_dev) {
  if (!q) return fail(VBH_ERR_INVALID_ARG, "null sets");
  if (n_req == 0) return VBH_OK;
  if (!clients_host || !limits_host || !recs_dev || !indices_dev || !n_out_dev || n_req > 4096)
    return fail(VBH_ERR_INVALID_ARG, "null argument or more than 4096 requests");
  std::vector<FetchReq> r(n_req);
  std::vector<char> seen(q->n_clients, 0);
  unsigned long long off = 0;
  for (uint32_t i = 0; i < n_req; ++i) {
    if (clients_host[i] >= q->n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
    if (seen[clients_host[i]]++) return fail(VBH_ERR_INVALID_ARG, "a client twice in one fetch");
    if (limits_host[i] == 0 || limits_host[i] > kMaxLimit)
      return fail(VBH_ERR_INVALID_ARG, "limits must be in 1..1024");
    r[i].client = clients_host[i];
    r[i].limit = limits_host[i];
    r[i].start = (unsigned int)q->next() & (q->S.cap - 1u);
    r[i].out = off;
    off += limits_host[i];
  }
  vbh_handle* h = q->h;
  VBH_CUDA(cudaMemcpyAsync(q->reqs_dev, r.data(), sizeof(FetchReq) * n_req,
                           cudaMemcpyHostToDevice, h->stream));
  k_sets_fetch<<<n_req, kSetThreads, 0, h->stream>>>(q->S, h->table(), h->pool(),
                                                     serve_log(q->server), q->reqs_dev,
                                                     reinterpret_cast<int4*>(recs_dev),
                                                     reinterpret_cast<uint4*>(indices_dev),
                                                     n_out_dev);
  h->launches += 1;
  VBH_CUDA(cudaGetLastError());
  return VBH_OK;
}

vbh_status vbh_sets_counts(vbh_sets* q, uint32_t* queued_host, uint32_t* tombs_host,
                           uint32_t* err_host) {
  if (!q) return fail(VBH_ERR_INVALID_ARG, "null sets");
  VBH_CUDA(cudaStreamSynchronize(q->h->stream));
  if (queued_host)
    VBH_CUDA(cudaMemcpy(queued_host, q->S.count, 4ull * q->n_clients, cudaMemcpyDeviceToHost));
  if (tombs_host)
    VBH_CUDA(cudaMemcpy(tombs_host, q->S.tombs, 4ull * q->n_clients, cudaMemcpyDeviceToHost));
  if (err_host) VBH_CUDA(cudaMemcpy(err_host, q->S.err, 4, cudaMemcpyDeviceToHost));
  return VBH_OK;
}

vbh_status vbh_sets_rebuild(vbh_sets* q, uint32_t client) {
  if (!q) return fail(VBH_ERR_INVALID_ARG, "null sets");
  if (client >= q->n_clients) return fail(VBH_ERR_INVALID_ARG, "client out of range");
  vbh_handle* h = q->h;
  cudaStream_t st = h->stream;
  VBH_CUDA(cudaMemsetAsync(q->n_list, 0, 4, st));
  k_sets_collect<<<h->L.sms * 4, 256, 0, st>>>(q->S, client, q->list, q->n_list);
  VBH_CUDA(cudaMemsetAsync(q->S.keys + (size_t)client * q->S.cap, 0xFF, 8ull * q->S.cap, st));
  VBH_CUDA(cudaMemsetAsync(q->S.count + client, 0, 4, st));
  VBH_CUDA(cudaMemsetAsync(q->S.tombs + client, 0, 4, st));
  k_sets_insert<<<q->grid, kSetThreads, 0, st>>>(q->S, h->pool(), nullptr, nullptr, nullptr,
                                                 nullptr, q->list, q->n_list, client, 1u, 0);
  h->launches += 2;
  VBH_CUDA(cudaGetLastError());
  return VBH_OK;
}

}  // extern "C"
