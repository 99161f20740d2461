// C ABI of libvbh (declared in include/vbh.h): handle lifetime, device memory, the ordering of
// the launches of each call, timing and counters.  No entry point calls into PyTorch; all
// compute runs in the kernels of hash.cu, frame.cu, erase.cu and mc.cu.
#include <unistd.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace vbh;

namespace vbh {

thread_local std::string g_last_error;

vbh_status fail(vbh_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

}  // namespace vbh


namespace {

vbh_status check_launch(vbh_handle* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VBH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  (void)h;
  return VBH_OK;
}

__global__ void k_init_pool(unsigned int* stack, unsigned int n) {
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    stack[i] = n - 1u - i;
}

// Stores the per-call control block and zeroes the counters the call accumulates into.
__global__ void k_setup(FrameCtl c, FrameCtl* dst, DevCounters* cnt) {
  if (threadIdx.x != 0) return;
  *dst = c;
  if (c.reset & kResetFrame) {
    cnt->n_cand = 0;
    cnt->n_touched = 0;
    cnt->n_new = 0;
    cnt->vox_updated = 0ull;
  }
  if (c.reset & kResetErase) cnt->n_erased = 0;
  if (c.reset & kResetMset) {
    cnt->n_mset = 0;
    cnt->n_tombrec = 0;
    if (c.n_entries_dev) *c.n_entries_dev = 0;
  }
}

// Frames the host may have queued on the GPU (vbh_process_frame waits beyond that).  With
// stream-out on, the host must drain the device ring of removed blocks, and it sees the ring's
// head only for frames that have run: it therefore lets at most kStreamOutAhead frames wait on
// the GPU, so that its view of the head is never more than these frames old (the ring keeps a
// quarter of its capacity free for them).
constexpr unsigned int kMaxAhead = 64;
constexpr unsigned int kStreamOutAhead = 3;

// Root node of the frame graph: the control block arrives by value (vbh_process_frame patches
// this node's argument before each launch, so the graph reads no host memory), is stored for
// the other kernels, the per-frame counters are zeroed and the frame's sequence number is
// reported to mapped host memory (the host's bound on queued frames).
__global__ void k_setup_frame(const FrameCtl c, unsigned long long seq,
                              unsigned long long* consumed, FrameCtl* dst, DevCounters* cnt) {
  *dst = c;
  cnt->n_cand = 0;
  cnt->n_touched = 0;
  cnt->n_new = 0;
  cnt->vox_updated = 0ull;
  cnt->n_erased = 0;
  cnt->n_mset = 0;
  cnt->n_tombrec = 0;
  if (c.n_entries_dev) *c.n_entries_dev = 0;
  // only a bound on the frames the host queues: no ordering with the writes above is needed
  *reinterpret_cast<volatile unsigned long long*>(consumed) = seq + 1;
}

// Non-blocking view of the counters: a copy enqueued on a side stream after each call, read by
// the next call if it has landed.  Used only for the tombstone clean-up heuristic.
void snapshot_counters(vbh_handle* h) {
  if (h->snap_pending) return;
  cudaEvent_t e = h->get_event();
  cudaEventRecord(e, h->stream);
  cudaStreamWaitEvent(h->side, e, 0);
  cudaMemcpyAsync(h->snap, h->cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->side);
  cudaEventRecord(h->snap_ev, h->side);
  h->ev_free.push_back(e);
  h->snap_pending = true;
}

vbh_status rebuild(vbh_handle* h) {
  const size_t bytes = (size_t)h->n_slots * sizeof(Slot);
  VBH_CUDA(cudaMemcpyAsync(h->shadow, h->slots, bytes, cudaMemcpyDeviceToDevice, h->stream));
  VBH_CUDA(cudaMemsetAsync(h->slots, 0xFF, bytes, h->stream));
  launch_rebuild(h->L, h->table(), h->shadow, h->n_slots, h->cnt);
  h->launches += 2;
  h->rebuilds++;
  return check_launch(h, "rebuild");
}

void free_batch_lists(vbh_handle* h) {
  BatchLists& b = h->blists;
  for (void* q : {(void*)b.ins_idx, (void*)b.ins_key, (void*)b.era_idx, (void*)b.era_key})
    if (q) cudaFree(q);
  b = BatchLists{};
  h->blists_cap = 0;
}

vbh_status maybe_rebuild(vbh_handle* h) {
  if (h->snap_pending && cudaEventQuery(h->snap_ev) == cudaSuccess) {
    h->snap_pending = false;
    const unsigned int tomb = h->snap->n_tomb, empty = h->snap->n_empty;
    // a running serving loop finds keys while frames run: entries must not move under it
    if (!h->serve_loop_active && tomb > h->n_slots / 64u && tomb > (tomb + empty) / 2u)
      return rebuild(h);
  }
  return VBH_OK;
}

FrameParams frame_params(const vbh_handle* h, const float* T) {
  const vbh_config& c = h->cfg;
  FrameParams fp{};
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) fp.R[3 * i + j] = T ? T[4 * i + j] : (i == j ? 1.f : 0.f);
    fp.t[i] = T ? T[4 * i + 3] : 0.f;
  }
  fp.s = c.voxel_size;
  fp.mu = c.trunc;
  fp.inv_mu = 1.0f / c.trunc;
  fp.wmax = c.max_weight;
  fp.ds = c.depth_scale;
  fp.zmax = c.zmax;
  // The validity test of a raw depth r (nonzero, and fl(r ds) <= zmax when zmax > 0) as one
  // range: fl(r ds) never decreases with r (ds > 0), so the valid values are 1..raw_max.
  fp.raw_max = 65535u;
  if (c.zmax > 0.f) {
    auto within = [&](unsigned int r) {
      volatile float d = (float)r * c.depth_scale;   // binary32 product, as on the device
      return d <= c.zmax;
    };
    if (!within(65535u)) {
      unsigned int lo = 0, hi = 65535u;   // within(lo), !within(hi)
      while (hi - lo > 1u) {
        const unsigned int mid = (lo + hi) / 2u;
        (within(mid) ? lo : hi) = mid;
      }
      fp.raw_max = lo;
    }
  }
  fp.fx = c.fx;
  fp.fy = c.fy;
  fp.cx = c.cx;
  fp.cy = c.cy;
  // binary32 host arithmetic, one rounding per operation (these feed the canonical decisions)
  fp.cxh = c.cx + 0.5f;
  fp.cyh = c.cy + 0.5f;
  const float bs = 8.0f * c.voxel_size;
  fp.inv_bs = 1.0f / bs;
  fp.fw = (float)c.width;
  fp.fh = (float)c.height;
  fp.width = c.width;
  fp.height = c.height;
  fp.J = h->J;
  fp.wait_limit = h->wait_limit;
  return fp;
}

FrameCtl base_ctl(const vbh_handle* h, const float* T) {
  FrameCtl c{};
  c.fp = frame_params(h, T);
  c.version = h->frame_version;
  c.slog = h->slog;
  c.so_tail = stream_out_tail(h);
  return c;
}

void set_stream_out(FrameCtl& c, const vbh_mc_stream* out) {
  c.rec_keys3 = out->keys3;
  c.rec_info = out->info;
  c.rec_off = out->offsets;
  c.rec_cnt = out->counts;
  c.ent_local = out->local;
  c.ent_idx = out->index;
  c.n_blocks_dev = out->n_blocks_dev;
  c.n_entries_dev = out->n_entries_dev;
  c.cap_blocks = out->cap_blocks;
  c.cap_entries = out->cap_entries;
}

void launch_setup(vbh_handle* h, const FrameCtl& c) {
  k_setup<<<1, 32, 0, h->stream>>>(c, h->ctl, h->cnt);
  h->launches += 1;
}

bool stream_ok(const vbh_mc_stream* out) {
  return out && out->n_blocks_dev && out->n_entries_dev &&
         !(out->cap_blocks && (!out->keys3 || !out->info || !out->offsets || !out->counts)) &&
         !(out->cap_entries && (!out->local || !out->index));
}

void read_frame_stats(vbh_handle* h, const DevCounters& d, vbh_frame_stats* st) {
  st->touched = d.n_touched;
  st->new_blocks = d.n_new;
  st->candidates = d.n_cand;
  st->error_flags = d.err;
  (void)h;
}

}  // namespace

namespace vbh {

vbh_status refresh_all_blocks(vbh_handle* h, unsigned int* counts_dev) {
  FrameCtl c = base_ctl(h, nullptr);
  c.epoch_mset = h->next_epoch();
  c.reset = kResetMset;
  c.serve_mark = 1u;
  c.store_only = 1u;
  c.n_blocks_dev = counts_dev;
  c.n_entries_dev = counts_dev + 1;
  launch_setup(h, c);
  launch_mset_scan(h->L, h->pool(), h->cnt, h->mset, 0, 0u);
  launch_mc_extract(h->L, h->table(), h->pool(), h->cnt, h->ctl, h->mset, h->tombrec);
  h->launches += 2;
  return check_launch(h, "refresh_all_blocks");
}

}  // namespace vbh

extern "C" {

int vbh_abi_version(void) { return VBH_ABI_VERSION; }
const char* vbh_last_error(void) { return g_last_error.c_str(); }

uint32_t vbh_bucket_of(int32_t x, int32_t y, int32_t z, uint32_t n_buckets, uint32_t hash_fn) {
  if (n_buckets == 0 || (n_buckets & (n_buckets - 1u)) || !key_ok(x, y, z)) return VBH_NONE;
  return home_bucket(pack_key(x, y, z), n_buckets - 1u, hash_fn);
}

vbh_status vbh_create(const vbh_config* cfg, void* cuda_stream, vbh_handle** out) {
  if (!cfg || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const vbh_config& c = *cfg;
  if (c.n_buckets < 2 || (c.n_buckets & (c.n_buckets - 1u)) || c.n_buckets > (1u << 28))
    return fail(VBH_ERR_INVALID_ARG, "n_buckets must be a power of two in [2, 2^28]");
  if (c.slots_per_bucket != 4) return fail(VBH_ERR_INVALID_ARG, "slots_per_bucket must be 4");
  if (c.hash_fn > 1) return fail(VBH_ERR_INVALID_ARG, "unknown hash_fn");
  if (c.max_blocks > (1u << 26)) return fail(VBH_ERR_INVALID_ARG, "max_blocks above 2^26");
  if (c.max_blocks > 0) {
    if (!(c.voxel_size > 0.f) || !(c.trunc > 0.f) || !(c.max_weight >= 1.f) ||
        !(c.depth_scale > 0.f) || !(c.zmax >= 0.f) || c.width <= 0 || c.height <= 0 ||
        c.width > 16384 || c.height > 16384 || !(c.fx > 0.f) || !(c.fy > 0.f) ||
        !std::isfinite(c.cx) || !std::isfinite(c.cy))
      return fail(VBH_ERR_INVALID_ARG, "invalid camera / volume parameters");
  }
  vbh_handle* h = new vbh_handle();
  h->cfg = c;
  if (h->cfg.max_batch == 0) h->cfg.max_batch = 1u << 22;
  h->stream = (cudaStream_t)cuda_stream;
  auto bail = [&](vbh_status st) {
    vbh_destroy(h);
    return st;
  };
#define CREATE_CUDA(call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      fail(VBH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
      return bail(VBH_ERR_CUDA);                                                       \
    }                                                                                  \
  } while (0)
  CREATE_CUDA(cudaGetDevice(&h->device));
  int sms = 0;
  CREATE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  h->L = Launch{h->stream, sms};
  CREATE_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CREATE_CUDA(cudaEventCreateWithFlags(&h->snap_ev, cudaEventDisableTiming));
  h->n_slots = c.n_buckets * 4u;
  const size_t tbytes = (size_t)h->n_slots * sizeof(Slot);
  CREATE_CUDA(cudaMalloc(&h->slots, tbytes));
  CREATE_CUDA(cudaMalloc(&h->shadow, tbytes));
  CREATE_CUDA(cudaMemsetAsync(h->slots, 0xFF, tbytes, h->stream));
  CREATE_CUDA(cudaMalloc(&h->cnt, sizeof(DevCounters)));
  CREATE_CUDA(cudaMalloc(&h->ctl, sizeof(FrameCtl)));
  CREATE_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CREATE_CUDA(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
  for (auto& e : h->fork_ev) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  {
    unsigned long long* ch = nullptr;
    CREATE_CUDA(cudaHostAlloc(&ch, sizeof(unsigned long long), cudaHostAllocMapped));
    *ch = 0ull;
    h->consumed_host = ch;
    CREATE_CUDA(cudaHostGetDevicePointer((void**)&h->consumed_dev, ch, 0));
  }
  CREATE_CUDA(cudaMallocHost(&h->snap, sizeof(DevCounters)));
  DevCounters init{};
  init.free_top = (int)c.max_blocks;
  init.n_empty = h->n_slots;
  CREATE_CUDA(cudaMemcpyAsync(h->cnt, &init, sizeof init, cudaMemcpyHostToDevice, h->stream));
  const unsigned int nb = c.max_blocks;
  if (nb > 0) {
    CREATE_CUDA(cudaMalloc(&h->vox, (size_t)nb * 512 * sizeof(float2)));
    CREATE_CUDA(cudaMalloc(&h->masks, (size_t)nb * 32 * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->pkeys, (size_t)nb * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&h->state, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->mark, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->version, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->stack, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->seq, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMemsetAsync(h->seq, 0, (size_t)nb * sizeof(unsigned int), h->stream));
    CREATE_CUDA(cudaMemsetAsync(h->pkeys, 0xFF, (size_t)nb * sizeof(unsigned long long), h->stream));
    CREATE_CUDA(cudaMemsetAsync(h->state, 0, (size_t)nb * sizeof(unsigned int), h->stream));
    CREATE_CUDA(cudaMemsetAsync(h->mark, 0, (size_t)nb * sizeof(unsigned int), h->stream));
    CREATE_CUDA(cudaMemsetAsync(h->version, 0, (size_t)nb * sizeof(unsigned int), h->stream));
    CREATE_CUDA(cudaMemsetAsync(h->masks, 0, (size_t)nb * 32 * sizeof(unsigned int), h->stream));
    k_init_pool<<<sms * 4, 256, 0, h->stream>>>(h->stack, nb);
    CREATE_CUDA(cudaGetLastError());
    h->J = (int)std::ceil(2.0 * (double)c.trunc / (double)c.voxel_size - 1e-6);
    if (h->J < 0 || h->J > 4096) {
      fail(VBH_ERR_INVALID_ARG, "truncation / voxel size ratio out of range");
      return bail(VBH_ERR_INVALID_ARG);
    }
    h->cand_cap = (unsigned int)std::min<uint64_t>(
        (uint64_t)c.width * c.height * (uint64_t)(h->J + 1), 0xFFFFFFF0ull);
    CREATE_CUDA(cudaMalloc(&h->cand, (size_t)h->cand_cap * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&h->cand_res, (size_t)h->cand_cap * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->cand_st, (size_t)h->cand_cap));
    CREATE_CUDA(cudaMalloc(&h->dimg, (size_t)c.width * c.height * sizeof(float)));
    CREATE_CUDA(cudaMalloc(&h->touched, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->tdepth, (size_t)nb * sizeof(float2)));
    CREATE_CUDA(cudaMalloc(&h->tkey, (size_t)nb * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&h->mset, (size_t)nb * sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&h->removed, (size_t)nb * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&h->tombrec, (size_t)nb * sizeof(unsigned long long)));
  }
  CREATE_CUDA(cudaStreamSynchronize(h->stream));
#undef CREATE_CUDA
  *out = h;
  return VBH_OK;
}

vbh_status vbh_destroy(vbh_handle* h) {
  if (!h) return VBH_OK;
  if (h->server) vbh_serve_destroy(h->server);
  host_pipe_release(h);
  stream_out_release(h);
  if (h->stream || h->slots) cudaStreamSynchronize(h->stream);
  free_batch_lists(h);
  if (h->stream || h->slots) cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->frame_exec) cudaGraphExecDestroy(h->frame_exec);
  if (h->frame_graph) cudaGraphDestroy(h->frame_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->cap_stream2) cudaStreamDestroy(h->cap_stream2);
  for (cudaEvent_t e : h->fork_ev)
    if (e) cudaEventDestroy(e);
  if (h->consumed_host) cudaFreeHost((void*)h->consumed_host);
  void* ptrs[] = {h->ctl, h->slots, h->shadow, h->cnt, h->vox, h->masks, h->pkeys, h->state, h->mark,
                  h->version, h->stack, h->seq, h->cand, h->cand_res, h->cand_st, h->touched, h->tdepth, h->tkey, h->mset,
                  h->removed, h->tombrec, h->dimg};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->snap) cudaFreeHost(h->snap);
  for (auto& s : h->pending) {
    cudaEventDestroy(s.a);
    cudaEventDestroy(s.b);
  }
  for (auto e : h->ev_free) cudaEventDestroy(e);
  if (h->snap_ev) cudaEventDestroy(h->snap_ev);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;
  return VBH_OK;
}

vbh_status vbh_set_stream(vbh_handle* h, void* cuda_stream) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  h->stream = (cudaStream_t)cuda_stream;
  h->L.stream = h->stream;
  return VBH_OK;
}

// Plain-map batches up to this size run as one cooperative launch (latency-bound otherwise).
constexpr uint32_t kSmallBatchMax = 1u << 17;
#ifndef VBH_FINISH_ERASE
#define VBH_FINISH_ERASE 1   // a plain map's pending insert values and erases share a launch
#endif

vbh_status vbh_hash_batch(vbh_handle* h, const uint8_t* ops_dev, const int32_t* keys3_dev,
                          const uint32_t* vals_dev, uint32_t* results_dev, uint8_t* status_dev,
                          uint32_t n) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (n == 0) return VBH_OK;
  if (n > h->cfg.max_batch) return fail(VBH_ERR_INVALID_ARG, "batch larger than max_batch");
  if (!ops_dev || !keys3_dev || !results_dev || !status_dev)
    return fail(VBH_ERR_INVALID_ARG, "null device pointer");
  vbh_status st = maybe_rebuild(h);
  if (st != VBH_OK) return st;
  // a small batch of a plain map: one cooperative launch, one thread per op, no op lists
  const bool small = h->cfg.max_blocks == 0 && n <= kSmallBatchMax && small_batch_fits(h->L, n);
  if (!small && h->blists_cap < n) {   // the compacted insert / erase lists, grown to n
    VBH_CUDA(cudaStreamSynchronize(h->stream));
    free_batch_lists(h);
    BatchLists& b = h->blists;
    if (cudaMalloc(&b.ins_idx, sizeof(unsigned int) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&b.ins_key, sizeof(unsigned long long) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&b.era_idx, sizeof(unsigned int) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&b.era_key, sizeof(unsigned long long) * (size_t)n) != cudaSuccess) {
      free_batch_lists(h);
      return fail(VBH_ERR_CUDA, "vbh_hash_batch: device memory for the op lists");
    }
    h->blists_cap = n;
  }
  const TableView t = h->table();
  const PoolView pool = h->pool();
  h->stage_begin(VBH_STAGE_HASH);
  h->blists.n = h->cnt->op_lists[h->batch_parity];
  h->blists.n_next = h->cnt->op_lists[h->batch_parity ^ 1u];
  h->batch_parity ^= 1u;
  if (small) {
    VBH_CUDA(launch_hash_batch_small(h->L, t, h->cnt, ops_dev, keys3_dev, vals_dev, results_dev,
                                     status_dev, n, h->blists.n_next, &h->gbar_base));
    h->launches += 1;
  } else {
    launch_hash_find(h->L, t, h->cnt, ops_dev, keys3_dev, results_dev, status_dev, n,
                     h->blists);
    launch_hash_insert(h->L, t, pool, h->cnt, h->blists.ins_key,
                       h->blists.n + 1, vals_dev, results_dev, status_dev, n,
                       h->blists.ins_idx);
#if VBH_FINISH_ERASE
    if (h->cfg.max_blocks == 0) {   // a plain map: pending values and erases in one launch
      launch_hash_finish_erase(h->L, t, pool, h->cnt, results_dev, status_dev, n, h->blists);
      h->launches += 3;
    } else
#endif
    {
      launch_hash_insert_finish(h->L, t, pool, h->cnt, h->blists.n + 1, results_dev, status_dev,
                                n, nullptr, nullptr, nullptr, nullptr, nullptr,
                                h->blists.ins_idx);
      launch_hash_erase(h->L, t, pool, h->cnt, results_dev, status_dev, n, h->blists);
      h->launches += 4;
    }
  }
  h->stage_end();
  st = check_launch(h, "vbh_hash_batch");
  snapshot_counters(h);
  return st;
}

vbh_status vbh_set_integration_mode(vbh_handle* h, uint32_t mode) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (mode > VBH_INTEGRATE_VISIBLE) return fail(VBH_ERR_INVALID_ARG, "unknown integration mode");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  h->integ_mode = mode;   // the frame graph is captured again at the next frame
  return VBH_OK;
}

vbh_status vbh_hash_rebuild(vbh_handle* h) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->serve_loop_active)
    return fail(VBH_ERR_UNSUPPORTED, "a device-resident serving loop reads this table");
  return rebuild(h);
}

vbh_status vbh_integrate_frame(vbh_handle* h, const uint16_t* depth_dev, const float* T_wc_host,
                               uint32_t frame_id, vbh_frame_stats* stats_host) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (!depth_dev || !T_wc_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_wc_host[i])) return fail(VBH_ERR_INVALID_ARG, "non-finite pose");
  if (frame_id >= 0x80000000u) return fail(VBH_ERR_INVALID_ARG, "frame_id must be < 2^31");
  vbh_status st = maybe_rebuild(h);
  if (st != VBH_OK) return st;
  FrameCtl c = base_ctl(h, T_wc_host);
  c.fp.depth = depth_dev;
  c.epoch_touch = h->next_epoch();
  c.reset = kResetFrame;
  c.visible = h->integ_mode == VBH_INTEGRATE_VISIBLE;
  const TableView t = h->table();
  const PoolView pool = h->pool();
  h->stage_begin(VBH_STAGE_ALLOC);
  launch_setup(h, c);
  launch_alloc_keys(h->L, h->ctl, h->cfg.width, h->cfg.height, h->cand, h->cand_cap, h->cnt,
                    h->dimg);
  launch_hash_insert(h->L, t, pool, h->cnt, h->cand, &h->cnt->n_cand, nullptr,
                     h->cand_res, h->cand_st, h->cand_cap);
  launch_hash_insert_finish(h->L, t, pool, h->cnt, &h->cnt->n_cand, h->cand_res, h->cand_st,
                            h->cand_cap, h->touched, h->tkey, h->tdepth, &h->cnt->n_touched,
                            h->ctl);
  h->launches += 3;
  if (h->integ_mode == VBH_INTEGRATE_VISIBLE) {
    launch_visible(h->L, h->ctl, pool, h->touched, h->tkey, h->tdepth, &h->cnt->n_touched);
    h->launches += 1;
  }
  h->stage_end();
  h->stage_begin(VBH_STAGE_INTEGRATE);
  launch_integrate(h->L, c.fp, h->dimg, pool, h->touched, h->tkey, h->tdepth,
                   &h->cnt->n_touched,
                   h->cnt);
  h->launches += 1;
  h->stage_end();
  h->frame_version = frame_id;
  h->have_frame = true;
  st = check_launch(h, "vbh_integrate_frame");
  if (st != VBH_OK) return st;
  if (stats_host) {
    DevCounters d;
    VBH_CUDA(cudaMemcpyAsync(&d, h->cnt, sizeof d, cudaMemcpyDeviceToHost, h->stream));
    VBH_CUDA(cudaStreamSynchronize(h->stream));
    read_frame_stats(h, d, stats_host);
    if (d.err & (kErrPool | kErrTable)) return fail(VBH_ERR_CAPACITY, "block pool or table full");
    if (d.err & kErrTimeout)
      return fail(VBH_ERR_TIMEOUT, "a bounded device wait gave up (fusion's voxel copy)");
  }
  snapshot_counters(h);
  return VBH_OK;
}

// Capture erase + allocation + fusion + MC set + MC extraction of one frame as a CUDA graph.
// All per-frame inputs reach the kernels through the control block written by the root
// (setup) node, so a frame is: update that node's argument, launch the graph.
// `tmask`: stages (VBH_STAGE_INTEGRATE, VBH_STAGE_MC) bracketed by event-record nodes.
static vbh_status build_frame_graph(vbh_handle* h, int tmask) {
  if (h->frame_exec) cudaGraphExecDestroy(h->frame_exec);
  if (h->frame_graph) cudaGraphDestroy(h->frame_graph);
  h->frame_exec = nullptr;
  h->frame_graph = nullptr;
  for (auto& nd : h->ev_node) nd = nullptr;
  const Launch Lc{h->cap_stream, h->L.sms};
  const TableView t = h->table();
  const PoolView pool = h->pool();
  const bool t_int = tmask & (1 << VBH_STAGE_INTEGRATE), t_mc = tmask & (1 << VBH_STAGE_MC);
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < 4; ++i)
    if ((i < 2 && t_int) || (i >= 2 && t_mc)) ev[i] = h->get_event();
  VBH_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  // the root node takes the control block by value: vbh_process_frame patches it
  k_setup_frame<<<1, 1, 0, h->cap_stream>>>(base_ctl(h, nullptr), 0ull, h->consumed_dev, h->ctl,
                                            h->cnt);
  // Two pairs of independent kernels run as parallel branches of the graph, so that the one
  // that leaves issue slots idle fills them beside the other: the band allocation (it reads the
  // depth image and writes the candidate list only) beside the erase (table, pool, removal and
  // stream-out lists), and the MC set (touched and removed lists, keys, table, marks, versions)
  // beside the fusion (voxels, masks, fresh states).
  const Launch L2{h->cap_stream2, h->L.sms};
  VBH_CUDA(cudaEventRecord(h->fork_ev[0], h->cap_stream));
  VBH_CUDA(cudaStreamWaitEvent(h->cap_stream2, h->fork_ev[0], 0));
  launch_alloc_keys(L2, h->ctl, h->cfg.width, h->cfg.height, h->cand, h->cand_cap, h->cnt,
                    h->dimg);
  VBH_CUDA(cudaEventRecord(h->fork_ev[1], h->cap_stream2));
  launch_erase_radius(Lc, t, pool, h->cnt, h->ctl, h->removed, h->cfg.max_blocks, nullptr,
                      nullptr, stream_list(h));
  if (h->so) launch_stream_gather(Lc, h->so_ring, h->ctl, pool, h->cnt, stream_list(h));
  VBH_CUDA(cudaStreamWaitEvent(h->cap_stream, h->fork_ev[1], 0));
  launch_hash_insert(Lc, t, pool, h->cnt, h->cand, &h->cnt->n_cand, nullptr,
                     h->cand_res, h->cand_st, h->cand_cap);
  launch_hash_insert_finish(Lc, t, pool, h->cnt, &h->cnt->n_cand, h->cand_res, h->cand_st,
                            h->cand_cap, h->touched, h->tkey, h->tdepth, &h->cnt->n_touched,
                            h->ctl);
  if (h->integ_mode == VBH_INTEGRATE_VISIBLE)
    launch_visible(Lc, h->ctl, pool, h->touched, h->tkey, h->tdepth, &h->cnt->n_touched);
  VBH_CUDA(cudaEventRecord(h->fork_ev[2], h->cap_stream));
  VBH_CUDA(cudaStreamWaitEvent(h->cap_stream2, h->fork_ev[2], 0));
  launch_mset_touched(L2, t, pool, h->cnt, h->ctl, h->touched, &h->cnt->n_touched, h->removed,
                      &h->cnt->n_removed, h->cfg.max_blocks, h->mset, h->tombrec);
  VBH_CUDA(cudaEventRecord(h->fork_ev[3], h->cap_stream2));
  if (t_int) cudaEventRecordWithFlags(ev[0], h->cap_stream, cudaEventRecordExternal);
  // the fusion node takes the frame parameters by value: vbh_process_frame patches them
  launch_integrate(Lc, base_ctl(h, nullptr).fp, h->dimg, pool, h->touched, h->tkey, h->tdepth,
                   &h->cnt->n_touched, h->cnt);
  if (t_int) cudaEventRecordWithFlags(ev[1], h->cap_stream, cudaEventRecordExternal);
  VBH_CUDA(cudaStreamWaitEvent(h->cap_stream, h->fork_ev[3], 0));
  if (t_mc) cudaEventRecordWithFlags(ev[2], h->cap_stream, cudaEventRecordExternal);
  launch_mc_extract(Lc, t, pool, h->cnt, h->ctl, h->mset, h->tombrec);
  if (t_mc) cudaEventRecordWithFlags(ev[3], h->cap_stream, cudaEventRecordExternal);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  cudaError_t le = cudaGetLastError();
  if (e != cudaSuccess || le != cudaSuccess || !g)
    return fail(VBH_ERR_CUDA, std::string("frame graph capture: ") +
                                  cudaGetErrorString(e != cudaSuccess ? e : le));
  h->frame_graph = g;
  {
    size_t n = 0;
    VBH_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    VBH_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    h->integ_node = nullptr;
    h->setup_node = nullptr;
    for (cudaGraphNode_t node : nodes) {
      cudaGraphNodeType ty;
      VBH_CUDA(cudaGraphNodeGetType(node, &ty));
      if (ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp{};
      VBH_CUDA(cudaGraphKernelNodeGetParams(node, &kp));
      if (kp.func == integrate_kernel()) {
        h->integ_node = node;
        h->integ_kp = kp;
      } else if (kp.func == reinterpret_cast<const void*>(&k_setup_frame)) {
        h->setup_node = node;
        h->setup_kp = kp;
      }
    }
    if (!h->integ_node || !h->setup_node)
      return fail(VBH_ERR_CUDA, "frame graph: fusion or setup node not found");
  }
  if (tmask) {
    size_t n = 0;
    VBH_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    VBH_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    for (cudaGraphNode_t node : nodes) {
      cudaGraphNodeType ty;
      VBH_CUDA(cudaGraphNodeGetType(node, &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t e_n = nullptr;
      VBH_CUDA(cudaGraphEventRecordNodeGetEvent(node, &e_n));
      for (int i = 0; i < 4; ++i)
        if (ev[i] && e_n == ev[i]) h->ev_node[i] = node;
    }
    for (int i = 0; i < 4; ++i)
      if (ev[i] && !h->ev_node[i]) return fail(VBH_ERR_CUDA, "frame graph: event nodes");
  }
  VBH_CUDA(cudaGraphInstantiate(&h->frame_exec, g, 0));
  h->graph_timed = tmask;
  h->graph_mode = h->integ_mode;
  h->graph_kernels = 8 + (h->so ? 1 : 0) + (h->integ_mode == VBH_INTEGRATE_VISIBLE ? 1 : 0);
  return VBH_OK;
}

vbh_status vbh_process_frame(vbh_handle* h, const uint16_t* depth_dev, const float* T_wc_host,
                             uint32_t frame_id, float erase_radius, const vbh_mc_stream* out) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (!depth_dev || !T_wc_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (!stream_ok(out)) return fail(VBH_ERR_INVALID_ARG, "incomplete output stream");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_wc_host[i])) return fail(VBH_ERR_INVALID_ARG, "non-finite pose");
  if (frame_id >= 0x80000000u) return fail(VBH_ERR_INVALID_ARG, "frame_id must be < 2^31");
  if (!(erase_radius >= 0.f) || !std::isfinite(erase_radius))
    return fail(VBH_ERR_INVALID_ARG, "invalid erase radius");
  vbh_status st = maybe_rebuild(h);
  if (st != VBH_OK) return st;
  if (h->so) {   // move landed stream-out copies to the host map (waits if the ring is full)
    st = stream_out_poll(h, false);
    if (st != VBH_OK) return st;
  }
  const int tmask = h->timing & ((1 << VBH_STAGE_INTEGRATE) | (1 << VBH_STAGE_MC));
  if (!h->frame_exec || tmask != h->graph_timed || h->integ_mode != h->graph_mode) {
    st = build_frame_graph(h, tmask);
    if (st != VBH_OK) return st;
  }
  FrameCtl c = base_ctl(h, T_wc_host);
  c.fp.depth = depth_dev;
  c.do_erase = erase_radius > 0.f;
  for (int i = 0; i < 3; ++i) c.erase_c[i] = T_wc_host[4 * i + 3];
  c.erase_r2 = erase_radius * erase_radius;   // binary32 product, one rounding
  c.epoch_touch = h->next_epoch();
  c.epoch_mset = h->next_epoch();
  c.version = frame_id;
  c.clear_removed = 1;
  c.reset = kResetFrame | kResetErase | kResetMset;
  c.serve_mark = h->slog != nullptr;
  c.visible = h->integ_mode == VBH_INTEGRATE_VISIBLE;
  set_stream_out(c, out);
  // wait (bounded) until the graph launched `ahead` frames ago has started: a bound on the
  // frames queued on the GPU
  const unsigned long long seq = h->host_seq;
  const unsigned long long ahead = h->so ? kStreamOutAhead : kMaxAhead;
  if (seq >= ahead) {
    const unsigned long long need = seq - ahead + 1;
    int spins = 0;
    while (*h->consumed_host < need) {
      if (++spins > 2000000) return fail(VBH_ERR_TIMEOUT, "queued frames did not start");
      if (spins > 1000) usleep(5);
    }
  }
  {   // the control block into the root node (applies to this and later launches only)
    unsigned long long* consumed = h->consumed_dev;
    FrameCtl* dst = h->ctl;
    DevCounters* cntp = h->cnt;
    void* args[] = {&c, (void*)&seq, &consumed, &dst, &cntp};
    cudaKernelNodeParams kp = h->setup_kp;
    kp.kernelParams = args;
    kp.extra = nullptr;
    VBH_CUDA(cudaGraphExecKernelNodeSetParams(h->frame_exec, h->setup_node, &kp));
  }
  {   // this frame's parameters into the fusion node (applies to this and later launches)
    FrameParams fpv = c.fp;
    const float* dimg = h->dimg;
    PoolView pv = h->pool();
    const unsigned int* touched = h->touched;
    const unsigned long long* tkey = h->tkey;
    const float2* tdepth = h->tdepth;
    const unsigned int* n_touched = &h->cnt->n_touched;
    DevCounters* cntp = h->cnt;
    void* args[] = {&fpv, &dimg, &pv, &touched, &tkey, &tdepth, &n_touched, &cntp};
    cudaKernelNodeParams kp = h->integ_kp;
    kp.kernelParams = args;
    kp.extra = nullptr;
    VBH_CUDA(cudaGraphExecKernelNodeSetParams(h->frame_exec, h->integ_node, &kp));
  }
  for (int sidx = 0; sidx < 2; ++sidx) {   // fresh events for the timed stages of this frame
    const int stage = sidx == 0 ? VBH_STAGE_INTEGRATE : VBH_STAGE_MC;
    if (tmask & (1 << stage)) {
      cudaEvent_t a = h->get_event(), b = h->get_event();
      VBH_CUDA(cudaGraphExecEventRecordNodeSetEvent(h->frame_exec, h->ev_node[2 * sidx], a));
      VBH_CUDA(cudaGraphExecEventRecordNodeSetEvent(h->frame_exec, h->ev_node[2 * sidx + 1], b));
      h->pending.push_back(StageEvents{stage, a, b, 1});
    } else {
      h->stage_launches[stage] += 1;
    }
  }
  VBH_CUDA(cudaGraphLaunch(h->frame_exec, h->stream));
  h->host_seq = seq + 1;
  h->launches += h->graph_kernels;
  h->frame_version = frame_id;
  h->have_frame = true;
  h->last_entries = out->n_entries_dev;
  snapshot_counters(h);
  return VBH_OK;
}

vbh_status vbh_erase_blocks(vbh_handle* h, const vbh_erase_selector* sel,
                            int32_t* erased_keys3_dev, uint32_t* n_erased_dev) {
  if (!h || !sel) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  const TableView t = h->table();
  const PoolView pool = h->pool();
  if (sel->mode == VBH_ERASE_RADIUS) {
    if (!(sel->radius >= 0.f) || !std::isfinite(sel->radius) || !std::isfinite(sel->centre[0]) ||
        !std::isfinite(sel->centre[1]) || !std::isfinite(sel->centre[2]))
      return fail(VBH_ERR_INVALID_ARG, "invalid erase radius / centre");
  } else if (sel->mode == VBH_ERASE_KEYS) {
    if (sel->n_keys && !sel->keys3_dev) return fail(VBH_ERR_INVALID_ARG, "null key list");
  } else if (sel->mode == VBH_ERASE_FRUSTUM) {
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(sel->T_wc[i])) return fail(VBH_ERR_INVALID_ARG, "non-finite pose");
    if (!(sel->zfar >= 0.f) || !std::isfinite(sel->zfar))
      return fail(VBH_ERR_INVALID_ARG, "invalid far limit");
  } else {
    return fail(VBH_ERR_INVALID_ARG, "unknown erase mode");
  }
  if (h->so) {
    vbh_status pst = stream_out_poll(h, false);
    if (pst != VBH_OK) return pst;
  }
  FrameCtl c = base_ctl(h, sel->mode == VBH_ERASE_FRUSTUM ? sel->T_wc : nullptr);
  c.reset = kResetErase;
  h->stage_begin(VBH_STAGE_ERASE);
  if (sel->mode == VBH_ERASE_FRUSTUM) {
    c.do_erase = 2;
    c.erase_zfar = sel->zfar;
    launch_setup(h, c);
    launch_erase_radius(h->L, t, pool, h->cnt, h->ctl, h->removed, h->cfg.max_blocks,
                        erased_keys3_dev, n_erased_dev, stream_list(h));
    h->launches += 1;
  } else if (sel->mode == VBH_ERASE_RADIUS) {
    c.do_erase = 1;
    for (int i = 0; i < 3; ++i) c.erase_c[i] = sel->centre[i];
    c.erase_r2 = sel->radius * sel->radius;   // binary32 product, one rounding
    launch_setup(h, c);
    launch_erase_radius(h->L, t, pool, h->cnt, h->ctl, h->removed, h->cfg.max_blocks,
                        erased_keys3_dev, n_erased_dev, stream_list(h));
    h->launches += 1;
  } else {
    launch_setup(h, c);
    launch_erase_keys(h->L, t, pool, h->cnt, sel->keys3_dev, sel->n_keys, h->removed,
                      h->cfg.max_blocks, erased_keys3_dev, n_erased_dev, stream_list(h));
    h->launches += sel->n_keys ? 1 : 0;
  }
  if (h->so) {
    launch_stream_gather(h->L, h->so_ring, h->ctl, pool, h->cnt, stream_list(h));
    h->launches += 1;
  }
  h->stage_end();
  vbh_status st = check_launch(h, "vbh_erase_blocks");
  snapshot_counters(h);
  return st;
}

vbh_status vbh_extract_mc_indices(vbh_handle* h, const vbh_mc_selector* sel,
                                  const vbh_mc_stream* out, uint64_t* needed_bytes_host) {
  if (!h || !sel || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (!stream_ok(out)) return fail(VBH_ERR_INVALID_ARG, "incomplete output stream");
  if (sel->mode > VBH_MC_SINCE) return fail(VBH_ERR_INVALID_ARG, "unknown extraction mode");
  if (sel->mode == VBH_MC_KEYS && sel->n_keys && !sel->keys3_dev)
    return fail(VBH_ERR_INVALID_ARG, "null key list");
  const TableView t = h->table();
  const PoolView pool = h->pool();
  FrameCtl c = base_ctl(h, nullptr);
  set_stream_out(c, out);
  c.epoch_mset = h->next_epoch();
  c.clear_removed = sel->mode == VBH_MC_TOUCHED;
  c.serve_mark = sel->mode == VBH_MC_TOUCHED && h->slog != nullptr;
  c.reset = kResetMset;
  h->stage_begin(VBH_STAGE_MCSET);
  launch_setup(h, c);
  switch (sel->mode) {
    case VBH_MC_TOUCHED:
      launch_mset_touched(h->L, t, pool, h->cnt, h->ctl, h->have_frame ? h->touched : nullptr,
                          h->have_frame ? &h->cnt->n_touched : nullptr, h->removed,
                          &h->cnt->n_removed, h->cfg.max_blocks, h->mset, h->tombrec);
      h->launches += 1;
      break;
    case VBH_MC_ALL:
    case VBH_MC_SINCE:
      launch_mset_scan(h->L, pool, h->cnt, h->mset, sel->mode == VBH_MC_SINCE, sel->since_version);
      h->launches += 1;
      break;
    default:
      launch_mset_keys(h->L, t, pool, h->cnt, h->ctl, sel->keys3_dev, sel->n_keys, h->mset);
      h->launches += sel->n_keys ? 1 : 0;
      break;
  }
  h->stage_end();
  h->stage_begin(VBH_STAGE_MC);
  launch_mc_extract(h->L, t, pool, h->cnt, h->ctl, h->mset, h->tombrec);
  h->launches += 1;
  h->stage_end();
  h->last_entries = out->n_entries_dev;
  vbh_status st = check_launch(h, "vbh_extract_mc_indices");
  if (st != VBH_OK) return st;
  if (needed_bytes_host) {
    uint32_t nb = 0, ne = 0;
    VBH_CUDA(cudaMemcpyAsync(&nb, out->n_blocks_dev, 4, cudaMemcpyDeviceToHost, h->stream));
    VBH_CUDA(cudaMemcpyAsync(&ne, out->n_entries_dev, 4, cudaMemcpyDeviceToHost, h->stream));
    VBH_CUDA(cudaStreamSynchronize(h->stream));
    *needed_bytes_host = (uint64_t)nb * (3 * sizeof(int32_t) + 3 * sizeof(uint32_t)) +
                         (uint64_t)ne * (sizeof(uint16_t) + sizeof(uint8_t));
    if (nb > out->cap_blocks || ne > out->cap_entries)
      return fail(VBH_ERR_BUFFER_TOO_SMALL, "MC stream capacity exceeded");
  }
  snapshot_counters(h);
  return VBH_OK;
}

vbh_status vbh_dump(vbh_handle* h, int32_t* keys3_host, float* tsdf_host, float* weight_host,
                    uint32_t* vals_host, uint32_t cap, uint32_t* n_host) {
  if (!h || !n_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if ((tsdf_host || weight_host) && h->cfg.max_blocks == 0)
    return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (cap && !keys3_host) return fail(VBH_ERR_INVALID_ARG, "null key buffer");
  DevCounters d;
  VBH_CUDA(cudaMemcpyAsync(&d, h->cnt, sizeof d, cudaMemcpyDeviceToHost, h->stream));
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  const unsigned int live = d.n_live;
  unsigned long long* dk = nullptr;
  unsigned int* dv = nullptr;
  unsigned int* dn = nullptr;
  float *dt = nullptr, *dw = nullptr;
  vbh_status st = VBH_OK;
  const unsigned int room = live + 1;
  std::vector<unsigned long long> hk;
  std::vector<unsigned int> hv;
  unsigned int n = 0;
  do {
    if (cudaMalloc(&dk, (size_t)room * 8) != cudaSuccess || cudaMalloc(&dv, (size_t)room * 4) != cudaSuccess ||
        cudaMalloc(&dn, 4) != cudaSuccess) {
      st = fail(VBH_ERR_CUDA, "vbh_dump: cudaMalloc failed");
      break;
    }
    cudaMemsetAsync(dn, 0, 4, h->stream);
    // the dump kernel appends every live slot; `room` bounds it (live is exact after a sync)
    launch_dump_table(h->L, h->table(), h->n_slots, dk, dv, room, dn);
    h->launches += 1;
    cudaMemcpyAsync(&n, dn, 4, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      st = fail(VBH_ERR_CUDA, "vbh_dump: kernel failed");
      break;
    }
    if (n > room) n = room;
    hk.resize(n);
    hv.resize(n);
    cudaMemcpy(hk.data(), dk, (size_t)n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(hv.data(), dv, (size_t)n * 4, cudaMemcpyDeviceToHost);
    const unsigned int m = n < cap ? n : cap;
    for (unsigned int i = 0; i < m; ++i) {
      int3 k = unpack_key(hk[i]);
      keys3_host[3 * i] = k.x;
      keys3_host[3 * i + 1] = k.y;
      keys3_host[3 * i + 2] = k.z;
      if (vals_host) vals_host[i] = hv[i];
    }
    if ((tsdf_host || weight_host) && m) {
      if (cudaMalloc(&dt, (size_t)m * 512 * 4) != cudaSuccess ||
          cudaMalloc(&dw, (size_t)m * 512 * 4) != cudaSuccess) {
        st = fail(VBH_ERR_CUDA, "vbh_dump: cudaMalloc failed");
        break;
      }
      launch_gather_blocks(h->L, h->pool(), dv, m, dt, dw);
      h->launches += 1;
      if (tsdf_host) cudaMemcpyAsync(tsdf_host, dt, (size_t)m * 512 * 4, cudaMemcpyDeviceToHost, h->stream);
      if (weight_host) cudaMemcpyAsync(weight_host, dw, (size_t)m * 512 * 4, cudaMemcpyDeviceToHost, h->stream);
      if (cudaStreamSynchronize(h->stream) != cudaSuccess) st = fail(VBH_ERR_CUDA, "vbh_dump: gather failed");
    }
  } while (0);
  for (void* p : {(void*)dk, (void*)dv, (void*)dn, (void*)dt, (void*)dw})
    if (p) cudaFree(p);
  *n_host = n;
  return st;
}

vbh_status vbh_load(vbh_handle* h, const int32_t* keys3_host, const float* tsdf_host,
                    const float* weight_host, uint32_t n) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (n == 0) return VBH_OK;
  if (!keys3_host || !tsdf_host || !weight_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  if (n > h->cfg.max_batch) return fail(VBH_ERR_INVALID_ARG, "more blocks than max_batch");
  int* dk = nullptr;
  unsigned char *dops = nullptr, *dst = nullptr;
  unsigned int* dres = nullptr;
  float *dt = nullptr, *dw = nullptr;
  vbh_status st = VBH_OK;
  std::vector<unsigned char> ops(n, (unsigned char)VBH_OP_INSERT), hst(n);
  do {
    if (cudaMalloc(&dk, (size_t)n * 12) != cudaSuccess || cudaMalloc(&dops, n) != cudaSuccess ||
        cudaMalloc(&dst, n) != cudaSuccess || cudaMalloc(&dres, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&dt, (size_t)n * 2048) != cudaSuccess || cudaMalloc(&dw, (size_t)n * 2048) != cudaSuccess) {
      st = fail(VBH_ERR_CUDA, "vbh_load: cudaMalloc failed");
      break;
    }
    cudaMemcpyAsync(dk, keys3_host, (size_t)n * 12, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dops, ops.data(), n, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dt, tsdf_host, (size_t)n * 2048, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dw, weight_host, (size_t)n * 2048, cudaMemcpyHostToDevice, h->stream);
    st = vbh_hash_batch(h, dops, dk, nullptr, dres, dst, n);
    if (st != VBH_OK) break;
    cudaMemcpyAsync(hst.data(), dst, n, cudaMemcpyDeviceToHost, h->stream);
    launch_scatter_blocks(h->L, h->pool(), dres, n, dt, dw);
    launch_block_masks(h->L, h->pool(), dres, n);
    h->launches += 2;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      st = fail(VBH_ERR_CUDA, "vbh_load: kernels failed");
      break;
    }
    for (unsigned int i = 0; i < n; ++i) {
      if (hst[i] == VBH_ST_INVALID) { st = fail(VBH_ERR_INVALID_ARG, "vbh_load: key out of range"); break; }
      if (hst[i] == VBH_ST_CAPACITY) { st = fail(VBH_ERR_CAPACITY, "vbh_load: pool or table full"); break; }
    }
  } while (0);
  for (void* p : {(void*)dk, (void*)dops, (void*)dst, (void*)dres, (void*)dt, (void*)dw})
    if (p) cudaFree(p);
  return st;
}

vbh_status vbh_get_counters(vbh_handle* h, vbh_counters* out) {
  if (!h || !out) return fail(VBH_ERR_INVALID_ARG, "null argument");
  DevCounters d;
  VBH_CUDA(cudaMemcpyAsync(&d, h->cnt, sizeof d, cudaMemcpyDeviceToHost, h->stream));
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  std::memset(out, 0, sizeof *out);
  out->live = d.n_live;
  out->tombstones = d.n_tomb;
  out->empty = d.n_empty;
  out->free_blocks = h->cfg.max_blocks ? (uint32_t)(d.free_top > 0 ? d.free_top : 0) : 0u;
  out->last_touched = d.n_touched;
  out->last_new = d.n_new;
  out->last_candidates = d.n_cand;
  out->error_flags = d.err;
  out->kernel_launches = h->launches;
  out->rebuilds = h->rebuilds;
  out->last_mc_blocks = d.mc_blocks;
  uint32_t ne = 0;
  if (h->last_entries) {
    VBH_CUDA(cudaMemcpy(&ne, h->last_entries, sizeof ne, cudaMemcpyDeviceToHost));
  }
  out->last_mc_entries = ne;
  out->last_erased = d.n_erased;
  out->voxels_written = d.vox_updated;
  out->total_frames = d.tot_frames;
  out->total_touched = d.tot_touched;
  out->total_new = d.tot_new;
  out->total_written = d.tot_written;
  return VBH_OK;
}

vbh_status vbh_set_wait_limit(vbh_handle* h, uint32_t polls) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  h->wait_limit = polls;
  return VBH_OK;
}

vbh_status vbh_clear_errors(vbh_handle* h) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  VBH_CUDA(cudaMemsetAsync(&h->cnt->err, 0, sizeof(unsigned int), h->stream));
  return VBH_OK;
}

vbh_status vbh_timing_enable(vbh_handle* h, int stage_mask) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  h->timing = stage_mask & ((1 << VBH_N_STAGES) - 1);
  return VBH_OK;
}

vbh_status vbh_timing_read(vbh_handle* h, double* ms_host, uint64_t* launches_host, int reset) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  VBH_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& s : h->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.a, s.b);
    h->ms[s.stage] += ms;
    h->stage_launches[s.stage] += s.launches;
    h->ev_free.push_back(s.a);
    h->ev_free.push_back(s.b);
  }
  h->pending.clear();
  for (int i = 0; i < VBH_N_STAGES; ++i) {
    if (ms_host) ms_host[i] = h->ms[i];
    if (launches_host) launches_host[i] = h->stage_launches[i];
    if (reset) {
      h->ms[i] = 0;
      h->stage_launches[i] = 0;
    }
  }
  return VBH_OK;
}

}  // extern "C"
