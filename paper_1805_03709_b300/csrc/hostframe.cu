// vbh_process_frame with host buffers, pipelined over consecutive calls, three frames deep.
//
// Call k (j = k mod 3) enqueues: the depth copy host -> device buffer j on the copy-in stream
// (after frame k-3, which read buffer j, has finished), the frame graph on the handle's stream into
// device stream j (after frame k-3's results, read from stream j, have been copied out), and a
// one-warp kernel that writes frame k's two totals to mapped pinned memory.  Then it moves the older frames along: frame
// k-1's records and entries start their copy into the caller's host buffers if its totals have
// already landed (no wait), and frame k-2 -- whose copy was started by now, waiting for its
// totals only if the GPU is two frames behind -- is waited for and marked done.  So the host
// blocks only when the GPU is behind, and the copy-out of a frame overlaps the next ones.
#include "handle.cuh"

#include <deque>

namespace vbh {

constexpr int kHostSlots = 3;

#ifndef VBH_HOST_TOTALS_KERNEL
#define VBH_HOST_TOTALS_KERNEL 1
#endif
// A frame's two stream totals to mapped pinned host memory, written by one warp on the frame's
// stream (a copy-engine transfer there would hand the stream to a copy engine and back after
// every frame); visible to the host once the frame's event has completed.
__global__ void k_frame_totals(const uint32_t* n_dev, uint32_t* n_host) {
  if (threadIdx.x < 2u) n_host[threadIdx.x] = __ldcg(n_dev + threadIdx.x);
  __threadfence_system();
}

struct HostPipe {
  struct Pending {
    vbh_mc_stream_host* out;
    uint32_t frame_id;
    int j;
    bool copying;   // its copy-out has been enqueued
  };
  cudaStream_t copy = nullptr;      // copies out (device -> host)
  cudaStream_t copy_in = nullptr;   // depth copies in, beside the copies out (the two
                                    // directions run on separate copy engines)
  uint16_t* depth[kHostSlots] = {};   // device depth images
  // device output streams and their totals (device) / totals copy (pinned host)
  int32_t* keys3[kHostSlots] = {};
  uint32_t* info[kHostSlots] = {};
  uint32_t* offsets[kHostSlots] = {};
  uint32_t* counts[kHostSlots] = {};
  uint16_t* local[kHostSlots] = {};
  uint8_t* index[kHostSlots] = {};
  uint32_t* n_dev[kHostSlots] = {};
  uint32_t* n_pin[kHostSlots] = {};       // mapped pinned host memory
  uint32_t* n_pin_dev[kHostSlots] = {};   // its device address
  uint32_t cap_blocks = 0, cap_entries = 0;
  cudaEvent_t e_h2d[kHostSlots] = {}, e_frame[kHostSlots] = {}, e_out[kHostSlots] = {};
  bool frame_used[kHostSlots] = {}, out_used[kHostSlots] = {};
  unsigned long long k = 0;      // frames enqueued
  std::deque<Pending> pending;   // enqueued frames not yet done, oldest first
};

namespace {

void free_streams(HostPipe* p) {
  for (int j = 0; j < kHostSlots; ++j) {
    void* d[] = {p->keys3[j], p->info[j], p->offsets[j], p->counts[j], p->local[j], p->index[j]};
    for (void* q : d)
      if (q) cudaFree(q);
    p->keys3[j] = nullptr;
    p->info[j] = p->offsets[j] = p->counts[j] = nullptr;
    p->local[j] = nullptr;
    p->index[j] = nullptr;
  }
  p->cap_blocks = p->cap_entries = 0;
}

vbh_status alloc_streams(HostPipe* p, uint32_t cb, uint32_t ce) {
  free_streams(p);
  for (int j = 0; j < kHostSlots; ++j) {
    VBH_CUDA(cudaMalloc(&p->keys3[j], sizeof(int32_t) * 3ull * cb));
    VBH_CUDA(cudaMalloc(&p->info[j], sizeof(uint32_t) * (size_t)cb));
    VBH_CUDA(cudaMalloc(&p->offsets[j], sizeof(uint32_t) * (size_t)cb));
    VBH_CUDA(cudaMalloc(&p->counts[j], sizeof(uint32_t) * (size_t)cb));
    VBH_CUDA(cudaMalloc(&p->local[j], sizeof(uint16_t) * (size_t)ce));
    VBH_CUDA(cudaMalloc(&p->index[j], (size_t)ce));
  }
  p->cap_blocks = cb;
  p->cap_entries = ce;
  return VBH_OK;
}

vbh_status create_pipe(vbh_handle* h) {
  HostPipe* p = new HostPipe();
  h->hp = p;
  VBH_CUDA(cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking));
  VBH_CUDA(cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking));
  const size_t db = sizeof(uint16_t) * (size_t)h->cfg.width * h->cfg.height;
  for (int j = 0; j < kHostSlots; ++j) {
    VBH_CUDA(cudaMalloc(&p->depth[j], db));
    VBH_CUDA(cudaMalloc(&p->n_dev[j], 2 * sizeof(uint32_t)));
#if VBH_HOST_TOTALS_KERNEL
    VBH_CUDA(cudaHostAlloc((void**)&p->n_pin[j], 2 * sizeof(uint32_t), cudaHostAllocMapped));
    VBH_CUDA(cudaHostGetDevicePointer((void**)&p->n_pin_dev[j], p->n_pin[j], 0));
#else
    VBH_CUDA(cudaMallocHost(&p->n_pin[j], 2 * sizeof(uint32_t)));
#endif
    VBH_CUDA(cudaEventCreateWithFlags(&p->e_h2d[j], cudaEventDisableTiming));
    VBH_CUDA(cudaEventCreateWithFlags(&p->e_frame[j], cudaEventDisableTiming));
    VBH_CUDA(cudaEventCreateWithFlags(&p->e_out[j], cudaEventDisableTiming));
  }
  return VBH_OK;
}

// Enqueue the copy of a pending frame's stream into its host buffers (its totals must have
// landed: with `wait`, wait for them; without, leave the frame if they have not).
vbh_status start_copy(HostPipe* p, HostPipe::Pending& f, bool wait) {
  if (f.copying) return VBH_OK;
  const int j = f.j;
  if (wait) {
    VBH_CUDA(cudaEventSynchronize(p->e_frame[j]));
  } else {
    const cudaError_t q = cudaEventQuery(p->e_frame[j]);
    if (q == cudaErrorNotReady) return VBH_OK;
    if (q != cudaSuccess) return fail(VBH_ERR_CUDA, cudaGetErrorString(q));
  }
  vbh_mc_stream_host* o = f.out;
  const uint32_t nb = p->n_pin[j][0], ne = p->n_pin[j][1];
  const uint32_t cb = nb < o->cap_blocks ? nb : o->cap_blocks;
  const uint32_t ce = ne < o->cap_entries ? ne : o->cap_entries;
  if (cb) {
    VBH_CUDA(cudaMemcpyAsync(o->keys3, p->keys3[j], sizeof(int32_t) * 3ull * cb,
                             cudaMemcpyDeviceToHost, p->copy));
    VBH_CUDA(cudaMemcpyAsync(o->info, p->info[j], sizeof(uint32_t) * (size_t)cb,
                             cudaMemcpyDeviceToHost, p->copy));
    VBH_CUDA(cudaMemcpyAsync(o->offsets, p->offsets[j], sizeof(uint32_t) * (size_t)cb,
                             cudaMemcpyDeviceToHost, p->copy));
    VBH_CUDA(cudaMemcpyAsync(o->counts, p->counts[j], sizeof(uint32_t) * (size_t)cb,
                             cudaMemcpyDeviceToHost, p->copy));
  }
  if (ce) {
    VBH_CUDA(cudaMemcpyAsync(o->local, p->local[j], sizeof(uint16_t) * (size_t)ce,
                             cudaMemcpyDeviceToHost, p->copy));
    VBH_CUDA(cudaMemcpyAsync(o->index, p->index[j], (size_t)ce, cudaMemcpyDeviceToHost,
                             p->copy));
  }
  VBH_CUDA(cudaEventRecord(p->e_out[j], p->copy));
  p->out_used[j] = true;
  f.copying = true;
  return VBH_OK;
}

// Complete the oldest pending frame: its copy started (waiting for its totals if needed) and
// landed; mark it done.
vbh_status complete_oldest(HostPipe* p) {
  if (p->pending.empty()) return VBH_OK;
  HostPipe::Pending f = p->pending.front();
  vbh_status st = start_copy(p, f, true);
  if (st != VBH_OK) return st;
  p->pending.pop_front();
  const int j = f.j;
  VBH_CUDA(cudaEventSynchronize(p->e_out[j]));
  vbh_mc_stream_host* o = f.out;
  const uint32_t nb = p->n_pin[j][0], ne = p->n_pin[j][1];
  o->n_blocks = nb;
  o->n_entries = ne;
  o->frame_id = f.frame_id;
  o->done = 1u;
  if (nb > o->cap_blocks || ne > o->cap_entries)
    return fail(VBH_ERR_BUFFER_TOO_SMALL, "host stream capacity exceeded (frame results cut)");
  return VBH_OK;
}

vbh_status complete_all(HostPipe* p) {
  vbh_status first = VBH_OK;
  while (!p->pending.empty()) {
    const vbh_status st = complete_oldest(p);
    if (st == VBH_ERR_BUFFER_TOO_SMALL) {
      if (first == VBH_OK) first = st;
    } else if (st != VBH_OK) {
      return st;
    }
  }
  return first;
}

}  // namespace

void host_pipe_release(vbh_handle* h) {
  HostPipe* p = h->hp;
  if (!p) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (cudaStream_t c : {p->copy, p->copy_in}) {
    if (!c) continue;
    cudaStreamSynchronize(c);
    cudaStreamDestroy(c);
  }
  free_streams(p);
  for (int j = 0; j < kHostSlots; ++j) {
    if (p->depth[j]) cudaFree(p->depth[j]);
    if (p->n_dev[j]) cudaFree(p->n_dev[j]);
    if (p->n_pin[j]) cudaFreeHost(p->n_pin[j]);
    for (cudaEvent_t e : {p->e_h2d[j], p->e_frame[j], p->e_out[j]})
      if (e) cudaEventDestroy(e);
  }
  delete p;
  h->hp = nullptr;
}

}  // namespace vbh

using namespace vbh;

vbh_status vbh_process_frame_host(vbh_handle* h, const uint16_t* depth_host,
                                  const float* T_wc_host, uint32_t frame_id, float erase_radius,
                                  vbh_mc_stream_host* out_host) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (h->cfg.max_blocks == 0) return fail(VBH_ERR_UNSUPPORTED, "plain map handle has no voxels");
  if (!depth_host || !T_wc_host || !out_host) return fail(VBH_ERR_INVALID_ARG, "null argument");
  const vbh_mc_stream_host& o = *out_host;
  if (o.cap_blocks == 0 || o.cap_entries == 0 || !o.keys3 || !o.info || !o.offsets ||
      !o.counts || !o.local || !o.index)
    return fail(VBH_ERR_INVALID_ARG, "incomplete host output stream");
  if (!h->hp) {
    vbh_status st = create_pipe(h);
    if (st != VBH_OK) {
      host_pipe_release(h);
      return st;
    }
  }
  HostPipe* p = h->hp;
  vbh_status done_st = VBH_OK;
  if (o.cap_blocks > p->cap_blocks || o.cap_entries > p->cap_entries) {
    // larger device streams: every frame in flight completes first
    done_st = complete_all(p);
    if (done_st != VBH_OK && done_st != VBH_ERR_BUFFER_TOO_SMALL) return done_st;
    VBH_CUDA(cudaStreamSynchronize(h->stream));
    VBH_CUDA(cudaStreamSynchronize(p->copy));
    VBH_CUDA(cudaStreamSynchronize(p->copy_in));
    const uint32_t cb = o.cap_blocks > p->cap_blocks ? o.cap_blocks : p->cap_blocks;
    const uint32_t ce = o.cap_entries > p->cap_entries ? o.cap_entries : p->cap_entries;
    vbh_status st = alloc_streams(p, cb, ce);
    if (st != VBH_OK) return st;
  }
  const int j = (int)(p->k % kHostSlots);
  // depth in: after frame k-3 (the last reader of buffer j) has finished
  if (p->frame_used[j]) VBH_CUDA(cudaStreamWaitEvent(p->copy_in, p->e_frame[j], 0));
  const size_t db = sizeof(uint16_t) * (size_t)h->cfg.width * h->cfg.height;
  VBH_CUDA(cudaMemcpyAsync(p->depth[j], depth_host, db, cudaMemcpyHostToDevice, p->copy_in));
  VBH_CUDA(cudaEventRecord(p->e_h2d[j], p->copy_in));
  // the frame: after its depth has landed and stream j's previous results were copied out
  VBH_CUDA(cudaStreamWaitEvent(h->stream, p->e_h2d[j], 0));
  if (p->out_used[j]) VBH_CUDA(cudaStreamWaitEvent(h->stream, p->e_out[j], 0));
  vbh_mc_stream s{p->keys3[j], p->info[j],  p->offsets[j], p->counts[j], p->local[j],
                  p->index[j], p->cap_blocks, p->cap_entries, p->n_dev[j], p->n_dev[j] + 1};
  out_host->done = 0u;
  vbh_status st = vbh_process_frame(h, p->depth[j], T_wc_host, frame_id, erase_radius, &s);
  if (st != VBH_OK) return st;
#if VBH_HOST_TOTALS_KERNEL
  k_frame_totals<<<1, 32, 0, h->stream>>>(p->n_dev[j], p->n_pin_dev[j]);
  VBH_CUDA(cudaGetLastError());
  h->launches += 1;
#else
  VBH_CUDA(cudaMemcpyAsync(p->n_pin[j], p->n_dev[j], 2 * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost, h->stream));
#endif
  VBH_CUDA(cudaEventRecord(p->e_frame[j], h->stream));
  p->frame_used[j] = true;
  ++p->k;
  p->pending.push_back(HostPipe::Pending{out_host, frame_id, j, false});
  // the frame before this one starts its copy-out if its totals are in; the one before that
  // completes (slot j of the next call is its slot)
  if (p->pending.size() >= 2) {
    st = start_copy(p, p->pending[p->pending.size() - 2], false);
    if (st != VBH_OK) return st;
  }
  if (done_st == VBH_OK && p->pending.size() >= (size_t)kHostSlots) done_st = complete_oldest(p);
  return done_st;
}

vbh_status vbh_process_frame_host_flush(vbh_handle* h) {
  if (!h) return fail(VBH_ERR_INVALID_ARG, "null handle");
  if (!h->hp) return VBH_OK;
  return complete_all(h->hp);
}
