// Host-side state of a libvbh handle, shared by the C ABI implementation files (api.cu,
// serve.cu).  Not part of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "vbh.h"
#include "vbh_internal.cuh"

namespace vbh {

// Records the message returned by vbh_last_error() and passes the status through.
vbh_status fail(vbh_status st, const std::string& msg);

#define VBH_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ::vbh::fail(VBH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct StreamOutHost;   // stream-out bookkeeping on the host (streamout.cu)
struct HostPipe;        // pipelined host-buffer frames (hostframe.cu)

struct StageEvents {
  int stage;
  cudaEvent_t a, b;
  uint64_t launches;
};

}  // namespace vbh

using vbh::StageEvents;
using vbh::Slot;
using vbh::DevCounters;
using vbh::FrameCtl;
using vbh::Launch;
using vbh::TableView;
using vbh::PoolView;

struct vbh_handle {
  vbh_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;     // snapshot copies of the counters, off the critical path
  int device = 0;
  Launch L{};
  unsigned int n_slots = 0;
  Slot* slots = nullptr;
  Slot* shadow = nullptr;
  DevCounters* cnt = nullptr;
  DevCounters* snap = nullptr;     // pinned host snapshot
  cudaEvent_t snap_ev = nullptr;
  bool snap_pending = false;
  // pool
  float2* vox = nullptr;
  unsigned int* masks = nullptr;
  unsigned long long* pkeys = nullptr;
  unsigned int *state = nullptr, *mark = nullptr, *version = nullptr, *stack = nullptr;
  unsigned int* seq = nullptr;
  // attached server (serve.cu): device-resident log/store state and its host object
  vbh::ServeLog* slog = nullptr;
  vbh_serve* server = nullptr;
  // stream-out (streamout.cu): device transfer ring, erased-block list, host side
  vbh::StreamRing* so_ring = nullptr;
  float2* so_data_dev = nullptr;             // the ring's slots (cap x 512) and keys
  unsigned long long* so_keys_dev = nullptr;
  unsigned int* so_p = nullptr;
  unsigned long long* so_k = nullptr;
  vbh::StreamOutHost* so = nullptr;
  vbh::HostPipe* hp = nullptr;   // vbh_process_frame_host state
  vbh::BatchLists blists;        // vbh_hash_batch: compacted insert / erase lists
  uint32_t blists_cap = 0;
  uint32_t batch_parity = 0;     // which set of list lengths the next vbh_hash_batch uses
  // per-frame lists
  int J = 0;
  unsigned long long* cand = nullptr;
  unsigned int cand_cap = 0;
  unsigned int* cand_res = nullptr;
  float* dimg = nullptr;           // the frame's metric depth (fl(raw ds), -inf when invalid)
  unsigned char* cand_st = nullptr;
  unsigned int* touched = nullptr;
  unsigned long long* tkey = nullptr;   // key of each touched block
  float2* tdepth = nullptr;        // camera depth of each touched block's origin (hi, lo)
  unsigned int* mset = nullptr;
  unsigned long long* removed = nullptr;
  unsigned long long* tombrec = nullptr;
  unsigned int epoch = 0;
  unsigned int frame_version = 0;
  bool have_frame = false;
  FrameCtl* ctl = nullptr;         // device-resident per-call control block
  unsigned int* last_entries = nullptr;   // n_entries_dev of the last extraction
  // whole-frame CUDA graph (vbh_process_frame)
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cap_stream2 = nullptr;            // the frame graph's second branch (capture)
  cudaEvent_t fork_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // its fork / join points
  cudaGraph_t frame_graph = nullptr;
  cudaGraphExec_t frame_exec = nullptr;
  // the control block of each vbh_process_frame is the by-value argument of the graph's root
  // node (patched before the launch); the root node reports the frame's sequence number back
  // through mapped memory, which bounds the frames the host queues
  volatile unsigned long long* consumed_host = nullptr;
  unsigned long long* consumed_dev = nullptr;
  unsigned long long host_seq = 0;
  cudaGraphNode_t setup_node = nullptr;
  cudaKernelNodeParams setup_kp{};
  cudaGraphNode_t ev_node[4] = {nullptr, nullptr, nullptr, nullptr};   // fusion, MC extraction
  cudaGraphNode_t integ_node = nullptr;   // fusion node: its by-value frame parameters are
  cudaKernelNodeParams integ_kp{};        // patched before every launch
  int graph_timed = 0;             // stage mask the captured graph brackets with events
  uint32_t integ_mode = 0;         // VBH_INTEGRATE_*
  uint32_t wait_limit = 1u << 24;  // polls of the fusion kernel's bounded copy wait
  uint32_t gbar_base = 0;          // small-batch barrier arrivals so far (the device counter's value)
  bool serve_loop_active = false;  // a device-resident serving loop reads the table: no rebuild
  uint32_t graph_mode = 0;         // integration mode the frame graph was captured with
  uint64_t graph_kernels = 0;
  // bookkeeping
  uint64_t launches = 0;
  uint32_t rebuilds = 0;
  int timing = 0;                  // bit mask of timed stages
  std::vector<StageEvents> pending;
  std::vector<cudaEvent_t> ev_free;
  double ms[VBH_N_STAGES] = {0};
  uint64_t stage_launches[VBH_N_STAGES] = {0};
  int cur_stage = -1;
  cudaEvent_t cur_a = nullptr;
  uint64_t cur_launch0 = 0;

  TableView table() const { return TableView{slots, cfg.n_buckets - 1u, cfg.hash_fn}; }
  PoolView pool() const {
    return PoolView{vox, masks, pkeys, state, mark, version, stack, seq, cfg.max_blocks};
  }
  unsigned int next_epoch() {
    ++epoch;
    if (epoch == 0) epoch = 1;
    return epoch;
  }
  cudaEvent_t get_event() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void stage_begin(int s) {
    cur_stage = s;
    cur_launch0 = launches;
    if (timing & (1 << s)) {
      cur_a = get_event();
      cudaEventRecord(cur_a, stream);
    }
  }
  void stage_end() {
    if (cur_stage >= 0 && (timing & (1 << cur_stage))) {
      cudaEvent_t b = get_event();
      cudaEventRecord(b, stream);
      pending.push_back(StageEvents{cur_stage, cur_a, b, launches - cur_launch0});
    } else if (cur_stage >= 0) {
      stage_launches[cur_stage] += launches - cur_launch0;
    }
    cur_stage = -1;
  }
};

namespace vbh {
// Copies filled ring slots to host memory and folds landed copies into the host map; with
// `wait`, first waits for the handle's stream and then for every copy.
vbh_status stream_out_poll(vbh_handle* h, bool wait);
unsigned long long stream_out_tail(const vbh_handle* h);
void stream_out_release(vbh_handle* h);
void host_pipe_release(vbh_handle* h);
inline StreamList stream_list(const vbh_handle* h);
// The volume handle and the device-resident log/store of a server (serve.cu).
vbh_handle* serve_handle(vbh_serve* s);
const ServeLog* serve_log(vbh_serve* s);
// What the device-resident request loop (serve_loop.cu) shares with its server.
struct ServeShared {
  vbh_handle* h;
  const ServeLog* sl;
  unsigned int* client_v;      // per-client versions (device)
  unsigned char* arena;        // the stream buffer
  uint64_t budget;             // its usable bytes (multiple of 256)
  unsigned int n_clients, log_cap;
};
ServeShared serve_shared(vbh_serve* s);
bool serve_idle(vbh_serve* s);
vbh_serve_loop* serve_loop_of(vbh_serve* s);
void serve_set_loop(vbh_serve* s, vbh_serve_loop* L);
vbh_status serve_reload_versions(vbh_serve* s);
// MC refresh of every live block into the attached server's store and log, with no stream
// output (enqueued on the handle's stream).  counts_dev: two device words of scratch.
vbh_status refresh_all_blocks(vbh_handle* h, unsigned int* counts_dev);
}  // namespace vbh

namespace vbh {
inline StreamList stream_list(const vbh_handle* h) {
  return h->so ? StreamList{h->so_p, h->so_k} : StreamList{nullptr, nullptr};
}
}  // namespace vbh
