/* vbh.h -- C ABI of the B300 voxel-block-hashing library (libvbh.so).
 *
 * The library implements, on one GPU, the per-frame data-parallel path of the SLAMCast
 * reconstruction server (Stotko et al., "SLAMCast: Large-Scale, Real-Time 3D Reconstruction and
 * Streaming for Immersive Multi-Client Live Telepresence"):
 *   - a GPU hash map of int3 voxel-block coordinates with guaranteed concurrent find / insert /
 *     erase and unique keys (Sec. 5, "Retrieval", "Insertion", "Removal");
 *   - block allocation from a depth frame and projective TSDF fusion into 8^3 voxel blocks
 *     (voxel block hashing, Sec. 4.1);
 *   - removal of blocks that leave the active region (Sec. 4.1, stream-out);
 *   - per-voxel 8-bit Marching Cubes indices of the updated blocks and their seven neighbours in
 *     negative direction, with indices 0 and 255 written as 0 (Sec. 4.2, the S^c equation),
 *     compacted into per-block streams.
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are device pointers owned by the caller (for example a torch
 *     tensor's data_ptr()); pointers named *_host are host pointers owned by the caller.  The
 *     handle owns its hash table, block pool, free list and per-frame lists.
 *   - All work is enqueued on the handle's CUDA stream and is asynchronous with respect to the
 *     host, except where a host output pointer is given: then the call synchronises the stream
 *     before it returns.  A handle is used from one host thread at a time.
 *   - Errors are returned as vbh_status; nothing throws across the ABI.  Capacity exhaustion
 *     inside a kernel (block pool or table full, output buffer too small) never drops work
 *     silently: the affected operation gets a per-op status or the stream reports the count it
 *     needed, and a sticky flag is raised that vbh_get_counters() reports.
 *   - Block coordinates are int32 triples (x, y, z) laid out as keys3[3*i + {0,1,2}], each in
 *     [-2^20, 2^20).  Voxel (lx, ly, lz) of a block has linear index lx + 8 ly + 64 lz.
 *   - A pose T_wc is 12 float32 (row-major 3x4 [R | t]) mapping camera to world: X = R p + t.
 *     Camera frame: x right, y down, z forward; pixel (u, v) is centred at (u, v).
 */
#ifndef VBH_H_
#define VBH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VBH_ABI_VERSION 1

typedef enum {
  VBH_OK = 0,
  VBH_ERR_INVALID_ARG = 1,      /* a pointer, size or configuration value is unusable */
  VBH_ERR_CAPACITY = 2,         /* block pool or hash table exhausted (per-op status set) */
  VBH_ERR_CUDA = 3,             /* a CUDA runtime call failed; see vbh_last_error() */
  VBH_ERR_TIMEOUT = 4,          /* a bounded device-side wait gave up */
  VBH_ERR_BUFFER_TOO_SMALL = 5, /* an output stream is smaller than what was produced */
  VBH_ERR_UNSUPPORTED = 6       /* the call does not apply to this kind of handle */
} vbh_status;

/* Hash operations (Sec. 5) and their per-op results. */
enum { VBH_OP_FIND = 0, VBH_OP_INSERT = 1, VBH_OP_ERASE = 2 };
enum {
  VBH_ST_FOUND = 1,      /* find: key present, result = its value */
  VBH_ST_NOT_FOUND = 2,  /* find / erase: key absent, result = 0xFFFFFFFF */
  VBH_ST_INSERTED = 3,   /* insert: this op added the key, result = its value */
  VBH_ST_EXISTS = 4,     /* insert: key already present (or added by a duplicate op of the
                            same batch), result = the value the key holds */
  VBH_ST_ERASED = 5,     /* erase: this op removed the key, result = the value it held */
  VBH_ST_CAPACITY = 6,   /* insert: table or block pool full; the key was not added */
  VBH_ST_INVALID = 7     /* unknown op code or key coordinate outside [-2^20, 2^20) */
};
#define VBH_NONE 0xFFFFFFFFu

enum { VBH_HASH_PRIMES = 0, /* b = (x p1 ^ y p2 ^ z p3) mod n, Sec. 5 "Retrieval" equation */
       VBH_HASH_MIX = 1     /* 64-bit avalanche mix of the packed key (default) */ };

typedef struct {
  float voxel_size;        /* s, metres (> 0) */
  float trunc;             /* truncation mu, metres (> 0) */
  float max_weight;        /* fusion weight cap Wmax (>= 1) */
  float depth_scale;       /* metres per raw uint16 depth unit (e.g. 0.001) */
  float zmax;              /* pixels with depth > zmax are ignored; 0 = no limit */
  int32_t width, height;   /* depth image size (pixels) */
  float fx, fy, cx, cy;    /* pinhole intrinsics (pixels) */
  uint32_t n_buckets;      /* hash buckets, a power of two >= 2 */
  uint32_t slots_per_bucket; /* must be 4 */
  uint32_t max_blocks;     /* voxel-block pool size; 0 = plain key -> uint32 map, no voxels */
  uint32_t hash_fn;        /* VBH_HASH_PRIMES or VBH_HASH_MIX */
  uint32_t max_batch;      /* largest n accepted by vbh_hash_batch (0 = 2^22) */
} vbh_config;

typedef struct vbh_handle vbh_handle;

/* Counters, read synchronously from the device. */
typedef struct {
  uint32_t live;            /* keys in the table */
  uint32_t tombstones;      /* erased slots not yet reused */
  uint32_t empty;           /* never-used slots */
  uint32_t free_blocks;     /* block pool entries available */
  uint32_t last_touched;    /* blocks allocated/updated by the last vbh_integrate_frame */
  uint32_t last_new;        /* of which newly allocated */
  uint32_t last_candidates; /* distinct block keys per image tile summed over tiles */
  uint32_t error_flags;     /* sticky: bit0 pool exhausted, bit1 table full, bit2 stream
                               overflow, bit3 bounded wait timed out, bit4 stream-out ring
                               without room (blocks counted as lost) */
  uint64_t kernel_launches; /* kernels this handle has launched since creation */
  uint32_t rebuilds;        /* table rebuilds performed (tombstone clean-up) */
  uint32_t last_mc_blocks;  /* records produced by the last extraction */
  uint32_t last_mc_entries; /* entries produced by the last extraction */
  uint32_t last_erased;     /* blocks removed by the last vbh_erase_blocks */
  uint64_t voxels_written;  /* voxels the last vbh_integrate_frame wrote (fused, or zeroed in
                               a new block) */
  uint64_t total_frames;    /* running totals over every fused frame of the handle */
  uint64_t total_touched;
  uint64_t total_new;
  uint64_t total_written;
} vbh_counters;

typedef struct {
  uint32_t touched;         /* blocks of this frame (allocated or already live) */
  uint32_t new_blocks;      /* of which new */
  uint32_t candidates;      /* per-tile distinct keys before the global de-duplication */
  uint32_t error_flags;     /* as in vbh_counters */
} vbh_frame_stats;

/* Lifecycle ---------------------------------------------------------------------------------
 * vbh_create: validates `cfg`, allocates the table (n_buckets * 4 slots * 16 B, plus an equal
 * rebuild buffer), the block pool (max_blocks * 4 KiB of (TSDF, weight) float pairs plus 160 B
 * of metadata per block) and the per-frame lists on the current device, and binds
 * `cuda_stream` (a cudaStream_t, or NULL for the legacy default stream).  *out receives the
 * handle.  The call synchronises. */
vbh_status vbh_create(const vbh_config* cfg, void* cuda_stream, vbh_handle** out);
vbh_status vbh_destroy(vbh_handle* h);
vbh_status vbh_set_stream(vbh_handle* h, void* cuda_stream);

/* Hash batch (Sec. 5; phased reading: all finds see the pre-batch state, then all inserts run,
 * then all erases).  ops_dev: n uint8 op codes; keys3_dev: n int3; vals_dev: n uint32 values to
 * insert (plain maps only; may be NULL = 0); results_dev: n uint32; status_dev: n uint8.
 * Among duplicate inserts of one key exactly one reports INSERTED and all return the same value;
 * among duplicate erases exactly one reports ERASED.  On a voxel-block handle (max_blocks > 0)
 * an insert takes a block from the pool (value = pool index; the new block reads as TSDF 0,
 * weight 0) and an erase returns it.  n may be 0.  n > max_batch -> VBH_ERR_INVALID_ARG.
 * A plain map's batch of at most 2^17 ops runs in one cooperative launch with one thread per
 * op: finds, then inserts, then erases, separated by grid barriers; a barrier that waits longer
 * than ~1 s gives up and raises error flag bit3 (the batch's results are then not to be
 * trusted).  Other batches run as phased launches over op lists.  The call is asynchronous on
 * the handle's stream, except that the first phased batch larger than any before it
 * synchronises and allocates the handle's op lists (36 B per op: the batch's finds, inserts
 * and erases as op index + packed key); VBH_ERR_CUDA if that allocation fails. */
vbh_status vbh_hash_batch(vbh_handle* h, const uint8_t* ops_dev, const int32_t* keys3_dev,
                          const uint32_t* vals_dev, uint32_t* results_dev, uint8_t* status_dev,
                          uint32_t n);

/* Rebuild the table from its live entries, turning every tombstone back into an empty slot
 * (live keys keep their values).  Runs automatically before a batch or frame once tombstones
 * outnumber half of the non-live slots; exposed for tests and maintenance. */
vbh_status vbh_hash_rebuild(vbh_handle* h);

/* Fusion of one frame (Sec. 4.1, voxel block hashing): every valid pixel samples its band
 * [d - mu, d + mu] at spacing s; each sample's block is found or inserted (new blocks start at
 * TSDF 0, weight 0); then every voxel of every touched block is projected into the frame and
 * fused with the projective TSDF running average.  depth_dev: height*width uint16 (raw units,
 * 0 = invalid), row-major; T_wc_host: 12 floats; frame_id: stored as the blocks' version by the
 * next touched-set extraction.  stats_host may be NULL (asynchronous) or receive the frame's
 * counts (synchronising).  Returns VBH_ERR_CAPACITY (only when stats_host is given) if the pool
 * or table ran out; the blocks that could be allocated are fused; VBH_ERR_TIMEOUT (likewise) if
 * a bounded device wait gave up (see vbh_set_wait_limit). */
vbh_status vbh_integrate_frame(vbh_handle* h, const uint16_t* depth_dev, const float* T_wc_host,
                               uint32_t frame_id, vbh_frame_stats* stats_host);

enum { VBH_ERASE_RADIUS = 0, VBH_ERASE_KEYS = 1, VBH_ERASE_FRUSTUM = 2 };
typedef struct {
  uint32_t mode;           /* VBH_ERASE_RADIUS, VBH_ERASE_KEYS or VBH_ERASE_FRUSTUM */
  float centre[3];         /* RADIUS: erase blocks whose centre (8k + 3.5) s is farther ... */
  float radius;            /* ... than `radius` metres from `centre` */
  const int32_t* keys3_dev;/* KEYS: n_keys block coordinates (absent keys are ignored) */
  uint32_t n_keys;
  float T_wc[12];          /* FRUSTUM (the scene reset of Sec. 4.1): erase every block in view
                              of this pose with the handle's camera -- its bounding sphere,
                              centre (8k + 3.5) s and radius 7 s, not outside the frustum
                              (side-plane margin 7 s G, G = max(fx, fy) + max(cx + 0.5,
                              W - cx - 0.5, cy + 0.5, H - cy - 0.5)) ... */
  float zfar;              /* ... and, when zfar > 0, no farther than zfar + 7 s in depth */
} vbh_erase_selector;

/* Removal of blocks that leave the active region (Sec. 4.1: blocks no longer in view are
 * streamed out and leave the GPU model).  Erased blocks go back to the pool and are remembered
 * for the next touched-set extraction, which reports them as removed.  erased_keys3_dev
 * (capacity: max_blocks keys) and n_erased_dev (one uint32) may be NULL. */
vbh_status vbh_erase_blocks(vbh_handle* h, const vbh_erase_selector* sel_host,
                            int32_t* erased_keys3_dev, uint32_t* n_erased_dev);

/* Fusion set of vbh_integrate_frame / vbh_process_frame.  TOUCHED (default): the blocks the
 * frame's truncation band allocated or reached (voxel block hashing, Sec. 4.1).  VISIBLE: those
 * and every live block in view of the frame (the FRUSTUM test above with zmax as far limit),
 * so that voxels the band does not reach are updated where they see free space (f = 1), and
 * surfaces that have moved away are carved; the extra blocks join the MC set too. */
enum { VBH_INTEGRATE_TOUCHED = 0, VBH_INTEGRATE_VISIBLE = 1 };
vbh_status vbh_set_integration_mode(vbh_handle* h, uint32_t mode);

enum { VBH_MC_TOUCHED = 0, /* blocks of the last fused frame + their seven negative neighbours,
                              plus removal records for blocks erased since the last call */
       VBH_MC_ALL = 1,     /* every live block */
       VBH_MC_KEYS = 2,    /* the given blocks + their seven negative neighbours (live only) */
       VBH_MC_SINCE = 3    /* every live block whose version is > since_version */ };
#define VBH_REC_REMOVED 0x80000000u  /* info bit: the block was erased (count = 0) */

typedef struct {
  uint32_t mode;
  const int32_t* keys3_dev; /* KEYS mode */
  uint32_t n_keys;
  uint32_t since_version;   /* SINCE mode */
} vbh_mc_selector;

/* Output stream of an extraction (all device buffers owned by the caller).
 * Record r (r < *n_blocks_dev): keys3[3r..3r+2] = block, info[r] = version | VBH_REC_REMOVED,
 * offsets[r], counts[r] = its entries' range in local/index.  Entry e: local[e] = voxel linear
 * index (0..511), index[e] = its MC cube index (never 0 or 255).  Only nonzero indices are
 * stored.  Records and entries are in no particular order.  *n_blocks_dev and *n_entries_dev
 * receive the totals produced; when they exceed the capacities the excess is not written. */
typedef struct {
  int32_t* keys3;
  uint32_t* info;
  uint32_t* offsets;
  uint32_t* counts;
  uint16_t* local;
  uint8_t* index;
  uint32_t cap_blocks;
  uint32_t cap_entries;
  uint32_t* n_blocks_dev;
  uint32_t* n_entries_dev;
} vbh_mc_stream;

/* Marching Cubes index extraction (Sec. 4.2).  Corner i of the cube at voxel g is g + c_i with
 * c = (000, 100, 110, 010, 001, 101, 111, 011) (x fastest); bit i is set iff the TSDF at that
 * corner is < 0; a cube with a corner in a missing block or with weight 0 gets index 0; indices
 * 0 and 255 are written as 0 and not stored.  In TOUCHED mode the extracted blocks get the
 * version of the last fused frame.  needed_bytes_host may be NULL (asynchronous); otherwise the
 * call synchronises, stores the bytes the stream needed, and returns VBH_ERR_BUFFER_TOO_SMALL
 * if a capacity was exceeded. */
vbh_status vbh_extract_mc_indices(vbh_handle* h, const vbh_mc_selector* sel_host,
                                  const vbh_mc_stream* out, uint64_t* needed_bytes_host);

/* One whole frame in one call: vbh_erase_blocks(RADIUS, camera position, erase_radius) (skipped
 * when erase_radius == 0), vbh_integrate_frame(depth, T_wc, frame_id) and
 * vbh_extract_mc_indices(VBH_MC_TOUCHED, out) -- the reconstruction client's per-frame update
 * and the server's MC conversion of Sec. 4.1-4.2 -- with the same results as those three calls.
 * The first call captures the frame's kernels as a CUDA graph on a private stream; every call
 * then updates the graph's per-frame inputs and launches it on the handle's stream, so a frame
 * costs two driver calls on the host.  Arguments as for the three calls; the erased keys are not
 * reported individually (the stream's removal records carry them).  Asynchronous. */
vbh_status vbh_process_frame(vbh_handle* h, const uint16_t* depth_dev, const float* T_wc_host,
                             uint32_t frame_id, float erase_radius, const vbh_mc_stream* out);

/* Host-side output of a frame: caller-owned host memory (pinned -- cudaHostAlloc or
 * cudaHostRegister -- lets the copy overlap the next frame), arrays as in vbh_mc_stream with
 * capacities cap_blocks / cap_entries.  n_blocks, n_entries, frame_id and done are written by
 * the library once the frame's results are complete: the totals the frame produced (when they
 * exceed the capacities only the first cap_* records / entries are copied, and the call that
 * completes the frame returns VBH_ERR_BUFFER_TOO_SMALL), the frame's id, and done = 1. */
typedef struct {
  int32_t* keys3;      /* cap_blocks x 3 */
  uint32_t* info;      /* cap_blocks */
  uint32_t* offsets;   /* cap_blocks */
  uint32_t* counts;    /* cap_blocks */
  uint16_t* local;     /* cap_entries */
  uint8_t* index;      /* cap_entries */
  uint32_t cap_blocks;
  uint32_t cap_entries;
  uint32_t n_blocks;   /* out */
  uint32_t n_entries;  /* out */
  uint32_t frame_id;   /* out */
  uint32_t done;       /* out: 0 while the frame is in flight, 1 once complete */
} vbh_mc_stream_host;

/* vbh_process_frame with host buffers, pipelined (Sec. 4.1-4.2 per frame, as vbh_process_frame):
 * the depth image is copied from host memory (depth_host: width x height uint16, reusable when
 * the call returns), the frame runs on one of three library-owned device streams, and its MC
 * stream is copied into out_host while the next frames are computed.  The call enqueues this
 * frame, starts the copy-out of the previous call's frame if that frame has finished, and
 * returns once the frame of TWO calls earlier is complete in its out_host (its `done` set; the
 * status of that completion is returned: VBH_ERR_BUFFER_TOO_SMALL if it was cut); it waits for
 * the GPU only when the GPU is two frames behind.  vbh_process_frame_host_flush completes every
 * frame still pending.  Each out_host must stay valid until its frame is done.  vbh_destroy
 * waits for the frames in flight but does not complete frames that were not flushed (their
 * `done` stays 0). */
vbh_status vbh_process_frame_host(vbh_handle* h, const uint16_t* depth_host,
                                  const float* T_wc_host, uint32_t frame_id, float erase_radius,
                                  vbh_mc_stream_host* out_host);
vbh_status vbh_process_frame_host_flush(vbh_handle* h);

/* Host copies of the live blocks (test and checkpoint path; synchronises).  keys3_host: cap
 * keys; tsdf_host, weight_host: cap*512 floats each (may be NULL); vals_host: cap uint32 (the
 * value of each key: pool index or the plain map's value; may be NULL); *n_host = live keys
 * (the first min(cap, live) are written, in no particular order). */
vbh_status vbh_dump(vbh_handle* h, int32_t* keys3_host, float* tsdf_host, float* weight_host,
                    uint32_t* vals_host, uint32_t cap, uint32_t* n_host);
/* Insert (or overwrite) n blocks with the given voxel values (synchronises). */
vbh_status vbh_load(vbh_handle* h, const int32_t* keys3_host, const float* tsdf_host,
                    const float* weight_host, uint32_t n);

vbh_status vbh_get_counters(vbh_handle* h, vbh_counters* out_host);
vbh_status vbh_clear_errors(vbh_handle* h);

/* Bounded device waits (failure detection; the paper states none).  The fusion kernel waits for
 * each block's asynchronous voxel copy with at most `polls` polls (default 2^24); a wait that
 * runs out raises error flag bit3, the warp drains its copy (bounded) and stops, the frame's
 * remaining voxels of that warp are left unfused, and vbh_integrate_frame with stats_host
 * returns VBH_ERR_TIMEOUT.  The flag is sticky until vbh_clear_errors; the handle stays usable.
 * polls = 0 makes every such wait give up at once (fault injection for tests).  Takes effect
 * from the next frame call. */
vbh_status vbh_set_wait_limit(vbh_handle* h, uint32_t polls);

/* Per-stage device timing: CUDA events are recorded on the handle's stream around each stage
 * whose bit (1 << stage) is set in `stage_mask` (0 = off).  vbh_timing_read synchronises and
 * returns, per stage since the last reset, the accumulated milliseconds of the timed stages and
 * the kernel launches of every stage. */
enum { VBH_STAGE_ERASE = 0, VBH_STAGE_ALLOC = 1, VBH_STAGE_INTEGRATE = 2, VBH_STAGE_MCSET = 3,
       VBH_STAGE_MC = 4, VBH_STAGE_HASH = 5, VBH_N_STAGES = 6 };
vbh_status vbh_timing_enable(vbh_handle* h, int stage_mask);
vbh_status vbh_timing_read(vbh_handle* h, double* ms_host /* VBH_N_STAGES */,
                           uint64_t* launches_host /* VBH_N_STAGES */, int reset);

/* Differentiable window fusion -- forward and hand-written backward of the fusion of Sec. 4.1
 * with respect to per-pixel depth and per-frame pose (an extension: the paper has no backward
 * pass).  A window of n_frames float32 metric depth images (0 = invalid) is fused at fixed
 * sample voxels g (world position g s); F(g) = mean over its valid frames of
 * clamp(sdf / trunc, -1, 1), sdf = D(u, v) - p_z with D bilinear in the depth; L = sum F^2.
 * Pose f is exp(xi_f) for an se(3) vector xi = (rho, omega) (rotation vector omega,
 * t = V(omega) rho).  Validity and the bilinear cell of every (sample, frame) are fixed at
 * nominal float32 poses T0 (3x4 row-major [R | t]) by canonical binary32 decisions (a cell is
 * valid when its four depths are > 0 and span at most trunc, and its bilinear sdf >= -trunc;
 * the term is live, f = sdf / trunc, when that sdf < trunc, else saturated, f = 1), so L is
 * smooth in (xi, depth) and the backward pass is exact for it; projections are recomputed in
 * the backward pass, not stored.  All pointers are caller-owned device memory; calls are
 * asynchronous on the handle's stream. */
typedef struct {
  float voxel_size, trunc;
  int32_t width, height;
  float fx, fy, cx, cy;
  uint32_t n_frames;             /* 1..256 */
} vbh_diff_config;
typedef struct vbh_diff vbh_diff;
vbh_status vbh_diff_create(const vbh_diff_config* cfg, void* cuda_stream, vbh_diff** out);
vbh_status vbh_diff_destroy(vbh_diff* d);
/* exp of n_frames se(3) vectors xi_dev (n_frames x 6 float: rho, omega) into T_dev
 * (n_frames x 12 float, [R | t]); T_dev may be NULL (the handle keeps the pose derivatives). */
vbh_status vbh_diff_poses(vbh_diff* d, const float* xi_dev, float* T_dev);
/* masks_dev: n x ceil(n_frames / 32) uint32, bit f of sample i set iff frame f is valid. */
vbh_status vbh_diff_masks(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                          const float* depth_dev, const float* T0_dev, uint32_t* masks_dev);
/* F_dev: n floats; loss_dev: one double (may be NULL). */
vbh_status vbh_diff_forward(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                            const float* depth_dev, const float* T0_dev, const float* xi_dev,
                            const uint32_t* masks_dev, float* F_dev, double* loss_dev);
/* dL/d depth into gdepth_dev (n_frames x height x width floats, overwritten) and dL/d xi into
 * gxi_dev (n_frames x 6 floats), given F_dev from the forward pass at the same xi. */
vbh_status vbh_diff_backward(vbh_diff* d, const int32_t* samples_dev, uint32_t n,
                             const float* depth_dev, const float* T0_dev, const float* xi_dev,
                             const uint32_t* masks_dev, const float* F_dev, float* gdepth_dev,
                             float* gxi_dev);

/* Marching Cubes indices of a caller's TSDF blocks, allocating nothing.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc -- code that runs inside another
 * framework's memory pool, real-time threads that must not risk an allocation's device-wide
 * synchronisation, hosts that reserve all memory at start-up -- and therefore cannot create a
 * vbh_handle.  It computes, for every input block, the stream record that
 * vbh_extract_mc_indices(VBH_MC_ALL) would produce for a volume holding exactly these blocks
 * (same corner order, S^c rule and compaction; info = 0), on `cuda_stream`.
 *   keys3_dev: n_blocks distinct block coordinates in [-2^20, 2^20); tsdf_dev, weight_dev:
 *   n_blocks * 512 floats each (voxel lx + 8 ly + 64 lz); out: as for vbh_extract_mc_indices;
 *   error_flags_dev (may be NULL): one uint32 that receives bit0 = a key out of range, bit1 = a
 *   repeated key, bit2 = the stream's capacity was exceeded (records beyond cap_blocks or
 *   entries beyond cap_entries are not written; a record whose entries did not fit keeps its
 *   offset and count, so offset + count > cap_entries: check this bit or the totals before
 *   reading entries).  All pointers are caller-owned device memory.
 * Scratch: a fixed 8 MiB + 256 B array in the library's device memory (every GPU that loads
 * the library holds it until exit); n_blocks is limited to 32768 and larger sizes return
 * VBH_ERR_INVALID_ARG without touching the device.  The call issues only memsets, kernels and a
 * device-to-device copy; it never calls cudaMalloc or cudaFree.  The first call on a device
 * looks up the array's device address on that device (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The address is kept for the life
 * of the process: do not use this entry point again on a device after cudaDeviceReset.  Every
 * call reuses the same array, so calls whose work overlaps on the GPU race: serialise them. */
vbh_status vbh_mc_from_tsdf_static(const int32_t* keys3_dev, const float* tsdf_dev,
                                   const float* weight_dev, uint32_t n_blocks,
                                   const vbh_mc_stream* out, void* cuda_stream,
                                   uint32_t* error_flags_dev);

/* Stream-out of blocks that leave the active model (Sec. 4.1: blocks no longer in the
 * sensor's view move to CPU memory) into a passive host map, and explicit stream-in.
 * After vbh_stream_out_enable, every erase (vbh_erase_blocks, and the erase step of
 * vbh_process_frame) copies the removed blocks' (TSDF, weight) and keys into a device transfer
 * ring of ring_blocks slots (0 = max_blocks) before their pool entries can be reused; copies to
 * pinned host memory run on a side stream and are folded into the host map -- key -> the
 * block's values at its last erase -- by the polls that every frame / erase call makes.  A
 * ring without room loses nothing silently: the blocks that did not fit are counted
 * (vbh_stream_out_stats) and error flag 16 is raised; the poll waits for copies while the ring
 * is more than half full.  Host memory: 4 KiB per slot pinned plus the map. */
vbh_status vbh_stream_out_enable(vbh_handle* h, uint32_t ring_blocks);   /* synchronises */
/* Non-blocking: start copies of filled slots, fold landed ones; *streamed_host (may be NULL)
 * = blocks folded into the host map so far. */
vbh_status vbh_stream_out_poll(vbh_handle* h, uint64_t* streamed_host);
/* Synchronises: every block erased so far is in the host map. */
vbh_status vbh_stream_out_flush(vbh_handle* h);
/* Synchronises; any pointer may be NULL: blocks folded in so far, blocks lost for want of ring
 * room, keys held by the host map. */
vbh_status vbh_stream_out_stats(vbh_handle* h, uint64_t* streamed_host, uint64_t* lost_host,
                                uint32_t* host_blocks_host);
/* The host map (synchronises): first min(cap, size) keys with their 512 TSDF / weight values
 * (tsdf_host, weight_host may be NULL), no particular order; *n_host = size. */
vbh_status vbh_host_map_dump(vbh_handle* h, int32_t* keys3_host, float* tsdf_host,
                             float* weight_host, uint32_t cap, uint32_t* n_host);
/* Stream-in (synchronises): every listed key that is in the host map and not live moves back
 * into the volume with its stored values (a live block is newer: it and its host copy stay);
 * *n_loaded_host (may be NULL) = blocks moved. */
vbh_status vbh_stream_in(vbh_handle* h, const int32_t* keys3_host, uint32_t n,
                         uint32_t* n_loaded_host);

/* Multi-client delta streaming: the server side of Sec. 4.2, where each client asks for the MC
 * blocks that changed since its last update (the paper keeps a hash set of changed block ids
 * per client and hands out capped random subsets; here each client holds one change sequence
 * number on the device, and requests are served by continuous batching).
 *
 * Change sequence.  While a server is attached, every MC refresh of a block -- the extraction
 * of a fused frame, vbh_process_frame or vbh_extract_mc_indices(VBH_MC_TOUCHED) -- gives the
 * block the next change sequence number and keeps its 512 dense cube indices; every removal
 * record gets a number too.  sigma is the last number assigned.  Attaching refreshes every
 * live block once.  Explicit-key, all and since extractions do not refresh.
 *
 * Result of a request of client c, admitted at snapshot sigma while c is at version v:
 *   - v > 0 and every change record after v still in the log: one record per block whose
 *     newest refresh has a number in (v, sigma] (info = the block's frame version, with its
 *     dense cube indices as of that refresh), and one per key whose newest removal has a number
 *     in (v, sigma] and that is not live (info = VBH_REC_REMOVED | frame of the removal, no
 *     indices); afterwards c is at sigma;
 *   - v = 0 (a new or reconnecting client) or records lost from the log: flag VBH_SERVE_RESET
 *     and one record per live block whose newest refresh is at or before sigma (a full model);
 *     afterwards c is at sigma.
 * Blocks refreshed after sigma are left to the client's next request.  A request is admitted
 * only after the same client's previous one completed; records come in no particular order.
 * A request whose worst case exceeds the whole budget is cut at the largest range that fits
 * (VBH_SERVE_PARTIAL; c moves to the end of that range).
 *
 * Serving loop (continuous batching).  vbh_serve_submit queues a request; each vbh_serve_step
 * retires the iterations that finished and, while fewer than max_inflight are queued, launches
 * one more: pending requests are admitted in arrival order while a slot is free (at most
 * max_batch requests in flight) and their worst-case output -- one 528 B record per change
 * record in their range, or per pool entry for a reset -- fits in the budget_bytes stream
 * buffer (a request that does not fit may be passed by later ones for bypass_iters
 * iterations); each admitted request then contributes a chunk of at most chunk_records change
 * records (0 = all) to the iteration, at most iter_records in total (oldest first; 0 = no
 * limit), and the whole batch is one persistent extraction/compaction launch on the volume
 * handle's stream, ordered with its frames.  max_batch = 1 with chunk_records = 0 serves one
 * request per launch (unbatched).
 *
 * Output of a completed request (vbh_serve_result): n_records headers of four int32 (x, y, z,
 * info as uint32 bits), then n_records x 512 cube indices (voxel lx + 8 ly + 64 lz; not written
 * for removal records), in the server's stream buffer until vbh_serve_release.
 * The server object is used from the handle's host thread; the handle must outlive it. */
enum { VBH_SERVE_RESET = 1u, VBH_SERVE_PARTIAL = 2u, VBH_SERVE_ERR_OVERRUN = 4u,
       VBH_SERVE_ERR_CAPACITY = 8u, VBH_SERVE_ERR_VERSION = 16u };
typedef struct {
  uint32_t n_clients;
  uint32_t max_batch;       /* requests in flight at once, 1..64 */
  uint32_t chunk_records;   /* change records per request per iteration (0 = no limit) */
  uint32_t iter_records;    /* change records per iteration (0 = no limit) */
  uint32_t max_inflight;    /* iterations queued on the stream at once (0 = 2) */
  uint32_t bypass_iters;    /* iterations a memory-blocked request may be passed */
  uint32_t log_bits;        /* change log of 2^log_bits records (0 = 22; >= 4 x max_blocks) */
  uint32_t rem_bits;        /* removal table of 2^rem_bits keys (0 = 22) */
  uint64_t budget_bytes;    /* stream buffer (>= 528 x max_blocks) */
} vbh_serve_config;
typedef struct {
  uint32_t id, client;
  uint32_t v_before, v_after;   /* client version before and after the request */
  uint32_t n_records, flags;    /* VBH_SERVE_* bits */
  uint64_t t_arrival_ns, t_admit_ns, t_done_ns;   /* vbh_serve_now_ns() clock */
  uint64_t bytes_reserved;
} vbh_serve_done;
typedef struct {
  const int32_t* recs_dev;      /* n_records x 4 */
  const uint8_t* indices_dev;   /* n_records x 512 */
  uint32_t n_records, flags;
} vbh_serve_view;
typedef struct {
  uint64_t iterations, requests_done, records_served, changes_scanned;
  uint64_t bytes_in_use, bytes_peak, deferred_memory;
  uint32_t err_flags;           /* kernel-side errors (removal table full ...) */
  uint32_t sigma;
} vbh_serve_stats;
/* A timed script for vbh_serve_run: events at t_ns (ascending, ns after the start); client >= 0
 * is a request of that client, -1 the next frame (vbh_process_frame with depth_dev[i], T_wc +
 * 12 i, frame_id[i], erase_radius, frame_out). */
typedef struct {
  uint32_t n_events;
  const uint64_t* t_ns;
  const int32_t* client;
  const uint16_t* const* depth_dev;
  const float* T_wc;
  const uint32_t* frame_id;
  float erase_radius;
  const vbh_mc_stream* frame_out;
} vbh_serve_script;
typedef struct vbh_serve vbh_serve;
/* Attach a server to a volume handle and refresh every live block (synchronises). */
vbh_status vbh_serve_create(vbh_handle* h, const vbh_serve_config* cfg, vbh_serve** out);
vbh_status vbh_serve_destroy(vbh_serve* s);
/* Change the scheduling fields (max_batch, chunk_records, iter_records, max_inflight,
 * bypass_iters) of an idle server. */
vbh_status vbh_serve_set_policy(vbh_serve* s, const vbh_serve_config* cfg);
/* Set / read client versions (synchronise; set only for clients without a request). */
vbh_status vbh_serve_set_versions(vbh_serve* s, const uint32_t* clients_host,
                                  const uint32_t* versions_host, uint32_t n);
vbh_status vbh_serve_get_versions(vbh_serve* s, uint32_t* versions_host /* n_clients */);
/* For each backlog b, the version v at which exactly min(b, live) live blocks have newer
 * refreshes (synchronises). */
vbh_status vbh_serve_versions_for_backlog(vbh_serve* s, const uint32_t* backlog_host, uint32_t n,
                                          uint32_t* versions_host);
vbh_status vbh_serve_submit(vbh_serve* s, uint32_t client, uint64_t t_arrival_ns /* 0 = now */,
                            uint32_t* id_host);
vbh_status vbh_serve_step(vbh_serve* s, uint32_t* launched_host /* may be NULL */);
/* Completed requests since the last poll (at most cap; the rest stay queued). */
vbh_status vbh_serve_poll(vbh_serve* s, vbh_serve_done* out_host, uint32_t cap, uint32_t* n_host);
vbh_status vbh_serve_result(vbh_serve* s, uint32_t id, vbh_serve_view* out_host);
vbh_status vbh_serve_release(vbh_serve* s, uint32_t id);
/* Step until nothing is pending or running (synchronises). */
vbh_status vbh_serve_drain(vbh_serve* s);
vbh_status vbh_serve_stats_read(vbh_serve* s, vbh_serve_stats* out_host);
/* Run a timed script in real time (frames and request arrivals), releasing every result as it
 * completes; writes the completions (at most cap) to out_host. */
vbh_status vbh_serve_run(vbh_serve* s, const vbh_serve_script* script, vbh_serve_done* out_host,
                         uint32_t cap, uint32_t* n_host);
uint64_t vbh_serve_now_ns(void);

/* Device-resident request loop (the same requests and results as above, Sec. 4.2 serving): one
 * persistent, cooperatively launched kernel on a library-owned non-blocking stream admits,
 * batches and serves requests while frames keep running on the volume's stream.
 *   - Requests go from the host into a ring in mapped host memory (id, client); the kernel's
 *     scheduler warp reads them, keeps every client's version and "request in flight" state on
 *     the device only, admits requests in arrival order (one per client at a time) when a slot
 *     (max_slots) is free and their worst case -- one 528 B record per change record of the
 *     range, or per pool entry for a reset -- fits in the server's budget_bytes stream buffer
 *     (a ring allocator over it; a memory-blocked request may be passed by later ones for
 *     bypass_rounds scheduler rounds), cuts the admitted ranges into chunks of chunk_records
 *     and hands chunks of all active requests out in rounds, smallest remainder first, as the
 *     workers drain them (continuous batching: a request that arrives while others run joins
 *     the next round).  Worker warps take tiles of 32 change records (64 while the request
 *     has at least 4096 left) by ticket, copy each current block's 512 cube indices and its
 *     header, and the warp that finishes a request's last tile moves
 *     the client to its new version and publishes the completion in mapped host memory.
 *   - Results are those of vbh_serve_step's requests, with sigma the last change number
 *     published when the request is admitted.  A block refreshed again while it is being
 *     copied is dropped from that result (its newer refresh is after sigma and goes to the
 *     client's next request), so concurrent frames never yield a torn block.
 *   - Every device wait is bounded: the scheduler stops the loop with VBH_ERR_TIMEOUT when the
 *     host has given no sign of life (no loop call) for idle_timeout_us; workers stop when the
 *     scheduler's heartbeat stalls.  While a loop runs, the volume's table rebuilds are
 *     deferred, the server's host scheduler calls (vbh_serve_submit / _step / _drain / _run /
 *     _set_versions / _set_policy) return VBH_ERR_UNSUPPORTED, and a device-wide
 *     synchronisation (cudaDeviceSynchronize, cudaFree) waits until the loop stops.
 * The loop object is used from one host thread. */
typedef struct {
  uint32_t ctas;             /* CTAs of 256 threads (0 = one per SM); all co-resident */
  uint32_t max_slots;        /* requests in flight at once, 1..64 (0 = 64) */
  uint32_t chunk_records;    /* change records per chunk (0 = 4096) */
  uint32_t bypass_rounds;    /* scheduler rounds a memory-blocked head may be passed */
  uint32_t ring;             /* request / completion ring entries, a power of two (0 = 4096) */
  uint32_t idle_timeout_us;  /* host silence that stops the loop (0 = 1000000) */
} vbh_serve_loop_config;
typedef struct {
  uint64_t requests_done, records_served, change_records_scanned, chunks, rounds;
  uint64_t deferred_memory;  /* admission attempts refused for want of stream buffer */
  uint64_t bytes_in_use, bytes_peak;
  uint32_t max_active;       /* most requests in flight at once */
  uint32_t status;           /* 0 running / stopped cleanly, else the vbh_status it stopped with */
  uint32_t launches;         /* kernel launches of the loop (1 per start) */
} vbh_serve_loop_stats;
typedef struct vbh_serve_loop vbh_serve_loop;
/* Start the loop (the server must be idle; synchronises the volume's stream first). */
vbh_status vbh_serve_loop_start(vbh_serve* s, const vbh_serve_loop_config* cfg,
                                vbh_serve_loop** out);
/* Queue a request (no device call); VBH_ERR_CAPACITY when the ring is full, VBH_ERR_TIMEOUT
 * if the loop has stopped by itself. */
vbh_status vbh_serve_loop_submit(vbh_serve_loop* L, uint32_t client, uint64_t t_arrival_ns,
                                 uint32_t* id_host);
/* Completions published since the last poll (at most cap; t_done_ns = when this poll saw
 * them; admission happens on the device, so t_admit_ns = t_done_ns minus the GPU timer's
 * interval from the request's admission to its publication, at least t_arrival_ns; a request
 * completed without work at admission has t_admit_ns = t_done_ns). */
vbh_status vbh_serve_loop_poll(vbh_serve_loop* L, vbh_serve_done* out_host, uint32_t cap,
                               uint32_t* n_host);
/* A completed request's records (device pointers into the stream buffer, valid until it is
 * released); release hands its region back to the device allocator. */
vbh_status vbh_serve_loop_result(vbh_serve_loop* L, uint32_t id, vbh_serve_view* out_host);
vbh_status vbh_serve_loop_release(vbh_serve_loop* L, uint32_t id);
/* Wait (bounded) until every submitted request has completed; VBH_ERR_TIMEOUT otherwise. */
vbh_status vbh_serve_loop_drain(vbh_serve_loop* L, uint64_t timeout_ns);
/* Real-time script as for vbh_serve_run (frames on the volume's stream, requests into the
 * loop), releasing every result as it completes. */
vbh_status vbh_serve_loop_run(vbh_serve_loop* L, const vbh_serve_script* script,
                              vbh_serve_done* out_host, uint32_t cap, uint32_t* n_host);
vbh_status vbh_serve_loop_stats_read(vbh_serve_loop* L, vbh_serve_loop_stats* out_host);
/* Stop the loop and free it: returns VBH_OK, or the status the loop stopped with by itself
 * (VBH_ERR_TIMEOUT after host silence); requests not completed are dropped. */
vbh_status vbh_serve_loop_stop(vbh_serve_loop* L);

/* Marching Cubes triangulation of an MC stream (Sec. 4.3: an exploration client builds its
 * mesh from the indices, vertices at edge midpoints, no interpolation).  The triangle table is
 * derived from the cube cases: corner i = (000, 100, 110, 010, 001, 101, 111, 011)[i] (bit i
 * set = TSDF < 0), edges 0-11 join corners (0,1) (1,2) (2,3) (3,0) (4,5) (5,6) (6,7) (7,4)
 * (0,4) (1,5) (2,6) (3,7); on each face, walked counter-clockwise from outside, a crossing out
 * of the inside joins the crossing into it that precedes it (ambiguous faces keep inside
 * corners apart); the joins close into loops, cut by ear clipping without diagonals on a
 * face; normals point to positive TSDF.  At most 5 triangles per index.
 * vbh_mc_tri_table (host only): n_host[256] triangle counts, edges_host[256 * 15] edge triples.
 * vbh_mc_triangulate: every entry of the device stream `in` (as written by
 * vbh_extract_mc_indices) becomes its triangles, 9 floats each (three vertices, metres: the
 * edge midpoints of the cube at voxel g, (g + m) * voxel_size), in no particular order;
 * *n_tris_dev (device) = triangles produced (the first cap_tris are written).  Asynchronous on
 * cuda_stream; allocates nothing (the table goes to constant memory at the first call). */
vbh_status vbh_mc_tri_table(uint8_t* n_host, uint8_t* edges_host);
vbh_status vbh_mc_triangulate(const vbh_mc_stream* in, float voxel_size, float* tris_dev,
                              uint32_t cap_tris, uint32_t* n_tris_dev, void* cuda_stream);

/* Per-client stream sets -- the paper's own serving design (Sec. 4.2), beside the version
 * server for comparison: each client has a hash set of queued block keys (2^cap_log2 slots);
 * vbh_sets_insert_last inserts the last extraction's refreshed blocks and removal keys into
 * every client's set (one launch over clients x blocks); vbh_sets_fill queues every live
 * block for one client (a (re)connect); vbh_sets_fetch serves n_req requests (distinct
 * clients, limits 1..1024) in one launch: each takes a random subset of at most its limit out
 * of its client's set by concurrent removal and writes, from record offset sum(limits before
 * it), headers (x, y, z, info: the block's frame version, or VBH_REC_REMOVED when it is not
 * live) into recs_dev (4 int32 each) and the block's dense cube indices (from the server's
 * store) into indices_dev (512 B each); n_out_dev[i] = records of request i.  Asynchronous on
 * the volume's stream, except vbh_sets_counts (synchronises).  The server and its volume must
 * outlive the sets. */
typedef struct vbh_sets vbh_sets;
vbh_status vbh_sets_create(vbh_serve* s, uint32_t n_clients, uint32_t cap_log2, vbh_sets** out);
vbh_status vbh_sets_destroy(vbh_sets* q);
vbh_status vbh_sets_insert_last(vbh_sets* q);
vbh_status vbh_sets_fill(vbh_sets* q, uint32_t client);
vbh_status vbh_sets_fetch(vbh_sets* q, const uint32_t* clients_host, const uint32_t* limits_host,
                          uint32_t n_req, int32_t* recs_dev, uint8_t* indices_dev,
                          uint32_t* n_out_dev);
/* queued keys and tombstones per client (n_clients each; may be NULL), error bits (bit0: a
 * set was full; may be NULL). */
vbh_status vbh_sets_counts(vbh_sets* q, uint32_t* queued_host, uint32_t* tombs_host,
                           uint32_t* err_host);
/* Rebuild one client's set without tombstones. */
vbh_status vbh_sets_rebuild(vbh_sets* q, uint32_t client);

/* Host-side helpers (no device work). */
int vbh_abi_version(void);
const char* vbh_last_error(void);
/* The bucket a key maps to under `hash_fn` for a table of n_buckets (power of two). */
uint32_t vbh_bucket_of(int32_t x, int32_t y, int32_t z, uint32_t n_buckets, uint32_t hash_fn);

#ifdef __cplusplus
}
#endif
#endif /* VBH_H_ */
