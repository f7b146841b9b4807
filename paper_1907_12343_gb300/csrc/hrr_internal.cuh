// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "hrr.h"

// ------------------------------------------------------------------------------------
// Host-side objects
// ------------------------------------------------------------------------------------

// Most slices hrr_cull_host splits the eyes into.
#define HRR_HOST_SLICES 8

// A library-owned shift tile, shared by reference: the context holds one reference, and
// every batch or served job that reads the context's tile holds another until its GPU
// work is over. A new hrr_set_shift_tile drops the context's reference only, so a batch's
// recorded graph or a job in flight keeps reading the tile it was created with.
struct hrr_tile_buf {
    uint32_t *dev = nullptr;
    std::atomic<int> refs{1};
};
inline void hrr_tile_retain(hrr_tile_buf *t) {
    if (t) t->refs.fetch_add(1, std::memory_order_relaxed);
}
// Drops one reference; the last one frees the tile, ordered after the work on `st` (every
// holder releases only once no GPU work of its own reads the tile).
inline void hrr_tile_release(hrr_tile_buf *t, cudaStream_t st) {
    if (t && t->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        if (t->dev) cudaFreeAsync(t->dev, st);
        delete t;
    }
}

struct hrr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // shift tile (library-owned copy, shared by reference; tile == tile_buf->dev)
    hrr_tile_buf *tile_buf = nullptr;
    uint32_t *tile = nullptr;
    uint32_t tile_w = 0, tile_h = 0, tile_d = 1;  // d layers of w x h (a space-time tile)
    // device counters of the last cull: [0] accepted pairs, [1] node visits, [2] flags,
    // [3] work cursor
    unsigned long long *counters = nullptr;
    unsigned long long *host_counters = nullptr;  // pinned mirror
    uint64_t last_visits = 0, last_accepted = 0;
    uint64_t launches = 0;
    // optional traversal-kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_start, ev_stop;  // recorded pairs, in order
    std::vector<cudaEvent_t> ev_pool;
    int sm_count = 0;
    // traversal stack spill area (grown on demand by hrr_cull)
    void *spill = nullptr;
    size_t spill_entries = 0;
    // hrr_cull_host: device copies of the eyes and two pair buffers (grown on demand), a
    // second compute stream and a copy stream, per-slice events and counters (device and
    // pinned), all created on first use
    void *host_eyes_dev = nullptr;
    size_t host_eyes_cap = 0;  // eyes
    void *host_pairs_dev = nullptr;
    size_t host_pairs_cap = 0;  // pairs per buffer
    // hrr_build_light_tree_host: device staging area for host lights (x, y, z, intensity)
    void *host_lights_dev = nullptr;
    size_t host_lights_cap = 0;  // lights
    cudaStream_t stream2 = nullptr, copy_stream = nullptr;
    cudaEvent_t ev_first = nullptr;
    cudaEvent_t ev_in[HRR_HOST_SLICES] = {}, ev_done[HRR_HOST_SLICES] = {}, ev_out[HRR_HOST_SLICES] = {};
    unsigned long long *slice_counters = nullptr;  // device, 4 per slice
    unsigned long long *sample_counters = nullptr;  // hrr_cull_samples: 40 device counters
    unsigned long long *host_slices = nullptr;     // pinned, 4 per slice
    std::string err;
};

// The top of a hierarchy, which the traversal's head evaluates from shared memory: the
// nodes of depth 0 .. HRR_TOP_LEVELS - 1 in heap order (slot 0 the root, the children of
// slot s in slots 2s + 1 and 2s + 2), three float4 per slot:
//   (box low corner, maximum intensity), (box high corner, first leaf as bits),
//   (last leaf as bits, node index as bits, kind as bits, 0)
// with kind HRR_TOP_EMPTY (no node: below a leaf), HRR_TOP_INTERNAL or HRR_TOP_LEAF (a light:
// its position and intensity, first = last = its sorted position). The root's box is not
// stored (the root is never tested). The slots follow the tree's binary records in the same
// allocation, at float4 offset 4 (n - 1).
#define HRR_TOP_LEVELS 6u
#define HRR_TOP_SLOTS 63u  // 2^HRR_TOP_LEVELS - 1
#define HRR_TOP_BYTES (HRR_TOP_SLOTS * 3u * 16u)
enum : uint32_t { HRR_TOP_EMPTY = 0u, HRR_TOP_INTERNAL = 1u, HRR_TOP_LEAF = 2u };

struct hrr_tree {
    int device = 0;
    uint32_t n = 0;
    uint32_t height = 0;
    // n - 1 records (one record with the single leaf if n == 1), followed by the top slots
    hrr_node *nodes = nullptr;
    uint32_t *perm = nullptr;   // n
    // The same hierarchy read with nodes of width four: for every internal node g a
    // 128-byte record of its four grandchild slots (hrr_derived_enqueue), at index g; a
    // traversal of width four reads the even-depth ones only. One record (the leaf in
    // slot 0) when n == 1.
    float4 *wide = nullptr;
};

// Fill the records derived from the binary ones: the top slots after tree->nodes, and
// tree->wide if the tree has it (one thread per internal node); skipped when *flags holds
// HRR_FLAG_NONFINITE (a failed refit leaves the hierarchy as it was).
cudaError_t hrr_derived_enqueue(hrr_tree *tree, const unsigned long long *flags, cudaStream_t st);
// Kernels hrr_derived_enqueue launches for the tree.
inline int hrr_derived_launches(const hrr_tree *tree) { return tree->wide ? 2 : 1; }
// Kernels a refit launches (hrr_refit_enqueue).
inline int hrr_refit_launches(const hrr_tree *tree) { return (tree->n > 1 ? 3 : 1) + hrr_derived_launches(tree); }

// Layer (sample mod d) of a w x h x d tile: the shifts one culling pass uses.
inline const uint32_t *hrr_tile_layer(const uint32_t *tile, uint32_t w, uint32_t h, uint32_t d,
                                      uint32_t sample) {
    return tile + (size_t)(sample % (d ? d : 1u)) * w * h;
}

// Status helpers (hrr_abi.cu)
int hrr_fail(hrr_ctx *ctx, int status, const std::string &msg);
int hrr_cuda_fail(hrr_ctx *ctx, cudaError_t e, const char *what);

#define HRR_CUDA(ctx, call)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return hrr_cuda_fail((ctx), e_, #call); \
    } while (0)

// RAII device selection for an API call
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// One frame of a traversal launch, as the kernel reads it (hrr_cull_kernel.cuh): a single frame
// for hrr_cull, an array of them for batches. 128 bytes.
struct hrr_cull_frame_t {
    const float *ex, *ey, *ez;
    const uint16_t *px, *py;
    const float4 *nodes;
    const uint32_t *perm;
    const uint32_t *tile;
    uint2 *pairs;
    unsigned long long cap;
    unsigned long long *counts;      // [0] accepted pairs, [1] node visits
    uint32_t *eye_visits;            // optional per-eye visit counts
    uint32_t n_lights, tile_w, tile_h, shift_offset;
    float tau;
    uint32_t eye_begin;              // first eye of the frame covered by this launch
    unsigned long long cursor_begin; // where the frame's eyes start on the launch's cursor
};

// Traversal defaults (the fastest form on the 1920x1080-eye, 2^20-light frame): node width,
// shared-memory stack ring per warp, threads per block, top levels evaluated from shared
// memory (1: the root only, every level walked).
#define HRR_DEFAULT_NODE_WIDTH 2u
#define HRR_DEFAULT_RING 256u
#define HRR_DEFAULT_THREADS 256u
#define HRR_DEFAULT_TOP_LEVELS HRR_TOP_LEVELS

// Launch parameters with the library defaults filled in.
inline hrr_tuning hrr_tuning_normalized(hrr_tuning t) {
    if (!t.node_width) t.node_width = HRR_DEFAULT_NODE_WIDTH;
    if (!t.ring_entries) t.ring_entries = HRR_DEFAULT_RING;
    if (!t.threads_per_block) t.threads_per_block = HRR_DEFAULT_THREADS;
    // the top levels come with binary records only: width four defaults to the root alone
    if (!t.top_levels) t.top_levels = t.node_width == 2 ? HRR_DEFAULT_TOP_LEVELS : 1u;
    return t;
}
// Levels the traversal's head evaluates from shared memory for a normalised tuning (0 = no
// head: the traversal starts at the root).
inline uint32_t hrr_tuning_top(const hrr_tuning &t) { return t.top_levels == 1u ? 0u : t.top_levels; }
inline hrr_tuning hrr_tuning_of(const hrr_cull_opts &o) {
    hrr_tuning t{};
    t.rangemin_variant = o.rangemin_variant;
    t.blocks_per_sm = o.blocks_per_sm;
    t.node_width = o.node_width;
    t.ring_entries = o.ring_entries;
    t.threads_per_block = o.threads_per_block;
    t.top_levels = o.top_levels;
    return hrr_tuning_normalized(t);
}
// Every combination that has a compiled traversal (zero fields stand for the defaults).
inline bool hrr_tuning_valid(const hrr_tuning &t0) {
    const hrr_tuning t = hrr_tuning_normalized(t0);
    if ((t.rangemin_variant != 0 && t.rangemin_variant != 2) || t.blocks_per_sm > 64) return false;
    if (t.threads_per_block != 128 && t.threads_per_block != 256) return false;
    if (t.top_levels != 1u && (t.top_levels != HRR_TOP_LEVELS || t.node_width != 2)) return false;
    if (t.node_width == 2) return t.ring_entries == 128 || t.ring_entries == 256;
    if (t.node_width == 4) return t.ring_entries == 256 || t.ring_entries == 512;
    return false;
}

// The traversal (hrr_cull_kernel.cuh). Frames of one batched launch (their descriptors are
// kernel parameters: 128 x 128 bytes):
#define HRR_CULL_MAX_FRAMES 128u
// Blocks of a traversal launch over `total` eyes (a whole number per SM, at most one warp per
// eye), for the single-frame or the batched kernel of a (normalised, valid) tuning.
unsigned hrr_cull_grid(int sm_count, const hrr_tuning &tuning, bool batch, unsigned long long total);
// Resident blocks per SM of the traversal kernel of a (normalised, valid) tuning.
int hrr_cull_max_blocks(const hrr_tuning &tuning, bool batch);
// Stack entries per warp that the spill area must hold for trees of the given height read
// with the given node width (the proven bound plus a margin), and the area's entries
// (8 bytes each) for a grid of the tuning's blocks.
uint32_t hrr_cull_spill_cap(uint32_t height, uint32_t width);
size_t hrr_cull_spill_entries(unsigned grid, uint32_t height, const hrr_tuning &tuning);
// The node records a traversal of the tuning's width reads (tree->nodes or tree->wide).
const float4 *hrr_cull_records(const hrr_tree *tree, const hrr_tuning &tuning);
// Enqueue one batched traversal over n_frames <= HRR_CULL_MAX_FRAMES frames (host array, copied
// into the launch) on st; a no-op when total == 0. A single frame runs the single-frame
// kernel (same results, frame fields in registers). The cursor and flags must be zero when the
// kernel starts. spill holds hrr_cull_spill_entries(grid, height) entries for the tallest tree
// of the frames, spill_cap = hrr_cull_spill_cap(height, tuning.node_width).
cudaError_t hrr_cull_batch_enqueue(unsigned grid, const hrr_cull_frame_t *frames, uint32_t n_frames,
                                   unsigned long long total, unsigned long long *cursor,
                                   unsigned long long *flags, void *spill, uint32_t spill_cap,
                                   const hrr_tuning &tuning, cudaStream_t st);

// Traversal timing (hrr_abi.cu)
void hrr_timing_begin(hrr_ctx *ctx);
void hrr_timing_end(hrr_ctx *ctx);

// Refit of a hierarchy for moved lights (hrr_build.cu): scratch of
// hrr_refit_scratch_bytes(tree->n) bytes (256-byte aligned); *flags must be zero and gets
// HRR_FLAG_NONFINITE (the hierarchy is then left unchanged) or HRR_FLAG_TOPOLOGY.
size_t hrr_refit_scratch_bytes(uint32_t n);
cudaError_t hrr_refit_enqueue(hrr_tree *tree, const hrr_lights &lights, void *scratch, unsigned long long *flags,
                              cudaStream_t st);

// Entry points implemented per translation unit
int hrr_build_impl(hrr_ctx *ctx, const hrr_lights &lights, uint32_t n, hrr_tree **out,
                   int topology = HRR_TOPOLOGY_RADIX, uint32_t cost_depth = 48);
int hrr_cull_impl(hrr_ctx *ctx, const hrr_eyes &eyes, uint32_t n_eyes, const hrr_tree *tree,
                  float tau, const hrr_cull_opts &opts, uint32_t *pairs, uint64_t cap,
                  uint64_t *out_count);
int hrr_cull_samples_impl(hrr_ctx *ctx, const hrr_eyes &eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                          const uint32_t *offsets, uint32_t n_samples, uint32_t *pairs, uint64_t cap,
                          uint64_t *out_counts, uint64_t *out_visits);
int hrr_cull_host_impl(hrr_ctx *ctx, const hrr_eyes &host_eyes, uint32_t n_eyes, const hrr_tree *tree,
                       float tau, const hrr_cull_opts &opts, uint32_t *host_pairs, uint64_t cap,
                       uint64_t *out_count);
int hrr_range_min_impl(hrr_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *r,
                       uint32_t *out_min, uint32_t *out_argmin, uint64_t n, int variant);

#include "hrr_math.cuh"
