// Batched culling: many frames (each its own eyes, hierarchy, tile, tau and output) culled
// by a few persistent traversal launches, optionally recorded once into a CUDA graph and
// replayed.
//
// A frame with enough eyes to fill the GPU by itself (kOwnLaunchEyes) gets a launch of its
// own, which runs the single-frame kernel (its frame fields are kernel parameters in
// registers); consecutive smaller frames share a batched launch of up to
// HRR_CULL_MAX_FRAMES frames, whose warps look their frame up by eye. Launches alternate
// between the context stream and a second stream of the batch, each with its own stack
// spill area, so a launch's first blocks fill the SMs its predecessor's last eyes leave
// idle; the second stream joins the context stream at the end.
//
// A batch keeps its frame descriptors on the host (they travel as kernel parameters) and its
// per-frame counters, the launches' eye cursors and the device flags in device memory.
// Replaying it resets the counters and runs every launch.
#include <algorithm>
#include <new>
#include <vector>

#include "hrr_internal.cuh"

struct hrr_batch {
    uint32_t n_frames = 0;
    unsigned long long total = 0;
    hrr_tuning tuning{};
    std::vector<hrr_cull_frame_t> desc;         // cursor offsets restart in every launch
    struct Part {
        uint32_t first = 0, count = 0;          // frames [first, first + count)
        unsigned long long total = 0;           // their eyes
        unsigned grid = 1;
    };
    std::vector<Part> parts;                    // one traversal launch each
    uint32_t spill_cap = 0;                     // stack spill entries per warp
    void *spill[2] = {};                        // stack spill area per stream (two launches may overlap)
    cudaStream_t side = nullptr;                // second stream (launches 1, 3, 5, ...)
    cudaEvent_t fork = nullptr, join = nullptr; // side stream starts after the counter reset, ends before results
    unsigned long long *dev_counts = nullptr;  // 2 per frame (accepted, visits), a cursor per part, flags
    unsigned long long *host_counts = nullptr; // pinned mirror
    std::vector<uint64_t> caps;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    hrr_tile_buf *ctx_tile = nullptr;           // the context tile the frames read, if any (a reference)
    cudaStream_t stream = nullptr;              // the context stream (runs the batch)

    size_t n_counters() const { return 2 * (size_t)n_frames + parts.size() + 1; }
};

namespace {

// Frames with at least this many eyes fill the GPU (152 SMs x 48 resident warps, one eye per
// warp, several eyes per warp over a launch) and run as launches of their own.
constexpr uint64_t kOwnLaunchEyes = 1u << 16;

int enqueue(hrr_ctx *ctx, hrr_batch *b, cudaStream_t st) {
    HRR_CUDA(ctx, cudaMemsetAsync(b->dev_counts, 0, sizeof(unsigned long long) * b->n_counters(), st));
    unsigned long long *cursors = b->dev_counts + 2 * (size_t)b->n_frames;
    unsigned long long *flags = cursors + b->parts.size();
    const bool two = b->parts.size() > 1;
    if (two) {
        HRR_CUDA(ctx, cudaEventRecord(b->fork, st));
        HRR_CUDA(ctx, cudaStreamWaitEvent(b->side, b->fork, 0));
    }
    for (size_t p = 0; p < b->parts.size(); ++p) {
        const hrr_batch::Part &pt = b->parts[p];
        const int k = two ? (int)(p & 1) : 0;
        HRR_CUDA(ctx, hrr_cull_batch_enqueue(pt.grid, b->desc.data() + pt.first, pt.count, pt.total, cursors + p,
                                             flags, b->spill[k], b->spill_cap, b->tuning, k ? b->side : st));
        if (pt.total) ++ctx->launches;
    }
    if (two) {
        HRR_CUDA(ctx, cudaEventRecord(b->join, b->side));
        HRR_CUDA(ctx, cudaStreamWaitEvent(st, b->join, 0));
    }
    return HRR_OK;
}

void release(hrr_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->dev_counts) cudaFree(b->dev_counts);
    if (b->host_counts) cudaFreeHost(b->host_counts);
    for (void *sp : b->spill)
        if (sp) cudaFree(sp);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->side) cudaStreamDestroy(b->side);
    hrr_tile_release(b->ctx_tile, b->stream);
    delete b;
}

}  // namespace

extern "C" {

int hrr_batch_create(hrr_ctx *ctx, const hrr_frame *frames, uint32_t n_frames, const hrr_tuning *tuning,
                     int use_graph, hrr_batch **out) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!frames || n_frames == 0 || n_frames > 65535)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "n_frames must be in [1, 65535]");
    const hrr_tuning tn = tuning ? *tuning : hrr_tuning{};
    if (!hrr_tuning_valid(tn)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "invalid tuning");
    hrr_batch *b = new (std::nothrow) hrr_batch();
    if (!b) return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the batch");
    b->n_frames = n_frames;
    b->tuning = hrr_tuning_normalized(tn);
    b->caps.resize(n_frames);
    b->desc.resize(n_frames);
    b->stream = ctx->stream;
    DeviceGuard g(ctx->device);
    unsigned long long cursor = 0;
    uint32_t height = 0;
    for (uint32_t i = 0; i < n_frames; ++i) {
        const hrr_frame &fr = frames[i];
        const char *bad = nullptr;
        int status = HRR_ERR_INVALID_ARG;
        if (!fr.tree || fr.tree->device != ctx->device) bad = "a frame's tree is NULL or on another device";
        else if (!(fr.tau >= 0.0f) || !(fr.tau < __builtin_huge_valf())) bad = "a frame's tau is not finite and >= 0";
        else if (fr.n_eyes && (!fr.eyes.x || !fr.eyes.y || !fr.eyes.z || !fr.eyes.px || !fr.eyes.py))
            bad = "a frame's eye array is NULL";
        else if (fr.cap && !fr.dev_pairs) bad = "a frame's dev_pairs is NULL";
        else if (((uintptr_t)fr.dev_pairs & 7u) != 0) bad = "a frame's dev_pairs is not 8-byte aligned";
        else if (fr.dev_tile && (fr.tile_w == 0 || fr.tile_h == 0 || fr.tile_w > 65536 || fr.tile_h > 65536 ||
                                 fr.tile_d > 65536))
            bad = "a frame's tile size is invalid";
        else if (!fr.dev_tile && !ctx->tile) {
            bad = "a frame has no tile and no context tile is set";
            status = HRR_ERR_NO_TILE;
        }
        if (bad) {
            release(b);
            return hrr_fail(ctx, status, bad);
        }
        // A new launch for a frame that fills the GPU, after one, or when the current
        // shared launch is full (frames or eyes).
        const bool big = fr.n_eyes >= kOwnLaunchEyes;
        if (b->parts.empty() || big || b->parts.back().count == HRR_CULL_MAX_FRAMES ||
            b->parts.back().total >= kOwnLaunchEyes) {
            b->parts.push_back(hrr_batch::Part{});
            b->parts.back().first = i;
            cursor = 0;
        }
        if (!fr.dev_tile && !b->ctx_tile) {  // keep the context tile alive while the batch exists
            b->ctx_tile = ctx->tile_buf;
            hrr_tile_retain(b->ctx_tile);
        }
        hrr_batch::Part &pt = b->parts.back();
        hrr_cull_frame_t &d = b->desc[i];
        d = hrr_cull_frame_t{};
        d.ex = fr.eyes.x; d.ey = fr.eyes.y; d.ez = fr.eyes.z; d.px = fr.eyes.px; d.py = fr.eyes.py;
        d.nodes = hrr_cull_records(fr.tree, b->tuning);
        if (!d.nodes) {
            release(b);
            return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a frame's tree has no records of the tuning's node width");
        }
        d.perm = fr.tree->perm;
        d.tile = fr.dev_tile ? hrr_tile_layer(fr.dev_tile, fr.tile_w, fr.tile_h, fr.tile_d, fr.sample_index)
                             : hrr_tile_layer(ctx->tile, ctx->tile_w, ctx->tile_h, ctx->tile_d, fr.sample_index);
        d.tile_w = fr.dev_tile ? fr.tile_w : ctx->tile_w;
        d.tile_h = fr.dev_tile ? fr.tile_h : ctx->tile_h;
        d.pairs = reinterpret_cast<uint2 *>(fr.dev_pairs);
        d.cap = fr.cap;
        d.eye_visits = fr.eye_visits;
        d.n_lights = fr.tree->n;
        d.shift_offset = fr.shift_offset;
        d.tau = fr.tau;
        d.eye_begin = 0;
        d.cursor_begin = cursor;
        cursor += fr.n_eyes;
        ++pt.count;
        pt.total = cursor;
        b->total += fr.n_eyes;
        b->caps[i] = fr.cap;
        height = std::max(height, fr.tree->height);
    }
    unsigned grid_max = 1;
    for (hrr_batch::Part &pt : b->parts) {
        pt.grid = hrr_cull_grid(ctx->sm_count, b->tuning, true, pt.total);
        grid_max = std::max(grid_max, pt.grid);
    }
    b->spill_cap = hrr_cull_spill_cap(height, b->tuning.node_width);
    const size_t spill_bytes = hrr_cull_spill_entries(grid_max, height, b->tuning) * sizeof(uint2);
    cudaError_t e = cudaMalloc(&b->spill[0], spill_bytes);
    if (e == cudaSuccess && b->parts.size() > 1) e = cudaMalloc(&b->spill[1], spill_bytes);
    if (e == cudaSuccess && b->parts.size() > 1) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->dev_counts, sizeof(unsigned long long) * b->n_counters());
    if (e == cudaSuccess) e = cudaMallocHost(&b->host_counts, sizeof(unsigned long long) * b->n_counters());
    if (e != cudaSuccess) {
        release(b);
        return hrr_cuda_fail(ctx, e, "batch allocation");
    }
    for (uint32_t i = 0; i < n_frames; ++i) b->desc[i].counts = b->dev_counts + 2 * (size_t)i;
    if (use_graph) {
        // Record [reset counters, traversal] once on a private stream; replays go to ctx->stream.
        cudaGraph_t graph = nullptr;
        e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const uint64_t launches = ctx->launches;
            const int st = enqueue(ctx, b, b->capture_stream);
            ctx->launches = launches;  // recording is not a launch
            const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &graph);
            e = st != HRR_OK ? cudaErrorUnknown : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            release(b);
            return hrr_cuda_fail(ctx, e, "batch graph capture");
        }
    }
    *out = b;
    return HRR_OK;
}

int hrr_batch_launch(hrr_ctx *ctx, hrr_batch *b) {
    if (!ctx || !b) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (b->exec) {
        HRR_CUDA(ctx, cudaGraphLaunch(b->exec, ctx->stream));
        for (const hrr_batch::Part &pt : b->parts) ctx->launches += pt.total ? 1 : 0;
        return HRR_OK;
    }
    return enqueue(ctx, b, ctx->stream);
}

int hrr_batch_results(hrr_ctx *ctx, hrr_batch *b, uint64_t *counts, uint64_t *visits) {
    if (!ctx || !b) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t n = b->n_counters();
    HRR_CUDA(ctx, cudaMemcpyAsync(b->host_counts, b->dev_counts, sizeof(unsigned long long) * n,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bool overflow = false;
    uint64_t acc = 0, vis = 0;
    for (uint32_t i = 0; i < b->n_frames; ++i) {
        const uint64_t c = b->host_counts[2 * (size_t)i];
        if (counts) counts[i] = c;
        if (visits) visits[i] = b->host_counts[2 * (size_t)i + 1];
        if (c > b->caps[i]) overflow = true;
        acc += c;
        vis += b->host_counts[2 * (size_t)i + 1];
    }
    ctx->last_accepted = acc;
    ctx->last_visits = vis;
    const unsigned long long flags = b->host_counts[n - 1];
    if (flags & HRR_FLAG_STACK) return hrr_fail(ctx, HRR_ERR_DEVICE, "traversal stack overflow");
    if (flags & HRR_FLAG_TOPOLOGY) return hrr_fail(ctx, HRR_ERR_DEVICE, "corrupt node record");
    if (overflow) return hrr_fail(ctx, HRR_ERR_OVERFLOW, "a frame's output capacity is too small");
    return HRR_OK;
}

int hrr_batch_destroy(hrr_ctx *ctx, hrr_batch *b) {
    if (!ctx || !b) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    release(b);
    return HRR_OK;
}

int hrr_cull_batch(hrr_ctx *ctx, const hrr_frame *frames, uint32_t n_frames, const hrr_tuning *tuning,
                   uint64_t *counts) {
    hrr_batch *b = nullptr;
    int st = hrr_batch_create(ctx, frames, n_frames, tuning, 0, &b);
    if (st != HRR_OK) return st;
    st = hrr_batch_launch(ctx, b);
    if (st == HRR_OK) st = hrr_batch_results(ctx, b, counts, nullptr);
    const std::string err = ctx->err;
    hrr_batch_destroy(ctx, b);
    ctx->err = err;
    return st;
}

}  // extern "C"
