// C ABI entry points: contexts, errors, shift tiles, argument checks and dispatch to the
// build / cull / range-minimum implementations.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "hrr_internal.cuh"

int hrr_fail(hrr_ctx *ctx, int status, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return status;
}

int hrr_cuda_fail(hrr_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    int st = (e == cudaErrorMemoryAllocation) ? HRR_ERR_OOM : HRR_ERR_CUDA;
    return hrr_fail(ctx, st, m);
}

void hrr_timing_begin(hrr_ctx *ctx) {
    if (!ctx->timing) return;
    cudaEvent_t a, b;
    if (ctx->ev_pool.size() >= 2) {
        a = ctx->ev_pool.back(); ctx->ev_pool.pop_back();
        b = ctx->ev_pool.back(); ctx->ev_pool.pop_back();
    } else {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    cudaEventRecord(a, ctx->stream);
    ctx->ev_start.push_back(a);
    ctx->ev_stop.push_back(b);
}

void hrr_timing_end(hrr_ctx *ctx) {
    if (!ctx->timing || ctx->ev_stop.empty()) return;
    cudaEventRecord(ctx->ev_stop.back(), ctx->stream);
}

static void release_events(hrr_ctx *ctx) {
    for (auto e : ctx->ev_start) ctx->ev_pool.push_back(e);
    for (auto e : ctx->ev_stop) ctx->ev_pool.push_back(e);
    ctx->ev_start.clear();
    ctx->ev_stop.clear();
}

extern "C" {

const char *hrr_status_string(int s) {
    switch (s) {
    case HRR_OK: return "HRR_OK";
    case HRR_ERR_INVALID_ARG: return "HRR_ERR_INVALID_ARG";
    case HRR_ERR_OOM: return "HRR_ERR_OOM";
    case HRR_ERR_NO_TILE: return "HRR_ERR_NO_TILE";
    case HRR_ERR_OVERFLOW: return "HRR_ERR_OVERFLOW";
    case HRR_ERR_TIMEOUT: return "HRR_ERR_TIMEOUT";
    case HRR_ERR_CUDA: return "HRR_ERR_CUDA";
    case HRR_ERR_DEVICE: return "HRR_ERR_DEVICE";
    case HRR_PENDING: return "HRR_PENDING";
    default: return "HRR_UNKNOWN_STATUS";
    }
}

const char *hrr_last_error(const hrr_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int hrr_default_tuning(hrr_tuning *out) {
    if (!out) return HRR_ERR_INVALID_ARG;
    *out = hrr_tuning_normalized(hrr_tuning{});
    return HRR_OK;
}

int hrr_create(hrr_ctx **out, int device, void *cuda_stream) {
    if (!out) return HRR_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev)
        return HRR_ERR_INVALID_ARG;
    hrr_ctx *ctx = new (std::nothrow) hrr_ctx();
    if (!ctx) return HRR_ERR_OOM;
    ctx->device = device;
    DeviceGuard g(device);
    if (!g.ok) { delete ctx; return HRR_ERR_CUDA; }
    int st = HRR_OK;
    do {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { st = HRR_ERR_CUDA; break; }
            ctx->own_stream = true;
        }
        if (cudaMalloc(&ctx->counters, 8 * sizeof(unsigned long long)) != cudaSuccess) { st = HRR_ERR_OOM; break; }
        if (cudaMallocHost(&ctx->host_counters, 8 * sizeof(unsigned long long)) != cudaSuccess) { st = HRR_ERR_OOM; break; }
        if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) { st = HRR_ERR_CUDA; break; }
    } while (0);
    if (st != HRR_OK) {
        hrr_destroy(ctx);
        return st;
    }
    *out = ctx;
    return HRR_OK;
}

int hrr_destroy(hrr_ctx *ctx) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    release_events(ctx);
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    hrr_tile_release(ctx->tile_buf, ctx->stream);  // batches or jobs may still hold it
    ctx->tile_buf = nullptr;
    ctx->tile = nullptr;
    if (ctx->counters) cudaFree(ctx->counters);
    if (ctx->host_counters) cudaFreeHost(ctx->host_counters);
    if (ctx->spill) cudaFree(ctx->spill);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->stream2) cudaStreamSynchronize(ctx->stream2);
    if (ctx->host_eyes_dev) cudaFree(ctx->host_eyes_dev);
    if (ctx->host_pairs_dev) cudaFree(ctx->host_pairs_dev);
    if (ctx->host_lights_dev) cudaFree(ctx->host_lights_dev);
    if (ctx->slice_counters) cudaFree(ctx->slice_counters);
    if (ctx->sample_counters) cudaFree(ctx->sample_counters);
    if (ctx->ev_first) cudaEventDestroy(ctx->ev_first);
    for (int i = 0; i < HRR_HOST_SLICES; ++i) {
        if (ctx->ev_in[i]) cudaEventDestroy(ctx->ev_in[i]);
        if (ctx->ev_done[i]) cudaEventDestroy(ctx->ev_done[i]);
        if (ctx->ev_out[i]) cudaEventDestroy(ctx->ev_out[i]);
    }
    if (ctx->host_slices) cudaFreeHost(ctx->host_slices);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return HRR_OK;
}

int hrr_launch_count(const hrr_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return HRR_ERR_INVALID_ARG;
    *out = ctx->launches;
    return HRR_OK;
}

int hrr_set_timing(hrr_ctx *ctx, int enable) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    release_events(ctx);
    ctx->timing = enable != 0;
    return HRR_OK;
}

int hrr_kernel_time(hrr_ctx *ctx, double *ms, uint64_t *launches) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double total = 0.0;
    for (size_t k = 0; k < ctx->ev_start.size(); ++k) {
        float t = 0.0f;
        HRR_CUDA(ctx, cudaEventElapsedTime(&t, ctx->ev_start[k], ctx->ev_stop[k]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = ctx->ev_start.size();
    return HRR_OK;
}

int hrr_build_light_tree(hrr_ctx *ctx, hrr_lights lights, uint32_t n_lights, hrr_tree **out) {
    return hrr_build_light_tree_ex(ctx, lights, n_lights, nullptr, out);
}

int hrr_build_light_tree_ex(hrr_ctx *ctx, hrr_lights lights, uint32_t n_lights, const hrr_build_opts *opts,
                            hrr_tree **out) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    const int topology = opts ? opts->topology : HRR_TOPOLOGY_RADIX;
    if (topology != HRR_TOPOLOGY_RADIX && topology != HRR_TOPOLOGY_COST)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "unknown topology");
    const uint32_t cost_depth = opts && opts->cost_depth ? opts->cost_depth : 48u;
    if (cost_depth > 64u) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "cost_depth must be in [0, 64]");
    if (!out) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_lights == 0 || n_lights > 0x7FFFFFFFu)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "n_lights must be in [1, 2^31 - 1]");
    if (!lights.x || !lights.y || !lights.z || !lights.intensity)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a light array is NULL");
    DeviceGuard g(ctx->device);
    return hrr_build_impl(ctx, lights, n_lights, out, topology, cost_depth);
}

int hrr_build_light_tree_host(hrr_ctx *ctx, hrr_lights H, uint32_t n_lights, const hrr_build_opts *opts,
                              hrr_tree **out) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_lights == 0 || n_lights > 0x7FFFFFFFu)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "n_lights must be in [1, 2^31 - 1]");
    if (!H.x || !H.y || !H.z || !H.intensity) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a light array is NULL");
    DeviceGuard g(ctx->device);
    const size_t stride = ((sizeof(float) * (size_t)n_lights + 255) & ~size_t(255)) / sizeof(float);
    if (ctx->host_lights_cap < n_lights) {
        HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->host_lights_dev) cudaFree(ctx->host_lights_dev);
        ctx->host_lights_dev = nullptr;
        ctx->host_lights_cap = 0;
        if (cudaMalloc(&ctx->host_lights_dev, 4 * sizeof(float) * stride) != cudaSuccess) {
            cudaGetLastError();
            return hrr_fail(ctx, HRR_ERR_OOM, "device staging area of the lights");
        }
        ctx->host_lights_cap = stride;
    }
    float *d = static_cast<float *>(ctx->host_lights_dev);
    const size_t cap = ctx->host_lights_cap;  // floats per array in the staging area
    const float *src[4] = {H.x, H.y, H.z, H.intensity};
    for (int k = 0; k < 4; ++k)
        HRR_CUDA(ctx, cudaMemcpyAsync(d + k * cap, src[k], sizeof(float) * (size_t)n_lights,
                                      cudaMemcpyHostToDevice, ctx->stream));
    const hrr_lights D{d, d + cap, d + 2 * cap, d + 3 * cap};
    return hrr_build_light_tree_ex(ctx, D, n_lights, opts, out);
}

int hrr_free_light_tree(hrr_ctx *ctx, hrr_tree *tree) {
    if (!ctx || !tree) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (tree->nodes) HRR_CUDA(ctx, cudaFreeAsync(tree->nodes, ctx->stream));
    if (tree->perm) HRR_CUDA(ctx, cudaFreeAsync(tree->perm, ctx->stream));
    if (tree->wide) HRR_CUDA(ctx, cudaFreeAsync(tree->wide, ctx->stream));
    delete tree;
    return HRR_OK;
}

int hrr_tree_perm(const hrr_tree *tree, const uint32_t **dev_perm) {
    if (!tree || !dev_perm) return HRR_ERR_INVALID_ARG;
    *dev_perm = tree->perm;
    return HRR_OK;
}

int hrr_tree_info(const hrr_tree *tree, uint32_t *n_lights, uint32_t *height,
                  const hrr_node **dev_nodes) {
    if (!tree) return HRR_ERR_INVALID_ARG;
    if (n_lights) *n_lights = tree->n;
    if (height) *height = tree->height;
    if (dev_nodes) *dev_nodes = tree->n > 1 ? tree->nodes : nullptr;
    return HRR_OK;
}

int hrr_tree_download(hrr_ctx *ctx, const hrr_tree *tree, hrr_node *host_nodes,
                      uint32_t *host_perm) {
    if (!ctx || !tree) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (host_nodes && tree->n > 1)
        HRR_CUDA(ctx, cudaMemcpyAsync(host_nodes, tree->nodes, sizeof(hrr_node) * (size_t)(tree->n - 1),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    if (host_perm)
        HRR_CUDA(ctx, cudaMemcpyAsync(host_perm, tree->perm, sizeof(uint32_t) * (size_t)tree->n,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HRR_OK;
}

int hrr_refit_light_tree(hrr_ctx *ctx, hrr_tree *tree, hrr_lights lights) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!tree || tree->device != ctx->device) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree is NULL or on another device");
    if (!lights.x || !lights.y || !lights.z || !lights.intensity)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a light array is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    unsigned long long *flags = ctx->counters + 2;
    HRR_CUDA(ctx, cudaMemsetAsync(flags, 0, sizeof(unsigned long long), st));
    void *scratch = nullptr;
    HRR_CUDA(ctx, cudaMallocAsync(&scratch, hrr_refit_scratch_bytes(tree->n), st));
    const cudaError_t e = hrr_refit_enqueue(tree, lights, scratch, flags, st);
    ctx->launches += hrr_refit_launches(tree);
    cudaFreeAsync(scratch, st);
    HRR_CUDA(ctx, e);
    HRR_CUDA(ctx, cudaMemcpyAsync(&ctx->host_counters[2], flags, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->host_counters[2] & HRR_FLAG_NONFINITE)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a light position or intensity is not finite");
    if (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY) return hrr_fail(ctx, HRR_ERR_DEVICE, "inconsistent tree records");
    return HRR_OK;
}

int hrr_set_shift_tile_3d(hrr_ctx *ctx, const uint32_t *host_tile, uint32_t w, uint32_t h, uint32_t d) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!host_tile || w == 0 || h == 0 || d == 0 || w > 65536 || h > 65536 || d > 65536 ||
        (uint64_t)w * h * d > (1ull << 30))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tile must be non-empty, w, h, d <= 65536, w*h*d <= 2^30");
    DeviceGuard g(ctx->device);
    const size_t bytes = sizeof(uint32_t) * (size_t)w * h * d;
    uint32_t *dev = nullptr;
    HRR_CUDA(ctx, cudaMallocAsync(&dev, bytes, ctx->stream));
    cudaError_t e = cudaMemcpyAsync(dev, host_tile, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dev, ctx->stream);
        return hrr_cuda_fail(ctx, e, "copy of the shift tile");
    }
    hrr_tile_buf *buf = new (std::nothrow) hrr_tile_buf();
    if (!buf) {
        cudaFreeAsync(dev, ctx->stream);
        return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the tile");
    }
    buf->dev = dev;
    // The old tile lives on while a batch or a served job still holds a reference to it.
    hrr_tile_release(ctx->tile_buf, ctx->stream);
    ctx->tile_buf = buf;
    ctx->tile = dev;
    ctx->tile_w = w;
    ctx->tile_h = h;
    ctx->tile_d = d;
    return HRR_OK;
}

int hrr_set_shift_tile(hrr_ctx *ctx, const uint32_t *host_tile, uint32_t w, uint32_t h) {
    return hrr_set_shift_tile_3d(ctx, host_tile, w, h, 1);
}

int hrr_cull_ex(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                const hrr_cull_opts *opts, uint32_t *dev_pairs, uint64_t cap,
                uint64_t *out_count) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out_count) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out_count is NULL");
    *out_count = 0;
    if (!tree) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree is NULL");
    if (tree->device != ctx->device) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree lives on another device");
    if (!(tau >= 0.0f) || !std::isfinite(tau)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (n_eyes > 0 && (!eyes.x || !eyes.y || !eyes.z || !eyes.px || !eyes.py))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "an eye array is NULL");
    if (cap > 0 && !dev_pairs) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs is NULL");
    if (!ctx->tile) return hrr_fail(ctx, HRR_ERR_NO_TILE, "no shift tile set");
    hrr_cull_opts o{};
    if (opts) o = *opts;
    if (!hrr_tuning_valid(hrr_tuning_of(o)))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG,
                        "rangemin_variant must be 0 or 2, blocks_per_sm <= 64, node_width 2 or 4, "
                        "threads_per_block 128 or 256, ring_entries 128/256 (width 2) or 256/512 (width 4)");
    DeviceGuard g(ctx->device);
    return hrr_cull_impl(ctx, eyes, n_eyes, tree, tau, o, dev_pairs, cap, out_count);
}

int hrr_cull(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
             uint32_t *dev_pairs, uint64_t cap, uint64_t *out_count) {
    return hrr_cull_ex(ctx, eyes, n_eyes, tree, tau, nullptr, dev_pairs, cap, out_count);
}

int hrr_cull_samples(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                     const uint32_t *offsets, uint32_t n_samples, uint32_t *dev_pairs, uint64_t cap,
                     uint64_t *out_counts, uint64_t *out_visits) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out_counts) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out_counts is NULL");
    if (n_samples < 1 || n_samples > 32) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "n_samples must be in [1, 32]");
    for (uint32_t s = 0; s < n_samples; ++s) out_counts[s] = 0;
    if (!offsets) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "offsets is NULL");
    if (!tree) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree is NULL");
    if (tree->device != ctx->device) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree lives on another device");
    if (!(tau >= 0.0f) || !std::isfinite(tau)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (n_eyes > 0 && (!eyes.x || !eyes.y || !eyes.z || !eyes.px || !eyes.py))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "an eye array is NULL");
    if (cap > 0 && !dev_pairs) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs is NULL");
    if (cap > (~0ull / 8) / 32) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "cap too large");
    if (!ctx->tile) return hrr_fail(ctx, HRR_ERR_NO_TILE, "no shift tile set");
    DeviceGuard g(ctx->device);
    return hrr_cull_samples_impl(ctx, eyes, n_eyes, tree, tau, offsets, n_samples, dev_pairs, cap, out_counts,
                                 out_visits);
}

int hrr_cull_host(hrr_ctx *ctx, hrr_eyes host_eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                  const hrr_cull_opts *opts, uint32_t *host_pairs, uint64_t cap, uint64_t *out_count) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out_count) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out_count is NULL");
    *out_count = 0;
    if (!tree) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree is NULL");
    if (tree->device != ctx->device) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tree lives on another device");
    if (!(tau >= 0.0f) || !std::isfinite(tau)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (n_eyes > 0 && (!host_eyes.x || !host_eyes.y || !host_eyes.z || !host_eyes.px || !host_eyes.py))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "an eye array is NULL");
    if (cap > 0 && !host_pairs) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "host_pairs is NULL");
    if (!ctx->tile) return hrr_fail(ctx, HRR_ERR_NO_TILE, "no shift tile set");
    hrr_cull_opts o{};
    if (opts) o = *opts;
    if (!hrr_tuning_valid(hrr_tuning_of(o)))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG,
                        "rangemin_variant must be 0 or 2, blocks_per_sm <= 64, node_width 2 or 4, "
                        "threads_per_block 128 or 256, ring_entries 128/256 (width 2) or 256/512 (width 4)");
    DeviceGuard g(ctx->device);
    return hrr_cull_host_impl(ctx, host_eyes, n_eyes, tree, tau, o, host_pairs, cap, out_count);
}

int hrr_last_cull_stats(const hrr_ctx *ctx, uint64_t *visits, uint64_t *accepted) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (visits) *visits = ctx->last_visits;
    if (accepted) *accepted = ctx->last_accepted;
    return HRR_OK;
}

int hrr_range_min(hrr_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *r,
                  uint32_t *out_min, uint32_t *out_argmin, uint64_t n, int variant) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (n == 0) return HRR_OK;
    if (!a || !b || !r || !out_min) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "NULL array");
    if (variant != 0 && variant != 2) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "variant must be 0 or 2");
    DeviceGuard g(ctx->device);
    return hrr_range_min_impl(ctx, a, b, r, out_min, out_argmin, n, variant);
}

}  // extern "C"
