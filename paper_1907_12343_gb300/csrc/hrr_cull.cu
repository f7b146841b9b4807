// Host entry points of the culling (Sec. 1): single frames, host buffers and batches;
// the traversal itself is in hrr_cull_kernel.cuh.
#include <algorithm>
#include <mutex>
#include <vector>

#include "hrr_cull_kernel.cuh"

namespace {

// ------------------------------------------------------------------------------------
// Instantiations and their dispatch
// ------------------------------------------------------------------------------------

// One compiled form of the traversal: range-minimum variant, node width, ring entries per
// warp, threads per block and top levels evaluated by the head, with its single-frame and
// batched kernels.
struct CullKernel {
    int variant, width, ring, threads, top;
    const void *single, *batch;
    int occ[2];  // resident blocks per SM (single, batched), 0 until first asked
};

template <int VARIANT, int W, int RING, int THREADS, int TOP>
CullKernel cull_entry() {
    return {VARIANT, W, RING, THREADS, TOP,
            reinterpret_cast<const void *>(cull_single_kernel<VARIANT, W, RING, THREADS, TOP>),
            reinterpret_cast<const void *>(cull_batch_kernel<VARIANT, W, RING, THREADS, TOP>), {0, 0}};
}

template <int VARIANT>
void add_entries(std::vector<CullKernel> &v) {
    constexpr int T = (int)HRR_TOP_LEVELS;
    v.push_back(cull_entry<VARIANT, 2, 256, 256, 0>());
    v.push_back(cull_entry<VARIANT, 2, 128, 256, 0>());
    v.push_back(cull_entry<VARIANT, 2, 256, 128, 0>());
    v.push_back(cull_entry<VARIANT, 2, 128, 128, 0>());
    v.push_back(cull_entry<VARIANT, 2, 256, 256, T>());
    v.push_back(cull_entry<VARIANT, 2, 128, 256, T>());
    v.push_back(cull_entry<VARIANT, 2, 256, 128, T>());
    v.push_back(cull_entry<VARIANT, 2, 128, 128, T>());
    v.push_back(cull_entry<VARIANT, 4, 256, 256, 0>());
    v.push_back(cull_entry<VARIANT, 4, 512, 256, 0>());
    v.push_back(cull_entry<VARIANT, 4, 256, 128, 0>());
    v.push_back(cull_entry<VARIANT, 4, 512, 128, 0>());
}

std::vector<CullKernel> &cull_kernels() {
    static std::vector<CullKernel> v = [] {
        std::vector<CullKernel> t;
        add_entries<0>(t);
        add_entries<2>(t);
        return t;
    }();
    return v;
}

// The compiled form for a normalised tuning (nullptr if there is none).
CullKernel *cull_kernel_for(const hrr_tuning &t) {
    for (CullKernel &k : cull_kernels())
        if (k.variant == t.rangemin_variant && k.width == (int)t.node_width && k.ring == (int)t.ring_entries &&
            k.threads == (int)t.threads_per_block && k.top == (int)hrr_tuning_top(t))
            return &k;
    return nullptr;
}

// The first call per form asks the runtime; the server's scheduler thread and a caller's
// thread may both get here, so the cache is filled under a lock.
int cull_occupancy(CullKernel &k, bool batch) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int &n = k.occ[batch ? 1 : 0];
    if (!n) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, batch ? k.batch : k.single, k.threads, 0) !=
                cudaSuccess || m < 1) {
            cudaGetLastError();
            m = 1;
        }
        n = m;
    }
    return n;
}

cudaError_t launch_single(CullKernel &k, unsigned grid, const Launch &Lc, const Frame &fr, cudaStream_t st) {
    Launch lc = Lc;
    Frame f = fr;
    void *args[] = {&lc, &f};
    return cudaLaunchKernel(k.single, dim3(grid), dim3(k.threads), args, 0, st);
}

cudaError_t launch_batch(CullKernel &k, unsigned grid, const Launch &Lc, const FrameArray<kMaxFrames> &fa,
                         cudaStream_t st) {
    Launch lc = Lc;
    void *args[] = {&lc, const_cast<FrameArray<kMaxFrames> *>(&fa)};
    return cudaLaunchKernel(k.batch, dim3(grid), dim3(k.threads), args, 0, st);
}

}  // namespace


unsigned hrr_cull_grid(int sm_count, const hrr_tuning &tuning, bool batch, unsigned long long total) {
    CullKernel *k = cull_kernel_for(tuning);
    if (!k) return 1;
    int per_sm = cull_occupancy(*k, batch);
    if (tuning.blocks_per_sm > 0 && (int)tuning.blocks_per_sm < per_sm) per_sm = (int)tuning.blocks_per_sm;
    const unsigned warps = (unsigned)k->threads / 32u;
    const unsigned long long needed = (total + warps - 1) / warps;
    return (unsigned)std::max<unsigned long long>(1ull, std::min<unsigned long long>((unsigned long long)per_sm * sm_count, needed));
}

int hrr_cull_max_blocks(const hrr_tuning &tuning, bool batch) {
    CullKernel *k = cull_kernel_for(tuning);
    return k ? cull_occupancy(*k, batch) : 0;
}

// The stack of a width-w traversal of a tree of height H holds at most (w - 1) 32 L + 32
// entries, L the depth levels a pushed node can sit at (binary: H - 1; width four: the even
// depths below the root, (H - 1) / 2); the spill writes stay below the stack size.
uint32_t hrr_cull_spill_cap(uint32_t height, uint32_t width) {
    const uint32_t levels = height == 0 ? 0u : (width == 4 ? (height - 1u) / 2u : height - 1u);
    return (width - 1u) * 32u * levels + 32u + 64u;
}

size_t hrr_cull_spill_entries(unsigned grid, uint32_t height, const hrr_tuning &tuning) {
    return (size_t)grid * (tuning.threads_per_block / 32u) * hrr_cull_spill_cap(height, tuning.node_width);
}

const float4 *hrr_cull_records(const hrr_tree *tree, const hrr_tuning &tuning) {
    return tuning.node_width == 4 ? tree->wide : reinterpret_cast<const float4 *>(tree->nodes);
}

namespace {

// Grows the context's stack spill area to hold `need` entries (synchronises the stream first).
int ensure_spill(hrr_ctx *ctx, size_t need) {
    if (need <= ctx->spill_entries) return HRR_OK;
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->spill) cudaFree(ctx->spill);
    ctx->spill = nullptr;
    ctx->spill_entries = 0;
    if (cudaMalloc(&ctx->spill, need * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        return hrr_fail(ctx, HRR_ERR_OOM, "traversal stack spill area");
    }
    ctx->spill_entries = need;
    return HRR_OK;
}

// The single-frame descriptor of one culling launch over eyes [eye_begin, eye_begin + n).
Frame single_frame(const hrr_ctx *ctx, const hrr_eyes &E, const hrr_tree *tree, float tau, const hrr_cull_opts &opts,
                   const hrr_tuning &tn, uint32_t *pairs, uint64_t cap, uint32_t eye_begin) {
    Frame fr{};
    fr.ex = E.x; fr.ey = E.y; fr.ez = E.z; fr.px = E.px; fr.py = E.py;
    fr.nodes = hrr_cull_records(tree, tn);
    fr.perm = tree->perm;
    fr.tile = hrr_tile_layer(ctx->tile, ctx->tile_w, ctx->tile_h, ctx->tile_d, opts.sample_index);
    fr.pairs = reinterpret_cast<uint2 *>(pairs);
    fr.cap = cap;
    fr.counts = ctx->counters;  // [0] accepted, [1] visits
    fr.eye_visits = opts.eye_visits;
    fr.n_lights = tree->n;
    fr.tile_w = ctx->tile_w; fr.tile_h = ctx->tile_h;
    fr.shift_offset = opts.shift_offset;
    fr.tau = tau;
    fr.eye_begin = eye_begin;
    fr.cursor_begin = 0;
    return fr;
}

// Reads the context's counters after a cull (synchronising the stream) and turns them into
// the call's status.
int finish_cull(hrr_ctx *ctx, uint64_t cap, uint64_t *out_count) {
    HRR_CUDA(ctx, cudaMemcpyAsync(ctx->host_counters, ctx->counters, 3 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    HRR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint64_t count = ctx->host_counters[0];
    ctx->last_accepted = count;
    ctx->last_visits = ctx->host_counters[1];
    *out_count = count;
    if (ctx->host_counters[2] & HRR_FLAG_STACK)
        return hrr_fail(ctx, HRR_ERR_DEVICE, "traversal stack overflow");
    if (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY)
        return hrr_fail(ctx, HRR_ERR_DEVICE, "corrupt node record");
    if (count > cap) return hrr_fail(ctx, HRR_ERR_OVERFLOW, "output capacity too small");
    return HRR_OK;
}

}  // namespace

int hrr_cull_impl(hrr_ctx *ctx, const hrr_eyes &E, uint32_t n_eyes, const hrr_tree *tree,
                  float tau, const hrr_cull_opts &opts, uint32_t *pairs, uint64_t cap,
                  uint64_t *out_count) {
    if (((uintptr_t)pairs & 7u) != 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs must be 8-byte aligned");
    const hrr_tuning tn = hrr_tuning_of(opts);
    CullKernel *kern = cull_kernel_for(tn);
    if (!kern) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "no compiled traversal for these options");
    if (!hrr_cull_records(tree, tn)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "the tree has no records of this width");
    cudaStream_t st = ctx->stream;
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(unsigned long long), st));
    if (n_eyes > 0) {
        const unsigned grid = hrr_cull_grid(ctx->sm_count, tn, false, n_eyes);
        if (int rc = ensure_spill(ctx, hrr_cull_spill_entries(grid, tree->height, tn))) return rc;
        const Frame fr = single_frame(ctx, E, tree, tau, opts, tn, pairs, cap, 0);
        const Launch Lc{1, hrr_cull_spill_cap(tree->height, tn.node_width), n_eyes, ctx->counters + 3,
                        ctx->counters + 2, reinterpret_cast<uint2 *>(ctx->spill)};
        hrr_timing_begin(ctx);
        const cudaError_t e = launch_single(*kern, grid, Lc, fr, st);
        hrr_timing_end(ctx);
        ++ctx->launches;
        HRR_CUDA(ctx, e);
    }
    return finish_cull(ctx, cap, out_count);
}

// Eyes from host memory, pairs to host memory. The eyes are culled in up to
// HRR_HOST_SLICES slices, one launch each, alternating between two streams so that a
// slice's blocks fill the SMs its predecessor's last eyes leave idle. Each slice counts
// into its own counters and appends to one of two device pair buffers (slice i to buffer
// i mod 2); the copy stream uploads every slice's eyes first and then downloads each
// slice's pairs, in slice order, once the host has read that slice's count. Slice i + 2
// is enqueued after slice i's download, on which it waits before reusing the buffer.
int hrr_cull_host_impl(hrr_ctx *ctx, const hrr_eyes &H, uint32_t n_eyes, const hrr_tree *tree, float tau,
                       const hrr_cull_opts &opts, uint32_t *host_pairs, uint64_t cap, uint64_t *out_count) {
    cudaStream_t st = ctx->stream;
    if (!ctx->copy_stream) {
        HRR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        HRR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
        HRR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_first, cudaEventDisableTiming));
        for (int i = 0; i < HRR_HOST_SLICES; ++i) {
            HRR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming));
            HRR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming));
            HRR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
        }
        if (cudaMalloc(&ctx->slice_counters, HRR_HOST_SLICES * 4 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&ctx->host_slices, HRR_HOST_SLICES * 4 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return hrr_fail(ctx, HRR_ERR_OOM, "slice counters");
        }
    }
    if (!ctx->host_slices || !ctx->slice_counters) return hrr_fail(ctx, HRR_ERR_OOM, "slice counters");
    // device copies: x, y, z (4 B each) and px, py (2 B each) per eye; two buffers of 8 B pairs
    auto grow = [&](void *&buf, size_t &have, size_t want, size_t unit, const char *what) -> int {
        if (want <= have) return HRR_OK;
        HRR_CUDA(ctx, cudaStreamSynchronize(st));
        if (buf) cudaFree(buf);
        buf = nullptr;
        have = 0;
        if (cudaMalloc(&buf, want * unit + 1024) != cudaSuccess) {
            cudaGetLastError();
            return hrr_fail(ctx, HRR_ERR_OOM, what);
        }
        have = want;
        return HRR_OK;
    };
    if (int rc = grow(ctx->host_eyes_dev, ctx->host_eyes_cap, n_eyes, 16, "device copy of the eyes")) return rc;
    if (int rc = grow(ctx->host_pairs_dev, ctx->host_pairs_cap, cap, 16, "device pair buffers")) return rc;
    char *eb = static_cast<char *>(ctx->host_eyes_dev);
    const size_t ne = ctx->host_eyes_cap;
    auto at = [&](const void *end) {
        const size_t off = (size_t)(static_cast<const char *>(end) - eb);
        return eb + ((off + 255) & ~size_t(255));
    };
    float *dx = reinterpret_cast<float *>(eb);
    float *dy = reinterpret_cast<float *>(at(dx + ne));
    float *dz = reinterpret_cast<float *>(at(dy + ne));
    uint16_t *dpx = reinterpret_cast<uint16_t *>(at(dz + ne));
    uint16_t *dpy = reinterpret_cast<uint16_t *>(at(dpx + ne));
    uint32_t *buf[2] = {static_cast<uint32_t *>(ctx->host_pairs_dev),
                        static_cast<uint32_t *>(ctx->host_pairs_dev) + 2 * ctx->host_pairs_cap};
    const hrr_eyes D{dx, dy, dz, dpx, dpy};

    // slices of about 2^18 eyes or more
    const uint32_t slices = n_eyes == 0 ? 0u : std::max(1u, std::min<uint32_t>(HRR_HOST_SLICES, (n_eyes + (1u << 17)) >> 18));
    const hrr_tuning tn = hrr_tuning_of(opts);
    CullKernel *kern = cull_kernel_for(tn);
    if (!kern) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "no compiled traversal for these options");
    if (!hrr_cull_records(tree, tn)) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "the tree has no records of this width");
    if (slices) {
        const unsigned grid = hrr_cull_grid(ctx->sm_count, tn, false, n_eyes);  // at least any slice's grid
        // two slices may run at once, each with its own spill area
        if (int rc = ensure_spill(ctx, 2 * hrr_cull_spill_entries(grid, tree->height, tn))) return rc;
    }
    cudaStream_t cs[2] = {st, ctx->stream2};
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(unsigned long long), st));
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->slice_counters, 0, HRR_HOST_SLICES * 4 * sizeof(unsigned long long), st));
    HRR_CUDA(ctx, cudaEventRecord(ctx->ev_first, st));
    HRR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream2, ctx->ev_first, 0));
    HRR_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_first, 0));
    // slice i holds a share min(4, slices - i) of the eyes: the last slices shrink, so the
    // download that nothing overlaps (the last slice's pairs) is short
    auto weight_before = [&](uint32_t i) {
        uint64_t w = 0;
        for (uint32_t k = 0; k < i; ++k) w += std::min<uint32_t>(4u, slices - k);
        return w;
    };
    const uint64_t w_all = weight_before(slices);
    auto bounds = [&](uint32_t i, uint32_t &e0, uint32_t &e1) {
        e0 = (uint32_t)((uint64_t)n_eyes * weight_before(i) / std::max<uint64_t>(w_all, 1));
        e1 = (uint32_t)((uint64_t)n_eyes * weight_before(i + 1) / std::max<uint64_t>(w_all, 1));
    };
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < slices && e == cudaSuccess; ++i) {  // every slice's eyes, in order
        uint32_t e0, e1;
        bounds(i, e0, e1);
        const size_t m = e1 - e0;
        cudaStream_t c = ctx->copy_stream;
        e = cudaMemcpyAsync(dx + e0, H.x + e0, m * 4, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy + e0, H.y + e0, m * 4, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dz + e0, H.z + e0, m * 4, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpx + e0, H.px + e0, m * 2, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpy + e0, H.py + e0, m * 2, cudaMemcpyHostToDevice, c);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in[i], c);
    }
    const unsigned grid_cap = hrr_cull_grid(ctx->sm_count, tn, false, n_eyes);
    auto enqueue = [&](uint32_t i) -> cudaError_t {
        uint32_t e0, e1;
        bounds(i, e0, e1);
        cudaStream_t s = cs[i & 1];
        unsigned long long *cnt = ctx->slice_counters + 4 * i;  // [0] accepted, [1] visits, [3] cursor
        cudaError_t r = cudaStreamWaitEvent(s, ctx->ev_in[i], 0);
        if (r == cudaSuccess && i >= 2) r = cudaStreamWaitEvent(s, ctx->ev_out[i - 2], 0);  // buffer reuse
        if (r != cudaSuccess) return r;
        Frame fr = single_frame(ctx, D, tree, tau, opts, tn, buf[i & 1], cap, e0);
        fr.counts = cnt;
        const Launch Lc{1, hrr_cull_spill_cap(tree->height, tn.node_width), (unsigned long long)(e1 - e0), cnt + 3,
                        ctx->counters + 2,
                        reinterpret_cast<uint2 *>(ctx->spill) + (i & 1) * hrr_cull_spill_entries(grid_cap, tree->height, tn)};
        r = launch_single(*kern, hrr_cull_grid(ctx->sm_count, tn, false, e1 - e0), Lc, fr, s);
        ++ctx->launches;
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(&ctx->host_slices[4 * i], cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess) r = cudaEventRecord(ctx->ev_done[i], s);
        return r;
    };
    uint32_t enqueued = 0;
    for (uint32_t i = 0; i < std::min(slices, 2u) && e == cudaSuccess; ++i)
        if ((e = enqueue(i)) == cudaSuccess) enqueued = i + 1;
    uint64_t need = 0, placed = 0, visits = 0;
    for (uint32_t i = 0; i < enqueued && e == cudaSuccess; ++i) {
        e = cudaEventSynchronize(ctx->ev_done[i]);
        if (e != cudaSuccess) break;
        const uint64_t c = ctx->host_slices[4 * i];
        visits += ctx->host_slices[4 * i + 1];
        const uint64_t fit = std::min<uint64_t>({c, cap, cap - placed});
        e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_done[i], 0);
        if (e == cudaSuccess && fit)
            e = cudaMemcpyAsync(host_pairs + 2 * placed, buf[i & 1], fit * 8, cudaMemcpyDeviceToHost, ctx->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out[i], ctx->copy_stream);
        need += c;
        placed += fit;
        if (e == cudaSuccess && i + 2 < slices) {
            if ((e = enqueue(i + 2)) == cudaSuccess) enqueued = i + 3;
        }
    }
    for (cudaStream_t s : {ctx->copy_stream, ctx->stream2, st}) {
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->host_counters, ctx->counters, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return hrr_cuda_fail(ctx, e, "culling with host buffers");
    ctx->last_accepted = need;
    ctx->last_visits = visits;
    *out_count = need;
    if (ctx->host_counters[2] & HRR_FLAG_STACK) return hrr_fail(ctx, HRR_ERR_DEVICE, "traversal stack overflow");
    if (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY) return hrr_fail(ctx, HRR_ERR_DEVICE, "corrupt node record");
    if (need > cap) return hrr_fail(ctx, HRR_ERR_OVERFLOW, "output capacity too small");
    return HRR_OK;
}

cudaError_t hrr_cull_batch_enqueue(unsigned grid, const hrr_cull_frame_t *frames, uint32_t n_frames,
                                   unsigned long long total, unsigned long long *cursor,
                                   unsigned long long *flags, void *spill, uint32_t spill_cap,
                                   const hrr_tuning &tuning, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    if (n_frames == 0 || n_frames > kMaxFrames) return cudaErrorInvalidValue;
    CullKernel *kern = cull_kernel_for(hrr_tuning_normalized(tuning));
    if (!kern) return cudaErrorInvalidValue;
    if (n_frames == 1 && frames[0].cursor_begin == 0) {
        // One frame (a served slice holding one job, a batch of one): the single-frame
        // kernel, whose frame is a plain kernel parameter held in registers, not looked up
        // per eye in the constant bank (about 2% faster per launch).
        const Launch Lc{1, spill_cap, total, cursor, flags, static_cast<uint2 *>(spill)};
        return launch_single(*kern, grid, Lc, frames[0], st);
    }
    FrameArray<kMaxFrames> fa;
    for (uint32_t i = 0; i < n_frames; ++i) fa.f[i] = frames[i];
    for (uint32_t i = n_frames; i < kMaxFrames; ++i) fa.f[i] = Frame{};
    const Launch Lc{n_frames, spill_cap, total, cursor, flags, static_cast<uint2 *>(spill)};
    return launch_batch(*kern, grid, Lc, fa, st);
}
