// Autotuning of the traversal's form and launch shape.
//
// The traversal's results do not depend on its tuning (range-minimum variant, node width,
// shared-memory stack ring, threads per block, top levels evaluated from shared memory,
// resident blocks per SM); only its speed does. hrr_autotune_all times every compiled
// form, at the most resident blocks per SM that fit and at one block fewer, on a
// caller-given eye sample; hrr_autotune keeps the fastest. A caller (the Python autotuner)
// caches one answer per size class of workload.
#include <algorithm>
#include <vector>

#include "hrr_internal.cuh"

namespace {

// Every candidate tuning, in a fixed order.
std::vector<hrr_tuning> candidates() {
    std::vector<hrr_tuning> out;
    for (int variant : {0, 2})
        for (uint32_t width : {2u, 4u})
            for (uint32_t top : {1u, HRR_TOP_LEVELS})
                for (uint32_t ring : {128u, 256u, 512u})
                    for (uint32_t threads : {128u, 256u}) {
                        hrr_tuning t{};
                        t.rangemin_variant = variant;
                        t.node_width = width;
                        t.ring_entries = ring;
                        t.threads_per_block = threads;
                        t.top_levels = top;
                        if (!hrr_tuning_valid(t)) continue;
                        const int most = hrr_cull_max_blocks(t, false);
                        for (int b = most; b >= std::max(1, most - 1); --b) {
                            t.blocks_per_sm = (uint32_t)b;
                            out.push_back(t);
                        }
                    }
    return out;
}

}  // namespace

extern "C" int hrr_autotune_all(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                                uint32_t *dev_pairs, uint64_t cap, hrr_tuning *tried, double *tried_ms,
                                uint32_t capacity, uint32_t *n_tried) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!n_tried) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "n_tried is NULL");
    *n_tried = 0;
    if (!tree || n_eyes == 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "autotuning needs a tree and eyes");
    DeviceGuard g(ctx->device);
    const std::vector<hrr_tuning> cands = candidates();
    if (!tried || !tried_ms || capacity < cands.size()) {
        *n_tried = (uint32_t)cands.size();  // the room the caller must provide
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "the candidate arrays are NULL or too small");
    }
    cudaEvent_t a = nullptr, b = nullptr;
    HRR_CUDA(ctx, cudaEventCreate(&a));
    HRR_CUDA(ctx, cudaEventCreate(&b));
    int status = HRR_OK;
    for (size_t c = 0; c < cands.size() && status == HRR_OK; ++c) {
        const hrr_tuning &t = cands[c];
        hrr_cull_opts o{};
        o.rangemin_variant = t.rangemin_variant;
        o.blocks_per_sm = t.blocks_per_sm;
        o.node_width = t.node_width;
        o.ring_entries = t.ring_entries;
        o.threads_per_block = t.threads_per_block;
        o.top_levels = t.top_levels;
        std::vector<double> ts;
        for (int rep = 0; rep < 4 && status == HRR_OK; ++rep) {
            uint64_t count = 0;
            cudaEventRecord(a, ctx->stream);
            status = hrr_cull_ex(ctx, eyes, n_eyes, tree, tau, &o, dev_pairs, cap, &count);
            cudaEventRecord(b, ctx->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) ts.push_back(ms);  // the first run warms caches
        }
        if (status != HRR_OK) break;
        std::sort(ts.begin(), ts.end());
        tried[c] = t;
        tried_ms[c] = ts[ts.size() / 2];
        *n_tried = (uint32_t)(c + 1);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return status;
}

extern "C" int hrr_autotune(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree,
                            float tau, uint32_t *dev_pairs, uint64_t cap, hrr_tuning *best,
                            double *best_ms) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!best) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "best is NULL");
    std::vector<hrr_tuning> tried(128);
    std::vector<double> ms(128);
    uint32_t n = 0;
    const int st = hrr_autotune_all(ctx, eyes, n_eyes, tree, tau, dev_pairs, cap, tried.data(), ms.data(),
                                    (uint32_t)tried.size(), &n);
    if (st != HRR_OK) return st;
    uint32_t k = 0;
    for (uint32_t i = 1; i < n; ++i)
        if (ms[i] < ms[k]) k = i;
    *best = tried[k];
    if (best_ms) *best_ms = ms[k];
    return HRR_OK;
}
