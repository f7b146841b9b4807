// Autotuning of the traversal's launch shape.
//
// The traversal's results do not depend on its launch parameters (range-minimum variant,
// resident blocks per SM), only its speed does. hrr_autotune runs
// every candidate on a caller-given eye sample and keeps the fastest; a caller (the Python
// autotuner) caches one answer per size class of workload.
#include <algorithm>
#include <vector>

#include "hrr_internal.cuh"

extern "C" int hrr_autotune(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree,
                            float tau, uint32_t *dev_pairs, uint64_t cap, hrr_tuning *best,
                            double *best_ms) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!best) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "best is NULL");
    if (!tree || n_eyes == 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "autotuning needs a tree and eyes");
    DeviceGuard g(ctx->device);
    cudaEvent_t a = nullptr, b = nullptr;
    HRR_CUDA(ctx, cudaEventCreate(&a));
    HRR_CUDA(ctx, cudaEventCreate(&b));
    const int variants[] = {0, 2};
    const uint32_t blocks[] = {4, 5, 6};
    double best_t = 1e300;
    int status = HRR_OK;
    for (int v : variants) {
        for (uint32_t bl : blocks) {
            {
                hrr_cull_opts o{};
                o.rangemin_variant = v;
                o.blocks_per_sm = bl;
                std::vector<double> t;
                for (int rep = 0; rep < 4 && status == HRR_OK; ++rep) {
                    uint64_t count = 0;
                    cudaEventRecord(a, ctx->stream);
                    status = hrr_cull_ex(ctx, eyes, n_eyes, tree, tau, &o, dev_pairs, cap, &count);
                    cudaEventRecord(b, ctx->stream);
                    cudaEventSynchronize(b);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, b);
                    if (rep > 0) t.push_back(ms);  // the first run warms caches
                }
                if (status != HRR_OK) break;
                std::sort(t.begin(), t.end());
                const double med = t[t.size() / 2];
                if (med < best_t) {
                    best_t = med;
                    best->rangemin_variant = v;
                    best->blocks_per_sm = bl;
                }
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (status != HRR_OK) return status;
    if (best_ms) *best_ms = best_t;
    return HRR_OK;
}
