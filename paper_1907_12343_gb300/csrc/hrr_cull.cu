// Hierarchical Russian-roulette culling with blue-noise dithered QMC sequences (Sec. 1).
//
// For eye j with shift r_j (tile entry at its pixel), the traversal starts at the root and,
// at every visited internal node, tests both children from the node's 64-byte record:
//   * a leaf child i is accepted iff brev(i) + r_j < ceil(p_ij 2^32) (exact float32 p);
//   * an internal child with leaf range [a, b) is descended unless the range minimum
//     v(a, b) = min_{i in [a,b)} (brev(i) + r_j) mod 2^32 is >= its conservative bound
//     T = ceil(P 2^32), P >= p_ij for every light below it (then none can be accepted).
// The accepted set therefore equals flat Russian roulette over all pairs.
//
// Execution: one eye per thread; a warp steps its 32 traversals together, one node per
// lane per iteration, so that accepted pairs can be counted with two ballots and staged
// in a per-warp shared-memory buffer; a full buffer is appended to the output with one
// atomic and coalesced 8-byte stores.
#include "hrr_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBuf = 256;     // staged pairs per warp
constexpr int kStack = 96;    // >= height of any radix tree over 95-bit ordering keys
constexpr uint32_t kNone = 0xFFFFFFFFu;

struct CullParams {
    const float *ex, *ey, *ez;
    const uint16_t *px, *py;
    uint32_t n_eyes;
    const float4 *nodes;
    const uint32_t *perm;
    uint32_t n_lights;
    const uint32_t *tile;
    uint32_t tile_w, tile_h, shift_offset;
    float tau;
    uint2 *pairs;
    unsigned long long cap;
    unsigned long long *counters;  // [0] accepted, [1] visits, [2] flags
    uint32_t *eye_visits;
};

template <int VARIANT>
__device__ __forceinline__ uint32_t range_min(uint32_t a, uint32_t b, uint32_t r) {
    uint32_t k;
    return VARIANT == 0 ? hrr_rangemin_closed(a, b, r, &k) : hrr_rangemin_alg2(a, b, r, &k);
}

// Append the warp's staged pairs to the output.
__device__ __forceinline__ void flush(const CullParams &P, const uint2 *wbuf, uint32_t cnt, int lane) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&P.counters[0], (unsigned long long)cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t k = lane; k < cnt; k += 32) {
        const unsigned long long o = base + k;
        if (o < P.cap) P.pairs[o] = wbuf[k];
    }
    __syncwarp();
}

// Stage up to two accepted leaves per lane (warp-collective).
__device__ __forceinline__ void emit(const CullParams &P, uint2 *wbuf, uint32_t &cnt, int lane,
                                     uint32_t j, uint32_t acc0, uint32_t acc1) {
    const unsigned b0 = __ballot_sync(0xFFFFFFFFu, acc0 != kNone);
    const unsigned b1 = __ballot_sync(0xFFFFFFFFu, acc1 != kNone);
    const uint32_t tot = __popc(b0) + __popc(b1);
    if (tot == 0) return;
    if (cnt + tot > kBuf) {
        flush(P, wbuf, cnt, lane);
        cnt = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    if (acc0 != kNone) wbuf[cnt + __popc(b0 & lt)] = make_uint2(j, __ldg(&P.perm[acc0]));
    if (acc1 != kNone) wbuf[cnt + __popc(b0) + __popc(b1 & lt)] = make_uint2(j, __ldg(&P.perm[acc1]));
    cnt += tot;
    __syncwarp();
}

template <int VARIANT>
__global__ void __launch_bounds__(kThreads) cull_kernel(const CullParams P) {
    __shared__ uint2 buf[kWarps][kBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint2 *wbuf = buf[warp];
    const uint32_t j = blockIdx.x * kThreads + threadIdx.x;
    bool alive = j < P.n_eyes;
    float ex = 0.f, ey = 0.f, ez = 0.f;
    uint32_t r = 0;
    if (alive) {
        ex = P.ex[j];
        ey = P.ey[j];
        ez = P.ez[j];
        const uint32_t tx = P.px[j] % P.tile_w, ty = P.py[j] % P.tile_h;
        r = P.tile[ty * P.tile_w + tx] + P.shift_offset;
    }
    const float tau = P.tau;
    uint32_t cnt = 0;
    uint32_t visits = 0;

    if (P.n_lights == 1) {  // the root is a leaf (record 0, slot 0)
        uint32_t acc = kNone;
        if (alive) {
            const float4 q0 = P.nodes[0];
            if ((unsigned long long)(__brev(0u) + r) < hrr_leaf_threshold(tau, q0.x, q0.y, q0.z, q0.w, ex, ey, ez))
                acc = 0;
        }
        emit(P, wbuf, cnt, lane, j, acc, kNone);
        alive = false;
    }

    uint32_t stack[kStack];
    int sp = 0;
    uint32_t node = 0;
    while (__any_sync(0xFFFFFFFFu, alive)) {
        uint32_t acc0 = kNone, acc1 = kNone;
        if (alive) {
            ++visits;
            const float4 q0 = __ldg(&P.nodes[4 * (size_t)node + 0]);
            const float4 q1 = __ldg(&P.nodes[4 * (size_t)node + 1]);
            const float4 q2 = __ldg(&P.nodes[4 * (size_t)node + 2]);
            const float4 q3 = __ldg(&P.nodes[4 * (size_t)node + 3]);
            const uint32_t split = __float_as_uint(q1.w);
            const uint32_t other = __float_as_uint(q3.w);
            const uint32_t first = min(node, other), last = max(node, other);
            if (last >= P.n_lights || split < first || split >= last) {  // corrupt record
                atomicOr(&P.counters[2], HRR_FLAG_TOPOLOGY);
                alive = false;
            } else {
                bool go0 = false, go1 = false;
                if (first == split) {
                    if ((unsigned long long)(__brev(split) + r) <
                        hrr_leaf_threshold(tau, q0.x, q0.y, q0.z, q0.w, ex, ey, ez))
                        acc0 = split;
                } else {
                    const unsigned long long T =
                        hrr_node_threshold(tau, q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q0.w, ex, ey, ez);
                    go0 = T > 0xFFFFFFFFull || range_min<VARIANT>(first, split + 1u, r) < T;
                }
                if (split + 1u == last) {
                    if ((unsigned long long)(__brev(last) + r) <
                        hrr_leaf_threshold(tau, q2.x, q2.y, q2.z, q2.w, ex, ey, ez))
                        acc1 = last;
                } else {
                    const unsigned long long T =
                        hrr_node_threshold(tau, q2.x, q2.y, q2.z, q3.x, q3.y, q3.z, q2.w, ex, ey, ez);
                    go1 = T > 0xFFFFFFFFull || range_min<VARIANT>(split + 1u, last + 1u, r) < T;
                }
                if (go0 && go1) {
                    if (sp < kStack) {
                        stack[sp++] = split + 1u;
                    } else {
                        atomicOr(&P.counters[2], HRR_FLAG_STACK);
                    }
                    node = split;
                } else if (go0) {
                    node = split;
                } else if (go1) {
                    node = split + 1u;
                } else if (sp > 0) {
                    node = stack[--sp];
                } else {
                    alive = false;
                }
            }
        }
        emit(P, wbuf, cnt, lane, j, acc0, acc1);
    }
    if (cnt) flush(P, wbuf, cnt, lane);
    if (P.eye_visits && j < P.n_eyes) P.eye_visits[j] = visits;
    const unsigned wsum = __reduce_add_sync(0xFFFFFFFFu, visits);
    if (lane == 0 && wsum) atomicAdd(&P.counters[1], (unsigned long long)wsum);
}

}  // namespace

int hrr_cull_impl(hrr_ctx *ctx, const hrr_eyes &E, uint32_t n_eyes, const hrr_tree *tree,
                  float tau, const hrr_cull_opts &opts, uint32_t *pairs, uint64_t cap,
                  uint64_t *out_count) {
    if (((uintptr_t)pairs & 7u) != 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs must be 8-byte aligned");
    cudaStream_t st = ctx->stream;
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(unsigned long long), st));
    if (n_eyes > 0) {
        CullParams P;
        P.ex = E.x; P.ey = E.y; P.ez = E.z; P.px = E.px; P.py = E.py;
        P.n_eyes = n_eyes;
        P.nodes = reinterpret_cast<const float4 *>(tree->nodes);
        P.perm = tree->perm;
        P.n_lights = tree->n;
        P.tile = ctx->tile; P.tile_w = ctx->tile_w; P.tile_h = ctx->tile_h;
        P.shift_offset = opts.shift_offset;
        P.tau = tau;
        P.pairs = reinterpret_cast<uint2 *>(pairs);
        P.cap = cap;
        P.counters = ctx->counters;
        P.eye_visits = opts.eye_visits;
        const unsigned grid = (n_eyes + kThreads - 1) / kThreads;
        hrr_timing_begin(ctx);
        if (opts.rangemin_variant == 0)
            cull_kernel<0><<<grid, kThreads, 0, st>>>(P);
        else
            cull_kernel<1><<<grid, kThreads, 0, st>>>(P);
        hrr_timing_end(ctx);
        ++ctx->launches;
        HRR_CUDA(ctx, cudaGetLastError());
    }
    HRR_CUDA(ctx, cudaMemcpyAsync(ctx->host_counters, ctx->counters, 3 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaStreamSynchronize(st));
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
