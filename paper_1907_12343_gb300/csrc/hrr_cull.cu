// Hierarchical Russian-roulette culling with blue-noise dithered QMC sequences (Sec. 1).
//
// For eye j with shift r_j (tile entry at its pixel), the traversal starts at the root and,
// at every visited internal node, tests both children from the node's 64-byte record:
//   * a leaf child i is accepted iff brev(i) + r_j < ceil(p_ij 2^32) (exact float32 p);
//   * an internal child with leaf range [a, b) is descended unless the range minimum
//     v(a, b) = min_{i in [a,b)} (brev(i) + r_j) mod 2^32 passes the conservative cull test
//     (v is at least the threshold of every light below; then none can be accepted).
// The accepted set therefore equals flat Russian roulette over all pairs.
//
// Execution: a persistent grid (a whole number of resident blocks per SM). Each lane of a
// warp traverses one eye; the warp steps its lanes together, one node per lane per
// iteration, so accepted pairs are counted with two ballots and staged in a per-warp
// shared-memory buffer that is appended to the output with one atomic and coalesced
// 8-byte stores. When lanes finish their eyes the warp refills them from a global eye
// cursor (one atomic per refill), which keeps the warp's lanes busy until the eyes run
// out instead of waiting for its slowest traversal. A node's range minimum is attained at
// its argmin, which lies in exactly one child; carrying the argmin down with the node
// means only the other child's minimum has to be computed.
#include "hrr_internal.cuh"

namespace {

// Launch shape, fixed at compile time (the values measured fastest on GB300).
#ifndef HRR_CULL_MIN_BLOCKS
#define HRR_CULL_MIN_BLOCKS 5  // resident 256-thread blocks per SM (caps registers at 48)
#endif
#ifndef HRR_CULL_REFILL_BELOW
#define HRR_CULL_REFILL_BELOW 29  // refill a warp's idle lanes once at least 4 are idle
#endif
#ifndef HRR_CULL_SMEM_LEVELS
#define HRR_CULL_SMEM_LEVELS 12  // traversal-stack levels kept in shared memory per thread
#endif
#ifndef HRR_CULL_BUF
#define HRR_CULL_BUF 128  // staged output pairs per warp
#endif
#ifndef HRR_CULL_PREFETCH
#define HRR_CULL_PREFETCH 0  // prefetch the children's records into L1 once the split is known
#endif

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBuf = HRR_CULL_BUF;  // staged pairs per warp
constexpr int kSmemLevels = HRR_CULL_SMEM_LEVELS;
constexpr int kStack = 96;        // >= height of any radix tree over 95-bit ordering keys
constexpr int kRefillBelow = HRR_CULL_REFILL_BELOW;
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
    unsigned long long *counters;  // [0] accepted, [1] visits, [2] flags, [3] eye cursor
    uint32_t *eye_visits;
};

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
    if (cnt + tot > (uint32_t)kBuf) {
        flush(P, wbuf, cnt, lane);
        cnt = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    if (acc0 != kNone) wbuf[cnt + __popc(b0 & lt)] = make_uint2(j, __ldg(&P.perm[acc0]));
    if (acc1 != kNone) wbuf[cnt + __popc(b0) + __popc(b1 & lt)] = make_uint2(j, __ldg(&P.perm[acc1]));
    cnt += tot;
    __syncwarp();
}

__device__ __forceinline__ uint32_t eye_shift(const CullParams &P, uint32_t j) {
    const uint32_t tx = P.px[j] % P.tile_w, ty = P.py[j] % P.tile_h;
    return P.tile[ty * P.tile_w + tx] + P.shift_offset;
}

// Argmin of the range minimum of (brev(i) + r) over [a, b); c = brev(2^32 - r).
template <int VARIANT>
__device__ __forceinline__ uint32_t range_argmin(uint32_t a, uint32_t b, uint32_t r, uint32_t c) {
    uint32_t k;
    if (VARIANT == 0) return hrr_range_argmin_select(a, b, c);
    if (VARIANT == 1) hrr_rangemin_alg2(a, b, r, &k);
    else hrr_rangemin_closed(a, b, r, &k);
    return k;
}

template <int VARIANT>
__global__ void __launch_bounds__(kThreads, VARIANT == 0 ? HRR_CULL_MIN_BLOCKS : 5)
cull_kernel(const CullParams P) {
    __shared__ uint2 buf[kWarps][kBuf];
    // The traversal stack: its first kSmemLevels levels in shared memory ([level][thread],
    // so that lanes at the same depth hit distinct banks), deeper levels in local memory.
    // Keeping the hot levels out of L1 leaves L1 to the node records.
    __shared__ uint2 sstack[kSmemLevels > 0 ? kSmemLevels : 1][kThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint2 *wbuf = buf[warp];
    const float tau = P.tau;

    bool alive = false;
    bool more = true;  // warp-uniform: the eye cursor may still hand out eyes
    uint32_t j = 0, r = 0, c = 0, node = 0, visits = 0, cnt = 0;
    // Argmin of the current node's range minimum. Exactly one child holds it and has the
    // same minimum, so each visit computes at most one new range minimum: the other
    // internal child's. The root's is computed when the eye starts.
    uint32_t kmin = 0;
    float ex = 0.f, ey = 0.f, ez = 0.f;
    unsigned long long visit_total = 0;
    uint2 deep[kStack - kSmemLevels];  // (node, argmin of its range minimum)
    int sp = 0;

    for (;;) {
        unsigned alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        if (more && __popc(alive_mask) < kRefillBelow) {
            const unsigned idle = ~alive_mask;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&P.counters[3], (unsigned long long)__popc(idle));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + __popc(idle) >= P.n_eyes) more = false;
            if (!alive) {
                const unsigned long long jj = base + __popc(idle & lt);
                if (jj < P.n_eyes) {
                    j = (uint32_t)jj;
                    ex = P.ex[j];
                    ey = P.ey[j];
                    ez = P.ez[j];
                    r = eye_shift(P, j);
                    c = __brev(0u - r);
                    node = 0;
                    kmin = range_argmin<VARIANT>(0u, P.n_lights, r, c);
                    sp = 0;
                    visits = 0;
                    alive = true;
                }
            }
            alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        }
        if (alive_mask == 0u) break;

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
            bool go0 = false, go1 = false;
            uint32_t k0 = kNone, k1 = kNone;
            if (last >= P.n_lights || split - first >= last - first) {  // needs first <= split < last
                atomicOr(&P.counters[2], HRR_FLAG_TOPOLOGY);               // corrupt record
                sp = 0;
            } else {
                const bool int0 = first != split, int1 = split + 1u != last;
#if HRR_CULL_PREFETCH
                // The next visit is most often a child (internal nodes split and split + 1,
                // adjacent records): start their transfer into L1 while this node is tested.
                if (int0) asm volatile("prefetch.global.L1 [%0];" ::"l"(&P.nodes[4 * (size_t)split]));
                if (int1) asm volatile("prefetch.global.L1 [%0];" ::"l"(&P.nodes[4 * (size_t)split + 4]));
#endif
                const bool kin0 = kmin <= split;
                uint32_t knew = kNone;
                if (kin0 ? int1 : int0)
                    knew = range_argmin<VARIANT>(kin0 ? split + 1u : first, kin0 ? last + 1u : split + 1u, r, c);
                k0 = kin0 ? kmin : knew;
                k1 = kin0 ? knew : kmin;
                float den0, rhs0, den1, rhs1;
                hrr_node_bound(tau, q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q0.w, ex, ey, ez, den0, rhs0);
                hrr_node_bound(tau, q2.x, q2.y, q2.z, q3.x, q3.y, q3.z, q2.w, ex, ey, ez, den1, rhs1);
                go0 = int0 && !hrr_node_culls(__brev(k0) + r, den0, rhs0);
                go1 = int1 && !hrr_node_culls(__brev(k1) + r, den1, rhs1);
                if (!int0 || !int1) {  // leaf children: one test site, a second for two leaves
                    const uint32_t i = !int0 ? split : last;
                    const float4 ql = !int0 ? q0 : q2;
                    if (hrr_leaf_accepts(__brev(i) + r, tau, ql.x, ql.y, ql.z, ql.w, ex, ey, ez)) acc0 = i;
                    if (!int0 && !int1 &&
                        hrr_leaf_accepts(__brev(last) + r, tau, q2.x, q2.y, q2.z, q2.w, ex, ey, ez))
                        acc1 = last;
                }
            }
            if (go0 && go1) {
                if (sp < kSmemLevels) {
                    sstack[sp++][threadIdx.x] = make_uint2(split + 1u, k1);
                } else if (sp < kStack) {
                    deep[sp++ - kSmemLevels] = make_uint2(split + 1u, k1);
                } else {
                    atomicOr(&P.counters[2], HRR_FLAG_STACK);
                }
                node = split;
                kmin = k0;
            } else if (go0) {
                node = split;
                kmin = k0;
            } else if (go1) {
                node = split + 1u;
                kmin = k1;
            } else if (sp > 0) {
                --sp;
                const uint2 e = sp < kSmemLevels ? sstack[sp][threadIdx.x] : deep[sp - kSmemLevels];
                node = e.x;
                kmin = e.y;
            } else {
                alive = false;
                visit_total += visits;
                if (P.eye_visits) P.eye_visits[j] = visits;
            }
        }
        emit(P, wbuf, cnt, lane, j, acc0, acc1);
    }
    if (cnt) flush(P, wbuf, cnt, lane);
    // visit_total < 2^32 per lane in practice; sum both halves to stay exact regardless
    const unsigned long long wsum =
        (unsigned long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(visit_total & 0xFFFFFFFFull)) +
        ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(visit_total >> 32)) << 32);
    if (lane == 0 && wsum) atomicAdd(&P.counters[1], wsum);
}

// A one-light hierarchy: the root is a leaf (record 0, slot 0).
__global__ void __launch_bounds__(kThreads) cull_single_light_kernel(const CullParams P) {
    __shared__ uint2 buf[kWarps][kBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t j = blockIdx.x * kThreads + threadIdx.x;
    uint32_t acc = kNone, cnt = 0;
    if (j < P.n_eyes) {
        const float4 q0 = P.nodes[0];
        if (hrr_leaf_accepts(__brev(0u) + eye_shift(P, j), P.tau, q0.x, q0.y, q0.z, q0.w, P.ex[j],
                             P.ey[j], P.ez[j]))
            acc = 0;
        if (P.eye_visits) P.eye_visits[j] = 0;
    }
    emit(P, buf[warp], cnt, lane, j, acc, kNone);
    if (cnt) flush(P, buf[warp], cnt, lane);
}

// Resident blocks per SM of the traversal kernel (the same on every device of one type).
template <int VARIANT>
int blocks_per_sm() {  // one cache per variant
    static int n = 0;
    if (!n) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, cull_kernel<VARIANT>, kThreads, 0) != cudaSuccess || m < 1)
            m = 1;
        n = m;
    }
    return n;
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
        hrr_timing_begin(ctx);
        if (tree->n == 1) {
            cull_single_light_kernel<<<(n_eyes + kThreads - 1) / kThreads, kThreads, 0, st>>>(P);
        } else {
            const int blocks_needed = (int)(((uint64_t)n_eyes + kThreads - 1) / kThreads);
            if (opts.rangemin_variant == 0)
                cull_kernel<0><<<min(blocks_per_sm<0>() * ctx->sm_count, blocks_needed), kThreads, 0, st>>>(P);
            else if (opts.rangemin_variant == 1)
                cull_kernel<1><<<min(blocks_per_sm<1>() * ctx->sm_count, blocks_needed), kThreads, 0, st>>>(P);
            else
                cull_kernel<2><<<min(blocks_per_sm<2>() * ctx->sm_count, blocks_needed), kThreads, 0, st>>>(P);
        }
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
