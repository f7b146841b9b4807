// Several samples per light in one traversal (Sec. 3: adaptive sampling and space-time
// shifts). Sample s of eye j uses the shift r_j,s = tile_s[pixel of j] + offset_s, where
// tile_s is layer s mod d of the context tile; for each sample the accepted set must equal
// the single-sample culling with that shift (Sec. 1), which is flat Russian roulette.
//
// The per-sample traversals of one eye visit largely the same nodes, so one traversal
// serves them all: a stack entry carries a node and the mask of samples for which the
// node is still alive. A visit fetches the node's record and computes each child's box
// bound once; for every sample of the mask it computes the child's range minimum under
// that sample's shift and the cull test, and the child is pushed with the mask of the
// samples that keep it. A leaf child is tested per sample of the mask. A node is thus
// visited for sample s exactly when the single-sample traversal with shift r_j,s visits it.
// Argmins are not inherited here (one per sample would not fit a stack entry), so each
// child's minimum is computed for every live sample.
//
// Execution mirrors the single-sample kernel: a persistent grid, one eye per warp, the
// warp's stack in a shared-memory ring spilling its oldest entries to a per-warp global
// area, survivors pushed as one compacted run. Accepted pairs are staged per warp with
// their sample index and appended to the sample's output with one atomic per sample in a
// chunk of 32. The shifts of the eye's samples live in lane s of the warp and are read by
// shuffles.
#include <algorithm>

#include "hrr_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBuf = 128;       // staged output entries per warp
constexpr uint32_t kRing = 256;  // stack entries per warp in shared memory
constexpr uint32_t kRingMask = kRing - 1;
constexpr int kMinBlocks = 5;    // resident blocks per SM the register budget is set for

struct SampleLaunch {
    const float *ex, *ey, *ez;
    const uint16_t *px, *py;
    const float4 *nodes;
    const uint32_t *perm;
    const uint32_t *tile;         // d layers of w x h
    uint32_t tile_w, tile_h, tile_d;
    uint32_t n_samples;           // 1 .. 32
    uint32_t offset[32];          // shift offset of each sample
    float tau;
    uint32_t n_lights;
    uint32_t n_eyes;
    uint32_t spill_cap;           // stack entries per warp in the spill area
    uint2 *pairs;                 // sample s: entries [s cap, (s + 1) cap)
    unsigned long long cap;
    unsigned long long *counts;   // [s] accepted of sample s (s < 32), [32] sample-visits,
                                  // [33] node visits, [34] eye cursor
    unsigned long long *flags;
    uint2 *spill;
};

// One 64-byte record as two 256-bit read-only loads that do not allocate in L1 (scattered
// records are rarely reused from L1; filling it would cost L1 data-pipe cycles).
__device__ __forceinline__ void load_record(const float4 *p, float4 &q0, float4 &q1, float4 &q2, float4 &q3) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(q0.x), "=f"(q0.y), "=f"(q0.z), "=f"(q0.w), "=f"(q1.x), "=f"(q1.y), "=f"(q1.z), "=f"(q1.w)
        : "l"(p));
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8+32];"
        : "=f"(q2.x), "=f"(q2.y), "=f"(q2.z), "=f"(q2.w), "=f"(q3.x), "=f"(q3.y), "=f"(q3.z), "=f"(q3.w)
        : "l"(p));
}

// Append the warp's cnt staged entries to their samples' outputs (warp-collective).
__device__ __forceinline__ void flush(const SampleLaunch &P, const uint2 *wbuf, const uint8_t *wsmp, uint32_t cnt,
                                      int lane) {
    for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
        const uint32_t k = k0 + lane;
        const bool has = k < cnt;
        const uint32_t s = has ? wsmp[k] : 0xFFFFFFFFu;
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, s);
        const int leader = __ffs(grp) - 1;
        const uint32_t rank = __popc(grp & ((1u << lane) - 1u));
        unsigned long long base = 0;
        if (has && lane == leader) base = atomicAdd(&P.counts[s], (unsigned long long)__popc(grp));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (has) {
            const unsigned long long o = base + rank;
            if (o < P.cap) __stcs(&P.pairs[(size_t)s * P.cap + o], wbuf[k]);  // streaming: written once
        }
    }
    __syncwarp();
}

// Stage the lanes' accepted samples of leaf i (bit s of acc: sample s accepts) as
// (j, original id of i) entries, one warp-uniform pass per sample (warp-collective).
__device__ __forceinline__ void emit(const SampleLaunch &P, uint2 *wbuf, uint8_t *wsmp, uint32_t &cnt, int lane,
                                     uint32_t j, uint32_t i, uint32_t acc) {
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t light = acc ? __ldg(&P.perm[i]) : 0u;
    for (uint32_t s = 0; s < P.n_samples; ++s) {
        const bool a = (acc >> s) & 1u;
        const unsigned b = __ballot_sync(0xFFFFFFFFu, a);
        if (!b) continue;
        if (cnt + __popc(b) > (uint32_t)kBuf) {
            flush(P, wbuf, wsmp, cnt, lane);
            cnt = 0;
        }
        if (a) {
            const uint32_t o = cnt + __popc(b & lt);
            wbuf[o] = make_uint2(j, light);
            wsmp[o] = (uint8_t)s;
        }
        cnt += __popc(b);
        __syncwarp();
    }
}

}  // namespace

namespace {

__global__ void __launch_bounds__(kThreads, kMinBlocks) cull_samples_kernel(const __grid_constant__ SampleLaunch P) {
    __shared__ uint2 buf[kWarps][kBuf];
    __shared__ uint8_t smp[kWarps][kBuf];
    __shared__ uint2 ring_all[kWarps][kRing];  // (node, mask of live samples)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint2 *wbuf = buf[warp];
    uint8_t *wsmp = smp[warp];
    uint2 *ring = ring_all[warp];
    uint2 *const spill = P.spill + ((size_t)blockIdx.x * kWarps + warp) * P.spill_cap;
    const uint32_t all = P.n_samples >= 32 ? 0xFFFFFFFFu : (1u << P.n_samples) - 1u;
    const float tau = P.tau;
    const float scale = hrr_node_scale(P.tau);  // the node test's scale
    uint32_t cnt = 0;
    unsigned long long node_visits = 0, sample_visits = 0;

    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(&P.counts[34], 1ull);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= P.n_eyes) break;
        const uint32_t j = (uint32_t)g;
        const float ex = P.ex[j], ey = P.ey[j], ez = P.ez[j];
        const uint32_t tx = P.px[j] % P.tile_w, ty = P.py[j] % P.tile_h;
        // lane s < n_samples: shift r of sample s and c = brev(2^32 - r)
        uint32_t rl = 0;
        if ((uint32_t)lane < P.n_samples)
            rl = P.tile[(size_t)((uint32_t)lane % P.tile_d) * P.tile_w * P.tile_h + ty * P.tile_w + tx] + P.offset[lane];
        const uint32_t cl = __brev(0u - rl);
        if (P.n_lights == 1) {  // the root is a leaf (record 0, slot 0)
            const float4 q0 = __ldg(&P.nodes[0]);
            uint32_t acc = 0;
            for (uint32_t s = 0; s < P.n_samples; ++s) {
                const uint32_t rs = __shfl_sync(0xFFFFFFFFu, rl, s);
                if (lane == 0 && hrr_leaf_accepts(__brev(0u) + rs, tau, scale, q0.x, q0.y, q0.z, q0.w, ex, ey, ez))
                    acc |= 1u << s;
            }
            emit(P, wbuf, wsmp, cnt, lane, j, 0u, acc);
            continue;
        }
        // Stack: logical entries [0, S); the newest R of them are in the ring at index & mask,
        // the others in the spill area at their logical index.
        uint32_t S = 1, R = 1, visits = 0;
        if (lane == 0) ring[0] = make_uint2(0u, all);
        __syncwarp();
        while (S > 0) {
            if (visits >= P.n_lights) {  // each internal node is visited at most once per eye
                if (lane == 0) atomicOr(P.flags, HRR_FLAG_TOPOLOGY);
                break;
            }
            const uint32_t m = min(32u, S);
            if (R < m) {  // bring spilled entries back into the ring
                const uint32_t fc = min(S - R, kRing / 2 - R);
                const uint32_t base = S - R - fc;
                for (uint32_t k = lane; k < fc; k += 32) ring[(base + k) & kRingMask] = spill[base + k];
                R += fc;
                __syncwarp();
            }
            const bool active = (uint32_t)lane < m;
            uint2 e = make_uint2(0u, 0u);
            if (active) e = ring[(S - m + lane) & kRingMask];
            S -= m;
            R -= m;
            visits += m;
            __syncwarp();

            bool valid = false, int0 = false, int1 = false;
            uint32_t split = 0, first = 0, last = 0;
            float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q2 = q0;
            float den0 = 0.f, rhs0 = 0.f, den1 = 0.f, rhs1 = 0.f;
            if (active) {
                sample_visits += __popc(e.y);
                float4 q1, q3;
                load_record(&P.nodes[4 * (size_t)e.x], q0, q1, q2, q3);
                split = __float_as_uint(q1.w);
                const uint32_t other = __float_as_uint(q3.w);
                first = min(e.x, other);
                last = max(e.x, other);
                if (last >= P.n_lights || split - first >= last - first) {  // needs first <= split < last
                    atomicOr(P.flags, HRR_FLAG_TOPOLOGY);                     // corrupt record
                } else {
                    valid = true;
                    int0 = first != split;
                    int1 = split + 1u != last;
                    hrr_node_bound(scale, q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q0.w, ex, ey, ez, den0, rhs0);
                    hrr_node_bound(scale, q2.x, q2.y, q2.z, q3.x, q3.y, q3.z, q2.w, ex, ey, ez, den1, rhs1);
                }
            }
            // per sample: the children's range minima and cull tests, or the leaf tests
            uint32_t mask0 = 0, mask1 = 0, acc0 = 0, acc1 = 0;
            for (uint32_t s = 0; s < P.n_samples; ++s) {
                const uint32_t rs = __shfl_sync(0xFFFFFFFFu, rl, s), cs = __shfl_sync(0xFFFFFFFFu, cl, s);
                if (valid && ((e.y >> s) & 1u)) {
                    const uint32_t bit = 1u << s;
                    if (int0) {
                        const uint32_t k = hrr_range_argmin_select(first, split + 1u, cs);
                        if (!hrr_node_culls(__brev(k) + rs, den0, rhs0)) mask0 |= bit;
                    } else if (hrr_leaf_accepts(__brev(split) + rs, tau, scale, q0.x, q0.y, q0.z, q0.w, ex, ey, ez)) {
                        acc0 |= bit;
                    }
                    if (int1) {
                        const uint32_t k = hrr_range_argmin_select(split + 1u, last + 1u, cs);
                        if (!hrr_node_culls(__brev(k) + rs, den1, rhs1)) mask1 |= bit;
                    } else if (hrr_leaf_accepts(__brev(last) + rs, tau, scale, q2.x, q2.y, q2.z, q2.w, ex, ey, ez)) {
                        acc1 |= bit;
                    }
                }
            }
            // Push the children that are alive for some sample as one compacted run.
            const bool go0 = mask0 != 0u, go1 = mask1 != 0u;
            const unsigned b0 = __ballot_sync(0xFFFFFFFFu, go0), b1 = __ballot_sync(0xFFFFFFFFu, go1);
            const uint32_t n = __popc(b0) + __popc(b1);
            if (n) {
                if (R + n > kRing) {  // move the oldest resident entries to the spill area
                    const uint32_t sp = (R + n - kRing + 31u) & ~31u;
                    const uint32_t base = S - R;
                    if (base + sp > P.spill_cap) {
                        if (lane == 0) atomicOr(P.flags, HRR_FLAG_STACK);
                        break;
                    }
                    for (uint32_t k = lane; k < sp; k += 32) spill[base + k] = ring[(base + k) & kRingMask];
                    R -= sp;
                    __syncwarp();
                }
                // lane by lane, siblings side by side (popped together by neighbouring lanes,
                // whose records are neighbours in memory)
                const uint32_t at = S + __popc(b0 & lt) + __popc(b1 & lt);
                if (go0) ring[at & kRingMask] = make_uint2(split, mask0);
                if (go1) ring[(at + (go0 ? 1u : 0u)) & kRingMask] = make_uint2(split + 1u, mask1);
                S += n;
                R += n;
                __syncwarp();
            }
            if (__any_sync(0xFFFFFFFFu, (acc0 | acc1) != 0u)) {
                emit(P, wbuf, wsmp, cnt, lane, j, split, acc0);
                emit(P, wbuf, wsmp, cnt, lane, j, last, acc1);
            }
        }
        node_visits += visits;
    }
    if (cnt) flush(P, wbuf, wsmp, cnt, lane);
    if (sample_visits) atomicAdd(&P.counts[32], sample_visits);
    if (lane == 0 && node_visits) atomicAdd(&P.counts[33], node_visits);
}

}  // namespace

int hrr_cull_samples_impl(hrr_ctx *ctx, const hrr_eyes &E, uint32_t n_eyes, const hrr_tree *tree, float tau,
                          const uint32_t *offsets, uint32_t n_samples, uint32_t *pairs, uint64_t cap,
                          uint64_t *out_counts, uint64_t *out_visits) {
    if (((uintptr_t)pairs & 7u) != 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs must be 8-byte aligned");
    cudaStream_t st = ctx->stream;
    if (!ctx->sample_counters) {
        if (cudaMalloc(&ctx->sample_counters, 40 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            ctx->sample_counters = nullptr;
            return hrr_fail(ctx, HRR_ERR_OOM, "sample counters");
        }
    }
    unsigned long long *counts = ctx->sample_counters;
    HRR_CUDA(ctx, cudaMemsetAsync(counts, 0, 40 * sizeof(unsigned long long), st));
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->counters + 2, 0, sizeof(unsigned long long), st));  // flags
    if (n_eyes > 0) {
        static int per_sm = 0;  // resident blocks per SM of the kernel
        if (!per_sm) {
            int m = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, cull_samples_kernel, kThreads, 0) != cudaSuccess ||
                m < 1)
                m = 1;
            per_sm = m;
        }
        const unsigned long long needed = ((unsigned long long)n_eyes + kWarps - 1) / kWarps;
        const unsigned grid =
            (unsigned)std::max<unsigned long long>(1ull, std::min<unsigned long long>((unsigned long long)per_sm * ctx->sm_count, needed));
        const uint32_t spill_cap = hrr_cull_spill_cap(tree->height, 2);  // binary records, two pushes a visit
        const size_t need = (size_t)grid * kWarps * spill_cap;
        if (need > ctx->spill_entries) {  // the stack spill area grows with the grid and tree height
            HRR_CUDA(ctx, cudaStreamSynchronize(st));
            if (ctx->spill) cudaFree(ctx->spill);
            ctx->spill = nullptr;
            ctx->spill_entries = 0;
            if (cudaMalloc(&ctx->spill, need * sizeof(uint2)) != cudaSuccess) {
                cudaGetLastError();
                return hrr_fail(ctx, HRR_ERR_OOM, "traversal stack spill area");
            }
            ctx->spill_entries = need;
        }
        SampleLaunch P{};
        P.ex = E.x; P.ey = E.y; P.ez = E.z; P.px = E.px; P.py = E.py;
        P.nodes = reinterpret_cast<const float4 *>(tree->nodes);
        P.perm = tree->perm;
        P.tile = ctx->tile;
        P.tile_w = ctx->tile_w; P.tile_h = ctx->tile_h; P.tile_d = ctx->tile_d ? ctx->tile_d : 1u;
        P.n_samples = n_samples;
        for (uint32_t s = 0; s < n_samples; ++s) P.offset[s] = offsets[s];
        P.tau = tau;
        P.n_lights = tree->n;
        P.n_eyes = n_eyes;
        P.spill_cap = spill_cap;
        P.pairs = reinterpret_cast<uint2 *>(pairs);
        P.cap = cap;
        P.counts = counts;
        P.flags = ctx->counters + 2;
        P.spill = reinterpret_cast<uint2 *>(ctx->spill);
        cull_samples_kernel<<<grid, kThreads, 0, st>>>(P);
        ++ctx->launches;
        HRR_CUDA(ctx, cudaGetLastError());
    }
    unsigned long long host[40];
    HRR_CUDA(ctx, cudaMemcpyAsync(host, counts, sizeof(host), cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaMemcpyAsync(&ctx->host_counters[2], ctx->counters + 2, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaStreamSynchronize(st));
    bool over = false;
    uint64_t total = 0;
    for (uint32_t s = 0; s < n_samples; ++s) {
        out_counts[s] = host[s];
        total += host[s];
        over = over || host[s] > cap;
    }
    if (out_visits) {
        out_visits[0] = host[32];
        out_visits[1] = host[33];
    }
    ctx->last_accepted = total;
    ctx->last_visits = host[32];
    if (ctx->host_counters[2] & HRR_FLAG_STACK) return hrr_fail(ctx, HRR_ERR_DEVICE, "traversal stack overflow");
    if (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY) return hrr_fail(ctx, HRR_ERR_DEVICE, "corrupt node record");
    if (over) return hrr_fail(ctx, HRR_ERR_OVERFLOW, "output capacity too small for a sample");
    return HRR_OK;
}
