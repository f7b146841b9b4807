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
// shared-memory buffer that is appended to the output with one atomic per frame and
// coalesced 8-byte stores. When lanes finish their eyes the warp refills them from a global
// eye cursor (one atomic per refill), which keeps the warp's lanes busy until the eyes run
// out instead of waiting for its slowest traversal. A node's range minimum is attained at
// its argmin, which lies in exactly one child; carrying the argmin down with the node
// means only the other child's minimum has to be computed.
//
// One launch may cover many frames (a batch): the cursor then runs over the eyes of all
// frames, each lane finds its frame by binary search over the frames' cursor offsets, and
// the frames' descriptors are staged in shared memory. Frames of different sizes share
// the launch without any per-frame tail.
#include "hrr_internal.cuh"

namespace {

// Launch shape, fixed at compile time (the values measured fastest on GB300).
#ifndef HRR_CULL_MIN_BLOCKS
#define HRR_CULL_MIN_BLOCKS 4  // resident 256-thread blocks per SM (64 registers: no spills, best measured)
#endif
#ifndef HRR_CULL_SMEM_LEVELS
#define HRR_CULL_SMEM_LEVELS 12  // traversal-stack levels kept in shared memory per thread
#endif
#ifndef HRR_CULL_BUF
#define HRR_CULL_BUF 128  // staged output pairs per warp
#endif
#ifndef HRR_CULL_BATCH_MIN_BLOCKS
#define HRR_CULL_BATCH_MIN_BLOCKS 4  // resident blocks per SM of the batched traversal (64 registers, no spills)
#endif

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBuf = HRR_CULL_BUF;
constexpr int kSmemLevels = HRR_CULL_SMEM_LEVELS;
constexpr int kStack = 96;       // >= height of any radix tree over 95-bit ordering keys
constexpr uint32_t kSmemFrames = 64;  // batch frames whose descriptors are staged in shared memory
constexpr uint32_t kNone = 0xFFFFFFFFu;

using Frame = hrr_cull_frame_t;
static_assert(sizeof(Frame) == 128, "frame descriptor layout");

struct Launch {
    const Frame *frames;            // batch: device array of n_frames descriptors
    uint32_t n_frames;
    uint32_t refill_below;          // refill a warp's idle lanes once fewer lanes are busy
    unsigned long long total;       // eyes of this launch over all frames
    unsigned long long *cursor;     // global eye cursor (starts at 0)
    unsigned long long *flags;      // HRR_FLAG_* bits
};

// Frame f of the launch: the kernel parameter for a single frame, shared memory (global
// memory beyond kSmemFrames) for a batch.
template <bool BATCH>
__device__ __forceinline__ const Frame &frame_at(const Frame &single, const Frame *sframes,
                                                 const Frame *glob, uint32_t f) {
    if constexpr (!BATCH) return single;
    else return f < kSmemFrames ? sframes[f] : glob[f];
}

// Append the warp's staged pairs to their frames' outputs: one atomic per frame present in
// each 32-entry chunk (a chunk rarely holds more than one frame).
template <bool BATCH>
__device__ __forceinline__ void flush(const Frame &single, const Frame *sframes, const Frame *glob,
                                      const uint2 *wbuf, const uint16_t *wfr, uint32_t cnt, int lane) {
    if constexpr (!BATCH) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&single.counts[0], (unsigned long long)cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (uint32_t k = lane; k < cnt; k += 32) {
            const unsigned long long o = base + k;
            if (o < single.cap) single.pairs[o] = wbuf[k];
        }
    } else {
        for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
            const uint32_t k = k0 + lane;
            const bool has = k < cnt;
            const uint32_t f = has ? wfr[k] : 0xFFFFFFFFu;
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, f);
            const int leader = __ffs(grp) - 1;
            const uint32_t rank = __popc(grp & ((1u << lane) - 1u));
            unsigned long long base = 0;
            if (has && lane == leader)
                base = atomicAdd(&frame_at<BATCH>(single, sframes, glob, f).counts[0],
                                 (unsigned long long)__popc(grp));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (has) {
                const Frame &fr = frame_at<BATCH>(single, sframes, glob, f);
                const unsigned long long o = base + rank;
                if (o < fr.cap) fr.pairs[o] = wbuf[k];
            }
        }
    }
    __syncwarp();
}

// Stage up to two accepted leaves per lane (warp-collective).
template <bool BATCH>
__device__ __forceinline__ void emit(const Frame &single, const Frame *sframes, const Frame *glob,
                                     uint2 *wbuf, uint16_t *wfr, uint32_t &cnt, int lane, uint32_t f,
                                     uint32_t j, uint32_t acc0, uint32_t acc1) {
    const unsigned b0 = __ballot_sync(0xFFFFFFFFu, acc0 != kNone);
    const unsigned b1 = __ballot_sync(0xFFFFFFFFu, acc1 != kNone);
    const uint32_t tot = __popc(b0) + __popc(b1);
    if (tot == 0) return;
    if (cnt + tot > (uint32_t)kBuf) {
        flush<BATCH>(single, sframes, glob, wbuf, wfr, cnt, lane);
        cnt = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t *perm = frame_at<BATCH>(single, sframes, glob, f).perm;
    if (acc0 != kNone) {
        const uint32_t o = cnt + __popc(b0 & lt);
        wbuf[o] = make_uint2(j, __ldg(&perm[acc0]));
        if constexpr (BATCH) wfr[o] = (uint16_t)f;
    }
    if (acc1 != kNone) {
        const uint32_t o = cnt + __popc(b0) + __popc(b1 & lt);
        wbuf[o] = make_uint2(j, __ldg(&perm[acc1]));
        if constexpr (BATCH) wfr[o] = (uint16_t)f;
    }
    cnt += tot;
    __syncwarp();
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

template <int VARIANT, bool BATCH>
__global__ void __launch_bounds__(kThreads, VARIANT != 0 ? 5 : (BATCH ? HRR_CULL_BATCH_MIN_BLOCKS : HRR_CULL_MIN_BLOCKS))
cull_kernel(const Launch Lc, const Frame single) {
    __shared__ uint2 buf[kWarps][kBuf];
    __shared__ uint16_t buf_frame[BATCH ? kWarps : 1][BATCH ? kBuf : 1];
    __shared__ Frame sframes[BATCH ? kSmemFrames : 1];
    // The traversal stack: its first kSmemLevels levels in shared memory ([level][thread],
    // so that lanes at the same depth hit distinct banks), deeper levels in local memory.
    // Keeping the hot levels out of L1 leaves L1 to the node records.
    __shared__ uint2 sstack[kSmemLevels > 0 ? kSmemLevels : 1][kThreads];

    if constexpr (BATCH) {
        const uint32_t ns = min(Lc.n_frames, kSmemFrames);
        const uint32_t words = ns * (uint32_t)(sizeof(Frame) / 4);
        for (uint32_t w = threadIdx.x; w < words; w += kThreads)
            reinterpret_cast<uint32_t *>(sframes)[w] = reinterpret_cast<const uint32_t *>(Lc.frames)[w];
        __syncthreads();
    }
    const Frame *glob = Lc.frames;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint2 *wbuf = buf[warp];
    uint16_t *wfr = BATCH ? buf_frame[warp] : nullptr;

    bool alive = false;
    bool more = true;  // warp-uniform: the eye cursor may still hand out eyes
    uint32_t f = 0, j = 0, r = 0, c = 0, node = 0, visits = 0, cnt = 0;
    // Argmin of the current node's range minimum. Exactly one child holds it and has the
    // same minimum, so each visit computes at most one new range minimum: the other
    // internal child's. The root's is computed when the eye starts.
    uint32_t kmin = 0;
    float ex = 0.f, ey = 0.f, ez = 0.f;
    // The current frame's hot fields, held in registers in a batch (a single frame reads
    // them from the kernel parameters).
    const float4 *f_nodes = single.nodes;
    float f_tau = single.tau;
    uint32_t f_nl = single.n_lights;
    unsigned long long visit_acc = 0;  // visits of finished eyes of frame f, not yet published
    uint2 deep[kStack - kSmemLevels];  // (node, argmin of its range minimum)
    int sp = 0;

    for (;;) {
        uint32_t acc0 = kNone, acc1 = kNone;
        unsigned alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        if (more && (uint32_t)__popc(alive_mask) < Lc.refill_below) {
            const unsigned idle = ~alive_mask;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(Lc.cursor, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + __popc(idle) >= Lc.total) more = false;
            if (!alive) {
                const unsigned long long g = base + __popc(idle & lt);
                if (g < Lc.total) {
                    if constexpr (BATCH) {  // last frame whose cursor offset is <= g
                        uint32_t lo = 0, hi = Lc.n_frames - 1;
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi + 1) >> 1;
                            if (frame_at<BATCH>(single, sframes, glob, mid).cursor_begin <= g) lo = mid;
                            else hi = mid - 1;
                        }
                        if (lo != f && visit_acc) {
                            atomicAdd(&frame_at<BATCH>(single, sframes, glob, f).counts[1], visit_acc);
                            visit_acc = 0;
                        }
                        f = lo;
                    }
                    const Frame &fr = frame_at<BATCH>(single, sframes, glob, f);
                    if constexpr (BATCH) {
                        f_nodes = fr.nodes;
                        f_tau = fr.tau;
                        f_nl = fr.n_lights;
                    }
                    j = fr.eye_begin + (uint32_t)(g - fr.cursor_begin);
                    ex = fr.ex[j];
                    ey = fr.ey[j];
                    ez = fr.ez[j];
                    const uint32_t tx = fr.px[j] % fr.tile_w, ty = fr.py[j] % fr.tile_h;
                    r = fr.tile[ty * fr.tile_w + tx] + fr.shift_offset;
                    if (fr.n_lights == 1) {  // the root is a leaf (record 0, slot 0)
                        const float4 q0 = fr.nodes[0];
                        if (hrr_leaf_accepts(__brev(0u) + r, fr.tau, q0.x, q0.y, q0.z, q0.w, ex, ey, ez))
                            acc0 = 0;
                        if (fr.eye_visits) fr.eye_visits[j] = 0;
                    } else {
                        c = __brev(0u - r);
                        node = 0;
                        kmin = range_argmin<VARIANT>(0u, fr.n_lights, r, c);
                        sp = 0;
                        visits = 0;
                        alive = true;
                    }
                }
            }
            alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        }
        if (alive_mask == 0u && !more) {
            emit<BATCH>(single, sframes, glob, wbuf, wfr, cnt, lane, f, j, acc0, acc1);
            break;
        }

        if (alive) {
            const float4 *nodes = BATCH ? f_nodes : single.nodes;
            const float tau = BATCH ? f_tau : single.tau;
            const uint32_t n_lights = BATCH ? f_nl : single.n_lights;
            ++visits;
            const float4 q0 = __ldg(&nodes[4 * (size_t)node + 0]);
            const float4 q1 = __ldg(&nodes[4 * (size_t)node + 1]);
            const float4 q2 = __ldg(&nodes[4 * (size_t)node + 2]);
            const float4 q3 = __ldg(&nodes[4 * (size_t)node + 3]);
            const uint32_t split = __float_as_uint(q1.w);
            const uint32_t other = __float_as_uint(q3.w);
            const uint32_t first = min(node, other), last = max(node, other);
            bool go0 = false, go1 = false;
            uint32_t k0 = kNone, k1 = kNone;
            if (last >= n_lights || split - first >= last - first) {  // needs first <= split < last
                atomicOr(Lc.flags, HRR_FLAG_TOPOLOGY);                   // corrupt record
                sp = 0;
            } else {
                const bool int0 = first != split, int1 = split + 1u != last;
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
                    atomicOr(Lc.flags, HRR_FLAG_STACK);
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
                visit_acc += visits;
                uint32_t *ev = frame_at<BATCH>(single, sframes, glob, f).eye_visits;
                if (ev) ev[j] = visits;
            }
        }
        emit<BATCH>(single, sframes, glob, wbuf, wfr, cnt, lane, f, j, acc0, acc1);
    }
    if (cnt) flush<BATCH>(single, sframes, glob, wbuf, wfr, cnt, lane);
    if constexpr (BATCH) {
        if (visit_acc) atomicAdd(&frame_at<BATCH>(single, sframes, glob, f).counts[1], visit_acc);
    } else {
        // visit_acc < 2^32 per lane in practice; sum both halves to stay exact regardless
        const unsigned long long wsum =
            (unsigned long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(visit_acc & 0xFFFFFFFFull)) +
            ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, (unsigned)(visit_acc >> 32)) << 32);
        if (lane == 0 && wsum) atomicAdd(&single.counts[1], wsum);
    }
}

// Resident blocks per SM of a traversal kernel (one cache per instantiation).
template <int VARIANT, bool BATCH>
int blocks_per_sm() {
    static int n = 0;
    if (!n) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, cull_kernel<VARIANT, BATCH>, kThreads, 0) !=
                cudaSuccess || m < 1)
            m = 1;
        n = m;
    }
    return n;
}

template <bool BATCH>
cudaError_t launch_variant(const hrr_tuning &tn, int sm_count, unsigned long long total, const Launch &Lc,
                           const Frame &single, cudaStream_t st) {
    const int variant = tn.rangemin_variant;
    const unsigned long long blocks_needed = (total + kThreads - 1) / kThreads;
    auto grid = [&](int per_sm) {
        if (tn.blocks_per_sm > 0 && (int)tn.blocks_per_sm < per_sm) per_sm = (int)tn.blocks_per_sm;
        return (unsigned)min((unsigned long long)per_sm * sm_count, blocks_needed);
    };
    if (variant == 0)
        cull_kernel<0, BATCH><<<grid(blocks_per_sm<0, BATCH>()), kThreads, 0, st>>>(Lc, single);
    else if (variant == 1)
        cull_kernel<1, BATCH><<<grid(blocks_per_sm<1, BATCH>()), kThreads, 0, st>>>(Lc, single);
    else
        cull_kernel<2, BATCH><<<grid(blocks_per_sm<2, BATCH>()), kThreads, 0, st>>>(Lc, single);
    return cudaGetLastError();
}

}  // namespace

int hrr_cull_impl(hrr_ctx *ctx, const hrr_eyes &E, uint32_t n_eyes, const hrr_tree *tree,
                  float tau, const hrr_cull_opts &opts, uint32_t *pairs, uint64_t cap,
                  uint64_t *out_count) {
    if (((uintptr_t)pairs & 7u) != 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs must be 8-byte aligned");
    cudaStream_t st = ctx->stream;
    HRR_CUDA(ctx, cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(unsigned long long), st));
    if (n_eyes > 0) {
        Frame fr{};
        fr.ex = E.x; fr.ey = E.y; fr.ez = E.z; fr.px = E.px; fr.py = E.py;
        fr.nodes = reinterpret_cast<const float4 *>(tree->nodes);
        fr.perm = tree->perm;
        fr.tile = ctx->tile;
        fr.pairs = reinterpret_cast<uint2 *>(pairs);
        fr.cap = cap;
        fr.counts = ctx->counters;  // [0] accepted, [1] visits
        fr.eye_visits = opts.eye_visits;
        fr.n_lights = tree->n;
        fr.tile_w = ctx->tile_w; fr.tile_h = ctx->tile_h;
        fr.shift_offset = opts.shift_offset;
        fr.tau = tau;
        fr.eye_begin = 0;
        fr.cursor_begin = 0;
        const hrr_tuning tn = hrr_tuning_of(opts);
        const Launch Lc{nullptr, 1, tn.refill_below, n_eyes, ctx->counters + 3, ctx->counters + 2};
        hrr_timing_begin(ctx);
        const cudaError_t e = launch_variant<false>(tn, ctx->sm_count, n_eyes, Lc, fr, st);
        hrr_timing_end(ctx);
        ++ctx->launches;
        HRR_CUDA(ctx, e);
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

cudaError_t hrr_cull_batch_enqueue(int sm_count, const hrr_cull_frame_t *dev_frames, uint32_t n_frames,
                                   unsigned long long total, unsigned long long *cursor,
                                   unsigned long long *flags, const hrr_tuning &tuning, cudaStream_t st) {
    const hrr_tuning tn = hrr_tuning_normalized(tuning);
    const Launch Lc{dev_frames, n_frames, tn.refill_below, total, cursor, flags};
    const Frame unused{};
    if (total == 0) return cudaSuccess;
    return launch_variant<true>(tn, sm_count, total, Lc, unused, st);
}
