// The culling traversal kernels and their launch helpers; hrr_cull.cu holds the host entry points.
//
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
// Execution: a persistent grid (a whole number of resident blocks per SM) in which each
// warp traverses one eye at a time. The warp's stack of pending nodes is a ring in shared
// memory; every step pops up to 32 nodes, one per lane, and the lanes push the children
// that survive their tests back as one compacted run (ballot + popc). All lanes of a step
// execute the same node test on the same eye, so the warp stays converged except at leaf
// children. When the ring would overflow, its oldest entries move to a per-warp area in
// global memory, and they come back when the ring runs low.
//
// Memory: the kernel is bound by the L1 data pipe (one scattered record per lane per
// step), so each record is fetched with two 256-bit loads instead of four 128-bit ones.
// A node's range minimum is attained at its argmin, which lies in exactly one child;
// carrying the argmin with each stack entry means only the other child's minimum has to be
// computed. Accepted pairs are staged per warp in shared memory and appended to the output
// with one atomic per frame and coalesced 8-byte stores.
//
// One launch may cover many frames (a batch): the eye cursor then runs over the eyes of all
// frames, each warp finds its eye's frame by binary search over the frames' cursor offsets,
// and the frames' descriptors are staged in shared memory. Frames of different sizes share
// the launch without any per-frame tail.
#pragma once

#include <algorithm>

#include "hrr_internal.cuh"

namespace {

// Launch shape, fixed at compile time (the values measured fastest on GB300).
#ifndef HRR_CULL_MIN_BLOCKS
#define HRR_CULL_MIN_BLOCKS 6  // resident 256-thread blocks per SM (40 registers, no spills)
#endif
#ifndef HRR_CULL_BATCH_MIN_BLOCKS
#define HRR_CULL_BATCH_MIN_BLOCKS 6  // the batched form: frame fields come from the constant cache
#endif
#ifndef HRR_CULL_RING
#define HRR_CULL_RING 256  // stack entries per warp kept in shared memory (a power of two)
#endif
#ifndef HRR_CULL_BUF
#define HRR_CULL_BUF 128  // staged output pairs per warp
#endif

constexpr int kThreads = HRR_CULL_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kBuf = HRR_CULL_BUF;
constexpr uint32_t kRing = HRR_CULL_RING;
constexpr uint32_t kRingMask = kRing - 1;
static_assert((kRing & kRingMask) == 0 && kRing >= 128, "ring size");
constexpr uint32_t kMaxFrames = HRR_CULL_MAX_FRAMES;  // frames of one batched launch
constexpr uint32_t kNone = 0xFFFFFFFFu;

using Frame = hrr_cull_frame_t;
static_assert(sizeof(Frame) == 128, "frame descriptor layout");

struct Launch {
    uint32_t n_frames;
    uint32_t spill_cap;             // stack entries per warp in the spill area
    unsigned long long total;       // eyes of this launch over all frames
    unsigned long long *cursor;     // global eye cursor (starts at 0)
    unsigned long long *flags;      // HRR_FLAG_* bits
    uint2 *spill;                   // grid warps x spill_cap stack entries
};

// The launch's frame descriptors travel as a kernel parameter, so the traversal reads them
// through the constant cache (and may re-read them instead of holding them in registers).
template <uint32_t N>
struct FrameArray {
    Frame f[N];
};

// Frame f of the launch (always the only one for a single frame).
template <bool BATCH>
__device__ __forceinline__ const Frame &frame_at(const Frame *F, uint32_t f) {
    if constexpr (!BATCH) return F[0];
    else return F[f];
}

// The 64-byte node record (both children) as two 256-bit read-only loads.
__device__ __forceinline__ void load_record(const float4 *p, float4 &q0, float4 &q1, float4 &q2,
                                            float4 &q3) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(q0.x), "=f"(q0.y), "=f"(q0.z), "=f"(q0.w), "=f"(q1.x), "=f"(q1.y), "=f"(q1.z), "=f"(q1.w)
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8+32];"
        : "=f"(q2.x), "=f"(q2.y), "=f"(q2.z), "=f"(q2.w), "=f"(q3.x), "=f"(q3.y), "=f"(q3.z), "=f"(q3.w)
        : "l"(p));
}

// Append the warp's staged pairs to their frames' outputs: one atomic per frame present in
// each 32-entry chunk (a chunk rarely holds more than one frame). The pairs are written
// once and never read by the kernel, so they are stored with the streaming (evict-first)
// hint: the output stream then does not push the node records out of L2.
template <bool BATCH>
__device__ __forceinline__ void flush(const Frame *F, const uint2 *wbuf, const uint16_t *wfr, uint32_t cnt,
                                      int lane) {
    if constexpr (!BATCH) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&F[0].counts[0], (unsigned long long)cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (uint32_t k = lane; k < cnt; k += 32) {
            const unsigned long long o = base + k;
            if (o < F[0].cap) __stcs(&F[0].pairs[o], wbuf[k]);
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
                base = atomicAdd(&frame_at<BATCH>(F, f).counts[0], (unsigned long long)__popc(grp));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (has) {
                const Frame &fr = frame_at<BATCH>(F, f);
                const unsigned long long o = base + rank;
                if (o < fr.cap) __stcs(&fr.pairs[o], wbuf[k]);
            }
        }
    }
    __syncwarp();
}

// Stage up to two accepted leaves per lane of eye j (warp-collective).
template <bool BATCH>
__device__ __forceinline__ void emit(const Frame *F, uint2 *wbuf, uint16_t *wfr, uint32_t &cnt, int lane,
                                     uint32_t f, uint32_t j, uint32_t acc0, uint32_t acc1) {
    const unsigned b0 = __ballot_sync(0xFFFFFFFFu, acc0 != kNone);
    const unsigned b1 = __ballot_sync(0xFFFFFFFFu, acc1 != kNone);
    const uint32_t tot = __popc(b0) + __popc(b1);
    if (tot == 0) return;
    if (cnt + tot > (uint32_t)kBuf) {
        flush<BATCH>(F, wbuf, wfr, cnt, lane);
        cnt = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t *perm = frame_at<BATCH>(F, f).perm;
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
    hrr_rangemin_closed(a, b, r, &k);
    return k;
}

// The traversal over the frames F (F[0] alone for a single frame).
template <int VARIANT, bool BATCH>
__device__ __forceinline__ void traverse(const Launch &Lc, const Frame *F) {
    __shared__ uint2 buf[kWarps][kBuf];
    __shared__ uint16_t buf_frame[BATCH ? kWarps : 1][BATCH ? kBuf : 1];
    __shared__ uint2 ring_all[kWarps][kRing];  // (node, argmin of its range minimum)

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint2 *wbuf = buf[warp];
    uint16_t *wfr = BATCH ? buf_frame[warp] : nullptr;
    uint2 *ring = ring_all[warp];
    // This warp's spill area (formed where it is used, so that it holds no registers).
#define HRR_WARP_SPILL (Lc.spill + ((size_t)blockIdx.x * kWarps + warp) * Lc.spill_cap)
    uint32_t cnt = 0, f = 0;
    unsigned long long visit_acc = 0;  // visits of finished eyes of frame f, not yet published

    for (;;) {
        // The warp's next eye (warp-uniform from here on).
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(Lc.cursor, 1ull);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g >= Lc.total) break;
        if constexpr (BATCH) {  // last frame whose cursor offset is <= g
            uint32_t lo = 0, hi = Lc.n_frames - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (frame_at<BATCH>(F, mid).cursor_begin <= g) lo = mid;
                else hi = mid - 1;
            }
            if (lo != f && visit_acc) {
                if (lane == 0) atomicAdd(&frame_at<BATCH>(F, f).counts[1], visit_acc);
                visit_acc = 0;
            }
            f = lo;
        }
        const Frame &fr = frame_at<BATCH>(F, f);
        const float4 *nodes = fr.nodes;
        const float tau = fr.tau;
        const uint32_t n_lights = fr.n_lights;
        const uint32_t j = fr.eye_begin + (uint32_t)(g - fr.cursor_begin);
        const float ex = fr.ex[j], ey = fr.ey[j], ez = fr.ez[j];
        const uint32_t tx = fr.px[j] % fr.tile_w, ty = fr.py[j] % fr.tile_h;
        const uint32_t r = fr.tile[ty * fr.tile_w + tx] + fr.shift_offset;
        if (n_lights == 1) {  // the root is a leaf (record 0, slot 0)
            uint32_t acc = kNone;
            if (lane == 0) {
                const float4 q0 = __ldg(&nodes[0]);
                if (hrr_leaf_accepts(__brev(0u) + r, tau, q0.x, q0.y, q0.z, q0.w, ex, ey, ez)) acc = 0;
                if (fr.eye_visits) fr.eye_visits[j] = 0;
            }
            emit<BATCH>(F, wbuf, wfr, cnt, lane, f, j, acc, kNone);
            continue;
        }
        const uint32_t c = __brev(0u - r);
        // Stack: logical entries [0, S); the newest R of them are in the ring at index & mask,
        // the others in the spill area at their logical index.
        uint32_t S = 1, R = 1, visits = 0;
        if (lane == 0) ring[0] = make_uint2(0u, range_argmin<VARIANT>(0u, n_lights, r, c));
        __syncwarp();
        while (S > 0) {
            if (visits >= n_lights) {  // each internal node is visited at most once per eye
                if (lane == 0) atomicOr(Lc.flags, HRR_FLAG_TOPOLOGY);
                break;
            }
            const uint32_t m = min(32u, S);
            if (R < m) {  // bring spilled entries back into the ring
                const uint32_t fc = min(S - R, kRing / 2 - R);
                const uint32_t base = S - R - fc;
                const uint2 *spill = HRR_WARP_SPILL;
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

            bool go0 = false, go1 = false;
            uint32_t k0 = 0, k1 = 0, split = 0;
            uint32_t acc0 = kNone, acc1 = kNone;
            if (active) {
                const uint32_t node = e.x, kmin = e.y;
                float4 q0, q1, q2, q3;
                load_record(&nodes[4 * (size_t)node], q0, q1, q2, q3);
                split = __float_as_uint(q1.w);
                const uint32_t other = __float_as_uint(q3.w);
                const uint32_t first = min(node, other), last = max(node, other);
                if (last >= n_lights || split - first >= last - first) {  // needs first <= split < last
                    atomicOr(Lc.flags, HRR_FLAG_TOPOLOGY);                   // corrupt record
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
            }
            // Push the surviving children as one compacted run.
            const unsigned b0 = __ballot_sync(0xFFFFFFFFu, go0), b1 = __ballot_sync(0xFFFFFFFFu, go1);
            const uint32_t n = __popc(b0) + __popc(b1);
            if (n) {
                if (R + n > kRing) {  // move the oldest resident entries to the spill area
                    const uint32_t s = (R + n - kRing + 31u) & ~31u;
                    const uint32_t base = S - R;
                    if (base + s > Lc.spill_cap) {
                        if (lane == 0) atomicOr(Lc.flags, HRR_FLAG_STACK);
                        break;
                    }
                    uint2 *spill = HRR_WARP_SPILL;
                    for (uint32_t k = lane; k < s; k += 32) spill[base + k] = ring[(base + k) & kRingMask];
                    R -= s;
                    __syncwarp();
                }
                if (go0) ring[(S + __popc(b0 & lt)) & kRingMask] = make_uint2(split, k0);
                if (go1) ring[(S + __popc(b0) + __popc(b1 & lt)) & kRingMask] = make_uint2(split + 1u, k1);
                S += n;
                R += n;
                __syncwarp();
            }
            if (__any_sync(0xFFFFFFFFu, (acc0 & acc1) != kNone))
                emit<BATCH>(F, wbuf, wfr, cnt, lane, f, j, acc0, acc1);
        }
        if (lane == 0) {
            uint32_t *ev = frame_at<BATCH>(F, f).eye_visits;
            if (ev) ev[j] = visits;
        }
        visit_acc += visits;
    }
    if (cnt) flush<BATCH>(F, wbuf, wfr, cnt, lane);
    if (lane == 0 && visit_acc) {
        if constexpr (BATCH) atomicAdd(&frame_at<BATCH>(F, f).counts[1], visit_acc);
        else atomicAdd(&F[0].counts[1], visit_acc);
    }
#undef HRR_WARP_SPILL
}

// A single frame travels as a plain kernel parameter; a batch's frames as a grid-constant
// array (indexed by the frame a warp is on).
template <int VARIANT>
__global__ void __launch_bounds__(kThreads, HRR_CULL_MIN_BLOCKS)
cull_single_kernel(const Launch Lc, const Frame fr) {
    traverse<VARIANT, false>(Lc, &fr);
}

template <int VARIANT>
__global__ void __launch_bounds__(kThreads, HRR_CULL_BATCH_MIN_BLOCKS)
cull_batch_kernel(const __grid_constant__ Launch Lc, const __grid_constant__ FrameArray<kMaxFrames> FA) {
    traverse<VARIANT, true>(Lc, FA.f);
}

template <int VARIANT, bool BATCH>
const void *kernel_fn() {
    if constexpr (BATCH) return reinterpret_cast<const void *>(cull_batch_kernel<VARIANT>);
    else return reinterpret_cast<const void *>(cull_single_kernel<VARIANT>);
}

// Resident blocks per SM of a traversal kernel (one cache per instantiation).
template <int VARIANT, bool BATCH>
int occupancy() {
    static int n = 0;
    if (!n) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, kernel_fn<VARIANT, BATCH>(), kThreads, 0) !=
                cudaSuccess || m < 1)
            m = 1;
        n = m;
    }
    return n;
}

template <bool BATCH>
int occupancy_of(int variant) {
    return variant == 0 ? occupancy<0, BATCH>() : occupancy<2, BATCH>();
}

cudaError_t launch_single(const hrr_tuning &tn, unsigned grid, const Launch &Lc, const Frame &fr, cudaStream_t st) {
    if (tn.rangemin_variant == 0) cull_single_kernel<0><<<grid, kThreads, 0, st>>>(Lc, fr);
    else cull_single_kernel<2><<<grid, kThreads, 0, st>>>(Lc, fr);
    return cudaGetLastError();
}

cudaError_t launch_batch(const hrr_tuning &tn, unsigned grid, const Launch &Lc, const FrameArray<kMaxFrames> &fa,
                         cudaStream_t st) {
    if (tn.rangemin_variant == 0) cull_batch_kernel<0><<<grid, kThreads, 0, st>>>(Lc, fa);
    else cull_batch_kernel<2><<<grid, kThreads, 0, st>>>(Lc, fa);
    return cudaGetLastError();
}

}  // namespace
