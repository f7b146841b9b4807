// The culling traversal kernels (device code only); hrr_cull.cu instantiates and launches them.
//
// Hierarchical Russian-roulette culling with blue-noise dithered QMC sequences (Sec. 1).
//
// For eye j with shift r_j (tile entry at its pixel), the traversal starts at the root and,
// at every visited node, tests the node's children from one record:
//   * a leaf child i is accepted iff brev(i) + r_j < ceil(p_ij 2^32) (exact float32 p);
//   * an internal child with leaf range [a, b) is descended unless the range minimum
//     v(a, b) = min_{i in [a,b)} (brev(i) + r_j) mod 2^32 passes the conservative cull test
//     (v is at least the threshold of every light below; then none can be accepted).
// The accepted set therefore equals flat Russian roulette over all pairs.
//
// Node width. The hierarchy is binary; a traversal reads it either with binary nodes
// (64-byte records: both children) or with nodes of width four (128-byte records: the four
// grandchildren, or a leaf child in place of its two slots), visiting only even-depth nodes.
// The cull test is monotone (a smaller box, a smaller maximum intensity and a range minimum
// over a sub-range never turn a cull into a visit), so both widths accept the same pairs;
// width four pops half as many nodes, with half the stack traffic and loop overhead per
// child tested, for one extra range minimum per visit.
//
// Execution: a persistent grid (a whole number of resident blocks per SM) in which each
// warp traverses one eye at a time. The warp's stack of pending nodes is a ring in shared
// memory; every step pops up to 32 nodes, one per lane, and the lanes push the children
// that survive their tests back as one compacted run (ballot + popc). All lanes of a step
// execute the same node test on the same eye, so the warp stays converged except at leaf
// children. When the ring would overflow, its oldest entries move to a per-warp area in
// global memory, and they come back when the ring runs low. The stack never exceeds
// (w - 1) * 32 * L + 32 entries for node width w and L depth levels of pushed nodes (each
// remainder of a pushed run below the top holds at most (w - 1) * 32 entries, and the
// shallowest depth of those runs grows from the bottom of the stack to its top), and the
// spill area is sized by that bound.
//
// Memory: the kernel is bound by the L1 data pipe (one scattered record per lane per
// step), so each record is fetched with 256-bit loads that do not allocate in L1. A node's
// range minimum is attained at its argmin, which lies in exactly one child; carrying the
// argmin with each stack entry means only the other children's minima have to be
// computed. Accepted pairs are staged
// per warp in shared memory and appended to the output with one atomic per frame and
// coalesced 8-byte stores.
//
// The head (forms with top levels, binary records): each eye starts by evaluating the 62
// nodes below the root of the top HRR_TOP_LEVELS levels, one per lane in two passes,
// instead of walking those levels one per step with 1, 2, 4, 8 and 16 lanes busy. A
// single-frame launch stages the top slots in shared memory once per block; in a batched
// launch, whose warps move between frames, each eye reads its frame's slots (3 KB, cached
// in L1 and L2) directly. The cull test is
// monotone: a child's box lies inside its parent's, its maximum intensity is at most the
// parent's and its range minimum at least the parent's, and the test culls at least as
// much for each, so a node below the root is visited iff its own test passes, whatever its
// ancestors' results. The head counts the root and the visited nodes above the deepest top
// level as visits, tests the top's leaves, and pushes the visited nodes of the deepest top
// level (with their argmins) as the stack the walk starts from: the same visited set, visit
// count and accepted set as a walk from the root.
//
// One launch may cover many frames (a batch): the eye cursor then runs over the eyes of all
// frames, each warp finds its eye's frame by binary search over the frames' cursor offsets,
// and the frames' descriptors are read through the constant cache. Frames of different
// sizes share the launch without any per-frame tail.
#pragma once

#include <algorithm>

#include "hrr_internal.cuh"

namespace {

#ifndef HRR_CULL_BUF
#define HRR_CULL_BUF 128  // staged output pairs per warp
#endif

constexpr int kBuf = HRR_CULL_BUF;
constexpr uint32_t kMaxFrames = HRR_CULL_MAX_FRAMES;  // frames of one batched launch
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Resident threads per SM each instantiation is compiled for (the register budget):
// 40 registers for binary records (6 blocks of 256 threads), 64 for width four.
template <int W>
constexpr int min_blocks(int threads) {
    return (W == 2 ? 1536 : 1024) / threads;
}

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

// 32 bytes (two float4) as one 256-bit read-only load that does not allocate in L1: the
// records are scattered and rarely reused from L1, and filling it with them would take
// L1 data-pipe cycles the kernel is bound by (they come from L2 either way).
__device__ __forceinline__ void load32(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
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

// Stage the accepted leaves (up to W per lane, kNone for none) of eye j (warp-collective).
template <bool BATCH, int W>
__device__ __forceinline__ void emit(const Frame *F, uint2 *wbuf, uint16_t *wfr, uint32_t &cnt, int lane,
                                     uint32_t f, uint32_t j, const uint32_t (&acc)[W]) {
    unsigned bal[W];
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        bal[k] = __ballot_sync(0xFFFFFFFFu, acc[k] != kNone);
        tot += __popc(bal[k]);
    }
    if (tot == 0) return;
    if (cnt + tot > (uint32_t)kBuf) {  // tot <= 32 W <= kBuf
        flush<BATCH>(F, wbuf, wfr, cnt, lane);
        cnt = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t *perm = frame_at<BATCH>(F, f).perm;
    uint32_t base = cnt;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if (acc[k] != kNone) {
            const uint32_t o = base + __popc(bal[k] & lt);
            wbuf[o] = make_uint2(j, __ldg(&perm[acc[k]]));
            if constexpr (BATCH) wfr[o] = (uint16_t)f;
        }
        base += __popc(bal[k]);
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

// The eye a traversal works on.
struct Eye {
    float x, y, z, tau;
    float scale;    // the node test's scale, hrr_node_scale(tau)
    uint32_t r, c;  // shift and brev(2^32 - r)
};

// What one lane's visit produces: up to W children to push (node, argmin of its range
// minimum) and up to W accepted leaves.
template <int W>
struct Visit {
    bool go[W];
    uint32_t node[W], karg[W], acc[W];
};

// Test one child slot: an internal child (range of more than one leaf) survives unless
// its range minimum at argmin k culls it; the box is (lo, imax, hi).
__device__ __forceinline__ bool survives(const Eye &E, const float4 &lo, const float4 &hi, uint32_t k) {
    float den, rhs;
    hrr_node_bound(E.scale, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, lo.w, E.x, E.y, E.z, den, rhs);
    return !hrr_node_culls(__brev(k) + E.r, den, rhs);
}

// A visit of binary node `node`: its 64-byte record holds both children (box low corner
// with the maximum intensity, box high corner with `split` / the range's other end).
template <int VARIANT>
__device__ __forceinline__ void visit(const float4 *nodes, uint32_t n_lights, uint32_t node, uint32_t kmin,
                                      const Eye &E, unsigned long long *flags, Visit<2> &V) {
    float4 q0, q1, q2, q3;
    load32(&nodes[4 * (size_t)node], q0, q1);
    load32(&nodes[4 * (size_t)node + 2], q2, q3);
    const uint32_t split = __float_as_uint(q1.w);
    const uint32_t other = __float_as_uint(q3.w);
    const uint32_t first = min(node, other), last = max(node, other);
    if (last >= n_lights || split - first >= last - first) {  // needs first <= split < last
        atomicOr(flags, HRR_FLAG_TOPOLOGY);                    // corrupt record
        return;
    }
    const bool int0 = first != split, int1 = split + 1u != last;
    const bool kin0 = kmin <= split;
    // the other child's argmin (unused when that child is a leaf: computing it anyway
    // keeps the warp on one path)
    const uint32_t knew = range_argmin<VARIANT>(kin0 ? split + 1u : first, kin0 ? last + 1u : split + 1u, E.r, E.c);
    V.karg[0] = kin0 ? kmin : knew;
    V.karg[1] = kin0 ? knew : kmin;
    V.node[0] = split;
    V.node[1] = split + 1u;
    V.go[0] = int0 && survives(E, q0, q1, V.karg[0]);
    V.go[1] = int1 && survives(E, q2, q3, V.karg[1]);
    if (!int0 || !int1) {  // leaf children: one test site, a second for two leaves
        const uint32_t i = !int0 ? split : last;
        const float4 ql = !int0 ? q0 : q2;
        if (hrr_leaf_accepts(__brev(i) + E.r, E.tau, E.scale, ql.x, ql.y, ql.z, ql.w, E.x, E.y, E.z)) V.acc[0] = i;
        if (!int0 && !int1 &&
            hrr_leaf_accepts(__brev(last) + E.r, E.tau, E.scale, q2.x, q2.y, q2.z, q2.w, E.x, E.y, E.z))
            V.acc[1] = last;
    }
}

// A visit of node g read with width four: its 128-byte record holds the four grandchild
// slots [first, s0], [s0 + 1, split], [split + 1, s1], [s1 + 1, last] (a leaf child fills its
// first slot and leaves the second empty). The parent's argmin lies in one child; one range
// minimum gives the other child's, and one more per internal child splits it between that
// child's two slots.
template <int VARIANT>
__device__ __forceinline__ void visit(const float4 *wide, uint32_t n_lights, uint32_t g, uint32_t kmin,
                                      const Eye &E, unsigned long long *flags, Visit<4> &V) {
    float4 q[8];
    load32(&wide[8 * (size_t)g], q[0], q[1]);
    load32(&wide[8 * (size_t)g + 2], q[2], q[3]);
    load32(&wide[8 * (size_t)g + 4], q[4], q[5]);
    load32(&wide[8 * (size_t)g + 6], q[6], q[7]);
    const uint32_t s0 = __float_as_uint(q[1].w), split = __float_as_uint(q[3].w);
    const uint32_t s1 = __float_as_uint(q[5].w), other = __float_as_uint(q[7].w);
    const uint32_t first = min(g, other), last = max(g, other);
    const bool c0int = first != split, c1int = split + 1u != last;
    // first <= s0 <= split < last, split < s1 <= last, and an internal child's split inside it
    // (so every internal slot is a node below g, with a record)
    if (last >= n_lights || s0 - first > split - first || split - first >= last - first ||
        s1 - split - 1u > last - split - 1u || (c0int && s0 == split) || (c1int && s1 == last)) {
        atomicOr(flags, HRR_FLAG_TOPOLOGY);  // corrupt record
        return;
    }
    const bool kin0 = kmin <= split;
    const uint32_t kc = range_argmin<VARIANT>(kin0 ? split + 1u : first, kin0 ? last + 1u : split + 1u, E.r, E.c);
    const uint32_t kA = kin0 ? kmin : kc, kB = kin0 ? kc : kmin;  // argmins of children 0 and 1
    uint32_t k[4] = {kA, kA, kB, kB};
    if (c0int) {
        const bool in0 = kA <= s0;
        const uint32_t kx = range_argmin<VARIANT>(in0 ? s0 + 1u : first, in0 ? split + 1u : s0 + 1u, E.r, E.c);
        k[0] = in0 ? kA : kx;
        k[1] = in0 ? kx : kA;
    }
    if (c1int) {
        const bool in2 = kB <= s1;
        const uint32_t ky = range_argmin<VARIANT>(in2 ? s1 + 1u : split + 1u, in2 ? last + 1u : s1 + 1u, E.r, E.c);
        k[2] = in2 ? kB : ky;
        k[3] = in2 ? ky : kB;
    }
    const uint32_t a[4] = {first, s0 + 1u, split + 1u, s1 + 1u};
    const uint32_t b[4] = {s0, split, s1, last};  // inclusive; a > b: an empty slot
    V.node[0] = s0;
    V.node[1] = s0 + 1u;
    V.node[2] = s1;
    V.node[3] = s1 + 1u;
    bool any_leaf = false;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        V.karg[t] = k[t];
        V.go[t] = a[t] < b[t] && survives(E, q[2 * t], q[2 * t + 1], k[t]);
        any_leaf |= a[t] == b[t];
    }
    if (any_leaf) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (a[t] == b[t] &&
                hrr_leaf_accepts(__brev(a[t]) + E.r, E.tau, E.scale, q[2 * t].x, q[2 * t].y, q[2 * t].z, q[2 * t].w, E.x,
                                 E.y, E.z))
                V.acc[t] = a[t];
    }
}

// The head of eye j's traversal over the top slots `top` (shared memory for a single frame,
// global memory for a batch): stages the top's accepted leaves, pushes the visited nodes of
// the deepest top level onto the empty ring, and returns the visits it accounts for (the
// root and the visited nodes above that level).
template <int VARIANT, bool BATCH, int W>
__device__ __forceinline__ uint32_t head(const float4 *top, const Eye &E, const Frame *F, uint2 *wbuf, uint16_t *wfr,
                                         uint32_t &cnt, int lane, uint32_t f, uint32_t j, uint2 *ring,
                                         uint32_t &pushed) {
    constexpr uint32_t kDeep = HRR_TOP_SLOTS / 2;  // first slot of the deepest top level
    const unsigned lt = (1u << lane) - 1u;
    uint32_t visits = 1, n = 0;  // the root
#pragma unroll
    for (uint32_t p = 0; p < (HRR_TOP_SLOTS + 31) / 32; ++p) {
        const uint32_t s = 1u + (uint32_t)lane + 32u * p;  // slots 1 .. HRR_TOP_SLOTS - 1
        bool vis = false;
        uint32_t acc[W];
#pragma unroll
        for (int t = 0; t < W; ++t) acc[t] = kNone;
        uint32_t node = 0, karg = 0;
        if (s < HRR_TOP_SLOTS) {
            float4 a, h, x;
            if constexpr (BATCH) {
                a = __ldg(&top[3 * s]);
                h = __ldg(&top[3 * s + 1]);
                x = __ldg(&top[3 * s + 2]);
            } else {
                a = top[3 * s];
                h = top[3 * s + 1];
                x = top[3 * s + 2];
            }
            const uint32_t kind = __float_as_uint(x.z);
            const uint32_t first = __float_as_uint(h.w), last = __float_as_uint(x.x);
            if (kind == HRR_TOP_INTERNAL) {
                karg = range_argmin<VARIANT>(first, last + 1u, E.r, E.c);
                vis = survives(E, a, h, karg);
                node = __float_as_uint(x.y);
            } else if (kind == HRR_TOP_LEAF &&
                       hrr_leaf_accepts(__brev(first) + E.r, E.tau, E.scale, a.x, a.y, a.z, a.w, E.x, E.y, E.z)) {
                acc[0] = first;
            }
        }
        const bool deep = s >= kDeep;
        visits += __popc(__ballot_sync(0xFFFFFFFFu, vis && !deep));
        const unsigned bp = __ballot_sync(0xFFFFFFFFu, vis && deep);
        if (vis && deep) ring[n + __popc(bp & lt)] = make_uint2(node, karg);
        n += __popc(bp);
        if (__any_sync(0xFFFFFFFFu, acc[0] != kNone)) emit<BATCH, W>(F, wbuf, wfr, cnt, lane, f, j, acc);
    }
    __syncwarp();
    pushed = n;
    return visits;
}

// The traversal over the frames F (F[0] alone for a single frame); TOP levels of the
// hierarchy evaluated by the head (0: none, the walk starts at the root).
template <int VARIANT, bool BATCH, int W, int RING, int THREADS, int TOP>
__device__ __forceinline__ void traverse(const Launch &Lc, const Frame *F) {
    constexpr int kWarps = THREADS / 32;
    constexpr uint32_t kRing = RING;
    constexpr uint32_t kRingMask = kRing - 1;
    // a step pushes at most 32 W entries; making room for them must only move entries that
    // are resident (see the spill below), which needs kRing >= 32 W + 31
    static_assert((kRing & kRingMask) == 0 && kRing >= 32 * W + 32, "ring size");
    static_assert(kBuf >= 32 * W, "output staging buffer");
    // the head reads the frames' binary records and pushes at most 32 entries
    static_assert(TOP == 0 || (TOP == (int)HRR_TOP_LEVELS && W == 2 && kRing >= 32), "top levels");
    __shared__ uint2 buf[kWarps][kBuf];
    __shared__ uint16_t buf_frame[BATCH ? kWarps : 1][BATCH ? kBuf : 1];
    __shared__ uint2 ring_all[kWarps][kRing];  // (node, argmin of its range minimum)
    constexpr bool kTopShared = TOP > 0 && !BATCH;
    __shared__ float4 top_s[kTopShared ? 3 * HRR_TOP_SLOTS : 1];
    if constexpr (kTopShared) {  // the top slots follow the frame's binary records
        if (F[0].n_lights > 1) {
            const float4 *src = F[0].nodes + 4 * (size_t)(F[0].n_lights - 1u);
            for (uint32_t k = threadIdx.x; k < 3 * HRR_TOP_SLOTS; k += THREADS) top_s[k] = __ldg(&src[k]);
        }
        __syncthreads();
    }

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
        unsigned long long gcur = 0;
        if (lane == 0) gcur = atomicAdd(Lc.cursor, 1ull);
        gcur = __shfl_sync(0xFFFFFFFFu, gcur, 0);
        if (gcur >= Lc.total) break;
        if constexpr (BATCH) {  // last frame whose cursor offset is <= gcur
            uint32_t lo = 0, hi = Lc.n_frames - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (frame_at<BATCH>(F, mid).cursor_begin <= gcur) lo = mid;
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
        const uint32_t n_lights = fr.n_lights;
        const uint32_t j = fr.eye_begin + (uint32_t)(gcur - fr.cursor_begin);
        Eye E;
        E.x = fr.ex[j];
        E.y = fr.ey[j];
        E.z = fr.ez[j];
        E.tau = fr.tau;
        E.scale = hrr_node_scale(fr.tau);
        const uint32_t tx = fr.px[j] % fr.tile_w, ty = fr.py[j] % fr.tile_h;
        E.r = fr.tile[ty * fr.tile_w + tx] + fr.shift_offset;
        if (n_lights == 1) {  // the root is a leaf (record 0, slot 0, in either layout)
            uint32_t acc[W];
#pragma unroll
            for (int t = 0; t < W; ++t) acc[t] = kNone;
            if (lane == 0) {
                const float4 q0 = __ldg(&nodes[0]);
                if (hrr_leaf_accepts(__brev(0u) + E.r, E.tau, E.scale, q0.x, q0.y, q0.z, q0.w, E.x, E.y, E.z)) acc[0] = 0;
                if (fr.eye_visits) fr.eye_visits[j] = 0;
            }
            emit<BATCH, W>(F, wbuf, wfr, cnt, lane, f, j, acc);
            continue;
        }
        E.c = __brev(0u - E.r);
        // Stack: logical entries [0, S); the newest R of them are in the ring at index & mask,
        // the others in the spill area at their logical index.
        uint32_t S = 1, R = 1, visits = 0;
        if constexpr (TOP > 0) {
            const float4 *top = kTopShared ? top_s : nodes + 4 * (size_t)(n_lights - 1u);
            visits = head<VARIANT, BATCH, W>(top, E, F, wbuf, wfr, cnt, lane, f, j, ring, S);
            R = S;
        } else {
            if (lane == 0) ring[0] = make_uint2(0u, range_argmin<VARIANT>(0u, n_lights, E.r, E.c));
            __syncwarp();
        }
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

            Visit<W> V;
#pragma unroll
            for (int t = 0; t < W; ++t) {
                V.go[t] = false;
                V.node[t] = 0;
                V.karg[t] = 0;
                V.acc[t] = kNone;
            }
            if (active) visit<VARIANT>(nodes, n_lights, e.x, e.y, E, Lc.flags, V);
            // Push the surviving children as one compacted run.
            unsigned bal[W];
            uint32_t n = 0;
#pragma unroll
            for (int t = 0; t < W; ++t) {
                bal[t] = __ballot_sync(0xFFFFFFFFu, V.go[t]);
                n += __popc(bal[t]);
            }
            if (n) {
                if (R + n > kRing) {  // move the oldest resident entries to the spill area
                    const uint32_t s = (R + n - kRing + 31u) & ~31u;
                    const uint32_t base = S - R;
                    if (base + s > Lc.spill_cap) {  // cannot happen: the area holds the bound
                        if (lane == 0) atomicOr(Lc.flags, HRR_FLAG_STACK);
                        break;
                    }
                    uint2 *spill = HRR_WARP_SPILL;
                    for (uint32_t k = lane; k < s; k += 32) spill[base + k] = ring[(base + k) & kRingMask];
                    R -= s;
                    __syncwarp();
                }
                // Lane by lane, each lane's survivors side by side: siblings (whose records
                // are neighbours in memory) are popped together by neighbouring lanes.
                uint32_t pos = S;
#pragma unroll
                for (int t = 0; t < W; ++t) pos += __popc(bal[t] & lt);
#pragma unroll
                for (int t = 0; t < W; ++t) {
                    if (V.go[t]) ring[pos & kRingMask] = make_uint2(V.node[t], V.karg[t]);
                    pos += V.go[t] ? 1u : 0u;
                }
                S += n;
                R += n;
                __syncwarp();
            }
            bool any_acc = false;
#pragma unroll
            for (int t = 0; t < W; ++t) any_acc |= V.acc[t] != kNone;
            if (__any_sync(0xFFFFFFFFu, any_acc)) emit<BATCH, W>(F, wbuf, wfr, cnt, lane, f, j, V.acc);
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
template <int VARIANT, int W, int RING, int THREADS, int TOP>
__global__ void __launch_bounds__(THREADS, min_blocks<W>(THREADS))
cull_single_kernel(const Launch Lc, const Frame fr) {
    traverse<VARIANT, false, W, RING, THREADS, TOP>(Lc, &fr);
}

template <int VARIANT, int W, int RING, int THREADS, int TOP>
__global__ void __launch_bounds__(THREADS, min_blocks<W>(THREADS))
cull_batch_kernel(const __grid_constant__ Launch Lc, const __grid_constant__ FrameArray<kMaxFrames> FA) {
    traverse<VARIANT, true, W, RING, THREADS, TOP>(Lc, FA.f);
}

}  // namespace
