// Light hierarchy builder: Morton keys, stable radix sort, binary radix tree, refit.
//
// Sec. 1 of the paper asks for light vertices sorted by a hierarchy in which every node
// is a contiguous range [a_n, b_n) of leaf indices, and notes that a spatial sort lets the
// sequence index inherit the radical inverse's stratification. This file builds such a
// hierarchy on the device:
//   1. morton_kernel     63-bit Morton keys (21 bits per axis) and finiteness checks;
//   2. radix_* kernels   stable LSD radix sort of (key, original index), 8 bits per pass;
//   3. gather_kernel     sorted (x, y, z, intensity) as float4;
//   4. topology_kernel   binary radix tree over (key, sorted position) in parallel: every
//                        internal node finds its range and split from its neighbours'
//                        common-prefix lengths (Karras, HPG 2012);
//   5. refit_kernel      bottom-up boxes / maximum intensities with one atomic counter per
//                        node (the second child to finish computes the parent), written
//                        straight into the parent's 64-byte record.
#include <algorithm>

#include "hrr_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // keys per sort block

// Spread the low 21 bits of v so that bit k moves to bit 3k.
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// floor(x * 2^21) clamped to [0, 2^21 - 1]; x * 2^21 is exact in float.
__device__ __forceinline__ uint32_t grid_cell(float x) {
    const float s = __fmul_rn(x, 2097152.0f);
    if (!(s >= 0.0f)) return 0u;
    const float f = floorf(s);
    return f >= 2097151.0f ? 2097151u : (uint32_t)f;
}

__global__ void __launch_bounds__(kThreads) morton_kernel(const float *__restrict__ x,
                                                          const float *__restrict__ y,
                                                          const float *__restrict__ z,
                                                          const float *__restrict__ inten,
                                                          uint32_t n, uint64_t *__restrict__ keys,
                                                          uint32_t *__restrict__ vals,
                                                          unsigned long long *flags) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const float px = x[i], py = y[i], pz = z[i], w = inten[i];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !isfinite(w))
        atomicOr(flags, HRR_FLAG_NONFINITE);
    keys[i] = (spread3(grid_cell(px)) << 2) | (spread3(grid_cell(py)) << 1) | spread3(grid_cell(pz));
    vals[i] = i;
}

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const uint64_t *__restrict__ keys,
                                                              uint32_t n, int shift,
                                                              uint32_t *__restrict__ hist,
                                                              uint32_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        const uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive prefix sums of each digit's row of the digit-major histogram
// hist[d * nblocks + b] (256 digits), in place, one warp per digit (8 consecutive counts per
// lane, a running carry over chunks of 256), and each digit's total in totals[d].
__global__ void __launch_bounds__(256) digit_scan_kernel(uint32_t *hist, uint32_t nblocks, uint32_t *totals) {
    const int lane = threadIdx.x & 31;
    const uint32_t d = blockIdx.x * 8u + (threadIdx.x >> 5);
    uint32_t *row = hist + (uint64_t)d * nblocks;
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nblocks; b0 += 256) {
        const uint32_t base = b0 + (uint32_t)lane * 8u;
        uint32_t v[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = base + k < nblocks ? row[base + k] : 0u;
            s += v[k];
        }
        uint32_t x = s;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = carry + x - s;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (base + k < nblocks) row[base + k] = run;
            run += v[k];
        }
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    if (lane == 0) totals[d] = carry;
}

// Stable scatter of one tile: items are taken in groups of 256 in tile order; an item's
// rank among equal digits is (earlier groups) + (earlier warps of its group) + (earlier
// lanes of its warp, from __match_any_sync); the digit's base comes first.
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, uint32_t n, int shift,
    const uint32_t *__restrict__ offsets, uint32_t nblocks, const uint32_t *__restrict__ totals) {
    static_assert(kThreads == 256, "one digit per thread");
    __shared__ uint32_t running[256];
    __shared__ uint32_t warp_cnt[kThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {  // the digit's base: exclusive prefix of the digit totals (a block scan)
        const uint32_t t = totals[threadIdx.x];
        uint32_t x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) running[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += running[w];
        __syncthreads();
        running[threadIdx.x] = offsets[(uint64_t)threadIdx.x * nblocks + blockIdx.x] + before + x - t;
    }
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) warp_cnt[w][threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int k = 0; k < kItems; ++k) {
        const uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
        const bool valid = i < n;
        const uint64_t key = valid ? keys_in[i] : 0ull;
        const uint32_t val = valid ? vals_in[i] : 0u;
        const uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += warp_cnt[w][d];
            const uint32_t pos = running[d] + before + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            tot += warp_cnt[w][threadIdx.x];
            warp_cnt[w][threadIdx.x] = 0;
        }
        running[threadIdx.x] += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) gather_kernel(const float *__restrict__ x,
                                                          const float *__restrict__ y,
                                                          const float *__restrict__ z,
                                                          const float *__restrict__ inten,
                                                          const uint32_t *__restrict__ perm,
                                                          uint32_t n, float4 *__restrict__ spos) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = perm[i];
    spos[i] = make_float4(x[v], y[v], z[v], inten[v]);
}

// Common-prefix length of the ordering keys (Morton key, sorted position) of leaves i, j;
// -1 outside [0, n).
__device__ __forceinline__ int prefix_len(const uint64_t *__restrict__ keys, int64_t n, int64_t i,
                                          int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t ki = keys[i], kj = keys[j];
    if (ki != kj) return __clzll((long long)(ki ^ kj));
    return 64 + __clz((uint32_t)(i ^ j));
}

__global__ void __launch_bounds__(kThreads) topology_kernel(const uint64_t *__restrict__ keys,
                                                            uint32_t n, hrr_node *__restrict__ nodes,
                                                            uint32_t *__restrict__ leaf_parent,
                                                            uint32_t *__restrict__ int_parent) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t N = n;
    if (i >= N - 1) return;
    const int d = (prefix_len(keys, N, i, i + 1) - prefix_len(keys, N, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = prefix_len(keys, N, i, i - d);
    int64_t lmax = 2;
    while (prefix_len(keys, N, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix_len(keys, N, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = prefix_len(keys, N, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (prefix_len(keys, N, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t first = i < j ? i : j, last = i < j ? j : i;
    nodes[i].split = (uint32_t)gamma;
    nodes[i].other_end = (uint32_t)j;
    const uint32_t code = (uint32_t)i << 1;
    if (first == gamma) leaf_parent[gamma] = code; else int_parent[gamma] = code;
    if (last == gamma + 1) leaf_parent[gamma + 1] = code | 1u; else int_parent[gamma + 1] = code | 1u;
}

__device__ __forceinline__ void store_slot(hrr_node *node, uint32_t slot, const float lo[3],
                                           const float hi[3], float imax) {
    float *f = reinterpret_cast<float *>(node) + (slot ? 8 : 0);
    f[0] = lo[0]; f[1] = lo[1]; f[2] = lo[2]; f[3] = imax;
    f[4] = hi[0]; f[5] = hi[1]; f[6] = hi[2];
}

__global__ void __launch_bounds__(kThreads) refit_kernel(const float4 *__restrict__ spos,
                                                         uint32_t n, hrr_node *nodes,
                                                         const uint32_t *__restrict__ leaf_parent,
                                                         const uint32_t *__restrict__ int_parent,
                                                         uint32_t *arrivals, uint32_t *child_height,
                                                         uint32_t *root_height,
                                                         unsigned long long *flags) {
    const uint32_t leaf = blockIdx.x * kThreads + threadIdx.x;
    if (leaf >= n || (*(volatile unsigned long long *)flags & HRR_FLAG_NONFINITE)) return;
    const float4 p = spos[leaf];
    float lo[3] = {p.x, p.y, p.z}, hi[3] = {p.x, p.y, p.z};
    float imax = p.w;
    uint32_t h = 0;
    uint32_t code = leaf_parent[leaf];
    for (;;) {
        const uint32_t node = code >> 1, slot = code & 1u;
        if (code == 0xFFFFFFFFu || node >= n - 1) {  // every link is set by topology_kernel
            atomicOr(flags, HRR_FLAG_TOPOLOGY);
            return;
        }
        store_slot(&nodes[node], slot, lo, hi, imax);
        child_height[2ull * node + slot] = h;
        __threadfence();
        if (atomicAdd(&arrivals[node], 1u) == 0u) return;  // the sibling finishes the node
        __threadfence();
        const float *f = reinterpret_cast<const float *>(&nodes[node]);
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(__ldcg(f + c), __ldcg(f + 8 + c));
            hi[c] = fmaxf(__ldcg(f + 4 + c), __ldcg(f + 12 + c));
        }
        imax = fmaxf(__ldcg(f + 3), __ldcg(f + 11));
        h = 1u + max(__ldcg(&child_height[2ull * node]), __ldcg(&child_height[2ull * node + 1]));
        if (node == 0) {
            *root_height = h;
            return;
        }
        code = int_parent[node];
    }
}

// Refit for moved lights: the leaves keep their order, so gather the new positions into
// that order (flagging non-finite values), rebuild the parent links from the records, and
// run refit_kernel again. The last two skip their work when the gather raised a flag, so
// the hierarchy is left as it was.
__global__ void __launch_bounds__(kThreads) gather_check_kernel(const float *__restrict__ x,
                                                                const float *__restrict__ y,
                                                                const float *__restrict__ z,
                                                                const float *__restrict__ inten,
                                                                const uint32_t *__restrict__ perm,
                                                                uint32_t n, float4 *__restrict__ spos,
                                                                unsigned long long *flags) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = perm[i];
    const float4 p = make_float4(x[v], y[v], z[v], inten[v]);
    if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z) || !isfinite(p.w)) atomicOr(flags, HRR_FLAG_NONFINITE);
    spos[i] = p;
}

__global__ void __launch_bounds__(kThreads) links_kernel(const hrr_node *__restrict__ nodes, uint32_t n,
                                                         uint32_t *__restrict__ leaf_parent,
                                                         uint32_t *__restrict__ int_parent,
                                                         unsigned long long *flags) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n - 1 || (*(volatile unsigned long long *)flags & HRR_FLAG_NONFINITE)) return;
    const uint32_t s = nodes[i].split, j = nodes[i].other_end;
    const uint32_t first = min(i, j), last = max(i, j);
    if (last >= n || s < first || s >= last) {
        atomicOr(flags, HRR_FLAG_TOPOLOGY);
        return;
    }
    const uint32_t code = i << 1;
    if (first == s) leaf_parent[s] = code; else int_parent[s] = code;
    if (last == s + 1) leaf_parent[s + 1] = code | 1u; else int_parent[s + 1] = code | 1u;
}

__global__ void single_leaf_kernel(const float *x, const float *y, const float *z,
                                   const float *inten, hrr_node *node, uint32_t *perm,
                                   unsigned long long *flags) {
    const float px = x[0], py = y[0], pz = z[0], w = inten[0];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !isfinite(w)) {
        atomicOr(flags, HRR_FLAG_NONFINITE);
        return;  // a build fails; a refit leaves the record as it was
    }
    const float lo[3] = {px, py, pz};
    store_slot(node, 0, lo, lo, w);
    store_slot(node, 1, lo, lo, w);
    node->split = 0;
    node->other_end = 0;
    perm[0] = 0;
}

// The top slots (HRR_TOP_SLOTS of them, layout in hrr_internal.cuh): thread s walks from the
// root along the path of heap slot s (the bits of s + 1 below its leading one, high to low:
// 0 = child 0, 1 = child 1), taking each child's box and maximum intensity from its parent's
// record. A slot below a leaf is empty; a record whose split is outside its node's range
// (not produced by the builder) empties the slots below it.
__global__ void __launch_bounds__(64) top_kernel(const float4 *__restrict__ nodes, uint32_t n,
                                                 float4 *__restrict__ top, const unsigned long long *flags) {
    const uint32_t s = threadIdx.x;
    if (s >= HRR_TOP_SLOTS) return;
    if (*(volatile const unsigned long long *)flags & HRR_FLAG_NONFINITE) return;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    uint32_t first = 0, last = 0, node = 0, kind = HRR_TOP_EMPTY;
    if (n > 1) {
        const uint32_t path = s + 1u;
        kind = HRR_TOP_INTERNAL;
        last = __float_as_uint(nodes[3].w);  // the root's range is [0, its other end]
        for (int b = 30 - __clz(path); b >= 0; --b) {
            if (kind != HRR_TOP_INTERNAL) {
                kind = HRR_TOP_EMPTY;
                break;
            }
            const float4 *r = nodes + 4 * (size_t)node;
            const uint32_t split = __float_as_uint(r[1].w);
            if (last >= n || split < first || split >= last) {
                kind = HRR_TOP_EMPTY;
                break;
            }
            if (((path >> b) & 1u) == 0u) {
                lo = r[0];
                hi = r[1];
                last = split;
                node = split;
            } else {
                lo = r[2];
                hi = r[3];
                first = split + 1u;
                node = split + 1u;
            }
            kind = first == last ? HRR_TOP_LEAF : HRR_TOP_INTERNAL;
        }
    }
    if (kind == HRR_TOP_EMPTY) {
        lo = hi = make_float4(0.f, 0.f, 0.f, 0.f);
        first = last = node = 0;
    }
    top[3 * s] = lo;
    top[3 * s + 1] = make_float4(hi.x, hi.y, hi.z, __uint_as_float(first));
    top[3 * s + 2] = make_float4(__uint_as_float(last), __uint_as_float(node), __uint_as_float(kind), 0.f);
}

// Records of width four. The record of internal node g holds, in this order, the slots of
// g's grandchildren over its leaf range [first, last] split at `split`:
//   slot 0: [first, s0]      slot 1: [s0 + 1, split]     (the children of child 0)
//   slot 2: [split + 1, s1]  slot 3: [s1 + 1, last]      (the children of child 1)
// each 32 bytes: box low corner, maximum intensity, box high corner, and one index word
// (s0, split, s1 and g's other range end, in slot order). A child that is a leaf takes its
// first slot as itself (s0 = split, or s1 = last) and leaves the second slot empty (an
// empty range). The internal slots are binary nodes s0, s0 + 1, s1, s1 + 1, whose own
// records sit at those indices. Since a node's record is the first 32 bytes of its
// children's binary records, re-labelled, the widening is a gather of the binary records.
__global__ void __launch_bounds__(kThreads) widen_kernel(const float4 *__restrict__ nodes, uint32_t n,
                                                         float4 *__restrict__ wide,
                                                         const unsigned long long *flags) {
    const uint32_t g = blockIdx.x * kThreads + threadIdx.x;
    if (*(volatile const unsigned long long *)flags & HRR_FLAG_NONFINITE) return;
    if (n == 1) {  // the single leaf in slot 0, the rest empty
        if (g == 0) {
            wide[0] = nodes[0];
            wide[1] = nodes[1];
            for (int k = 2; k < 8; ++k) wide[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    if (g >= n - 1) return;
    const float4 *r = nodes + 4 * (size_t)g;
    const float4 c0l = r[0], c0h = r[1], c1l = r[2], c1h = r[3];
    const uint32_t split = __float_as_uint(c0h.w), other = __float_as_uint(c1h.w);
    const uint32_t first = min(g, other), last = max(g, other);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 *w = wide + 8 * (size_t)g;
    if (first == split) {  // child 0 is a leaf: slot 0 is the leaf, slot 1 empty
        w[0] = c0l;
        w[1] = make_float4(c0h.x, c0h.y, c0h.z, __uint_as_float(split));
        w[2] = zero;
        w[3] = make_float4(0.f, 0.f, 0.f, __uint_as_float(split));
    } else {  // the children of internal node `split`
        const float4 *a = nodes + 4 * (size_t)split;
        w[0] = a[0];
        w[1] = a[1];  // its .w is the child's split, s0
        w[2] = a[2];
        const float4 h = a[3];
        w[3] = make_float4(h.x, h.y, h.z, __uint_as_float(split));
    }
    if (split + 1u == last) {  // child 1 is a leaf
        w[4] = c1l;
        w[5] = make_float4(c1h.x, c1h.y, c1h.z, __uint_as_float(last));
        w[6] = zero;
        w[7] = make_float4(0.f, 0.f, 0.f, __uint_as_float(other));
    } else {  // the children of internal node split + 1
        const float4 *b = nodes + 4 * (size_t)(split + 1u);
        w[4] = b[0];
        w[5] = b[1];  // s1
        w[6] = b[2];
        const float4 h = b[3];
        w[7] = make_float4(h.x, h.y, h.z, __uint_as_float(other));
    }
}

template <typename T>
T *carve(char *&p, size_t count) {
    T *r = reinterpret_cast<T *>(p);
    p += (sizeof(T) * count + 255) & ~size_t(255);
    return r;
}

// ------------------------------------------------------------------------------------
// Cost-driven topology over the Morton order
// ------------------------------------------------------------------------------------
//
// A top-down build, one level per pass: every range [f, l] of the level splits at the k
// (children [f, k], [k+1, l]) that minimises C(k) = w(L) + w(R) over every k in [f, l),
//     w(X) = u^2 ((A + 0.1 P) + 1e-4) c sqrt(c),
// with c the child's light count, u its maximum intensity (clamped at 0) times the
// reciprocal of the range's, A = dx dy + dy dz + dz dx and P = dx + dy + dz of its box; in
// float with every operation rounded separately (no contraction; sqrt and the reciprocal
// correctly rounded). A non-finite C never wins; ties go to the least |c_L - c_R|, then
// the least k. Ranges deeper than the cost depth (root = 1)
// take the radix split, which bounds the height. Node numbering and parent links are those
// of topology_kernel, so refit_kernel finishes the hierarchy unchanged.
//
// Boxes and maxima are min / max reductions, exact in any order, so parallel scans give
// the same prefix and suffix aggregates at every k as a serial sweep, and the same costs
// bit for bit. A range of up to 32 lights: one warp builds its whole subtree, a light per
// lane; up to 256: one warp, a run of 8 lights per lane; larger ones: tiles of 1024
// lights, one block per tile and a run of 4 lights per thread. tile_agg_kernel reduces each tile, and the last tile of a
// range to finish scans the range's tile aggregates; tile_cost_kernel evaluates every
// split in its tile, and the last tile of a range to finish picks the range's split.

constexpr int kSplitThreads = 256;  // block size of every split kernel
constexpr int kTileRun = 4;         // lights per thread in a tile
constexpr uint32_t kSegTile = kSplitThreads * kTileRun;
constexpr int kMidRun = 8;          // lights per lane for ranges of 33..256 lights
constexpr uint32_t kSmallMax = 32, kMidMax = 32 * kMidRun;
constexpr uint32_t kNoSplit = 0xFFFFFFFFu;

struct Seg {
    uint32_t node, f, l, depth;
};

struct Agg {  // box and maximum intensity of a set of lights
    float lo[3], hi[3], m;
};

struct __align__(16) AggRec {  // (lo xyz, m), (hi xyz, 0)
    float4 a, b;
};

struct Best {  // a candidate split, ordered by (c, d, k)
    float c;
    uint32_t d, k;
};

// The next level's range lists, filled by commit_split. Small ranges fill their list from
// the front, ranges below the cost depth from the back (radix_end[-1], radix_end[-2], ...):
// the ranges of a level are disjoint, so together they number at most n / 2.
struct SplitOut {
    hrr_node *nodes;
    uint32_t *leaf_parent, *int_parent;
    uint32_t cost_depth;
    Seg *small, *radix_end, *mid, *big;
    uint32_t *big_t0;                // first tile of each big range (increasing)
    uint32_t *counts;                // [0] small, [1] mid, [2] radix
    unsigned long long *big_count;   // (big ranges << 32) | tiles
};

__device__ __forceinline__ Agg agg_empty() {
    Agg a;
    for (int c = 0; c < 3; ++c) {
        a.lo[c] = __int_as_float(0x7f800000);
        a.hi[c] = -__int_as_float(0x7f800000);
    }
    a.m = -__int_as_float(0x7f800000);
    return a;
}
__device__ __forceinline__ Agg agg_of(float4 p) {
    Agg a;
    a.lo[0] = a.hi[0] = p.x;
    a.lo[1] = a.hi[1] = p.y;
    a.lo[2] = a.hi[2] = p.z;
    a.m = p.w;
    return a;
}
__device__ __forceinline__ Agg agg_join(const Agg &a, const Agg &b) {
    Agg r;
    for (int c = 0; c < 3; ++c) {
        r.lo[c] = fminf(a.lo[c], b.lo[c]);
        r.hi[c] = fmaxf(a.hi[c], b.hi[c]);
    }
    r.m = fmaxf(a.m, b.m);
    return r;
}
__device__ __forceinline__ Agg agg_shfl(const Agg &a, int delta, bool up) {
    Agg r;
    for (int c = 0; c < 3; ++c) {
        r.lo[c] = up ? __shfl_up_sync(0xFFFFFFFFu, a.lo[c], delta) : __shfl_down_sync(0xFFFFFFFFu, a.lo[c], delta);
        r.hi[c] = up ? __shfl_up_sync(0xFFFFFFFFu, a.hi[c], delta) : __shfl_down_sync(0xFFFFFFFFu, a.hi[c], delta);
    }
    r.m = up ? __shfl_up_sync(0xFFFFFFFFu, a.m, delta) : __shfl_down_sync(0xFFFFFFFFu, a.m, delta);
    return r;
}
__device__ __forceinline__ AggRec agg_pack(const Agg &a) {
    return {make_float4(a.lo[0], a.lo[1], a.lo[2], a.m), make_float4(a.hi[0], a.hi[1], a.hi[2], 0.f)};
}
__device__ __forceinline__ Agg agg_unpack(float4 x, float4 y) {
    Agg a;
    a.lo[0] = x.x; a.lo[1] = x.y; a.lo[2] = x.z; a.m = x.w;
    a.hi[0] = y.x; a.hi[1] = y.y; a.hi[2] = y.z;
    return a;
}
// Written by other blocks of the running kernel: read past L1.
__device__ __forceinline__ Agg agg_load_cg(const AggRec *r) { return agg_unpack(__ldcg(&r->a), __ldcg(&r->b)); }

// w(X) of a child of c lights, given the reciprocal of the range's maximum intensity
__device__ __forceinline__ float child_cost(const Agg &x, float inv, uint32_t c) {
    const float u = __fmul_rn(fmaxf(x.m, 0.f), inv);
    const float dx = __fsub_rn(x.hi[0], x.lo[0]), dy = __fsub_rn(x.hi[1], x.lo[1]), dz = __fsub_rn(x.hi[2], x.lo[2]);
    const float a = __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
    const float p = __fadd_rn(__fadd_rn(dx, dy), dz);
    const float g = __fadd_rn(__fadd_rn(a, __fmul_rn(0.1f, p)), 1e-4f);
    const float cf = __uint2float_rn(c);
    return __fmul_rn(__fmul_rn(__fmul_rn(u, u), g), __fmul_rn(cf, __fsqrt_rn(cf)));
}

// Reciprocal of a range's maximum intensity m: 0 for a dark range, and a maximum below the
// smallest normal float counts as that float.
__device__ __forceinline__ float range_inv(float m) {
    const float mx = fmaxf(m, 0.f);
    return mx > 0.f ? __fdiv_rn(1.f, fmaxf(mx, __int_as_float(0x00800000))) : 0.f;
}

// C(k) for children of cl and cr lights, given range_inv of the range's maximum (the larger
// of the children's)
__device__ __forceinline__ float split_cost(const Agg &L, const Agg &R, uint32_t cl, uint32_t cr, float inv) {
    return __fadd_rn(child_cost(L, inv, cl), child_cost(R, inv, cr));
}

__device__ __forceinline__ Best best_none() { return {__int_as_float(0x7f800000), kNoSplit, kNoSplit}; }
// o < b in (cost, |c_L - c_R|, k) order; a NaN cost never wins
__device__ __forceinline__ void best_take(Best &b, const Best &o) {
    if (o.c < b.c || (o.c == b.c && (o.d < b.d || (o.d == b.d && o.k < b.k)))) b = o;
}
__device__ __forceinline__ Best warp_best(Best b) {  // the warp's best, in lane 0
    for (int d = 16; d > 0; d >>= 1) {
        const Best o = {__shfl_down_sync(0xFFFFFFFFu, b.c, d), __shfl_down_sync(0xFFFFFFFFu, b.d, d),
                        __shfl_down_sync(0xFFFFFFFFu, b.k, d)};
        best_take(b, o);
    }
    return b;
}
// The block's best, in thread 0; sh holds one entry per warp.
__device__ __forceinline__ Best block_best(Best b, Best *sh) {
    b = warp_best(b);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kSplitThreads / 32; ++w) best_take(b, sh[w]);
    __syncthreads();
    return b;
}

// Exclusive scans over the lanes of a warp: the aggregates of lanes [0, lane) and (lane, 31].
__device__ __forceinline__ void warp_scans(const Agg &x, Agg &before, Agg &after) {
    const int lane = threadIdx.x & 31;
    Agg pre = x, suf = x;
    for (int d = 1; d < 32; d <<= 1) {
        const Agg u = agg_shfl(pre, d, true), v = agg_shfl(suf, d, false);
        if (lane >= d) pre = agg_join(pre, u);
        if (lane + d < 32) suf = agg_join(suf, v);
    }
    before = agg_shfl(pre, 1, true);
    after = agg_shfl(suf, 1, false);
    if (lane == 0) before = agg_empty();
    if (lane == 31) after = agg_empty();
}

// Exclusive scans over the threads of a block, and the block's total; sh holds one entry
// per warp.
__device__ __forceinline__ void block_scans(const Agg &x, Agg &before, Agg &after, Agg &total, Agg *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Agg wb, wa;
    warp_scans(x, wb, wa);
    if (lane == 31) sh[w] = agg_join(wb, x);
    __syncthreads();
    Agg bb = agg_empty(), ba = agg_empty();
    total = agg_empty();
    for (int v = 0; v < kSplitThreads / 32; ++v) {
        const Agg s = sh[v];
        if (v < w) bb = agg_join(bb, s);
        if (v > w) ba = agg_join(ba, s);
        total = agg_join(total, s);
    }
    before = agg_join(bb, wb);
    after = agg_join(wa, ba);
    __syncthreads();
}

// The lights [a, min(a + R, end)) of a thread's run; returns their count.
template <int R>
__device__ __forceinline__ uint32_t load_run(const float4 *__restrict__ spos, uint32_t a, uint32_t end, float4 (&p)[R]) {
    const uint32_t cnt = a < end ? min((uint32_t)R, end - a) : 0u;
#pragma unroll
    for (int i = 0; i < R; ++i) p[i] = (uint32_t)i < cnt ? spos[a + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    return cnt;
}
template <int R>
__device__ __forceinline__ Agg run_agg(const float4 (&p)[R], uint32_t cnt) {
    Agg x = agg_empty();
#pragma unroll
    for (int i = 0; i < R; ++i)
        if ((uint32_t)i < cnt) x = agg_join(x, agg_of(p[i]));
    return x;
}
// Every split k = a + i (k < l) of a run, given the aggregates of [f, a) and of the lights
// of [f, l] after the run.
template <int R>
__device__ __forceinline__ void run_best(const float4 (&p)[R], uint32_t cnt, uint32_t a, const Agg &before,
                                         const Agg &after, uint32_t f, uint32_t l, Best &b) {
    Agg suf[R + 1];  // suf[i]: lights a + i .. of the run, then the rest of the range
    suf[R] = after;
#pragma unroll
    for (int i = R - 1; i >= 0; --i) suf[i] = (uint32_t)i < cnt ? agg_join(agg_of(p[i]), suf[i + 1]) : suf[i + 1];
    const float inv = range_inv(fmaxf(before.m, suf[0].m));  // the same for every split of the range
    Agg pre = before;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        if ((uint32_t)i < cnt) {
            pre = agg_join(pre, agg_of(p[i]));
            const uint32_t k = a + i;
            if (k < l) {
                const uint32_t cl = k - f + 1, cr = l - k;
                best_take(b, {split_cost(pre, suf[i + 1], cl, cr, inv), cl > cr ? cl - cr : cr - cl, k});
            }
        }
    }
}

// Radix split of [f, l]: the last k whose ordering key (Morton key, position) has a 0 at
// the highest bit where the keys of f and l differ (binary search; the digit is sorted).
__device__ uint32_t radix_split(const uint64_t *__restrict__ keys, uint32_t f, uint32_t l) {
    const uint64_t kf = keys[f], kl = keys[l];
    uint32_t lo = f, hi = l;  // digit(lo) = 0, digit(hi) = 1
    if (kf != kl) {
        const int bit = 63 - __clzll((long long)(kf ^ kl));
        while (hi - lo > 1) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if ((keys[mid] >> bit) & 1ull) hi = mid; else lo = mid;
        }
    } else {
        const int bit = 31 - __clz(f ^ l);
        while (hi - lo > 1) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if ((mid >> bit) & 1u) hi = mid; else lo = mid;
        }
    }
    return lo;
}

// Record the split s of range g: the node's record and its children's parent links.
__device__ __forceinline__ void record_split(const Seg &g, uint32_t s, const SplitOut &o) {
    o.nodes[g.node].split = s;
    o.nodes[g.node].other_end = g.node == g.f ? g.l : g.f;
    const uint32_t code = g.node << 1;
    if (s == g.f) o.leaf_parent[s] = code; else o.int_parent[s] = code;
    if (s + 1 == g.l) o.leaf_parent[s + 1] = code | 1u; else o.int_parent[s + 1] = code | 1u;
}

// Record the split of range g and queue its internal children for the next level.
__device__ void commit_split(const Seg &g, uint32_t s, const SplitOut &o) {
    if (s == kNoSplit) s = g.f;  // no finite cost: non-finite lights, which fail the build
    record_split(g, s, o);
    const Seg kids[2] = {{s, g.f, s, g.depth + 1}, {s + 1, s + 1, g.l, g.depth + 1}};
    for (int c = 0; c < 2; ++c) {
        const Seg &k = kids[c];
        if (k.f == k.l) continue;
        const uint32_t m = k.l - k.f + 1;
        if (k.depth > o.cost_depth) {
            o.radix_end[-1 - (int64_t)atomicAdd(&o.counts[2], 1u)] = k;
        } else if (m <= kSmallMax) {
            o.small[atomicAdd(&o.counts[0], 1u)] = k;
        } else if (m <= kMidMax) {
            o.mid[atomicAdd(&o.counts[1], 1u)] = k;
        } else {
            const unsigned long long old = atomicAdd(o.big_count, (1ull << 32) | ((m + kSegTile - 1) / kSegTile));
            const uint32_t i = (uint32_t)(old >> 32);
            o.big[i] = k;
            o.big_t0[i] = (uint32_t)old;
        }
    }
}

// Ranges below the cost depth: one thread each.
__global__ void __launch_bounds__(kSplitThreads) split_radix_kernel(const Seg *__restrict__ segs, uint32_t n_segs,
                                                                    const uint64_t *__restrict__ keys, SplitOut o) {
    const uint32_t i = blockIdx.x * kSplitThreads + threadIdx.x;
    if (i >= n_segs) return;
    const Seg g = segs[i];
    commit_split(g, radix_split(keys, g.f, g.l), o);
}

// Ranges of up to 32 lights: one warp builds the whole subtree, one level of it per
// iteration. Lane j holds light f0 + j and the range of the level that holds it; scans and
// the reduction to the range's first lane are segmented by those ranges.
__global__ void __launch_bounds__(kSplitThreads) subtree_warp_kernel(const Seg *__restrict__ segs, uint32_t n_segs,
                                                                     const float4 *__restrict__ spos,
                                                                     const uint64_t *__restrict__ keys, SplitOut o) {
    const uint32_t w = (blockIdx.x * kSplitThreads + threadIdx.x) >> 5;
    if (w >= n_segs) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const Seg g0 = segs[w];
    const uint32_t i = g0.f + (uint32_t)lane;
    const bool valid = i <= g0.l;
    const Agg self = valid ? agg_of(spos[i]) : agg_empty();
    Seg g = valid ? g0 : Seg{i, i, i, 0u};  // lanes past the range: a closed range of their own
    // a range of at most 32 lights is at most 31 levels deep
    for (int level = 0; level < 32 && __any_sync(0xFFFFFFFFu, g.l > g.f); ++level) {
        const int lf = (int)(g.f - g0.f), ll = (int)(g.l - g0.f);  // this lane's range, as lanes
        Agg pre = self, suf = self;  // inclusive scans within the range
        for (int d = 1; d < 32; d <<= 1) {
            const Agg u = agg_shfl(pre, d, true), v = agg_shfl(suf, d, false);
            if (lane - d >= lf) pre = agg_join(pre, u);
            if (lane + d <= ll) suf = agg_join(suf, v);
        }
        const Agg right = agg_shfl(suf, 1, false);  // [i + 1, l] for i < l
        Best b = best_none();
        if (lane < ll) {
            const uint32_t cl = i - g.f + 1, cr = g.l - i;
            b = {split_cost(pre, right, cl, cr, range_inv(fmaxf(pre.m, right.m))), cl > cr ? cl - cr : cr - cl, i};
        }
        for (int d = 1; d < 32; d <<= 1) {  // the range's best split, in its first lane
            const Best ob = {__shfl_down_sync(0xFFFFFFFFu, b.c, d), __shfl_down_sync(0xFFFFFFFFu, b.d, d),
                             __shfl_down_sync(0xFFFFFFFFu, b.k, d)};
            if (lane + d <= ll) best_take(b, ob);
        }
        uint32_t s = 0;
        if (lane == lf && ll > lf) {
            s = g.depth <= o.cost_depth ? (b.k == kNoSplit ? g.f : b.k) : radix_split(keys, g.f, g.l);
            record_split(g, s, o);
        }
        s = __shfl_sync(0xFFFFFFFFu, s, lf);
        if (ll > lf) g = i <= s ? Seg{s, g.f, s, g.depth + 1} : Seg{s + 1, s + 1, g.l, g.depth + 1};
    }
}

// Ranges of up to 32 R lights: one warp each, a run of R lights per lane.
template <int R>
__global__ void __launch_bounds__(kSplitThreads) split_warp_kernel(const Seg *__restrict__ segs, uint32_t n_segs,
                                                                   const float4 *__restrict__ spos, SplitOut o) {
    const uint32_t w = (blockIdx.x * kSplitThreads + threadIdx.x) >> 5;
    if (w >= n_segs) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const Seg g = segs[w];
    const uint32_t a = g.f + (uint32_t)lane * R;
    float4 p[R];
    const uint32_t cnt = load_run<R>(spos, a, g.l + 1, p);
    Agg before, after;
    warp_scans(run_agg<R>(p, cnt), before, after);
    Best b = best_none();
    run_best<R>(p, cnt, a, before, after, g.f, g.l, b);
    b = warp_best(b);
    if (lane == 0) commit_split(g, b.k, o);
}

// The big range holding tile t: the last i with big_t0[i] <= t.
__device__ __forceinline__ uint32_t range_of_tile(const uint32_t *__restrict__ big_t0, uint32_t n_big, uint32_t t) {
    uint32_t lo = 0, hi = n_big;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (big_t0[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

struct TileSite {  // a tile of a big range
    Seg g;
    uint32_t i, t0, nt, start, end;  // range index, first tile, tiles, lights [start, end)
};

__device__ __forceinline__ TileSite tile_site(const Seg *__restrict__ big, const uint32_t *__restrict__ big_t0,
                                              uint32_t n_big, uint32_t *s_i) {
    if (threadIdx.x == 0) *s_i = range_of_tile(big_t0, n_big, blockIdx.x);
    __syncthreads();
    TileSite s;
    s.i = *s_i;
    s.g = big[s.i];
    s.t0 = big_t0[s.i];
    s.nt = (s.g.l - s.g.f + 1 + kSegTile - 1) / kSegTile;
    s.start = s.g.f + (blockIdx.x - s.t0) * kSegTile;
    s.end = s.g.l + 1 - s.start > kSegTile ? s.start + kSegTile : s.g.l + 1;
    return s;
}

// Tile aggregates of ranges of more than one tile; the last tile of a range to finish
// writes, for every tile, the aggregates of the range's tiles before it and after it.
__global__ void __launch_bounds__(kSplitThreads) tile_agg_kernel(
    const Seg *__restrict__ big, const uint32_t *__restrict__ big_t0, uint32_t n_big, const float4 *__restrict__ spos,
    AggRec *tile_agg, AggRec *tile_pre, AggRec *tile_suf, uint32_t *done) {
    __shared__ Agg sh[kSplitThreads / 32];
    __shared__ uint32_t s_i;
    __shared__ int s_last;
    const TileSite s = tile_site(big, big_t0, n_big, &s_i);
    if (s.nt == 1) return;  // block-uniform
    float4 p[kTileRun];
    const uint32_t cnt = load_run<kTileRun>(spos, s.start + threadIdx.x * kTileRun, s.end, p);
    Agg before, after, total;
    block_scans(run_agg<kTileRun>(p, cnt), before, after, total, sh);
    if (threadIdx.x == 0) {
        tile_agg[blockIdx.x] = agg_pack(total);
        __threadfence();
        s_last = atomicAdd(&done[s.i], 1u) == s.nt - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    Agg carry = agg_empty();
    for (uint32_t base = 0; base < s.nt; base += kSplitThreads) {  // tiles before
        const uint32_t j = base + threadIdx.x;
        const Agg y = j < s.nt ? agg_load_cg(&tile_agg[s.t0 + j]) : agg_empty();
        block_scans(y, before, after, total, sh);
        if (j < s.nt) tile_pre[s.t0 + j] = agg_pack(agg_join(carry, before));
        carry = agg_join(carry, total);
    }
    carry = agg_empty();
    for (uint32_t base = (s.nt - 1) / kSplitThreads * kSplitThreads;; base -= kSplitThreads) {  // tiles after
        const uint32_t j = base + threadIdx.x;
        const Agg y = j < s.nt ? agg_load_cg(&tile_agg[s.t0 + j]) : agg_empty();
        block_scans(y, before, after, total, sh);
        if (j < s.nt) tile_suf[s.t0 + j] = agg_pack(agg_join(after, carry));
        carry = agg_join(carry, total);
        if (base == 0) break;
    }
    if (threadIdx.x == 0) done[s.i] = 0;
}

// Every split in a tile of a big range; a range of one tile records its split here, else
// the last tile of the range to finish reduces the tiles' best splits and records it.
__global__ void __launch_bounds__(kSplitThreads) tile_cost_kernel(
    const Seg *__restrict__ big, const uint32_t *__restrict__ big_t0, uint32_t n_big, const float4 *__restrict__ spos,
    const AggRec *__restrict__ tile_pre, const AggRec *__restrict__ tile_suf, Best *tile_best, uint32_t *done,
    SplitOut o) {
    __shared__ Agg sh[kSplitThreads / 32];
    __shared__ Best shb[kSplitThreads / 32];
    __shared__ uint32_t s_i;
    __shared__ int s_last;
    const TileSite s = tile_site(big, big_t0, n_big, &s_i);
    const uint32_t a = s.start + threadIdx.x * kTileRun;
    float4 p[kTileRun];
    const uint32_t cnt = load_run<kTileRun>(spos, a, s.end, p);
    Agg before, after, total;
    block_scans(run_agg<kTileRun>(p, cnt), before, after, total, sh);
    if (s.nt > 1) {
        const AggRec pre = tile_pre[blockIdx.x], suf = tile_suf[blockIdx.x];
        before = agg_join(agg_unpack(pre.a, pre.b), before);
        after = agg_join(after, agg_unpack(suf.a, suf.b));
    }
    Best b = best_none();
    run_best<kTileRun>(p, cnt, a, before, after, s.g.f, s.g.l, b);
    b = block_best(b, shb);
    if (s.nt == 1) {  // block-uniform
        if (threadIdx.x == 0) commit_split(s.g, b.k, o);
        return;
    }
    if (threadIdx.x == 0) {
        tile_best[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(&done[s.i], 1u) == s.nt - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    Best r = best_none();
    for (uint32_t j = threadIdx.x; j < s.nt; j += kSplitThreads) {
        const Best *q = &tile_best[s.t0 + j];
        best_take(r, {__ldcg(&q->c), __ldcg(&q->d), __ldcg(&q->k)});
    }
    r = block_best(r, shb);
    if (threadIdx.x == 0) {
        done[s.i] = 0;
        commit_split(s.g, r.k, o);
    }
}

}  // namespace

namespace {

// The cost-driven topology for n >= 2 sorted lights: writes split / other_end of every
// record and the parent links, level by level (one host round trip per level).
int cost_topology(hrr_ctx *ctx, const float4 *spos, const uint64_t *keys, uint32_t n, uint32_t cost_depth,
                  hrr_node *nodes, uint32_t *leaf_parent, uint32_t *int_parent, cudaStream_t st) {
    const size_t cap_s = (size_t)n / 2 + 1;                    // ranges of >= 2 lights in a level
    const size_t cap_m = (size_t)n / (kSmallMax + 1) + 1;      // ... of > 32
    const size_t cap_b = (size_t)n / (kMidMax + 1) + 1;        // ... of > 256
    const size_t cap_t = (size_t)n / kSegTile + cap_b + 1;     // tiles of those
    auto rup = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t bytes = 2 * (rup(sizeof(Seg) * cap_s) + rup(sizeof(Seg) * cap_m) + rup(sizeof(Seg) * cap_b) +
                              rup(sizeof(uint32_t) * cap_b)) +
                         3 * rup(sizeof(AggRec) * cap_t) + rup(sizeof(Best) * cap_t) + rup(sizeof(uint32_t) * cap_b) +
                         256;
    char *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, st);
    if (e != cudaSuccess) return hrr_cuda_fail(ctx, e, "topology scratch");
    struct Lists {
        Seg *small, *radix_end, *mid, *big;
        uint32_t *big_t0;
    } in, out;
    char *p = scratch;
    for (Lists *L : {&in, &out}) {
        L->small = carve<Seg>(p, cap_s);
        L->radix_end = L->small + cap_s;
        L->mid = carve<Seg>(p, cap_m);
        L->big = carve<Seg>(p, cap_b);
        L->big_t0 = carve<uint32_t>(p, cap_b);
    }
    AggRec *tile_agg = carve<AggRec>(p, cap_t), *tile_pre = carve<AggRec>(p, cap_t), *tile_suf = carve<AggRec>(p, cap_t);
    Best *tile_best = carve<Best>(p, cap_t);
    uint32_t *done = carve<uint32_t>(p, cap_b);
    uint32_t *counts = carve<uint32_t>(p, 6);  // small, mid, radix, pad, big (64-bit)
    unsigned long long *big_count = reinterpret_cast<unsigned long long *>(counts + 4);

    const Seg root{0u, 0u, n - 1, 1u};
    uint32_t ns = 0, nm = 0, nr = 0, nb = 0, ntiles = 0;
    Seg *root_list;
    if (n <= kSmallMax) { ns = 1; root_list = in.small; }
    else if (n <= kMidMax) { nm = 1; root_list = in.mid; }
    else { nb = 1; ntiles = (uint32_t)(((size_t)n + kSegTile - 1) / kSegTile); root_list = in.big; }
    e = cudaMemcpyAsync(root_list, &root, sizeof(Seg), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(in.big_t0, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(done, 0, sizeof(uint32_t) * cap_b, st);
    uint32_t *host = reinterpret_cast<uint32_t *>(&ctx->host_counters[5]);  // 6 words of pinned memory
    int rc = HRR_OK;
    for (int level = 0; e == cudaSuccess && ns + nm + nr + nb > 0; ++level) {
        if (level > (int)cost_depth + 100) {  // the radix split bounds the height
            rc = hrr_fail(ctx, HRR_ERR_DEVICE, "topology build did not terminate");
            break;
        }
        if ((e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 6, st)) != cudaSuccess) break;
        const SplitOut o{nodes, leaf_parent, int_parent, cost_depth, out.small, out.radix_end, out.mid, out.big,
                         out.big_t0, counts, big_count};
        if (nr) {
            split_radix_kernel<<<(nr + kSplitThreads - 1) / kSplitThreads, kSplitThreads, 0, st>>>(in.radix_end - nr,
                                                                                               nr, keys, o);
            ++ctx->launches;
        }
        if (ns) {
            subtree_warp_kernel<<<(unsigned)(((size_t)ns * 32 + kSplitThreads - 1) / kSplitThreads), kSplitThreads, 0,
                                  st>>>(in.small, ns, spos, keys, o);
            ++ctx->launches;
        }
        if (nm) {
            split_warp_kernel<kMidRun><<<(unsigned)(((size_t)nm * 32 + kSplitThreads - 1) / kSplitThreads), kSplitThreads,
                                         0, st>>>(in.mid, nm, spos, o);
            ++ctx->launches;
        }
        if (nb) {
            if (ntiles > nb) {  // some range spans several tiles
                tile_agg_kernel<<<ntiles, kSplitThreads, 0, st>>>(in.big, in.big_t0, nb, spos, tile_agg, tile_pre,
                                                                  tile_suf, done);
                ++ctx->launches;
            }
            tile_cost_kernel<<<ntiles, kSplitThreads, 0, st>>>(in.big, in.big_t0, nb, spos, tile_pre, tile_suf,
                                                               tile_best, done, o);
            ++ctx->launches;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(host, counts, sizeof(uint32_t) * 6, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        ns = host[0];
        nm = host[1];
        nr = host[2];
        const unsigned long long bc = (unsigned long long)host[4] | ((unsigned long long)host[5] << 32);
        nb = (uint32_t)(bc >> 32);
        ntiles = (uint32_t)bc;
        std::swap(in, out);
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return hrr_cuda_fail(ctx, e, "topology build");
    return rc;
}

}  // namespace

int hrr_build_impl(hrr_ctx *ctx, const hrr_lights &L, uint32_t n, hrr_tree **out, int topology, uint32_t cost_depth) {
    cudaStream_t st = ctx->stream;
    hrr_tree *tree = new (std::nothrow) hrr_tree();
    if (!tree) return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the tree");
    tree->device = ctx->device;
    tree->n = n;
    auto fail = [&](int status) {
        if (tree->nodes) cudaFreeAsync(tree->nodes, st);
        if (tree->perm) cudaFreeAsync(tree->perm, st);
        if (tree->wide) cudaFreeAsync(tree->wide, st);
        delete tree;
        return status;
    };
    const uint32_t n_rec = n > 1 ? n - 1 : 1;
    cudaError_t e = cudaMallocAsync(&tree->nodes, sizeof(hrr_node) * (size_t)n_rec + HRR_TOP_BYTES, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&tree->perm, sizeof(uint32_t) * (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&tree->wide, 8 * sizeof(float4) * (size_t)n_rec, st);
    if (e != cudaSuccess) return fail(hrr_cuda_fail(ctx, e, "tree allocation"));
    unsigned long long *flags = ctx->counters + 2;
    if ((e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long), st)) != cudaSuccess)
        return fail(hrr_cuda_fail(ctx, e, "flag reset"));

    if (n == 1) {
        single_leaf_kernel<<<1, 1, 0, st>>>(L.x, L.y, L.z, L.intensity, tree->nodes, tree->perm, flags);
        ++ctx->launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(hrr_cuda_fail(ctx, e, "single_leaf_kernel"));
        tree->height = 0;
    } else {
        const uint32_t nblocks = (n + kTile - 1) / kTile;
        const uint64_t hist_n = 256ull * (nblocks + 1);  // digit-major counts, then the digit totals
        const size_t bytes = 2 * ((sizeof(uint64_t) * (size_t)n + 255) & ~size_t(255)) +
                             ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)) +
                             ((sizeof(uint32_t) * hist_n + 255) & ~size_t(255)) +
                             ((sizeof(float4) * (size_t)n + 255) & ~size_t(255)) +
                             2 * ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)) +
                             ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)) +
                             ((sizeof(uint32_t) * 2 * (size_t)n + 255) & ~size_t(255)) + 256 + 1024;
        char *scratch = nullptr;
        if ((e = cudaMallocAsync(&scratch, bytes, st)) != cudaSuccess) return fail(hrr_cuda_fail(ctx, e, "build scratch"));
        char *p = scratch;
        uint64_t *keys0 = carve<uint64_t>(p, n), *keys1 = carve<uint64_t>(p, n);
        uint32_t *vals1 = carve<uint32_t>(p, n);
        uint32_t *hist = carve<uint32_t>(p, hist_n);
        float4 *spos = carve<float4>(p, n);
        uint32_t *leaf_parent = carve<uint32_t>(p, n), *int_parent = carve<uint32_t>(p, n);
        uint32_t *arrivals = carve<uint32_t>(p, n);
        uint32_t *child_height = carve<uint32_t>(p, 2 * (size_t)n);
        uint32_t *root_height = carve<uint32_t>(p, 1);
        uint32_t *vals0 = tree->perm;

        const unsigned g = (n + kThreads - 1) / kThreads;
        int rc = HRR_OK;
        do {
            morton_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, n, keys0, vals0, flags);
            ++ctx->launches;
            uint64_t *kin = keys0, *kout = keys1;
            uint32_t *vin = vals0, *vout = vals1;
            for (int shift = 0; shift < 64; shift += 8) {
                radix_hist_kernel<<<nblocks, kThreads, 0, st>>>(kin, n, shift, hist, nblocks);
                digit_scan_kernel<<<32, 256, 0, st>>>(hist, nblocks, hist + 256 * (size_t)nblocks);
                radix_scatter_kernel<<<nblocks, kThreads, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblocks,
                                                                     hist + 256 * (size_t)nblocks);
                ctx->launches += 3;
                uint64_t *tk = kin; kin = kout; kout = tk;
                uint32_t *tv = vin; vin = vout; vout = tv;
            }
            // eight passes: the sorted keys are back in keys0 and the permutation in vals0
            gather_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, vals0, n, spos);
            if ((e = cudaMemsetAsync(arrivals, 0, sizeof(uint32_t) * (size_t)n, st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "memset"); break; }
            if ((e = cudaMemsetAsync(leaf_parent, 0xFF, 2 * ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)), st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "memset"); break; }
            const unsigned gi = (n - 1 + kThreads - 1) / kThreads;
            if (topology == HRR_TOPOLOGY_COST) {
                if ((rc = cost_topology(ctx, spos, keys0, n, cost_depth, tree->nodes, leaf_parent, int_parent, st)) != HRR_OK) break;
            } else {
                topology_kernel<<<gi, kThreads, 0, st>>>(keys0, n, tree->nodes, leaf_parent, int_parent);
                ++ctx->launches;
            }
            refit_kernel<<<g, kThreads, 0, st>>>(spos, n, tree->nodes, leaf_parent, int_parent, arrivals,
                                                 child_height, root_height, flags);
            ctx->launches += 2;
            if ((e = cudaGetLastError()) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "build kernels"); break; }
            if ((e = cudaMemcpyAsync(&ctx->host_counters[4], root_height, sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "height copy"); break; }
        } while (0);
        cudaFreeAsync(scratch, st);
        if (rc != HRR_OK) return fail(rc);
    }
    if ((e = hrr_derived_enqueue(tree, flags, st)) != cudaSuccess)
        return fail(hrr_cuda_fail(ctx, e, "top and widen kernels"));
    ctx->launches += hrr_derived_launches(tree);
    if ((e = cudaMemcpyAsync(&ctx->host_counters[2], flags, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(hrr_cuda_fail(ctx, e, "flag copy"));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(hrr_cuda_fail(ctx, e, "build"));
    if (n > 1) tree->height = (uint32_t)(ctx->host_counters[4] & 0xFFFFFFFFull);
    if (ctx->host_counters[2] & HRR_FLAG_NONFINITE)
        return fail(hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a light position or intensity is not finite"));
    if (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY)
        return fail(hrr_fail(ctx, HRR_ERR_DEVICE, "inconsistent radix-tree links"));
    *out = tree;
    return HRR_OK;
}

// ------------------------------------------------------------------------------------
// Refit for moved lights
// ------------------------------------------------------------------------------------

size_t hrr_refit_scratch_bytes(uint32_t n) {
    const size_t un = (size_t)n;
    return ((sizeof(float4) * un + 255) & ~size_t(255)) + 2 * ((sizeof(uint32_t) * un + 255) & ~size_t(255)) +
           ((sizeof(uint32_t) * un + 255) & ~size_t(255)) + ((sizeof(uint32_t) * 2 * un + 255) & ~size_t(255)) +
           256 + 1024;
}

cudaError_t hrr_refit_enqueue(hrr_tree *tree, const hrr_lights &L, void *scratch_mem, unsigned long long *flags,
                              cudaStream_t st) {
    const uint32_t n = tree->n;
    if (n == 1) {
        // one leaf: rewrite the single record unless the light is not finite (checked there)
        single_leaf_kernel<<<1, 1, 0, st>>>(L.x, L.y, L.z, L.intensity, tree->nodes, tree->perm, flags);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? hrr_derived_enqueue(tree, flags, st) : e;
    }
    char *p = static_cast<char *>(scratch_mem);
    float4 *spos = carve<float4>(p, n);
    uint32_t *leaf_parent = carve<uint32_t>(p, n), *int_parent = carve<uint32_t>(p, n);
    uint32_t *arrivals = carve<uint32_t>(p, n);
    uint32_t *child_height = carve<uint32_t>(p, 2 * (size_t)n);
    uint32_t *root_height = carve<uint32_t>(p, 1);
    const unsigned g = (n + kThreads - 1) / kThreads, gi = (n - 1 + kThreads - 1) / kThreads;
    gather_check_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, tree->perm, n, spos, flags);
    cudaError_t e = cudaMemsetAsync(arrivals, 0, sizeof(uint32_t) * (size_t)n, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(leaf_parent, 0xFF, 2 * ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)), st);
    if (e != cudaSuccess) return e;
    links_kernel<<<gi, kThreads, 0, st>>>(tree->nodes, n, leaf_parent, int_parent, flags);
    refit_kernel<<<g, kThreads, 0, st>>>(spos, n, tree->nodes, leaf_parent, int_parent, arrivals, child_height,
                                         root_height, flags);
    e = cudaGetLastError();
    return e == cudaSuccess ? hrr_derived_enqueue(tree, flags, st) : e;
}

cudaError_t hrr_derived_enqueue(hrr_tree *tree, const unsigned long long *flags, cudaStream_t st) {
    const uint32_t n = tree->n;
    const float4 *nodes = reinterpret_cast<const float4 *>(tree->nodes);
    const size_t n_rec = n > 1 ? n - 1 : 1;
    top_kernel<<<1, 64, 0, st>>>(nodes, n, reinterpret_cast<float4 *>(tree->nodes) + 4 * n_rec, flags);
    if (!tree->wide) return cudaGetLastError();
    const unsigned g = n > 1 ? (n - 1 + kThreads - 1) / kThreads : 1;
    widen_kernel<<<g, kThreads, 0, st>>>(nodes, n, tree->wide, flags);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Build without allocation
// ------------------------------------------------------------------------------------
//
// hrr_build_light_tree_static runs the same kernels as hrr_build_light_tree, but takes
// its working memory from one file-scope device array instead of allocating, and writes
// the hierarchy into arrays the caller provides. Host code must not hand the array's name
// to a kernel (in host code it names a host-side stand-in); its device address is looked
// up once per device with cudaGetSymbolAddress and cached.

#include <cstdio>
#include <mutex>

namespace {

constexpr uint32_t kStaticMaxLights = HRR_STATIC_BUILD_MAX_LIGHTS;

constexpr size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr size_t static_scratch_bytes(size_t n) {
    return 2 * pad256(sizeof(uint64_t) * n)                               // keys, ping-pong
           + pad256(sizeof(uint32_t) * n)                                 // second value buffer
           + pad256(sizeof(uint32_t) * 256 * ((n + kTile - 1) / kTile + 1)) // digit histograms, totals
           + pad256(sizeof(float4) * n)                                   // sorted lights
           + 2 * pad256(sizeof(uint32_t) * n)                             // parent links
           + pad256(sizeof(uint32_t) * n)                                 // arrival counters
           + pad256(sizeof(uint32_t) * 2 * n)                             // child heights
           + pad256(sizeof(uint32_t))                                     // root height
           + pad256(sizeof(unsigned long long));                          // error flags
}

// The shared working memory of every hrr_build_light_tree_static call on a device
// (about 3.6 MiB for 65536 lights), held by each device that loads the library.
static __device__ __align__(256) unsigned char g_static_build_scratch[static_scratch_bytes(kStaticMaxLights)];

std::mutex g_static_mutex;
void *g_static_scratch_ptr[128] = {};

void set_err(char *err, size_t len, const char *msg) {
    if (err && len) snprintf(err, len, "%s", msg);
}

}  // namespace

extern "C" int hrr_build_light_tree_static(hrr_lights L, uint32_t n, hrr_node *dev_nodes,
                                           uint32_t *dev_perm, uint32_t *out_height,
                                           void *cuda_stream, char *err, size_t err_len) {
    set_err(err, err_len, "");
    if (n == 0 || n > kStaticMaxLights) {
        char msg[160];
        snprintf(msg, sizeof msg, "n_lights = %u is outside [1, %u], the most this call's fixed "
                 "working memory holds; use hrr_build_light_tree for larger light sets", n, kStaticMaxLights);
        set_err(err, err_len, msg);
        return HRR_ERR_INVALID_ARG;
    }
    if (!L.x || !L.y || !L.z || !L.intensity || !dev_nodes || !dev_perm) {
        set_err(err, err_len, "a light, node or permutation array is NULL");
        return HRR_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        set_err(err, err_len, "no usable current CUDA device");
        return HRR_ERR_CUDA;
    }
    char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_build_scratch);
            if (e != cudaSuccess || !p) {
                set_err(err, err_len, "cudaGetSymbolAddress of the build working memory failed");
                return HRR_ERR_CUDA;
            }
            g_static_scratch_ptr[dev] = p;
        }
        scratch = static_cast<char *>(g_static_scratch_ptr[dev]);
    }
    char *p = scratch;
    uint64_t *keys0 = carve<uint64_t>(p, kStaticMaxLights), *keys1 = carve<uint64_t>(p, kStaticMaxLights);
    uint32_t *vals1 = carve<uint32_t>(p, kStaticMaxLights);
    uint32_t *hist = carve<uint32_t>(p, 256 * ((kStaticMaxLights + kTile - 1) / kTile + 1));
    float4 *spos = carve<float4>(p, kStaticMaxLights);
    uint32_t *leaf_parent = carve<uint32_t>(p, kStaticMaxLights), *int_parent = carve<uint32_t>(p, kStaticMaxLights);
    uint32_t *arrivals = carve<uint32_t>(p, kStaticMaxLights);
    uint32_t *child_height = carve<uint32_t>(p, 2 * (size_t)kStaticMaxLights);
    uint32_t *root_height = carve<uint32_t>(p, 1);
    unsigned long long *flags = carve<unsigned long long>(p, 1);

    // Every call reuses the array: clear what the kernels expect to start cleared.
    e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(root_height, 0, sizeof(uint32_t), st);
    if (n == 1) {
        if (e == cudaSuccess) {
            single_leaf_kernel<<<1, 1, 0, st>>>(L.x, L.y, L.z, L.intensity, dev_nodes, dev_perm, flags);
            e = cudaGetLastError();
        }
    } else {
        const uint32_t nblocks = (n + kTile - 1) / kTile;
        if (e == cudaSuccess) e = cudaMemsetAsync(arrivals, 0, sizeof(uint32_t) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(leaf_parent, 0xFF, sizeof(uint32_t) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(int_parent, 0xFF, sizeof(uint32_t) * (size_t)n, st);
        if (e == cudaSuccess) {
            const unsigned g = (n + kThreads - 1) / kThreads;
            morton_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, n, keys0, dev_perm, flags);
            uint64_t *kin = keys0, *kout = keys1;
            uint32_t *vin = dev_perm, *vout = vals1;
            for (int shift = 0; shift < 64; shift += 8) {
                radix_hist_kernel<<<nblocks, kThreads, 0, st>>>(kin, n, shift, hist, nblocks);
                digit_scan_kernel<<<32, 256, 0, st>>>(hist, nblocks, hist + 256 * (size_t)nblocks);
                radix_scatter_kernel<<<nblocks, kThreads, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblocks,
                                                                     hist + 256 * (size_t)nblocks);
                uint64_t *tk = kin; kin = kout; kout = tk;
                uint32_t *tv = vin; vin = vout; vout = tv;
            }
            gather_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, dev_perm, n, spos);
            const unsigned gi = (n - 1 + kThreads - 1) / kThreads;
            topology_kernel<<<gi, kThreads, 0, st>>>(keys0, n, dev_nodes, leaf_parent, int_parent);
            refit_kernel<<<g, kThreads, 0, st>>>(spos, n, dev_nodes, leaf_parent, int_parent, arrivals,
                                                 child_height, root_height, flags);
            e = cudaGetLastError();
        }
    }
    uint32_t height = 0;
    unsigned long long host_flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&height, root_height, sizeof height, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flags, flags, sizeof host_flags, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof msg, "CUDA error in the build: %s", cudaGetErrorString(e));
        set_err(err, err_len, msg);
        return HRR_ERR_CUDA;
    }
    if (host_flags & HRR_FLAG_NONFINITE) {
        set_err(err, err_len, "a light position or intensity is not finite");
        return HRR_ERR_INVALID_ARG;
    }
    if (host_flags & HRR_FLAG_TOPOLOGY) {
        set_err(err, err_len, "inconsistent radix-tree links");
        return HRR_ERR_DEVICE;
    }
    if (out_height) *out_height = height;
    return HRR_OK;
}
