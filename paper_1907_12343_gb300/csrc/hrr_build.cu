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

// Exclusive prefix sum of `total` counts in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(uint32_t *data, uint64_t total) {
    __shared__ uint32_t sums[1024];
    const uint64_t per = (total + 1023) / 1024;
    const uint64_t beg = min((uint64_t)threadIdx.x * per, total);
    const uint64_t end = min(beg + per, total);
    uint32_t s = 0;
    for (uint64_t i = beg; i < end; ++i) s += data[i];
    sums[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? sums[threadIdx.x - off] : 0u;
        __syncthreads();
        sums[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? sums[threadIdx.x - 1] : 0u;
    for (uint64_t i = beg; i < end; ++i) {
        const uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// Stable scatter of one tile: items are taken 256 at a time in tile order; an item's
// rank among equal digits is (earlier rounds) + (earlier warps this round) + (earlier
// lanes of its warp, from __match_any_sync).
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, uint32_t n, int shift,
    const uint32_t *__restrict__ offsets, uint32_t nblocks) {
    __shared__ uint32_t running[256];
    __shared__ uint32_t warp_cnt[kThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = offsets[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
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

template <typename T>
T *carve(char *&p, size_t count) {
    T *r = reinterpret_cast<T *>(p);
    p += (sizeof(T) * count + 255) & ~size_t(255);
    return r;
}

}  // namespace

int hrr_build_impl(hrr_ctx *ctx, const hrr_lights &L, uint32_t n, hrr_tree **out) {
    cudaStream_t st = ctx->stream;
    hrr_tree *tree = new (std::nothrow) hrr_tree();
    if (!tree) return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the tree");
    tree->device = ctx->device;
    tree->n = n;
    auto fail = [&](int status) {
        if (tree->nodes) cudaFreeAsync(tree->nodes, st);
        if (tree->perm) cudaFreeAsync(tree->perm, st);
        delete tree;
        return status;
    };
    const uint32_t n_rec = n > 1 ? n - 1 : 1;
    cudaError_t e = cudaMallocAsync(&tree->nodes, sizeof(hrr_node) * (size_t)n_rec, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&tree->perm, sizeof(uint32_t) * (size_t)n, st);
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
        const uint64_t hist_n = 256ull * nblocks;
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
                exclusive_scan_kernel<<<1, 1024, 0, st>>>(hist, hist_n);
                radix_scatter_kernel<<<nblocks, kThreads, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblocks);
                ctx->launches += 3;
                uint64_t *tk = kin; kin = kout; kout = tk;
                uint32_t *tv = vin; vin = vout; vout = tv;
            }
            // eight passes: the sorted keys are back in keys0 and the permutation in vals0
            gather_kernel<<<g, kThreads, 0, st>>>(L.x, L.y, L.z, L.intensity, vals0, n, spos);
            if ((e = cudaMemsetAsync(arrivals, 0, sizeof(uint32_t) * (size_t)n, st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "memset"); break; }
            if ((e = cudaMemsetAsync(leaf_parent, 0xFF, 2 * ((sizeof(uint32_t) * (size_t)n + 255) & ~size_t(255)), st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "memset"); break; }
            const unsigned gi = (n - 1 + kThreads - 1) / kThreads;
            topology_kernel<<<gi, kThreads, 0, st>>>(keys0, n, tree->nodes, leaf_parent, int_parent);
            refit_kernel<<<g, kThreads, 0, st>>>(spos, n, tree->nodes, leaf_parent, int_parent, arrivals,
                                                 child_height, root_height, flags);
            ctx->launches += 3;
            if ((e = cudaGetLastError()) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "build kernels"); break; }
            if ((e = cudaMemcpyAsync(&ctx->host_counters[4], root_height, sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess) { rc = hrr_cuda_fail(ctx, e, "height copy"); break; }
        } while (0);
        cudaFreeAsync(scratch, st);
        if (rc != HRR_OK) return fail(rc);
    }
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
        return cudaGetLastError();
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
           + pad256(sizeof(uint32_t) * 256 * ((n + kTile - 1) / kTile))   // digit histograms
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
    uint32_t *hist = carve<uint32_t>(p, 256 * ((kStaticMaxLights + kTile - 1) / kTile));
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
        const uint64_t hist_n = 256ull * nblocks;
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
                exclusive_scan_kernel<<<1, 1024, 0, st>>>(hist, hist_n);
                radix_scatter_kernel<<<nblocks, kThreads, 0, st>>>(kin, vin, kout, vout, n, shift, hist, nblocks);
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
