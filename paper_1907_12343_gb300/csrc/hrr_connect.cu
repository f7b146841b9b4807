// Connection evaluation: the step after the culling (the connections it keeps are what a
// bidirectional path tracer then evaluates).
//
// Every accepted pair (eye j, light id) carries the Russian-roulette weight
// (I / max(d^2, 1e-4)) / p_ij, with d^2 and p_ij the acceptance rule's own float32 values,
// times the visibility of the open segment eye -> light against a triangle scene. The
// per-eye sums of the weights are unbiased estimates of the eyes' unculled sums.
//
// The scene is a bounding-volume hierarchy over the triangles: the light-hierarchy builder
// orders the triangles by the Morton keys of their centroids and builds the same binary
// radix tree over them; a refit then replaces the records' point boxes with triangle
// boxes, widened so that floating-point slab tests can never reject a box that holds a
// crossing. Each lane of a persistent grid traces one pair's shadow segment at a time (any
// hit ends it) and takes the next pair when it is done.
#include <algorithm>
#include <new>

#include "hrr_internal.cuh"

struct hrr_scene {
    int device = 0;
    uint32_t n = 0;
    hrr_tree *tree = nullptr;  // records: child boxes of the triangles; perm: sorted -> original
    float *tris = nullptr;     // sorted triangles, 16 floats each: v0, e1 = v1 - v0, e2 = v2 - v0, pad
};

namespace {

constexpr int kThreads = 256;
constexpr int kStack = 128;  // >= height of the radix tree (at most 96) + 2
constexpr int kTriFloats = 16;  // a sorted triangle's stride (64 bytes: aligned 256-bit loads)

__global__ void __launch_bounds__(kThreads) centroid_kernel(const float *__restrict__ tri, uint32_t n,
                                                             float *cx, float *cy, float *cz, float *zero,
                                                             unsigned long long *flags) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const float *t = tri + 9 * (size_t)i;
    float s[3];
    for (int c = 0; c < 3; ++c) {
        const float a = t[c], b = t[3 + c], d = t[6 + c];
        if (!isfinite(a) || !isfinite(b) || !isfinite(d)) atomicOr(flags, HRR_FLAG_NONFINITE);
        s[c] = (a + b + d) * (1.0f / 3.0f);
    }
    cx[i] = s[0];
    cy[i] = s[1];
    cz[i] = s[2];
    zero[i] = 0.0f;
}

// A box that surely holds a triangle: its vertices' bounds widened by 2^-16 of the
// larger of their magnitude and the box's extent (float32 rounding in the slab and
// triangle tests is below 2^-20 of those).
__device__ __forceinline__ void tri_box(const float *t, float lo[3], float hi[3]) {
    for (int c = 0; c < 3; ++c) {
        const float a = fminf(fminf(t[c], t[3 + c]), t[6 + c]);
        const float b = fmaxf(fmaxf(t[c], t[3 + c]), t[6 + c]);
        const float m = fmaxf(fmaxf(fabsf(a), fabsf(b)), b - a) * 1.52587890625e-05f + 1e-30f;
        lo[c] = a - m;
        hi[c] = b + m;
    }
}

__device__ __forceinline__ void store_box(hrr_node *node, uint32_t slot, const float lo[3], const float hi[3]) {
    float *f = reinterpret_cast<float *>(node) + (slot ? 8 : 0);
    f[0] = lo[0]; f[1] = lo[1]; f[2] = lo[2]; f[3] = 0.0f;
    f[4] = hi[0]; f[5] = hi[1]; f[6] = hi[2];
}

// Sorted triangles, and the bottom-up refit of the records with triangle boxes (the same
// arrival scheme as the light refit: the second child to arrive finishes its parent).
__global__ void __launch_bounds__(kThreads) tri_refit_kernel(const float *__restrict__ tri, const uint32_t *perm,
                                                             uint32_t n, hrr_node *nodes, float *sorted,
                                                             const uint32_t *__restrict__ leaf_parent,
                                                             const uint32_t *__restrict__ int_parent,
                                                             uint32_t *arrivals, unsigned long long *flags) {
    const uint32_t leaf = blockIdx.x * kThreads + threadIdx.x;
    if (leaf >= n) return;
    const float *t = tri + 9 * (size_t)perm[leaf];
    // v0 and the edges e1, e2 (the segment test's first six roundings, done once here), so
    // that one 256-bit load and one 32-bit load fetch a triangle
    float *o = sorted + kTriFloats * (size_t)leaf;
    o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
    o[3] = __fsub_rn(t[3], t[0]); o[4] = __fsub_rn(t[4], t[1]); o[5] = __fsub_rn(t[5], t[2]);
    o[6] = __fsub_rn(t[6], t[0]); o[7] = __fsub_rn(t[7], t[1]); o[8] = __fsub_rn(t[8], t[2]);
    for (int c = 9; c < kTriFloats; ++c) o[c] = 0.0f;
    float lo[3], hi[3];
    tri_box(t, lo, hi);
    if (n == 1) {
        store_box(nodes, 0, lo, hi);
        store_box(nodes, 1, lo, hi);
        return;
    }
    uint32_t code = leaf_parent[leaf];
    for (;;) {
        const uint32_t node = code >> 1, slot = code & 1u;
        if (code == 0xFFFFFFFFu || node >= n - 1) {
            atomicOr(flags, HRR_FLAG_TOPOLOGY);
            return;
        }
        store_box(&nodes[node], slot, lo, hi);
        __threadfence();
        if (atomicAdd(&arrivals[node], 1u) == 0u) return;
        __threadfence();
        const float *f = reinterpret_cast<const float *>(&nodes[node]);
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(__ldcg(f + c), __ldcg(f + 8 + c));
            hi[c] = fmaxf(__ldcg(f + 4 + c), __ldcg(f + 12 + c));
        }
        if (node == 0) return;
        code = int_parent[node];
    }
}

__global__ void __launch_bounds__(kThreads) scene_links_kernel(const hrr_node *__restrict__ nodes, uint32_t n,
                                                               uint32_t *__restrict__ leaf_parent,
                                                               uint32_t *__restrict__ int_parent,
                                                               unsigned long long *flags) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n - 1) return;
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

// Open segment e -> e + D, t in (1e-4, 1 - 1e-4), against the closed triangle (v0, v1, v2),
// stored as v0, e1 = v1 - v0, e2 = v2 - v0: Moller-Trumbore with every product and sum
// rounded separately (no fused operations), dot products summed x + y then + z, one
// correctly rounded reciprocal of det.
__device__ __forceinline__ bool segment_hits(const float e[3], const float D[3], const float *__restrict__ tri) {
    float v0x, v0y, v0z, e1x, e1y, e1z, e2x, e2y;
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v0x), "=f"(v0y), "=f"(v0z), "=f"(e1x), "=f"(e1y), "=f"(e1z), "=f"(e2x), "=f"(e2y)
        : "l"(tri));
    const float e2z = __ldg(tri + 8);
    const float Px = __fsub_rn(__fmul_rn(D[1], e2z), __fmul_rn(D[2], e2y));
    const float Py = __fsub_rn(__fmul_rn(D[2], e2x), __fmul_rn(D[0], e2z));
    const float Pz = __fsub_rn(__fmul_rn(D[0], e2y), __fmul_rn(D[1], e2x));
    const float det = __fadd_rn(__fadd_rn(__fmul_rn(e1x, Px), __fmul_rn(e1y, Py)), __fmul_rn(e1z, Pz));
    if (det == 0.0f) return false;
    const float inv = __frcp_rn(det);
    const float Tx = __fsub_rn(e[0], v0x), Ty = __fsub_rn(e[1], v0y), Tz = __fsub_rn(e[2], v0z);
    const float u = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(Tx, Px), __fmul_rn(Ty, Py)), __fmul_rn(Tz, Pz)), inv);
    if (!(u >= 0.0f && u <= 1.0f)) return false;
    const float Qx = __fsub_rn(__fmul_rn(Ty, e1z), __fmul_rn(Tz, e1y));
    const float Qy = __fsub_rn(__fmul_rn(Tz, e1x), __fmul_rn(Tx, e1z));
    const float Qz = __fsub_rn(__fmul_rn(Tx, e1y), __fmul_rn(Ty, e1x));
    const float v = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(D[0], Qx), __fmul_rn(D[1], Qy)), __fmul_rn(D[2], Qz)), inv);
    if (!(v >= 0.0f && __fadd_rn(u, v) <= 1.0f)) return false;
    const float t = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(e2x, Qx), __fmul_rn(e2y, Qy)), __fmul_rn(e2z, Qz)), inv);
    return t > 1e-4f && t < 1.0f - 1e-4f;
}

// Slab test of the segment's [0, 1] against a box, widened by 2^-20 on both ends.
__device__ __forceinline__ bool box_hit(const float e[3], const float inv[3], const float lo[3], const float hi[3]) {
    float tn = 0.0f, tf = 1.0f;
    for (int c = 0; c < 3; ++c) {
        const float a = (lo[c] - e[c]) * inv[c], b = (hi[c] - e[c]) * inv[c];
        tn = fmaxf(tn, fminf(a, b));
        tf = fminf(tf, fmaxf(a, b));
    }
    return tn * (1.0f - 9.5367431640625e-07f) <= tf * (1.0f + 9.5367431640625e-07f);
}

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

struct ConnectArgs {
    hrr_eyes eyes;
    uint32_t n_eyes;
    hrr_lights lights;
    uint32_t n_lights;
    float tau;
    const uint2 *pairs;
    unsigned long long n_pairs;
    const float4 *nodes;  // scene, or NULL
    const float *tris;    // sorted triangles, kTriFloats each
    uint32_t n_tris;
    float *weight;        // per pair, or NULL
    uint8_t *visible;     // per pair, or NULL
    float *eye_sum;       // per eye
    unsigned long long *flags;
    unsigned long long *cursor;  // next pair to trace (starts at 0)
};

#ifndef HRR_CONNECT_REFILL_BELOW
#define HRR_CONNECT_REFILL_BELOW 24
#endif
constexpr uint32_t kRefillBelow = HRR_CONNECT_REFILL_BELOW;  // refill idle lanes once fewer are busy

// The outputs of pair k (eye j): weight times visibility, the visibility bit, the eye's sum.
__device__ __forceinline__ void finish(const ConnectArgs &A, unsigned long long k, uint32_t j, float w, bool vis) {
    const float out = vis ? w : 0.0f;
    if (A.weight) A.weight[k] = out;
    if (A.visible) A.visible[k] = vis ? 1 : 0;
    if (out != 0.0f) atomicAdd(&A.eye_sum[j], out);
}

// Without a scene every connection is visible: one thread per pair, grid-stride.
__global__ void __launch_bounds__(kThreads) weights_kernel(const ConnectArgs A) {
    const unsigned long long stride = (unsigned long long)gridDim.x * kThreads;
    for (unsigned long long k = (unsigned long long)blockIdx.x * kThreads + threadIdx.x; k < A.n_pairs; k += stride) {
        const uint2 pr = A.pairs[k];
        if (pr.x >= A.n_eyes || pr.y >= A.n_lights) {
            atomicOr(A.flags, HRR_FLAG_RANGE);
            continue;
        }
        const float dx = __fsub_rn(A.lights.x[pr.y], A.eyes.x[pr.x]);
        const float dy = __fsub_rn(A.lights.y[pr.y], A.eyes.y[pr.x]);
        const float dz = __fsub_rn(A.lights.z[pr.y], A.eyes.z[pr.x]);
        const float inten = A.lights.intensity[pr.y];
        float d2 = __fmul_rn(dx, dx);
        d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
        d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
        const float den = fmaxf(d2, 1e-4f);
        const float p = fminf(1.0f, __fdiv_rn(__fmul_rn(A.tau, inten), den));
        finish(A, k, pr.x, __fdiv_rn(__fdiv_rn(inten, den), p), true);
    }
}

// Persistent segments: each lane traces one pair's segment, one hierarchy node per step,
// and a warp refills its idle lanes from the global pair cursor (one atomic per refill), so
// lanes do not idle behind the warp's longest segment. A segment ends at its first
// crossing (occluded) or when its stack runs dry (visible).
__global__ void __launch_bounds__(kThreads) connect_kernel(const ConnectArgs A) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    bool alive = false, more = true;
    unsigned long long k = 0;
    uint32_t j = 0, node = 0, steps = 0;
    int sp = 0;
    float w = 0.0f;
    float e[3] = {0.f, 0.f, 0.f}, D[3] = {0.f, 0.f, 0.f}, inv[3] = {0.f, 0.f, 0.f};
    uint32_t stack[kStack];
    for (;;) {
        unsigned alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        if (more && (uint32_t)__popc(alive_mask) < kRefillBelow) {
            const unsigned idle = ~alive_mask;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(A.cursor, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + __popc(idle) >= A.n_pairs) more = false;
            if (!alive) {
                k = base + __popc(idle & lt);
                if (k < A.n_pairs) {
                    const uint2 pr = A.pairs[k];
                    if (pr.x >= A.n_eyes || pr.y >= A.n_lights) {
                        atomicOr(A.flags, HRR_FLAG_RANGE);
                    } else {
                        j = pr.x;
                        e[0] = A.eyes.x[j]; e[1] = A.eyes.y[j]; e[2] = A.eyes.z[j];
                        const float l0 = A.lights.x[pr.y], l1 = A.lights.y[pr.y], l2 = A.lights.z[pr.y];
                        const float inten = A.lights.intensity[pr.y];
                        D[0] = __fsub_rn(l0, e[0]); D[1] = __fsub_rn(l1, e[1]); D[2] = __fsub_rn(l2, e[2]);
                        // the weight: the acceptance rule's d^2 and p, then (I / den) / p
                        float d2 = __fmul_rn(D[0], D[0]);
                        d2 = __fadd_rn(d2, __fmul_rn(D[1], D[1]));
                        d2 = __fadd_rn(d2, __fmul_rn(D[2], D[2]));
                        const float den = fmaxf(d2, 1e-4f);
                        const float p = fminf(1.0f, __fdiv_rn(__fmul_rn(A.tau, inten), den));
                        w = __fdiv_rn(__fdiv_rn(inten, den), p);
                        if (A.n_tris == 1) {
                            finish(A, k, j, w, !segment_hits(e, D, A.tris));
                        } else {
                            // a zero component is taken as 1e-30: its slab then admits exactly
                            // the boxes whose range holds e (up to 1e-30, a conservative margin)
                            for (int c = 0; c < 3; ++c) inv[c] = __frcp_rn(D[c] == 0.0f ? 1e-30f : D[c]);
                            node = 0;
                            sp = 0;
                            steps = 0;
                            alive = true;
                        }
                    }
                }
            }
            alive_mask = __ballot_sync(0xFFFFFFFFu, alive);
        }
        if (alive_mask == 0u && !more) break;
        if (!alive) continue;
        float4 q0, q1, q2, q3;
        load_record(&A.nodes[4 * (size_t)node], q0, q1, q2, q3);
        const uint32_t split = __float_as_uint(q1.w), other = __float_as_uint(q3.w);
        const uint32_t first = min(node, other), last = max(node, other);
        if (last >= A.n_tris || split < first || split >= last || sp >= kStack || ++steps >= A.n_tris) {
            // corrupt records: out-of-range links, an impossible depth, or more steps than
            // the hierarchy has internal nodes
            atomicOr(A.flags, HRR_FLAG_TOPOLOGY);
            alive = false;
            continue;
        }
        const float lo0[3] = {q0.x, q0.y, q0.z}, hi0[3] = {q1.x, q1.y, q1.z};
        const float lo1[3] = {q2.x, q2.y, q2.z}, hi1[3] = {q3.x, q3.y, q3.z};
        const bool h0 = box_hit(e, inv, lo0, hi0), h1 = box_hit(e, inv, lo1, hi1);
        const bool leaf0 = first == split, leaf1 = split + 1 == last;
        bool hit = false;
        if (h0 && leaf0) {
            hit = segment_hits(e, D, A.tris + kTriFloats * (size_t)split);
        }
        if (!hit && h1 && leaf1) {
            hit = segment_hits(e, D, A.tris + kTriFloats * (size_t)(split + 1));
        }
        const bool go0 = h0 && !leaf0, go1 = h1 && !leaf1;
        if (hit) {
            finish(A, k, j, w, false);
            alive = false;
        } else if (go0 && go1) {
            stack[sp++] = split + 1;
            node = split;
        } else if (go0) {
            node = split;
        } else if (go1) {
            node = split + 1;
        } else if (sp > 0) {
            node = stack[--sp];
        } else {
            finish(A, k, j, w, true);
            alive = false;
        }
    }
}

}  // namespace

extern "C" {

int hrr_build_scene(hrr_ctx *ctx, const float *dev_tris, uint32_t n_tris, hrr_scene **out) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!out) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!dev_tris || n_tris == 0 || n_tris > 0x7FFFFFFFu)
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "need 1 .. 2^31 - 1 triangles");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    unsigned long long *flags = ctx->counters + 2;
    const size_t n = n_tris;
    float *cen = nullptr;
    HRR_CUDA(ctx, cudaMallocAsync(&cen, sizeof(float) * 4 * n, st));
    const unsigned gr = (unsigned)((n + kThreads - 1) / kThreads);
    HRR_CUDA(ctx, cudaMemsetAsync(flags, 0, sizeof(unsigned long long), st));
    centroid_kernel<<<gr, kThreads, 0, st>>>(dev_tris, n_tris, cen, cen + n, cen + 2 * n, cen + 3 * n, flags);
    ++ctx->launches;
    HRR_CUDA(ctx, cudaMemcpyAsync(&ctx->host_counters[2], flags, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->host_counters[2] & HRR_FLAG_NONFINITE) {
        cudaFreeAsync(cen, st);
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a triangle vertex is not finite");
    }
    hrr_tree *tree = nullptr;
    const hrr_lights L{cen, cen + n, cen + 2 * n, cen + 3 * n};
    int rc = hrr_build_impl(ctx, L, n_tris, &tree);  // the centroids' radix tree (synchronous)
    cudaFreeAsync(cen, st);
    if (rc != HRR_OK) return rc;
    if (tree->wide) {  // the segment walk reads the binary records only
        cudaFreeAsync(tree->wide, st);
        tree->wide = nullptr;
    }
    hrr_scene *sc = new (std::nothrow) hrr_scene();
    if (!sc) {
        hrr_free_light_tree(ctx, tree);
        return hrr_fail(ctx, HRR_ERR_OOM, "host allocation of the scene");
    }
    sc->device = ctx->device;
    sc->n = n_tris;
    sc->tree = tree;
    uint32_t *links = nullptr;
    cudaError_t e = cudaMallocAsync(&sc->tris, sizeof(float) * kTriFloats * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&links, sizeof(uint32_t) * 3 * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(links, 0xFF, sizeof(uint32_t) * 2 * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(links + 2 * n, 0, sizeof(uint32_t) * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        if (n > 1) {
            scene_links_kernel<<<(unsigned)((n - 1 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                tree->nodes, n_tris, links, links + n, flags);
            ++ctx->launches;
        }
        tri_refit_kernel<<<gr, kThreads, 0, st>>>(dev_tris, tree->perm, n_tris, tree->nodes, sc->tris, links,
                                                  links + n, links + 2 * n, flags);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (links) cudaFreeAsync(links, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ctx->host_counters[2], flags, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || (ctx->host_counters[2] & HRR_FLAG_TOPOLOGY)) {
        hrr_free_scene(ctx, sc);
        return e != cudaSuccess ? hrr_cuda_fail(ctx, e, "scene build") : hrr_fail(ctx, HRR_ERR_DEVICE, "scene links");
    }
    *out = sc;
    return HRR_OK;
}

int hrr_free_scene(hrr_ctx *ctx, hrr_scene *scene) {
    if (!ctx || !scene) return HRR_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (scene->tree) hrr_free_light_tree(ctx, scene->tree);
    if (scene->tris) cudaFreeAsync(scene->tris, ctx->stream);
    delete scene;
    return HRR_OK;
}

int hrr_connect(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, hrr_lights lights, uint32_t n_lights, float tau,
                const uint32_t *dev_pairs, uint64_t n_pairs, const hrr_scene *scene, float *dev_weight,
                uint8_t *dev_visible, float *dev_eye_sum) {
    if (!ctx) return HRR_ERR_INVALID_ARG;
    if (!(tau >= 0.0f) || !(tau < __builtin_huge_valf())) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (n_pairs && (!dev_pairs || !eyes.x || !eyes.y || !eyes.z || !lights.x || !lights.y || !lights.z ||
                    !lights.intensity))
        return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a pair, eye or light array is NULL");
    if (n_eyes && !dev_eye_sum) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_eye_sum is NULL");
    if (((uintptr_t)dev_pairs & 7u) != 0) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "dev_pairs must be 8-byte aligned");
    if (scene && scene->device != ctx->device) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "scene lives on another device");
    DeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    unsigned long long *flags = ctx->counters + 2;
    HRR_CUDA(ctx, cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned long long), st));  // flags, pair cursor
    if (n_eyes) HRR_CUDA(ctx, cudaMemsetAsync(dev_eye_sum, 0, sizeof(float) * (size_t)n_eyes, st));
    if (n_pairs) {
        ConnectArgs A{};
        A.eyes = eyes;
        A.n_eyes = n_eyes;
        A.lights = lights;
        A.n_lights = n_lights;
        A.tau = tau;
        A.pairs = reinterpret_cast<const uint2 *>(dev_pairs);
        A.n_pairs = n_pairs;
        A.nodes = scene ? reinterpret_cast<const float4 *>(scene->tree->nodes) : nullptr;
        A.tris = scene ? scene->tris : nullptr;
        A.n_tris = scene ? scene->n : 0;
        A.weight = dev_weight;
        A.visible = dev_visible;
        A.eye_sum = dev_eye_sum;
        A.flags = flags;
        A.cursor = ctx->counters + 3;
        const void *fn = scene ? reinterpret_cast<const void *>(connect_kernel) : reinterpret_cast<const void *>(weights_kernel);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const unsigned long long want = (n_pairs + kThreads - 1) / kThreads;
        const unsigned grid = (unsigned)std::min<unsigned long long>(want, (unsigned long long)per_sm * ctx->sm_count);
        hrr_timing_begin(ctx);
        if (scene) connect_kernel<<<grid, kThreads, 0, st>>>(A);
        else weights_kernel<<<grid, kThreads, 0, st>>>(A);
        hrr_timing_end(ctx);
        ++ctx->launches;
        HRR_CUDA(ctx, cudaGetLastError());
    }
    HRR_CUDA(ctx, cudaMemcpyAsync(&ctx->host_counters[2], flags, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    HRR_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->host_counters[2] & HRR_FLAG_RANGE) return hrr_fail(ctx, HRR_ERR_INVALID_ARG, "a pair's eye or light index is out of range");
    if (ctx->host_counters[2] & (HRR_FLAG_STACK | HRR_FLAG_TOPOLOGY))
        return hrr_fail(ctx, HRR_ERR_DEVICE, "corrupt scene records");
    return HRR_OK;
}

}  // extern "C"
