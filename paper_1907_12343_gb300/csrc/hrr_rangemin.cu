// Batched range minimum of the shifted base-2 radical inverse (Sec. 2).
//
// One query reads (a, b, r) and writes the minimum and its index: 12 + 8 bytes that are
// touched once, so the kernel is a streaming pass bounded by HBM bandwidth. Threads take
// four queries at a time with 16-byte loads and stores when every array is 16-byte
// aligned; the grid is a whole number of waves of resident blocks and strides over the
// queries.
#include "hrr_internal.cuh"

namespace {

template <int VARIANT>
__device__ __forceinline__ uint32_t one_query(uint32_t a, uint32_t b, uint32_t r, uint32_t *k) {
    if (a >= b) {  // empty range: no minimum
        *k = 0xFFFFFFFFu;
        return 0xFFFFFFFFu;
    }
    if (VARIANT == 0) {
        *k = hrr_range_argmin_select(a, b, __brev(0u - r));
        return __brev(*k) + r;
    }
    return hrr_rangemin_closed(a, b, r, k);
}

template <int VARIANT, bool ARGMIN>
__global__ void __launch_bounds__(256) rangemin_vec4_kernel(const uint4 *__restrict__ a,
                                                            const uint4 *__restrict__ b,
                                                            const uint4 *__restrict__ r,
                                                            uint4 *__restrict__ vmin,
                                                            uint4 *__restrict__ argmin,
                                                            uint64_t n4) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const uint4 va = __ldcs(a + q), vb = __ldcs(b + q), vr = __ldcs(r + q);
        uint4 vm, vk;
        vm.x = one_query<VARIANT>(va.x, vb.x, vr.x, &vk.x);
        vm.y = one_query<VARIANT>(va.y, vb.y, vr.y, &vk.y);
        vm.z = one_query<VARIANT>(va.z, vb.z, vr.z, &vk.z);
        vm.w = one_query<VARIANT>(va.w, vb.w, vr.w, &vk.w);
        __stcs(vmin + q, vm);
        if (ARGMIN) __stcs(argmin + q, vk);
    }
}

template <int VARIANT>
__global__ void __launch_bounds__(256) rangemin_scalar_kernel(const uint32_t *__restrict__ a,
                                                              const uint32_t *__restrict__ b,
                                                              const uint32_t *__restrict__ r,
                                                              uint32_t *__restrict__ vmin,
                                                              uint32_t *__restrict__ argmin,
                                                              uint64_t begin, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        uint32_t k;
        const uint32_t v = one_query<VARIANT>(a[q], b[q], r[q], &k);
        vmin[q] = v;
        if (argmin) argmin[q] = k;
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <int VARIANT>
int launch(hrr_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *r, uint32_t *vmin,
           uint32_t *argmin, uint64_t n) {
    const int threads = 256;
    const uint64_t waves_blocks = (uint64_t)ctx->sm_count * 8;  // 2048 resident threads per SM
    uint64_t done = 0;
    const bool vec = aligned16(a) && aligned16(b) && aligned16(r) && aligned16(vmin) &&
                     (!argmin || aligned16(argmin));
    if (vec && n >= 4) {
        const uint64_t n4 = n / 4;
        uint64_t blocks = (n4 + threads - 1) / threads;
        if (blocks > waves_blocks * 4) blocks = waves_blocks * 4;
        if (argmin)
            rangemin_vec4_kernel<VARIANT, true><<<(unsigned)blocks, threads, 0, ctx->stream>>>(
                (const uint4 *)a, (const uint4 *)b, (const uint4 *)r, (uint4 *)vmin, (uint4 *)argmin, n4);
        else
            rangemin_vec4_kernel<VARIANT, false><<<(unsigned)blocks, threads, 0, ctx->stream>>>(
                (const uint4 *)a, (const uint4 *)b, (const uint4 *)r, (uint4 *)vmin, nullptr, n4);
        ++ctx->launches;
        done = n4 * 4;
    }
    if (done < n) {
        uint64_t rest = n - done;
        uint64_t blocks = (rest + threads - 1) / threads;
        if (blocks > waves_blocks * 4) blocks = waves_blocks * 4;
        rangemin_scalar_kernel<VARIANT><<<(unsigned)blocks, threads, 0, ctx->stream>>>(
            a, b, r, vmin, argmin, done, n);
        ++ctx->launches;
    }
    HRR_CUDA(ctx, cudaGetLastError());
    return HRR_OK;
}

}  // namespace

int hrr_range_min_impl(hrr_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *r,
                       uint32_t *out_min, uint32_t *out_argmin, uint64_t n, int variant) {
    if (variant == 0) return launch<0>(ctx, a, b, r, out_min, out_argmin, n);
    return launch<2>(ctx, a, b, r, out_min, out_argmin, n);
}
