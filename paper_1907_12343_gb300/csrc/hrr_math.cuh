// Device-side definitions shared by the library's kernels: the flags the kernels raise and
// the method's arithmetic (range minimum, node bound, leaf test).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Device flags reported through counters[2]
enum : unsigned long long {
    HRR_FLAG_STACK = 1ull,     // traversal stack spill area would overflow (not seen for any tree)
    HRR_FLAG_NONFINITE = 2ull, // a light position or intensity is not finite
    HRR_FLAG_TOPOLOGY = 4ull,  // a node record or parent link is out of range
    HRR_FLAG_RANGE = 8ull,     // an input index (a pair's eye or light) is out of range
};

// ------------------------------------------------------------------------------------
// Device math
// ------------------------------------------------------------------------------------

// Range minimum of the shifted radical inverse, closed form.
//
// With T = (2^32 - r) mod 2^32 (the threshold 1 - r of Sec. 2), the minimum of
// (brev(i) + r) mod 2^32 over [a,b) sits at the smallest brev(i) >= T if any (cases one
// and two of Sec. 2's split), else at the smallest brev(i) (case three, Alg. 1). The
// values brev(i) form a binary trie whose level-k digit is bit k of i, and a level-k
// prefix p is present iff a + ((p - a) mod 2^k) < b. With c = brev(T) (the paper's k_r),
// D = c - a and L = b - a, every quantity of the successor walk is an O(1) bit
// expression:
//   * c is in the range (case one)               iff D < L;
//   * the right sibling of T's path at level k   exists iff bit k of c is 0 and
//     ((D xor 2^k) mod 2^(k+1)) < L;
//   * with h = fls(L), that holds for every zero bit k < h of c, for k = h iff bit h of D
//     is set or (D mod 2^h) < L - 2^h, and above h only for K = h + 1 + ctz(D >> (h+1))
//     when (D mod 2^(h+1)) < L.
// The deepest such level k* fixes the low k*+1 bits of the answer; its members form the
// progression i0, i0 + 2^(k*+1), ... <= b - 1, and by the identity
// Phi_2(l + n 2^d) = 2^-d Phi_2(n) + Phi_2(l) (Sec. 4) the smallest value among them is at
// the multiplier with the most trailing zeros: for s in [x, y], x >= 1, that is y with
// its bits below fls((x-1) xor y) cleared (the same rule, on [a,b), gives case three).
__device__ __forceinline__ uint32_t hrr_most_trailing_zeros(uint32_t x, uint32_t y) {
    // the number in [x, y] with the most trailing zero bits
    if (x == 0u) return 0u;
    const uint32_t h = 31u - __clz((x - 1u) ^ y);
    return y & ~((1u << h) - 1u);
}

__device__ __forceinline__ uint32_t hrr_rangemin_closed(uint32_t a, uint32_t b, uint32_t r,
                                                        uint32_t *argmin) {
    const uint32_t T = 0u - r;
    const uint32_t c = __brev(T);
    const uint32_t L = b - a;
    const uint32_t D = c - a;
    uint32_t k;
    if (D < L) {
        k = c;
    } else {
        const int h = 31 - __clz(L);
        int ks = -1;
        const uint32_t lowD = D & ((2u << h) - 1u);  // 2u << 31 wraps to 0: mask = all ones
        if (lowD < L) {                               // only possible when h <= 30
            const int K = h + __ffs(D >> (h + 1));    // h + 1 + ctz; D >> (h+1) != 0 here
            if (!((c >> K) & 1u)) ks = K;
        }
        if (ks < 0 && !((c >> h) & 1u)) {
            if (((D >> h) & 1u) || (D & ((1u << h) - 1u)) < L - (1u << h)) ks = h;
        }
        if (ks < 0) {
            const uint32_t low = ~c & ((1u << h) - 1u);
            if (low) ks = 31 - __clz(low);
        }
        if (ks >= 0) {
            const uint32_t mask = (2u << ks) - 1u;
            const uint32_t i0 = a + ((D ^ (1u << ks)) & mask);
            const uint32_t s_lo = (i0 >> ks) >> 1;
            const uint32_t s_hi = s_lo + (((b - 1u - i0) >> ks) >> 1);
            const uint32_t s = hrr_most_trailing_zeros(s_lo, s_hi);
            k = ((s << ks) << 1) | (i0 & mask);
        } else {
            k = hrr_most_trailing_zeros(a, b - 1u);
        }
    }
    *argmin = k;
    return __brev(k) + r;
}

// The same computation without branches, for warps whose lanes take different cases. c =
// brev(2^32 - r) is the eye's k_r, passed in because it is constant along a traversal.
// Returns the argmin; the minimum is brev(argmin) + r.
//   * The levels k where the trie branches above k_r's path form a bit mask: every zero
//     bit of c below h = fls(L); bit h when it is zero in c and (D has bit h set or
//     D mod 2^h < L mod 2^h); and bit K = h + 1 + ctz(D >> (h+1)) when it is zero in c and
//     D mod 2^(h+1) < L. The deepest level is ks = fls(mask) (-1: case three).
//   * With P = 2^(ks+1) (1 in case three), the answer lies in the residue class
//     q = i0 mod P, i0 = a + ((D xor 2^ks) mod P): among q + X .. q + Y (multiples of P,
//     X = i0 - q, Y = (b - 1 - q) rounded down to a multiple of P) the smallest Phi_2 is
//     at the one with the most trailing zeros, Y with the bits below
//     fls((X - P) xor Y) cleared (or q itself when X = 0).
//   * P - 1 is all ones shifted right by clz(mask) (a clamped shift: 0 in case three), and
//     2^ks its top bit; the bits below fls(t) are all ones shifted right by clz(t) + 1.
__device__ __forceinline__ uint32_t hrr_range_argmin_select(uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t L = b - a;
    const uint32_t D = c - a;
    const int h = 31 - __clz(L);
    const uint32_t bh = 1u << h;
    const uint32_t mh = bh - 1u;
    const uint32_t Z = ~c;
    uint32_t levels = Z & mh;
    if (((D & bh) != 0u) || (D & mh) < (L & mh)) levels |= Z & bh;
    const uint32_t hiD = (D >> h) >> 1;
    if ((D & (mh | bh)) < L && hiD != 0u) levels |= Z & (bh << __ffs(hiD));  // bit K
    const uint32_t pm = __funnelshift_rc(0xFFFFFFFFu, 0u, (uint32_t)__clz(levels));  // P - 1
    const uint32_t bit = pm & ~(pm >> 1);                                            // 2^ks
    const uint32_t i0 = a + ((D ^ bit) & pm);
    const uint32_t q = i0 & pm;
    const uint32_t X = i0 & ~pm;
    const uint32_t Y = (b - 1u - q) & ~pm;
    // (X - P) xor Y is nonzero whenever X != 0 (X - P < X <= Y); the 1 keeps clz below 32
    const uint32_t t = ((X - pm - 1u) ^ Y) | 1u;
    const uint32_t k = X == 0u ? q : (q | (Y & ~(0x7FFFFFFFu >> __clz(t))));
    return D < L ? c : k;
}

// Exact per-pair test (round to nearest, canonical order, no FMA): accept iff
// xi < ceil(p 2^32), p = min(1, (tau I) / max(d2, 1e-4)). For 0 < p < 1, p 2^32 is an
// exact float below 2^32, so its ceiling fits in 32 bits.
//
// Most tested pairs are rejected, so the test first applies the node test to the light
// alone (a box of one point; den is exactly the pair's max(d2, 1e-4); scale =
// hrr_node_scale(tau)): when RD(RD(xi) den) >= RU(scale I), xi is at least the pair's
// threshold by the node test's soundness, and the pair is rejected without the division.
// Only the pairs that test leaves undecided go on to the exact quotient, so the result is
// the exact rule's in every case.
__device__ __forceinline__ bool hrr_leaf_accepts(uint32_t xi, float tau, float scale, float lx, float ly,
                                                 float lz, float inten, float ex, float ey,
                                                 float ez) {
    const float dx = __fsub_rn(lx, ex);
    const float dy = __fsub_rn(ly, ey);
    const float dz = __fsub_rn(lz, ez);
    float d2 = __fmul_rn(dx, dx);
    d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
    d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
    const float den = fmaxf(d2, 1e-4f);
    if (__fmul_rd(__uint2float_rd(xi), den) >= __fmul_ru(scale, inten)) return false;
    const float num = __fmul_rn(tau, inten);
    const float p = fminf(1.0f, __fdiv_rn(num, den));
    if (p >= 1.0f) return true;
    if (!(p > 0.0f)) return false;
    return xi < __float2uint_ru(__fmul_rn(p, 4294967296.0f));
}

// max(a, b, c) in one instruction (three-operand max of sm_100 and later; a NaN operand
// is ignored as in fmaxf). Exact, so the same as fmaxf(a, fmaxf(b, c)).
__device__ __forceinline__ float hrr_max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The node test's scale for a frame's tau: RU(tau 2^32 (1 + 2^-22)); tau 2^32 is exact (a
// power-of-two scaling), infinite when it overflows.
__device__ __forceinline__ float hrr_node_scale(float tau) {
    return __fmul_ru(tau * 4294967296.0f, 1.0f + 0x1p-22f);
}

// Conservative cull test of a node with box [lo, hi] and maximum intensity imax, for an eye
// at e, with the scale s = hrr_node_scale(tau):
//   den = max(d2, 1e-4), d2 = RD(gz^2 + RD(gy^2 + RD(gx^2))) (fused, rounded down) with
//         per-axis gaps g = max(0, RD(lo - e), RD(e - hi)): at most the float32 max(d^2, 1e-4)
//         of any light in the box;
//   rhs = RU(s imax) >= 2^32 tau imax (1 + 2^-22) >= 2^32 RN(tau I) (1 + 2^-24)(1 + 2^-23) of
//         every light with 0 < I <= imax, when tau I is a normal float.
// The node is culled at range minimum v iff RD(RD(v) den) >= rhs. Then for every such light,
// v den_i >= 2^32 RN(tau I_i) (1 + 2^-23) >= 2^32 RN(RN(tau I_i) / den_i), so v is at least
// its threshold ceil(p_i 2^32). The cases outside that chain are sound as well: rhs <= 0
// (tau imax <= 0: no light below has p > 0) culls at any v, v = 0 included, and otherwise
// v = 0 never culls; if tau I is subnormal the light's threshold is at most 1 and a cull
// needs v >= 1 (rhs > 0); rhs = +inf or NaN (tau 2^32 overflows) never culls.
__device__ __forceinline__ void hrr_node_bound(float scale, float lox, float loy, float loz,
                                               float hix, float hiy, float hiz, float imax,
                                               float ex, float ey, float ez, float &den,
                                               float &rhs) {
    const float gx = hrr_max3(0.0f, __fsub_rd(lox, ex), __fsub_rd(ex, hix));
    const float gy = hrr_max3(0.0f, __fsub_rd(loy, ey), __fsub_rd(ey, hiy));
    const float gz = hrr_max3(0.0f, __fsub_rd(loz, ez), __fsub_rd(ez, hiz));
    float d2 = __fmul_rd(gx, gx);
    d2 = __fmaf_rd(gy, gy, d2);
    d2 = __fmaf_rd(gz, gz, d2);
    den = fmaxf(d2, 1e-4f);
    rhs = __fmul_ru(scale, imax);
}

__device__ __forceinline__ bool hrr_node_culls(uint32_t v, float den, float rhs) {
    return __fmul_rd(__uint2float_rd(v), den) >= rhs;
}
