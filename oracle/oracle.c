/*
 * CPU oracle for blue-noise dithered QMC hierarchical Russian roulette.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU baseline are
 * its only callers; the CUDA library never links or loads it, and the two share no code.
 * Everything here is written for clarity, not speed. Build with -ffp-contract=off and
 * -frounding-math: the float32 expressions below are evaluated one rounded operation at
 * a time, in the order written.
 *
 * Parity pins (tests/test_oracle_*.py) tie each function to what the paper fixes:
 *   brev / Phi_2 ........ permutation of {m/2^k} over [0,2^k); the Sec. 4 identity
 *                         Phi_2(l + n 2^d) = 2^-d Phi_2(n) + Phi_2(l); involution.
 *   scan ................ the definition of v(a,b) itself (Sec. 1).
 *   trie ................ equals scan exhaustively for small B; three-case value ranges.
 *   Alg. 1 .............. equals the scan argmin at r = 0 exhaustively for small B.
 *   Alg. 2 / Alg. 3 ..... worked examples of Sec. 2; equals scan for every a > 0.
 *   thresholds .......... directed-rounding pins; a node culls only ranges whose minimum
 *                         is >= every leaf threshold inside, and culls tightly.
 *   tree ................ partition / containment invariants; brute-force radix split.
 *   culling ............. hierarchical set == flat brute-force set (Sec. 1: the
 *                         hierarchy only removes work, never changes the result).
 */
#include "oracle.h"

#include <fenv.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FENV_ACCESS ON

/* ------------------------------------------------------------------------------------ */
/* Bits                                                                                  */
/* ------------------------------------------------------------------------------------ */

/* Reverse the B low binary digits of x (Sec. 2: Phi_2 reverses the binary expansion of i
 * behind the radix point, so with B digits Phi_2(i) = brev_B(i) / 2^B). */
uint32_t or_brev(uint32_t x, int B)
{
    uint32_t y = 0;
    for (int k = 0; k < B; ++k)
        if ((x >> k) & 1u)
            y |= 1u << (B - 1 - k);
    return y;
}

static uint64_t word_mask(int B) { return (B >= 64) ? ~0ull : ((1ull << B) - 1ull); }

/* Highest set bit, 0-based; -1 for zero (the paper leaves fls(0) undefined). */
static int fls64(uint64_t x)
{
    int h = -1;
    for (int k = 0; k < 64; ++k)
        if ((x >> k) & 1ull)
            h = k;
    return h;
}

/* Lowest set bit, 0-based; B for zero (the paper leaves ffs(0) undefined). */
static int ffs_b(uint64_t x, int B)
{
    for (int k = 0; k < B; ++k)
        if ((x >> k) & 1ull)
            return k;
    return B;
}

static int in_range(uint64_t k, uint64_t a, uint64_t b) { return k >= a && k < b; }

static uint32_t shifted_value(uint64_t i, uint32_t r, int B)
{
    return (uint32_t)(((uint64_t)or_brev((uint32_t)i, B) + r) & word_mask(B));
}

/* ------------------------------------------------------------------------------------ */
/* Range minimum of the shifted radical inverse                                          */
/* ------------------------------------------------------------------------------------ */

/* v(a,b) = min over i in [a,b) of (Phi_2(i) + r) mod 1, and its argmin (Sec. 1 and the
 * argmin restatement in Sec. 2), by trying every index. */
uint32_t or_rangemin_scan(uint64_t a, uint64_t b, uint32_t r, int B, uint64_t *argmin)
{
    uint32_t best = 0;
    uint64_t best_i = a;
    for (uint64_t i = a; i < b; ++i) {
        uint32_t v = shifted_value(i, r, B);
        if (i == a || v < best) {
            best = v;
            best_i = i;
        }
    }
    if (argmin)
        *argmin = best_i;
    return best;
}

/* The same scan over every index of [a,b) with 32-bit words, carrying the reversed index
 * along instead of reversing each i from scratch: going from i - 1 to i flips the low
 * ctz(i) + 1 binary digits of the index (its trailing ones and the zero above them), so
 * the reversal flips the top ctz(i) + 1 digits. Used where every short range of a large
 * query set is scanned. */
uint32_t or_rangemin_scan_inc(uint64_t a, uint64_t b, uint32_t r, uint64_t *argmin)
{
    uint32_t rev = or_brev((uint32_t)a, 32);
    uint32_t best = rev + r;
    uint64_t best_i = a;
    for (uint64_t i = a + 1; i < b; ++i) {
        int t = __builtin_ctzll(i);
        rev ^= 0xFFFFFFFFu << (31 - t);
        uint32_t v = rev + r;
        if (v < best) {
            best = v;
            best_i = i;
        }
    }
    if (argmin)
        *argmin = best_i;
    return best;
}

/* Does some i in [a,b) end in the k binary digits p (i mod 2^k == p)? The first i >= a
 * with that ending is a + ((p - a) mod 2^k). */
static int has_ending(uint64_t a, uint64_t b, uint64_t p, int k)
{
    uint64_t first = a + ((p - a) & word_mask(k));
    return first < b;
}

/* Range minimum as a successor search. The values brev(i), i in [a,b), form a binary trie
 * whose level-k digit is bit k of i. With T = 1 - r (Sec. 2's threshold), the minimum of
 * (Phi_2(i) + r) mod 1 is at the smallest brev(i) >= T when one exists (cases one and two
 * of the three-case split), else at the smallest brev(i) overall (case three). */
uint32_t or_rangemin_trie(uint64_t a, uint64_t b, uint32_t r, int B, uint64_t *argmin)
{
    uint64_t M = word_mask(B);
    uint64_t T = (0ull - (uint64_t)r) & M;
    uint64_t path = 0;          /* low digits of the index spelling T's leading digits */
    int followed = 1;           /* T's whole digit string is present */
    int branch = -1;            /* deepest level where a larger digit than T's exists */
    uint64_t branch_prefix = 0;

    for (int k = 0; k < B; ++k) {
        uint64_t t = (T >> (B - 1 - k)) & 1ull;
        if (t == 0) {
            uint64_t up = path | (1ull << k);
            if (has_ending(a, b, up, k + 1)) {
                branch = k;
                branch_prefix = up;
            }
        }
        uint64_t next = path | (t << k);
        if (!has_ending(a, b, next, k + 1)) {
            followed = 0;
            break;
        }
        path = next;
    }

    uint64_t idx;
    if (followed) {
        idx = path; /* brev(idx) == T: the shifted value is 0 */
    } else {
        /* smallest completion below the branch (or below the root for case three):
         * prefer digit 0 whenever some index of the range continues that way */
        uint64_t pre = (branch >= 0) ? branch_prefix : 0;
        for (int k = (branch >= 0) ? branch + 1 : 0; k < B; ++k)
            if (!has_ending(a, b, pre, k + 1))
                pre |= 1ull << k;
        idx = pre;
    }
    if (argmin)
        *argmin = idx;
    return shifted_value(idx, r, B);
}

/* Alg. 1: the number in [a,b) with the most trailing zero digits, i.e. the argmin of the
 * unshifted Phi_2 (Sec. 2). Starting from a, repeatedly clear the current digit and set
 * the next one up, keeping every candidate that stays inside the range. */
uint64_t or_alg1(uint64_t a, uint64_t b, int B)
{
    (void)B;
    if (a == 0 || a == b - 1)
        return a;
    int b_h = fls64(b);
    int b_l = ffs_b(a, 64);
    uint64_t k = a, m = a;
    for (int i = b_l; i <= b_h - 1; ++i) {
        m &= ~(1ull << i);
        m |= 1ull << (i + 1);
        if (in_range(m, a, b))
            k = m;
    }
    return k;
}

/* Alg. 3, refine(m, i, [a,b)): keep digits [0,i) of m; walk its remaining set digits from
 * the lowest, and at each try the next integer whose digit there is 0 (adding 2^i), which
 * lands in the lower-ordered subset I_0... of Sec. 2.1.1 whenever it stays in range. */
static uint64_t refine(uint64_t m, int i, uint64_t a, uint64_t b, int B)
{
    i = ffs_b(m & ~word_mask(i), B);
    while (i < B - 1) {
        uint64_t k = m + (1ull << i);
        if (in_range(k, a, b))
            m = k;
        i = ffs_b(m & ~word_mask(i + 1), B);
    }
    return m;
}

/* Alg. 2 as printed: case one (k_r in range), the left-to-right sweep of Sec. 2.1 from
 * b_h down to k_p with refinement, then the right-to-left sweep of Sec. 2.2. */
uint64_t or_alg2_printed(uint64_t a, uint64_t b, uint32_t r, int B)
{
    uint64_t M = word_mask(B);
    uint64_t k_r = or_brev((uint32_t)((0ull - (uint64_t)r) & M), B); /* Phi_2^-1(1 - r) */
    if (in_range(k_r, a, b))
        return k_r;

    int b_h = fls64(b);
    int k_p = ffs_b(k_r, B);

    /* m = k_r with every digit above b_h cleared */
    uint64_t m = k_r & word_mask(b_h + 1);

    for (int i = b_h; i >= k_p; --i) {
        if ((m >> i) & 1ull) {
            m &= ~(1ull << i);
        } else {
            uint64_t m_i = m | (1ull << i);
            if (m_i < a)
                m_i |= 1ull << (i + 1);
            m_i = refine(m_i, i + 1, a, b, B);
            if (in_range(m_i, a, b))
                return m_i;
        }
        if ((a >> i) & 1ull)
            m |= 1ull << i; /* keep a's digit so the candidate does not fall below a */
    }

    m = a;
    uint64_t k = b; /* b marks "nothing found yet" */
    for (int i = 0; i < B; ++i) {
        if (in_range(k, a, b) && i == k_p)
            return k;
        if (i > 0)
            m &= ~(1ull << (i - 1));
        m |= 1ull << i;
        if (m < a)
            m |= 1ull << (i + 1);
        uint64_t m_i = refine(m, i + 1, a, b, B);
        if (in_range(m_i, a, b))
            k = m_i;
    }
    return k;
}

/* Alg. 2 with this build's reading for a = 0: when the printed algorithm returns an index
 * outside [a,b), or (for r != 0) one whose Phi_2 lies below 1 - r although it was looking
 * for the smallest value above it, the answer is case three, the unshifted minimum of
 * Alg. 1. */
uint64_t or_alg2_fixed(uint64_t a, uint64_t b, uint32_t r, int B)
{
    uint64_t M = word_mask(B);
    uint64_t T = (0ull - (uint64_t)r) & M;
    uint64_t k = or_alg2_printed(a, b, r, B);
    if (!in_range(k, a, b) || (r != 0 && or_brev((uint32_t)k, B) < T))
        k = or_alg1(a, b, B);
    return k;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int pick_threads(int nthreads)
{
    int mx = or_max_threads();
    return (nthreads <= 0 || nthreads > mx) ? mx : nthreads;
}

void or_rangemin_batch(const uint32_t *a, const uint32_t *b, const uint32_t *r, uint64_t n,
                       int method, int B, uint32_t *vmin, uint32_t *argmin, int nthreads)
{
    int nt = pick_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nt)
    for (int64_t q = 0; q < (int64_t)n; ++q) {
        uint64_t k = 0;
        uint32_t v;
        switch (method) {
        case 0: v = or_rangemin_scan(a[q], b[q], r[q], B, &k); break;
        case 1: v = or_rangemin_trie(a[q], b[q], r[q], B, &k); break;
        case 2: k = or_alg2_fixed(a[q], b[q], r[q], B); v = shifted_value(k, r[q], B); break;
        case 3: k = or_alg2_printed(a[q], b[q], r[q], B); v = shifted_value(k, r[q], B); break;
        case 5:
            v = B == 32 ? or_rangemin_scan_inc(a[q], b[q], r[q], &k) : or_rangemin_scan(a[q], b[q], r[q], B, &k);
            break;
        default: k = or_alg1(a[q], b[q], B); v = shifted_value(k, 0, B); break;
        }
        vmin[q] = v;
        if (argmin)
            argmin[q] = (uint32_t)k;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Float32 arithmetic with a chosen rounding direction                                   */
/* ------------------------------------------------------------------------------------ */

/* One IEEE-754 binary32 operation under the requested rounding direction. The operands
 * pass through volatile storage so that the operation is performed between the two mode
 * switches. */
__attribute__((noinline)) float or_fround(int op, float x, float y, int mode)
{
    int old = fegetround();
    fesetround(mode < 0 ? FE_DOWNWARD : (mode > 0 ? FE_UPWARD : FE_TONEAREST));
    volatile float vx = x, vy = y;
    volatile float res;
    switch (op) {
    case 0: res = vx + vy; break;
    case 1: res = vx - vy; break;
    case 2: res = vx * vy; break;
    default: res = vx / vy; break;
    }
    fesetround(old);
    return res;
}

static float sub_rd(float x, float y) { return or_fround(1, x, y, -1); }
static float add_rd(float x, float y) { return or_fround(0, x, y, -1); }
static float mul_rd(float x, float y) { return or_fround(2, x, y, -1); }
static float mul_ru(float x, float y) { return or_fround(2, x, y, +1); }

/* RD(x y + z) with one rounding, for finite floats. The product is exact in double (24 + 24
 * significant bits); s = RN(x y + z) in double and its rounding error e are recovered
 * exactly (two-sum). The float below x y + z is the float below s, unless s is itself a
 * float and the exact sum lies below it (e < 0): then it is the next float down. (A float
 * other than s cannot lie between s and s + e: both are doubles, |e| is at most half a
 * double ulp of s.) */
float or_fma_rd(float x, float y, float z)
{
    volatile double p = (double)x * (double)y;
    volatile double sum = p + (double)z;
    volatile double bb = sum - p;
    volatile double e = (p - (sum - bb)) + ((double)z - bb);
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    volatile float f = (float)sum;
    fesetround(old);
    if ((double)f == sum && e < 0.0)
        f = nextafterf(f, -INFINITY);
    return f;
}

static float fma_rd(float x, float y, float z) { return or_fma_rd(x, y, z); }

/* ------------------------------------------------------------------------------------ */
/* Acceptance thresholds                                                                  */
/* ------------------------------------------------------------------------------------ */

static const float kMinDist2 = 1e-4f;

/* ceil(p * 2^32) as an integer in [0, 2^32]; p <= 0 gives 0. p * 2^32 is exact in float
 * (a power-of-two scaling), so only the ceiling rounds. */
static uint64_t fixed_point_ceil(float p)
{
    if (!(p > 0.0f))
        return 0;
    if (p >= 1.0f)
        return 1ull << 32;
    return (uint64_t)ceilf(p * 4294967296.0f);
}

/* Russian-roulette acceptance threshold of one (eye, light) pair. The shifted sample xi
 * (Sec. 1) accepts the connection iff xi / 2^32 < p, i.e. iff xi < ceil(p 2^32). The
 * probability p = min(1, tau I / max(d^2, 1e-4)) is the culling shape of the
 * hierarchical Russian roulette the paper builds on (Sec. 1), evaluated in float32 with
 * round-to-nearest in exactly this order: dx = l - e per axis; d2 = (dx^2 + dy^2) + dz^2;
 * q = (tau I) / max(d2, 1e-4); p = min(1, q). */
uint64_t or_leaf_threshold(float tau, const float l[3], float intensity, const float e[3])
{
    float dx = l[0] - e[0];
    float dy = l[1] - e[1];
    float dz = l[2] - e[2];
    float d2 = dx * dx;
    d2 = d2 + dy * dy;
    d2 = d2 + dz * dz;
    float num = tau * intensity;
    float q = num / fmaxf(d2, kMinDist2);
    return fixed_point_ceil(fminf(1.0f, q));
}

/* u32 -> float rounded toward -inf, by truncating the bits below the 24 significant
 * ones (truncation is rounding down for a non-negative integer). */
static float u32_to_float_rd(uint32_t v)
{
    int h = fls64(v);
    if (h > 23)
        v = (v >> (h - 23)) << (h - 23);
    return (float)v; /* exact: at most 24 significant bits */
}

/* Can a node with box [lo,hi] and maximum intensity imax be culled when the minimum of the
 * eye's shifted sequence over its range is v? It can when v is at least the threshold of
 * every light inside. Per axis the gap to the box is max(0, RD(lo - e), RD(e - hi)); the
 * squared gaps are summed with fused multiply-adds rounded down and floored at 1e-4:
 * den_D <= the float32 max(d^2, 1e-4) of any light in the box. With the scale
 * s = RU(tau' (1 + 2^-22)), tau' = tau 2^32 (exact), the right side RU(s imax) is at least
 * tau' imax (1 + 2^-22) >= 2^32 RN(tau I) (1 + 2^-24)(1 + 2^-23) for any light with
 * 0 < I <= imax (when tau I is a normal float), and each light's quotient
 * RN(RN(tau I) / den) is at most its numerator over den_D times (1 + 2^-24). So the node is
 * culled iff
 *     RD(RD(v) den_D) >= RU(s imax),
 * a division-free test whose left side is a lower bound of v den_D. Outside that chain it
 * is sound too: a right side <= 0 (tau imax <= 0: no light below has p > 0) culls at any v,
 * and otherwise v = 0 never culls; if tau I is subnormal the light's threshold is at most
 * 1 and a cull needs v >= 1; a right side of +inf or NaN (tau' overflows) never culls. */
int or_node_culls(float tau, const float lo[3], const float hi[3], float imax, const float e[3],
                  uint32_t v)
{
    float g[3];
    for (int k = 0; k < 3; ++k) {
        float below = sub_rd(lo[k], e[k]);
        float above = sub_rd(e[k], hi[k]);
        g[k] = fmaxf(0.0f, fmaxf(below, above));
    }
    float d2 = mul_rd(g[0], g[0]);
    d2 = fma_rd(g[1], g[1], d2);
    d2 = fma_rd(g[2], g[2], d2);
    float den = fmaxf(d2, kMinDist2);
    float tau32 = tau * 4294967296.0f; /* exact: a power-of-two scaling */
    float scale = mul_ru(tau32, 1.0f + 0x1p-22f);
    float rhs = mul_ru(scale, imax);
    float lhs = mul_rd(u32_to_float_rd(v), den);
    return lhs >= rhs;
}

/* ------------------------------------------------------------------------------------ */
/* Light hierarchy                                                                        */
/* ------------------------------------------------------------------------------------ */

/* Cell of x on a 2^21 grid over [0,1): floor(x 2^21) clamped to [0, 2^21 - 1]. */
static uint32_t grid_cell(float x)
{
    float s = x * 2097152.0f;
    if (!(s >= 0.0f))
        return 0;
    float f = floorf(s);
    if (f >= 2097151.0f)
        return 2097151u;
    return (uint32_t)f;
}

/* Morton key: bit k of the x cell goes to key bit 3k+2, y to 3k+1, z to 3k. Sorting the
 * light vertices by this key is the spatial sort of Sec. 1 that lets the sequence index i
 * inherit the spatial stratification. */
uint64_t or_morton(float x, float y, float z)
{
    uint32_t cx = grid_cell(x), cy = grid_cell(y), cz = grid_cell(z);
    uint64_t key = 0;
    for (int k = 0; k < 21; ++k) {
        key |= (uint64_t)((cx >> k) & 1u) << (3 * k + 2);
        key |= (uint64_t)((cy >> k) & 1u) << (3 * k + 1);
        key |= (uint64_t)((cz >> k) & 1u) << (3 * k);
    }
    return key;
}

typedef struct {
    uint64_t key;
    uint32_t id;
} keyed_light;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed_light *x = (const keyed_light *)pa, *y = (const keyed_light *)pb;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

/* Does the sorted leaf k carry a 0 at the splitting bit? The ordering key of leaf k is the
 * 96-bit concatenation (Morton key, k): leaves with equal Morton keys are told apart by
 * their position. bit >= 32 addresses Morton bit (bit - 32), bit < 32 position bit. */
static int digit_of(const or_tree *t, uint32_t k, int bit)
{
    if (bit >= 32)
        return (int)((t->key[k] >> (bit - 32)) & 1ull);
    return (int)((k >> bit) & 1u);
}

/* Highest bit where the ordering keys of sorted leaves i and j differ. */
static int highest_difference(const or_tree *t, uint32_t i, uint32_t j)
{
    if (t->key[i] != t->key[j])
        return 32 + fls64(t->key[i] ^ t->key[j]);
    return fls64((uint64_t)(i ^ j));
}

/* Boxes and maximum intensities of every internal node, straight from the leaves of its
 * range (the bound the node test of Sec. 1 needs). */
static void boxes_from_leaves(or_tree *t)
{
    uint32_t ni = t->n - 1;
    for (uint32_t k = 0; k < ni; ++k) {
        float *lo = &t->lo[3 * k], *hi = &t->hi[3 * k];
        for (int c = 0; c < 3; ++c)
            lo[c] = hi[c] = t->pos[3 * t->first[k] + c];
        float im = t->inten[t->first[k]];
        for (uint32_t i = t->first[k]; i <= t->last[k]; ++i) {
            for (int c = 0; c < 3; ++c) {
                lo[c] = fminf(lo[c], t->pos[3 * i + c]);
                hi[c] = fmaxf(hi[c], t->pos[3 * i + c]);
            }
            im = fmaxf(im, t->inten[i]);
        }
        t->imax[k] = im;
    }
}

/* Cost of one child in the cost-driven split: m its maximum intensity clamped at 0, inv
 * the reciprocal of the range's clamped maximum (0 for a dark range), (dx, dy, dz) its box
 * extent and c its light count. With u = m inv (in [0, 1]), A = dx dy + dy dz + dz dx and
 * P = dx + dy + dz, the cost is u^2 ((A + 0.1 P) + 1e-4) c sqrt(c), in float with every
 * operation rounded separately, in this order. */
static float child_cost(float m, float inv, float dx, float dy, float dz, float c)
{
    float u = m * inv;
    float a = dx * dy + dy * dz + dz * dx;
    float p = dx + dy + dz;
    float g = (a + 0.1f * p) + 1e-4f;
    return ((u * u) * g) * (c * sqrtf(c));
}

/* Cost-driven split of the range [f, l] (l > f) over the same leaf order: among the
 * candidate splits k (children [f, k] and [k+1, l]), the one minimising
 * C(k) = child_cost(left) + child_cost(right). A node is visited about in proportion to
 * its count times its maximum intensity over its squared distance; the weights (intensity
 * squared, count to the 1.5, a perimeter term beside the half area) were chosen by the
 * visits they save on several synthetic scenes. Every k in [f, l) is a candidate; a
 * non-finite C never wins. Ties go to the split nearest the middle (the least
 * |c_L - c_R|), then to the smaller k; with no finite C the split is f. The counts are
 * converted to float with rounding to nearest. suf holds 7 floats per leaf of scratch. */
static uint32_t cost_split(const or_tree *t, uint32_t f, uint32_t l, float *suf)
{
    /* suffix boxes and maxima: suf[7 * (i - f)] = lo xyz, hi xyz, max intensity of [i, l] */
    for (uint32_t i = l + 1; i-- > f;) {
        float *o = &suf[7 * (uint64_t)(i - f)];
        const float *p = &t->pos[3 * (uint64_t)i];
        for (int c = 0; c < 3; ++c)
            o[c] = o[3 + c] = p[c];
        o[6] = t->inten[i];
        if (i < l) {
            const float *q = o + 7;
            for (int c = 0; c < 3; ++c) {
                o[c] = fminf(o[c], q[c]);
                o[3 + c] = fmaxf(o[3 + c], q[3 + c]);
            }
            o[6] = fmaxf(o[6], q[6]);
        }
    }
    float lo[3], hi[3], m = -INFINITY;
    for (int c = 0; c < 3; ++c) {
        lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    float best = INFINITY;
    uint32_t best_k = f;
    int64_t best_dist = INT64_MAX;
    for (uint32_t k = f; k < l; ++k) {
        const float *p = &t->pos[3 * (uint64_t)k];
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], p[c]);
            hi[c] = fmaxf(hi[c], p[c]);
        }
        m = fmaxf(m, t->inten[k]);
        const float *r = &suf[7 * (uint64_t)(k + 1 - f)];
        float dxl = hi[0] - lo[0], dyl = hi[1] - lo[1], dzl = hi[2] - lo[2];
        float dxr = r[3] - r[0], dyr = r[4] - r[1], dzr = r[5] - r[2];
        float ml = fmaxf(m, 0.0f), mr = fmaxf(r[6], 0.0f);
        float mx = fmaxf(ml, mr);
        float inv = mx > 0.0f ? 1.0f / fmaxf(mx, FLT_MIN) : 0.0f;
        float cl = (float)(k - f + 1), cr = (float)(l - k);
        float cost = child_cost(ml, inv, dxl, dyl, dzl, cl) + child_cost(mr, inv, dxr, dyr, dzr, cr);
        int64_t dist = (int64_t)(k - f + 1) - (int64_t)(l - k);
        if (dist < 0)
            dist = -dist;
        if (cost < best || (cost == best && dist < best_dist)) {
            best = cost;
            best_k = k;
            best_dist = dist;
        }
    }
    return best_k;
}

static or_tree *tree_build(const float *pos, const float *intensity, uint32_t n, uint32_t cost_depth);

or_tree *or_tree_build(const float *pos, const float *intensity, uint32_t n)
{
    return tree_build(pos, intensity, n, 0);
}

/* Cost splits for the nodes of depth (root = 1) up to cost_depth (0 means 48); deeper
 * nodes take the radix split, which bounds the height by cost_depth + 96 whatever the
 * intensities. */
or_tree *or_tree_build_cost(const float *pos, const float *intensity, uint32_t n, uint32_t cost_depth)
{
    return tree_build(pos, intensity, n, cost_depth ? cost_depth : 48);
}

static or_tree *tree_build(const float *pos, const float *intensity, uint32_t n, uint32_t cost_depth)
{
    if (n == 0)
        return NULL;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    t->n = n;
    keyed_light *kl = (keyed_light *)malloc(sizeof(keyed_light) * n);
    for (uint32_t i = 0; i < n; ++i) {
        kl[i].key = or_morton(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
        kl[i].id = i;
    }
    qsort(kl, n, sizeof(keyed_light), cmp_keyed);
    t->perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * n);
    t->pos = (float *)malloc(sizeof(float) * 3 * n);
    t->inten = (float *)malloc(sizeof(float) * n);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t id = kl[i].id;
        t->perm[i] = id;
        t->key[i] = kl[i].key;
        memcpy(&t->pos[3 * i], &pos[3 * id], 3 * sizeof(float));
        t->inten[i] = intensity[id];
    }
    free(kl);

    uint32_t ni = n - 1;
    t->first = (uint32_t *)malloc(sizeof(uint32_t) * (ni ? ni : 1));
    t->last = (uint32_t *)malloc(sizeof(uint32_t) * (ni ? ni : 1));
    t->split = (uint32_t *)malloc(sizeof(uint32_t) * (ni ? ni : 1));
    t->lo = (float *)malloc(sizeof(float) * 3 * (ni ? ni : 1));
    t->hi = (float *)malloc(sizeof(float) * 3 * (ni ? ni : 1));
    t->imax = (float *)malloc(sizeof(float) * (ni ? ni : 1));
    for (uint32_t k = 0; k < ni; ++k)
        t->first[k] = t->last[k] = t->split[k] = 0xFFFFFFFFu;
    t->height = 0;
    if (ni == 0)
        return t;

    /* Top-down binary radix tree: a range [f,l] splits where the highest differing bit of
     * its end keys changes from 0 to 1. The root is internal node 0; the children of a
     * node split at s are numbered s and s+1. */
    typedef struct { uint32_t id, f, l, depth; } job;
    job *stack = (job *)malloc(sizeof(job) * 512);
    float *suf = cost_depth ? (float *)malloc(sizeof(float) * 7 * (uint64_t)n) : NULL;
    int sp = 0;
    stack[sp++] = (job){0, 0, n - 1, 1};
    while (sp > 0) {
        job j = stack[--sp];
        uint32_t s = j.f;
        if (j.depth <= cost_depth) {
            s = cost_split(t, j.f, j.l, suf);
        } else {
            int bit = highest_difference(t, j.f, j.l);
            for (uint32_t k = j.f; k < j.l; ++k)
                if (digit_of(t, k, bit) == 0)
                    s = k;
        }
        t->first[j.id] = j.f;
        t->last[j.id] = j.l;
        t->split[j.id] = s;
        if (j.depth > t->height)
            t->height = j.depth;
        if (s != j.f)
            stack[sp++] = (job){s, j.f, s, j.depth + 1};
        if (s + 1 != j.l)
            stack[sp++] = (job){s + 1, s + 1, j.l, j.depth + 1};
    }
    free(stack);
    free(suf);

    boxes_from_leaves(t);
    return t;
}

void or_tree_refit(or_tree *t, const float *pos, const float *intensity)
{
    /* Same leaf order and topology (they came from the build's keys); the leaves take the
     * new positions and intensities of their original lights. */
    for (uint32_t i = 0; i < t->n; ++i) {
        uint32_t id = t->perm[i];
        memcpy(&t->pos[3 * i], &pos[3 * id], 3 * sizeof(float));
        t->inten[i] = intensity[id];
    }
    boxes_from_leaves(t);
}

void or_tree_free(or_tree *t)
{
    if (!t)
        return;
    free(t->perm); free(t->key); free(t->pos); free(t->inten);
    free(t->first); free(t->last); free(t->split);
    free(t->lo); free(t->hi); free(t->imax);
    free(t);
}

/* ------------------------------------------------------------------------------------ */
/* Culling                                                                                */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    uint32_t *ids;
    uint64_t n, cap;
} id_list;

static void list_push(id_list *L, uint32_t v)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->ids = (uint32_t *)realloc(L->ids, sizeof(uint32_t) * L->cap);
    }
    L->ids[L->n++] = v;
}

static double now_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* The eye's Cranley-Patterson shift: the tile entry at its pixel (Sec. 1, blue-noise
 * dithering of the shifts over the image plane). */
static uint32_t eye_shift(const uint32_t *tile, uint32_t w, uint32_t h, uint16_t px, uint16_t py)
{
    return tile[(uint64_t)(py % h) * w + (px % w)];
}

static or_cull_result *gather(id_list *lists, uint32_t n_eyes, const uint32_t *eye_ids,
                              const or_tree *t)
{
    or_cull_result *res = (or_cull_result *)calloc(1, sizeof(or_cull_result));
    res->count = (uint32_t *)calloc(n_eyes ? n_eyes : 1, sizeof(uint32_t));
    uint64_t total = 0;
    for (uint32_t j = 0; j < n_eyes; ++j)
        total += lists[j].n;
    res->n_pairs = total;
    res->pairs = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (total ? total : 1));
    uint64_t o = 0;
    for (uint32_t j = 0; j < n_eyes; ++j) {
        res->count[j] = (uint32_t)lists[j].n;
        for (uint64_t q = 0; q < lists[j].n; ++q) {
            res->pairs[2 * o] = eye_ids ? eye_ids[j] : j;
            res->pairs[2 * o + 1] = t->perm[lists[j].ids[q]];
            ++o;
        }
        free(lists[j].ids);
    }
    free(lists);
    return res;
}

/* Flat Russian roulette over every (eye, light) pair: the definition of the result. Light
 * i (sorted position) is accepted for eye j iff (brev(i) + r_j) mod 2^32 < t_ij. */
or_cull_result *or_cull_flat(const or_tree *t, const float *eye_pos, const uint16_t *px,
                             const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                             const uint32_t *tile, uint32_t w, uint32_t h, float tau,
                             int nthreads)
{
    int nt = pick_threads(nthreads);
    (void)nt;
    id_list *lists = (id_list *)calloc(n_eyes ? n_eyes : 1, sizeof(id_list));
    uint32_t *seq = (uint32_t *)malloc(sizeof(uint32_t) * t->n);
    for (uint32_t i = 0; i < t->n; ++i)
        seq[i] = or_brev(i, 32);
    uint64_t marginal = 0;
    double t0 = now_seconds();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt) reduction(+ : marginal)
    for (int64_t jj = 0; jj < (int64_t)n_eyes; ++jj) {
        uint32_t j = (uint32_t)jj;
        const float *e = &eye_pos[3 * (uint64_t)j];
        uint32_t r = eye_shift(tile, w, h, px[j], py[j]);
        for (uint32_t i = 0; i < t->n; ++i) {
            uint32_t xi = seq[i] + r;
            uint64_t thr = or_leaf_threshold(tau, &t->pos[3 * (uint64_t)i], t->inten[i], e);
            if ((uint64_t)xi < thr)
                list_push(&lists[j], i);
            /* acceptance margin in double precision, for reporting only */
            double dx = (double)t->pos[3 * (uint64_t)i] - e[0];
            double dy = (double)t->pos[3 * (uint64_t)i + 1] - e[1];
            double dz = (double)t->pos[3 * (uint64_t)i + 2] - e[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double p = (double)tau * t->inten[i] / (d2 > 1e-4 ? d2 : 1e-4);
            if (p > 1.0)
                p = 1.0;
            double x = (double)xi * (1.0 / 4294967296.0);
            if (p > 0.0 && fabs(x - p) < 1e-6 * p)
                ++marginal;
        }
    }
    double t1 = now_seconds();
    free(seq);
    or_cull_result *res = gather(lists, n_eyes, eye_ids, t);
    res->n_marginal = marginal;
    res->seconds = t1 - t0;
    res->threads = nt;
    return res;
}

/* One child of a visited node during the hierarchical traversal: the leaf range [f, l]
 * (inclusive) of that child and, if it is internal, its node number k. A leaf (f == l) is
 * accepted by the exact pair test; an internal child is pushed unless the minimum of the
 * eye's shifted sequence over [f, l] passes the conservative cull test (or_node_culls),
 * in which case no light below it can be accepted. */
static void consider_child(const or_tree *t, uint32_t f, uint32_t l, uint32_t k, uint32_t r, float tau,
                           const float *e, id_list *acc, uint32_t *stack, int *sp)
{
    if (f == l) {
        uint32_t xi = or_brev(f, 32) + r;
        if ((uint64_t)xi < or_leaf_threshold(tau, &t->pos[3 * (uint64_t)f], t->inten[f], e))
            list_push(acc, f);
        return;
    }
    uint64_t arg;
    uint32_t v = or_rangemin_trie(f, (uint64_t)l + 1, r, 32, &arg);
    if (!or_node_culls(tau, &t->lo[3 * (uint64_t)k], &t->hi[3 * (uint64_t)k], t->imax[k], e, v))
        stack[(*sp)++] = k;
}

/* Hierarchical Russian roulette (Sec. 1): top-down traversal from the root. With width 2
 * each visited internal node tests its two children. With width 4 the binary tree is read
 * as a tree of nodes of width four: a visited node tests its grandchildren (and any child
 * that is a leaf), never its internal children, and only even-depth nodes are visited.
 * Both give the flat set: the cull test is monotone (a smaller box, a smaller maximum
 * intensity and a range minimum over a sub-range never turn a cull into a visit), so a
 * grandchild whose parent would have been culled is culled too. The root is always
 * visited; visits are counted per visited node of the traversal's width. */
or_cull_result *or_cull_hier_w(const or_tree *t, const float *eye_pos, const uint16_t *px,
                               const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                               const uint32_t *tile, uint32_t w, uint32_t h, float tau, int width,
                               int nthreads)
{
    int nt = pick_threads(nthreads);
    (void)nt;
    id_list *lists = (id_list *)calloc(n_eyes ? n_eyes : 1, sizeof(id_list));
    uint64_t *visits = (uint64_t *)calloc(n_eyes ? n_eyes : 1, sizeof(uint64_t));
    uint64_t total_visits = 0;
    double t0 = now_seconds();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt) reduction(+ : total_visits)
    for (int64_t jj = 0; jj < (int64_t)n_eyes; ++jj) {
        uint32_t j = (uint32_t)jj;
        const float *e = &eye_pos[3 * (uint64_t)j];
        uint32_t r = eye_shift(tile, w, h, px[j], py[j]);
        if (t->n == 1) {
            uint32_t xi = or_brev(0, 32) + r;
            if ((uint64_t)xi < or_leaf_threshold(tau, &t->pos[0], t->inten[0], e))
                list_push(&lists[j], 0);
            continue;
        }
        /* depth-first: at most 3 pending nodes per level (width 4; 1 for width 2) plus the
         * last visit's pushes, height <= 144 */
        uint32_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        uint64_t v_count = 0;
        while (sp > 0) {
            uint32_t node = stack[--sp];
            ++v_count;
            uint32_t s = t->split[node];
            uint32_t cf[2] = {t->first[node], s + 1};
            uint32_t cl[2] = {s, t->last[node]};
            uint32_t ck[2] = {s, s + 1};
            for (int c = 0; c < 2; ++c) {
                if (width == 2 || cf[c] == cl[c]) {
                    consider_child(t, cf[c], cl[c], ck[c], r, tau, e, &lists[j], stack, &sp);
                } else { /* an internal child: test its two children instead */
                    uint32_t s2 = t->split[ck[c]];
                    consider_child(t, cf[c], s2, s2, r, tau, e, &lists[j], stack, &sp);
                    consider_child(t, s2 + 1, cl[c], s2 + 1, r, tau, e, &lists[j], stack, &sp);
                }
            }
        }
        visits[j] = v_count;
        total_visits += v_count;
        /* leaves arrive in traversal order; report them by leaf position */
        id_list *L = &lists[j];
        for (uint64_t x = 1; x < L->n; ++x) {
            uint32_t v = L->ids[x];
            uint64_t y = x;
            while (y > 0 && L->ids[y - 1] > v) {
                L->ids[y] = L->ids[y - 1];
                --y;
            }
            L->ids[y] = v;
        }
    }
    double t1 = now_seconds();
    or_cull_result *res = gather(lists, n_eyes, eye_ids, t);
    res->visits = visits;
    res->total_visits = total_visits;
    res->seconds = t1 - t0;
    res->threads = nt;
    return res;
}

or_cull_result *or_cull_hier(const or_tree *t, const float *eye_pos, const uint16_t *px,
                             const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                             const uint32_t *tile, uint32_t w, uint32_t h, float tau,
                             int nthreads)
{
    return or_cull_hier_w(t, eye_pos, px, py, eye_ids, n_eyes, tile, w, h, tau, 2, nthreads);
}

void or_cull_free(or_cull_result *res)
{
    if (!res)
        return;
    free(res->pairs);
    free(res->count);
    free(res->visits);
    free(res);
}

/* ------------------------------------------------------------------------------------ */
/* Connection evaluation: the step after the culling                                      */
/* ------------------------------------------------------------------------------------ */

/* An accepted connection carries the light's unoccluded contribution I / max(d^2, 1e-4)
 * divided by its acceptance probability p (Russian roulette keeps the sum over accepted
 * lights an unbiased estimate of the sum over all lights). d^2 and p are the acceptance
 * rule's own float32 values; every operation rounds to nearest, none is fused. */
void or_pair_weight(float tau, const float l[3], float intensity, const float e[3], float *weight, float *p_out)
{
    float dx = l[0] - e[0];
    float dy = l[1] - e[1];
    float dz = l[2] - e[2];
    float d2 = dx * dx;
    d2 = d2 + dy * dy;
    d2 = d2 + dz * dz;
    float den = fmaxf(d2, kMinDist2);
    float p = fminf(1.0f, (tau * intensity) / den);
    float base = intensity / den;
    *weight = base / p;
    if (p_out)
        *p_out = p;
}

static const float kSegTMin = 1e-4f, kSegTMax = 1.0f - 1e-4f;

/* Does the open segment e + t (l - e), t in (1e-4, 1 - 1e-4), cross the closed triangle
 * (v0, v1, v2)? Moller-Trumbore: with D = l - e, e1 = v1 - v0, e2 = v2 - v0, P = D x e2,
 * det = e1 . P, T = e - v0, Q = T x e1, the barycentrics are u = (T . P) / det and
 * v = (D . Q) / det and the ray parameter t = (e2 . Q) / det. det == 0 (segment parallel
 * to the plane) is no hit. float32, each product and sum rounded separately, dot products
 * summed x + y then + z, 1 / det rounded once. */
int or_segment_hits(const float e[3], const float l[3], const float tri[9])
{
    float D[3], e1[3], e2[3], T[3], P[3], Q[3];
    for (int c = 0; c < 3; ++c) {
        D[c] = l[c] - e[c];
        e1[c] = tri[3 + c] - tri[c];
        e2[c] = tri[6 + c] - tri[c];
        T[c] = e[c] - tri[c];
    }
    P[0] = D[1] * e2[2] - D[2] * e2[1];
    P[1] = D[2] * e2[0] - D[0] * e2[2];
    P[2] = D[0] * e2[1] - D[1] * e2[0];
    float det = e1[0] * P[0];
    det = det + e1[1] * P[1];
    det = det + e1[2] * P[2];
    if (det == 0.0f)
        return 0;
    float inv = 1.0f / det;
    float tp = T[0] * P[0];
    tp = tp + T[1] * P[1];
    tp = tp + T[2] * P[2];
    float u = tp * inv;
    if (!(u >= 0.0f && u <= 1.0f))
        return 0;
    Q[0] = T[1] * e1[2] - T[2] * e1[1];
    Q[1] = T[2] * e1[0] - T[0] * e1[2];
    Q[2] = T[0] * e1[1] - T[1] * e1[0];
    float dq = D[0] * Q[0];
    dq = dq + D[1] * Q[1];
    dq = dq + D[2] * Q[2];
    float v = dq * inv;
    if (!(v >= 0.0f && u + v <= 1.0f))
        return 0;
    float eq = e2[0] * Q[0];
    eq = eq + e2[1] * Q[1];
    eq = eq + e2[2] * Q[2];
    float t = eq * inv;
    return t > kSegTMin && t < kSegTMax;
}

/* Weight of every accepted pair (eye id, light id) times its visibility against all
 * triangles (brute force; n_tri = 0 means nothing occludes), and the per-eye sums in
 * double precision, added in pair order. */
void or_connect(const float *eye_pos, uint32_t n_eyes, const float *light_pos, const float *intensity,
                const uint32_t *pairs, uint64_t n_pairs, float tau, const float *tris, uint32_t n_tri,
                float *weight, uint8_t *visible, double *eye_sum, int nthreads)
{
    int nt = pick_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
    for (int64_t k = 0; k < (int64_t)n_pairs; ++k) {
        uint32_t j = pairs[2 * k], id = pairs[2 * k + 1];
        const float *e = &eye_pos[3 * (uint64_t)j], *l = &light_pos[3 * (uint64_t)id];
        float w;
        or_pair_weight(tau, l, intensity[id], e, &w, NULL);
        int vis = 1;
        for (uint32_t q = 0; q < n_tri && vis; ++q)
            if (or_segment_hits(e, l, &tris[9 * (uint64_t)q]))
                vis = 0;
        weight[k] = vis ? w : 0.0f;
        visible[k] = (uint8_t)vis;
    }
    for (uint32_t j = 0; j < n_eyes; ++j)
        eye_sum[j] = 0.0;
    for (uint64_t k = 0; k < n_pairs; ++k)
        eye_sum[pairs[2 * k]] += (double)weight[k];
}
