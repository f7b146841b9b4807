/*
 * CPU oracle for blue-noise dithered QMC hierarchical Russian roulette (Pantaleoni,
 * "Blue-Noise Dithered QMC Hierarchical Russian Roulette").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this
 * code: it exists so that tests, the smoke check and the benchmark's CPU baseline can
 * compare the CUDA library against a plain, slow, independently written restatement of
 * the paper. It shares no code, header or constant table with the CUDA library.
 *
 * Conventions (B-bit words; the library uses B = 32):
 *  - Phi_2(i) = brev_B(i) / 2^B for i < 2^B (Sec. 2, radical inverse definition).
 *  - A shift r is a B-bit fixed-point number r / 2^B; the shifted sequence value of
 *    index i is xi(i) = (brev_B(i) + r) mod 2^B (Sec. 1, Cranley-Patterson rotation).
 *  - Ranges are half-open [a, b) with 0 <= a < b <= 2^B.
 *  - The threshold 1 - r of the three-case split (Sec. 2) is T = (2^B - r) mod 2^B.
 */
#ifndef HRR_ORACLE_H
#define HRR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- radical inverse and range minimum (Sec. 2) ---- */
uint32_t or_brev(uint32_t x, int B);
/* Linear scan: the definition of v(a,b) and its argmin (Sec. 1, Sec. 2). */
uint32_t or_rangemin_scan(uint64_t a, uint64_t b, uint32_t r, int B, uint64_t *argmin);
/* The scan with 32-bit words, the reversed index updated from one index to the next
 * (brev(i) and brev(i - 1) differ in their top ctz(i) + 1 digits); a < b. */
uint32_t or_rangemin_scan_inc(uint64_t a, uint64_t b, uint32_t r, uint64_t *argmin);
/* Successor search in the binary trie of {brev(i) : i in [a,b)}: independent of Alg. 2. */
uint32_t or_rangemin_trie(uint64_t a, uint64_t b, uint32_t r, int B, uint64_t *argmin);
/* Alg. 1: the index in [a,b) with the most trailing zeros (the unshifted argmin). */
uint64_t or_alg1(uint64_t a, uint64_t b, int B);
/* Alg. 2 with Alg. 3 exactly as the paper states them (wrong for some a = 0 ranges). */
uint64_t or_alg2_printed(uint64_t a, uint64_t b, uint32_t r, int B);
/* Alg. 2 with the a = 0 reading: fall back to Alg. 1 when the result is invalid. */
uint64_t or_alg2_fixed(uint64_t a, uint64_t b, uint32_t r, int B);
/* Batched range minimum with B-bit words (b <= 2^B - 1 when B = 32). method: 0 scan,
 * 1 trie, 2 Alg. 2 fixed, 3 Alg. 2 printed, 4 Alg. 1 (r ignored), 5 the incremental scan. The index returned by
 * methods 3 and 4 may lie outside [a,b) when the algorithm fails; its value is still
 * reported. argmin may be NULL. nthreads <= 0 uses every available thread. */
void or_rangemin_batch(const uint32_t *a, const uint32_t *b, const uint32_t *r, uint64_t n,
                       int method, int B, uint32_t *vmin, uint32_t *argmin, int nthreads);

/* ---- directed rounding primitives (exposed so tests can pin them) ---- */
/* op: 0 add, 1 sub, 2 mul, 3 div; mode: -1 toward -inf, 0 nearest, +1 toward +inf */
float or_fround(int op, float x, float y, int mode);
/* x y + z rounded once toward -inf (a fused multiply-add rounded down). */
float or_fma_rd(float x, float y, float z);

/* ---- acceptance thresholds (float32, canonical operation order) ---- */
/* t_ij = ceil(p_ij * 2^32), p_ij = min(1, (tau*I) / max(d^2, 1e-4)), round to nearest. */
uint64_t or_leaf_threshold(float tau, const float l[3], float intensity, const float e[3]);
/* Conservative cull test: 1 only if v >= t_ij for every light in the box [lo,hi] with
 * intensity <= imax (v: minimum of the eye's shifted sequence over the node's range). */
int or_node_culls(float tau, const float lo[3], const float hi[3], float imax, const float e[3],
                  uint32_t v);

/* ---- light hierarchy ---- */
uint64_t or_morton(float x, float y, float z);

typedef struct or_tree {
    uint32_t n;          /* lights */
    uint32_t height;     /* internal nodes on the longest root-to-leaf path */
    uint32_t *perm;      /* sorted leaf i -> original light id */
    uint64_t *key;       /* Morton key of sorted leaf i */
    float *pos;          /* sorted positions, 3 per leaf */
    float *inten;        /* sorted intensities */
    /* internal nodes, numbered as in a binary radix tree (root 0; the children of a
     * node split at s are s and s+1, each a leaf when its range has one element) */
    uint32_t *first, *last, *split;
    float *lo, *hi;      /* 3 per internal node */
    float *imax;
} or_tree;

or_tree *or_tree_build(const float *pos, const float *intensity, uint32_t n);
/* The same leaf order with cost-driven splits down to depth cost_depth (0: 48), radix
 * splits below. */
or_tree *or_tree_build_cost(const float *pos, const float *intensity, uint32_t n, uint32_t cost_depth);
void or_tree_free(or_tree *t);
/* New positions (3 per light) and intensities for the same lights (indexed by original id):
 * the leaf order and topology stay, boxes and maximum intensities are recomputed. */
void or_tree_refit(or_tree *t, const float *pos, const float *intensity);

/* ---- culling ---- */
typedef struct or_cull_result {
    uint64_t n_pairs;
    uint32_t *pairs;       /* 2*n_pairs: (eye id, original light id), by eye then leaf */
    uint32_t *count;       /* accepted per eye (n_eyes) */
    uint64_t *visits;      /* internal nodes visited per eye (hierarchical only) */
    uint64_t total_visits;
    uint64_t n_marginal;   /* pairs with |xi/2^32 - p| < 1e-6 p, p in double (flat only) */
    double seconds;
    int threads;
} or_cull_result;

/* eyes: pos (n_eyes*3), px, py; eye_ids (may be NULL -> 0..n_eyes-1) label the output.
 * tile: w*h shifts, r_j = tile[(py mod h)*w + (px mod w)]. */
or_cull_result *or_cull_flat(const or_tree *t, const float *eye_pos, const uint16_t *px,
                             const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                             const uint32_t *tile, uint32_t w, uint32_t h, float tau,
                             int nthreads);
or_cull_result *or_cull_hier(const or_tree *t, const float *eye_pos, const uint16_t *px,
                             const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                             const uint32_t *tile, uint32_t w, uint32_t h, float tau,
                             int nthreads);
/* The same traversal over the tree read with nodes of width 2 (each visit tests two
 * children, as or_cull_hier) or 4 (each visit tests the grandchildren, and leaf children;
 * only even-depth nodes are visited): the same accepted set, visits counted per node of
 * that width. */
or_cull_result *or_cull_hier_w(const or_tree *t, const float *eye_pos, const uint16_t *px,
                               const uint16_t *py, const uint32_t *eye_ids, uint32_t n_eyes,
                               const uint32_t *tile, uint32_t w, uint32_t h, float tau, int width,
                               int nthreads);
void or_cull_free(or_cull_result *res);

int or_max_threads(void);

/* ---- connection evaluation (after the culling) ---- */
/* weight = (I / max(d^2, 1e-4)) / p of one accepted connection; p the acceptance
 * probability (p_out may be NULL). */
void or_pair_weight(float tau, const float l[3], float intensity, const float e[3], float *weight, float *p_out);
/* 1 iff the open segment e -> l (t in (1e-4, 1 - 1e-4)) crosses the closed triangle
 * tri = (v0, v1, v2), 9 floats (Moller-Trumbore in float32). */
int or_segment_hits(const float e[3], const float l[3], const float tri[9]);
/* Per accepted pair (eye id, light id): weight times visibility against n_tri triangles
 * (brute force), the visibility bit, and per-eye sums (double, in pair order). */
void or_connect(const float *eye_pos, uint32_t n_eyes, const float *light_pos, const float *intensity,
                const uint32_t *pairs, uint64_t n_pairs, float tau, const float *tris, uint32_t n_tri,
                float *weight, uint8_t *visible, double *eye_sum, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
