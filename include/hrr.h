/*
 * hrr.h - C ABI of the GB300 (sm_103a) library for blue-noise dithered QMC hierarchical
 * Russian roulette (Pantaleoni, "Blue-Noise Dithered QMC Hierarchical Russian Roulette").
 *
 * The problem (Sec. 1): eye vertices e_j, j in [0, N_e), and light vertices l_i sorted by
 * a hierarchy whose nodes are leaf ranges [a_n, b_n). Each eye owns a Cranley-Patterson
 * rotated base-2 radical-inverse sequence
 *     xi_j(i) = (Phi_2(i) + r_j) mod 1,
 * with its shift r_j read from a blue-noise tile at the eye's pixel. Light i is connected
 * to eye j iff xi_j(i) < p_ij (Russian roulette). A top-down traversal culls every
 * subtree whose range minimum v(a_n, b_n) = min_{i in [a_n,b_n)} xi_j(i) is at least a
 * conservative bound on p over the subtree, so the accepted set equals the brute-force
 * set over all N_e * N_l pairs while visiting a sub-linear number of nodes.
 *
 * Number formats (exact, no rounding anywhere in the sequence arithmetic):
 *   - A shift r is a uint32 fixed-point number r / 2^32; Phi_2(i) = brev32(i) / 2^32
 *     (Sec. 2, radical inverse); xi_j(i) = brev32(i) + r_j (mod 2^32) as a uint32.
 *   - The acceptance probability of a pair is the float32 expression
 *       p = fminf(1, (tau * I_i) / fmaxf(d2, 1e-4f)),  d2 = (dx*dx + dy*dy) + dz*dz,
 *     dx = l.x - e.x etc., every operation rounded to nearest, in that order, without
 *     fused multiply-add. Its fixed-point threshold is t = ceil(p * 2^32) in [0, 2^32]
 *     (t = 0 when p <= 0) and the pair is accepted iff xi < t.
 *   - The node bound uses the same expression with directed rounding (gap to the box
 *     and its squares and sums rounded down, numerator and quotient rounded up), so that
 *     it is never below the threshold of any light in the subtree.
 *
 * Conventions for every call:
 *   - Functions return an hrr_status. On failure hrr_last_error(ctx) describes it.
 *   - "device pointer" = memory on the context's GPU; the caller owns it and must keep it
 *     valid until the call's work on the context stream has completed.
 *   - All work is enqueued on the context stream. Calls that return a host-visible
 *     result (a count, an info field) synchronise that stream before returning; this is
 *     stated per call.
 *   - A context is not thread-safe: use one per host thread.
 *   - The library never frees caller memory and never keeps caller pointers after a
 *     call returns.
 */
#ifndef HRR_H
#define HRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hrr_status {
    HRR_OK = 0,
    HRR_ERR_INVALID_ARG = 1, /* bad pointer, size, value or handle */
    HRR_ERR_OOM = 2,         /* device or pinned-host allocation failed */
    HRR_ERR_NO_TILE = 3,     /* hrr_cull before hrr_set_shift_tile */
    HRR_ERR_OVERFLOW = 4,    /* output capacity too small; *out_count holds the need */
    HRR_ERR_TIMEOUT = 5,     /* a bounded device wait or queue wait ran out */
    HRR_ERR_CUDA = 6,        /* a CUDA runtime call failed */
    HRR_ERR_DEVICE = 7,      /* a kernel reported an internal error flag */
    HRR_PENDING = 8          /* a served job has not finished yet (not an error) */
} hrr_status;

typedef struct hrr_ctx hrr_ctx;   /* opaque, library-owned */
typedef struct hrr_tree hrr_tree; /* opaque, library-owned, device-resident */

/* Light vertices, device pointers, structure of arrays, n_lights entries each. Positions
 * are quantised for the spatial sort over the unit cube [0,1)^3 (values outside are
 * clamped to the border cells: still correct, only less coherent). All values must be
 * finite; intensities should be >= 0 (negative ones are never accepted). */
typedef struct hrr_lights {
    const float *x, *y, *z;
    const float *intensity;
} hrr_lights;

/* Eye vertices, device pointers, structure of arrays, n_eyes entries each. (px, py) is
 * the eye's pixel; its shift is tile[(py mod h) * w + (px mod w)] (Sec. 1). */
typedef struct hrr_eyes {
    const float *x, *y, *z;
    const uint16_t *px, *py;
} hrr_eyes;

/* Internal node record of the light hierarchy (64 bytes, 16-byte aligned). Internal
 * node n is a binary radix-tree node over the Morton-sorted leaves; its leaf range is
 * [min(n, other_end), max(n, other_end)] (inclusive) and it splits after leaf `split`:
 * child 0 covers [first, split], child 1 covers [split + 1, last]. A child whose range
 * has one leaf is that leaf; otherwise child 0 is internal node `split` and child 1 is
 * internal node `split + 1`. The record stores each child's bounding box and maximum
 * intensity (for a leaf child: its position, twice, and its intensity), so a traversal
 * tests both children from one fetch. The root is internal node 0. */
typedef struct hrr_node {
    float c0_lo[3];
    float c0_imax;
    float c0_hi[3];
    uint32_t split;
    float c1_lo[3];
    float c1_imax;
    float c1_hi[3];
    uint32_t other_end;
} hrr_node;

/* Optional knobs of a culling call; a NULL pointer means all defaults (zeros). */
typedef struct hrr_cull_opts {
    /* device pointer to n_eyes uint32, or NULL: receives the number of internal nodes
     * each eye visited (the root counts; a node is visited iff no ancestor culled it) */
    uint32_t *eye_visits;
    /* range-minimum variant, both with identical results: 0 = closed-form successor search
     * evaluated without branches (default), 2 = the same closed form with branches. (1 is
     * not accepted: the paper's Alg. 2 + 3, which the oracle restates, is not built into the
     * library; it is O(B^2) and 50x slower as a traversal's range minimum.) */
    int rangemin_variant;
    /* added (mod 2^32) to every eye's shift: the sample offset psi(n) of the adaptive
     * sampling variant (Sec. 3), absorbed into the shift; 0 for the plain method */
    uint32_t shift_offset;
    /* launch shape (results do not depend on it): resident blocks per SM of the
     * persistent grid, 0 = as many as fit (at most 64); see hrr_autotune */
    uint32_t blocks_per_sm;
    /* sample index n: selects layer n mod d of a space-time tile (hrr_set_shift_tile_3d);
     * 0 for a plain tile */
    uint32_t sample_index;
    /* traversal form (results do not depend on it; 0 = the library default for each, see
     * hrr_default_tuning: width 2, 256 ring entries, 256 threads, 6 top levels):
     *   node_width: 2 = binary records (a visit tests both children), 4 = the hierarchy read
     *     with nodes of width four (a visit tests the four grandchildren);
     *   ring_entries: stack entries per warp kept in shared memory, 128 or 256 for width 2,
     *     256 or 512 for width 4;
     *   threads_per_block: 128 or 256 (one eye per warp);
     *   top_levels: 1 = every level is walked from the root; 6 (width 2 only) = each block
     *     stages the top six levels of the hierarchy (63 nodes) in shared memory, and each
     *     eye first evaluates the 62 nodes below the root there in two warp-wide passes.
     *     The cull test is monotone (a child's smaller box, smaller maximum intensity and
     *     larger range minimum never turn its parent's cull into a visit), so a node below
     *     the root is visited iff its own test passes, and those levels need not be walked
     *     one level per step. Batched launches of several frames read each frame's top
     *     slots from global memory instead. */
    uint32_t node_width;
    uint32_t ring_entries;
    uint32_t threads_per_block;
    uint32_t top_levels;
} hrr_cull_opts;

/* Launch parameters of the traversal (see hrr_cull_opts); none changes any result. Zero
 * fields take the library defaults. */
typedef struct hrr_tuning {
    int rangemin_variant;
    uint32_t blocks_per_sm;
    uint32_t node_width;
    uint32_t ring_entries;
    uint32_t threads_per_block;
    uint32_t top_levels;
} hrr_tuning;

/* The tuning the library uses for zero fields (rangemin_variant 0, blocks_per_sm 0 = as many
 * as fit, and the default node width, ring size, threads per block and top levels). */
int hrr_default_tuning(hrr_tuning *out);

/* ---- context --------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`. cuda_stream is a cudaStream_t on that device
 * (for example torch.cuda.current_stream().cuda_stream) or NULL for a stream owned by the
 * context. Allocates a few bytes of device counters and pinned host memory. */
int hrr_create(hrr_ctx **out, int device, void *cuda_stream);
/* Waits for the context stream, then releases the context (not trees built with it). */
int hrr_destroy(hrr_ctx *ctx);
/* Text of the last error on this context ("" if none). Valid until the next call. */
const char *hrr_last_error(const hrr_ctx *ctx);
/* Static name of a status code. */
const char *hrr_status_string(int status);
/* Number of kernels this context has launched so far. */
int hrr_launch_count(const hrr_ctx *ctx, uint64_t *out);
/* Enable (1) or disable (0) CUDA-event timing of the traversal kernel on the context
 * stream; hrr_kernel_time returns the summed device time (ms) and launch count since it
 * was enabled, synchronising the stream. */
int hrr_set_timing(hrr_ctx *ctx, int enable);
int hrr_kernel_time(hrr_ctx *ctx, double *ms, uint64_t *launches);

/* ---- light hierarchy (Sec. 1: lights sorted by a hierarchy of leaf ranges) -------------- */

/* Build the light hierarchy: 63-bit Morton keys (21 bits per axis, cell =
 * floor(x * 2^21) clamped to [0, 2^21 - 1]; bit k of the x, y, z cells at key bits
 * 3k+2, 3k+1, 3k), a stable radix sort by (key, original index), a binary radix tree over
 * (key, sorted position), and a bottom-up refit of boxes and maximum intensities. Leaf
 * i of the tree is the i-th light in sorted order; i is the index of the radical-inverse
 * sequence (Sec. 1: spatially sorted lights inherit the sequence's stratification).
 * 1 <= n_lights <= 2^31 - 1. Synchronises the context stream; returns
 * HRR_ERR_INVALID_ARG if any position or intensity is not finite. */
int hrr_build_light_tree(hrr_ctx *ctx, hrr_lights lights, uint32_t n_lights, hrr_tree **out);

/* Hierarchy shapes over the same Morton leaf order (so the same accepted set, Sec. 1):
 * RADIX splits every range at the highest differing bit of its end keys (a binary radix
 * tree); COST splits each range down to depth cost_depth (root = 1) where w(L) + w(R) is
 * least, w(X) = u^2 ((A + 0.1 P) + 1e-4) c sqrt(c) for a child of c lights whose maximum
 * intensity (clamped at 0) is u times the range's, A = dx dy + dy dz + dz dx and
 * P = dx + dy + dz of its box (float, each operation rounded separately; every split a
 * candidate; ties to the most even split, then the smaller one), and takes radix splits
 * below, which bound the height by cost_depth + 96. COST trees take fewer node visits to
 * cull (about 15% on the frame workload) and about a millisecond more to build. */
typedef enum hrr_topology { HRR_TOPOLOGY_RADIX = 0, HRR_TOPOLOGY_COST = 1 } hrr_topology;

typedef struct hrr_build_opts {
    int topology;        /* hrr_topology */
    uint32_t cost_depth; /* COST: 1..64, the deepest level split by cost; 0 = 48 */
} hrr_build_opts;

/* hrr_build_light_tree with options (NULL: the defaults, a radix tree). HRR_ERR_INVALID_ARG
 * for an unknown topology or a cost_depth above 64. */
int hrr_build_light_tree_ex(hrr_ctx *ctx, hrr_lights lights, uint32_t n_lights, const hrr_build_opts *opts,
                            hrr_tree **out);

/* hrr_build_light_tree_ex with the lights in host memory (host SoA, n_lights entries each):
 * the library copies them into a device staging area of the context (16 bytes a light,
 * grown on demand, freed by hrr_destroy) on the context stream, then builds as
 * hrr_build_light_tree_ex does. Pinned host memory lets the copies run at full bandwidth.
 * Synchronous; statuses as hrr_build_light_tree_ex. */
int hrr_build_light_tree_host(hrr_ctx *ctx, hrr_lights host_lights, uint32_t n_lights, const hrr_build_opts *opts,
                              hrr_tree **out);

/* Moved lights (the same lights, new positions and intensities; device SoA of the tree's
 * n lights, indexed by original light id): refit `tree` in place. The leaf order and the
 * topology of the build stay, so a light keeps its sequence index i (its position in the
 * build's Morton order, Sec. 1) and culling equals flat culling over that order; the boxes
 * and maximum intensities are recomputed. Synchronous. HRR_ERR_INVALID_ARG if a value is
 * not finite (the tree is then unchanged). The tree must not be in use by work in flight. */
int hrr_refit_light_tree(hrr_ctx *ctx, hrr_tree *tree, hrr_lights lights);
/* Release a hierarchy (stream-ordered on ctx). */
int hrr_free_light_tree(hrr_ctx *ctx, hrr_tree *tree);
/* Device pointer to the sorted-leaf -> original light id permutation (n_lights entries). */
int hrr_tree_perm(const hrr_tree *tree, const uint32_t **dev_perm);
/* Size facts of a hierarchy: lights, height (internal nodes on the longest root-to-leaf
 * path; 0 for one light), device pointer to its n_lights - 1 node records (NULL for one
 * light). Any output pointer may be NULL. */
int hrr_tree_info(const hrr_tree *tree, uint32_t *n_lights, uint32_t *height,
                  const hrr_node **dev_nodes);
/* Copy the node records and the permutation to host memory (n_lights - 1 records and
 * n_lights ids; either pointer may be NULL). Synchronises the context stream. */
int hrr_tree_download(hrr_ctx *ctx, const hrr_tree *tree, hrr_node *host_nodes,
                      uint32_t *host_perm);

/* Build a hierarchy without allocating any memory. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc. Examples are a renderer
 * whose device memory is owned by its own pool, a real-time thread where an allocation
 * may stall the device, or code that must run in a fixed memory footprint. The result is
 * the same hierarchy as hrr_build_light_tree's: n_lights - 1 node records written to
 * dev_nodes (one record holding the single leaf when n_lights == 1) and the
 * sorted-leaf -> original id permutation written to dev_perm (n_lights entries), both
 * device memory the caller owns. *out_height (may be NULL) receives the height.
 *   - Working memory is one library-wide static device array sized for
 *     HRR_STATIC_BUILD_MAX_LIGHTS lights (about 3.6 MiB), which every GPU that loads
 *     the library keeps until the process exits. Larger n_lights is rejected with
 *     HRR_ERR_INVALID_ARG.
 *   - Runs on the calling thread's current device, on cuda_stream (NULL = the legacy
 *     default stream), and synchronises that stream before returning.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, which may load the library's GPU code); make that first
 *     call before any stream capture. The address is kept for the life of the process:
 *     after a cudaDeviceReset of a device, do not call this entry point on it again.
 *   - All calls on a device share the array: calls whose GPU work overlaps (for
 *     example on two streams) race and produce garbage. Serialise them.
 *   - err (may be NULL) receives a message of at most err_len bytes on failure. */
#define HRR_STATIC_BUILD_MAX_LIGHTS 65536u
int hrr_build_light_tree_static(hrr_lights lights, uint32_t n_lights, hrr_node *dev_nodes,
                                uint32_t *dev_perm, uint32_t *out_height, void *cuda_stream,
                                char *err, size_t err_len);

/* ---- shifts (Sec. 1: blue-noise dithered Cranley-Patterson rotations) ------------------- */

/* Copy a w x h tile of uint32 shifts (row-major, host memory) into the context. The
 * eye at pixel (px, py) uses tile[(py mod h) * w + (px mod w)]. 1 <= w, h <= 65536.
 * Synchronises the context stream. Same as hrr_set_shift_tile_3d with d = 1. */
int hrr_set_shift_tile(hrr_ctx *ctx, const uint32_t *host_tile, uint32_t w, uint32_t h);

/* A space-time tile psi(j, n) (Sec. 3): d layers of w x h shifts (layer-major, then
 * row-major). Sample n of the eye at pixel (px, py) uses
 * tile[((n mod d) * h + (py mod h)) * w + (px mod w)]; the sample index n is the
 * sample_index of hrr_cull_opts, hrr_frame or hrr_job. 1 <= w, h <= 65536, 1 <= d <= 65536,
 * w * h * d <= 2^30. Synchronises the context stream. */
int hrr_set_shift_tile_3d(hrr_ctx *ctx, const uint32_t *host_tile, uint32_t w, uint32_t h, uint32_t d);

/* ---- culling (Sec. 1: hierarchical Russian roulette with QMC sequences) ----------------- */

/* Cull all eye x light connections. Writes the accepted pairs to dev_pairs as
 * (eye index j, original light id) uint32 pairs, 2 * cap uint32 of device memory, in no
 * particular order; sets *out_count to the number of accepted pairs. If that number
 * exceeds cap, returns HRR_ERR_OVERFLOW (the first cap slots hold some accepted pairs,
 * unspecified which) and the caller may retry with a larger buffer. tau >= 0 and finite.
 * n_eyes may be 0. Synchronises the context stream (to read the count). */
int hrr_cull(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
             uint32_t *dev_pairs, uint64_t cap, uint64_t *out_count);
/* hrr_cull with options (see hrr_cull_opts). opts may be NULL. */
int hrr_cull_ex(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree,
                float tau, const hrr_cull_opts *opts, uint32_t *dev_pairs, uint64_t cap,
                uint64_t *out_count);
/* Several samples per light in one traversal (Sec. 3: n samples per light with shifts
 * r_j + psi(n), and space-time shifts psi(j, n)). Sample s of eye j uses the shift
 * tile_s[pixel of j] + offsets[s] (mod 2^32), where tile_s is layer s mod d of the context
 * tile (the tile itself when it has one layer); its pairs are exactly those hrr_cull_ex
 * gives with shift_offset = offsets[s] and sample_index = s. One traversal per eye visits
 * the union of the samples' nodes and fetches each record once. n_samples in [1, 32];
 * offsets: host array of n_samples. dev_pairs: n_samples * cap pairs (2 uint32 each,
 * 8-byte aligned), sample s's pairs at dev_pairs + 2 * cap * s, as (eye index, original
 * light id) in unspecified order. out_counts: host array of n_samples, sample s's count.
 * out_visits: NULL or a host array of 2: the node visits summed over the samples (equal
 * to the total of hrr_cull_ex over the samples) and the node records fetched.
 * HRR_ERR_OVERFLOW if a sample's count exceeds cap (its first cap pairs are written).
 * Synchronous. */
int hrr_cull_samples(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                     const uint32_t *offsets, uint32_t n_samples, uint32_t *dev_pairs, uint64_t cap,
                     uint64_t *out_counts, uint64_t *out_visits);

/* hrr_cull with host buffers: the eyes are read from host memory (host_eyes: host SoA,
 * n_eyes entries each) and the accepted pairs written to host memory (host_pairs: 2 * cap
 * uint32), as (eye index, original light id) with the same set as hrr_cull_ex gives for the
 * same eyes and options. Pinned host memory lets the copies overlap the culling: the eyes
 * are culled in up to eight slices of at least about 2^18 eyes, launched alternately on the
 * context stream and a second stream so that consecutive slices overlap; each slice's eyes
 * are copied in ahead of it and its pairs copied out while the next slice runs. The
 * context keeps device copies of the eyes and two pair buffers of cap pairs (grown on
 * demand, freed by hrr_destroy), a second stream and a copy stream. Statuses as in
 * hrr_cull_ex (HRR_ERR_OVERFLOW: *out_count holds the need, the first cap pairs of the
 * buffer are written). opts may be NULL; its eye_visits, if set, is device memory.
 * Synchronous. */
int hrr_cull_host(hrr_ctx *ctx, hrr_eyes host_eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                  const hrr_cull_opts *opts, uint32_t *host_pairs, uint64_t cap, uint64_t *out_count);
/* Statistics of the last hrr_cull/hrr_cull_ex on this context: total internal-node
 * visits and accepted pairs (both exact, computed on the device). */
int hrr_last_cull_stats(const hrr_ctx *ctx, uint64_t *visits, uint64_t *accepted);

/* Roofline denominators measured on this GPU (not from the paper; measurement only). */
typedef struct hrr_peaks {
    double l2_read_gbs;          /* streaming 128-bit reads of a 32 MiB L2-resident buffer */
    double record_fetches_per_s; /* 64-byte records at random indices of a 64 MiB L2-resident
                                    array, each as two 256-bit loads (the traversal's fetch) */
    double int_ops_per_s;        /* independent 32-bit lop3 / add chains, 8 per thread */
} hrr_peaks;

/* Run the three microbenchmarks on the context stream (best of five timed launches of a
 * few milliseconds each, about 60 ms in all) and fill *out. Allocates and frees 64 MiB of
 * device memory. Synchronous. */
int hrr_measure_peaks(hrr_ctx *ctx, hrr_peaks *out);

/* ---- batched culling (many frames in one persistent launch) ---------------------------- */

/* One frame of a batch: its eyes, hierarchy, shifts, culling scale and output. Pairs are
 * written as (eye index within the frame, original light id), as in hrr_cull. */
typedef struct hrr_frame {
    hrr_eyes eyes;              /* device SoA, n_eyes entries */
    uint32_t n_eyes;            /* may be 0 */
    const hrr_tree *tree;       /* built on the batch's context device */
    const uint32_t *dev_tile;   /* device tile_w x tile_h shifts, or NULL for the context tile */
    uint32_t tile_w, tile_h;
    float tau;                  /* finite, >= 0 */
    uint32_t shift_offset;      /* as in hrr_cull_opts */
    uint32_t *dev_pairs;        /* 2 * cap uint32 of device memory, 8-byte aligned */
    uint64_t cap;
    uint32_t *eye_visits;       /* optional per-eye visit counts (device, n_eyes), or NULL */
    uint32_t tile_d;            /* layers of dev_tile (0 means 1); ignored for the context tile */
    uint32_t sample_index;      /* layer sample_index mod d of the frame's tile */
} hrr_frame;

typedef struct hrr_batch hrr_batch; /* opaque, library-owned */

/* Prepare a batch of 1..65535 frames for repeated culling: validates the frames, uploads
 * their descriptors and per-frame counters to the device and, when use_graph != 0, records
 * the launch (counter reset + one persistent traversal over every frame's eyes) into a
 * CUDA graph. tuning may be NULL (defaults). The frames' memory must stay valid while the
 * batch exists. Frames without a tile read the context's tile as it is now: the batch keeps
 * a reference to it, so a later hrr_set_shift_tile does not change (or free) what the batch
 * reads. Destroy a batch before its context. Synchronous.
 * Status HRR_ERR_NO_TILE if a frame has no tile and the context has none. */
int hrr_batch_create(hrr_ctx *ctx, const hrr_frame *frames, uint32_t n_frames,
                     const hrr_tuning *tuning, int use_graph, hrr_batch **out);
/* Enqueue one run of the batch on the context stream (a graph replay when recorded).
 * Asynchronous. */
int hrr_batch_launch(hrr_ctx *ctx, hrr_batch *batch);
/* Wait for the last run and copy its per-frame accepted-pair counts and node visits to
 * host arrays of n_frames (either may be NULL). HRR_ERR_OVERFLOW if any frame's count
 * exceeds its cap (its count is still reported). */
int hrr_batch_results(hrr_ctx *ctx, hrr_batch *batch, uint64_t *counts, uint64_t *visits);
/* Wait for the context stream and release the batch. */
int hrr_batch_destroy(hrr_ctx *ctx, hrr_batch *batch);
/* One-shot batch: create (no graph), launch, results, destroy. */
int hrr_cull_batch(hrr_ctx *ctx, const hrr_frame *frames, uint32_t n_frames,
                   const hrr_tuning *tuning, uint64_t *counts);

/* ---- served culling (continuous batching) --------------------------------------------- */

/* A culling job: eyes against a device-resident hierarchy and tile. The server reserves
 * cap output pairs for it. All pointers must stay valid until the job is released. A job
 * without a tile reads the submitting context's tile as it is at submission; the job keeps
 * a reference to it until hrr_server_release, so a later hrr_set_shift_tile on that
 * context does not change (or free) the job's tile. */
typedef struct hrr_job {
    hrr_eyes eyes;              /* device SoA */
    uint32_t n_eyes;
    const hrr_tree *tree;       /* built on the server's device, kept resident by the caller */
    const uint32_t *dev_tile;   /* device tile, or NULL for the submitting context's tile */
    uint32_t tile_w, tile_h;
    float tau;
    uint32_t shift_offset;
    uint64_t cap;               /* output pairs to reserve */
    uint32_t tile_d;            /* layers of dev_tile (0 means 1); ignored for the context tile */
    uint32_t sample_index;      /* layer sample_index mod d of the job's tile */
    /* moved lights for this frame, or all NULL: the server refits `tree` to them (as
     * hrr_refit_light_tree does) in the job's stream before its first eyes, once every job
     * submitted earlier that reads the same tree is done; jobs submitted later see the
     * refitted tree. A light that is not finite fails the job with HRR_ERR_INVALID_ARG and
     * leaves the tree unchanged. With refit set the server writes `tree` (const above
     * because other jobs only read it). */
    hrr_lights refit;
} hrr_job;

typedef struct hrr_job_result {
    int status;                 /* HRR_PENDING, HRR_OK, HRR_ERR_OVERFLOW (count > cap; the
                                   buffer holds cap of the pairs), HRR_ERR_OOM (the job's
                                   reservation exceeds the budget), HRR_ERR_DEVICE */
    uint64_t count;             /* accepted pairs */
    uint64_t visits;            /* internal-node visits */
    const uint32_t *dev_pairs;  /* server-owned device buffer of min(count, cap) pairs
                                   (eye index within the job, original light id), valid
                                   until hrr_server_release */
    double queue_s;             /* submission to admission (so far, while waiting) */
    double latency_s;           /* submission to completion (so far, while pending) */
} hrr_job_result;

typedef struct hrr_server_info {
    uint64_t slices, launches, jobs_done, jobs_waiting, jobs_active, bytes_reserved;
    uint32_t max_active;        /* most jobs admitted at once so far */
} hrr_server_info;

typedef struct hrr_server hrr_server; /* opaque, library-owned */

/* Start a server on ctx's device with its own stream and scheduler thread. Jobs are
 * admitted in arrival order while their output reservations (cap * 8 bytes) fit in
 * hbm_budget_bytes and fewer than max_jobs are admitted; the GPU then runs slices, each
 * one batched traversal over up to slice_eyes (0: 2^20) of the admitted jobs' remaining
 * eyes, oldest job first, so jobs arriving while others run join a slice as soon as the
 * older jobs leave room. Each job's result is exactly what hrr_cull would produce for it
 * alone. Slices alternate between two streams so that each one's tail overlaps the next.
 * Job outputs come from a memory pool of the server that keeps freed memory up to the
 * budget. The server never makes the GPU wait on the host. tuning may be NULL (defaults). */
int hrr_server_create(hrr_ctx *ctx, uint64_t hbm_budget_bytes, uint32_t slice_eyes,
                      uint32_t max_jobs, const hrr_tuning *tuning, hrr_server **out);
/* Queue a job (thread-safe, non-blocking); *ticket identifies it. ctx (may be NULL when the
 * job has its own tile) receives the error text of a rejected job. */
int hrr_server_submit(hrr_server *server, hrr_ctx *ctx, const hrr_job *job, uint64_t *ticket);
/* HRR_OK with the result when the job has finished, HRR_PENDING otherwise (non-blocking). */
int hrr_server_poll(hrr_server *server, uint64_t ticket, hrr_job_result *result);
/* Block until the job finishes (HRR_OK) or timeout_s passes (HRR_ERR_TIMEOUT). */
int hrr_server_wait(hrr_server *server, uint64_t ticket, double timeout_s, hrr_job_result *result);
/* Copy up to max_pairs of a finished job's pairs (min(count, cap) are stored) to host
 * memory; *copied receives the number copied. Synchronous. */
int hrr_server_copy_pairs(hrr_server *server, uint64_t ticket, uint32_t *host_pairs,
                          uint64_t max_pairs, uint64_t *copied);
/* Free a finished job's output buffer and reservation; the ticket becomes invalid. */
int hrr_server_release(hrr_server *server, uint64_t ticket);
/* Counters of the scheduler. */
int hrr_server_stats(hrr_server *server, hrr_server_info *info);
/* Finish every submitted job, stop the scheduler and free everything the server owns. */
int hrr_server_destroy(hrr_server *server);

/* ---- autotuning ---------------------------------------------------------------------- */

/* Time every compiled form of the traversal on the given eyes (a sample of a workload's
 * size class): range-minimum variants 0 and 2, node widths 2 and 4, both ring sizes of
 * each width, 128 and 256 threads per block, each at the most resident blocks per SM that
 * fit and at one block fewer. Fills tried[k] and tried_ms[k] (median of three timed runs
 * after a warm-up) for k < *n_tried, in a fixed order. capacity is the length of both
 * arrays; if it is too small (or an array is NULL) nothing is timed, *n_tried receives the
 * number needed and the call returns HRR_ERR_INVALID_ARG. dev_pairs / cap as in hrr_cull
 * and large enough for the sample. Results of every candidate are identical; only the time
 * differs. Synchronous. */
int hrr_autotune_all(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                     uint32_t *dev_pairs, uint64_t cap, hrr_tuning *tried, double *tried_ms,
                     uint32_t capacity, uint32_t *n_tried);
/* hrr_autotune_all, keeping the fastest candidate in *best (its median time in *best_ms,
 * may be NULL). */
int hrr_autotune(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, const hrr_tree *tree, float tau,
                 uint32_t *dev_pairs, uint64_t cap, hrr_tuning *best, double *best_ms);

/* ---- connection evaluation (after the culling) --------------------------------------- */

typedef struct hrr_scene hrr_scene; /* opaque, library-owned: a triangle hierarchy */

/* Build a bounding-volume hierarchy over n_tris triangles (device memory, 9 floats each:
 * v0, v1, v2), copied into the scene. 1 <= n_tris <= 2^31 - 1. Synchronous.
 * HRR_ERR_INVALID_ARG if a vertex is not finite. */
int hrr_build_scene(hrr_ctx *ctx, const float *dev_tris, uint32_t n_tris, hrr_scene **out);
int hrr_free_scene(hrr_ctx *ctx, hrr_scene *scene);

/* Evaluate accepted connections (the step after the culling, Sec. 1): for each of the
 * n_pairs pairs (eye index, light id) in dev_pairs (as hrr_cull writes them), the
 * Russian-roulette weight (I / max(d^2, 1e-4)) / p, with d^2 and p the acceptance rule's
 * float32 values, times the visibility of the open segment eye -> light (t in
 * (1e-4, 1 - 1e-4)) against the scene's triangles (scene NULL: every connection is
 * visible). Writes the weights (dev_weight, n_pairs floats, may be NULL), the visibility
 * bits (dev_visible, n_pairs bytes, may be NULL) and the per-eye sums (dev_eye_sum, n_eyes
 * floats, zeroed first; float atomics, so the last bits depend on the order). lights are
 * the SoA indexed by original light id. Synchronous. HRR_ERR_INVALID_ARG if a pair's index
 * is out of range. */
int hrr_connect(hrr_ctx *ctx, hrr_eyes eyes, uint32_t n_eyes, hrr_lights lights, uint32_t n_lights,
                float tau, const uint32_t *dev_pairs, uint64_t n_pairs, const hrr_scene *scene,
                float *dev_weight, uint8_t *dev_visible, float *dev_eye_sum);

/* ---- range minimum (Sec. 2) ----------------------------------------------------------- */

/* For q in [0, n): out_min[q] = min_{i in [a[q], b[q])} (brev32(i) + r[q]) mod 2^32 and
 * out_argmin[q] = the unique index attaining it (v(a,b) and k of Sec. 1-2 in 32-bit fixed
 * point). Device pointers; out_argmin may be NULL. An empty range (a >= b) gives
 * out_min = 0xFFFFFFFF and out_argmin = 0xFFFFFFFF. variant (0 or 2) as in
 * hrr_cull_opts; any other value is HRR_ERR_INVALID_ARG.
 * Asynchronous (no stream synchronisation). */
int hrr_range_min(hrr_ctx *ctx, const uint32_t *a, const uint32_t *b, const uint32_t *r,
                  uint32_t *out_min, uint32_t *out_argmin, uint64_t n, int variant);

#ifdef __cplusplus
}
#endif
#endif /* HRR_H */
