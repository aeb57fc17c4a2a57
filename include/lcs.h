/*
 * lcs.h -- C ABI of the GB300 (sm_103a) DIST hot path of the Lu-Lin parallel
 * LCS method, as implemented in "Parallel Longest Common SubSequence
 * Analysis In Chapel" (arXiv 2309.09072).
 *
 * Problem (Sec. I, Sec. II-A, Fig. 1).  String a (length m) labels the rows
 * and string b (length n) the columns of a grid graph with (m+1) x (n+1)
 * vertices; right and down edges weigh 0 and the diagonal edge into vertex
 * (r, c) weighs 1 iff a_r = b_c.  With top and bottom boundary vertices
 * numbered 0..n,
 *
 *     DIST(i, j) = heaviest path from top vertex i to bottom vertex j
 *                = LCS(a, b[i:j])                for j >= i,
 *     DIST(i, j) = -infinity (the sentinel)      for j <  i,
 *
 * and LCS(a, b) = DIST(0, n).  The library builds DIST strip by strip (rows
 * of a in groups of h), combines strips up a binary tree with the (max,+)
 * product D(i, j) = max_k U(i, k) + L(k, j) (Sec. II-A, Sec. II-B-1) taken
 * under the Monge bound K(i, j-1) <= K(i, j) <= K(i+1, j), and walks the
 * leftmost maximisers K back down the tree to one LCS (Sec. II-C..II-E).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an lcs_status and never throws or aborts.
 *  - Pointers named *_host are host pointers; all other buffer pointers are
 *    DEVICE pointers on the context's device.  The caller owns every buffer
 *    it passes; the library never frees caller memory.  The context owns its
 *    workspace (device memory it allocates itself, within the budget given to
 *    lcs_create).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device-only calls are asynchronous on that stream; calls that
 *    return a value through a *_host pointer synchronise it first.
 *  - Dense DIST matrices are (n+1) x ld, row-major: row i = top vertex i,
 *    column j = bottom vertex j.  ld is in elements, ld >= n+1, ld times the
 *    element size is a multiple of 16 bytes, and the base is 16-byte aligned.
 *    The lower triangle (j < i) holds the sentinel INT32_MIN (LCS_I32) or
 *    INT16_MIN (LCS_I16).
 *  - Rows belong to the first string `a`.  The orientation is part of the
 *    contract: it decides which of several optimal LCS strings is returned.
 *  - Empty strings are legal: the length is 0 and DIST has 0 on and above
 *    the diagonal.
 *  - A context is not re-entrant: use one per host thread or serialise.
 *  - Results are exact integers and independent of strip height, tile shape
 *    and schedule: every maximiser is the smallest one (ties go to the lower
 *    index, as the "<=" comparison of Algorithm 2 does).
 */
#ifndef LCS_GB300_H
#define LCS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lcs_ctx lcs_ctx;

typedef enum {
    LCS_OK = 0,
    LCS_EINVAL = 1,     /* an argument is out of range, misaligned or NULL      */
    LCS_ENOMEM = 2,     /* the workspace would exceed the budget / cudaMalloc failed */
    LCS_ETIMEOUT = 3,   /* a bounded device-side wait gave up                   */
    LCS_ECUDA = 4,      /* a CUDA runtime call failed (details: lcs_last_error) */
    LCS_EAGAIN = 5,     /* no room now: retry later (batch admission)           */
    LCS_EOVERFLOW = 6   /* a result does not fit the requested type / capacity  */
} lcs_status;

typedef enum {
    LCS_I32 = 0,        /* int32_t entries, sentinel INT32_MIN                  */
    LCS_I16 = 1         /* int16_t entries, sentinel INT16_MIN; legal iff
                           m < 32768 and n < 32768 (values <= min(m, n))        */
} lcs_dtype;

/* Counters of the last call on a context (lcs_get_stats). */
typedef struct {
    int64_t workspace_bytes;        /* device workspace currently held          */
    int64_t peak_workspace_bytes;   /* high-water mark since lcs_create          */
    int32_t strip_height;           /* h used by the last call                   */
    int32_t strips;                 /* ceil(m / h)                               */
    int32_t merges;                 /* (max,+) merges in the tree                */
    int32_t tree_levels;            /* merge levels above the strips             */
    int32_t kernel_launches;        /* kernels the last call launched            */
    int32_t tile;                   /* merge tile edge (vertices)                */
    int32_t depth_first;            /* 1: the last call's tree was built depth
                                       first (see lcs_set_schedule)              */
    int32_t chunk_strips;           /* strips per strip launch of the last call  */
    int64_t plan_bytes;             /* workspace the last call's plan needs      */
} lcs_stats;

/* Per-kernel-class timing of the calls made while profiling is on
 * (lcs_set_profiling).  Kinds: 0 strip builder, 1 coarse argmax grid,
 * 2 merge tile refinement, 3 traceback level argmax, 4 traceback leaves,
 * 5 compaction, 6 dense fills / packing.  `ms` is the summed device time of
 * the launches measured with CUDA events on the launching stream; `bytes`
 * and `ops` are the algorithmic DRAM bytes and INT32 word operations of
 * those launches (see lcs_get_profile). */
typedef struct {
    int32_t kind;
    int32_t launches;
    double ms;
    double bytes;
    double ops;
} lcs_kernel_profile;

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the
 * workspace (0 = 64 GiB).  No device memory is allocated until the first
 * call that needs it.  *out receives the context.
 * Errors: EINVAL (out NULL, bad device), ECUDA. */
lcs_status lcs_create(lcs_ctx **out, int device, size_t mem_budget_bytes);

/* Free the workspace and the context (synchronises the device first). */
lcs_status lcs_destroy(lcs_ctx *ctx);

/* Static description of a status code. */
const char *lcs_strerror(lcs_status status);

/* Text of the last error recorded on ctx (a CUDA error string or the
 * argument that failed validation); "" if none.  Never NULL. */
const char *lcs_last_error(lcs_ctx *ctx);

/* Rows per strip for later calls; 0 restores the automatic choice.  Legal
 * values are 1..256.  The results do not depend on it (leftmost rule).
 * Errors: EINVAL. */
lcs_status lcs_set_strip_height(lcs_ctx *ctx, int32_t h);

/* Kernel that computes the tree's merge tiles (Sec. II-B-3: every entry of
 * D(i, j) = max_k U(i, k) + L(k, j)).  All give the same D, so the choice
 * changes speed only.
 *   LCS_MERGE_AUTO      LCS_MERGE_DPX when every merge operand of the tree
 *                       fits int16 values <= 16383 (strips of <= 16383 rows
 *                       below the root), else LCS_MERGE_EXACT.
 *   LCS_MERGE_EXACT     Monge-windowed refinement of each 64 x 64 tile from
 *                       its corner maximisers, with the exact leftmost argmax.
 *   LCS_MERGE_DPX       (max,+) product of each 64 x 64 tile on DPX
 *                       instructions (D only) over the band [x, y]: y the
 *                       smallest maximiser of the tile's bottom-right corner,
 *                       x the largest maximiser of its top-left corner that
 *                       is <= y; where the operands do not fit int16, EXACT
 *                       is used.
 * Applies to lcs_solve* and lcs_dist* on this ctx; lcs_merge, which returns
 * the argmax, always refines exactly.  Errors: EINVAL. */
enum { LCS_MERGE_AUTO = 0, LCS_MERGE_EXACT = 1, LCS_MERGE_DPX = 2 };
lcs_status lcs_set_merge_kernel(lcs_ctx *ctx, int32_t kind);

/* Failure detection, for tests.  Every device-side wait of the merge
 * kernels (a TMA band copy landing on its mbarrier) is bounded: after
 * wait_limit_ns of global time (0 restores the default of 2 s) the kernel
 * records a timeout, gives copies that are only late a second wait of the
 * same length, skips the tile and returns; lcs_sync (or the synchronous call)
 * then returns LCS_ETIMEOUT and the context stays usable.  With hold_band
 * set, the first tile of every later exact-merge launch (lcs_merge, and
 * lcs_solve / lcs_dist with LCS_MERGE_EXACT) announces its band on its
 * barrier but copies nothing, so that wait runs out with nothing in flight:
 * the way to exercise the timeout without faulting or hanging the GPU.
 * Outputs of such a call are unspecified.  hold_band = 0 and
 * wait_limit_ns = 0 restore normal operation.  Errors: EINVAL (ctx NULL,
 * wait_limit_ns < 0). */
lcs_status lcs_set_fault_injection(lcs_ctx *ctx, int32_t hold_band, int64_t wait_limit_ns);

/* Order in which the tree of strips is built (Sec. II-A's recursion).
 *   LCS_SCHED_AUTO    the retained tree when it needs at most 4 GiB and
 *                     fits the budget, else depth first.
 *   LCS_SCHED_RETAIN  breadth first: all strips in one launch, every merge
 *                     of a tree level in one launch, and every node kept
 *                     until the traceback has read it (fastest for small
 *                     problems; memory (2S - 1) node triangles).
 *   LCS_SCHED_DEPTH   depth first: `chunk` strips at a time (0: the largest
 *                     of 32, 16, .., 1 whose plan fits both the budget and
 *                     16 GiB, else the largest that fits the budget), merged as
 *                     soon as both halves exist, so that only the chunk's
 *                     nodes and one pending node per tree level are alive;
 *                     freed nodes are never re-read: the traceback
 *                     recomputes, per node from the root down, the row of
 *                     the upper child's DIST and the column of the lower
 *                     child's that the path needs, by one bit-vector sweep
 *                     each (Hirschberg's split), beside the tree on a side
 *                     stream.  A call that wants no DIST builds no tree.
 * The results do not depend on the schedule.  With an LCS wanted, a tree
 * half of more than 16384 rows keeps the retained tree.  Errors: EINVAL. */
enum { LCS_SCHED_AUTO = 0, LCS_SCHED_RETAIN = 1, LCS_SCHED_DEPTH = 2 };
lcs_status lcs_set_schedule(lcs_ctx *ctx, int32_t mode, int32_t chunk);

/* The tree plan of a solve that writes DIST (Sec. II-A: strips of h rows of
 * a, combined pairwise up a binary tree of (max,+) merges), as lcs_plan
 * reports it. */
typedef struct {
    int64_t workspace_bytes;   /* device workspace the plan needs (the caller's
                                  outputs not counted)                        */
    int32_t fits;              /* 1: workspace_bytes is within budget_bytes;
                                  0: a solve would return ENOMEM             */
    int32_t strip_height;      /* h                                          */
    int32_t strips;            /* S = ceil(m / h); 0 when m or n is 0        */
    int32_t nodes;             /* 2S - 1 (strips, then merge outputs)        */
    int32_t levels;            /* merges on the longest strip-to-root chain  */
    int32_t depth_first;       /* 0: retained tree, 1: depth first           */
    int32_t chunk;             /* strips per strip launch                    */
    int32_t launches;          /* strip launches + merge-group launches      */
    int32_t root;              /* node id of the root                        */
    int32_t tile;              /* merge tile edge (vertices)                 */
} lcs_plan_info;

/* One node of the plan.  Node ids: strips 0 .. S-1 in row order, then the
 * merge outputs.  Launches are numbered 0 .. launches-1 in stream order. */
typedef struct {
    int64_t row0, rows;        /* the rows of a the node covers              */
    int64_t offset, bytes;     /* its stored triangle in the workspace (0, 0
                                  for the root: the caller's matrix)         */
    int64_t grid_offset, grid_bytes;  /* merge outputs: the merge's argmax and
                                  value grids in the workspace (0, 0 for
                                  strips)                                    */
    int32_t upper, lower;      /* children (merge outputs; -1 for strips)    */
    int32_t parent;            /* -1 for the root                            */
    int32_t level;             /* 0 for strips, else 1 + the children's      */
    int32_t made_by;           /* the launch that writes it                  */
    int32_t last_use;          /* the last launch of the tree that needs its
                                  storage (the merge that consumes it when
                                  depth first; `launches` when the tree is
                                  retained for the traceback)                */
    int32_t grid_last_use;     /* the same for its grids (depth first: the
                                  launch that makes it; they are reused by
                                  later launches)                            */
} lcs_plan_node;

/* Host only: no device, no context, no CUDA call.  The plan a solve of an
 * m x n pair would use for its tree, chosen as lcs_solve chooses it: h (0:
 * the automatic strip height), `schedule` and `chunk` as lcs_set_schedule
 * takes them, budget_bytes as lcs_create takes mem_budget_bytes (0: 64
 * GiB), want_lcs (1: the solve also wants an LCS, which keeps the retained
 * tree when a tree half would exceed 16384 rows), root_dtype the dtype of
 * the DIST output.  Fills *info and the first min(cap, info->nodes) node
 * records (nodes may be NULL when cap is 0).  For sizing a budget before
 * lcs_create and for checking the schedule: the storage of nodes alive
 * during a launch (made_by <= launch <= last_use) and the grids in use
 * (made_by <= launch <= grid_last_use) never share workspace bytes.  A
 * context that holds host-call staging (lcs_solve_host) has that much less
 * of its budget for the workspace.
 * Errors: EINVAL (negative lengths, h outside 0..256, an unknown schedule,
 * chunk < 0, a bad dtype, LCS_I16 with m or n >= 32768, info NULL, cap < 0,
 * nodes NULL with cap > 0). */
lcs_status lcs_plan(int64_t m, int64_t n, int32_t h, int32_t schedule, int32_t chunk, size_t budget_bytes,
                    int32_t want_lcs, lcs_dtype root_dtype, lcs_plan_info *info, lcs_plan_node *nodes,
                    int64_t cap);

/* CUDA-graph replay of lcs_solve (1) or plain launches (0, the default).
 * With graphs on, the first lcs_solve with a given set of arguments runs as
 * usual and is then captured (on a private stream) into a graph; later
 * calls with the same arguments, strip height, merge kernel and device plan
 * replay it with one launch on the caller's stream.  One graph is kept: a
 * call with other arguments re-captures.  Calls with profiling on, and
 * empty strings, always launch directly.  Errors: EINVAL, ECUDA. */
lcs_status lcs_set_graphs(lcs_ctx *ctx, int32_t enable);

/* Autotuner: times the caller's solve (the same outputs: dist may be NULL,
 * out_lcs may be NULL) at strip heights 64, 128 and 256 and, where the
 * plan allows both, with the DPX and the exact merge kernel, and keeps the
 * fastest for the size bucket (floor(log2 m), floor(log2 n), dtype).  Later
 * solves with the automatic strip height (lcs_set_strip_height(ctx, 0)) and
 * merge kernel in that bucket use it.  The outputs hold the last timed
 * solve's results, which do not depend on the choice.  Synchronous.
 * h_out, merge_out, ms_out (nullable) receive the choice and its time.
 * Errors: EINVAL, ENOMEM (no candidate fits the budget), ECUDA, ETIMEOUT. */
lcs_status lcs_autotune(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, lcs_dtype dtype,
                        void *dist, int64_t ld, uint8_t *out_lcs, int64_t cap, void *stream,
                        int32_t *h_out, int32_t *merge_out, float *ms_out);

/* Counters of the last call (see lcs_stats).  Errors: EINVAL. */
lcs_status lcs_get_stats(lcs_ctx *ctx, lcs_stats *out);

/* Turn per-launch event timing on (1) or off (0); turning it on clears the
 * accumulated profile.  Adds two event records per launch.  Errors: EINVAL. */
lcs_status lcs_set_profiling(lcs_ctx *ctx, int32_t enable);

/* Synchronise the device and return the accumulated profile, one entry per
 * kernel kind that launched (at most cap entries; *count receives the
 * number written), then clear it.  Algorithmic bytes: strip builder = the
 * DIST tiles it writes; merge tile = both operand triangles read once plus
 * the output triangle written once, (n+1)(n+2)/2 entries each.  Algorithmic
 * ops (strip builder) = per (strip, source i, column j > i) step, 3 integer
 * instructions per 32-bit word of the strip's bit vector (and, add with
 * carry, and-not/or) plus 2 (carry out, accumulate).  Errors: EINVAL, ECUDA. */
lcs_status lcs_get_profile(lcs_ctx *ctx, lcs_kernel_profile *out, int32_t cap, int32_t *count);

/* Measured INT32 ALU throughput of the device: a kernel of independent
 * 32-bit integer add/logic operations filling every SM, timed with events.
 * *gops_out receives 10^9 operations per second; *sm_mhz_out (nullable)
 * the SM clock the kernel's own timer saw.  Errors: EINVAL, ECUDA. */
lcs_status lcs_measure_int32_peak(int device, double *gops_out, double *sm_mhz_out);

/* Synchronise `stream` and report device-side failures of earlier
 * asynchronous calls on ctx (ETIMEOUT from a bounded wait, EOVERFLOW from a
 * capacity check); clears the device error word.  Errors: ECUDA, ETIMEOUT,
 * EOVERFLOW. */
lcs_status lcs_sync(lcs_ctx *ctx, void *stream);

/* DIST of one strip of h rows (Sec. II-B-3 for h = 1; Sec. II-B-1's matrix
 * of a block of consecutive rows otherwise): dist(i, j) = LCS(a_strip,
 * b[i:j]).  Each column step applies the prefix-max over the strip's rows
 * F_j(r) = max(F_j(r-1), F_{j-1}(r), F_{j-1}(r-1) + [a_r = b_j]) to all h
 * rows at once.  a_strip: h device bytes; b: n device bytes; dist: dense
 * (n+1) x ld in `dtype`.  1 <= h <= 256 (values are at most h, so they fit
 * either dtype).  Asynchronous.
 * Errors: EINVAL (h out of range, n < 0, ld/alignment), ENOMEM, ECUDA. */
lcs_status lcs_strip_dist(lcs_ctx *ctx, const uint8_t *a_strip, int32_t h,
                          const uint8_t *b, int64_t n, lcs_dtype dtype,
                          void *dist, int64_t ld, void *stream);

/* (max,+) merge of the DIST of an upper strip U and a lower strip L over
 * the same columns (Sec. II-A's split through a middle vertex, Sec. II-B-1's
 * combination in its DIST form):
 *     dist_out(i, j) = max_{i <= k <= j} dist_u(i, k) + dist_l(k, j),
 * evaluated under the Monge bound (U and L must be DIST matrices of strips:
 * unit steps and the Monge inequality; arbitrary matrices are not legal
 * input).  argmax_out (nullable, dense int32, same ld) receives the smallest
 * maximising k (-1 below the diagonal).  All matrices dense (n+1) x ld in
 * `dtype`; dist_out may not alias the inputs.  Asynchronous.
 * Errors: EINVAL, ENOMEM, ECUDA; ETIMEOUT / EOVERFLOW via lcs_sync. */
lcs_status lcs_merge(lcs_ctx *ctx, const void *dist_u, const void *dist_l, int64_t n,
                     lcs_dtype dtype, int64_t ld, void *dist_out, int32_t *argmax_out,
                     void *stream);

/* lcs_merge without any device allocation, for callers that must not
 * allocate device memory: code running under a framework that owns all
 * device memory through its own pool, or a latency-critical loop in which a
 * cudaMalloc would synchronise the device.  The paper has no counterpart; it
 * is an interface convenience of this library.
 * Same arguments and results as lcs_merge, but no context: every scratch
 * byte comes from one static device array of 6 MiB that each GPU loading the
 * library holds until the process exits, which limits n to 1024 (both
 * dtypes; larger n returns EINVAL).  The call runs on the current device:
 * `stream` must belong to it, and so must every pointer.  Each call looks up
 * that device's copy of the array (cudaGetSymbolAddress, with the device
 * current), so a context torn down and created again is handled.  All calls
 * on a device share the array and it keeps the last call's contents (each
 * call clears what must start at zero); calls that overlap on the GPU race,
 * so serialise them.  Synchronous: returns after the merge has finished on
 * `stream`.
 * Errors: EINVAL (n > 1024, bad layout, inputs that are not strip DIST
 * matrices), ECUDA, ETIMEOUT, EOVERFLOW. */
lcs_status lcs_merge_static(const void *dist_u, const void *dist_l, int64_t n, lcs_dtype dtype, int64_t ld,
                            void *dist_out, int32_t *argmax_out, void *stream);

/* Full DIST of the whole grid: dist(i, j) = LCS(a, b[i:j]).  dist: dense
 * (n+1) x ld in dtype (LCS_I16 needs m, n < 32768).  Asynchronous.
 * Errors: EINVAL, ENOMEM, ECUDA. */
lcs_status lcs_dist(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    lcs_dtype dtype, void *dist, int64_t ld, void *stream);

/* LCS length = DIST(0, n) (Sec. I).  Synchronises the stream and writes
 * *out_len_host.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
lcs_status lcs_length(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                      int64_t *out_len_host, void *stream);

/* One LCS: the letters of a on the leftmost heaviest path (Sec. II-C..II-E),
 * found by walking the leftmost maximisers down the merge tree.  out_lcs:
 * device buffer of cap >= min(m, n) bytes.  Synchronises the stream and
 * writes *out_len_host (the number of letters written).
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW (cap too small). */
lcs_status lcs_traceback(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         uint8_t *out_lcs, int64_t cap, int64_t *out_len_host, void *stream);

/* ------------------------------------------------------------------------
 * Breakout (D-form) matrices: the paper's compact form of a strip's DIST
 * (Sec. II-B-1).  D(i, w) = min{ j >= i : DIST(i, j) >= w } is the leftmost
 * bottom vertex reached from top vertex i with weight w; D(i, 0) = i; an
 * unreachable weight holds INT32_MAX (LCS_I32) or INT16_MAX (LCS_I16).  A
 * strip of h rows takes (n+1) x (h+1) entries, row-major with leading
 * dimension ld (elements), row i = D(i, 0..h).  Device pointers, owned by
 * the caller; asynchronous on `stream`.
 * ---------------------------------------------------------------------- */

/* D-forms of the S = ceil(m / h) strips of h (1..256) rows of a (m
 * letters; the last strip may be shorter, its unreachable weights hold the
 * infinity) against b (n columns), in one launch.  Strip s is stored at
 * dform + s * (n+1) * ldf elements.  ldf >= h + 1; S <= 65535.  LCS_I16
 * needs n < 32767.  Errors: EINVAL, ECUDA. */
lcs_status lcs_strip_dform(lcs_ctx *ctx, const uint8_t *a, int64_t m, int32_t h, const uint8_t *b, int64_t n,
                           lcs_dtype dtype, void *dform, int64_t ldf, void *stream);

/* The combination of Sec. II-B-3 of an upper (hu rows) and a lower (hl
 * rows) strip over the same b:
 *     out(i, w) = min_{0 <= k <= w} dl(du(i, k), w - k),   w = 0 .. hu + hl,
 * terms with du(i, k) unreachable or w - k > hl left out.  Computed by
 * monotone column minima per top vertex (Algorithm 1 cut to two levels:
 * the exact minimum of every 32nd column bounds the rows of the columns in
 * between).  hu + hl <= 16384; ldu >= hu + 1, ldl >= hl + 1,
 * ldo >= hu + hl + 1.  Errors: EINVAL, ECUDA. */
lcs_status lcs_dform_merge(lcs_ctx *ctx, const void *du, int32_t hu, int64_t ldu, const void *dl, int32_t hl,
                           int64_t ldl, int64_t n, lcs_dtype dtype, void *out, int64_t ldo, void *stream);

/* The leftmost heaviest path itself, as the list of its grid vertices
 * (Sec. II-D: each row's horizontal run between consecutive cross vertices,
 * the runs placed in row order by a prefix sum).  Vertex (r, c) is the
 * grid point after r letters of a and c letters of b; the list runs from
 * (0, 0) to (m, n) and has m + n + 1 - L entries (a match diagonal enters
 * a row one column right of where the previous row's run ended).
 * path: device int32 array of 2 * cap entries receiving (row, col) pairs.
 * Synchronises the stream and writes *out_count_host (the vertex count).
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT; EOVERFLOW when cap is below the
 * vertex count (nothing written to path, *out_count_host untouched). */
lcs_status lcs_path(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int32_t *path, int64_t cap, int64_t *out_count_host, void *stream);

/* The whole hot path in one call: strips, merge tree, and any of
 *   dist  (nullable): dense (n+1) x ld DIST in dtype;
 *   out_lcs (nullable): the LCS letters (cap >= min(m, n) bytes);
 *   cross (nullable): int32 device array of m+1 cross vertices v[0..m],
 *        v[r] = leftmost column of the path in row r (Sec. II-C);
 *   out_len_device (nullable): int64 device word receiving the length.
 * Asynchronous (nothing is read back).  With every output NULL the call
 * still builds the tree and leaves the length in an internal word.
 * Errors: EINVAL, ENOMEM, ECUDA; ETIMEOUT / EOVERFLOW via lcs_sync. */
lcs_status lcs_solve(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     lcs_dtype dtype, void *dist, int64_t ld,
                     uint8_t *out_lcs, int64_t cap, int32_t *cross,
                     int64_t *out_len_device, void *stream);

/* lcs_solve on HOST buffers: copies a and b to the device, runs the whole
 * path, returns the requested outputs (dist_host: (n+1) x ld in dtype;
 * lcs_host: cap bytes, of which the first *out_len_host hold the LCS) and
 * writes *out_len_host.  A pinned dist_host that the device can address
 * (16-byte aligned rows) is written by the kernels directly: its lower
 * triangle while the tree is built, the rest by the root merge while the
 * traceback runs.  Any other dist_host is filled by a copy from device
 * staging (pageable memory works, slower).  Synchronous.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW. */
lcs_status lcs_solve_host(lcs_ctx *ctx, const uint8_t *a_host, int64_t m,
                          const uint8_t *b_host, int64_t n, lcs_dtype dtype,
                          void *dist_host, int64_t ld, uint8_t *lcs_host, int64_t cap,
                          int64_t *out_len_host, void *stream);

/* ------------------------------------------------------------------------
 * Batches of independent pairs.  The paper treats one pair; serving many
 * pairs of uneven lengths is this library's extension of it.  A pair whose a
 * has at most 16384 letters is one strip (all its rows fit one bit vector),
 * so its tree has no merge level: the length is the strip's DIST(0, n) and
 * one LCS the strip's leftmost heaviest path.  Pairs of up to 4096 rows run a
 * warp per pair in one launch per size class (a up to 2048 and up to 4096
 * rows), the classes side by side; pairs of 4097..16384 rows spread their
 * vector over several warps and find the LCS from forward and backward
 * sweeps.  Taller pairs go through the strip tree of lcs_solve, one after
 * another, inside lcs_batch_submit.  Each batch runs on streams of its own:
 * a process with many batches in flight should raise the
 * CUDA_DEVICE_MAX_CONNECTIONS environment variable (32, say) before CUDA is
 * initialised, or the batches' kernels queue behind one another in the
 * default 8 hardware queues.
 * ---------------------------------------------------------------------- */
#define LCS_WANT_STRING 1u

typedef struct {
    const uint8_t *a;       /* m device bytes (rows)                             */
    int64_t m;
    const uint8_t *b;       /* n device bytes (columns)                          */
    int64_t n;
    uint32_t flags;         /* LCS_WANT_STRING: also return one LCS              */
} lcs_pair;

typedef struct {
    int64_t len;            /* LCS length                                        */
    int64_t string_offset;  /* offset of the pair's LCS (len bytes) in the
                               ticket's string buffer, -1 without LCS_WANT_STRING */
    lcs_status status;      /* of this pair                                      */
    double t_submit;        /* steady host clock (s) when the batch was submitted */
    double t_done;          /* when the batch finished on the device, same clock  */
} lcs_result;

/* Queue `count` pairs (descriptors in host memory; the strings they point to
 * stay valid until the batch is done) and return a ticket.  The batch runs
 * asynchronously on a stream of its own; its device memory (descriptors,
 * results, strings, and the column vectors of the pairs that want their LCS)
 * counts against the context's budget.
 * Errors: EINVAL (a NULL or negative argument), EAGAIN (the batch does not
 * fit the budget next to what the context holds now: release finished
 * batches or submit fewer pairs), ENOMEM, ECUDA. */
lcs_status lcs_batch_submit(lcs_ctx *ctx, const lcs_pair *pairs_host, int64_t count, uint64_t *ticket_host);

/* Wait up to timeout_ms (0: just look, < 0: until done) for a batch.  When
 * it is done, write min(count, cap) results in submission order and set
 * *n_done_host = count; otherwise *n_done_host = 0.  The batch keeps its
 * memory until lcs_batch_release.
 * Errors: EINVAL (unknown ticket), EOVERFLOW (cap < count; the first cap are
 * written), ECUDA. */
lcs_status lcs_batch_poll(lcs_ctx *ctx, uint64_t ticket, lcs_result *results_host, int64_t cap,
                          int64_t *n_done_host, int32_t timeout_ms);

/* Copy the string buffer of a finished batch (the LCS of pair p at
 * results[p].string_offset, results[p].len bytes) to `out` (host or device
 * memory), waiting for the batch first; *bytes_host receives its size.
 * Errors: EINVAL, EOVERFLOW (cap too small; nothing copied), ECUDA. */
lcs_status lcs_batch_strings(lcs_ctx *ctx, uint64_t ticket, uint8_t *out, int64_t cap, int64_t *bytes_host);

/* Wait for a batch and free its device memory.  Errors: EINVAL, ECUDA. */
lcs_status lcs_batch_release(lcs_ctx *ctx, uint64_t ticket);

#ifdef __cplusplus
}
#endif

#endif /* LCS_GB300_H */
