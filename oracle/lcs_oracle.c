/*
 * lcs_oracle.c -- plain, slow CPU oracle for the Lu-Lin DIST method of
 * "Parallel Longest Common SubSequence Analysis In Chapel" (arXiv 2309.09072).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, loads or calls
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Notation (Sec. II-A, Fig. 1): string a (length m) labels the grid rows,
 * string b (length n) the columns.  The grid graph has (m+1) x (n+1)
 * vertices; right and down edges weigh 0, the diagonal edge into vertex
 * (r, c) weighs 1 iff a_r = b_c (1-based letters; zero-weight diagonals are
 * left out, Fig. 1 caption).  Top and bottom boundary vertices are numbered
 * 0..n here (0-based), and
 *
 *     DIST(i, j) = weight of the heaviest path from top vertex i to bottom
 *                  vertex j = LCS(a, b[i:j])          for j >= i,
 *     DIST(i, j) = -infinity (stored as INT32_MIN)    for j <  i.
 *
 * Every function is the plain definition written out, or the paper's steps
 * in the paper's order; none of them is blocked, fused or reordered.
 */
#include <limits.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_NEG_INF INT32_MIN
#define ORACLE_INF INT64_MAX

static int32_t max_i32(int32_t x, int32_t y) { return x > y ? x : y; }

/* ------------------------------------------------------------------------
 * LCS length by the textbook O(mn) dynamic programme (Sec. I: "a simple
 * dynamic programming approach ... in O(mn) time"), kept to two rows.
 * F(r, c) = LCS(a[0:r], b[0:c]).
 * ---------------------------------------------------------------------- */
int64_t oracle_lcs_length(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n)
{
    if (m <= 0 || n <= 0) return 0;
    int32_t *prev = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *cur = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    for (int64_t r = 1; r <= m; ++r) {
        cur[0] = 0;
        for (int64_t c = 1; c <= n; ++c) {
            if (a[r - 1] == b[c - 1]) cur[c] = prev[c - 1] + 1;
            else cur[c] = max_i32(prev[c], cur[c - 1]);
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    int64_t out = prev[n];
    free(prev); free(cur);
    return out;
}

/* ------------------------------------------------------------------------
 * One row of DIST (Sec. II-B, the matrix of heaviest paths from a top vertex
 * to every bottom vertex): for source i, the DP of a against b[i:n]; its last
 * row is DIST(i, j), j = i..n.  Entries j < i get the -infinity sentinel.
 * ---------------------------------------------------------------------- */
int oracle_dist_row(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int64_t i, int32_t *row)
{
    if (i < 0 || i > n) return -1;
    for (int64_t c = 0; c < i; ++c) row[c] = ORACLE_NEG_INF;
    int64_t w = n - i;                          /* columns i..n -> 0..w */
    int32_t *prev = (int32_t *)calloc((size_t)w + 1, sizeof(int32_t));
    int32_t *cur = (int32_t *)calloc((size_t)w + 1, sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    /* The heaviest path into vertex (r, c) arrives by the down edge, the
     * right edge or the diagonal (weight [a_r = b_c]), so each cell is the
     * maximum of those three terms. */
    for (int64_t r = 1; r <= m; ++r) {
        cur[0] = 0;
        for (int64_t c = 1; c <= w; ++c) {
            const int32_t diag = prev[c - 1] + (a[r - 1] == b[i + c - 1] ? 1 : 0);
            cur[c] = max_i32(max_i32(prev[c], cur[c - 1]), diag);
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    for (int64_t c = 0; c <= w; ++c) row[i + c] = prev[c];
    free(prev); free(cur);
    return 0;
}

/* Sources are independent, so they may be spread over host threads; each
 * row is still computed by oracle_dist_row exactly as above. */
typedef struct {
    const uint8_t *a, *b;
    int64_t m, n;
    const int64_t *rows;     /* NULL: rows 0..n */
    int64_t nrows;
    int32_t *out;
    int64_t ld;
    int tid, nthreads;
    int err;
} dist_job;

static void *dist_worker(void *p)
{
    dist_job *J = (dist_job *)p;
    for (int64_t t = J->tid; t < J->nrows; t += J->nthreads) {
        int64_t i = J->rows ? J->rows[t] : t;
        if (oracle_dist_row(J->a, J->m, J->b, J->n, i, J->out + t * J->ld) != 0) J->err = 1;
    }
    return NULL;
}

static int resolve_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

static int run_dist(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    const int64_t *rows, int64_t nrows, int32_t *out, int64_t ld, int nthreads)
{
    nthreads = resolve_threads(nthreads);
    if (nthreads > nrows) nthreads = (int)(nrows > 0 ? nrows : 1);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    dist_job *jobs = (dist_job *)calloc((size_t)nthreads, sizeof(dist_job));
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    int err = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (dist_job){a, b, m, n, rows, nrows, out, ld, t, nthreads, 0};
        if (pthread_create(&th[t], NULL, dist_worker, &jobs[t]) != 0) {
            dist_worker(&jobs[t]);      /* run inline if a thread cannot start */
            th[t] = 0;
        }
    }
    for (int t = 0; t < nthreads; ++t) {
        if (th[t]) pthread_join(th[t], NULL);
        err |= jobs[t].err;
    }
    free(th); free(jobs);
    return err ? -1 : nthreads;
}

/* Full (n+1) x (n+1) DIST, row i at dist + i*ld.  Returns the thread count
 * used, or -1 on error. */
int oracle_dist(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                int32_t *dist, int64_t ld, int nthreads)
{
    if (ld < n + 1) return -1;
    return run_dist(a, m, b, n, NULL, n + 1, dist, ld, nthreads);
}

/* Selected rows of DIST: out[t*(n+1) + j] = DIST(rows[t], j). */
int oracle_dist_rows(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     const int64_t *rows, int64_t nrows, int32_t *out, int nthreads)
{
    return run_dist(a, m, b, n, rows, nrows, out, n + 1, nthreads);
}

/* ------------------------------------------------------------------------
 * The (max,+) combination of an upper and a lower strip (Sec. II-A: the
 * heaviest path a -> b through a middle vertex c; Eq. for D_G in Sec. II-B-1
 * in its DIST form):
 *     D(i, j) = max_{i <= k <= j} U(i, k) + L(k, j),
 * brute force over every k, O(n^3).  K(i, j) is the smallest maximising k
 * (ties go to the lower index, as the "<=" comparison of Algorithm 2 does).
 * Lower-triangle cells get the sentinel and K = -1.
 * ---------------------------------------------------------------------- */
void oracle_merge(const int32_t *U, const int32_t *L, int64_t n, int64_t ld,
                  int32_t *D, int32_t *K)
{
    for (int64_t i = 0; i <= n; ++i) {
        for (int64_t j = 0; j <= n; ++j) {
            if (j < i) {
                D[i * ld + j] = ORACLE_NEG_INF;
                if (K) K[i * ld + j] = -1;
                continue;
            }
            int64_t best = INT64_MIN, bk = -1;
            for (int64_t k = i; k <= j; ++k) {
                int64_t v = (int64_t)U[i * ld + k] + (int64_t)L[k * ld + j];
                if (v > best) { best = v; bk = k; }
            }
            D[i * ld + j] = (int32_t)best;
            if (K) K[i * ld + j] = (int32_t)bk;
        }
    }
}

/* ------------------------------------------------------------------------
 * One LCS: the leftmost heaviest path (Sec. II-C..II-E).  With
 *     F(r, c) = LCS(a[0:r], b[0:c])   (forward table),
 *     B(r, c) = LCS(a[r:m], b[c:n])   (backward table),  L = F(m, n),
 * the cross vertex of row r (the leftmost vertex of the path in that row,
 * Sec. II-C) is v[r] = min{ c : F(r, c) + B(r, c) = L }.  Letter a_r is
 * emitted (Sec. II-E) iff the step between the cross vertices of rows r-1 and
 * r gains weight 1: F(r, v[r]) - F(r-1, v[r-1]) = 1.  Marked letters are
 * emitted in row order.
 * Returns L (the number of letters written to out), or -1 on error.
 * v (nullable) receives v[0..m].
 * ---------------------------------------------------------------------- */
static int64_t leftmost_path(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                             uint8_t *out, int64_t *v, uint8_t *gain)
{
    int64_t W = n + 1;
    int32_t *Bt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1) * (size_t)W);
    int32_t *Fp = (int32_t *)calloc((size_t)W, sizeof(int32_t));
    int32_t *Fc = (int32_t *)calloc((size_t)W, sizeof(int32_t));
    if (!Bt || !Fp || !Fc) { free(Bt); free(Fp); free(Fc); return -1; }
    for (int64_t c = 0; c <= n; ++c) Bt[m * W + c] = 0;
    for (int64_t r = m - 1; r >= 0; --r) {
        Bt[r * W + n] = 0;
        for (int64_t c = n - 1; c >= 0; --c) {
            if (a[r] == b[c]) Bt[r * W + c] = Bt[(r + 1) * W + c + 1] + 1;
            else Bt[r * W + c] = max_i32(Bt[(r + 1) * W + c], Bt[r * W + c + 1]);
        }
    }
    int32_t L = Bt[0];
    int64_t vprev = 0;                 /* F(0, c) = 0 and B(0, 0) = L, so v[0] = 0 */
    if (v) v[0] = 0;
    if (gain) gain[0] = 0;
    int64_t len = 0;
    for (int64_t r = 1; r <= m; ++r) {
        Fc[0] = 0;
        for (int64_t c = 1; c <= n; ++c) {
            if (a[r - 1] == b[c - 1]) Fc[c] = Fp[c - 1] + 1;
            else Fc[c] = max_i32(Fp[c], Fc[c - 1]);
        }
        int64_t vr = -1;
        for (int64_t c = 0; c <= n; ++c) {
            if (Fc[c] + Bt[r * W + c] == L) { vr = c; break; }
        }
        if (vr < 0) { len = -1; break; }
        const int g = Fc[vr] - Fp[vprev] == 1;
        if (gain) gain[r] = (uint8_t)g;
        if (g) {
            if (out) out[len] = a[r - 1];
            ++len;
        }
        if (v) v[r] = vr;
        vprev = vr;
        int32_t *t = Fp; Fp = Fc; Fc = t;
    }
    free(Bt); free(Fp); free(Fc);
    return len;
}

int64_t oracle_traceback(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         uint8_t *out, int64_t *v)
{
    return leftmost_path(a, m, b, n, out, v, NULL);
}

/* ------------------------------------------------------------------------
 * The vertex list of the same leftmost heaviest path (Sec. II-D): in row r
 * the path runs right from its cross vertex v[r] to the column where it
 * leaves the row, then steps down into row r+1 at v[r+1].  The step gains
 * weight 1 (F(r+1, v[r+1]) - F(r, v[r]) = 1) only on a match diagonal, which
 * leaves row r at column v[r+1] - 1; otherwise it is vertical and leaves at
 * v[r+1].  The last row runs to column n.  The runs are concatenated in row
 * order.  rows/cols (capacity m + n + 1 each) receive the vertices from
 * (0, 0) to (m, n).  Returns the vertex count, or -1 on error.
 * ---------------------------------------------------------------------- */
int64_t oracle_path(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int64_t *rows, int64_t *cols)
{
    int64_t *v = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    uint8_t *gain = (uint8_t *)malloc((size_t)m + 1);
    if (!v || !gain) { free(v); free(gain); return -1; }
    int64_t cnt = -1;
    if (leftmost_path(a, m, b, n, NULL, v, gain) >= 0) {
        cnt = 0;
        for (int64_t r = 0; r <= m; ++r) {
            const int64_t end = (r == m) ? n : (gain[r + 1] ? v[r + 1] - 1 : v[r + 1]);
            for (int64_t c = v[r]; c <= end; ++c) {
                rows[cnt] = r;
                cols[cnt] = c;
                ++cnt;
            }
        }
    }
    free(v); free(gain);
    return cnt;
}

/* ------------------------------------------------------------------------
 * DIST -> breakout form D_G (Sec. II-B-1): D_G(i, w) is the leftmost bottom
 * vertex reachable from top vertex i by a path of weight w,
 *     D(i, w) = min{ j >= i : DIST(i, j) >= w },  infinity if none,
 * with the paper's 0th breakout D(i, 0) = i (Sec. II-B-3).
 * Output (n+1) x (wmax+1), infinity = INT64_MAX.
 * ---------------------------------------------------------------------- */
void oracle_dform(const int32_t *dist, int64_t n, int64_t ld, int64_t wmax, int64_t *D)
{
    for (int64_t i = 0; i <= n; ++i) {
        for (int64_t w = 0; w <= wmax; ++w) {
            int64_t found = ORACLE_INF;
            for (int64_t j = i; j <= n; ++j) {
                if (dist[i * ld + j] >= w) { found = j; break; }
            }
            D[i * (wmax + 1) + w] = found;
        }
    }
}

/* ------------------------------------------------------------------------
 * The two-row leaf D_{G_h} by the paper's own construction (Sec. II-B-3),
 * in the paper's 1-based vertex numbering: out[k-1] = first breakout of top
 * vertex k, k = 1..n.
 *   1. find the match positions j_1 < ... < j_r with b_{j} = a_h;
 *   2. D(1) = j_1 + 1 and D(j_{k-1} + 1) = j_k - j_{k-1} for 1 < k <= r;
 *      every other entry is "not yet computed" (0 in the sum below);
 *   3. prefix sum D(k) = sum_{t <= k} D(t) over the computed range;
 *   4. infinity for the vertices after the last match.
 * The text gives the ranges of steps 3 and 4 as 1..j_r+1 and j_r+2..n, but
 * the worked example prints infinity from position j_r+1 on, which is also
 * what the breakout definition gives (vertex j_r+1 has no match to its
 * right); the example is followed: sum over 1..j_r, infinity from j_r+1.
 * gaps (nullable) receives the vector after step 2 (0 = not computed).
 * Infinity = INT64_MAX.
 * ---------------------------------------------------------------------- */
void oracle_leaf_dform(uint8_t ah, const uint8_t *b, int64_t n, int64_t *out, int64_t *gaps)
{
    int64_t *D = (int64_t *)calloc((size_t)n + 2, sizeof(int64_t));   /* 1-based */
    int64_t prev = -1, last = 0;
    for (int64_t j = 1; j <= n; ++j) {
        if (b[j - 1] != ah) continue;
        if (prev < 0) D[1] = j + 1;
        else D[prev + 1] = j - prev;
        prev = j;
        last = j;
    }
    if (gaps) for (int64_t k = 1; k <= n; ++k) gaps[k - 1] = D[k];
    int64_t acc = 0;
    for (int64_t k = 1; k <= n; ++k) {
        if (k <= last) { acc += D[k]; out[k - 1] = acc; }
        else out[k - 1] = ORACLE_INF;
    }
    free(D);
}

/* ------------------------------------------------------------------------
 * The paper's combination of breakout matrices (Sec. II-B-1):
 *     D_G(i, w) = min( D_GU(i, w), D_GL(i, w), D_GL(D_GU(i, k), w - k) ),
 * 1 <= k <= w.  With the 0th breakout D(x, 0) = x the first two terms are
 * the k = w and k = 0 cases of the third, so this is the min over 0..w.
 * A term is infinity when D_GU(i, k) is infinity or w - k exceeds the
 * lower half's largest weight wl.  DU is (n+1) x (wu+1), DL is
 * (n+1) x (wl+1), D is (n+1) x (wu+wl+1); infinity = INT64_MAX.
 * ---------------------------------------------------------------------- */
void oracle_dform_combine(const int64_t *DU, int64_t wu, const int64_t *DL, int64_t wl,
                          int64_t n, int64_t *D)
{
    int64_t w_out = wu + wl;
    for (int64_t i = 0; i <= n; ++i) {
        for (int64_t w = 0; w <= w_out; ++w) {
            int64_t best = ORACLE_INF;
            for (int64_t k = 0; k <= w; ++k) {
                if (k > wu || w - k > wl) continue;
                int64_t x = DU[i * (wu + 1) + k];
                if (x == ORACLE_INF) continue;
                int64_t y = DL[x * (wl + 1) + (w - k)];
                if (y < best) best = y;
            }
            D[i * (w_out + 1) + w] = best;
        }
    }
}
