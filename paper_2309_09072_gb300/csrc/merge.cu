// merge.cu -- the (max,+) merge of two strip DISTs under the Monge bound.
//
//     D(i, j) = max_{i <= k <= j} U(i, k) + L(k, j),   K(i, j) = smallest maximiser
//
// (Sec. II-A's split of a heaviest path at the boundary row between the upper
// and lower halves; Sec. II-B-1's combination formula in its DIST form).  U
// and L are DIST matrices of strips, hence Monge, and with ties broken to the
// smallest k the maximiser is monotone: K(i, j) <= K(i, j') for j <= j' and
// K(i, j) <= K(i', j) for i <= i' (the column-minima monotonicity that
// Algorithm 1 relies on, read for maxima).  So once K is known at two points
// (i_lo, j_lo) <= (i, j) <= (i_hi, j_hi), only k in [K(i_lo, j_lo),
// K(i_hi, j_hi)] ∩ [i, j] needs scanning.
//
// Schedule (no serial wavefront, so there is no chain of n dependent waves):
//   1. coarse_kernel, one launch per level: K on the grid of tile corners
//      (multiples of T, plus n).  The first level scans full windows on a
//      sparse sub-grid (stride sigma0); every later level halves the stride
//      and scans only the window between the enclosing coarser points.
//   2. tile_kernel: one CTA per output tile (T x T vertices plus the far edges
//      shared with the neighbours).  The CTA stages the U rows and L columns
//      of the tile's k-window into shared memory with TMA bulk copies
//      (cp.async.bulk + mbarrier), then refines K from the four corners at
//      stride 32, 16, .., 1 -- each level first the points with one new
//      coordinate, then the points with two, every point bounded by already
//      known neighbours (a warp per grid row, a lane per point) -- and
//      finally writes D out: a TMA bulk store of the tile for internal nodes,
//      plain stores for a dense matrix.
//      Tiles whose k-window exceeds the shared-memory band fall back to the
//      same refinement reading global memory.
//   3. tile_dpx_kernel (int16 operands, D only): persistent CTAs take tiles
//      from a counter; a tile's band [kl, kh] (narrowed at its low end to the
//      largest maximiser of the near corner that is <= kh) streams through
//      shared memory from its top chunk down, and the band's (max,+) product
//      runs on DPX; packed output tiles go from the accumulators to global
//      memory, the root's dense tile through shared memory.
#include <algorithm>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int64_t grid_vertex(int64_t p, int64_t n) { return min(p * T, n); }
// Vertex of coarse-grid index p at spacing 2^gshift (gshift 0: T).
__device__ __forceinline__ int64_t grid_vertex_s(int64_t p, int64_t n, int gshift) {
    return min(p << (gshift ? gshift : T_SHIFT), n);
}

// Point rem of the upper triangle t <= u of a cnt x cnt grid, row by row:
// row t starts at t cnt - t (t - 1) / 2.
__device__ __forceinline__ void tri_point(int64_t rem, int64_t cnt, int64_t &t, int64_t &u) {
    auto start = [&](int64_t x) { return x * cnt - x * (x - 1) / 2; };
    const float b = 2.0f * (float)cnt + 1.0f;
    int64_t r = (int64_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)rem, 0.0f))) * 0.5f);
    r = max((int64_t)0, min(r, cnt - 1));
    while (r + 1 < cnt && start(r + 1) <= rem) ++r;
    while (r > 0 && start(r) > rem) --r;
    t = r;
    u = r + (rem - start(r));
}

// Warp-wide (value, k) reduction: largest value, smallest k among equals.
__device__ __forceinline__ void warp_argmax(int &v, int &k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const int ov = __shfl_xor_sync(0xFFFFFFFFu, v, off);
        const int ok = __shfl_xor_sync(0xFFFFFFFFu, k, off);
        if (ov > v || (ov == v && ok < k)) { v = ov; k = ok; }
    }
}

// ------------------------------------------------------------------ coarse
int64_t coarse_sigma0(int64_t P) {
    // Full scans on a sub-grid of about 33 x 33 points; each later level
    // halves the stride down to 1.
    int64_t s = 1;
    while (s * 32 < P) s <<= 1;
    return s;
}

template <typename TIn>
__global__ void __launch_bounds__(256) coarse_kernel(MergeParams p) {
    pdl_wait_and_release();
    const int64_t P = p.P, n = p.n, sigma = p.sigma;
    const int64_t cnt = P / sigma + 1 + ((P % sigma) ? 1 : 0);   // points 0, s, 2s, .., P
    const int64_t per_job = cnt * (cnt + 1) / 2;                  // t <= u
    const int64_t total = per_job * p.njobs;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp0; w < total; w += nwarps) {
        const int job = (int)(w / per_job);
        int64_t t, u;
        tri_point(w - (int64_t)job * per_job, cnt, t, u);
        const int64_t xp = min(t * sigma, P), xq = min(u * sigma, P);
        if (xp > xq) continue;
        const bool newp = (t & 1) && xp < P;
        const bool newq = (u & 1) && xq < P;
        if (!p.full && !newp && !newq) continue;
        const MergeJob jb = p.jobs[job];
        int32_t *kg = jb.kgrid;
        const int gi = (int)grid_vertex_s(xp, n, p.gshift), gj = (int)grid_vertex_s(xq, n, p.gshift);
        int lo = gi, hi = gj;
        if (!p.full) {
            const int64_t td = newp ? t - 1 : t, tu = newp ? t + 1 : t;
            const int64_t ud = newq ? u - 1 : u, uu = newq ? u + 1 : u;
            const int64_t pd = min(td * sigma, P), pu = min(tu * sigma, P);
            const int64_t qd = min(ud * sigma, P), qu = min(uu * sigma, P);
            lo = max(lo, kg[pd * (P + 1) + qd]);
            hi = min(hi, kg[pu * (P + 1) + qu]);
        }
        const TIn *U = reinterpret_cast<const TIn *>(jb.U);
        const TIn *L = reinterpret_cast<const TIn *>(jb.L);
        int best = INT32_MIN, bk = INT32_MAX;
        // Walk the window one K-tile at a time: within a tile both U's row gi
        // and L's column gj are contiguous, so each lane reads k = base + lane
        // and base + 32 with the tile bases computed once per tile.
        const int64_t Ib = gi >> T_SHIFT, Jb = gj >> T_SHIFT;
        const int ro = (gi & (T - 1)) * Fmt<TIn>::P, co = (gj & (T - 1)) * Fmt<TIn>::P;
#pragma unroll 8
        for (int kt = lo >> T_SHIFT; kt <= (hi >> T_SHIFT); ++kt) {
            const TIn *ub = U + row_tile(Ib, kt, p.NT) * Fmt<TIn>::ELEMS + ro;
            const TIn *lb = L + col_tile(kt, Jb) * Fmt<TIn>::ELEMS + co;
            const int k0 = kt * T;
            const int ka = max(lo, k0), kz = min(hi, k0 + T - 1);
            const int k1 = k0 + lane, k2 = k0 + 32 + lane;
            const bool v1 = k1 >= ka && k1 <= kz, v2 = k2 >= ka && k2 <= kz;
            const int x1 = v1 ? (int)ub[lane] + (int)lb[lane] : INT32_MIN;
            const int x2 = v2 ? (int)ub[32 + lane] + (int)lb[32 + lane] : INT32_MIN;
            if (x1 > best) { best = x1; bk = k1; }     // k increases: first max per lane
            if (x2 > best) { best = x2; bk = k2; }
        }
        warp_argmax(best, bk);
        if (lane == 0) {
            if (bk == INT32_MAX) { set_error(p.err, ERR_BOUNDS); bk = gi; best = 0; }
            kg[xp * (P + 1) + xq] = bk;
            jb.vgrid[xp * (P + 1) + xq] = best;
        }
    }
}

// The full-scan level: windows span up to n, so a whole CTA takes one grid
// point (threads over k, then a block-wide leftmost argmax).
template <typename TIn>
__global__ void __launch_bounds__(256) coarse_full_kernel(MergeParams p) {
    pdl_wait_and_release();
    __shared__ int sv[8], sk[8];
    const int64_t P = p.P, n = p.n, sigma = p.sigma;
    const int64_t cnt = P / sigma + 1 + ((P % sigma) ? 1 : 0);
    const int64_t per_job = cnt * (cnt + 1) / 2;                  // t <= u
    const int job = (int)(blockIdx.x / per_job);
    int64_t t, u;
    tri_point(blockIdx.x - (int64_t)job * per_job, cnt, t, u);
    const int64_t xp = min(t * sigma, P), xq = min(u * sigma, P);
    if (xp > xq) return;
    const MergeJob jb = p.jobs[job];
    const TIn *U = reinterpret_cast<const TIn *>(jb.U);
    const TIn *L = reinterpret_cast<const TIn *>(jb.L);
    const int gi = (int)grid_vertex_s(xp, n, p.gshift), gj = (int)grid_vertex_s(xq, n, p.gshift);
    int best = INT32_MIN, bk = INT32_MAX;
#pragma unroll 4
    for (int k = gi + (int)threadIdx.x; k <= gj; k += blockDim.x) {
        const int v = (int)U[row_elem<TIn>(gi, k, p.NT)] + (int)L[col_elem<TIn>(k, gj)];
        if (v > best) { best = v; bk = k; }     // k increases: first max per thread
    }
    warp_argmax(best, bk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sv[warp] = best; sk[warp] = bk; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && sk[w] < bk)) { best = sv[w]; bk = sk[w]; }
        if (bk == INT32_MAX) { set_error(p.err, ERR_BOUNDS); bk = gi; best = 0; }
        jb.kgrid[xp * (P + 1) + xq] = bk;
        jb.vgrid[xp * (P + 1) + xq] = best;
    }
}

// One full-scan coarse point by a whole CTA, int16 operands: the leftmost
// argmax of U(gi, k) + L(k, gj) over every k in [gi, gj].  A thread reads four
// consecutive k of U's stored row gi and of L's stored column gj per 8-byte
// load, then a block-wide (largest value, smallest k) reduction.  sv, sk: a
// slot per warp.
__device__ __forceinline__ void coarse_point_cta16(const MergeParams &p, int64_t sigma, int64_t w, int *sv,
                                                   int *sk) {
    const int64_t P = p.P, n = p.n;
    const int64_t cnt = P / sigma + 1 + ((P % sigma) ? 1 : 0);
    const int64_t per_job = cnt * (cnt + 1) / 2;                  // t <= u
    const int job = (int)(w / per_job);
    int64_t t, u;
    tri_point(w - (int64_t)job * per_job, cnt, t, u);
    const int64_t xp = min(t * sigma, P), xq = min(u * sigma, P);
    if (xp > xq) return;                          // the same for the whole CTA
    const MergeJob jb = p.jobs[job];
    const int16_t *U = reinterpret_cast<const int16_t *>(jb.U);
    const int16_t *L = reinterpret_cast<const int16_t *>(jb.L);
    const int gi = (int)grid_vertex_s(xp, n, p.gshift), gj = (int)grid_vertex_s(xq, n, p.gshift);
    const int64_t Ib = gi >> T_SHIFT, Jb = gj >> T_SHIFT;
    constexpr int PI = Fmt<int16_t>::P;
    constexpr int64_t EI = Fmt<int16_t>::ELEMS;
    const int ro = (gi & (T - 1)) * PI, co = (gj & (T - 1)) * PI;
    // Thread t takes offset 4 (t mod 16) of K-tiles Ib + t / 16, + 16, ..:
    // row_tile(Ib, kt) and col_tile(kt, Jb) both grow by one tile per K-tile,
    // so the two pointers advance by a constant.  A group of four k inside
    // [gi, gj] is added as two packed pairs (every value there is a DIST
    // entry in [0, 16383], so a pair's sum never carries across halves) and
    // kept by two packed maxima, one running maximum per k mod 4; a group cut
    // by the window's ends goes one k at a time.  Ties keep the first k of
    // each track: the leftmost maximiser.
    const int kl = (int)(threadIdx.x >> 4), o = 4 * (int)(threadIdx.x & 15);
    const int64_t step = (int64_t)(blockDim.x >> 4) * EI;
    const int16_t *up = U + row_tile(Ib, Ib + kl, p.NT) * EI + ro + o;
    const int16_t *lp = L + col_tile(Ib + kl, Jb) * EI + co + o;
    uint32_t bx = 0x80008000u, by = 0x80008000u;  // tracks k = 0, 1 (mod 4) and 2, 3
    int ix0 = INT32_MAX, ix1 = INT32_MAX, iy0 = INT32_MAX, iy1 = INT32_MAX;
    int best = INT32_MIN, bk = INT32_MAX;          // the cut groups
    for (int64_t kt = Ib + kl; kt <= Jb; kt += blockDim.x >> 4, up += step, lp += step) {
        const int kb = (int)(kt << T_SHIFT) + o;
        if (kb > gj) break;
        const uint2 uu = *reinterpret_cast<const uint2 *>(up);
        const uint2 ll = *reinterpret_cast<const uint2 *>(lp);
        if (kb >= gi && kb + 3 <= gj) {
            // A halfword of the running maximum changes only where the new
            // sum is strictly greater: its k is then the track's first.
            const uint32_t nx = __vmaxs2(bx, uu.x + ll.x), ny = __vmaxs2(by, uu.y + ll.y);
            const uint32_t cx = nx ^ bx, cy = ny ^ by;
            if (cx & 0xFFFFu) ix0 = kb;
            if (cx >> 16) ix1 = kb + 1;
            if (cy & 0xFFFFu) iy0 = kb + 2;
            if (cy >> 16) iy1 = kb + 3;
            bx = nx;
            by = ny;
        } else {
            const uint32_t uw[2] = {uu.x, uu.y}, lw[2] = {ll.x, ll.y};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = kb + e;
                const int v = (int)(int16_t)(uw[e >> 1] >> (16 * (e & 1))) + (int)(int16_t)(lw[e >> 1] >> (16 * (e & 1)));
                if (k >= gi && k <= gj && v > best) { best = v; bk = k; }
            }
        }
    }
    auto fold = [&](int v, int k) {
        if (k != INT32_MAX && (v > best || (v == best && k < bk))) { best = v; bk = k; }
    };
    fold((int)(int16_t)(bx & 0xFFFFu), ix0);
    fold((int)(int16_t)(bx >> 16), ix1);
    fold((int)(int16_t)(by & 0xFFFFu), iy0);
    fold((int)(int16_t)(by >> 16), iy1);
    warp_argmax(best, bk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sv[warp] = best; sk[warp] = bk; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (sv[q] > best || (sv[q] == best && sk[q] < bk)) { best = sv[q]; bk = sk[q]; }
        if (bk == INT32_MAX) { set_error(p.err, ERR_BOUNDS); bk = gi; best = 0; }
        jb.kgrid[xp * (P + 1) + xq] = bk;
        jb.vgrid[xp * (P + 1) + xq] = best;
    }
    __syncthreads();                              // sv, sk free again
}

// The full-scan level for int16 operands: a CTA per point, four k per load.
__global__ void __launch_bounds__(256) coarse_full16_kernel(MergeParams p) {
    pdl_wait_and_release();
    __shared__ int sv[8], sk[8];
    coarse_point_cta16(p, p.sigma, (int64_t)blockIdx.x, sv, sk);
}

cudaError_t launch_coarse(const MergeParams &p, int in_dtype, cudaStream_t st) {
    if (p.full) {
        const int64_t cnt = p.P / p.sigma + 1 + ((p.P % p.sigma) ? 1 : 0);
        const unsigned blocks = (unsigned)(cnt * (cnt + 1) / 2 * p.njobs);
        switch (in_dtype) {
            case DT_U8: return launch_pdl(coarse_full_kernel<uint8_t>, dim3(blocks), dim3(256), 0, st, p);
            case DT_I16: {
                // A CTA per point: its fixed cost (index, reduction) is per
                // warp, the scan's per k; short rows (n up to ~6000) take 4
                // warps, longer ones 8.
                const unsigned threads = p.n <= 6000 ? 128u : 256u;
                return launch_pdl(coarse_full16_kernel, dim3(blocks), dim3(threads), 0, st, p);
            }
            case DT_I32: return launch_pdl(coarse_full_kernel<int32_t>, dim3(blocks), dim3(256), 0, st, p);
            default: return cudaErrorInvalidValue;
        }
    }
    const int64_t cnt = p.P / p.sigma + 1 + ((p.P % p.sigma) ? 1 : 0);
    const int64_t warps = cnt * (cnt + 1) / 2 * p.njobs;
    int64_t blocks = ceil_div(warps, 8);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    switch (in_dtype) {
        case DT_U8: return launch_pdl(coarse_kernel<uint8_t>, dim3((unsigned)blocks), dim3(256), 0, st, p);
        case DT_I16: return launch_pdl(coarse_kernel<int16_t>, dim3((unsigned)blocks), dim3(256), 0, st, p);
        case DT_I32: return launch_pdl(coarse_kernel<int32_t>, dim3((unsigned)blocks), dim3(256), 0, st, p);
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ tile
constexpr int TP1 = T + 1;              // box points per side (with the far edge)
constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;

__host__ __device__ constexpr size_t align16c(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory band buffer of one K-tile: T+1 rows at the stored pitch.
template <typename V> struct Band {
    static constexpr int BUF = (int)(align16c((size_t)TP1 * Fmt<V>::P * sizeof(V)) / sizeof(V));
};

struct TileSmem {
    size_t ks, ds, us, ls, total;
};
__host__ __device__ inline TileSmem tile_smem_layout(int in_dt, int out_dt, int cap) {
    TileSmem s;
    const size_t in_sz = dt_bytes(in_dt), out_sz = dt_bytes(out_dt);
    const size_t buf = align16c((size_t)TP1 * tile_pitch(in_dt) * in_sz);
    size_t off = 16;                                  // mbarrier
    s.ks = off; off = align16c(off + (size_t)TP1 * TP1 * 4);
    s.ds = off; off = align16c(off + (size_t)T * tile_pitch(out_dt) * out_sz);
    s.us = off; off = align16c(off + (size_t)cap * buf);
    s.ls = off; off = align16c(off + (size_t)cap * buf);
    s.total = off;
    return s;
}

size_t tile_smem_bytes(int in_dtype, int out_dtype, int cap) {
    return tile_smem_layout(in_dtype, out_dtype, cap).total;
}

template <typename V> struct DtOf;
template <> struct DtOf<uint8_t> { static constexpr int v = DT_U8; };
template <> struct DtOf<int16_t> { static constexpr int v = DT_I16; };
template <> struct DtOf<int32_t> { static constexpr int v = DT_I32; };

// Number of s-grid points of [0, B] that are new at stride s (odd multiples
// of s below B) and old (even multiples below B, plus B itself).
__device__ __forceinline__ void level_counts(int B, int s, int &nnew, int &nold, int &neven) {
    const int ms = (B + s - 1) / s;     // multiples of s in [0, B)
    nnew = ms >> 1;
    neven = (ms + 1) >> 1;
    nold = neven + 1;
    if (B == 0) { nnew = 0; neven = 0; nold = 1; }
}
__device__ __forceinline__ int old_coord(int q, int neven, int s, int B) { return q < neven ? 2 * q * s : B; }

// Leftmost-argmax key of a candidate k: the value in the high half and the
// complement of k's offset in the low half, so the largest key has the largest
// value and, among equals, the smallest k (the tie rule of Algorithm 2).
template <typename TIn> struct Key { using type = uint32_t; static constexpr int SHIFT = 16; };
template <> struct Key<int32_t> { using type = uint64_t; static constexpr int SHIFT = 32; };

template <typename K> __device__ __forceinline__ K warp_max_key(K v);
template <> __device__ __forceinline__ uint32_t warp_max_key<uint32_t>(uint32_t v) {
    return __reduce_max_sync(0xFFFFFFFFu, v);
}
template <> __device__ __forceinline__ uint64_t warp_max_key<uint64_t>(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

// Operand access for the refinement: the staged shared-memory band, or the
// tile-packed matrices in global memory (tiles whose window fits no band).
template <typename TIn, bool SMEM> struct Operands;
template <typename TIn> struct Operands<TIn, true> {
    const TIn *Us, *Ls;
    int kbase;
    __device__ __forceinline__ int value(int x, int y, int k) const {
        const int off = k - kbase;
        const int e = (off >> T_SHIFT) * Band<TIn>::BUF + (off & (T - 1));
        return (int)Us[x * Fmt<TIn>::P + e] + (int)Ls[y * Fmt<TIn>::P + e];
    }
};
template <typename TIn> struct Operands<TIn, false> {
    const TIn *Ug, *Lg;
    int64_t NT;
    int ia, ja;
    __device__ __forceinline__ int value(int x, int y, int k) const {
        return (int)Ug[row_elem<TIn>(ia + x, k, NT)] + (int)Lg[col_elem<TIn>(k, ja + y)];
    }
};

// x / d for 0 <= x < 2^16 and 1 <= d <= 2^16 by one multiply-high
// (d > 1: m = ceil(2^32 / d) makes the quotient exact in that range).
struct FastDiv {
    uint32_t d, m;
    __device__ __forceinline__ explicit FastDiv(uint32_t dd)
        : d(dd), m(dd > 1 ? (uint32_t)((0x100000000ull + dd - 1) / dd) : 0u) {}
    __device__ __forceinline__ uint32_t div(uint32_t x) const { return d > 1 ? __umulhi(x, m) : x; }
};

// Coarse-to-fine refinement of K (and D) over the box [0, Bi] x [0, Bj] of a
// tile whose four corners are known.  Each level s first resolves the points
// with exactly one coordinate that is an odd multiple of s (bounded by the
// two neighbours at distance s along that coordinate), then the points with
// both (bounded by the four points just resolved).  Windows are short on
// average (about 1.9 candidates at s = 1, which holds three quarters of the
// points) but heavy-tailed (the 99th percentile is near 40), and a warp runs
// as long as its widest lane.  So a lane resolves its own point when the
// window has at most kLaneWindow candidates; wider points go to a shared-
// memory queue that whole warps then scan, lanes over k.  Keys carry
// (value, -k) so a plain max is the leftmost argmax.
constexpr int kLaneWindow = 16;
constexpr int kQueueCap = 512;

template <typename TIn, typename TOut, bool SMEM>
__device__ __forceinline__ void refine_tile(const Operands<TIn, SMEM> op, int32_t *Ks, TOut *Ds, int layout,
                                            int ia, int ja, int Bi, int Bj, int klo, int khi, int *err,
                                            uint32_t *queue, int *qcount) {
    using KeyT = typename Key<TIn>::type;
    constexpr int SH = Key<TIn>::SHIFT;
    constexpr KeyT LOW = (KeyT(1) << SH) - 1;
    constexpr int PO = Fmt<TOut>::P;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int kb = 0;
    if constexpr (SMEM) kb = op.kbase;
    const int ds_sx = layout == LAYOUT_COL ? 1 : PO, ds_sy = layout == LAYOUT_COL ? PO : 1;

    auto store = [&](int x, int y, bool found, int best, int bk) {
        if (!found) {                          // empty window: not a Monge input
            set_error(err, ERR_BOUNDS);
            best = 0;
        }
        if (best > MaxVal<TOut>::value) set_error(err, ERR_OVERFLOW);
        Ks[x * TP1 + y] = bk;
        if (x < T && y < T) Ds[x * ds_sx + y * ds_sy] = (TOut)best;
    };
    // One lane scans [lo, hi] (already clamped), left to right, one K-tile
    // segment at a time.  `vcap` bounds D(x, y) from above (D is monotone,
    // so a resolved neighbour above or to the right bounds it): the first k
    // that reaches vcap is the leftmost maximiser and ends the scan.
    auto lane_scan = [&](int x, int y, int lo, int hi, int vcap) {
        if constexpr (SMEM) {
            KeyT key = 0;
            int off = lo - kb;
            const int offhi = hi - kb;
            const TIn *ur = op.Us + x * Fmt<TIn>::P;
            const TIn *lr = op.Ls + y * Fmt<TIn>::P;
            bool done = false;
            while (off <= offhi && !done) {
                const int seg_end = min(offhi, off | (T - 1));
                const int e0 = (off >> T_SHIFT) * Band<TIn>::BUF + (off & (T - 1));
                const TIn *up = ur + e0;
                const TIn *lp = lr + e0;
                for (; off <= seg_end; ++off, ++up, ++lp) {
                    const int v = (int)*up + (int)*lp;
                    const KeyT c = ((KeyT)(uint32_t)v << SH) | (LOW - (KeyT)off);
                    key = c > key ? c : key;
                    if (v >= vcap) { done = true; break; }
                }
            }
            store(x, y, key != 0, (int)(key >> SH), key != 0 ? kb + (int)(LOW - (key & LOW)) : lo);
        } else {
            int best = INT32_MIN, bk = lo;
            for (int k = lo; k <= hi; ++k) {
                const int v = op.value(x, y, k);
                if (v > best) { best = v; bk = k; }
            }
            store(x, y, lo <= hi, best, bk);
        }
    };
    // D of a resolved owned point, or "no bound" for the far edges.
    auto dval = [&](int x, int y) -> int {
        return (x < T && y < T) ? (int)Ds[x * ds_sx + y * ds_sy] : INT32_MAX;
    };
    // Resolve or enqueue one point.
    auto point = [&](int x, int y, int lo, int hi, int vcap, int *qc) {
        if constexpr (SMEM) {
            lo = max(lo, klo);
            hi = min(hi, khi);
            if (hi - lo >= kLaneWindow) {
                const int slot = atomicAdd(qc, 1);
                if (slot < kQueueCap) {
                    // x, y < 128 and band offsets < 2^12 (cap <= 32 K-tiles).
                    queue[2 * slot] = (uint32_t)x | ((uint32_t)y << 8);
                    queue[2 * slot + 1] = (uint32_t)(lo - kb) | ((uint32_t)(hi - kb) << 16);
                    return;
                }
            }
        }
        lane_scan(x, y, lo, hi, vcap);
    };
    // Whole warps drain the queue (lanes over k).
    auto drain = [&](int count) {
        if constexpr (SMEM) {
            for (int q = warp; q < count; q += kTileWarps) {
                const uint32_t w0 = queue[2 * q], w1 = queue[2 * q + 1];
                const int x = (int)(w0 & 0xFF), y = (int)(w0 >> 8);
                const int lo = kb + (int)(w1 & 0xFFFF), hi = kb + (int)(w1 >> 16);
                KeyT key = 0;
                for (int k = lo + lane; k <= hi; k += 32) {
                    const KeyT c = ((KeyT)(uint32_t)op.value(x, y, k) << SH) | (LOW - (KeyT)(k - kb));
                    key = c > key ? c : key;
                }
                key = warp_max_key<KeyT>(key);
                if (lane == 0) store(x, y, key != 0, (int)(key >> SH), key != 0 ? kb + (int)(LOW - (key & LOW)) : lo);
            }
        }
    };

    int sub = 0;
    for (int s = T / 2; s >= 1; s >>= 1) {
        int nnx, nox, nex, nny, noy, ney;
        level_counts(Bi, s, nnx, nox, nex);
        level_counts(Bj, s, nny, noy, ney);
        const int cA = nnx * noy, cB = nox * nny, cC = nnx * nny;
        const FastDiv dnoy((uint32_t)noy), dnny((uint32_t)nny);
        for (int step = 0; step < 2; ++step, ++sub) {
            // Three rotating counters: the next sub-step's counter was last
            // read two sub-steps ago, and resetting it here is ordered
            // before its next use by the barrier below.
            int *qc = qcount + sub % 3;
            if (threadIdx.x == 0) qcount[(sub + 1) % 3] = 0;
            const int cnt = step == 0 ? cA + cB : cC;
            for (int idx = threadIdx.x; idx < cnt; idx += kTileThreads) {
                int x, y, lo, hi, vcap;
                if (step == 1) {                 // both coordinates new
                    const int qx = (int)dnny.div((uint32_t)idx), qy = idx - qx * nny;
                    x = (2 * qx + 1) * s;
                    y = (2 * qy + 1) * s;
                    const int xu = min(x + s, Bi), yu = min(y + s, Bj);
                    lo = max(Ks[x * TP1 + (y - s)], Ks[(x - s) * TP1 + y]);
                    hi = min(Ks[x * TP1 + yu], Ks[xu * TP1 + y]);
                    vcap = min(dval(x - s, y), dval(x, yu));
                } else if (idx < cA) {           // x new, y old
                    const int qx = (int)dnoy.div((uint32_t)idx), qy = idx - qx * noy;
                    x = (2 * qx + 1) * s;
                    y = qy < ney ? 2 * qy * s : Bj;
                    lo = Ks[(x - s) * TP1 + y];
                    hi = Ks[min(x + s, Bi) * TP1 + y];
                    vcap = dval(x - s, y);
                } else {                         // x old, y new
                    const int id2 = idx - cA;
                    const int qx = (int)dnny.div((uint32_t)id2), qy = id2 - qx * nny;
                    x = qx < nex ? 2 * qx * s : Bi;
                    y = (2 * qy + 1) * s;
                    const int yu = min(y + s, Bj);
                    lo = Ks[x * TP1 + (y - s)];
                    hi = Ks[x * TP1 + yu];
                    vcap = dval(x, yu);
                }
                const int i = ia + x, j = ja + y;
                if (i <= j) point(x, y, max(lo, i), min(hi, j), vcap, qc);
            }
            __syncthreads();
            const int queued = min(*qc, kQueueCap);
            if (queued > 0) {
                drain(queued);
                __syncthreads();
            }
        }
    }
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kTileThreads) tile_kernel(MergeParams p) {
    pdl_wait_and_release();
    constexpr int PI = Fmt<TIn>::P, PO = Fmt<TOut>::P;
    constexpr int EI = Fmt<TIn>::ELEMS, EO = Fmt<TOut>::ELEMS;
    constexpr int BUF = Band<TIn>::BUF;
    extern __shared__ __align__(128) unsigned char smem[];
    const TileSmem SL = tile_smem_layout(DtOf<TIn>::v, DtOf<TOut>::v, p.cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int32_t *Ks = reinterpret_cast<int32_t *>(smem + SL.ks);
    TOut *Ds = reinterpret_cast<TOut *>(smem + SL.ds);
    TIn *Us = reinterpret_cast<TIn *>(smem + SL.us);
    TIn *Ls = reinterpret_cast<TIn *>(smem + SL.ls);
    __shared__ int s_ok;
    __shared__ uint32_t s_queue[2 * kQueueCap];
    __shared__ int s_qcount[3];

    const int64_t NT = p.NT, P = p.P;
    const int n = (int)p.n;
    const MergeJob jb = p.jobs[blockIdx.y];
    // Tile index -> (I, J), row-major over the upper triangle of tiles.
    const int64_t tix = blockIdx.x;
    int64_t I;
    {
        int64_t lo = 0, hi = NT - 1;
        while (lo < hi) {                 // largest I with row_tile(I, I) <= tix
            const int64_t mid = (lo + hi + 1) >> 1;
            if (row_tile(mid, mid, NT) <= tix) lo = mid; else hi = mid - 1;
        }
        I = lo;
    }
    const int64_t J = I + (tix - row_tile(I, I, NT));
    const int ia = (int)(I * T), ja = (int)(J * T);
    const int Bi = min(ia + T, n) - ia, Bj = min(ja + T, n) - ja;
    const int64_t pa = I, pb = min(I + 1, P), qa = J, qb = min(J + 1, P);
    auto kcorner = [&](int64_t pp, int64_t qq) -> int {
        const int64_t gi = grid_vertex(pp, n), gj = grid_vertex(qq, n);
        return gi > gj ? (int)gj : jb.kgrid[pp * (P + 1) + qq];
    };
    int klo = kcorner(pa, qa), khi = kcorner(pb, qb);
    // K(ia, ja) lies in [ia, ja] and K(ib, jb) in [ib, jb]; anything else
    // means the inputs are not DIST matrices: flag it and stage nothing.
    const bool corners_ok = klo >= ia && klo <= ja && khi >= ia + Bi && khi <= ja + Bj && klo <= khi;
    if (!corners_ok) {
        if (threadIdx.x == 0) set_error(p.err, ERR_BOUNDS);
        klo = ia;
        khi = ja + Bj;
    }
    const int kt0 = klo >> T_SHIFT, kt1 = khi >> T_SHIFT;
    const int nK = kt1 - kt0 + 1;
    const int kbase = kt0 * T;
    // Two launches share the tiles: the main one (spill == 0) takes every
    // tile whose band fits p.cap K-tiles, the spill one (spill == 1, larger
    // band) the rest; a tile wider than even that reads global memory.
    // DIST is nonincreasing in i and nondecreasing in j (so is D), so the
    // tile's smallest value sits at its bottom-left corner (ib, ja) and its
    // largest at the top-right corner (ia, jb).  When the two agree (typical
    // far from the diagonal in low merges, where both halves saturate) the
    // tile is constant and needs neither staging nor refinement.
    bool constant = false;
    int cval = 0;
    if (p.const_tiles && corners_ok && I != J) {
        const int vmin = jb.vgrid[pb * (P + 1) + qa], vmax = jb.vgrid[pa * (P + 1) + qb];
        constant = vmin == vmax;
        cval = vmax;
    }
    if (constant) {
        if (p.spill == 1) return;            // the main launch writes it
        const int layout = jb.d_layout;
        if (layout == LAYOUT_DENSE) {
            TOut *out = reinterpret_cast<TOut *>(p.dense_out);
            const int rows = min(T, n + 1 - ia), cols = min(T, n + 1 - ja);
            for (int idx = threadIdx.x; idx < rows * T; idx += blockDim.x) {
                const int x = idx >> T_SHIFT, y = idx & (T - 1);
                if (y < cols) out[(int64_t)(ia + x) * p.ld + ja + y] = (TOut)cval;
            }
        } else {
            const int64_t tile = (layout == LAYOUT_COL) ? col_tile(I, J) : row_tile(I, J, NT);
            TOut *dst = reinterpret_cast<TOut *>(jb.D) + tile * EO;
            const TOut c = (TOut)cval;
            // 16-byte stores of the replicated value (EO * size is a multiple of 16).
            uint4 v;
            TOut *vp = reinterpret_cast<TOut *>(&v);
#pragma unroll
            for (int t = 0; t < (int)(16 / sizeof(TOut)); ++t) vp[t] = c;
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (int c4 = threadIdx.x; c4 < (int)(EO * sizeof(TOut) / 16); c4 += blockDim.x) d4[c4] = v;
        }
        return;
    }
    if (p.spill == 0 && corners_ok && nK > p.cap) return;
    if (p.spill == 1 && corners_ok && nK <= p.cap_main) return;
    const bool in_smem = corners_ok && nK <= p.cap;
    const TIn *Ug = reinterpret_cast<const TIn *>(jb.U);
    const TIn *Lg = reinterpret_cast<const TIn *>(jb.L);

    if (threadIdx.x == 0) {
        s_ok = 1;
        s_qcount[0] = 0;
        s_qcount[1] = 0;
        s_qcount[2] = 0;
        if (in_smem) {
            mbar_init(bar, 1);
            fence_mbar_init();
            const uint32_t tileB = (uint32_t)(EI * sizeof(TIn)), rowB = (uint32_t)(T * sizeof(TIn));
            const int ltop = min(kt1, (int)J);
            const int ufirst = max(kt0, (int)I + 1);
            const int ltop2 = min(kt1, (int)J + 1);
            uint32_t bytes = (uint32_t)nK * tileB + (uint32_t)(ltop - kt0 + 1) * tileB;
            if (Bi == T && kt1 >= ufirst) bytes += (uint32_t)(kt1 - ufirst + 1) * rowB;
            if (Bj == T) bytes += (uint32_t)(ltop2 - kt0 + 1) * rowB;
            mbar_arrive_expect_tx(bar, bytes);
            // Fault injection (tests only): the band of the launch's first
            // tile is announced on the barrier but never copied, so its wait
            // runs out and the tile reports ERR_TIMEOUT with nothing in flight.
            const bool held = p.hold_band && blockIdx.x == 0 && blockIdx.y == 0;
            for (int kt = kt0; kt <= kt1 && !held; ++kt) {
                TIn *dst = Us + (kt - kt0) * BUF;
                bulk_g2s(dst, Ug + row_tile(I, kt, NT) * EI, tileB, bar);
                if (Bi == T && kt >= ufirst) bulk_g2s(dst + T * PI, Ug + row_tile(I + 1, kt, NT) * EI, rowB, bar);
            }
            for (int kt = kt0; kt <= ltop && !held; ++kt)
                bulk_g2s(Ls + (kt - kt0) * BUF, Lg + col_tile(kt, J) * EI, tileB, bar);
            if (Bj == T && !held)
                for (int kt = kt0; kt <= ltop2; ++kt)
                    bulk_g2s(Ls + (kt - kt0) * BUF + T * PI, Lg + col_tile(kt, J + 1) * EI, rowB, bar);
        }
    }

    // Box initialisation (overlaps the copies).  Only a diagonal tile has
    // lower-triangle points; they hold j, the k <= j bound.  Every other
    // point is written before it is read.
    if (I == J) {
        for (int idx = threadIdx.x; idx < TP1 * TP1; idx += blockDim.x) {
            const int x = idx / TP1, y = idx - x * TP1;
            if (x > y) Ks[idx] = ja + y;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Ks[0] = klo;
        Ks[Bj] = kcorner(pa, qb);
        Ks[Bi * TP1] = kcorner(pb, qa);
        Ks[Bi * TP1 + Bj] = khi;
        // One thread waits for the band (bounded); the others park at the barrier.
        const uint64_t lim = p.wait_ns ? p.wait_ns : kWaitLimitNs;
        if (in_smem && !mbar_wait_bounded(bar, 0, lim)) {
            set_error(p.err, ERR_TIMEOUT);
            s_ok = 0;
            // Copies that are only late still land before the CTA's shared
            // memory is released (a second bounded wait).
            mbar_wait_bounded(bar, 0, lim);
        }
    }
    __syncthreads();
    if (!s_ok) return;           // a timed-out tile is skipped by every thread

    const int layout = jb.d_layout;
    // D at the corners that this tile owns (K known from the coarse grid).
    if (threadIdx.x < 4) {
        const int x = (threadIdx.x & 1) ? Bi : 0, y = (threadIdx.x & 2) ? Bj : 0;
        const bool dup = (threadIdx.x == 1 && Bi == 0) || (threadIdx.x == 2 && Bj == 0) ||
                         (threadIdx.x == 3 && (Bi == 0 || Bj == 0));
        if (!dup && x < T && y < T && ia + x <= ja + y) {
            const int k = Ks[x * TP1 + y];
            int v;
            if (in_smem) v = Operands<TIn, true>{Us, Ls, kbase}.value(x, y, k);
            else v = Operands<TIn, false>{Ug, Lg, NT, ia, ja}.value(x, y, k);
            Ds[layout == LAYOUT_COL ? y * PO + x : x * PO + y] = (TOut)v;
        }
    }
    __syncthreads();
    if (in_smem)
        refine_tile<TIn, TOut, true>(Operands<TIn, true>{Us, Ls, kbase}, Ks, Ds, layout, ia, ja, Bi, Bj, klo, khi,
                                     p.err, s_queue, s_qcount);
    else
        refine_tile<TIn, TOut, false>(Operands<TIn, false>{Ug, Lg, NT, ia, ja}, Ks, Ds, layout, ia, ja, Bi, Bj,
                                      klo, khi, p.err, s_queue, s_qcount);

    // Output.
    if (layout == LAYOUT_DENSE) {
        TOut *out = reinterpret_cast<TOut *>(p.dense_out);
        int32_t *Kout = p.dense_K;
        const int rows = min(T, n + 1 - ia), cols = min(T, n + 1 - ja);
        for (int idx = threadIdx.x; idx < rows * T; idx += blockDim.x) {
            const int x = idx >> T_SHIFT, y = idx & (T - 1);
            if (y >= cols) continue;
            const int64_t i = ia + x, j = ja + y;
            out[i * p.ld + j] = (i > j) ? Sentinel<TOut>::value : Ds[x * PO + y];
            if (Kout) Kout[i * p.ld + j] = (i > j) ? -1 : Ks[x * TP1 + y];
        }
    } else if (threadIdx.x == 0) {
        // TMA bulk store of the whole tile image (pitch included).
        const int64_t tile = (layout == LAYOUT_COL) ? col_tile(I, J) : row_tile(I, J, NT);
        fence_proxy_async_smem();
        bulk_s2g(reinterpret_cast<TOut *>(jb.D) + tile * EO, Ds, (uint32_t)(EO * sizeof(TOut)));
        bulk_commit();
        bulk_wait_read0();
    }
}

template <typename TIn, typename TOut>
static cudaError_t launch_tile_t(const MergeParams &p, cudaStream_t st) {
    const size_t smem = tile_smem_layout(DtOf<TIn>::v, DtOf<TOut>::v, p.cap).total;
    auto kern = tile_kernel<TIn, TOut>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)num_tiles_tri(p.NT), (unsigned)p.njobs);
    return launch_pdl(kern, grid, dim3(kTileThreads), smem, st, p);
}

cudaError_t launch_tile(const MergeParams &p, int in_dtype, int out_dtype, cudaStream_t st) {
#define LCS_TILE_CASE(TI, TO, DI, DO) \
    if (in_dtype == DI && out_dtype == DO) return launch_tile_t<TI, TO>(p, st);
    LCS_TILE_CASE(uint8_t, uint8_t, DT_U8, DT_U8)
    LCS_TILE_CASE(uint8_t, int16_t, DT_U8, DT_I16)
    LCS_TILE_CASE(uint8_t, int32_t, DT_U8, DT_I32)
    LCS_TILE_CASE(int16_t, int16_t, DT_I16, DT_I16)
    LCS_TILE_CASE(int16_t, int32_t, DT_I16, DT_I32)
    LCS_TILE_CASE(int32_t, int32_t, DT_I32, DT_I32)
    LCS_TILE_CASE(int32_t, int16_t, DT_I32, DT_I16)
#undef LCS_TILE_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ DPX max-plus tile
// For the merges of the tree the argmax is not needed (the traceback
// recomputes it from the retained children), only D.  Within a tile every
// K(i, j) lies in the band [K(ia, ja), K(ib, jb)] of the corners, so
//     D(i, j) = max over k in the band, k in [i, j], of U(i, k) + L(k, j),
// a (max,+) product of a 64 x W slice of U by a W x 64 slice of L.  It runs
// on the DPX instruction __viaddmax_s16x2 (max(a + b, c) on two int16
// lanes): the pair is taken along k, so a U row and an L column (a row of
// the column-layout L) feed it straight from the tile-packed layout, and each
// accumulator ends as max(low half, high half).  Entries with k < i (U) or
// k > j (L) are set to -16384 in shared memory first; with every DIST value
// at most 16383 such a sum stays negative.  Each of 128 threads owns an
// 8 x 4 block of outputs (rows ty + 8a, columns tx + 16b).
// The CTAs are persistent: a CTA takes every G-th tile of the launch (all
// jobs), warp 0 classifies 32 of them at a time (a lane per tile: corner
// argmax and values, constant or not, band), and thread 0 issues the bulk
// copies of the next staged tile's band as soon as the current tile's
// product has read the shared-memory band, so they land while the current
// tile is stored and the constant tiles in between are written.
constexpr int kDpxThreads = 128;
constexpr int kDpxCap = 2;
constexpr int16_t kNegInf16 = -16384;

struct DpxSmem {
    size_t ds, us, ls, total;
};
// The output tile is staged in shared memory only for a launch that writes
// the caller's dense matrix (`dense`); packed tiles go from registers to
// global memory.
__host__ __device__ inline DpxSmem dpx_smem_layout(int out_dt, int cap, bool dense) {
    DpxSmem s;
    const size_t tileb = (size_t)T * tile_pitch(DT_I16) * 2;   // 8704
    size_t off = 16;
    s.ds = off;
    if (dense) off = align16c(off + (size_t)T * tile_pitch(out_dt) * dt_bytes(out_dt));
    s.us = off; off = align16c(off + (size_t)cap * tileb);
    s.ls = off; off = align16c(off + (size_t)cap * tileb);
    s.total = off;
    return s;
}

// Rows [0, rows) of an output tile into the caller's dense matrix, entry
// (x, y) = val(x, y).  A tile whose T columns all exist is written with
// 16-byte stores (its rows start 16-byte aligned: ld and the column offset
// are multiples of 16 bytes), which matters when the matrix is pinned host
// memory written over the CPU-GPU link; the last tile column element-wise.
template <typename TOut, typename F>
__device__ __forceinline__ void store_dense_tile(TOut *out, int64_t ld, int64_t ia, int64_t ja, int rows, int cols,
                                                 F val) {
    constexpr int E = 16 / (int)sizeof(TOut);   // elements per 16-byte word
    constexpr int WPR = T / E;                  // words per tile row
    if (cols == T) {
        for (int idx = threadIdx.x; idx < rows * WPR; idx += blockDim.x) {
            const int x = idx / WPR, y0 = (idx % WPR) * E;
            uint4 v4;
            TOut *vp = reinterpret_cast<TOut *>(&v4);
#pragma unroll
            for (int e = 0; e < E; ++e) vp[e] = val(x, y0 + e);
            *reinterpret_cast<uint4 *>(out + (ia + x) * ld + ja + y0) = v4;
        }
    } else {
        for (int idx = threadIdx.x; idx < rows * T; idx += blockDim.x) {
            const int x = idx >> T_SHIFT, y = idx & (T - 1);
            if (y < cols) out[(ia + x) * ld + ja + y] = val(x, y);
        }
    }
}

// A tile of the launch as classified by warp 0.
struct DpxMeta {
    int32_t job, I, J;
    int32_t kl, kh;            // band of k (inclusive)
    int32_t cst;               // corner values agree: constant `val`
    int32_t val;
    int32_t valid;             // a tile of this CTA (else past the end)
    int32_t va;                // D at the top-left corner (ia, ja)
    int32_t ok;                // corners are a DIST merge's (else the band is every k)
};

template <typename TOut>
__global__ void __launch_bounds__(kDpxThreads) tile_dpx_kernel(MergeParams p) {
    pdl_wait_and_release();
    using TIn = int16_t;
    constexpr int PI = Fmt<TIn>::P, PO = Fmt<TOut>::P;
    constexpr int EI = Fmt<TIn>::ELEMS, EO = Fmt<TOut>::ELEMS;
    constexpr uint32_t tileB = (uint32_t)(EI * sizeof(TIn));
    extern __shared__ __align__(128) unsigned char smem[];
    const DpxSmem SL = dpx_smem_layout(DtOf<TOut>::v, p.cap, p.dense_out != nullptr);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    TOut *Ds = reinterpret_cast<TOut *>(smem + SL.ds);
    TIn *Us = reinterpret_cast<TIn *>(smem + SL.us);
    TIn *Ls = reinterpret_cast<TIn *>(smem + SL.ls);
    __shared__ int s_ok;
    __shared__ DpxMeta s_meta[32];
    __shared__ int64_t s_grab;

    const int64_t NT = p.NT, P = p.P;
    const int n = (int)p.n;
    const int64_t tiles = num_tiles_tri(NT), total = tiles * p.njobs, G = gridDim.x;
    const int knT = n >> T_SHIFT, kn = n & (T - 1);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lane = threadIdx.x & 31;
    const uint64_t lim = p.wait_ns ? p.wait_ns : kWaitLimitNs;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // Thread 0's view of the staging buffer: the K-tiles it holds (or is
    // loading) and the barrier parity to wait for.
    int st_tile = -1, st_c0 = -1;             // batch slot and first K-tile staged
    uint32_t phase = 0;
    auto issue = [&](const DpxMeta &m, int c0) {
        const int c1 = min(m.kh >> T_SHIFT, c0 + p.cap - 1);
        const MergeJob jb = p.jobs[m.job];
        const TIn *Ug = reinterpret_cast<const TIn *>(jb.U);
        const TIn *Lg = reinterpret_cast<const TIn *>(jb.L);
        mbar_arrive_expect_tx(bar, 2u * (uint32_t)(c1 - c0 + 1) * tileB);
        for (int kt = c0; kt <= c1; ++kt) {
            bulk_g2s(Us + (kt - c0) * EI, Ug + row_tile(m.I, kt, NT) * EI, tileB, bar);
            bulk_g2s(Ls + (kt - c0) * EI, Lg + col_tile(kt, m.J) * EI, tileB, bar);
        }
    };

    // First K-tile of a tile's top chunk: chunks of p.cap K-tiles aligned at
    // the band's first K-tile.
    auto top_chunk = [&](const DpxMeta &m) {
        const int t0 = m.kl >> T_SHIFT;
        return t0 + (((m.kh >> T_SHIFT) - t0) / p.cap) * p.cap;
    };

    // Batches of tiles: with a counter, p.grab (1..32) consecutive tiles
    // taken from it (tile costs differ by orders of magnitude -- constant
    // tiles read nothing, wide bands stream several chunks -- so a static
    // split leaves SMs idle at the end); without one, 32 tiles strided by the
    // grid.
    const int64_t bstride = p.sched ? 1 : G;
    const int bcount = p.sched ? p.grab : 32;
    for (int64_t it = 0;; ++it) {
        __syncthreads();                       // the previous batch's metadata is consumed
        int64_t b0;
        if (p.sched) {
            if (threadIdx.x == 0) s_grab = (int64_t)atomicAdd(p.sched, (unsigned)bcount);
            __syncthreads();
            b0 = s_grab;
        } else {
            b0 = blockIdx.x + it * 32 * G;
        }
        if (b0 >= total) break;
        if (threadIdx.x < 32) {
            // Lane l classifies tile b0 + l * bstride.
            const int64_t g = b0 + lane * bstride;
            DpxMeta m{};
            if (lane < bcount && g < total) {
                m.valid = 1;
                m.job = (int)(g / tiles);
                const int64_t tix = g - m.job * tiles;
                int64_t lo = 0, hi = NT - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (row_tile(mid, mid, NT) <= tix) lo = mid; else hi = mid - 1;
                }
                m.I = (int)lo;
                m.J = (int)(lo + (tix - row_tile(lo, lo, NT)));
                const MergeJob jb = p.jobs[m.job];
                const int ia = m.I * T, ja = m.J * T;
                const int Bi = min(ia + T, n) - ia, Bj = min(ja + T, n) - ja;
                const int64_t pa = m.I, pb = (m.I + 1 < P) ? m.I + 1 : P, qa = m.J, qb = (m.J + 1 < P) ? m.J + 1 : P;
                auto kcorner = [&](int64_t pp, int64_t qq) -> int {
                    const int64_t gi = grid_vertex(pp, n), gj = grid_vertex(qq, n);
                    return gi > gj ? (int)gj : jb.kgrid[pp * (P + 1) + qq];
                };
                const int klo = kcorner(pa, qa), khi = kcorner(pb, qb);
                const int vmin = jb.vgrid[pb * (P + 1) + qa], vmax = jb.vgrid[pa * (P + 1) + qb];
                const bool ok = klo >= ia && klo <= ja && khi >= ia + Bi && khi <= ja + Bj && klo <= khi;
                m.cst = (ok && m.I != m.J && vmin == vmax) ? 1 : 0;
                m.val = vmax;
                // Band [klo, khi], k <= ja + T - 1 for owned columns.  Corners
                // that are not a DIST's (invalid input) fall back to every k
                // of the tile, [ia, ja + T - 1], and are flagged.
                m.kl = ok ? klo : ia;
                m.kh = ok ? min(khi, ja + T - 1) : min(ja + T - 1, n);
                m.va = jb.vgrid[pa * (P + 1) + qa];
                m.ok = ok ? 1 : 0;
                if (!ok) set_error(p.err, ERR_BOUNDS);
            }
            s_meta[lane] = m;
        }
        __syncthreads();
        for (int l = 0; l < 32; ++l) {
            const DpxMeta m = s_meta[l];
            if (!m.valid) break;
            const MergeJob jb = p.jobs[m.job];
            const int layout = jb.d_layout;
            const bool col_out = layout == LAYOUT_COL;
            const int ia = m.I * T, ja = m.J * T;
            if (m.cst) {
                // Constant tile: written here, nothing staged.
                if (layout == LAYOUT_DENSE) {
                    const TOut cv = (TOut)m.val;
                    store_dense_tile<TOut>(reinterpret_cast<TOut *>(p.dense_out), p.ld, ia, ja, min(T, n + 1 - ia),
                                           min(T, n + 1 - ja), [&](int, int) { return cv; });
                } else {
                    const int64_t tile = (layout == LAYOUT_COL) ? col_tile(m.I, m.J) : row_tile(m.I, m.J, NT);
                    uint4 v4;
                    TOut *vp = reinterpret_cast<TOut *>(&v4);
#pragma unroll
                    for (int k = 0; k < (int)(16 / sizeof(TOut)); ++k) vp[k] = (TOut)m.val;
                    uint4 *d4 = reinterpret_cast<uint4 *>(reinterpret_cast<TOut *>(jb.D) + tile * EO);
                    for (int c4 = threadIdx.x; c4 < (int)(EO * sizeof(TOut) / 16); c4 += blockDim.x) d4[c4] = v4;
                }
                continue;
            }
            const int kt0 = m.kl >> T_SHIFT, ktop = m.kh >> T_SHIFT;
            int kbeg = m.kl & ~3;
            const int kend = m.kh | 3;
            uint32_t acc[8][4];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0xC000C000u;
            // The band streams through shared memory p.cap K-tiles at a time
            // (one chunk for most tiles), from its top chunk down, with the
            // chunks aligned at kt0; accumulators persist.
            //
            // The band's low end: x, the largest maximiser of the corner
            // (ia, ja) that is <= kh (kh is the smallest maximiser of the far
            // corner).  For every entry (i, j) of the tile a maximiser below x
            // can be replaced by x and one above kh by kh (Monge), so [x, kh]
            // keeps a maximiser of every entry.  U's row ia and L's column ja
            // are row 0 of the staged K-tiles: warp 0 searches each staged
            // chunk that holds k <= ja from the top down for the largest k
            // with U(ia, k) + L(k, ja) = D(ia, ja); the chunk that holds it is
            // the last one the tile needs.
            bool narrowed = !m.ok;             // corners that are not a DIST merge's: the whole band
            for (int c0 = top_chunk(m);; c0 -= p.cap) {
                const int c1 = min(ktop, c0 + p.cap - 1);
                if (threadIdx.x == 0) {
                    if (!(st_tile == l && st_c0 == c0)) issue(m, c0);   // not prefetched
                    st_tile = -1;
                    s_ok = 1;
                    if (!mbar_wait_bounded(bar, phase, lim)) {
                        set_error(p.err, ERR_TIMEOUT);
                        s_ok = 0;
                        // Before the early return: copies that are only late
                        // land (a second bounded wait), and no bulk copy of
                        // this CTA is left in flight.
                        mbar_wait_bounded(bar, phase, lim);
                        bulk_wait_all0();
                    }
                    phase ^= 1u;
                }
                __syncthreads();
                if (!s_ok) return;
                // Mask k < i in U's diagonal tile, k > j in L's diagonal tile,
                // and every k > n (stored tiles carry unspecified values past
                // the last vertex).  Masked + masked = -32768 still fits
                // int16; a sentinel or stale value could wrap, so none is
                // left in the band.
                bool masked = false;
                for (int kt = c0; kt <= c1; ++kt) {
                    const bool mu = kt == m.I || kt == knT, ml = kt == m.J || kt == knT;
                    if (!mu && !ml) continue;
                    masked = true;
                    TIn *Ut = Us + (kt - c0) * EI;
                    TIn *Lt = Ls + (kt - c0) * EI;
                    for (int idx = threadIdx.x; idx < T2; idx += blockDim.x) {
                        const int r = idx >> T_SHIFT, c = idx & (T - 1);
                        if (mu && ((kt == m.I && c < r) || (kt == knT && c > kn))) Ut[r * PI + c] = kNegInf16;
                        if (ml && ((kt == m.J && c > r) || (kt == knT && c > kn))) Lt[r * PI + c] = kNegInf16;
                    }
                }
                if (masked) __syncthreads();
                if (!narrowed && c0 * T <= ja) {
                    // Every warp runs the same search on the same staged
                    // data (a ballot or two), so no barrier hands x over.
                    const int top = min(min(m.kh, ja), c1 * T + T - 1), bot = max(m.kl, c0 * T);
                    int x = -1;
                    for (int t = top; t >= bot && x < 0; t -= 32) {
                        const int k = t - lane;
                        bool hit = false;
                        if (k >= bot) {
                            const int o = ((k >> T_SHIFT) - c0) * EI + (k & (T - 1));
                            hit = (int)Us[o] + (int)Ls[o] == m.va;
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, hit);
                        if (bal) x = t - (__ffs(bal) - 1);
                    }
                    if (x >= 0) {
                        kbeg = x & ~3;
                        narrowed = true;
                    }
                }
                const bool last = narrowed || c0 == kt0;
                for (int kt = max(c0, kbeg >> T_SHIFT); kt <= min(c1, kend >> T_SHIFT); ++kt) {
                    const int lo = max(kbeg, kt * T) & (T - 1), hi = min(kend, kt * T + T - 1) & (T - 1);
                    // Thread (tx, ty) owns the 8 x 4 entries at stored-tile
                    // rows ty + 8a and columns tx + 16b of the output image:
                    // D rows x of U's rows and D columns y of L's stored rows
                    // in row (and dense) layout, transposed in column layout,
                    // so that the 16 lanes of a half-warp store consecutive
                    // elements either way.  (max,+) is symmetric in its two
                    // operands, so only the roles of the staged tiles swap.
                    const TIn *Ab = (col_out ? Ls : Us) + (kt - c0) * EI + ty * PI;
                    const TIn *Bb = (col_out ? Us : Ls) + (kt - c0) * EI + tx * PI;
                    // Four k per step; the next step's operands load while
                    // this step computes, and the two k pairs of a step go
                    // through all 32 accumulators in turn, so that dependent
                    // DPX instructions are 32 apart.
                    uint2 u[8], lv[4];
#pragma unroll
                    for (int a = 0; a < 8; ++a) u[a] = *reinterpret_cast<const uint2 *>(Ab + a * 8 * PI + lo);
#pragma unroll
                    for (int b = 0; b < 4; ++b) lv[b] = *reinterpret_cast<const uint2 *>(Bb + b * 16 * PI + lo);
                    for (int kk = lo; kk <= hi; kk += 4) {
                        const int kn = kk + 4 <= hi ? kk + 4 : kk;   // stays inside the staged tile
                        uint2 un[8], ln[4];
#pragma unroll
                        for (int a = 0; a < 8; ++a) un[a] = *reinterpret_cast<const uint2 *>(Ab + a * 8 * PI + kn);
#pragma unroll
                        for (int b = 0; b < 4; ++b) ln[b] = *reinterpret_cast<const uint2 *>(Bb + b * 16 * PI + kn);
#pragma unroll
                        for (int a = 0; a < 8; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[a][b] = __viaddmax_s16x2(u[a].x, lv[b].x, acc[a][b]);
#pragma unroll
                        for (int a = 0; a < 8; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[a][b] = __viaddmax_s16x2(u[a].y, lv[b].y, acc[a][b]);
#pragma unroll
                        for (int a = 0; a < 8; ++a) u[a] = un[a];
#pragma unroll
                        for (int b = 0; b < 4; ++b) lv[b] = ln[b];
                    }
                }
                __syncthreads();                // the band is read
                if (threadIdx.x == 0) {
                    if (!last) {
                        issue(m, c0 - p.cap);   // next chunk of this tile, below
                        st_tile = l;
                        st_c0 = c0 - p.cap;
                    } else {
                        // Prefetch the next staged tile of the batch.
                        for (int l2 = l + 1; l2 < 32; ++l2) {
                            const DpxMeta m2 = s_meta[l2];
                            if (!m2.valid) break;
                            if (m2.cst) continue;
                            issue(m2, top_chunk(m2));
                            st_tile = l2;
                            st_c0 = top_chunk(m2);
                            break;
                        }
                    }
                }
                if (last) break;
            }
            if (layout == LAYOUT_DENSE) {
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int v = max((int)(int16_t)(acc[a][b] & 0xFFFFu), (int)(int16_t)(acc[a][b] >> 16));
                        Ds[(ty + 8 * a) * PO + tx + 16 * b] = (TOut)v;
                    }
                __syncthreads();
                store_dense_tile<TOut>(reinterpret_cast<TOut *>(p.dense_out), p.ld, ia, ja, min(T, n + 1 - ia),
                                       min(T, n + 1 - ja), [&](int x, int y) {
                                           return ia + x > ja + y ? Sentinel<TOut>::value : Ds[x * PO + y];
                                       });
                __syncthreads();                // Ds read before the next tile writes it
            } else {
                // The tile image straight from the accumulators: entry
                // (ty + 8a, tx + 16b) of the stored tile (rows past n and
                // below the diagonal carry unspecified values, as in every
                // stored tile).
                const int64_t tile = col_out ? col_tile(m.I, m.J) : row_tile(m.I, m.J, NT);
                TOut *dt = reinterpret_cast<TOut *>(jb.D) + tile * EO + ty * PO + tx;
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int v = max((int)(int16_t)(acc[a][b] & 0xFFFFu), (int)(int16_t)(acc[a][b] >> 16));
                        dt[a * 8 * PO + b * 16] = (TOut)v;
                    }
            }
        }
    }
    if (threadIdx.x == 0) {
        // A copy still in flight (prefetched past an error) lands before the
        // CTA's shared memory goes away.
        if (st_tile >= 0 && !mbar_wait_bounded(bar, phase, lim)) set_error(p.err, ERR_TIMEOUT);
        bulk_wait_all0();
    }
}

template <typename TOut>
static cudaError_t launch_dpx_t(const MergeParams &p, cudaStream_t st) {
    const size_t smem = dpx_smem_layout(DtOf<TOut>::v, p.cap, p.dense_out != nullptr).total;
    auto kern = tile_dpx_kernel<TOut>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDpxThreads, smem)) != cudaSuccess) return e;
    const int64_t work = p.njobs * num_tiles_tri(p.NT);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)sms * std::max(per_sm, 1)));
    // Tiles per grab: larger grabs amortise the classification's load
    // latency, smaller ones shorten the tail; measured best at 2 with ~20
    // tiles per CTA (4096) and 4-8 with ~1000 (16384).
    MergeParams q = p;
    const int64_t per_cta = work / grid;
    q.grab = per_cta >= 96 ? 8 : per_cta >= 48 ? 4 : per_cta >= 16 ? 2 : 1;
    return launch_pdl(kern, dim3((unsigned)grid), dim3(kDpxThreads), smem, st, q);
}

cudaError_t launch_tile_dpx(MergeParams p, int out_dtype, cudaStream_t st) {
    p.spill = 0;
    p.cap = kDpxCap;
    if (out_dtype == DT_I16) return launch_dpx_t<int16_t>(p, st);
    if (out_dtype == DT_I32) return launch_dpx_t<int32_t>(p, st);
    return cudaErrorInvalidValue;
}

static size_t band_bytes(int in_dt) { return align16c((size_t)TP1 * tile_pitch(in_dt) * dt_bytes(in_dt)); }

int tile_cap_main(int in_dtype) { return in_dtype == DT_I32 ? 2 : 4; }

int tile_cap_spill(int in_dtype, int out_dtype) {
    // 227 KB per block, minus the kernel's static shared memory (the queue).
    const size_t limit = 227 * 1024 - (2 * kQueueCap + 8) * 4 - 64;
    const size_t fixed = tile_smem_layout(in_dtype, out_dtype, 0).total;
    const size_t cap = (limit - fixed) / (2 * band_bytes(in_dtype));
    return (int)(cap > 32 ? 32 : cap);
}

cudaError_t launch_tile_pair(MergeParams p, int in_dtype, int out_dtype, cudaStream_t st) {
    const int cap_main = tile_cap_main(in_dtype);
    p.spill = 0;
    p.cap = cap_main;
    p.cap_main = cap_main;
    cudaError_t e = launch_tile(p, in_dtype, out_dtype, st);
    if (e != cudaSuccess) return e;
    p.spill = 1;
    p.cap = tile_cap_spill(in_dtype, out_dtype);
    return launch_tile(p, in_dtype, out_dtype, st);
}

// ------------------------------------------------------------------ pack
// Dense (n+1) x ld -> tile-packed (one CTA per tile I <= J); the column
// layout transposes each tile through shared memory.
template <typename V>
__global__ void __launch_bounds__(256) pack_kernel(const V *src, int64_t ld, int64_t n, int64_t NT,
                                                   V *dst, int layout) {
    pdl_wait_and_release();
    constexpr int P = Fmt<V>::P, E = Fmt<V>::ELEMS;
    __shared__ V tile[T][T + 1];
    const int64_t tix = blockIdx.x;
    int64_t lo = 0, hi = NT - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (row_tile(mid, mid, NT) <= tix) lo = mid; else hi = mid - 1;
    }
    const int64_t I = lo, J = I + (tix - row_tile(I, I, NT));
    for (int idx = threadIdx.x; idx < T2; idx += blockDim.x) {
        const int x = idx >> T_SHIFT, y = idx & (T - 1);
        const int64_t i = I * T + x, j = J * T + y;
        tile[x][y] = (i <= n && j <= n) ? src[i * ld + j] : (V)0;
    }
    __syncthreads();
    V *d = dst + ((layout == LAYOUT_COL) ? col_tile(I, J) : row_tile(I, J, NT)) * E;
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) {
        const int r = idx / P, c = idx - r * P;
        V v = (V)0;
        if (c < T) v = (layout == LAYOUT_COL) ? tile[c][r] : tile[r][c];
        d[idx] = v;
    }
}

cudaError_t launch_pack(const void *src, int dtype, int64_t n, int64_t ld, void *dst, int layout,
                        cudaStream_t st) {
    const int64_t NT = num_tiles_side(n);
    const unsigned blocks = (unsigned)num_tiles_tri(NT);
    if (dtype == DT_I32)
        return launch_pdl(pack_kernel<int32_t>, dim3(blocks), dim3(256), 0, st, (const int32_t *)src, ld, n, NT,
                          (int32_t *)dst, layout);
    else if (dtype == DT_I16)
        return launch_pdl(pack_kernel<int16_t>, dim3(blocks), dim3(256), 0, st, (const int16_t *)src, ld, n, NT,
                          (int16_t *)dst, layout);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dense fill
template <typename V>
__global__ void fill_dense_kernel(V *out, int64_t n, int64_t ld, V lower, V upper, int fill_upper,
                                  int32_t *K) {
    pdl_wait_and_release();
    for (int64_t i = blockIdx.x; i <= n; i += gridDim.x) {
        // Lower triangle outside the diagonal tile: columns [0, (i/T)*T).
        const int64_t jl = fill_upper ? i : ((i >> T_SHIFT) << T_SHIFT);
        for (int64_t j = threadIdx.x; j < jl; j += blockDim.x) {
            out[i * ld + j] = lower;
            if (K) K[i * ld + j] = -1;
        }
        if (fill_upper)
            for (int64_t j = i + threadIdx.x; j <= n; j += blockDim.x) out[i * ld + j] = upper;
    }
}

template <typename V>
__global__ void __launch_bounds__(256) fill_lower_kernel(V *out, int64_t n, int64_t ld, V lower) {
    pdl_wait_and_release();
    uint4 v4;
    V *vp = reinterpret_cast<V *>(&v4);
#pragma unroll
    for (int k = 0; k < (int)(16 / sizeof(V)); ++k) vp[k] = lower;
    for (int64_t i = blockIdx.x; i <= n; i += gridDim.x) {
        // Columns [0, (i / T) T): whole 16-byte words (T elements are 64 or
        // 128 bytes), starting at a 16-byte aligned row.
        const int64_t words = ((i >> T_SHIFT) << T_SHIFT) * (int64_t)sizeof(V) / 16;
        uint4 *row = reinterpret_cast<uint4 *>(out + i * ld);
        for (int64_t w = threadIdx.x; w < words; w += blockDim.x) row[w] = v4;
    }
}

cudaError_t launch_fill_lower(void *out, int dtype, int64_t n, int64_t ld, int lower, int blocks, cudaStream_t st) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, n + 1));
    if (dtype == DT_I32)
        return launch_pdl(fill_lower_kernel<int32_t>, dim3(g), dim3(256), 0, st, (int32_t *)out, n, ld,
                          (int32_t)lower);
    if (dtype == DT_I16)
        return launch_pdl(fill_lower_kernel<int16_t>, dim3(g), dim3(256), 0, st, (int16_t *)out, n, ld,
                          (int16_t)lower);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fill_dense(void *out, int dtype, int64_t n, int64_t ld, int lower, int upper,
                              int fill_upper, int32_t *K, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 1) < 8192 ? (n + 1) : 8192);
    if (dtype == DT_I32)
        return launch_pdl(fill_dense_kernel<int32_t>, dim3(blocks), dim3(256), 0, st, (int32_t *)out, n, ld,
                          (int32_t)lower, (int32_t)upper, fill_upper, K);
    if (dtype == DT_I16)
        return launch_pdl(fill_dense_kernel<int16_t>, dim3(blocks), dim3(256), 0, st, (int16_t *)out, n, ld,
                          (int16_t)lower, (int16_t)upper, fill_upper, K);
    return cudaErrorInvalidValue;
}

}  // namespace lcsg
