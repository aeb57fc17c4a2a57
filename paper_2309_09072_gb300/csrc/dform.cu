// dform.cu -- the breakout (D-form) representation of a strip's DIST.
//
// D(i, w) = min{ j >= i : DIST(i, j) >= w } is the leftmost bottom vertex
// reached from top vertex i by a path of weight w (Sec. II-B-1), D(i, 0) = i,
// and "infinity" (the dtype's maximum) when no path from i reaches weight w.
// A strip of h rows needs (n+1) x (h+1) entries instead of the (n+1)^2 of
// its DIST.  Two stacked strips combine as (Sec. II-B-3)
//     D(i, w) = min_{0 <= k <= w} D_L(D_U(i, k), w - k),
// terms with D_U(i, k) infinite or w - k above L's height left out.
//
// Strip: the strip builder's bit-vector sweep (strip.cu) run from each
// source, a lane per source, every strip of a in one launch; the carry out
// of the top row at column j is the unit step DIST(i, j) - DIST(i, j-1), so
// column j is the next breakout.
//
// Merge: for one top vertex i the terms form a matrix M(k, w) =
// D_L(D_U(i, k), w - k) whose leftmost minimising row is nondecreasing in w
// (the monotone matrix of Sec. II-B-1 that Algorithm 1 exploits).  Algorithm
// 1 finds column minima by recursive halving of the columns; here the
// recursion is cut to two levels that suit a warp: the exact leftmost
// minimum of every 32nd column (lanes over rows, a warp reduction), then
// the 31 columns between two such columns, a lane each, scanning only the
// rows between the two known minimisers -- the same rows for every lane, so
// D_U(i, k) is a broadcast and D_L's row is read by consecutive lanes at
// consecutive columns.
#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

template <typename V> struct DInf;
template <> struct DInf<int32_t> { static constexpr int32_t value = INT32_MAX; };
template <> struct DInf<int16_t> { static constexpr int16_t value = INT16_MAX; };

// ------------------------------------------------------------------ strip
constexpr int kDfWarps = 4;

template <typename V, int W>
__global__ void __launch_bounds__(kDfWarps * 32) dform_strip_kernel(DformStripParams p) {
    pdl_wait_and_release();
    extern __shared__ __align__(16) uint32_t dmasks[];     // [256][W] row masks per letter
    const int64_t r0 = (int64_t)blockIdx.y * p.h;           // strip blockIdx.y: rows r0 .. r0 + hs - 1
    const int hs = (int)min((int64_t)p.h, p.m - r0);
    for (int t = threadIdx.x; t < 256 * W; t += blockDim.x) dmasks[t] = 0u;
    __syncthreads();
    for (int r = threadIdx.x; r < hs; r += blockDim.x)
        atomicOr(&dmasks[p.a[r0 + r] * W + (r >> 5)], 1u << (r & 31));
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * kDfWarps + warp) * 32;
    if (i0 > p.n) return;
    const int64_t i = i0 + lane;
    const bool live = i <= p.n;
    V *row = reinterpret_cast<V *>(p.out) + ((int64_t)blockIdx.y * (p.n + 1) + (live ? i : 0)) * p.ld;
    if (live) row[0] = (V)i;
    uint32_t Vb[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Vb[w] = 0xFFFFFFFFu;
    int d = 0;
    // Columns in blocks of 32: one coalesced load of the block's letters (a
    // lane each), then a shuffle per column; the loop is partly unrolled so
    // that the next columns' masks load while a column steps.
    for (int64_t jb = i0 + 1; jb <= p.n; jb += 32) {
        if (__all_sync(0xFFFFFFFFu, !live || d >= hs)) break;      // every source saturated
        const int64_t jl = jb + lane;
        const int myc = jl <= p.n ? (int)p.b[jl - 1] : 0;
        const int cnt = (int)min((int64_t)32, p.n - jb + 1);
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            const int ch = __shfl_sync(0xFFFFFFFFu, myc, t);
            const int64_t j = jb + t;
            const bool step = live && j > i;
            uint32_t M[W];
#pragma unroll
            for (int w = 0; w < W; ++w) M[w] = step ? dmasks[ch * W + w] : 0u;   // no mask: V unchanged, no carry
            if (column_step<W>(Vb, M)) {
                ++d;
                row[d] = (V)j;
            }
        }
    }
    if (live)
        for (int w = d + 1; w <= p.h; ++w) row[w] = DInf<V>::value;   // a shorter last strip: also past hs
}

template <typename V, int W>
static cudaError_t launch_dfs(const DformStripParams &p, cudaStream_t st) {
    const unsigned blocks = (unsigned)ceil_div(p.n + 1, 32 * kDfWarps);
    const unsigned strips = (unsigned)ceil_div(p.m, p.h);
    return launch_pdl(dform_strip_kernel<V, W>, dim3(blocks, strips), dim3(kDfWarps * 32), (size_t)256 * W * 4, st, p);
}

cudaError_t launch_dform_strip(const DformStripParams &p, int dtype, int words, cudaStream_t st) {
#define LCS_DFS(V)                                          \
    switch (words) {                                        \
        case 1: return launch_dfs<V, 1>(p, st);             \
        case 2: return launch_dfs<V, 2>(p, st);             \
        case 4: return launch_dfs<V, 4>(p, st);             \
        case 8: return launch_dfs<V, 8>(p, st);             \
        default: return cudaErrorInvalidValue;              \
    }
    if (dtype == DT_I32) { LCS_DFS(int32_t) }
    if (dtype == DT_I16) { LCS_DFS(int16_t) }
#undef LCS_DFS
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ merge
constexpr int kDmWarps = 4;
constexpr int kDmStride = 32;                 // sampled columns: every 32nd, and the last

template <typename V>
__global__ void __launch_bounds__(kDmWarps * 32) dform_merge_kernel(DformMergeParams p) {
    pdl_wait_and_release();
    extern __shared__ int32_t kmin_all[];     // [warps][samples] leftmost minimiser of each sampled column
    constexpr int INF = DInf<V>::value;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hu = p.hu, hl = p.hl, wout = hu + hl;
    const int ns = wout / kDmStride + 1 + ((wout % kDmStride) ? 1 : 0);
    int32_t *kmin = kmin_all + warp * ns;
    const V *DU = reinterpret_cast<const V *>(p.du);
    const V *DL = reinterpret_cast<const V *>(p.dl);
    V *out = reinterpret_cast<V *>(p.out);
    const int64_t nw = (int64_t)gridDim.x * kDmWarps;
    for (int64_t i = (int64_t)blockIdx.x * kDmWarps + warp; i <= p.n; i += nw) {
        const V *du = DU + i * p.ldu;
        V *o = out + i * p.ldo;
        // term (k, w): D_L(D_U(i, k), w - k), infinite when D_U(i, k) is or
        // w - k lies outside [0, hl].  An entry of D_U that is no vertex
        // (outside [0, n]; not a breakout matrix) counts as unreachable, so
        // every read stays inside D_L.
        auto term = [&](int k, int w) -> int {
            const int x = (int)du[k];
            if (x == INF || x < 0 || x > p.n || w - k < 0 || w - k > hl) return INF;
            return (int)DL[(int64_t)x * p.ldl + (w - k)];
        };
        // 1. exact leftmost minimum of the sampled columns.
        for (int s = 0; s < ns; ++s) {
            const int w = min(s * kDmStride, wout);
            const int lo = max(0, w - hl), hi = min(w, hu);
            int best = INF, bk = INT32_MAX;
            for (int k = lo + lane; k <= hi; k += 32) {
                const int v = term(k, w);
                if (v < best) { best = v; bk = k; }        // k ascending per lane: first minimum
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const int ov = __shfl_xor_sync(0xFFFFFFFFu, best, off);
                const int ok = __shfl_xor_sync(0xFFFFFFFFu, bk, off);
                if (ov < best || (ov == best && ok < bk)) { best = ov; bk = ok; }
            }
            if (lane == 0) {
                kmin[s] = best == INF ? -1 : bk;
                o[w] = (V)best;
            }
        }
        __syncwarp();
        // 2. the columns between two sampled ones: a lane each, rows from the
        // left column's minimiser to the right one's (or to the last row when
        // the right column is infinite; a left column that is infinite makes
        // every later column infinite).
        for (int s = 0; s + 1 < ns; ++s) {
            const int wl = s * kDmStride, wr = min((s + 1) * kDmStride, wout);
            const int w = wl + 1 + lane;
            const bool mine = w < wr;
            const int kl = kmin[s], kr = kmin[s + 1];
            int best = INF;
            if (kl >= 0) {
                const int khi = kr >= 0 ? kr : min(hu, wr);
#pragma unroll 4
                for (int k = kl; k <= khi; ++k) {
                    const int v = mine ? term(k, w) : INF;
                    best = v < best ? v : best;
                }
            }
            if (mine) o[w] = (V)best;
        }
        __syncwarp();
    }
}

template <typename V>
static cudaError_t launch_dfm(const DformMergeParams &p, cudaStream_t st) {
    const int wout = p.hu + p.hl;
    const int ns = wout / kDmStride + 2;
    const size_t smem = (size_t)kDmWarps * ns * 4;
    auto kern = dform_merge_kernel<V>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>(ceil_div(p.n + 1, kDmWarps), (int64_t)sms * 16);
    return launch_pdl(kern, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(kDmWarps * 32), smem, st, p);
}

cudaError_t launch_dform_merge(const DformMergeParams &p, int dtype, cudaStream_t st) {
    if (dtype == DT_I32) return launch_dfm<int32_t>(p, st);
    if (dtype == DT_I16) return launch_dfm<int16_t>(p, st);
    return cudaErrorInvalidValue;
}

}  // namespace lcsg
