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
//      known neighbours -- and finally writes D (and K) out in the layout the
//      consumer wants.  Tiles whose k-window exceeds the shared-memory band
//      fall back to the same refinement reading global memory.
#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int64_t grid_vertex(int64_t p, int64_t n) { return min(p * T, n); }

// Warp-wide (value, k) reduction: largest value, smallest k among equals.
__device__ __forceinline__ void warp_argmax(int &v, int64_t &k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const int ov = __shfl_xor_sync(0xFFFFFFFFu, v, off);
        const int64_t ok = __shfl_xor_sync(0xFFFFFFFFu, k, off);
        if (ov > v || (ov == v && ok < k)) { v = ov; k = ok; }
    }
}

// ------------------------------------------------------------------ coarse
int64_t coarse_sigma0(int64_t P) {
    // Full scans on a sub-grid of about 17 x 17 points; each later level
    // halves the stride down to 1.
    int64_t s = 1;
    while (s * 16 < P) s <<= 1;
    return s;
}

template <typename TIn>
__global__ void __launch_bounds__(256) coarse_kernel(MergeParams p) {
    const int64_t P = p.P, n = p.n, sigma = p.sigma;
    const int64_t cnt = P / sigma + 1 + ((P % sigma) ? 1 : 0);   // points 0, s, 2s, .., P
    const int64_t per_job = cnt * cnt;
    const int64_t total = per_job * p.njobs;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp0; w < total; w += nwarps) {
        const int job = (int)(w / per_job);
        const int64_t rem = w - (int64_t)job * per_job;
        const int64_t t = rem / cnt, u = rem - t * cnt;
        const int64_t xp = min(t * sigma, P), xq = min(u * sigma, P);
        if (xp > xq) continue;
        const bool newp = (t & 1) && xp < P;
        const bool newq = (u & 1) && xq < P;
        if (!p.full && !newp && !newq) continue;
        const MergeJob jb = p.jobs[job];
        int32_t *kg = jb.kgrid;
        const int64_t gi = grid_vertex(xp, n), gj = grid_vertex(xq, n);
        int64_t lo = gi, hi = gj;
        if (!p.full) {
            const int64_t td = newp ? t - 1 : t, tu = newp ? t + 1 : t;
            const int64_t ud = newq ? u - 1 : u, uu = newq ? u + 1 : u;
            const int64_t pd = min(td * sigma, P), pu = min(tu * sigma, P);
            const int64_t qd = min(ud * sigma, P), qu = min(uu * sigma, P);
            lo = max(lo, (int64_t)kg[pd * (P + 1) + qd]);
            hi = min(hi, (int64_t)kg[pu * (P + 1) + qu]);
        }
        const TIn *U = reinterpret_cast<const TIn *>(jb.U);
        const TIn *L = reinterpret_cast<const TIn *>(jb.L);
        int best = INT32_MIN;
        int64_t bk = INT64_MAX;
        for (int64_t k = lo + lane; k <= hi; k += 32) {
            const int v = (int)U[row_elem(gi, k, p.NT)] + (int)L[col_elem(k, gj)];
            if (v > best) { best = v; bk = k; }     // k increases: first max per lane
        }
        warp_argmax(best, bk);
        if (lane == 0) {
            if (bk == INT64_MAX) { set_error(p.err, ERR_BOUNDS); bk = gi; }
            kg[xp * (P + 1) + xq] = (int32_t)bk;
        }
    }
}

cudaError_t launch_coarse(const MergeParams &p, int in_dtype, cudaStream_t st) {
    const int64_t cnt = p.P / p.sigma + 2;
    const int64_t warps = cnt * cnt * p.njobs;
    int64_t blocks = ceil_div(warps, 8);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    switch (in_dtype) {
        case DT_U8: coarse_kernel<uint8_t><<<(unsigned)blocks, 256, 0, st>>>(p); break;
        case DT_I16: coarse_kernel<int16_t><<<(unsigned)blocks, 256, 0, st>>>(p); break;
        case DT_I32: coarse_kernel<int32_t><<<(unsigned)blocks, 256, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ tile
constexpr int TP1 = T + 1;              // box points per side (with the far edge)
constexpr int kTileThreads = 256;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct TileSmem {
    size_t ks, ds, us, ls, total;
};
__host__ __device__ inline TileSmem tile_smem_layout(int in_sz, int out_sz, int cap) {
    TileSmem s;
    size_t off = 16;                                  // mbarrier
    s.ks = off; off = align16(off + (size_t)TP1 * TP1 * 4);
    s.ds = off; off = align16(off + (size_t)T2 * out_sz);
    s.us = off; off = align16(off + (size_t)cap * TP1 * T * in_sz);
    s.ls = off; off = align16(off + (size_t)cap * TP1 * T * in_sz);
    s.total = off;
    return s;
}

static int dt_size(int dt) { return dt == DT_U8 ? 1 : (dt == DT_I16 ? 2 : 4); }

size_t tile_smem_bytes(int in_dtype, int out_dtype, int cap) {
    return tile_smem_layout(dt_size(in_dtype), dt_size(out_dtype), cap).total;
}

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

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kTileThreads) tile_kernel(MergeParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const TileSmem L = tile_smem_layout((int)sizeof(TIn), (int)sizeof(TOut), p.cap);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int32_t *Ks = reinterpret_cast<int32_t *>(smem + L.ks);
    TOut *Ds = reinterpret_cast<TOut *>(smem + L.ds);
    TIn *Us = reinterpret_cast<TIn *>(smem + L.us);
    TIn *Ls = reinterpret_cast<TIn *>(smem + L.ls);

    const int64_t n = p.n, NT = p.NT, P = p.P;
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
    const int64_t ia = I * T, ja = J * T;
    const int Bi = (int)(min(ia + T, n) - ia), Bj = (int)(min(ja + T, n) - ja);
    const int64_t pa = I, pb = min(I + 1, P), qa = J, qb = min(J + 1, P);
    auto kcorner = [&](int64_t pp, int64_t qq) -> int32_t {
        const int64_t gi = grid_vertex(pp, n), gj = grid_vertex(qq, n);
        return gi > gj ? (int32_t)gj : jb.kgrid[pp * (P + 1) + qq];
    };
    int32_t klo = kcorner(pa, qa), khi = kcorner(pb, qb);
    // K(ia, ja) lies in [ia, ja] and K(ib, jb) in [ib, jb]; anything else
    // means the inputs are not DIST matrices: flag it and stage nothing.
    const bool corners_ok = klo >= ia && klo <= ja && khi >= ia + Bi && khi <= ja + Bj && klo <= khi;
    if (!corners_ok) {
        if (threadIdx.x == 0) set_error(p.err, ERR_BOUNDS);
        klo = (int32_t)ia;
        khi = (int32_t)(ja + Bj);
    }
    const int64_t kt0 = klo >> T_SHIFT, kt1 = khi >> T_SHIFT;
    const int nK = (int)(kt1 - kt0 + 1);
    const int64_t kbase = kt0 * T;
    const bool in_smem = corners_ok && nK <= p.cap;
    const TIn *Ug = reinterpret_cast<const TIn *>(jb.U);
    const TIn *Lg = reinterpret_cast<const TIn *>(jb.L);
    constexpr int TT = TP1 * T;         // elements per staged K-tile (T+1 rows)

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (in_smem && threadIdx.x == 0) {
        // Byte count first, then the copies.
        uint32_t bytes = 0;
        const uint32_t tileB = (uint32_t)(T2 * sizeof(TIn)), rowB = (uint32_t)(T * sizeof(TIn));
        const int64_t ltop = min(kt1, J);
        bytes += (uint32_t)nK * tileB;                              // U band
        const int64_t uextra = kt1 - max(kt0, I + 1) + 1;
        if (Bi == T && uextra > 0) bytes += (uint32_t)uextra * rowB;
        bytes += (uint32_t)(ltop - kt0 + 1) * tileB;                // L band
        if (Bj == T) bytes += (uint32_t)(min(kt1, J + 1) - kt0 + 1) * rowB;
        mbar_arrive_expect_tx(bar, bytes);
        for (int64_t kt = kt0; kt <= kt1; ++kt) {
            TIn *dst = Us + (kt - kt0) * TT;
            bulk_g2s(dst, Ug + row_tile(I, kt, NT) * T2, tileB, bar);
            if (Bi == T && kt >= I + 1) bulk_g2s(dst + T2, Ug + row_tile(I + 1, kt, NT) * T2, rowB, bar);
        }
        for (int64_t kt = kt0; kt <= ltop; ++kt)
            bulk_g2s(Ls + (kt - kt0) * TT, Lg + col_tile(kt, J) * T2, tileB, bar);
        if (Bj == T)
            for (int64_t kt = kt0; kt <= min(kt1, J + 1); ++kt)
                bulk_g2s(Ls + (kt - kt0) * TT + T2, Lg + col_tile(kt, J + 1) * T2, rowB, bar);
    }

    // Box initialisation: lower-triangle points hold j (k <= j bounds), the
    // four corners come from the coarse grid, everything else is unknown.
    for (int idx = threadIdx.x; idx < TP1 * TP1; idx += blockDim.x) {
        const int x = idx / TP1, y = idx - x * TP1;
        int32_t v = -1;
        if (x <= Bi && y <= Bj && ia + x > ja + y) v = (int32_t)(ja + y);
        Ks[idx] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Ks[0] = klo;
        Ks[Bj] = kcorner(pa, qb);
        Ks[Bi * TP1] = kcorner(pb, qa);
        Ks[Bi * TP1 + Bj] = khi;
    }
    bool ok = true;
    if (in_smem) ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (!ok) set_error(p.err, ERR_TIMEOUT);
    __syncthreads();
    // Every thread must agree on `ok`; a timed-out tile is skipped entirely.
    ok = __syncthreads_and(ok);
    if (!ok) return;

    const int layout = jb.d_layout;
    auto ds_index = [&](int x, int y) -> int { return layout == LAYOUT_COL ? y * T + x : x * T + y; };

    // Value of k for (x, y): SMEM band or global memory.
    auto eval = [&](int x, int y, int64_t lo, int64_t hi, int &best, int64_t &bk) {
        const int64_t i = ia + x, j = ja + y;
        best = INT32_MIN;
        if (in_smem) {
            // A no-op for Monge inputs (every window lies in [klo, khi]); it
            // keeps shared-memory reads inside the staged band for any input.
            lo = max(lo, (int64_t)klo);
            hi = min(hi, (int64_t)khi);
        }
        bk = lo;
        if (lo > hi) { set_error(p.err, ERR_BOUNDS); return; }
        if (in_smem) {
            const TIn *ur = Us + x * T;
            const TIn *lr = Ls + y * T;
            for (int64_t k = lo; k <= hi; ++k) {
                const int off = (int)(k - kbase);
                const int e = (off >> T_SHIFT) * TT + (off & (T - 1));
                const int v = (int)ur[e] + (int)lr[e];
                if (v > best) { best = v; bk = k; }
            }
        } else {
            for (int64_t k = lo; k <= hi; ++k) {
                const int v = (int)Ug[row_elem(i, k, NT)] + (int)Lg[col_elem(k, j)];
                if (v > best) { best = v; bk = k; }
            }
        }
    };
    auto finish = [&](int x, int y, int best, int64_t bk) {
        if (best > MaxVal<TOut>::value) set_error(p.err, ERR_OVERFLOW);
        Ks[x * TP1 + y] = (int32_t)bk;
        if (x < T && y < T) Ds[ds_index(x, y)] = (TOut)best;
    };

    // D at the corners that this tile owns (K known from the coarse grid).
    if (threadIdx.x < 4) {
        const int x = (threadIdx.x & 1) ? Bi : 0, y = (threadIdx.x & 2) ? Bj : 0;
        const bool dup = (threadIdx.x == 1 && Bi == 0) || (threadIdx.x == 2 && Bj == 0) ||
                         (threadIdx.x == 3 && (Bi == 0 || Bj == 0));
        if (!dup && x < T && y < T && ia + x <= ja + y) {
            const int64_t k = Ks[x * TP1 + y];
            int best;
            int64_t bk;
            eval(x, y, k, k, best, bk);
            finish(x, y, best, bk);
        }
    }
    __syncthreads();

    for (int s = T / 2; s >= 1; s >>= 1) {
        int nnx, nox, nex, nny, noy, ney;
        level_counts(Bi, s, nnx, nox, nex);
        level_counts(Bj, s, nny, noy, ney);
        // Points with exactly one new coordinate.
        const int cA = nnx * noy, cB = nox * nny;
        for (int idx = threadIdx.x; idx < cA + cB; idx += blockDim.x) {
            int x, y, xd, xu, yd, yu;
            if (idx < cA) {
                const int qx = idx / noy, qy = idx - qx * noy;
                x = (2 * qx + 1) * s; y = old_coord(qy, ney, s, Bj);
                xd = x - s; xu = min(x + s, Bi); yd = yu = y;
            } else {
                const int id2 = idx - cA;
                const int qx = id2 / nny, qy = id2 - qx * nny;
                x = old_coord(qx, nex, s, Bi); y = (2 * qy + 1) * s;
                xd = xu = x; yd = y - s; yu = min(y + s, Bj);
            }
            const int64_t i = ia + x, j = ja + y;
            if (i > j) continue;
            const int64_t lo = max(i, (int64_t)Ks[xd * TP1 + yd]);
            const int64_t hi = min(j, (int64_t)Ks[xu * TP1 + yu]);
            int best;
            int64_t bk;
            eval(x, y, lo, hi, best, bk);
            finish(x, y, best, bk);
        }
        __syncthreads();
        // Points with two new coordinates, bounded by the four just computed.
        const int cC = nnx * nny;
        for (int idx = threadIdx.x; idx < cC; idx += blockDim.x) {
            const int qx = idx / nny, qy = idx - qx * nny;
            const int x = (2 * qx + 1) * s, y = (2 * qy + 1) * s;
            const int64_t i = ia + x, j = ja + y;
            if (i > j) continue;
            const int xu = min(x + s, Bi), yu = min(y + s, Bj);
            int64_t lo = max((int64_t)Ks[x * TP1 + (y - s)], (int64_t)Ks[(x - s) * TP1 + y]);
            int64_t hi = min((int64_t)Ks[x * TP1 + yu], (int64_t)Ks[xu * TP1 + y]);
            lo = max(lo, i);
            hi = min(hi, j);
            int best;
            int64_t bk;
            eval(x, y, lo, hi, best, bk);
            finish(x, y, best, bk);
        }
        __syncthreads();
    }

    // Output.
    if (layout == LAYOUT_DENSE) {
        TOut *out = reinterpret_cast<TOut *>(p.dense_out);
        int32_t *Kout = p.dense_K;
        const int rows = (int)min((int64_t)T, n + 1 - ia), cols = (int)min((int64_t)T, n + 1 - ja);
        for (int idx = threadIdx.x; idx < rows * T; idx += blockDim.x) {
            const int x = idx >> T_SHIFT, y = idx & (T - 1);
            if (y >= cols) continue;
            const int64_t i = ia + x, j = ja + y;
            out[i * p.ld + j] = (i > j) ? Sentinel<TOut>::value : Ds[x * T + y];
            if (Kout) Kout[i * p.ld + j] = (i > j) ? -1 : Ks[x * TP1 + y];
        }
    } else {
        const int64_t tile = (layout == LAYOUT_COL) ? col_tile(I, J) : row_tile(I, J, NT);
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<TOut *>(jb.D) + tile * T2);
        const uint4 *src = reinterpret_cast<const uint4 *>(Ds);
        constexpr int chunks = T2 * (int)sizeof(TOut) / 16;
        for (int c = threadIdx.x; c < chunks; c += blockDim.x) dst[c] = src[c];
    }
}

template <typename TIn, typename TOut>
static cudaError_t launch_tile_t(const MergeParams &p, cudaStream_t st) {
    const size_t smem = tile_smem_layout((int)sizeof(TIn), (int)sizeof(TOut), p.cap).total;
    auto kern = tile_kernel<TIn, TOut>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)num_tiles_tri(p.NT), (unsigned)p.njobs);
    kern<<<grid, kTileThreads, smem, st>>>(p);
    return cudaGetLastError();
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

// ------------------------------------------------------------------ pack
// Dense (n+1) x ld -> tile-packed (one CTA per tile I <= J); the column
// layout transposes each tile through shared memory.
template <typename V>
__global__ void __launch_bounds__(256) pack_kernel(const V *src, int64_t ld, int64_t n, int64_t NT,
                                                   V *dst, int layout) {
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
    if (layout == LAYOUT_COL) {
        V *d = dst + col_tile(I, J) * T2;
        for (int idx = threadIdx.x; idx < T2; idx += blockDim.x) {
            const int y = idx >> T_SHIFT, x = idx & (T - 1);
            d[idx] = tile[x][y];
        }
    } else {
        V *d = dst + row_tile(I, J, NT) * T2;
        for (int idx = threadIdx.x; idx < T2; idx += blockDim.x) d[idx] = tile[idx >> T_SHIFT][idx & (T - 1)];
    }
}

cudaError_t launch_pack(const void *src, int dtype, int64_t n, int64_t ld, void *dst, int layout,
                        cudaStream_t st) {
    const int64_t NT = num_tiles_side(n);
    const unsigned blocks = (unsigned)num_tiles_tri(NT);
    if (dtype == DT_I32)
        pack_kernel<int32_t><<<blocks, 256, 0, st>>>((const int32_t *)src, ld, n, NT, (int32_t *)dst, layout);
    else if (dtype == DT_I16)
        pack_kernel<int16_t><<<blocks, 256, 0, st>>>((const int16_t *)src, ld, n, NT, (int16_t *)dst, layout);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dense fill
template <typename V>
__global__ void fill_dense_kernel(V *out, int64_t n, int64_t ld, V lower, V upper, int fill_upper,
                                  int32_t *K) {
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

cudaError_t launch_fill_dense(void *out, int dtype, int64_t n, int64_t ld, int lower, int upper,
                              int fill_upper, int32_t *K, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 1) < 8192 ? (n + 1) : 8192);
    if (dtype == DT_I32)
        fill_dense_kernel<int32_t><<<blocks, 256, 0, st>>>((int32_t *)out, n, ld, (int32_t)lower,
                                                           (int32_t)upper, fill_upper, K);
    else if (dtype == DT_I16)
        fill_dense_kernel<int16_t><<<blocks, 256, 0, st>>>((int16_t *)out, n, ld, (int16_t)lower,
                                                           (int16_t)upper, fill_upper, K);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lcsg
