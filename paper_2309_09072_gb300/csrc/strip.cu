// strip.cu -- DIST of a strip of h consecutive rows of a, for every source.
//
// For one source (top vertex) i the strip's column state after bottom vertex
// j is F_j(r) = LCS(a_strip[0:r], b[i:j]), r = 0..h.  F_j is nondecreasing in
// r with steps of 0 or 1, so it is held as an h-bit vector V whose zero bits
// mark the rows where F steps up.  One column step of the prefix-max
//     F_j(r) = max(F_j(r-1), F_{j-1}(r), F_{j-1}(r-1) + [a_r = b_j])
// over all h rows is then (Allison-Dix / Hyyro bit-vector LCS, restated)
//     u = V & M[b_j];   V' = (V + u) | (V & ~M[b_j]),
// where M[c] has bit r set iff a_r = c: the carry chain of the integer add
// carries the running maximum down the rows, and the carry out of the top
// row is exactly DIST(i, j) - DIST(i, j-1).  The add runs as one
// add.cc/addc chain over 32-bit words, so 32..256 rows cost a handful of
// INT32 instructions per (i, j).
//
// Work mapping: a pair of warps owns one band of T = 64 sources (one per
// lane) and sweeps j across the band's tiles J >= I in lock step, so the
// match mask of column j is warp-uniform (one broadcast shared-memory load
// per step); a named barrier per pair orders the shared column masks and
// staging tile.  Each finished T x T tile is staged in shared memory (padded
// pitch, conflict-free) and written out with coalesced stores in the layout
// its consumer wants (row or column tile-packed, or dense).
// Once every source of a band has matched all rows of the strip, DIST stays
// at h for the rest of the band's row, so the band's remaining tiles are
// written as constants without further column steps.
#include <type_traits>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

template <typename OutT>
struct StagePitch {
    // Row-layout staging writes 32 lanes x 1 element at rows lane, lane+32 of
    // one column; the padded pitch of a stored tile (T + 4 or T + 1
    // elements) spreads them over the banks, and a staged tile is then
    // written out as one contiguous image.
    static constexpr int value = Fmt<OutT>::P;
};

constexpr int kStripWarps = 4;
constexpr int kStripBands = kStripWarps / 2;   // a pair of warps per band

// Write words [w0, w1) of one staged T x T tile: a contiguous image for the
// tile-packed layouts, rows [w0, w1) for a dense matrix.
template <typename OutT>
__device__ __forceinline__ void write_tile_part(const StripParams &p, OutT *out, const OutT *stage, int layout,
                                                int64_t I, int64_t J, int64_t i0, int64_t jb, int cmax, int lane,
                                                int half) {
    constexpr int P = Fmt<OutT>::P;
    if (layout == LAYOUT_DENSE) {
        const int64_t rows = min((int64_t)T, p.n + 1 - i0);
        for (int r = half * (T / 2); r < min(rows, (int64_t)(half + 1) * (T / 2)); ++r) {
            OutT *dst = out + (i0 + r) * p.ld + jb;
            for (int c = lane; c < cmax; c += 32) dst[c] = stage[r * P + c];
        }
    } else {
        const int64_t tile = (layout == LAYOUT_COL) ? col_tile(I, J) : row_tile(I, J, p.NT);
        uint32_t *dst = reinterpret_cast<uint32_t *>(out + tile * Fmt<OutT>::ELEMS);
        constexpr int WT = Fmt<OutT>::ELEMS * (int)sizeof(OutT) / 4;   // 32-bit words per tile
        const uint32_t *src = reinterpret_cast<const uint32_t *>(stage);
        for (int w = half * (WT / 2) + lane; w < (half ? WT : WT / 2); w += 32) dst[w] = src[w];
    }
}

template <typename OutT, int W>
__global__ void __launch_bounds__(kStripWarps * 32) strip_kernel(StripParams p) {
    pdl_wait_and_release();
    constexpr int P = StagePitch<OutT>::value;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *masks = reinterpret_cast<uint32_t *>(smem);             // [256][W]
    uint32_t *colm_all = masks + 256 * W;                             // [bands][T][W]
    OutT *stage_all = reinterpret_cast<OutT *>(colm_all + kStripBands * T * W);  // [bands][T][P]
    __shared__ int s_sat[kStripBands][2];

    const int s = blockIdx.y;
    const int64_t r0 = (int64_t)s * p.h;
    const int hs = (int)min((int64_t)p.h, p.m - r0);

    for (int t = threadIdx.x; t < 256 * W; t += blockDim.x) masks[t] = 0u;
    __syncthreads();
    for (int r = threadIdx.x; r < hs; r += blockDim.x) {
        const uint8_t ch = p.a[r0 + r];
        atomicOr(&masks[ch * W + (r >> 5)], 1u << (r & 31));
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int band = warp >> 1, half = warp & 1;
    const int64_t I = (int64_t)p.band_first + (int64_t)blockIdx.x * kStripBands + band;
    if (I >= p.NT) return;     // both warps of the pair; no block-wide barrier below this point
    // The pair's named barrier (a constant id per branch keeps the CTA's
    // hardware barrier count small).
    auto pair_sync = [&]() {
        if (band == 0) named_bar_sync(1, 64);
        else named_bar_sync(2, 64);
    };

    uint32_t *colm = colm_all + band * T * W;
    OutT *stage = stage_all + band * T * P;
    const int64_t n = p.n;
    const int64_t i0 = I * T;
    const int layout = p.dense ? (int)LAYOUT_DENSE : p.outs[s].layout;
    OutT *out = p.dense ? reinterpret_cast<OutT *>(p.dense) : reinterpret_cast<OutT *>(p.outs[s].base);

    uint32_t V[W];
#pragma unroll
    for (int w = 0; w < W; ++w) V[w] = 0xFFFFFFFFu;
    int d = 0;
    const int r = half * 32 + lane;            // this lane's source is i0 + r, row r of the staged tile

    // Column c of tile J consumes letter b[J T + c - 1]; each lane of the
    // pair reads one column's letter, one tile ahead, so that the global
    // load's latency passes behind a tile of column steps.
    auto letter = [&](int64_t Jt) -> int {
        const int64_t j = Jt * T + half * 32 + lane;
        return (Jt < p.NT && j >= 1 && j <= n) ? (int)p.b[j - 1] : -1;
    };
    int ch_next = letter(I);
    // Rows are matched from the top of the strip down: once the first 32 w
    // rows of a source have all stepped (its low words are zero), they stay
    // so, and the column step runs from word w on (column_step_tail).  w0 is
    // the warp's smallest such w, refreshed after every tile.
    int w0 = 0;
    for (int64_t J = I; J < p.NT; ++J) {
        const int64_t jb = J * T;
        // Column masks of this tile (each warp of the pair builds half).
        {
            const int c = half * 32 + lane;
            const int ch = ch_next;
            ch_next = letter(J + 1);
#pragma unroll
            for (int w = 0; w < W; ++w) colm[c * W + w] = ch >= 0 ? masks[ch * W + w] : 0u;
        }
        // The masks are complete, and the previous tile has left the stage.
        pair_sync();
        const int cmax = (int)min((int64_t)T, n + 1 - jb);
        if (J == I) {
            // Diagonal tile: source i0+r starts at column r (DIST(i,i) = 0).
            for (int c = 0; c < cmax; ++c) {
                uint32_t M[W];
#pragma unroll
                for (int w = 0; w < W; ++w) M[w] = (c > r) ? colm[c * W + w] : 0u;
                d += (int)column_step<W>(V, M);
                const OutT v = (c < r) ? Sentinel<OutT>::value : (OutT)d;
                if (layout == LAYOUT_COL) stage[c * P + r] = v;
                else stage[r * P + c] = v;
            }
        } else {
            // Column c + 1's masks load while column c's carry chain runs;
            // the staging stride is a constant of each layout's loop, and
            // the first live word S of the warp's vectors is a constant of
            // each instantiation.
            auto sweep = [&](auto col_layout, auto start) {
                constexpr int SC = decltype(col_layout)::value ? P : 1, SR = decltype(col_layout)::value ? 1 : P;
                constexpr int S = decltype(start)::value;
                uint32_t Mn[W] = {};
#pragma unroll
                for (int w = S; w < W; ++w) Mn[w] = colm[w];
#pragma unroll 4
                for (int c = 0; c < cmax; ++c) {
                    uint32_t M[W] = {};
#pragma unroll
                    for (int w = S; w < W; ++w) M[w] = Mn[w];
                    const int cn = c + 1 < cmax ? c + 1 : c;
#pragma unroll
                    for (int w = S; w < W; ++w) Mn[w] = colm[cn * W + w];
                    d += (int)column_step_tail<W, S>(V, M);
                    stage[c * SC + r * SR] = (OutT)d;
                }
            };
            dispatch_start<W>(w0, [&](auto start) {
                if (layout == LAYOUT_COL) sweep(std::true_type{}, start);
                else sweep(std::false_type{}, start);
            });
        }
        {
            int z = W;
#pragma unroll
            for (int w = W - 1; w >= 0; --w)
                if (V[w] != 0u) z = w;
            if (i0 + r > n) z = W;             // no source in this lane
            w0 = __reduce_min_sync(0xFFFFFFFFu, z);
        }
        // Once every source of the band has matched all hs rows, DIST stays
        // hs for the rest of the row: the remaining tiles are constant.
        const bool sat_w = __all_sync(0xFFFFFFFFu, d >= hs || i0 + r > n);
        if (lane == 0) s_sat[band][half] = sat_w ? 1 : 0;
        pair_sync();         // the tile and both saturation flags are in
        write_tile_part<OutT>(p, out, stage, layout, I, J, i0, jb, cmax, lane, half);
        const bool saturated = s_sat[band][0] && s_sat[band][1];
        if (saturated && J + 1 < p.NT) {
            pair_sync();     // both halves written before the stage is refilled
            for (int e = half * 32 + lane; e < T * P; e += 64) stage[e] = (OutT)hs;
            pair_sync();
            for (int64_t J2 = J + 1; J2 < p.NT; ++J2) {
                const int64_t jb2 = J2 * T;
                write_tile_part<OutT>(p, out, stage, layout, I, J2, i0, jb2, (int)min((int64_t)T, n + 1 - jb2), lane,
                                      half);
            }
            break;
        }
    }
}

template <typename OutT, int W>
static cudaError_t launch_t(const StripParams &p, cudaStream_t st) {
    constexpr int P = StagePitch<OutT>::value;
    const size_t smem = (size_t)256 * W * 4 + (size_t)kStripBands * T * W * 4 +
                        (size_t)kStripBands * T * P * sizeof(OutT);
    auto kern = strip_kernel<OutT, W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t bands = p.NT - p.band_first;
    dim3 grid((unsigned)ceil_div(bands, kStripBands), (unsigned)p.S);
    return launch_pdl(kern, grid, dim3(kStripWarps * 32), smem, st, p);
}

template <typename OutT>
static cudaError_t launch_w(const StripParams &p, int words, cudaStream_t st) {
    switch (words) {
        case 1: return launch_t<OutT, 1>(p, st);
        case 2: return launch_t<OutT, 2>(p, st);
        case 4: return launch_t<OutT, 4>(p, st);
        case 8: return launch_t<OutT, 8>(p, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_strip(const StripParams &p, int out_dtype, int words, cudaStream_t st) {
    if (p.NT <= p.band_first || p.S <= 0) return cudaSuccess;
    switch (out_dtype) {
        case DT_U8: return launch_w<uint8_t>(p, words, st);
        case DT_I16: return launch_w<int16_t>(p, words, st);
        case DT_I32: return launch_w<int32_t>(p, words, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lcsg
