// batch.cu -- many independent pairs in one submission (lcs_batch_submit).
//
// A pair whose string a has at most 16384 letters is one strip: its rows all
// fit one bit vector of W = ceil(m / 32) words, so the merge tree has no
// level, the length is the strip's DIST(0, n) (Sec. I) and one LCS is the
// strip's leftmost heaviest path from top vertex 0 to bottom vertex n
// (Sec. II-C..II-E).  Only source 0 is needed, so a warp carries that one
// source through the column sweep of the strip builder
//     u = V & M[b_j];  V' = (V + u) | (V & ~M[b_j]),
// lane l holding the WPL consecutive words l*WPL .. l*WPL + WPL - 1.  The add
// runs through a lane's words serially; its carries cross the lanes by carry
// look-ahead: with G the ballot of lanes whose words overflowed and P the
// ballot of lanes whose words summed to all ones (a carry in passes through
// them), the carries into the lanes are the carries of the 32-bit addition
// (G | P) + G.
// Each column vector, with the count of ones below each of its words, is
// stored when the pair wants its string; a backward walk from (m, n) then
// keeps every row's segment as far left as it can go (left while F keeps its
// value, else the match diagonal if it is tight, else up), which is the
// leftmost heaviest path; a diagonal step into row r marks a_r.  F(r, c) = r
// minus the ones among the first r bits of V_c is one stored count plus one
// masked popcount, read from a small shared-memory window of the columns and
// words the walk is at.
#include <algorithm>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

constexpr int kBatchLetters = 32;        // distinct letters of a with a shared mask table
constexpr int kWalkCols = 32;            // columns staged per walk window (a lane each)

// Per-warp shared memory of the words-per-lane class WPL.
template <int WPL>
struct BatchCfg {
    static constexpr int W = 32 * WPL;                                  // words of the tallest a
    static constexpr int kWarps = WPL <= 2 ? 4 : (WPL == 4 ? 2 : 1);    // warps (pairs in flight) per CTA
    static constexpr size_t o_msk = 0;                                  // [kBatchLetters][W] row masks
    static constexpr size_t o_win = o_msk + (size_t)kBatchLetters * W * 4;   // walk window: [kWalkCols][2]
                                                                        // words, then [kWalkCols][2] counts
    static constexpr size_t o_a = o_win + (size_t)kWalkCols * 2 * 4 + (size_t)kWalkCols * 2 * 4;
    static constexpr size_t o_lmap = o_a + (size_t)W * 32;              // letter -> mask row (255: absent)
    static constexpr size_t o_present = o_lmap + 256;                   // letters of a, a bit each
    static constexpr size_t warp_bytes = (o_present + 32 + 15) / 16 * 16;
};

// Carries into the 32 lanes' word blocks (bit l: into lane l), given each
// lane's generate g and propagate p.
__device__ __forceinline__ uint32_t lane_carries(bool g, bool p) {
    const uint32_t G = __ballot_sync(0xFFFFFFFFu, g), P = __ballot_sync(0xFFFFFFFFu, p);
    const uint32_t A = G | P;
    return (A + G) ^ A ^ G;
}

template <int WPL>
__global__ void __launch_bounds__(BatchCfg<WPL>::kWarps * 32) batch_strip_kernel(BatchParams bp) {
    using C = BatchCfg<WPL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ws = smem_raw + warp * C::warp_bytes;
    uint32_t(*msk)[C::W] = reinterpret_cast<uint32_t(*)[C::W]>(ws + C::o_msk);
    uint32_t(*wword)[2] = reinterpret_cast<uint32_t(*)[2]>(ws + C::o_win);
    uint32_t(*wcnt)[2] = reinterpret_cast<uint32_t(*)[2]>(ws + C::o_win + kWalkCols * 2 * 4);
    uint8_t *sa = ws + C::o_a;
    uint8_t *lmap = ws + C::o_lmap;
    uint32_t *present = reinterpret_cast<uint32_t *>(ws + C::o_present);
    // Pairs come from the batch's device work queue: each warp takes the next
    // pair of the processing order (largest first) from an atomic counter as
    // soon as it is free, so that pairs of very different costs spread over
    // the warps as they finish.
    for (;;) {
        unsigned q32 = 0;
        if (lane == 0) q32 = atomicAdd(bp.queue, 1u);
        const int64_t q = (int64_t)__shfl_sync(0xFFFFFFFFu, q32, 0);
        if (q >= bp.count) break;
        const BatchPair pr = bp.pairs[bp.order ? bp.order[q] : q];
        const int m = (int)pr.m;
        const int64_t n = pr.n;
        if (m <= 0 || n <= 0 || m > 32 * C::W) {
            if (lane == 0) {
                pr.len_out[0] = 0;
                if (m > 32 * C::W) set_error(bp.err, ERR_BOUNDS);
            }
            continue;
        }
        const int Wu = (m + 31) >> 5;          // words in use; rows >= m are padding
        // Stage a, rank its letters, build the row masks.
        if (lane < 8) present[lane] = 0u;
        __syncwarp();
        for (int r = lane; r < m; r += 32) {
            const uint8_t ch = pr.a[r];
            sa[r] = ch;
            atomicOr(&present[ch >> 5], 1u << (ch & 31));
        }
        __syncwarp();
        int nlet = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) nlet += __popc(present[t]);
        const bool table = nlet <= kBatchLetters;
        if (table) {
            for (int c = lane; c < 256; c += 32) {
                const uint32_t word = present[c >> 5], bit = 1u << (c & 31);
                int rank = 0;
                for (int t = 0; t < (c >> 5); ++t) rank += __popc(present[t]);
                rank += __popc(word & (bit - 1u));
                lmap[c] = (word & bit) ? (uint8_t)rank : (uint8_t)255;
            }
            for (int t = lane; t < nlet * C::W; t += 32) (&msk[0][0])[t] = 0u;
            __syncwarp();
            for (int r = lane; r < m; r += 32) atomicOr(&msk[lmap[sa[r]]][r >> 5], 1u << (r & 31));
        }
        __syncwarp();
        const int w0 = lane * WPL;                // this lane's first word
        auto masks = [&](uint8_t ch, uint32_t (&M)[WPL]) {
            if (table) {
                const uint8_t k = lmap[ch];
#pragma unroll
                for (int t = 0; t < WPL; ++t) M[t] = (k == 255 || w0 + t >= Wu) ? 0u : msk[k][w0 + t];
            } else {
                // More than kBatchLetters letters in a: compare the rows.
#pragma unroll
                for (int t = 0; t < WPL; ++t) {
                    uint32_t mk = 0u;
                    const int r0 = (w0 + t) * 32;
                    for (int b = 0; b < 32 && r0 + b < m; ++b) mk |= (uint32_t)(sa[r0 + b] == ch) << b;
                    M[t] = mk;
                }
            }
        };
        uint32_t V[WPL];
#pragma unroll
        for (int t = 0; t < WPL; ++t) V[t] = 0xFFFFFFFFu;
        // Scratch of a pair that wants its string: (n+1) x Wu column words,
        // then (n+1) x (Wu+1) 16-bit counts of the ones below each word
        // (entry Wu: all of them).
        uint32_t *col = bp.scratch ? bp.scratch + pr.scratch_off : nullptr;
        uint16_t *cnt = col ? reinterpret_cast<uint16_t *>(col + (n + 1) * Wu) : nullptr;
        const bool want = pr.want && col != nullptr;
        auto store_col = [&](int64_t c) {
            uint32_t *cv = col + c * Wu;
            uint16_t *pv = cnt + c * (Wu + 1);
            int ones[WPL], tot = 0;
#pragma unroll
            for (int t = 0; t < WPL; ++t) {
                ones[t] = w0 + t < Wu ? __popc(V[t]) : 0;
                tot += ones[t];
            }
            int below = tot;                      // inclusive scan of the lanes' totals
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, below, off);
                if (lane >= off) below += y;
            }
            below -= tot;
#pragma unroll
            for (int t = 0; t < WPL; ++t) {
                if (w0 + t <= Wu) pv[w0 + t] = (uint16_t)below;
                if (w0 + t < Wu) cv[w0 + t] = V[t];
                below += ones[t];
            }
            if (lane == 31 && Wu == C::W) pv[Wu] = (uint16_t)below;   // no lane holds index Wu
        };
        if (want) store_col(0);
        uint32_t bnext = (lane < n) ? pr.b[lane] : 0u;      // b[blk + lane], one block ahead
        for (int64_t blk = 0; blk < n; blk += 32) {
            const uint32_t bcur = bnext;
            bnext = (blk + 32 + lane < n) ? pr.b[blk + 32 + lane] : 0u;
            const int cnt = (int)min((int64_t)32, n - blk);
#pragma unroll 2
            for (int t = 0; t < cnt; ++t) {
                const uint8_t ch = (uint8_t)__shfl_sync(0xFFFFFFFFu, bcur, t);
                uint32_t M[WPL], s[WPL];
                masks(ch, M);
                // This lane's words of V + (V & M) with no carry in: generate
                // and propagate of the lane.
                // This lane's words of V + (V & M) with no carry in (one
                // add-with-carry chain): generate and propagate of the lane.
                uint32_t u[WPL];
#pragma unroll
                for (int k = 0; k < WPL; ++k) u[k] = V[k] & M[k];
                const uint32_t carry = addn_cin<WPL>(s, V, u, 0u);
                // below[k]: every word under k is all ones, so a carry into
                // the lane reaches word k (computed while the ballots run).
                uint32_t below[WPL];
                below[0] = 1u;
#pragma unroll
                for (int k = 1; k < WPL; ++k) below[k] = below[k - 1] & (s[k - 1] == 0xFFFFFFFFu ? 1u : 0u);
                const bool ones = (below[WPL - 1] & (s[WPL - 1] == 0xFFFFFFFFu ? 1u : 0u)) != 0u;
                const uint32_t cin = (lane_carries(carry != 0u, ones) >> lane) & 1u;
#pragma unroll
                for (int k = 0; k < WPL; ++k) V[k] = (s[k] + (cin & below[k])) | (V[k] & ~M[k]);
                if (want) store_col(blk + t + 1);
            }
        }
        // Length = F(m, n) = zeros among the first m bits.
        auto ones_below = [&](const uint32_t (&v)[WPL], int r) -> int {
            int ones = 0;
#pragma unroll
            for (int k = 0; k < WPL; ++k) {
                const int bits = min(max(r - 32 * (w0 + k), 0), 32);
                ones += __popc(v[k] & (bits == 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u)));
            }
            return __reduce_add_sync(0xFFFFFFFFu, ones);
        };
        const int L = m - ones_below(V, m);
        if (lane == 0) pr.len_out[0] = L;
        if (!want) continue;
        __syncwarp();
        // Backward walk.  F(r, c) needs word w = r / 32 of V_c and the count
        // of ones below it; the window holds words w-1 and w (and their
        // counts) of kWalkCols columns, a lane loading one column.  The walk
        // asks for its current column c or c - 1 with c never growing, and
        // for rows that never grow: a window that misses is reloaded to end
        // one column past the asked one and to hold the asked word on top.
        int64_t wlo = 0, whi = -1;
        int wbase = -2;                          // words wbase, wbase + 1 are staged
        auto F = [&](int64_t c, int r) -> int {
            const int w = r >> 5, bits = r & 31;
            if (c < wlo || c > whi || w < wbase || w > wbase + 1) {
                __syncwarp();
                whi = min(n, c + 1);
                wlo = max((int64_t)0, whi - kWalkCols + 1);
                wbase = max(0, w - 1);
                const int64_t cc = wlo + lane;
                if (cc <= whi) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int wk = wbase + k;
                        wword[lane][k] = wk < Wu ? col[cc * Wu + wk] : 0u;
                        wcnt[lane][k] = wk <= Wu ? cnt[cc * (Wu + 1) + wk] : 0u;
                    }
                }
                __syncwarp();
            }
            const int slot = (int)(c - wlo), k = w - wbase;
            int ones = (int)wcnt[slot][k];
            if (bits) ones += __popc(wword[slot][k] & ((1u << bits) - 1u));
            return r - ones;
        };
        uint8_t *str = bp.strings + pr.str_off;
        int r = m;
        int64_t c = n;
        int pos = L;
        int fc = F(c, r);
        int64_t bbase = -64;                     // b[bbase + lane] in breg
        uint32_t breg = 0u;
        auto bchar = [&](int64_t j) -> uint8_t {   // b[j], warp-uniform j
            if (j < bbase || j >= bbase + 32) {
                bbase = max((int64_t)0, j - 31);
                breg = (bbase + lane < n) ? pr.b[bbase + lane] : 0u;
            }
            return (uint8_t)__shfl_sync(0xFFFFFFFFu, breg, (int)(j - bbase));
        };
        while (r > 0) {
            if (c > 0) {
                if (F(c - 1, r) == fc) {         // left along row r
                    --c;
                    continue;
                }
                if (sa[r - 1] == bchar(c - 1) && F(c - 1, r - 1) == fc - 1) {   // diagonal into row r
                    --pos;
                    if (lane == 0 && pos >= 0) str[pos] = sa[r - 1];
                    --r;
                    --c;
                    --fc;
                    continue;
                }
            }
            --r;                                 // up
            fc = F(c, r);
        }
        if (pos != 0 && lane == 0) set_error(bp.err, ERR_BOUNDS);
    }
}

int batch_max_rows() { return 32 * BatchCfg<16>::W; }

int batch_words_per_lane(int64_t m) {
    const int64_t w = (m + 31) / 32;
    return w <= 64 ? 2 : (w <= 128 ? 4 : (w <= 256 ? 8 : 16));
}

template <int WPL>
static cudaError_t launch_wpl(const BatchParams &bp, cudaStream_t st) {
    using C = BatchCfg<WPL>;
    const size_t smem = (size_t)C::kWarps * C::warp_bytes;
    auto kern = batch_strip_kernel<WPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::kWarps * 32, smem)) != cudaSuccess)
        return e;
    const int64_t need = ceil_div(bp.count, C::kWarps);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * std::max(per_sm, 1)));
    kern<<<(unsigned)grid, C::kWarps * 32, smem, st>>>(bp);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pairs split in two
// A CTA per split pair: the halves' columns from the split column c.
__global__ void split_fix_kernel(const SplitPair *sp, int64_t count) {
    const SplitPair s = sp[blockIdx.x];
    if (threadIdx.x == 0) {
        int64_t c = s.pathI[s.lower];
        if (c < 0 || c > s.n) {
            set_error(s.err, ERR_BOUNDS);
            c = 0;
        }
        s.sub0->b = s.b;
        s.sub0->n = c;
        s.sub1->b = s.b + c;
        s.sub1->n = s.n - c;
    }
    __syncthreads();
    // A half on the tall kernels with its string keeps its cross vertices
    // after its column vectors: m + 1 words set above any column.
    for (int h = 0; h < 2; ++h) {
        const BatchPair bp = h ? *s.sub1 : *s.sub0;
        if (!(h ? s.big1 : s.big0) || !bp.want || bp.m <= 0 || bp.n <= 0) continue;
        const int64_t wu = (bp.m + 31) / 32;
        int32_t *v = reinterpret_cast<int32_t *>(s.scratch + bp.scratch_off + 2 * wu * (bp.n + 1));
        for (int64_t r = threadIdx.x; r <= bp.m; r += blockDim.x) v[r] = 0x7F7F7F7F;
    }
}

// A CTA per split pair: length = len0 + len1, the lower half's string after
// the upper half's.
__global__ void split_join_kernel(const SplitPair *sp, int64_t count) {
    const SplitPair s = sp[blockIdx.x];
    const int64_t l0 = *s.sub0->len_out, l1 = *s.sub1->len_out;
    if (threadIdx.x == 0) *s.len_out = l0 + l1;
    if (s.str && s.str1)
        for (int64_t k = threadIdx.x; k < l1; k += blockDim.x) s.str[l0 + k] = s.str1[k];
}

cudaError_t launch_split_fix(const SplitPair *sp, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    split_fix_kernel<<<(unsigned)count, 256, 0, st>>>(sp, count);
    return cudaGetLastError();
}

cudaError_t launch_split_join(const SplitPair *sp, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    split_join_kernel<<<(unsigned)count, 256, 0, st>>>(sp, count);
    return cudaGetLastError();
}

cudaError_t launch_batch_strip(const BatchParams &bp, int wpl, cudaStream_t st) {
    if (bp.count <= 0) return cudaSuccess;
    if (!bp.queue) return cudaErrorInvalidValue;
    switch (wpl) {
        case 2: return launch_wpl<2>(bp, st);
        case 4: return launch_wpl<4>(bp, st);
        case 8: return launch_wpl<8>(bp, st);
        case 16: return launch_wpl<16>(bp, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lcsg
