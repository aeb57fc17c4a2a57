// batch.cu -- many independent pairs in one launch (lcs_batch_submit).
//
// A pair whose string a has at most 2048 letters is one strip: its rows all
// fit one bit vector of W = ceil(m / 32) <= 64 words, so the merge tree has
// no level, the length is the strip's DIST(0, n) (Sec. I) and one LCS is the
// strip's leftmost heaviest path from top vertex 0 to bottom vertex n
// (Sec. II-C..II-E).  Only source 0 is needed, so a warp carries that one
// source through the column sweep of the strip builder
//     u = V & M[b_j];  V' = (V + u) | (V & ~M[b_j])
// with the W words spread over the lanes (lane l holds words l and l + 32),
// and the add's carries crossing the lanes by carry look-ahead: with G the
// ballot of words whose sum overflowed and P the ballot of words that summed
// to all ones (a carry in passes through them), the carries into the words
// are the carries of the 32-bit addition (G | P) + G.
// Each column vector is stored when the pair wants its string; a backward
// walk from (m, n) then keeps every row's segment as far left as it can go
// (left while F keeps its value, else the match diagonal if it is tight,
// else up), which is the leftmost heaviest path; a diagonal step into row r
// marks a_r.  F(r, c) = r minus the ones among the first r bits of V_c is a
// masked popcount reduced over the warp.
#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

constexpr int kBatchWarps = 4;           // warps (pairs in flight) per CTA
constexpr int kBatchWords = 64;          // bit-vector words of the largest a (2048 rows)
constexpr int kBatchLetters = 32;        // distinct letters of a with a shared mask table
constexpr int kWalkCols = 16;            // column vectors staged per walk window

struct BatchWarpSmem {
    uint32_t msk[kBatchLetters][kBatchWords];   // row masks per letter of a
    uint32_t win[kWalkCols][kBatchWords];       // the walk's window of column vectors
    uint8_t a[kBatchWords * 32];                // the pair's a
    uint8_t lmap[256];                          // letter -> mask row (255: not in a)
    uint32_t present[8];                        // letters of a, one bit each
};

// Carries into the 32 words of one half (bit l: into lane l's word), given
// each lane's generate g and propagate p and the carry into the half; *cout
// receives the carry out of its top word.
__device__ __forceinline__ uint32_t carry_in(bool g, bool p, uint32_t cin, uint32_t *cout) {
    const uint32_t G = __ballot_sync(0xFFFFFFFFu, g), P = __ballot_sync(0xFFFFFFFFu, p);
    const uint64_t A = (uint64_t)(G | P), B = (uint64_t)G;
    const uint64_t sum = A + B + cin;
    *cout = (uint32_t)(sum >> 32);
    return (uint32_t)(sum ^ A ^ B);
}

__global__ void __launch_bounds__(kBatchWarps * 32) batch_small_kernel(BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BatchWarpSmem &S = reinterpret_cast<BatchWarpSmem *>(smem_raw)[warp];
    const int64_t warps = (int64_t)gridDim.x * kBatchWarps;
    for (int64_t q = (int64_t)blockIdx.x * kBatchWarps + warp; q < bp.count; q += warps) {
        const BatchPair pr = bp.pairs[bp.order ? bp.order[q] : q];
        const int m = (int)pr.m;
        const int64_t n = pr.n;
        if (m <= 0 || n <= 0) {
            if (lane == 0) pr.len_out[0] = 0;
            continue;
        }
        const int W = (m + 31) >> 5;
        // Stage a, rank its letters, build the row masks.
        for (int t = lane; t < 8; t += 32) S.present[t] = 0u;
        __syncwarp();
        for (int r = lane; r < m; r += 32) {
            const uint8_t ch = pr.a[r];
            S.a[r] = ch;
            atomicOr(&S.present[ch >> 5], 1u << (ch & 31));
        }
        __syncwarp();
        int nlet = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) nlet += __popc(S.present[t]);
        const bool table = nlet <= kBatchLetters;
        if (table) {
            for (int c = lane; c < 256; c += 32) {
                const uint32_t word = S.present[c >> 5], bit = 1u << (c & 31);
                int rank = 0;
                for (int t = 0; t < (c >> 5); ++t) rank += __popc(S.present[t]);
                rank += __popc(word & (bit - 1u));
                S.lmap[c] = (word & bit) ? (uint8_t)rank : (uint8_t)255;
            }
            for (int t = lane; t < nlet * kBatchWords; t += 32) (&S.msk[0][0])[t] = 0u;
            __syncwarp();
            for (int r = lane; r < m; r += 32) atomicOr(&S.msk[S.lmap[S.a[r]]][r >> 5], 1u << (r & 31));
        }
        __syncwarp();
        // Rows of lane l: word l (rows 32l..) and word l + 32; rows >= m are
        // padding, set in V and never in a mask.
        const bool hi_used = W > 32;
        auto mask_of = [&](uint8_t ch, int w) -> uint32_t {
            if (w >= W) return 0u;
            if (table) {
                const uint8_t k = S.lmap[ch];
                return k == 255 ? 0u : S.msk[k][w];
            }
            uint32_t mk = 0u;                    // more than kBatchLetters letters: compare
            const int r0 = w * 32;
            for (int t = 0; t < 32 && r0 + t < m; ++t) mk |= (uint32_t)(S.a[r0 + t] == ch) << t;
            return mk;
        };
        uint32_t V0 = 0xFFFFFFFFu, V1 = 0xFFFFFFFFu;
        uint32_t *col = bp.scratch ? bp.scratch + pr.scratch_off : nullptr;   // (n+1) x W words
        const bool want = pr.want && col != nullptr;
        if (want) {
            if (lane < W) col[lane] = V0;
            if (lane + 32 < W) col[lane + 32] = V1;
        }
        uint32_t bnext = (lane < n) ? pr.b[lane] : 0u;      // b[blk + lane], one block ahead
        for (int64_t blk = 0; blk < n; blk += 32) {
            const uint32_t bcur = bnext;
            bnext = (blk + 32 + lane < n) ? pr.b[blk + 32 + lane] : 0u;
            const int cnt = (int)min((int64_t)32, n - blk);
            for (int t = 0; t < cnt; ++t) {
                const uint8_t ch = (uint8_t)__shfl_sync(0xFFFFFFFFu, bcur, t);
                const uint32_t M0 = mask_of(ch, lane), M1 = hi_used ? mask_of(ch, lane + 32) : 0u;
                const uint32_t u0 = V0 & M0, u1 = V1 & M1;
                const uint32_t s0 = V0 + u0, s1 = V1 + u1;
                uint32_t c_lo, dummy;
                const uint32_t cin_lo = carry_in(s0 < V0, s0 == 0xFFFFFFFFu, 0u, &c_lo);
                const uint32_t cin_hi = hi_used ? carry_in(s1 < V1, s1 == 0xFFFFFFFFu, c_lo, &dummy) : 0u;
                const uint32_t f0 = s0 + ((cin_lo >> lane) & 1u), f1 = s1 + ((cin_hi >> lane) & 1u);
                V0 = f0 | (V0 & ~M0);
                V1 = f1 | (V1 & ~M1);
                if (want) {
                    uint32_t *cv = col + (blk + t + 1) * W;
                    if (lane < W) cv[lane] = V0;
                    if (lane + 32 < W) cv[lane + 32] = V1;
                }
            }
        }
        // Length = F(m, n) = zeros among the first m bits.
        auto ones_below = [&](uint32_t v0, uint32_t v1, int r) -> int {
            const int b0 = min(max(r - 32 * lane, 0), 32), b1 = min(max(r - 32 * (lane + 32), 0), 32);
            const uint32_t m0 = b0 == 32 ? 0xFFFFFFFFu : ((1u << b0) - 1u);
            const uint32_t m1 = b1 == 32 ? 0xFFFFFFFFu : ((1u << b1) - 1u);
            return __reduce_add_sync(0xFFFFFFFFu, __popc(v0 & m0) + __popc(v1 & m1));
        };
        const int L = m - ones_below(V0, V1, m);
        if (lane == 0) pr.len_out[0] = L;
        if (!want) continue;
        __syncwarp();
        // Backward walk over the stored columns, a window of kWalkCols at a
        // time in shared memory; the warp moves together (every lane computes
        // the same F values).
        // The walk asks for its current column c or c - 1, c never growing:
        // a window that misses the asked column is reloaded to end one past
        // it, so that it holds the current column as well.
        int64_t wlo = 0, whi = -1;               // columns [wlo, whi] are staged
        auto column = [&](int64_t c, uint32_t &v0, uint32_t &v1) {
            if (c < wlo || c > whi) {
                __syncwarp();
                whi = min(n, c + 1);
                wlo = max((int64_t)0, whi - kWalkCols + 1);
                const int64_t nc = whi - wlo + 1;
                for (int64_t e = lane; e < nc * W; e += 32) {
                    const int64_t cc = e / W;
                    const int w = (int)(e - cc * W);
                    S.win[cc][w] = col[(wlo + cc) * W + w];
                }
                __syncwarp();
            }
            const uint32_t *v = S.win[c - wlo];
            v0 = lane < W ? v[lane] : 0xFFFFFFFFu;
            v1 = lane + 32 < W ? v[lane + 32] : 0xFFFFFFFFu;
        };
        auto F = [&](int64_t c, int r) -> int {
            uint32_t v0, v1;
            column(c, v0, v1);
            return r - ones_below(v0, v1, r);
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
                if (S.a[r - 1] == bchar(c - 1) && F(c - 1, r - 1) == fc - 1) {   // diagonal into row r
                    --pos;
                    if (lane == 0 && pos >= 0) str[pos] = S.a[r - 1];
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

size_t batch_smem_bytes() { return (size_t)kBatchWarps * sizeof(BatchWarpSmem); }
int batch_max_rows() { return kBatchWords * 32; }

cudaError_t launch_batch_small(const BatchParams &bp, cudaStream_t st) {
    if (bp.count <= 0) return cudaSuccess;
    const size_t smem = batch_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_small_kernel, kBatchWarps * 32, smem)) !=
        cudaSuccess)
        return e;
    const int64_t need = ceil_div(bp.count, kBatchWarps);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * std::max(per_sm, 1)));
    batch_small_kernel<<<(unsigned)grid, kBatchWarps * 32, smem, st>>>(bp);
    return cudaGetLastError();
}

}  // namespace lcsg
