// batch_big.cu -- tall pairs of a batch (more than 4096 rows): several warps
// per sweep, and the LCS without a serial walk.
//
// A batch pair with more than 4096 rows takes this path instead of the
// one-warp kernel of batch.cu: its sweep spreads the vector over several
// warps, and when it wants its string the one-warp walk (whose ~m + n
// dependent steps would dominate such a pair) is replaced as follows.  With F the strip's DP from the source (0, 0)
// and B the DP from the sink (m, n), the vertices on heaviest paths are those
// with F(r, c) + B(r, c) = L, so the leftmost heaviest path enters row r at
//     v[r] = min{ c : F(r, c) + B(r, c) = L }            (Sec. II-C),
// and the step into row r is a match diagonal, marking letter a_r
// (Sec. II-E), exactly when v[r] > v[r-1] and a_r = b_{v[r]}: the rule of
// the single-pair leaf (traceback.cu), on one strip of the whole pair.
//   1. big_sweep_kernel: a CTA sweeps the pair forward (a against b) and
//      another backward (reversed a against reversed b), each with the strip
//      builder's column step, the vector spread over four warps (carry
//      look-ahead within and across them), storing every column's vector
//      word-major (word w of column c at w * (n+1) + c, so that 32
//      consecutive columns read one word coalesced).  The forward CTA also
//      gives the length.
//   2. big_cross_kernel: a lane per column runs down the rows, its count of
//      ones moving by (forward bit - backward bit); hits are collected as
//      32-row masks, transposed across the warp, and the smallest column of
//      each row is folded in with atomicMin.
//   3. big_marks_kernel: a CTA per pair marks the rows and writes the LCS.
#include <algorithm>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

constexpr int kBigLetters = 32;           // distinct letters with a mask table, else direct compares

template <int WPL>
struct BigCfg {
    static constexpr int W = 32 * WPL;                                  // words of the tallest a
    static constexpr int NW = WPL / 4;                                  // warps per sweep (4 words per lane)
    static constexpr int WL = WPL / NW;                                 // words per lane
    static constexpr size_t o_msk = 0;                                  // [kBigLetters][W]
    static constexpr size_t o_a = o_msk + (size_t)kBigLetters * W * 4;  // the strip's letters, in sweep order
    static constexpr size_t o_lmap = o_a + (size_t)W * 32;
    static constexpr size_t o_present = o_lmap + 256;
    static constexpr size_t o_xchg = o_present + 32;                    // [2][NW] warp generate/propagate
    // Column vectors staged 32 at a time for coalesced stores: measured to pay
    // with 4 warps (16384 rows: 6.3 -> 5.7 ms), not with 2 (8192: 2.4 -> 2.8).
    static constexpr bool STAGE = NW >= 4;
    static constexpr int CP = W + 1;                                    // stage pitch (odd: no bank conflicts)
    static constexpr size_t o_cols = (o_xchg + 2 * NW * 4 + 15) / 16 * 16;   // [32][CP] staged columns
    static constexpr size_t bytes = (o_cols + (STAGE ? (size_t)32 * CP * 4 : 0) + 15) / 16 * 16;
};

// Block 2q sweeps pair q forward, block 2q + 1 backward (only for a pair
// that wants its string).  The m-bit vector is spread over NW warps (4
// words per lane), lane l of warp w holding words (32 w + l) WL .. + WL - 1.  Within a warp the carries cross the lanes by
// the look-ahead on two ballots; across the warps each warp publishes its
// block's generate (carry out with no carry in) and propagate (every word
// all ones) bits, a named barrier per column, and a warp's carry in is then
// the carry of the chain of the warps below it.
template <int WPL>
__global__ void __launch_bounds__(BigCfg<WPL>::NW * 32) big_sweep_kernel(BigParams p) {
    pdl_wait_and_release();
    using C = BigCfg<WPL>;
    constexpr int WL = C::WL, NW = C::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t(*msk)[C::W] = reinterpret_cast<uint32_t(*)[C::W]>(smem_raw + C::o_msk);
    uint8_t *sa = smem_raw + C::o_a;
    uint8_t *lmap = smem_raw + C::o_lmap;
    uint32_t *present = reinterpret_cast<uint32_t *>(smem_raw + C::o_present);
    uint32_t *xchg = reinterpret_cast<uint32_t *>(smem_raw + C::o_xchg);   // bit 0: generate, bit 1: propagate
    uint32_t *cols = reinterpret_cast<uint32_t *>(smem_raw + C::o_cols);   // 32 columns' vectors, column-major
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.x >> 1;
    const bool back = (blockIdx.x & 1) != 0;
    if (q >= p.count) return;
    const BatchPair pr = p.pairs[q];
    const bool want = pr.want != 0;
    if (back && !want) return;                   // length only: no backward sweep
    const int m = (int)pr.m;
    const int64_t n = pr.n;
    if (m <= 0 || n <= 0 || m > 32 * C::W) {
        if (tid == 0 && !back) {
            pr.len_out[0] = 0;
            if (m > 32 * C::W) set_error(p.err, ERR_BOUNDS);
        }
        return;
    }
    const int Wu = (m + 31) >> 5;
    uint32_t *vec = p.scratch + pr.scratch_off + (back ? (int64_t)Wu * (n + 1) : 0);
    // Rows in sweep order: the backward sweep takes a reversed.
    if (tid < 8) present[tid] = 0u;
    __syncthreads();
    for (int r = tid; r < m; r += blockDim.x) {
        const uint8_t ch = pr.a[back ? m - 1 - r : r];
        sa[r] = ch;
        atomicOr(&present[ch >> 5], 1u << (ch & 31));
    }
    __syncthreads();
    int nlet = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) nlet += __popc(present[t]);
    const bool table = nlet <= kBigLetters;
    if (table) {
        for (int c = tid; c < 256; c += blockDim.x) {
            const uint32_t word = present[c >> 5], bit = 1u << (c & 31);
            int rank = 0;
            for (int t = 0; t < (c >> 5); ++t) rank += __popc(present[t]);
            rank += __popc(word & (bit - 1u));
            lmap[c] = (word & bit) ? (uint8_t)rank : (uint8_t)255;
        }
        for (int t = tid; t < nlet * C::W; t += blockDim.x) (&msk[0][0])[t] = 0u;
        __syncthreads();
        for (int r = tid; r < m; r += blockDim.x) atomicOr(&msk[lmap[sa[r]]][r >> 5], 1u << (r & 31));
    }
    __syncthreads();
    const int w0 = (warp * 32 + lane) * WL;      // this lane's first word
    auto masks = [&](uint8_t ch, uint32_t (&M)[WL]) {
        if (table) {
            const uint8_t k = lmap[ch];
#pragma unroll
            for (int t = 0; t < WL; ++t) M[t] = (k == 255 || w0 + t >= Wu) ? 0u : msk[k][w0 + t];
        } else {
#pragma unroll
            for (int t = 0; t < WL; ++t) {
                uint32_t mk = 0u;
                const int r0 = (w0 + t) * 32;
                for (int b = 0; b < 32 && r0 + b < m; ++b) mk |= (uint32_t)(sa[r0 + b] == ch) << b;
                M[t] = mk;
            }
        }
    };
    uint32_t V[WL];
#pragma unroll
    for (int t = 0; t < WL; ++t) V[t] = 0xFFFFFFFFu;
    // Column vectors, word-major: with STAGE, 32 columns at a time staged in
    // shared memory (lane words contiguous) and then written 32 consecutive
    // columns of one word per warp store; else each lane writes its words.
    auto stage = [&](int slot, int64_t c) {
        if (!want) return;
        if constexpr (C::STAGE) {
#pragma unroll
            for (int t = 0; t < WL; ++t) cols[slot * C::CP + w0 + t] = V[t];
        } else {
#pragma unroll
            for (int t = 0; t < WL; ++t)
                if (w0 + t < Wu) vec[(int64_t)(w0 + t) * (n + 1) + c] = V[t];
        }
    };
    auto flush = [&](int64_t c0, int cnt) {
        if constexpr (!C::STAGE) return;
        if (!want) return;
        __syncthreads();
        for (int w = warp; w < Wu; w += NW)
            if (lane < cnt) vec[(int64_t)w * (n + 1) + c0 + lane] = cols[lane * C::CP + w];
        __syncthreads();
    };
    stage(0, 0);
    flush(0, 1);
    int dist = 0;
    int par = 0;
    // Column c' of the sweep takes b[c' - 1] forward, b[n - c'] backward.
    auto letter_at = [&](int64_t cc) -> uint32_t { return back ? pr.b[n - cc] : pr.b[cc - 1]; };
    uint32_t bnext = (1 + lane <= n) ? letter_at(1 + lane) : 0u;
    for (int64_t blk = 1; blk <= n; blk += 32) {
        const uint32_t bcur = bnext;
        bnext = (blk + 32 + lane <= n) ? letter_at(blk + 32 + lane) : 0u;
        const int cnt = (int)min((int64_t)32, n - blk + 1);
        for (int t = 0; t < cnt; ++t) {
            const uint8_t ch = (uint8_t)__shfl_sync(0xFFFFFFFFu, bcur, t);
            uint32_t M[WL], s[WL], u[WL];
            masks(ch, M);
#pragma unroll
            for (int k = 0; k < WL; ++k) u[k] = V[k] & M[k];
            const uint32_t carry = addn_cin<WL>(s, V, u, 0u);
            uint32_t below[WL];
            below[0] = 1u;
#pragma unroll
            for (int k = 1; k < WL; ++k) below[k] = below[k - 1] & (s[k - 1] == 0xFFFFFFFFu ? 1u : 0u);
            const bool ones = (below[WL - 1] & (s[WL - 1] == 0xFFFFFFFFu ? 1u : 0u)) != 0u;
            const uint32_t G = __ballot_sync(0xFFFFFFFFu, carry != 0u), Pb = __ballot_sync(0xFFFFFFFFu, ones);
            const uint32_t A = G | Pb;
            // The warp's generate and propagate, published for the warps above.
            const uint32_t wg = (uint32_t)(((uint64_t)A + G) >> 32), wp = Pb == 0xFFFFFFFFu ? 1u : 0u;
            if (lane == 0) xchg[par * NW + warp] = wg | (wp << 1);
            named_bar_sync(1, NW * 32);
            uint32_t cw = 0u;                        // carry into this warp
            uint32_t ctop = 0u;                      // carry out of the whole vector
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t e = xchg[par * NW + w];
                const uint32_t cout = (e & 1u) | ((e >> 1) & ctop);
                if (w == warp) cw = ctop;
                ctop = cout;
            }
            par ^= 1;
            const uint64_t S = (uint64_t)A + G + cw;
            const uint32_t cin = (((uint32_t)S ^ A ^ G) >> lane) & 1u;
            dist += (int)ctop;                       // DIST(i, j) - DIST(i, j-1)
#pragma unroll
            for (int k = 0; k < WL; ++k) V[k] = (s[k] + (cin & below[k])) | (V[k] & ~M[k]);
            stage(t, blk + t);
        }
        flush(blk, cnt);
    }
    if (!back && tid == 0) {
        pr.len_out[0] = dist;                     // DIST(0, n) = LCS(a, b)
        p.lens[q] = dist;
    }
}

// Warp g of pair q (blockIdx.y) takes columns 32 g .. 32 g + 31.
__global__ void __launch_bounds__(128) big_cross_kernel(BigParams p) {
    pdl_wait_and_release();
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.y;
    const BatchPair pr = p.pairs[q];
    const int m = (int)pr.m;
    const int64_t n = pr.n;
    const int64_t grp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (!pr.want || m <= 0 || n <= 0 || grp * 32 > n) return;
    const int Wu = (m + 31) >> 5;
    const uint32_t *fwd = p.scratch + pr.scratch_off;
    const uint32_t *bwd = fwd + (int64_t)Wu * (n + 1);
    int32_t *v = reinterpret_cast<int32_t *>(const_cast<uint32_t *>(bwd + (int64_t)Wu * (n + 1)));
    const int L = p.lens[q];
    const int target = m - L;                  // ones(F, < r) + ones(B, < m - r) = m - L on the path
    const int64_t c = grp * 32 + lane;
    const bool live = c <= n;
    const int64_t cb = n - c;                  // the backward sweep's column for c
    auto fword = [&](int w) -> uint32_t { return live && w >= 0 && w < Wu ? fwd[(int64_t)w * (n + 1) + c] : 0u; };
    auto bword = [&](int w) -> uint32_t { return live && w >= 0 && w < Wu ? bwd[(int64_t)w * (n + 1) + cb] : 0u; };
    // r = 0: every one of the backward vector's first m bits.
    int d = INT32_MIN / 2;
    if (live) {
        d = 0;
        for (int w = 0; w < Wu; ++w) {
            const int k = min(m - 32 * w, 32);
            d += __popc(bword(w) & (k == 32 ? 0xFFFFFFFFu : ((1u << k) - 1u)));
        }
    }
    for (int w = 0; w < Wu; ++w) {
        // Rows 32 w + 1 .. 32 w + 32 use forward bits 32 w + t and backward
        // bits m - 1 - 32 w - t: the 32 backward bits from q0 = m - 32 - 32 w
        // up, reversed.
        const uint32_t fw0 = fword(w);
        const int q0 = m - 32 - 32 * w;
        const int wq = q0 >= 0 ? (q0 >> 5) : -1, sq = q0 - 32 * wq;
        const uint64_t pairw = ((uint64_t)bword(wq + 1) << 32) | bword(wq);
        const uint32_t gw0 = __brev((uint32_t)(pairw >> sq));
        uint32_t fw = fw0, gw = gw0, hits = 0u;
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
            d += (int)(fw & 1u) - (int)(gw & 1u);
            fw >>= 1;
            gw >>= 1;
            hits |= (d == target ? 1u : 0u) << t;
        }
        const int valid = m - 32 * w;              // rows past m in the last word: dropped
        if (valid < 32) hits &= (1u << valid) - 1u;
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
            const uint32_t mk = sh == 16 ? 0x0000FFFFu : sh == 8 ? 0x00FF00FFu : sh == 4 ? 0x0F0F0F0Fu
                                                             : sh == 2 ? 0x33333333u : 0x55555555u;
            const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, hits, sh);
            hits = (lane & sh) ? ((hits & ~mk) | ((y & ~mk) >> sh)) : ((hits & mk) | ((y & mk) << sh));
        }
        if (hits) atomicMin(&v[32 * w + lane + 1], (int32_t)(grp * 32 + __ffs(hits) - 1));
    }
}

// A CTA per pair: marks, their ranks (block scan in chunks), the LCS.
__global__ void __launch_bounds__(1024) big_marks_kernel(BigParams p) {
    pdl_wait_and_release();
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    __shared__ int bad;
    const int64_t q = blockIdx.x;
    const BatchPair pr = p.pairs[q];
    const int m = (int)pr.m;
    const int64_t n = pr.n;
    if (!pr.want || m <= 0 || n <= 0) return;
    const int Wu = (m + 31) >> 5;
    const int32_t *v = reinterpret_cast<const int32_t *>(p.scratch + pr.scratch_off + 2 * (int64_t)Wu * (n + 1));
    uint8_t *str = p.strings + pr.str_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        bad = 0;
    }
    __syncthreads();
    for (int base = 0; base < m; base += 1024) {
        const int r = base + (int)threadIdx.x + 1;   // rows 1 .. m
        bool mark = false;
        if (r <= m) {
            const int32_t cr = v[r], cp = r == 1 ? 0 : v[r - 1];
            if (cr < 0 || cr > n || cp < 0 || cp > n) bad = 1;
            else mark = cr > cp && pr.a[r - 1] == pr.b[cr - 1];
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, mark);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = carry + __popc(bal & ((1u << lane) - 1u)), tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) before += wsum[w];
            tot += wsum[w];
        }
        if (mark && before < p.lens[q]) str[before] = pr.a[r - 1];
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && (bad || carry != p.lens[q])) set_error(p.err, ERR_BOUNDS);
}

cudaError_t launch_big(const BigParams &p, int wpl, cudaStream_t st) {
    if (p.count <= 0) return cudaSuccess;
    cudaError_t e;
    if (wpl == 8) {
        auto k = big_sweep_kernel<8>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BigCfg<8>::bytes)) != cudaSuccess)
            return e;
        if ((e = launch_pdl(k, dim3((unsigned)(2 * p.count)), dim3(BigCfg<8>::NW * 32), BigCfg<8>::bytes, st, p)) != cudaSuccess) return e;
    } else if (wpl == 16) {
        auto k = big_sweep_kernel<16>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BigCfg<16>::bytes)) != cudaSuccess)
            return e;
        if ((e = launch_pdl(k, dim3((unsigned)(2 * p.count)), dim3(BigCfg<16>::NW * 32), BigCfg<16>::bytes, st, p)) != cudaSuccess) return e;
    } else {
        return cudaErrorInvalidValue;
    }
    const int64_t groups = ceil_div(p.max_n + 1, 32);
    if ((e = launch_pdl(big_cross_kernel, dim3((unsigned)ceil_div(groups, 4), (unsigned)p.count), dim3(128), 0, st, p)) !=
        cudaSuccess)
        return e;
    return launch_pdl(big_marks_kernel, dim3((unsigned)p.count), dim3(1024), 0, st, p);
}

}  // namespace lcsg
