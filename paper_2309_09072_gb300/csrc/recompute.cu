// recompute.cu -- the traceback of a tree whose nodes were not kept.
//
// When the merge tree is built depth first with bounded memory, a node's
// DIST is freed once its parent has been merged, so the traceback cannot read
// the children.  It recomputes what it needs instead, node by node from the
// root down, as Hirschberg's split does: at a node covering rows [r0, r1)
// whose part of the path runs from top vertex i to bottom vertex j, with the
// halves split at row rm, the path crosses row rm at the smallest maximiser
//     c = min argmax_{i <= k <= j} U(i, k) + L(k, j)            (Sec. II-D)
// where U(i, k) = LCS(a[r0:rm], b[i:k]) is one row of the upper child's DIST
// and L(k, j) = LCS(a[rm:r1], b[k:j]) one column of the lower child's.  Both
// come from one bit-vector sweep each (the strip builder's column step):
// forward over a[r0:rm] from column i, where the carry out of the top row at
// column k is U(i, k) - U(i, k - 1), and backward over the reversed a[rm:r1]
// against the reversed b[i:j], where after t columns the count is L(j - t, j).
// The children then get (i, c) and (c, j); the strips at the bottom are
// resolved by the leaf kernel as before.
//
// node_sweep_kernel: block 2q sweeps node q of one depth forward, block
// 2q + 1 backward.  The vector is spread over NW warps of 32 lanes x 4 words
// (up to 4096 NW rows); rows past the half's height never match, which
// leaves the counts unchanged.  The sweep runs as a wavefront: lane g takes
// column c at step c + g with the carry that lane g - 1 produced for the same
// column one step earlier (a shuffle within a warp, shared memory and one
// named barrier per step across warps).
// node_pick_kernel: a CTA per node takes the smallest maximiser and hands the
// two sub-paths down.
#include <algorithm>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

namespace {

constexpr int kRcWL = 4;                     // words per lane
constexpr int kRcLetters = 32;               // distinct letters with a mask table

template <int NW>
struct RcCfg {
    static constexpr int W = 32 * NW * kRcWL;                          // words of the vector
    static constexpr size_t o_msk = 0;                                 // [kRcLetters][W]
    static constexpr size_t o_a = o_msk + (size_t)kRcLetters * W * 4;  // the half's letters, sweep order
    static constexpr size_t o_lmap = o_a + (size_t)W * 32;
    static constexpr size_t o_present = o_lmap + 256;
    static constexpr size_t o_xchg = o_present + 32;                   // [2][NW]
    static constexpr size_t o_b = (o_xchg + 2 * NW * 4 + 15) / 16 * 16;  // column letters, sweep order
    static constexpr int kBCols = 16384;                                // staged when the span fits
    static constexpr size_t bytes = o_b + kBCols + 64;
};

template <int NW, bool PAIRS>
__global__ void __launch_bounds__(NW * 32) node_sweep_kernel(SweepParams p) {
    pdl_wait_and_release();
    using C = RcCfg<NW>;
    constexpr int WL = kRcWL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t(*msk)[C::W] = reinterpret_cast<uint32_t(*)[C::W]>(smem_raw + C::o_msk);
    uint8_t *sa = smem_raw + C::o_a;
    uint8_t *lmap = smem_raw + C::o_lmap;
    uint32_t *present = reinterpret_cast<uint32_t *>(smem_raw + C::o_present);
    uint32_t *xchg = reinterpret_cast<uint32_t *>(smem_raw + C::o_xchg);
    uint8_t *sb = smem_raw + C::o_b;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.x >> 1;
    const bool back = (blockIdx.x & 1) != 0;
    if (q >= p.count) return;
    const SweepNode nd = p.nodes[q];
    // A tree's nodes share a and b; a batch's split pairs (PAIRS) each have
    // their own strings, no longer than p.n.
    const int64_t n = PAIRS ? p.pairs[q].n : p.n;
    const uint8_t *A = PAIRS ? p.pairs[q].a : p.a, *Bs = PAIRS ? p.pairs[q].b : p.b;
    int64_t i = p.pathI[nd.node], j = p.pathJ[nd.node];
    if (i < 0 || j > n || i > j || n > p.n) {             // never for a consistent tree
        if (tid == 0) set_error(p.err, ERR_BOUNDS);
        i = j = 0;
    }
    const int r0 = back ? nd.rm : nd.r0, h = back ? nd.r1 - nd.rm : nd.rm - nd.r0;
    if (h > 32 * C::W) {
        if (tid == 0) set_error(p.err, ERR_BOUNDS);
        return;
    }
    int32_t *cnt = (back ? p.bcnt : p.fcnt) + (int64_t)q * (p.n + 1);
    const int64_t span = j - i;
    // Rows in sweep order (backward: reversed), and the letters present;
    // the columns' letters in sweep order (sb[c] for column c, 1-based,
    // sb[0] and past the span unused) when they fit.
    if (tid < 8) present[tid] = 0u;
    const bool staged_b = span <= C::kBCols;
    if (staged_b)
        for (int c = tid; c < (int)span; c += blockDim.x) sb[c + 1] = back ? Bs[j - 1 - c] : Bs[i + c];
    __syncthreads();
    for (int r = tid; r < h; r += blockDim.x) {
        const uint8_t ch = A[back ? r0 + h - 1 - r : r0 + r];
        sa[r] = ch;
        atomicOr(&present[ch >> 5], 1u << (ch & 31));
    }
    __syncthreads();
    int nlet = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) nlet += __popc(present[t]);
    const bool table = nlet < kRcLetters;            // one row kept clear for absent letters
    if (table) {
        for (int c = tid; c < 256; c += blockDim.x) {
            const uint32_t word = present[c >> 5], bit = 1u << (c & 31);
            int rank = 0;
            for (int t = 0; t < (c >> 5); ++t) rank += __popc(present[t]);
            rank += __popc(word & (bit - 1u));
            lmap[c] = (word & bit) ? (uint8_t)rank : (uint8_t)255;
        }
        for (int t = tid; t < min(nlet + 1, kRcLetters) * C::W; t += blockDim.x) (&msk[0][0])[t] = 0u;
        __syncthreads();
        for (int r = tid; r < h; r += blockDim.x) atomicOr(&msk[lmap[sa[r]]][r >> 5], 1u << (r & 31));
    }
    __syncthreads();
    // The sweep as a wavefront: lane g (of NW * 32) holds rows 128 g .. 128 g
    // + 127 (4 words) and takes column c at step t = c + g, with the carry
    // out of lane g - 1's words for the same column, made one step earlier
    // (a shuffle within a warp; across warps through shared memory, one named
    // barrier per step).  A column then costs one add-with-carry chain of 4
    // words plus one shuffle on the critical path instead of a whole-vector
    // carry resolution.  Lanes above the half's height only pass carries
    // (their rows never match), so the carry out of the top lane that holds
    // rows of the half, gtop, is the count's increment.
    const int g = warp * 32 + lane;
    const int gtop = min(NW * 32, (h + 127) >> 7) - 1;
    const int w0 = g * WL;
    // The table's rows are zero past the half's height (those bits are never set),
    // and a lane above gtop never reads its mask; a letter absent from the
    // half reads the zero row nlet (cleared with the others below).
    auto masks = [&](uint8_t ch, uint32_t (&M)[WL]) {
        if (table) {
            const uint8_t k = lmap[ch];
            const uint4 q = *reinterpret_cast<const uint4 *>(&msk[k == 255 ? nlet : k][min(w0, C::W - WL)]);
            M[0] = q.x; M[1] = q.y; M[2] = q.z; M[3] = q.w;
        } else {
#pragma unroll
            for (int t = 0; t < WL; ++t) {
                uint32_t mk = 0u;
                const int rb = (w0 + t) * 32;
                for (int b = 0; b < 32 && rb + b < h; ++b) mk |= (uint32_t)(sa[rb + b] == ch) << b;
                M[t] = mk;
            }
        }
    };
    // Sweep column c (1-based) takes b[i + c - 1] forward, b[j - c] backward.
    const int span32 = (int)span;
    auto letter_at = [&](int c) -> uint8_t {
        if (c < 1 || c > span32) return (uint8_t)0;
        return staged_b ? sb[c] : (back ? Bs[j - c] : Bs[i + c - 1]);
    };
    uint32_t V[WL];
#pragma unroll
    for (int t = 0; t < WL; ++t) V[t] = 0xFFFFFFFFu;
    if (tid == 0) cnt[back ? span : 0] = 0;             // U(i, i) = 0, L(j, j) = 0
    int dist = 0;
    uint32_t cout = 0u;
    const int steps = span32 + gtop;
    // Operands one and two steps ahead: this lane's column at step t is t - g.
    uint8_t ch1 = letter_at(1 - g), ch2 = letter_at(2 - g);
    uint32_t Mn[WL];
    masks(ch1, Mn);
    for (int t = 1; t <= steps; ++t) {
        const int c = t - g;
        uint32_t cin = __shfl_up_sync(0xFFFFFFFFu, cout, 1);
        if constexpr (NW > 1) {
            if (lane == 0) cin = warp == 0 ? 0u : xchg[((t - 1) & 1) * NW + warp - 1];
        } else {
            if (lane == 0) cin = 0u;
        }
        uint32_t M[WL];
#pragma unroll
        for (int k = 0; k < WL; ++k) M[k] = Mn[k];
        // The next step's mask and the letter after it load while this
        // step's chain runs.
        masks(ch2, Mn);
        ch2 = letter_at(t + 2 - g);
        const bool active = c >= 1 && c <= span32 && g <= gtop;
        uint32_t co = 0u;
        if (active) {
            uint32_t u[WL], sum[WL];
#pragma unroll
            for (int k = 0; k < WL; ++k) u[k] = V[k] & M[k];
            co = addn_cin<WL>(sum, V, u, cin);
#pragma unroll
            for (int k = 0; k < WL; ++k) V[k] = sum[k] | (V[k] & ~M[k]);
            if (g == gtop) {
                dist += (int)co;
                cnt[back ? span - c : c] = dist;   // U(i, i + c), or L(j - c, j)
            }
        }
        cout = co;
        if constexpr (NW > 1) {
            if (lane == 31) xchg[(t & 1) * NW + warp] = co;
            named_bar_sync(1, NW * 32);
        }
    }
}

__global__ void __launch_bounds__(256) node_pick_kernel(SweepParams p) {
    pdl_wait_and_release();
    __shared__ int sv[8];
    __shared__ int64_t sk[8];
    const int q = blockIdx.x;
    const SweepNode nd = p.nodes[q];
    const int64_t n = p.pairs ? p.pairs[q].n : p.n;
    int64_t i = p.pathI[nd.node], j = p.pathJ[nd.node];
    if (i < 0 || j > n || i > j || n > p.n) i = j = 0;  // flagged by the sweep
    const int32_t *f = p.fcnt + (int64_t)q * (p.n + 1), *g = p.bcnt + (int64_t)q * (p.n + 1);
    int best = INT32_MIN;
    int64_t bk = INT64_MAX;
    for (int64_t k = i + threadIdx.x; k <= j; k += blockDim.x) {
        const int v = f[k - i] + g[k - i];
        if (v > best) { best = v; bk = k; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const int ov = __shfl_xor_sync(0xFFFFFFFFu, best, off);
        const int64_t ok = __shfl_xor_sync(0xFFFFFFFFu, bk, off);
        if (ov > best || (ov == best && ok < bk)) { best = ov; bk = ok; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sv[warp] = best; sk[warp] = bk; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && sk[w] < bk)) { best = sv[w]; bk = sk[w]; }
        const int32_t c = (int32_t)bk;
        p.pathI[nd.upper] = (int32_t)i;
        p.pathJ[nd.upper] = c;
        p.pathI[nd.lower] = c;
        p.pathJ[nd.lower] = (int32_t)j;
        if (p.pairs) {
            if (p.pairs[q].len_out) *p.pairs[q].len_out = best;
        } else if (nd.node == p.root_node && p.len_out) {
            *p.len_out = best;
        }
    }
}

template <int NW>
cudaError_t launch_sweep_t(const SweepParams &p, cudaStream_t st) {
    const size_t smem = RcCfg<NW>::bytes;
    auto kern = p.pairs ? node_sweep_kernel<NW, true> : node_sweep_kernel<NW, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, dim3((unsigned)(2 * p.count)), dim3(NW * 32), smem, st, p);
}

}  // namespace

int sweep_max_rows() { return 32 * RcCfg<4>::W; }

cudaError_t launch_node_sweep(const SweepParams &p, int max_rows, cudaStream_t st) {
    if (p.count <= 0) return cudaSuccess;
    if (max_rows <= 32 * RcCfg<1>::W) return launch_sweep_t<1>(p, st);
    if (max_rows <= 32 * RcCfg<2>::W) return launch_sweep_t<2>(p, st);
    if (max_rows <= 32 * RcCfg<4>::W) return launch_sweep_t<4>(p, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_node_pick(const SweepParams &p, cudaStream_t st) {
    if (p.count <= 0) return cudaSuccess;
    return launch_pdl(node_pick_kernel, dim3((unsigned)p.count), dim3(256), 0, st, p);
}

}  // namespace lcsg
