// traceback.cu -- one LCS from the merge tree (Sec. II-C..II-E).
//
// The cross vertex v[r] of row r is the leftmost vertex of the heaviest path
// in that row (Sec. II-C).  At a tree node covering rows [r0, r1) whose path
// runs from top vertex i = v[r0] to bottom vertex j, the cross vertex on the
// boundary row s between its halves is the smallest maximiser
//     c = min argmax_{i <= k <= j} U(i, k) + L(k, j)
// (Sec. II-D: it is a by-product of the merge), and the two halves get the
// sub-paths (i, c) and (c, j).  tb_path_kernel resolves every split above
// the strips in one launch (a CTA per strip walks from the root down to its
// strip); tb_level_kernel resolves one tree level per launch (the root level
// alone gives the length).  Inside a strip (leaf) the rows are resolved
// directly from the bit vectors of F(r, c) = LCS(a_strip[0:r], b[i:c]) and
// of the backward B: the path enters row r at the smallest c with
// F + B = L (see leaf_kernel); letter a_r is marked when the path enters row
// r by a weight-1 diagonal (Sec. II-E).  The marked letters of all strips, in
// row order, are the LCS.
#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

// ------------------------------------------------------------------ per-node argmax
// The smallest maximiser c of U(i, k) + L(k, j) over i <= k <= j for merge mg,
// and the maximum, by the whole CTA (returned to every thread).  sv, sk: a
// slot per warp.
__device__ void node_argmax(const TbParams &p, const TbMerge &mg, int64_t i, int64_t j, int *sv, int64_t *sk,
                            int32_t &c_out, int &best_out) {
    // The leftmost argmax is monotone in both coordinates (Monge), so with the
    // merge's argmax grid it lies between the grid's values at the tile
    // corners around (i, j).
    int64_t lo = i, hi = j;
    if (mg.kgrid) {
        const int64_t P = (p.n + T - 1) >> T_SHIFT;
        const int64_t I0 = min(i >> T_SHIFT, P), J0 = min(j >> T_SHIFT, P);
        const int64_t I1 = min(I0 + 1, P), J1 = min(J0 + 1, P);
        lo = max(lo, (int64_t)mg.kgrid[I0 * (P + 1) + J0]);
        hi = min(hi, (int64_t)mg.kgrid[I1 * (P + 1) + J1]);
        if (lo > hi) {                       // not a DIST merge's grid: the whole row
            lo = i;
            hi = j;
        }
    }
    int best = INT32_MIN;
    int64_t bk = INT64_MAX;
    if (mg.in_dtype == DT_I16) {
        // Thread t takes four consecutive k at offset 4 (t mod 16) of K-tiles
        // lo/T + t/16, + 16, .. (8-byte loads of U's stored row i and L's
        // stored column j; both tiles advance by one per K-tile).
        constexpr int PI = Fmt<int16_t>::P;
        constexpr int64_t EI = Fmt<int16_t>::ELEMS;
        const int16_t *U = reinterpret_cast<const int16_t *>(mg.U);
        const int16_t *L = reinterpret_cast<const int16_t *>(mg.L);
        const int64_t Ib = i >> T_SHIFT, Jb = j >> T_SHIFT, K0 = lo >> T_SHIFT;
        const int kl = (int)(threadIdx.x >> 4), o = 4 * (int)(threadIdx.x & 15);
        const int64_t step = (int64_t)(blockDim.x >> 4) * EI;
        const int16_t *up = U + row_tile(Ib, K0 + kl, p.NT) * EI + (i & (T - 1)) * PI + o;
        const int16_t *lp = L + col_tile(K0 + kl, Jb) * EI + (j & (T - 1)) * PI + o;
        for (int64_t kt = K0 + kl; kt <= (hi >> T_SHIFT); kt += blockDim.x >> 4, up += step, lp += step) {
            const int64_t kb = (kt << T_SHIFT) + o;
            if (kb > hi) break;
            const uint2 uu = *reinterpret_cast<const uint2 *>(up);
            const uint2 ll = *reinterpret_cast<const uint2 *>(lp);
            const uint32_t uw[2] = {uu.x, uu.y}, lw[2] = {ll.x, ll.y};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t k = kb + e;
                const int v = (int)(int16_t)(uw[e >> 1] >> (16 * (e & 1))) + (int)(int16_t)(lw[e >> 1] >> (16 * (e & 1)));
                if (k >= lo && k <= hi && v > best) { best = v; bk = k; }   // k increases: first max per thread
            }
        }
    } else {
        for (int64_t k = lo + threadIdx.x; k <= hi; k += blockDim.x) {
            const int v = load_row_any(mg.U, i, k, p.NT, mg.in_dtype) + load_col_any(mg.L, k, j, mg.in_dtype);
            if (v > best) { best = v; bk = k; }
        }
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
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (sv[w] > best || (sv[w] == best && sk[w] < bk)) { best = sv[w]; bk = sk[w]; }
    __syncthreads();                         // sv, sk free again
    c_out = (int32_t)bk;
    best_out = best;
}

__global__ void __launch_bounds__(256) tb_level_kernel(TbParams p) {
    pdl_wait_and_release();
    __shared__ int sv[8];
    __shared__ int64_t sk[8];
    const TbMerge mg = p.merges[blockIdx.x];
    int64_t i = p.pathI[mg.node], j = p.pathJ[mg.node];
    if (i < 0 || j > p.n || i > j) {          // never for a consistent tree
        if (threadIdx.x == 0) set_error(p.err, ERR_BOUNDS);
        i = 0;
        j = 0;
    }
    int32_t c;
    int best;
    node_argmax(p, mg, i, j, sv, sk, c, best);
    if (threadIdx.x == 0) {
        p.pathI[mg.upper] = (int32_t)i;
        p.pathJ[mg.upper] = c;
        p.pathI[mg.lower] = c;
        p.pathJ[mg.lower] = (int32_t)j;
        if (mg.node == p.root_node && p.len_out) *p.len_out = best;
    }
}

// One CTA per strip walks the tree from the root down to the strip, taking
// the split of every node on its way (the upper nodes' splits are taken by
// every CTA under them, the same values), so the whole traceback above the
// leaves is one launch.  chain[s * depth_max + d] is the tb merge of depth d
// on strip s's way down (depth[s] of them).
__global__ void __launch_bounds__(256) tb_path_kernel(TbParams p, const int32_t *chain, const int32_t *depth,
                                                      int32_t depth_max) {
    pdl_wait_and_release();
    __shared__ int sv[8];
    __shared__ int64_t sk[8];
    const int s = blockIdx.x;
    int64_t i = 0, j = p.n;
    const int nd = depth[s];
    if (s == 0 && threadIdx.x == 0) {
        p.pathI[p.root_node] = 0;            // the whole path, source to sink
        p.pathJ[p.root_node] = (int32_t)p.n;
    }
    for (int d = 0; d < nd; ++d) {
        const TbMerge mg = p.merges[chain[(int64_t)s * depth_max + d]];
        int32_t c;
        int best;
        node_argmax(p, mg, i, j, sv, sk, c, best);
        if (threadIdx.x == 0) {
            p.pathI[mg.upper] = (int32_t)i;
            p.pathJ[mg.upper] = c;
            p.pathI[mg.lower] = c;
            p.pathJ[mg.lower] = (int32_t)j;
            if (d == 0 && p.len_out) *p.len_out = best;
        }
        const int32_t next = d + 1 < nd ? p.merges[chain[(int64_t)s * depth_max + d + 1]].node : s;
        if (next == mg.upper) j = c;
        else i = c;
    }
}

cudaError_t launch_tb_path(const TbParams &p, const int32_t *chain, const int32_t *depth, int32_t depth_max,
                           int32_t strips, cudaStream_t st) {
    if (strips <= 0) return cudaSuccess;
    return launch_pdl(tb_path_kernel, dim3((unsigned)strips), dim3(256), 0, st, p, chain, depth, depth_max);
}

__global__ void root_path_kernel(int32_t *pI, int32_t *pJ, int32_t root, int32_t n) {
    pdl_wait_and_release();
    pI[root] = 0;
    pJ[root] = n;
}

cudaError_t launch_root_path(int32_t *pathI, int32_t *pathJ, int32_t root, int64_t n, cudaStream_t st) {
    return launch_pdl(root_path_kernel, dim3(1), dim3(1), 0, st, pathI, pathJ, root, (int32_t)n);
}

cudaError_t launch_tb_level(const TbParams &p, cudaStream_t st) {
    if (p.count <= 0) return cudaSuccess;
    return launch_pdl(tb_level_kernel, dim3((unsigned)p.count), dim3(256), 0, st, p);
}

// ------------------------------------------------------------------ leaves
// One CTA per strip, whose part of the path runs from (0, i) to (hs, j).
// With F(r, c) = LCS(a_strip[0:r], b[i:c]) (forward from the source) and
// B(r, c) = LCS(a_strip[r:hs], b[c:j]) (backward from the sink), the
// vertices on heaviest paths are those with F + B = L = F(hs, j), so the
// leftmost heaviest path enters row r at
//     v[r] = min{ c in [i, j] : F(r, c) + B(r, c) = L }     (Sec. II-C),
// and the step into row r is a match diagonal, marking letter a_r
// (Sec. II-E), exactly when v[r] > v[r-1] and a_r = b_{v[r]} (a vertical
// step where the diagonal into the same vertex matches would give up one
// unit of weight).  Warp 0 sweeps the columns forward and warp 1 backward
// (the reversed strip against the reversed segment of b), both with the
// bit-vector step of the strip builder, storing every column's vector; then
// all warps test F + B = L for a slice of the columns, a lane per group of
// rows, and the first hit of each row is its cross vertex.
constexpr int kLeafThreads = 256;
constexpr int kLeafSmemCols = 1024;   // columns whose vectors fit shared memory

struct LeafSmem {
    size_t fm, fmr, vf, vb, vr, vmin, wsum, sa, sb, total;
};
__host__ __device__ constexpr LeafSmem leaf_smem_layout(int W) {
    LeafSmem L{};
    size_t off = 0;
    L.fm = off;   off += (size_t)256 * W * 4;                      // forward row masks per letter
    L.fmr = off;  off += (size_t)256 * W * 4;                      // the same over reversed rows
    L.vf = off;   off += (size_t)(kLeafSmemCols + 1) * W * 4;      // forward column vectors
    L.vb = off;   off += (size_t)(kLeafSmemCols + 1) * W * 4;      // backward column vectors
    L.vr = off;   off += (size_t)(kLeafSmemCols + 1) * W * 4;      // backward ones, in forward row order
    L.vmin = off; off += (size_t)(256 + 1) * 4;                    // cross vertex per row
    L.wsum = off; off += 16 * 4;                                   // scan of the marks
    L.sa = off;   off += 256;                                      // the strip's letters
    L.sb = off;   off += kLeafSmemCols;                            // b[i .. j - 1]
    L.total = (off + 15) / 16 * 16;
    return L;
}

// Ones among the first `bits` bits of a W-word vector.
template <int W>
__device__ __forceinline__ int prefix_ones(const uint32_t (&v)[W], int bits) {
    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int k = min(max(bits - 32 * w, 0), 32);
        const uint32_t mask = k == 32 ? 0xFFFFFFFFu : ((1u << k) - 1u);
        ones += __popc(v[w] & mask);
    }
    return ones;
}

// W words to shared memory with the widest stores their alignment allows
// (a column's vector starts on a 4 W-byte boundary).
template <int W>
__device__ __forceinline__ void store_words(uint32_t *dst, const uint32_t (&v)[W]) {
    if constexpr (W >= 4) {
#pragma unroll
        for (int w = 0; w < W; w += 4)
            *reinterpret_cast<uint4 *>(dst + w) = make_uint4(v[w], v[w + 1], v[w + 2], v[w + 3]);
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1]);
    } else {
        dst[0] = v[0];
    }
}

// Sweep of `ncol` columns from the all-ones vector; column c (1-based) uses
// the masks of letter seg[rev ? ncol - c : c - 1].  Every lane steps the
// whole vector (one add-with-carry chain per column, no cross-lane traffic
// on the dependent path), and every column's
// vector, column 0 included (lane 0 writes it).  The letter and its masks
// are fetched two and one columns ahead.
template <int W>
__device__ __forceinline__ void leaf_sweep(const uint32_t *masks, const uint8_t *seg, int ncol, bool rev,
                                           uint32_t *out, int lane) {
    uint32_t V[W];
#pragma unroll
    for (int w = 0; w < W; ++w) V[w] = 0xFFFFFFFFu;
    if (lane == 0) store_words<W>(out, V);
    auto letter = [&](int c) -> int { return seg[rev ? ncol - c : c - 1]; };   // 1 <= c <= ncol
    uint32_t M[W];
    int chn = 0;
    if (ncol > 0) {
        const uint32_t *m0 = masks + letter(1) * W;
#pragma unroll
        for (int w = 0; w < W; ++w) M[w] = m0[w];
        chn = letter(ncol > 1 ? 2 : 1);
    }
    for (int c = 1; c <= ncol; ++c) {
        uint32_t Mn[W];
        const uint32_t *mn = masks + chn * W;
#pragma unroll
        for (int w = 0; w < W; ++w) Mn[w] = mn[w];
        chn = letter(c + 2 <= ncol ? c + 2 : ncol);
        column_step<W>(V, M);
        if (lane == 0) store_words<W>(out + c * W, V);
#pragma unroll
        for (int w = 0; w < W; ++w) M[w] = Mn[w];
    }
}

// Strips whose segment of b is longer than kLeafSmemCols: warp 0 alone, the
// forward vectors in the global scratch, then one lane walks back from the
// sink: left while F keeps its value, else along the match diagonal if it
// is tight, else up (which leaves each row at its leftmost vertex).
template <int W>
__device__ void leaf_walk_global(const LeafParams &p, int s, int64_t r0, int hs, int64_t i, int64_t j,
                                 const uint32_t *fm, const uint8_t *sa, int lane) {
    uint32_t *vb = p.vbuf + (i + s) * (int64_t)W;
    uint32_t V[W];
#pragma unroll
    for (int w = 0; w < W; ++w) V[w] = 0xFFFFFFFFu;
    if (lane < W) vb[lane] = 0xFFFFFFFFu;
    for (int64_t c = i + 1; c <= j; ++c) {
        const uint32_t *m = fm + p.b[c - 1] * W;
        uint32_t M[W];
#pragma unroll
        for (int w = 0; w < W; ++w) M[w] = m[w];
        column_step<W>(V, M);
        uint32_t mine = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) mine = lane == w ? V[w] : mine;
        if (lane < W) vb[(c - i) * W + lane] = mine;
    }
    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) ones += __popc(V[w]);
    const int Ltot = 32 * W - ones;              // padding bits stay 1
    __syncwarp();
    if (lane != 0) return;
    auto F = [&](int64_t c, int r) -> int {
        uint32_t vv[W];
#pragma unroll
        for (int w = 0; w < W; ++w) vv[w] = vb[(c - i) * W + w];
        return r - prefix_ones<W>(vv, r);
    };
    int r = hs;
    int64_t c = j;
    int pos = Ltot;
    int fc = F(c, r);
    while (r > 0) {
        if (c > i) {
            if (F(c - 1, r) == fc) {
                --c;
                continue;
            }
            if (sa[r - 1] == p.b[c - 1] && F(c - 1, r - 1) == fc - 1) {
                if (p.cross) p.cross[r0 + r] = (int32_t)c;
                --pos;
                if (pos >= 0) p.slots[(int64_t)s * p.h + pos] = sa[r - 1];
                --r;
                --c;
                --fc;
                continue;
            }
        }
        if (p.cross) p.cross[r0 + r] = (int32_t)c;
        --r;
        fc = F(c, r);
    }
    if (s == 0 && p.cross) p.cross[0] = (int32_t)i;
    p.counts[s] = Ltot;
    if (pos != 0) set_error(p.err, ERR_BOUNDS);
}

template <int W>
__global__ void __launch_bounds__(kLeafThreads, 1) leaf_kernel(LeafParams p) {
    pdl_wait_and_release();
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr LeafSmem SL = leaf_smem_layout(W);
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + SL.fm);
    uint32_t *fmr = reinterpret_cast<uint32_t *>(smem + SL.fmr);
    uint32_t *vf = reinterpret_cast<uint32_t *>(smem + SL.vf);
    uint32_t *vbk = reinterpret_cast<uint32_t *>(smem + SL.vb);
    uint32_t *vr = reinterpret_cast<uint32_t *>(smem + SL.vr);
    int32_t *vmin = reinterpret_cast<int32_t *>(smem + SL.vmin);
    int32_t *wsum = reinterpret_cast<int32_t *>(smem + SL.wsum);
    uint8_t *sa = smem + SL.sa;
    uint8_t *sb = smem + SL.sb;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = blockIdx.x;
    const int64_t r0 = (int64_t)s * p.h;
    const int hs = (int)min((int64_t)p.h, p.m - r0);
    const int64_t i = p.pathI[s], j = p.pathJ[s];

    for (int t = tid; t < 256 * W; t += kLeafThreads) {
        fm[t] = 0u;
        fmr[t] = 0u;
    }
    for (int t = tid; t <= 256; t += kLeafThreads) vmin[t] = INT32_MAX;
    __syncthreads();
    for (int r = tid; r < hs; r += kLeafThreads) {
        const uint8_t ch = p.a[r0 + r];
        sa[r] = ch;
        atomicOr(&fm[ch * W + (r >> 5)], 1u << (r & 31));
        const int rr = hs - 1 - r;               // row r of the reversed strip
        atomicOr(&fmr[ch * W + (rr >> 5)], 1u << (rr & 31));
    }
    const bool valid = !(i < 0 || j < i || j > p.n);
    const int64_t ncol64 = valid ? j - i : 0;
    if (valid && ncol64 <= kLeafSmemCols)
        for (int64_t t = tid; t < ncol64; t += kLeafThreads) sb[t] = p.b[i + t];
    __syncthreads();
    if (!valid) {
        if (tid == 0) {
            set_error(p.err, ERR_BOUNDS);
            p.counts[s] = 0;
        }
        return;
    }
    if (ncol64 > kLeafSmemCols) {
        if (warp == 0) leaf_walk_global<W>(p, s, r0, hs, i, j, fm, sa, lane);
        return;
    }
    const int ncol = (int)ncol64;
    if (warp == 0) leaf_sweep<W>(fm, sb, ncol, false, vf, lane);
    else if (warp == 1) leaf_sweep<W>(fmr, sb, ncol, true, vbk, lane);
    __syncthreads();

    // Backward vectors in forward row order: bit q of vr[c'] is bit
    // hs - 1 - q of vbk[c'] (reverse all 32 W bits, then drop the 32 W - hs
    // padding rows that land at the bottom).  A thread per column.
    {
        const int sft = 32 * W - hs, q0 = sft >> 5, sb5 = sft & 31;
        for (int c = tid; c <= ncol; c += kLeafThreads) {
            // Word k of the reversed vector is brev(vbk word W - 1 - k); word
            // w of the result joins reversed words w + q0 and w + q0 + 1.
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int klo = W - 1 - (w + q0), khi = klo - 1;
                const uint32_t lo = klo >= 0 ? __brev(vbk[c * W + klo]) : 0u;
                const uint32_t hi = khi >= 0 ? __brev(vbk[c * W + khi]) : 0u;
                vr[c * W + w] = sb5 ? ((lo >> sb5) | (hi << (32 - sb5))) : lo;
            }
        }
    }
    __syncthreads();

    // L = F(hs, j).  Vertex (r, c) lies on a heaviest path iff F + B = L,
    // i.e. ones(vf[c - i], bits < r) + ones(vr[j - c], bits r .. hs-1)
    // = hs - L.  A lane per column (32 consecutive columns per warp and
    // group) runs down the rows, the count moving by (forward bit - backward
    // bit) of row r - 1, and collects its hits as bit masks of 32 rows; a
    // warp bit-matrix transpose then gives lane t, for row 32 w + t + 1, the
    // mask of the group's columns with a hit, whose lowest bit is the
    // group's smallest such column.
    uint32_t last[W];
#pragma unroll
    for (int w = 0; w < W; ++w) last[w] = vf[ncol * W + w];
    const int L = hs - prefix_ones<W>(last, hs);
    const int target = hs - L;
    const int nw = kLeafThreads / 32;
    for (int grp = warp; grp * 32 <= ncol; grp += nw) {
        const int c = grp * 32 + lane;
        const bool live = c <= ncol;
        const uint32_t *fc = vf + c * W, *gc = vr + (ncol - c) * W;
        int d = INT32_MIN / 2;                   // dead lanes never hit
        if (live) {
            d = 0;                               // r = 0: all of B's ones
            for (int w = 0; w < W; ++w) {
                const int k = min(max(hs - 32 * w, 0), 32);
                d += __popc(gc[w] & (k == 32 ? 0xFFFFFFFFu : ((1u << k) - 1u)));
            }
        }
        for (int w = 0; w < W && 32 * w < hs; ++w) {
            uint32_t fw = live ? fc[w] : 0u, gw = live ? gc[w] : 0u, hits = 0u;
            // Partly unrolled: fully unrolled rows of every word would not
            // fit the instruction cache.
#pragma unroll 8
            for (int t = 0; t < 32; ++t) {
                d += (int)(fw & 1u) - (int)(gw & 1u);
                fw >>= 1;
                gw >>= 1;
                hits |= (d == target ? 1u : 0u) << t;
            }
            // Rows past hs within the word carry padding bits: drop them.
            const int valid = hs - 32 * w;
            if (valid < 32) hits &= (1u << valid) - 1u;
            // Transpose: afterwards lane t holds bit l = hit of lane l's
            // column in row 32 w + t + 1.
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
                const uint32_t m = sh == 16 ? 0x0000FFFFu : sh == 8 ? 0x00FF00FFu : sh == 4 ? 0x0F0F0F0Fu
                                                            : sh == 2 ? 0x33333333u : 0x55555555u;
                const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, hits, sh);
                hits = (lane & sh) ? ((hits & ~m) | ((y & ~m) >> sh)) : ((hits & m) | ((y & m) << sh));
            }
            if (hits) atomicMin(&vmin[32 * w + lane + 1], grp * 32 + __ffs(hits) - 1);
        }
    }
    __syncthreads();

    // Marks, their ranks (block scan), the cross vertices and the letters.
    const int r = tid + 1;                       // one row per thread (hs <= 256)
    bool mark = false, bad = false;
    int32_t v = 0;
    if (r <= hs) {
        const int32_t cr = vmin[r], cp = r == 1 ? 0 : vmin[r - 1];
        bad = cr == INT32_MAX || cp == INT32_MAX;
        if (!bad) {
            v = (int32_t)i + cr;
            mark = cr > cp && sa[r - 1] == sb[cr - 1];
        }
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, mark);
    if (lane == 0) wsum[warp] = __popc(bal);
    if (__syncthreads_or(bad)) {
        if (tid == 0) {
            set_error(p.err, ERR_BOUNDS);
            p.counts[s] = 0;
        }
        return;
    }
    int before = __popc(bal & ((1u << lane) - 1u)), total = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
    if (r <= hs) {
        if (p.cross) p.cross[r0 + r] = v;
        if (mark) p.slots[(int64_t)s * p.h + before] = sa[r - 1];
    }
    if (tid == 0) {
        if (s == 0 && p.cross) p.cross[0] = (int32_t)i;
        p.counts[s] = total;
        if (total != L) set_error(p.err, ERR_BOUNDS);
    }
}

template <int W>
static cudaError_t launch_leaf_t(const LeafParams &p, cudaStream_t st, int priority) {
    constexpr size_t smem = leaf_smem_layout(W).total;
    auto kern = leaf_kernel<W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl_prio(kern, dim3((unsigned)p.S), dim3(kLeafThreads), smem, st, priority, p);
}

cudaError_t launch_leaf(const LeafParams &p, cudaStream_t st, int priority) {
    if (p.S <= 0) return cudaSuccess;
    switch (p.words) {
        case 1: return launch_leaf_t<1>(p, st, priority);
        case 2: return launch_leaf_t<2>(p, st, priority);
        case 4: return launch_leaf_t<4>(p, st, priority);
        case 8: return launch_leaf_t<8>(p, st, priority);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ compaction
__global__ void __launch_bounds__(1024) compact_kernel(CompactParams p, int32_t *offsets) {
    pdl_wait_and_release();
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Exclusive scan of counts in chunks of 1024.
    for (int base = 0; base < p.S; base += 1024) {
        const int s = base + threadIdx.x;
        const int v = (s < p.S) ? p.counts[s] : 0;
        int x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = warp_sums[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, w, off);
                if (lane >= off) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? warp_sums[warp - 1] : 0);
        if (s < p.S) offsets[s] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    const int64_t total = carry;
    if (threadIdx.x == 0) {
        if (p.len_out) *p.len_out = total;
        if (p.len_out2) *p.len_out2 = total;
        if (p.out && total > p.cap) set_error(p.err, ERR_OVERFLOW);
    }
    if (!p.out || total > p.cap) return;
    for (int s = warp; s < p.S; s += 32) {
        const int cnt = p.counts[s], off = offsets[s];
        for (int t = lane; t < cnt; t += 32) p.out[off + t] = p.slots[(int64_t)s * p.h + t];
    }
}

cudaError_t launch_compact(const CompactParams &p, cudaStream_t st) {
    // offsets live right after the counts array (the planner reserves 2*S ints).
    return launch_pdl(compact_kernel, dim3(1), dim3(1024), 0, st, p, const_cast<int32_t *>(p.counts) + p.S);
}

// ------------------------------------------------------------------ path listing
// The leftmost heaviest path as a vertex list (Sec. II-D: the horizontal
// runs between consecutive cross vertices, placed by a prefix sum).  Row r's
// run starts at its cross vertex v[r] and ends where the path steps down.
// The step into row r+1 lands on v[r+1]; it is a match diagonal exactly
// when v[r+1] > v[r] and a_{r+1} = b_{v[r+1]} (a vertical step at a column
// where the diagonal into it matches would give up one unit of weight, so a
// heaviest path never takes it), and then the run ends at v[r+1] - 1; else
// at v[r+1].  The last row runs to n.  The vertex count is m + n + 1 - L.
__device__ __forceinline__ int64_t path_run(const PathParams &p, int64_t r, bool &bad) {
    const int64_t v0 = p.cross[r];
    if (v0 < 0 || v0 > p.n) {
        bad = true;
        return 1;
    }
    int64_t e = p.n;
    if (r < p.m) {
        const int64_t v1 = p.cross[r + 1];
        if (v1 < v0 || v1 > p.n) {
            bad = true;
            return 1;
        }
        e = (v1 > v0 && p.a[r] == p.b[v1 - 1]) ? v1 - 1 : v1;
    }
    if (v0 > e) {
        bad = true;
        return 1;
    }
    return e - v0 + 1;
}

__global__ void __launch_bounds__(1024) path_kernel(PathParams p) {
    pdl_wait_and_release();
    __shared__ int32_t warp_sums[32];
    __shared__ int64_t carry;
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        carry = 0;
        s_bad = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rows = p.m + 1;
    for (int64_t base = 0; base < rows; base += 1024) {
        const int64_t r = base + threadIdx.x;
        bool bad = false;
        const int32_t v = r < rows ? (int32_t)path_run(p, r, bad) : 0;
        if (bad) s_bad = 1;
        int32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = warp_sums[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int32_t y = __shfl_up_sync(0xFFFFFFFFu, w, off);
                if (lane >= off) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int32_t incl = x + (warp > 0 ? warp_sums[warp - 1] : 0);
        if (r < rows) p.offsets[r] = (int32_t)carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    const int64_t total = carry;
    const int64_t want = p.m + p.n + 1 - *p.len;
    if (threadIdx.x == 0) {
        if (p.count_out) *p.count_out = total;
        if (s_bad || total != want) set_error(p.err, ERR_BOUNDS);
        else if (total > p.cap) set_error(p.err, ERR_OVERFLOW);
    }
    if (s_bad || total != want || total > p.cap) return;
    for (int64_t r = warp; r < rows; r += 32) {
        bool bad = false;
        const int64_t len = path_run(p, r, bad), off = p.offsets[r], v0 = p.cross[r];
        for (int64_t t = lane; t < len; t += 32) {
            p.path[2 * (off + t)] = (int32_t)r;
            p.path[2 * (off + t) + 1] = (int32_t)(v0 + t);
        }
    }
}

cudaError_t launch_path(const PathParams &p, cudaStream_t st) {
    return launch_pdl(path_kernel, dim3(1), dim3(1024), 0, st, p);
}

cudaError_t launch_copy_len(const int64_t *src, int64_t *dst, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

}  // namespace lcsg
