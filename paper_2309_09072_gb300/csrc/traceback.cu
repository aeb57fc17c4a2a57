// traceback.cu -- one LCS from the merge tree (Sec. II-C..II-E).
//
// The cross vertex v[r] of row r is the leftmost vertex of the heaviest path
// in that row (Sec. II-C).  At a tree node covering rows [r0, r1) whose path
// runs from top vertex i = v[r0] to bottom vertex j, the cross vertex on the
// boundary row s between its halves is the smallest maximiser
//     c = min argmax_{i <= k <= j} U(i, k) + L(k, j)
// (Sec. II-D: it is a by-product of the merge), and the two halves get the
// sub-paths (i, c) and (c, j).  tb_level_kernel resolves one tree level per
// launch, top down.  Inside a strip (leaf) the rows are resolved directly
// from the forward bit vectors of F(r, c) = LCS(a_strip[0:r], b[i:c]) by a
// backward walk that keeps every row's segment as far left as it can go (see
// leaf_kernel); letter a_r is marked when the path enters row r by a weight-1
// diagonal (Sec. II-E).  The marked letters of all strips, in row order, are
// the LCS.
#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {

// ------------------------------------------------------------------ per-level argmax
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
    int best = INT32_MIN;
    int64_t bk = INT64_MAX;
    for (int64_t k = i + threadIdx.x; k <= j; k += blockDim.x) {
        const int v = load_row_any(mg.U, i, k, p.NT, mg.in_dtype) + load_col_any(mg.L, k, j, mg.in_dtype);
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
        p.pathI[mg.upper] = (int32_t)i;
        p.pathJ[mg.upper] = c;
        p.pathI[mg.lower] = c;
        p.pathJ[mg.lower] = (int32_t)j;
        if (mg.node == p.root_node && p.len_out) *p.len_out = best;
    }
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
constexpr int kLeafWarps = 2;
constexpr int kLeafSmemCols = 1024;   // forward bit-vectors kept in shared memory

// Shared memory of one leaf warp: match masks, column vectors, the strip's
// letters and b's segment.
__host__ __device__ constexpr size_t leaf_warp_bytes(int W) {
    return ((size_t)(256 * W + kLeafSmemCols * W) * 4 + (size_t)kLeafSmemCols * (W + 1) * 2 + 256 +
            kLeafSmemCols + 15) / 16 * 16;
}

// F(r, c) of a strip = zeros among the first r bits of its column vector V_c
// (a zero bit marks a row where the DP steps up).
template <int W>
__device__ __forceinline__ int f_at(const uint32_t *v, int r) {
    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int bits = min(max(r - 32 * w, 0), 32);          // of word w, the first `bits` rows
        const uint32_t mask = bits == 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
        ones += __popc(v[w] & mask);
    }
    return r - ones;
}

// Forward sweep and backward walk of one strip whose path runs from (0, i)
// to (hs, j): column vectors in vb and b's segment in sb (shared memory,
// kSmem) or vb in the global scratch and b read from global memory.
template <int W, bool kSmem>
__device__ __forceinline__ void leaf_path(const LeafParams &p, int s, int64_t r0, int hs, int64_t i, int64_t j,
                                          const uint32_t *fm, uint32_t *vb, uint16_t *pp, const uint8_t *sa,
                                          const uint8_t *sb, int lane) {
    auto bch = [&](int64_t c) -> uint8_t {
        if constexpr (kSmem) return sb[c - 1 - i];
        else return p.b[c - 1];
    };
    // Forward sweep (every lane computes V; lane w stores word w).
    // With the column vectors in shared memory, lane w <= W also stores the
    // ones in the words below w, so that the walk's F(r, c) is one table
    // entry plus one masked popcount.
    uint32_t V[W];
#pragma unroll
    for (int w = 0; w < W; ++w) V[w] = 0xFFFFFFFFu;
    if (lane < W) vb[lane] = 0xFFFFFFFFu;
    if (kSmem && lane <= W) pp[lane] = (uint16_t)(32 * lane);
    for (int64_t c = i + 1; c <= j; ++c) {
        const uint32_t *M = fm + bch(c) * W;
        uint32_t u[W], sm[W];
#pragma unroll
        for (int w = 0; w < W; ++w) u[w] = V[w] & M[w];
        uint32_t carry = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t t = (uint64_t)V[w] + (uint64_t)u[w] + carry;
            sm[w] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        uint32_t mine = 0;                       // word `lane` of V, picked without branches
        int below = 0;                           // ones in the words below `lane`
#pragma unroll
        for (int w = 0; w < W; ++w) {
            V[w] = sm[w] | (V[w] & ~M[w]);
            mine = lane == w ? V[w] : mine;
            below += w < lane ? __popc(V[w]) : 0;
        }
        if (lane < W) vb[(c - i) * W + lane] = mine;
        if (kSmem && lane <= W) pp[(c - i) * (W + 1) + lane] = (uint16_t)below;
    }
    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) ones += __popc(V[w]);
    const int Ltot = 32 * W - ones;              // padding bits stay 1
    __syncwarp();
    if (lane != 0) return;

    // Backward walk (one lane).  F(r, c) = r minus the ones among the first
    // r bits of V_c.
    auto F = [&](int64_t c, int r) -> int {
        const uint32_t *v = vb + (c - i) * W;
        if constexpr (kSmem) {
            const int w = r >> 5, bits = r & 31;
            int ones = pp[(c - i) * (W + 1) + w];
            if (bits) ones += __popc(v[w] & ((1u << bits) - 1u));
            return r - ones;
        } else {
            uint32_t vv[W];
#pragma unroll
            for (int w = 0; w < W; ++w) vv[w] = v[w];
            return f_at<W>(vv, r);
        }
    };
    int r = hs;
    int64_t c = j;
    int pos = Ltot;
    int fc = F(c, r);
    while (r > 0) {
        if (c > i) {
            if (F(c - 1, r) == fc) {              // left along row r
                --c;
                continue;
            }
            if (sa[r - 1] == bch(c) && F(c - 1, r - 1) == fc - 1) {   // diagonal into row r
                if (p.cross) p.cross[r0 + r] = (int32_t)c;
                --pos;
                if (pos >= 0) p.slots[(int64_t)s * p.h + pos] = sa[r - 1];
                --r;
                --c;
                --fc;
                continue;
            }
        }
        if (p.cross) p.cross[r0 + r] = (int32_t)c;   // up: row r is entered at c
        --r;
        fc = F(c, r);
    }
    // Row 0 of the strip is entered at its source i (the path may run along
    // that row before stepping down, so the walk may stop right of i).
    if (s == 0 && p.cross) p.cross[0] = (int32_t)i;
    p.counts[s] = Ltot;
    if (pos != 0) set_error(p.err, ERR_BOUNDS);
}

// One warp per strip.  A forward bit-vector sweep from the strip's source i
// stores V_c, c = i..j.  Then one lane walks back from the strip's sink
// (h, j): left while F keeps its value (the heaviest path may run along the
// row), else along the match diagonal if it is tight, else up.  Moving left
// first keeps every row's segment as far left as it can go, so the row a
// step leaves is left at its cross vertex v[r] = min{c : F(r,c)+B(r,c) =
// DIST_strip(i, j)}: the leftmost heaviest path (Sec. II-C); a diagonal step
// into row r marks letter a_r (Sec. II-E).
template <int W>
__global__ void __launch_bounds__(kLeafWarps * 32) leaf_kernel(LeafParams p) {
    pdl_wait_and_release();
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *fm = reinterpret_cast<uint32_t *>(smem + warp * leaf_warp_bytes(W));   // [256][W] match masks
    uint32_t *vs = fm + 256 * W;                                                  // [kLeafSmemCols][W]
    uint16_t *pp = reinterpret_cast<uint16_t *>(vs + kLeafSmemCols * W);          // [kLeafSmemCols][W + 1]
    uint8_t *sa = reinterpret_cast<uint8_t *>(pp + kLeafSmemCols * (W + 1));      // the strip's letters
    uint8_t *sb = sa + 256;                                                       // b[i .. j - 1]
    const int s = blockIdx.x * kLeafWarps + warp;
    if (s >= p.S) return;
    const int64_t r0 = (int64_t)s * p.h;
    const int hs = (int)min((int64_t)p.h, p.m - r0);
    const int64_t i = p.pathI[s], j = p.pathJ[s];

    for (int t = lane; t < 256 * W; t += 32) fm[t] = 0u;
    __syncwarp();
    for (int r = lane; r < hs; r += 32) {
        const uint8_t ch = p.a[r0 + r];
        sa[r] = ch;
        atomicOr(&fm[ch * W + (r >> 5)], 1u << (r & 31));
    }
    __syncwarp();
    if (i < 0 || j < i || j > p.n) {
        if (lane == 0) { set_error(p.err, ERR_BOUNDS); p.counts[s] = 0; }
        return;
    }
    const int64_t ncol = j - i + 1;
    if (ncol <= kLeafSmemCols) {
        // The letters the serial sweep and walk compare, and the column
        // vectors, live in shared memory; a global access per step would
        // dominate the walk.
        for (int64_t t = lane; t < ncol - 1; t += 32) sb[t] = p.b[i + t];
        __syncwarp();
        leaf_path<W, true>(p, s, r0, hs, i, j, fm, vs, pp, sa, sb, lane);
    } else {
        leaf_path<W, false>(p, s, r0, hs, i, j, fm, p.vbuf + (i + s) * (int64_t)W, nullptr, sa, nullptr, lane);
    }
}

template <int W>
static cudaError_t launch_leaf_t(const LeafParams &p, cudaStream_t st) {
    const size_t smem = (size_t)kLeafWarps * leaf_warp_bytes(W);
    auto kern = leaf_kernel<W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, dim3((unsigned)ceil_div(p.S, kLeafWarps)), dim3(kLeafWarps * 32), smem, st, p);
}

cudaError_t launch_leaf(const LeafParams &p, cudaStream_t st) {
    if (p.S <= 0) return cudaSuccess;
    switch (p.words) {
        case 1: return launch_leaf_t<1>(p, st);
        case 2: return launch_leaf_t<2>(p, st);
        case 4: return launch_leaf_t<4>(p, st);
        case 8: return launch_leaf_t<8>(p, st);
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
