// quad.cu -- the tree's (max,+) merge on DPX instructions, by 32 x 32 quadrants.
//
//     D(i, j) = max_{i <= k <= j} U(i, k) + L(k, j)
//
// (Sec. II-A's split of a heaviest path at the boundary row between the two
// halves; Sec. II-B-1's combination formula in its DIST form.)  Only D is
// produced: the traceback recomputes the maximiser at the one (i, j) of each
// node that the path uses.
//
// The band of a quadrant.  U and L are DIST matrices, hence Monge, and for
// two points a <= c (both coordinates) with maximisers k_a of a and k_c of c,
// k_a > k_c implies that k_a also maximises c and k_c also maximises a (add
// the two Monge inequalities of U and L; the sum can only be an equality).
// Take the quadrant's top-left corner a = (ia, ja) and bottom-right corner
// b = (ia + 32, ja + 32), y = K(b) the smallest maximiser of b, and x the
// largest maximiser of a that is <= y (x >= K(a), since K is monotone).
// For every (i, j) of the quadrant a <= (i, j) <= b, so a maximiser k of
// (i, j) below x can be replaced by x and one above y by y: the band [x, y]
// holds a maximiser of every entry.  Against the band [K(a), K(b)] of the
// smallest maximisers this drops the ties at a, and against a 64 x 64 tile's
// band it drops about two thirds of the (max,+) terms on the tree merges of
// the 4096 and 16384 pairs (measured on the oracle's merges).
//
// Work layout.  Every warp is on its own: it takes quadrants from a launch-
// wide counter, classifies each (corner values from the coarse grid at
// spacing 32, x by a ballot over U(ia, k) + L(k, ja) = D(a) read from L2),
// writes constant quadrants straight away, and streams the others' bands
// through two shared-memory slots of one 32-wide k-chunk each (U rows
// i = ia..ia+31 and L columns j = ja..ja+31, cp.async 8-byte pieces): the
// next chunk -- of this quadrant or the next -- lands while the current one
// is multiplied.  A lane owns 8 x 4 outputs (rows ty + 4a, columns tx + 8b),
// loads 12 operand words per 4 k and issues 64 __viaddmax_s16x2 (max(a + b,
// c) on two int16 lanes, the pair taken along k).  Masked entries (k < i in
// U, k > j in L, k > n) hold -16384; every DIST value is at most 16383, so a
// masked sum stays negative and never wraps.  The quadrant leaves through
// the slot it was computed from: rows of 8-byte stores into the tile-packed
// node, or 16-byte stores into the caller's dense matrix.
//
// There is no spin-wait: cp.async groups complete by themselves.
#include <algorithm>
#include <cstdint>

#include "lcs_common.cuh"
#include "lcs_kernels.h"

namespace lcsg {
namespace {

constexpr int Q = 32;                       // quadrant edge
constexpr int kQuadWarps = 4;               // warps per CTA, each independent
constexpr int kQuadThreads = 32 * kQuadWarps;
constexpr int KC = T;                       // k per staged chunk: one K-tile
constexpr int SP = T + 4;                   // slot row pitch = the stored tile's (68 int16)
constexpr int kHalfBytes = Q * SP * 2;      // 32 stored rows of a tile: 4352 contiguous bytes
constexpr int kSlotElems = 2 * Q * SP;      // U rows then L rows
constexpr int kSlotBytes = kSlotElems * 2;  // 8704
constexpr int kWarpBytes = 2 * kSlotBytes + 16;   // two slots and their two mbarriers
constexpr int16_t kNeg = -16384;

__device__ __forceinline__ int64_t gv(int64_t p, int64_t n) { return min(p << 5, n); }

struct QMeta {
    int job, ia, ja;        // merge of the launch, top-left vertex
    int x, y;               // band of k
};

template <typename TOut>
__global__ void __launch_bounds__(kQuadThreads, 3) quad_dpx_kernel(MergeParams p) {
    pdl_wait_and_release();
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int16_t *slots = reinterpret_cast<int16_t *>(smem + warp * kWarpBytes);
    constexpr int64_t EI16 = Fmt<int16_t>::ELEMS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + warp * kWarpBytes + 2 * kSlotBytes);
    const uint64_t lim = p.wait_ns ? p.wait_ns : kWaitLimitNs;
    if (lane == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phases = 0u, pend = 0u;          // bit t: slot t's barrier parity / a copy in flight
    const int n = (int)p.n;
    const int64_t NT = p.NT, P = p.P;
    const int64_t NQ = (n + Q) / Q;                         // quadrant rows: ceil((n+1) / 32)
    const int64_t per_job = NQ * (NQ + 1) / 2, total = per_job * p.njobs;
    const int tx = lane & 7, ty = lane >> 3;

    // Destination of output row r (0..31) of a quadrant in a tile-packed
    // node: row layout (i-major tiles) or column layout (tiles stored
    // transposed, so a quadrant "row" is a column j).
    auto packed_row = [&](const MergeJob &jb, int ia, int ja, int r) -> TOut * {
        TOut *D = reinterpret_cast<TOut *>(jb.D);
        const int I = ia >> T_SHIFT, J = ja >> T_SHIFT;
        if (jb.d_layout == LAYOUT_COL)
            return D + col_tile(I, J) * Fmt<TOut>::ELEMS + ((ja & (T - 1)) + r) * Fmt<TOut>::P + (ia & (T - 1));
        return D + row_tile(I, J, NT) * Fmt<TOut>::ELEMS + ((ia & (T - 1)) + r) * Fmt<TOut>::P + (ja & (T - 1));
    };
    // Entry (x, y) of the quadrant at (ia, ja) = val(x, y), stored by the
    // whole warp: into the caller's dense matrix (rows of 16-byte stores when
    // all 32 columns exist; the sentinel below the diagonal; nothing past n),
    // or into a tile-packed node (8-byte pieces of int16 rows).
    auto store = [&](const MergeJob &jb, int ia, int ja, auto val) {
        const int rows = min(Q, n + 1 - ia), cols = min(Q, n + 1 - ja);
        if (jb.d_layout == LAYOUT_DENSE) {
            TOut *out = reinterpret_cast<TOut *>(p.dense_out);
            constexpr int E = 16 / (int)sizeof(TOut), PR = Q / E;   // elements per piece, pieces per row
            if (cols == Q) {
                for (int c = lane; c < rows * PR; c += 32) {
                    const int x = c / PR, y0 = (c % PR) * E;
                    uint4 v4;
                    TOut *vp = reinterpret_cast<TOut *>(&v4);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        vp[e] = ia + x > ja + y0 + e ? Sentinel<TOut>::value : (TOut)val(x, y0 + e);
                    *reinterpret_cast<uint4 *>(out + (int64_t)(ia + x) * p.ld + ja + y0) = v4;
                }
            } else {
                for (int c = lane; c < rows * Q; c += 32) {
                    const int x = c >> 5, y = c & 31;
                    if (y < cols)
                        out[(int64_t)(ia + x) * p.ld + ja + y] =
                            ia + x > ja + y ? Sentinel<TOut>::value : (TOut)val(x, y);
                }
            }
        } else if (sizeof(TOut) == 2) {
            const bool col = jb.d_layout == LAYOUT_COL;
            for (int c = lane; c < Q * 8; c += 32) {
                const int r = c >> 3, y0 = (c & 7) * 4;
                uint2 v2;
                TOut *vp = reinterpret_cast<TOut *>(&v2);
#pragma unroll
                for (int e = 0; e < 4; ++e) vp[e] = (TOut)(col ? val(y0 + e, r) : val(r, y0 + e));
                *reinterpret_cast<uint2 *>(packed_row(jb, ia, ja, r) + y0) = v2;
            }
        } else {
            const bool col = jb.d_layout == LAYOUT_COL;
            for (int c = lane; c < Q * Q; c += 32) {
                const int r = c >> 5, y = c & 31;
                packed_row(jb, ia, ja, r)[y] = (TOut)(col ? val(y, r) : val(r, y));
            }
        }
    };
    // The accumulators (the pair's two halves maximised) through the slot.
    auto write_quadrant = [&](const MergeJob &jb, int ia, int ja, uint32_t (&acc)[8][4], int16_t *sl) {
        TOut *st = reinterpret_cast<TOut *>(sl);
        constexpr int SPO = Q + 4;           // staged row pitch: 32 x 36 int32 fill the 4608-byte slot
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int x = ty + 4 * a, y = tx + 8 * b;
                const int v = max((int)(int16_t)(acc[a][b] & 0xFFFFu), (int)(int16_t)(acc[a][b] >> 16));
                st[x * SPO + y] = (TOut)v;
            }
        __syncwarp();
        store(jb, ia, ja, [&](int x, int y) { return (int)st[x * SPO + y]; });
    };

    // Batches of quadrants: p.grab (1..32) consecutive quadrants from the
    // launch's counter, classified a lane each -- corner values from the
    // coarse grid, constant quadrants written at once, then x for four
    // staged quadrants at a time (their scans' loads in flight together) --
    // so that the latency of the loads is paid once per batch.  The staged
    // ones are kept in this warp's part of shared memory.
    QMeta *batch = reinterpret_cast<QMeta *>(smem + kQuadWarps * kWarpBytes) + warp * 32;
    int b_pos = 0, b_len = 0;
    bool drained = false;
    auto classify_batch = [&]() -> bool {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(p.sched, (unsigned)p.grab);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        const int64_t base = g0;
        const int cnt = (int)max((int64_t)0, min((int64_t)p.grab, total - base));
        if (cnt <= 0) return false;
        QMeta m{0, 0, 0, 0, -1};
        int va = 0, cval = 0;
        bool cst = false, live = lane < cnt, y_ok = true;
        if (live) {
            const int64_t g = base + lane;
            m.job = (int)(g / per_job);
            const int64_t t = g - (int64_t)m.job * per_job;
            int64_t lo = 0, hi = NQ - 1;                  // quadrant row: largest r with start(r) <= t
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (mid * NQ - mid * (mid - 1) / 2 <= t) lo = mid; else hi = mid - 1;
            }
            const int I2 = (int)lo, J2 = (int)(lo + (t - (lo * NQ - lo * (lo - 1) / 2)));
            m.ia = I2 * Q;
            m.ja = J2 * Q;
            const MergeJob jb = p.jobs[m.job];
            const int64_t pa = I2, pb = min((int64_t)I2 + 1, P), qa = J2, qb = min((int64_t)J2 + 1, P);
            int y = jb.kgrid[pb * (P + 1) + qb];
            va = jb.vgrid[pa * (P + 1) + qa];
            if (I2 < J2) {
                // D is nonincreasing in i and nondecreasing in j: the
                // quadrant's smallest value is at (ib, ja), its largest at (ia, jb).
                const int vmin = jb.vgrid[pb * (P + 1) + qa], vmax = jb.vgrid[pa * (P + 1) + qb];
                cst = vmin == vmax;
                cval = vmax;
            }
            y_ok = y >= m.ia && y <= (int)gv(qb, n);
            if (!y_ok) set_error(p.err, ERR_BOUNDS);
            m.y = min(y_ok ? y : n, min(m.ja + Q - 1, n));
            m.x = m.ia == m.ja ? m.ia : -1;               // on the diagonal, a's only k is ia
            if (!y_ok) m.x = m.ia;                        // not a DIST merge's corners: every k
        }
        // Constant quadrants, and the dense matrix's lower-left quadrant of
        // each diagonal tile (no quadrant of the enumeration; written with
        // the tile's odd diagonal quadrant), by the whole warp.
        unsigned todo = __ballot_sync(0xffffffffu, live && cst);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const MergeJob jb = p.jobs[__shfl_sync(0xffffffffu, m.job, l)];
            store(jb, __shfl_sync(0xffffffffu, m.ia, l), __shfl_sync(0xffffffffu, m.ja, l),
                  [v = __shfl_sync(0xffffffffu, cval, l)](int, int) { return v; });
        }
        todo = __ballot_sync(0xffffffffu, live && m.ia == m.ja && ((m.ia >> 5) & 1));
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const MergeJob jb = p.jobs[__shfl_sync(0xffffffffu, m.job, l)];
            if (jb.d_layout == LAYOUT_DENSE) {
                const int ia = __shfl_sync(0xffffffffu, m.ia, l);
                store(jb, ia, ia - Q, [](int, int) { return 0; });   // every entry has i > j
            }
        }
        // x: the largest k <= y with U(ia, k) + L(k, ja) = D(a), k <= ja (the
        // entries of a); four quadrants' first 32 candidates per round.
        unsigned need = __ballot_sync(0xffffffffu, live && !cst && m.x < 0);
        while (need) {
            int ls[4], tops[4], vas[4], ias[4], jas[4];
            const int16_t *us[4], *lsp[4];
            int16_t fu[4], fl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ls[q] = -1;
                if (need) {
                    const int l = __ffs(need) - 1;
                    need &= need - 1;
                    ls[q] = l;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fu[q] = fl[q] = 0;
                if (ls[q] < 0) continue;                  // warp-uniform
                const int l = ls[q];
                const MergeJob jb = p.jobs[__shfl_sync(0xffffffffu, m.job, l)];
                ias[q] = __shfl_sync(0xffffffffu, m.ia, l);
                jas[q] = __shfl_sync(0xffffffffu, m.ja, l);
                tops[q] = min(__shfl_sync(0xffffffffu, m.y, l), jas[q]);
                vas[q] = __shfl_sync(0xffffffffu, va, l);
                us[q] = reinterpret_cast<const int16_t *>(jb.U);
                lsp[q] = reinterpret_cast<const int16_t *>(jb.L);
                const int k = tops[q] - lane;
                if (k >= ias[q]) {
                    fu[q] = us[q][row_elem<int16_t>(ias[q], k, NT)];
                    fl[q] = lsp[q][col_elem<int16_t>(k, jas[q])];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (ls[q] < 0) continue;
                const int k = tops[q] - lane;
                unsigned bal = __ballot_sync(0xffffffffu, k >= ias[q] && (int)fu[q] + (int)fl[q] == vas[q]);
                int x = bal ? tops[q] - (__ffs(bal) - 1) : -1;
                // Rarely the maximiser lies further down: 32 more at a time.
                for (int top = tops[q] - 32; x < 0 && top >= ias[q]; top -= 32) {
                    const int kk = top - lane;
                    bool hit = false;
                    if (kk >= ias[q])
                        hit = (int)us[q][row_elem<int16_t>(ias[q], kk, NT)] +
                                  (int)lsp[q][col_elem<int16_t>(kk, jas[q])] == vas[q];
                    bal = __ballot_sync(0xffffffffu, hit);
                    if (bal) x = top - (__ffs(bal) - 1);
                }
                if (x < 0) {                              // not a DIST's (invalid input): every k
                    if (lane == 0) set_error(p.err, ERR_BOUNDS);
                    x = ias[q];
                }
                if (lane == ls[q]) m.x = x;
            }
        }
        // Keep the staged quadrants, in order.
        const bool keep = live && !cst;
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        if (keep) batch[__popc(kb & ((1u << lane) - 1u))] = m;
        __syncwarp();
        b_pos = 0;
        b_len = __popc(kb);
        return true;
    };
    // The next staged quadrant of this warp (false: the launch is done).
    auto next_quadrant = [&](QMeta &m) -> bool {
        while (b_pos >= b_len) {
            if (drained || !classify_batch()) {
                drained = true;
                return false;
            }
        }
        m = batch[b_pos++];
        return true;
    };

    // Stage K-tile kt of quadrant m in slot sl: U's rows ia..ia+31 and L's
    // columns ja..ja+31 of that K-tile are 32 consecutive stored rows each, so
    // one TMA bulk copy apiece, completing on the slot's mbarrier.
    auto issue = [&](const QMeta &m, int kt, int sl) {
        if (lane == 0) {
            const MergeJob jb = p.jobs[m.job];
            const int16_t *U = reinterpret_cast<const int16_t *>(jb.U);
            const int16_t *L = reinterpret_cast<const int16_t *>(jb.L);
            int16_t *dst = slots + sl * kSlotElems;
            fence_proxy_async_smem();            // the slot's last generic writes come first
            mbar_arrive_expect_tx(bars + sl, 2u * kHalfBytes);
            bulk_g2s(dst, U + row_tile(m.ia >> T_SHIFT, kt, NT) * EI16 + (m.ia & (T - 1)) * SP, kHalfBytes, bars + sl);
            bulk_g2s(dst + Q * SP, L + col_tile(kt, m.ja >> T_SHIFT) * EI16 + (m.ja & (T - 1)) * SP, kHalfBytes,
                     bars + sl);
        }
        pend |= 1u << sl;
    };
    // Wait (bounded) for slot sl; on a timeout, flag it, give both slots'
    // copies a second bounded wait so nothing lands after the warp leaves,
    // and report false.
    auto wait_slot = [&](int sl) -> bool {
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(bars + sl, (phases >> sl) & 1u, lim) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                set_error(p.err, ERR_TIMEOUT);
                for (int t = 0; t < 2; ++t)
                    if ((pend >> t) & 1u) mbar_wait_bounded(bars + t, (phases >> t) & 1u, lim);
            }
            __syncwarp();
            return false;
        }
        // The phase has completed: every lane's own wait returns at once and
        // makes the copied bytes visible to it.
        if (lane != 0) mbar_wait_bounded(bars + sl, (phases >> sl) & 1u, lim);
        phases ^= 1u << sl;
        pend &= ~(1u << sl);
        return true;
    };

    // --- first staged quadrant
    QMeta cur, nxt;
    int cur_k0 = 0;
    {
        if (!next_quadrant(cur)) return;
        cur_k0 = cur.x & ~(KC - 1);
        issue(cur, cur_k0 >> T_SHIFT, 0);
    }
    int s = 0;
    uint32_t acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0xC000C000u;

    for (;;) {
        int16_t *sl = slots + s * kSlotElems;
        // The task after this one: the next chunk of this quadrant, or the
        // first chunk of the next staged quadrant (constant ones are written
        // as they are met).
        bool more = true;
        QMeta tm = cur;
        int t_k0 = cur_k0 + KC;
        if (t_k0 > cur.y) {
            if (!next_quadrant(nxt)) {
                more = false;
            } else {
                tm = nxt;
                t_k0 = nxt.x & ~(KC - 1);
            }
        }
        if (more) issue(tm, t_k0 >> T_SHIFT, s ^ 1);
        if (!wait_slot(s)) return;

        // Mask k < i (U), k > j (L) and k > n (both) where the chunk reaches
        // them (stored tiles hold unspecified values there).
        const int kmax = cur_k0 + KC - 1;
        if (cur_k0 <= cur.ia + Q - 1 || kmax > cur.ja || kmax > n) {
            const int i = cur.ia + lane, j = cur.ja + lane;
            int16_t *ur = sl + lane * SP, *lr = sl + (Q + lane) * SP;
            for (int kk = 0; kk < KC; kk += 4) {
                uint2 uu = *reinterpret_cast<uint2 *>(ur + kk), ll = *reinterpret_cast<uint2 *>(lr + kk);
                int16_t *up = reinterpret_cast<int16_t *>(&uu), *lp = reinterpret_cast<int16_t *>(&ll);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = cur_k0 + kk + e;
                    if (k < i || k > n) up[e] = kNeg;
                    if (k > j || k > n) lp[e] = kNeg;
                }
                *reinterpret_cast<uint2 *>(ur + kk) = uu;
                *reinterpret_cast<uint2 *>(lr + kk) = ll;
            }
            __syncwarp();
        }
        // (max,+) over this chunk's part of the band, 4 k per step.
        const int lo = (max(cur.x, cur_k0) - cur_k0) & ~3;
        const int hi = (min(cur.y, kmax) - cur_k0) | 3;
        {
            const int16_t *Ub = sl + ty * SP;
            const int16_t *Lb = sl + (Q + tx) * SP;
            uint2 u[8], lv[4];
#pragma unroll
            for (int a = 0; a < 8; ++a) u[a] = *reinterpret_cast<const uint2 *>(Ub + a * 4 * SP + lo);
#pragma unroll
            for (int b = 0; b < 4; ++b) lv[b] = *reinterpret_cast<const uint2 *>(Lb + b * 8 * SP + lo);
            for (int kk = lo; kk <= hi; kk += 4) {
                const int kn = kk + 4 <= hi ? kk + 4 : kk;
                uint2 un[8], ln[4];
#pragma unroll
                for (int a = 0; a < 8; ++a) un[a] = *reinterpret_cast<const uint2 *>(Ub + a * 4 * SP + kn);
#pragma unroll
                for (int b = 0; b < 4; ++b) ln[b] = *reinterpret_cast<const uint2 *>(Lb + b * 8 * SP + kn);
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
        if (cur_k0 + KC > cur.y) {
            // Last chunk of the quadrant: results through this slot.
            __syncwarp();
            write_quadrant(p.jobs[cur.job], cur.ia, cur.ja, acc, sl);
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0xC000C000u;
        }
        __syncwarp();
        if (!more) break;
        cur = tm;
        cur_k0 = t_k0;
        s ^= 1;
    }
}

}  // namespace

cudaError_t launch_quad_dpx(MergeParams p, int out_dtype, cudaStream_t st) {
    if (!p.sched || p.gshift != 5) return cudaErrorInvalidValue;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e;
        const size_t smem = (size_t)kQuadWarps * (kWarpBytes + 32 * sizeof(QMeta));
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQuadThreads, smem)) != cudaSuccess)
            return e;
        const int64_t NQ = (p.n + Q) / Q;
        const int64_t work = p.njobs * NQ * (NQ + 1) / 2;
        const int64_t warps = std::max<int64_t>(1, (int64_t)sms * std::max(per_sm, 1) * kQuadWarps);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, kQuadWarps),
                                                                    (int64_t)sms * std::max(per_sm, 1)));
        // Quadrants per batch: a quarter of a warp's share (at most 32, a
        // lane each), so that batches amortise the classification's load
        // latency and still leave the tail short.
        const int64_t per_warp = work / warps;
        p.grab = (int32_t)std::max<int64_t>(1, std::min<int64_t>(32, per_warp / 4));
        return launch_pdl(kern, dim3((unsigned)grid), dim3(kQuadThreads), smem, st, p);
    };
    switch (out_dtype) {
        case DT_I16: return go(quad_dpx_kernel<int16_t>);
        case DT_I32: return go(quad_dpx_kernel<int32_t>);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lcsg
