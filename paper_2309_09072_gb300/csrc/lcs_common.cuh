// lcs_common.cuh -- layout, types and PTX helpers shared by the GB300 kernels.
//
// Internal DIST storage ("tile-packed").  A DIST matrix over vertices 0..n is
// cut into T x T tiles (T = 64); only tiles (I, J) with I <= J exist.  Each
// stored tile has a row pitch of T + 4/sizeof(element) elements: 4 bytes of
// padding per row make rows that are 2 apart fall into different shared-
// memory banks once a tile is copied byte for byte into shared memory.  A node
// that the merge above it reads by ROWS (the upper operand U) is stored in
// row layout: tiles ordered by I then J, each tile row-major (i-major).  A
// node read by COLUMNS (the lower operand L) is stored in column layout:
// tiles ordered by J then I, each tile j-major (the tile is stored
// transposed).  In both layouts the band of tiles a merge tile needs --
// U(i in tile I, k in K-tiles) or L(k in K-tiles, j in tile J) -- is one
// contiguous run of whole tiles, so it is staged into shared memory with one
// TMA bulk copy per tile, and every scan over k reads consecutive addresses.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace lcsg {

constexpr int T = 64;          // tile edge in vertices
constexpr int T_SHIFT = 6;
constexpr int T2 = T * T;

enum DType : int { DT_I32 = 0, DT_I16 = 1, DT_U8 = 2 };
enum Layout : int { LAYOUT_ROW = 0, LAYOUT_COL = 1, LAYOUT_DENSE = 2 };

// Device error word bits (read back by lcs_sync).
enum ErrBits : int { ERR_TIMEOUT = 1, ERR_OVERFLOW = 2, ERR_BOUNDS = 4 };

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t num_tiles_side(int64_t n) { return ceil_div(n + 1, T); }
__host__ __device__ inline int64_t num_tiles_tri(int64_t NT) { return NT * (NT + 1) / 2; }
// Row layout: tile (I, J >= I) -> I*NT - I*(I-1)/2 + (J - I).
__host__ __device__ inline int64_t row_tile(int64_t I, int64_t J, int64_t NT) {
    return I * NT - I * (I - 1) / 2 + (J - I);
}
// Column layout: tile (I <= J, J) -> J*(J+1)/2 + I.
__host__ __device__ inline int64_t col_tile(int64_t I, int64_t J) { return J * (J + 1) / 2 + I; }

__host__ __device__ inline int dt_bytes(int dt) { return dt == 2 ? 1 : (dt == 1 ? 2 : 4); }
// Stored tile: T rows of pitch T + 4 elements (int8/int16) or T + 1 (int32):
// a few bytes per row so that rows fall into different shared-memory banks,
// and, for int16, rows that start on 8-byte boundaries (64-bit loads).
__host__ __device__ inline int tile_pitch(int dt) { return dt == 0 ? T + 1 : T + 4; }
__host__ __device__ inline int64_t tile_elems(int dt) { return (int64_t)T * tile_pitch(dt); }
template <typename V> struct Fmt {
    static constexpr int P = sizeof(V) == 4 ? T + 1 : T + 4;
    static constexpr int ELEMS = T * P;
};

// Element (i, k) of a row-layout matrix, k >= i.
template <typename V>
__device__ __forceinline__ int64_t row_elem(int64_t i, int64_t k, int64_t NT) {
    return row_tile(i >> T_SHIFT, k >> T_SHIFT, NT) * Fmt<V>::ELEMS + (i & (T - 1)) * Fmt<V>::P + (k & (T - 1));
}
// Element (k, j) of a column-layout matrix, k <= j.
template <typename V>
__device__ __forceinline__ int64_t col_elem(int64_t k, int64_t j) {
    return col_tile(k >> T_SHIFT, j >> T_SHIFT) * Fmt<V>::ELEMS + (j & (T - 1)) * Fmt<V>::P + (k & (T - 1));
}

template <typename V> struct Sentinel;
template <> struct Sentinel<int32_t> { static constexpr int32_t value = INT32_MIN; };
template <> struct Sentinel<int16_t> { static constexpr int16_t value = INT16_MIN; };
template <> struct Sentinel<uint8_t> { static constexpr uint8_t value = 0xFF; };

template <typename V> struct MaxVal;
template <> struct MaxVal<int32_t> { static constexpr int value = INT32_MAX; };
template <> struct MaxVal<int16_t> { static constexpr int value = INT16_MAX; };
template <> struct MaxVal<uint8_t> { static constexpr int value = 255; };

// U(i, k) of a row-layout matrix / L(k, j) of a column-layout matrix whose
// element type is known only at run time.
__device__ __forceinline__ int load_row_any(const void *p, int64_t i, int64_t k, int64_t NT, int dt) {
    if (dt == DT_U8) return ((const uint8_t *)p)[row_elem<uint8_t>(i, k, NT)];
    if (dt == DT_I16) return ((const int16_t *)p)[row_elem<int16_t>(i, k, NT)];
    return ((const int32_t *)p)[row_elem<int32_t>(i, k, NT)];
}
__device__ __forceinline__ int load_col_any(const void *p, int64_t k, int64_t j, int dt) {
    if (dt == DT_U8) return ((const uint8_t *)p)[col_elem<uint8_t>(k, j)];
    if (dt == DT_I16) return ((const int16_t *)p)[col_elem<int16_t>(k, j)];
    return ((const int32_t *)p)[col_elem<int32_t>(k, j)];
}

__device__ __forceinline__ void set_error(int *err, int bits) {
    if (err) atomicOr(err, bits);
}

// ---------------------------------------------------------------- PTX: mbarrier + TMA bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One TMA bulk copy global -> shared, completing `bytes` transactions on bar.
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Programmatic dependent launch.  A kernel of the solve chain begins with
// pdl_wait_and_release(): it waits until the kernel before it in the stream
// has completed and its writes are visible (griddepcontrol.wait), then lets
// the next kernel be scheduled (griddepcontrol.launch_dependents).  Launched
// with launch_pdl, the next kernel's CTAs are placed while this one runs and
// block in their own wait, which hides the launch gap between the two.
// Without the launch attribute (or after a copy or an event) both
// instructions do nothing and the stream orders the kernels as usual.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// launch_pdl with a scheduling priority for the launch (0: the stream's):
// pending CTAs of a higher-priority launch are placed first as SMs free up.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_prio(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   int priority, Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = priority ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Barrier among `count` threads (a multiple of 32) of the CTA on hardware
// barrier `id` (1..15; 0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~max_ns of global time
// and returns false (the caller records ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint64_t max_ns) {
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > max_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

// TMA bulk copy shared -> global (one bulk group); the caller fences the
// generic-proxy writes first and waits for the reads before reusing smem.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ------------------------------------------------------------------ bit-vector step
// s = x + y over W words; returns the carry out of the top word.
template <int W> struct AddChain;
template <> struct AddChain<1> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[1], const uint32_t (&x)[1],
                                                   const uint32_t (&y)[1]) {
        uint32_t c;
        asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, 0, 0;" : "=r"(s[0]), "=r"(c) : "r"(x[0]), "r"(y[0]));
        return c;
    }
};
template <> struct AddChain<2> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[2], const uint32_t (&x)[2],
                                                   const uint32_t (&y)[2]) {
        uint32_t c;
        asm("add.cc.u32 %0, %3, %5;\n\t"
            "addc.cc.u32 %1, %4, %6;\n\t"
            "addc.u32 %2, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(y[0]), "r"(y[1]));
        return c;
    }
};
template <> struct AddChain<4> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[4], const uint32_t (&x)[4],
                                                   const uint32_t (&y)[4]) {
        uint32_t c;
        asm("add.cc.u32 %0, %5, %9;\n\t"
            "addc.cc.u32 %1, %6, %10;\n\t"
            "addc.cc.u32 %2, %7, %11;\n\t"
            "addc.cc.u32 %3, %8, %12;\n\t"
            "addc.u32 %4, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]));
        return c;
    }
};
template <> struct AddChain<8> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[8], const uint32_t (&x)[8],
                                                   const uint32_t (&y)[8]) {
        uint32_t c;
        asm("add.cc.u32 %0, %9, %17;\n\t"
            "addc.cc.u32 %1, %10, %18;\n\t"
            "addc.cc.u32 %2, %11, %19;\n\t"
            "addc.cc.u32 %3, %12, %20;\n\t"
            "addc.cc.u32 %4, %13, %21;\n\t"
            "addc.cc.u32 %5, %14, %22;\n\t"
            "addc.cc.u32 %6, %15, %23;\n\t"
            "addc.cc.u32 %7, %16, %24;\n\t"
            "addc.u32 %8, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]),
              "=r"(s[7]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]),
              "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]));
        return c;
    }
};

template <> struct AddChain<3> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[3], const uint32_t (&x)[3],
                                                   const uint32_t (&y)[3]) {
        uint32_t c;
        asm("add.cc.u32 %0, %4, %7;\n\t"
            "addc.cc.u32 %1, %5, %8;\n\t"
            "addc.cc.u32 %2, %6, %9;\n\t"
            "addc.u32 %3, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(y[0]), "r"(y[1]), "r"(y[2]));
        return c;
    }
};
template <> struct AddChain<5> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[5], const uint32_t (&x)[5],
                                                   const uint32_t (&y)[5]) {
        uint32_t c;
        asm("add.cc.u32 %0, %6, %11;\n\t"
            "addc.cc.u32 %1, %7, %12;\n\t"
            "addc.cc.u32 %2, %8, %13;\n\t"
            "addc.cc.u32 %3, %9, %14;\n\t"
            "addc.cc.u32 %4, %10, %15;\n\t"
            "addc.u32 %5, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]));
        return c;
    }
};
template <> struct AddChain<6> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[6], const uint32_t (&x)[6],
                                                   const uint32_t (&y)[6]) {
        uint32_t c;
        asm("add.cc.u32 %0, %7, %13;\n\t"
            "addc.cc.u32 %1, %8, %14;\n\t"
            "addc.cc.u32 %2, %9, %15;\n\t"
            "addc.cc.u32 %3, %10, %16;\n\t"
            "addc.cc.u32 %4, %11, %17;\n\t"
            "addc.cc.u32 %5, %12, %18;\n\t"
            "addc.u32 %6, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]));
        return c;
    }
};
template <> struct AddChain<7> {
    static __device__ __forceinline__ uint32_t run(uint32_t (&s)[7], const uint32_t (&x)[7],
                                                   const uint32_t (&y)[7]) {
        uint32_t c;
        asm("add.cc.u32 %0, %8, %15;\n\t"
            "addc.cc.u32 %1, %9, %16;\n\t"
            "addc.cc.u32 %2, %10, %17;\n\t"
            "addc.cc.u32 %3, %11, %18;\n\t"
            "addc.cc.u32 %4, %12, %19;\n\t"
            "addc.cc.u32 %5, %13, %20;\n\t"
            "addc.cc.u32 %6, %14, %21;\n\t"
            "addc.u32 %7, 0, 0;"
            : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(c)
            : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]));
        return c;
    }
};

// One bit-vector column step (u = V & M, V' = (V + u) | (V & ~M), the
// Allison-Dix / Hyyro step restated) for one source; returns the carry out
// of the top row, the increment of DIST.
template <int W>
__device__ __forceinline__ uint32_t column_step(uint32_t (&V)[W], const uint32_t (&M)[W]) {
    uint32_t u[W], s[W];
#pragma unroll
    for (int w = 0; w < W; ++w) u[w] = V[w] & M[w];
    uint32_t c = AddChain<W>::run(s, V, u);
#pragma unroll
    for (int w = 0; w < W; ++w) V[w] = s[w] | (V[w] & ~M[w]);
    return c;
}

// The same step over words [S, W) only, for a vector whose words below S are
// zero: a zero word gives no carry and stays zero (u = 0, V + 0 = 0), so the
// chain starts at word S with no carry in.  The carry out is the same.
template <int W, int S>
__device__ __forceinline__ uint32_t column_step_tail(uint32_t (&V)[W], const uint32_t (&M)[W]) {
    constexpr int N = W - S;
    if constexpr (N <= 0) {
        return 0u;
    } else {
        uint32_t x[N], u[N], s[N];
#pragma unroll
        for (int w = 0; w < N; ++w) {
            x[w] = V[S + w];
            u[w] = x[w] & M[S + w];
        }
        const uint32_t c = AddChain<N>::run(s, x, u);
#pragma unroll
        for (int w = 0; w < N; ++w) V[S + w] = s[w] | (x[w] & ~M[S + w]);
        return c;
    }
}

// Calls f(std::integral_constant<int, w0>{}) for a run-time w0 in [0, W].
template <int W, int K = 0, typename F>
__device__ __forceinline__ void dispatch_start(int w0, F &&f) {
    if constexpr (K <= W) {
        if (w0 == K) {
            f(std::integral_constant<int, K>{});
            return;
        }
        dispatch_start<W, K + 1>(w0, f);
    }
}

// ------------------------------------------------------------------ multi-word adds with carry in
// s = x + y + cin (cin 0 or 1) over 4 words as one add-with-carry chain;
// returns the carry out of the top word.  The carry in enters the chain
// through the carry flag: cin + 0xFFFFFFFF carries exactly when cin = 1.
__device__ __forceinline__ uint32_t add4_cin(uint32_t *s, const uint32_t *x, const uint32_t *y, uint32_t cin) {
    uint32_t c;
    asm("{\n\t.reg .u32 ci;\n\t"
        "add.cc.u32 ci, %13, -1;\n\t"
        "addc.cc.u32 %0, %5, %9;\n\t"
        "addc.cc.u32 %1, %6, %10;\n\t"
        "addc.cc.u32 %2, %7, %11;\n\t"
        "addc.cc.u32 %3, %8, %12;\n\t"
        "addc.u32 %4, 0, 0;\n\t}"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c)
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(cin));
    return c;
}
__device__ __forceinline__ uint32_t add2_cin(uint32_t *s, const uint32_t *x, const uint32_t *y, uint32_t cin) {
    uint32_t c;
    asm("{\n\t.reg .u32 ci;\n\t"
        "add.cc.u32 ci, %7, -1;\n\t"
        "addc.cc.u32 %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, 0, 0;\n\t}"
        : "=r"(s[0]), "=r"(s[1]), "=r"(c)
        : "r"(x[0]), "r"(x[1]), "r"(y[0]), "r"(y[1]), "r"(cin));
    return c;
}
// s = x + y + cin over N words (N = 2 or a multiple of 4), blocks of four
// chained through their carries; returns the carry out.
template <int N>
__device__ __forceinline__ uint32_t addn_cin(uint32_t (&s)[N], const uint32_t (&x)[N], const uint32_t (&y)[N],
                                             uint32_t cin) {
    static_assert(N == 2 || N % 4 == 0, "words per lane: 2 or a multiple of 4");
    if constexpr (N == 2) {
        return add2_cin(s, x, y, cin);
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 4) cin = add4_cin(s + k, x + k, y + k, cin);
        return cin;
    }
}

}  // namespace lcsg
