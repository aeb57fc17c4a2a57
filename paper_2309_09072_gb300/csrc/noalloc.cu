// noalloc.cu -- lcs_merge_static: the (max,+) merge of lcs_merge for callers
// that cannot allocate device memory.
//
// lcs_merge keeps its scratch (both operands re-laid out as tile-packed
// matrices, the coarse argmax grid, a job descriptor, an error word) in a
// workspace that the context allocates with cudaMalloc.  Some callers may
// not call cudaMalloc at all: code that runs inside a framework which owns
// every byte of device memory through its own pool, or a latency-critical
// loop where an allocation would synchronise the device.  This entry point
// gives them the same merge with every scratch byte taken from one
// file-scope device array, so the call itself allocates nothing; the caller
// still passes the inputs and outputs.
//
// The array is static device memory: every GPU that loads the library holds
// kStaticScratchBytes of it until the process exits.  In host code its name
// is only a host-side stand-in, so each call looks the device address up with
// cudaGetSymbolAddress, with the call's device current.  The lookup is cheap
// next to the synchronous merge, and it stays right when the device's context
// is torn down and created again (cudaDeviceReset reloads the module, and the
// array may then sit at another address).  All calls on a device share the
// array and it keeps the last call's contents; whatever must start at zero is
// cleared by each call, and calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cstdint>

#include "lcs.h"
#include "lcs_common.cuh"
#include "lcs_kernels.h"

using namespace lcsg;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)6 << 20;   // 6 MiB per device
constexpr int64_t kStaticMaxN = 1024;                     // documented in lcs.h

static __device__ __align__(256) unsigned char g_merge_scratch[kStaticScratchBytes];

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of g_merge_scratch in the current device's context.
lcs_status scratch_address(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_merge_scratch) != cudaSuccess || !p) return LCS_ECUDA;
    *out = p;
    return LCS_OK;
}

}  // namespace

extern "C" lcs_status lcs_merge_static(const void *dist_u, const void *dist_l, int64_t n, lcs_dtype dtype,
                                       int64_t ld, void *dist_out, int32_t *argmax_out, void *stream) {
    if (n < 0 || n > kStaticMaxN) return LCS_EINVAL;          // beyond the static scratch
    if (dtype != LCS_I32 && dtype != LCS_I16) return LCS_EINVAL;
    const int dt = dtype == LCS_I16 ? DT_I16 : DT_I32;
    const int esz = dt_bytes(dt);
    auto dense_ok = [&](const void *p) {
        return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld >= n + 1 && (ld * esz) % 16 == 0;
    };
    if (!dense_ok(dist_u) || !dense_ok(dist_l) || !dense_ok(dist_out)) return LCS_EINVAL;
    if (argmax_out && (reinterpret_cast<uintptr_t>(argmax_out) & 15) != 0) return LCS_EINVAL;
    if (dist_out == dist_u || dist_out == dist_l) return LCS_EINVAL;

    void *base = nullptr;
    lcs_status s = scratch_address(&base);
    if (s != LCS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    // Carve the scratch: error word, job descriptor, packed U, packed L,
    // argmax and value grids.
    const int64_t NT = num_tiles_side(n), P = ceil_div(n, T);
    const size_t packed = round256((size_t)num_tiles_tri(NT) * tile_elems(dt) * esz);
    const size_t grids = round256(2 * (size_t)(P + 1) * (P + 1) * sizeof(int32_t));
    char *c = static_cast<char *>(base);
    int *err = reinterpret_cast<int *>(c);
    MergeJob *jobd = reinterpret_cast<MergeJob *>(c + 256);
    char *Up = c + 512, *Lp = Up + packed;
    int32_t *kgrid = reinterpret_cast<int32_t *>(Lp + packed);
    if (512 + 2 * packed + grids > kStaticScratchBytes) return LCS_EINVAL;

    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return LCS_ECUDA;
    if (launch_pack(dist_u, dt, n, ld, Up, LAYOUT_ROW, st) != cudaSuccess) return LCS_ECUDA;
    if (launch_pack(dist_l, dt, n, ld, Lp, LAYOUT_COL, st) != cudaSuccess) return LCS_ECUDA;
    MergeJob job{};
    job.U = Up;
    job.L = Lp;
    job.D = nullptr;
    job.kgrid = kgrid;
    job.vgrid = kgrid + (P + 1) * (P + 1);
    job.d_layout = LAYOUT_DENSE;
    // A pageable-to-device copy is staged before the call returns, so `job`
    // may go out of scope; nothing is allocated.
    if (cudaMemcpyAsync(jobd, &job, sizeof(job), cudaMemcpyHostToDevice, st) != cudaSuccess) return LCS_ECUDA;

    MergeParams mp{};
    mp.jobs = jobd;
    mp.njobs = 1;
    mp.n = n;
    mp.NT = NT;
    mp.P = P;
    mp.ld = ld;
    mp.err = err;
    mp.dense_out = dist_out;
    mp.dense_K = argmax_out;
    mp.const_tiles = argmax_out ? 0 : 1;
    const int64_t sigma0 = coarse_sigma0(P > 1 ? P : 1);
    mp.sigma = (int32_t)sigma0;
    mp.full = 1;
    if (launch_coarse(mp, dt, st) != cudaSuccess) return LCS_ECUDA;
    for (int64_t sg = sigma0 / 2; sg >= 1; sg /= 2) {
        mp.sigma = (int32_t)sg;
        mp.full = 0;
        if (launch_coarse(mp, dt, st) != cudaSuccess) return LCS_ECUDA;
    }
    if (launch_tile_pair(mp, dt, dt, st) != cudaSuccess) return LCS_ECUDA;
    if (launch_fill_dense(dist_out, dt, n, ld, dt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 0, argmax_out, st) !=
        cudaSuccess)
        return LCS_ECUDA;

    // Synchronous: wait, then report what the kernels flagged.
    int flags = 0;
    if (cudaMemcpyAsync(&flags, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LCS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LCS_ECUDA;
    if (flags & ERR_TIMEOUT) return LCS_ETIMEOUT;
    if (flags & ERR_OVERFLOW) return LCS_EOVERFLOW;
    if (flags) return LCS_EINVAL;          // inputs that are not strip DIST matrices
    return LCS_OK;
}
