// lcs_kernels.h -- host-side declarations of the kernel launchers and the
// job descriptors they read from device memory.  Internal to the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lcsg {

// ------------------------------------------------------------- strip builder
struct StripOut {
    void *base;        // tile-packed storage of this strip's DIST
    int32_t layout;    // LAYOUT_ROW or LAYOUT_COL
    int32_t pad;
};

struct StripParams {
    const uint8_t *a;      // first row of strip 0
    int64_t m;             // rows in all strips together
    int32_t h;             // rows per strip (the last strip may be shorter)
    int32_t S;             // number of strips
    const uint8_t *b;
    int64_t n;
    int64_t NT;            // tiles per side = ceil((n+1)/T)
    const StripOut *outs;  // [S] packed outputs (device array), or
    void *dense;           // dense (n+1) x ld output of strip 0 (S must be 1)
    int64_t ld;
    int32_t band_first;    // first band (tile row) this launch covers
    int32_t pad;
};

// out_dtype: DT_*; words = 32-bit words per source (1, 2, 4 or 8).
cudaError_t launch_strip(const StripParams &p, int out_dtype, int words, cudaStream_t st);

// ------------------------------------------------------------- merge
struct MergeJob {
    const void *U;       // upper operand, row layout
    const void *L;       // lower operand, column layout
    void *D;             // output: packed (row/col layout) or dense (n+1) x ld
    int32_t *kgrid;      // (P+1) x (P+1) argmax on the T-grid (scratch)
    int32_t *vgrid;      // (P+1) x (P+1) maximum (D itself) on the T-grid (scratch)
    int32_t d_layout;    // LAYOUT_ROW / LAYOUT_COL / LAYOUT_DENSE
    int32_t pad;
};

struct MergeParams {
    const MergeJob *jobs;  // device array
    int32_t njobs;
    int32_t cap;           // K-tiles of a band held in shared memory
    int64_t n, NT, P;      // P = ceil(n / T): T-grid points 0..P
    int64_t ld;            // dense leading dimension (elements)
    int *err;              // device error word
    int32_t sigma;         // coarse level stride (grid units)
    int32_t full;          // 1: full-scan coarse level
    void *dense_out;       // output of LAYOUT_DENSE jobs (per call)
    int32_t *dense_K;      // optional dense argmax of LAYOUT_DENSE jobs (per call)
    int32_t spill;         // 0: tiles whose band fits `cap`; 1: the others
    int32_t cap_main;      // the main launch's cap (spill launches only)
    int32_t const_tiles;   // 1: write tiles whose corner values agree as constants
    int32_t grab;          // DPX launch: tiles taken from `sched` at a time (set by the launcher)
    unsigned int *sched;   // DPX launch: tile counter (zero at launch) for dynamic scheduling, or null
    uint64_t wait_ns;      // limit of each bounded device wait (0: kWaitLimitNs)
    int32_t hold_band;     // test only: the first staged tile arms its barrier but copies nothing
    int32_t gshift;        // coarse grid spacing 2^gshift vertices (0: T = 64); P = ceil(n / 2^gshift)
};

// K-tiles per band for the main tile launch and the spill launch.
int tile_cap_main(int in_dtype);
int tile_cap_spill(int in_dtype, int out_dtype);
// Main launch then spill launch of the tile kernel (2 kernel launches).
cudaError_t launch_tile_pair(MergeParams p, int in_dtype, int out_dtype, cudaStream_t st);
// DPX (max,+) merge of every tile of every job, for int16 operands whose
// values are at most 16383 (D only, no argmax): one launch of persistent
// CTAs after the coarse levels.
cudaError_t launch_tile_dpx(MergeParams p, int out_dtype, cudaStream_t st);

// One pair of a batch on the one-strip path (batch.cu).
struct BatchPair {
    const uint8_t *a, *b;
    int64_t m, n;
    int64_t str_off;       // byte offset of the pair's LCS in BatchParams::strings
    int64_t scratch_off;   // word offset of its (n+1) x ceil(m/32) column vectors
    int64_t *len_out;      // device word receiving the length
    int32_t want;          // store the columns and walk back for the LCS
    int32_t pad;
};
struct BatchParams {
    const BatchPair *pairs;
    const int32_t *order;  // processing order (largest first), nullable
    int64_t count;
    uint32_t *scratch;
    uint8_t *strings;
    int *err;
    unsigned int *queue;   // work queue: the next position of `order` to take (zero at launch)
};
// A batch pair taller than one strip (up to two strips' rows) split at row
// rm: the split column c comes from the recomputing sweeps (recompute.cu),
// and its two halves (a[0:rm], b[0:c]) and (a[rm:m], b[c:n]) are ordinary
// one-strip pairs of the batch.
struct SplitPair {
    BatchPair *sub0, *sub1;   // device descriptors of the halves (their b and n are set from c)
    const uint8_t *b;
    int64_t n;
    int32_t lower;            // node id of the lower half: c = pathI[lower]
    int32_t big0, big1;       // 1: the half runs on the tall kernels (cross vertices initialised here)
    int32_t pad;
    const int32_t *pathI;
    uint32_t *scratch;        // the batch's scratch (tall halves' cross vertices)
    int64_t *len_out;         // the pair's length: len0 + len1
    uint8_t *str;             // the pair's string (the upper half's goes here), nullable
    const uint8_t *str1;      // the lower half's string, appended after the upper's, nullable
    int *err;
};
// Set the halves' columns (before the batch's kernels run).
cudaError_t launch_split_fix(const SplitPair *sp, int64_t count, cudaStream_t st);
// Join the halves' lengths and strings (after them).
cudaError_t launch_split_join(const SplitPair *sp, int64_t count, cudaStream_t st);

// The pairs of one words-per-lane class wpl (2, 4, 8 or 16: a up to
// 1024 wpl rows) on one launch, a warp per pair.
cudaError_t launch_batch_strip(const BatchParams &bp, int wpl, cudaStream_t st);
int batch_words_per_lane(int64_t m);
int batch_max_rows();

// Coarse argmax on the T-grid: one launch per level, sigma = sigma0 (full
// scans) then sigma0/2 .. 1 (windows bounded by the coarser level).
cudaError_t launch_coarse(const MergeParams &p, int in_dtype, cudaStream_t st);
// Tile refinement + output.
cudaError_t launch_tile(const MergeParams &p, int in_dtype, int out_dtype, cudaStream_t st);
size_t tile_smem_bytes(int in_dtype, int out_dtype, int cap);
int64_t coarse_sigma0(int64_t P);

// Dense (n+1) x ld matrix -> tile-packed storage in row or column layout.
cudaError_t launch_pack(const void *src, int dtype, int64_t n, int64_t ld, void *dst, int layout,
                        cudaStream_t st);

// ------------------------------------------------------------- dense fills
// Lower triangle (j < i) of a dense matrix outside the diagonal T-tiles gets
// `lower`; with `fill_upper` the whole upper triangle (j >= i) gets `upper`.
cudaError_t launch_fill_dense(void *out, int dtype, int64_t n, int64_t ld, int lower, int upper,
                              int fill_upper, int32_t *K, cudaStream_t st);
// The lower triangle outside the diagonal tiles (row i, columns
// [0, 64 floor(i / 64))) set to `lower` with 16-byte stores by `blocks`
// blocks of 256 threads: the region no merge tile writes, so it can be
// filled on a side stream while the tree is built.  out and ld * element
// size must be 16-byte aligned.
cudaError_t launch_fill_lower(void *out, int dtype, int64_t n, int64_t ld, int lower, int blocks, cudaStream_t st);

// ------------------------------------------------------------- traceback
struct TbMerge {
    const void *U;        // upper child (row layout)
    const void *L;        // lower child (column layout)
    const int32_t *kgrid; // the merge's argmax on the T-grid (complete when the level runs), or null
    int32_t in_dtype;
    int32_t node;         // index of the merged node (its path endpoints)
    int32_t upper;        // child node indices
    int32_t lower;
};

struct TbParams {
    const TbMerge *merges; // device array (one tree level)
    int32_t count;
    int32_t pad;
    int64_t n, NT;
    int32_t *pathI;       // [nodes] path endpoints (top vertex i, bottom vertex j)
    int32_t *pathJ;
    int64_t *len_out;     // written by the root merge: its maximum (the LCS length)
    int32_t root_node;
    int32_t pad2;
    int *err;
};
cudaError_t launch_tb_level(const TbParams &p, cudaStream_t st);
// The whole traceback above the leaves in one launch: a CTA per strip takes the
// splits of the tb merges chain[s * depth_max .. + depth[s]) from the root down.
cudaError_t launch_tb_path(const TbParams &p, const int32_t *chain, const int32_t *depth, int32_t depth_max,
                           int32_t strips, cudaStream_t st);
// pathI[root] = 0, pathJ[root] = n: the whole path, source to sink.
cudaError_t launch_root_path(int32_t *pathI, int32_t *pathJ, int32_t root, int64_t n, cudaStream_t st);

// Traceback of a tree whose nodes were freed (recompute.cu): per depth, a
// forward and a backward bit-vector sweep per node give one row of the upper
// child's DIST and one column of the lower child's; the smallest maximiser
// of their sum splits the node's sub-path.
struct SweepNode {
    int32_t node;          // merged node: its path endpoints pathI/pathJ[node]
    int32_t upper, lower;  // its children
    int32_t r0, rm, r1;    // rows: upper child [r0, rm), lower child [rm, r1)
};
// Strings of node q's pair when a launch covers nodes of several pairs.
struct SweepPair {
    const uint8_t *a, *b;
    int64_t n;
    int64_t *len_out;        // the node's maximum, nullable
};
struct SweepParams {
    const SweepNode *nodes;  // the nodes of one depth (device array)
    int32_t count;
    int32_t root_node;
    const uint8_t *a, *b;
    int64_t n;               // also the row stride of fcnt / bcnt (n + 1)
    int32_t *pathI, *pathJ;
    int32_t *fcnt, *bcnt;    // [count][n + 1] scratch: U(i, i + t), L(i + t, j)
    int64_t *len_out;        // the root's maximum (the LCS length), nullable
    int *err;
    const SweepPair *pairs;  // nullable: node q's strings and length word are pairs[q]'s
};
int sweep_max_rows();
cudaError_t launch_node_sweep(const SweepParams &p, int max_rows, cudaStream_t st);
cudaError_t launch_node_pick(const SweepParams &p, cudaStream_t st);

struct LeafParams {
    const uint8_t *a;
    int64_t m;
    int32_t h, S;
    const uint8_t *b;
    int64_t n;
    const int32_t *pathI; // strip s is node s
    const int32_t *pathJ;
    uint32_t *vbuf;       // forward bit-vectors, (n + S + 1) * words
    int32_t words;
    int32_t pad;
    uint8_t *slots;       // [S][h] emitted letters per strip
    int32_t *counts;      // [S]
    int32_t *cross;       // nullable [m+1]
    int *err;
};
// priority: the launch's scheduling priority (0: the stream's).
cudaError_t launch_leaf(const LeafParams &p, cudaStream_t st, int priority = 0);

struct CompactParams {
    const uint8_t *slots;
    const int32_t *counts;
    int32_t S, h;
    uint8_t *out;         // nullable
    int64_t cap;
    int64_t *len_out;     // nullable (device)
    int64_t *len_out2;    // nullable (device, caller's word)
    int *err;
};
cudaError_t launch_compact(const CompactParams &p, cudaStream_t st);

// Vertex list of the leftmost heaviest path from the cross vertices
// (traceback.cu): one CTA scans the rows' run lengths and writes the runs.
struct PathParams {
    const uint8_t *a, *b;
    int64_t m, n;
    const int32_t *cross;  // v[0..m]
    int32_t *offsets;      // m + 1 ints of scratch
    int32_t *path;         // 2 * cap ints: (row, col) pairs
    int64_t cap;
    const int64_t *len;    // device word holding the LCS length
    int64_t *count_out;    // device word receiving the vertex count
    int *err;
};
cudaError_t launch_path(const PathParams &p, cudaStream_t st);

// Tall batch pairs that want their string (batch_big.cu): scratch per pair
// of 2 * ceil(m/32) * (n+1) words (forward then backward column vectors,
// word-major) followed by m + 1 ints of cross vertices, set to a value
// above n before the launch.
struct BigParams {
    const BatchPair *pairs;  // the tall pairs of one words-per-lane class
    int64_t count;
    int64_t max_n;           // largest n among them
    uint32_t *scratch;
    int32_t *lens;           // count ints: the lengths, for the later kernels
    uint8_t *strings;
    int *err;
};
cudaError_t launch_big(const BigParams &p, int wpl, cudaStream_t st);

// Breakout (D-form) matrices (dform.cu).
struct DformStripParams {
    const uint8_t *a;      // m letters: strips of h rows (the last one may be shorter)
    int64_t m;
    int32_t h, pad;
    const uint8_t *b;
    int64_t n;
    void *out;             // strip s at out + s * (n+1) * ld: (n+1) x ld, row i = D(i, 0..h)
    int64_t ld;
};
cudaError_t launch_dform_strip(const DformStripParams &p, int dtype, int words, cudaStream_t st);
struct DformMergeParams {
    const void *du, *dl;   // (n+1) x (hu+1), (n+1) x (hl+1)
    int64_t ldu, ldl;
    int32_t hu, hl;
    int64_t n;
    void *out;             // (n+1) x (hu+hl+1)
    int64_t ldo;
};
cudaError_t launch_dform_merge(const DformMergeParams &p, int dtype, cudaStream_t st);

// Copy the internal length word to the caller's word (device to device).
cudaError_t launch_copy_len(const int64_t *src, int64_t *dst, cudaStream_t st);

}  // namespace lcsg
