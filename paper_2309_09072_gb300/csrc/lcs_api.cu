// lcs_api.cu -- the C ABI (include/lcs.h): context, tree planner, executor.
//
// Planner.  Rows of a are cut into S = ceil(m / h) strips.  Strips are merged
// pairwise, level by level (an odd node at the end of a level is carried up
// unchanged), into one root: the binary tree of Sec. II-A's recursive split,
// with the strip builder standing in for the bottom log2(h) levels.  Every
// node is stored in the narrowest integer type that holds the values of the
// merge that reads it (DIST of a node is at most its row count), and in the
// orientation that merge reads it in (upper operand by rows, lower operand by
// columns).  All merges of one level run in one launch of each kernel.
//
// Executor.  strips -> per level: coarse K grid, tile refinement -> (root
// merge into the caller's dense matrix if DIST is wanted) -> traceback: root
// path, per level leftmost argmax top down, leaves, compaction.  Every node
// of the tree stays resident until the traceback has passed it; the context
// workspace is sized from the plan and never exceeds the budget.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <thread>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lcs.h"
#include "lcs_common.cuh"
#include "lcs_kernels.h"

using namespace lcsg;

namespace {

int dt_size(int dt) { return dt == DT_U8 ? 1 : (dt == DT_I16 ? 2 : 4); }
int dt_for(int64_t maxval) { return maxval <= 255 ? DT_U8 : (maxval <= 32767 ? DT_I16 : DT_I32); }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int words_for(int h) {
    const int w = (h + 31) / 32;
    return w <= 1 ? 1 : (w <= 2 ? 2 : (w <= 4 ? 4 : 8));
}


struct Node {
    int64_t row0 = 0, rows = 0;
    int level = 0;
    int dtype = DT_U8;
    int layout = LAYOUT_ROW;
    int parent = -1;
    bool root = false;
    size_t off = 0;        // storage offset in the workspace (non-root nodes)
    size_t bytes = 0;      // its stored triangle (non-root nodes)
};

struct Merge {
    int u = -1, l = -1, out = -1;
    int level = 0;
    int in_dt = DT_U8, out_dt = DT_U8;
    size_t kgrid_off = 0;
};

struct Group {               // merges of one level launched together
    int level, in_dt, out_dt;
    int begin, count;        // range in the job array
    bool root;
};

// A launch of the depth-first schedule: strips [begin, begin + count) in one
// strip launch, or merge group `begin`.
struct Step {
    bool strips;
    int begin, count;
};

struct Plan {
    int64_t m = -1, n = -1;
    int h = 0, words = 1, S = 0, levels = 0, root = -1;
    // Depth first (bounded memory): strips are built `chunk` at a time and
    // merged as soon as both halves exist, nodes live in a pool of reused
    // slots, and the traceback recomputes what it needs (recompute.cu).
    bool depth_first = false;
    int chunk = 0;
    int pool_slots = 0;
    std::vector<Step> steps;
    std::vector<SweepNode> h_sweep;                  // merge nodes by depth from the root
    std::vector<std::pair<int, int>> sweep_levels;   // top-down ranges in h_sweep
    std::vector<int> sweep_rows;                     // tallest half per depth
    size_t off_sweep = 0, off_fcnt = 0, off_bcnt = 0, off_counters = 0;
    int max_depth_nodes = 0;
    bool dpx = false;        // every merge on the DPX (max,+) kernel, int16 nodes
    int64_t NT = 0, P = 0;   // tiles per side; coarse-grid points per side - 1 (spacing 64)
    int root_dt = DT_I32;    // dtype the root merge writes (caller's)
    std::vector<Node> nodes;
    std::vector<Merge> merges;         // in job order
    std::vector<Group> groups;         // bottom-up
    std::vector<std::pair<int, int>> tb_levels;   // top-down ranges in the tb array
    // device arrays (offsets in the workspace)
    size_t off_strip_outs = 0, off_jobs = 0, off_tb = 0, off_path = 0, off_counts = 0;
    size_t off_slots = 0, off_vbuf = 0, total = 0;
    std::vector<StripOut> h_strip_outs;
    std::vector<MergeJob> h_jobs;
    std::vector<TbMerge> h_tb;
    // Retained plans: strip s's tb merges from the root down (h_chain[s * depth_max + d], h_depth[s] of them).
    std::vector<int32_t> h_chain, h_depth;
    int32_t depth_max = 0;
    size_t off_chain = 0, off_depth = 0;
};

constexpr size_t kHeaderBytes = 256;   // err word (int) at 0, length word (int64) at 8,
                                       // DPX tile counters (one per tree level) at 64
constexpr size_t kSchedOffset = 64;
constexpr int kSchedSlots = 32;

// A submitted batch: its stream, completion events and one device block
// holding descriptors, lengths, strings, column vectors and an error word.
constexpr int kBatchClasses = 4;       // words per lane 2, 4, 8, 16
// The streams and events of one batch in flight, reused across batches.
struct BatchLane {
    cudaStream_t stream = nullptr;
    cudaStream_t aux[kBatchClasses] = {};  // one per words-per-lane class, forked from `stream`
    cudaEvent_t ev_join[kBatchClasses] = {};
    cudaEvent_t ev_start = nullptr, ev_done = nullptr, ev_fork = nullptr;
};
void destroy_lane(BatchLane &l) {
    if (l.stream) cudaStreamDestroy(l.stream);
    for (int c = 0; c < kBatchClasses; ++c) {
        if (l.aux[c]) cudaStreamDestroy(l.aux[c]);
        if (l.ev_join[c]) cudaEventDestroy(l.ev_join[c]);
    }
    if (l.ev_start) cudaEventDestroy(l.ev_start);
    if (l.ev_done) cudaEventDestroy(l.ev_done);
    if (l.ev_fork) cudaEventDestroy(l.ev_fork);
    l = BatchLane{};
}
bool create_lane(BatchLane &l) {
    bool ok = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&l.ev_start) == cudaSuccess && cudaEventCreate(&l.ev_done) == cudaSuccess &&
              cudaEventCreateWithFlags(&l.ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int c = 0; ok && c < kBatchClasses; ++c)
        ok = cudaStreamCreateWithFlags(&l.aux[c], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&l.ev_join[c], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_lane(l);
    }
    return ok;
}

struct BatchTicket {
    int64_t count = 0;
    BatchLane lane;
    double t_submit = 0.0;
    char *dev = nullptr;
    size_t bytes = 0;
    int64_t *d_lens = nullptr;
    uint8_t *d_strings = nullptr;
    int *d_err = nullptr;
    int64_t strings_bytes = 0;
    std::vector<int64_t> str_off;          // -1: no string wanted
    std::vector<lcs_status> host_status;   // pairs solved at submit (the strip tree)
};

double steady_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct lcs_ctx {
    int device = 0;
    size_t budget = 0;
    int32_t strip_h = 0;
    int32_t merge_kernel = LCS_MERGE_AUTO;
    uint64_t wait_ns = 0;        // bounded device waits (0: the kernels' default)
    int32_t hold_band = 0;       // fault injection (lcs_set_fault_injection)
    char *ws = nullptr;          // plan workspace
    size_t ws_bytes = 0;
    char *io = nullptr;          // host-call staging (lcs_solve_host, lcs_merge)
    size_t io_bytes = 0;
    size_t peak = 0;
    std::string last_error;
    lcs_stats stats{};
    Plan plan;
    bool plan_uploaded = false;
    bool auto_h = false;         // the current plan's h was chosen automatically
    int launches = 0;
    // profiling (lcs_set_profiling)
    bool profiling = false;
    struct Rec { int kind; cudaEvent_t e0, e1; double bytes, ops; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // batches (lcs_batch_submit)
    std::map<uint64_t, BatchTicket> tickets;
    uint64_t next_ticket = 1;
    size_t batch_bytes = 0;
    std::vector<BatchLane> free_lanes;    // streams/events of released batches
    cudaMemPool_t mempool = nullptr;      // batches' device memory (stream ordered, no device sync)
    // solve_device: the root merge group beside the traceback
    cudaStream_t root_side = nullptr;
    // depth-first solves: the recomputing traceback beside the tree
    cudaStream_t tb_side = nullptr;
    cudaEvent_t ev_tb_fork = nullptr, ev_tb = nullptr;
    int32_t schedule = LCS_SCHED_AUTO, sched_chunk = 0;
    std::vector<int64_t> sched_key;       // inputs of the current plan's schedule choice
    cudaEvent_t ev_fork = nullptr, ev_root = nullptr;
    cudaEvent_t ev_tbl = nullptr;         // the traceback's argmax levels are done (the root tiles may start)
    int leaf_priority = 0;                // the leaf kernel's launch priority (the device's greatest)
    // lcs_solve_host: DIST copied on a side stream while the traceback runs
    cudaStream_t side = nullptr;
    cudaEvent_t ev_dist = nullptr, ev_copied = nullptr;
    int64_t *host_hdr = nullptr;          // pinned: error word and length, read once per call
    // CUDA-graph replay of lcs_solve (lcs_set_graphs)
    bool graphs = false;
    cudaStream_t cap_stream = nullptr;    // private stream the solve is captured on
    cudaGraphExec_t gexec = nullptr;
    std::vector<int64_t> gkey;            // the arguments and plan state the graph was captured for
    int32_t glaunches = 0;
    // autotuner (lcs_autotune): (m bucket, n bucket, root dtype, wants dist) -> (h, merge kernel)
    std::map<std::vector<int64_t>, std::pair<int32_t, int32_t>> tuned;
    int32_t tuned_merge = -1;             // merge kernel chosen with the current automatic h, -1: none
    int64_t tune_gen = 0;                 // bumped by every lcs_autotune
    int64_t plan_gen = 0;                 // bumped whenever the device copy of the plan is rewritten
};

namespace {

lcs_status fail(lcs_ctx *ctx, lcs_status s, const std::string &what) {
    if (ctx) ctx->last_error = what;
    return s;
}

lcs_status cuda_fail(lcs_ctx *ctx, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, LCS_ENOMEM, msg);
    return fail(ctx, LCS_ECUDA, msg);
}

#define LCS_CK(ctx, expr)                                      \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

enum Kind { K_STRIP = 0, K_COARSE = 1, K_TILE = 2, K_TB = 3, K_LEAF = 4, K_COMPACT = 5, K_FILL = 6, K_KINDS = 7 };

double tri_entries(int64_t n) { return (double)(n + 1) * (double)(n + 2) / 2.0; }
// Strip builder: per (strip, source i, column j > i) step, 3 integer
// instructions per 32-bit word (and, add with carry, and-not/or) plus 2
// (carry out, accumulate).
double strip_ops(int strips, int64_t n, int words) {
    return (double)strips * (double)n * (double)(n + 1) / 2.0 * (3.0 * words + 2.0);
}

cudaEvent_t take_event(lcs_ctx *ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Event pair around one launch when profiling is on (else a no-op).
int prof_begin(lcs_ctx *ctx, cudaStream_t st) {
    if (!ctx->profiling) return -1;
    lcs_ctx::Rec r{0, take_event(ctx), take_event(ctx), 0.0, 0.0};
    if (!r.e0 || !r.e1) {                  // out of events: this launch goes untimed
        if (r.e0) ctx->pool.push_back(r.e0);
        if (r.e1) ctx->pool.push_back(r.e1);
        return -1;
    }
    cudaEventRecord(r.e0, st);
    ctx->recs.push_back(r);
    return (int)ctx->recs.size() - 1;
}
void prof_end(lcs_ctx *ctx, int idx, cudaStream_t st, int kind, double bytes, double ops) {
    if (idx < 0) return;
    lcs_ctx::Rec &r = ctx->recs[idx];
    r.kind = kind; r.bytes = bytes; r.ops = ops;
    cudaEventRecord(r.e1, st);
}

#define LCS_LAUNCHK(ctx, st, kind, bytes, ops, expr)              \
    do {                                                          \
        const int pi_ = prof_begin(ctx, st);                      \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);  \
        (ctx)->launches++;                                        \
        prof_end(ctx, pi_, st, kind, bytes, ops);                 \
    } while (0)

// The side stream of a solve (the early dense fill, the root merge group)
// and its fork / join events, created on first use.
lcs_status ensure_root_side(lcs_ctx *ctx) {
    if (!ctx->root_side) LCS_CK(ctx, cudaStreamCreateWithFlags(&ctx->root_side, cudaStreamNonBlocking));
    if (!ctx->ev_fork) LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_root) LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_root, cudaEventDisableTiming));
    if (!ctx->ev_tbl) {
        LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_tbl, cudaEventDisableTiming));
        int least = 0, greatest = 0;
        LCS_CK(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        ctx->leaf_priority = greatest;
    }
    return LCS_OK;
}

lcs_status ensure_tb_side(lcs_ctx *ctx) {
    if (!ctx->tb_side) LCS_CK(ctx, cudaStreamCreateWithFlags(&ctx->tb_side, cudaStreamNonBlocking));
    if (!ctx->ev_tb_fork) LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_tb_fork, cudaEventDisableTiming));
    if (!ctx->ev_tb) LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_tb, cudaEventDisableTiming));
    return LCS_OK;
}

// Strip height when none is set: 256 rows (eight 32-bit words per bit
// vector), or m for a shorter a.  Halving h doubles the strips but adds a
// tree level of merges, the dominant cost, so at m = n = 4096 the
// autotuner's candidates 64, 128 and 256 rank in that order, slowest first.
// Memory is bounded by the schedule (depth first), not by the strip height.
int auto_strip_height(int64_t m, int64_t n) {
    (void)n;
    if (m <= 256) return (int)std::max<int64_t>(m, 1);
    return 256;
}

Plan build_plan(int64_t m, int64_t n, int h, int root_dt) {
    Plan P;
    P.m = m; P.n = n; P.h = h; P.words = words_for(h); P.root_dt = root_dt;
    P.S = (int)ceil_div(m, h);
    P.NT = num_tiles_side(n);
    P.P = ceil_div(n, T);
    for (int s = 0; s < P.S; ++s) {
        Node nd;
        nd.row0 = (int64_t)s * h;
        nd.rows = std::min<int64_t>(h, m - nd.row0);
        P.nodes.push_back(nd);
    }
    std::vector<int> cur(P.S);
    for (int s = 0; s < P.S; ++s) cur[s] = s;
    int level = 0;
    std::vector<Merge> merges;
    while (cur.size() > 1) {
        ++level;
        std::vector<int> next;
        for (size_t q = 0; q < cur.size(); q += 2) {
            if (q + 1 < cur.size()) {
                Node nd;
                nd.row0 = P.nodes[cur[q]].row0;
                nd.rows = P.nodes[cur[q]].rows + P.nodes[cur[q + 1]].rows;
                nd.level = level;
                P.nodes.push_back(nd);
                const int out = (int)P.nodes.size() - 1;
                Merge mg;
                mg.u = cur[q]; mg.l = cur[q + 1]; mg.out = out; mg.level = level;
                P.nodes[mg.u].parent = out; P.nodes[mg.u].layout = LAYOUT_ROW;
                P.nodes[mg.l].parent = out; P.nodes[mg.l].layout = LAYOUT_COL;
                merges.push_back(mg);
                next.push_back(out);
            } else {
                next.push_back(cur[q]);
            }
        }
        cur.swap(next);
    }
    P.levels = level;
    P.root = cur[0];
    P.nodes[P.root].root = true;
    // The DPX kernel adds int16 pairs: every operand value must stay at or
    // below 16383 (a node's DIST is at most its row count).
    P.dpx = true;
    for (auto &mg : merges)
        if (std::max(P.nodes[mg.u].rows, P.nodes[mg.l].rows) > 16383) P.dpx = false;
    for (auto &mg : merges) {
        mg.in_dt = P.dpx ? (int)DT_I16 : dt_for(std::max(P.nodes[mg.u].rows, P.nodes[mg.l].rows));
        P.nodes[mg.u].dtype = mg.in_dt;
        P.nodes[mg.l].dtype = mg.in_dt;
    }
    for (auto &mg : merges) mg.out_dt = (mg.out == P.root) ? root_dt : P.nodes[mg.out].dtype;
    // Strips need a dtype even when S == 1 (unused then).
    // Job order: level ascending, then (in_dt, out_dt), the root merge last.
    std::stable_sort(merges.begin(), merges.end(), [&](const Merge &x, const Merge &y) {
        const bool rx = x.out == P.root, ry = y.out == P.root;
        if (x.level != y.level) return x.level < y.level;
        if (rx != ry) return ry;
        if (x.in_dt != y.in_dt) return x.in_dt < y.in_dt;
        return x.out_dt < y.out_dt;
    });
    P.merges = merges;

    // Workspace layout.
    size_t off = kHeaderBytes;
    const int64_t tiles = num_tiles_tri(P.NT);
    for (size_t v = 0; v < P.nodes.size(); ++v) {
        Node &nd = P.nodes[v];
        if (nd.root) continue;
        nd.off = off;
        nd.bytes = (size_t)tiles * tile_elems(nd.dtype) * dt_size(nd.dtype);
        off = align256(off + nd.bytes);
    }
    for (auto &mg : P.merges) {
        mg.kgrid_off = off;                       // kgrid then vgrid
        off = align256(off + 2 * (size_t)(P.P + 1) * (P.P + 1) * 4);
    }
    P.off_strip_outs = off; off = align256(off + sizeof(StripOut) * P.S);
    P.off_jobs = off; off = align256(off + sizeof(MergeJob) * std::max<size_t>(1, P.merges.size()));
    P.off_tb = off; off = align256(off + sizeof(TbMerge) * std::max<size_t>(1, P.merges.size()));
    P.off_path = off; off = align256(off + sizeof(int32_t) * 2 * P.nodes.size());
    P.depth_max = std::max(1, P.levels);
    P.off_chain = off; off = align256(off + sizeof(int32_t) * (size_t)P.S * P.depth_max);
    P.off_depth = off; off = align256(off + sizeof(int32_t) * (size_t)P.S);
    P.off_counts = off; off = align256(off + sizeof(int32_t) * 2 * P.S);
    P.off_slots = off; off = align256(off + (size_t)P.S * h);
    P.off_vbuf = off; off = align256(off + (size_t)(n + P.S + 1) * P.words * 4);
    P.total = off;

    // Groups (bottom-up) and traceback ranges (top-down).
    for (int q = 0; q < (int)P.merges.size();) {
        const Merge &a = P.merges[q];
        int e = q + 1;
        while (e < (int)P.merges.size()) {
            const Merge &b = P.merges[e];
            if (b.level != a.level || b.in_dt != a.in_dt || b.out_dt != a.out_dt ||
                (b.out == P.root) != (a.out == P.root))
                break;
            ++e;
        }
        P.groups.push_back(Group{a.level, a.in_dt, a.out_dt, q, e - q, a.out == P.root});
        q = e;
    }
    // tb array: level descending.
    std::vector<int> order(P.merges.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return P.merges[x].level > P.merges[y].level; });
    for (size_t q = 0; q < order.size();) {
        size_t e = q + 1;
        while (e < order.size() && P.merges[order[e]].level == P.merges[order[q]].level) ++e;
        P.tb_levels.push_back({(int)q, (int)(e - q)});
        q = e;
    }
    P.h_tb.resize(order.size());
    for (size_t q = 0; q < order.size(); ++q) {
        const Merge &mg = P.merges[order[q]];
        TbMerge t{};
        t.U = reinterpret_cast<const void *>(P.nodes[mg.u].off);   // relocated at upload
        t.L = reinterpret_cast<const void *>(P.nodes[mg.l].off);
        t.in_dtype = mg.in_dt;
        t.node = mg.out; t.upper = mg.u; t.lower = mg.l;
        // The root's grid is computed beside the traceback (the root merge
        // group runs on a side stream): the root level scans its whole row.
        t.kgrid = (mg.out == P.root) ? nullptr : reinterpret_cast<const int32_t *>(mg.kgrid_off);
        P.h_tb[q] = t;
    }
    // Each strip's tb merges from the root down, for the one-launch traceback.
    // Every pairing level puts at most one merge above a node, so no strip
    // lies deeper than `levels` (= depth_max).
    {
        std::vector<int32_t> tb_of_node(P.nodes.size(), -1);
        for (size_t q = 0; q < P.h_tb.size(); ++q) tb_of_node[P.h_tb[q].node] = (int32_t)q;
        P.h_chain.assign((size_t)P.S * P.depth_max, 0);
        P.h_depth.assign(P.S, 0);
        for (int st = 0; st < P.S; ++st) {
            std::vector<int32_t> up;
            for (int v = st; v != P.root && P.nodes[v].parent >= 0; v = P.nodes[v].parent) up.push_back(tb_of_node[P.nodes[v].parent]);
            P.h_depth[st] = (int32_t)std::min<size_t>(up.size(), (size_t)P.depth_max);
            for (size_t d = 0; d < up.size() && (int)d < P.depth_max; ++d) P.h_chain[(size_t)st * P.depth_max + d] = up[up.size() - 1 - d];
        }
    }
    P.h_jobs.resize(P.merges.size());
    for (size_t q = 0; q < P.merges.size(); ++q) {
        const Merge &mg = P.merges[q];
        MergeJob j{};
        j.U = reinterpret_cast<const void *>(P.nodes[mg.u].off);
        j.L = reinterpret_cast<const void *>(P.nodes[mg.l].off);
        j.D = (mg.out == P.root) ? nullptr : reinterpret_cast<void *>(P.nodes[mg.out].off);
        j.kgrid = reinterpret_cast<int32_t *>(mg.kgrid_off);
        j.vgrid = reinterpret_cast<int32_t *>(mg.kgrid_off + (size_t)(P.P + 1) * (P.P + 1) * 4);
        j.d_layout = (mg.out == P.root) ? LAYOUT_DENSE : P.nodes[mg.out].layout;
        P.h_jobs[q] = j;
    }
    P.h_strip_outs.resize(P.S);
    for (int s = 0; s < P.S; ++s) {
        StripOut o{};
        o.base = reinterpret_cast<void *>(P.nodes[s].off);
        o.layout = P.nodes[s].layout;
        P.h_strip_outs[s] = o;
    }
    return P;
}

// Depth-first plan.  Strips are built `chunk` at a time; the strips of a
// chunk are merged level by level into one node (one launch per level), and
// that node enters a binary counter: while the counter holds a node of the
// same level, the two are merged at once (the earlier rows are the upper
// half).  At the end the counter's nodes are merged from the last rows up.
// Every node is consumed by its parent right after it is made, so only the
// chunk's nodes and one pending node per level are alive at a time; they
// live in a pool of slots that the planner assigns by simulating the
// launches (a merge's output slot is taken before its operands' slots are
// released).  The root is the caller's dense matrix.  The tree's shape
// differs from the breadth-first one when the strip count is not a power of
// two; DIST is the same, and so is the LCS (the leftmost heaviest path does
// not depend on the tree).
Plan build_plan_depth_first(int64_t m, int64_t n, int h, int root_dt, int chunk) {
    Plan P;
    P.m = m; P.n = n; P.h = h; P.words = words_for(h); P.root_dt = root_dt;
    P.S = (int)ceil_div(m, h);
    P.NT = num_tiles_side(n);
    P.P = ceil_div(n, T);
    P.depth_first = true;
    P.chunk = chunk = std::max(1, std::min(chunk, P.S));
    for (int s = 0; s < P.S; ++s) {
        Node nd;
        nd.row0 = (int64_t)s * h;
        nd.rows = std::min<int64_t>(h, m - nd.row0);
        P.nodes.push_back(nd);
    }
    std::vector<Merge> merges;
    auto merge = [&](int u, int l, int level) -> int {
        Node nd;
        nd.row0 = P.nodes[u].row0;
        nd.rows = P.nodes[u].rows + P.nodes[l].rows;
        nd.level = level;
        P.nodes.push_back(nd);
        const int out = (int)P.nodes.size() - 1;
        Merge mg;
        mg.u = u; mg.l = l; mg.out = out; mg.level = level;
        P.nodes[u].parent = out; P.nodes[u].layout = LAYOUT_ROW;
        P.nodes[l].parent = out; P.nodes[l].layout = LAYOUT_COL;
        merges.push_back(mg);
        return out;
    };
    std::vector<std::pair<int, int>> counter;      // (node, level)
    std::vector<std::pair<int, int>> group_ranges;  // merge ranges launched together
    for (int s0 = 0; s0 < P.S; s0 += chunk) {
        const int cnt = std::min(chunk, P.S - s0);
        P.steps.push_back(Step{true, s0, cnt});
        std::vector<int> cur;
        for (int s = s0; s < s0 + cnt; ++s) cur.push_back(s);
        int level = 0;
        while (cur.size() > 1) {
            ++level;
            std::vector<int> next;
            const int gb = (int)merges.size();
            for (size_t q = 0; q < cur.size(); q += 2)
                next.push_back(q + 1 < cur.size() ? merge(cur[q], cur[q + 1], level) : cur[q]);
            group_ranges.push_back({gb, (int)merges.size() - gb});
            P.steps.push_back(Step{false, (int)group_ranges.size() - 1, 0});
            cur.swap(next);
        }
        int node = cur[0];
        while (!counter.empty() && counter.back().second == level) {
            const int u = counter.back().first;
            counter.pop_back();
            ++level;
            const int gb = (int)merges.size();
            node = merge(u, node, level);
            group_ranges.push_back({gb, 1});
            P.steps.push_back(Step{false, (int)group_ranges.size() - 1, 0});
        }
        counter.push_back({node, level});
    }
    int node = counter.back().first;
    int top = counter.back().second;
    counter.pop_back();
    while (!counter.empty()) {
        const int u = counter.back().first;
        top = std::max(top, counter.back().second) + 1;
        counter.pop_back();
        const int gb = (int)merges.size();
        node = merge(u, node, top);
        group_ranges.push_back({gb, 1});
        P.steps.push_back(Step{false, (int)group_ranges.size() - 1, 0});
    }
    P.root = node;
    P.nodes[P.root].root = true;
    P.levels = 0;
    for (auto &mg : merges) P.levels = std::max(P.levels, mg.level);
    P.dpx = true;
    for (auto &mg : merges)
        if (std::max(P.nodes[mg.u].rows, P.nodes[mg.l].rows) > 16383) P.dpx = false;
    for (auto &mg : merges) {
        mg.in_dt = P.dpx ? (int)DT_I16 : dt_for(std::max(P.nodes[mg.u].rows, P.nodes[mg.l].rows));
        P.nodes[mg.u].dtype = mg.in_dt;
        P.nodes[mg.l].dtype = mg.in_dt;
    }
    for (auto &mg : merges) mg.out_dt = (mg.out == P.root) ? root_dt : P.nodes[mg.out].dtype;
    P.merges = merges;
    // Launch groups; a group whose merges differ in type is split.
    std::vector<int> step_of_range(group_ranges.size());
    {
        std::vector<Step> steps;
        for (const Step &st : P.steps) {
            if (st.strips) { steps.push_back(st); continue; }
            const auto rg = group_ranges[st.begin];
            for (int q = rg.first; q < rg.first + rg.second;) {
                const Merge &a = P.merges[q];
                int e = q + 1;
                while (e < rg.first + rg.second && P.merges[e].in_dt == a.in_dt && P.merges[e].out_dt == a.out_dt) ++e;
                P.groups.push_back(Group{a.level, a.in_dt, a.out_dt, q, e - q, a.out == P.root});
                steps.push_back(Step{false, (int)P.groups.size() - 1, 0});
                q = e;
            }
        }
        P.steps.swap(steps);
    }
    // Pool slots by simulation.
    std::vector<int> slot(P.nodes.size(), -1), free_slots;
    int nslots = 0;
    auto take = [&]() { if (!free_slots.empty()) { int x = free_slots.back(); free_slots.pop_back(); return x; } return nslots++; };
    size_t max_group = 1;
    for (const Step &st : P.steps) {
        if (st.strips) {
            for (int s = st.begin; s < st.begin + st.count; ++s)
                if (!P.nodes[s].root) slot[s] = take();
            continue;
        }
        const Group &g = P.groups[st.begin];
        max_group = std::max(max_group, (size_t)g.count);
        for (int q = g.begin; q < g.begin + g.count; ++q)
            if (P.merges[q].out != P.root) slot[P.merges[q].out] = take();
        for (int q = g.begin; q < g.begin + g.count; ++q) {
            free_slots.push_back(slot[P.merges[q].u]);
            free_slots.push_back(slot[P.merges[q].l]);
        }
    }
    P.pool_slots = nslots;
    int max_dt_size = 1;
    for (auto &nd : P.nodes) if (!nd.root) max_dt_size = std::max(max_dt_size, dt_size(nd.dtype));
    const int slot_dt = max_dt_size == 4 ? DT_I32 : (max_dt_size == 2 ? DT_I16 : DT_U8);
    const size_t slot_bytes = align256((size_t)num_tiles_tri(P.NT) * tile_elems(slot_dt) * dt_size(slot_dt));
    size_t off = kHeaderBytes;
    const size_t pool = off;
    off += (size_t)nslots * slot_bytes;
    for (size_t v = 0; v < P.nodes.size(); ++v) {
        Node &nd = P.nodes[v];
        if (nd.root) continue;
        nd.off = pool + (size_t)slot[v] * slot_bytes;
        nd.bytes = (size_t)num_tiles_tri(P.NT) * tile_elems(nd.dtype) * dt_size(nd.dtype);
    }
    // Coarse grids: one per merge of the largest group, reused group after group.
    const size_t kg_bytes = align256(2 * (size_t)(P.P + 1) * (P.P + 1) * 4);
    const size_t kg_base = off;
    off += max_group * kg_bytes;
    for (auto &g : P.groups)
        for (int q = g.begin; q < g.begin + g.count; ++q) P.merges[q].kgrid_off = kg_base + (size_t)(q - g.begin) * kg_bytes;
    P.off_counters = off; off = align256(off + sizeof(unsigned) * std::max<size_t>(1, P.groups.size()));
    P.off_strip_outs = off; off = align256(off + sizeof(StripOut) * P.S);
    P.off_jobs = off; off = align256(off + sizeof(MergeJob) * std::max<size_t>(1, P.merges.size()));
    // Traceback by recompute: merge nodes by depth from the root.
    std::vector<int> depth(P.nodes.size(), -1);
    depth[P.root] = 0;
    std::vector<int> order(P.merges.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    for (int q = (int)P.merges.size() - 1; q >= 0; --q) {      // parents after children in job order
        const Merge &mg = P.merges[q];
        depth[mg.u] = depth[mg.out] + 1;
        depth[mg.l] = depth[mg.out] + 1;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return depth[P.merges[x].out] < depth[P.merges[y].out]; });
    for (size_t q = 0; q < order.size();) {
        size_t e = q + 1;
        while (e < order.size() && depth[P.merges[order[e]].out] == depth[P.merges[order[q]].out]) ++e;
        int rows = 0;
        for (size_t t = q; t < e; ++t) {
            const Merge &mg = P.merges[order[t]];
            rows = std::max<int>(rows, (int)std::max(P.nodes[mg.u].rows, P.nodes[mg.l].rows));
        }
        P.sweep_levels.push_back({(int)q, (int)(e - q)});
        P.sweep_rows.push_back(rows);
        P.max_depth_nodes = std::max(P.max_depth_nodes, (int)(e - q));
        q = e;
    }
    for (int q : order) {
        const Merge &mg = P.merges[q];
        SweepNode sn{};
        sn.node = mg.out; sn.upper = mg.u; sn.lower = mg.l;
        sn.r0 = (int32_t)P.nodes[mg.u].row0;
        sn.rm = (int32_t)P.nodes[mg.l].row0;
        sn.r1 = (int32_t)(P.nodes[mg.l].row0 + P.nodes[mg.l].rows);
        P.h_sweep.push_back(sn);
    }
    P.off_sweep = off; off = align256(off + sizeof(SweepNode) * std::max<size_t>(1, P.h_sweep.size()));
    P.off_fcnt = off; off = align256(off + (size_t)std::max(1, P.max_depth_nodes) * (n + 1) * 4);
    P.off_bcnt = off; off = align256(off + (size_t)std::max(1, P.max_depth_nodes) * (n + 1) * 4);
    P.off_tb = off; off = align256(off + sizeof(TbMerge));
    P.off_path = off; off = align256(off + sizeof(int32_t) * 2 * P.nodes.size());
    P.off_counts = off; off = align256(off + sizeof(int32_t) * 2 * P.S);
    P.off_slots = off; off = align256(off + (size_t)P.S * h);
    P.off_vbuf = off; off = align256(off + (size_t)(n + P.S + 1) * P.words * 4);
    P.total = off;
    P.h_jobs.resize(P.merges.size());
    for (size_t q = 0; q < P.merges.size(); ++q) {
        const Merge &mg = P.merges[q];
        MergeJob j{};
        j.U = reinterpret_cast<const void *>(P.nodes[mg.u].off);
        j.L = reinterpret_cast<const void *>(P.nodes[mg.l].off);
        j.D = (mg.out == P.root) ? nullptr : reinterpret_cast<void *>(P.nodes[mg.out].off);
        j.kgrid = reinterpret_cast<int32_t *>(mg.kgrid_off);
        j.vgrid = reinterpret_cast<int32_t *>(mg.kgrid_off + (size_t)(P.P + 1) * (P.P + 1) * 4);
        j.d_layout = (mg.out == P.root) ? LAYOUT_DENSE : P.nodes[mg.out].layout;
        P.h_jobs[q] = j;
    }
    P.h_strip_outs.resize(P.S);
    for (int s = 0; s < P.S; ++s) {
        StripOut o{};
        o.base = reinterpret_cast<void *>(P.nodes[s].off);
        o.layout = P.nodes[s].layout;
        P.h_strip_outs[s] = o;
    }
    return P;
}

template <typename X> X *reloc(char *base, X *off) {
    return reinterpret_cast<X *>(base + reinterpret_cast<uintptr_t>(off));
}

lcs_status ensure_workspace(lcs_ctx *ctx, size_t bytes) {
    if (bytes + ctx->io_bytes > ctx->budget)
        return fail(ctx, LCS_ENOMEM, "workspace of " + std::to_string(bytes) + " bytes exceeds the budget");
    if (ctx->ws_bytes >= bytes) return LCS_OK;
    if (ctx->ws) {
        LCS_CK(ctx, cudaDeviceSynchronize());
        LCS_CK(ctx, cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    LCS_CK(ctx, cudaMalloc(&ctx->ws, bytes));
    LCS_CK(ctx, cudaMemset(ctx->ws, 0, kHeaderBytes));
    ctx->ws_bytes = bytes;
    ctx->peak = std::max(ctx->peak, ctx->ws_bytes + ctx->io_bytes);
    ctx->plan_uploaded = false;
    return LCS_OK;
}

lcs_status ensure_io(lcs_ctx *ctx, size_t bytes) {
    if (ctx->io_bytes >= bytes) return LCS_OK;
    if (bytes + ctx->ws_bytes > ctx->budget)
        return fail(ctx, LCS_ENOMEM, "staging of " + std::to_string(bytes) + " bytes exceeds the budget");
    if (ctx->io) {
        LCS_CK(ctx, cudaDeviceSynchronize());
        LCS_CK(ctx, cudaFree(ctx->io));
        ctx->io = nullptr;
        ctx->io_bytes = 0;
    }
    LCS_CK(ctx, cudaMalloc(&ctx->io, bytes));
    ctx->io_bytes = bytes;
    ctx->peak = std::max(ctx->peak, ctx->ws_bytes + ctx->io_bytes);
    return LCS_OK;
}

// The budget left for the workspace (host-call staging holds the rest).
size_t room_of(const lcs_ctx *ctx) { return ctx->budget > ctx->io_bytes ? ctx->budget - ctx->io_bytes : 0; }

// Size bucket of the autotuner: floor(log2) of each length and the root
// dtype (the dense output, when asked for, changes the root merge's work).
std::vector<int64_t> tune_key(int64_t m, int64_t n, int root_dt) {
    auto lg = [](int64_t x) { int64_t b = 0; while (x > 1) { x >>= 1; ++b; } return b; };
    return {lg(m), lg(n), (int64_t)root_dt};
}

// Retained (breadth-first) tree when it fits comfortably, else depth first
// with the largest chunk of strips whose plan stays within both the budget
// and kDepthTarget (larger chunks mean fewer, fuller launches: at m = n =
// 16384 a chunk of 32 strips needs about 14 GB against the retained tree's
// 36 GB).  Forced either way by lcs_set_schedule.  The recomputing
// traceback sweeps a tree half of at most sweep_max_rows() rows in one CTA,
// so a taller half keeps the retained tree when an LCS is wanted.
constexpr size_t kRetainLimit = (size_t)4 << 30;
constexpr size_t kDefaultBudget = (size_t)64 << 30;   // lcs_create's mem_budget_bytes = 0
constexpr size_t kDepthTarget = (size_t)16 << 30;

Plan pick_plan(int schedule, int sched_chunk, size_t room, int64_t m, int64_t n, int h, int root_dt, bool want_tb) {
    Plan R = build_plan(m, n, h, root_dt);
    if (schedule == LCS_SCHED_RETAIN || R.S <= 1) return R;
    if (schedule == LCS_SCHED_AUTO && R.total <= std::min(room, kRetainLimit)) return R;
    auto too_tall = [&](const Plan &D) {
        for (auto &mg : D.merges)
            if (std::max(D.nodes[mg.u].rows, D.nodes[mg.l].rows) > sweep_max_rows()) return true;
        return false;
    };
    std::vector<int> chunks;
    if (sched_chunk > 0) chunks.push_back(sched_chunk);
    else chunks = {32, 16, 8, 4, 2, 1};
    const size_t target = sched_chunk > 0 ? room : std::min(room, kDepthTarget);
    Plan D;
    for (int c : chunks) {
        if (c > R.S && c > 1 && sched_chunk == 0) continue;
        D = build_plan_depth_first(m, n, h, root_dt, c);
        if (want_tb && too_tall(D)) return R;
        if (D.total <= target) return D;
    }
    // Nothing within the target: the smallest chunk that fits the budget.
    if (D.total <= room) return D;
    return R.total <= room ? R : D;      // neither fits: ensure_workspace reports ENOMEM
}

Plan choose_plan(lcs_ctx *ctx, int64_t m, int64_t n, int h, int root_dt, bool want_tb) {
    return pick_plan(ctx->schedule, ctx->sched_chunk, room_of(ctx), m, n, h, root_dt, want_tb);
}

// Make ctx->plan match (m, n, h, root dtype) and upload its device arrays.
lcs_status prepare(lcs_ctx *ctx, int64_t m, int64_t n, int root_dt, bool want_tb) {
    Plan &P = ctx->plan;
    int h = ctx->strip_h;
    ctx->tuned_merge = -1;
    if (h <= 0) {
        // A tuned choice for this size bucket, else the current plan's
        // choice for the same shape, else the rule.
        auto it = ctx->tuned.find(tune_key(m, n, root_dt));
        if (it != ctx->tuned.end()) {
            h = it->second.first;
            ctx->tuned_merge = it->second.second;
        } else {
            h = (P.m == m && P.n == n && P.root_dt == root_dt && ctx->auto_h) ? P.h
                                                                               : auto_strip_height(m, n);
        }
        ctx->auto_h = true;
    } else {
        ctx->auto_h = false;
    }
    const std::vector<int64_t> key = {m, n, h, root_dt, ctx->schedule, ctx->sched_chunk, want_tb ? 1 : 0,
                                      (int64_t)ctx->budget};
    if (key != ctx->sched_key || P.m < 0) {
        Plan np = choose_plan(ctx, m, n, h, root_dt, want_tb);
        if (!(P.m == m && P.n == n && P.h == h && P.root_dt == root_dt && P.depth_first == np.depth_first &&
              P.chunk == np.chunk)) {
            // Kernels of an earlier call may still read the old descriptors.
            LCS_CK(ctx, cudaDeviceSynchronize());
            ctx->plan = std::move(np);
            ctx->plan_uploaded = false;
        }
        ctx->sched_key = key;
    }
    lcs_status s = ensure_workspace(ctx, ctx->plan.total);
    if (s != LCS_OK) return s;
    if (!ctx->plan_uploaded) {
        Plan &Q = ctx->plan;
        char *base = ctx->ws;
        std::vector<StripOut> so = Q.h_strip_outs;
        for (auto &o : so) o.base = reloc(base, (char *)o.base);
        std::vector<MergeJob> jobs = Q.h_jobs;
        for (auto &j : jobs) {
            j.U = reloc(base, (const char *)j.U);
            j.L = reloc(base, (const char *)j.L);
            if (j.D) j.D = reloc(base, (char *)j.D);
            j.kgrid = reloc(base, j.kgrid);
            j.vgrid = reloc(base, j.vgrid);
        }
        std::vector<TbMerge> tb = Q.h_tb;
        for (auto &t : tb) {
            t.U = reloc(base, (const char *)t.U);
            t.L = reloc(base, (const char *)t.L);
            if (t.kgrid) t.kgrid = reloc(base, t.kgrid);
        }
        LCS_CK(ctx, cudaMemcpy(base + Q.off_strip_outs, so.data(), sizeof(StripOut) * so.size(),
                               cudaMemcpyHostToDevice));
        if (!Q.h_sweep.empty())
            LCS_CK(ctx, cudaMemcpy(base + Q.off_sweep, Q.h_sweep.data(), sizeof(SweepNode) * Q.h_sweep.size(),
                                   cudaMemcpyHostToDevice));
        if (!jobs.empty()) {
            LCS_CK(ctx, cudaMemcpy(base + Q.off_jobs, jobs.data(), sizeof(MergeJob) * jobs.size(),
                                   cudaMemcpyHostToDevice));
            LCS_CK(ctx, cudaMemcpy(base + Q.off_tb, tb.data(), sizeof(TbMerge) * tb.size(),
                                   cudaMemcpyHostToDevice));
        }
        if (!Q.h_chain.empty()) {
            LCS_CK(ctx, cudaMemcpy(base + Q.off_chain, Q.h_chain.data(), sizeof(int32_t) * Q.h_chain.size(),
                                   cudaMemcpyHostToDevice));
            LCS_CK(ctx, cudaMemcpy(base + Q.off_depth, Q.h_depth.data(), sizeof(int32_t) * Q.h_depth.size(),
                                   cudaMemcpyHostToDevice));
        }
        ctx->plan_uploaded = true;
        ++ctx->plan_gen;
    }
    return LCS_OK;
}

int *err_word(lcs_ctx *ctx) { return reinterpret_cast<int *>(ctx->ws); }
int64_t *len_word(lcs_ctx *ctx) { return reinterpret_cast<int64_t *>(ctx->ws + 8); }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

lcs_status check_dense(lcs_ctx *ctx, const void *p, int64_t n, int64_t ld, int dt, const char *name) {
    if (!p) return fail(ctx, LCS_EINVAL, std::string(name) + " is NULL");
    if (ld < n + 1) return fail(ctx, LCS_EINVAL, std::string(name) + ": ld < n+1");
    if ((ld * dt_size(dt)) % 16 != 0) return fail(ctx, LCS_EINVAL, std::string(name) + ": ld*size % 16 != 0");
    if (!aligned16(p)) return fail(ctx, LCS_EINVAL, std::string(name) + " is not 16-byte aligned");
    return LCS_OK;
}

int api_dt(lcs_dtype d) { return d == LCS_I16 ? DT_I16 : DT_I32; }

// The whole path with a depth-first plan.  The traceback needs only a and
// b (it recomputes the rows and columns of freed nodes), so it runs on a side
// stream from the start, beside the tree; the tree is built only when the
// DIST is wanted.
lcs_status solve_depth_first(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, int rdt,
                             void *dist, int64_t ld, uint8_t *out_lcs, int64_t cap, int32_t *cross,
                             int64_t *len_dev_out, bool want_tb, bool want_len, cudaStream_t st,
                             cudaEvent_t dist_ready, bool early_fill) {
    Plan &P = ctx->plan;
    char *base = ctx->ws;
    int *err = err_word(ctx);
    int32_t *pathI = reinterpret_cast<int32_t *>(base + P.off_path);
    int32_t *pathJ = pathI + P.nodes.size();
    int32_t *counts = reinterpret_cast<int32_t *>(base + P.off_counts);
    uint8_t *letters = reinterpret_cast<uint8_t *>(base + P.off_slots);
    bool tb_forked = false, fill_side = false;
    const int sentinel = rdt == DT_I16 ? INT16_MIN : INT32_MIN;

    // 1. traceback / length: root down, per depth a sweep pair and a pick.
    if (want_tb || want_len) {
        lcs_status ss = ensure_tb_side(ctx);
        if (ss != LCS_OK) return ss;
        LCS_CK(ctx, cudaEventRecord(ctx->ev_tb_fork, st));
        LCS_CK(ctx, cudaStreamWaitEvent(ctx->tb_side, ctx->ev_tb_fork, 0));
        cudaStream_t ts = ctx->tb_side;
        LCS_LAUNCHK(ctx, ts, K_TB, 0.0, 0.0, launch_root_path(pathI, pathJ, P.root, n, ts));
        const SweepNode *sweep = reinterpret_cast<const SweepNode *>(base + P.off_sweep);
        for (size_t d = 0; d < P.sweep_levels.size(); ++d) {
            SweepParams sp{};
            sp.nodes = sweep + P.sweep_levels[d].first;
            sp.count = P.sweep_levels[d].second;
            sp.root_node = P.root;
            sp.a = a; sp.b = b; sp.n = n;
            sp.pathI = pathI; sp.pathJ = pathJ;
            sp.fcnt = reinterpret_cast<int32_t *>(base + P.off_fcnt);
            sp.bcnt = reinterpret_cast<int32_t *>(base + P.off_bcnt);
            sp.len_out = d == 0 ? len_word(ctx) : nullptr;
            sp.err = err;
            LCS_LAUNCHK(ctx, ts, K_TB, 0.0, 0.0, launch_node_sweep(sp, P.sweep_rows[d], ts));
            LCS_LAUNCHK(ctx, ts, K_TB, 0.0, 0.0, launch_node_pick(sp, ts));
            if (!want_tb) break;               // the root's maximum is the length
        }
        if (want_tb || P.S == 1) {
            LeafParams lp{};
            lp.a = a; lp.m = m; lp.h = P.h; lp.S = P.S; lp.b = b; lp.n = n;
            lp.pathI = pathI; lp.pathJ = pathJ;
            lp.vbuf = reinterpret_cast<uint32_t *>(base + P.off_vbuf);
            lp.words = P.words; lp.slots = letters; lp.counts = counts; lp.cross = cross; lp.err = err;
            LCS_LAUNCHK(ctx, ts, K_LEAF, 0.0, 0.0, launch_leaf(lp, ts));
            CompactParams cp{};
            cp.slots = letters; cp.counts = counts; cp.S = P.S; cp.h = P.h;
            cp.out = out_lcs; cp.cap = cap; cp.len_out = len_word(ctx); cp.len_out2 = len_dev_out; cp.err = err;
            LCS_LAUNCHK(ctx, ts, K_COMPACT, 0.0, 0.0, launch_compact(cp, ts));
        } else if (len_dev_out) {
            LCS_CK(ctx, launch_copy_len(len_word(ctx), len_dev_out, ts));
        }
        LCS_CK(ctx, cudaEventRecord(ctx->ev_tb, ts));
        tb_forked = true;
    }

    // 2. the DIST tree, depth first.
    if (dist) {
        if (P.S == 1) {
            StripParams sp{};
            sp.a = a; sp.m = m; sp.h = P.h; sp.S = 1; sp.b = b; sp.n = n; sp.NT = P.NT;
            sp.outs = nullptr; sp.dense = dist; sp.ld = ld; sp.band_first = 0;
            LCS_LAUNCHK(ctx, st, K_STRIP, tri_entries(n) * dt_size(rdt), strip_ops(1, n, P.words),
                        launch_strip(sp, rdt, P.words, st));
            if (P.NT > 1)
                LCS_LAUNCHK(ctx, st, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                            launch_fill_dense(dist, rdt, n, ld, sentinel, 0, 0, nullptr, st));
        } else {
            if (early_fill) {
                lcs_status ss = ensure_root_side(ctx);
                if (ss != LCS_OK) return ss;
                int sms = 0;
                LCS_CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
                LCS_CK(ctx, cudaEventRecord(ctx->ev_fork, st));
                LCS_CK(ctx, cudaStreamWaitEvent(ctx->root_side, ctx->ev_fork, 0));
                LCS_LAUNCHK(ctx, ctx->root_side, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                            launch_fill_lower(dist, rdt, n, ld, sentinel, std::max(1, sms / 2), ctx->root_side));
                LCS_CK(ctx, cudaEventRecord(ctx->ev_root, ctx->root_side));
                fill_side = true;
            }
            unsigned int *counters = reinterpret_cast<unsigned int *>(base + P.off_counters);
            LCS_CK(ctx, cudaMemsetAsync(counters, 0, sizeof(unsigned) * std::max<size_t>(1, P.groups.size()), st));
            const StripOut *outs = reinterpret_cast<const StripOut *>(base + P.off_strip_outs);
            const int64_t sigma0 = coarse_sigma0(P.P);
            const int mk = ctx->merge_kernel != LCS_MERGE_AUTO ? ctx->merge_kernel
                           : (ctx->tuned_merge >= 0 ? ctx->tuned_merge : (int)LCS_MERGE_AUTO);
            for (const Step &stp : P.steps) {
                if (stp.strips) {
                    StripParams sp{};
                    sp.a = a + (int64_t)stp.begin * P.h;
                    sp.m = 0;
                    for (int q = stp.begin; q < stp.begin + stp.count; ++q) sp.m += P.nodes[q].rows;
                    sp.h = P.h; sp.S = stp.count; sp.b = b; sp.n = n; sp.NT = P.NT;
                    sp.outs = outs + stp.begin; sp.dense = nullptr; sp.ld = 0; sp.band_first = 0;
                    // The strips of a chunk share one dtype unless the last
                    // chunk's short strip feeds a different merge type.
                    bool same = true;
                    for (int q = stp.begin; q < stp.begin + stp.count; ++q)
                        if (P.nodes[q].dtype != P.nodes[stp.begin].dtype) same = false;
                    if (same) {
                        LCS_LAUNCHK(ctx, st, K_STRIP, stp.count * tri_entries(n) * dt_size(P.nodes[stp.begin].dtype),
                                    strip_ops(stp.count, n, P.words),
                                    launch_strip(sp, P.nodes[stp.begin].dtype, P.words, st));
                    } else {
                        for (int q = stp.begin; q < stp.begin + stp.count; ++q) {
                            StripParams one = sp;
                            one.a = a + (int64_t)q * P.h; one.m = P.nodes[q].rows; one.S = 1; one.outs = outs + q;
                            LCS_LAUNCHK(ctx, st, K_STRIP, tri_entries(n) * dt_size(P.nodes[q].dtype),
                                        strip_ops(1, n, P.words), launch_strip(one, P.nodes[q].dtype, P.words, st));
                        }
                    }
                    continue;
                }
                const Group &g = P.groups[stp.begin];
                MergeParams mp{};
                mp.jobs = reinterpret_cast<const MergeJob *>(base + P.off_jobs) + g.begin;
                mp.njobs = g.count;
                mp.n = n; mp.NT = P.NT; mp.P = P.P; mp.ld = ld; mp.err = err;
                    mp.dense_out = g.root ? dist : nullptr;
                mp.dense_K = nullptr;
                mp.const_tiles = 1;
                mp.wait_ns = ctx->wait_ns; mp.hold_band = ctx->hold_band;
                const int64_t sg0 = sigma0;
                mp.sigma = (int32_t)sg0; mp.full = 1;
                LCS_LAUNCHK(ctx, st, K_COARSE, 0.0, 0.0, launch_coarse(mp, g.in_dt, st));
                for (int64_t sg = sg0 / 2; sg >= 1; sg /= 2) {
                    mp.sigma = (int32_t)sg; mp.full = 0;
                    LCS_LAUNCHK(ctx, st, K_COARSE, 0.0, 0.0, launch_coarse(mp, g.in_dt, st));
                }
                const double bytes = g.count * tri_entries(n) * (2.0 * dt_size(g.in_dt) + dt_size(g.out_dt));
                if (P.dpx && mk != LCS_MERGE_EXACT) {
                    mp.sched = counters + stp.begin;
                    LCS_LAUNCHK(ctx, st, K_TILE, bytes, 0.0,
                                launch_tile_dpx(mp, g.out_dt, st));
                } else {
                    LCS_LAUNCHK(ctx, st, K_TILE, bytes, 0.0, launch_tile_pair(mp, g.in_dt, g.out_dt, st));
                    ctx->launches++;   // the pair is two kernel launches
                }
                if (g.root && !fill_side)
                    LCS_LAUNCHK(ctx, st, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                                launch_fill_dense(dist, rdt, n, ld, sentinel, 0, 0, nullptr, st));
            }
            if (fill_side) LCS_CK(ctx, cudaStreamWaitEvent(st, ctx->ev_root, 0));
        }
        if (dist_ready) LCS_CK(ctx, cudaEventRecord(dist_ready, st));
    }
    if (tb_forked) LCS_CK(ctx, cudaStreamWaitEvent(st, ctx->ev_tb, 0));   // join the traceback
    ctx->stats.strip_height = P.h;
    ctx->stats.strips = P.S;
    ctx->stats.merges = (int32_t)P.merges.size();
    ctx->stats.tree_levels = P.levels;
    ctx->stats.kernel_launches = ctx->launches;
    ctx->stats.tile = T;
    return LCS_OK;
}

// The whole hot path on device buffers (see lcs_solve in lcs.h).
// dist_ready (nullable): recorded once the dense DIST is complete, on the
// stream that completes it, before the traceback kernels that follow.
// early_fill: dist is pinned host memory; its lower triangle is filled on
// the side stream while the merge levels run.
lcs_status solve_device(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        lcs_dtype dtype, void *dist, int64_t ld, uint8_t *out_lcs, int64_t cap,
                        int32_t *cross, int64_t *len_dev_out, bool need_len, cudaStream_t st,
                        cudaEvent_t dist_ready = nullptr, bool early_fill = false) {
    ctx->launches = 0;
    const int rdt = api_dt(dtype);
    if (m < 0 || n < 0) return fail(ctx, LCS_EINVAL, "negative length");
    if (n >= INT32_MAX / 2 || m >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "length too large");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    if (dtype == LCS_I16 && (m >= 32768 || n >= 32768)) return fail(ctx, LCS_EINVAL, "LCS_I16 needs m, n < 32768");
    if (dist) {
        lcs_status s = check_dense(ctx, dist, n, ld, rdt, "dist");
        if (s != LCS_OK) return s;
    }
    if (out_lcs && cap < std::min(m, n)) return fail(ctx, LCS_EOVERFLOW, "cap < min(m, n)");
    if ((m > 0 && !a) || (n > 0 && !b)) return fail(ctx, LCS_EINVAL, "a or b is NULL");
    const bool want_tb = out_lcs || cross;
    const bool want_len = need_len || len_dev_out;
    bool forked = false;                 // the root merge group runs on ctx->root_side
    bool fill_side = false;              // the dense fill runs on ctx->root_side
    // The root group's tile launch, when it waits for the traceback levels.
    bool root_deferred = false;
    Group root_defer{};
    MergeParams root_defer_mp{};

    // Degenerate grids: no rows or no columns.
    if (m == 0 || n == 0) {
        lcs_status s = ensure_workspace(ctx, std::max(ctx->ws_bytes, kHeaderBytes));
        if (s != LCS_OK) return s;
        if (dist) {
            LCS_LAUNCHK(ctx, st, K_FILL, tri_entries(n) * dt_size(rdt), 0.0, launch_fill_dense(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 1,
                                              nullptr, st));
        }
        if (dist_ready) LCS_CK(ctx, cudaEventRecord(dist_ready, st));
        LCS_CK(ctx, cudaMemsetAsync(len_word(ctx), 0, sizeof(int64_t), st));
        if (len_dev_out) LCS_CK(ctx, cudaMemsetAsync(len_dev_out, 0, sizeof(int64_t), st));
        if (cross) {
            // v[r] = 0 for every row when n == 0; with m == 0 there is only v[0] = 0.
            LCS_CK(ctx, cudaMemsetAsync(cross, 0, sizeof(int32_t) * (m + 1), st));
        }
        ctx->stats.strips = 0; ctx->stats.merges = 0; ctx->stats.tree_levels = 0;
        ctx->stats.kernel_launches = ctx->launches;
        return LCS_OK;
    }

    lcs_status s = prepare(ctx, m, n, rdt, want_tb);
    if (s != LCS_OK) return s;
    Plan &P = ctx->plan;
    ctx->stats.depth_first = P.depth_first ? 1 : 0;
    ctx->stats.chunk_strips = P.depth_first ? P.chunk : P.S;
    ctx->stats.plan_bytes = (int64_t)P.total;
    if (P.depth_first)
        return solve_depth_first(ctx, a, m, b, n, rdt, dist, ld, out_lcs, cap, cross, len_dev_out, want_tb, want_len,
                                 st, dist_ready, early_fill);
    char *base = ctx->ws;
    int *err = err_word(ctx);
    int32_t *pathI = reinterpret_cast<int32_t *>(base + P.off_path);
    int32_t *pathJ = pathI + P.nodes.size();
    int32_t *counts = reinterpret_cast<int32_t *>(base + P.off_counts);
    uint8_t *slots = reinterpret_cast<uint8_t *>(base + P.off_slots);

    // DPX merge tile counters, one per tree level (zero at each launch).
    unsigned int *sched = reinterpret_cast<unsigned int *>(base + kSchedOffset);
    if (P.dpx && P.S > 1) LCS_CK(ctx, cudaMemsetAsync(sched, 0, kSchedSlots * sizeof(unsigned int), st));

    const int64_t sigma0 = coarse_sigma0(P.P);
    int dpx_launch = 0;
    const int mk = ctx->merge_kernel != LCS_MERGE_AUTO ? ctx->merge_kernel
                   : (ctx->tuned_merge >= 0 ? ctx->tuned_merge : (int)LCS_MERGE_AUTO);
    // A group's tile launch and, for the root, the dense fill and events.
    auto tiles = [&](const Group &g, MergeParams mp, cudaStream_t gs) -> lcs_status {
        if (P.dpx && mk != LCS_MERGE_EXACT) {
            // A zeroed work counter per launch (zeroed above, once per solve).
            mp.sched = dpx_launch < kSchedSlots ? sched + dpx_launch : nullptr;
            ++dpx_launch;
            LCS_LAUNCHK(ctx, gs, K_TILE, g.count * tri_entries(n) * (2.0 * dt_size(g.in_dt) + dt_size(g.out_dt)),
                        0.0, launch_tile_dpx(mp, g.out_dt, gs));
        } else {
            LCS_LAUNCHK(ctx, gs, K_TILE, g.count * tri_entries(n) * (2.0 * dt_size(g.in_dt) + dt_size(g.out_dt)),
                        0.0, launch_tile_pair(mp, g.in_dt, g.out_dt, gs));
            ctx->launches++;   // the pair is two kernel launches
        }
        if (g.root) {
            if (!fill_side) {
                LCS_LAUNCHK(ctx, gs, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                            launch_fill_dense(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 0,
                                              nullptr, gs));
            } else if (!forked) {
                // The early fill ran on the side stream: the DIST is
                // complete once it has (on the side stream it precedes
                // the root group anyway).
                LCS_CK(ctx, cudaStreamWaitEvent(st, ctx->ev_root, 0));
            }
            if (dist_ready) LCS_CK(ctx, cudaEventRecord(dist_ready, gs));
            if (forked) LCS_CK(ctx, cudaEventRecord(ctx->ev_root, gs));
        }
        return LCS_OK;
    };
    // 1. strips
    if (P.S == 1) {
        if (dist) {
            StripParams sp{};
            sp.a = a; sp.m = m; sp.h = P.h; sp.S = 1; sp.b = b; sp.n = n; sp.NT = P.NT;
            sp.outs = nullptr; sp.dense = dist; sp.ld = ld; sp.band_first = 0;
            LCS_LAUNCHK(ctx, st, K_STRIP, tri_entries(n) * dt_size(rdt), strip_ops(1, n, P.words), launch_strip(sp, rdt, P.words, st));
            if (P.NT > 1)
                LCS_LAUNCHK(ctx, st, K_FILL, tri_entries(n) * dt_size(rdt), 0.0, launch_fill_dense(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 0,
                                                  nullptr, st));
            if (dist_ready) LCS_CK(ctx, cudaEventRecord(dist_ready, st));
        }
    } else {
        // The dense DIST's lower triangle outside the diagonal tiles is
        // written by no merge tile.  When the DIST is pinned host memory
        // (early_fill), that fill crosses the CPU-GPU link, so it runs on the
        // side stream from the start, beside the strip builder and the merge
        // levels, instead of after the root; half the SMs get one block each.
        // A device DIST is filled after the root merge instead (a few
        // microseconds of HBM writes, where a concurrent fill measurably
        // slows the latency-bound strip builder).
        if (dist && early_fill) {
            lcs_status ss = ensure_root_side(ctx);
            if (ss != LCS_OK) return ss;
            int sms = 0;
            LCS_CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            LCS_CK(ctx, cudaEventRecord(ctx->ev_fork, st));
            LCS_CK(ctx, cudaStreamWaitEvent(ctx->root_side, ctx->ev_fork, 0));
            LCS_LAUNCHK(ctx, ctx->root_side, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                        launch_fill_lower(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN,
                                          std::max(1, sms / 2), ctx->root_side));
            LCS_CK(ctx, cudaEventRecord(ctx->ev_root, ctx->root_side));
            fill_side = true;
        }
        // All strips share one dtype here (heights <= h, h <= 256 -> u8/i16).
        StripParams sp{};
        sp.a = a; sp.m = m; sp.h = P.h; sp.S = P.S; sp.b = b; sp.n = n; sp.NT = P.NT;
        sp.outs = reinterpret_cast<const StripOut *>(base + P.off_strip_outs);
        sp.dense = nullptr; sp.ld = 0; sp.band_first = 0;
        // Strips feeding merges of different input types: launch per dtype.
        int dts[3] = {DT_U8, DT_I16, DT_I32};
        for (int dt : dts) {
            bool any = false, all = true;
            for (int q = 0; q < P.S; ++q) {
                if (P.nodes[q].dtype == dt) any = true; else all = false;
            }
            if (!any) continue;
            if (all) {
                LCS_LAUNCHK(ctx, st, K_STRIP, P.S * tri_entries(n) * dt_size(dt), strip_ops(P.S, n, P.words), launch_strip(sp, dt, P.words, st));
            } else {
                for (int q = 0; q < P.S; ++q) {
                    if (P.nodes[q].dtype != dt) continue;
                    StripParams one = sp;
                    one.a = a + (int64_t)q * P.h;
                    one.m = P.nodes[q].rows;
                    one.S = 1;
                    one.outs = sp.outs + q;
                    LCS_LAUNCHK(ctx, st, K_STRIP, tri_entries(n) * dt_size(dt), strip_ops(1, n, P.words), launch_strip(one, dt, P.words, st));
                }
            }
        }
        // A device DIST's lower triangle outside the diagonal tiles: filled on
        // the side stream once the strips are done, beside the merge levels
        // (bound by their (max,+) arithmetic, where the fill's HBM writes
        // cost little), instead of after the root merge.
        if (dist && !early_fill) {
            lcs_status ss = ensure_root_side(ctx);
            if (ss != LCS_OK) return ss;
            int sms = 0;
            LCS_CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            LCS_CK(ctx, cudaEventRecord(ctx->ev_fork, st));
            LCS_CK(ctx, cudaStreamWaitEvent(ctx->root_side, ctx->ev_fork, 0));
            LCS_LAUNCHK(ctx, ctx->root_side, K_FILL, tri_entries(n) * dt_size(rdt), 0.0,
                        launch_fill_lower(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN,
                                          std::max(1, sms / 4), ctx->root_side));
            LCS_CK(ctx, cudaEventRecord(ctx->ev_root, ctx->root_side));
            fill_side = true;
        }
        // 2. merges, level by level
        for (const Group &g : P.groups) {
            if (g.root && !dist) continue;
            // The root merge writes only the dense DIST, which the traceback
            // does not read (it reads the root's children): with a traceback
            // to run, the root group goes to a side stream and the traceback
            // overlaps it.
            cudaStream_t gs = st;
            if (g.root && want_tb) {
                lcs_status ss = ensure_root_side(ctx);
                if (ss != LCS_OK) return ss;
                LCS_CK(ctx, cudaEventRecord(ctx->ev_fork, st));
                LCS_CK(ctx, cudaStreamWaitEvent(ctx->root_side, ctx->ev_fork, 0));
                gs = ctx->root_side;
                forked = true;
            }
            MergeParams mp{};
            mp.jobs = reinterpret_cast<const MergeJob *>(base + P.off_jobs) + g.begin;
            mp.njobs = g.count;
            mp.n = n; mp.NT = P.NT; mp.P = P.P; mp.ld = ld; mp.err = err;
            mp.dense_out = g.root ? dist : nullptr;
            mp.dense_K = nullptr;
            mp.const_tiles = 1;
            mp.wait_ns = ctx->wait_ns; mp.hold_band = ctx->hold_band;
            const int64_t sg0 = sigma0;
            mp.sigma = (int32_t)sg0; mp.full = 1;
            LCS_LAUNCHK(ctx, gs, K_COARSE, 0.0, 0.0, launch_coarse(mp, g.in_dt, gs));
            for (int64_t sg = sg0 / 2; sg >= 1; sg /= 2) {
                mp.sigma = (int32_t)sg; mp.full = 0;
                LCS_LAUNCHK(ctx, gs, K_COARSE, 0.0, 0.0, launch_coarse(mp, g.in_dt, gs));
            }
            if (forked && g.root) {
                // The root's tile launch waits for the traceback's argmax
                // levels (below): its persistent grid fills every SM, and the
                // leaf kernel, launched first and at a higher priority, then
                // runs beside it instead of after it.
                root_defer = g;
                root_defer_mp = mp;
                root_deferred = true;
                continue;
            }
            lcs_status ss = tiles(g, mp, gs);
            if (ss != LCS_OK) return ss;
        }
    }

    // 3. traceback / length
    if (want_tb || (want_len && P.S == 1)) {
        const TbMerge *tbd = reinterpret_cast<const TbMerge *>(base + P.off_tb);
        if (P.S > 1) {
            // The splits above the leaves in one launch: a CTA per strip walks
            // from the root down to its strip.
            TbParams tp{};
            tp.merges = tbd; tp.count = (int32_t)P.merges.size();
            tp.n = n; tp.NT = P.NT; tp.pathI = pathI; tp.pathJ = pathJ;
            tp.len_out = nullptr; tp.root_node = P.root; tp.err = err;
            LCS_LAUNCHK(ctx, st, K_TB, 0.0, 0.0,
                        launch_tb_path(tp, reinterpret_cast<const int32_t *>(base + P.off_chain),
                                       reinterpret_cast<const int32_t *>(base + P.off_depth), P.depth_max, P.S, st));
        } else {
            LCS_LAUNCHK(ctx, st, K_TB, 0.0, 0.0, launch_root_path(pathI, pathJ, P.root, n, st));
        }
        if (root_deferred) {
            LCS_CK(ctx, cudaEventRecord(ctx->ev_tbl, st));
            LCS_CK(ctx, cudaStreamWaitEvent(ctx->root_side, ctx->ev_tbl, 0));
            lcs_status ss = tiles(root_defer, root_defer_mp, ctx->root_side);
            if (ss != LCS_OK) return ss;
        }
        LeafParams lp{};
        lp.a = a; lp.m = m; lp.h = P.h; lp.S = P.S; lp.b = b; lp.n = n;
        lp.pathI = pathI; lp.pathJ = pathJ;
        lp.vbuf = reinterpret_cast<uint32_t *>(base + P.off_vbuf);
        lp.words = P.words; lp.slots = slots; lp.counts = counts; lp.cross = cross; lp.err = err;
        LCS_LAUNCHK(ctx, st, K_LEAF, 0.0, 0.0, launch_leaf(lp, st, root_deferred ? ctx->leaf_priority : 0));
        CompactParams cp{};
        cp.slots = slots; cp.counts = counts; cp.S = P.S; cp.h = P.h;
        cp.out = out_lcs; cp.cap = cap; cp.len_out = len_word(ctx); cp.len_out2 = len_dev_out; cp.err = err;
        LCS_LAUNCHK(ctx, st, K_COMPACT, 0.0, 0.0, launch_compact(cp, st));
    } else if (want_len) {
        // Root maximum only: the first traceback level.
        LCS_LAUNCHK(ctx, st, K_TB, 0.0, 0.0, launch_root_path(pathI, pathJ, P.root, n, st));
        const TbMerge *tbd = reinterpret_cast<const TbMerge *>(base + P.off_tb);
        TbParams tp{};
        tp.merges = tbd + P.tb_levels[0].first; tp.count = P.tb_levels[0].second;
        tp.n = n; tp.NT = P.NT; tp.pathI = pathI; tp.pathJ = pathJ;
        tp.len_out = len_word(ctx); tp.root_node = P.root; tp.err = err;
        LCS_LAUNCHK(ctx, st, K_TB, 0.0, 0.0, launch_tb_level(tp, st));
        if (len_dev_out) LCS_CK(ctx, launch_copy_len(len_word(ctx), len_dev_out, st));
    }
    if (forked || fill_side) LCS_CK(ctx, cudaStreamWaitEvent(st, ctx->ev_root, 0));   // join the side stream
    ctx->stats.strip_height = P.h;
    ctx->stats.strips = P.S;
    ctx->stats.merges = (int32_t)P.merges.size();
    ctx->stats.tree_levels = P.levels;
    ctx->stats.kernel_launches = ctx->launches;
    ctx->stats.tile = T;
    return LCS_OK;
}

// Synchronise and read the error and length words (one 16-byte copy).
lcs_status read_back(lcs_ctx *ctx, cudaStream_t st, int64_t *len_host) {
    int64_t hdr[2] = {0, 0};
    LCS_CK(ctx, cudaMemcpyAsync(hdr, ctx->ws, 16, cudaMemcpyDeviceToHost, st));
    LCS_CK(ctx, cudaStreamSynchronize(st));
    const int errbits = (int)(hdr[0] & 0xFFFFFFFF);
    if (errbits) {
        LCS_CK(ctx, cudaMemset(ctx->ws, 0, 4));
        if (errbits & ERR_TIMEOUT) return fail(ctx, LCS_ETIMEOUT, "a device-side wait timed out");
        if (errbits & ERR_OVERFLOW) return fail(ctx, LCS_EOVERFLOW, "a value or the output exceeded its capacity");
        return fail(ctx, LCS_ECUDA, "device-side consistency check failed");
    }
    if (len_host) *len_host = hdr[1];
    return LCS_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

lcs_status lcs_create(lcs_ctx **out, int device, size_t mem_budget_bytes) {
    if (!out) return LCS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return LCS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return LCS_ECUDA;
    lcs_ctx *ctx = new (std::nothrow) lcs_ctx();
    if (!ctx) return LCS_ENOMEM;
    ctx->device = device;
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : kDefaultBudget;
    *out = ctx;
    return LCS_OK;
}

lcs_status lcs_destroy(lcs_ctx *ctx) {
    if (!ctx) return LCS_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->io) cudaFree(ctx->io);
    for (auto &kv : ctx->tickets) {
        BatchTicket &t = kv.second;
        if (t.dev) cudaFreeAsync(t.dev, t.lane.stream);
        cudaStreamSynchronize(t.lane.stream);
        destroy_lane(t.lane);
    }
    for (auto &l : ctx->free_lanes) destroy_lane(l);
    if (ctx->mempool) cudaMemPoolDestroy(ctx->mempool);
    for (auto &r : ctx->recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->root_side) cudaStreamDestroy(ctx->root_side);
    if (ctx->ev_tbl) cudaEventDestroy(ctx->ev_tbl);
    if (ctx->tb_side) cudaStreamDestroy(ctx->tb_side);
    if (ctx->ev_tb_fork) cudaEventDestroy(ctx->ev_tb_fork);
    if (ctx->ev_tb) cudaEventDestroy(ctx->ev_tb);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_root) cudaEventDestroy(ctx->ev_root);
    if (ctx->ev_dist) cudaEventDestroy(ctx->ev_dist);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->host_hdr) cudaFreeHost(ctx->host_hdr);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return LCS_OK;
}

const char *lcs_strerror(lcs_status s) {
    switch (s) {
        case LCS_OK: return "ok";
        case LCS_EINVAL: return "invalid argument";
        case LCS_ENOMEM: return "out of memory (workspace budget or device)";
        case LCS_ETIMEOUT: return "device-side wait timed out";
        case LCS_ECUDA: return "CUDA error";
        case LCS_EAGAIN: return "try again";
        case LCS_EOVERFLOW: return "value or output exceeds its capacity";
    }
    return "unknown status";
}

const char *lcs_last_error(lcs_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

lcs_status lcs_set_strip_height(lcs_ctx *ctx, int32_t h) {
    if (!ctx || h < 0 || h > 256) return fail(ctx, LCS_EINVAL, "strip height must be 0..256");
    ctx->strip_h = h;
    return LCS_OK;
}

lcs_status lcs_set_merge_kernel(lcs_ctx *ctx, int32_t kind) {
    if (!ctx || kind < LCS_MERGE_AUTO || kind > LCS_MERGE_DPX) return fail(ctx, LCS_EINVAL, "unknown merge kernel");
    ctx->merge_kernel = kind;
    return LCS_OK;
}

lcs_status lcs_set_schedule(lcs_ctx *ctx, int32_t mode, int32_t chunk) {
    if (!ctx || mode < LCS_SCHED_AUTO || mode > LCS_SCHED_DEPTH || chunk < 0)
        return fail(ctx, LCS_EINVAL, "schedule arguments");
    ctx->schedule = mode;
    ctx->sched_chunk = chunk;
    return LCS_OK;
}

lcs_status lcs_plan(int64_t m, int64_t n, int32_t h, int32_t schedule, int32_t chunk, size_t budget_bytes,
                    int32_t want_lcs, lcs_dtype root_dtype, lcs_plan_info *info, lcs_plan_node *nodes,
                    int64_t cap) {
    if (!info || m < 0 || n < 0 || h < 0 || h > 256 || schedule < LCS_SCHED_AUTO || schedule > LCS_SCHED_DEPTH ||
        chunk < 0 || cap < 0 || (cap > 0 && !nodes))
        return LCS_EINVAL;
    if (n >= INT32_MAX / 2 || m >= INT32_MAX / 2) return LCS_EINVAL;
    if (root_dtype != LCS_I32 && root_dtype != LCS_I16) return LCS_EINVAL;
    if (root_dtype == LCS_I16 && (m >= 32768 || n >= 32768)) return LCS_EINVAL;
    *info = lcs_plan_info{};
    info->tile = T;
    info->root = -1;
    const size_t budget = budget_bytes ? budget_bytes : kDefaultBudget;
    if (m == 0 || n == 0) {
        // No tree: the solve writes the degenerate DIST and length directly.
        info->workspace_bytes = (int64_t)kHeaderBytes;
        info->fits = kHeaderBytes <= budget ? 1 : 0;
        return LCS_OK;
    }
    const int rdt = api_dt(root_dtype);
    if (h == 0) h = auto_strip_height(m, n);
    const Plan P = pick_plan(schedule, chunk, budget, m, n, h, rdt, want_lcs != 0);
    // Launches in stream order: the retained tree builds every strip in one
    // launch and then launches each merge group; the depth-first plan runs
    // its steps.
    std::vector<int32_t> made(P.nodes.size(), -1), last(P.nodes.size(), -1);
    int32_t launches = 0;
    auto group_launch = [&](const Group &g, int32_t L) {
        for (int q = g.begin; q < g.begin + g.count; ++q) {
            const Merge &mg = P.merges[q];
            made[mg.out] = L;
            last[mg.u] = L;
            last[mg.l] = L;
        }
    };
    if (P.depth_first) {
        for (const Step &st : P.steps) {
            if (st.strips) {
                for (int s = st.begin; s < st.begin + st.count; ++s) made[s] = launches;
            } else {
                group_launch(P.groups[st.begin], launches);
            }
            ++launches;
        }
    } else {
        for (int s = 0; s < P.S; ++s) made[s] = 0;
        launches = 1;
        for (const Group &g : P.groups) group_launch(g, launches++);
        for (auto &x : last) x = launches;   // every node is kept for the traceback
    }
    if (P.root >= 0) last[P.root] = launches;
    info->workspace_bytes = (int64_t)P.total;
    info->fits = P.total <= budget ? 1 : 0;
    info->strip_height = P.h;
    info->strips = P.S;
    info->nodes = (int32_t)P.nodes.size();
    info->levels = P.levels;
    info->depth_first = P.depth_first ? 1 : 0;
    info->chunk = P.depth_first ? P.chunk : P.S;
    info->launches = launches;
    info->root = P.root;
    const int64_t count = std::min<int64_t>(cap, (int64_t)P.nodes.size());
    for (int64_t v = 0; v < count; ++v) {
        const Node &nd = P.nodes[v];
        lcs_plan_node r{};
        r.row0 = nd.row0;
        r.rows = nd.rows;
        r.offset = nd.root ? 0 : (int64_t)nd.off;
        r.bytes = nd.root ? 0 : (int64_t)nd.bytes;
        r.upper = r.lower = -1;
        r.parent = nd.parent;
        r.level = nd.level;
        r.made_by = made[v];
        r.last_use = last[v];
        r.grid_last_use = -1;
        nodes[v] = r;
    }
    const int64_t grid_bytes = 2 * (int64_t)(P.P + 1) * (P.P + 1) * 4;   // argmax grid, then value grid
    for (const Merge &mg : P.merges) {
        if (mg.out >= count) continue;
        lcs_plan_node &r = nodes[mg.out];
        r.upper = mg.u;
        r.lower = mg.l;
        r.grid_offset = (int64_t)mg.kgrid_off;
        r.grid_bytes = grid_bytes;
        r.grid_last_use = P.depth_first ? made[mg.out] : launches;
    }
    return LCS_OK;
}

lcs_status lcs_set_fault_injection(lcs_ctx *ctx, int32_t hold_band, int64_t wait_limit_ns) {
    if (!ctx || wait_limit_ns < 0) return fail(ctx, LCS_EINVAL, "fault injection arguments");
    ctx->hold_band = hold_band ? 1 : 0;
    ctx->wait_ns = (uint64_t)wait_limit_ns;
    ctx->gkey.clear();           // a captured solve holds the old launch parameters
    return LCS_OK;
}

lcs_status lcs_set_graphs(lcs_ctx *ctx, int32_t enable) {
    if (!ctx) return LCS_EINVAL;
    ctx->graphs = enable != 0;
    if (!ctx->graphs && ctx->gexec) {
        LCS_CK(ctx, cudaSetDevice(ctx->device));
        LCS_CK(ctx, cudaDeviceSynchronize());
        LCS_CK(ctx, cudaGraphExecDestroy(ctx->gexec));
        ctx->gexec = nullptr;
        ctx->gkey.clear();
    }
    return LCS_OK;
}

lcs_status lcs_autotune(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, lcs_dtype dtype,
                        void *dist, int64_t ld, uint8_t *out_lcs, int64_t cap, void *stream,
                        int32_t *h_out, int32_t *merge_out, float *ms_out) {
    if (!ctx) return LCS_EINVAL;
    if (m <= 0 || n <= 0) return fail(ctx, LCS_EINVAL, "autotune needs m, n > 0");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int root_dt = api_dt(dtype);
    const std::vector<int64_t> key = tune_key(m, n, root_dt);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(ctx, LCS_ECUDA, cudaGetErrorString(cudaGetLastError()));
    }
    const int32_t keep_h = ctx->strip_h, keep_mk = ctx->merge_kernel;
    const bool keep_prof = ctx->profiling, keep_graphs = ctx->graphs;
    ctx->profiling = false;
    ctx->graphs = false;
    ctx->tuned.erase(key);
    float best_ms = -1.0f;
    int32_t best_h = 0, best_mk = LCS_MERGE_AUTO;
    lcs_status s = LCS_OK;
    const int32_t hs[3] = {64, 128, 256};
    const int32_t mks[2] = {LCS_MERGE_DPX, LCS_MERGE_EXACT};
    for (int32_t h : hs) {
        if (h > m && h != hs[0]) continue;          // taller than the pair: same plan as a shorter h
        for (int32_t mk : mks) {
            ctx->strip_h = std::min<int64_t>(h, m);
            ctx->merge_kernel = mk;
            s = solve_device(ctx, a, m, b, n, dtype, dist, ld, out_lcs, cap, nullptr, nullptr, true, st);
            if (s == LCS_ENOMEM) { s = LCS_OK; continue; }      // does not fit the budget: not a candidate
            if (s != LCS_OK) break;
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && s == LCS_OK; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) { s = LCS_ECUDA; break; }
                s = solve_device(ctx, a, m, b, n, dtype, dist, ld, out_lcs, cap, nullptr, nullptr, true, st);
                if (s != LCS_OK) break;
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { s = LCS_ECUDA; break; }
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                ms = std::min(ms, t);
            }
            if (s != LCS_OK) break;
            if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; best_h = ctx->strip_h; best_mk = mk; }
            if (!ctx->plan.dpx) break;               // the plan has no DPX merge: one kernel to time
        }
        if (s != LCS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->strip_h = keep_h;
    ctx->merge_kernel = keep_mk;
    ctx->profiling = keep_prof;
    ctx->graphs = keep_graphs;
    if (s != LCS_OK) return s;
    if (best_ms < 0.0f) return fail(ctx, LCS_ENOMEM, "no strip height fits the budget");
    ctx->tuned[key] = {best_h, best_mk};
    ++ctx->tune_gen;
    if (h_out) *h_out = best_h;
    if (merge_out) *merge_out = best_mk;
    if (ms_out) *ms_out = best_ms;
    return read_back(ctx, st, nullptr);
}

lcs_status lcs_get_stats(lcs_ctx *ctx, lcs_stats *out) {
    if (!ctx || !out) return LCS_EINVAL;
    ctx->stats.workspace_bytes = (int64_t)(ctx->ws_bytes + ctx->io_bytes);
    ctx->stats.peak_workspace_bytes = (int64_t)ctx->peak;
    *out = ctx->stats;
    return LCS_OK;
}

lcs_status lcs_set_profiling(lcs_ctx *ctx, int32_t enable) {
    if (!ctx) return LCS_EINVAL;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    LCS_CK(ctx, cudaDeviceSynchronize());
    for (auto &r : ctx->recs) { ctx->pool.push_back(r.e0); ctx->pool.push_back(r.e1); }
    ctx->recs.clear();
    ctx->profiling = enable != 0;
    return LCS_OK;
}

lcs_status lcs_get_profile(lcs_ctx *ctx, lcs_kernel_profile *out, int32_t cap, int32_t *count) {
    if (!ctx || !count || (cap > 0 && !out)) return LCS_EINVAL;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    LCS_CK(ctx, cudaDeviceSynchronize());
    lcs_kernel_profile acc[K_KINDS];
    for (int k = 0; k < K_KINDS; ++k) acc[k] = lcs_kernel_profile{k, 0, 0.0, 0.0, 0.0};
    for (auto &r : ctx->recs) {
        float ms = 0.f;
        LCS_CK(ctx, cudaEventElapsedTime(&ms, r.e0, r.e1));
        acc[r.kind].launches += 1;
        acc[r.kind].ms += ms;
        acc[r.kind].bytes += r.bytes;
        acc[r.kind].ops += r.ops;
        ctx->pool.push_back(r.e0);
        ctx->pool.push_back(r.e1);
    }
    ctx->recs.clear();
    int c = 0;
    for (int k = 0; k < K_KINDS; ++k)
        if (acc[k].launches > 0 && c < cap) out[c++] = acc[k];
    *count = c;
    return LCS_OK;
}

lcs_status lcs_sync(lcs_ctx *ctx, void *stream) {
    if (!ctx) return LCS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->ws) {
        LCS_CK(ctx, cudaStreamSynchronize(st));
        return LCS_OK;
    }
    return read_back(ctx, st, nullptr);
}

lcs_status lcs_strip_dist(lcs_ctx *ctx, const uint8_t *a_strip, int32_t h, const uint8_t *b, int64_t n,
                          lcs_dtype dtype, void *dist, int64_t ld, void *stream) {
    if (!ctx) return LCS_EINVAL;
    ctx->launches = 0;
    if (h < 1 || h > 256) return fail(ctx, LCS_EINVAL, "h must be 1..256");
    if (n < 0 || n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "n out of range");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    if (dtype == LCS_I16 && n >= 32768) return fail(ctx, LCS_EINVAL, "LCS_I16 needs n < 32768");
    if (!a_strip || (n > 0 && !b)) return fail(ctx, LCS_EINVAL, "a_strip or b is NULL");
    const int rdt = api_dt(dtype);
    lcs_status s = check_dense(ctx, dist, n, ld, rdt, "dist");
    if (s != LCS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    StripParams sp{};
    sp.a = a_strip; sp.m = h; sp.h = h; sp.S = 1; sp.b = b; sp.n = n; sp.NT = num_tiles_side(n);
    sp.outs = nullptr; sp.dense = dist; sp.ld = ld; sp.band_first = 0;
    LCS_LAUNCHK(ctx, st, K_STRIP, tri_entries(n) * dt_size(rdt), strip_ops(1, n, words_for(h)), launch_strip(sp, rdt, words_for(h), st));
    if (sp.NT > 1)
        LCS_LAUNCHK(ctx, st, K_FILL, tri_entries(n) * dt_size(rdt), 0.0, launch_fill_dense(dist, rdt, n, ld, rdt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 0, nullptr, st));
    ctx->stats.kernel_launches = ctx->launches;
    return LCS_OK;
}

lcs_status lcs_strip_dform(lcs_ctx *ctx, const uint8_t *a, int64_t m, int32_t h, const uint8_t *b, int64_t n,
                           lcs_dtype dtype, void *dform, int64_t ldf, void *stream) {
    if (!ctx) return LCS_EINVAL;
    ctx->launches = 0;
    if (h < 1 || h > 256) return fail(ctx, LCS_EINVAL, "h must be 1..256");
    if (m < 1 || ceil_div(m, h) > 65535) return fail(ctx, LCS_EINVAL, "m must be 1 .. 65535 h");
    if (n < 0 || n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "n out of range");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    if (dtype == LCS_I16 && n >= INT16_MAX) return fail(ctx, LCS_EINVAL, "LCS_I16 needs n < 32767");
    if (!a || (n > 0 && !b) || !dform) return fail(ctx, LCS_EINVAL, "a, b or dform is NULL");
    if (ldf < h + 1) return fail(ctx, LCS_EINVAL, "ldf < h+1");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    DformStripParams dp{};
    dp.a = a; dp.m = m; dp.h = h; dp.b = b; dp.n = n; dp.out = dform; dp.ld = ldf;
    LCS_LAUNCHK(ctx, st, K_STRIP, (double)ceil_div(m, h) * (n + 1) * (h + 1) * dt_size(api_dt(dtype)), 0.0,
                launch_dform_strip(dp, api_dt(dtype), words_for(h), st));
    ctx->stats.kernel_launches = ctx->launches;
    return LCS_OK;
}

lcs_status lcs_dform_merge(lcs_ctx *ctx, const void *du, int32_t hu, int64_t ldu, const void *dl, int32_t hl,
                           int64_t ldl, int64_t n, lcs_dtype dtype, void *out, int64_t ldo, void *stream) {
    if (!ctx) return LCS_EINVAL;
    ctx->launches = 0;
    if (hu < 0 || hl < 0 || hu + hl > 16384) return fail(ctx, LCS_EINVAL, "hu, hl must be >= 0 with hu + hl <= 16384");
    if (n < 0 || n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "n out of range");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    if (dtype == LCS_I16 && n >= INT16_MAX) return fail(ctx, LCS_EINVAL, "LCS_I16 needs n < 32767");
    if (!du || !dl || !out) return fail(ctx, LCS_EINVAL, "du, dl or out is NULL");
    if (ldu < hu + 1 || ldl < hl + 1 || ldo < hu + hl + 1) return fail(ctx, LCS_EINVAL, "leading dimension too small");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    DformMergeParams mp{};
    mp.du = du; mp.dl = dl; mp.ldu = ldu; mp.ldl = ldl; mp.hu = hu; mp.hl = hl; mp.n = n; mp.out = out; mp.ldo = ldo;
    LCS_LAUNCHK(ctx, st, K_TILE, (double)(n + 1) * (2 * hu + hl + 2) * dt_size(api_dt(dtype)), 0.0,
                launch_dform_merge(mp, api_dt(dtype), st));
    ctx->stats.kernel_launches = ctx->launches;
    return LCS_OK;
}

lcs_status lcs_merge(lcs_ctx *ctx, const void *dist_u, const void *dist_l, int64_t n, lcs_dtype dtype,
                     int64_t ld, void *dist_out, int32_t *argmax_out, void *stream) {
    if (!ctx) return LCS_EINVAL;
    ctx->launches = 0;
    if (n < 0 || n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "n out of range");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    const int dt = api_dt(dtype);
    lcs_status s;
    if ((s = check_dense(ctx, dist_u, n, ld, dt, "dist_u")) != LCS_OK) return s;
    if ((s = check_dense(ctx, dist_l, n, ld, dt, "dist_l")) != LCS_OK) return s;
    if ((s = check_dense(ctx, dist_out, n, ld, dt, "dist_out")) != LCS_OK) return s;
    if (argmax_out && !aligned16(argmax_out)) return fail(ctx, LCS_EINVAL, "argmax_out is not 16-byte aligned");
    if (dist_out == dist_u || dist_out == dist_l) return fail(ctx, LCS_EINVAL, "dist_out aliases an input");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t NT = num_tiles_side(n), P = ceil_div(n, T);
    const size_t packed = align256((size_t)num_tiles_tri(NT) * tile_elems(dt) * dt_size(dt));
    const size_t kg = align256(2 * (size_t)(P + 1) * (P + 1) * 4);   // kgrid + vgrid
    const size_t need = kHeaderBytes + 2 * packed + kg + align256(sizeof(MergeJob));
    if ((s = ensure_workspace(ctx, std::max(ctx->ws_bytes, kHeaderBytes))) != LCS_OK) return s;
    if ((s = ensure_io(ctx, need)) != LCS_OK) return s;
    char *io = ctx->io;
    char *Up = io + kHeaderBytes, *Lp = Up + packed;
    int32_t *kgrid = reinterpret_cast<int32_t *>(Lp + packed);
    MergeJob *jobd = reinterpret_cast<MergeJob *>(Lp + packed + kg);
    LCS_LAUNCHK(ctx, st, K_FILL, 0.0, 0.0, launch_pack(dist_u, dt, n, ld, Up, LAYOUT_ROW, st));
    LCS_LAUNCHK(ctx, st, K_FILL, 0.0, 0.0, launch_pack(dist_l, dt, n, ld, Lp, LAYOUT_COL, st));
    MergeJob job{};
    job.U = Up; job.L = Lp; job.D = nullptr; job.kgrid = kgrid; job.d_layout = LAYOUT_DENSE;
    job.vgrid = kgrid + (P + 1) * (P + 1);
    LCS_CK(ctx, cudaMemcpyAsync(jobd, &job, sizeof(job), cudaMemcpyHostToDevice, st));
    MergeParams mp{};
    mp.jobs = jobd; mp.njobs = 1;
    mp.n = n; mp.NT = NT; mp.P = P; mp.ld = ld; mp.err = err_word(ctx);
    mp.dense_out = dist_out; mp.dense_K = argmax_out;
    mp.const_tiles = argmax_out ? 0 : 1;      // a constant tile has no argmax to report
    mp.wait_ns = ctx->wait_ns; mp.hold_band = ctx->hold_band;
    const int64_t sigma0 = coarse_sigma0(std::max<int64_t>(P, 1));
    mp.sigma = (int32_t)sigma0; mp.full = 1;
    LCS_LAUNCHK(ctx, st, K_COARSE, 0.0, 0.0, launch_coarse(mp, dt, st));
    for (int64_t sg = sigma0 / 2; sg >= 1; sg /= 2) {
        mp.sigma = (int32_t)sg; mp.full = 0;
        LCS_LAUNCHK(ctx, st, K_COARSE, 0.0, 0.0, launch_coarse(mp, dt, st));
    }
    LCS_LAUNCHK(ctx, st, K_TILE, tri_entries(n) * 3.0 * dt_size(dt), 0.0, launch_tile_pair(mp, dt, dt, st));
    ctx->launches++;
    LCS_LAUNCHK(ctx, st, K_FILL, 0.0, 0.0, launch_fill_dense(dist_out, dt, n, ld, dt == DT_I16 ? INT16_MIN : INT32_MIN, 0, 0, argmax_out, st));
    // The job descriptor lives on the host stack: make sure the copy is done.
    LCS_CK(ctx, cudaStreamSynchronize(st));
    ctx->stats.kernel_launches = ctx->launches;
    return LCS_OK;
}

lcs_status lcs_solve(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, lcs_dtype dtype,
                     void *dist, int64_t ld, uint8_t *out_lcs, int64_t cap, int32_t *cross,
                     int64_t *out_len_device, void *stream) {
    if (!ctx) return LCS_EINVAL;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->graphs || ctx->profiling || m == 0 || n == 0)
        return solve_device(ctx, a, m, b, n, dtype, dist, ld, out_lcs, cap, cross, out_len_device, false, st);
    // Graph replay: the launch sequence depends only on the arguments and on
    // the plan state (strip height, merge kernel, workspace), so a solve with
    // the same key replays the captured graph.
    std::vector<int64_t> key = {(int64_t)(uintptr_t)a, m, (int64_t)(uintptr_t)b, n, (int64_t)dtype,
                                (int64_t)(uintptr_t)dist, ld, (int64_t)(uintptr_t)out_lcs, cap,
                                (int64_t)(uintptr_t)cross, (int64_t)(uintptr_t)out_len_device,
                                ctx->strip_h, ctx->merge_kernel, ctx->tune_gen, ctx->schedule, ctx->sched_chunk};
    // The captured kernels read the plan's descriptors from the workspace:
    // a graph stays valid only while that copy of the plan is the one it
    // was captured with.
    auto with_plan = [&](std::vector<int64_t> k) {
        k.push_back((int64_t)(uintptr_t)ctx->ws);
        k.push_back(ctx->plan_gen);
        return k;
    };
    if (ctx->gexec && ctx->gkey == with_plan(key)) {
        LCS_CK(ctx, cudaGraphLaunch(ctx->gexec, st));
        ctx->launches = ctx->glaunches;
        ctx->stats.kernel_launches = ctx->glaunches;
        return LCS_OK;
    }
    // Miss: run eagerly (this prepares the plan and workspace, so the
    // capture below makes no allocation or synchronous copy), then capture
    // the same solve on the private stream for the next calls.
    lcs_status s = solve_device(ctx, a, m, b, n, dtype, dist, ld, out_lcs, cap, cross, out_len_device, false, st);
    if (s != LCS_OK) return s;
    if (!ctx->cap_stream) LCS_CK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (ctx->gexec) {
        LCS_CK(ctx, cudaGraphExecDestroy(ctx->gexec));
        ctx->gexec = nullptr;
    }
    const lcs_stats keep = ctx->stats;
    const std::vector<int64_t> full = with_plan(key);
    LCS_CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    s = solve_device(ctx, a, m, b, n, dtype, dist, ld, out_lcs, cap, cross, out_len_device, false, ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (s != LCS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (ec != cudaSuccess) return cuda_fail(ctx, ec, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        ctx->gexec = nullptr;
        return cuda_fail(ctx, ei, "cudaGraphInstantiate");
    }
    ctx->gkey = full;
    ctx->glaunches = ctx->launches;
    ctx->stats = keep;
    return LCS_OK;
}

lcs_status lcs_dist(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, lcs_dtype dtype,
                    void *dist, int64_t ld, void *stream) {
    if (!ctx) return LCS_EINVAL;
    if (!dist) return fail(ctx, LCS_EINVAL, "dist is NULL");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    return solve_device(ctx, a, m, b, n, dtype, dist, ld, nullptr, 0, nullptr, nullptr, false,
                        (cudaStream_t)stream);
}

lcs_status lcs_length(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                      int64_t *out_len_host, void *stream) {
    if (!ctx) return LCS_EINVAL;
    if (!out_len_host) return fail(ctx, LCS_EINVAL, "out_len_host is NULL");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    lcs_status s = solve_device(ctx, a, m, b, n, LCS_I32, nullptr, 0, nullptr, 0, nullptr, nullptr, true, st);
    if (s != LCS_OK) return s;
    return read_back(ctx, st, out_len_host);
}

lcs_status lcs_traceback(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         uint8_t *out_lcs, int64_t cap, int64_t *out_len_host, void *stream) {
    if (!ctx) return LCS_EINVAL;
    if (!out_lcs || !out_len_host) return fail(ctx, LCS_EINVAL, "out_lcs or out_len_host is NULL");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    lcs_status s = solve_device(ctx, a, m, b, n, LCS_I32, nullptr, 0, out_lcs, cap, nullptr, nullptr, true, st);
    if (s != LCS_OK) return s;
    return read_back(ctx, st, out_len_host);
}

lcs_status lcs_path(lcs_ctx *ctx, const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int32_t *path, int64_t cap, int64_t *out_count_host, void *stream) {
    if (!ctx) return LCS_EINVAL;
    if (!out_count_host) return fail(ctx, LCS_EINVAL, "out_count_host is NULL");
    if (cap < 0 || (cap > 0 && !path)) return fail(ctx, LCS_EINVAL, "path is NULL or cap < 0");
    if (m < 0 || n < 0 || m >= INT32_MAX / 2 || n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "length");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // Staging: cross vertices, run offsets, the vertex count.
    const size_t rows_b = align256((size_t)(m + 1) * sizeof(int32_t));
    lcs_status s = ensure_io(ctx, 2 * rows_b + 256);
    if (s != LCS_OK) return s;
    int32_t *cross = reinterpret_cast<int32_t *>(ctx->io);
    int32_t *offs = reinterpret_cast<int32_t *>(ctx->io + rows_b);
    int64_t *cnt = reinterpret_cast<int64_t *>(ctx->io + 2 * rows_b);
    s = solve_device(ctx, a, m, b, n, LCS_I32, nullptr, 0, nullptr, 0, cross, nullptr, true, st);
    if (s != LCS_OK) return s;
    PathParams pp{};
    pp.a = a; pp.b = b; pp.m = m; pp.n = n; pp.cross = cross; pp.offsets = offs;
    pp.path = path; pp.cap = cap; pp.len = len_word(ctx); pp.count_out = cnt; pp.err = err_word(ctx);
    LCS_LAUNCHK(ctx, st, K_COMPACT, 0.0, 0.0, launch_path(pp, st));
    ctx->stats.kernel_launches = ctx->launches;
    int64_t len = 0;
    s = read_back(ctx, st, &len);
    if (s != LCS_OK) return s;
    *out_count_host = m + n + 1 - len;
    return LCS_OK;
}

lcs_status lcs_solve_host(lcs_ctx *ctx, const uint8_t *a_host, int64_t m, const uint8_t *b_host, int64_t n,
                          lcs_dtype dtype, void *dist_host, int64_t ld, uint8_t *lcs_host, int64_t cap,
                          int64_t *out_len_host, void *stream) {
    if (!ctx) return LCS_EINVAL;
    if (!out_len_host) return fail(ctx, LCS_EINVAL, "out_len_host is NULL");
    if (m < 0 || n < 0) return fail(ctx, LCS_EINVAL, "negative length");
    if ((m > 0 && !a_host) || (n > 0 && !b_host)) return fail(ctx, LCS_EINVAL, "a_host or b_host is NULL");
    if (dtype != LCS_I32 && dtype != LCS_I16) return fail(ctx, LCS_EINVAL, "dtype");
    if (dist_host && ld < n + 1) return fail(ctx, LCS_EINVAL, "ld < n+1");
    if (lcs_host && cap < std::min(m, n)) return fail(ctx, LCS_EOVERFLOW, "cap < min(m, n)");
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int rdt = api_dt(dtype);
    // Pinned host memory the device can address: the root merge writes the
    // dense DIST straight into it (over the CPU-GPU link, beside the
    // traceback), with no staging copy.  Anything else (pageable memory,
    // rows not 16-byte aligned) goes through device staging and a copy.
    void *direct = nullptr;
    if (dist_host) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, dist_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer && aligned16(pa.devicePointer) && (ld * dt_size(rdt)) % 16 == 0)
            direct = pa.devicePointer;
        else
            (void)cudaGetLastError();
    }
    const bool staged = dist_host && !direct;
    const int64_t ldd = staged ? ((n + 1) * dt_size(rdt) + 15) / 16 * 16 / dt_size(rdt) : (direct ? ld : 0);
    const size_t dist_bytes = staged ? align256((size_t)(n + 1) * ldd * dt_size(rdt)) : 0;
    const size_t a_off = 0, b_off = align256((size_t)m), l_off = b_off + align256((size_t)n);
    const size_t d_off = l_off + align256((size_t)std::max<int64_t>(cap, 1));
    lcs_status s = ensure_io(ctx, d_off + dist_bytes + 256);
    if (s != LCS_OK) return s;
    char *io = ctx->io;
    if (m) LCS_CK(ctx, cudaMemcpyAsync(io + a_off, a_host, m, cudaMemcpyHostToDevice, st));
    if (n) LCS_CK(ctx, cudaMemcpyAsync(io + b_off, b_host, n, cudaMemcpyHostToDevice, st));
    void *dd = direct ? direct : (staged ? (void *)(io + d_off) : nullptr);
    uint8_t *ld_lcs = lcs_host ? reinterpret_cast<uint8_t *>(io + l_off) : nullptr;
    if (!ctx->side) {
        LCS_CK(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_dist, cudaEventDisableTiming));
        LCS_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming));
        LCS_CK(ctx, cudaMallocHost(&ctx->host_hdr, 64));
    }
    s = solve_device(ctx, reinterpret_cast<const uint8_t *>(io + a_off), m, reinterpret_cast<const uint8_t *>(io + b_off),
                     n, dtype, dd, ldd, ld_lcs, cap, nullptr, nullptr, true, st, staged ? ctx->ev_dist : nullptr,
                     direct != nullptr);
    if (s != LCS_OK) return s;
    // A staged DIST leaves on the side stream as soon as it is complete,
    // while the traceback kernels still run; the LCS (cap bytes) and the
    // error / length words follow the solve on st; one synchronisation.
    if (staged) {
        LCS_CK(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_dist, 0));
        LCS_CK(ctx, cudaMemcpy2DAsync(dist_host, (size_t)ld * dt_size(rdt), dd, (size_t)ldd * dt_size(rdt),
                                      (size_t)(n + 1) * dt_size(rdt), (size_t)(n + 1), cudaMemcpyDeviceToHost,
                                      ctx->side));
        LCS_CK(ctx, cudaEventRecord(ctx->ev_copied, ctx->side));
    }
    if (lcs_host && cap > 0) LCS_CK(ctx, cudaMemcpyAsync(lcs_host, ld_lcs, (size_t)cap, cudaMemcpyDeviceToHost, st));
    LCS_CK(ctx, cudaMemcpyAsync(ctx->host_hdr, ctx->ws, 16, cudaMemcpyDeviceToHost, st));
    if (staged) LCS_CK(ctx, cudaStreamWaitEvent(st, ctx->ev_copied, 0));
    LCS_CK(ctx, cudaStreamSynchronize(st));
    const int errbits = (int)(ctx->host_hdr[0] & 0xFFFFFFFF);
    if (errbits) {
        LCS_CK(ctx, cudaMemset(ctx->ws, 0, 4));
        if (errbits & ERR_TIMEOUT) return fail(ctx, LCS_ETIMEOUT, "a device-side wait timed out");
        if (errbits & ERR_OVERFLOW) return fail(ctx, LCS_EOVERFLOW, "a value or the output exceeded its capacity");
        return fail(ctx, LCS_ECUDA, "device-side consistency check failed");
    }
    *out_len_host = ctx->host_hdr[1];
    return LCS_OK;
}

// ----------------------------------------------------------------------------- batches
// Pairs with more rows than this take the tall path (batch_big.cu): a sweep
// over several warps, and for the string no one-warp walk.
constexpr int64_t kBatchBigRows = 4096;

lcs_status lcs_batch_submit(lcs_ctx *ctx, const lcs_pair *pairs, int64_t count, uint64_t *ticket_out) {
    if (!ctx || !ticket_out || count < 0 || (count > 0 && !pairs)) return LCS_EINVAL;
    *ticket_out = 0;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    const int64_t max_rows = batch_max_rows();
    // Work items: the caller's pairs, and for each pair with more rows than
    // one strip but at most two strips' worth, its two halves split at row
    // rm (the items count + 2 s and count + 2 s + 1 of split pair s).  A
    // split pair's halves are one-strip pairs like the others; their columns
    // come from the split column that the recomputing sweeps find on the
    // device (Sec. II-D's argmax at the boundary row), and a join kernel adds
    // the halves' lengths and appends the lower half's string to the upper's.
    std::vector<lcs_pair> items(pairs, pairs + count);
    std::vector<int64_t> split_parent, split_rm;            // per split pair
    for (int64_t q = 0; q < count; ++q) {
        const lcs_pair &pr = pairs[q];
        if (pr.m > max_rows && pr.m <= 2 * max_rows && pr.n > 0 && pr.a && pr.b) {
            const int64_t rm = (pr.m + 1) / 2;
            split_parent.push_back(q);
            split_rm.push_back(rm);
        }
    }
    const int64_t n_split = (int64_t)split_parent.size();
    std::vector<char> is_split(count, 0);
    for (int64_t k = 0; k < n_split; ++k) {
        const lcs_pair &pr = pairs[split_parent[k]];
        is_split[split_parent[k]] = 1;
        lcs_pair h0 = pr, h1 = pr;
        h0.m = split_rm[k];
        h1.a = pr.a + split_rm[k];
        h1.m = pr.m - split_rm[k];
        items.push_back(h0);       // b, n: placeholders (the whole b) until the split is known
        items.push_back(h1);
    }
    const int64_t nitems = (int64_t)items.size();
    // Layout of the batch's device block.
    int64_t n_small = 0, n_big = 0, str_bytes = 0, scr_words = 0;
    std::vector<int64_t> str_off(nitems, -1), scr_off(nitems, 0);
    std::vector<char> big(nitems, 0);
    for (int64_t q = 0; q < nitems; ++q) {
        const lcs_pair &pr = items[q];
        if (q < count) {
            if (pr.m < 0 || pr.n < 0 || (pr.m > 0 && !pr.a) || (pr.n > 0 && !pr.b))
                return fail(ctx, LCS_EINVAL, "batch pair " + std::to_string(q) + ": bad string");
            if (pr.m >= INT32_MAX / 2 || pr.n >= INT32_MAX / 2) return fail(ctx, LCS_EINVAL, "batch pair too long");
        }
        const bool want = (pr.flags & LCS_WANT_STRING) != 0;
        if (want) {
            if (q >= count && ((q - count) & 1) == 0) {
                str_off[q] = str_off[split_parent[(q - count) / 2]];   // the upper half writes the pair's slot
            } else {
                str_off[q] = str_bytes;                                // a pair, or a lower half's own slot
                str_bytes += std::min(pr.m, pr.n);
            }
        }
        if (q < count && is_split[q]) continue;
        if (pr.m <= max_rows) {
            ++n_small;
            if (pr.m > kBatchBigRows && pr.n > 0) {
                // Tall pair (batch_big.cu); with its string: forward and
                // backward column vectors, then m + 1 cross vertices.
                big[q] = 1;
                ++n_big;
                if (want) {
                    const int64_t wu = (pr.m + 31) / 32;
                    scr_off[q] = scr_words;
                    scr_words += (2 * (pr.n + 1) * wu + pr.m + 1 + 3) / 4 * 4;
                }
            } else if (want && pr.m > 0 && pr.n > 0) {
                // (n+1) column words per row word, then (n+1) x (words+1)
                // 16-bit counts (batch.cu), rounded to 16 bytes.
                const int64_t wu = (pr.m + 31) / 32;
                scr_off[q] = scr_words;
                scr_words += ((pr.n + 1) * wu + ((pr.n + 1) * (wu + 1) + 1) / 2 + 3) / 4 * 4;
            }
        }
    }
    const size_t o_pairs = 0;
    const size_t o_order = align256(o_pairs + sizeof(BatchPair) * std::max<int64_t>(1, nitems));
    const size_t o_lens = align256(o_order + sizeof(int32_t) * std::max<int64_t>(1, nitems));
    const size_t o_err = align256(o_lens + sizeof(int64_t) * std::max<int64_t>(1, nitems));
    const size_t o_str = align256(o_err + sizeof(int));
    const size_t o_big = align256(o_str + (size_t)std::max<int64_t>(1, str_bytes));
    const size_t o_blens = align256(o_big + sizeof(BatchPair) * std::max<int64_t>(1, n_big));
    const size_t o_queue = align256(o_blens + sizeof(int32_t) * std::max<int64_t>(1, n_big));
    // Split pairs: their descriptors, sweep nodes and pairs, path endpoints
    // (nodes 3 s, 3 s + 1, 3 s + 2: the pair, its upper and lower half) and
    // the sweeps' count rows.
    int64_t split_nmax = 0;
    int split_rows = 0;
    for (int64_t k = 0; k < n_split; ++k) {
        const lcs_pair &pr = pairs[split_parent[k]];
        split_nmax = std::max(split_nmax, pr.n);
        split_rows = std::max<int>(split_rows, (int)std::max(split_rm[k], pr.m - split_rm[k]));
    }
    const int64_t ns1 = std::max<int64_t>(1, n_split);
    const size_t o_split = align256(o_queue + sizeof(unsigned) * kBatchClasses);
    const size_t o_snode = align256(o_split + sizeof(SplitPair) * ns1);
    const size_t o_spair = align256(o_snode + sizeof(SweepNode) * ns1);
    const size_t o_spath = align256(o_spair + sizeof(SweepPair) * ns1);
    const size_t o_fcnt = align256(o_spath + sizeof(int32_t) * 2 * 3 * ns1);
    const size_t o_bcnt = align256(o_fcnt + sizeof(int32_t) * (size_t)(n_split ? n_split * (split_nmax + 1) : 1));
    const size_t o_scr = align256(o_bcnt + sizeof(int32_t) * (size_t)(n_split ? n_split * (split_nmax + 1) : 1));
    const size_t total = align256(o_scr + (size_t)scr_words * 4);
    if (ctx->ws_bytes + ctx->io_bytes + ctx->batch_bytes + total > ctx->budget)
        return fail(ctx, LCS_EAGAIN, "batch does not fit the budget now");

    BatchTicket t;
    t.count = count;
    t.str_off = str_off;
    t.strings_bytes = str_bytes;
    t.host_status.assign(count, LCS_OK);
    t.t_submit = steady_seconds();
    // A lane (streams, events) from the free list, memory from the
    // context's pool: no call here synchronises the device, so a batch
    // submitted while others run overlaps with them.
    if (!ctx->mempool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        if (cudaMemPoolCreate(&ctx->mempool, &props) != cudaSuccess) {
            cudaGetLastError();
            ctx->mempool = nullptr;
            return fail(ctx, LCS_ECUDA, "batch memory pool");
        }
        uint64_t keep = UINT64_MAX;               // keep freed blocks for the next batches
        cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (!ctx->free_lanes.empty()) {
        t.lane = ctx->free_lanes.back();
        ctx->free_lanes.pop_back();
    } else if (!create_lane(t.lane)) {
        return fail(ctx, LCS_ECUDA, "batch streams/events");
    }
    auto cleanup = [&]() {
        if (t.dev) cudaFreeAsync(t.dev, t.lane.stream);
        cudaStreamSynchronize(t.lane.stream);
        ctx->free_lanes.push_back(t.lane);
    };
    if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&t.dev), total, ctx->mempool, t.lane.stream) != cudaSuccess) {
        cudaGetLastError();
        t.dev = nullptr;
        cleanup();
        return fail(ctx, LCS_ENOMEM, "batch device memory");
    }
    t.bytes = total;
    t.d_lens = reinterpret_cast<int64_t *>(t.dev + o_lens);
    t.d_strings = reinterpret_cast<uint8_t *>(t.dev + o_str);
    t.d_err = reinterpret_cast<int *>(t.dev + o_err);
    cudaStream_t st = t.lane.stream;
    // Descriptors by words-per-lane class (class c holds a up to 2048 << c
    // rows), each class's processing order largest pair first, so that the
    // last warps to finish have small ones.
    std::vector<BatchPair> hp;
    std::vector<int32_t> order;
    // Where each half's descriptor goes: index in hp (>= 0) or -1 - index in hb.
    std::vector<int64_t> half_desc(2 * n_split, 0);
    int64_t cls_begin[kBatchClasses + 1] = {0, 0, 0, 0, 0};
    for (int c = 0; c < kBatchClasses; ++c) {
        const int wpl = 2 << c;
        cls_begin[c] = (int64_t)hp.size();
        for (int64_t q = 0; q < nitems; ++q) {
            const lcs_pair &pr = items[q];
            if ((q < count && is_split[q]) || pr.m > max_rows || big[q] || batch_words_per_lane(pr.m) != wpl) continue;
            if (q >= count) half_desc[q - count] = (int64_t)hp.size();
            BatchPair b{};
            b.a = pr.a; b.b = pr.b; b.m = pr.m; b.n = pr.n;
            b.str_off = str_off[q] < 0 ? 0 : str_off[q];
            b.scratch_off = scr_off[q];
            b.len_out = t.d_lens + q;
            b.want = str_off[q] >= 0 ? 1 : 0;
            order.push_back((int32_t)(hp.size() - cls_begin[c]));
            hp.push_back(b);
        }
        std::stable_sort(order.begin() + cls_begin[c], order.end(), [&](int32_t x, int32_t y) {
            const BatchPair &u = hp[cls_begin[c] + x], &v = hp[cls_begin[c] + y];
            return u.m * u.n > v.m * v.n;
        });
    }
    cls_begin[kBatchClasses] = (int64_t)hp.size();
    // Tall pairs that want their string, by words-per-lane class (8, 16).
    std::vector<BatchPair> hb;
    std::vector<char> hb_half;
    int64_t big_begin[3] = {0, 0, 0}, big_max_n[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        big_begin[g] = (int64_t)hb.size();
        for (int64_t q = 0; q < nitems; ++q) {
            const lcs_pair &pr = items[q];
            if (!big[q] || batch_words_per_lane(pr.m) != (8 << g)) continue;
            if (q >= count) half_desc[q - count] = -1 - (int64_t)hb.size();
            BatchPair b{};
            b.a = pr.a; b.b = pr.b; b.m = pr.m; b.n = pr.n;
            b.str_off = str_off[q] < 0 ? 0 : str_off[q];
            b.scratch_off = scr_off[q];
            b.len_out = t.d_lens + q;
            b.want = str_off[q] >= 0 ? 1 : 0;
            hb.push_back(b);
            hb_half.push_back(q >= count ? 1 : 0);
            big_max_n[g] = std::max(big_max_n[g], pr.n);
        }
    }
    big_begin[2] = (int64_t)hb.size();
    lcs_status s = LCS_OK;
    do {
        if (cudaEventRecord(t.lane.ev_start, st) != cudaSuccess ||
            cudaMemsetAsync(t.dev + o_err, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(t.d_lens, 0, sizeof(int64_t) * std::max<int64_t>(1, nitems), st) != cudaSuccess) {
            s = fail(ctx, LCS_ECUDA, "batch setup");
            break;
        }
        // Pairs taller than two strips: the strip tree, one after another.
        for (int64_t q = 0; q < count && s == LCS_OK; ++q) {
            const lcs_pair &pr = pairs[q];
            if (pr.m <= max_rows || is_split[q]) continue;
            lcs_status ps = solve_device(ctx, pr.a, pr.m, pr.b, pr.n, LCS_I32, nullptr, 0,
                                         str_off[q] >= 0 ? t.d_strings + str_off[q] : nullptr,
                                         std::min(pr.m, pr.n), nullptr, t.d_lens + q, true, st);
            if (ps == LCS_OK) ps = read_back(ctx, st, nullptr);
            t.host_status[q] = ps;
            if (ps == LCS_ECUDA) s = ps;
        }
        if (s != LCS_OK) break;
        uint32_t *scr = reinterpret_cast<uint32_t *>(t.dev + o_scr);
        if (!hp.empty() &&
            (cudaMemcpyAsync(t.dev + o_pairs, hp.data(), sizeof(BatchPair) * hp.size(), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess ||
             cudaMemcpyAsync(t.dev + o_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice,
                             st) != cudaSuccess)) {
            s = fail(ctx, LCS_ECUDA, "batch descriptors");
            break;
        }
        if (!hb.empty()) {
            if (cudaMemcpyAsync(t.dev + o_big, hb.data(), sizeof(BatchPair) * hb.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
                s = fail(ctx, LCS_ECUDA, "batch tall descriptors");
                break;
            }
            for (size_t x = 0; x < hb.size(); ++x) {
                const BatchPair &b = hb[x];
                if (!b.want || hb_half[x]) continue;         // a half's are set by the split kernel
                const int64_t wu = (b.m + 31) / 32;
                // Cross vertices start above any column (0x7F7F7F7F > n).
                if (cudaMemsetAsync(scr + b.scratch_off + 2 * wu * (b.n + 1), 0x7F, sizeof(int32_t) * (b.m + 1), st) !=
                    cudaSuccess) {
                    s = fail(ctx, LCS_ECUDA, "batch tall setup");
                    break;
                }
            }
            if (s != LCS_OK) break;
        }
        // Split pairs: the root's forward and backward sweeps (a CTA each per
        // pair), the smallest maximiser per pair (the split column), then the
        // halves' columns in their descriptors, before any class kernel runs.
        if (n_split > 0) {
            std::vector<SplitPair> hs(n_split);
            std::vector<SweepNode> hn(n_split);
            std::vector<SweepPair> hq(n_split);
            std::vector<int32_t> hpath(2 * 3 * n_split, 0);
            int32_t *pathI = reinterpret_cast<int32_t *>(t.dev + o_spath), *pathJ = pathI + 3 * n_split;
            auto desc = [&](int64_t h) -> BatchPair * {
                const int64_t x = half_desc[h];
                return x >= 0 ? reinterpret_cast<BatchPair *>(t.dev + o_pairs) + x
                              : reinterpret_cast<BatchPair *>(t.dev + o_big) + (-1 - x);
            };
            for (int64_t k = 0; k < n_split; ++k) {
                const int64_t q = split_parent[k];
                const lcs_pair &pr = pairs[q];
                hn[k] = SweepNode{(int32_t)(3 * k), (int32_t)(3 * k + 1), (int32_t)(3 * k + 2), 0,
                                  (int32_t)split_rm[k], (int32_t)pr.m};
                hq[k] = SweepPair{pr.a, pr.b, pr.n, nullptr};
                hpath[3 * k] = 0;                            // pathI[root] = 0
                hpath[3 * n_split + 3 * k] = (int32_t)pr.n;  // pathJ[root] = n
                SplitPair sp{};
                sp.sub0 = desc(2 * k);
                sp.sub1 = desc(2 * k + 1);
                sp.b = pr.b;
                sp.n = pr.n;
                sp.lower = (int32_t)(3 * k + 2);
                sp.big0 = half_desc[2 * k] < 0 ? 1 : 0;
                sp.big1 = half_desc[2 * k + 1] < 0 ? 1 : 0;
                sp.pathI = pathI;
                sp.scratch = scr;
                sp.len_out = t.d_lens + q;
                sp.str = str_off[q] >= 0 ? t.d_strings + str_off[q] : nullptr;
                sp.str1 = str_off[count + 2 * k + 1] >= 0 ? t.d_strings + str_off[count + 2 * k + 1] : nullptr;
                sp.err = t.d_err;
                hs[k] = sp;
            }
            SweepParams swp{};
            swp.nodes = reinterpret_cast<const SweepNode *>(t.dev + o_snode);
            swp.count = (int32_t)n_split;
            swp.root_node = -1;
            swp.n = split_nmax;
            swp.pathI = pathI;
            swp.pathJ = pathJ;
            swp.fcnt = reinterpret_cast<int32_t *>(t.dev + o_fcnt);
            swp.bcnt = reinterpret_cast<int32_t *>(t.dev + o_bcnt);
            swp.err = t.d_err;
            swp.pairs = reinterpret_cast<const SweepPair *>(t.dev + o_spair);
            if (cudaMemcpyAsync(t.dev + o_split, hs.data(), sizeof(SplitPair) * n_split, cudaMemcpyHostToDevice,
                                st) != cudaSuccess ||
                cudaMemcpyAsync(t.dev + o_snode, hn.data(), sizeof(SweepNode) * n_split, cudaMemcpyHostToDevice,
                                st) != cudaSuccess ||
                cudaMemcpyAsync(t.dev + o_spair, hq.data(), sizeof(SweepPair) * n_split, cudaMemcpyHostToDevice,
                                st) != cudaSuccess ||
                cudaMemcpyAsync(pathI, hpath.data(), sizeof(int32_t) * hpath.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                launch_node_sweep(swp, split_rows, st) != cudaSuccess || launch_node_pick(swp, st) != cudaSuccess ||
                launch_split_fix(reinterpret_cast<const SplitPair *>(t.dev + o_split), n_split, st) != cudaSuccess) {
                s = fail(ctx, LCS_ECUDA, std::string("batch split pairs: ") + cudaGetErrorString(cudaGetLastError()));
                break;
            }
        }
        // The classes run side by side, each on a stream forked from the
        // batch's; the tall pairs' kernels run on the batch's stream beside
        // them; the classes join back before ev_done.  Each class's kernel
        // pulls its pairs from a zeroed work-queue counter.
        unsigned *queues = reinterpret_cast<unsigned *>(t.dev + o_queue);
        if (cudaMemsetAsync(queues, 0, sizeof(unsigned) * kBatchClasses, st) != cudaSuccess ||
            cudaEventRecord(t.lane.ev_fork, st) != cudaSuccess) {
            s = fail(ctx, LCS_ECUDA, "batch fork");
            break;
        }
        bool joined[kBatchClasses] = {false, false, false, false};
        for (int c = 0; c < kBatchClasses && s == LCS_OK; ++c) {
            const int64_t k0 = cls_begin[c], k1 = cls_begin[c + 1];
            if (k1 == k0) continue;
            BatchParams bp{};
            bp.pairs = reinterpret_cast<const BatchPair *>(t.dev + o_pairs) + k0;
            bp.order = reinterpret_cast<const int32_t *>(t.dev + o_order) + k0;
            bp.count = k1 - k0;
            bp.scratch = scr;
            bp.strings = t.d_strings;
            bp.err = t.d_err;
            bp.queue = queues + c;
            if (cudaStreamWaitEvent(t.lane.aux[c], t.lane.ev_fork, 0) != cudaSuccess ||
                launch_batch_strip(bp, 2 << c, t.lane.aux[c]) != cudaSuccess ||
                cudaEventRecord(t.lane.ev_join[c], t.lane.aux[c]) != cudaSuccess)
                s = fail(ctx, LCS_ECUDA, std::string("batch kernel: ") + cudaGetErrorString(cudaGetLastError()));
            else
                joined[c] = true;
        }
        for (int g = 0; g < 2 && s == LCS_OK; ++g) {
            if (big_begin[g + 1] == big_begin[g]) continue;
            BigParams gp{};
            gp.pairs = reinterpret_cast<const BatchPair *>(t.dev + o_big) + big_begin[g];
            gp.count = big_begin[g + 1] - big_begin[g];
            gp.max_n = big_max_n[g];
            gp.scratch = scr;
            gp.lens = reinterpret_cast<int32_t *>(t.dev + o_blens) + big_begin[g];
            gp.strings = t.d_strings;
            gp.err = t.d_err;
            if (launch_big(gp, 8 << g, st) != cudaSuccess)
                s = fail(ctx, LCS_ECUDA, std::string("batch tall kernels: ") + cudaGetErrorString(cudaGetLastError()));
        }
        for (int c = 0; c < kBatchClasses; ++c)
            if (joined[c] && cudaStreamWaitEvent(st, t.lane.ev_join[c], 0) != cudaSuccess && s == LCS_OK)
                s = fail(ctx, LCS_ECUDA, "batch join");
        if (s != LCS_OK) break;
        if (n_split > 0 &&
            launch_split_join(reinterpret_cast<const SplitPair *>(t.dev + o_split), n_split, st) != cudaSuccess) {
            s = fail(ctx, LCS_ECUDA, "batch split join");
            break;
        }
        // (The descriptor copies come from pageable host memory, which the
        // runtime stages before cudaMemcpyAsync returns.)
        if (cudaEventRecord(t.lane.ev_done, st) != cudaSuccess) s = fail(ctx, LCS_ECUDA, "batch event");
    } while (false);
    if (s != LCS_OK) {
        cleanup();
        return s;
    }
    const uint64_t id = ctx->next_ticket++;
    ctx->batch_bytes += t.bytes;
    ctx->peak = std::max(ctx->peak, ctx->ws_bytes + ctx->io_bytes + ctx->batch_bytes);
    ctx->tickets.emplace(id, std::move(t));
    *ticket_out = id;
    return LCS_OK;
}

lcs_status lcs_batch_poll(lcs_ctx *ctx, uint64_t ticket, lcs_result *results, int64_t cap, int64_t *n_done,
                          int32_t timeout_ms) {
    if (!ctx || !n_done || cap < 0 || (cap > 0 && !results)) return LCS_EINVAL;
    *n_done = 0;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, LCS_EINVAL, "unknown batch ticket");
    BatchTicket &t = it->second;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    const double t0 = steady_seconds();
    for (;;) {
        const cudaError_t q = cudaEventQuery(t.lane.ev_done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return fail(ctx, LCS_ECUDA, cudaGetErrorString(q));
        if (timeout_ms >= 0 && (steady_seconds() - t0) * 1e3 >= timeout_ms) return LCS_OK;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    std::vector<int64_t> lens(t.count);
    int err = 0;
    if (t.count) LCS_CK(ctx, cudaMemcpy(lens.data(), t.d_lens, sizeof(int64_t) * t.count, cudaMemcpyDeviceToHost));
    LCS_CK(ctx, cudaMemcpy(&err, t.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    float ms = 0.0f;
    LCS_CK(ctx, cudaEventElapsedTime(&ms, t.lane.ev_start, t.lane.ev_done));
    const lcs_status dev_status = (err & ERR_TIMEOUT) ? LCS_ETIMEOUT : (err ? LCS_ECUDA : LCS_OK);
    const int64_t nw = std::min(cap, t.count);
    for (int64_t q = 0; q < nw; ++q) {
        lcs_result &r = results[q];
        r.len = lens[q];
        r.string_offset = t.str_off[q];
        r.status = t.host_status[q] != LCS_OK ? t.host_status[q] : dev_status;
        r.t_submit = t.t_submit;
        r.t_done = t.t_submit + ms * 1e-3;
    }
    *n_done = t.count;
    return cap < t.count ? fail(ctx, LCS_EOVERFLOW, "results capacity below the batch size") : LCS_OK;
}

lcs_status lcs_batch_strings(lcs_ctx *ctx, uint64_t ticket, uint8_t *out, int64_t cap, int64_t *bytes) {
    if (!ctx || !bytes || cap < 0) return LCS_EINVAL;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, LCS_EINVAL, "unknown batch ticket");
    BatchTicket &t = it->second;
    *bytes = t.strings_bytes;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    LCS_CK(ctx, cudaEventSynchronize(t.lane.ev_done));
    if (cap < t.strings_bytes) return fail(ctx, LCS_EOVERFLOW, "string buffer too small");
    if (t.strings_bytes > 0) {
        if (!out) return LCS_EINVAL;
        LCS_CK(ctx, cudaMemcpy(out, t.d_strings, (size_t)t.strings_bytes, cudaMemcpyDefault));
    }
    return LCS_OK;
}

lcs_status lcs_batch_release(lcs_ctx *ctx, uint64_t ticket) {
    if (!ctx) return LCS_EINVAL;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, LCS_EINVAL, "unknown batch ticket");
    BatchTicket &t = it->second;
    LCS_CK(ctx, cudaSetDevice(ctx->device));
    LCS_CK(ctx, cudaStreamSynchronize(t.lane.stream));
    LCS_CK(ctx, cudaFreeAsync(t.dev, t.lane.stream));     // stream ordered: no device synchronisation
    ctx->free_lanes.push_back(t.lane);
    ctx->batch_bytes -= t.bytes;
    ctx->tickets.erase(it);
    return LCS_OK;
}

}  // extern "C"
