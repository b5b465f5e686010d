// Internal data structures of the IFGF library (host and device views).
//
// Layout in device memory (one plan):
//   points, Morton order:  xs, ys, zs            double [N]
//   perm                   int32 [N]             sorted position -> caller index
//   per level d = 1..D:
//     key[nbox]            uint64  Morton key of the box's integer coordinate
//     start[nbox+1]        int32   point range of the box (Morton order)
//     pt_box[N]            int32   box of every sorted point
//     parent[nbox]         int32   box at level d-1
//     child_start[nbox+1]  int32   children at level d+1 form a contiguous range
//     nbr[nbox][27]        int32   neighbours (Sec. 3.3.1), ascending, -1 padded
//     center[nbox][3]      double  x_k^d (Eq. defboxsizesandcenters)
//   per level d = 3..D (cone levels):
//     cous_start/cous      int32   CSR cousin lists (Eq. defcousinboxes)
//     tables               double  cos(k pi/n_C), node radii h/s_a, sin/cos of the
//                                  theta and phi interpolation nodes
//     bits[nbox][words]    uint64  relevant-cone bitmap (Eq. defallrelevantconesegments)
//     rank[nbox][words]    int32   slot of the first cone of each bitmap word
//     act_start/act_cone/act_box   relevant cones in (box, cone id) order
//     F[nact][P][nrhs]     complex values of F_k^d at the interpolation points
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cstdio>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include <cuda_runtime.h>

#include "ifgf.h"

#define IFGF_MAX_LEVELS 20

#define IFGF_MAX_P 8

struct LevelDev {
    int nbox = 0;
    int ns = 0, nc = 0;     // cone grid n_{s,d}, n_{C,d}
    int ncone = 0;          // n_s * n_C * 2 n_C
    int words = 0;          // bitmap words per box
    int nact = 0;           // relevant cones at this level
    double H = 0, h = 0, ds = 0, dth = 0;
    const uint64_t *key = nullptr;
    const int *start = nullptr;        // [nbox+1] first point of each box (start[nbox] = N)
    const int *end = nullptr;          // [nbox] one past the last point of each box (start[b+1] in a
                                       // uniform tree; adaptive trees have points of coarser leaves
                                       // between the boxes of a level)
    const unsigned char *leaf = nullptr;  // [nbox] the box is a leaf (not subdivided)
    const int *pt_box = nullptr;       // [N] box of every point at this level, -1 for points of
                                       // coarser leaves (adaptive trees)
    const int *parent = nullptr;
    const int *child_start = nullptr;
    const int *nbr = nullptr;          // [nbox][27]
    const int *cous_start = nullptr;
    const int *cous = nullptr;
    // near field of the leaf boxes of this level (d >= 3): CSR of point ranges [lo, hi),
    // ascending; the uniform tree's level-D lists are the 27 neighbours' ranges
    const int *near_start = nullptr;
    const int *near_lo = nullptr;
    const int *near_hi = nullptr;
    // relevant cone slots of the leaf boxes of this level (their analytic factors come from
    // their points); nullptr with nleaf_slots = nact: every slot
    const int *leaf_slots = nullptr;
    int nleaf_slots = 0;
    const double *center = nullptr;    // [nbox][3]
    const double *cosk = nullptr;      // [nc+1]
    const float *coskf = nullptr;      // [nc+1] the same in FP32 (cell decisions of the FP32 path)
    const double *nodeR = nullptr;     // [ns*Ps]
    const double *sth = nullptr, *cth = nullptr;  // [nc*Pang]
    const double *sph = nullptr, *cph = nullptr;  // [2nc*Pang]
    const double *cs_edge = nullptr;   // [2nc+1][2] cos, sin of k pi / n_C (cell start angles)
    double hds = 0;                    // h / Delta_s
    float inv_dth = 0;                 // 1 / Delta_theta
    const uint64_t *bits = nullptr;    // [nbox*words]
    const int *rank = nullptr;         // [nbox*words]
    const int *act_start = nullptr;    // [nbox+1]
    const int *act_cone = nullptr;     // [nact]
    const int *act_box = nullptr;      // [nact]
    void *F = nullptr;                 // forward values
    void *Fadj = nullptr;              // adjoint values
    const int *tl_start = nullptr;     // adjoint: per slot, cousin targets landing in it
    const int *tl = nullptr;
    const int *tl_cache = nullptr;     // per entry of tl, its evaluation's index in tcache
    const int *ul_start = nullptr;     // adjoint: per slot, parent (slot*P + node) landing in it
    const int *ul = nullptr;
    // batched plans: per entry of tl, the target's local coordinates in its cone
    // (x, y, z = s, theta, phi in [-1, 1]) and its centred factor G(x, x_k^d)
    const float4 *tl_loc = nullptr;
    const float2 *tl_fac = nullptr;
    // Upward table of the step from this level d to d-1 (absent: computed on the fly).
    // Rows are the distinct relevant cone ids of level d-1 (union bitmap + rank);
    // entry (row, octant, node) holds the child cone id, the Lagrange weights of the
    // node in that child cone and the re-centring factor.
    int urows = 0;
    const uint64_t *ubits = nullptr;   // [words of level d-1]
    const int *urank = nullptr;        // [words of level d-1]
    const int *uids = nullptr;         // [urows] cone id of each row
    const void *utab = nullptr;        // [urows][8][P] entries
    // Evaluation caches (plan time, when they fit the memory budget):
    // cousin targets of level d: point i's evaluations, in cousin-list order, at
    // tcache[toff[i] .. toff[i+1]); upward step d -> d-1 of an untabled level:
    // (parent slot s, node q, child c) at ucache[uoff[s] + q * nchild + c].
    const int *toff = nullptr;
    const void *tcache = nullptr;
    const int *uoff = nullptr;
    const void *ucache = nullptr;
};

constexpr int kNearTargets = 32;  // targets per near-field block
// most near-field point ranges of one leaf box (its 27 neighbours, and in an adaptive tree
// the leaf neighbours of its ancestors); plans that need more are rejected
constexpr int kMaxNearRanges = 27 * 8;

struct PlanDev {
    int n = 0, D = 0, Ps = 0, Pang = 0, P = 0;
    int pingpong = 0;   // level buffers alternate: target evaluation runs level by level
    double kappa = 0;
    double ts[IFGF_MAX_P] = {}, ta[IFGF_MAX_P] = {};    // Chebyshev nodes
    double its[IFGF_MAX_P] = {}, ita[IFGF_MAX_P] = {};  // 1 / prod_{e != a} (t_a - t_e)
    float tsf[IFGF_MAX_P] = {}, taf[IFGF_MAX_P] = {};   // the same in FP32, for FP32 weights
    float itsf[IFGF_MAX_P] = {}, itaf[IFGF_MAX_P] = {};
    const double *xs = nullptr, *ys = nullptr, *zs = nullptr;
    const float4 *leaf_off = nullptr;  // [N] x_j - centre of its leaf box, and its squared norm (FP32)
    const int *perm = nullptr;
    const int *ptlev = nullptr;        // [N] level of every point's leaf box (all D in a uniform tree)
    int adaptive = 0;                  // the tree has leaves above level D
    // near-field work items: (leaf box, first target, level) for each run of at most
    // kNearTargets consecutive targets of a leaf box
    const int4 *near_tile = nullptr;
    int n_near_tile = 0;
    int *err = nullptr;                                  // device invariant-failure counter
    int *sched = nullptr;  // [IFGF_MAX_LEVELS + 1] work counters of the batched cone kernel
    int flags = 0;         // the plan's option flags (test switches read by kernels)
    // batched path tile shapes (set by the autotuner, ifgf_plan_autotune): the leaf
    // kernel's register tile (0: 16 RHS threads x 8 node groups, 1: 32 x 4, 2: 8 x 16)
    // and the tensor-core cone kernel's persistent CTAs per SM (1 or 2)
    int tune_leaf = 0;
    int tune_cone_ctas = 2;
    int batched_f16 = 0;   // IFGF_BATCHED_FP16: the tensor-core contraction takes FP16 operands
    LevelDev lev[IFGF_MAX_LEVELS + 1];
};

// Per-stage CUDA-event timing of one call (enabled by ifgf_plan_set_profiling).
enum IfgfStage {
    STAGE_PERMUTE_IN = 0, STAGE_LEAF, STAGE_UPWARD, STAGE_EVAL, STAGE_PERMUTE_OUT,
    STAGE_ADJ_LEVEL, STAGE_ADJ_EVAL, STAGE_ADJ_LISTS, STAGE_COUNT
};

struct StageTimer {
    static constexpr int kMax = 2048;  // marks per evaluation (an adjoint built just in time marks per list range)
    bool on = false;
    int n = 0;
    cudaEvent_t ev[kMax] = {};
    int stage[kMax] = {};
    int launches[kMax] = {};
    bool external = false;  // capturing a CUDA graph: the records become event-record nodes
    void mark(int s, int nlaunch, cudaStream_t st)
    {
        if (!on || n >= kMax) return;
        if (external) cudaEventRecordWithFlags(ev[n], st, cudaEventRecordExternal);
        else cudaEventRecord(ev[n], st);
        stage[n] = s;
        launches[n] = nlaunch;
        ++n;
    }
};

// NVTX range for profilers (nsys timelines, ncu --nvtx-include): the plan build, each
// evaluation, and each stage and level of its launches.  Header-only NVTX: a no-op
// unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    NvtxRange(const char *stage, int level)
    {
        char buf[48];
        snprintf(buf, sizeof buf, "%s d=%d", stage, level);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct LevelHost {
    int64_t nbox = 0, nnbr = 0, ncous = 0, nact = 0;
    int ns = 0, nc = 0;
    int64_t cousin_evals = 0, upward_evals = 0;
    int64_t words = 0;
    int64_t table_rows = 0;   // rows of the upward table of step d -> d-1 (0: none)
    int act_sets = 0;         // rule (ii) of level d marked per distinct parent cone id (1) or per node (0)
    int64_t union_rows = 0;   // distinct relevant cone ids of level d-1 (the rows a table would have)
};

struct ifgf_plan {
    int64_t n = 0;
    int D = 0, Ps = 0, Pang = 0, P = 0;
    double kappa = 0;
    int precision = IFGF_FP64;
    int max_nrhs = 1;
    int flags = 0;
    int leaf_max = 0;          // adaptive tree: boxes of level >= 3 with at most leaf_max points are leaves
    int device = 0;            // the CUDA device current at ifgf_plan_create (owns every buffer)
    double timeout_s = 0;      // host-side wait limit of an evaluation (0: none)
    size_t value_budget = 0;   // bytes for cone values (0: 85% of the free memory less buffers and reserve)
    bool pingpong = false;     // two alternating level buffers instead of one per level
    size_t cache_bytes = 0;    // evaluation caches (0: none)
    int rhs_chunk = 1;         // right-hand sides per internal pass
    double H1 = 0, corner[3] = {0, 0, 0};
    PlanDev dev;
    LevelHost lh[IFGF_MAX_LEVELS + 1];
    int64_t near_pairs = 0;
    int64_t leaf_evals = 0;
    double build_ms = 0;
    size_t device_bytes = 0;
    std::vector<void *> allocs;
    void *sig_sorted = nullptr;   // [N][max_nrhs] complex
    void *u_sorted = nullptr;     // [N][max_nrhs] complex
    void *stage_in = nullptr;     // staging for host-pointer calls
    void *stage_out = nullptr;
    bool adjoint_ready = false;
    bool adjoint_values_ready = false;
    int last_nrhs = 1;
    cudaStream_t build_stream = nullptr;
    std::string last_error;
    StageTimer timer;
    double stage_ms[STAGE_COUNT] = {};
    int64_t stage_launches[STAGE_COUNT] = {};
    int64_t stage_calls = 0;
    // CUDA graphs of evaluations (ifgf_plan_set_graphs): the launches of one evaluation
    // for fixed device buffers, right-hand-side count, mode and direction, captured on
    // capture_stream at the first such call and replayed on the caller's stream after.
    // A graph captured with profiling on records the stage timer's events itself; it
    // keeps the stage and launch count of each mark for the attribution after a replay.
    struct GraphEntry {
        const void *in;
        void *out;
        int nrhs, mode, adjoint;
        bool timed;
        cudaGraphExec_t exec;
        uint64_t used;
        int tn;
        std::vector<int> tstage, tlaunch;
    };
    static constexpr int kMaxGraphs = 8;
    bool use_graphs = false;
    std::vector<GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
    uint64_t graph_clock = 0;
    int64_t graph_captures = 0, graph_replays = 0;
};

// complex element size of the plan's data type
inline size_t ifgf_elem_bytes(int precision) { return precision == IFGF_FP64 ? 16 : 8; }

// plans whose interpolation contractions run on the tensor cores
inline bool ifgf_is_batched(int precision) { return precision == IFGF_BATCHED_BF16 || precision == IFGF_BATCHED_FP16; }
// largest nrhs of one tensor-core pass at the given radial order (defined with the kernels)
int ifgf_batched_max_nrhs(int Ps);

// Upward-table entry for value type T and NW = P_s + 2 P_ang weights.
template <typename T, int NW> struct UpEntry {
    T w[NW];
    T fr, fi;
    int cone;
};

// The entry of FP32 plans (24 bytes): the local coordinates of the node in its child cone
// and the re-centring factor; the Lagrange weights are expanded from the coordinates by
// the same FP32 operations that would have produced stored weights.
struct UpEntry32 {
    float t[3];
    float fr, fi;
    int cone;
};

template <typename T, int NW> struct UpEntryOf { using type = UpEntry<T, NW>; };
template <int NW> struct UpEntryOf<float, NW> { using type = UpEntry32; };

// Cached geometry of one cousin-target evaluation.  FP64 plans: the Lagrange weights
// and the centred factor; float plans: the local coordinates and the factor.
struct TEntry64 {
    double w[13];
    double gr, gi;
    int slot, pad;
};
struct TEntry32 {
    float t[3];
    int slot;
    float gr, gi;
};

// Transpose lists built just in time for one level, for the adjoint of plans whose
// lists do not stay resident (two-buffer plans): CSR over the level-d slots [s0, s1)
// (start[s - s0] .. start[s - s0 + 1] index list).  Target lists hold point indices;
// upward lists hold parent slot * P + node, read as unsigned.
// A device buffer that only grows: the list builds of one adjoint call reuse it, so that
// hundreds of ranges do not each allocate and free gigabytes.
struct GrowBuf {
    void *ptr = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        if (ptr && bytes <= cap) return true;
        release();
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
            return false;
        }
        cap = bytes;
        return true;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
};

struct JitLists {
    int s0 = 0, s1 = 0;
    int *start = nullptr;
    int *list = nullptr;
    GrowBuf mem;   // holds start and list
};

// scratch of the list builds of one adjoint call (counts, offsets, unsorted and sorted
// keys, values, sort and scan temporaries)
struct JitWork {
    GrowBuf cnt, off, keys, vals, sorted, sort_tmp, scan_tmp;
    void release()
    {
        cnt.release(); off.release(); keys.release(); vals.release();
        sorted.release(); sort_tmp.release(); scan_tmp.release();
    }
};

// plan.cu
ifgf_status ifgf_build_plan(ifgf_plan *p, const double *points, cudaStream_t st);
// cousin-target transpose lists of level d (all slots)
ifgf_status ifgf_jit_targets(ifgf_plan *p, int d, JitLists *out, JitWork *w, cudaStream_t st);
// upward transpose lists of level d for the parent boxes [b0, b1) of level d-1
ifgf_status ifgf_jit_upward(ifgf_plan *p, int d, int b0, int b1, JitLists *out, JitWork *w, cudaStream_t st);
void ifgf_jit_release(JitLists *l);
// apply_f64.cu / apply_f32.cu: the adjoint with just-in-time lists (one RHS chunk)
ifgf_status ifgf_run_adjoint_jit_f64(ifgf_plan *p, int nrhs, const void *in, void *out, int mode, cudaStream_t st);
ifgf_status ifgf_run_adjoint_jit_f32(ifgf_plan *p, int nrhs, const void *in, void *out, int mode, cudaStream_t st);
// parent-box ranges of level d-1 whose upward lists hold at most max_entries each
ifgf_status ifgf_jit_chunks(ifgf_plan *p, int d, int64_t max_entries, std::vector<int> *bounds);
ifgf_status ifgf_build_adjoint_lists(ifgf_plan *p, cudaStream_t st);
ifgf_status ifgf_alloc_adjoint_values(ifgf_plan *p);
cudaError_t ifgf_cache_target_geometry(const PlanDev &pd, int d, float4 *loc, float2 *fac, int64_t m, cudaStream_t st);
void *ifgf_dalloc(ifgf_plan *p, size_t bytes);
// apply_*.cu: fill the upward table of level d (entries already allocated)
cudaError_t ifgf_build_uptable_f64(const PlanDev &pd, int d, void *tab, cudaStream_t st);
cudaError_t ifgf_build_uptable_f32(const PlanDev &pd, int d, void *tab, cudaStream_t st);
size_t ifgf_uptable_entry_bytes(int precision, int Ps, int Pang);
// fill the evaluation caches of level d (offsets and storage already set in pd)
cudaError_t ifgf_build_evalcache_f64(const PlanDev &pd, int d, int which, cudaStream_t st);
cudaError_t ifgf_build_evalcache_f32(const PlanDev &pd, int d, int which, cudaStream_t st);
// apply.cu
ifgf_status ifgf_run_apply(ifgf_plan *p, const void *sigma, void *u, int nrhs, int mode,
                           int adjoint, cudaStream_t st);
