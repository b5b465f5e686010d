// Plan construction on the GPU: the pre-computation stage of Algorithm 1.
//
//   root cube -> leaf integer coordinates -> Morton keys -> stable radix sort
//   -> per-level relevant boxes (unique keys), parents, children, centres
//   -> neighbours (Sec. 3.3.1) and cousins (Eq. defcousinboxes)
//   -> relevant cone segments, top-down d = 3..D (Sec. 3.3.2): rule (i) cousin
//      surface points, rule (ii) interpolation points of the parent's relevant
//      cones; deduplicated in a per-box bitmap, numbered by a rank directory.
//
// Radix sort and prefix sums use CUB (the CUDA toolkit's header library); every
// other step is a kernel in this file.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>

#include <cub/cub.cuh>

#include "ifgf_device.cuh"

using namespace ifgf;

namespace {

constexpr int kThreads = 256;

inline int nblocks(int64_t n, int t = kThreads)
{
    int64_t b = (n + t - 1) / t;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 30));
}

// ---------------------------------------------------------------------------------
// Root cube: componentwise min/max and finiteness.
// ---------------------------------------------------------------------------------
__global__ void k_bbox_partial(const double *pts, int n, double *part, int *bad)
{
    __shared__ double smin[3][kThreads], smax[3][kThreads];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            double v = pts[3 * (size_t)i + c];
            if (!isfinite(v)) atomicAdd(bad, 1);
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    }
    for (int c = 0; c < 3; ++c) { smin[c][threadIdx.x] = lo[c]; smax[c][threadIdx.x] = hi[c]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) {
                smin[c][threadIdx.x] = fmin(smin[c][threadIdx.x], smin[c][threadIdx.x + s]);
                smax[c][threadIdx.x] = fmax(smax[c][threadIdx.x], smax[c][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            part[6 * blockIdx.x + c] = smin[c][0];
            part[6 * blockIdx.x + 3 + c] = smax[c][0];
        }
}

__global__ void k_bbox_final(const double *part, int nb, double *out)
{
    if (threadIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], part[6 * b + c]);
            hi[c] = fmax(hi[c], part[6 * b + 3 + c]);
        }
    for (int c = 0; c < 3; ++c) { out[c] = lo[c]; out[3 + c] = hi[c]; }
}

// ---------------------------------------------------------------------------------
// Leaf integer coordinate k = clamp(floor((x - corner) / H_D), 0, 2^{D-1}-1), Morton key.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}
__device__ __forceinline__ uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}

__global__ void k_morton(const double *pts, int n, double c0, double c1, double c2, double HD,
                         int nside, uint64_t *key, int *idx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double cr[3] = {c0, c1, c2};
    uint64_t k[3];
    for (int c = 0; c < 3; ++c) {
        double q = floor(__ddiv_rn(__dsub_rn(pts[3 * (size_t)i + c], cr[c]), HD));
        k[c] = q < 0.0 ? 0 : (q > (double)(nside - 1) ? (uint64_t)(nside - 1) : (uint64_t)q);
    }
    key[i] = spread3(k[0]) | (spread3(k[1]) << 1) | (spread3(k[2]) << 2);
    idx[i] = i;
}

__global__ void k_gather_points(const double *pts, const int *idx, int n, double *xs, double *ys,
                                double *zs, int *perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = idx[i];
    xs[i] = pts[3 * (size_t)j];
    ys[i] = pts[3 * (size_t)j + 1];
    zs[i] = pts[3 * (size_t)j + 2];
    perm[i] = j;
}

// Box boundaries of level d among the points that still lie in boxes of level d (their
// leaf level ptlev >= d; all points in a uniform tree): flag[i] = 1 where such a point
// starts a box, i.e. where the level key changes or the previous point lies in a coarser
// leaf.
__device__ __forceinline__ bool level_start(const uint64_t *leafkey, const int *ptlev, int i, int d, int shift)
{
    return ptlev[i] >= d && (i == 0 || ptlev[i - 1] < d || (leafkey[i] >> shift) != (leafkey[i - 1] >> shift));
}

__global__ void k_level_flags(const uint64_t *leafkey, const int *ptlev, int n, int d, int shift, int *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = level_start(leafkey, ptlev, i, d, shift) ? 1 : 0;
}

// pt_box = inclusive scan - 1 (-1 for points of coarser leaves); box starts, ends and keys
__global__ void k_level_boxes(const uint64_t *leafkey, const int *ptlev, const int *incl, int n, int d, int shift,
                              int nbox, int *pt_box, int *start, int *end, uint64_t *key)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) start[nbox] = n;
    if (ptlev[i] < d) {
        pt_box[i] = -1;
        return;
    }
    int b = incl[i] - 1;
    pt_box[i] = b;
    if (level_start(leafkey, ptlev, i, d, shift)) {
        start[b] = i;
        key[b] = leafkey[i] >> shift;
    }
    if (i == n - 1 || ptlev[i + 1] < d || (leafkey[i + 1] >> shift) != (leafkey[i] >> shift)) end[b] = i + 1;
}

// Leaves of level d: every box of level D; with leaf_max > 0 (adaptive tree), also the
// boxes of levels 3..D-1 that hold at most leaf_max points.  The points of a leaf above
// level D take its level as their leaf level.
__global__ void k_level_leaves(const int *start, const int *end, int nbox, int d, int D, int leaf_max,
                               unsigned char *leaf)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    leaf[b] = (d == D || (leaf_max > 0 && d >= 3 && end[b] - start[b] <= leaf_max)) ? 1 : 0;
}

__global__ void k_max_int(const int *v, int n, int *mx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, v[i]);
}

__global__ void k_any_leaf(const unsigned char *leaf, int nbox, int *any)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox && leaf[b]) atomicExch(any, 1);
}

__global__ void k_mark_leaf_points(const int *pt_box, const unsigned char *leaf, int n, int d, int *ptlev)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = pt_box[i];
    if (b >= 0 && leaf[b]) ptlev[i] = d;
}

// offset of every point from the centre of its leaf box, and its squared norm: formed
// in FP64, stored in FP32 (for the FP32 leaf factor), with the rounding remainder of
// the offset in FP32 (for FP32 near-field distances that stay exact for close pairs)
__global__ void k_leaf_offsets(PlanDev pd, float4 *off)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    const LevelDev &L = pd.lev[pd.ptlev[i]];
    const double *c = L.center + 3 * (size_t)L.pt_box[i];
    double dx = pd.xs[i] - c[0], dy = pd.ys[i] - c[1], dz = pd.zs[i] - c[2];
    off[i] = make_float4((float)dx, (float)dy, (float)dz, (float)(dx * dx + dy * dy + dz * dz));
}

// Near-field work items: the targets of each leaf box of level d in runs of kNearTargets.
__global__ void k_near_tile_count(const int *start, const int *end, const unsigned char *leaf, int nbox, int *cnt)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbox) return;
    cnt[b] = b < nbox && leaf[b] ? (end[b] - start[b] + kNearTargets - 1) / kNearTargets : 0;
}

__global__ void k_near_tile_emit(const int *start, int nbox, int d, const int *tstart, int4 *tile)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    for (int t = tstart[b]; t < tstart[b + 1]; ++t)
        tile[t] = make_int4(b, start[b] + (t - tstart[b]) * kNearTargets, d, 0);
}

// Near-field ranges of the leaf boxes of level l (the near relation of adaptive trees):
// the points of every neighbour of the box at level l, and for each level d = 3..l-1 the
// points of the leaf neighbours of its ancestor at level d; ascending by first point.
// With leaves on level D only these are the 27 neighbours' ranges.
template <bool FILL>
__global__ void k_near_ranges(PlanDev pd, int l, int *count, const int *nstart, int *lo, int *hi)
{
    const LevelDev &L = pd.lev[l];
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= L.nbox) return;
    if (!L.leaf[b]) {
        if (!FILL) count[b] = 0;
        return;
    }
    int m = 0;
    const int o = FILL ? nstart[b] : 0;
    auto add = [&](int s, int e) {
        if (FILL) {  // insertion by first point (the lists are short)
            int j = m;
            while (j > 0 && lo[o + j - 1] > s) {
                lo[o + j] = lo[o + j - 1];
                hi[o + j] = hi[o + j - 1];
                --j;
            }
            lo[o + j] = s;
            hi[o + j] = e;
        }
        ++m;
    };
    for (int e = 0; e < 27; ++e) {
        const int q = L.nbr[27 * (size_t)b + e];
        if (q < 0) break;
        add(L.start[q], L.end[q]);
    }
    int a = b;
    for (int d = l - 1; d >= 3; --d) {
        a = pd.lev[d + 1].parent[a];
        const LevelDev &La = pd.lev[d];
        for (int e = 0; e < 27; ++e) {
            const int q = La.nbr[27 * (size_t)a + e];
            if (q < 0) break;
            if (La.leaf[q]) add(La.start[q], La.end[q]);
        }
    }
    if (!FILL) count[b] = m;
}

// relevant cone slots of the leaf boxes of level d
__global__ void k_leaf_slot_count(const int *act_start, const unsigned char *leaf, int nbox, int *cnt)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbox) return;
    cnt[b] = b < nbox && leaf[b] ? act_start[b + 1] - act_start[b] : 0;
}

__global__ void k_leaf_slot_emit(const int *act_start, const unsigned char *leaf, int nbox, const int *off,
                                 int *slots)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox || !leaf[b]) return;
    for (int s = act_start[b]; s < act_start[b + 1]; ++s) slots[off[b] + s - act_start[b]] = s;
}

// Points must be pairwise distinct (Eq. field1 sums over m != l; the method's
// factorisation divides by |x_l - x_m|).  Equal points share their level-D Morton key,
// so each point is compared with the later points of its key run.
__global__ void k_duplicates(PlanDev pd, const uint64_t *leafkey, int *found)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    const double x = pd.xs[i], y = pd.ys[i], z = pd.zs[i];
    for (int j = i + 1; j < pd.n && leafkey[j] == leafkey[i]; ++j)
        if (pd.xs[j] == x && pd.ys[j] == y && pd.zs[j] == z) {
            atomicExch(found, 1);
            return;
        }
}

__global__ void k_parents(const int *start, int nbox, const int *pt_box_parent, int *parent)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    parent[b] = pt_box_parent[start[b]];
}

// children of parent box p (level d-1) are the contiguous level-d boxes with parent p:
// child_start[p] = the first level-d box whose parent is >= p (leaves have none)
__global__ void k_child_start(const int *parent, int nbox, int nparent, int *child_start)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nparent) return;
    int lo = 0, hi = nbox;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (parent[mid] < p) lo = mid + 1; else hi = mid;
    }
    child_start[p] = lo;
}

// x_k^d = corner + (k + 1/2) H_d   (Eq. defboxsizesandcenters, 0-based k)
__global__ void k_centers(const uint64_t *key, int nbox, double c0, double c1, double c2, double H,
                          double *center)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    uint64_t kk = key[b];
    double cr[3] = {c0, c1, c2};
    for (int c = 0; c < 3; ++c) {
        double k = (double)compact3(kk >> c);
        center[3 * (size_t)b + c] = __dadd_rn(cr[c], __dmul_rn(k + 0.5, H));
    }
}

__device__ __forceinline__ int find_key(const uint64_t *keys, int n, uint64_t key)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

// neighbours N B: relevant boxes a with |a - k|_inf <= 1 (including k), ascending
__global__ void k_neighbours(const uint64_t *key, int nbox, int side, int *nbr)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    uint64_t kk = key[b];
    int k[3] = {(int)compact3(kk), (int)compact3(kk >> 1), (int)compact3(kk >> 2)};
    int list[27];
    int m = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int a0 = k[0] + dx, a1 = k[1] + dy, a2 = k[2] + dz;
                if (a0 < 0 || a1 < 0 || a2 < 0 || a0 >= side || a1 >= side || a2 >= side) continue;
                uint64_t ck = spread3(a0) | (spread3(a1) << 1) | (spread3(a2) << 2);
                int f = find_key(key, nbox, ck);
                if (f >= 0) {
                    int j = m++;
                    while (j > 0 && list[j - 1] > f) { list[j] = list[j - 1]; --j; }
                    list[j] = f;
                }
            }
    for (int j = 0; j < 27; ++j) nbr[27 * (size_t)b + j] = j < m ? list[j] : -1;
}

// cousins M B (Eq. defcousinboxes): children of the parent's neighbours that are
// not neighbours of B.  Parents' neighbours are ascending and children ranges are
// ordered by parent, so the list comes out ascending.
template <bool FILL>
__global__ void k_cousins(const uint64_t *key, int nbox, const int *parent, const int *pnbr,
                          const int *pchild_start, int *count, const int *cstart, int *cous)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    uint64_t kk = key[b];
    int k[3] = {(int)compact3(kk), (int)compact3(kk >> 1), (int)compact3(kk >> 2)};
    int p = parent[b];
    int m = 0;
    int out = FILL ? cstart[b] : 0;
    for (int e = 0; e < 27; ++e) {
        int q = pnbr[27 * (size_t)p + e];
        if (q < 0) break;
        for (int c = pchild_start[q]; c < pchild_start[q + 1]; ++c) {
            uint64_t ck = key[c];
            int a0 = (int)compact3(ck), a1 = (int)compact3(ck >> 1), a2 = (int)compact3(ck >> 2);
            int dd = max(abs(a0 - k[0]), max(abs(a1 - k[1]), abs(a2 - k[2])));
            if (dd > 1) {
                if (FILL) cous[out + m] = c;
                ++m;
            }
        }
    }
    if (!FILL) count[b] = m;
}

// ---------------------------------------------------------------------------------
// Relevant cones (Sec. 3.3.2).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void set_bit(uint64_t *bits, int words, int box, int cone)
{
    atomicOr((unsigned long long *)&bits[(size_t)box * words + (cone >> 6)], 1ull << (cone & 63));
}

// rule (i): every cousin surface point of box k marks its cone around x_k.
// Written per point over the boxes that have it as a cousin point (the cousin
// relation is symmetric).
__global__ void k_activate_cousins(PlanDev pd, int d, uint64_t *bits)
{
    const LevelDev &L = pd.lev[d];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    int b = L.pt_box[i];
    if (b < 0) return;  // a point of a coarser leaf (adaptive tree)
    double x = pd.xs[i], y = pd.ys[i], z = pd.zs[i];
    for (int e = L.cous_start[b]; e < L.cous_start[b + 1]; ++e) {
        int k = L.cous[e];
        const double *c = L.center + 3 * (size_t)k;
        ConeGeom g = cone_of_mixed(L, __dsub_rn(x, c[0]), __dsub_rn(y, c[1]), __dsub_rn(z, c[2]));
        // neighbouring points of a leaf mostly mark the same cone of the same cousin
        const unsigned grp = __activemask();
        const unsigned long long key = ((unsigned long long)(unsigned)k << 32) | (unsigned)g.cone;
        const unsigned same = __match_any_sync(grp, key);
        if ((threadIdx.x & 31) == __ffs(same) - 1) set_bit(bits, L.words, k, g.cone);
    }
}

// rule (ii): every interpolation point of a relevant parent cone marks its cone
// around each child centre.  Both activation kernels take cells from cone_of_mixed,
// which equals the correctly rounded cone_of bit for bit (FP32 decisions only outside a
// margin around the cell boundaries, cone_of inside it) at a fraction of its FP64 cost.
// The lanes of a warp hold consecutive nodes of one or two parent cones and mostly mark the
// same few child cones: only one lane per distinct (child, cone) pair issues the atomic OR.
__global__ void k_activate_parent(PlanDev pd, int d, uint64_t *bits)
{
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < (int64_t)Lp.nact * pd.P;
    if (__all_sync(0xffffffffu, !valid)) return;  // whole warps past the end
    const int slot = valid ? (int)(t / pd.P) : 0, node = valid ? (int)(t % pd.P) : 0;
    const int j = valid ? Lp.act_box[slot] : 0;
    const int k0 = valid ? Lp.child_start[j] : 0, nch = valid ? Lp.child_start[j + 1] - k0 : 0;
    const int maxch = __reduce_max_sync(0xffffffffu, nch);
    const double hh = L.H * 0.5;
    for (int kk = 0; kk < maxch; ++kk) {
        unsigned long long key = ~0ull;  // (child box, cone) of this lane, or none
        if (kk < nch) {
            const int k = k0 + kk;
            double v[3];
            node_rel(Lp, pd.Ps, pd.Pang, Lp.act_cone[slot], node, hh, (int)(L.key[k] & 7u), v, nullptr);
            ConeGeom g = cone_of_mixed(L, v[0], v[1], v[2]);
            key = ((unsigned long long)(unsigned)k << 32) | (unsigned)g.cone;
        }
        const unsigned same = __match_any_sync(0xffffffffu, key);
        if (key != ~0ull && (threadIdx.x & 31) == __ffs(same) - 1)
            set_bit(bits, L.words, (int)(key >> 32), (int)(key & 0xffffffffu));
    }
}

// Rule (ii) by parent cone id.  The cell of a parent interpolation point seen from a child
// centre depends only on (parent cone id, child octant, node): the point relative to the
// child centre is R dir - delta (node_rel).  So the set of child cones that one parent cone
// id marks in the child of one octant is the same for every box; it is computed once per
// distinct parent cone id of the level (the union of the boxes' relevant cones) and octant,
// and every (parent slot, child) pair then sets those bits.  The sets are the ones the
// per-node kernel marks, bit for bit.  At most kConeSet cells are kept per (id, octant); a
// larger set is stored as count -1 and its pairs take the per-node path.
constexpr int kConeSet = 4;

// one warp per (union row, octant): count, then the distinct cells in order of first node
__global__ void k_cone_sets(PlanDev pd, int d, const int *uids, int rows, int *sets)
{
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)rows * 8) return;  // the whole warp
    const int row = (int)(wid >> 3), oct = (int)(wid & 7);
    const double hh = L.H * 0.5;
    int found[kConeSet];
#pragma unroll
    for (int i = 0; i < kConeSet; ++i) found[i] = -1;
    int n = 0;  // distinct cells so far (the same in every lane)
    bool over = false;
    for (int n0 = 0; n0 < pd.P; n0 += 32) {
        const int node = n0 + lane;
        int cone = -1;
        if (node < pd.P) {
            double v[3];
            node_rel(Lp, pd.Ps, pd.Pang, uids[row], node, hh, oct, v, nullptr);
            cone = cone_of_mixed(L, v[0], v[1], v[2]).cone;
        }
        unsigned pending = __ballot_sync(0xffffffffu, cone >= 0);
        while (pending) {
            const int c = __shfl_sync(0xffffffffu, cone, __ffs(pending) - 1);
            pending &= ~__ballot_sync(0xffffffffu, cone == c);
            bool known = false;
#pragma unroll
            for (int i = 0; i < kConeSet; ++i) known = known || (i < n && found[i] == c);
            if (!known) {
                if (n < kConeSet) {
#pragma unroll
                    for (int i = 0; i < kConeSet; ++i)
                        if (i == n) found[i] = c;
                    ++n;
                } else {
                    over = true;
                }
            }
        }
    }
    if (lane == 0) {
        int *out = sets + (size_t)wid * (kConeSet + 1);
        out[0] = over ? -1 : n;
#pragma unroll
        for (int i = 0; i < kConeSet; ++i) out[1 + i] = found[i];
    }
}

// One thread per (child position, parent slot), slots innermost: the lanes of a warp hold
// consecutive slots, mostly of one parent box, so they mark cones of the same child box.
// Lanes that set bits in the same bitmap word combine them first (match, then an OR
// reduction over the group) and one of them issues the atomic: the slots of a box all
// write into a few words of each child, and one atomic each would serialise in L2.
__global__ void k_activate_parent_sets(PlanDev pd, int d, const uint64_t *ubits, const int *urank, const int *sets,
                                       uint64_t *bits)
{
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)Lp.nact * 8;
    if (__all_sync(0xffffffffu, t >= total)) return;  // whole warps past the end
    bool valid = t < total;
    const int kk = valid ? (int)(t / Lp.nact) : 0, slot = valid ? (int)(t % Lp.nact) : 0;
    int k = 0, oct = 0, pcone = 0, cnt = 0;
    const int *set = nullptr;
    if (valid) {
        const int j = Lp.act_box[slot];
        const int k0 = Lp.child_start[j], nch = Lp.child_start[j + 1] - k0;
        valid = kk < nch;
        if (valid) {
            k = k0 + kk;
            oct = (int)(L.key[k] & 7u);
            pcone = Lp.act_cone[slot];
            const int row = table_row(ubits, urank, pcone);
            if (row < 0) {  // every relevant cone id is in the union
                atomicAdd(pd.err, 1);
                valid = false;
            } else {
                set = sets + ((size_t)row * 8 + oct) * (kConeSet + 1);
                cnt = set[0];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kConeSet; ++i) {
        unsigned long long key = ~0ull, bit = 0;
        if (valid && i < cnt) {
            const int cone = set[1 + i];
            key = (unsigned long long)k * L.words + (unsigned)(cone >> 6);
            bit = 1ull << (cone & 63);
        }
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const unsigned lo = __reduce_or_sync(grp, (unsigned)bit), hi = __reduce_or_sync(grp, (unsigned)(bit >> 32));
        if (key != ~0ull && (threadIdx.x & 31) == __ffs(grp) - 1)
            atomicOr((unsigned long long *)&bits[key], ((unsigned long long)hi << 32) | lo);
    }
    if (valid && cnt < 0) {  // more than kConeSet cells: node by node
        const double hh = L.H * 0.5;
        for (int node = 0; node < pd.P; ++node) {
            double v[3];
            node_rel(Lp, pd.Ps, pd.Pang, pcone, node, hh, oct, v, nullptr);
            set_bit(bits, L.words, k, cone_of_mixed(L, v[0], v[1], v[2]).cone);
        }
    }
}

// union over boxes of a level's relevant-cone bitmaps
__global__ void k_union_bits(const uint64_t *bits, int nbox, int words, uint64_t *ubits)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nbox * words) return;
    uint64_t v = bits[t];
    if (v) atomicOr((unsigned long long *)&ubits[t % words], (unsigned long long)v);
}

__global__ void k_popc(const uint64_t *bits, int64_t nw, int *cnt)
{
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) cnt[w] = __popcll(bits[w]);
}

__global__ void k_expand(const uint64_t *bits, const int *rank, int64_t nw, int words, int *act_cone,
                         int *act_box)
{
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint64_t v = bits[w];
    int s = rank[w];
    int box = (int)(w / words);
    int base = (int)(w % words) * 64;
    while (v) {
        int j = __ffsll((long long)v) - 1;
        act_cone[s] = base + j;
        act_box[s] = box;
        ++s;
        v &= v - 1;
    }
}

__global__ void k_act_start(const int *rank, int nbox, int words, int nact, int *act_start)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbox) return;
    act_start[b] = b < nbox ? rank[(size_t)b * words] : nact;
}

// statistics: cousin evaluations = sum over points of the cousin count of their box
__global__ void k_count_cousin_evals(PlanDev pd, int d, unsigned long long *acc)
{
    const LevelDev &L = pd.lev[d];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < pd.n) {
        int b = L.pt_box[i];
        if (b >= 0) v = (unsigned long long)(L.cous_start[b + 1] - L.cous_start[b]);
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

__global__ void k_count_near(PlanDev pd, unsigned long long *acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < pd.n) {
        const LevelDev &L = pd.lev[pd.ptlev[i]];
        int b = L.pt_box[i];
        for (int e = L.near_start[b]; e < L.near_start[b + 1]; ++e)
            v += (unsigned long long)(L.near_hi[e] - L.near_lo[e]);
        v -= 1;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

__global__ void k_count_upward(PlanDev pd, int d, unsigned long long *acc)
{
    const LevelDev &Lp = pd.lev[d - 1];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (s < Lp.nact) {
        int j = Lp.act_box[s];
        v = (unsigned long long)(Lp.child_start[j + 1] - Lp.child_start[j]) * pd.P;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

__global__ void k_count_leaf(PlanDev pd, int d, unsigned long long *acc)
{
    const LevelDev &L = pd.lev[d];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (s < L.nact && L.leaf[L.act_box[s]]) {
        int b = L.act_box[s];
        v = (unsigned long long)(L.end[b] - L.start[b]) * pd.P;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc, v);
}

// ---------------------------------------------------------------------------------
// Transpose lists for the adjoint.
// ---------------------------------------------------------------------------------

// (slot, target) pairs of all cousin evaluations of level d; offsets from a scan
// of the per-point cousin counts.
__global__ void k_emit_tlist(PlanDev pd, int d, const int *off, int *keys, int *vals)
{
    const LevelDev &L = pd.lev[d];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    int b = L.pt_box[i];
    if (b < 0) return;  // a point of a coarser leaf
    double x = pd.xs[i], y = pd.ys[i], z = pd.zs[i];
    int o = off[i];
    for (int e = L.cous_start[b]; e < L.cous_start[b + 1]; ++e, ++o) {
        int k = L.cous[e];
        const double *c = L.center + 3 * (size_t)k;
        ConeGeom g = cone_of(L, __dsub_rn(x, c[0]), __dsub_rn(y, c[1]), __dsub_rn(z, c[2]));
        int sl = cone_slot(L, k, g.cone);
        if (sl < 0) { atomicAdd(pd.err, 1); sl = 0; }
        keys[o] = sl;
        vals[o] = i;
    }
}

__global__ void k_iota(int *a, int64_t m)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = (int)i;
}

// out[j] = src[idx[j]]
__global__ void k_gather_int(int *out, const int *src, const int *idx, int64_t m)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) out[j] = src[idx[j]];
}

__global__ void k_point_cousin_count(PlanDev pd, int d, int *cnt)
{
    const LevelDev &L = pd.lev[d];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    int b = L.pt_box[i];
    cnt[i] = b < 0 ? 0 : L.cous_start[b + 1] - L.cous_start[b];
}

__global__ void k_parent_slot_count(PlanDev pd, int d, int *cnt)
{
    const LevelDev &Lp = pd.lev[d - 1];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Lp.nact) return;
    int j = Lp.act_box[s];
    cnt[s] = (Lp.child_start[j + 1] - Lp.child_start[j]) * pd.P;
}

// (child slot, parent slot * P + node) pairs of all upward evaluations of level d
__global__ void k_emit_ulist(PlanDev pd, int d, const int *off, int *keys, int *vals)
{
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Lp.nact * pd.P) return;
    int slot = (int)(t / pd.P), node = (int)(t % pd.P);
    int j = Lp.act_box[slot];
    int nch = Lp.child_start[j + 1] - Lp.child_start[j];
    const double hh = L.H * 0.5;
    int o = off[slot] + node * nch;
    for (int k = Lp.child_start[j]; k < Lp.child_start[j + 1]; ++k, ++o) {
        double v[3];
        node_rel(Lp, pd.Ps, pd.Pang, Lp.act_cone[slot], node, hh, (int)(L.key[k] & 7u), v, nullptr);
        ConeGeom g = cone_of(L, v[0], v[1], v[2]);
        int sl = cone_slot(L, k, g.cone);
        if (sl < 0) { atomicAdd(pd.err, 1); sl = 0; }
        keys[o] = sl;
        vals[o] = (int)t;
    }
}

// Upward evaluations of level d whose parent slots are [q0, q1), for just-in-time
// lists: cnt[q - q0] = entries of parent slot q
__global__ void k_parent_slot_count_range(PlanDev pd, int d, int q0, int q1, int *cnt)
{
    const LevelDev &Lp = pd.lev[d - 1];
    int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    int j = Lp.act_box[q];
    cnt[q - q0] = (Lp.child_start[j + 1] - Lp.child_start[j]) * pd.P;
}

// (child slot - s0, parent slot * P + node) pairs of those evaluations; the second
// member is stored as the bits of an unsigned value (it can exceed 2^31 - 1)
__global__ void k_emit_ulist_range(PlanDev pd, int d, int q0, int q1, int s0, const int *off, int *keys,
                                   int *vals)
{
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int64_t t = (int64_t)q0 * pd.P + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)q1 * pd.P) return;
    const int slot = (int)(t / pd.P), node = (int)(t % pd.P);
    const int j = Lp.act_box[slot];
    const int nch = Lp.child_start[j + 1] - Lp.child_start[j];
    const double hh = L.H * 0.5;
    int o = off[slot - q0] + node * nch;
    for (int k = Lp.child_start[j]; k < Lp.child_start[j + 1]; ++k, ++o) {
        double v[3];
        node_rel(Lp, pd.Ps, pd.Pang, Lp.act_cone[slot], node, hh, (int)(L.key[k] & 7u), v, nullptr);
        ConeGeom g = cone_of(L, v[0], v[1], v[2]);
        int sl = cone_slot(L, k, g.cone);
        if (sl < 0) { atomicAdd(pd.err, 1); sl = s0; }
        keys[o] = sl - s0;
        vals[o] = (int)(unsigned)t;
    }
}

// CSR starts from sorted keys: start[s] = first position with key >= s
__global__ void k_csr_from_sorted(const int *keys, int64_t m, int nslot, int *start)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nslot) return;
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < s) lo = mid + 1; else hi = mid;
    }
    start[s] = (int)lo;
}

}  // namespace

// ===================================================================================
// Host orchestration
// ===================================================================================

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            p->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;          \
        }                                                                                 \
    } while (0)

void *ifgf_dalloc(ifgf_plan *p, size_t bytes)
{
    void *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    p->allocs.push_back(ptr);
    p->device_bytes += bytes;
    return ptr;
}

template <typename T> static T *dalloc(ifgf_plan *p, size_t count)
{
    return (T *)ifgf_dalloc(p, count * sizeof(T));
}

#define DALLOC(var, T, count)                                                        \
    T *var = dalloc<T>(p, (size_t)(count));                                          \
    if (!var) {                                                                      \
        p->last_error = "device allocation failed (" #var ")";                      \
        return IFGF_ENOMEM;                                                          \
    }

// temporary device buffer freed at scope exit
struct Scratch {
    void *ptr = nullptr;
    ~Scratch() { if (ptr) cudaFree(ptr); }
    bool alloc(size_t bytes)
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        return cudaMalloc(&ptr, bytes ? bytes : 16) == cudaSuccess;
    }
};

static ifgf_status cub_inclusive_sum(ifgf_plan *p, const int *in, int *out, int64_t n, cudaStream_t st)
{
    size_t bytes = 0;
    CK(cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out, n, st));
    Scratch tmp;
    if (!tmp.alloc(bytes)) { p->last_error = "scan scratch"; return IFGF_ENOMEM; }
    CK(cub::DeviceScan::InclusiveSum(tmp.ptr, bytes, in, out, n, st));
    CK(cudaStreamSynchronize(st));
    return IFGF_OK;
}

static ifgf_status cub_exclusive_sum(ifgf_plan *p, const int *in, int *out, int64_t n, cudaStream_t st)
{
    size_t bytes = 0;
    CK(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, st));
    Scratch tmp;
    if (!tmp.alloc(bytes)) { p->last_error = "scan scratch"; return IFGF_ENOMEM; }
    CK(cub::DeviceScan::ExclusiveSum(tmp.ptr, bytes, in, out, n, st));
    CK(cudaStreamSynchronize(st));
    return IFGF_OK;
}

static inline double cheb_node(int k, int n)
{
    return cos(((double)(2 * k + 1) * M_PI) / (double)(2 * n));
}

// device memory kept free at plan time for the adjoint's transpose lists and workspace
constexpr size_t kReserveBytes = (size_t)24 << 30;

ifgf_status ifgf_build_plan(ifgf_plan *p, const double *points, cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    const int n = (int)p->n, D = p->D, Ps = p->Ps, Pang = p->Pang, P = p->P;
    PlanDev &pd = p->dev;
    pd.n = n; pd.D = D; pd.Ps = Ps; pd.Pang = Pang; pd.P = P; pd.kappa = p->kappa;
    for (int a = 0; a < Ps; ++a) pd.ts[a] = cheb_node(a, Ps);
    for (int a = 0; a < Pang; ++a) pd.ta[a] = cheb_node(a, Pang);
    for (int a = 0; a < Ps; ++a) {
        double v = 1.0;
        for (int e = 0; e < Ps; ++e) if (e != a) v *= pd.ts[a] - pd.ts[e];
        pd.its[a] = 1.0 / v;
    }
    for (int a = 0; a < Pang; ++a) {
        double v = 1.0;
        for (int e = 0; e < Pang; ++e) if (e != a) v *= pd.ta[a] - pd.ta[e];
        pd.ita[a] = 1.0 / v;
    }
    for (int a = 0; a < IFGF_MAX_P; ++a) {
        pd.tsf[a] = (float)pd.ts[a];
        pd.taf[a] = (float)pd.ta[a];
        pd.itsf[a] = (float)pd.its[a];
        pd.itaf[a] = (float)pd.ita[a];
    }
    DALLOC(d_err, int, 1);
    CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    pd.err = d_err;
    DALLOC(d_sched, int, IFGF_MAX_LEVELS + 1);
    pd.sched = d_sched;

    // points to the device (AoS, caller order)
    Scratch pts;
    if (!pts.alloc((size_t)n * 3 * sizeof(double))) { p->last_error = "points scratch"; return IFGF_ENOMEM; }
    CK(cudaMemcpyAsync(pts.ptr, points, (size_t)n * 3 * sizeof(double), cudaMemcpyDefault, st));
    const double *dpts = (const double *)pts.ptr;

    // root cube (reading: bounding cube of the points, centred at the bbox midpoint)
    {
        int nb = std::min(nblocks(n), 1024);
        Scratch part, out;
        if (!part.alloc((size_t)nb * 6 * sizeof(double)) || !out.alloc(6 * sizeof(double) + sizeof(int)))
            return IFGF_ENOMEM;
        int *bad = (int *)((double *)out.ptr + 6);
        CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_bbox_partial<<<nb, kThreads, 0, st>>>(dpts, n, (double *)part.ptr, bad);
        k_bbox_final<<<1, 32, 0, st>>>((double *)part.ptr, nb, (double *)out.ptr);
        CK(cudaGetLastError());
        double h[6];
        int hbad = 0;
        CK(cudaMemcpyAsync(h, out.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hbad) { p->last_error = "non-finite point coordinates"; return IFGF_EINVAL; }
        double H1 = 0.0;
        for (int c = 0; c < 3; ++c)
            if (h[3 + c] - h[c] > H1) H1 = h[3 + c] - h[c];
        if (!(H1 > 0.0)) { p->last_error = "all points coincide"; return IFGF_EINVAL; }
        p->H1 = H1;
        for (int c = 0; c < 3; ++c) p->corner[c] = (h[c] + h[3 + c]) * 0.5 - H1 * 0.5;
    }
    double Hd[IFGF_MAX_LEVELS + 1];
    for (int d = 1; d <= D; ++d) Hd[d] = ldexp(p->H1, -(d - 1));

    // Morton keys and stable sort (ties keep the caller order)
    DALLOC(xs, double, n);
    DALLOC(ys, double, n);
    DALLOC(zs, double, n);
    DALLOC(perm, int, n);
    pd.xs = xs; pd.ys = ys; pd.zs = zs; pd.perm = perm;
    Scratch keyA, keyB, idxA, idxB;
    if (!keyA.alloc((size_t)n * 8) || !keyB.alloc((size_t)n * 8) || !idxA.alloc((size_t)n * 4) ||
        !idxB.alloc((size_t)n * 4)) {
        p->last_error = "sort scratch";
        return IFGF_ENOMEM;
    }
    k_morton<<<nblocks(n), kThreads, 0, st>>>(dpts, n, p->corner[0], p->corner[1], p->corner[2], Hd[D],
                                              1 << (D - 1), (uint64_t *)keyA.ptr, (int *)idxA.ptr);
    CK(cudaGetLastError());
    {
        size_t bytes = 0;
        CK(cub::DeviceRadixSort::SortPairs(nullptr, bytes, (uint64_t *)keyA.ptr, (uint64_t *)keyB.ptr,
                                           (int *)idxA.ptr, (int *)idxB.ptr, n, 0, 3 * (D - 1), st));
        Scratch tmp;
        if (!tmp.alloc(bytes)) { p->last_error = "sort temp"; return IFGF_ENOMEM; }
        CK(cub::DeviceRadixSort::SortPairs(tmp.ptr, bytes, (uint64_t *)keyA.ptr, (uint64_t *)keyB.ptr,
                                           (int *)idxA.ptr, (int *)idxB.ptr, n, 0, 3 * (D - 1), st));
    }
    const uint64_t *leafkey = (const uint64_t *)keyB.ptr;
    k_gather_points<<<nblocks(n), kThreads, 0, st>>>(dpts, (int *)idxB.ptr, n, xs, ys, zs, perm);
    CK(cudaGetLastError());

    // relevant boxes of every level.  A box exists when its parent exists and is not a
    // leaf (every box of levels 1..D-1 in a uniform tree); the points of a leaf above
    // level D lie in no box of the finer levels (ptlev < d there).
    DALLOC(ptlev, int, n);
    {
        std::vector<int> hD(n, D);
        CK(cudaMemcpyAsync(ptlev, hD.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    pd.ptlev = ptlev;
    pd.adaptive = 0;
    Scratch flag, incl;
    if (!flag.alloc((size_t)n * 4) || !incl.alloc((size_t)n * 4)) return IFGF_ENOMEM;
    for (int d = 1; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        int shift = 3 * (D - d);
        k_level_flags<<<nblocks(n), kThreads, 0, st>>>(leafkey, ptlev, n, d, shift, (int *)flag.ptr);
        CK(cudaGetLastError());
        ifgf_status s = cub_inclusive_sum(p, (int *)flag.ptr, (int *)incl.ptr, n, st);
        if (s != IFGF_OK) return s;
        int nbox = 0;
        CK(cudaMemcpy(&nbox, (int *)incl.ptr + (n - 1), sizeof(int), cudaMemcpyDeviceToHost));
        L.nbox = nbox;
        p->lh[d].nbox = nbox;
        DALLOC(pt_box, int, n);
        DALLOC(start, int, nbox + 1);
        DALLOC(bend, int, nbox + 1);
        DALLOC(key, uint64_t, nbox + 1);
        DALLOC(leaf, unsigned char, nbox + 1);
        k_level_boxes<<<nblocks(n), kThreads, 0, st>>>(leafkey, ptlev, (int *)incl.ptr, n, d, shift, nbox, pt_box,
                                                       start, bend, key);
        k_level_leaves<<<nblocks(nbox), kThreads, 0, st>>>(start, bend, nbox, d, D, p->leaf_max, leaf);
        if (d < D && d >= 3 && p->leaf_max > 0)
            k_mark_leaf_points<<<nblocks(n), kThreads, 0, st>>>(pt_box, leaf, n, d, ptlev);
        CK(cudaGetLastError());
        L.pt_box = pt_box; L.start = start; L.end = bend; L.key = key; L.leaf = leaf;
        L.H = Hd[d];
        DALLOC(center, double, 3 * (size_t)nbox);
        k_centers<<<nblocks(nbox), kThreads, 0, st>>>(key, nbox, p->corner[0], p->corner[1], p->corner[2],
                                                      Hd[d], center);
        CK(cudaGetLastError());
        L.center = center;
        DALLOC(nbr, int, 27 * (size_t)nbox);
        k_neighbours<<<nblocks(nbox), kThreads, 0, st>>>(key, nbox, 1 << (d - 1), nbr);
        CK(cudaGetLastError());
        L.nbr = nbr;
    }
    {
        CK(cudaMemsetAsync(flag.ptr, 0, sizeof(int), st));
        k_duplicates<<<nblocks(n), kThreads, 0, st>>>(pd, leafkey, (int *)flag.ptr);
        CK(cudaGetLastError());
        int dup = 0;
        CK(cudaMemcpy(&dup, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        if (dup) {
            p->last_error = "duplicate points (the points must be pairwise distinct)";
            return IFGF_EINVAL;
        }
    }
    for (int d = 2; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        LevelDev &Lp = pd.lev[d - 1];
        DALLOC(parent, int, L.nbox);
        k_parents<<<nblocks(L.nbox), kThreads, 0, st>>>(L.start, L.nbox, Lp.pt_box, parent);
        DALLOC(cstart, int, Lp.nbox + 1);
        k_child_start<<<nblocks(Lp.nbox + 1), kThreads, 0, st>>>(parent, L.nbox, Lp.nbox, cstart);
        CK(cudaGetLastError());
        L.parent = parent;
        Lp.child_start = cstart;
    }
    {
        DALLOC(off, float4, n);
        k_leaf_offsets<<<nblocks(n), kThreads, 0, st>>>(pd, off);
        CK(cudaGetLastError());
        pd.leaf_off = off;
    }
    // leaves above level D make the tree adaptive
    for (int d = 3; d < D; ++d) {
        int any = 0;
        if (p->leaf_max > 0 && pd.lev[d].nbox > 0) {
            Scratch c;
            if (!c.alloc(sizeof(int))) return IFGF_ENOMEM;
            CK(cudaMemsetAsync(c.ptr, 0, sizeof(int), st));
            k_any_leaf<<<nblocks(pd.lev[d].nbox), kThreads, 0, st>>>(pd.lev[d].leaf, pd.lev[d].nbox, (int *)c.ptr);
            CK(cudaMemcpy(&any, c.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        }
        if (any) pd.adaptive = 1;
    }
    // near-field ranges of the leaf boxes of every level, and the work items: runs of at
    // most kNearTargets targets of a leaf box
    {
        int ntile = 0;
        Scratch tstarts[IFGF_MAX_LEVELS + 1];
        int nt_level[IFGF_MAX_LEVELS + 1] = {};
        for (int d = 3; d <= D; ++d) {
            LevelDev &L = pd.lev[d];
            const int nb = L.nbox;
            Scratch cnt;
            if (!cnt.alloc((size_t)(nb + 1) * 4)) return IFGF_ENOMEM;
            CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(nb + 1) * 4, st));
            if (nb > 0) k_near_ranges<false><<<nblocks(nb), kThreads, 0, st>>>(pd, d, (int *)cnt.ptr, nullptr, nullptr, nullptr);
            CK(cudaGetLastError());
            {
                Scratch mx;
                if (!mx.alloc(sizeof(int))) return IFGF_ENOMEM;
                CK(cudaMemsetAsync(mx.ptr, 0, sizeof(int), st));
                if (nb > 0) k_max_int<<<nblocks(nb), kThreads, 0, st>>>((int *)cnt.ptr, nb, (int *)mx.ptr);
                int hmax = 0;
                CK(cudaMemcpy(&hmax, mx.ptr, sizeof(int), cudaMemcpyDeviceToHost));
                if (hmax > kMaxNearRanges) {
                    p->last_error = "a leaf box has more than " + std::to_string(kMaxNearRanges) +
                                    " near-field ranges (use fewer levels or a smaller leaf_max)";
                    return IFGF_EINVAL;
                }
            }
            DALLOC(nstart, int, nb + 1);
            ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, nstart, nb + 1, st);
            if (s != IFGF_OK) return s;
            int m = 0;
            CK(cudaMemcpy(&m, nstart + nb, sizeof(int), cudaMemcpyDeviceToHost));
            DALLOC(nlo, int, m + 1);
            DALLOC(nhi, int, m + 1);
            L.near_start = nstart;
            L.near_lo = nlo;
            L.near_hi = nhi;
            if (nb > 0) k_near_ranges<true><<<nblocks(nb), kThreads, 0, st>>>(pd, d, nullptr, nstart, nlo, nhi);
            CK(cudaGetLastError());
            if (!tstarts[d].alloc((size_t)(nb + 1) * 4)) return IFGF_ENOMEM;
            CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(nb + 1) * 4, st));
            k_near_tile_count<<<nblocks(nb + 1), kThreads, 0, st>>>(L.start, L.end, L.leaf, nb, (int *)cnt.ptr);
            CK(cudaGetLastError());
            s = cub_exclusive_sum(p, (int *)cnt.ptr, (int *)tstarts[d].ptr, nb + 1, st);
            if (s != IFGF_OK) return s;
            CK(cudaMemcpy(&nt_level[d], (int *)tstarts[d].ptr + nb, sizeof(int), cudaMemcpyDeviceToHost));
            ntile += nt_level[d];
        }
        DALLOC(tile, int4, ntile + 1);
        int o = 0;
        for (int d = D; d >= 3; --d) {  // finest leaves first (the uniform tree: level D only)
            if (nt_level[d] == 0) continue;
            k_near_tile_emit<<<nblocks(pd.lev[d].nbox), kThreads, 0, st>>>(pd.lev[d].start, pd.lev[d].nbox, d,
                                                                         (int *)tstarts[d].ptr, tile + o);
            CK(cudaGetLastError());
            o += nt_level[d];
        }
        CK(cudaStreamSynchronize(st));
        pd.near_tile = tile;
        pd.n_near_tile = ntile;
    }
    // cousins of levels 3..D
    for (int d = 3; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        LevelDev &Lp = pd.lev[d - 1];
        Scratch cnt;
        if (!cnt.alloc((size_t)(L.nbox + 1) * 4)) return IFGF_ENOMEM;
        CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(L.nbox + 1) * 4, st));
        k_cousins<false><<<nblocks(L.nbox), kThreads, 0, st>>>(L.key, L.nbox, L.parent, Lp.nbr,
                                                               Lp.child_start, (int *)cnt.ptr, nullptr, nullptr);
        CK(cudaGetLastError());
        DALLOC(cstart, int, L.nbox + 1);
        ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, cstart, L.nbox + 1, st);
        if (s != IFGF_OK) return s;
        int total = 0;
        CK(cudaMemcpy(&total, cstart + L.nbox, sizeof(int), cudaMemcpyDeviceToHost));
        DALLOC(cous, int, total);
        k_cousins<true><<<nblocks(L.nbox), kThreads, 0, st>>>(L.key, L.nbox, L.parent, Lp.nbr,
                                                              Lp.child_start, nullptr, cstart, cous);
        CK(cudaGetLastError());
        L.cous_start = cstart;
        L.cous = cous;
        p->lh[d].ncous = total;
    }

    // cone levels: n_{.,d-1} = a_d n_{.,d}, a_d = 2 iff 2 kappa H_d > 1
    int ns[IFGF_MAX_LEVELS + 1], nc[IFGF_MAX_LEVELS + 1];
    ns[D] = p->lh[D].ns;
    nc[D] = p->lh[D].nc;
    for (int d = D; d >= 4; --d) {
        int a = (2.0 * p->kappa * Hd[d] > 1.0) ? 2 : 1;
        ns[d - 1] = a * ns[d];
        nc[d - 1] = a * nc[d];
    }
    const double eta = sqrt(3.0) / 3.0;
    for (int d = 3; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        int64_t ncone64 = (int64_t)ns[d] * nc[d] * 2 * nc[d];
        if (ncone64 >= (int64_t)1 << 30) {
            p->last_error = "too many cone cells per box at level " + std::to_string(d);
            return IFGF_EINVAL;
        }
        L.ns = ns[d]; L.nc = nc[d]; L.ncone = (int)ncone64;
        L.words = (L.ncone + 63) / 64;
        L.h = sqrt(3.0) * 0.5 * Hd[d];
        L.ds = eta / (double)ns[d];
        L.dth = M_PI / (double)nc[d];
        p->lh[d].ns = ns[d];
        p->lh[d].nc = nc[d];
        p->lh[d].words = L.words;
        std::vector<double> tab;
        size_t o_cosk = tab.size();
        for (int k = 0; k <= nc[d]; ++k) tab.push_back(cos(((double)k * M_PI) / (double)nc[d]));
        size_t o_R = tab.size();
        for (int g = 0; g < ns[d]; ++g)
            for (int a = 0; a < Ps; ++a) {
                double s = L.ds * ((double)g + (1.0 + pd.ts[a]) * 0.5);
                tab.push_back(L.h / s);
            }
        size_t o_sth = tab.size();
        for (int g = 0; g < nc[d]; ++g)
            for (int b = 0; b < Pang; ++b) tab.push_back(sin(L.dth * ((double)g + (1.0 + pd.ta[b]) * 0.5)));
        size_t o_cth = tab.size();
        for (int g = 0; g < nc[d]; ++g)
            for (int b = 0; b < Pang; ++b) tab.push_back(cos(L.dth * ((double)g + (1.0 + pd.ta[b]) * 0.5)));
        size_t o_sph = tab.size();
        for (int g = 0; g < 2 * nc[d]; ++g)
            for (int c = 0; c < Pang; ++c) tab.push_back(sin(L.dth * ((double)g + (1.0 + pd.ta[c]) * 0.5)));
        size_t o_cph = tab.size();
        for (int g = 0; g < 2 * nc[d]; ++g)
            for (int c = 0; c < Pang; ++c) tab.push_back(cos(L.dth * ((double)g + (1.0 + pd.ta[c]) * 0.5)));
        size_t o_cs = tab.size();
        for (int k = 0; k <= 2 * nc[d]; ++k) {
            double a = ((double)k * M_PI) / (double)nc[d];
            tab.push_back(cos(a));
            tab.push_back(sin(a));
        }
        L.hds = L.h / L.ds;
        L.inv_dth = (float)(1.0 / L.dth);
        DALLOC(dtab, double, tab.size());
        CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        L.cosk = dtab + o_cosk; L.nodeR = dtab + o_R;
        L.sth = dtab + o_sth; L.cth = dtab + o_cth; L.sph = dtab + o_sph; L.cph = dtab + o_cph;
        L.cs_edge = dtab + o_cs;
        std::vector<float> ftab(tab.begin() + o_cosk, tab.begin() + o_cosk + nc[d] + 1);
        DALLOC(coskf, float, ftab.size());
        CK(cudaMemcpyAsync(coskf, ftab.data(), ftab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        L.coskf = coskf;
    }

    // relevant cones, top-down
    for (int d = 3; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        int64_t nw = (int64_t)L.nbox * L.words;
        DALLOC(bits, uint64_t, nw);
        DALLOC(rank, int, nw + 1);
        CK(cudaMemsetAsync(bits, 0, nw * sizeof(uint64_t), st));
        L.bits = bits;
        L.rank = rank;
        k_activate_cousins<<<nblocks(n), kThreads, 0, st>>>(pd, d, bits);
        CK(cudaGetLastError());
        if (d >= 4) {
            // rule (ii): per distinct parent cone id where they are few against the parent
            // slots (each slot has up to 8 children of P nodes), else per node (flags bit
            // 12 forces the per-node kernel; the marked bits are the same)
            const LevelDev &Lp = pd.lev[d - 1];
            const int64_t pw = Lp.words;
            Scratch ub, ucnt, ur;
            if (!ub.alloc((size_t)pw * 8) || !ucnt.alloc((size_t)(pw + 1) * 4) || !ur.alloc((size_t)(pw + 1) * 4))
                return IFGF_ENOMEM;
            CK(cudaMemsetAsync(ub.ptr, 0, (size_t)pw * 8, st));
            CK(cudaMemsetAsync(ucnt.ptr, 0, (size_t)(pw + 1) * 4, st));
            const int64_t tot = (int64_t)Lp.nbox * Lp.words;
            k_union_bits<<<nblocks(tot), kThreads, 0, st>>>(Lp.bits, Lp.nbox, Lp.words, (uint64_t *)ub.ptr);
            k_popc<<<nblocks(pw), kThreads, 0, st>>>((const uint64_t *)ub.ptr, pw, (int *)ucnt.ptr);
            CK(cudaGetLastError());
            ifgf_status su = cub_exclusive_sum(p, (int *)ucnt.ptr, (int *)ur.ptr, pw + 1, st);
            if (su != IFGF_OK) return su;
            int rows = 0;
            CK(cudaMemcpy(&rows, (int *)ur.ptr + pw, sizeof(int), cudaMemcpyDeviceToHost));
            if (!(p->flags & 4096) && rows > 0 && 2 * (int64_t)rows <= Lp.nact) {
                Scratch uid, dummy, sets;
                if (!uid.alloc((size_t)rows * 4) || !dummy.alloc((size_t)rows * 4) ||
                    !sets.alloc((size_t)rows * 8 * (kConeSet + 1) * 4))
                    return IFGF_ENOMEM;
                k_expand<<<nblocks(pw), kThreads, 0, st>>>((const uint64_t *)ub.ptr, (const int *)ur.ptr, pw, (int)pw,
                                                          (int *)uid.ptr, (int *)dummy.ptr);
                k_cone_sets<<<nblocks((int64_t)rows * 8 * 32), kThreads, 0, st>>>(pd, d, (const int *)uid.ptr, rows,
                                                                                   (int *)sets.ptr);
                k_activate_parent_sets<<<nblocks((int64_t)Lp.nact * 8), kThreads, 0, st>>>(
                    pd, d, (const uint64_t *)ub.ptr, (const int *)ur.ptr, (const int *)sets.ptr, bits);
                CK(cudaGetLastError());
                CK(cudaStreamSynchronize(st));
                p->lh[d].act_sets = 1;
            } else {
                int64_t nt = (int64_t)Lp.nact * P;
                k_activate_parent<<<nblocks(nt), kThreads, 0, st>>>(pd, d, bits);
                CK(cudaGetLastError());
            }
        }
        Scratch cnt;
        if (!cnt.alloc((size_t)(nw + 1) * 4)) return IFGF_ENOMEM;
        CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(nw + 1) * 4, st));
        k_popc<<<nblocks(nw), kThreads, 0, st>>>(bits, nw, (int *)cnt.ptr);
        CK(cudaGetLastError());
        ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, rank, nw + 1, st);
        if (s != IFGF_OK) return s;
        int nact = 0;
        CK(cudaMemcpy(&nact, rank + nw, sizeof(int), cudaMemcpyDeviceToHost));
        L.nact = nact;
        p->lh[d].nact = nact;
        DALLOC(act_cone, int, nact);
        DALLOC(act_box, int, nact);
        DALLOC(act_start, int, L.nbox + 1);
        k_expand<<<nblocks(nw), kThreads, 0, st>>>(bits, rank, nw, L.words, act_cone, act_box);
        k_act_start<<<nblocks(L.nbox + 1), kThreads, 0, st>>>(rank, L.nbox, L.words, nact, act_start);
        CK(cudaGetLastError());
        L.act_cone = act_cone; L.act_box = act_box; L.act_start = act_start;
        // relevant cones of the leaf boxes (every slot of level D in a uniform tree)
        if (!pd.adaptive) {
            L.leaf_slots = nullptr;
            L.nleaf_slots = d == D ? nact : 0;
        } else {
            Scratch lc;
            if (!lc.alloc((size_t)(L.nbox + 1) * 4)) return IFGF_ENOMEM;
            k_leaf_slot_count<<<nblocks(L.nbox + 1), kThreads, 0, st>>>(act_start, L.leaf, L.nbox, (int *)lc.ptr);
            CK(cudaGetLastError());
            DALLOC(loff, int, L.nbox + 1);
            s = cub_exclusive_sum(p, (int *)lc.ptr, loff, L.nbox + 1, st);
            if (s != IFGF_OK) return s;
            int nls = 0;
            CK(cudaMemcpy(&nls, loff + L.nbox, sizeof(int), cudaMemcpyDeviceToHost));
            DALLOC(lslots, int, nls + 1);
            if (L.nbox > 0) k_leaf_slot_emit<<<nblocks(L.nbox), kThreads, 0, st>>>(act_start, L.leaf, L.nbox, loff, lslots);
            CK(cudaGetLastError());
            L.leaf_slots = lslots;
            L.nleaf_slots = nls;
        }
    }

    // statistics of one apply
    {
        Scratch acc;
        if (!acc.alloc(sizeof(unsigned long long) * (IFGF_MAX_LEVELS + 4))) return IFGF_ENOMEM;
        unsigned long long *a = (unsigned long long *)acc.ptr;
        CK(cudaMemsetAsync(a, 0, sizeof(unsigned long long) * (IFGF_MAX_LEVELS + 4), st));
        for (int d = 3; d <= D; ++d) k_count_cousin_evals<<<nblocks(n), kThreads, 0, st>>>(pd, d, a + d);
        k_count_near<<<nblocks(n), kThreads, 0, st>>>(pd, a + 0);
        for (int d = 3; d <= D; ++d)
            if (pd.lev[d].nact > 0) k_count_leaf<<<nblocks(pd.lev[d].nact), kThreads, 0, st>>>(pd, d, a + 1);
        CK(cudaGetLastError());
        unsigned long long h[IFGF_MAX_LEVELS + 4];
        CK(cudaMemcpyAsync(h, a, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        p->near_pairs = (int64_t)h[0];
        p->leaf_evals = (int64_t)h[1];
        for (int d = 3; d <= D; ++d) p->lh[d].cousin_evals = (int64_t)h[d];
        CK(cudaMemsetAsync(a, 0, sizeof(unsigned long long) * (IFGF_MAX_LEVELS + 4), st));
        for (int d = 4; d <= D; ++d)
            k_count_upward<<<nblocks(pd.lev[d - 1].nact), kThreads, 0, st>>>(pd, d, a + d);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h, a, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int d = 4; d <= D; ++d) p->lh[d].upward_evals = (int64_t)h[d];
    }

    // Value buffers.  All levels stay resident when that fits the budget; otherwise
    // two buffers alternate between levels d and d-1 (the only two an evaluation
    // step reads and writes), and right-hand sides are processed in chunks.
    const size_t eb = ifgf_elem_bytes(p->precision);
    size_t all_levels = 0, max_pair = 0, max_level = 0;
    for (int d = 3; d <= D; ++d) {
        size_t b = (size_t)pd.lev[d].nact * P * eb;
        all_levels += b;
        max_level = std::max(max_level, b);
        if (d > 3) max_pair = std::max(max_pair, b + (size_t)pd.lev[d - 1].nact * P * eb);
    }
    if (D == 3) max_pair = max_level;
    size_t budget = p->value_budget;
    if (budget == 0) {
        // 85% of the free memory less the sorted density and field buffers and a reserve
        // for the adjoint's transpose lists and workspace; the upward tables and
        // evaluation caches come after the values, from what is left
        size_t freeb = 0, totalb = 0;
        CK(cudaMemGetInfo(&freeb, &totalb));
        const size_t sorted = (size_t)2 * n * p->max_nrhs * eb + std::min(kReserveBytes, totalb / 10);
        budget = freeb > sorted ? (size_t)((freeb - sorted) * 0.85) : 0;
    }
    if (all_levels * p->max_nrhs <= budget) {
        p->pingpong = false;
        p->rhs_chunk = p->max_nrhs;
    } else {
        p->pingpong = true;
        int64_t c = max_pair ? (int64_t)(budget / max_pair) : p->max_nrhs;
        if (c < 1) { p->last_error = "cone values of two levels do not fit in device memory"; return IFGF_ENOMEM; }
        // the fewest passes, then chunks as equal as possible (8 right-hand sides that fit
        // 5 at a time run as 4 + 4)
        const int64_t passes = (p->max_nrhs + std::min<int64_t>(c, p->max_nrhs) - 1) / std::min<int64_t>(c, p->max_nrhs);
        p->rhs_chunk = (int)((p->max_nrhs + passes - 1) / passes);
    }
    if (p->flags & 8) {  // force ping-pong buffers (tests)
        p->pingpong = true;
        p->rhs_chunk = p->max_nrhs;
    }
    if (p->flags & 16) p->rhs_chunk = std::min(p->rhs_chunk, 2);  // force small chunks (tests)
    pd.pingpong = p->pingpong ? 1 : 0;
    size_t value_bytes = 0;  // forward cone values of all levels (plans that keep every level)
    if (!p->pingpong) {
        for (int d = 3; d <= D; ++d) {
            LevelDev &L = pd.lev[d];
            value_bytes += (size_t)L.nact * P * p->rhs_chunk * eb;
            L.F = ifgf_dalloc(p, (size_t)L.nact * P * p->rhs_chunk * eb);
            if (!L.F) { p->last_error = "cone value buffer"; return IFGF_ENOMEM; }
        }
    } else {
        size_t even = 0, odd = 0;
        for (int d = 3; d <= D; ++d) {
            size_t b = (size_t)pd.lev[d].nact * P * p->rhs_chunk * eb;
            if (d & 1) odd = std::max(odd, b); else even = std::max(even, b);
        }
        void *bufs[2] = {ifgf_dalloc(p, even), ifgf_dalloc(p, odd)};
        if (!bufs[0] || !bufs[1]) { p->last_error = "cone value buffers"; return IFGF_ENOMEM; }
        for (int d = 3; d <= D; ++d) pd.lev[d].F = bufs[d & 1];
    }
    p->sig_sorted = ifgf_dalloc(p, (size_t)n * p->rhs_chunk * eb);
    p->u_sorted = ifgf_dalloc(p, (size_t)n * p->rhs_chunk * eb);
    if (!p->sig_sorted || !p->u_sorted) { p->last_error = "sorted density buffers"; return IFGF_ENOMEM; }

    // Upward tables: the geometry of the step d -> d-1 depends only on (parent cone id,
    // child octant, node).  Tabulate it where the table has at most half as many
    // entries as the level has upward evaluations per apply and fits the memory left
    // after the value buffers (finest levels first): all of it but the reserve in
    // two-buffer plans, whose adjoint builds its transpose lists level by level inside
    // the reserve, and half of it otherwise.
    const size_t entry_bytes = ifgf_uptable_entry_bytes(p->precision, Ps, Pang);
    for (int d = D; d >= 4; --d) {
        LevelDev &L = pd.lev[d];
        LevelDev &Lp = pd.lev[d - 1];
        int64_t nw = Lp.words;
        DALLOC(ubits, uint64_t, nw);
        CK(cudaMemsetAsync(ubits, 0, nw * sizeof(uint64_t), st));
        int64_t tot = (int64_t)Lp.nbox * Lp.words;
        k_union_bits<<<nblocks(tot), kThreads, 0, st>>>(Lp.bits, Lp.nbox, Lp.words, ubits);
        CK(cudaGetLastError());
        Scratch cnt;
        if (!cnt.alloc((size_t)(nw + 1) * 4)) return IFGF_ENOMEM;
        CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(nw + 1) * 4, st));
        k_popc<<<nblocks(nw), kThreads, 0, st>>>(ubits, nw, (int *)cnt.ptr);
        CK(cudaGetLastError());
        DALLOC(urank, int, nw + 1);
        ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, urank, nw + 1, st);
        if (s != IFGF_OK) return s;
        int rows = 0;
        CK(cudaMemcpy(&rows, urank + nw, sizeof(int), cudaMemcpyDeviceToHost));
        p->lh[d].union_rows = rows;
        int64_t entries = (int64_t)rows * 8 * P;
        size_t bytes = (size_t)entries * entry_bytes;
        size_t freeb = 0, totalb = 0;
        CK(cudaMemGetInfo(&freeb, &totalb));
        // keep room for the adjoint's cone values, allocated on the first adjoint call
        // (as large as the forward values of a plan that keeps every level)
        const size_t reserve = std::min(kReserveBytes, totalb / 10) + (p->pingpong ? 0 : value_bytes);
        const size_t room = freeb > reserve ? (p->pingpong ? freeb - reserve : (freeb - reserve) / 2) : 0;
        if ((p->flags & 2) || rows == 0 || 2 * entries > p->lh[d].upward_evals || bytes > room) continue;
        DALLOC(uids, int, rows);
        Scratch dummy;
        if (!dummy.alloc((size_t)rows * 4)) return IFGF_ENOMEM;
        k_expand<<<nblocks(nw), kThreads, 0, st>>>(ubits, urank, nw, Lp.words, uids, (int *)dummy.ptr);
        CK(cudaGetLastError());
        void *tab = ifgf_dalloc(p, bytes);
        if (!tab) { p->last_error = "upward table"; return IFGF_ENOMEM; }
        L.ubits = ubits;
        L.urank = urank;
        L.uids = uids;
        L.urows = rows;
        CK(p->precision == IFGF_FP64 ? ifgf_build_uptable_f64(pd, d, tab, st)
                                     : ifgf_build_uptable_f32(pd, d, tab, st));
        L.utab = tab;
        p->lh[d].table_rows = rows;
        CK(cudaStreamSynchronize(st));
    }

    // Evaluation caches: the cousin targets' slots, weights and centred factors, and
    // the geometry of untabled upward levels, computed once here instead of at every
    // apply.  Built when they take at most a quarter of the free memory (flags bit 5
    // turns them off; batched plans have their own target cache).
    if (!(p->flags & 32) && !ifgf_is_batched(p->precision)) {
        const bool f64 = p->precision == IFGF_FP64;
        const size_t te = Ps == 3 && Pang == 5 ? (f64 ? sizeof(TEntry64) : sizeof(TEntry32)) : 0;
        const size_t ue = ifgf_uptable_entry_bytes(p->precision, Ps, Pang);
        size_t need = 0;
        bool fits32 = true;
        for (int d = 3; d <= D; ++d) {
            need += (size_t)p->lh[d].cousin_evals * te;
            fits32 = fits32 && p->lh[d].cousin_evals < ((int64_t)1 << 31);
            if (d >= 4 && !pd.lev[d].utab) {
                need += (size_t)p->lh[d].upward_evals * ue;
                fits32 = fits32 && p->lh[d].upward_evals < ((int64_t)1 << 31);
            }
        }
        size_t freeb = 0, totalb = 0;
        CK(cudaMemGetInfo(&freeb, &totalb));
        if (fits32 && need > 0 && need <= freeb / 4) {
            for (int d = 3; d <= D; ++d) {
                LevelDev &L = pd.lev[d];
                if (te > 0 && p->lh[d].cousin_evals > 0) {
                    Scratch cnt;
                    if (!cnt.alloc((size_t)(n + 1) * 4)) return IFGF_ENOMEM;
                    CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(n + 1) * 4, st));
                    k_point_cousin_count<<<nblocks(n), kThreads, 0, st>>>(pd, d, (int *)cnt.ptr);
                    CK(cudaGetLastError());
                    DALLOC(toff, int, n + 1);
                    ifgf_status s2 = cub_exclusive_sum(p, (int *)cnt.ptr, toff, n + 1, st);
                    if (s2 != IFGF_OK) return s2;
                    void *tc = ifgf_dalloc(p, (size_t)p->lh[d].cousin_evals * te);
                    if (!tc) { p->last_error = "target cache"; return IFGF_ENOMEM; }
                    L.toff = toff;
                    L.tcache = tc;
                    CK(f64 ? ifgf_build_evalcache_f64(pd, d, 0, st) : ifgf_build_evalcache_f32(pd, d, 0, st));
                }
                if (d >= 4 && !L.utab && p->lh[d].upward_evals > 0) {
                    LevelDev &Lp = pd.lev[d - 1];
                    Scratch cnt;
                    if (!cnt.alloc((size_t)(Lp.nact + 1) * 4)) return IFGF_ENOMEM;
                    CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(Lp.nact + 1) * 4, st));
                    k_parent_slot_count<<<nblocks(Lp.nact), kThreads, 0, st>>>(pd, d, (int *)cnt.ptr);
                    CK(cudaGetLastError());
                    DALLOC(uoff, int, Lp.nact + 1);
                    ifgf_status s2 = cub_exclusive_sum(p, (int *)cnt.ptr, uoff, Lp.nact + 1, st);
                    if (s2 != IFGF_OK) return s2;
                    void *uc = ifgf_dalloc(p, (size_t)p->lh[d].upward_evals * ue);
                    if (!uc) { p->last_error = "upward cache"; return IFGF_ENOMEM; }
                    L.uoff = uoff;
                    L.ucache = uc;
                    CK(f64 ? ifgf_build_evalcache_f64(pd, d, 1, st) : ifgf_build_evalcache_f32(pd, d, 1, st));
                }
            }
            CK(cudaStreamSynchronize(st));
            p->cache_bytes = need;
        }
    }

    CK(cudaStreamSynchronize(st));
    int herr = 0;
    CK(cudaMemcpy(&herr, pd.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) { p->last_error = "plan build: internal invariant failed"; return IFGF_EINTERNAL; }
    p->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return IFGF_OK;
}

// Transpose lists for the adjoint: for every relevant cone slot of level d, the
// cousin targets whose interpolation reads it, and the parent interpolation points
// (parent slot * P + node) whose upward interpolation reads it; both in ascending
// order within a slot (stable radix sort by slot).
static ifgf_status sort_to_csr(ifgf_plan *p, int *keys, int *vals, int64_t m, int nslot, int **start_out,
                               int **list_out, cudaStream_t st)
{
    DALLOC(list, int, m);
    DALLOC(start, int, nslot + 1);
    Scratch kb;
    if (!kb.alloc((size_t)m * 4)) { p->last_error = "adjoint list sort"; return IFGF_ENOMEM; }
    int end_bit = 1;
    while (end_bit < 31 && (1 << end_bit) <= nslot) ++end_bit;
    size_t bytes = 0;
    CK(cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys, (int *)kb.ptr, vals, list, m, 0, end_bit, st));
    Scratch tmp;
    if (!tmp.alloc(bytes)) { p->last_error = "adjoint list sort temp"; return IFGF_ENOMEM; }
    CK(cub::DeviceRadixSort::SortPairs(tmp.ptr, bytes, keys, (int *)kb.ptr, vals, list, m, 0, end_bit, st));
    k_csr_from_sorted<<<nblocks(nslot + 1), kThreads, 0, st>>>((int *)kb.ptr, m, nslot, start);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    *start_out = start;
    *list_out = list;
    return IFGF_OK;
}

// adjoint cone-value buffers (allocated on the first adjoint call)
ifgf_status ifgf_alloc_adjoint_values(ifgf_plan *p)
{
    if (p->adjoint_values_ready) return IFGF_OK;
    const size_t eb = ifgf_elem_bytes(p->precision);
    if (!p->pingpong) {
        for (int d = 3; d <= p->D; ++d) {
            LevelDev &L = p->dev.lev[d];
            L.Fadj = ifgf_dalloc(p, (size_t)L.nact * p->P * p->rhs_chunk * eb);
            if (!L.Fadj) { p->last_error = "adjoint value buffer"; return IFGF_ENOMEM; }
        }
    } else {
        // the adjoint needs levels d-1 and d at a time, like the forward step, and a plan
        // runs one evaluation at a time on its stream: the adjoint reuses the forward's
        // two alternating buffers
        for (int d = 3; d <= p->D; ++d) p->dev.lev[d].Fadj = p->dev.lev[d].F;
    }
    p->adjoint_values_ready = true;
    return IFGF_OK;
}

ifgf_status ifgf_build_adjoint_lists(ifgf_plan *p, cudaStream_t st)
{
    if (p->adjoint_ready) return IFGF_OK;
    PlanDev &pd = p->dev;
    const int n = (int)p->n, D = p->D, P = p->P;
    const size_t eb = ifgf_elem_bytes(p->precision);
    (void)eb;
    for (int d = 3; d <= D; ++d) {
        LevelDev &L = pd.lev[d];
        // targets
        {
            Scratch cnt, off;
            if (!cnt.alloc((size_t)(n + 1) * 4) || !off.alloc((size_t)(n + 1) * 4)) return IFGF_ENOMEM;
            CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(n + 1) * 4, st));
            k_point_cousin_count<<<nblocks(n), kThreads, 0, st>>>(pd, d, (int *)cnt.ptr);
            CK(cudaGetLastError());
            ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, (int *)off.ptr, n + 1, st);
            if (s != IFGF_OK) return s;
            int m = 0;
            CK(cudaMemcpy(&m, (int *)off.ptr + n, sizeof(int), cudaMemcpyDeviceToHost));
            Scratch keys, vals;
            if (!keys.alloc((size_t)m * 4) || !vals.alloc((size_t)m * 4)) return IFGF_ENOMEM;
            k_emit_tlist<<<nblocks(n), kThreads, 0, st>>>(pd, d, (int *)off.ptr, (int *)keys.ptr, (int *)vals.ptr);
            CK(cudaGetLastError());
            int *start = nullptr, *list = nullptr;
            if (L.tcache && P == 75 && m > 0) {
                // an entry's emission offset is its index in the level's target cache
                // (both are the per-point cousin-count prefix): sort the offsets, then
                // gather the points, so the adjoint reads the cached geometry
                Scratch idx;
                if (!idx.alloc((size_t)m * 4)) return IFGF_ENOMEM;
                k_iota<<<nblocks(m), kThreads, 0, st>>>((int *)idx.ptr, m);
                CK(cudaGetLastError());
                s = sort_to_csr(p, (int *)keys.ptr, (int *)idx.ptr, m, L.nact, &start, &list, st);
                if (s != IFGF_OK) return s;
                DALLOC(pts_list, int, m);
                k_gather_int<<<nblocks(m), kThreads, 0, st>>>(pts_list, (const int *)vals.ptr, list, m);
                CK(cudaGetLastError());
                CK(cudaStreamSynchronize(st));
                L.tl_start = start;
                L.tl = pts_list;
                L.tl_cache = list;
            } else {
                s = sort_to_csr(p, (int *)keys.ptr, (int *)vals.ptr, m, L.nact, &start, &list, st);
                if (s != IFGF_OK) return s;
                L.tl_start = start;
                L.tl = list;
            }
            if (ifgf_is_batched(p->precision) && !(p->flags & 4) && m > 0) {
                DALLOC(tloc, float4, m);
                DALLOC(tfac, float2, m);
                CK(ifgf_cache_target_geometry(pd, d, tloc, tfac, m, st));
                L.tl_loc = tloc;
                L.tl_fac = tfac;
            }
        }
        if (d >= 4) {
            LevelDev &Lp = pd.lev[d - 1];
            Scratch cnt, off;
            if (!cnt.alloc((size_t)(Lp.nact + 1) * 4) || !off.alloc((size_t)(Lp.nact + 1) * 4)) return IFGF_ENOMEM;
            CK(cudaMemsetAsync(cnt.ptr, 0, (size_t)(Lp.nact + 1) * 4, st));
            k_parent_slot_count<<<nblocks(Lp.nact), kThreads, 0, st>>>(pd, d, (int *)cnt.ptr);
            CK(cudaGetLastError());
            ifgf_status s = cub_exclusive_sum(p, (int *)cnt.ptr, (int *)off.ptr, Lp.nact + 1, st);
            if (s != IFGF_OK) return s;
            int m = 0;
            CK(cudaMemcpy(&m, (int *)off.ptr + Lp.nact, sizeof(int), cudaMemcpyDeviceToHost));
            Scratch keys, vals;
            if (!keys.alloc((size_t)m * 4) || !vals.alloc((size_t)m * 4)) return IFGF_ENOMEM;
            int64_t nt = (int64_t)Lp.nact * P;
            k_emit_ulist<<<nblocks(nt), kThreads, 0, st>>>(pd, d, (int *)off.ptr, (int *)keys.ptr, (int *)vals.ptr);
            CK(cudaGetLastError());
            int *start = nullptr, *list = nullptr;
            s = sort_to_csr(p, (int *)keys.ptr, (int *)vals.ptr, m, L.nact, &start, &list, st);
            if (s != IFGF_OK) return s;
            L.ul_start = start;
            L.ul = list;
        }
    }
    int herr = 0;
    CK(cudaMemcpy(&herr, pd.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) { p->last_error = "adjoint lists: a cone lookup missed"; return IFGF_EINTERNAL; }
    p->adjoint_ready = true;
    return IFGF_OK;
}

// ---------------------------------------------------------------------------------
// Just-in-time transpose lists (adjoint of two-buffer plans).  The resident lists of
// ifgf_build_adjoint_lists cost 4 bytes per cousin and per upward evaluation for all
// levels at once (about 190 GB for the 256-wavelength sphere); these are built for one
// level, and the upward ones for a range of parent boxes, right before use.
// ---------------------------------------------------------------------------------
namespace {

// stable sort of (key, value) pairs by key into list, and CSR starts over nslot keys
ifgf_status sort_into_csr(ifgf_plan *p, int *keys, int *vals, int64_t m, int nslot, int *start, int *list,
                          JitWork *w, cudaStream_t st)
{
    if (!w->sorted.ensure((size_t)m * 4)) { p->last_error = "adjoint list sort"; return IFGF_ENOMEM; }
    int end_bit = 1;
    while (end_bit < 31 && (1 << end_bit) <= nslot) ++end_bit;
    size_t bytes = 0;
    CK(cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys, (int *)w->sorted.ptr, vals, list, m, 0, end_bit, st));
    if (!w->sort_tmp.ensure(bytes)) { p->last_error = "adjoint list sort temp"; return IFGF_ENOMEM; }
    CK(cub::DeviceRadixSort::SortPairs(w->sort_tmp.ptr, bytes, keys, (int *)w->sorted.ptr, vals, list, m, 0, end_bit,
                                       st));
    k_csr_from_sorted<<<nblocks(nslot + 1), kThreads, 0, st>>>((int *)w->sorted.ptr, m, nslot, start);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return IFGF_OK;
}

// exclusive prefix sum with the scan temporary of the workspace
ifgf_status jit_exclusive_sum(ifgf_plan *p, const int *in, int *out, int64_t n, JitWork *w, cudaStream_t st)
{
    size_t bytes = 0;
    CK(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, st));
    if (!w->scan_tmp.ensure(bytes)) { p->last_error = "scan scratch"; return IFGF_ENOMEM; }
    CK(cub::DeviceScan::ExclusiveSum(w->scan_tmp.ptr, bytes, in, out, n, st));
    CK(cudaStreamSynchronize(st));
    return IFGF_OK;
}

// start [nslot + 1] and list [m] in the list's own (grow-only) buffer
ifgf_status jit_alloc(ifgf_plan *p, JitLists *out, int nslot, int64_t m)
{
    const size_t sb = ((size_t)(nslot + 1) * 4 + 255) / 256 * 256;
    if (!out->mem.ensure(sb + (size_t)m * 4 + 16)) {
        p->last_error = "just-in-time adjoint lists";
        return IFGF_ENOMEM;
    }
    out->start = (int *)out->mem.ptr;
    out->list = (int *)((char *)out->mem.ptr + sb);
    return IFGF_OK;
}

}  // namespace

void ifgf_jit_release(JitLists *l)
{
    l->mem.release();
    *l = JitLists();
}

ifgf_status ifgf_jit_targets(ifgf_plan *p, int d, JitLists *out, JitWork *w, cudaStream_t st)
{
    PlanDev &pd = p->dev;
    const LevelDev &L = pd.lev[d];
    const int n = (int)p->n;
    if (!w->cnt.ensure((size_t)(n + 1) * 4) || !w->off.ensure((size_t)(n + 1) * 4)) return IFGF_ENOMEM;
    int *cnt = (int *)w->cnt.ptr, *off = (int *)w->off.ptr;
    CK(cudaMemsetAsync(cnt, 0, (size_t)(n + 1) * 4, st));
    k_point_cousin_count<<<nblocks(n), kThreads, 0, st>>>(pd, d, cnt);
    CK(cudaGetLastError());
    ifgf_status s = jit_exclusive_sum(p, cnt, off, n + 1, w, st);
    if (s != IFGF_OK) return s;
    int m = 0;
    CK(cudaMemcpy(&m, off + n, sizeof(int), cudaMemcpyDeviceToHost));
    if (!w->keys.ensure((size_t)m * 4) || !w->vals.ensure((size_t)m * 4)) return IFGF_ENOMEM;
    k_emit_tlist<<<nblocks(n), kThreads, 0, st>>>(pd, d, off, (int *)w->keys.ptr, (int *)w->vals.ptr);
    CK(cudaGetLastError());
    s = jit_alloc(p, out, L.nact, m);
    if (s != IFGF_OK) return s;
    out->s0 = 0;
    out->s1 = L.nact;
    return sort_into_csr(p, (int *)w->keys.ptr, (int *)w->vals.ptr, m, L.nact, out->start, out->list, w, st);
}

ifgf_status ifgf_jit_chunks(ifgf_plan *p, int d, int64_t max_entries, std::vector<int> *bounds)
{
    const LevelDev &Lp = p->dev.lev[d - 1];
    const int nb = Lp.nbox;
    std::vector<int> as(nb + 1), cs(nb + 1);
    CK(cudaMemcpy(as.data(), Lp.act_start, (size_t)(nb + 1) * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cs.data(), Lp.child_start, (size_t)(nb + 1) * 4, cudaMemcpyDeviceToHost));
    bounds->assign(1, 0);
    int64_t acc = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t e = (int64_t)(as[b + 1] - as[b]) * p->P * (cs[b + 1] - cs[b]);
        if (e > INT32_MAX) { p->last_error = "a parent box with more than 2^31 upward evaluations"; return IFGF_EINVAL; }
        if (acc > 0 && acc + e > max_entries) {
            bounds->push_back(b);
            acc = 0;
        }
        acc += e;
    }
    bounds->push_back(nb);
    return IFGF_OK;
}

ifgf_status ifgf_jit_upward(ifgf_plan *p, int d, int b0, int b1, JitLists *out, JitWork *w, cudaStream_t st)
{
    PlanDev &pd = p->dev;
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    int q[2], cb[2], sl[2];
    CK(cudaMemcpy(&q[0], Lp.act_start + b0, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&q[1], Lp.act_start + b1, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&cb[0], Lp.child_start + b0, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&cb[1], Lp.child_start + b1, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&sl[0], L.act_start + cb[0], 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&sl[1], L.act_start + cb[1], 4, cudaMemcpyDeviceToHost));
    const int nq = q[1] - q[0], ns = sl[1] - sl[0];
    if (!w->cnt.ensure((size_t)(nq + 1) * 4) || !w->off.ensure((size_t)(nq + 1) * 4)) return IFGF_ENOMEM;
    int *cnt = (int *)w->cnt.ptr, *off = (int *)w->off.ptr;
    CK(cudaMemsetAsync(cnt, 0, (size_t)(nq + 1) * 4, st));
    if (nq > 0) k_parent_slot_count_range<<<nblocks(nq), kThreads, 0, st>>>(pd, d, q[0], q[1], cnt);
    CK(cudaGetLastError());
    ifgf_status s = jit_exclusive_sum(p, cnt, off, nq + 1, w, st);
    if (s != IFGF_OK) return s;
    int m = 0;
    CK(cudaMemcpy(&m, off + nq, sizeof(int), cudaMemcpyDeviceToHost));
    if (!w->keys.ensure((size_t)m * 4) || !w->vals.ensure((size_t)m * 4)) return IFGF_ENOMEM;
    const int64_t nt = (int64_t)nq * pd.P;
    if (nt > 0)
        k_emit_ulist_range<<<nblocks(nt), kThreads, 0, st>>>(pd, d, q[0], q[1], sl[0], off, (int *)w->keys.ptr,
                                                             (int *)w->vals.ptr);
    CK(cudaGetLastError());
    s = jit_alloc(p, out, ns, m);
    if (s != IFGF_OK) return s;
    out->s0 = sl[0];
    out->s1 = sl[1];
    if (m == 0) {
        CK(cudaMemsetAsync(out->start, 0, (size_t)(ns + 1) * 4, st));
        CK(cudaStreamSynchronize(st));
        return IFGF_OK;
    }
    return sort_into_csr(p, (int *)w->keys.ptr, (int *)w->vals.ptr, m, ns, out->start, out->list, w, st);
}
