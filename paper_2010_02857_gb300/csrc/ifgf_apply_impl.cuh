// Evaluation kernels of the IFGF method (Algorithm 1, evaluation stage) and of its
// exact adjoint, templated on the value type T (double: all-FP64; float: FP64
// geometry and phase arguments, FP32 interpolation and accumulation), on the
// number R of right-hand sides a thread carries, and on the interpolation orders
// (PS, PA) = (P_s, P_ang).
//
// Forward (u = A sigma), all in pull form so every output has one writer and a
// fixed summation order (bitwise reproducible, no atomics):
//   k_leaf    F_k^D at the interpolation points of every relevant leaf cone
//             (Eq. I_k with d = D): one thread per (cone, point).
//   k_upward  F_j^{d-1} at the parent cones' interpolation points from the children's
//             interpolants, re-centred by G(x, x_k^d) / G(x, x_j^{d-1}): one thread
//             per (parent cone, point), looping over the children.
//   k_near_staged  per run of at most 32 targets of a leaf box (one block): level-D
//             direct sums over the neighbouring boxes (skipping the self term), the
//             sources staged through shared memory with cp.async; also the adjoint's
//             conjugated sums.
//   k_eval    per target: for d = D..3, interpolation from every cousin box's cone
//             times G(x, x_k^d), added to the near field.
// Adjoint (w = A^H v), same data, transposed:
//   k_adj_level1 / k_adj_level  per relevant cone slot of level d (one warp per slot):
//             conjugated contributions of the cousin targets that read the slot and of
//             the parent interpolation points that read it (transpose lists); the
//             first sum-factorised for one right-hand side, the second R-blocked.
//   k_adj_eval   per source: conj(g) of its leaf's cone values, added to the
//             conjugated near field.
#pragma once

#include "ifgf_device.cuh"

// launch of the FP32 kernels blocked for 4 right-hand sides (ifgf_apply_f32_r4.cu)
cudaError_t ifgf_launch_f32_r4(const PlanDev &pd, int nrhs, const void *in, void *out, int mode, int adjoint,
                               cudaStream_t st, StageTimer &tm);
// the FP32 upward step d -> d-1 for more than 4 right-hand sides: the run kernel on
// blocks of 4 (ifgf_apply_f32_r4.cu)
void ifgf_upward_runs_blocks(const PlanDev &pd, int d, int nrhs, cudaStream_t st);

namespace ifgf {

constexpr double kInv4Pi = 0.079577471545947667884441881686257181;

inline int grid_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <typename T> struct Vec { using type = double2; };
template <> struct Vec<float> { using type = float2; };

template <typename T> __device__ __forceinline__ cpx<T> ld(const void *base, size_t i)
{
    if constexpr (sizeof(T) == 8) {
        double2 v = __ldg((const double2 *)base + i);
        return {v.x, v.y};
    } else {
        float2 v = __ldg((const float2 *)base + i);
        return {v.x, v.y};
    }
}
template <typename T> __device__ __forceinline__ void st(void *base, size_t i, cpx<T> v)
{
    if constexpr (sizeof(T) == 8) ((double2 *)base)[i] = make_double2(v.x, v.y);
    else ((float2 *)base)[i] = make_float2(v.x, v.y);
}

// Lagrange weights of the three local coordinates
template <typename T, int PS, int PA>
__device__ __forceinline__ void weights3(const PlanDev &pd, const double *loc, T *ws, T *wt, T *wp)
{
    if constexpr (sizeof(T) == 8) {
        lagrange<T>(PS, pd.ts, pd.its, loc[0], ws);
        lagrange<T>(PA, pd.ta, pd.ita, loc[1], wt);
        lagrange<T>(PA, pd.ta, pd.ita, loc[2], wp);
    } else {
        lagrange(PS, pd.tsf, pd.itsf, (float)loc[0], ws);
        lagrange(PA, pd.taf, pd.itaf, (float)loc[1], wt);
        lagrange(PA, pd.taf, pd.itaf, (float)loc[2], wp);
    }
}

// sum_{a,b,c} ws[a] wt[b] wp[c] F[(a PA + b) PA + c][r], sum-factorised (phi, theta, s)
template <typename T, int R, int PS, int PA>
__device__ __forceinline__ void contract(const void *F, size_t base, int nrhs, int r0, const T *ws,
                                         const T *wt, const T *wp, cpx<T> *out)
{
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = {T(0), T(0)};
#pragma unroll
    for (int a = 0; a < PS; ++a) {
        cpx<T> mid[R];
#pragma unroll
        for (int r = 0; r < R; ++r) mid[r] = {T(0), T(0)};
#pragma unroll
        for (int b = 0; b < PA; ++b) {
            cpx<T> in[R];
#pragma unroll
            for (int r = 0; r < R; ++r) in[r] = {T(0), T(0)};
#pragma unroll
            for (int c = 0; c < PA; ++c) {
                size_t idx = (base + (size_t)((a * PA + b) * PA + c)) * nrhs + r0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (R == 1 || r0 + r < nrhs) {
                        cpx<T> f = ld<T>(F, idx + r);
                        in[r].x += wp[c] * f.x;
                        in[r].y += wp[c] * f.y;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) { mid[r].x += wt[b] * in[r].x; mid[r].y += wt[b] * in[r].y; }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) { out[r].x += ws[a] * mid[r].x; out[r].y += ws[a] * mid[r].y; }
    }
}

// |v| in FP64.  Double plans: correctly rounded sqrt.  Float plans: FP32 rsqrt plus
// one FP64 Newton step (relative error < 1e-13), enough for phase arguments.
template <typename T> __device__ __forceinline__ double dist(double dx, double dy, double dz)
{
    double r2 = dx * dx + dy * dy + dz * dz;
    if constexpr (sizeof(T) == 8) {
        return sqrt(r2);
    } else {
        double y = (double)rsqrtf((float)r2);
        y = y * (1.5 - 0.5 * r2 * y * y);
        return r2 * y;
    }
}

// 1/sqrt(r2) in FP64 without an FP64 square root or division: the FP32 estimate
// (relative error about 2^-23) and two Newton steps, each of which squares the
// relative error, so the result is within a few ulp.  Outside the FP32 range of r2 the
// plain FP64 operations are used.
__device__ __forceinline__ double rsqrt64(double r2)
{
    if (!(r2 > 1e-30 && r2 < 1e30)) return 1.0 / sqrt(r2);
    double y = (double)rsqrtf((float)r2);
    y = y * fma(-0.5 * r2, y * y, 1.5);
    y = y * fma(-0.5 * r2, y * y, 1.5);
    return y;
}

// e^{i kappa r} / (4 pi r) in FP64 from r^2
__device__ __forceinline__ cpx<double> green_r2_64(double kappa, double r2)
{
    const double y = rsqrt64(r2);
    const double a = kInv4Pi * y;
    if (kappa == 0.0) return {a, 0.0};  // Laplace kernel: no phase
    double c, s;
    expi(kappa * (r2 * y), c, s);
    return {a * c, a * s};
}

// e^{i kappa r} / (4 pi r)
template <typename T> __device__ __forceinline__ cpx<T> green_r(double kappa, double r)
{
    T a;
    if constexpr (sizeof(T) == 8) a = kInv4Pi / r;
    else a = (float)kInv4Pi / (float)r;
    if (kappa == 0.0) return {a, T(0)};  // Laplace kernel: no phase
    T c, s;
    expi(kappa * r, c, s);
    return {a * c, a * s};
}

// Near-field distances of float plans without FP64 per pair.  Target and source
// positions relative to the centre c of the target's leaf box are formed once each in
// FP64 and split into FP32 high and low parts (the near-field kernels stage the
// sources' splits in shared memory).  The difference of the high parts is exact when
// the two points are close (Sterbenz), so r = |p - o_j| has FP32 relative accuracy for
// every pair; the phase kappa r then carries an absolute error of about kappa r * 6e-8.
struct Rel32 {
    float hx, hy, hz, lx, ly, lz;
};

__device__ __forceinline__ Rel32 rel32(double x, double y, double z, const double *c)
{
    const double px = x - c[0], py = y - c[1], pz = z - c[2];
    Rel32 p;
    p.hx = (float)px;
    p.hy = (float)py;
    p.hz = (float)pz;
    p.lx = (float)(px - (double)p.hx);
    p.ly = (float)(py - (double)p.hy);
    p.lz = (float)(pz - (double)p.hz);
    return p;
}

// e^{i kappa r} / (4 pi r) for r = |p - o_j| (FP32 only)
__device__ __forceinline__ cpx<float> green_near32(const Rel32 &p, const float4 &oh, const float4 &ol, float kf)
{
    const float dx = (p.hx - oh.x) + (p.lx - ol.x);
    const float dy = (p.hy - oh.y) + (p.ly - ol.y);
    const float dz = (p.hz - oh.z) + (p.lz - ol.z);
    // r^2 > 0 (the self term is skipped by index); 1/r from the SFU's reciprocal square root
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float y = rsqrtf(r2);
    const float a = (float)kInv4Pi * y;
    if (kf == 0.f) return {a, 0.f};  // Laplace kernel: no phase
    float c, s;
    expi_f32(kf * (r2 * y), c, s);
    return {a * c, a * s};
}

// Analytic factor g(q, x_j) = (R/|q - x_j|) e^{i kappa (|q - x_j| - R)} (Eq. factored_f) for
// an interpolation point q = x_k + R dir of a leaf cone and a source x_j = x_k + delta in
// the same leaf box.  Double plans evaluate it as written.  Float plans use
// |q - x_j| - R = (|delta|^2 - 2 R dir.delta) / (|q - x_j| + R), all in FP32 from the
// stored FP32 offset delta and |delta|^2: no difference of nearly equal numbers is
// formed, so the absolute error of the numerator is about eps32 * 2 R |delta| and the
// phase error about kappa |delta| eps32 (below 1e-6 rad for leaf boxes of a wavelength
// at kappa = 800).
// FP32 leaf factor from the node's FP32 constants (R, dir, kappa) and the source's
// stored offset o = (delta, |delta|^2)
__device__ __forceinline__ cpx<float> leaf_factor32(float Rf, float dx, float dy, float dz, float kf, const float4 &o)
{
    const float num = fmaf(-2.0f * Rf, fmaf(dx, o.x, fmaf(dy, o.y, dz * o.z)), o.w);
    // |q - x_j|^2 and its reciprocal square root (the SFU's, 2 ulp): the amplitude R / r1
    // and r1 itself from one special-function operation
    const float r2 = fmaxf(fmaf(Rf, Rf, num), 0.f);
    const float y = rsqrtf(r2);
    const float a = Rf * y;
    if (kf == 0.f) return {a, 0.f};  // Laplace kernel: no phase
    const float ph = __fdividef(kf * num, fmaf(r2, y, Rf));
    float c, s;
    expi_f32(ph, c, s);
    return {a * c, a * s};
}

template <typename T>
__device__ __forceinline__ cpx<T> leaf_factor(const PlanDev &pd, double R, const double *q, const double *dir, int j)
{
    if constexpr (sizeof(T) == 8) {
        const double dx = q[0] - pd.xs[j], dy = q[1] - pd.ys[j], dz = q[2] - pd.zs[j];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double y = rsqrt64(r2);
        const double a = R * y;
        if (pd.kappa == 0.0) return {a, 0.0};  // Laplace kernel: no phase
        double c, s;
        expi(pd.kappa * (r2 * y - R), c, s);
        return {a * c, a * s};
    } else {
        // the quotient and the reciprocal square root need FP32 relative accuracy only
        // (their arguments lie far inside the range where the fast forms are accurate to
        // 2 ulp)
        return leaf_factor32((float)R, (float)dir[0], (float)dir[1], (float)dir[2], (float)pd.kappa, pd.leaf_off[j]);
    }
}

// cone cell (bit-identical to cone_of), Lagrange weights and distance of the vector v
template <typename T, int PS, int PA>
__device__ __forceinline__ ConeGeom geom_weights(const PlanDev &pd, const LevelDev &L, double vx, double vy,
                                                 double vz, T *w)
{
    ConeGeom g = sizeof(T) == 8 ? cone_of_fast(L, vx, vy, vz) : cone_of_mixed(L, vx, vy, vz);
    if constexpr (sizeof(T) == 8) {
        double loc[3];
        local_coords(L, g, vx, vy, vz, loc);
        weights3<T, PS, PA>(pd, loc, w, w + PS, w + PS + PA);
    } else {
        float t[3];
        local_coords_f32(L, g, vx, vy, vz, t);
        lagrange(PS, pd.tsf, pd.itsf, t[0], w);
        lagrange(PA, pd.taf, pd.itaf, t[1], w + PS);
        lagrange(PA, pd.taf, pd.itaf, t[2], w + PS + PA);
    }
    return g;
}

// Re-centring factor G(q, x_k) / G(q, x_j) = (r_j / r_k) e^{i kappa (r_k - r_j)} for the
// interpolation point q = x_j + Rj dir, child centre x_k = x_j + delta, r_k = |q - x_k|.
// r_k - r_j = (|delta|^2 - 2 Rj dir.delta) / (r_k + r_j) avoids the cancellation of
// the plain difference.  Float plans evaluate it in FP32: the absolute error of the
// numerator is about eps32 * 2 Rj |delta|, so the phase error is about
// kappa |delta| eps32 (2e-5 rad for the coarsest level of a 256-wavelength sphere).
template <typename T>
__device__ __forceinline__ cpx<T> recentre(double kappa, double Rj, const double *dir, double rk,
                                           double dx, double dy, double dz)
{
    if constexpr (sizeof(T) == 8) {
        T a = Rj / rk;
        if (kappa == 0.0) return {a, T(0)};  // Laplace kernel: a real ratio
        double dd = dx * dx + dy * dy + dz * dz;
        double yd = dir[0] * dx + dir[1] * dy + dir[2] * dz;
        double diff = (dd - 2.0 * Rj * yd) / (rk + Rj);
        T c, s;
        expi(kappa * diff, c, s);
        return {a * c, a * s};
    } else {
        const float Rf = (float)Rj, rkf = (float)rk;
        const float a = __fdividef(Rf, rkf);
        if (kappa == 0.0) return {a, 0.f};  // Laplace kernel: a real ratio
        const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
        const float dd = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        const float yd = fmaf((float)dir[0], fx, fmaf((float)dir[1], fy, (float)dir[2] * fz));
        const float diff = __fdividef(fmaf(-2.0f * Rf, yd, dd), rkf + Rf);
        float c, s;
        expi_f32((float)kappa * diff, c, s);
        return {a * c, a * s};
    }
}

// ---------------------------------------------------------------------------------
template <typename T>
__global__ void k_permute_in(const void *in, void *out, const int *perm, int n, int nrhs)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    int i = (int)(t / nrhs), r = (int)(t % nrhs);
    st<T>(out, t, ld<T>(in, (size_t)r * n + perm[i]));
}

template <typename T>
__global__ void k_permute_out(const void *in, void *out, const int *perm, int n, int nrhs)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    int i = (int)(t / nrhs), r = (int)(t % nrhs);
    st<T>(out, (size_t)r * n + perm[i], ld<T>(in, t));
}

// ---------------------------------------------------------------------------------
// Leaf level: F_k^D(q) = sum_{x' in B_k} sigma(x') |q - x_k| / |q - x'| e^{i kappa (|q - x'| - |q - x_k|)}
// ---------------------------------------------------------------------------------
// One thread per (relevant cone of a leaf box of level d, node): every slot of level D in
// a uniform tree; the leaf boxes' slots of any level in an adaptive one.
template <typename T, int R, int PS, int PA>
__global__ void __launch_bounds__(128) k_leaf(PlanDev pd, int d, int nrhs, const void *sig)
{
    constexpr int P = PS * PA * PA;
    const LevelDev &L = pd.lev[d];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)L.nleaf_slots * P) return;
    const int li = (int)(t / P), node = (int)(t % P);
    const int slot = L.leaf_slots ? L.leaf_slots[li] : li;
    int b = L.act_box[slot];
    const double *c = L.center + 3 * (size_t)b;
    double q[3], dir[3];
    double R0 = node_pos(L, PS, PA, L.act_cone[slot], node, c[0], c[1], c[2], q, dir);
    const int j0 = L.start[b], j1 = L.end[b];
    // FP32 factors: the node's radius, direction and kappa converted once, not per source
    const float Rf = (float)R0, dxf = (float)dir[0], dyf = (float)dir[1], dzf = (float)dir[2];
    const float kf = (float)pd.kappa;
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        cpx<T> acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = {T(0), T(0)};
        for (int j = j0; j < j1; ++j) {
            cpx<T> g;
            if constexpr (sizeof(T) == 8) g = leaf_factor<T>(pd, R0, q, dir, j);
            else g = leaf_factor32(Rf, dxf, dyf, dzf, kf, pd.leaf_off[j]);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (R == 1 || r0 + r < nrhs) {
                    cpx<T> s = ld<T>(sig, (size_t)j * nrhs + r0 + r);
                    cpx<T> m = cmul(s, g);
                    acc[r].x += m.x;
                    acc[r].y += m.y;
                }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r0 + r < nrhs) st<T>(L.F, ((size_t)slot * P + node) * nrhs + r0 + r, acc[r]);
    }
}

// ---------------------------------------------------------------------------------
// Upward step d -> d-1 (d > 3)
// ---------------------------------------------------------------------------------

// Geometry of one upward evaluation: the parent node (cone id `pcone`, node) seen from
// the child centre in octant `oct`: child cone id, Lagrange weights, re-centring
// factor.  Returns false if r = 0 (cannot happen for s <= 1 nodes).
template <typename T, int PS, int PA>
__device__ __forceinline__ int up_geometry(const PlanDev &pd, const LevelDev &L, const LevelDev &Lp, int pcone,
                                           int node, int oct, T *w, cpx<T> &f)
{
    const double hh = L.H * 0.5;
    double v[3], dir[3];
    double Rj = node_rel(Lp, PS, PA, pcone, node, hh, oct, v, dir);
    ConeGeom g = geom_weights<T, PS, PA>(pd, L, v[0], v[1], v[2], w);
    f = recentre<T>(pd.kappa, Rj, dir, g.r, (oct & 1) ? hh : -hh, (oct & 2) ? hh : -hh, (oct & 4) ? hh : -hh);
    return g.cone;
}

// The same geometry for FP32 plans as local coordinates (the form the FP32 tables store).
template <int PS, int PA>
__device__ __forceinline__ int up_geometry_t(const PlanDev &pd, const LevelDev &L, const LevelDev &Lp, int pcone,
                                             int node, int oct, float *tl, cpx<float> &f)
{
    const double hh = L.H * 0.5;
    double v[3], dir[3];
    double Rj = node_rel(Lp, PS, PA, pcone, node, hh, oct, v, dir);
    ConeGeom g = cone_of_mixed(L, v[0], v[1], v[2]);
    local_coords_f32(L, g, v[0], v[1], v[2], tl);
    f = recentre<float>(pd.kappa, Rj, dir, g.r, (oct & 1) ? hh : -hh, (oct & 2) ? hh : -hh, (oct & 4) ? hh : -hh);
    return g.cone;
}

// Weights, factor and child cone from an upward table or cache entry.
template <typename T, int PS, int PA>
__device__ __forceinline__ int up_entry(const PlanDev &pd, const typename UpEntryOf<T, PS + 2 * PA>::type &e, T *w,
                                        cpx<T> &f)
{
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int m = 0; m < PS + 2 * PA; ++m) w[m] = e.w[m];
        f = {e.fr, e.fi};
    } else {
        lagrange(PS, pd.tsf, pd.itsf, e.t[0], w);
        lagrange(PA, pd.taf, pd.itaf, e.t[1], w + PS);
        lagrange(PA, pd.taf, pd.itaf, e.t[2], w + PS + PA);
        f = {e.fr, e.fi};
    }
    return e.cone;
}

// The table or cache entry of one upward evaluation.
template <typename T, int PS, int PA>
__device__ __forceinline__ typename UpEntryOf<T, PS + 2 * PA>::type make_up_entry(const PlanDev &pd, const LevelDev &L,
                                                                                   const LevelDev &Lp, int pcone,
                                                                                   int node, int oct)
{
    typename UpEntryOf<T, PS + 2 * PA>::type e;
    cpx<T> f;
    if constexpr (sizeof(T) == 8) e.cone = up_geometry<T, PS, PA>(pd, L, Lp, pcone, node, oct, e.w, f);
    else e.cone = up_geometry_t<PS, PA>(pd, L, Lp, pcone, node, oct, e.t, f);
    e.fr = f.x;
    e.fi = f.y;
    return e;
}

template <typename T, int PS, int PA>
__global__ void __launch_bounds__(128) k_build_uptable(PlanDev pd, int d, typename UpEntryOf<T, PS + 2 * PA>::type *tab)
{
    constexpr int P = PS * PA * PA;
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)L.urows * 8 * P) return;
    int node = (int)(t % P);
    int oct = (int)((t / P) % 8);
    int row = (int)(t / (8 * P));
    typename UpEntryOf<T, PS + 2 * PA>::type e = make_up_entry<T, PS, PA>(pd, L, Lp, L.uids[row], node, oct);
    // the table's cone id must be the one relevance rule (ii) marked: take the
    // correctly rounded cell (cone_of_fast agrees by construction; this is a check)
    {
        double v[3];
        node_rel(Lp, PS, PA, L.uids[row], node, L.H * 0.5, oct, v, nullptr);
        if (cone_of(L, v[0], v[1], v[2]).cone != e.cone) atomicAdd(pd.err, 1);
    }
    tab[t] = e;
}

template <typename T, int R, int PS, int PA, bool TAB>
__global__ void __launch_bounds__(128) k_upward(PlanDev pd, int d, int nrhs)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Lp.nact * P) return;
    int slot = (int)(t / P), node = (int)(t % P);
    int j = Lp.act_box[slot];
    const int pcone = Lp.act_cone[slot];
    using Entry = typename UpEntryOf<T, NW>::type;
    const Entry *tab = nullptr;
    if constexpr (TAB) {
        int row = table_row(L.ubits, L.urank, pcone);
        if (row < 0) { atomicAdd(pd.err, 1); return; }
        tab = (const Entry *)L.utab + (size_t)row * 8 * P + node;
    }
    const int k0 = Lp.child_start[j], k1 = Lp.child_start[j + 1];
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        cpx<T> acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = {T(0), T(0)};
        for (int k = k0; k < k1; ++k) {
            const int oct = (int)(L.key[k] & 7u);
            T w[NW];
            cpx<T> f;
            int cone;
            if constexpr (TAB) {
                cone = up_entry<T, PS, PA>(pd, tab[(size_t)oct * P], w, f);
            } else if (L.ucache) {
                cone = up_entry<T, PS, PA>(
                    pd, ((const Entry *)L.ucache)[(size_t)L.uoff[slot] + (size_t)node * (k1 - k0) + (k - k0)], w, f);
            } else {
                cone = up_geometry<T, PS, PA>(pd, L, Lp, pcone, node, oct, w, f);
            }
            int sl = cone_slot(L, k, cone);
            if (sl < 0) { atomicAdd(pd.err, 1); continue; }
            cpx<T> val[R];
            contract<T, R, PS, PA>(L.F, (size_t)sl * P, nrhs, r0, w, w + PS, w + PS + PA, val);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cpx<T> m = cmul(f, val[r]);
                acc[r].x += m.x;
                acc[r].y += m.y;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r0 + r < nrhs) st<T>(Lp.F, ((size_t)slot * P + node) * nrhs + r0 + r, acc[r]);
    }
}

// 8- and 16-byte asynchronous copies global -> shared (cp.async), and their wait
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"((uint64_t)__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"((uint64_t)__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// FP32 upward step with the children's cone values staged in shared memory (used where
// the geometry is computed on the fly: one node per lane keeps the FP64 work of the
// geometry dense in every warp).
//
// The thread layout and the arithmetic are those of k_upward (one thread per (parent
// slot, node); children in order; the same sum-factorised contraction), but a warp
// reads cone values from shared memory instead of from L1.  In k_upward the 32 lanes of
// a warp interpolate, at each child step, from the 2-3 child cones their nodes fall in,
// so every value load costs 2-3 L1 wavefronts and the kernel is bound by L1 throughput.
// Here, at each child step, the warp finds the distinct child slots of its lanes
// (__match_any_sync), copies the values of up to kUpStage of them into its shared-memory
// stage (coalesced 16-byte or 8-byte loads), and each lane contracts from its cone's
// copy.  A staged cone takes P * nrhs complex values; the copies follow one another
// without padding, so the copies start 600 * nrhs (mod 32) banks apart: for nrhs = 1..4
// the same node of up to four cones lies in disjoint banks, and a warp's load is one
// shared-memory wavefront whichever of the staged cones its lanes read.  Lanes whose
// cone is beyond the first kUpStage distinct ones (rare) read from global memory.  Every
// lane sums its children in the same order with the same operations as k_upward.
// nrhs <= R <= 4.
constexpr int kUpStage = 4;
constexpr int kUpWarps = 4;

template <int R, int PS, int PA>
__device__ __forceinline__ void contract_staged(const float2 *s, int nrhs, const float *ws, const float *wt,
                                                const float *wp, cpx<float> *out)
{
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < PS; ++a) {
        cpx<float> mid[R];
#pragma unroll
        for (int r = 0; r < R; ++r) mid[r] = {0.f, 0.f};
#pragma unroll
        for (int b = 0; b < PA; ++b) {
            cpx<float> in[R];
#pragma unroll
            for (int r = 0; r < R; ++r) in[r] = {0.f, 0.f};
#pragma unroll
            for (int c = 0; c < PA; ++c) {
                const int idx = (a * PA + b) * PA + c;
                if (R == 4 && nrhs == 4) {
                    const float4 v01 = reinterpret_cast<const float4 *>(s)[idx * 2];
                    const float4 v23 = reinterpret_cast<const float4 *>(s)[idx * 2 + 1];
                    const float v[8] = {v01.x, v01.y, v01.z, v01.w, v23.x, v23.y, v23.z, v23.w};
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        in[r].x += wp[c] * v[2 * r];
                        in[r].y += wp[c] * v[2 * r + 1];
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (R == 1 || r < nrhs) {
                            const float2 v = s[idx * nrhs + r];
                            in[r].x += wp[c] * v.x;
                            in[r].y += wp[c] * v.y;
                        }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) { mid[r].x += wt[b] * in[r].x; mid[r].y += wt[b] * in[r].y; }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) { out[r].x += ws[a] * mid[r].x; out[r].y += ws[a] * mid[r].y; }
    }
}

template <int R, int PS, int PA, bool TAB>
__global__ void __launch_bounds__(32 * kUpWarps) k_upward_staged(PlanDev pd, int d, int nrhs)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) float2 s_up_stage[];
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = t < (int64_t)Lp.nact * P;
    if (__all_sync(kFull, !valid)) return;  // whole warps past the end
    const int slot = valid ? (int)(t / P) : 0, node = valid ? (int)(t % P) : 0;
    const int j = valid ? Lp.act_box[slot] : 0;
    const int pcone = valid ? Lp.act_cone[slot] : 0;
    const UpEntry32 *tab = nullptr;
    if constexpr (TAB) {
        if (valid) {
            const int row = table_row(L.ubits, L.urank, pcone);
            if (row < 0) { atomicAdd(pd.err, 1); valid = false; }
            else tab = (const UpEntry32 *)L.utab + (size_t)row * 8 * P + node;
        }
    }
    const int k0 = valid ? Lp.child_start[j] : 0;
    const int nch = valid ? Lp.child_start[j + 1] - k0 : 0;
    const int maxch = __reduce_max_sync(kFull, nch);
    const int vals = P * nrhs;  // complex values per staged cone
    float2 *stg = s_up_stage + (size_t)warp * kUpStage * vals;
    cpx<float> acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = {0.f, 0.f};
    for (int kk = 0; kk < maxch; ++kk) {
        int sl = -1;
        float w[NW];
        cpx<float> f = {0.f, 0.f};
        if (kk < nch) {
            const int k = k0 + kk;
            const int oct = (int)(L.key[k] & 7u);
            int cone;
            if constexpr (TAB) {
                cone = up_entry<float, PS, PA>(pd, tab[(size_t)oct * P], w, f);
            } else if (L.ucache) {
                cone = up_entry<float, PS, PA>(
                    pd, ((const UpEntry32 *)L.ucache)[(size_t)L.uoff[slot] + (size_t)node * nch + kk], w, f);
            } else {
                cone = up_geometry<float, PS, PA>(pd, L, Lp, pcone, node, oct, w, f);
            }
            sl = cone_slot(L, k, cone);
            if (sl < 0) atomicAdd(pd.err, 1);
        }
        // the warp's distinct child slots; the first kUpStage are staged
        const unsigned same = __match_any_sync(kFull, sl);
        const int leader = __ffs(same) - 1;
        const unsigned leaders = __ballot_sync(kFull, lane == leader && sl >= 0);
        const int mine = sl >= 0 ? __popc(leaders & ((1u << leader) - 1u)) : -1;
        const int nst = min(__popc(leaders), kUpStage);
        unsigned rem = leaders;
        for (int g = 0; g < nst; ++g) {
            const int src = __ffs(rem) - 1;
            rem &= rem - 1u;
            const int gsl = __shfl_sync(kFull, sl, src);
            const float2 *from = (const float2 *)L.F + (size_t)gsl * vals;
            float2 *to = stg + (size_t)g * vals;
            if ((vals & 1) == 0) {
                for (int e = lane; e < vals / 2; e += 32)
                    reinterpret_cast<float4 *>(to)[e] = __ldg(reinterpret_cast<const float4 *>(from) + e);
            } else {
                for (int e = lane; e < vals; e += 32) to[e] = __ldg(from + e);
            }
        }
        __syncwarp();
        if (sl >= 0) {
            cpx<float> val[R];
            if (mine < kUpStage) contract_staged<R, PS, PA>(stg + (size_t)mine * vals, nrhs, w, w + PS, w + PS + PA, val);
            else contract<float, R, PS, PA>(L.F, (size_t)sl * P, nrhs, 0, w, w + PS, w + PS + PA, val);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cpx<float> m = cmul(f, val[r]);
                acc[r].x += m.x;
                acc[r].y += m.y;
            }
        }
        __syncwarp();  // the stage is read before the next child step overwrites it
    }
    if (valid) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r < nrhs) st<float>(Lp.F, ((size_t)slot * P + node) * nrhs + r, acc[r]);
    }
}

// FP32 upward step, one warp per parent cone slot, in runs of nodes that share a child cone.
//
// k_upward gives each thread one (parent slot, node) and interpolates, child by child, from
// the child cone its node falls in.  Every evaluation then reads all P * nrhs values of its
// cone into its registers: one 16-byte load per two complex values and three FMAs per load
// on average, which binds the kernel to the 128 bytes per clock that L1 and shared memory
// deliver.  Here a warp takes one parent slot and, for each child in order:
//   A. computes the geometry of the P nodes (table, cache or on the fly; three per lane)
//      into shared memory: local coordinates, factor, child cone slot;
//   B. groups the nodes by child cone slot (ballots) and cuts each group into runs of at
//      most kRunK nodes, in node order;
//   C. copies the values of the first run_stage_cones(P) cones into the warp's shared-memory stage
//      (coalesced 16-byte loads);
//   D. gives each lane one run: it reads each value of its cone once and applies it to the
//      run's kRunK evaluations (the weight products (ws wt) wp per node, so that only
//      accumulators and weights stay live), and adds factor times value to the node's
//      accumulator in shared memory.
// Every node sums its children in the same order as k_upward; the contraction associates
// its products differently (the same polynomial, equal to FP32 rounding).  Cones beyond
// the first run_stage_cones(P) of a child step are read from global memory.  A child step has at
// most P runs (every group of g nodes gives ceil(g / kRunK)); lanes take them 32 apart, so
// a step with more than 32 runs gives some lanes a second one (each node is in one run,
// so no two lanes write the same accumulator).
constexpr int kRunK = 3;
// cones staged per child step: 4 at (3, 5); 2 at (4, 7), whose cones are 2.6 times larger
// (a parent cone's nodes fall into 1 or 2 cones of a child nearly always)
__host__ __device__ constexpr int run_stage_cones(int P) { return P > 100 ? 2 : 4; }
constexpr int kRunWarps = 2;  // 2 x 14.3 KB of shared memory per CTA (4 right-hand sides), under the 48 KB default

// Shape of the run kernel per register blocking R and cone size P: whether the contraction
// unrolls its angular loops (compile-time weight indices and value offsets, more
// registers), and the CTAs per SM its register budget is sized for.
//   - one right-hand side: unrolled, 6 CTAs (the select chains of the rolled form cost
//     more than its FMAs);
//   - four at (3, 5): rolled, 8 CTAs (measured faster on the 256-wavelength sphere than
//     unrolled at 6; shared memory admits 7 CTAs of 30 KB, which takes 128 registers too);
//   - four at (4, 7): unrolled, 4 CTAs (shared memory admits 4 CTAs of 53 KB).
template <int R, int P>
struct RunShape {
    static constexpr bool unroll_angular = R == 1 || P > 100;
    static constexpr int min_ctas = R == 1 ? 6 : (P > 100 ? 4 : 8);
};

// the run's evaluations: values src[node * stride + r] (r < nb) of one child cone, per evaluation e
// the weights w[e] = (ws (PS), wt (PA), wp (PA)); out[e][r] = sum over the nodes (a, b, c) of
// (ws[a] wt[b]) wp[c] src[(a PA + b) PA + c][r], in node order.  Each value is read once and
// applied to the run's kRunK evaluations; per evaluation only the accumulators and the
// weights are live.  Rolled indices take their weights by selects, so that w stays in
// registers.
template <int R, int PS, int PA>
__device__ __forceinline__ void run_values(const float2 *p, int stride, int nb, float *v)
{
    if (R == 4 && nb == 4 && stride == 4) {
        const float4 v01 = reinterpret_cast<const float4 *>(p)[0];
        const float4 v23 = reinterpret_cast<const float4 *>(p)[1];
        v[0] = v01.x; v[1] = v01.y; v[2] = v01.z; v[3] = v01.w;
        v[4] = v23.x; v[5] = v23.y; v[6] = v23.z; v[7] = v23.w;
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = make_float2(0.f, 0.f);
            if (R == 1 || r < nb) x = p[r];
            v[2 * r] = x.x;
            v[2 * r + 1] = x.y;
        }
    }
}

template <int R, int PS, int PA>
__device__ __forceinline__ void run_fma(const float (*w)[PS + 2 * PA], const float *wab, int c, const float *v,
                                        cpx<float> (*out)[R])
{
#pragma unroll
    for (int e = 0; e < kRunK; ++e) {
        const float wn = wab[e] * w[e][PS + PA + c];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            out[e][r].x += wn * v[2 * r];
            out[e][r].y += wn * v[2 * r + 1];
        }
    }
}

template <int R, int PS, int PA, bool FULL>
__device__ __forceinline__ void contract_run(const float2 *src, int stride_, int nb_, const float (*w)[PS + 2 * PA],
                                             cpx<float> (*out)[R])
{
    // FULL: a packed block of R right-hand sides (the common case), with compile-time strides
    const int stride = FULL ? R : stride_, nb = FULL ? R : nb_;
#pragma unroll
    for (int e = 0; e < kRunK; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) out[e][r] = {0.f, 0.f};
    if constexpr (RunShape<R, PS * PA * PA>::unroll_angular) {
        // a rolled; b and c unrolled
#pragma unroll 1
        for (int a = 0; a < PS; ++a) {
            float wa[kRunK];
#pragma unroll
            for (int e = 0; e < kRunK; ++e) {
                wa[e] = w[e][0];
#pragma unroll
                for (int m = 1; m < PS; ++m)
                    if (a == m) wa[e] = w[e][m];
            }
            const float2 *sa = src + (size_t)a * PA * PA * stride;
#pragma unroll
            for (int b = 0; b < PA; ++b) {
                float wab[kRunK];
#pragma unroll
                for (int e = 0; e < kRunK; ++e) wab[e] = wa[e] * w[e][PS + b];
#pragma unroll
                for (int c = 0; c < PA; ++c) {
                    float v[2 * R];
                    run_values<R, PS, PA>(sa + (size_t)(b * PA + c) * stride, stride, nb, v);
                    run_fma<R, PS, PA>(w, wab, c, v, out);
                }
            }
        }
    } else {
        // (a, b) rolled; c unrolled
#pragma unroll 1
        for (int ab = 0; ab < PS * PA; ++ab) {
            const int a = ab / PA, b = ab - a * PA;
            float wab[kRunK];
#pragma unroll
            for (int e = 0; e < kRunK; ++e) {
                float wa = w[e][0], wb = w[e][PS];
#pragma unroll
                for (int m = 1; m < PS; ++m)
                    if (a == m) wa = w[e][m];
#pragma unroll
                for (int m = 1; m < PA; ++m)
                    if (b == m) wb = w[e][PS + m];
                wab[e] = wa * wb;
            }
            const float2 *sab = src + (size_t)ab * PA * stride;
#pragma unroll
            for (int c = 0; c < PA; ++c) {
                float v[2 * R];
                run_values<R, PS, PA>(sab + (size_t)c * stride, stride, nb, v);
                run_fma<R, PS, PA>(w, wab, c, v, out);
            }
        }
    }
}

// Shared memory of one warp of k_upward_runs for P nodes and nrhs right-hand sides, in this
// order (each array starts on a boundary of its element type; 8-byte arrays first):
//   stage [run_stage_cones(P)][P][nb] complex   (16-byte aligned: the 16-byte copies)
//   acc   [P][R] complex, f [P] complex  (8 bytes)
//   t     [P][3] float, slot [P], runs [P][kRunK], run group [P]  (4 bytes)
// The warp's block is a multiple of 16 bytes, so every warp's stage stays 16-byte aligned.
__host__ __device__ constexpr size_t run_stage_floats(int P, int nb) { return (size_t)run_stage_cones(P) * P * nb * 2; }
__host__ __device__ constexpr size_t run_warp_bytes(int P, int R, int nb)
{
    return ((run_stage_floats(P, nb) + (size_t)P * R * 2 + (size_t)P * 2 + (size_t)P * 3) * 4 + (size_t)P * 4 +
            (size_t)P * kRunK * 4 + (size_t)P * 4 + 15) / 16 * 16;
}

template <int R, int PS, int PA, bool TAB>
__global__ void __launch_bounds__(32 * kRunWarps, RunShape<R, PS * PA * PA>::min_ctas)
    k_upward_runs(PlanDev pd, int d, int nrhs, int r0, int nb)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    constexpr int NCH = (P + 31) / 32;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) float s_runs_raw[];
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = blockIdx.x * kRunWarps + warp;
    if (slot >= Lp.nact) return;  // the whole warp
    // this warp's shared memory
    float *base = (float *)((unsigned char *)s_runs_raw + (size_t)warp * run_warp_bytes(P, R, nb));
    float2 *stage = (float2 *)base;
    float2 *acc = (float2 *)(base + run_stage_floats(P, nb));  // [P][R]
    float2 *gf = acc + (size_t)P * R;                           // [P]
    float *gt = (float *)(gf + P);                              // [P][3]
    int *gsl = (int *)(gt + (size_t)P * 3);                     // [P]
    int *runs = gsl + P;                                        // [P][kRunK]
    int *rgrp = runs + P * kRunK;                               // [P] group of each run
    const int j = Lp.act_box[slot];
    const int pcone = Lp.act_cone[slot];
    const int k0 = Lp.child_start[j], nch = Lp.child_start[j + 1] - k0;
    const UpEntry32 *tab = nullptr;
    if constexpr (TAB) {
        const int row = table_row(L.ubits, L.urank, pcone);
        if (row < 0) {
            if (lane == 0) atomicAdd(pd.err, 1);
            return;
        }
        tab = (const UpEntry32 *)L.utab + (size_t)row * 8 * P;
    }
    for (int q = lane; q < P * R; q += 32) acc[q] = make_float2(0.f, 0.f);
    const int rstep = (pd.flags & 1024) ? 8 : 32;  // lanes taking runs (flags bit 10: 8, testing)
    for (int kk = 0; kk < nch; ++kk) {
        const int k = k0 + kk;
        const int oct = (int)(L.key[k] & 7u);
        // A. geometry of the P nodes
        int sl_c[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int node = lane + 32 * c;
            sl_c[c] = -1;
            if (node < P) {
                float tl[3];
                cpx<float> f;
                int cone;
                if constexpr (TAB) {
                    const UpEntry32 en = tab[(size_t)oct * P + node];
                    tl[0] = en.t[0]; tl[1] = en.t[1]; tl[2] = en.t[2];
                    f = {en.fr, en.fi};
                    cone = en.cone;
                } else if (L.ucache) {
                    const UpEntry32 en = ((const UpEntry32 *)L.ucache)[(size_t)L.uoff[slot] + (size_t)node * nch + kk];
                    tl[0] = en.t[0]; tl[1] = en.t[1]; tl[2] = en.t[2];
                    f = {en.fr, en.fi};
                    cone = en.cone;
                } else {
                    cone = up_geometry_t<PS, PA>(pd, L, Lp, pcone, node, oct, tl, f);
                }
                const int sl = cone_slot(L, k, cone);
                if (sl < 0) atomicAdd(pd.err, 1);
                sl_c[c] = sl;
                gt[3 * node] = tl[0];
                gt[3 * node + 1] = tl[1];
                gt[3 * node + 2] = tl[2];
                gf[node] = make_float2(f.x, f.y);
                gsl[node] = sl;
            }
        }
        // B. groups of nodes with one child slot, in order of their first node; runs
        unsigned pend[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) pend[c] = __ballot_sync(kFull, sl_c[c] >= 0);
        int nruns = 0, ngroups = 0;
        for (int q = lane; q < P * kRunK; q += 32) runs[q] = -1;
        __syncwarp();
        while (true) {
            int c0 = -1;
#pragma unroll
            for (int c = NCH - 1; c >= 0; --c)
                if (pend[c]) c0 = c;
            if (c0 < 0) break;
            unsigned pc = 0;
            int slc = -1;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                if (c == c0) { pc = pend[c]; slc = sl_c[c]; }
            const int g_sl = __shfl_sync(kFull, slc, __ffs(pc) - 1);
            const int g = ngroups++;
            int before = 0;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const bool mem = sl_c[c] == g_sl && ((pend[c] >> lane) & 1u);
                const unsigned m = __ballot_sync(kFull, mem);
                if (mem) {
                    const int rank = before + __popc(m & ((1u << lane) - 1u));
                    runs[(nruns + rank / kRunK) * kRunK + rank % kRunK] = lane + 32 * c;
                }
                before += __popc(m);
                pend[c] &= ~m;
            }
            const int nr = (before + kRunK - 1) / kRunK;
            for (int q = nruns + lane; q < nruns + nr; q += 32) rgrp[q] = g;
            // C. stage this group's cone values (asynchronous copies: the groups' loads
            // overlap, and all complete at the wait below)
            if (g < run_stage_cones(P)) {
                // values [r0, r0 + nb) of each node, packed as [P][nb]
                const float2 *from = (const float2 *)L.F + (size_t)g_sl * P * nrhs + r0;
                float2 *to = stage + (size_t)g * P * nb;
                if (nb == nrhs && (P * nb) % 2 == 0) {  // the whole cone, contiguous
                    for (int q = lane; q < P * nb / 2; q += 32) cp_async16(to + 2 * q, from + 2 * q);
                } else if (nb % 2 == 0 && nrhs % 2 == 0 && r0 % 2 == 0) {  // 16-byte pairs per node
                    for (int q = lane; q < P * nb / 2; q += 32) {
                        const int node = q / (nb / 2), h = q - node * (nb / 2);
                        cp_async16(to + node * nb + 2 * h, from + (size_t)node * nrhs + 2 * h);
                    }
                } else {
                    for (int q = lane; q < P * nb; q += 32) {
                        const int node = q / nb, r = q - node * nb;
                        cp_async8(to + q, from + (size_t)node * nrhs + r);
                    }
                }
            }
            nruns += nr;
        }
        cp_async_wait_all();
        __syncwarp();
        // D. the runs, lane l taking runs l, l + rstep, ...
        if (lane < rstep) {
            for (int r = lane; r < nruns; r += rstep) {
                int nodes[kRunK];
                float w[kRunK][NW];
#pragma unroll
                for (int e = 0; e < kRunK; ++e) {
                    nodes[e] = runs[r * kRunK + e];
                    const int nd = nodes[e] < 0 ? 0 : nodes[e];
                    lagrange(PS, pd.tsf, pd.itsf, gt[3 * nd], w[e]);
                    lagrange(PA, pd.taf, pd.itaf, gt[3 * nd + 1], w[e] + PS);
                    lagrange(PA, pd.taf, pd.itaf, gt[3 * nd + 2], w[e] + PS + PA);
                }
                const int g = rgrp[r];
                cpx<float> val[kRunK][R];
                if (g < run_stage_cones(P)) {
                    const float2 *sg = stage + (size_t)g * P * nb;
                    if (nb == R) contract_run<R, PS, PA, true>(sg, R, R, w, val);
                    else contract_run<R, PS, PA, false>(sg, nb, nb, w, val);
                } else {
                    const int sl = gsl[nodes[0]];
                    contract_run<R, PS, PA, false>((const float2 *)L.F + (size_t)sl * P * nrhs + r0, nrhs, nb, w, val);
                }
#pragma unroll
                for (int e = 0; e < kRunK; ++e) {
                    if (nodes[e] < 0) continue;
                    const float2 f = gf[nodes[e]];
                    const cpx<float> fc = {f.x, f.y};
#pragma unroll
                    for (int rr = 0; rr < R; ++rr) {
                        const cpx<float> m = cmul(fc, val[e][rr]);
                        float2 &a = acc[nodes[e] * R + rr];
                        a.x += m.x;
                        a.y += m.y;
                    }
                }
            }
        }
        __syncwarp();  // the stage, runs and geometry are read before the next child overwrites them
    }
    for (int q = lane; q < P; q += 32)
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r < nb) {
                const float2 a = acc[q * R + r];
                st<float>(Lp.F, ((size_t)slot * P + q) * nrhs + r0 + r, cpx<float>{a.x, a.y});
            }
}

// Dynamic shared memory of the run kernel, at most: (4, 7) with 4 right-hand sides per block
// takes 53 KB per CTA, above the 48 KB default, so every instantiation is given this
// limit once at plan creation (ifgf_prepare_runs).
constexpr int kRunSmemMax = 64 * 1024;

template <int R, int PS, int PA>
inline cudaError_t set_run_smem_limit()
{
    cudaError_t e = cudaFuncSetAttribute(k_upward_runs<R, PS, PA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kRunSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_upward_runs<R, PS, PA, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRunSmemMax);
    return e;
}

// One launch of the run kernel for right-hand sides [r0, r0 + nb) of nrhs (nb <= R).
template <int R, int PS, int PA>
inline void launch_runs(const PlanDev &pd, int d, int nrhs, int r0, int nb, cudaStream_t st)
{
    constexpr int P = PS * PA * PA;
    const size_t smem = (size_t)kRunWarps * run_warp_bytes(P, R, nb);
    const int nslot = pd.lev[d - 1].nact;
    const int grid = (nslot + kRunWarps - 1) / kRunWarps;
    if (pd.lev[d].utab) k_upward_runs<R, PS, PA, true><<<grid, 32 * kRunWarps, smem, st>>>(pd, d, nrhs, r0, nb);
    else k_upward_runs<R, PS, PA, false><<<grid, 32 * kRunWarps, smem, st>>>(pd, d, nrhs, r0, nb);
}

// Launch of the upward step d -> d-1 for FP32 values: the run kernel where the geometry is
// stored (table or cache; flags bit 11: also where it is computed on the fly), with up to 4
// right-hand sides per launch (blocks of 4 for more); the staged kernel where the geometry
// is computed on the fly (up to 4 right-hand sides); k_upward otherwise, and for FP64
// values (flags bit 9 selects k_upward for FP32 too, for comparison tests).
template <typename T, int R, int PS, int PA>
inline void launch_upward(const PlanDev &pd, int d, int nrhs, int64_t np, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        constexpr int P = PS * PA * PA;
        const bool stored = pd.lev[d].utab || pd.lev[d].ucache || (pd.flags & 2048);
        if (!(pd.flags & 512)) {
            if constexpr (R <= 4) {
                if (nrhs <= R) {
                    if (stored) {
                        launch_runs<R, PS, PA>(pd, d, nrhs, 0, nrhs, st);
                        return;
                    }
                    const size_t ssmem = (size_t)kUpWarps * kUpStage * P * nrhs * sizeof(float2);
                    if (ssmem <= 48 * 1024) {
                        k_upward_staged<R, PS, PA, false>
                            <<<grid_for(np, 32 * kUpWarps), 32 * kUpWarps, ssmem, st>>>(pd, d, nrhs);
                        return;
                    }
                }
            } else if (stored) {
                // more than 4 right-hand sides: blocks of 4 (the kernels of the 4-wide
                // translation unit)
                ifgf_upward_runs_blocks(pd, d, nrhs, st);
                return;
            }
        }
    }
    if (pd.lev[d].utab) k_upward<T, R, PS, PA, true><<<grid_for(np, 128), 128, 0, st>>>(pd, d, nrhs);
    else k_upward<T, R, PS, PA, false><<<grid_for(np, 128), 128, 0, st>>>(pd, d, nrhs);
}

// Leaf analytic factors of the leaf boxes of level d; returns the threads launched.
template <typename T, int R, int PS, int PA>
inline int64_t launch_leaf(const PlanDev &pd, int d, int nrhs, const void *sig, cudaStream_t st)
{
    const int64_t nt = (int64_t)pd.lev[d].nleaf_slots * (PS * PA * PA);
    if (nt > 0) {
        NvtxRange range("leaf", d);
        k_leaf<T, R, PS, PA><<<grid_for(nt, 128), 128, 0, st>>>(pd, d, nrhs, sig);
    }
    return nt;
}

// ---------------------------------------------------------------------------------
// Targets: near field + interpolation from every cousin box of every level
// ---------------------------------------------------------------------------------
// Near field (Algorithm 1's direct evaluations at level D) with the sources staged
// through shared memory.  A block holds one work item of the plan's near tile list: up to
// kNearTargets consecutive targets of one leaf box.  The sources of the box's neighbours
// (at most 27 ranges, each contiguous in Morton order) form one list of ns entries, which
// the block copies in tiles of kNearTile into shared memory: FP64 plans copy positions
// and densities with cp.async; float plans convert each source once to its offset from
// the box centre split into FP32 high and low parts (see Rel32), so that the difference
// of two close points loses nothing.  The 128 threads form q = 128 / nt groups over the
// nt targets: group g sums, for each target, the tile entries g, g + q, ...  Small leaf
// boxes (a few points, the common case) therefore keep every lane busy, and a large box
// spreads over several blocks.  The groups' partial sums are added in group order.  The
// self term is skipped by index; conj = 1 gives the adjoint's conjugated sums.  The order
// of every sum is fixed by the plan, so results repeat bitwise.
constexpr int kNearTile = 128;
constexpr int kNearThreads = 128;
static_assert(kNearThreads >= kNearTargets, "every target of a work item needs a thread");

// The sources of the near field of leaf box b of level LD as one list (one warp, the
// first of the block): the box's near ranges [near_lo, near_hi) (its neighbours'
// points in a uniform tree; reading R13 in an adaptive one), ascending; sbeg[e] is the
// first point of range e and spre[e] the list position where it starts; spre[nr] is the
// list length.  Returns nr.
__device__ __forceinline__ int near_ranges(const LevelDev &LD, int b, int lane, int *sbeg, int *spre)
{
    const int e0 = LD.near_start[b], nr = LD.near_start[b + 1] - e0;
    int carry = 0;
    for (int c0 = 0; c0 < nr; c0 += 32) {
        const int e = c0 + lane;
        int beg = 0, cnt = 0;
        if (e < nr) {
            beg = LD.near_lo[e0 + e];
            cnt = LD.near_hi[e0 + e] - beg;
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (e < nr) {
            sbeg[e] = beg;
            spre[e + 1] = carry + inc;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) spre[0] = 0;
    return nr;
}

// The point at position g of that list.
__device__ __forceinline__ int near_source(const int *sbeg, const int *spre, int nr, int g)
{
    int lo = 0, hi = nr;  // the range e with spre[e] <= g < spre[e + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (spre[mid] <= g) lo = mid; else hi = mid;
    }
    return sbeg[lo] + (g - spre[lo]);
}

template <typename T, int R>
__global__ void __launch_bounds__(kNearThreads) k_near_staged(PlanDev pd, int nrhs, const void *in, void *out,
                                                              int conj)
{
    // positions: FP64 plans x, y, z [kNearTile] doubles; float plans the split offsets
    // (high, low) [kNearTile] float4 each
    __shared__ __align__(16) unsigned char spos[kNearTile * 32];
    __shared__ __align__(16) cpx<T> ssig[kNearTile * R];
    __shared__ __align__(16) cpx<T> spart[kNearThreads * R];
    __shared__ int sidx[kNearTile];
    __shared__ int sbeg[kMaxNearRanges], spre[kMaxNearRanges + 1];
    __shared__ int snr;
    double *sx = (double *)spos, *sy = sx + kNearTile, *sz = sy + kNearTile;
    float4 *soh = (float4 *)spos, *sol = soh + kNearTile;
    const int tid = threadIdx.x;
    const int4 item = pd.near_tile[blockIdx.x];
    const LevelDev &LD = pd.lev[item.z];
    const int b = item.x, t0 = item.y;
    const int nt = min(kNearTargets, LD.end[b] - t0);  // 1 .. kNearTargets
    if (tid < 32) {
        const int nr = near_ranges(LD, b, tid, sbeg, spre);
        if (tid == 0) snr = nr;
    }
    __syncthreads();
    const int nr = snr;
    const int ns = spre[nr];
    const int q = kNearThreads / nt;
    const int tt = tid % nt, grp = tid / nt;
    const bool tv = grp < q;
    const int i = t0 + tt;
    const double *cb = LD.center + 3 * (size_t)b;
    const float kf = (float)pd.kappa;
    double x = 0, y = 0, z = 0;
    if (tv) {
        x = pd.xs[i];
        y = pd.ys[i];
        z = pd.zs[i];
    }
    Rel32 pt;
    if constexpr (sizeof(T) == 4) pt = rel32(x, y, z, cb);
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        const int rv = min(R, nrhs - r0);
        cpx<T> acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = {T(0), T(0)};
        for (int g0 = 0; g0 < ns; g0 += kNearTile) {
            const int cnt = min(kNearTile, ns - g0);
            for (int s = tid; s < cnt; s += kNearThreads) {
                const int j = near_source(sbeg, spre, nr, g0 + s);
                sidx[s] = j;
                if constexpr (sizeof(T) == 8) {
                    cp_async8(sx + s, pd.xs + j);
                    cp_async8(sy + s, pd.ys + j);
                    cp_async8(sz + s, pd.zs + j);
                } else {
                    const Rel32 ps = rel32(pd.xs[j], pd.ys[j], pd.zs[j], cb);
                    soh[s] = make_float4(ps.hx, ps.hy, ps.hz, 0.f);
                    sol[s] = make_float4(ps.lx, ps.ly, ps.lz, 0.f);
                }
                for (int r = 0; r < rv; ++r) {
                    const cpx<T> *src = (const cpx<T> *)in + (size_t)j * nrhs + r0 + r;
                    if constexpr (sizeof(T) == 8) cp_async16(ssig + s * R + r, src);
                    else cp_async8(ssig + s * R + r, src);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            if (tv) {
                for (int s = grp; s < cnt; s += q) {
                    if (sidx[s] == i) continue;
                    cpx<T> G;
                    if constexpr (sizeof(T) == 8) {
                        const double dx = x - sx[s], dy = y - sy[s], dz = z - sz[s];
                        G = green_r2_64(pd.kappa, dx * dx + dy * dy + dz * dz);
                    } else {
                        G = green_near32(pt, soh[s], sol[s], kf);
                    }
                    if (conj) G = cconj(G);
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (R == 1 || r < rv) {
                            const cpx<T> m = cmul(G, ssig[s * R + r]);
                            acc[r].x += m.x;
                            acc[r].y += m.y;
                        }
                }
            }
            __syncthreads();  // the tile is read before the next copy overwrites it
        }
#pragma unroll
        for (int r = 0; r < R; ++r) spart[tid * R + r] = acc[r];
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (R == 1 || r < rv) {
                    cpx<T> v = spart[tt * R + r];
                    for (int g = 1; g < q; ++g) {
                        const cpx<T> o = spart[(g * nt + tt) * R + r];
                        v.x += o.x;
                        v.y += o.y;
                    }
                    st<T>(out, (size_t)i * nrhs + r0 + r, v);
                }
        }
        __syncthreads();  // the partial sums are read before the next chunk writes them
    }
}

template <typename T, int R, int PS, int PA>
__global__ void __launch_bounds__(128) k_eval(PlanDev pd, int nrhs, const void *sig, void *us, int mode, int d_hi,
                                              int d_lo, int accumulate)
{
    constexpr int P = PS * PA * PA;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    const double x = pd.xs[i], y = pd.ys[i], z = pd.zs[i];
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        cpx<T> acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = {T(0), T(0)};
        if (mode & 2) {
            for (int d = d_hi; d >= d_lo; --d) {
                const LevelDev &L = pd.lev[d];
                int b = L.pt_box[i];
                if (b < 0) continue;  // below the point's leaf (adaptive tree)
                for (int e = L.cous_start[b]; e < L.cous_start[b + 1]; ++e) {
                    int k = L.cous[e];
                    const double *ck = L.center + 3 * (size_t)k;
                    T w[PS + 2 * PA];
                    int sl;
                    cpx<T> G;
                    bool cached = false;
                    if constexpr (PS + 2 * PA <= 13) {
                        if (L.tcache) {
                            const size_t o = (size_t)L.toff[i] + (e - L.cous_start[b]);
                            if constexpr (sizeof(T) == 8) {
                                const TEntry64 &en = ((const TEntry64 *)L.tcache)[o];
#pragma unroll
                                for (int m = 0; m < PS + 2 * PA; ++m) w[m] = en.w[m];
                                G = {en.gr, en.gi};
                                sl = en.slot;
                            } else {
                                const TEntry32 en = ((const TEntry32 *)L.tcache)[o];
                                lagrange(PS, pd.tsf, pd.itsf, en.t[0], w);
                                lagrange(PA, pd.taf, pd.itaf, en.t[1], w + PS);
                                lagrange(PA, pd.taf, pd.itaf, en.t[2], w + PS + PA);
                                G = {en.gr, en.gi};
                                sl = en.slot;
                            }
                            cached = true;
                        }
                    }
                    if (!cached) {
                        double vx = __dsub_rn(x, ck[0]), vy = __dsub_rn(y, ck[1]), vz = __dsub_rn(z, ck[2]);
                        ConeGeom g = geom_weights<T, PS, PA>(pd, L, vx, vy, vz, w);
                        sl = cone_slot(L, k, g.cone);
                        if (sl < 0) { atomicAdd(pd.err, 1); continue; }
                        G = green_r<T>(pd.kappa, g.r);
                    }
                    cpx<T> val[R];
                    contract<T, R, PS, PA>(L.F, (size_t)sl * P, nrhs, r0, w, w + PS, w + PS + PA, val);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        cpx<T> m = cmul(G, val[r]);
                        acc[r].x += m.x;
                        acc[r].y += m.y;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r0 + r < nrhs) {
                size_t o = (size_t)i * nrhs + r0 + r;
                if (accumulate) {
                    cpx<T> prev = ld<T>(us, o);
                    acc[r].x += prev.x;
                    acc[r].y += prev.y;
                }
                st<T>(us, o, acc[r]);
            }
    }
}

// ---------------------------------------------------------------------------------
// Adjoint: cone slots of level d gather from their readers (one warp per slot).
// ---------------------------------------------------------------------------------
constexpr int kAdjWarps = 4;

// AdjLists: the transpose lists a launch reads (CSR over level-d slots, start[s - base]),
// the slots [s0, s1) it covers, the passes it runs (bit 0 cousin targets, bit 1 parent
// interpolation points) and whether it adds to the adjoint values instead of storing.
struct AdjLists {
    const int *tstart, *tlist;
    int tbase;
    const int *ustart, *ulist;
    int ubase;
    int s0, s1, passes, accumulate;
    const int *tcache_idx;  // per entry of tlist, its index in the level's target cache (or null)
};

// Weights and conjugated factor of one reader of a level-d cone slot of box k (centre ck):
// pass 0 a cousin target (item = point index, e its list position), pass 1 a parent
// interpolation point (item = parent slot * P + node).  Cached geometry is used where
// the plan holds it: the target cache through the list's cache index, the upward table,
// or the upward cache of an untabled level (indexed by parent slot, node and the child's
// position among the parent box's children); otherwise it is computed here.
template <typename T, int PS, int PA>
__device__ __forceinline__ void adj_reader(const PlanDev &pd, const LevelDev &L, int d, int k, const double *ck,
                                           int pass, unsigned item, int e, const AdjLists &al, T *w, cpx<T> &f)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    if (pass == 0) {
        if constexpr (NW <= 13) {
            if (al.tcache_idx && L.tcache) {
                const size_t o = (size_t)al.tcache_idx[e];
                if constexpr (sizeof(T) == 8) {
                    const TEntry64 &en = ((const TEntry64 *)L.tcache)[o];
#pragma unroll
                    for (int m = 0; m < NW; ++m) w[m] = en.w[m];
                    f = cconj(cpx<T>{en.gr, en.gi});
                } else {
                    const TEntry32 en = ((const TEntry32 *)L.tcache)[o];
                    lagrange(PS, pd.tsf, pd.itsf, en.t[0], w);
                    lagrange(PA, pd.taf, pd.itaf, en.t[1], w + PS);
                    lagrange(PA, pd.taf, pd.itaf, en.t[2], w + PS + PA);
                    f = cconj(cpx<T>{en.gr, en.gi});
                }
                return;
            }
        }
        const double vx = __dsub_rn(pd.xs[item], ck[0]), vy = __dsub_rn(pd.ys[item], ck[1]),
                     vz = __dsub_rn(pd.zs[item], ck[2]);
        ConeGeom g = geom_weights<T, PS, PA>(pd, L, vx, vy, vz, w);
        f = cconj(green_r<T>(pd.kappa, g.r));
        return;
    }
    const LevelDev &Lp = pd.lev[d - 1];
    const int psl = item / P, pnode = item % P;
    const int oct = (int)(L.key[k] & 7u);
    const int pcone = Lp.act_cone[psl];
    const int row = L.utab ? table_row(L.ubits, L.urank, pcone) : -1;
    using Entry = typename UpEntryOf<T, NW>::type;
    if (row >= 0) {
        cpx<T> ff;
        up_entry<T, PS, PA>(pd, ((const Entry *)L.utab)[((size_t)row * 8 + oct) * P + pnode], w, ff);
        f = cconj(ff);
    } else if (L.ucache) {
        const int j = Lp.act_box[psl];
        const int k0 = Lp.child_start[j], nch = Lp.child_start[j + 1] - k0;
        cpx<T> ff;
        up_entry<T, PS, PA>(pd, ((const Entry *)L.ucache)[(size_t)L.uoff[psl] + (size_t)pnode * nch + (k - k0)], w, ff);
        f = cconj(ff);
    } else {
        cpx<T> ff;
        up_geometry<T, PS, PA>(pd, L, Lp, pcone, pnode, oct, w, ff);
        f = cconj(ff);
    }
}

template <typename T, int R, int PS, int PA>
__global__ void __launch_bounds__(32 * kAdjWarps) k_adj_level(PlanDev pd, int d, int nrhs, const void *vs, int mode,
                                                               AdjLists al)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    constexpr int NPL = (P + 31) / 32;  // nodes per lane
    __shared__ T sw[kAdjWarps][32][NW];
    __shared__ cpx<T> sc[kAdjWarps][32][R];
    const LevelDev &L = pd.lev[d];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kAdjWarps + warp;
    const int nwarps = gridDim.x * kAdjWarps;
    for (int slot = al.s0 + gw; slot < al.s1; slot += nwarps) {
        const int k = L.act_box[slot];
        const double *ck = L.center + 3 * (size_t)k;
        for (int r0 = 0; r0 < nrhs; r0 += R) {
            cpx<T> acc[NPL][R];
#pragma unroll
            for (int h = 0; h < NPL; ++h)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[h][r] = {T(0), T(0)};
            for (int pass = 0; pass < 2; ++pass) {
                if (!((al.passes >> pass) & 1)) continue;
                const int *lst;
                int e_begin, e_end;
                if (pass == 0) {
                    lst = al.tlist;
                    e_begin = al.tstart[slot - al.tbase];
                    e_end = al.tstart[slot - al.tbase + 1];
                } else {
                    if (d <= 3 || !(mode & 2)) break;
                    lst = al.ulist;
                    e_begin = al.ustart[slot - al.ubase];
                    e_end = al.ustart[slot - al.ubase + 1];
                }
                for (int e0 = e_begin; e0 < e_end; e0 += 32) {
                    int e = e0 + lane;
                    if (e < e_end) {
                        // a point index, or parent slot * P + node (can exceed 2^31 - 1)
                        const unsigned item = (unsigned)lst[e];
                        const int psl = (int)(item / P), pnode = (int)(item % P);  // pass 1
                        T w[NW];
                        cpx<T> f;
                        adj_reader<T, PS, PA>(pd, L, d, k, ck, pass, item, e, al, w, f);
#pragma unroll
                        for (int m = 0; m < NW; ++m) sw[warp][lane][m] = w[m];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            cpx<T> src = {T(0), T(0)};
                            if (R == 1 || r0 + r < nrhs) {
                                if (pass == 0) src = ld<T>(vs, (size_t)item * nrhs + r0 + r);
                                else src = ld<T>(pd.lev[d - 1].Fadj, ((size_t)psl * P + pnode) * nrhs + r0 + r);
                            }
                            sc[warp][lane][r] = cmul(f, src);
                        }
                    }
                    __syncwarp();
                    int cnt = min(32, e_end - e0);
                    for (int m = 0; m < cnt; ++m) {
#pragma unroll
                        for (int h = 0; h < NPL; ++h) {
                            int p = lane + 32 * h;
                            if (p < P) {
                                int a = p / (PA * PA), b = (p / PA) % PA, c = p % PA;
                                T w = sw[warp][m][a] * sw[warp][m][PS + b] * sw[warp][m][PS + PA + c];
#pragma unroll
                                for (int r = 0; r < R; ++r) {
                                    acc[h][r].x += w * sc[warp][m][r].x;
                                    acc[h][r].y += w * sc[warp][m][r].y;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
#pragma unroll
            for (int h = 0; h < NPL; ++h) {
                int p = lane + 32 * h;
                if (p < P)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (R == 1 || r0 + r < nrhs) {
                            const size_t o = ((size_t)slot * P + p) * nrhs + r0 + r;
                            cpx<T> v = acc[h][r];
                            if (al.accumulate) {
                                const cpx<T> old = ld<T>(L.Fadj, o);
                                v.x += old.x;
                                v.y += old.y;
                            }
                            st<T>(L.Fadj, o, v);
                        }
            }
        }
    }
}

// One right-hand side: the same sums, sum-factorised.  The contribution of a reader
// with weights w (Lagrange weights of its local coordinates), factor f and value v to
// node (a, b, c) of the slot is w_c t_ab with t_ab = w_a w_b conj(f) v.  Each lane forms
// the PS PA values t_ab of the reader it loads; the warp then adds w_c t_ab at the nodes
// of two readers at a time (2P node slots over the lanes, 150 of 160 for P = 75): two
// FMAs per node and reader instead of a weight product and two FMAs on 75 of 96 slots.
// A node's sum over the even readers of each batch of 32 and its sum over the odd ones
// are added at the end, so the order of every sum is fixed.
constexpr int kAdj1Warps = 2;

template <typename T, int PS, int PA>
__global__ void __launch_bounds__(32 * kAdj1Warps) k_adj_level1(PlanDev pd, int d, const void *vs, int mode,
                                                                 AdjLists al)
{
    constexpr int P = PS * PA * PA;
    constexpr int NW = PS + 2 * PA;
    constexpr int NAB = PS * PA;
    constexpr int NS = (2 * P + 31) / 32;  // node slots per lane (two readers)
    constexpr int NPL = (P + 31) / 32;     // nodes per lane
    static_assert(2 * P <= 32 * NAB, "the partial sums reuse the t_ab buffer");
    __shared__ cpx<T> stab[kAdj1Warps][32][NAB];
    __shared__ T swc[kAdj1Warps][32][PA];
    const LevelDev &L = pd.lev[d];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kAdj1Warps + warp;
    const int nwarps = gridDim.x * kAdj1Warps;
    for (int slot = al.s0 + gw; slot < al.s1; slot += nwarps) {
        const int k = L.act_box[slot];
        const double *ck = L.center + 3 * (size_t)k;
        cpx<T> acc[NS];
#pragma unroll
        for (int h = 0; h < NS; ++h) acc[h] = {T(0), T(0)};
        for (int pass = 0; pass < 2; ++pass) {
            if (!((al.passes >> pass) & 1)) continue;
            const int *lst;
            int e_begin, e_end;
            if (pass == 0) {
                lst = al.tlist;
                e_begin = al.tstart[slot - al.tbase];
                e_end = al.tstart[slot - al.tbase + 1];
            } else {
                if (d <= 3 || !(mode & 2)) break;
                lst = al.ulist;
                e_begin = al.ustart[slot - al.ubase];
                e_end = al.ustart[slot - al.ubase + 1];
            }
            for (int e0 = e_begin; e0 < e_end; e0 += 32) {
                const int e = e0 + lane;
                if (e < e_end) {
                    // a point index, or parent slot * P + node (can exceed 2^31 - 1)
                    const unsigned item = (unsigned)lst[e];
                    T w[NW];
                    cpx<T> f;
                    adj_reader<T, PS, PA>(pd, L, d, k, ck, pass, item, e, al, w, f);
                    const cpx<T> v = pass == 0 ? ld<T>(vs, (size_t)item) : ld<T>(pd.lev[d - 1].Fadj, (size_t)item);
                    const cpx<T> z = cmul(f, v);
#pragma unroll
                    for (int a = 0; a < PS; ++a)
#pragma unroll
                        for (int b = 0; b < PA; ++b) {
                            const T wab = w[a] * w[PS + b];
                            stab[warp][lane][a * PA + b] = {wab * z.x, wab * z.y};
                        }
#pragma unroll
                    for (int c = 0; c < PA; ++c) swc[warp][lane][c] = w[PS + PA + c];
                }
                __syncwarp();
                const int cnt = min(32, e_end - e0);
                for (int m = 0; m < cnt; m += 2) {
#pragma unroll
                    for (int h = 0; h < NS; ++h) {
                        const int s = lane + 32 * h;
                        const int eo = s >= P ? 1 : 0;
                        const int pn = s - eo * P;
                        if (s < 2 * P && m + eo < cnt) {
                            const cpx<T> t = stab[warp][m + eo][pn / PA];
                            const T wc = swc[warp][m + eo][pn % PA];
                            acc[h].x += wc * t.x;
                            acc[h].y += wc * t.y;
                        }
                    }
                }
                __syncwarp();
            }
        }
        // node p: the even readers' sum (slot p) plus the odd readers' sum (slot p + P)
        cpx<T> *part = &stab[warp][0][0];
#pragma unroll
        for (int h = 0; h < NS; ++h) {
            const int s = lane + 32 * h;
            if (s < 2 * P) part[s] = acc[h];
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < NPL; ++h) {
            const int pn = lane + 32 * h;
            if (pn < P) {
                cpx<T> v = {part[pn].x + part[pn + P].x, part[pn].y + part[pn + P].y};
                const size_t o = (size_t)slot * P + pn;
                if (al.accumulate) {
                    const cpx<T> old = ld<T>(L.Fadj, o);
                    v.x += old.x;
                    v.y += old.y;
                }
                st<T>(L.Fadj, o, v);
            }
        }
        __syncwarp();  // the partial sums are read before the next slot's readers overwrite them
    }
}

// Launch of the adjoint level kernel for slots [al.s0, al.s1): the sum-factorised
// single-RHS kernel for one right-hand side, else the R-blocked one.
template <typename T, int R, int PS, int PA>
inline void launch_adj_level(const PlanDev &pd, int d, int nrhs, const void *vs, int mode, const AdjLists &al,
                             cudaStream_t st)
{
    const int64_t ns = al.s1 - al.s0;
    if (ns <= 0) return;
    if constexpr (R == 1) {
        const int blocks = (int)std::min<int64_t>((ns + kAdj1Warps - 1) / kAdj1Warps, 152 * 128);
        k_adj_level1<T, PS, PA><<<blocks, 32 * kAdj1Warps, 0, st>>>(pd, d, vs, mode, al);
    } else {
        const int blocks = (int)std::min<int64_t>((ns + kAdjWarps - 1) / kAdjWarps, 152 * 64);
        k_adj_level<T, R, PS, PA><<<blocks, 32 * kAdjWarps, 0, st>>>(pd, d, nrhs, vs, mode, al);
    }
}

// Adjoint per source: conj(g(q, x')) times the adjoint values of its leaf box's cones,
// stored or added to the conjugated near field (accumulate).  only_level >= 3 restricts
// the launch to the sources whose leaf box lies on that level (two-buffer adjoints of
// adaptive trees run it level by level, while the level's values are resident).
template <typename T, int R, int PS, int PA>
__global__ void __launch_bounds__(128) k_adj_eval(PlanDev pd, int nrhs, const void *vs, void *ws, int mode,
                                                  int accumulate, int only_level)
{
    constexpr int P = PS * PA * PA;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= pd.n) return;
    const int lv = pd.ptlev[j];  // the level of the point's leaf box
    if (only_level >= 3 && lv != only_level) return;
    const LevelDev &LD = pd.lev[lv];
    const int b = LD.pt_box[j];
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        cpx<T> acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = {T(0), T(0)};
        if (mode & 2) {
            const double *c = LD.center + 3 * (size_t)b;
            for (int slot = LD.act_start[b]; slot < LD.act_start[b + 1]; ++slot) {
                int cone = LD.act_cone[slot];
                for (int node = 0; node < P; ++node) {
                    double q[3], dir[3];
                    double R0 = node_pos(LD, PS, PA, cone, node, c[0], c[1], c[2], q, dir);
                    cpx<T> g = cconj(leaf_factor<T>(pd, R0, q, dir, j));
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (R == 1 || r0 + r < nrhs) {
                            cpx<T> m = cmul(g, ld<T>(LD.Fadj, ((size_t)slot * P + node) * nrhs + r0 + r));
                            acc[r].x += m.x;
                            acc[r].y += m.y;
                        }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (R == 1 || r0 + r < nrhs) {
                cpx<T> v = acc[r];
                if (accumulate) {
                    const cpx<T> old = ld<T>(ws, (size_t)j * nrhs + r0 + r);
                    v.x += old.x;
                    v.y += old.y;
                }
                st<T>(ws, (size_t)j * nrhs + r0 + r, v);
            }
    }
}

// ---------------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------------

template <typename T, int R, int PS, int PA>
cudaError_t launch_forward(const PlanDev &pd, int nrhs, const void *sig, void *us, int mode, cudaStream_t st,
                           StageTimer &tm)
{
    constexpr int P = PS * PA * PA;
    if (!pd.pingpong) {
        if (mode & 2) {
            int64_t nt = launch_leaf<T, R, PS, PA>(pd, pd.D, nrhs, sig, st);
            tm.mark(STAGE_LEAF, nt > 0, st);
            int nl = 0;
            for (int d = pd.D; d >= 4; --d) {
                int64_t np = (int64_t)pd.lev[d - 1].nact * P;
                if (np == 0) continue;
                NvtxRange range("upward", d);
                launch_upward<T, R, PS, PA>(pd, d, nrhs, np, st);
                // leaves of level d-1 (adaptive tree): their slots take the analytic factors
                // of their own points, after the upward step has written the level
                nl += 1 + (launch_leaf<T, R, PS, PA>(pd, d - 1, nrhs, sig, st) > 0);
            }
            tm.mark(STAGE_UPWARD, nl, st);
        }
        {
            NvtxRange range("near field and targets");
            if (mode & 1) k_near_staged<T, R><<<pd.n_near_tile, kNearThreads, 0, st>>>(pd, nrhs, sig, us, 0);
            if (mode & 2)
                k_eval<T, R, PS, PA><<<grid_for(pd.n, 128), 128, 0, st>>>(pd, nrhs, sig, us, 2, pd.D, 3, mode & 1);
        }
        tm.mark(STAGE_EVAL, 1 + ((mode & 3) == 3), st);
        return cudaGetLastError();
    }
    // two alternating level buffers: each level's targets are evaluated before the
    // upward step overwrites the buffer of level d-1's parent
    if (mode & 1) {
        NvtxRange range("near field");
        k_near_staged<T, R><<<pd.n_near_tile, kNearThreads, 0, st>>>(pd, nrhs, sig, us, 0);
    } else {
        cudaMemsetAsync(us, 0, (size_t)pd.n * nrhs * sizeof(cpx<T>), st);
    }
    tm.mark(STAGE_EVAL, 1, st);
    if (mode & 2) {
        int64_t nt = launch_leaf<T, R, PS, PA>(pd, pd.D, nrhs, sig, st);
        tm.mark(STAGE_LEAF, nt > 0, st);
        for (int d = pd.D; d >= 3; --d) {
            NvtxRange range("targets and upward", d);
            k_eval<T, R, PS, PA><<<grid_for(pd.n, 128), 128, 0, st>>>(pd, nrhs, sig, us, 2, d, d, 1);
            tm.mark(STAGE_EVAL, 1, st);
            if (d > 3) {
                int64_t np = (int64_t)pd.lev[d - 1].nact * P;
                if (np > 0) launch_upward<T, R, PS, PA>(pd, d, nrhs, np, st);
                const int64_t nl = launch_leaf<T, R, PS, PA>(pd, d - 1, nrhs, sig, st);
                tm.mark(STAGE_UPWARD, (np > 0) + (nl > 0), st);
            }
        }
    }
    return cudaGetLastError();
}

template <typename T, int R, int PS, int PA>
cudaError_t launch_adjoint(const PlanDev &pd, int nrhs, const void *vs, void *ws, int mode, cudaStream_t st,
                           StageTimer &tm)
{
    if (mode & 2) {
        int nl = 0;
        for (int d = 3; d <= pd.D; ++d) {
            int nact = pd.lev[d].nact;
            if (nact == 0) continue;
            NvtxRange range("adjoint level", d);
            const LevelDev &L = pd.lev[d];
            const AdjLists al = {L.tl_start, L.tl, 0, L.ul_start, L.ul, 0, 0, nact, 3, 0, L.tl_cache};
            launch_adj_level<T, R, PS, PA>(pd, d, nrhs, vs, mode, al, st);
            ++nl;
        }
        tm.mark(STAGE_ADJ_LEVEL, nl, st);
    }
    if (mode & 1) k_near_staged<T, R><<<pd.n_near_tile, kNearThreads, 0, st>>>(pd, nrhs, vs, ws, 1);
    if (mode & 2) k_adj_eval<T, R, PS, PA><<<grid_for(pd.n, 128), 128, 0, st>>>(pd, nrhs, vs, ws, 2, mode & 1, -1);
    tm.mark(STAGE_ADJ_EVAL, 1 + ((mode & 3) == 3), st);
    return cudaGetLastError();
}

// Adjoint of a two-buffer plan with transpose lists built just in time: per level d =
// 3..D, the cousin-target lists of the level (one launch over all slots, storing), then
// the upward lists in ranges of parent boxes of at most max_entries evaluations (one
// launch per range over the child slots of that range, adding).  The child slots of a
// range of parent boxes are contiguous, and every child slot takes all of its upward
// entries from one range, so each slot's sum has a fixed order.
template <typename T, int R, int PS, int PA>
ifgf_status launch_adjoint_jit(ifgf_plan *p, int nrhs, const void *vs, void *ws, int mode, cudaStream_t st,
                               int64_t max_entries)
{
    const PlanDev &pd = p->dev;
    StageTimer &tm = p->timer;
    JitLists tl, ul;
    JitWork work;  // reused by every list build of this call
    ifgf_status s = IFGF_OK;
    // the conjugated near field first (it stores), then per level the adjoint values and,
    // in adaptive trees, the sources whose leaf box lies on that level (they add)
    if (mode & 1) {
        k_near_staged<T, R><<<pd.n_near_tile, kNearThreads, 0, st>>>(pd, nrhs, vs, ws, 1);
        tm.mark(STAGE_ADJ_EVAL, 1, st);
    }
    if (mode & 2) {
        for (int d = 3; d <= pd.D && s == IFGF_OK; ++d) {
            const int nact = pd.lev[d].nact;
            if (nact == 0) {
                if (pd.adaptive || d == pd.D) {
                    k_adj_eval<T, R, PS, PA><<<grid_for(pd.n, 128), 128, 0, st>>>(pd, nrhs, vs, ws, 2, mode & 1, d);
                    tm.mark(STAGE_ADJ_EVAL, 1, st);
                }
                continue;
            }
            NvtxRange range("adjoint level (lists built here)", d);
            s = ifgf_jit_targets(p, d, &tl, &work, st);
            if (s != IFGF_OK) break;
            tm.mark(STAGE_ADJ_LISTS, 0, st);
            {
                const AdjLists al = {tl.start, tl.list, 0, nullptr, nullptr, 0, 0, nact, 1, 0, nullptr};
                launch_adj_level<T, R, PS, PA>(pd, d, nrhs, vs, mode, al, st);
                if (cudaGetLastError() != cudaSuccess) { p->last_error = "adjoint level launch"; s = IFGF_ECUDA; break; }
                tm.mark(STAGE_ADJ_LEVEL, 1, st);
            }
            if (d > 3) {
                std::vector<int> bounds;
                s = ifgf_jit_chunks(p, d, max_entries, &bounds);
                for (size_t c = 0; c + 1 < bounds.size() && s == IFGF_OK; ++c) {
                    s = ifgf_jit_upward(p, d, bounds[c], bounds[c + 1], &ul, &work, st);
                    tm.mark(STAGE_ADJ_LISTS, 0, st);
                    if (s != IFGF_OK || ul.s1 == ul.s0) continue;
                    const AdjLists al = {nullptr, nullptr, 0, ul.start, ul.list, ul.s0, ul.s0, ul.s1, 2, 1, nullptr};
                    launch_adj_level<T, R, PS, PA>(pd, d, nrhs, vs, mode, al, st);
                    if (cudaGetLastError() != cudaSuccess) { p->last_error = "adjoint level launch"; s = IFGF_ECUDA; }
                    tm.mark(STAGE_ADJ_LEVEL, 1, st);
                    // the lists are freed (and rebuilt) only after the launch has read them
                    if (cudaStreamSynchronize(st) != cudaSuccess) { p->last_error = "adjoint level"; s = IFGF_ECUDA; }
                }
            }
            // the sources of this level's leaves, before level d + 2 reuses the buffer
            if (pd.adaptive || d == pd.D) {
                k_adj_eval<T, R, PS, PA><<<grid_for(pd.n, 128), 128, 0, st>>>(pd, nrhs, vs, ws, 2, mode & 1, d);
                tm.mark(STAGE_ADJ_EVAL, 1, st);
            }
            if (cudaStreamSynchronize(st) != cudaSuccess) { p->last_error = "adjoint level"; s = IFGF_ECUDA; }
        }
    }
    ifgf_jit_release(&tl);
    ifgf_jit_release(&ul);
    work.release();
    if (s != IFGF_OK) return s;
    if (cudaGetLastError() != cudaSuccess) { p->last_error = "adjoint launch"; return IFGF_ECUDA; }
    return IFGF_OK;
}

// permute, just-in-time adjoint, un-permute (FP64 or FP32 plans, one right-hand-side chunk)
template <typename T>
ifgf_status run_adjoint_jit(ifgf_plan *p, int nrhs, const void *in_user, void *out_user, int mode, cudaStream_t st)
{
    const PlanDev &pd = p->dev;
    const int64_t tot = (int64_t)pd.n * nrhs;
    const int64_t max_entries = (p->flags & 64) ? 4096 : ((int64_t)1 << 28);
    p->timer.mark(-1, 0, st);
    k_permute_in<T><<<grid_for(tot, 256), 256, 0, st>>>(in_user, p->sig_sorted, pd.perm, pd.n, nrhs);
    p->timer.mark(STAGE_PERMUTE_IN, 1, st);
    constexpr int RB = sizeof(T) == 8 ? 4 : 8;
    ifgf_status s;
    if (pd.Ps == 3 && pd.Pang == 5) {
        if (nrhs == 1)
            s = launch_adjoint_jit<T, 1, 3, 5>(p, nrhs, p->sig_sorted, p->u_sorted, mode, st, max_entries);
        else if (sizeof(T) == 4 && nrhs <= 4)
            // FP32 with 2..4 right-hand sides: blocked for 4, as the forward (more warps per SM)
            s = launch_adjoint_jit<T, 4, 3, 5>(p, nrhs, p->sig_sorted, p->u_sorted, mode, st, max_entries);
        else
            s = launch_adjoint_jit<T, RB, 3, 5>(p, nrhs, p->sig_sorted, p->u_sorted, mode, st, max_entries);
    } else if (pd.Ps == 4 && pd.Pang == 7)
        s = nrhs == 1 ? launch_adjoint_jit<T, 1, 4, 7>(p, nrhs, p->sig_sorted, p->u_sorted, mode, st, max_entries)
                      : launch_adjoint_jit<T, RB, 4, 7>(p, nrhs, p->sig_sorted, p->u_sorted, mode, st, max_entries);
    else
        return IFGF_EINVAL;
    if (s != IFGF_OK) return s;
    k_permute_out<T><<<grid_for(tot, 256), 256, 0, st>>>(p->u_sorted, out_user, pd.perm, pd.n, nrhs);
    p->timer.mark(STAGE_PERMUTE_OUT, 1, st);
    if (cudaGetLastError() != cudaSuccess) { p->last_error = "permute launch"; return IFGF_ECUDA; }
    return IFGF_OK;
}

template <typename T, int PS, int PA>
cudaError_t launch_orders(const PlanDev &pd, int nrhs, const void *in, void *out, int mode, int adjoint,
                          cudaStream_t st, StageTimer &tm)
{
    if (nrhs == 1) {
        return adjoint ? launch_adjoint<T, 1, PS, PA>(pd, nrhs, in, out, mode, st, tm)
                       : launch_forward<T, 1, PS, PA>(pd, nrhs, in, out, mode, st, tm);
    }
    // FP32 with 2..4 right-hand sides: kernels blocked for 4 (half the accumulator
    // registers of the 8-wide blocking, so more warps per SM; instantiated in
    // ifgf_apply_f32_r4.cu)
    if constexpr (sizeof(T) == 4)
        if (nrhs <= 4) return ifgf_launch_f32_r4(pd, nrhs, in, out, mode, adjoint, st, tm);
    constexpr int RB = sizeof(T) == 8 ? 4 : 8;
    return adjoint ? launch_adjoint<T, RB, PS, PA>(pd, nrhs, in, out, mode, st, tm)
                   : launch_forward<T, RB, PS, PA>(pd, nrhs, in, out, mode, st, tm);
}

// Evaluation caches.  which = 0: cousin targets of level d; which = 1: upward step
// d -> d-1 per (parent slot, node, child).
template <typename T, int PS, int PA>
__global__ void __launch_bounds__(128) k_build_tcache(PlanDev pd, int d)
{
    constexpr int NW = PS + 2 * PA;
    const LevelDev &L = pd.lev[d];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.n) return;
    const int b = L.pt_box[i];
    if (b < 0) return;  // a point of a coarser leaf: no cousin evaluations at this level
    const double x = pd.xs[i], y = pd.ys[i], z = pd.zs[i];
    int o = L.toff[i];
    for (int e = L.cous_start[b]; e < L.cous_start[b + 1]; ++e, ++o) {
        const int k = L.cous[e];
        const double *ck = L.center + 3 * (size_t)k;
        double vx = __dsub_rn(x, ck[0]), vy = __dsub_rn(y, ck[1]), vz = __dsub_rn(z, ck[2]);
        ConeGeom g = sizeof(T) == 8 ? cone_of_fast(L, vx, vy, vz) : cone_of_mixed(L, vx, vy, vz);
        int sl = cone_slot(L, k, g.cone);
        if (sl < 0) { atomicAdd(pd.err, 1); sl = 0; }
        if constexpr (sizeof(T) == 8) {
            TEntry64 en;
            double loc[3];
            local_coords(L, g, vx, vy, vz, loc);
            weights3<double, PS, PA>(pd, loc, en.w, en.w + PS, en.w + PS + PA);
            for (int m = NW; m < 13; ++m) en.w[m] = 0.0;
            cpx<double> G = green_r<double>(pd.kappa, g.r);
            en.gr = G.x;
            en.gi = G.y;
            en.slot = sl;
            en.pad = 0;
            ((TEntry64 *)L.tcache)[o] = en;
        } else {
            TEntry32 en;
            local_coords_f32(L, g, vx, vy, vz, en.t);
            cpx<float> G = green_r<float>(pd.kappa, g.r);
            en.gr = G.x;
            en.gi = G.y;
            en.slot = sl;
            ((TEntry32 *)L.tcache)[o] = en;
        }
    }
}

template <typename T, int PS, int PA>
__global__ void __launch_bounds__(128) k_build_ucache(PlanDev pd, int d)
{
    constexpr int P = PS * PA * PA;
    const LevelDev &L = pd.lev[d];
    const LevelDev &Lp = pd.lev[d - 1];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Lp.nact * P) return;
    const int slot = (int)(t / P), node = (int)(t % P);
    const int j = Lp.act_box[slot];
    const int k0 = Lp.child_start[j], k1 = Lp.child_start[j + 1];
    const int pcone = Lp.act_cone[slot];
    for (int k = k0; k < k1; ++k) {
        const int oct = (int)(L.key[k] & 7u);
        ((typename UpEntryOf<T, PS + 2 * PA>::type *)L.ucache)[(size_t)L.uoff[slot] + (size_t)node * (k1 - k0) + (k - k0)] =
            make_up_entry<T, PS, PA>(pd, L, Lp, pcone, node, oct);
    }
}

template <typename T>
cudaError_t build_evalcache(const PlanDev &pd, int d, int which, cudaStream_t st)
{
    int64_t n = which == 0 ? pd.n : (int64_t)pd.lev[d - 1].nact * pd.P;
    if (n == 0) return cudaSuccess;
    if (pd.Ps == 3 && pd.Pang == 5) {
        if (which == 0) k_build_tcache<T, 3, 5><<<grid_for(n, 128), 128, 0, st>>>(pd, d);
        else k_build_ucache<T, 3, 5><<<grid_for(n, 128), 128, 0, st>>>(pd, d);
    } else if (pd.Ps == 4 && pd.Pang == 7) {
        if (which == 0) return cudaSuccess;  // 18 weights do not fit the 13-weight target entry
        k_build_ucache<T, 4, 7><<<grid_for(n, 128), 128, 0, st>>>(pd, d);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t build_uptable(const PlanDev &pd, int d, void *tab, cudaStream_t st)
{
    int64_t n = (int64_t)pd.lev[d].urows * 8 * pd.P;
    if (n == 0) return cudaSuccess;
    if (pd.Ps == 3 && pd.Pang == 5)
        k_build_uptable<T, 3, 5><<<grid_for(n, 128), 128, 0, st>>>(pd, d, (typename UpEntryOf<T, 13>::type *)tab);
    else if (pd.Ps == 4 && pd.Pang == 7)
        k_build_uptable<T, 4, 7><<<grid_for(n, 128), 128, 0, st>>>(pd, d, (typename UpEntryOf<T, 18>::type *)tab);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// entry used by the per-type translation units
template <typename T>
cudaError_t run_typed(const PlanDev &pd, int nrhs, const void *in_user, void *out_user, void *in_sorted,
                      void *out_sorted, int mode, int adjoint, cudaStream_t st, StageTimer &tm)
{
    int64_t tot = (int64_t)pd.n * nrhs;
    tm.mark(-1, 0, st);
    k_permute_in<T><<<grid_for(tot, 256), 256, 0, st>>>(in_user, in_sorted, pd.perm, pd.n, nrhs);
    tm.mark(STAGE_PERMUTE_IN, 1, st);
    cudaError_t e;
    if (pd.Ps == 3 && pd.Pang == 5) e = launch_orders<T, 3, 5>(pd, nrhs, in_sorted, out_sorted, mode, adjoint, st, tm);
    else if (pd.Ps == 4 && pd.Pang == 7) e = launch_orders<T, 4, 7>(pd, nrhs, in_sorted, out_sorted, mode, adjoint, st, tm);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    k_permute_out<T><<<grid_for(tot, 256), 256, 0, st>>>(out_sorted, out_user, pd.perm, pd.n, nrhs);
    tm.mark(STAGE_PERMUTE_OUT, 1, st);
    return cudaGetLastError();
}

}  // namespace ifgf
