// Device helpers shared by the plan and apply kernels.
//
// Index path (box coordinates, cone cells, interpolation-point positions): only
// correctly rounded double operations (__dadd_rn, __dsub_rn, __dmul_rn,
// __ddiv_rn, __dsqrt_rn) in a fixed order, never contracted into FMAs, and
// trigonometric values only from host-computed tables.  This makes every box
// and cone index a deterministic function of the input bits.
#pragma once

#include <cstdint>

#include "ifgf_internal.h"

namespace ifgf {

template <typename T> struct cpx { T x, y; };

template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }

// ----------------------------------------------------------------------------------
// Cone cell of the vector v = y - c at level L (cells of Eq. defconedomain and
// defconedomainproduct).  Cells are half-open; the theta cell is the number of
// k in 1..n_C-1 with v_z/r <= cos(k pi/n_C); the phi cell is found the same way
// from v_x/rho on [0, pi] (v_y >= 0) and on (pi, 2 pi) (v_y < 0, where the cell
// boundaries are -cos(k pi/n_C)).  On the axis (rho == 0) the pole rule of
// Eq. (defconedomain) applies: theta = 0 lies in the first phi cell, theta = pi
// in the last.  Returns the linear id (g1 n_C + g2) 2 n_C + g3 and the
// quantities that the local coordinates need.
// ----------------------------------------------------------------------------------
struct ConeGeom {
    double r, rho, s_over_ds;   // distance, distance to the axis, s / Delta_s
    int g1, g2, g3;
    int cone;
};

__device__ __forceinline__ ConeGeom cone_of(const LevelDev &L, double vx, double vy, double vz)
{
    ConeGeom o;
    double rho2 = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
    double r = __dsqrt_rn(__dadd_rn(rho2, __dmul_rn(vz, vz)));
    double rho = __dsqrt_rn(rho2);
    o.r = r;
    o.rho = rho;
    const int nc = L.nc, ns = L.ns;
    if (r == 0.0) {
        o.g1 = o.g2 = o.g3 = 0;
        o.s_over_ds = 0.0;
    } else {
        double s = __ddiv_rn(L.h, r);
        double q = __ddiv_rn(s, L.ds);
        o.s_over_ds = q;
        double fq = floor(q);
        o.g1 = fq < 0.0 ? 0 : (fq > (double)(ns - 1) ? ns - 1 : (int)fq);
        double ct = __ddiv_rn(vz, r);
        // cosk is strictly decreasing: count k in [1, nc-1] with ct <= cosk[k]
        int lo = 1, hi = nc;  // answer m in [0, nc-1]: cosk[1..m] >= ct
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (ct <= L.cosk[mid]) lo = mid + 1; else hi = mid;
        }
        o.g2 = lo - 1;
        if (rho == 0.0) {
            o.g3 = vz > 0.0 ? 0 : 2 * nc - 1;
        } else {
            double cp = __ddiv_rn(vx, rho);
            if (vy >= 0.0) {
                // count j in [1, nc] with cp <= cosk[j]
                int a = 1, b = nc + 1;
                while (a < b) {
                    int mid = (a + b) >> 1;
                    if (cp <= L.cosk[mid]) a = mid + 1; else b = mid;
                }
                o.g3 = a - 1;
            } else {
                // nc + count j in [1, nc-1] with cp >= -cosk[j]  (-cosk increasing)
                int a = 1, b = nc;
                while (a < b) {
                    int mid = (a + b) >> 1;
                    if (cp >= -L.cosk[mid]) a = mid + 1; else b = mid;
                }
                o.g3 = nc + a - 1;
            }
        }
    }
    o.cone = (o.g1 * nc + o.g2) * (2 * nc) + o.g3;
    return o;
}

// ----------------------------------------------------------------------------------
// Fast cone cell: the same cell as cone_of, for a fraction of its FP64 cost.
// 1/r and 1/rho start from FP32 rsqrt (relative error < 2^-22) and take one FP64
// Newton step (error < 1.5 * 2^-44 < 1e-13), so s/Delta_s, v_z/r and v_x/rho are
// known to better than 1e-13 relative.  When every such estimate is farther than
// 1e-11 (relative for s/Delta_s, absolute for the cosines) from the cell boundaries
// that decide it, the cells equal those of the correctly rounded path; otherwise the
// correctly rounded cone_of decides.  The estimates of r, rho and s/Delta_s feed
// the value path (1e-13 relative).
// ----------------------------------------------------------------------------------
__device__ __forceinline__ int count_le(const double *tab, int lo, int hi, double x)
{
    // number of k in [lo, hi) with x <= tab[k], tab strictly decreasing
    int a = lo, b = hi;
    while (a < b) {
        int mid = (a + b) >> 1;
        if (x <= tab[mid]) a = mid + 1; else b = mid;
    }
    return a - lo;
}

__device__ __forceinline__ bool near_edge(double x, const double *tab, int k, int lo, int hi)
{
    // x lies within 1e-11 of tab[k-1] or tab[k] (the boundaries around position k)
    const double m = 1e-11;
    return (k - 1 >= lo && fabs(x - tab[k - 1]) < m) || (k < hi && fabs(x - tab[k]) < m);
}

__device__ __forceinline__ ConeGeom cone_of_fast(const LevelDev &L, double vx, double vy, double vz)
{
    const int nc = L.nc, ns = L.ns;
    float fx = (float)vx, fy = (float)vy, fz = (float)vz;
    float rho2f = fx * fx + fy * fy;
    float r2f = rho2f + fz * fz;
    if (!(rho2f > 1e-30f) || !(r2f > 1e-30f)) return cone_of(L, vx, vy, vz);
    double rho2 = vx * vx + vy * vy;
    double r2 = rho2 + vz * vz;
    double ri = (double)rsqrtf(r2f);
    ri = ri * (1.5 - 0.5 * r2 * ri * ri);
    double hi = (double)rsqrtf(rho2f);
    hi = hi * (1.5 - 0.5 * rho2 * hi * hi);
    ConeGeom o;
    o.r = r2 * ri;
    o.rho = rho2 * hi;
    double q = L.hds * ri;
    o.s_over_ds = q;
    double fq = floor(q);
    double fr = q - fq;
    double mq = 1e-11 * fmax(q, 1.0);
    bool edge = (fr < mq) || (1.0 - fr < mq);
    o.g1 = fq < 0.0 ? 0 : (fq > (double)(ns - 1) ? ns - 1 : (int)fq);
    double ct = vz * ri;
    int m2 = count_le(L.cosk, 1, nc, ct);
    edge = edge || near_edge(ct, L.cosk, m2 + 1, 1, nc);
    o.g2 = m2;
    double cp = vx * hi;
    if (vy >= 0.0) {
        int m3 = count_le(L.cosk, 1, nc + 1, cp);
        edge = edge || near_edge(cp, L.cosk, m3 + 1, 1, nc + 1);
        o.g3 = m3;
    } else {
        // -cosk increasing: count j in [1, nc-1] with cp >= -cosk[j]  <=>  -cp <= cosk[j]
        int m3 = count_le(L.cosk, 1, nc, -cp);
        edge = edge || near_edge(-cp, L.cosk, m3 + 1, 1, nc);
        o.g3 = nc + m3;
    }
    if (edge) {
        ConeGeom e = cone_of(L, vx, vy, vz);
        e.r = o.r;
        e.rho = o.rho;
        e.s_over_ds = q;
        return e;
    }
    o.cone = (o.g1 * nc + o.g2) * (2 * nc) + o.g3;
    return o;
}

// Cone cell for the FP32 value path, with FP64 only where the value path needs it.
// r, 1/r, s / Delta_s and rho are formed in FP64 (1/r and 1/rho from FP32 estimates and
// one FP64 Newton step each, relative error < 1e-13): the local coordinates need them to
// ~1e-10.  The theta and phi cells are decided in FP32 instead: v_z/r and v_x/rho are
// estimated to within 6e-7 (FP32 rounding of the operands, of the product and of the
// FP32 reciprocal square root) and compared with FP32 copies of the boundary cosines
// (rounding 6e-8).  When an estimate lies farther than 2e-6 from both boundaries that
// decide its cell, every comparison has the sign the correctly rounded path finds;
// otherwise, and for a radial quotient within 1e-11 of a boundary or a vector on or
// near the axis, the correctly rounded cone_of decides.  The cells therefore equal
// those of cone_of (and of the plan's activation) bit for bit.
__device__ __forceinline__ int count_le_f(const float *tab, int lo, int hi, float x)
{
    // number of k in [lo, hi) with x <= tab[k], tab strictly decreasing
    int a = lo, b = hi;
    while (a < b) {
        int mid = (a + b) >> 1;
        if (x <= tab[mid]) a = mid + 1; else b = mid;
    }
    return a - lo;
}

__device__ __forceinline__ bool near_edge_f(float x, const float *tab, int k, int lo, int hi)
{
    const float m = 2e-6f;
    return (k - 1 >= lo && fabsf(x - tab[k - 1]) < m) || (k < hi && fabsf(x - tab[k]) < m);
}

__device__ __forceinline__ ConeGeom cone_of_mixed(const LevelDev &L, double vx, double vy, double vz)
{
    const int nc = L.nc, ns = L.ns;
    const float fx = (float)vx, fy = (float)vy, fz = (float)vz;
    const float rho2f = fx * fx + fy * fy;
    const float r2f = rho2f + fz * fz;
    if (!(rho2f > 1e-30f) || !(r2f > 1e-30f) || !(r2f < 1e30f)) return cone_of(L, vx, vy, vz);
    const double rho2 = vx * vx + vy * vy;
    const double r2 = rho2 + vz * vz;
    const float rif = rsqrtf(r2f), hif = rsqrtf(rho2f);
    double ri = (double)rif;
    ri = ri * fma(-0.5 * r2, ri * ri, 1.5);
    double hi = (double)hif;
    hi = hi * fma(-0.5 * rho2, hi * hi, 1.5);
    ConeGeom o;
    o.r = r2 * ri;
    o.rho = rho2 * hi;
    const double q = L.hds * ri;
    o.s_over_ds = q;
    const double fq = floor(q);
    const double fr = q - fq;
    const double mq = 1e-11 * fmax(q, 1.0);
    bool edge = (fr < mq) || (1.0 - fr < mq);
    o.g1 = fq < 0.0 ? 0 : (fq > (double)(ns - 1) ? ns - 1 : (int)fq);
    const float ct = fz * rif;
    const int m2 = count_le_f(L.coskf, 1, nc, ct);
    edge = edge || near_edge_f(ct, L.coskf, m2 + 1, 1, nc);
    o.g2 = m2;
    const float cp = fx * hif;
    if (vy >= 0.0) {
        const int m3 = count_le_f(L.coskf, 1, nc + 1, cp);
        edge = edge || near_edge_f(cp, L.coskf, m3 + 1, 1, nc + 1);
        o.g3 = m3;
    } else {
        const int m3 = count_le_f(L.coskf, 1, nc, -cp);
        edge = edge || near_edge_f(-cp, L.coskf, m3 + 1, 1, nc);
        o.g3 = nc + m3;
    }
    if (edge) {
        ConeGeom e = cone_of(L, vx, vy, vz);
        e.r = o.r;
        e.rho = o.rho;
        e.s_over_ds = q;
        return e;
    }
    o.cone = (o.g1 * nc + o.g2) * (2 * nc) + o.g3;
    return o;
}

// Local coordinates with FP32 angles: the polar and azimuthal angles are rotated to
// the start of their cell in FP64 (no input rounding), and only the in-cell angle,
// in [0, Delta_theta), goes through FP32 atan2 (relative error ~1e-7 of the in-cell
// angle, i.e. ~2e-7 in the local coordinate).
__device__ __forceinline__ void local_coords_f32(const LevelDev &L, const ConeGeom &g, double vx, double vy,
                                                 double vz, float *t)
{
    t[0] = (float)(2.0 * (g.s_over_ds - (double)g.g1) - 1.0);
    double c2 = L.cs_edge[2 * g.g2], s2 = L.cs_edge[2 * g.g2 + 1];
    // angle from the z axis measured from theta_g2 = g2 Delta_theta
    double yt = g.rho * c2 - vz * s2, xt = vz * c2 + g.rho * s2;
    t[1] = 2.0f * (atan2f((float)yt, (float)xt) * L.inv_dth) - 1.0f;
    if (g.rho == 0.0) {
        t[2] = 0.0f;
    } else {
        double c3 = L.cs_edge[2 * g.g3], s3 = L.cs_edge[2 * g.g3 + 1];
        double yp = vy * c3 - vx * s3, xp = vx * c3 + vy * s3;
        t[2] = 2.0f * (atan2f((float)yp, (float)xp) * L.inv_dth) - 1.0f;
    }
}

// Local coordinates in [-1, 1] of (s, theta, phi) inside the cell (value path).
__device__ __forceinline__ void local_coords(const LevelDev &L, const ConeGeom &g, double vx,
                                             double vy, double vz, double *t)
{
    t[0] = 2.0 * (g.s_over_ds - (double)g.g1) - 1.0;
    double th = atan2(g.rho, vz);
    t[1] = 2.0 * (th / L.dth - (double)g.g2) - 1.0;
    if (g.rho == 0.0) {
        t[2] = 0.0;
    } else {
        double ph = atan2(vy, vx);
        if (ph < 0.0) ph += 6.283185307179586476925286766559;
        t[2] = 2.0 * (ph / L.dth - (double)g.g3) - 1.0;
    }
}

// Interpolation point `node` = (a, b, c) of cone `cone` around centre (cx, cy, cz),
// Eq. (interp_pts): centre + (h/s_a) (sin th_b cos ph_c, sin th_b sin ph_c, cos th_b).
// Exact-rounding order; returns the radius h/s_a and the unit direction.
__device__ __forceinline__ double node_pos(const LevelDev &L, int Ps, int Pang, int cone, int node,
                                           double cx, double cy, double cz, double *q, double *dir)
{
    const int nc = L.nc;
    int g3 = cone % (2 * nc);
    int g2 = (cone / (2 * nc)) % nc;
    int g1 = cone / (2 * nc) / nc;
    int a = node / (Pang * Pang), b = (node / Pang) % Pang, c = node % Pang;
    double R = L.nodeR[g1 * Ps + a];
    double st = L.sth[g2 * Pang + b], ct = L.cth[g2 * Pang + b];
    double sp = L.sph[g3 * Pang + c], cp = L.cph[g3 * Pang + c];
    double dx = __dmul_rn(st, cp), dy = __dmul_rn(st, sp);
    q[0] = __dadd_rn(cx, __dmul_rn(R, dx));
    q[1] = __dadd_rn(cy, __dmul_rn(R, dy));
    q[2] = __dadd_rn(cz, __dmul_rn(R, ct));
    if (dir) { dir[0] = dx; dir[1] = dy; dir[2] = ct; }
    return R;
}

// Interpolation point `node` of the level-(d-1) cone `cone` (level params Lp) seen
// from the centre of the child box in octant `oct` (bit 0: x, 1: y, 2: z): the point
// is x_j + R dir (Eq. interp_pts) and the child centre x_j + delta with
// delta_i = +-H_d/2 exactly (Eq. defboxsizesandcenters), so v = R dir - delta.  This
// form does not depend on where the boxes are, which makes the upward geometry of
// a level a function of (cone, node, octant) only.  hh = H_d / 2.
__device__ __forceinline__ double node_rel(const LevelDev &Lp, int Ps, int Pang, int cone, int node,
                                           double hh, int oct, double *v, double *dir)
{
    const int nc = Lp.nc;
    int g3 = cone % (2 * nc);
    int g2 = (cone / (2 * nc)) % nc;
    int g1 = cone / (2 * nc) / nc;
    int a = node / (Pang * Pang), b = (node / Pang) % Pang, c = node % Pang;
    double R = Lp.nodeR[g1 * Ps + a];
    double st = Lp.sth[g2 * Pang + b], ct = Lp.cth[g2 * Pang + b];
    double sp = Lp.sph[g3 * Pang + c], cp = Lp.cph[g3 * Pang + c];
    double dx = __dmul_rn(st, cp), dy = __dmul_rn(st, sp);
    v[0] = __dsub_rn(__dmul_rn(R, dx), (oct & 1) ? hh : -hh);
    v[1] = __dsub_rn(__dmul_rn(R, dy), (oct & 2) ? hh : -hh);
    v[2] = __dsub_rn(__dmul_rn(R, ct), (oct & 4) ? hh : -hh);
    if (dir) { dir[0] = dx; dir[1] = dy; dir[2] = ct; }
    return R;
}

// Row of cone id `cone` in a level's upward table (union bitmap + rank), -1 if absent.
__device__ __forceinline__ int table_row(const uint64_t *ubits, const int *urank, int cone)
{
    uint64_t word = ubits[cone >> 6];
    uint64_t bit = 1ull << (cone & 63);
    if (!(word & bit)) return -1;
    return urank[cone >> 6] + __popcll(word & (bit - 1));
}

// Slot of cone id `cone` of box b via the bitmap rank directory; -1 if not relevant.
__device__ __forceinline__ int cone_slot(const LevelDev &L, int b, int cone)
{
    size_t w = (size_t)b * L.words + (cone >> 6);
    uint64_t word = L.bits[w];
    uint64_t bit = 1ull << (cone & 63);
    if (!(word & bit)) return -1;
    return L.rank[w] + __popcll(word & (bit - 1));
}

// Lagrange basis at the first-kind Chebyshev nodes: w_a = inv_a prod_{e != a}(t - t_e).
template <typename W>
__device__ __forceinline__ void lagrange(int n, const double *nodes, const double *inv, W t, W *w)
{
    W d[IFGF_MAX_P];
#pragma unroll
    for (int e = 0; e < IFGF_MAX_P; ++e)
        if (e < n) d[e] = t - (W)nodes[e];
#pragma unroll
    for (int a = 0; a < IFGF_MAX_P; ++a) {
        if (a < n) {
            W v = (W)inv[a];
#pragma unroll
            for (int e = 0; e < IFGF_MAX_P; ++e)
                if (e < n && e != a) v *= d[e];
            w[a] = v;
        }
    }
}

// The same in FP32 from FP32 copies of the nodes and weights, so that no call
// converts from FP64.
__device__ __forceinline__ void lagrange(int n, const float *nodes, const float *inv, float t, float *w)
{
    float d[IFGF_MAX_P];
#pragma unroll
    for (int e = 0; e < IFGF_MAX_P; ++e)
        if (e < n) d[e] = t - nodes[e];
#pragma unroll
    for (int a = 0; a < IFGF_MAX_P; ++a) {
        if (a < n) {
            float v = inv[a];
#pragma unroll
            for (int e = 0; e < IFGF_MAX_P; ++e)
                if (e < n && e != a) v *= d[e];
            w[a] = v;
        }
    }
}

// exp(i arg) with the argument in FP64: full FP64 sincos for double results; for
// float results the argument is reduced modulo 2 pi in FP64 (Cody-Waite, two-part
// 2 pi) and the reduced angle, in [-pi, pi], goes to the special-function unit's sine
// and cosine (__sincosf, absolute error below 2^-21 there by CUDA's documented bound).
__device__ __forceinline__ void expi(double arg, double &c, double &s) { sincos(arg, &s, &c); }
__device__ __forceinline__ void expi(double arg, float &c, float &s)
{
    const double inv2pi = 0.15915494309189533577;
    const double twopi_hi = 6.283185307179586232;      // nearest double to 2 pi
    const double twopi_lo = 2.4492935982947064e-16;    // 2 pi - twopi_hi
    double k = rint(arg * inv2pi);
    double red = fma(-k, twopi_hi, arg);
    red = fma(-k, twopi_lo, red);
    __sincosf((float)red, &s, &c);
}

// exp(i x) for an FP32 argument of moderate size (|x| below 2^16 * 2 pi).  Cody-Waite
// reduction (W. J. Cody and W. Waite, Software Manual for the Elementary Functions, 1980)
// by 2 pi split as 201/32 (8 significant bits, so k * 201/32 is exact for |k| < 2^16) plus
// the FP32 remainder 2 pi - 201/32 (error 1e-11); the reduced angle, in [-pi, pi], goes to
// __sincosf (absolute error below 2^-21 there).  Against FP32 sincosf this adds at most
// about 4e-7 to each factor, far below the error of the FP32 argument itself.
__device__ __forceinline__ void expi_f32(float x, float &c, float &s)
{
    const float k = rintf(x * 0.159154943f);
    float r = fmaf(-k, 6.28125f, x);
    r = fmaf(-k, 1.93530717e-3f, r);
    __sincosf(r, &s, &c);
}

}  // namespace ifgf
