// Batched right-hand sides on tensor cores (IFGF_BATCHED_BF16 and IFGF_BATCHED_FP16 plans).
//
// With many right-hand sides the interpolation of Algorithm 1 is a set of small
// dense contractions that share their cone values: every evaluation that reads
// relevant cone s of level d (a cousin target of Algorithm 1's target step, or a
// parent interpolation point of its upward step) computes
//     out[row][r] = f_row * sum_p W[row][p] F_s^d[p][r],   p < P = 75,
// with real Lagrange weights W (Eq. defchebyshevinterpooperator, Lagrange form) and
// a complex factor f_row (the centred factor G(x, x_k^d) of Eq. I_k for targets,
// the re-centring factor G(x, x_k^d)/G(x, x_j^{d-1}) for parent points).  Grouping
// the rows by source cone turns this into one GEMM per cone,
//     D (rows x 2 nrhs) = A (rows x 80) * B (80 x 2 nrhs),
// with B = the cone's values (re/im interleaved, 75 rows padded to 80) loaded once.
//
// k_cone_mma: persistent CTAs (two per SM) walk the relevant cones of a level in
// chunks of 128 rows.  For each cone B goes to shared memory as BF16 hi + lo parts;
// for each chunk A (hi + lo) is written and one thread issues tcgen05.mma
// (kind::f16, BF16 inputs, FP32 accumulation in tensor memory): Ahi Bhi + Ahi Blo +
// Alo Bhi per K block of 16, which keeps ~16 significant bits of both operands.  With
// FP16 operands (IFGF_BATCHED_FP16) the hi + lo split keeps ~22 bits; the values of
// each cone are scaled by a power of two into [-1, 1] (FP16's range is narrow) and the
// row factors of its chunks carry the inverse power.
// While the tensor cores run, the threads compute the rows of the CTA's next chunk.
// The epilogue reads the accumulator with tcgen05.ld, multiplies each row by its
// complex factor, transposes 32 rows through shared memory and adds them to their
// destinations with warp-coalesced red.global.add.v4.f32 (one 128-byte row segment
// per 8 lanes).  Destinations receive contributions from several cones, so the
// summation order (and the last bits of the result) varies from run to run on this
// path.
//
// The level-D direct sums (near field) and the leaf analytic factors run on CUDA cores:
// the near field by warps whose lanes own right-hand sides, each Green-function value
// computed once per pair and broadcast; the leaf factors by blocks that stage a chunk
// of sources' densities and factors in shared memory and contract them from there.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ifgf_apply_impl.cuh"

namespace ifgf {
namespace batched {

// Interpolation order of a batched plan: P = P_s P_ang^2 nodes per cone, the contraction
// length K (P padded to a multiple of 16, the K of one kind::f16 MMA), NW Lagrange weights.
template <int PS_, int PA_> struct Ord {
    static constexpr int PS = PS_, PA = PA_;
    static constexpr int P = PS * PA * PA;
    static constexpr int K = (P + 15) / 16 * 16;
    static constexpr int NW = PS + 2 * PA;
    static constexpr uint32_t SBO_A = (K / 8) * 128;  // byte stride of 8-row groups of A
};
using Ord35 = Ord<3, 5>;  // 75 nodes, K = 80
using Ord47 = Ord<4, 7>;  // 196 nodes, K = 208
// largest even nrhs of the tensor-core path per order (shared memory: A and B hi + lo)
constexpr int kMaxBatched35 = 64, kMaxBatched47 = 48;
constexpr int kM = 128;       // rows per MMA
constexpr int kThreads = 128;
constexpr int kWaitLimit = 1 << 22;
constexpr int kBatch = 16;     // cone-value loads in flight per thread
constexpr int kStageStride = 32 * 4 + 16;  // one epilogue pass: 32 floats per row, padded

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, LBO = byte
// stride between 8x16-byte core matrices along K, SBO = byte stride along M/N.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: FP32 accumulate, A and B both BF16 (F16 = false) or both FP16
// (F16 = true), A K-major, B MN-major
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, bool f16 = false)
{
    return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// x = hi + lo + O(2^-16 |x|) in BF16 (F16 = false), or + O(2^-22 |x|) in FP16 (F16 = true,
// for |x| within the FP16 range: the cone values are scaled into [-1, 1] per cone)
template <bool F16> __device__ __forceinline__ uint32_t split_hi_lo(float x, uint16_t &lo)
{
    if constexpr (F16) {
        const __half h = __float2half_rn(x);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
        return __half_as_ushort(h);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
        return __bfloat16_as_ushort(h);
    }
}

// A (kM x K, K-major): element (m, k) at (m/8)*SBO_A + (k/8)*128 + (m%8)*16 + (k%8)*2
template <class O> __device__ __forceinline__ uint32_t a_off(int m, int k)
{
    return (m >> 3) * O::SBO_A + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2;
}
// B (K x Npad, MN-major): element (k, n) at (k/8)*LBO_B + (n/8)*128 + (k%8)*16 + (n%8)*2, LBO_B = Npad/8*128
__device__ __forceinline__ uint32_t b_off(int k, int n, uint32_t lbo_b)
{
    return (k >> 3) * lbo_b + (n >> 3) * 128 + (k & 7) * 16 + (n & 7) * 2;
}

struct ConeKernelArgs {
    int d;            // level of the cones
    int nrhs;
    int npad;         // 2 nrhs rounded up to a multiple of 16, <= 256
    int tmem_cols;    // power of two >= max(32, npad)
    int do_targets;   // cousin targets of level d -> u
    int do_upward;    // parent interpolation points (d > 3) -> F^{d-1}
    float2 *u;        // sorted fields [N][nrhs]
    int *work;        // cone counter of this launch, zero at launch
    int wait_limit;   // iterations of the bounded wait for a chunk's MMAs
    int skip_mma;     // testing: issue no MMA, so that the waits run out
};

// One CTA job: 128 rows (a chunk) of the evaluations that read relevant cone `slot`,
// the CTA's cone number q.
struct ConeJob {
    int slot, c0, rows, rows_t, t0, u0, q;
};

// The CTA takes its cones one at a time from a level-wide counter, in slot order
// (slots are box-major in Morton order), so that all CTAs work on neighbouring boxes
// and the destinations of their reductions stay in L2.  sq[q % 2] holds the slot of
// the CTA's cone q, fetched one cone ahead by thread 0 (take_cone).
__device__ __forceinline__ bool next_job(const LevelDev &L, const ConeKernelArgs &a, const int *sq, ConeJob &j)
{
    if (j.slot >= 0 && j.c0 + kM < j.rows) {
        j.c0 += kM;
        return true;
    }
    const int q = j.slot < 0 ? 0 : j.q + 1;
    const int s = sq[q & 1];
    if (s >= L.nact) {
        j.slot = L.nact;
        return false;
    }
    const bool up = a.do_upward && a.d > 3;
    j.slot = s;
    j.q = q;
    j.c0 = 0;
    j.t0 = a.do_targets ? L.tl_start[s] : 0;
    j.rows_t = a.do_targets ? L.tl_start[s + 1] - j.t0 : 0;
    j.u0 = up ? L.ul_start[s] : 0;
    j.rows = j.rows_t + (up ? L.ul_start[s + 1] - j.u0 : 0);  // an empty cone is one empty chunk
    return true;
}

__device__ __forceinline__ int take_cone(const ConeKernelArgs &a) { return atomicAdd(a.work, 1); }

struct RowData {
    float2 *dest;   // destination row (nrhs complex values), nullptr past the job's rows
    float fr, fi;   // complex factor of the row
};

// Lagrange weights w[NW] and factor of row `row` of job j: a cousin target (centred
// factor G(x, x_k^d)) or a parent interpolation point (re-centring factor)
template <class O>
__device__ __forceinline__ RowData row_geometry(const PlanDev &pd, const LevelDev &L, const LevelDev *Lp,
                                                const ConeKernelArgs &a, const ConeJob &j, bool tab, int row,
                                                float *w)
{
    RowData rd = {nullptr, 0.f, 0.f};
    const int r = j.c0 + row;
    if (r >= j.rows) return rd;
    cpx<float> f;
    if (r < j.rows_t) {
        const int e = j.t0 + r;
        const int i = L.tl[e];
        if (L.tl_loc) {
            float4 t = L.tl_loc[e];
            float2 G = L.tl_fac[e];
            lagrange(O::PS, pd.tsf, pd.itsf, t.x, w);
            lagrange(O::PA, pd.taf, pd.itaf, t.y, w + O::PS);
            lagrange(O::PA, pd.taf, pd.itaf, t.z, w + O::PS + O::PA);
            f = {G.x, G.y};
        } else {
            const double *ck = L.center + 3 * (size_t)L.act_box[j.slot];
            double vx = __dsub_rn(pd.xs[i], ck[0]), vy = __dsub_rn(pd.ys[i], ck[1]), vz = __dsub_rn(pd.zs[i], ck[2]);
            ConeGeom g = geom_weights<float, O::PS, O::PA>(pd, L, vx, vy, vz, w);
            f = green_r<float>(pd.kappa, g.r);
        }
        rd.dest = a.u + (size_t)i * a.nrhs;
    } else {
        const int e = L.ul[j.u0 + r - j.rows_t];
        const int psl = e / O::P, node = e % O::P;
        const int pcone = Lp->act_cone[psl];
        const int oct = (int)(L.key[L.act_box[j.slot]] & 7u);
        const int trow = tab ? table_row(L.ubits, L.urank, pcone) : -1;
        if (trow >= 0) {
            up_entry<float, O::PS, O::PA>(pd, ((const UpEntry32 *)L.utab)[((size_t)trow * 8 + oct) * O::P + node], w, f);
        } else {
            up_geometry<float, O::PS, O::PA>(pd, L, *Lp, pcone, node, oct, w, f);
        }
        rd.dest = (float2 *)Lp->F + ((size_t)psl * O::P + node) * a.nrhs;
    }
    rd.fr = f.x;
    rd.fi = f.y;
    return rd;
}

// A row `row` from its weights: W[p] = ws[a] wt[b] wp[c], p = (a P_ang + b) P_ang + c, as
// hi and lo parts (BF16 or FP16); zero for an empty row and for the padding columns p >= P
template <bool F16, class O>
__device__ __forceinline__ void write_A_row(const float *w, bool valid, int row, unsigned char *A_hi,
                                            unsigned char *A_lo)
{
#pragma unroll
    for (int kc = 0; kc < O::K / 8; ++kc) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h2[2], l2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = kc * 8 + q * 2 + h;
                float x = 0.f;
                if (valid && p < O::P) {
                    const int ia = p / (O::PA * O::PA), ib = (p / O::PA) % O::PA, ic = p % O::PA;
                    x = w[ia] * w[O::PS + ib] * w[O::PS + O::PA + ic];
                }
                uint16_t lo;
                h2[h] = split_hi_lo<F16>(x, lo);
                l2[h] = lo;
            }
            hv[q] = h2[0] | (h2[1] << 16);
            lv[q] = l2[0] | (l2[1] << 16);
        }
        const uint32_t off = a_off<O>(row, kc * 8);
        *(uint4 *)(A_hi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *(uint4 *)(A_lo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

// The cone's values as B (hi, lo), times `scale`: complex -> (re, im) columns 2r, 2r+1.
// Lane l of a warp converts (p, r) = (8 pb + l / 4, 4 rb + l % 4) of a tile (pb, rb), so
// that its 32 four-byte stores fill one core matrix (no bank conflicts) and its loads read
// eight 32-byte runs.  Batches of kBatch independent loads per thread before any
// conversion; nt threads (a multiple of 32) take part, t is this thread's index.
template <bool F16, class O>
__device__ __forceinline__ void load_cone_B(const LevelDev &L, int slot, int nrhs, int npad, uint32_t lbo_b,
                                            unsigned char *B_hi, unsigned char *B_lo, int t, int nt, float scale)
{
    const float2 *F = (const float2 *)L.F + (size_t)slot * O::P * nrhs;
    const int ntr = npad / 8;               // r tiles of 4: npad / 2 columns pairs
    const int tot = (O::K / 8) * ntr * 32;  // (p tiles) x (r tiles) x 32 lanes
    for (int base = t; base < tot; base += kBatch * nt) {
        float2 v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = base + u * nt, tile = idx >> 5, l = idx & 31;
            const int p = (tile / ntr) * 8 + (l >> 2), r = (tile % ntr) * 4 + (l & 3);
            v[u] = (idx < tot && p < O::P && r < nrhs) ? __ldg(F + (size_t)p * nrhs + r) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = base + u * nt, tile = idx >> 5, l = idx & 31;
            const int p = (tile / ntr) * 8 + (l >> 2), r = (tile % ntr) * 4 + (l & 3);
            if (idx < tot && p < O::P) {
                uint16_t l0, l1;
                const uint32_t h0 = split_hi_lo<F16>(v[u].x * scale, l0);
                const uint32_t h1 = split_hi_lo<F16>(v[u].y * scale, l1);
                const uint32_t off = b_off(p, 2 * r, lbo_b);
                *(uint32_t *)(B_hi + off) = h0 | (h1 << 16);
                *(uint32_t *)(B_lo + off) = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
        }
    }
}

// Largest |value| (as its non-negative float bits) of the cone's values, over the block.
template <class O>
__device__ __forceinline__ void cone_max_abs(const LevelDev &L, int slot, int nrhs, int t, int nt, unsigned *smax)
{
    const float2 *F = (const float2 *)L.F + (size_t)slot * O::P * nrhs;
    float m = 0.f;
    for (int q = t; q < O::P * nrhs; q += nt) {
        const float2 v = __ldg(F + q);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0 && m > 0.f) atomicMax(smax, __float_as_uint(m));
}

// 3 K / 16 MMAs (the K blocks x {hi.hi, hi.lo, lo.hi}) into the accumulator, then a commit
// that arrives on mbar when they have completed
template <class O>
__device__ __forceinline__ void issue_cone_mma(uint32_t tmem, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                               uint32_t lbo_b, uint32_t idesc, uint32_t mbar)
{
#pragma unroll
    for (int kb = 0; kb < O::K / 16; ++kb) {
        const uint64_t dah = umma_desc(ah + kb * 256, 128, O::SBO_A);
        const uint64_t dal = umma_desc(al + kb * 256, 128, O::SBO_A);
        const uint64_t dbh = umma_desc(bh + kb * 2 * lbo_b, lbo_b, 128);
        const uint64_t dbl = umma_desc(bl + kb * 2 * lbo_b, lbo_b, 128);
        const uint32_t acc0 = kb > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0)
                     : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dah), "l"(dbl), "r"(idesc), "r"(1u)
                     : "memory");
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(dal), "l"(dbh), "r"(idesc), "r"(1u)
                     : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta)
        : "memory");
}

// One pass of 32 accumulator columns [c, c + 32): thread tid writes its row times the
// row's factor to the warp's stage rows; then the warp reads four 128-byte row
// segments per step (16 bytes per lane) and adds them to their destinations with
// red.global.add.v4.f32, so that the additions are coalesced per row.  All stage
// reads and pointer shuffles come before the reductions.
__device__ __forceinline__ void epilogue_pass(const uint32_t (&v)[32], int c, int ncols, int lane, const RowData &rd,
                                              float *srow, const unsigned char *swarp)
{
    const int lr = lane >> 3, lc = (lane & 7) * 4;
    const int ncol = min(32, ncols - c);  // a multiple of 4: nrhs is even
    const unsigned long long dest_u = (unsigned long long)rd.dest;
    __syncwarp();  // the previous pass has read the stage
    if (rd.dest) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            if (j < ncol) {
                const float r0 = __uint_as_float(v[j]), i0 = __uint_as_float(v[j + 1]);
                const float r1 = __uint_as_float(v[j + 2]), i1 = __uint_as_float(v[j + 3]);
                *(float4 *)(srow + j) = make_float4(rd.fr * r0 - rd.fi * i0, rd.fr * i0 + rd.fi * r0,
                                                    rd.fr * r1 - rd.fi * i1, rd.fr * i1 + rd.fi * r1);
            }
        }
    }
    __syncwarp();
    float4 x[8];
    unsigned long long d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int rr = 4 * q + lr;  // the warp's row read by this lane
        d[q] = __shfl_sync(0xffffffffu, dest_u, rr);
        x[q] = *(const float4 *)(swarp + (size_t)rr * kStageStride + lc * 4);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (d[q] != 0ull && lc < ncol)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"((float *)d[q] + c + lc), "f"(x[q].x),
                         "f"(x[q].y), "f"(x[q].z), "f"(x[q].w)
                         : "memory");
    }
}

// Epilogue of one chunk: row tid of the accumulator times the row's factor, added to
// the row's destination; 64 columns are read from tensor memory per wait.
__device__ __forceinline__ void cone_epilogue(uint32_t tmem, int tid, int nrhs, const RowData &rd,
                                              unsigned char *stage)
{
    const int warp = tid >> 5, lane = tid & 31;
    float *srow = (float *)(stage + (size_t)tid * kStageStride);
    const unsigned char *swarp = stage + (size_t)warp * 32 * kStageStride;
    const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
    const int ncols = 2 * nrhs;
    for (int cb = 0; cb < ncols; cb += 64) {
        uint32_t v0[32], v1[32];
        const bool two = cb + 32 < ncols;
        __syncwarp();  // tcgen05.ld / wait::ld are .sync.aligned: the warp must be converged
        tmem_ld32(base + (uint32_t)cb, v0);
        if (two) tmem_ld32(base + (uint32_t)(cb + 32), v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        epilogue_pass(v0, cb, ncols, lane, rd, srow, swarp);
        if (two) epilogue_pass(v1, cb + 32, ncols, lane, rd, srow, swarp);
    }
}

// k_cone_mma: two CTAs of 128 threads per SM; each walks its (cone, 128-row chunk)
// jobs.  Per job: B (when the job starts a cone) and A are written to shared memory,
// one thread issues the MMAs, and while the tensor cores run, every thread computes
// its row of the next job (weights, factor, destination: the global loads of the
// row), then drains this job's accumulator.
template <bool F16, class O>
__global__ void __launch_bounds__(kThreads, 2) k_cone_mma(PlanDev pd, ConeKernelArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int sq[2];  // slots of the CTA's cones q and q + 1 (entry q % 2)
    __shared__ unsigned smax;  // FP16 operands: the cone's largest |value| (float bits)
    const int tid = threadIdx.x, warp = tid >> 5;
    const LevelDev &L = pd.lev[a.d];
    const int npad = a.npad, nrhs = a.nrhs;
    const uint32_t lbo_b = (uint32_t)(npad / 8) * 128;
    unsigned char *A_hi = sm;
    unsigned char *A_lo = A_hi + kM * O::K * 2;
    unsigned char *B_hi = A_lo + kM * O::K * 2;
    unsigned char *B_lo = B_hi + O::K * npad * 2;
    unsigned char *stage = B_lo + O::K * npad * 2;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sq[0] = take_cone(a);
        sq[1] = take_cone(a);
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // padding rows p = P..K-1 of B stay zero for the whole kernel
    for (int idx = tid; idx < (O::K - O::P) * npad; idx += kThreads) {
        const int p = O::P + idx / npad, n = idx % npad;
        *(__nv_bfloat16 *)(B_hi + b_off(p, n, lbo_b)) = __float2bfloat16_rn(0.f);
        *(__nv_bfloat16 *)(B_lo + b_off(p, n, lbo_b)) = __float2bfloat16_rn(0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t idesc = umma_idesc(kM, npad, F16);
    const LevelDev *Lp = a.d > 3 ? &pd.lev[a.d - 1] : nullptr;
    const bool tab = a.do_upward && a.d > 3 && L.utab != nullptr;
    uint32_t phase = 0;

    ConeJob cur;
    cur.slot = -1;
    cur.c0 = 0;
    cur.rows = 0;
    bool have = next_job(L, a, sq, cur);
    float w[O::NW];
    RowData rd = {nullptr, 0.f, 0.f};
    if (have) rd = row_geometry<O>(pd, L, Lp, a, cur, tab, tid, w);
    float unscale = 1.f;  // FP16 operands: the cone's values are scaled by 1 / unscale (a power of two)
    while (have) {
        // the previous job's MMAs have completed: B and A may be rewritten
        if (cur.c0 == 0) {
            float scale = 1.f;
            if constexpr (F16) {
                if (tid == 0) smax = 0u;
                __syncthreads();
                cone_max_abs<O>(L, cur.slot, nrhs, tid, kThreads, &smax);
                __syncthreads();
                const float mx = __uint_as_float(smax);
                int e = 0;
                if (mx > 0.f) frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
                scale = ldexpf(1.f, -e);
                unscale = ldexpf(1.f, e);
            }
            load_cone_B<F16, O>(L, cur.slot, nrhs, npad, lbo_b, B_hi, B_lo, tid, kThreads, scale);
        }
        if constexpr (F16) {
            rd.fr *= unscale;
            rd.fi *= unscale;
        }
        write_A_row<F16, O>(w, rd.dest != nullptr, tid, A_hi, A_lo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !a.skip_mma) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_cone_mma<O>(tmem, smem_u32(A_hi), smem_u32(A_lo), smem_u32(B_hi), smem_u32(B_lo), lbo_b, idesc,
                              smem_u32(&mbar));
        }
        // the next job's row while the tensor cores run this one
        ConeJob nxt = cur;
        const bool have_n = next_job(L, a, sq, nxt);
        // entering cone q: the entry of cone q - 1 takes cone q + 1 (read from the next
        // iteration on, after the barriers below)
        if (tid == 0 && have_n && nxt.c0 == 0) sq[(nxt.q + 1) & 1] = take_cone(a);
        float wn[O::NW];
        RowData rn = {nullptr, 0.f, 0.f};
        if (have_n) rn = row_geometry<O>(pd, L, Lp, a, nxt, tab, tid, wn);
        uint32_t done = 0;
        for (int it = 0; it < a.wait_limit && !done; ++it) {
            asm volatile(
                "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"(phase)
                : "memory");
        }
        // the decision must be the same for every thread of the CTA
        if (__syncthreads_or(done ? 0 : 1)) {
            if (tid == 0) atomicAdd(pd.err, 1);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        cone_epilogue(tmem, tid, nrhs, rd, stage);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        cur = nxt;
        rd = rn;
#pragma unroll
        for (int m = 0; m < O::NW; ++m) w[m] = wn[m];
        have = have_n;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    __syncwarp();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// Plan-time cache of the target rows' geometry: for every entry e of the transpose
// list of level d (cousin target i of the box k of slot s), the local coordinates of
// x_i in its cone and the centred factor G(x_i, x_k^d).  These do not depend on the
// densities; the apply then only expands the Lagrange weights.
__global__ void k_cache_target_geometry(PlanDev pd, int d, float4 *loc, float2 *fac, int64_t m)
{
    const LevelDev &L = pd.lev[d];
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    // slot of entry e: last s with tl_start[s] <= e
    int lo = 0, hi = L.nact;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (L.tl_start[mid] <= e) lo = mid; else hi = mid;
    }
    const int k = L.act_box[lo];
    const int i = L.tl[e];
    const double *ck = L.center + 3 * (size_t)k;
    double vx = __dsub_rn(pd.xs[i], ck[0]), vy = __dsub_rn(pd.ys[i], ck[1]), vz = __dsub_rn(pd.zs[i], ck[2]);
    ConeGeom g = cone_of_fast(L, vx, vy, vz);
    if (g.cone != L.act_cone[lo]) atomicAdd(pd.err, 1);
    float t[3];
    local_coords_f32(L, g, vx, vy, vz, t);
    loc[e] = make_float4(t[0], t[1], t[2], 0.f);
    cpx<float> G = green_r<float>(pd.kappa, g.r);
    fac[e] = make_float2(G.x, G.y);
}

// Near field of the batched path (Algorithm 1's level-D direct evaluations), one block
// per near work item of the plan (up to 32 consecutive targets of one leaf box).  The
// sources of the box's neighbours form one list (near_ranges), copied in chunks of
// kNearKT: the densities [kNearKT][nrhs] with cp.async, the positions as FP64 offsets
// from the box centre split into FP32 high and low parts (Rel32).  The Green function of
// every (target, source) pair of the chunk is computed once into shared memory (zero for
// the self pair), and thread (tx, ty) accumulates targets ty + 8 i and right-hand sides
// tx + 16 k in registers.  Every output is one thread's sum over the sources in list
// order.
constexpr int kNearKT = 32;

template <int RPT>
__global__ void __launch_bounds__(128) k_near_tiled(PlanDev pd, int nrhs, const float2 *sig, float2 *us)
{
    constexpr int TX = 16, NG = 8;
    constexpr int TPT = (kNearTargets + NG - 1) / NG;  // targets per thread
    __shared__ float4 sth[kNearTargets], stl[kNearTargets];  // targets: split offsets
    __shared__ float4 ssh[kNearKT], ssl[kNearKT];            // the chunk's sources
    __shared__ float2 sG[kNearTargets][kNearKT + 1];
    __shared__ __align__(16) float2 ssig[kNearKT * TX * RPT];
    __shared__ int sj[kNearKT];                              // the chunk's point indices
    __shared__ int sbeg[kMaxNearRanges], spre[kMaxNearRanges + 1];
    __shared__ int snr;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int4 item = pd.near_tile[blockIdx.x];
    const LevelDev &LD = pd.lev[item.z];
    const int b = item.x, t0 = item.y;
    const int nt = min(kNearTargets, LD.end[b] - t0);
    const double *cb = LD.center + 3 * (size_t)b;
    const float kf = (float)pd.kappa;
    if (tid < 32) {
        const int nr = near_ranges(LD, b, tid, sbeg, spre);
        if (tid == 0) snr = nr;
    }
    if (tid < nt) {
        const Rel32 p = rel32(pd.xs[t0 + tid], pd.ys[t0 + tid], pd.zs[t0 + tid], cb);
        sth[tid] = make_float4(p.hx, p.hy, p.hz, 0.f);
        stl[tid] = make_float4(p.lx, p.ly, p.lz, 0.f);
    }
    __syncthreads();
    const int nr = snr;
    const int ns = spre[nr];
    float2 acc[TPT][RPT];
#pragma unroll
    for (int i = 0; i < TPT; ++i)
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[i][k] = make_float2(0.f, 0.f);
    const int pieces = nrhs / 2;  // 16-byte pieces of a density row (nrhs is even)
    for (int g0 = 0; g0 < ns; g0 += kNearKT) {
        const int cnt = min(kNearKT, ns - g0);
        if (tid < cnt) {
            const int j = near_source(sbeg, spre, nr, g0 + tid);
            sj[tid] = j;
            const Rel32 p = rel32(pd.xs[j], pd.ys[j], pd.zs[j], cb);
            ssh[tid] = make_float4(p.hx, p.hy, p.hz, 0.f);
            ssl[tid] = make_float4(p.lx, p.ly, p.lz, 0.f);
        }
        __syncthreads();  // sj is complete
        for (int q = tid; q < cnt * pieces; q += blockDim.x) {
            const int s = q / pieces, c = q - s * pieces;
            cp_async16(ssig + s * nrhs + 2 * c, sig + (size_t)sj[s] * nrhs + 2 * c);
        }
        cp_async_wait_all();
        __syncthreads();
        for (int e = tid; e < nt * cnt; e += blockDim.x) {
            const int t = e / cnt, s = e - t * cnt;
            float2 g = make_float2(0.f, 0.f);
            if (sj[s] != t0 + t) {
                const float4 th = sth[t], tl = stl[t];
                const Rel32 pt = {th.x, th.y, th.z, tl.x, tl.y, tl.z};
                const cpx<float> G = green_near32(pt, ssh[s], ssl[s], kf);
                g = make_float2(G.x, G.y);
            }
            sG[t][s] = g;
        }
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            float2 v[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = tx + TX * k;
                v[k] = r < nrhs ? ssig[s * nrhs + r] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                const int t = ty + NG * i;
                if (t < nt) {
                    const float2 g = sG[t][s];
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        acc[i][k].x += g.x * v[k].x - g.y * v[k].y;
                        acc[i][k].y += g.x * v[k].y + g.y * v[k].x;
                    }
                }
            }
        }
        __syncthreads();  // the chunk is read before the next copy overwrites it
    }
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
        const int t = ty + NG * i;
        if (t >= nt) continue;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = tx + TX * k;
            if (r < nrhs) us[(size_t)(t0 + t) * nrhs + r] = acc[i][k];
        }
    }
}

// Leaf analytic factors (Eq. factored_f at the interpolation points of every relevant
// leaf cone, summed over the sources of the cone's box), one block per relevant leaf
// cone.  Per chunk of kLeafKT sources of the box, the densities [kLeafKT][nrhs] are
// copied into shared memory with cp.async and the factors g(q_n, x_j) of the 75 nodes
// are computed once into shared memory (FP32, from the node's FP32 constants and the
// source's stored offset).  The contraction F[n][r] = sum_j g(q_n, x_j) sigma_j[r] then
// runs from shared memory on register tiles: the 128 threads are TX along the
// right-hand sides times NG = 128 / TX along the nodes; thread (tx, ty) holds nodes
// ty + NG i and right-hand sides tx + TX k (k < RPT).  TX is the tile shape the
// autotuner chooses (8, 16 or 32).  Every output is one thread's sum over the sources
// in order, so the result does not depend on the shape.
constexpr int kLeafKT = 32;
constexpr int kLeafShapes = 3;  // TX = 16, 32, 8 (launch_leaf); order (3, 5)

template <int TX, int RPT>
__global__ void __launch_bounds__(128) k_leaf_tiled(PlanDev pd, int nrhs, const float2 *sig)
{
    constexpr int NG = 128 / TX;
    constexpr int NPT = (Ord35::P + NG - 1) / NG;  // nodes per thread
    __shared__ float4 snode[Ord35::P];              // R and dir of each node (FP32)
    __shared__ float4 soff[kLeafKT];          // the chunk's source offsets (delta, |delta|^2)
    __shared__ float2 sg[Ord35::P][kLeafKT + 1];    // g(q_n, x_j); padded against bank conflicts
    __shared__ __align__(16) float2 ssig[kLeafKT * TX * RPT];
    const LevelDev &L = pd.lev[pd.D];
    const int slot = blockIdx.x;
    const int b = L.act_box[slot];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const float kf = (float)pd.kappa;
    if (tid < Ord35::P) {
        const double *c = L.center + 3 * (size_t)b;
        double q[3], dir[3];
        const double R0 = node_pos(L, 3, 5, L.act_cone[slot], tid, c[0], c[1], c[2], q, dir);
        snode[tid] = make_float4((float)R0, (float)dir[0], (float)dir[1], (float)dir[2]);
    }
    float2 acc[NPT][RPT];
#pragma unroll
    for (int i = 0; i < NPT; ++i)
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[i][k] = make_float2(0.f, 0.f);
    const int j0 = L.start[b], j1 = L.end[b];
    for (int jb = j0; jb < j1; jb += kLeafKT) {
        const int cnt = min(kLeafKT, j1 - jb);
        __syncthreads();  // the previous chunk is consumed (and the node constants are written)
        // nrhs is even: a chunk's rows are cnt * nrhs / 2 aligned 16-byte pieces
        const int pieces = cnt * nrhs / 2;
        for (int q = tid; q < pieces; q += blockDim.x) cp_async16(ssig + 2 * q, sig + (size_t)jb * nrhs + 2 * q);
        if (tid < cnt) soff[tid] = pd.leaf_off[jb + tid];
        cp_async_wait_all();
        __syncthreads();
        for (int e = tid; e < Ord35::P * cnt; e += blockDim.x) {
            const int n = e / cnt, t = e - n * cnt;
            const float4 nd = snode[n];
            const cpx<float> g = leaf_factor32(nd.x, nd.y, nd.z, nd.w, kf, soff[t]);
            sg[n][t] = make_float2(g.x, g.y);
        }
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            float2 s[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = tx + TX * k;
                s[k] = r < nrhs ? ssig[t * nrhs + r] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                const int n = ty + NG * i;
                if (n < Ord35::P) {
                    const float2 g = sg[n][t];
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        acc[i][k].x += g.x * s[k].x - g.y * s[k].y;
                        acc[i][k].y += g.x * s[k].y + g.y * s[k].x;
                    }
                }
            }
        }
    }
    float2 *F = (float2 *)L.F + (size_t)slot * Ord35::P * nrhs;
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
        const int n = ty + NG * i;
        if (n >= Ord35::P) continue;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = tx + TX * k;
            if (r < nrhs) F[(size_t)n * nrhs + r] = acc[i][k];
        }
    }
}

// right-hand sides per thread: the fewest of 1, 2, 4, 8 with TX * RPT >= nrhs (nrhs <= 64)
template <int TX>
void launch_leaf_shape(const PlanDev &pd, int nrhs, const float2 *sig, int nact, cudaStream_t st)
{
    const int rpt = (nrhs + TX - 1) / TX;
    if (rpt <= 1) {
        k_leaf_tiled<TX, 1><<<nact, 128, 0, st>>>(pd, nrhs, sig);
    } else if (rpt <= 2) {
        k_leaf_tiled<TX, 2><<<nact, 128, 0, st>>>(pd, nrhs, sig);
    } else {
        if constexpr (TX <= 16) {
            if (rpt <= 4) k_leaf_tiled<TX, 4><<<nact, 128, 0, st>>>(pd, nrhs, sig);
            else if constexpr (TX <= 8) k_leaf_tiled<TX, 8><<<nact, 128, 0, st>>>(pd, nrhs, sig);
        }
    }
}

// leaf factors of all relevant leaf cones with tile shape `shape` (an index of kLeafTX);
// order (4, 7) plans run the mixed path's leaf kernel (one thread per node, right-hand
// sides in blocks of 8)
inline void launch_leaf(const PlanDev &pd, int nrhs, const float2 *sig, int shape, cudaStream_t st)
{
    const int nact = pd.lev[pd.D].nact;
    if (nact == 0) return;
    if (pd.Ps == 4) {
        ifgf::launch_leaf<float, 8, 4, 7>(pd, pd.D, nrhs, sig, st);
        return;
    }
    if (shape == 1) launch_leaf_shape<32>(pd, nrhs, sig, nact, st);
    else if (shape == 2) launch_leaf_shape<8>(pd, nrhs, sig, nact, st);
    else launch_leaf_shape<16>(pd, nrhs, sig, nact, st);
}

// the CUDA-core stages of the batched path: leaf factors, near field
inline cudaError_t launch_cuda_core(const PlanDev &pd, int nrhs, const float2 *sig, float2 *us, int mode,
                                    cudaStream_t st, StageTimer &tm)
{
    if (mode & 2) {
        launch_leaf(pd, nrhs, sig, pd.tune_leaf, st);
        tm.mark(STAGE_LEAF, pd.lev[pd.D].nact > 0, st);
    }
    if (mode & 1) {
        if (nrhs <= 16) k_near_tiled<1><<<pd.n_near_tile, 128, 0, st>>>(pd, nrhs, sig, us);
        else if (nrhs <= 32) k_near_tiled<2><<<pd.n_near_tile, 128, 0, st>>>(pd, nrhs, sig, us);
        else k_near_tiled<4><<<pd.n_near_tile, 128, 0, st>>>(pd, nrhs, sig, us);
    } else {
        const cudaError_t e = cudaMemsetAsync(us, 0, (size_t)pd.n * nrhs * sizeof(float2), st);
        if (e != cudaSuccess) return e;
    }
    tm.mark(STAGE_EVAL, 1, st);
    return cudaGetLastError();
}

}  // namespace batched
}  // namespace ifgf

// Shared memory of k_cone_mma for npad columns and contraction length K.
static size_t cone_mma_smem(int npad, int K)
{
    using namespace ifgf::batched;
    return (size_t)2 * kM * K * 2 + (size_t)2 * K * npad * 2 + (size_t)kM * kStageStride;
}

// Raises k_cone_mma's dynamic shared-memory limit to what the largest batch of each order
// needs (64 right-hand sides, 128 columns, at order (3, 5): 98 KB, two CTAs per SM; 48, 96
// columns, at order (4, 7): 205 KB, one CTA per SM).  Called once per batched plan, so
// that evaluations queue only stream-ordered work (and can be captured into CUDA graphs).
cudaError_t ifgf_batched_prepare()
{
    using namespace ifgf::batched;
    const int s35 = (int)cone_mma_smem(2 * kMaxBatched35, Ord35::K);
    const int s47 = (int)cone_mma_smem(2 * kMaxBatched47, Ord47::K);
    cudaError_t e = cudaFuncSetAttribute(k_cone_mma<false, Ord35>, cudaFuncAttributeMaxDynamicSharedMemorySize, s35);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cone_mma<true, Ord35>, cudaFuncAttributeMaxDynamicSharedMemorySize, s35);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cone_mma<false, Ord47>, cudaFuncAttributeMaxDynamicSharedMemorySize, s47);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cone_mma<true, Ord47>, cudaFuncAttributeMaxDynamicSharedMemorySize, s47);
    return e;
}

// the largest nrhs the tensor-core path takes for a plan's order
int ifgf_batched_max_nrhs(int Ps) { return Ps == 4 ? ifgf::batched::kMaxBatched47 : ifgf::batched::kMaxBatched35; }

// The tensor-core cone kernels of levels D..3 (targets of every level, parent
// interpolation points above level 3), ctas persistent CTAs per SM.
static cudaError_t launch_cones(const PlanDev &pd, int nrhs, float2 *us, int ctas, cudaStream_t st, int *launches)
{
    using namespace ifgf;
    using namespace ifgf::batched;
    const int npad = ((2 * nrhs + 15) / 16) * 16;
    int tcols = 32;
    while (tcols < npad) tcols *= 2;
    const bool o47 = pd.Ps == 4;
    // within the limit ifgf_batched_prepare set
    const size_t smem = cone_mma_smem(npad, o47 ? Ord47::K : Ord35::K);
    const int P = o47 ? Ord47::P : Ord35::P;
    for (int d = pd.D; d >= 3; --d) {
        const LevelDev &L = pd.lev[d];
        if (d > 3) {
            const LevelDev &Lp = pd.lev[d - 1];
            const cudaError_t e = cudaMemsetAsync(Lp.F, 0, (size_t)Lp.nact * P * nrhs * sizeof(float2), st);
            if (e != cudaSuccess) return e;
        }
        if (L.nact == 0) continue;
        NvtxRange range("tensor-core cones", d);
        ConeKernelArgs a;
        a.d = d;
        a.nrhs = nrhs;
        a.npad = npad;
        a.tmem_cols = tcols;
        a.do_targets = 1;
        a.do_upward = d > 3;
        a.u = us;
        a.work = pd.sched + d;
        a.skip_mma = (pd.flags & 256) ? 1 : 0;
        a.wait_limit = a.skip_mma ? (1 << 10) : kWaitLimit;
        const cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        // one CTA per SM when two do not fit (order (4, 7))
        const int per_sm = (ctas == 1 || 2 * smem > 227 * 1024) ? 1 : 2;
        const int grid = std::min(L.nact, per_sm * 152);
        if (o47) {
            if (pd.batched_f16) k_cone_mma<true, Ord47><<<grid, kThreads, smem, st>>>(pd, a);
            else k_cone_mma<false, Ord47><<<grid, kThreads, smem, st>>>(pd, a);
        } else {
            if (pd.batched_f16) k_cone_mma<true, Ord35><<<grid, kThreads, smem, st>>>(pd, a);
            else k_cone_mma<false, Ord35><<<grid, kThreads, smem, st>>>(pd, a);
        }
        ++*launches;
    }
    return cudaGetLastError();
}

// Autotuner of the batched path for nrhs right-hand sides (even, <= 64): times each
// leaf tile shape and each cone-kernel grid (1 or 2 persistent CTAs per SM) on this
// plan's relevant cones, over reps runs after one warm-up run, and keeps the fastest
// of each in pd.  The runs read sig (Morton-ordered densities, [N][nrhs]) and write the
// plan's cone values and us (scratch).  ms[] receives the mean time of every
// candidate: leaf shapes 0..2, then cone grids of 1 and 2 CTAs per SM.  Synchronises
// the stream.
cudaError_t ifgf_batched_autotune(PlanDev &pd, int nrhs, const void *sig, void *us, cudaStream_t st, int reps,
                                  float *ms)
{
    using namespace ifgf;
    using namespace ifgf::batched;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cudaGetLastError();
    }
    cudaError_t err = cudaSuccess;
    auto timed = [&](auto &&run) -> float {
        run();  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) run();
        cudaEventRecord(e1, st);
        float t = 0.f;
        const cudaError_t s = cudaEventSynchronize(e1);
        if (s != cudaSuccess || (err = cudaGetLastError()) != cudaSuccess) {
            if (err == cudaSuccess) err = s;
            return 0.f;
        }
        cudaEventElapsedTime(&t, e0, e1);
        return t / reps;
    };
    int best = 0;
    for (int s = 0; s < kLeafShapes && err == cudaSuccess; ++s) {
        ms[s] = timed([&] { launch_leaf(pd, nrhs, (const float2 *)sig, s, st); });
        if (ms[s] < ms[best]) best = s;
    }
    int best_ctas = 2;
    for (int c = 1; c <= 2 && err == cudaSuccess; ++c) {
        int nl = 0;
        ms[kLeafShapes + c - 1] = timed([&] {
            const cudaError_t le = launch_cones(pd, nrhs, (float2 *)us, c, st, &nl);
            if (le != cudaSuccess && err == cudaSuccess) err = le;
        });
    }
    if (err == cudaSuccess) {
        best_ctas = ms[kLeafShapes] < ms[kLeafShapes + 1] ? 1 : 2;
        pd.tune_leaf = best;
        pd.tune_cone_ctas = best_ctas;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

// Forward apply of a batched plan (device pointers to Morton-ordered buffers).
cudaError_t ifgf_run_batched(const PlanDev &pd, int nrhs, const void *in_user, void *out_user, void *in_sorted,
                             void *out_sorted, int mode, cudaStream_t st, StageTimer &tm)
{
    using namespace ifgf;
    using namespace ifgf::batched;
    const int n = pd.n;
    int64_t tot = (int64_t)n * nrhs;
    tm.mark(-1, 0, st);
    k_permute_in<float><<<grid_for(tot, 256), 256, 0, st>>>(in_user, in_sorted, pd.perm, n, nrhs);
    tm.mark(STAGE_PERMUTE_IN, 1, st);
    const float2 *sig = (const float2 *)in_sorted;
    float2 *us = (float2 *)out_sorted;
    cudaError_t e;
    e = launch_cuda_core(pd, nrhs, sig, us, mode, st, tm);
    if (e != cudaSuccess) return e;
    if (mode & 2) {
        int nl = 0;
        e = launch_cones(pd, nrhs, us, pd.tune_cone_ctas, st, &nl);
        tm.mark(STAGE_UPWARD, nl, st);
        if (e != cudaSuccess) return e;
    }
    k_permute_out<float><<<grid_for(tot, 256), 256, 0, st>>>(out_sorted, out_user, pd.perm, n, nrhs);
    tm.mark(STAGE_PERMUTE_OUT, 1, st);
    return cudaGetLastError();
}

cudaError_t ifgf_cache_target_geometry(const PlanDev &pd, int d, float4 *loc, float2 *fac, int64_t m, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    ifgf::batched::k_cache_target_geometry<<<(int)((m + 255) / 256), 256, 0, st>>>(pd, d, loc, fac, m);
    return cudaGetLastError();
}
