/*
 * ifgf.h - C ABI of the GB300 (sm_103a) IFGF library.
 *
 * The library evaluates the discrete Helmholtz single-layer operator of
 * Bauinger & Bruno, "Interpolated Factored Green Function method for accelerated
 * solution of scattering problems" (arXiv 2010.02857), Eq. (field1) with the
 * kernel of Eq. (greensfunction):
 *
 *     u_r(x_l) = sum_{m != l} sigma_r(x_m) exp(i kappa |x_l - x_m|) / (4 pi |x_l - x_m|),
 *
 * for l = 1..N and right-hand sides r = 0..nrhs-1, by the IFGF method of
 * Algorithm 1 (Sec. 3.3.3): a box octree of D levels (Sec. 3.3.1), per-box cone
 * segments in the (s, theta, phi) variables of Eq. (defparametrizationins), and
 * Chebyshev interpolation of the analytic factor of Eq. (factored_f) with
 * P = P_s * P_ang^2 points per cone (Eq. interp_pts).
 *
 * Conventions for every entry point:
 *   - Every call returns an ifgf_status; none aborts, traps or exits.
 *   - Complex data are interleaved (re, im) pairs.  FP64 plans take complex128
 *     (double pairs); all other precisions take complex64 (float pairs).
 *   - Densities and fields are row-major [nrhs][N] in the caller's point order.
 *   - Array arguments may be host or device pointers unless stated otherwise;
 *     the library detects which with cudaPointerGetAttributes.  With device
 *     pointers the call is asynchronous on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream).  With host pointers the call copies through
 *     plan-owned device buffers and returns after the result is on the host.
 *   - The caller owns every array it passes; the plan copies what it needs
 *     (the points) and keeps no caller pointer after a call returns.
 *   - A plan is not thread-safe: calls on one plan must be serialised by the
 *     caller (the plan owns the intermediate cone-value buffers).
 */
#ifndef IFGF_H
#define IFGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifgf_plan ifgf_plan;

typedef enum {
    IFGF_OK = 0,
    IFGF_EINVAL = 1,    /* invalid argument (sizes, levels, non-finite points, nrhs) */
    IFGF_ENOMEM = 2,    /* device or host allocation failed */
    IFGF_ECUDA = 3,     /* a CUDA runtime call failed; see ifgf_last_error */
    IFGF_ETIMEOUT = 4,  /* a host-side wait exceeded its limit */
    IFGF_EINTERNAL = 5  /* an internal invariant failed (e.g. a cone lookup missed) */
} ifgf_status;

typedef enum {
    /* all arithmetic in FP64; complex128 data */
    IFGF_FP64 = 0,
    /* FP64 for point differences, distances, spherical coordinates and phase
     * arguments; FP32 interpolation, accumulation and reduced-phase sincos;
     * complex64 data */
    IFGF_MIXED = 1,
    /* IFGF_MIXED with the per-cone interpolation contraction on tensor cores
     * (tcgen05, BF16 hi+lo operand split, FP32 accumulate), grouped by source cone;
     * for many right-hand sides.  Used by ifgf_apply for even nrhs up to 64 at
     * (P_s, P_ang) = (3, 5) (contraction length 80) and up to 48 at (4, 7) (length 208,
     * one CTA per SM); other nrhs and the adjoint run the IFGF_MIXED kernels.
     * Contributions are added to their destinations with FP32 atomic reductions, so the
     * last bits of the result vary from run to run. */
    IFGF_BATCHED_BF16 = 2,
    /* IFGF_BATCHED_BF16 with FP16 operands: the hi + lo split keeps ~22 significant bits
     * (~16 for BF16); each cone's values are scaled by a power of two into [-1, 1] before
     * the split (FP16's exponent range is narrow) and the rows of the cone carry the
     * inverse power. */
    IFGF_BATCHED_FP16 = 3
} ifgf_precision;

typedef struct {
    int leaf_ns;    /* n_{s,D}: radial cone intervals at the leaf level; 0 = default */
    int leaf_nc;    /* n_{C,D}: polar intervals at the leaf level (2 n_C azimuthal); 0 = default */
    int max_nrhs;   /* largest nrhs a later apply may use; 0 = 1 */
    int precision;  /* an ifgf_precision */
    int flags;      /* bit 0: build the adjoint's transpose lists at plan time;
                       bit 1: no upward tables (compute the upward geometry per
                       evaluation; by default a level whose geometry table is at most
                       half its evaluation count gets one);
                       bit 2: IFGF_BATCHED_BF16 plans do not cache the cousin
                       targets' local coordinates and centred factors at plan time
                       (24 bytes per cousin evaluation; cached by default);
                       bit 3: keep only two levels' cone values (always on when the
                       values of all levels exceed the budget below);
                       bit 4: process at most 2 right-hand sides per pass (testing);
                       bit 5: no evaluation caches.  By default, when they take at most a
                       quarter of the free device memory, FP64 and IFGF_MIXED plans
                       store at plan time each cousin-target evaluation's cone slot,
                       weights (local coordinates for IFGF_MIXED) and centred factor,
                       and the geometry of every upward evaluation of levels without an
                       upward table; the evaluations, forward and adjoint, then skip
                       that geometry (the adjoint's transpose lists then also hold each
                       cousin-target entry's cache index, 4 bytes per evaluation);
                       bit 6: adjoints of two-level plans build their upward transpose
                       lists in ranges of at most 4096 evaluations (testing; the
                       default range is 2^28).  Two-level plans build the adjoint's
                       transpose lists level by level right before use, unless bit 0
                       built them at plan time;
                       bit 7: host-side waits never see the device finish, so they
                       end with IFGF_ETIMEOUT (testing; the limit is timeout_s, or
                       0.05 s when that is 0);
                       bit 8: the tensor-core cone kernel of IFGF_BATCHED_BF16 plans
                       issues no MMA, so its bounded waits for them run out (after a
                       shortened limit) and the device error counter records it
                       (testing; see ifgf_plan_check);
                       bit 9: FP32 upward steps run one thread per parent node, reading
                       the child cone values from L1, instead of one warp per parent cone
                       in runs of nodes that share a child cone (testing: the two kernels
                       sum in the same order);
                       bit 10: the run kernel's runs are taken by 8 lanes instead of 32
                       (testing: every lane then takes several runs of a child step);
                       bit 11: FP32 upward steps whose geometry is computed on the fly use
                       the run kernel too (by default they use one node per lane, which
                       keeps the FP64 geometry work dense; testing and measurement);
                       bit 12: plan creation marks the cones of relevance rule (ii) node by
                       node for every parent slot, instead of once per distinct parent cone
                       id and child octant (testing: both mark the same cones). */
    long long value_budget_bytes; /* device bytes for cone values; 0 = 85% of the free
                       memory at plan time less the sorted density and field buffers and
                       a reserve of min(24 GB, a tenth of the device) for the adjoint's
                       transpose lists and workspace.  When the values of every level for
                       max_nrhs right-hand sides exceed it, the plan keeps two levels
                       (d and d-1) and applies right-hand sides in chunks that fit; the
                       per-level values returned by ifgf_plan_get_values are then those
                       of the last two levels written */
    double timeout_s;   /* limit of the host-side waits of an evaluation (calls with host
                       buffers wait for their result; profiling waits for its events):
                       past it the call returns IFGF_ETIMEOUT and the queued work
                       completes on its own; 0 = no limit */
    int leaf_max;       /* 0: the uniform octree of `levels` levels (Sec. 3.3.1).  > 0: an
                       adaptive octree, which Sec. 4 names as an improvement: a box of
                       level >= 3 with at most leaf_max points is not subdivided (a leaf),
                       boxes of level `levels` are leaves.  A leaf's points take the
                       analytic factors of its cones directly; the direct sums of a target
                       cover the points of its leaf's neighbours and the leaf neighbours of
                       its leaf's ancestors (every pair is covered once).  IFGF_FP64 and
                       IFGF_MIXED plans only. */
} ifgf_options;

/*
 * Build a plan: the octree, cousin lists and relevant cone segments of every level
 * (Sec. 3.3.1, Eq. defcousinboxes and defallrelevantconesegments; the
 * pre-computation stage of Algorithm 1), on the GPU.
 *   points    [N][3] double, x y z per point, host or device; pairwise distinct.
 *   n         N >= 2 (and < 2^31).
 *   kappa     wavenumber >= 0 (kappa = 0 gives the Laplace kernel 1/(4 pi r)).
 *   levels    D >= 3, <= 20: the number of octree levels, root = level 1 (Sec. 3.3.1).
 *   p_radial  P_s  >= 1, <= 8: Chebyshev points per cone along s.
 *   p_angular P_ang >= 1, <= 8: Chebyshev points per cone along theta and along phi.
 *   opt       NULL for defaults.  Default leaf cones: (n_s, n_C) = (1, 2) for leaf boxes
 *             up to a quarter wavelength, doubled per doubling of the leaf size
 *             (Sec. 4 uses (1, 2) at H_D ~ lambda / 4).
 *   stream    cudaStream_t used for the build; the call synchronises it before return.
 *   out       receives the plan (NULL on failure).
 * Errors: IFGF_EINVAL for bad arguments (including coinciding points), IFGF_ENOMEM,
 * IFGF_ECUDA.
 */
ifgf_status ifgf_plan_create(const double *points, int64_t n, double kappa, int levels,
                             int p_radial, int p_angular, const ifgf_options *opt,
                             void *stream, ifgf_plan **out);

/*
 * u = A sigma: the IFGF evaluation stage of Algorithm 1 (level-D direct sums over
 * neighbouring boxes, analytic factors at the leaf cones' interpolation points,
 * and for d = D..3 interpolation to cousin targets and, for d > 3, to the parent
 * cones' interpolation points with re-centring).
 *   sigma  [nrhs][N] complex (complex128 for IFGF_FP64 plans, complex64 otherwise).
 *   u      [nrhs][N] complex output, same type; overwritten.
 *   nrhs   1 <= nrhs <= max_nrhs of the plan.
 * Errors: IFGF_EINVAL (nrhs, NULL), IFGF_ECUDA.
 */
ifgf_status ifgf_apply(ifgf_plan *plan, const void *sigma, void *u, int nrhs, void *stream);

/*
 * w = A^H v: the exact conjugate transpose of the operator that ifgf_apply
 * computes (every linear step of Algorithm 1 transposed and conjugated, run from
 * targets to cone nodes to sources).  The paper has no adjoint; this is the
 * linear algebra of the same steps.  Arguments as for ifgf_apply.
 */
ifgf_status ifgf_apply_adjoint(ifgf_plan *plan, const void *v, void *w, int nrhs, void *stream);

/*
 * Partial evaluation for stage-wise checks: mode bit 0 = level-D direct
 * neighbour sums only, bit 1 = interpolated (far) contributions only, 3 = both
 * (= ifgf_apply).  `adjoint` != 0 selects the adjoint.
 */
ifgf_status ifgf_apply_partial(ifgf_plan *plan, const void *in, void *out, int nrhs, int mode,
                               int adjoint, void *stream);

/*
 * u = A sigma like ifgf_apply, but allocating nothing.  The paper has no
 * counterpart; this entry point exists for callers that may not allocate device
 * memory during an evaluation (their memory belongs to a framework pool or a fixed
 * budget, or they cannot afford an allocation's implicit synchronisation): it calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   - All scratch of the evaluation (densities and fields in Morton order, the cone
 *     values of every level) comes from one fixed device array of 64 MiB,
 *     2 N nrhs + sum_d A_d P nrhs complex elements (each part rounded up to 256
 *     bytes); a plan whose evaluation needs more is rejected with IFGF_EINVAL.
 *     The array is a static device variable of the library: every GPU that loads
 *     the library holds it until the process exits.
 *   - sigma and u must be device pointers of the plan's device ([nrhs][N] complex,
 *     as for ifgf_apply), and the plan's device must be current.
 *   - The evaluation runs on the CUDA-core kernels of the plan's data type, all nrhs
 *     in one pass: IFGF_BATCHED_BF16 plans are evaluated by the IFGF_MIXED kernels
 *     (FP32 contraction, not the tensor cores), so their result differs from
 *     ifgf_apply's by the BF16 operand rounding.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress).  The first call on a device may load the library's
 *     device code there; make that first call before any stream capture.
 *   - Every call shares the array and it keeps the last call's contents; each call
 *     overwrites all of the scratch it reads, so nothing is cleared.  Calls whose
 *     work overlaps on the GPU (different streams, or different threads) race on
 *     the array and give wrong results: serialise them.
 * Errors: IFGF_EINVAL (sizes, host pointers or another device's pointers, another
 * device current, scratch limit), IFGF_ECUDA.
 */
ifgf_status ifgf_apply_noalloc(ifgf_plan *plan, const void *sigma, void *u, int nrhs, void *stream);

/* Release every device and host resource of the plan.  NULL is accepted. */
ifgf_status ifgf_plan_destroy(ifgf_plan *plan);

/* ---------------------------------------------------------------------------
 * Introspection (host outputs; the call synchronises the plan's work first).
 * ------------------------------------------------------------------------- */

/*
 * Per-level counts of level d (1..D), written to info[0..7]:
 * nbox, neighbour entries, cousin entries, relevant cones, n_s, n_C,
 * cousin evaluations per apply, upward evaluations per apply.
 */
ifgf_status ifgf_plan_level_info(const ifgf_plan *plan, int level, int64_t *info);

/* perm[i] = caller index of the i-th point in Morton order ([N] int64, host). */
ifgf_status ifgf_plan_get_perm(const ifgf_plan *plan, int64_t *perm);

/* Relevant boxes of level d: keys[nbox] (Morton key of the integer box
 * coordinate) and start[nbox+1] (ranges into the Morton-ordered points). */
ifgf_status ifgf_plan_get_boxes(const ifgf_plan *plan, int level, uint64_t *keys, int64_t *start);

/* Point ranges and leaves of level d: end[nbox] (box b holds the sorted points
 * start[b] .. end[b]-1, start from ifgf_plan_get_boxes) and leaf[nbox] (1: the box is
 * not subdivided).  In a uniform tree end[b] = start[b+1] and the leaves are the boxes
 * of level D. */
ifgf_status ifgf_plan_get_box_ends(const ifgf_plan *plan, int level, int64_t *end, int64_t *leaf);

/* Level of every point's leaf box, levels[N] in Morton order (all D in a uniform tree). */
ifgf_status ifgf_plan_get_point_levels(const ifgf_plan *plan, int64_t *levels);

/* Near-field point ranges of the leaf boxes of level d >= 3: *count receives their number;
 * with start != NULL also start[nbox+1] (CSR over the boxes) and the ranges
 * [lo[e], hi[e]) of sorted points, ascending per box. */
ifgf_status ifgf_plan_get_near(const ifgf_plan *plan, int level, int64_t *count, int64_t *start, int64_t *lo,
                               int64_t *hi);

/* Cousin lists of level d >= 3 (Eq. defcousinboxes) in CSR form. */
ifgf_status ifgf_plan_get_cousins(const ifgf_plan *plan, int level, int64_t *start, int64_t *list);

/* Relevant cones of level d >= 3 (Eq. defallrelevantconesegments) in CSR form:
 * start[nbox+1], cones[nact] = linear cone id (g1 n_C + g2) 2 n_C + g3. */
ifgf_status ifgf_plan_get_active(const ifgf_plan *plan, int level, int64_t *start, int64_t *cones);

/* Cone values F_k^d at the interpolation points of level d after the last apply:
 * [nact][P][nrhs] complex of the plan's data type (host). */
ifgf_status ifgf_plan_get_values(const ifgf_plan *plan, int level, void *out);

/*
 * Cone cells (Eq. defconedomain, defconedomainproduct) of the vectors v[n][3]
 * (host; a vector is a point minus a box centre) at level d >= 3, by the two
 * device paths the library uses: exact[i] from correctly rounded FP64 operations
 * (plan construction) and fast[i] from the evaluation path of the plan's precision
 * (FP64 plans: Newton-refined FP64 estimates; other plans: FP64 radius and FP32 angle
 * decisions with a margin), each with a correctly rounded fallback near cell
 * boundaries.  Both are linear cone ids
 * (g1 n_C + g2) 2 n_C + g3 and must be equal; for tests.
 */
ifgf_status ifgf_plan_cone_ids(const ifgf_plan *plan, int level, int64_t n, const double *v,
                               int32_t *exact, int32_t *fast);

/* Root cube: geom[0] = H_1, geom[1..3] = lower corner. */
ifgf_status ifgf_plan_geometry(const ifgf_plan *plan, double *geom);

/* JSON statistics into buf[cap] (IFGF_EINVAL when cap is too small): sizes, near pairs,
 * leaf evaluations, build time, device bytes, the two-buffer and chunking choices, cache
 * bytes, the captured CUDA graphs ("graphs", "graph_captures", "graph_replays"), the
 * batched tile shapes ("tune_leaf", "tune_cone_ctas"), and per level the box, cousin and
 * relevant-cone counts, cone intervals, and cousin and upward evaluation counts. */
ifgf_status ifgf_plan_stats(const ifgf_plan *plan, char *buf, size_t cap);

/* Status of the device-side invariant checks of all calls since the last query
 * (0 = none failed); synchronises the plan's stream and clears the flag. */
ifgf_status ifgf_plan_check(ifgf_plan *plan, int *device_errors);

/*
 * Per-stage timing.  With profiling on, every apply records CUDA events on its
 * stream between stages and waits for them before returning, adding the elapsed
 * times per stage.  Turning it on or off clears the totals.
 */
ifgf_status ifgf_plan_set_profiling(ifgf_plan *plan, int on);

/*
 * Autotuner of the batched tensor-core path (IFGF_BATCHED_BF16 and IFGF_BATCHED_FP16
 * plans).  On this plan's relevant cones with nrhs right-hand sides (even, 2..the order's
 * maximum (64 at (3, 5), 48 at (4, 7)) and max_nrhs) it times:
 *   - each register-tile shape of the leaf analytic-factor kernel, written as threads
 *     along the right-hand sides x thread groups along the 75 nodes of a cone:
 *     0 = 16 x 8 (the default), 1 = 32 x 4, 2 = 8 x 16 (order (4, 7) plans run one leaf
 *     kernel, so the three times are of the same kernel);
 *   - each grid of the persistent tensor-core cone kernel: 1 or 2 CTAs per SM (2 is
 *     the default; order (4, 7) fits one);
 * reps runs of each after one warm-up run, and keeps the fastest of each for the
 * plan's later evaluations.  ms (NULL or [5]) receives the candidates' mean times in
 * milliseconds in the order above (the 3 leaf shapes, then 1 and 2 CTAs per SM);
 * choice (NULL or [2]) receives {leaf shape, CTAs per SM}.  The shapes change how the
 * work is split, not the result (the cone kernel's reductions vary in order from run to
 * run whatever the shape).  The runs use the plan's own buffers (densities zeroed),
 * never the caller's; captured CUDA graphs of the plan are dropped.  Synchronises the
 * stream.  Errors: IFGF_EINVAL for another precision, an odd or out-of-range nrhs or
 * reps < 1; IFGF_ECUDA for a failed launch.
 */
ifgf_status ifgf_plan_autotune(ifgf_plan *plan, int nrhs, int reps, double *ms, int *choice, void *stream);

/*
 * Sets the batched path's tile shapes directly (for instance to reuse what
 * ifgf_plan_autotune chose for an earlier plan of the same geometry): leaf_shape in
 * 0..2 as listed above, cone_ctas_per_sm 1 or 2.  Drops the plan's captured CUDA
 * graphs.  Plans of other precisions keep the setting and ignore it.  Errors:
 * IFGF_EINVAL for values out of range.
 */
ifgf_status ifgf_plan_set_tiles(ifgf_plan *plan, int leaf_shape, int cone_ctas_per_sm);

/*
 * Persistent tune cache.  The shapes ifgf_plan_autotune chooses depend on the device and
 * on the workload's sizes, not on the densities, so they can be kept in a text file and
 * reused by later plans and processes.  The file holds one line per workload,
 *     <key> <leaf_shape> <cone_ctas_per_sm>
 * with the values of ifgf_plan_set_tiles; lines are appended whole, the last valid line
 * for a key wins and malformed or out-of-range lines are skipped (so the file may be
 * shared by processes and edited by hand).  Host code only: no device work.
 *
 * ifgf_plan_tune_key writes the plan's key for nrhs right-hand sides into buf (cap
 * bytes, at most 481 used): the device's name, SM count and compute capability, the
 * precision, (P_s, P_ang), nrhs, N, the depth, the leaf factor count and the rows of the
 * cone contraction (cousin plus upward evaluations), as one token without whitespace.
 * Errors: IFGF_EINVAL (cap too small), IFGF_ECUDA (device query failed).
 *
 * ifgf_tune_cache_lookup sets *found to 1 and choice[2] to {leaf_shape,
 * cone_ctas_per_sm} when path holds a valid line for key, else *found = 0 (also when the
 * file does not exist).  Errors: IFGF_EINVAL for a NULL argument or a key that is empty,
 * longer than 480 bytes or contains whitespace.
 *
 * ifgf_tune_cache_store appends the line for key and choice[2] to path (creating it).
 * Errors: IFGF_EINVAL for a bad key, values out of range, or a file that cannot be
 * written.
 *
 * ifgf_plan_autotune_cached looks the plan's key up in path: on a hit it sets the cached
 * shapes (ifgf_plan_set_tiles) and sets *hit = 1 without any device work; otherwise it
 * runs ifgf_plan_autotune(plan, nrhs, reps, ...) and appends the choice.  choice (NULL or
 * [2]) receives the shapes in use.  Errors: those of ifgf_plan_autotune (checked on a hit
 * too), and IFGF_EINVAL when the file cannot be written.
 */
ifgf_status ifgf_plan_tune_key(const ifgf_plan *plan, int nrhs, char *buf, int cap);
ifgf_status ifgf_tune_cache_lookup(const char *path, const char *key, int *found, int *choice);
ifgf_status ifgf_tune_cache_store(const char *path, const char *key, const int *choice);
ifgf_status ifgf_plan_autotune_cached(ifgf_plan *plan, int nrhs, int reps, const char *path, int *choice, int *hit,
                                      void *stream);

/*
 * CUDA-graph replay of evaluations.  With on != 0, the launches of an evaluation
 * (ifgf_apply, ifgf_apply_adjoint, ifgf_apply_partial) are captured into a CUDA graph
 * the first time the plan evaluates with a given input buffer, output buffer, nrhs,
 * mode and direction, and that graph is replayed on the caller's stream by later such
 * calls (host-pointer calls use the plan's own device staging buffers, so they share
 * one graph per nrhs, mode and direction).  A replay runs the same kernels in the same
 * order as the plain launches, so the results are the same.  The graph keeps the
 * buffer addresses, not their contents.  At most 8 graphs are kept (the least recently
 * used is dropped); on = 0 frees them.  With profiling on (ifgf_plan_set_profiling),
 * separate graphs are captured that record the stage events themselves, so per-stage
 * times stay available.  Graphs are not used for the adjoint of two-buffer plans, whose
 * transpose lists are built between launches.  Off by default.  Errors: IFGF_EINVAL
 * for a NULL plan; a capture that fails makes the evaluation return IFGF_ECUDA.
 */
ifgf_status ifgf_plan_set_graphs(ifgf_plan *plan, int on);

/*
 * Totals since profiling was turned on: ms[s] milliseconds and launches[s] kernel
 * launches of stage s, calls = profiled calls; count >= 8.  Stages: 0 density
 * permutation, 1 leaf analytic factors, 2 upward interpolation (all levels),
 * 3 target evaluation (near + cousin interpolation), 4 output permutation,
 * 5 adjoint cone levels, 6 adjoint source evaluation (and the conjugated near field),
 * 7 transpose lists that the adjoint of a two-buffer plan builds between its launches
 * (launch count 0: their sorts are library kernels).
 */
ifgf_status ifgf_plan_timings(const ifgf_plan *plan, double *ms, int64_t *launches, int64_t *calls,
                              int count);

/*
 * Roofline probe (not part of the paper's method): the device's sustained fused
 * multiply-add rate, *tflops in TFLOP/s (2 flops per FMA), for which = 0 (FP64) or
 * which = 1 (FP32), measured on the current device by a kernel of independent FMA
 * chains with no memory traffic (best of 5 timed runs after a warm-up, CUDA events on
 * `stream`; synchronises it).  The FP64 and mixed evaluation kernels are bound by these
 * pipes, so their roofline fractions divide by these rates.
 * Errors: IFGF_EINVAL (which, NULL), IFGF_ECUDA.
 */
ifgf_status ifgf_device_peak(int which, double *tflops, void *stream);

/* Message of the last failed call on this plan (or of the last failed
 * ifgf_plan_create when plan is NULL).  Never NULL. */
const char *ifgf_last_error(const ifgf_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* IFGF_H */
