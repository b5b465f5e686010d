// ifgf_apply_noalloc: u = A sigma with every scratch buffer taken from a fixed,
// file-scope device array instead of device memory the library allocates.
//
// Who needs it: callers whose device memory is owned by someone else and who may
// not call cudaMalloc/cudaFree themselves or let a library do so during the
// evaluation - for example code that runs under a framework's memory pool or a
// hard device-memory budget, or a latency-bound loop that cannot afford the
// implicit synchronisation of an allocation.  They build the plan once (which does
// allocate the tree and relevant-cone tables) and afterwards evaluate with this
// entry point, which calls no allocating routine.
//
// The scratch of one evaluation is: the densities and fields in Morton order
// (2 x N x nrhs complex) and the cone values of every level (sum_d A_d x P x nrhs
// complex), each rounded up to 256 bytes.  It must fit in
// IFGF_NOALLOC_SCRATCH_BYTES (64 MiB); larger requests are rejected.
//
// Every plan is evaluated by the CUDA-core kernels of its data type in one pass over all
// nrhs right-hand sides, with every level's cone values resident: FP64 plans by the FP64
// kernels, IFGF_MIXED and IFGF_BATCHED_BF16 plans by the mixed-precision kernels (the
// tensor-core path needs buffers this entry point does not have).  A batched plan thus
// gives the mixed path's result here, which differs from ifgf_apply's tensor-core result
// by the BF16 operand rounding; plans with two level buffers or right-hand-side chunks
// give the same operator as ifgf_apply.
#include <string>

#include "ifgf_internal.h"

cudaError_t ifgf_run_typed_f64(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm);
cudaError_t ifgf_run_typed_f32(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm);

#define IFGF_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

// One array per device that loads the library, held until the process exits.  Every
// call shares it: it keeps the previous call's contents, and calls whose work
// overlaps on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IFGF_NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device memory.  Every
// call looks up the array's device address for the current device (cudaGetSymbolAddress,
// cheap once the library's device code is loaded) instead of caching it: after a
// cudaDeviceReset or a new primary context the array may live at another address.
static cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// A device (or managed) pointer of the given device.
static bool on_device(const void *ptr, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" ifgf_status ifgf_apply_noalloc(ifgf_plan *plan, const void *sigma, void *u, int nrhs, void *stream)
{
    if (!plan || !sigma || !u) return IFGF_EINVAL;
    if (nrhs < 1 || nrhs > plan->max_nrhs) {
        plan->last_error = "nrhs must be in [1, max_nrhs]";
        return IFGF_EINVAL;
    }
    int cur_dev = -1;
    if (cudaGetDevice(&cur_dev) != cudaSuccess || cur_dev != plan->device) {
        cudaGetLastError();
        plan->last_error = "ifgf_apply_noalloc: make the plan's device current";
        return IFGF_EINVAL;
    }
    if (!on_device(sigma, plan->device) || !on_device(u, plan->device)) {
        plan->last_error = "ifgf_apply_noalloc takes device pointers of the plan's device only";
        return IFGF_EINVAL;
    }
    const size_t eb = ifgf_elem_bytes(plan->precision);
    const size_t vec = round256((size_t)plan->n * nrhs * eb);
    size_t need = 2 * vec;
    for (int d = 3; d <= plan->D; ++d) need += round256((size_t)plan->dev.lev[d].nact * plan->P * nrhs * eb);
    if (need > IFGF_NOALLOC_SCRATCH_BYTES) {
        plan->last_error = "ifgf_apply_noalloc: this plan needs " + std::to_string(need) +
                           " bytes of scratch, more than the fixed " +
                           std::to_string((size_t)IFGF_NOALLOC_SCRATCH_BYTES) + " bytes";
        return IFGF_EINVAL;
    }
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        plan->last_error = std::string("scratch address lookup failed: ") + cudaGetErrorString(e);
        return IFGF_ECUDA;
    }
    // Carve the scratch.  Every kernel below overwrites the whole region it uses
    // (sorted densities, every relevant cone value of every level, every sorted
    // field), so nothing needs clearing between calls.
    unsigned char *cur = (unsigned char *)base;
    void *sig_sorted = cur;
    cur += vec;
    void *u_sorted = cur;
    cur += vec;
    PlanDev pd = plan->dev;
    for (int d = 3; d <= plan->D; ++d) {
        pd.lev[d].F = cur;
        cur += round256((size_t)plan->dev.lev[d].nact * plan->P * nrhs * eb);
    }
    StageTimer off;
    cudaStream_t st = (cudaStream_t)stream;
    e = plan->precision == IFGF_FP64
            ? ifgf_run_typed_f64(pd, nrhs, sigma, u, sig_sorted, u_sorted, 3, 0, st, off)
            : ifgf_run_typed_f32(pd, nrhs, sigma, u, sig_sorted, u_sorted, 3, 0, st, off);
    if (e != cudaSuccess) {
        plan->last_error = std::string("kernel launch failed: ") + cudaGetErrorString(e);
        return IFGF_ECUDA;
    }
    return IFGF_OK;
}
