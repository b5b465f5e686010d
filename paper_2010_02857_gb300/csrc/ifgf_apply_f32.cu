// Mixed-precision instantiation of the evaluation kernels (IFGF_MIXED plans): FP64
// geometry and phase arguments, FP32 values, interpolation and accumulation.
#include "ifgf_apply_impl.cuh"

cudaError_t ifgf_run_typed_f32(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm)
{
    return ifgf::run_typed<float>(pd, nrhs, in_user, out_user, in_sorted, out_sorted, mode, adjoint, st, tm);
}

cudaError_t ifgf_prepare_runs_r1()
{
    cudaError_t e = ifgf::set_run_smem_limit<1, 3, 5>();
    return e == cudaSuccess ? ifgf::set_run_smem_limit<1, 4, 7>() : e;
}

cudaError_t ifgf_build_uptable_f32(const PlanDev &pd, int d, void *tab, cudaStream_t st)
{
    return ifgf::build_uptable<float>(pd, d, tab, st);
}

cudaError_t ifgf_build_evalcache_f32(const PlanDev &pd, int d, int which, cudaStream_t st)
{
    return ifgf::build_evalcache<float>(pd, d, which, st);
}

ifgf_status ifgf_run_adjoint_jit_f32(ifgf_plan *p, int nrhs, const void *in, void *out, int mode, cudaStream_t st)
{
    return ifgf::run_adjoint_jit<float>(p, nrhs, in, out, mode, st);
}
