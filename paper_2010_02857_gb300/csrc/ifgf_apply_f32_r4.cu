// Mixed-precision kernels blocked for up to 4 right-hand sides per thread (IFGF_MIXED
// plans called with 2..4 right-hand sides, or with chunks of at most 4).  A separate
// translation unit so that the build compiles it in parallel with the others.
#include "ifgf_apply_impl.cuh"

void ifgf_upward_runs_blocks(const PlanDev &pd, int d, int nrhs, cudaStream_t st)
{
    using namespace ifgf;
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
        const int nb = nrhs - r0 < 4 ? nrhs - r0 : 4;
        if (pd.Ps == 3 && pd.Pang == 5) launch_runs<4, 3, 5>(pd, d, nrhs, r0, nb, st);
        else if (pd.Ps == 4 && pd.Pang == 7) launch_runs<4, 4, 7>(pd, d, nrhs, r0, nb, st);
    }
}

cudaError_t ifgf_prepare_runs_r4()
{
    cudaError_t e = ifgf::set_run_smem_limit<4, 3, 5>();
    return e == cudaSuccess ? ifgf::set_run_smem_limit<4, 4, 7>() : e;
}

cudaError_t ifgf_launch_f32_r4(const PlanDev &pd, int nrhs, const void *in, void *out, int mode, int adjoint,
                               cudaStream_t st, StageTimer &tm)
{
    using namespace ifgf;
    if (pd.Ps == 3 && pd.Pang == 5)
        return adjoint ? launch_adjoint<float, 4, 3, 5>(pd, nrhs, in, out, mode, st, tm)
                       : launch_forward<float, 4, 3, 5>(pd, nrhs, in, out, mode, st, tm);
    if (pd.Ps == 4 && pd.Pang == 7)
        return adjoint ? launch_adjoint<float, 4, 4, 7>(pd, nrhs, in, out, mode, st, tm)
                       : launch_forward<float, 4, 4, 7>(pd, nrhs, in, out, mode, st, tm);
    return cudaErrorInvalidValue;
}
