// FP64 instantiation of the evaluation kernels (IFGF_FP64 plans).
#include "ifgf_apply_impl.cuh"

cudaError_t ifgf_run_typed_f64(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm)
{
    return ifgf::run_typed<double>(pd, nrhs, in_user, out_user, in_sorted, out_sorted, mode, adjoint, st, tm);
}

cudaError_t ifgf_build_uptable_f64(const PlanDev &pd, int d, void *tab, cudaStream_t st)
{
    return ifgf::build_uptable<double>(pd, d, tab, st);
}

size_t ifgf_uptable_entry_bytes(int precision, int Ps, int Pang)
{
    bool big = (Ps == 4 && Pang == 7);
    if (precision == IFGF_FP64) return big ? sizeof(UpEntry<double, 18>) : sizeof(UpEntry<double, 13>);
    return sizeof(UpEntry32);
}

cudaError_t ifgf_build_evalcache_f64(const PlanDev &pd, int d, int which, cudaStream_t st)
{
    return ifgf::build_evalcache<double>(pd, d, which, st);
}

ifgf_status ifgf_run_adjoint_jit_f64(ifgf_plan *p, int nrhs, const void *in, void *out, int mode, cudaStream_t st)
{
    return ifgf::run_adjoint_jit<double>(p, nrhs, in, out, mode, st);
}
