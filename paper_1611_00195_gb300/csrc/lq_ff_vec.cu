// Float-float instantiations of the vector kernels (lq_kernels.cuh): the update step of the
// recurrences, start vectors, recombination, layout conversions of spinors and links, and the
// derivative direction dU/dt.
#include "lq_kernels.cuh"

namespace lq {

cudaError_t launch_update_ff(const UpdArgs& a, dim3 grid, cudaStream_t st) {
    k_update<ff><<<grid, kUpdThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tsl_init_ff(int nf, const InitArgs& a, dim3 grid, cudaStream_t st) {
    if (nf == 1) k_tsl_init<ff, 1><<<grid, kUpdThreads, 0, st>>>(a);
    else k_tsl_init<ff, 2><<<grid, kUpdThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_recombine_ff(int nf, const RecArgs& a, dim3 grid, size_t smem, cudaStream_t st) {
    if (nf == 1) {
        cudaFuncSetAttribute(k_recombine<ff, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_recombine<ff, 1><<<grid, kRecThreads, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_recombine<ff, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_recombine<ff, 2><<<grid, kRecThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_internal_ff(const double* x, void* f, size_t V, int nfields, dim3 grid, cudaStream_t st) {
    k_to_internal<ff><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<float4*>(f), V, nfields);
    return cudaGetLastError();
}

cudaError_t launch_to_boundary_ff(const void* f, double* x, size_t V, int nfields, dim3 grid, cudaStream_t st) {
    k_to_boundary<ff><<<grid, 128, 0, st>>>(reinterpret_cast<const float4*>(f), reinterpret_cast<double2*>(x), V, nfields);
    return cudaGetLastError();
}

cudaError_t launch_links_internal_ff(const double* U, void* L, size_t V, dim3 grid, cudaStream_t st) {
    k_links_internal<ff><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), reinterpret_cast<cff*>(L), V);
    return cudaGetLastError();
}

cudaError_t launch_direction_ff(const double* U, const double* w, int kind, void* Y, size_t V, dim3 grid, cudaStream_t st) {
    k_direction<ff><<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(U), w, kind, reinterpret_cast<cff*>(Y), V);
    return cudaGetLastError();
}

}  // namespace lq
