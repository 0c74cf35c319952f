// Float-float block stencil, derivative mode 2 (a link direction: the hops with the links
// Y = dU/dt): the instantiations of k_hop (lq_kernels.cuh) for lq::ff, schedule 0.
#include "lq_kernels.cuh"

namespace lq {

cudaError_t launch_hop_ff2(const HopArgs& a, bool dot, cudaStream_t st) {
    const dim3 grid((unsigned)((a.V + kHopThreads - 1) / kHopThreads), (unsigned)a.nsides, (unsigned)a.nsrc);
    if (dot) k_hop<ff, 2, 2, true, 1><<<grid, kHopThreads, 0, st>>>(a);
    else k_hop<ff, 2, 2, false, 1><<<grid, kHopThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// schedules 1 / 2: one thread per (site, output field), the four outputs of 32 sites in a block,
// at least 3 / 4 resident blocks per SM (170 / 128 registers)
cudaError_t launch_roles_ff2(const HopArgs& a, bool dot, cudaStream_t st) {
    const dim3 grid((unsigned)((a.V + kRoleSites - 1) / kRoleSites), (unsigned)a.nsrc, 1);
    if (a.variant == 2) {
        if (dot) k_hop_roles<ff, 2, true, kRoleSites, 4><<<grid, 4 * kRoleSites, 0, st>>>(a);
        else k_hop_roles<ff, 2, false, kRoleSites, 4><<<grid, 4 * kRoleSites, 0, st>>>(a);
    } else {
        if (dot) k_hop_roles<ff, 2, true, kRoleSites, 3><<<grid, 4 * kRoleSites, 0, st>>>(a);
        else k_hop_roles<ff, 2, false, kRoleSites, 3><<<grid, 4 * kRoleSites, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lq
