// Float-float block stencil, derivative mode 0 (no derivative term; also the plain operator,
// one field per side): the instantiations of k_hop (lq_kernels.cuh) for lq::ff, schedule 0.
#include "lq_kernels.cuh"

namespace lq {

cudaError_t launch_hop_ff0(const HopArgs& a, int nf, bool dot, cudaStream_t st) {
    const dim3 grid((unsigned)((a.V + kHopThreads - 1) / kHopThreads), (unsigned)a.nsides, (unsigned)a.nsrc);
    if (nf == 1) {
        if (dot) k_hop<ff, 1, 0, true, 1><<<grid, kHopThreads, 0, st>>>(a);
        else k_hop<ff, 1, 0, false, 1><<<grid, kHopThreads, 0, st>>>(a);
    } else {
        if (dot) k_hop<ff, 2, 0, true, 1><<<grid, kHopThreads, 0, st>>>(a);
        else k_hop<ff, 2, 0, false, 1><<<grid, kHopThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// schedules 1 / 2: one thread per (site, output field), the four outputs of 32 sites in a block,
// at least 3 / 4 resident blocks per SM (170 / 128 registers)
cudaError_t launch_roles_ff0(const HopArgs& a, bool dot, cudaStream_t st) {
    const dim3 grid((unsigned)((a.V + kRoleSites - 1) / kRoleSites), (unsigned)a.nsrc, 1);
    if (a.variant == 2) {
        if (dot) k_hop_roles<ff, 0, true, kRoleSites, 4><<<grid, 4 * kRoleSites, 0, st>>>(a);
        else k_hop_roles<ff, 0, false, kRoleSites, 4><<<grid, 4 * kRoleSites, 0, st>>>(a);
    } else {
        if (dot) k_hop_roles<ff, 0, true, kRoleSites, 3><<<grid, 4 * kRoleSites, 0, st>>>(a);
        else k_hop_roles<ff, 0, false, kRoleSites, 3><<<grid, 4 * kRoleSites, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lq
