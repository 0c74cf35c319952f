// Inner linear solves of the shift-and-invert eigensolver (lq_compute_deflation): conjugate
// gradients on the normal equations (CGNR), A^dag A x = A^dag b, for several systems at once, each
// with its own operator A_s in {H(mu), H(mu)^dag}.  Vectors live in the internal FP32 layout
// (float4 chunks [6][V] per system); the CG scalars are FP64 and stay on the device, so an
// iteration needs no host synchronisation: two stencil launches (by the caller) and the three
// kernels below.  The driver in lq_api.cu wraps the FP32 solve in FP64 defect correction.
//
// CGNR (Hestenes & Stiefel's CG applied to A^dag A; Saad, "Iterative Methods for Sparse Linear
// Systems", 2nd ed., Sec. 8.3):  r = b - A x,  z = A^dag r,  p = z,  g = |z|^2;  repeat
//   q = A p;  alpha = g / |q|^2;  x += alpha p;  r -= alpha q;  z = A^dag r;
//   g' = |z|^2;  p = z + (g' / g) p;  g = g'.
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

namespace lq {
namespace {

constexpr int kCgThreads = 256;
constexpr int kCgBlocks = 304;   // blocks per system: two per SM of the 152

// Sum over the system's elements of |v|^2 into scal[sys * kCgNs + slot] (last-block reduction).
__global__ void __launch_bounds__(kCgThreads) k_cg_norm(CgArgs a, const float4* __restrict__ v, int slot) {
    __shared__ CSum smem[32];
    const int sys = blockIdx.y;
    if (a.scal[sys * kCgNs + CG_DONE] != 0.0) return;
    const float4* vs = v + (size_t)sys * a.ne;
    float acc = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.ne; e += (size_t)gridDim.x * blockDim.x) {
        const float4 t = vs[e];
        acc = fmaf(t.x, t.x, fmaf(t.y, t.y, fmaf(t.z, t.z, fmaf(t.w, t.w, acc))));
    }
    CSum s[1] = {{(double)acc, 0.0}};
    block_reduce_cs<1>(s, smem);
    double* part = a.part + ((size_t)sys * kCgBlocks + blockIdx.x) * 2;
    if (threadIdx.x == 0) { part[0] = s[0].s; part[1] = s[0].e; }
    if (last_block(a.counters + sys * 3 + 0, gridDim.x)) {
        double res[1];
        reduce_partials<1>(a.part + (size_t)sys * kCgBlocks * 2, gridDim.x, res, smem);
        if (threadIdx.x == 0) a.scal[sys * kCgNs + slot] = res[0];
    }
}

// x += alpha p, r -= alpha q with alpha = g / |q|^2; |r|^2 into CG_RR.
__global__ void __launch_bounds__(kCgThreads) k_cg_xr(CgArgs a) {
    __shared__ CSum smem[32];
    const int sys = blockIdx.y;
    const double* sc = a.scal + sys * kCgNs;
    if (sc[CG_DONE] != 0.0) return;
    const double qq = sc[CG_QQ];
    const float al = qq > 0.0 ? (float)(sc[CG_G0 + (a.it & 1)] / qq) : 0.f;
    float4* x = a.x + (size_t)sys * a.ne;
    float4* r = a.r + (size_t)sys * a.ne;
    const float4* p = a.p + (size_t)sys * a.ne;
    const float4* q = a.q + (size_t)sys * a.ne;
    float acc = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.ne; e += (size_t)gridDim.x * blockDim.x) {
        const float4 pe = p[e], qe = q[e];
        float4 xe = x[e], re = r[e];
        xe.x = fmaf(al, pe.x, xe.x); xe.y = fmaf(al, pe.y, xe.y); xe.z = fmaf(al, pe.z, xe.z); xe.w = fmaf(al, pe.w, xe.w);
        re.x = fmaf(-al, qe.x, re.x); re.y = fmaf(-al, qe.y, re.y); re.z = fmaf(-al, qe.z, re.z); re.w = fmaf(-al, qe.w, re.w);
        x[e] = xe;
        r[e] = re;
        acc = fmaf(re.x, re.x, fmaf(re.y, re.y, fmaf(re.z, re.z, fmaf(re.w, re.w, acc))));
    }
    CSum s[1] = {{(double)acc, 0.0}};
    block_reduce_cs<1>(s, smem);
    double* part = a.part + ((size_t)sys * kCgBlocks + blockIdx.x) * 2;
    if (threadIdx.x == 0) { part[0] = s[0].s; part[1] = s[0].e; }
    if (last_block(a.counters + sys * 3 + 1, gridDim.x)) {
        double res[1];
        reduce_partials<1>(a.part + (size_t)sys * kCgBlocks * 2, gridDim.x, res, smem);
        if (threadIdx.x == 0) a.scal[sys * kCgNs + CG_RR] = res[0];
    }
}

// p = z + (g' / g) p, g' in slot CG_G0 + ((it + 1) & 1), g in CG_G0 + (it & 1).
__global__ void __launch_bounds__(kCgThreads) k_cg_p(CgArgs a) {
    const int sys = blockIdx.y;
    const double* sc = a.scal + sys * kCgNs;
    if (sc[CG_DONE] != 0.0) return;
    const double g = sc[CG_G0 + (a.it & 1)];
    const float be = g > 0.0 ? (float)(sc[CG_G0 + ((a.it + 1) & 1)] / g) : 0.f;
    float4* p = a.p + (size_t)sys * a.ne;
    const float4* z = a.z + (size_t)sys * a.ne;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.ne; e += (size_t)gridDim.x * blockDim.x) {
        const float4 ze = z[e];
        float4 pe = p[e];
        pe.x = fmaf(be, pe.x, ze.x); pe.y = fmaf(be, pe.y, ze.y); pe.z = fmaf(be, pe.z, ze.z); pe.w = fmaf(be, pe.w, ze.w);
        p[e] = pe;
    }
}

}  // namespace

size_t cg_partial_doubles(int nsys) { return (size_t)nsys * kCgBlocks * 2; }

cudaError_t launch_cg_norm(const CgArgs& a, const float4* v, int slot, cudaStream_t st) {
    k_cg_norm<<<dim3(kCgBlocks, (unsigned)a.nb), kCgThreads, 0, st>>>(a, v, slot);
    return cudaGetLastError();
}
cudaError_t launch_cg_xr(const CgArgs& a, cudaStream_t st) {
    k_cg_xr<<<dim3(kCgBlocks, (unsigned)a.nb), kCgThreads, 0, st>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_cg_p(const CgArgs& a, cudaStream_t st) {
    k_cg_p<<<dim3(kCgBlocks, (unsigned)a.nb), kCgThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lq
