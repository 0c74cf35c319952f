// Deflation of Sec. 3 on FP64 vectors in the boundary layout:
//   * k_bdots      -- all inner products <X_a | Y_b> of two sets of vectors (compensated FP64);
//   * k_bcombine   -- Z_b = W_b + sum_a coef[b][a] X_a (several vector sets at once).
// The projections Pbar x = x - sum_i R_i <L_i|x>, the exact parts of Eqs. (3.1) and (3.4) and
// the eigenvector-derivative assembly are all combinations of these two operations, with the
// small coefficient matrices formed on the host.
#include "lq_internal.cuh"
#include "lq_launch.h"

namespace lq {

constexpr int kDotThreads = 256;

// partial[pair][blockIdx.x] for pair = a * ny + b, then k_bdots_finish sums the partials.
__global__ void __launch_bounds__(kDotThreads) k_bdots(const double2* __restrict__ X, size_t xs, int nx,
                                                       const double2* __restrict__ Y, size_t ys, int ny, size_t n,
                                                       double* __restrict__ partial) {
    __shared__ CSum smem[32 * 2];
    const int pair = blockIdx.y;
    const int a = pair / ny, b = pair % ny;
    const double2* x = X + (size_t)a * xs;
    const double2* y = Y + (size_t)b * ys;
    CSum acc[2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 u = x[i], v = y[i];
        cs_add_prod(acc[0], u.x, v.x); cs_add_prod(acc[0], u.y, v.y);     // Re conj(u) v
        cs_add_prod(acc[1], u.x, v.y); cs_add_prod(acc[1], -u.y, v.x);    // Im conj(u) v
    }
    block_reduce_cs<2>(acc, smem);
    if (threadIdx.x == 0) {
        double* p = partial + ((size_t)pair * gridDim.x + blockIdx.x) * 4;
        p[0] = acc[0].s; p[1] = acc[0].e; p[2] = acc[1].s; p[3] = acc[1].e;
    }
}

__global__ void k_bdots_finish(const double* __restrict__ partial, int nblocks, int npairs, double2* __restrict__ out) {
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    if (pair >= npairs) return;
    CSum re{0.0, 0.0}, im{0.0, 0.0};
    for (int q = 0; q < nblocks; ++q) {
        const double* p = partial + ((size_t)pair * nblocks + q) * 4;
        re = cs_merge(re, CSum{p[0], p[1]});
        im = cs_merge(im, CSum{p[2], p[3]});
    }
    out[pair] = make_double2(re.s + re.e, im.s + im.e);
}

// Z_b = W_b + sum_{a < nx} coef[b * nx + a] X_a  (W may alias Z; W null means 0)
__global__ void k_bcombine(double2* __restrict__ Z, const double2* W, size_t zs, int nz,
                           const double2* __restrict__ X, size_t xs, int nx, const double2* __restrict__ coef, size_t n) {
    const int b = blockIdx.y;
    const double2* cb = coef + (size_t)b * nx;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 acc = W ? W[(size_t)b * zs + i] : make_double2(0.0, 0.0);
        for (int a = 0; a < nx; ++a) acc = cfma(__ldg(cb + a), __ldg(X + (size_t)a * xs + i), acc);
        Z[(size_t)b * zs + i] = acc;
    }
}

// Z = a1 X1 + a2 X2 + a3 X3 elementwise over n doubles (real coefficients; X3 may be null)
__global__ void k_axpby3(double* __restrict__ Z, double a1, const double* __restrict__ X1, double a2,
                         const double* __restrict__ X2, double a3, const double* __restrict__ X3, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = a1 * X1[i] + a2 * X2[i];
        if (X3) v += a3 * X3[i];
        Z[i] = v;
    }
}

cudaError_t launch_axpby3(double* Z, double a1, const double* X1, double a2, const double* X2, double a3, const double* X3,
                          size_t n, cudaStream_t st) {
    k_axpby3<<<1216, 256, 0, st>>>(Z, a1, X1, a2, X2, a3, X3, n);
    return cudaGetLastError();
}

constexpr int kDotBlocks = 32;

cudaError_t launch_bdots(const double* X, size_t xs, int nx, const double* Y, size_t ys, int ny, size_t n,
                         double* partial, double* out, cudaStream_t st) {
    if (nx <= 0 || ny <= 0) return cudaSuccess;
    dim3 grid(kDotBlocks, (unsigned)(nx * ny));
    k_bdots<<<grid, kDotThreads, 0, st>>>(reinterpret_cast<const double2*>(X), xs / 2, nx,
                                          reinterpret_cast<const double2*>(Y), ys / 2, ny, n / 2, partial);
    k_bdots_finish<<<(nx * ny + 127) / 128, 128, 0, st>>>(partial, kDotBlocks, nx * ny, reinterpret_cast<double2*>(out));
    return cudaGetLastError();
}

cudaError_t launch_bcombine(double* Z, const double* W, size_t zs, int nz, const double* X, size_t xs, int nx,
                            const double* coef, size_t n, cudaStream_t st) {
    if (nz <= 0) return cudaSuccess;
    dim3 grid(256, (unsigned)nz);
    k_bcombine<<<grid, 256, 0, st>>>(reinterpret_cast<double2*>(Z), reinterpret_cast<const double2*>(W), zs / 2, nz,
                                     reinterpret_cast<const double2*>(X), xs / 2, nx, reinterpret_cast<const double2*>(coef), n / 2);
    return cudaGetLastError();
}

size_t bdots_partial_doubles(int npairs) { return (size_t)npairs * kDotBlocks * 4; }

// Per-source inner products <X_s | Y_s> (compensated FP64), partial[s][blockIdx.x]; summed by
// k_bdots_finish.  Source s of a set starts at s * xs (or s * ys) complex numbers.
__global__ void __launch_bounds__(kDotThreads) k_sdots(const double2* __restrict__ X, size_t xs,
                                                       const double2* __restrict__ Y, size_t ys, size_t n,
                                                       double* __restrict__ partial) {
    __shared__ CSum smem[32 * 2];
    const int src = blockIdx.y;
    const double2* x = X + (size_t)src * xs;
    const double2* y = Y + (size_t)src * ys;
    CSum acc[2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 u = x[i], v = y[i];
        cs_add_prod(acc[0], u.x, v.x); cs_add_prod(acc[0], u.y, v.y);
        cs_add_prod(acc[1], u.x, v.y); cs_add_prod(acc[1], -u.y, v.x);
    }
    block_reduce_cs<2>(acc, smem);
    if (threadIdx.x == 0) {
        double* p = partial + ((size_t)src * gridDim.x + blockIdx.x) * 4;
        p[0] = acc[0].s; p[1] = acc[0].e; p[2] = acc[1].s; p[3] = acc[1].e;
    }
}

cudaError_t launch_sdots(const double* X, const double* Y, size_t stride, size_t n, int nsrc, double* partial, double* out,
                         cudaStream_t st) {
    if (nsrc <= 0) return cudaSuccess;
    k_sdots<<<dim3(kDotBlocks, (unsigned)nsrc), kDotThreads, 0, st>>>(reinterpret_cast<const double2*>(X), stride / 2,
                                                                      reinterpret_cast<const double2*>(Y), stride / 2, n / 2, partial);
    k_bdots_finish<<<(nsrc + 127) / 128, 128, 0, st>>>(partial, kDotBlocks, nsrc, reinterpret_cast<double2*>(out));
    return cudaGetLastError();
}

// Per-source combinations Z_s = c[s][0] X0_s + c[s][1] X1_s + c[s][2] X2_s (complex coefficients;
// X1, X2 may be null; Z may alias any X: element i is read before it is written)
__global__ void k_scomb(double2* Z, const double2* X0, const double2* X1, const double2* X2, const double2* __restrict__ coef,
                        size_t stride, size_t n) {
    const int src = blockIdx.y;
    const double2 c0 = coef[src * 3], c1 = coef[src * 3 + 1], c2 = coef[src * 3 + 2];
    const size_t o = (size_t)src * stride;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = cmul(c0, X0[o + i]);
        if (X1) v = cfma(c1, X1[o + i], v);
        if (X2) v = cfma(c2, X2[o + i], v);
        Z[o + i] = v;
    }
}

cudaError_t launch_scomb(double* Z, const double* X0, const double* X1, const double* X2, const double* coef, size_t stride,
                         size_t n, int nsrc, cudaStream_t st) {
    if (nsrc <= 0) return cudaSuccess;
    k_scomb<<<dim3(256, (unsigned)nsrc), 256, 0, st>>>(reinterpret_cast<double2*>(Z), reinterpret_cast<const double2*>(X0),
                                                       reinterpret_cast<const double2*>(X1), reinterpret_cast<const double2*>(X2),
                                                       reinterpret_cast<const double2*>(coef), stride / 2, n / 2);
    return cudaGetLastError();
}

// out = cx x + cs gamma5 s on boundary-layout FP64 fields (x may be null); gamma5 = diag(1, 1, -1, -1)
// on spin.  With cx = 1 + m/2, cs = 1 - m/2 and s = sgn(H) x: the massive overlap operator D(m) x.
__global__ void k_g5axpy(double2* out, const double2* x, double cx, const double2* s, double cs, size_t ncomp) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncomp; i += (size_t)gridDim.x * blockDim.x) {
        const double g = (i % 12 < 6) ? cs : -cs;
        const double2 v = s[i];
        double2 r = make_double2(g * v.x, g * v.y);
        if (x) { const double2 xv = x[i]; r.x += cx * xv.x; r.y += cx * xv.y; }
        out[i] = r;
    }
}

cudaError_t launch_g5axpy(double* out, const double* x, double cx, const double* s, double cs, size_t nsites, cudaStream_t st) {
    k_g5axpy<<<1216, 256, 0, st>>>(reinterpret_cast<double2*>(out), reinterpret_cast<const double2*>(x), cx,
                                   reinterpret_cast<const double2*>(s), cs, nsites * 12);
    return cudaGetLastError();
}

// Overlap operator of Eq. (1.1) from the sign and its derivative, in place on boundary-layout
// FP64 fields: s <- x + gamma5 s (D_ov x), d <- gamma5 d (d D_ov x; d may be null).  gamma5 =
// diag(1, 1, -1, -1) on spin: the first six of a site's twelve components keep their sign.
__global__ void k_overlap(const double2* __restrict__ x, double2* __restrict__ s, double2* __restrict__ d, size_t ncomp) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncomp; i += (size_t)gridDim.x * blockDim.x) {
        const double g = (i % 12 < 6) ? 1.0 : -1.0;
        const double2 v = s[i], xv = x[i];
        s[i] = make_double2(xv.x + g * v.x, xv.y + g * v.y);
        if (d) { const double2 w = d[i]; d[i] = make_double2(g * w.x, g * w.y); }
    }
}

cudaError_t launch_overlap(const double* x, double* s, double* d, size_t nsites, cudaStream_t st) {
    k_overlap<<<1216, 256, 0, st>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(s),
                                    reinterpret_cast<double2*>(d), nsites * 12);
    return cudaGetLastError();
}

}  // namespace lq
