// Nested two-sided Lanczos evaluation of the projected sign sgn(T_k) e_1 (Sec. 4: one level of
// nesting, inner Krylov subspace of size 100).  The inner process is the two-sided Lanczos
// recurrence of Sec. 2 on the k x k matrix
//     M = T / c + c T^{-1},
// started at e_1 (or at a given vector).  M is a function of T with the same sign, since
// Re(z / c + c / z) = Re(z) (1/c + c/|z|^2), and it folds the eigenvalue moduli of T about c (|z|
// and c^2/|z| land on one circle), so m << k inner steps resolve what k outer steps produced.
// Then sgn(T) e_1 ~ |e| V'_m sgn(T'_m) e_1 with the inner m x m tridiagonal T'_m, whose sign the
// batched device Newton iteration takes.  The result is checked by a second pass started at the
// first pass's result: sgn^2 = 1, so ||sgn(T) s - e_1|| measures the error.
//
// One block per source.  T^{-1} (and T^{-H}) are applied through a pivoted tridiagonal LU
// factorisation computed once per source (Gaussian elimination with partial pivoting; Golub &
// Van Loan, "Matrix Computations", Sec. 4.3): its forward and back substitutions are O(k) and
// sequential, two of them (M v and M^H w) run by two warps of the block in parallel, everything
// else (the tridiagonal products, the dots, the recurrences) over all threads.
#include "lq_internal.cuh"
#include "lq_launch.h"

namespace lq {
namespace {

constexpr int kNestThreads = 256;

__device__ __forceinline__ double2 crecip(double2 z) {
    const double r = 1.0 / (z.x * z.x + z.y * z.y);
    return make_double2(z.x * r, -z.y * r);
}
__device__ __forceinline__ double2 cconj(double2 z) { return make_double2(z.x, -z.y); }

// Per-source workspace (complex entries, row length kmax): the two factorisations, the inner
// vectors and the inner basis.
struct NestWork {
    double2 *fl, *fu0, *fu1, *fu2;          // T = P L U: multipliers, 1/u0, u1, u2 (piv in fpiv)
    double2 *gl, *gu0, *gu1, *gu2;          // the same for T^H
    double2 *v, *w, *vp, *wp, *t1, *t2, *y1, *y2;
    double2* basis;                          // [m][kmax]
    unsigned char* fpiv;                     // [2][kmax] pivot flags (T, T^H)
};
__device__ __forceinline__ NestWork nest_work(const NestArgs& a, int src) {
    double2* b = a.work + (size_t)src * a.work_stride;
    const size_t K = (size_t)a.kmax;
    NestWork w;
    w.fl = b; w.fu0 = b + K; w.fu1 = b + 2 * K; w.fu2 = b + 3 * K;
    w.gl = b + 4 * K; w.gu0 = b + 5 * K; w.gu1 = b + 6 * K; w.gu2 = b + 7 * K;
    w.v = b + 8 * K; w.w = b + 9 * K; w.vp = b + 10 * K; w.wp = b + 11 * K;
    w.t1 = b + 12 * K; w.t2 = b + 13 * K; w.y1 = b + 14 * K; w.y2 = b + 15 * K;
    w.basis = b + 16 * K;
    w.fpiv = reinterpret_cast<unsigned char*>(b + 16 * K + (size_t)a.m * K);
    return w;
}
// nest_work uses 16 kmax + m kmax complex entries plus 2 kmax bytes
}  // namespace

size_t nest_work_entries(int kmax, int m) { return (size_t)(16 + m) * kmax + ((size_t)2 * kmax + 15) / 16 + 1; }

namespace {

__device__ __forceinline__ int nest_k(const NestArgs& a, int src) { return a.state ? a.state[src].k_eff : a.kfix; }

// Entries of T (sub = delta real) or of T^H.
struct Tri {
    const double2* al; const double2* be; const double* de; bool herm;
    __device__ double2 d(int i) const { return herm ? cconj(al[i]) : al[i]; }
    __device__ double2 up(int i) const { return herm ? make_double2(de[i], 0.0) : be[i]; }   // (i, i+1)
    __device__ double2 lo(int i) const { return herm ? cconj(be[i]) : make_double2(de[i], 0.0); }   // (i+1, i)
};

// P L U of the k x k tridiagonal (partial pivoting between rows i and i + 1 at each step).
__device__ void tri_factor(const Tri& T, int k, double2* fl, double2* fu0, double2* fu1, double2* fu2, unsigned char* piv) {
    double2 a = T.d(0), b = (k > 1) ? T.up(0) : make_double2(0.0, 0.0);   // active row: cols i, i+1
    for (int i = 0; i < k - 1; ++i) {
        const double2 s = T.lo(i), d = T.d(i + 1);
        const double2 u = (i + 1 < k - 1) ? T.up(i + 1) : make_double2(0.0, 0.0);
        if (s.x * s.x + s.y * s.y > a.x * a.x + a.y * a.y) {
            // pivot row R_{i+1} = (s, d, u); active' = A_i - l R_{i+1}
            const double2 l = cmul(a, crecip(s));
            piv[i] = 1; fl[i] = l; fu0[i] = crecip(s); fu1[i] = d; fu2[i] = u;
            a = csub(b, cmul(l, d));
            b = make_double2(-(l.x * u.x - l.y * u.y), -(l.x * u.y + l.y * u.x));
        } else {
            const double2 l = cmul(s, crecip(a));
            piv[i] = 0; fl[i] = l; fu0[i] = crecip(a); fu1[i] = b; fu2[i] = make_double2(0.0, 0.0);
            a = csub(d, cmul(l, b));
            b = u;
        }
    }
    piv[k - 1] = 0; fl[k - 1] = make_double2(0.0, 0.0); fu0[k - 1] = crecip(a);
    fu1[k - 1] = make_double2(0.0, 0.0); fu2[k - 1] = make_double2(0.0, 0.0);
}

// x = (P L U)^{-1} rhs (sequential); x may alias nothing in rhs.
__device__ void tri_apply_inverse(int k, const double2* fl, const double2* fu0, const double2* fu1, const double2* fu2,
                                  const unsigned char* piv, const double2* rhs, double2* x) {
    double2 cx = rhs[0];
    for (int i = 0; i < k - 1; ++i) {
        const double2 nx = rhs[i + 1];
        if (piv[i]) { x[i] = nx; cx = csub(cx, cmul(fl[i], nx)); }
        else { x[i] = cx; cx = csub(nx, cmul(fl[i], cx)); }
    }
    x[k - 1] = cx;
    double2 x1 = cmul(x[k - 1], fu0[k - 1]), x2 = make_double2(0.0, 0.0);
    x[k - 1] = x1;
    for (int i = k - 2; i >= 0; --i) {
        double2 t = csub(x[i], cmul(fu1[i], x1));
        t = csub(t, cmul(fu2[i], x2));
        t = cmul(t, fu0[i]);
        x[i] = t;
        x2 = x1;
        x1 = t;
    }
}

// Block sum of NV doubles (plain FP64; result in every thread).
template <int NV>
__device__ __forceinline__ void nest_sum(double (&v)[NV], double* sh) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[warp * NV + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += sh[q * NV + i];
        v[i] = s;
    }
    __syncthreads();
}

__global__ void k_nest_factor(NestArgs a) {
    const int src = blockIdx.x;
    if (a.sel && !a.sel[src]) return;
    const int k = nest_k(a, src);
    if (k <= 0 || threadIdx.x >= 2) return;
    NestWork w = nest_work(a, src);
    const Tri T{a.alpha + (size_t)src * a.kmax, a.beta + (size_t)src * a.kmax, a.delta + (size_t)src * a.kmax, threadIdx.x == 1};
    if (threadIdx.x == 0) tri_factor(T, k, w.fl, w.fu0, w.fu1, w.fu2, w.fpiv);
    else tri_factor(T, k, w.gl, w.gu0, w.gu1, w.gu2, w.fpiv + a.kmax);
}

// The inner process (m steps) for one source per block.
__global__ void __launch_bounds__(kNestThreads) k_nest_lanczos(NestArgs a) {
    __shared__ double sh[32 * 8];
    const int src = blockIdx.x;
    if (a.sel && !a.sel[src]) return;
    const int k = nest_k(a, src);
    TslState& is = a.istate[src];
    if (k <= 0) {
        if (threadIdx.x == 0) { is.k_eff = 0; is.status = LQ_ERR_NOT_READY; }
        return;
    }
    const int m = min(a.m, k);
    NestWork w = nest_work(a, src);
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    const double c = a.cscale[src], ic = 1.0 / c;
    double2* ia = a.ialpha + (size_t)src * a.kmax;
    double2* ib = a.ibeta + (size_t)src * a.kmax;
    double* id = a.idelta + (size_t)src * a.kmax;
    const double2* x0 = a.start ? a.start + (size_t)src * a.kmax : nullptr;
    // v_1 = w_1 = x0 / |x0|
    double nn[1] = {0.0};
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double2 z = x0 ? x0[i] : make_double2(i == 0 ? 1.0 : 0.0, 0.0);
        nn[0] += z.x * z.x + z.y * z.y;
    }
    nest_sum<1>(nn, sh);
    const double xn = sqrt(nn[0]);
    if (threadIdx.x == 0) { a.snorm[src] = xn; is.status = 0; is.k_eff = 0; }
    if (!(xn > 0.0) || !isfinite(xn)) {
        if (threadIdx.x == 0) is.status = isfinite(xn) ? LQ_ERR_ARG : LQ_ERR_NONFINITE;
        return;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double2 z = x0 ? x0[i] : make_double2(i == 0 ? 1.0 : 0.0, 0.0);
        const double2 v = make_double2(z.x / xn, z.y / xn);
        w.v[i] = v; w.w[i] = v;
        w.vp[i] = make_double2(0.0, 0.0); w.wp[i] = make_double2(0.0, 0.0);
    }
    double2 beta_p = make_double2(0.0, 0.0);
    double delta_p = 0.0;
    int meff = m;
    for (int j = 0; j < m; ++j) {
        __syncthreads();
        double2* bj = w.basis + (size_t)j * a.kmax;
        // t1 = T v / c, t2 = T^H w / c; the basis keeps v_j
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const double2 vi = w.v[i], wi = w.w[i];
            double2 s = cmul(al[i], vi);
            double2 h = cmul(cconj(al[i]), wi);
            if (i + 1 < k) {
                s = cadd(s, cmul(be[i], w.v[i + 1]));
                h = cadd(h, cscale(w.w[i + 1], de[i]));
            }
            if (i > 0) {
                s = cadd(s, cscale(w.v[i - 1], de[i - 1]));
                h = cadd(h, cmul(cconj(be[i - 1]), w.w[i - 1]));
            }
            w.t1[i] = cscale(s, ic);
            w.t2[i] = cscale(h, ic);
            bj[i] = vi;
        }
        __syncthreads();
        // y1 = T^{-1} v (warp 0), y2 = T^{-H} w (warp 1)
        if (threadIdx.x == 0) tri_apply_inverse(k, w.fl, w.fu0, w.fu1, w.fu2, w.fpiv, w.v, w.y1);
        if (threadIdx.x == 32) tri_apply_inverse(k, w.gl, w.gu0, w.gu1, w.gu2, w.fpiv + a.kmax, w.w, w.y2);
        __syncthreads();
        // t = M v, M^H w; alpha_j = <w_j, M v_j>
        double r[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const double2 t1 = cadd(w.t1[i], cscale(w.y1[i], c));
            const double2 t2 = cadd(w.t2[i], cscale(w.y2[i], c));
            w.t1[i] = t1; w.t2[i] = t2;
            const double2 wi = w.w[i];
            r[0] += wi.x * t1.x + wi.y * t1.y;
            r[1] += wi.x * t1.y - wi.y * t1.x;
        }
        nest_sum<2>(r, sh);
        const double2 alj = make_double2(r[0], r[1]);
        if (threadIdx.x == 0) ia[j] = alj;
        if (j == m - 1) break;
        // vh = t1 - alpha v - beta_{j-1} v_{j-1};  wh = t2 - conj(alpha) w - conj(delta_{j-1}) w_{j-1}
        double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // Re <wh, vh>, Im, |vh|^2, |wh|^2, |t1|^2 + |t2|^2 scale
        double tt[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const double2 t1 = w.t1[i], t2 = w.t2[i];
            double2 vh = csub(csub(t1, cmul(alj, w.v[i])), cmul(beta_p, w.vp[i]));
            double2 wh = csub(csub(t2, cmul(cconj(alj), w.w[i])), cscale(w.wp[i], delta_p));
            w.t1[i] = vh; w.t2[i] = wh;
            q[0] += wh.x * vh.x + wh.y * vh.y;
            q[1] += wh.x * vh.y - wh.y * vh.x;
            q[2] += vh.x * vh.x + vh.y * vh.y;
            q[3] += wh.x * wh.x + wh.y * wh.y;
            tt[0] += t1.x * t1.x + t1.y * t1.y;
            tt[1] += t2.x * t2.x + t2.y * t2.y;
        }
        nest_sum<5>(q, sh);
        nest_sum<2>(tt, sh);
        const double om = hypot(q[0], q[1]);
        // an invariant subspace or a serious breakdown ends the inner process (as in the outer one)
        if (q[2] <= 1e-20 * tt[0] || q[3] <= 1e-20 * tt[1] || om < 1e-14 * sqrt(q[2]) * sqrt(q[3]) || !isfinite(om)) {
            meff = j + 1;
            if (!isfinite(om) && threadIdx.x == 0) is.status = LQ_ERR_NONFINITE;
            break;
        }
        const double dl = sqrt(om);
        const double2 bt = make_double2(q[0] / dl, q[1] / dl);
        if (threadIdx.x == 0) { id[j] = dl; ib[j] = bt; }
        const double2 ibc = crecip(cconj(bt));    // w_{j+1} = wh / conj(beta)
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            w.vp[i] = w.v[i]; w.wp[i] = w.w[i];
            w.v[i] = cscale(w.t1[i], 1.0 / dl);
            w.w[i] = cmul(w.t2[i], ibc);
        }
        beta_p = bt;
        delta_p = dl;
    }
    if (threadIdx.x == 0) is.k_eff = meff;
}

// out = |x0| V' s' (s' = sgn(T'_m) e_1 from the Newton iteration, row stride kmax) for rows < k.
__global__ void k_nest_combine(NestArgs a, const double2* __restrict__ sp, double2* __restrict__ out) {
    const int src = blockIdx.y;
    if (a.sel && !a.sel[src]) return;
    const int k = nest_k(a, src);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.kmax) return;
    const int meff = a.istate[src].k_eff;
    double2 acc = make_double2(0.0, 0.0);
    if (i < k && a.istate[src].status == 0) {
        const double2* s = sp + (size_t)src * a.kmax;
        const double2* B = nest_work(a, src).basis;
        for (int j = 0; j < meff; ++j) acc = cadd(acc, cmul(s[j], B[(size_t)j * a.kmax + i]));
        acc = cscale(acc, a.snorm[src]);
    }
    out[(size_t)src * a.kmax + i] = acc;
}

// check[src] = || q - e_1 || over the first k rows (the involution residual of the two passes).
__global__ void k_nest_check(NestArgs a, const double2* __restrict__ q, double* __restrict__ check) {
    __shared__ double sh[32];
    const int src = blockIdx.x;
    if (a.sel && !a.sel[src]) return;
    const int k = nest_k(a, src);
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double2 z = q[(size_t)src * a.kmax + i];
        const double ex = (i == 0) ? 1.0 : 0.0;
        s[0] += (z.x - ex) * (z.x - ex) + z.y * z.y;
    }
    nest_sum<1>(s, sh);
    if (threadIdx.x == 0) check[src] = (a.istate[src].status == 0 && k > 0) ? sqrt(s[0]) : INFINITY;
}

}  // namespace

cudaError_t nest_factor(const NestArgs& a, cudaStream_t st) {
    k_nest_factor<<<a.nb, 32, 0, st>>>(a);
    return cudaGetLastError();
}
cudaError_t nest_lanczos(const NestArgs& a, cudaStream_t st) {
    k_nest_lanczos<<<a.nb, kNestThreads, 0, st>>>(a);
    return cudaGetLastError();
}
cudaError_t nest_combine(const NestArgs& a, const double2* sp, double2* out, cudaStream_t st) {
    k_nest_combine<<<dim3((unsigned)((a.kmax + 127) / 128), (unsigned)a.nb), 128, 0, st>>>(a, sp, out);
    return cudaGetLastError();
}
cudaError_t nest_check(const NestArgs& a, const double2* q, double* check, cudaStream_t st) {
    k_nest_check<<<a.nb, 256, 0, st>>>(a, q, check);
    return cudaGetLastError();
}

}  // namespace lq
