// Adjoint of the two-sided Lanczos sign: the gradient of S = Re <y| sgn(H(mu)) |x> with respect
// to every link (the fermionic force, 8 su(3) components per link) and to mu.
//
// For f analytic on the spectrum tr(L_f(A, E) B) = tr(E L_f(A, B)), so every direction E gives
// dS/dt = Re tr(E G) with G = L_sgn(H, x y^H).  With V_1, T_1 from the Lanczos process started at
// x and W_2, T_2 from the process started at y, Mathias' block identity (Eq. (2.5)) applied to the
// projected block matrix [[T_1, |x||y| e_1 e_1^T], [0, T_2]] gives G ~ |x||y| V_1 X W_2^H, X the
// top-right block of sgn([[T_1, e_1 e_1^T], [0, T_2]]).  The quadrature of the projected sign
// makes X a sum of 2N rank-one terms:
//     X = - sum_q w_q a_q b_q^T,  a_q = (T_1 + i tau_q)^{-1} e_1,  b_q = (T_2 + i tau_q)^{-T} e_1,
// so Re tr(E G) = Re sum_q <omega_q| E |nu_q> with nu_q = -w_q |x||y| V_1 a_q and
// omega_q = W_2 conj(b_q): 2N vector pairs, contracted link by link.
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

namespace lq {

// Gaussian elimination with partial pivoting for a complex tridiagonal matrix given by
// accessors (diagonal D, super-diagonal Up, sub-diagonal Lo), right-hand side B(i) read in row
// order; U factors into sd/s1/s2 and w * x into sx, all at stride ld.
template <class DF, class UF, class LF, class BF>
__device__ void tri_solve_gen(int n, DF D, UF Up, LF Lo, BF B, double2* sd, double2* s1, double2* s2, double2* sx,
                              size_t ld, double2 w) {
    double2 cd = D(0), cu = (n > 1) ? Up(0) : make_double2(0.0, 0.0), cx = B(0);
    for (int i = 0; i < n - 1; ++i) {
        const double2 l = Lo(i);
        const double2 nd = D(i + 1);
        const double2 nu = (i + 1 < n - 1) ? Up(i + 1) : make_double2(0.0, 0.0);
        const double2 nx = B(i + 1);
        const size_t o = (size_t)i * ld;
        if (l.x * l.x + l.y * l.y > cd.x * cd.x + cd.y * cd.y) {
            const double2 f = cdiv(cd, l);
            sd[o] = l; s1[o] = nd; s2[o] = nu; sx[o] = nx;
            const double2 ncd = csub(cu, cmul(f, nd));
            const double2 ncu = make_double2(-(f.x * nu.x - f.y * nu.y), -(f.x * nu.y + f.y * nu.x));
            cx = csub(cx, cmul(f, nx));
            cd = ncd;
            cu = ncu;
        } else {
            const double2 f = cdiv(l, cd);
            sd[o] = cd; s1[o] = cu; s2[o] = make_double2(0.0, 0.0); sx[o] = cx;
            cd = csub(nd, cmul(f, cu));
            cu = nu;
            cx = csub(nx, cmul(f, cx));
        }
    }
    double2 x1 = cdiv(cx, cd), x2 = make_double2(0.0, 0.0);
    sx[(size_t)(n - 1) * ld] = cmul(x1, w);
    for (int i = n - 2; i >= 0; --i) {
        const size_t o = (size_t)i * ld;
        double2 v = csub(sx[o], cmul(s1[o], x1));
        v = csub(v, cmul(s2[o], x2));
        v = cdiv(v, sd[o]);
        sx[o] = cmul(v, w);
        x2 = x1;
        x1 = v;
    }
}

// One block of 2 * 2N threads: threads [0, 2N) solve for a_q with T_1 (source 0), threads
// [2N, 4N) for b_q with T_2^T (source 1).  Writes the recombination coefficients
//   cnu[q][j] = -w_q |x||y| a_q[j] s_j     (right basis of source 0, scales s_j)
//   com[q][j] = conj(b_q[j]) u_j           (left basis of source 1, scales u_j)
__global__ void k_adj_pairs(AdjArgs a) {
    const int nq = a.npairs;        // 2N
    const int t = threadIdx.x;
    const int side = t / nq;        // 0: a_q, 1: b_q
    const int q = t % nq;
    const int N = nq / 2;
    const int src = side;           // T_1 is source 0, T_2 source 1
    const int n = a.state[src].k_eff;
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    double2* base = a.work + (size_t)src * a.kmax * 4 * a.nth_max;
    double2* sd = base + q;
    double2* s1 = base + (size_t)a.kmax * a.nth_max + q;
    double2* s2 = base + (size_t)2 * a.kmax * a.nth_max + q;
    double2* sx = base + (size_t)3 * a.kmax * a.nth_max + q;
    const int j = q >> 1;
    const double sg = (q & 1) ? -1.0 : 1.0;
    const double c = a.c;
    const double th = (j + 0.5) * 3.14159265358979323846 / (2.0 * N);
    const double ct = cos(th);
    const double tau = sg * c * tan(th);
    const double w = c / (2.0 * N) / (ct * ct);
    auto B = [&](int i) -> double2 { return make_double2(i == 0 ? 1.0 : 0.0, 0.0); };
    auto D = [&](int i) -> double2 { double2 v = al[i]; v.y += tau; return v; };
    if (n > 0) {
        if (side == 0) {
            auto Up = [&](int i) -> double2 { return be[i]; };
            auto Lo = [&](int i) -> double2 { return make_double2(de[i], 0.0); };
            tri_solve_gen(n, D, Up, Lo, B, sd, s1, s2, sx, a.nth_max, make_double2(1.0, 0.0));
        } else {   // transpose: super-diagonal delta, sub-diagonal beta
            auto Up = [&](int i) -> double2 { return make_double2(de[i], 0.0); };
            auto Lo = [&](int i) -> double2 { return be[i]; };
            tri_solve_gen(n, D, Up, Lo, B, sd, s1, s2, sx, a.nth_max, make_double2(1.0, 0.0));
        }
    }
    double2* out = (side == 0 ? a.cnu : a.com) + (size_t)q * a.kmax;
    const double xy = a.state[0].xnorm * a.state[1].xnorm;
    for (int i = 0; i < a.kmax; ++i) {
        double2 v = make_double2(0.0, 0.0);
        if (i < n) {
            const double2 z = sx[(size_t)i * a.nth_max];
            if (side == 0) {
                const double f = -w * xy * a.scale[i];                       // scales of source 0
                v = make_double2(f * z.x, f * z.y);
            } else {
                const double2 u = a.uscale[(size_t)a.kmax + i];              // scales of source 1
                v = cmul(make_double2(z.x, -z.y), u);
            }
        }
        out[i] = v;
    }
}

// Deflated adjoint (the eigenpairs of Sec. 3 applied to G = L_sgn(H, x y^H)): with spectral
// projectors Pi = sum_j R_j L_j and Pbar = 1 - Pi, the blocks Pi G Pbar and Pbar G Pi are
//   sum_j R_j c_j u_j^H,  u_j = h_{conj lambda_j}(A^H) y',     sum_j v_j d_j L_j,  v_j = h_{lambda_j}(A) x',
// h_l(z) = (sgn z - sgn l) / (z - l), x' = Pbar x, y' = Pbar^H y, c_j = L_j x, d_j = y^H R_j.  With the
// quadrature sgn(z) ~ Q(z) = sum_q w_q (z + i tau_q)^{-1} of k_adj_pairs and the resolvent identity,
//   h_l(T) e_1 = -sum_q w_q (l + i tau_q)^{-1} (T + i tau_q)^{-1} e_1 + (Q(l) - sgn l) (T - l)^{-1} e_1,
// so v_j and u_j are combinations of the node solves a_q, b_q already in cnu / com plus one shifted
// tridiagonal solve.  Thread (j, side) writes the basis coefficients of d_j v_j (side 0, right basis
// of source 0) or conj(c_j) u_j (side 1, left basis of source 1).
__global__ void k_defl_coef(AdjArgs a) {
    const int nd = a.ndefl;
    const int t = threadIdx.x;
    if (t >= 2 * nd) return;
    const int side = t / nd, j = t % nd;
    const int nq = a.npairs, N = nq / 2;
    const int src = side;
    const int n = a.state[src].k_eff;
    const double2 lj = a.dlam[j];
    const double sl = lj.x > 0.0 ? 1.0 : -1.0;                    // sgn(lambda_j) = sign of Re
    const double2 l = side == 0 ? lj : make_double2(lj.x, -lj.y);  // lambda_j or its conjugate
    const double c = a.c;
    // per node: g_q = 1 / (l + i s tau_q) with s = +1 for v (T_1 + i tau_q) and s = -1 for u, whose
    // left solves b_q belong to T_2^H - i tau_q; the scalar quadrature Q(l) over all nodes
    double2 Q = make_double2(0.0, 0.0);
    for (int q = 0; q < nq; ++q) {
        const int jj = q >> 1;
        const double sg = (q & 1) ? -1.0 : 1.0;
        const double th = (jj + 0.5) * 3.14159265358979323846 / (2.0 * N);
        const double ct = cos(th);
        const double w = c / (2.0 * N) / (ct * ct);
        const double2 g = cdiv(make_double2(1.0, 0.0), make_double2(l.x, l.y + sg * c * tan(th)));
        Q = make_double2(Q.x + w * g.x, Q.y + w * g.y);
    }
    const double2 corr = make_double2(Q.x - sl, Q.y);   // Q(l) - sgn l
    // (T_1 - lambda_j)^{-1} e_1, or (T_2^T - lambda_j)^{-1} e_1 whose conjugate is (T_2^H - conj lambda_j)^{-1} e_1
    const double2* al = a.alpha + (size_t)src * a.kmax;
    const double2* be = a.beta + (size_t)src * a.kmax;
    const double* de = a.delta + (size_t)src * a.kmax;
    double2* base = a.work + (size_t)src * a.kmax * 4 * a.nth_max;
    const int col = nq + j;
    double2* sd = base + col;
    double2* s1 = base + (size_t)a.kmax * a.nth_max + col;
    double2* s2 = base + (size_t)2 * a.kmax * a.nth_max + col;
    double2* sx = base + (size_t)3 * a.kmax * a.nth_max + col;
    auto B = [&](int i) -> double2 { return make_double2(i == 0 ? 1.0 : 0.0, 0.0); };
    auto D = [&](int i) -> double2 { return csub(al[i], lj); };
    if (n > 0) {
        if (side == 0) {
            auto Up = [&](int i) -> double2 { return be[i]; };
            auto Lo = [&](int i) -> double2 { return make_double2(de[i], 0.0); };
            tri_solve_gen(n, D, Up, Lo, B, sd, s1, s2, sx, a.nth_max, make_double2(1.0, 0.0));
        } else {
            auto Up = [&](int i) -> double2 { return make_double2(de[i], 0.0); };
            auto Lo = [&](int i) -> double2 { return be[i]; };
            tri_solve_gen(n, D, Up, Lo, B, sd, s1, s2, sx, a.nth_max, make_double2(1.0, 0.0));
        }
    }
    const double nx = a.state[0].xnorm, ny = a.state[1].xnorm;
    const double2 fold = side == 0 ? a.ddy[j] : make_double2(a.dcx[j].x, -a.dcx[j].y);   // d_j or conj(c_j)
    double2* out = (side == 0 ? a.cnu + (size_t)(nq + 2 * nd + j) * a.kmax : a.com + (size_t)(nq + nd + j) * a.kmax);
    for (int i = 0; i < a.kmax; ++i) {
        double2 v = make_double2(0.0, 0.0);
        if (i < n) {
            for (int q = 0; q < nq; ++q) {
                const int jj = q >> 1;
                const double sg = (q & 1) ? -1.0 : 1.0;
                const double th = (jj + 0.5) * 3.14159265358979323846 / (2.0 * N);
                const double ct = cos(th);
                const double w = c / (2.0 * N) / (ct * ct);
                const double tau = sg * c * tan(th);
                if (side == 0) {
                    // cnu[q][i] = -w_q |x'||y'| a_q[i] s_i, so |x'| (-w_q g_q) a_q[i] s_i = cnu[q][i] g_q / |y'|
                    const double2 g = cdiv(make_double2(1.0, 0.0), make_double2(l.x, l.y + tau));
                    v = cfma(a.cnu[(size_t)q * a.kmax + i], make_double2(g.x / ny, g.y / ny), v);
                } else {
                    // com[q][i] = conj(b_q[i]) u_i and W_2 conj(b_q) = W_2 (T_2^H - i tau_q)^{-1} e_1
                    const double2 g = cdiv(make_double2(1.0, 0.0), make_double2(l.x, l.y - tau));
                    v = cfma(a.com[(size_t)q * a.kmax + i], make_double2(-w * ny * g.x, -w * ny * g.y), v);
                }
            }
            const double2 z = sx[(size_t)i * a.nth_max];
            if (side == 0) {
                const double2 r = cmul(corr, z);
                v = make_double2(v.x + nx * a.scale[i] * r.x, v.y + nx * a.scale[i] * r.y);
            } else {
                const double2 r = cmul(cmul(corr, make_double2(z.x, -z.y)), a.uscale[(size_t)a.kmax + i]);
                v = make_double2(v.x + ny * r.x, v.y + ny * r.y);
            }
        }
        out[i] = cmul(fold, v);
    }
}

// out[q] = sum_{j < k} coef[q][j] basis_j for QB outputs per thread (internal layout).
constexpr int kQB = 8;
template <typename R>
__global__ void __launch_bounds__(128) k_recomb_multi(const typename Tr<R>::Chunk* __restrict__ basis, size_t vec_stride,
                                                      int k, const double2* __restrict__ coef, int kmax, int nq,
                                                      typename Tr<R>::Chunk* __restrict__ out, size_t F) {
    using Chunk = typename Tr<R>::Chunk;
    extern __shared__ double2 sc[];    // [kQB][k] (FP64 and float-float bases), or float2 [kQB][k] for FP32 ones
    float2* scf = reinterpret_cast<float2*>(sc);
    const int q0 = blockIdx.y * kQB;
    for (int i = threadIdx.x; i < kQB * k; i += blockDim.x) {
        const int qq = i / k, j = i % k;
        const double2 cv = (q0 + qq < nq) ? coef[(size_t)(q0 + qq) * kmax + j] : make_double2(0.0, 0.0);
        if (Tr<R>::kKind == 0) sc[i] = cv;
        else if (Tr<R>::kKind == 2) {   // float-float coefficient (re.hi, re.lo, im.hi, im.lo)
            const ff re(cv.x), im(cv.y);
            reinterpret_cast<float4*>(sc)[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        } else scf[i] = make_float2((float)cv.x, (float)cv.y);
    }
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F) return;
    if constexpr (Tr<R>::kKind == 2) {
        // float-float basis: unnormalised float-float sums of the exact products (FP32 operations
        // only), renormalised once and stored as float-float
        FFSum ar[kQB], ai[kQB];
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq) { ar[qq] = FFSum{0.f, 0.f}; ai[qq] = FFSum{0.f, 0.f}; }
        const float4* scq = reinterpret_cast<const float4*>(sc);
        for (int j = 0; j < k; ++j) {
            const float4 q = reinterpret_cast<const float4*>(basis)[(size_t)j * vec_stride + e];
            const ff vr(q.x, q.y), vi(q.z, q.w);
#pragma unroll
            for (int qq = 0; qq < kQB; ++qq) {
                const float4 cf = scq[qq * k + j];
                const ff cr(cf.x, cf.y), ci(cf.z, cf.w);
                ffsum_add_prod<false>(ar[qq], cr, vr);
                ffsum_add_prod<true>(ar[qq], ci, vi);
                ffsum_add_prod<false>(ai[qq], cr, vi);
                ffsum_add_prod<false>(ai[qq], ci, vr);
            }
        }
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq)
            if (q0 + qq < nq) {
                const ff re = ff_two_sum(ar[qq].s, ar[qq].e), im = ff_two_sum(ai[qq].s, ai[qq].e);
                reinterpret_cast<float4*>(out)[(size_t)(q0 + qq) * F + e] = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
    } else if (Tr<R>::kKind == 0) {
        double2 acc[kQB];
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq) acc[qq] = make_double2(0.0, 0.0);
        for (int j = 0; j < k; ++j) {
            const double2 v = reinterpret_cast<const double2*>(basis)[(size_t)j * vec_stride + e];
#pragma unroll
            for (int qq = 0; qq < kQB; ++qq) acc[qq] = cfma(sc[qq * k + j], v, acc[qq]);
        }
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq)
            if (q0 + qq < nq) reinterpret_cast<double2*>(out)[(size_t)(q0 + qq) * F + e] = acc[qq];
    } else {
        float2 a0[kQB], a1[kQB];
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq) { a0[qq] = make_float2(0.f, 0.f); a1[qq] = make_float2(0.f, 0.f); }
        for (int j = 0; j < k; ++j) {
            const float4 v = reinterpret_cast<const float4*>(basis)[(size_t)j * vec_stride + e];
            const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
            for (int qq = 0; qq < kQB; ++qq) {
                const float2 cf = scf[qq * k + j];
                a0[qq] = cfma(cf, v0, a0[qq]);
                a1[qq] = cfma(cf, v1, a1[qq]);
            }
        }
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq)
            if (q0 + qq < nq)
                reinterpret_cast<float4*>(out)[(size_t)(q0 + qq) * F + e] = make_float4(a0[qq].x, a0[qq].y, a1[qq].x, a1[qq].y);
    }
}

// The same over a window [j0, j1) of Krylov indices whose vectors sit in ring slots j % ring
// (the second pass of a two-pass run), added to out (accumulate) or written.  FP64 accumulation
// within the window for both precisions; the window sums are added in FP64 (FP32 fields are
// widened, added, and rounded once per window).
template <typename R>
__global__ void __launch_bounds__(128) k_recomb_window(const typename Tr<R>::Chunk* __restrict__ basis, size_t vec_stride,
                                                       int j0, int j1, int ring, const double2* __restrict__ coef, int kmax,
                                                       int nq, typename Tr<R>::Chunk* __restrict__ out, size_t F, int accumulate) {
    using Chunk = typename Tr<R>::Chunk;
    __shared__ double2 sc[kQB * kTwoPassRing];
    const int q0 = blockIdx.y * kQB;
    const int w = j1 - j0;
    for (int i = threadIdx.x; i < kQB * w; i += blockDim.x) {
        const int qq = i / w, j = i % w;
        sc[i] = (q0 + qq < nq) ? coef[(size_t)(q0 + qq) * kmax + j0 + j] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F) return;
    constexpr int PC = Tr<R>::kPerChunk;     // complex numbers per chunk
    double2 acc[kQB][PC];
#pragma unroll
    for (int qq = 0; qq < kQB; ++qq)
#pragma unroll
        for (int p = 0; p < PC; ++p) acc[qq][p] = make_double2(0.0, 0.0);
    for (int j = 0; j < w; ++j) {
        const int slot = ring > 0 ? (j0 + j) % ring : j0 + j;
        const Chunk v = basis[(size_t)slot * vec_stride + e];
        double2 vv[PC];
        if constexpr (Tr<R>::kKind == 2) {
            const float4 f = reinterpret_cast<const float4&>(v);
            vv[0] = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
        } else if constexpr (PC == 1) {
            vv[0] = make_double2((double)reinterpret_cast<const double2&>(v).x, (double)reinterpret_cast<const double2&>(v).y);
        } else {
            const float4 f = reinterpret_cast<const float4&>(v); vv[0] = make_double2(f.x, f.y); vv[1] = make_double2(f.z, f.w);
        }
#pragma unroll
        for (int qq = 0; qq < kQB; ++qq)
#pragma unroll
            for (int p = 0; p < PC; ++p) acc[qq][p] = cfma(sc[qq * w + j], vv[p], acc[qq][p]);
    }
#pragma unroll
    for (int qq = 0; qq < kQB; ++qq) {
        if (q0 + qq >= nq) continue;
        Chunk* o = out + (size_t)(q0 + qq) * F + e;
        if constexpr (Tr<R>::kKind == 2) {
            double2 r = acc[qq][0];
            if (accumulate) {
                const float4 t = *reinterpret_cast<const float4*>(o);
                r.x += (double)t.x + (double)t.y; r.y += (double)t.z + (double)t.w;
            }
            const ff re(r.x), im(r.y);
            *reinterpret_cast<float4*>(o) = make_float4(re.hi, re.lo, im.hi, im.lo);
        } else if constexpr (PC == 1) {
            double2 r = acc[qq][0];
            if (accumulate) { const double2 t = *reinterpret_cast<const double2*>(o); r.x += t.x; r.y += t.y; }
            *reinterpret_cast<double2*>(o) = r;
        } else {
            double2 r0 = acc[qq][0], r1 = acc[qq][1];
            if (accumulate) {
                const float4 t = *reinterpret_cast<const float4*>(o);
                r0.x += t.x; r0.y += t.y; r1.x += t.z; r1.y += t.w;
            }
            *reinterpret_cast<float4*>(o) = make_float4((float)r0.x, (float)r0.y, (float)r1.x, (float)r1.y);
        }
    }
}

// Spinor loads in FP64 from either internal precision.
__device__ __forceinline__ void load_d(const double2* f, size_t V, size_t s, double2 (&o)[12]) { load_spinor(f, V, s, o); }
__device__ __forceinline__ void load_d(const float4* f, size_t V, size_t s, double2 (&o)[12]) {
    float2 t[12];
    load_spinor(f, V, s, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = make_double2((double)t[c].x, (double)t[c].y);
}
// float-float fields (one complex per float4 chunk), widened exactly
__device__ __forceinline__ void load_d_ff(const float4* f, size_t V, size_t s, double2 (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float4 q = __ldg(f + (size_t)c * V + s);
        o[c] = make_double2((double)q.x + (double)q.y, (double)q.z + (double)q.w);
    }
}
template <typename R, typename Chunk>
__device__ __forceinline__ void load_dk(const Chunk* f, size_t V, size_t s, double2 (&o)[12]) {
    if constexpr (Tr<R>::kKind == 2) load_d_ff(f, V, s, o);
    else load_d(f, V, s, o);
}

// (gamma5 (1 + SP gamma_NU) psi) in the chiral basis: (h, SP B^dag h) with the lower half negated.
template <int NU, int SP>
__device__ __forceinline__ void g5_proj(const double2 (&psi)[12], double2 (&out)[12]) {
    double2 h[6];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        const double2 u0 = psi[col], u1 = psi[3 + col], d2 = psi[6 + col], d3 = psi[9 + col];
        double2 b0, b1;
        if (NU == 0) { b0 = cmul_mi(d3); b1 = cmul_mi(d2); }
        else if (NU == 1) { b0 = make_double2(-d3.x, -d3.y); b1 = d2; }
        else if (NU == 2) { b0 = cmul_mi(d2); b1 = cmul_i(d3); }
        else { b0 = d2; b1 = d3; }
        h[col] = (SP > 0) ? cadd(u0, b0) : csub(u0, b0);
        h[3 + col] = (SP > 0) ? cadd(u1, b1) : csub(u1, b1);
    }
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        const double2 g0 = h[col], g1 = h[3 + col];
        double2 l0, l1;
        if (NU == 0) { l0 = cmul_i(g1); l1 = cmul_i(g0); }
        else if (NU == 1) { l0 = g1; l1 = make_double2(-g0.x, -g0.y); }
        else if (NU == 2) { l0 = cmul_i(g0); l1 = cmul_mi(g1); }
        else { l0 = g0; l1 = g1; }
        out[col] = g0;
        out[3 + col] = g1;
        // lower half: SP * B^dag h, then gamma5 flips its sign
        out[6 + col] = (SP > 0) ? make_double2(-l0.x, -l0.y) : l0;
        out[9 + col] = (SP > 0) ? make_double2(-l1.x, -l1.y) : l1;
    }
}

// P[c][c'] += sum_s conj(w[s][c]) g[s][c']
__device__ __forceinline__ void outer_acc(const double2 (&w)[12], const double2 (&g)[12], double2 (&P)[9]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) P[c * 3 + cc] = cfmac(w[sp * 3 + c], g[sp * 3 + cc], P[c * 3 + cc]);
}

template <typename R, int NU>
__device__ __forceinline__ void force_dir(const AdjArgs& a, size_t s, const int (&x)[4], double& dmu_acc) {
    using Chunk = typename Tr<R>::Chunk;
    const size_t V = a.V;
    const size_t F = field_elems<R>(V);
    const int ext = a.dims[NU];
    const size_t stride = a.strides[NU];
    const size_t sp = (x[NU] == ext - 1) ? s - (size_t)(ext - 1) * stride : s + stride;
    const double bs = (NU == 3 && a.apbc && x[NU] == ext - 1) ? -1.0 : 1.0;
    const Chunk* nu = reinterpret_cast<const Chunk*>(a.nu);
    const Chunk* om = reinterpret_cast<const Chunk*>(a.om);
    double2 Pf[9], Pb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) { Pf[i] = make_double2(0.0, 0.0); Pb[i] = make_double2(0.0, 0.0); }
    const int np = a.npairs_force > 0 ? a.npairs_force : a.npairs;
    for (int q = 0; q < np; ++q) {
        double2 w[12], v[12], g[12];
        // forward hop: conj(omega(x)) . gamma5 (1 - gamma) nu(x + nu)
        load_dk<R>(om + (size_t)q * F, V, s, w);
        load_dk<R>(nu + (size_t)q * F, V, sp, v);
        g5_proj<NU, -1>(v, g);
        outer_acc(w, g, Pf);
        // backward hop: conj(omega(x + nu)) . gamma5 (1 + gamma) nu(x)
        load_dk<R>(om + (size_t)q * F, V, sp, w);
        load_dk<R>(nu + (size_t)q * F, V, s, v);
        g5_proj<NU, +1>(v, g);
        outer_acc(w, g, Pb);
    }
    // Q = (i/4) bs [ -f+ U Pf^T + f- Pb^T U^dag ];  F^a = Re tr(lambda_a Q)
    const double2* U = a.Ub + ((size_t)NU * V + s) * 9;
    double2 u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = U[e];
    const double fp = (NU == 3) ? a.efwd : 1.0, fm = (NU == 3) ? a.ebwd : 1.0;
    double2 M[9];   // -f+ U Pf^T + f- Pb^T U^dag
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            double2 t1 = make_double2(0.0, 0.0), t2 = make_double2(0.0, 0.0);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                t1 = cfma(u[r * 3 + m], Pf[cc * 3 + m], t1);                       // (U Pf^T)[r][cc]
                t2 = cfma(Pb[m * 3 + r], make_double2(u[cc * 3 + m].x, -u[cc * 3 + m].y), t2);   // (Pb^T U^dag)[r][cc]
            }
            M[r * 3 + cc] = make_double2(-fp * t1.x + fm * t2.x, -fp * t1.y + fm * t2.y);
        }
    // Q = (i bs / 4) M;  Re tr(lambda_a Q) = -(bs/4) Im tr(lambda_a M)
    auto imtr = [&](int r0, int c0) { return M[c0 * 3 + r0].y; };        // Im of (lambda entry at (r0,c0)) x M[c0][r0]
    auto retr = [&](int r0, int c0) { return M[c0 * 3 + r0].x; };
    // tr(lambda M) = sum_{r,c} lambda[r][c] M[c][r]
    double im[8];
    im[0] = imtr(0, 1) + imtr(1, 0);                                      // lambda_1
    im[1] = retr(1, 0) - retr(0, 1);                                      // lambda_2: Im( -i M10 + i M01 ) ...
    im[2] = imtr(0, 0) - imtr(1, 1);                                      // lambda_3
    im[3] = imtr(0, 2) + imtr(2, 0);                                      // lambda_4
    im[4] = retr(2, 0) - retr(0, 2);                                      // lambda_5
    im[5] = imtr(1, 2) + imtr(2, 1);                                      // lambda_6
    im[6] = retr(2, 1) - retr(1, 2);                                      // lambda_7
    im[7] = (imtr(0, 0) + imtr(1, 1) - 2.0 * imtr(2, 2)) * 0.57735026918962576451;   // lambda_8
    double* out = a.force + ((size_t)NU * V + s) * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = -0.25 * bs * im[i];
    if (NU == 3) {
        // d/dmu: <omega| dH/dmu |nu> = -1/2 e^mu bs tr(U Pf^T) + 1/2 e^-mu bs tr(U^dag Pb^T)
        double2 trf = make_double2(0.0, 0.0), trb = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                trf = cfma(u[r * 3 + m], Pf[r * 3 + m], trf);                                       // sum U[r][m] Pf[r][m]
                trb = cfma(make_double2(u[m * 3 + r].x, -u[m * 3 + r].y), Pb[r * 3 + m], trb);     // sum conj(U[m][r]) Pb[r][m]
            }
        dmu_acc += bs * (-0.5 * a.efwd * trf.x + 0.5 * a.ebwd * trb.x);
    }
}

template <typename R>
__global__ void __launch_bounds__(128) k_force(AdjArgs a) {
    __shared__ double red[128];
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dmu = 0.0;
    if (s < a.V) {
        int x[4];
        unsigned r = (unsigned)s;
        x[0] = (int)(r % (unsigned)a.dims[0]); r /= (unsigned)a.dims[0];
        x[1] = (int)(r % (unsigned)a.dims[1]); r /= (unsigned)a.dims[1];
        x[2] = (int)(r % (unsigned)a.dims[2]); r /= (unsigned)a.dims[2];
        x[3] = (int)r;
        force_dir<R, 0>(a, s, x, dmu);
        force_dir<R, 1>(a, s, x, dmu);
        force_dir<R, 2>(a, s, x, dmu);
        force_dir<R, 3>(a, s, x, dmu);
    }
    red[threadIdx.x] = dmu;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.dmu_part[blockIdx.x] = red[0];
}

cudaError_t launch_adj_pairs(const AdjArgs& a, cudaStream_t st) {
    k_adj_pairs<<<1, 2 * a.npairs, 0, st>>>(a);
    return cudaGetLastError();
}

namespace {
// element counts of a field and the kernels' chunk type per precision
size_t adj_field_elems(int prec, size_t V) { return prec == LQ_MIXED ? field_elems<float>(V) : field_elems<double>(V); }

template <typename R>
cudaError_t adj_window_t(const AdjArgs& a, const void* basis, size_t bstride, const void* lbasis, size_t lstride, int j0,
                         int j1, int ring, size_t F, cudaStream_t st) {
    using Chunk = typename Tr<R>::Chunk;
    const dim3 grid((unsigned)((F + 127) / 128), (unsigned)((a.npairs + kQB - 1) / kQB));
    const int acc = j0 > 0 ? 1 : 0;
    k_recomb_window<R><<<grid, 128, 0, st>>>(reinterpret_cast<const Chunk*>(basis), bstride, j0, j1, ring, a.cnu, a.kmax,
                                             a.npairs, reinterpret_cast<Chunk*>(a.nu), F, acc);
    k_recomb_window<R><<<grid, 128, 0, st>>>(reinterpret_cast<const Chunk*>(lbasis), lstride, j0, j1, ring, a.com, a.kmax,
                                             a.npairs, reinterpret_cast<Chunk*>(a.om), F, acc);
    return cudaGetLastError();
}

template <typename R>
cudaError_t adjoint_t(const AdjArgs& a, const void* basis, size_t bstride, const void* lbasis, size_t lstride, int k,
                      size_t F, cudaStream_t st) {
    using Chunk = typename Tr<R>::Chunk;
    const dim3 grid((unsigned)((F + 127) / 128), (unsigned)((a.npairs + kQB - 1) / kQB));
    const size_t sm = (size_t)kQB * k * sizeof(double2);
    cudaFuncSetAttribute(k_recomb_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_recomb_multi<R><<<grid, 128, sm, st>>>(reinterpret_cast<const Chunk*>(basis), bstride, k, a.cnu, a.kmax, a.npairs,
                                             reinterpret_cast<Chunk*>(a.nu), F);
    k_recomb_multi<R><<<grid, 128, sm, st>>>(reinterpret_cast<const Chunk*>(lbasis), lstride, k, a.com, a.kmax, a.npairs,
                                             reinterpret_cast<Chunk*>(a.om), F);
    if (a.ndefl > 0) {
        const int nq = a.npairs, nd = a.ndefl;
        const dim3 gd((unsigned)((F + 127) / 128), (unsigned)((nd + kQB - 1) / kQB));
        k_defl_coef<<<1, 2 * nd, 0, st>>>(a);
        k_recomb_multi<R><<<gd, 128, sm, st>>>(reinterpret_cast<const Chunk*>(basis), bstride, k,
                                               a.cnu + (size_t)(nq + 2 * nd) * a.kmax, a.kmax, nd,
                                               reinterpret_cast<Chunk*>(a.nu) + (size_t)(nq + 2 * nd) * F, F);
        k_recomb_multi<R><<<gd, 128, sm, st>>>(reinterpret_cast<const Chunk*>(lbasis), lstride, k,
                                               a.com + (size_t)(nq + nd) * a.kmax, a.kmax, nd,
                                               reinterpret_cast<Chunk*>(a.om) + (size_t)(nq + nd) * F, F);
    }
    k_force<R><<<(unsigned)((a.V + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adj_window(int prec, const AdjArgs& a, const void* basis, size_t basis_vec_stride, const void* lbasis,
                              size_t lbasis_vec_stride, int j0, int j1, int ring, cudaStream_t st) {
    if (j1 - j0 > kTwoPassRing || j1 <= j0) return cudaErrorInvalidValue;
    const size_t F = adj_field_elems(prec, a.V);
    if (prec == LQ_FP64) return adj_window_t<double>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, j0, j1, ring, F, st);
    if (prec == LQ_FLOAT_FLOAT) return adj_window_t<ff>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, j0, j1, ring, F, st);
    return adj_window_t<float>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, j0, j1, ring, F, st);
}

cudaError_t launch_adj_force(int prec, const AdjArgs& a, cudaStream_t st) {
    const unsigned g = (unsigned)((a.V + 127) / 128);
    if (prec == LQ_FP64) k_force<double><<<g, 128, 0, st>>>(a);
    else if (prec == LQ_FLOAT_FLOAT) k_force<ff><<<g, 128, 0, st>>>(a);
    else k_force<float><<<g, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(int prec, const AdjArgs& a, const void* basis, size_t basis_vec_stride, const void* lbasis,
                           size_t lbasis_vec_stride, int k, cudaStream_t st) {
    k_adj_pairs<<<1, 2 * a.npairs, 0, st>>>(a);
    const size_t F = adj_field_elems(prec, a.V);
    if (prec == LQ_FP64) return adjoint_t<double>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, k, F, st);
    if (prec == LQ_FLOAT_FLOAT) return adjoint_t<ff>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, k, F, st);
    return adjoint_t<float>(a, basis, basis_vec_stride, lbasis, lbasis_vec_stride, k, F, st);
}

}  // namespace lq
