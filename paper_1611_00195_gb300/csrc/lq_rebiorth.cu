// Periodic re-biorthogonalisation of the two-sided Lanczos process (Sec. 2).  In finite precision
// the new pair (vh_{j+1}, wh_{j+1}) of the three-term recurrences slowly loses its
// biorthogonality to the earlier pairs; with lq_opts.rebiorth = p, the pairs of two consecutive
// updates per period (steps j with j + 1 or j a multiple of p) are projected against all j + 1
// earlier pairs before omega_j is formed:
//     vh <- vh - sum_i v_i <w_i, vh>,    wh <- wh - sum_i w_i <v_i, wh>,    i = 0 .. j,
// with v_i = s_i vh_i and w_i = u_i wh_i the stored (unnormalised) vectors and their scales.  T
// keeps its three-term entries.  Three launches per correction, in every precision of the
// library:
//   k_rb_dots   the 2 (j + 1) inner products per source, each thread holding a few chunks of the
//               new pair in registers while it streams the earlier vectors; fixed-order block sums;
//   k_rb_coef   the block sums reduced in a fixed order into the coefficients
//               c_i = s_i conj(u_i) <wh_i, vh> and d_i = s_i u_i <vh_i, wh>;
//   k_rb_apply  the two corrections (float-float sums for FP32 data), the stored copies of the new
//               pair, omega and the norms, and (last block) the scalar step the update left to it
//               (UpdArgs.defer).
// Inner products are accumulated as the update's are (compensated FP64, float-float for FP32 and
// float-float data).  A correction reads the 2 (j + 1) earlier vectors twice: O(j n) bytes.
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

#include <algorithm>

namespace lq {
namespace {

// re + i im += <w, v> over the complex numbers of one chunk
__device__ __forceinline__ void rb_cdot(DotAcc<double>& re, DotAcc<double>& im, double2 w, double2 v) {
    add_cdot(re, im, w, v);
}
__device__ __forceinline__ void rb_cdot(DotAcc<float>& re, DotAcc<float>& im, float4 w, float4 v) {
    add_cdot(re, im, make_float2(w.x, w.y), make_float2(v.x, v.y));
    add_cdot(re, im, make_float2(w.z, w.w), make_float2(v.z, v.w));
}
__device__ __forceinline__ void rb_cdot(DotAcc<ff>& re, DotAcc<ff>& im, float4 w, float4 v) {
    add_cdot(re, im, cff_from_chunk(w), cff_from_chunk(v));
}

// The corrected chunk x - sum_i c_i b_i, accumulated over i in the data's own type for FP64 and
// float-float data and in float-float for FP32 data (rounded once to FP32 when stored): the terms
// can exceed the result by the condition |v_i| |w_i| of the biorthogonal pairs (1e4 and more on
// the Wilson kernel at mu > 0), and an FP32 rounding of every term would add more error than the
// correction removes.  c_i comes as the FP64 coefficient or its float-float split (re.hi, re.lo,
// im.hi, im.lo).
template <typename R> struct RbAcc;
template <> struct RbAcc<double> {
    double2 v;
    __device__ __forceinline__ void load(double2 x) { v = x; }
    __device__ __forceinline__ void sub(double2 b, double2 c, float4) { v = cfma(make_double2(-c.x, -c.y), b, v); }
    __device__ __forceinline__ double2 get() const { return v; }
};
template <> struct RbAcc<float> {
    cff a, b;   // the chunk's two complex numbers
    __device__ __forceinline__ void load(float4 x) {
        a.x = ff(x.x); a.y = ff(x.y);
        b.x = ff(x.z); b.y = ff(x.w);
    }
    __device__ __forceinline__ void sub(float4 q, double2, float4 f) {
        cff c, q0, q1;
        c.x = ff(-f.x, -f.y); c.y = ff(-f.z, -f.w);
        q0.x = ff(q.x); q0.y = ff(q.y);
        q1.x = ff(q.z); q1.y = ff(q.w);
        a = cfma(c, q0, a);
        b = cfma(c, q1, b);
    }
    __device__ __forceinline__ float4 get() const {
        return make_float4(a.x.hi + a.x.lo, a.y.hi + a.y.lo, b.x.hi + b.x.lo, b.y.hi + b.y.lo);
    }
};
template <> struct RbAcc<ff> {
    cff v;
    __device__ __forceinline__ void load(float4 x) { v = cff_from_chunk(x); }
    __device__ __forceinline__ void sub(float4 q, double2, float4 f) {
        cff c;
        c.x = ff(-f.x, -f.y); c.y = ff(-f.z, -f.w);
        v = cfma(c, cff_from_chunk(q), v);
    }
    __device__ __forceinline__ float4 get() const { return cff_to_chunk(v); }
};

template <typename R>
__global__ void __launch_bounds__(kRbThreads) k_rb_dots(RbArgs a) {
    using Chunk = typename Tr<R>::Chunk;
    __shared__ CSum smem[32 * 4];
    const int src = blockIdx.y;
    if (a.u.state[src].status != 0) return;   // block-uniform
    const size_t N = a.u.nelem;
    const Chunk* vn = reinterpret_cast<const Chunk*>(a.u.v_next) + (size_t)src * a.u.src_stride_basis;
    const Chunk* wn = reinterpret_cast<const Chunk*>(a.u.w_next) + (size_t)src * a.u.src_stride_left;
    const Chunk* vb = reinterpret_cast<const Chunk*>(a.vbasis) + (size_t)src * a.u.src_stride_basis;
    const Chunk* wb = reinterpret_cast<const Chunk*>(a.wbasis) + (size_t)src * a.u.src_stride_store;
    // element q of this thread: e0 + q span; the grid (rb_dot_blocks) covers N with kRbPerThread
    const size_t span = (size_t)gridDim.x * kRbThreads;
    const size_t e0 = (size_t)blockIdx.x * kRbThreads + threadIdx.x;
    const Chunk zero{};
    Chunk x[kRbPerThread], y[kRbPerThread];
#pragma unroll
    for (int q = 0; q < kRbPerThread; ++q) {
        const size_t e = e0 + q * span;
        x[q] = e < N ? vn[e] : zero;
        y[q] = e < N ? wn[e] : zero;
    }
    for (int i = 0; i < a.m; ++i) {
        const Chunk* vi = vb + (size_t)i * a.vec_stride;
        const Chunk* wi = wb + (size_t)i * a.vec_stride;
        DotAcc<R> d[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) d[t].zero();
#pragma unroll
        for (int q = 0; q < kRbPerThread; ++q) {
            const size_t e = e0 + q * span;
            if (e < N) {
                rb_cdot(d[0], d[1], __ldg(wi + e), x[q]);   // <wh_i, vh_new>
                rb_cdot(d[2], d[3], __ldg(vi + e), y[q]);   // <vh_i, wh_new>
            }
        }
        CSum tot[4];
        block_total<R, 4>(d, tot, smem);
        if (threadIdx.x == 0) {
            double* p = a.part + (((size_t)src * a.u.kmax + i) * a.dot_blocks + blockIdx.x) * 8;
#pragma unroll
            for (int t = 0; t < 4; ++t) { p[2 * t] = tot[t].s; p[2 * t + 1] = tot[t].e; }
        }
    }
}

__global__ void __launch_bounds__(kRbThreads) k_rb_coef(RbArgs a) {
    const int src = blockIdx.x;
    if (a.u.state[src].status != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t km = a.u.kmax;
    for (int i = warp; i < a.m; i += kRbThreads / 32) {   // warp-uniform: every lane shuffles
        CSum acc[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) { acc[t].s = 0.0; acc[t].e = 0.0; }
        const double* p = a.part + ((size_t)src * km + i) * a.dot_blocks * 8;
        for (unsigned b = lane; b < a.dot_blocks; b += 32)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                CSum v;
                v.s = __ldcg(p + (size_t)b * 8 + 2 * t);
                v.e = __ldcg(p + (size_t)b * 8 + 2 * t + 1);
                acc[t] = cs_merge(acc[t], v);
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[t] = cs_merge(acc[t], cs_shfl_down(acc[t], off));
        if (lane == 0) {
            const double2 av = make_double2(acc[0].s + acc[0].e, acc[1].s + acc[1].e);   // <wh_i, vh_new>
            const double2 bw = make_double2(acc[2].s + acc[2].e, acc[3].s + acc[3].e);   // <vh_i, wh_new>
            const double s = a.scale[src * km + i];
            const double2 u = a.uscale[src * km + i];
            // v_i <w_i, vh> = s_i conj(u_i) <wh_i, vh> vh_i;  w_i <v_i, wh> = u_i s_i <vh_i, wh> wh_i
            const double2 c = make_double2(s * (u.x * av.x + u.y * av.y), s * (u.x * av.y - u.y * av.x));
            const double2 d = make_double2(s * (u.x * bw.x - u.y * bw.y), s * (u.x * bw.y + u.y * bw.x));
            a.coef[(2 * (size_t)src) * km + i] = c;
            a.coef[(2 * (size_t)src + 1) * km + i] = d;
            const ff cx(c.x), cy(c.y), dx(d.x), dy(d.y);
            a.coef_f[(2 * (size_t)src) * km + i] = make_float4(cx.hi, cx.lo, cy.hi, cy.lo);
            a.coef_f[(2 * (size_t)src + 1) * km + i] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kRbThreads) k_rb_apply(RbArgs a) {
    using Chunk = typename Tr<R>::Chunk;
    __shared__ CSum smem[32 * 6];
    const int src = blockIdx.y;
    TslState& st = a.u.state[src];
    if (st.status != 0) return;
    const size_t N = a.u.nelem;
    const size_t km = a.u.kmax;
    Chunk* vn = reinterpret_cast<Chunk*>(a.u.v_next) + (size_t)src * a.u.src_stride_basis;
    Chunk* wn = reinterpret_cast<Chunk*>(a.u.w_next) + (size_t)src * a.u.src_stride_left;
    Chunk* ws = reinterpret_cast<Chunk*>(a.u.w_store) + (size_t)src * a.u.src_stride_store;
    const Chunk* vb = reinterpret_cast<const Chunk*>(a.vbasis) + (size_t)src * a.u.src_stride_basis;
    const Chunk* wb = reinterpret_cast<const Chunk*>(a.wbasis) + (size_t)src * a.u.src_stride_store;
    const double2* cr = a.coef + 2 * (size_t)src * km;
    const double2* cl = cr + km;
    const float4* fr = a.coef_f + 2 * (size_t)src * km;
    const float4* fl = fr + km;
    DotAcc<R> d[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) d[t].zero();
    const size_t stride = (size_t)gridDim.x * kRbThreads;
    for (size_t e = (size_t)blockIdx.x * kRbThreads + threadIdx.x; e < N; e += stride) {
        RbAcc<R> ax, ay;
        ax.load(vn[e]);
        ay.load(wn[e]);
        for (int i = 0; i < a.m; ++i) {
            ax.sub(__ldg(vb + (size_t)i * a.vec_stride + e), __ldg(cr + i), __ldg(fr + i));
            ay.sub(__ldg(wb + (size_t)i * a.vec_stride + e), __ldg(cl + i), __ldg(fl + i));
        }
        const Chunk x = ax.get(), y = ay.get();
        vn[e] = x;
        wn[e] = y;
        ws[e] = y;
        dot_chunk<R>(d, y, x);   // omega = <wh, vh>, |vh|^2, |wh|^2
    }
    CSum tot[6];
    block_total<R, 6>(d, tot, smem);
    double* part = a.u.partials + ((size_t)src * a.u.partial_stride + blockIdx.x) * 12;
    if (threadIdx.x == 0)
        for (int t = 0; t < 6; ++t) { part[2 * t] = tot[t].s; part[2 * t + 1] = tot[t].e; }
    if (last_block(a.u.counters + a.u.nsrc + src, gridDim.x)) {
        double res[6];
        reduce_partials<6>(a.u.partials + (size_t)src * a.u.partial_stride * 12, gridDim.x, res, smem);
        if (threadIdx.x == 0) {
            res[4] = st.rb_nr;   // |B vh_j|^2, |B^dag wh_j|^2 from the update
            res[5] = st.rb_nl;
            update_scalars<R>(a.u, src, res);
        }
    }
}

template <typename R>
cudaError_t rebiorth_t(const RbArgs& a, cudaStream_t st) {
    const unsigned nb = rb_dot_blocks(a.u.nelem);
    k_rb_dots<R><<<dim3(nb, (unsigned)a.u.nsrc), kRbThreads, 0, st>>>(a);
    k_rb_coef<<<(unsigned)a.u.nsrc, kRbThreads, 0, st>>>(a);
    const size_t want = (a.u.nelem + kRbThreads - 1) / kRbThreads;
    const unsigned na = (unsigned)std::max<size_t>(1, std::min(want, a.u.partial_stride));
    k_rb_apply<R><<<dim3(na, (unsigned)a.u.nsrc), kRbThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rebiorth(int prec, const RbArgs& a, cudaStream_t st) {
    if (a.m < 1 || a.dot_blocks != rb_dot_blocks(a.u.nelem)) return cudaErrorInvalidValue;
    if (prec == LQ_FP64) return rebiorth_t<double>(a, st);
    if (prec == LQ_FLOAT_FLOAT) return rebiorth_t<ff>(a, st);
    return rebiorth_t<float>(a, st);
}

}  // namespace lq
