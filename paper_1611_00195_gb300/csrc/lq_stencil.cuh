// Device helpers shared by the stencil kernels of the two-sided Lanczos path: compensated
// accumulators for the inner products, block / grid reductions, and the spin-colour algebra of
// one Wilson hop (projection to half spinors, SU(3) multiply, reconstruction).
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "lq_internal.cuh"
#include "lq_launch.h"

namespace lq {

// ---------------------------------------------------------------------------------------
// float-float accumulator with exact products (for FP32 data); double CSum for FP64 data
// ---------------------------------------------------------------------------------------
struct FF { float h, l; };
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
    s = a + b;
    float z = s - a;
    t = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void ff_add_prod(FF& acc, float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float s, t;
    two_sum_f(acc.h, p, s, t);
    acc.h = s;
    acc.l += t + pe;
}
__device__ __forceinline__ FF ff_merge(FF a, FF b) {
    float s, t;
    two_sum_f(a.h, b.h, s, t);
    FF r; r.h = s; r.l = a.l + b.l + t;
    return r;
}

template <typename R> struct DotAcc;
template <> struct DotAcc<double> {
    CSum v;
    __device__ __forceinline__ void zero() { v.s = 0.0; v.e = 0.0; }
    __device__ __forceinline__ void add_prod(double a, double b) { cs_add_prod(v, a, b); }
    // a plain FMA term (for sums that only feed a threshold: the compensation, several FP64
    // operations per term, is what bounds the FP64 update on this GPU)
    __device__ __forceinline__ void add_plain(double a, double b) { v.s = fma(a, b, v.s); }
    // warp-level reduction then conversion to a double compensated sum (valid in lane 0)
    __device__ __forceinline__ CSum warp_total() {
        CSum r = v;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r = cs_merge(r, cs_shfl_down(r, off));
        return r;
    }
};
template <> struct DotAcc<float> {
    FF v;
    __device__ __forceinline__ void zero() { v.h = 0.f; v.l = 0.f; }
    __device__ __forceinline__ void add_prod(float a, float b) { ff_add_prod(v, a, b); }
    // a plain FMA term (sums that only feed a threshold)
    __device__ __forceinline__ void add_plain(float a, float b) { v.h = fmaf(a, b, v.h); }
    __device__ __forceinline__ CSum warp_total() {   // valid in lane 0 only
        FF r = v;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            FF o; o.h = __shfl_down_sync(0xffffffffu, r.h, off); o.l = __shfl_down_sync(0xffffffffu, r.l, off);
            r = ff_merge(r, o);
        }
        CSum c{0.0, 0.0};
        if ((threadIdx.x & 31) == 0) { c.s = (double)r.h; c.e = (double)r.l; }
        return c;
    }
};

// float-float data: float-float products added into a float-float accumulator (FP32 operations
// only, as for FP32 data)
template <> struct DotAcc<ff> {
    FF v;
    __device__ __forceinline__ void zero() { v.h = 0.f; v.l = 0.f; }
    __device__ __forceinline__ void add_prod(ff a, ff b) {
        const ff p = a * b;
        float s, t;
        two_sum_f(v.h, p.hi, s, t);
        v.h = s;
        v.l += t + p.lo;
    }
    __device__ __forceinline__ void add_plain(ff a, ff b) { v.h = fmaf(a.hi, b.hi, v.h); }
    __device__ __forceinline__ CSum warp_total() {   // valid in lane 0 only
        FF r = v;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            FF o; o.h = __shfl_down_sync(0xffffffffu, r.h, off); o.l = __shfl_down_sync(0xffffffffu, r.l, off);
            r = ff_merge(r, o);
        }
        CSum c{0.0, 0.0};
        if ((threadIdx.x & 31) == 0) { c.s = (double)r.h; c.e = (double)r.l; }
        return c;
    }
};

// re += Re conj(w) a, im += Im conj(w) a.  FP64: each complex term is formed with one product
// and one FMA and then added by a compensated two-sum, so the long sums over sites and elements
// stay compensated while a term costs a few FP64 operations instead of two exact products (FP64
// is slow on this GPU).  FP32: exact products in float-float.
__device__ __forceinline__ void add_cdot(DotAcc<double>& re, DotAcc<double>& im, double2 w, double2 a) {
    cs_add(re.v, fma(w.x, a.x, w.y * a.y));
    cs_add(im.v, fma(w.x, a.y, -(w.y * a.x)));
}
__device__ __forceinline__ void add_cdot(DotAcc<float>& re, DotAcc<float>& im, float2 w, float2 a) {
    re.add_prod(w.x, a.x); re.add_prod(w.y, a.y);
    im.add_prod(w.x, a.y); im.add_prod(-w.y, a.x);
}
__device__ __forceinline__ void add_cdot(DotAcc<ff>& re, DotAcc<ff>& im, cff w, cff a) {
    re.add_prod(w.x, a.x); re.add_prod(w.y, a.y);
    im.add_prod(w.x, a.y); im.add_prod(-w.y, a.x);
}

// Reduce NV per-thread accumulators to one compensated double per value for the block.
// Valid in thread 0.  smem holds 32 * NV CSum.  FP32 data stays in float-float up to the block
// total (one conversion per value in thread 0): FP64 is slow on this GPU and has no place in the
// body of an FP32 kernel.
template <typename R, int NV>
__device__ __forceinline__ void block_total(DotAcc<R> (&acc)[NV], CSum (&out)[NV], CSum* smem) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if constexpr (sizeof(R) == 4) {
        FF* fs = reinterpret_cast<FF*>(smem);
        FF w[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            FF r = acc[i].v;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                FF o; o.h = __shfl_down_sync(0xffffffffu, r.h, off); o.l = __shfl_down_sync(0xffffffffu, r.l, off);
                r = ff_merge(r, o);
            }
            w[i] = r;
        }
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < NV; ++i) fs[warp * NV + i] = w[i];
        __syncthreads();
        if (threadIdx.x == 0)
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                FF t = fs[i];
                for (int v = 1; v < nw; ++v) t = ff_merge(t, fs[v * NV + i]);
                out[i].s = (double)t.h;
                out[i].e = (double)t.l;
            }
        __syncthreads();
    } else {
        CSum w[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) w[i] = acc[i].warp_total();
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < NV; ++i) smem[warp * NV + i] = w[i];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                if (lane < nw) w[i] = smem[lane * NV + i];
                else { w[i].s = 0.0; w[i].e = 0.0; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int i = 0; i < NV; ++i) w[i] = cs_merge(w[i], cs_shfl_down(w[i], off));
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < NV; ++i) out[i] = w[i];
        }
        __syncthreads();
    }
}

// "Last block done" election: every block of a source publishes its partials, then the
// block that finishes last (atomic counter) reduces them.  Returns true in that block.
__device__ __forceinline__ bool last_block(int* counter, int nblocks) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int prev = atomicAdd(counter, 1);
        is_last = (prev == nblocks - 1);
        if (is_last) *counter = 0;   // reset for the next launch
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// Sum nb partials (stride NV values of (s, e) pairs) in a fixed order -> deterministic.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int nb, double (&res)[NV], CSum* smem) {
    CSum acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) { acc[i].s = 0.0; acc[i].e = 0.0; }
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            CSum p; p.s = __ldcg(part + (size_t)b * 2 * NV + 2 * i); p.e = __ldcg(part + (size_t)b * 2 * NV + 2 * i + 1);
            acc[i] = cs_merge(acc[i], p);
        }
    block_reduce_cs<NV>(acc, smem);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) res[i] = acc[i].s + acc[i].e;
}

// ---------------------------------------------------------------------------------------
// Spin structure in the chiral basis: gamma_nu = [[0, B_nu], [B_nu^dag, 0]] with
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.  Then
// (1 + s gamma_nu) psi = (h, s B^dag h) with h = psi_up + s B psi_dn  (s = +-1),
// so every hop only needs the two-component half spinor h (Wilson projector, r = 1).
// ---------------------------------------------------------------------------------------
template <typename C, int NU, int SP>
__device__ __forceinline__ void project(const C (&p)[12], C (&h)[6]) {
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        C u0 = p[col], u1 = p[3 + col], d2 = p[6 + col], d3 = p[9 + col];
        C b0, b1;
        if (NU == 0) { b0 = cmul_mi(d3); b1 = cmul_mi(d2); }
        else if (NU == 1) { b0 = cmk<C>(-d3.x, -d3.y); b1 = d2; }
        else if (NU == 2) { b0 = cmul_mi(d2); b1 = cmul_i(d3); }
        else { b0 = d2; b1 = d3; }
        if (SP > 0) { h[col] = cadd(u0, b0); h[3 + col] = cadd(u1, b1); }
        else { h[col] = csub(u0, b0); h[3 + col] = csub(u1, b1); }
    }
}

// Float-float accumulator step a += s b (s = +-1) without renormalising: TwoSum of the high
// parts, the rest into the low part.  The accumulators of a site's output spinor take eight such
// steps per component and are renormalised once, in finish(), by its float-float FMA.
template <bool NEG>
__device__ __forceinline__ void ff_acc_add(ff& a, ff b) {
    float s, t;
    two_sum_f(a.hi, NEG ? -b.hi : b.hi, s, t);
    a.hi = s;
    a.lo += t + (NEG ? -b.lo : b.lo);
}

// acc += (g, s B^dag g)
template <typename C, int NU, int SP>
__device__ __forceinline__ void reconstruct_add(const C (&g)[6], C (&acc)[12]) {
    if constexpr (std::is_same_v<C, cff>) {
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            const cff g0 = g[col], g1 = g[3 + col];
            cff l0, l1;   // B^dag g
            if (NU == 0) { l0 = cmul_i(g1); l1 = cmul_i(g0); }
            else if (NU == 1) { l0 = g1; l1 = cmk<cff>(-g0.x, -g0.y); }
            else if (NU == 2) { l0 = cmul_i(g0); l1 = cmul_mi(g1); }
            else { l0 = g0; l1 = g1; }
            ff_acc_add<false>(acc[col].x, g0.x); ff_acc_add<false>(acc[col].y, g0.y);
            ff_acc_add<false>(acc[3 + col].x, g1.x); ff_acc_add<false>(acc[3 + col].y, g1.y);
            ff_acc_add<(SP < 0)>(acc[6 + col].x, l0.x); ff_acc_add<(SP < 0)>(acc[6 + col].y, l0.y);
            ff_acc_add<(SP < 0)>(acc[9 + col].x, l1.x); ff_acc_add<(SP < 0)>(acc[9 + col].y, l1.y);
        }
        return;
    }
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        C g0 = g[col], g1 = g[3 + col];
        C l0, l1;   // B^dag g
        if (NU == 0) { l0 = cmul_i(g1); l1 = cmul_i(g0); }
        else if (NU == 1) { l0 = g1; l1 = cmk<C>(-g0.x, -g0.y); }
        else if (NU == 2) { l0 = cmul_i(g0); l1 = cmul_mi(g1); }
        else { l0 = g0; l1 = g1; }
        acc[col] = cadd(acc[col], g0);
        acc[3 + col] = cadd(acc[3 + col], g1);
        if (SP > 0) { acc[6 + col] = cadd(acc[6 + col], l0); acc[9 + col] = cadd(acc[9 + col], l1); }
        else { acc[6 + col] = csub(acc[6 + col], l0); acc[9 + col] = csub(acc[9 + col], l1); }
    }
}

// Float-float accumulation of a sum of products without renormalising after every term: the
// high parts of the exact products (one product and one FMA each) are added by TwoSum into s,
// everything of order u |term| (the products' errors, the cross terms hi * lo, the TwoSum
// errors) into e in FP32; one TwoSum of (s, e) at the end.  Twelve FP32 operations per real
// product instead of about twenty-six for a float-float multiply followed by an add.
struct FFSum {
    float s, e;
};
template <bool NEG>
__device__ __forceinline__ void ffsum_add_prod(FFSum& a, ff x, ff y) {
    float p = x.hi * y.hi;
    float pe = fmaf(x.hi, y.hi, -p);
    pe = fmaf(x.hi, y.lo, pe);
    pe = fmaf(x.lo, y.hi, pe);
    if (NEG) { p = -p; pe = -pe; }
    float s, t;
    two_sum_f(a.s, p, s, t);
    a.s = s;
    a.e += t + pe;
}

template <typename C, bool DAG>
__device__ __forceinline__ void su3_mul(const C (&u)[9], const C (&h)[6], C (&g)[6]) {
    if constexpr (std::is_same_v<C, cff>) {
        // float-float: each output component as one FFSum over its six real products
#pragma unroll
        for (int sc = 0; sc < 2; ++sc)
#pragma unroll
            for (int row = 0; row < 3; ++row) {
                FFSum re{0.f, 0.f}, im{0.f, 0.f};
#pragma unroll
                for (int col = 0; col < 3; ++col) {
                    const cff uu = DAG ? u[col * 3 + row] : u[row * 3 + col];
                    const cff hh = h[sc * 3 + col];
                    // U h: (ux hx - uy hy, ux hy + uy hx);  U^dag h: (ux hx + uy hy, ux hy - uy hx)
                    ffsum_add_prod<false>(re, uu.x, hh.x);
                    ffsum_add_prod<!DAG>(re, uu.y, hh.y);
                    ffsum_add_prod<false>(im, uu.x, hh.y);
                    ffsum_add_prod<DAG>(im, uu.y, hh.x);
                }
                g[sc * 3 + row].x = ff_two_sum(re.s, re.e);
                g[sc * 3 + row].y = ff_two_sum(im.s, im.e);
            }
        return;
    }
#pragma unroll
    for (int sc = 0; sc < 2; ++sc)
#pragma unroll
        for (int row = 0; row < 3; ++row) {
            C a = cmk<C>(0, 0);
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                if (!DAG) a = cfma(u[row * 3 + col], h[sc * 3 + col], a);
                else a = cfmac(u[col * 3 + row], h[sc * 3 + col], a);
            }
            g[sc * 3 + row] = a;
        }
}

template <typename C>
__device__ __forceinline__ void load_link(const C* __restrict__ L, size_t V, int nu, size_t s, C (&u)[9]) {
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = __ldg(L + ((size_t)nu * 9 + e) * V + s);
}
__device__ __forceinline__ void load_link(const cff* __restrict__ L, size_t V, int nu, size_t s, cff (&u)[9]) {
    const float4* L4 = reinterpret_cast<const float4*>(L);
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = cff_from_chunk(__ldg(L4 + ((size_t)nu * 9 + e) * V + s));
}
// The gauge links of the operator: FP32 or FP64 entries, or BF16 pairs widened to FP32.
__device__ __forceinline__ void load_gauge(const HopArgs& a, size_t V, int nu, size_t s, double2 (&u)[9]) {
    load_link(reinterpret_cast<const double2*>(a.U), V, nu, s, u);
}
__device__ __forceinline__ void load_gauge(const HopArgs& a, size_t V, int nu, size_t s, cff (&u)[9]) {
    load_link(reinterpret_cast<const cff*>(a.U), V, nu, s, u);
}
__device__ __forceinline__ void load_gauge(const HopArgs& a, size_t V, int nu, size_t s, float2 (&u)[9]) {
    if (a.link_bf16) {
        const __nv_bfloat162* L = reinterpret_cast<const __nv_bfloat162*>(a.U);
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = __bfloat1622float2(__ldg(L + ((size_t)nu * 9 + e) * V + s));
    } else {
        load_link(reinterpret_cast<const float2*>(a.U), V, nu, s, u);
    }
}

template <typename C>
__device__ __forceinline__ void hscale(C (&h)[6], decltype(C::x) f) {
#pragma unroll
    for (int i = 0; i < 6; ++i) h[i] = cscale(h[i], f);
}
template <typename C>
__device__ __forceinline__ void haxpy(C (&h)[6], decltype(C::x) f, const C (&x)[6]) {  // h += f x
#pragma unroll
    for (int i = 0; i < 6; ++i) { h[i].x = fma(f, x[i].x, h[i].x); h[i].y = fma(f, x[i].y, h[i].y); }
}

// Hop factors in the kernel's precision (FP32 copies are prepared on the host).
template <typename R> __device__ __forceinline__ R fac_a(const HopArgs& a, int side, int nu, bool fwd);
template <> __device__ __forceinline__ double fac_a<double>(const HopArgs& a, int side, int nu, bool fwd) { return fwd ? a.a_fwd[side][nu] : a.a_bwd[side][nu]; }
template <> __device__ __forceinline__ float fac_a<float>(const HopArgs& a, int side, int nu, bool fwd) { return fwd ? a.af_fwd[side][nu] : a.af_bwd[side][nu]; }
template <typename R> __device__ __forceinline__ R fac_e(const HopArgs& a, int side, int nu, bool fwd);
template <> __device__ __forceinline__ double fac_e<double>(const HopArgs& a, int side, int nu, bool fwd) { return fwd ? a.e_fwd[side][nu] : a.e_bwd[side][nu]; }
template <> __device__ __forceinline__ float fac_e<float>(const HopArgs& a, int side, int nu, bool fwd) { return fwd ? a.ef_fwd[side][nu] : a.ef_bwd[side][nu]; }
template <typename R> __device__ __forceinline__ R fac_diag(const HopArgs& a);
template <> __device__ __forceinline__ double fac_diag<double>(const HopArgs& a) { return a.diag; }
template <> __device__ __forceinline__ float fac_diag<float>(const HopArgs& a) { return a.diag_f; }
template <> __device__ __forceinline__ ff fac_a<ff>(const HopArgs& a, int side, int nu, bool fwd) { return ff(fwd ? a.a_fwd[side][nu] : a.a_bwd[side][nu]); }
template <> __device__ __forceinline__ ff fac_e<ff>(const HopArgs& a, int side, int nu, bool fwd) { return ff(fwd ? a.e_fwd[side][nu] : a.e_bwd[side][nu]); }
template <> __device__ __forceinline__ ff fac_diag<ff>(const HopArgs& a) { return ff(a.diag); }

// Site coordinates (x, y, z, t) from the linear site index (32-bit arithmetic: V < 2^31).
__device__ __forceinline__ void site_coords(const HopArgs& a, size_t s, int (&x)[4]) {
    unsigned r = (unsigned)s;
    const unsigned d0 = (unsigned)a.dims[0], d1 = (unsigned)a.dims[1], d2 = (unsigned)a.dims[2];
    unsigned q = r / d0; x[0] = (int)(r - q * d0); r = q;
    q = r / d1; x[1] = (int)(r - q * d1); r = q;
    q = r / d2; x[2] = (int)(r - q * d2);
    x[3] = (int)q;
}


// gamma5 [diag * psi + acc]
template <typename C>
__device__ __forceinline__ void finish(const C (&psi)[12], decltype(C::x) diag, C (&acc)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        C v = cmk<C>(fma(diag, psi[c].x, acc[c].x), fma(diag, psi[c].y, acc[c].y));
        acc[c] = (c < 6) ? v : cmk<C>(-v.x, -v.y);
    }
}

// ---------------------------------------------------------------------------------------
// Update step of the Lanczos recurrences (Sec. 2): elementwise part and the scalar step that
// the last block of a source takes once omega, |vh|^2, |wh|^2, |B vh|^2, |B^dag wh|^2 are summed.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ typename Tr<R>::Chunk axpy3(typename Tr<R>::Chunk r, typename Tr<R>::Chunk v, typename Tr<R>::Chunk p,
                                                      const typename Tr<R>::C (&c)[3], bool has_prev);

template <>
__device__ __forceinline__ double2 axpy3<double>(double2 r, double2 v, double2 p, const double2 (&c)[3], bool has_prev) {
    double2 o = cmul(c[0], r);
    o = cfma(c[1], v, o);
    if (has_prev) o = cfma(c[2], p, o);
    return o;
}
template <>
__device__ __forceinline__ float4 axpy3<float>(float4 r, float4 v, float4 p, const float2 (&c)[3], bool has_prev) {
    float2 o0 = cmul(c[0], make_float2(r.x, r.y));
    float2 o1 = cmul(c[0], make_float2(r.z, r.w));
    o0 = cfma(c[1], make_float2(v.x, v.y), o0);
    o1 = cfma(c[1], make_float2(v.z, v.w), o1);
    if (has_prev) {
        o0 = cfma(c[2], make_float2(p.x, p.y), o0);
        o1 = cfma(c[2], make_float2(p.z, p.w), o1);
    }
    return make_float4(o0.x, o0.y, o1.x, o1.y);
}

template <>
__device__ __forceinline__ float4 axpy3<ff>(float4 r, float4 v, float4 p, const cff (&c)[3], bool has_prev) {
    const cff rr = cff_from_chunk(r), vv = cff_from_chunk(v);
    cff o = cmul(c[0], rr);
    o = cfma(c[1], vv, o);
    if (has_prev) o = cfma(c[2], cff_from_chunk(p), o);
    return cff_to_chunk(o);
}

template <typename R>
__device__ __forceinline__ void dot_chunk(DotAcc<R> (&d)[6], typename Tr<R>::Chunk w, typename Tr<R>::Chunk v);
// omega = <w, v> compensated over the elements (it becomes delta_j and beta_j); the norms
// |v|^2, |w|^2 only set the breakdown thresholds and are summed plainly
template <>
__device__ __forceinline__ void dot_chunk<double>(DotAcc<double> (&d)[6], double2 w, double2 v) {
    add_cdot(d[0], d[1], w, v);
    d[2].add_plain(v.x, v.x); d[2].add_plain(v.y, v.y);
    d[3].add_plain(w.x, w.x); d[3].add_plain(w.y, w.y);
}
template <>
__device__ __forceinline__ void dot_chunk<float>(DotAcc<float> (&d)[6], float4 w, float4 v) {
    d[0].add_prod(w.x, v.x); d[0].add_prod(w.y, v.y); d[0].add_prod(w.z, v.z); d[0].add_prod(w.w, v.w);
    d[1].add_prod(w.x, v.y); d[1].add_prod(-w.y, v.x); d[1].add_prod(w.z, v.w); d[1].add_prod(-w.w, v.z);
    d[2].add_plain(v.x, v.x); d[2].add_plain(v.y, v.y); d[2].add_plain(v.z, v.z); d[2].add_plain(v.w, v.w);
    d[3].add_plain(w.x, w.x); d[3].add_plain(w.y, w.y); d[3].add_plain(w.z, w.z); d[3].add_plain(w.w, w.w);
}
template <>
__device__ __forceinline__ void dot_chunk<ff>(DotAcc<ff> (&d)[6], float4 w4, float4 v4) {
    const cff w = cff_from_chunk(w4), v = cff_from_chunk(v4);
    add_cdot(d[0], d[1], w, v);
    d[2].add_plain(v.x, v.x); d[2].add_plain(v.y, v.y);
    d[3].add_plain(w.x, w.x); d[3].add_plain(w.y, w.y);
}
// |B vh_j|^2 (d[4]) and |B^dag wh_j|^2 (d[5]): the scale against which an invariant subspace is
// detected (plain sums, thresholds only)
__device__ __forceinline__ void norm_chunk(DotAcc<double> (&d)[6], double2 r, double2 l) {
    d[4].add_plain(r.x, r.x); d[4].add_plain(r.y, r.y);
    d[5].add_plain(l.x, l.x); d[5].add_plain(l.y, l.y);
}
__device__ __forceinline__ void norm_chunk(DotAcc<ff> (&d)[6], float4 r, float4 l) {
    d[4].add_plain(ff(r.x), ff(r.x)); d[4].add_plain(ff(r.z), ff(r.z));
    d[5].add_plain(ff(l.x), ff(l.x)); d[5].add_plain(ff(l.z), ff(l.z));
}
__device__ __forceinline__ void norm_chunk(DotAcc<float> (&d)[6], float4 r, float4 l) {
    d[4].add_plain(r.x, r.x); d[4].add_plain(r.y, r.y); d[4].add_plain(r.z, r.z); d[4].add_plain(r.w, r.w);
    d[5].add_plain(l.x, l.x); d[5].add_plain(l.y, l.y); d[5].add_plain(l.z, l.z); d[5].add_plain(l.w, l.w);
}

// An invariant subspace: the new vector has cancelled to this fraction of |B v_j| (right) or
// |B^dag w_j| (left), a few hundred times the rounding level of the vectors' precision.  A
// regular step of these processes keeps the ratio of order one.
template <typename R> __host__ __device__ constexpr double invariant_tol();
template <> __host__ __device__ constexpr double invariant_tol<double>() { return 1e-10; }
template <> __host__ __device__ constexpr double invariant_tol<float>() { return 1e-5; }
template <> __host__ __device__ constexpr double invariant_tol<ff>() { return 1e-10; }

// The scalar step after omega_j = <wh_{j+1}, vh_{j+1}> (res[0], res[1]) and the norms res[2..5]:
// breakdown and invariant-subspace tests, delta_j = sqrt|omega|, beta_j = omega / delta_j and the
// scales of the next step.  One thread.
template <typename R>
__device__ inline void update_scalars(const UpdArgs& a, int src, const double (&res)[6]) {
    TslState& st = a.state[src];
    // omega = <wh_{j+1}, vh_{j+1}>; delta_j = sqrt|omega|; beta_j = omega / delta_j
    const double om_re = res[0], om_im = res[1];
    const double nv2 = res[2], nw2 = res[3];
    const double om = hypot(om_re, om_im);
    const int j = a.j;
    if (!isfinite(om) || !isfinite(nv2) || !isfinite(nw2)) { st.status = LQ_ERR_NONFINITE; return; }
    // |B v_j|^2 = |s_j|^2 |B vh_j|^2 and |B^dag w_j|^2 = |u_j|^2 |B^dag wh_j|^2 (cv[0] = s_j, cw[0] = u_j)
    const double tol2 = invariant_tol<R>() * invariant_tol<R>();
    const double rr = (st.cv[0].x * st.cv[0].x + st.cv[0].y * st.cv[0].y) * res[4];
    const double ll = (st.cw[0].x * st.cw[0].x + st.cw[0].y * st.cw[0].y) * res[5];
    // vh_{j+1} = s_j B vh_j - ... is in the units of B v_j already (likewise wh_{j+1})
    if (nv2 <= tol2 * rr || nw2 <= tol2 * ll) { st.status = LQ_ERR_BREAKDOWN; return; }
    if (om < st.breakdown_tol * sqrt(nv2) * sqrt(nw2) || om == 0.0) { st.status = LQ_ERR_BREAKDOWN; return; }
    const double dl = sqrt(om);
    const double2 be = make_double2(om_re / dl, om_im / dl);
    a.delta[(size_t)src * a.kmax + j] = dl;
    a.beta[(size_t)src * a.kmax + j] = be;
    st.s_prev = st.s_cur;
    st.u_prev = st.u_cur;
    st.beta_prev = be;
    st.delta_prev = dl;
    st.s_cur = 1.0 / dl;
    // u_{j+1} = 1 / conj(beta_j)
    const double bn = be.x * be.x + be.y * be.y;
    st.u_cur = make_double2(be.x / bn, be.y / bn);
}

// Lanczos scalar step after alpha_j: record alpha_j and prepare the update coefficients
//   vh_{j+1} = s_j B vh_j - alpha_j s_j vh_j - beta_{j-1} s_{j-1} vh_{j-1}
//   wh_{j+1} = u_j B^dag wh_j - conj(alpha_j) u_j wh_j - delta_{j-1} u_{j-1} wh_{j-1}
__device__ inline void tsl_alpha_step(const HopArgs& a, int src, double dre, double dim) {
    TslState& st = a.state[src];
    const int j = a.j;
    const double2 uj = st.u_cur;
    const double sj = st.s_cur;
    // alpha = conj(u_j) s_j <wh_j, B vh_j>
    double2 al;
    al.x = sj * (uj.x * dre + uj.y * dim);
    al.y = sj * (uj.x * dim - uj.y * dre);
    a.alpha[(size_t)src * a.kmax + j] = al;
    a.scale[(size_t)src * a.kmax + j] = sj;
    if (a.uscale) a.uscale[(size_t)src * a.kmax + j] = uj;
    st.k_eff = j + 1;
    if (!isfinite(al.x) || !isfinite(al.y)) { st.status = LQ_ERR_NONFINITE; return; }
    st.cv[0] = make_double2(sj, 0.0);
    st.cv[1] = make_double2(-al.x * sj, -al.y * sj);
    st.cw[0] = uj;
    // -conj(alpha) u_j
    st.cw[1] = make_double2(-(al.x * uj.x + al.y * uj.y), -(al.x * uj.y - al.y * uj.x));
    if (j > 0) {
        st.cv[2] = make_double2(-st.beta_prev.x * st.s_prev, -st.beta_prev.y * st.s_prev);
        st.cw[2] = make_double2(-st.delta_prev * st.u_prev.x, -st.delta_prev * st.u_prev.y);
    } else {
        st.cv[2] = make_double2(0.0, 0.0);
        st.cw[2] = make_double2(0.0, 0.0);
    }
    if (j == a.kmax_run - 1) st.status = 1;   // k reached
}

}  // namespace lq
