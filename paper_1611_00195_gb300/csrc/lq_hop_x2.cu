// Packed-FP32 block stencil of the two-sided Lanczos step (schedules 7 and 8, FP32 contexts).
//
// It applies the block operator B = [[A, E], [0, A]] of Eq. (2.5) to the right vectors and B^dag
// to the left vectors of every source, A = H(mu) = gamma5 Dw(mu) of Eq. (1.1), with the Lanczos
// alpha dot in the epilogue -- the same work, thread decomposition (one thread per site and side)
// and results as schedule 3 of k_hop, bit for bit.  What changes is the instruction stream:
//
//   * complex arithmetic on sm_100+ packed FP32 pairs (__ffma2_rn / __fadd2_rn / __fmul2_rn): one
//     instruction updates the real and the imaginary part.  A complex multiply-add acc += u h is
//     the two packed FMAs  acc = (ux, ux) * (hx, hy) + acc;  acc = (-uy, uy) * (hy, hx) + acc,
//     which round exactly like the four scalar FMAs of the scalar kernel, in the same order;
//   * links stored pre-broadcast as float4 (ux, ux, -uy, uy) (HopArgs::Up / Yp), so that both
//     operand pairs come straight from one 16-byte load; the second operand of the pair is the
//     swapped half spinor (hy, hx), or (-hy, -hx) for the adjoint link of a backward hop, formed
//     once per projection;
//   * the common factor -1/2 of the hops in Dw is applied once per output component instead of
//     once per hop: every hop is accumulated with its factor times -2 (exactly 1 on spatial hops,
//     so nothing is multiplied there) and the sum is scaled by -1/2 in the epilogue.  Scaling by
//     a power of two commutes with every rounding, so the result is unchanged bit for bit.
//
// Schedule 8 adds a software pipeline: while a thread computes one hop it has the two neighbour
// spinors of its next hop in flight into its own slice of shared memory (cp.async, double
// buffered; each thread reads only what it copied, so no barrier is needed), so that the L2/HBM
// latency of a hop overlaps the arithmetic of the previous one.
#include "lq_internal.cuh"
#include "lq_launch.h"
#include "lq_stencil.cuh"

namespace lq {
namespace {

__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded like the scalar subtraction: fma(b, -1, a) is exactly a - b before rounding
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Projection to the half spinor h of the hop in direction NU (see project<> in lq_stencil.cuh)
// and its partner operand hx: (hy, hx) for a forward hop (link U), (-hy, -hx) for a backward hop
// (link U^dag).
template <int NU, int SP>
__device__ __forceinline__ void project_x2(const float2 (&p)[12], float2 (&h)[6], float2 (&hx)[6]) {
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        const float2 u0 = p[col], u1 = p[3 + col], d2 = p[6 + col], d3 = p[9 + col];
        float2 a, b;
        if (NU == 1) {          // B psi_dn = (-d3, d2): pairs as they are
            if (SP > 0) { a = sub2(u0, d3); b = add2(u1, d2); }
            else { a = add2(u0, d3); b = sub2(u1, d2); }
        } else if (NU == 3) {   // B psi_dn = (d2, d3)
            if (SP > 0) { a = add2(u0, d2); b = add2(u1, d3); }
            else { a = sub2(u0, d2); b = sub2(u1, d3); }
        } else {                // x, z: factors of +-i swap the components (scalar adds)
            float2 b0, b1;
            if (NU == 0) { b0 = cmul_mi(d3); b1 = cmul_mi(d2); }
            else { b0 = cmul_mi(d2); b1 = cmul_i(d3); }
            if (SP > 0) { a = cadd(u0, b0); b = cadd(u1, b1); }
            else { a = csub(u0, b0); b = csub(u1, b1); }
        }
        h[col] = a;
        h[3 + col] = b;
        if (SP > 0) { hx[col] = make_float2(-a.y, -a.x); hx[3 + col] = make_float2(-b.y, -b.x); }
        else { hx[col] = make_float2(a.y, a.x); hx[3 + col] = make_float2(b.y, b.x); }
    }
}

// g = U h (DAG false) or U^dag h (DAG true) with pre-broadcast link elements (ux, ux, -uy, uy).
template <bool DAG>
__device__ __forceinline__ void su3_mul_x2(const float4 (&u)[9], const float2 (&h)[6], const float2 (&hx)[6],
                                           float2 (&g)[6]) {
#pragma unroll
    for (int sc = 0; sc < 2; ++sc)
#pragma unroll
        for (int row = 0; row < 3; ++row) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                const float4 e = DAG ? u[col * 3 + row] : u[row * 3 + col];
                a = fma2(make_float2(e.x, e.y), h[sc * 3 + col], a);
                a = fma2(make_float2(e.z, e.w), hx[sc * 3 + col], a);
            }
            g[sc * 3 + row] = a;
        }
}

// acc += (g, s B^dag g) (see reconstruct_add<> in lq_stencil.cuh)
template <int NU, int SP>
__device__ __forceinline__ void reconstruct_x2(const float2 (&g)[6], float2 (&acc)[12]) {
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        const float2 g0 = g[col], g1 = g[3 + col];
        acc[col] = add2(acc[col], g0);
        acc[3 + col] = add2(acc[3 + col], g1);
        if (NU == 1) {          // B^dag g = (g1, -g0)
            if (SP > 0) { acc[6 + col] = add2(acc[6 + col], g1); acc[9 + col] = sub2(acc[9 + col], g0); }
            else { acc[6 + col] = sub2(acc[6 + col], g1); acc[9 + col] = add2(acc[9 + col], g0); }
        } else if (NU == 3) {   // B^dag g = (g0, g1)
            if (SP > 0) { acc[6 + col] = add2(acc[6 + col], g0); acc[9 + col] = add2(acc[9 + col], g1); }
            else { acc[6 + col] = sub2(acc[6 + col], g0); acc[9 + col] = sub2(acc[9 + col], g1); }
        } else {
            float2 l0, l1;
            if (NU == 0) { l0 = cmul_i(g1); l1 = cmul_i(g0); }
            else { l0 = cmul_i(g0); l1 = cmul_mi(g1); }
            if (SP > 0) { acc[6 + col] = cadd(acc[6 + col], l0); acc[9 + col] = cadd(acc[9 + col], l1); }
            else { acc[6 + col] = csub(acc[6 + col], l0); acc[9 + col] = csub(acc[9 + col], l1); }
        }
    }
}

__device__ __forceinline__ void load_link_x2(const float4* __restrict__ L, size_t V, int nu, size_t s, float4 (&u)[9]) {
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = __ldg(L + ((size_t)nu * 9 + e) * V + s);
}

// h *= f, hx *= f (temporal hops; spatial hops carry the factor 1 after the -1/2 is taken out)
__device__ __forceinline__ void scale_x2(float2 (&h)[6], float2 (&hx)[6], float f) {
#pragma unroll
    for (int i = 0; i < 6; ++i) { h[i] = mul2(h[i], bc2(f)); hx[i] = mul2(hx[i], bc2(f)); }
}
// t = fa h + fe e (the d/dmu time hop, which shares the link between A and E)
__device__ __forceinline__ void axpby_x2(float2 (&t)[6], float2 (&tx)[6], float fa, const float2 (&h)[6],
                                         const float2 (&hx)[6], float fe, const float2 (&e)[6], const float2 (&ex)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        t[i] = fma2(bc2(fe), e[i], mul2(h[i], bc2(fa)));
        tx[i] = fma2(bc2(fe), ex[i], mul2(hx[i], bc2(fa)));
    }
}

// Hop factors times -2 (exact in FP32): 1 on spatial hops.
__device__ __forceinline__ float fa2(const HopArgs& a, int side, int nu, bool fwd) { return -2.f * fac_a<float>(a, side, nu, fwd); }
__device__ __forceinline__ float fe2(const HopArgs& a, int side, int nu, bool fwd) { return -2.f * fac_e<float>(a, side, nu, fwd); }

// One hop (direction NU, SP = -1 forward / +1 backward) for both fields of one side; psi0 / psi1
// are the neighbour spinors of the two input fields.  Mirrors do_hop<float, 2, EMODE, NU, SP>.
template <int EMODE, int NU, int SP>
__device__ __forceinline__ void hop_x2(const HopArgs& a, int side, size_t V, size_t lsite, float bsign,
                                       const float2 (&psi0)[12], const float2 (&psi1)[12], float2 (&acc0)[12],
                                       float2 (&acc1)[12]) {
    constexpr bool DAG = SP > 0;
    constexpr bool TIME = NU == 3;
    float4 u[9];
    load_link_x2(reinterpret_cast<const float4*>(a.Up), V, NU, lsite, u);
    float2 h0[6], h0x[6], h1[6], h1x[6], g[6];
    project_x2<NU, SP>(psi0, h0, h0x);
    project_x2<NU, SP>(psi1, h1, h1x);
    const float fa = fa2(a, side, NU, SP < 0) * bsign;
    const float fe = fe2(a, side, NU, SP < 0) * bsign;
    const bool emu = (EMODE == 1) && TIME;
    // the operand that carries the derivative: right side E b (b = field 1), left side E^dag p (field 0)
    if (side == 0) {
        // out0 += U (fa h0 [+ fe h1 for d/dmu]) [+ Y (fe h1)];  out1 += U (fa h1)
        if (emu) {
            float2 t[6], tx[6];
            axpby_x2(t, tx, fa, h0, h0x, fe, h1, h1x);
            su3_mul_x2<DAG>(u, t, tx, g);
        } else if (TIME) {
            float2 t[6], tx[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) { t[i] = mul2(h0[i], bc2(fa)); tx[i] = mul2(h0x[i], bc2(fa)); }
            su3_mul_x2<DAG>(u, t, tx, g);
        } else {
            su3_mul_x2<DAG>(u, h0, h0x, g);
        }
        reconstruct_x2<NU, SP>(g, acc0);
        if (EMODE == 2) {
            float4 y[9];
            load_link_x2(reinterpret_cast<const float4*>(a.Yp), V, NU, lsite, y);
            if (TIME) {
                float2 t[6], tx[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) { t[i] = mul2(h1[i], bc2(fe)); tx[i] = mul2(h1x[i], bc2(fe)); }
                su3_mul_x2<DAG>(y, t, tx, g);
            } else {
                su3_mul_x2<DAG>(y, h1, h1x, g);
            }
            reconstruct_x2<NU, SP>(g, acc0);
        }
        if (TIME) scale_x2(h1, h1x, fa);
        su3_mul_x2<DAG>(u, h1, h1x, g);
        reconstruct_x2<NU, SP>(g, acc1);
    } else {
        // out0 += U (fa h0);  out1 += U (fa h1 [+ fe h0]) [+ Y (fe h0)]
        if (emu) {
            float2 t[6], tx[6];
            axpby_x2(t, tx, fa, h1, h1x, fe, h0, h0x);
            su3_mul_x2<DAG>(u, t, tx, g);
        } else if (TIME) {
            float2 t[6], tx[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) { t[i] = mul2(h1[i], bc2(fa)); tx[i] = mul2(h1x[i], bc2(fa)); }
            su3_mul_x2<DAG>(u, t, tx, g);
        } else {
            su3_mul_x2<DAG>(u, h1, h1x, g);
        }
        reconstruct_x2<NU, SP>(g, acc1);
        if (EMODE == 2) {
            float4 y[9];
            load_link_x2(reinterpret_cast<const float4*>(a.Yp), V, NU, lsite, y);
            if (TIME) {
                float2 t[6], tx[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) { t[i] = mul2(h0[i], bc2(fe)); tx[i] = mul2(h0x[i], bc2(fe)); }
                su3_mul_x2<DAG>(y, t, tx, g);
            } else {
                su3_mul_x2<DAG>(y, h0, h0x, g);
            }
            reconstruct_x2<NU, SP>(g, acc1);
        }
        if (TIME) scale_x2(h0, h0x, fa);
        su3_mul_x2<DAG>(u, h0, h0x, g);
        reconstruct_x2<NU, SP>(g, acc0);
    }
}

// Neighbour of site s in direction NU (FWD: +NU), its link site and the antiperiodic sign.
template <int NU, bool FWD>
__device__ __forceinline__ size_t nb_site(const HopArgs& a, size_t s, const int (&x)[4], size_t& lsite, float& bsign) {
    const int ext = a.dims[NU];
    const size_t stride = a.strides[NU];
    if (FWD) {
        const size_t sf = (x[NU] == ext - 1) ? s - (size_t)(ext - 1) * stride : s + stride;
        bsign = (NU == 3 && a.apbc && x[NU] == ext - 1) ? -1.f : 1.f;
        lsite = s;
        return sf;
    }
    const size_t sb = (x[NU] == 0) ? s + (size_t)(ext - 1) * stride : s - stride;
    bsign = (NU == 3 && a.apbc && x[NU] == 0) ? -1.f : 1.f;
    lsite = sb;
    return sb;
}

// gamma5 [diag psi - acc / 2] for the unscaled hop sum acc (see finish<> in lq_stencil.cuh):
// -(x) on the lower spin components is computed as fma(-diag, psi, acc / 2), rounded identically.
__device__ __forceinline__ void finish_x2(const float2 (&psi)[12], float diag, float2 (&acc)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        if (c < 6) acc[c] = fma2(bc2(diag), psi[c], mul2(acc[c], bc2(-0.5f)));
        else acc[c] = fma2(bc2(-diag), psi[c], mul2(acc[c], bc2(0.5f)));
    }
}

// cp.async of 16 bytes, global -> shared (the thread's own slice), and its completion waits
__device__ __forceinline__ void cpa16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kPfBuf = 2 * 2 * 6;   // float4 per thread: 2 buffers x 2 fields x 6 chunks

// Hop HOP (0..7: direction HOP / 2, forward when even) of the site; PF: read the neighbour spinors
// from the thread's shared-memory buffer HOP & 1 (filled one hop earlier) and start the copies of
// hop HOP + 1 into the other buffer first.
template <int EMODE, bool PF, int HOP>
__device__ __forceinline__ void step_x2(const HopArgs& a, int side, size_t V, size_t s, const int (&x)[4], bool active,
                                        const float4* in0, const float4* in1, float4* pf, float2 (&acc0)[12],
                                        float2 (&acc1)[12]) {
    constexpr int NU = HOP / 2;
    constexpr bool FWD = (HOP % 2) == 0;
    size_t lsite;
    float bsign;
    const size_t nb = nb_site<NU, FWD>(a, s, x, lsite, bsign);
    float2 psi0[12], psi1[12];
    if (PF) {
        if (HOP < 7) {
            constexpr int NNU = (HOP + 1) / 2;
            constexpr bool NFWD = ((HOP + 1) % 2) == 0;
            size_t ls2;
            float b2;
            const size_t nn = nb_site<NNU, NFWD>(a, s, x, ls2, b2);
            float4* dst = pf + ((HOP + 1) & 1) * 12 * kHopThreads + threadIdx.x;
            if (active) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    cpa16(dst + q * kHopThreads, in0 + (size_t)q * V + nn);
                    cpa16(dst + (6 + q) * kHopThreads, in1 + (size_t)q * V + nn);
                }
            }
            cpa_commit();
            cpa_wait<1>();       // everything but the copies just started: hop HOP's buffer is complete
        } else {
            cpa_wait<0>();
        }
        const float4* src = pf + (HOP & 1) * 12 * kHopThreads + threadIdx.x;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v0 = src[q * kHopThreads], v1 = src[(6 + q) * kHopThreads];
            psi0[2 * q] = make_float2(v0.x, v0.y); psi0[2 * q + 1] = make_float2(v0.z, v0.w);
            psi1[2 * q] = make_float2(v1.x, v1.y); psi1[2 * q + 1] = make_float2(v1.z, v1.w);
        }
    } else if (active) {
        load_spinor(in0, V, nb, psi0);
        load_spinor(in1, V, nb, psi1);
    }
    if (active) hop_x2<EMODE, NU, FWD ? -1 : +1>(a, side, V, lsite, bsign, psi0, psi1, acc0, acc1);
}

template <int EMODE, bool DOT, bool PF>
__global__ void __launch_bounds__(kHopThreads, 4) k_hop_x2(HopArgs a) {
    using C = float2;
    using Chunk = float4;
    extern __shared__ float4 pf_smem[];
    __shared__ CSum smem[32 * 2];
    const int side = blockIdx.y + a.side0;
    const unsigned bx = blockIdx.x;
    const int src = blockIdx.z;
    if (a.state != nullptr && a.state[src].status != 0) return;   // source finished / failed
    const size_t V = a.V;
    const size_t s = (size_t)bx * blockDim.x + threadIdx.x;
    const bool active = s < V;
    const Chunk* in0 = reinterpret_cast<const Chunk*>(a.in[side]) + (size_t)src * a.src_stride_in[side];
    const Chunk* in1 = in0 + field_elems<float>(V);
    Chunk* out0 = reinterpret_cast<Chunk*>(a.out[side]) + (size_t)src * a.src_stride_out[side];
    Chunk* out1 = out0 + field_elems<float>(V);

    C acc0[12], acc1[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) { acc0[c] = make_float2(0.f, 0.f); acc1[c] = make_float2(0.f, 0.f); }
    DotAcc<float> d[2];
    d[0].zero(); d[1].zero();
    int x[4] = {0, 0, 0, 0};
    const size_t sa = active ? s : 0;    // inactive threads still take part in the copy groups
    if (active) site_coords(a, s, x);
    float4* pf = PF ? pf_smem : nullptr;
    if (PF) {
        size_t ls;
        float b;
        const size_t nn = nb_site<0, true>(a, sa, x, ls, b);
        float4* dst = pf + threadIdx.x;
        if (active) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                cpa16(dst + q * kHopThreads, in0 + (size_t)q * V + nn);
                cpa16(dst + (6 + q) * kHopThreads, in1 + (size_t)q * V + nn);
            }
        }
        cpa_commit();
    }
    step_x2<EMODE, PF, 0>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 1>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 2>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 3>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 4>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 5>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 6>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    step_x2<EMODE, PF, 7>(a, side, V, sa, x, active, in0, in1, pf, acc0, acc1);
    if (active) {
        const float diag = fac_diag<float>(a);
        C psi[12];
        load_spinor(in0, V, s, psi);
        finish_x2(psi, diag, acc0);
        store_spinor(out0, V, s, acc0);
        load_spinor(in1, V, s, psi);
        finish_x2(psi, diag, acc1);
        store_spinor(out1, V, s, acc1);
        if (DOT && side == 0) {
            // <w_j, B vh_j> restricted to this site: left inputs at s (conj) times outputs
            const Chunk* l0 = reinterpret_cast<const Chunk*>(a.in[1]) + (size_t)src * a.src_stride_in[1];
            C w[12];
            load_spinor(l0, V, s, w);
#pragma unroll
            for (int c = 0; c < 12; ++c) add_cdot(d[0], d[1], w[c], acc0[c]);
            load_spinor(l0 + field_elems<float>(V), V, s, w);
#pragma unroll
            for (int c = 0; c < 12; ++c) add_cdot(d[0], d[1], w[c], acc1[c]);
        }
    }
    if (DOT && side == 0) {
        const int nbx = (int)gridDim.x;
        CSum tot[2];
        block_total<float, 2>(d, tot, smem);
        double* part = a.partials + ((size_t)src * a.partial_stride + bx) * 4;
        if (threadIdx.x == 0) { part[0] = tot[0].s; part[1] = tot[0].e; part[2] = tot[1].s; part[3] = tot[1].e; }
        if (last_block(a.counters + src, nbx)) {
            double res[2];
            reduce_partials<2>(a.partials + (size_t)src * a.partial_stride * 4, nbx, res, smem);
            if (threadIdx.x == 0) tsl_alpha_step(a, src, res[0], res[1]);
        }
    }
}

constexpr size_t kPfSmem = (size_t)kPfBuf * kHopThreads * sizeof(float4);   // 48 KB

template <int EMODE, bool DOT, bool PF>
cudaError_t launch_x2_k(const HopArgs& a, cudaStream_t st) {
    const dim3 grid((unsigned)((a.V + kHopThreads - 1) / kHopThreads), (unsigned)a.nsides, (unsigned)a.nsrc);
    if (PF) {
        static bool attr = false;   // opt in to 48 KB of dynamic shared memory next to the static part
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_hop_x2<EMODE, DOT, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kPfSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
    }
    k_hop_x2<EMODE, DOT, PF><<<grid, kHopThreads, PF ? kPfSmem : 0, st>>>(a);
    return cudaGetLastError();
}

// links (ux, uy) [4][9][V] -> (ux, ux, -uy, uy)
__global__ void k_links_packed(const float2* __restrict__ L, float4* __restrict__ P, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 u = L[i];
    P[i] = make_float4(u.x, u.x, -u.y, u.y);
}

}  // namespace

cudaError_t launch_hop_x2(const HopArgs& a, int emode, bool dot, bool prefetch, cudaStream_t st) {
    if (!a.Up || (emode == 2 && !a.Yp)) return cudaErrorInvalidValue;
    if (prefetch) {
        if (emode == 0) return dot ? launch_x2_k<0, true, true>(a, st) : launch_x2_k<0, false, true>(a, st);
        if (emode == 1) return dot ? launch_x2_k<1, true, true>(a, st) : launch_x2_k<1, false, true>(a, st);
        return dot ? launch_x2_k<2, true, true>(a, st) : launch_x2_k<2, false, true>(a, st);
    }
    if (emode == 0) return dot ? launch_x2_k<0, true, false>(a, st) : launch_x2_k<0, false, false>(a, st);
    if (emode == 1) return dot ? launch_x2_k<1, true, false>(a, st) : launch_x2_k<1, false, false>(a, st);
    return dot ? launch_x2_k<2, true, false>(a, st) : launch_x2_k<2, false, false>(a, st);
}

cudaError_t launch_links_packed(const void* L, void* P, size_t V, cudaStream_t st) {
    const size_t n = V * 36;
    k_links_packed<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float2*>(L),
                                                                 reinterpret_cast<float4*>(P), n);
    return cudaGetLastError();
}

}  // namespace lq
