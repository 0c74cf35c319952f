// Internal definitions of the GB300 two-sided-Lanczos library: context, field layouts,
// complex helpers and compensated FP64 reductions shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lq.h"
#include "lq_ff.cuh"

namespace lq {

// ---------------------------------------------------------------------------------------
// Internal field layout (device).  A colour-spinor field of V sites is stored as
// "component-major" chunks so that one warp touching 32 consecutive sites issues fully
// coalesced 512-byte requests:
//   FP64: 12 chunks of double2 (one complex each):  f[c * V + s], c = 3*spin + colour
//   FP32:  6 chunks of float4  (two complex each):  f[q * V + s] holds c = 2q, 2q+1
//   float-float: 12 chunks of float4 (one complex each: re.hi, re.lo, im.hi, im.lo)
// Links: [4 directions][9 elements (row*3+col)][V] of double2 / float2 / float-float complex.
// A block vector (top, bottom) of Eq. (2.6) is two consecutive fields.
// ---------------------------------------------------------------------------------------
template <typename R> struct Tr;
template <> struct Tr<double> {
    using C = double2;        // complex
    using Chunk = double2;    // storage unit of a spinor field
    static constexpr int kChunks = 12;
    static constexpr int kPerChunk = 1;
    static constexpr int kKind = 0;
};
template <> struct Tr<float> {
    using C = float2;
    using Chunk = float4;
    static constexpr int kChunks = 6;
    static constexpr int kPerChunk = 2;
    static constexpr int kKind = 1;
};
template <> struct Tr<ff> {
    using C = cff;
    using Chunk = float4;
    static constexpr int kChunks = 12;
    static constexpr int kPerChunk = 1;
    static constexpr int kKind = 2;
};

template <typename R> __host__ __device__ inline size_t field_elems(size_t V) {
    return (size_t)Tr<R>::kChunks * V;   // in Chunk units
}
template <typename R> __host__ __device__ inline size_t field_bytes(size_t V) {
    return field_elems<R>(V) * sizeof(typename Tr<R>::Chunk);
}

// ---- complex arithmetic on double2 / float2 ---------------------------------------------
template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) { return cmk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a)*b
template <typename C> __device__ __forceinline__ C cdiv(C a, C b) {   // a / b (Smith's scaling)
    if (fabs(b.x) >= fabs(b.y)) {
        auto r = b.y / b.x, d = b.x + b.y * r;
        return cmk<C>((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        auto r = b.x / b.y, d = b.x * r + b.y;
        return cmk<C>((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C cmul_i(C a) { return cmk<C>(-a.y, a.x); }      // i*a
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmk<C>(a.y, -a.x); }     // -i*a
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {  // acc + a*b
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
template <typename C> __device__ __forceinline__ C cfmac(C a, C b, C acc) {  // acc + conj(a)*b
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// ---- spinor load / store in the internal layout ---------------------------------------
__device__ __forceinline__ void load_spinor(const double2* __restrict__ f, size_t V, size_t s, double2 (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = __ldg(f + c * V + s);
}
__device__ __forceinline__ void load_spinor(const float4* __restrict__ f, size_t V, size_t s, float2 (&o)[12]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float4 v = __ldg(f + q * V + s);
        o[2 * q] = make_float2(v.x, v.y);
        o[2 * q + 1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ void load_spinor(const float4* __restrict__ f, size_t V, size_t s, cff (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = cff_from_chunk(__ldg(f + c * V + s));
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ f, size_t V, size_t s, const double2 (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) f[c * V + s] = o[c];
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ f, size_t V, size_t s, const float2 (&o)[12]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) f[q * V + s] = make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ f, size_t V, size_t s, const cff (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) f[c * V + s] = cff_to_chunk(o[c]);
}

// ---- error-free transformations (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26 (2005)) --
// A compensated sum is carried as (s, e): value = s + e.
struct CSum { double s, e; };
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& t) {
    s = a + b;
    double z = s - a;
    t = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void cs_add(CSum& acc, double x) {
    double s, t;
    two_sum(acc.s, x, s, t);
    acc.s = s;
    acc.e += t;
}
__device__ __forceinline__ void cs_add_prod(CSum& acc, double a, double b) {  // acc += a*b exactly-rounded-ish
    double p = a * b;
    double pe = fma(a, b, -p);
    cs_add(acc, p);
    acc.e += pe;
}
__device__ __forceinline__ CSum cs_merge(CSum a, CSum b) {
    double s, t;
    two_sum(a.s, b.s, s, t);
    CSum r; r.s = s; r.e = a.e + b.e + t;
    return r;
}
__device__ __forceinline__ CSum cs_shfl_down(CSum a, int off) {
    CSum b;
    b.s = __shfl_down_sync(0xffffffffu, a.s, off);
    b.e = __shfl_down_sync(0xffffffffu, a.e, off);
    return b;
}

// Reduce NV compensated sums across the block; result valid in thread 0.
// smem must hold (blockDim.x/32) * NV CSum.
template <int NV>
__device__ __forceinline__ void block_reduce_cs(CSum (&v)[NV], CSum* smem) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = cs_merge(v[i], cs_shfl_down(v[i], off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            if (lane < nw) v[i] = smem[lane * NV + i];
            else { v[i].s = 0.0; v[i].e = 0.0; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = cs_merge(v[i], cs_shfl_down(v[i], off));
    }
    __syncthreads();
}

// ---- per-source Lanczos state (device) ---------------------------------------------------
// Vectors are stored unnormalised: v_j = s_j * vh_j (right), w_j = u_j * wh_j (left).
struct TslState {
    int status;        // 0 running, 1 stopped normally (k reached), <0 LQ_ERR_* code
    int k_eff;         // number of alpha's computed
    double xnorm;      // |x|
    double s_prev, s_cur;              // right scales s_{j-1}, s_j (real)
    double2 u_prev, u_cur;             // left scales u_{j-1}, u_j
    double2 beta_prev;                 // beta_{j-1}
    double delta_prev;                 // delta_{j-1}
    double2 cv[3];                     // update coefficients (right) for the current step
    double2 cw[3];                     // update coefficients (left)
    double breakdown_tol;
    double rb_nr, rb_nl;               // |B vh_j|^2, |B^dag wh_j|^2 of an update whose scalar step
                                       // waits for the re-biorthogonalisation
};

// Per-source slices of the projected tridiagonal T_k: alpha[k], beta[k], delta[k], scale[k]
// (scale[j] = s_j, so that v_j = scale[j] * vh_j) live in separate device arrays.

}  // namespace lq

// ---- the context (opaque to callers) -------------------------------------------------------
struct lq_ctx {
    lq_lattice_desc desc;
    int dims[4];           // nx, ny, nz, nt (direction order x, y, z, t)
    size_t V = 0;
    int prec = LQ_FP64;              // LQ_FP64 or LQ_MIXED (the arithmetic of every kernel)
    bool link_bf16 = false;          // LQ_MIXED_BF16: the stencil's links stored in BF16
    int device = 0;
    std::string err;

    // gauge field in the internal layout/precision
    void* U = nullptr;
    double* Ub = nullptr;            // FP64 copy in the boundary layout (direction builder)
    bool gauge_ready = false;
    // derivative direction: dU/dt = Y (internal layout/precision); kind of the current one
    void* Y = nullptr;
    void* Up = nullptr;              // FP32 contexts: links as float4 (ux, ux, -uy, uy), packed stencil
    void* Yp = nullptr;              // the same for Y
    double* dir_scratch = nullptr;   // staging for the direction coefficients
    int dir_kind = -1;

    // workspace (lq_reserve)
    int kmax = 0, nsrc = 0, block = 0;
    int ring = 0;                    // basis slots per source when reserved for two-pass runs only
    void* basis = nullptr;           // [nsrc][kmax][NF] fields
    void* left = nullptr;            // [nsrc][3][NF] fields (ring)
    void* rout = nullptr;            // [nsrc][NF] fields: B vh_j
    void* lout = nullptr;            // [nsrc][NF] fields: B^dag wh_j
    double* io = nullptr;            // [6][nsrc][V][12] complex128 boundary staging (device)
    double* norms = nullptr;         // [3][nsrc] norm results
    double* partials = nullptr;      // reduction partials
    int* counters = nullptr;         // last-block counters
    lq::TslState* state = nullptr;   // [nsrc]
    double2* alpha = nullptr;        // [nsrc][kmax]
    double2* beta = nullptr;         // [nsrc][kmax]
    double* delta = nullptr;         // [nsrc][kmax]
    double* scale = nullptr;         // [nsrc][kmax]
    // Newton workspace
    double2* nx_X = nullptr;         // [nsrc][kmax][kmax]
    double2* nx_Y = nullptr;         // [nsrc][kmax][kmax]
    double2* nx_F = nullptr;         // [nsrc][kmax]
    int* nx_perm = nullptr;          // [nsrc][kmax]
    double* nx_scal = nullptr;       // [nsrc][16] Newton scalars
    double* nx_partials = nullptr;   // Newton reduction partials
    int* nx_counters = nullptr;
    // projected coefficients and quadrature workspace
    double2* proj_c = nullptr;       // [nsrc][kmax] sgn(T_k) e_1
    double2* quad_q = nullptr;       // [nsrc][kmax] involution check vector
    double2* quad_work = nullptr;    // [nsrc][4][kmax][2 * kQuadMaxNodes]
    double* quad_c = nullptr;        // [nsrc]
    double* quad_check = nullptr;    // [nsrc]
    int* quad_nodes = nullptr;       // [nsrc] nodes of the current quadrature pass per source
    double2* quad_part = nullptr;    // [nsrc][2 * kQuadRetryMaxNodes / 32][kmax] block row sums of the quadrature
    int* proj_sel = nullptr;         // [nsrc] sources finished by the Newton fallback
    // nested projected sign: inner state and coefficients, its first columns and results
    lq::TslState* nest_state = nullptr;   // [nsrc]
    double2* nest_alpha = nullptr;        // [nsrc][kmax]
    double2* nest_beta = nullptr;         // [nsrc][kmax]
    double* nest_delta = nullptr;         // [nsrc][kmax]
    double2* nest_s = nullptr;            // [nsrc][kmax] inner sgn(T') e_1
    double2* nest_q = nullptr;            // [nsrc][kmax] second-pass result
    double* nest_norm = nullptr;          // [nsrc]
    double* nest_check = nullptr;         // [nsrc]
    double* nest_c = nullptr;             // [nsrc] staged scales (lq_nested_sign)
    size_t partial_blocks = 0;       // capacity per source of the TSL partials
    size_t nx_partial_blocks = 0;

    // adjoint workspace (lq_reserve flag LQ_RESERVE_ADJOINT)
    void* lbasis = nullptr;          // [nsrc][kmax][lbasis_nf] left Lanczos vectors
    int lbasis_nf = 0;               // fields per stored left vector: 1 (adjoint), NF (re-biorthogonalisation)
    double2* uscale = nullptr;       // [nsrc][kmax] left scales
    // re-biorthogonalisation workspace (lq_reserve flag LQ_RESERVE_REBIORTH)
    double* rb_part = nullptr;       // [nsrc][kmax][rb_dot_blocks][8]
    double2* rb_coef = nullptr;      // [nsrc][2][kmax]
    float4* rb_coef_f = nullptr;     // [nsrc][2][kmax]
    bool rebiorth = false;
    double2* adj_coef = nullptr;     // [2][2 * kQuadMaxNodes][kmax]
    void* adj_nu = nullptr;          // [2 * kQuadMaxNodes] fields
    void* adj_om = nullptr;          // [2 * kQuadMaxNodes] fields
    double* adj_force = nullptr;     // [4][V][8]
    double* adj_dmu = nullptr;       // [V / 128 + 1]
    bool adjoint = false;

    // deflation space (Sec. 3), FP64 boundary layout: V = [R_0..R_{l-1}, dR_0..dR_{l-1}],
    // W = [Lk_0..Lk_{l-1}, dLk_0..dLk_{l-1}] with <Lk_i|R_j> = delta_ij (Lk_i = L_i^dag)
    int defl_l = 0, defl_cap = 0;
    std::vector<double2> defl_lam, defl_dlam;
    double* defl_V = nullptr;
    double* defl_W = nullptr;
    double* defl_work = nullptr;     // [6][cap][n] scratch vectors for the derivative preparation
    double* defl_scr = nullptr;      // dot partials and coefficient matrices
    size_t defl_scr_doubles = 0;
    double* gen_scr = nullptr;       // general dot / combine scratch (lq_reserve)
    double* solve_ws = nullptr;      // overlap solver: [9][nsrc][V][12] complex (LQ_RESERVE_SOLVE)
    size_t gen_scr_doubles = 0;
    double2* defl_shift = nullptr;   // [nsrc] resolvent shifts
    double defl_resid = 0.0;         // largest relative residual of the last shifted solves
    // the eigenvector derivatives of the generalised deflation along d/dmu are kept until the
    // space, the links, mu, the Jordan blocks or the shifted-solve depth change
    long long defl_version = 0;      // bumped by every change of the space or the links
    bool defl_prep_ok = false;
    long long defl_prep_version = -1;
    double defl_prep_mu = 0.0;
    int defl_prep_ld = 0, defl_prep_kd = 0, defl_prep_prec = 0;
    lq_eig_stats eig_stats{};        // statistics of the last lq_compute_deflation

    // stencil autotuning: chosen variant per (batch size, nf, emode) of the Lanczos step
    struct Tuned { int nsrc, nf, emode, variant; };
    std::vector<Tuned> tuned;

    // CUDA graphs of the Krylov loop, one per configuration (cleared when the workspace is
    // reserved again); captured on cap_stream, launched on the caller's stream
    struct GraphKey {
        int k, nsrc, nf, emode, variant, store_left, ring;
        double mu;
        int groups;        // source groups run as concurrent branches (1: none)
        int update;        // update kernel (UpdArgs.bulk)
        int rebiorth;      // re-biorthogonalisation period (0: none)
        bool operator==(const GraphKey& o) const {
            return k == o.k && nsrc == o.nsrc && nf == o.nf && emode == o.emode && variant == o.variant &&
                   store_left == o.store_left && ring == o.ring && mu == o.mu && groups == o.groups &&
                   update == o.update && rebiorth == o.rebiorth;
        }
    };
    struct GraphEntry { GraphKey key; cudaGraphExec_t exec; };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;   // the second source group's branch

    // profiling (lq_profile_enable): event pairs per kernel class, summed at sync points
    int prof_on = 0;
    long long launches = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double prof_ms[4] = {0, 0, 0, 0};       // hop, update, newton, other
    long long prof_n[4] = {0, 0, 0, 0};
};
