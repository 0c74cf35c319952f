// Kernel argument blocks and host launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "lq_internal.cuh"

namespace lq {

constexpr int kHopThreads = 128;
constexpr int kUpdThreads = 256;
constexpr int kRecThreads = 128;
constexpr int kTwoPassRing = 32;     // basis slots per source of a two-pass run
constexpr int kTwoPassWindow = 16;   // Krylov vectors recombined at a time in the second pass

// Arguments of the stencil kernel k_hop (Eq. (1.1), block operator of Eq. (2.5)).
struct HopArgs {
    int dims[4];           // x, y, z, t extents
    size_t strides[4];     // site-index strides of the four directions
    size_t V;
    int apbc;
    int nsrc, nsides;
    int side0;             // side of blockIdx.y == 0 (0 = right / A, 1 = left / A^dag)
    int variant;           // 0: one thread per (site, side); 1: one thread per (site, output field)
    double diag;           // 4r + m_w
    // hop factors, including the -1/2 of Dw: [side][direction]
    double a_fwd[2][4], a_bwd[2][4];   // operator A (side 0) / A^dag (side 1)
    double e_fwd[2][4], e_bwd[2][4];   // derivative E (side 0) / E^dag (side 1)
    float af_fwd[2][4], af_bwd[2][4], ef_fwd[2][4], ef_bwd[2][4];   // FP32 copies (no conversion in kernels)
    float diag_f;
    const void* U;         // links (internal)
    const void* Y;         // dU/dt (internal), EMODE 2
    int link_bf16;         // FP32 kernels: U holds __nv_bfloat162 entries instead of float2
    const void* Up;        // FP32 links pre-broadcast as float4 (ux, ux, -uy, uy) (schedules 7, 8)
    const void* Yp;        // the same for dU/dt
    const void* in[2];     // per side: NF consecutive fields of source 0
    void* out[2];
    size_t src_stride_in[2], src_stride_out[2];   // Chunk units between sources
    // Lanczos alpha dot (DOT)
    TslState* state;       // may be null (plain operator application)
    double* partials;
    size_t partial_stride; // blocks per source capacity
    int* counters;
    double2* alpha;
    double* scale;
    double2* uscale;       // left scales u_j (stored when the left basis is kept), may be null
    int kmax;              // row length of alpha/beta/delta/scale
    int kmax_run;          // k of this run
    int j;                 // 0-based Lanczos step
};

struct UpdArgs {
    size_t nelem;          // Chunk elements per source and side (NF fields)
    int nsrc;
    int j;
    const void* rout; const void* lout;
    const void* v_cur; const void* v_prev; void* v_next;
    const void* w_cur; const void* w_prev; void* w_next;
    void* w_store;         // copy of wh_{j+1} into the left basis (adjoint), may be null
    size_t src_stride_io, src_stride_basis, src_stride_left, src_stride_store;
    TslState* state;
    double* partials;
    size_t partial_stride;
    int* counters;
    double2* beta;
    double* delta;
    int kmax;
    int bulk;              // FP32: 1 = k_update_bulk (inputs staged by bulk copies), 0 = k_update
    int defer;             // 1: keep the norm terms in the state and leave the scalar step to the
                           // re-biorthogonalisation that follows (k_update only)
};

struct InitArgs {
    size_t V;
    int nsrc;
    const double* x;       // boundary layout, device (bottom of a block source)
    const double* xt;      // top of a block source (boundary layout) or null for (0, x)
    void* v1; void* w1;
    void* w1_store;        // copy of wh_1 into the left basis (adjoint), may be null
    size_t src_stride_basis, src_stride_left, src_stride_store;
    TslState* state;
    double* partials;
    size_t partial_stride;
    int* counters;
    double breakdown_tol;
};

struct RecArgs {
    size_t V;
    int nsrc;
    const void* basis;
    size_t src_stride_basis;   // Chunk units
    size_t vec_stride;         // Chunk units between consecutive Krylov vectors
    const TslState* state;
    const double* scale;
    int kmax;
    const double2* coef;       // [nsrc][kmax] sgn(T_k) e_1
    double* y0; double* y1;    // boundary layout outputs (device), field 0 / field 1
    int j0, j1;                // window of Krylov indices [j0, j1) (j1 = 0: up to k_eff)
    int ring;                  // basis slots of a ring (two-pass runs), 0: vector j in slot j
    int accumulate;            // 1: y += window sum; 0: y = window sum
};


cudaError_t launch_hop(int prec, const HopArgs& a, int nf, int emode, bool dot, cudaStream_t st);
// CGNR inner solves of the shift-and-invert eigensolver (lq_eig.cu): nb systems of ne float4
// elements each (internal FP32 layout), FP64 scalars per system in scal[sys * kCgNs + slot].
enum { CG_G0 = 0, CG_G1 = 1, CG_QQ = 2, CG_RR = 3, CG_BB = 4, CG_DONE = 5 };
constexpr int kCgNs = 8;
struct CgArgs {
    size_t ne;             // float4 elements per system
    int nb;                // systems
    int it;                // iteration (selects the slot of g in the two-slot rotation)
    float4* x; float4* r; float4* p; const float4* q; const float4* z;   // [nb][ne]
    double* scal;          // [nb][kCgNs]
    double* part;          // cg_partial_doubles(nb)
    int* counters;         // [nb][3], zero
};
size_t cg_partial_doubles(int nsys);
cudaError_t launch_cg_norm(const CgArgs& a, const float4* v, int slot, cudaStream_t st);   // |v_s|^2 -> slot
cudaError_t launch_cg_xr(const CgArgs& a, cudaStream_t st);     // x += alpha p, r -= alpha q, |r|^2
cudaError_t launch_cg_p(const CgArgs& a, cudaStream_t st);      // p = z + beta p
// packed-FP32 block stencil (lq_hop_x2.cu): schedule 7, or 8 with the neighbour prefetch
// float-float instantiations of the kernel templates (lq_ff_hop0.cu .. lq_ff_hop2.cu: the block
// stencil for derivative mode 0 (and the plain operator), 1 and 2; lq_ff_vec.cu: the rest), called
// by the launchers above with their grids
cudaError_t launch_hop_ff0(const HopArgs& a, int nf, bool dot, cudaStream_t st);
cudaError_t launch_hop_ff1(const HopArgs& a, bool dot, cudaStream_t st);
cudaError_t launch_hop_ff2(const HopArgs& a, bool dot, cudaStream_t st);
cudaError_t launch_roles_ff0(const HopArgs& a, bool dot, cudaStream_t st);   // schedule 1, block operator
cudaError_t launch_roles_ff1(const HopArgs& a, bool dot, cudaStream_t st);
cudaError_t launch_roles_ff2(const HopArgs& a, bool dot, cudaStream_t st);
cudaError_t launch_update_ff(const UpdArgs& a, dim3 grid, cudaStream_t st);
cudaError_t launch_tsl_init_ff(int nf, const InitArgs& a, dim3 grid, cudaStream_t st);
cudaError_t launch_recombine_ff(int nf, const RecArgs& a, dim3 grid, size_t smem, cudaStream_t st);
cudaError_t launch_to_internal_ff(const double* x, void* f, size_t V, int nfields, dim3 grid, cudaStream_t st);
cudaError_t launch_to_boundary_ff(const void* f, double* x, size_t V, int nfields, dim3 grid, cudaStream_t st);
cudaError_t launch_links_internal_ff(const double* U, void* L, size_t V, dim3 grid, cudaStream_t st);
cudaError_t launch_direction_ff(const double* U, const double* w, int kind, void* Y, size_t V, dim3 grid, cudaStream_t st);
cudaError_t launch_hop_x2(const HopArgs& a, int emode, bool dot, bool prefetch, cudaStream_t st);
cudaError_t launch_links_packed(const void* L, void* P, size_t V, cudaStream_t st);   // float2 -> (ux, ux, -uy, uy)
constexpr int kHopSchedules = 10;    // FP32 block-stencil schedules 0..9 (FP64: 0, 1)
bool tile_ok(const int (&dims)[4]);   // schedule 6 (shared-memory tiles) covers this lattice
cudaError_t launch_update(int prec, const UpdArgs& a, cudaStream_t st);
cudaError_t launch_tsl_init(int prec, int nf, const InitArgs& a, cudaStream_t st);
cudaError_t launch_recombine(int prec, int nf, const RecArgs& a, cudaStream_t st);
cudaError_t launch_to_internal(int prec, const double* x, void* f, size_t V, int nfields, cudaStream_t st);
cudaError_t launch_to_boundary(int prec, const void* f, double* x, size_t V, int nfields, cudaStream_t st);
cudaError_t launch_links_internal(int prec, const double* U, void* L, size_t V, cudaStream_t st);
// BF16 link storage: round the boundary-layout FP64 links in place (FP64 -> FP32 -> BF16, nearest
// even) and write the internal BF16 copy [4][9][V] of __nv_bfloat162
cudaError_t launch_links_bf16(double* U, void* L, size_t V, cudaStream_t st);
cudaError_t launch_direction(int prec, const double* U, const double* w, int kind, void* Y, size_t V, cudaStream_t st);
unsigned update_grid(size_t nelem, int nsrc, size_t cap);
// the bulk-copy FP32 update (lq_update_bulk.cu)
cudaError_t launch_update_bulk(const UpdArgs& a, cudaStream_t st);
bool update_bulk_ready();                 // opts in to its shared memory (once); false: unavailable
unsigned update_bulk_grid(size_t nelem, int nsrc, size_t cap);
void update_bulk_prepare();               // every one-time device query, before a stream capture
// Periodic re-biorthogonalisation of the new Lanczos pair (lq_rebiorth.cu): the pair written by
// an update with defer = 1 is projected against the m earlier pairs, then omega and the scalar
// step are formed from the corrected pair.  Needs the whole right basis and the stored left
// basis (a full left basis: LQ_RESERVE_REBIORTH).
constexpr int kRbThreads = 256;
constexpr int kRbPerThread = 4;           // chunks of each new vector a dot thread holds
inline unsigned rb_dot_blocks(size_t nelem) {
    const size_t per = (size_t)kRbThreads * kRbPerThread;
    return (unsigned)(nelem == 0 ? 1 : (nelem + per - 1) / per);
}
struct RbArgs {
    UpdArgs u;             // the update of this step: new pair slots, state, scalars, partials
    int m;                 // earlier pairs: j + 1
    const void* vbasis;    // right basis vh_0 ..: per source u.src_stride_basis (Chunk units)
    const void* wbasis;    // stored left basis wh_0 ..: per source u.src_stride_store
    size_t vec_stride;     // Chunk elements per basis vector
    const double* scale;   // s_i [src][kmax]
    const double2* uscale; // u_i [src][kmax]
    double* part;          // [src][kmax][dot_blocks][8] block sums of the dots
    unsigned dot_blocks;   // rb_dot_blocks(u.nelem)
    double2* coef;         // [src][2][kmax]: c_i (right), d_i (left)
    float4* coef_f;        // the same split into float-float (re.hi, re.lo, im.hi, im.lo)
};
cudaError_t launch_rebiorth(int prec, const RbArgs& a, cudaStream_t st);
// Deflation vector algebra on FP64 boundary-layout vectors (lq_deflate.cu).  Sizes and strides
// are in doubles (2 per complex number).
cudaError_t launch_bdots(const double* X, size_t xs, int nx, const double* Y, size_t ys, int ny, size_t n,
                         double* partial, double* out, cudaStream_t st);      // out[a * ny + b] = <X_a|Y_b>
cudaError_t launch_bcombine(double* Z, const double* W, size_t zs, int nz, const double* X, size_t xs, int nx,
                            const double* coef, size_t n, cudaStream_t st);   // Z_b = W_b + sum_a coef[b*nx+a] X_a
size_t bdots_partial_doubles(int npairs);
cudaError_t launch_axpby3(double* Z, double a1, const double* X1, double a2, const double* X2, double a3, const double* X3,
                          size_t n, cudaStream_t st);
cudaError_t launch_norm2(const double* a, const double* b, double sigma, size_t n, int nsrc, double* out, cudaStream_t st);
// s <- x + gamma5 s, d <- gamma5 d (d may be null) over nsites boundary-layout sites (Eq. (1.1))
cudaError_t launch_overlap(const double* x, double* s, double* d, size_t nsites, cudaStream_t st);
// Overlap solver (lq_deflate.cu).  Sizes and strides in doubles.
// out[s] = <X_s|Y_s> for nsrc sources; partial: bdots_partial_doubles(nsrc)
cudaError_t launch_sdots(const double* X, const double* Y, size_t stride, size_t n, int nsrc, double* partial, double* out,
                         cudaStream_t st);
// Z_s = c[s][0] X0_s + c[s][1] X1_s + c[s][2] X2_s (complex coef [nsrc][3] on the device)
cudaError_t launch_scomb(double* Z, const double* X0, const double* X1, const double* X2, const double* coef, size_t stride,
                         size_t n, int nsrc, cudaStream_t st);
// out = cx x + cs gamma5 s over nsites boundary-layout sites (x may be null)
cudaError_t launch_g5axpy(double* out, const double* x, double cx, const double* s, double cs, size_t nsites, cudaStream_t st);

// Newton sign iteration (lq_newton.cu)
struct NewtonArgs {
    int k;                 // matrix dimension (padded)
    int nb;                // batch
    int ld;                // leading dimension of the per-matrix storage (>= k)
    double2* X;            // [nb][ld][ld] iterate
    double2* Y;            // [nb][ld][ld] work (inverse)
    double2* F;            // [nb][ld] multipliers
    int* perm;             // [nb][ld]
    double* scal;          // [nb][16] scalars
    double* partials;
    size_t partial_stride;
    int* counters;
    double tol;
    int max_iter;
    // tridiagonal source (Lanczos): may be null when X is initialised densely
    const TslState* state;
    const double2* alpha; const double2* beta; const double* delta;
    int kmax;
};
// scal layout per matrix
enum { NS_NORMX = 0, NS_NORMY, NS_MU, NS_CHANGE, NS_DONE, NS_ITERS, NS_SCALING, NS_STATUS, NS_PREVCHANGE, NS_KEFF };

// Adjoint / force (lq_adjoint.cu)
struct AdjArgs {
    int npairs;            // 2N quadrature terms
    int kmax;
    int nth_max;
    double c;              // contour scale
    const TslState* state; // sources 0 (x) and 1 (y)
    const double2* alpha; const double2* beta; const double* delta;
    const double* scale;   // right scales (source 0 row)
    const double2* uscale; // left scales (source 1 row at offset kmax)
    double2* work;         // quadrature workspace
    double2* cnu;          // [npairs][kmax] coefficients for nu_q
    double2* com;          // [npairs][kmax] coefficients for omega_q
    void* nu; void* om;    // [npairs] internal fields
    // lattice
    size_t V;
    int dims[4];
    size_t strides[4];
    int apbc;
    double efwd, ebwd;     // exp(+mu), exp(-mu)
    const double2* Ub;     // FP64 links, boundary layout [4][V][9]
    double* force;         // [4][V][8]
    double* dmu_part;      // [blocks]
    // deflated adjoint (ndefl = 0 without deflation): the mixed-block vectors d_j v_j and
    // conj(c_j) u_j (coefficient rows 2N + 2l + j of cnu and 2N + l + j of com) and the pairs
    // contracted by k_force (npairs_force, 2N + 3l; 0 means npairs)
    int ndefl;
    int npairs_force;
    const double2* dlam;   // [l] eigenvalues lambda_j
    const double2* dcx;    // [l] c_j = L_j x'  (before deflation: L_j x)
    const double2* ddy;    // [l] d_j = y^H R_j
};
cudaError_t launch_adjoint(int prec, const AdjArgs& a, const void* basis, size_t basis_vec_stride, const void* lbasis,
                           size_t lbasis_vec_stride, int k, cudaStream_t st);
// the same in three parts for a two-pass run: the pair coefficients (after the first pass), the
// pair vectors accumulated over a window [j0, j1) of ring slots (second pass), the contraction
cudaError_t launch_adj_pairs(const AdjArgs& a, cudaStream_t st);
cudaError_t launch_adj_window(int prec, const AdjArgs& a, const void* basis, size_t basis_vec_stride, const void* lbasis,
                              size_t lbasis_vec_stride, int j0, int j1, int ring, cudaStream_t st);
cudaError_t launch_adj_force(int prec, const AdjArgs& a, cudaStream_t st);

// Nested two-sided Lanczos projected sign (lq_nested.cu)
struct NestArgs {
    int nb;                // sources
    int kmax;              // row stride of every per-source array
    int kfix;              // k when state is null
    int m;                 // inner steps
    const TslState* state; // outer k_eff per source, or null
    const double2* alpha; const double2* beta; const double* delta;   // outer T (stride kmax)
    const double* cscale;  // [nb] c of M = T/c + c T^{-1}
    double2* work;         // per source nest_work_entries(kmax, m) complex entries
    size_t work_stride;
    const double2* start;  // [nb][kmax] start vector, or null for e_1
    TslState* istate;      // [nb] inner: k_eff, status
    double2* ialpha; double2* ibeta; double* idelta;   // [nb][kmax] inner coefficients
    double* snorm;         // [nb] |start|
    const int* sel;        // [nb] sources to process, or null for all
};
size_t nest_work_entries(int kmax, int m);
cudaError_t nest_factor(const NestArgs& a, cudaStream_t st);
cudaError_t nest_lanczos(const NestArgs& a, cudaStream_t st);
cudaError_t nest_combine(const NestArgs& a, const double2* sp, double2* out, cudaStream_t st);
cudaError_t nest_check(const NestArgs& a, const double2* q, double* check, cudaStream_t st);

// Quadrature projected sign (lq_newton.cu)
struct QuadArgs {
    int k;                 // padded dimension
    int nb;
    int kmax;              // row stride of alpha/beta/delta/s/q
    int nth_max;           // thread capacity of the work array (2 * max nodes)
    const TslState* state; // [nb] per-source dimension (k_eff)
    const double2* alpha; const double2* beta; const double* delta;
    double* c;             // [nb] contour scale
    double2* work;         // [nb][4][kmax][nth_max]
    const int* nodes;      // [nb] quadrature nodes per source (0: skip the source), sign quadrature only
    double2* part;         // [nb][part_blocks][kmax] per-block row sums of the sign quadrature
    int part_blocks;
    double2* s;            // [nb][kmax] sgn(T) e_1
    double2* q;            // [nb][kmax] sgn(T) s (involution check)
    double* check;         // [nb] ||q - e_1||
};
constexpr int kQuadMaxNodes = 128;        // opts.quad_nodes and the adjoint's rank-one terms
constexpr int kQuadRetryMaxNodes = 2048;  // LQ_PROJ_AUTO retries a failing source once with this many nodes
constexpr int kQuadBlk = 32;              // shifted solves per block of the sign quadrature
constexpr int kQuadFinish = 256;          // threads of the summing kernel
// sgn(T) e_1 and the involution check for the sources with a.nodes[src] > 0 (at most max_nodes;
// contour scales recomputed when `scale`).  a.work needs 2 * max_nodes columns (nth_max).
cudaError_t quad_sign_e1(const QuadArgs& a, int max_nodes, bool scale, cudaStream_t st);
cudaError_t quad_scale(const QuadArgs& a, cudaStream_t st);   // contour scales c only
// c = (sigma_src - T)^{-1} e_1 into a.s (per-source complex shifts, device array)
cudaError_t proj_resolvent(const QuadArgs& a, const double2* shifts, cudaStream_t st);
cudaError_t newton_first_column(const NewtonArgs& a, double2* out, int ldo, cudaStream_t st, const int* sel = nullptr);

cudaError_t newton_init_tridiag(const NewtonArgs& a, cudaStream_t st);
cudaError_t newton_init_dense(const NewtonArgs& a, const double2* Xin, cudaStream_t st);
cudaError_t newton_iteration(const NewtonArgs& a, cudaStream_t st);
cudaError_t newton_copy_out(const NewtonArgs& a, double2* Sout, cudaStream_t st);

}  // namespace lq
