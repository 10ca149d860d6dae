// Internal declarations shared by the CUDA translation units of libbah.
//
// Grid conventions (2-D): n1 x n2 cells, x_1 fastest, point (i, j) at index
// j*n1 + i.  Every acoustic block lives on the same padded n1 x n2 index
// space at each level; its unknowns are
//   type 0 (u1, nodal along x_1): i >= 1
//   type 1 (u2, nodal along x_2): j >= 1
//   type 2 (p,  cell-centred):    all points
// and the remaining (boundary-normal) points hold structural zeros.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bah.h"

namespace bah {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Hot kernels begin with pdl_prologue(): wait
// until the preceding kernel of the stream has completed and flushed its
// memory (so nothing produced upstream is read early and nothing read
// upstream is overwritten early), then allow the next kernel to start
// launching.  Launched with launch_pdl(), the next kernel's launch overlaps
// this kernel's execution; launched normally, both instructions are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// thread-block cluster: hardware barrier over all threads of all CTAs of the
// cluster (release/acquire at cluster scope: shared and global memory writes
// before it are visible to every thread of the cluster after it), the CTA's
// rank, the cluster's CTA count, and the cluster's index in the grid (x)
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_nrank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// NVTX range over a host scope (setup phases, solves, restart cycles, FGMRES
// steps), visible in a timeline profiler; costs nothing when none is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// precision traits: V = complex vector element, R = real arithmetic type,
// C / CC = stored real / complex coefficient types
// ---------------------------------------------------------------------------
template <int MODE> struct Prec;
template <> struct Prec<BAH_FP64> {
    using V = double2; using R = double; using C = double; using CC = double2;
};
template <> struct Prec<BAH_MIXED> {
    using V = float2; using R = float; using C = __nv_bfloat16; using CC = __nv_bfloat162;
};

__host__ __device__ __forceinline__ double ldr(double x) { return x; }
__device__ __forceinline__ float ldr(__nv_bfloat16 x) { return __bfloat162float(x); }
__host__ __device__ __forceinline__ double2 ldc(double2 x) { return x; }
__device__ __forceinline__ float2 ldc(__nv_bfloat162 x) { return __bfloat1622float2(x); }

template <class V> struct VecTraits;
template <> struct VecTraits<double2> { using R = double; };
template <> struct VecTraits<float2> { using R = float; };

// complex helpers (x = re, y = im)
template <class V> __host__ __device__ __forceinline__ V cmk(typename VecTraits<V>::R a, typename VecTraits<V>::R b) { V v; v.x = a; v.y = b; return v; }
template <class V> __host__ __device__ __forceinline__ V czero() { return cmk<V>(0, 0); }
template <class V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <class V> __host__ __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <class V> __host__ __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class V> __host__ __device__ __forceinline__ V cscale(V a, typename VecTraits<V>::R s) { return cmk<V>(a.x * s, a.y * s); }
template <class V> __host__ __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
// a * conj-free reciprocal: b / a
template <class V> __host__ __device__ __forceinline__ V cdiv(V b, V a) {
    typename VecTraits<V>::R d = a.x * a.x + a.y * a.y;
    return cmk<V>((b.x * a.x + b.y * a.y) / d, (b.y * a.x - b.x * a.y) / d);
}
template <class To, class From> __host__ __device__ __forceinline__ To cconv(From a) {
    return cmk<To>((typename VecTraits<To>::R)a.x, (typename VecTraits<To>::R)a.y);
}

__host__ __device__ __forceinline__ bool valid_pt(int type, int i, int j) {
    return (type == 0) ? (i >= 1) : (type == 1) ? (j >= 1) : true;
}

// ---------------------------------------------------------------------------
// operator coefficients of H (FP64, Eq. 2.6), all pre-scaled by 1/h^2 or 1/h
// ---------------------------------------------------------------------------
struct OpCoef {
    int n1, n2;
    const double* cx;    // mu_c / h1^2 at cells     (u1 own-direction, x-neighbours)
    const double* cz;    // mu_c / h2^2 at cells     (u2 own-direction)
    const double* nx;    // mu_node / h1^2 at nodes (i,j), zero on boundary nodes
    const double* nz;    // mu_node / h2^2
    const double2* d1;   // diagonal of A_1 incl. -omega^2 rho~ (unshifted)
    const double2* d2;   // diagonal of A_2
    const double* cinv;  // 1 / (lambda + mu)
    double ihx, ihz;     // 1/h1, 1/h2
};

// the same coefficients as double-float pairs (hi, lo), for the operator
// applied to FP32 vectors in double-float arithmetic
struct OpCoefDF {
    int n1, n2;
    const float2 *cx, *cz, *nx, *nz, *cinv;
    const float4 *d1, *d2;
    float2 ihx, ihz;
};

// ---------------------------------------------------------------------------
// multigrid level-0 (fine) operators: 5-point stencils from per-point arrays
// (Eq. 2.6 blocks with the shift of Eq. 2.8; H_p,s of Eq. 3.4; A_p of Eq. 3.2)
// ---------------------------------------------------------------------------
template <class C, class CC> struct Fine5 {
    int n1, n2;
    const C *cx, *cz, *nx, *nz;   // as OpCoef
    const C *wx, *wz;             // w / h^2, w = (lambda+2mu)/(lambda+mu)  (H_p off-diagonals)
    const CC *dg0, *dg1, *dg2;    // shifted diagonals of A_1,s, A_2,s, H_p,s
    const CC *dAp;                // diagonal of A_p (unshifted)
};

// one block's data on one level, for batched launches over blocks
template <class V, class CC> struct LvlBlk {
    int type;
    const CC* S;       // stencil [(2rz+1)(2rx+1)][n1*n2] (levels >= 1)
    int rx, rz;
    const V* b;        // right-hand side
    const V* xin;      // current iterate
    V* xout;           // output iterate / residual
    size_t sb, sxi, sxo;   // element strides between right-hand sides (blockIdx.z)
};
template <class V, class CC> struct LvlSet {
    int nb;            // blocks in the set (1..3)
    int n1, n2;        // level grid
    LvlBlk<V, CC> blk[3];
    int nrhs;          // right-hand sides in the launch (blockIdx.z)
    const int* active; // per right-hand side, or nullptr
    int staged;        // Galerkin-level sweeps may stage their inputs in shared memory
};

constexpr int kMaxLevels = 16;
// shared-memory-resident cluster multigrid (mixed mode): levels l0 .. L-1 of
// one block set, one cluster per block and right-hand side; lv[k] is level
// l0 + k, its rows split in slabs of rp rows per CTA, and off_* are byte
// offsets of its arrays in each CTA's dynamic shared memory
struct SmLevel {
    int n1, n2, rp;
    float inv_rp, inv_n1;     // 1/rp and 1/n1 (row and column from a flat or row index)
    float w;                  // Jacobi damping
    unsigned off_c, off_x, off_t, off_b;
};
struct SmArgs {
    SmLevel lv[kMaxLevels];
    int nlev, b0, nb, nu_pre, nu_post, intergrid, wcycle, warm;
    int rx[2][kMaxLevels], rz[2][kMaxLevels];
    const __nv_bfloat162* S[2][kMaxLevels];   // global stencils (levels below the coarsest)
    const float2* gb[2];      // level-l0 right-hand sides (right-hand side r at r * points)
    float2* gx[2];            // level-l0 iterates / results
    const double2* inv[2];    // coarsest FP64 inverses (global memory; the product is formed in FP64)
    unsigned off_g;           // gathered coarsest right-hand side
    const int* active;
};
// fills the shared-memory layout of a (n1, n2, slot counts per level from l0);
// returns the bytes of dynamic shared memory per CTA
size_t smmg_layout(SmArgs& a, const int* n1, const int* n2, const int* nslot_max, int nlev, int cs);
// sets the kernel attributes; returns how many clusters of cs CTAs fit (0: none)
int smmg_prepare(int rm, int cs, size_t smem);
int launch_cluster_mg(const SmArgs& a, int rm, int nrhs, int cs, size_t smem, cudaStream_t st);

// right-hand-side batching: element strides between consecutive right-hand
// sides for up to three pointers of a launch (blockIdx.y or .z is the
// right-hand side), and an optional per-right-hand-side active flag
struct RhsStride {
    size_t s0 = 0, s1 = 0, s2 = 0;
    const int* active = nullptr;
};

// FP64 stencil of one block on one level (setup and test hook)
struct StencilF64 {
    double2* S = nullptr;   // [(2rz+1)(2rx+1)][n1*n2]
    int rx = 1, rz = 1;
    int n1 = 0, n2 = 0;
};

// ---------------------------------------------------------------------------
// launchers (host functions, all asynchronous on `st`)
// ---------------------------------------------------------------------------
// setup (k_setup.cu)
void launch_medium_prep(int n1, int n2, double h1, double h2, double omega, double alpha,
                        const double* lam, const double* mu, const double* rho, const double* gam,
                        double* cx, double* cz, double* nx, double* nz, double* wx, double* wz,
                        double2* d1, double2* d2, double* cinv,
                        double2* dg0, double2* dg1, double2* dg2, double2* dAp, cudaStream_t st);
void launch_fine_stencil(int type, int n1, int n2, const double* cx, const double* cz, const double* nx,
                         const double* nz, const double* wx, const double* wz, const double2* dg,
                         double2* S, cudaStream_t st);
void launch_galerkin(int type, int intergrid, const StencilF64& fine, StencilF64& coarse, cudaStream_t st);
void launch_round_real(const double* src, void* dst, size_t n, int mode, cudaStream_t st);
void launch_round_cplx(const double2* src, void* dst, size_t n, int mode, cudaStream_t st);
int  coarse_invert(int type, const StencilF64& S, double2* inv, double2* work, int* piv_work, cudaStream_t st);

// operator (k_ops.cu)
template <class Vin>
void launch_elastic_apply(const OpCoef& c, const Vin* x, double2* y, const double2* b, int conj, cudaStream_t st,
                          int nrhs = 1, RhsStride rs = RhsStride());
// y = H x written as double-float (float4) for the double-float Krylov basis
template <class Vin>
void launch_elastic_apply_df(const OpCoef& c, const Vin* x, float4* y, cudaStream_t st, int nrhs, RhsStride rs);
// y = H x for FP32 x in double-float arithmetic (no FP64 instructions), y as double-float
void launch_elastic_apply_dfa(const OpCoefDF& c, const float2* x, float4* y, cudaStream_t st, int nrhs, RhsStride rs);
// the same, rounded once to FP64 on output (the FP64 Krylov basis)
void launch_elastic_apply_dfa(const OpCoefDF& c, const float2* x, double2* y, cudaStream_t st, int nrhs, RhsStride rs);
// FP64 arrays to double-float pairs
void launch_to_df(const double* src, float2* dst, size_t n, cudaStream_t st);
void launch_to_df_c(const double2* src, float4* dst, size_t n, cudaStream_t st);

// multigrid (k_mg.cu)
template <int MODE>
void launch_jacobi(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                   const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w, int zero_init,
                   cudaStream_t st);
template <int MODE>
void launch_residual(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                     const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, cudaStream_t st);
template <int MODE>
void launch_restrict(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                     typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st, size_t coarse_stride = 0);
template <int MODE>
void launch_prolong_add(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                        const typename Prec<MODE>::V* const* coarse_x, cudaStream_t st, size_t coarse_stride = 0);
template <int MODE>
void launch_coarse_apply(int nb, int npts, const double2* const* inv, const typename Prec<MODE>::V* const* b,
                         typename Prec<MODE>::V* const* x, cudaStream_t st, int nrhs = 1, RhsStride rs = RhsStride());
template <int MODE, class RIN = double2>
void launch_distributor(int n1, int n2, double ihx, double ihz,
                        const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>& f5,
                        const RIN* r, typename Prec<MODE>::V* tp, cudaStream_t st, int nrhs = 1,
                        RhsStride rs = RhsStride());
template <int MODE, class RIN = double2>
void launch_u_rhs(int n1, int n2, double ihx, double ihz, const RIN* r, const typename Prec<MODE>::V* ep,
                  typename Prec<MODE>::V* su1, typename Prec<MODE>::V* su2, cudaStream_t st, int nrhs = 1,
                  RhsStride rs = RhsStride());
// y = A x (b null) or y = b - A x for one acoustic block's FP64 fine operator
void launch_block_apply64(const Fine5<double, double2>& f5, int type, const double2* x, double2* y, const double2* b,
                          cudaStream_t st);
void launch_sanitize(double2* v, int n1, int n2, int nvec, cudaStream_t st);
template <class Vin, class Vout>
void launch_convert(const Vin* x, Vout* y, size_t n, cudaStream_t st);

// Krylov (k_krylov.cu), batched over right-hand sides
constexpr int RED_CTAS = 296;   // partial sums per reduction (2 per SM on 148+ SMs)
struct KS {                     // per-right-hand-side element strides and active flags
    size_t sv = 0;              // basis V (m+1 vectors)
    size_t sw = 0;              // work vector w
    size_t sp = 0;              // dot partials
    size_t so = 0;              // small per-rhs arrays (h1, h2, cs, sn, g, y)
    size_t sh = 0;              // Hessenberg matrix
    size_t sz = 0;              // flexible basis Z
    size_t sx = 0;              // solution x
    const int* active = nullptr;
};
void launch_dot_norm(const double2* V, int k, const double2* w, size_t n, double2* partial, double2* out,
                     const int* flag, int nrhs, const KS& ks, cudaStream_t st);
void launch_axpy_norm(const double2* V, int k, const double2* coef, double2* w, size_t n, double* npart,
                      const int* flag, int nrhs, const KS& ks, cudaStream_t st);
// flag = 1 (second pass) when ||w'||^2 < eta2 ||w||^2 (DGKS criterion; eta2 = 1/2 classically)
void launch_dgks_decide(const double* npart, const double2* h1norm, int k, int* flag, double* sc, int nrhs,
                        const KS& ks, cudaStream_t st, double eta2 = 0.5);
void launch_pass2_norm(const double* npart, const int* flag, double* sc, int nrhs, const KS& ks, cudaStream_t st);
void launch_norm2(const double2* w, size_t n, double* partial, double* sc, int slot, int nrhs, const KS& ks,
                  cudaStream_t st);
template <class Vz>
void launch_update_x(const Vz* Z, const int* kk, const double2* y, double2* x, size_t n, int nrhs, const KS& ks,
                     cudaStream_t st);
void launch_sub(const double2* a, const double2* b, double2* c, size_t n, cudaStream_t st);
void launch_scale_copy(const double2* w, const double* sc, int slot, double2* v, size_t n, size_t sw, size_t sv,
                       int nrhs, const KS& ks, cudaStream_t st);
void launch_arnoldi_givens(double2* Hm, int ldh, const double2* h1, const double2* h2, const double* sc, int j,
                           double2* cs, double2* sn, double2* g, double* status, int nrhs, const KS& ks,
                           cudaStream_t st);
void launch_triangular_solve(const double2* Hm, int ldh, const double2* g, const int* kk, double2* y, int nrhs,
                             const KS& ks, cudaStream_t st);
void launch_init_arnoldi(const double* sc, double2* g, int m, double* status, int nrhs, const KS& ks, cudaStream_t st);

// double-float Krylov kernels (k_krylov_df.cu)
void launch_dot_norm_df(const float4* V, int k, const float4* w, size_t n, double2* partial, double2* out,
                        const int* flag, int nrhs, const KS& ks, cudaStream_t st);
void launch_axpy_norm_df(const float4* V, int k, const double2* coef, float4* w, size_t n, double* npart,
                         const int* flag, int nrhs, const KS& ks, cudaStream_t st);
void launch_scale_copy_df(const void* w, bool from64, const double* sc, int slot, float4* v, size_t n, size_t sw,
                          size_t sv, int nrhs, const KS& ks, cudaStream_t st);

// block FGMRES kernels (k_block.cu); s <= 16 columns; rows of A (and Z) for
// block i, column a at A + a * sa + i * n
void launch_block_dot(const double2* A, size_t sa, int k, int s, const double2* W, size_t n, double2* partial,
                      double2* C, cudaStream_t st);
void launch_block_update(const double2* A, size_t sa, int k, int s, const double2* C, double2* W, size_t n,
                         int subtract, cudaStream_t st);
void launch_block_scale(const double2* W, int s, const double2* T, double2* V, size_t sv, size_t n, cudaStream_t st);
template <class Vz>
void launch_block_xupdate(const Vz* Z, size_t sz, int k, int s, const double2* Y, double2* X, size_t n,
                          cudaStream_t st);
// allow the block update kernels the given dynamic shared memory
void block_kernels_smem(size_t bytes);

// adjoint gradient (k_grad.cu)
void launch_conj(double2* v, size_t n, cudaStream_t st);
void launch_misfit(const double2* x, const double2* d, const int* rec, int nrec, int nrhs, size_t vlen, double2* adj,
                   double* misfit, cudaStream_t st);
void launch_gradient(int n1, int n2, double h1, double h2, double omega, const double* cinv, const double* gamma,
                     size_t vlen, int nrhs, const double2* X, const double2* Y, double* gl, double* gm, double* gr,
                     cudaStream_t st);

// three-dimensional grids (k_3d.cu).  FP64 operator coefficients of H on
// n[0] x n[1] x n[2] cells; mue[e] is the edge mean of mu for the pair of axes
// other than e, zero on boundary edges.
struct Op3 {
    int n[3];
    double ih[3], ih2[3];     // 1/h_a, 1/h_a^2
    const double* muc;        // mu at cells
    const double* mue[3];
    const double2* dg[3];     // diagonal of A_a (unshifted, with -omega^2 A_f(rho~))
    const double* cinv;       // 1/(lambda+mu)
    const double2* mrt;       // omega^2 rho~ at cells
};
void launch_prep3(const Op3& op, double omega, double alpha, const double* lam, const double* mu, const double* rho,
                  const double* gam, double* cinv, double2* mrt, double* const* mue, double2* const* dg,
                  double2* const* S, cudaStream_t st);
template <class Vin>
void launch_apply3(const Op3& op, const Vin* x, double2* y, const double2* b, int conj, int nrhs, size_t sx, size_t sy,
                   size_t sb, cudaStream_t st);
void launch_sanitize3(double2* v, int n1, int n2, int n3, int nvec, cudaStream_t st);
template <class V>
void launch_distrib3(const Op3& op, const double2* r, V* tp, cudaStream_t st);
template <class V>
void launch_urhs3(const Op3& op, const double2* r, const V* ep, V* const* su, cudaStream_t st);
// the level kernels run blocks type0 .. type0 + nq - 1 (nq <= 3) of one level in
// one launch, block y on the y-th pointer of each array
template <class V>
// S: stencil entries, FP64 complex (V = double2) or bfloat16 complex (V = float2)
void launch_jacobi3(int type0, int nq, const int* n, int ns, const void* const* S, const V* const* b,
                    const V* const* xin, V* const* xout, double w, int zero, int res, cudaStream_t st);
template <class V>
void launch_restrict3(int type0, int nq, const int* nf, const V* const* r, V* const* bc, cudaStream_t st);
template <class V>
void launch_prolong3(int type0, int nq, const int* nf, const V* const* ec, V* const* x, cudaStream_t st);
void launch_galerkin3(int type, const int* nf, int nsf, const double2* Sf, double2* Sc, int* err, cudaStream_t st);
int coarse_invert3(int type, const int* n, const double2* S, double2* inv, double2* work, int* flag, cudaStream_t st);
// dense FP64 inverse X = A^{-1} of an n x n matrix by Gauss-Jordan elimination
// (A is overwritten; X enters as the identity; f holds n scratch entries)
int gauss_jordan(int n, double2* A, double2* X, double2* f, int* flag, cudaStream_t st);

// error handling
void set_error(const std::string& msg);
}  // namespace bah

#define BAH_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            bah::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));           \
            return BAH_ERR_CUDA;                                                            \
        }                                                                                   \
    } while (0)
