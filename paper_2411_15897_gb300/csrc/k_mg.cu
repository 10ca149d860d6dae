// Multigrid level kernels for the acoustic blocks (Sec. 2.2, Algorithm 1;
// Sec. 4.4.1): damped Jacobi relaxation, residual, restriction (Eq. 4.1, 4.2,
// 4.4), bilinear prolongation and the dense FP64 coarsest solve.  Every kernel
// is batched over the blocks of one set (blockIdx.y = block) so the d
// independent displacement blocks run in one launch.
//
// Level 0 reads the 5-point operator from per-point coefficient arrays
// (Fine5); coarser levels read explicit Galerkin stencils of radius (rx, rz).
#include "bah_internal.cuh"
#include "intergrid.cuh"
#include "mg_device.cuh"

#include <algorithm>
#include <cstdlib>

namespace bah {


template <class LS>
static inline int max_radius(const LS& s) {
    int r = 0;
    for (int z = 0; z < s.nb; ++z) r = std::max(r, std::max(s.blk[z].rx, s.blk[z].rz));
    return r;
}

// ---------------------------------------------------------------------------
// damped Jacobi:  x_out = x_in + w D^{-1} (b - A x_in)   (zero_init: w D^{-1} b)
// ---------------------------------------------------------------------------
template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_jacobi(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                typename MGT<MODE>::R w, int zero_init) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.z;
    if (t >= np || (s.active && !s.active[rr])) return;
    V* __restrict__ xout = B.xout + rr * B.sxo;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) { xout[t] = czero<V>(); return; }
    const V b = B.b[rr * B.sb + t];
    if (zero_init) {
        const V dg = diag_only<MODE>(L0 ? &f5 : nullptr, B, np, t);
        xout[t] = cscale(cdiv(b, dg), w);
        return;
    }
    const V* __restrict__ xin = B.xin + rr * B.sxi;
    auto X = [&](int g) { return xin[g]; };
    V ax;
    if (L0) ax = apply_fine5_fn<MODE>(f5, B.type, i, j, t, X);
    else ax = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, i, j, t, X);
    const V dg = diag_only<MODE>(L0 ? &f5 : nullptr, B, np, t);
    const V corr = cdiv(csub(b, ax), dg);
    const V x = xin[t];
    xout[t] = cmk<V>(x.x + w * corr.x, x.y + w * corr.y);
}

// ---------------------------------------------------------------------------
// residual:  r = b - A x
// ---------------------------------------------------------------------------
template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_residual(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                  Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.z;
    if (t >= np || (s.active && !s.active[rr])) return;
    V* __restrict__ xout = B.xout + rr * B.sxo;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) { xout[t] = czero<V>(); return; }
    const V* __restrict__ xin = B.xin + rr * B.sxi;
    auto X = [&](int g) { return xin[g]; };
    V ax;
    if (L0) ax = apply_fine5_fn<MODE>(f5, B.type, i, j, t, X);
    else ax = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, i, j, t, X);
    xout[t] = csub(B.b[rr * B.sb + t], ax);
}

// ---------------------------------------------------------------------------
// Jacobi sweep (RES = false) or residual (RES = true) on a Galerkin level with
// the CTA's inputs staged in shared memory first: every stencil coefficient of
// its 256 points and the iterate over the points' rows plus RM rows on each
// side are requested with asynchronous copies (cp.async) before any is used,
// so the number of loads in flight no longer depends on how many registers
// the compiler keeps for them.  Arithmetic as in k_jacobi / k_residual.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
template <class T>
__device__ __forceinline__ void cpa(T* dst, const T* src) {
    if constexpr (sizeof(T) == 4) cpa4(dst, src);
    else if constexpr (sizeof(T) == 8) cpa8(dst, src);
    else cpa16(dst, src);
}

template <int MODE, int RM, bool RES>
__global__ void __launch_bounds__(256) k_stencil_staged(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                        typename MGT<MODE>::R w) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using CC = typename MGT<MODE>::CC;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int rr = blockIdx.z;
    if (s.active && !s.active[rr]) return;              // uniform over the CTA
    const int t0 = blockIdx.x * 256;
    const int nsl = (2 * B.rx + 1) * (2 * B.rz + 1);
    const int halo = RM * n1 + RM;
    const int xbase = t0 - halo, xlen = 256 + 2 * halo;
    extern __shared__ __align__(16) unsigned char stage_raw[];
    V* xs = reinterpret_cast<V*>(stage_raw);
    CC* cs = reinterpret_cast<CC*>(stage_raw + (size_t)xlen * sizeof(V));
    const V* __restrict__ xin = B.xin + rr * B.sxi;
    for (int e = threadIdx.x; e < xlen; e += 256) {
        const int g = xbase + e;
        if (g >= 0 && g < np) cpa(xs + e, xin + g);
    }
    for (int e = threadIdx.x; e < nsl * 256; e += 256) {
        const int g = t0 + (e & 255);
        if (g < np) cpa(cs + e, B.S + (size_t)(e >> 8) * np + g);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int t = t0 + threadIdx.x;
    if (t >= np) return;
    V* __restrict__ xout = B.xout + rr * B.sxo;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) { xout[t] = czero<V>(); return; }
    auto X = [&](int g) { return xs[g - xbase]; };
    auto S = [&](int slot) { return cs[slot * 256 + threadIdx.x]; };
    const V ax = apply_stencil_acc<MODE, RM>(S, B.rx, B.rz, n1, n2, i, j, t, X);
    const V b = B.b[rr * B.sb + t];
    if (RES) {
        xout[t] = csub(b, ax);
    } else {
        const V dg = ldc(S(B.rz * (2 * B.rx + 1) + B.rx));
        const V corr = cdiv(csub(b, ax), dg);
        const V x = X(t);
        xout[t] = cmk<V>(x.x + w * corr.x, x.y + w * corr.y);
    }
}

// bytes of shared memory the staged kernel needs on this set (0: use the plain kernel)
template <int MODE>
static size_t staged_smem(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s, int rm) {
    if (!s.staged || MODE != BAH_MIXED) return 0;
    int nsl = 0;
    for (int z = 0; z < s.nb; ++z) nsl = std::max(nsl, (2 * s.blk[z].rx + 1) * (2 * s.blk[z].rz + 1));
    const size_t xlen = 256 + 2 * ((size_t)rm * s.n1 + rm);
    const size_t bytes = xlen * sizeof(typename Prec<MODE>::V) + (size_t)nsl * 256 * sizeof(typename Prec<MODE>::CC);
    return bytes <= 48 * 1024 ? bytes : 0;
}

template <int MODE>
void launch_jacobi(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                   const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w, int zero_init,
                   cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb, s.nrhs);
    using R = typename Prec<MODE>::R;
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    const int rm = f5 ? 1 : max_radius(s);
    const size_t sm = (f5 || zero_init) ? 0 : staged_smem<MODE>(s, rm);
    if (f5) launch_pdl(k_jacobi<MODE, true, 1>, dim3(g), dim3(256), 0, st, s, *f5, (R)w, zero_init);
    else if (sm && rm <= 1) launch_pdl(k_stencil_staged<MODE, 1, false>, dim3(g), dim3(256), sm, st, s, (R)w);
    else if (sm) launch_pdl(k_stencil_staged<MODE, 2, false>, dim3(g), dim3(256), sm, st, s, (R)w);
    else if (rm <= 1) launch_pdl(k_jacobi<MODE, false, 1>, dim3(g), dim3(256), 0, st, s, nof, (R)w, zero_init);
    else launch_pdl(k_jacobi<MODE, false, 2>, dim3(g), dim3(256), 0, st, s, nof, (R)w, zero_init);
}
template <int MODE>
void launch_residual(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                     const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb, s.nrhs);
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    using R = typename Prec<MODE>::R;
    const int rm = f5 ? 1 : max_radius(s);
    const size_t sm = f5 ? 0 : staged_smem<MODE>(s, rm);
    if (f5) launch_pdl(k_residual<MODE, true, 1>, dim3(g), dim3(256), 0, st, s, *f5);
    else if (sm && rm <= 1) launch_pdl(k_stencil_staged<MODE, 1, true>, dim3(g), dim3(256), sm, st, s, (R)0);
    else if (sm) launch_pdl(k_stencil_staged<MODE, 2, true>, dim3(g), dim3(256), sm, st, s, (R)0);
    else if (rm <= 1) launch_pdl(k_residual<MODE, false, 1>, dim3(g), dim3(256), 0, st, s, nof);
    else launch_pdl(k_residual<MODE, false, 2>, dim3(g), dim3(256), 0, st, s, nof);
}

// ---------------------------------------------------------------------------
// restriction: b_c = R r_f  (r_f in blk.xout of the fine set)
// ---------------------------------------------------------------------------

// support of a 1-D restriction row for coarse index c: first fine index

template <int MODE>
__global__ void __launch_bounds__(256) k_restrict(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> fine,
                                                  PtrSet<typename MGT<MODE>::V> cb, int intergrid) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = fine.blk[blockIdx.y];
    const int n1 = fine.n1, n2 = fine.n2, n1c = n1 / 2, n2c = n2 / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.z;
    if (t >= n1c * n2c || (fine.active && !fine.active[rr])) return;
    const int I = t % n1c, J = t / n1c;
    V acc = czero<V>();
    if (valid_pt(B.type, I, J)) {
        const bool nodx = B.type == 0, nodz = B.type == 1;
        const V* r = B.xout + rr * B.sxo;
        const int bx = rbase(nodx, intergrid, I), bz = rbase(nodz, intergrid, J);
        R wxs[4], wzs[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            wxs[q] = rw_axis_t<R>(nodx, intergrid, n1, I, bx + q);
            wzs[q] = rw_axis_t<R>(nodz, intergrid, n2, J, bz + q);
        }
        V v[16];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = wzs[a] != R(0) && wxs[q] != R(0);
                v[a * 4 + q] = r[ok ? (bz + a) * n1 + (bx + q) : 0];
            }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const R wgt = wzs[a] * wxs[q];
                acc.x += wgt * v[a * 4 + q].x;
                acc.y += wgt * v[a * 4 + q].y;
            }
    }
    pick(cb, (int)blockIdx.y)[rr * cb.s + t] = acc;
}

template <int MODE>
void launch_restrict(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                     typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st, size_t coarse_stride) {
    PtrSet<typename Prec<MODE>::V> cb;
    for (int z = 0; z < 3; ++z) cb.p[z] = z < fine.nb ? coarse_b[z] : nullptr;
    cb.s = coarse_stride;
    const int npc = (fine.n1 / 2) * (fine.n2 / 2);
    dim3 g((npc + 255) / 256, fine.nb, fine.nrhs);
    launch_pdl(k_restrict<MODE>, dim3(g), dim3(256), 0, st, fine, cb, intergrid);
}

// ---------------------------------------------------------------------------
// prolongation and correction: x_f += P e_c  (x_f = blk.xout of the fine set)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_prolong_add(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> fine,
                                                     PtrSet<typename MGT<MODE>::V> ce) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = fine.blk[blockIdx.y];
    const int n1 = fine.n1, n2 = fine.n2, n1c = n1 / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.z;
    if (t >= n1 * n2 || (fine.active && !fine.active[rr])) return;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) return;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    const V* e = pick(ce, (int)blockIdx.y) + rr * ce.s;
    V* xo = B.xout + rr * B.sxo;
    R px[3], pz[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        px[q] = pw_axis_t<R>(nodx, n1, i, (i >> 1) - 1 + q);
        pz[q] = pw_axis_t<R>(nodz, n2, j, (j >> 1) - 1 + q);
    }
    V v[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const bool ok = pz[a] != R(0) && px[q] != R(0);
            v[a * 3 + q] = e[ok ? ((j >> 1) - 1 + a) * n1c + ((i >> 1) - 1 + q) : 0];
        }
    V acc = xo[t];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const R wgt = pz[a] * px[q];
            acc.x += wgt * v[a * 3 + q].x;
            acc.y += wgt * v[a * 3 + q].y;
        }
    xo[t] = acc;
}

template <int MODE>
void launch_prolong_add(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                        const typename Prec<MODE>::V* const* coarse_x, cudaStream_t st, size_t coarse_stride) {
    PtrSet<typename Prec<MODE>::V> ce;
    for (int z = 0; z < 3; ++z) ce.p[z] = z < fine.nb ? const_cast<typename Prec<MODE>::V*>(coarse_x[z]) : nullptr;
    ce.s = coarse_stride;
    const int np = fine.n1 * fine.n2;
    dim3 g((np + 255) / 256, fine.nb, fine.nrhs);
    launch_pdl(k_prolong_add<MODE>, dim3(g), dim3(256), 0, st, fine, ce);
}

// ---------------------------------------------------------------------------
// coarsest level: x = A_c^{-1} b with the stored FP64 inverse (one warp per
// row).  The product is formed in FP64 in both modes -- the coarsest-grid
// solve is one of the steps kept in FP64 -- from the right-hand side in the
// cycle's precision; the result is rounded once to the cycle's precision.
// Each lane issues its eight row loads before the first multiply-add.
// ---------------------------------------------------------------------------
constexpr int kCoarseSmem = 3072;   // points staged in shared memory

template <class V>
__global__ void __launch_bounds__(256) k_coarse_apply(int npts, PtrSet<const double2> inv, PtrSet<const V> b,
                                                      PtrSet<V> x, const int* active) {
    pdl_prologue();
    const int z = blockIdx.y;
    const int rr = blockIdx.z;
    if (active && !active[rr]) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char coarse_raw[];
    V* bsh = reinterpret_cast<V*>(coarse_raw);
    const V* bb = pick(b, z) + rr * b.s;
    const bool staged = npts <= kCoarseSmem;
    if (staged) {
        for (int c = threadIdx.x; c < npts; c += blockDim.x) bsh[c] = bb[c];
        __syncthreads();
    }
    if (warp >= npts) return;
    const double2* row = pick(inv, z) + (size_t)warp * npts;
    double re = 0.0, im = 0.0;
    auto mac = [&](const double2& a, const V& v) {
        const double vx = (double)v.x, vy = (double)v.y;
        re = fma(a.x, vx, re);
        re = fma(-a.y, vy, re);
        im = fma(a.x, vy, im);
        im = fma(a.y, vx, im);
    };
    constexpr int kU = 8;
    int c = lane;
    for (; c + 32 * (kU - 1) < npts; c += 32 * kU) {
        double2 a[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) a[u] = __ldg(row + c + 32 * u);
#pragma unroll
        for (int u = 0; u < kU; ++u) mac(a[u], staged ? bsh[c + 32 * u] : bb[c + 32 * u]);
    }
    for (; c < npts; c += 32) mac(__ldg(row + c), staged ? bsh[c] : bb[c]);
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) pick(x, z)[rr * x.s + warp] = cmk<V>((typename VecTraits<V>::R)re, (typename VecTraits<V>::R)im);
}

template <int MODE>
void launch_coarse_apply(int nb, int npts, const double2* const* inv, const typename Prec<MODE>::V* const* b,
                         typename Prec<MODE>::V* const* x, cudaStream_t st, int nrhs, RhsStride rs) {
    using V = typename Prec<MODE>::V;
    PtrSet<const double2> pi;
    PtrSet<const V> pb;
    PtrSet<V> px;
    for (int z = 0; z < 3; ++z) {
        pi.p[z] = z < nb ? inv[z] : nullptr;
        pb.p[z] = z < nb ? b[z] : nullptr;
        px.p[z] = z < nb ? x[z] : nullptr;
    }
    pb.s = rs.s0;
    px.s = rs.s1;
    dim3 g((npts * 32 + 255) / 256, nb, nrhs);
    const size_t smem = npts <= kCoarseSmem ? (size_t)npts * sizeof(V) : 0;
    launch_pdl(k_coarse_apply<V>, dim3(g), dim3(256), smem, st, npts, pi, pb, px, rs.active);
}

// ---------------------------------------------------------------------------
// one acoustic block's fine operator in FP64 (the 5-point stencil of Eq. 2.6 /
// 3.4 with the diagonals given in f5): y = A x, or y = b - A x.  The operator
// of the inner block solves of the exact-block preconditioner.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_block_apply64(Fine5<double, double2> f5, int type,
                                                       const double2* __restrict__ x, double2* __restrict__ y,
                                                       const double2* __restrict__ b) {
    pdl_prologue();
    const int n1 = f5.n1, n2 = f5.n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n1 * n2) return;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(type, i, j)) { y[t] = make_double2(0.0, 0.0); return; }
    const double2 ax = apply_fine5_fn<BAH_FP64>(f5, type, i, j, t, [&](int g) { return x[g]; });
    y[t] = b ? csub(b[t], ax) : ax;
}
void launch_block_apply64(const Fine5<double, double2>& f5, int type, const double2* x, double2* y, const double2* b,
                          cudaStream_t st) {
    const int np = f5.n1 * f5.n2;
    launch_pdl(k_block_apply64, dim3((np + 255) / 256), dim3(256), 0, st, f5, type, x, y, b);
}

#define INST(MODE)                                                                                                 \
    template void launch_jacobi<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                                \
                                      const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double, int, cudaStream_t);     \
    template void launch_residual<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                              \
                                        const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, cudaStream_t);                \
    template void launch_restrict<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&, Prec<MODE>::V* const*, int,  \
                                        cudaStream_t, size_t);                                                     \
    template void launch_prolong_add<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                           \
                                           const Prec<MODE>::V* const*, cudaStream_t, size_t);                     \
    template void launch_coarse_apply<MODE>(int, int, const double2* const*, const Prec<MODE>::V* const*,   \
                                            Prec<MODE>::V* const*, cudaStream_t, int, RhsStride);
INST(BAH_FP64)
INST(BAH_MIXED)

}  // namespace bah
