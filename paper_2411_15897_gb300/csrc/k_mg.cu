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

// A x and diag(A) at point t of a level-0 block
template <int MODE>
__device__ __forceinline__ void apply_fine5(const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>& f, int type,
                                            int i, int j, int t, const typename MGT<MODE>::V* __restrict__ x,
                                            typename MGT<MODE>::V& ax, typename MGT<MODE>::V& dg) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const int n1 = f.n1, n2 = f.n2;
    const auto* dgp = type == 0 ? f.dg0 : (type == 1 ? f.dg1 : f.dg2);
    dg = ldc(dgp[t]);
    V acc = cmul(dg, x[t]);
    auto sub = [&](R k, V v) { acc.x -= k * v.x; acc.y -= k * v.y; };
    if (type == 0) {
        if (i - 1 >= 1) sub(ldr(f.cx[t - 1]), x[t - 1]);
        if (i + 1 <= n1 - 1) sub(ldr(f.cx[t]), x[t + 1]);
        if (j >= 1) sub(ldr(f.nz[t]), x[t - n1]);
        if (j + 1 <= n2 - 1) sub(ldr(f.nz[t + n1]), x[t + n1]);
    } else if (type == 1) {
        if (j - 1 >= 1) sub(ldr(f.cz[t - n1]), x[t - n1]);
        if (j + 1 <= n2 - 1) sub(ldr(f.cz[t]), x[t + n1]);
        if (i >= 1) sub(ldr(f.nx[t]), x[t - 1]);
        if (i + 1 <= n1 - 1) sub(ldr(f.nx[t + 1]), x[t + 1]);
    } else {
        if (i >= 1) sub(ldr(f.wx[t - 1]), x[t - 1]);
        if (i + 1 < n1) sub(ldr(f.wx[t + 1]), x[t + 1]);
        if (j >= 1) sub(ldr(f.wz[t - n1]), x[t - n1]);
        if (j + 1 < n2) sub(ldr(f.wz[t + n1]), x[t + n1]);
    }
    ax = acc;
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
// fused pre-smoothing + residual + restriction (one thread per coarse point):
//   x = w D^{-1} b  (one damped Jacobi sweep from the zero guess),
//   b_c = R (b - A x),
// with x recomputed on the fly at every fine point the restriction touches;
// the thread also writes x on the 2x2 fine points it owns.
// ---------------------------------------------------------------------------
template <class V> struct PtrSetF { V* p[3]; };

template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_smooth_restrict(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                         Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                         typename MGT<MODE>::R w, PtrSetF<typename MGT<MODE>::V> cb,
                                                         int intergrid) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, n1c = n1 / 2, n2c = n2 / 2;
    const int np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n1c * n2c) return;
    const int I = t % n1c, J = t / n1c;
    const int type = B.type;
    // zero-guess Jacobi iterate at fine index g
    auto X = [&](int g) -> V {
        const int gi = g % n1, gj = g / n1;
        if (!valid_pt(type, gi, gj)) return czero<V>();
        const V dg = diag_only<MODE>(L0 ? &f5 : nullptr, B, np, g);
        return cscale(cdiv(B.b[g], dg), w);
    };
    // the owned 2x2 fine points
    for (int q = 0; q < 4; ++q) {
        const int fi = 2 * I + (q & 1), fj = 2 * J + (q >> 1);
        B.xout[fj * n1 + fi] = X(fj * n1 + fi);
    }
    V acc = czero<V>();
    if (valid_pt(type, I, J)) {
        const bool nodx = type == 0, nodz = type == 1;
        for (int fj = 2 * J - 2; fj <= 2 * J + 3; ++fj) {
            const R wz = rw_axis_t<R>(nodz, intergrid, n2, J, fj);
            if (wz == R(0)) continue;
            for (int fi = 2 * I - 2; fi <= 2 * I + 3; ++fi) {
                const R wxw = rw_axis_t<R>(nodx, intergrid, n1, I, fi);
                if (wxw == R(0)) continue;
                const int f = fj * n1 + fi;
                V ax;
                if (L0) ax = apply_fine5_fn<MODE>(f5, type, fi, fj, f, X);
                else ax = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, fi, fj, f, X);
                const V r = csub(B.b[f], ax);
                const R wgt = wz * wxw;
                acc.x += wgt * r.x;
                acc.y += wgt * r.y;
            }
        }
    }
    cb.p[blockIdx.y][t] = acc;
}

// ---------------------------------------------------------------------------
// fused prolongation + correction + one damped Jacobi sweep (one thread per
// fine point): y = x + P e_c evaluated on the fly at the point and its
// stencil neighbours, then x_out = y + w D^{-1} (b - A y).
// ---------------------------------------------------------------------------
template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_prolong_smooth(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                        Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                        typename MGT<MODE>::R w, PtrSetF<const typename MGT<MODE>::V> ce) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, n1c = n1 / 2;
    const int np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int i = t % n1, j = t / n1;
    const int type = B.type;
    if (!valid_pt(type, i, j)) { B.xout[t] = czero<V>(); return; }
    const bool nodx = type == 0, nodz = type == 1;
    const V* e = ce.p[blockIdx.y];
    auto Y = [&](int g) -> V {
        const int gi = g % n1, gj = g / n1;
        if (!valid_pt(type, gi, gj)) return czero<V>();
        V acc = B.xin[g];
        for (int cj = (gj >> 1) - 1; cj <= (gj >> 1) + 1; ++cj) {
            const R pz = pw_axis_t<R>(nodz, n2, gj, cj);
            if (pz == R(0)) continue;
            for (int ci = (gi >> 1) - 1; ci <= (gi >> 1) + 1; ++ci) {
                const R px = pw_axis_t<R>(nodx, n1, gi, ci);
                if (px == R(0)) continue;
                const V v = e[cj * n1c + ci];
                acc.x += px * pz * v.x;
                acc.y += px * pz * v.y;
            }
        }
        return acc;
    };
    V ay;
    if (L0) ay = apply_fine5_fn<MODE>(f5, type, i, j, t, Y);
    else ay = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, i, j, t, Y);
    const V dg = diag_only<MODE>(L0 ? &f5 : nullptr, B, np, t);
    const V corr = cdiv(csub(B.b[t], ay), dg);
    const V y = Y(t);
    B.xout[t] = cmk<V>(y.x + w * corr.x, y.y + w * corr.y);
}

template <int MODE>
void launch_smooth_restrict(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                            const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                            typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st) {
    PtrSetF<typename Prec<MODE>::V> cb;
    for (int z = 0; z < 3; ++z) cb.p[z] = z < s.nb ? coarse_b[z] : nullptr;
    const int npc = (s.n1 / 2) * (s.n2 / 2);
    dim3 g((npc + 255) / 256, s.nb);
    using R = typename Prec<MODE>::R;
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    if (f5) k_smooth_restrict<MODE, true, 1><<<g, 256, 0, st>>>(s, *f5, (R)w, cb, intergrid);
    else if (max_radius(s) <= 1) k_smooth_restrict<MODE, false, 1><<<g, 256, 0, st>>>(s, nof, (R)w, cb, intergrid);
    else k_smooth_restrict<MODE, false, 2><<<g, 256, 0, st>>>(s, nof, (R)w, cb, intergrid);
}
template <int MODE>
void launch_prolong_smooth(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                           const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                           const typename Prec<MODE>::V* const* coarse_x, cudaStream_t st) {
    PtrSetF<const typename Prec<MODE>::V> ce;
    for (int z = 0; z < 3; ++z) ce.p[z] = z < s.nb ? coarse_x[z] : nullptr;
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb);
    using R = typename Prec<MODE>::R;
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    if (f5) k_prolong_smooth<MODE, true, 1><<<g, 256, 0, st>>>(s, *f5, (R)w, ce);
    else if (max_radius(s) <= 1) k_prolong_smooth<MODE, false, 1><<<g, 256, 0, st>>>(s, nof, (R)w, ce);
    else k_prolong_smooth<MODE, false, 2><<<g, 256, 0, st>>>(s, nof, (R)w, ce);
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
    cb.p[blockIdx.y][rr * cb.s + t] = acc;
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
    const V* e = ce.p[blockIdx.y] + rr * ce.s;
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
// coarsest level: x = A_c^{-1} b with the stored inverse (one warp per row).
// The inverse is computed in FP64 at setup and stored in the cycle's vector
// type: FP64 in the FP64 mode, rounded once to FP32 in the mixed mode, where
// the product is accumulated in FP32 like the rest of the cycle.
// ---------------------------------------------------------------------------
constexpr int kCoarseSmem = 3072;   // points staged in shared memory (48 KB of FP64 complex)

template <int MODE>
__global__ void __launch_bounds__(256) k_coarse_apply(int npts, PtrSet<const typename MGT<MODE>::V> inv,
                                                      PtrSet<const typename MGT<MODE>::V> b,
                                                      PtrSet<typename MGT<MODE>::V> x, const int* active) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const int z = blockIdx.y;
    const int rr = blockIdx.z;
    if (active && !active[rr]) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char coarse_raw[];
    V* bsh = reinterpret_cast<V*>(coarse_raw);
    const V* bb = b.p[z] + rr * b.s;
    const bool staged = npts <= kCoarseSmem;
    if (staged) {
        for (int c = threadIdx.x; c < npts; c += blockDim.x) bsh[c] = bb[c];
        __syncthreads();
    }
    if (warp >= npts) return;
    const V* row = inv.p[z] + (size_t)warp * npts;
    R re = 0, im = 0;
    for (int c = lane; c < npts; c += 32) {
        const V a = row[c];
        const V v = staged ? bsh[c] : bb[c];
        re += a.x * v.x - a.y * v.y;
        im += a.x * v.y + a.y * v.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) x.p[z][rr * x.s + warp] = cmk<V>(re, im);
}

template <int MODE>
void launch_coarse_apply(int nb, int npts, const typename Prec<MODE>::V* const* inv,
                         const typename Prec<MODE>::V* const* b, typename Prec<MODE>::V* const* x, cudaStream_t st,
                         int nrhs, RhsStride rs) {
    PtrSet<const typename Prec<MODE>::V> pi;
    PtrSet<const typename Prec<MODE>::V> pb;
    PtrSet<typename Prec<MODE>::V> px;
    for (int z = 0; z < 3; ++z) {
        pi.p[z] = z < nb ? inv[z] : nullptr;
        pb.p[z] = z < nb ? b[z] : nullptr;
        px.p[z] = z < nb ? x[z] : nullptr;
    }
    pb.s = rs.s0;
    px.s = rs.s1;
    dim3 g((npts * 32 + 255) / 256, nb, nrhs);
    const size_t smem = npts <= kCoarseSmem ? (size_t)npts * sizeof(typename Prec<MODE>::V) : 0;
    launch_pdl(k_coarse_apply<MODE>, dim3(g), dim3(256), smem, st, npts, pi, pb, px, rs.active);
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
    template void launch_coarse_apply<MODE>(int, int, const Prec<MODE>::V* const*, const Prec<MODE>::V* const*,   \
                                            Prec<MODE>::V* const*, cudaStream_t, int, RhsStride);                 \
    template void launch_smooth_restrict<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                       \
                                               const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double,                \
                                               Prec<MODE>::V* const*, int, cudaStream_t);                          \
    template void launch_prolong_smooth<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                        \
                                              const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double,                 \
                                              const Prec<MODE>::V* const*, cudaStream_t);
INST(BAH_FP64)
INST(BAH_MIXED)

}  // namespace bah

// ===========================================================================
// Cooperative multigrid: all levels l0..L-1 of a block set in one launch.
// A persistent grid (co-residency checked by the cooperative launch) walks
// the cycle phase by phase -- zero-guess Jacobi, residual, restriction, ...,
// coarsest FP64 solve, prolongation, post-smoothing -- with a grid barrier
// between phases.  The barrier's spin is bounded: on time-out it raises the
// error flag and the kernel carries on without waiting (the host reports
// the flag as a failed solve).
// ===========================================================================
namespace bah {

template <int MODE>
__device__ __forceinline__ typename MGT<MODE>::V coop_x0(const typename MGT<MODE>::CC* S, int rx, int rz, int np,
                                                         int type, int n1, int g, const typename MGT<MODE>::V* b,
                                                         typename MGT<MODE>::R w) {
    using V = typename MGT<MODE>::V;
    const int gi = g % n1, gj = g / n1;
    if (!valid_pt(type, gi, gj)) return czero<V>();
    const V dg = ldc(S[(size_t)(rz * (2 * rx + 1) + rx) * np + g]);
    return cscale(cdiv(b[g], dg), w);
}

__constant__ unsigned g_barrier_sleep_ns = 32;

__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vg = gen;
        const unsigned g = *vg;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vg == g) {
                if (++spins > (1ull << 24)) {      // well over a second with the back-off below
                    atomicExch(err, 1);
                    break;
                }
                if (g_barrier_sleep_ns) __nanosleep(g_barrier_sleep_ns);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

template <int MODE, int RM>
__global__ void __launch_bounds__(256) k_coop_cycle(CoopArgs a) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    using CC = typename MGT<MODE>::CC;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gsz = (long long)gridDim.x * blockDim.x;
    const int nb = a.nb;
    auto lvl = [&](int l) -> const CoopLevel& { return a.lv[l]; };
    auto sync = [&]() { grid_barrier(a.bar_count, a.bar_gen, a.err); };
    auto apply = [&](const CoopLevel& L, int z, int t, const V* x) -> V {
        const int n1 = L.n1, n2 = L.n2;
        auto X = [&](int g) { return x[g]; };
        return apply_stencil_fn<MODE, RM>((const CC*)L.S[z], L.rx[z], L.rz[z], n1, n2, t % n1, t / n1, t, X);
    };
    auto diag = [&](const CoopLevel& L, int z, int t) -> V {
        const int np = L.n1 * L.n2;
        return ldc(((const CC*)L.S[z])[(size_t)(L.rz[z] * (2 * L.rx[z] + 1) + L.rx[z]) * np + t]);
    };
    // phase: x_out = x_in + w D^-1 (b - A x_in)  (zero: w D^-1 b)
    auto jacobi = [&](int l, V* const* xin, V* const* xout, bool zero) {
        const CoopLevel& L = lvl(l);
        const int np = L.n1 * L.n2;
        const R w = (R)L.w;
        for (long long idx = gtid; idx < (long long)nb * np; idx += gsz) {
            const int z = (int)(idx / np), t = (int)(idx % np);
            const int type = a.b0 + z;
            const V* b = (const V*)L.b[z];
            if (!valid_pt(type, t % L.n1, t / L.n1)) { xout[z][t] = czero<V>(); continue; }
            const V dg = diag(L, z, t);
            if (zero) { xout[z][t] = cscale(cdiv(b[t], dg), w); continue; }
            const V ax = apply(L, z, t, xin[z]);
            const V corr = cdiv(csub(b[t], ax), dg);
            const V xv = xin[z][t];
            xout[z][t] = cmk<V>(xv.x + w * corr.x, xv.y + w * corr.y);
        }
    };
    auto residual = [&](int l, V* const* x, V* const* r) {
        const CoopLevel& L = lvl(l);
        const int np = L.n1 * L.n2;
        for (long long idx = gtid; idx < (long long)nb * np; idx += gsz) {
            const int z = (int)(idx / np), t = (int)(idx % np);
            const int type = a.b0 + z;
            if (!valid_pt(type, t % L.n1, t / L.n1)) { r[z][t] = czero<V>(); continue; }
            r[z][t] = csub(((const V*)L.b[z])[t], apply(L, z, t, x[z]));
        }
    };
    auto restrict_ = [&](int l, V* const* r) {      // into level l+1's right-hand side
        const CoopLevel& L = lvl(l);
        const CoopLevel& Lc = lvl(l + 1);
        const int n1 = L.n1, n2 = L.n2, n1c = Lc.n1, npc = Lc.n1 * Lc.n2;
        const bool to_coarsest = (l + 1 == a.L - 1);
        for (long long idx = gtid; idx < (long long)nb * npc; idx += gsz) {
            const int z = (int)(idx / npc), t = (int)(idx % npc);
            const int type = a.b0 + z;
            const int I = t % n1c, J = t / n1c;
            V acc = czero<V>();
            if (valid_pt(type, I, J)) {
                const bool nodx = type == 0, nodz = type == 1;
                for (int fj = 2 * J - 2; fj <= 2 * J + 3; ++fj) {
                    const R wz = rw_axis_t<R>(nodz, a.intergrid, n2, J, fj);
                    if (wz == R(0)) continue;
                    for (int fi = 2 * I - 2; fi <= 2 * I + 3; ++fi) {
                        const R wxw = rw_axis_t<R>(nodx, a.intergrid, n1, I, fi);
                        if (wxw == R(0)) continue;
                        const V v = r[z][fj * n1 + fi];
                        acc.x += wz * wxw * v.x;
                        acc.y += wz * wxw * v.y;
                    }
                }
            }
            if (to_coarsest) a.bc64[z][t] = make_double2((double)acc.x, (double)acc.y);
            else ((V*)Lc.b[z])[t] = acc;
        }
    };
    auto prolong = [&](int l, V* const* x, const V* const* e) {
        const CoopLevel& L = lvl(l);
        const int n1 = L.n1, n2 = L.n2, n1c = n1 / 2, np = n1 * n2;
        for (long long idx = gtid; idx < (long long)nb * np; idx += gsz) {
            const int z = (int)(idx / np), t = (int)(idx % np);
            const int type = a.b0 + z;
            const int i = t % n1, j = t / n1;
            if (!valid_pt(type, i, j)) continue;
            const bool nodx = type == 0, nodz = type == 1;
            V acc = czero<V>();
            for (int cj = (j >> 1) - 1; cj <= (j >> 1) + 1; ++cj) {
                const R pz = pw_axis_t<R>(nodz, n2, j, cj);
                if (pz == R(0)) continue;
                for (int ci = (i >> 1) - 1; ci <= (i >> 1) + 1; ++ci) {
                    const R px = pw_axis_t<R>(nodx, n1, i, ci);
                    if (px == R(0)) continue;
                    const V v = e[z][cj * n1c + ci];
                    acc.x += px * pz * v.x;
                    acc.y += px * pz * v.y;
                }
            }
            x[z][t] = cadd(x[z][t], acc);
        }
    };
    auto coarse = [&]() {                            // x_{L-1} = A_c^{-1} b_{L-1} (FP64 sums), one warp per row
        const CoopLevel& L = lvl(a.L - 1);
        const int npts = L.n1 * L.n2;
        const long long warp = gtid >> 5, nwarps = gsz >> 5;
        const int lane = threadIdx.x & 31;
        for (long long row = warp; row < (long long)nb * npts; row += nwarps) {
            const int z = (int)(row / npts), rr = (int)(row % npts);
            const V* arow = (const V*)a.inv[z] + (size_t)rr * npts;
            const double2* bb = a.bc64[z];
            double re = 0.0, im = 0.0;
            for (int c = lane; c < npts; c += 32) {
                const V m = arow[c];
                const double2 v = bb[c];
                re += (double)m.x * v.x - (double)m.y * v.y;
                im += (double)m.x * v.y + (double)m.y * v.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) ((V*)L.x[z])[rr] = cmk<V>((R)re, (R)im);
        }
    };

    V* X[3]; V* T[3];
    // ---- down ----
    for (int l = a.l0; l < a.L - 1; ++l) {
        const CoopLevel& L = lvl(l);
        for (int z = 0; z < nb; ++z) { X[z] = (V*)L.x[z]; T[z] = (V*)L.t[z]; }
        jacobi(l, nullptr, X, true);
        sync();
        for (int s = 1; s < a.nu_pre; ++s) {
            jacobi(l, X, T, false);
            sync();
            for (int z = 0; z < nb; ++z) { V* q = X[z]; X[z] = T[z]; T[z] = q; }
        }
        residual(l, X, T);
        sync();
        restrict_(l, T);
        sync();
    }
    coarse();
    sync();
    // ---- up ----
    for (int l = a.L - 2; l >= a.l0; --l) {
        const CoopLevel& L = lvl(l);
        const CoopLevel& Lc = lvl(l + 1);
        // the pre-smoothing result sits in L.x (nu_pre - 1 swaps are undone by the pairing below)
        for (int z = 0; z < nb; ++z) {
            X[z] = (a.nu_pre % 2 == 1) ? (V*)L.x[z] : (V*)L.t[z];
            T[z] = (a.nu_pre % 2 == 1) ? (V*)L.t[z] : (V*)L.x[z];
        }
        const V* E[3];
        for (int z = 0; z < nb; ++z) E[z] = (const V*)Lc.x[z];
        prolong(l, X, E);
        sync();
        for (int s = 0; s < a.nu_post; ++s) {
            jacobi(l, X, T, false);
            sync();
            for (int z = 0; z < nb; ++z) { V* q = X[z]; X[z] = T[z]; T[z] = q; }
        }
        if (X[0] != (V*)L.x[0]) {                     // leave the result in L.x
            const int np = L.n1 * L.n2;
            for (long long idx = gtid; idx < (long long)nb * np; idx += gsz) {
                const int z = (int)(idx / np), t = (int)(idx % np);
                ((V*)L.x[z])[t] = X[z][t];
            }
            sync();
        }
    }
}

template <int MODE>
int launch_coop_cycle(const CoopArgs& a, int max_radius, int nsm, cudaStream_t st) {
    const void* fn = max_radius <= 1 ? (const void*)k_coop_cycle<MODE, 1> : (const void*)k_coop_cycle<MODE, 2>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return -1;
    }
    int cap = 1;
    if (const char* e = getenv("BAH_COOP_CTAS_PER_SM")) cap = atoi(e) > 0 ? atoi(e) : 1;
    per_sm = per_sm > cap ? cap : per_sm;
    static bool sleep_set = false;
    if (!sleep_set) {
        unsigned ns = 32;
        if (const char* e = getenv("BAH_COOP_SLEEP_NS")) ns = (unsigned)atoi(e);
        cudaMemcpyToSymbol(g_barrier_sleep_ns, &ns, sizeof(ns));
        sleep_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsm * per_sm);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = max_radius <= 1 ? cudaLaunchKernelEx(&cfg, k_coop_cycle<MODE, 1>, a)
                                    : cudaLaunchKernelEx(&cfg, k_coop_cycle<MODE, 2>, a);
    return e == cudaSuccess ? 0 : (int)e;
}
template int launch_coop_cycle<BAH_FP64>(const CoopArgs&, int, int, cudaStream_t);
template int launch_coop_cycle<BAH_MIXED>(const CoopArgs&, int, int, cudaStream_t);

// ===========================================================================
// Cluster multigrid: the levels l0..L-1 of a V-cycle for one block and one
// right-hand side in one thread-block cluster.  The small levels of the
// hierarchy (a few thousand points) cannot fill the GPU, so separate launches
// cost their launch latency and tail many times per cycle.  Here the cluster
// walks the same phases as the separate kernels -- zero-guess Jacobi, Jacobi,
// residual, restriction, the coarsest solve, prolongation and correction --
// each phase spread over the cluster's threads, with the hardware cluster
// barrier (release/acquire at cluster scope, which orders the global-memory
// writes of one phase before the reads of the next) between phases.  All
// CTAs of a cluster are co-scheduled by the hardware, every thread of every
// CTA reaches every barrier (no early exit except a whole cluster at once),
// so the barrier always completes.  Clusters are independent: the grid is
// (cluster size) x (blocks) x (right-hand sides) CTAs.
// ===========================================================================
template <int MODE, int RM>
__global__ void __launch_bounds__(256) k_cluster_cycle(ClusterArgs a) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    using CC = typename MGT<MODE>::CC;
    const unsigned cid = cluster_index();
    const int z = (int)(cid % (unsigned)a.nb), rr = (int)(cid / (unsigned)a.nb);
    if (a.active && !a.active[rr]) return;          // uniform over the cluster
    const int tid = (int)(cluster_rank() * blockDim.x + threadIdx.x);
    const int nth = (int)(cluster_nrank() * blockDim.x);
    const int type = a.b0 + z;
    const bool nodx = type == 0, nodz = type == 1;
    extern __shared__ __align__(16) unsigned char cluster_raw[];
    V* bsh = reinterpret_cast<V*>(cluster_raw);     // coarsest right-hand side, staged per CTA

    struct Lv { int n1, n2, rx, rz; R w; const CC* S; V* b; V* x; V* t; };
    auto level = [&](int l) {
        const CoopLevel& q = a.lv[l];
        const size_t off = (size_t)rr * q.n1 * q.n2;
        Lv v;
        v.n1 = q.n1; v.n2 = q.n2; v.rx = q.rx[z]; v.rz = q.rz[z]; v.w = (R)q.w;
        v.S = (const CC*)q.S[z];
        v.b = (V*)q.b[z] + off; v.x = (V*)q.x[z] + off; v.t = (V*)q.t[z] + off;
        return v;
    };
    auto diag = [&](const Lv& L, int t) -> V {
        return ldc(L.S[(size_t)(L.rz * (2 * L.rx + 1) + L.rx) * L.n1 * L.n2 + t]);
    };
    auto jacobi = [&](const Lv& L, const V* xin, V* xout, bool zero) {
        const int np = L.n1 * L.n2;
        for (int t = tid; t < np; t += nth) {
            const int i = t % L.n1, j = t / L.n1;
            if (!valid_pt(type, i, j)) { xout[t] = czero<V>(); continue; }
            const V dg = diag(L, t);
            const V b = L.b[t];
            if (zero) { xout[t] = cscale(cdiv(b, dg), L.w); continue; }
            auto X = [&](int g) { return xin[g]; };
            const V ax = apply_stencil_fn<MODE, RM>(L.S, L.rx, L.rz, L.n1, L.n2, i, j, t, X);
            const V corr = cdiv(csub(b, ax), dg);
            const V xv = xin[t];
            xout[t] = cmk<V>(xv.x + L.w * corr.x, xv.y + L.w * corr.y);
        }
    };
    auto residual = [&](const Lv& L, const V* x, V* r) {
        const int np = L.n1 * L.n2;
        for (int t = tid; t < np; t += nth) {
            const int i = t % L.n1, j = t / L.n1;
            if (!valid_pt(type, i, j)) { r[t] = czero<V>(); continue; }
            auto X = [&](int g) { return x[g]; };
            r[t] = csub(L.b[t], apply_stencil_fn<MODE, RM>(L.S, L.rx, L.rz, L.n1, L.n2, i, j, t, X));
        }
    };
    auto restrict_ = [&](const Lv& L, const V* r, V* bc) {     // b_c = R r
        const int n1c = L.n1 / 2, npc = n1c * (L.n2 / 2);
        for (int t = tid; t < npc; t += nth) {
            const int I = t % n1c, J = t / n1c;
            V acc = czero<V>();
            if (valid_pt(type, I, J)) {
                const int bx = rbase(nodx, a.intergrid, I), bz = rbase(nodz, a.intergrid, J);
                R wxs[4], wzs[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    wxs[q] = rw_axis_t<R>(nodx, a.intergrid, L.n1, I, bx + q);
                    wzs[q] = rw_axis_t<R>(nodz, a.intergrid, L.n2, J, bz + q);
                }
                V v[16];
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool ok = wzs[e] != R(0) && wxs[q] != R(0);
                        v[e * 4 + q] = r[ok ? (bz + e) * L.n1 + (bx + q) : 0];
                    }
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const R wgt = wzs[e] * wxs[q];
                        acc.x += wgt * v[e * 4 + q].x;
                        acc.y += wgt * v[e * 4 + q].y;
                    }
            }
            bc[t] = acc;
        }
    };
    auto prolong = [&](const Lv& L, V* x, const V* e) {         // x += P e
        const int np = L.n1 * L.n2, n1c = L.n1 / 2;
        for (int t = tid; t < np; t += nth) {
            const int i = t % L.n1, j = t / L.n1;
            if (!valid_pt(type, i, j)) continue;
            R px[3], pz[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                px[q] = pw_axis_t<R>(nodx, L.n1, i, (i >> 1) - 1 + q);
                pz[q] = pw_axis_t<R>(nodz, L.n2, j, (j >> 1) - 1 + q);
            }
            V v[9];
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const bool ok = pz[e2] != R(0) && px[q] != R(0);
                    v[e2 * 3 + q] = e[ok ? ((j >> 1) - 1 + e2) * n1c + ((i >> 1) - 1 + q) : 0];
                }
            V acc = x[t];
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const R wgt = pz[e2] * px[q];
                    acc.x += wgt * v[e2 * 3 + q].x;
                    acc.y += wgt * v[e2 * 3 + q].y;
                }
            x[t] = acc;
        }
    };
    auto coarse = [&](const Lv& L) {                             // x = A_c^{-1} b, one warp per row
        const int npts = L.n1 * L.n2;
        const bool staged = npts <= kCoarseSmem;
        if (staged) {
            for (int c = threadIdx.x; c < npts; c += blockDim.x) bsh[c] = L.b[c];
            __syncthreads();
        }
        const V* inv = (const V*)a.inv[z];
        const int lane = threadIdx.x & 31;
        for (int row = tid >> 5; row < npts; row += nth >> 5) {
            const V* arow = inv + (size_t)row * npts;
            R re = 0, im = 0;
            for (int c = lane; c < npts; c += 32) {
                const V m = arow[c];
                const V v = staged ? bsh[c] : L.b[c];
                re += m.x * v.x - m.y * v.y;
                im += m.x * v.y + m.y * v.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) L.x[row] = cmk<V>(re, im);
        }
    };

    // The cycle from level l0 down and back up, as an explicit walk over the
    // recursion: one visit of the coarse problem for a V-cycle; two for a
    // W-cycle (the second starting from the first one's result), except where
    // the coarse level is the coarsest, solved exactly once.  Every visit
    // leaves its result in the level's x buffer.
    V* xs[kMaxLevels];
    V* ts[kMaxLevels];
    int stage[kMaxLevels];
    bool warm[kMaxLevels];
    int l = a.l0;
    stage[l] = 0;
    warm[l] = a.warm != 0;
    while (true) {
        if (l == a.L - 1) {
            coarse(level(l));
            cluster_barrier();
            --l;
            continue;
        }
        const Lv L = level(l);
        if (stage[l] == 0) {
            // pre-smoothing (from zero, or from the x buffer on a warm visit), residual, restriction
            V* x = L.x;
            V* t = L.t;
            int s0 = 0;
            if (!warm[l]) {
                if (a.nu_pre >= 1) {
                    jacobi(L, nullptr, x, true);
                    s0 = 1;
                } else {
                    for (int g = tid; g < L.n1 * L.n2; g += nth) x[g] = czero<V>();
                }
                cluster_barrier();
            }
            for (int s = s0; s < a.nu_pre; ++s) {
                jacobi(L, x, t, false);
                cluster_barrier();
                V* q = x; x = t; t = q;
            }
            residual(L, x, t);
            cluster_barrier();
            restrict_(L, t, level(l + 1).b);
            cluster_barrier();
            xs[l] = x;
            ts[l] = t;
            stage[l] = 1;
            ++l;
            stage[l] = 0;
            warm[l] = false;
            continue;
        }
        if (stage[l] == 1 && a.wcycle && l + 1 < a.L - 1) {
            stage[l] = 2;
            ++l;
            stage[l] = 0;
            warm[l] = true;
            continue;
        }
        // prolongation and correction, post-smoothing
        V* x = xs[l];
        V* t = ts[l];
        prolong(L, x, level(l + 1).x);
        cluster_barrier();
        for (int s = 0; s < a.nu_post; ++s) {
            jacobi(L, x, t, false);
            cluster_barrier();
            V* q = x; x = t; t = q;
        }
        if (x != L.x) {
            for (int g = tid; g < L.n1 * L.n2; g += nth) L.x[g] = x[g];
            cluster_barrier();
        }
        if (l == a.l0) break;
        --l;
    }
}

template <int MODE>
static const void* cluster_fn(int max_radius) {
    return max_radius <= 1 ? (const void*)k_cluster_cycle<MODE, 1> : (const void*)k_cluster_cycle<MODE, 2>;
}

template <int MODE>
int cluster_size_for(int max_radius, int want, int coarse_pts) {
    const void* fn = cluster_fn<MODE>(max_radius);
    if (want > 8) {
        // both radius variants: a block set may launch either
        for (int r = 1; r <= 2; ++r)
            if (cudaFuncSetAttribute(cluster_fn<MODE>(r), cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
                cudaGetLastError();
                want = 8;
            }
    }
    const size_t smem = coarse_pts <= kCoarseSmem ? (size_t)coarse_pts * sizeof(typename Prec<MODE>::V) : 0;
    for (int cs = want; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) return cs;
        cudaGetLastError();
    }
    return 0;
}

template <int MODE>
int launch_cluster_cycle(const ClusterArgs& a, int max_radius, int nrhs, int csize, int coarse_pts, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize * a.nb * nrhs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = coarse_pts <= kCoarseSmem ? (size_t)coarse_pts * sizeof(typename Prec<MODE>::V) : 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e = max_radius <= 1 ? cudaLaunchKernelEx(&cfg, k_cluster_cycle<MODE, 1>, a)
                                    : cudaLaunchKernelEx(&cfg, k_cluster_cycle<MODE, 2>, a);
    return e == cudaSuccess ? 0 : (int)e;
}
template int cluster_size_for<BAH_FP64>(int, int, int);
template int cluster_size_for<BAH_MIXED>(int, int, int);
template int launch_cluster_cycle<BAH_FP64>(const ClusterArgs&, int, int, int, int, cudaStream_t);
template int launch_cluster_cycle<BAH_MIXED>(const ClusterArgs&, int, int, int, int, cudaStream_t);

}  // namespace bah
