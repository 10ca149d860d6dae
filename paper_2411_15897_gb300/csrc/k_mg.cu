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

#include <algorithm>
#include <cstdlib>

namespace bah {

template <int MODE>
struct MGT {
    using V = typename Prec<MODE>::V;
    using R = typename Prec<MODE>::R;
    using C = typename Prec<MODE>::C;
    using CC = typename Prec<MODE>::CC;
};

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


// A x at point (i, j) of a level-0 block where x is given by an accessor X(index).
// The four neighbour terms are loaded unconditionally with clamped indices and
// masked, so the loads issue together.
template <int MODE, class XF>
__device__ __forceinline__ typename MGT<MODE>::V apply_fine5_fn(const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>& f,
                                                               int type, int i, int j, int t, XF X) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const int n1 = f.n1, n2 = f.n2;
    const auto* dgp = type == 0 ? f.dg0 : (type == 1 ? f.dg1 : f.dg2);
    // neighbours W, E, S, N: existence, coefficient index and array per block type
    bool ok[4];
    int ci[4];
    const typename MGT<MODE>::C* arr[4];
    if (type == 0) {
        ok[0] = i - 1 >= 1;       ci[0] = t - 1;  arr[0] = f.cx;
        ok[1] = i + 1 <= n1 - 1;  ci[1] = t;      arr[1] = f.cx;
        ok[2] = j >= 1;           ci[2] = t;      arr[2] = f.nz;
        ok[3] = j + 1 <= n2 - 1;  ci[3] = t + n1; arr[3] = f.nz;
    } else if (type == 1) {
        ok[0] = i >= 1;           ci[0] = t;      arr[0] = f.nx;
        ok[1] = i + 1 <= n1 - 1;  ci[1] = t + 1;  arr[1] = f.nx;
        ok[2] = j - 1 >= 1;       ci[2] = t - n1; arr[2] = f.cz;
        ok[3] = j + 1 <= n2 - 1;  ci[3] = t;      arr[3] = f.cz;
    } else {
        ok[0] = i >= 1;           ci[0] = t - 1;  arr[0] = f.wx;
        ok[1] = i + 1 < n1;       ci[1] = t + 1;  arr[1] = f.wx;
        ok[2] = j >= 1;           ci[2] = t - n1; arr[2] = f.wz;
        ok[3] = j + 1 < n2;       ci[3] = t + n1; arr[3] = f.wz;
    }
    const int nb[4] = {t - 1, t + 1, t - n1, t + n1};
    R k[4];
    V xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        k[q] = ldr(arr[q][ok[q] ? ci[q] : t]);
        xv[q] = X(ok[q] ? nb[q] : t);
    }
    const V dg = ldc(dgp[t]);
    V acc = cmul(dg, X(t));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R kk = ok[q] ? k[q] : R(0);
        acc.x -= kk * xv[q].x;
        acc.y -= kk * xv[q].y;
    }
    return acc;
}

// RM is the compile-time maximum radius (1 or 2); rx, rz <= RM are the block's
// radii.  The loops unroll fully and every candidate load is issued with an
// index clamped into range (out-of-range terms are masked to zero), so all
// loads go out back to back instead of waiting behind per-neighbour branches.
template <int MODE, int RM, class XF>
__device__ __forceinline__ typename MGT<MODE>::V apply_stencil_fn(const typename MGT<MODE>::CC* __restrict__ S, int rx,
                                                                 int rz, int n1, int n2, int i, int j, int t, XF X) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const size_t np = (size_t)n1 * n2;
    const int wx = 2 * rx + 1;
    V sv[(2 * RM + 1) * (2 * RM + 1)], xv[(2 * RM + 1) * (2 * RM + 1)];
    bool in[(2 * RM + 1) * (2 * RM + 1)];
#pragma unroll
    for (int dz = -RM; dz <= RM; ++dz) {
#pragma unroll
        for (int dx = -RM; dx <= RM; ++dx) {
            const int q = (dz + RM) * (2 * RM + 1) + (dx + RM);
            const int ii = i + dx, jj = j + dz;
            in[q] = dx >= -rx && dx <= rx && dz >= -rz && dz <= rz && ii >= 0 && ii < n1 && jj >= 0 && jj < n2;
            const int slot = in[q] ? (dz + rz) * wx + (dx + rx) : 0;
            sv[q] = ldc(S[(size_t)slot * np + t]);
            xv[q] = X(in[q] ? jj * n1 + ii : t);
        }
    }
    V acc = czero<V>();
#pragma unroll
    for (int q = 0; q < (2 * RM + 1) * (2 * RM + 1); ++q) {
        const R m = in[q] ? R(1) : R(0);
        acc.x += m * (sv[q].x * xv[q].x - sv[q].y * xv[q].y);
        acc.y += m * (sv[q].x * xv[q].y + sv[q].y * xv[q].x);
    }
    return acc;
}

template <int MODE>
__device__ __forceinline__ typename MGT<MODE>::V diag_only(const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>* f5,
                                                          const LvlBlk<typename MGT<MODE>::V, typename MGT<MODE>::CC>& B,
                                                          int np, int t) {
    if (f5) {
        const auto* dgp = B.type == 0 ? f5->dg0 : (B.type == 1 ? f5->dg1 : f5->dg2);
        return ldc(dgp[t]);
    }
    return ldc(B.S[(size_t)(B.rz * (2 * B.rx + 1) + B.rx) * np + t]);
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

template <int MODE>
void launch_jacobi(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                   const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w, int zero_init,
                   cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb, s.nrhs);
    using R = typename Prec<MODE>::R;
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    if (f5) launch_pdl(k_jacobi<MODE, true, 1>, dim3(g), dim3(256), 0, st, s, *f5, (R)w, zero_init);
    else if (max_radius(s) <= 1) launch_pdl(k_jacobi<MODE, false, 1>, dim3(g), dim3(256), 0, st, s, nof, (R)w, zero_init);
    else launch_pdl(k_jacobi<MODE, false, 2>, dim3(g), dim3(256), 0, st, s, nof, (R)w, zero_init);
}
template <int MODE>
void launch_residual(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                     const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb, s.nrhs);
    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    if (f5) launch_pdl(k_residual<MODE, true, 1>, dim3(g), dim3(256), 0, st, s, *f5);
    else if (max_radius(s) <= 1) launch_pdl(k_residual<MODE, false, 1>, dim3(g), dim3(256), 0, st, s, nof);
    else launch_pdl(k_residual<MODE, false, 2>, dim3(g), dim3(256), 0, st, s, nof);
}

// ---------------------------------------------------------------------------
// restriction: b_c = R r_f  (r_f in blk.xout of the fine set)
// ---------------------------------------------------------------------------
template <class V> struct PtrSet { V* p[3]; size_t s = 0; };

// support of a 1-D restriction row for coarse index c: first fine index
__host__ __device__ __forceinline__ int rbase(bool nodal, int intergrid, int c) {
    return nodal ? 2 * c - 1 : (intergrid == BAH_INTERGRID_MIXED ? 2 * c : 2 * c - 1);
}

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
// coarsest level: x = A_c^{-1} b with the stored FP64 inverse (one warp per row)
// ---------------------------------------------------------------------------
constexpr int kCoarseSmem = 3072;   // points staged in shared memory (48 KB of FP64 complex)

template <int MODE>
__global__ void __launch_bounds__(256) k_coarse_apply(int npts, PtrSet<const double2> inv,
                                                      PtrSet<const typename MGT<MODE>::V> b,
                                                      PtrSet<typename MGT<MODE>::V> x, const int* active) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    const int z = blockIdx.y;
    const int rr = blockIdx.z;
    if (active && !active[rr]) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    extern __shared__ double2 bsh[];
    const V* bb = b.p[z] + rr * b.s;
    const bool staged = npts <= kCoarseSmem;
    if (staged) {
        // the right-hand side in FP64, converted once per CTA
        for (int c = threadIdx.x; c < npts; c += blockDim.x) bsh[c] = make_double2((double)bb[c].x, (double)bb[c].y);
        __syncthreads();
    }
    if (warp >= npts) return;
    const double2* row = inv.p[z] + (size_t)warp * npts;
    double re = 0.0, im = 0.0;
    for (int c = lane; c < npts; c += 32) {
        const double2 a = row[c];
        double2 v;
        if (staged) v = bsh[c];
        else v = make_double2((double)bb[c].x, (double)bb[c].y);
        re += a.x * v.x - a.y * v.y;
        im += a.x * v.y + a.y * v.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) x.p[z][rr * x.s + warp] = cmk<V>((typename MGT<MODE>::R)re, (typename MGT<MODE>::R)im);
}

template <int MODE>
void launch_coarse_apply(int nb, int npts, const double2* const* inv, const typename Prec<MODE>::V* const* b,
                         typename Prec<MODE>::V* const* x, cudaStream_t st, int nrhs, RhsStride rs) {
    PtrSet<const double2> pi;
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
    const size_t smem = npts <= kCoarseSmem ? (size_t)npts * sizeof(double2) : 0;
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
    template void launch_coarse_apply<MODE>(int, int, const double2* const*, const Prec<MODE>::V* const*,         \
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
    auto coarse = [&]() {                            // x_{L-1} = A_c^{-1} b_{L-1} (FP64), one warp per row
        const CoopLevel& L = lvl(a.L - 1);
        const int npts = L.n1 * L.n2;
        const long long warp = gtid >> 5, nwarps = gsz >> 5;
        const int lane = threadIdx.x & 31;
        for (long long row = warp; row < (long long)nb * npts; row += nwarps) {
            const int z = (int)(row / npts), rr = (int)(row % npts);
            const double2* arow = a.inv[z] + (size_t)rr * npts;
            const double2* bb = a.bc64[z];
            double re = 0.0, im = 0.0;
            for (int c = lane; c < npts; c += 32) {
                const double2 m = arow[c], v = bb[c];
                re += m.x * v.x - m.y * v.y;
                im += m.x * v.y + m.y * v.x;
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

}  // namespace bah
