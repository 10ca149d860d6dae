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

namespace bah {

template <int MODE>
struct MGT {
    using V = typename Prec<MODE>::V;
    using R = typename Prec<MODE>::R;
    using C = typename Prec<MODE>::C;
    using CC = typename Prec<MODE>::CC;
};

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

// A x and diag(A) at point t from an explicit stencil
template <int MODE>
__device__ __forceinline__ void apply_stencil(const typename MGT<MODE>::CC* __restrict__ S, int rx, int rz, int n1,
                                              int n2, int i, int j, int t, const typename MGT<MODE>::V* __restrict__ x,
                                              typename MGT<MODE>::V& ax, typename MGT<MODE>::V& dg) {
    using V = typename MGT<MODE>::V;
    const size_t np = (size_t)n1 * n2;
    const int wx = 2 * rx + 1;
    V acc = czero<V>();
    for (int dz = -rz; dz <= rz; ++dz) {
        const int jj = j + dz;
        if (jj < 0 || jj >= n2) continue;
        for (int dx = -rx; dx <= rx; ++dx) {
            const int ii = i + dx;
            if (ii < 0 || ii >= n1) continue;
            const V s = ldc(S[(size_t)((dz + rz) * wx + (dx + rx)) * np + t]);
            const V v = x[jj * n1 + ii];
            acc.x += s.x * v.x - s.y * v.y;
            acc.y += s.x * v.y + s.y * v.x;
        }
    }
    ax = acc;
    dg = ldc(S[(size_t)(rz * wx + rx) * np + t]);
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
template <int MODE, bool L0>
__global__ void __launch_bounds__(256) k_jacobi(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                typename MGT<MODE>::R w, int zero_init) {
    using V = typename MGT<MODE>::V;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) { B.xout[t] = czero<V>(); return; }
    const V b = B.b[t];
    if (zero_init) {
        const V dg = diag_only<MODE>(L0 ? &f5 : nullptr, B, np, t);
        B.xout[t] = cscale(cdiv(b, dg), w);
        return;
    }
    V ax, dg;
    if (L0) apply_fine5<MODE>(f5, B.type, i, j, t, B.xin, ax, dg);
    else apply_stencil<MODE>(B.S, B.rx, B.rz, n1, n2, i, j, t, B.xin, ax, dg);
    const V corr = cdiv(csub(b, ax), dg);
    const V x = B.xin[t];
    B.xout[t] = cmk<V>(x.x + w * corr.x, x.y + w * corr.y);
}

// ---------------------------------------------------------------------------
// residual:  r = b - A x
// ---------------------------------------------------------------------------
template <int MODE, bool L0>
__global__ void __launch_bounds__(256) k_residual(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                  Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5) {
    using V = typename MGT<MODE>::V;
    const auto& B = s.blk[blockIdx.y];
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) { B.xout[t] = czero<V>(); return; }
    V ax, dg;
    if (L0) apply_fine5<MODE>(f5, B.type, i, j, t, B.xin, ax, dg);
    else apply_stencil<MODE>(B.S, B.rx, B.rz, n1, n2, i, j, t, B.xin, ax, dg);
    B.xout[t] = csub(B.b[t], ax);
}

template <int MODE>
void launch_jacobi(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                   const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w, int zero_init,
                   cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb);
    using R = typename Prec<MODE>::R;
    if (f5) k_jacobi<MODE, true><<<g, 256, 0, st>>>(s, *f5, (R)w, zero_init);
    else k_jacobi<MODE, false><<<g, 256, 0, st>>>(s, Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>{}, (R)w,
                                                  zero_init);
}
template <int MODE>
void launch_residual(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                     const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, cudaStream_t st) {
    const int np = s.n1 * s.n2;
    dim3 g((np + 255) / 256, s.nb);
    if (f5) k_residual<MODE, true><<<g, 256, 0, st>>>(s, *f5);
    else k_residual<MODE, false><<<g, 256, 0, st>>>(s, Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>{});
}

// ---------------------------------------------------------------------------
// restriction: b_c = R r_f  (r_f in blk.xout of the fine set)
// ---------------------------------------------------------------------------
template <class V> struct PtrSet { V* p[3]; };

template <int MODE>
__global__ void __launch_bounds__(256) k_restrict(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> fine,
                                                  PtrSet<typename MGT<MODE>::V> cb, int intergrid) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = fine.blk[blockIdx.y];
    const int n1 = fine.n1, n2 = fine.n2, n1c = n1 / 2, n2c = n2 / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n1c * n2c) return;
    const int I = t % n1c, J = t / n1c;
    V acc = czero<V>();
    if (valid_pt(B.type, I, J)) {
        const bool nodx = B.type == 0, nodz = B.type == 1;
        const V* r = B.xout;
        for (int fj = 2 * J - 2; fj <= 2 * J + 3; ++fj) {
            const double wz = rw_axis(nodz, intergrid, n2, J, fj);
            if (wz == 0.0) continue;
            for (int fi = 2 * I - 2; fi <= 2 * I + 3; ++fi) {
                const double wxw = rw_axis(nodx, intergrid, n1, I, fi);
                if (wxw == 0.0) continue;
                const R wgt = (R)(wz * wxw);
                const V v = r[fj * n1 + fi];
                acc.x += wgt * v.x;
                acc.y += wgt * v.y;
            }
        }
    }
    cb.p[blockIdx.y][t] = acc;
}

template <int MODE>
void launch_restrict(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                     typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st) {
    PtrSet<typename Prec<MODE>::V> cb;
    for (int z = 0; z < 3; ++z) cb.p[z] = z < fine.nb ? coarse_b[z] : nullptr;
    const int npc = (fine.n1 / 2) * (fine.n2 / 2);
    dim3 g((npc + 255) / 256, fine.nb);
    k_restrict<MODE><<<g, 256, 0, st>>>(fine, cb, intergrid);
}

// ---------------------------------------------------------------------------
// prolongation and correction: x_f += P e_c  (x_f = blk.xout of the fine set)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_prolong_add(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> fine,
                                                     PtrSet<typename MGT<MODE>::V> ce) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    const auto& B = fine.blk[blockIdx.y];
    const int n1 = fine.n1, n2 = fine.n2, n1c = n1 / 2, n2c = n2 / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n1 * n2) return;
    const int i = t % n1, j = t / n1;
    if (!valid_pt(B.type, i, j)) return;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    const V* e = ce.p[blockIdx.y];
    V acc = czero<V>();
    for (int cj = (j >> 1) - 1; cj <= (j >> 1) + 1; ++cj) {
        const double pz = pw_axis(nodz, n2, j, cj);
        if (pz == 0.0) continue;
        for (int ci = (i >> 1) - 1; ci <= (i >> 1) + 1; ++ci) {
            const double px = pw_axis(nodx, n1, i, ci);
            if (px == 0.0) continue;
            const R wgt = (R)(px * pz);
            const V v = e[cj * n1c + ci];
            acc.x += wgt * v.x;
            acc.y += wgt * v.y;
        }
    }
    V x = B.xout[t];
    B.xout[t] = cadd(x, acc);
}

template <int MODE>
void launch_prolong_add(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& fine,
                        const typename Prec<MODE>::V* const* coarse_x, cudaStream_t st) {
    PtrSet<typename Prec<MODE>::V> ce;
    for (int z = 0; z < 3; ++z) ce.p[z] = z < fine.nb ? const_cast<typename Prec<MODE>::V*>(coarse_x[z]) : nullptr;
    const int np = fine.n1 * fine.n2;
    dim3 g((np + 255) / 256, fine.nb);
    k_prolong_add<MODE><<<g, 256, 0, st>>>(fine, ce);
}

// ---------------------------------------------------------------------------
// coarsest level: x = A_c^{-1} b with the stored FP64 inverse (one warp per row)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_coarse_apply(int npts, PtrSet<const double2> inv,
                                                      PtrSet<const typename MGT<MODE>::V> b,
                                                      PtrSet<typename MGT<MODE>::V> x) {
    using V = typename MGT<MODE>::V;
    const int z = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= npts) return;
    const double2* row = inv.p[z] + (size_t)warp * npts;
    const V* bb = b.p[z];
    double re = 0.0, im = 0.0;
    for (int c = lane; c < npts; c += 32) {
        const double2 a = row[c];
        const V v = bb[c];
        const double vx = (double)v.x, vy = (double)v.y;
        re += a.x * vx - a.y * vy;
        im += a.x * vy + a.y * vx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) x.p[z][warp] = cmk<V>((typename MGT<MODE>::R)re, (typename MGT<MODE>::R)im);
}

template <int MODE>
void launch_coarse_apply(int nb, int npts, const double2* const* inv, const typename Prec<MODE>::V* const* b,
                         typename Prec<MODE>::V* const* x, cudaStream_t st) {
    PtrSet<const double2> pi;
    PtrSet<const typename Prec<MODE>::V> pb;
    PtrSet<typename Prec<MODE>::V> px;
    for (int z = 0; z < 3; ++z) {
        pi.p[z] = z < nb ? inv[z] : nullptr;
        pb.p[z] = z < nb ? b[z] : nullptr;
        px.p[z] = z < nb ? x[z] : nullptr;
    }
    dim3 g((npts * 32 + 255) / 256, nb);
    k_coarse_apply<MODE><<<g, 256, 0, st>>>(npts, pi, pb, px);
}

#define INST(MODE)                                                                                                 \
    template void launch_jacobi<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                                \
                                      const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double, int, cudaStream_t);     \
    template void launch_residual<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                              \
                                        const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, cudaStream_t);                \
    template void launch_restrict<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&, Prec<MODE>::V* const*, int,  \
                                        cudaStream_t);                                                             \
    template void launch_prolong_add<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                           \
                                           const Prec<MODE>::V* const*, cudaStream_t);                             \
    template void launch_coarse_apply<MODE>(int, int, const double2* const*, const Prec<MODE>::V* const*,         \
                                            Prec<MODE>::V* const*, cudaStream_t);
INST(BAH_FP64)
INST(BAH_MIXED)

}  // namespace bah
