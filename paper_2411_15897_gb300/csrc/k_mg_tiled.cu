// Tiled fused multigrid level kernels (Sec. 2.2, Algorithm 1; Sec. 4.4.1).
//
// A V(1,2) or W(1,2) visit of a level with a zero initial guess runs six
// dependent sweeps: damped Jacobi from zero, residual, restriction, then --
// after the coarse correction -- prolongation with correction and two Jacobi
// sweeps.  On the levels above the cluster-resident ones each of these is a
// launch of a few microseconds over a grid that is too small to hide its
// latency.  Here the six become two launches:
//
//   down:  x = w D^{-1} b on a tile plus halo, r = b - A x on the tile plus
//          one point, x written on the tile, b_c = R r on the tile's coarse
//          points;
//   up:    x + P e on the tile plus two stencil radii, one sweep on the tile
//          plus one radius, the second sweep on the tile, written out.
//
// Each CTA owns a TX x TY tile of fine points and recomputes the halo values
// it needs in shared memory (cheap: the zero-guess sweep is a division, the
// prolongation 9 taps), so no other CTA's results are read within a launch.
// The per-point arithmetic is the one of the separate kernels (the helpers of
// mg_device.cuh with the same accumulation order), so both schedules give the
// same iterates up to the compiler's contraction of multiply-adds.
#include "bah_internal.cuh"
#include "intergrid.cuh"
#include "mg_device.cuh"

#include <algorithm>

namespace bah {

constexpr int kTX = 32, kTY = 16;   // fine tile (even, so a tile owns whole coarse cells)

template <class LS>
static inline int max_radius_t(const LS& s) {
    int r = 0;
    for (int z = 0; z < s.nb; ++z) r = std::max(r, std::max(s.blk[z].rx, s.blk[z].rz));
    return r;
}

// accessor from a flat grid index g near own point t (|di|, |dj| <= 2) to the
// shared tile in which t sits at local index lb; n1 >= 8 makes the rounded
// quotient the row offset exactly
template <class V>
struct TileX {
    const V* tile;
    int lb, t, n1, tw;
    float inv_n1;
    __device__ __forceinline__ V operator()(int g) const {
        const int d = g - t;
        const int dz = __float2int_rn((float)d * inv_n1);
        const int dx = d - dz * n1;
        return tile[lb + dz * tw + dx];
    }
};

template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_down_tiled(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                    Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                    typename MGT<MODE>::R w, PtrSet<typename MGT<MODE>::V> cb,
                                                    int intergrid) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    constexpr int RR = L0 ? 1 : RM;                       // stencil radius
    constexpr int XW = kTX + 2 + 2 * RR, XH = kTY + 2 + 2 * RR;
    constexpr int RW = kTX + 2, RH = kTY + 2;
    __shared__ V xs[XH * XW];
    __shared__ V rs[RH * RW];
    const auto& B = s.blk[blockIdx.y];
    const int rr = blockIdx.z;
    if (s.active && !s.active[rr]) return;
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int ntx = (n1 + kTX - 1) / kTX;
    const int x0 = (blockIdx.x % ntx) * kTX, y0 = (blockIdx.x / ntx) * kTY;
    const V* b = B.b + rr * B.sb;
    V* xo = B.xout + rr * B.sxo;
    const float inv_n1 = 1.0f / (float)n1;
    const auto* pf5 = L0 ? &f5 : nullptr;
    // zero-guess damped Jacobi on the tile and a halo of 1 + RR
    for (int e = threadIdx.x; e < XH * XW; e += blockDim.x) {
        const int i = x0 - 1 - RR + e % XW, j = y0 - 1 - RR + e / XW;
        V v = czero<V>();
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && valid_pt(B.type, i, j)) {
            const int t = j * n1 + i;
            v = cscale(cdiv(b[t], diag_only<MODE>(pf5, B, np, t)), w);
        }
        xs[e] = v;
    }
    __syncthreads();
    // residual on the tile and a halo of 1
    for (int e = threadIdx.x; e < RH * RW; e += blockDim.x) {
        const int li = e % RW, lj = e / RW;
        const int i = x0 - 1 + li, j = y0 - 1 + lj;
        V v = czero<V>();
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && valid_pt(B.type, i, j)) {
            const int t = j * n1 + i;
            const TileX<V> X{xs, (lj + RR) * XW + li + RR, t, n1, XW, inv_n1};
            V ax;
            if constexpr (L0) ax = apply_fine5_fn<MODE>(f5, B.type, i, j, t, X);
            else ax = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, i, j, t, X);
            v = csub(b[t], ax);
        }
        rs[e] = v;
    }
    __syncthreads();
    // the smoothed iterate on the tile
    for (int e = threadIdx.x; e < kTX * kTY; e += blockDim.x) {
        const int i = x0 + e % kTX, j = y0 + e / kTX;
        if (i < n1 && j < n2) xo[j * n1 + i] = xs[(e / kTX + 1 + RR) * XW + e % kTX + 1 + RR];
    }
    // restriction to the tile's coarse points (support within the residual tile)
    const int n1c = n1 / 2, n2c = n2 / 2;
    V* bc = cb.p[blockIdx.y] + rr * cb.s;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    for (int e = threadIdx.x; e < (kTX / 2) * (kTY / 2); e += blockDim.x) {
        const int I = x0 / 2 + e % (kTX / 2), J = y0 / 2 + e / (kTX / 2);
        if (I >= n1c || J >= n2c) continue;
        V acc = czero<V>();
        if (valid_pt(B.type, I, J)) {
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
                    v[a * 4 + q] = rs[ok ? (bz + a - (y0 - 1)) * RW + (bx + q - (x0 - 1)) : 0];
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
        bc[J * n1c + I] = acc;
    }
}

template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_up_tiled(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                  Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                  typename MGT<MODE>::R w, PtrSet<typename MGT<MODE>::V> ce) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    constexpr int RR = L0 ? 1 : RM;
    constexpr int AW = kTX + 4 * RR, AH = kTY + 4 * RR;   // prolonged iterate
    constexpr int BW = kTX + 2 * RR, BH = kTY + 2 * RR;   // after the first sweep
    __shared__ V xa[AH * AW];
    __shared__ V xb[BH * BW];
    const auto& B = s.blk[blockIdx.y];
    const int rr = blockIdx.z;
    if (s.active && !s.active[rr]) return;
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2, n1c = n1 / 2;
    const int ntx = (n1 + kTX - 1) / kTX;
    const int x0 = (blockIdx.x % ntx) * kTX, y0 = (blockIdx.x / ntx) * kTY;
    const V* b = B.b + rr * B.sb;
    const V* xi = B.xin + rr * B.sxi;
    V* xo = B.xout + rr * B.sxo;
    const V* ec = ce.p[blockIdx.y] + rr * ce.s;
    const float inv_n1 = 1.0f / (float)n1;
    const auto* pf5 = L0 ? &f5 : nullptr;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    // x + P e on the tile and a halo of 2 RR
    for (int e = threadIdx.x; e < AH * AW; e += blockDim.x) {
        const int i = x0 - 2 * RR + e % AW, j = y0 - 2 * RR + e / AW;
        V acc = czero<V>();
        if (i >= 0 && i < n1 && j >= 0 && j < n2) {
            acc = xi[j * n1 + i];
            if (valid_pt(B.type, i, j)) {
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
                        v[a * 3 + q] = ec[ok ? ((j >> 1) - 1 + a) * n1c + ((i >> 1) - 1 + q) : 0];
                    }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const R wgt = pz[a] * px[q];
                        acc.x += wgt * v[a * 3 + q].x;
                        acc.y += wgt * v[a * 3 + q].y;
                    }
            }
        }
        xa[e] = acc;
    }
    __syncthreads();
    // one damped Jacobi sweep of x (source tile, halo in src) at grid point (i, j)
    auto sweep = [&](const V* src, int sw, int lb, int i, int j) -> V {
        if (!valid_pt(B.type, i, j)) return czero<V>();
        const int t = j * n1 + i;
        const TileX<V> X{src, lb, t, n1, sw, inv_n1};
        V ax;
        if constexpr (L0) ax = apply_fine5_fn<MODE>(f5, B.type, i, j, t, X);
        else ax = apply_stencil_fn<MODE, RM>(B.S, B.rx, B.rz, n1, n2, i, j, t, X);
        const V dg = diag_only<MODE>(pf5, B, np, t);
        const V corr = cdiv(csub(b[t], ax), dg);
        const V xv = src[lb];
        return cmk<V>(xv.x + w * corr.x, xv.y + w * corr.y);
    };
    // first sweep on the tile and a halo of RR
    for (int e = threadIdx.x; e < BH * BW; e += blockDim.x) {
        const int li = e % BW, lj = e / BW;
        const int i = x0 - RR + li, j = y0 - RR + lj;
        xb[e] = (i >= 0 && i < n1 && j >= 0 && j < n2) ? sweep(xa, AW, (lj + RR) * AW + li + RR, i, j) : czero<V>();
    }
    __syncthreads();
    // second sweep on the tile, written out
    for (int e = threadIdx.x; e < kTX * kTY; e += blockDim.x) {
        const int li = e % kTX, lj = e / kTX;
        const int i = x0 + li, j = y0 + lj;
        if (i < n1 && j < n2) xo[j * n1 + i] = sweep(xb, BW, (lj + RR) * BW + li + RR, i, j);
    }
}

template <int MODE>
void launch_down_tiled(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                       const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                       typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st, size_t coarse_stride) {
    using R = typename Prec<MODE>::R;
    PtrSet<typename Prec<MODE>::V> cb;
    for (int z = 0; z < 3; ++z) cb.p[z] = z < s.nb ? coarse_b[z] : nullptr;
    cb.s = coarse_stride;
    Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    const int tiles = ((s.n1 + kTX - 1) / kTX) * ((s.n2 + kTY - 1) / kTY);
    dim3 g(tiles, s.nb, s.nrhs);
    if (f5) launch_pdl(k_down_tiled<MODE, true, 1>, g, dim3(256), 0, st, s, *f5, (R)w, cb, intergrid);
    else if (max_radius_t(s) <= 1) launch_pdl(k_down_tiled<MODE, false, 1>, g, dim3(256), 0, st, s, nof, (R)w, cb, intergrid);
    else launch_pdl(k_down_tiled<MODE, false, 2>, g, dim3(256), 0, st, s, nof, (R)w, cb, intergrid);
}

template <int MODE>
void launch_up_tiled(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                     const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                     const typename Prec<MODE>::V* const* coarse_x, cudaStream_t st, size_t coarse_stride) {
    using R = typename Prec<MODE>::R;
    PtrSet<typename Prec<MODE>::V> ce;
    for (int z = 0; z < 3; ++z) ce.p[z] = z < s.nb ? const_cast<typename Prec<MODE>::V*>(coarse_x[z]) : nullptr;
    ce.s = coarse_stride;
    Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    const int tiles = ((s.n1 + kTX - 1) / kTX) * ((s.n2 + kTY - 1) / kTY);
    dim3 g(tiles, s.nb, s.nrhs);
    if (f5) launch_pdl(k_up_tiled<MODE, true, 1>, g, dim3(256), 0, st, s, *f5, (R)w, ce);
    else if (max_radius_t(s) <= 1) launch_pdl(k_up_tiled<MODE, false, 1>, g, dim3(256), 0, st, s, nof, (R)w, ce);
    else launch_pdl(k_up_tiled<MODE, false, 2>, g, dim3(256), 0, st, s, nof, (R)w, ce);
}

#define INST_TILED(MODE)                                                                                          \
    template void launch_down_tiled<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                           \
                                          const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double, Prec<MODE>::V* const*, \
                                          int, cudaStream_t, size_t);                                              \
    template void launch_up_tiled<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                             \
                                        const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double,                      \
                                        const Prec<MODE>::V* const*, cudaStream_t, size_t);
INST_TILED(BAH_FP64)
INST_TILED(BAH_MIXED)

}  // namespace bah
