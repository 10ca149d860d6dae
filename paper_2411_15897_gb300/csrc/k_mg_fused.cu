// Fused level visits for the multigrid levels above the cluster-resident ones
// (Sec. 2.2, Algorithm 1; Sec. 4.4.1).
//
// A zero-guess visit of a level in a V(1, nu) or W(1, nu) cycle is a chain of
// dependent sweeps: damped Jacobi from zero, residual, restriction, then --
// after the coarse correction -- prolongation with correction and nu damped
// Jacobi sweeps.  Run as separate launches each link is a few microseconds of
// launch and grid ramp over a grid that is small for the GPU.  Here the chain
// becomes two launches per level:
//
//   down:  x = w D^{-1} b on the tile plus a halo of 1 + r, the residual
//          b - A x on the tile plus 1 point, x written on the tile, and
//          b_c = R (b - A x) on the coarse points the tile owns;
//   up:    y = x + P e on the tile plus a halo of nu r, then nu sweeps, each
//          on a region r smaller than the last, the final one on the tile.
//
// r is the stencil radius (1 on the fine level, the Galerkin radius below).
// Each CTA owns a TX x TY tile of points and recomputes the halo values it
// needs in shared memory, so no CTA reads another's results within a launch.
// The per-point arithmetic is the separate kernels' (the accessors of
// mg_device.cuh, same operand order), so both schedules give the same
// iterates up to the compiler's contraction of multiply-adds.
#include "bah_internal.cuh"
#include "intergrid.cuh"
#include "mg_device.cuh"

#include <algorithm>

namespace bah {

// a rectangular region of the level grid, [i0, i0 + w) x [j0, j0 + h), held
// in shared memory with x fastest
struct Reg {
    int i0, j0, w, h;
    __device__ __forceinline__ int idx(int i, int j) const { return (j - j0) * w + (i - i0); }
    __device__ __forceinline__ int size() const { return w * h; }
};
__device__ __forceinline__ Reg grow(int x0, int y0, int tx, int ty, int halo) {
    return Reg{x0 - halo, y0 - halo, tx + 2 * halo, ty + 2 * halo};
}

// A x at (i, j) with x in a shared-memory region (level 0: the 5-point
// operator from the per-point arrays; below: the Galerkin stencil of radius
// <= RM from global memory)
template <int MODE, bool L0, int RM>
__device__ __forceinline__ typename MGT<MODE>::V ax_tile(const LvlBlk<typename MGT<MODE>::V, typename MGT<MODE>::CC>& B,
                                                         const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>& f5,
                                                         int n1, int n2, int i, int j, int t,
                                                         const typename MGT<MODE>::V* buf, const Reg& rg) {
    const int c = rg.idx(i, j);
    const int w = rg.w;
    auto X = [&](int dx, int dz) { return buf[c + dz * w + dx]; };
    if constexpr (L0) {
        return apply_fine5_rel<MODE>(f5, B.type, i, j, t, X);
    } else {
        const size_t np = (size_t)n1 * n2;
        const auto* S = B.S;
        return apply_stencil_rel<MODE, RM>([&](int slot) { return S[(size_t)slot * np + t]; }, B.rx, B.rz, n1, n2, i,
                                           j, X);
    }
}

// ---------------------------------------------------------------------------
// down: zero-guess damped Jacobi, residual, restriction.  Tile TX x TY (even,
// so the tile owns whole coarse cells).  Dynamic shared memory: the iterate on
// the tile plus 1 + r, the residual on the tile plus 1.
// ---------------------------------------------------------------------------
template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_level_down(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                    Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                    typename MGT<MODE>::R w, PtrSet<typename MGT<MODE>::V> cb,
                                                    int intergrid, int tx, int ty) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    constexpr int RR = L0 ? 1 : RM;
    const auto& B = s.blk[blockIdx.y];
    const int rr = blockIdx.z;
    if (s.active && !s.active[rr]) return;
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2;
    const int ntx = (n1 + tx - 1) / tx;
    const int x0 = (blockIdx.x % ntx) * tx, y0 = (blockIdx.x / ntx) * ty;
    const V* b = B.b + rr * B.sb;
    V* xo = B.xout + rr * B.sxo;
    const auto* pf5 = L0 ? &f5 : nullptr;
    extern __shared__ __align__(16) unsigned char fused_raw[];
    const Reg rx = grow(x0, y0, tx, ty, 1 + RR), rrg = grow(x0, y0, tx, ty, 1);
    V* xs = reinterpret_cast<V*>(fused_raw);
    V* rs = xs + rx.size();
    // x = w D^{-1} b on the tile plus 1 + r (zero outside the grid and on structural zeros)
    for (int e = threadIdx.x; e < rx.size(); e += blockDim.x) {
        const int i = rx.i0 + e % rx.w, j = rx.j0 + e / rx.w;
        V v = czero<V>();
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && valid_pt(B.type, i, j)) {
            const int t = j * n1 + i;
            v = cscale(cdiv(b[t], diag_only<MODE>(pf5, B, np, t)), w);
        }
        xs[e] = v;
    }
    __syncthreads();
    // r = b - A x on the tile plus 1
    for (int e = threadIdx.x; e < rrg.size(); e += blockDim.x) {
        const int i = rrg.i0 + e % rrg.w, j = rrg.j0 + e / rrg.w;
        V v = czero<V>();
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && valid_pt(B.type, i, j)) {
            const int t = j * n1 + i;
            v = csub(b[t], ax_tile<MODE, L0, RM>(B, f5, n1, n2, i, j, t, xs, rx));
        }
        rs[e] = v;
    }
    // the smoothed iterate on the tile
    for (int e = threadIdx.x; e < tx * ty; e += blockDim.x) {
        const int i = x0 + e % tx, j = y0 + e / tx;
        if (i < n1 && j < n2) xo[j * n1 + i] = xs[rx.idx(i, j)];
    }
    __syncthreads();
    // b_c = R r on the tile's coarse points (their support lies in the residual region)
    const int n1c = n1 / 2, n2c = n2 / 2;
    V* bc = cb.p[blockIdx.y] + rr * cb.s;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    for (int e = threadIdx.x; e < (tx / 2) * (ty / 2); e += blockDim.x) {
        const int I = x0 / 2 + e % (tx / 2), J = y0 / 2 + e / (tx / 2);
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
                    v[a * 4 + q] = rs[ok ? rrg.idx(bx + q, bz + a) : 0];
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

// ---------------------------------------------------------------------------
// up: prolongation with correction, then nu damped Jacobi sweeps.  Dynamic
// shared memory: y on the tile plus nu r (buffer A), the first sweep's result
// on the tile plus (nu - 1) r (buffer B), and b on that region.  Sweep k reads
// one buffer and writes the other on a region r smaller per side; the last
// sweep writes the tile to global memory.
// ---------------------------------------------------------------------------
template <int MODE, bool L0, int RM>
__global__ void __launch_bounds__(256) k_level_up(LvlSet<typename MGT<MODE>::V, typename MGT<MODE>::CC> s,
                                                  Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC> f5,
                                                  typename MGT<MODE>::R w, PtrSet<typename MGT<MODE>::V> ce, int nu,
                                                  int tx, int ty) {
    pdl_prologue();
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
    constexpr int RR = L0 ? 1 : RM;
    const auto& B = s.blk[blockIdx.y];
    const int rr = blockIdx.z;
    if (s.active && !s.active[rr]) return;
    const int n1 = s.n1, n2 = s.n2, np = n1 * n2, n1c = n1 / 2;
    const int ntx = (n1 + tx - 1) / tx;
    const int x0 = (blockIdx.x % ntx) * tx, y0 = (blockIdx.x / ntx) * ty;
    const V* b = B.b + rr * B.sb;
    const V* xi = B.xin + rr * B.sxi;
    V* xo = B.xout + rr * B.sxo;
    const V* ec = ce.p[blockIdx.y] + rr * ce.s;
    const auto* pf5 = L0 ? &f5 : nullptr;
    const bool nodx = B.type == 0, nodz = B.type == 1;
    extern __shared__ __align__(16) unsigned char fused_raw[];
    const Reg ra = grow(x0, y0, tx, ty, nu * RR), rb1 = grow(x0, y0, tx, ty, (nu - 1) * RR);
    V* bufA = reinterpret_cast<V*>(fused_raw);
    V* bufB = bufA + ra.size();
    V* bs = bufB + rb1.size();
    // y = x + P e on the tile plus nu r; b on the tile plus (nu - 1) r
    for (int e = threadIdx.x; e < ra.size(); e += blockDim.x) {
        const int i = ra.i0 + e % ra.w, j = ra.j0 + e / ra.w;
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
        bufA[e] = acc;
    }
    for (int e = threadIdx.x; e < rb1.size(); e += blockDim.x) {
        const int i = rb1.i0 + e % rb1.w, j = rb1.j0 + e / rb1.w;
        bs[e] = (i >= 0 && i < n1 && j >= 0 && j < n2) ? b[j * n1 + i] : czero<V>();
    }
    __syncthreads();
    // one damped Jacobi sweep at (i, j) from the region rin held in src
    auto sweep = [&](const V* src, const Reg& rin, int i, int j) -> V {
        if (!valid_pt(B.type, i, j)) return czero<V>();
        const int t = j * n1 + i;
        const V ax = ax_tile<MODE, L0, RM>(B, f5, n1, n2, i, j, t, src, rin);
        const V dg = diag_only<MODE>(pf5, B, np, t);
        const V corr = cdiv(csub(bs[rb1.idx(i, j)], ax), dg);
        const V xv = src[rin.idx(i, j)];
        return cmk<V>(xv.x + w * corr.x, xv.y + w * corr.y);
    };
    const V* src = bufA;
    V* dst = bufB;
    Reg rin = ra;
    for (int k = 1; k < nu; ++k) {
        const Reg rout = grow(x0, y0, tx, ty, (nu - k) * RR);
        for (int e = threadIdx.x; e < rout.size(); e += blockDim.x) {
            const int i = rout.i0 + e % rout.w, j = rout.j0 + e / rout.w;
            dst[e] = (i >= 0 && i < n1 && j >= 0 && j < n2) ? sweep(src, rin, i, j) : czero<V>();
        }
        __syncthreads();
        rin = rout;
        const V* t_ = dst;
        dst = const_cast<V*>(src);
        src = t_;
    }
    // the last sweep on the tile, written out
    for (int e = threadIdx.x; e < tx * ty; e += blockDim.x) {
        const int i = x0 + e % tx, j = y0 + e / tx;
        if (i < n1 && j < n2) xo[j * n1 + i] = sweep(src, rin, i, j);
    }
}

// tile shape per level: 32 x 32 on grids of at least 512 x 256 points, else
// 32 x 16 (twice the CTAs on the smaller grids, where the GPU is not filled)
static void fused_tile(int n1, int n2, int& tx, int& ty) {
    tx = 32;
    ty = ((long long)n1 * n2 >= 512LL * 256) ? 32 : 16;
}

template <class LS>
static inline int max_radius_f(const LS& s) {
    int r = 0;
    for (int z = 0; z < s.nb; ++z) r = std::max(r, std::max(s.blk[z].rx, s.blk[z].rz));
    return r;
}

static bool set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <int MODE>
size_t fused_down_smem(int n1, int n2, bool l0, int rm) {
    int tx, ty;
    fused_tile(n1, n2, tx, ty);
    const int rr = l0 ? 1 : rm;
    const size_t a = (size_t)(tx + 2 + 2 * rr) * (ty + 2 + 2 * rr), r = (size_t)(tx + 2) * (ty + 2);
    return (a + r) * sizeof(typename Prec<MODE>::V);
}
template <int MODE>
size_t fused_up_smem(int n1, int n2, bool l0, int rm, int nu) {
    int tx, ty;
    fused_tile(n1, n2, tx, ty);
    const int rr = l0 ? 1 : rm;
    const size_t a = (size_t)(tx + 2 * nu * rr) * (ty + 2 * nu * rr);
    const size_t b1 = (size_t)(tx + 2 * (nu - 1) * rr) * (ty + 2 * (nu - 1) * rr);
    return (a + 2 * b1) * sizeof(typename Prec<MODE>::V);
}

template <int MODE>
int launch_level_down(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                      const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                      typename Prec<MODE>::V* const* coarse_b, int intergrid, cudaStream_t st, size_t coarse_stride) {
    using R = typename Prec<MODE>::R;
    PtrSet<typename Prec<MODE>::V> cb;
    for (int z = 0; z < 3; ++z) cb.p[z] = z < s.nb ? coarse_b[z] : nullptr;
    cb.s = coarse_stride;
    Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    int tx, ty;
    fused_tile(s.n1, s.n2, tx, ty);
    const int rm = f5 ? 1 : max_radius_f(s);
    const size_t smem = fused_down_smem<MODE>(s.n1, s.n2, f5 != nullptr, rm);
    const int tiles = ((s.n1 + tx - 1) / tx) * ((s.n2 + ty - 1) / ty);
    dim3 g(tiles, s.nb, s.nrhs);
    if (f5) {
        if (!set_smem((const void*)k_level_down<MODE, true, 1>, smem)) return -1;
        launch_pdl(k_level_down<MODE, true, 1>, g, dim3(256), smem, st, s, *f5, (R)w, cb, intergrid, tx, ty);
    } else if (rm <= 1) {
        if (!set_smem((const void*)k_level_down<MODE, false, 1>, smem)) return -1;
        launch_pdl(k_level_down<MODE, false, 1>, g, dim3(256), smem, st, s, nof, (R)w, cb, intergrid, tx, ty);
    } else {
        if (!set_smem((const void*)k_level_down<MODE, false, 2>, smem)) return -1;
        launch_pdl(k_level_down<MODE, false, 2>, g, dim3(256), smem, st, s, nof, (R)w, cb, intergrid, tx, ty);
    }
    return 0;
}

template <int MODE>
int launch_level_up(const LvlSet<typename Prec<MODE>::V, typename Prec<MODE>::CC>& s,
                    const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>* f5, double w,
                    const typename Prec<MODE>::V* const* coarse_x, int nu, cudaStream_t st, size_t coarse_stride) {
    using R = typename Prec<MODE>::R;
    PtrSet<typename Prec<MODE>::V> ce;
    for (int z = 0; z < 3; ++z) ce.p[z] = z < s.nb ? const_cast<typename Prec<MODE>::V*>(coarse_x[z]) : nullptr;
    ce.s = coarse_stride;
    Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> nof{};
    int tx, ty;
    fused_tile(s.n1, s.n2, tx, ty);
    const int rm = f5 ? 1 : max_radius_f(s);
    const size_t smem = fused_up_smem<MODE>(s.n1, s.n2, f5 != nullptr, rm, nu);
    const int tiles = ((s.n1 + tx - 1) / tx) * ((s.n2 + ty - 1) / ty);
    dim3 g(tiles, s.nb, s.nrhs);
    if (f5) {
        if (!set_smem((const void*)k_level_up<MODE, true, 1>, smem)) return -1;
        launch_pdl(k_level_up<MODE, true, 1>, g, dim3(256), smem, st, s, *f5, (R)w, ce, nu, tx, ty);
    } else if (rm <= 1) {
        if (!set_smem((const void*)k_level_up<MODE, false, 1>, smem)) return -1;
        launch_pdl(k_level_up<MODE, false, 1>, g, dim3(256), smem, st, s, nof, (R)w, ce, nu, tx, ty);
    } else {
        if (!set_smem((const void*)k_level_up<MODE, false, 2>, smem)) return -1;
        launch_pdl(k_level_up<MODE, false, 2>, g, dim3(256), smem, st, s, nof, (R)w, ce, nu, tx, ty);
    }
    return 0;
}

#define INST_FUSED(MODE)                                                                                          \
    template size_t fused_down_smem<MODE>(int, int, bool, int);                                                  \
    template size_t fused_up_smem<MODE>(int, int, bool, int, int);                                                \
    template int launch_level_down<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                            \
                                         const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double, Prec<MODE>::V* const*, \
                                         int, cudaStream_t, size_t);                                               \
    template int launch_level_up<MODE>(const LvlSet<Prec<MODE>::V, Prec<MODE>::CC>&,                              \
                                       const Fine5<Prec<MODE>::C, Prec<MODE>::CC>*, double,                       \
                                       const Prec<MODE>::V* const*, int, cudaStream_t, size_t);
INST_FUSED(BAH_FP64)
INST_FUSED(BAH_MIXED)

}  // namespace bah
