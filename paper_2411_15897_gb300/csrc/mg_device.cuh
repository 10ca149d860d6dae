// Per-point multigrid arithmetic shared by the level kernels: the level-0
// 5-point operator read from per-point coefficient arrays, the Galerkin stencil of radius
// (rx, rz) <= RM, and the diagonal.  The iterate is read through an accessor
// X(flat index), so callers may serve it from global or shared memory; the
// arithmetic (and its order) is the same for every caller.
#pragma once
#include "bah_internal.cuh"

namespace bah {

// one pointer per block of a set, with the element stride between right-hand sides;
// pick() selects without indexing the kernel-parameter array at a run-time index
// (which would copy it to the stack)
template <class V> struct PtrSet { V* p[3]; size_t s = 0; };
template <class V> __device__ __forceinline__ V* pick(const PtrSet<V>& s, int y) {
    return y == 0 ? s.p[0] : (y == 1 ? s.p[1] : s.p[2]);
}

template <int MODE>
struct MGT {
    using V = typename Prec<MODE>::V;
    using R = typename Prec<MODE>::R;
    using C = typename Prec<MODE>::C;
    using CC = typename Prec<MODE>::CC;
};

// A x at point (i, j) of a level-0 block where x is given by an accessor
// XR(dx, dz) relative to the point (a global or a shared-memory tile).
// The four neighbour terms are loaded unconditionally with clamped offsets and
// masked, so the loads issue together.
template <int MODE, class XR>
__device__ __forceinline__ typename MGT<MODE>::V apply_fine5_rel(const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>& f,
                                                                int type, int i, int j, int t, XR X) {
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
    const int ddx[4] = {-1, 1, 0, 0}, ddz[4] = {0, 0, -1, 1};
    R k[4];
    V xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        k[q] = ldr(arr[q][ok[q] ? ci[q] : t]);
        xv[q] = X(ok[q] ? ddx[q] : 0, ok[q] ? ddz[q] : 0);
    }
    const V dg = ldc(dgp[t]);
    V acc = cmul(dg, X(0, 0));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R kk = ok[q] ? k[q] : R(0);
        acc.x -= kk * xv[q].x;
        acc.y -= kk * xv[q].y;
    }
    return acc;
}
// the same with x given by a flat-index accessor X(index)
template <int MODE, class XF>
__device__ __forceinline__ typename MGT<MODE>::V apply_fine5_fn(const Fine5<typename MGT<MODE>::C, typename MGT<MODE>::CC>& f,
                                                               int type, int i, int j, int t, XF X) {
    const int n1 = f.n1;
    return apply_fine5_rel<MODE>(f, type, i, j, t, [&](int dx, int dz) { return X(t + dz * n1 + dx); });
}

// Galerkin stencil product at point (i, j) of a level >= 1: coefficients
// through an accessor S(slot), x through XR(dx, dz).  RM is the compile-time
// maximum radius (1 or 2); rx, rz <= RM are the block's radii.  The loops
// unroll fully and every candidate load is issued with an offset clamped into
// range (out-of-range terms are masked to zero), so all loads go out back to
// back instead of waiting behind per-neighbour branches.
template <int MODE, int RM, class SF, class XR>
__device__ __forceinline__ typename MGT<MODE>::V apply_stencil_rel(SF S, int rx, int rz, int n1, int n2, int i, int j,
                                                                  XR X) {
    using V = typename MGT<MODE>::V;
    using R = typename MGT<MODE>::R;
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
            sv[q] = ldc(S(slot));
            xv[q] = X(in[q] ? dx : 0, in[q] ? dz : 0);
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

// the stencil read from global memory (slot-major [slots][points]), x by flat index
template <int MODE, int RM, class XF>
__device__ __forceinline__ typename MGT<MODE>::V apply_stencil_fn(const typename MGT<MODE>::CC* __restrict__ S, int rx,
                                                                 int rz, int n1, int n2, int i, int j, int t, XF X) {
    const size_t np = (size_t)n1 * n2;
    return apply_stencil_rel<MODE, RM>([&](int slot) { return S[(size_t)slot * np + t]; }, rx, rz, n1, n2, i, j,
                                       [&](int dx, int dz) { return X(t + dz * n1 + dx); });
}

// the stencil through an accessor S(slot) (e.g. shared memory), x by flat index
template <int MODE, int RM, class SF, class XF>
__device__ __forceinline__ typename MGT<MODE>::V apply_stencil_acc(SF S, int rx, int rz, int n1, int n2, int i, int j,
                                                                  int t, XF X) {
    return apply_stencil_rel<MODE, RM>(S, rx, rz, n1, n2, i, j, [&](int dx, int dz) { return X(t + dz * n1 + dx); });
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

}  // namespace bah
