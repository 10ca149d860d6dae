// 1-D intergrid weights shared by the Galerkin setup and the multigrid
// transfer kernels.
#pragma once
#include "bah_internal.cuh"

namespace bah {

// ---------------------------------------------------------------------------
// 1-D intergrid weights.  P is bilinear interpolation (rows sum to one), the
// restriction is R = P^T / 2 per axis (1/4[1 2 1] nodal, 1/8[1 3 3 1] cell,
// Eq. 4.1, 4.2) or the mixed 1/2[1 1] along cell axes (Eq. 4.4).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double pw_nodal(int nfine, int f, int c) {
    const int nc = nfine / 2;
    if (f < 1 || f > nfine - 1 || c < 1 || c > nc - 1) return 0.0;
    const int d = f - 2 * c;
    return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);
}
__host__ __device__ __forceinline__ double pw_cell(int nfine, int f, int c) {
    const int nc = nfine / 2;
    if (f < 0 || f > nfine - 1 || c < 0 || c > nc - 1) return 0.0;
    const int J = f >> 1;
    int nb = (f & 1) ? J + 1 : J - 1;
    nb = nb < 0 ? 0 : (nb > nc - 1 ? nc - 1 : nb);
    return (c == J ? 0.75 : 0.0) + (c == nb ? 0.25 : 0.0);
}
__host__ __device__ __forceinline__ double pw_axis(bool nodal, int nfine, int f, int c) {
    return nodal ? pw_nodal(nfine, f, c) : pw_cell(nfine, f, c);
}
__host__ __device__ __forceinline__ double rw_axis(bool nodal, int intergrid, int nfine, int c, int f) {
    if (nodal) return 0.5 * pw_nodal(nfine, f, c);
    if (intergrid == BAH_INTERGRID_MIXED) {
        const int nc = nfine / 2;
        if (f < 0 || f > nfine - 1 || c < 0 || c > nc - 1) return 0.0;
        return (f >> 1) == c ? 0.5 : 0.0;
    }
    return 0.5 * pw_cell(nfine, f, c);
}

// Same weights evaluated in the arithmetic type T of the caller (the values
// 0, 1/8, 1/4, 3/8, 1/2, 3/4, 1 are exact in FP32), so the FP32 multigrid
// kernels do no FP64 arithmetic.
template <class T>
__host__ __device__ __forceinline__ T pw_axis_t(bool nodal, int nfine, int f, int c) {
    const int nc = nfine / 2;
    if (nodal) {
        if (f < 1 || f > nfine - 1 || c < 1 || c > nc - 1) return T(0);
        const int d = f - 2 * c;
        return d == 0 ? T(1) : ((d == 1 || d == -1) ? T(0.5) : T(0));
    }
    if (f < 0 || f > nfine - 1 || c < 0 || c > nc - 1) return T(0);
    const int J = f >> 1;
    int nb = (f & 1) ? J + 1 : J - 1;
    nb = nb < 0 ? 0 : (nb > nc - 1 ? nc - 1 : nb);
    return (c == J ? T(0.75) : T(0)) + (c == nb ? T(0.25) : T(0));
}
template <class T>
__host__ __device__ __forceinline__ T rw_axis_t(bool nodal, int intergrid, int nfine, int c, int f) {
    if (!nodal && intergrid == BAH_INTERGRID_MIXED) {
        const int nc = nfine / 2;
        if (f < 0 || f > nfine - 1 || c < 0 || c > nc - 1) return T(0);
        return (f >> 1) == c ? T(0.5) : T(0);
    }
    return T(0.5) * pw_axis_t<T>(nodal, nfine, f, c);
}

// first fine index of the 4-wide restriction support of coarse index c
__host__ __device__ __forceinline__ int rbase(bool nodal, int intergrid, int c) {
    return nodal ? 2 * c - 1 : (intergrid == BAH_INTERGRID_MIXED ? 2 * c : 2 * c - 1);
}

}  // namespace bah
