// The three rows of y = H x at one cell of a 2-D grid (Eq. 2.6), in FP64:
//   u1 row:  (diag A_1) u1 - sum of the four mu-weighted neighbours + (grad_h p)_1
//   u2 row:  the same along x_2
//   p row:   (B u - C p) = -div_h u - p / (lambda + mu)
// The entries of x are read through accessors U1(i, j), U2(i, j) (zero
// outside the unknowns of the component) and P(flat index), so every kernel
// that needs H x (the operator launches and the allocation-free residual)
// shares one definition of the stencil.  sg = -1 applies H^H = conj(H).
#pragma once
#include "bah_internal.cuh"

namespace bah {

template <class FU1, class FU2, class FP>
__device__ __forceinline__ void elastic_rows(const OpCoef& c, int i, int j, int t, double sg, FU1 U1, FU2 U2, FP P,
                                             double2& y1, double2& y2, double2& yp) {
    const int n1 = c.n1, n2 = c.n2;
    const double2 z = make_double2(0.0, 0.0);
    const double2 p = P(t);
    y1 = z;
    y2 = z;
    if (i >= 1) {
        const double2 u = U1(i, j);
        double2 d = c.d1[t];
        d.y *= sg;
        double2 a = cmul(d, u);
        const double2 uw = U1(i - 1, j), ue = U1(i + 1, j), us = U1(i, j - 1), un = U1(i, j + 1);
        const double kw = c.cx[t - 1], ke = c.cx[t];
        const double ks = c.nz[t], kn = (j + 1 < n2) ? c.nz[t + n1] : 0.0;
        a.x -= kw * uw.x + ke * ue.x + ks * us.x + kn * un.x;
        a.y -= kw * uw.y + ke * ue.y + ks * us.y + kn * un.y;
        const double2 pw = P(t - 1);
        a.x += c.ihx * (p.x - pw.x);
        a.y += c.ihx * (p.y - pw.y);
        y1 = a;
    }
    if (j >= 1) {
        const double2 u = U2(i, j);
        double2 d = c.d2[t];
        d.y *= sg;
        double2 a = cmul(d, u);
        const double2 us = U2(i, j - 1), un = U2(i, j + 1), uw = U2(i - 1, j), ue = U2(i + 1, j);
        const double ks = c.cz[t - n1], kn = c.cz[t];
        const double kw = c.nx[t], ke = (i + 1 < n1) ? c.nx[t + 1] : 0.0;
        a.x -= ks * us.x + kn * un.x + kw * uw.x + ke * ue.x;
        a.y -= ks * us.y + kn * un.y + kw * uw.y + ke * ue.y;
        const double2 ps = P(t - n1);
        a.x += c.ihz * (p.x - ps.x);
        a.y += c.ihz * (p.y - ps.y);
        y2 = a;
    }
    const double2 u1c = U1(i, j), u1e = U1(i + 1, j), u2c = U2(i, j), u2n = U2(i, j + 1);
    const double ci = c.cinv[t];
    yp.x = c.ihx * (u1c.x - u1e.x) + c.ihz * (u2c.x - u2n.x) - ci * p.x;
    yp.y = c.ihx * (u1c.y - u1e.y) + c.ihz * (u2c.y - u2n.y) - ci * p.y;
}

}  // namespace bah
