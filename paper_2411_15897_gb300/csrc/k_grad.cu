// Kernels of the adjoint gradient of a receiver misfit
// J = 1/2 sum_s ||Q x_s - d_s||^2 with respect to lambda, mu, rho:
//   * adjoint source Q^H (Q x_s - d_s) and the per-source misfit;
//   * element-wise conjugation (H^H = conj(H) for the complex-symmetric H of
//     Eq. 2.6, so H^H y = b is solved as H conj(y) = conj(b));
//   * the pointwise gradient  dJ/dm_k = -Re sum_s y_s^H (dH/dm_k) x_s, written
//     out per cell from the structure of H: lambda enters through
//     -C = -diag(1/(lambda+mu)), mu through A_e(mu) (own-direction
//     derivatives at the cell, cross derivatives at the 4 nodes around it
//     with weight 1/4) and through C, rho through the face mass
//     A_f(rho (1 - i gamma/omega)) of the faces around the cell.
#include "bah_internal.cuh"

namespace bah {

__global__ void k_conj(double2* v, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        v[e].y = -v[e].y;
}
void launch_conj(double2* v, size_t n, cudaStream_t st) {
    k_conj<<<RED_CTAS * 2, 256, 0, st>>>(v, n);
}

// adj_s = Q^H (Q x_s - d_s) (adj zeroed beforehand): adj[s][rec[q]] gathers
// x[s][rec[q]] - d[s][q] of every q naming that entry, so a receiver listed
// twice is counted twice, as in J; one thread adds them in the order of q, so
// the result does not depend on scheduling.  misfit[s] = 1/2 sum_q |x - d|^2
// (one CTA per source, fixed-order block reduction).
__global__ void __launch_bounds__(256) k_misfit(const double2* __restrict__ x, const double2* __restrict__ d,
                                                const int* __restrict__ rec, int nrec, size_t vlen, double2* adj,
                                                double* misfit) {
    const int s = blockIdx.x;
    const double2* xs = x + (size_t)s * vlen;
    const double2* ds = d + (size_t)s * nrec;
    double2* as = adj + (size_t)s * vlen;
    double acc = 0.0;
    for (int q = threadIdx.x; q < nrec; q += blockDim.x) {
        const double2 r = csub(xs[rec[q]], ds[q]);
        acc += r.x * r.x + r.y * r.y;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < nrec; ++q) {
            const int i = rec[q];
            as[i] = cadd(as[i], csub(xs[i], ds[q]));
        }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) misfit[s] = 0.5 * sh[0];
}
void launch_misfit(const double2* x, const double2* d, const int* rec, int nrec, int nrhs, size_t vlen, double2* adj,
                   double* misfit, cudaStream_t st) {
    k_misfit<<<nrhs, 256, 0, st>>>(x, d, rec, nrec, vlen, adj, misfit);
}

struct GradArgs {
    int n1, n2;
    double ih1, ih2, omega;
    const double* cinv;     // 1/(lambda+mu)
    const double* gamma;
    size_t vlen;
    int nrhs;
};

// one cell per thread; accumulates over the nrhs (forward, adjoint) pairs
__global__ void __launch_bounds__(256) k_gradient(GradArgs a, const double2* __restrict__ X, const double2* __restrict__ Y,
                                                  double* g_lambda, double* g_mu, double* g_rho) {
    const int n1 = a.n1, n2 = a.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int i = t % n1, j = t / n1;
    const double z0 = 0.0;
    double gl = 0.0, gm = 0.0, gr_re = 0.0, gr_im = 0.0;
    for (int s = 0; s < a.nrhs; ++s) {
        const double2* x1 = X + (size_t)s * a.vlen;
        const double2* x2 = x1 + np;
        const double2* xp = x1 + 2 * np;
        const double2* y1 = Y + (size_t)s * a.vlen;
        const double2* y2 = y1 + np;
        const double2* yp = y1 + 2 * np;
        auto U1 = [&](const double2* u, int ii, int jj) {
            return (ii >= 1 && ii < n1 && jj >= 0 && jj < n2) ? u[jj * n1 + ii] : make_double2(z0, z0);
        };
        auto U2 = [&](const double2* u, int ii, int jj) {
            return (ii >= 0 && ii < n1 && jj >= 1 && jj < n2) ? u[jj * n1 + ii] : make_double2(z0, z0);
        };
        auto rdot = [](double2 a_, double2 b_) { return a_.x * b_.x + a_.y * b_.y; };   // Re(conj(a) b)
        // C term: lambda and mu
        const double ci = a.cinv[t];
        const double cterm = rdot(yp[t], xp[t]) * ci * ci;
        gl += cterm;
        gm += cterm;
        // own-direction derivatives at the cell: d1 u1 and d2 u2
        {
            const double2 dx = cscale(csub(U1(x1, i + 1, j), U1(x1, i, j)), a.ih1);
            const double2 dy = cscale(csub(U1(y1, i + 1, j), U1(y1, i, j)), a.ih1);
            gm += rdot(dy, dx);
            const double2 ex = cscale(csub(U2(x2, i, j + 1), U2(x2, i, j)), a.ih2);
            const double2 ey = cscale(csub(U2(y2, i, j + 1), U2(y2, i, j)), a.ih2);
            gm += rdot(ey, ex);
        }
        // cross derivatives at the interior nodes around the cell (weight 1/4):
        // d2 u1 and d1 u2 at node (ni, nj)
        for (int q = 0; q < 4; ++q) {
            const int ni = i + (q & 1), nj = j + (q >> 1);
            if (ni < 1 || ni > n1 - 1 || nj < 1 || nj > n2 - 1) continue;
            const double2 ax = cscale(csub(U1(x1, ni, nj), U1(x1, ni, nj - 1)), a.ih2);
            const double2 ay = cscale(csub(U1(y1, ni, nj), U1(y1, ni, nj - 1)), a.ih2);
            const double2 bx = cscale(csub(U2(x2, ni, nj), U2(x2, ni - 1, nj)), a.ih1);
            const double2 by = cscale(csub(U2(y2, ni, nj), U2(y2, ni - 1, nj)), a.ih1);
            gm += 0.25 * (rdot(ay, ax) + rdot(by, bx));
        }
        // faces around the cell: sum conj(y_f) x_f (u1 faces i, i+1; u2 faces j, j+1)
        double sre = 0.0, sim = 0.0;
        auto acc = [&](double2 yv, double2 xv) {
            sre += yv.x * xv.x + yv.y * xv.y;
            sim += yv.x * xv.y - yv.y * xv.x;
        };
        acc(U1(y1, i, j), U1(x1, i, j));
        acc(U1(y1, i + 1, j), U1(x1, i + 1, j));
        acc(U2(y2, i, j), U2(x2, i, j));
        acc(U2(y2, i, j + 1), U2(x2, i, j + 1));
        gr_re += sre;
        gr_im += sim;
    }
    // rho: -Re[ y^H (-omega^2 1/2 (1 - i gamma/omega)) x ] = Re[ omega^2/2 (1 - i gamma/omega) S ]
    const double om2 = a.omega * a.omega;
    const double gk = a.gamma[t] / a.omega;
    const double gr = 0.5 * om2 * (gr_re + gk * gr_im);
    g_lambda[t] += -gl;
    g_mu[t] += -gm;
    g_rho[t] += gr;
}
void launch_gradient(int n1, int n2, double h1, double h2, double omega, const double* cinv, const double* gamma,
                     size_t vlen, int nrhs, const double2* X, const double2* Y, double* gl, double* gm, double* gr,
                     cudaStream_t st) {
    GradArgs a{n1, n2, 1.0 / h1, 1.0 / h2, omega, cinv, gamma, vlen, nrhs};
    const int np = n1 * n2;
    k_gradient<<<(np + 255) / 256, 256, 0, st>>>(a, X, Y, gl, gm, gr);
}

}  // namespace bah
