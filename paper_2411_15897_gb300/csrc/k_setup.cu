// Setup kernels: operator coefficients (Eq. 2.6, 3.2, 3.4 with the shift of
// Eq. 2.8), Galerkin coarse operators R A P (Eq. 4.3) with the intergrid
// stencils of Eq. 4.1, 4.2, 4.4, and the FP64 inverse of the coarsest level
// (the direct coarse solve of Sec. 4.4.1).  All FP64; run once per context.
#include "bah_internal.cuh"
#include "intergrid.cuh"

#include <cmath>

namespace bah {

// ---------------------------------------------------------------------------
// medium preparation
// ---------------------------------------------------------------------------
__device__ __forceinline__ double node_mu(const double* mu, int n1, int n2, int i, int j) {
    // arithmetic mean of the four cells around node (i, j); zero on boundary nodes
    if (i < 1 || j < 1 || i > n1 - 1 || j > n2 - 1) return 0.0;
    return 0.25 * (mu[(j - 1) * n1 + i - 1] + mu[(j - 1) * n1 + i] + mu[j * n1 + i - 1] + mu[j * n1 + i]);
}

__global__ void k_medium_prep(int n1, int n2, double ih1, double ih2, double omega, double alpha,
                              const double* __restrict__ lam, const double* __restrict__ mu,
                              const double* __restrict__ rho, const double* __restrict__ gam,
                              double* cx, double* cz, double* nx, double* nz, double* wx, double* wz,
                              double2* d1, double2* d2, double* cinv,
                              double2* dg0, double2* dg1, double2* dg2, double2* dAp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n1 * n2) return;
    const int i = t % n1, j = t / n1;
    const double ih1s = ih1 * ih1, ih2s = ih2 * ih2, om2 = omega * omega;
    const double muc = mu[t];
    const double lm = lam[t] + muc;
    cx[t] = muc * ih1s;
    cz[t] = muc * ih2s;
    const double mn = node_mu(mu, n1, n2, i, j);
    nx[t] = mn * ih1s;
    nz[t] = mn * ih2s;
    const double w = (lam[t] + 2.0 * muc) / lm;
    wx[t] = w * ih1s;
    wz[t] = w * ih2s;
    cinv[t] = 1.0 / lm;
    auto rt = [&](int c) { return make_double2(rho[c], -rho[c] * gam[c] / omega); };   // rho (1 - i gamma/omega)

    // u1 on the x_1-face below cell (i, j): A_1 diagonal (Eq. 2.6) and its shift (Eq. 2.8)
    if (i >= 1) {
        const int w_ = t - 1;
        double2 m = make_double2(0.5 * (rt(w_).x + rt(t).x), 0.5 * (rt(w_).y + rt(t).y));
        double ms = 0.5 * (rho[w_] + rho[t]);
        double lap = (mu[w_] + muc) * ih1s + (node_mu(mu, n1, n2, i, j) + node_mu(mu, n1, n2, i, j + 1)) * ih2s;
        d1[t] = make_double2(lap - om2 * m.x, -om2 * m.y);
        dg0[t] = make_double2(lap - om2 * m.x, -om2 * m.y + alpha * om2 * ms);
    } else {
        d1[t] = make_double2(0.0, 0.0);
        dg0[t] = make_double2(0.0, 0.0);
    }
    // u2 on the x_2-face below cell (i, j)
    if (j >= 1) {
        const int s_ = t - n1;
        double2 m = make_double2(0.5 * (rt(s_).x + rt(t).x), 0.5 * (rt(s_).y + rt(t).y));
        double ms = 0.5 * (rho[s_] + rho[t]);
        double lap = (mu[s_] + muc) * ih2s + (node_mu(mu, n1, n2, i, j) + node_mu(mu, n1, n2, i + 1, j)) * ih1s;
        d2[t] = make_double2(lap - om2 * m.x, -om2 * m.y);
        dg1[t] = make_double2(lap - om2 * m.x, -om2 * m.y + alpha * om2 * ms);
    } else {
        d2[t] = make_double2(0.0, 0.0);
        dg1[t] = make_double2(0.0, 0.0);
    }
    // p: number of existing neighbours per axis (zero-flux boundary, Eq. 3.2 / 3.4)
    const double nbx = (i >= 1 ? 1.0 : 0.0) + (i + 1 < n1 ? 1.0 : 0.0);
    const double nbz = (j >= 1 ? 1.0 : 0.0) + (j + 1 < n2 ? 1.0 : 0.0);
    const double2 r = rt(t);
    // A_p = B B^T diag(mu) - omega^2 diag(rho~)
    dAp[t] = make_double2(nbx * cx[t] + nbz * cz[t] - om2 * r.x, -om2 * r.y);
    // H_p = B B^T diag(w) - omega^2 diag(rho~/(lambda+mu)), shifted by + i alpha omega^2 rho/(lambda+mu)
    dg2[t] = make_double2(nbx * wx[t] + nbz * wz[t] - om2 * r.x / lm, -om2 * r.y / lm + alpha * om2 * rho[t] / lm);
}

void launch_medium_prep(int n1, int n2, double h1, double h2, double omega, double alpha,
                        const double* lam, const double* mu, const double* rho, const double* gam,
                        double* cx, double* cz, double* nx, double* nz, double* wx, double* wz,
                        double2* d1, double2* d2, double* cinv,
                        double2* dg0, double2* dg1, double2* dg2, double2* dAp, cudaStream_t st) {
    int n = n1 * n2;
    k_medium_prep<<<(n + 255) / 256, 256, 0, st>>>(n1, n2, 1.0 / h1, 1.0 / h2, omega, alpha, lam, mu, rho, gam,
                                                   cx, cz, nx, nz, wx, wz, d1, d2, cinv, dg0, dg1, dg2, dAp);
}

// ---------------------------------------------------------------------------
// level-0 shifted block as an explicit 3x3 stencil (slot (dz+1)*3 + (dx+1))
// ---------------------------------------------------------------------------
__global__ void k_fine_stencil(int type, int n1, int n2, const double* cx, const double* cz, const double* nx,
                               const double* nz, const double* wx, const double* wz, const double2* dg,
                               double2* S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = n1 * n2;
    if (t >= np) return;
    const int i = t % n1, j = t / n1;
    double c[9];
    for (int s = 0; s < 9; ++s) c[s] = 0.0;
    double2 ctr = make_double2(0.0, 0.0);
    if (valid_pt(type, i, j)) {
        ctr = dg[t];
        if (type == 0) {            // u1: own-direction x (cells i-1, i), tangential z (nodes (i,j), (i,j+1))
            if (i - 1 >= 1) c[3] = -cx[t - 1];
            if (i + 1 <= n1 - 1) c[5] = -cx[t];
            if (j - 1 >= 0) c[1] = -nz[t];
            if (j + 1 <= n2 - 1) c[7] = -nz[t + n1];
        } else if (type == 1) {     // u2: own-direction z, tangential x
            if (j - 1 >= 1) c[1] = -cz[t - n1];
            if (j + 1 <= n2 - 1) c[7] = -cz[t];
            if (i - 1 >= 0) c[3] = -nx[t];
            if (i + 1 <= n1 - 1) c[5] = -nx[t + 1];
        } else {                    // p: H_p weights the Laplacian from the right
            if (i >= 1) c[3] = -wx[t - 1];
            if (i + 1 < n1) c[5] = -wx[t + 1];
            if (j >= 1) c[1] = -wz[t - n1];
            if (j + 1 < n2) c[7] = -wz[t + n1];
        }
    }
    for (int s = 0; s < 9; ++s) S[(size_t)s * np + t] = (s == 4) ? ctr : make_double2(c[s], 0.0);
}

void launch_fine_stencil(int type, int n1, int n2, const double* cx, const double* cz, const double* nx,
                         const double* nz, const double* wx, const double* wz, const double2* dg, double2* S,
                         cudaStream_t st) {
    int n = n1 * n2;
    k_fine_stencil<<<(n + 255) / 256, 256, 0, st>>>(type, n1, n2, cx, cz, nx, nz, wx, wz, dg, S);
}

// ---------------------------------------------------------------------------
// Galerkin coarse operator A_c = R A P (Eq. 4.3), one coarse point per thread
// ---------------------------------------------------------------------------
__global__ void k_galerkin(int type, int intergrid, const double2* __restrict__ Sf, int rxf, int rzf, int n1, int n2,
                           double2* Sc, int rxc, int rzc) {
    const int n1c = n1 / 2, n2c = n2 / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int npc = n1c * n2c, npf = n1 * n2;
    if (t >= npc) return;
    const int I = t % n1c, J = t / n1c;
    const int wxc = 2 * rxc + 1, nsc = wxc * (2 * rzc + 1);
    const int wxf = 2 * rxf + 1;
    double2 acc[25];
    for (int s = 0; s < nsc; ++s) acc[s] = make_double2(0.0, 0.0);
    const bool nodx = (type == 0), nodz = (type == 1);
    if (valid_pt(type, I, J)) {
        for (int fj = 2 * J - 2; fj <= 2 * J + 3; ++fj) {
            const double rz = rw_axis(nodz, intergrid, n2, J, fj);
            if (rz == 0.0) continue;
            for (int fi = 2 * I - 2; fi <= 2 * I + 3; ++fi) {
                const double rx = rw_axis(nodx, intergrid, n1, I, fi);
                if (rx == 0.0) continue;
                const double r = rx * rz;
                const int f = fj * n1 + fi;
                for (int dz = -rzf; dz <= rzf; ++dz) {
                    const int gj = fj + dz;
                    if (gj < 0 || gj >= n2) continue;
                    for (int dx = -rxf; dx <= rxf; ++dx) {
                        const int gi = fi + dx;
                        if (gi < 0 || gi >= n1) continue;
                        const double2 a = Sf[(size_t)((dz + rzf) * wxf + (dx + rxf)) * npf + f];
                        if (a.x == 0.0 && a.y == 0.0) continue;
                        // coarse points whose interpolation reaches g = (gi, gj)
                        for (int cj = (gj >> 1) - 1; cj <= (gj >> 1) + 1; ++cj) {
                            const double pz = pw_axis(nodz, n2, gj, cj);
                            if (pz == 0.0) continue;
                            for (int ci = (gi >> 1) - 1; ci <= (gi >> 1) + 1; ++ci) {
                                const double px = pw_axis(nodx, n1, gi, ci);
                                if (px == 0.0) continue;
                                const int ox = ci - I, oz = cj - J;
                                if (ox < -rxc || ox > rxc || oz < -rzc || oz > rzc) continue;   // cannot happen
                                const double wgt = r * px * pz;
                                double2& o = acc[(oz + rzc) * wxc + (ox + rxc)];
                                o.x += wgt * a.x;
                                o.y += wgt * a.y;
                            }
                        }
                    }
                }
            }
        }
    }
    for (int s = 0; s < nsc; ++s) Sc[(size_t)s * npc + t] = acc[s];
}

void launch_galerkin(int type, int intergrid, const StencilF64& fine, StencilF64& coarse, cudaStream_t st) {
    int npc = (fine.n1 / 2) * (fine.n2 / 2);
    k_galerkin<<<(npc + 127) / 128, 128, 0, st>>>(type, intergrid, fine.S, fine.rx, fine.rz, fine.n1, fine.n2,
                                                  coarse.S, coarse.rx, coarse.rz);
}

// ---------------------------------------------------------------------------
// storage rounding: FP64 -> bfloat16 (round to nearest even) or FP64 copy
// ---------------------------------------------------------------------------
__global__ void k_round_real(const double* src, void* dst, size_t n, int mode) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (mode == BAH_MIXED) ((__nv_bfloat16*)dst)[t] = __double2bfloat16(src[t]);
    else ((double*)dst)[t] = src[t];
}
__global__ void k_round_cplx(const double2* src, void* dst, size_t n, int mode) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (mode == BAH_MIXED) {
        __nv_bfloat162 v;
        v.x = __double2bfloat16(src[t].x);
        v.y = __double2bfloat16(src[t].y);
        ((__nv_bfloat162*)dst)[t] = v;
    } else {
        ((double2*)dst)[t] = src[t];
    }
}
void launch_round_real(const double* src, void* dst, size_t n, int mode, cudaStream_t st) {
    k_round_real<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n, mode);
}
void launch_round_cplx(const double2* src, void* dst, size_t n, int mode, cudaStream_t st) {
    k_round_cplx<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n, mode);
}

// ---------------------------------------------------------------------------
// coarsest level: dense FP64 inverse by Gauss-Jordan elimination with
// partial pivoting.  Rows of non-unknown (boundary-normal) points are
// identity rows, so the inverse maps their zero entries to zero.
// ---------------------------------------------------------------------------
__global__ void k_dense_assemble(int type, const double2* S, int rx, int rz, int n1, int n2, double2* A, double2* X) {
    const int np = n1 * n2;
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= np || r >= np) return;
    const int i = r % n1, j = r / n1;
    double2 v = make_double2(0.0, 0.0);
    if (valid_pt(type, i, j)) {
        const int ci = c % n1, cj = c / n1;
        const int ox = ci - i, oz = cj - j;
        if (ox >= -rx && ox <= rx && oz >= -rz && oz <= rz)
            v = S[(size_t)((oz + rz) * (2 * rx + 1) + (ox + rx)) * np + r];
    } else if (c == r) {
        v = make_double2(1.0, 0.0);
    }
    A[(size_t)r * np + c] = v;
    X[(size_t)r * np + c] = make_double2(c == r ? 1.0 : 0.0, 0.0);
}

__global__ void k_gj_pivot(int n, int k, double2* A, double2* X, double2* f, int* flag) {
    __shared__ double bestv[256];
    __shared__ int besti[256];
    double bv = -1.0;
    int bi = k;
    for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
        double2 a = A[(size_t)r * n + k];
        double m = a.x * a.x + a.y * a.y;
        if (m > bv) { bv = m; bi = r; }
    }
    bestv[threadIdx.x] = bv;
    besti[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            if (bestv[threadIdx.x + s] > bestv[threadIdx.x] ||
                (bestv[threadIdx.x + s] == bestv[threadIdx.x] && besti[threadIdx.x + s] < besti[threadIdx.x])) {
                bestv[threadIdx.x] = bestv[threadIdx.x + s];
                besti[threadIdx.x] = besti[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    const int p = besti[0];
    if (bestv[0] <= 0.0) {
        if (threadIdx.x == 0) *flag = 1;
        return;
    }
    if (p != k) {
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double2 t1 = A[(size_t)k * n + c]; A[(size_t)k * n + c] = A[(size_t)p * n + c]; A[(size_t)p * n + c] = t1;
            double2 t2 = X[(size_t)k * n + c]; X[(size_t)k * n + c] = X[(size_t)p * n + c]; X[(size_t)p * n + c] = t2;
        }
    }
    __syncthreads();
    const double2 piv = A[(size_t)k * n + k];
    const double2 ip = cdiv(make_double2(1.0, 0.0), piv);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        A[(size_t)k * n + c] = cmul(A[(size_t)k * n + c], ip);
        X[(size_t)k * n + c] = cmul(X[(size_t)k * n + c], ip);
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) f[r] = (r == k) ? make_double2(0.0, 0.0) : A[(size_t)r * n + k];
}

__global__ void k_gj_eliminate(int n, int k, double2* A, double2* X, const double2* f) {
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == k || c >= n) return;
    const double2 fr = f[r];
    if (fr.x == 0.0 && fr.y == 0.0) return;
    if (c >= k) {
        double2 a = A[(size_t)r * n + c];
        A[(size_t)r * n + c] = csub(a, cmul(fr, A[(size_t)k * n + c]));
    }
    double2 x = X[(size_t)r * n + c];
    X[(size_t)r * n + c] = csub(x, cmul(fr, X[(size_t)k * n + c]));
}

int coarse_invert(int type, const StencilF64& S, double2* inv, double2* work, int* flag, cudaStream_t st) {
    const int n = S.n1 * S.n2;
    double2* A = work;                       // n*n
    double2* f = work + (size_t)n * n;       // n
    dim3 g((n + 127) / 128, n);
    k_dense_assemble<<<g, 128, 0, st>>>(type, S.S, S.rx, S.rz, S.n1, S.n2, A, inv);
    return gauss_jordan(n, A, inv, f, flag, st);
}

int gauss_jordan(int n, double2* A, double2* X, double2* f, int* flag, cudaStream_t st) {
    dim3 g((n + 127) / 128, n);
    BAH_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    for (int k = 0; k < n; ++k) {
        k_gj_pivot<<<1, 256, 0, st>>>(n, k, A, X, f, flag);
        k_gj_eliminate<<<g, 128, 0, st>>>(n, k, A, X, f);
    }
    BAH_CUDA_TRY(cudaGetLastError());
    int h = 0;
    BAH_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        set_error("coarsest-level operator is singular to working precision");
        return BAH_ERR_ARG;
    }
    return BAH_OK;
}

}  // namespace bah
