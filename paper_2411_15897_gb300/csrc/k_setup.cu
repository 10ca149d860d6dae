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

// ---------------------------------------------------------------------------
// Dense FP64 inverse by Gauss-Jordan elimination with partial pivoting on
// [A | X], X = I at entry, in one launch of one thread-block cluster.  The
// matrices stay in global memory (they fit in L2); CTA q of the cluster owns
// the rows r = q (mod CTAs).  Per column k:
//   1. each CTA finds its largest |A[r][k]|, r >= k, among its rows;
//   2. every CTA reads the candidates of all CTAs from distributed shared
//      memory and takes the same winner p (largest, lowest index on ties);
//   3. rows k and p are swapped in A and X (columns split over the CTAs);
//   4. row k is scaled by 1 / A[k][k] (column k itself is never read again);
//   5. every other row r subtracts A[r][k] times row k.
// A hardware cluster barrier separates the steps: the control flow is the
// same in every CTA (the winner, and so a singular pivot, is seen by all), so
// every CTA arrives at every barrier.
// ---------------------------------------------------------------------------
constexpr int kGjThreads = 512;

__device__ __forceinline__ uint32_t gj_mapa(const void* p, unsigned rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ double gj_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int gj_ld_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__global__ void __launch_bounds__(kGjThreads, 1) k_gj_cluster(int n, double2* A, double2* X, int* flag) {
    const unsigned q = cluster_rank(), nq = cluster_nrank();
    const int tid = threadIdx.x, nth = blockDim.x;
    __shared__ double wv[kGjThreads / 32];
    __shared__ int wi[kGjThreads / 32];
    __shared__ double cand_v;          // this CTA's pivot candidate, read by every CTA
    __shared__ int cand_i;
    __shared__ int piv_row;
    __shared__ int singular;
    for (int k = 0; k < n; ++k) {
        // 1. local candidate among own rows r >= k
        double bv = -1.0;
        int bi = n;
        for (int r = (int)q + (int)nq * tid; r < n; r += (int)nq * nth) {
            if (r < k) continue;
            const double2 a = A[(size_t)r * n + k];
            const double m = a.x * a.x + a.y * a.y;
            if (m > bv || (m == bv && r < bi)) { bv = m; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { wv[tid >> 5] = bv; wi[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nth / 32; ++w)
                if (wv[w] > bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
            cand_v = bv;
            cand_i = bi;
        }
        cluster_barrier();
        // 2. the common winner
        if (tid == 0) {
            double best = -1.0;
            int p = n;
            for (unsigned s = 0; s < nq; ++s) {
                const double v = gj_ld_f64(gj_mapa(&cand_v, s));
                const int i = gj_ld_s32(gj_mapa(&cand_i, s));
                if (v > best || (v == best && i < p)) { best = v; p = i; }
            }
            piv_row = p;
            singular = !(best > 0.0) || p >= n;
        }
        __syncthreads();
        if (singular) {
            if (q == 0 && tid == 0) *flag = 1;
            cluster_barrier();              // no CTA exits while another still reads its candidate
            break;                          // taken by every CTA at the same k
        }
        const int p = piv_row;
        // 3. swap rows k and p (columns split over the cluster)
        if (p != k) {
            for (int c = (int)q * nth + tid; c < n; c += (int)nq * nth) {
                double2 t1 = A[(size_t)k * n + c]; A[(size_t)k * n + c] = A[(size_t)p * n + c]; A[(size_t)p * n + c] = t1;
                double2 t2 = X[(size_t)k * n + c]; X[(size_t)k * n + c] = X[(size_t)p * n + c]; X[(size_t)p * n + c] = t2;
            }
        }
        cluster_barrier();
        // 4. scale the pivot row (A[k][k] is left as is: column k is never read again)
        const double2 ip = cdiv(make_double2(1.0, 0.0), A[(size_t)k * n + k]);
        for (int c = (int)q * nth + tid; c < n; c += (int)nq * nth) {
            if (c > k) A[(size_t)k * n + c] = cmul(A[(size_t)k * n + c], ip);
            X[(size_t)k * n + c] = cmul(X[(size_t)k * n + c], ip);
        }
        cluster_barrier();
        // 5. eliminate column k from every other own row: columns c > k of A, all of X
        const int nown = (n - (int)q + (int)nq - 1) / (int)nq;
        const int w2 = 2 * n;
        for (int e = tid; e < nown * w2; e += nth) {
            const int r = (int)q + (int)nq * (e / w2), c = e % w2;
            if (r == k) continue;
            const double2 f = A[(size_t)r * n + k];
            if (c < n) {
                if (c > k) A[(size_t)r * n + c] = csub(A[(size_t)r * n + c], cmul(f, A[(size_t)k * n + c]));
            } else {
                const int cx = c - n;
                X[(size_t)r * n + cx] = csub(X[(size_t)r * n + cx], cmul(f, X[(size_t)k * n + cx]));
            }
        }
        cluster_barrier();
    }
}

int coarse_invert(int type, const StencilF64& S, double2* inv, double2* work, int* flag, cudaStream_t st) {
    const int n = S.n1 * S.n2;
    double2* A = work;                       // n*n
    double2* f = work + (size_t)n * n;       // n
    dim3 g((n + 127) / 128, n);
    k_dense_assemble<<<g, 128, 0, st>>>(type, S.S, S.rx, S.rz, S.n1, S.n2, A, inv);
    return gauss_jordan(n, A, inv, f, flag, st);
}

// CTAs per cluster for the Gauss-Jordan kernel: 16 where the device allows
// non-portable clusters, else 8
static int gj_cluster_size() {
    static int cs = 0;
    if (cs) return cs;
    cs = 8;
    if (cudaFuncSetAttribute((const void*)k_gj_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kGjThreads);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, (const void*)k_gj_cluster, &cfg) == cudaSuccess && nc >= 1) cs = 16;
    }
    cudaGetLastError();
    return cs;
}

int gauss_jordan(int n, double2* A, double2* X, double2* /*f*/, int* flag, cudaStream_t st) {
    BAH_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    const int cs = gj_cluster_size();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kGjThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BAH_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster, n, A, X, flag));
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
