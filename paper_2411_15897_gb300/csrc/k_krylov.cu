// FP64 kernels of the flexible GMRES outer iteration: block dot products and
// norms (warp-shuffle + shared-memory reductions in two deterministic stages),
// the Gram-Schmidt updates, the Givens update of the Hessenberg least-squares
// problem, the triangular solve and the solution update x += Z y.
#include "bah_internal.cuh"

namespace bah {

__device__ __forceinline__ double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of a double2 (blockDim.x = 256); result valid in thread 0
__device__ __forceinline__ double2 block_sum2(double2 v) {
    __shared__ double2 sh[8];
    v = warp_sum2(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : make_double2(0.0, 0.0);
        r = warp_sum2(r);
    }
    __syncthreads();
    return r;
}

// stage 1: partial[y * RED_CTAS + x] = sum over the CTA's chunk of conj(V_y) w
__global__ void __launch_bounds__(256) k_multi_dot_partial(const double2* __restrict__ V, size_t ldv,
                                                           const double2* __restrict__ w, size_t n,
                                                           double2* __restrict__ partial) {
    const double2* v = V + (size_t)blockIdx.y * ldv;
    double2 acc = make_double2(0.0, 0.0);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = v[e], b = w[e];
        acc.x += a.x * b.x + a.y * b.y;
        acc.y += a.x * b.y - a.y * b.x;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// stage 2: out[y] = sum of the RED_CTAS partials of row y (fixed order)
__global__ void __launch_bounds__(256) k_reduce_partials2(const double2* __restrict__ partial, int np,
                                                          double2* __restrict__ out) {
    double2 acc = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const double2 a = partial[(size_t)blockIdx.y * np + e];
        acc.x += a.x;
        acc.y += a.y;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) out[blockIdx.y] = acc;
}

// ---------------------------------------------------------------------------
// Gram-Schmidt with selective reorthogonalisation (Daniel-Gragg-Kaufman-Stewart
// criterion): pass 1 forms h1 = V^H w together with ||w||^2 and then
// w' = w - V h1 together with ||w'||^2; a second pass runs only if
// ||w'|| < ||w|| / sqrt(2).  The pass-2 kernels read the device flag and
// return at once when it is clear.
// ---------------------------------------------------------------------------
// rows 0..k-1: conj(V_y) w; row k: |w|^2 (imaginary part 0)
__global__ void __launch_bounds__(256) k_dot_norm_partial(const double2* __restrict__ V, size_t ldv, int k,
                                                          const double2* __restrict__ w, size_t n,
                                                          double2* __restrict__ partial, const int* flag) {
    if (flag && *flag == 0) return;
    const int y = blockIdx.y;
    double2 acc = make_double2(0.0, 0.0);
    if (y < k) {
        const double2* v = V + (size_t)y * ldv;
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
            const double2 a = v[e], b = w[e];
            acc.x += a.x * b.x + a.y * b.y;
            acc.y += a.x * b.y - a.y * b.x;
        }
    } else {
        for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
            const double2 b = w[e];
            acc.x += b.x * b.x + b.y * b.y;
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) partial[(size_t)y * gridDim.x + blockIdx.x] = acc;
}
__global__ void __launch_bounds__(256) k_reduce_rows(const double2* __restrict__ partial, int np, double2* out,
                                                     const int* flag) {
    if (flag && *flag == 0) {
        if (threadIdx.x == 0) out[blockIdx.y] = make_double2(0.0, 0.0);
        return;
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const double2 a = partial[(size_t)blockIdx.y * np + e];
        acc.x += a.x;
        acc.y += a.y;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) out[blockIdx.y] = acc;
}
void launch_dot_norm(const double2* V, size_t ldv, int k, const double2* w, size_t n, double2* partial, double2* out,
                     const int* flag, cudaStream_t st) {
    k_dot_norm_partial<<<dim3(RED_CTAS, k + 1), 256, 0, st>>>(V, ldv, k, w, n, partial, flag);
    k_reduce_rows<<<dim3(1, k + 1), 256, 0, st>>>(partial, RED_CTAS, out, flag);
}

// w -= sum_i coef[i] V_i, and per-CTA partial sums of |w_new|^2
__global__ void __launch_bounds__(256) k_axpy_norm(const double2* __restrict__ V, size_t ldv, int k,
                                                   const double2* __restrict__ coef, double2* __restrict__ w, size_t n,
                                                   double* __restrict__ npart, const int* flag) {
    if (flag && *flag == 0) return;
    __shared__ double2 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = coef[threadIdx.x];
    __syncthreads();
    double nn = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc = w[e];
        for (int i = 0; i < k; ++i) {
            const double2 v = V[(size_t)i * ldv + e];
            acc.x -= c[i].x * v.x - c[i].y * v.y;
            acc.y -= c[i].x * v.y + c[i].y * v.x;
        }
        w[e] = acc;
        nn += acc.x * acc.x + acc.y * acc.y;
    }
    double2 r = block_sum2(make_double2(nn, 0.0));
    if (threadIdx.x == 0) npart[blockIdx.x] = r.x;
}
void launch_axpy_norm(const double2* V, size_t ldv, int k, const double2* coef, double2* w, size_t n, double* npart,
                      const int* flag, cudaStream_t st) {
    k_axpy_norm<<<RED_CTAS, 256, 0, st>>>(V, ldv, k, coef, w, n, npart, flag);
}

// reduce the pass-1 norm, decide on the second pass, set ||w|| for the Givens step
// wn[0] = ||w_final||; flag = 1 when ||w'||^2 < ||w||^2 / 2
__global__ void __launch_bounds__(256) k_dgks_decide(const double* npart, int np, const double2* h1norm, int k,
                                                     int* flag, double* wn) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += npart[e];
    double2 r = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) {
        const double w0 = h1norm[k].x;          // ||w||^2 before pass 1
        const int f = (r.x < 0.5 * w0) ? 1 : 0;
        *flag = f;
        wn[0] = sqrt(r.x);
        wn[1] += (double)f;                      // count of second passes (diagnostic)
    }
}
void launch_dgks_decide(const double* npart, const double2* h1norm, int k, int* flag, double* wn, cudaStream_t st) {
    k_dgks_decide<<<1, 256, 0, st>>>(npart, RED_CTAS, h1norm, k, flag, wn);
}
// after pass 2: ||w''|| replaces ||w'||
__global__ void __launch_bounds__(256) k_pass2_norm(const double* npart, int np, const int* flag, double* wn) {
    if (*flag == 0) return;
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += npart[e];
    double2 r = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) wn[0] = sqrt(r.x);
}
void launch_pass2_norm(const double* npart, const int* flag, double* wn, cudaStream_t st) {
    k_pass2_norm<<<1, 256, 0, st>>>(npart, RED_CTAS, flag, wn);
}

void launch_multi_dot(const double2* V, size_t ldv, int k, const double2* w, size_t n, double2* partial, double2* out,
                      cudaStream_t st) {
    k_multi_dot_partial<<<dim3(RED_CTAS, k), 256, 0, st>>>(V, ldv, w, n, partial);
    k_reduce_partials2<<<dim3(1, k), 256, 0, st>>>(partial, RED_CTAS, out);
}

__global__ void __launch_bounds__(256) k_norm2_partial(const double2* __restrict__ w, size_t n, double* partial) {
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 b = w[e];
        acc += b.x * b.x + b.y * b.y;
    }
    double2 r = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) partial[blockIdx.x] = r.x;
}
__global__ void __launch_bounds__(256) k_norm2_final(const double* partial, int np, double* out) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += partial[e];
    double2 r = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) *out = sqrt(r.x);
}
void launch_norm2(const double2* w, size_t n, double* partial, double* out, cudaStream_t st) {
    k_norm2_partial<<<RED_CTAS, 256, 0, st>>>(w, n, partial);
    k_norm2_final<<<1, 256, 0, st>>>(partial, RED_CTAS, out);
}

// w -= sum_i coef[i] V_i
__global__ void __launch_bounds__(256) k_multi_axpy_sub(const double2* __restrict__ V, size_t ldv, int k,
                                                        const double2* __restrict__ coef, double2* __restrict__ w,
                                                        size_t n) {
    __shared__ double2 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = coef[threadIdx.x];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc = w[e];
        for (int i = 0; i < k; ++i) {
            const double2 v = V[(size_t)i * ldv + e];
            acc.x -= c[i].x * v.x - c[i].y * v.y;
            acc.y -= c[i].x * v.y + c[i].y * v.x;
        }
        w[e] = acc;
    }
}
void launch_multi_axpy_sub(const double2* V, size_t ldv, int k, const double2* coef, double2* w, size_t n,
                           cudaStream_t st) {
    k_multi_axpy_sub<<<RED_CTAS * 4, 256, 0, st>>>(V, ldv, k, coef, w, n);
}

// x += sum_i y_i Z_i  (Z in the preconditioner's precision, x in FP64)
template <class Vz>
__global__ void __launch_bounds__(256) k_update_x(const Vz* __restrict__ Z, size_t ldz, int k,
                                                  const double2* __restrict__ y, double2* __restrict__ x, size_t n) {
    __shared__ double2 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc = x[e];
        for (int i = 0; i < k; ++i) {
            const Vz zv = Z[(size_t)i * ldz + e];
            const double zx = (double)zv.x, zy = (double)zv.y;
            acc.x += c[i].x * zx - c[i].y * zy;
            acc.y += c[i].x * zy + c[i].y * zx;
        }
        x[e] = acc;
    }
}
template <class Vz>
void launch_update_x(const Vz* Z, size_t ldz, int k, const double2* y, double2* x, size_t n, cudaStream_t st) {
    k_update_x<Vz><<<RED_CTAS * 4, 256, 0, st>>>(Z, ldz, k, y, x, n);
}
template void launch_update_x<double2>(const double2*, size_t, int, const double2*, double2*, size_t, cudaStream_t);
template void launch_update_x<float2>(const float2*, size_t, int, const double2*, double2*, size_t, cudaStream_t);

// v = w / nrm  (inverse = 1)  or  v = w * nrm (inverse = 0)
__global__ void k_scale_copy(const double2* __restrict__ w, const double* nrm, double2* __restrict__ v, size_t n,
                             int inverse) {
    const double s = inverse ? 1.0 / *nrm : *nrm;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = w[e];
        v[e] = make_double2(a.x * s, a.y * s);
    }
}
void launch_scale_copy(const double2* w, const double* nrm, double2* v, size_t n, int inverse, cudaStream_t st) {
    k_scale_copy<<<RED_CTAS * 4, 256, 0, st>>>(w, nrm, v, n, inverse);
}

// ---------------------------------------------------------------------------
// Hessenberg column j = h1 + h2 (two Gram-Schmidt passes) with subdiagonal
// ||w||; apply the previous Givens rotations, form the new one, update g.
// Rotation [c s; -conj(s) c] with c real.  status[0] = |g_{j+1}|,
// status[1] = h_{j+1,j}, status[2] = 1 if a non-finite value appeared.
// ---------------------------------------------------------------------------
__global__ void k_arnoldi_givens(double2* Hcol, const double2* h1, const double2* h2, const double* wnorm, int j,
                                 double2* cs, double2* sn, double2* g, double* status) {
    __shared__ double2 h[66];
    __shared__ double2 ssn[65];
    __shared__ double scs[65];
    // the warp stages the column and the previous rotations
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        h[i] = h2 ? cadd(h1[i], h2[i]) : h1[i];
        if (i < j) { scs[i] = cs[i].x; ssn[i] = sn[i]; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double wn = *wnorm;
    h[j + 1] = make_double2(wn, 0.0);
    bool bad = !isfinite(wn);
    for (int i = 0; i <= j; ++i) bad |= !isfinite(h[i].x) || !isfinite(h[i].y);
    for (int i = 0; i < j; ++i) {
        const double c = scs[i];
        const double2 s = ssn[i];
        const double2 a = h[i], b = h[i + 1];
        h[i] = cadd(cscale(a, c), cmul(s, b));
        h[i + 1] = csub(cscale(b, c), cmul(cconj(s), a));
    }
    const double2 a = h[j], b = h[j + 1];
    const double na2 = a.x * a.x + a.y * a.y, nb2 = b.x * b.x + b.y * b.y;
    double c;
    double2 s;
    if (nb2 == 0.0) {
        c = 1.0; s = make_double2(0.0, 0.0);
    } else if (na2 == 0.0) {
        c = 0.0; s = cscale(cconj(b), 1.0 / sqrt(nb2));
    } else {
        const double na = sqrt(na2), r = sqrt(na2 + nb2);
        c = na / r;
        s = cscale(cmul(a, cconj(b)), 1.0 / (na * r));
    }
    cs[j] = make_double2(c, 0.0);
    sn[j] = s;
    h[j] = cadd(cscale(a, c), cmul(s, b));
    h[j + 1] = make_double2(0.0, 0.0);
    for (int i = 0; i <= j + 1; ++i) Hcol[i] = h[i];
    const double2 gj = g[j];
    g[j] = cscale(gj, c);
    const double2 gn = cscale(cmul(cconj(s), gj), -1.0);
    g[j + 1] = gn;
    status[0] = sqrt(gn.x * gn.x + gn.y * gn.y);
    status[1] = wn;
    status[2] = bad ? 1.0 : 0.0;
}
void launch_arnoldi_givens(double2* Hcol, const double2* h1, const double2* h2, const double* wnorm, int j,
                           double2* cs, double2* sn, double2* g, double* status, cudaStream_t st) {
    k_arnoldi_givens<<<1, 32, 0, st>>>(Hcol, h1, h2, wnorm, j, cs, sn, g, status);
}

// R y = g(0..k-1), R upper triangular stored column-major with leading dimension ldh
__global__ void k_triangular_solve(const double2* Hm, int ldh, const double2* g, int k, double2* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int c = i + 1; c < k; ++c) acc = csub(acc, cmul(Hm[(size_t)c * ldh + i], y[c]));
        y[i] = cdiv(acc, Hm[(size_t)i * ldh + i]);
    }
}
void launch_triangular_solve(const double2* Hm, int ldh, const double2* g, int k, double2* y, cudaStream_t st) {
    k_triangular_solve<<<1, 32, 0, st>>>(Hm, ldh, g, k, y);
}

__global__ void k_init_arnoldi(const double* beta, double2* g, int m, double* status) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = make_double2(i == 0 ? *beta : 0.0, 0.0);
    if (threadIdx.x == 0) { status[0] = *beta; status[1] = 0.0; status[2] = 0.0; }
}
void launch_init_arnoldi(const double* beta, double2* g, int m, double* status, cudaStream_t st) {
    k_init_arnoldi<<<1, 128, 0, st>>>(beta, g, m, status);
}

}  // namespace bah
