// FP64 kernels of the flexible GMRES outer iteration, batched over
// right-hand sides (blockIdx.z or .y = right-hand side, strides in KS):
// block dot products and norms (warp-shuffle + shared-memory reductions in two
// deterministic stages), the Gram-Schmidt updates with selective
// reorthogonalisation, the Givens update of the Hessenberg least-squares
// problem, the triangular solve and the solution update x += Z y.
// A right-hand side whose active flag is 0 is skipped by every kernel.
#include "bah_internal.cuh"
#include "df.cuh"

namespace bah {

__device__ __forceinline__ double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// block-wide sum of a double2 (blockDim.x a multiple of 32, at most 1024); result valid in thread 0
__device__ __forceinline__ double2 block_sum2(double2 v) {
    __shared__ double2 sh[32];   // one per warp, up to 1024 threads
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

__device__ __forceinline__ bool inactive(const KS& ks, int r) { return ks.active && !ks.active[r]; }

// ---------------------------------------------------------------------------
// Gram-Schmidt with selective reorthogonalisation (Daniel-Gragg-Kaufman-Stewart
// criterion): pass 1 forms h1 = V^H w together with ||w||^2 and then
// w' = w - V h1 together with ||w'||^2; a second pass runs only if
// ||w'|| < ||w|| / sqrt(2).  The pass-2 kernels read the per-right-hand-side
// flag and return at once when it is clear.
// ---------------------------------------------------------------------------
// The FP64 pipe (2 FMA/clk/SM on GB300, 1/64 of FP32) bounds these kernels,
// so every complex multiply-add is written as four explicit fused
// multiply-adds into the accumulator (a plain "acc += a*b + c*d" compiles to a
// multiply, an FMA and an add: six FP64 instructions per complex MAC).
__device__ __forceinline__ void cmac_conj(double2& acc, const double2& a, const double2& b) {   // acc += conj(a) b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmsub(double2& acc, const double2& c, const double2& v) {       // acc -= c v
    acc.x = fma(-c.x, v.x, acc.x);
    acc.x = fma(c.y, v.y, acc.x);
    acc.y = fma(-c.x, v.y, acc.y);
    acc.y = fma(-c.y, v.x, acc.y);
}

// Partial sums of rows y0 .. y0+kG-1 (blockIdx.y = row group): row y < k is
// conj(V_y) w, row k is |w|^2 (imaginary part 0).  Each thread loads w once per
// element for the kG rows of its group.  The kG complex partials of the CTA are
// reduced through shared memory: thread t sums quantity t / 16 over a slice of
// 16 threads, then 16-lane shuffles finish it (few FP64 adds per thread).
constexpr int kDotG = 8;
__global__ void __launch_bounds__(256) k_dot_norm_partial(const double2* __restrict__ V, int k,
                                                          const double2* __restrict__ w, size_t n,
                                                          double2* __restrict__ partial, const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive(ks, r) || (flag && flag[r] == 0)) return;
    V += r * ks.sv;
    w += r * ks.sw;
    partial += r * ks.sp;
    const int y0 = blockIdx.y * kDotG;
    const int ny = min(kDotG, k + 1 - y0);          // rows of this group (the norm row is row k)
    double2 acc[kDotG];
#pragma unroll
    for (int q = 0; q < kDotG; ++q) acc[q] = make_double2(0.0, 0.0);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride) {
        const double2 b = __ldg(w + e);
        double2 a[kDotG];
#pragma unroll
        for (int q = 0; q < kDotG; ++q)
            if (q < ny && y0 + q < k) a[q] = __ldg(V + (size_t)(y0 + q) * n + e);
#pragma unroll
        for (int q = 0; q < kDotG; ++q) {
            if (q >= ny) break;
            if (y0 + q < k) {
                cmac_conj(acc[q], a[q], b);
            } else {
                acc[q].x = fma(b.x, b.x, acc[q].x);
                acc[q].x = fma(b.y, b.y, acc[q].x);
            }
        }
    }
    __shared__ double sh[2 * kDotG][256];
#pragma unroll
    for (int q = 0; q < kDotG; ++q) {
        sh[2 * q][threadIdx.x] = acc[q].x;
        sh[2 * q + 1][threadIdx.x] = acc[q].y;
    }
    __syncthreads();
    const int qv = threadIdx.x >> 4, sl = threadIdx.x & 15;     // quantity, slice
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 16; ++u) s += sh[qv][sl * 16 + u];
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (sl == 0 && (qv >> 1) < ny) {
        double* dst = reinterpret_cast<double*>(partial + (size_t)(y0 + (qv >> 1)) * gridDim.x + blockIdx.x);
        dst[qv & 1] = s;
    }
}
__global__ void __launch_bounds__(256) k_reduce_rows(const double2* __restrict__ partial, int np, double2* out,
                                                     const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive(ks, r)) return;
    partial += r * ks.sp;
    out += r * ks.so;
    if (flag && flag[r] == 0) {
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
void launch_dot_norm(const double2* V, int k, const double2* w, size_t n, double2* partial, double2* out,
                     const int* flag, int nrhs, const KS& ks, cudaStream_t st) {
    const int groups = (k + 1 + kDotG - 1) / kDotG;
    launch_pdl(k_dot_norm_partial, dim3(dim3(RED_CTAS, groups, nrhs)), dim3(256), 0, st, V, k, w, n, partial, flag, ks);
    launch_pdl(k_reduce_rows, dim3(dim3(1, k + 1, nrhs)), dim3(256), 0, st, partial, RED_CTAS, out, flag, ks);
}

// w -= sum_i coef[i] V_i, and per-CTA partial sums of |w_new|^2
__global__ void __launch_bounds__(512) k_axpy_norm(const double2* __restrict__ V, int k,
                                                   const double2* __restrict__ coef, double2* __restrict__ w, size_t n,
                                                   double* __restrict__ npart, const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive(ks, r) || (flag && flag[r] == 0)) return;
    V += r * ks.sv;
    w += r * ks.sw;
    coef += r * ks.so;
    npart += r * RED_CTAS;
    __shared__ double2 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = coef[threadIdx.x];
    __syncthreads();
    double nn = 0.0;
    constexpr int kU = 8;   // rows whose loads go out together
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc = w[e];
        int i = 0;
        for (; i + kU <= k; i += kU) {
            double2 v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = __ldg(V + (size_t)(i + u) * n + e);
#pragma unroll
            for (int u = 0; u < kU; ++u) cmsub(acc, c[i + u], v[u]);
        }
        for (; i < k; ++i) cmsub(acc, c[i], __ldg(V + (size_t)i * n + e));
        w[e] = acc;
        nn = fma(acc.x, acc.x, nn);
        nn = fma(acc.y, acc.y, nn);
    }
    double2 rs = block_sum2(make_double2(nn, 0.0));
    if (threadIdx.x == 0) npart[blockIdx.x] = rs.x;
}
void launch_axpy_norm(const double2* V, int k, const double2* coef, double2* w, size_t n, double* npart,
                      const int* flag, int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_axpy_norm, dim3(dim3(RED_CTAS, 1, nrhs)), dim3(512), 0, st, V, k, coef, w, n, npart, flag, ks);
}

// reduce the pass-1 norm, decide on the second pass, set ||w|| for the Givens
// step: sc[2] = ||w_final||, sc[3] counts second passes; flag = 1 when
// ||w'||^2 < ||w||^2 / 2
__global__ void __launch_bounds__(256) k_dgks_decide(const double* npart, int np, const double2* h1norm, int k,
                                                     int* flag, double* sc, double eta2, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    if (inactive(ks, r)) return;
    npart += r * RED_CTAS;
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += npart[e];
    double2 s = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) {
        const double w0 = h1norm[r * ks.so + k].x;          // ||w||^2 before pass 1
        const int f = (s.x < eta2 * w0) ? 1 : 0;
        flag[r] = f;
        sc[r * 8 + 2] = sqrt(s.x);
        sc[r * 8 + 3] += (double)f;
    }
}
void launch_dgks_decide(const double* npart, const double2* h1norm, int k, int* flag, double* sc, int nrhs,
                        const KS& ks, cudaStream_t st, double eta2) {
    launch_pdl(k_dgks_decide, dim3(nrhs), dim3(256), 0, st, npart, RED_CTAS, h1norm, k, flag, sc, eta2, ks);
}
// after pass 2: ||w''|| replaces ||w'||
__global__ void __launch_bounds__(256) k_pass2_norm(const double* npart, int np, const int* flag, double* sc, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    if (inactive(ks, r) || flag[r] == 0) return;
    npart += r * RED_CTAS;
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += npart[e];
    double2 s = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) sc[r * 8 + 2] = sqrt(s.x);
}
void launch_pass2_norm(const double* npart, const int* flag, double* sc, int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_pass2_norm, dim3(nrhs), dim3(256), 0, st, npart, RED_CTAS, flag, sc, ks);
}

// ---------------------------------------------------------------------------
// 2-norm of w per right-hand side: sc[r*8 + slot] = ||w_r||
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_norm2_partial(const double2* __restrict__ w, size_t n, double* partial, KS ks) {
    pdl_prologue();
    const int r = blockIdx.y;
    if (inactive(ks, r)) return;
    w += r * ks.sw;
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 b = w[e];
        acc += b.x * b.x + b.y * b.y;
    }
    double2 s = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) partial[r * RED_CTAS + blockIdx.x] = s.x;
}
__global__ void __launch_bounds__(256) k_norm2_final(const double* partial, int np, double* sc, int slot, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    if (inactive(ks, r)) return;
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) acc += partial[r * RED_CTAS + e];
    double2 s = block_sum2(make_double2(acc, 0.0));
    if (threadIdx.x == 0) sc[r * 8 + slot] = sqrt(s.x);
}
void launch_norm2(const double2* w, size_t n, double* partial, double* sc, int slot, int nrhs, const KS& ks,
                  cudaStream_t st) {
    launch_pdl(k_norm2_partial, dim3(dim3(RED_CTAS, nrhs)), dim3(256), 0, st, w, n, partial, ks);
    launch_pdl(k_norm2_final, dim3(nrhs), dim3(256), 0, st, partial, RED_CTAS, sc, slot, ks);
}

// x += sum_i y_i Z_i  (Z in the preconditioner's precision, x in FP64), k per right-hand side
template <class Vz>
__global__ void __launch_bounds__(256) k_update_x(const Vz* __restrict__ Z, const int* kk, const double2* __restrict__ y,
                                                  double2* __restrict__ x, size_t n, KS ks) {
    pdl_prologue();
    const int r = blockIdx.y;
    const int k = kk[r];
    if (k <= 0) return;
    Z += r * ks.sz;
    y += r * ks.so;
    x += r * ks.sx;
    __shared__ double2 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc = x[e];
        for (int i = 0; i < k; ++i) {
            const Vz zv = Z[(size_t)i * n + e];
            const double zx = (double)zv.x, zy = (double)zv.y;
            acc.x += c[i].x * zx - c[i].y * zy;
            acc.y += c[i].x * zy + c[i].y * zx;
        }
        x[e] = acc;
    }
}
// FP32 Z (mixed mode): the k products in double-float arithmetic (y split
// once per CTA into double-float pairs, every product an error-free FP32
// product, every sum a two-sum), added to the FP64 x once per element; the
// loads of kU rows go out together
template <>
__global__ void __launch_bounds__(256) k_update_x<float2>(const float2* __restrict__ Z, const int* kk,
                                                          const double2* __restrict__ y, double2* __restrict__ x,
                                                          size_t n, KS ks) {
    pdl_prologue();
    const int r = blockIdx.y;
    const int k = kk[r];
    if (k <= 0) return;
    Z += r * ks.sz;
    y += r * ks.so;
    x += r * ks.sx;
    __shared__ float4 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = cdf_from_double2(y[threadIdx.x]);
    __syncthreads();
    constexpr int kU = 8;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        dfacc ar, ai;
        auto mac = [&](const float2& zv, const float4& cc) {
            // (cr + i ci)(zx + i zy) = (cr zx - ci zy) + i (cr zy + ci zx)
            const dfl cr = re_of(cc), ci = im_of(cc);
            ar.add(df_mul_f(cr, zv.x));
            ar.add(df_neg(df_mul_f(ci, zv.y)));
            ai.add(df_mul_f(cr, zv.y));
            ai.add(df_mul_f(ci, zv.x));
        };
        int i = 0;
        for (; i + kU <= k; i += kU) {
            float2 zv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) zv[u] = __ldg(Z + (size_t)(i + u) * n + e);
#pragma unroll
            for (int u = 0; u < kU; ++u) mac(zv[u], c[i + u]);
        }
        for (; i < k; ++i) mac(__ldg(Z + (size_t)i * n + e), c[i]);
        double2 acc = x[e];
        acc.x += ar.value();
        acc.y += ai.value();
        x[e] = acc;
    }
}
template <class Vz>
void launch_update_x(const Vz* Z, const int* kk, const double2* y, double2* x, size_t n, int nrhs, const KS& ks,
                     cudaStream_t st) {
    launch_pdl(k_update_x<Vz>, dim3(dim3(RED_CTAS * 2, nrhs)), dim3(256), 0, st, Z, kk, y, x, n, ks);
}
template void launch_update_x<double2>(const double2*, const int*, const double2*, double2*, size_t, int, const KS&,
                                       cudaStream_t);
template void launch_update_x<float2>(const float2*, const int*, const double2*, double2*, size_t, int, const KS&,
                                      cudaStream_t);

// v = w / sc[slot]  (per right-hand side)
__global__ void k_scale_copy(const double2* __restrict__ w, const double* sc, int slot, double2* __restrict__ v,
                             size_t n, size_t sw, size_t sv, KS ks) {
    pdl_prologue();
    const int r = blockIdx.y;
    if (inactive(ks, r)) return;
    w += r * sw;
    v += r * sv;
    const double s = 1.0 / sc[r * 8 + slot];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = w[e];
        v[e] = make_double2(a.x * s, a.y * s);
    }
}
// c = a - b
__global__ void k_sub(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ c, size_t n) {
    pdl_prologue();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        c[e] = csub(a[e], b[e]);
}
void launch_sub(const double2* a, const double2* b, double2* c, size_t n, cudaStream_t st) {
    launch_pdl(k_sub, dim3(RED_CTAS * 2), dim3(256), 0, st, a, b, c, n);
}

void launch_scale_copy(const double2* w, const double* sc, int slot, double2* v, size_t n, size_t sw, size_t sv,
                       int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_scale_copy, dim3(dim3(RED_CTAS * 2, nrhs)), dim3(256), 0, st, w, sc, slot, v, n, sw, sv, ks);
}

// ---------------------------------------------------------------------------
// Hessenberg column j = h1 + h2 (two Gram-Schmidt passes) with subdiagonal
// ||w||; apply the previous Givens rotations, form the new one, update g.
// Rotation [c s; -conj(s) c] with c real.  status[0] = |g_{j+1}|,
// status[1] = h_{j+1,j}, status[2] = 1 if a non-finite value appeared.
// ---------------------------------------------------------------------------
__global__ void k_arnoldi_givens(double2* Hm, int ldh, const double2* h1, const double2* h2, const double* sc, int j,
                                 double2* cs, double2* sn, double2* g, double* status, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    if (inactive(ks, r)) return;
    double2* Hcol = Hm + r * ks.sh + (size_t)j * ldh;
    h1 += r * ks.so;
    h2 += r * ks.so;
    cs += r * ks.so;
    sn += r * ks.so;
    g += r * ks.so;
    status += r * 4;
    __shared__ double2 h[66];
    __shared__ double2 ssn[65];
    __shared__ double scs[65];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        h[i] = cadd(h1[i], h2[i]);
        if (i < j) { scs[i] = cs[i].x; ssn[i] = sn[i]; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double wn = sc[r * 8 + 2];
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
        const double na = sqrt(na2), rr = sqrt(na2 + nb2);
        c = na / rr;
        s = cscale(cmul(a, cconj(b)), 1.0 / (na * rr));
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
void launch_arnoldi_givens(double2* Hm, int ldh, const double2* h1, const double2* h2, const double* sc, int j,
                           double2* cs, double2* sn, double2* g, double* status, int nrhs, const KS& ks,
                           cudaStream_t st) {
    launch_pdl(k_arnoldi_givens, dim3(nrhs), dim3(32), 0, st, Hm, ldh, h1, h2, sc, j, cs, sn, g, status, ks);
}

// R y = g(0..k-1), R upper triangular stored column-major with leading dimension ldh
__global__ void k_triangular_solve(const double2* Hm, int ldh, const double2* g, const int* kk, double2* y, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    const int k = kk[r];
    if (threadIdx.x != 0 || k <= 0) return;
    Hm += r * ks.sh;
    g += r * ks.so;
    y += r * ks.so;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int c = i + 1; c < k; ++c) acc = csub(acc, cmul(Hm[(size_t)c * ldh + i], y[c]));
        y[i] = cdiv(acc, Hm[(size_t)i * ldh + i]);
    }
}
void launch_triangular_solve(const double2* Hm, int ldh, const double2* g, const int* kk, double2* y, int nrhs,
                             const KS& ks, cudaStream_t st) {
    launch_pdl(k_triangular_solve, dim3(nrhs), dim3(32), 0, st, Hm, ldh, g, kk, y, ks);
}

// g = beta e_1, status = (beta, 0, 0)
__global__ void k_init_arnoldi(const double* sc, double2* g, int m, double* status, KS ks) {
    pdl_prologue();
    const int r = blockIdx.x;
    if (inactive(ks, r)) return;
    g += r * ks.so;
    const double beta = sc[r * 8 + 0];
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
    if (threadIdx.x == 0) { status[r * 4 + 0] = beta; status[r * 4 + 1] = 0.0; status[r * 4 + 2] = 0.0; }
}
void launch_init_arnoldi(const double* sc, double2* g, int m, double* status, int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_init_arnoldi, dim3(nrhs), dim3(128), 0, st, sc, g, m, status, ks);
}

}  // namespace bah
