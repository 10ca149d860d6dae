// Gram-Schmidt kernels on double-float Krylov vectors (see df.cuh): the basis
// V and the work vector w are float4 double-floats, the Hessenberg entries
// and norms come out in FP64.  Same batching, flags and reductions as the
// FP64 kernels of k_krylov.cu; only the element arithmetic differs: every
// product and sum is an error-free FP32 transformation, so the inner loops
// issue no FP64 instruction.
#include "bah_internal.cuh"
#include "df.cuh"

namespace bah {

__device__ __forceinline__ double2 warp_sum2_df(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double2 block_sum2_df(double2 v) {
    __shared__ double2 sh[32];   // one per warp, up to 1024 threads
    v = warp_sum2_df(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : make_double2(0.0, 0.0);
        r = warp_sum2_df(r);
    }
    __syncthreads();
    return r;
}
__device__ __forceinline__ bool inactive_df(const KS& ks, int r) { return ks.active && !ks.active[r]; }

// rows 0..k-1: conj(V_y) w; row k: |w|^2
__global__ void __launch_bounds__(256) k_dot_norm_partial_df(const float4* __restrict__ V, int k,
                                                             const float4* __restrict__ w, size_t n,
                                                             double2* __restrict__ partial, const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive_df(ks, r) || (flag && flag[r] == 0)) return;
    V += r * ks.sv;
    w += r * ks.sw;
    partial += r * ks.sp;
    const int y = blockIdx.y;
    dfacc are, aim;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    // conj(a) b = (ar br + ai bi) + i (ar bi - ai br), accumulated in element
    // order; the loads of kU elements go out together before any arithmetic
    auto mac = [&](const float4& a, const float4& b) {
        const dfl ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
        are.add_prod(ar, br);
        are.add_prod(ai, bi);
        aim.add_prod(ar, bi);
        aim.add_prod(df_neg(ai), br);
    };
    auto sq = [&](const float4& b) {
        const dfl br = re_of(b), bi = im_of(b);
        are.add_prod(br, br);
        are.add_prod(bi, bi);
    };
    constexpr int kU = 4;
    if (y < k) {
        const float4* v = V + (size_t)y * n;
        for (; e + (kU - 1) * stride < n; e += kU * stride) {
            float4 a[kU], b[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                a[u] = __ldg(v + e + u * stride);
                b[u] = __ldg(w + e + u * stride);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) mac(a[u], b[u]);
        }
        for (; e < n; e += stride) mac(__ldg(v + e), __ldg(w + e));
    } else {
        for (; e + (kU - 1) * stride < n; e += kU * stride) {
            float4 b[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) b[u] = __ldg(w + e + u * stride);
#pragma unroll
            for (int u = 0; u < kU; ++u) sq(b[u]);
        }
        for (; e < n; e += stride) sq(__ldg(w + e));
    }
    double2 acc = block_sum2_df(make_double2(are.value(), aim.value()));
    if (threadIdx.x == 0) partial[(size_t)y * gridDim.x + blockIdx.x] = acc;
}
__global__ void __launch_bounds__(256) k_reduce_rows_df(const double2* __restrict__ partial, int np, double2* out,
                                                        const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive_df(ks, r)) return;
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
    acc = block_sum2_df(acc);
    if (threadIdx.x == 0) out[blockIdx.y] = acc;
}
void launch_dot_norm_df(const float4* V, int k, const float4* w, size_t n, double2* partial, double2* out,
                        const int* flag, int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_dot_norm_partial_df, dim3(dim3(RED_CTAS, k + 1, nrhs)), dim3(256), 0, st, V, k, w, n, partial, flag, ks);
    launch_pdl(k_reduce_rows_df, dim3(dim3(1, k + 1, nrhs)), dim3(256), 0, st, partial, RED_CTAS, out, flag, ks);
}

// w -= sum_i coef[i] V_i (coef FP64, split once per CTA), per-CTA |w_new|^2
__global__ void __launch_bounds__(512) k_axpy_norm_df(const float4* __restrict__ V, int k,
                                                      const double2* __restrict__ coef, float4* __restrict__ w,
                                                      size_t n, double* __restrict__ npart, const int* flag, KS ks) {
    pdl_prologue();
    const int r = blockIdx.z;
    if (inactive_df(ks, r) || (flag && flag[r] == 0)) return;
    V += r * ks.sv;
    w += r * ks.sw;
    coef += r * ks.so;
    npart += r * RED_CTAS;
    __shared__ float4 c[64];
    if (threadIdx.x < k) c[threadIdx.x] = cdf_from_double2(coef[threadIdx.x]);
    __syncthreads();
    dfacc nn;
    constexpr int kU = 8;   // rows whose loads go out together
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float4 w0 = w[e];
        dfacc xr, xi;
        xr.hi = w0.x; xr.lo = w0.y;
        xi.hi = w0.z; xi.lo = w0.w;
        // w -= c v = (cr vr - ci vi) + i (cr vi + ci vr), rows in order
        auto sub = [&](const float4& v, const float4& cc) {
            const dfl vr = re_of(v), vi = im_of(v), cr = re_of(cc), ci = im_of(cc);
            xr.add_prod(df_neg(cr), vr);
            xr.add_prod(ci, vi);
            xi.add_prod(df_neg(cr), vi);
            xi.add_prod(df_neg(ci), vr);
        };
        int i = 0;
        for (; i + kU <= k; i += kU) {
            float4 v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = __ldg(V + (size_t)(i + u) * n + e);
#pragma unroll
            for (int u = 0; u < kU; ++u) sub(v[u], c[i + u]);
        }
        for (; i < k; ++i) sub(__ldg(V + (size_t)i * n + e), c[i]);
        w[e] = make_float4(xr.hi, xr.lo, xi.hi, xi.lo);
        nn.add_prod(dfl{xr.hi, xr.lo}, dfl{xr.hi, xr.lo});
        nn.add_prod(dfl{xi.hi, xi.lo}, dfl{xi.hi, xi.lo});
    }
    double2 rs = block_sum2_df(make_double2(nn.value(), 0.0));
    if (threadIdx.x == 0) npart[blockIdx.x] = rs.x;
}
void launch_axpy_norm_df(const float4* V, int k, const double2* coef, float4* w, size_t n, double* npart,
                         const int* flag, int nrhs, const KS& ks, cudaStream_t st) {
    launch_pdl(k_axpy_norm_df, dim3(dim3(RED_CTAS, 1, nrhs)), dim3(512), 0, st, V, k, coef, w, n, npart, flag, ks);
}

// v = w / sc[slot]: from a double-float w, or (from64) from an FP64 vector
template <bool FROM64>
__global__ void k_scale_copy_df(const void* __restrict__ wsrc, const double* sc, int slot, float4* __restrict__ v,
                                size_t n, size_t sw, size_t sv, KS ks) {
    pdl_prologue();
    const int r = blockIdx.y;
    if (inactive_df(ks, r)) return;
    v += r * sv;
    const dfl s = df_from_double(1.0 / sc[r * 8 + slot]);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        float4 a;
        if (FROM64) a = cdf_from_double2(((const double2*)wsrc)[r * sw + e]);
        else a = ((const float4*)wsrc)[r * sw + e];
        v[e] = cdf_make(df_mul(re_of(a), s), df_mul(im_of(a), s));
    }
}
void launch_scale_copy_df(const void* w, bool from64, const double* sc, int slot, float4* v, size_t n, size_t sw,
                          size_t sv, int nrhs, const KS& ks, cudaStream_t st) {
    if (from64) launch_pdl(k_scale_copy_df<true>, dim3(dim3(RED_CTAS * 2, nrhs)), dim3(256), 0, st, w, sc, slot, v, n, sw, sv, ks);
    else launch_pdl(k_scale_copy_df<false>, dim3(dim3(RED_CTAS * 2, nrhs)), dim3(256), 0, st, w, sc, slot, v, n, sw, sv, ks);
}

}  // namespace bah
