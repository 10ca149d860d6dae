// Kernels of block FGMRES: one Krylov space for a block of s right-hand sides
// (the batched form of the outer solve; FGMRES of Sec. 2.2 and Sec. 4 applied
// to a block).  The block basis uses the batched layout of the lockstep
// solver: column a of basis block i is V + a * sv + i * n (sv = the per-
// right-hand-side basis stride), W and X hold column b at b * n.
//
//   block dot    C[(i, a), b] = sum_e conj(V_i[a][e]) W[b][e]      ((k s) x s, k blocks)
//   block update W[b][e] -= sum_(i, a) V_i[a][e] C[(i, a), b]
//   block scale  V[b][e] = sum_(b' <= b) W[b'][e] T[b', b]          (W R^{-1}, CholQR)
//   solution     X[b][e] += sum_(i, a) Z_i[a][e] Y[(i, a), b]       (Z in the multigrid's precision)
//
// FP64 arithmetic with explicit fused multiply-adds; the dot partial sums are
// reduced in a fixed order.
#include "bah_internal.cuh"

namespace bah {

constexpr int kBlockMaxS = 16;     // right-hand sides per block (columns)

__device__ __forceinline__ void bmac_conj(double2& acc, const double2& a, const double2& b) {   // acc += conj(a) b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void bmac(double2& acc, const double2& a, const double2& b) {        // acc += a b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void bmsub(double2& acc, const double2& a, const double2& b) {       // acc -= a b
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// partial[row][b][cta] for row = i * s + a (i < k), one row per blockIdx.y;
// rows of A are at A + a * sa + i * n
template <int S>
__global__ void __launch_bounds__(256) k_bdot_partial(const double2* __restrict__ A, size_t sa, int s,
                                                      const double2* __restrict__ W, size_t n,
                                                      double2* __restrict__ partial) {
    pdl_prologue();
    const int row = blockIdx.y;
    const int i = row / s, a = row % s;
    const double2* v = A + (size_t)a * sa + (size_t)i * n;
    double2 acc[S];
#pragma unroll
    for (int b = 0; b < S; ++b) acc[b] = make_double2(0.0, 0.0);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 x = __ldg(v + e);
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (b < s) bmac_conj(acc[b], x, __ldg(W + (size_t)b * n + e));
    }
    __shared__ double2 sh[256 / 32][S];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        double2 t = acc[b];
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) sh[wp][b] = t;
    }
    __syncthreads();
    if (threadIdx.x < s) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t.x += sh[w][threadIdx.x].x;
            t.y += sh[w][threadIdx.x].y;
        }
        partial[((size_t)row * s + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}
// C[row * s + b] = sum over the CTAs' partials (fixed order)
__global__ void __launch_bounds__(256) k_bdot_reduce(const double2* __restrict__ partial, int np, double2* C) {
    pdl_prologue();
    const int q = blockIdx.x;                       // row * s + b
    double2 t = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const double2 v = partial[(size_t)q * np + e];
        t.x += v.x;
        t.y += v.y;
    }
    __shared__ double2 sh[256];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { sh[threadIdx.x].x += sh[threadIdx.x + o].x; sh[threadIdx.x].y += sh[threadIdx.x + o].y; }
        __syncthreads();
    }
    if (threadIdx.x == 0) C[q] = sh[0];
}
template <int S>
static void bdot_t(const double2* A, size_t sa, int k, int s, const double2* W, size_t n, double2* partial, double2* C,
                   cudaStream_t st) {
    launch_pdl(k_bdot_partial<S>, dim3(RED_CTAS, k * s), dim3(256), 0, st, A, sa, s, W, n, partial);
    launch_pdl(k_bdot_reduce, dim3(k * s * s), dim3(256), 0, st, (const double2*)partial, RED_CTAS, C);
}
void launch_block_dot(const double2* A, size_t sa, int k, int s, const double2* W, size_t n, double2* partial,
                      double2* C, cudaStream_t st) {
    if (s <= 4) bdot_t<4>(A, sa, k, s, W, n, partial, C, st);
    else if (s <= 8) bdot_t<8>(A, sa, k, s, W, n, partial, C, st);
    else bdot_t<16>(A, sa, k, s, W, n, partial, C, st);
}

// W[b][e] -= sum over rows (i, a) < k s of V_i[a][e] C[row, b]; coefficients in shared memory
template <int S>
__global__ void __launch_bounds__(256) k_bupdate(const double2* __restrict__ A, size_t sa, int k, int s,
                                                 const double2* __restrict__ C, double2* __restrict__ W, size_t n,
                                                 int subtract) {
    pdl_prologue();
    extern __shared__ double2 cs[];                  // (k s) x s
    for (int q = threadIdx.x; q < k * s * s; q += blockDim.x) cs[q] = C[q];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc[S];
#pragma unroll
        for (int b = 0; b < S; ++b) acc[b] = b < s ? W[(size_t)b * n + e] : make_double2(0.0, 0.0);
        for (int row = 0; row < k * s; ++row) {
            const int i = row / s, a = row % s;
            const double2 v = __ldg(A + (size_t)a * sa + (size_t)i * n + e);
#pragma unroll
            for (int b = 0; b < S; ++b)
                if (b < s) {
                    if (subtract) bmsub(acc[b], v, cs[row * s + b]);
                    else bmac(acc[b], v, cs[row * s + b]);
                }
        }
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (b < s) W[(size_t)b * n + e] = acc[b];
    }
}
void launch_block_update(const double2* A, size_t sa, int k, int s, const double2* C, double2* W, size_t n,
                         int subtract, cudaStream_t st) {
    const size_t smem = (size_t)k * s * s * sizeof(double2);
    if (s <= 4) launch_pdl(k_bupdate<4>, dim3(RED_CTAS * 2), dim3(256), smem, st, A, sa, k, s, C, W, n, subtract);
    else if (s <= 8) launch_pdl(k_bupdate<8>, dim3(RED_CTAS * 2), dim3(256), smem, st, A, sa, k, s, C, W, n, subtract);
    else launch_pdl(k_bupdate<16>, dim3(RED_CTAS * 2), dim3(256), smem, st, A, sa, k, s, C, W, n, subtract);
}

// V[b] (at V + b * sv) = sum_(b' <= b) W[b'] T[b', b] (T upper triangular, s x s, row-major)
template <int S>
__global__ void __launch_bounds__(256) k_bscale(const double2* W, int s, const double2* __restrict__ T, double2* V,
                                                size_t sv, size_t n) {
    pdl_prologue();
    __shared__ double2 ts[S * S];
    for (int q = threadIdx.x; q < s * s; q += blockDim.x) ts[q] = T[q];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 w[S];
#pragma unroll
        for (int b = 0; b < S; ++b) w[b] = b < s ? W[(size_t)b * n + e] : make_double2(0.0, 0.0);
#pragma unroll
        for (int b = 0; b < S; ++b) {
            if (b >= s) break;
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q <= b; ++q) bmac(acc, w[q], ts[q * s + b]);
            V[(size_t)b * sv + e] = acc;
        }
    }
}
void launch_block_scale(const double2* W, int s, const double2* T, double2* V, size_t sv, size_t n, cudaStream_t st) {
    if (s <= 4) launch_pdl(k_bscale<4>, dim3(RED_CTAS * 2), dim3(256), 0, st, W, s, T, V, sv, n);
    else if (s <= 8) launch_pdl(k_bscale<8>, dim3(RED_CTAS * 2), dim3(256), 0, st, W, s, T, V, sv, n);
    else launch_pdl(k_bscale<16>, dim3(RED_CTAS * 2), dim3(256), 0, st, W, s, T, V, sv, n);
}

// X[b][e] += sum over rows (i, a) < k s of Z_i[a][e] Y[row, b]  (Z FP32 or FP64 complex)
template <int S, class Vz>
__global__ void __launch_bounds__(256) k_bxupdate(const Vz* __restrict__ Z, size_t sz, int k, int s,
                                                  const double2* __restrict__ Y, double2* __restrict__ X, size_t n) {
    pdl_prologue();
    extern __shared__ double2 ys[];
    for (int q = threadIdx.x; q < k * s * s; q += blockDim.x) ys[q] = Y[q];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 acc[S];
#pragma unroll
        for (int b = 0; b < S; ++b) acc[b] = b < s ? X[(size_t)b * n + e] : make_double2(0.0, 0.0);
        for (int row = 0; row < k * s; ++row) {
            const int i = row / s, a = row % s;
            const Vz zv = Z[(size_t)a * sz + (size_t)i * n + e];
            const double2 z = make_double2((double)zv.x, (double)zv.y);
#pragma unroll
            for (int b = 0; b < S; ++b)
                if (b < s) bmac(acc[b], z, ys[row * s + b]);
        }
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (b < s) X[(size_t)b * n + e] = acc[b];
    }
}
template <class Vz>
void launch_block_xupdate(const Vz* Z, size_t sz, int k, int s, const double2* Y, double2* X, size_t n,
                          cudaStream_t st) {
    const size_t smem = (size_t)k * s * s * sizeof(double2);
    if (s <= 4) launch_pdl(k_bxupdate<4, Vz>, dim3(RED_CTAS * 2), dim3(256), smem, st, Z, sz, k, s, Y, X, n);
    else if (s <= 8) launch_pdl(k_bxupdate<8, Vz>, dim3(RED_CTAS * 2), dim3(256), smem, st, Z, sz, k, s, Y, X, n);
    else launch_pdl(k_bxupdate<16, Vz>, dim3(RED_CTAS * 2), dim3(256), smem, st, Z, sz, k, s, Y, X, n);
}
void block_kernels_smem(size_t bytes) {
    if (bytes <= 48 * 1024) return;
    const void* fns[] = {(const void*)k_bupdate<4>, (const void*)k_bupdate<8>, (const void*)k_bupdate<16>,
                         (const void*)k_bxupdate<4, float2>, (const void*)k_bxupdate<8, float2>,
                         (const void*)k_bxupdate<16, float2>, (const void*)k_bxupdate<4, double2>,
                         (const void*)k_bxupdate<8, double2>, (const void*)k_bxupdate<16, double2>};
    for (const void* f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaGetLastError();
}
template void launch_block_xupdate<float2>(const float2*, size_t, int, int, const double2*, double2*, size_t,
                                           cudaStream_t);
template void launch_block_xupdate<double2>(const double2*, size_t, int, int, const double2*, double2*, size_t,
                                            cudaStream_t);

}  // namespace bah
