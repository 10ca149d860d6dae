// bah_residual_norm_static: the true relative residual ||b - H x|| / ||b|| of
// up to BAH_STATIC_MAX_RHS right-hand sides, computed without allocating any
// memory.
//
// Why it exists: some callers cannot call cudaMalloc at the point where they
// need this number -- real-time or embedded loops that forbid allocator calls
// after start-up (an allocation can block for an unbounded time), and hosts
// whose device memory all belongs to another allocator (a framework's caching
// pool, which a direct cudaMalloc would bypass or find exhausted).  The rest
// of the library keeps its scratch in the context; this entry point keeps its
// scratch (the per-block partial sums of the reduction) in one file-scope
// device array instead, so a call only launches kernels.
//
// The kernel is a variant of the library's residual + norm pair: one pass
// forms b - H x cell by cell (with the same per-cell operator rows as the
// operator kernels, op_rows.cuh) and reduces |b - Hx|^2 and |b|^2 per block
// into the static array; a second kernel sums the partials in a fixed order
// and writes the ratio.  The results agree with the relative residual
// bah_solve reports up to rounding order.
//
// The device address of the array is looked up once per device and kept for
// the life of the process.  cudaDeviceReset unloads the library's device code
// and with it the array, so the cached address is stale afterwards: this
// entry point must not be called on a device after cudaDeviceReset.
#include "bah_internal.cuh"
#include "op_rows.cuh"

namespace bah {

constexpr int kStaticCtas = RED_CTAS;       // partial sums per right-hand side and quantity

// Shared by every call in the process on this device; 2 * 64 * 296 doubles
// (296 KiB).  Each call overwrites every slot it reads, so nothing needs
// clearing; calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_static_scratch[2 * BAH_STATIC_MAX_RHS * kStaticCtas];

// device address of g_static_scratch per device, looked up on the first call
static double* g_scratch_addr[64] = {nullptr};

__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double sh[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// blockIdx.y = right-hand side; partial layout [rhs][quantity][cta]
__global__ void __launch_bounds__(256) k_static_residual_partial(OpCoef c, const double2* __restrict__ bb,
                                                                 const double2* __restrict__ xx, size_t vlen,
                                                                 double* scratch) {
    const int n1 = c.n1, n2 = c.n2, np = n1 * n2;
    const int rhs = blockIdx.y;
    const double2* x = xx + (size_t)rhs * vlen;
    const double2* b = bb + (size_t)rhs * vlen;
    const double2* x1 = x;
    const double2* x2 = x + np;
    const double2* xp = x + 2 * np;
    const double2 z = make_double2(0.0, 0.0);
    double rr = 0.0, bn = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < np; t += gridDim.x * blockDim.x) {
        const int i = t % n1, j = t / n1;
        auto U1 = [&](int ii, int jj) { return (ii >= 1 && ii < n1 && jj >= 0 && jj < n2) ? x1[jj * n1 + ii] : z; };
        auto U2 = [&](int ii, int jj) { return (ii >= 0 && ii < n1 && jj >= 1 && jj < n2) ? x2[jj * n1 + ii] : z; };
        auto P = [&](int g) { return xp[g]; };
        double2 y1, y2, yp;
        elastic_rows(c, i, j, t, 1.0, U1, U2, P, y1, y2, yp);
        if (i >= 1) {
            const double2 r = csub(b[t], y1);
            rr += r.x * r.x + r.y * r.y;
            bn += b[t].x * b[t].x + b[t].y * b[t].y;
        }
        if (j >= 1) {
            const double2 r = csub(b[np + t], y2);
            rr += r.x * r.x + r.y * r.y;
            bn += b[np + t].x * b[np + t].x + b[np + t].y * b[np + t].y;
        }
        const double2 r = csub(b[2 * np + t], yp);
        rr += r.x * r.x + r.y * r.y;
        bn += b[2 * np + t].x * b[2 * np + t].x + b[2 * np + t].y * b[2 * np + t].y;
    }
    rr = block_sum_d(rr);
    bn = block_sum_d(bn);
    if (threadIdx.x == 0) {
        scratch[((size_t)rhs * 2 + 0) * kStaticCtas + blockIdx.x] = rr;
        scratch[((size_t)rhs * 2 + 1) * kStaticCtas + blockIdx.x] = bn;
    }
}

__global__ void __launch_bounds__(256) k_static_residual_final(const double* scratch, double* relres) {
    const int rhs = blockIdx.x;
    double rr = 0.0, bn = 0.0;
    for (int e = threadIdx.x; e < kStaticCtas; e += blockDim.x) {
        rr += scratch[((size_t)rhs * 2 + 0) * kStaticCtas + e];
        bn += scratch[((size_t)rhs * 2 + 1) * kStaticCtas + e];
    }
    rr = block_sum_d(rr);
    bn = block_sum_d(bn);
    if (threadIdx.x == 0) relres[rhs] = bn > 0.0 ? sqrt(rr) / sqrt(bn) : 0.0;
}

// operator coefficients of a context (defined in solver.cu)
const OpCoef* context_op(const bah_ctx* ctx);
size_t context_vec_len(const bah_ctx* ctx);

}  // namespace bah

extern "C" int bah_residual_norm_static(bah_ctx* ctx, const void* b, const void* x, int nrhs, double* relres,
                                        void* stream) {
    using namespace bah;
    if (!ctx || !b || !x || !relres || nrhs < 0) { set_error("bad argument"); return BAH_ERR_ARG; }
    if (nrhs > BAH_STATIC_MAX_RHS) {
        set_error("bah_residual_norm_static: nrhs exceeds BAH_STATIC_MAX_RHS (64), the size of its static scratch");
        return BAH_ERR_ARG;
    }
    if (!context_op(ctx)) {
        set_error("bah_residual_norm_static is implemented for 2-D grids");
        return BAH_ERR_UNSUPPORTED;
    }
    if (nrhs == 0) return BAH_OK;
    int dev = 0;
    BAH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index out of range"); return BAH_ERR_ARG; }
    if (!g_scratch_addr[dev]) {
        // set-up, once per device, with that device current: the device address
        // of the file-scope array (its host-side name is only a stand-in)
        void* p = nullptr;
        BAH_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_addr[dev] = (double*)p;
    }
    double* scratch = g_scratch_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    const OpCoef* op = context_op(ctx);
    k_static_residual_partial<<<dim3(kStaticCtas, nrhs), 256, 0, st>>>(*op, (const double2*)b, (const double2*)x,
                                                                      context_vec_len(ctx), scratch);
    k_static_residual_final<<<nrhs, 256, 0, st>>>(scratch, relres);
    BAH_CUDA_TRY(cudaGetLastError());
    return BAH_OK;
}
