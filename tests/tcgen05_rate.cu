// Tensor-core rate at the shapes of a block Gram-Schmidt step (test program,
// built and run by tests/test_gpu_tcgen05_rate.py).
//
// A block Gram-Schmidt product C = V^H W with p basis vectors and s right-hand
// sides, written as a real GEMM, has M = p (tiles of 128), N = 2 s <= 32 and a
// K of twice the vector length.  This program measures what the fifth-
// generation tensor cores deliver at M = 128, K = 16 per instruction and
// N = 16 ... 256: tcgen05.mma (kind::f16, bfloat16 operands, FP32
// accumulator in tensor memory) issued by one thread per CTA, operands in
// shared memory in the K-major core-matrix layout without swizzle (8 rows x
// 16 bytes per core matrix; consecutive core matrices 128 bytes apart along
// K and (K / 8) x 128 bytes apart along M or N), one CTA per SM.
//
// First a check: D = A B^T for small integer operands, read back from tensor
// memory with tcgen05.ld, must equal the exact product.  Then, for each N, a
// timed launch of R x 4 accumulating instructions per CTA.  Every wait on the
// completion barrier is bounded; a CTA that gives up sets a flag, and the
// program reports it and exits non-zero.  Output: one JSON line per
// measurement.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {

constexpr int kM = 128, kK = 64;          // rows per tile, K staged per CTA (4 instructions of K = 16)
constexpr long kWaitLimit = 20000000L;    // try_wait rounds before a CTA gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading-dimension byte offset (K
// direction), stride-dimension byte offset (M/N direction), descriptor
// version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor, kind::f16: FP32 accumulator, bfloat16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// byte offset of element (row, k) of a K-major operand with kK columns
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((row / 8) * (kK / 8) * 128 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2);
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
    for (long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// D (kM x n, row-major FP32) = A (kM x kK) B (n x kK)^T, reps x 4 accumulating
// instructions (reps = 1: the product itself); one CTA of 128 threads
__global__ void __launch_bounds__(128, 1) k_mma(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                                                int n, int ncols, long reps, float* __restrict__ D, int* __restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sa = sm;
    unsigned char* sb = sm + kM * kK * 2;
    for (int e = tid; e < kM * kK; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(sa + core_off(e / kK, e % kK)) = A[e];
    for (int e = tid; e < n * kK; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(sb + core_off(e / kK, e % kK)) = B[e];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");       // generic-proxy writes -> tensor core reads
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem;
    const uint32_t idesc = instr_desc(kM, n);
    const uint32_t kcore = 128, mcore = (kK / 8) * 128;
    if (tid == 0) {
        uint64_t da[kK / 16], db[kK / 16];
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
            da[kk] = smem_desc(smem_u32(sa) + kk * 2 * kcore, kcore, mcore);
            db[kk] = smem_desc(smem_u32(sb) + kk * 2 * kcore, kcore, mcore);
        }
        for (long r = 0; r < reps; ++r)
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk) {
                const uint32_t acc = (r > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tbase),
                    "l"(da[kk]), "l"(db[kk]), "r"(idesc), "r"(acc)
                    : "memory");
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                     : "memory");
    }
    const bool ok = wait_parity(smem_u32(&bar), 0);
    if (!ok && tid == 0) atomicExch(flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && D) {
        // warp w reads lanes 32w .. 32w+31 (rows), 16 columns per load
        for (int c0 = 0; c0 < n; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int row = warp * 32 + lane;
            for (int c = 0; c < 16; ++c)
                D[((size_t)blockIdx.x * kM + row) * n + c0 + c] = __uint_as_float(r[c]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols) : "memory");
}

int ceil_pow2(int v) {
    int c = 32;
    while (c < v) c <<= 1;
    return c;
}

}  // namespace

int main() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nmax = 256;
    std::vector<float> fa((size_t)kM * kK), fb((size_t)nmax * kK);
    std::vector<__nv_bfloat16> ha(fa.size()), hb(fb.size());
    srand(7);
    for (size_t i = 0; i < fa.size(); ++i) { fa[i] = (float)(rand() % 17 - 8); ha[i] = __float2bfloat16(fa[i]); }
    for (size_t i = 0; i < fb.size(); ++i) { fb[i] = (float)(rand() % 17 - 8); hb[i] = __float2bfloat16(fb[i]); }
    __nv_bfloat16 *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    int* dflag = nullptr;
    cudaMalloc(&dA, ha.size() * 2);
    cudaMalloc(&dB, hb.size() * 2);
    cudaMalloc(&dD, (size_t)kM * nmax * 4);
    cudaMalloc(&dflag, 4);
    cudaMemcpy(dA, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice);
    cudaMemset(dflag, 0, 4);
    // dynamic shared memory: operands (48 KB at most), padded to keep one CTA per SM
    const size_t smem = 160 * 1024;
    if (cudaFuncSetAttribute(k_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        printf("{\"error\": \"shared memory attribute\"}\n");
        return 2;
    }
    // check: one CTA, exact integer product, N = 32 and N = 256
    for (int n : {32, 256}) {
        cudaMemset(dD, 0, (size_t)kM * n * 4);
        k_mma<<<1, 128, smem>>>(dA, dB, n, ceil_pow2(n), 1, dD, dflag);
        const cudaError_t e = cudaDeviceSynchronize();
        int flag = 0;
        cudaMemcpy(&flag, dflag, 4, cudaMemcpyDeviceToHost);
        std::vector<float> hd((size_t)kM * n);
        cudaMemcpy(hd.data(), dD, hd.size() * 4, cudaMemcpyDeviceToHost);
        double maxerr = 0;
        for (int i = 0; i < kM; ++i)
            for (int j = 0; j < n; ++j) {
                double ref = 0;
                for (int k = 0; k < kK; ++k) ref += (double)fa[(size_t)i * kK + k] * fb[(size_t)j * kK + k];
                maxerr = std::fmax(maxerr, std::fabs(ref - hd[(size_t)i * n + j]));
            }
        printf("{\"check\": true, \"n\": %d, \"cuda\": \"%s\", \"timeout\": %d, \"maxerr\": %g}\n", n,
               cudaGetErrorString(e), flag, maxerr);
        if (e != cudaSuccess || flag || maxerr != 0.0) return 1;
    }
    // rate: one CTA per SM, reps x 4 instructions each
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int n : {16, 32, 64, 128, 256}) {
        const long reps = 16384;
        k_mma<<<nsm, 128, smem>>>(dA, dB, n, ceil_pow2(n), 64, nullptr, dflag);    // warm-up
        cudaEventRecord(e0);
        k_mma<<<nsm, 128, smem>>>(dA, dB, n, ceil_pow2(n), reps, nullptr, dflag);
        cudaEventRecord(e1);
        const cudaError_t e = cudaEventSynchronize(e1);
        int flag = 0;
        cudaMemcpy(&flag, dflag, 4, cudaMemcpyDeviceToHost);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * nsm * reps * 4.0 * kM * n * 16.0;
        printf("{\"n\": %d, \"m\": %d, \"k_per_instr\": 16, \"ctas\": %d, \"instr_per_cta\": %ld, \"ms\": %.4f, "
               "\"tflops\": %.2f, \"cuda\": \"%s\", \"timeout\": %d}\n",
               n, kM, nsm, reps * 4, ms, flops / (ms * 1e-3) / 1e12, cudaGetErrorString(e), flag);
        if (e != cudaSuccess || flag) return 1;
    }
    return 0;
}
