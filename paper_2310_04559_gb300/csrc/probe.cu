// probe.cu -- peak-rate microbenchmarks of the arithmetic units the precision
// modes run on, so that every mode's throughput has a roofline measured on the
// same GPU in the same run:
//
//   CC_PROBE_DMMA        FP64 tensor-core MMA (mma.sync.m8n8k4.f64), the FP64 mode's GEMMs
//   CC_PROBE_DFMA        scalar FP64 fused multiply-add
//   CC_PROBE_TC_BF16     tcgen05.mma kind::f16 with BF16 operands, M=128 N=256 K=16 (emulated
//                        FP64 slices and the BF16 mode)
//   CC_PROBE_TC_TF32     tcgen05.mma kind::tf32, M=128 N=256 K=8 (the TF32 mode)
//   CC_PROBE_IMMA        legacy INT8 tensor-core MMA (mma.sync.m16n8k32.s8), the only INT8 MMA that
//                        assembles for sm_103a (tcgen05 has no kind::i8 there), for the record
//
// Each probe keeps the unit busy from registers or shared memory only (no
// global-memory operands), times itself with CUDA events around the launch and
// reports flops per second of the whole GPU.  The tensor-core probes issue MMAs
// back to back from one thread per SM on fixed shared-memory tiles into a TMEM
// accumulator; their only wait (for the last MMAs) is bounded by the global timer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cc_internal.cuh"

namespace cc {
namespace {

__device__ double g_probe_sink;  // keeps the probes' results observable
__device__ int g_probe_status;   // set when a tensor-core probe's wait ran out

__global__ void __launch_bounds__(256) dmma_probe_kernel(int iters, double seed)
{
    double a = seed + threadIdx.x * 1e-9, b = 1.0 - seed * 1e-3;
    double d[8][2];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q][0] = d[q][1] = q * 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(d[q][0]), "+d"(d[q][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += d[q][0] + d[q][1];
    if (s == 1234.5678) g_probe_sink = s;
}

__global__ void __launch_bounds__(256) imma_probe_kernel(int iters, int seed)
{
    const int a = seed * 0x01010101 + (int)threadIdx.x, b = 0x02030405 ^ seed;
    int d[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q][0] = d[q][1] = d[q][2] = d[q][3] = q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%4,%4,%4}, {%5,%5}, "
                         "{%0,%1,%2,%3};"
                         : "+r"(d[q][0]), "+r"(d[q][1]), "+r"(d[q][2]), "+r"(d[q][3])
                         : "r"(a), "r"(b));
    }
    int s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += d[q][0] + d[q][1] + d[q][2] + d[q][3];
    if (s == 1234567) g_probe_sink = s;
}

__global__ void __launch_bounds__(256) dfma_probe_kernel(int iters, double seed)
{
    double x[8];
    const double m = 1.0 - 1e-9 * seed, c = 1e-12 * threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = seed + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = fma(x[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q];
    if (s == 1234.5678) g_probe_sink = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 128-byte swizzled operand tile (8-row groups 1024 bytes apart), descriptor version 1.
__device__ __forceinline__ unsigned long long probe_desc(const void* p)
{
    const unsigned long long addr = smem_u32(p);
    return ((addr >> 4) & 0x3fffull) | (1ull << 16) | ((unsigned long long)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

template <bool TF32>
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int iters, unsigned long long limit_ns)
{
    constexpr int BM = 128, BN = 256;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* A = base;                 // 128 rows x 128 bytes
    unsigned char* B = base + BM * 128;      // 256 rows x 128 bytes
    __shared__ unsigned long long bar;
    __shared__ uint32_t tmem_base;
    // small values (exact in bf16 / tf32) so the arithmetic is real work
    for (int q = threadIdx.x; q < (BM + BN) * 128 / 4; q += blockDim.x) {
        const float f = (float)((q * 7 + blockIdx.x) % 13 - 6);
        uint32_t w;
        if (TF32) {
            w = __float_as_uint(f);
        } else {
            const uint32_t h = __float_as_uint(f) >> 16;
            w = h | (h << 16);
        }
        ((uint32_t*)base)[q] = w;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t fmt = TF32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(BM >> 4) << 24);
        const unsigned long long ad = probe_desc(A), bd = probe_desc(B);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // four K-steps of 32 bytes per 128-byte row
                const uint32_t acc = (it | k) ? 1u : 0u;
                if (TF32)
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(tmem), "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(idesc), "r"(acc));
                else
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(tmem), "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar))
                     : "memory");
    }
    // every thread waits for the MMAs (bounded by the global timer)
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(smem_u32(&bar))
                     : "memory");
        if (ok) break;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            atomicOr(&g_probe_status, 1);
            break;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

}  // namespace
}  // namespace cc

extern "C" int cc_ladder_peak_probe(int which, int iters, void* stream, double* tflops)
{
    using namespace cc;
    if (!tflops) return CC_ERR_NULL;
    if (which < CC_PROBE_DMMA || which > CC_PROBE_IMMA || iters < 1 || iters > (1 << 24)) return CC_ERR_ARG;
    const bool tc = which == CC_PROBE_TC_BF16 || which == CC_PROBE_TC_TF32;
    if (tc && !tc_gemm_available()) return CC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int nsm = device_sm_count();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CC_ERR_CUDA;
    const int zero = 0;
    double flops = 0.0;
    cudaError_t err = cudaMemcpyToSymbolAsync(g_probe_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    // 48 KB of operand tiles, padded so that one CTA fills an SM (its tensor core and TMEM)
    const size_t tc_smem = 120 * 1024;
    if (err == cudaSuccess && tc) {
        err = cudaFuncSetAttribute(tc_probe_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(tc_probe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
    }
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {  // rep 0 warms up
        cudaEventRecord(e0, st);
        switch (which) {
        case CC_PROBE_DMMA:
            dmma_probe_kernel<<<nsm * 8, 256, 0, st>>>(iters, 0.5);
            flops = (double)nsm * 8 * (256 / 32) * iters * 8 * (2.0 * 8 * 8 * 4);
            break;
        case CC_PROBE_DFMA:
            dfma_probe_kernel<<<nsm * 8, 256, 0, st>>>(iters, 0.5);
            flops = (double)nsm * 8 * 256 * iters * 8 * 2.0;
            break;
        case CC_PROBE_IMMA:
            imma_probe_kernel<<<nsm * 8, 256, 0, st>>>(iters, 3);
            flops = (double)nsm * 8 * (256 / 32) * iters * 8 * (2.0 * 16 * 8 * 32);
            break;
        case CC_PROBE_TC_BF16:
            tc_probe_kernel<false><<<nsm, 128, tc_smem, st>>>(iters, 2000000000ull);
            flops = (double)nsm * iters * 4 * (2.0 * 128 * 256 * 16);
            break;
        default:
            tc_probe_kernel<true><<<nsm, 128, tc_smem, st>>>(iters, 2000000000ull);
            flops = (double)nsm * iters * 4 * (2.0 * 128 * 256 * 8);
            break;
        }
        count_launch();
        cudaEventRecord(e1, st);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    }
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    int h = 0;
    if (err == cudaSuccess) err = cudaMemcpyFromSymbol(&h, g_probe_status, sizeof(int));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return CC_ERR_CUDA;
    if (h) return CC_ERR_DEVICE_TIMEOUT;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return CC_OK;
}
