// gemm_tc.cu -- Blackwell (sm_103a) tensor-core GEMM for the emulated-FP64
// (Ozaki, BF16 slices) and mixed-precision (BF16 / TF32) modes.
//
//   C[rmap(m) + cmap(n)] (= or +=) sum_passes 2^(eA[m] + eB[n] + base - beta*level)
//                                  * sum_{k in pass range} sum_{i+j=level} A_i(m,k) B_j(n,k)
//
// Both operands are K-major slice stacks D[slice][row][pitch].  One CTA owns a
// 128 x 256 output tile and runs the pass list; within a pass the products
// A_i B_j^T with i + j = level are accumulated in FP32 in tensor memory (exact
// for integer-valued slices while partial sums stay below 2^24); at the end of a
// pass the epilogue adds the scaled FP32 tile into C in FP64.  Two TMEM
// accumulators (2 x 256 columns) let the MMAs of pass p+1 run while the
// epilogue drains pass p.
//
// Warp roles (192 threads):
//   warp 0      TMA producer: 128B-swizzled tiles of A (128 x 128 B) and B
//               (256 x 128 B) per stage, 4 stages, mbarrier complete_tx.
//   warp 1      TMEM allocator and MMA issuer: tcgen05.mma.cta_group::1
//               (M=128, N=256, K=16 bf16 / K=8 tf32) into TMEM, tcgen05.commit
//               to free a stage / publish an accumulator.
//   warps 2..5  epilogue: tcgen05.ld (32 lanes x 32 columns), transpose
//               through shared memory, scaled FP64 read-modify-write of C with
//               coalesced 256-byte row segments.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the CTA raises a
// shared abort flag and the device status word, drains the copies and MMAs it
// has in flight (with a fixed bound), frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int BM = 128, BN = 256, STAGES = 4;
constexpr int ROW_BYTES = 128;                    // K bytes per stage row (one swizzle atom)
constexpr int A_BYTES = BM * ROW_BYTES;           // 16 KB
constexpr int B_BYTES = BN * ROW_BYTES;           // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;
constexpr unsigned long long kDrainLimitNs = 1000000000ull;  // bound on the abort-path drains

struct SmemCtl {
    unsigned long long full[STAGES];
    unsigned long long empty[STAGES];
    unsigned long long tfull[2];
    unsigned long long tempty[2];
    unsigned long long drain;
    unsigned int tmem_base;
    volatile int abort;
    long long rowoff[BM];
    int eA[BM];
    int eB[BN];
    float stage[EPI_WARPS][32][33];
};
constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + sizeof(SmemCtl);

struct Params {
    int M, N, K;
    long long rowA0, rowB0;
    const int* eA; const int* eB;
    int scale_base, beta, nslices;
    int nlevel, level0;
    int kchunk[9];   // per level: K elements per pass (multiple of the stage K), 0 = whole K
    OutDesc out;
    int* status;
    unsigned long long wait_ns;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(unsigned long long* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the abort flag) when the bound expires
// or another role has aborted.
__device__ __noinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, SmemCtl* ctl, int* status,
                                       unsigned long long limit_ns)
{
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtime();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 63) == 0) {
            if (ctl->abort) return false;
            if (gtime() - t0 > limit_ns) {
                ctl->abort = 1;
                atomicOr(status, 1);
                return false;
            }
        }
    }
}

// Wait used only on the abort path: fixed bound, ignores the abort flag.
__device__ __noinline__ void mbar_drain_wait(unsigned long long* b, uint32_t parity, int* status)
{
    const unsigned long long t0 = gtime();
    while (!mbar_try(b, parity)) {
        if (gtime() - t0 > kDrainLimitNs) { atomicOr(status, 2); return; }
    }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ unsigned long long smem_desc(const void* p)
{
    const unsigned long long addr = smem_u32(p);
    unsigned long long d = 0;
    d |= (addr >> 4) & 0x3fffull;              // start address
    d |= (unsigned long long)1 << 16;          // leading byte offset (unused for swizzled K-major)
    d |= (unsigned long long)(1024 >> 4) << 32;  // stride byte offset
    d |= (unsigned long long)1 << 46;          // version
    d |= (unsigned long long)2 << 61;          // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format (1 = BF16, 2 = TF32),
// both K-major, N = 256, M = 128.
template <int KIND>
__device__ __forceinline__ uint32_t instr_desc()
{
    const uint32_t fmt = KIND == TC_BF16 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, unsigned long long adesc, unsigned long long bdesc, uint32_t idesc,
                                    uint32_t accumulate)
{
    if (KIND == TC_BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ double pow2(int e)
{
    e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Pass sequence, shared by all roles: levels level0 .. level0+nlevel-1, each cut
// into K-chunks.  Returns false past the end.
struct PassIter {
    int level, k0, k1;
    int li;
    __device__ void begin(const Params& p)
    {
        li = 0;
        level = p.level0;
        k0 = 0;
        const int kc = p.kchunk[0];
        k1 = (kc > 0 && kc < p.K) ? kc : p.K;
    }
    __device__ bool next(const Params& p)
    {
        if (k1 < p.K) {
            k0 = k1;
            const int kc = p.kchunk[li];
            k1 = (kc > 0 && k0 + kc < p.K) ? k0 + kc : p.K;
            return true;
        }
        if (++li >= p.nlevel) return false;
        level = p.level0 + li;
        k0 = 0;
        const int kc = p.kchunk[li];
        k1 = (kc > 0 && kc < p.K) ? kc : p.K;
        return true;
    }
};

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* tiles = base;
    SmemCtl* ctl = (SmemCtl*)(base + STAGES * STAGE_BYTES);

    constexpr int KSTEP = KIND == TC_BF16 ? 64 : 32;  // K elements per stage
    constexpr int KMMA = KIND == TC_BF16 ? 16 : 8;    // K per tcgen05.mma
    constexpr int NMMA = KSTEP / KMMA;                // 4

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    // ---- set-up: barriers, TMEM, per-tile row offsets and exponents
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&ctl->full[s], 1); mbar_init(&ctl->empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&ctl->tfull[b], 1); mbar_init(&ctl->tempty[b], EPI_WARPS); }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int r = threadIdx.x; r < BM; r += THREADS) {
        const int m = m0 + r;
        ctl->rowoff[r] = (m < p.M) ? map2(p.out.rmap, m) : -1;
        ctl->eA[r] = (p.eA && m < p.M) ? p.eA[p.rowA0 + m] : 0;
    }
    for (int c = threadIdx.x; c < BN; c += THREADS) {
        const int n = n0 + c;
        ctl->eB[c] = (p.eB && n < p.N) ? p.eB[p.rowB0 + n] : 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;
            bool ok = true;
            PassIter it;
            it.begin(p);
            do {
                const int lo = it.level - (p.nslices - 1) > 0 ? it.level - (p.nslices - 1) : 0;
                const int hi = it.level < p.nslices - 1 ? it.level : p.nslices - 1;
                for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                    for (int i = lo; i <= hi && ok; ++i) {
                        if (!mbar_wait(&ctl->empty[stage], phase ^ 1, ctl, p.status, p.wait_ns)) { ok = false; break; }
                        unsigned char* sa = tiles + stage * STAGE_BYTES;
                        mbar_expect_tx(&ctl->full[stage], STAGE_BYTES);
                        tma_load_3d(sa, &tmA, &ctl->full[stage], kb, (int)(p.rowA0 + m0), i);
                        tma_load_3d(sa + A_BYTES, &tmB, &ctl->full[stage], kb, (int)(p.rowB0 + n0), it.level - i);
                        ++issued;
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                }
            } while (ok && it.next(p));
            if (!ok) {
                // drain: the last min(issued, STAGES) stages may still have copies in flight
                const long long n = issued < STAGES ? issued : STAGES;
                for (long long q = 1; q <= n; ++q) {
                    const long long u = issued - q;  // use index of that copy
                    mbar_drain_wait(&ctl->full[u % STAGES], (uint32_t)((u / STAGES) & 1), p.status);
                }
            }
        }
    } else if (warp == 1) {
        // ----------------------------------------------------------------- MMA
        if (lane == 0) {
            const uint32_t idesc = instr_desc<KIND>();
            int stage = 0;
            uint32_t phase = 0;
            int pass = 0;
            bool ok = true, any = false;
            PassIter it;
            it.begin(p);
            do {
                const int buf = pass & 1;
                const uint32_t use = (uint32_t)(pass >> 1);
                if (!mbar_wait(&ctl->tempty[buf], (use & 1) ^ 1, ctl, p.status, p.wait_ns)) { ok = false; break; }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                const int lo = it.level - (p.nslices - 1) > 0 ? it.level - (p.nslices - 1) : 0;
                const int hi = it.level < p.nslices - 1 ? it.level : p.nslices - 1;
                uint32_t acc = 0;
                for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                    for (int i = lo; i <= hi; ++i) {
                        if (!mbar_wait(&ctl->full[stage], phase, ctl, p.status, p.wait_ns)) { ok = false; break; }
                        fence_after();
                        unsigned char* sa = tiles + stage * STAGE_BYTES;
                        const unsigned long long ad = smem_desc(sa), bd = smem_desc(sa + A_BYTES);
#pragma unroll
                        for (int j = 0; j < NMMA; ++j) {
                            // advance the start address by 32 bytes per MMA K-step
                            mma<KIND>(d, ad + (unsigned long long)((j * 32) >> 4), bd + (unsigned long long)((j * 32) >> 4),
                                      idesc, acc);
                            acc = 1;
                        }
                        any = true;
                        mma_commit(&ctl->empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                }
                if (!ok) break;
                mma_commit(&ctl->tfull[buf]);
                ++pass;
            } while (it.next(p));
            if (!ok && any) {
                mma_commit(&ctl->drain);
                mbar_drain_wait(&ctl->drain, 0, p.status);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int row0 = q * 32;
        float(*stg)[33] = ctl->stage[warp - 2];
        int pass = 0;
        PassIter it;
        it.begin(p);
        do {
            const int buf = pass & 1;
            const uint32_t use = (uint32_t)(pass >> 1);
            if (!mbar_wait(&ctl->tfull[buf], use & 1, ctl, p.status, p.wait_ns)) break;
            fence_after();
            const bool store_only = (pass == 0) && !p.out.accumulate;
            const int lvl_shift = p.scale_base - p.beta * it.level;
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)row0 << 16) + (uint32_t)(buf * BN + c * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane][j] = v[j];
                __syncwarp();
                const int n = n0 + c * 32 + lane;
                const bool ncol = n < p.N;
                const long long co = ncol ? map2(p.out.cmap, n) : 0;
                const int eb = ctl->eB[c * 32 + lane] + lvl_shift;
                for (int r = 0; r < 32; ++r) {
                    const long long ro = ctl->rowoff[row0 + r];
                    if (ro < 0 || !ncol) continue;
                    const double x = (double)stg[r][lane] * pow2(ctl->eA[row0 + r] + eb);
                    double* dst = p.out.C + ro + co;
                    *dst = store_only ? x : *dst + x;
                }
                __syncwarp();
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
            ++pass;
        } while (it.next(p));
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// 3-D map over a slice stack [slices][rows][pitch] with extent K in the inner dim.
bool make_map(CUtensorMap* m, const void* base, int kind, long long K, long long pitch, long long rows, int slices,
              int box_rows)
{
    auto enc = get_encode();
    if (!enc) return false;
    const int esz = kind == TC_BF16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * esz), (cuuint64_t)(pitch * esz * rows)};
    cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / esz), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, kind == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

int tc_gemm_available() { return get_encode() != nullptr; }

cudaError_t gemm_tc(const GemmTc& g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.K <= 0 || g.slices < 1 || g.slices > 8 || g.nlevel < 1 || g.nlevel > 9) return cudaErrorInvalidValue;
    if (g.level0 < 0 || g.level0 + g.nlevel - 1 > 2 * (g.slices - 1)) return cudaErrorInvalidValue;
    const int kstep = g.kind == TC_BF16 ? 64 : 32;
    Params p{};
    p.M = g.M; p.N = g.N; p.K = g.K;
    p.rowA0 = g.rowA0; p.rowB0 = g.rowB0;
    p.eA = g.eA; p.eB = g.eB;
    p.scale_base = g.scale_base; p.beta = g.beta; p.nslices = g.slices;
    p.nlevel = g.nlevel;
    p.level0 = g.level0;
    for (int i = 0; i < g.nlevel; ++i) {
        if (g.kchunk[i] < 0 || g.kchunk[i] % kstep) return cudaErrorInvalidValue;
        p.kchunk[i] = g.kchunk[i];
    }
    p.out = g.out;
    p.status = g.status;
    p.wait_ns = g.wait_ns;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.kind, g.K, g.pitchA, g.rowsA, g.slices, BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb, g.B, g.kind, g.K, g.pitchB, g.rowsB, g.slices, BN)) return cudaErrorInvalidValue;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    static bool attr_done[2] = {false, false};
    if (g.kind == TC_BF16) {
        if (!attr_done[0]) {
            cudaFuncSetAttribute(gemm_tc_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
            attr_done[0] = true;
        }
        gemm_tc_kernel<TC_BF16><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, p);
    } else {
        if (!attr_done[1]) {
            cudaFuncSetAttribute(gemm_tc_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
            attr_done[1] = true;
        }
        gemm_tc_kernel<TC_TF32><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, p);
    }
    return cudaGetLastError();
}

}  // namespace cc
