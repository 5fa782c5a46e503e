// gemm_tc.cu -- Blackwell (sm_103a) tensor-core GEMM for the emulated-FP64
// (Ozaki, BF16 slices) and mixed-precision (BF16 / TF32) modes.
//
//   C[rmap(m) + cmap(n)] (= or +=) sum_levels 2^(eA[m] + eB[n] + base - beta*level)
//                                  * sum_{i+j=level} A_i(m,:) . B_j(n,:)
//
// Operands are K-major slice stacks D[slice][row][pitch].  One CTA owns a
// 128 x 256 output tile.  The slice-product levels are processed in groups of
// at most two (a "pass" = one group over one K-range); each level of a group
// accumulates in FP32 in its own TMEM accumulator (2 x 256 columns), exact for
// integer-valued slices while partial sums stay below 2^24.
//
// Operand reuse: for every K-step (64 bf16 / 32 tf32 elements = one 128-byte
// swizzle atom per row) each slice tile the group needs is loaded once.  The B
// slices stream in order j = lo..hi through a ring of 32 KB slots; the A slices
// arrive in order i = hi..lo through a ring of 16 KB slots, so B_j meets every
// A_i with i + j in the group while A_i lives only until its last partner
// B_{L2-i} has passed (about two B steps).  For 6 slices the 21 slice products
// of a K-step cost 24 tile loads instead of 42.
//
// Epilogues:
//   FIXED64  every pass adds its levels, converted exactly to a signed 64-bit
//            fixed-point number (2^-F of a level-0 unit), into the output tile
//            held as int64; the last pass scales it once into FP64.  No FP64
//            arithmetic until that single conversion (GB300's FP64 pipe is slow).
//   FIXED64_RED  as FIXED64 but the output stays int64 fixed point: the first pass
//            stores, later passes add with red.global (no loads in the epilogue); the
//            split kernel that consumes the intermediate applies the exponents.
//   FIXED64_ADD  split-K: every pass of every CTA adds with red.global into an int64
//            tile zeroed beforehand; fixed_to_f64 converts it afterwards.
//   FP64RMW  every pass adds 2^e * acc into the FP64 output (mixed modes, and
//            accumulation into caller data).  Single-level passes alternate the
//            two accumulators so the MMAs of pass p+1 overlap the drain of pass p.
//
// Warp roles (352 threads): warp 0 TMA producer, warps 1-2 MMA issuers
// (tcgen05.mma.cta_group::1, M=128, N=256; warp 1 also allocates TMEM), warps 3..10 epilogue:
// two warps per TMEM lane quarter, each owning one half of the tile's columns (tcgen05.ld of
// 32 lanes x 16 columns, transpose through shared memory, global accesses of two rows x 128
// contiguous bytes per instruction).  The epilogue of a pass keeps the MMA warps waiting, so
// it is kept short: both levels of a pair are combined into one int64 per element.  CTAs are rastered in groups of M-tiles so the
// CTAs resident at once share their A and B tiles in L2.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the CTA raises a
// shared abort flag and the device status word, drains the copies and MMAs it
// has in flight (with a fixed bound), frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int BM = 128, BN = 256;
constexpr int ROW_BYTES = 128;                 // K bytes per tile row: one 128-byte swizzle atom
constexpr int A_TILE = BM * ROW_BYTES;         // 16 KB per A slice tile
constexpr int B_TILE = BN * ROW_BYTES;         // 32 KB per B slice tile
constexpr int NA = 4, NB = 4;                  // A ring and B ring slots (powers of two)
static_assert((NA & (NA - 1)) == 0 && (NB & (NB - 1)) == 0, "ring sizes must be powers of two");
constexpr int TILE_SMEM = NA * A_TILE + NB * B_TILE;  // 192 KB
constexpr int MAX_SLICES = 8;
constexpr int EPI_WARPS = 8;                   // two per TMEM lane quarter
constexpr int ISSUERS = 2;                     // MMA-issuing warps (one per level of a pair)
constexpr int THREADS = 32 * (1 + ISSUERS + EPI_WARPS);
constexpr int TMEM_COLS = 512;
constexpr unsigned long long kDrainLimitNs = 1000000000ull;  // bound on the abort-path drains

struct SmemCtl {
    unsigned long long afull[NA], aempty[NA];
    unsigned long long bfull[NB], bempty[NB];
    unsigned long long tfull[2], tempty[2];
    unsigned long long drain[ISSUERS];
    unsigned int tmem_base;
    volatile int abort;
    long long rowoff[BM];
    long long coloff[BN];   // -1 for columns beyond N
    int eA[BM];
    int eB[BN];
    float stage[EPI_WARPS][32][17];
};
constexpr size_t SMEM_BYTES = 1024 + TILE_SMEM + sizeof(SmemCtl);

struct Params {
    int M, N, K;
    long long rowA0, rowB0;
    const int* eA; const int* eB;
    int scale_base, beta, nslices;
    int ngroups;
    int glo[kMaxGroups], gn[kMaxGroups], gkc[kMaxGroups];
    int epi, fixF;
    int ksplit, kper;            // K split: CTA split s owns [s*kper, min(K, (s+1)*kper))
    long long tri_rdiv, tri_cdiv;  // triangular tile skip (0 = off)
    int tiles_m, tiles_n, group_m;
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
    d |= (addr >> 4) & 0x3fffull;                 // start address
    d |= (unsigned long long)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (unsigned long long)(1024 >> 4) << 32;   // stride byte offset: 8 rows x 128 B
    d |= (unsigned long long)1 << 46;             // version
    d |= (unsigned long long)2 << 61;             // SWIZZLE_128B
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

// 32 lanes x 16 columns of TMEM into registers (no wait: pair with tmem_wait_ld).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Fire-and-forget int64 store / add for the fixed-point epilogue: no result, no ordering with
// other memory operations, so the 16 of a sub-chunk issue back to back.
__device__ __forceinline__ void st_cg_s64(long long* p, long long x)
{
    asm volatile("st.global.cg.s64 [%0], %1;" ::"l"(p), "l"(x));
}
__device__ __forceinline__ void red_add_u64(long long* p, long long x)
{
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(x));
}

__device__ __forceinline__ double pow2(int e)
{
    e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Pass sequence shared by all roles: groups in order, each cut into K-chunks, over
// this CTA's K range [kbeg, kend).
struct PassIter {
    int g, k0, k1, idx, kbeg, kend;
    __device__ int chunk_end(const Params& p, int from) const
    {
        const int kc = p.gkc[g];
        return (kc > 0 && from + kc < kend) ? from + kc : kend;
    }
    __device__ void begin(const Params& p, int split)
    {
        kbeg = split * p.kper;
        kend = min(p.K, kbeg + p.kper);
        g = 0; k0 = kbeg; k1 = chunk_end(p, kbeg); idx = 0;
    }
    __device__ bool next(const Params& p)
    {
        ++idx;
        if (k1 < kend) { k0 = k1; k1 = chunk_end(p, k0); return true; }
        if (++g >= p.ngroups) return false;
        k0 = kbeg;
        k1 = chunk_end(p, kbeg);
        return true;
    }
    __device__ bool last(const Params& p) const { return k1 >= kend && g == p.ngroups - 1; }
    // slice index range whose products land in the group's levels
    __device__ void ranges(const Params& p, int& lo, int& hi) const
    {
        const int L1 = p.glo[g], L2 = p.glo[g] + p.gn[g] - 1, s1 = p.nslices - 1;
        lo = L1 - s1 > 0 ? L1 - s1 : 0;
        hi = L2 < s1 ? L2 : s1;
    }
};

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* aring = base;                      // NA x A_TILE
    unsigned char* bring = base + NA * A_TILE;        // NB x B_TILE
    SmemCtl* ctl = (SmemCtl*)(base + TILE_SMEM);

    constexpr int KSTEP = KIND == TC_BF16 ? 64 : 32;  // K elements per 128-byte row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // grouped raster: consecutive CTAs walk group_m M-tiles before the next N-tile
    const int per_group = p.group_m * p.tiles_n;
    const int ntiles = p.tiles_m * p.tiles_n;            // tiles per K split
    const int split = (int)blockIdx.x / ntiles;          // this CTA's K split
    const int t = (int)blockIdx.x % ntiles;
    const int first_m = (t / per_group) * p.group_m;
    const int gm = min(p.tiles_m - first_m, p.group_m);
    const int m0 = (first_m + (t % per_group) % gm) * BM;
    const int n0 = ((t % per_group) / gm) * BN;
    // triangular skip: every element of the tile has b(n) < a(m), so nothing of it is
    // needed; leave before any barrier or TMEM is touched
    if (p.tri_rdiv > 0) {
        const long long nmax = min((long long)p.N - 1, (long long)n0 + BN - 1);
        if (nmax / p.tri_cdiv < (long long)m0 / p.tri_rdiv) return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; ++s) { mbar_init(&ctl->afull[s], 1); mbar_init(&ctl->aempty[s], ISSUERS); }
        for (int s = 0; s < NB; ++s) { mbar_init(&ctl->bfull[s], 1); mbar_init(&ctl->bempty[s], ISSUERS); }
        for (int b = 0; b < 2; ++b) { mbar_init(&ctl->tfull[b], 1); mbar_init(&ctl->tempty[b], EPI_WARPS); }
        for (int q = 0; q < ISSUERS; ++q) mbar_init(&ctl->drain[q], 1);
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
        ctl->coloff[c] = (n < p.N) ? map2(p.out.cmap, n) : -1;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // Per K-step: for j = lo..hi, first the A tiles (in order i = hi..lo) down to
        // the lowest i that B_j needs, then B_j.
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
            long long a_issued = 0, b_issued = 0;
            bool ok = true;
            PassIter it;
            it.begin(p, split);
            do {
                int lo, hi;
                it.ranges(p, lo, hi);
                const int L1 = p.glo[it.g];
                for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                    int a_here = 0;
                    for (int j = lo; j <= hi && ok; ++j) {
                        const int imin = L1 - j > lo ? L1 - j : lo;
                        while (a_here < hi - imin + 1) {
                            const int as = (int)(a_issued & (NA - 1));
                            const uint32_t par = (uint32_t)(((a_issued / NA) & 1) ^ 1);
                            if (!mbar_try(&ctl->aempty[as], par) &&
                                !mbar_wait(&ctl->aempty[as], par, ctl, p.status, p.wait_ns)) {
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(&ctl->afull[as], A_TILE);
                            tma_load_3d(aring + as * A_TILE, &tmA, &ctl->afull[as], kb, (int)(p.rowA0 + m0), hi - a_here);
                            ++a_issued;
                            ++a_here;
                        }
                        if (!ok) break;
                        const int bs = (int)(b_issued & (NB - 1));
                        const uint32_t bpar = (uint32_t)(((b_issued / NB) & 1) ^ 1);
                        if (!mbar_try(&ctl->bempty[bs], bpar) &&
                            !mbar_wait(&ctl->bempty[bs], bpar, ctl, p.status, p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&ctl->bfull[bs], B_TILE);
                        tma_load_3d(bring + bs * B_TILE, &tmB, &ctl->bfull[bs], kb, (int)(p.rowB0 + n0), j);
                        ++b_issued;
                    }
                }
            } while (ok && it.next(p));
            if (!ok) {
                // drain: the newest copy into each A slot and each B slot may still be in flight
                for (long long q = 1; q <= (a_issued < NA ? a_issued : NA); ++q) {
                    const long long u = a_issued - q;
                    mbar_drain_wait(&ctl->afull[u % NA], (uint32_t)((u / NA) & 1), p.status);
                }
                for (long long q = 1; q <= (b_issued < NB ? b_issued : NB); ++q) {
                    const long long u = b_issued - q;
                    mbar_drain_wait(&ctl->bfull[u % NB], (uint32_t)((u / NB) & 1), p.status);
                }
            }
        }
    } else if (warp <= ISSUERS) {
        // ----------------------------------------------------------------- MMA
        // Two issuing warps: issuing one tcgen05.mma costs the issuing thread about half
        // of the MMA's own duration and the hardware queue is shallow, so a single issuer
        // with per-tile barrier bookkeeping leaves the tensor pipe idle.  In a two-level
        // pass issuer `me` owns level L1+me and its accumulator; both walk the same tile
        // sequence, wait for the same tiles and release every slot (arrival count 2), so
        // neither can run a phase ahead of the other.  In a one-level pass issuer 0 does
        // all MMAs and issuer 1 only paces and releases.  Bookkeeping stays in registers;
        // slot descriptors are slot 0's plus an offset; barrier tests take an inline fast path.
        if (lane == 0) {
            const int me = warp - 1;
            const uint32_t idesc = instr_desc<KIND>();
            // slot q's descriptor = slot 0's + q * tile_bytes / 16 in the start-address field
            // (shared addresses stay below 256 KB, so the 14-bit field never carries over)
            const unsigned long long adesc0 = smem_desc(aring), bdesc0 = smem_desc(bring);
            uint32_t a_used = 0, b_used = 0;
            uint32_t tuse0 = 0, tuse1 = 0;
            int toggle = 0;
            bool ok = true, any = false;
            PassIter it;
            it.begin(p, split);
            do {
                int lo, hi;
                it.ranges(p, lo, hi);
                const int L1 = p.glo[it.g], nl = p.gn[it.g], L2 = L1 + nl - 1;
                const bool active = me < nl;
                const int buf = nl == 2 ? me : toggle;
                if (nl == 1) toggle ^= 1;
                const int mylevel = L1 + me;
                if (active) {
                    const uint32_t par = ((buf ? tuse1 : tuse0) & 1) ^ 1;
                    if (!mbar_try(&ctl->tempty[buf], par) && !mbar_wait(&ctl->tempty[buf], par, ctl, p.status, p.wait_ns))
                        ok = false;
                }
                if (!ok) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                uint32_t acc = 0;
                for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                    int a_wait = 0, a_free = 0;  // A tiles of this K-step waited for / released (i = hi - index)
                    for (int j = lo; j <= hi; ++j) {
                        const int imin = L1 - j > lo ? L1 - j : lo;
                        while (a_wait < hi - imin + 1) {
                            const uint32_t u = a_used + (uint32_t)a_wait;
                            unsigned long long* bar = &ctl->afull[u & (NA - 1)];
                            const uint32_t par = (u / NA) & 1;
                            if (!mbar_try(bar, par) && !mbar_wait(bar, par, ctl, p.status, p.wait_ns)) {
                                ok = false;
                                break;
                            }
                            ++a_wait;
                        }
                        if (!ok) break;
                        const int bs = (int)(b_used & (NB - 1));
                        {
                            unsigned long long* bar = &ctl->bfull[bs];
                            const uint32_t par = (b_used / NB) & 1;
                            if (!mbar_try(bar, par) && !mbar_wait(bar, par, ctl, p.status, p.wait_ns)) {
                                ok = false;
                                break;
                            }
                        }
                        if (active) {
                            const unsigned long long bd = bdesc0 + ((unsigned long long)bs << 11);
                            // products of my level(s) with this B slice
                            const int i_hi = (nl == 2 ? mylevel : L2) - j < hi ? (nl == 2 ? mylevel : L2) - j : hi;
                            const int i_lo = (nl == 2 ? mylevel : L1) - j > lo ? (nl == 2 ? mylevel : L1) - j : lo;
                            for (int i = i_hi; i >= i_lo; --i) {
                                const unsigned long long ad =
                                    adesc0 + ((unsigned long long)((a_used + (uint32_t)(hi - i)) & (NA - 1)) << 10);
                                // four MMAs per 128-byte row: advance the start address by 32 bytes each
                                mma<KIND>(d, ad, bd, idesc, acc);
                                mma<KIND>(d, ad + 2, bd + 2, idesc, 1u);
                                mma<KIND>(d, ad + 4, bd + 4, idesc, 1u);
                                mma<KIND>(d, ad + 6, bd + 6, idesc, 1u);
                                acc = 1;
                                any = true;
                            }
                        }
                        mma_commit(&ctl->bempty[bs]);
                        ++b_used;
                        // release the A tiles no later B of this K-step needs: i > min(hi, L2 - j - 1)
                        const int keep = j < hi ? (L2 - j - 1 < hi ? L2 - j - 1 : hi) : lo - 1;
                        while (a_free < hi - keep) {
                            mma_commit(&ctl->aempty[(a_used + (uint32_t)a_free) & (NA - 1)]);
                            ++a_free;
                        }
                    }
                    if (!ok) break;
                    a_used += (uint32_t)(hi - lo + 1);
                }
                if (!ok) break;
                if (active) {
                    mma_commit(&ctl->tfull[buf]);
                    if (buf) ++tuse1; else ++tuse0;
                }
            } while (it.next(p));
            if (!ok && any) {
                mma_commit(&ctl->drain[me]);
                mbar_drain_wait(&ctl->drain[me], 0, p.status);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // Warp e = warp - 1 - ISSUERS may read TMEM lanes 32 (warp % 4) .. + 31 (rows row0..) and
        // owns columns half*128 .. +127 of the tile, in sub-chunks of 16 columns.  A sub-chunk
        // of one level is read lane = row, staged, and re-read lane = column: lane L handles
        // column cl = L % 16 of rows 2k + rp (rp = L / 16, k < 16).
        const int e = warp - 1 - ISSUERS;
        const int q4 = warp & 3;
        const int row0 = q4 * 32;
        const int half = e >> 2;
        const int cl = lane & 15, rp = lane >> 4;
        float(*stg)[17] = ctl->stage[e];
        // output row offsets of this lane's 16 rows (fixed for the CTA), kept in registers
        long long ro_reg[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) ro_reg[k] = ctl->rowoff[row0 + 2 * k + rp];
        uint32_t tuse0 = 0, tuse1 = 0;
        int toggle = 0;
        PassIter it;
        it.begin(p, split);
        bool ok = true;
        // one level of one sub-chunk, from registers r (lane = row) to a[k] = acc(row0 + 2k + rp, col + cl)
        auto transpose = [&](const uint32_t (&r)[16], float (&a)[16]) {
#pragma unroll
            for (int j = 0; j < 16; ++j) stg[lane][j] = __uint_as_float(r[j]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = stg[2 * k + rp][cl];
            __syncwarp();
        };
        do {
            const int L1 = p.glo[it.g], nl = p.gn[it.g];
            // buffer of level L1 + q is (q ? 1 : buf0)
            const int buf0 = nl == 2 ? 0 : toggle;
            const int nb = nl;
            const bool use0 = nl == 2 || buf0 == 0, use1 = nl == 2 || buf0 == 1;
            if (nl == 1) toggle ^= 1;
            if (use0 && !mbar_wait(&ctl->tfull[0], tuse0 & 1, ctl, p.status, p.wait_ns)) ok = false;
            if (ok && use1 && !mbar_wait(&ctl->tfull[1], tuse1 & 1, ctl, p.status, p.wait_ns)) ok = false;
            if (!ok) break;
            fence_after();
            const bool first = it.idx == 0, last = it.last(p);
            const uint32_t tl = tmem + ((uint32_t)row0 << 16);
            for (int sc = 0; sc < BN / 32; ++sc) {
                const int col = half * (BN / 2) + sc * 16;  // tile column of the sub-chunk
                const long long co = ctl->coloff[col + cl];
                const bool ncol = co >= 0;
                float a0[16], a1[16];
                uint32_t r0[16], r1[16];
                tmem_ld16(tl + (uint32_t)(buf0 * BN + col), r0);
                if (nb == 2) tmem_ld16(tl + (uint32_t)(BN + col), r1);
                tmem_wait_ld();
                transpose(r0, a0);
                if (nb == 2) transpose(r1, a1);
                if (p.epi != EPI_FP64_RMW) {
                    // exact int64 fixed point (2^-fixF of a level-0 unit); a level pair is combined
                    // as (acc_L1 * 2^beta + acc_L2) before the one shift to the fixed-point scale
                    long long X[16];
                    const int sh = p.fixF - p.beta * (L1 + nb - 1);
                    if (nb == 2) {
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            X[k] = ((long long)__float2int_rn(a0[k]) << p.beta) + (long long)__float2int_rn(a1[k]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k) X[k] = (long long)__float2int_rn(a0[k]);
                    }
                    if (sh >= 0) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) X[k] <<= sh;
                    } else {
                        const long long rnd = 1ll << (-sh - 1);
#pragma unroll
                        for (int k = 0; k < 16; ++k) X[k] = (X[k] + rnd) >> (-sh);
                    }
                    if (p.epi == EPI_FIXED64_RED || p.epi == EPI_FIXED64_ADD) {
                        // int64 result for a consumer that scales it: store (first pass of an
                        // unsplit tile), then add without reading
                        const bool store = first && p.epi == EPI_FIXED64_RED;
                        if (ncol) {
                            long long* cb = (long long*)(p.out.C + co);
                            if (store) {
#pragma unroll
                                for (int k = 0; k < 16; ++k)
                                    if (ro_reg[k] >= 0) st_cg_s64(cb + ro_reg[k], X[k]);
                            } else {
#pragma unroll
                                for (int k = 0; k < 16; ++k)
                                    if (ro_reg[k] >= 0) red_add_u64(cb + ro_reg[k], X[k]);
                            }
                        }
                        continue;
                    }
                    // all loads of the sub-chunk are issued before any store (no aliasing stalls)
                    if (!first) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const long long ro = ctl->rowoff[row0 + 2 * k + rp];
                            if (ro >= 0 && ncol) X[k] += __ldcg((const long long*)(p.out.C + ro + co));
                        }
                    }
                    const int eb = ctl->eB[col + cl] + p.scale_base - p.fixF;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int r = row0 + 2 * k + rp;
                        const long long ro = ctl->rowoff[r];
                        if (ro < 0 || !ncol) continue;
                        long long* dst = (long long*)(p.out.C + ro + co);
                        if (last) __stcg((double*)dst, (double)X[k] * pow2(ctl->eA[r] + eb));
                        else __stcg(dst, X[k]);
                    }
                } else {
                    // FP64 read-modify-write of 2^e * acc (both levels of a pair at once)
                    const bool store_only = first && !p.out.accumulate;
                    const int eb0 = ctl->eB[col + cl] + p.scale_base - p.beta * L1;
                    double old[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const long long ro = ctl->rowoff[row0 + 2 * k + rp];
                        old[k] = (!store_only && ro >= 0 && ncol) ? __ldcg(p.out.C + ro + co) : 0.0;
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int r = row0 + 2 * k + rp;
                        const long long ro = ctl->rowoff[r];
                        if (ro < 0 || !ncol) continue;
                        double val = (double)a0[k] * pow2(ctl->eA[r] + eb0);
                        if (nb == 2) val += (double)a1[k] * pow2(ctl->eA[r] + eb0 - p.beta);
                        __stcg(p.out.C + ro + co, old[k] + val);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) {
                if (use0) mbar_arrive(&ctl->tempty[0]);
                if (use1) mbar_arrive(&ctl->tempty[1]);
            }
            if (use0) ++tuse0;
            if (use1) ++tuse1;
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

// 3-D map over a slice stack [slices][rows][pitch] with extent K in the inner dim;
// box = one 128-byte swizzle atom of K by box_rows rows.
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

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    return n;
}

namespace {
__global__ void fixed_to_f64_kernel(int M, int N, const OutDesc out, const int* __restrict__ eA, long long rowA0,
                                    const int* __restrict__ eB, long long rowB0, int base, int zero)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const long long co = map2(out.cmap, n);
    const int en = (eB ? eB[rowB0 + n] : 0) + base;
    for (int m = blockIdx.y; m < M; m += gridDim.y) {
        double* dst = out.C + map2(out.rmap, m) + co;
        if (zero) {
            *(long long*)dst = 0;
        } else {
            const long long X = *(const long long*)dst;
            *dst = (double)X * pow2((eA ? eA[rowA0 + m] : 0) + en);
        }
    }
}
}  // namespace

cudaError_t zero_out(int M, int N, const OutDesc& out, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    fixed_to_f64_kernel<<<dim3((N + 255) / 256, M < 65535 ? M : 65535), 256, 0, s>>>(M, N, out, nullptr, 0, nullptr, 0,
                                                                                     0, 1);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fixed_to_f64(int M, int N, const OutDesc& out, const int* eA, long long rowA0, const int* eB,
                         long long rowB0, int base, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    fixed_to_f64_kernel<<<dim3((N + 255) / 256, M < 65535 ? M : 65535), 256, 0, s>>>(M, N, out, eA, rowA0, eB, rowB0,
                                                                                     base, 0);
    count_launch();
    return cudaGetLastError();
}

cudaError_t gemm_tc(const GemmTc& g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.K <= 0 || g.slices < 1 || g.slices > MAX_SLICES || g.ngroups < 1 || g.ngroups > kMaxGroups)
        return cudaErrorInvalidValue;
    const int kstep = g.kind == TC_BF16 ? 64 : 32;
    Params p{};
    p.M = g.M; p.N = g.N; p.K = g.K;
    p.rowA0 = g.rowA0; p.rowB0 = g.rowB0;
    p.eA = g.eA; p.eB = g.eB;
    p.scale_base = g.scale_base; p.beta = g.beta; p.nslices = g.slices;
    p.ngroups = g.ngroups;
    for (int i = 0; i < g.ngroups; ++i) {
        if (g.gn[i] < 1 || g.gn[i] > 2 || g.glo[i] < 0 || g.glo[i] + g.gn[i] - 1 > 2 * (g.slices - 1))
            return cudaErrorInvalidValue;
        if (g.gkc[i] < 0 || g.gkc[i] % kstep) return cudaErrorInvalidValue;
        p.glo[i] = g.glo[i]; p.gn[i] = g.gn[i]; p.gkc[i] = g.gkc[i];
    }
    if (g.epi != EPI_FP64_RMW && g.out.accumulate) return cudaErrorInvalidValue;
    p.epi = g.epi;
    p.fixF = g.fixF;
    p.ksplit = g.ksplit > 1 ? g.ksplit : 1;
    if (p.ksplit > 1 && g.epi != EPI_FIXED64_ADD) return cudaErrorInvalidValue;
    p.kper = (int)((((long long)g.K + p.ksplit - 1) / p.ksplit + kstep - 1) / kstep * kstep);
    for (int i = 0; i < g.ngroups; ++i)
        if (p.ksplit > 1 && g.gkc[i] != 0) return cudaErrorInvalidValue;
    if ((g.tri_rdiv > 0) != (g.tri_cdiv > 0) || g.tri_rdiv < 0) return cudaErrorInvalidValue;
    p.tri_rdiv = g.tri_rdiv;
    p.tri_cdiv = g.tri_cdiv;
    p.out = g.out;
    p.status = g.status;
    p.wait_ns = g.wait_ns;
    p.tiles_m = (g.M + BM - 1) / BM;
    p.tiles_n = (g.N + BN - 1) / BN;
    p.group_m = p.tiles_m < 8 ? p.tiles_m : 8;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.kind, g.K, g.pitchA, g.rowsA, g.slices, BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb, g.B, g.kind, g.K, g.pitchB, g.rowsB, g.slices, BN)) return cudaErrorInvalidValue;
    const long long nctas = (long long)p.tiles_m * p.tiles_n * p.ksplit;
    if (nctas > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(gemm_tc_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        cudaFuncSetAttribute(gemm_tc_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    });
    cudaError_t err;
    if (g.kind == TC_BF16)
        err = (gemm_tc_kernel<TC_BF16><<<(unsigned)nctas, THREADS, SMEM_BYTES, s>>>(ma, mb, p), cudaGetLastError());
    else
        err = (gemm_tc_kernel<TC_TF32><<<(unsigned)nctas, THREADS, SMEM_BYTES, s>>>(ma, mb, p), cudaGetLastError());
    if (err != cudaSuccess) return err;
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
