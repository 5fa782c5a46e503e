// gemm_tc.cu -- Blackwell (sm_103a) tensor-core GEMM for the emulated-FP64
// (Ozaki, BF16 slices) and mixed-precision (BF16 / TF32) modes.
//
//   C[rmap(m) + cmap(n)] (= or +=) sum_levels 2^(eA[m] + eB[n] + base - beta*level)
//                                  * sum_{i+j=level} A_i(m,:) . B_j(n,:)
//
// Operands are K-major slice stacks D[slice][row][pitch].  One CTA per SM owns a
// 128 x 128 output tile at a time and issues tcgen05.mma.cta_group::1 (M = N = 128, 64 clocks
// of the tensor pipe each) into its tensor memory.  The kernel is persistent: every CTA takes
// (tile, K-split) items from a global counter, in raster order.  (Pairs of SMs on one 256-row
// tile, cta_group::2, were measured slower here: every slot of the operand rings then waits for
// handshakes between the two SMs, which cut the copy throughput per SM to about a third, and this
// GEMM streams about one operand tile per slice product.)
//
// Passes.  The slice-product levels L (products A_i B_j with i + j = L) are
// processed in groups of at most two; a "pass" is one group over one K-chunk, and
// each level of the pass accumulates in FP32 in its own 128-column TMEM region.
// Two such buffers (2 x 2 x 128 = all 512 columns) alternate between passes, so
// the epilogue drains pass p while the MMAs of pass p + 1 run.
//
// Exactness of the emulated mode.  Slices are balanced base-2^7 digits, |d| <= 64,
// so one product is at most 2^12 in magnitude and a level with q products per K
// element grows by at most q * 2^12 per element.  A pass covers at most
// 4096 / q K elements of its levels (the host chooses the chunks), so every
// partial FP32 sum is an integer below 2^24 and exact, whatever the input.  The
// epilogue converts each pass exactly to a signed 64-bit fixed-point number
// (2^-fixF of a level-0 unit; a level pair as acc_L1 * 2^beta + acc_L2) and adds
// it to a running sum held in the epilogue threads' registers: 128 x 128 int64
// per CTA, one row and 64 columns per thread.  The sum is written once per item:
// scaled to FP64 (final outputs, = or +=), stored as int64 (intermediates, whose
// consumer applies the exponents), or added with red.global (K split across pairs).
// In the mixed modes the running sum is FP64.
//
// Operand reuse: for every K-step (64 bf16 / 32 tf32 elements = one 128-byte
// swizzle atom per row) each slice tile a pass needs is loaded once.  The B
// slices stream in order j = lo..hi through a ring; the A slices arrive in order
// i = hi..lo through a FIFO, so B_j meets every A_i with i + j in the pass while
// A_i lives only until its last partner has passed.
//
// Roles (512 threads, four warpgroups): warps 0, 4 (A slices) and 3, 7 (B slices) are TMA
// producers, each issuing every other copy of its operand -- one thread keeps only about one
// copy in flight per 0.3 us (measured), fewer than the tensor pipe consumes.  Warps 1 (A) and
// 5 (B) wait for the copies to land and publish per-operand counts in shared memory; one
// thread of warp 2 issues all MMAs and slot releases (warp 2 also allocates TMEM), reading
// those counts instead of testing a barrier per tile -- a barrier test stalls the issuing
// thread for about as long as two MMAs take, which with per-tile tests kept the tensor pipe
// busy only about a third of the time (measured).  Warp 6 idles; warps 8-15 are the epilogue
// (two per TMEM lane quarter).  setmaxnreg moves registers from warpgroups 0-1 to the
// epilogue warpgroups, which hold the running sums.
//
// Every mbarrier wait is bounded (globaltimer); on expiry the CTA raises a
// shared abort flag and the device status word, drains what it has in flight
// (with a fixed bound), frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int BM = 128;                        // output rows per tile
constexpr int BN = 128;                        // output columns per tile
constexpr int ROW_BYTES = 128;                 // K bytes per tile row: one 128-byte swizzle atom
constexpr int A_TILE = BM * ROW_BYTES;         // 16 KB per A slice tile
constexpr int B_TILE = BN * ROW_BYTES;         // 16 KB per B slice tile
constexpr int NS = 6;                          // ring slots per operand
constexpr int TILE_SMEM = NS * (A_TILE + B_TILE);  // 192 KB
constexpr int MAX_SLICES = 8;
constexpr int QN = 8;                          // item queue slots
constexpr int kCounterSlots = 64;              // item counters, one per launch in flight
constexpr int EPI_WARPS = 8;                   // two per TMEM lane quarter
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int THREADS = 32 * 8 + EPI_THREADS;  // 512: producers, waiters and MMA issuer, then the epilogue
constexpr int TMEM_COLS = 512;                 // 2 buffers x 2 levels x BN columns
constexpr int COLS_PER_THREAD = BN / 2;        // 64 accumulator columns per epilogue thread
// setmaxnreg split of the 512 x 128 registers of the launch: warpgroups 0-1 (producers, waiters,
// MMA issuer) keep 64, the two epilogue warpgroups (running sums) get 192: 256 * 64 + 256 * 192 = 512 * 128.
constexpr int REG_LAUNCH = 128, REG_LOW = 64, REG_HIGH = 192;
// Warp roles.  A warp runs on SM sub-partition warp % 4: the MMA issuer (warp 2) shares its
// sub-partition only with the idle warp 6 and two epilogue warps, not with a producer or a
// waiter (that measured 3-4% faster).  Producers: warps 0, 4 (A slices) and 3, 7 (B slices).
constexpr int WARP_WAIT_A = 1, WARP_WAIT_B = 5, WARP_MMA = 2;
static_assert(256 * REG_LOW + 256 * REG_HIGH <= THREADS * REG_LAUNCH, "register split exceeds the launch's share");
constexpr unsigned long long kDrainLimitNs = 1000000000ull;  // bound on the abort-path drains

enum OutKind { OUT_F64 = 0, OUT_I64 = 1, OUT_I64_RED = 2 };

__device__ int g_item_counter[kCounterSlots];  // see the item schedule below

struct SmemCtl {
    unsigned long long afull[NS], bfull[NS];
    unsigned long long empty[NS];              // slot s of both rings released
    unsigned long long tfull[2], tempty[2];
    unsigned long long drain;
    unsigned int ready_a;                      // A tiles landed, in sequence order
    unsigned int ready_braw;                   // B tiles landed, in sequence order
    unsigned int ready_b;                      // B tiles landed with every A tile they meet
    volatile int item_q[QN];                   // this CTA's items in order (-1: no work left)
    unsigned int items_pub;                    // items written to item_q
    unsigned int items_done;                   // items the epilogue has finished
    volatile int epi_item;                     // the epilogue's current item, shared at its first epi_sync
    unsigned int tmem_base;
    volatile int abort;
    long long coloff[BN];                      // -1 for columns beyond N
    int eB[BN];
};
constexpr size_t SMEM_BYTES = 1024 + TILE_SMEM + sizeof(SmemCtl);
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

struct Params {
    int M, N, K;
    long long rowA0, rowB0;
    const int* eA; const int* eB;
    int scale_base, beta, nslices;
    int ngroups;
    int glo[kMaxGroups], gn[kMaxGroups], gkc[kMaxGroups];
    int out_kind, fixF;
    int ksplit, kper;              // K split: item split s owns [s*kper, min(K, (s+1)*kper))
    long long tri_rdiv, tri_cdiv;  // triangular tile skip (0 = off)
    int tiles_m, tiles_n, group_m, nitems;
    int* counter;                  // next item to hand out (zero at launch)
    OutDesc out;
    int* status;
    unsigned long long wait_ns;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
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
// or another role has aborted.  Inlined: code under setmaxnreg calls no functions.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, SmemCtl* ctl, int* status,
                                       unsigned long long limit_ns)
{
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtime();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(b, parity)) return true;
        // (each failed try_wait has already suspended the thread for a while)
        if (it == 1 || (it & 7) == 0) {
            if (ctl->abort) return false;
            if (gtime() - t0 > limit_ns) {
                ctl->abort = 1;
                atomicOr(status, kStatusWaitExpired);
                return false;
            }
        }
    }
}

__device__ __forceinline__ bool wait_fast(unsigned long long* b, uint32_t parity, SmemCtl* ctl, const Params& p)
{
    return mbar_try(b, parity) || mbar_wait(b, parity, ctl, p.status, p.wait_ns);
}

// Wait used only on the abort path: fixed bound, ignores the abort flag.
__device__ __forceinline__ void mbar_drain_wait(unsigned long long* b, uint32_t parity, int* status)
{
    const unsigned long long t0 = gtime();
    while (!mbar_try(b, parity)) {
        if (gtime() - t0 > kDrainLimitNs) { atomicOr(status, kStatusDrainExpired); return; }
    }
}

__device__ __forceinline__ void publish(unsigned int* ctr, unsigned int v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(ctr)), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int observe(unsigned int* ctr)
{
    unsigned int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(ctr)) : "memory");
    return v;
}

// Tile `idx` of a sequence has landed once the published count exceeds it.  `known` caches
// the last count read, so the common case costs one register compare; a miss spins on the
// shared counter with the same bound and abort check as the barrier waits.
template <bool BACKOFF = false>
__device__ __forceinline__ bool landed(unsigned int* ctr, uint32_t idx, uint32_t& known, SmemCtl* ctl, const Params& p)
{
    if ((int)(known - idx) > 0) return true;
    known = observe(ctr);
    if ((int)(known - idx) > 0) return true;
    const unsigned long long t0 = gtime();
    for (unsigned it = 1;; ++it) {
        if (BACKOFF) __nanosleep(32);  // a waiter's spin yields issue slots to its sub-partition
        known = observe(ctr);
        if ((int)(known - idx) > 0) return true;
        if ((it & 15) == 0) {
            if (ctl->abort) return false;
            if (gtime() - t0 > p.wait_ns) {
                ctl->abort = 1;
                atomicOr(p.status, kStatusWaitExpired);
                return false;
            }
        }
    }
}

// Bounded spin until the shared count *ctr exceeds `v` (sleeping between looks: the caller is
// not on the critical path); false on expiry or abort.
__device__ __forceinline__ bool await_count(unsigned int* ctr, uint32_t v, SmemCtl* ctl, const Params& p)
{
    if ((int)(observe(ctr) - v) > 0) return true;
    const unsigned long long t0 = gtime();
    for (unsigned it = 1;; ++it) {
        __nanosleep(64);
        if ((int)(observe(ctr) - v) > 0) return true;
        if ((it & 15) == 0) {
            if (ctl->abort) return false;
            if (gtime() - t0 > p.wait_ns) {
                ctl->abort = 1;
                atomicOr(p.status, kStatusWaitExpired);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
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
// both K-major, N = BN, M = BM.
template <int KIND>
__device__ __forceinline__ uint32_t instr_desc()
{
    const uint32_t fmt = KIND == TC_BF16 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         uint32_t idesc, uint32_t accumulate)
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

// Arrive on `bar` once this thread's prior MMAs complete.
__device__ __forceinline__ void mma_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 8 columns.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Pins 8 running sums at this point of the instruction stream: their updates cannot sink
// below the next (volatile) TMEM load, so one chunk's loaded values die before the next
// chunk's arrive and the sums plus one chunk fit the epilogue's registers.
template <typename T>
__device__ __forceinline__ void pin8(T* x)
{
    static_assert(sizeof(T) == 8, "8-byte sums");
    long long* v = reinterpret_cast<long long*>(x);
    asm volatile("" : "+l"(v[0]), "+l"(v[1]), "+l"(v[2]), "+l"(v[3]), "+l"(v[4]), "+l"(v[5]), "+l"(v[6]), "+l"(v[7]));
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

// Epilogue-only named barrier (the 256 epilogue threads).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory"); }

// Work item i: K split i / (tiles_m tiles_n), tile i % (tiles_m tiles_n), rastered in groups
// of group_m tile rows so that the items resident at once share A and B tiles in L2.
struct Item {
    int split, m0, n0;
    bool skip;
};

__device__ __forceinline__ Item item_of(const Params& p, int i)
{
    const int ntiles = p.tiles_m * p.tiles_n;
    const int t = i % ntiles;
    const int per_group = p.group_m * p.tiles_n;
    const int first_m = (t / per_group) * p.group_m;
    const int gm = min(p.tiles_m - first_m, p.group_m);
    Item it;
    it.split = i / ntiles;
    it.m0 = (first_m + (t % per_group) % gm) * BM;
    it.n0 = ((t % per_group) / gm) * BN;
    // triangular skip: every element of the tile has b(n) < a(m)
    it.skip = false;
    if (p.tri_rdiv > 0) {
        const long long nmax = min((long long)p.N - 1, (long long)it.n0 + BN - 1);
        it.skip = nmax / p.tri_cdiv < (long long)it.m0 / p.tri_rdiv;
    }
    return it;
}

// Items are handed out in order from a global counter, one at a time to whichever CTA asks
// next, so that the items resident at once stay a contiguous run of the raster and share
// their operand tiles in L2.  (A fixed stride of items per CTA let the CTAs drift apart over
// thousands of items: a 42000 x 160000 x 2000 GEMM then read about 1.9 TB from HBM.)  One
// producer thread fetches; every role reads the items from a queue in shared memory.

// The fetching thread's item k: -1 when no work is left (or on abort).  Slot k % QN is
// reused only after the epilogue, the last role to read the queue, has finished item k - QN.
__device__ __forceinline__ int fetch_item(SmemCtl* ctl, const Params& p, uint32_t k)
{
    int item = -1;
    if (k < QN || await_count(&ctl->items_done, k - QN, ctl, p)) {
        do {
            item = atomicAdd(p.counter, 1);
        } while (item < p.nitems && item_of(p, item).skip);
        if (item >= p.nitems) item = -1;
    }
    ctl->item_q[k % QN] = item;
    publish(&ctl->items_pub, k + 1);
    return item;
}

// Item k of this CTA for the other roles (-1: no work left, or abort).
__device__ __forceinline__ int item_at(SmemCtl* ctl, const Params& p, uint32_t k)
{
    if (!await_count(&ctl->items_pub, k, ctl, p)) return -1;
    return ctl->item_q[k % QN];
}

// Pass sequence of one item shared by all roles: groups in order, each cut into
// K-chunks, over the item's K range [kbeg, kend).
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

// MMA issuer state carried across K-steps and passes.
struct IssueState {
    unsigned long long adesc0, bdesc0;  // descriptors of ring slot 0
    uint32_t idesc, d0, fresh;          // instruction descriptor, pass buffer, levels not yet written
    uint32_t used;                      // tiles of either operand consumed so far (the counts agree)
    uint32_t slot0;                     // ring slot of the current K-step's first tile (= used % NS)
    uint32_t known_a, known_braw, known_b;  // last landed counts read
};

__device__ __forceinline__ uint32_t slot_add(uint32_t a, int k)  // (a + k) % NS for a < NS, k <= 2 NS
{
    uint32_t r = a + (uint32_t)k;
    r = r >= (uint32_t)NS ? r - NS : r;
    return r >= (uint32_t)NS ? r - NS : r;
}

// One K-step of a pass over levels L1 = hi - nl + 1 .. hi, slices 0 .. hi (the host admits no
// level above slices - 1, so every pass has this shape).  B_j meets A_i for each level L of the
// pass (i = L - j).  The A tiles arrive in order i = hi .. 0, so A tile number j (slice hi - j)
// is last used with B_j: both tiles number j of the K-step sit in the same ring slot and leave
// with one commit.  HI >= 0 fixes the shape at compile time (the loops unroll and the slot
// arithmetic folds -- with the shape at run time the issuing thread, not the tensor pipe, set
// the pace); HI < 0 takes any shape at run time.
template <int KIND, int HI, int NL>
__device__ __forceinline__ bool issue_kstep(IssueState& st, int hi_rt, int nl_rt, SmemCtl* ctl, const Params& p)
{
    const int hi = HI >= 0 ? HI : hi_rt;
    const int nl = HI >= 0 ? NL : nl_rt;
    const int L1 = hi - nl + 1;
#pragma unroll
    for (int j = 0; j <= hi; ++j) {
        const uint32_t idx = st.used + (uint32_t)j;
        const int imin = L1 - j > 0 ? L1 - j : 0;  // lowest A slice that B_j meets
        if ((int)(st.known_b - idx) <= 0) {
            st.known_b = observe(&ctl->ready_b);
            if ((int)(st.known_b - idx) <= 0) {
                // late tiles: watch the two raw counts, not the combined one, which would add
                // the second waiter's reaction to every late A tile
                if (!landed(&ctl->ready_a, st.used + (uint32_t)(hi - imin), st.known_a, ctl, p) ||
                    !landed(&ctl->ready_braw, idx, st.known_braw, ctl, p))
                    return false;
            }
            fence_after();
        }
        const uint32_t bs = slot_add(st.slot0, j);
        const unsigned long long bd = st.bdesc0 + (unsigned long long)bs * (B_TILE >> 4);
#pragma unroll
        for (int lv = 0; lv < nl; ++lv) {
            const int i = L1 + lv - j;
            if (i < 0 || i > hi) continue;
            const unsigned long long ad = st.adesc0 + (unsigned long long)slot_add(st.slot0, hi - i) * (A_TILE >> 4);
            const uint32_t d = st.d0 + (uint32_t)(lv * BN);
            // four MMAs per 128-byte row: advance the start address by 32 bytes each
            mma<KIND>(d, ad, bd, st.idesc, ((st.fresh >> lv) & 1u) ^ 1u);
            mma<KIND>(d, ad + 2, bd + 2, st.idesc, 1u);
            mma<KIND>(d, ad + 4, bd + 4, st.idesc, 1u);
            mma<KIND>(d, ad + 6, bd + 6, st.idesc, 1u);
            st.fresh &= ~(1u << lv);
        }
        mma_commit(&ctl->empty[bs]);
    }
    st.used += (uint32_t)(hi + 1);
    st.slot0 = slot_add(st.slot0, hi + 1);
    return true;
}

template <int KIND, int HI, int NL>
__device__ __forceinline__ bool issue_pass(IssueState& st, int nk, int hi, int nl, SmemCtl* ctl, const Params& p)
{
    for (int k = 0; k < nk; ++k)
        if (!issue_kstep<KIND, HI, NL>(st, hi, nl, ctl, p)) return false;
    return true;
}

template <int KIND, bool FIXED>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* aring = base;                      // NS x A_TILE
    unsigned char* bring = base + NS * A_TILE;        // NS x B_TILE
    SmemCtl* ctl = (SmemCtl*)(base + TILE_SMEM);

    constexpr int KSTEP = KIND == TC_BF16 ? 64 : 32;  // K elements per 128-byte row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&ctl->afull[s], 1);
            mbar_init(&ctl->bfull[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) { mbar_init(&ctl->tfull[b], 1); mbar_init(&ctl->tempty[b], EPI_WARPS); }
        mbar_init(&ctl->drain, 1);
        ctl->ready_a = 0;
        ctl->ready_b = 0;
        ctl->ready_braw = 0;
        ctl->items_pub = 0;
        ctl->items_done = 0;
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp < 8) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_LOW));
        const int prod = warp == 0 ? 0 : warp == 4 ? 1 : warp == 3 ? 2 : warp == 7 ? 3 : -1;
        if (prod >= 0 && lane == 0) {
            // -------------------------------------------------------- producers
            // Four producer threads (warps 0, 3: A slices; 4, 5: B slices), each issuing every
            // other copy of its operand: one thread keeps only about one copy in flight per 0.3 us,
            // which alone would starve the tensor pipe.  All walk the same sequence -- per K-step,
            // for j = lo..hi, the A tiles (i = hi..lo) down to the lowest i that B_j needs, then
            // B_j -- and count every copy of their operand.
            const bool isA = prod < 2;
            const long long mine = prod & 1;
            const CUtensorMap* map = isA ? &tmA : &tmB;
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)map) : "memory");
            const uint32_t tile = isA ? A_TILE : B_TILE;
            unsigned char* ring = isA ? aring : bring;
            unsigned long long* full = isA ? ctl->afull : ctl->bfull;
            unsigned long long* empty = ctl->empty;
            long long issued = 0;  // copies of this operand in the sequence so far (all producers')
            bool ok = true;
            auto load = [&](int kb, int row, int slice) -> bool {
                const long long u = issued++;
                if ((u & 1) != mine) return true;
                const int s = (int)(u % NS);
                if (!wait_fast(&empty[s], (uint32_t)(((u / NS) & 1) ^ 1), ctl, p)) return false;
                mbar_expect_tx(&full[s], tile);
                tma_load_3d(ring + s * tile, map, &full[s], kb, row, slice);
                return true;
            };
            // producer 0 fetches the items, item k + 1 as soon as item k starts, so that the
            // fetch (a global atomic) overlaps item k's copies
            int next = -1;
            for (uint32_t k = 0; ok; ++k) {
                const int item = prod == 0 ? (k == 0 ? fetch_item(ctl, p, 0) : next) : item_at(ctl, p, k);
                if (item < 0) break;
                if (prod == 0) next = fetch_item(ctl, p, k + 1);
                const Item w = item_of(p, item);
                const int rowA = (int)(p.rowA0 + w.m0), rowB = (int)(p.rowB0 + w.n0);
                PassIter it;
                it.begin(p, w.split);
                do {
                    int lo, hi;
                    it.ranges(p, lo, hi);
                    const int L1 = p.glo[it.g];
                    for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                        int a_here = 0;
                        for (int j = lo; j <= hi && ok; ++j) {
                            const int imin = L1 - j > lo ? L1 - j : lo;
                            for (; a_here < hi - imin + 1 && ok; ++a_here)
                                if (isA) ok = load(kb, rowA, hi - a_here);
                            if (ok && !isA) ok = load(kb, rowB, j);
                        }
                    }
                } while (ok && it.next(p));
            }
            if (ok) {
                // tail: the last use of every slot this producer filled is released, so no commit
                // still targets the barriers when the CTA leaves
                for (long long u = issued - 1; u >= 0 && u >= issued - NS && ok; --u)
                    if ((u & 1) == mine) ok = wait_fast(&empty[u % NS], (uint32_t)((u / NS) & 1), ctl, p);
            }
            if (!ok) {
                // the newest copy into each of its slots may still be in flight
                for (long long u = issued - 1; u >= 0 && u >= issued - NS; --u)
                    if ((u & 1) == mine) mbar_drain_wait(&full[u % NS], (uint32_t)((u / NS) & 1), p.status);
            }
        } else if (warp == WARP_WAIT_A && lane == 0) {
            // ------------------------------------------------------------ waiters
            // Two threads wait for the copies to land and publish counts in shared memory; the
            // MMA issuer then compares one shared count per B tile instead of testing barriers:
            // a barrier test blocks the issuing thread for about 70 ns, as long as two of its
            // MMAs take, and per-tile tests left the tensor pipe idle most of the time.  This one
            // counts the A tiles landed, in sequence order.
            uint32_t u = 0;  // A tiles waited for
            bool ok = true;
            for (uint32_t k = 0; ok; ++k) {
                const int item = item_at(ctl, p, k);
                if (item < 0) break;
                uint32_t end = u;  // the item's A tiles (as many as its B tiles)
                PassIter it;
                it.begin(p, item_of(p, item).split);
                do {
                    int lo, hi;
                    it.ranges(p, lo, hi);
                    end += (uint32_t)((it.k1 - it.k0 + KSTEP - 1) / KSTEP) * (uint32_t)(hi - lo + 1);
                } while (it.next(p));
                for (; u < end && ok; ++u) {
                    ok = wait_fast(&ctl->afull[u % NS], (u / NS) & 1, ctl, p);
                    if (ok) publish(&ctl->ready_a, u + 1);
                }
            }
        } else if (warp == WARP_WAIT_B && lane == 0) {
            // The other counts the B tiles that have landed (raw) and those that have landed
            // together with every A tile they meet (the A count is the first thread's).  The
            // issuer compares the combined count once per B tile and reads the raw counts only
            // when tiles are late (one compare instead of two measured +9% where the issue loop
            // sets the pace).
            uint32_t nb = 0, a_done = 0, known_a = 0;  // B tiles published, A tiles of past K-steps
            bool ok = true;
            for (uint32_t k = 0; ok; ++k) {
                const int item = item_at(ctl, p, k);
                if (item < 0) break;
                PassIter it;
                it.begin(p, item_of(p, item).split);
                do {
                    int lo, hi;
                    it.ranges(p, lo, hi);
                    const int L1 = p.glo[it.g];
                    for (int kb = it.k0; kb < it.k1 && ok; kb += KSTEP) {
                        for (int j = lo; j <= hi && ok; ++j) {
                            const int imin = L1 - j > lo ? L1 - j : lo;  // lowest A slice B_j meets
                            ok = wait_fast(&ctl->bfull[nb % NS], (nb / NS) & 1, ctl, p);
                            if (ok) publish(&ctl->ready_braw, nb + 1);
                            ok = ok && landed<true>(&ctl->ready_a, a_done + (uint32_t)(hi - imin), known_a, ctl, p);
                            if (ok) publish(&ctl->ready_b, nb + 1);
                            ++nb;
                        }
                        a_done += (uint32_t)(hi - lo + 1);
                    }
                } while (ok && it.next(p));
            }
        } else if (warp == WARP_MMA && lane == 0) {
            // ------------------------------------------------------------ MMA
            // One issuing thread for both levels of a pass (accumulator columns lv * BN of the
            // pass's buffer).  It walks the producers' tile sequence, learns from the waiters'
            // counters which tiles have landed, and releases every slot with a commit once the
            // MMAs that read it are done.
            IssueState st;
            st.idesc = instr_desc<KIND>();
            // slot q's descriptor = slot 0's + q * tile_bytes / 16 in the start-address field
            // (shared addresses stay below 256 KB, so the 14-bit field never carries over)
            st.adesc0 = smem_desc(aring);
            st.bdesc0 = smem_desc(bring);
            st.used = 0;
            st.slot0 = 0;
            st.known_a = 0;
            st.known_braw = 0;
            st.known_b = 0;
            uint32_t npass = 0;
            bool ok = true, any = false;
            for (uint32_t k = 0; ok; ++k) {
                const int item = item_at(ctl, p, k);
                if (item < 0) break;
                PassIter it;
                it.begin(p, item_of(p, item).split);
                do {
                    int lo, hi;
                    it.ranges(p, lo, hi);  // lo = 0 and hi = the pass's top level
                    const int nl = p.gn[it.g];
                    const int buf = (int)(npass & 1);
                    const uint32_t use = npass >> 1;  // earlier passes on this buffer
                    if (!wait_fast(&ctl->tempty[buf], (use & 1) ^ 1, ctl, p)) { ok = false; break; }
                    fence_after();
                    st.d0 = tmem + (uint32_t)(buf * 2 * BN);
                    st.fresh = (1u << nl) - 1;
                    const int nk = (it.k1 - it.k0 + KSTEP - 1) / KSTEP;
                    switch (hi * 4 + nl) {  // the shapes the host builds for up to 8 slices
                        case 0 * 4 + 1: ok = issue_pass<KIND, 0, 1>(st, nk, hi, nl, ctl, p); break;
                        case 1 * 4 + 2: ok = issue_pass<KIND, 1, 2>(st, nk, hi, nl, ctl, p); break;
                        case 3 * 4 + 2: ok = issue_pass<KIND, 3, 2>(st, nk, hi, nl, ctl, p); break;
                        case 5 * 4 + 2: ok = issue_pass<KIND, 5, 2>(st, nk, hi, nl, ctl, p); break;
                        case 7 * 4 + 2: ok = issue_pass<KIND, 7, 2>(st, nk, hi, nl, ctl, p); break;
                        default: ok = issue_pass<KIND, -1, 0>(st, nk, hi, nl, ctl, p); break;
                    }
                    if (!ok) break;
                    any = true;
                    mma_commit(&ctl->tfull[buf]);
                    ++npass;
                } while (it.next(p));
            }
            if (ok) {
                // tail: both buffers' last drains are done
                for (uint32_t q = npass > 2 ? npass - 2 : 0; q < npass && ok; ++q)
                    ok = wait_fast(&ctl->tempty[q & 1], (q >> 1) & 1, ctl, p);
            }
            if (any) {
                // every MMA this thread issued has completed before TMEM is released
                mma_commit(&ctl->drain);
                mbar_drain_wait(&ctl->drain, 0, p.status);
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_HIGH));
        // ------------------------------------------------------------ epilogue
        // Warp e = warp - 8 reads TMEM lanes 32 (warp % 4) .. + 31 and owns columns
        // half * 64 .. + 63 of the tile: one output row and 64 columns per thread.
        const int e = warp - 8;
        const int q4 = warp & 3;
        const int row = q4 * 32 + lane;  // TMEM lane = row of this CTA's 128
        const int half = e >> 2;
        const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
        typedef typename std::conditional<FIXED, long long, double>::type acc_t;
        acc_t sum[COLS_PER_THREAD];
        uint32_t npass = 0;
        bool ok = true;
        // One thread reads each item from the queue and shares it at the item's first epi_sync,
        // so every epilogue warp walks the same items and meets every epi_sync even after an
        // abort (it then skips the waits and TMEM reads): no warp can be left at a named
        // barrier that a warp which gave up will never reach.
        for (uint32_t k = 0;; ++k) {
            if (e == 0 && lane == 0) {
                // this thread has finished items 0 .. k-1 (the queue slots are read once per item)
                if (k > 0) publish(&ctl->items_done, k);
                ctl->epi_item = item_at(ctl, p, k);
            }
            epi_sync();
            const int item = ctl->epi_item;
            if (item < 0) break;
            const Item w = item_of(p, item);
            // this item's output row and column tables (the previous item's writes are done)
            const int m = w.m0 + row;
            const long long ro = (m < p.M) ? map2(p.out.rmap, m) : -1;
            const int eAr = (p.eA && m < p.M) ? p.eA[p.rowA0 + m] : 0;
            epi_sync();
            for (int c = e * 32 + lane; c < BN; c += EPI_THREADS) {
                const int n = w.n0 + c;
                ctl->coloff[c] = (n < p.N) ? map2(p.out.cmap, n) : -1;
                ctl->eB[c] = (p.eB && n < p.N) ? p.eB[p.rowB0 + n] : 0;
            }
            epi_sync();
            PassIter it;
            it.begin(p, w.split);
            do {
                const int L1 = p.glo[it.g], nl = p.gn[it.g];
                const int buf = (int)(npass & 1);
                if (ok && !wait_fast(&ctl->tfull[buf], (npass >> 1) & 1, ctl, p)) ok = false;
                if (!ok) continue;  // (continue in a do-while goes to it.next())
                fence_after();
                const bool first = it.idx == 0;
                const int sh = p.fixF - p.beta * (L1 + nl - 1);
                const uint32_t tb = tl + (uint32_t)(buf * 2 * BN + half * COLS_PER_THREAD);
#pragma unroll
                for (int cc = 0; cc < COLS_PER_THREAD / 8; ++cc) {
                    uint32_t r0[8], r1[8];
                    tmem_ld8(tb + (uint32_t)(cc * 8), r0);
                    if (nl == 2) tmem_ld8(tb + (uint32_t)(BN + cc * 8), r1);
                    tmem_wait_ld();
                    if (cc == COLS_PER_THREAD / 8 - 1) {
                        // the buffer is read: hand it back to the MMA issuer
                        fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
                    }
                    if (FIXED) {
                        // exact int64 fixed point (2^-fixF of a level-0 unit); a level pair is combined
                        // as (acc_L1 * 2^beta + acc_L2) before the one shift to the fixed-point scale
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            long long X = (long long)__float2int_rn(__uint_as_float(r0[k]));
                            if (nl == 2) X = (X << p.beta) + (long long)__float2int_rn(__uint_as_float(r1[k]));
                            X = sh >= 0 ? (X << sh) : ((X + (1ll << (-sh - 1))) >> (-sh));
                            sum[cc * 8 + k] = first ? (acc_t)X : sum[cc * 8 + k] + (acc_t)X;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const double X = (double)__uint_as_float(r0[k]);
                            sum[cc * 8 + k] = first ? (acc_t)X : sum[cc * 8 + k] + (acc_t)X;
                        }
                    }
                    pin8(&sum[cc * 8]);
                }
                ++npass;
                if (it.last(p) && ro >= 0) {
                    // the item's result: one row, 64 columns of this thread
                    const int col0 = half * COLS_PER_THREAD;
                    double* Crow = p.out.C + ro;
                    const int ebase = eAr + p.scale_base - (FIXED ? p.fixF : 0);
#pragma unroll
                    for (int k0 = 0; k0 < COLS_PER_THREAD; k0 += 8) {
                        // eight columns at a time: keeps the table loads from being hoisted
                        // ahead of all stores (they would need more registers than the sums leave)
                        asm volatile("" ::: "memory");
#pragma unroll
                        for (int k = k0; k < k0 + 8; ++k) {
                            const long long co = ctl->coloff[col0 + k];
                            if (co < 0) continue;
                            if (p.out_kind == OUT_F64) {
                                const double val = (double)sum[k] * pow2(ebase + ctl->eB[col0 + k]);
                                Crow[co] = p.out.accumulate ? Crow[co] + val : val;
                            } else if (p.out_kind == OUT_I64) {
                                __stcg((long long*)(Crow + co), (long long)sum[k]);
                            } else {
                                red_add_u64((long long*)(Crow + co), (long long)sum[k]);
                            }
                        }
                    }
                }
            } while (it.next(p));
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == WARP_MMA) {
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

template <int KIND, bool FIXED>
cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, const Params& p, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int max_ctas = 0;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(gemm_tc_kernel<KIND, FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SMEM_BYTES);
        // persistent: as many CTAs as are resident on the device at once (one per SM)
        int per_sm = 0;
        if (attr_err != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_tc_kernel<KIND, FIXED>, THREADS, SMEM_BYTES) !=
                cudaSuccess ||
            per_sm <= 0) {
            cudaGetLastError();
            per_sm = 1;
        }
        max_ctas = per_sm * device_sm_count();
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int ctas = p.nitems < max_ctas ? p.nitems : max_ctas;
    gemm_tc_kernel<KIND, FIXED><<<ctas, THREADS, SMEM_BYTES, s>>>(ma, mb, p);
    return cudaGetLastError();
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
    const bool fixed = g.epi != EPI_FP64_RMW;
    Params p{};
    p.M = g.M; p.N = g.N; p.K = g.K;
    p.rowA0 = g.rowA0; p.rowB0 = g.rowB0;
    p.eA = g.eA; p.eB = g.eB;
    p.scale_base = g.scale_base; p.beta = g.beta; p.nslices = g.slices;
    p.ngroups = g.ngroups;
    for (int i = 0; i < g.ngroups; ++i) {
        // levels up to slices - 1 only: every pass then has the shape the MMA issuer assumes
        if (g.gn[i] < 1 || g.gn[i] > 2 || g.glo[i] < 0 || g.glo[i] + g.gn[i] - 1 > g.slices - 1)
            return cudaErrorInvalidValue;
        if (g.gkc[i] < 0 || g.gkc[i] % kstep) return cudaErrorInvalidValue;
        if (!fixed && g.gn[i] != 1) return cudaErrorInvalidValue;  // FP64 sums take one level per pass
        p.glo[i] = g.glo[i]; p.gn[i] = g.gn[i]; p.gkc[i] = g.gkc[i];
    }
    if ((g.epi == EPI_FIXED64_RED || g.epi == EPI_FIXED64_ADD) && g.out.accumulate) return cudaErrorInvalidValue;
    p.out_kind = g.epi == EPI_FIXED64_RED ? OUT_I64 : (g.epi == EPI_FIXED64_ADD ? OUT_I64_RED : OUT_F64);
    p.fixF = g.fixF;
    p.ksplit = g.ksplit > 1 ? g.ksplit : 1;
    if (p.ksplit > 1 && g.epi != EPI_FIXED64_ADD) return cudaErrorInvalidValue;
    p.kper = (int)((((long long)g.K + p.ksplit - 1) / p.ksplit + kstep - 1) / kstep * kstep);
    if ((long long)p.kper * (p.ksplit - 1) >= g.K) return cudaErrorInvalidValue;  // every split owns some K
    if ((g.tri_rdiv > 0) != (g.tri_cdiv > 0) || g.tri_rdiv < 0) return cudaErrorInvalidValue;
    p.tri_rdiv = g.tri_rdiv;
    p.tri_cdiv = g.tri_cdiv;
    p.out = g.out;
    p.status = g.status;
    p.wait_ns = g.wait_ns;
    p.tiles_m = (g.M + BM - 1) / BM;
    p.tiles_n = (g.N + BN - 1) / BN;
    p.group_m = p.tiles_m < 8 ? p.tiles_m : 8;
    const long long nitems = (long long)p.tiles_m * p.tiles_n * p.ksplit;
    // (the item counter runs past nitems by at most two per CTA)
    if (nitems > 0x7fffffffll - (1 << 20)) return cudaErrorInvalidConfiguration;
    p.nitems = (int)nitems;
    // item counter: a slot of a small ring (launches in flight on other streams take other
    // slots), zeroed in stream order before the launch
    static std::atomic<unsigned> next_slot{0};
    int* counters = nullptr;
    cudaError_t cerr = cudaGetSymbolAddress((void**)&counters, g_item_counter);
    if (cerr != cudaSuccess) return cerr;
    p.counter = counters + (next_slot.fetch_add(1) % kCounterSlots);
    cerr = cudaMemsetAsync(p.counter, 0, sizeof(int), s);
    if (cerr != cudaSuccess) return cerr;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.kind, g.K, g.pitchA, g.rowsA, g.slices, BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb, g.B, g.kind, g.K, g.pitchB, g.rowsB, g.slices, BN)) return cudaErrorInvalidValue;
    cudaError_t err;
    if (g.kind == TC_BF16)
        err = fixed ? launch<TC_BF16, true>(ma, mb, p, s) : launch<TC_BF16, false>(ma, mb, p, s);
    else
        err = fixed ? launch<TC_TF32, true>(ma, mb, p, s) : launch<TC_TF32, false>(ma, mb, p, s);
    if (err != cudaSuccess) return err;
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
