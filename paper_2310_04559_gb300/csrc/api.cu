// api.cu -- the C ABI of include/cc_ladder.h: argument validation, the planner
// (contraction order, block of `a` values, workspace carve), and the sequence of
// device steps for the forward, the adjoint and the pair energy.
//
// Forward, integral-first order (Section 3.2, the for-loop over `a` widened to
// blocks of A values):
//   for each block a0 .. a0+A-1:
//     KG1  V[a,b,c,d] = sum_P L[P,a,c] L[P,b,d]              (Eq. 5; GEMM M=A*v, N=v^2, K=n)
//     KG2  R[ij,a,b]  = sum_(c,d) t2[ij,c,d] V[a,b,c,d]       (Eq. 6; GEMM M=o^2, N=A*v, K=v^2)
// Forward, Cholesky-first order (Section 3.2, the L.t intermediate):
//     CF1  X[ij,a,P,d] = sum_c L[P,a,c] t2[ij,c,d]            (GEMM M=A*n, N=o^2*v, K=v)
//     CF2  R[ij,a,b]   = sum_(P,d) X[ij,a,P,d] L[P,b,d]        (GEMM M=o^2*A, N=v, K=n*v)
// Pair-symmetric amplitudes (CC_FLAG_SYMMETRIC_T), integral-first, tensor-core modes
// ("packed" path, pm.cu): since (ac|bd) = (bd|ac) for any L, a block only needs the
// integrals with b >= a (KG1 skips the tiles below that diagonal), and the ladder
// GEMM is done on the parts of t2 and of the integrals symmetric and antisymmetric
// under c <-> d, packed over c <= d:
//     KG1   V[al][b'][c][d], b = a0 + b' >= a                   (GEMM M=A*v, N=(v-a0)*v, K=n)
//     R+[i<=j][(a,b>=a)] = sum_{c<=d} T+[ij][cd] V+[ab][cd]      (GEMM M=o(o+1)/2, K=v(v+1)/2)
//     R-[i< j][(a,b>=a)] = sum_{c< d} T-[ij][cd] V-[ab][cd]      (GEMM M=o(o-1)/2, K=v(v-1)/2)
//     R[i,j,a,b] = R[j,i,b,a] = R+ + R-,  R[j,i,a,b] = R[i,j,b,a] = R+ - R-
// which issues about (n + o^2/2) v^4 multiply-adds instead of 2 (n + o(o+1)/2) v^4.
// In the emulated-FP64 and mixed modes every GEMM operand is first turned into
// a slice stack (split.cu, pm.cu) and the GEMM runs on the tensor cores (gemm_tc.cu);
// in the FP64 mode the GEMMs run on DMMA (gemm_f64.cu) straight from FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <utility>
#include <vector>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "cc_internal.cuh"

using namespace cc;

namespace {

constexpr int kDefaultSlices = 6;
constexpr int kBeta = 7;                 // bits per Ozaki slice (balanced digits in [-64, 64])
constexpr int kMixedChunk = 16384;       // K elements per FP32 accumulation in the BF16 / TF32 modes
constexpr int kFixF = 26;                // fixed-point fraction bits (of a level-0 unit) in the Ozaki epilogue
constexpr int kFixedBase = 2 - 2 * kBeta - kFixF;  // exponent of one fixed-point unit, before row/col exponents
constexpr size_t kDefaultBudget = 150ull << 30;

std::atomic<unsigned long long> g_wait_ns{2000000000ull};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
inline long long pitch_for(long long K, int esz) { const long long q = 16 / esz; return (K + q - 1) / q * q; }

struct Carve {
    size_t cur = 0;
    size_t take(size_t bytes)
    {
        const size_t o = cur;
        cur = al256(cur + bytes);
        return o;
    }
};

bool is_tc(int mode) { return mode == CC_OZAKI_BF16 || mode == CC_BF16 || mode == CC_TF32; }
int esz_of(int mode) { return mode == CC_TF32 ? 4 : 2; }
int slices_of(int mode, int slices) { return mode == CC_OZAKI_BF16 ? (slices > 0 ? slices : kDefaultSlices) : 1; }

struct Ctx {
    int o, v, n;
    int mode, order, flags, s;
    bool sym, exch;
    long long pairs;  // GEMM rows for (i,j)
    bool packed;      // pair-symmetric integral-first tensor-core path (R+ / R- over c <= d)
    long long pp, pm; // packed path: pairs i <= j and i < j
    long long Kp, Km; // packed path: v(v+1)/2 and v(v-1)/2
    bool host;        // t2 and R are page-locked host memory, read and written over the host link
    long long PB;     // packed path: pairs (i <= j) per pair block (o(o+1)/2 unless host)
    bool hostL;       // L is page-locked host memory, streamed to the device in chunks of Cholesky vectors
    long long PC;     // hostL: Cholesky vectors per chunk (n otherwise)
    int* status = nullptr;  // device status word of the call (the splits flag non-finite inputs there)
};

// Blocks of `a` values [a0, a0 + Ab) covering [alo, ahi).  Unpacked paths: Ab = P
// for every block.  Packed path: a block holds the integrals (a, b >= a0), so its
// size is Ab * (v - a0) rows; P bounds that product and blocks widen as a0 grows.
std::vector<std::pair<int, int>> block_list(const Ctx& c, long long P, int alo, int ahi, int forced)
{
    std::vector<std::pair<int, int>> out;
    for (int a0 = alo; a0 < ahi;) {
        int Ab;
        if (!c.packed) Ab = (int)std::min<long long>(P, ahi - a0);
        else if (forced > 0) Ab = std::min(forced, ahi - a0);
        else Ab = (int)std::max(1ll, std::min<long long>(P / (c.v - a0), ahi - a0));
        out.emplace_back(a0, Ab);
        a0 += Ab;
    }
    return out;
}

// ------------------------------------------------------------------ workspace
struct FwdLayout {
    size_t status, pairtab, t2x, Rc, epart, epair;
    // packed path
    size_t pairtab_m, rtab, Tp, eTp, Tm, eTm, Vp, eVp, Vm, eVm, Rpc, Rmc;
    // integral-first
    size_t V, Lw, eL, colmax, tw, et, Vw, eV, Lraw;
    // Cholesky-first
    size_t X2, LwA, eLA, twB, etB, X2w, eX2, LwB, eLB;
    size_t total;
};

// Packed path: P = capacity in integral rows (a, b), P >= max over blocks of Ab * (v - a0).
FwdLayout layout_packed(const Ctx& c, long long P)
{
    FwdLayout L{};
    Carve cv;
    const long long o = c.o, v = c.v, n = c.n, vv = v * v;
    const bool f64 = c.mode == CC_FP64;  // packed operands stay FP64 (DMMA), no slices
    const int es = f64 ? 8 : esz_of(c.mode);
    const long long s = f64 ? 1 : c.s;
    L.status = cv.take(256);
    L.pairtab = cv.take(8 * c.pp);
    L.pairtab_m = cv.take(8 * std::max(1ll, c.pm));
    if (c.exch) L.t2x = cv.take(8 * o * o * vv);
    L.epart = cv.take(8 * energy_scratch_doubles(c.o, c.v));
    L.epair = cv.take(8 * o * o);
    L.V = cv.take(8 * P * vv);
    if (c.hostL) L.Lraw = cv.take(2 * 8 * c.PC * vv);  // two FP64 chunks of L: one arriving, one in use
    const long long nk = c.hostL ? c.PC : n;           // K of the L slices held at once
    if (!f64) {
        L.Lw = cv.take(es * s * vv * pitch_for(nk, es));
        L.eL = cv.take(4 * vv);
        L.colmax = cv.take(8 * vv);
    }
    const long long pbm = std::min(c.PB, c.pm);  // pairs i < j in one pair block
    L.Tp = cv.take(es * s * c.PB * pitch_for(c.Kp, es));
    L.eTp = cv.take(4 * c.PB);
    L.Tm = cv.take(es * s * pbm * pitch_for(c.Km, es));
    L.eTm = cv.take(4 * pbm);
    L.rtab = cv.take(8 * P);
    L.Vp = cv.take(es * s * P * pitch_for(c.Kp, es));
    L.eVp = cv.take(4 * P);
    L.Vm = cv.take(es * s * P * pitch_for(c.Km, es));
    L.eVm = cv.take(4 * P);
    L.Rpc = cv.take(8 * c.PB * P);
    L.Rmc = cv.take(8 * pbm * P);
    L.total = cv.cur;
    return L;
}

FwdLayout layout_fwd(const Ctx& c, long long A)
{
    if (c.packed) return layout_packed(c, A);
    FwdLayout L{};
    Carve cv;
    const long long o = c.o, v = c.v, n = c.n, vv = v * v, P = c.pairs;
    L.status = cv.take(256);
    if (c.sym) L.pairtab = cv.take(8 * P);
    if (c.exch) L.t2x = cv.take(8 * o * o * vv);
    if (c.sym) L.Rc = cv.take(8 * P * vv);
    L.epart = cv.take(8 * energy_scratch_doubles(c.o, c.v));
    L.epair = cv.take(8 * o * o);
    const int es = esz_of(c.mode);
    const long long s = c.s;
    if (c.order == CC_ORDER_INTEGRAL_FIRST) {
        L.V = cv.take(8 * (long long)A * v * vv);
        if (is_tc(c.mode)) {
            L.Lw = cv.take(es * s * vv * pitch_for(n, es));
            L.eL = cv.take(4 * vv);
            L.colmax = cv.take(8 * vv);
            L.tw = cv.take(es * s * P * pitch_for(vv, es));
            L.et = cv.take(4 * P);
            L.Vw = cv.take(es * s * (long long)A * v * pitch_for(vv, es));
            L.eV = cv.take(4 * (long long)A * v);
        }
    } else {
        L.X2 = cv.take(8 * P * (long long)A * n * v);
        if (is_tc(c.mode)) {
            L.LwA = cv.take(es * s * v * n * pitch_for(v, es));
            L.eLA = cv.take(4 * v * n);
            L.twB = cv.take(es * s * P * v * pitch_for(v, es));
            L.etB = cv.take(4 * P * v);
            L.colmax = cv.take(8 * P * v);
            L.X2w = cv.take(es * s * P * (long long)A * pitch_for(n * v, es));
            L.eX2 = cv.take(4 * P * (long long)A);
            L.LwB = cv.take(es * s * v * pitch_for(n * v, es));
            L.eLB = cv.take(4 * v);
        }
    }
    L.total = cv.cur;
    return L;
}

struct BwdLayout {
    size_t status, LT, Wx, tx, M1, fwd;  // fwd = nested forward workspace for dt2
    size_t Lw, eL, Ww, eW, tw, et, colmax, M1w, eM1;
    size_t total;
};

// ------------------------------------------------------------------ planner
double flops_if(const Ctx& c)
{
    if (c.packed)
        return std::pow((double)c.v, 2) * (c.n * (double)c.v * (c.v + 1) + 2.0 * ((double)c.pp * c.Kp + (double)c.pm * c.Km));
    return 2.0 * ((double)c.pairs + c.n) * std::pow((double)c.v, 4);
}
double flops_cf(const Ctx& c) { return 4.0 * c.n * (double)c.pairs * std::pow((double)c.v, 3); }

// ---------------------------------------------------------------- autotuner
// Orders decided by timed trials (cc_ladder_autotune), per shape and mode; also kept
// in a text file when CC_LADDER_CACHE names one ("o v n mode flags order" per line).
struct TuneKey {
    int o, v, n, mode, flags;
    bool operator<(const TuneKey& b) const
    {
        return std::tie(o, v, n, mode, flags) < std::tie(b.o, b.v, b.n, b.mode, b.flags);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
bool g_cache_loaded = false;

int tune_flags(int flags) { return flags & (CC_FLAG_SYMMETRIC_T | CC_FLAG_EXCHANGE); }

void load_cache_locked()
{
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char* path = getenv("CC_LADDER_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    TuneKey k;
    int order;
    while (fscanf(f, "%d %d %d %d %d %d", &k.o, &k.v, &k.n, &k.mode, &k.flags, &order) == 6)
        if (order == CC_ORDER_INTEGRAL_FIRST || order == CC_ORDER_CHOLESKY_FIRST) g_tuned[k] = order;
    fclose(f);
}

int cached_order(const TuneKey& k)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    auto it = g_tuned.find(k);
    return it == g_tuned.end() ? 0 : it->second;
}

void store_order(const TuneKey& k, int order)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    g_tuned[k] = order;
    const char* path = getenv("CC_LADDER_CACHE");
    if (path && *path) {
        if (FILE* f = fopen(path, "a")) {
            fprintf(f, "%d %d %d %d %d %d\n", k.o, k.v, k.n, k.mode, k.flags, order);
            fclose(f);
        }
    }
}

int pick_order(const Ctx& c, int requested)
{
    if (requested == CC_ORDER_INTEGRAL_FIRST || requested == CC_ORDER_CHOLESKY_FIRST) return requested;
    if (const int t = cached_order(TuneKey{c.o, c.v, c.n, c.mode, tune_flags(c.flags)})) return t;
    // Cost model: tensor-core flops, with the Cholesky-first order charged for its
    // larger intermediate traffic (it writes and re-reads o^2 n v^2 per block).
    const double cf = flops_cf(c) * 1.15, itf = flops_if(c);
    return cf < itf ? CC_ORDER_CHOLESKY_FIRST : CC_ORDER_INTEGRAL_FIRST;
}

// Layout parameter fitting `bytes`: the block size A (unpacked paths: largest A, then
// evened out over the blocks it implies), or the integral-row capacity P (packed path:
// largest P in [v, v^2]; a requested a_block A means P = A v).  -1 if nothing fits.
long long pick_block_pb(const Ctx& c, size_t bytes, int requested, size_t* need);

// Host-resident t2 / R: the device holds one block of pairs at a time.  Pair blocks cost a new
// split of their t2 rows for every integral block and shorter ladder GEMMs, so the largest pair
// block (halving from all pairs) that leaves room for integral blocks of at least 4 `a` values
// (or all of them) is taken; when no pair block does, the largest one that fits one `a` per block.
long long pick_block_host(Ctx& c, size_t bytes, int requested, size_t* need);

// Streamed L: the chunk of Cholesky vectors starts at the caller's chol_chunk or at the one whose
// two FP64 buffers and slices take an eighth of the budget, and halves until a plan fits.
long long pick_block(Ctx& c, size_t bytes, int requested, size_t* need)
{
    if (!c.hostL) return pick_block_host(c, bytes, requested, need);
    const long long vv = (long long)c.v * c.v;
    const long long per = vv * (16 + (c.mode == CC_FP64 ? 0 : esz_of(c.mode) * (long long)c.s));
    long long pc = c.PC > 0 ? std::min<long long>(c.PC, c.n)
                            : std::max(1ll, std::min<long long>(c.n, (long long)(bytes / 8) / per));
    for (;; pc = (pc + 1) / 2) {
        c.PC = pc;
        const long long P = pick_block_host(c, bytes, requested, need);
        if (P >= 0 || pc == 1) return P;
    }
}

long long pick_block_host(Ctx& c, size_t bytes, int requested, size_t* need)
{
    if (!(c.host && c.packed)) return pick_block_pb(c, bytes, requested, need);
    const long long want = (long long)std::min(c.v, 4) * c.v;
    long long fallback = -1;
    for (long long pb = c.pp;; pb = (pb + 1) / 2) {
        c.PB = pb;
        const long long P = pick_block_pb(c, bytes, requested, need);
        if (P >= 0 && (P >= want || requested > 0)) return P;
        if (P >= 0 && fallback < 0) fallback = pb;
        if (pb == 1) break;
    }
    if (fallback < 0) return -1;
    c.PB = fallback;
    return pick_block_pb(c, bytes, requested, need);
}

long long pick_block_pb(const Ctx& c, size_t bytes, int requested, size_t* need)
{
    const long long unit = c.packed ? c.v : 1;
    if (requested > 0) {
        const long long P = (long long)std::min(requested, c.v) * unit;
        *need = layout_fwd(c, P).total;
        return *need <= bytes ? P : -1;
    }
    if (layout_fwd(c, unit).total > bytes) { *need = layout_fwd(c, unit).total; return -1; }
    long long lo = unit, hi = (long long)c.v * unit;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (layout_fwd(c, mid).total <= bytes) lo = mid; else hi = mid - 1;
    }
    long long P = lo;
    if (!c.packed) {
        const long long nb = (c.v + lo - 1) / lo;
        P = (c.v + nb - 1) / nb;
    }
    *need = layout_fwd(c, P).total;
    return P;
}

int make_ctx(const cc_ladder_args* a, Ctx* c)
{
    if (!a) return CC_ERR_NULL;
    if (a->o < 1 || a->v < 1 || a->n_chol < 1) return CC_ERR_SHAPE;
    if ((double)a->o * a->o * a->v * a->v > 4.0e12 || (double)a->n_chol * a->v * a->v > 4.0e12) return CC_ERR_SHAPE;
    if (a->v > 46340 || a->o > 46340) return CC_ERR_SHAPE;
    if (a->mode == CC_OZAKI_INT8) return CC_ERR_UNSUPPORTED;
    if (a->mode < CC_FP64 || a->mode > CC_BF16) return CC_ERR_ARG;
    if (a->order < CC_ORDER_AUTO || a->order > CC_ORDER_CHOLESKY_FIRST) return CC_ERR_ARG;
    if (a->a_block < 0) return CC_ERR_ARG;
    if (a->flags & ~(CC_FLAG_ACCUMULATE | CC_FLAG_SYMMETRIC_T | CC_FLAG_EXCHANGE | CC_FLAG_NO_STATUS_SYNC |
                     CC_FLAG_HOST_T2R | CC_FLAG_HOST_L))
        return CC_ERR_ARG;
    if (a->chol_chunk < 0) return CC_ERR_ARG;
    if (a->mode == CC_OZAKI_BF16 && a->slices != 0 && (a->slices < 2 || a->slices > 8)) return CC_ERR_ARG;
    if (a->a_lo < 0 || a->a_hi < 0 || a->a_lo > a->v || a->a_hi > a->v || (a->a_hi && a->a_hi <= a->a_lo))
        return CC_ERR_ARG;
    c->o = a->o; c->v = a->v; c->n = a->n_chol;
    c->mode = a->mode; c->flags = a->flags;
    c->s = slices_of(a->mode, a->slices);
    c->sym = (a->flags & CC_FLAG_SYMMETRIC_T) != 0;
    c->exch = (a->flags & CC_FLAG_EXCHANGE) != 0;
    c->pairs = c->sym ? (long long)a->o * (a->o + 1) / 2 : (long long)a->o * a->o;
    c->pp = (long long)a->o * (a->o + 1) / 2;
    c->pm = (long long)a->o * (a->o - 1) / 2;
    c->Kp = (long long)a->v * (a->v + 1) / 2;
    c->Km = (long long)a->v * (a->v - 1) / 2;
    // the packed path needs the pair symmetry and runs the tensor-core modes integral-first;
    // the order's cost model sees the packed flop count
    const bool can_pack = c->sym;
    c->packed = can_pack;
    // host-resident amplitudes and streamed L run through the integral-first order only
    const bool hostflags = (a->flags & (CC_FLAG_HOST_T2R | CC_FLAG_HOST_L)) != 0;
    c->order = (hostflags && a->order == CC_ORDER_AUTO) ? (int)CC_ORDER_INTEGRAL_FIRST : pick_order(*c, a->order);
    c->packed = can_pack && c->order == CC_ORDER_INTEGRAL_FIRST;
    c->host = (a->flags & CC_FLAG_HOST_T2R) != 0;
    c->PB = c->pp;
    c->hostL = (a->flags & CC_FLAG_HOST_L) != 0;
    c->PC = c->hostL ? a->chol_chunk : c->n;
    // host-resident amplitudes run on the packed path only, without the exchange copy
    if (c->host && (!c->packed || c->exch)) return CC_ERR_UNSUPPORTED;
    if (c->hostL && !c->packed) return CC_ERR_UNSUPPORTED;
    return CC_OK;
}

bool aligned(const void* p, size_t al) { return ((uintptr_t)p % al) == 0; }

int check_cuda(cudaError_t e) { return e == cudaSuccess ? CC_OK : CC_ERR_CUDA; }

int run_f64(const char* name, const GemmF64& g, cudaStream_t st, double elems = -1.0)
{
    ProfScope ps(name, st, 2.0 * (elems >= 0 ? elems : g.M * (double)g.N) * g.K);
    return check_cuda(gemm_f64(g, st));
}

#define CC_TRY(x)                      \
    do {                               \
        const int _st = (x);           \
        if (_st != CC_OK) return _st;  \
    } while (0)
#define CC_CU(x) CC_TRY(check_cuda(x))

// cc_status of a device status word: an expired wait first, then non-finite input.
int status_of(int h)
{
    if (h & (kStatusWaitExpired | kStatusDrainExpired)) return CC_ERR_DEVICE_TIMEOUT;
    if (h & kStatusNonfinite) return CC_ERR_NONFINITE;
    return CC_OK;
}

int finish(void* ws_status, int flags, cudaStream_t s)
{
    CC_CU(cudaGetLastError());
    if (flags & CC_FLAG_NO_STATUS_SYNC) return CC_OK;
    CC_CU(cudaStreamSynchronize(s));
    int h = 0;
    CC_CU(cudaMemcpy(&h, ws_status, sizeof(int), cudaMemcpyDeviceToHost));
    return status_of(h);
}

// ---------------------------------------------------- tensor-core operand prep
struct Operand {
    void* D; int* e; long long pitch, rows;
};

int prep_rows(const Ctx& c, const RowSrc& src, Operand& op, cudaStream_t st)
{
    ProfScope ps("split", st);
    op.rows = src.rows;
    op.pitch = pitch_for(src.K, esz_of(c.mode));
    if (c.mode == CC_TF32) return check_cuda(convert_rows_tf32(src, (float*)op.D, op.pitch, st));
    const int s = c.mode == CC_OZAKI_BF16 ? c.s : 0;
    return check_cuda(split_rows_bf16(src, s, kBeta, op.D, op.pitch, op.e, c.status, st));
}

// Split of an intermediate left as int64 fixed point by run_tc(..., intermediate=true).
int prep_fixed(const Ctx& c, const FixedSrc& src, Operand& op, cudaStream_t st)
{
    ProfScope ps("split", st);
    op.rows = src.rows;
    op.pitch = pitch_for((long long)src.outer * src.inner, esz_of(c.mode));
    return check_cuda(split_fixed_rows_bf16(src, c.s, kBeta, op.D, op.pitch, op.e, st));
}


int prep_cols(const Ctx& c, const ColSrc& src, Operand& op, unsigned long long* colmax, cudaStream_t st)
{
    ProfScope ps("split", st);
    op.rows = src.rows;
    op.pitch = pitch_for(src.K, esz_of(c.mode));
    if (c.mode == CC_TF32) return check_cuda(convert_cols_tf32(src, (float*)op.D, op.pitch, st));
    const int s = c.mode == CC_OZAKI_BF16 ? c.s : 0;
    return check_cuda(split_cols_bf16(src, s, kBeta, op.D, op.pitch, op.e, colmax, c.status, st));
}

double tc_products(const Ctx& c) { return c.mode == CC_OZAKI_BF16 ? c.s * (c.s + 1) / 2.0 : 1.0; }

// Output elements of an M x N slice GEMM that lie in tiles the triangular skip keeps
// (a(m) = m / tri, b(n) = n / tri; a tile goes when b < a for all its elements).
// Tile edges TM x TN: 128 x 128 in gemm_tc.cu, 64 x 64 in gemm_f64.cu.
double tri_elems(long long M, long long N, long long tri, long long TM = 128, long long TN = 128)
{
    if (tri <= 0) return (double)M * N;
    double e = 0.0;
    for (long long m0 = 0; m0 < M; m0 += TM) {
        const long long need = (m0 / tri) * tri;  // smallest n whose b reaches a(m0)
        if (need > N - 1) continue;
        const long long t0 = need >= TN - 1 ? (need - TN + 1 + TN - 1) / TN : 0;
        e += (double)std::min(TM, M - m0) * (double)(N - t0 * TN);
    }
    return e;
}

// Longest K-chunk over which the FP32 sums of the levels glo .. glo + gn - 1 stay exact for any
// input: balanced digits are at most 2^(beta-1) in magnitude, so a level with q products per K
// element grows by at most q 2^(2 beta - 2) per element, and below 2^24 every partial sum is an
// exact FP32 integer.  Rounded down to whole K-steps of the GEMM (64 bf16 elements).
constexpr long long kReuseK = 2048;  // longest K split of a GEMM with more tiles than SMs

int exact_chunk(int glo, int gn, int s)
{
    int q = 1;
    for (int L = glo; L < glo + gn; ++L) q = std::max(q, std::min(L, s - 1) - std::max(0, L - s + 1) + 1);
    const long long per = 1ll << (2 * kBeta - 2);
    const long long kc = ((1ll << 24) / (q * per)) / 64 * 64;
    return (int)std::max(64ll, kc);
}

// intermediate: the output feeds another slice GEMM through split_fixed_rows, so in
// the emulated mode it stays int64 fixed point (no FP64 work, no loads in the epilogue).
// tri > 0: triangular tile skip with a(m) = m / tri, b(n) = n / tri.
// add_int64 (intermediate only): add the int64 result into the output instead of storing it
// (later chunks of a contraction split on the host, e.g. streamed Cholesky vectors).
int run_tc(const char* name, const Ctx& c, int M, int N, int K, const Operand& A, long long rowA0, const Operand& B,
           long long rowB0, const OutDesc& out, int* status, cudaStream_t st, bool intermediate = false,
           long long tri = 0, bool add_int64 = false)
{
    // algorithmic bytes: every slice of both operands read once, the kept output written once
    // (8 bytes per element; read as well when accumulated)
    const double out_el = tri_elems(M, N, tri);
    const int opb = c.mode == CC_TF32 ? 4 : 2;
    const double bytes = (double)opb * c.s * ((double)M + N) * K + out_el * 8.0 * (out.accumulate ? 2 : 1);
    ProfScope ps(name, st, 2.0 * out_el * K * tc_products(c), bytes);
    // C = A B^T and C^T = B A^T are the same GEMM; the tiles are square (128 x 128), so the
    // orientation changes no padding: the longer operand is kept as A, whose rows are the
    // slowest-moving index of the tile raster (not with the triangular skip, which is one-sided)
    const bool swap = tri == 0 && N > M;
    const Operand& Aop = swap ? B : A;
    const Operand& Bop = swap ? A : B;
    OutDesc o = out;
    if (swap) std::swap(o.rmap, o.cmap);
    if (swap) { std::swap(M, N); std::swap(rowA0, rowB0); }
    GemmTc g{};
    g.kind = c.mode == CC_TF32 ? TC_TF32 : TC_BF16;
    g.M = M; g.N = N; g.K = K;
    g.A = Aop.D; g.pitchA = Aop.pitch; g.rowsA = Aop.rows; g.rowA0 = rowA0;
    g.B = Bop.D; g.pitchB = Bop.pitch; g.rowsB = Bop.rows; g.rowB0 = rowB0;
    g.slices = c.s;
    g.eA = c.mode == CC_TF32 ? nullptr : Aop.e;
    g.eB = c.mode == CC_TF32 ? nullptr : Bop.e;
    g.beta = kBeta;
    g.scale_base = c.mode == CC_OZAKI_BF16 ? 2 - 2 * kBeta : 0;
    if (c.mode == CC_OZAKI_BF16) {
        // levels 0 .. s-1 (all products i + j <= s-1), paired from the top; each pass covers at
        // most exact_chunk() K elements, so every FP32 level sum is exact for any input
        g.ngroups = 0;
        for (int L = c.s - 1; L >= 0; L -= 2) {
            g.glo[g.ngroups] = L >= 1 ? L - 1 : 0;
            g.gn[g.ngroups] = L >= 1 ? 2 : 1;
            g.gkc[g.ngroups] = exact_chunk(g.glo[g.ngroups], g.gn[g.ngroups], c.s);
            ++g.ngroups;
        }
        g.epi = intermediate ? (add_int64 ? EPI_FIXED64_ADD : EPI_FIXED64_RED) : EPI_FIXED64;
        g.fixF = kFixF;
        // Few tiles of long K: split K over CTAs so that the items fill whole waves of
        // the device (int64 adds into a zeroed output, then one conversion pass for final outputs)
        if (!o.accumulate) {
            const long long tiles = (long long)((M + 127) / 128) * ((N + 127) / 128);
            const int nsm = std::max(1, device_sm_count());
            auto eff = [&](int S) {
                const double w = (double)tiles * S / nsm;
                return w / std::ceil(w);
            };
            int best = 1;
            for (int S = 2; S <= 8 && (long long)K / S >= 8192; ++S)
                if (eff(S) > eff(best) + 0.02) best = S;
            // L2 reuse: the items resident at once (one per SM) share operand rows, and while they
            // run in step one copy of a K-step's rows in L2 serves them all.  Over a long K they
            // drift apart and re-read the rows from HBM.  Items are ordered split-major, so
            // short splits keep the resident items within one K window: a 36540 x 820 x 80200
            // GEMM measured 1080 TFLOP/s issued unsplit, 1130 with splits of 8192, 1200 with 2048.
            // Not for intermediates (the integral blocks): there the split's zeroing pass and
            // red.global adds on the large int64 output cost more than the reuse gains (o=60,
            // v=600, n=3000: KG1 6.58 s split, 5.87 s whole; its R+- GEMMs 3.48 s split, 4.81 s
            // whole).
            if (tiles > nsm && !intermediate)
                while ((K + best - 1) / best > kReuseK) ++best;
            if (best > 1) {
                // the kernel rounds a split up to whole K-steps: count the splits that leaves
                const long long kper = ((K + best - 1) / best + 63) / 64 * 64;
                best = (int)((K + kper - 1) / kper);
            }
            if (best > 1) {
                g.epi = EPI_FIXED64_ADD;
                g.ksplit = best;
            }
        }
    } else {
        g.ngroups = 1;
        g.glo[0] = 0; g.gn[0] = 1; g.gkc[0] = kMixedChunk;
        g.epi = EPI_FP64_RMW;
        g.fixF = 0;
    }
    g.tri_rdiv = g.tri_cdiv = tri;
    g.out = o;
    g.status = status;
    g.wait_ns = g_wait_ns.load();
    if (g.epi == EPI_FIXED64_ADD) {
        if (!add_int64) CC_CU(zero_out(M, N, o, st));
        CC_CU(gemm_tc(g, st));
        // an intermediate stays int64 fixed point: its consumer applies the exponents
        if (intermediate) return CC_OK;
        return check_cuda(fixed_to_f64(M, N, o, g.eA, rowA0, g.eB, rowB0, kFixedBase, st));
    }
    return check_cuda(gemm_tc(g, st));
}

template <typename T>
T* at(void* ws, size_t off) { return (T*)((char*)ws + off); }

// ----------------------------------------------------------------- forward
// Packed path (pair-symmetric t2, integral-first, tensor-core modes): see the header
// comment.  R receives R[i,j,a,b] and R[i,j,b,a] for all i, j, a in [alo, ahi), b >= a.
int fwd_packed(const Ctx& c, const cc_ladder_args* a, const double* Lsrc, const double* t2, long long P,
               const FwdLayout& Lo, void* ws, int* status, cudaStream_t st, int alo, int ahi)
{
    const long long v = c.v, n = c.n, vv = v * v;
    const bool ozaki = c.mode == CC_OZAKI_BF16, f64 = c.mode == CC_FP64;
    const int kind = ozaki ? 0 : (c.mode == CC_BF16 ? 1 : (f64 ? 3 : 2));
    const int es = f64 ? 8 : esz_of(c.mode);
    long long* pairtab = at<long long>(ws, Lo.pairtab);
    long long* pairtab_m = at<long long>(ws, Lo.pairtab_m);
    long long* rtab = at<long long>(ws, Lo.rtab);
    CC_CU(fill_pairs(c.o, c.v, 0, pairtab, st));
    CC_CU(fill_pairs(c.o, c.v, 1, pairtab_m, st));
    const bool minus = c.pm > 0 && c.Km > 0;

    Operand Lw{}, Tp{}, Tm{}, Vp{}, Vm{};
    Lw.D = at<void>(ws, Lo.Lw); Lw.e = at<int>(ws, Lo.eL);
    Tp.D = at<void>(ws, Lo.Tp); Tp.e = at<int>(ws, Lo.eTp); Tp.rows = c.pp; Tp.pitch = pitch_for(c.Kp, es);
    Tm.D = at<void>(ws, Lo.Tm); Tm.e = at<int>(ws, Lo.eTm); Tm.rows = c.pm; Tm.pitch = pitch_for(c.Km, es);
    Vp.D = at<void>(ws, Lo.Vp); Vp.e = at<int>(ws, Lo.eVp); Vp.pitch = Tp.pitch;
    Vm.D = at<void>(ws, Lo.Vm); Vm.e = at<int>(ws, Lo.eVm); Vm.pitch = Tm.pitch;
    unsigned long long* colmax = at<unsigned long long>(ws, Lo.colmax);
    // Streamed L (CC_FLAG_HOST_L): chunks of PC Cholesky vectors are copied from page-locked host
    // memory into two device buffers on a second stream, so that chunk q + 1 arrives while chunk q
    // is split and contracted (the batches of Cholesky vectors of Section 5, overlapped); events
    // order every copy after the last use of its buffer.  Stream and events belong to this call.
    struct Streamer {
        cudaStream_t cs = nullptr;
        cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
        ~Streamer()
        {
            for (int b = 0; b < 2; ++b) {
                if (copied[b]) cudaEventDestroy(copied[b]);
                if (freed[b]) cudaEventDestroy(freed[b]);
            }
            if (cs) cudaStreamDestroy(cs);
        }
    } sm;
    double* Lraw = c.hostL ? at<double>(ws, Lo.Lraw) : nullptr;
    if (c.hostL) {
        CC_CU(cudaStreamCreateWithFlags(&sm.cs, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CC_CU(cudaEventCreateWithFlags(&sm.copied[b], cudaEventDisableTiming));
            CC_CU(cudaEventCreateWithFlags(&sm.freed[b], cudaEventDisableTiming));
        }
    }
    // consume(buf, P0, Pq): enqueue on st the work that reads chunk [P0, P0 + Pq) of L in buf.
    // The chunk counter runs on across calls, so the first copies of a pass still wait for the
    // last readers of their buffers in the pass before.
    long long q = 0;
    auto stream_L = [&](auto&& consume) -> int {
        for (long long P0 = 0; P0 < n; P0 += c.PC, ++q) {
            const long long Pq = std::min<long long>(c.PC, n - P0);
            const int b = (int)(q & 1);
            double* buf = Lraw + b * c.PC * vv;
            if (q >= 2) CC_CU(cudaStreamWaitEvent(sm.cs, sm.freed[b], 0));
            CC_CU(cudaMemcpyAsync(buf, Lsrc + P0 * vv, (size_t)(Pq * vv) * 8, cudaMemcpyHostToDevice, sm.cs));
            CC_CU(cudaEventRecord(sm.copied[b], sm.cs));
            CC_CU(cudaStreamWaitEvent(st, sm.copied[b], 0));
            CC_TRY(consume(buf, P0, Pq));
            CC_CU(cudaEventRecord(sm.freed[b], st));
        }
        return CC_OK;
    };
    if (!f64 && !c.hostL) {
        // L rows (a,c) are contiguous in L[P][a][c]; K = P is strided
        ColSrc ls{Lsrc, vv, vv, n, 0, plain_map(0)};
        CC_TRY(prep_cols(c, ls, Lw, colmax, st));
    } else if (ozaki && c.hostL) {
        // row scales of the Ozaki split need every Cholesky vector: one streaming pass for the maxima
        CC_CU(cudaMemsetAsync(colmax, 0, 8 * vv, st));
        CC_TRY(stream_L([&](const double* buf, long long, long long Pq) {
            ColSrc ls{buf, vv, vv, Pq, 0, plain_map(0)};
            return check_cuda(cols_max(ls, colmax, c.status, st));
        }));
    }
    // Pair blocks [q0, q1) of the i <= j pairs; their pairs i < j are [s0, s1) in the strict
    // enumeration (s(p) = p - i - [j > i] pairs i < j precede pair p = (i, j)).
    auto strict_before = [&](long long p) -> long long {
        if (p >= c.pp) return c.pm;
        long long i = 0, rem = p;
        while (rem >= c.o - i) { rem -= c.o - i; ++i; }
        return p - i - (rem > 0 ? 1 : 0);
    };
    std::vector<std::pair<long long, long long>> pblocks;
    for (long long q0 = 0; q0 < c.pp; q0 += c.PB) pblocks.emplace_back(q0, std::min(c.pp, q0 + c.PB));
    // T+ / T- of one pair block (t2 rows read where they are: device or page-locked host memory)
    auto split_t = [&](long long q0, long long q1) -> int {
        ProfScope ps("split", st);
        const long long s0 = strict_before(q0), s1 = strict_before(q1);
        Tp.rows = q1 - q0;
        Tm.rows = s1 - s0;
        CC_CU(pm_split_f64(t2, pairtab + q0, 1, q1 - q0, c.v, +1, 1.0, kind, c.s, kBeta, Tp.D, Tp.pitch, Tp.e, c.status, st));
        if (minus && s1 > s0)
            CC_CU(pm_split_f64(t2, pairtab_m + s0, 1, s1 - s0, c.v, -1, 1.0, kind, c.s, kBeta, Tm.D, Tm.pitch, Tm.e,
                               c.status, st));
        return CC_OK;
    };
    if (pblocks.size() == 1) CC_TRY(split_t(0, c.pp));
    double* V = at<double>(ws, Lo.V);
    double* Rpc = at<double>(ws, Lo.Rpc);
    double* Rmc = at<double>(ws, Lo.Rmc);
    const int accum = (c.flags & CC_FLAG_ACCUMULATE) ? 1 : 0;
    for (const auto& blk : block_list(c, P, alo, ahi, a->a_block)) {
        const int a0 = blk.first, Ab = blk.second, Nb = c.v - a0;
        const long long nr = (long long)Ab * Nb - (long long)Ab * (Ab - 1) / 2;
        // KG1: V[al][b'][c][d] = sum_P L[P, a0+al, c] L[P, a0+b', d], tiles with b < a skipped
        OutDesc o1{V, split_map(v, (long long)Nb * vv, v), split_map(v, vv, 1), 0};
        if (c.hostL) {
            // the block's integrals summed over the chunks of Cholesky vectors (additive in P)
            CC_TRY(stream_L([&](const double* buf, long long P0, long long Pq) -> int {
                OutDesc oq = o1;
                if (f64) {
                    GemmF64 g{};
                    g.M = Ab * c.v; g.N = Nb * c.v; g.K = (int)Pq;
                    g.A = buf; g.am = plain_map(1, (long long)a0 * v); g.ak = plain_map(vv);
                    g.B = buf; g.bm = plain_map(1, (long long)a0 * v); g.bk = plain_map(vv);
                    oq.accumulate = P0 > 0;
                    g.out = oq;
                    g.tri = v;
                    return run_f64("kg1_f64", g, st, tri_elems(g.M, g.N, v, 64, 64));
                }
                ColSrc ls{buf, vv, vv, Pq, 0, plain_map(0)};
                if (ozaki) {
                    ProfScope ps("split", st);
                    Lw.rows = vv;
                    Lw.pitch = pitch_for(Pq, es);
                    CC_CU(split_cols_bf16(ls, c.s, kBeta, Lw.D, Lw.pitch, Lw.e, colmax, c.status, st, true));
                } else {
                    CC_TRY(prep_cols(c, ls, Lw, colmax, st));
                    oq.accumulate = P0 > 0;  // mixed modes: FP64 integral block
                }
                return run_tc("kg1_tc", c, Ab * c.v, Nb * c.v, (int)Pq, Lw, (long long)a0 * v, Lw, (long long)a0 * v,
                              oq, status, st, true, v, ozaki && P0 > 0);
            }));
        } else if (f64) {
            GemmF64 g{};
            g.M = Ab * c.v; g.N = Nb * c.v; g.K = c.n;
            g.A = Lsrc; g.am = plain_map(1, (long long)a0 * v); g.ak = plain_map(vv);
            g.B = Lsrc; g.bm = plain_map(1, (long long)a0 * v); g.bk = plain_map(vv);
            g.out = o1;
            g.tri = v;
            CC_TRY(run_f64("kg1_f64", g, st, tri_elems(g.M, g.N, v, 64, 64)));
        } else {
            CC_TRY(run_tc("kg1_tc", c, Ab * c.v, Nb * c.v, c.n, Lw, (long long)a0 * v, Lw, (long long)a0 * v, o1,
                          status, st, true, v));
        }
        CC_CU(fill_rtab(Ab, Nb, rtab, st));
        Vp.rows = nr; Vm.rows = nr;
        {
            ProfScope ps("split", st);
            if (ozaki) {
                // V[al][b'][c][d] = X * 2^(eL[(a0+al)v + c] + eL[(a0+b')v + d] + base)
                PmFixedSrc fs{(const long long*)V, rtab, nr, vv, c.v, Lw.e, split_map(Nb, v, 0, (long long)a0 * v),
                              Lw.e, split_map(Nb, 0, v, (long long)a0 * v), kFixedBase};
                CC_CU(pm_split_fixed(fs, c.s, kBeta, Vp.D, Vp.pitch, Vp.e, minus ? Vm.D : nullptr, Vm.pitch, Vm.e, st));
            } else {
                CC_CU(pm_split_f64(V, rtab, vv, nr, c.v, +1, 0.5, kind, c.s, kBeta, Vp.D, Vp.pitch, Vp.e, nullptr, st));
                if (minus)
                    CC_CU(pm_split_f64(V, rtab, vv, nr, c.v, -1, 0.5, kind, c.s, kBeta, Vm.D, Vm.pitch, Vm.e, nullptr, st));
            }
        }
        OutDesc op{Rpc, plain_map(nr), plain_map(1), 0};
        OutDesc om{Rmc, plain_map(nr), plain_map(1), 0};
        for (const auto& pb : pblocks) {
            const long long q0 = pb.first, q1 = pb.second;
            const long long s0 = strict_before(q0), s1 = strict_before(q1);
            if (pblocks.size() > 1) CC_TRY(split_t(q0, q1));
            const bool mb = minus && s1 > s0;
            if (f64) {
                for (int sg = 0; sg < (mb ? 2 : 1); ++sg) {
                    const Operand& T = sg ? Tm : Tp;
                    const Operand& Vx = sg ? Vm : Vp;
                    GemmF64 g{};
                    g.M = (int)(sg ? s1 - s0 : q1 - q0); g.N = (int)nr; g.K = (int)(sg ? c.Km : c.Kp);
                    g.A = (const double*)T.D; g.am = plain_map(T.pitch); g.ak = plain_map(1);
                    g.B = (const double*)Vx.D; g.bm = plain_map(Vx.pitch); g.bk = plain_map(1);
                    g.out = sg ? om : op;
                    CC_TRY(run_f64("kg2_f64", g, st));
                }
            } else {
                CC_TRY(run_tc("kg2_tc", c, (int)(q1 - q0), (int)nr, (int)c.Kp, Tp, 0, Vp, 0, op, status, st));
                if (mb) CC_TRY(run_tc("kg2_tc", c, (int)(s1 - s0), (int)nr, (int)c.Km, Tm, 0, Vm, 0, om, status, st));
            }
            ProfScope ps("scatter", st);
            CC_CU(pm_combine(c.o, c.v, a0, Ab, Nb, nr, q0, q1, s0, Rpc, mb ? Rmc : nullptr, a->R, accum, st));
        }
    }
    return CC_OK;
}

int fwd_impl(const cc_ladder_args* a, const double* Lsrc_override = nullptr)
{
    Ctx c;
    CC_TRY(make_ctx(a, &c));
    const double* Lsrc = Lsrc_override ? Lsrc_override : a->L;
    if (!Lsrc || !a->t2 || !a->R || !a->workspace) return CC_ERR_NULL;
    if (!aligned(Lsrc, 16) || !aligned(a->t2, 16) || !aligned(a->R, 16) || !aligned(a->workspace, 256) ||
        (a->energy && !aligned(a->energy, 8)))
        return CC_ERR_ALIGN;
    if (is_tc(c.mode) && !tc_gemm_available()) return CC_ERR_UNSUPPORTED;
    if (c.host) {
        // t2 and R must be page-locked host memory the device can address
        cudaPointerAttributes pa{};
        for (const void* hp : {(const void*)a->t2, (const void*)a->R}) {
            if (cudaPointerGetAttributes(&pa, hp) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
                pa.devicePointer != hp) {
                cudaGetLastError();
                return CC_ERR_ARG;
            }
        }
    }
    if (c.hostL) {
        // L must be page-locked host memory (the source of asynchronous copies)
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, Lsrc) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return CC_ERR_ARG;
        }
    }
    size_t need = 0;
    const long long Pblk = pick_block(c, a->ws_bytes, a->a_block, &need);
    if (Pblk < 0) return CC_ERR_WORKSPACE;
    const FwdLayout Lo = layout_fwd(c, Pblk);
    const int A = (int)Pblk;
    if (const char* vb = getenv("CC_LADDER_VERBOSE")) {
        if (*vb && *vb != '0')
            fprintf(stderr, "cc_ladder: o=%d v=%d n=%d mode=%d order=%s packed=%d host=%d block-param=%lld "
                            "pair-blocks=%lld workspace=%zu B of %zu\n",
                    c.o, c.v, c.n, c.mode, c.order == CC_ORDER_INTEGRAL_FIRST ? "integral-first" : "cholesky-first",
                    (int)c.packed, (int)c.host, Pblk, c.packed ? (c.pp + c.PB - 1) / c.PB : 1ll, need, a->ws_bytes);
    }
    void* ws = a->workspace;
    cudaStream_t st = (cudaStream_t)a->stream;
    const long long o = c.o, v = c.v, n = c.n, vv = v * v;
    int* status = at<int>(ws, Lo.status);
    c.status = status;
    const int alo = a->a_hi ? a->a_lo : 0, ahi = a->a_hi ? a->a_hi : c.v;
    // an a-range's share of the energy is defined where the range owns both R_ijab and R_ijba of
    // its terms: the packed path (entries with min(a, b) in the range)
    if (a->energy && (alo != 0 || ahi != c.v) && !c.packed) return CC_ERR_UNSUPPORTED;
    CC_CU(cudaMemsetAsync(status, 0, 256, st));

    const double* t2 = a->t2;
    if (c.exch) {  // Eq. 7 = Eq. 6 applied to t2 with c <-> d swapped
        CC_CU(swap_last2(o * o, c.v, a->t2, at<double>(ws, Lo.t2x), st));
        t2 = at<double>(ws, Lo.t2x);
    }
    if (c.packed) {
        CC_TRY(fwd_packed(c, a, Lsrc, t2, Pblk, Lo, ws, status, st, alo, ahi));
        if (a->energy) {
            ProfScope ps("energy", st);
            CC_CU(energy_pairs(c.o, c.v, a->R, a->t2, at<double>(ws, Lo.epart), at<double>(ws, Lo.epair), st, alo,
                               ahi));
            CC_CU(energy_total((long long)c.o * c.o, at<double>(ws, Lo.epair), a->energy, st));
        }
        return finish(status, c.flags, st);
    }
    long long* pairtab = c.sym ? at<long long>(ws, Lo.pairtab) : nullptr;
    if (c.sym) CC_CU(fill_pair_table(c.o, c.v, pairtab, st));
    // rows of t2 used as GEMM rows: all (i,j), or the pairs i <= j
    const Map2 trows = c.sym ? table_map(pairtab) : plain_map(vv);
    double* Rdst = c.sym ? at<double>(ws, Lo.Rc) : a->R;
    const int accum = (!c.sym && (c.flags & CC_FLAG_ACCUMULATE)) ? 1 : 0;

    if (c.order == CC_ORDER_INTEGRAL_FIRST) {
        double* V = at<double>(ws, Lo.V);
        Operand Lw{}, tw{}, Vw{};
        if (is_tc(c.mode)) {
            Lw.D = at<void>(ws, Lo.Lw); Lw.e = at<int>(ws, Lo.eL);
            tw.D = at<void>(ws, Lo.tw); tw.e = at<int>(ws, Lo.et);
            Vw.D = at<void>(ws, Lo.Vw); Vw.e = at<int>(ws, Lo.eV);
            // L rows (a,c) are contiguous in L[P][a][c]; K = P is strided
            ColSrc ls{Lsrc, vv, vv, n, 0, plain_map(0)};
            CC_TRY(prep_cols(c, ls, Lw, at<unsigned long long>(ws, Lo.colmax), st));
            RowSrc ts{t2, trows, plain_map(1), c.pairs, vv};
            CC_TRY(prep_rows(c, ts, tw, st));
        }
        for (int a0 = alo; a0 < ahi; a0 += A) {
            const int Ab = std::min(A, ahi - a0);
            // KG1: V[al][b][c][d], GEMM rows (al,c), cols (b,d)
            OutDesc o1{V, split_map(v, v * vv, v), split_map(v, vv, 1), 0};
            if (c.mode == CC_FP64) {
                GemmF64 g{};
                g.M = Ab * c.v; g.N = (int)vv; g.K = c.n;
                g.A = Lsrc; g.am = plain_map(1, (long long)a0 * v); g.ak = plain_map(vv);
                g.B = Lsrc; g.bm = plain_map(1); g.bk = plain_map(vv);
                g.out = o1;
                CC_TRY(run_f64("kg1_f64", g, st));
            } else {
                CC_TRY(run_tc("kg1_tc", c, Ab * c.v, (int)vv, c.n, Lw, (long long)a0 * v, Lw, 0, o1, status, st, true));
            }
            // KG2: R[ij][a0+al][b] = sum_(c,d) t2[ij][(c,d)] V[al][b][(c,d)]
            OutDesc o2{Rdst, plain_map(vv), plain_map(1, (long long)a0 * v), accum};
            if (c.mode == CC_FP64) {
                GemmF64 g{};
                g.M = (int)c.pairs; g.N = Ab * c.v; g.K = (int)vv;
                g.A = t2; g.am = trows; g.ak = plain_map(1);
                g.B = V; g.bm = plain_map(vv); g.bk = plain_map(1);
                g.out = o2;
                CC_TRY(run_f64("kg2_f64", g, st));
            } else {
                if (c.mode == CC_OZAKI_BF16) {
                    // V[al][b][c][d] = X * 2^(eL[(a0+al)v + c] + eL[b v + d] + base)
                    FixedSrc fs{(const long long*)V, (long long)Ab * v, vv, c.v, c.v, Lw.e,
                                split_map(v, v, 0, (long long)a0 * v), Lw.e, split_map(v, 0, v), kFixedBase};
                    CC_TRY(prep_fixed(c, fs, Vw, st));
                } else {
                    RowSrc vs{V, plain_map(vv), plain_map(1), (long long)Ab * v, vv};
                    CC_TRY(prep_rows(c, vs, Vw, st));
                }
                CC_TRY(run_tc("kg2_tc", c, (int)c.pairs, Ab * c.v, (int)vv, tw, 0, Vw, 0, o2, status, st));
            }
        }
    } else {
        // Cholesky-first.  Rows of CF1's B operand are (p, d): t2 rows p, element c*v + d.
        double* X2 = at<double>(ws, Lo.X2);
        Operand LwA{}, twB{}, X2w{}, LwB{};
        if (is_tc(c.mode)) {
            LwA.D = at<void>(ws, Lo.LwA); LwA.e = at<int>(ws, Lo.eLA);
            twB.D = at<void>(ws, Lo.twB); twB.e = at<int>(ws, Lo.etB);
            X2w.D = at<void>(ws, Lo.X2w); X2w.e = at<int>(ws, Lo.eX2);
            LwB.D = at<void>(ws, Lo.LwB); LwB.e = at<int>(ws, Lo.eLB);
            // CF1 A: rows (a, P) over all a, K = c contiguous: L[P][a][c]
            RowSrc la{Lsrc, split_map(n, v, vv), plain_map(1), v * n, v};
            CC_TRY(prep_rows(c, la, LwA, st));
            // CF1 B: rows (p, d), K = c: batched, rows d contiguous within t2[p]
            ColSrc tb{t2, v, c.pairs * v, v, v, c.sym ? table_map(pairtab) : plain_map(vv)};
            CC_TRY(prep_cols(c, tb, twB, at<unsigned long long>(ws, Lo.colmax), st));
            // CF2 B: rows b, K = (P, d): L[P][b][d]
            RowSrc lb{Lsrc, plain_map(v), split_map(v, vv, 1), v, n * v};
            CC_TRY(prep_rows(c, lb, LwB, st));
        }
        for (int a0 = alo; a0 < ahi; a0 += A) {
            const int Ab = std::min(A, ahi - a0);
            // CF1: rows (al, P), cols (p, d), K = c  ->  X2[(p, al), (P, d)]
            OutDesc o1{X2, split_map(n, n * v, v), split_map(v, (long long)Ab * n * v, 1), 0};
            if (c.mode == CC_FP64) {
                GemmF64 g{};
                g.M = Ab * c.n; g.N = (int)(c.pairs * v); g.K = c.v;
                g.A = Lsrc; g.am = split_map(n, v, vv, (long long)a0 * v); g.ak = plain_map(1);
                g.B = t2; g.bm = c.sym ? table_map(pairtab, v, 1) : split_map(v, vv, 1); g.bk = plain_map(v);
                g.out = o1;
                CC_TRY(run_f64("cf1_f64", g, st));
            } else {
                CC_TRY(run_tc("cf1_tc", c, Ab * c.n, (int)(c.pairs * v), c.v, LwA, (long long)a0 * n, twB, 0, o1, status, st,
                              true));
            }
            // CF2: rows (p, al), cols b, K = (P, d)  ->  R[p][a0+al][b]
            OutDesc o2{Rdst, split_map(Ab, vv, v, (long long)a0 * v), plain_map(1), accum};
            if (c.mode == CC_FP64) {
                GemmF64 g{};
                g.M = (int)(c.pairs * Ab); g.N = c.v; g.K = (int)(n * v);
                g.A = X2; g.am = plain_map(n * v); g.ak = plain_map(1);
                g.B = Lsrc; g.bm = plain_map(v); g.bk = split_map(v, vv, 1);
                g.out = o2;
                CC_TRY(run_f64("cf2_f64", g, st));
            } else {
                if (c.mode == CC_OZAKI_BF16) {
                    // X2[(p, al)][(P, d)] = X * 2^(eLA[(a0+al) n + P] + etB[p v + d] + base)
                    FixedSrc fs{(const long long*)X2, c.pairs * Ab, n * v, c.n, c.v, LwA.e,
                                split_map(Ab, 0, n, (long long)a0 * n), twB.e, split_map(Ab, v, 0), kFixedBase};
                    CC_TRY(prep_fixed(c, fs, X2w, st));
                } else {
                    RowSrc xs{X2, plain_map(n * v), plain_map(1), c.pairs * Ab, n * v};
                    CC_TRY(prep_rows(c, xs, X2w, st));
                }
                CC_TRY(run_tc("cf2_tc", c, (int)(c.pairs * Ab), c.v, (int)(n * v), X2w, 0, LwB, 0, o2, status, st));
            }
        }
    }
    if (c.sym) {
        ProfScope ps("scatter", st);
        CC_CU(scatter_pairs(c.o, c.v, alo, ahi, at<double>(ws, Lo.Rc), a->R, (c.flags & CC_FLAG_ACCUMULATE) ? 1 : 0,
                            st));
    }
    if (a->energy) {
        ProfScope ps("energy", st);
        CC_CU(energy_pairs(c.o, c.v, a->R, a->t2, at<double>(ws, Lo.epart), at<double>(ws, Lo.epair), st));
        CC_CU(energy_total((long long)c.o * c.o, at<double>(ws, Lo.epair), a->energy, st));
    }
    return finish(status, c.flags, st);
}

// ------------------------------------------------- two-block terms (Eq. 8, 9)
// G[i,j,p,q] = sum_cd (sum_P A[P,p,c] B[P,q,d]) t2[i,j,c,d], A: n x np x v, B: n x nq x v, the
// contraction shared by the ladder and the two further Cholesky terms of Section 6.1:
//   Eq. 8  tt_ijkl: A = B = Lov (np = nq = o),   Eq. 9  tt_ijbk: A = Lov, B = Lvv (output [i][j][b][k]).
// Integral-first in blocks of p, exactly like the ladder's unpacked path:
//   KG1  V[pl][q][c][d] = sum_P A[P,p0+pl,c] B[P,q,d]    (GEMM M = Pb v, N = nq v, K = n)
//   KG2  G[ij][p0+pl][q] = sum_(c,d) t2[ij,c,d] V[pl][q][c][d]  (GEMM M = o^2, N = Pb nq, K = v^2)
struct TermCtx {
    Ctx c;           // o, v, n, mode, s (pairs = o^2, no symmetry)
    int np_, nq;
    bool same;       // A and B are the same array (one set of slices)
    int which;
};

struct TermLayout {
    size_t status, V, Aw, eA, Bw, eB, colmax, tw, et, Vw, eV, total;
};

TermLayout layout_term(const TermCtx& tc, long long Pb)
{
    const Ctx& c = tc.c;
    TermLayout L{};
    Carve cv;
    const long long o = c.o, v = c.v, n = c.n, vv = v * v;
    L.status = cv.take(256);
    L.V = cv.take(8 * Pb * tc.nq * vv);
    if (is_tc(c.mode)) {
        const int es = esz_of(c.mode);
        const long long s = c.s;
        L.Aw = cv.take(es * s * tc.np_ * v * pitch_for(n, es));
        L.eA = cv.take(4 * tc.np_ * v);
        if (!tc.same) {
            L.Bw = cv.take(es * s * tc.nq * v * pitch_for(n, es));
            L.eB = cv.take(4 * tc.nq * v);
        }
        L.colmax = cv.take(8 * std::max(tc.np_, tc.nq) * v);
        L.tw = cv.take(es * s * o * o * pitch_for(vv, es));
        L.et = cv.take(4 * o * o);
        L.Vw = cv.take(es * s * Pb * tc.nq * pitch_for(vv, es));
        L.eV = cv.take(4 * Pb * tc.nq);
    }
    L.total = cv.cur;
    return L;
}

int term_ctx(int which, int o, int v, int n, int mode, int slices, TermCtx* tc)
{
    if (which != CC_TERM_IJKL && which != CC_TERM_IJBK) return CC_ERR_ARG;
    cc_ladder_args a{};
    a.o = o; a.v = v; a.n_chol = n; a.mode = mode; a.slices = slices; a.order = CC_ORDER_INTEGRAL_FIRST;
    CC_TRY(make_ctx(&a, &tc->c));
    if ((double)o * o * o * v > 4.0e12 || (double)n * o * v > 4.0e12) return CC_ERR_SHAPE;
    tc->which = which;
    tc->np_ = o;
    tc->nq = which == CC_TERM_IJKL ? o : v;
    tc->same = which == CC_TERM_IJKL;
    return CC_OK;
}

// Largest block of p fitting `bytes` (-1 if one p does not fit), evened over the blocks.
long long pick_term_block(const TermCtx& tc, size_t bytes, size_t* need)
{
    if (layout_term(tc, 1).total > bytes) { *need = layout_term(tc, 1).total; return -1; }
    long long lo = 1, hi = tc.np_;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (layout_term(tc, mid).total <= bytes) lo = mid; else hi = mid - 1;
    }
    const long long nb = (tc.np_ + lo - 1) / lo;
    const long long P = (tc.np_ + nb - 1) / nb;
    *need = layout_term(tc, P).total;
    return P;
}

int term_impl(int which, int o, int v, int n, const double* Lov, const double* Lvv, const double* t2, double* T,
              int mode, int flags, int slices, void* ws, size_t ws_bytes, void* stream)
{
    TermCtx tc;
    CC_TRY(term_ctx(which, o, v, n, mode, slices, &tc));
    if (flags & ~CC_FLAG_NO_STATUS_SYNC) return CC_ERR_ARG;
    const double* A = Lov;
    const double* Bm = which == CC_TERM_IJKL ? Lov : Lvv;
    if (!A || !Bm || !t2 || !T || !ws) return CC_ERR_NULL;
    if (!aligned(A, 16) || !aligned(Bm, 16) || !aligned(t2, 16) || !aligned(T, 16) || !aligned(ws, 256))
        return CC_ERR_ALIGN;
    Ctx c = tc.c;
    if (is_tc(c.mode) && !tc_gemm_available()) return CC_ERR_UNSUPPORTED;
    size_t need = 0;
    const long long Pb = pick_term_block(tc, ws_bytes, &need);
    if (Pb < 0 || need > ws_bytes) return CC_ERR_WORKSPACE;
    const TermLayout Lo = layout_term(tc, Pb);
    cudaStream_t st = (cudaStream_t)stream;
    const long long v_ = v, vv = v_ * v, np_ = tc.np_, nq = tc.nq;
    int* status = at<int>(ws, Lo.status);
    c.status = status;
    CC_CU(cudaMemsetAsync(status, 0, 256, st));
    double* V = at<double>(ws, Lo.V);
    Operand Aw{}, Bw{}, tw{}, Vw{};
    if (is_tc(c.mode)) {
        Aw.D = at<void>(ws, Lo.Aw); Aw.e = at<int>(ws, Lo.eA);
        tw.D = at<void>(ws, Lo.tw); tw.e = at<int>(ws, Lo.et);
        Vw.D = at<void>(ws, Lo.Vw); Vw.e = at<int>(ws, Lo.eV);
        // rows (p, c) of A[P][p][c] are contiguous; K = P is strided
        ColSrc as{A, np_ * v_, np_ * v_, n, 0, plain_map(0)};
        CC_TRY(prep_cols(c, as, Aw, at<unsigned long long>(ws, Lo.colmax), st));
        if (tc.same) {
            Bw = Aw;
        } else {
            Bw.D = at<void>(ws, Lo.Bw); Bw.e = at<int>(ws, Lo.eB);
            ColSrc bs{Bm, nq * v_, nq * v_, n, 0, plain_map(0)};
            CC_TRY(prep_cols(c, bs, Bw, at<unsigned long long>(ws, Lo.colmax), st));
        }
        RowSrc ts{t2, plain_map(vv), plain_map(1), (long long)o * o, vv};
        CC_TRY(prep_rows(c, ts, tw, st));
    }
    for (long long p0 = 0; p0 < np_; p0 += Pb) {
        const int Ab = (int)std::min(Pb, np_ - p0);
        // KG1: V[pl][q][c][d], GEMM rows (pl, c), cols (q, d)
        OutDesc o1{V, split_map(v_, nq * vv, v_), split_map(v_, vv, 1), 0};
        if (c.mode == CC_FP64) {
            GemmF64 g{};
            g.M = Ab * v; g.N = (int)(nq * v_); g.K = n;
            g.A = A; g.am = plain_map(1, p0 * v_); g.ak = plain_map(np_ * v_);
            g.B = Bm; g.bm = plain_map(1); g.bk = plain_map(nq * v_);
            g.out = o1;
            CC_TRY(run_f64("term_kg1_f64", g, st));
        } else {
            CC_TRY(run_tc("term_kg1_tc", c, Ab * v, (int)(nq * v_), n, Aw, p0 * v_, Bw, 0, o1, status, st, true));
        }
        // KG2: T[ij][p0 + pl][q] (Eq. 8: [i][j][k][l]) or T[ij][q][p0 + pl] (Eq. 9: [i][j][b][k])
        const Map2 ocol = which == CC_TERM_IJKL ? plain_map(1, p0 * nq) : split_map(nq, 1, np_, p0);
        OutDesc o2{T, plain_map(np_ * nq), ocol, 0};
        if (c.mode == CC_FP64) {
            GemmF64 g{};
            g.M = o * o; g.N = (int)(Ab * nq); g.K = (int)vv;
            g.A = t2; g.am = plain_map(vv); g.ak = plain_map(1);
            g.B = V; g.bm = plain_map(vv); g.bk = plain_map(1);
            g.out = o2;
            CC_TRY(run_f64("term_kg2_f64", g, st));
        } else {
            if (c.mode == CC_OZAKI_BF16) {
                // V[pl][q][c][d] = X * 2^(eA[(p0+pl) v + c] + eB[q v + d] + base)
                FixedSrc fs{(const long long*)V, Ab * nq, vv, v, v, Aw.e, split_map(nq, v_, 0, p0 * v_), Bw.e,
                            split_map(nq, 0, v_), kFixedBase};
                CC_TRY(prep_fixed(c, fs, Vw, st));
            } else {
                RowSrc vs{V, plain_map(vv), plain_map(1), Ab * nq, vv};
                CC_TRY(prep_rows(c, vs, Vw, st));
            }
            CC_TRY(run_tc("term_kg2_tc", c, o * o, (int)(Ab * nq), (int)vv, tw, 0, Vw, 0, o2, status, st));
        }
    }
    return finish(status, flags, st);
}

// ----------------------------------------------------------------- adjoint
// dt2 = forward with L'[P,a,c] = L[P,c,a] applied to W (integral symmetry (ac|bd)).
// dL  = T1[W, t] + T1[W^swap, t^swap], T1[X,t][P,e,f] = sum_(b,d) L[P,b,d] M1[e,f,b,d],
//       M1[e,f,b,d] = sum_ij X[ij,e,b] t[ij,f,d]; for pair-symmetric t this is T1[W + W^swap, t].
struct BwdPlan {
    Ctx c;      // c.pairs = o*o (W has no pair symmetry)
    int E;      // e-block for M1
    cc_ladder_args fa;  // nested forward for dt2
    size_t fwd_bytes;
    BwdLayout L;
};

BwdLayout layout_bwd(const Ctx& c, int E, size_t fwd_bytes, bool sym)
{
    BwdLayout L{};
    Carve cv;
    const long long o = c.o, v = c.v, n = c.n, vv = v * v, P = (long long)o * o;
    L.status = cv.take(256);
    L.LT = cv.take(8 * n * vv);
    L.Wx = cv.take(8 * P * vv);
    if (!sym) L.tx = cv.take(8 * P * vv);
    L.M1 = cv.take(8 * (long long)E * v * vv);
    if (is_tc(c.mode)) {
        const int es = esz_of(c.mode);
        const long long s = c.s;
        L.Lw = cv.take(es * s * n * pitch_for(vv, es));
        L.eL = cv.take(4 * n);
        L.Ww = cv.take(es * s * (long long)E * v * pitch_for(P, es));
        L.eW = cv.take(4 * (long long)E * v);
        L.tw = cv.take(es * s * vv * pitch_for(P, es));
        L.et = cv.take(4 * vv);
        L.colmax = cv.take(8 * vv);
        L.M1w = cv.take(es * s * (long long)E * v * pitch_for(vv, es));
        L.eM1 = cv.take(4 * (long long)E * v);
    }
    L.fwd = cv.take(fwd_bytes);
    L.total = cv.cur;
    return L;
}

int bwd_plan(int o, int v, int n, int mode, int flags, int slices, size_t bytes, bool for_query, BwdPlan* bp)
{
    cc_ladder_args fa{};
    fa.o = o; fa.v = v; fa.n_chol = n; fa.mode = mode; fa.order = CC_ORDER_INTEGRAL_FIRST; fa.slices = slices;
    fa.flags = flags & CC_FLAG_NO_STATUS_SYNC;
    Ctx c;
    CC_TRY(make_ctx(&fa, &c));
    const bool sym = (flags & CC_FLAG_SYMMETRIC_T) != 0;
    // Split the budget: find the largest block E (used for both the nested forward's
    // integral block and the M1 block) such that everything fits.
    auto total_for = [&](int A) {
        const size_t fb = layout_fwd(c, A).total;
        return layout_bwd(c, A, fb, sym).total;
    };
    if (total_for(1) > bytes) return for_query ? CC_ERR_BUDGET : CC_ERR_WORKSPACE;
    int lo = 1, hi = v;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (total_for(mid) <= bytes) lo = mid; else hi = mid - 1;
    }
    const int nb = (v + lo - 1) / lo;
    const int A = (v + nb - 1) / nb;
    bp->c = c;
    bp->E = A;
    bp->fwd_bytes = layout_fwd(c, A).total;
    bp->L = layout_bwd(c, A, bp->fwd_bytes, sym);
    bp->fa = fa;
    bp->fa.a_block = A;
    return CC_OK;
}

int bwd_impl(int o, int v, int n, const double* L, const double* t2, const double* W, double* dL, double* dt2, int mode,
             int flags, int slices, void* ws, size_t ws_bytes, void* stream)
{
    if (flags & ~(CC_FLAG_SYMMETRIC_T | CC_FLAG_NO_STATUS_SYNC)) return CC_ERR_ARG;
    BwdPlan bp;
    {
        cc_ladder_args probe{};
        probe.o = o; probe.v = v; probe.n_chol = n; probe.mode = mode; probe.slices = slices;
        Ctx tmp;
        CC_TRY(make_ctx(&probe, &tmp));
    }
    if (!L || !t2 || !W || !ws) return CC_ERR_NULL;
    if (!aligned(L, 16) || !aligned(t2, 16) || !aligned(W, 16) || !aligned(ws, 256) || (dL && !aligned(dL, 16)) ||
        (dt2 && !aligned(dt2, 16)))
        return CC_ERR_ALIGN;
    CC_TRY(bwd_plan(o, v, n, mode, flags, slices, ws_bytes, false, &bp));
    if (is_tc(mode) && !tc_gemm_available()) return CC_ERR_UNSUPPORTED;
    Ctx c = bp.c;
    const BwdLayout& Lo = bp.L;
    cudaStream_t st = (cudaStream_t)stream;
    const long long vv = (long long)v * v, P = (long long)o * o;
    int* status = at<int>(ws, Lo.status);
    c.status = status;
    CC_CU(cudaMemsetAsync(status, 0, 256, st));
    const bool sym = (flags & CC_FLAG_SYMMETRIC_T) != 0;

    if (dt2) {
        double* LT = at<double>(ws, Lo.LT);
        CC_CU(transpose_last2(n, v, L, LT, st));
        cc_ladder_args fa = bp.fa;
        fa.L = LT; fa.t2 = W; fa.R = dt2; fa.energy = nullptr;
        fa.workspace = at<void>(ws, Lo.fwd); fa.ws_bytes = bp.fwd_bytes;
        fa.stream = stream;
        fa.flags = CC_FLAG_NO_STATUS_SYNC;
        CC_TRY(fwd_impl(&fa));
        // the nested call has its own status word; fold it into ours
        int* st2 = at<int>(fa.workspace, 0);
        CC_CU(cudaMemcpyAsync(status + 1, st2, sizeof(int), cudaMemcpyDeviceToDevice, st));
    }
    if (dL) {
        double* Wx = at<double>(ws, Lo.Wx);
        const double* tt[2];
        const double* Xs[2];
        int npass;
        if (sym) {
            CC_CU(add_pair_swap(o, v, W, Wx, 1, st));  // W + W^swap
            Xs[0] = Wx; tt[0] = t2; npass = 1;
        } else {
            double* tx = at<double>(ws, Lo.tx);
            CC_CU(add_pair_swap(o, v, W, Wx, 0, st));   // W^swap
            CC_CU(add_pair_swap(o, v, t2, tx, 0, st));  // t^swap
            Xs[0] = W; tt[0] = t2; Xs[1] = Wx; tt[1] = tx; npass = 2;
        }
        double* M1 = at<double>(ws, Lo.M1);
        const int E = bp.E;
        Operand Lw{}, Ww{}, tw{}, M1w{};
        if (is_tc(mode)) {
            Lw.D = at<void>(ws, Lo.Lw); Lw.e = at<int>(ws, Lo.eL);
            Ww.D = at<void>(ws, Lo.Ww); Ww.e = at<int>(ws, Lo.eW);
            tw.D = at<void>(ws, Lo.tw); tw.e = at<int>(ws, Lo.et);
            M1w.D = at<void>(ws, Lo.M1w); M1w.e = at<int>(ws, Lo.eM1);
            RowSrc ls{L, plain_map(vv), plain_map(1), n, vv};  // T1 A: rows P, K = (b,d)
            CC_TRY(prep_rows(c, ls, Lw, st));
        }
        for (int pass = 0; pass < npass; ++pass) {
            if (is_tc(mode)) {
                ColSrc ts{tt[pass], vv, vv, P, 0, plain_map(0)};  // M1 B: rows (f,d), K = ij
                CC_TRY(prep_cols(c, ts, tw, at<unsigned long long>(ws, Lo.colmax), st));
            }
            for (int e0 = 0; e0 < v; e0 += E) {
                const int Eb = std::min(E, v - e0);
                // M1: rows (el,b), cols (f,d), K = ij  ->  M1[el][f][b][d]
                OutDesc o1{M1, split_map(v, v * vv, v), split_map(v, vv, 1), 0};
                if (mode == CC_FP64) {
                    GemmF64 g{};
                    g.M = Eb * v; g.N = (int)vv; g.K = (int)P;
                    g.A = Xs[pass]; g.am = plain_map(1, (long long)e0 * v); g.ak = plain_map(vv);
                    g.B = tt[pass]; g.bm = plain_map(1); g.bk = plain_map(vv);
                    g.out = o1;
                    CC_TRY(run_f64("m1_f64", g, st));
                } else {
                    ColSrc ws_{Xs[pass] + (long long)e0 * v, vv, (long long)Eb * v, P, 0, plain_map(0)};
                    CC_TRY(prep_cols(c, ws_, Ww, at<unsigned long long>(ws, Lo.colmax), st));
                    CC_TRY(run_tc("m1_tc", c, Eb * v, (int)vv, (int)P, Ww, 0, tw, 0, o1, status, st, true));
                }
                // T1: dL[P][e0+el][f] (+)= sum_(b,d) L[P][(b,d)] M1[(el,f)][(b,d)]
                OutDesc o2{dL, plain_map(vv), plain_map(1, (long long)e0 * v), pass > 0 ? 1 : 0};
                if (mode == CC_FP64) {
                    GemmF64 g{};
                    g.M = n; g.N = Eb * v; g.K = (int)vv;
                    g.A = L; g.am = plain_map(vv); g.ak = plain_map(1);
                    g.B = M1; g.bm = plain_map(vv); g.bk = plain_map(1);
                    g.out = o2;
                    CC_TRY(run_f64("t1_f64", g, st));
                } else {
                    if (mode == CC_OZAKI_BF16) {
                        // M1[el][f][b][d] = X * 2^(eW[el v + b] + et[f v + d] + base)
                        FixedSrc fs{(const long long*)M1, (long long)Eb * v, vv, v, v, Ww.e, split_map(v, v, 0), tw.e,
                                    split_map(v, 0, v), kFixedBase};
                        CC_TRY(prep_fixed(c, fs, M1w, st));
                    } else {
                        RowSrc ms{M1, plain_map(vv), plain_map(1), (long long)Eb * v, vv};
                        CC_TRY(prep_rows(c, ms, M1w, st));
                    }
                    CC_TRY(run_tc("t1_tc", c, n, Eb * v, (int)vv, Lw, 0, M1w, 0, o2, status, st));
                }
            }
        }
    }
    CC_CU(cudaGetLastError());
    if (flags & CC_FLAG_NO_STATUS_SYNC) return CC_OK;
    CC_CU(cudaStreamSynchronize(st));
    int h[2] = {0, 0};
    CC_CU(cudaMemcpy(h, status, sizeof(h), cudaMemcpyDeviceToHost));
    return status_of(h[0] | h[1]);
}

}  // namespace

// ======================================================================= ABI
extern "C" {

const char* cc_ladder_strerror(int status)
{
    switch (status) {
    case CC_OK: return "ok";
    case CC_ERR_SHAPE: return "invalid shape (o, v, n_chol must be >= 1 and not overflow)";
    case CC_ERR_NULL: return "required pointer is NULL";
    case CC_ERR_ALIGN: return "pointer misaligned (tensors 16 bytes, workspace 256 bytes)";
    case CC_ERR_WORKSPACE: return "workspace smaller than the plan needs";
    case CC_ERR_BUDGET: return "budget below the smallest plan";
    case CC_ERR_UNSUPPORTED: return "mode/order/flag combination not supported on this device";
    case CC_ERR_CUDA: return "CUDA runtime error";
    case CC_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait expired; results are invalid";
    case CC_ERR_ARG: return "invalid argument";
    case CC_ERR_NOALLOC_LIMIT: return "problem exceeds the fixed scratch of cc_ladder_energy_noalloc";
    case CC_ERR_NONFINITE: return "an input holds NaN or Inf (emulated FP64 mode); results are invalid";
    default: return "unknown status";
    }
}

const char* cc_ladder_version(void) { return "cc_ladder 0.1 (sm_103a)"; }

void cc_ladder_set_wait_limit_ns(unsigned long long ns) { g_wait_ns.store(ns ? ns : 2000000000ull); }

int cc_ladder_workspace_size_ex(const cc_ladder_args* args, size_t* bytes)
{
    if (!bytes) return CC_ERR_NULL;
    Ctx c;
    CC_TRY(make_ctx(args, &c));
    const size_t budget = args->budget_bytes ? args->budget_bytes : kDefaultBudget;
    size_t need = 0;
    if (pick_block(c, budget, args->a_block, &need) < 0) return CC_ERR_BUDGET;
    *bytes = need;
    return CC_OK;
}

int cc_ladder_workspace_size(int o, int v, int n_chol, int mode, size_t budget_bytes, size_t* bytes)
{
    cc_ladder_args a{};
    a.o = o; a.v = v; a.n_chol = n_chol; a.mode = mode; a.budget_bytes = budget_bytes;
    return cc_ladder_workspace_size_ex(&a, bytes);
}

int cc_ladder_plan_query(const cc_ladder_args* args, cc_ladder_plan* plan)
{
    if (!plan) return CC_ERR_NULL;
    Ctx c;
    CC_TRY(make_ctx(args, &c));
    size_t need = 0;
    const size_t bytes = args->ws_bytes ? args->ws_bytes : (args->budget_bytes ? args->budget_bytes : kDefaultBudget);
    const long long P = pick_block(c, bytes, args->a_block, &need);
    if (P < 0) return CC_ERR_WORKSPACE;
    const int alo = args->a_hi ? args->a_lo : 0, ahi = args->a_hi ? args->a_hi : c.v;
    const auto blocks = block_list(c, P, alo, ahi, args->a_block);
    plan->order = c.order;
    plan->a_block = blocks.empty() ? 0 : blocks[0].second;
    plan->n_blocks = (int)blocks.size();
    plan->slices = c.s;
    plan->pairs = (int)c.pairs;
    plan->ws_bytes = need;
    const double v = c.v, o2 = (double)c.o * c.o, frac = (double)(ahi - alo) / c.v;
    plan->flops_algorithmic = (c.order == CC_ORDER_INTEGRAL_FIRST ? 2.0 * (o2 + c.n) * v * v * v * v
                                                                  : 4.0 * c.n * o2 * v * v * v) * frac;
    const double nprod = tc_products(c);
    double issued = 0.0;
    if (c.packed) {
        for (const auto& b : blocks) {
            const long long Ab = b.second, Nb = c.v - b.first;
            const double nr = (double)Ab * Nb - (double)Ab * (Ab - 1) / 2;
            const double e1 = c.mode == CC_FP64 ? tri_elems(Ab * c.v, Nb * c.v, c.v, 64, 64)
                                                : tri_elems(Ab * c.v, Nb * c.v, c.v);
            issued += 2.0 * c.n * e1 + 2.0 * nr * ((double)c.pp * c.Kp + (double)c.pm * c.Km);
        }
    } else {
        issued = (c.order == CC_ORDER_INTEGRAL_FIRST ? 2.0 * ((double)c.pairs + c.n) * v * v * v * v
                                                     : 4.0 * c.n * (double)c.pairs * v * v * v) * frac;
    }
    plan->flops_issued = issued * nprod;
    plan->pair_blocks = c.packed ? (int)((c.pp + c.PB - 1) / c.PB) : 1;
    return CC_OK;
}

int cc_ladder_fwd_ex(const cc_ladder_args* args) { return fwd_impl(args); }

int cc_ladder_partition(const cc_ladder_args* args, int parts, int* bounds)
{
    if (!bounds) return CC_ERR_NULL;
    Ctx c;
    CC_TRY(make_ctx(args, &c));
    if (parts < 1 || parts > c.v) return CC_ERR_ARG;
    // Work of the `a` values below a: on the packed path a column a builds the integrals (a, b >= a)
    // and the ladder columns of the same pairs, so its work is proportional to v - a; on the other
    // paths every `a` costs the same.
    const double v = c.v;
    auto W = [&](int a) { return c.packed ? (double)a * v - (double)a * (a - 1) / 2.0 : (double)a; };
    const double total = W(c.v);
    bounds[0] = 0;
    for (int g = 1; g < parts; ++g) {
        const double target = total * g / parts;
        // candidates keep every part non-empty: bounds[g-1] < a <= v - (parts - g)
        int lo = bounds[g - 1] + 1, hi = c.v - (parts - g);
        while (lo < hi) {  // smallest a in [lo, hi] with W(a) >= target
            const int mid = (lo + hi) / 2;
            if (W(mid) >= target) hi = mid; else lo = mid + 1;
        }
        int a = lo;
        if (a - 1 > bounds[g - 1] && std::fabs(W(a - 1) - target) < std::fabs(W(a) - target)) --a;
        bounds[g] = a;
    }
    bounds[parts] = c.v;
    return CC_OK;
}

int cc_ladder_autotune(const cc_ladder_args* args, cc_ladder_plan* plan, double* ms_if, double* ms_cf)
{
    Ctx c;
    CC_TRY(make_ctx(args, &c));
    if (!args->L || !args->t2 || !args->R || !args->workspace) return CC_ERR_NULL;
    cudaStream_t st = (cudaStream_t)args->stream;
    const int orders[2] = {CC_ORDER_INTEGRAL_FIRST, CC_ORDER_CHOLESKY_FIRST};
    double est[2] = {-1.0, -1.0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CC_ERR_CUDA;
    int status = CC_OK;
    for (int q = 0; q < 2 && status == CC_OK; ++q) {
        cc_ladder_args a = *args;
        a.order = orders[q];
        a.energy = nullptr;
        a.flags &= ~CC_FLAG_ACCUMULATE;
        Ctx cq;
        make_ctx(&a, &cq);
        size_t need = 0;
        const long long P = pick_block(cq, a.ws_bytes, a.a_block, &need);
        if (P < 0) continue;  // this order does not fit the workspace
        // time one block and (when there is one) two blocks: fixed cost + per-block cost
        // (packed blocks are sized to about equal work, so the extrapolation holds there too)
        double t[2] = {0.0, 0.0};
        const auto blocks = block_list(cq, P, 0, c.v, a.a_block);
        const int nb = (int)blocks.size();
        const int reps = nb >= 2 ? 2 : 1;
        for (int r = 0; r < reps && status == CC_OK; ++r) {
            a.a_lo = 0;
            a.a_hi = blocks[r].first + blocks[r].second;
            status = fwd_impl(&a);  // warm (first use of the shape)
            if (status != CC_OK) break;
            cudaEventRecord(e0, st);
            status = fwd_impl(&a);
            cudaEventRecord(e1, st);
            if (status != CC_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t[r] = ms;
        }
        if (status != CC_OK) break;
        est[q] = reps == 2 ? t[0] + (nb - 1) * (t[1] - t[0]) : t[0];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != CC_OK) return status;
    if (est[0] < 0 && est[1] < 0) return CC_ERR_WORKSPACE;
    const int best = (est[1] >= 0 && (est[0] < 0 || est[1] < est[0])) ? orders[1] : orders[0];
    store_order(TuneKey{c.o, c.v, c.n, c.mode, tune_flags(c.flags)}, best);
    if (ms_if) *ms_if = est[0];
    if (ms_cf) *ms_cf = est[1];
    if (plan) {
        cc_ladder_args a = *args;
        a.order = best;
        a.a_lo = a.a_hi = 0;
        return cc_ladder_plan_query(&a, plan);
    }
    return CC_OK;
}

int cc_ladder_fwd(int o, int v, int n_chol, const double* L, const double* t2, double* R, int mode, double* energy,
                  void* workspace, size_t ws_bytes, void* stream)
{
    cc_ladder_args a{};
    a.o = o; a.v = v; a.n_chol = n_chol; a.L = L; a.t2 = t2; a.R = R; a.energy = energy; a.mode = mode;
    a.workspace = workspace; a.ws_bytes = ws_bytes; a.stream = stream;
    return fwd_impl(&a);
}

int cc_ladder_bwd_workspace_size(int o, int v, int n_chol, int mode, size_t budget_bytes, size_t* bytes)
{
    if (!bytes) return CC_ERR_NULL;
    BwdPlan bp;
    CC_TRY(bwd_plan(o, v, n_chol, mode, 0, 0, budget_bytes ? budget_bytes : kDefaultBudget, true, &bp));
    *bytes = bp.L.total;
    return CC_OK;
}

int cc_ladder_bwd_ex(int o, int v, int n_chol, const double* L, const double* t2, const double* dR, double* dL,
                     double* dt2, int mode, int flags, int slices, void* workspace, size_t ws_bytes, void* stream)
{
    return bwd_impl(o, v, n_chol, L, t2, dR, dL, dt2, mode, flags, slices, workspace, ws_bytes, stream);
}

int cc_ladder_bwd(int o, int v, int n_chol, const double* L, const double* t2, const double* dR, double* dL,
                  double* dt2, int mode, void* workspace, size_t ws_bytes, void* stream)
{
    return bwd_impl(o, v, n_chol, L, t2, dR, dL, dt2, mode, 0, 0, workspace, ws_bytes, stream);
}

int cc_ladder_energy_workspace_size(int o, int v, size_t* bytes)
{
    if (!bytes) return CC_ERR_NULL;
    if (o < 1 || v < 1 || o > 46340 || v > 46340) return CC_ERR_SHAPE;
    *bytes = al256(8 * (size_t)energy_scratch_doubles(o, v)) + al256(8 * (size_t)o * o);
    return CC_OK;
}

int cc_ladder_energy(int o, int v, const double* R, const double* t2, double* energy, double* e_pair, void* workspace,
                     size_t ws_bytes, void* stream)
{
    if (o < 1 || v < 1 || o > 46340 || v > 46340) return CC_ERR_SHAPE;
    if (!R || !t2 || !energy || !workspace) return CC_ERR_NULL;
    if (!aligned(R, 16) || !aligned(t2, 16) || !aligned(workspace, 256) || !aligned(energy, 8)) return CC_ERR_ALIGN;
    size_t need = 0;
    cc_ladder_energy_workspace_size(o, v, &need);
    if (ws_bytes < need) return CC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)workspace;
    double* ep = e_pair ? e_pair : (double*)((char*)workspace + al256(8 * (size_t)energy_scratch_doubles(o, v)));
    CC_CU(energy_pairs(o, v, R, t2, part, ep, st));
    CC_CU(energy_total((long long)o * o, ep, energy, st));
    CC_CU(cudaGetLastError());
    return CC_OK;
}

static size_t gemm_ws(int mode, int M, int N, int K, int s)
{
    Carve cv;
    cv.take(256);
    if (is_tc(mode)) {
        const int es = esz_of(mode);
        cv.take((size_t)es * s * M * pitch_for(K, es));
        cv.take(4 * (size_t)M);
        cv.take((size_t)es * s * N * pitch_for(K, es));
        cv.take(4 * (size_t)N);
    }
    return cv.cur;
}

int cc_ladder_gemm_workspace_size(int mode, int M, int N, int K, int slices, size_t* bytes)
{
    if (!bytes) return CC_ERR_NULL;
    if (M < 1 || N < 1 || K < 1) return CC_ERR_SHAPE;
    if (mode == CC_OZAKI_INT8) return CC_ERR_UNSUPPORTED;
    if (mode < CC_FP64 || mode > CC_BF16) return CC_ERR_ARG;
    if (mode == CC_OZAKI_BF16 && slices != 0 && (slices < 2 || slices > 8)) return CC_ERR_ARG;
    *bytes = gemm_ws(mode, M, N, K, slices_of(mode, slices));
    return CC_OK;
}

int cc_ladder_gemm(int mode, int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                   int ldc, int accumulate, int slices, void* workspace, size_t ws_bytes, void* stream)
{
    size_t need = 0;
    CC_TRY(cc_ladder_gemm_workspace_size(mode, M, N, K, slices, &need));
    if (!A || !B || !C || !workspace) return CC_ERR_NULL;
    if (lda < K || ldb < K || ldc < N) return CC_ERR_ARG;
    if (!aligned(A, 16) || !aligned(B, 16) || !aligned(C, 16) || !aligned(workspace, 256)) return CC_ERR_ALIGN;
    if (ws_bytes < need) return CC_ERR_WORKSPACE;
    if (is_tc(mode) && !tc_gemm_available()) return CC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = (int*)workspace;
    CC_CU(cudaMemsetAsync(status, 0, 256, st));
    OutDesc out{C, plain_map(ldc), plain_map(1), accumulate ? 1 : 0};
    if (mode == CC_FP64) {
        GemmF64 g{};
        g.M = M; g.N = N; g.K = K;
        g.A = A; g.am = plain_map(lda); g.ak = plain_map(1);
        g.B = B; g.bm = plain_map(ldb); g.bk = plain_map(1);
        g.out = out;
        CC_TRY(run_f64("gemm_f64", g, st));
    } else {
        Ctx c{};
        c.mode = mode;
        c.s = slices_of(mode, slices);
        c.status = status;
        const int es = esz_of(mode);
        Carve cv;
        cv.take(256);
        Operand oa{}, ob{};
        oa.D = at<void>(workspace, cv.take((size_t)es * c.s * M * pitch_for(K, es)));
        oa.e = at<int>(workspace, cv.take(4 * (size_t)M));
        ob.D = at<void>(workspace, cv.take((size_t)es * c.s * N * pitch_for(K, es)));
        ob.e = at<int>(workspace, cv.take(4 * (size_t)N));
        RowSrc ra{A, plain_map(lda), plain_map(1), M, K};
        RowSrc rb{B, plain_map(ldb), plain_map(1), N, K};
        CC_TRY(prep_rows(c, ra, oa, st));
        CC_TRY(prep_rows(c, rb, ob, st));
        CC_TRY(run_tc("gemm_tc", c, M, N, K, oa, 0, ob, 0, out, status, st));
    }
    return finish(status, 0, st);
}

int cc_ladder_term_workspace_size(int which, int o, int v, int n_chol, int mode, int slices, size_t budget_bytes,
                                  size_t* bytes)
{
    if (!bytes) return CC_ERR_NULL;
    TermCtx tc;
    CC_TRY(term_ctx(which, o, v, n_chol, mode, slices, &tc));
    size_t need = 0;
    if (pick_term_block(tc, budget_bytes ? budget_bytes : kDefaultBudget, &need) < 0) return CC_ERR_BUDGET;
    *bytes = need;
    return CC_OK;
}

int cc_ladder_term(int which, int o, int v, int n_chol, const double* Lov, const double* Lvv, const double* t2,
                   double* T, int mode, int flags, int slices, void* workspace, size_t ws_bytes, void* stream)
{
    return term_impl(which, o, v, n_chol, Lov, Lvv, t2, T, mode, flags, slices, workspace, ws_bytes, stream);
}

int cc_ladder_tijkl(int o, int v, int n_chol, const double* Lov, const double* t2, double* T, int mode,
                    void* workspace, size_t ws_bytes, void* stream)
{
    return term_impl(CC_TERM_IJKL, o, v, n_chol, Lov, nullptr, t2, T, mode, 0, 0, workspace, ws_bytes, stream);
}

int cc_ladder_tijbk(int o, int v, int n_chol, const double* Lov, const double* Lvv, const double* t2, double* T,
                    int mode, void* workspace, size_t ws_bytes, void* stream)
{
    return term_impl(CC_TERM_IJBK, o, v, n_chol, Lov, Lvv, t2, T, mode, 0, 0, workspace, ws_bytes, stream);
}

int cc_ladder_device_status(void* workspace, void* stream)
{
    if (!workspace) return CC_ERR_NULL;
    CC_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int h[2] = {0, 0};
    CC_CU(cudaMemcpy(h, workspace, sizeof(h), cudaMemcpyDeviceToHost));
    CC_CU(cudaMemset(workspace, 0, sizeof(h)));
    return status_of(h[0] | h[1]);
}

}  // extern "C"
