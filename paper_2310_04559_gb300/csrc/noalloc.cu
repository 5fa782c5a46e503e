// noalloc.cu -- the pair energy for callers that cannot allocate device memory.
//
// cc_ladder_energy needs a caller-provided workspace for its per-tile partial
// sums.  Some callers have no way to provide one: code whose device memory is
// owned by another framework's pool (a CC driver embedding this library inside
// a larger simulation that has handed out its whole memory budget), or code that
// must not call cudaMalloc / cudaFree at all because those calls can block or
// synchronise the whole device in the middle of a latency-sensitive loop.
// cc_ladder_energy_noalloc computes the same energy with the same kernels but
// keeps its partial sums in a fixed array that lives in the library itself, so
// the call allocates nothing.
//
// The array (kScratchDoubles doubles, 16 MiB) is a file-scope __device__
// variable: every GPU on which the library is loaded holds one copy of it until
// the process exits.  Host code cannot use the array's name as a device address,
// so the first call in each CUDA context looks the address up with
// cudaGetSymbolAddress (with that context's device current) and caches it under
// the context's unique id.  A device reset creates a new context (and may load
// the module at a new address), so the next call looks the address up again
// instead of using a stale pointer.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "cc_internal.cuh"

namespace {

constexpr long long kScratchDoubles = 1ll << 21;  // 16 MiB
constexpr int kCacheSlots = 64;

static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

struct Slot {
    unsigned long long ctx_id;  // 0 = empty (context ids start at 1)
    double* ptr;
};

std::mutex g_mu;
Slot g_cache[kCacheSlots] = {};
int g_next = 0;

// Unique id of the current CUDA context (0 if it cannot be had), via the driver entry points.
unsigned long long current_ctx_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)f;
    });
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_energy_scratch in the current context (nullptr on failure).
double* scratch_address()
{
    // 0 when no context is current yet: the lookup below then creates the runtime's
    // context, and the next call finds it
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (id)
        for (const Slot& s : g_cache)
            if (s.ctx_id == id) return s.ptr;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    if (id) {
        g_cache[g_next] = Slot{id, (double*)p};
        g_next = (g_next + 1) % kCacheSlots;
    }
    return (double*)p;
}

}  // namespace

extern "C" int cc_ladder_energy_noalloc(int o, int v, const double* R, const double* t2, double* energy,
                                        double* e_pair, void* stream)
{
    if (o < 1 || v < 1 || o > 46340 || v > 46340) return CC_ERR_SHAPE;
    if (!R || !t2 || !energy) return CC_ERR_NULL;
    if (((uintptr_t)R % 16) || ((uintptr_t)t2 % 16) || ((uintptr_t)energy % 8) || (e_pair && ((uintptr_t)e_pair % 8)))
        return CC_ERR_ALIGN;
    const long long part = cc::energy_scratch_doubles(o, v);
    const long long need = part + (e_pair ? 0 : (long long)o * o);
    if (need > kScratchDoubles) return CC_ERR_NOALLOC_LIMIT;
    double* scratch = scratch_address();
    if (!scratch) return CC_ERR_CUDA;
    // Every partial the two kernels read is written earlier in the same call, so the
    // array needs no clearing.
    cudaStream_t st = (cudaStream_t)stream;
    double* ep = e_pair ? e_pair : scratch + part;
    if (cc::energy_pairs(o, v, R, t2, scratch, ep, st) != cudaSuccess) return CC_ERR_CUDA;
    if (cc::energy_total((long long)o * o, ep, energy, st) != cudaSuccess) return CC_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}
