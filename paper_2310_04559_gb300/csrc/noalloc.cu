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
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <cuda_runtime.h>

#include <mutex>

#include "cc_internal.cuh"

namespace {

constexpr long long kScratchDoubles = 1ll << 21;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of g_energy_scratch, per device

}  // namespace

extern "C" int cc_ladder_energy_noalloc(int o, int v, const double* R, const double* t2, double* energy,
                                        double* e_pair, void* stream)
{
    if (o < 1 || v < 1) return CC_ERR_SHAPE;
    if (!R || !t2 || !energy) return CC_ERR_NULL;
    if (((uintptr_t)R % 16) || ((uintptr_t)t2 % 16) || ((uintptr_t)energy % 8) || (e_pair && ((uintptr_t)e_pair % 8)))
        return CC_ERR_ALIGN;
    const long long part = cc::energy_scratch_doubles(o, v);
    const long long need = part + (e_pair ? 0 : (long long)o * o);
    if (need > kScratchDoubles) return CC_ERR_NOALLOC_LIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CC_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) return CC_ERR_CUDA;
            g_scratch_ptr[dev] = (double*)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    // Every partial the two kernels read is written earlier in the same call, so the
    // array needs no clearing.
    cudaStream_t st = (cudaStream_t)stream;
    double* ep = e_pair ? e_pair : scratch + part;
    if (cc::energy_pairs(o, v, R, t2, scratch, ep, st) != cudaSuccess) return CC_ERR_CUDA;
    if (cc::energy_total(o * o, ep, energy, st) != cudaSuccess) return CC_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}
