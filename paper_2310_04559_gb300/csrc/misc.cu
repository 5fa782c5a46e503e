// misc.cu -- memory-bound helpers around the two contractions: the closed-shell
// pair energy, the scatter of pair-symmetric results, and batched v x v
// transposes.  All transposes stage 32x32 tiles through shared memory so that
// both the read and the write are coalesced.
#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int T = 32;  // tile edge
constexpr int TR = 8;  // rows of threads per tile (block = 32 x 8)

// (i, j) of pair index p in the i-major enumeration of i <= j.
__device__ __forceinline__ void pair_of(int o, int p, int& i, int& j)
{
    int ii = 0, rem = p;
    while (rem >= o - ii) { rem -= o - ii; ++ii; }
    i = ii;
    j = ii + rem;
}

// Index of this block in a batch spread over gridDim.y x gridDim.z (see batch_grid).
__device__ __forceinline__ long long batch_index() { return (long long)blockIdx.y + (long long)blockIdx.z * gridDim.y; }

// E_ij = sum_ab (2 R_ijab - R_ijba) t_ijab for one (i,j) per batch index, over the terms
// with lo <= min(a, b) < hi (all of them for lo = 0, hi = v); partial per 32x32 (a,b) tile
// written to part[ij][tile]; a second kernel sums them.
__global__ void energy_tiles_kernel(long long npairs, int v, int lo, int hi, const double* __restrict__ R,
                                    const double* __restrict__ t2, double* __restrict__ part)
{
    __shared__ double Rt[T][T + 1];
    __shared__ double red[T * TR];
    const long long ij = batch_index();
    if (ij >= npairs) return;
    const int ntile = (v + T - 1) / T;
    const int ta = blockIdx.x / ntile, tb = blockIdx.x % ntile;
    const double* Rij = R + ij * (long long)v * v;
    const double* tij = t2 + ij * (long long)v * v;
    const int a0 = ta * T, b0 = tb * T;
    // mirrored tile: Rt[b - b0][a - a0] = R[ij, b, a]
    for (int y = threadIdx.y; y < T; y += TR) {
        const int b = b0 + y, a = a0 + threadIdx.x;
        Rt[y][threadIdx.x] = (b < v && a < v) ? Rij[(long long)b * v + a] : 0.0;
    }
    __syncthreads();
    double s = 0.0;
    for (int y = threadIdx.y; y < T; y += TR) {
        const int a = a0 + y, b = b0 + threadIdx.x;
        const int m = a < b ? a : b;  // terms owned by the range [lo, hi): min(a, b) inside it
        if (a < v && b < v && m >= lo && m < hi) {
            const long long q = (long long)a * v + b;
            s += (2.0 * Rij[q] - Rt[threadIdx.x][y]) * tij[q];
        }
    }
    const int tid = threadIdx.y * T + threadIdx.x;
    red[tid] = s;
    __syncthreads();
    for (int w = (T * TR) / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) part[ij * (long long)gridDim.x + blockIdx.x] = red[0];
}

// Deterministic sum of `len` values per row of `x` (rows = gridDim.x) into y.
__global__ void row_sum_kernel(long long len, const double* __restrict__ x, double* __restrict__ y)
{
    __shared__ double red[256];
    const double* xr = x + (long long)blockIdx.x * len;
    double s = 0.0;
    for (long long q = threadIdx.x; q < len; q += 256) s += xr[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[blockIdx.x] = red[0];
}

// Y[b][c][d] = X[b][d][c] over batch b (blockIdx.z / y split), v x v each.
__global__ void transpose_kernel(long long batch, int v, const double* __restrict__ X, double* __restrict__ Y)
{
    __shared__ double S[T][T + 1];
    const int ntile = (v + T - 1) / T;
    const int tr = blockIdx.x / ntile, tc = blockIdx.x % ntile;
    const long long b = batch_index();
    if (b >= batch) return;
    const double* Xb = X + b * (long long)v * v;
    double* Yb = Y + b * (long long)v * v;
    // read X[d][c] rows d in tile tr, cols c in tile tc
    for (int y = threadIdx.y; y < T; y += TR) {
        const int d = tr * T + y, c = tc * T + threadIdx.x;
        if (d < v && c < v) S[y][threadIdx.x] = Xb[(long long)d * v + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < T; y += TR) {
        const int c = tc * T + y, d = tr * T + threadIdx.x;
        if (d < v && c < v) Yb[(long long)c * v + d] = S[threadIdx.x][y];
    }
}

// R[i,j,a,b] (=|+=) Rc[p,a,b]; for i < j also R[j,i,b,a] (=|+=) Rc[p,a,b]; a in [a_lo, a_hi).
__global__ void scatter_pairs_kernel(int o, int v, int a_lo, int a_hi, const double* __restrict__ Rc,
                                     double* __restrict__ R, int accumulate)
{
    __shared__ double S[T][T + 1];
    const long long pb = batch_index();
    if (pb >= (long long)o * (o + 1) / 2) return;  // uniform over the block
    const int ntile = (v + T - 1) / T;
    const int ta = blockIdx.x / ntile, tb = blockIdx.x % ntile;
    const int a0 = a_lo + ta * T;
    const int p = (int)pb;
    int i, j;
    pair_of(o, p, i, j);
    const long long vv = (long long)v * v;
    const double* Rp = Rc + (long long)p * vv;
    double* Rij = R + ((long long)i * o + j) * vv;
    double* Rji = R + ((long long)j * o + i) * vv;
    for (int y = threadIdx.y; y < T; y += TR) {
        const int a = a0 + y, b = tb * T + threadIdx.x;
        if (a < a_hi && b < v) {
            const long long q = (long long)a * v + b;
            const double x = Rp[q];
            S[y][threadIdx.x] = x;
            Rij[q] = accumulate ? Rij[q] + x : x;
        }
    }
    if (i == j) return;
    __syncthreads();
    for (int y = threadIdx.y; y < T; y += TR) {
        const int b = tb * T + y, a = a0 + threadIdx.x;
        if (a < a_hi && b < v) {
            const long long q = (long long)b * v + a;
            const double x = S[threadIdx.x][y];
            Rji[q] = accumulate ? Rji[q] + x : x;
        }
    }
}

// Y[i,j,a,b] = alpha * X[i,j,a,b] + X[j,i,b,a]
__global__ void add_pair_swap_kernel(int o, int v, const double* __restrict__ X, double* __restrict__ Y, int alpha)
{
    __shared__ double S[T][T + 1];
    const long long ij = batch_index();
    if (ij >= (long long)o * o) return;
    const int ntile = (v + T - 1) / T;
    const int ta = blockIdx.x / ntile, tb = blockIdx.x % ntile;
    const int i = (int)(ij / o), j = (int)(ij % o);
    const long long vv = (long long)v * v;
    const double* Xji = X + ((long long)j * o + i) * vv;
    const double* Xij = X + (long long)ij * vv;
    double* Yij = Y + (long long)ij * vv;
    // S[b - b0][a - a0] = X[j,i,b,a]
    for (int y = threadIdx.y; y < T; y += TR) {
        const int b = tb * T + y, a = ta * T + threadIdx.x;
        if (a < v && b < v) S[y][threadIdx.x] = Xji[(long long)b * v + a];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < T; y += TR) {
        const int a = ta * T + y, b = tb * T + threadIdx.x;
        if (a < v && b < v) {
            const long long q = (long long)a * v + b;
            Yij[q] = alpha ? Xij[q] + S[threadIdx.x][y] : S[threadIdx.x][y];
        }
    }
}

__global__ void fill_pair_table_kernel(int o, long long vv, long long* tab)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= o * (o + 1) / 2) return;
    int i, j;
    pair_of(o, p, i, j);
    tab[p] = ((long long)i * o + j) * vv;
}

// Grid for `batch` independent blocks of ntile2 tiles: batch index = y + z * gridDim.y, with
// gridDim.y and gridDim.z within the 65535 limit for any batch up to 65535^2 (blocks with an
// index beyond the batch return at once).
dim3 batch_grid(int ntile2, long long batch)
{
    const long long gz = (batch + 65534) / 65535;
    const long long gy = (batch + gz - 1) / gz;
    return dim3(ntile2, (unsigned)(gy > 0 ? gy : 1), (unsigned)(gz > 0 ? gz : 1));
}

}  // namespace

cudaError_t energy_pairs(int o, int v, const double* R, const double* t2, double* part, double* e_pair,
                         cudaStream_t s, int lo, int hi)
{
    if (hi < 0) hi = v;
    const int ntile = (v + T - 1) / T;
    const long long np = (long long)o * o;
    energy_tiles_kernel<<<batch_grid(ntile * ntile, np), dim3(T, TR), 0, s>>>(np, v, lo, hi, R, t2, part);
    row_sum_kernel<<<(unsigned)np, 256, 0, s>>>((long long)ntile * ntile, part, e_pair);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t energy_total(long long npairs, const double* e_pair, double* E, cudaStream_t s)
{
    row_sum_kernel<<<1, 256, 0, s>>>(npairs, e_pair, E);
    count_launch();
    return cudaGetLastError();
}

cudaError_t scatter_pairs(int o, int v, int a_lo, int a_hi, const double* Rc, double* R, int accumulate,
                          cudaStream_t s)
{
    const int ntile = (v + T - 1) / T;
    const int ntile_a = (a_hi - a_lo + T - 1) / T;
    const long long np = (long long)o * (o + 1) / 2;
    scatter_pairs_kernel<<<batch_grid(ntile_a * ntile, np), dim3(T, TR), 0, s>>>(o, v, a_lo, a_hi, Rc, R, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t swap_last2(long long batch, int v, const double* X, double* Y, cudaStream_t s)
{
    const int ntile = (v + T - 1) / T;
    transpose_kernel<<<batch_grid(ntile * ntile, batch), dim3(T, TR), 0, s>>>(batch, v, X, Y);
    count_launch();
    return cudaGetLastError();
}

cudaError_t transpose_last2(long long batch, int v, const double* X, double* Y, cudaStream_t s)
{
    return swap_last2(batch, v, X, Y, s);
}

cudaError_t add_pair_swap(int o, int v, const double* X, double* Y, int alpha, cudaStream_t s)
{
    const int ntile = (v + T - 1) / T;
    add_pair_swap_kernel<<<batch_grid(ntile * ntile, (long long)o * o), dim3(T, TR), 0, s>>>(o, v, X, Y, alpha);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fill_pair_table(int o, int v, long long* tab, cudaStream_t s)
{
    const int np = o * (o + 1) / 2;
    fill_pair_table_kernel<<<(np + 127) / 128, 128, 0, s>>>(o, (long long)v * v, tab);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
