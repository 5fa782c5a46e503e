// gemm_f64.cu -- FP64 GEMM on the FP64 tensor-core instruction (DMMA,
// mma.sync.m8n8k4.f64) for the plain-FP64 precision mode.
//
// Computes C[rmap(m) + cmap(n)] (= or +=) sum_k A(m,k) B(n,k) for the two
// contractions of the integral-first order (Section 3.2): the integral block
// (ac|bd) = sum_P L_Pac L_Pbd (Eq. 5) and the ladder GEMM sum_cd (ac|bd) t_ijcd
// (Eq. 6), and for the adjoint's contractions.
//
// GB300 executes FP64 at a small fraction of its BF16 rate, so this kernel is
// bound by the FP64 pipe at any reasonable tiling: 64x64 CTA tiles, 4 warps of
// 32x32, k-tiles of 16 staged through shared memory with a register prefetch.
#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int BM = 64, BN = 64, BKT = 16, THREADS = 128;

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// Loads one BM x BKT (or BN x BKT) tile into registers.  KMAJ: k contiguous in
// memory -> thread t takes row t/2 and 8 consecutive k; otherwise rows are
// contiguous -> thread t takes row t%64 and 8 k values.
template <bool KMAJ>
struct TileLoader {
    long long rowoff;  // map of this thread's row (or -1 if out of range)
    int r, kofs;
    __device__ void init(const Map2& rm, int row0, int nrows)
    {
        const int t = threadIdx.x;
        if (KMAJ) { r = t >> 1; kofs = (t & 1) * 8; }
        else      { r = t & 63; kofs = (t >> 6) * 8; }
        rowoff = (row0 + r < nrows) ? map2(rm, row0 + r) : -1;
    }
    __device__ void load(const double* __restrict__ X, const Map2& km, int k0, int K, double (&v)[8]) const
    {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + kofs + q;
            v[q] = (rowoff >= 0 && k < K) ? __ldg(X + rowoff + map2(km, k)) : 0.0;
        }
    }
    __device__ void store(double (*S)[BM + 1], const double (&v)[8]) const
    {
#pragma unroll
        for (int q = 0; q < 8; ++q) S[kofs + q][r] = v[q];
    }
};

template <bool AK, bool BK>
__global__ void __launch_bounds__(THREADS) gemm_f64_kernel(const GemmF64 g)
{
    __shared__ double As[2][BKT][BM + 1];
    __shared__ double Bs[2][BKT][BN + 1];

    // one-dimensional grid over the tiles (no gridDim.y limit on M)
    const int tiles_n = (g.N + BN - 1) / BN;
    const int m0 = (int)(blockIdx.x / tiles_n) * BM, n0 = (int)(blockIdx.x % tiles_n) * BN;
    if (g.tri > 0 && (long long)min(g.N - 1, n0 + BN - 1) / g.tri < (long long)m0 / g.tri) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    TileLoader<AK> la;
    TileLoader<BK> lb;
    la.init(g.am, m0, g.M);
    lb.init(g.bm, n0, g.N);

    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    double ra[8], rb[8];
    la.load(g.A, g.ak, 0, g.K, ra);
    lb.load(g.B, g.bk, 0, g.K, rb);
    la.store(As[0], ra);
    lb.store(Bs[0], rb);
    __syncthreads();

    const int nk = (g.K + BKT - 1) / BKT;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) {
            la.load(g.A, g.ak, (kt + 1) * BKT, g.K, ra);
            lb.load(g.B, g.bk, (kt + 1) * BKT, g.K, rb);
        }
#pragma unroll
        for (int kk = 0; kk < BKT; kk += 4) {
            double fa[4], fb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) fa[i] = As[cur][kk + (lane & 3)][wm + i * 8 + (lane >> 2)];
#pragma unroll
            for (int j = 0; j < 4; ++j) fb[j] = Bs[cur][kk + (lane & 3)][wn + j * 8 + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) dmma(acc[i][j], fa[i], fb[j]);
        }
        if (kt + 1 < nk) {
            la.store(As[cur ^ 1], ra);
            lb.store(Bs[cur ^ 1], rb);
        }
        __syncthreads();
    }

    // D fragment: row lane/4, columns 2*(lane%4) + {0,1} of each 8x8 sub-tile.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + wm + i * 8 + (lane >> 2);
        if (m >= g.M) continue;
        const long long ro = map2(g.out.rmap, m);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n = n0 + wn + j * 8 + (lane & 3) * 2 + h;
                if (n >= g.N) continue;
                double* p = g.out.C + ro + map2(g.out.cmap, n);
                *p = g.out.accumulate ? *p + acc[i][j][h] : acc[i][j][h];
            }
        }
    }
}

}  // namespace

cudaError_t gemm_f64(const GemmF64& g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const bool ak = (g.ak.div == 0 && !g.ak.tab && g.ak.s1 == 1);
    const bool bk = (g.bk.div == 0 && !g.bk.tab && g.bk.s1 == 1);
    const long long tiles = (long long)((g.N + BN - 1) / BN) * ((g.M + BM - 1) / BM);
    if (tiles > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)tiles);
    if (ak && bk) gemm_f64_kernel<true, true><<<grid, THREADS, 0, s>>>(g);
    else if (ak && !bk) gemm_f64_kernel<true, false><<<grid, THREADS, 0, s>>>(g);
    else if (!ak && bk) gemm_f64_kernel<false, true><<<grid, THREADS, 0, s>>>(g);
    else gemm_f64_kernel<false, false><<<grid, THREADS, 0, s>>>(g);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
