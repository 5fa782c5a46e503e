// split.cu -- operand preparation for the tensor-core slice GEMM.
//
// Ozaki-style splitting (error-free transformation of an FP64 matrix into a sum
// of low-precision matrices with a per-row power-of-two scale): every row x of
// an FP64 operand is scaled by 2^-e with max|x| < 2^e, rounded ONCE to a signed
// integer X with |X| <= 2^(beta*s-1), and X is cut into s balanced base-2^beta
// digits d_0 (most significant) .. d_{s-1}:
//
//     x ~= sum_k d_k * 2^(e - beta + 1 - beta*k),   |d_k| <= 2^(beta-1).
//
// Digits of at most 2^8 in magnitude are exact in bf16, so a product of two
// digit matrices summed on the tensor cores in FP32 is an exact integer while
// the partial sums stay below 2^24.
//
// GB300 executes FP64 arithmetic at a small fraction of its integer rate, so
// the whole transformation is done on the IEEE-754 bit pattern with 64-bit
// integer operations: the only FP64->integer step is the reinterpretation of
// the bits.  Rows are split either from a K-contiguous source (t2, integral
// blocks) or from a row-contiguous source (Cholesky vectors L[P][a][c], whose
// GEMM rows (a,c) are contiguous and whose K index P is strided), the latter
// through a shared-memory transpose.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;  // |x| bit patterns >= this are Inf or NaN

// Exponent e with max|row| < 2^e from the largest |x| bit pattern (0 for a zero row).
__device__ __forceinline__ int row_exponent(unsigned long long maxbits)
{
    if (maxbits == 0) return 0;
    const int ex = (int)(maxbits >> 52);
    return ex == 0 ? -1022 : ex - 1022;
}

// X = round(x * 2^(total_bits - 1 - e)) as a signed 64-bit integer.
__device__ __forceinline__ long long fixed_point(double x, int e, int total_bits)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0x000fffffffffffffull;
    if (ex == 0 && mant == 0) return 0;
    int exe = ex;
    if (ex == 0) exe = 1; else mant |= 0x0010000000000000ull;
    // x = mant * 2^(exe - 1075)
    const int sh = exe - 1075 + total_bits - 1 - e;
    long long X;
    if (sh >= 0) X = (long long)(mant << sh);
    else if (sh > -64) X = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    else X = 0;
    return (bits >> 63) ? -X : X;
}

// bf16 bit pattern of a small integer (|d| <= 256, exact): the float 1.5*2^23 + d has unit
// spacing, so subtracting 1.5*2^23 gives d exactly, and d has at most 8 significant bits.
__device__ __forceinline__ unsigned short bf16_small(int d)
{
    return (unsigned short)(__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16);
}

// Writes the s balanced base-2^beta digits of X (d_0 most significant, |X| <= 2^(beta s - 1))
// as bf16.  With H = half * sum_{k<s} 2^(beta k), X + H holds every digit plus `half` as a
// plain base-2^beta digit, so each digit is one shift and mask (no carry chain).
__device__ __forceinline__ void digits_bf16(long long X, int s, int beta, __nv_bfloat16* out, long long slice_stride)
{
    long long H = 0;
    for (int k = 0; k < s; ++k) H = (H << beta) | (1ll << (beta - 1));
    const unsigned long long Y = (unsigned long long)(X + H);
    const int half = 1 << (beta - 1), mask = (1 << beta) - 1;
    unsigned short* o = (unsigned short*)out;
    o[0] = bf16_small((int)(Y >> (beta * (s - 1))) - half);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        if (k >= s) break;
        o[k * slice_stride] = bf16_small(((int)(Y >> (beta * (s - 1 - k))) & mask) - half);
    }
}

template <int TPR>  // threads per row: 256 (one CTA per row) or 32 (one warp per row)
__global__ void split_rows_kernel(const RowSrc src, int s, int beta, __nv_bfloat16* __restrict__ D, long long pitch,
                                  int* __restrict__ e_out, int* __restrict__ status)
{
    __shared__ unsigned long long red[256];
    const int lane = threadIdx.x % TPR;
    const long long r = (long long)blockIdx.x * (256 / TPR) + threadIdx.x / TPR;
    const bool live = r < src.rows;
    const double* X = src.X + (live ? map2(src.rm, r) : 0);
    const long long K = src.K;
    const long long slice_stride = src.rows * pitch;
    __nv_bfloat16* Dr = D + r * pitch;

    if (s == 0) {  // plain bf16 copy, unit scale
        if (live) {
            for (long long k = lane; k < K; k += TPR) Dr[k] = __double2bfloat16(X[map2(src.km, k)]);
            if (lane == 0) e_out[r] = 0;
        }
        return;
    }
    unsigned long long mx = 0;
    if (live)
        for (long long k = lane; k < K; k += TPR) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(X[map2(src.km, k)]) & kAbsMask;
            mx = b > mx ? b : mx;
        }
    if (TPR == 32) {
        for (int w = 16; w > 0; w >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, w);
            mx = o > mx ? o : mx;
        }
    } else {
        red[threadIdx.x] = mx;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x] > red[threadIdx.x + w] ? red[threadIdx.x] : red[threadIdx.x + w];
            __syncthreads();
        }
        mx = red[0];
    }
    if (!live) return;
    const int e = row_exponent(mx);
    if (lane == 0) {
        e_out[r] = e;
        if (status && mx >= kInfBits) atomicOr(status, kStatusNonfinite);
    }
    const int total = beta * s;
    for (long long k = lane; k < K; k += TPR)
        digits_bf16(fixed_point(X[map2(src.km, k)], e, total), s, beta, Dr + k, slice_stride);
}

__device__ __forceinline__ long long col_off(const ColSrc& s, long long r)
{
    if (s.brows == 0) return r;
    return map2(s.bmap, r / s.brows) + r % s.brows;
}

// Column-source max: mx[r] = max_k |X[r + k*ldk]| (bit pattern), atomically over k-chunks.
__global__ void col_max_kernel(const ColSrc src, long long kchunk, unsigned long long* __restrict__ mx,
                               int* __restrict__ status)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= src.rows) return;
    const long long roff = col_off(src, r);
    unsigned long long m = 0;
    // chunks blockIdx.y, blockIdx.y + gridDim.y, ... (gridDim.y is capped at 65535)
    for (long long k0 = (long long)blockIdx.y * kchunk; k0 < src.K; k0 += (long long)gridDim.y * kchunk) {
        const long long k1 = min(src.K, k0 + kchunk);
        for (long long k = k0; k < k1; ++k) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(src.X[roff + k * src.ldk]) & kAbsMask;
            m = b > m ? b : m;
        }
    }
    if (m) atomicMax(mx + r, m);
    if (status && m >= kInfBits) atomicOr(status, kStatusNonfinite);
}

constexpr int CT_R = 32, CT_K = 32;  // transpose tile: 32 rows x 32 k

// Transposing split: tile of 32 rows x 32 k; reads are coalesced along rows,
// digit writes along k.
__global__ void split_cols_kernel(const ColSrc src, int s, int beta, const unsigned long long* __restrict__ mx,
                                  __nv_bfloat16* __restrict__ D, long long pitch, int* __restrict__ e_out)
{
    __shared__ double S[CT_K][CT_R + 1];
    const long long r0 = (long long)blockIdx.x * CT_R;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const long long slice_stride = src.rows * pitch;
    // k tiles blockIdx.y, blockIdx.y + gridDim.y, ... (gridDim.y is capped at 65535)
    for (long long k0 = (long long)blockIdx.y * CT_K; k0 < src.K; k0 += (long long)gridDim.y * CT_K) {
        __syncthreads();
        for (int y = ty; y < CT_K; y += 8) {
            const long long k = k0 + y, r = r0 + tx;
            S[y][tx] = (k < src.K && r < src.rows) ? src.X[col_off(src, r) + k * src.ldk] : 0.0;
        }
        __syncthreads();
        for (int y = ty; y < CT_R; y += 8) {
            const long long r = r0 + y, k = k0 + tx;
            if (r >= src.rows || k >= src.K) continue;
            const double x = S[tx][y];
            __nv_bfloat16* out = D + r * pitch + k;
            if (s == 0) {
                out[0] = __double2bfloat16(x);
                if (k == 0) e_out[r] = 0;
                continue;
            }
            const int e = row_exponent(mx[r]);
            if (k == 0) e_out[r] = e;
            digits_bf16(fixed_point(x, e, beta * s), s, beta, out, slice_stride);
        }
    }
}

// X * 2^sh rounded to an integer (round half up for right shifts); |result| < 2^62.
__device__ __forceinline__ long long shift_round(long long X, int sh)
{
    if (sh >= 0) return X << sh;
    if (sh <= -63) return 0;
    return (X + (1ll << (-sh - 1))) >> (-sh);
}

// One CTA (8 warps) per row; warp w walks outer indices w, w+8, ..., lanes the inner index.
__global__ void split_fixed_kernel(const FixedSrc src, int s, int beta, __nv_bfloat16* __restrict__ D, long long pitch,
                                   int* __restrict__ e_out)
{
    extern __shared__ int esm[];  // outer entries of eA, then inner entries of eB
    __shared__ int red[8];
    const long long r = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long ab = map2(src.amap, r), bb = map2(src.bmap, r);
    for (int q = threadIdx.x; q < src.outer; q += 256) esm[q] = src.eA[ab + q];
    for (int q = threadIdx.x; q < src.inner; q += 256) esm[src.outer + q] = src.eB[bb + q];
    __syncthreads();
    const int* eo = esm;
    const int* ei = esm + src.outer;
    const long long* Xr = src.X + r * src.ldx;
    // pass 1: E = max over the row of bitlength(|X|) + e, so that max |value| < 2^E
    int mx = INT_MIN;
    for (int o = warp; o < src.outer; o += 8) {
        const long long* Xo = Xr + (long long)o * src.inner;
        for (int i = lane; i < src.inner; i += 32) {
            const long long x = __ldcs(Xo + i);
            if (x) {
                const unsigned long long ax = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
                const int c = 64 - __clzll((long long)ax) + eo[o] + ei[i];
                mx = c > mx ? c : mx;
            }
        }
    }
    for (int w = 16; w > 0; w >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, w));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = red[0];
        for (int w = 1; w < 8; ++w) m = max(m, red[w]);
        red[0] = m;
    }
    __syncthreads();
    const bool zero = red[0] == INT_MIN;
    const int E = zero ? 0 : red[0] + src.base;
    if (threadIdx.x == 0) e_out[r] = E;
    // pass 2: digits of round(value * 2^(beta*s - 1 - E))
    const int total = beta * s;
    const long long slice_stride = src.rows * pitch;
    __nv_bfloat16* Dr = D + r * pitch;
    for (int o = warp; o < src.outer; o += 8) {
        const long long* Xo = Xr + (long long)o * src.inner;
        for (int i = lane; i < src.inner; i += 32) {
            const long long x = zero ? 0 : __ldcs(Xo + i);
            const long long X = shift_round(x, eo[o] + ei[i] + src.base + total - 1 - E);
            digits_bf16(X, s, beta, Dr + (long long)o * src.inner + i, slice_stride);
        }
    }
}

__device__ __forceinline__ float to_tf32(double x)
{
    const float f = (float)x;
    unsigned int u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
    return __uint_as_float(u);
}

__global__ void convert_rows_tf32_kernel(const RowSrc src, float* __restrict__ D, long long pitch)
{
    const long long r = blockIdx.x;
    const double* X = src.X + map2(src.rm, r);
    for (long long k = threadIdx.x; k < src.K; k += blockDim.x) D[r * pitch + k] = to_tf32(X[map2(src.km, k)]);
}

__global__ void convert_cols_tf32_kernel(const ColSrc src, float* __restrict__ D, long long pitch)
{
    __shared__ double S[CT_K][CT_R + 1];
    const long long r0 = (long long)blockIdx.x * CT_R;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (long long k0 = (long long)blockIdx.y * CT_K; k0 < src.K; k0 += (long long)gridDim.y * CT_K) {
        __syncthreads();
        for (int y = ty; y < CT_K; y += 8) {
            const long long k = k0 + y, r = r0 + tx;
            S[y][tx] = (k < src.K && r < src.rows) ? src.X[col_off(src, r) + k * src.ldk] : 0.0;
        }
        __syncthreads();
        for (int y = ty; y < CT_R; y += 8) {
            const long long r = r0 + y, k = k0 + tx;
            if (r < src.rows && k < src.K) D[r * pitch + k] = to_tf32(S[tx][y]);
        }
    }
}

}  // namespace

cudaError_t split_rows_bf16(const RowSrc& src, int s, int beta, void* D, long long pitch, int* e, int* status,
                            cudaStream_t st)
{
    if (src.rows <= 0) return cudaSuccess;
    if (s < 0 || s > 8 || (s > 0 && (beta < 2 || beta > 9 || beta * s > 62))) return cudaErrorInvalidValue;
    if (src.K >= 4096) {
        split_rows_kernel<256><<<(unsigned)src.rows, 256, 0, st>>>(src, s, beta, (__nv_bfloat16*)D, pitch, e, status);
    } else {
        split_rows_kernel<32><<<(unsigned)((src.rows + 7) / 8), 256, 0, st>>>(src, s, beta, (__nv_bfloat16*)D, pitch, e,
                                                                             status);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t cols_max(const ColSrc& src, unsigned long long* mx, int* status, cudaStream_t st)
{
    if (src.rows <= 0 || src.K <= 0) return cudaSuccess;
    const long long kchunk = 256;
    dim3 g((unsigned)((src.rows + 255) / 256), (unsigned)std::min(65535ll, (src.K + kchunk - 1) / kchunk));
    col_max_kernel<<<g, 256, 0, st>>>(src, kchunk, mx, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t split_cols_bf16(const ColSrc& src, int s, int beta, void* D, long long pitch, int* e,
                            unsigned long long* scratch_max, int* status, cudaStream_t st, bool premax)
{
    if (src.rows <= 0) return cudaSuccess;
    if (s < 0 || s > 8 || (s > 0 && (beta < 2 || beta > 9 || beta * s > 62))) return cudaErrorInvalidValue;
    if (s > 0 && !premax) {
        cudaError_t err = cudaMemsetAsync(scratch_max, 0, sizeof(unsigned long long) * src.rows, st);
        if (err != cudaSuccess) return err;
        err = cols_max(src, scratch_max, status, st);
        if (err != cudaSuccess) return err;
    }
    dim3 g2((unsigned)((src.rows + CT_R - 1) / CT_R), (unsigned)std::min(65535ll, (src.K + CT_K - 1) / CT_K));
    split_cols_kernel<<<g2, dim3(32, 8), 0, st>>>(src, s, beta, scratch_max, (__nv_bfloat16*)D, pitch, e);
    count_launch();
    return cudaGetLastError();
}

cudaError_t split_fixed_rows_bf16(const FixedSrc& src, int s, int beta, void* D, long long pitch, int* e,
                                  cudaStream_t st)
{
    if (src.rows <= 0) return cudaSuccess;
    if (s < 1 || s > 8 || beta < 2 || beta > 9 || beta * s > 62) return cudaErrorInvalidValue;
    const size_t smem = sizeof(int) * ((size_t)src.outer + src.inner);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {  // opt in to the larger dynamic shared memory
        const cudaError_t e =
            cudaFuncSetAttribute(split_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    split_fixed_kernel<<<(unsigned)src.rows, 256, smem, st>>>(src, s, beta, (__nv_bfloat16*)D, pitch, e);
    count_launch();
    return cudaGetLastError();
}

cudaError_t convert_rows_tf32(const RowSrc& src, float* D, long long pitch, cudaStream_t st)
{
    if (src.rows <= 0) return cudaSuccess;
    convert_rows_tf32_kernel<<<(unsigned)src.rows, 256, 0, st>>>(src, D, pitch);
    count_launch();
    return cudaGetLastError();
}

cudaError_t convert_cols_tf32(const ColSrc& src, float* D, long long pitch, cudaStream_t st)
{
    if (src.rows <= 0) return cudaSuccess;
    dim3 g2((unsigned)((src.rows + CT_R - 1) / CT_R), (unsigned)std::min(65535ll, (src.K + CT_K - 1) / CT_K));
    convert_cols_tf32_kernel<<<g2, dim3(32, 8), 0, st>>>(src, D, pitch);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
