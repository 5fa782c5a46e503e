// pm.cu -- symmetric / antisymmetric packing of the pair-symmetric ladder.
//
// For amplitudes with t[i,j,c,d] = t[j,i,d,c] the ladder term splits into a part
// symmetric and a part antisymmetric under c <-> d (closed-shell CC codes call these
// the t+ / t- amplitudes).  With V_ab[c,d] = (ac|bd) (Eq. 5) and, for c < d,
//
//     T+[ij][c<=d] = t_ijcd + t_ijdc  (t_ijcc on the diagonal)
//     T-[ij][c< d] = t_ijcd - t_ijdc
//     V+[ab][c<=d] = (V_ab[c,d] + V_ab[d,c]) / 2  (V_ab[c,c] on the diagonal)
//     V-[ab][c< d] = (V_ab[c,d] - V_ab[d,c]) / 2
//
// the sum of Eq. 6 is  sum_cd t_ijcd V_ab[c,d] = R+_ijab + R-_ijab  with
// R+ = sum_{c<=d} T+ V+ and R- = sum_{c<d} T- V-.  Because (ac|bd) = (bd|ac),
// V+ is symmetric and V- antisymmetric under a <-> b; T+ is symmetric and T-
// antisymmetric under i <-> j.  Hence R+ is needed for i <= j, a <= b only, R-
// for i < j, a < b only, and
//
//     R[i,j,a,b] = R[j,i,b,a] = R+ + R-,    R[j,i,a,b] = R[i,j,b,a] = R+ - R-.
//
// The two ladder GEMMs then have K = v(v+1)/2 and v(v-1)/2 and about o^2/2 rows,
// a quarter of the unpacked product each.  Packed column index of (c, d):
//     kp(c,d) = c*v - c(c-1)/2 + (d - c)       (c <= d, v(v+1)/2 entries)
//     km(c,d) = c*(v-1) - c(c-1)/2 + (d - c - 1)  (c < d, v(v-1)/2 entries)
//
// Rows of the integral block used here are the pairs (a, b) with b >= a of a block
// a0 <= a < a0 + A, b in [a0, v): packed row r = rowbase(al) + (b' - al) with
// al = a - a0, b' = b - a0, Nb = v - a0 and rowbase(al) = al*Nb - al(al-1)/2.
//
// Every v x v matrix is visited as pairs of 32 x 32 tiles (C, D) and (D, C) staged
// in shared memory, so that X[c][d] and X[d][c] are both read coalesced.
#include <cuda_bf16.h>

#include <climits>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int TT = 32;   // tile edge
constexpr int TY = 8;    // thread rows per tile (256 threads)
constexpr unsigned long long kAbs = 0x7fffffffffffffffull;

__device__ __forceinline__ long long kp_of(long long c, long long d, long long v) { return c * v - c * (c - 1) / 2 + (d - c); }
__device__ __forceinline__ long long km_of(long long c, long long d, long long v)
{
    return c * (v - 1) - c * (c - 1) / 2 + (d - c - 1);
}

// bf16 bit pattern of a small integer (|d| <= 256, exact): the float 1.5*2^23 + d has unit
// spacing, so subtracting 1.5*2^23 gives d exactly, and d has at most 8 significant bits.
__device__ __forceinline__ unsigned short bf16_small(int d)
{
    return (unsigned short)(__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16);
}

// H = half * sum_{k<s} 2^(beta k): X + H holds the balanced digits of X plus `half` each as
// plain base-2^beta digits (no carries to propagate), for |X| <= 2^(beta s - 1) < H.
__device__ __forceinline__ long long digit_bias(int s, int beta)
{
    long long H = 0;
    for (int k = 0; k < s; ++k) H = (H << beta) | (1ll << (beta - 1));
    return H;
}

// Balanced base-2^beta digits of X (d_0 most significant) as bf16, same convention as
// the row splits: x ~= sum_k d_k 2^(e - beta + 1 - beta k) for X = round(x 2^(beta s - 1 - e)).
__device__ __forceinline__ void put_digits(long long X, long long H, int s, int beta, __nv_bfloat16* out,
                                           long long stride)
{
    const unsigned long long Y = (unsigned long long)(X + H);
    const int half = 1 << (beta - 1), mask = (1 << beta) - 1;
    unsigned short* o = (unsigned short*)out;
    o[0] = bf16_small((int)(Y >> (beta * (s - 1))) - half);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        if (k >= s) break;
        o[k * stride] = bf16_small(((int)(Y >> (beta * (s - 1 - k))) & mask) - half);
    }
}

// X * 2^sh rounded to an integer (round half up on right shifts).
__device__ __forceinline__ long long shr_round(long long X, int sh)
{
    if (sh >= 0) return X << sh;
    if (sh <= -63) return 0;
    return (X + (1ll << (-sh - 1))) >> (-sh);
}

// round(x * 2^(total - 1 - e)) from the bit pattern of x (|x| < 2^e).
__device__ __forceinline__ long long fixed_of(double x, int e, int total)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0x000fffffffffffffull;
    if (ex == 0 && mant == 0) return 0;
    int exe = ex;
    if (ex == 0) exe = 1; else mant |= 0x0010000000000000ull;
    const int sh = exe - 1075 + total - 1 - e;
    long long X;
    if (sh >= 0) X = (long long)(mant << sh);
    else if (sh > -64) X = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    else X = 0;
    return (bits >> 63) ? -X : X;
}

__device__ __forceinline__ int exp_of_maxbits(unsigned long long b)
{
    if (b == 0) return 0;
    const int ex = (int)(b >> 52);
    return ex == 0 ? -1022 : ex - 1022;
}

__device__ __forceinline__ float tf32_of(double x)
{
    const float f = (float)x;
    unsigned int u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
    return __uint_as_float(u);
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long m, unsigned long long* red)
{
    for (int w = 16; w > 0; w >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, w);
        m = o > m ? o : m;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    unsigned long long r = red[0];
    for (int w = 1; w < 8; ++w) r = red[w] > r ? red[w] : r;
    return r;
}

// Value of the packed entry (c, d) of one sign from x1 = X[c][d], x2 = X[d][c].
__device__ __forceinline__ double pm_value(double x1, double x2, bool diag, int sign, double h)
{
    if (diag) return x1;
    return sign > 0 ? (x1 + x2) * h : (x1 - x2) * h;
}

// FP64 source: one row r is the v x v matrix at X + rowtab[r] * rowmul (rowtab NULL: r * rowmul).
// kind: 0 = Ozaki digits (s slices, exponent per row), 1 = bf16 copy (e = 0), 2 = tf32 copy,
// 3 = FP64 copy.
__global__ void pm_f64_kernel(const double* __restrict__ X0, const long long* __restrict__ rowtab, long long rowmul,
                              int v, int sign, double h, int kind, int s, int beta, void* __restrict__ D,
                              long long pitch, long long rows, int* __restrict__ e_out, int* __restrict__ status)
{
    __shared__ double S1[TT][TT + 1], S2[TT][TT + 1];
    __shared__ unsigned long long red[8];
    const long long r = blockIdx.x;
    const double* X = X0 + (rowtab ? rowtab[r] : r) * rowmul;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int nt = (v + TT - 1) / TT;
    const long long vv = v;
    const long long slice_stride = rows * pitch;
    const int total = beta * s;
    const long long H = kind == 0 ? digit_bias(s, beta) : 0;
    int e = 0;
    for (int pass = (kind == 0 ? 0 : 1); pass < 2; ++pass) {
        unsigned long long mx = 0;
        for (int tc = 0; tc < nt; ++tc) {
            for (int td = tc; td < nt; ++td) {
                __syncthreads();
                for (int y = ty; y < TT; y += TY) {
                    const int c = tc * TT + y, d = td * TT + tx;
                    S1[y][tx] = (c < v && d < v) ? X[c * vv + d] : 0.0;
                    const int d2 = td * TT + y, c2 = tc * TT + tx;
                    S2[y][tx] = (d2 < v && c2 < v) ? X[d2 * vv + c2] : 0.0;
                }
                __syncthreads();
                for (int y = ty; y < TT; y += TY) {
                    const int c = tc * TT + y, d = td * TT + tx;
                    if (c >= v || d >= v || d < c || (sign < 0 && d == c)) continue;
                    const double z = pm_value(S1[y][tx], S2[tx][y], c == d, sign, h);
                    const long long k = sign > 0 ? kp_of(c, d, vv) : km_of(c, d, vv);
                    if (pass == 0) {
                        const unsigned long long b = (unsigned long long)__double_as_longlong(z) & kAbs;
                        mx = b > mx ? b : mx;
                    } else if (kind == 0) {
                        put_digits(fixed_of(z, e, total), H, s, beta, (__nv_bfloat16*)D + r * pitch + k, slice_stride);
                    } else if (kind == 1) {
                        ((__nv_bfloat16*)D)[r * pitch + k] = __double2bfloat16(z);
                    } else if (kind == 3) {
                        ((double*)D)[r * pitch + k] = z;
                    } else {
                        ((float*)D)[r * pitch + k] = tf32_of(z);
                    }
                }
            }
        }
        if (pass == 0) {
            const unsigned long long bm = block_max_u64(mx, red);
            e = exp_of_maxbits(bm);
            // NaN or Inf in the row (or an overflowing sum t_cd + t_dc): flag the call
            if (threadIdx.x == 0 && status && bm >= 0x7ff0000000000000ull) atomicOr(status, kStatusNonfinite);
        }
    }
    if (threadIdx.x == 0 && e_out) e_out[r] = e;
}

// Int64 fixed-point integral block (output of the integral GEMM kept as int64): packed
// row r is the unpacked row ru = rtab[r], X[c][d] = V[ru*ldx + c*v + d] * 2^(eo[c] + ei[d]
// + base) with eo = eA + amap(ru), ei = eB + bmap(ru).  Writes V+ and V- digits with one
// shared row exponent E (max |V| < 2^E bounds both halves).  Integer arithmetic only.
__global__ void pm_fixed_kernel(const PmFixedSrc src, int s, int beta, __nv_bfloat16* __restrict__ Dp,
                                long long pitchp, int* __restrict__ ep, __nv_bfloat16* __restrict__ Dm,
                                long long pitchm, int* __restrict__ em)
{
    extern __shared__ int esm[];  // eo[v], ei[v]
    __shared__ long long S1[TT][TT + 1], S2[TT][TT + 1];
    __shared__ int redi[8];
    const long long r = blockIdx.x;
    const long long ru = src.rtab[r];
    const int v = src.v;
    const long long vv = v;
    const long long ab = map2(src.amap, ru), bb = map2(src.bmap, ru);
    for (int q = threadIdx.x; q < v; q += 256) {
        esm[q] = src.eA[ab + q];
        esm[v + q] = src.eB[bb + q];
    }
    __syncthreads();
    const int* eo = esm;
    const int* ei = esm + v;
    const long long* X = src.X + ru * src.ldx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pass 1: E = max over the row of bitlength(|X|) + exponent, so max |V| < 2^E
    int mx = INT_MIN;
    for (int c = warp; c < v; c += 8) {
        const long long* Xc = X + c * vv;
        const int ec = eo[c];
#pragma unroll 4
        for (int d = lane; d < v; d += 32) {
            const long long x = __ldcs(Xc + d);
            const unsigned long long ax = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
            const int b = x ? 64 - __clzll((long long)ax) + ec + ei[d] : INT_MIN;
            mx = b > mx ? b : mx;
        }
    }
    for (int w = 16; w > 0; w >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, w));
    if (lane == 0) redi[warp] = mx;
    __syncthreads();
    int m = redi[0];
    for (int w = 1; w < 8; ++w) m = max(m, redi[w]);
    const bool zero = m == INT_MIN;
    const int E = zero ? 0 : m + src.base;
    if (threadIdx.x == 0) {
        ep[r] = E;
        if (em) em[r] = E;
    }
    // pass 2: Y = round(V * 2^(total - E)) (one guard bit), V+- = (Y1 +- Y2) / 4 at the
    // digit scale 2^(total - 1 - E); the diagonal of V+ is Y1 / 2.  Tile pairs (tc <= td)
    // in order; the next pair's loads are issued before the current pair is split.
    const int total = beta * s;
    const long long H = digit_bias(s, beta);
    const int tx = lane, ty = warp;
    const int nt = (v + TT - 1) / TT;
    const long long sp = src.rows * pitchp, sm = src.rows * pitchm;
    const int sh0 = src.base + total - E;
    long long q1[TT / TY], q2[TT / TY];
    auto fetch = [&](int tc, int td) {
#pragma unroll
        for (int u = 0; u < TT / TY; ++u) {
            const int y = ty + u * TY;
            const int c = tc * TT + y, d = td * TT + tx;
            q1[u] = (!zero && c < v && d < v) ? __ldcs(X + c * vv + d) : 0;
            const int d2 = td * TT + y, c2 = tc * TT + tx;
            q2[u] = (!zero && d2 < v && c2 < v) ? __ldcs(X + d2 * vv + c2) : 0;
        }
    };
    int tc = 0, td = 0;
    fetch(0, 0);
    while (tc < nt) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TT / TY; ++u) {
            S1[ty + u * TY][tx] = q1[u];
            S2[ty + u * TY][tx] = q2[u];
        }
        __syncthreads();
        int nc = tc, nd = td + 1;
        if (nd == nt) { ++nc; nd = nc; }
        if (nc < nt) fetch(nc, nd);
        for (int y = ty; y < TT; y += TY) {
            const int c = tc * TT + y, d = td * TT + tx;
            if (c >= v || d >= v || d < c) continue;
            const long long Y1 = shr_round(S1[y][tx], eo[c] + ei[d] + sh0);
            if (c == d) {
                put_digits((Y1 + 1) >> 1, H, s, beta, Dp + r * pitchp + kp_of(c, d, vv), sp);
            } else {
                const long long Y2 = shr_round(S2[tx][y], eo[d] + ei[c] + sh0);
                put_digits((Y1 + Y2 + 2) >> 2, H, s, beta, Dp + r * pitchp + kp_of(c, d, vv), sp);
                if (Dm) put_digits((Y1 - Y2 + 2) >> 2, H, s, beta, Dm + r * pitchm + km_of(c, d, vv), sm);
            }
        }
        tc = nc;
        td = nd;
    }
}

// rtab[rowbase(al) + b' - al] = al * Nb + b' for b' in [al, Nb)
__global__ void fill_rtab_kernel(int Ab, int Nb, long long* __restrict__ rtab)
{
    const int al = blockIdx.x;
    const long long base = (long long)al * Nb - (long long)al * (al - 1) / 2;
    for (int b = al + threadIdx.x; b < Nb; b += blockDim.x) rtab[base + (b - al)] = (long long)al * Nb + b;
}

__device__ __forceinline__ void pair_ij(int o, int p, int& i, int& j)
{
    int ii = 0, rem = p;
    while (rem >= o - ii) { rem -= o - ii; ++ii; }
    i = ii;
    j = ii + rem;
}

// R from R+ (rows: pairs q0 <= p < q1, i <= j) and R- (rows: their pairs i < j, from strict index
// s0) of one block; columns are packed rows r (al, b' >= al).  Grid: x = pair p - q0, y = al.
__global__ void pm_combine_kernel(int o, int v, int a0, int Nb, long long nr, long long q0, long long s0,
                                  const double* __restrict__ Rp, const double* __restrict__ Rm,
                                  double* __restrict__ R, int accumulate)
{
    const long long pl = blockIdx.x;
    const int p = (int)(q0 + pl), al = blockIdx.y;
    int i, j;
    pair_ij(o, p, i, j);
    const long long q = p - (i + 1) - s0;  // row among this block's pairs i < j
    const long long vv = (long long)v * v;
    const long long base = (long long)al * Nb - (long long)al * (al - 1) / 2;
    const int a = a0 + al;
    double* Rij = R + ((long long)i * o + j) * vv;
    double* Rji = R + ((long long)j * o + i) * vv;
    const double* rp = Rp + pl * nr + base - al;
    const double* rm = (i < j && Rm) ? Rm + q * nr + base - al : nullptr;
    for (int bq = al + threadIdx.x; bq < Nb; bq += blockDim.x) {
        const int b = a0 + bq;
        const double plus = rp[bq];
        const double minus = (rm && b != a) ? rm[bq] : 0.0;
        const double e1 = plus + minus, e2 = plus - minus;
        const long long ab = (long long)a * v + b, ba = (long long)b * v + a;
        if (accumulate) {
            Rij[ab] += e1;
            if (!(i == j && a == b)) Rji[ba] += e1;
            if (i != j && a != b) { Rji[ab] += e2; Rij[ba] += e2; }
        } else {
            Rij[ab] = e1;
            if (!(i == j && a == b)) Rji[ba] = e1;
            if (i != j && a != b) { Rji[ab] = e2; Rij[ba] = e2; }
        }
    }
}

// tab[q] = (i*o + j) * v*v for the pairs i < j (strict) or i <= j, i-major.
__global__ void fill_pairs_kernel(int o, int v, int strict, long long* __restrict__ tab)
{
    const int i = blockIdx.x;
    const long long vv = (long long)v * v;
    const long long base = strict ? (long long)i * (o - 1) - (long long)i * (i - 1) / 2
                                  : (long long)i * o - (long long)i * (i - 1) / 2;
    for (int j = i + strict + threadIdx.x; j < o; j += blockDim.x)
        tab[base + (j - i - strict)] = ((long long)i * o + j) * vv;
}

}  // namespace

cudaError_t pm_split_f64(const double* X, const long long* rowtab, long long rowmul, long long rows, int v, int sign,
                         double h, int kind, int s, int beta, void* D, long long pitch, int* e, int* status,
                         cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    if (v < 1 || (sign < 0 && v < 2)) return cudaErrorInvalidValue;
    if (kind == 0 && (s < 1 || s > 8 || beta < 2 || beta > 9 || beta * s > 62)) return cudaErrorInvalidValue;
    if (rows > 0x7fffffffll) return cudaErrorInvalidValue;
    pm_f64_kernel<<<(unsigned)rows, 256, 0, st>>>(X, rowtab, rowmul, v, sign, h, kind, s, beta, D, pitch, rows, e,
                                                   status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t pm_split_fixed(const PmFixedSrc& src, int s, int beta, void* Dp, long long pitchp, int* ep, void* Dm,
                           long long pitchm, int* em, cudaStream_t st)
{
    if (src.rows <= 0) return cudaSuccess;
    if (s < 1 || s > 8 || beta < 2 || beta > 9 || beta * s > 62 || src.v < 1) return cudaErrorInvalidValue;
    // 8 v bytes of row / column exponents next to 17 KB of static tiles; above the 48 KB
    // default the kernel opts in to the larger dynamic shared memory (v up to about 26000)
    const size_t smem = sizeof(int) * 2 * (size_t)src.v;
    if (smem > 200 * 1024 || src.rows > 0x7fffffffll) return cudaErrorInvalidValue;
    if (smem > 30 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pm_fixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pm_fixed_kernel<<<(unsigned)src.rows, 256, smem, st>>>(src, s, beta, (__nv_bfloat16*)Dp, pitchp, ep,
                                                           (__nv_bfloat16*)Dm, pitchm, em);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fill_rtab(int Ab, int Nb, long long* rtab, cudaStream_t st)
{
    if (Ab <= 0) return cudaSuccess;
    fill_rtab_kernel<<<Ab, 256, 0, st>>>(Ab, Nb, rtab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t pm_combine(int o, int v, int a0, int Ab, int Nb, long long nr, long long q0, long long q1, long long s0,
                       const double* Rp, const double* Rm, double* R, int accumulate, cudaStream_t st)
{
    const long long np = q1 - q0;
    if (Ab <= 0 || np <= 0) return cudaSuccess;
    if (Ab > 65535 || np > 0x7fffffffll || q0 < 0 || q1 > (long long)o * (o + 1) / 2) return cudaErrorInvalidValue;
    pm_combine_kernel<<<dim3((unsigned)np, (unsigned)Ab), 256, 0, st>>>(o, v, a0, Nb, nr, q0, s0, Rp, Rm, R,
                                                                        accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fill_pairs(int o, int v, int strict, long long* tab, cudaStream_t st)
{
    if (o - strict <= 0) return cudaSuccess;
    fill_pairs_kernel<<<o, 64, 0, st>>>(o, v, strict, tab);
    count_launch();
    return cudaGetLastError();
}

}  // namespace cc
