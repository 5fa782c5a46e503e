// cc_internal.cuh -- internal interfaces between the C ABI (api.cu), the planner
// and the kernels.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cc_ladder.h"

namespace cc {

// Bits of the device status word at the start of every workspace.
constexpr int kStatusWaitExpired = 1;   // a bounded device-side wait ran out
constexpr int kStatusDrainExpired = 2;  // the abort path's drain ran out as well
constexpr int kStatusNonfinite = 16;    // an Ozaki split met NaN or Inf in its FP64 input

// Two-level index map: off(i) = (i / div) * s0 + (i % div) * s1 + base, where the
// outer term is tab[i / div] instead when a device table is given.  div == 0 means
// a plain stride: off(i) = i * s1 + base (or tab[i] + base).
struct Map2 {
    long long div, s0, s1, base;
    const long long* tab;
};

__host__ __device__ inline long long map2(const Map2& m, long long i)
{
    if (m.tab) {
        if (m.div == 0) return m.tab[i] + m.base;
        return m.tab[i / m.div] + (i % m.div) * m.s1 + m.base;
    }
    if (m.div == 0) return i * m.s1 + m.base;
    return (i / m.div) * m.s0 + (i % m.div) * m.s1 + m.base;
}

inline Map2 plain_map(long long stride, long long base = 0) { return Map2{0, 0, stride, base, nullptr}; }
inline Map2 split_map(long long div, long long s0, long long s1, long long base = 0)
{
    return Map2{div, s0, s1, base, nullptr};
}
inline Map2 table_map(const long long* tab, long long div = 0, long long s1 = 0, long long base = 0)
{
    return Map2{div, 0, s1, base, tab};
}

// Output of every GEMM: C[rmap(m) + cmap(n)] (= or +=) alpha * sum_k A(m,k) B(n,k).
struct OutDesc {
    double* C;
    Map2 rmap, cmap;
    int accumulate;  // 1: C += ..., 0: C = ...
};

// ---------------------------------------------------------------- FP64 DMMA GEMM
// A(m,k) = A[am(m) + ak(k)], B(n,k) = B[bm(n) + bk(k)].  An operand whose k map is
// the unit stride is loaded k-contiguously, any other one row-contiguously.
struct GemmF64 {
    int M, N, K;
    const double* A; Map2 am, ak;
    const double* B; Map2 bm, bk;
    OutDesc out;
    long long tri;  // triangular tile skip (0 = off): tiles with n / tri < m / tri everywhere are skipped
};
cudaError_t gemm_f64(const GemmF64& g, cudaStream_t s);

// ------------------------------------------------------- tensor-core slice GEMM
// Operands are K-major "slice stacks": D[slice][row][pitch] of bf16 (or fp32 for
// TF32), with one int32 exponent per row (row scale 2^e).  The slice-product
// levels L (products A_i B_j^T with i + j = L) are computed in groups of one or
// two levels, each group over K-chunks of gkc elements (one pass per chunk), in
// FP32 on the tensor cores; the epilogue turns level L of a pass into
// 2^(eA[m] + eB[n] + scale_base - beta*L) * acc, either added into the FP64 output
// after every pass (EPI_FP64_RMW) or summed exactly as int64 fixed point with
// 2^-fixF resolution of a level-0 unit and converted once (EPI_FIXED64).
enum TcKind { TC_BF16 = 0, TC_TF32 = 1 };
enum TcEpi { EPI_FP64_RMW = 0, EPI_FIXED64 = 1, EPI_FIXED64_RED = 2, EPI_FIXED64_ADD = 3 };
constexpr int kMaxGroups = 8;

struct GemmTc {
    int kind;  // TcKind
    int M, N, K;
    const void* A; long long pitchA, rowsA, rowA0;  // GEMM row m is stack row rowA0 + m
    const void* B; long long pitchB, rowsB, rowB0;
    int slices;                 // slices per operand (1 for the mixed modes)
    const int* eA; const int* eB;  // per stack-row exponents (nullable = 0)
    int scale_base, beta;
    int ngroups;
    int glo[kMaxGroups];        // lowest level of each group
    int gn[kMaxGroups];         // levels in the group (1 or 2)
    int gkc[kMaxGroups];        // K elements per pass (0 = whole K; else a multiple of 64 bf16 / 32 tf32)
    int epi, fixF;              // TcEpi; fixed-point fraction bits for EPI_FIXED64
    int ksplit;                 // K split across this many CTAs per tile (EPI_FIXED64_ADD only; 1 = none)
    // Triangular tile skip (0 = off): with a(m) = m / tri_rdiv and b(n) = n / tri_cdiv, a CTA
    // whose tile has b(n) < a(m) for every element writes nothing (integral blocks with b >= a).
    long long tri_rdiv, tri_cdiv;
    OutDesc out;
    int* status;                // device status word (bit 0: wait bound expired)
    unsigned long long wait_ns; // bound on every device-side wait
};
cudaError_t gemm_tc(const GemmTc& g, cudaStream_t s);
int tc_gemm_available();
int device_sm_count();
// C[rmap(m) + cmap(n)] (int64 fixed point) -> FP64: X * 2^(eA[rowA0+m] + eB[rowB0+n] + base)
cudaError_t fixed_to_f64(int M, int N, const OutDesc& out, const int* eA, long long rowA0, const int* eB,
                         long long rowB0, int base, cudaStream_t s);
// C[rmap(m) + cmap(n)] = 0 (as int64) for m < M, n < N
cudaError_t zero_out(int M, int N, const OutDesc& out, cudaStream_t s);

// ------------------------------------------------------------------- splitting
// Row source: X(r, k) = X[rm(r) + km(k)], k contiguous (km.s1 == 1 for the inner level).
struct RowSrc {
    const double* X; Map2 rm; Map2 km; long long rows, K;
};
// Ozaki split of each row into `s` balanced base-2^beta digits stored as bf16 in
// D[s][rows][pitch] with exponent e[r] (max |row| < 2^e).  s == 0: plain bf16 copy
// (e = 0).  D must hold s*rows*pitch bf16.
// status (nullable): kStatusNonfinite is or-ed in when a split row holds NaN or Inf (s > 0).
cudaError_t split_rows_bf16(const RowSrc& src, int s, int beta, void* D, long long pitch, int* e, int* status,
                            cudaStream_t st);
// Column source, rows contiguous: X(r, k) = X[bmap(r / brows) + r % brows + k * ldk]
// for r in [0, rows); brows == 0 means one batch (X[r + k * ldk]).
struct ColSrc {
    const double* X; long long ldk; long long rows, K;
    long long brows; Map2 bmap;
};
// premax: scratch_max already holds every row's max |x| bit pattern (over a K range that may be
// longer than this call's, e.g. all Cholesky vectors when L arrives in chunks): rows are split
// with those exponents and nothing is recomputed.
cudaError_t split_cols_bf16(const ColSrc& src, int s, int beta, void* D, long long pitch, int* e,
                            unsigned long long* scratch_max, int* status, cudaStream_t st, bool premax = false);
// mx[r] = max(mx[r], max_k |X(r, k)| as a bit pattern) (atomic; mx is not cleared).
cudaError_t cols_max(const ColSrc& src, unsigned long long* mx, int* status, cudaStream_t st);
// Ozaki split of an int64 fixed-point intermediate (a slice-GEMM output kept as
// EPI_FIXED64_RED).  Row r, element k = o*inner + i is X[r*ldx + k] * 2^e with
// e = eA[amap(r) + o] + eB[bmap(r) + i] + base.  Integer arithmetic only.
struct FixedSrc {
    const long long* X; long long rows, ldx;
    int outer, inner;
    const int* eA; Map2 amap;
    const int* eB; Map2 bmap;
    int base;
};
cudaError_t split_fixed_rows_bf16(const FixedSrc& src, int s, int beta, void* D, long long pitch, int* e,
                                  cudaStream_t st);
// Symmetric / antisymmetric packing (pm.cu) for pair-symmetric amplitudes.
// Packed rows of an FP64 source: row r is the v x v matrix at X + (rowtab ? rowtab[r] : r) * rowmul;
// sign > 0 writes the c <= d part (X[c][d] + X[d][c]) * h (diagonal X[c][c]) at c*v - c(c-1)/2 + d - c,
// sign < 0 the c < d part (X[c][d] - X[d][c]) * h at c*(v-1) - c(c-1)/2 + d - c - 1.  kind 0: Ozaki
// digits with a row exponent, 1: bf16 copy (e = 0), 2: tf32 copy (e may be NULL), 3: FP64 copy.
// status (nullable, kind 0): kStatusNonfinite is or-ed in when a packed row holds NaN or Inf.
cudaError_t pm_split_f64(const double* X, const long long* rowtab, long long rowmul, long long rows, int v, int sign,
                         double h, int kind, int s, int beta, void* D, long long pitch, int* e, int* status,
                         cudaStream_t st);
// Int64 fixed-point integral block: packed row r is unpacked row ru = rtab[r] of X (ldx per row),
// X[c][d] * 2^(eA[amap(ru) + c] + eB[bmap(ru) + d] + base).  Writes V+ (h = 1/2) and, if Dm is not
// NULL, V- digits, both with the row exponent of max |V|.
struct PmFixedSrc {
    const long long* X; const long long* rtab; long long rows, ldx;
    int v;
    const int* eA; Map2 amap;
    const int* eB; Map2 bmap;
    int base;
};
cudaError_t pm_split_fixed(const PmFixedSrc& src, int s, int beta, void* Dp, long long pitchp, int* ep, void* Dm,
                           long long pitchm, int* em, cudaStream_t st);
// rtab[rowbase(al) + b' - al] = al * Nb + b' for al < Ab, al <= b' < Nb (rowbase(al) = al Nb - al(al-1)/2)
cudaError_t fill_rtab(int Ab, int Nb, long long* rtab, cudaStream_t st);
// R[i,j,a,b], R[j,i,b,a] (=|+=) R+ + R-;  R[j,i,a,b], R[i,j,b,a] (=|+=) R+ - R-  for the block
// a = a0 + al (al < Ab), b = a0 + b' (al <= b' < Nb) and the pairs q0 <= p < q1 (i <= j):
// Rp[p - q0][r]; Rm[s(p) - s0][r] for their pairs i < j (s = index among the pairs i < j).
cudaError_t pm_combine(int o, int v, int a0, int Ab, int Nb, long long nr, long long q0, long long q1, long long s0,
                       const double* Rp, const double* Rm, double* R, int accumulate, cudaStream_t st);
// tab = (i*o + j) * v*v for the pairs i < j (strict = 1) or i <= j (strict = 0), i-major
cudaError_t fill_pairs(int o, int v, int strict, long long* tab, cudaStream_t st);
// Plain fp64 -> tf32 (stored as fp32) copies, K-major.
cudaError_t convert_rows_tf32(const RowSrc& src, float* D, long long pitch, cudaStream_t st);
cudaError_t convert_cols_tf32(const ColSrc& src, float* D, long long pitch, cudaStream_t st);

// -------------------------------------------------------------------- misc
// R[i,j,a,b] (=|+=) Rc[p, a, b] for p = pair(i<=j), and R[j,i,b,a] likewise for i<j,
// for a in [a_lo, a_hi).
cudaError_t scatter_pairs(int o, int v, int a_lo, int a_hi, const double* Rc, double* R, int accumulate,
                          cudaStream_t s);
// Y[ij][c][d] = X[ij][d][c]
cudaError_t swap_last2(long long batch, int v, const double* X, double* Y, cudaStream_t s);
// Y[ij][a][b] = alpha * X[ij][a][b] + X[ji][b][a]   (alpha = 0 or 1)
cudaError_t add_pair_swap(int o, int v, const double* X, double* Y, int alpha, cudaStream_t s);
// tab[p] = (i*o + j) * v*v for the pairs i <= j in i-major order
cudaError_t fill_pair_table(int o, int v, long long* tab, cudaStream_t s);
// Y[P][a][c] = X[P][c][a]
cudaError_t transpose_last2(long long batch, int v, const double* X, double* Y, cudaStream_t s);
// energy
// part: o*o*ceil(v/32)^2 doubles of scratch; e_pair: o*o results
// Terms with lo <= min(a, b) < hi only (hi < 0: all of them).
cudaError_t energy_pairs(int o, int v, const double* R, const double* t2, double* part, double* e_pair, cudaStream_t s,
                         int lo = 0, int hi = -1);
inline long long energy_scratch_doubles(int o, int v) { const long long t = (v + 31) / 32; return (long long)o * o * t * t; }
cudaError_t energy_total(long long npairs, const double* e_pair, double* E, cudaStream_t s);

// ------------------------------------------------------------------- tracing
void count_launch(int n = 1);
// Records CUDA events around a phase on `s` when profiling is enabled.
class ProfScope {
  public:
    ProfScope(const char* name, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    double flops_, bytes_;
    void* e0_;
};

}  // namespace cc
