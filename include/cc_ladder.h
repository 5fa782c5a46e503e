/*
 * cc_ladder.h -- C ABI of the GB300 (sm_103a) particle-particle ladder library.
 *
 * The library evaluates the rate-determining term of the closed-shell CCD/CCSD
 * vector function with Cholesky-decomposed integrals (arXiv:2310.04559):
 *
 *   Eq. 4   0 = ... + sum_cd <ab|cd> t_ij^cd + ...
 *   Eq. 5   <ab|cd> ~= sum_P L^P_ac L^P_bd
 *   Eq. 6   R[i,j,a,b] = sum_{c,d} ( sum_P L[P,a,c] L[P,b,d] ) t2[i,j,c,d]
 *
 * without ever storing the v^4 integral tensor: the integrals (ac|bd) are
 * assembled on the device for one block of `a` values at a time (the for-loop
 * over `a` of Section 3.2, widened to blocks), then contracted with t2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All tensors are row-major, contiguous FP64 (IEEE binary64) DEVICE arrays
 *    owned by the caller; the library keeps no pointer after a call returns.
 *      L  [n_chol][v][v]   Cholesky vectors L[P,a,c]        (Eq. 5)
 *      t2 [o][o][v][v]     amplitudes t2[i,j,c,d]
 *      R  [o][o][v][v]     result R[i,j,a,b]                (Eq. 6)
 *    The paper stores amplitudes as t[i,a,j,b] (Section 3.1); a caller with
 *    that layout permutes axes 1 and 2 first.
 *  - Every pointer must be 16-byte aligned (CC_ERR_ALIGN otherwise).
 *  - The library never allocates device memory.  Scratch comes from the
 *    caller's `workspace` (256-byte aligned); query its size first.  The
 *    planner sizes the block of `a` values so that the workspace fits the
 *    caller's budget.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Unless CC_FLAG_NO_STATUS_SYNC is given, the call synchronises
 *    the stream once at the end to read the device status word, so the
 *    returned status covers device-side failures (CC_ERR_DEVICE_TIMEOUT).
 *  - Return value: CC_OK (0) or a negative cc_status.  Argument errors are
 *    detected before anything is enqueued.  No C++ exception crosses the ABI.
 *  - Thread safety: calls on different streams with different workspaces may
 *    run concurrently; the plan cache is guarded by a mutex.
 */
#ifndef CC_LADDER_H
#define CC_LADDER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum cc_status {
    CC_OK = 0,
    CC_ERR_SHAPE = -1,          /* o, v or n_chol < 1, or a product overflows      */
    CC_ERR_NULL = -2,           /* a required pointer is NULL                       */
    CC_ERR_ALIGN = -3,          /* a pointer is not 16-byte (workspace: 256) aligned */
    CC_ERR_WORKSPACE = -4,      /* ws_bytes smaller than the plan needs             */
    CC_ERR_BUDGET = -5,         /* budget below the smallest plan (one `a` per block) */
    CC_ERR_UNSUPPORTED = -6,    /* mode / order / flag combination not available    */
    CC_ERR_CUDA = -7,           /* a CUDA runtime call failed                       */
    CC_ERR_DEVICE_TIMEOUT = -8, /* a bounded device-side wait ran out; results invalid */
    CC_ERR_ARG = -9,            /* other invalid argument (unknown mode, bad a_block) */
    CC_ERR_NOALLOC_LIMIT = -10, /* problem larger than cc_ladder_energy_noalloc's fixed scratch */
    CC_ERR_NONFINITE = -11      /* CC_OZAKI_BF16: an input (L, t2, the adjoint's dR, a GEMM operand)
                                   holds NaN or Inf, which the integer slices cannot carry; the
                                   outputs are invalid.  The other modes propagate NaN / Inf into
                                   the outputs as IEEE arithmetic does and never return this. */
};

/* Arithmetic used for the two contractions (integral build and ladder GEMM). */
enum cc_precision {
    CC_FP64 = 0,       /* FP64 tensor-core MMA (DMMA), FP64 accumulation              */
    CC_OZAKI_BF16 = 1, /* FP64 emulated by split BF16 integer slices (Ozaki scheme) on
                          tcgen05 tensor cores: each operand row is scaled by a power of two and
                          rounded once to a 42-bit integer cut into 6 balanced 7-bit digits (2..8
                          slices selectable); the slice products of each level are summed in FP32
                          on the tensor cores and drained to exact int64 at most every
                          4096 / (products in the level) contraction elements, so every FP32 sum
                          stays an exact integer below 2^24 for ANY input (sign-aligned data,
                          constant matrices, Gram diagonals included); levels are recombined in
                          int64 and converted to FP64 once.  Error: the 42-bit rounding of the
                          inputs and the dropped levels, about 1e-11 relative.  NaN / Inf inputs
                          give CC_ERR_NONFINITE. */
    CC_OZAKI_INT8 = 2, /* INT8-slice emulation: tcgen05 has no kind::i8 on sm_103a;
                          always returns CC_ERR_UNSUPPORTED                           */
    CC_TF32 = 3,       /* TF32 inputs, FP32 accumulation per K-chunk, FP64 across chunks */
    CC_BF16 = 4        /* BF16 inputs, FP32 accumulation per K-chunk, FP64 across chunks */
};

/* Contraction order (Section 3.2). */
enum cc_order {
    CC_ORDER_AUTO = 0,           /* planner picks the cheaper one for the shape           */
    CC_ORDER_INTEGRAL_FIRST = 1, /* (ac|bd) block first: 2 n v^4 + 2 o^2 v^4 flops         */
    CC_ORDER_CHOLESKY_FIRST = 2  /* L.t intermediate first: 4 n o^2 v^3 flops              */
};

/* Bit flags for cc_ladder_args.flags. */
enum cc_flags {
    CC_FLAG_ACCUMULATE = 1,     /* R += term (the paper's `t_new += ...`, Section 3) instead of R = term */
    CC_FLAG_SYMMETRIC_T = 2,    /* caller promises t2[i,j,c,d] == t2[j,i,d,c], so R[j,i,b,a] = R[i,j,a,b].
                                   Integral-first (every mode): the integrals are built for b >= a only
                                   ((ac|bd) = (bd|ac) holds for any L) and the ladder GEMM runs on the
                                   parts of t2 and (ac|bd) symmetric / antisymmetric in c <-> d, packed
                                   over c <= d (about half the flops).  The Cholesky-first order
                                   computes the pairs i <= j and mirrors them.                         */
    CC_FLAG_EXCHANGE = 4,       /* evaluate the exchange partner of Eq. 7 instead:
                                   R[i,j,a,b] = sum_cd (sum_P L_Pad L_Pbc) t2[i,j,c,d]                */
    CC_FLAG_NO_STATUS_SYNC = 8, /* do not synchronise the stream at the end; device-side failures are
                                   then reported by cc_ladder_device_status()                         */
    CC_FLAG_HOST_T2R = 16,      /* t2 and R are page-locked HOST memory (cudaHostAlloc / cudaHostRegister,
                                   addressable from the device); L, energy and the workspace stay on the
                                   device.  The kernels read t2 and write R over the host link, so
                                   o^2 v^2 may exceed device memory: the device holds one block of
                                   pairs (i <= j) at a time.  Needs CC_FLAG_SYMMETRIC_T and the
                                   integral-first order, not CC_FLAG_EXCHANGE (else CC_ERR_UNSUPPORTED);
                                   CC_ERR_ARG if t2 or R is not page-locked host memory.              */
    CC_FLAG_HOST_L = 32         /* L is page-locked HOST memory: the library copies it to the device in
                                   chunks of chol_chunk Cholesky vectors (the batches over the Cholesky
                                   index of Section 5), double-buffered on a stream of its own so that
                                   the copy of chunk q + 1 overlaps the split and integral GEMM of
                                   chunk q; the integrals of a block are summed over the chunks.  L is
                                   read once for the emulated mode's row scales and once per block of
                                   `a`, so n_chol v^2 may exceed device memory.  Needs
                                   CC_FLAG_SYMMETRIC_T and the integral-first order (else
                                   CC_ERR_UNSUPPORTED); combines with CC_FLAG_HOST_T2R; CC_ERR_ARG if
                                   L is not page-locked host memory.  Forward only.                    */
};

/* Full argument block for cc_ladder_fwd_ex / cc_ladder_workspace_size_ex. */
typedef struct cc_ladder_args {
    int o, v, n_chol;      /* occupied, virtual, Cholesky-vector counts (>= 1)                */
    const double* L;       /* device [n_chol][v][v]                                             */
    const double* t2;      /* device [o][o][v][v] (page-locked host memory with CC_FLAG_HOST_T2R) */
    double* R;             /* device [o][o][v][v] (host, as t2); overwritten unless
                              CC_FLAG_ACCUMULATE                                                */
    double* energy;        /* nullable device scalar: E = sum_ijab (2 R_ijab - R_ijba) t2_ijab.
                              With an a-range (a_lo, a_hi below) on the pair-symmetric
                              integral-first path: the terms with min(a, b) in the range, whose
                              R_ijab and R_ijba the call writes, so the energies of disjoint
                              ranges add up to E; other paths need the complete range
                              (CC_ERR_UNSUPPORTED otherwise).                                  */
    int mode;              /* cc_precision                                                      */
    int order;             /* cc_order                                                          */
    int a_block;           /* 0 = planner's choice; else the number of `a` values per block     */
    int flags;             /* cc_flags                                                          */
    int slices;            /* Ozaki modes: BF16 slices per operand (0 = default 6; 2..8)         */
    void* workspace;       /* device scratch, 256-byte aligned                                  */
    size_t ws_bytes;       /* its size                                                          */
    size_t budget_bytes;   /* workspace_size_ex only: upper bound for the plan (0 = 150 GB)     */
    void* stream;          /* cudaStream_t                                                      */
    int a_lo, a_hi;        /* range of virtual indices `a` to compute (both 0 = all of 0..v-1).
                              Entries written: R[i,j,a,b] for a in [a_lo, a_hi).  With
                              CC_FLAG_SYMMETRIC_T, integral-first: R[i,j,a,b] and R[i,j,b,a] for
                              all i, j, a in the range and b >= a; Cholesky-first: R[i,j,a,b]
                              (i <= j) and R[j,i,b,a] (i < j) for a in the range.  Either way
                              disjoint ranges write disjoint entries, so ranges spread over
                              devices (each R zeroed first) assemble R by a sum
                              (cc_ladder_partition balances the ranges' work).                   */
    int chol_chunk;        /* CC_FLAG_HOST_L: Cholesky vectors per streamed chunk of L (0 = planner's
                              choice: two chunks and their slices in about an eighth of the budget,
                              halved until the plan fits); ignored otherwise                       */
} cc_ladder_args;

/* What the planner decided for a call (for reporting and tests). */
typedef struct cc_ladder_plan {
    int order;             /* CC_ORDER_INTEGRAL_FIRST or CC_ORDER_CHOLESKY_FIRST */
    int a_block;           /* `a` values in the first block                      */
    int n_blocks;          /* number of blocks (pair-symmetric integral-first plans widen their
                              blocks as the b >= a range shrinks)                 */
    int slices;            /* Ozaki slices (1 for the non-emulated modes)        */
    int pairs;             /* GEMM rows used for (i,j): o*o, or o(o+1)/2 with symmetry */
    size_t ws_bytes;       /* workspace the plan needs                           */
    double flops_algorithmic; /* 2(o^2+n)v^4 (integral-first) or 4 n o^2 v^3     */
    double flops_issued;      /* tensor-core flops actually issued (slice products, padding) */
    int pair_blocks;          /* blocks of pairs (i <= j) the device holds one at a time (1 unless
                                 CC_FLAG_HOST_T2R splits them to fit the workspace) */
} cc_ladder_plan;

/* Workspace bytes for cc_ladder_fwd with (mode, default order/flags) under `budget_bytes`
 * (0 = 150 GB).  Writes *bytes.  CC_ERR_BUDGET if even one `a` per block does not fit. */
int cc_ladder_workspace_size(int o, int v, int n_chol, int mode, size_t budget_bytes, size_t* bytes);

/* Same for an explicit argument block (uses o, v, n_chol, mode, order, a_block, flags,
 * slices, budget_bytes; pointers may be NULL). */
int cc_ladder_workspace_size_ex(const cc_ladder_args* args, size_t* bytes);

/* The plan cc_ladder_fwd_ex would run for `args` with its ws_bytes (pointers may be NULL). */
int cc_ladder_plan_query(const cc_ladder_args* args, cc_ladder_plan* plan);

/* R = sum_cd (ac|bd) t2_ijcd (Eq. 6) with default order (auto) and no flags.
 * energy: nullable device scalar for E (see cc_ladder_args).  Returns cc_status. */
int cc_ladder_fwd(int o, int v, int n_chol, const double* L, const double* t2, double* R, int mode,
                  double* energy, void* workspace, size_t ws_bytes, void* stream);

/* Forward with every option (order, a-block, accumulate, pair symmetry, exchange, slices). */
int cc_ladder_fwd_ex(const cc_ladder_args* args);

/* Work-balanced partition of the `a` range of one problem over `parts` devices (or ranks), for
 * running one problem on several GPUs without any exchange of data between them: part g calls
 * cc_ladder_fwd_ex with a_lo = bounds[g], a_hi = bounds[g + 1] on its own zeroed R, the parts'
 * R add up to the full R, and (pair-symmetric integral-first path) their energies add up to the
 * full energy (see cc_ladder_args.energy).  The output is not part of the paper, which leaves
 * multi-GPU execution to future work; the partition follows its for-loop over `a` (Section 3.2).
 * Reads o, v, n_chol, mode, order and flags of `args` (pointers may be NULL).  bounds: host
 * array of parts + 1 ints, bounds[0] = 0 < bounds[1] < ... < bounds[parts] = v.  On the packed
 * pair-symmetric path the work of column a is proportional to v - a (it builds the integrals
 * (a, b >= a) and their ladder columns), so the parts get equal sums of v - a; elsewhere equal
 * counts.  CC_ERR_ARG unless 1 <= parts <= v.  Host-only: launches nothing. */
int cc_ladder_partition(const cc_ladder_args* args, int parts, int* bounds);

/* Autotuner: times both contraction orders (Section 3.2) on this shape with the caller's
 * buffers and workspace (one and two blocks of `a` per order, extrapolated to all blocks), and
 * records the faster one for (o, v, n_chol, mode, symmetric/exchange flags).  Later calls with
 * order = CC_ORDER_AUTO use the recorded order; without a record they use the flop cost model.
 * If the environment variable CC_LADDER_CACHE names a file, records are appended to it and read
 * back by later processes.  R (and only R) is overwritten with partial results.  Synchronous.
 * plan (nullable) receives the chosen plan; ms_if / ms_cf (nullable) the estimated milliseconds
 * of each order (-1 where the order does not fit the workspace). */
int cc_ladder_autotune(const cc_ladder_args* args, cc_ladder_plan* plan, double* ms_if, double* ms_cf);

/* Workspace bytes for cc_ladder_bwd. */
int cc_ladder_bwd_workspace_size(int o, int v, int n_chol, int mode, size_t budget_bytes, size_t* bytes);

/* Adjoint of the forward for loss = sum W_ijab R_ijab, W = dR (device [o][o][v][v]):
 *   dt2[i,j,c,d] = sum_ab W_ijab (ac|bd)                                 (nullable)
 *   dL[P,e,f]    = sum_{ij,b,d} W_ijeb L_Pbd t_ijfd + sum_{ij,a,c} W_ijae L_Pac t_ijcf   (nullable)
 * The (ac|bd) blocks are rebuilt (a-block recomputation), never stored whole.
 * flags: CC_FLAG_SYMMETRIC_T lets dL use one pass with W + W^swap.  Overwrites dL / dt2. */
int cc_ladder_bwd(int o, int v, int n_chol, const double* L, const double* t2, const double* dR,
                  double* dL, double* dt2, int mode, void* workspace, size_t ws_bytes, void* stream);

/* Adjoint with flags (CC_FLAG_SYMMETRIC_T, CC_FLAG_NO_STATUS_SYNC) and slices. */
int cc_ladder_bwd_ex(int o, int v, int n_chol, const double* L, const double* t2, const double* dR,
                     double* dL, double* dt2, int mode, int flags, int slices, void* workspace,
                     size_t ws_bytes, void* stream);

/* E = sum_ijab (2 R_ijab - R_ijba) t2_ijab into the device scalar `energy`, and, if e_pair is not
 * NULL, e_pair[i*o+j] = the (i,j) part (device [o][o]).  Deterministic FP64 tree.
 * Needs cc_ladder_energy_workspace_size() bytes of workspace. */
int cc_ladder_energy(int o, int v, const double* R, const double* t2, double* energy, double* e_pair,
                     void* workspace, size_t ws_bytes, void* stream);
int cc_ladder_energy_workspace_size(int o, int v, size_t* bytes);

/* Pair energy without any allocation and without a workspace (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory -- e.g. code whose device
 * memory belongs to another framework's pool, or code that must not call cudaMalloc/cudaFree
 * because those calls can block or synchronise the device).  Same result and kernels as
 * cc_ladder_energy; the partial sums live in a 16 MiB array inside the library that every GPU
 * loading the library holds until the process exits.
 *   Limit: ceil(v/32)^2 * o^2 doubles of partials, plus o^2 when e_pair is NULL, must not exceed
 *   2^21 (e.g. o = 60 with v <= 640); larger problems return CC_ERR_NOALLOC_LIMIT and launch nothing.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress, with
 *   that device current); make that first call before capturing the stream into a graph.
 *   All calls share the one array: calls whose kernels may overlap on the GPU (different streams,
 *   or different host threads on one device) race and must be serialised by the caller.
 *   Nothing is synchronised; errors of the kernels surface at the caller's next synchronisation. */
int cc_ladder_energy_noalloc(int o, int v, const double* R, const double* t2, double* energy, double* e_pair,
                             void* stream);

/* The two further Cholesky terms of the CCSD vector function that share the ladder's contraction
 * (Section 6.1, Eq. 8 and Eq. 9; the paper benchmarks both as the contraction "abcd,ecfd->efab"),
 * with Lov[P][k][c] the occupied-virtual block of the Cholesky vectors (device [n_chol][o][v]) and
 * Lvv the virtual-virtual block (the L of cc_ladder_fwd, device [n_chol][v][v]):
 *   CC_TERM_IJKL  Eq. 8  T[i,j,k,l] = sum_{P,c,d} Lov[P,k,c] Lov[P,l,d] t2[i,j,c,d]   T: [o][o][o][o]
 *   CC_TERM_IJBK  Eq. 9  T[i,j,b,k] = sum_{P,c,d} Lvv[P,b,d] Lov[P,k,c] t2[i,j,c,d]   T: [o][o][v][o]
 * Computed like the ladder, integral-first: the four-index integrals (kc|ld) or (kc|bd) are built on
 * the device for a block of k at a time and contracted with t2 over (c,d); no symmetry is assumed.
 * Same precision modes, conventions and error behaviour as cc_ladder_fwd (T is overwritten;
 * Lvv may be NULL for CC_TERM_IJKL).  flags: CC_FLAG_NO_STATUS_SYNC only. */
enum cc_term { CC_TERM_IJKL = 1, CC_TERM_IJBK = 2 };
int cc_ladder_term_workspace_size(int which, int o, int v, int n_chol, int mode, int slices, size_t budget_bytes,
                                  size_t* bytes);
int cc_ladder_term(int which, int o, int v, int n_chol, const double* Lov, const double* Lvv, const double* t2,
                   double* T, int mode, int flags, int slices, void* workspace, size_t ws_bytes, void* stream);
int cc_ladder_tijkl(int o, int v, int n_chol, const double* Lov, const double* t2, double* T, int mode,
                    void* workspace, size_t ws_bytes, void* stream);
int cc_ladder_tijbk(int o, int v, int n_chol, const double* Lov, const double* Lvv, const double* t2, double* T,
                    int mode, void* workspace, size_t ws_bytes, void* stream);

/* Device status word of a workspace after calls made with CC_FLAG_NO_STATUS_SYNC
 * (synchronises `stream`; returns CC_OK or CC_ERR_DEVICE_TIMEOUT and clears the word). */
int cc_ladder_device_status(void* workspace, void* stream);

/* Test knob: the bound, in nanoseconds, on every device-side wait (0 = library default of
 * 2 s).  Applies to calls made after it on this process. */
void cc_ladder_set_wait_limit_ns(unsigned long long ns);

/* Building block used by every contraction above, exposed for direct use and testing:
 *   C[m*ldc + n] (= or +=) sum_k A[m*lda + k] * B[n*ldb + k]     (row-major, K-contiguous FP64)
 * in the arithmetic of `mode` (CC_FP64: DMMA; CC_OZAKI_BF16: split BF16 slices on tcgen05 with
 * FP64 recombination; CC_TF32 / CC_BF16: one rounded copy, FP32 accumulation per K-chunk).
 * accumulate != 0 adds into C.  Workspace from cc_ladder_gemm_workspace_size.
 * CC_OZAKI_BF16 is exact in its FP32 level sums for any K and any input (see cc_precision). */
int cc_ladder_gemm_workspace_size(int mode, int M, int N, int K, int slices, size_t* bytes);
int cc_ladder_gemm(int mode, int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                   int ldc, int accumulate, int slices, void* workspace, size_t ws_bytes, void* stream);

/* Tracing.  cc_ladder_profile_enable(1) resets and starts per-phase timing: every phase of
 * every later call records CUDA events on its stream.  cc_ladder_profile_read synchronises
 * those events and fills up to max_entries totals (phase name, launches, milliseconds,
 * tensor-core or FP64 flops issued, algorithmic bytes); it returns the number of phases.  Profiling adds two
 * events per phase and is off by default.  cc_ladder_launch_count is the number of kernels
 * the library has launched in this process.  Every phase is also an NVTX range of the same name
 * (visible in timeline profilers; free when none is attached), and with the environment variable
 * CC_LADDER_VERBOSE set to a non-zero value every forward call prints its plan to stderr. */
typedef struct cc_ladder_profile_entry {
    char name[32];
    int launches;
    double ms;
    double flops;
    double bytes;   /* algorithmic DRAM bytes of the slice GEMMs: every operand slice read once and
                       the output written once (read too when accumulated); 0 for other phases */
} cc_ladder_profile_entry;
void cc_ladder_profile_enable(int on);
int cc_ladder_profile_read(cc_ladder_profile_entry* out, int max_entries);
long long cc_ladder_launch_count(void);

/* Peak-rate probes (no counterpart in the paper: measurement support, so that each precision
 * mode's throughput can be set against the rate of the unit it runs on, measured on the same GPU).
 * Launches one microbenchmark kernel twice (warm-up, then timed with CUDA events on `stream`,
 * synchronised) and writes the whole GPU's rate in TFLOP/s to *tflops (host pointer).
 *   CC_PROBE_DMMA     mma.sync.m8n8k4.f64 from registers (the FP64 mode's GEMM instruction)
 *   CC_PROBE_DFMA     scalar FP64 fma from registers
 *   CC_PROBE_TC_BF16  tcgen05.mma kind::f16, BF16 operands in shared memory, M=128 N=256 K=16,
 *                     one issuing thread per SM (the emulated-FP64 and BF16 modes)
 *   CC_PROBE_TC_TF32  tcgen05.mma kind::tf32, M=128 N=256 K=8 (the TF32 mode)
 *   CC_PROBE_IMMA     mma.sync.m16n8k32.s8 from registers (TOP/s): legacy INT8 MMA, the only INT8
 *                     tensor-core form sm_103a assembles (ptxas rejects tcgen05 kind::i8 there)
 * iters (1 .. 2^24): loop trips per thread (tensor-core probes: groups of four MMAs).  The
 * tensor-core probes' wait for their last MMAs is bounded (2 s, CC_ERR_DEVICE_TIMEOUT).
 * Allocates no device memory. */
enum cc_probe { CC_PROBE_DMMA = 1, CC_PROBE_DFMA = 2, CC_PROBE_TC_BF16 = 3, CC_PROBE_TC_TF32 = 4, CC_PROBE_IMMA = 5 };
int cc_ladder_peak_probe(int which, int iters, void* stream, double* tflops);

/* Static description of a status code. */
const char* cc_ladder_strerror(int status);

/* Library version string. */
const char* cc_ladder_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CC_LADDER_H */
