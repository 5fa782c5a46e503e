/*
 * ladder_oracle.c -- plain FP64 CPU oracle for the particle-particle ladder term.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The product
 * path (the CUDA library under paper_2310_04559_gb300/) never links, imports or
 * calls it, and the two share no code, headers or tables.
 *
 * Paper: Kriebel, Tecmer, Galynska, Leszczyk, Boguslawski, "Accelerating
 * Pythonic coupled cluster implementations: a comparison between CPUs and
 * GPUs" (arXiv:2310.04559).
 *
 *   Eq. 4   0 = ... + sum_cd <ab|cd> t_ij^cd + ...       (the ladder term)
 *   Eq. 5   <ab|cd> ~= sum_x L^x_ac L^x_bd              (Cholesky-decomposed ERI)
 *   Eq. 6   t~_ij^ab = ... + sum_xcd L^x_ac L^x_bd t_ij^cd + ...
 *
 * so the quantity computed here is
 *
 *   R[i,j,a,b] = sum_{c,d} ( sum_P L[P,a,c] L[P,b,d] ) t2[i,j,c,d].
 *
 * No prefactor: the paper prints the term without one (Eq. 4, Eq. 6).
 * Layouts (row-major, FP64): L[P][a][c] (n x v x v), t2[i][j][c][d] and
 * R[i][j][a][b] (o x o x v x v).
 *
 * Everything is plain nested loops in FP64, in the order the definition reads;
 * OpenMP only distributes independent output entries over threads.  Optional
 * Neumaier compensation of the long sums is available for checking the plain
 * sums.  Parity status of every function: pinned (see tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double s; /* running sum            */
    double c; /* Neumaier compensation */
} nsum_t;

static inline void nsum_add(nsum_t* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double nsum_get(const nsum_t* a) { return a->s + a->c; }

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Eq. 5 + Eq. 6, evaluated like the for-loop over `a` of Section 3.2: for one
 * (a, b) pair build the v x v slice of integrals (ac|bd) = sum_P L_Pac L_Pbd,
 * then contract it with every t_ij.
 *
 * a_list / na select which virtual indices `a` to compute (a_list == NULL:
 * all a = 0..v-1, na ignored).  Output layout: R[i][j][k][b] where k is the
 * position of a in a_list (for the full case this is R[i][j][a][b]).
 * compensated != 0 uses Neumaier summation for both sums.
 */
void oracle_ladder(int o, int v, int n, const double* L, const double* t2, double* R,
                   const int* a_list, int na, int compensated, int nthreads)
{
    set_threads(nthreads);
    const int nav = a_list ? na : v;
    const size_t vv = (size_t)v * v;
    const long long npairs = (long long)nav * v;
#pragma omp parallel
    {
        double* Vab = (double*)malloc(sizeof(double) * vv);
        double* Vc = (double*)malloc(sizeof(double) * vv);
#pragma omp for schedule(dynamic, 1)
        for (long long pair = 0; pair < npairs; ++pair) {
            const int k = (int)(pair / v);
            const int b = (int)(pair % v);
            const int a = a_list ? a_list[k] : k;
            /* (ac|bd) = sum_P L[P,a,c] L[P,b,d]   (Eq. 5).  Every entry is summed
             * over P = 0..n-1 in increasing order; looping P outermost only
             * changes which entry is visited first, not any entry's sum. */
            if (compensated) {
                for (size_t q = 0; q < vv; ++q) { Vab[q] = 0.0; Vc[q] = 0.0; }
                for (int P = 0; P < n; ++P) {
                    const double* La = L + (size_t)P * vv + (size_t)a * v;
                    const double* Lb = L + (size_t)P * vv + (size_t)b * v;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d) {
                            nsum_t s = {Vab[(size_t)c * v + d], Vc[(size_t)c * v + d]};
                            nsum_add(&s, La[c] * Lb[d]);
                            Vab[(size_t)c * v + d] = s.s;
                            Vc[(size_t)c * v + d] = s.c;
                        }
                }
                for (size_t q = 0; q < vv; ++q) Vab[q] += Vc[q];
            } else {
                for (size_t q = 0; q < vv; ++q) Vab[q] = 0.0;
                for (int P = 0; P < n; ++P) {
                    const double* La = L + (size_t)P * vv + (size_t)a * v;
                    const double* Lb = L + (size_t)P * vv + (size_t)b * v;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d) Vab[(size_t)c * v + d] += La[c] * Lb[d];
                }
            }
            /* R_ij,ab = sum_c sum_d (ac|bd) t_ij,cd   (Eq. 6) */
            for (int i = 0; i < o; ++i) {
                for (int j = 0; j < o; ++j) {
                    const double* tij = t2 + ((size_t)i * o + j) * vv;
                    double r;
                    if (compensated) {
                        nsum_t s = {0.0, 0.0};
                        for (int c = 0; c < v; ++c)
                            for (int d = 0; d < v; ++d)
                                nsum_add(&s, Vab[(size_t)c * v + d] * tij[(size_t)c * v + d]);
                        r = nsum_get(&s);
                    } else {
                        double s = 0.0;
                        for (int c = 0; c < v; ++c)
                            for (int d = 0; d < v; ++d)
                                s += Vab[(size_t)c * v + d] * tij[(size_t)c * v + d];
                        r = s;
                    }
                    R[(((size_t)i * o + j) * nav + k) * v + b] = r;
                }
            }
        }
        free(Vab);
        free(Vc);
    }
}

/*
 * Selected entries R[i,j,a,b] of Eq. 6, one by one, for spot checks of workloads whose full
 * oracle would take hours.  idx[k] = ((i*o + j)*v + a)*v + b.  Each entry builds its own
 * slice (ac|bd) over all (c, d) (Eq. 5, P in increasing order) and contracts it with t_ij
 * (c then d), the same sums in the same order as oracle_ladder's entry.
 */
void oracle_ladder_entries(int o, int v, int n, const double* L, const double* t2, const long long* idx,
                           int nidx, double* out, int nthreads)
{
    set_threads(nthreads);
    const size_t vv = (size_t)v * v;
#pragma omp parallel
    {
        double* Vab = (double*)malloc(sizeof(double) * vv);
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < nidx; ++k) {
            long long q = idx[k];
            const int b = (int)(q % v); q /= v;
            const int a = (int)(q % v); q /= v;
            const int j = (int)(q % o); q /= o;
            const int i = (int)q;
            for (size_t e = 0; e < vv; ++e) Vab[e] = 0.0;
            for (int P = 0; P < n; ++P) {
                const double* La = L + (size_t)P * vv + (size_t)a * v;
                const double* Lb = L + (size_t)P * vv + (size_t)b * v;
                for (int c = 0; c < v; ++c)
                    for (int d = 0; d < v; ++d) Vab[(size_t)c * v + d] += La[c] * Lb[d];
            }
            const double* tij = t2 + ((size_t)i * o + j) * vv;
            double r = 0.0;
            for (int c = 0; c < v; ++c)
                for (int d = 0; d < v; ++d) r += Vab[(size_t)c * v + d] * tij[(size_t)c * v + d];
            out[k] = r;
        }
        free(Vab);
    }
}

/*
 * Brute force for tiny inputs, the integral-first path of Section 3.2: build
 * the whole dense integral tensor ERI[a][c][b][d] = sum_P L_Pac L_Pbd
 * (Eq. 5, v^4 doubles), then contract it with t over (c, d) (Eq. 4).
 * ERI is caller-provided scratch of v^4 doubles.
 */
void oracle_ladder_eri(int o, int v, int n, const double* L, const double* t2, double* R,
                       double* ERI)
{
    const size_t vv = (size_t)v * v;
    for (int a = 0; a < v; ++a)
        for (int c = 0; c < v; ++c)
            for (int b = 0; b < v; ++b)
                for (int d = 0; d < v; ++d) {
                    double s = 0.0;
                    for (int P = 0; P < n; ++P)
                        s += L[(size_t)P * vv + (size_t)a * v + c] * L[(size_t)P * vv + (size_t)b * v + d];
                    ERI[(((size_t)a * v + c) * v + b) * v + d] = s;
                }
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += ERI[(((size_t)a * v + c) * v + b) * v + d] *
                                 t2[(((size_t)i * o + j) * v + c) * v + d];
                    R[(((size_t)i * o + j) * v + a) * v + b] = s;
                }
}

/*
 * Closed-shell pair energy in the form E = sum_ijab (2 R_ijab - R_ijba) t_ijab
 * (the paper implies an energy evaluation in every CC iteration step, Table 2,
 * but prints no formula; this is the spin-adapted closed-shell form).
 * Neumaier-compensated.  e_pair (nullable) receives e_ij = sum_ab (...), o x o.
 */
double oracle_energy(int o, int v, const double* R, const double* t2, double* e_pair)
{
    const size_t vv = (size_t)v * v;
    nsum_t tot = {0.0, 0.0};
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j) {
            nsum_t s = {0.0, 0.0};
            const size_t ij = ((size_t)i * o + j) * vv;
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b)
                    nsum_add(&s, (2.0 * R[ij + (size_t)a * v + b] - R[ij + (size_t)b * v + a]) *
                                     t2[ij + (size_t)a * v + b]);
            if (e_pair) e_pair[(size_t)i * o + j] = nsum_get(&s);
            nsum_add(&tot, nsum_get(&s));
        }
    return nsum_get(&tot);
}

/*
 * The share of the pair energy that one part of an `a`-range partition owns:
 * the terms (2 R_ijab - R_ijba) t_ijab of the sum above whose smaller virtual
 * index min(a, b) lies in [lo, hi).  Both R_ijab and R_ijba of such a term belong
 * to that part (the pair-symmetric path writes R[.,.,a,b] and R[.,.,b,a] for the
 * a of its range and every b >= a), and the shares of disjoint ranges covering
 * [0, v) add up to the full sum.  Plain loops over every (i, j, a, b), Neumaier sums.
 */
double oracle_energy_range(int o, int v, const double* R, const double* t2, int lo, int hi)
{
    const size_t vv = (size_t)v * v;
    nsum_t tot = {0.0, 0.0};
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j) {
            const size_t ij = ((size_t)i * o + j) * vv;
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b) {
                    const int m = a < b ? a : b;
                    if (m < lo || m >= hi) continue;
                    nsum_add(&tot, (2.0 * R[ij + (size_t)a * v + b] - R[ij + (size_t)b * v + a]) *
                                       t2[ij + (size_t)a * v + b]);
                }
        }
    return nsum_get(&tot);
}

/*
 * Gradient of loss = sum_ijab W_ijab R_ijab, R from Eq. 6, with respect to
 * t2 and L, written out literally (no symmetry of L or t2 assumed):
 *
 *   dt2[i,j,c,d] = sum_{a,b} W_ijab (sum_P L_Pac L_Pbd)
 *   dL[P,e,f]    = sum_{ij,b,d} W_ijeb L_Pbd t_ijfd      (L appears as L_Pac, a=e, c=f)
 *                + sum_{ij,a,c} W_ijae L_Pac t_ijcf      (L appears as L_Pbd, b=e, d=f)
 *
 * Either output pointer may be NULL.  Cost O((o^2 + n) v^4); small sizes only.
 */
void oracle_ladder_grad(int o, int v, int n, const double* L, const double* t2, const double* W,
                        double* dL, double* dt2, int nthreads)
{
    set_threads(nthreads);
    const size_t vv = (size_t)v * v;
    if (dt2) {
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
        for (int c = 0; c < v; ++c)
            for (int d = 0; d < v; ++d) {
                for (int i = 0; i < o; ++i)
                    for (int j = 0; j < o; ++j) {
                        const double* Wij = W + ((size_t)i * o + j) * vv;
                        double s = 0.0;
                        for (int a = 0; a < v; ++a)
                            for (int b = 0; b < v; ++b) {
                                double eri = 0.0;
                                for (int P = 0; P < n; ++P)
                                    eri += L[(size_t)P * vv + (size_t)a * v + c] *
                                           L[(size_t)P * vv + (size_t)b * v + d];
                                s += Wij[(size_t)a * v + b] * eri;
                            }
                        dt2[((size_t)i * o + j) * vv + (size_t)c * v + d] = s;
                    }
            }
    }
    if (dL) {
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
        for (int e = 0; e < v; ++e)
            for (int f = 0; f < v; ++f) {
                for (int P = 0; P < n; ++P) {
                    const double* LP = L + (size_t)P * vv;
                    double s1 = 0.0, s2 = 0.0;
                    for (int i = 0; i < o; ++i)
                        for (int j = 0; j < o; ++j) {
                            const size_t ij = ((size_t)i * o + j) * vv;
                            for (int b = 0; b < v; ++b)
                                for (int d = 0; d < v; ++d)
                                    s1 += W[ij + (size_t)e * v + b] * LP[(size_t)b * v + d] *
                                          t2[ij + (size_t)f * v + d];
                            for (int a = 0; a < v; ++a)
                                for (int c = 0; c < v; ++c)
                                    s2 += W[ij + (size_t)a * v + e] * LP[(size_t)a * v + c] *
                                          t2[ij + (size_t)c * v + f];
                        }
                    dL[(size_t)P * vv + (size_t)e * v + f] = s1 + s2;
                }
            }
    }
}

/*
 * Selected gradient entries, one by one, for full-size spot checks.
 * dt2_idx[k] = (i, j, c, d) flattened as ((i*o+j)*v+c)*v+d; dL_idx[k] = (P, e, f)
 * flattened as (P*v+e)*v+f.  Same formulas as oracle_ladder_grad.
 */
void oracle_ladder_grad_entries(int o, int v, int n, const double* L, const double* t2,
                                const double* W, const long long* dt2_idx, int ndt2, double* dt2_out,
                                const long long* dL_idx, int ndL, double* dL_out, int nthreads)
{
    set_threads(nthreads);
    const size_t vv = (size_t)v * v;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < ndt2; ++k) {
        long long q = dt2_idx[k];
        const int d = (int)(q % v); q /= v;
        const int c = (int)(q % v); q /= v;
        const int j = (int)(q % o); q /= o;
        const int i = (int)q;
        const double* Wij = W + ((size_t)i * o + j) * vv;
        double s = 0.0;
        for (int a = 0; a < v; ++a)
            for (int b = 0; b < v; ++b) {
                double eri = 0.0;
                for (int P = 0; P < n; ++P)
                    eri += L[(size_t)P * vv + (size_t)a * v + c] * L[(size_t)P * vv + (size_t)b * v + d];
                s += Wij[(size_t)a * v + b] * eri;
            }
        dt2_out[k] = s;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < ndL; ++k) {
        long long q = dL_idx[k];
        const int f = (int)(q % v); q /= v;
        const int e = (int)(q % v); q /= v;
        const int P = (int)q;
        const double* LP = L + (size_t)P * vv;
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < o; ++i)
            for (int j = 0; j < o; ++j) {
                const size_t ij = ((size_t)i * o + j) * vv;
                for (int b = 0; b < v; ++b)
                    for (int d = 0; d < v; ++d)
                        s1 += W[ij + (size_t)e * v + b] * LP[(size_t)b * v + d] * t2[ij + (size_t)f * v + d];
                for (int a = 0; a < v; ++a)
                    for (int c = 0; c < v; ++c)
                        s2 += W[ij + (size_t)a * v + e] * LP[(size_t)a * v + c] * t2[ij + (size_t)c * v + f];
            }
        dL_out[k] = s1 + s2;
    }
}

/*
 * Exchange ladder of Eq. 7: X[i,j,a,b] = sum_{c,d} (sum_P L_Pad L_Pbc) t_ijcd,
 * the c <-> d partner of Eq. 6 that the paper benchmarks for completeness
 * (contraction "abcd,edfc->eafb").  Same a_list convention as oracle_ladder.
 */
void oracle_exchange(int o, int v, int n, const double* L, const double* t2, double* X,
                     const int* a_list, int na, int nthreads)
{
    set_threads(nthreads);
    const int nav = a_list ? na : v;
    const size_t vv = (size_t)v * v;
    const long long npairs = (long long)nav * v;
#pragma omp parallel
    {
        double* Kab = (double*)malloc(sizeof(double) * vv);
#pragma omp for schedule(dynamic, 1)
        for (long long pair = 0; pair < npairs; ++pair) {
            const int k = (int)(pair / v);
            const int b = (int)(pair % v);
            const int a = a_list ? a_list[k] : k;
            for (int c = 0; c < v; ++c)
                for (int d = 0; d < v; ++d) {
                    double s = 0.0;
                    for (int P = 0; P < n; ++P)
                        s += L[(size_t)P * vv + (size_t)a * v + d] * L[(size_t)P * vv + (size_t)b * v + c];
                    Kab[(size_t)c * v + d] = s;
                }
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    const double* tij = t2 + ((size_t)i * o + j) * vv;
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d) s += Kab[(size_t)c * v + d] * tij[(size_t)c * v + d];
                    X[(((size_t)i * o + j) * nav + k) * v + b] = s;
                }
        }
        free(Kab);
    }
}

/*
 * The two further Cholesky terms of the CCSD vector function that share the
 * ladder's contraction pattern (Section 6.1, the contraction the paper benchmarks
 * as "abcd,ecfd->efab"), with Lov[P][k][c] the occupied-virtual block of the
 * Cholesky vectors (k occupied, c virtual):
 *
 *   Eq. 8   tt_ijkl = sum_{P,c,d} L^P_kc L^P_ld t_ij^cd        O(n o^4 v^2)
 *   Eq. 9   tt_ijbk = sum_{P,c,d} L^P_bd L^P_kc t_ij^cd        O(n o^3 v^3)
 *
 * Both are G[i,j,p,q] = sum_{c,d} (sum_P A[P,p,c] B[P,q,d]) t2[i,j,c,d]:
 *   tt_ijkl[i,j,k,l] = G with A = B = Lov (np = nq = o);
 *   tt_ijbk[i,j,b,k] = G[i,j,k,b] with A = Lov (np = o), B = Lvv (nq = v).
 * Evaluated like the ladder: for each (p, q) build the v x v slice
 * W[c][d] = sum_P A[P,p,c] B[P,q,d] (P in increasing order), then contract it
 * with every t_ij.  A is n x np x v, B is n x nq x v, G is o x o x np x nq.
 */
void oracle_general(int o, int v, int n, int np_, int nq, const double* A, const double* B,
                    const double* t2, double* G, int nthreads)
{
    set_threads(nthreads);
    const size_t vv = (size_t)v * v;
    const long long npairs = (long long)np_ * nq;
#pragma omp parallel
    {
        double* W = (double*)malloc(sizeof(double) * vv);
#pragma omp for schedule(dynamic, 1)
        for (long long pair = 0; pair < npairs; ++pair) {
            const int p = (int)(pair / nq);
            const int q = (int)(pair % nq);
            for (size_t x = 0; x < vv; ++x) W[x] = 0.0;
            for (int P = 0; P < n; ++P) {
                const double* Ap = A + ((size_t)P * np_ + p) * v;
                const double* Bq = B + ((size_t)P * nq + q) * v;
                for (int c = 0; c < v; ++c)
                    for (int d = 0; d < v; ++d) W[(size_t)c * v + d] += Ap[c] * Bq[d];
            }
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    const double* tij = t2 + ((size_t)i * o + j) * vv;
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d) s += W[(size_t)c * v + d] * tij[(size_t)c * v + d];
                    G[(((size_t)i * o + j) * np_ + p) * nq + q] = s;
                }
        }
        free(W);
    }
}
