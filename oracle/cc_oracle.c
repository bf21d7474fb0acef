/*
 * cc_oracle.c -- plain, slow, explicit-loop FP64 CPU oracle for spin-orbital
 * coupled-cluster (CCSD) residuals, energies and the Jacobi+DIIS iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (arxiv 2409.06759, Sec. II A):
 *   * the CC amplitude equations <Phi_l| exp(-T) H_N exp(T) |Phi_0> = 0 and the
 *     energy <Phi_0| exp(-T) H_N exp(T) |Phi_0> = E - E_HF (Eq. amp), with
 *     T = T1 + T2, t1[i][a], t2[i][j][a][b] stored unpacked and antisymmetric
 *     (the cluster-operator definitions with the 1 and 1/4 prefactors);
 *   * the Hamiltonian of Eq. ham2q with antisymmetrised integrals <pq||rs>,
 *     here built from a factorised chemist tensor (pq|rs) = sum_L B_pq^L B_rs^L
 *     as <pq||rs> = (pr|qs) - (ps|qr);  the Fock matrix is diagonal (eps).
 *   * The residual is written out in the Stanton-Gauss intermediate form of the
 *     spin-orbital CCSD equations (the pedagogical presentation the paper
 *     follows for its diagram rules), with R = RHS - D*t.  Its correctness is
 *     pinned by a determinant-space brute force, FCI for two electrons and the
 *     MP2 closed form (tests), not by this file.
 *
 * Memory: the full n^4 antisymmetrised integral tensor is held (small systems).
 * The sampled-element routines at the end work from B directly for large n.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long ll;

/* The same source is compiled twice: real (orc_*) and, with CC_COMPLEX,
 * complex double (orz_*) for complex Hermitian integrals (relativistic
 * spinors).  The CC equations are polynomial in t and <pq||rs> with no
 * conjugation, so only the scalar type changes; norms and DIIS overlaps use
 * Re<x|y>, orbital energies and denominators stay real. */
#ifdef CC_COMPLEX
typedef double complex sc;
#define FN(name) orz_##name
#define ABS2(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define RDOT(a, b) (creal(a) * creal(b) + cimag(a) * cimag(b))
#else
typedef double sc;
#define FN(name) orc_##name
#define ABS2(x) ((x) * (x))
#define RDOT(a, b) ((a) * (b))
#endif

/* ---------------------------------------------------------------- integrals */

/* <pq||rs> = (pr|qs) - (ps|qr),  (pq|rs) = sum_L B[L][p][q] B[L][r][s]. */
int FN(antisym_integrals)(int o, int v, int L, const sc *B, sc *V)
{
    const ll n = o + v;
    sc *chem = (sc *)malloc(sizeof(sc) * n * n * n * n);
    if (!chem) return 1;
#pragma omp parallel for schedule(static)
    for (ll pq = 0; pq < n * n; pq++) {
        for (ll rs = 0; rs < n * n; rs++) {
            sc s = 0.0;
            for (ll l = 0; l < L; l++) s += B[l * n * n + pq] * B[l * n * n + rs];
            chem[pq * n * n + rs] = s;
        }
    }
#pragma omp parallel for schedule(static)
    for (ll p = 0; p < n; p++)
        for (ll q = 0; q < n; q++)
            for (ll r = 0; r < n; r++)
                for (ll s = 0; s < n; s++) {
                    sc prqs = chem[((p * n + r) * n + q) * n + s];
                    sc psqr = chem[((p * n + s) * n + q) * n + r];
                    V[((p * n + q) * n + r) * n + s] = prqs - psqr;
                }
    free(chem);
    return 0;
}

/* ------------------------------------------------------------- CCSD terms */

#define VV(p, q, r, s) V[(((ll)(p) * n + (q)) * n + (r)) * n + (s)]
#define T1(i, a) t1[(ll)(i) * v + (a)]
#define T2(i, j, a, b) t2[(((ll)(i) * o + (j)) * v + (a)) * v + (b)]
#define O4(x, i, j, a, b) x[(((ll)(i) * o + (j)) * v + (a)) * v + (b)]

/* Residual R = <Phi_l|Hbar|Phi_0> for l = singles, doubles.  eps[n] holds the
 * diagonal Fock matrix (occupied first).  Returns 0 on success. */
int FN(ccsd_residual)(int o, int v, const double *eps, const sc *V,
                      const sc *t1, const sc *t2, sc *r1, sc *r2)
{
    const ll n = o + v;
    const ll ov2 = (ll)o * o * v * v;
    sc *tau = malloc(sizeof(sc) * ov2);
    sc *taut = malloc(sizeof(sc) * ov2);
    sc *Fae = malloc(sizeof(sc) * v * v);
    sc *Fmi = malloc(sizeof(sc) * o * o);
    sc *Fme = malloc(sizeof(sc) * o * v);
    sc *Fbe2 = malloc(sizeof(sc) * v * v);   /* F_be - 1/2 sum_m t_m^b F_me */
    sc *Fmj2 = malloc(sizeof(sc) * o * o);   /* F_mj + 1/2 sum_e t_j^e F_me */
    sc *Wmnij = malloc(sizeof(sc) * o * o * o * o);
    sc *Wabef = malloc(sizeof(sc) * (ll)v * v * v * v);
    sc *Wmbej = malloc(sizeof(sc) * (ll)o * v * v * o);
    sc *X = malloc(sizeof(sc) * ov2);
    if (!tau || !taut || !Fae || !Fmi || !Fme || !Fbe2 || !Fmj2 || !Wmnij || !Wabef || !Wmbej || !X)
        return 1;

    /* tau = t2 + t_i^a t_j^b - t_i^b t_j^a ; tau~ with a factor 1/2 on the t1 part */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc p = T1(i, a) * T1(j, b) - T1(i, b) * T1(j, a);
                    O4(tau, i, j, a, b) = T2(i, j, a, b) + p;
                    O4(taut, i, j, a, b) = T2(i, j, a, b) + 0.5 * p;
                }

    /* F_ae = sum_mf t_m^f <ma||fe> - 1/2 sum_mnf tau~_mn^af <mn||ef>   (f_ae off-diagonal = 0, f_me = 0) */
#pragma omp parallel for
    for (int a = 0; a < v; a++)
        for (int e = 0; e < v; e++) {
            sc s = 0.0;
            for (int m = 0; m < o; m++)
                for (int f = 0; f < v; f++) s += T1(m, f) * VV(m, o + a, o + f, o + e);
            for (int m = 0; m < o; m++)
                for (int nn = 0; nn < o; nn++)
                    for (int f = 0; f < v; f++) s -= 0.5 * O4(taut, m, nn, a, f) * VV(m, nn, o + e, o + f);
            Fae[a * v + e] = s;
        }
    /* F_mi = sum_en t_n^e <mn||ie> + 1/2 sum_nef tau~_in^ef <mn||ef> */
    for (int m = 0; m < o; m++)
        for (int i = 0; i < o; i++) {
            sc s = 0.0;
            for (int e = 0; e < v; e++)
                for (int nn = 0; nn < o; nn++) s += T1(nn, e) * VV(m, nn, i, o + e);
            for (int nn = 0; nn < o; nn++)
                for (int e = 0; e < v; e++)
                    for (int f = 0; f < v; f++) s += 0.5 * O4(taut, i, nn, e, f) * VV(m, nn, o + e, o + f);
            Fmi[m * o + i] = s;
        }
    /* F_me = sum_nf t_n^f <mn||ef> */
    for (int m = 0; m < o; m++)
        for (int e = 0; e < v; e++) {
            sc s = 0.0;
            for (int nn = 0; nn < o; nn++)
                for (int f = 0; f < v; f++) s += T1(nn, f) * VV(m, nn, o + e, o + f);
            Fme[m * v + e] = s;
        }
    for (int b = 0; b < v; b++)
        for (int e = 0; e < v; e++) {
            sc s = Fae[b * v + e];
            for (int m = 0; m < o; m++) s -= 0.5 * T1(m, b) * Fme[m * v + e];
            Fbe2[b * v + e] = s;
        }
    for (int m = 0; m < o; m++)
        for (int j = 0; j < o; j++) {
            sc s = Fmi[m * o + j];
            for (int e = 0; e < v; e++) s += 0.5 * T1(j, e) * Fme[m * v + e];
            Fmj2[m * o + j] = s;
        }

    /* W_mnij = <mn||ij> + P(ij) sum_e t_j^e <mn||ie> + 1/4 sum_ef tau_ij^ef <mn||ef> */
    for (int m = 0; m < o; m++)
        for (int nn = 0; nn < o; nn++)
            for (int i = 0; i < o; i++)
                for (int j = 0; j < o; j++) {
                    sc s = VV(m, nn, i, j);
                    for (int e = 0; e < v; e++)
                        s += T1(j, e) * VV(m, nn, i, o + e) - T1(i, e) * VV(m, nn, j, o + e);
                    for (int e = 0; e < v; e++)
                        for (int f = 0; f < v; f++) s += 0.25 * O4(tau, i, j, e, f) * VV(m, nn, o + e, o + f);
                    Wmnij[((m * o + nn) * o + i) * o + j] = s;
                }

    /* W_abef = <ab||ef> - P(ab) sum_m t_m^b <am||ef> + 1/4 sum_mn tau_mn^ab <mn||ef> */
#pragma omp parallel for
    for (int a = 0; a < v; a++)
        for (int b = 0; b < v; b++)
            for (int e = 0; e < v; e++)
                for (int f = 0; f < v; f++) {
                    sc s = VV(o + a, o + b, o + e, o + f);
                    for (int m = 0; m < o; m++)
                        s -= T1(m, b) * VV(o + a, m, o + e, o + f) - T1(m, a) * VV(o + b, m, o + e, o + f);
                    for (int m = 0; m < o; m++)
                        for (int nn = 0; nn < o; nn++) s += 0.25 * O4(tau, m, nn, a, b) * VV(m, nn, o + e, o + f);
                    Wabef[(((ll)a * v + b) * v + e) * v + f] = s;
                }

    /* W_mbej = <mb||ej> + sum_f t_j^f <mb||ef> - sum_n t_n^b <mn||ej>
     *          - sum_nf (1/2 t_jn^fb + t_j^f t_n^b) <mn||ef>                   */
#pragma omp parallel for
    for (int m = 0; m < o; m++)
        for (int b = 0; b < v; b++)
            for (int e = 0; e < v; e++)
                for (int j = 0; j < o; j++) {
                    sc s = VV(m, o + b, o + e, j);
                    for (int f = 0; f < v; f++) s += T1(j, f) * VV(m, o + b, o + e, o + f);
                    for (int nn = 0; nn < o; nn++) s -= T1(nn, b) * VV(m, nn, o + e, j);
                    for (int nn = 0; nn < o; nn++)
                        for (int f = 0; f < v; f++)
                            s -= (0.5 * T2(j, nn, f, b) + T1(j, f) * T1(nn, b)) * VV(m, nn, o + e, o + f);
                    Wmbej[(((ll)m * v + b) * v + e) * o + j] = s;
                }

    /* ---- T1 residual */
    for (int i = 0; i < o; i++)
        for (int a = 0; a < v; a++) {
            sc s = 0.0;
            for (int e = 0; e < v; e++) s += T1(i, e) * Fae[a * v + e];
            for (int m = 0; m < o; m++) s -= T1(m, a) * Fmi[m * o + i];
            for (int m = 0; m < o; m++)
                for (int e = 0; e < v; e++) s += T2(i, m, a, e) * Fme[m * v + e];
            for (int nn = 0; nn < o; nn++)
                for (int f = 0; f < v; f++) s -= T1(nn, f) * VV(nn, o + a, i, o + f);
            for (int m = 0; m < o; m++)
                for (int e = 0; e < v; e++)
                    for (int f = 0; f < v; f++) s -= 0.5 * T2(i, m, e, f) * VV(m, o + a, o + e, o + f);
            for (int m = 0; m < o; m++)
                for (int e = 0; e < v; e++)
                    for (int nn = 0; nn < o; nn++) s -= 0.5 * T2(m, nn, a, e) * VV(nn, m, o + e, i);
            s -= (eps[i] - eps[o + a]) * T1(i, a);
            r1[(ll)i * v + a] = s;
        }

    /* ---- T2 residual: start from <ab||ij> - D t2 (the doubles projection of
     * H|Phi_0> creates a, b and annihilates i, j; equal to <ij||ab> only for
     * real orbitals) */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++)
                    O4(r2, i, j, a, b) = VV(o + a, o + b, i, j)
                        - (eps[i] + eps[j] - eps[o + a] - eps[o + b]) * T2(i, j, a, b);

    /* + P(ab) sum_e t_ij^ae (F_be - 1/2 sum_m t_m^b F_me) */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int e = 0; e < v; e++) s += T2(i, j, a, e) * Fbe2[b * v + e];
                    O4(X, i, j, a, b) = s;
                }
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) O4(r2, i, j, a, b) += O4(X, i, j, a, b) - O4(X, i, j, b, a);

    /* - P(ij) sum_m t_im^ab (F_mj + 1/2 sum_e t_j^e F_me) */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int m = 0; m < o; m++) s += T2(i, m, a, b) * Fmj2[m * o + j];
                    O4(X, i, j, a, b) = s;
                }
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) O4(r2, i, j, a, b) -= O4(X, i, j, a, b) - O4(X, j, i, a, b);

    /* + 1/2 sum_mn tau_mn^ab W_mnij  + 1/2 sum_ef tau_ij^ef W_abef */
#pragma omp parallel for
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int m = 0; m < o; m++)
                        for (int nn = 0; nn < o; nn++)
                            s += 0.5 * O4(tau, m, nn, a, b) * Wmnij[((m * o + nn) * o + i) * o + j];
                    for (int e = 0; e < v; e++)
                        for (int f = 0; f < v; f++)
                            s += 0.5 * O4(tau, i, j, e, f) * Wabef[(((ll)a * v + b) * v + e) * v + f];
                    O4(r2, i, j, a, b) += s;
                }

    /* + P(ij)P(ab) sum_me (t_im^ae W_mbej - t_i^e t_m^a <mb||ej>) */
#pragma omp parallel for
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int m = 0; m < o; m++)
                        for (int e = 0; e < v; e++)
                            s += T2(i, m, a, e) * Wmbej[(((ll)m * v + b) * v + e) * o + j]
                               - T1(i, e) * T1(m, a) * VV(m, o + b, o + e, j);
                    O4(X, i, j, a, b) = s;
                }
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++)
                    O4(r2, i, j, a, b) += O4(X, i, j, a, b) - O4(X, j, i, a, b)
                                        - O4(X, i, j, b, a) + O4(X, j, i, b, a);

    /* + P(ij) sum_e t_i^e <ab||ej> */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int e = 0; e < v; e++) s += T1(i, e) * VV(o + a, o + b, o + e, j);
                    O4(X, i, j, a, b) = s;
                }
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) O4(r2, i, j, a, b) += O4(X, i, j, a, b) - O4(X, j, i, a, b);

    /* - P(ab) sum_m t_m^a <mb||ij> */
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc s = 0.0;
                    for (int m = 0; m < o; m++) s += T1(m, a) * VV(m, o + b, i, j);
                    O4(X, i, j, a, b) = s;
                }
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) O4(r2, i, j, a, b) -= O4(X, i, j, a, b) - O4(X, i, j, b, a);

    free(tau); free(taut); free(Fae); free(Fmi); free(Fme); free(Fbe2); free(Fmj2);
    free(Wmnij); free(Wabef); free(Wmbej); free(X);
    return 0;
}

/* E_CC - E_ref = sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b  (f_ia = 0) */
sc FN(ccsd_energy)(int o, int v, const sc *V, const sc *t1, const sc *t2)
{
    const ll n = o + v;
    sc e = 0.0;
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++)
                    e += VV(i, j, o + a, o + b) * (0.25 * T2(i, j, a, b) + 0.5 * T1(i, a) * T1(j, b));
    return e;
}

/* ------------------------------------------------------------------ DIIS */

/* Solve [B 1; 1^T 0][c; lambda] = [0; 1] (size m+1) by Gaussian elimination with
 * partial pivoting.  B is first scaled by 1/max(diag B).  Returns 0, or 1 if a
 * pivot falls below 1e-14 in magnitude (caller drops the oldest vector). */
#ifndef CC_COMPLEX
int orc_diis_coeffs(int m, const double *Bmat, double *c)
{
    int N = m + 1;
    double A[17][18];
    double dmax = 0.0;
    for (int k = 0; k < m; k++) if (Bmat[k * m + k] > dmax) dmax = Bmat[k * m + k];
    if (!(dmax > 0.0)) return 1;
    for (int r = 0; r < N; r++)
        for (int col = 0; col <= N; col++) A[r][col] = 0.0;
    for (int r = 0; r < m; r++) {
        for (int col = 0; col < m; col++) A[r][col] = Bmat[r * m + col] / dmax;
        A[r][m] = 1.0;
        A[m][r] = 1.0;
    }
    A[m][N] = 1.0;                          /* right-hand side column */
    for (int col = 0; col < N; col++) {
        int piv = col;
        for (int r = col + 1; r < N; r++) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (fabs(A[piv][col]) < 1e-14) return 1;
        if (piv != col)
            for (int k = 0; k <= N; k++) { double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
        for (int r = col + 1; r < N; r++) {
            double fac = A[r][col] / A[col][col];
            for (int k = col; k <= N; k++) A[r][k] -= fac * A[col][k];
        }
    }
    double x[17];
    for (int r = N - 1; r >= 0; r--) {
        double s = A[r][N];
        for (int k = r + 1; k < N; k++) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    for (int k = 0; k < m; k++) c[k] = x[k];
    return 0;
}

#else
int orc_diis_coeffs(int m, const double *Bmat, double *c);
#endif

/* Jacobi + DIIS on x = (t1, t2).  Iteration k: R_k = R(x_k), E_k = E(x_k),
 * |R_k| = Frobenius norm over the full t1 and t2 residual arrays.  Stop when
 * |R_k| < tol.  Otherwise x'_{k+1} = x_k + R_k/D, e_k = R_k/D; keep the last
 * diis_max pairs (x', e); with two or more stored, x_{k+1} = sum_l c_l x'_l with
 * c from orc_diis_coeffs (oldest dropped while the solve is singular), else
 * x_{k+1} = x'_{k+1}.  t1/t2 hold the start on entry and the last x_k on exit.
 * energies/rnorms receive E_k and |R_k| (maxiter entries).  Returns 0 when
 * converged, 2 when maxiter is reached, 3 on a non-finite or exploding norm. */
int FN(ccsd_solve)(int o, int v, const double *eps, const sc *V, sc *t1, sc *t2,
                   double tol, int maxiter, int diis_max, sc *energies, double *rnorms, int *iters)
{
    const ll n1 = (ll)o * v, n2 = (ll)o * o * v * v, nx = n1 + n2;
    if (diis_max > 16) diis_max = 16;
    sc *r1 = malloc(sizeof(sc) * n1), *r2 = malloc(sizeof(sc) * n2);
    double *D = malloc(sizeof(double) * nx);
    sc *hx = malloc(sizeof(sc) * nx * (diis_max > 0 ? diis_max : 1));
    sc *he = malloc(sizeof(sc) * nx * (diis_max > 0 ? diis_max : 1));
    if (!r1 || !r2 || !D || !hx || !he) return 1;
    for (int i = 0; i < o; i++)
        for (int a = 0; a < v; a++) D[(ll)i * v + a] = eps[i] - eps[o + a];
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++)
                    D[n1 + (((ll)i * o + j) * v + a) * v + b] = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    int nstored = 0, status = 2;
    double best = INFINITY;
    int k;
    for (k = 0; k < maxiter; k++) {
        FN(ccsd_residual)(o, v, eps, V, t1, t2, r1, r2);
        sc e = FN(ccsd_energy)(o, v, V, t1, t2);
        double s = 0.0;
        for (ll q = 0; q < n1; q++) s += ABS2(r1[q]);
        for (ll q = 0; q < n2; q++) s += ABS2(r2[q]);
        double rn = sqrt(s);
        energies[k] = e;
        rnorms[k] = rn;
        if (!isfinite(rn) || rn > 1e3 * best) { status = 3; k++; break; }
        if (rn < best) best = rn;
        if (rn < tol) { status = 0; k++; break; }
        /* push (x', e) as the newest entry; drop the oldest when full */
        if (diis_max > 0 && nstored == diis_max) {
            memmove(hx, hx + nx, sizeof(sc) * nx * (diis_max - 1));
            memmove(he, he + nx, sizeof(sc) * nx * (diis_max - 1));
            nstored--;
        }
        sc *xn = hx + nx * (diis_max > 0 ? nstored : 0);
        sc *en = he + nx * (diis_max > 0 ? nstored : 0);
        for (ll q = 0; q < n1; q++) { en[q] = r1[q] / D[q]; xn[q] = t1[q] + en[q]; }
        for (ll q = 0; q < n2; q++) { en[n1 + q] = r2[q] / D[n1 + q]; xn[n1 + q] = t2[q] + en[n1 + q]; }
        if (diis_max > 0) nstored++;
        if (nstored >= 2) {
            double Bm[256], c[16];
            int ok;
            for (;;) {
                int m = nstored;
                for (int a = 0; a < m; a++)
                    for (int b = 0; b < m; b++) {
                        double d = 0.0;
                        for (ll q = 0; q < nx; q++) d += RDOT(he[nx * a + q], he[nx * b + q]);
                        Bm[a * m + b] = d;
                    }
                ok = (orc_diis_coeffs(m, Bm, c) == 0);
                if (ok || m <= 2) break;
                memmove(hx, hx + nx, sizeof(sc) * nx * (m - 1));
                memmove(he, he + nx, sizeof(sc) * nx * (m - 1));
                nstored--;
            }
            if (ok) {
                for (ll q = 0; q < nx; q++) {
                    sc s2 = 0.0;
                    for (int a = 0; a < nstored; a++) s2 += c[a] * hx[nx * a + q];
                    if (q < n1) t1[q] = s2; else t2[q - n1] = s2;
                }
            } else {
                const sc *xl = hx + nx * (nstored - 1);
                memcpy(t1, xl, sizeof(sc) * n1);
                memcpy(t2, xl + n1, sizeof(sc) * n2);
            }
        } else {
            memcpy(t1, xn, sizeof(sc) * n1);
            memcpy(t2, xn + n1, sizeof(sc) * n2);
        }
    }
    *iters = k;
    free(r1); free(r2); free(D); free(hx); free(he);
    return status;
}

#ifndef CC_COMPLEX
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
#endif

/* --------------------------------------------------------- sampled R2 elements
 *
 * Selected elements R_ij^ab of the same CCSD residual (same equations as
 * orc_ccsd_residual), for systems whose n^4 integral tensor does not fit:
 * integrals are formed from B on demand, <pq||rs> = sum_L B_pr B_qs - B_ps B_qr.
 * Built once: the oovv, ooov and ovvv blocks, tau, tau~ and the one-particle
 * intermediates.  Per sample: the W_mnij(.,.,i,j), W_abef(a,b,.,.) and
 * W_mbej(.,d,.,q) slices that element needs.  OpenMP over samples.
 */
typedef struct {
    int o, v, n, L;
    const sc *Bt;                     /* [p][r][L] */
    sc *oovv, *ooov, *ovvv;           /* <mn||ef>, <mn||ie>, <ma||ef> */
} vsrc;

static sc vint(const vsrc *S, int p, int q, int r, int s)
{
    const sc *a = S->Bt + ((ll)p * S->n + r) * S->L, *b = S->Bt + ((ll)q * S->n + s) * S->L;
    const sc *c = S->Bt + ((ll)p * S->n + s) * S->L, *d = S->Bt + ((ll)q * S->n + r) * S->L;
    sc x = 0.0;
    for (int l = 0; l < S->L; l++) x += a[l] * b[l] - c[l] * d[l];
    return x;
}

#define OOVV(m, nn, e, f) S.oovv[(((ll)(m) * o + (nn)) * v + (e)) * v + (f)]
#define OOOV(m, nn, i, e) S.ooov[(((ll)(m) * o + (nn)) * o + (i)) * v + (e)]
#define OVVV(m, a, e, f) S.ovvv[(((ll)(m) * v + (a)) * v + (e)) * v + (f)]

/* X_pqcd = sum_me ( t_pm^ce W_mdeq - t_p^e t_m^c <md||eq> ) for the ring term */
static sc ring_x(const vsrc *Sp, const sc *t1, const sc *t2, int p, int q, int c, int dd)
{
    const vsrc S = *Sp;
    const int o = S.o, v = S.v;
    sc x = 0.0;
    for (int m = 0; m < o; m++)
        for (int e = 0; e < v; e++) {
            /* W_mbej with b = dd, j = q */
            sc w = vint(&S, m, o + dd, o + e, q);
            for (int f = 0; f < v; f++) w += T1(q, f) * OVVV(m, dd, e, f);
            for (int nn = 0; nn < o; nn++) w += T1(nn, dd) * OOOV(m, nn, q, e);   /* -t_n^b <mn||ej> */
            for (int nn = 0; nn < o; nn++)
                for (int f = 0; f < v; f++)
                    w -= (0.5 * T2(q, nn, f, dd) + T1(q, f) * T1(nn, dd)) * OOVV(m, nn, e, f);
            x += T2(p, m, c, e) * w - T1(p, e) * T1(m, c) * vint(&S, m, o + dd, o + e, q);
        }
    return x;
}

/* What the per-element evaluation reads: the integral source, tau, tau~ and the
 * one-particle intermediates, built once per (B, t1, t2). */
typedef struct {
    vsrc S;
    const double *eps;
    const sc *t1, *t2;
    sc *Bt, *tau, *taut, *Fae, *Fmi, *Fme, *Fbe2, *Fmj2;
} FN(r2s);

void FN(ccsd_r2_sample_free)(void *h)
{
    FN(r2s) *R = (FN(r2s) *)h;
    if (!R) return;
    free(R->Bt); free(R->S.oovv); free(R->S.ooov); free(R->S.ovvv); free(R->tau); free(R->taut);
    free(R->Fae); free(R->Fmi); free(R->Fme); free(R->Fbe2); free(R->Fmj2);
    free(R);
}

/* Builds the shared part; eps, t1, t2 are kept by pointer and must outlive the
 * handle.  Returns NULL when an allocation fails. */
void *FN(ccsd_r2_sample_prepare)(int o, int v, int L, const sc *B, const double *eps, const sc *t1,
                                 const sc *t2)
{
    const ll n = o + v;
    FN(r2s) *R = calloc(1, sizeof(FN(r2s)));
    if (!R) return NULL;
    vsrc S;
    S.o = o; S.v = v; S.n = (int)n; S.L = L;
    sc *Bt = malloc(sizeof(sc) * n * n * L);
    S.oovv = malloc(sizeof(sc) * (ll)o * o * v * v);
    S.ooov = malloc(sizeof(sc) * (ll)o * o * o * v);
    S.ovvv = malloc(sizeof(sc) * (ll)o * v * v * v);
    sc *tau = malloc(sizeof(sc) * (ll)o * o * v * v), *taut = malloc(sizeof(sc) * (ll)o * o * v * v);
    sc *Fae = malloc(sizeof(sc) * v * v), *Fmi = malloc(sizeof(sc) * o * o);
    sc *Fme = malloc(sizeof(sc) * o * v), *Fbe2 = malloc(sizeof(sc) * v * v);
    sc *Fmj2 = malloc(sizeof(sc) * o * o);
    R->Bt = Bt; R->S = S; R->tau = tau; R->taut = taut; R->Fae = Fae; R->Fmi = Fmi; R->Fme = Fme;
    R->Fbe2 = Fbe2; R->Fmj2 = Fmj2; R->eps = eps; R->t1 = t1; R->t2 = t2;
    if (!Bt || !S.oovv || !S.ooov || !S.ovvv || !tau || !taut || !Fae || !Fmi || !Fme || !Fbe2 || !Fmj2) {
        FN(ccsd_r2_sample_free)(R);
        return NULL;
    }
#pragma omp parallel for
    for (ll pr = 0; pr < n * n; pr++)
        for (int l = 0; l < L; l++) Bt[pr * L + l] = B[(ll)l * n * n + pr];
    S.Bt = Bt;
#pragma omp parallel for collapse(2)
    for (int m = 0; m < o; m++)
        for (int nn = 0; nn < o; nn++) {
            for (int e = 0; e < v; e++)
                for (int f = 0; f < v; f++) OOVV(m, nn, e, f) = vint(&S, m, nn, o + e, o + f);
            for (int i = 0; i < o; i++)
                for (int e = 0; e < v; e++) OOOV(m, nn, i, e) = vint(&S, m, nn, i, o + e);
        }
#pragma omp parallel for collapse(2)
    for (int m = 0; m < o; m++)
        for (int a = 0; a < v; a++)
            for (int e = 0; e < v; e++)
                for (int f = 0; f < v; f++) OVVV(m, a, e, f) = vint(&S, m, o + a, o + e, o + f);
    for (int i = 0; i < o; i++)
        for (int j = 0; j < o; j++)
            for (int a = 0; a < v; a++)
                for (int b = 0; b < v; b++) {
                    sc p = T1(i, a) * T1(j, b) - T1(i, b) * T1(j, a);
                    O4(tau, i, j, a, b) = T2(i, j, a, b) + p;
                    O4(taut, i, j, a, b) = T2(i, j, a, b) + 0.5 * p;
                }
#pragma omp parallel for
    for (int a = 0; a < v; a++)
        for (int e = 0; e < v; e++) {
            sc s = 0.0;
            for (int m = 0; m < o; m++)
                for (int f = 0; f < v; f++) s += T1(m, f) * OVVV(m, a, f, e);
            for (int m = 0; m < o; m++)
                for (int nn = 0; nn < o; nn++)
                    for (int f = 0; f < v; f++) s -= 0.5 * O4(taut, m, nn, a, f) * OOVV(m, nn, e, f);
            Fae[a * v + e] = s;
        }
    for (int m = 0; m < o; m++)
        for (int i = 0; i < o; i++) {
            sc s = 0.0;
            for (int e = 0; e < v; e++)
                for (int nn = 0; nn < o; nn++) s += T1(nn, e) * OOOV(m, nn, i, e);
            for (int nn = 0; nn < o; nn++)
                for (int e = 0; e < v; e++)
                    for (int f = 0; f < v; f++) s += 0.5 * O4(taut, i, nn, e, f) * OOVV(m, nn, e, f);
            Fmi[m * o + i] = s;
        }
    for (int m = 0; m < o; m++)
        for (int e = 0; e < v; e++) {
            sc s = 0.0;
            for (int nn = 0; nn < o; nn++)
                for (int f = 0; f < v; f++) s += T1(nn, f) * OOVV(m, nn, e, f);
            Fme[m * v + e] = s;
        }
    for (int b = 0; b < v; b++)
        for (int e = 0; e < v; e++) {
            sc s = Fae[b * v + e];
            for (int m = 0; m < o; m++) s -= 0.5 * T1(m, b) * Fme[m * v + e];
            Fbe2[b * v + e] = s;
        }
    for (int m = 0; m < o; m++)
        for (int j = 0; j < o; j++) {
            sc s = Fmi[m * o + j];
            for (int e = 0; e < v; e++) s += 0.5 * T1(j, e) * Fme[m * v + e];
            Fmj2[m * o + j] = s;
        }
    R->S = S;
    return R;
}

/* R_ij^ab for each row (i, j, a, b) of idx[ns][4], from a prepared handle. */
int FN(ccsd_r2_sample_eval)(void *h, int ns, const int *idx, sc *out)
{
    const FN(r2s) *R = (const FN(r2s) *)h;
    if (!R) return 1;
    const vsrc S = R->S;
    const int o = S.o, v = S.v;
    const double *eps = R->eps;
    const sc *t1 = R->t1, *t2 = R->t2, *tau = R->tau, *Fbe2 = R->Fbe2, *Fmj2 = R->Fmj2;

#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < ns; k++) {
        const int i = idx[4 * k], j = idx[4 * k + 1], a = idx[4 * k + 2], b = idx[4 * k + 3];
        sc r = vint(&S, o + a, o + b, i, j) - (eps[i] + eps[j] - eps[o + a] - eps[o + b]) * T2(i, j, a, b);
        /* P(ab) sum_e t_ij^ae Fbe2_be  and  -P(ij) sum_m t_im^ab Fmj2_mj */
        for (int e = 0; e < v; e++) r += T2(i, j, a, e) * Fbe2[b * v + e] - T2(i, j, b, e) * Fbe2[a * v + e];
        for (int m = 0; m < o; m++) r -= T2(i, m, a, b) * Fmj2[m * o + j] - T2(j, m, a, b) * Fmj2[m * o + i];
        /* 1/2 sum_mn tau_mn^ab W_mnij */
        for (int m = 0; m < o; m++)
            for (int nn = 0; nn < o; nn++) {
                sc w = vint(&S, m, nn, i, j);
                for (int e = 0; e < v; e++) w += T1(j, e) * OOOV(m, nn, i, e) - T1(i, e) * OOOV(m, nn, j, e);
                for (int e = 0; e < v; e++)
                    for (int f = 0; f < v; f++) w += 0.25 * O4(tau, i, j, e, f) * OOVV(m, nn, e, f);
                r += 0.5 * O4(tau, m, nn, a, b) * w;
            }
        /* 1/2 sum_ef tau_ij^ef W_abef, <am||ef> = -<ma||ef> */
        for (int e = 0; e < v; e++)
            for (int f = 0; f < v; f++) {
                sc w = vint(&S, o + a, o + b, o + e, o + f);
                for (int m = 0; m < o; m++) w -= -T1(m, b) * OVVV(m, a, e, f) + T1(m, a) * OVVV(m, b, e, f);
                for (int m = 0; m < o; m++)
                    for (int nn = 0; nn < o; nn++) w += 0.25 * O4(tau, m, nn, a, b) * OOVV(m, nn, e, f);
                r += 0.5 * O4(tau, i, j, e, f) * w;
            }
        /* P(ij) P(ab) X */
        r += ring_x(&S, t1, t2, i, j, a, b) - ring_x(&S, t1, t2, j, i, a, b)
           - ring_x(&S, t1, t2, i, j, b, a) + ring_x(&S, t1, t2, j, i, b, a);
        /* P(ij) sum_e t_i^e <ab||ej>  and  -P(ab) sum_m t_m^a <mb||ij> */
        for (int e = 0; e < v; e++)
            r += T1(i, e) * vint(&S, o + a, o + b, o + e, j) - T1(j, e) * vint(&S, o + a, o + b, o + e, i);
        for (int m = 0; m < o; m++)
            r -= T1(m, a) * vint(&S, m, o + b, i, j) - T1(m, b) * vint(&S, m, o + a, i, j);
        out[k] = r;
    }
    return 0;
}

int FN(ccsd_r2_sample)(int o, int v, int L, const sc *B, const double *eps, const sc *t1,
                       const sc *t2, int ns, const int *idx, sc *out)
{
    void *h = FN(ccsd_r2_sample_prepare)(o, v, L, B, eps, t1, t2);
    if (!h) return 1;
    int rc = FN(ccsd_r2_sample_eval)(h, ns, idx, out);
    FN(ccsd_r2_sample_free)(h);
    return rc;
}
