/*
 * cc_definition.c -- coupled-cluster residual elements and energies straight
 * from their definition, with no CC equations:
 *
 *     R_l = <Phi_l| exp(-T) H_N exp(T) |Phi_0>,   E - E_ref = <Phi_0| H_N exp(T) |Phi_0>
 *
 * (arxiv 2409.06759 Sec. II A, Eq. amp; H_N of Eq. ham2q with the integrals
 * <pq||rs> = (pr|qs) - (ps|qr), (pq|rs) = sum_L B_pq^L B_rs^L).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU legs may load this code.  It shares nothing with the CUDA path, and it
 * does not use the contraction lists or the code that derives them.
 *
 * The three factors:
 *   * Psi = exp(T) Phi_0 = sum_D c_D Phi_D with Phi_D = X_D Phi_0,
 *     X_D = a+_{p1} .. a+_{pk} a_{hk} .. a_{h1} (h, p ascending), and
 *     T = sum_n sum_{I<, A<} t_I^A X_(I,A).  The excitation operators commute
 *     and square to zero, so c_D is the sum over the ways of splitting D's
 *     holes and particles into blocks of equal size n (a rank present in T) of
 *     the product of the blocks' amplitudes, times the sign that orders the
 *     blocks' operators into X_D.  Splits are enumerated by the block that
 *     holds the lowest remaining hole.
 *   * <Phi_m| H_N |Psi> = sum_D <Phi_m| H_N |Phi_D> c_D over the determinants
 *     D that differ from Phi_m in at most two spin orbitals (Slater-Condon),
 *     with h_pq = eps_p delta_pq - sum_i <pi||qi> so that the Fock operator of
 *     H is diag(eps), and E_ref = sum_i eps_i - 1/2 sum_ij <ij||ij>.
 *   * <Phi_l| exp(-T) |Phi_m> is non-zero only for Phi_m inside Phi_l: the same
 *     block sum over the excitation l \ m with amplitudes -t.
 *
 * Cost per element: a few (o v)^2 determinants, each with a block sum over at
 * most five hole-particle pairs -- polynomial, so elements of o = 8, v = 64
 * CCSDT (or o = 40, v = 200 CCSD) are reachable one at a time.
 * Pins (tests): the determinant-space brute force (full matrices) at small
 * sizes, for CCSD and CCSDT, real and complex.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long ll;
#ifdef CC_COMPLEX
typedef double complex sc;
#define FN(name) orz_##name
#else
typedef double sc;
#define FN(name) orc_##name
#endif

#define MAXN 256    /* spin orbitals */
#define MAXK 8      /* excitation level handled by the block sums */

typedef struct {
    int o, v, n, L;
    const sc *Bt;          /* [p][r][L] */
    const sc *t[4];        /* t[1], t[2], t[3] (NULL: rank absent) */
    sc *h;                 /* [n][n] one-body part */
    sc eref;
} Ctx;

static sc vint(const Ctx *C, int p, int q, int r, int s)
{
    const sc *a = C->Bt + ((ll)p * C->n + r) * C->L, *b = C->Bt + ((ll)q * C->n + s) * C->L;
    const sc *c = C->Bt + ((ll)p * C->n + s) * C->L, *d = C->Bt + ((ll)q * C->n + r) * C->L;
    sc x = 0.0;
    for (int l = 0; l < C->L; l++) x += a[l] * b[l] - c[l] * d[l];
    return x;
}

/* amplitude t_{H}^{P} of rank s for sorted hole orbitals and particle orbitals */
static sc amp(const Ctx *C, int s, const int *hs, const int *ps)
{
    const int o = C->o, v = C->v;
    const sc *t = C->t[s];
    if (s == 1) return t[(ll)hs[0] * v + (ps[0] - o)];
    if (s == 2) return t[(((ll)hs[0] * o + hs[1]) * v + (ps[0] - o)) * v + (ps[1] - o)];
    return t[(((((ll)hs[0] * o + hs[1]) * o + hs[2]) * v + (ps[0] - o)) * v + (ps[1] - o)) * v + (ps[2] - o)];
}

/* inversions of a descending merge / ascending merge between two sorted sets */
static int inv_gt(const int *x, int nx, const int *y, int ny)
{
    int c = 0;
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++) c += x[a] > y[b];
    return c;
}

/* c_D of the excitation (H, P) (k pairs, sorted): sum over block splits.
 * neg: amplitudes enter as -t (exp(-T)). */
static sc block_sum(const Ctx *C, const int *H, const int *P, int k, int neg)
{
    if (k == 0) return 1.0;
    sc total = 0.0;
    for (int s = 1; s <= 3 && s <= k; s++) {
        if (!C->t[s]) continue;
        /* other holes of the block: (s-1)-subsets of H[1..k-1]; particles: s-subsets of P */
        int hsel[3], psel[3];
        int hi[3] = {0, 0, 0}, pi[3] = {0, 0, 0};
        /* iterate hole subsets */
        int nh = k - 1, ns = s - 1;
        int hidx[3];
        for (int q = 0; q < ns; q++) hidx[q] = q;
        for (;;) {
            hsel[0] = H[0];
            for (int q = 0; q < ns; q++) hsel[q + 1] = H[1 + hidx[q]];
            int pidx[3];
            for (int q = 0; q < s; q++) pidx[q] = q;
            for (;;) {
                for (int q = 0; q < s; q++) psel[q] = P[pidx[q]];
                /* the rest, sorted */
                int Hr[MAXK], Pr[MAXK], nr = 0, nrp = 0;
                for (int q = 0; q < k; q++) {
                    int in = 0;
                    for (int z = 0; z < s; z++) in |= H[q] == hsel[z];
                    if (!in) Hr[nr++] = H[q];
                }
                for (int q = 0; q < k; q++) {
                    int in = 0;
                    for (int z = 0; z < s; z++) in |= P[q] == psel[z];
                    if (!in) Pr[nrp++] = P[q];
                }
                /* X_block X_rest = sign X_full: creators ascending, annihilators descending */
                const int r = k - s;
                int par = s * r + inv_gt(psel, s, Pr, r) + inv_gt(Hr, r, hsel, s);
                sc a = amp(C, s, hsel, psel);
                if (neg) a = -a;
                sc sub = block_sum(C, Hr, Pr, r, neg);
                total += (par & 1) ? -a * sub : a * sub;
                /* next particle subset */
                int q = s - 1;
                while (q >= 0 && pidx[q] == k - s + q) q--;
                if (q < 0) break;
                pidx[q]++;
                for (int z = q + 1; z < s; z++) pidx[z] = pidx[z - 1] + 1;
            }
            (void)hi; (void)pi;
            /* next hole subset */
            int q = ns - 1;
            while (q >= 0 && hidx[q] == nh - ns + q) q--;
            if (q < 0) break;
            hidx[q]++;
            for (int z = q + 1; z < ns; z++) hidx[z] = hidx[z - 1] + 1;
        }
    }
    return total;
}

/* ---- determinants as bit strings: |q1 < q2 < ...> = a+_q1 a+_q2 .. |vac> */
typedef struct { uint64_t w[MAXN / 64]; } Det;

static int bit(const Det *d, int p) { return (int)((d->w[p >> 6] >> (p & 63)) & 1u); }
static void setb(Det *d, int p) { d->w[p >> 6] |= 1ull << (p & 63); }
static void clrb(Det *d, int p) { d->w[p >> 6] &= ~(1ull << (p & 63)); }
static int below(const Det *d, int p)
{
    int c = 0;
    for (int q = 0; q < (p >> 6); q++) c += __builtin_popcountll(d->w[q]);
    if (p & 63) c += __builtin_popcountll(d->w[p >> 6] & ((1ull << (p & 63)) - 1));
    return c;
}
/* a_p / a+_p applied in place; returns the sign (0 when the result vanishes) */
static int ann(Det *d, int p)
{
    if (!bit(d, p)) return 0;
    int s = (below(d, p) & 1) ? -1 : 1;
    clrb(d, p);
    return s;
}
static int cre(Det *d, int p)
{
    if (bit(d, p)) return 0;
    int s = (below(d, p) & 1) ? -1 : 1;
    setb(d, p);
    return s;
}

/* X_(H,P) Phi_0 = sign * |bits> */
static int excite(const Ctx *C, const int *H, const int *P, int k, Det *out)
{
    memset(out, 0, sizeof(*out));
    for (int i = 0; i < C->o; i++) setb(out, i);
    int s = 1;
    for (int q = 0; q < k; q++) s *= ann(out, H[q]);          /* a_h1 first */
    for (int q = k - 1; q >= 0; q--) s *= cre(out, P[q]);     /* then a+_pk .. a+_p1 */
    return s;
}

/* (H, P) of a determinant relative to Phi_0 (sorted); returns k, or -1 beyond MAXK */
static int excitation_of(const Ctx *C, const Det *d, int *H, int *P)
{
    int k = 0, kp = 0;
    for (int i = 0; i < C->o; i++)
        if (!bit(d, i)) { if (k >= MAXK) return -1; H[k++] = i; }
    for (int a = C->o; a < C->n; a++)
        if (bit(d, a)) { if (kp >= MAXK) return -1; P[kp++] = a; }
    return k == kp ? k : -1;
}

/* c_D and the sign s_D of X_D Phi_0 = s_D |D>: returns s_D * c_D */
static sc coef_of_bits(const Ctx *C, const Det *d)
{
    int H[MAXK], P[MAXK];
    int k = excitation_of(C, d, H, P);
    if (k < 0) return 0.0;
    Det chk;
    int s = excite(C, H, P, k, &chk);
    sc c = block_sum(C, H, P, k, 0);
    return s < 0 ? -c : c;
}

/* <m|H_N|Psi> over the bit-string determinant m (returns <bits_m| H_N |Psi>) */
static sc h_psi(const Ctx *C, const Det *m)
{
    const int n = C->n;
    int occ[MAXN], uno[MAXN], N = 0, U = 0;
    for (int p = 0; p < n; p++) {
        if (bit(m, p)) occ[N++] = p; else uno[U++] = p;
    }
    /* diagonal */
    sc diag = -C->eref;
    for (int a = 0; a < N; a++) {
        diag += C->h[(ll)occ[a] * n + occ[a]];
        for (int b = a + 1; b < N; b++) diag += vint(C, occ[a], occ[b], occ[a], occ[b]);
    }
    sc total = diag * coef_of_bits(C, m);
    /* singles: D = m with x -> y;  <m|H|D> = (h_xy + sum_k in D <xk||yk>) * phase */
    sc *part = calloc((size_t)N * N + 1, sizeof(sc));
    if (!part) return 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < N; a++) {
        const int x = occ[a];
        sc acc = 0.0;
        for (int u = 0; u < U; u++) {
            const int y = uno[u];
            Det D = *m;
            clrb(&D, x);
            setb(&D, y);
            sc c = coef_of_bits(C, &D);
            if (c == 0.0) continue;
            Det t = D;
            int ph = ann(&t, y);
            ph *= cre(&t, x);
            sc val = C->h[(ll)x * n + y];
            for (int z = 0; z < N; z++) {
                const int kk = occ[z];
                if (kk == x) continue;
                val += vint(C, x, kk, y, kk);
            }
            acc += ph * val * c;
        }
        part[a] = acc;
    }
    for (int a = 0; a < N; a++) total += part[a];
    /* doubles: D = m with x1 < x2 -> y1 < y2;  <m|H|D> = <x1 x2||y1 y2> * phase */
    const int npair = N * (N - 1) / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int pr = 0; pr < npair; pr++) {
        int a = 0, rem = pr;
        while (rem >= N - 1 - a) { rem -= N - 1 - a; a++; }
        const int b = a + 1 + rem;
        const int x1 = occ[a], x2 = occ[b];
        sc acc = 0.0;
        for (int u1 = 0; u1 < U; u1++)
            for (int u2 = u1 + 1; u2 < U; u2++) {
                const int y1 = uno[u1], y2 = uno[u2];
                Det D = *m;
                clrb(&D, x1); clrb(&D, x2);
                setb(&D, y1); setb(&D, y2);
                sc c = coef_of_bits(C, &D);
                if (c == 0.0) continue;
                Det t = D;
                int ph = ann(&t, y1);        /* a+_x1 a+_x2 a_y2 a_y1 |D> */
                ph *= ann(&t, y2);
                ph *= cre(&t, x2);
                ph *= cre(&t, x1);
                acc += ph * vint(C, x1, x2, y1, y2) * c;
            }
        part[pr] = acc;
    }
    for (int pr = 0; pr < npair; pr++) total += part[pr];
    free(part);
    return total;
}

static int setup(Ctx *C, int o, int v, int L, const sc *B, const double *eps, const sc *t1, const sc *t2,
                 const sc *t3)
{
    const int n = o + v;
    if (n > MAXN) return 2;
    C->o = o; C->v = v; C->n = n; C->L = L;
    C->t[0] = NULL; C->t[1] = t1; C->t[2] = t2; C->t[3] = t3;
    sc *Bt = malloc(sizeof(sc) * (size_t)n * n * L);
    C->h = malloc(sizeof(sc) * (size_t)n * n);
    if (!Bt || !C->h) { free(Bt); free(C->h); return 1; }
    for (ll pr = 0; pr < (ll)n * n; pr++)
        for (int l = 0; l < L; l++) Bt[pr * L + l] = B[(ll)l * n * n + pr];
    C->Bt = Bt;
#pragma omp parallel for collapse(2)
    for (int p = 0; p < n; p++)
        for (int q = 0; q < n; q++) {
            sc x = p == q ? eps[p] : 0.0;
            for (int i = 0; i < o; i++) x -= vint(C, p, i, q, i);
            C->h[(ll)p * n + q] = x;
        }
    sc e = 0.0;
    for (int i = 0; i < o; i++) {
        e += eps[i];
        for (int j = 0; j < o; j++) e -= 0.5 * vint(C, i, j, i, j);
    }
    C->eref = e;
    return 0;
}

static void teardown(Ctx *C)
{
    free((void *)C->Bt);
    free(C->h);
}

/* sorts x[0..k) ascending, returns the permutation parity (0/1); -1 on a repeat */
static int sort_parity(int *x, int k)
{
    int par = 0;
    for (int a = 0; a < k; a++)
        for (int b = a + 1; b < k; b++) {
            if (x[a] == x[b]) return -1;
            if (x[a] > x[b]) { int t = x[a]; x[a] = x[b]; x[b] = t; par ^= 1; }
        }
    return par;
}

/*
 * Residual elements of rank `rank` (1..3; 0: the energy E - E_ref, idx unused)
 * for ns index tuples idx[ns][2*rank] = (i.., a..) (occupied 0..o-1, virtual
 * 0..v-1, any order; the result follows the antisymmetry of R).
 * B[L][n][n]; t1 [o][v], t2 [o][o][v][v], t3 [o]^3[v]^3 (t2 / t3 may be NULL:
 * that rank is absent from T).  Returns 0, 1 on allocation failure, 2 when
 * o + v > 256.
 */
int FN(cc_definition_elements)(int o, int v, int L, const sc *B, const double *eps, const sc *t1, const sc *t2,
                               const sc *t3, int rank, int ns, const int *idx, sc *out)
{
    Ctx C;
    int st = setup(&C, o, v, L, B, eps, t1, t2, t3);
    if (st) return st;
    if (rank == 0) {
        Det d;
        excite(&C, NULL, NULL, 0, &d);
        out[0] = h_psi(&C, &d);
        teardown(&C);
        return 0;
    }
    for (int e = 0; e < ns; e++) {
        int H[MAXK], P[MAXK];
        for (int q = 0; q < rank; q++) {
            H[q] = idx[e * 2 * rank + q];
            P[q] = o + idx[e * 2 * rank + rank + q];
        }
        int ph = sort_parity(H, rank), pp = sort_parity(P, rank);
        if (ph < 0 || pp < 0) { out[e] = 0.0; continue; }
        const int sgn = (ph ^ pp) ? -1 : 1;
        /* R_l = sum over Phi_m inside Phi_l of <l|exp(-T)|m> <m|H_N|Psi> */
        sc r = 0.0;
        for (int j = 0; j <= rank; j++) {
            /* j-subsets of H and of P */
            int hs[MAXK], psb[MAXK];
            for (int q = 0; q < j; q++) hs[q] = q;
            for (;;) {
                for (int q = 0; q < j; q++) psb[q] = q;
                for (;;) {
                    int Hm[MAXK], Pm[MAXK], Hd[MAXK], Pd[MAXK], nd = 0, ndp = 0;
                    for (int q = 0; q < j; q++) { Hm[q] = H[hs[q]]; Pm[q] = P[psb[q]]; }
                    for (int q = 0; q < rank; q++) {
                        int in = 0;
                        for (int z = 0; z < j; z++) in |= hs[z] == q;
                        if (!in) Hd[nd++] = H[q];
                        in = 0;
                        for (int z = 0; z < j; z++) in |= psb[z] == q;
                        if (!in) Pd[ndp++] = P[q];
                    }
                    /* <l|exp(-T)|m> = c^-(l \ m) * sign(X_m X_(l\m) = sign X_l) */
                    sc em = block_sum(&C, Hd, Pd, nd, 1);
                    if (em != 0.0) {
                        const int par = j * nd + inv_gt(Pm, j, Pd, nd) + inv_gt(Hd, nd, Hm, j);
                        Det dm;
                        const int sm = excite(&C, Hm, Pm, j, &dm);
                        sc g = h_psi(&C, &dm);                  /* <bits_m|H_N|Psi> */
                        sc term = em * g * (sc)sm;              /* <Phi_m| = s_m <bits_m| */
                        r += (par & 1) ? -term : term;
                    }
                    int q = j - 1;
                    while (q >= 0 && psb[q] == rank - j + q) q--;
                    if (q < 0) break;
                    psb[q]++;
                    for (int z = q + 1; z < j; z++) psb[z] = psb[z - 1] + 1;
                }
                int q = j - 1;
                while (q >= 0 && hs[q] == rank - j + q) q--;
                if (q < 0) break;
                hs[q]++;
                for (int z = q + 1; z < j; z++) hs[z] = hs[z - 1] + 1;
            }
        }
        out[e] = sgn < 0 ? -r : r;
    }
    teardown(&C);
    return 0;
}
