// kernels.h -- host-side launchers of the ccb300 CUDA kernels and the small
// descriptor structs they take.  Shared by the planner/executor (C++) and the
// kernel translation units (CUDA).  No torch types anywhere.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ccb {

constexpr int kMaxDims = 8;     // dims of one tensor view
constexpr int kMaxPerms = 36;   // terms of an expanded permutation operator (3! x 3! for triples)

// Multiplication by a constant alpha, classified on the host.  alpha = +-2^k
// (|k| < 512) is applied exactly with integer operations on the exponent and
// sign bits (B300 issues FP64 instructions, conversions included, at ~1/64 of
// the FP32 rate); any other alpha is a plain FP64 multiply.
struct Scale {
    int general;                    // 1: multiply by value
    int kexp;                       // alpha = (sflip ? -1 : 1) * 2^kexp when !general
    uint32_t sflip;                 // 0x80000000 when alpha < 0
    double value;                   // alpha
};
inline Scale make_scale(double a) {
    Scale s{1, 0, 0u, a};
    if (a != 0.0 && a == a) {
        double m = a < 0 ? -a : a;
        int k = 0;
        while (m >= 2.0 && k < 512) { m *= 0.5; k++; }
        while (m < 1.0 && k > -512) { m *= 2.0; k--; }
        if (m == 1.0 && k > -512 && k < 512) { s.general = 0; s.kexp = k; s.sflip = a < 0 ? 0x80000000u : 0u; }
    }
    return s;
}

// Mixed-radix index group: a fused matrix index decomposed into nd digits
// (digit 0 outermost, digit nd-1 fastest); offset = sum digit_d * str[d].
struct Grp {
    int nd;
    int64_t ext[6];
    int64_t str[6];
};

// out[offset(idx)] = beta * out[...] + alpha * sum_p sign[p] * src[sum_d idx_d * sstr[p][d]]
// over the nd-dimensional index box ext[]; the output is visited in the
// row-major order of ext (out strides arbitrary).  Covers permutes (TTGT
// transposes), copies, and the antisymmetrising epilogues P(..).
// two_src: each term is the product src[sstr . idx] * src2[sstr2 . idx] (an
// outer product with permutation operators, formed directly in the output).
// cplx: elements are interleaved complex doubles (strides count complex
// elements); conj_a / conj_b conjugate src / src2 as they are read.
struct AccumDesc {
    int nd;
    int nperm;
    int64_t total;
    int64_t ext[kMaxDims];
    int64_t ostr[kMaxDims];
    int64_t sstr[kMaxPerms][kMaxDims];
    double sign[kMaxPerms];
    double alpha, beta;
    int two_src;
    int64_t sstr2[kMaxPerms][kMaxDims];
    int cplx, conj_a, conj_b;
    // set by launch_accum from sign/alpha/beta (the kernels never compare
    // doubles per element: those compares run on the narrow FP64 pipe)
    unsigned long long negmask;     // bit p: sign[p] < 0
    Scale as;                       // make_scale(alpha)
    int bcase;                      // beta_case(beta)
    // has_add (beta must be 1): the accumulated-onto value is add[sum idx_d * astr[d]]
    // instead of out's own (a copy "out = add" fused into the step: out = add + alpha sum ...)
    int has_add;
    int64_t astr[kMaxDims];
};

// beta classes for epilogues: 0 -> 0, 1 -> 1, other -> 2
inline int beta_case(double b) { return b == 0.0 ? 0 : b == 1.0 ? 1 : 2; }

// C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n), FP64.
// A(m,k) = A[m*sAm + k*sAk] with sAm == 1 or sAk == 1; B(k,n) = B[k*sBk + n*sBn]
// likewise; C addressed through two mixed-radix groups.
// splitk > 1: grid z = splitk slices of K; each writes its raw partial sum to
// partials[z][n][m] (m fastest) and launch_splitk_reduce applies alpha/beta.
// cplx: complex double operands and output (strides in complex elements, four
// real FMAs per complex product); conj_a / conj_b conjugate A / B.
// f32 (real only): operands rounded to FP32 as they are staged and multiplied
// and accumulated in FP32 (the SIMT FP32 rate); output FP64.
struct GemmF64Desc {
    int64_t M, N, K;
    int64_t sAm, sAk, sBk, sBn;
    Grp cm, cn;
    double alpha, beta;
    int splitk;
    int cplx, conj_a, conj_b;
    int f32;
    int bcase;                      // set by launch_gemm_f64 from beta
    Scale as;                       // make_scale(alpha), same launcher
    int red;                        // beta = 1, no split K: add C by red.global.add.f64 (no read)
};

// Narrow GEMM: C(r, c) = alpha * sum_k X(r, k) Y(k, c) + beta * C(r, c) for
// many rows r and a short side c (the rank-o updates of T3, products with T1
// and the F intermediates: shapes that tensor tiles would pad).  Every operand
// and the output are read through mixed-radix groups, so no operand is
// permuted first; one thread per row, Y staged in shared memory in chunks of
// 64 contraction indices by up to 64 columns.
// f32: products and sums in FP32 (FP64 data, one rounding per operand).
struct RowsGemmDesc {
    int64_t R;
    int nc, K;
    Grp xr, xk;     // X(r, k) = X[xr(r) + xk(k)]
    Grp yk, yc;     // Y(k, c) = Y[yk(k) + yc(c)]
    Grp cr, cc;     // C(r, c) = C[cr(r) + cc(c)]
    double alpha, beta;
    int f32;
    int bcase;                      // set by launch_rows_gemm from beta
    Scale as;                       // make_scale(alpha), same launcher
    int red;                        // beta = 1: add C by red.global.add.f64 (no read)
    int kc;                         // set by the launchers: X read with lanes along K (FP32 only)
};

// Long contraction with at most 8 columns, the large operand X read in place:
//   C(m, n) = alpha * sum_k X(m, k) Y(k, n) + beta * C(m, n),
// k = (ko, j) with j the contraction's inner run, contiguous in X (unit
// stride) and of stride sy in Y: X(m, k) = X[xm(m) + xko(ko) + j],
// Y(k, n) = Y[yko(ko) + j sy + yn(n)].  A work item is four rows and either
// seg elements of one inner run or kper whole runs (seg = L).
// f32: products and lane sums in FP32 (FP64 data), the rest in FP64.
struct NarrowKDesc {
    int64_t M;
    int N;
    int64_t Ko, L, sy, kper, seg;
    Grp xm, xko;
    Grp yko, yn;
    Grp cm, cn;
    double alpha, beta;
    int f32;
};

// Several narrow GEMMs into one output, accumulated in one pass (K
// concatenation on the narrow kernel):
//   C(r, c) += sum_s alpha_s sum_k X_s(r, k) Y_s(k, c)
// each member with its own operands and strides; the members' Y blocks sit in
// shared memory one after the other (alpha_s applied there), so each output
// element is read and written once whatever the number of members.
constexpr int kMaxRowsMembers = 8;
struct RowsMember {
    Grp xr, xk;     // X_s(r, k) = X_s[xr(r) + xk(k)]
    Grp yk, yc;     // Y_s(k, c) = Y_s[yk(k) + yc(c)]
    int K;
    double alpha;
    const double *X, *Y;            // set at launch
};
struct RowsMultiDesc {
    int64_t R;
    int nc, nm;
    Grp cr, cc;     // C(r, c) = C[cr(r) + cc(c)]
    int f32;
    int red;                        // add C by red.global.add.f64 (no read)
    RowsMember m[kMaxRowsMembers];
};
// shared memory of one block of the multi-member narrow kernel (0: too large)
int64_t rows_multi_smem_bytes(const RowsMultiDesc &d);

// Packed index pairs.  A pair (p < q) of letters with extent n has the index
// P(p, q) = p (2n - p - 1) / 2 + (q - p - 1): q runs fastest.
// pack:   dst[P1][P2] = scale * src[p s0 + q s1 + r s2 + u s3] over p < q
//         (extent n1) and r < u (extent n2), dst contiguous
// row0, rows: the launch covers packed rows [row0, row0 + rows) and writes
// them to dst[0 ..); pbase is subtracted from the first letter before its
// stride s0 (a source holding only part of that letter's range).
struct PackDesc {
    int64_t n1, n2, P1, P2;
    int64_t s0, s1, s2, s3;
    double scale;
    int64_t row0, rows, pbase;
};
// unpack: out(x) = beta * out(x) + alpha * sign * C[PA(a1, a2) cA + PB(b1, b2) cB]
// over the 4-index output box (dims in storage order, ext/ostr), where
// (a1, a2) = the digits at dims da1, da2 and (b1, b2) those at db1, db2; a
// digit pair out of order takes the swapped pair with a minus sign; equal
// digits give 0
struct UnpackDesc {
    int64_t ext[4], ostr[4];
    int da1, da2, db1, db2;
    int64_t nA, nB, cA, cB;
    double alpha, beta;
    int bcase;                      // set by launch_unpack_pairs from beta
    Scale as;                       // make_scale(alpha), same launcher
};
cudaError_t launch_pack_pairs(const PackDesc &d, const double *src, double *dst, cudaStream_t s);
// amplitude packing of a [o][o][v][v] array antisymmetric in both pairs
// (cplx: interleaved complex elements): packed[P(i,j)][P(a,b)] over i<j, a<b
cudaError_t launch_pack_t2(int o, int v, int cplx, const double *full, double *packed, cudaStream_t s);
cudaError_t launch_unpack_t2(int o, int v, int cplx, const double *packed, double *full, cudaStream_t s);
cudaError_t launch_unpack_pairs(const UnpackDesc &d, const double *C, double *out, cudaStream_t s);

// Split an FP64 strided view X(r, k) (r, k mixed-radix groups) into nplanes
// bf16 planes P_p[r][k] of a K-major matrix [Rp][Kp]:
//   hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid); rows >= R and
//   columns >= K are written as zeros.  The planner passes Rp = R: the
//   tensor-core kernels read the rows past a plane as zeros through TMA.
// Complex sources (gr, gk give complex-element offsets in doubles) enter the
// real GEMM that carries a complex product C = A B (4M, one GEMM):
//   cplx 1, stacked:  X(r, 2k + c) = component c of X(r, k)
//                     (conj: the c = 1 column negated)
//   cplx 2, embedded: X(2r + cr, 2k + ck) = s * component (cr ^ ck) of X(r, k),
//                     s = -1 for (cr, ck) = (0, 1) (conj: also for cr ^ ck = 1)
// so that [C_re; C_im] = embedded(A) stacked(B) and likewise with the roles of
// the operands swapped.  R and K count the real rows and columns.
// K concatenation (several contractions into one output, one GEMM): the
// operand fills the plane columns [kdst, kdst + kend) of rows that are Kp long
// (columns K..kend-1 with zeros; kend = 0 means the whole row, kdst = 0), each
// value multiplied by `scale` first when `scaled` (the contraction's factor).
struct SplitDesc {
    int64_t R, K, Rp, Kp;
    Grp gr, gk;
    int nplanes;
    int cplx, conj;
    int64_t kdst, kend;
    double scale;
    int scaled;
};

// Split-bf16 GEMM on tcgen05: D[m][n] = sum_{(p,q) in products} A_p[m][:] . B_q[n][:]
// (fp32 in TMEM), then C(m,n) = alpha * D + beta * C(m,n) in FP64.
// bn: N tile (64, 128 or 256; the ceil(N / bn) column tiles share N evenly);
// splitk > 1: each CTA covers one slice of the K blocks and stores its raw
// fp32 tile (as double) to partials[z][n][m].
struct TcGemmDesc {
    int64_t M, N, Mp, Np, Kp;
    int nplanes_a, nplanes_b;
    int nprod;                 // number of (p,q) products
    int prod_a[8], prod_b[8];  // plane indices of each product
    Grp cm, cn;
    double alpha, beta;
    int bn;
    int splitk;
    int bcase;                      // set by launch_tc_gemm from beta
    Scale as;                       // make_scale(alpha), same launcher
    int red;                        // beta = 1, no split K: add the tile with red.global.add.f64
};

cudaError_t launch_accum(const AccumDesc &d, const double *src, double *out, cudaStream_t s,
                         const double *src2 = nullptr, const double *add = nullptr);
cudaError_t launch_zero(double *p, int64_t n, cudaStream_t s);
cudaError_t launch_gemm_f64(const GemmF64Desc &d, const double *A, const double *B, double *C, double *partials,
                            cudaStream_t s);
// C(m,n) = alpha * sum_z partials[z][n][m] + beta * C(m,n) (fixed summation order)
cudaError_t launch_splitk_reduce(int64_t M, int64_t N, int splitk, const double *partials, const Grp &cm, const Grp &cn,
                                 double alpha, double beta, double *C, cudaStream_t s);
cudaError_t launch_rows_gemm(const RowsGemmDesc &d, const double *X, const double *Y, double *C, cudaStream_t s);
cudaError_t launch_rows_multi(const RowsMultiDesc &d, double *C, cudaStream_t s);
cudaError_t launch_narrow_k(const NarrowKDesc &d, const double *X, const double *Y, double *C, cudaStream_t s);
// C(m,n) *= beta over an M x N output addressed by two mixed-radix groups
cudaError_t launch_scale_grp(int64_t M, int64_t N, const Grp &cm, const Grp &cn, double beta, double *C, cudaStream_t s);
// the split kernels' double -> float rounding (mine) next to the library's (ref)
cudaError_t launch_convert_selftest(const double *in, int64_t n, float *mine, float *ref, cudaStream_t s);
// 1/D for rank 1..3 amplitude arrays (complex: the same value on both parts)
cudaError_t launch_inv_denominators(int rank, int o, int v, const double *fo, const double *fv, double *out, int cplx,
                                    cudaStream_t s);
// Jacobi step with precomputed 1/D over n doubles: e = r * dinv, x' = t + e
cudaError_t launch_jacobi_inv(int64_t n, const double *t, const double *r, const double *dinv, double *xo, double *eo,
                              cudaStream_t s);
// one CTA whose mbarrier wait is never satisfied: *timed_out = 1 after budget_cycles
cudaError_t launch_wait_selftest(long long budget_cycles, int *timed_out, cudaStream_t s);
cudaError_t launch_split_bf16(const SplitDesc &d, const double *x, void *planes, cudaStream_t s);
cudaError_t launch_tc_gemm(const TcGemmDesc &d, const void *Aplanes, const void *Bplanes, double *C,
                           double *partials, int *err_flag, cudaStream_t s);

// ---- grouped execution: one plan step over a batch of systems whose plans
// have the same steps (a launch covers every system; entries of systems whose
// active[sys] is 0 are skipped).  Each entry's work items follow those of the
// entries before it (item0 / tile0: the entry's first item in the launch).
struct alignas(64) TmapBytes {
    unsigned char b[128];           // a CUtensorMap, encoded on the host
};
struct GroupedSplit {               // one operand split of one system (real, bf16 planes)
    SplitDesc d;
    const double *x;
    void *planes;
    int64_t tile0;
    uint32_t rtiles;                // tiled splits: row tiles; long contiguous K: 1 = vector loads
    int sys;
};
struct alignas(64) GroupedGemm {    // one system's split-bf16 GEMM (accumulating or assigning)
    TmapBytes ma, mbw, mbn;         // A planes; B planes at the wide / narrow column tile
    int64_t M, N, Kp;
    int n_tiles, cs_base, cs_extra; // column tiles and their even split (16-column units)
    Grp cm, cn;
    Scale as;
    int bcase;                      // 0 store, 1 read-modify-write, 2 reductions
    double *C;
    int nslices, kb_per;            // K slices (> 1: raw slice sums to P[z][n][m], reduced after)
    double *P;
    int64_t tile0;
    int sys;
};
// K slices of a grouped GEMM whose entries have fewer than 2 x 148 output
// tiles in all (tiles_all): long contractions with small outputs are cut into
// slices of about 32 K blocks of 64 (partials of at most 16 MB)
inline int grouped_kslices(int64_t M, int64_t N, int64_t Kp, int64_t tiles_all) {
    const int64_t kb = Kp / 64;
    if (kb <= 48 || tiles_all >= 2 * 148) return 1;
    int64_t ns = (kb + 31) / 32;
    if (ns > 64) ns = 64;
    const int64_t cap = ((int64_t)16 << 20) / (M * N * 8 > 0 ? M * N * 8 : 1);
    if (ns > cap) ns = cap;
    return ns < 2 ? 1 : (int)ns;
}
struct GroupedRows {                // one system's narrow GEMM (bcase / as prepared)
    RowsGemmDesc d;
    const double *X, *Y;
    double *C;
    int64_t item0;
    int sys;
};
void prepare_grouped_rows(GroupedRows &g);
int grouped_rows_nc(int nc_max);                       // the column chunk of a launch
int64_t grouped_rows_items(const GroupedRows &g, int nc);
cudaError_t launch_grouped_rows(const GroupedRows *tab, int n, int64_t total, int nc, bool f32, const int *active,
                                cudaStream_t s);
// one-column narrow GEMMs (GEMVs) of a batch: warps over rows, lanes along K
constexpr int kGemvKmax = 2048;                 // longest K (staged in shared memory)
bool grouped_gemv_ok(const GroupedRows &g);     // prepared entry: nc = 1, K <= kGemvKmax, 32-bit X offsets
int64_t grouped_gemv_items(const GroupedRows &g);
// the same with X running along the rows and a long K: lanes along rows, K over the block's warps
bool grouped_gemvr_ok(const GroupedRows &g);
int64_t grouped_gemvr_items(const GroupedRows &g);
cudaError_t launch_grouped_gemvr(const GroupedRows *tab, int n, int64_t total, bool f32, const int *active,
                                 cudaStream_t s);
cudaError_t launch_grouped_gemv(const GroupedRows *tab, int n, int64_t total, bool f32, const int *active,
                                cudaStream_t s);
struct GroupedReduce {              // C = alpha sum_z P[z][n][m] + beta C of one sliced GEMM
    int64_t M, N;
    int nslices;
    const double *P;
    Grp cm, cn;
    Scale as;
    int bcase;
    double *C;
    int64_t item0;
    int sys;
};
struct GroupedGemmParams {          // what every entry of a grouped GEMM shares
    int nprod;
    int prod_a[8], prod_b[8];
};
struct GroupedAccum {               // one system's elementwise step
    AccumDesc d;                    // prepared (prepare_grouped_accum): dims merged, negmask / as / bcase set
    const double *src, *src2, *add;
    double *out;
    int row_path;                   // the row path applies (rows of the innermost dim, stride 0 / 1)
    uint32_t rows, ncb;             // row path: rows, column blocks
    int rch;                        // row path: rows per work item
    int64_t item0;
    int sys;
};
// An elementwise step of one system in compact form (grouped launches): at
// most kEwDims dims and kEwTerms terms, every offset below 2^31, so a lane keeps
// 32-bit running offsets and steps them instead of decomposing each element.
constexpr int kEwDims = 4;
constexpr int kEwTerms = 4;
struct GroupedEw {
    int nd, nterms, has_add;
    uint32_t total;                 // output elements
    unsigned long long negmask;     // bit p: term p subtracts
    Scale as;                       // alpha
    int ext[kEwDims];
    int ostr[kEwDims], astr[kEwDims];
    int sstr[kEwTerms][kEwDims], sstr2[kEwTerms][kEwDims];
    // the offset change when digit k wraps into digit k - 1 (str[k-1] - ext[k] str[k], k >= 1),
    // and at k = 0 the change of a 32-element step of the innermost digit (32 str[nd-1])
    int wo[kEwDims], wa[kEwDims], ws[kEwTerms][kEwDims], ws2[kEwTerms][kEwDims];
    const double *src, *src2, *add;
    double *out;
    int64_t item0;
    int sys;
};
constexpr int64_t kEwRun = 256;     // output elements per work item (a warp's run)
// the compact form of a prepared entry; false when it does not fit
bool grouped_ew_from(const GroupedAccum &g, GroupedEw &e);
cudaError_t launch_grouped_ew(const GroupedEw *tab, int n, int64_t total, bool acc, int nperm, bool two,
                              const int *active, cudaStream_t s);
// the denominator update of the residuals (R -= D T, real) and the
// partial sums of the energy and of |R1|^2, |R2|^2 of one system
struct GroupedPost {
    int o, v;
    const double *fo, *fv, *t1, *t2, *oovv;
    double *r1, *r2;
    double *partials;               // [3][chunks]: energy, |R1|^2, |R2|^2 per chunk
    double *scal;                   // scal[0] = E, scal[1] = 0, scal[2] = |R1|^2, scal[3] = |R2|^2
    int64_t item0, chunks;
    int sys;
};
constexpr int64_t kPostChunk = 4096;    // elements of (R1 | R2) per post work item

// host: an entry of a grouped GEMM from a planned TcGemmDesc (two planes,
// no split K) at column tile width bn; false when a map cannot be encoded
bool grouped_gemm_entry(GroupedGemm &g, const TcGemmDesc &d, const void *A, const void *B, double *C, int bn,
                        int nslices, double *P);
// host: the split kernel's lane orientation for a descriptor (lanes along K)
bool split_lanes_along_k(const SplitDesc &d);
void prepare_grouped_accum(GroupedAccum &g);
// work items of an entry: mode 0 generic (runs of 256), 1 row path, 2 generic
// with four elements' loads in flight per lane (runs of 128; one or two terms)
int64_t grouped_accum_items(const GroupedAccum &g, int mode);
// the launches: tab (device) holds n entries; total = the work items of all
// long contiguous-K splits of a batch (vector loads, warps over (row, span) items)
// 0: not this path; 1: scalar loads; 2: vector loads
int grouped_split_vec_ok(const SplitDesc &d, const double *x);
int64_t grouped_split_vec_items(const SplitDesc &d);
cudaError_t launch_grouped_split_vec(const GroupedSplit *tab, int n, int64_t total, const int *active,
                                     cudaStream_t s);
cudaError_t launch_grouped_split(const GroupedSplit *tab, int n, int64_t total, bool lk, const int *active,
                                 cudaStream_t s);
cudaError_t launch_grouped_gemm(const GroupedGemm *tab, int n, int64_t total, int bn, const GroupedGemmParams &p,
                                const int *active, int *err_flag, cudaStream_t s);
cudaError_t launch_grouped_accum(const GroupedAccum *tab, int n, int64_t total, bool acc, int mode, int nperm,
                                 bool two, const int *active, cudaStream_t s);
cudaError_t launch_grouped_post(const GroupedPost *tab, int n, int64_t total, const int *active, cudaStream_t s);
cudaError_t launch_grouped_reduce(const GroupedReduce *tab, int n, int64_t total, const int *active, cudaStream_t s);

// R -= D * T for rank 1..3 residuals: D from the orbital energies (real);
// cplx: t and r are interleaved complex.
cudaError_t launch_denom_sub(int rank, int o, int v, const double *fo, const double *fv,
                             const double *t, double *r, int cplx, cudaStream_t s);
// y = a*x + b*y over n elements
cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s);
// partial sums for dot products: partials[b] = sum over block b of x*y (fixed grid)
constexpr int kRedBlocks = 592;
// Jacobi step over the concatenated amplitude vector (up to three rank
// segments of seg_n[l] doubles: t[l], r[l]) fused with the DIIS overlaps of the
// new error vector: e = r * dinv, x' = t + e written to xo / eo (contiguous),
// and partials[h][block] of <e, he[h]> for h < m (he[h] == eo: the new vector
// itself).  Fixed grid and order: deterministic.
struct JacobiSegs {
    int nseg;
    int64_t n[3];
    const double *t[3];
    const double *r[3];
    const double *he[16];
    int m;
};
cudaError_t launch_jacobi_dots(const JacobiSegs &g, const double *dinv, double *xo, double *eo, double *partials,
                               cudaStream_t s);
cudaError_t launch_dot_partials(const double *x, const double *y, int64_t n, double *partials,
                                cudaStream_t s);
// energy partials: sum_ijab V[ijab] (1/4 t2[ijab] + 1/2 t1[ia] t1[jb]); t1 may be NULL.
// cplx: complex inputs; two partial rows (real part, then imaginary part).
cudaError_t launch_energy_partials(int o, int v, const double *Voovv, const double *t1,
                                   const double *t2, double *partials, int cplx, cudaStream_t s);
// out[k] = sum of partials[k][0..kRedBlocks) for k < count (fixed order)
cudaError_t launch_reduce_partials(const double *partials, int count, double *out, cudaStream_t s);
// DIIS on device.  gram16[16*16] holds <e_a|e_b> by history slot; order_host
// lists the m stored slots oldest first.  Writes coef (for the newest
// status[0] vectors) and status[0] = vectors used (0: no usable solve).
cudaError_t launch_diis_solve(const double *gram16, const int *order_host, int m, double *coef, int *status,
                              cudaStream_t s);
// reduce `count` partial rows into gram16 at the symmetric pairs (a_k, b_k)
cudaError_t launch_gram_scatter(const double *partials, int count, const int *a_host, const int *b_host,
                                double *gram16, cudaStream_t s);
// x = sum_k c_k xs[m - used + k] over n elements (used read from used_dev);
// xs_host: host array of m device pointers, oldest first.
cudaError_t launch_combine(const double *const *xs_host, const double *coef, const int *used_dev, int m, int64_t n,
                           double *x, cudaStream_t s);

// ---- batched Jacobi + DIIS (many independent systems, one launch per kernel)
// One system of a batched iteration; the host rewrites the table every
// iteration (one copy) and the four kernels below read it on the device.
constexpr int kBatchBlocks = 64;    // blocks per system of the batched kernels
struct BatchSys {
    int active;                // 0: converged or stopped (the kernels skip it)
    int o, v, cplx;
    const double *fo, *fv;
    double *t[4], *r[4];       // amplitudes and residuals by rank (NULL: absent)
    int64_t n[4];              // doubles per rank
    int64_t nx;                // doubles of x (the ranks concatenated)
    double *hx, *he;           // DIIS history (x', e) slots of nx doubles
    int slot;                  // the slot this iteration's Jacobi step writes
    int nstored;               // stored slots after this step (order[] oldest first)
    int order[16];
    double *gram;              // [16][16] by slot
    double *coef;              // [16]
    int *used;                 // newest vectors the DIIS solve used (0: none)
    double *partials;          // [16][kBatchBlocks]
    const double *dinv;        // 1/D of every amplitude, concatenated like x (set once per solve)
};
// x'_slot = t + R (1/D), e_slot = R (1/D) for every active system
cudaError_t launch_batched_jacobi(const BatchSys *sys, int nsys, cudaStream_t s);
// <e_slot | e_order[q]> for q < nstored, reduced into gram; the DIIS solve when
// nstored >= 2 (coef, used); deterministic fixed-grid reductions
cudaError_t launch_batched_diis(const BatchSys *sys, int nsys, cudaStream_t s);
// t = sum_k coef_k x'_order[nstored-used+k] (used == 0: the newest x'), or the
// new x' when fewer than two are stored
cudaError_t launch_batched_combine(const BatchSys *sys, int nsys, cudaStream_t s);

}  // namespace ccb
