/*
 * cc.h -- C ABI of ccb300: the coupled-cluster amplitude residual, energy and
 * Jacobi+DIIS iteration on one NVIDIA B300 (sm_103a).
 *
 * The method (arxiv 2409.06759, "Generating coupled cluster code for modern
 * distributed memory tensor software"):
 *   * Sec. II A, Eq. amp: the CC equations <Phi_l| exp(-T) H_N exp(T) |Phi_0> = 0
 *     and the energy <Phi_0| exp(-T) H_N exp(T) |Phi_0> = E - E_HF, with
 *     T1 = sum t_i^a a+_a a_i and T2 = 1/4 sum t_ij^ab a+_a a+_b a_j a_i
 *     (amplitudes stored unpacked and fully antisymmetric);
 *   * Sec. II C: the residual is evaluated as an ordered list of binary tensor
 *     contractions ("Contraction" objects: a factor, permutation operators, at
 *     most two tensors, an output), written in text as
 *       OUT[idx] (=|+=|-=) factor P(..) A[idx] * B[idx]
 *     and executed transpose-transpose-GEMM-transpose (TTGT, Sec. I C);
 *   * Sec. III B, Eq. ham2q: the Hamiltonian with antisymmetrised integrals
 *     <pq||rs>; i,j,k,l (and m,n) are occupied, a..h are virtual (Sec. II A).
 *
 * Conventions shared by every call:
 *   * All tensors are caller-owned DEVICE memory, row-major, in the orders
 *     given below.  The library never frees them.  Scratch comes from the
 *     caller's workspace argument; the hot path allocates no device memory.
 *   * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and return without synchronising,
 *     except cc_solve, which reads |R| back to the host once per iteration.
 *   * Errors: every call returns a cc_status and never aborts.  On error the
 *     outputs are unspecified, the inputs are untouched, and cc_last_error()
 *     returns a message (thread-local, valid until the next call).
 *   * dtype CC_F64: double.  CC_C128: interleaved complex double (re, im)
 *     for every tensor (integral blocks, amplitudes, residuals); orbital
 *     energies stay real.  Complex integrals are Hermitian,
 *     <pq||rs> = conj(<rs||pq>); a list names each integral in the
 *     orientation the projection fixes (the doubles driver is <ab||ij>).
 */
#ifndef CCB300_CC_H
#define CCB300_CC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CC_API __attribute__((visibility("default")))
#else
#define CC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CC_OK = 0,
    CC_ERR_INVALID_ARG = 1,   /* NULL pointer, bad size or option */
    CC_ERR_PARSE = 2,         /* contraction text does not parse */
    CC_ERR_SHAPE = 3,         /* index spaces / extents inconsistent */
    CC_ERR_UNSUPPORTED = 4,   /* valid request this build does not implement */
    CC_ERR_OOM = 5,           /* host allocation failed */
    CC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    CC_ERR_NOT_CONVERGED = 7, /* cc_solve: maxiter reached or divergence */
    CC_ERR_TIMEOUT = 8,       /* a bounded device wait expired */
    CC_ERR_WORKSPACE = 9      /* workspace too small or misaligned */
} cc_status;

typedef enum { CC_F64 = 0, CC_C128 = 1 } cc_dtype;

/* Arithmetic of the bulk contractions (those of at least 2e8 flops; smaller
 * ones run in FP32 on CC_PREC_BF16X3 plans and in FP64 on the others).
 *   CC_PREC_FP64:   every GEMM in FP64 (SIMT DFMA).
 *   CC_PREC_BF16X3: each FP64 operand split into bf16 hi + lo planes, products
 *                   hi*hi + hi*lo + lo*hi on tcgen05 tensor cores with FP32
 *                   accumulation in TMEM, recombined into FP64 outputs.
 *   CC_PREC_BF16X6: three planes (hi, mid, lo), six products, accumulators
 *                   drained into float-float registers every 128 K.
 *   CC_PREC_SLICES: FP64-grade: every operand row scaled by a power of two and
 *                   cut into six exact 7-bit bf16 slices; the 21 slice
 *                   products of weight <= 5 summed exactly in FP32 over
 *                   128-long K chunks and drained into float-float registers
 *                   (error ~2^-40 of K max|A row| max|B column|).  Meant as
 *                   the refine plan of cc_solve. */
typedef enum { CC_PREC_FP64 = 0, CC_PREC_BF16X3 = 2, CC_PREC_BF16X6 = 3, CC_PREC_SLICES = 4 } cc_precision;

typedef struct cc_plan_s *cc_plan;

/* Antisymmetrised integrals <pq||rs> (Eq. ham2q) in six canonical blocks, each
 * dense [p][q][r][s] with the spaces in its name (o = occupied, v = virtual),
 * every element stored (no permutational packing).  Any other space pattern
 * is read from these through <pq||rs> = -<qp||rs> = -<pq||sr> and
 * <rs||pq> = conj(<pq||rs>).  f_occ[o], f_vir[v]: the diagonal Fock matrix
 * (orbital energies, always double). */
typedef struct {
    const double *f_occ;
    const double *f_vir;
    const void *oooo;   /* [o][o][o][o] */
    const void *ooov;   /* [o][o][o][v] */
    const void *oovv;   /* [o][o][v][v] */
    const void *ovov;   /* [o][v][o][v] */
    const void *ovvv;   /* [o][v][v][v] */
    const void *vvvv;   /* [v][v][v][v] */
    /* optional: <ab||ef> for a < b, e < f as a dense [P(a,b)][P(e,f)] matrix,
     * P(p,q) = p (2v - p - 1)/2 + (q - p - 1) (a quarter of vvvv; real only).
     * Read instead of vvvv by plans created with packed_vvvv = 1. */
    const void *vvvv_packed;
} cc_integrals;

/* Cluster amplitudes: t1[i][a], t2[i][j][a][b], t3[i][j][k][a][b][c] (NULL when
 * the plan has no triples).  Antisymmetric in occupied and in virtual indices. */
typedef struct {
    void *t1;
    void *t2;
    void *t3;
} cc_amps;

/* Residuals R = <Phi_l|Hbar|Phi_0>, same layouts as the amplitudes. */
typedef struct {
    void *r1;
    void *r2;
    void *r3;
} cc_resid;

typedef struct {
    int struct_size;      /* sizeof(cc_plan_opts) */
    int verbose;          /* 1: print the plan to stderr at creation */
    int fuse_permutes;    /* reserved, 0 */
    int packed_vvvv;      /* 1: a packed-pair contraction over <ab||ef> in its stored
                           * orientation (declared (ab)(ef)) reads ints->vvvv_packed */
    int no_kconcat;       /* 1: plan every statement on its own.  By default, on the
                           * split-bf16 precisions (real), statements that accumulate
                           * into the same intermediate with its indices split the same
                           * way between their operands run as one tensor-core GEMM
                           * whose K concatenates theirs (one pass over the output) */
    int uniform_steps;    /* 1 (split-bf16 precisions, real): every contraction on the
                           * tensor-core split route and none merged, so that plans of
                           * one list have the same steps at any o, v.  cc_solve_batched
                           * then runs the batch step by step, one launch per step for
                           * all systems (grouped execution) */
} cc_plan_opts;

/* cc_plan_create -- parse a contraction list and plan its execution.
 * Defined by: Sec. II C (the residual as an ordered list of binary
 * "Contraction" objects, their text form in Fig. representations) and
 * Sec. I C (each contraction executed transpose-transpose-GEMM-transpose).
 *   text: one statement per line, '#' starts a comment:
 *       OUT[idx]..  (=|+=|-=)  [factor] [P(pq)|P(p/qr)]...  A[idx].. [* B[idx]..]
 *     Index letters i..n (or h1, h2, ...) are occupied, a..h (or p1, p2, ...)
 *     virtual.  Reserved tensors: T1 T2 T3 (amplitudes; occupied indices are
 *     matched to the occupied slots and virtual to the virtual slots, so
 *     t[ab][ij] and T2[ijab] name the same tensor), R1 R2 R3 (residual
 *     outputs, same rule), V (integrals, <pq||rs> = V[pq][rs]).  Any other name
 *     is an intermediate; its first statement must be '=' and fixes its index
 *     order (storage order).  P(pq) = 1 - (p<->q); P(p/qr) = 1 - (p<->q) - (p<->r).
 *     The list must not contain the diagonal Fock terms: cc_residual adds
 *     -D*t itself (D_i^a = f_ii - f_aa, D_ij^ab = f_ii + f_jj - f_aa - f_bb).
 *   o, v: occupied / virtual extents (>= 1).
 *   opts: NULL for defaults.
 *   out: receives the plan (host object; creating it touches no GPU).
 * Errors: CC_ERR_PARSE / CC_ERR_SHAPE with the line number in cc_last_error(). */
CC_API cc_status cc_plan_create(const char *text, int o, int v, cc_dtype dtype, cc_precision precision,
                                const cc_plan_opts *opts, cc_plan *out);

/* Device workspace that cc_residual needs (bytes, 256-byte aligned base). */
CC_API cc_status cc_plan_workspace_bytes(cc_plan plan, size_t *bytes);

/* Writes a JSON description of the planned steps (permutes, GEMMs with
 * M,N,K and flops, epilogues) into buf (NUL-terminated, truncated at len);
 * *needed receives the full length + 1.  Host only. */
CC_API cc_status cc_plan_describe(cc_plan plan, char *buf, size_t len, size_t *needed);

/* Total dense GEMM flops of one residual evaluation (2*M*N*K summed). */
CC_API cc_status cc_plan_flops(cc_plan plan, double *flops);

CC_API cc_status cc_plan_destroy(cc_plan plan);

/* Per-step timing with CUDA events recorded on each call's stream (off by
 * default).  enable = 1 creates the events (a host call: make it before any
 * timed region) and clears the totals; 0 stops recording.  When a refine plan
 * runs inside cc_solve, its own profile records its steps. */
CC_API cc_status cc_plan_profile_enable(cc_plan plan, int enable);

/* Accumulated device milliseconds per plan step (the order of
 * cc_plan_describe's steps) over `calls` residual evaluations since enabling.
 * ms_kernel[k] is the GEMM kernel alone (the split kernels of a split-bf16
 * step excluded), or the whole step for permutes and epilogues.  Waits for the
 * events of the last evaluation.  Arrays may be NULL; cap bounds the writes. */
CC_API cc_status cc_plan_profile_read(cc_plan plan, double *ms_step, double *ms_kernel, int cap, int *nsteps,
                                      int *calls);

/* Number of kernels launched so far by calls on this plan (residual steps,
 * operand splits, epilogues, and in cc_solve the iteration kernels). */
CC_API cc_status cc_plan_launch_count(cc_plan plan, long long *count);

/* cc_residual -- evaluate R1, R2 (, R3) for the given amplitudes.
 * Defined by: Sec. II A, Eq. amp (R_l = <Phi_l| exp(-T) H_N exp(T) |Phi_0>,
 * projected on singles, doubles and triples), with H_N of Eq. ham2q.
 *   ints, amps: inputs (device, unchanged).  res: outputs (device), fully
 *   overwritten.  ws: device workspace of at least cc_plan_workspace_bytes.
 * Ownership: nothing is retained after the call returns. */
CC_API cc_status cc_residual(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, cc_resid *res,
                             void *ws, size_t ws_bytes, void *stream);

/* cc_plan_autotune -- picks, for every contraction of the plan, the GEMM
 * configuration (tensor-core tile width 64/128/256, split-K factor and, for
 * an accumulating contraction, read-modify-write or reduction epilogue on the
 * split-bf16 route; split-K factor on the FP64/FP32 tiled route) that runs
 * fastest on this device for these inputs: each candidate the plan prepared
 * room for is timed reps times (CUDA events, minimum taken) in place of the
 * planned one, the steps running in list order so every operand is real.
 * Results stay in the plan (cc_plan_describe reports "tuned") and in a
 * process-wide cache keyed by the contraction's route, shape (M, N, K), product
 * count, arithmetic, dtype, beta and candidate set: a contraction of that key
 * in any later autotuned plan (e.g. a same-sized system of a batch) takes the
 * stored pick without timing.  The paper has no counterpart (its contractions
 * run in ExaTENSOR).
 *   ints, amps, ws: as for cc_residual.  res: receives unspecified values.
 *   reps: 1..100 timings per candidate.  Synchronises the stream. */
CC_API cc_status cc_plan_autotune(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, cc_resid *res,
                                  void *ws, size_t ws_bytes, void *stream, int reps);

/* cc_autotune_cache -- the process-wide tuning cache of cc_plan_autotune:
 * clear = 1 empties it; *entries / *hits (either may be NULL) receive its size
 * and the number of contractions served from it since the last clear.  Host
 * only; thread-safe. */
CC_API cc_status cc_autotune_cache(int clear, long long *entries, long long *hits);

/* cc_plan_set_gemm_config -- sets the configuration of one contraction step
 * (the steps of cc_plan_describe, 0-based) to one of its autotuning
 * candidates, e.g. to replay a configuration chosen by cc_plan_autotune.
 *   bn: tensor-core tile width (64, 128, 256; 0 on the FP64/FP32 route);
 *   splitk: split-K factor; red: 1 = epilogue by red.global.add.f64 (only
 *   for accumulating contractions without split K), else 0.
 * Returns CC_ERR_INVALID_ARG when the step has no such candidate. */
CC_API cc_status cc_plan_set_gemm_config(cc_plan plan, int step, int bn, int splitk, int red);

/* cc_energy -- E_CC - E_ref = 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b
 * (f_ia = 0).  Defined by: Sec. II A, Eq. amp (the Phi_0 projection of
 * exp(-T) H_N exp(T)).  e_dev: device double[2] receiving (Re E, Im E) (Im E = 0 for
 * CC_F64).  Uses the first 10 KiB of ws as scratch. */
CC_API cc_status cc_energy(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, double *e_dev,
                           void *ws, size_t ws_bytes, void *stream);

typedef struct {
    int struct_size;          /* sizeof(cc_solve_opts) */
    int max_iter;             /* iterations of this call (default 100) */
    double tol;               /* stop when |R|_2 < tol (default 1e-8); 0 = never */
    int diis_max;             /* stored vectors (default 8, 0 = plain Jacobi) */
    int resume;               /* 1: continue the DIIS history kept in ws */
    cc_plan refine_plan;      /* optional FP64 plan used after the switch */
    double switch_tol;        /* switch to refine_plan when |R| < switch_tol */
    int verbose;              /* 1: one line per iteration on stderr */
} cc_solve_opts;

typedef struct {
    int iterations;           /* iterations done by this call */
    int converged;            /* 1 when |R| < tol */
    int switched_at;          /* iteration index of the switch to refine_plan, -1 if none */
    double energy;            /* Re E(x_k) of the last evaluated iterate */
    double rnorm;             /* |R(x_k)|_2 of the last evaluated iterate */
    double *energies;         /* optional host array [max_iter] (NULL = skip) */
    double *rnorms;           /* optional host array [max_iter] (NULL = skip) */
    double energy_im;         /* Im E(x_k) (0 for CC_F64) */
    double *energies_im;      /* optional host array [max_iter] of Im E (NULL = skip) */
} cc_solve_report;

/* Workspace of cc_solve: cc_plan_workspace_bytes plus the DIIS history and
 * residual buffers (and the refine plan's workspace when given). */
CC_API cc_status cc_solve_workspace_bytes(cc_plan plan, const cc_solve_opts *opts, size_t *bytes);

/* cc_solve -- Jacobi + DIIS on x = (t1, t2[, t3]).  Solves the equations of
 * Sec. II A, Eq. amp; the paper leaves the iteration to DIRAC-ExaCorr and
 * reports only "the norm of the residual vector" (Tables h2o/lih), so the
 * Jacobi + Pulay DIIS reading below is this library's.  Iteration k evaluates
 * R_k = R(x_k), E_k = E(x_k) and |R_k|_2 (Frobenius norm over the full stored
 * residual arrays) and stops when |R_k| < tol; otherwise x'_{k+1} = x_k + R_k/D,
 * e_k = R_k/D, the last diis_max pairs (x', e) are kept and, once two are
 * stored, x_{k+1} = sum_l c_l x'_l with [B 1; 1^T 0][c; lambda] = [0; 1],
 * B_kl = Re<e_k|e_l> (complex vectors as real ones of twice the length),
 * solved in FP64 on the device (B scaled by 1/max diag, partial pivoting, the
 * oldest vector dropped while a pivot is below 1e-14).
 *   amps: in = start (zeros give MP2 at k = 1); out = the converged x_k, or,
 *   when max_iter ends the call, the next iterate x_{k+1} (resume = 1 continues
 *   from it with the DIIS history and the static integral caches kept in ws:
 *   resume only with the same integrals, plan and ws).
 * With refine_plan (an FP64 plan of the same system), iterations run on `plan`
 * until |R| < max(switch_tol, tol) or |R| stops improving for two iterations;
 * then the DIIS history restarts and the iteration turns defect-corrected: an
 * outer step evaluates R64(x) with refine_plan (convergence is judged on this
 * FP64 residual only) and Rp(x) with plan, keeping delta = R64 - Rp; up to four
 * inner steps use Rp(x) + delta, and a new outer step starts once the
 * corrected |R| drops below 0.02 |R64|.
 * Returns CC_OK when converged, CC_ERR_NOT_CONVERGED when max_iter is reached
 * or |R| stops being finite or grows 1e3 times above its best value. */
CC_API cc_status cc_solve(cc_plan plan, const cc_integrals *ints, cc_amps *amps, const cc_solve_opts *opts,
                          cc_solve_report *report, void *ws, size_t ws_bytes, void *stream);

/* cc_solve_batched -- Jacobi + DIIS on n independent systems at once (their
 * own plans, integrals and amplitudes; sizes may differ).  Iteration 0 runs
 * each system's residual directly (filling the static caches); later
 * iterations replay one CUDA graph holding every system's residual, energy and
 * norm as independent branches, then four batched kernels (Jacobi, Gram row,
 * DIIS solve, combine) update all systems that are still iterating, driven by
 * a per-system table the host rewrites each iteration.  The per-system
 * arithmetic and stopping rule are those of cc_solve (converged systems stop
 * updating; their residuals are still evaluated by the graph).
 * Grouped execution: when the n >= 2 plans have the same steps (made with
 * cc_plan_opts.uniform_steps at CC_PREC_BF16X3 from one list writing R1 and
 * R2), the residuals of the whole batch run as one launch per step instead --
 * each step's elementwise pass, operand splits and tensor-core GEMM take a
 * table with one entry per system (the GEMM is one persistent tcgen05 kernel
 * walking the tiles of every system), then one grouped pass applies the
 * denominators and forms every system's energy and norms.  Converged systems
 * are skipped inside those launches.  The workspace size accounts for the
 * tables.
 *   plans: n distinct plans (one per system), each writing R2.
 *   ints, amps: arrays of n structs; amps in = start, out = final iterates.
 *   opts: shared options (refine_plan and resume are not supported: CC_ERR_UNSUPPORTED).
 *   reports: NULL or n reports (their optional arrays as in cc_solve).
 *   ws: cc_solve_batched_workspace_bytes bytes, 256-byte aligned.
 * Returns CC_OK when every system converged, CC_ERR_NOT_CONVERGED otherwise
 * (the message counts them). */
CC_API cc_status cc_solve_batched_workspace_bytes(int n, const cc_plan *plans, const cc_solve_opts *opts,
                                                  size_t *bytes);
CC_API cc_status cc_solve_batched(int n, const cc_plan *plans, const cc_integrals *ints, cc_amps *amps,
                                  const cc_solve_opts *opts, cc_solve_report *reports, void *ws, size_t ws_bytes,
                                  void *stream);

/* Integral construction (setup step; the antisymmetrised integrals of Eq.
 * ham2q, Sec. III B):  (pq|rs) = sum_L B[L][p][q] B[L][r][s]
 * and <pq||rs> = (pr|qs) - (ps|qr) for the six canonical blocks (Eq. ham2q).
 *   B: device [L][n][n] (n = o + v, occupied first), double or complex
 *   double (dtype); complex B gives <pq||rs> = sum_L B_pr B_qs - B_ps B_qr
 *   with no conjugation (B[L][q][p] = conj(B[L][p][q]) makes them Hermitian).
 *   blocks: device outputs (NULL skips a block), sizes from
 *   cc_integral_block_elems (elements).
 *   ws: device workspace of cc_build_integrals_workspace_bytes. */
CC_API cc_status cc_integral_block_elems(int o, int v, size_t elems[6]);
/* The packed <ab||ef> block (cc_integrals.vvvv_packed) from B, built in chunks
 * of a so that the full vvvv block is never held (real only: CC_F64).
 *   out: device, (v(v-1)/2)^2 doubles.  ws: cc_build_vvvv_packed_workspace_bytes. */
CC_API cc_status cc_build_vvvv_packed_workspace_bytes(int o, int v, int L, cc_dtype dtype, size_t *bytes);
CC_API cc_status cc_build_vvvv_packed(int o, int v, int L, cc_dtype dtype, const void *B, void *out, void *ws,
                                      size_t ws_bytes, void *stream);
CC_API cc_status cc_build_integrals_workspace_bytes(int o, int v, int L, cc_dtype dtype, size_t *bytes);
CC_API cc_status cc_build_integrals(int o, int v, int L, cc_dtype dtype, const void *B, void *oooo, void *ooov,
                                    void *oovv, void *ovov, void *ovvv, void *vvvv, void *ws, size_t ws_bytes,
                                    void *stream);

/* cc_pack_t2 / cc_unpack_t2 -- the doubles amplitudes t_ij^ab are
 * antisymmetric in (i, j) and in (a, b) (Eq. amp), so their unique content is
 * the i < j, a < b quarter.  Packed layout: t_packed[P(i,j)][P(a,b)] with the
 * pair index P(p, q) = p (2n - p - 1) / 2 + (q - p - 1) (q fastest; n = o for
 * (i, j), v for (a, b)), cc_packed_t2_elems(o, v) elements.  Moving amplitudes
 * between host and device in this form carries a quarter of the bytes.
 *   pack:   t_full (device, o*o*v*v, [i][j][a][b]) -> t_packed (device); reads
 *           only the i < j, a < b elements.
 *   unpack: t_packed -> t_full, writing every element (sign-flipped orbit
 *           members, exact zeros on i = j or a = b).
 * Elements are doubles (CC_F64) or interleaved complex doubles (CC_C128).
 * Asynchronous on stream; no workspace. */
CC_API int64_t cc_packed_t2_elems(int o, int v);
CC_API cc_status cc_pack_t2(int o, int v, cc_dtype dtype, const void *t_full, void *t_packed, void *stream);
CC_API cc_status cc_unpack_t2(int o, int v, cc_dtype dtype, const void *t_packed, void *t_full, void *stream);

/* cc_energy_noalloc -- the energy of cc_energy (E_CC - E_ref = 1/4 sum
 * <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b, FP64 or complex128) for
 * callers that cannot allocate device memory: code running under a host
 * application that owns the device heap, or in a region where a cudaMalloc
 * would be refused or would synchronise the device.  The paper has no
 * counterpart; it is a convenience of this library.  The block partial sums
 * live in a fixed device array of the library (64 KiB: 4096 real and 4096
 * imaginary partials, each covering 16384 elements), held on every GPU that
 * loads the library until the process exits; nothing is allocated and no
 * workspace is taken.
 *   o, v: extents; o^2 v^2 must not exceed 67,108,864, otherwise the call
 *   returns CC_ERR_INVALID_ARG before touching any pointer.
 *   dtype: CC_F64 (double tensors) or CC_C128 (interleaved complex double);
 *   it says how ints->oovv, amps->t1 and amps->t2 are read.
 *   ints->oovv, amps->t2 (and amps->t1, may be NULL): device inputs.
 *   e_dev: device double[2] receiving (Re E, Im E) (Im E = 0 for CC_F64).
 * The array's device address is looked up on every call with the caller's
 * device current; the first call on a device may load the library's device
 * code there, so make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's partials: calls that
 * overlap on the GPU (different streams or threads, same device) race. */
CC_API cc_status cc_energy_noalloc(int o, int v, cc_dtype dtype, const cc_integrals *ints, const cc_amps *amps,
                                   double *e_dev, void *stream);

/* cc_selftest_wait_timeout -- checks the bounded-wait mechanism of the
 * tensor-core kernels on this device: one CTA waits, with the kernels' own
 * bounded mbarrier wait and a budget of budget_cycles (1e3..4e9 SM cycles), on
 * a barrier that nothing arrives at.  Returns CC_ERR_TIMEOUT when the wait
 * gave up and the kernel returned (the expected outcome; the context stays
 * usable), CC_ERR_CUDA otherwise.  Diagnostic; the paper has no counterpart.
 * Allocates and frees 4 bytes of device memory and synchronises. */
CC_API cc_status cc_selftest_wait_timeout(long long budget_cycles);

/* cc_selftest_convert -- the split kernels' double -> float rounding (integer
 * pipe, round to nearest even) next to the library conversion, for testing:
 * in: device double[n]; mine, ref: device float[n].  Synchronises.
 * Diagnostic; the paper has no counterpart. */
CC_API cc_status cc_selftest_convert(const double *in, long long n, float *mine, float *ref);

CC_API const char *cc_status_string(cc_status s);
CC_API const char *cc_last_error(void);

/* Library version and the device architecture it was built for. */
CC_API const char *cc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CCB300_CC_H */
