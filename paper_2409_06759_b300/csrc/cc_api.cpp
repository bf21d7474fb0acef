// cc_api.cpp -- the C ABI of include/cc.h: plan objects, the residual
// executor, energy, the Jacobi+DIIS solver and the integral builder.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "../../include/cc.h"
#include "kernels.h"
#include "plan.h"

using namespace ccb;

namespace {

thread_local std::string g_err;

cc_status fail(cc_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CC_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(CC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct SolverState {
    int nstored = 0;
    int order[16] = {0};        // history slots, oldest first
    int pending_m = 0;          // m passed to the last device DIIS solve (0 = none)
    int iter = 0;
    double best = INFINITY;
    int phase = 0;              // 0: plan, 1: defect-corrected with the refine plan
    int stall = 0;
    int inner = 0;              // phase 1: corrected iterations since the last FP64 evaluation
    double rn64 = INFINITY;     // phase 1: |R| of the last FP64 evaluation
};

// Phase 1 of cc_solve with a refine plan: every outer step evaluates the FP64
// residual R64(x) (convergence is judged on it alone) and the plan's residual
// Rp(x) at the same point, keeps delta = R64 - Rp, and the following inner
// iterations use Rp(x) + delta.  A new outer step starts after kInnerMax inner
// iterations or once the corrected |R| falls below kInnerDrop * |R64|.
constexpr int kInnerMax = 4;
constexpr double kInnerDrop = 0.02;

}  // namespace

void ccb_set_last_error(const std::string &msg) { g_err = msg; }

// Per-step CUDA-event timing (cc_plan_profile_enable).
struct Profile {
    bool on = false;
    bool pending = false;           // events of the last run not yet harvested
    std::vector<cudaEvent_t> ev;    // 3 per step: start, after the operand splits, end
    std::vector<double> ms_step, ms_gemm;
    int calls = 0;
};

struct cc_plan_s {
    Plan plan;
    bool cache_filled = false;  // static split planes valid (inside one cc_solve call)
    SolverState solver;
    Profile prof;
    long long launches = 0;     // kernels launched by calls on this plan
};

namespace {

const void *block_ptr(const cc_integrals *I, int b) {
    const void *p[7] = {I->oooo, I->ooov, I->oovv, I->ovov, I->ovvv, I->vvvv, I->vvvv_packed};
    return p[b];
}

double *resolve(const BufRef &r, const cc_integrals *I, const cc_amps *A, const cc_resid *R, char *ws) {
    switch (r.where) {
        case BufRef::AMP: return (double *)(r.slot == 1 ? A->t1 : r.slot == 2 ? A->t2 : A->t3);
        case BufRef::RES: return (double *)(r.slot == 1 ? R->r1 : r.slot == 2 ? R->r2 : R->r3);
        case BufRef::INTEG: return (double *)block_ptr(I, r.slot);
        case BufRef::WS: return (double *)(ws + r.off);
        default: return nullptr;
    }
}

bool aligned256(const void *p) { return ((uintptr_t)p & 255) == 0; }

cc_status check_inputs(const Plan &P, const cc_integrals *I, const cc_amps *A, const cc_resid *R, void *ws,
                       size_t wsb) {
    if (!I || !A || !R) return fail(CC_ERR_INVALID_ARG, "NULL integrals, amplitudes or residual struct");
    if (!I->f_occ || !I->f_vir) return fail(CC_ERR_INVALID_ARG, "NULL orbital energies");
    for (auto &t : P.tensors) {
        if (t.kind == TKind::INTEGRAL) {
            if (P.integ_used[t.slot] && !block_ptr(I, t.slot))
                return fail(CC_ERR_INVALID_ARG, "integral block " + t.name + " is NULL but the list uses it");
        } else if (t.kind == TKind::AMP) {
            void *p = t.slot == 1 ? A->t1 : t.slot == 2 ? A->t2 : A->t3;
            if (!p) return fail(CC_ERR_INVALID_ARG, "amplitude " + t.name + " is NULL but the list uses it");
        } else if (t.kind == TKind::RES) {
            void *p = t.slot == 1 ? R->r1 : t.slot == 2 ? R->r2 : R->r3;
            if (!p) return fail(CC_ERR_INVALID_ARG, "residual " + t.name + " is NULL but the list writes it");
        }
    }
    if ((int64_t)wsb < P.ws_bytes)
        return fail(CC_ERR_WORKSPACE, "workspace too small: need " + std::to_string(P.ws_bytes) + " bytes");
    if (!ws || !aligned256(ws)) return fail(CC_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    return CC_OK;
}

cc_status harvest_profile(cc_plan_s *pl) {
    Profile &pf = pl->prof;
    if (!pf.pending) return CC_OK;
    CC_CUDA(cudaEventSynchronize(pf.ev.back()));
    for (size_t k = 0; k < pl->plan.steps.size(); k++) {
        float a = 0.f, b = 0.f;
        CC_CUDA(cudaEventElapsedTime(&a, pf.ev[3 * k], pf.ev[3 * k + 2]));
        CC_CUDA(cudaEventElapsedTime(&b, pf.ev[3 * k + 1], pf.ev[3 * k + 2]));
        pf.ms_step[k] += a;
        pf.ms_gemm[k] += b;
    }
    pf.calls++;
    pf.pending = false;
    return CC_OK;
}

// One step of a plan.  splits: run the operand splits of a split-bf16 GEMM
// (false re-runs only its GEMM, for autotuning).  mark: event recorded after
// the splits, just before the GEMM kernel (profiling), or NULL.
cc_status exec_step(cc_plan_s *pl, const Step &stp, const cc_integrals *I, const cc_amps *A, const cc_resid *R,
                    char *w, cudaStream_t s, bool splits, cudaEvent_t mark) {
    const Plan &P = pl->plan;
    switch (stp.kind) {
        case StepKind::ZERO:
            CC_CUDA(launch_zero(resolve(stp.out, I, A, R, w), stp.zero_elems, s));
            pl->launches++;
            break;
        case StepKind::ACCUM:
            if (!(stp.static_src && pl->cache_filled)) {
                CC_CUDA(launch_accum(stp.acc, resolve(stp.a, I, A, R, w), resolve(stp.out, I, A, R, w), s,
                                     stp.acc.two_src ? resolve(stp.b, I, A, R, w) : nullptr,
                                     stp.acc.has_add ? resolve(stp.c, I, A, R, w) : nullptr));
                pl->launches++;
            }
            break;
        case StepKind::PACK:
            if (!(stp.static_src && pl->cache_filled)) {
                CC_CUDA(launch_pack_pairs(stp.pk, resolve(stp.a, I, A, R, w), resolve(stp.out, I, A, R, w), s));
                pl->launches++;
            }
            break;
        case StepKind::UNPACK:
            CC_CUDA(launch_unpack_pairs(stp.up, resolve(stp.a, I, A, R, w), resolve(stp.out, I, A, R, w), s));
            pl->launches++;
            break;
        case StepKind::GEMM:
            if (stp.nk) {
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_narrow_k(stp.nkd, resolve(stp.a, I, A, R, w), resolve(stp.b, I, A, R, w),
                                        resolve(stp.out, I, A, R, w), s));
                pl->launches += stp.nkd.beta != 1.0 ? 2 : 1;
            } else if (stp.rows && !stp.kcat.empty()) {
                RowsMultiDesc d = stp.rm;
                for (size_t k = 0; k < stp.kcat.size(); k++) {
                    d.m[k].X = resolve(stp.kcat[k].a, I, A, R, w);
                    d.m[k].Y = resolve(stp.kcat[k].b, I, A, R, w);
                }
                d.red = stp.rg.red;
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_rows_multi(d, resolve(stp.out, I, A, R, w), s));
                pl->launches++;
            } else if (stp.rows) {
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_rows_gemm(stp.rg, resolve(stp.a, I, A, R, w), resolve(stp.b, I, A, R, w),
                                         resolve(stp.out, I, A, R, w), s));
                pl->launches++;
            } else if (!stp.mixed) {
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_gemm_f64(stp.gemm, resolve(stp.a, I, A, R, w), resolve(stp.b, I, A, R, w),
                                        resolve(stp.out, I, A, R, w), resolve(stp.partials, I, A, R, w), s));
                pl->launches += stp.gemm.splitk > 1 ? 2 : 1;
            } else if (!stp.kcat.empty()) {
                // K-concatenated members: each fills its own K columns of the shared planes
                void *pa = w + stp.planes_a_off, *pb = w + stp.planes_b_off;
                if (splits) {
                    for (const KMember &m : stp.kcat) {
                        CC_CUDA(launch_split_bf16(m.split_a, resolve(m.a, I, A, R, w), pa, s));
                        CC_CUDA(launch_split_bf16(m.split_b, resolve(m.b, I, A, R, w), pb, s));
                        pl->launches += 2;
                    }
                }
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_tc_gemm(stp.tc, pa, pb, resolve(stp.out, I, A, R, w), resolve(stp.partials, I, A, R, w),
                                       (int *)(w + P.flags_off), s));
                pl->launches += stp.tc.splitk > 1 ? 2 : 1;
            } else {
                void *pa = w + stp.planes_a_off, *pb = w + stp.planes_b_off;
                if (splits && !(stp.a_static && pl->cache_filled) && !stp.skip_a) {
                    CC_CUDA(launch_split_bf16(stp.split_a, resolve(stp.a, I, A, R, w), pa, s));
                    pl->launches++;
                }
                if (splits && !(stp.b_static && pl->cache_filled) && !stp.skip_b) {
                    CC_CUDA(launch_split_bf16(stp.split_b, resolve(stp.b, I, A, R, w), pb, s));
                    pl->launches++;
                }
                if (mark) CC_CUDA(cudaEventRecord(mark, s));
                CC_CUDA(launch_tc_gemm(stp.tc, pa, pb, resolve(stp.out, I, A, R, w), resolve(stp.partials, I, A, R, w),
                                       (int *)(w + P.flags_off), s));
                pl->launches += stp.tc.splitk > 1 ? 2 : 1;
            }
            break;
    }
    return CC_OK;
}

cc_status run_residual(cc_plan_s *pl, const cc_integrals *I, const cc_amps *A, const cc_resid *R, void *ws,
                       size_t wsb, cudaStream_t s, bool use_cache) {
    const Plan &P = pl->plan;
    cc_status st = check_inputs(P, I, A, R, ws, wsb);
    if (st != CC_OK) return st;
    char *w = (char *)ws;
    Profile &pf = pl->prof;
    if (pf.on) {
        st = harvest_profile(pl);
        if (st != CC_OK) return st;
    }
    size_t si = 0;
    if (!use_cache) pl->cache_filled = false;
    if (P.flops_mixed > 0 && !pl->cache_filled)   // clear the bounded-wait status word (once per solve)
        CC_CUDA(cudaMemsetAsync(w + P.flags_off, 0, sizeof(int), s));
    for (const Step &stp : P.steps) {
        if (pf.on) CC_CUDA(cudaEventRecord(pf.ev[3 * si], s));
        st = exec_step(pl, stp, I, A, R, w, s, true, pf.on ? pf.ev[3 * si + 1] : nullptr);
        if (st != CC_OK) return st;
        if (pf.on) {
            if (stp.kind != StepKind::GEMM) CC_CUDA(cudaEventRecord(pf.ev[3 * si + 1], s));
            CC_CUDA(cudaEventRecord(pf.ev[3 * si + 2], s));
        }
        si++;
    }
    if (pf.on) pf.pending = true;
    if (use_cache) pl->cache_filled = true;
    // R -= D * t for every residual the list writes
    for (int l = 1; l <= 3; l++) {
        if (!P.res_used[l]) continue;
        const double *t = (const double *)(l == 1 ? A->t1 : l == 2 ? A->t2 : A->t3);
        double *r = (double *)(l == 1 ? R->r1 : l == 2 ? R->r2 : R->r3);
        if (t) {
            CC_CUDA(launch_denom_sub(l, P.o, P.v, I->f_occ, I->f_vir, t, r, P.dtype == CC_C128, s));
            pl->launches++;
        }
    }
    return CC_OK;
}

int64_t amp_count(int rank, int o, int v) {
    int64_t n = 1;
    for (int k = 0; k < rank; k++) n *= (int64_t)o * v;
    return n;
}

constexpr int64_t kAlign = 256;
int64_t al(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// solver region layout (bytes, relative to its start).  Counts are in
// doubles: a complex amplitude is two, and the DIIS overlaps are Re<x|y>.
struct SolverLayout {
    int64_t n[4] = {0, 0, 0, 0};    // doubles per rank (1..3)
    int64_t nx = 0;                 // elements of x = concatenation of the ranks in use
    int64_t r_off[4] = {0, 0, 0, 0};
    int64_t hist_x = 0, hist_e = 0; // diis_max vectors of nx each
    int64_t gram = 0, coef = 0, used = 0, scal = 0, partials = 0, delta = 0, dinv = 0;
    int64_t bytes = 0;
    int diis = 0;
};

SolverLayout solver_layout(const Plan &P, int diis_max) {
    SolverLayout L;
    int64_t off = 0;
    for (int l = 1; l <= 3; l++) {
        if (!P.res_used[l]) continue;
        L.n[l] = amp_count(l, P.o, P.v) * (P.dtype == CC_C128 ? 2 : 1);
        L.nx += L.n[l];
        L.r_off[l] = off;
        off += al(L.n[l] * 8);
    }
    L.diis = std::max(diis_max, 1);
    L.hist_x = off;
    off += al((int64_t)L.diis * L.nx * 8);
    L.hist_e = off;
    off += al((int64_t)L.diis * L.nx * 8);
    L.delta = off;
    off += al(L.nx * 8);
    L.dinv = off;                   // 1/D of every amplitude (Jacobi), set at the start of a solve
    off += al(L.nx * 8);
    L.gram = off; off += al(256 * 8);
    L.coef = off; off += al(16 * 8);
    L.used = off; off += al(16);
    L.scal = off; off += al(8 * 8);
    L.partials = off; off += al((int64_t)20 * kRedBlocks * 8);
    L.bytes = off;
    return L;
}

// scal[0] = Re E, scal[1] = Im E, scal[2..] = |R_l|^2 for the residual ranks in use
cc_status reduce_energy_norm(const Plan &P, const cc_integrals *I, const cc_amps *A, double *const r[4],
                             const int64_t n[4], double *partials, double *scal, cudaStream_t s) {
    const int cplx = P.dtype == CC_C128;
    CC_CUDA(launch_energy_partials(P.o, P.v, (const double *)I->oovv, (const double *)A->t1, (const double *)A->t2,
                                   partials, cplx, s));
    if (!cplx) CC_CUDA(cudaMemsetAsync(partials + kRedBlocks, 0, kRedBlocks * sizeof(double), s));
    int cnt = 2;
    for (int l = 1; l <= 3; l++) {
        if (!r[l]) continue;
        CC_CUDA(launch_dot_partials(r[l], r[l], n[l], partials + (int64_t)cnt * kRedBlocks, s));
        cnt++;
    }
    CC_CUDA(launch_reduce_partials(partials, cnt, scal, s));
    return CC_OK;
}

}  // namespace

extern "C" {

const char *cc_status_string(cc_status s) {
    switch (s) {
        case CC_OK: return "ok";
        case CC_ERR_INVALID_ARG: return "invalid argument";
        case CC_ERR_PARSE: return "parse error";
        case CC_ERR_SHAPE: return "shape error";
        case CC_ERR_UNSUPPORTED: return "unsupported";
        case CC_ERR_OOM: return "out of memory";
        case CC_ERR_CUDA: return "CUDA error";
        case CC_ERR_NOT_CONVERGED: return "not converged";
        case CC_ERR_TIMEOUT: return "device wait timed out";
        case CC_ERR_WORKSPACE: return "workspace error";
    }
    return "unknown status";
}

const char *cc_last_error(void) { return g_err.c_str(); }

const char *cc_version(void) { return "ccb300 0.1 (sm_103a)"; }

cc_status cc_plan_create(const char *text, int o, int v, cc_dtype dtype, cc_precision precision,
                         const cc_plan_opts *opts, cc_plan *out) {
    if (!text || !out) return fail(CC_ERR_INVALID_ARG, "NULL text or output handle");
    if (o < 1 || v < 1) return fail(CC_ERR_INVALID_ARG, "o and v must be >= 1");
    if (dtype != CC_F64 && dtype != CC_C128) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    const int prec = (int)precision;
    const int base = prec >= 100 ? prec - 100 : prec;
    if (base != CC_PREC_FP64 && base != CC_PREC_BF16X3 && base != CC_PREC_BF16X6 && base != CC_PREC_SLICES)
        return fail(CC_ERR_INVALID_ARG, "unknown precision");
    cc_plan_s *pl = new (std::nothrow) cc_plan_s();
    if (!pl) return fail(CC_ERR_OOM, "plan allocation failed");
    std::string err;
    int flags = 0;
    if (opts && opts->struct_size >= (int)(offsetof(cc_plan_opts, packed_vvvv) + sizeof(int)) && opts->packed_vvvv)
        flags |= 1;
    if (opts && opts->struct_size >= (int)(offsetof(cc_plan_opts, no_kconcat) + sizeof(int)) && opts->no_kconcat)
        flags |= 2;
    int prec_eff = prec;
    if (opts && opts->struct_size >= (int)(offsetof(cc_plan_opts, uniform_steps) + sizeof(int)) &&
        opts->uniform_steps) {
        if (dtype != CC_F64 || (base != CC_PREC_BF16X3 && base != CC_PREC_BF16X6)) {
            delete pl;
            return fail(CC_ERR_UNSUPPORTED, "uniform_steps needs a real split-bf16 plan");
        }
        flags |= 2 | 4;
        prec_eff = base + 100;
    }
    if (!build_plan(text, o, v, (int)dtype, prec_eff, pl->plan, err, flags)) {
        delete pl;
        return fail(err.find("index spaces") != std::string::npos ? CC_ERR_SHAPE : CC_ERR_PARSE, err);
    }
    if (opts && opts->struct_size >= (int)(2 * sizeof(int)) && opts->verbose) {
        pl->plan.verbose = 1;
        std::fprintf(stderr, "%s\n", describe_plan(pl->plan).c_str());
    }
    *out = pl;
    return CC_OK;
}

cc_status cc_plan_workspace_bytes(cc_plan plan, size_t *bytes) {
    if (!plan || !bytes) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    *bytes = (size_t)plan->plan.ws_bytes;
    return CC_OK;
}

cc_status cc_plan_describe(cc_plan plan, char *buf, size_t len, size_t *needed) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    std::string d = describe_plan(plan->plan);
    if (needed) *needed = d.size() + 1;
    if (buf && len) {
        size_t n = std::min(len - 1, d.size());
        std::memcpy(buf, d.data(), n);
        buf[n] = 0;
    }
    return CC_OK;
}

cc_status cc_plan_flops(cc_plan plan, double *flops) {
    if (!plan || !flops) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    *flops = plan->plan.flops;
    return CC_OK;
}

cc_status cc_plan_destroy(cc_plan plan) {
    if (!plan) return CC_OK;
    for (cudaEvent_t e : plan->prof.ev) cudaEventDestroy(e);
    delete plan;
    return CC_OK;
}

cc_status cc_plan_profile_enable(cc_plan plan, int enable) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    Profile &pf = plan->prof;
    if (enable) {
        const size_t need = 3 * plan->plan.steps.size();
        while (pf.ev.size() < need) {
            cudaEvent_t e;
            CC_CUDA(cudaEventCreate(&e));
            pf.ev.push_back(e);
        }
        pf.ms_step.assign(plan->plan.steps.size(), 0.0);
        pf.ms_gemm.assign(plan->plan.steps.size(), 0.0);
        pf.calls = 0;
        pf.pending = false;
        pf.on = true;
    } else {
        cc_status st = harvest_profile(plan);
        pf.on = false;
        if (st != CC_OK) return st;
    }
    return CC_OK;
}

cc_status cc_plan_profile_read(cc_plan plan, double *ms_step, double *ms_kernel, int cap, int *nsteps, int *calls) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    cc_status st = harvest_profile(plan);
    if (st != CC_OK) return st;
    const Profile &pf = plan->prof;
    const int n = (int)pf.ms_step.size();
    if (nsteps) *nsteps = (int)plan->plan.steps.size();
    if (calls) *calls = pf.calls;
    for (int k = 0; k < n && k < cap; k++) {
        if (ms_step) ms_step[k] = pf.ms_step[k];
        if (ms_kernel) ms_kernel[k] = pf.ms_gemm[k];
    }
    return CC_OK;
}

cc_status cc_plan_launch_count(cc_plan plan, long long *count) {
    if (!plan || !count) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    *count = plan->launches;
    return CC_OK;
}

cc_status cc_residual(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, cc_resid *res, void *ws,
                      size_t ws_bytes, void *stream) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    return run_residual(plan, ints, amps, res, ws, ws_bytes, (cudaStream_t)stream, false);
}

}  // extern "C"

namespace {
// Shape-keyed tuning results shared by every plan of the process: a contraction
// whose route, shape and candidate set were timed before (on any plan, e.g. a
// same-sized system of a batch) takes the stored pick without timing again.
struct TuneKey {
    int route;                  // 0 tiled GEMM, 1 narrow, 2 split route
    int64_t M, N, K;
    int prod, f32, cplx, beta, ncand;
    bool operator<(const TuneKey &o) const {
        return std::tie(route, M, N, K, prod, f32, cplx, beta, ncand) <
               std::tie(o.route, o.M, o.N, o.K, o.prod, o.f32, o.cplx, o.beta, o.ncand);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 3>> g_tune;
long long g_tune_hits = 0;

TuneKey tune_key(const Step &st) {
    TuneKey k{};
    k.route = st.mixed ? 2 : st.rows ? 1 : 0;
    k.M = st.mixed ? st.tc.M : st.gemm.M;
    k.N = st.mixed ? st.tc.N : st.gemm.N;
    k.K = st.mixed ? st.tc.Kp : st.gemm.K;
    k.prod = st.mixed ? st.tc.nprod : 0;
    k.f32 = st.gemm.f32;
    k.cplx = st.mixed ? st.split_a.cplx : st.gemm.cplx;
    k.beta = beta_case(st.mixed ? st.tc.beta : st.rows ? st.rg.beta : st.gemm.beta);
    k.ncand = (int)st.cands.size();
    return k;
}
}  // namespace

extern "C" {

cc_status cc_autotune_cache(int clear, long long *entries, long long *hits) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (clear) {
        g_tune.clear();
        g_tune_hits = 0;
    }
    if (entries) *entries = (long long)g_tune.size();
    if (hits) *hits = g_tune_hits;
    return CC_OK;
}

cc_status cc_plan_autotune(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, cc_resid *res, void *ws,
                           size_t ws_bytes, void *stream, int reps) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    if (plan->prof.on) return fail(CC_ERR_INVALID_ARG, "disable profiling before autotuning");
    if (reps < 1 || reps > 100) return fail(CC_ERR_INVALID_ARG, "reps must be in [1, 100]");
    cudaStream_t s = (cudaStream_t)stream;
    // one full residual first: static caches filled, kernels warm
    cc_status st = run_residual(plan, ints, amps, res, ws, ws_bytes, s, false);
    if (st != CC_OK) return st;
    plan->cache_filled = true;
    Plan &P = plan->plan;
    char *w = (char *)ws;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CC_CUDA(cudaEventCreate(&e0));
    CC_CUDA(cudaEventCreate(&e1));
    cc_status result = CC_OK;
    for (Step &stp : P.steps) {
        // the step once as planned (its operands are then in place), then every candidate
        st = exec_step(plan, stp, ints, amps, res, w, s, true, nullptr);
        if (st != CC_OK) { result = st; break; }
        if (stp.cands.size() < 2) continue;
        const TuneKey key = tune_key(stp);
        std::array<int, 3> pick = stp.cands[0];
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end() &&
                std::find(stp.cands.begin(), stp.cands.end(), it->second) != stp.cands.end()) {
                pick = it->second;
                cached = true;
                g_tune_hits++;
            }
        }
        double best = 1e30;
        for (const auto &c : stp.cands) {
            if (cached) break;
            Step trial = stp;
            if (trial.mixed) {
                trial.tc.bn = c[0];
                trial.tc.splitk = c[1];
                trial.tc.red = c[2];
            } else {
                trial.gemm.splitk = c[1];
                trial.gemm.red = c[2];
                trial.rg.red = c[2];
            }
            float ms = 0.f, acc = 0.f;
            for (int r = 0; r < reps; r++) {
                if (cudaEventRecord(e0, s) != cudaSuccess) { result = fail(CC_ERR_CUDA, "event record"); break; }
                st = exec_step(plan, trial, ints, amps, res, w, s, false, nullptr);
                if (st != CC_OK) { result = st; break; }
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    result = fail(CC_ERR_CUDA, "event timing");
                    break;
                }
                acc = r == 0 ? ms : std::min(acc, ms);
            }
            if (result != CC_OK) break;
            if (acc < best) { best = acc; pick = c; }
        }
        if (result != CC_OK) break;
        if (!cached) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = pick;
        }
        if (stp.mixed) {
            stp.tc.bn = pick[0];
            stp.tc.splitk = pick[1];
            stp.tc.red = pick[2];
        } else {
            stp.gemm.splitk = pick[1];
            stp.gemm.red = pick[2];
            stp.rg.red = pick[2];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result == CC_OK) {
        P.tuned = true;
        plan->cache_filled = false;
    }
    return result;
}

int64_t cc_packed_t2_elems(int o, int v) {
    if (o < 0 || v < 0) return 0;
    return ((int64_t)o * (o - 1) / 2) * ((int64_t)v * (v - 1) / 2);
}

static cc_status t2_pack_args(int o, int v, cc_dtype dtype, const void *x, const void *y) {
    if (o < 1 || v < 1 || o > 4096 || v > 65535) return fail(CC_ERR_INVALID_ARG, "o, v out of range");
    if (dtype != CC_F64 && dtype != CC_C128) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    if (!x || !y) return fail(CC_ERR_INVALID_ARG, "NULL array");
    if ((uintptr_t)x % (dtype == CC_C128 ? 16 : 8) || (uintptr_t)y % (dtype == CC_C128 ? 16 : 8))
        return fail(CC_ERR_INVALID_ARG, "arrays must be aligned to their element size");
    return CC_OK;
}

cc_status cc_pack_t2(int o, int v, cc_dtype dtype, const void *t_full, void *t_packed, void *stream) {
    cc_status st = t2_pack_args(o, v, dtype, t_full, t_packed);
    if (st != CC_OK) return st;
    CC_CUDA(launch_pack_t2(o, v, dtype == CC_C128, (const double *)t_full, (double *)t_packed, (cudaStream_t)stream));
    return CC_OK;
}

cc_status cc_unpack_t2(int o, int v, cc_dtype dtype, const void *t_packed, void *t_full, void *stream) {
    cc_status st = t2_pack_args(o, v, dtype, t_packed, t_full);
    if (st != CC_OK) return st;
    CC_CUDA(launch_unpack_t2(o, v, dtype == CC_C128, (const double *)t_packed, (double *)t_full,
                             (cudaStream_t)stream));
    return CC_OK;
}

cc_status cc_plan_set_gemm_config(cc_plan plan, int step, int bn, int splitk, int red) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "NULL plan");
    Plan &P = plan->plan;
    if (step < 0 || step >= (int)P.steps.size()) return fail(CC_ERR_INVALID_ARG, "step index out of range");
    Step &stp = P.steps[step];
    const std::array<int, 3> want{bn, splitk, red};
    bool found = false;
    for (const auto &c : stp.cands) found = found || c == want;
    if (!found) return fail(CC_ERR_INVALID_ARG, "not a candidate configuration of this step");
    if (stp.mixed) {
        stp.tc.bn = bn;
        stp.tc.splitk = splitk;
        stp.tc.red = red;
    } else {
        stp.gemm.splitk = splitk;
        stp.gemm.red = red;
        stp.rg.red = red;
    }
    return CC_OK;
}

cc_status cc_energy(cc_plan plan, const cc_integrals *ints, const cc_amps *amps, double *e_dev, void *ws,
                    size_t ws_bytes, void *stream) {
    if (!plan || !ints || !amps || !e_dev) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    if (!ints->oovv || !amps->t2) return fail(CC_ERR_INVALID_ARG, "energy needs the oovv block and t2");
    if (!ws || ws_bytes < (size_t)2 * kRedBlocks * 8 || !aligned256(ws))
        return fail(CC_ERR_WORKSPACE, "energy needs 10 KiB of 256-byte aligned workspace");
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = (double *)ws;
    const int cplx = plan->plan.dtype == CC_C128;
    CC_CUDA(launch_energy_partials(plan->plan.o, plan->plan.v, (const double *)ints->oovv, (const double *)amps->t1,
                                   (const double *)amps->t2, partials, cplx, s));
    CC_CUDA(launch_reduce_partials(partials, cplx ? 2 : 1, e_dev, s));
    if (!cplx) CC_CUDA(cudaMemsetAsync(e_dev + 1, 0, sizeof(double), s));
    return CC_OK;
}

cc_status cc_solve_workspace_bytes(cc_plan plan, const cc_solve_opts *opts, size_t *bytes) {
    if (!plan || !bytes) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    int diis = opts ? opts->diis_max : 8;
    if (diis < 0 || diis > 16) return fail(CC_ERR_INVALID_ARG, "diis_max must be in [0, 16]");
    // the refine plan gets a region of its own: the plan's cached split planes
    // must survive the FP64 evaluations of the corrected phase
    int64_t pw = al(plan->plan.ws_bytes);
    if (opts && opts->refine_plan) pw += al(opts->refine_plan->plan.ws_bytes);
    *bytes = (size_t)(pw + solver_layout(plan->plan, diis).bytes);
    return CC_OK;
}

cc_status cc_solve(cc_plan plan, const cc_integrals *ints, cc_amps *amps, const cc_solve_opts *opts,
                   cc_solve_report *report, void *ws, size_t ws_bytes, void *stream) {
    if (!plan || !ints || !amps) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    cc_solve_opts o{};
    o.struct_size = sizeof(o);
    o.max_iter = 100;
    o.tol = 1e-8;
    o.diis_max = 8;
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.diis_max < 0 || o.diis_max > 16) return fail(CC_ERR_INVALID_ARG, "bad solve options");
    cc_plan refine = o.refine_plan;
    if (refine && (refine->plan.o != plan->plan.o || refine->plan.v != plan->plan.v ||
                   refine->plan.dtype != plan->plan.dtype))
        return fail(CC_ERR_INVALID_ARG, "refine plan has different o/v or dtype");
    const Plan &P = plan->plan;
    if (!P.res_used[2]) return fail(CC_ERR_INVALID_ARG, "cc_solve needs a list that writes R2");
    if (refine) {
        for (int l = 1; l <= 3; l++)
            if (refine->plan.res_used[l] != P.res_used[l])
                return fail(CC_ERR_INVALID_ARG, "refine plan writes different residuals");
    }
    size_t need = 0;
    cc_status st = cc_solve_workspace_bytes(plan, &o, &need);
    if (st != CC_OK) return st;
    if (ws_bytes < need || !ws || !aligned256(ws))
        return fail(CC_ERR_WORKSPACE, "solve workspace too small: need " + std::to_string(need));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t pw = al(P.ws_bytes);
    const int64_t rw = refine ? al(refine->plan.ws_bytes) : 0;
    char *pws = (char *)ws;
    char *rws = (char *)ws + pw;
    char *sreg = (char *)ws + pw + rw;
    SolverLayout L = solver_layout(P, o.diis_max);
    const int o_ = P.o, v_ = P.v;
    double *r[4] = {nullptr, nullptr, nullptr, nullptr};
    double *t[4] = {nullptr, (double *)amps->t1, (double *)amps->t2, (double *)amps->t3};
    for (int l = 1; l <= 3; l++)
        if (P.res_used[l]) {
            r[l] = (double *)(sreg + L.r_off[l]);
            if (!t[l]) return fail(CC_ERR_INVALID_ARG, "amplitude buffer missing for a residual the list writes");
        }
    cc_resid R{r[1], r[2], r[3]};
    double *hx = (double *)(sreg + L.hist_x), *he = (double *)(sreg + L.hist_e);
    double *gram = (double *)(sreg + L.gram), *coef = (double *)(sreg + L.coef);
    int *used_dev = (int *)(sreg + L.used);
    double *scal = (double *)(sreg + L.scal), *partials = (double *)(sreg + L.partials);
    SolverState &S = plan->solver;
    if (!o.resume) {
        S = SolverState();
        CC_CUDA(cudaMemsetAsync(used_dev, 0, 16, s));
    }
    // host staging for the per-iteration scalars (E, |R|, DIIS bookkeeping):
    // 56 bytes read once per iteration right before the stream synchronisation,
    // so plain stack memory serves (no host or device allocation in the call)
    alignas(16) double h_scal[16] = {};
    if (report) { report->iterations = 0; report->converged = 0; report->switched_at = -1; }
    const int cplx = P.dtype == CC_C128;
    // the static caches (permuted and split integral blocks) are rebuilt at the
    // start of a solve; a resumed solve continues with them
    if (!o.resume) {
        plan->cache_filled = false;
        if (refine) refine->cache_filled = false;
    }
    g_err.clear();
    cc_status result = CC_ERR_NOT_CONVERGED;
    double last_e = NAN, last_ei = NAN, last_rn = NAN;
    int k = 0;
    double *dl = (double *)(sreg + L.delta);
    double *dlr[4] = {nullptr, nullptr, nullptr, nullptr};
    {
        int64_t off = 0;
        for (int l = 1; l <= 3; l++)
            if (r[l]) { dlr[l] = dl + off; off += L.n[l]; }
    }
    cc_resid Rd{dlr[1], dlr[2], dlr[3]};
    double *dinv = (double *)(sreg + L.dinv);
    if (!o.resume) {
        // 1/D of every amplitude; a resumed solve (same integrals, plan and ws) keeps it
        int64_t off = 0;
        for (int l = 1; l <= 3; l++) {
            if (!r[l]) continue;
            CC_CUDA(launch_inv_denominators(l, o_, v_, ints->f_occ, ints->f_vir, dinv + off, cplx, s));
            plan->launches++;
            off += L.n[l];
        }
    }
    for (k = 0; k < o.max_iter; k++) {
        const bool corrected = S.phase == 1 && refine != nullptr;
        const bool outer = corrected && S.inner == 0;
        if (corrected && outer) {
            st = run_residual(refine, ints, amps, &R, rws, (size_t)rw, s, true);
            if (st != CC_OK) return st;
        }
        // the plan's residual: R itself, or (outer) Rp into the delta buffer
        st = run_residual(plan, ints, amps, (corrected && outer) ? &Rd : &R, pws, (size_t)pw, s, true);
        if (st != CC_OK) return st;
        if (corrected) {
            // delta = R64 - Rp (outer), or R = Rp + delta (inner)
            for (int l = 1; l <= 3; l++) {
                if (!r[l]) continue;
                if (outer) CC_CUDA(launch_axpby(L.n[l], 1.0, r[l], -1.0, dlr[l], s));
                else CC_CUDA(launch_axpby(L.n[l], 1.0, dlr[l], 1.0, r[l], s));
                plan->launches++;
            }
        }
        st = reduce_energy_norm(P, ints, amps, r, L.n, partials, scal, s);
        if (st != CC_OK) return st;
        plan->launches += 2 + (r[1] != nullptr) + (r[2] != nullptr) + (r[3] != nullptr);
        CC_CUDA(cudaMemcpyAsync(h_scal, scal, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaMemcpyAsync(h_scal + 6, used_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaMemcpyAsync(h_scal + 7, pws + plan->plan.flags_off, sizeof(int), cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaStreamSynchronize(s));
        if (plan->plan.flops_mixed > 0 && *(int *)(h_scal + 7) != 0)
            return fail(CC_ERR_TIMEOUT, "a bounded tensor-core pipeline wait expired");
        // history bookkeeping of the previous device DIIS solve: drop what it dropped
        if (S.pending_m >= 2) {
            int used = *(int *)(h_scal + 6);
            int keep = used == 0 ? 2 : used;
            while (S.nstored > keep) {
                for (int q = 0; q + 1 < S.nstored; q++) S.order[q] = S.order[q + 1];
                S.nstored--;
            }
            S.pending_m = 0;
        }
        double rr = 0.0;
        for (int l = 1, c = 2; l <= 3; l++)
            if (r[l]) rr += h_scal[c++];
        const double e = h_scal[0], rn = std::sqrt(rr);
        last_e = e;
        last_ei = h_scal[1];
        last_rn = rn;
        if (report && report->energies) report->energies[k] = e;
        if (report && report->energies_im) report->energies_im[k] = h_scal[1];
        if (report && report->rnorms) report->rnorms[k] = rn;
        if (o.verbose)
            std::fprintf(stderr, "cc_solve iter %d phase %d%s E %.14f |R| %.3e\n", S.iter, S.phase,
                         corrected ? (outer ? " fp64" : " corrected") : "", e, rn);
        S.iter++;
        if (!std::isfinite(rn) || rn > 1e3 * S.best) {
            g_err = "divergence: |R| not finite or 1e3 above its best value";
            k++;
            break;
        }
        if (rn < S.best) { S.best = rn; S.stall = 0; } else S.stall++;
        if (refine && S.phase == 0 && (rn < std::max(o.switch_tol, o.tol) || S.stall >= 2)) {
            // switch: the next iteration is an FP64 evaluation at the same amplitudes
            S.phase = 1;
            S.inner = 0;
            S.nstored = 0;
            S.best = INFINITY;
            S.stall = 0;
            if (report) report->switched_at = k;
            continue;
        }
        if (corrected) {
            if (outer) {
                S.rn64 = rn;
                if (o.tol > 0 && rn < o.tol) { result = CC_OK; k++; break; }
                S.inner = 1;
            } else {
                S.inner++;
                if (S.inner > kInnerMax || rn < kInnerDrop * S.rn64) S.inner = 0;
            }
        }
        if (!corrected && o.tol > 0 && rn < o.tol) { result = CC_OK; k++; break; }
        // Jacobi step into a history slot
        int slot = 0;
        if (o.diis_max > 0 && S.nstored == o.diis_max) {
            slot = S.order[0];
            for (int q = 0; q + 1 < S.nstored; q++) S.order[q] = S.order[q + 1];
            S.nstored--;
        } else if (o.diis_max > 0) {
            for (;; slot++) {
                bool busy = false;
                for (int q = 0; q < S.nstored; q++) busy |= S.order[q] == slot;
                if (!busy) break;
            }
        }
        double *xs = hx + (int64_t)slot * L.nx, *es = he + (int64_t)slot * L.nx;
        if (o.diis_max > 0) {
            // Jacobi step and the new Gram row <e_new, e_q> in one pass
            S.order[S.nstored++] = slot;
            JacobiSegs g{};
            for (int l = 1; l <= 3; l++) {
                if (!r[l]) continue;
                g.t[g.nseg] = t[l];
                g.r[g.nseg] = r[l];
                g.n[g.nseg] = L.n[l];
                g.nseg++;
            }
            int a_[16], b_[16];
            g.m = S.nstored;
            for (int q = 0; q < S.nstored; q++) {
                g.he[q] = he + (int64_t)S.order[q] * L.nx;
                a_[q] = slot;
                b_[q] = S.order[q];
            }
            CC_CUDA(launch_jacobi_dots(g, dinv, xs, es, partials, s));
            CC_CUDA(launch_gram_scatter(partials, S.nstored, a_, b_, gram, s));
            plan->launches += 2;
        } else {
            int64_t off = 0;
            for (int l = 1; l <= 3; l++) {
                if (!r[l]) continue;
                CC_CUDA(launch_jacobi_inv(L.n[l], t[l], r[l], dinv + off, xs + off, es + off, s));
                plan->launches++;
                off += L.n[l];
            }
        }
        if (S.nstored >= 2) {
            CC_CUDA(launch_diis_solve(gram, S.order, S.nstored, coef, used_dev, s));
            plan->launches++;
            int64_t off2 = 0;
            for (int l = 1; l <= 3; l++) {
                if (!r[l]) continue;
                const double *xq[16];
                for (int q = 0; q < S.nstored; q++) xq[q] = hx + (int64_t)S.order[q] * L.nx + off2;
                CC_CUDA(launch_combine(xq, coef, used_dev, S.nstored, L.n[l], t[l], s));
                plan->launches++;
                off2 += L.n[l];
            }
            S.pending_m = S.nstored;
        } else {
            int64_t off2 = 0;
            for (int l = 1; l <= 3; l++) {
                if (!r[l]) continue;
                CC_CUDA(cudaMemcpyAsync(t[l], xs + off2, L.n[l] * 8, cudaMemcpyDeviceToDevice, s));
                off2 += L.n[l];
            }
        }
    }
    if (report) {
        report->iterations = k;
        report->converged = result == CC_OK;
        report->energy = last_e;
        report->energy_im = last_ei;
        report->rnorm = last_rn;
    }
    if (result != CC_OK && g_err.empty()) g_err = "maximum iterations reached";
    return result;
}

}  // extern "C"

// ------------------------------------------------------------------ batched
namespace {

// ---- grouped execution of a batch.  When every plan of a batch has the same
// steps (plans made with uniform_steps: real, split-bf16, all contractions on
// the tensor-core route, none merged), a residual evaluation of the whole batch
// is one launch per step: the step's elementwise pass, operand splits and
// tensor-core GEMM each take a table with one entry per system (grouped
// kernels), followed by one grouped denominator/energy/norm pass.  Systems
// whose active flag is 0 (converged) are skipped inside the launches.
bool same_split_route(const Step &a, const Step &b) {
    if (!b.mixed || b.rows || b.nk || !b.kcat.empty() || b.tc.nplanes_a != 2 || b.tc.nplanes_b != 2) return false;
    if (b.tc.nprod != a.tc.nprod || beta_case(b.tc.beta) == 2 || beta_case(b.tc.beta) != beta_case(a.tc.beta))
        return false;
    for (int k = 0; k < b.tc.nprod; k++)
        if (b.tc.prod_a[k] != a.tc.prod_a[k] || b.tc.prod_b[k] != a.tc.prod_b[k]) return false;
    return a.a_static == b.a_static && a.b_static == b.b_static && a.skip_a == b.skip_a && a.skip_b == b.skip_b &&
           b.split_a.cplx == 0 && b.split_b.cplx == 0 && b.split_a.nplanes == 2 && b.split_b.nplanes == 2;
}

bool batch_groupable(int n, const cc_plan *plans) {
    if (n < 2) return false;
    const Plan &P0 = plans[0]->plan;
    for (int i = 0; i < n; i++) {
        const Plan &P = plans[i]->plan;
        if (P.precision != CC_PREC_BF16X3 || P.dtype != CC_F64 || P.res_used[3] || !P.res_used[1] ||
            !P.res_used[2] || P.steps.size() != P0.steps.size() || P.packed_vvvv)
            return false;
        for (size_t k = 0; k < P.steps.size(); k++) {
            const Step &a = P0.steps[k], &b = P.steps[k];
            if (a.kind != b.kind) return false;
            if (b.kind == StepKind::ACCUM) {
                const int bc = beta_case(b.acc.beta);
                if (bc == 2 || bc != beta_case(a.acc.beta) || b.acc.cplx || a.static_src != b.static_src ||
                    a.acc.two_src != b.acc.two_src || a.acc.has_add != b.acc.has_add)
                    return false;
            } else if (b.kind == StepKind::GEMM && a.rows) {
                if (!b.rows || b.nk || !b.kcat.empty() || b.mixed || b.gemm.f32 != a.gemm.f32 ||
                    beta_case(b.rg.beta) == 2 || beta_case(b.rg.beta) != beta_case(a.rg.beta))
                    return false;
            } else if (b.kind == StepKind::GEMM) {
                if (!same_split_route(a, b) || !same_split_route(a, a)) return false;
            } else {
                return false;
            }
        }
    }
    return true;
}

// output tiles of step k over the batch (unsliced), at the column tile width
// the grouped GEMM takes (128 when some output has more than 96 columns)
int grouped_bn(int n, const cc_plan *plans, size_t k) {
    int64_t nmax = 0;
    for (int i = 0; i < n; i++) nmax = std::max<int64_t>(nmax, plans[i]->plan.steps[k].tc.N);
    return nmax > 96 ? 128 : 64;
}
int64_t grouped_tiles(int n, const cc_plan *plans, size_t k) {
    const int bn = grouped_bn(n, plans, k);
    int64_t t = 0;
    for (int i = 0; i < n; i++) {
        const TcGemmDesc &d = plans[i]->plan.steps[k].tc;
        t += (d.M + 127) / 128 * ((d.N + bn - 1) / bn);
    }
    return t;
}

// device bytes of the grouped tables of a batch (an upper bound: every table
// 256-byte aligned)
int64_t grouped_bytes(int n, const cc_plan *plans) {
    const Plan &P0 = plans[0]->plan;
    int64_t b = 0;
    for (size_t k = 0; k < P0.steps.size(); k++) {
        if (P0.steps[k].kind == StepKind::ACCUM) {
            b += al((int64_t)n * (int64_t)sizeof(GroupedAccum));
            continue;
        }
        if (P0.steps[k].rows) {
            b += al((int64_t)n * (int64_t)sizeof(GroupedRows));
            continue;
        }
        b += 4 * al((int64_t)n * (int64_t)sizeof(GroupedSplit)) + al((int64_t)n * (int64_t)sizeof(GroupedGemm)) +
             al((int64_t)n * (int64_t)sizeof(GroupedReduce));
        const int64_t tiles = grouped_tiles(n, plans, k);
        for (int i = 0; i < n; i++) {
            const TcGemmDesc &t = plans[i]->plan.steps[k].tc;
            const int ns = grouped_kslices(t.M, t.N, t.Kp, tiles);
            if (ns > 1) b += al((int64_t)ns * t.M * t.N * 8);
        }
    }
    b += al((int64_t)n * (int64_t)sizeof(GroupedPost)) + al((int64_t)n * 4);
    for (int i = 0; i < n; i++) {
        const int64_t e = amp_count(1, plans[i]->plan.o, plans[i]->plan.v) + amp_count(2, plans[i]->plan.o, plans[i]->plan.v);
        b += al(3 * ((e + kPostChunk - 1) / kPostChunk) * 8);
    }
    return b;
}

struct BatchLayout {
    std::vector<int64_t> base, pw;      // per system: region start, plan workspace bytes
    std::vector<SolverLayout> L;
    int64_t tab = 0, scal = 0, used = 0, bytes = 0;
    bool grouped = false;
    int64_t grp = 0, grp_bytes = 0;     // grouped tables (when the plans allow it)
};

BatchLayout batch_layout(int n, const cc_plan *plans, int diis) {
    BatchLayout B;
    int64_t off = 0;
    for (int i = 0; i < n; i++) {
        B.base.push_back(off);
        const int64_t pw = al(plans[i]->plan.ws_bytes);
        B.pw.push_back(pw);
        B.L.push_back(solver_layout(plans[i]->plan, diis));
        off += pw + al(B.L.back().bytes);
    }
    B.tab = off; off += al((int64_t)n * (int64_t)sizeof(BatchSys));
    B.scal = off; off += al((int64_t)n * 8 * 8);
    B.used = off; off += al((int64_t)n * 4);
    B.grouped = batch_groupable(n, plans);
    if (B.grouped) {
        B.grp = off;
        B.grp_bytes = grouped_bytes(n, plans);
        off += B.grp_bytes;
    }
    B.bytes = off;
    return B;
}

// compact elementwise tables take the space sized for GroupedAccum tables
static_assert(sizeof(GroupedEw) <= sizeof(GroupedAccum), "grouped elementwise table size");

// one launch of a grouped residual evaluation
struct GroupedLaunch {
    int kind = 0;                 // 0 elementwise, 1 split, 2 GEMM, 3 K-slice reduction, 4 narrow GEMM,
                                  // 5 one-column narrow GEMM (GEMV), 6 long contiguous-K split,
                                  // 7 GEMV with X along the rows
    bool first_only = false;      // static sources / cached planes: the first evaluation only
    int64_t off = 0;              // table offset in the grouped region
    int n = 0;                    // entries
    int64_t total = 0;            // work items of all entries
    bool flag = false;            // elementwise: accumulate; split: lanes along K
    int mode = 0;                 // elementwise: 0 generic, 1 row path, 2 generic, four loads per lane,
                                  // 3 compact entries (GroupedEw)
    bool two = false;             // elementwise: products of two sources
    int nperm = 1;
    int bn = 64;
    GroupedGemmParams gp{};
};

struct GroupedBatch {
    std::vector<GroupedLaunch> launches;
    int64_t post_off = 0, post_total = 0, active_off = 0;
    int n = 0;
    int *err_flag = nullptr;
};

// The tables of every step (device pointers into the systems' workspaces),
// built on the host and copied into the grouped region once per call.
cc_status build_grouped(GroupedBatch &GB, int n, const cc_plan *plans, const cc_integrals *ints, const cc_amps *amps,
                        const std::vector<cc_resid> &R, char *W, const BatchLayout &BL, double *d_scal,
                        cudaStream_t s) {
    std::vector<unsigned char> img((size_t)BL.grp_bytes, 0);
    int64_t off = 0;
    auto put = [&](const void *src, int64_t bytes) {
        const int64_t at = off;
        std::memcpy(img.data() + at, src, (size_t)bytes);
        off += al(bytes);
        return at;
    };
    GB = GroupedBatch();
    GB.n = n;
    const Plan &P0 = plans[0]->plan;
    char *G = W + BL.grp;
    for (size_t k = 0; k < P0.steps.size(); k++) {
        const Step &s0 = P0.steps[k];
        if (s0.kind == StepKind::ACCUM) {
            std::vector<GroupedAccum> t(n);
            int64_t items = 0;
            bool rowp = true;
            int nperm = 1;
            for (int i = 0; i < n; i++) {
                const Step &st = plans[i]->plan.steps[k];
                char *w = W + BL.base[i];
                GroupedAccum &g = t[i];
                g.d = st.acc;
                prepare_grouped_accum(g);
                g.src = resolve(st.a, &ints[i], &amps[i], &R[i], w);
                g.src2 = st.acc.two_src ? resolve(st.b, &ints[i], &amps[i], &R[i], w) : nullptr;
                g.add = st.acc.has_add ? resolve(st.c, &ints[i], &amps[i], &R[i], w) : nullptr;
                g.out = resolve(st.out, &ints[i], &amps[i], &R[i], w);
                if (!g.src || !g.out || (st.acc.two_src && !g.src2) || (st.acc.has_add && !g.add))
                    return fail(CC_ERR_INVALID_ARG, "grouped batch: an operand buffer is missing");
                g.sys = i;
                rowp = rowp && g.row_path;
                nperm = std::max(nperm, g.d.nperm);
            }
            // one or two terms: the generic path with four elements' loads in flight
            // per lane (short rows leave the row path's lanes idle); else the row
            // path when it holds for every system, else the plain generic one
            bool small = true;            // 32-bit element indices
            for (int i = 0; i < n; i++) small = small && t[i].d.total < ((int64_t)1 << 31);
            // every entry in compact form (32-bit running offsets): that kernel
            std::vector<GroupedEw> te(n);
            bool compact = nperm <= kEwTerms && (!s0.acc.two_src || nperm <= 2);
            for (int i = 0; i < n && compact; i++) compact = grouped_ew_from(t[i], te[i]);
            if (compact) {
                for (int i = 0; i < n; i++) {
                    te[i].item0 = items;
                    items += (te[i].total + kEwRun - 1) / kEwRun;
                }
                GroupedLaunch L;
                L.kind = 0;
                L.first_only = s0.static_src;
                L.n = n;
                L.total = items;
                L.flag = beta_case(s0.acc.beta) == 1;
                L.mode = 3;
                L.nperm = nperm;
                L.two = s0.acc.two_src != 0;
                L.off = put(te.data(), (int64_t)sizeof(GroupedEw) * n);
                GB.launches.push_back(L);
                continue;
            }
            const int mode = nperm <= 2 && small ? 2 : rowp ? 1 : 0;
            for (int i = 0; i < n; i++) {
                t[i].item0 = items;
                items += grouped_accum_items(t[i], mode);
            }
            GroupedLaunch L;
            L.kind = 0;
            L.first_only = s0.static_src;
            L.n = n;
            L.total = items;
            L.flag = beta_case(s0.acc.beta) == 1;
            L.mode = mode;
            L.nperm = nperm;
            L.two = s0.acc.two_src != 0;
            L.off = put(t.data(), (int64_t)sizeof(GroupedAccum) * n);
            GB.launches.push_back(L);
            continue;
        }
        if (s0.rows) {
            // the narrow kernel: operands read in place, no splits
            std::vector<GroupedRows> t(n);
            int nc_max = 1;
            for (int i = 0; i < n; i++) {
                const Step &st = plans[i]->plan.steps[k];
                char *w = W + BL.base[i];
                GroupedRows &g = t[i];
                g.d = st.rg;
                prepare_grouped_rows(g);
                g.X = resolve(st.a, &ints[i], &amps[i], &R[i], w);
                g.Y = resolve(st.b, &ints[i], &amps[i], &R[i], w);
                g.C = resolve(st.out, &ints[i], &amps[i], &R[i], w);
                if (!g.X || !g.Y || !g.C || g.d.R > 0xffffffffLL)
                    return fail(CC_ERR_INVALID_ARG, "grouped batch: a narrow GEMM operand is missing");
                g.sys = i;
                nc_max = std::max(nc_max, g.d.nc);
            }
            // one column in every system: the warp-per-row GEMV
            // (lanes along K), or with X along the rows and a long K (lanes along rows)
            bool gemv = true, gemvr = true;
            for (int i = 0; i < n && gemv; i++) gemv = grouped_gemv_ok(t[i]);
            for (int i = 0; i < n && gemvr; i++) gemvr = !gemv && grouped_gemvr_ok(t[i]);
            const int nc = grouped_rows_nc(nc_max);
            int64_t items = 0;
            for (int i = 0; i < n; i++) {
                t[i].item0 = items;
                items += gemv ? grouped_gemv_items(t[i]) : gemvr ? grouped_gemvr_items(t[i]) : grouped_rows_items(t[i], nc);
            }
            GroupedLaunch L;
            L.kind = gemv ? 5 : gemvr ? 7 : 4;
            L.n = n;
            L.total = items;
            L.bn = nc;
            L.flag = s0.gemm.f32 != 0;
            L.off = put(t.data(), (int64_t)sizeof(GroupedRows) * n);
            GB.launches.push_back(L);
            continue;
        }
        // operand splits: A then B, the entries of each lane orientation in one launch
        for (int side = 0; side < 2; side++) {
            if (side == 0 ? s0.skip_a : s0.skip_b) continue;
            // mode 0 / 1: tiles with lanes along rows / K; mode 2: long contiguous K
            // (vector loads, (row, span) items)
            for (int mode = 0; mode < 3; mode++) {
                std::vector<GroupedSplit> t;
                int64_t tiles = 0;
                for (int i = 0; i < n; i++) {
                    const Step &st = plans[i]->plan.steps[k];
                    const SplitDesc &d = side == 0 ? st.split_a : st.split_b;
                    char *w = W + BL.base[i];
                    GroupedSplit g{};
                    g.d = d;
                    g.x = resolve(side == 0 ? st.a : st.b, &ints[i], &amps[i], &R[i], w);
                    g.planes = w + (side == 0 ? st.planes_a_off : st.planes_b_off);
                    if (!g.x) return fail(CC_ERR_INVALID_ARG, "grouped batch: an operand buffer is missing");
                    // the (row, span) items where the vector loads apply, or where the
                    // operand has fewer rows than a 64-row tile
                    const int vk = grouped_split_vec_ok(d, g.x);
                    const bool vec = vk == 2 || (vk == 1 && d.R < 64);
                    if (vec ? mode != 2 : (int)split_lanes_along_k(d) != mode) continue;
                    const int64_t kcols = d.kend ? d.kend : d.Kp;
                    g.rtiles = vec ? (uint32_t)(vk == 2) : (uint32_t)((d.Rp + 63) / 64);
                    g.tile0 = tiles;
                    g.sys = i;
                    tiles += vec ? grouped_split_vec_items(d) : (int64_t)g.rtiles * ((kcols + 63) / 64);
                    t.push_back(g);
                }
                if (t.empty()) continue;
                GroupedLaunch L;
                L.kind = mode == 2 ? 6 : 1;
                L.first_only = side == 0 ? s0.a_static : s0.b_static;
                L.n = (int)t.size();
                L.total = tiles;
                L.flag = mode == 1;
                L.off = put(t.data(), (int64_t)sizeof(GroupedSplit) * (int64_t)t.size());
                GB.launches.push_back(L);
            }
        }
        // the GEMMs: 128-wide column tiles when some output has more than 96 columns
        const int bn = grouped_bn(n, plans, k);
        const int64_t tiles_all = grouped_tiles(n, plans, k);
        std::vector<GroupedGemm> t(n);
        std::vector<GroupedReduce> red;
        int64_t tiles = 0, ritems = 0;
        for (int i = 0; i < n; i++) {
            const Step &st = plans[i]->plan.steps[k];
            char *w = W + BL.base[i];
            double *C = resolve(st.out, &ints[i], &amps[i], &R[i], w);
            // long K, small output: K slices into partials (after the tables), reduced in order
            const int ns = grouped_kslices(st.tc.M, st.tc.N, st.tc.Kp, tiles_all);
            double *P = nullptr;
            if (ns > 1) {
                P = (double *)(G + off);
                off += al((int64_t)ns * st.tc.M * st.tc.N * 8);
            }
            if (!C || !grouped_gemm_entry(t[i], st.tc, w + st.planes_a_off, w + st.planes_b_off, C, bn, ns, P))
                return fail(CC_ERR_CUDA, "grouped batch: a GEMM entry could not be encoded");
            t[i].tile0 = tiles;
            t[i].sys = i;
            tiles += (t[i].M + 127) / 128 * t[i].n_tiles * t[i].nslices;
            if (t[i].nslices > 1) {
                GroupedReduce r{};
                r.M = t[i].M;
                r.N = t[i].N;
                r.nslices = t[i].nslices;
                r.P = P;
                r.cm = st.tc.cm;
                r.cn = st.tc.cn;
                r.as = make_scale(st.tc.alpha);
                r.bcase = beta_case(st.tc.beta) != 0;
                r.C = C;
                r.item0 = ritems;
                r.sys = i;
                ritems += (r.M * r.N + 255) / 256;
                red.push_back(r);
            }
        }
        GroupedLaunch L;
        L.kind = 2;
        L.n = n;
        L.total = tiles;
        L.bn = bn;
        L.gp.nprod = s0.tc.nprod;
        for (int q = 0; q < s0.tc.nprod; q++) {
            L.gp.prod_a[q] = s0.tc.prod_a[q];
            L.gp.prod_b[q] = s0.tc.prod_b[q];
        }
        L.off = put(t.data(), (int64_t)sizeof(GroupedGemm) * n);
        GB.launches.push_back(L);
        if (!red.empty()) {
            GroupedLaunch Q;
            Q.kind = 3;
            Q.n = (int)red.size();
            Q.total = ritems;
            Q.off = put(red.data(), (int64_t)sizeof(GroupedReduce) * (int64_t)red.size());
            GB.launches.push_back(Q);
        }
    }
    // the denominator / energy / norm pass and its partials
    {
        std::vector<GroupedPost> t(n);
        std::vector<int64_t> part_at(n);
        int64_t items = 0;
        for (int i = 0; i < n; i++) {
            const Plan &P = plans[i]->plan;
            GroupedPost &g = t[i];
            g.o = P.o;
            g.v = P.v;
            g.fo = ints[i].f_occ;
            g.fv = ints[i].f_vir;
            g.t1 = (const double *)amps[i].t1;
            g.t2 = (const double *)amps[i].t2;
            g.oovv = (const double *)ints[i].oovv;
            g.r1 = (double *)R[i].r1;
            g.r2 = (double *)R[i].r2;
            if (!g.fo || !g.fv || !g.t1 || !g.t2 || !g.oovv || !g.r1 || !g.r2)
                return fail(CC_ERR_INVALID_ARG, "grouped batch: a solver buffer is missing");
            g.scal = d_scal + 8 * i;
            g.chunks = (amp_count(1, P.o, P.v) + amp_count(2, P.o, P.v) + kPostChunk - 1) / kPostChunk;
            g.item0 = items;
            g.sys = i;
            items += g.chunks;
        }
        // partials after the tables
        GB.post_total = items;
        const int64_t post_at = off;
        off += al((int64_t)sizeof(GroupedPost) * n);
        for (int i = 0; i < n; i++) {
            t[i].partials = (double *)(G + off);
            off += al(3 * t[i].chunks * 8);
        }
        std::memcpy(img.data() + post_at, t.data(), sizeof(GroupedPost) * n);
        GB.post_off = post_at;
    }
    GB.active_off = off;
    off += al((int64_t)n * 4);
    if (off > BL.grp_bytes) return fail(CC_ERR_WORKSPACE, "grouped batch tables exceed their region");
    GB.err_flag = (int *)(W + BL.base[0] + plans[0]->plan.flags_off);
    CC_CUDA(cudaMemcpyAsync(G, img.data(), (size_t)off, cudaMemcpyHostToDevice, s));
    CC_CUDA(cudaMemsetAsync(GB.err_flag, 0, sizeof(int), s));
    CC_CUDA(cudaStreamSynchronize(s));
    return CC_OK;
}

// one residual evaluation of the whole batch (grouped launches); the caller
// has set the active flags
cc_status grouped_residual(const GroupedBatch &GB, char *G, bool first, long long &launches, cudaStream_t s) {
    const int *active = (const int *)(G + GB.active_off);
    for (const GroupedLaunch &L : GB.launches) {
        if (L.first_only && !first) continue;
        if (L.kind == 0 && L.mode == 3)
            CC_CUDA(launch_grouped_ew((const GroupedEw *)(G + L.off), L.n, L.total, L.flag, L.nperm, L.two, active, s));
        else if (L.kind == 0)
            CC_CUDA(launch_grouped_accum((const GroupedAccum *)(G + L.off), L.n, L.total, L.flag, L.mode, L.nperm,
                                         L.two, active, s));
        else if (L.kind == 1)
            CC_CUDA(launch_grouped_split((const GroupedSplit *)(G + L.off), L.n, L.total, L.flag, active, s));
        else if (L.kind == 2)
            CC_CUDA(launch_grouped_gemm((const GroupedGemm *)(G + L.off), L.n, L.total, L.bn, L.gp, active,
                                        GB.err_flag, s));
        else if (L.kind == 4)
            CC_CUDA(launch_grouped_rows((const GroupedRows *)(G + L.off), L.n, L.total, L.bn, L.flag, active, s));
        else if (L.kind == 5)
            CC_CUDA(launch_grouped_gemv((const GroupedRows *)(G + L.off), L.n, L.total, L.flag, active, s));
        else if (L.kind == 7)
            CC_CUDA(launch_grouped_gemvr((const GroupedRows *)(G + L.off), L.n, L.total, L.flag, active, s));
        else if (L.kind == 6)
            CC_CUDA(launch_grouped_split_vec((const GroupedSplit *)(G + L.off), L.n, L.total, active, s));
        else
            CC_CUDA(launch_grouped_reduce((const GroupedReduce *)(G + L.off), L.n, L.total, active, s));
        launches++;
    }
    CC_CUDA(launch_grouped_post((const GroupedPost *)(G + GB.post_off), GB.n, GB.post_total, active, s));
    launches += 2;
    return CC_OK;
}

// host resources of one batched call, released on every exit path
struct BatchHost {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t main = nullptr;
    cudaEvent_t sync_ev = nullptr;
    BatchSys *tab = nullptr;
    double *scal = nullptr;
    int *used = nullptr, *flags = nullptr, *active = nullptr;
    ~BatchHost() {
        if (active) cudaFreeHost(active);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : ev) cudaEventDestroy(e);
        for (auto x : st) cudaStreamDestroy(x);
        if (sync_ev) cudaEventDestroy(sync_ev);
        if (main) cudaStreamDestroy(main);
        if (tab) cudaFreeHost(tab);
        if (scal) cudaFreeHost(scal);
        if (used) cudaFreeHost(used);
        if (flags) cudaFreeHost(flags);
    }
};

}  // namespace

extern "C" {

cc_status cc_solve_batched_workspace_bytes(int n, const cc_plan *plans, const cc_solve_opts *opts, size_t *bytes) {
    if (n < 1 || !plans || !bytes) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < n; i++)
        if (!plans[i]) return fail(CC_ERR_INVALID_ARG, "NULL plan in the batch");
    const int diis = opts ? opts->diis_max : 8;
    if (diis < 0 || diis > 16) return fail(CC_ERR_INVALID_ARG, "diis_max must be in [0, 16]");
    *bytes = (size_t)batch_layout(n, plans, diis).bytes;
    return CC_OK;
}

cc_status cc_solve_batched(int n, const cc_plan *plans, const cc_integrals *ints, cc_amps *amps,
                           const cc_solve_opts *opts, cc_solve_report *reports, void *ws, size_t ws_bytes,
                           void *stream) {
    if (n < 1 || !plans || !ints || !amps) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    cc_solve_opts o{};
    o.struct_size = sizeof(o);
    o.max_iter = 100;
    o.tol = 1e-8;
    o.diis_max = 8;
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.diis_max < 0 || o.diis_max > 16) return fail(CC_ERR_INVALID_ARG, "bad solve options");
    if (o.refine_plan) return fail(CC_ERR_UNSUPPORTED, "cc_solve_batched takes no refine plan");
    if (o.resume) return fail(CC_ERR_UNSUPPORTED, "cc_solve_batched does not resume");
    for (int i = 0; i < n; i++) {
        if (!plans[i]) return fail(CC_ERR_INVALID_ARG, "NULL plan in the batch");
        if (!plans[i]->plan.res_used[2]) return fail(CC_ERR_INVALID_ARG, "every plan must write R2");
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return fail(CC_ERR_INVALID_ARG, "each system needs a plan of its own");
    }
    const BatchLayout BL = batch_layout(n, plans, o.diis_max);
    if ((int64_t)ws_bytes < BL.bytes || !ws || !aligned256(ws))
        return fail(CC_ERR_WORKSPACE, "batched workspace too small: need " + std::to_string(BL.bytes));
    char *W = (char *)ws;
    BatchHost H;
    // the work runs on a stream of its own (capturable even when the caller
    // passes the legacy default stream), ordered after and before the caller's
    cudaStream_t user = (cudaStream_t)stream;
    CC_CUDA(cudaStreamCreateWithFlags(&H.main, cudaStreamNonBlocking));
    CC_CUDA(cudaEventCreateWithFlags(&H.sync_ev, cudaEventDisableTiming));
    CC_CUDA(cudaEventRecord(H.sync_ev, user));
    CC_CUDA(cudaStreamWaitEvent(H.main, H.sync_ev, 0));
    cudaStream_t s = H.main;
    CC_CUDA(cudaMallocHost(&H.tab, sizeof(BatchSys) * n));
    CC_CUDA(cudaMallocHost(&H.scal, sizeof(double) * 8 * n));
    CC_CUDA(cudaMallocHost(&H.used, sizeof(int) * n));
    CC_CUDA(cudaMallocHost(&H.flags, sizeof(int) * n));
    BatchSys *d_tab = (BatchSys *)(W + BL.tab);
    double *d_scal = (double *)(W + BL.scal);
    int *d_used = (int *)(W + BL.used);
    CC_CUDA(cudaMemsetAsync(d_used, 0, sizeof(int) * n, s));
    CC_CUDA(cudaMemsetAsync(d_scal, 0, sizeof(double) * 8 * n, s));

    // per-system views
    std::vector<std::array<double *, 4>> r(n), t(n);
    std::vector<cc_resid> R(n);
    std::vector<SolverState> S(n);
    std::vector<int> state(n, 0);        // 0 active, 1 converged, 2 stopped (divergence)
    std::vector<double> last_e(n, NAN), last_ei(n, NAN), last_rn(n, NAN);
    std::vector<int> iters(n, 0);
    for (int i = 0; i < n; i++) {
        const Plan &P = plans[i]->plan;
        const SolverLayout &L = BL.L[i];
        char *sreg = W + BL.base[i] + BL.pw[i];
        t[i] = {nullptr, (double *)amps[i].t1, (double *)amps[i].t2, (double *)amps[i].t3};
        for (int l = 0; l < 4; l++) r[i][l] = nullptr;
        for (int l = 1; l <= 3; l++)
            if (P.res_used[l]) {
                r[i][l] = (double *)(sreg + L.r_off[l]);
                if (!t[i][l]) return fail(CC_ERR_INVALID_ARG, "amplitude buffer missing for a residual the list writes");
            }
        R[i] = cc_resid{r[i][1], r[i][2], r[i][3]};
        plans[i]->cache_filled = false;
        // 1/D of every amplitude (the Jacobi steps multiply by it, as cc_solve does)
        double *dinv = (double *)(sreg + L.dinv);
        int64_t doff = 0;
        for (int l = 1; l <= 3; l++) {
            if (!r[i][l]) continue;
            CC_CUDA(launch_inv_denominators(l, P.o, P.v, ints[i].f_occ, ints[i].f_vir, dinv + doff,
                                            P.dtype == CC_C128, s));
            doff += L.n[l];
        }
        if (reports) { reports[i].iterations = 0; reports[i].converged = 0; reports[i].switched_at = -1; }
    }
    g_err.clear();

    // grouped execution (plans with the same steps): tables built once per call
    GroupedBatch GB;
    int *d_active = nullptr;
    if (BL.grouped) {
        cc_status gs = build_grouped(GB, n, plans, ints, amps, R, W, BL, d_scal, s);
        if (gs != CC_OK) return gs;
        d_active = (int *)(W + BL.grp + GB.active_off);
        CC_CUDA(cudaMallocHost(&H.active, sizeof(int) * n));
        for (int i = 0; i < n; i++) H.active[i] = 1;
        CC_CUDA(cudaMemcpyAsync(d_active, H.active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    }
    // the grouped residual of the batch + energy/norm into d_scal[i], read back
    auto grouped_phase = [&](bool first) -> cc_status {
        long long la = 0;
        cc_status gst = grouped_residual(GB, W + BL.grp, first, la, s);
        if (gst != CC_OK) return gst;
        plans[0]->launches += la;
        CC_CUDA(cudaMemcpyAsync(H.scal, d_scal, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaMemcpyAsync(H.used, d_used, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaMemcpyAsync(H.flags, GB.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        for (int i = 1; i < n; i++) H.flags[i] = 0;
        return CC_OK;
    };

    // residual phase of every system: run_residual + energy/norm into d_scal[i]
    auto residual_phase = [&](bool capture) -> cc_status {
        for (int i = 0; i < n; i++) {
            cudaStream_t si = capture ? H.st[i] : s;
            if (capture) CC_CUDA(cudaStreamWaitEvent(si, H.ev[0], 0));
            const Plan &P = plans[i]->plan;
            const SolverLayout &L = BL.L[i];
            char *sreg = W + BL.base[i] + BL.pw[i];
            cc_status st = run_residual(plans[i], &ints[i], &amps[i], &R[i], W + BL.base[i], (size_t)BL.pw[i], si,
                                        true);
            if (st != CC_OK) return st;
            double *rr[4] = {nullptr, r[i][1], r[i][2], r[i][3]};
            st = reduce_energy_norm(P, &ints[i], &amps[i], rr, L.n, (double *)(sreg + L.partials), d_scal + 8 * i, si);
            if (st != CC_OK) return st;
            plans[i]->launches += 2 + (rr[1] != nullptr) + (rr[2] != nullptr) + (rr[3] != nullptr);
            if (capture) {
                CC_CUDA(cudaEventRecord(H.ev[1 + i], si));
                CC_CUDA(cudaStreamWaitEvent(s, H.ev[1 + i], 0));
            }
        }
        CC_CUDA(cudaMemcpyAsync(H.scal, d_scal, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaMemcpyAsync(H.used, d_used, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        for (int i = 0; i < n; i++)
            CC_CUDA(cudaMemcpyAsync(H.flags + i, W + BL.base[i] + plans[i]->plan.flags_off, sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        return CC_OK;
    };

    // iteration 0 runs directly (it fills the static caches); later ones replay a graph
    cc_status st = BL.grouped ? grouped_phase(true) : residual_phase(false);
    if (st != CC_OK) return st;
    CC_CUDA(cudaStreamSynchronize(s));
    std::vector<long long> per_replay(n, 0);
    if (o.max_iter > 1 && BL.grouped) {
        const long long before = plans[0]->launches;
        CC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cc_status cst = grouped_phase(false);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        H.graph = g;
        if (cst != CC_OK) return cst;
        if (ce != cudaSuccess) return fail(CC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        CC_CUDA(cudaGraphInstantiate(&H.exec, H.graph, 0));
        per_replay[0] = plans[0]->launches - before;
        plans[0]->launches = before;
    } else if (o.max_iter > 1) {
        H.st.resize(n);
        for (int i = 0; i < n; i++) CC_CUDA(cudaStreamCreateWithFlags(&H.st[i], cudaStreamNonBlocking));
        H.ev.resize(n + 1);
        for (int i = 0; i <= n; i++) CC_CUDA(cudaEventCreateWithFlags(&H.ev[i], cudaEventDisableTiming));
        std::vector<long long> before(n);
        for (int i = 0; i < n; i++) before[i] = plans[i]->launches;
        CC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cc_status cst = cudaEventRecord(H.ev[0], s) == cudaSuccess ? residual_phase(true)
                                                                   : fail(CC_ERR_CUDA, "event record in capture");
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        H.graph = g;
        if (cst != CC_OK) return cst;
        if (ce != cudaSuccess) return fail(CC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        CC_CUDA(cudaGraphInstantiate(&H.exec, H.graph, 0));
        for (int i = 0; i < n; i++) {
            per_replay[i] = plans[i]->launches - before[i];
            plans[i]->launches = before[i];
        }
    }

    cc_status result = CC_OK;
    int k = 0;
    for (k = 0; k < o.max_iter; k++) {
        if (k > 0) {
            if (BL.grouped) {
                // converged (or stopped) systems are skipped inside the grouped launches
                for (int i = 0; i < n; i++) H.active[i] = state[i] == 0;
                CC_CUDA(cudaMemcpyAsync(d_active, H.active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
            }
            CC_CUDA(cudaGraphLaunch(H.exec, s));
            CC_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i < n; i++) plans[i]->launches += per_replay[i];
        }
        int nact = 0;
        for (int i = 0; i < n; i++) {
            BatchSys &b = H.tab[i];
            std::memset(&b, 0, sizeof(b));
            if (state[i] != 0) continue;
            const Plan &P = plans[i]->plan;
            SolverState &Z = S[i];
            if (P.flops_mixed > 0 && H.flags[i] != 0)
                return fail(CC_ERR_TIMEOUT, "a bounded tensor-core pipeline wait expired (system " +
                                                std::to_string(i) + ")");
            if (Z.pending_m >= 2) {
                const int keep = H.used[i] == 0 ? 2 : H.used[i];
                while (Z.nstored > keep) {
                    for (int q = 0; q + 1 < Z.nstored; q++) Z.order[q] = Z.order[q + 1];
                    Z.nstored--;
                }
                Z.pending_m = 0;
            }
            double rr = 0.0;
            for (int l = 1, c = 2; l <= 3; l++)
                if (r[i][l]) rr += H.scal[8 * i + c++];
            const double e = H.scal[8 * i], rn = std::sqrt(rr);
            last_e[i] = e;
            last_ei[i] = H.scal[8 * i + 1];
            last_rn[i] = rn;
            if (reports && reports[i].energies) reports[i].energies[k] = e;
            if (reports && reports[i].energies_im) reports[i].energies_im[k] = H.scal[8 * i + 1];
            if (reports && reports[i].rnorms) reports[i].rnorms[k] = rn;
            iters[i] = k + 1;
            if (!std::isfinite(rn) || rn > 1e3 * Z.best) { state[i] = 2; continue; }
            if (rn < Z.best) Z.best = rn;
            if (o.tol > 0 && rn < o.tol) { state[i] = 1; continue; }
            // Jacobi step into a history slot (the same bookkeeping as cc_solve)
            int slot = 0;
            if (o.diis_max > 0 && Z.nstored == o.diis_max) {
                slot = Z.order[0];
                for (int q = 0; q + 1 < Z.nstored; q++) Z.order[q] = Z.order[q + 1];
                Z.nstored--;
            } else if (o.diis_max > 0) {
                for (;; slot++) {
                    bool busy = false;
                    for (int q = 0; q < Z.nstored; q++) busy |= Z.order[q] == slot;
                    if (!busy) break;
                }
            }
            if (o.diis_max > 0) Z.order[Z.nstored++] = slot;
            const SolverLayout &L = BL.L[i];
            char *sreg = W + BL.base[i] + BL.pw[i];
            b.active = 1;
            b.o = P.o;
            b.v = P.v;
            b.cplx = P.dtype == CC_C128;
            b.fo = ints[i].f_occ;
            b.fv = ints[i].f_vir;
            for (int l = 1; l <= 3; l++) {
                b.t[l] = r[i][l] ? t[i][l] : nullptr;
                b.r[l] = r[i][l];
                b.n[l] = r[i][l] ? L.n[l] : 0;
            }
            b.nx = L.nx;
            b.hx = (double *)(sreg + L.hist_x);
            b.he = (double *)(sreg + L.hist_e);
            b.slot = slot;
            b.nstored = o.diis_max > 0 ? Z.nstored : 0;
            for (int q = 0; q < 16; q++) b.order[q] = Z.order[q];
            b.gram = (double *)(sreg + L.gram);
            b.coef = (double *)(sreg + L.coef);
            b.used = d_used + i;
            b.partials = (double *)(sreg + L.partials);
            b.dinv = (const double *)(sreg + L.dinv);
            Z.pending_m = b.nstored;
            Z.iter++;
            nact++;
        }
        if (nact == 0) { k++; break; }
        CC_CUDA(cudaMemcpyAsync(d_tab, H.tab, sizeof(BatchSys) * n, cudaMemcpyHostToDevice, s));
        CC_CUDA(launch_batched_jacobi(d_tab, n, s));
        CC_CUDA(launch_batched_diis(d_tab, n, s));
        CC_CUDA(launch_batched_combine(d_tab, n, s));
        plans[0]->launches += 4;
    }
    CC_CUDA(cudaStreamSynchronize(s));
    CC_CUDA(cudaEventRecord(H.sync_ev, s));
    CC_CUDA(cudaStreamWaitEvent(user, H.sync_ev, 0));
    int nconv = 0;
    for (int i = 0; i < n; i++) {
        nconv += state[i] == 1;
        if (reports) {
            reports[i].iterations = iters[i];
            reports[i].converged = state[i] == 1;
            reports[i].energy = last_e[i];
            reports[i].energy_im = last_ei[i];
            reports[i].rnorm = last_rn[i];
        }
    }
    if (nconv < n) {
        result = CC_ERR_NOT_CONVERGED;
        g_err = std::to_string(n - nconv) + " of " + std::to_string(n) + " systems did not converge";
    }
    return result;
}

}  // extern "C"

extern "C" {

cc_status cc_build_vvvv_packed_workspace_bytes(int o, int v, int L, cc_dtype dtype, size_t *bytes) {
    if (o < 1 || v < 2 || L < 1 || !bytes) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    if (dtype != CC_F64) return fail(CC_ERR_UNSUPPORTED, "the packed vvvv block is real only");
    const int64_t v3 = (int64_t)v * v * v;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(v, ((int64_t)1 << 30) / (v3 * 8)));
    *bytes = (size_t)(al((int64_t)L * v * v * 8) + al(chunk * v3 * 8));
    return CC_OK;
}

cc_status cc_build_vvvv_packed(int o, int v, int L, cc_dtype dtype, const void *B, void *out, void *ws,
                               size_t ws_bytes, void *stream) {
    size_t need = 0;
    cc_status st = cc_build_vvvv_packed_workspace_bytes(o, v, L, dtype, &need);
    if (st != CC_OK) return st;
    if (!B || !out || !ws || ws_bytes < need || !aligned256(ws)) return fail(CC_ERR_WORKSPACE, "bad B, out or workspace");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = o + v, v2 = (int64_t)v * v, v3 = v2 * v;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(v, ((int64_t)1 << 30) / (v3 * 8)));
    double *Bvv = (double *)ws;                                   // [L][v][v]
    double *S = (double *)((char *)ws + al((int64_t)L * v2 * 8)); // [a - a0][b][e][f] of one chunk
    {
        AccumDesc d{};
        d.nd = 3;
        d.nperm = 1;
        d.ext[0] = L; d.ext[1] = v; d.ext[2] = v;
        d.ostr[0] = v2; d.ostr[1] = v; d.ostr[2] = 1;
        d.sstr[0][0] = n * n; d.sstr[0][1] = n; d.sstr[0][2] = 1;
        d.total = (int64_t)L * v2;
        d.sign[0] = 1.0;
        d.alpha = 1.0;
        CC_CUDA(launch_accum(d, (const double *)B + (int64_t)o * n + o, Bvv, s));
    }
    const int64_t P = (int64_t)v * (v - 1) / 2;
    auto start = [&](int64_t a) { return a * (2 * (int64_t)v - a - 1) / 2; };
    for (int64_t a0 = 0; a0 < v - 1; a0 += chunk) {
        const int64_t a1 = std::min<int64_t>(a0 + chunk, v - 1), ca = a1 - a0;
        // S[a][b][e][f] = sum_L Bvv[a][e] Bvv[b][f] - Bvv[a][f] Bvv[b][e] for a in [a0, a1)
        for (int term = 0; term < 2; term++) {
            GemmF64Desc g{};
            g.M = ca * v;            // rows (a, e) or (a, f)
            g.N = v2;                // cols (b, f) or (b, e)
            g.K = L;
            g.sAm = 1;
            g.sAk = v2;
            g.sBk = v2;
            g.sBn = 1;
            g.cm.nd = 2; g.cm.ext[0] = ca; g.cm.ext[1] = v; g.cm.str[0] = v3;
            g.cn.nd = 2; g.cn.ext[0] = v; g.cn.ext[1] = v; g.cn.str[0] = v2;
            g.cm.str[1] = term == 0 ? v : 1;     // e | f
            g.cn.str[1] = term == 0 ? 1 : v;     // f | e
            g.alpha = term == 0 ? 1.0 : -1.0;
            g.beta = term == 0 ? 0.0 : 1.0;
            g.splitk = 1;
            CC_CUDA(launch_gemm_f64(g, Bvv + a0 * v, Bvv, S, nullptr, s));
        }
        PackDesc pd{};
        pd.n1 = v;
        pd.n2 = v;
        pd.P1 = P;
        pd.P2 = P;
        pd.s0 = v3; pd.s1 = v2; pd.s2 = v; pd.s3 = 1;
        pd.scale = 1.0;
        pd.row0 = start(a0);
        pd.rows = start(a1) - start(a0);
        pd.pbase = a0;
        CC_CUDA(launch_pack_pairs(pd, S, (double *)out + pd.row0 * P, s));
    }
    return CC_OK;
}

cc_status cc_selftest_convert(const double *in, long long n, float *mine, float *ref) {
    if (!in || !mine || !ref || n < 0) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    CC_CUDA(launch_convert_selftest(in, n, mine, ref, nullptr));
    CC_CUDA(cudaDeviceSynchronize());
    return CC_OK;
}

cc_status cc_selftest_wait_timeout(long long budget_cycles) {
    if (budget_cycles < 1000 || budget_cycles > 4000000000LL)
        return fail(CC_ERR_INVALID_ARG, "budget_cycles must be in [1e3, 4e9]");
    int *d = nullptr, h = -1;
    CC_CUDA(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) e = launch_wait_selftest(budget_cycles, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    if (h == 1) return fail(CC_ERR_TIMEOUT, "the bounded wait gave up as designed");
    return fail(CC_ERR_CUDA, "the never-satisfied wait did not time out");
}

cc_status cc_integral_block_elems(int o, int v, size_t elems[6]) {
    if (o < 1 || v < 1 || !elems) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    for (int b = 0; b < 6; b++) {
        int64_t e[4];
        integral_block_dims(o, v, b, e);
        elems[b] = (size_t)(e[0] * e[1] * e[2] * e[3]);
    }
    return CC_OK;
}

cc_status cc_build_integrals_workspace_bytes(int o, int v, int L, cc_dtype dtype, size_t *bytes) {
    if (o < 1 || v < 1 || L < 1 || !bytes) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    if (dtype != CC_F64 && dtype != CC_C128) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    const int64_t n = o + v, esz = dtype == CC_C128 ? 16 : 8;
    *bytes = (size_t)(al((int64_t)L * n * n * esz) + 4 * kAlign);
    return CC_OK;
}

cc_status cc_build_integrals(int o, int v, int L, cc_dtype dtype, const void *B, void *oooo, void *ooov, void *oovv,
                             void *ovov, void *ovvv, void *vvvv, void *ws, size_t ws_bytes, void *stream) {
    size_t need = 0;
    cc_status st = cc_build_integrals_workspace_bytes(o, v, L, dtype, &need);
    if (st != CC_OK) return st;
    if (!B || !ws || ws_bytes < need || !aligned256(ws)) return fail(CC_ERR_WORKSPACE, "bad B or workspace");
    void *blocks[6] = {oooo, ooov, oovv, ovov, ovvv, vvvv};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = o + v;
    const int64_t ext[2] = {o, v}, base[2] = {0, o};
    const int cplx = dtype == CC_C128;
    const int64_t esz = cplx ? 16 : 8, ew = cplx ? 2 : 1;   // bytes and doubles per element
    // sub-blocks Bsub[x][y] = B[L][x-range][y-range], contiguous [L][X][Y]
    double *sub[2][2];
    int64_t off = 0;
    for (int x = 0; x < 2; x++)
        for (int y = 0; y < 2; y++) {
            sub[x][y] = (double *)((char *)ws + off);
            off += (int64_t)L * ext[x] * ext[y] * esz;
            AccumDesc d{};
            d.nd = 3;
            d.nperm = 1;
            d.ext[0] = L; d.ext[1] = ext[x]; d.ext[2] = ext[y];
            d.ostr[0] = ext[x] * ext[y]; d.ostr[1] = ext[y]; d.ostr[2] = 1;
            d.sstr[0][0] = n * n; d.sstr[0][1] = n; d.sstr[0][2] = 1;
            d.total = (int64_t)L * ext[x] * ext[y];
            d.sign[0] = 1.0;
            d.alpha = 1.0;
            d.beta = 0.0;
            d.cplx = cplx;
            CC_CUDA(launch_accum(d, (const double *)B + (base[x] * n + base[y]) * ew, sub[x][y], s));
        }
    static const char *nm[6] = {"oooo", "ooov", "oovv", "ovov", "ovvv", "vvvv"};
    for (int b = 0; b < 6; b++) {
        if (!blocks[b]) continue;
        int64_t e[4];
        integral_block_dims(o, v, b, e);
        int sp[4];
        for (int q = 0; q < 4; q++) sp[q] = nm[b][q] == 'o' ? 0 : 1;
        const int64_t str[4] = {e[1] * e[2] * e[3], e[2] * e[3], e[3], 1};
        // <pq||rs> = sum_L B_pr B_qs - sum_L B_ps B_qr  (rows: (p, r|s), columns: (q, s|r))
        for (int term = 0; term < 2; term++) {
            const int ri = term == 0 ? 2 : 3, si = term == 0 ? 3 : 2;
            GemmF64Desc g{};
            g.M = e[0] * e[ri];
            g.N = e[1] * e[si];
            g.K = L;
            g.sAm = 1;
            g.sAk = e[0] * e[ri];
            g.sBk = e[1] * e[si];
            g.sBn = 1;
            g.cm.nd = 2; g.cm.ext[0] = e[0]; g.cm.ext[1] = e[ri]; g.cm.str[0] = str[0]; g.cm.str[1] = str[ri];
            g.cn.nd = 2; g.cn.ext[0] = e[1]; g.cn.ext[1] = e[si]; g.cn.str[0] = str[1]; g.cn.str[1] = str[si];
            g.alpha = term == 0 ? 1.0 : -1.0;
            g.beta = term == 0 ? 0.0 : 1.0;
            g.splitk = 1;
            g.cplx = cplx;
            CC_CUDA(launch_gemm_f64(g, sub[sp[0]][sp[ri]], sub[sp[1]][sp[si]], (double *)blocks[b], nullptr, s));
        }
    }
    return CC_OK;
}

}  // extern "C"
