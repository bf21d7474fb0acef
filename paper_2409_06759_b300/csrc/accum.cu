// accum.cu -- the elementwise half of the TTGT residual (sm_103a): permuted
// copies, outer products with permutation operators, and the antisymmetrising
// epilogues out = beta * out + alpha * sum_p sign_p * src[sigma_p(idx)].
//
// These steps move whole amplitude-sized arrays (o^2 v^2 doubles) and do a
// few operations per element, so HBM bandwidth is their roofline.  Two rules
// follow from B300's shape: keep many independent loads in flight per thread
// (each kernel issues all of an element batch's loads before its arithmetic),
// and spend as few FP64 instructions per element as the sum itself needs --
// the FP64 pipe issues ~2 per clock per SM, so one FP64 instruction per
// element of a 64M-element array costs ~0.1 ms, the time HBM takes to move
// 700 MB.  Signs, alpha = +-2^k and beta in {0, 1} therefore cost integer
// operations or one add (scalar.cuh, fp_bits.cuh).
//
// Kernel choice (launch_accum), after merging dims that are contiguous in
// every operand:
//   antisym_pairs   out = alpha P(ij) P(ab) src (4 terms, same index order):
//                   each orbit {ijab, jiab, ijba, jiba} is read and written once
//   antisym_triple  the six-term antisymmetriser of a triple of dims (leading
//                   or innermost), one orbit read and written once
//   accum_rows      every term reads its sources with stride 0 or 1 along the
//                   output's innermost dim (copies, outer products T1 x T1,
//                   and a copy fused into the next step: out = add + ...)
//   accum_tiled     some term runs along another dim: 32 x 32 tiles through
//                   shared memory (TTGT transposes, P(..) gathers)
//   accum_kernel    anything else (odometer over the flat output index)
#include <cstdint>
#include <cuda_runtime.h>

#include "grouped.cuh"
#include "kernels.h"
#include "scalar.cuh"

namespace ccb {

// ------------------------------------------------------------ generic path
// Each warp owns a contiguous run of 32*kAccChunk output elements; lane l
// visits run_start + l + 32*j, so stores to a contiguous output coalesce.
// The multi-index is decomposed once per run and advanced as an odometer.
constexpr int kAccChunk = 8;

// the run of 32*kAccChunk output elements starting at r0, by one warp
template <typename T, bool ACC>
__device__ __forceinline__ void accum_run(const AccumDesc &d, const T *__restrict__ src, T *__restrict__ out,
                                          const T *__restrict__ src2, const T *__restrict__ add, int64_t r0,
                                          int lane) {
    {
        int64_t e = r0 + lane;
        if (e >= d.total) return;
        int dig[kMaxDims];
        {
            int64_t x = e;
            for (int k = d.nd - 1; k >= 0; k--) {
                dig[k] = (int)(x % d.ext[k]);
                x /= d.ext[k];
            }
        }
        for (int j = 0; j < kAccChunk && e < d.total; j++) {
            int64_t oo = 0;
            for (int k = 0; k < d.nd; k++) oo += dig[k] * d.ostr[k];
            T acc = zero<T>();
            for (int p = 0; p < d.nperm; p++) {
                int64_t so = 0;
                for (int k = 0; k < d.nd; k++) so += dig[k] * d.sstr[p][k];
                T x = cj(ld(src + so), d.conj_a);
                if (d.two_src) {
                    int64_t so2 = 0;
                    for (int k = 0; k < d.nd; k++) so2 += dig[k] * d.sstr2[p][k];
                    x = mul(x, cj(ld(src2 + so2), d.conj_b));
                }
                acc = signed_term(p == 0, (d.negmask >> p) & 1ull, x, acc);
            }
            T old = zero<T>();
            if (ACC) {
                if (d.has_add) {
                    int64_t ao = 0;
                    for (int k = 0; k < d.nd; k++) ao += dig[k] * d.astr[k];
                    old = add[ao];
                } else {
                    old = out[oo];
                }
            }
            out[oo] = finish<ACC>(d.as, acc, old);
            // advance by 32 elements (compare-and-subtract carries)
            e += 32;
            int carry = 32;
            for (int k = d.nd - 1; k >= 0 && carry; k--) {
                int t = dig[k] + carry;
                carry = 0;
                const int ex = (int)d.ext[k];
                while (t >= ex) { t -= ex; carry++; }
                dig[k] = t;
            }
        }
    }
}

template <typename T, bool ACC>
__global__ void __launch_bounds__(256) accum_kernel(const AccumDesc d, const T *__restrict__ src,
                                                    T *__restrict__ out, const T *__restrict__ src2,
                                                    const T *__restrict__ add) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t run = 32 * kAccChunk;
    for (int64_t r0 = warp * run; r0 < d.total; r0 += nwarps * run) accum_run<T, ACC>(d, src, out, src2, add, r0, lane);
}

// The generic path with the loads of four elements per lane in flight (one
// or two terms): a lane takes the flat elements r0 + lane + 32 j, j < 4,
// decomposes each once (32-bit divisions), issues every term's loads for all
// four, then sums and stores.  TWO: products of two sources.
template <bool ACC, int NP, bool TWO>
__device__ __forceinline__ void accum_run4(const AccumDesc &d, const double *__restrict__ src,
                                           double *__restrict__ out, const double *__restrict__ src2,
                                           const double *__restrict__ add, int64_t r0, int lane) {
    constexpr int J = 4;
    int64_t oo[J], ao[J], so[NP][J], so2[NP][J];
    bool ok[J];
#pragma unroll
    for (int j = 0; j < J; j++) {
        const int64_t e = r0 + lane + 32 * j;
        ok[j] = e < d.total;
        uint32_t x = ok[j] ? (uint32_t)e : 0u;
        oo[j] = ao[j] = 0;
#pragma unroll
        for (int p = 0; p < NP; p++) so[p][j] = so2[p][j] = 0;
#pragma unroll
        for (int k = kMaxDims - 1; k >= 0; k--) {
            if (k >= d.nd) continue;
            const uint32_t ex = (uint32_t)d.ext[k], q = x / ex, dg = x - q * ex;
            x = q;
            oo[j] += (int64_t)dg * d.ostr[k];
            if (ACC && d.has_add) ao[j] += (int64_t)dg * d.astr[k];
#pragma unroll
            for (int p = 0; p < NP; p++) {
                so[p][j] += (int64_t)dg * d.sstr[p][k];
                if (TWO) so2[p][j] += (int64_t)dg * d.sstr2[p][k];
            }
        }
    }
    double xs[NP][J], ys[NP][J], old[J];
#pragma unroll
    for (int p = 0; p < NP; p++)
#pragma unroll
        for (int j = 0; j < J; j++) {
            const bool on = ok[j] && p < d.nperm;
            xs[p][j] = on ? __ldg(src + so[p][j]) : 0.0;
            ys[p][j] = (TWO && on) ? __ldg(src2 + so2[p][j]) : 0.0;
        }
#pragma unroll
    for (int j = 0; j < J; j++) old[j] = (ACC && ok[j]) ? (d.has_add ? add[ao[j]] : out[oo[j]]) : 0.0;
    // accumulating products start from the old value and add each term with
    // one FMA, the sign and alpha (+-2^k) riding on a factor: nterms FP64
    // operations per element instead of 2 nterms
    if (TWO && ACC && !d.as.general) {
        const bool fold = !(d.as.kexp == 0 && d.as.sflip == 0);
#pragma unroll
        for (int j = 0; j < J; j++) {
            if (!ok[j]) continue;
            double acc = old[j];
#pragma unroll
            for (int p = 0; p < NP; p++) {
                if (p >= d.nperm) break;
                double sa = ((d.negmask >> p) & 1ull) ? neg(xs[p][j]) : xs[p][j];
                if (fold) sa = scale_f64(sa, d.as);
                acc = fma(sa, ys[p][j], acc);
            }
            out[oo[j]] = acc;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < J; j++) {
        if (!ok[j]) continue;
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p < NP; p++) {
            if (p >= d.nperm) break;
            const double t = TWO ? xs[p][j] * ys[p][j] : xs[p][j];
            acc = signed_term(p == 0, (d.negmask >> p) & 1ull, t, acc);
        }
        out[oo[j]] = finish<ACC>(d.as, acc, old[j]);
    }
}

template <bool ACC, int NP, bool TWO>
__global__ void __launch_bounds__(256) grouped_accum4_kernel(const GroupedAccum *__restrict__ tab, int n, int64_t total,
                                                             const int *__restrict__ active) {
    const int lane = threadIdx.x & 31;
    const WorkRange wr = work_range(total, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                    (int64_t)gridDim.x * (blockDim.x >> 5));
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedAccum> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedAccum &e = tab[walk.at(it)];
        if (!active[e.sys]) { it = walk.next - 1; continue; }   // the rest of a converged system
        accum_run4<ACC, NP, TWO>(e.d, e.src, e.out, e.src2, e.add, (it - e.item0) * 128, lane);
    }
}

// The grouped form (real): entry e's runs are the work items [e.item0,
// e.item0 + ceil(total / run)); each warp takes a contiguous range of items
// (grouped.cuh).
template <bool ACC>
__global__ void __launch_bounds__(256) grouped_accum_kernel(const GroupedAccum *__restrict__ tab, int n, int64_t total,
                                                            const int *__restrict__ active) {
    const int lane = threadIdx.x & 31;
    const WorkRange wr = work_range(total, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                    (int64_t)gridDim.x * (blockDim.x >> 5));
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedAccum> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedAccum &e = tab[walk.at(it)];
        if (!active[e.sys]) { it = walk.next - 1; continue; }
        accum_run<double, ACC>(e.d, e.src, e.out, e.src2, e.add, (it - e.item0) * (32 * kAccChunk), lane);
    }
}

// ------------------------------------------------------ grouped, compact
// The grouped elementwise pass on compact entries (GroupedEw): a warp's run
// is kEwRun consecutive output elements, lane l taking r0 + l + 32 j.  A lane
// decomposes its first element once and then steps its digits by 32 with
// carries, moving each operand's 32-bit offset by the strides it crosses, so an
// element costs a few integer adds instead of a mixed-radix decomposition.
// Four elements' loads are issued before their arithmetic.
template <int NP, bool TWO> struct EwLane {
    int dig[kEwDims];
    uint32_t oo, ao, so[NP], so2[NP];
};

template <int NP, bool TWO, bool ACC>
__device__ __forceinline__ void ew_step32(const GroupedEw &d, EwLane<NP, TWO> &L) {
    const int k0 = d.nd - 1;
#pragma unroll
    for (int k = 0; k < kEwDims; k++)            // static indices keep the digits in registers
        if (k == k0) L.dig[k] += 32;
    // the 32-element step of the innermost digit (deltas precomputed on the host)
    L.oo += (uint32_t)d.wo[0];
    if (ACC && d.has_add) L.ao += (uint32_t)d.wa[0];
#pragma unroll
    for (int p = 0; p < NP; p++) {
        L.so[p] += (uint32_t)d.ws[p][0];
        if (TWO) L.so2[p] += (uint32_t)d.ws2[p][0];
    }
    // carries from the innermost digit outwards (no early exit: the digits stay
    // in registers); each wrap adds its precomputed offset changes
    bool carry = true;
#pragma unroll
    for (int k = kEwDims - 1; k > 0; k--) {
        if (k > k0 || !carry) continue;
        carry = L.dig[k] >= d.ext[k];
        if (!carry) continue;
        do {                                       // wrap digit k into digit k - 1
            L.dig[k] -= d.ext[k];
            L.dig[k - 1]++;
            L.oo += (uint32_t)d.wo[k];
            if (ACC && d.has_add) L.ao += (uint32_t)d.wa[k];
#pragma unroll
            for (int p = 0; p < NP; p++) {
                L.so[p] += (uint32_t)d.ws[p][k];
                if (TWO) L.so2[p] += (uint32_t)d.ws2[p][k];
            }
        } while (L.dig[k] >= d.ext[k]);
    }
}

template <bool ACC, int NP, bool TWO>
__device__ __forceinline__ void ew_run(const GroupedEw &d, int64_t r0, int lane) {
    constexpr int J = 4;
    uint32_t e = (uint32_t)r0 + (uint32_t)lane;
    if (e >= d.total) return;
    EwLane<NP, TWO> L;
    {
        uint32_t x = e;
        L.oo = L.ao = 0;
#pragma unroll
        for (int p = 0; p < NP; p++) L.so[p] = L.so2[p] = 0;
#pragma unroll
        for (int k = kEwDims - 1; k >= 0; k--) {
            L.dig[k] = 0;
            if (k >= d.nd) continue;
            const uint32_t ex = (uint32_t)d.ext[k], q = x / ex, dg = x - q * ex;
            x = q;
            L.dig[k] = (int)dg;
            L.oo += dg * (uint32_t)d.ostr[k];
            if (ACC && d.has_add) L.ao += dg * (uint32_t)d.astr[k];
#pragma unroll
            for (int p = 0; p < NP; p++) {
                L.so[p] += dg * (uint32_t)d.sstr[p][k];
                if (TWO) L.so2[p] += dg * (uint32_t)d.sstr2[p][k];
            }
        }
    }
    const uint32_t end = (uint32_t)min((int64_t)d.total, r0 + kEwRun);
    const bool chain = TWO && ACC && !d.as.general;
    const bool fold = chain && !(d.as.kexp == 0 && d.as.sflip == 0);
    for (int b = 0; b < (int)(kEwRun / (32 * J)); b++) {
        uint32_t oo[J], ao[J], so[NP][J], so2[NP][J];
        bool ok[J];
#pragma unroll
        for (int j = 0; j < J; j++) {
            ok[j] = e < end;
            oo[j] = L.oo;
            ao[j] = L.ao;
#pragma unroll
            for (int p = 0; p < NP; p++) {
                so[p][j] = L.so[p];
                so2[p][j] = L.so2[p];
            }
            e += 32;
            if (e < end) ew_step32<NP, TWO, ACC>(d, L);
        }
        double xs[NP][J], ys[NP][J], old[J];
#pragma unroll
        for (int p = 0; p < NP; p++)
#pragma unroll
            for (int j = 0; j < J; j++) {
                const bool on = ok[j] && p < d.nterms;
                xs[p][j] = on ? __ldg(d.src + so[p][j]) : 0.0;
                ys[p][j] = (TWO && on) ? __ldg(d.src2 + so2[p][j]) : 0.0;
            }
#pragma unroll
        for (int j = 0; j < J; j++) old[j] = (ACC && ok[j]) ? (d.has_add ? d.add[ao[j]] : d.out[oo[j]]) : 0.0;
#pragma unroll
        for (int j = 0; j < J; j++) {
            if (!ok[j]) continue;
            double acc;
            if (chain) {
                // start from the old value, one FMA per term, sign and alpha = +-2^k on a factor
                acc = old[j];
#pragma unroll
                for (int p = 0; p < NP; p++) {
                    if (p >= d.nterms) break;
                    double sa = ((d.negmask >> p) & 1ull) ? neg(xs[p][j]) : xs[p][j];
                    if (fold) sa = scale_f64(sa, d.as);
                    acc = fma(sa, ys[p][j], acc);
                }
            } else {
                acc = 0.0;
#pragma unroll
                for (int p = 0; p < NP; p++) {
                    if (p >= d.nterms) break;
                    const double t = TWO ? xs[p][j] * ys[p][j] : xs[p][j];
                    acc = signed_term(p == 0, (d.negmask >> p) & 1ull, t, acc);
                }
                acc = finish<ACC>(d.as, acc, old[j]);
            }
            d.out[oo[j]] = acc;
        }
        if (e >= end) break;
    }
}

template <bool ACC, int NP, bool TWO>
__global__ void __launch_bounds__(256, 3) grouped_ew_kernel(const GroupedEw *__restrict__ tab, int n, int64_t total,
                                                         const int *__restrict__ active) {
    // each warp keeps its current entry in shared memory: the lanes re-read its
    // fields at every step, and shared loads return sooner than L1 hits
    static_assert(sizeof(GroupedEw) % 16 == 0, "entry staging");
    __shared__ GroupedEw sd[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WorkRange wr = work_range(total, (int64_t)blockIdx.x * (blockDim.x >> 5) + warp,
                                    (int64_t)gridDim.x * (blockDim.x >> 5));
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedEw> walk(tab, n, wr.begin);
    int staged = -1;
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const int ei = walk.at(it);
        if (!active[tab[ei].sys]) { it = walk.next - 1; continue; }
        if (ei != staged) {
            __syncwarp();                        // the lanes are done with the previous entry
            const int4 *src4 = reinterpret_cast<const int4 *>(tab + ei);
            int4 *dst4 = reinterpret_cast<int4 *>(&sd[warp]);
            for (int q = lane; q < (int)(sizeof(GroupedEw) / 16); q += 32) dst4[q] = src4[q];
            __syncwarp();
            staged = ei;
        }
        const GroupedEw &e = sd[warp];
        ew_run<ACC, NP, TWO>(e, (it - e.item0) * kEwRun, lane);
    }
}

// --------------------------------------------------------------- row path
// Work item = (chunk of rch consecutive output rows, block of 32*kRowU
// columns of the innermost dim d0 = nd-1).  A warp decomposes the chunk's
// first row once (32-bit divisions; rows < 2^32) and then steps the row
// digits as an odometer, keeping each term's row offsets in registers; lane l
// handles columns cb + l + 32u, u < U, with every load of the batch issued
// before the arithmetic.  NP: the term count rounded up (1, 2, 4, 8).  U: 8
// columns per lane for one-source terms, 4 for products (their operand pairs
// would otherwise cost the occupancy that hides the loads' latency).
template <bool TWO> __host__ __device__ constexpr int rows_u() { return TWO ? 4 : 8; }

// one work item `it` of the row path, by one warp
template <typename T, int NP, bool TWO, bool ACC>
__device__ __forceinline__ void accum_rows_item(const AccumDesc &d, const T *__restrict__ src,
                                                const T *__restrict__ src2, T *__restrict__ out,
                                                const T *__restrict__ add, uint32_t rows, int rch, uint32_t ncb,
                                                uint64_t it, int lane) {
    constexpr int kRowU = rows_u<TWO>();
    const int d0 = d.nd - 1;
    const int E0 = (int)d.ext[d0];                     // < 2^31 (launch_accum checks)
    // along the innermost dim every source (and the addend) has stride 0 or 1
    // and the output stride 1: a column's offset is its index or 0
    bool u0[NP], u02[NP];
#pragma unroll
    for (int p = 0; p < NP; p++) {
        u0[p] = p < d.nperm && d.sstr[p][d0] != 0;
        u02[p] = TWO && p < d.nperm && d.sstr2[p][d0] != 0;
    }
    const bool ua = d.has_add && d.astr[d0] != 0;
    // accumulating outer products start from the old value and add each term
    // with one FMA, alpha (+-2^k) riding on a factor: nterms FP64 operations per
    // element instead of nterms + 1
    const bool chain = TWO && ACC && !d.as.general;
    const bool fold = chain && !(d.as.kexp == 0 && d.as.sflip == 0);
    {
        const uint32_t chunk = (uint32_t)(it / ncb);
        const int cb = (int)(it - (uint64_t)chunk * ncb) * (32 * kRowU);
        const uint32_t r0 = chunk * (uint32_t)rch;
        // row digits of r0 over dims d0-1 .. 0, unrolled so they live in registers
        uint32_t dig[kMaxDims - 1];
        int64_t obase = 0, abase = 0, sb[NP], sb2[NP];
#pragma unroll
        for (int p = 0; p < NP; p++) sb[p] = sb2[p] = 0;
        uint32_t x = r0;
#pragma unroll
        for (int k = kMaxDims - 2; k >= 0; k--) {
            dig[k] = 0;
            if (k < d0) {
                const uint32_t e = (uint32_t)d.ext[k], q = x / e;
                dig[k] = x - q * e;
                x = q;
                obase += (int64_t)dig[k] * d.ostr[k];
                if (ACC && d.has_add) abase += (int64_t)dig[k] * d.astr[k];
#pragma unroll
                for (int p = 0; p < NP; p++)
                    if (p < d.nperm) {
                        sb[p] += (int64_t)dig[k] * d.sstr[p][k];
                        if (TWO) sb2[p] += (int64_t)dig[k] * d.sstr2[p][k];
                    }
            }
        }
        const int nr = rows - r0 < (uint32_t)rch ? (int)(rows - r0) : rch;
        for (int rr = 0; rr < nr; rr++) {
            // the row's base pointers
            T *orow = out + obase;
            const T *irow = d.has_add ? add + abase : orow;
            T old[kRowU], acc[kRowU];
#pragma unroll
            for (int u = 0; u < kRowU; u++) {
                const int i = cb + lane + 32 * u;
                old[u] = (ACC && i < E0) ? irow[d.has_add ? (ua ? i : 0) : i] : zero<T>();
                acc[u] = old[u];
            }
#pragma unroll
            for (int p = 0; p < NP; p++) {
                if (p >= d.nperm) break;
                const bool ng = (d.negmask >> p) & 1ull;
                const T *arow = src + sb[p];
                const T *brow = TWO ? src2 + sb2[p] : nullptr;
                T a[kRowU], b[kRowU];
#pragma unroll
                for (int u = 0; u < kRowU; u++) {
                    const int i = cb + lane + 32 * u;
                    a[u] = i < E0 ? cj(ld(arow + (u0[p] ? i : 0)), d.conj_a) : zero<T>();
                    if (TWO) b[u] = i < E0 ? cj(ld(brow + (u02[p] ? i : 0)), d.conj_b) : zero<T>();
                }
#pragma unroll
                for (int u = 0; u < kRowU; u++) {
                    if (cb + 32 * u >= E0) continue;             // the whole warp is past the row's end
                    if (TWO) {
                        T sa = ng ? neg(a[u]) : a[u];              // the sign rides on a factor
                        if (chain) {
                            if (fold) sa = scale_f64(sa, d.as);
                            acc[u] = cfma(sa, b[u], acc[u]);
                        } else {
                            acc[u] = p == 0 ? mul(sa, b[u]) : cfma(sa, b[u], acc[u]);
                        }
                    } else {
                        acc[u] = signed_term(p == 0, ng, a[u], acc[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kRowU; u++) {
                const int i = cb + lane + 32 * u;
                if (i < E0) orow[i] = chain ? acc[u] : finish<ACC>(d.as, acc[u], old[u]);
            }
            // next row: odometer step with carries
#pragma unroll
            for (int k = kMaxDims - 2; k >= 0; k--) {
                if (k < d0) {
                    obase += d.ostr[k];
                    if (ACC && d.has_add) abase += d.astr[k];
#pragma unroll
                    for (int p = 0; p < NP; p++)
                        if (p < d.nperm) {
                            sb[p] += d.sstr[p][k];
                            if (TWO) sb2[p] += d.sstr2[p][k];
                        }
                    if (++dig[k] < (uint32_t)d.ext[k]) break;
                    dig[k] = 0;
                    obase -= d.ext[k] * d.ostr[k];
                    if (ACC && d.has_add) abase -= d.ext[k] * d.astr[k];
#pragma unroll
                    for (int p = 0; p < NP; p++)
                        if (p < d.nperm) {
                            sb[p] -= d.ext[k] * d.sstr[p][k];
                            if (TWO) sb2[p] -= d.ext[k] * d.sstr2[p][k];
                        }
                }
            }
        }
    }
}

template <typename T, int NP, bool TWO, bool ACC>
__global__ void __launch_bounds__(256) accum_rows_kernel(const AccumDesc d, const T *__restrict__ src,
                                                         const T *__restrict__ src2, T *__restrict__ out,
                                                         const T *__restrict__ add, uint32_t rows, int rch,
                                                         uint32_t ncb) {
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (uint32_t)((rows + (uint32_t)rch - 1) / (uint32_t)rch);
    const uint64_t items = (uint64_t)nchunks * ncb;
    for (uint64_t it = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5); it < items; it += (uint64_t)gridDim.x * 8)
        accum_rows_item<T, NP, TWO, ACC>(d, src, src2, out, add, rows, rch, ncb, it, lane);
}

// The grouped row path (real): entry e's items are [e.item0, e.item0 +
// ceil(rows / rch) * ncb); each warp takes a contiguous range of items.
template <int NP, bool TWO, bool ACC>
__global__ void __launch_bounds__(256) grouped_accum_rows_kernel(const GroupedAccum *__restrict__ tab, int n,
                                                                 int64_t total, const int *__restrict__ active) {
    const int lane = threadIdx.x & 31;
    const WorkRange wr = work_range(total, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                    (int64_t)gridDim.x * (blockDim.x >> 5));
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedAccum> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedAccum &e = tab[walk.at(it)];
        if (!active[e.sys]) { it = walk.next - 1; continue; }
        accum_rows_item<double, NP, TWO, ACC>(e.d, e.src, e.src2, e.out, e.add, e.rows, e.rch, e.ncb,
                                              (uint64_t)(it - e.item0), lane);
    }
}

// ------------------------------------------------------------- tiled path
// 32 x 32 tiles over two output dims, d0 = the innermost output dim and d1 = a
// dim that carries some term's unit source stride; every other dim is a batch
// index of the tile.  Each term reads its source tile either directly (lanes
// along d0) or through shared memory (lanes along d1, then transposed), so
// reads and writes stay coalesced for the P(..) gathers.  Blocks loop over
// tiles; tile and batch indices are decomposed with 32-bit divisions.
template <typename T, bool ACC>
__global__ void __launch_bounds__(256) accum_tiled_kernel(const AccumDesc d, const T *__restrict__ src,
                                                          T *__restrict__ out, int d0, int d1, uint64_t tmask,
                                                          uint32_t tiles0, uint32_t tiles1, uint32_t ntiles) {
    __shared__ T sm[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8 threads
    const int64_t E0 = d.ext[d0], E1 = d.ext[d1];
    const int64_t os0 = d.ostr[d0], os1 = d.ostr[d1];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t bid = t;
        const uint32_t t0 = bid % tiles0;
        bid /= tiles0;
        const uint32_t t1 = bid % tiles1;
        bid /= tiles1;
        // batch digits (all dims except d0, d1), row-major over the remaining dims
        uint32_t dig[kMaxDims];
#pragma unroll
        for (int k = kMaxDims - 1; k >= 0; k--) {
            dig[k] = 0;
            if (k < d.nd && k != d0 && k != d1) {
                const uint32_t e = (uint32_t)d.ext[k], q = bid / e;
                dig[k] = bid - q * e;
                bid = q;
            }
        }
        int64_t obase = 0;
#pragma unroll
        for (int k = 0; k < kMaxDims; k++)
            if (k < d.nd) obase += (int64_t)dig[k] * d.ostr[k];
        const int64_t i0b = (int64_t)t0 * 32, i1b = (int64_t)t1 * 32;
        T acc[4] = {zero<T>(), zero<T>(), zero<T>(), zero<T>()};
        T old[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t i1 = ty + 8 * r;
            const bool ok = i0b + tx < E0 && i1b + i1 < E1;
            old[r] = (ACC && ok) ? out[obase + (i0b + tx) * os0 + (i1b + i1) * os1] : zero<T>();
        }
        for (int p = 0; p < d.nperm; p++) {
            int64_t base = 0;
#pragma unroll
            for (int k = 0; k < kMaxDims; k++)
                if (k < d.nd) base += (int64_t)dig[k] * d.sstr[p][k];     // dig[d0] = dig[d1] = 0
            const int64_t s0 = d.sstr[p][d0], s1 = d.sstr[p][d1];
            base += i0b * s0 + i1b * s1;
            const bool ng = (d.negmask >> p) & 1ull;
            if (!((tmask >> p) & 1ull)) {
                T x[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int64_t i1 = ty + 8 * r;
                    x[r] = (i0b + tx < E0 && i1b + i1 < E1) ? cj(ld(src + base + tx * s0 + i1 * s1), d.conj_a)
                                                            : zero<T>();
                }
#pragma unroll
                for (int r = 0; r < 4; r++) acc[r] = signed_term(p == 0, ng, x[r], acc[r]);
            } else {
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int64_t i0 = ty + 8 * r;
                    sm[tx][i0] = (i1b + tx < E1 && i0b + i0 < E0) ? ld(src + base + tx * s1 + i0 * s0) : zero<T>();
                }
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 4; r++) acc[r] = signed_term(p == 0, ng, cj(sm[ty + 8 * r][tx], d.conj_a), acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t i1 = ty + 8 * r;
            if (i0b + tx < E0 && i1b + i1 < E1)
                out[obase + (i0b + tx) * os0 + (i1b + i1) * os1] = finish<ACC>(d.as, acc[r], old[r]);
        }
    }
}

// ------------------------------------------------------ pair antisymmetriser
// out(i,j,a,b) = beta out + alpha [z(ijab) - z(jiab) - z(ijba) + z(jiba)]
// with z(i,j,a,b) = src[i S0 + j S1 + a S2 + b S3] and the output addressed by
// O0..O3 (ext: n1 = ext i = ext j, n2 = ext a = ext b).  The value at ijab
// fixes the whole orbit: out(jiab) = out(ijba) = -out(ijab), out(jiba) =
// out(ijab).  A block takes one (i <= j, A <= B) pair of 32-wide a/b tiles,
// reads the four source tiles once (two of them transposed through shared
// memory), forms X(a,b) = (z_ij(a,b) - z_ij(b,a)) - (z_ji(a,b) - z_ji(b,a))
// and writes the four output tiles, so every element of src and out moves
// once.  i == j and a == b give exact zeros (x - x); A == B and i == j skip
// the duplicate writes.
struct PairSym {
    int64_t n1, n2;
    int64_t S[4], O[4];
};

template <bool ACC, typename T> __device__ __forceinline__ void pair_store(T *out, int64_t off, T v) {
    out[off] = ACC ? add(v, out[off]) : v;
}

template <typename T, bool ACC>
__global__ void __launch_bounds__(256) antisym_pairs_kernel(const AccumDesc d, const PairSym g,
                                                            const T *__restrict__ src, T *__restrict__ out,
                                                            uint32_t nt, uint32_t items) {
    __shared__ T s1[32][33], s2[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n2 = g.n2;
    for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
        // item = ((i * n1 + j) * nt + A) * nt + B, only i <= j and A <= B work
        uint32_t x = it;
        const uint32_t B = x % nt;
        x /= nt;
        const uint32_t A = x % nt;
        x /= nt;
        const uint32_t j = x % (uint32_t)g.n1, i = x / (uint32_t)g.n1;
        if (i > j || A > B) continue;
        const int64_t a0 = (int64_t)A * 32, b0 = (int64_t)B * 32;
        const int64_t zij = i * g.S[0] + j * g.S[1], zji = j * g.S[0] + i * g.S[1];
        const int64_t oij = i * g.O[0] + j * g.O[1], oji = j * g.O[0] + i * g.O[1];
        T z1[4], z2[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t a = a0 + ty + 8 * r, b = b0 + tx;
            const bool ok = a < n2 && b < n2;
            const int64_t off = a * g.S[2] + b * g.S[3];
            z1[r] = ok ? cj(ld(src + zij + off), d.conj_a) : zero<T>();
            z2[r] = ok ? cj(ld(src + zji + off), d.conj_a) : zero<T>();
        }
        __syncthreads();                    // previous item's reads of s1/s2 are done
#pragma unroll
        for (int r = 0; r < 4; r++) {
            // s(b', a') = z(., ., b0 + b', a0 + a'), lanes along a'
            const int64_t bb = b0 + ty + 8 * r, aa = a0 + tx;
            const bool ok = bb < n2 && aa < n2;
            const int64_t off = bb * g.S[2] + aa * g.S[3];
            s1[ty + 8 * r][tx] = ok ? cj(ld(src + zij + off), d.conj_a) : zero<T>();
            s2[ty + 8 * r][tx] = ok ? cj(ld(src + zji + off), d.conj_a) : zero<T>();
        }
        __syncthreads();
        T X[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            // z(i,j,b,a) for a = a0 + ty + 8r, b = b0 + tx sits at s(b - b0, a - a0)
            X[r] = scale_f64(sub(sub(z1[r], s1[tx][ty + 8 * r]), sub(z2[r], s2[tx][ty + 8 * r])), d.as);
        }
        const bool offdiag = i != j;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t a = a0 + ty + 8 * r, b = b0 + tx;
            if (a < n2 && b < n2) {
                const int64_t off = a * g.O[2] + b * g.O[3];
                pair_store<ACC>(out, oij + off, X[r]);
                if (offdiag) pair_store<ACC>(out, oji + off, neg(X[r]));
            }
        }
        if (A != B) {
            __syncthreads();                // s1 is reused for X
#pragma unroll
            for (int r = 0; r < 4; r++) s1[ty + 8 * r][tx] = X[r];     // s1(a', b') = X(a0 + a', b0 + b')
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; r++) {
                // out(i,j,b,a) = -X(a,b): lanes along a' = tx, b' = ty + 8r
                const int64_t bb = b0 + ty + 8 * r, aa = a0 + tx;
                if (bb < n2 && aa < n2) {
                    const T v = s1[tx][ty + 8 * r];
                    const int64_t off = bb * g.O[2] + aa * g.O[3];
                    pair_store<ACC>(out, oij + off, offdiag ? neg(v) : v);
                    if (offdiag) pair_store<ACC>(out, oji + off, v);
                }
            }
        }
    }
}

// ------------------------------------------------ triple-orbit antisymmetriser
// out(., t, .) (+)= alpha sum_p sign_p src(., pi_p t, .) where t = (t0, t1, t2)
// runs over three dims of equal extent n and the six terms are the six
// permutations of those dims with their parities (the full antisymmetriser
// of a triple, e.g. P(i/jk) P(jk) of the triples residual, Eq. amp).  The dims
// before the triple form a batch index (stride sb / ob) and the dims after it
// one contiguous run of C elements.  A work item is (multiset i <= j <= k,
// batch, 256-column chunk): for i < j < k the six source rows are read once,
// X = sum_p sign_p src_p formed (five adds) and sgn(sigma) X written to the six
// output rows sigma(i, j, k), so every element moves once; a multiset with a
// repeated index is an exact zero (skipped when accumulating, written as
// zeros otherwise).
struct TripleSym {
    int64_t n, C, nb;
    int64_t S[6][3];      // term p's source strides of the three dims
    int64_t O[3];         // output strides of the three dims
    int64_t sb, ob;       // batch strides (one collapsed batch dim)
};

// sigma applied to (i, j, k): the six orderings with their parities
__device__ __forceinline__ void triple_perm(int q, int64_t i, int64_t j, int64_t k, int64_t &a, int64_t &b,
                                            int64_t &c, bool &odd) {
    switch (q) {
        case 0: a = i; b = j; c = k; odd = false; break;
        case 1: a = j; b = i; c = k; odd = true; break;
        case 2: a = i; b = k; c = j; odd = true; break;
        case 3: a = k; b = j; c = i; odd = true; break;
        case 4: a = j; b = k; c = i; odd = false; break;
        default: a = k; b = i; c = j; odd = false; break;
    }
}

template <typename T, bool ACC>
__global__ void __launch_bounds__(256) antisym_triple_rows_kernel(const AccumDesc d, const TripleSym g,
                                                                  const T *__restrict__ src, T *__restrict__ out,
                                                                  uint32_t nms, uint32_t nchunk, uint64_t items) {
    constexpr int U = 4;                          // columns per thread per item: chunk = 1024
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        uint64_t x = it;
        const uint32_t ch = (uint32_t)(x % nchunk);
        x /= nchunk;
        const uint32_t ms = (uint32_t)(x % nms);
        const int64_t bidx = (int64_t)(x / nms);
        // multiset index -> i <= j <= k (k fastest)
        int64_t i = 0, j = 0, k = 0;
        {
            uint32_t r = ms;
            for (i = 0; i < g.n; i++) {
                const uint32_t cnt = (uint32_t)((g.n - i) * (g.n - i + 1) / 2);   // pairs j <= k in [i, n)
                if (r < cnt) break;
                r -= cnt;
            }
            for (j = i; j < g.n; j++) {
                const uint32_t cnt = (uint32_t)(g.n - j);
                if (r < cnt) break;
                r -= cnt;
            }
            k = j + r;
        }
        const bool distinct = i < j && j < k;
        if (!distinct && ACC) continue;                    // adds an exact zero
        const int64_t c0 = (int64_t)ch * (256 * U);
        const int64_t sbase = bidx * g.sb, obase = bidx * g.ob;
        if (!distinct) {
            // rows of a repeated index: the distinct orderings of the multiset get zeros
            for (int q = 0; q < 6; q++) {
                int64_t a, b, c;
                bool odd;
                triple_perm(q, i, j, k, a, b, c, odd);
                T *orow = out + obase + a * g.O[0] + b * g.O[1] + c * g.O[2];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t col = c0 + threadIdx.x + 256 * u;
                    if (col < g.C) orow[col] = zero<T>();
                }
            }
            continue;
        }
        const T *srow[6];
#pragma unroll
        for (int p = 0; p < 6; p++) srow[p] = src + sbase + i * g.S[p][0] + j * g.S[p][1] + k * g.S[p][2];
        T X[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t col = c0 + threadIdx.x + 256 * u;
            T w[6];
#pragma unroll
            for (int p = 0; p < 6; p++) w[p] = col < g.C ? cj(ld(srow[p] + col), d.conj_a) : zero<T>();
            T acc = zero<T>();
#pragma unroll
            for (int p = 0; p < 6; p++) acc = signed_term(p == 0, (d.negmask >> p) & 1ull, w[p], acc);
            X[u] = scale_f64(acc, d.as);
        }
#pragma unroll
        for (int q = 0; q < 6; q++) {
            int64_t a, b, c;
            bool odd;
            triple_perm(q, i, j, k, a, b, c, odd);
            T *orow = out + obase + a * g.O[0] + b * g.O[1] + c * g.O[2];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t col = c0 + threadIdx.x + 256 * u;
                if (col < g.C) {
                    const T v = odd ? neg(X[u]) : X[u];
                    orow[col] = ACC ? add(v, orow[col]) : v;
                }
            }
        }
    }
}

// The same antisymmetriser over the three innermost dims (e.g. the virtual
// triple of W3 = P(a/bc) P(bc) Z3): the orbit {sigma(a, b, c)} spans a whole
// n^3 cube of one batch row, so its members are strided.  A work item is
// (batch row, eight pairs a < b); warp w takes one pair and its lanes the c >
// b, reading the six orbit members, forming X once and writing +-X to all
// six.  Consecutive items share a row, so the blocks running at once work on a
// few cubes that L2 holds, and every element still moves once through HBM.
// In store mode, items past the orbits zero the cube's repeated-index planes.
template <typename T, bool ACC>
__global__ void __launch_bounds__(256) antisym_triple_inner_kernel(const AccumDesc d, const TripleSym g,
                                                                   const T *__restrict__ src, T *__restrict__ out,
                                                                   uint32_t npair_items, uint64_t items) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = g.n;
    const uint64_t orbit_items = (uint64_t)g.nb * npair_items;
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        if (it >= orbit_items) {
            // store mode: zero the planes with a repeated index, row (it - orbit_items) / n, plane x
            const uint64_t z = it - orbit_items;
            const int64_t row = (int64_t)(z / (uint64_t)n), x = (int64_t)(z % (uint64_t)n);
            T *o = out + row * g.ob;
            for (int64_t y = threadIdx.x; y < n; y += blockDim.x) {
                o[x * g.O[0] + x * g.O[1] + y * g.O[2]] = zero<T>();
                o[x * g.O[0] + y * g.O[1] + x * g.O[2]] = zero<T>();
                o[y * g.O[0] + x * g.O[1] + x * g.O[2]] = zero<T>();
            }
            continue;
        }
        const int64_t row = (int64_t)(it / npair_items);
        const uint32_t pi = (uint32_t)(it % npair_items) * 8 + warp;       // this warp's pair index
        // pair index -> a < b (b fastest)
        int64_t a = 0, b = 0;
        {
            uint32_t r = pi;
            bool found = false;
            for (a = 0; a + 1 < n; a++) {
                const uint32_t cnt = (uint32_t)(n - 1 - a);
                if (r < cnt) { b = a + 1 + r; found = true; break; }
                r -= cnt;
            }
            if (!found) continue;                                          // past the last pair
        }
        const T *sr = src + row * g.sb;
        T *orow = out + row * g.ob;
        for (int64_t c = b + 1 + lane; c < n; c += 32) {
            T acc = zero<T>();
#pragma unroll
            for (int p = 0; p < 6; p++) {
                const T w = cj(ld(sr + a * g.S[p][0] + b * g.S[p][1] + c * g.S[p][2]), d.conj_a);
                acc = signed_term(p == 0, (d.negmask >> p) & 1ull, w, acc);
            }
            const T X = scale_f64(acc, d.as);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                int64_t x, y, z;
                bool odd;
                triple_perm(q, a, b, c, x, y, z, odd);
                T *op = orow + x * g.O[0] + y * g.O[1] + z * g.O[2];
                const T v = odd ? neg(X) : X;
                *op = ACC ? add(v, *op) : v;
            }
        }
    }
}

// The inner-triple antisymmetriser by tile orbits: a work item is (batch row,
// tile multiset A <= B <= C) of 8 x 8 x 8 tiles of the n^3 cube.  The block
// reads each term's source tile with lanes along that term's contiguous dim
// (64-byte runs), sums the six signed terms into the representative tile in
// shared memory (term by term, in the order of the terms), then writes the six
// output tiles sigma(A, B, C), each with lanes along the output's contiguous
// dim: every element a < b < c is written with its sign to its six orbit
// members.  Each global access is a full 64-byte run, where the warp-per-pair
// form's strided members touched one sector per element.
constexpr int kTriTile = 8;

// 3 x the position of each dim of a (distinct) stride triple in memory order,
// fastest first: the shift of the dim's digit in a tile's linear index
__device__ __forceinline__ void digit_shifts(const int64_t *st, int sh[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) sh[k] = 3 * ((st[(k + 1) % 3] < st[k]) + (st[(k + 2) % 3] < st[k]));
}

// one term's tile of a work item: element l = tid + 256 h in the term's memory
// order (digit shifts sh), read into w[h]
template <typename T>
__device__ __forceinline__ void tri_tile_load(const AccumDesc &d, const TripleSym &g, const T *__restrict__ sr,
                                              const int tl[3], const int sh[3], int p, T w[2]) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int l = threadIdx.x + 256 * h;
        const int64_t t0 = tl[0] * kTriTile + ((l >> sh[0]) & 7), t1 = tl[1] * kTriTile + ((l >> sh[1]) & 7),
                      t2 = tl[2] * kTriTile + ((l >> sh[2]) & 7);
        w[h] = (t0 < g.n && t1 < g.n && t2 < g.n)
                   ? cj(ld(sr + t0 * g.S[p][0] + t1 * g.S[p][1] + t2 * g.S[p][2]), d.conj_a)
                   : zero<T>();
    }
}

// tile multiset index -> A <= B <= C
__device__ __forceinline__ void tri_tiles(uint32_t r, int nt, int tl[3]) {
    int A = 0, B = 0;
    for (A = 0; A < nt; A++) {
        const uint32_t cnt = (uint32_t)((nt - A) * (nt - A + 1) / 2);
        if (r < cnt) break;
        r -= cnt;
    }
    for (B = A; B < nt; B++) {
        const uint32_t cnt = (uint32_t)(nt - B);
        if (r < cnt) break;
        r -= cnt;
    }
    tl[0] = A; tl[1] = B; tl[2] = B + (int)r;
}

// Tile-local offsets of a thread's elements, which do not change from item to
// item: per term, the source offset of element l of the tile in that term's
// memory order, and the output offset of element l in the output's memory
// order (32-bit: the host takes this kernel for n^3 < 2^31 only).  With them
// an interior tile triple A < B < C (every element valid) costs an add per
// access instead of the digit arithmetic and bounds checks of the general path.
struct TriTabs {
    int src[6][kTriTile * kTriTile * kTriTile];
    int dst[kTriTile * kTriTile * kTriTile];
};
template <typename T> struct TriTabsSel { using type = TriTabs; };
template <> struct TriTabsSel<double2> { using type = char; };   // no room beside the complex tiles

template <typename T, bool ACC>
__global__ void __launch_bounds__(256) antisym_triple_tiles_kernel(const AccumDesc d, const TripleSym g,
                                                                   const T *__restrict__ src, T *__restrict__ out,
                                                                   uint32_t ntm, uint64_t items) {
    // output position m of orbit member q holds t[kPi[q][m]] (the six orderings of
    // (a, b, c) as in triple_perm), with parity kOdd[q]
    constexpr int kPi[6][3] = {{0, 1, 2}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}, {1, 2, 0}, {2, 0, 1}};
    constexpr bool kOdd[6] = {false, true, true, true, false, false};
    constexpr int kT3 = kTriTile * kTriTile * kTriTile;
    constexpr bool kTabs = sizeof(T) == 8;
    __shared__ T tiles[6][kT3];                 // the terms' tiles, canonical (a, b, c) order; X in tiles[0]
    __shared__ typename TriTabsSel<T>::type tabs;
    const int tid = threadIdx.x;
    const int64_t n = g.n;
    const int nt = (int)((n + kTriTile - 1) / kTriTile);
    const uint64_t orbit_items = (uint64_t)g.nb * ntm;
    int fs[6][3], gs[3];
#pragma unroll
    for (int p = 0; p < 6; p++) digit_shifts(g.S[p], fs[p]);
    digit_shifts(g.O, gs);
    if constexpr (kTabs) {
        TriTabs &tb = *reinterpret_cast<TriTabs *>(&tabs);
        for (int l = tid; l < kT3; l += blockDim.x) {
#pragma unroll
            for (int p = 0; p < 6; p++) {
                int64_t o = 0;
#pragma unroll
                for (int k = 0; k < 3; k++) o += (int64_t)((l >> fs[p][k]) & 7) * g.S[p][k];
                tb.src[p][l] = (int)o;
            }
            int64_t o = 0;
#pragma unroll
            for (int m = 0; m < 3; m++) o += (int64_t)((l >> gs[m]) & 7) * g.O[m];
            tb.dst[l] = (int)o;
        }
        __syncthreads();
    }
    // an interior triple of distinct tiles: every element is a valid orbit representative
    auto interior = [&](const int t3[3]) {
        return kTabs && t3[0] < t3[1] && t3[1] < t3[2] && (int64_t)(t3[2] + 1) * kTriTile <= n;
    };
    // the item's loads (element l of each term's tile in the term's memory order)
    auto load_item = [&](uint64_t item, int t3[3], T wv[6][2]) {
        tri_tiles((uint32_t)(item % ntm), nt, t3);
        const T *sr = src + (int64_t)(item / ntm) * g.sb;
        if constexpr (kTabs) {
            if (interior(t3)) {
                const TriTabs &tb = *reinterpret_cast<const TriTabs *>(&tabs);
#pragma unroll
                for (int p = 0; p < 6; p++) {
                    const T *base = sr + (int64_t)t3[0] * kTriTile * g.S[p][0] + (int64_t)t3[1] * kTriTile * g.S[p][1] +
                                    (int64_t)t3[2] * kTriTile * g.S[p][2];
#pragma unroll
                    for (int h = 0; h < 2; h++) wv[p][h] = cj(ld(base + tb.src[p][tid + 256 * h]), d.conj_a);
                }
                return;
            }
        }
#pragma unroll
        for (int p = 0; p < 6; p++) tri_tile_load(d, g, sr, t3, fs[p], p, wv[p]);
    };
    // the loads of the block's first orbit item, then per item: stage, issue the
    // next item's loads, sum, write
    T w[6][2];
    uint64_t it = blockIdx.x;
    int tl[3] = {0, 0, 0};
    if (it < orbit_items) load_item(it, tl, w);
    for (; it < orbit_items; it += gridDim.x) {
        const int64_t row = (int64_t)(it / ntm);
        const int ctl[3] = {tl[0], tl[1], tl[2]};
        __syncthreads();                        // the previous item's reads of the tiles are done
#pragma unroll
        for (int p = 0; p < 6; p++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int l = tid + 256 * h;
                tiles[p][((((l >> fs[p][0]) & 7) * kTriTile) + ((l >> fs[p][1]) & 7)) * kTriTile +
                         ((l >> fs[p][2]) & 7)] = w[p][h];
            }
        __syncthreads();
        const uint64_t nx = it + gridDim.x;
        if (nx < orbit_items) load_item(nx, tl, w);   // in flight while this item is summed and written
        // X = sum_p sign_p term_p, in the order of the terms, for this thread's two elements
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int l = tid + 256 * h;
            T x = zero<T>();
#pragma unroll
            for (int p = 0; p < 6; p++) x = signed_term(p == 0, (d.negmask >> p) & 1ull, tiles[p][l], x);
            tiles[0][l] = x;                    // only this thread reads or writes element l here
        }
        __syncthreads();
        T *orow = out + row * g.ob;
        const bool fast = interior(ctl);
        // the six output tiles, lanes along the output's contiguous dim
#pragma unroll
        for (int q = 0; q < 6; q++) {
            T *obase = orow;
            if (fast) {
#pragma unroll
                for (int m = 0; m < 3; m++) obase += (int64_t)ctl[kPi[q][m]] * kTriTile * g.O[m];
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int l = tid + 256 * h;
                int lx[3], lt[3];
#pragma unroll
                for (int m = 0; m < 3; m++) lx[m] = (l >> gs[m]) & 7;
#pragma unroll
                for (int m = 0; m < 3; m++) lt[kPi[q][m]] = lx[m];
                T *op;
                if (fast) {
                    if constexpr (kTabs) op = obase + reinterpret_cast<const TriTabs *>(&tabs)->dst[l];
                    else op = nullptr;
                } else {
                    int64_t x[3], t[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) t[k] = (int64_t)ctl[k] * kTriTile + lt[k];
#pragma unroll
                    for (int m = 0; m < 3; m++) x[m] = t[kPi[q][m]];
                    if (!(t[0] < t[1] && t[1] < t[2] && t[2] < n)) continue;
                    op = orow + x[0] * g.O[0] + x[1] * g.O[1] + x[2] * g.O[2];
                }
                const T X = scale_f64(tiles[0][(lt[0] * kTriTile + lt[1]) * kTriTile + lt[2]], d.as);
                const T v = kOdd[q] ? neg(X) : X;
                *op = ACC ? add(v, *op) : v;
            }
        }
    }
    // store mode: zero the planes with a repeated index, one (row, plane x) per item
    for (uint64_t z = it - orbit_items; z < items - orbit_items; z += gridDim.x) {
        const int64_t row = (int64_t)(z / (uint64_t)n), x = (int64_t)(z % (uint64_t)n);
        T *o = out + row * g.ob;
        for (int64_t y = tid; y < n; y += blockDim.x) {
            o[x * g.O[0] + x * g.O[1] + y * g.O[2]] = zero<T>();
            o[x * g.O[0] + y * g.O[1] + x * g.O[2]] = zero<T>();
            o[y * g.O[0] + x * g.O[1] + x * g.O[2]] = zero<T>();
        }
    }
}

// ---------------------------------------------------------------- host side
// Drop unit dims and merge neighbours k, k+1 that are contiguous in the
// output and in every term's source(s): the kernels then see the fewest dims
// (a plain copy becomes one dim).
static void collapse_dims(AccumDesc &d) {
    int w = 0;
    for (int k = 0; k < d.nd; k++) {
        if (d.ext[k] == 1 && d.nd > 1) continue;
        d.ext[w] = d.ext[k];
        d.ostr[w] = d.ostr[k];
        d.astr[w] = d.astr[k];
        for (int p = 0; p < d.nperm; p++) {
            d.sstr[p][w] = d.sstr[p][k];
            if (d.two_src) d.sstr2[p][w] = d.sstr2[p][k];
        }
        w++;
    }
    if (w == 0) w = 1;
    d.nd = w;
    for (int k = d.nd - 2; k >= 0; k--) {
        const int64_t e = d.ext[k + 1];
        bool ok = d.ostr[k] == d.ostr[k + 1] * e && (!d.has_add || d.astr[k] == d.astr[k + 1] * e);
        for (int p = 0; p < d.nperm && ok; p++) {
            ok = d.sstr[p][k] == d.sstr[p][k + 1] * e;
            if (ok && d.two_src) ok = d.sstr2[p][k] == d.sstr2[p][k + 1] * e;
        }
        if (!ok) continue;
        // merge k+1 into k, shift the rest down
        d.ext[k] *= e;
        d.ostr[k] = d.ostr[k + 1];
        d.astr[k] = d.astr[k + 1];
        for (int p = 0; p < d.nperm; p++) {
            d.sstr[p][k] = d.sstr[p][k + 1];
            if (d.two_src) d.sstr2[p][k] = d.sstr2[p][k + 1];
        }
        for (int m = k + 1; m + 1 < d.nd; m++) {
            d.ext[m] = d.ext[m + 1];
            d.ostr[m] = d.ostr[m + 1];
            d.astr[m] = d.astr[m + 1];
            for (int p = 0; p < d.nperm; p++) {
                d.sstr[p][m] = d.sstr[p][m + 1];
                if (d.two_src) d.sstr2[p][m] = d.sstr2[p][m + 1];
            }
        }
        d.nd--;
    }
}

// Is d the pair antisymmetriser over dims (0,1) and (2,3)?  The term with a
// +-1 sign taken as base gives S; the other three must be its (01), (23) and
// (01)(23) swaps with signs -, -, + relative to it.  alpha_sign gets the
// base's sign.
static bool match_pair_antisym(const AccumDesc &d, PairSym &g, double &alpha_sign) {
    if (d.two_src || d.nd != 4 || d.nperm != 4) return false;
    if (d.ext[0] != d.ext[1] || d.ext[2] != d.ext[3] || d.ext[0] < 1 || d.ext[2] < 1) return false;
    if (d.ext[0] > 0x7fffffffLL || d.ext[2] > 0x7fffffffLL) return false;
    for (int p = 0; p < 4; p++)
        if (d.sign[p] != 1.0 && d.sign[p] != -1.0) return false;
    const int64_t *S = d.sstr[0];
    if (S[0] == S[1] || S[2] == S[3]) return false;
    const double s0 = d.sign[0];
    bool f01 = false, f23 = false, fb = false;
    for (int p = 1; p < 4; p++) {
        const int64_t *Q = d.sstr[p];
        const double rel = d.sign[p] * s0;
        if (Q[0] == S[1] && Q[1] == S[0] && Q[2] == S[2] && Q[3] == S[3] && rel < 0) f01 = true;
        else if (Q[0] == S[0] && Q[1] == S[1] && Q[2] == S[3] && Q[3] == S[2] && rel < 0) f23 = true;
        else if (Q[0] == S[1] && Q[1] == S[0] && Q[2] == S[3] && Q[3] == S[2] && rel > 0) fb = true;
        else return false;
    }
    if (!(f01 && f23 && fb)) return false;
    g.n1 = d.ext[0];
    g.n2 = d.ext[2];
    for (int k = 0; k < 4; k++) {
        g.S[k] = S[k];
        g.O[k] = d.ostr[k];
    }
    alpha_sign = s0;
    return true;
}

// Is d the triple antisymmetriser over three consecutive dims t..t+2 (equal
// extents), with one batch dim before them (or none) and a contiguous run
// after them (unit strides in src and out)?  Term p's strides on the three
// dims must be a permutation of term 0's, and its sign term 0's times the
// permutation's parity.
static bool match_triple_antisym(const AccumDesc &d0, TripleSym &g, bool inner = false) {
    if (d0.two_src || d0.has_add || d0.nperm != 6) return false;
    AccumDesc d = d0;
    for (int t = inner ? d.nd - 3 : 0; t >= 0 && t + 2 < d.nd; t++) {
        const int64_t n = d.ext[t];
        if (n < 3 || d.ext[t + 1] != n || d.ext[t + 2] != n || n > 4096) continue;
        // every other dim: the same stride in all terms
        bool ok = true;
        for (int k = 0; k < d.nd && ok; k++) {
            if (k >= t && k <= t + 2) continue;
            for (int p = 1; p < 6 && ok; p++) ok = d.sstr[p][k] == d.sstr[0][k];
        }
        if (!ok) continue;
        // the inner run: dims after t+2 contiguous with unit innermost stride in src and out
        int64_t C = 1, so = 1, oo = 1;
        for (int k = d.nd - 1; k > t + 2 && ok; k--) {
            ok = d.sstr[0][k] == so && d.ostr[k] == oo;
            so *= d.ext[k];
            oo *= d.ext[k];
            C *= d.ext[k];
        }
        if (!ok || (inner ? t + 3 != d.nd : C < 64)) continue;
        // the batch: dims before t collapse into one strided index
        int64_t nb = 1, sb = 0, ob = 0;
        for (int k = t - 1; k >= 0 && ok; k--) {
            if (d.ext[k] == 1) continue;
            if (nb == 1) { sb = d.sstr[0][k]; ob = d.ostr[k]; nb = d.ext[k]; }
            else if (d.sstr[0][k] == sb * nb && d.ostr[k] == ob * nb) nb *= d.ext[k];
            else ok = false;
        }
        if (!ok) continue;
        // the six terms: permutations of term 0's strides with parity signs
        const int64_t *B = &d.sstr[0][t];
        if (B[0] == B[1] || B[1] == B[2] || B[0] == B[2]) continue;
        bool seen[6] = {false, false, false, false, false, false};
        static const int perm[6][3] = {{0, 1, 2}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}, {1, 2, 0}, {2, 0, 1}};
        static const bool odd[6] = {false, true, true, true, false, false};
        for (int p = 0; p < 6 && ok; p++) {
            int hit = -1;
            for (int q = 0; q < 6; q++)
                if (d.sstr[p][t] == B[perm[q][0]] && d.sstr[p][t + 1] == B[perm[q][1]] &&
                    d.sstr[p][t + 2] == B[perm[q][2]])
                    hit = q;
            if (hit < 0 || seen[hit]) { ok = false; break; }
            seen[hit] = true;
            const double want = odd[hit] ? -d.sign[0] : d.sign[0];
            ok = d.sign[p] == want && (d.sign[p] == 1.0 || d.sign[p] == -1.0);
        }
        if (!ok) continue;
        g.n = n;
        g.C = C;
        g.nb = nb;
        g.sb = sb;
        g.ob = ob;
        for (int p = 0; p < 6; p++)
            for (int q = 0; q < 3; q++) g.S[p][q] = d.sstr[p][t + q];
        for (int q = 0; q < 3; q++) g.O[q] = d.ostr[t + q];
        return true;
    }
    return false;
}

static int64_t grid_cap(int64_t want, int64_t cap) { return want < 1 ? 1 : want > cap ? cap : want; }

// out *= beta over the output view (a general beta before an accumulating pass)
template <typename T>
__global__ void __launch_bounds__(256) scale_view_kernel(const AccumDesc d, T *__restrict__ out, double beta) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = e, off = 0;
        for (int k = d.nd - 1; k >= 0; k--) {
            const int64_t q = x / d.ext[k];
            off += (x - q * d.ext[k]) * d.ostr[k];
            x = q;
        }
        out[off] = scal(beta, out[off]);
    }
}

template <typename T, bool ACC>
static cudaError_t accum_generic(const AccumDesc &d, const T *src, T *out, cudaStream_t s, const T *src2,
                                 const T *add) {
    int64_t runs = (d.total + 32 * kAccChunk - 1) / (32 * kAccChunk);
    accum_kernel<T, ACC><<<(unsigned)grid_cap((runs + 7) / 8, 148 * 16), 256, 0, s>>>(d, src, out, src2, add);
    return cudaGetLastError();
}

template <typename T, int NP, bool ACC>
static cudaError_t rows_launch(const AccumDesc &d, const T *src, T *out, cudaStream_t s, const T *src2, const T *add) {
    const int64_t E0 = d.ext[d.nd - 1];
    const int64_t rows = d.total / E0;
    constexpr int U1 = rows_u<false>(), U2 = rows_u<true>();
    const int64_t cw = 32 * (d.two_src ? U2 : U1);                 // columns per work item
    const int64_t ncb = (E0 + cw - 1) / cw;
    // about four work items per resident warp (148 SMs x 64 warps), at most 16 rows each
    int64_t rch = rows * ncb / (148 * 64 * 4);
    rch = rch < 1 ? 1 : rch > 16 ? 16 : rch;
    const int64_t items = (rows + rch - 1) / rch * ncb;
    const unsigned blocks = (unsigned)grid_cap((items + 7) / 8, 148 * 16);
    if (d.two_src)
        accum_rows_kernel<T, NP, true, ACC><<<blocks, 256, 0, s>>>(d, src, src2, out, add, (uint32_t)rows, (int)rch,
                                                                   (uint32_t)ncb);
    else
        accum_rows_kernel<T, NP, false, ACC><<<blocks, 256, 0, s>>>(d, src, src2, out, add, (uint32_t)rows,
                                                                    (int)rch, (uint32_t)ncb);
    return cudaGetLastError();
}

template <typename T, bool ACC>
static cudaError_t accum_t(const AccumDesc &d0, const T *src, T *out, cudaStream_t s, const T *src2, const T *add) {
    PairSym g;
    double sg = 1.0;
    if (!d0.has_add && match_pair_antisym(d0, g, sg)) {
        AccumDesc d = d0;
        if (sg < 0) {
            d.alpha = -d.alpha;
            d.as = make_scale(d.alpha);
        }
        const int64_t nt = (g.n2 + 31) / 32;
        const int64_t items = g.n1 * g.n1 * nt * nt;
        if (items <= 0xffffffffLL) {
            antisym_pairs_kernel<T, ACC><<<(unsigned)grid_cap(items, 148 * 32), 256, 0, s>>>(
                d, g, src, out, (uint32_t)nt, (uint32_t)items);
            return cudaGetLastError();
        }
    }
    TripleSym tg;
    if (match_triple_antisym(d0, tg)) {
        const int64_t nms = tg.n * (tg.n + 1) * (tg.n + 2) / 6;          // multisets i <= j <= k
        const int64_t nchunk = (tg.C + 1023) / 1024;
        const uint64_t items = (uint64_t)nms * (uint64_t)tg.nb * (uint64_t)nchunk;
        antisym_triple_rows_kernel<T, ACC><<<(unsigned)grid_cap((int64_t)items, 148 * 16), 256, 0, s>>>(
            d0, tg, src, out, (uint32_t)nms, (uint32_t)nchunk, items);
        return cudaGetLastError();
    }
    // tile-local offsets (at most 7 per dim times a stride) kept in 32 bits
    auto small_strides = [](const TripleSym &t) {
        for (int k = 0; k < 3; k++) {
            if (t.O[k] < 0 || t.O[k] >= ((int64_t)1 << 27)) return false;
            for (int p = 0; p < 6; p++)
                if (t.S[p][k] < 0 || t.S[p][k] >= ((int64_t)1 << 27)) return false;
        }
        return true;
    };
    if (match_triple_antisym(d0, tg, true) && tg.n >= 3 && tg.n <= 1024 && small_strides(tg)) {
        const int64_t nt = (tg.n + kTriTile - 1) / kTriTile;
        const int64_t ntm = nt * (nt + 1) * (nt + 2) / 6;                  // tile multisets
        const uint64_t items = (uint64_t)tg.nb * (uint64_t)ntm + (ACC ? 0 : (uint64_t)tg.nb * (uint64_t)tg.n);
        antisym_triple_tiles_kernel<T, ACC><<<(unsigned)grid_cap((int64_t)items, 148 * 8), 256, 0, s>>>(
            d0, tg, src, out, (uint32_t)ntm, items);
        return cudaGetLastError();
    }
    if (match_triple_antisym(d0, tg, true) && tg.n <= 4096) {
        const int64_t npairs = tg.n * (tg.n - 1) / 2;
        const int64_t npair_items = (npairs + 7) / 8;
        const uint64_t items = (uint64_t)tg.nb * (uint64_t)npair_items + (ACC ? 0 : (uint64_t)tg.nb * (uint64_t)tg.n);
        if (npair_items <= 0xffffffffLL) {
            antisym_triple_inner_kernel<T, ACC><<<(unsigned)grid_cap((int64_t)items, 148 * 16), 256, 0, s>>>(
                d0, tg, src, out, (uint32_t)npair_items, items);
            return cudaGetLastError();
        }
    }
    AccumDesc d = d0;
    collapse_dims(d);
    const int dl = d.nd - 1;
    const int64_t rows = d.total / d.ext[dl];
    // row path: every source (and a fused copy's source) runs with stride 0 or 1
    // along the innermost output dim, and the output with stride 1
    bool rowok = d.nperm <= 8 && rows <= 0xffffffffLL && d.ext[dl] >= 8 && d.ext[dl] < 0x7fff0000LL &&
                 d.ostr[dl] == 1 && (!d.has_add || d.astr[dl] == 0 || d.astr[dl] == 1);
    for (int p = 0; p < d.nperm && rowok; p++) {
        rowok = d.sstr[p][dl] == 0 || d.sstr[p][dl] == 1;
        if (rowok && d.two_src) rowok = d.sstr2[p][dl] == 0 || d.sstr2[p][dl] == 1;
    }
    for (int k = 0; k < dl && rowok; k++) rowok = d.ext[k] <= 0xffffffffLL;
    if (rowok) {
        if (d.nperm <= 1) return rows_launch<T, 1, ACC>(d, src, out, s, src2, add);
        if (d.nperm <= 2) return rows_launch<T, 2, ACC>(d, src, out, s, src2, add);
        if (d.nperm <= 4) return rows_launch<T, 4, ACC>(d, src, out, s, src2, add);
        return rows_launch<T, 8, ACC>(d, src, out, s, src2, add);
    }
    // tiled path: the output's innermost dim and a partner dim both of extent >= 16
    if (!d.two_src && !d.has_add && d.nd >= 2 && d.ext[dl] >= 16) {
        int d1 = -1;
        uint64_t tmask = 0;
        // partner: the dim holding a term's smallest source stride, when that is not d0
        for (int p = 0; p < d.nperm; p++) {
            int kmin = 0;
            for (int k = 1; k < d.nd; k++)
                if (d.ext[k] > 1 && (d.ext[kmin] <= 1 || d.sstr[p][k] < d.sstr[p][kmin])) kmin = k;
            if (kmin != dl && d.sstr[p][kmin] < d.sstr[p][dl]) {
                if (d1 < 0) d1 = kmin;
                if (kmin == d1) tmask |= 1ull << p;
            }
        }
        if (d1 < 0) {
            // no transposed term: pair d0 with the largest remaining dim
            for (int k = 0; k < d.nd - 1; k++)
                if (d1 < 0 || d.ext[k] > d.ext[d1]) d1 = k;
        }
        if (d.ext[d1] >= 16) {
            const int64_t tiles0 = (d.ext[dl] + 31) / 32, tiles1 = (d.ext[d1] + 31) / 32;
            const int64_t ntiles = tiles0 * tiles1 * (d.total / (d.ext[dl] * d.ext[d1]));
            bool fits = ntiles <= 0xffffffffLL;
            for (int k = 0; k < d.nd && fits; k++) fits = d.ext[k] <= 0xffffffffLL;
            if (fits) {
                accum_tiled_kernel<T, ACC><<<(unsigned)grid_cap(ntiles, 148 * 8), 256, 0, s>>>(
                    d, src, out, dl, d1, tmask, (uint32_t)tiles0, (uint32_t)tiles1, (uint32_t)ntiles);
                return cudaGetLastError();
            }
        }
    }
    return accum_generic<T, ACC>(d, src, out, s, src2, add);
}

template <typename T>
static cudaError_t accum_dispatch(AccumDesc &d, const T *src, T *out, cudaStream_t s, const T *src2, const T *add) {
    if (d.bcase == 2) {
        // general beta: out *= beta first, then accumulate with beta = 1
        scale_view_kernel<T><<<(unsigned)grid_cap((d.total + 255) / 256, 148 * 16), 256, 0, s>>>(d, out, d.beta);
        if (cudaError_t e = cudaGetLastError()) return e;
        d.beta = 1.0;
        d.bcase = 1;
    }
    return d.bcase ? accum_t<T, true>(d, src, out, s, src2, add) : accum_t<T, false>(d, src, out, s, src2, add);
}

// the row path's test of launch_accum: after merging dims, every source (and
// a fused copy's source) runs with stride 0 or 1 along the output's innermost
// dim, and the output with stride 1
static bool row_path_ok(const AccumDesc &d) {
    const int dl = d.nd - 1;
    const int64_t rows = d.total / d.ext[dl];
    bool ok = d.nperm <= 8 && rows <= 0xffffffffLL && d.ext[dl] >= 8 && d.ext[dl] < 0x7fff0000LL &&
              d.ostr[dl] == 1 && (!d.has_add || d.astr[dl] == 0 || d.astr[dl] == 1);
    for (int p = 0; p < d.nperm && ok; p++) {
        ok = d.sstr[p][dl] == 0 || d.sstr[p][dl] == 1;
        if (ok && d.two_src) ok = d.sstr2[p][dl] == 0 || d.sstr2[p][dl] == 1;
    }
    for (int k = 0; k < dl && ok; k++) ok = d.ext[k] <= 0xffffffffLL;
    return ok;
}

void prepare_grouped_accum(GroupedAccum &g) {
    AccumDesc &d = g.d;
    d.negmask = 0;
    for (int p = 0; p < d.nperm; p++)
        if (d.sign[p] < 0.0) d.negmask |= 1ull << p;
    d.as = make_scale(d.alpha);
    d.bcase = beta_case(d.beta);
    collapse_dims(d);
    g.row_path = row_path_ok(d) ? 1 : 0;
    g.rows = 1;
    g.rch = 1;
    g.ncb = 1;
    if (g.row_path) {
        const int64_t E0 = d.ext[d.nd - 1];
        g.rows = (uint32_t)(d.total / E0);
        const int64_t cw = 32 * (d.two_src ? rows_u<true>() : rows_u<false>());
        g.ncb = (uint32_t)((E0 + cw - 1) / cw);
        g.rch = 2;
    }
}

int64_t grouped_accum_items(const GroupedAccum &g, int mode) {
    if (mode == 1) return ((int64_t)g.rows + g.rch - 1) / g.rch * (int64_t)g.ncb;
    if (mode == 2) return (g.d.total + 127) / 128;
    return (g.d.total + 32 * kAccChunk - 1) / (32 * kAccChunk);
}

bool grouped_ew_from(const GroupedAccum &g, GroupedEw &e) {
    const AccumDesc &d = g.d;
    if (d.cplx || d.nd < 1 || d.nd > kEwDims || d.nperm < 1 || d.nperm > kEwTerms || d.total <= 0 ||
        d.total >= ((int64_t)1 << 31) || d.bcase == 2)
        return false;
    // every operand's offsets (and a wrap's stride difference) below 2^31
    auto fits = [&](const int64_t *str) {
        int64_t m = 0;
        for (int k = 0; k < d.nd; k++) {
            if (str[k] < 0 || d.ext[k] >= ((int64_t)1 << 31)) return false;
            m += (d.ext[k] - 1) * str[k];
        }
        return m < ((int64_t)1 << 30) && 32 * str[d.nd - 1] < ((int64_t)1 << 30);
    };
    if (!fits(d.ostr) || (d.has_add && !fits(d.astr))) return false;
    for (int p = 0; p < d.nperm; p++)
        if (!fits(d.sstr[p]) || (d.two_src && !fits(d.sstr2[p]))) return false;
    e = GroupedEw{};
    e.nd = d.nd;
    e.nterms = d.nperm;
    e.has_add = d.has_add;
    e.total = (uint32_t)d.total;
    e.negmask = d.negmask;
    e.as = d.as;
    for (int k = 0; k < d.nd; k++) {
        e.ext[k] = (int)d.ext[k];
        e.ostr[k] = (int)d.ostr[k];
        e.astr[k] = d.has_add ? (int)d.astr[k] : 0;
        for (int p = 0; p < d.nperm; p++) {
            e.sstr[p][k] = (int)d.sstr[p][k];
            e.sstr2[p][k] = d.two_src ? (int)d.sstr2[p][k] : 0;
        }
    }
    // the offset deltas of the digit steps: [0] the 32-element step of the
    // innermost digit, [k >= 1] a wrap of digit k into digit k - 1
    const int k0 = e.nd - 1;
    auto deltas = [&](const int *str, int *w) {
        w[0] = 32 * str[k0];
        for (int k = 1; k < e.nd; k++) w[k] = str[k - 1] - e.ext[k] * str[k];
    };
    deltas(e.ostr, e.wo);
    deltas(e.astr, e.wa);
    for (int p = 0; p < e.nterms; p++) {
        deltas(e.sstr[p], e.ws[p]);
        deltas(e.sstr2[p], e.ws2[p]);
    }
    e.src = g.src;
    e.src2 = g.src2;
    e.add = g.add;
    e.out = g.out;
    e.sys = g.sys;
    return true;
}

cudaError_t launch_grouped_ew(const GroupedEw *tab, int n, int64_t total, bool acc, int nperm, bool two,
                              const int *active, cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    if (nperm > kEwTerms || (two && nperm > 2)) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)grid_cap((total + 7) / 8, 148 * 16);
#define CCB_EW(A, P, T) grouped_ew_kernel<A, P, T><<<blocks, 256, 0, s>>>(tab, n, total, active)
    if (two) {
        if (acc) { if (nperm <= 1) CCB_EW(true, 1, true); else CCB_EW(true, 2, true); }
        else { if (nperm <= 1) CCB_EW(false, 1, true); else CCB_EW(false, 2, true); }
    } else if (acc) {
        if (nperm <= 1) CCB_EW(true, 1, false);
        else if (nperm <= 2) CCB_EW(true, 2, false);
        else CCB_EW(true, 4, false);
    } else {
        if (nperm <= 1) CCB_EW(false, 1, false);
        else if (nperm <= 2) CCB_EW(false, 2, false);
        else CCB_EW(false, 4, false);
    }
#undef CCB_EW
    return cudaGetLastError();
}

cudaError_t launch_grouped_accum(const GroupedAccum *tab, int n, int64_t total, bool acc, int mode, int nperm,
                                 bool two, const int *active, cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)grid_cap((total + 7) / 8, 148 * 16);
    if (mode == 2) {
        if (nperm > 2) return cudaErrorInvalidValue;
#define CCB_ACC4(A, P, T) grouped_accum4_kernel<A, P, T><<<blocks, 256, 0, s>>>(tab, n, total, active)
        if (acc) {
            if (nperm <= 1) { if (two) CCB_ACC4(true, 1, true); else CCB_ACC4(true, 1, false); }
            else { if (two) CCB_ACC4(true, 2, true); else CCB_ACC4(true, 2, false); }
        } else {
            if (nperm <= 1) { if (two) CCB_ACC4(false, 1, true); else CCB_ACC4(false, 1, false); }
            else { if (two) CCB_ACC4(false, 2, true); else CCB_ACC4(false, 2, false); }
        }
#undef CCB_ACC4
        return cudaGetLastError();
    }
    if (mode == 0) {
        if (acc) grouped_accum_kernel<true><<<blocks, 256, 0, s>>>(tab, n, total, active);
        else grouped_accum_kernel<false><<<blocks, 256, 0, s>>>(tab, n, total, active);
        return cudaGetLastError();
    }
#define CCB_GROUPED_ROWS(NPV)                                                                                        \
    do {                                                                                                             \
        if (two) {                                                                                                   \
            if (acc) grouped_accum_rows_kernel<NPV, true, true><<<blocks, 256, 0, s>>>(tab, n, total, active);      \
            else grouped_accum_rows_kernel<NPV, true, false><<<blocks, 256, 0, s>>>(tab, n, total, active);         \
        } else {                                                                                                     \
            if (acc) grouped_accum_rows_kernel<NPV, false, true><<<blocks, 256, 0, s>>>(tab, n, total, active);     \
            else grouped_accum_rows_kernel<NPV, false, false><<<blocks, 256, 0, s>>>(tab, n, total, active);        \
        }                                                                                                            \
    } while (0)
    if (nperm <= 1) CCB_GROUPED_ROWS(1);
    else if (nperm <= 2) CCB_GROUPED_ROWS(2);
    else if (nperm <= 4) CCB_GROUPED_ROWS(4);
    else CCB_GROUPED_ROWS(8);
#undef CCB_GROUPED_ROWS
    return cudaGetLastError();
}

cudaError_t launch_accum(const AccumDesc &d0, const double *src, double *out, cudaStream_t s, const double *src2,
                         const double *add) {
    if (d0.total <= 0) return cudaSuccess;
    if (d0.nd < 1 || d0.nd > kMaxDims || d0.nperm < 1 || d0.nperm > kMaxPerms) return cudaErrorInvalidValue;
    if (d0.has_add && (!add || d0.beta != 1.0)) return cudaErrorInvalidValue;
    AccumDesc d = d0;
    d.negmask = 0;
    for (int p = 0; p < d.nperm; p++)
        if (d.sign[p] < 0.0) d.negmask |= 1ull << p;
    d.as = make_scale(d.alpha);
    d.bcase = beta_case(d.beta);
    if (d.cplx)
        return accum_dispatch<double2>(d, reinterpret_cast<const double2 *>(src), reinterpret_cast<double2 *>(out), s,
                                       reinterpret_cast<const double2 *>(src2), reinterpret_cast<const double2 *>(add));
    return accum_dispatch<double>(d, src, out, s, src2, add);
}

}  // namespace ccb
