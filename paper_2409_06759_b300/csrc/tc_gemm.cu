// tc_gemm.cu -- split-bf16 route of the bulk contractions (sm_103a):
//   split_bf16   FP64 strided view -> K-major bf16 planes (hi, mid, lo), the
//                TTGT transpose fused into the precision split
//   tc_gemm      tcgen05 GEMM over the plane products, FP32 accumulation in
//                TMEM, FP64 epilogue into the output
#include <atomic>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fp_bits.cuh"
#include "grouped.cuh"
#include "kernels.h"

namespace ccb {

__device__ __forceinline__ int64_t grp_off(const Grp &g, int64_t x) {
    if (g.nd == 1) return x * g.str[0];
    int64_t off = 0;
    for (int k = g.nd - 1; k >= 0; k--) {
        int64_t q = x / g.ext[k];
        off += (x - q * g.ext[k]) * g.str[k];
        x = q;
    }
    return off;
}

// C[roff + co[j]] = v[j] (bcase 0) or += v[j] (bcase 1; a general beta was
// applied to C beforehand), skipping co[j] < 0.  The branch is taken once per
// batch, so the FP64 add exists only on the accumulating side.
// fire-and-forget FP64 add in L2 (no value returns to the SM)
__device__ __forceinline__ void red_add_tc(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// (co may point to shared memory: each offset is read where it is used;
// bcase 2 means red: C += v by reductions)
template <int NB>
__device__ __forceinline__ void store_batch(double *__restrict__ C, int64_t roff, const int64_t *co, const double *v,
                                            int bcase) {
    if (bcase == 2) {
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) red_add_tc(C + roff + co[j], v[j]);
    } else if (bcase == 0) {
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) C[roff + co[j]] = v[j];
    } else {
        double old[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) old[j] = co[j] >= 0 ? C[roff + co[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) C[roff + co[j]] = v[j] + old[j];
    }
}
// the same from raw FP32 accumulator bits: alpha * r[j] is formed as each
// value is stored (integer pipe for alpha = +-2^k, a multiply otherwise, the
// choice made once per batch), so only the bits and the old values are live
template <int NB>
__device__ __forceinline__ void store_batch_f32(double *__restrict__ C, int64_t roff, const int64_t *co,
                                                const uint32_t *r, const Scale &as, int bcase) {
    if (as.general) {
        double v[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) v[j] = (double)__uint_as_float(r[j]) * as.value;
        store_batch<NB>(C, roff, co, v, bcase);
    } else if (bcase == 0) {
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) C[roff + co[j]] = f32_to_f64_pow2(__uint_as_float(r[j]), as.kexp, as.sflip);
    } else if (bcase == 2) {
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) red_add_tc(C + roff + co[j], f32_to_f64_pow2(__uint_as_float(r[j]), as.kexp, as.sflip));
    } else {
        double old[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) old[j] = co[j] >= 0 ? C[roff + co[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (co[j] >= 0) C[roff + co[j]] = f32_to_f64_pow2(__uint_as_float(r[j]), as.kexp, as.sflip) + old[j];
    }
}

__global__ void convert_selftest_kernel(const double *in, int64_t n, float *mine, float *ref) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        mine[e] = f64_to_f32_rn(in[e]);
        ref[e] = __double2float_rn(in[e]);
    }
}

// The split runs in FP32 after one rounding of x to FP32 on the integer pipe
// (24 significant bits, as many as three bf16 planes hold): the remainders
// x_f - hi and r - mid are exact in FP32, so no FP64 instruction is spent.
__device__ __forceinline__ void split3(double x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    const float xf = f64_to_f32_rn(x);
    h = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Source element X(r, k) of a split, real or complex (see SplitDesc):
// roff = row_offset(d, r) of a valid row.
__device__ __forceinline__ int64_t row_offset(const SplitDesc &d, int64_t r) {
    return grp_off(d.gr, d.cplx == 2 ? (r >> 1) : r);
}
__device__ __forceinline__ double src_at(const SplitDesc &d, const double *__restrict__ x, int64_t r, int64_t roff,
                                         int64_t k) {
    if (d.cplx == 0) return __ldg(x + roff + grp_off(d.gk, k));
    const int kc = (int)(k & 1);
    if (d.cplx == 1) {
        const double val = __ldg(x + roff + grp_off(d.gk, k >> 1) + kc);
        return (d.conj && kc) ? -val : val;
    }
    const int rc = (int)(r & 1), comp = rc ^ kc;
    const double val = __ldg(x + roff + grp_off(d.gk, k >> 1) + comp);
    const bool neg = (rc == 0 && kc == 1) != (d.conj && comp == 1);
    return neg ? -val : val;
}

// Long contiguous K: warps take (row, 1024-column span) items; lane l converts
// columns [8l, 8l+8) of each 256-column chunk and stores 16 bytes per plane.
// When the K group's innermost index has unit stride and every other stride
// keeps 16-byte alignment, the eight sources are read as four double2 loads.
// eight FP32 values -> NPL bf16 planes (hi, mid[, lo]); the remainders are exact in FP32
template <int NPL>
__device__ __forceinline__ void split8(const float *f, uint4 &H, uint4 &M, uint4 &L) {
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        const float2 hf = __bfloat1622float2(h2);
        const float r0 = f[2 * j] - hf.x, r1 = f[2 * j + 1] - hf.y;
        const __nv_bfloat162 m2 = __floats2bfloat162_rn(r0, r1);
        h[j] = *reinterpret_cast<const uint32_t *>(&h2);
        m[j] = *reinterpret_cast<const uint32_t *>(&m2);
        if (NPL == 3) {
            const float2 mf = __bfloat1622float2(m2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
            l[j] = *reinterpret_cast<const uint32_t *>(&l2);
        } else {
            l[j] = 0u;
        }
    }
    H = make_uint4(h[0], h[1], h[2], h[3]);
    M = make_uint4(m[0], m[1], m[2], m[3]);
    L = make_uint4(l[0], l[1], l[2], l[3]);
}

// one work item (row r, 1024-column span from kspan) by one warp
__device__ __forceinline__ void split_vec_item(const SplitDesc &d, const double *__restrict__ x,
                                               __nv_bfloat16 *__restrict__ planes, int vec, int64_t r, int64_t kspan,
                                               int lane) {
    const int64_t plane_elems = d.Rp * d.Kp;
    const int64_t kcols = d.kend ? d.kend : d.Kp;       // plane columns this split fills
    const double sc = d.scaled ? d.scale : 1.0;
    const int64_t kend = kspan + 1024 < kcols ? kspan + 1024 : kcols;
    const bool row_ok = r < d.R;
    const int64_t roff = row_ok ? row_offset(d, r) : 0;
    for (int64_t k0 = kspan + (int64_t)lane * 8; k0 < kend; k0 += 256) {
        // the eight source values (loads first), then FP32 rounding on the integer
        // pipe and two values per bf16 conversion (split8): the planes are built in
        // registers
        double v8[8];
        if (row_ok && vec && k0 + 7 < d.K) {
            // real: eight consecutive doubles; stacked complex: four
            // consecutive complex elements (re, im pairs)
            const double2 *src = reinterpret_cast<const double2 *>(
                x + roff + (d.cplx ? grp_off(d.gk, k0 >> 1) : grp_off(d.gk, k0)));
            const double sy = (d.cplx && d.conj) ? -1.0 : 1.0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const double2 v2 = __ldg(src + j);
                v8[2 * j] = v2.x;
                v8[2 * j + 1] = d.cplx ? sy * v2.y : v2.y;
            }
        } else if (d.cplx == 0 && row_ok && d.gk.nd >= 1) {
            // real, scalar loads: k0 decomposed once, then the innermost K digit
            // stepped (a new decomposition only where the run crosses it)
            const int64_t ein = d.gk.ext[d.gk.nd - 1], sin = d.gk.str[d.gk.nd - 1];
            int64_t off = grp_off(d.gk, k0), dig = k0 % ein;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int64_t k = k0 + j;
                v8[j] = k < d.K ? __ldg(x + roff + off) : 0.0;
                if (++dig == ein) {
                    dig = 0;
                    off = k + 1 < d.K ? grp_off(d.gk, k + 1) : 0;
                } else {
                    off += sin;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int64_t k = k0 + j;
                v8[j] = (row_ok && k < d.K) ? src_at(d, x, r, roff, k) : 0.0;
            }
        }
        float f[8];
#pragma unroll
        for (int j = 0; j < 8; j++) f[j] = f64_to_f32_rn(d.scaled ? v8[j] * sc : v8[j]);
        uint4 H, M, L;
        if (d.nplanes == 3) split8<3>(f, H, M, L);
        else split8<2>(f, H, M, L);
        __nv_bfloat16 *p0 = planes + r * d.Kp + d.kdst + k0;
        *reinterpret_cast<uint4 *>(p0) = H;
        *reinterpret_cast<uint4 *>(p0 + plane_elems) = M;
        if (d.nplanes == 3) *reinterpret_cast<uint4 *>(p0 + 2 * plane_elems) = L;
    }
}

__global__ void __launch_bounds__(256) split_bf16_kernel(const SplitDesc d, const double *__restrict__ x,
                                                         __nv_bfloat16 *__restrict__ planes, int vec) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    const int64_t kcols = d.kend ? d.kend : d.Kp;
    // work items: (row, 1024-column span); a warp takes one item at a time
    const int64_t spans = (kcols + 1023) / 1024;
    for (int64_t it = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); it < d.Rp * spans; it += nwarps) {
        const int64_t r = it / spans;
        split_vec_item(d, x, planes, vec, r, (it - r * spans) * 1024, lane);
    }
}

// The grouped form for long contiguous K: entry e's items are its (row,
// 1024-column span) pairs from e.tile0 (e.rtiles: 1 where the entry takes the
// vector loads); each warp takes a contiguous range of items (grouped.cuh).
__global__ void __launch_bounds__(256) grouped_split_vec_kernel(const GroupedSplit *__restrict__ tab, int n,
                                                                int64_t total, const int *__restrict__ active) {
    const int lane = threadIdx.x & 31;
    const WorkRange wr = work_range(total, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), (int64_t)gridDim.x * 8);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedSplit> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedSplit &e = tab[walk.at(it)];
        if (!active[e.sys]) { it = walk.next - 1; continue; }
        const int64_t kcols = e.d.kend ? e.d.kend : e.d.Kp;
        const int64_t spans = (kcols + 1023) / 1024, local = it - e.tile0, r = local / spans;
        split_vec_item(e.d, e.x, (__nv_bfloat16 *)e.planes, (int)e.rtiles, r, (local - r * spans) * 1024, lane);
    }
}

// Tiled split for every layout but the long contiguous-K one: a 64-row x
// 64-column tile whose row and column offsets are decomposed once per tile
// (one mixed-radix decomposition per row and per column, kept in shared
// memory) instead of once per element.  LK: lanes run along K (the source's
// unit stride is K's innermost digit), else along rows.  The 16 loads of a
// thread are issued before any arithmetic; each value is rounded to FP32 as
// it arrives -- alternately by the conversion instruction (FP64 pipe) and on
// the integer pipe, so neither pipe limits the kernel -- and the FP32 tile is
// staged in shared memory and written K-major, 16 bytes per lane per plane,
// two values per bf16 conversion.  NPL: planes (2 or 3); CPLX: complex modes.
__device__ __forceinline__ double src_tile(const SplitDesc &d, const double *__restrict__ x, int64_t r, int64_t ro,
                                           int64_t k, int64_t ko) {
    const int kc = (int)(k & 1);
    if (d.cplx == 1) {
        const double val = __ldg(x + ro + ko + kc);
        return (d.conj && kc) ? -val : val;
    }
    const int rc = (int)(r & 1), comp = rc ^ kc;
    const double val = __ldg(x + ro + ko + comp);
    const bool neg = (rc == 0 && kc == 1) != (d.conj && comp == 1);
    return neg ? -val : val;
}

// one 64 x 64 tile at (r0, k0) of a split, by the whole block (block-uniform call)
template <bool LK, int NPL, bool CPLX>
__device__ __forceinline__ void split_tile_one(const SplitDesc &d, const double *__restrict__ x,
                                               __nv_bfloat16 *__restrict__ planes, int64_t r0, int64_t k0,
                                               float (*tile)[65], int64_t *ro, int64_t *ko) {
    const int64_t plane_elems = d.Rp * d.Kp;
    const int64_t kcols = d.kend ? d.kend : d.Kp;       // plane columns this split fills
    const double sc = d.scaled ? d.scale : 1.0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        __syncthreads();                       // the previous tile's reads of tile/ro/ko are done
        if (tid < 64) {
            const int64_t r = r0 + tid;
            ro[tid] = r < d.R ? row_offset(d, r) : -1;
        } else if (tid < 128) {
            const int64_t k = k0 + tid - 64;
            ko[tid - 64] = k < d.K ? grp_off(d.gk, CPLX ? (k >> 1) : k) : -1;
        }
        __syncthreads();
        double v[16];
        // element e of the thread: (row, col) = LK ? (warp + 8 (e/2), lane + 32 (e%2))
        //                                          : (lane + 32 (e%2), warp + 8 (e/2))
        const int64_t oA = LK ? ko[lane] : ro[lane], oB = LK ? ko[lane + 32] : ro[lane + 32];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int w = warp + 8 * i;
            const int64_t ow = LK ? ro[w] : ko[w];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int64_t oo = h ? oB : oA;
                const int q = lane + 32 * h;
                const int rr = LK ? w : q, kk = LK ? q : w;
                const bool ok = ow >= 0 && oo >= 0;
                if (CPLX)
                    v[2 * i + h] = ok ? src_tile(d, x, r0 + rr, ro[rr], k0 + kk, ko[kk]) : 0.0;
                else
                    v[2 * i + h] = ok ? __ldg(x + ow + oo) : 0.0;
            }
        }
        if (d.scaled) {
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] *= sc;
        }
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int w = warp + 8 * i, q = lane + 32 * h;
                const float f = h ? f64_to_f32_rn(v[2 * i + h]) : __double2float_rn(v[2 * i + h]);
                if (LK) tile[w][q] = f;
                else tile[q][w] = f;
            }
        __syncthreads();
        // 64 rows x 8 runs of 8 columns: two runs per thread
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int run = tid + 256 * q, rr = run >> 3, kk = (run & 7) * 8;
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; j++) f[j] = tile[rr][kk + j];
            uint4 H, M, L;
            split8<NPL>(f, H, M, L);
            if (r0 + rr < d.Rp && k0 + kk < kcols) {
                __nv_bfloat16 *p0 = planes + (r0 + rr) * d.Kp + d.kdst + k0 + kk;
                *reinterpret_cast<uint4 *>(p0) = H;
                *reinterpret_cast<uint4 *>(p0 + plane_elems) = M;
                if (NPL == 3) *reinterpret_cast<uint4 *>(p0 + 2 * plane_elems) = L;
            }
        }
    }
}

template <bool LK, int NPL, bool CPLX>
__global__ void __launch_bounds__(256, 5) split_tile_kernel(const SplitDesc d, const double *__restrict__ x,
                                                         __nv_bfloat16 *__restrict__ planes, uint32_t rtiles,
                                                         uint32_t ntiles) {
    __shared__ float tile[64][65];
    __shared__ int64_t ro[64], ko[64];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x)
        split_tile_one<LK, NPL, CPLX>(d, x, planes, (int64_t)(t % rtiles) * 64, (int64_t)(t / rtiles) * 64, tile, ro,
                                      ko);
}

// The grouped form: the tiles of every entry one after the other; each block
// takes a contiguous range of tiles (grouped.cuh) and stages an entry's
// descriptor in shared memory when it reaches the entry.
template <bool LK>
__global__ void __launch_bounds__(256, 5) grouped_split_kernel(const GroupedSplit *__restrict__ tab, int n,
                                                            int64_t total, const int *__restrict__ active) {
    __shared__ float tile[64][65];
    __shared__ int64_t ro[64], ko[64];
    __shared__ SplitDesc sd;                   // the current entry's descriptor
    static_assert(sizeof(SplitDesc) % 8 == 0 && sizeof(SplitDesc) / 8 <= 256, "descriptor staging");
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedSplit> walk(tab, n, wr.begin);
    int staged = -1;
    for (int64_t t = wr.begin; t < wr.end; t++) {
        const int ei = walk.at(t);
        const GroupedSplit &e = tab[ei];
        if (!active[e.sys]) { t = walk.next - 1; continue; }   // block-uniform
        if (ei != staged) {
            __syncthreads();                   // the previous tile's reads of sd are done
            if (threadIdx.x < sizeof(SplitDesc) / 8)
                reinterpret_cast<int64_t *>(&sd)[threadIdx.x] = reinterpret_cast<const int64_t *>(&e.d)[threadIdx.x];
            __syncthreads();                   // staged: split_tile_one reads sd before its own barrier
            staged = ei;
        }
        const int64_t lt = t - e.tile0;
        split_tile_one<LK, 2, false>(sd, e.x, (__nv_bfloat16 *)e.planes, (lt % e.rtiles) * 64, (lt / e.rtiles) * 64,
                                     tile, ro, ko);
    }
}

template <bool LK>
static void split_tile_launch(const SplitDesc &d, const double *x, void *planes, unsigned blocks, uint32_t rtiles,
                              uint32_t ntiles, cudaStream_t s) {
    __nv_bfloat16 *p = (__nv_bfloat16 *)planes;
    if (d.cplx) {
        if (d.nplanes == 3) split_tile_kernel<LK, 3, true><<<blocks, 256, 0, s>>>(d, x, p, rtiles, ntiles);
        else split_tile_kernel<LK, 2, true><<<blocks, 256, 0, s>>>(d, x, p, rtiles, ntiles);
    } else {
        if (d.nplanes == 3) split_tile_kernel<LK, 3, false><<<blocks, 256, 0, s>>>(d, x, p, rtiles, ntiles);
        else split_tile_kernel<LK, 2, false><<<blocks, 256, 0, s>>>(d, x, p, rtiles, ntiles);
    }
}

// ------------------------------------------------------------ exact slices
// The FP64-grade split (kSlices = 6 planes): every row r of the operand gets an
// exponent E_r with max_k |X(r,k)| < 2^E_r, and each element is cut into six
// signed 7-bit slices of its fixed-point value |x| 2^-E_r:
//     x = sign 2^E_r sum_s q_s 2^-7(s+1) + t,   0 <= q_s <= 127,  |t| < 2^(E_r-42).
// A slice is stored as the bf16 number sign q_s 2^-7(s+1) (at most 7
// significant bits, so exact).  A product of slices s and t is then an integer
// multiple of 2^-7(s+t+2) below 2^-7(s+t) in magnitude, and a sum of fewer
// than 2^24 such units is exact in FP32 whatever the order of the additions:
// the tensor cores accumulate the slice products of one weight s + t exactly
// over 128-long K chunks (tc_gemm_slices_kernel).  The fixed-point value is
// taken from the 53-bit significand shifted by E_r - e_x, on the integer pipe.
// The row exponents (biased: the largest IEEE exponent field of the row, so
// E_r = field - 1022) follow the planes in the same buffer, one int per row.
constexpr int kSlices = 6;

__host__ __device__ inline int64_t slice_plane_bytes(int64_t R, int64_t Kp) { return (int64_t)kSlices * R * Kp * 2; }

// biased exponent field of |x| (0 for zeros and subnormals, 2047 for inf/NaN)
__device__ __forceinline__ int exp_field(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffull);
}

// pass 1: the row exponents (atomicMax into exps[], which starts at zero)
template <bool LK, bool CPLX>
__global__ void __launch_bounds__(256, 5) slice_exp_kernel(const SplitDesc d, const double *__restrict__ x,
                                                         int *__restrict__ exps, uint32_t rtiles, uint32_t ntiles) {
    __shared__ int64_t ro[64], ko[64];
    __shared__ int srow[64];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = (int64_t)(t % rtiles) * 64, k0 = (int64_t)(t / rtiles) * 64;
        __syncthreads();
        if (tid < 64) {
            const int64_t r = r0 + tid;
            ro[tid] = r < d.R ? row_offset(d, r) : -1;
            srow[tid] = 0;
        } else if (tid < 128) {
            const int64_t k = k0 + tid - 64;
            ko[tid - 64] = k < d.K ? grp_off(d.gk, CPLX ? (k >> 1) : k) : -1;
        }
        __syncthreads();
        int ex[16];
        const int64_t oA = LK ? ko[lane] : ro[lane], oB = LK ? ko[lane + 32] : ro[lane + 32];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int w = warp + 8 * i;
            const int64_t ow = LK ? ro[w] : ko[w];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int64_t oo = h ? oB : oA;
                const int q = lane + 32 * h;
                const int rr = LK ? w : q, kk = LK ? q : w;
                const bool ok = ow >= 0 && oo >= 0;
                double v;
                if (CPLX) v = ok ? src_tile(d, x, r0 + rr, ro[rr], k0 + kk, ko[kk]) : 0.0;
                else v = ok ? __ldg(x + ow + oo) : 0.0;
                ex[2 * i + h] = exp_field(v);
            }
        }
        if (LK) {
            // row warp + 8i: the warp's 64 values of that row
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int m = __reduce_max_sync(0xffffffffu, (unsigned)max(ex[2 * i], ex[2 * i + 1]));
                if (lane == 0 && m > 0) atomicMax(&srow[warp + 8 * i], m);
            }
        } else {
            // rows lane and lane + 32: eight values of each per thread
            int m0 = 0, m1 = 0;
#pragma unroll
            for (int i = 0; i < 8; i++) { m0 = max(m0, ex[2 * i]); m1 = max(m1, ex[2 * i + 1]); }
            if (m0 > 0) atomicMax(&srow[lane], m0);
            if (m1 > 0) atomicMax(&srow[lane + 32], m1);
        }
        __syncthreads();
        if (tid < 64 && r0 + tid < d.R && srow[tid] > 0) atomicMax(exps + r0 + tid, srow[tid]);
    }
}

// six slices of one element: out[s] = sign q_s 2^-7(s+1) (biased row exponent eb)
__device__ __forceinline__ void slice6(double x, int eb, float (&out)[kSlices]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ffull);
    if (ex == 0x7ff) {                       // inf / NaN: carried by the top slice
#pragma unroll
        for (int s = 0; s < kSlices; s++) out[s] = s == 0 ? __uint_as_float(0x7fc00000u) : 0.f;
        return;
    }
    const int dsh = eb - ex;
    unsigned long long a = 0ull;
    if (ex != 0 && dsh < 53) a = ((b & 0xfffffffffffffull) | (1ull << 52)) >> (dsh > 0 ? dsh : 0);
    const bool neg = (b >> 63) != 0ull;
    float sc = 0.0078125f;                   // 2^-7
#pragma unroll
    for (int s = 0; s < kSlices; s++) {
        const float f = __int2float_rn((int)((a >> (46 - 7 * s)) & 127ull)) * sc;
        out[s] = neg ? -f : f;
        sc *= 0.0078125f;
    }
}

// pass 2: the six planes, K-major, 16 bytes per lane per plane (the tile
// layout of split_tile_kernel; the FP64 tile is staged in shared memory)
template <bool LK, bool CPLX>
__global__ void __launch_bounds__(256, 3) slice_planes_kernel(const SplitDesc d, const double *__restrict__ x,
                                                            __nv_bfloat16 *__restrict__ planes,
                                                            const int *__restrict__ exps, uint32_t rtiles,
                                                            uint32_t ntiles) {
    __shared__ double tile[64][65];
    __shared__ int64_t ro[64], ko[64];
    const int64_t plane_elems = d.Rp * d.Kp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = (int64_t)(t % rtiles) * 64, k0 = (int64_t)(t / rtiles) * 64;
        __syncthreads();
        if (tid < 64) {
            const int64_t r = r0 + tid;
            ro[tid] = r < d.R ? row_offset(d, r) : -1;
        } else if (tid < 128) {
            const int64_t k = k0 + tid - 64;
            ko[tid - 64] = k < d.K ? grp_off(d.gk, CPLX ? (k >> 1) : k) : -1;
        }
        __syncthreads();
        double v[16];
        const int64_t oA = LK ? ko[lane] : ro[lane], oB = LK ? ko[lane + 32] : ro[lane + 32];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int w = warp + 8 * i;
            const int64_t ow = LK ? ro[w] : ko[w];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int64_t oo = h ? oB : oA;
                const int q = lane + 32 * h;
                const int rr = LK ? w : q, kk = LK ? q : w;
                const bool ok = ow >= 0 && oo >= 0;
                if (CPLX) v[2 * i + h] = ok ? src_tile(d, x, r0 + rr, ro[rr], k0 + kk, ko[kk]) : 0.0;
                else v[2 * i + h] = ok ? __ldg(x + ow + oo) : 0.0;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int w = warp + 8 * i, q = lane + 32 * h;
                if (LK) tile[w][q] = v[2 * i + h];
                else tile[q][w] = v[2 * i + h];
            }
        __syncthreads();
#pragma unroll 1
        for (int qd = 0; qd < 2; qd++) {
            const int run = tid + 256 * qd, rr = run >> 3, kk = (run & 7) * 8;
            if (r0 + rr >= d.Rp) continue;
            const int eb = exps[r0 + rr];
            uint32_t pk[kSlices][4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float s0[kSlices], s1[kSlices];
                slice6(tile[rr][kk + 2 * j], eb, s0);
                slice6(tile[rr][kk + 2 * j + 1], eb, s1);
#pragma unroll
                for (int sl = 0; sl < kSlices; sl++) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(s0[sl], s1[sl]);
                    pk[sl][j] = *reinterpret_cast<const uint32_t *>(&b2);
                }
            }
            __nv_bfloat16 *p0 = planes + (r0 + rr) * d.Kp + k0 + kk;
#pragma unroll
            for (int sl = 0; sl < kSlices; sl++)
                *reinterpret_cast<uint4 *>(p0 + sl * plane_elems) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
        }
    }
}

template <bool LK, bool CPLX>
static void slice_launch(const SplitDesc &d, const double *x, void *planes, int *exps, unsigned blocks,
                         uint32_t rtiles, uint32_t ntiles, cudaStream_t s) {
    slice_exp_kernel<LK, CPLX><<<blocks, 256, 0, s>>>(d, x, exps, rtiles, ntiles);
    slice_planes_kernel<LK, CPLX><<<blocks, 256, 0, s>>>(d, x, (__nv_bfloat16 *)planes, exps, rtiles, ntiles);
}

static cudaError_t launch_slices(const SplitDesc &d, const double *x, void *planes, cudaStream_t s) {
    int *exps = reinterpret_cast<int *>(static_cast<char *>(planes) + slice_plane_bytes(d.Rp, d.Kp));
    if (cudaError_t e = cudaMemsetAsync(exps, 0, sizeof(int) * (size_t)d.Rp, s)) return e;
    const int64_t rtiles = (d.Rp + 63) / 64, ntiles = rtiles * (d.Kp / 64);
    if (ntiles > 0xffffffffLL) return cudaErrorInvalidValue;
    const bool lk = split_lanes_along_k(d);
    const unsigned blocks = (unsigned)(ntiles < 148 * 6 ? ntiles : 148 * 6);
    if (d.cplx) {
        if (lk) slice_launch<true, true>(d, x, planes, exps, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
        else slice_launch<false, true>(d, x, planes, exps, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
    } else {
        if (lk) slice_launch<true, false>(d, x, planes, exps, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
        else slice_launch<false, false>(d, x, planes, exps, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const SplitDesc &d, const double *x, void *planes, cudaStream_t s) {
    if (d.Kp % 64 || d.Rp <= 0 || (d.nplanes != kSlices && (d.nplanes < 2 || d.nplanes > 3)) || d.cplx < 0 ||
        d.cplx > 2)
        return cudaErrorInvalidValue;
    if (d.cplx && (d.K % 2 || (d.cplx == 2 && d.R % 2))) return cudaErrorInvalidValue;
    if (d.nplanes == kSlices) return launch_slices(d, x, planes, s);
    // source unit stride inside the row group and not in K: transposed tiles
    // (for complex sources the unit is one complex element, two doubles)
    const int64_t unit = d.cplx ? 2 : 1;
    // vector path: long contiguous K (whole 1024-column spans per warp item)
    int vec = d.cplx != 2 && d.gk.nd >= 1 && d.gk.str[d.gk.nd - 1] == unit &&
              d.gk.ext[d.gk.nd - 1] % (d.cplx ? 4 : 8) == 0 && ((uintptr_t)x & 15) == 0;
    for (int q = 0; q + 1 < d.gk.nd; q++) vec &= (d.gk.str[q] % 2) == 0;
    for (int q = 0; q < d.gr.nd; q++) vec &= (d.gr.str[q] % 2) == 0;
    // K concatenation: the split fills plane columns [kdst, kdst + kcols) in runs
    // of eight (16-byte stores), so both stay multiples of 8
    const int64_t kcols = d.kend ? d.kend : d.Kp;
    if (d.kdst % 8 || kcols % 8 || d.kdst + kcols > d.Kp || kcols < d.K) return cudaErrorInvalidValue;
    const int64_t rtiles = (d.Rp + 63) / 64, ntiles = rtiles * ((kcols + 63) / 64);
    if (!(vec && d.K >= 512) && ntiles <= 0xffffffffLL) {
        const bool lk = split_lanes_along_k(d);
        const unsigned blocks = (unsigned)(ntiles < 148 * 5 ? ntiles : 148 * 5);
        if (lk) split_tile_launch<true>(d, x, planes, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
        else split_tile_launch<false>(d, x, planes, blocks, (uint32_t)rtiles, (uint32_t)ntiles, s);
        return cudaGetLastError();
    }
    // vec: innermost K digit contiguous with an extent that keeps the 8-column
    // runs inside it (4 complex elements when stacked), every other stride even
    // (16-byte aligned double2), base aligned; not for embedded
    const int64_t items = d.Rp * ((kcols + 1023) / 1024);
    int64_t blocks = (items + 7) / 8;
    if (blocks > 148 * 16) blocks = 148 * 16;
    split_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, x, (__nv_bfloat16 *)planes, vec);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ tcgen05
// Split-bf16 GEMM D = sum_products A_p B_q^T on the tensor cores.  One CTA per
// SM (persistent) computes output tiles of 128 rows by at most BN columns (the
// column tiles share N evenly, in steps of 16):
//   warp 0      TMA producer (one elected lane): all A and B planes of a
//               64-wide K block land in one pipeline stage (SWIZZLE_128B)
//   warp 1      TMEM allocator + MMA issuer (one lane): tcgen05.mma kind::f16,
//               bf16 x bf16 -> fp32 accumulators of 128 lanes x BN columns
//   warps 2..9  epilogue: tcgen05.ld of the accumulator, alpha/beta update of
//               the FP64 output through the mixed-radix addressing
// Every mbarrier wait is bounded (clock64 budget); on expiry the CTA sets
// err_flag, stops issuing work, waits (bounded) for what it already issued,
// frees its TMEM and returns.
namespace tc {

constexpr int BM = 128, BK = 64;
constexpr long long kWaitBudget = 4000000000LL;   // cycles (~2 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// false when the budget runs out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget = kWaitBudget) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// Self-test of the bounded wait: an mbarrier that expects one arrival nobody
// makes.  The wait gives up after `budget` cycles and the kernel records it and
// returns normally (nothing is in flight).
__global__ void wait_selftest_kernel(long long budget, int *timed_out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) *timed_out = mbar_wait(&bar, 0, budget) ? 0 : 1;
}

// box {64 columns, rows, 1 plane} at column x (a multiple of 64), row y, plane z;
// rows past the plane's row count arrive as zeros (the tile padding)
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major bf16 tile written by TMA with
// SWIZZLE_128B: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                     // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), fp32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Column tiles of an N-column output at tile width BN: the n_tiles =
// ceil(N / BN) tiles share the ceil(N / 16) 16-column units (16 is the MMA's
// N step at M = 128) as evenly as possible, the first `extra` tiles one unit
// wider; a tile's last columns may pass N by less than 16 (TMA reads zeros).
struct ColSplit {
    int base, extra;
    __host__ __device__ int width(int nb) const { return 16 * (base + (nb < extra ? 1 : 0)); }
    __host__ __device__ int64_t n0(int nb) const { return 16 * ((int64_t)nb * base + (nb < extra ? nb : extra)); }
    __host__ __device__ int wide() const { return 16 * (base + (extra > 0 ? 1 : 0)); }
};
static inline ColSplit col_split(int64_t N, int BN) {
    const int64_t n_tiles = (N + BN - 1) / BN, units = (N + 15) / 16;
    return ColSplit{(int)(units / n_tiles), (int)(units % n_tiles)};
}

template <int NP, int BN, int STAGES>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = NP * (A_BYTES + B_BYTES);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 1024 /*barriers, offsets*/ + BN * 8;
};

// ---- persistent variant (two planes): one CTA per SM walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... of the (tile, K-slice) space.
// The producer streams K blocks of consecutive tiles through the stage ring
// without a break; the MMA issuer alternates between two TMEM accumulators so
// the epilogue of one tile overlaps the main loop of the next.  Eight epilogue
// warps (2..9): warp w reads TMEM lanes 32*(w%4).. and the column half (w-2)/4
// of the tile, so twice as many output loads are in flight as with four.
// Column tiles share N evenly (ColSplit): e.g. N = 1600 at BN = 256 runs two
// 240-wide and five 224-wide tiles instead of six full ones and a quarter-full
// seventh, so no MMA works on padding and tiles of one row block cost about
// the same (their CTAs stay in step, which keeps the shared A block in L2).
template <int NP, int BN, int STAGES>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_persistent_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBw,
                              const __grid_constant__ CUtensorMap mapBn, const TcGemmDesc d,
                              double *__restrict__ C, double *__restrict__ partials, int kb_per_split, int nslices,
                              int64_t ntiles, const ColSplit cs, int *err_flag) {
    using G = Cfg<NP, BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = smem;
    uint64_t *full = (uint64_t *)(smem + STAGES * G::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;             // [2]
    uint64_t *acce = accf + 2;                   // [2]
    uint32_t *tmem_slot = (uint32_t *)(acce + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *epi_abort = abort_flag + 1;    // written by epilogue warps only (uniform decision)
    int64_t *coloff = (int64_t *)(smem + STAGES * G::STAGE_BYTES + 1024);   // [BN]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (int)((d.N + BN - 1) / BN);   // tiles past N would read padding only
    const int kb_total = (int)(d.Kp / BK);
    const int64_t total = ntiles * nslices;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 8);              // one arrival per epilogue warp
        }
        *abort_flag = 0;
        *epi_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 2 * BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    auto tile_coords = [&](int64_t t, int64_t &m0, int64_t &n0, int &nw, int &kb0, int &kb1) {
        const int64_t tile = t % ntiles;
        const int z = (int)(t / ntiles);
        m0 = (tile / n_tiles) * BM;
        const int nb = (int)(tile % n_tiles);
        n0 = cs.n0(nb);
        nw = cs.width(nb);
        kb0 = z * kb_per_split;
        kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
    };

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;                       // K blocks issued by this CTA so far
            bool stop = false;
            for (int64_t t = blockIdx.x; t < total && !stop; t += gridDim.x) {
                int64_t m0, n0;
                int nw, kb0, kb1;
                tile_coords(t, m0, n0, nw, kb0, kb1);
                const CUtensorMap *mb = nw == cs.wide() ? &mapBw : &mapBn;
                const uint32_t bytes = (uint32_t)(NP * (G::A_BYTES + nw * BK * 2));
                for (int kb = kb0; kb < kb1; kb++, g++) {
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    uint8_t *st = tiles + s * G::STAGE_BYTES;
                    mbar_expect_tx(&full[s], bytes);
                    for (int p = 0; p < NP; p++)
                        tma_load_3d(st + p * G::A_BYTES, &mapA, &full[s], kb * BK, (int)m0, p);
                    for (int q = 0; q < NP; q++)
                        tma_load_3d(st + NP * G::A_BYTES + q * G::B_BYTES, mb, &full[s], kb * BK, (int)n0, q);
                }
            }
            if (stop) {
                // let the last STAGES issued copies land before the CTA can exit
                for (int64_t k = (g > STAGES ? g - STAGES : 0); k < g; k++)
                    mbar_wait(&full[k % STAGES], (uint32_t)(k / STAGES) & 1u);
                atomicOr(err_flag, 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int64_t g = 0;
            int j = 0;                           // local tile counter
            for (int64_t t = blockIdx.x; t < total; t += gridDim.x, j++) {
                if (*abort_flag) break;
                int64_t m0, n0;
                int nw, kb0, kb1;
                tile_coords(t, m0, n0, nw, kb0, kb1);
                const uint32_t idesc = idesc_bf16(BM, nw);
                const int b = j & 1;
                if (j >= 2) {
                    if (!mbar_wait(&acce[b], (uint32_t)((j >> 1) - 1) & 1u)) {
                        *abort_flag = 1;
                        atomicOr(err_flag, 1);
                    }
                    fence_after();
                }
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                for (int kb = kb0; kb < kb1 && !*abort_flag; kb++, g++) {
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (!mbar_wait(&full[s], ph)) {
                        *abort_flag = 1;
                        atomicOr(err_flag, 1);
                        break;
                    }
                    fence_after();
                    const uint32_t st = smem_u32(tiles + s * G::STAGE_BYTES);
                    for (int pr = 0; pr < d.nprod; pr++) {
                        const uint32_t a0 = st + d.prod_a[pr] * G::A_BYTES;
                        const uint32_t b0 = st + NP * G::A_BYTES + d.prod_b[pr] * G::B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; kk++)
                            mma_bf16(dt, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                                     ((kb - kb0) | pr | kk) != 0);
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&accf[b]);            // tile j's accumulator (complete, or abandoned on abort)
            }
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;        // column half of the tile
        const int et = threadIdx.x - 64;         // 0..255
        int j = 0;
        for (int64_t t = blockIdx.x; t < total; t += gridDim.x, j++) {
            int64_t m0, n0;
            int nw, kb0, kb1;
            tile_coords(t, m0, n0, nw, kb0, kb1);
            const int b = j & 1;
            const bool split = nslices > 1;
            asm volatile("bar.sync 1, 256;" ::: "memory");   // previous tile's coloff reads are done
            for (int c = et; c < BN; c += 256) {
                const int64_t n = n0 + c;
                coloff[c] = (c < nw && n < d.N) ? (split ? n : grp_off(d.cn, n)) : -1;
            }
            const int64_t m = m0 + q * 32 + lane;
            const bool mok = m < d.M;
            const int64_t roff = mok ? (split ? 0 : grp_off(d.cm, m)) : 0;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            bool ok = mbar_wait(&accf[b], (uint32_t)(j >> 1) & 1u);
            fence_after();
            ok = __all_sync(0xffffffffu, ok && !*abort_flag);
            if (!ok) *epi_abort = 1;
            // all eight epilogue warps take the same decision (only they write epi_abort)
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (*epi_abort) {
                *abort_flag = 1;
                if (lane == 0) atomicOr(err_flag, 1);
                break;
            }
            double *P = split ? partials + (t / ntiles) * d.M * d.N : nullptr;
#pragma unroll 1
            for (int cc = 0; cc < BN / 2; cc += 32) {
                const int c0 = half * (BN / 2) + cc;
                if (c0 >= nw) break;             // warp-uniform: past the tile's columns
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0), r);
                tmem_ld_wait();
                if (mok) {
                    if (split) {
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) {
                            const int64_t n = coloff[c0 + jj];
                            if (n >= 0) P[n * d.M + m] = f32_to_f64_pow2(__uint_as_float(r[jj]), 0, 0u);
                        }
                    } else {
                        // read-modify-write in two batches of 16 (loads issued before the stores)
                        store_batch_f32<16>(C, roff, coloff + c0, r, d.as, d.bcase);
                        store_batch_f32<16>(C, roff, coloff + c0 + 16, r + 16, d.as, d.bcase);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ---- grouped variant (two planes): the tiles of a batch of GEMMs, one per
// system, in one persistent launch.  Entry e owns the global tiles
// [e.tile0, e.tile0 + row tiles * e.n_tiles); its tensor maps, extents,
// output addressing and scale live in the entry (global memory), so the roles
// look the entry up by binary search for each tile.  Tiles of a system whose
// active flag is 0 are skipped by all three roles alike (the accumulator
// buffer index counts only the tiles worked), so converged systems cost
// nothing but the lookup.  No split K: the tile count of a batch fills the GPU.
__device__ __forceinline__ int grouped_entry(const GroupedGemm *__restrict__ tab, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_grouped_kernel(const GroupedGemm *__restrict__ tab, int n, int64_t total, const GroupedGemmParams gp,
                           const int *__restrict__ active, int *err_flag) {
    constexpr int NP = 2;
    using G = Cfg<NP, BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = smem;
    uint64_t *full = (uint64_t *)(smem + STAGES * G::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;             // [2]
    uint64_t *acce = accf + 2;                   // [2]
    uint32_t *tmem_slot = (uint32_t *)(acce + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *epi_abort = abort_flag + 1;
    int64_t *coloff = (int64_t *)(smem + STAGES * G::STAGE_BYTES + 1024);   // [BN]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 8);
        }
        *abort_flag = 0;
        *epi_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 2 * BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    // item t of entry e: K slice z (its K blocks [kb0, kb1)), row block, first column, width
    auto coords = [&](const GroupedGemm &e, int64_t t, int64_t &m0, int64_t &n0, int &nw, int &z, int &kb0,
                      int &kb1) {
        const int64_t per_slice = (e.M + BM - 1) / BM * e.n_tiles;
        const int64_t local = t - e.tile0;
        z = (int)(local / per_slice);
        const int64_t tile = local - (int64_t)z * per_slice;
        m0 = (tile / e.n_tiles) * BM;
        const int nb = (int)(tile % e.n_tiles);
        const ColSplit cs{e.cs_base, e.cs_extra};
        n0 = cs.n0(nb);
        nw = cs.width(nb);
        const int kb_total = (int)(e.Kp / BK);
        kb0 = z * e.kb_per;
        kb1 = kb0 + e.kb_per < kb_total ? kb0 + e.kb_per : kb_total;
    };

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;
            bool stop = false;
            int last = -1;
            for (int64_t t = blockIdx.x; t < total && !stop; t += gridDim.x) {
                const int ie = grouped_entry(tab, n, t);
                const GroupedGemm &e = tab[ie];
                if (!active[e.sys]) continue;
                int64_t m0, n0;
                int nw, z, kb0, kb1;
                coords(e, t, m0, n0, nw, z, kb0, kb1);
                const ColSplit cs{e.cs_base, e.cs_extra};
                const CUtensorMap *ma = reinterpret_cast<const CUtensorMap *>(&e.ma);
                const CUtensorMap *mb = reinterpret_cast<const CUtensorMap *>(nw == cs.wide() ? &e.mbw : &e.mbn);
                if (ie != last) {
                    // the entry's maps live in global memory: order them for the tensor-map proxy
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.ma) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.mbw) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.mbn) : "memory");
                    last = ie;
                }
                const uint32_t bytes = (uint32_t)(NP * (G::A_BYTES + nw * BK * 2));
                for (int kb = kb0; kb < kb1; kb++, g++) {
                    const int q = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (*abort_flag || !mbar_wait(&empty[q], ph ^ 1u)) {
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    uint8_t *st = tiles + q * G::STAGE_BYTES;
                    mbar_expect_tx(&full[q], bytes);
                    for (int p = 0; p < NP; p++) tma_load_3d(st + p * G::A_BYTES, ma, &full[q], kb * BK, (int)m0, p);
                    for (int p = 0; p < NP; p++)
                        tma_load_3d(st + NP * G::A_BYTES + p * G::B_BYTES, mb, &full[q], kb * BK, (int)n0, p);
                }
            }
            if (stop) {
                for (int64_t k = (g > STAGES ? g - STAGES : 0); k < g; k++)
                    mbar_wait(&full[k % STAGES], (uint32_t)(k / STAGES) & 1u);
                atomicOr(err_flag, 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int64_t g = 0;
            int j = 0;                           // tiles worked by this CTA
            for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
                if (*abort_flag) break;
                const GroupedGemm &e = tab[grouped_entry(tab, n, t)];
                if (!active[e.sys]) continue;
                int64_t m0, n0;
                int nw, z, kb0, kb1;
                coords(e, t, m0, n0, nw, z, kb0, kb1);
                const uint32_t idesc = idesc_bf16(BM, nw);
                const int b = j & 1;
                if (j >= 2) {
                    if (!mbar_wait(&acce[b], (uint32_t)((j >> 1) - 1) & 1u)) {
                        *abort_flag = 1;
                        atomicOr(err_flag, 1);
                    }
                    fence_after();
                }
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                for (int kb = kb0; kb < kb1 && !*abort_flag; kb++, g++) {
                    const int q = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (!mbar_wait(&full[q], ph)) {
                        *abort_flag = 1;
                        atomicOr(err_flag, 1);
                        break;
                    }
                    fence_after();
                    const uint32_t st = smem_u32(tiles + q * G::STAGE_BYTES);
                    for (int pr = 0; pr < gp.nprod; pr++) {
                        const uint32_t a0 = st + gp.prod_a[pr] * G::A_BYTES;
                        const uint32_t b0 = st + NP * G::A_BYTES + gp.prod_b[pr] * G::B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; kk++)
                            mma_bf16(dt, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                                     ((kb - kb0) | pr | kk) != 0);
                    }
                    mma_commit(&empty[q]);
                }
                mma_commit(&accf[b]);
                j++;
            }
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int et = threadIdx.x - 64;
        int j = 0;
        for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
            const GroupedGemm &e = tab[grouped_entry(tab, n, t)];
            if (!active[e.sys]) continue;        // uniform over the CTA
            int64_t m0, n0;
            int nw, z, kb0, kb1;
            coords(e, t, m0, n0, nw, z, kb0, kb1);
            const bool split = e.nslices > 1;
            const int b = j & 1;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            for (int c = et; c < BN; c += 256) {
                const int64_t nn = n0 + c;
                coloff[c] = (c < nw && nn < e.N) ? (split ? nn : grp_off(e.cn, nn)) : -1;
            }
            const int64_t m = m0 + q * 32 + lane;
            const bool mok = m < e.M;
            const int64_t roff = mok ? (split ? 0 : grp_off(e.cm, m)) : 0;
            double *P = split ? e.P + (int64_t)z * e.M * e.N : nullptr;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            bool ok = mbar_wait(&accf[b], (uint32_t)(j >> 1) & 1u);
            fence_after();
            ok = __all_sync(0xffffffffu, ok && !*abort_flag);
            if (!ok) *epi_abort = 1;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (*epi_abort) {
                *abort_flag = 1;
                if (lane == 0) atomicOr(err_flag, 1);
                break;
            }
#pragma unroll 1
            for (int cc = 0; cc < BN / 2; cc += 32) {
                const int c0 = half * (BN / 2) + cc;
                if (c0 >= nw) break;
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0), r);
                tmem_ld_wait();
                if (mok) {
                    if (split) {
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) {
                            const int64_t nn = coloff[c0 + jj];
                            if (nn >= 0) P[nn * e.M + m] = f32_to_f64_pow2(__uint_as_float(r[jj]), 0, 0u);
                        }
                    } else {
                        store_batch_f32<16>(e.C, roff, coloff + c0, r, e.as, e.bcase);
                        store_batch_f32<16>(e.C, roff, coloff + c0 + 16, r + 16, e.as, e.bcase);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
            j++;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ---- chunked-accumulation variant (the accurate split route, three planes)
// TMEM holds two 128 x BN fp32 accumulators.  The MMA issuer alternates
// between them every CH K blocks; eight epilogue warps drain the finished one
// into float-float (hi, lo) registers with an exact two-sum, so fp32 rounding
// only ever acts on CH*64-long partial sums.  Warp w (2..9) owns TMEM lanes
// 32*(w%4).. and the column half (w-2)/4 of the tile.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int NP, int BN, int STAGES, int CH>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_chunked_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBw,
                           const __grid_constant__ CUtensorMap mapBn, const TcGemmDesc d, double *__restrict__ C,
                           double *__restrict__ partials, int kb_per_split, const ColSplit cs, int *err_flag) {
    using G = Cfg<NP, BN, STAGES>;
    constexpr int HALF = BN / 2;                 // columns per epilogue warp
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = smem;
    uint64_t *full = (uint64_t *)(smem + STAGES * G::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;             // [2] accumulator b complete
    uint64_t *acce = accf + 2;                   // [2] accumulator b drained
    uint32_t *tmem_slot = (uint32_t *)(acce + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *consumed = abort_flag + 1;
    int64_t *coloff = (int64_t *)(smem + STAGES * G::STAGE_BYTES + 1024);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (int)((d.N + BN - 1) / BN);   // tiles past N would read padding only
    const int tile = blockIdx.x;
    const int64_t m0 = (int64_t)(tile / n_tiles) * BM;
    const int64_t n0 = cs.n0(tile % n_tiles);     // column tiles share N evenly (as the persistent kernel)
    const int nw = cs.width(tile % n_tiles);
    const int kb_total = (int)(d.Kp / BK);
    const int kb0 = (int)blockIdx.y * kb_per_split;
    const int kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
    const int kblocks = kb1 - kb0;
    const int nch = (kblocks + CH - 1) / CH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 8);              // one arrival per epilogue warp
        }
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 2 * BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < kblocks; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                uint8_t *st = tiles + s * G::STAGE_BYTES;
                mbar_expect_tx(&full[s], (uint32_t)(NP * (G::A_BYTES + nw * BK * 2)));
                for (int p = 0; p < NP; p++)
                    tma_load_3d(st + p * G::A_BYTES, &mapA, &full[s], (kb0 + kb) * BK, (int)m0, p);
                for (int q = 0; q < NP; q++)
                    tma_load_3d(st + NP * G::A_BYTES + q * G::B_BYTES, nw == cs.wide() ? &mapBw : &mapBn,
                                &full[s], (kb0 + kb) * BK, (int)n0, q);
                issued = kb + 1;
            }
            if (*abort_flag) {
                for (int kb = *consumed; kb < issued; kb++) mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u);
                atomicOr(err_flag, 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, nw);
            int committed = -1;              // last chunk whose accumulator was committed
            for (int kb = 0; kb < kblocks; kb++) {
                const int c = kb / CH, b = c & 1;
                const bool first = (kb % CH) == 0;
                if (first && c >= 2) {
                    // the epilogue must have drained this buffer's previous chunk
                    if (*abort_flag || !mbar_wait(&acce[b], (uint32_t)((c >> 1) - 1) & 1u)) {
                        *abort_flag = 1;
                        break;
                    }
                    fence_after();
                }
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&full[s], ph)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t st = smem_u32(tiles + s * G::STAGE_BYTES);
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                for (int pr = 0; pr < d.nprod; pr++) {
                    const uint32_t a0 = st + d.prod_a[pr] * G::A_BYTES;
                    const uint32_t b0 = st + NP * G::A_BYTES + d.prod_b[pr] * G::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; kk++)
                        mma_bf16(dt, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                                 !(first && pr == 0 && kk == 0));
                }
                mma_commit(&empty[s]);
                *consumed = kb + 1;
                if ((kb % CH) == CH - 1 || kb == kblocks - 1) {
                    mma_commit(&accf[b]);
                    committed = c;
                }
            }
            // on abort, still complete the pending chunks' barriers so the epilogue can finish
            for (int c = committed + 1; c < nch; c++) mma_commit(&accf[c & 1]);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;              // column half
        const int et = threadIdx.x - 64;            // 0..255
        for (int c = et; c < BN; c += 256) {
            const int64_t n = n0 + c;
            coloff[c] = (c < nw && n < d.N) ? grp_off(d.cn, n) : -1;
        }
        const int64_t m = m0 + q * 32 + lane;
        const bool mok = m < d.M;
        const int64_t roff = mok ? grp_off(d.cm, m) : 0;
        asm volatile("bar.sync 1, 256;" ::: "memory");
        float hi[HALF], lo[HALF];
#pragma unroll
        for (int j = 0; j < HALF; j++) { hi[j] = 0.f; lo[j] = 0.f; }
        bool good = true;
        for (int c = 0; c < nch; c++) {
            const int b = c & 1;
            bool ok = mbar_wait(&accf[b], (uint32_t)(c >> 1) & 1u);
            fence_after();
            ok = __all_sync(0xffffffffu, ok && !*abort_flag);
            if (!ok) {
                good = false;
                *abort_flag = 1;
                if (lane == 0) atomicOr(err_flag, 1);
                break;
            }
#pragma unroll
            for (int c0 = 0; c0 < HALF; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * HALF + c0), r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    float s2, e2;
                    two_sum(hi[c0 + j], __uint_as_float(r[j]), s2, e2);
                    hi[c0 + j] = s2;
                    lo[c0 + j] += e2;
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])) : "memory");
        }
        if (good && mok) {
            if (gridDim.y > 1) {
                double *P = partials + (int64_t)blockIdx.y * d.M * d.N;
#pragma unroll
                for (int j = 0; j < HALF; j++) {
                    const int64_t n = n0 + h * HALF + j;
                    if (h * HALF + j < nw && n < d.N) P[n * d.M + m] = f32_to_f64_pow2(hi[j], 0, 0u) + f32_to_f64_pow2(lo[j], 0, 0u);
                }
            } else {
#pragma unroll
                for (int j0 = 0; j0 < HALF; j0 += 16) {
                    double v[16];
                    int64_t co[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        co[j] = coloff[h * HALF + j0 + j];
                        v[j] = scale_f64(f32_to_f64_pow2(hi[j0 + j], 0, 0u) + f32_to_f64_pow2(lo[j0 + j], 0, 0u),
                                         d.as);
                    }
                    store_batch<16>(C, roff, co, v, d.bcase);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ---- exact-slice variant (the FP64-grade route, six planes)
// Stage s holds the six A slices (128 x 32 bf16 each) and the six B slices
// (BN x 32) of one 32-wide K block (SWIZZLE_64B).  The 21 slice products with
// weight g = s + t <= 5 accumulate in six TMEM accumulators, one per weight
// (columns g * BN ..): each holds integer multiples of 2^-7(g+2) below
// 6 * 128 * 2^(14 - 7(g+2)) after a 128-long K chunk (four K blocks), so its
// FP32 sums are exact.  After each chunk the eight epilogue warps drain weight
// g into float-float (hi, lo) registers (exact two-sum) as soon as that
// weight's MMAs of the chunk complete, and the MMA issuer starts weight g of
// the next chunk once its accumulator is drained.  The tile's value is
// alpha 2^(E_m + E_n) (hi + lo), E from the operands' row exponents.
constexpr int SBK = 32, SCHUNK = 4;           // K block, K blocks per exact chunk

__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset between 8-row groups (rows of 64 bytes)
    d |= (uint64_t)1 << 46;                     // descriptor version of tcgen05
    d |= (uint64_t)4 << 61;                     // SWIZZLE_64B
    return d;
}

template <int BN, int STAGES>
struct SlCfg {
    static constexpr int A_BYTES = BM * SBK * 2;
    static constexpr int B_BYTES = BN * SBK * 2;
    static constexpr int STAGE_BYTES = kSlices * (A_BYTES + B_BYTES);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 1024 /*barriers*/ + BN * 8;
};

__device__ __noinline__ double ldexp_slow(double x, int k) { return ldexp(x, k); }

// 2^k (hi + lo) in FP64: exact power-of-two re-encodings for the usual range
__device__ __forceinline__ double ff_to_f64_pow2(float hi, float lo, int k) {
    if (k > -500 && k < 500) return f32_to_f64_pow2(hi, k, 0u) + f32_to_f64_pow2(lo, k, 0u);
    return ldexp_slow((double)hi + (double)lo, k);
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_slices_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBw,
                          const __grid_constant__ CUtensorMap mapBn, const TcGemmDesc d, double *__restrict__ C,
                          double *__restrict__ partials, int kb_per_split, const ColSplit cs,
                          const int *__restrict__ expA, const int *__restrict__ expB, int *err_flag) {
    using G = SlCfg<BN, STAGES>;
    constexpr int HALF = BN / 2;                 // columns per epilogue warp
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = smem;
    uint64_t *full = (uint64_t *)(smem + STAGES * G::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;             // [kSlices] weight g of the chunk complete
    uint64_t *acce = accf + kSlices;             // [kSlices] weight g drained
    uint32_t *tmem_slot = (uint32_t *)(acce + kSlices);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *consumed = abort_flag + 1;
    int64_t *coloff = (int64_t *)(smem + STAGES * G::STAGE_BYTES + 1024);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (int)((d.N + BN - 1) / BN);
    const int tile = blockIdx.x;
    const int64_t m0 = (int64_t)(tile / n_tiles) * BM;
    const int64_t n0 = cs.n0(tile % n_tiles);
    const int nw = cs.width(tile % n_tiles);
    const int kb_total = (int)(d.Kp / SBK);
    const int kb0 = (int)blockIdx.y * kb_per_split;
    const int kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
    const int kblocks = kb1 - kb0;
    const int nch = (kblocks + SCHUNK - 1) / SCHUNK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int g = 0; g < kSlices; g++) {
            mbar_init(&accf[g], 1);
            mbar_init(&acce[g], 8);              // one arrival per epilogue warp
        }
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);              // kSlices * BN = 384 columns in use
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            const CUtensorMap *mb = nw == cs.wide() ? &mapBw : &mapBn;
            for (int kb = 0; kb < kblocks; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                uint8_t *st = tiles + s * G::STAGE_BYTES;
                mbar_expect_tx(&full[s], (uint32_t)(kSlices * (G::A_BYTES + nw * SBK * 2)));
                for (int p = 0; p < kSlices; p++)
                    tma_load_3d(st + p * G::A_BYTES, &mapA, &full[s], (kb0 + kb) * SBK, (int)m0, p);
                for (int q = 0; q < kSlices; q++)
                    tma_load_3d(st + kSlices * G::A_BYTES + q * G::B_BYTES, mb, &full[s], (kb0 + kb) * SBK, (int)n0,
                                q);
                issued = kb + 1;
            }
            if (*abort_flag) {
                for (int kb = *consumed; kb < issued; kb++) mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u);
                atomicOr(err_flag, 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, nw);
            int committed = -1;                  // last chunk whose weights were all committed
            bool stop = false;
            for (int kb = 0; kb < kblocks && !stop; kb++) {
                const int c = kb / SCHUNK;
                const bool first = (kb % SCHUNK) == 0;
                const bool last = (kb % SCHUNK) == SCHUNK - 1 || kb == kblocks - 1;
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&full[s], ph)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t st = smem_u32(tiles + s * G::STAGE_BYTES);
                for (int g = 0; g < kSlices; g++) {
                    if (first && c >= 1) {
                        // weight g of the previous chunk must be drained
                        if (*abort_flag || !mbar_wait(&acce[g], (uint32_t)((c - 1) & 1))) {
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        fence_after();
                    }
                    const uint32_t dt = tmem + (uint32_t)(g * BN);
                    for (int sa = 0; sa <= g; sa++) {
                        const uint32_t a0 = st + sa * G::A_BYTES;
                        const uint32_t b0 = st + kSlices * G::A_BYTES + (g - sa) * G::B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < SBK / 16; kk++)
                            mma_bf16(dt, sw64_desc(a0 + kk * 32), sw64_desc(b0 + kk * 32), idesc,
                                     !(first && sa == 0 && kk == 0));
                    }
                    if (last) mma_commit(&accf[g]);
                }
                if (stop) break;
                mma_commit(&empty[s]);
                *consumed = kb + 1;
                if (last) committed = c;
            }
            // on abort, still complete the pending chunks' barriers so the epilogue can finish
            for (int c = committed + 1; c < nch; c++)
                for (int g = 0; g < kSlices; g++) mma_commit(&accf[g]);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;              // column half
        const int et = threadIdx.x - 64;            // 0..255
        for (int c = et; c < BN; c += 256) {
            const int64_t n = n0 + c;
            coloff[c] = (c < nw && n < d.N) ? grp_off(d.cn, n) : -1;
        }
        const int64_t m = m0 + q * 32 + lane;
        const bool mok = m < d.M;
        const int64_t roff = mok && gridDim.y == 1 ? grp_off(d.cm, m) : 0;
        const int em = mok ? expA[m] - 1022 : 0;
        asm volatile("bar.sync 1, 256;" ::: "memory");
        float hi[HALF], lo[HALF];
#pragma unroll
        for (int j = 0; j < HALF; j++) { hi[j] = 0.f; lo[j] = 0.f; }
        bool good = true;
        for (int c = 0; c < nch && good; c++) {
#pragma unroll 1
            for (int g = 0; g < kSlices; g++) {
                bool ok = mbar_wait(&accf[g], (uint32_t)(c & 1));
                fence_after();
                ok = __all_sync(0xffffffffu, ok && !*abort_flag);
                if (!ok) {
                    good = false;
                    *abort_flag = 1;
                    if (lane == 0) atomicOr(err_flag, 1);
                    break;
                }
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * BN + h * HALF), r);
                tmem_ld_wait();
                fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[g])) : "memory");
#pragma unroll
                for (int j = 0; j < HALF; j++) {
                    float s2, e2;
                    two_sum(hi[j], __uint_as_float(r[j]), s2, e2);
                    hi[j] = s2;
                    lo[j] += e2;
                }
            }
        }
        if (good && mok) {
            if (gridDim.y > 1) {
                double *P = partials + (int64_t)blockIdx.y * d.M * d.N;
#pragma unroll
                for (int j = 0; j < HALF; j++) {
                    const int64_t n = n0 + h * HALF + j;
                    if (h * HALF + j < nw && n < d.N) P[n * d.M + m] = ff_to_f64_pow2(hi[j], lo[j], em + expB[n] - 1022);
                }
            } else {
#pragma unroll
                for (int j0 = 0; j0 < HALF; j0 += 16) {
                    double v[16];
                    int64_t co[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int c = h * HALF + j0 + j;
                        co[j] = coloff[c];
                        const int en = co[j] >= 0 ? expB[n0 + c] - 1022 : 0;
                        v[j] = co[j] >= 0 ? scale_f64(ff_to_f64_pow2(hi[j0 + j], lo[j0 + j], em + en), d.as) : 0.0;
                    }
                    store_batch<16>(C, roff, co, v, d.bcase);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3-D map over the planes [nplanes][rows][Kp] bf16 (rows unpadded: the
// box rows past `rows` read as zeros), box {64, box_rows, 1}
static bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t Kp, int nplanes, int box_rows,
                     int box_k = BK) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
    cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The dynamic shared-memory opt-in of a kernel holds per device: it is set once
// on each device the kernel runs on (bit `dev` of *done; a device index past 63
// sets it at every launch).  Setting it twice is harmless, so racing threads
// need no lock.
template <typename K>
static cudaError_t smem_opt_in(K *kernel, int bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    if (cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) return e;
    done.fetch_or(bit, std::memory_order_relaxed);
    return cudaSuccess;
}

template <int NP, int BN, int STAGES>
static cudaError_t launch_persistent(const TcGemmDesc &d, const void *A, const void *B, double *C, double *partials,
                                     int *err, cudaStream_t s) {
    using G = Cfg<NP, BN, STAGES>;
    static std::atomic<unsigned long long> opted{0};
    if (cudaError_t e = smem_opt_in(tc_gemm_persistent_kernel<NP, BN, STAGES>, G::SMEM, opted)) return e;
    if (d.Mp % BM || d.Kp % BK || d.Mp < d.M) return cudaErrorInvalidValue;
    const ColSplit cs = col_split(d.N, BN);
    CUtensorMap ma, mbw, mbn;
    if (!make_map(&ma, A, d.M, d.Kp, NP, BM) || !make_map(&mbw, B, d.N, d.Kp, NP, cs.wide()) ||
        !make_map(&mbn, B, d.N, d.Kp, NP, 16 * cs.base))
        return cudaErrorInvalidValue;
    const int64_t ntiles = (d.Mp / BM) * ((d.N + BN - 1) / BN);
    const int kb_total = (int)(d.Kp / BK);
    const int sk = d.splitk > 1 ? d.splitk : 1;
    const int per = (kb_total + sk - 1) / sk;
    const int zs = (kb_total + per - 1) / per;
    if (zs > 1 && !partials) return cudaErrorInvalidValue;
    const int64_t total = ntiles * zs;
    const int grid = (int)(total < 148 ? total : 148);
    tc_gemm_persistent_kernel<NP, BN, STAGES>
        <<<grid, 320, G::SMEM, s>>>(ma, mbw, mbn, d, C, partials, per, zs, ntiles, cs, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || zs == 1) return e;
    return launch_splitk_reduce(d.M, d.N, zs, partials, d.cm, d.cn, d.alpha, d.beta, C, s);
}

template <int NP, int BN, int STAGES, int CH>
static cudaError_t launch_chunked(const TcGemmDesc &d, const void *A, const void *B, double *C, double *partials,
                                  int *err, cudaStream_t s) {
    using G = Cfg<NP, BN, STAGES>;
    static std::atomic<unsigned long long> opted{0};
    if (cudaError_t e = smem_opt_in(tc_gemm_chunked_kernel<NP, BN, STAGES, CH>, G::SMEM, opted)) return e;
    if (d.Mp % BM || d.Kp % BK || d.Mp < d.M) return cudaErrorInvalidValue;
    const ColSplit cs = col_split(d.N, BN);
    CUtensorMap ma, mbw, mbn;
    if (!make_map(&ma, A, d.M, d.Kp, NP, BM) || !make_map(&mbw, B, d.N, d.Kp, NP, cs.wide()) ||
        !make_map(&mbn, B, d.N, d.Kp, NP, 16 * cs.base))
        return cudaErrorInvalidValue;
    const int64_t tiles = (d.Mp / BM) * ((d.N + BN - 1) / BN);
    if (tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const int kb_total = (int)(d.Kp / BK);
    const int sk = d.splitk > 1 ? d.splitk : 1;
    const int per = (kb_total + sk - 1) / sk;
    const int zs = (kb_total + per - 1) / per;
    if (zs > 1 && !partials) return cudaErrorInvalidValue;
    if (zs > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)tiles, (unsigned)zs);
    tc_gemm_chunked_kernel<NP, BN, STAGES, CH><<<grid, 320, G::SMEM, s>>>(ma, mbw, mbn, d, C, partials, per, cs, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || zs == 1) return e;
    return launch_splitk_reduce(d.M, d.N, zs, partials, d.cm, d.cn, d.alpha, d.beta, C, s);
}

template <int BN, int STAGES>
static cudaError_t launch_slices_gemm(const TcGemmDesc &d, const void *A, const void *B, double *C, double *partials,
                                     int *err, cudaStream_t s) {
    using G = SlCfg<BN, STAGES>;
    static std::atomic<unsigned long long> opted{0};
    if (cudaError_t e = smem_opt_in(tc_gemm_slices_kernel<BN, STAGES>, G::SMEM, opted)) return e;
    if (d.Mp % BM || d.Kp % 64 || d.Mp < d.M) return cudaErrorInvalidValue;
    const ColSplit cs = col_split(d.N, BN);
    CUtensorMap ma, mbw, mbn;
    if (!make_map(&ma, A, d.M, d.Kp, kSlices, BM, SBK) || !make_map(&mbw, B, d.N, d.Kp, kSlices, cs.wide(), SBK) ||
        !make_map(&mbn, B, d.N, d.Kp, kSlices, 16 * cs.base, SBK))
        return cudaErrorInvalidValue;
    const int *expA = reinterpret_cast<const int *>(static_cast<const char *>(A) + slice_plane_bytes(d.M, d.Kp));
    const int *expB = reinterpret_cast<const int *>(static_cast<const char *>(B) + slice_plane_bytes(d.N, d.Kp));
    const int64_t tiles = (d.Mp / BM) * ((d.N + BN - 1) / BN);
    if (tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const int kb_total = (int)(d.Kp / SBK);
    const int sk = d.splitk > 1 ? d.splitk : 1;
    // K slices hold whole exact chunks
    int per = (kb_total + sk - 1) / sk;
    per = (per + SCHUNK - 1) / SCHUNK * SCHUNK;
    const int zs = (kb_total + per - 1) / per;
    if (zs > 1 && !partials) return cudaErrorInvalidValue;
    if (zs > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)tiles, (unsigned)zs);
    tc_gemm_slices_kernel<BN, STAGES><<<grid, 320, G::SMEM, s>>>(ma, mbw, mbn, d, C, partials, per, cs, expA, expB, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || zs == 1) return e;
    return launch_splitk_reduce(d.M, d.N, zs, partials, d.cm, d.cn, d.alpha, d.beta, C, s);
}

}  // namespace tc

cudaError_t launch_convert_selftest(const double *in, int64_t n, float *mine, float *ref, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    convert_selftest_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, n, mine, ref);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long budget_cycles, int *timed_out, cudaStream_t s) {
    if (budget_cycles < 0 || budget_cycles > tc::kWaitBudget) return cudaErrorInvalidValue;
    tc::wait_selftest_kernel<<<1, 32, 0, s>>>(budget_cycles, timed_out);
    return cudaGetLastError();
}

bool split_lanes_along_k(const SplitDesc &d) {
    // lanes along K when K's innermost digit is the unit stride, or when
    // neither side has one and K's innermost stride is the smaller
    const int64_t unit = d.cplx ? 2 : 1;
    const bool k_unit = d.gk.nd >= 1 && d.gk.str[d.gk.nd - 1] == unit;
    const bool r_unit = d.gr.nd >= 1 && d.gr.str[d.gr.nd - 1] == unit;
    const int64_t ks = d.gk.nd >= 1 ? d.gk.str[d.gk.nd - 1] : 0, rs = d.gr.nd >= 1 ? d.gr.str[d.gr.nd - 1] : 0;
    return k_unit || (!r_unit && ks <= rs);
}

int grouped_split_vec_ok(const SplitDesc &d, const double *x) {
    // real, two or three planes, long K whose innermost digit is contiguous
    if (d.cplx || d.nplanes < 2 || d.nplanes > 3 || d.K < 512 || d.gk.nd < 1 || d.gk.str[d.gk.nd - 1] != 1)
        return 0;
    const int64_t kcols = d.kend ? d.kend : d.Kp;
    if (d.kdst % 8 || kcols % 8 || d.kdst + kcols > d.Kp || kcols < d.K) return 0;
    // the vector loads (four double2 per lane): 16-byte aligned runs of eight
    // inside the innermost digit (one digit: the tail takes the scalar loads)
    bool vec = ((uintptr_t)x & 15) == 0 && (d.gk.nd == 1 || d.gk.ext[d.gk.nd - 1] % 8 == 0);
    for (int q = 0; q + 1 < d.gk.nd; q++) vec = vec && d.gk.str[q] % 2 == 0;
    for (int q = 0; q < d.gr.nd; q++) vec = vec && d.gr.str[q] % 2 == 0;
    return vec ? 2 : 1;
}

int64_t grouped_split_vec_items(const SplitDesc &d) {
    const int64_t kcols = d.kend ? d.kend : d.Kp;
    return d.Rp * ((kcols + 1023) / 1024);
}

cudaError_t launch_grouped_split_vec(const GroupedSplit *tab, int n, int64_t total, const int *active,
                                     cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 7) / 8 < 148 * 16 ? (total + 7) / 8 : 148 * 16);
    grouped_split_vec_kernel<<<blocks, 256, 0, s>>>(tab, n, total, active);
    return cudaGetLastError();
}

cudaError_t launch_grouped_split(const GroupedSplit *tab, int n, int64_t total, bool lk, const int *active,
                                 cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 5 ? total : 148 * 5);
    if (lk) grouped_split_kernel<true><<<blocks, 256, 0, s>>>(tab, n, total, active);
    else grouped_split_kernel<false><<<blocks, 256, 0, s>>>(tab, n, total, active);
    return cudaGetLastError();
}

bool grouped_gemm_entry(GroupedGemm &g, const TcGemmDesc &d, const void *A, const void *B, double *C, int bn,
                        int nslices, double *P) {
    using namespace tc;
    if (d.nplanes_a != 2 || d.nplanes_b != 2 || d.Kp % BK || d.Kp < BK || d.M <= 0 || d.N <= 0 || bn < 64 ||
        bn > 256 || beta_case(d.beta) == 2 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return false;
    g = GroupedGemm{};
    const ColSplit cs = col_split(d.N, bn);
    if (!make_map(reinterpret_cast<CUtensorMap *>(&g.ma), A, d.M, d.Kp, 2, BM) ||
        !make_map(reinterpret_cast<CUtensorMap *>(&g.mbw), B, d.N, d.Kp, 2, cs.wide()) ||
        !make_map(reinterpret_cast<CUtensorMap *>(&g.mbn), B, d.N, d.Kp, 2, 16 * cs.base))
        return false;
    g.M = d.M;
    g.N = d.N;
    g.Kp = d.Kp;
    g.n_tiles = (int)((d.N + bn - 1) / bn);
    g.cs_base = cs.base;
    g.cs_extra = cs.extra;
    g.cm = d.cm;
    g.cn = d.cn;
    g.as = make_scale(d.alpha);
    g.bcase = beta_case(d.beta);
    // accumulating: each output element gets exactly one addition per launch
    // (K slices go through the partials), so a reduction in L2 gives the same
    // sum as a read-modify-write and spares the epilogue the loads' latency
    if (g.bcase == 1) g.bcase = 2;
    g.C = C;
    const int kb_total = (int)(d.Kp / BK);
    g.nslices = nslices > 1 ? nslices : 1;
    g.kb_per = (kb_total + g.nslices - 1) / g.nslices;
    g.nslices = (kb_total + g.kb_per - 1) / g.kb_per;   // no empty slice
    g.P = g.nslices > 1 ? P : nullptr;
    return g.nslices == 1 || P != nullptr;
}

cudaError_t launch_grouped_gemm(const GroupedGemm *tab, int n, int64_t total, int bn, const GroupedGemmParams &p,
                                const int *active, int *err_flag, cudaStream_t s) {
    using namespace tc;
    if (n <= 0 || total <= 0) return cudaSuccess;
    if (p.nprod < 1 || p.nprod > 8) return cudaErrorInvalidValue;
    const int grid = (int)(total < 148 ? total : 148);
    if (bn == 64) {
        using G = Cfg<2, 64, 4>;
        static std::atomic<unsigned long long> opted{0};
        if (cudaError_t e = smem_opt_in(tc_gemm_grouped_kernel<64, 4>, G::SMEM, opted)) return e;
        tc_gemm_grouped_kernel<64, 4><<<grid, 320, G::SMEM, s>>>(tab, n, total, p, active, err_flag);
    } else if (bn == 128) {
        using G = Cfg<2, 128, 3>;
        static std::atomic<unsigned long long> opted{0};
        if (cudaError_t e = smem_opt_in(tc_gemm_grouped_kernel<128, 3>, G::SMEM, opted)) return e;
        tc_gemm_grouped_kernel<128, 3><<<grid, 320, G::SMEM, s>>>(tab, n, total, p, active, err_flag);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcGemmDesc &d0, const void *Aplanes, const void *Bplanes, double *C, double *partials,
                           int *err_flag, cudaStream_t s) {
    if (d0.M <= 0 || d0.N <= 0) return cudaSuccess;
    TcGemmDesc d = d0;
    d.bcase = beta_case(d.beta);
    d.as = make_scale(d.alpha);
    if (d.nplanes_a != d.nplanes_b || d.nprod < 1 || (d.nprod > 8 && d.nplanes_a != kSlices))
        return cudaErrorInvalidValue;
    if (d.bcase == 2 && d.splitk <= 1) {
        // general beta: C *= beta first, then accumulate
        if (cudaError_t e = launch_scale_grp(d.M, d.N, d.cm, d.cn, d.beta, C, s)) return e;
        d.beta = 1.0;
        d.bcase = 1;
    }
    // the kernels' store mode: 0 store, 1 read-modify-write, 2 reductions
    if (d.bcase == 1 && d.red && d.splitk <= 1) d.bcase = 2;
    if (((uintptr_t)Aplanes & 1023) || ((uintptr_t)Bplanes & 1023) || d.Kp < 64) {
        // TMA needs 16-byte aligned bases; the planner hands out 256-byte aligned workspace
        if (((uintptr_t)Aplanes & 15) || ((uintptr_t)Bplanes & 15)) return cudaErrorMisalignedAddress;
    }
    if (d.nplanes_a == 2) {
        if (d.bn == 256) return tc::launch_persistent<2, 256, 2>(d, Aplanes, Bplanes, C, partials, err_flag, s);
        if (d.bn == 128) return tc::launch_persistent<2, 128, 3>(d, Aplanes, Bplanes, C, partials, err_flag, s);
        if (d.bn == 64) return tc::launch_persistent<2, 64, 4>(d, Aplanes, Bplanes, C, partials, err_flag, s);
    } else if (d.nplanes_a == 3) {
        // three planes: the accurate route, chunked float-float accumulation
        if (d.bn == 128) return tc::launch_chunked<3, 128, 2, 2>(d, Aplanes, Bplanes, C, partials, err_flag, s);
        if (d.bn == 64) return tc::launch_chunked<3, 64, 3, 2>(d, Aplanes, Bplanes, C, partials, err_flag, s);
    } else if (d.nplanes_a == kSlices) {
        // six exact slices: the FP64-grade route
        if (d.bn == 64) return tc::launch_slices_gemm<64, 3>(d, Aplanes, Bplanes, C, partials, err_flag, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ccb
