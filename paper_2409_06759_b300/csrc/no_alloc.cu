// no_alloc.cu -- cc_energy_noalloc: the CC energy for callers that cannot
// allocate device memory.
//
// Some callers run inside a host application whose memory policy forbids
// cudaMalloc/cudaFree on the calling thread (a custom allocator owns the
// device heap, or the call sits in a region where allocation is not allowed
// or would synchronise the device).  cc_energy needs a few KiB of scratch
// for its block partial sums, which those callers would have to carve out of
// a workspace they allocate.  This variant keeps that scratch in a
// file-scope device array instead, so the caller passes only inputs and the
// output.
//
// The array is a fixed part of the library image: every GPU that loads the
// library holds it (2 x kNoAllocPartials doubles, 64 KiB: real parts, then
// imaginary parts) until the process exits.  One block partial covers
// kElemsPerPartial elements of the o^2 v^2 sum, so the largest system
// accepted has o^2 v^2 <= kNoAllocPartials * kElemsPerPartial (67,108,864)
// for either dtype; larger ones are rejected with CC_ERR_INVALID_ARG.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/cc.h"

namespace {

constexpr int kNoAllocPartials = 4096;
constexpr int64_t kElemsPerPartial = 16384;   // 256 threads x 64 elements

static __device__ __align__(256) double g_energy_partials[2 * kNoAllocPartials];

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per partial: sum over its kElemsPerPartial elements of
// V[ijab] (1/4 t2[ijab] + 1/2 t1[ia] t1[jb]), fixed summation order.  The
// element index fits 32 bits (o^2 v^2 <= 67,108,864), so (i, j, a, b) come
// from 32-bit divisions.  Complex: the same polynomial in complex arithmetic
// (no conjugation), real parts to partials[k], imaginary parts to
// partials[kNoAllocPartials + k].
template <bool CPLX>
__global__ void __launch_bounds__(256) energy_partials_noalloc(uint32_t o, uint32_t v, const double *V,
                                                               const double *t1, const double *t2, uint32_t n,
                                                               double *partials) {
    if (blockIdx.x >= (unsigned)kNoAllocPartials) return;   // second guard behind the host's size check
    __shared__ double sh[2][256];
    const uint32_t base = blockIdx.x * (uint32_t)kElemsPerPartial;
    const uint32_t end = min(n, base + (uint32_t)kElemsPerPartial);
    double sr = 0.0, si = 0.0;
    for (uint32_t e = base + threadIdx.x; e < end; e += 256) {
        uint32_t x = e;
        const uint32_t b = x % v; x /= v;
        const uint32_t a = x % v; x /= v;
        const uint32_t j = x % o;
        const uint32_t i = x / o;
        if constexpr (!CPLX) {
            double w = 0.25 * t2[e];
            if (t1) w += 0.5 * t1[i * v + a] * t1[j * v + b];
            sr = fma(V[e], w, sr);
        } else {
            const double2 *V2 = reinterpret_cast<const double2 *>(V);
            const double2 *t12 = reinterpret_cast<const double2 *>(t1);
            const double2 *t22 = reinterpret_cast<const double2 *>(t2);
            const double2 tt = t22[e];
            double2 w = make_double2(0.25 * tt.x, 0.25 * tt.y);
            if (t1) {
                const double2 p = cmul(t12[i * v + a], t12[j * v + b]);
                w.x += 0.5 * p.x;
                w.y += 0.5 * p.y;
            }
            const double2 r = cmul(V2[e], w);
            sr += r.x;
            si += r.y;
        }
    }
    sh[0][threadIdx.x] = sr;
    sh[1][threadIdx.x] = si;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sh[0][0];
        if (CPLX) partials[kNoAllocPartials + blockIdx.x] = sh[1][0];
    }
}

// e_dev[0] = sum of the real partials, e_dev[1] = sum of the imaginary ones
// (0 for real inputs), in a fixed order.
__global__ void __launch_bounds__(256) energy_reduce_noalloc(const double *partials, int count, int cplx,
                                                             double *e_dev) {
    __shared__ double sh[2][256];
    count = min(count, kNoAllocPartials);
    double sr = 0.0, si = 0.0;
    for (int k = threadIdx.x; k < count; k += 256) {
        sr += partials[k];
        if (cplx) si += partials[kNoAllocPartials + k];
    }
    sh[0][threadIdx.x] = sr;
    sh[1][threadIdx.x] = si;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        e_dev[0] = sh[0][0];
        e_dev[1] = sh[1][0];
    }
}

}  // namespace

// message for cc_last_error() (defined with the rest of the C ABI)
void ccb_set_last_error(const std::string &msg);

extern "C" {

// The device address of the static partials array on the current device.
// Host code only holds a stand-in for the array, so the address is looked up
// through cudaGetSymbolAddress, with the caller's device current, on every
// call (no allocation; cheap next to the two launches), so a device reset
// between calls cannot leave a stale address behind.  The first lookup on a
// device may load the library's device code there.
static cc_status scratch_address(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energy_partials);
    if (e != cudaSuccess || !p) {
        ccb_set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return CC_ERR_CUDA;
    }
    *out = (double *)p;
    return CC_OK;
}

cc_status cc_energy_noalloc(int o, int v, cc_dtype dtype, const cc_integrals *ints, const cc_amps *amps,
                            double *e_dev, void *stream) {
    if (o < 1 || v < 1) { ccb_set_last_error("o and v must be >= 1"); return CC_ERR_INVALID_ARG; }
    if (dtype != CC_F64 && dtype != CC_C128) { ccb_set_last_error("dtype must be CC_F64 or CC_C128"); return CC_ERR_INVALID_ARG; }
    const int64_t n = (int64_t)o * o * v * v;
    const int64_t parts = (n + kElemsPerPartial - 1) / kElemsPerPartial;
    if (parts > kNoAllocPartials) {
        ccb_set_last_error("o^2 v^2 = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                           std::to_string((int64_t)kNoAllocPartials * kElemsPerPartial) + " elements");
        return CC_ERR_INVALID_ARG;
    }
    if (!ints || !amps || !e_dev || !ints->oovv || !amps->t2) {
        ccb_set_last_error("energy needs the oovv block, t2 and e_dev");
        return CC_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    cc_status st = scratch_address(&scratch);
    if (st != CC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int cplx = dtype == CC_C128;
    if (cplx)
        energy_partials_noalloc<true><<<(unsigned)parts, 256, 0, s>>>(
            (uint32_t)o, (uint32_t)v, (const double *)ints->oovv, (const double *)amps->t1,
            (const double *)amps->t2, (uint32_t)n, scratch);
    else
        energy_partials_noalloc<false><<<(unsigned)parts, 256, 0, s>>>(
            (uint32_t)o, (uint32_t)v, (const double *)ints->oovv, (const double *)amps->t1,
            (const double *)amps->t2, (uint32_t)n, scratch);
    energy_reduce_noalloc<<<1, 256, 0, s>>>(scratch, (int)parts, cplx, e_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ccb_set_last_error(std::string("launch: ") + cudaGetErrorString(e)); return CC_ERR_CUDA; }
    return CC_OK;
}

}  // extern "C"
