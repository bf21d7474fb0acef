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
// library holds it (kNoAllocPartials doubles, 32 KiB) until the process
// exits.  One block partial covers kElemsPerPartial elements of the o^2 v^2
// sum, so the largest system accepted has o^2 v^2 <= kNoAllocPartials *
// kElemsPerPartial (67,108,864); larger ones are rejected with
// CC_ERR_INVALID_ARG.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/cc.h"

namespace {

constexpr int kNoAllocPartials = 4096;
constexpr int64_t kElemsPerPartial = 16384;   // 256 threads x 64 elements
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kNoAllocPartials];

// One block per partial: sum over its kElemsPerPartial elements of
// V[ijab] (1/4 t2[ijab] + 1/2 t1[ia] t1[jb]), fixed summation order.
__global__ void __launch_bounds__(256) energy_partials_noalloc(int o, int v, const double *V, const double *t1,
                                                               const double *t2, int64_t n, double *partials) {
    __shared__ double sh[256];
    const int64_t base = (int64_t)blockIdx.x * kElemsPerPartial;
    double s = 0.0;
    for (int64_t e = base + threadIdx.x; e < base + kElemsPerPartial && e < n; e += 256) {
        double w = 0.25 * t2[e];
        if (t1) {
            int64_t x = e;
            const int b = (int)(x % v); x /= v;
            const int a = (int)(x % v); x /= v;
            const int j = (int)(x % o); x /= o;
            const int i = (int)x;
            w += 0.5 * t1[(int64_t)i * v + a] * t1[(int64_t)j * v + b];
        }
        s = fma(V[e], w, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) energy_reduce_noalloc(const double *partials, int count, double *e_dev) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < count; k += 256) s += partials[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        e_dev[0] = sh[0];
        e_dev[1] = 0.0;
    }
}

std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

}  // namespace

// message for cc_last_error() (defined with the rest of the C ABI)
void ccb_set_last_error(const std::string &msg);

extern "C" {

// The device address of the static partials array: host code only holds a
// stand-in for it, so it is looked up once per device (with that device
// current) through cudaGetSymbolAddress.
static cc_status scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { ccb_set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return CC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { ccb_set_last_error("device index out of range"); return CC_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_partials);
        if (e != cudaSuccess || !p) {
            ccb_set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return CC_ERR_CUDA;
        }
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return CC_OK;
}

cc_status cc_energy_noalloc(int o, int v, const cc_integrals *ints, const cc_amps *amps, double *e_dev,
                            void *stream) {
    if (o < 1 || v < 1) { ccb_set_last_error("o and v must be >= 1"); return CC_ERR_INVALID_ARG; }
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
    energy_partials_noalloc<<<(unsigned)parts, 256, 0, s>>>(o, v, (const double *)ints->oovv, (const double *)amps->t1,
                                                            (const double *)amps->t2, n, scratch);
    energy_reduce_noalloc<<<1, 256, 0, s>>>(scratch, (int)parts, e_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ccb_set_last_error(std::string("launch: ") + cudaGetErrorString(e)); return CC_ERR_CUDA; }
    return CC_OK;
}

}  // extern "C"
