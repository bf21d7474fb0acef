// tc_gemm.cu -- split-bf16 route of the bulk contractions (sm_103a):
//   split_bf16   FP64 strided view -> K-major bf16 planes (hi, mid, lo), the
//                TTGT transpose fused into the precision split
//   tc_gemm      tcgen05 GEMM over the plane products, FP32 accumulation in
//                TMEM, FP64 epilogue into the output
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

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

// One block per row (grid-stride over rows), each thread 4 consecutive columns.
__global__ void __launch_bounds__(256) split_bf16_kernel(const SplitDesc d, const double *__restrict__ x,
                                                         __nv_bfloat16 *__restrict__ planes) {
    const int64_t plane_elems = d.Rp * d.Kp;
    for (int64_t r = blockIdx.x; r < d.Rp; r += gridDim.x) {
        const bool row_ok = r < d.R;
        const int64_t roff = row_ok ? grp_off(d.gr, r) : 0;
        for (int64_t k0 = (int64_t)threadIdx.x * 4; k0 < d.Kp; k0 += 1024) {
            // digits of k0 in the K group, advanced as an odometer
            int dig[6];
            int64_t coff = 0;
            {
                int64_t t = k0 < d.K ? k0 : 0;
                for (int q = d.gk.nd - 1; q >= 0; q--) {
                    dig[q] = (int)(t % d.gk.ext[q]);
                    t /= d.gk.ext[q];
                    coff += dig[q] * d.gk.str[q];
                }
            }
            __align__(8) __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t k = k0 + j;
                double val = 0.0;
                if (row_ok && k < d.K) {
                    val = __ldg(x + roff + coff);
                    for (int q = d.gk.nd - 1; q >= 0; q--) {
                        coff += d.gk.str[q];
                        if (++dig[q] < d.gk.ext[q]) break;
                        coff -= dig[q] * d.gk.str[q];
                        dig[q] = 0;
                    }
                }
                h[j] = __double2bfloat16(val);
                double r1 = val - (double)__bfloat162float(h[j]);
                m[j] = __double2bfloat16(r1);
                double r2 = r1 - (double)__bfloat162float(m[j]);
                l[j] = __double2bfloat16(r2);
            }
            // Kp is a multiple of 64, so the 4 columns are always in range
            __nv_bfloat16 *p0 = planes + r * d.Kp + k0;
            *reinterpret_cast<uint2 *>(p0) = *reinterpret_cast<uint2 *>(h);
            *reinterpret_cast<uint2 *>(p0 + plane_elems) = *reinterpret_cast<uint2 *>(m);
            if (d.nplanes == 3) *reinterpret_cast<uint2 *>(p0 + 2 * plane_elems) = *reinterpret_cast<uint2 *>(l);
        }
    }
}

cudaError_t launch_split_bf16(const SplitDesc &d, const double *x, void *planes, cudaStream_t s) {
    if (d.Kp % 64 || d.Rp <= 0 || d.nplanes < 2 || d.nplanes > 3) return cudaErrorInvalidValue;
    int64_t blocks = d.Rp < 148 * 32 ? d.Rp : 148 * 32;
    split_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, x, (__nv_bfloat16 *)planes);
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcGemmDesc &d, const void *Aplanes, const void *Bplanes, double *C, int *err_flag,
                           cudaStream_t s) {
    (void)d; (void)Aplanes; (void)Bplanes; (void)C; (void)err_flag; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace ccb
