// kernels.cu -- FP64 kernels of the TTGT residual path (sm_103a):
//   gemm_f64     FP64 SIMT GEMM with generalised (mixed-radix) output addressing
//   denom/jacobi/energy/dot reductions and the DIIS solve of the iteration
#include <cstdint>
#include <cuda_runtime.h>

#include "grouped.cuh"
#include "kernels.h"
#include "scalar.cuh"

namespace ccb {

__global__ void zero_kernel(double *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

cudaError_t launch_zero(double *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    zero_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ scale_grp
// C(m,n) *= beta over an output addressed by two mixed-radix groups (applies a
// general beta before an accumulating epilogue; the planner itself only emits
// beta = 0 or 1)
__device__ __forceinline__ int64_t grp_offset(const Grp &g, int64_t x);

template <typename T>
__global__ void __launch_bounds__(256) scale_grp_kernel(int64_t M, int64_t N, const Grp cm, const Grp cn, double beta,
                                                        T *__restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = e / M, m = e - n * M;
        T *p = C + grp_offset(cm, m) + grp_offset(cn, n);
        *p = beta == 0.0 ? zero<T>() : scal(beta, *p);     // beta = 0 clears (whatever was there)
    }
}

template <typename T>
static cudaError_t scale_grp_t(int64_t M, int64_t N, const Grp &cm, const Grp &cn, double beta, T *C, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    int64_t blocks = (M * N + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    scale_grp_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(M, N, cm, cn, beta, C);
    return cudaGetLastError();
}

cudaError_t launch_scale_grp(int64_t M, int64_t N, const Grp &cm, const Grp &cn, double beta, double *C, cudaStream_t s) {
    return scale_grp_t<double>(M, N, cm, cn, beta, C, s);
}

// --------------------------------------------------------------- gemm_f64
// 64x64 output tile, BK = 16, 256 threads as 16x16, each thread a 4x4
// strided micro-tile.  Operand tiles go global -> registers -> shared memory
// (k-major, padded), double-buffered through registers.  The FP64 pipe of
// sm_103a is narrow, so the kernel is built to keep it issuing: 16 DFMA per
// 8 shared loads.
constexpr int GBM = 64, GBN = 64, GBK = 16, GPAD = 1;

__device__ __forceinline__ int64_t grp_offset(const Grp &g, int64_t x) {
    if (g.nd == 1) return x * g.str[0];
    int64_t off = 0;
    for (int k = g.nd - 1; k >= 0; k--) {
        int64_t q = x / g.ext[k];
        off += (x - q * g.ext[k]) * g.str[k];
        x = q;
    }
    return off;
}

// CT: compute type (T, or float for FP64 data multiplied in FP32)
template <typename T, typename CT, bool A_KCONTIG, bool B_KCONTIG>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmF64Desc d, const T *__restrict__ A,
                                                       const T *__restrict__ B, T *__restrict__ C,
                                                       T *__restrict__ partials, int thread_m_fast, int64_t kchunk) {
    __shared__ CT As[GBK][GBM + GPAD];
    __shared__ CT Bs[GBK][GBN + GPAD];
    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.x * GBM;
    const int64_t n0 = (int64_t)blockIdx.y * GBN;
    const int tm = thread_m_fast ? (tid & 15) : (tid >> 4);
    const int tn = thread_m_fast ? (tid >> 4) : (tid & 15);

    CT ra[4], rb[4];
    auto load_tiles = [&](int64_t k0, int64_t klim) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int e = tid + 256 * r;
            int mm, kk;
            if (A_KCONTIG) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
            int64_t gm = m0 + mm, gk = k0 + kk;
            ra[r] = (gm < d.M && gk < klim) ? down<CT>(cj(ld(A + gm * d.sAm + gk * d.sAk), d.conj_a)) : zero<CT>();
            int nn;
            if (B_KCONTIG) { kk = e & 15; nn = e >> 4; } else { nn = e & 63; kk = e >> 6; }
            int64_t gn = n0 + nn;
            gk = k0 + kk;
            rb[r] = (gn < d.N && gk < klim) ? down<CT>(cj(ld(B + gk * d.sBk + gn * d.sBn), d.conj_b)) : zero<CT>();
        }
    };
    auto store_tiles = [&]() {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int e = tid + 256 * r;
            if (A_KCONTIG) As[e & 15][e >> 4] = ra[r]; else As[e >> 6][e & 63] = ra[r];
            if (B_KCONTIG) Bs[e & 15][e >> 4] = rb[r]; else Bs[e >> 6][e & 63] = rb[r];
        }
    };

    CT acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = zero<CT>();

    // K slice of this CTA (the whole K unless split)
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = kbeg + kchunk < d.K ? kbeg + kchunk : d.K;
    load_tiles(kbeg, kend);
    for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
        __syncthreads();
        store_tiles();
        __syncthreads();
        if (k0 + GBK < kend) load_tiles(k0 + GBK, kend);
#pragma unroll
        for (int k = 0; k < GBK; k++) {
            CT a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][tm + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[k][tn + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
    }
    if (gridDim.z > 1) {
        // split K: raw partial sums, [z][n][m]
        T *P = partials + (int64_t)blockIdx.z * d.M * d.N;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t m = m0 + tm + 16 * i, n = n0 + tn + 16 * j;
                if (m < d.M && n < d.N) P[n * d.M + m] = up(acc[i][j]);
            }
        return;
    }
    // the tile's row and column offsets, decomposed once per CTA
    __shared__ int64_t s_ro[GBM], s_co[GBN];
    __syncthreads();
    if (tid < GBM) s_ro[tid] = m0 + tid < d.M ? grp_offset(d.cm, m0 + tid) : 0;
    else if (tid < GBM + GBN) s_co[tid - GBM] = n0 + tid - GBM < d.N ? grp_offset(d.cn, n0 + tid - GBM) : 0;
    __syncthreads();
    int64_t ro[4], co[4];
    bool rv[4], cv[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        rv[i] = m0 + tm + 16 * i < d.M;
        ro[i] = s_ro[tm + 16 * i];
        cv[i] = n0 + tn + 16 * i < d.N;
        co[i] = s_co[tn + 16 * i];
    }
    // beta is 0 or 1 here (a general beta was applied to C beforehand); the
    // branch is taken once, so the FP64 add exists only on the accumulating side
    if (d.bcase == 0) {
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (rv[i] && cv[j]) C[ro[i] + co[j]] = epi_scale(acc[i][j], d.as);
    } else if (d.red) {
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (rv[i] && cv[j]) red_add(C + ro[i] + co[j], epi_scale(acc[i][j], d.as));
    } else {
        T old[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) old[i][j] = (rv[i] && cv[j]) ? C[ro[i] + co[j]] : zero<T>();
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (rv[i] && cv[j]) C[ro[i] + co[j]] = add(epi_scale(acc[i][j], d.as), old[i][j]);
    }
}

// ------------------------------------------------------------ packed pairs
__device__ __forceinline__ int64_t pair_start(int64_t p, int64_t n) { return p * (2 * n - p - 1) / 2; }
// (p, q), p < q, of the packed index P
__device__ __forceinline__ void pair_of(int64_t P, int64_t n, int64_t &p, int64_t &q) {
    const double b = 2.0 * (double)n - 1.0;
    int64_t x = (int64_t)((b - sqrt(b * b - 8.0 * (double)P)) * 0.5);
    if (x < 0) x = 0;
    while (x + 1 < n && pair_start(x + 1, n) <= P) x++;
    while (x > 0 && pair_start(x, n) > P) x--;
    p = x;
    q = P - pair_start(x, n) + x + 1;
}

__global__ void __launch_bounds__(256) pack_pairs_kernel(const PackDesc d, const double *__restrict__ src,
                                                         double *__restrict__ dst) {
    const int64_t total = d.rows * d.P2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = e / d.P2, J = e - I * d.P2;
        int64_t p, q, r, u;
        pair_of(d.row0 + I, d.n1, p, q);
        pair_of(J, d.n2, r, u);
        dst[e] = d.scale * __ldg(src + (p - d.pbase) * d.s0 + q * d.s1 + r * d.s2 + u * d.s3);
    }
}

__global__ void __launch_bounds__(256) unpack_pairs_kernel(const UnpackDesc d, const double *__restrict__ C,
                                                           double *__restrict__ out) {
    const int64_t total = d.ext[0] * d.ext[1] * d.ext[2] * d.ext[3];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t dig[4], x = e, off = 0;
        for (int k = 3; k >= 0; k--) {
            dig[k] = x % d.ext[k];
            x /= d.ext[k];
            off += dig[k] * d.ostr[k];
        }
        const int64_t a1 = dig[d.da1], a2 = dig[d.da2], b1 = dig[d.db1], b2 = dig[d.db2];
        double val = 0.0;
        if (a1 != a2 && b1 != b2) {
            const int64_t pa = a1 < a2 ? pair_start(a1, d.nA) + a2 - a1 - 1 : pair_start(a2, d.nA) + a1 - a2 - 1;
            const int64_t pb = b1 < b2 ? pair_start(b1, d.nB) + b2 - b1 - 1 : pair_start(b2, d.nB) + b1 - b2 - 1;
            val = __ldg(C + pa * d.cA + pb * d.cB);
            if ((a1 > a2) != (b1 > b2)) val = -val;
        }
        double r = scale_f64(val, d.as);
        if (d.bcase != 0) r += out[off];           // a general beta was applied to out before
        out[off] = r;
    }
}

// Amplitude packing.  pack: one block per packed row P(i, j), i < j (found
// once per block); the block walks a = 0..v-2 and its lanes the run b = a+1..
// v-1, which is contiguous in both arrays.  unpack: one block per full row
// (i, j); column (a, b) reads packed[P(min)][P(a, b) or P(b, a)] with the sign
// of the two swaps, and i = j or a = b write exact zeros.
template <typename T>
__global__ void __launch_bounds__(256) pack_t2_kernel(int o, int v, const T *__restrict__ full, T *__restrict__ packed) {
    const int64_t P2 = (int64_t)v * (v - 1) / 2;
    const int64_t prow = blockIdx.x;
    int64_t i, j;
    pair_of(prow, o, i, j);
    const T *src = full + (i * o + j) * (int64_t)v * v;
    T *dst = packed + prow * P2;
    for (int a = 0; a + 1 < v; a++) {
        const int64_t pa = pair_start(a, v) - a - 1;                 // + b gives P(a, b)
        for (int b = a + 1 + (int)threadIdx.x; b < v; b += blockDim.x) dst[pa + b] = src[(int64_t)a * v + b];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) unpack_t2_kernel(int o, int v, const T *__restrict__ packed, T *__restrict__ full) {
    const int64_t P2 = (int64_t)v * (v - 1) / 2;
    const uint32_t row = blockIdx.x, i = row / (uint32_t)o, j = row - i * (uint32_t)o;
    const uint32_t ncol = (uint32_t)v * (uint32_t)v;
    T *dst = full + (int64_t)row * ncol;
    if (i == j) {
        for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) dst[c] = zero<T>();
        return;
    }
    const int64_t pij = i < j ? pair_start(i, o) + j - i - 1 : pair_start(j, o) + i - j - 1;
    const bool nrow = i > j;
    const T *src = packed + pij * P2;
    for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) {
        const uint32_t a = c / (uint32_t)v, b = c - a * (uint32_t)v;
        T x = zero<T>();
        if (a != b) {
            const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
            x = src[pair_start(lo, v) + hi - lo - 1];
            if (nrow != (a > b)) x = neg(x);
        }
        dst[c] = x;
    }
}

cudaError_t launch_pack_t2(int o, int v, int cplx, const double *full, double *packed, cudaStream_t s) {
    if (o < 2 || v < 2) return cudaSuccess;
    const unsigned rows = (unsigned)((int64_t)o * (o - 1) / 2);
    if (cplx)
        pack_t2_kernel<double2><<<rows, 256, 0, s>>>(o, v, reinterpret_cast<const double2 *>(full),
                                                     reinterpret_cast<double2 *>(packed));
    else
        pack_t2_kernel<double><<<rows, 256, 0, s>>>(o, v, full, packed);
    return cudaGetLastError();
}

cudaError_t launch_unpack_t2(int o, int v, int cplx, const double *packed, double *full, cudaStream_t s) {
    if (o < 1 || v < 1) return cudaSuccess;
    const unsigned rows = (unsigned)((int64_t)o * o);
    if (cplx)
        unpack_t2_kernel<double2><<<rows, 256, 0, s>>>(o, v, reinterpret_cast<const double2 *>(packed),
                                                       reinterpret_cast<double2 *>(full));
    else
        unpack_t2_kernel<double><<<rows, 256, 0, s>>>(o, v, packed, full);
    return cudaGetLastError();
}

cudaError_t launch_pack_pairs(const PackDesc &d, const double *src, double *dst, cudaStream_t s) {
    if (d.row0 < 0 || d.rows < 0 || d.row0 + d.rows > d.P1) return cudaErrorInvalidValue;
    const int64_t total = d.rows * d.P2;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    pack_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_unpack_pairs(const UnpackDesc &d0, const double *C, double *out, cudaStream_t s) {
    UnpackDesc d = d0;
    d.bcase = beta_case(d.beta);
    d.as = make_scale(d.alpha);
    if (d.bcase == 2) {
        // out *= beta over the 4-index view first (rows of the two outer indices)
        Grp gm{2, {d.ext[0], d.ext[1]}, {d.ostr[0], d.ostr[1]}}, gn{2, {d.ext[2], d.ext[3]}, {d.ostr[2], d.ostr[3]}};
        if (cudaError_t e = launch_scale_grp(d.ext[0] * d.ext[1], d.ext[2] * d.ext[3], gm, gn, d.beta, out, s)) return e;
        d.beta = 1.0;
        d.bcase = 1;
    }
    const int64_t total = d.ext[0] * d.ext[1] * d.ext[2] * d.ext[3];
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    unpack_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, C, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ rows_gemm
// offset of a mixed-radix index below 2^32 with 32-bit divisions
__device__ __forceinline__ int64_t grp_offset32(const Grp &g, uint32_t x) {
    int64_t off = 0;
    for (int k = g.nd - 1; k >= 0; k--) {
        const uint32_t e = (uint32_t)g.ext[k];
        const uint32_t q = x / e;
        off += (int64_t)(x - q * e) * g.str[k];
        x = q;
    }
    return off;
}

// resident blocks per SM the accumulators allow without spilling
template <typename CT, int NC> constexpr int rows_min_blocks() {
    // FP32: the 24- and 32-column instances need more than 85 registers with the
    // K-contiguous path beside the row path
    return sizeof(CT) == 4 ? ((NC <= 16 || NC == 40) ? 3 : 2) : (NC <= 24 ? 3 : NC <= 48 ? 2 : 1);
}

// acc[c] += a * y[c] over a row of NC values in shared memory (16-byte aligned),
// read four floats or two doubles at a time: one shared load per 4 (2) FMAs
template <int NC> __device__ __forceinline__ void row_fma(float a, const float *y, float *acc) {
    const float4 *y4 = reinterpret_cast<const float4 *>(y);
#pragma unroll
    for (int c = 0; c < NC / 4; c++) {
        const float4 v = y4[c];
        acc[4 * c] = fmaf(a, v.x, acc[4 * c]);
        acc[4 * c + 1] = fmaf(a, v.y, acc[4 * c + 1]);
        acc[4 * c + 2] = fmaf(a, v.z, acc[4 * c + 2]);
        acc[4 * c + 3] = fmaf(a, v.w, acc[4 * c + 3]);
    }
}
template <int NC> __device__ __forceinline__ void row_fma(double a, const double *y, double *acc) {
    const double2 *y2 = reinterpret_cast<const double2 *>(y);
#pragma unroll
    for (int c = 0; c < NC / 2; c++) {
        const double2 v = y2[c];
        acc[2 * c] = fma(a, v.x, acc[2 * c]);
        acc[2 * c + 1] = fma(a, v.y, acc[2 * c + 1]);
    }
}

// Y rows [k0, k0 + 64) by columns [c0, c0 + NC) of a narrow GEMM, staged in
// shared memory with the X offsets of those K indices and the C offsets of
// those columns (block-wide; the caller places barriers around it)
template <typename CT, int NC> struct RowsSmem {
    __align__(16) CT ys[64 * NC];
    int64_t xko[64], cco[NC];
};
template <typename CT, int NC>
__device__ __forceinline__ void rows_stage(const RowsGemmDesc &d, const double *__restrict__ Y, int k0, int c0,
                                           RowsSmem<CT, NC> &S) {
    for (int e = threadIdx.x; e < 64 * NC; e += blockDim.x) {
        const int k = e / NC, c = e - k * NC;
        // K and the column count are ints: 32-bit digit divisions
        S.ys[e] = (k0 + k < d.K && c0 + c < d.nc)
                      ? down<CT>(__ldg(Y + grp_offset32(d.yk, (uint32_t)(k0 + k)) +
                                       grp_offset32(d.yc, (uint32_t)(c0 + c))))
                      : zero<CT>();
    }
    for (int k = threadIdx.x; k < 64; k += blockDim.x)
        S.xko[k] = k0 + k < d.K ? grp_offset32(d.xk, (uint32_t)(k0 + k)) : 0;
    for (int c = threadIdx.x; c < NC; c += blockDim.x)
        S.cco[c] = c0 + c < d.nc ? grp_offset32(d.cc, (uint32_t)(c0 + c)) : 0;
}

// X running along K (unit stride in K's innermost digit) with rows that are
// not contiguous: one row per thread would make every warp load touch 32
// lines, and the L1 then spends a cycle per line.  Instead each warp reads its
// 32 rows x 16 K with lanes along K (two rows per load instruction, two or
// three lines), rounds to FP32 into a warp-private tile in shared memory, and
// each thread then takes its own row from the tile (pitch 17: no bank
// conflicts).  FP32 compute only (the tile would not fit beside FP64 Y chunks).
struct RowsKc {
    float tile[8][32][17];
    int64_t xo[8][32];                  // the warp's row offsets (-1: past the last row)
};
template <typename CT> struct RowsKcSel { using type = char; };
template <> struct RowsKcSel<float> { using type = RowsKc; };

// One work item of a narrow GEMM: 256 rows (one per thread) by the column
// chunk cc (NC columns), all of K in chunks of 64 staged in shared memory.
// `staged` (block-uniform) names the column chunk already in shared memory
// when K fits one chunk (then Y is loaded once for many items), else -1.
template <typename CT, int NC, int KB = 8>
__device__ __forceinline__ void rows_item(const RowsGemmDesc &d, const double *__restrict__ X,
                                          const double *__restrict__ Y, double *__restrict__ C, int64_t rb, int cc,
                                          RowsSmem<CT, NC> &S, int64_t &staged, int64_t key, void *kcp) {
    const int nkc = (d.K + 63) / 64;
    const int64_t r = rb * 256 + threadIdx.x;
    const bool rok = r < d.R;
    const int64_t xo = rok ? grp_offset32(d.xr, (uint32_t)r) : 0, co = rok ? grp_offset32(d.cr, (uint32_t)r) : 0;
    const int c0 = cc * NC;
    CT acc[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) acc[c] = zero<CT>();
    for (int kc = 0; kc < nkc; kc++) {
        if (nkc > 1 || staged != key) {
            __syncthreads();                     // the block is done with the staged chunk
            rows_stage<CT, NC>(d, Y, kc * 64, c0, S);
            __syncthreads();
            staged = nkc == 1 ? key : -1;
        }
        const int kn = d.K - kc * 64 < 64 ? d.K - kc * 64 : 64;
        if constexpr (sizeof(CT) == 4) {
            if (d.kc) {
                RowsKc &Kc = *reinterpret_cast<RowsKc *>(kcp);
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                Kc.xo[warp][lane] = rok ? xo : -1;
                __syncwarp();
                for (int k16 = 0; k16 < kn; k16 += 16) {
                    const int kk = k16 + (lane & 15);
                    const bool kok = kk < kn;
                    const int64_t xk = kok ? S.xko[kk] : 0;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        double v[8];
#pragma unroll
                        for (int q = 0; q < 8; q++) {
                            const int64_t ro = Kc.xo[warp][2 * (8 * h + q) + (lane >> 4)];
                            v[q] = (kok && ro >= 0) ? __ldg(X + ro + xk) : 0.0;
                        }
#pragma unroll
                        for (int q = 0; q < 8; q++) Kc.tile[warp][2 * (8 * h + q) + (lane >> 4)][lane & 15] = down<CT>(v[q]);
                    }
                    __syncwarp();
                    // tile columns past K hold zeros and so do the staged Y rows
#pragma unroll
                    for (int k = 0; k < 16; k++) row_fma<NC>(Kc.tile[warp][lane][k], S.ys + (k16 + k) * NC, acc);
                    __syncwarp();               // the tile is refilled next
                }
                continue;
            }
        }
        if (rok) {
            // eight loads in flight per thread before their products (ys rows past K are zero)
            for (int k0 = 0; k0 < kn; k0 += KB) {
                // the KB loads first: a conversion may call out on its rare path
                double ad[KB];
                CT a[KB];
#pragma unroll
                for (int j = 0; j < KB; j++) ad[j] = k0 + j < kn ? __ldg(X + xo + S.xko[k0 + j]) : 0.0;
#pragma unroll
                for (int j = 0; j < KB; j++) a[j] = down<CT>(ad[j]);
#pragma unroll
                for (int j = 0; j < KB; j++) row_fma<NC>(a[j], S.ys + (k0 + j) * NC, acc);
            }
        }
    }
    if (!rok) return;
    const int ncc = d.nc - c0 < NC ? d.nc - c0 : NC;
    // beta 0: plain stores; beta 1: read-modify-write in batches of eight
    // (loads issued before the stores) or reductions; a general beta was applied before
    if (d.bcase == 0) {
#pragma unroll
        for (int c = 0; c < NC; c++)
            if (c < ncc) C[co + S.cco[c]] = epi_scale(acc[c], d.as);
    } else if (d.red) {
#pragma unroll
        for (int c = 0; c < NC; c++)
            if (c < ncc) red_add(C + co + S.cco[c], epi_scale(acc[c], d.as));
    } else {
#pragma unroll
        for (int cb = 0; cb < NC; cb += 8) {
            double old[8];
#pragma unroll
            for (int j = 0; j < 8; j++) old[j] = cb + j < ncc ? C[co + S.cco[cb + j]] : 0.0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (cb + j < ncc) C[co + S.cco[cb + j]] = epi_scale(acc[cb + j], d.as) + old[j];
        }
    }
}

// items: (column chunk, block of 256 rows), column chunk outermost so a block
// keeps one chunk of Y staged across its items
template <typename CT, int NC>
__global__ void __launch_bounds__(256, rows_min_blocks<CT, NC>()) rows_gemm_kernel(const RowsGemmDesc d, const double *__restrict__ X,
                                                        const double *__restrict__ Y, double *__restrict__ C) {
    __shared__ RowsSmem<CT, NC> S;
    __shared__ typename RowsKcSel<CT>::type KC;
    const int64_t rblocks = (d.R + 255) / 256;
    const int64_t items = rblocks * ((d.nc + NC - 1) / NC);
    int64_t staged = -1;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int cc = (int)(it / rblocks);
        rows_item<CT, NC>(d, X, Y, C, it - (int64_t)cc * rblocks, cc, S, staged, cc, &KC);
    }
}

// the grouped form: entry e's items follow item0; each block takes a
// contiguous range of items (grouped.cuh), so each entry's Y is staged once per
// (entry, column chunk) the block meets
template <typename CT, int NC>
__global__ void __launch_bounds__(256, rows_min_blocks<CT, NC>()) grouped_rows_kernel(const GroupedRows *__restrict__ tab,
                                                                                      int n, int64_t total,
                                                                                      const int *__restrict__ active) {
    __shared__ RowsSmem<CT, NC> S;
    __shared__ typename RowsKcSel<CT>::type KC;
    int64_t staged = -1;
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedRows> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const int lo = walk.at(it);
        const GroupedRows &e = tab[lo];
        if (!active[e.sys]) { it = walk.next - 1; continue; }   // block-uniform
        const int64_t rblocks = (e.d.R + 255) / 256, local = it - e.item0;
        const int cc = (int)(local / rblocks);
        // four loads per batch at the widest chunks: the grouped bookkeeping would
        // otherwise push the accumulators into local memory
        rows_item<CT, NC, (NC >= 40 ? 4 : 8)>(e.d, e.X, e.Y, e.C, local - (int64_t)cc * rblocks, cc, S, staged,
                                            (int64_t)lo * 4096 + cc, &KC);
    }
}

template <typename CT, int NC> constexpr int rows_grid_cap() { return 148 * rows_min_blocks<CT, NC>(); }

template <typename CT>
static cudaError_t rows_t(const RowsGemmDesc &d, const double *X, const double *Y, double *C, cudaStream_t s) {
    // accumulators: the column count rounded up to a multiple of 8 (chunks of 64 beyond)
    const int nc8 = d.nc > 64 ? 64 : (d.nc + 7) / 8 * 8;
    const int64_t items = (d.R + 255) / 256 * ((d.nc + nc8 - 1) / nc8);
    int64_t blocks = items < 148 * 3 ? items : 148 * 3;
    const unsigned b = (unsigned)blocks;
    switch (nc8 / 8) {
        case 1: rows_gemm_kernel<CT, 8><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 2: rows_gemm_kernel<CT, 16><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 3: rows_gemm_kernel<CT, 24><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 4: rows_gemm_kernel<CT, 32><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 5: rows_gemm_kernel<CT, 40><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 6: rows_gemm_kernel<CT, 48><<<b, 256, 0, s>>>(d, X, Y, C); break;
        default: rows_gemm_kernel<CT, 64><<<b, 256, 0, s>>>(d, X, Y, C); break;
    }
    return cudaGetLastError();
}

// the K-contiguous path's test: X's unit stride in K's innermost digit, not
// in the rows', FP32 compute
static int rows_kc(const RowsGemmDesc &d) {
    return d.f32 && d.xk.nd >= 1 && d.xk.str[d.xk.nd - 1] == 1 && !(d.xr.nd >= 1 && d.xr.str[d.xr.nd - 1] == 1);
}

cudaError_t launch_rows_gemm(const RowsGemmDesc &d0, const double *X, const double *Y, double *C, cudaStream_t s) {
    if (d0.R <= 0) return cudaSuccess;
    RowsGemmDesc d = d0;
    d.kc = rows_kc(d);
    d.bcase = beta_case(d.beta);
    d.as = make_scale(d.alpha);
    if (d.nc < 1 || d.K < 1 || d.R > 0xffffffffLL) return cudaErrorInvalidValue;
    if (d.bcase == 2) {
        if (cudaError_t e = launch_scale_grp(d.R, d.nc, d.cr, d.cc, d.beta, C, s)) return e;
        d.beta = 1.0;
        d.bcase = 1;
    }
    return d.f32 ? rows_t<float>(d, X, Y, C, s) : rows_t<double>(d, X, Y, C, s);
}

void prepare_grouped_rows(GroupedRows &g) {
    g.d.kc = rows_kc(g.d);
    g.d.bcase = beta_case(g.d.beta);
    g.d.as = make_scale(g.d.alpha);
    // one addition per output element and launch: a reduction in L2 gives the
    // same sum as a read-modify-write, without the loads' latency
    if (g.d.bcase == 1) g.d.red = 1;
}

int grouped_rows_nc(int nc_max) { return nc_max > 48 ? 64 : (nc_max + 7) / 8 * 8; }   // the kernels' widths

int64_t grouped_rows_items(const GroupedRows &g, int nc) {
    return (g.d.R + 255) / 256 * ((g.d.nc + nc - 1) / nc);
}

cudaError_t launch_grouped_rows(const GroupedRows *tab, int n, int64_t total, int nc, bool f32, const int *active,
                                cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 3 ? total : 148 * 3);
#define CCB_GROUPED_ROWS_NC(NCV)                                                                                     \
    do {                                                                                                             \
        if (f32) grouped_rows_kernel<float, NCV><<<blocks, 256, 0, s>>>(tab, n, total, active);                     \
        else grouped_rows_kernel<double, NCV><<<blocks, 256, 0, s>>>(tab, n, total, active);                        \
    } while (0)
    switch (nc / 8) {
        case 1: CCB_GROUPED_ROWS_NC(8); break;
        case 2: CCB_GROUPED_ROWS_NC(16); break;
        case 3: CCB_GROUPED_ROWS_NC(24); break;
        case 4: CCB_GROUPED_ROWS_NC(32); break;
        case 5: CCB_GROUPED_ROWS_NC(40); break;
        case 6: CCB_GROUPED_ROWS_NC(48); break;
        case 8: CCB_GROUPED_ROWS_NC(64); break;
        default: return cudaErrorInvalidValue;
    }
#undef CCB_GROUPED_ROWS_NC
    return cudaGetLastError();
}

// ------------------------------------------------------------ grouped GEMV
// Narrow GEMMs with one column (C(r) = alpha sum_k X(r, k) Y(k) + beta C(r))
// in a grouped launch.  The thread-per-row kernel above leaves such steps with
// a few hundred rows per system and K up to o v long, one dependent K loop per
// thread and, where X runs along K, 32 sectors per warp load.  Here a warp
// takes kGemvRQ consecutive rows and its lanes run along K, so the X loads
// coalesce; it is used where X's unit stride runs along K (grouped_gemv_ok).
// The block stages its entry's K offsets of X and the Y vector (in the
// compute type) in shared memory once per entry.
constexpr int kGemvRQ = 4;                   // rows per warp
constexpr int kGemvRows = 8 * kGemvRQ;       // rows per work item (block of 8 warps)

template <typename CT>
__global__ void __launch_bounds__(256) grouped_gemv_kernel(const GroupedRows *__restrict__ tab, int n, int64_t total,
                                                           const int *__restrict__ active) {
    __shared__ int xko[kGemvKmax];
    __shared__ CT ys[kGemvKmax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedRows> walk(tab, n, wr.begin);
    int staged = -1;
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const int ei = walk.at(it);
        const GroupedRows &e = tab[ei];
        if (!active[e.sys]) { it = walk.next - 1; continue; }   // block-uniform
        const RowsGemmDesc &d = e.d;
        const int K = d.K;
        if (ei != staged) {
            __syncthreads();                     // the previous entry's reads are done
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                xko[k] = (int)grp_offset(d.xk, k);
                ys[k] = down<CT>(__ldg(e.Y + grp_offset(d.yk, k)));   // column 0: yc(0) = 0
            }
            __syncthreads();
            staged = ei;
        }
        const int64_t r0 = (it - e.item0) * kGemvRows + warp * kGemvRQ;
        bool rok[kGemvRQ];
        int64_t xo[kGemvRQ];
#pragma unroll
        for (int q = 0; q < kGemvRQ; q++) {
            rok[q] = r0 + q < d.R;
            xo[q] = rok[q] ? grp_offset32(d.xr, (uint32_t)(r0 + q)) : 0;
        }
        CT acc[kGemvRQ];
#pragma unroll
        for (int q = 0; q < kGemvRQ; q++) acc[q] = zero<CT>();
        for (int kb = 0; kb < K; kb += 128) {
            // every load of the batch before its products
            double xv[4][kGemvRQ];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int k = kb + lane + 32 * u;
                const int ko = k < K ? xko[k] : 0;
#pragma unroll
                for (int q = 0; q < kGemvRQ; q++) xv[u][q] = (k < K && rok[q]) ? __ldg(e.X + xo[q] + ko) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int k = kb + lane + 32 * u;
                const CT y = k < K ? ys[k] : zero<CT>();
#pragma unroll
                for (int q = 0; q < kGemvRQ; q++) acc[q] = fma(down<CT>(xv[u][q]), y, acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kGemvRQ; q++)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        if (lane < kGemvRQ) {
            CT a = acc[0];
#pragma unroll
            for (int q = 1; q < kGemvRQ; q++)
                if (lane == q) a = acc[q];
            if (rok[lane]) {
                double *c = e.C + grp_offset32(d.cr, (uint32_t)(r0 + lane));
                if (d.bcase == 0) *c = epi_scale(a, d.as);
                else if (d.red) red_add(c, epi_scale(a, d.as));
                else *c = epi_scale(a, d.as) + *c;
            }
        }
    }
}

// One-column narrow GEMMs whose large operand X runs along the rows (unit
// stride in the rows' innermost digit) and whose K is long (the V_ovvv t1
// contraction into F_ae, K = o v): a work item is 32 consecutive rows, lanes
// along the rows (coalesced), and the block's eight warps each take one eighth
// of K, so a row's K loop is spread over eight warps instead of one thread.
// The eight partial sums of a row are added in warp order in shared memory.
template <typename CT>
__global__ void __launch_bounds__(256) grouped_gemvr_kernel(const GroupedRows *__restrict__ tab, int n, int64_t total,
                                                            const int *__restrict__ active) {
    __shared__ int xko[kGemvKmax];
    __shared__ CT ys[kGemvKmax];
    __shared__ CT part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedRows> walk(tab, n, wr.begin);
    int staged = -1;
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const int ei = walk.at(it);
        const GroupedRows &e = tab[ei];
        if (!active[e.sys]) { it = walk.next - 1; continue; }   // block-uniform
        const RowsGemmDesc &d = e.d;
        const int K = d.K;
        if (ei != staged) {
            __syncthreads();                     // the previous entry's reads are done
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                xko[k] = (int)grp_offset(d.xk, k);
                ys[k] = down<CT>(__ldg(e.Y + grp_offset(d.yk, k)));
            }
            __syncthreads();
            staged = ei;
        }
        const int64_t r = (it - e.item0) * 32 + lane;
        const bool rok = r < d.R;
        const int64_t xo = rok ? grp_offset32(d.xr, (uint32_t)r) : 0;
        const int kper = (K + 7) / 8, kb = warp * kper, ke = min(K, kb + kper);
        CT acc = zero<CT>();
        for (int k0 = kb; k0 < ke; k0 += 8) {
            double xv[8];
#pragma unroll
            for (int j = 0; j < 8; j++) xv[j] = (rok && k0 + j < ke) ? __ldg(e.X + xo + xko[k0 + j]) : 0.0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (k0 + j < ke) acc = fma(down<CT>(xv[j]), ys[k0 + j], acc);
        }
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && rok) {
            CT a = part[0][lane];
#pragma unroll
            for (int w = 1; w < 8; w++) a += part[w][lane];
            double *c = e.C + grp_offset32(d.cr, (uint32_t)r);
            if (d.bcase == 0) *c = epi_scale(a, d.as);
            else if (d.red) red_add(c, epi_scale(a, d.as));
            else *c = epi_scale(a, d.as) + *c;
        }
        __syncthreads();                         // part is reused by the next item
    }
}

bool grouped_gemvr_ok(const GroupedRows &g) {
    const RowsGemmDesc &d = g.d;
    if (d.nc != 1 || d.K < 64 || d.K > kGemvKmax || d.R > 0xffffffffLL || d.bcase == 2) return false;
    if (d.xr.nd < 1 || d.xr.str[d.xr.nd - 1] != 1) return false;
    int64_t xmax = 0;
    for (int k = 0; k < d.xk.nd; k++) xmax += (d.xk.ext[k] - 1) * d.xk.str[k];
    return xmax >= 0 && xmax < ((int64_t)1 << 31);
}

int64_t grouped_gemvr_items(const GroupedRows &g) { return (g.d.R + 31) / 32; }

cudaError_t launch_grouped_gemvr(const GroupedRows *tab, int n, int64_t total, bool f32, const int *active,
                                 cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 6 ? total : 148 * 6);
    if (f32) grouped_gemvr_kernel<float><<<blocks, 256, 0, s>>>(tab, n, total, active);
    else grouped_gemvr_kernel<double><<<blocks, 256, 0, s>>>(tab, n, total, active);
    return cudaGetLastError();
}

bool grouped_gemv_ok(const GroupedRows &g) {
    const RowsGemmDesc &d = g.d;
    // lanes along K pay off where X's unit stride runs along K (the innermost K digit)
    if (d.nc != 1 || d.K < 1 || d.K > kGemvKmax || d.R > 0xffffffffLL || d.bcase == 2) return false;
    if (d.xk.nd < 1 || d.xk.str[d.xk.nd - 1] != 1) return false;
    int64_t xmax = 0;
    for (int k = 0; k < d.xk.nd; k++) xmax += (d.xk.ext[k] - 1) * d.xk.str[k];
    return xmax >= 0 && xmax < ((int64_t)1 << 31);
}

int64_t grouped_gemv_items(const GroupedRows &g) { return (g.d.R + kGemvRows - 1) / kGemvRows; }

cudaError_t launch_grouped_gemv(const GroupedRows *tab, int n, int64_t total, bool f32, const int *active,
                                cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 6 ? total : 148 * 6);
    if (f32) grouped_gemv_kernel<float><<<blocks, 256, 0, s>>>(tab, n, total, active);
    else grouped_gemv_kernel<double><<<blocks, 256, 0, s>>>(tab, n, total, active);
    return cudaGetLastError();
}

// ------------------------------------------------------------ rows_multi
// The narrow kernel over several members into one output: every member's Y
// block (alpha_s folded in, K rounded up to 8 with zero rows) is staged in
// shared memory, one thread per row runs through all members' K, and the row's
// outputs are read and written once at the end.
static inline int64_t rows_multi_krows(const RowsMultiDesc &d) {
    int64_t k = 0;
    for (int s = 0; s < d.nm; s++) k += (d.m[s].K + 7) / 8 * 8;
    return k;
}

template <int NC> static int64_t rows_multi_bytes(const RowsMultiDesc &d, int esz) {
    const int64_t kr = rows_multi_krows(d);
    return kr * NC * esz + kr * 8 + NC * 8;
}

// blocks per SM: the staged Y blocks (up to 96 KB) allow two
template <typename CT, int NC> constexpr int rows_multi_min_blocks() { return sizeof(CT) == 4 || NC <= 24 ? 2 : 1; }

template <typename CT, int NC>
__global__ void __launch_bounds__(256, rows_multi_min_blocks<CT, NC>()) rows_multi_kernel(const RowsMultiDesc d, double *__restrict__ C) {
    extern __shared__ __align__(16) unsigned char rm_smem[];
    int kr = 0;
    for (int s = 0; s < d.nm; s++) kr += (d.m[s].K + 7) / 8 * 8;
    CT *ys = reinterpret_cast<CT *>(rm_smem);
    int64_t *xko = reinterpret_cast<int64_t *>(rm_smem + (size_t)kr * NC * sizeof(CT));
    int64_t *cco = xko + kr;
    int kb = 0;
    for (int s = 0; s < d.nm; s++) {
        const RowsMember &m = d.m[s];
        const int k8 = (m.K + 7) / 8 * 8;
        for (int e = threadIdx.x; e < k8 * NC; e += blockDim.x) {
            const int k = e / NC, c = e - k * NC;
            ys[(kb + k) * NC + c] = (k < m.K && c < d.nc)
                                        ? down<CT>(m.alpha * __ldg(m.Y + grp_offset(m.yk, k) + grp_offset(m.yc, c)))
                                        : zero<CT>();
        }
        for (int k = threadIdx.x; k < k8; k += blockDim.x) xko[kb + k] = k < m.K ? grp_offset(m.xk, k) : 0;
        kb += k8;
    }
    for (int c = threadIdx.x; c < NC; c += blockDim.x) cco[c] = c < d.nc ? grp_offset(d.cc, c) : 0;
    __syncthreads();
    const Scale one = {0, 0, 0u, 1.0};
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < d.R; r += (int64_t)gridDim.x * blockDim.x) {
        CT acc[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) acc[c] = zero<CT>();
        kb = 0;
        for (int s = 0; s < d.nm; s++) {
            const RowsMember &m = d.m[s];
            const double *X = m.X;
            const int64_t xo = grp_offset32(m.xr, (uint32_t)r);
            // eight loads in flight before their products (the padded Y rows are zero)
            for (int k0 = 0; k0 < m.K; k0 += 8) {
                double ad[8];
                CT a[8];
#pragma unroll
                for (int j = 0; j < 8; j++) ad[j] = k0 + j < m.K ? __ldg(X + xo + xko[kb + k0 + j]) : 0.0;
#pragma unroll
                for (int j = 0; j < 8; j++) a[j] = down<CT>(ad[j]);
#pragma unroll
                for (int j = 0; j < 8; j++) row_fma<NC>(a[j], ys + (kb + k0 + j) * NC, acc);
            }
            kb += (m.K + 7) / 8 * 8;
        }
        const int64_t co = grp_offset32(d.cr, (uint32_t)r);
        if (d.red) {
#pragma unroll
            for (int c = 0; c < NC; c++)
                if (c < d.nc) red_add(C + co + cco[c], epi_scale(acc[c], one));
        } else {
#pragma unroll
            for (int c0 = 0; c0 < NC; c0 += 8) {
                double old[8];
#pragma unroll
                for (int j = 0; j < 8; j++) old[j] = c0 + j < d.nc ? C[co + cco[c0 + j]] : 0.0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (c0 + j < d.nc) C[co + cco[c0 + j]] = epi_scale(acc[c0 + j], one) + old[j];
            }
        }
    }
}

template <typename CT, int NC> static cudaError_t rows_multi_t(const RowsMultiDesc &d, double *C, cudaStream_t s) {
    const int64_t smem = rows_multi_bytes<NC>(d, (int)sizeof(CT));
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        if (cudaError_t e = cudaFuncSetAttribute(rows_multi_kernel<CT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem))
            return e;
    }
    int64_t blocks = (d.R + 255) / 256;
    if (blocks > 148 * rows_multi_min_blocks<CT, NC>()) blocks = 148 * rows_multi_min_blocks<CT, NC>();
    rows_multi_kernel<CT, NC><<<(unsigned)blocks, 256, (size_t)smem, s>>>(d, C);
    return cudaGetLastError();
}

template <typename CT> static cudaError_t rows_multi_ct(const RowsMultiDesc &d, double *C, cudaStream_t s) {
    switch ((d.nc + 7) / 8) {
        case 1: return rows_multi_t<CT, 8>(d, C, s);
        case 2: return rows_multi_t<CT, 16>(d, C, s);
        case 3: return rows_multi_t<CT, 24>(d, C, s);
        case 4: return rows_multi_t<CT, 32>(d, C, s);
        case 5: return rows_multi_t<CT, 40>(d, C, s);
        case 6: return rows_multi_t<CT, 48>(d, C, s);
        default: return rows_multi_t<CT, 64>(d, C, s);
    }
}

int64_t rows_multi_smem_bytes(const RowsMultiDesc &d) {
    if (d.nc < 1 || d.nc > 64) return 0;
    const int nc8 = (d.nc + 7) / 8 * 8;
    const int64_t kr = rows_multi_krows(d);
    const int64_t b = kr * nc8 * (d.f32 ? 4 : 8) + kr * 8 + nc8 * 8;
    return b > 200 * 1024 ? 0 : b;
}

cudaError_t launch_rows_multi(const RowsMultiDesc &d, double *C, cudaStream_t s) {
    if (d.R <= 0) return cudaSuccess;
    if (d.nm < 1 || d.nm > kMaxRowsMembers || d.nc < 1 || d.nc > 64 || d.R > 0xffffffffLL ||
        rows_multi_smem_bytes(d) == 0)
        return cudaErrorInvalidValue;
    for (int k = 0; k < d.nm; k++)
        if (d.m[k].K < 1 || !d.m[k].X || !d.m[k].Y) return cudaErrorInvalidValue;
    return d.f32 ? rows_multi_ct<float>(d, C, s) : rows_multi_ct<double>(d, C, s);
}

// ------------------------------------------------------------ narrow_k
// Long contraction, at most 8 columns, the large operand read in place: a warp
// takes four rows and a segment of the contraction (seg elements of one inner
// run, or kper whole runs); its lanes read the contiguous run of the four rows
// (coalesced) and the matching Y values once for all four.  Each lane issues
// the loads of two steps before converting any of them (a conversion may call
// out on its rare path, and loads are not moved across calls).  Lane sums
// meet in a shuffle tree and are added to C by reductions in L2 (C cleared or
// scaled beforehand for beta != 1).
template <typename CT, int NN>
__global__ void __launch_bounds__(256) narrow_k_kernel(const NarrowKDesc d, const double *__restrict__ X,
                                                       const double *__restrict__ Y, double *__restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int64_t groups = (d.M + 3) / 4, chunks = (d.Ko + d.kper - 1) / d.kper, nseg = (d.L + d.seg - 1) / d.seg;
    const int64_t per_group = chunks * nseg, items = groups * per_group;
    int yn[NN];     // the columns' offsets in Y (Y below 2^31 elements: checked by the planner)
#pragma unroll
    for (int n = 0; n < NN; n++) yn[n] = n < d.N ? (int)grp_offset(d.yn, n) : 0;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += nwarps) {
        const int64_t g = it / per_group, rem = it - g * per_group;
        const int64_t kc = rem / nseg, sg = rem - kc * nseg;
        int64_t xr[4];
        bool ok[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t m = 4 * g + r;
            ok[r] = m < d.M;
            xr[r] = ok[r] ? grp_offset(d.xm, m) : 0;
        }
        CT acc[4][NN];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int n = 0; n < NN; n++) acc[r][n] = zero<CT>();
        const int64_t ko1 = (kc + 1) * d.kper < d.Ko ? (kc + 1) * d.kper : d.Ko;
        const int64_t j0 = sg * d.seg, j1 = j0 + d.seg < d.L ? j0 + d.seg : d.L;
        for (int64_t ko = kc * d.kper; ko < ko1; ko++) {
            const int64_t xo = grp_offset(d.xko, ko), yo = grp_offset(d.yko, ko);
            for (int64_t j = j0 + lane; j < j1; j += 64) {
                const bool two = j + 32 < j1;
                double xd[2][4], yd[2][NN];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int64_t jj = j + 32 * u;
                    const bool on = u == 0 || two;
#pragma unroll
                    for (int n = 0; n < NN; n++) yd[u][n] = on && n < d.N ? __ldg(Y + yo + jj * d.sy + yn[n]) : 0.0;
#pragma unroll
                    for (int r = 0; r < 4; r++) xd[u][r] = on && ok[r] ? __ldg(X + xr[r] + xo + jj) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    CT y[NN], x[4];
#pragma unroll
                    for (int n = 0; n < NN; n++) y[n] = down<CT>(yd[u][n]);
#pragma unroll
                    for (int r = 0; r < 4; r++) x[r] = down<CT>(xd[u][r]);
#pragma unroll
                    for (int r = 0; r < 4; r++)
#pragma unroll
                        for (int n = 0; n < NN; n++) acc[r][n] = cfma(x[r], y[n], acc[r][n]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int n = 0; n < NN; n++) {
                double v = up(acc[r][n]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && ok[r] && n < d.N)
                    red_add(C + grp_offset(d.cm, 4 * g + r) + grp_offset(d.cn, n), d.alpha * v);
            }
    }
}

template <typename CT>
static cudaError_t narrow_k_t(const NarrowKDesc &d, const double *X, const double *Y, double *C, cudaStream_t s) {
    const int64_t items = ((d.M + 3) / 4) * ((d.Ko + d.kper - 1) / d.kper) * ((d.L + d.seg - 1) / d.seg);
    int64_t blocks = (items + 7) / 8;
    if (blocks > 148 * 8) blocks = 148 * 8;
    const unsigned b = (unsigned)blocks;
    switch (d.N) {
        case 1: narrow_k_kernel<CT, 1><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 2: narrow_k_kernel<CT, 2><<<b, 256, 0, s>>>(d, X, Y, C); break;
        case 3: case 4: narrow_k_kernel<CT, 4><<<b, 256, 0, s>>>(d, X, Y, C); break;
        default: narrow_k_kernel<CT, 8><<<b, 256, 0, s>>>(d, X, Y, C); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_narrow_k(const NarrowKDesc &d, const double *X, const double *Y, double *C, cudaStream_t s) {
    if (d.M <= 0) return cudaSuccess;
    if (d.N < 1 || d.N > 8 || d.Ko < 1 || d.L < 1 || d.kper < 1 || d.seg < 1) return cudaErrorInvalidValue;
    if (d.beta != 1.0)
        if (cudaError_t e = launch_scale_grp(d.M, d.N, d.cm, d.cn, d.beta, C, s)) return e;
    return d.f32 ? narrow_k_t<float>(d, X, Y, C, s) : narrow_k_t<double>(d, X, Y, C, s);
}

// ------------------------------------------------------------------ gemv
// y(r) = alpha * sum_k X(r,k) x(k) + beta * y(r): the GEMM shapes with one
// output dimension of extent 1 are memory-bound matrix-vector products.
// X(r,k) = X[r*sr + k*sk]; x(k) = x[k*incx]; y addressed through a group;
// cX / cx conjugate X / x.  K-contiguous X (sk == 1): one warp per row;
// otherwise one thread per row.
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shfl_xor(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
template <typename T>
__global__ void __launch_bounds__(256) gemv_rowwarp_kernel(int64_t R, int64_t K, const T *__restrict__ X, int64_t sr,
                                                           const T *__restrict__ x, int64_t incx, const Grp gy,
                                                           double alpha, double beta, T *__restrict__ y, int cX,
                                                           int cx) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    for (int64_t r = w0; r < R; r += (int64_t)gridDim.x * 8) {
        const T *row = X + r * sr;
        T s0 = zero<T>(), s1 = zero<T>();
        int64_t k = lane;
        for (; k + 32 < K; k += 64) {
            s0 = cfma(cj(ld(row + k), cX), cj(ld(x + k * incx), cx), s0);
            s1 = cfma(cj(ld(row + k + 32), cX), cj(ld(x + (k + 32) * incx), cx), s1);
        }
        if (k < K) s0 = cfma(cj(ld(row + k), cX), cj(ld(x + k * incx), cx), s0);
        T s = add(s0, s1);
        for (int o = 16; o > 0; o >>= 1) s = add(s, shfl_xor(s, o));
        if (lane == 0) {
            T *p = y + grp_offset(gy, r);
            T val = scal(alpha, s);
            if (beta != 0.0) val = axpy(beta, *p, val);
            *p = val;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gemv_rowthread_kernel(int64_t R, int64_t K, const T *__restrict__ X,
                                                             int64_t sk, const T *__restrict__ x, int64_t incx,
                                                             const Grp gy, double alpha, double beta,
                                                             T *__restrict__ y, int cX, int cx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        T s0 = zero<T>(), s1 = zero<T>(), s2 = zero<T>(), s3 = zero<T>();
        int64_t k = 0;
        for (; k + 3 < K; k += 4) {
            s0 = cfma(cj(ld(X + r + k * sk), cX), cj(ld(x + k * incx), cx), s0);
            s1 = cfma(cj(ld(X + r + (k + 1) * sk), cX), cj(ld(x + (k + 1) * incx), cx), s1);
            s2 = cfma(cj(ld(X + r + (k + 2) * sk), cX), cj(ld(x + (k + 2) * incx), cx), s2);
            s3 = cfma(cj(ld(X + r + (k + 3) * sk), cX), cj(ld(x + (k + 3) * incx), cx), s3);
        }
        for (; k < K; k++) s0 = cfma(cj(ld(X + r + k * sk), cX), cj(ld(x + k * incx), cx), s0);
        T *p = y + grp_offset(gy, r);
        T val = scal(alpha, add(add(s0, s1), add(s2, s3)));
        if (beta != 0.0) val = axpy(beta, *p, val);
        *p = val;
    }
}

template <typename T>
static cudaError_t launch_gemv(int64_t R, int64_t K, const T *X, int64_t sr, int64_t sk, const T *x, int64_t incx,
                               const Grp &gy, double alpha, double beta, T *y, int cX, int cx, cudaStream_t s) {
    if (sk == 1 || K == 1) {
        int64_t blocks = (R + 7) / 8;
        if (blocks > 148 * 16) blocks = 148 * 16;
        gemv_rowwarp_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(R, K, X, sr, x, incx, gy, alpha, beta, y, cX, cx);
    } else {
        int64_t blocks = (R + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        gemv_rowthread_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(R, K, X, sk, x, incx, gy, alpha, beta, y, cX, cx);
    }
    return cudaGetLastError();
}

// C(m,n) = alpha * a(m) b(n) + beta * C(m,n): the K = 1 (outer product) shape,
// memory-bound; threads run along the output direction with the smaller stride.
template <typename T>
__global__ void __launch_bounds__(256) outer_kernel(int64_t M, int64_t N, const T *__restrict__ a, int64_t sa,
                                                    const T *__restrict__ b, int64_t sb, const Grp cm, const Grp cn,
                                                    double alpha, double beta, T *__restrict__ C, int m_fast, int ca,
                                                    int cb) {
    const int64_t MN = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t m, n;
        if (m_fast) { n = e / M; m = e - n * M; } else { m = e / N; n = e - m * N; }
        T *p = C + grp_offset(cm, m) + grp_offset(cn, n);
        T val = scal(alpha, mul(cj(ld(a + m * sa), ca), cj(ld(b + n * sb), cb)));
        if (beta != 0.0) val = axpy(beta, *p, val);
        *p = val;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) splitk_reduce_kernel(int64_t M, int64_t N, int nz, const T *__restrict__ P,
                                                            const Grp cm, const Grp cn, double alpha, double beta,
                                                            T *__restrict__ C) {
    const int64_t MN = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
        T acc = zero<T>();
        for (int z = 0; z < nz; z++) acc = add(acc, P[z * MN + e]);
        const int64_t n = e / M, m = e - n * M;
        T *p = C + grp_offset(cm, m) + grp_offset(cn, n);
        T val = scal(alpha, acc);
        if (beta != 0.0) val = axpy(beta, *p, val);
        *p = val;
    }
}

template <typename T>
static cudaError_t splitk_reduce_t(int64_t M, int64_t N, int splitk, const T *partials, const Grp &cm, const Grp &cn,
                                   double alpha, double beta, T *C, cudaStream_t s) {
    int64_t blocks = (M * N + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    splitk_reduce_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(M, N, splitk, partials, cm, cn, alpha, beta, C);
    return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(int64_t M, int64_t N, int splitk, const double *partials, const Grp &cm, const Grp &cn,
                                 double alpha, double beta, double *C, cudaStream_t s) {
    return splitk_reduce_t<double>(M, N, splitk, partials, cm, cn, alpha, beta, C, s);
}

template <typename T, typename CT>
static cudaError_t gemm_t(GemmF64Desc d, const T *A, const T *B, T *C, T *partials, cudaStream_t s) {
    if (d.K == 1 && d.M > 1 && d.N > 1) {
        int64_t sm = d.cm.nd ? d.cm.str[d.cm.nd - 1] : 0, sn = d.cn.nd ? d.cn.str[d.cn.nd - 1] : 0;
        int64_t blocks = (d.M * d.N + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        outer_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d.M, d.N, A, d.sAm, B, d.sBn, d.cm, d.cn, d.alpha, d.beta, C,
                                                         sm <= sn ? 1 : 0, d.conj_a, d.conj_b);
        return cudaGetLastError();
    }
    // matrix-vector shapes: rows m of A against the single column of B, or
    // rows n of B^T against the single row of A
    if (d.N == 1 && d.M > 1 && (d.sAk == 1 || d.sAm == 1))
        return launch_gemv<T>(d.M, d.K, A, d.sAm, d.sAk, B, d.sBk, d.cm, d.alpha, d.beta, C, d.conj_a, d.conj_b, s);
    if (d.M == 1 && d.N > 1 && (d.sBk == 1 || d.sBn == 1))
        return launch_gemv<T>(d.N, d.K, B, d.sBn, d.sBk, A, d.sAk, d.cn, d.alpha, d.beta, C, d.conj_b, d.conj_a, s);
    const int sk = d.splitk > 1 ? d.splitk : 1;
    const int64_t kchunk = sk > 1 ? ((d.K + sk - 1) / sk + GBK - 1) / GBK * GBK : (d.K > 0 ? d.K : 1);
    const int zs = (int)((d.K + kchunk - 1) / kchunk);
    dim3 grid((unsigned)((d.M + GBM - 1) / GBM), (unsigned)((d.N + GBN - 1) / GBN), (unsigned)zs);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    if (zs > 1 && !partials) return cudaErrorInvalidValue;
    // threads run fastest along the output direction with the smaller stride
    int64_t sm = d.cm.nd ? d.cm.str[d.cm.nd - 1] : 0, sn = d.cn.nd ? d.cn.str[d.cn.nd - 1] : 0;
    int m_fast = (d.cm.nd && (!d.cn.nd || sm <= sn)) ? 1 : 0;
    const bool ak = d.sAk == 1 && !(d.sAm == 1 && d.K == 1);
    const bool bk = d.sBk == 1 && !(d.sBn == 1 && d.K == 1);
    if (zs > 1) m_fast = 1;
    if (zs == 1 && d.bcase == 2) {
        // general beta: C *= beta first, then the kernel accumulates
        if (cudaError_t e = scale_grp_t<T>(d.M, d.N, d.cm, d.cn, d.beta, C, s)) return e;
        d.beta = 1.0;
        d.bcase = 1;
    }
    if (ak && bk) gemm_f64_kernel<T, CT, true, true><<<grid, 256, 0, s>>>(d, A, B, C, partials, m_fast, kchunk);
    else if (ak) gemm_f64_kernel<T, CT, true, false><<<grid, 256, 0, s>>>(d, A, B, C, partials, m_fast, kchunk);
    else if (bk) gemm_f64_kernel<T, CT, false, true><<<grid, 256, 0, s>>>(d, A, B, C, partials, m_fast, kchunk);
    else gemm_f64_kernel<T, CT, false, false><<<grid, 256, 0, s>>>(d, A, B, C, partials, m_fast, kchunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || zs == 1) return e;
    return splitk_reduce_t<T>(d.M, d.N, zs, partials, d.cm, d.cn, d.alpha, d.beta, C, s);
}

cudaError_t launch_gemm_f64(const GemmF64Desc &d0, const double *A, const double *B, double *C, double *partials,
                            cudaStream_t s) {
    if (d0.M <= 0 || d0.N <= 0) return cudaSuccess;
    GemmF64Desc d = d0;
    d.bcase = beta_case(d.beta);
    d.as = make_scale(d.alpha);
    if (d.cplx)
        return gemm_t<double2, double2>(d, reinterpret_cast<const double2 *>(A), reinterpret_cast<const double2 *>(B),
                                        reinterpret_cast<double2 *>(C), reinterpret_cast<double2 *>(partials), s);
    if (d.f32) return gemm_t<double, float>(d, A, B, C, partials, s);
    return gemm_t<double, double>(d, A, B, C, partials, s);
}

// ------------------------------------------------------- iteration kernels
// Residual arrays are [occupied tuple][virtual tuple] row-major with
// nvt = v^rank virtual tuples per occupied tuple.  One block row per occupied
// tuple: its orbital-energy sum is formed once; the virtual tuple's is formed
// from 32-bit digits.  D = sum f_occ - sum f_vir.
__device__ __forceinline__ double occ_sum(int rank, int o, const double *fo, int64_t row) {
    double s = 0.0;
    for (int k = 0; k < rank; k++) { s += fo[row % o]; row /= o; }
    return s;
}
__device__ __forceinline__ double vir_sum(int rank, int v, const double *fv, uint32_t col) {
    double s = 0.0;
    for (int k = 0; k < rank; k++) { s += fv[col % (uint32_t)v]; col /= (uint32_t)v; }
    return s;
}

// cplx: the arrays are interleaved complex; column c of a row is component
// c & 1 of virtual tuple c >> 1 (D is real).
// sum of the rank virtual energies of a tuple with rank - 1 adds (the FP64
// pipe issues ~2 operations per clock per SM: the per-element update below
// is rank + 1 of them)
__device__ __forceinline__ double vir_sum_lean(int rank, int v, const double *fv, uint32_t col) {
    double s = fv[col % (uint32_t)v];
    for (int k = 1; k < rank; k++) {
        col /= (uint32_t)v;
        s += fv[col % (uint32_t)v];
    }
    return s;
}

__global__ void __launch_bounds__(256) denom_sub_kernel(int rank, int o, int v, const double *fo, const double *fv,
                                                        const double *__restrict__ t, double *__restrict__ r,
                                                        int64_t rows, uint32_t nvt, int cplx) {
    const uint32_t ncol = nvt << cplx;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const double so = occ_sum(rank, o, fo, row);
        const int64_t base = row * ncol;
        for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) {
            const double d = so - vir_sum_lean(rank, v, fv, c >> cplx);
            r[base + c] = fma(neg(d), t[base + c], r[base + c]);
        }
    }
}

// The same update with a table in shared memory, two FP64 operations per
// element instead of rank + 1.  Rank 2: the pair sums f_vir[a] + f_vir[b] of
// all v^2 columns (formed once per block; the sum commutes, so D stays exactly
// symmetric in a, b and the update keeps T2's antisymmetry bit for bit), d =
// sum f_occ - pair[c].  Rank >= 3: per row, tab[q] = sum f_occ - sum f_vir over
// the outer virtual digits q (all but the last), d = tab[q] - f_vir[c].
constexpr int kDenomTab = 6144;              // doubles of the table (48 KB)
__global__ void __launch_bounds__(256) denom_sub_tab_kernel(int rank, int o, int v, const double *fo,
                                                            const double *fv, const double *__restrict__ t,
                                                            double *__restrict__ r, int64_t rows, uint32_t nvt,
                                                            int cplx) {
    extern __shared__ double tab[];
    const uint32_t vv = (uint32_t)v, nout = nvt / vv, ncol = nvt << cplx;
    const bool pairs = rank == 2;
    if (pairs) {
        for (uint32_t c = threadIdx.x; c < nvt; c += blockDim.x) tab[c] = vir_sum_lean(2, v, fv, c);
        __syncthreads();
    }
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const double so = occ_sum(rank, o, fo, row);
        const int64_t base = row * ncol;
        if (pairs) {
            for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) {
                const double d = so - tab[c >> cplx];
                r[base + c] = fma(neg(d), t[base + c], r[base + c]);
            }
            continue;
        }
        __syncthreads();                         // the previous row's reads of tab are done
        for (uint32_t q = threadIdx.x; q < nout; q += blockDim.x) tab[q] = so - vir_sum_lean(rank - 1, v, fv, q);
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) {
            const uint32_t x = c >> cplx, q = x / vv, b = x - q * vv;
            const double d = tab[q] - fv[b];
            r[base + c] = fma(neg(d), t[base + c], r[base + c]);
        }
    }
}

static void rows_cols(int rank, int o, int v, int64_t &rows, uint32_t &nvt) {
    rows = 1;
    int64_t c = 1;
    for (int k = 0; k < rank; k++) { rows *= o; c *= v; }
    nvt = (uint32_t)c;
}

cudaError_t launch_denom_sub(int rank, int o, int v, const double *fo, const double *fv, const double *t, double *r,
                             int cplx, cudaStream_t s) {
    int64_t rows;
    uint32_t nvt;
    rows_cols(rank, o, v, rows, nvt);
    int64_t blocks = rows < 148 * 16 ? rows : 148 * 16;
    const uint32_t ntab = rank == 2 ? nvt : nvt / (uint32_t)v;
    if (rank >= 2 && ntab <= (uint32_t)kDenomTab) {
        const size_t shm = (size_t)ntab * sizeof(double);
        denom_sub_tab_kernel<<<(unsigned)blocks, 256, shm, s>>>(rank, o, v, fo, fv, t, r, rows, nvt, cplx ? 1 : 0);
        return cudaGetLastError();
    }
    denom_sub_kernel<<<(unsigned)blocks, 256, 0, s>>>(rank, o, v, fo, fv, t, r, rows, nvt, cplx ? 1 : 0);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) inv_denominators_kernel(int rank, int o, int v, const double *fo,
                                                                const double *fv, double *out, int64_t rows,
                                                                uint32_t nvt, int cplx) {
    const uint32_t ncol = nvt << cplx;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const double so = occ_sum(rank, o, fo, row);
        for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x)
            out[row * ncol + c] = 1.0 / (so - vir_sum(rank, v, fv, c >> cplx));
    }
}

cudaError_t launch_inv_denominators(int rank, int o, int v, const double *fo, const double *fv, double *out, int cplx,
                                    cudaStream_t s) {
    int64_t rows;
    uint32_t nvt;
    rows_cols(rank, o, v, rows, nvt);
    int64_t blocks = rows < 148 * 16 ? rows : 148 * 16;
    inv_denominators_kernel<<<(unsigned)blocks, 256, 0, s>>>(rank, o, v, fo, fv, out, rows, nvt, cplx ? 1 : 0);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) jacobi_inv_kernel(int64_t n, const double *__restrict__ t,
                                                         const double *__restrict__ r, const double *__restrict__ dinv,
                                                         double *__restrict__ xo, double *__restrict__ eo) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double q = r[e] * dinv[e];
        eo[e] = q;
        xo[e] = t[e] + q;
    }
}

cudaError_t launch_jacobi_inv(int64_t n, const double *t, const double *r, const double *dinv, double *xo, double *eo,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    jacobi_inv_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, t, r, dinv, xo, eo);
    return cudaGetLastError();
}

__global__ void axpby_kernel(int64_t n, double a, const double *__restrict__ x, double b, double *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = a * x[e] + b * y[e];
}

cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    axpby_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, a, x, b, y);
    return cudaGetLastError();
}

// deterministic block reduction (fixed grid, fixed order)
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double sh[256];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) dot_partials_kernel(const double *x, const double *y, int64_t n,
                                                           double *partials) {
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)kRedBlocks * 256)
        s = fma(x[e], y[e], s);
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One pass over e: each thread walks its fixed strided slice of the vector,
// issuing every overlap's load for an element before its FMAs; one block sum
// per overlap.  The history vectors are read once and the new error vector is
// never re-read, so m overlaps cost (m + 3.5) vector passes instead of 2m + 5.
template <int M>
__global__ void __launch_bounds__(256) jacobi_dots_kernel(const JacobiSegs g, const double *__restrict__ dinv,
                                                          double *__restrict__ xo, double *__restrict__ eo,
                                                          double *__restrict__ partials) {
    double acc[M];
#pragma unroll
    for (int h = 0; h < M; h++) acc[h] = 0.0;
    const int64_t stride = (int64_t)kRedBlocks * 256;
    int64_t base = 0;
    for (int l = 0; l < g.nseg; l++) {
        const double *__restrict__ t = g.t[l];
        const double *__restrict__ r = g.r[l];
        const int64_t n = g.n[l];
        if constexpr (M <= 4) {
            // up to four overlaps: two elements per pass, every load of both
            // issued before the stores (a history slot is not known not to alias
            // the outputs, so the compiler would not move a later element's loads
            // above them).  The per-thread order of the dot-product terms is the
            // plain grid-stride order, as below.
            for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += 2 * stride) {
                const int64_t e1 = e + stride;
                const bool two = e1 < n;
                const int64_t x0 = base + e, x1 = base + e1;
                const double r0 = r[e], d0 = dinv[x0], t0 = t[e];
                const double r1 = two ? r[e1] : 0.0, d1 = two ? dinv[x1] : 0.0, t1 = two ? t[e1] : 0.0;
                double h0[M], h1[M];
#pragma unroll
                for (int h = 0; h < M; h++) {
                    // g.he[h] == eo: the slot the new error vector goes to (its overlap is q.q)
                    const bool rd = h < g.m && g.he[h] != eo;
                    h0[h] = rd ? g.he[h][x0] : 0.0;
                    h1[h] = rd && two ? g.he[h][x1] : 0.0;
                }
                const double q0 = r0 * d0, q1 = r1 * d1;
                eo[x0] = q0;
                xo[x0] = t0 + q0;
                if (two) {
                    eo[x1] = q1;
                    xo[x1] = t1 + q1;
                }
#pragma unroll
                for (int h = 0; h < M; h++)
                    if (h < g.m) {
                        const bool c = g.he[h] == eo;
                        acc[h] = fma(q0, c ? q0 : h0[h], acc[h]);
                        if (two) acc[h] = fma(q1, c ? q1 : h1[h], acc[h]);
                    }
            }
        } else {
            // more overlaps: one element per pass (the registers of a second
            // element would cut the resident warps)
            for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += stride) {
                const int64_t x = base + e;
                const double q = r[e] * dinv[x];
                eo[x] = q;
                xo[x] = t[e] + q;
                double hv[M];
#pragma unroll
                for (int h = 0; h < M; h++) hv[h] = (h < g.m && g.he[h] != eo) ? g.he[h][x] : q;
#pragma unroll
                for (int h = 0; h < M; h++)
                    if (h < g.m) acc[h] = fma(q, hv[h], acc[h]);
            }
        }
        base += n;
    }
#pragma unroll
    for (int h = 0; h < M; h++) {
        if (h >= g.m) break;
        const double sum = block_sum(acc[h]);
        if (threadIdx.x == 0) partials[(int64_t)h * kRedBlocks + blockIdx.x] = sum;
    }
}

cudaError_t launch_jacobi_dots(const JacobiSegs &g, const double *dinv, double *xo, double *eo, double *partials,
                               cudaStream_t s) {
    if (g.nseg < 1 || g.nseg > 3 || g.m < 0 || g.m > 16) return cudaErrorInvalidValue;
    if (g.m <= 4) jacobi_dots_kernel<4><<<kRedBlocks, 256, 0, s>>>(g, dinv, xo, eo, partials);
    else if (g.m <= 8) jacobi_dots_kernel<8><<<kRedBlocks, 256, 0, s>>>(g, dinv, xo, eo, partials);
    else jacobi_dots_kernel<16><<<kRedBlocks, 256, 0, s>>>(g, dinv, xo, eo, partials);
    return cudaGetLastError();
}

cudaError_t launch_dot_partials(const double *x, const double *y, int64_t n, double *partials, cudaStream_t s) {
    dot_partials_kernel<<<kRedBlocks, 256, 0, s>>>(x, y, n, partials);
    return cudaGetLastError();
}

// E = sum_ijab <ij||ab> (t2_ijab / 4 + t1_ia t1_jb / 2), the spin-orbital
// CC energy (the projection on Phi_0 of Eq. amp, Sec. II A), summed as
// 1/4 sum V (t2 + 2 t1_ia t1_jb): the factor 4 is a power of two, so the
// scaling commutes with every rounding (no subnormals) and is applied once per
// block.  Warps take rows (i, j, a) (a fixed mapping, so the sum order is
// deterministic), lanes run along b; the row's 2 t1_ia is formed once, so an
// element costs two FMAs and the loop body holds only loads and FMAs (no call
// that would keep the next iteration's loads from being issued early).
template <typename T>
__global__ void __launch_bounds__(256) energy_partials_kernel(int o, int v, const T *__restrict__ V,
                                                              const T *__restrict__ t1, const T *__restrict__ t2,
                                                              double *partials) {
    const int lane = threadIdx.x & 31;
    const uint32_t rows = (uint32_t)o * (uint32_t)o * (uint32_t)v;
    T s = zero<T>();
    for (uint32_t row = blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += kRedBlocks * 8) {
        const uint32_t a = row % (uint32_t)v, ij = row / (uint32_t)v;
        const uint32_t j = ij % (uint32_t)o, i = ij / (uint32_t)o;
        const T *__restrict__ vr = V + (int64_t)row * v;
        const T *__restrict__ tr = t2 + (int64_t)row * v;
        if (t1) {
            const T x = ld(t1 + (int64_t)i * v + a);
            const T c = add(x, x);
            const T *__restrict__ t1j = t1 + (int64_t)j * v;
            for (int b = lane; b < v; b += 32) s = cfma(ld(vr + b), cfma(c, ld(t1j + b), ld(tr + b)), s);
        } else {
            for (int b = lane; b < v; b += 32) s = cfma(ld(vr + b), ld(tr + b), s);
        }
    }
    if constexpr (sizeof(T) == sizeof(double)) {
        const double r = block_sum(s);
        if (threadIdx.x == 0) partials[blockIdx.x] = 0.25 * r;
    } else {
        const double re = block_sum(s.x), im = block_sum(s.y);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = 0.25 * re;
            partials[kRedBlocks + blockIdx.x] = 0.25 * im;
        }
    }
}

cudaError_t launch_energy_partials(int o, int v, const double *Voovv, const double *t1, const double *t2,
                                   double *partials, int cplx, cudaStream_t s) {
    if (cplx)
        energy_partials_kernel<double2><<<kRedBlocks, 256, 0, s>>>(
            o, v, reinterpret_cast<const double2 *>(Voovv), reinterpret_cast<const double2 *>(t1),
            reinterpret_cast<const double2 *>(t2), partials);
    else
        energy_partials_kernel<double><<<kRedBlocks, 256, 0, s>>>(o, v, Voovv, t1, t2, partials);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) reduce_partials_kernel(const double *partials, int count, double *out) {
    for (int c = 0; c < count; c++) {
        double s = 0.0;
        for (int k = threadIdx.x; k < kRedBlocks; k += 256) s += partials[(int64_t)c * kRedBlocks + k];
        s = block_sum(s);
        if (threadIdx.x == 0) out[c] = s;
    }
}

cudaError_t launch_reduce_partials(const double *partials, int count, double *out, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, count, out);
    return cudaGetLastError();
}

// ---- grouped post step: for every system of a batch, R -= D T over (R1 | R2)
// and the chunk partials of E = sum_ijab V (1/4 t2 + 1/2 t1 t1), |R1|^2, |R2|^2
// (one block per kPostChunk elements), then one warp per system sums its
// partials in a fixed order into scal.
__global__ void __launch_bounds__(256) grouped_post_kernel(const GroupedPost *__restrict__ tab, int n, int64_t total,
                                                          const int *__restrict__ active) {
    const Scale kTwo = {0, 1, 0u, 2.0};
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedPost> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedPost &g = tab[walk.at(it)];
        if (!active[g.sys]) { it = walk.next - 1; continue; }   // block-uniform
        const int64_t c = it - g.item0;
        const uint32_t o = (uint32_t)g.o, v = (uint32_t)g.v;
        const int64_t n1 = (int64_t)o * v, n2 = n1 * n1;
        double se = 0.0, s1 = 0.0, s2 = 0.0;
        const int64_t e1 = (c + 1) * kPostChunk < n1 + n2 ? (c + 1) * kPostChunk : n1 + n2;
        for (int64_t e = c * kPostChunk + threadIdx.x; e < e1; e += blockDim.x) {
            if (e < n1) {
                const uint32_t i = (uint32_t)e / v, a = (uint32_t)e - i * v;
                const double d = g.fo[i] - g.fv[a];
                const double r = fma(neg(d), g.t1[e], g.r1[e]);
                g.r1[e] = r;
                s1 = fma(r, r, s1);
            } else {
                const int64_t x = e - n1;
                // 32-bit division where the system's o^2 v^2 allows it (block-uniform)
                const uint32_t row = n2 <= 0xffffffffLL ? (uint32_t)x / v : (uint32_t)(x / v);
                const uint32_t b = (uint32_t)(x - (int64_t)row * v);
                const uint32_t a = row % v, ij = row / v, j = ij % o, i = ij / o;
                const double t2 = g.t2[x];
                const double d = (g.fo[i] + g.fo[j]) - (g.fv[a] + g.fv[b]);
                const double r = fma(neg(d), t2, g.r2[x]);
                g.r2[x] = r;
                s2 = fma(r, r, s2);
                // 2 t1_ia by the exponent field (exact, no FP64 instruction)
                const double tt =
                    g.t1 ? fma(scale_f64(g.t1[(int64_t)i * v + a], kTwo), g.t1[(int64_t)j * v + b], t2) : t2;
                se = fma(g.oovv[x], tt, se);
            }
        }
        se = block_sum(se);
        s1 = block_sum(s1);
        s2 = block_sum(s2);
        if (threadIdx.x == 0) {
            g.partials[c] = 0.25 * se;
            g.partials[g.chunks + c] = s1;
            g.partials[2 * g.chunks + c] = s2;
        }
    }
}

__global__ void __launch_bounds__(256) grouped_post_reduce_kernel(const GroupedPost *__restrict__ tab, int n,
                                                                 const int *__restrict__ active) {
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.x * 8 + (threadIdx.x >> 5); q < n; q += gridDim.x * 8) {
        const GroupedPost &g = tab[q];
        if (!active[g.sys]) continue;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; k++) {
            for (int64_t c = lane; c < g.chunks; c += 32) acc[k] += g.partials[k * g.chunks + c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
        }
        if (lane == 0) {
            g.scal[0] = acc[0];
            g.scal[1] = 0.0;
            g.scal[2] = acc[1];
            g.scal[3] = acc[2];
        }
    }
}

__global__ void __launch_bounds__(256) grouped_reduce_kernel(const GroupedReduce *__restrict__ tab, int n,
                                                            int64_t total, const int *__restrict__ active) {
    const WorkRange wr = work_range(total, blockIdx.x, gridDim.x);
    if (wr.begin >= wr.end) return;
    EntryWalk<GroupedReduce> walk(tab, n, wr.begin);
    for (int64_t it = wr.begin; it < wr.end; it++) {
        const GroupedReduce &g = tab[walk.at(it)];
        if (!active[g.sys]) { it = walk.next - 1; continue; }
        const int64_t e = (it - g.item0) * 256 + threadIdx.x, mn = g.M * g.N;
        if (e >= mn) continue;
        const int64_t nn = e / g.M, m = e - nn * g.M;
        double acc = 0.0;
        for (int z = 0; z < g.nslices; z++) acc += g.P[(int64_t)z * mn + e];
        double *c = g.C + grp_offset(g.cm, m) + grp_offset(g.cn, nn);
        const double v = scale_f64(acc, g.as);
        *c = g.bcase ? *c + v : v;
    }
}

cudaError_t launch_grouped_reduce(const GroupedReduce *tab, int n, int64_t total, const int *active, cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 16 ? total : 148 * 16);
    grouped_reduce_kernel<<<blocks, 256, 0, s>>>(tab, n, total, active);
    return cudaGetLastError();
}

cudaError_t launch_grouped_post(const GroupedPost *tab, int n, int64_t total, const int *active, cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(total < 148 * 8 ? total : 148 * 8);
    grouped_post_kernel<<<blocks, 256, 0, s>>>(tab, n, total, active);
    if (cudaError_t e = cudaGetLastError()) return e;
    grouped_post_reduce_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(tab, n, active);
    return cudaGetLastError();
}

struct Order {
    int s[16];
};

// DIIS: the bordered system [B 1; 1^T 0][c; l] = [0; 1] with B scaled by
// 1/max(diag B), Gaussian elimination with partial pivoting; while a pivot is
// below 1e-14 the oldest vector is dropped and the solve repeated (down to
// two vectors).  Returns the number of newest vectors used (0: none usable).
__device__ int diis_solve_dev(const double *gram16, const int *ord, int m, double *coef) {
    for (int mm = m; mm >= 2; mm--) {
        const int off = m - mm;     // drop the `off` oldest
        const int N = mm + 1;
        auto G = [&](int r, int c) { return gram16[ord[off + r] * 16 + ord[off + c]]; };
        double Am[17][18];
        double dmax = 0.0;
        for (int k = 0; k < mm; k++) dmax = fmax(dmax, G(k, k));
        if (!(dmax > 0.0)) continue;
        for (int r = 0; r < N; r++)
            for (int c = 0; c <= N; c++) Am[r][c] = 0.0;
        for (int r = 0; r < mm; r++) {
            for (int c = 0; c < mm; c++) Am[r][c] = G(r, c) / dmax;
            Am[r][mm] = 1.0;
            Am[mm][r] = 1.0;
        }
        Am[mm][N] = 1.0;
        bool ok = true;
        for (int c = 0; c < N && ok; c++) {
            int piv = c;
            for (int r = c + 1; r < N; r++)
                if (fabs(Am[r][c]) > fabs(Am[piv][c])) piv = r;
            if (fabs(Am[piv][c]) < 1e-14) { ok = false; break; }
            if (piv != c)
                for (int k = 0; k <= N; k++) { double t = Am[c][k]; Am[c][k] = Am[piv][k]; Am[piv][k] = t; }
            for (int r = c + 1; r < N; r++) {
                double f = Am[r][c] / Am[c][c];
                for (int k = c; k <= N; k++) Am[r][k] -= f * Am[c][k];
            }
        }
        if (!ok) continue;
        double x[17];
        for (int r = N - 1; r >= 0; r--) {
            double s = Am[r][N];
            for (int k = r + 1; k < N; k++) s -= Am[r][k] * x[k];
            x[r] = s / Am[r][r];
        }
        for (int k = 0; k < mm; k++) coef[k] = x[k];
        return mm;
    }
    return 0;
}

__global__ void diis_solve_kernel(const double *gram16, Order ord, int m, double *coef, int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    status[0] = diis_solve_dev(gram16, ord.s, m, coef);
}

cudaError_t launch_diis_solve(const double *gram16, const int *order_host, int m, double *coef, int *status,
                              cudaStream_t s) {
    Order o{};
    for (int k = 0; k < m && k < 16; k++) o.s[k] = order_host[k];
    diis_solve_kernel<<<1, 32, 0, s>>>(gram16, o, m, coef, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched
// offset of rank l inside a system's x vector
__device__ __forceinline__ int64_t rank_offset(const BatchSys &b, int l) {
    int64_t off = 0;
    for (int q = 1; q < l; q++) off += b.n[q];
    return off;
}

__global__ void __launch_bounds__(256) batched_jacobi_kernel(const BatchSys *__restrict__ sys) {
    const BatchSys &b = sys[blockIdx.y];
    if (!b.active) return;
    double *xs = b.hx + (int64_t)b.slot * b.nx, *es = b.he + (int64_t)b.slot * b.nx;
    for (int l = 1; l <= 3; l++) {
        if (!b.t[l]) continue;
        const int64_t off = rank_offset(b, l);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b.n[l];
             e += (int64_t)gridDim.x * blockDim.x) {
            const double q = b.r[l][e] * b.dinv[off + e];
            es[off + e] = q;
            xs[off + e] = b.t[l][e] + q;
        }
    }
}

// block partials of <e_slot | e_order[q]>, q < nstored: partials[q][blockIdx.x]
__global__ void __launch_bounds__(256) batched_dots_kernel(const BatchSys *__restrict__ sys) {
    const BatchSys &b = sys[blockIdx.y];
    if (!b.active) return;
    const double *es = b.he + (int64_t)b.slot * b.nx;
    for (int q = 0; q < b.nstored; q++) {
        const double *eq = b.he + (int64_t)b.order[q] * b.nx;
        double acc = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < b.nx; e += (int64_t)kBatchBlocks * 256)
            acc = fma(es[e], eq[e], acc);
        acc = block_sum(acc);
        if (threadIdx.x == 0) b.partials[q * kBatchBlocks + blockIdx.x] = acc;
    }
}

// one block per system: the Gram row of the new slot, then the DIIS solve
__global__ void __launch_bounds__(256) batched_gram_solve_kernel(const BatchSys *__restrict__ sys) {
    const BatchSys &b = sys[blockIdx.x];
    if (!b.active) return;
    for (int q = 0; q < b.nstored; q++) {
        double x = threadIdx.x < kBatchBlocks ? b.partials[q * kBatchBlocks + threadIdx.x] : 0.0;
        x = block_sum(x);
        if (threadIdx.x == 0) {
            b.gram[b.slot * 16 + b.order[q]] = x;
            b.gram[b.order[q] * 16 + b.slot] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *b.used = b.nstored >= 2 ? diis_solve_dev(b.gram, b.order, b.nstored, b.coef) : 0;
}

__global__ void __launch_bounds__(256) batched_combine_kernel(const BatchSys *__restrict__ sys) {
    const BatchSys &b = sys[blockIdx.y];
    if (!b.active) return;
    const int m = b.nstored;
    const int used = m >= 2 ? *b.used : 0;
    for (int l = 1; l <= 3; l++) {
        if (!b.t[l]) continue;
        const int64_t off = rank_offset(b, l);
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b.n[l];
             e += (int64_t)gridDim.x * blockDim.x) {
            double x;
            if (used == 0) {
                x = b.hx[(int64_t)(m >= 2 ? b.order[m - 1] : b.slot) * b.nx + off + e];
            } else {
                x = 0.0;
                for (int k = 0; k < used; k++) x += b.coef[k] * b.hx[(int64_t)b.order[m - used + k] * b.nx + off + e];
            }
            b.t[l][e] = x;
        }
    }
}

cudaError_t launch_batched_jacobi(const BatchSys *sys, int nsys, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    batched_jacobi_kernel<<<dim3(kBatchBlocks, (unsigned)nsys), 256, 0, s>>>(sys);
    return cudaGetLastError();
}

cudaError_t launch_batched_diis(const BatchSys *sys, int nsys, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    batched_dots_kernel<<<dim3(kBatchBlocks, (unsigned)nsys), 256, 0, s>>>(sys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batched_gram_solve_kernel<<<(unsigned)nsys, 256, 0, s>>>(sys);
    return cudaGetLastError();
}

cudaError_t launch_batched_combine(const BatchSys *sys, int nsys, cudaStream_t s) {
    if (nsys <= 0) return cudaSuccess;
    batched_combine_kernel<<<dim3(kBatchBlocks, (unsigned)nsys), 256, 0, s>>>(sys);
    return cudaGetLastError();
}

struct PairPack {
    int2 p[16];
};

// gram16[a_k*16 + b_k] = gram16[b_k*16 + a_k] = sum of partials row k (fixed order)
__global__ void __launch_bounds__(256) gram_scatter_kernel(const double *partials, int count, PairPack pk,
                                                           double *gram16) {
    for (int c = 0; c < count; c++) {
        double s = 0.0;
        for (int k = threadIdx.x; k < kRedBlocks; k += 256) s += partials[(int64_t)c * kRedBlocks + k];
        s = block_sum(s);
        if (threadIdx.x == 0) {
            int2 pr = pk.p[c];
            gram16[pr.x * 16 + pr.y] = s;
            gram16[pr.y * 16 + pr.x] = s;
        }
    }
}

cudaError_t launch_gram_scatter(const double *partials, int count, const int *a_host, const int *b_host,
                                double *gram16, cudaStream_t s) {
    PairPack pk{};
    for (int k = 0; k < count && k < 16; k++) pk.p[k] = make_int2(a_host[k], b_host[k]);
    gram_scatter_kernel<<<1, 256, 0, s>>>(partials, count, pk, gram16);
    return cudaGetLastError();
}

struct PtrPack {
    const double *p[16];
};

// x = sum_k coef[k] * xs[m - used + k] over the `used` newest vectors
// (used read from the device; used == 0 copies the newest vector).
__global__ void combine_kernel(PtrPack xs, const double *coef, const int *used_dev, int m, int64_t n, double *x) {
    const int used = *used_dev;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s;
        if (used == 0) {
            s = xs.p[m - 1][e];
        } else {
            s = 0.0;
            for (int k = 0; k < used; k++) s += coef[k] * xs.p[m - used + k][e];
        }
        x[e] = s;
    }
}

cudaError_t launch_combine(const double *const *xs_host, const double *coef, const int *used_dev, int m, int64_t n,
                           double *x, cudaStream_t s) {
    PtrPack pk{};
    for (int k = 0; k < m && k < 16; k++) pk.p[k] = xs_host[k];
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(pk, coef, used_dev, m, n, x);
    return cudaGetLastError();
}

}  // namespace ccb
