// accumulate.cu -- the estimator side of the sampler (Eq. 1/C, Eq. tr, Sec. 2.3):
//   * folding the sweep's FP32 diagonal partials into FP64 per-chain-group sums,
//   * the FP32 CUDA-core block contraction  blk += Z_R W_S^dagger  (one cycle),
//   * folding block batches into FP64 sums and batch-mean second moments,
//   * means and Monte Carlo standard errors in FP64.
#include <algorithm>

#include "internal.h"

namespace mcinv {

// acc[g][perm[p]] += sum over the group's units of part[u][p]; part is
// cleared.  Units are grouped contiguously: group g owns units
// [g*upg, (g+1)*upg); part is indexed by position p, acc by row.
template <typename T, int NV>
__global__ void diag_fold_kernel(int n, int units, int G, const int *__restrict__ perm,
                                 T *__restrict__ part, double *__restrict__ acc)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (p >= n) return;
    const int upg = units / G;
    const int i = perm[p];
    double s[NV] = {};
    for (int k = 0; k < upg; ++k) {
        T *src = part + (size_t)(g * upg + k) * n + p;
        const float *f = (const float *)src;
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += (double)f[v];
        *src = T{};
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[((size_t)g * n + i) * NV + v] += s[v];
}

cudaError_t launch_diag_fold(int cplx, int n, int units, int G, const int *perm, void *diag_part,
                             double *acc, cudaStream_t s)
{
    dim3 grid((n + 255) / 256, G);
    if (cplx) diag_fold_kernel<float2, 2><<<grid, 256, 0, s>>>(n, units, G, perm, (float2 *)diag_part, acc);
    else diag_fold_kernel<float, 1><<<grid, 256, 0, s>>>(n, units, G, perm, (float *)diag_part, acc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 SIMT block contraction for one cycle: blk[a][b] += sum_c z[R_a][c] conj(w[S_b][c]).
// 64x64 output tile per CTA, 256 threads with a 4x4 register tile each; chains
// are the contraction dimension, staged through shared memory 16 at a time.
// ---------------------------------------------------------------------------
template <bool CPLX>
struct BlkT;
template <> struct BlkT<false> { using T = float; };
template <> struct BlkT<true> { using T = float2; };

template <bool CPLX>
__global__ void __launch_bounds__(256) block_simt_kernel(int K, const typename BlkT<CPLX>::T *__restrict__ z,
                                                         const typename BlkT<CPLX>::T *__restrict__ w,
                                                         const int *__restrict__ R, int nR,
                                                         const int *__restrict__ S, int nS,
                                                         float *__restrict__ blk)
{
    using T = typename BlkT<CPLX>::T;
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int a0 = blockIdx.y * BM, b0 = blockIdx.x * BN;
    float acc[4][4][CPLX ? 2 : 1] = {};
    // loader mapping: 256 threads cover 64 rows x 16 chains with 4 loads each
    const int lc = tid % BK, lr = tid / BK;  // lr in [0,16)
    for (int c0 = 0; c0 < K; c0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lr + 16 * q;
            const int c = c0 + lc;
            T va{}, vb{};
            if (c < K && a0 + r < nR) va = z[(size_t)R[a0 + r] * K + c];
            if (c < K && b0 + r < nS) vb = w[(size_t)S[b0 + r] * K + c];
            As[lc][r] = va;
            Bs[lc][r] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T ra[4], rb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { ra[q] = As[kk][ty + 16 * q]; rb[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    if constexpr (!CPLX) {
                        acc[x][y][0] = fmaf(ra[x], rb[y], acc[x][y][0]);
                    } else {  // z conj(w)
                        acc[x][y][0] = fmaf(ra[x].x, rb[y].x, fmaf(ra[x].y, rb[y].y, acc[x][y][0]));
                        acc[x][y][1] = fmaf(ra[x].y, rb[y].x, fmaf(-ra[x].x, rb[y].y, acc[x][y][1]));
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int a = a0 + ty + 16 * x, b = b0 + tx + 16 * y;
            if (a < nR && b < nS) {
                const size_t o = ((size_t)a * nS + b) * (CPLX ? 2 : 1);
                blk[o] += acc[x][y][0];
                if constexpr (CPLX) blk[o + 1] += acc[x][y][1];
            }
        }
}

cudaError_t launch_block_simt(int cplx, int K, const void *z, const void *w, const int *R, int nR,
                              const int *S, int nS, float *blk, cudaStream_t s)
{
    dim3 grid((nS + 63) / 64, (nR + 63) / 64);
    if (cplx) block_simt_kernel<true><<<grid, 256, 0, s>>>(K, (const float2 *)z, (const float2 *)w, R, nR, S, nS, blk);
    else block_simt_kernel<false><<<grid, 256, 0, s>>>(K, (const float *)z, (const float *)w, R, nR, S, nS, blk);
    return cudaGetLastError();
}

// sum += blk; sq += blk^2 * scale_sq (scale_sq = 1/(K^2 B) makes sq the
// batch-length-weighted second moment of the batch means); optionally blk = 0.
// sum += x, sq += x^2 scale for the FP32 batch product x, eight elements a
// thread per step with every load issued before the stores (16-byte accesses)
// to keep enough bytes in flight; explicit round-to-nearest double operations.
__global__ void block_fold_kernel(long long elems, double scale_sq, float *__restrict__ blk,
                                  double *__restrict__ sum, double *__restrict__ sq, int zero_blk, int vec)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n8 = vec ? elems / 8 : 0;  // whole octets first when the arrays are 16-byte aligned
    float4 *__restrict__ D4 = (float4 *)blk;
    double2 *__restrict__ s2 = (double2 *)sum;
    double2 *__restrict__ q2 = (double2 *)sq;
    for (long long e = e0; e < n8; e += stride) {
        const float4 v0 = D4[2 * e], v1 = D4[2 * e + 1];
        double2 a[4], c[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) { a[h] = s2[4 * e + h]; c[h] = q2[4 * e + h]; }
        const double x[8] = {(double)v0.x, (double)v0.y, (double)v0.z, (double)v0.w,
                             (double)v1.x, (double)v1.y, (double)v1.z, (double)v1.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            a[h].x = __dadd_rn(a[h].x, x[2 * h]);
            a[h].y = __dadd_rn(a[h].y, x[2 * h + 1]);
            c[h].x = __fma_rn(__dmul_rn(x[2 * h], x[2 * h]), scale_sq, c[h].x);
            c[h].y = __fma_rn(__dmul_rn(x[2 * h + 1], x[2 * h + 1]), scale_sq, c[h].y);
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) { s2[4 * e + h] = a[h]; q2[4 * e + h] = c[h]; }
        if (zero_blk) {
            D4[2 * e] = make_float4(0.f, 0.f, 0.f, 0.f);
            D4[2 * e + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (long long e = 8 * n8 + e0; e < elems; e += stride) {
        const double x = blk[e];
        sum[e] = __dadd_rn(sum[e], x);
        sq[e] = __fma_rn(__dmul_rn(x, x), scale_sq, sq[e]);
        if (zero_blk) blk[e] = 0.f;
    }
}

cudaError_t launch_block_fold(int cplx, long long elems, double scale_sq, float *blk, double *sum,
                              double *sq, int zero_blk, cudaStream_t s)
{
    const long long total = elems * (cplx ? 2 : 1);
    const int vec = ((uintptr_t)blk % 16 == 0 && (uintptr_t)sum % 16 == 0 && (uintptr_t)sq % 16 == 0) ? 1 : 0;
    long long blocks = ((vec ? total / 8 : total) + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    if (blocks < 1) blocks = 1;
    block_fold_kernel<<<(unsigned)blocks, 256, 0, s>>>(total, scale_sq, blk, sum, sq, zero_blk, vec);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Estimates.  Group SE: with group sums A_g over n_g chains and `samples`
// cycles, m_g = A_g/(n_g samples), m = sum A_g/(N samples) and
// SE^2 = sum_g n_g (m_g - m)^2 / ((G-1) N).  Real and imaginary parts apart.
// ---------------------------------------------------------------------------
template <int NV>
__global__ void diag_estimate_kernel(int n, int G, const double *__restrict__ counts, double samples,
                                     const double *__restrict__ acc, double *__restrict__ mean,
                                     double *__restrict__ se)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double N = 0.0;
    for (int g = 0; g < G; ++g) N += counts[g];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot += acc[((size_t)g * n + i) * NV + v];
        const double m = tot / (N * samples);
        double ss = 0.0;
        for (int g = 0; g < G; ++g) {
            const double mg = acc[((size_t)g * n + i) * NV + v] / (counts[g] * samples);
            ss += counts[g] * (mg - m) * (mg - m);
        }
        mean[(size_t)i * NV + v] = m;
        se[(size_t)i * NV + v] = G > 1 ? sqrt(ss / ((G - 1) * N)) : nan("");
    }
}

cudaError_t launch_diag_estimate(int cplx, int n, int G, const double *counts, double samples,
                                 const double *acc, double *mean, double *se, cudaStream_t s)
{
    if (cplx) diag_estimate_kernel<2><<<(n + 255) / 256, 256, 0, s>>>(n, G, counts, samples, acc, mean, se);
    else diag_estimate_kernel<1><<<(n + 255) / 256, 256, 0, s>>>(n, G, counts, samples, acc, mean, se);
    return cudaGetLastError();
}

// tr(Q C^-1) per group: t_g = sum_i q_i A_g[i] (fixed-order block reduction),
// then the same group mean / SE as above.  out = [mean (NV), se (NV)].
template <int NV>
__global__ void __launch_bounds__(1024) trace_estimate_kernel(int n, int G, const double *__restrict__ counts,
                                                              double samples, const double *__restrict__ acc,
                                                              const double *__restrict__ q,
                                                              double *__restrict__ out)
{
    __shared__ double red[1024];
    __shared__ double tg[1024][NV];  // G <= 1024
    for (int g = 0; g < G; ++g) {
        for (int v = 0; v < NV; ++v) {
            double s = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) s += q[i] * acc[((size_t)g * n + i) * NV + v];
            red[threadIdx.x] = s;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) tg[g][v] = red[0];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        double N = 0.0;
        for (int g = 0; g < G; ++g) N += counts[g];
        for (int v = 0; v < NV; ++v) {
            double tot = 0.0;
            for (int g = 0; g < G; ++g) tot += tg[g][v];
            const double m = tot / (N * samples);
            double ss = 0.0;
            for (int g = 0; g < G; ++g) {
                const double mg = tg[g][v] / (counts[g] * samples);
                ss += counts[g] * (mg - m) * (mg - m);
            }
            out[v] = m;
            out[NV + v] = G > 1 ? sqrt(ss / ((G - 1) * N)) : nan("");
        }
    }
}

cudaError_t launch_trace_estimate(int cplx, int n, int G, const double *counts, double samples,
                                  const double *acc, const double *q, double *out, cudaStream_t s)
{
    if (G > 1024) return cudaErrorInvalidValue;
    if (cplx) trace_estimate_kernel<2><<<1, 1024, 0, s>>>(n, G, counts, samples, acc, q, out);
    else trace_estimate_kernel<1><<<1, 1024, 0, s>>>(n, G, counts, samples, acc, q, out);
    return cudaGetLastError();
}

// Block: batch means.  sum = sum_b X_b, sq = sum_b X_b^2/(K^2 B_b) = sum_b B_b m_b^2,
// T = sum_b B_b cycles, nb batches: m = sum/(K T),
// SE^2 = (sq - m^2 T) / (T (nb - 1)).
__global__ void block_estimate_kernel(long long elems, double K, double T, double nb,
                                      const double *__restrict__ sum, const double *__restrict__ sq,
                                      double *__restrict__ mean, double *__restrict__ se)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < elems;
         e += (long long)gridDim.x * blockDim.x) {
        const double m = sum[e] / (K * T);
        const double v = fmax(sq[e] - m * m * T, 0.0);
        mean[e] = m;
        se[e] = nb > 1 ? sqrt(v / (T * (nb - 1))) : nan("");
    }
}

cudaError_t launch_block_estimate(int cplx, long long elems, double K, double T, double nb,
                                  const double *sum, const double *sq, double *mean, double *se,
                                  cudaStream_t s)
{
    const long long total = elems * (cplx ? 2 : 1);
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    block_estimate_kernel<<<(unsigned)blocks, 256, 0, s>>>(total, K, T, nb, sum, sq, mean, se);
    return cudaGetLastError();
}

__global__ void series_fold_kernel(int ncyc, int ctas, int warps, const float *__restrict__ tpart, double K,
                                   double *__restrict__ series, long long first)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncyc) return;
    double s = 0.0;
    for (int k = 0; k < ctas * warps; ++k) s += (double)tpart[(size_t)c * ctas * warps + k];
    series[first + c] = s / K;
}

cudaError_t launch_series_fold(int ncyc, int ctas, int warps, const float *tpart, double K, double *series,
                               long long first, cudaStream_t s)
{
    series_fold_kernel<<<(ncyc + 127) / 128, 128, 0, s>>>(ncyc, ctas, warps, tpart, K, series, first);
    return cudaGetLastError();
}

// max_i |d_i| of two length-n vectors (float or float2), as float bits in out[0], out[1]
// (non-negative floats order like their integer bit patterns)
template <int NV>
__global__ void maxabs2_kernel(int n, const float *__restrict__ a, const float *__restrict__ b, unsigned *out)
{
    float ma = 0.f, mb = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (NV == 1) {
            ma = fmaxf(ma, fabsf(a[i]));
            mb = fmaxf(mb, fabsf(b[i]));
        } else {
            ma = fmaxf(ma, hypotf(a[2 * i], a[2 * i + 1]));
            mb = fmaxf(mb, hypotf(b[2 * i], b[2 * i + 1]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // NaN (a diverged difference) has the largest bit pattern, so it never passes the test
        atomicMax(&out[0], __float_as_uint(ma));
        atomicMax(&out[1], __float_as_uint(mb));
    }
}

cudaError_t launch_maxabs2(int cplx, int n, const void *a, const void *b, unsigned *out, cudaStream_t s)
{
    const int blocks = std::min((n + 255) / 256, 152 * 4);
    if (cplx) maxabs2_kernel<2><<<blocks, 256, 0, s>>>(n, (const float *)a, (const float *)b, out);
    else maxabs2_kernel<1><<<blocks, 256, 0, s>>>(n, (const float *)a, (const float *)b, out);
    return cudaGetLastError();
}

// d = (1, 2, ..., n): the difference z* - z of the coupled starts of Algorithm 1, step 1
template <int NV>
__global__ void iota1_kernel(int n, float *d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d[NV * i] = (float)(i + 1);
    if (NV == 2) d[2 * i + 1] = 0.f;
}

cudaError_t launch_iota1(int cplx, int n, void *d, cudaStream_t s)
{
    if (cplx) iota1_kernel<2><<<(n + 255) / 256, 256, 0, s>>>(n, (float *)d);
    else iota1_kernel<1><<<(n + 255) / 256, 256, 0, s>>>(n, (float *)d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block partition (Sec. 4): the products z_r conj(w_s) of the rows of one
// diagonal block, per chain group, summed in FP64 in chain order (one thread
// per (entry, group)); the estimate maps them through S_b^-1 on both sides.
template <int NV>
__global__ void pblock_acc_kernel(int nent, const int *__restrict__ ent_r, const int *__restrict__ ent_s, int K,
                                  int G, const int *__restrict__ gch, const float *__restrict__ z,
                                  const float *__restrict__ w, double *__restrict__ acc)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nent * G) return;
    const int e = (int)(t % nent), g = (int)(t / nent);
    const size_t r = (size_t)ent_r[e], s = (size_t)ent_s[e];
    double re = 0.0, im = 0.0;
    for (int c = gch[g]; c < gch[g + 1]; ++c) {
        if (NV == 1) {
            re += (double)z[r * K + c] * (double)w[s * K + c];
        } else {
            const double zr = z[(r * K + c) * 2], zi = z[(r * K + c) * 2 + 1];
            const double wr = w[(s * K + c) * 2], wi = w[(s * K + c) * 2 + 1];
            re += zr * wr + zi * wi;  // z conj(w)
            im += zi * wr - zr * wi;
        }
    }
    acc[((size_t)g * nent + e) * NV] += re;
    if (NV == 2) acc[((size_t)g * nent + e) * NV + 1] += im;
}

cudaError_t launch_pblock_acc(int cplx, int nent, const int *ent_r, const int *ent_s, int K, int G, const int *gch,
                              const void *z, const void *w, double *acc, cudaStream_t s)
{
    const long long threads = (long long)nent * G;
    if (threads == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (cplx)
        pblock_acc_kernel<2><<<blocks, 256, 0, s>>>(nent, ent_r, ent_s, K, G, gch, (const float *)z, (const float *)w, acc);
    else
        pblock_acc_kernel<1><<<blocks, 256, 0, s>>>(nent, ent_r, ent_s, K, G, gch, (const float *)z, (const float *)w, acc);
    return cudaGetLastError();
}

__global__ void scatter_kernel(int count, const long long *__restrict__ idx, const double *__restrict__ val,
                               double *__restrict__ dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) dst[idx[k]] = val[k];
}

cudaError_t launch_scatter(int count, const long long *idx, const double *val, double *dst, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    scatter_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, idx, val, dst);
    return cudaGetLastError();
}

}  // namespace mcinv
