// diagnostics.cu -- convergence and efficiency diagnostics of the chains, on the device.
//
// Sec. 3.1 judges samplers by the integrated autocorrelation time kappa of the tau^2 chain, the
// effective sample size N / kappa and the cost per effective sample CES = kappa T / N, and by
// Gelman plots (potential scale reduction over chains).  Here:
//   * trace_iat_kernel: one block per chain; the last N values of a parameter trace, kappa by
//     Geyer's initial monotone sequence estimator (Geyer 1992, Statistical Science 7, Sec. 3.3),
//     and the chain's mean and variance;
//   * trace_psrf_kernel: the potential scale reduction factor over chains (Gelman & Rubin 1992
//     with the (m + 1)/m factor of Brooks & Gelman 1998) from those moments;
//   * site_psrf_kernel: the same factor for every site, from the running means and M2 of the
//     accumulated sweeps, in natural site order, and its maximum.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

constexpr int kDiagBlock = 256;

// Deterministic block sum in FP64: thread-strided partial sums, a shuffle tree per warp, then the
// warps' sums in order by thread 0; every thread gets the result.
__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kDiagBlock / 32; ++w) s += red[w];
        red[kDiagBlock / 32] = s;
    }
    __syncthreads();
    return red[kDiagBlock / 32];
}

// Potential scale reduction factor from m chains' means and variances (divisor N - 1).
__device__ double psrf_from_moments(const double *mean, const double *var, int m, long long N, int stride)
{
    if (m < 2 || N < 2) return nan("");
    double W = 0.0, mm = 0.0;
    for (int c = 0; c < m; ++c) {
        W += var[c * stride];
        mm += mean[c * stride];
    }
    W /= m;
    mm /= m;
    double BN = 0.0;
    for (int c = 0; c < m; ++c) {
        const double d = mean[c * stride] - mm;
        BN += d * d;
    }
    BN /= (m - 1);
    if (!(W > 0.0)) return nan("");
    const double V = static_cast<double>(N - 1) / static_cast<double>(N) * W + static_cast<double>(m + 1) / m * BN;
    return sqrt(V / W);
}

__global__ void __launch_bounds__(kDiagBlock) trace_iat_kernel(const DiagArgs a)
{
    __shared__ double red[kDiagBlock / 32 + 1];
    __shared__ double gam[kDiagBlock];
    __shared__ int done;
    const int c = blockIdx.x;
    const double *tr = a.trace + static_cast<int64_t>(c) * a.cap;
    double *x = a.work + static_cast<int64_t>(c) * a.N;
    const long long N = a.N;
    // Gather the last N values (oldest first) from the ring buffer.
    for (long long q = threadIdx.x; q < N; q += kDiagBlock) {
        const long long sw = a.sweep - N + q;
        const double v = tr[sw % a.cap];
        x[q] = a.reciprocal ? 1.0 / v : v;
    }
    __syncthreads();
    double s = 0.0;
    for (long long q = threadIdx.x; q < N; q += kDiagBlock) s += x[q];
    const double mean = block_sum(s, red) / static_cast<double>(N);
    double s2 = 0.0;
    for (long long q = threadIdx.x; q < N; q += kDiagBlock) {
        const double d = x[q] - mean;
        s2 += d * d;
    }
    const double g0 = block_sum(s2, red) / static_cast<double>(N);
    double *out = a.out + static_cast<int64_t>(c) * 4;
    if (N < 4 || !(g0 > 0.0)) {
        if (threadIdx.x == 0) {
            out[0] = nan("");
            out[1] = nan("");
            out[2] = mean;
            out[3] = N > 1 ? g0 * N / (N - 1) : nan("");
        }
        return;
    }
    // Autocovariances lag by lag, one lag per thread, chunk by chunk until the initial positive
    // sequence ends; thread 0 walks the pairs (gamma(2m), gamma(2m + 1)) of each chunk in order.
    double sum = 0.0, run_min = 1e300;
    if (threadIdx.x == 0) done = 0;
    __syncthreads();
    for (long long k0 = 0; k0 < N; k0 += kDiagBlock) {
        const long long k = k0 + threadIdx.x;
        double g = 0.0;
        if (k < N) {
            double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;  // four chains of dependent FP64 adds
            long long t = 0;
            for (; t + 3 + k < N; t += 4) {
                p0 += (x[t] - mean) * (x[t + k] - mean);
                p1 += (x[t + 1] - mean) * (x[t + 1 + k] - mean);
                p2 += (x[t + 2] - mean) * (x[t + 2 + k] - mean);
                p3 += (x[t + 3] - mean) * (x[t + 3 + k] - mean);
            }
            for (; t + k < N; ++t) p0 += (x[t] - mean) * (x[t + k] - mean);
            g = ((p0 + p1) + (p2 + p3)) / static_cast<double>(N);
        }
        gam[threadIdx.x] = g;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j + 1 < kDiagBlock && !done; j += 2) {
                const long long m = (k0 + j) / 2;
                if (2 * m + 1 > N - 1) {
                    done = 1;
                    break;
                }
                const double G = gam[j] + gam[j + 1];
                if (m > 0 && !(G > 0.0)) {
                    done = 1;
                    break;
                }
                run_min = G < run_min ? G : run_min;
                sum += run_min;
                if (!(G > 0.0)) done = 1;
            }
        }
        __syncthreads();
        if (done) break;
    }
    if (threadIdx.x == 0) {
        double kappa = (-g0 + 2.0 * sum) / g0;
        const double floor_k = 1.0 / log10(static_cast<double>(N));
        kappa = kappa < floor_k ? floor_k : kappa;
        out[0] = kappa;
        out[1] = static_cast<double>(N) / kappa;
        out[2] = mean;
        out[3] = g0 * N / (N - 1);
    }
}

__global__ void trace_psrf_kernel(const DiagArgs a)
{
    a.psrf[0] = psrf_from_moments(a.out + 2, a.out + 3, a.chains, a.N, 4);
}

template <typename T>
__global__ void site_psrf_kernel(const FieldDev *fields, int32_t fidx, int32_t Cp, int32_t C, const T *mean,
                                 const T *m2, long long count, const int32_t *perm_inv, double *out,
                                 unsigned long long *max_bits)
{
    const FieldDev f = fields[fidx];
    double mu[kMaxChains], var[kMaxChains];
    unsigned long long local = 0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < f.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = f.slot0 + (f.kind == kCsr ? perm_inv[f.csr0 + i] : lattice_slot_of_site(f, i));
        for (int c = 0; c < C; ++c) {
            mu[c] = static_cast<double>(mean[slot * Cp + c]);
            var[c] = static_cast<double>(m2[slot * Cp + c]) / static_cast<double>(count - 1);
        }
        const double r = psrf_from_moments(mu, var, C, count, 1);
        out[i] = r;
        if (r == r) {
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(r));
            local = b > local ? b : local;
        }
    }
    if (local) atomicMax(max_bits, local);
}

}  // namespace

cudaError_t launch_trace_diagnostics(const DiagArgs &a, cudaStream_t stream)
{
    trace_iat_kernel<<<a.chains, kDiagBlock, 0, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    trace_psrf_kernel<<<1, 1, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_site_psrf(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t Cp,
                             int32_t C, const void *mean, const void *m2, long long count, const int32_t *perm_inv,
                             double *out, unsigned long long *max_bits, cudaStream_t stream)
{
    int64_t g = (static_cast<int64_t>(f.n) + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    if (precision == 0)
        site_psrf_kernel<float><<<static_cast<int>(g), 256, 0, stream>>>(
            fields_dev, fidx, Cp, C, static_cast<const float *>(mean), static_cast<const float *>(m2), count, perm_inv,
            out, max_bits);
    else
        site_psrf_kernel<double><<<static_cast<int>(g), 256, 0, stream>>>(
            fields_dev, fidx, Cp, C, static_cast<const double *>(mean), static_cast<const double *>(m2), count,
            perm_inv, out, max_bits);
    return cudaGetLastError();
}

}  // namespace gmrf
