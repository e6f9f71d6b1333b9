// wos_spectral.cu -- spectral diagnostics of one operator from its SVD (paper
// Sec. 5.2 items (i)-(iv); Eq. (Lambda_tilde_nu), (rho omega1 MC),
// (eigenfunctions_MC), (tsvd solution simulations)), FP64 throughout.
//
// From U, S, V of B = diag(nu) A_1 diag(sigma)^{-1/2} and the counts:
//   lambda_j      = S_j^2, the eigenvalues of Lambda^nu (Prop. coro:B-Lambda);
//   eigfun(l, j)  = S_j^{-1} sum_i nu_i U_ij rho_i(l), rho_i(l) = A_il / sigma_l;
//   density(l)    = (1 / M_D) sum_i rho_i(l);
//   u^(r)         = diag(sigma)^{-1/2} V_r Sigma_r^{-1} U_r^T diag(nu) b,
//                   b = u^D - A_0 u^0, for every r = 1..r_max (prefix sums of
//                   one coefficient vector);
//   uD^(r)        = A_1 u^(r) + A_0 u^0.
// The TSVD family uses the arithmetic of wos_reconstruct in the same order,
// so u^(r) and uD^(r) equal a reconstruction at truncation r bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "wos.h"
#include "wos_internal.h"

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL, v, o);
    return __shfl_sync(FULL, v, 0);
}

__global__ void lambda_kernel(const double *S, int k, double *lam)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x)
        lam[j] = S[j] * S[j];
}

// One thread per (l, j): the sum over the points runs down a count column
// (one address per block) and along a row of U (coalesced over j).
__global__ void eigfun_kernel(const double *U, const double *S, int M_D, int k,
                              const uint32_t *counts, int M_tot, double invN,
                              const int *g1_idx, const double *nu, const double *sigma,
                              double *eigfun)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (j >= k)
        return;
    const int col = g1_idx[l];
    const double nu_def = 1.0 / sqrt(double(M_D));
    double s = 0.0;
    for (int i = 0; i < M_D; ++i)
        s = fma((nu ? nu[i] : nu_def) * U[size_t(i) * k + j],
                double(counts[size_t(i) * M_tot + col]), s);
    const double sj = S[j];
    eigfun[size_t(l) * k + j] = sj > 0.0 ? s * invN / (sigma[col] * sj) : 0.0;
}

// density(l) = (1 / M_D) sum_i C[i][g1_l] / (N sigma): one warp per l.
__global__ void density_kernel(const uint32_t *counts, int M_D, int M_tot, double invN,
                               const int *g1_idx, int M_1, const double *sigma,
                               double *density)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int l = gw; l < M_1; l += nw) {
        const int col = g1_idx[l];
        double s = 0.0;
        for (int i = lane; i < M_D; i += 32)
            s += double(counts[size_t(i) * M_tot + col]);
        s = warp_sum(s);
        if (lane == 0)
            density[l] = s * invN / (double(M_D) * sigma[col]);
    }
}

__global__ void scatter_kernel(const int *idx, int n, const double *vals, double *f)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        f[idx[q]] = vals ? vals[q] : 0.0;
}

// y[i] = x[i] + alpha (C f)[i] / N, one warp per row.
__global__ void counts_matvec_kernel(const uint32_t *counts, int M_D, int M_tot, double invN,
                                     const double *f, const double *x, double alpha,
                                     double *y)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < M_D; i += nw) {
        const uint32_t *row = counts + size_t(i) * M_tot;
        double s = 0.0;
        for (int j = lane; j < M_tot; j += 32)
            s = fma(double(row[j]), f[j], s);
        s = warp_sum(s);
        if (lane == 0)
            y[i] = (x ? x[i] : 0.0) + alpha * s * invN;
    }
}

// t_c = sum_i U[i][c] nu_i b_i / S_c, c < r (one warp per c).
__global__ void coef_kernel(const double *U, const double *S, int M_D, int k, int r,
                            const double *nu, const double *b, double *t)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const double nu_def = 1.0 / sqrt(double(M_D));
    for (int c = gw; c < r; c += nw) {
        double s = 0.0;
        for (int i = lane; i < M_D; i += 32)
            s = fma(U[size_t(i) * k + c], (nu ? nu[i] : nu_def) * b[i], s);
        s = warp_sum(s);
        if (lane == 0) {
            const double sc = S[c];
            t[c] = (sc > 0.0 ? 1.0 / sc : 0.0) * s;
        }
    }
}

// u_sweep[r][l] = sum_{c <= r} V[l][c] t_c / sqrt(sigma): prefix sums, one
// thread per element.
__global__ void usweep_kernel(const double *V, int M_1, int k, int r_max, const double *t,
                              const int *g1_idx, const double *sigma, double *u_sweep)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M_1;
         l += gridDim.x * blockDim.x) {
        const double sq = sqrt(sigma[g1_idx[l]]);
        double s = 0.0;
        for (int c = 0; c < r_max; ++c) {
            s = fma(V[size_t(l) * k + c], t[c], s);
            u_sweep[size_t(c) * M_1 + l] = s / sq;
        }
    }
}

// Every row of F starts as f0 (u0 on Gamma_0, zero on Gamma_1) ...
__global__ void fill_f_kernel(const double *f0, int M_tot, int r_max, double *F)
{
    const size_t n = size_t(r_max) * M_tot;
    for (size_t q = size_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
         q += size_t(gridDim.x) * blockDim.x)
        F[q] = f0[q % M_tot];
}

// ... then F[r][g1_l] = u_sweep[r][l].
__global__ void fill_g1_kernel(const double *u_sweep, int M_1, int r_max, const int *g1_idx,
                               int M_tot, double *F)
{
    const size_t n = size_t(r_max) * M_1;
    for (size_t q = size_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
         q += size_t(gridDim.x) * blockDim.x) {
        const size_t r = q / M_1, l = q - r * M_1;
        F[r * M_tot + g1_idx[l]] = u_sweep[q];
    }
}

// uD_sweep[r][i] = (C F_r)[i] / N, one warp per (i, r).
__global__ void udsweep_kernel(const uint32_t *counts, int M_D, int M_tot, double invN,
                               const double *F, int r_max, double *uD_sweep)
{
    const int lane = threadIdx.x & 31;
    const size_t gw = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const size_t nw = (size_t(gridDim.x) * blockDim.x) >> 5;
    const size_t n = size_t(M_D) * r_max;
    for (size_t q = gw; q < n; q += nw) {
        const size_t r = q / M_D, i = q - r * M_D;
        const uint32_t *row = counts + i * M_tot;
        const double *f = F + r * M_tot;
        double s = 0.0;
        for (int j = lane; j < M_tot; j += 32)
            s = fma(double(row[j]), f[j], s);
        s = warp_sum(s);
        if (lane == 0)
            uD_sweep[q] = 0.0 + 1.0 * s * invN;
    }
}

}  // namespace

extern "C" wos_status wos_spectral(wos_context *ctx, const double *U, const double *S,
                                   const double *V, int32_t M_D, int32_t k,
                                   const uint32_t *counts, int32_t M_tot, uint32_t N,
                                   const uint8_t *gamma1, const double *nu,
                                   const double *sigma, const double *uD, const double *u0,
                                   int32_t r_max, double *lambda, double *eigfun,
                                   double *density, double *u_sweep, double *uD_sweep,
                                   void *stream)
{
    if (!ctx || !U || !S || !V || !counts || !gamma1 || !sigma || M_D < 1 || M_tot < 1 ||
        N < 1 || k < 1 || r_max < 0 || r_max > k)
        return WOS_INVALID_ARG;
    if ((u_sweep || uD_sweep) && (r_max < 1 || !uD || !u_sweep))
        return WOS_INVALID_ARG;  // the fitted data need the solutions
    std::vector<int> g1, g0;
    for (int j = 0; j < M_tot; ++j)
        (gamma1[j] ? g1 : g0).push_back(j);
    const int M_1 = int(g1.size()), M_0 = int(g0.size());
    if (M_1 < 1 || k > std::min(M_D, M_1))
        return WOS_INVALID_ARG;
    cudaSetDevice(wos::ctx_device(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = wos::ctx_sm_count(ctx);
    const double invN = 1.0 / double(N);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_g1 = 0, o_g0 = o_g1 + al(size_t(M_1) * 4), o_f = o_g0 + al(size_t(M_0) * 4 + 4);
    const size_t o_b = o_f + al(size_t(M_tot) * 8), o_t = o_b + al(size_t(M_D) * 8);
    const size_t o_F = o_t + al(size_t(std::max(r_max, 1)) * 8);
    const size_t bytes = o_F + (uD_sweep ? size_t(r_max) * M_tot * 8 : 0);
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), bytes, st);
    if (e != cudaSuccess)
        return wos::cuda_status(e);
    int *d_g1 = reinterpret_cast<int *>(base + o_g1);
    int *d_g0 = reinterpret_cast<int *>(base + o_g0);
    double *f = reinterpret_cast<double *>(base + o_f);
    double *b = reinterpret_cast<double *>(base + o_b);
    double *t = reinterpret_cast<double *>(base + o_t);
    double *F = reinterpret_cast<double *>(base + o_F);
    cudaMemcpyAsync(d_g1, g1.data(), size_t(M_1) * 4, cudaMemcpyHostToDevice, st);
    if (M_0)
        cudaMemcpyAsync(d_g0, g0.data(), size_t(M_0) * 4, cudaMemcpyHostToDevice, st);
    int launches = 0;
    if (lambda) {
        lambda_kernel<<<std::max(1, (k + 255) / 256), 256, 0, st>>>(S, k, lambda);
        ++launches;
    }
    if (eigfun) {
        eigfun_kernel<<<dim3((k + 127) / 128, M_1), 128, 0, st>>>(
            U, S, M_D, k, counts, M_tot, invN, d_g1, nu, sigma, eigfun);
        ++launches;
    }
    if (density) {
        density_kernel<<<sms, 256, 0, st>>>(counts, M_D, M_tot, invN, d_g1, M_1, sigma,
                                            density);
        ++launches;
    }
    if (u_sweep) {
        // b = uD - A_0 u0 (f holds u0 on Gamma_0, zero elsewhere)
        cudaMemsetAsync(f, 0, size_t(M_tot) * 8, st);
        if (u0 && M_0) {
            scatter_kernel<<<sms, 256, 0, st>>>(d_g0, M_0, u0, f);
            ++launches;
        }
        counts_matvec_kernel<<<sms * 2, 256, 0, st>>>(counts, M_D, M_tot, invN, f, uD, -1.0,
                                                      b);
        coef_kernel<<<std::max(1, (r_max + 7) / 8), 256, 0, st>>>(U, S, M_D, k, r_max, nu, b,
                                                                   t);
        usweep_kernel<<<std::max(1, (M_1 + 255) / 256), 256, 0, st>>>(V, M_1, k, r_max, t,
                                                                      d_g1, sigma, u_sweep);
        launches += 3;
        if (uD_sweep) {
            fill_f_kernel<<<sms * 4, 256, 0, st>>>(f, M_tot, r_max, F);
            fill_g1_kernel<<<sms * 4, 256, 0, st>>>(u_sweep, M_1, r_max, d_g1, M_tot, F);
            udsweep_kernel<<<sms * 8, 256, 0, st>>>(counts, M_D, M_tot, invN, F, r_max,
                                                    uD_sweep);
            launches += 3;
        }
    }
    wos::count_launches(ctx, launches);
    e = cudaGetLastError();
    cudaFreeAsync(base, st);
    return wos::cuda_status(e);
}
