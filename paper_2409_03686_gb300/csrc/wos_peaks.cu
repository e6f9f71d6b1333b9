// wos_peaks.cu -- measured throughput of the execution pipes the kernels of
// this library lean on (the denominators of their rooflines are the
// recipe's unit counts; these measurements check them on the GPU at hand).
//
// Every kernel runs SMs x 8 CTAs of 256 threads; each thread advances eight
// independent dependency chains of one PTX operation (so latency hides
// behind the other chains and warps) and stores them at the end (so nothing
// is dead code).  The operations are written in inline PTX so that the
// measured instruction is the one named:
//   FFMA   fma.rn.f32                        (the move, the direction map)
//   MUFU   sin.approx.f32 + cos.approx.f32   (the 2-D direction)
//   IMADW  mul.wide.u32 + the xor of its halves (a Philox half-round)
//   LOP3   lop3.b32                          (the Philox xors, masks)
//   DFMA   fma.rn.f64                        (the SVD)
//   ISSUE  fma.rn.f32 and lop3.b32 alternately (two pipes: the issue limit)
#include <cuda_runtime.h>

#include <cstdint>

#include "wos.h"
#include "wos_internal.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 8;
constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(kPeakThreads)
pipe_kernel(int iters, uint32_t seed, float *fout, uint32_t *uout, double *dout)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t s = seed ^ uint32_t(gid);
    if (OP == WOS_PIPE_FFMA || OP == WOS_PIPE_MUFU) {
        float x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j)
            x[j] = float(s & 0xffu) * 1e-3f + float(j);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) {
                if (OP == WOS_PIPE_FFMA) {
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[j]) : "f"(0.999f), "f"(1e-3f));
                } else {
                    float sn, cs;
                    asm volatile("sin.approx.f32 %0, %1;" : "=f"(sn) : "f"(x[j]));
                    asm volatile("cos.approx.f32 %0, %1;" : "=f"(cs) : "f"(x[j]));
                    x[j] = sn + cs;
                }
            }
        }
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < kChains; ++j)
            acc += x[j];
        fout[gid] = acc;
    } else if (OP == WOS_PIPE_IMAD_WIDE || OP == WOS_PIPE_LOP3 || OP == WOS_PIPE_ISSUE) {
        uint32_t u[kChains];
        float f[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            u[j] = s * 0x9E3779B9u + uint32_t(j);
            f[j] = float(j);
        }
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) {
                if (OP == WOS_PIPE_IMAD_WIDE) {
                    uint64_t p;
                    asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(u[j]), "r"(0xD2511F53u));
                    u[j] = uint32_t(p >> 32) ^ uint32_t(p);
                } else if (OP == WOS_PIPE_LOP3) {
                    // u ^ k ^ (u >> 0 of another constant): a three-input xor
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[j]) : "r"(0x85EBCA6Bu), "r"(uint32_t(it)));
                } else {
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(0.999f), "f"(1e-3f));
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[j]) : "r"(0x85EBCA6Bu), "r"(uint32_t(it)));
                }
            }
        }
        uint32_t acc = 0u;
        float facc = 0.f;
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            acc ^= u[j];
            facc += f[j];
        }
        uout[gid] = acc;
        fout[gid] = facc;
    } else {
        double d[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j)
            d[j] = double(s & 0xffu) * 1e-3 + double(j);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < kChains; ++j)
                asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[j]) : "d"(0.999), "d"(1e-3));
        }
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < kChains; ++j)
            acc += d[j];
        dout[gid] = acc;
    }
}

template <int OP>
cudaError_t time_pipe(int grid, int iters, float *fo, uint32_t *uo, double *dop, cudaStream_t st,
                      cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    pipe_kernel<OP><<<grid, kPeakThreads, 0, st>>>(iters / 8, 1u, fo, uo, dop);  // warm-up
    cudaEventRecord(e0, st);
    pipe_kernel<OP><<<grid, kPeakThreads, 0, st>>>(iters, 2u, fo, uo, dop);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess)
        return e;
    return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace

extern "C" wos_status wos_measure_pipes(wos_context *ctx, double *out, void *stream)
{
    if (!ctx || !out)
        return WOS_INVALID_ARG;
    cudaSetDevice(wos::ctx_device(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = wos::ctx_sm_count(ctx) * kPeakCtasPerSm;
    const size_t nthr = size_t(grid) * kPeakThreads;
    float *fo = nullptr;
    uint32_t *uo = nullptr;
    double *dop = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&fo), nthr * 4, st);
    if (e == cudaSuccess)
        e = cudaMallocAsync(reinterpret_cast<void **>(&uo), nthr * 4, st);
    if (e == cudaSuccess)
        e = cudaMallocAsync(reinterpret_cast<void **>(&dop), nthr * 8, st);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    // iterations per kernel: about a millisecond at the nominal rates
    const int it_f = 4096, it_m = 512, it_w = 2048, it_l = 4096, it_d = 64, it_i = 2048;
    float ms[WOS_PIPE_COUNT] = {0};
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_FFMA>(grid, it_f, fo, uo, dop, st, e0, e1, &ms[WOS_PIPE_FFMA]);
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_MUFU>(grid, it_m, fo, uo, dop, st, e0, e1, &ms[WOS_PIPE_MUFU]);
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_IMAD_WIDE>(grid, it_w, fo, uo, dop, st, e0, e1,
                                          &ms[WOS_PIPE_IMAD_WIDE]);
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_LOP3>(grid, it_l, fo, uo, dop, st, e0, e1, &ms[WOS_PIPE_LOP3]);
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_DFMA>(grid, it_d, fo, uo, dop, st, e0, e1, &ms[WOS_PIPE_DFMA]);
    if (e == cudaSuccess)
        e = time_pipe<WOS_PIPE_ISSUE>(grid, it_i, fo, uo, dop, st, e0, e1, &ms[WOS_PIPE_ISSUE]);
    wos::count_launches(ctx, 2 * WOS_PIPE_COUNT);
    if (e == cudaSuccess) {
        const double lanes = double(nthr) * kChains;
        const int iters[WOS_PIPE_COUNT] = {it_f, it_m, it_w, it_l, it_d, it_i};
        // operations per chain step: 1, except MUFU (sine and cosine) and
        // ISSUE (an FMA and a LOP3): 2 instructions each
        for (int q = 0; q < WOS_PIPE_COUNT; ++q) {
            const double per = (q == WOS_PIPE_MUFU || q == WOS_PIPE_ISSUE) ? 2.0 : 1.0;
            out[q] = ms[q] > 0.f ? lanes * iters[q] * per / (double(ms[q]) * 1e-3) : 0.0;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (fo) cudaFreeAsync(fo, st);
    if (uo) cudaFreeAsync(uo, st);
    if (dop) cudaFreeAsync(dop, st);
    return wos::cuda_status(e);
}
