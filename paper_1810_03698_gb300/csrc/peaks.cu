// Arithmetic-pipe throughput of the device (measurement support, not a step of the
// method): the FP32 FMA, FP64 FMA and the special-function (MUFU) reciprocal square
// root and base-2 exponential rates that bound the treecode and direct pair
// kernels, which are ALU-bound elementwise arithmetic rather than contractions.
//
// Each kernel runs CH independent dependency chains per thread (enough to cover
// the pipe latency with a full SM) for `iters` steps, every step one instruction
// per chain, written as inline PTX so the compiler keeps every instruction.  The
// chains' final values are stored (conditionally on an impossible flag) so no
// chain is dead.  Grids are SMs x blocks-per-SM x 256 threads, timed with CUDA
// events after a warm-up launch; the best of `reps` launches is kept.
#include <cmath>
#include <string>

#include "internal.h"

namespace bp {
namespace {

constexpr int CH = 8;
constexpr int PK_TPB = 256;

__global__ void __launch_bounds__(PK_TPB) ffma_kernel(int iters, float seed, int flag, float* out) {
  float a[CH];
  const float b = 1.0f - 1e-7f * seed, c = 1e-7f;
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = seed + (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_TPB) dfma_kernel(int iters, double seed, int flag, double* out) {
  double a[CH];
  const double b = 1.0 - 1e-12 * seed, c = 1e-12;
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = seed + (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(b), "d"(c));
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// MUFU chains: x <- rsqrt(x) (fixed point 1) or x <- 2^(-x) (fixed point ~0.64); both
// stay finite and in range for any positive start.
template <int OP>
__global__ void __launch_bounds__(PK_TPB) mufu_kernel(int iters, float seed, int flag, float* out) {
  float a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = 0.5f + 1e-3f * (seed + (float)(threadIdx.x + k));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if (OP == 0)
        asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
      else
        asm volatile("{ .reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t; }" : "+f"(a[k]));
    }
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct Ev {
  cudaEvent_t a = nullptr, b = nullptr;
  Ev() {
    BP_CUDA(cudaEventCreate(&a));
    BP_CUDA(cudaEventCreate(&b));
  }
  ~Ev() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// best-of-reps time (ms) of `fn` launched on `s`, after one untimed launch
template <typename F>
double best_ms(F&& fn, int reps, cudaStream_t s) {
  Ev e;
  fn();
  BP_CHECK_LAUNCH();
  double best = 1e300;
  for (int r = 0; r < reps; ++r) {
    BP_CUDA(cudaEventRecord(e.a, s));
    fn();
    BP_CUDA(cudaEventRecord(e.b, s));
    BP_CUDA(cudaEventSynchronize(e.b));
    float ms = 0;
    BP_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
    best = std::min(best, (double)ms);
  }
  BP_CHECK_LAUNCH();
  return best;
}

}  // namespace
}  // namespace bp

extern "C" bempol_status bempol_measure_peaks(int device, int iters, int reps, bempol_peaks* out) {
  using namespace bp;
  if (!out || iters < 1 || reps < 1) return BEMPOL_ERR_ARG;
  try {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
      (void)cudaGetLastError();
      return BEMPOL_ERR_CUDA;
    }
    BP_CUDA(cudaSetDevice(device));
    const int sms = num_sms(device);
    int clk_khz = 0;
    BP_CUDA(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device));
    const int bps = 8;  // 8 blocks x 256 threads = 64 warps per SM
    const dim3 grid(sms * bps), block(PK_TPB);
    const double threads = (double)grid.x * PK_TPB;
    cudaStream_t s = nullptr;
    float* f = nullptr;   // never written (flag = 0)
    double* d = nullptr;
    const double ops = threads * (double)iters * CH;  // instructions of one launch
    const double t_ffma = best_ms([&] { ffma_kernel<<<grid, block, 0, s>>>(iters, 1.0f, 0, f); }, reps, s);
    const double t_dfma = best_ms([&] { dfma_kernel<<<grid, block, 0, s>>>(iters / 8 + 1, 1.0, 0, d); }, reps, s);
    const double ops_d = threads * (double)(iters / 8 + 1) * CH;
    const double t_rsq = best_ms([&] { mufu_kernel<0><<<grid, block, 0, s>>>(iters / 4 + 1, 1.0f, 0, f); }, reps, s);
    const double t_ex2 = best_ms([&] { mufu_kernel<1><<<grid, block, 0, s>>>(iters / 4 + 1, 1.0f, 0, f); }, reps, s);
    const double ops_m = threads * (double)(iters / 4 + 1) * CH;
    out->fp32_fma_tflops = 2.0 * ops / (t_ffma * 1e-3) / 1e12;
    out->fp64_fma_tflops = 2.0 * ops_d / (t_dfma * 1e-3) / 1e12;
    out->mufu_rsqrt_gops = ops_m / (t_rsq * 1e-3) / 1e9;
    out->mufu_ex2_gops = ops_m / (t_ex2 * 1e-3) / 1e9;
    out->ms_fp32 = t_ffma;
    out->ms_fp64 = t_dfma;
    out->ms_rsqrt = t_rsq;
    out->ms_ex2 = t_ex2;
    out->sm_count = sms;
    out->clock_mhz_attr = clk_khz / 1000.0;
    return BEMPOL_OK;
  } catch (const Error& e) {
    return e.st;
  }
}
