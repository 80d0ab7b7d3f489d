// Throughput microbenchmarks of this GPU: the FP64 FMA rate and the tcgen05 MMA rate
// (kind::tf32 and kind::f16 with bf16), the denominators of the FP64 and tensor-core
// rooflines that the measured copy/GEMM peaks do not provide; and the diagnostic wait that
// runs out. Tools only; no assembly path calls them.
#include <cuda_runtime.h>
#include <cstdint>
#include "../../include/coffee.h"
#include "../../include/coffee_peaks.h"
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {
using namespace tc;

// 8 independent FMA chains per thread, 16 links per loop trip
__global__ void k_peak_fp64(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int PEAK_SMEM = 120 * 1024;  // one CTA (one MMA issuer, one TMEM owner) per SM

// One thread per CTA issues `iters` back-to-back M=128 x N x K=32-byte MMAs on fixed
// shared-memory operands into one TMEM accumulator, then waits for them (bounded).
template <bool TF32, int N>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, unsigned* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  uint8_t* sA = smem;               // 128 rows x 32 bytes
  uint8_t* sB = smem + 128 * 32;    // N rows x 32 bytes
  const uint32_t half = TF32 ? 0x3F000000u : 0x3F003F00u;  // 0.5 (tf32) or two bf16 0.5
  for (int i = threadIdx.x; i < (128 + N) * 32 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(smem)[i] = half;
  fence_proxy_async();
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)), "r"(N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  if (threadIdx.x == 0) {
    const uint32_t idesc = make_idesc(TF32 ? 2 : 1, 128, N);
    const uint64_t ad = make_desc(smem_u32(sA), 8u * 32u), bd = make_desc(smem_u32(sB), 8u * 32u);
    for (int i = 0; i < iters; ++i) mma<TF32>(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
    tc_commit(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 0, err);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N) : "memory");
  }
}

// One thread waits on an mbarrier that nothing arrives at, through the library's bounded wait:
// it gives up after the bound, sets the timeout bit of the error word and returns.
__global__ void k_diag_wait(unsigned* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err);
}

template <class L>
int time_launch(L launch, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return COFFEE_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return COFFEE_ERR_CUDA;
  }
  launch();  // warm-up
  cudaEventRecord(a);
  launch();
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e == cudaSuccess ? COFFEE_OK : fail(COFFEE_ERR_CUDA, cudaGetErrorString(e));
}

template <bool TF32, int N>
int run_mma(int sms, int iters, unsigned* err, float* ms) {
  cudaError_t e = cudaFuncSetAttribute(k_peak_mma<TF32, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_SMEM);
  if (e != cudaSuccess) return fail(COFFEE_ERR_CUDA, cudaGetErrorString(e));
  return time_launch([&] { k_peak_mma<TF32, N><<<sms, 128, PEAK_SMEM>>>(iters, err); }, ms);
}

}  // namespace

int launch_diag_wait(unsigned* err, void* stream) {
  k_diag_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err);
  return (int)cudaGetLastError();
}

}  // namespace coffee

using namespace coffee;

extern "C" int coffee_peak_fp64(double* tflops) {
  if (!tflops) return fail(COFFEE_ERR_INVALID_ARG, "tflops is NULL");
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0 /* current */) != cudaSuccess || sms <= 0)
    return fail(COFFEE_ERR_CUDA, "no CUDA device");
  const int blocks = sms * 8, threads = 256, iters = 250;  // ~16 ms at 1.25 TFLOP/s
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return fail(COFFEE_ERR_NOMEM, "cudaMalloc");
  float ms = 0.f;
  const int rc = time_launch([&] { k_peak_fp64<<<blocks, threads>>>(out, iters, 0.999, 1e-3); }, &ms);
  cudaFree(out);
  if (rc != COFFEE_OK) return rc;
  *tflops = 2.0 * 8 * 16 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return COFFEE_OK;
}

extern "C" int coffee_peak_mma(int precision, int n, double* tflops) {
  if (!tflops) return fail(COFFEE_ERR_INVALID_ARG, "tflops is NULL");
  if (!(precision == PREC_TF32 || precision == PREC_BF16)) return fail(COFFEE_ERR_INVALID_ARG, "precision: TF32 or BF16");
  if (!(n == 128 || n == 256)) return fail(COFFEE_ERR_INVALID_ARG, "n must be 128 or 256");
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0)
    return fail(COFFEE_ERR_CUDA, "no CUDA device");
  unsigned* err = nullptr;
  if (cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) return fail(COFFEE_ERR_NOMEM, "cudaMalloc");
  cudaMemset(err, 0, sizeof(unsigned));
  const int iters = 20000;
  float ms = 0.f;
  const bool tf32 = precision == PREC_TF32;
  int rc = tf32 ? (n == 256 ? run_mma<true, 256>(sms, iters, err, &ms) : run_mma<true, 128>(sms, iters, err, &ms))
                : (n == 256 ? run_mma<false, 256>(sms, iters, err, &ms) : run_mma<false, 128>(sms, iters, err, &ms));
  unsigned w = 0;
  cudaMemcpy(&w, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (rc != COFFEE_OK) return rc;
  if (w) return fail(COFFEE_ERR_TIMEOUT, "peak MMA loop: a wait gave up");
  const double k = tf32 ? 8.0 : 16.0;  // K elements per 32-byte operand row
  *tflops = 2.0 * 128.0 * n * k * (double)iters * sms / (ms * 1e-3) / 1e12;
  return COFFEE_OK;
}
