// Peak rates of the arithmetic pipes the M-RA kernels use, timed with CUDA
// events on this GPU: FP64 FMA (DFMA), FP64 mma.sync (DMMA, m8n8k4), and the
// two tcgen05 MMA shapes of the library's engines -- kind::f16 bf16
// 128 x 64 x 16 (the FP64-emulation engine) and kind::tf32 128 x 64 x 8 (the
// 3xTF32 engine) -- issued back to back by one thread per SM on staged
// shared-memory tiles into a tensor-memory accumulator.  Prints one JSON line.
#include <cstdio>
#include <cuda_runtime.h>
#include "mra_emu.cuh"

using namespace mra;

__global__ void dfma_kernel(double* out, int iters) {
  double a[8];
  for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  const double b = 0.999999, c = 1e-9;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  double s = 0;
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 12345.678) out[0] = s;   // keeps the loop alive
}

__global__ void dmma_kernel(double* out, int iters) {
  double acc[4][2] = {};
  const double a = 1.0 + 1e-6 * threadIdx.x, b = 0.5;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(acc[j][0]), "+d"(acc[j][1])
                   : "d"(a), "d"(b));
  double s = 0;
  for (int j = 0; j < 4; ++j) s += acc[j][0] + acc[j][1];
  if (s == 12345.678) out[0] = s;
}

template <bool BF16>
__global__ void __launch_bounds__(128) mma_kernel(int iters, int* fail) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  // zero the 32 KB the two tiles span (the tf32 descriptor strides 1 KB per 8-row group)
  for (int t = threadIdx.x; t < 32768 / 4; t += blockDim.x) reinterpret_cast<uint32_t*>(dsm)[t] = 0u;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(64u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  if (threadIdx.x == 0) {
    const uint32_t a0 = smem_addr(dsm), b0 = smem_addr(dsm + 4096 * 2);
    const uint64_t da = BF16 ? em_desc(a0) : tc_desc(a0), db = BF16 ? em_desc(b0) : tc_desc(b0);
    for (int it = 0; it < iters && ok; it += 64) {
      for (int j = 0; j < 64; ++j) {
        if (BF16) em_issue(tmem, da, db, (it + j) ? 1u : 0u);
        else tc_issue(tmem, da, db, (it + j) ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar)));
      ok = tc_wait_phase(&mbar, phase);
    }
    if (!ok) atomicExch(fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u));
}

template <typename F>
static float time_ms(F launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  double* out;
  int* fail;
  cudaMalloc(&out, 8);
  cudaMalloc(&fail, 4);
  cudaMemset(fail, 0, 4);
  const int it_f = 1 << 16, it_d = 1 << 14, it_m = 1 << 15;
  const dim3 gf(sms * 8), bf(256);
  const float ms_f = time_ms([&] { dfma_kernel<<<gf, bf>>>(out, it_f); });
  const float ms_d = time_ms([&] { dmma_kernel<<<gf, bf>>>(out, it_d); });
  const size_t smem = 120 * 1024;   // one CTA per SM
  cudaFuncSetAttribute(mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const float ms_b = time_ms([&] { mma_kernel<true><<<sms, 128, smem>>>(it_m, fail); });
  const float ms_t = time_ms([&] { mma_kernel<false><<<sms, 128, smem>>>(it_m, fail); });
  int hf = 0;
  cudaMemcpy(&hf, fail, 4, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  const double thr = (double)gf.x * bf.x;
  const double dfma = 2.0 * 8 * it_f * thr / (ms_f * 1e-3) / 1e12;
  const double dmma = 512.0 * 4 * it_d * (thr / 32) / (ms_d * 1e-3) / 1e12;
  const double bf16 = 2.0 * 128 * 64 * 16 * (double)it_m * sms / (ms_b * 1e-3) / 1e12;
  const double tf32 = 2.0 * 128 * 64 * 8 * (double)it_m * sms / (ms_t * 1e-3) / 1e12;
  printf("{\"sms\": %d, \"dfma_tflops\": %.4f, \"dmma_tflops\": %.4f, \"bf16_128x64x16_tflops\": %.2f, "
         "\"tf32_128x64x8_tflops\": %.2f, \"ms\": [%.3f, %.3f, %.3f, %.3f], \"timeout\": %d, \"cuda\": \"%s\"}\n",
         sms, dfma, dmma, bf16, tf32, ms_f, ms_d, ms_b, ms_t, hf, cudaGetErrorString(e));
  return e == cudaSuccess && !hf ? 0 : 1;
}
