// Arithmetic peaks of the device, measured: FP32 FMA throughput of the CUDA
// cores and TF32 throughput of the tcgen05 tensor cores. They are the
// denominators of the ALU and tensor-core roofline fractions of the library's
// kernels (the plane kernels' FFT arithmetic, the projector GEMMs).
#include <cuda_runtime.h>

#include <string>

#include "tddft_testing.h"
#include "umma.cuh"

namespace tddft {

constexpr int PEAK_FMA_THREADS = 256;
constexpr int PEAK_FMA_CHAINS = 16;

// Independent FMA chains per thread (no memory traffic in the loop); the result
// is stored so that the chains are not removed.
__global__ void __launch_bounds__(PEAK_FMA_THREADS) k_peak_fma(float a, float b, int iters, float* __restrict__ out) {
  float x[PEAK_FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_FMA_CHAINS; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PEAK_FMA_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PEAK_FMA_CHAINS; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One CTA per SM: one thread issues back-to-back tcgen05.mma.kind::tf32 of shape
// M = 128, N = 256, K = 8 from a fixed pair of shared-memory tiles into one tensor-
// memory accumulator, committing every PEAK_MMA_BATCH MMAs to an mbarrier and keeping
// at most two batches in flight. Every wait is bounded (on timeout the CTA records
// an error and stops issuing).
constexpr int PEAK_MMA_N = 256;
constexpr int PEAK_MMA_BATCH = 64;
constexpr int PEAK_A_BYTES = 128 * 32 * 4;          // A: 128 rows x 32 k (TF32), canonical K-major
constexpr int PEAK_B_BYTES = PEAK_MMA_N * 32 * 4;   // B: 256 rows x 32 k
constexpr int PEAK_SMEM_USED = PEAK_A_BYTES + PEAK_B_BYTES + 64;
constexpr int PEAK_SMEM = 120 * 1024;  // more than half an SM's shared memory: one CTA per SM

__host__ __device__ constexpr uint32_t peak_idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PEAK_MMA_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ bool peak_wait(uint32_t bar, uint32_t phase) {
  for (long long polls = 0; polls < UMMA_WAIT_LIMIT; ++polls) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) k_peak_tf32(int batches, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char peak_smem[];
  unsigned char* a = peak_smem;
  unsigned char* b = a + PEAK_A_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b + PEAK_B_BYTES);  // two barriers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b + PEAK_B_BYTES + 32);
  const int tid = threadIdx.x, warp = tid >> 5;
  // operand tiles: small values, the same for every MMA
  for (int e = tid; e < (PEAK_A_BYTES + PEAK_B_BYTES) / 4; e += 128)
    reinterpret_cast<uint32_t*>(a)[e] = to_tf32(1.0f + (float)(e & 7) * 0.125f);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(PEAK_MMA_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    constexpr uint32_t idesc = peak_idesc_tf32();
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    for (int bt = 0; bt < batches && ok; ++bt) {
      const int slot = bt & 1;
      if (bt >= 2) {  // the batch that used this barrier two batches ago has finished
        ok = peak_wait(smem_u32(mbar + slot), phase[slot]);
        phase[slot] ^= 1u;
      }
      for (int i = 0; i < PEAK_MMA_BATCH; ++i) {
        const uint32_t koff = (uint32_t)(i & 3) * 256;  // 8 tf32 = 2 core matrices along K
        umma_tf32(tmem, umma_desc(smem_u32(a) + koff), umma_desc(smem_u32(b) + koff), idesc,
                  (bt > 0 || i > 0) ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(mbar + slot)));
    }
    // drain the (up to two) batches still in flight
    for (int bt = (batches > 2 ? batches - 2 : 0); bt < batches && ok; ++bt) {
      const int slot = bt & 1;
      ok = peak_wait(smem_u32(mbar + slot), phase[slot]);
      phase[slot] ^= 1u;
    }
    if (!ok) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(PEAK_MMA_N));
  }
}

}  // namespace tddft

using namespace tddft;

extern "C" tddft_status tddft_testing_peak(int which, double* tflops, double* ms) {
  if (!tflops || (which != 0 && which != 1)) return TDDFT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TDDFT_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TDDFT_ECUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TDDFT_ECUDA;
  double flops = 0.0;
  float best = 1e30f;
  tddft_status st = TDDFT_OK;
  void* buf = nullptr;
  if (which == 0) {
    const int blocks = sms * 8, iters = 1 << 14;
    if (cudaMalloc(&buf, (size_t)blocks * PEAK_FMA_THREADS * sizeof(float)) != cudaSuccess) st = TDDFT_ENOMEM;
    flops = 2.0 * PEAK_FMA_CHAINS * (double)iters * blocks * PEAK_FMA_THREADS;
    for (int rep = 0; rep < 4 && st == TDDFT_OK; ++rep) {  // first launch warms up
      cudaEventRecord(e0);
      k_peak_fma<<<blocks, PEAK_FMA_THREADS>>>(0.999f, 1e-4f, iters, (float*)buf);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = TDDFT_ECUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0 && t < best) best = t;
    }
  } else {
    const int batches = 2048;
    if (cudaMalloc(&buf, sizeof(int)) != cudaSuccess) st = TDDFT_ENOMEM;
    if (st == TDDFT_OK) cudaMemset(buf, 0, sizeof(int));
    if (st == TDDFT_OK &&
        cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_SMEM) != cudaSuccess)
      st = TDDFT_ECUDA;
    flops = 2.0 * 128.0 * PEAK_MMA_N * 8.0 * PEAK_MMA_BATCH * (double)batches * sms;
    for (int rep = 0; rep < 4 && st == TDDFT_OK; ++rep) {
      cudaEventRecord(e0);
      k_peak_tf32<<<sms, 128, PEAK_SMEM>>>(batches, (int*)buf);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = TDDFT_ECUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0 && t < best) best = t;
    }
    int flag = 0;
    if (st == TDDFT_OK && cudaMemcpy(&flag, buf, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = TDDFT_ECUDA;
    if (st == TDDFT_OK && flag) st = TDDFT_ETIMEOUT;
  }
  if (st == TDDFT_OK && cudaGetLastError() != cudaSuccess) st = TDDFT_ECUDA;
  if (buf) cudaFree(buf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TDDFT_OK) return st;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return TDDFT_OK;
}
