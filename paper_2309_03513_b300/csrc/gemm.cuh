// Complex GEMMs of the occupied-subspace projector P^c = 1 - Phi Phi^dagger
// (plain SIMT path; used by the FP64 path, and by the FP32 path for the
// small orthogonality checks).
//
//   overlap:  C[m][n] = sum_g conj(Phi[m][g]) Y[n][g]      (Phi [M][K], Y [Nn][K])
//   update:   Y[n][g] += s * sum_m Phi[m][g] C[m][n]
#pragma once
#include "fft.cuh"

namespace tddft {

// Split-K overlap: block (bm, bn, split) writes Cp[split][m][n].
template <typename T>
__global__ void __launch_bounds__(256)
    k_overlap(const cplx<T>* __restrict__ phi, int M, const cplx<T>* __restrict__ Y, int Nn, int K, int kchunk,
              cplx<T>* __restrict__ Cp) {
  constexpr int BM = 32, BN = 32, BK = 16;
  __shared__ cplx<T> sa[BK][BM + 1];
  __shared__ cplx<T> sb[BK][BN + 1];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int tm = (tid / 16) * 2, tn = (tid % 16) * 2;
  cplx<T> acc[2][2] = {};
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int i = tid; i < BM * BK; i += 256) {
      const int r = i / BK, c = i - r * BK;
      const int m = m0 + r, k = k0 + c;
      sa[c][r] = (m < M && k < kend) ? phi[(long long)m * K + k] : cplx<T>{T(0), T(0)};
      const int n = n0 + r;
      sb[c][r] = (n < Nn && k < kend) ? Y[(long long)n * K + k] : cplx<T>{T(0), T(0)};
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < BK; ++c) {
      cplx<T> a0 = sa[c][tm], a1 = sa[c][tm + 1], b0 = sb[c][tn], b1 = sb[c][tn + 1];
      acc[0][0] = cadd(acc[0][0], cmulc(a0, b0));
      acc[0][1] = cadd(acc[0][1], cmulc(a0, b1));
      acc[1][0] = cadd(acc[1][0], cmulc(a1, b0));
      acc[1][1] = cadd(acc[1][1], cmulc(a1, b1));
    }
    __syncthreads();
  }
  cplx<T>* out = Cp + (long long)blockIdx.z * M * Nn;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + tm + i, n = n0 + tn + j;
      if (m < M && n < Nn) out[(long long)m * Nn + n] = acc[i][j];
    }
}

// C[i] = sum_s Cp[s][i]
template <typename T>
__global__ void k_reduce_split(const cplx<T>* __restrict__ Cp, int nsplit, long long len, cplx<T>* __restrict__ C) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    cplx<T> a = {T(0), T(0)};
    for (int s = 0; s < nsplit; ++s) a = cadd(a, Cp[(long long)s * len + i]);
    C[i] = a;
  }
}

// Y[n][g] += s * sum_m Phi[m][g] C[m][n]. Block tile 32 (n) x 64 (g).
template <typename T>
__global__ void __launch_bounds__(256)
    k_update(const cplx<T>* __restrict__ phi, int M, const cplx<T>* __restrict__ C, int Nn, int K, T s,
             cplx<T>* __restrict__ Y) {
  constexpr int BN = 32, BG = 64, BM = 16;
  __shared__ cplx<T> sc[BM][BN + 1];
  __shared__ cplx<T> sp[BM][BG + 1];
  const int tid = threadIdx.x;
  const int n0 = blockIdx.y * BN, g0 = blockIdx.x * BG;
  const int tn = (tid / 16) * 2, tg = tid % 16;
  cplx<T> acc[2][4] = {};
  for (int m0 = 0; m0 < M; m0 += BM) {
    for (int i = tid; i < BM * BN; i += 256) {
      const int r = i / BN, c = i - r * BN;
      const int m = m0 + r, n = n0 + c;
      sc[r][c] = (m < M && n < Nn) ? C[(long long)m * Nn + n] : cplx<T>{T(0), T(0)};
    }
    for (int i = tid; i < BM * BG; i += 256) {
      const int r = i / BG, c = i - r * BG;
      const int m = m0 + r, g = g0 + c;
      sp[r][c] = (m < M && g < K) ? phi[(long long)m * K + g] : cplx<T>{T(0), T(0)};
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < BM; ++r) {
      cplx<T> c0 = sc[r][tn], c1 = sc[r][tn + 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        cplx<T> p = sp[r][tg + 16 * j];
        acc[0][j] = cadd(acc[0][j], cmul(p, c0));
        acc[1][j] = cadd(acc[1][j], cmul(p, c1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn + i, g = g0 + tg + 16 * j;
      if (n < Nn && g < K) {
        cplx<T>* y = Y + (long long)n * K + g;
        *y = cadd(*y, cscale(acc[i][j], s));
      }
    }
}

}  // namespace tddft
