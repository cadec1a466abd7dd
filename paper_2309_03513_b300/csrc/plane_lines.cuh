// Register-line xy passes of compact pair densities (FP32, N = 32, 48, 64).
//
// Every line of an xy plane is held by two lanes of one warp: lane h of a line
// holds its points n + h N/2 (n < N/2). The first decimation-in-frequency
// butterfly (radix 2) pairs point n with point n + N/2 and is exchanged with
// __shfl_xor between the two lanes; the rest of the line transform (length N/2)
// runs in registers with constant-memory twiddles (fft_reg). The plane is
// transposed once through shared memory between the two axes, so a point makes
// one shared-memory round trip per xy pass (the staged kernels of
// plane_kernels.cuh make one per radix stage and axis).
//
// Lane h of a line ends the forward transform with the frequencies 2 k' + h,
// k' in the digit-reversed order of the N/2 plan; each value is stored at the
// position of its frequency in the digit-reversed order of the N plan, so the
// planes these kernels write and read are laid out exactly as those of the
// staged kernels (the z pass, the kernel tables and the sphere map are shared).
//
// Compact planes only: plane z of an item holds the nact columns of the 2 G_max
// disc (see stage_in_plane), addressed through cmapT[px * N + py] = compact
// index of position (px, py), or -1 outside the disc.
#pragma once
#include <type_traits>

#include "plane_kernels.cuh"

namespace tddft {

template <typename T, int N>
__host__ __device__ constexpr bool xy_lines_ok() {
  return sizeof(T) == 4 && (N == 32 || N == 48 || N == 64) && tw_offset(N / 2) >= 0;
}

// position of frequency k in the digit-reversed order of the N plan
template <int N>
__host__ __device__ constexpr int dif_pos(int k) {
  int pos = 0, len = N, kk = k;
  for (int s = 0; s < Plan<N>::S; ++s) {
    const int r = Plan<N>::r[s];
    const int m = len / r;
    pos += m * (kk % r);
    kk /= r;
    len = m;
  }
  return pos;
}
// the frequency at position p of that order
template <int N>
__host__ __device__ constexpr int dif_freq(int p) {
  for (int k = 0; k < N; ++k)
    if (dif_pos<N>(k) == p) return k;
  return -1;
}
// position (N plan) of the value in register j of lane h after a line transform
template <int N, int J>
struct LinePos {
  static constexpr int kp = dif_freq<N / 2>(J);
  static constexpr int p0 = dif_pos<N>(2 * kp);
  static constexpr int p1 = dif_pos<N>(2 * kp + 1);
};

template <int J, int END, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (J < END) {
    f(std::integral_constant<int, J>{});
    static_for<J + 1, END>(f);
  }
}

// forward line transform: natural points n + h N/2 in, frequencies 2 k' + h (k' in the
// digit-reversed order of the N/2 plan) out
template <typename T, int N>
__device__ __forceinline__ void line_fwd(cplx<T>* v, int h) {
  constexpr int H = N / 2;
  TwConst<T, N> twn;
#pragma unroll
  for (int n = 0; n < H; ++n) {  // lane 0: x_n + x_(n+H); lane 1: (x_n - x_(n+H)) W_N^n
    const cplx<T> p = shfl_xor_c(v[n], 16);
    v[n] = h ? cmul(csub(p, v[n]), twn(n)) : cadd(v[n], p);
  }
  fft_reg<T, H, FWD>(v, TwConst<T, H>{});
}

// inverse line transform (unnormalised): the layout of line_fwd's output in, natural
// points n + h N/2 out
template <typename T, int N>
__device__ __forceinline__ void line_inv(cplx<T>* v, int h) {
  constexpr int H = N / 2;
  fft_reg<T, H, INV>(v, TwConst<T, H>{});
  TwConst<T, N> twn;
#pragma unroll
  for (int n = 0; n < H; ++n) {  // lane 0: A_n + conj(W_N^n) B_n; lane 1: A_n - conj(W_N^n) B_n
    // lane 1 scales its own B_n first, so that one product per point suffices
    const cplx<T> x = h ? cmulc(twn(n), v[n]) : v[n];
    const cplx<T> p = shfl_xor_c(x, 16);
    v[n] = h ? csub(p, x) : cadd(x, p);
  }
}

// Lanes per line: 1 (a thread holds a whole line of N points, so the first radix stage
// needs no exchange: fewest instructions) or 2 (half the registers per thread).
template <int N, int L>
__host__ __device__ constexpr int lines_threads() {
  return L * N;
}

// position (N plan) of the value in register j of lane h after a forward line transform
template <int N, int L, int J>
__device__ __forceinline__ int line_pos(int h) {
  if constexpr (L == 1) return J;
  else return h ? LinePos<N, J>::p1 : LinePos<N, J>::p0;
}

template <typename T, int N, int L>
__device__ __forceinline__ void line_fwd_any(cplx<T>* v, int h) {
  if constexpr (L == 1) fft_reg<T, N, FWD>(v, TwConst<T, N>{});
  else line_fwd<T, N>(v, h);
}
template <typename T, int N, int L>
__device__ __forceinline__ void line_inv_any(cplx<T>* v, int h) {
  if constexpr (L == 1) fft_reg<T, N, INV>(v, TwConst<T, N>{});
  else line_inv<T, N>(v, h);
}

// Forward xy pass of compact pair densities. MODE_PRODUCT: plane = conj(Q) R;
// MODE_LOAD: plane = R. Grid (N, items). One lane per line: thread i holds line i;
// two lanes per line: lanes 0-15 of a warp hold the first halves of 16 lines, lanes
// 16-31 the second halves. Columns (y) first, read straight from global memory, then
// the rows (x); compact columns out.
template <typename T, int N, int MODE, int L>
__global__ void __launch_bounds__(lines_threads<N, L>())
    k_xy_fwd_lines(const cplx<T>* __restrict__ qb, const cplx<T>* __restrict__ rb, PairMap pm,
                   cplx<T>* __restrict__ ibuf, const int* __restrict__ cmapT, int nact) {
  constexpr int H = N / L, PITCH = N + 1, N2 = N * N;
  constexpr long long N3 = (long long)N * N2;
  __shared__ cplx<T> s[N * PITCH];
  const int tid = threadIdx.x, z = blockIdx.x, item = blockIdx.y;
  const int lane = tid & 31, h = L == 1 ? 0 : lane >> 4;
  const int line = L == 1 ? tid : (tid >> 5) * 16 + (lane & 15);
  const int t = item / pm.kdim, k = item - t * pm.kdim;
  long long qi = pm.q0 + (long long)k * pm.qk + (long long)t * pm.qt;
  long long ri = pm.r0 + (long long)k * pm.rk + (long long)t * pm.rt;
  if (pm.list) {
    const int2 pr = pm.list[item];
    qi = pr.x;
    ri = pr.y;
  }
  cplx<T> v[H];
  {
    const cplx<T>* R = plane_ptr(rb, ri, z, N3, N2) + h * H * N + line;
    if constexpr (MODE == XY_PRODUCT) {
      const cplx<T>* Q = plane_ptr(qb, qi, z, N3, N2) + h * H * N + line;
#pragma unroll
      for (int n = 0; n < H; ++n) v[n] = cmulc(Q[n * N], R[n * N]);
    } else {
#pragma unroll
      for (int n = 0; n < H; ++n) v[n] = R[n * N];
    }
  }
  // pass 0: column `line` along y, then the transpose; pass 1: the row at y position `line`
  // along x. One copy of the line-transform code serves both (a smaller instruction footprint:
  // the warps of an SM are at different points of the kernel)
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    line_fwd_any<T, N, L>(v, h);
    if (pass == 0) {
      static_for<0, H>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        s[line_pos<N, L, j>(h) * PITCH + line] = v[j];
      });
      __syncthreads();
#pragma unroll
      for (int n = 0; n < H; ++n) v[n] = s[line * PITCH + n + h * H];
    }
  }
  cplx<T>* O = ibuf + (long long)item * N3 + (long long)z * nact;
  static_for<0, H>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    const int c = __ldg(cmapT + line_pos<N, L, j>(h) * N + line);
    if (c >= 0) O[c] = v[j];
  });
}

// Inverse xy pass of compact pair densities. INV_ATOMIC: one CTA per (plane, item),
// O_(t) += scale * P_(t,k) * IFFT_xy(item) with atomics; INV_WRITE: out field
// (o0 + t*ot) plane z = scale * IFFT_xy(item t). Rows (x) first from the compact
// columns, then the columns (y), whose results go to global memory directly.
template <typename T, int N, int MODE, int L>
__global__ void __launch_bounds__(lines_threads<N, L>(), L == 1 ? 6 : 1)
    k_xy_inv_lines(const cplx<T>* __restrict__ ibuf, cplx<T>* ob, const cplx<T>* __restrict__ pb, PairMap pm,
                   T scale, const int* __restrict__ cmapT, int nact) {
  constexpr int H = N / L, PITCH = N + 1, N2 = N * N;
  constexpr long long N3 = (long long)N * N2;
  __shared__ cplx<T> s[N * PITCH];
  const int tid = threadIdx.x, z = blockIdx.x, item = blockIdx.y;
  const int lane = tid & 31, h = L == 1 ? 0 : lane >> 4;
  const int line = L == 1 ? tid : (tid >> 5) * 16 + (lane & 15);
  cplx<T> v[H];
  {
    const cplx<T>* I = ibuf + (long long)item * N3 + (long long)z * nact;
    static_for<0, H>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      const int c = __ldg(cmapT + line_pos<N, L, j>(h) * N + line);
      v[j] = c >= 0 ? I[c] : cplx<T>{T(0), T(0)};
    });
  }
  // pass 0: the row at y position `line` along x, then the transpose; pass 1: column `line`
  // along y (points y = n + h H). One copy of the line-transform code serves both
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    line_inv_any<T, N, L>(v, h);
    if (pass == 0) {
#pragma unroll
      for (int n = 0; n < H; ++n) s[line * PITCH + n + h * H] = v[n];
      __syncthreads();
      static_for<0, H>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        v[j] = s[line_pos<N, L, j>(h) * PITCH + line];
      });
    }
  }
  if constexpr (MODE == INV_ATOMIC) {
    const int tt = item / pm.kdim, k = item - tt * pm.kdim;
    const cplx<T>* P = plane_ptr(pb, pm.p0 + (long long)k * pm.pk + (long long)tt * pm.pt, z, N3, N2) + h * H * N + line;
    cplx<T>* O = ob + (long long)(pm.o0 + (long long)tt * pm.ot) * N3 + (long long)z * N2 + h * H * N + line;
#pragma unroll
    for (int n = 0; n < H; ++n) atomic_cadd(O + n * N, cscale(cmul(P[n * N], v[n]), scale));
  } else if (pm.tile_nf) {
    const long long f = pm.o0 + (long long)item * pm.ot;
    const long long r = (long long)z * N2 + h * H * N + line;  // point of n = 0; N is a multiple of POINT_TILE
    cplx<T>* O = ob + ((r / POINT_TILE) * pm.tile_nf + f) * POINT_TILE + r % POINT_TILE;
#pragma unroll
    for (int n = 0; n < H; ++n) O[(long long)n * (N / POINT_TILE) * pm.tile_nf * POINT_TILE] = cscale(v[n], scale);
  } else {
    cplx<T>* O = ob + (long long)(pm.o0 + (long long)item * pm.ot) * N3 + (long long)z * N2 + h * H * N + line;
#pragma unroll
    for (int n = 0; n < H; ++n) O[n * N] = cscale(v[n], scale);
  }
}

}  // namespace tddft
