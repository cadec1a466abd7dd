// Plane kernels of the pair convolutions: the forward xy pass, the z pass
// and the inverse xy pass (templated on the real type T and the grid size N).
//
// Field layout: a real-space field is N^3 complex values indexed [z][y][x]
// (x fastest). A reciprocal-space field produced by the forward kernels is
// the same array with each axis in the digit-reversed order of its radix plan.
#pragma once
#include "fft.cuh"

namespace tddft {

// Affine description of a batch of pair convolutions. Item i = t * kdim + k
// (t = target slot, k = source slot) convolves conj(Q) * R and, in the
// accumulate mode, adds scale * P * Conv[conj(Q) R] to output field o.
struct PairMap {
  int kdim;
  int q0, qk, qt;
  int r0, rk, rt;
  int p0, pk, pt;
  int o0, ot;
  // optional explicit (q, r) field indices per item for the forward pass (pair lists)
  const int2* list = nullptr;
  // INV_WRITE of the register-line kernels: when > 0, the output is point-tiled: field f
  // at point r goes to ((r / POINT_TILE) * tile_nf + f) * POINT_TILE + r % POINT_TILE
  // (tile_nf fields in the buffer), so that the values of every field at POINT_TILE
  // consecutive points are one contiguous run per tile
  long long tile_nf = 0;
};
constexpr int POINT_TILE = 8;

// A copy of p that the compiler cannot relate to p: walking it again for the stores of a
// column keeps one address live instead of one per element (runtime column strides).
template <typename T>
__device__ __forceinline__ T* opaque_ptr(T* p) {
  asm volatile("" : "+l"(p));
  return p;
}

template <typename T>
__device__ __forceinline__ const cplx<T>* plane_ptr(const cplx<T>* base, long long field, int z, long long n3, int n2) {
  return base + field * n3 + (long long)z * n2;
}

// Compact intermediate of pair densities (ccols != nullptr): a pair density
// ρ = conj(q) r of two fields band-limited to |G| < G_max is band-limited to
// 2 G_max, so after the xy transform only the nact columns (x, y) inside that
// disk can be non-zero, for every z. Plane z of an item then holds just those
// columns, densely: element c of the plane is column ccols[c] (= y * N + x in
// the digit-reversed positions), at item base + z * nact + c. The other columns
// are zero and are neither stored, transformed along z nor read back.
// Plane z of an item (full or compact) into the shared-memory plane s (row pitch PITCH).
// Compact: ccols lists all N^2 positions, the nact stored columns first, so every
// position of the plane is written once (data or zero).
template <typename T, int N, int NT, int PITCH>
__device__ __forceinline__ void stage_in_plane(cplx<T>* s, const cplx<T>* item, int z, const int* __restrict__ ccols,
                                               int nact, int tid) {
  constexpr int N2 = N * N;
  if (ccols) {
    const cplx<T>* I = item + (long long)z * nact;
#pragma unroll 4
    for (int c = tid; c < N2; c += NT) {
      const int q = ccols[c], y = q / N;
      s[y * PITCH + q - y * N] = c < nact ? I[c] : cplx<T>{T(0), T(0)};
    }
  } else {
    const cplx<T>* I = item + (long long)z * N2;
#pragma unroll 4
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      s[y * PITCH + x] = I[e];
    }
  }
}

// ---------------------------------------------------------------------------
// Forward xy pass. MODE_PRODUCT: plane = conj(Q) * R; MODE_LOAD: plane = R.
// Grid (N, items). Output item i goes to ibuf field i (digit-reversed in x, y;
// compact when ccols is given).
// ---------------------------------------------------------------------------
constexpr int XY_LOAD = 0;
constexpr int XY_PRODUCT = 1;

// element i (= y) of column `line` of the plane conj(Q) * R (or R) in global memory
template <typename T, int N, bool PRODUCT>
struct PairLd {
  const cplx<T>* Q;
  const cplx<T>* R;
  int line;
  __device__ __forceinline__ cplx<T> operator()(int i) const {
    const int e = i * N + line;
    if constexpr (PRODUCT) return cmulc(Q[e], R[e]);
    else return R[e];
  }
};

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(plane_threads<N>())
    k_xy_fwd(const cplx<T>* __restrict__ qb, const cplx<T>* __restrict__ rb, PairMap pm,
             cplx<T>* __restrict__ ibuf, const cplx<T>* __restrict__ twg, const int* __restrict__ ccols, int nact) {
  constexpr int NT = plane_threads<N>(), PITCH = plane_pitch<N>(), N2 = N * N;
  constexpr long long N3 = (long long)N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* s = tw + tw_table_len<N>();
  const int tid = threadIdx.x, z = blockIdx.x, item = blockIdx.y;
  const int t = item / pm.kdim, k = item - t * pm.kdim;
  for (int i = tid; i < tw_table_len<N>(); i += NT) tw[i] = twg[i];
  long long qi = pm.q0 + (long long)k * pm.qk + (long long)t * pm.qt;
  long long ri = pm.r0 + (long long)k * pm.rk + (long long)t * pm.rt;
  if (pm.list) {
    const int2 pr = pm.list[item];
    qi = pr.x;
    ri = pr.y;
  }
  const cplx<T>* R = plane_ptr(rb, ri, z, N3, N2);
  const cplx<T>* Q = MODE == XY_PRODUCT ? plane_ptr(qb, qi, z, N3, N2) : nullptr;
  __syncthreads();  // twiddle tables
  // columns first, their first stage straight from global memory (consecutive threads take
  // consecutive x), then the rows
  const int line = tid % N, g = tid / N;
  fft_lines_from<T, N, FWD, false>(s, tw, line, g, PairLd<T, N, MODE == XY_PRODUCT>{Q, R, line});
  fft_lines<T, N, FWD, true>(s, tw, line, g);
  if (ccols) {
    cplx<T>* O = ibuf + (long long)item * N3 + (long long)z * nact;
#pragma unroll 4
    for (int c = tid; c < nact; c += NT) {
      const int q = ccols[c], y = q / N;
      O[c] = s[y * PITCH + q - y * N];
    }
  } else {
    cplx<T>* O = ibuf + (long long)item * N3 + (long long)z * N2;
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      O[e] = s[y * PITCH + x];
    }
  }
}

// ---------------------------------------------------------------------------
// z pass over the xz-plane at fixed y of every item.
// Z_CONV: forward z, multiply by kernel * kscale, inverse z.  Z_FWD / Z_INV: one direction.
// kernel is real, [N^3] in digit-reversed (position) order.
// ---------------------------------------------------------------------------
constexpr int Z_CONV = 0;
constexpr int Z_FWD = 1;
constexpr int Z_INV = 2;

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(plane_threads<N>())
    k_z(cplx<T>* __restrict__ ibuf, const T* __restrict__ kern, T kscale, const cplx<T>* __restrict__ twg) {
  constexpr int NT = plane_threads<N>(), PITCH = plane_pitch<N>(), N2 = N * N;
  constexpr long long N3 = (long long)N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* s = tw + tw_table_len<N>();
  const int tid = threadIdx.x, y = blockIdx.x, item = blockIdx.y;
  for (int i = tid; i < tw_table_len<N>(); i += NT) tw[i] = twg[i];
  cplx<T>* B = ibuf + (long long)item * N3 + (long long)y * N;
  for (int e = tid; e < N2; e += NT) {
    const int z = e / N, x = e - z * N;
    s[z * PITCH + x] = B[(long long)z * N2 + x];
  }
  __syncthreads();
  const int line = tid % N, g = tid / N;
  if constexpr (MODE != Z_INV) fft_lines<T, N, FWD, false>(s, tw, line, g);
  if constexpr (MODE == Z_CONV) {
    const T* K = kern + (long long)y * N;
    for (int e = tid; e < N2; e += NT) {
      const int z = e / N, x = e - z * N;
      s[z * PITCH + x] = cscale(s[z * PITCH + x], K[(long long)z * N2 + x] * kscale);
    }
    __syncthreads();
  }
  if constexpr (MODE != Z_FWD) fft_lines<T, N, INV, false>(s, tw, line, g);
  for (int e = tid; e < N2; e += NT) {
    const int z = e / N, x = e - z * N;
    B[(long long)z * N2 + x] = s[z * PITCH + x];
  }
}

// Register-resident z pass: one thread per (x, y) column holds the whole
// column of N values, so the transform needs neither shared memory nor a
// barrier; loads and stores of a warp cover 32 consecutive columns of one
// z-plane (coalesced). Used where the column fits the register file.
template <typename T, int N>
__host__ __device__ constexpr bool z_in_registers() {
  return sizeof(T) == 4 && N >= 8 && N <= 80;
}
constexpr int ZREG_THREADS = 128;

// COMPACT: compact items (see stage_in_plane): thread i < nact takes compact
// column i, and kern is the compact kernel table [z][nact].
template <typename T, int N, int MODE, bool COMPACT = false>
__global__ void __launch_bounds__(ZREG_THREADS)
    k_z_reg(cplx<T>* __restrict__ ibuf, const T* __restrict__ kern, T kscale, int nact) {
  constexpr int N2 = N * N;
  constexpr long long N3 = (long long)N * N * N;
  const int i = blockIdx.x * ZREG_THREADS + threadIdx.x;
  const int stride = COMPACT ? nact : N2;
  if (i >= stride) return;
  cplx<T>* B = ibuf + (long long)blockIdx.y * N3 + i;
  cplx<T> v[N];
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = B[(long long)z * stride];
  TwConst<T, N> tw;
  if constexpr (MODE != Z_INV) fft_reg<T, N, FWD>(v, tw);
  if constexpr (MODE == Z_CONV) {
    const T* K = kern + i;
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = cscale(v[z], K[(long long)z * stride] * kscale);
  }
  if constexpr (MODE != Z_FWD) fft_reg<T, N, INV>(v, tw);
#pragma unroll
  for (int z = 0; z < N; ++z) B[(long long)z * stride] = v[z];
}

// Register-resident z pass of compact pair densities with two threads per
// column (half the registers of k_z_reg, so more warps per SM hide the memory
// latency). Lanes 2c and 2c + 1 hold the points n and n + N/2 of column c; the
// first radix-2 decimation-in-frequency butterfly is exchanged with __shfl_xor,
// then each lane transforms its N/2 points in registers: lane h ends with the
// frequencies 2 k' + h in the digit-reversed order of the N/2 plan, which is the
// order of the kernel table kern2 [(h N/2 + j)][nact]. The inverse runs the same
// steps backwards (decimation-in-time butterfly, conjugate twiddles).
// (also at N = 96, where a whole column does not fit one thread's registers but a half does)
template <typename T, int N>
__host__ __device__ constexpr bool z_pair_ok() {
  return (z_in_registers<T, N>() || (sizeof(T) == 4 && N == 96)) && N % 2 == 0 && tw_offset(N / 2) >= 0;
}

template <typename T>
__device__ __forceinline__ cplx<T> shfl_xor_c(cplx<T> v, int mask) {
  return {__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask)};
}

template <typename T, int N>
__global__ void __launch_bounds__(ZREG_THREADS)
    k_z_pair(cplx<T>* __restrict__ ibuf, const T* __restrict__ kern2, T kscale, int nact) {
  constexpr int H = N / 2;
  constexpr long long N3 = (long long)N * N * N;
  const int gt = blockIdx.x * ZREG_THREADS + threadIdx.x;
  const int h = gt & 1;
  int c = gt >> 1;
  const bool valid = c < nact;
  if (!valid) c = nact - 1;  // both lanes of every pair take part in the exchanges; no store
  cplx<T>* B = ibuf + (long long)blockIdx.y * N3 + c + (long long)h * H * nact;
  cplx<T> v[H];
  {
    const cplx<T>* p = B;
#pragma unroll
    for (int n = 0; n < H; ++n, p += nact) v[n] = *p;
  }
  TwConst<T, N> twn;
#pragma unroll
  for (int n = 0; n < H; ++n) {  // lane 0: x_n + x_(n+H); lane 1: (x_n - x_(n+H)) W_N^n
    const cplx<T> p = shfl_xor_c(v[n], 1);
    v[n] = h ? cmul(csub(p, v[n]), twn(n)) : cadd(v[n], p);
  }
  // scalar halves (no packed pairs): packed operands need aligned register pairs, which
  // would cost this memory-bound kernel a third of its resident warps
  TwConst<T, H> twh;
  fft_reg<T, H, FWD, TwConst<T, H>, 0, false>(v, twh);
  const T* K = opaque_ptr(kern2 + c + (long long)h * H * nact);
#pragma unroll
  for (int j = 0; j < H; ++j, K += nact) v[j] = cscale(v[j], *K * kscale);
  fft_reg<T, H, INV, TwConst<T, H>, 0, false>(v, twh);
#pragma unroll
  for (int n = 0; n < H; ++n) {  // lane 0: A_n + conj(W_N^n) B_n; lane 1: A_n - conj(W_N^n) B_n
    const cplx<T> p = shfl_xor_c(v[n], 1);
    const cplx<T> w = twn(n);
    v[n] = h ? csub(p, cmulc(w, v[n])) : cadd(v[n], cmulc(w, p));
  }
  if (valid) {
    cplx<T>* q = opaque_ptr(B);
#pragma unroll
    for (int n = 0; n < H; ++n, q += nact) *q = v[n];
  }
}

// ---------------------------------------------------------------------------
// Inverse xy pass.
// INV_WRITE: out field (o0 + t*ot) plane z = scale * IFFT_xy(ibuf item t).
// INV_ACCUM: out field (o0 + t*ot) plane z += scale * sum_k P_(t,k) * IFFT_xy(ibuf item t*kdim+k).
//            Grid (N, targets); each CTA loops over the sources of its target.
// INV_ATOMIC: the same sum with one CTA per item (grid (N, targets*kdim)),
//            added to the output with atomics (summation order not fixed). In INV_WRITE mode ob may be ibuf itself (in place: each
// CTA reads its whole plane before it writes it back), unless the items are compact (ccols).
// ---------------------------------------------------------------------------
constexpr int INV_WRITE = 0;
constexpr int INV_ACCUM = 1;
constexpr int INV_ATOMIC = 2;  // one CTA per pair item, atomic accumulation into the target

template <typename T>
__device__ __forceinline__ void atomic_cadd(cplx<T>* p, cplx<T> v);
template <>
__device__ __forceinline__ void atomic_cadd<float>(cplx<float>* p, cplx<float> v) {
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}
template <>
__device__ __forceinline__ void atomic_cadd<double>(cplx<double>* p, cplx<double> v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// Last stage of the inverse (columns, element i = y of column `line`) into global memory.
template <typename T, int N>
struct AtomicSt {  // O += scale * P * v with atomics
  const cplx<T>* P;
  cplx<T>* O;
  T scale;
  int line;
  __device__ __forceinline__ void operator()(int i, cplx<T> v) const {
    const int e = i * N + line;
    atomic_cadd(O + e, cscale(cmul(P[e], v), scale));
  }
};
template <typename T, int N>
struct WriteSt {  // O = scale * v
  cplx<T>* O;
  T scale;
  int line;
  __device__ __forceinline__ void operator()(int i, cplx<T> v) const { O[i * N + line] = cscale(v, scale); }
};

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(plane_threads<N>())
    k_xy_inv(const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* __restrict__ pb, PairMap pm,
             T scale, const cplx<T>* __restrict__ twg, const int* __restrict__ ccols, int nact) {
  constexpr int NT = plane_threads<N>(), PITCH = plane_pitch<N>(), N2 = N * N;
  constexpr int EPT = (N2 + NT - 1) / NT;
  constexpr long long N3 = (long long)N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* s = tw + tw_table_len<N>();
  const int tid = threadIdx.x, z = blockIdx.x, t = blockIdx.y;
  for (int i = tid; i < tw_table_len<N>(); i += NT) tw[i] = twg[i];
  const int line = tid % N, g = tid / N;
  cplx<T>* O = ob + (long long)(pm.o0 + (long long)t * pm.ot) * N3 + (long long)z * N2;
  // rows first, then the columns, whose last stage writes to global memory directly
  // (consecutive threads take consecutive x); every read of the input plane comes
  // before the first barrier, so INV_WRITE may overwrite its own input (full planes)
  if constexpr (MODE == INV_WRITE) {
    stage_in_plane<T, N, NT, PITCH>(s, ibuf + (long long)t * N3, z, ccols, nact, tid);
    __syncthreads();
    fft_lines<T, N, INV, true>(s, tw, line, g);
    fft_lines_to<T, N, INV, false>(s, tw, line, g, WriteSt<T, N>{O, scale, line});
  } else if constexpr (MODE == INV_ATOMIC) {
    const int item = t;
    const int tt = item / pm.kdim, k = item - tt * pm.kdim;
    stage_in_plane<T, N, NT, PITCH>(s, ibuf + (long long)item * N3, z, ccols, nact, tid);
    __syncthreads();
    const cplx<T>* P = plane_ptr(pb, pm.p0 + (long long)k * pm.pk + (long long)tt * pm.pt, z, N3, N2);
    cplx<T>* Oa = ob + (long long)(pm.o0 + (long long)tt * pm.ot) * N3 + (long long)z * N2;
    fft_lines<T, N, INV, true>(s, tw, line, g);
    fft_lines_to<T, N, INV, false>(s, tw, line, g, AtomicSt<T, N>{P, Oa, scale, line});
  } else {
    cplx<T> acc[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) acc[i] = {T(0), T(0)};
    for (int k = 0; k < pm.kdim; ++k) {
      const long long item = (long long)t * pm.kdim + k;
      stage_in_plane<T, N, NT, PITCH>(s, ibuf + item * N3, z, ccols, nact, tid);
      __syncthreads();
      fft_lines<T, N, INV, false>(s, tw, line, g);
      fft_lines<T, N, INV, true>(s, tw, line, g);
      const cplx<T>* P = plane_ptr(pb, pm.p0 + (long long)k * pm.pk + (long long)t * pm.pt, z, N3, N2);
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + i * NT;
        if (e < N2) {
          const int y = e / N, x = e - y * N;
          acc[i] = cadd(acc[i], cmul(P[e], s[y * PITCH + x]));
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * NT;
      if (e < N2) O[e] = cadd(O[e], cscale(acc[i], scale));
    }
  }
}

}  // namespace tddft
