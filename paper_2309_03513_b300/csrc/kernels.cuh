// CUDA kernels of the Liouville-operator path (templated on the real type T
// and, for the plane kernels, on the grid size N).
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
};

template <typename T>
__device__ __forceinline__ const cplx<T>* plane_ptr(const cplx<T>* base, long long field, int z, long long n3, int n2) {
  return base + field * n3 + (long long)z * n2;
}

// ---------------------------------------------------------------------------
// Forward xy pass. MODE_PRODUCT: plane = conj(Q) * R; MODE_LOAD: plane = R.
// Grid (N, items). Output item i goes to ibuf field i (digit-reversed in x, y).
// ---------------------------------------------------------------------------
constexpr int XY_LOAD = 0;
constexpr int XY_PRODUCT = 1;

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(plane_threads<N>())
    k_xy_fwd(const cplx<T>* __restrict__ qb, const cplx<T>* __restrict__ rb, PairMap pm,
             cplx<T>* __restrict__ ibuf, const cplx<T>* __restrict__ twg) {
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
  if constexpr (MODE == XY_PRODUCT) {
    const cplx<T>* Q = plane_ptr(qb, qi, z, N3, N2);
#pragma unroll 4
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      s[y * PITCH + x] = cmulc(Q[e], R[e]);
    }
  } else {
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      s[y * PITCH + x] = R[e];
    }
  }
  __syncthreads();
  const int line = tid % N, g = tid / N;
  fft_lines<T, N, FWD, true>(s, tw, line, g);
  fft_lines<T, N, FWD, false>(s, tw, line, g);
  cplx<T>* O = ibuf + (long long)item * N3 + (long long)z * N2;
  for (int e = tid; e < N2; e += NT) {
    const int y = e / N, x = e - y * N;
    O[e] = s[y * PITCH + x];
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

// cols (optional): the N^2 column positions with the nact columns that can be
// non-zero first (ascending), then the others (ascending). Threads of the
// first kind transform their column; threads of the second kind only write
// zeros, which is what the transform of an all-zero column gives exactly.
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(ZREG_THREADS)
    k_z_reg(cplx<T>* __restrict__ ibuf, const T* __restrict__ kern, T kscale, const int* __restrict__ cols,
            int nact) {
  constexpr int N2 = N * N;
  constexpr long long N3 = (long long)N * N * N;
  const int i = blockIdx.x * ZREG_THREADS + threadIdx.x;
  if (i >= N2) return;
  const int c = cols ? cols[i] : i;
  cplx<T>* B = ibuf + (long long)blockIdx.y * N3 + c;
  if (cols && i >= nact) {
#pragma unroll 8
    for (int z = 0; z < N; ++z) B[(long long)z * N2] = cplx<T>{T(0), T(0)};
    return;
  }
  cplx<T> v[N];
#pragma unroll
  for (int z = 0; z < N; ++z) v[z] = B[(long long)z * N2];
  TwConst<T, N> tw;
  if constexpr (MODE != Z_INV) fft_reg<T, N, FWD>(v, tw);
  if constexpr (MODE == Z_CONV) {
    const T* K = kern + c;
#pragma unroll
    for (int z = 0; z < N; ++z) v[z] = cscale(v[z], K[(long long)z * N2] * kscale);
  }
  if constexpr (MODE != Z_FWD) fft_reg<T, N, INV>(v, tw);
#pragma unroll
  for (int z = 0; z < N; ++z) B[(long long)z * N2] = v[z];
}

// ---------------------------------------------------------------------------
// Inverse xy pass.
// INV_WRITE: out field (o0 + t*ot) plane z = scale * IFFT_xy(ibuf item t).
// INV_ACCUM: out field (o0 + t*ot) plane z += scale * sum_k P_(t,k) * IFFT_xy(ibuf item t*kdim+k).
//            Grid (N, targets); each CTA loops over the sources of its target.
// INV_ATOMIC: the same sum with one CTA per item (grid (N, targets*kdim)),
//            added to the output with atomics (summation order not fixed). In INV_WRITE mode ob may be ibuf itself (in place: each
// CTA reads its whole plane before it writes it back).
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

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(plane_threads<N>())
    k_xy_inv(const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* __restrict__ pb, PairMap pm,
             T scale, const cplx<T>* __restrict__ twg) {
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
  if constexpr (MODE == INV_WRITE) {
    const cplx<T>* I = ibuf + (long long)t * N3 + (long long)z * N2;
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      s[y * PITCH + x] = I[e];
    }
    __syncthreads();
    fft_lines<T, N, INV, false>(s, tw, line, g);
    fft_lines<T, N, INV, true>(s, tw, line, g);
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      O[e] = cscale(s[y * PITCH + x], scale);
    }
  } else if constexpr (MODE == INV_ATOMIC) {
    const int item = t;
    const int tt = item / pm.kdim, k = item - tt * pm.kdim;
    const cplx<T>* I = ibuf + (long long)item * N3 + (long long)z * N2;
#pragma unroll 4
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      s[y * PITCH + x] = I[e];
    }
    __syncthreads();
    fft_lines<T, N, INV, false>(s, tw, line, g);
    fft_lines<T, N, INV, true>(s, tw, line, g);
    const cplx<T>* P = plane_ptr(pb, pm.p0 + (long long)k * pm.pk + (long long)tt * pm.pt, z, N3, N2);
    cplx<T>* Oa = ob + (long long)(pm.o0 + (long long)tt * pm.ot) * N3 + (long long)z * N2;
#pragma unroll 4
    for (int e = tid; e < N2; e += NT) {
      const int y = e / N, x = e - y * N;
      atomic_cadd(Oa + e, cscale(cmul(P[e], s[y * PITCH + x]), scale));
    }
  } else {
    cplx<T> acc[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) acc[i] = {T(0), T(0)};
    for (int k = 0; k < pm.kdim; ++k) {
      const long long item = (long long)t * pm.kdim + k;
      const cplx<T>* I = ibuf + item * N3 + (long long)z * N2;
      for (int e = tid; e < N2; e += NT) {
        const int y = e / N, x = e - y * N;
        s[y * PITCH + x] = I[e];
      }
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

// ---------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------

// drho[b](r) = sum_v conj(phi_v(r)) a_{b,v}(r)
template <typename T>
__global__ void k_delta_rho(const cplx<T>* __restrict__ phi, const cplx<T>* __restrict__ a, cplx<T>* __restrict__ drho,
                            int nocc, int nb, long long n3) {
  const long long total = (long long)nb * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n3, r = i - b * n3;
    cplx<T> acc = {T(0), T(0)};
    const cplx<T>* ab = a + b * nocc * n3 + r;
    for (int v = 0; v < nocc; ++v) acc = cadd(acc, cmulc(phi[(long long)v * n3 + r], ab[(long long)v * n3]));
    drho[i] = acc;
  }
}

// out[b,v](r) = vloc(r) a_{b,v}(r) + phi_v(r) W_b(r), where
// W_b = [Conv_H drho_b] and/or its conjugate (hmode bits 1, 2: the K1e and K2e
// Hartree parts; Conv_H[conj drho] = conj Conv_H[drho] for the real, even
// kernel) + fxc (drho_b and/or conj drho_b) (xmode bits 1, 2).
// vloc == nullptr: no local term; hmode = xmode = 0: no phi_v W_b term.
template <typename T>
__global__ void k_init_out(const cplx<T>* __restrict__ a, const cplx<T>* __restrict__ phi, const T* __restrict__ vloc,
                           const cplx<T>* __restrict__ wconv, const T* __restrict__ fxc, const cplx<T>* __restrict__ drho,
                           cplx<T>* __restrict__ out, int nocc, int nb, long long n3, int hmode, int xmode) {
  const long long total = (long long)nb * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n3, r = i - b * n3;
    cplx<T> W = {T(0), T(0)};
    if (hmode) {
      const cplx<T> w = wconv[i];
      if (hmode & 1) W = cadd(W, w);
      if (hmode & 2) W = cadd(W, cplx<T>{w.x, -w.y});
    }
    if (xmode) {
      const cplx<T> d = drho[i];
      const T f = fxc[r];
      if (xmode & 1) W = cadd(W, cscale(d, f));
      if (xmode & 2) W = cadd(W, cscale(cplx<T>{d.x, -d.y}, f));
    }
    const bool k1e = (hmode | xmode) != 0;
    const T vl = vloc ? vloc[r] : T(0);
    for (int v = 0; v < nocc; ++v) {
      const long long o = (b * nocc + v) * n3 + r;
      cplx<T> val = {T(0), T(0)};
      if (vloc) val = cscale(a[o], vl);
      if (k1e) val = cadd(val, cmul(phi[(long long)v * n3 + r], W));
      out[o] = val;
    }
  }
}

// cube[f][pos[g]] = s * c[f][g]  (cube zeroed beforehand)
template <typename T>
__global__ void k_scatter(const cplx<T>* __restrict__ c, cplx<T>* __restrict__ cube, const int* __restrict__ pos, int npw,
                          int nf, T s, long long n3) {
  const long long total = (long long)nf * npw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npw, g = i - f * npw;
    cube[f * n3 + pos[g]] = cscale(c[i], s);
  }
}

// out[f][g] = s * cube[f][pos[g]] (+ (g2h[g] - eps[(f0+f) % nocc]) * A[f][g] when A != null)
template <typename T>
__global__ void k_gather(const cplx<T>* __restrict__ cube, const int* __restrict__ pos, int npw, int nf, T s,
                         const cplx<T>* __restrict__ A, const T* __restrict__ g2h, const T* __restrict__ eps, int nocc,
                         int f0, cplx<T>* __restrict__ out, long long n3) {
  const long long total = (long long)nf * npw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npw, g = i - f * npw;
    cplx<T> v = cscale(cube[f * n3 + pos[g]], s);
    if (A) v = cadd(v, cscale(A[i], eps ? g2h[g] - eps[(f0 + f) % nocc] : g2h[g]));
    out[i] = v;
  }
}

// K1d contraction for one block of pairs (v in I = [i0, i0+ti), v' in J = [j0, j0+tj)),
// tau[(vi*tj + vj)] = Conv_x[conj(phi_v') phi_v] in real space:
//   out[b, i0+vi] += s * sum_vj a[b, j0+vj] tau[vi][vj]
//   and, when I != J, out[b, j0+vj] += s * sum_vi a[b, i0+vi] conj(tau[vi][vj])
//   (tau_{v'v} = conj(tau_{vv'}) because the kernel is real and even).
// keep (optional, [nocc][nocc], symmetric): pairs with keep = 0 are truncated
// (their tau is taken as zero on both sides).
// A CTA of 256 threads takes PTS consecutive grid points: the tau values of
// those points are staged once in shared memory with coalesced loads, then
// thread (q, l) computes orbital q of each side for the points l + 16 j, for
// every trial vector b. Each (b, orbital, point) is written once.
constexpr int K1D_THREADS = 256;
template <typename T, int TB, int PTS>
__global__ void __launch_bounds__(K1D_THREADS)
    k_k1d_contract(const cplx<T>* __restrict__ tau, const cplx<T>* __restrict__ a, cplx<T>* __restrict__ out, int i0,
                   int ti, int j0, int tj, int nocc, int nb, T s, long long n3, const unsigned char* __restrict__ keep) {
  static_assert(K1D_THREADS == TB * 16 && PTS % 16 == 0, "thread layout");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* st = reinterpret_cast<cplx<T>*>(smem_raw);  // [TB*TB][PTS]
  const long long r0 = (long long)blockIdx.x * PTS;
  const int npts = (int)min((long long)PTS, n3 - r0);
  // the whole TB x TB tile is written (zeros outside ti x tj and past the last point)
  for (int e = threadIdx.x; e < TB * TB * PTS; e += K1D_THREADS) {
    const int slot = e / PTS, p = e - slot * PTS;
    const int vi = slot / TB, vj = slot - vi * TB;
    const bool kept = vi < ti && vj < tj && p < npts && (!keep || keep[(long long)(i0 + vi) * nocc + j0 + vj]);
    st[e] = kept ? tau[(long long)(vi * tj + vj) * n3 + r0 + p] : cplx<T>{T(0), T(0)};
  }
  __syncthreads();
  const int q = threadIdx.x / 16, l = threadIdx.x - q * 16;
  constexpr int PPT = PTS / 16;
  const bool offdiag = (i0 != j0);
  for (int side = 0; side < (offdiag ? 2 : 1); ++side) {
    const int nq = side == 0 ? ti : tj, nk = side == 0 ? tj : ti;
    if (q >= nq) continue;
    const int src0 = side == 0 ? j0 : i0, dst = (side == 0 ? i0 : j0) + q;
    for (int b = 0; b < nb; ++b) {
      const cplx<T>* ab = a + ((long long)b * nocc + src0) * n3 + r0;
      cplx<T>* ob = out + ((long long)b * nocc + dst) * n3 + r0;
      // issue every load of this (side, b) before using any of them
      cplx<T> av[PPT][TB], ov[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = l + 16 * j;
        const bool okp = p < npts;
        ov[j] = okp ? ob[p] : cplx<T>{T(0), T(0)};
#pragma unroll
        for (int k = 0; k < TB; ++k) av[j][k] = (okp && k < nk) ? ab[(long long)k * n3 + p] : cplx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = l + 16 * j;
        cplx<T> acc = {T(0), T(0)};
#pragma unroll
        for (int k = 0; k < TB; ++k) {
          const cplx<T> tv = side == 0 ? st[(q * TB + k) * PTS + p] : cconj(st[(k * TB + q) * PTS + p]);
          acc = cadd(acc, cmul(av[j][k], tv));
        }
        if (p < npts) ob[p] = cadd(ov[j], cscale(acc, s));
      }
    }
  }
}

// K1d contraction over a list of kept pairs (pair truncation, Sec. 3.2).
// tau[slot] (slot < np) holds Conv_x[conj(phi_n) phi_m] of the batch's pairs.
// Output rows: row i adds to orbital row_out[i], over its entries
// e in [row_ptr[i], row_ptr[i+1]): ent[e] = (n << 1 | c, slot):
//   out[b, row_out[i]] += s * sum_e a[b, n] * (c ? conj(tau[slot]) : tau[slot]).
// Rows are distinct orbitals, so each (b, orbital, point) is written by one
// thread. A CTA takes PTS points: the tau values of all np slots at those points
// are staged in shared memory once and reused for every b.
template <typename T, int PTS>
__global__ void __launch_bounds__(K1D_THREADS)
    k_k1d_sparse(const cplx<T>* __restrict__ tau, int np, const cplx<T>* __restrict__ a, cplx<T>* __restrict__ out,
                 const int* __restrict__ row_ptr, const int* __restrict__ row_out, int nrows,
                 const int2* __restrict__ ent, int nocc, int nb, T s, long long n3) {
  static_assert(PTS % 16 == 0, "thread layout");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* st = reinterpret_cast<cplx<T>*>(smem_raw);  // [np][PTS]
  const long long r0 = (long long)blockIdx.x * PTS;
  const int npts = (int)min((long long)PTS, n3 - r0);
  for (int e = threadIdx.x; e < np * PTS; e += K1D_THREADS) {
    const int slot = e / PTS, p = e - slot * PTS;
    st[e] = p < npts ? tau[(long long)slot * n3 + r0 + p] : cplx<T>{T(0), T(0)};
  }
  __syncthreads();
  const int q = threadIdx.x / 16, l = threadIdx.x - q * 16;
  constexpr int PPT = PTS / 16;
  for (int i = q; i < nrows; i += K1D_THREADS / 16) {
    const int e0 = row_ptr[i], e1 = row_ptr[i + 1], dst = row_out[i];
    for (int b = 0; b < nb; ++b) {
      const cplx<T>* ab = a + (long long)b * nocc * n3 + r0;
      cplx<T>* ob = out + ((long long)b * nocc + dst) * n3 + r0;
      cplx<T> acc[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) acc[j] = {T(0), T(0)};
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const int2 en = ent[e];
        const int n = en.x >> 1;
        const bool cj = en.x & 1;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const int p = l + 16 * j;
          if (p < npts) {
            const cplx<T> tv = st[en.y * PTS + p];
            acc[j] = cadd(acc[j], cmul(ab[(long long)n * n3 + p], cj ? cconj(tv) : tv));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = l + 16 * j;
        if (p < npts) ob[p] = cadd(ob[p], cscale(acc[j], s));
      }
    }
  }
}

}  // namespace tddft
