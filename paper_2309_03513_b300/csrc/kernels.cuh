// Pointwise and K1d-contraction kernels of the Liouville-operator path
// (templated on the real type T). Field layout as in plane_kernels.cuh.
#pragma once
#include "plane_kernels.cuh"

namespace tddft {

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
// A CTA takes PTS consecutive grid points: the tau values of those points are
// staged once in shared memory with coalesced loads. Thread (p, g) then works on
// point p for the trial vectors b = g, g + K1D_GROUPS, ...: it holds the TB
// output orbitals of a side in registers, reads each source value a[b, v'](p)
// once (consecutive points across a warp) and tau from shared memory (consecutive
// points, no bank conflicts), and writes each (b, orbital, point) once.
constexpr int K1D_THREADS = 256;
template <typename T, int TB, int PTS>
__global__ void __launch_bounds__(K1D_THREADS)
    k_k1d_contract(const cplx<T>* __restrict__ tau, const cplx<T>* __restrict__ a, cplx<T>* __restrict__ out, int i0,
                   int ti, int j0, int tj, int nocc, int nb, T s, long long n3, const unsigned char* __restrict__ keep) {
  static_assert(K1D_THREADS % PTS == 0, "thread layout");
  constexpr int GROUPS = K1D_THREADS / PTS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* st = reinterpret_cast<cplx<T>*>(smem_raw);  // [TB*TB][PTS]
  const long long r0 = (long long)blockIdx.x * PTS;
  const int npts = (int)min((long long)PTS, n3 - r0);
  // the whole TB x TB tile is written (zeros outside ti x tj, for truncated pairs and past the last point)
  for (int e = threadIdx.x; e < TB * TB * PTS; e += K1D_THREADS) {
    const int slot = e / PTS, p = e - slot * PTS;
    const int vi = slot / TB, vj = slot - vi * TB;
    const bool kept = vi < ti && vj < tj && p < npts && (!keep || keep[(long long)(i0 + vi) * nocc + j0 + vj]);
    st[e] = kept ? tau[(long long)(vi * tj + vj) * n3 + r0 + p] : cplx<T>{T(0), T(0)};
  }
  __syncthreads();
  const int p = threadIdx.x % PTS, g = threadIdx.x / PTS;
  if (p >= npts) return;
  const bool offdiag = (i0 != j0);
  for (int b = g; b < nb; b += GROUPS) {
    for (int side = 0; side < (offdiag ? 2 : 1); ++side) {
      const int nq = side == 0 ? ti : tj, nk = side == 0 ? tj : ti;
      const int src0 = side == 0 ? j0 : i0, dst0 = side == 0 ? i0 : j0;
      const cplx<T>* ab = a + ((long long)b * nocc + src0) * n3 + r0 + p;
      cplx<T>* ob = out + ((long long)b * nocc + dst0) * n3 + r0 + p;
      cplx<T> acc[TB];
#pragma unroll
      for (int q = 0; q < TB; ++q) acc[q] = {T(0), T(0)};
      // sources four at a time: their loads are in flight together
#pragma unroll 1
      for (int k0 = 0; k0 < nk; k0 += 4) {
        cplx<T> a4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a4[j] = k0 + j < nk ? ab[(long long)(k0 + j) * n3] : cplx<T>{T(0), T(0)};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + j;
          if (k >= TB) break;
#pragma unroll
          for (int q = 0; q < TB; ++q) {
            const cplx<T> tv = side == 0 ? st[(q * TB + k) * PTS + p] : cconj(st[(k * TB + q) * PTS + p]);
            acc[q] = cadd(acc[q], cmul(a4[j], tv));
          }
        }
      }
#pragma unroll
      for (int q = 0; q < TB; ++q)
        if (q < nq) ob[(long long)q * n3] = cadd(ob[(long long)q * n3], cscale(acc[q], s));
    }
  }
}

// K1d contraction over a list of kept pairs (pair truncation, Sec. 3.2).
// tau[slot] (slot < np) holds Conv_x[conj(phi_n) phi_m] of the batch's pairs.
// Output rows: row i adds to orbital row_out[i], over its entries
// e in [row_ptr[i], row_ptr[i+1]): ent[e] = (n << 1 | c, slot):
//   out[b, row_out[i]] += s * sum_e a[b, n] * (c ? conj(tau[slot]) : tau[slot]).
// A CTA takes PTS points: the tau values of all np slots at those points are
// staged in shared memory once. Thread (p, g) then works on point p for the
// trial vectors b = g, g + K1D_THREADS / PTS, ..., row after row, so each
// (b, orbital, point) is written by one thread and each source value is read once
// per row entry (consecutive points across a warp).
template <typename T, int PTS>
__global__ void __launch_bounds__(K1D_THREADS)
    k_k1d_sparse(const cplx<T>* __restrict__ tau, int np, const cplx<T>* __restrict__ a, cplx<T>* __restrict__ out,
                 const int* __restrict__ row_ptr, const int* __restrict__ row_out, int nrows,
                 const int2* __restrict__ ent, int nocc, int nb, T s, long long n3) {
  static_assert(K1D_THREADS % PTS == 0, "thread layout");
  constexpr int GROUPS = K1D_THREADS / PTS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* st = reinterpret_cast<cplx<T>*>(smem_raw);  // [np][PTS]
  const long long r0 = (long long)blockIdx.x * PTS;
  const int npts = (int)min((long long)PTS, n3 - r0);
  for (int e = threadIdx.x; e < np * PTS; e += K1D_THREADS) {
    const int slot = e / PTS, p = e - slot * PTS;
    st[e] = p < npts ? tau[(long long)slot * n3 + r0 + p] : cplx<T>{T(0), T(0)};
  }
  __syncthreads();
  const int p = threadIdx.x % PTS, g = threadIdx.x / PTS;
  if (p >= npts) return;
  for (int b = g; b < nb; b += GROUPS) {
    const cplx<T>* ab = a + (long long)b * nocc * n3 + r0 + p;
    cplx<T>* ob = out + (long long)b * nocc * n3 + r0 + p;
#pragma unroll 1
    for (int i = 0; i < nrows; ++i) {
      const int e0 = row_ptr[i], e1 = row_ptr[i + 1], dst = row_out[i];
      cplx<T> acc = {T(0), T(0)};
#pragma unroll 1
      for (int e = e0; e < e1; e += 4) {
        cplx<T> av[4], tv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (e + j < e1) {
            const int2 en = ent[e + j];
            av[j] = ab[(long long)(en.x >> 1) * n3];
            const cplx<T> t = st[en.y * PTS + p];
            tv[j] = (en.x & 1) ? cconj(t) : t;
          } else {
            av[j] = {T(0), T(0)};
            tv[j] = {T(0), T(0)};
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc = cadd(acc, cmul(av[j], tv[j]));
      }
      ob[(long long)dst * n3] = cadd(ob[(long long)dst * n3], cscale(acc, s));
    }
  }
}

}  // namespace tddft
