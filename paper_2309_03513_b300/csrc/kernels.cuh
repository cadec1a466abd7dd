// Pointwise and K1d-contraction kernels of the Liouville-operator path
// (templated on the real type T). Field layout as in plane_kernels.cuh.
#pragma once
#include <cstdint>

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

// K1d from the tau of every unordered orbital pair at once (Eq. 6), FP32:
//   out[b][v] += s * sum_v' a[b][v'] tau_vv',   tau_v'v = conj(tau_vv').
// tau is point-tiled (PairMap::tile_nf): for the POINT_TILE points of tile t, the values
// of all nf pair fields follow each other, field f at (t * nf + f) * POINT_TILE. The
// fields are ordered block pair after block pair (16 x 16 orbital blocks I <= J, field
// vi * tj + vj of block pair (I, J) at K1dAll::off[I][J]; diagonal blocks hold both
// orders), so the tau of one block pair at one tile is one contiguous run, which a
// bulk copy (cp.async.bulk, completion on an mbarrier) brings into shared memory.
// A CTA takes one tile and every output row (nocc <= 128): thread (row quad, point) holds
// rows v, v + 4, v + 8, v + 12 of one block at one point and keeps the sums of NB trial
// vectors for the four in registers, so that each trial-vector value read from shared
// memory serves four rows and each tau value NB vectors; the four row quads of a block and
// the eight points of the tile make one warp (one block per warp). The trial vectors of the
// tile are staged once per group of NB. The
// off-diagonal block pairs are visited in rounds of disjoint pairs (the round-robin
// pairing of the blocks, K1dAll::pi/pj): in a round every block meets one partner and
// the rows of both blocks read the round's tiles (the I rows as tau, the J rows
// conjugated and transposed), so each tau value leaves global memory once. The copies
// of round r + 1 are in flight while round r is computed (two buffers); the diagonal
// blocks come last, into both buffers once the last round is done. Every wait on an mbarrier is bounded: on
// timeout the CTA sets *err, waits (bounded) for the copies it issued and returns.
constexpr int K1D_ALL_THREADS = 256;
constexpr int K1D_ALL_PTS = POINT_TILE;
constexpr int K1D_ALL_BLOCKS = 8;  // orbital blocks (nocc <= 128)
constexpr int K1D_ALL_ROWS = 16 * K1D_ALL_BLOCKS;
constexpr int K1D_ALL_SLOT = 256 * K1D_ALL_PTS;   // elements of one block-pair tile
constexpr long long K1D_ALL_WAIT_LIMIT = 1LL << 22;
struct K1dAll {
  long long off[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS];  // field offset of block pair (I <= J)
  // per round and block: partner block (-1: none), slot of the pair in the round, 1 if the block is I
  signed char partner[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS];
  signed char slot[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS];
  signed char first[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS];
  signed char pi[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS / 2];  // (I, J) of slot k in round r, -1 unused
  signed char pj[K1D_ALL_BLOCKS][K1D_ALL_BLOCKS / 2];
  int rounds, nblk;
  long long nf;  // fields per tile
};

// acc += x * t as four fused multiply-adds (the product is not rounded before the sum)
__device__ __forceinline__ void k1d_cmac(cplx<float>& acc, float xr, float xi, float tr, float ti) {
  acc.x = fmaf(xr, tr, acc.x);
  acc.x = fmaf(-xi, ti, acc.x);
  acc.y = fmaf(xr, ti, acc.y);
  acc.y = fmaf(xi, tr, acc.y);
}
// acc[h][q] += a_q * t[h] for the four rows of a thread; av: trial vector 0 of the partner row
template <int NB>
__device__ __forceinline__ void k1d_all_mac(cplx<float> (&acc)[4][NB], const cplx<float>* av, const cplx<float> (&t)[4]) {
  constexpr int QS = K1D_ALL_ROWS * K1D_ALL_PTS;  // stride of one trial vector in the staged block
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const cplx<float> x = av[q * QS];
#pragma unroll
    for (int h = 0; h < 4; ++h) k1d_cmac(acc[h][q], x.x, x.y, t[h].x, t[h].y);
  }
}
__device__ __forceinline__ cplx<float> k1d_ld(const cplx<float>* p, bool ok) {
  return ok ? *p : cplx<float>{0.f, 0.f};
}

__device__ __forceinline__ uint32_t k1d_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// bounded wait for phase `parity` of the mbarrier at bar; false on timeout
__device__ __forceinline__ bool k1d_bar_wait(uint32_t bar, uint32_t parity) {
  for (long long polls = 0; polls < K1D_ALL_WAIT_LIMIT; ++polls) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
  }
  return false;
}
// one bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared
// memory, counted on the mbarrier at bar
__device__ __forceinline__ void k1d_bulk_copy(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   k1d_smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int NB>
__global__ void __launch_bounds__(K1D_ALL_THREADS, 1)
    k_k1d_all(const cplx<float>* __restrict__ tau, K1dAll kt, const cplx<float>* __restrict__ a,
              cplx<float>* __restrict__ out, int nocc, int nb, float s, long long n3, int* __restrict__ err) {
  using T = float;
  constexpr int PTS = K1D_ALL_PTS;
  constexpr int QS = K1D_ALL_ROWS * PTS;
  constexpr int NBUF = K1D_ALL_BLOCKS / 2 * K1D_ALL_SLOT;  // elements of one round buffer
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);  // two mbarriers
  cplx<T>* as = reinterpret_cast<cplx<T>*>(smem_raw + 128);  // [NB][K1D_ALL_ROWS][PTS]
  cplx<T>* ts = as + NB * QS;                                 // two round buffers, [slot][field][PTS]
  const int tid = threadIdx.x;
  const int p = tid % PTS, rq = tid / PTS;  // point p; rq: row quad 0..31
  const int B = rq / 4, vb = rq % 4;        // rows 16 B + vb + 4 h, h < 4
  const int v0 = 16 * B + vb;
  const long long tile = blockIdx.x, r0 = tile * PTS;
  const cplx<T>* tt = tau + tile * kt.nf * PTS;  // this tile's fields
  auto bsize = [nocc](int blk) { return min(16, nocc - 16 * blk); };
  const bool live = B < kt.nblk;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(k1d_smem_u32(bars)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(k1d_smem_u32(bars + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // copies of stage g (round r of a group, or the diagonal blocks) go to buffer g & 1
  uint32_t issued = 0, waited = 0;  // stages issued / completed
  auto issue = [&](int r) {        // thread 0: round r's tiles, or the diagonal tiles for r < 0
    cplx<T>* buf = ts + (issued & 1) * NBUF;
    uint32_t bytes = 0;
    const uint32_t bar = k1d_smem_u32(bars + (issued & 1));
    if (r >= 0) {
      for (int k = 0; k < K1D_ALL_BLOCKS / 2; ++k)
        if (kt.pi[r][k] >= 0) bytes += (uint32_t)(bsize(kt.pi[r][k]) * bsize(kt.pj[r][k]) * PTS * sizeof(cplx<T>));
    } else {
      for (int blk = 0; blk < kt.nblk; ++blk) bytes += (uint32_t)(bsize(blk) * bsize(blk) * PTS * sizeof(cplx<T>));
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    if (r >= 0) {
      for (int k = 0; k < K1D_ALL_BLOCKS / 2; ++k) {
        const int I = kt.pi[r][k], J = kt.pj[r][k];
        if (I < 0) continue;
        k1d_bulk_copy(buf + k * K1D_ALL_SLOT, tt + kt.off[I][J] * PTS,
                      (uint32_t)(bsize(I) * bsize(J) * PTS * sizeof(cplx<T>)), bar);
      }
    } else {
      for (int blk = 0; blk < kt.nblk; ++blk)  // diagonal block blk at slot blk of the two buffers
        k1d_bulk_copy(ts + blk * K1D_ALL_SLOT, tt + kt.off[blk][blk] * PTS,
                      (uint32_t)(bsize(blk) * bsize(blk) * PTS * sizeof(cplx<T>)), bar);
    }
  };
  bool ok = true;
  for (int b0 = 0; b0 < nb && ok; b0 += NB) {
    const int nbc = min(NB, nb - b0);
    __syncthreads();  // the previous group's reads of the staged values and buffers are done
    if (tid == 0) {
      if (kt.rounds > 0) issue(0);
      else issue(-1);
      ++issued;
    }
    for (int e = 2 * tid; e < NB * QS; e += 2 * K1D_ALL_THREADS) {  // two points per 16-byte copy
      const int pp = e % PTS, rest = e / PTS, vv = rest % K1D_ALL_ROWS, bb = rest / K1D_ALL_ROWS;
      *reinterpret_cast<float4*>(as + e) =
          (bb < nbc && vv < nocc) ? *reinterpret_cast<const float4*>(a + ((long long)(b0 + bb) * nocc + vv) * n3 + r0 + pp)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cplx<T> acc[4][NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) acc[0][q] = acc[1][q] = acc[2][q] = acc[3][q] = {T(0), T(0)};
    for (int r = 0; r <= kt.rounds && ok; ++r) {  // r == rounds: the diagonal blocks
      __syncthreads();  // staged trial vectors visible; the buffer of stage `issued` is free
      if (tid == 0) {
        if (r + 1 < kt.rounds) {  // the next round's copies, in flight during this one
          issue(r + 1);
          ++issued;
        } else if (r == kt.rounds && kt.rounds > 0) {  // the diagonal blocks fill both buffers: after the last round
          issue(-1);
          ++issued;
        }
      }
      const int stage_buf = waited & 1;
      if (!k1d_bar_wait(k1d_smem_u32(bars + stage_buf), (waited >> 1) & 1)) ok = false;
      ++waited;
      if (__syncthreads_or(ok ? 0 : 1)) {
        ok = false;
        break;
      }
      const cplx<T>* buf = ts + stage_buf * NBUF;
      if (r < kt.rounds) {
        const int partner = live ? kt.partner[r][B] : -1;
        if (partner >= 0) {
          const cplx<T>* tile_s = buf + kt.slot[r][B] * K1D_ALL_SLOT;
          const cplx<T>* av = as + partner * 16 * PTS + p;
          const int np = bsize(partner), nself = bsize(B);
          if (kt.first[r][B]) {  // rows of I: tau_(v, J*16 + vj), field vi * tj + vj
#pragma unroll 4
            for (int vj = 0; vj < np; ++vj) {
              cplx<T> t[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) t[h] = k1d_ld(tile_s + ((vb + 4 * h) * np + vj) * PTS + p, vb + 4 * h < nself);
              k1d_all_mac<NB>(acc, av + vj * PTS, t);
            }
          } else {  // rows of J: tau_(v, I*16 + vi) = conj(tau_(I*16 + vi, v)), field vi * tj + vj
#pragma unroll 4
            for (int vi = 0; vi < np; ++vi) {
              cplx<T> t[4];
#pragma unroll
              for (int h = 0; h < 4; ++h)
                t[h] = cconj(k1d_ld(tile_s + (vi * nself + vb + 4 * h) * PTS + p, vb + 4 * h < nself));
              k1d_all_mac<NB>(acc, av + vi * PTS, t);
            }
          }
        }
      } else if (live) {  // diagonal block B at slot B of the buffers (which follow each other)
        const cplx<T>* tile_s = ts + B * K1D_ALL_SLOT;
        const int tb = bsize(B);
        const cplx<T>* av = as + B * 16 * PTS + p;
#pragma unroll 4
        for (int vj = 0; vj < tb; ++vj) {
          cplx<T> t[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) t[h] = k1d_ld(tile_s + ((vb + 4 * h) * tb + vj) * PTS + p, vb + 4 * h < tb);
          k1d_all_mac<NB>(acc, av + vj * PTS, t);
        }
      }
    }
    if (!ok) break;
    if (live) {
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nbc) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int v = v0 + 4 * h;
            if (v < nocc)  // the only contribution to this value in this launch: one rounding, as a plain add
              atomicAdd(reinterpret_cast<float2*>(out + ((long long)(b0 + q) * nocc + v) * n3 + r0 + p),
                        make_float2(s * acc[h][q].x, s * acc[h][q].y));
          }
        }
    }
  }
  if (!ok) {
    // a wait ran out: report, and wait (bounded) for the copies this CTA still has in flight
    if (tid == 0) {
      atomicExch(err, 1);
      for (; waited < issued; ++waited) k1d_bar_wait(k1d_smem_u32(bars + (waited & 1)), (waited >> 1) & 1);
    }
    __syncthreads();
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
