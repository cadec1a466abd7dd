// Tensor-core (tcgen05, Blackwell 5th generation) real GEMM D = A * B^T with
// split-precision TF32 products ("3xTF32": a_hi b_hi + a_hi b_lo + a_lo b_hi,
// FP32 accumulation in tensor memory). Used for the occupied-subspace
// projector; the complex GEMMs are written as real GEMMs by the loaders.
//
// One CTA of 128 threads computes a 128 x 128 tile of D for one split of K:
//   * every thread stages its share of the A and B chunks (128 x 32 values)
//     into shared memory in the canonical K-major layout without swizzle
//     (8-row x 16-byte core matrices; K-adjacent cores 128 B apart, 8-row
//     groups 1024 B apart), split into TF32 high and low parts;
//   * one thread issues the MMAs (K = 8 each) and commits them to an mbarrier;
//   * all threads wait on the mbarrier (bounded: on timeout an error flag is
//     set and the CTA stops issuing work), then read the accumulator from
//     tensor memory, one row per thread, and hand it to the epilogue.
#pragma once
#include <cstdint>

#include "fft.cuh"

namespace tddft {

constexpr int UMMA_M = 128, UMMA_N = 128, UMMA_KC = 32;     // tile rows, tile columns, K per chunk
constexpr int UMMA_TILE_BYTES = UMMA_M * UMMA_KC * 4;        // 16 KB per operand part
constexpr int UMMA_SMEM = 4 * UMMA_TILE_BYTES + 64;          // A hi/lo, B hi/lo, barrier, TMEM slot
constexpr long long UMMA_WAIT_LIMIT = 1LL << 22;             // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of element (row, k) of a 128 x 32 K-major tile in the canonical layout
__device__ __forceinline__ int umma_offset(int row, int k) {
  return ((row >> 3) * 8 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor (no swizzle): start, LBO = 128 B (K-adjacent
// core matrices), SBO = 1024 B (adjacent 8-row groups), descriptor version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;  // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128
__host__ __device__ constexpr uint32_t umma_idesc_tf32() {
  return (1u << 4)                       // D format F32
         | (2u << 7)                     // A format TF32
         | (2u << 10)                    // B format TF32
         | ((uint32_t)(UMMA_N >> 3) << 17)
         | ((uint32_t)(UMMA_M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Loader / epilogue interface:
//   float LA::operator()(int m, int k) const   (A element, 0 outside)
//   float LB::operator()(int n, int k) const   (B element, 0 outside)
//   void  EP::operator()(int m, int n, float v, int split) const
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(128)
    k_umma_gemm(LA la, LB lb, EP ep, int kchunks, int chunks_per_split, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char umma_smem[];
  unsigned char* a_hi = umma_smem;
  unsigned char* a_lo = a_hi + UMMA_TILE_BYTES;
  unsigned char* b_hi = a_lo + UMMA_TILE_BYTES;
  unsigned char* b_lo = b_hi + UMMA_TILE_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + UMMA_TILE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_lo + UMMA_TILE_BYTES + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * UMMA_M, n0 = blockIdx.x * UMMA_N, split = blockIdx.z;
  const int c0 = split * chunks_per_split, c1 = min(kchunks, c0 + chunks_per_split);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(UMMA_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  uint32_t phase = 0;
  bool ok = true;
  for (int c = c0; c < c1 && ok; ++c) {
    const int k0 = c * UMMA_KC;
    // stage the A and B chunks (128 rows x 32 k), k fastest across threads
    for (int e = tid; e < UMMA_M * UMMA_KC; e += 128) {
      const int row = e / UMMA_KC, k = e - row * UMMA_KC;
      const int off = umma_offset(row, k);
      const float av = la(m0 + row, k0 + k);
      const uint32_t ah = to_tf32(av);
      const uint32_t al = to_tf32(av - __uint_as_float(ah));
      *reinterpret_cast<uint32_t*>(a_hi + off) = ah;
      *reinterpret_cast<uint32_t*>(a_lo + off) = al;
      const float bv = lb(n0 + row, k0 + k);
      const uint32_t bh = to_tf32(bv);
      const uint32_t bl = to_tf32(bv - __uint_as_float(bh));
      *reinterpret_cast<uint32_t*>(b_hi + off) = bh;
      *reinterpret_cast<uint32_t*>(b_lo + off) = bl;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      constexpr uint32_t idesc = umma_idesc_tf32();
#pragma unroll
      for (int kk = 0; kk < UMMA_KC / 8; ++kk) {
        const uint32_t koff = kk * 256;  // 8 tf32 = 2 core matrices along K
        const uint64_t ah = umma_desc(smem_u32(a_hi) + koff), al = umma_desc(smem_u32(a_lo) + koff);
        const uint64_t bh = umma_desc(smem_u32(b_hi) + koff), bl = umma_desc(smem_u32(b_lo) + koff);
        const uint32_t acc0 = (c > c0 || kk > 0) ? 1u : 0u;
        umma_tf32(tmem, ah, bh, idesc, acc0);
        umma_tf32(tmem, ah, bl, idesc, 1u);
        umma_tf32(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(mbar)));
    }
    // wait for the MMAs of this chunk (they read the staged tiles)
    long long polls = 0;
    uint32_t done = 0;
    while (!done) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(phase));
      if (!done && ++polls > UMMA_WAIT_LIMIT) break;
    }
    // the decision to stop is taken by the whole CTA at once
    const int timed_out = __syncthreads_or(done ? 0 : 1);
    if (timed_out) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
  }

  if (ok && c1 > c0) {
    // accumulator row (m0 + tid) from tensor memory, 16 columns at a time
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int cb = 0; cb < UMMA_N; cb += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + lane_base + (uint32_t)cb));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) ep(m0 + tid, n0 + cb + j, __uint_as_float(r[j]), split);
    }
  } else if (c1 <= c0) {
#pragma unroll 1
    for (int j = 0; j < UMMA_N; ++j) ep(m0 + tid, n0 + j, 0.f, split);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UMMA_N));
  }
}

// ---------------------------------------------------------------------------
// Projector loaders. Complex values are split into real GEMMs:
// overlap  C[u][r] = sum_g conj(P[u][g]) Y[r][g]
//   A(u, k') = [Re P | Im P],  B(n', k') = n' <  R: [Re Y_n' | Im Y_n']
//                                         n' >= R: [Im Y | -Re Y] of row n' - R
//   D(u, n') = Re C[u][n'] (n' < R), Im C[u][n'-R] (n' >= R)
// update   Y[r][g] -= sum_u P[u][g] C[u][r]
//   A(r, u') = [Re C[:, r] | Im C[:, r]],  B(n', u') = n' <  G: [Re P[:, g] | -Im P[:, g]]
//                                                      n' >= G: [Im P[:, g] |  Re P[:, g]]
//   D(r, n') = Re (n' < G) or Im (n' >= G) of sum_u P[u][g] C[u][r]
// Kp, Up, Gp, Rp: padded extents (multiples of the tile); real and imaginary
// halves of a padded dimension never share a chunk or a tile.
// ---------------------------------------------------------------------------
struct OvA {
  const cplx<float>* p;
  int M, K, Kp;
  __device__ __forceinline__ float operator()(int m, int k) const {
    if (m >= M) return 0.f;
    if (k < Kp) return k < K ? p[(long long)m * K + k].x : 0.f;
    k -= Kp;
    return k < K ? p[(long long)m * K + k].y : 0.f;
  }
};
struct OvB {
  const cplx<float>* y;
  int R, Rp, K, Kp;
  __device__ __forceinline__ float operator()(int n, int k) const {
    const bool im = n >= Rp;
    const int r = im ? n - Rp : n;
    if (r >= R) return 0.f;
    const bool kim = k >= Kp;
    const int g = kim ? k - Kp : k;
    if (g >= K) return 0.f;
    const cplx<float> v = y[(long long)r * K + g];
    return !im ? (kim ? v.y : v.x) : (kim ? -v.x : v.y);
  }
};
struct OvEp {
  cplx<float>* part;  // [split][M][R]
  int M, R, Rp;
  __device__ __forceinline__ void operator()(int m, int n, float v, int split) const {
    const bool im = n >= Rp;
    const int r = im ? n - Rp : n;
    if (m >= M || r >= R) return;
    float* d = reinterpret_cast<float*>(part + ((long long)split * M + m) * R + r);
    d[im ? 1 : 0] = v;
  }
  // two-phase form of the packed path's epilogue: load the value a store needs (none here), then store
  __device__ __forceinline__ float load(int, int, int) const { return 0.f; }
  __device__ __forceinline__ void store(int m, int n, float, float v, int split) const { (*this)(m, n, v, split); }
};
struct UpA {
  const cplx<float>* c;  // [U][R]
  int U, Up, R;
  __device__ __forceinline__ float operator()(int r, int k) const {
    if (r >= R) return 0.f;
    const bool im = k >= Up;
    const int u = im ? k - Up : k;
    if (u >= U) return 0.f;
    const cplx<float> v = c[(long long)u * R + r];
    return im ? v.y : v.x;
  }
};
struct UpB {
  const cplx<float>* p;  // [U][G]
  int U, Up, G, Gp;
  __device__ __forceinline__ float operator()(int n, int k) const {
    const bool oim = n >= Gp;
    const int g = oim ? n - Gp : n;
    if (g >= G) return 0.f;
    const bool kim = k >= Up;
    const int u = kim ? k - Up : k;
    if (u >= U) return 0.f;
    const cplx<float> v = p[(long long)u * G + g];
    return !oim ? (kim ? -v.y : v.x) : (kim ? v.x : v.y);
  }
};
struct UpEp {
  cplx<float>* y;  // [R][G], updated in place: y += s * D
  int R, G, Gp;
  float s;
  __device__ __forceinline__ void operator()(int r, int n, float v, int) const {
    const bool im = n >= Gp;
    const int g = im ? n - Gp : n;
    if (r >= R || g >= G) return;
    float* d = reinterpret_cast<float*>(y + (long long)r * G + g);
    d[im ? 1 : 0] += s * v;
  }
  __device__ __forceinline__ float* addr(int r, int n) const {
    const bool im = n >= Gp;
    const int g = im ? n - Gp : n;
    if (r >= R || g >= G) return nullptr;
    return reinterpret_cast<float*>(y + (long long)r * G + g) + (im ? 1 : 0);
  }
  __device__ __forceinline__ float load(int r, int n, int) const {
    const float* d = addr(r, n);
    return d ? *d : 0.f;
  }
  __device__ __forceinline__ void store(int r, int n, float old, float v, int) const {
    float* d = addr(r, n);
    if (d) *d = old + s * v;
  }
};

// ---------------------------------------------------------------------------
// Packed-operand path (used where the packed operands fit the handle's buffer).
// k_umma_pack writes a real operand, given by one of the loaders above, as TF32
// high and low tiles in the canonical layout of the MMA (the image that the
// staging loop of k_umma_gemm builds in shared memory): tile (row block rb, K
// chunk c) at ((rb * kchunks + c) * 2 + part) * UMMA_M * UMMA_KC words, part 0 =
// high, 1 = low. Consecutive threads write consecutive words.
// k_umma_tiles brings the tile pairs of a K chunk into shared memory with one bulk
// copy per operand (cp.async.bulk, completion counted on an mbarrier), in a ring of
// UMMA_STAGES stages; one thread waits for a stage's copies, issues its 12 MMAs,
// commits them to the stage's second mbarrier and refills the stage once those
// MMAs are done, so copies of later chunks overlap the MMAs of earlier ones and no
// thread touches the operands in between. The accumulator tile goes through shared
// memory to the epilogue, one row after the other across the CTA's threads
// (consecutive threads take consecutive columns). Every wait is bounded: on a
// timeout the CTA waits (bounded) for what it issued, sets *err, frees its tensor
// memory and returns.
// ---------------------------------------------------------------------------
constexpr int UMMA_TILE_WORDS = UMMA_M * UMMA_KC;           // 4096
constexpr int UMMA_PAIR_BYTES = 2 * UMMA_TILE_BYTES;        // high + low tile, 32 KB
constexpr int UMMA_STAGES = 3;
constexpr int UMMA_STAGE_BYTES = 2 * UMMA_PAIR_BYTES;       // A pair + B pair
constexpr int UMMA_DPITCH = UMMA_N + 1;                     // epilogue staging row pitch (words)
constexpr int UMMA_TILES_SMEM = UMMA_STAGES * UMMA_STAGE_BYTES + 128;

template <class LD>
__global__ void __launch_bounds__(256) k_umma_pack(LD ld, int kchunks, uint32_t* __restrict__ out) {
  const int c = blockIdx.x, rb = blockIdx.y;
  uint32_t* hi = out + (size_t)(rb * kchunks + c) * 2 * UMMA_TILE_WORDS;
  uint32_t* lo = hi + UMMA_TILE_WORDS;
  for (int o = threadIdx.x; o < UMMA_TILE_WORDS; o += 256) {
    // word o = ((row / 8) * 8 + k / 4) * 32 + (row % 8) * 4 + k % 4 (see umma_offset)
    const int row = (o >> 8) * 8 + ((o >> 2) & 7), k = ((o >> 5) & 7) * 4 + (o & 3);
    const float v = ld(rb * UMMA_M + row, c * UMMA_KC + k);
    const uint32_t h = to_tf32(v);
    hi[o] = h;
    lo[o] = to_tf32(v - __uint_as_float(h));
  }
}

__device__ __forceinline__ bool umma_bar_wait(uint32_t bar, uint32_t parity) {
  for (long long polls = 0; polls < UMMA_WAIT_LIMIT; ++polls) {
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

// pa: packed A [mtiles][kchunks][2][4096]; pb: packed B [ntiles][kchunks][2][4096]
template <class EP>
__global__ void __launch_bounds__(128)
    k_umma_tiles(const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb, EP ep, int kchunks,
                 int chunks_per_split, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char umma_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(umma_smem + UMMA_STAGES * UMMA_STAGE_BYTES);
  uint64_t* empty = full + UMMA_STAGES;
  uint64_t* done = empty + UMMA_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * UMMA_M, n0 = blockIdx.x * UMMA_N, split = blockIdx.z;
  const int c0 = split * chunks_per_split, c1 = min(kchunks, c0 + chunks_per_split), nch = max(0, c1 - c0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(UMMA_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < 2 * UMMA_STAGES + 1; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + s)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  int bad = 0;
  if (tid == 0 && nch > 0) {
    const uint32_t* abase = pa + (size_t)blockIdx.y * kchunks * 2 * UMMA_TILE_WORDS;
    const uint32_t* bbase = pb + (size_t)blockIdx.x * kchunks * 2 * UMMA_TILE_WORDS;
    int loaded = 0, consumed = 0;
    auto load = [&](int i) {  // chunk c0 + i into stage i % UMMA_STAGES
      unsigned char* st = umma_smem + (i % UMMA_STAGES) * UMMA_STAGE_BYTES;
      const uint32_t bar = smem_u32(full + i % UMMA_STAGES);
      const size_t off = (size_t)(c0 + i) * 2 * UMMA_TILE_WORDS;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(2 * UMMA_PAIR_BYTES)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       smem_u32(st)),
                   "l"(abase + off), "r"(UMMA_PAIR_BYTES), "r"(bar)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       smem_u32(st + UMMA_PAIR_BYTES)),
                   "l"(bbase + off), "r"(UMMA_PAIR_BYTES), "r"(bar)
                   : "memory");
      ++loaded;
    };
    for (int i = 0; i < min(UMMA_STAGES, nch); ++i) load(i);
    constexpr uint32_t idesc = umma_idesc_tf32();
    for (int i = 0; i < nch && !bad; ++i) {
      const int s = i % UMMA_STAGES;
      const uint32_t ph = (uint32_t)(i / UMMA_STAGES) & 1u;
      if (!umma_bar_wait(smem_u32(full + s), ph)) {
        bad = 1;
        break;
      }
      ++consumed;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t sa = smem_u32(umma_smem + s * UMMA_STAGE_BYTES), sb = sa + UMMA_PAIR_BYTES;
#pragma unroll
      for (int kk = 0; kk < UMMA_KC / 8; ++kk) {
        const uint32_t koff = kk * 256;  // 8 tf32 = 2 core matrices along K
        const uint64_t ah = umma_desc(sa + koff), al = umma_desc(sa + UMMA_TILE_BYTES + koff);
        const uint64_t bh = umma_desc(sb + koff), bl = umma_desc(sb + UMMA_TILE_BYTES + koff);
        const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
        umma_tf32(tmem, ah, bh, idesc, acc0);
        umma_tf32(tmem, ah, bl, idesc, 1u);
        umma_tf32(tmem, al, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(empty + s)));
      // refill the previous chunk's stage once its MMAs have read it (this chunk's MMAs queue behind them)
      const int ip = i - 1;
      if (ip >= 0 && ip + UMMA_STAGES < nch) {
        if (!umma_bar_wait(smem_u32(empty + ip % UMMA_STAGES), (uint32_t)(ip / UMMA_STAGES) & 1u)) {
          bad = 1;
          break;
        }
        load(ip + UMMA_STAGES);
      }
    }
    // all MMAs issued so far complete before the accumulator is read (or the CTA leaves)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_u32(done)));
    if (!umma_bar_wait(smem_u32(done), 0u)) bad = 1;
    // copies still in flight (after a timeout) land before the shared memory is reused
    for (; consumed < loaded; ++consumed)
      umma_bar_wait(smem_u32(full + consumed % UMMA_STAGES), (uint32_t)(consumed / UMMA_STAGES) & 1u);
    if (bad) atomicExch(err, 1);
  }
  const int failed = __syncthreads_or(bad);
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (!failed) {
    float* dst = reinterpret_cast<float*>(umma_smem);  // [UMMA_M][UMMA_DPITCH], over the stage buffers
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int cb = 0; cb < UMMA_N; cb += 16) {
      uint32_t r[16];
      if (nch > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + lane_base + (uint32_t)cb));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[tid * UMMA_DPITCH + cb + j] = __uint_as_float(r[j]);
    }
    __syncthreads();
    // rows in groups of 16: the group's loads (for read-modify-write epilogues) are in flight together
#pragma unroll 1
    for (int mg = 0; mg < UMMA_M; mg += 16) {
      float old[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) old[j] = ep.load(m0 + mg + j, n0 + tid, split);
#pragma unroll
      for (int j = 0; j < 16; ++j) ep.store(m0 + mg + j, n0 + tid, old[j], dst[(mg + j) * UMMA_DPITCH + tid], split);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UMMA_N));
  }
}

}  // namespace tddft
