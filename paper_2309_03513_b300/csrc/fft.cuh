// Shared-memory 3D FFT building blocks for the pair-convolution path.
//
// A 3D transform of an N^3 field is done plane by plane: an xy-plane pass
// (x lines then y lines) and a z pass over xz-planes. Each 1D transform is an
// in-place mixed-radix Cooley-Tukey FFT:
//   forward  = decimation in frequency (DIF): natural order in, digit-reversed out;
//   inverse  = the DIF stages undone in reverse order (DIT): digit-reversed in,
//              natural order out.
// No reordering pass exists: every array that lives in reciprocal space (the
// convolution kernels, the sphere map) is stored in the digit-reversed order.
// Sign convention: forward exp(-2 pi i jk/N), inverse exp(+2 pi i jk/N), both
// unnormalised.
//
// Twiddles W_N^e = exp(-2 pi i e/N) come from a table computed on the host in
// FP64 with std::cos/std::sin and rounded once to the working precision.
#pragma once
#include <cuda_runtime.h>

namespace tddft {

template <typename T>
struct __align__(2 * sizeof(T)) cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <typename T>
__device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.x * s, a.y * s}; }

// Sums and differences of two plain complex values (neither one a rotated view such as
// mul_di(a), whose swapped halves would first have to be moved into place). In FP32 the
// two halves go through one packed instruction (add/sub.rn.f32x2, sm_100 and later):
// the same two IEEE round-to-nearest operations, half the instructions to issue.
__device__ __forceinline__ unsigned long long pack2(cplx<float> a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ cplx<float> unpack2(unsigned long long r) {
  cplx<float> a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
// PK = false keeps both halves as separate scalar instructions (for kernels whose register
// budget does not allow the aligned register pairs that packed operands need)
template <bool PK = true, typename T>
__device__ __forceinline__ cplx<T> padd(cplx<T> a, cplx<T> b) {
  if constexpr (PK && sizeof(T) == 4) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(d);
  } else {
    return cadd(a, b);
  }
}
template <bool PK = true, typename T>
__device__ __forceinline__ cplx<T> psub(cplx<T> a, cplx<T> b) {
  if constexpr (PK && sizeof(T) == 4) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(d);
  } else {
    return csub(a, b);
  }
}


template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.x, -a.y}; }
// multiply by +i / -i
template <typename T>
__device__ __forceinline__ cplx<T> mul_pi(cplx<T> a) { return {-a.y, a.x}; }
template <typename T>
__device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) { return {a.y, -a.x}; }

constexpr int FWD = -1;  // exp(-2 pi i ...)
constexpr int INV = +1;  // exp(+2 pi i ...)

// multiply by (DIR i): forward -> -i, inverse -> +i
template <int DIR, typename T>
__device__ __forceinline__ cplx<T> mul_di(cplx<T> a) {
  if constexpr (DIR == FWD) return mul_mi(a);
  else return mul_pi(a);
}

// a * w (forward) or a * conj(w) (inverse), w a table twiddle W_N^e
template <int DIR, typename T>
__device__ __forceinline__ cplx<T> twmul(cplx<T> a, cplx<T> w) {
  if constexpr (DIR == FWD) return cmul(a, w);
  else return cmulc(w, a);
}

// Twiddle accessors: tw(e) = W_N^e = exp(-2 pi i e / N) for the N of the transform.
// TwPtr reads a table in shared memory; TwConst (below) reads the constant-memory
// table, where a compile-time index becomes an immediate constant operand.
template <typename T>
struct TwPtr {
  const cplx<T>* p;
  __device__ __forceinline__ cplx<T> operator()(int e) const { return p[e]; }
};

// ---------------------------------------------------------------------------
// Radix codelets: v[k] <- sum_n v[n] exp(DIR 2 pi i n k / R), natural order.
// Mathematical constants: sqrt(3)/2, cos/sin(2 pi/5), cos/sin(4 pi/5), 1/sqrt(2).
// ---------------------------------------------------------------------------
template <int DIR, bool PK = true, typename T>
__device__ __forceinline__ void dft2(cplx<T>* v) {
  cplx<T> a = v[0], b = v[1];
  v[0] = padd<PK>(a, b);
  v[1] = psub<PK>(a, b);
}

template <int DIR, bool PK = true, typename T>
__device__ __forceinline__ void dft3(cplx<T>* v) {
  const T c = T(-0.5);
  const T s = T(0.86602540378443864676372317075293618);
  cplx<T> t1 = padd<PK>(v[1], v[2]);
  cplx<T> t2 = cadd(v[0], cscale(t1, c));
  cplx<T> t3 = cscale(psub<PK>(v[1], v[2]), s);
  v[0] = padd<PK>(v[0], t1);
  cplx<T> it3 = mul_di<DIR>(t3);
  v[1] = cadd(t2, it3);
  v[2] = csub(t2, it3);
}

template <int DIR, bool PK = true, typename T>
__device__ __forceinline__ void dft4(cplx<T>* v) {
  cplx<T> t0 = padd<PK>(v[0], v[2]), t1 = psub<PK>(v[0], v[2]);
  cplx<T> t2 = padd<PK>(v[1], v[3]), t3 = mul_di<DIR>(psub<PK>(v[1], v[3]));
  v[0] = padd<PK>(t0, t2);
  v[2] = psub<PK>(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <int DIR, bool PK = true, typename T>
__device__ __forceinline__ void dft5(cplx<T>* v) {
  const T c1 = T(0.30901699437494742410229341718281906);
  const T c2 = T(-0.80901699437494742410229341718281906);
  const T s1 = T(0.95105651629515357211643933337938214);
  const T s2 = T(0.58778525229247312916870595463907277);
  cplx<T> a1 = padd<PK>(v[1], v[4]), b1 = psub<PK>(v[1], v[4]);
  cplx<T> a2 = padd<PK>(v[2], v[3]), b2 = psub<PK>(v[2], v[3]);
  cplx<T> x0 = v[0];
  v[0] = padd<PK>(x0, padd<PK>(a1, a2));
  cplx<T> r1 = cadd(x0, cadd(cscale(a1, c1), cscale(a2, c2)));
  cplx<T> r2 = cadd(x0, cadd(cscale(a1, c2), cscale(a2, c1)));
  cplx<T> i1 = mul_di<DIR>(cadd(cscale(b1, s1), cscale(b2, s2)));
  cplx<T> i2 = mul_di<DIR>(csub(cscale(b1, s2), cscale(b2, s1)));
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

// Multiply by exp(DIR 2 pi i E / R); exact for multiples of pi/4, table otherwise.
// tw points at the length-N table, twstride = N / R.
template <int DIR, int R, int E, typename T, typename TW>
__device__ __forceinline__ cplx<T> rot(cplx<T> a, const TW& tw, int twstride) {
  constexpr int e = E % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr ((4 * e) % R == 0) {
    constexpr int q = (4 * e) / R;  // quarter turns
    if constexpr (q == 1) return mul_di<DIR>(a);
    else if constexpr (q == 2) return {-a.x, -a.y};
    else return mul_di<-DIR>(a);
  } else if constexpr ((8 * e) % R == 0) {
    constexpr int o = (8 * e) / R;  // odd number of eighth turns: 1, 3, 5, 7
    const T h = T(0.70710678118654752440084436210484904);
    // exp(DIR i pi o/4) a from s = a.x + a.y and d = a.x - a.y, each half written in its
    // final place and sign (no swapped view left for a packed consumer to move into place);
    // the inverse turn by o eighths is the forward turn by 8 - o
    constexpr int of = (DIR == FWD) ? o : 8 - o;
    const T sh = (a.x + a.y) * h, dh = (a.x - a.y) * h;
    if constexpr (of == 1) return {sh, -dh};
    else if constexpr (of == 3) return {-dh, -sh};
    else if constexpr (of == 5) return {-sh, dh};
    else return {dh, sh};
  } else {
    return twmul<DIR>(a, tw(e * twstride));
  }
}

template <int R, int DIR, bool PK = true, typename T, typename TW>
__device__ __forceinline__ void dft(cplx<T>* v, const TW& tw, int twstride);

template <int P, int Q, int DIR, typename T, int Q0, int K1, typename TW>
__device__ __forceinline__ void comp_rot(cplx<T>* t, cplx<T>* u, const TW& tw, int twstride) {
  if constexpr (K1 < P) {
    u[Q0 * P + K1] = rot<DIR, P * Q, Q0 * K1>(t[K1], tw, twstride);
    comp_rot<P, Q, DIR, T, Q0, K1 + 1>(t, u, tw, twstride);
  }
}

// Composite codelet R = P * Q: input index n = q + Q p, output k = k1 + P k2.
template <int P, int Q, int DIR, bool PK, typename T, int Q0 = 0, typename TW>
__device__ __forceinline__ void comp_first(cplx<T>* v, cplx<T>* u, const TW& tw, int twstride) {
  if constexpr (Q0 < Q) {
    cplx<T> t[P];
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = v[Q0 + Q * p];
    dft<P, DIR, PK>(t, tw, twstride * Q);
    comp_rot<P, Q, DIR, T, Q0, 0>(t, u, tw, twstride);
    comp_first<P, Q, DIR, PK, T, Q0 + 1>(v, u, tw, twstride);
  }
}

template <int P, int Q, int DIR, bool PK, typename T, typename TW>
__device__ __forceinline__ void dft_comp(cplx<T>* v, const TW& tw, int twstride) {
  cplx<T> u[P * Q];
  comp_first<P, Q, DIR, PK, T, 0>(v, u, tw, twstride);
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    cplx<T> t[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) t[q] = u[q * P + k1];
    dft<Q, DIR, PK>(t, tw, twstride * P);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
  }
}

// twstride: index step in the length-N table for W_R (N / R).
template <int R, int DIR, bool PK, typename T, typename TW>
__device__ __forceinline__ void dft(cplx<T>* v, const TW& tw, int twstride) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<DIR, PK>(v);
  } else if constexpr (R == 3) {
    dft3<DIR, PK>(v);
  } else if constexpr (R == 4) {
    dft4<DIR, PK>(v);
  } else if constexpr (R == 5) {
    dft5<DIR, PK>(v);
  } else if constexpr (R == 6) {
    dft_comp<2, 3, DIR, PK>(v, tw, twstride);
  } else if constexpr (R == 8) {
    dft_comp<2, 4, DIR, PK>(v, tw, twstride);
  } else if constexpr (R == 9) {
    dft_comp<3, 3, DIR, PK>(v, tw, twstride);
  } else if constexpr (R == 12) {
    dft_comp<4, 3, DIR, PK>(v, tw, twstride);
  } else if constexpr (R == 16) {
    dft_comp<4, 4, DIR, PK>(v, tw, twstride);
  } else {
    static_assert(R == 2, "unsupported radix");
  }
}

// ---------------------------------------------------------------------------
// Radix plans. Stage s has radix R_s; the stage operates on blocks of length
// L_s = N / (R_0 ... R_{s-1}) and butterflies of stride M_s = L_s / R_s.
// ---------------------------------------------------------------------------
template <int N>
struct Plan;
#define TDDFT_PLAN(NN, ...)                                \
  template <>                                              \
  struct Plan<NN> {                                        \
    static constexpr int r[] = {__VA_ARGS__};              \
    static constexpr int S = sizeof(r) / sizeof(int);      \
  };
TDDFT_PLAN(8, 8)
TDDFT_PLAN(12, 4, 3)
TDDFT_PLAN(16, 16)
TDDFT_PLAN(24, 8, 3)
TDDFT_PLAN(32, 8, 4)
TDDFT_PLAN(36, 4, 9)
TDDFT_PLAN(48, 16, 3)
TDDFT_PLAN(64, 8, 8)
TDDFT_PLAN(72, 8, 9)
TDDFT_PLAN(80, 16, 5)
TDDFT_PLAN(96, 12, 8)
TDDFT_PLAN(108, 12, 9)
TDDFT_PLAN(128, 8, 16)
#undef TDDFT_PLAN

template <int N, int S>
__host__ __device__ constexpr int plan_block() {  // L_s
  int l = N;
  for (int i = 0; i < S; ++i) l /= Plan<N>::r[i];
  return l;
}

// Per-stage twiddle tables: stage s stores W_{L_s}^{n1 k2} at [k2 * M_s + n1]
// (k2 < R_s, n1 < M_s), L_s entries, so that lanes with consecutive n1 read
// consecutive words. The tables of all stages follow each other.
template <int N, int S>
__host__ __device__ constexpr int stage_tw_off() {
  int off = 0;
  for (int i = 0; i < S; ++i) {
    int l = N;
    for (int j = 0; j < i; ++j) l /= Plan<N>::r[j];
    off += l;
  }
  return off;
}
template <int N>
__host__ __device__ constexpr int stage_tw_len() {
  return stage_tw_off<N, Plan<N>::S>();
}
// Shared-memory twiddle region of the staged kernels: the length-N table
// followed by the per-stage tables.
template <int N>
__host__ __device__ constexpr int tw_table_len() {
  return N + stage_tw_len<N>();
}

// Threads per line: a CTA of N * G threads works on N lines at once.
template <int N>
__host__ __device__ constexpr int lines_group() {
  return N <= 16 ? 16 : (N <= 32 ? 8 : 4);
}
template <int N>
__host__ __device__ constexpr int plane_threads() {
  return N * lines_group<N>();
}
// Row pitch (complex elements) of a plane in shared memory: odd, so that
// threads walking different lines hit different banks.
template <int N>
__host__ __device__ constexpr int plane_pitch() {
  return N + 1;
}

// One DIF stage (forward) or its inverse over all N lines of a plane in smem.
// Line l is a row (elements l*PITCH + i) when ROWS, a column (i*PITCH + l) otherwise.
// The butterfly inputs come from ld(i) and the outputs go to st(i, v) (element i of
// the line): by default the plane in shared memory; the first or last stage of a
// pass can read from or write to global memory instead.
template <typename T, int N, int ROWS>
struct PlaneLd {
  const cplx<T>* s;
  int line;
  __device__ __forceinline__ cplx<T> operator()(int i) const {
    constexpr int PITCH = plane_pitch<N>();
    return ROWS ? s[line * PITCH + i] : s[i * PITCH + line];
  }
};
template <typename T, int N, int ROWS>
struct PlaneSt {
  cplx<T>* s;
  int line;
  __device__ __forceinline__ void operator()(int i, cplx<T> v) const {
    constexpr int PITCH = plane_pitch<N>();
    if (ROWS) s[line * PITCH + i] = v;
    else s[i * PITCH + line] = v;
  }
};

template <typename T, int N, int S, int DIR, bool ROWS, typename LD, typename ST>
__device__ __forceinline__ void stage_io(const cplx<T>* tw, int g, const LD& ld, const ST& st) {
  constexpr int R = Plan<N>::r[S];
  constexpr int L = plan_block<N, S>();
  constexpr int M = L / R;
  constexpr int G = lines_group<N>();
  constexpr int NB = N / R;         // butterflies per line
  const cplx<T>* stw = tw + N + stage_tw_off<N, S>();  // [k2 * M + n1]
#pragma unroll 1
  for (int j = g; j < NB; j += G) {
    const int blk = j / M, n1 = j - blk * M;
    const int base = blk * L + n1;
    cplx<T> v[R];
    if constexpr (DIR == FWD) {
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) v[n2] = ld(base + M * n2);
      dft<R, FWD>(v, TwPtr<T>{tw}, N / R);
#pragma unroll
      for (int k2 = 1; k2 < R; ++k2)
        if (n1) v[k2] = twmul<FWD>(v[k2], stw[k2 * M + n1]);
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) st(base + M * k2, v[k2]);
    } else {
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) {
        v[k2] = ld(base + M * k2);
        if (k2 && n1) v[k2] = twmul<INV>(v[k2], stw[k2 * M + n1]);
      }
      dft<R, INV>(v, TwPtr<T>{tw}, N / R);
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) st(base + M * n2, v[n2]);
    }
  }
}

template <typename T, int N, int S, int DIR, bool ROWS>
__device__ __forceinline__ void stage(cplx<T>* s, const cplx<T>* tw, int line, int g) {
  stage_io<T, N, S, DIR, ROWS>(tw, g, PlaneLd<T, N, ROWS>{s, line}, PlaneSt<T, N, ROWS>{s, line});
}

// Full 1D transform of all lines of the plane (syncs between stages and at the end).
template <typename T, int N, int DIR, bool ROWS, int S = 0>
__device__ __forceinline__ void fft_lines(cplx<T>* s, const cplx<T>* tw, int line, int g) {
  constexpr int NS = Plan<N>::S;
  if constexpr (S < NS) {
    constexpr int st = (DIR == FWD) ? S : (NS - 1 - S);
    stage<T, N, st, DIR, ROWS>(s, tw, line, g);
    __syncthreads();
    fft_lines<T, N, DIR, ROWS, S + 1>(s, tw, line, g);
  }
}

// The same with the first stage reading its inputs through ld (instead of the plane).
template <typename T, int N, int DIR, bool ROWS, typename LD>
__device__ __forceinline__ void fft_lines_from(cplx<T>* s, const cplx<T>* tw, int line, int g, const LD& ld) {
  constexpr int NS = Plan<N>::S;
  constexpr int st0 = (DIR == FWD) ? 0 : NS - 1;
  stage_io<T, N, st0, DIR, ROWS>(tw, g, ld, PlaneSt<T, N, ROWS>{s, line});
  __syncthreads();
  if constexpr (NS > 1) fft_lines<T, N, DIR, ROWS, 1>(s, tw, line, g);
}

// The same with the last stage writing its outputs through st (no barrier after it).
template <typename T, int N, int DIR, bool ROWS, typename ST, int S = 0>
__device__ __forceinline__ void fft_lines_to(cplx<T>* s, const cplx<T>* tw, int line, int g, const ST& st) {
  constexpr int NS = Plan<N>::S;
  constexpr int stg = (DIR == FWD) ? S : (NS - 1 - S);
  if constexpr (S + 1 < NS) {
    stage<T, N, stg, DIR, ROWS>(s, tw, line, g);
    __syncthreads();
    fft_lines_to<T, N, DIR, ROWS, ST, S + 1>(s, tw, line, g, st);
  } else {
    stage_io<T, N, stg, DIR, ROWS>(tw, g, PlaneLd<T, N, ROWS>{s, line}, st);
  }
}

// ---------------------------------------------------------------------------
// Constant-memory twiddle tables (one per translation unit; filled by the
// launchers' prepare()) and the register-resident 1D transform.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tw_offset(int n) {
  constexpr int sizes[] = {8, 12, 16, 24, 32, 36, 48, 64, 72, 80, 96, 108, 128};
  int off = 0;
  for (int s : sizes) {
    if (s == n) return off;
    off += s;
  }
  return -1;
}
constexpr int TW_TOTAL = 724;  // sum of the supported sizes
static __constant__ cplx<float> c_tw_f32[TW_TOTAL];
static __constant__ cplx<double> c_tw_f64[TW_TOTAL];

template <typename T, int N>
struct TwConst {
  __device__ __forceinline__ cplx<T> operator()(int e) const {
    if constexpr (sizeof(T) == 4) return c_tw_f32[tw_offset(N) + e];
    else return c_tw_f64[tw_offset(N) + e];
  }
};

// Whole length-N transform of v[0..N) held in registers: forward = DIF
// (natural in, digit-reversed out), inverse = DIT (digit-reversed in, natural out).
template <typename T, int N, int DIR, typename TW, int S = 0, bool PK = true>
__device__ __forceinline__ void fft_reg(cplx<T>* v, const TW& tw) {
  constexpr int NS = Plan<N>::S;
  if constexpr (S < NS) {
    constexpr int st = (DIR == FWD) ? S : (NS - 1 - S);
    constexpr int R = Plan<N>::r[st];
    constexpr int L = plan_block<N, st>();
    constexpr int M = L / R;
    constexpr int TWS = N / L;
#pragma unroll
    for (int blk = 0; blk < N / L; ++blk) {
#pragma unroll
      for (int n1 = 0; n1 < M; ++n1) {
        const int base = blk * L + n1;
        cplx<T> x[R];
        if constexpr (DIR == FWD) {
#pragma unroll
          for (int n2 = 0; n2 < R; ++n2) x[n2] = v[base + M * n2];
          dft<R, FWD, PK>(x, tw, N / R);
#pragma unroll
          for (int k2 = 1; k2 < R; ++k2)
            if (n1) x[k2] = twmul<FWD>(x[k2], tw(n1 * k2 * TWS));
#pragma unroll
          for (int k2 = 0; k2 < R; ++k2) v[base + M * k2] = x[k2];
        } else {
#pragma unroll
          for (int k2 = 0; k2 < R; ++k2) {
            x[k2] = v[base + M * k2];
            if (k2 && n1) x[k2] = twmul<INV>(x[k2], tw(n1 * k2 * TWS));
          }
          dft<R, INV, PK>(x, tw, N / R);
#pragma unroll
          for (int n2 = 0; n2 < R; ++n2) v[base + M * n2] = x[n2];
        }
      }
    }
    fft_reg<T, N, DIR, TW, S + 1, PK>(v, tw);
  }
}

}  // namespace tddft
