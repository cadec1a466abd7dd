// Host-side launchers of the plane kernels for one (T, N), and the dispatch
// table that picks them by grid size at run time.
#pragma once
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "plane_lines.cuh"

namespace tddft {

// Launch accounting (defined in tddft_api.cu). note_launch() counts every
// kernel launch of the library; when the profiler is enabled, prof_begin /
// prof_end bracket each plane-kernel launch with CUDA events on its stream and
// add the launch's algorithmic bytes to its class.
enum KernelClass { KC_XY_FWD = 0, KC_Z = 1, KC_XY_INV = 2, KC_COUNT = 3 };
void note_launch();
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double bytes);

// z = 0: shared-memory staged z pass; 1: register-resident columns (FP32, n <= 80);
// 2: as 1, with the compact pair-density convolutions on two threads per column (FP32,
// n <= 80 and n = 96; at 96 the other z passes are the staged ones).
struct KernelChoice {
  int z = 1;
};

// Compact pair-density columns (see stage_in_plane in plane_kernels.cuh):
// the nact column positions that can be non-zero; nullptr = full planes. The
// three passes of a convolution get the same list; it is only given when the
// register-resident z pass runs (the staged z pass takes full planes).
struct ColumnList {
  const int* cols = nullptr;
  int nact = 0;
  // compact index of every (x, y) position, transposed ([x][y], -1 outside the disc): when
  // given (and the register-line kernels exist for N), the xy passes of compact planes run
  // on the register-line kernels of plane_lines.cuh
  const int* cmapT = nullptr;
  int lanes_fwd = 1;  // register-line kernels: lanes per line (1 or 2) of the forward pass
  int lanes_inv = 2;  // and of the inverse pass
};

template <typename T>
struct PlaneOps {
  int n = 0;
  bool reg_ok = false;   // the register-resident z pass exists for this (T, N)
  bool pair_ok = false;  // the two-threads-per-column z pass exists for this (T, N)
  bool lines_ok = false; // the register-line xy passes exist for this (T, N)
  KernelChoice kc;
  cudaError_t (*prepare)() = nullptr;
  void (*f_xy_fwd)(int mode, const cplx<T>* qb, const cplx<T>* rb, PairMap pm, int items, cplx<T>* ibuf,
                   const cplx<T>* tw, ColumnList cl, cudaStream_t st) = nullptr;
  void (*f_z)(KernelChoice kc, int mode, cplx<T>* ibuf, int items, const T* kern, T kscale, const cplx<T>* tw,
              ColumnList cl, cudaStream_t st) = nullptr;
  void (*f_xy_inv)(int mode, const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* pb, PairMap pm, int targets, T scale,
                   const cplx<T>* tw, ColumnList cl, cudaStream_t st) = nullptr;
  void xy_fwd(int mode, const cplx<T>* qb, const cplx<T>* rb, PairMap pm, int items, cplx<T>* ibuf,
              const cplx<T>* tw, cudaStream_t st, ColumnList cl = ColumnList{}) const {
    f_xy_fwd(mode, qb, rb, pm, items, ibuf, tw, cl, st);
  }
  void z(int mode, cplx<T>* ibuf, int items, const T* kern, T kscale, const cplx<T>* tw, cudaStream_t st,
         ColumnList cl = ColumnList{}) const {
    f_z(kc, mode, ibuf, items, kern, kscale, tw, cl, st);
  }
  void xy_inv(int mode, const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* pb, PairMap pm, int targets, T scale,
              const cplx<T>* tw, cudaStream_t st, ColumnList cl = ColumnList{}) const {
    f_xy_inv(mode, ibuf, ob, pb, pm, targets, scale, tw, cl, st);
  }
};

template <typename T, int N>
struct PlaneLaunch {
  static constexpr int NT = plane_threads<N>();
  static constexpr size_t SMEM = (size_t)(tw_table_len<N>() + N * plane_pitch<N>()) * sizeof(cplx<T>);

  static cudaError_t prepare() {
    cudaError_t e;
#define TDDFT_ATTR(K)                                                                         \
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);        \
  if (e != cudaSuccess) return e;
    TDDFT_ATTR((k_xy_fwd<T, N, XY_LOAD>))
    TDDFT_ATTR((k_xy_fwd<T, N, XY_PRODUCT>))
    TDDFT_ATTR((k_z<T, N, Z_CONV>))
    TDDFT_ATTR((k_z<T, N, Z_FWD>))
    TDDFT_ATTR((k_z<T, N, Z_INV>))
    TDDFT_ATTR((k_xy_inv<T, N, INV_WRITE>))
    TDDFT_ATTR((k_xy_inv<T, N, INV_ACCUM>))
    TDDFT_ATTR((k_xy_inv<T, N, INV_ATOMIC>))
#undef TDDFT_ATTR
    // prefer shared memory over L1 so that several plane CTAs fit on an SM
#define TDDFT_CARVE(K)                                                                                   \
  e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared); \
  if (e != cudaSuccess) return e;
    TDDFT_CARVE((k_xy_fwd<T, N, XY_LOAD>))
    TDDFT_CARVE((k_xy_fwd<T, N, XY_PRODUCT>))
    TDDFT_CARVE((k_z<T, N, Z_CONV>))
    TDDFT_CARVE((k_z<T, N, Z_FWD>))
    TDDFT_CARVE((k_z<T, N, Z_INV>))
    TDDFT_CARVE((k_xy_inv<T, N, INV_WRITE>))
    TDDFT_CARVE((k_xy_inv<T, N, INV_ACCUM>))
    TDDFT_CARVE((k_xy_inv<T, N, INV_ATOMIC>))
    if constexpr (xy_lines_ok<T, N>()) {
      TDDFT_CARVE((k_xy_fwd_lines<T, N, XY_LOAD, 1>))
      TDDFT_CARVE((k_xy_fwd_lines<T, N, XY_PRODUCT, 1>))
      TDDFT_CARVE((k_xy_inv_lines<T, N, INV_WRITE, 1>))
      TDDFT_CARVE((k_xy_inv_lines<T, N, INV_ATOMIC, 1>))
      TDDFT_CARVE((k_xy_fwd_lines<T, N, XY_LOAD, 2>))
      TDDFT_CARVE((k_xy_fwd_lines<T, N, XY_PRODUCT, 2>))
      TDDFT_CARVE((k_xy_inv_lines<T, N, INV_WRITE, 2>))
      TDDFT_CARVE((k_xy_inv_lines<T, N, INV_ATOMIC, 2>))
    }
#undef TDDFT_CARVE
    // constant-memory twiddles W_N^e for the register-resident transforms,
    // computed in FP64 on the host and rounded once
    std::vector<cplx<T>> t(N);
    for (int k = 0; k < N; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)N;
      t[k] = {(T)std::cos(ang), (T)std::sin(ang)};
    }
    if constexpr (sizeof(T) == 4)
      e = cudaMemcpyToSymbol(c_tw_f32, t.data(), N * sizeof(cplx<T>), tw_offset(N) * sizeof(cplx<T>));
    else
      e = cudaMemcpyToSymbol(c_tw_f64, t.data(), N * sizeof(cplx<T>), tw_offset(N) * sizeof(cplx<T>));
    if (e != cudaSuccess) return e;
    if constexpr (z_pair_ok<T, N>()) {  // the half-length table of the paired z pass
      constexpr int H = N / 2;
      std::vector<cplx<T>> th(H);
      for (int k = 0; k < H; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)H;
        th[k] = {(T)std::cos(ang), (T)std::sin(ang)};
      }
      if constexpr (sizeof(T) == 4)
        e = cudaMemcpyToSymbol(c_tw_f32, th.data(), H * sizeof(cplx<T>), tw_offset(H) * sizeof(cplx<T>));
      else
        e = cudaMemcpyToSymbol(c_tw_f64, th.data(), H * sizeof(cplx<T>), tw_offset(H) * sizeof(cplx<T>));
    }
    return e;
  }

  static void xy_fwd(int mode, const cplx<T>* qb, const cplx<T>* rb, PairMap pm, int items, cplx<T>* ibuf,
                     const cplx<T>* tw, ColumnList cl, cudaStream_t st) {
    if (items <= 0) return;
    dim3 grid(N, items);
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    const double fout = cl.cols ? (double)cl.nact / ((double)N * N) : 1.0;  // share of the plane written
    prof_begin(KC_XY_FWD, st);
    bool done = false;
    if constexpr (xy_lines_ok<T, N>()) {
      if (cl.cols && cl.cmapT) {
        done = true;
        if (cl.lanes_fwd == 2) {
          if (mode == XY_PRODUCT)
            k_xy_fwd_lines<T, N, XY_PRODUCT, 2><<<grid, lines_threads<N, 2>(), 0, st>>>(qb, rb, pm, ibuf, cl.cmapT,
                                                                                     cl.nact);
          else
            k_xy_fwd_lines<T, N, XY_LOAD, 2><<<grid, lines_threads<N, 2>(), 0, st>>>(qb, rb, pm, ibuf, cl.cmapT, cl.nact);
        } else {
          if (mode == XY_PRODUCT)
            k_xy_fwd_lines<T, N, XY_PRODUCT, 1><<<grid, lines_threads<N, 1>(), 0, st>>>(qb, rb, pm, ibuf, cl.cmapT,
                                                                                     cl.nact);
          else
            k_xy_fwd_lines<T, N, XY_LOAD, 1><<<grid, lines_threads<N, 1>(), 0, st>>>(qb, rb, pm, ibuf, cl.cmapT, cl.nact);
        }
      }
    }
    if (done) {
    } else if (mode == XY_PRODUCT)
      k_xy_fwd<T, N, XY_PRODUCT><<<grid, NT, SMEM, st>>>(qb, rb, pm, ibuf, tw, cl.cols, cl.nact);
    else
      k_xy_fwd<T, N, XY_LOAD><<<grid, NT, SMEM, st>>>(qb, rb, pm, ibuf, tw, cl.cols, cl.nact);
    note_launch();
    prof_end(KC_XY_FWD, st, ((mode == XY_PRODUCT ? 2.0 : 1.0) + fout) * F * items);
  }

  static void zl(KernelChoice kc, int mode, cplx<T>* ibuf, int items, const T* kern, T kscale, const cplx<T>* tw,
                 ColumnList cl, cudaStream_t st) {
    if (items <= 0) return;
    dim3 grid(N, items);
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    const double fcol = cl.cols ? (double)cl.nact / ((double)N * N) : 1.0;
    prof_begin(KC_Z, st);
    bool done = false;
    if constexpr (z_pair_ok<T, N>()) {
      if (kc.z == 2 && cl.cols && mode == Z_CONV) {
        done = true;
        dim3 g((2 * cl.nact + ZREG_THREADS - 1) / ZREG_THREADS, items);
        k_z_pair<T, N><<<g, ZREG_THREADS, 0, st>>>(ibuf, kern, kscale, cl.nact);
      }
    }
    if constexpr (z_in_registers<T, N>()) {
      if (!done && kc.z >= 1) {
        done = true;
        const int ncol = cl.cols ? cl.nact : N * N;
        dim3 g((ncol + ZREG_THREADS - 1) / ZREG_THREADS, items);
        if (mode == Z_CONV && cl.cols)
          k_z_reg<T, N, Z_CONV, true><<<g, ZREG_THREADS, 0, st>>>(ibuf, kern, kscale, cl.nact);
        else if (mode == Z_CONV)
          k_z_reg<T, N, Z_CONV><<<g, ZREG_THREADS, 0, st>>>(ibuf, kern, kscale, 0);
        else if (mode == Z_FWD)
          k_z_reg<T, N, Z_FWD><<<g, ZREG_THREADS, 0, st>>>(ibuf, kern, kscale, 0);
        else
          k_z_reg<T, N, Z_INV><<<g, ZREG_THREADS, 0, st>>>(ibuf, kern, kscale, 0);
      }
    }
    if (!done) {
      if (mode == Z_CONV)
        k_z<T, N, Z_CONV><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
      else if (mode == Z_FWD)
        k_z<T, N, Z_FWD><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
      else
        k_z<T, N, Z_INV><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
    }
    note_launch();
    prof_end(KC_Z, st, fcol * (2.0 * F * items + (mode == Z_CONV ? F / 2.0 : 0.0)));
  }

  static void xy_inv(int mode, const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* pb, PairMap pm, int targets, T scale,
                     const cplx<T>* tw, ColumnList cl, cudaStream_t st) {
    if (targets <= 0) return;
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    const double fin = cl.cols ? (double)cl.nact / ((double)N * N) : 1.0;  // share of the plane read
    prof_begin(KC_XY_INV, st);
    bool done = false;
    if constexpr (xy_lines_ok<T, N>()) {
      if (cl.cols && cl.cmapT && mode != INV_ACCUM) {
        done = true;
        const dim3 g(N, mode == INV_ATOMIC ? targets * pm.kdim : targets);
        if (cl.lanes_inv == 2) {
          if (mode == INV_ATOMIC)
            k_xy_inv_lines<T, N, INV_ATOMIC, 2><<<g, lines_threads<N, 2>(), 0, st>>>(ibuf, ob, pb, pm, scale, cl.cmapT,
                                                                                   cl.nact);
          else
            k_xy_inv_lines<T, N, INV_WRITE, 2><<<g, lines_threads<N, 2>(), 0, st>>>(ibuf, ob, pb, pm, scale, cl.cmapT,
                                                                                  cl.nact);
        } else {
          if (mode == INV_ATOMIC)
            k_xy_inv_lines<T, N, INV_ATOMIC, 1><<<g, lines_threads<N, 1>(), 0, st>>>(ibuf, ob, pb, pm, scale, cl.cmapT,
                                                                                   cl.nact);
          else
            k_xy_inv_lines<T, N, INV_WRITE, 1><<<g, lines_threads<N, 1>(), 0, st>>>(ibuf, ob, pb, pm, scale, cl.cmapT,
                                                                                  cl.nact);
        }
      }
    }
    if (done) {
    } else if (mode == INV_ACCUM)
      k_xy_inv<T, N, INV_ACCUM><<<dim3(N, targets), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw, cl.cols, cl.nact);
    else if (mode == INV_ATOMIC)
      k_xy_inv<T, N, INV_ATOMIC><<<dim3(N, targets * pm.kdim), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw, cl.cols,
                                                                            cl.nact);
    else
      k_xy_inv<T, N, INV_WRITE><<<dim3(N, targets), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw, cl.cols, cl.nact);
    note_launch();
    prof_end(KC_XY_INV, st,
             mode == INV_WRITE ? (fin + 1.0) * F * targets : ((fin + 1.0) * pm.kdim + 2.0) * F * targets);
  }

  static PlaneOps<T> ops() {
    PlaneOps<T> o;
    o.n = N;
    o.reg_ok = z_in_registers<T, N>();
    o.pair_ok = z_pair_ok<T, N>();
    o.lines_ok = xy_lines_ok<T, N>();
    o.kc.z = o.pair_ok ? 2 : (o.reg_ok ? 1 : 0);
    o.prepare = &prepare;
    o.f_xy_fwd = &xy_fwd;
    o.f_z = &zl;
    o.f_xy_inv = &xy_inv;
    return o;
  }
};

// Host twiddle table of the staged kernels for grid size N (see tw_table_len):
// W_N^e for e < N, then per stage W_{L_s}^{n1 k2} at [k2 * M_s + n1]; FP64
// std::cos / std::sin, rounded once to T.
template <typename T>
std::vector<cplx<T>> host_twiddles(int n, const std::vector<int>& radices) {
  std::vector<cplx<T>> t;
  auto w = [n](long long e) {
    const double ang = -2.0 * M_PI * (double)e / (double)n;
    return cplx<T>{(T)std::cos(ang), (T)std::sin(ang)};
  };
  for (int e = 0; e < n; ++e) t.push_back(w(e));
  int l = n;
  for (int r : radices) {
    const int m = l / r, tws = n / l;
    for (int k2 = 0; k2 < r; ++k2)
      for (int n1 = 0; n1 < m; ++n1) t.push_back(w((long long)n1 * k2 * tws));
    l = m;
  }
  return t;
}

// Dispatch by grid size; returns ops with n == 0 for an unsupported size.
template <typename T>
PlaneOps<T> plane_ops_for(int n);

}  // namespace tddft
