// Host-side launchers of the plane kernels for one (T, N), and the dispatch
// table that picks them by grid size at run time.
#pragma once
#include "kernels.cuh"

namespace tddft {

// Launch accounting (defined in tddft_api.cu). note_launch() counts every
// kernel launch of the library; when the profiler is enabled, prof_begin /
// prof_end bracket each plane-kernel launch with CUDA events on its stream and
// add the launch's algorithmic bytes to its class.
enum KernelClass { KC_XY_FWD = 0, KC_Z = 1, KC_XY_INV = 2, KC_COUNT = 3 };
void note_launch();
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double bytes);

template <typename T>
struct PlaneOps {
  int n = 0;
  cudaError_t (*prepare)() = nullptr;
  void (*xy_fwd)(int mode, const cplx<T>* qb, const cplx<T>* rb, PairMap pm, int items, cplx<T>* ibuf,
                 const cplx<T>* tw, cudaStream_t st) = nullptr;
  void (*z)(int mode, cplx<T>* ibuf, int items, const T* kern, T kscale, const cplx<T>* tw, cudaStream_t st) = nullptr;
  void (*xy_inv)(int mode, const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* pb, PairMap pm, int targets, T scale,
                 const cplx<T>* tw, cudaStream_t st) = nullptr;
};

template <typename T, int N>
struct PlaneLaunch {
  static constexpr int NT = plane_threads<N>();
  static constexpr size_t SMEM = (size_t)(N + N * plane_pitch<N>()) * sizeof(cplx<T>);

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
#undef TDDFT_CARVE
    return cudaSuccess;
  }

  static void xy_fwd(int mode, const cplx<T>* qb, const cplx<T>* rb, PairMap pm, int items, cplx<T>* ibuf,
                     const cplx<T>* tw, cudaStream_t st) {
    if (items <= 0) return;
    dim3 grid(N, items);
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    prof_begin(KC_XY_FWD, st);
    if (mode == XY_PRODUCT)
      k_xy_fwd<T, N, XY_PRODUCT><<<grid, NT, SMEM, st>>>(qb, rb, pm, ibuf, tw);
    else
      k_xy_fwd<T, N, XY_LOAD><<<grid, NT, SMEM, st>>>(qb, rb, pm, ibuf, tw);
    note_launch();
    prof_end(KC_XY_FWD, st, (mode == XY_PRODUCT ? 3.0 : 2.0) * F * items);
  }

  static void z(int mode, cplx<T>* ibuf, int items, const T* kern, T kscale, const cplx<T>* tw, cudaStream_t st) {
    if (items <= 0) return;
    dim3 grid(N, items);
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    prof_begin(KC_Z, st);
    if (mode == Z_CONV)
      k_z<T, N, Z_CONV><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
    else if (mode == Z_FWD)
      k_z<T, N, Z_FWD><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
    else
      k_z<T, N, Z_INV><<<grid, NT, SMEM, st>>>(ibuf, kern, kscale, tw);
    note_launch();
    prof_end(KC_Z, st, 2.0 * F * items + (mode == Z_CONV ? F / 2.0 : 0.0));
  }

  static void xy_inv(int mode, const cplx<T>* ibuf, cplx<T>* ob, const cplx<T>* pb, PairMap pm, int targets, T scale,
                     const cplx<T>* tw, cudaStream_t st) {
    if (targets <= 0) return;
    constexpr double F = (double)N * N * N * sizeof(cplx<T>);
    prof_begin(KC_XY_INV, st);
    if (mode == INV_ACCUM) {
      k_xy_inv<T, N, INV_ACCUM><<<dim3(N, targets), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw);
    } else if (mode == INV_ATOMIC) {
      k_xy_inv<T, N, INV_ATOMIC><<<dim3(N, targets * pm.kdim), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw);
    } else {
      k_xy_inv<T, N, INV_WRITE><<<dim3(N, targets), NT, SMEM, st>>>(ibuf, ob, pb, pm, scale, tw);
    }
    note_launch();
    prof_end(KC_XY_INV, st, mode == INV_WRITE ? 2.0 * F * targets : (2.0 * pm.kdim + 2.0) * F * targets);
  }

  static PlaneOps<T> ops() {
    PlaneOps<T> o;
    o.n = N;
    o.prepare = &prepare;
    o.xy_fwd = &xy_fwd;
    o.z = &z;
    o.xy_inv = &xy_inv;
    return o;
  }
};

// Dispatch by grid size; returns ops with n == 0 for an unsupported size.
template <typename T>
PlaneOps<T> plane_ops_for(int n);

}  // namespace tddft
