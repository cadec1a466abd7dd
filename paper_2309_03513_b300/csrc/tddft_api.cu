// C ABI of the Liouville-operator library: system set-up, L.A, the adjoint of
// omega = <X|L X>, and a block-Davidson driver. Host code plus the small
// pointwise kernels; the FFT plane kernels live in plane_f32.cu / plane_f64.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/tddft.h"
#include "../../include/tddft_testing.h"
#include "gemm.cuh"
#include "plane_ops.cuh"
#include "umma.cuh"

using namespace tddft;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static tddft_status fail(tddft_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// ---------------------------------------------------------------------------
// host-side fault injection (tddft_testing_inject_fault; TDDFT_FAULT when the library is
// loaded): the library reports an allocation or a device wait as failed without any
// failure on the GPU, so callers' error handling can be tested
// ---------------------------------------------------------------------------
namespace {
std::mutex g_fault_mu;
std::atomic<bool> g_fault_armed{false};
int g_fault_alloc = -1;     // allocations to let through before the injected failure; -1: none
bool g_fault_wait = false;  // the next check of a device-wait flag reports a wait that ran out
thread_local bool t_alloc_injected = false;

void fault_rearm_locked() { g_fault_armed.store(g_fault_alloc >= 0 || g_fault_wait, std::memory_order_release); }

// TDDFT_FAULT = "alloc" (the first allocation), "alloc:N" (allocation N, counted from 0) or
// "wait"; anything else is ignored
struct FaultFromEnvironment {
  FaultFromEnvironment() {
    const char* v = std::getenv("TDDFT_FAULT");
    if (!v) return;
    const std::string e(v);
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (e == "wait") {
      g_fault_wait = true;
    } else if (e == "alloc") {
      g_fault_alloc = 0;
    } else if (e.rfind("alloc:", 0) == 0 && e.size() > 6) {
      char* end = nullptr;
      const long n = std::strtol(e.c_str() + 6, &end, 10);
      if (end && *end == 0 && n >= 0 && n < INT_MAX) g_fault_alloc = (int)n;
    }
    fault_rearm_locked();
  }
} g_fault_from_environment;

bool fault_take_alloc() {
  if (!g_fault_armed.load(std::memory_order_acquire)) return false;
  std::lock_guard<std::mutex> lk(g_fault_mu);
  if (g_fault_alloc < 0) return false;
  const bool now = g_fault_alloc == 0;
  --g_fault_alloc;  // -1 once it has fired
  fault_rearm_locked();
  return now;
}

bool fault_take_wait() {
  if (!g_fault_armed.load(std::memory_order_acquire)) return false;
  std::lock_guard<std::mutex> lk(g_fault_mu);
  const bool now = g_fault_wait;
  g_fault_wait = false;
  fault_rearm_locked();
  return now;
}
}  // namespace

// cudaMalloc of the library's device memory, through the fault injector
static cudaError_t lib_malloc(void** p, size_t bytes) {
  t_alloc_injected = false;
  if (fault_take_alloc()) {
    *p = nullptr;
    t_alloc_injected = true;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

static std::string alloc_error(size_t bytes, cudaError_t e) {
  return "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e) +
         (t_alloc_injected ? " (injected fault)" : "");
}

// Every entry point runs its body through abi_guard: a C++ exception (host memory exhausted, a
// worker thread that cannot start) becomes a status and a last-error message, never crossing
// the C ABI.
template <typename F>
static tddft_status abi_guard(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    try {
      return fail(TDDFT_ENOMEM, "host memory exhausted");
    } catch (...) {
      return TDDFT_ENOMEM;
    }
  } catch (const std::exception& e) {
    try {
      return fail(TDDFT_ENOMEM, std::string("host exception: ") + e.what());
    } catch (...) {
      return TDDFT_ENOMEM;
    }
  } catch (...) {
    return TDDFT_ENOMEM;
  }
}

#define CUDA_TRY(expr)                                                                                 \
  do {                                                                                                 \
    cudaError_t _e = (expr);                                                                           \
    if (_e != cudaSuccess)                                                                             \
      return fail(_e == cudaErrorMemoryAllocation ? TDDFT_ENOMEM : TDDFT_ECUDA,                        \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                                 \
  } while (0)

#define STATUS_TRY(expr)                  \
  do {                                    \
    tddft_status _s = (expr);             \
    if (_s != TDDFT_OK) return _s;        \
  } while (0)

static tddft_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TDDFT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return TDDFT_OK;
}

// ---------------------------------------------------------------------------
// launch accounting and the optional per-class profiler (process-wide, not thread-safe)
// ---------------------------------------------------------------------------
namespace {
struct Profiler {
  bool on = false;
  long long launches = 0;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cls;        // class of event pair i
  std::vector<double> bytes;   // algorithmic bytes of event pair i
  size_t used = 0;
  cudaEvent_t pending = nullptr;
};
Profiler g_prof;
}  // namespace

void tddft::note_launch() { ++g_prof.launches; }

void tddft::prof_begin(int c, cudaStream_t st) {
  if (!g_prof.on) return;
  const size_t need = 2 * (g_prof.used + 1);
  while (g_prof.pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      g_prof.on = false;
      return;
    }
    g_prof.pool.push_back(e);
  }
  cudaEventRecord(g_prof.pool[2 * g_prof.used], st);
  (void)c;
}

void tddft::prof_end(int c, cudaStream_t st, double bytes) {
  if (!g_prof.on) return;
  cudaEventRecord(g_prof.pool[2 * g_prof.used + 1], st);
  if (g_prof.cls.size() <= g_prof.used) {
    g_prof.cls.push_back(c);
    g_prof.bytes.push_back(bytes);
  } else {
    g_prof.cls[g_prof.used] = c;
    g_prof.bytes[g_prof.used] = bytes;
  }
  ++g_prof.used;
}

static int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (int)std::max(1LL, std::min(g, 148LL * 32));
}

// ---------------------------------------------------------------------------
// sphere and radix plans (host)
// ---------------------------------------------------------------------------
struct Miller {
  long long m2;
  int x, y, z;
};

static tddft_status build_sphere(int n, double a, double ecut, std::vector<Miller>& out) {
  if (n < 2 || (n & 1)) return fail(TDDFT_EINVAL, "grid size must be even and >= 2");
  if (!(a > 0.0) || !(ecut > 0.0)) return fail(TDDFT_EINVAL, "cell side and cutoff must be positive");
  const int h = n / 2;
  const double tpiba = 2.0 * M_PI / a;
  const double tpiba2 = tpiba * tpiba;
  out.clear();
  for (int z = -h; z < n - h; ++z)
    for (int y = -h; y < n - h; ++y)
      for (int x = -h; x < n - h; ++x) {
        const long long m2 = (long long)x * x + (long long)y * y + (long long)z * z;
        const double g2 = tpiba2 * (double)m2;
        if (0.5 * g2 < ecut) {
          if (std::abs(x) >= h || std::abs(y) >= h || std::abs(z) >= h)
            return fail(TDDFT_EINVAL, "wavefunction sphere does not fit inside the FFT grid");
          out.push_back({m2, x, y, z});
        }
      }
  std::sort(out.begin(), out.end(), [](const Miller& p, const Miller& q) {
    return std::tie(p.m2, p.x, p.y, p.z) < std::tie(q.m2, q.x, q.y, q.z);
  });
  return TDDFT_OK;
}

static std::vector<int> plan_radices(int n) {
  switch (n) {
#define TDDFT_CASE(NN) \
  case NN:             \
    return std::vector<int>(std::begin(Plan<NN>::r), std::end(Plan<NN>::r));
    TDDFT_CASE(8)
    TDDFT_CASE(12)
    TDDFT_CASE(16)
    TDDFT_CASE(24)
    TDDFT_CASE(32)
    TDDFT_CASE(36)
    TDDFT_CASE(48)
    TDDFT_CASE(64)
    TDDFT_CASE(72)
    TDDFT_CASE(80)
    TDDFT_CASE(96)
    TDDFT_CASE(108)
    TDDFT_CASE(128)
#undef TDDFT_CASE
    default:
      return {};
  }
}

// Position of frequency k after the in-place DIF stages of the plan.
static int dif_position(int k, const std::vector<int>& radices, int n) {
  int pos = 0, len = n, kk = k;
  for (int r : radices) {
    const int m = len / r;
    pos += m * (kk % r);
    kk /= r;
    len = m;
  }
  return pos;
}

// ---------------------------------------------------------------------------
// pointwise kernels used by the adjoint and Davidson
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_cast(const cplx<double>* __restrict__ in, cplx<T>* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = {(T)in[i].x, (T)in[i].y};
}

template <typename T>
__global__ void k_widen(const cplx<T>* __restrict__ in, cplx<double>* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = {(double)in[i].x, (double)in[i].y};
}

// out[r] = s * in[r] for real tables
template <typename T>
__global__ void k_real_cast(const double* __restrict__ in, T* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

// omega[b] = Re sum_i conj(p[b][i]) y[b][i], one block per b (FP64 accumulation)
template <typename T>
__global__ void k_bilinear(const cplx<T>* __restrict__ p, const cplx<T>* __restrict__ y, long long len,
                           double* __restrict__ omega) {
  __shared__ double red[256];
  const long long b = blockIdx.x;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    const cplx<T> u = p[b * len + i], v = y[b * len + i];
    acc += (double)u.x * (double)v.x + (double)u.y * (double)v.y;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) omega[b] = red[0];
}

// g[u](r) += w * p[u](r) * conj(W(r))   (u over nocc fields)
template <typename T>
__global__ void k_grad_k1e(const cplx<T>* __restrict__ p, const cplx<T>* __restrict__ W, cplx<T>* __restrict__ g,
                           int nocc, T w, long long n3) {
  const long long total = (long long)nocc * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i % n3;
    g[i] = cadd(g[i], cscale(cmul(p[i], cconj(W[r])), w));
  }
}

// W(r) += fxc(r) drho(r)   (fxc may be null)
template <typename T>
__global__ void k_add_fxc(cplx<T>* __restrict__ W, const T* __restrict__ fxc, const cplx<T>* __restrict__ drho,
                          long long n3) {
  if (!fxc) return;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n3; r += (long long)gridDim.x * blockDim.x)
    W[r] = cadd(W[r], cscale(drho[r], fxc[r]));
}

// gv[r] += s * sum_v |p[v](r)|^2
template <typename T>
__global__ void k_grad_vloc(const cplx<T>* __restrict__ p, int nocc, double s, double* __restrict__ gv, long long n3) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n3; r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int v = 0; v < nocc; ++v) {
      const cplx<T> u = p[(long long)v * n3 + r];
      acc += (double)u.x * (double)u.x + (double)u.y * (double)u.y;
    }
    gv[r] += s * acc;
  }
}

// Ct[k][u] = -w[k / nocc] * conj(C[u][k])   (C is [M][K])
template <typename T>
__global__ void k_proj_grad_coef(const cplx<T>* __restrict__ C, int M, int K, int nocc, const double* __restrict__ w,
                                 cplx<T>* __restrict__ Ct) {
  const long long total = (long long)M * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long u = i / K, k = i - u * K;
    const T s = (T)(-w[k / nocc]);
    const cplx<T> c = C[i];
    Ct[k * M + u] = {s * c.x, -s * c.y};
  }
}

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct Buffers {
  void* tw = nullptr;          // [n] twiddles
  void* kx = nullptr;          // [n^3] real, exchange kernel / N_r, position order
  void* kh = nullptr;          // [n^3] real, Hartree kernel / N_r
  int* pos = nullptr;          // [npw] cube position of each sphere point
  void* g2h = nullptr;         // [npw] real, |G|^2 / 2
  void* eps = nullptr;         // [nocc_src] real
  void* phi_src_pw = nullptr;  // [nocc_src][npw]
  void* phi_tgt_pw = nullptr;  // [nocc_tgt][npw] (aliases phi_src_pw for SC)
  cplx<double>* phi_tgt_pw64 = nullptr;  // FP64 copy for Davidson
  cplx<double>* phi_src_pw64 = nullptr;  // FP64 copy of the given (canonical) source orbitals
  void* phi_src_r = nullptr;   // [nocc_src][n^3]
  void* phi_tgt_r = nullptr;   // [nocc_tgt][n^3] (aliases for SC)
  void* vloc = nullptr;        // [n^3] real or null
  void* fxc = nullptr;         // [n^3] real or null
  void* a_r = nullptr;         // [nb_chunk*nocc_src][n^3]
  void* out_r = nullptr;       // [nb_chunk*nocc_src][n^3]
  void* drho = nullptr;        // [nb_chunk][n^3]
  void* wb = nullptr;          // [nb_chunk][n^3]
  void* ibuf = nullptr;        // [ibuf_fields][n^3]
  void* cpart = nullptr;       // projector split-K partials
  void* cmat = nullptr;        // projector overlaps [nocc_tgt][nb_max*nocc_src]
  void* ctmp = nullptr;        // [nb_max*nocc_src][nocc_tgt]
  void* io_a = nullptr;        // staging for host-buffer calls / adjoint [nb_max][nocc_src][npw]
  void* io_b = nullptr;
  void* grad_r = nullptr;      // [nocc_src][n^3] (adjoint)
  double* wdev = nullptr;      // [nb_max]
  int* dev_err = nullptr;      // set by a device wait that ran out of polls
  int* zcols = nullptr;        // [n*n] column positions, the ncols_act that a pair density can occupy first
  int* cmapT = nullptr;        // [n*n] compact index of position (x, y) at [x][y], -1 outside the disc
  void* kx_c = nullptr;        // [n][ncols_act] exchange kernel on those columns (compact pair densities)
  void* kh_c = nullptr;        // [n][ncols_act] Hartree kernel on those columns
  void* kx_p = nullptr;        // [n][ncols_act] exchange kernel in the order of the paired z pass
  void* kh_p = nullptr;        // [n][ncols_act] Hartree kernel in that order
};

struct tddft_system {
  tddft_desc d{};
  int npw = 0, n = 0;
  long long n3 = 0;
  int nb_chunk = 0;
  int ibuf_fields = 0;
  int tile_targets = 128, tile_sources = 8, k1d_block = 16;
  int accumulate = INV_ATOMIC;
  int projector_tc = 1;  // FP32 projector GEMMs on tcgen05 tensor cores (3xTF32): 1 packed operands with
                         // bulk copies where they fit, 2 operands staged through registers; 0: SIMT
  uint32_t* tc_pack = nullptr;  // packed TF32 operands of the tensor-core GEMMs (k_umma_pack)
  size_t tc_pack_words = 0;
  bool prune = true;     // pair convolutions keep only the columns a pair density can occupy (compact)
  int xy_lines = 1;      // compact xy passes on the register-line kernels where they exist (tuning.xy_kernel)
  // adaptively compressed exchange for the exchange term inside D (tddft_ace_build)
  bool ace_on = false;
  int n_ace = 0;
  void* ace_xi = nullptr;    // [n_ace][npw] working precision
  void* ace_c = nullptr;     // [n_ace][nb_max * nocc_src]
  void* ace_part = nullptr;  // split-K partials [2 * nsplit][n_ace][nb_max * nocc_src]
  // localised frame (tddft_set_localization): the handle's source orbitals are
  // phi~ = U^dagger phi, trial vectors are rotated in and results rotated out
  bool loc_on = false;
  int loc_kept = 0;
  void* loc_Uc = nullptr;    // [nocc][nocc]: C[v][n] = conj(U_vn)   (A~ = U^dagger A)
  void* loc_Ut = nullptr;    // [nocc][nocc]: C[n][v] = U_vn         (L A = U L~ A~)
  void* loc_E = nullptr;     // [nocc][nocc]: C[n'][n] = eps~_nn' = sum_v conj(U_vn) eps_v U_vn'
  void* loc_a = nullptr;     // [nb_max][nocc][npw] A~
  void* loc_b = nullptr;     // [nb_max][nocc][npw] L~ A~
  unsigned char* loc_keep = nullptr;        // device [nocc][nocc]
  std::vector<unsigned char> loc_keep_host;
  // kept unique pairs as batches of a pair list (k1d_sparse path)
  struct PairBatch {
    int pair0, np;   // slots [pair0, pair0 + np) of loc_list
    int rp0, nrows;  // row pointers loc_rowptr[rp0 .. rp0 + nrows], outputs loc_rowout[rp0 .. rp0 + nrows)
  };
  std::vector<PairBatch> loc_batches;
  int2* loc_list = nullptr;    // (q = n, r = m) per kept unique pair (m <= n)
  int* loc_rowptr = nullptr;
  int* loc_rowout = nullptr;
  int2* loc_ent = nullptr;     // (n << 1 | conj, slot)
  bool loc_sparse_auto = false;
  int k1d_sparse = 2;          // 0 blocks, 1 pair list, 2 automatic
  // K1d from stored tau (tuning.k1d_cache): tau_vv' of every unordered block pair of the source
  // orbitals, device-resident; built from the orbitals of the given frame
  bool k1d_cache = false;
  void* tau_cache = nullptr;
  size_t tau_cache_bytes = 0;
  bool k1d_cache_req = false;  // tuning.k1d_cache as set (the stored tau live where K1d runs)
  bool tau_cache_tiled = false;  // the stored tau are point-tiled (k_k1d_all reads them)
  // K1d of the recomputing path with the tau of every pair materialised in device scratch per
  // application (tuning.k1d_all), allocated at the first K1d outside stream capture when it fits
  bool k1d_all = true;
  bool tau_all_tried = false;
  void* tau_all = nullptr;
  size_t tau_all_bytes = 0;
  // Exchange terms (D_EXX, K1d, K2d) on a smaller grid on which they are exact (tuning.exchange_grid):
  // an internal system on that grid and its plane-wave results [nb_max][nocc_src][npw]
  tddft_system* xsub = nullptr;
  bool use_xsub = true;
  void* x_pw = nullptr;
  std::vector<double> eps64;  // the given eigenvalues
  int ncols_act = 0;     // number of such columns (0 = no list: the grid aliases pair densities)
  int nsplit = 1;
  size_t bytes = 0;
  Buffers b;
  // CUDA-graph replay of tddft_apply_liouville (tuning.graph): the launch
  // sequence is captured on the handle's own stream once per (nb, A, LA, mask)
  // and replayed on the caller's stream.
  bool use_graph = false;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_nb = -1;
  const void* g_A = nullptr;
  void* g_LA = nullptr;
  unsigned g_mask = 0;
  std::vector<void*> allocations;
  PlaneOps<float> ops32;
  PlaneOps<double> ops64;
  bool sf() const { return d.spin_mode == TDDFT_SPIN_FLIP; }
  size_t esz() const { return d.precision == TDDFT_PREC_FP64 ? 16 : 8; }
  size_t rsz() const { return d.precision == TDDFT_PREC_FP64 ? 8 : 4; }
};

template <typename T>
static PlaneOps<T>& ops_of(tddft_system* h);

// Compact pair-density columns for the three passes of a pair convolution
// (plane_kernels.cuh): given when pruning is on, the grid does not alias pair
// densities and the register-resident z pass runs; otherwise full planes.
template <typename T>
static ColumnList pair_columns(tddft_system* h) {
  ColumnList cl;
  const PlaneOps<T>& o = ops_of<T>(h);
  if (h->prune && h->b.zcols && ((o.reg_ok && o.kc.z >= 1) || (o.pair_ok && o.kc.z == 2))) {
    cl.cols = h->b.zcols;
    cl.nact = h->ncols_act;
    if (h->xy_lines && o.lines_ok) {
      // 1: one thread per line in both passes; 2: two lanes per line in both; 3: forward
      // pass one thread per line, inverse two lanes per line
      cl.cmapT = h->b.cmapT;
      cl.lanes_fwd = h->xy_lines == 2 ? 2 : 1;
      cl.lanes_inv = h->xy_lines == 1 ? 1 : 2;
    }
  }
  return cl;
}

// the convolution kernel in the layout of the column list (compact table when compact)
template <typename T>
static const T* pair_kernel(tddft_system* h, const T* kern, const ColumnList& cl) {
  if (!cl.cols) return kern;
  const PlaneOps<T>& o = ops_of<T>(h);
  const bool paired = o.pair_ok && o.kc.z == 2 && h->b.kx_p;
  if (kern == (const T*)h->b.kx) return (const T*)(paired ? h->b.kx_p : h->b.kx_c);
  if (kern == (const T*)h->b.kh) return (const T*)(paired ? h->b.kh_p : h->b.kh_c);
  return kern;
}

static tddft_status dalloc(tddft_system* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return TDDFT_OK;
  cudaError_t e = lib_malloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TDDFT_ENOMEM, alloc_error(bytes, e));
  }
  h->allocations.push_back(*p);
  h->bytes += bytes;
  return TDDFT_OK;
}

namespace {
// temporaries of one call, released on every exit path
struct TempAllocs {
  std::vector<void*> p;
  tddft_status get(void** out, size_t bytes) {
    cudaError_t e = lib_malloc(out, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *out = nullptr;
      return fail(TDDFT_ENOMEM, alloc_error(bytes, e));
    }
    p.push_back(*out);
    return TDDFT_OK;
  }
  ~TempAllocs() {
    for (void* q : p) cudaFree(q);
  }
};
}  // namespace

template <typename T>
static PlaneOps<T>& ops_of(tddft_system* h);
template <>
PlaneOps<float>& ops_of<float>(tddft_system* h) { return h->ops32; }
template <>
PlaneOps<double>& ops_of<double>(tddft_system* h) { return h->ops64; }

// ---------------------------------------------------------------------------
// building blocks of the apply (templated on the working precision)
// ---------------------------------------------------------------------------

// real-space fields dst[f] (f < nf) from plane-wave rows src[f] (Omega^{-1/2} normalisation)
template <typename T>
static tddft_status pw_to_real(tddft_system* h, const cplx<T>* src, int nf, cplx<T>* dst, cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  cplx<T>* ib = (cplx<T>*)h->b.ibuf;
  const T s = (T)(1.0 / std::sqrt(h->d.a * h->d.a * h->d.a));
  for (int f0 = 0; f0 < nf; f0 += h->ibuf_fields) {
    const int cnt = std::min(h->ibuf_fields, nf - f0);
    CUDA_TRY(cudaMemsetAsync(ib, 0, (size_t)cnt * h->n3 * sizeof(cplx<T>), st));
    { k_scatter<T><<<grid_for((long long)cnt * h->npw, 256), 256, 0, st>>>(src + (long long)f0 * h->npw, ib, h->b.pos,
                                                                         h->npw, cnt, s, h->n3); note_launch(); }
    o.z(Z_INV, ib, cnt, nullptr, T(1), tw, st);
    PairMap pm{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, f0, 1};
    o.xy_inv(INV_WRITE, ib, dst, nullptr, pm, cnt, T(1), tw, st);
  }
  return check_launch("pw_to_real");
}

// plane-wave rows dst[f] = Omega^{1/2}/N_r F[src[f]] on the sphere, plus the
// diagonal term (|G|^2/2 - eps_v) A[f] when A is given (v = (f0 + f) % nocc_src).
template <typename T>
static tddft_status real_to_pw(tddft_system* h, const cplx<T>* src, int nf, cplx<T>* dst, const cplx<T>* A,
                               cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  cplx<T>* ib = (cplx<T>*)h->b.ibuf;
  const T s = (T)(std::sqrt(h->d.a * h->d.a * h->d.a) / (double)h->n3);
  for (int f0 = 0; f0 < nf; f0 += h->ibuf_fields) {
    const int cnt = std::min(h->ibuf_fields, nf - f0);
    PairMap pm{1, 0, 0, 0, f0, 0, 1, 0, 0, 0, 0, 0};
    o.xy_fwd(XY_LOAD, nullptr, src, pm, cnt, ib, tw, st);
    o.z(Z_FWD, ib, cnt, nullptr, T(1), tw, st);
    { k_gather<T><<<grid_for((long long)cnt * h->npw, 256), 256, 0, st>>>(
        ib, h->b.pos, h->npw, cnt, s, A ? A + (long long)f0 * h->npw : nullptr, (const T*)h->b.g2h,
        h->loc_on ? nullptr : (const T*)h->b.eps, h->d.nocc_src, f0, dst + (long long)f0 * h->npw, h->n3); note_launch(); }
  }
  return check_launch("real_to_pw");
}

// Y[n][:] -= sum_m Phi[m][:] <Phi_m|Y_n>  for nrows rows of length npw
// Complex GEMMs on tcgen05 tensor cores (FP32 data, 3xTF32 products, FP32 accumulation).
// At most 256 chunks of 32 real K values (8192 products) accumulate in one TMEM
// accumulator chain: the accumulator's rounding error grows about linearly with
// the chain length (measured: 3e-5 relative on a projected 49k-plane-wave row with
// one split of the whole K, 4e-6 with nine), so long K is always split.
constexpr int TC_CHAIN_CHUNKS = 256;

// Packed operands of the tensor-core GEMMs: words for mt + nt row blocks of kchunks K chunks
// (high and low tiles), at most TC_PACK_MAX_WORDS; the buffer grows on demand outside stream
// capture (otherwise, and beyond the limit, the GEMM stages its operands through registers).
constexpr size_t TC_PACK_MAX_WORDS = (size_t)1 << 28;  // 1 GiB
static size_t tc_pack_words(int mt, int nt, int kchunks) {
  return (size_t)(mt + nt) * kchunks * 2 * UMMA_TILE_WORDS;
}
static bool tc_pack_ready(tddft_system* h, size_t words, cudaStream_t st) {
  if (words > TC_PACK_MAX_WORDS) return false;
  if (words <= h->tc_pack_words) return true;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  if (h->tc_pack) {
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaFree(h->tc_pack) != cudaSuccess) {
      cudaGetLastError();
      h->tc_pack = nullptr;
      h->bytes -= h->tc_pack_words * 4;
      h->tc_pack_words = 0;
      return false;
    }
    h->bytes -= h->tc_pack_words * 4;
    h->tc_pack = nullptr;
    h->tc_pack_words = 0;
  }
  if (lib_malloc((void**)&h->tc_pack, words * 4) != cudaSuccess) {
    cudaGetLastError();
    h->tc_pack = nullptr;
    return false;
  }
  h->tc_pack_words = words;
  h->bytes += words * 4;
  return true;
}

// overlap: C[u][r] = sum_g conj(P[u][g]) Y[r][g]   (C: [M][nrows], split-K partials in part)

static tddft_status tc_overlap(tddft_system* h, const cplx<float>* P, int M, const cplx<float>* Y, int nrows,
                               cplx<float>* part, int max_splits, cplx<float>* C, cudaStream_t st) {
  const int K = h->npw;
  const int Kp = (K + UMMA_KC - 1) / UMMA_KC * UMMA_KC;
  const int Rp = (nrows + UMMA_N - 1) / UMMA_N * UMMA_N;
  const int kchunks = 2 * Kp / UMMA_KC;
  const int mt = (M + UMMA_M - 1) / UMMA_M;
  const int nt = 2 * Rp / UMMA_N;
  const int min_splits = (kchunks + TC_CHAIN_CHUNKS - 1) / TC_CHAIN_CHUNKS;
  int splits = std::max(min_splits, std::min(kchunks, 296 / std::max(1, nt * mt)));
  splits = std::max(1, std::min(splits, max_splits));
  const int per = (kchunks + splits - 1) / splits;
  splits = (kchunks + per - 1) / per;
  OvA la{P, M, K, Kp};
  OvB lb{Y, nrows, Rp, K, Kp};
  OvEp ep{part, M, nrows, Rp};
  if (h->projector_tc == 1 && tc_pack_ready(h, tc_pack_words(mt, nt, kchunks), st)) {
    uint32_t* pa = h->tc_pack;
    uint32_t* pb = pa + (size_t)mt * kchunks * 2 * UMMA_TILE_WORDS;
    { k_umma_pack<OvA><<<dim3(kchunks, mt), 256, 0, st>>>(la, kchunks, pa); note_launch(); }
    { k_umma_pack<OvB><<<dim3(kchunks, nt), 256, 0, st>>>(lb, kchunks, pb); note_launch(); }
    { k_umma_tiles<OvEp><<<dim3(nt, mt, splits), 128, UMMA_TILES_SMEM, st>>>(pa, pb, ep, kchunks, per, h->b.dev_err);
      note_launch(); }
  } else {
    k_umma_gemm<OvA, OvB, OvEp><<<dim3(nt, mt, splits), 128, UMMA_SMEM, st>>>(la, lb, ep, kchunks, per, h->b.dev_err);
    note_launch();
  }
  { k_reduce_split<float><<<grid_for((long long)M * nrows, 256), 256, 0, st>>>(part, splits, (long long)M * nrows, C); note_launch(); }
  return check_launch("overlap (tensor cores)");
}

// update: Y[r][g] += s * sum_u P[u][g] C[u][r]
static tddft_status tc_update(tddft_system* h, const cplx<float>* P, int M, const cplx<float>* C, cplx<float>* Y,
                              int nrows, float s, cudaStream_t st) {
  const int K = h->npw;
  const int Up = (M + UMMA_KC - 1) / UMMA_KC * UMMA_KC;
  const int Gp = (K + UMMA_N - 1) / UMMA_N * UMMA_N;
  UpA la{C, M, Up, nrows};
  UpB lb{P, M, Up, K, Gp};
  UpEp ep{Y, nrows, K, Gp, s};
  const int kc2 = 2 * Up / UMMA_KC;
  const int nt = 2 * Gp / UMMA_N, mt = (nrows + UMMA_M - 1) / UMMA_M;
  if (h->projector_tc == 1 && tc_pack_ready(h, tc_pack_words(mt, nt, kc2), st)) {
    uint32_t* pa = h->tc_pack;
    uint32_t* pb = pa + (size_t)mt * kc2 * 2 * UMMA_TILE_WORDS;
    { k_umma_pack<UpA><<<dim3(kc2, mt), 256, 0, st>>>(la, kc2, pa); note_launch(); }
    { k_umma_pack<UpB><<<dim3(kc2, nt), 256, 0, st>>>(lb, kc2, pb); note_launch(); }
    { k_umma_tiles<UpEp><<<dim3(nt, mt, 1), 128, UMMA_TILES_SMEM, st>>>(pa, pb, ep, kc2, kc2, h->b.dev_err);
      note_launch(); }
  } else {
    k_umma_gemm<UpA, UpB, UpEp><<<dim3(nt, mt, 1), 128, UMMA_SMEM, st>>>(la, lb, ep, kc2, kc2, h->b.dev_err);
    note_launch();
  }
  return check_launch("update (tensor cores)");
}

// C[u][r] = sum_g conj(P[u][g]) Y[r][g] for u < M, r < nrows (tensor cores for FP32 when enabled)
template <typename T>
static tddft_status gemm_overlap(tddft_system* h, const cplx<T>* P, int M, const cplx<T>* Y, int nrows, cplx<T>* part,
                                 cplx<T>* C, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (h->projector_tc) return tc_overlap(h, P, M, Y, nrows, part, 2 * h->nsplit, C, st);
  }
  const int K = h->npw;
  const int nsplit = h->nsplit;
  const int kchunk = ((K + nsplit - 1) / nsplit + 15) / 16 * 16;
  dim3 g1((M + 31) / 32, (nrows + 31) / 32, nsplit);
  { k_overlap<T><<<g1, 256, 0, st>>>(P, M, Y, nrows, K, kchunk, part); note_launch(); }
  { k_reduce_split<T><<<grid_for((long long)M * nrows, 256), 256, 0, st>>>(part, nsplit, (long long)M * nrows, C); note_launch(); }
  return check_launch("overlap");
}

// Y[r][g] += s * sum_u P[u][g] C[u][r]
template <typename T>
static tddft_status gemm_update(tddft_system* h, const cplx<T>* P, int M, const cplx<T>* C, cplx<T>* Y, int nrows,
                                T s, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (h->projector_tc) return tc_update(h, P, M, C, Y, nrows, s, st);
  }
  const int K = h->npw;
  dim3 g2((K + 63) / 64, (nrows + 31) / 32);
  { k_update<T><<<g2, 256, 0, st>>>(P, M, C, nrows, K, s, Y); note_launch(); }
  return check_launch("update");
}

// Y[n][:] -= sum_m Phi[m][:] <Phi_m|Y_n>  for nrows rows of length npw
template <typename T>
static tddft_status project_rows(tddft_system* h, const cplx<T>* phi, int M, cplx<T>* Y, int nrows, cudaStream_t st) {
  if (nrows <= 0 || M <= 0) return TDDFT_OK;
  cplx<T>* C = (cplx<T>*)h->b.cmat;
  STATUS_TRY(gemm_overlap<T>(h, phi, M, Y, nrows, (cplx<T>*)h->b.cpart, C, st));
  return gemm_update<T>(h, phi, M, C, Y, nrows, T(-1), st);
}

// Conv_kappa of nf fields src[f] into dst[f] (dst may equal src)
template <typename T>
static tddft_status convolve_fields(tddft_system* h, const cplx<T>* src, int nf, const T* kern, T kscale, cplx<T>* dst,
                                    cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  cplx<T>* ib = (cplx<T>*)h->b.ibuf;
  for (int f0 = 0; f0 < nf; f0 += h->ibuf_fields) {
    const int cnt = std::min(h->ibuf_fields, nf - f0);
    PairMap pin{1, 0, 0, 0, f0, 0, 1, 0, 0, 0, 0, 0};
    // the fields are pair-density sums (Delta rho): compact when pruning; dst may equal src, never ib
    const ColumnList cl = pair_columns<T>(h);
    o.xy_fwd(XY_LOAD, nullptr, src, pin, cnt, ib, tw, st, cl);
    o.z(Z_CONV, ib, cnt, pair_kernel<T>(h, kern, cl), kscale, tw, st, cl);
    PairMap pout{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, f0, 1};
    o.xy_inv(INV_WRITE, ib, dst, nullptr, pout, cnt, T(1), tw, st, cl);
  }
  return check_launch("convolve_fields");
}

// out[o0 + t*ot] += scale * sum_k P_(t,k) Conv_x[conj(Q_(t,k)) R_(t,k)] over a grid of
// ntargets x nsources pairs, tiled into batches that fit the intermediate buffer.
// qm/rm/pm give the affine field maps in terms of (t, k) relative to the tile origin.
struct PairGrid {
  int ntargets, nsources;
  // field index = base + k * ks + t * ts
  int q_base, q_ks, q_ts;
  int r_base, r_ks, r_ts;
  int p_base, p_ks, p_ts;
  int o_base, o_ts;
};

template <typename T>
static tddft_status pair_accumulate(tddft_system* h, const cplx<T>* qb, const cplx<T>* rb, const cplx<T>* pb,
                                    cplx<T>* ob, const PairGrid& pg, const T* kern, T scale, cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  cplx<T>* ib = (cplx<T>*)h->b.ibuf;
  const ColumnList cl = pair_columns<T>(h);  // pair densities: compact intermediates when pruning
  int TT = std::max(1, std::min(h->tile_targets, pg.ntargets));
  int KS = std::max(1, std::min(h->tile_sources, pg.nsources));
  while (TT * KS > h->ibuf_fields) {  // shrink the targets to 32 first, then the sources
    if (TT > 32) TT = (TT + 1) / 2;
    else if (KS > 1) KS = (KS + 1) / 2;
    else TT = (TT + 1) / 2;
  }
  for (int t0 = 0; t0 < pg.ntargets; t0 += TT) {
    const int tt = std::min(TT, pg.ntargets - t0);
    for (int k0 = 0; k0 < pg.nsources; k0 += KS) {
      const int kk = std::min(KS, pg.nsources - k0);
      PairMap pm;
      pm.kdim = kk;
      pm.q0 = pg.q_base + k0 * pg.q_ks + t0 * pg.q_ts;
      pm.qk = pg.q_ks;
      pm.qt = pg.q_ts;
      pm.r0 = pg.r_base + k0 * pg.r_ks + t0 * pg.r_ts;
      pm.rk = pg.r_ks;
      pm.rt = pg.r_ts;
      pm.p0 = pg.p_base + k0 * pg.p_ks + t0 * pg.p_ts;
      pm.pk = pg.p_ks;
      pm.pt = pg.p_ts;
      pm.o0 = pg.o_base + t0 * pg.o_ts;
      pm.ot = pg.o_ts;
      o.xy_fwd(XY_PRODUCT, qb, rb, pm, tt * kk, ib, tw, st, cl);
      o.z(Z_CONV, ib, tt * kk, pair_kernel<T>(h, kern, cl), T(1), tw, st, cl);
      o.xy_inv(h->accumulate, ib, ob, pb, pm, tt, scale, tw, st, cl);
    }
  }
  return check_launch("pair_accumulate");
}

// K1d: out[b][v] -= alpha sum_v' a[b][v'] Conv_x[conj(phi_v') phi_v], tau computed once per
// unordered block pair (I <= J) and shared by every b of the chunk.
// pair-list K1d: points per CTA and the largest batch whose tau values fit in shared memory
constexpr int K1D_SPARSE_PTS = 32;
template <typename T>
constexpr int k1d_sparse_np_max() { return sizeof(T) == 4 ? 384 : 192; }

// Stored tau: Conv_x[conj(phi_v') phi_v] of every unordered block pair (I <= J) of
// K1D_CACHE_BLOCK source orbitals, block pair after block pair (I, then J), each block pair
// in the field order k_k1d_contract reads (vi * tj + vj). The tau depend on the occupied
// orbitals only, so one build serves every application.
constexpr int K1D_CACHE_BLOCK = 16;

static size_t tau_cache_fields(int nocc) {
  size_t f = 0;
  for (int i0 = 0; i0 < nocc; i0 += K1D_CACHE_BLOCK) {
    const int ti = std::min(K1D_CACHE_BLOCK, nocc - i0);
    for (int j0 = i0; j0 < nocc; j0 += K1D_CACHE_BLOCK) f += (size_t)ti * std::min(K1D_CACHE_BLOCK, nocc - j0);
  }
  return f;
}

// tau_vv' = Conv_x[conj(phi_v') phi_v] of every unordered 16 x 16 block pair of the source
// orbitals (I <= J, block pair after block pair, field vi * tj + vj; diagonal blocks in both
// orders) into dst. Plain layout: field after field. Point-tiled layout (tiled; only with the
// register-line inverse pass of compact intermediates, see PairMap::tile_nf): the values of
// all fields at POINT_TILE consecutive points follow each other.
template <typename T>
static tddft_status build_tau_fields(tddft_system* h, void* dst, bool tiled, cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  const cplx<T>* phi = (const cplx<T>*)h->b.phi_src_r;
  const int nocc = h->d.nocc_src;
  cplx<T>* blk = (cplx<T>*)dst;
  const ColumnList cl = pair_columns<T>(h);
  if (tiled && !(cl.cols && cl.cmapT)) return fail(TDDFT_EINVAL, "point-tiled tau need the register-line passes");
  const long long nf = (long long)tau_cache_fields(nocc);
  long long f0 = 0;
  for (int i0 = 0; i0 < nocc; i0 += K1D_CACHE_BLOCK) {
    const int ti = std::min(K1D_CACHE_BLOCK, nocc - i0);
    for (int j0 = i0; j0 < nocc; j0 += K1D_CACHE_BLOCK) {
      const int tj = std::min(K1D_CACHE_BLOCK, nocc - j0);
      // the pair convolutions of k1d_term, written straight into the block pair's slot
      // (through compact intermediates in the pair buffer when the grid allows them)
      PairMap pm{tj, j0, 1, 0, i0, 0, 1, 0, 0, 0, 0, 1};
      PairMap pw{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
      if (cl.cols && ti * tj <= h->ibuf_fields) {
        cplx<T>* ib = (cplx<T>*)h->b.ibuf;
        o.xy_fwd(XY_PRODUCT, phi, phi, pm, ti * tj, ib, tw, st, cl);
        o.z(Z_CONV, ib, ti * tj, pair_kernel<T>(h, (const T*)h->b.kx, cl), T(1), tw, st, cl);
        if (tiled) {
          pw.o0 = (int)f0;
          pw.tile_nf = nf;
          o.xy_inv(INV_WRITE, ib, (cplx<T>*)dst, nullptr, pw, ti * tj, T(1), tw, st, cl);
        } else {
          o.xy_inv(INV_WRITE, ib, blk, nullptr, pw, ti * tj, T(1), tw, st, cl);
        }
      } else {
        if (tiled) return fail(TDDFT_EINVAL, "point-tiled tau need compact intermediates");
        o.xy_fwd(XY_PRODUCT, phi, phi, pm, ti * tj, blk, tw, st);
        o.z(Z_CONV, blk, ti * tj, (const T*)h->b.kx, T(1), tw, st);
        o.xy_inv(INV_WRITE, blk, blk, nullptr, pw, ti * tj, T(1), tw, st);
      }
      blk += (long long)ti * tj * h->n3;
      f0 += (long long)ti * tj;
    }
  }
  return check_launch("tau build");
}

// the point-tiled tau of every pair and their one-pass contraction (k_k1d_all) apply: FP32, at
// most 128 source orbitals, the register-line passes of compact intermediates, whole point tiles
template <typename T>
static bool k1d_all_layout_ok(tddft_system* h) {
  const ColumnList cl = pair_columns<T>(h);
  return sizeof(T) == 4 && h->d.nocc_src <= K1D_ALL_ROWS && cl.cols && cl.cmapT &&
         K1D_CACHE_BLOCK * K1D_CACHE_BLOCK <= h->ibuf_fields && h->n3 % K1D_ALL_PTS == 0;
}

// stored tau: point-tiled (contracted by k_k1d_all) where that layout applies, else block pair
// after block pair (contracted by k_k1d_contract)
template <typename T>
static tddft_status build_tau_cache(tddft_system* h, cudaStream_t st) {
  h->tau_cache_tiled = k1d_all_layout_ok<T>(h);
  return build_tau_fields<T>(h, h->tau_cache, h->tau_cache_tiled, st);
}

// the round-robin schedule of the all-pairs K1d contraction (k_k1d_all) and the
// field offsets of the block pairs in the tau layout of build_tau_fields
static K1dAll k1d_all_table(int nocc) {
  K1dAll t{};
  const int nblk = (nocc + K1D_CACHE_BLOCK - 1) / K1D_CACHE_BLOCK;
  t.nblk = nblk;
  long long f = 0;
  for (int i = 0; i < nblk; ++i)
    for (int j = i; j < nblk; ++j) {
      t.off[i][j] = f;
      f += (long long)std::min(K1D_CACHE_BLOCK, nocc - i * K1D_CACHE_BLOCK) *
           std::min(K1D_CACHE_BLOCK, nocc - j * K1D_CACHE_BLOCK);
    }
  t.nf = f;
  const int M = nblk + (nblk & 1), m1 = M - 1;
  t.rounds = nblk >= 2 ? m1 : 0;
  for (int r = 0; r < K1D_ALL_BLOCKS; ++r)
    for (int b = 0; b < K1D_ALL_BLOCKS; ++b) {
      t.partner[r][b] = -1;
      t.slot[r][b] = 0;
      t.first[r][b] = 0;
      if (b < K1D_ALL_BLOCKS / 2) t.pi[r][b] = t.pj[r][b] = -1;
    }
  for (int r = 0; r < t.rounds; ++r)
    for (int k = 0; k < M / 2; ++k) {
      int p = k == 0 ? M - 1 : (r + k) % m1, q = k == 0 ? r : (r - k + m1) % m1;
      const int I = std::min(p, q), J = std::max(p, q);
      if (J >= nblk) continue;
      t.pi[r][k] = (signed char)I;
      t.pj[r][k] = (signed char)J;
      t.partner[r][I] = (signed char)J;
      t.slot[r][I] = (signed char)k;
      t.first[r][I] = 1;
      t.partner[r][J] = (signed char)I;
      t.slot[r][J] = (signed char)k;
      t.first[r][J] = 0;
    }
  return t;
}

template <int NB>
static constexpr size_t k1d_all_smem() {
  return 128 + ((size_t)NB * K1D_ALL_ROWS * K1D_ALL_PTS + (size_t)2 * (K1D_ALL_BLOCKS / 2) * K1D_ALL_SLOT) *
                   sizeof(cplx<float>);
}

// K1d from point-tiled tau of every pair (k_k1d_all), trial vectors in groups of up to 8
static tddft_status k1d_all_launch(tddft_system* h, const cplx<float>* tau, int nbc, cudaStream_t st) {
  const int nocc = h->d.nocc_src;
  const K1dAll kt = k1d_all_table(nocc);
  const unsigned blocks = (unsigned)(h->n3 / K1D_ALL_PTS);
  const float s = (float)(-h->d.alpha);
  const cplx<float>* a = (const cplx<float>*)h->b.a_r;
  cplx<float>* out = (cplx<float>*)h->b.out_r;
  // the smallest group of trial vectors that covers nbc (one pass when nbc <= 8)
  const int nbg = nbc <= 1 ? 1 : nbc <= 2 ? 2 : nbc <= 4 ? 4 : 8;
#define TDDFT_K1D_ALL(NBG)                                                                                   \
  {                                                                                                          \
    constexpr size_t smem = k1d_all_smem<NBG>();                                                             \
    CUDA_TRY(cudaFuncSetAttribute(k_k1d_all<NBG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));  \
    k_k1d_all<NBG><<<blocks, K1D_ALL_THREADS, smem, st>>>(tau, kt, a, out, nocc, nbc, s, h->n3, h->b.dev_err); \
    note_launch();                                                                                           \
  }
  if (nbg == 1) TDDFT_K1D_ALL(1)
  else if (nbg == 2) TDDFT_K1D_ALL(2)
  else if (nbg == 4) TDDFT_K1D_ALL(4)
  else TDDFT_K1D_ALL(8)
#undef TDDFT_K1D_ALL
  return check_launch("k1d (all pairs)");
}

template <typename T>
static tddft_status k1d_term(tddft_system* h, int nbc, cudaStream_t st) {
  PlaneOps<T>& o = ops_of<T>(h);
  const cplx<T>* tw = (const cplx<T>*)h->b.tw;
  cplx<T>* ib = (cplx<T>*)h->b.ibuf;
  const cplx<T>* phi = (const cplx<T>*)h->b.phi_src_r;
  const int nocc = h->d.nocc_src;
  int TB = std::min(h->k1d_block, nocc);
  while (TB * TB > h->ibuf_fields) --TB;
  const T s = (T)(-h->d.alpha);
  if (h->loc_on && (h->k1d_sparse == 1 || (h->k1d_sparse == 2 && h->loc_sparse_auto))) {
    // only the kept pairs: tau of each batch of the pair list, then the row-wise contraction
    for (const auto& pb : h->loc_batches) {
      PairMap pm{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
      pm.list = h->loc_list + pb.pair0;
      o.xy_fwd(XY_PRODUCT, phi, phi, pm, pb.np, ib, tw, st);
      o.z(Z_CONV, ib, pb.np, (const T*)h->b.kx, T(1), tw, st);  // full planes: the inverse runs in place
      PairMap pw{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
      o.xy_inv(INV_WRITE, ib, ib, nullptr, pw, pb.np, T(1), tw, st);
      const size_t smem = (size_t)pb.np * K1D_SPARSE_PTS * sizeof(cplx<T>);
      const unsigned blocks = (unsigned)((h->n3 + K1D_SPARSE_PTS - 1) / K1D_SPARSE_PTS);
      { k_k1d_sparse<T, K1D_SPARSE_PTS><<<blocks, K1D_THREADS, smem, st>>>(
          ib, pb.np, (const cplx<T>*)h->b.a_r, (cplx<T>*)h->b.out_r, h->loc_rowptr + pb.rp0, h->loc_rowout + pb.rp0,
          pb.nrows, h->loc_ent, nocc, nbc, s, h->n3); note_launch(); }
    }
    return check_launch("k1d_term (pair list)");
  }
  // the tau of every pair at once: FP32, register-line passes of compact intermediates
  // (point-tiled tau), at most 128 orbitals, recomputing path
  const bool all_ok = h->k1d_all && !h->loc_on && !h->k1d_cache && k1d_all_layout_ok<T>(h);
  if (all_ok) {
    if (!h->tau_all && !h->tau_all_tried) {
      // scratch for the tau of every pair: allocated once, outside stream capture, when it
      // takes at most a quarter of the free device memory
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      CUDA_TRY(cudaStreamIsCapturing(st, &cs));
      if (cs == cudaStreamCaptureStatusNone) {
        h->tau_all_tried = true;
        const size_t bytes = tau_cache_fields(nocc) * (size_t)h->n3 * sizeof(cplx<T>);
        size_t freeb = 0, totalb = 0;
        CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
        if (bytes <= freeb / 4) {
          if (lib_malloc(&h->tau_all, bytes) == cudaSuccess) {
            h->tau_all_bytes = bytes;
            h->bytes += bytes;
          } else {
            cudaGetLastError();
            h->tau_all = nullptr;
          }
        }
      }
    }
    if (h->tau_all) {
      STATUS_TRY(build_tau_fields<T>(h, h->tau_all, true, st));
      if constexpr (sizeof(T) == 4) return k1d_all_launch(h, (const cplx<float>*)h->tau_all, nbc, st);
    }
  }
  if (h->k1d_cache && h->tau_cache && !h->loc_on && h->tau_cache_tiled) {
    // stored point-tiled tau: the one-pass contraction alone
    if constexpr (sizeof(T) == 4) return k1d_all_launch(h, (const cplx<float>*)h->tau_cache, nbc, st);
  }
  if (h->k1d_cache && h->tau_cache && !h->loc_on && !h->tau_cache_tiled) {
    // stored tau: the contraction alone, block pair after block pair in the build order
    const cplx<T>* blk = (const cplx<T>*)h->tau_cache;
    for (int i0 = 0; i0 < nocc; i0 += K1D_CACHE_BLOCK) {
      const int ti = std::min(K1D_CACHE_BLOCK, nocc - i0);
      for (int j0 = i0; j0 < nocc; j0 += K1D_CACHE_BLOCK) {
        const int tj = std::min(K1D_CACHE_BLOCK, nocc - j0);
        constexpr int KB = K1D_CACHE_BLOCK, PTS = 32;
        const size_t smem = (size_t)KB * KB * PTS * sizeof(cplx<T>);
        const unsigned blocks = (unsigned)((h->n3 + PTS - 1) / PTS);
        { k_k1d_contract<T, KB, PTS><<<blocks, K1D_THREADS, smem, st>>>(
            blk, (const cplx<T>*)h->b.a_r, (cplx<T>*)h->b.out_r, i0, ti, j0, tj, nocc, nbc, s, h->n3, nullptr); note_launch(); }
        blk += (long long)ti * tj * h->n3;
      }
    }
    return check_launch("k1d_term (stored tau)");
  }
  // truncated pairs of the localised frame: blocks without a kept pair are skipped
  const unsigned char* keep = h->loc_on ? h->loc_keep : nullptr;
  // compact pair-density intermediates when the grid allows them and the pair buffer holds
  // both the intermediates and the tau fields of a block pair
  const ColumnList ccl = pair_columns<T>(h);
  const bool compact = ccl.cols && 2 * TB * TB <= h->ibuf_fields;
  auto block_kept = [&](int i0, int ti, int j0, int tj) {
    for (int i = i0; i < i0 + ti; ++i)
      for (int j = j0; j < j0 + tj; ++j)
        if (h->loc_keep_host[(size_t)i * nocc + j]) return true;
    return false;
  };
  for (int i0 = 0; i0 < nocc; i0 += TB) {
    const int ti = std::min(TB, nocc - i0);
    for (int j0 = i0; j0 < nocc; j0 += TB) {
      const int tj = std::min(TB, nocc - j0);
      if (keep && !block_kept(i0, ti, j0, tj)) continue;
      // item = vi * tj + vj : Q = phi[j0 + vj], R = phi[i0 + vi]
      PairMap pm{tj, j0, 1, 0, i0, 0, 1, 0, 0, 0, 0, 1};
      PairMap pw{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
      const cplx<T>* tau = ib;
      if (compact) {
        // compact intermediates in the first half of the pair buffer, tau in the second
        cplx<T>* taub = ib + (long long)TB * TB * h->n3;
        o.xy_fwd(XY_PRODUCT, phi, phi, pm, ti * tj, ib, tw, st, ccl);
        o.z(Z_CONV, ib, ti * tj, pair_kernel<T>(h, (const T*)h->b.kx, ccl), T(1), tw, st, ccl);
        o.xy_inv(INV_WRITE, ib, taub, nullptr, pw, ti * tj, T(1), tw, st, ccl);
        tau = taub;
      } else {
        o.xy_fwd(XY_PRODUCT, phi, phi, pm, ti * tj, ib, tw, st);
        o.z(Z_CONV, ib, ti * tj, (const T*)h->b.kx, T(1), tw, st);  // full planes: the inverse runs in place
        o.xy_inv(INV_WRITE, ib, ib, nullptr, pw, ti * tj, T(1), tw, st);
      }
      {
        constexpr int KB = 16, PTS = 32;
        const size_t smem = (size_t)KB * KB * PTS * sizeof(cplx<T>);
        const unsigned blocks = (unsigned)((h->n3 + PTS - 1) / PTS);
        { k_k1d_contract<T, KB, PTS><<<blocks, K1D_THREADS, smem, st>>>(
            tau, (const cplx<T>*)h->b.a_r, (cplx<T>*)h->b.out_r, i0, ti, j0, tj, nocc, nbc, s, h->n3, keep); note_launch(); }
      }
    }
  }
  return check_launch("k1d_term");
}

// y += x (element-wise)
template <typename T>
__global__ void k_accumulate(cplx<T>* __restrict__ y, const cplx<T>* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = cadd(y[i], x[i]);
}

// (L A) for nb trial vectors in the handle's orbital frame; terms of `mask`
// (PROJ bit included or not). In the localised frame the eigenvalue part of D
// is left out here (it is a matrix there, added by apply_impl).
template <typename T>
static tddft_status apply_core(tddft_system* h, int nb, const cplx<T>* A, cplx<T>* LA, unsigned mask, cudaStream_t st) {
  const int nocc = h->d.nocc_src, npw = h->npw;
  const long long n3 = h->n3;
  const cplx<T>* phis = (const cplx<T>*)h->b.phi_src_r;
  const cplx<T>* phit = (const cplx<T>*)h->b.phi_tgt_r;
  cplx<T>* a_r = (cplx<T>*)h->b.a_r;
  cplx<T>* out_r = (cplx<T>*)h->b.out_r;
  cplx<T>* drho = (cplx<T>*)h->b.drho;
  cplx<T>* wb = (cplx<T>*)h->b.wb;
  if (h->sf() && (mask & (TDDFT_TERM_K2E_H | TDDFT_TERM_K2E_XC | TDDFT_TERM_K2D)))
    return fail(TDDFT_ENOTSUP, "K2 terms are implemented for spin-conserving systems");
  // Hartree and xc parts of K1e (W) and K2e (conj W); spin-flip has no Hartree part
  const int hmode = (((mask & TDDFT_TERM_K1E_H) && !h->sf()) ? 1 : 0) | ((mask & TDDFT_TERM_K2E_H) ? 2 : 0);
  const int xmode = h->b.fxc ? (((mask & TDDFT_TERM_K1E_XC) ? 1 : 0) | ((mask & TDDFT_TERM_K2E_XC) ? 2 : 0)) : 0;
  const bool vloc = (mask & TDDFT_TERM_D_VLOC) && h->b.vloc;
  // the pair-convolution terms on the exchange grid: same plane-wave result, fewer points
  unsigned xmask = 0;
  if (h->xsub && h->use_xsub && h->xsub->loc_on == h->loc_on && h->d.alpha != 0.0) {
    xmask = mask & (TDDFT_TERM_K1D | TDDFT_TERM_K2D | (h->ace_on ? 0u : TDDFT_TERM_D_EXX));
    if (xmask) STATUS_TRY(apply_core<T>(h->xsub, nb, A, (cplx<T>*)h->x_pw, xmask, st));
    mask &= ~xmask;
  }
  for (int b0 = 0; b0 < nb; b0 += h->nb_chunk) {
    const int nbc = std::min(h->nb_chunk, nb - b0);
    const int nf = nbc * nocc;
    const cplx<T>* Ab = A + (long long)b0 * nocc * npw;
    STATUS_TRY(pw_to_real<T>(h, Ab, nf, a_r, st));
    if (hmode || xmode)
      { k_delta_rho<T><<<grid_for((long long)nbc * n3, 256), 256, 0, st>>>(phis, a_r, drho, nocc, nbc, n3); note_launch(); }
    if (hmode) STATUS_TRY(convolve_fields<T>(h, drho, nbc, (const T*)h->b.kh, T(1), wb, st));
    { k_init_out<T><<<grid_for((long long)nbc * n3, 256), 256, 0, st>>>(
        a_r, phis, vloc ? (const T*)h->b.vloc : nullptr, wb, (const T*)h->b.fxc, drho, out_r, nocc, nbc, n3, hmode,
        xmode); note_launch(); }
    STATUS_TRY(check_launch("init_out"));
    if ((mask & TDDFT_TERM_D_EXX) && h->d.alpha != 0.0 && !h->ace_on) {
      // out[t] += -alpha sum_w phi_w Conv_x[conj(phi_w) a_t],  t = (b, v)
      PairGrid pg{nf, h->d.nocc_tgt, 0, 1, 0, 0, 0, 1, 0, 1, 0, 0, 1};
      STATUS_TRY(pair_accumulate<T>(h, phit, a_r, phit, out_r, pg, (const T*)h->b.kx, (T)(-h->d.alpha), st));
    }
    if ((mask & TDDFT_TERM_K1D) && h->d.alpha != 0.0) STATUS_TRY(k1d_term<T>(h, nbc, st));
    if ((mask & TDDFT_TERM_K2D) && h->d.alpha != 0.0) {
      // out[b,v] += -alpha sum_v' phi_v' Conv_x[conj(a_{b,v'}) phi_v]  (Eq. 7): per b, targets v, sources v'
      for (int b = 0; b < nbc; ++b) {
        PairGrid pg{nocc, nocc, b * nocc, 1, 0, 0, 0, 1, 0, 1, 0, b * nocc, 1};
        STATUS_TRY(pair_accumulate<T>(h, a_r, phis, phis, out_r, pg, (const T*)h->b.kx, (T)(-h->d.alpha), st));
      }
    }
    STATUS_TRY(real_to_pw<T>(h, out_r, nf, LA + (long long)b0 * nocc * npw,
                             (mask & TDDFT_TERM_D_KIN) ? Ab : nullptr, st));
  }
  if (xmask) {
    const long long len = (long long)nb * nocc * npw;
    { k_accumulate<T><<<grid_for(len, 256), 256, 0, st>>>(LA, (const cplx<T>*)h->x_pw, len); note_launch(); }
    STATUS_TRY(check_launch("exchange-grid terms"));
  }
  if ((mask & TDDFT_TERM_D_EXX) && h->d.alpha != 0.0 && h->ace_on) {
    // alpha V_X^ACE a = -alpha sum_k xi_k <xi_k|a>, in plane waves
    const cplx<T>* xi = (const cplx<T>*)h->ace_xi;
    cplx<T>* C = (cplx<T>*)h->ace_c;
    STATUS_TRY(gemm_overlap<T>(h, xi, h->n_ace, A, nb * nocc, (cplx<T>*)h->ace_part, C, st));
    STATUS_TRY(gemm_update<T>(h, xi, h->n_ace, C, LA, nb * nocc, (T)(-h->d.alpha), st));
  }
  if (mask & TDDFT_TERM_PROJ)
    STATUS_TRY(project_rows<T>(h, (const cplx<T>*)h->b.phi_tgt_pw, h->d.nocc_tgt, LA, nb * nocc, st));
  return TDDFT_OK;
}

// (L A) for nb trial vectors (terms of `mask`). In the localised frame
// (Sec. 3.2, Eq. 31) every term except the eigenvalue part of D is covariant
// under the rotation phi_v = sum_n U_vn phi~_n, so L A = U [L~ A~ - eps~ A~]
// with A~ = U^dagger A, L~ the operator on phi~ with K1d's truncated pairs
// left out and eps~ = U^dagger diag(eps) U; P^c is the same in both frames.
template <typename T>
static tddft_status apply_impl(tddft_system* h, int nb, const cplx<T>* A, cplx<T>* LA, unsigned mask, cudaStream_t st) {
  if (!h->loc_on) return apply_core<T>(h, nb, A, LA, mask, st);
  const int nocc = h->d.nocc_src;
  const long long len = (long long)nocc * h->npw;
  cplx<T>* At = (cplx<T>*)h->loc_a;
  cplx<T>* Lt = (cplx<T>*)h->loc_b;
  CUDA_TRY(cudaMemsetAsync(At, 0, (size_t)nb * len * sizeof(cplx<T>), st));
  for (int b = 0; b < nb; ++b)
    STATUS_TRY(gemm_update<T>(h, A + b * len, nocc, (const cplx<T>*)h->loc_Uc, At + b * len, nocc, T(1), st));
  STATUS_TRY(apply_core<T>(h, nb, At, Lt, mask & ~TDDFT_TERM_PROJ, st));
  if (mask & TDDFT_TERM_D_KIN)
    for (int b = 0; b < nb; ++b)
      STATUS_TRY(gemm_update<T>(h, At + b * len, nocc, (const cplx<T>*)h->loc_E, Lt + b * len, nocc, T(-1), st));
  if (mask & TDDFT_TERM_PROJ)
    STATUS_TRY(project_rows<T>(h, (const cplx<T>*)h->b.phi_tgt_pw, h->d.nocc_tgt, Lt, nb * nocc, st));
  CUDA_TRY(cudaMemsetAsync(LA, 0, (size_t)nb * len * sizeof(cplx<T>), st));
  for (int b = 0; b < nb; ++b)
    STATUS_TRY(gemm_update<T>(h, Lt + b * len, nocc, (const cplx<T>*)h->loc_Ut, LA + b * len, nocc, T(1), st));
  return TDDFT_OK;
}

// ---------------------------------------------------------------------------
// init
// ---------------------------------------------------------------------------
static bool supported_n(int n, int prec) {
  static const int sizes[] = {8, 12, 16, 24, 32, 36, 48, 64, 72, 80, 96, 108, 128};
  for (int s : sizes)
    if (s == n) return !(prec == TDDFT_PREC_FP64 && n == 128);
  return false;
}

// Smallest supported grid on which the exchange terms equal those computed on the n grid.
// With M = max |m_i| over the sphere, a pair density occupies |m_i| <= 2M and its
// convolution times an orbital |m_i| <= 3M. On a grid of N > 4M points per axis no two
// pair-density components fold onto one another, the kernel is sampled at the same G,
// and a product component can only fold onto |m_i| >= N - 3M > M, outside the sphere:
// the plane-wave result on the sphere is the alias-free one, the same on every such grid.
// Returns n when no smaller grid qualifies (in particular when n itself folds).
static int exchange_grid_for(int n, int prec, const std::vector<Miller>& sph) {
  int M = 0;
  for (const Miller& m : sph) M = std::max(M, std::max(std::abs(m.x), std::max(std::abs(m.y), std::abs(m.z))));
  static const int sizes[] = {8, 12, 16, 24, 32, 36, 48, 64, 72, 80, 96, 108, 128};
  for (int g : sizes)
    if (g < n && g > 4 * M && supported_n(g, prec)) return g;
  return n;
}

template <typename T>
static tddft_status init_impl(tddft_system* h, const tddft_inputs* in, cudaStream_t st) {
  const int n = h->n, npw = h->npw;
  const long long n3 = h->n3;
  const tddft_desc& d = h->d;
  PlaneOps<T>& o = ops_of<T>(h);
  o = plane_ops_for<T>(n);
  if (o.n != n) return fail(TDDFT_EINVAL, "unsupported grid size");
  CUDA_TRY(o.prepare());
  CUDA_TRY(cudaFuncSetAttribute(k_k1d_contract<T, 16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(16 * 16 * 32 * sizeof(cplx<T>))));
  CUDA_TRY(cudaFuncSetAttribute(k_k1d_sparse<T, K1D_SPARSE_PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(k1d_sparse_np_max<T>() * K1D_SPARSE_PTS * sizeof(cplx<T>))));
  CUDA_TRY(cudaFuncSetAttribute(k_umma_gemm<OvA, OvB, OvEp>, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_SMEM));
  CUDA_TRY(cudaFuncSetAttribute(k_umma_gemm<UpA, UpB, UpEp>, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_SMEM));
  CUDA_TRY(cudaFuncSetAttribute(k_umma_tiles<OvEp>, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_TILES_SMEM));
  CUDA_TRY(cudaFuncSetAttribute(k_umma_tiles<UpEp>, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_TILES_SMEM));
  STATUS_TRY(dalloc(h, (void**)&h->b.dev_err, sizeof(int)));
  CUDA_TRY(cudaMemsetAsync(h->b.dev_err, 0, sizeof(int), st));

  std::vector<int> radices = plan_radices(n);
  std::vector<int> rev(n);
  for (int k = 0; k < n; ++k) rev[k] = dif_position(k, radices, n);

  // twiddles W_n^e = exp(-2 pi i e / n) and the per-stage tables, FP64 on the host, rounded once
  std::vector<cplx<T>> tw = host_twiddles<T>(n, radices);
  // kernels in position order, divided by N_r
  const double tpiba = 2.0 * M_PI / d.a, tpiba2 = tpiba * tpiba;
  std::vector<T> kx(n3), kh(n3);
  auto mof = [n](int k) { return k < n - n / 2 ? k : k - n; };
  for (int kz = 0; kz < n; ++kz)
    for (int ky = 0; ky < n; ++ky)
      for (int kxx = 0; kxx < n; ++kxx) {
        const long long m2 = (long long)mof(kz) * mof(kz) + (long long)mof(ky) * mof(ky) + (long long)mof(kxx) * mof(kxx);
        const double g2 = tpiba2 * (double)m2;
        const double vx = m2 == 0 ? d.kx_g0 : 4.0 * M_PI / g2;
        const double vh = m2 == 0 ? 0.0 : 4.0 * M_PI / g2;
        const long long p = ((long long)rev[kz] * n + rev[ky]) * n + rev[kxx];
        kx[p] = (T)(vx / (double)n3);
        kh[p] = (T)(vh / (double)n3);
      }
  std::vector<Miller> sph;
  STATUS_TRY(build_sphere(n, d.a, d.ecut, sph));
  std::vector<int> pos(npw);
  std::vector<T> g2h(npw);
  for (int i = 0; i < npw; ++i) {
    const int px = rev[(sph[i].x % n + n) % n], py = rev[(sph[i].y % n + n) % n], pz = rev[(sph[i].z % n + n) % n];
    pos[i] = (pz * n + py) * n + px;
    g2h[i] = (T)(0.5 * (tpiba2 * (double)sph[i].m2));
  }
  std::vector<T> eps(d.nocc_src);
  // the eigenvalues on the host (the input may be host or device memory)
  std::vector<double> eps_in(d.nocc_src);
  CUDA_TRY(cudaMemcpy(eps_in.data(), in->eps_src, d.nocc_src * sizeof(double), cudaMemcpyDefault));
  for (int v = 0; v < d.nocc_src; ++v) eps[v] = (T)eps_in[v];
  // z-pass columns of pair densities: the product of two sphere functions has
  // |m| < 2 R_m (R_m = sqrt(2 ecut) / tpiba); without aliasing (2 max|m_i| <=
  // n/2 - 1) every (k_x, k_y) column with m_x^2 + m_y^2 > 4 R_m^2 is exactly
  // zero. Positions are digit-reversed; the list holds the others after them.
  int mmax = 0;
  for (const Miller& q : sph) mmax = std::max(mmax, std::max(std::abs(q.x), std::max(std::abs(q.y), std::abs(q.z))));
  std::vector<int> zcols;
  if (2 * mmax <= n / 2 - 1) {
    std::vector<int> irev(n);
    for (int k = 0; k < n; ++k) irev[rev[k]] = k;
    const double r2 = 4.0 * (2.0 * d.ecut / tpiba2) * (1.0 + 1e-12);
    std::vector<int> rest;
    for (int py = 0; py < n; ++py)
      for (int px = 0; px < n; ++px) {
        const double mx = mof(irev[px]), my = mof(irev[py]);
        if (mx * mx + my * my <= r2) zcols.push_back(py * n + px);
        else rest.push_back(py * n + px);
      }
    if (o.lines_ok) {
      // register-line xy passes: ordered by x position, then y position, so that the 16
      // lanes writing rows y..y+15 of one x position store to consecutive entries
      auto by_x = [n](int p, int q) { return std::make_pair(p % n, p / n) < std::make_pair(q % n, q / n); };
      std::sort(zcols.begin(), zcols.end(), by_x);
      std::sort(rest.begin(), rest.end(), by_x);
    } else {
      // Within each part, interleave the 16 shared-memory bank classes of the positions
      // (8-byte words y * (n + 1) + x in the plane kernels): the compact planes are staged
      // with 16 consecutive list entries per half-warp, which then hit distinct banks.
      auto interleave_banks = [n](std::vector<int>& v) {
        std::vector<std::vector<int>> cls(16);
        for (int q : v) cls[((q / n) * (n + 1) + q % n) % 16].push_back(q);
        std::vector<int> out;
        out.reserve(v.size());
        std::vector<size_t> at(16, 0);
        while (out.size() < v.size())
          for (int k = 0; k < 16; ++k)
            if (at[k] < cls[k].size()) out.push_back(cls[k][at[k]++]);
        v.swap(out);
      };
      interleave_banks(zcols);
      interleave_banks(rest);
    }
    h->ncols_act = (int)zcols.size();
    zcols.insert(zcols.end(), rest.begin(), rest.end());
  }

  Buffers& B = h->b;
  const size_t ez = sizeof(cplx<T>), rz = sizeof(T);
  STATUS_TRY(dalloc(h, &B.tw, tw.size() * ez));
  STATUS_TRY(dalloc(h, &B.kx, n3 * rz));
  STATUS_TRY(dalloc(h, &B.kh, n3 * rz));
  STATUS_TRY(dalloc(h, (void**)&B.pos, npw * sizeof(int)));
  STATUS_TRY(dalloc(h, &B.g2h, npw * rz));
  STATUS_TRY(dalloc(h, &B.eps, d.nocc_src * rz));
  std::vector<T> kx_c, kh_c, kx_p, kh_p;
  if (!zcols.empty()) {
    STATUS_TRY(dalloc(h, (void**)&B.zcols, zcols.size() * sizeof(int)));
    CUDA_TRY(cudaMemcpyAsync(B.zcols, zcols.data(), zcols.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (o.lines_ok) {
      std::vector<int> cmapT((size_t)n * n, -1);
      for (int c = 0; c < h->ncols_act; ++c) cmapT[(size_t)(zcols[c] % n) * n + zcols[c] / n] = c;
      STATUS_TRY(dalloc(h, (void**)&B.cmapT, cmapT.size() * sizeof(int)));
      CUDA_TRY(cudaMemcpy(B.cmapT, cmapT.data(), cmapT.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    // kernels on the compact columns: [z][c] = kappa at (z, zcols[c])
    const int na = h->ncols_act;
    kx_c.resize((size_t)n * na);
    kh_c.resize((size_t)n * na);
    for (int z = 0; z < n; ++z)
      for (int c = 0; c < na; ++c) {
        kx_c[(size_t)z * na + c] = kx[(size_t)z * n * n + zcols[c]];
        kh_c[(size_t)z * na + c] = kh[(size_t)z * n * n + zcols[c]];
      }
    STATUS_TRY(dalloc(h, &B.kx_c, kx_c.size() * rz));
    STATUS_TRY(dalloc(h, &B.kh_c, kh_c.size() * rz));
    CUDA_TRY(cudaMemcpyAsync(B.kx_c, kx_c.data(), kx_c.size() * rz, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(B.kh_c, kh_c.data(), kh_c.size() * rz, cudaMemcpyHostToDevice, st));
    if (o.pair_ok) {
      // paired z pass: lane h, register j holds k_z = 2 k' + h, with k' the natural index
      // of position j of the N/2 plan's digit-reversed order
      const int hn = n / 2;
      const std::vector<int> rad_h = plan_radices(hn);
      std::vector<int> irev_h(hn);
      for (int k = 0; k < hn; ++k) irev_h[dif_position(k, rad_h, hn)] = k;
      kx_p.resize((size_t)n * na);
      kh_p.resize((size_t)n * na);
      for (int hh = 0; hh < 2; ++hh)
        for (int j = 0; j < hn; ++j) {
          const int pz = rev[2 * irev_h[j] + hh];
          for (int c = 0; c < na; ++c) {
            kx_p[(size_t)(hh * hn + j) * na + c] = kx_c[(size_t)pz * na + c];
            kh_p[(size_t)(hh * hn + j) * na + c] = kh_c[(size_t)pz * na + c];
          }
        }
      STATUS_TRY(dalloc(h, &B.kx_p, kx_p.size() * rz));
      STATUS_TRY(dalloc(h, &B.kh_p, kh_p.size() * rz));
      CUDA_TRY(cudaMemcpyAsync(B.kx_p, kx_p.data(), kx_p.size() * rz, cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(B.kh_p, kh_p.data(), kh_p.size() * rz, cudaMemcpyHostToDevice, st));
    }
  }
  CUDA_TRY(cudaMemcpyAsync(B.tw, tw.data(), tw.size() * ez, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B.kx, kx.data(), n3 * rz, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B.kh, kh.data(), n3 * rz, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B.pos, pos.data(), npw * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B.g2h, g2h.data(), npw * rz, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B.eps, eps.data(), d.nocc_src * rz, cudaMemcpyHostToDevice, st));
  h->eps64 = eps_in;

  // orbitals: FP64 upload, orthonormality check, cast to the working precision
  const int nsets = h->sf() ? 2 : 1;
  const int ntgt = d.nocc_tgt;
  STATUS_TRY(dalloc(h, (void**)&B.phi_tgt_pw64, (size_t)ntgt * npw * sizeof(cplx<double>)));
  cplx<double>* phi_src64 = nullptr;
  STATUS_TRY(dalloc(h, (void**)&phi_src64, (size_t)d.nocc_src * npw * sizeof(cplx<double>)));
  B.phi_src_pw64 = phi_src64;
  CUDA_TRY(cudaMemcpyAsync(phi_src64, in->phi_src, (size_t)d.nocc_src * npw * 16, cudaMemcpyDefault, st));
  if (h->sf())
    CUDA_TRY(cudaMemcpyAsync(B.phi_tgt_pw64, in->phi_tgt, (size_t)ntgt * npw * 16, cudaMemcpyDefault, st));
  else
    CUDA_TRY(cudaMemcpyAsync(B.phi_tgt_pw64, phi_src64, (size_t)ntgt * npw * 16, cudaMemcpyDeviceToDevice, st));

  // projector scratch sized for nb_max * nocc_src rows (also used for the checks below)
  const int maxrows = std::max(d.nb_max * d.nocc_src, std::max(d.nocc_src, ntgt));
  h->nsplit = std::max(1, std::min(32, npw / 512));
  STATUS_TRY(dalloc(h, &B.cmat, (size_t)std::max(ntgt, d.nocc_src) * maxrows * sizeof(cplx<double>)));
  STATUS_TRY(dalloc(h, &B.cpart, (size_t)h->nsplit * std::max(ntgt, d.nocc_src) * maxrows * sizeof(cplx<double>)));
  STATUS_TRY(dalloc(h, &B.ctmp, (size_t)std::max(ntgt, d.nocc_src) * maxrows * sizeof(cplx<double>)));

  for (int set = 0; set < nsets; ++set) {
    const cplx<double>* P = set == 0 ? phi_src64 : B.phi_tgt_pw64;
    const int M = set == 0 ? d.nocc_src : ntgt;
    cplx<double>* C = (cplx<double>*)B.cmat;
    cplx<double>* Cp = (cplx<double>*)B.cpart;
    const int kchunk = ((npw + h->nsplit - 1) / h->nsplit + 15) / 16 * 16;
    dim3 g1((M + 31) / 32, (M + 31) / 32, h->nsplit);
    { k_overlap<double><<<g1, 256, 0, st>>>(P, M, P, M, npw, kchunk, Cp); note_launch(); }
    { k_reduce_split<double><<<grid_for((long long)M * M, 256), 256, 0, st>>>(Cp, h->nsplit, (long long)M * M, C); note_launch(); }
    STATUS_TRY(check_launch("orthonormality check"));
    std::vector<cplx<double>> hc((size_t)M * M);
    CUDA_TRY(cudaMemcpyAsync(hc.data(), C, hc.size() * 16, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    double dev = 0.0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        const cplx<double> c = hc[(size_t)i * M + j];
        dev = std::max(dev, std::hypot(c.x - (i == j ? 1.0 : 0.0), c.y));
      }
    if (!(dev <= 1e-10))
      return fail(TDDFT_EINVAL, "orbitals are not orthonormal: max |Phi^H Phi - I| = " + std::to_string(dev));
  }

  STATUS_TRY(dalloc(h, &B.phi_src_pw, (size_t)d.nocc_src * npw * ez));
  { k_cast<T><<<grid_for((long long)d.nocc_src * npw, 256), 256, 0, st>>>(phi_src64, (cplx<T>*)B.phi_src_pw,
                                                                        (long long)d.nocc_src * npw); note_launch(); }
  if (h->sf()) {
    STATUS_TRY(dalloc(h, &B.phi_tgt_pw, (size_t)ntgt * npw * ez));
    { k_cast<T><<<grid_for((long long)ntgt * npw, 256), 256, 0, st>>>(B.phi_tgt_pw64, (cplx<T>*)B.phi_tgt_pw,
                                                                    (long long)ntgt * npw); note_launch(); }
  } else {
    B.phi_tgt_pw = B.phi_src_pw;
  }
  STATUS_TRY(check_launch("orbital cast"));

  // local fields
  TempAllocs tmp;
  double* tmp64 = nullptr;
  if (in->vloc || in->fxc) STATUS_TRY(tmp.get((void**)&tmp64, n3 * sizeof(double)));
  if (in->vloc) {
    STATUS_TRY(dalloc(h, &B.vloc, n3 * rz));
    CUDA_TRY(cudaMemcpyAsync(tmp64, in->vloc, n3 * 8, cudaMemcpyDefault, st));
    { k_real_cast<T><<<grid_for(n3, 256), 256, 0, st>>>(tmp64, (T*)B.vloc, n3); note_launch(); }
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (in->fxc) {
    STATUS_TRY(dalloc(h, &B.fxc, n3 * rz));
    CUDA_TRY(cudaMemcpyAsync(tmp64, in->fxc, n3 * 8, cudaMemcpyDefault, st));
    { k_real_cast<T><<<grid_for(n3, 256), 256, 0, st>>>(tmp64, (T*)B.fxc, n3); note_launch(); }
    CUDA_TRY(cudaStreamSynchronize(st));
  }

  // workspace: chunk of trial vectors and the pair-batch buffer, bounded to leave
  // room on the device (cfg-independent: at most ~60% of free memory)
  size_t freeb = 0, totalb = 0;
  CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
  const size_t field = (size_t)n3 * ez;
  h->ibuf_fields = std::max(16, std::min(1024, (int)((size_t)(2u << 30) / field)));
  const size_t fixed = field * ((size_t)h->ibuf_fields + (size_t)d.nocc_src + (h->sf() ? ntgt : 0));
  const size_t per_b = field * (2 * (size_t)d.nocc_src + 2);
  const size_t budget = (size_t)(0.6 * (double)freeb);
  if (budget < fixed + per_b) return fail(TDDFT_ENOMEM, "not enough device memory for one trial vector");
  h->nb_chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)d.nb_max, (budget - fixed) / per_b));

  STATUS_TRY(dalloc(h, &B.ibuf, (size_t)h->ibuf_fields * field));
  STATUS_TRY(dalloc(h, &B.phi_src_r, (size_t)d.nocc_src * field));
  STATUS_TRY(dalloc(h, &B.a_r, (size_t)h->nb_chunk * d.nocc_src * field));
  STATUS_TRY(dalloc(h, &B.out_r, (size_t)h->nb_chunk * d.nocc_src * field));
  STATUS_TRY(dalloc(h, &B.drho, (size_t)h->nb_chunk * field));
  STATUS_TRY(dalloc(h, &B.wb, (size_t)h->nb_chunk * field));
  STATUS_TRY(pw_to_real<T>(h, (const cplx<T>*)B.phi_src_pw, d.nocc_src, (cplx<T>*)B.phi_src_r, st));
  if (h->sf()) {
    STATUS_TRY(dalloc(h, &B.phi_tgt_r, (size_t)ntgt * field));
    STATUS_TRY(pw_to_real<T>(h, (const cplx<T>*)B.phi_tgt_pw, ntgt, (cplx<T>*)B.phi_tgt_r, st));
  } else {
    B.phi_tgt_r = B.phi_src_r;
  }
  const size_t iob = (size_t)d.nb_max * d.nocc_src * npw * ez;
  STATUS_TRY(dalloc(h, &B.io_a, iob));
  STATUS_TRY(dalloc(h, &B.io_b, iob));
  STATUS_TRY(dalloc(h, (void**)&B.wdev, (size_t)d.nb_max * sizeof(double)));
  CUDA_TRY(cudaStreamSynchronize(st));
  return check_launch("init");
}

// ---------------------------------------------------------------------------
// adaptively compressed exchange (Sec. 3.1)
// ---------------------------------------------------------------------------

// A = L L^dagger for Hermitian positive definite A (row-major n x n, lower L
// returned in A); false if a pivot is not positive.
static bool cholesky_lower(int n, std::vector<std::complex<double>>& A) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(A[(size_t)j * n + k]);
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    A[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      std::complex<double> v = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * std::conj(A[(size_t)j * n + k]);
      A[(size_t)i * n + j] = v / ljj;
    }
    for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0.0;
  }
  return true;
}

// inverse of a lower-triangular L (row-major), by forward substitution per column
static std::vector<std::complex<double>> lower_inverse(int n, const std::vector<std::complex<double>>& L) {
  std::vector<std::complex<double>> X((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      std::complex<double> v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = v / L[(size_t)i * n + i];
    }
  }
  return X;
}


template <typename T>
static tddft_status ace_build_impl(tddft_system* h, int n_extra, const double* extra, cudaStream_t st) {
  const int nt = h->d.nocc_tgt, na = nt + n_extra, npw = h->npw;
  const size_t row64 = (size_t)npw * sizeof(cplx<double>), rowT = (size_t)npw * sizeof(cplx<T>);
  TempAllocs tmp;
  cplx<double>* psi64 = nullptr;
  cplx<double>* w64 = nullptr;
  cplx<T>* psi = nullptr;
  cplx<T>* W = nullptr;
  cplx<double>* m64 = nullptr;
  cplx<double>* p64 = nullptr;
  cplx<T>* cm = nullptr;
  STATUS_TRY(tmp.get((void**)&psi64, row64 * na));
  STATUS_TRY(tmp.get((void**)&w64, row64 * na));
  STATUS_TRY(tmp.get((void**)&psi, rowT * na));
  STATUS_TRY(tmp.get((void**)&W, rowT * na));
  STATUS_TRY(tmp.get((void**)&m64, sizeof(cplx<double>) * na * na));
  STATUS_TRY(tmp.get((void**)&p64, sizeof(cplx<double>) * h->nsplit * na * na));
  STATUS_TRY(tmp.get((void**)&cm, sizeof(cplx<T>) * na * na));
  CUDA_TRY(cudaMemcpyAsync(psi64, h->b.phi_tgt_pw64, row64 * nt, cudaMemcpyDeviceToDevice, st));
  if (n_extra) CUDA_TRY(cudaMemcpyAsync(psi64 + (size_t)nt * npw, extra, row64 * n_extra, cudaMemcpyHostToDevice, st));
  const int kchunk = ((npw + h->nsplit - 1) / h->nsplit + 15) / 16 * 16;
  auto overlap64 = [&](const cplx<double>* A, const cplx<double>* B, std::vector<std::complex<double>>& out) -> tddft_status {
    dim3 g1((na + 31) / 32, (na + 31) / 32, h->nsplit);
    { k_overlap<double><<<g1, 256, 0, st>>>(A, na, B, na, npw, kchunk, p64); note_launch(); }
    { k_reduce_split<double><<<grid_for((long long)na * na, 256), 256, 0, st>>>(p64, h->nsplit, (long long)na * na, m64); note_launch(); }
    STATUS_TRY(check_launch("ace overlap"));
    out.resize((size_t)na * na);
    CUDA_TRY(cudaMemcpyAsync(out.data(), m64, out.size() * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDDFT_OK;
  };
  // the build set must be orthonormal (the occupied orbitals followed by the extra rows)
  std::vector<std::complex<double>> S;
  STATUS_TRY(overlap64(psi64, psi64, S));
  double dev = 0.0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < na; ++j) dev = std::max(dev, std::abs(S[(size_t)i * na + j] - (i == j ? 1.0 : 0.0)));
  if (!(dev <= 1e-10))
    return fail(TDDFT_EINVAL, "ACE build vectors are not orthonormal and orthogonal to the orbitals: max dev " +
                                  std::to_string(dev));
  { k_cast<T><<<grid_for((long long)na * npw, 256), 256, 0, st>>>(psi64, psi, (long long)na * npw); note_launch(); }
  // W = V_X Psi with the exact pair convolutions, in chunks of the real-space workspace
  const int cap = h->nb_chunk * h->d.nocc_src;
  cplx<T>* a_r = (cplx<T>*)h->b.a_r;
  cplx<T>* out_r = (cplx<T>*)h->b.out_r;
  const cplx<T>* phit = (const cplx<T>*)h->b.phi_tgt_r;
  for (int r0 = 0; r0 < na; r0 += cap) {
    const int cnt = std::min(cap, na - r0);
    STATUS_TRY(pw_to_real<T>(h, psi + (size_t)r0 * npw, cnt, a_r, st));
    CUDA_TRY(cudaMemsetAsync(out_r, 0, (size_t)cnt * h->n3 * sizeof(cplx<T>), st));
    PairGrid pg{cnt, nt, 0, 1, 0, 0, 0, 1, 0, 1, 0, 0, 1};
    STATUS_TRY(pair_accumulate<T>(h, phit, a_r, phit, out_r, pg, (const T*)h->b.kx, T(-1), st));
    STATUS_TRY(real_to_pw<T>(h, out_r, cnt, W + (size_t)r0 * npw, nullptr, st));
  }
  { k_widen<T><<<grid_for((long long)na * npw, 256), 256, 0, st>>>(W, w64, (long long)na * npw); note_launch(); }
  // M = Psi^dagger W (FP64), -M = L L^dagger, xi = W L^{-dagger}
  std::vector<std::complex<double>> M;
  STATUS_TRY(overlap64(psi64, w64, M));
  std::vector<std::complex<double>> negM((size_t)na * na);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < na; ++j)
      negM[(size_t)i * na + j] = -0.5 * (M[(size_t)i * na + j] + std::conj(M[(size_t)j * na + i]));
  if (!cholesky_lower(na, negM)) return fail(TDDFT_ENUMERIC, "-Psi^dagger V_X Psi is not positive definite");
  const std::vector<std::complex<double>> Linv = lower_inverse(na, negM);
  // xi[k][g] = sum_i conj(Linv[k][i]) W[i][g]  ->  update with C[i][k] = conj(Linv[k][i])
  std::vector<cplx<T>> ch((size_t)na * na);
  for (int i = 0; i < na; ++i)
    for (int k = 0; k < na; ++k) {
      const std::complex<double> c = std::conj(Linv[(size_t)k * na + i]);
      ch[(size_t)i * na + k] = {(T)c.real(), (T)c.imag()};
    }
  CUDA_TRY(cudaMemcpyAsync(cm, ch.data(), ch.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
  // persistent buffers (replaced on a rebuild)
  const int rows = h->d.nb_max * h->d.nocc_src;
  for (void** q : {&h->ace_xi, &h->ace_c, &h->ace_part}) {
    if (*q) {
      cudaFree(*q);
      h->allocations.erase(std::remove(h->allocations.begin(), h->allocations.end(), *q), h->allocations.end());
      *q = nullptr;
    }
  }
  h->ace_on = false;
  STATUS_TRY(dalloc(h, &h->ace_xi, rowT * na));
  STATUS_TRY(dalloc(h, &h->ace_c, sizeof(cplx<T>) * (size_t)na * rows));
  STATUS_TRY(dalloc(h, &h->ace_part, sizeof(cplx<T>) * (size_t)2 * h->nsplit * na * rows));
  CUDA_TRY(cudaMemsetAsync(h->ace_xi, 0, rowT * na, st));
  { dim3 g2((npw + 63) / 64, (na + 31) / 32);
    k_update<T><<<g2, 256, 0, st>>>(W, na, cm, na, npw, T(1), (cplx<T>*)h->ace_xi); note_launch(); }
  STATUS_TRY(check_launch("ace build"));
  CUDA_TRY(cudaStreamSynchronize(st));
  h->n_ace = na;
  h->ace_on = true;
  return TDDFT_OK;
}

// ---------------------------------------------------------------------------
// localised frame and pair truncation (Sec. 3.2, Eq. 31)
// ---------------------------------------------------------------------------

namespace {
void drop_graphs(tddft_system* h);  // forgets captured graphs that contain h's launches
}  // namespace

// part[z][m][n] = sum over the z-th slice of points of d_m(r) d_n(r), d = |phi(r)|^2,
// FP64 accumulation of the products. 16 x 16 (m, n) tile per CTA, points staged
// in shared memory 64 at a time.
constexpr int DG_TILE = 16, DG_PTS = 64;
template <typename T>
__global__ void __launch_bounds__(DG_TILE * DG_TILE)
    k_density_gram(const cplx<T>* __restrict__ phi, int nocc, long long n3, long long per_slice,
                   double* __restrict__ part) {
  __shared__ double dm[DG_TILE][DG_PTS + 1], dn[DG_TILE][DG_PTS + 1];
  const int m0 = blockIdx.y * DG_TILE, n0 = blockIdx.x * DG_TILE;
  const int tm = threadIdx.x / DG_TILE, tn = threadIdx.x % DG_TILE;
  const long long r_begin = (long long)blockIdx.z * per_slice;
  const long long r_end = min(n3, r_begin + per_slice);
  double acc = 0.0;
  for (long long r0 = r_begin; r0 < r_end; r0 += DG_PTS) {
    for (int e = threadIdx.x; e < DG_TILE * DG_PTS; e += DG_TILE * DG_TILE) {
      const int o = e / DG_PTS, p = e % DG_PTS;
      const long long r = r0 + p;
      double vm = 0.0, vn = 0.0;
      if (r < r_end) {
        if (m0 + o < nocc) {
          const cplx<T> c = phi[(long long)(m0 + o) * n3 + r];
          vm = (double)c.x * c.x + (double)c.y * c.y;
        }
        if (n0 + o < nocc) {
          const cplx<T> c = phi[(long long)(n0 + o) * n3 + r];
          vn = (double)c.x * c.x + (double)c.y * c.y;
        }
      }
      dm[o][p] = vm;
      dn[o][p] = vn;
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < DG_PTS; ++p) acc += dm[tm][p] * dn[tn][p];
    __syncthreads();
  }
  if (m0 + tm < nocc && n0 + tn < nocc) part[((long long)blockIdx.z * nocc + m0 + tm) * nocc + n0 + tn] = acc;
}

// phi_src (PW, handle precision) and its real-space copy from FP64 rows
template <typename T>
static tddft_status load_source_orbitals(tddft_system* h, const cplx<double>* phi64, cudaStream_t st) {
  const long long cnt = (long long)h->d.nocc_src * h->npw;
  { k_cast<T><<<grid_for(cnt, 256), 256, 0, st>>>(phi64, (cplx<T>*)h->b.phi_src_pw, cnt); note_launch(); }
  STATUS_TRY(check_launch("orbital cast"));
  return pw_to_real<T>(h, (const cplx<T>*)h->b.phi_src_pw, h->d.nocc_src, (cplx<T>*)h->b.phi_src_r, st);
}

// Kept unique pairs (m <= n, by m then n) in batches of at most
// min(ibuf_fields, k1d_sparse_np_max) slots, each with its rows: orbital m gets
// (n, slot) and, for m != n, orbital n gets (m, slot) with tau conjugated.
template <typename T>
static tddft_status build_pair_batches(tddft_system* h, cudaStream_t st) {
  const int nocc = h->d.nocc_src;
  const int npmax = std::max(1, std::min(h->ibuf_fields, k1d_sparse_np_max<T>()));
  std::vector<int2> list;
  for (int m = 0; m < nocc; ++m)
    for (int n = m; n < nocc; ++n)
      if (h->loc_keep_host[(size_t)m * nocc + n]) list.push_back(make_int2(n, m));
  const size_t unique_total = (size_t)nocc * (nocc + 1) / 2;
  h->loc_sparse_auto = 2 * list.size() < unique_total;
  std::vector<int> rowptr, rowout;
  std::vector<int2> ent;
  h->loc_batches.clear();
  for (size_t p0 = 0; p0 < list.size(); p0 += npmax) {
    const int np = (int)std::min<size_t>(npmax, list.size() - p0);
    std::vector<std::vector<int2>> rows(nocc);
    for (int j = 0; j < np; ++j) {
      const int n = list[p0 + j].x, m = list[p0 + j].y;
      rows[m].push_back(make_int2(n << 1, j));
      if (m != n) rows[n].push_back(make_int2((m << 1) | 1, j));
    }
    tddft_system::PairBatch pb{(int)p0, np, (int)rowptr.size(), 0};
    for (int o = 0; o < nocc; ++o) {
      if (rows[o].empty()) continue;
      rowptr.push_back((int)ent.size());
      rowout.push_back(o);
      ent.insert(ent.end(), rows[o].begin(), rows[o].end());
      ++pb.nrows;
    }
    rowptr.push_back((int)ent.size());
    rowout.push_back(-1);  // keeps rowout aligned with rowptr; never read
    h->loc_batches.push_back(pb);
  }
  for (void** q : {(void**)&h->loc_list, (void**)&h->loc_rowptr, (void**)&h->loc_rowout, (void**)&h->loc_ent}) {
    if (*q) {
      cudaFree(*q);
      h->allocations.erase(std::remove(h->allocations.begin(), h->allocations.end(), *q), h->allocations.end());
      *q = nullptr;
    }
  }
  if (list.empty()) return TDDFT_OK;
  STATUS_TRY(dalloc(h, (void**)&h->loc_list, list.size() * sizeof(int2)));
  STATUS_TRY(dalloc(h, (void**)&h->loc_rowptr, rowptr.size() * sizeof(int)));
  STATUS_TRY(dalloc(h, (void**)&h->loc_rowout, rowout.size() * sizeof(int)));
  STATUS_TRY(dalloc(h, (void**)&h->loc_ent, ent.size() * sizeof(int2)));
  CUDA_TRY(cudaMemcpyAsync(h->loc_list, list.data(), list.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_rowptr, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_rowout, rowout.data(), rowout.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_ent, ent.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
  return TDDFT_OK;
}

template <typename T>
static tddft_status localization_impl(tddft_system* h, const double* Uh, double s_thr, double* S_out, int* kept,
                                      cudaStream_t st) {
  using C = std::complex<double>;
  const int nocc = h->d.nocc_src, npw = h->npw;
  const C* U = reinterpret_cast<const C*>(Uh);
  drop_graphs(h);
  if (!U) {  // back to the given orbitals
    h->loc_on = false;
    STATUS_TRY(load_source_orbitals<T>(h, h->b.phi_src_pw64, st));
    if (h->xsub) {
      drop_graphs(h->xsub);
      h->xsub->loc_on = false;
      STATUS_TRY(load_source_orbitals<T>(h->xsub, h->xsub->b.phi_src_pw64, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (kept) *kept = nocc * nocc;
    return TDDFT_OK;
  }
  double dev = 0.0;
  for (int i = 0; i < nocc; ++i)
    for (int j = 0; j < nocc; ++j) {
      C g = 0.0;
      for (int v = 0; v < nocc; ++v) g += std::conj(U[(size_t)v * nocc + i]) * U[(size_t)v * nocc + j];
      dev = std::max(dev, std::abs(g - (i == j ? 1.0 : 0.0)));
    }
  if (!(dev <= 1e-10)) return fail(TDDFT_EINVAL, "U is not unitary: max |U^H U - I| = " + std::to_string(dev));
  if (!h->loc_a) {
    const size_t rows = (size_t)h->d.nb_max * nocc * npw * sizeof(cplx<T>);
    STATUS_TRY(dalloc(h, &h->loc_a, rows));
    STATUS_TRY(dalloc(h, &h->loc_b, rows));
    STATUS_TRY(dalloc(h, &h->loc_Uc, (size_t)nocc * nocc * sizeof(cplx<T>)));
    STATUS_TRY(dalloc(h, &h->loc_Ut, (size_t)nocc * nocc * sizeof(cplx<T>)));
    STATUS_TRY(dalloc(h, &h->loc_E, (size_t)nocc * nocc * sizeof(cplx<T>)));
    STATUS_TRY(dalloc(h, (void**)&h->loc_keep, (size_t)nocc * nocc));
  }
  h->loc_on = false;
  // phi~_n = sum_v conj(U_vn) phi_v in FP64, then the handle's orbitals
  TempAllocs tmp;
  cplx<double>* phil = nullptr;
  cplx<double>* c64 = nullptr;
  STATUS_TRY(tmp.get((void**)&phil, (size_t)nocc * npw * sizeof(cplx<double>)));
  STATUS_TRY(tmp.get((void**)&c64, (size_t)nocc * nocc * sizeof(cplx<double>)));
  std::vector<cplx<double>> cu((size_t)nocc * nocc);
  std::vector<cplx<T>> cuT(cu.size()), ctT(cu.size()), ceT(cu.size());
  const std::vector<double>& eps = h->eps64;
  for (int v = 0; v < nocc; ++v)
    for (int n = 0; n < nocc; ++n) {
      const C u = U[(size_t)v * nocc + n];
      cu[(size_t)v * nocc + n] = {std::conj(u).real(), std::conj(u).imag()};
      cuT[(size_t)v * nocc + n] = {(T)u.real(), (T)(-u.imag())};
      ctT[(size_t)n * nocc + v] = {(T)u.real(), (T)u.imag()};
    }
  for (int n = 0; n < nocc; ++n)
    for (int np = 0; np < nocc; ++np) {
      C e = 0.0;
      for (int v = 0; v < nocc; ++v) e += std::conj(U[(size_t)v * nocc + n]) * eps[v] * U[(size_t)v * nocc + np];
      ceT[(size_t)np * nocc + n] = {(T)e.real(), (T)e.imag()};
    }
  CUDA_TRY(cudaMemcpyAsync(c64, cu.data(), cu.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(phil, 0, (size_t)nocc * npw * sizeof(cplx<double>), st));
  { dim3 g2((npw + 63) / 64, (nocc + 31) / 32);
    k_update<double><<<g2, 256, 0, st>>>(h->b.phi_src_pw64, nocc, c64, nocc, npw, 1.0, phil); note_launch(); }
  STATUS_TRY(check_launch("localised orbitals"));
  STATUS_TRY(load_source_orbitals<T>(h, phil, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_Uc, cuT.data(), cuT.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_Ut, ctT.data(), ctT.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(h->loc_E, ceT.data(), ceT.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
  // overlap function S_mn of the localised orbitals (densities of the handle's real-space orbitals)
  const long long n3 = h->n3;
  const int slices = (int)std::max(1LL, std::min(64LL, n3 / 4096));
  const long long per = (n3 + slices - 1) / slices;
  double* part = nullptr;
  STATUS_TRY(tmp.get((void**)&part, (size_t)slices * nocc * nocc * sizeof(double)));
  { dim3 g((nocc + DG_TILE - 1) / DG_TILE, (nocc + DG_TILE - 1) / DG_TILE, slices);
    k_density_gram<T><<<g, DG_TILE * DG_TILE, 0, st>>>((const cplx<T>*)h->b.phi_src_r, nocc, n3, per, part); note_launch(); }
  STATUS_TRY(check_launch("density gram"));
  std::vector<double> ph((size_t)slices * nocc * nocc);
  CUDA_TRY(cudaMemcpyAsync(ph.data(), part, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> Q((size_t)nocc * nocc, 0.0);
  for (int z = 0; z < slices; ++z)
    for (size_t i = 0; i < Q.size(); ++i) Q[i] += ph[(size_t)z * Q.size() + i];
  h->loc_keep_host.assign((size_t)nocc * nocc, 0);
  int cnt = 0;
  for (int m = 0; m < nocc; ++m)
    for (int n = 0; n < nocc; ++n) {
      // symmetric by construction: (Q_mn + Q_nm) / 2 against the diagonal
      const double q = 0.5 * (Q[(size_t)m * nocc + n] + Q[(size_t)n * nocc + m]);
      const double S = q / std::sqrt(Q[(size_t)m * nocc + m] * Q[(size_t)n * nocc + n]);
      if (S_out) S_out[(size_t)m * nocc + n] = S;
      const unsigned char k = S >= s_thr ? 1 : 0;
      h->loc_keep_host[(size_t)m * nocc + n] = k;
      cnt += k;
    }
  CUDA_TRY(cudaMemcpyAsync(h->loc_keep, h->loc_keep_host.data(), h->loc_keep_host.size(), cudaMemcpyHostToDevice, st));
  STATUS_TRY(build_pair_batches<T>(h, st));
  if (h->xsub) {
    // the exchange-grid system (D_EXX, K1d, K2d) works in the same frame with the same kept
    // pairs (the overlap function of the caller's grid decides them)
    tddft_system* x = h->xsub;
    drop_graphs(x);
    x->loc_on = false;
    STATUS_TRY(load_source_orbitals<T>(x, phil, st));
    if (!x->loc_keep) STATUS_TRY(dalloc(x, (void**)&x->loc_keep, (size_t)nocc * nocc));
    x->loc_keep_host = h->loc_keep_host;
    CUDA_TRY(cudaMemcpyAsync(x->loc_keep, x->loc_keep_host.data(), x->loc_keep_host.size(), cudaMemcpyHostToDevice, st));
    STATUS_TRY(build_pair_batches<T>(x, st));
    x->loc_kept = cnt;
    x->loc_on = true;
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  h->loc_kept = cnt;
  if (kept) *kept = cnt;
  h->loc_on = true;
  return TDDFT_OK;
}

// ---------------------------------------------------------------------------
// adjoint (spin-conserving)
// ---------------------------------------------------------------------------
template <typename T>
static tddft_status adjoint_impl(tddft_system* h, int nb, const cplx<T>* X, const double* w, double* omega,
                                 cplx<T>* grad_phi, double* grad_vloc, cudaStream_t st) {
  const int nocc = h->d.nocc_src, ntgt = h->d.nocc_tgt, npw = h->npw;
  const bool sf = h->sf();
  const long long n3 = h->n3, rows = (long long)nb * nocc;
  Buffers& B = h->b;
  const int gfields = nocc + (sf ? ntgt : 0);
  if (!B.grad_r) STATUS_TRY(dalloc(h, &B.grad_r, (size_t)gfields * n3 * sizeof(cplx<T>)));
  cplx<T>* P = (cplx<T>*)B.io_a;   // P^c X
  cplx<T>* Y = (cplx<T>*)B.io_b;   // M P^c X
  // source-spin rows (K1e, K1d) and target-spin rows (V_X in D, P^c); the same rows when spin-conserving
  cplx<T>* Gs = (cplx<T>*)B.grad_r;
  cplx<T>* Gt = sf ? Gs + (long long)nocc * n3 : Gs;
  cplx<T>* grad_t = sf ? grad_phi + (long long)nocc * npw : grad_phi;
  const cplx<T>* phi = (const cplx<T>*)B.phi_tgt_pw;  // projector orbitals
  const cplx<T>* phi_r = (const cplx<T>*)B.phi_src_r;
  const cplx<T>* phit_r = (const cplx<T>*)B.phi_tgt_r;
  CUDA_TRY(cudaMemcpyAsync(P, X, (size_t)rows * npw * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st));
  STATUS_TRY(project_rows<T>(h, phi, ntgt, P, (int)rows, st));
  const unsigned mask = TDDFT_TERMS_ALL & ~TDDFT_TERM_PROJ;
  STATUS_TRY(apply_impl<T>(h, nb, P, Y, mask, st));
  { k_bilinear<T><<<nb, 256, 0, st>>>(P, Y, (long long)nocc * npw, omega); note_launch(); }
  STATUS_TRY(check_launch("bilinear"));

  // real-space part of the gradient, one trial vector at a time
  CUDA_TRY(cudaMemsetAsync(Gs, 0, (size_t)gfields * n3 * sizeof(cplx<T>), st));
  if (grad_vloc) CUDA_TRY(cudaMemsetAsync(grad_vloc, 0, (size_t)n3 * sizeof(double), st));
  cplx<T>* p_r = (cplx<T>*)B.a_r;
  cplx<T>* drho = (cplx<T>*)B.drho;
  cplx<T>* wb = (cplx<T>*)B.wb;
  const double vol = h->d.a * h->d.a * h->d.a;
  for (int b = 0; b < nb; ++b) {
    if (w[b] == 0.0) continue;
    STATUS_TRY(pw_to_real<T>(h, P + (long long)b * nocc * npw, nocc, p_r, st));
    const T wa = (T)(-h->d.alpha * w[b]);
    if (h->d.alpha != 0.0) {
      // -alpha w sum_v p_v Conv_x[conj(p_v) phi_u]:  target-spin orbital u, source v
      PairGrid ga{ntgt, nocc, 0, 1, 0, 0, 0, 1, 0, 1, 0, 0, 1};
      STATUS_TRY(pair_accumulate<T>(h, p_r, phit_r, p_r, Gt, ga, (const T*)B.kx, wa, st));
      // -alpha w sum_v phi_v Conv_x[conj(p_v) p_u]:  source-spin orbital u
      PairGrid gb{nocc, nocc, 0, 1, 0, 0, 0, 1, 0, 1, 0, 0, 1};
      STATUS_TRY(pair_accumulate<T>(h, p_r, p_r, phi_r, Gs, gb, (const T*)B.kx, wa, st));
    }
    // K1e: w p_u conj(W), W = Conv_H[drho] + f_xc drho (spin-flip: f_xc^SF drho only)
    { k_delta_rho<T><<<grid_for(n3, 256), 256, 0, st>>>(phi_r, p_r, drho, nocc, 1, n3); note_launch(); }
    if (sf) CUDA_TRY(cudaMemsetAsync(wb, 0, (size_t)n3 * sizeof(cplx<T>), st));
    else STATUS_TRY(convolve_fields<T>(h, drho, 1, (const T*)B.kh, T(1), wb, st));
    { k_add_fxc<T><<<grid_for(n3, 256), 256, 0, st>>>(wb, (const T*)B.fxc, drho, n3); note_launch(); }
    { k_grad_k1e<T><<<grid_for((long long)nocc * n3, 256), 256, 0, st>>>(p_r, wb, Gs, nocc, (T)w[b], n3); note_launch(); }
    STATUS_TRY(check_launch("adjoint k1e"));
    if (grad_vloc)
      { k_grad_vloc<T><<<grid_for(n3, 256), 256, 0, st>>>(p_r, nocc, w[b] * vol / (double)n3, grad_vloc, n3); note_launch(); }
  }
  STATUS_TRY(real_to_pw<T>(h, Gs, gfields, grad_phi, nullptr, st));

  // projector terms: -sum_k w_b(k) [ <x_k|phi_u> y_k + <y_k|phi_u> x_k ]
  CUDA_TRY(cudaMemcpyAsync(B.wdev, w, (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, st));
  cplx<T>* C = (cplx<T>*)B.cmat;
  cplx<T>* Cp = (cplx<T>*)B.cpart;
  cplx<T>* Ct = (cplx<T>*)B.ctmp;
  const int nsplit = h->nsplit;
  const int kchunk = ((npw + nsplit - 1) / nsplit + 15) / 16 * 16;
  for (int pass = 0; pass < 2; ++pass) {
    const cplx<T>* V = pass == 0 ? X : Y;        // overlap partner
    const cplx<T>* Wv = pass == 0 ? Y : X;       // vectors that get the coefficients
    dim3 g1((ntgt + 31) / 32, (unsigned)((rows + 31) / 32), nsplit);
    { k_overlap<T><<<g1, 256, 0, st>>>(phi, ntgt, V, (int)rows, npw, kchunk, Cp); note_launch(); }
    { k_reduce_split<T><<<grid_for((long long)ntgt * rows, 256), 256, 0, st>>>(Cp, nsplit, (long long)ntgt * rows, C); note_launch(); }
    { k_proj_grad_coef<T><<<grid_for((long long)ntgt * rows, 256), 256, 0, st>>>(C, ntgt, (int)rows, nocc, B.wdev, Ct); note_launch(); }
    dim3 g2((npw + 63) / 64, (ntgt + 31) / 32);
    { k_update<T><<<g2, 256, 0, st>>>(Wv, (int)rows, Ct, ntgt, npw, T(1), grad_t); note_launch(); }
  }
  return check_launch("adjoint projector terms");
}

static tddft_status apply_dispatch(tddft_system* h, int nb, const void* A, void* LA, unsigned mask, cudaStream_t st) {
  if (h->d.precision == TDDFT_PREC_FP64)
    return apply_impl<double>(h, nb, (const cplx<double>*)A, (cplx<double>*)LA, mask, st);
  return apply_impl<float>(h, nb, (const cplx<float>*)A, (cplx<float>*)LA, mask, st);
}

static tddft_status ensure_capture_stream(tddft_system* h) {
  if (!h->cap) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  return TDDFT_OK;
}

// Capture one apply of h into a graph (on h->cap), returning the graph.
static tddft_status capture_apply(tddft_system* h, int nb, const void* A, void* LA, cudaGraph_t* g) {
  STATUS_TRY(ensure_capture_stream(h));
  CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  tddft_status s = apply_dispatch(h, nb, A, LA, h->d.term_mask, h->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  if (s != TDDFT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(TDDFT_ECUDA, std::string("stream capture: ") + cudaGetErrorString(e));
  *g = graph;
  return TDDFT_OK;
}

static tddft_status apply_graph(tddft_system* h, int nb, const void* A, void* LA, cudaStream_t st) {
  if (!(h->gexec && h->g_nb == nb && h->g_A == A && h->g_LA == LA && h->g_mask == h->d.term_mask)) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    // work queued earlier on the caller's stream must finish before the
    // capture stream is used for the capture itself (capture launches nothing)
    cudaGraph_t g = nullptr;
    STATUS_TRY(capture_apply(h, nb, A, LA, &g));
    cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      return fail(TDDFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    h->g_nb = nb;
    h->g_A = A;
    h->g_LA = LA;
    h->g_mask = h->d.term_mask;
  }
  CUDA_TRY(cudaGraphLaunch(h->gexec, st));
  return TDDFT_OK;
}

// One graph for several systems: each system's apply is a branch forked from
// the first handle's capture stream, so that independent systems of uneven
// size run concurrently when replayed with a single graph launch.
namespace {
struct MultiKey {
  std::vector<const void*> k;
  bool operator==(const MultiKey& o) const { return k == o.k; }
};
struct MultiGraph {
  MultiKey key;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;
};
MultiGraph g_multi;

// Forget the captured graphs that contain h's launches.
void drop_graphs(tddft_system* h) {
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  if (g_multi.exec && std::find(g_multi.key.k.begin(), g_multi.key.k.end(), (const void*)h) != g_multi.key.k.end()) {
    cudaGraphExecDestroy(g_multi.exec);
    g_multi.exec = nullptr;
    g_multi.key.k.clear();
  }
}
}  // namespace

static tddft_status build_multi_graph(int nsys, const tddft_handle* hs, const int* nb, const void* const* A,
                                      void* const* LA, cudaGraphExec_t* out, std::vector<cudaEvent_t>& events) {
  for (int i = 0; i < nsys; ++i) STATUS_TRY(ensure_capture_stream(hs[i]));
  while ((int)events.size() < nsys + 1) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    events.push_back(e);
  }
  cudaStream_t origin = hs[0]->cap;
  CUDA_TRY(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
  tddft_status s = TDDFT_OK;
  cudaError_t e = cudaEventRecord(events[nsys], origin);
  for (int i = 0; i < nsys && s == TDDFT_OK && e == cudaSuccess; ++i) {
    cudaStream_t si = hs[i]->cap;
    if (si != origin) e = cudaStreamWaitEvent(si, events[nsys], 0);
    if (e != cudaSuccess) break;
    if (nb[i] > 0) s = apply_dispatch(hs[i], nb[i], A[i], LA[i], hs[i]->d.term_mask, si);
    if (s == TDDFT_OK && si != origin) {
      e = cudaEventRecord(events[i], si);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, events[i], 0);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
  if (s != TDDFT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(TDDFT_ECUDA, std::string("multi-system capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaError_t e3 = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return fail(TDDFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
  return TDDFT_OK;
}

// Reads (and clears) the device error flag; synchronises the stream.
static tddft_status check_device_flag(tddft_system* h, cudaStream_t st) {
  if (!h->b.dev_err) return TDDFT_OK;
  if (fault_take_wait()) {
    CUDA_TRY(cudaStreamSynchronize(st));
    return fail(TDDFT_ETIMEOUT, "a bounded device wait ran out (injected fault); results of the call are invalid");
  }
  int flag = 0;
  CUDA_TRY(cudaMemcpyAsync(&flag, h->b.dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (flag) {
    CUDA_TRY(cudaMemsetAsync(h->b.dev_err, 0, sizeof(int), st));
    return fail(TDDFT_ETIMEOUT, "a bounded device wait (tensor-core projector) ran out; results of the call are invalid");
  }
  return TDDFT_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* tddft_status_string(tddft_status s) {
  switch (s) {
    case TDDFT_OK: return "ok";
    case TDDFT_EINVAL: return "invalid argument";
    case TDDFT_ENOMEM: return "out of memory";
    case TDDFT_ECUDA: return "CUDA error";
    case TDDFT_ETIMEOUT: return "device wait timed out";
    case TDDFT_ENUMERIC: return "numerical failure";
    case TDDFT_ENOTCONV: return "not converged";
    case TDDFT_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char* tddft_last_error(void) { return g_last_error.c_str(); }

tddft_status tddft_sphere_size(int n, double a, double ecut, int* npw) {
  return abi_guard([&]() -> tddft_status {
    if (!npw) return fail(TDDFT_EINVAL, "null output");
    std::vector<Miller> s;
    STATUS_TRY(build_sphere(n, a, ecut, s));
    *npw = (int)s.size();
    return TDDFT_OK;
  });
}

tddft_status tddft_sphere_miller(int n, double a, double ecut, int* miller) {
  return abi_guard([&]() -> tddft_status {
    if (!miller) return fail(TDDFT_EINVAL, "null output");
    std::vector<Miller> s;
    STATUS_TRY(build_sphere(n, a, ecut, s));
    for (size_t i = 0; i < s.size(); ++i) {
      miller[3 * i] = s[i].x;
      miller[3 * i + 1] = s[i].y;
      miller[3 * i + 2] = s[i].z;
    }
    return TDDFT_OK;
  });
}

// Local exchange-correlation kernels from a ground-state spin density (host, FP64), for the local
// density approximation: Slater exchange, E_x = -(3/4)(6/pi)^(1/3) sum_sigma int rho_sigma^(4/3), and
// the Perdew-Zunger (1981) parametrisation of the correlation energy per electron with its
// spin interpolation eps_c = eps_U + f(zeta) (eps_P - eps_U).
namespace {
struct PzBranch {  // one of the two spin limits (U: unpolarised, P: fully polarised)
  double gamma, beta1, beta2, A, B, C, D;
};
constexpr PzBranch kPzU{-0.1423, 1.0529, 0.3334, 0.0311, -0.048, 0.0020, -0.0116};
constexpr PzBranch kPzP{-0.0843, 1.3981, 0.2611, 0.01555, -0.0269, 0.0007, -0.0048};

// eps(rs) and its first two derivatives of one branch
void pz_eps(const PzBranch& q, double rs, double* e, double* de, double* dde) {
  if (rs >= 1.0) {
    const double sr = std::sqrt(rs), den = 1.0 + q.beta1 * sr + q.beta2 * rs;
    const double g = 0.5 * q.beta1 / sr + q.beta2, dg = -0.25 * q.beta1 / (rs * sr);  // d den / d rs and its derivative
    *e = q.gamma / den;
    *de = -q.gamma * g / (den * den);
    *dde = -q.gamma * (dg / (den * den) - 2.0 * g * g / (den * den * den));
  } else {
    const double l = std::log(rs);
    *e = q.A * l + q.B + q.C * rs * l + q.D * rs;
    *de = q.A / rs + q.C * (l + 1.0) + q.D;
    *dde = -q.A / (rs * rs) + q.C / rs;
  }
}

// V_xc of both spins (Ha) and d V_xc,up / d rho_up (Ha bohr^3) at one point, in closed form;
// zero where the density vanishes
void lda_point(double ru, double rd, double* vu, double* vd, double* fuu) {
  ru = std::max(ru, 0.0);
  rd = std::max(rd, 0.0);
  const double rho = ru + rd;
  if (!(rho > 1e-14)) {
    *vu = *vd = *fuu = 0.0;
    return;
  }
  const double cx = std::cbrt(6.0 / M_PI);
  const double vxu = -cx * std::cbrt(ru), vxd = -cx * std::cbrt(rd);
  const double rs = std::cbrt(3.0 / (4.0 * M_PI * rho));
  const double zeta = std::min(1.0, std::max(-1.0, (ru - rd) / rho));
  const double den = 2.0 * std::cbrt(2.0) - 2.0;  // 2^(4/3) - 2
  const double zp = std::cbrt(1.0 + zeta), zm = std::cbrt(1.0 - zeta);
  const double f = ((1.0 + zeta) * zp + (1.0 - zeta) * zm - 2.0) / den;
  const double df = (4.0 / 3.0) * (zp - zm) / den;
  double eu, deu, ddeu, ep, dep, ddep;
  pz_eps(kPzU, rs, &eu, &deu, &ddeu);
  pz_eps(kPzP, rs, &ep, &dep, &ddep);
  // E(rs, zeta) = eps_U + f(zeta) (eps_P - eps_U) and its partial derivatives
  const double E = eu + f * (ep - eu), Er = deu + f * (dep - deu), Ez = df * (ep - eu);
  const double Err = ddeu + f * (ddep - ddeu), Erz = df * (dep - deu);
  // V_c,sigma = E - (rs/3) E_r + (s_sigma - zeta) E_z, s_up = +1, s_dn = -1
  const double base = E - rs / 3.0 * Er;
  *vu = vxu + base + (1.0 - zeta) * Ez;
  *vd = vxd + base - (1.0 + zeta) * Ez;
  // d V_c,up / d rho_up with d rs / d rho_up = -rs / (3 rho), d zeta / d rho_up = (1 - zeta) / rho:
  // dV/drs = (2/3) E_r - (rs/3) E_rr + (1 - zeta) E_rz, dV/dzeta = -(rs/3) E_rz + (1 - zeta) E_zz.
  // (1 - zeta)^2 E_zz stays finite as zeta -> 1; as zeta -> -1 (rho_up -> 0) it grows like the
  // exchange term, rho_up^(-2/3)
  double fx = 0.0, term_zz = 0.0;
  if (ru > 0.0) {
    fx = -(1.0 / 3.0) * cx * std::cbrt(ru) / ru;
    const double opz = 1.0 + zeta, omz = 1.0 - zeta;  // d^2 f / d zeta^2 = (4/9)((1+z)^(-2/3) + (1-z)^(-2/3)) / den
    const double a = opz > 0.0 ? 1.0 / (std::cbrt(opz) * std::cbrt(opz)) : 0.0;
    const double b = omz > 0.0 ? omz * omz / (std::cbrt(omz) * std::cbrt(omz)) : 0.0;  // (1-z)^(4/3)
    // (1 - zeta)^2 E_zz = (1 - zeta)^2 f''(zeta) (eps_P - eps_U)
    term_zz = (4.0 / 9.0) * (omz * omz * a + b) / den * (ep - eu);
  }
  const double dVdrs = (2.0 / 3.0) * Er - rs / 3.0 * Err + (1.0 - zeta) * Erz;
  const double dVdz_times_omz = -(rs / 3.0) * Erz * (1.0 - zeta) + term_zz;
  *fuu = ru > 0.0 ? fx + (dVdrs * (-rs / 3.0) + dVdz_times_omz) / rho : 0.0;  // diverges as rho_up -> 0
}
}  // namespace

tddft_status tddft_lda_kernels(long long npts, const double* rho_up, const double* rho_dn, double sf_cutoff,
                               double* vxc_up, double* vxc_dn, double* fxc, double* fxc_sf) {
  return abi_guard([&]() -> tddft_status {
    if (npts < 0 || !rho_up || !rho_dn) return fail(TDDFT_EINVAL, "need npts >= 0 and both densities");
    if (!(sf_cutoff >= 0.0)) return fail(TDDFT_EINVAL, "sf_cutoff must be >= 0");
    for (long long i = 0; i < npts; ++i) {
      if (!(rho_up[i] >= 0.0) || !(rho_dn[i] >= 0.0))
        return fail(TDDFT_EINVAL, "densities must be finite and non-negative (point " + std::to_string(i) + ")");
    }
    for (long long i = 0; i < npts; ++i) {
      const double ru = rho_up[i], rd = rho_dn[i];
      double vu, vd, fuu;
      lda_point(ru, rd, &vu, &vd, &fuu);
      if (vxc_up) vxc_up[i] = vu;
      if (vxc_dn) vxc_dn[i] = vd;
      if (fxc) fxc[i] = fuu;
      if (fxc_sf) {
        // spin-flip kernel (V_xc,up - V_xc,dn) / (rho_up - rho_dn), zero where the spin density is
        // below the cutoff (Sec. 2.3; the cutoff of the Supporting Information is 1e-3)
        const double sd = ru - rd;
        fxc_sf[i] = std::abs(sd) < sf_cutoff || sd == 0.0 ? 0.0 : (vu - vd) / sd;
      }
    }
    return TDDFT_OK;
  });
}

// Maximally localised orbitals at the Gamma point (host, FP64): the localised frame of the pair
// truncation of Sec. 3.2 (Eq. 31). Spread functional of a cubic cell (Resta; Silvestrelli):
// Omega = (a/2pi)^2 sum_alpha sum_n (1 - |Z^alpha_nn|^2), Z^alpha_mn = <phi_m| exp(i 2 pi r_alpha / a) |phi_n>,
// minimised over unitary rotations by maximising sum_alpha sum_n |Z^alpha_nn|^2, i.e. by the joint
// approximate diagonalisation of the six Hermitian matrices (Z + Z^H)/2, (Z - Z^H)/2i with complex
// Jacobi rotations in closed form (Cardoso and Souloumiac, SIAM J. Matrix Anal. Appl. 17, 161 (1996);
// for Wannier functions: Gygi, Fattebert and Schwegler, Comput. Phys. Commun. 155, 1 (2003)).
namespace {
using cd = std::complex<double>;

// eigenvector of the largest eigenvalue of a real symmetric 3 x 3 matrix (cyclic Jacobi)
void top_eigvec3(double A[3][3], double v[3]) {
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double th = 0.5 * std::atan2(2.0 * A[p][q], A[q][q] - A[p][p]);
        const double c = std::cos(th), s = std::sin(th);
        for (int k = 0; k < 3; ++k) {  // A <- J^T A J, J the rotation in the (p, q) plane
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int k = 1; k < 3; ++k)
    if (A[k][k] > A[best][best]) best = k;
  for (int k = 0; k < 3; ++k) v[k] = V[k][best];
}

// Z^alpha (alpha = x, y, z) of nocc plane-wave rows c [nocc][npw] on the sphere sph:
// Z_mn = sum_G conj(c_m(G)) c_n(G - b_alpha), the coefficients of exp(i b_alpha . r) phi_n being
// c_n(G - b_alpha); exact on the basis (both G and G - b_alpha on the sphere)
void position_matrices(int n, const std::vector<Miller>& sph, int nocc, const cd* c, std::vector<cd> Z[3]) {
  const int npw = (int)sph.size(), h = n / 2;
  std::vector<int> cube((size_t)n * n * n, -1);
  auto at = [n, h](int x, int y, int z) { return ((size_t)(z + h) * n + (y + h)) * n + (x + h); };
  for (int g = 0; g < npw; ++g) cube[at(sph[g].x, sph[g].y, sph[g].z)] = g;
  const int nthr = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  for (int al = 0; al < 3; ++al) {
    std::vector<int> sh(npw);
    for (int g = 0; g < npw; ++g) {
      int x = sph[g].x - (al == 0), y = sph[g].y - (al == 1), z = sph[g].z - (al == 2);
      sh[g] = (x < -h || y < -h || z < -h) ? -1 : cube[at(x, y, z)];
    }
    std::vector<cd> cs((size_t)nocc * npw);  // shifted rows
    for (int v = 0; v < nocc; ++v)
      for (int g = 0; g < npw; ++g) cs[(size_t)v * npw + g] = sh[g] >= 0 ? c[(size_t)v * npw + sh[g]] : cd(0.0, 0.0);
    Z[al].assign((size_t)nocc * nocc, cd(0.0, 0.0));
    std::vector<std::thread> pool;
    for (int t = 0; t < nthr; ++t)
      pool.emplace_back([&, t] {
        for (int m = t; m < nocc; m += nthr)
          for (int k = 0; k < nocc; ++k) {
            double re = 0.0, im = 0.0;
            const cd* a = c + (size_t)m * npw;
            const cd* b = cs.data() + (size_t)k * npw;
            for (int g = 0; g < npw; ++g) {  // conj(a) b
              re += a[g].real() * b[g].real() + a[g].imag() * b[g].imag();
              im += a[g].real() * b[g].imag() - a[g].imag() * b[g].real();
            }
            Z[al][(size_t)m * nocc + k] = cd(re, im);
          }
      });
    for (auto& th : pool) th.join();
  }
}

double spread_of(const std::vector<cd> M[6], int nocc, double a) {
  double s = 0.0;
  for (int al = 0; al < 3; ++al)
    for (int v = 0; v < nocc; ++v) {
      const double x = M[2 * al][(size_t)v * nocc + v].real(), y = M[2 * al + 1][(size_t)v * nocc + v].real();
      s += 1.0 - (x * x + y * y);
    }
  return s * (a / (2.0 * M_PI)) * (a / (2.0 * M_PI));
}
}  // namespace

tddft_status tddft_localize(int n, double a, double ecut, int nocc, const double* phi_pw, int max_sweeps, double tol,
                            double* U, double* spread, int* sweeps) {
  return abi_guard([&]() -> tddft_status {
    if (!phi_pw || !U) return fail(TDDFT_EINVAL, "null argument");
    if (nocc < 1 || max_sweeps < 0 || !(tol > 0.0)) return fail(TDDFT_EINVAL, "need nocc >= 1, max_sweeps >= 0, tol > 0");
    std::vector<Miller> sph;
    STATUS_TRY(build_sphere(n, a, ecut, sph));
    if ((int)sph.size() < nocc) return fail(TDDFT_EINVAL, "sphere smaller than the number of orbitals");
    std::vector<cd> Z[3];
    position_matrices(n, sph, nocc, reinterpret_cast<const cd*>(phi_pw), Z);
    // the six Hermitian matrices: Z = A + i B with A = (Z + Z^H)/2, B = (Z - Z^H)/2i
    std::vector<cd> M[6];
    for (int al = 0; al < 3; ++al) {
      M[2 * al].resize((size_t)nocc * nocc);
      M[2 * al + 1].resize((size_t)nocc * nocc);
      for (int i = 0; i < nocc; ++i)
        for (int j = 0; j < nocc; ++j) {
          const cd zij = Z[al][(size_t)i * nocc + j], zji = std::conj(Z[al][(size_t)j * nocc + i]);
          M[2 * al][(size_t)i * nocc + j] = 0.5 * (zij + zji);
          M[2 * al + 1][(size_t)i * nocc + j] = (zij - zji) / cd(0.0, 2.0);
        }
    }
    const double before = spread_of(M, nocc, a);
    // accumulated rotation, stored transposed (RT[n][v] = R_vn, w_n = sum_v R_vn phi_v) so that the
    // column updates of R run over contiguous memory
    std::vector<cd> RT((size_t)nocc * nocc, cd(0.0, 0.0));
    for (int i = 0; i < nocc; ++i) RT[(size_t)i * nocc + i] = 1.0;
    int done = 0;
    bool converged = max_sweeps == 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      double maxrot = 0.0;
      for (int i = 0; i < nocc; ++i)
        for (int j = i + 1; j < nocc; ++j) {
          // diagonal difference of every matrix after the rotation = h_k . v for a unit v; the best
          // v is the top eigenvector of G = sum_k h_k h_k^T, h_k = (M_ii - M_jj, 2 Re M_ij, 2 Im M_ij)
          double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          for (int k = 0; k < 6; ++k) {
            const std::vector<cd>& Mk = M[k];
            const double hk[3] = {Mk[(size_t)i * nocc + i].real() - Mk[(size_t)j * nocc + j].real(),
                                  2.0 * Mk[(size_t)i * nocc + j].real(), 2.0 * Mk[(size_t)i * nocc + j].imag()};
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) G[p][q] += hk[p] * hk[q];
          }
          double v[3];
          top_eigvec3(G, v);
          if (v[0] < 0.0) v[0] = -v[0], v[1] = -v[1], v[2] = -v[2];
          const double c = std::sqrt(0.5 * (1.0 + std::min(1.0, v[0])));
          const double sr = v[1] / (2.0 * c), si = -v[2] / (2.0 * c);  // s = sr + i si
          const double as = std::hypot(sr, si);
          if (!(as > 1e-15)) continue;
          maxrot = std::max(maxrot, as);
          // R = identity but R_ii = c, R_ji = s, R_ij = -conj(s), R_jj = c. Each M is Hermitian, so
          // M <- R^H M R is its rows i, j updated (row i <- c row i + conj(s) row j, row j <- -s row i
          // + c row j) off the 2 x 2 block, the columns i, j their conjugates, and the block itself
          for (int k = 0; k < 6; ++k) {
            cd* X = M[k].data();
            cd* Xi = X + (size_t)i * nocc;
            cd* Xj = X + (size_t)j * nocc;
            const cd a = Xi[i], b = Xi[j], d = Xj[j];
            for (int q = 0; q < nocc; ++q) {
              const double air = Xi[q].real(), aii = Xi[q].imag(), bjr = Xj[q].real(), bji = Xj[q].imag();
              const double nir = c * air + sr * bjr + si * bji, nii = c * aii + sr * bji - si * bjr;
              const double njr = -sr * air + si * aii + c * bjr, nji = -sr * aii - si * air + c * bji;
              Xi[q] = cd(nir, nii);
              Xj[q] = cd(njr, nji);
              X[(size_t)q * nocc + i] = cd(nir, -nii);
              X[(size_t)q * nocc + j] = cd(njr, -nji);
            }
            // the 2 x 2 block: M'_ii = c^2 a + |s|^2 d + 2c Re(s b), M'_jj = |s|^2 a + c^2 d - 2c Re(s b),
            // M'_ij = c^2 b - conj(s)^2 conj(b) + c conj(s) (d - a)
            const cd sc(sr, -si);  // conj(s)
            const double resb = sr * b.real() - si * b.imag();
            const double s2 = sr * sr + si * si;
            const double mii = c * c * a.real() + s2 * d.real() + 2.0 * c * resb;
            const double mjj = s2 * a.real() + c * c * d.real() - 2.0 * c * resb;
            const cd mij = c * c * b - sc * sc * std::conj(b) + c * sc * (d - a);
            Xi[i] = mii;
            Xj[j] = mjj;
            Xi[j] = mij;
            Xj[i] = std::conj(mij);
          }
          // R_total <- R_total R: columns i, j of R = rows i, j of RT
          cd* Ri = RT.data() + (size_t)i * nocc;
          cd* Rj = RT.data() + (size_t)j * nocc;
          for (int p = 0; p < nocc; ++p) {
            const double xr = Ri[p].real(), xi_ = Ri[p].imag(), yr = Rj[p].real(), yi = Rj[p].imag();
            Ri[p] = cd(c * xr + sr * yr - si * yi, c * xi_ + sr * yi + si * yr);   // c x + s y
            Rj[p] = cd(-sr * xr - si * xi_ + c * yr, -sr * xi_ + si * xr + c * yi);  // -conj(s) x + c y
          }
        }
      done = sweep + 1;
      if (maxrot < tol) {
        converged = true;
        break;
      }
    }
    std::vector<cd> R((size_t)nocc * nocc);
    for (int n = 0; n < nocc; ++n)
      for (int v = 0; v < nocc; ++v) R[(size_t)v * nocc + n] = RT[(size_t)n * nocc + v];
    // the library's convention for the localised frame: phi_v = sum_n U_vn phi~_n, so U = conj(R)
    cd* u = reinterpret_cast<cd*>(U);
    for (size_t e = 0; e < R.size(); ++e) u[e] = std::conj(R[e]);
    if (spread) {
      spread[0] = before;
      spread[1] = spread_of(M, nocc, a);
    }
    if (sweeps) *sweeps = done;
    return converged ? TDDFT_OK : fail(TDDFT_ENOTCONV, "localisation sweeps did not converge (U is the last iterate)");
  });
}

tddft_status tddft_exchange_grid(int n, double a, double ecut, int precision, int* n_exchange) {
  return abi_guard([&]() -> tddft_status {
    if (!n_exchange) return fail(TDDFT_EINVAL, "null output");
    if (precision != TDDFT_PREC_FP64 && precision != TDDFT_PREC_FP32) return fail(TDDFT_EINVAL, "unknown precision");
    if (!supported_n(n, precision)) return fail(TDDFT_EINVAL, "unsupported grid size " + std::to_string(n));
    std::vector<Miller> s;
    STATUS_TRY(build_sphere(n, a, ecut, s));
    *n_exchange = exchange_grid_for(n, precision, s);
    return TDDFT_OK;
  });
}

tddft_status tddft_profile_enable(int enable) {
  return abi_guard([&]() -> tddft_status {
    g_prof.on = enable != 0;
    g_prof.used = 0;
    return TDDFT_OK;
  });
}

tddft_status tddft_profile_read(double* ms, long long* launches, double* bytes, long long* total_launches) {
  return abi_guard([&]() -> tddft_status {
    if (total_launches) *total_launches = g_prof.launches;
    for (int c = 0; c < TDDFT_PROFILE_CLASSES; ++c) {
      if (ms) ms[c] = 0.0;
      if (launches) launches[c] = 0;
      if (bytes) bytes[c] = 0.0;
    }
    for (size_t i = 0; i < g_prof.used; ++i) {
      CUDA_TRY(cudaEventSynchronize(g_prof.pool[2 * i + 1]));
      float t = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&t, g_prof.pool[2 * i], g_prof.pool[2 * i + 1]));
      const int c = g_prof.cls[i];
      if (ms) ms[c] += t;
      if (launches) launches[c] += 1;
      if (bytes) bytes[c] += g_prof.bytes[i];
    }
    return TDDFT_OK;
  });
}

tddft_status tddft_destroy(tddft_handle h) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return TDDFT_OK;
    // a cached multi-system graph that refers to this handle is dropped
    if (g_multi.exec && std::find(g_multi.key.k.begin(), g_multi.key.k.end(), (const void*)h) != g_multi.key.k.end()) {
      cudaGraphExecDestroy(g_multi.exec);
      g_multi.exec = nullptr;
      g_multi.key.k.clear();
    }
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (void* p : h->allocations) cudaFree(p);
    if (h->tau_cache) cudaFree(h->tau_cache);
    if (h->tau_all) cudaFree(h->tau_all);
    if (h->tc_pack) cudaFree(h->tc_pack);
    if (h->xsub) tddft_destroy(h->xsub);
    delete h;
    return TDDFT_OK;
  });
}

tddft_status tddft_init_system(const tddft_desc* desc, const tddft_inputs* in, void* stream, tddft_handle* out) {
  return abi_guard([&]() -> tddft_status {
    if (!desc || !in || !out) return fail(TDDFT_EINVAL, "null argument");
    *out = nullptr;
    const tddft_desc& d = *desc;
    if (d.spin_mode != TDDFT_SPIN_CONSERVING && d.spin_mode != TDDFT_SPIN_FLIP)
      return fail(TDDFT_EINVAL, "unknown spin mode");
    if (d.precision != TDDFT_PREC_FP64 && d.precision != TDDFT_PREC_FP32) return fail(TDDFT_EINVAL, "unknown precision");
    if (!supported_n(d.n, d.precision)) return fail(TDDFT_EINVAL, "unsupported grid size " + std::to_string(d.n));
    if (d.nocc_src < 1 || d.nb_max < 1) return fail(TDDFT_EINVAL, "nocc_src and nb_max must be >= 1");
    if (d.spin_mode == TDDFT_SPIN_CONSERVING && d.nocc_tgt != d.nocc_src)
      return fail(TDDFT_EINVAL, "spin-conserving systems need nocc_tgt == nocc_src");
    if (d.nocc_tgt < 1) return fail(TDDFT_EINVAL, "nocc_tgt must be >= 1");
    if (d.term_mask & ~TDDFT_TERMS_ZVEC) return fail(TDDFT_EINVAL, "unknown term bits");
    if (d.spin_mode == TDDFT_SPIN_FLIP && (d.term_mask & ~TDDFT_TERMS_ALL))
      return fail(TDDFT_ENOTSUP, "K2 terms are implemented for spin-conserving systems");
    if (!in->phi_src || !in->eps_src) return fail(TDDFT_EINVAL, "orbitals and eigenvalues are required");
    if (d.spin_mode == TDDFT_SPIN_FLIP && !in->phi_tgt) return fail(TDDFT_EINVAL, "spin-flip needs phi_tgt");
    std::vector<Miller> sph;
    STATUS_TRY(build_sphere(d.n, d.a, d.ecut, sph));
    if ((int)sph.size() < std::max(d.nocc_src, d.nocc_tgt))
      return fail(TDDFT_EINVAL, "sphere smaller than the number of orbitals");
    tddft_system* h = new tddft_system();
    h->d = d;
    h->n = d.n;
    h->n3 = (long long)d.n * d.n * d.n;
    h->npw = (int)sph.size();
    cudaStream_t st = (cudaStream_t)stream;
    tddft_status s = d.precision == TDDFT_PREC_FP64 ? init_impl<double>(h, in, st) : init_impl<float>(h, in, st);
    if (s != TDDFT_OK) {
      std::string msg = g_last_error;
      tddft_destroy(h);
      g_last_error = msg;
      return s;
    }
    const int nx = exchange_grid_for(d.n, d.precision, sph);
    if (nx < d.n) {
      // the exchange terms on the nx grid: an internal system with the same orbitals and no
      // local fields; without room for it the n grid serves (same result, more points)
      tddft_desc dx = d;
      dx.n = nx;
      tddft_inputs ix = *in;
      ix.vloc = nullptr;
      ix.fxc = nullptr;
      const std::string saved = g_last_error;
      tddft_handle hx = nullptr;
      if (tddft_init_system(&dx, &ix, stream, &hx) == TDDFT_OK) {
        void* xpw = nullptr;
        // the same sphere in the same order (it fits: N_x > 4M), so plane-wave rows are shared
        if (hx->npw == h->npw && dalloc(h, &xpw, (size_t)d.nb_max * d.nocc_src * h->npw * h->esz()) == TDDFT_OK) {
          h->xsub = hx;
          h->x_pw = xpw;
        } else {
          tddft_destroy(hx);
        }
      }
      g_last_error = saved;
    }
    *out = h;
    return TDDFT_OK;
  });
}

tddft_status tddft_query(tddft_handle h, tddft_info* info) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !info) return fail(TDDFT_EINVAL, "null argument");
    STATUS_TRY(check_device_flag(h, nullptr));
    info->npw = h->npw;
    info->n = h->n;
    info->nb_chunk = h->nb_chunk;
    info->precision = h->d.precision;
    info->device_bytes = h->bytes;
    info->n_exchange = h->n;
    if (h->xsub) {
      STATUS_TRY(check_device_flag(h->xsub, nullptr));
      info->device_bytes += h->xsub->bytes;
      if (h->use_xsub) info->n_exchange = h->xsub->n;
    }
    return TDDFT_OK;
  });
}

tddft_status tddft_set_terms(tddft_handle h, unsigned term_mask) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (term_mask & ~TDDFT_TERMS_ZVEC) return fail(TDDFT_EINVAL, "unknown term bits");
    if (h->sf() && (term_mask & ~TDDFT_TERMS_ALL))
      return fail(TDDFT_ENOTSUP, "K2 terms are implemented for spin-conserving systems");
    h->d.term_mask = term_mask;  // a cached graph is re-captured when the mask differs
    return TDDFT_OK;
  });
}

// tuning.k1d_cache: build the stored tau (synchronises) or release them
static tddft_status set_tau_cache(tddft_system* h, bool on) {
  if (!on) {
    if (h->tau_cache) {
      CUDA_TRY(cudaFree(h->tau_cache));
      h->bytes -= h->tau_cache_bytes;
    }
    h->tau_cache = nullptr;
    h->tau_cache_bytes = 0;
    h->k1d_cache = false;
    return TDDFT_OK;
  }
  if (h->tau_cache) {
    h->k1d_cache = true;
    return TDDFT_OK;
  }
  // the source orbitals must be the given ones (the localised frame replaces them while it is on)
  if (h->loc_on) return fail(TDDFT_ENOTSUP, "stored tau are built in the given frame: switch localisation off first");
  const size_t bytes = tau_cache_fields(h->d.nocc_src) * (size_t)h->n3 * h->esz();
  cudaError_t e = lib_malloc(&h->tau_cache, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->tau_cache = nullptr;
    return fail(TDDFT_ENOMEM, "stored tau: " + alloc_error(bytes, e));
  }
  h->tau_cache_bytes = bytes;
  h->bytes += bytes;
  tddft_status s = ensure_capture_stream(h);
  if (s == TDDFT_OK) {
    // work queued on other streams (orbital loads) completes first; the build runs on the handle's stream
    cudaError_t e2 = cudaDeviceSynchronize();
    if (e2 != cudaSuccess) s = fail(TDDFT_ECUDA, std::string("before the tau build: ") + cudaGetErrorString(e2));
  }
  if (s == TDDFT_OK)
    s = h->d.precision == TDDFT_PREC_FP64 ? build_tau_cache<double>(h, h->cap) : build_tau_cache<float>(h, h->cap);
  if (s == TDDFT_OK) {
    cudaError_t e3 = cudaStreamSynchronize(h->cap);
    if (e3 != cudaSuccess) s = fail(TDDFT_ECUDA, std::string("tau build: ") + cudaGetErrorString(e3));
  }
  if (s != TDDFT_OK) {
    cudaFree(h->tau_cache);
    h->bytes -= bytes;
    h->tau_cache = nullptr;
    h->tau_cache_bytes = 0;
    return s;
  }
  h->k1d_cache = true;
  return TDDFT_OK;
}

// the stored tau where K1d runs (the exchange-grid system when it is in use), none elsewhere
static tddft_status sync_tau_cache(tddft_system* h) {
  tddft_system* run = (h->xsub && h->use_xsub) ? h->xsub : h;
  tddft_system* idle = run == h ? h->xsub : h;
  if (idle) STATUS_TRY(set_tau_cache(idle, false));
  const tddft_status s = set_tau_cache(run, h->k1d_cache_req);
  if (s != TDDFT_OK) h->k1d_cache_req = false;
  return s;
}

static bool z_kernel_ok(const tddft_system* h, int z) {
  const bool reg = h->d.precision == TDDFT_PREC_FP32 ? h->ops32.reg_ok : h->ops64.reg_ok;
  const bool pair = h->d.precision == TDDFT_PREC_FP32 ? h->ops32.pair_ok : h->ops64.pair_ok;
  return z == 0 || (z == 1 && reg) || (z == 2 && pair);
}

tddft_status tddft_set_tuning(tddft_handle h, const tddft_tuning* t) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !t) return fail(TDDFT_EINVAL, "null argument");
    if (t->targets < 0 || t->sources < 0 || t->k1d_block < 0 || t->k1d_block > 16)
      return fail(TDDFT_EINVAL, "tile sizes must be >= 0 and k1d_block <= 16");
    if (t->accumulate < -1 || t->accumulate > 1) return fail(TDDFT_EINVAL, "accumulate must be -1, 0 or 1");
    if (t->graph < -1 || t->graph > 1) return fail(TDDFT_EINVAL, "graph must be -1, 0 or 1");
    if (t->targets) h->tile_targets = t->targets;
    if (t->sources) h->tile_sources = t->sources;
    if (t->k1d_block) h->k1d_block = t->k1d_block;
    if (t->accumulate >= 0) h->accumulate = t->accumulate == 1 ? INV_ATOMIC : INV_ACCUM;
    if (t->graph >= 0) h->use_graph = t->graph == 1;
    if (t->prune >= 0) {
      if (t->prune > 1) return fail(TDDFT_EINVAL, "prune must be 0 or 1");
      h->prune = t->prune == 1;
    }
    if (t->projector >= 0) {
      if (t->projector > 2) return fail(TDDFT_EINVAL, "projector must be 0, 1 or 2");
      h->projector_tc = t->projector;
    }
    if (t->k1d_sparse >= 0) {
      if (t->k1d_sparse > 2) return fail(TDDFT_EINVAL, "k1d_sparse must be 0, 1 or 2");
      h->k1d_sparse = t->k1d_sparse;
    }
    if (t->z_kernel >= 0) {
      if (t->z_kernel > 2) return fail(TDDFT_EINVAL, "z_kernel must be 0, 1 or 2");
      const bool reg = h->d.precision == TDDFT_PREC_FP32 ? h->ops32.reg_ok : h->ops64.reg_ok;
      const bool pair = h->d.precision == TDDFT_PREC_FP32 ? h->ops32.pair_ok : h->ops64.pair_ok;
      if (t->z_kernel == 1 && !reg) return fail(TDDFT_EINVAL, "the register-resident z pass needs FP32 and n <= 80");
      if (t->z_kernel == 2 && !pair)
        return fail(TDDFT_EINVAL, "the paired z pass needs FP32, n <= 80 or n = 96, and a supported n / 2");
      h->ops32.kc.z = t->z_kernel;
      h->ops64.kc.z = t->z_kernel;
    }
    if (t->k1d_all >= 0) {
      if (t->k1d_all > 1) return fail(TDDFT_EINVAL, "k1d_all must be 0 or 1");
      h->k1d_all = t->k1d_all == 1;
      if (!h->k1d_all && h->tau_all) {
        CUDA_TRY(cudaDeviceSynchronize());
        CUDA_TRY(cudaFree(h->tau_all));
        h->bytes -= h->tau_all_bytes;
        h->tau_all = nullptr;
        h->tau_all_bytes = 0;
      }
      h->tau_all_tried = false;
    }
    if (t->xy_kernel >= 0) {
      if (t->xy_kernel > 3) return fail(TDDFT_EINVAL, "xy_kernel must be 0, 1, 2 or 3");
      h->xy_lines = t->xy_kernel;
    }
    tddft_status cs = TDDFT_OK;
    if (t->exchange_grid > 1) cs = fail(TDDFT_EINVAL, "exchange_grid must be 0 or 1");
    if (t->k1d_cache > 1) cs = fail(TDDFT_EINVAL, "k1d_cache must be 0 or 1");
    if (cs == TDDFT_OK && h->xsub) {
      // the same schedule for the exchange-grid system (its z pass where that grid has it)
      tddft_tuning tx = *t;
      tx.k1d_cache = -1;
      tx.exchange_grid = -1;
      if (tx.z_kernel >= 0 && !z_kernel_ok(h->xsub, tx.z_kernel)) tx.z_kernel = -1;
      cs = tddft_set_tuning(h->xsub, &tx);
    }
    if (cs == TDDFT_OK && (t->exchange_grid >= 0 || t->k1d_cache >= 0)) {
      if (t->exchange_grid >= 0) h->use_xsub = t->exchange_grid == 1;
      if (t->k1d_cache >= 0) h->k1d_cache_req = t->k1d_cache == 1;
      cs = sync_tau_cache(h);
    }
    drop_graphs(h);  // the schedule changed: the next graph call captures again
    return cs;
  });
}

tddft_status tddft_get_tuning(tddft_handle h, tddft_tuning* t) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !t) return fail(TDDFT_EINVAL, "null argument");
    t->targets = h->tile_targets;
    t->sources = h->tile_sources;
    t->k1d_block = h->k1d_block;
    t->accumulate = h->accumulate == INV_ATOMIC ? 1 : 0;
    t->batch_fields = h->ibuf_fields;
    t->graph = h->use_graph ? 1 : 0;
    const KernelChoice kc = h->d.precision == TDDFT_PREC_FP32 ? h->ops32.kc : h->ops64.kc;
    t->prune = h->prune ? 1 : 0;
    t->z_kernel = kc.z;
    t->projector = h->projector_tc;
    t->k1d_sparse = h->k1d_sparse;
    t->k1d_cache = h->k1d_cache_req ? 1 : 0;
    t->exchange_grid = h->use_xsub ? 1 : 0;
    t->xy_kernel = h->xy_lines;
    t->k1d_all = h->k1d_all ? 1 : 0;
    return TDDFT_OK;
  });
}

tddft_status tddft_apply_liouville(tddft_handle h, int nb, const void* A, void* LA, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (nb < 0 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [0, nb_max]");
    if (nb == 0) return TDDFT_OK;
    if (!A || !LA) return fail(TDDFT_EINVAL, "null buffer");
    if (A == LA) return fail(TDDFT_EINVAL, "A and LA must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->use_graph) return apply_graph(h, nb, A, LA, st);
    return apply_dispatch(h, nb, A, LA, h->d.term_mask, st);
  });
}

tddft_status tddft_apply_liouville_host(tddft_handle h, int nb, const void* A_host, void* LA_host, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (nb < 0 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [0, nb_max]");
    if (nb == 0) return TDDFT_OK;
    if (!A_host || !LA_host) return fail(TDDFT_EINVAL, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)nb * h->d.nocc_src * h->npw * h->esz();
    CUDA_TRY(cudaMemcpyAsync(h->b.io_a, A_host, bytes, cudaMemcpyHostToDevice, st));
    STATUS_TRY(tddft_apply_liouville(h, nb, h->b.io_a, h->b.io_b, stream));
    CUDA_TRY(cudaMemcpyAsync(LA_host, h->b.io_b, bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return check_device_flag(h, st);
  });
}

tddft_status tddft_apply_liouville_multi(int nsys, const tddft_handle* hs, const int* nb, const void* const* A,
                                         void* const* LA, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (nsys < 1 || !hs || !nb || !A || !LA) return fail(TDDFT_EINVAL, "null or empty argument");
    for (int i = 0; i < nsys; ++i) {
      if (!hs[i]) return fail(TDDFT_EINVAL, "null handle in the list");
      if (nb[i] < 0 || nb[i] > hs[i]->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [0, nb_max] for system " + std::to_string(i));
      if (nb[i] > 0 && (!A[i] || !LA[i] || A[i] == LA[i])) return fail(TDDFT_EINVAL, "bad buffers for system " + std::to_string(i));
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) return fail(TDDFT_EINVAL, "a handle appears twice (one workspace per handle)");
    }
    MultiKey key;
    for (int i = 0; i < nsys; ++i) {
      key.k.push_back(hs[i]);
      key.k.push_back((const void*)(size_t)nb[i]);
      key.k.push_back(A[i]);
      key.k.push_back(LA[i]);
      key.k.push_back((const void*)(size_t)hs[i]->d.term_mask);
    }
    if (!(g_multi.exec && g_multi.key == key)) {
      if (g_multi.exec) {
        cudaGraphExecDestroy(g_multi.exec);
        g_multi.exec = nullptr;
      }
      STATUS_TRY(build_multi_graph(nsys, hs, nb, A, LA, &g_multi.exec, g_multi.events));
      g_multi.key = key;
    }
    CUDA_TRY(cudaGraphLaunch(g_multi.exec, (cudaStream_t)stream));
    return TDDFT_OK;
  });
}

tddft_status tddft_ace_build(tddft_handle h, int n_extra, const double* extra, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (n_extra < 0 || (n_extra > 0 && !extra)) return fail(TDDFT_EINVAL, "bad extra rows");
    if (h->d.nocc_tgt + n_extra > h->npw) return fail(TDDFT_EINVAL, "more ACE vectors than plane waves");
    cudaStream_t st = (cudaStream_t)stream;
    drop_graphs(h);  // a captured graph would keep the old exchange path
    if (h->d.precision == TDDFT_PREC_FP64) return ace_build_impl<double>(h, n_extra, extra, st);
    return ace_build_impl<float>(h, n_extra, extra, st);
  });
}

tddft_status tddft_set_localization(tddft_handle h, const double* U, double s_thr, double* S, int* kept_pairs,
                                    void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (U && !(s_thr >= 0.0)) return fail(TDDFT_EINVAL, "s_thr must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d.precision == TDDFT_PREC_FP64) return localization_impl<double>(h, U, s_thr, S, kept_pairs, st);
    return localization_impl<float>(h, U, s_thr, S, kept_pairs, st);
  });
}

tddft_status tddft_ace_enable(tddft_handle h, int enable) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (enable && !h->ace_xi) return fail(TDDFT_EINVAL, "ACE has not been built");
    h->ace_on = enable != 0;
    drop_graphs(h);
    return TDDFT_OK;
  });
}

tddft_status tddft_autotune(tddft_handle h, int nb, const void* A, void* LA, void* stream, tddft_tuning* best) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !A || !LA) return fail(TDDFT_EINVAL, "null argument");
    if (nb < 1 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [1, nb_max]");
    cudaStream_t st = (cudaStream_t)stream;
    struct Cand {
      int tt, ks, acc, kb;
    };
    const Cand cands[] = {{64, 8, 1, 16}, {128, 8, 1, 16}, {32, 8, 1, 16}, {64, 16, 1, 16}, {16, 8, 1, 16},
                          {32, 4, 1, 16}, {32, 8, 0, 16}, {8, 8, 1, 8}};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const bool graph = h->use_graph;
    h->use_graph = false;
    float best_ms = 1e30f;
    Cand bc = cands[0];
    tddft_status s = TDDFT_OK;
    auto set_tiles = [h](const Cand& c) {
      for (tddft_system* x : {h, h->xsub}) {
        if (!x) continue;
        x->tile_targets = c.tt;
        x->tile_sources = c.ks;
        x->accumulate = c.acc ? INV_ATOMIC : INV_ACCUM;
        x->k1d_block = c.kb;
      }
    };
    for (const Cand& c : cands) {
      set_tiles(c);
      s = apply_dispatch(h, nb, A, LA, h->d.term_mask, st);  // warm
      if (s != TDDFT_OK) break;
      cudaEventRecord(e0, st);
      s = apply_dispatch(h, nb, A, LA, h->d.term_mask, st);
      if (s != TDDFT_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        s = fail(TDDFT_ECUDA, "autotune timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        bc = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->use_graph = graph;
    set_tiles(bc);
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    if (s != TDDFT_OK) return s;
    if (best) STATUS_TRY(tddft_get_tuning(h, best));
    return TDDFT_OK;
  });
}

tddft_status tddft_apply_liouville_adjoint(tddft_handle h, int nb, const void* X, const double* w, double* omega,
                                           void* grad_phi, double* grad_vloc, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (h->ace_on) return fail(TDDFT_ENOTSUP, "the adjoint differentiates the exact exchange; disable ACE first");
    if (h->loc_on) return fail(TDDFT_ENOTSUP, "the adjoint differentiates the exact K1d; disable the localised frame first");
    if (nb < 1 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [1, nb_max]");
    if (!X || !w || !omega || !grad_phi) return fail(TDDFT_EINVAL, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d.precision == TDDFT_PREC_FP64)
      return adjoint_impl<double>(h, nb, (const cplx<double>*)X, w, omega, (cplx<double>*)grad_phi, grad_vloc, st);
    return adjoint_impl<float>(h, nb, (const cplx<float>*)X, w, omega, (cplx<float>*)grad_phi, grad_vloc, st);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// density responses of the force expression (Sec. 2.2, Sec. 2.3)
// ---------------------------------------------------------------------------

// out[r] += s * sum_v Re(conj(f_v(r)) g_v(r))
template <typename T>
__global__ void k_density_accum(const cplx<T>* __restrict__ f, const cplx<T>* __restrict__ g, int nocc, double s,
                                double* __restrict__ out, long long n3) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n3; r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int v = 0; v < nocc; ++v) {
      const cplx<T> a = f[(long long)v * n3 + r], b = g[(long long)v * n3 + r];
      acc += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
    }
    out[r] += s * acc;
  }
}

template <typename T>
static tddft_status relaxed_density_impl(tddft_system* h, int nb, const cplx<T>* X, const cplx<T>* Z, const double* w,
                                         double* drho, cudaStream_t st) {
  const int nocc = h->d.nocc_src, npw = h->npw;
  const long long n3 = h->n3, len = (long long)nocc * npw;
  const bool sf = h->sf();
  CUDA_TRY(cudaMemsetAsync(drho, 0, (size_t)(sf ? 2 : 1) * n3 * sizeof(double), st));
  cplx<T>* a_r = (cplx<T>*)h->b.a_r;
  cplx<T>* f_r = (cplx<T>*)h->b.out_r;
  cplx<T>* psi = (cplx<T>*)h->b.io_a;
  const cplx<T>* phi_r = (const cplx<T>*)h->b.phi_src_r;
  std::vector<cplx<T>> S((size_t)nocc * nocc), St(S.size());
  cplx<T>* C = (cplx<T>*)h->b.cmat;
  for (int b = 0; b < nb; ++b) {
    if (w[b] == 0.0) continue;
    const cplx<T>* Xb = X + b * len;
    // sum_v |a_v|^2: the target-spin channel (channel 0)
    STATUS_TRY(pw_to_real<T>(h, Xb, nocc, a_r, st));
    { k_density_accum<T><<<grid_for(n3, 256), 256, 0, st>>>(a_r, a_r, nocc, w[b], drho, n3); note_launch(); }
    // -sum_vv' conj(phi_v) phi_v' <a_v|a_v'>: psi_v = sum_v' <a_v|a_v'> phi_v' in plane waves
    STATUS_TRY(gemm_overlap<T>(h, Xb, nocc, Xb, nocc, (cplx<T>*)h->b.cpart, C, st));  // C[u][r] = <a_u|a_r>
    CUDA_TRY(cudaMemcpyAsync(S.data(), C, S.size() * sizeof(cplx<T>), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int v = 0; v < nocc; ++v)
      for (int vp = 0; vp < nocc; ++vp) St[(size_t)vp * nocc + v] = S[(size_t)v * nocc + vp];  // [v'][v] = <a_v|a_v'>
    CUDA_TRY(cudaMemcpyAsync(C, St.data(), St.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(psi, 0, (size_t)len * sizeof(cplx<T>), st));
    STATUS_TRY(gemm_update<T>(h, (const cplx<T>*)h->b.phi_src_pw, nocc, C, psi, nocc, T(1), st));
    STATUS_TRY(pw_to_real<T>(h, psi, nocc, f_r, st));
    { k_density_accum<T><<<grid_for(n3, 256), 256, 0, st>>>(phi_r, f_r, nocc, -w[b], sf ? drho + n3 : drho, n3);
      note_launch(); }
    if (Z) {  // 2 Re sum_v conj(phi_v) Z_v
      STATUS_TRY(pw_to_real<T>(h, Z + b * len, nocc, f_r, st));
      { k_density_accum<T><<<grid_for(n3, 256), 256, 0, st>>>(phi_r, f_r, nocc, 2.0 * w[b], drho, n3); note_launch(); }
    }
    STATUS_TRY(check_launch("relaxed density"));
  }
  return TDDFT_OK;
}

extern "C" tddft_status tddft_relaxed_density(tddft_handle h, int nb, const void* X, const void* Z, const double* w,
                                              double* drho, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (nb < 1 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [1, nb_max]");
    if (!X || !w || !drho) return fail(TDDFT_EINVAL, "null buffer");
    if (Z && h->sf()) return fail(TDDFT_ENOTSUP, "the Z-vector part is implemented for spin-conserving systems");
    if (h->loc_on) return fail(TDDFT_ENOTSUP, "disable the localised frame first (the density uses the given orbitals)");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d.precision == TDDFT_PREC_FP64)
      return relaxed_density_impl<double>(h, nb, (const cplx<double>*)X, (const cplx<double>*)Z, w, drho, st);
    return relaxed_density_impl<float>(h, nb, (const cplx<float>*)X, (const cplx<float>*)Z, w, drho, st);
  });
}

// ---------------------------------------------------------------------------
// Z-vector equation (Eq. 19) by conjugate gradients with the inexact Krylov
// switch (Sec. 3.3)
// ---------------------------------------------------------------------------

// per state b (rows of length len): Z_b += step_b p_b, r_b -= step_b q_b
template <typename T>
__global__ void k_zv_step(cplx<T>* __restrict__ Z, cplx<T>* __restrict__ r, const cplx<T>* __restrict__ p,
                          const cplx<T>* __restrict__ q, const double* __restrict__ step, long long len,
                          long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const double a = step[i / len];
    if (a == 0.0) continue;
    const cplx<T> pv = p[i], qv = q[i];
    Z[i] = {(T)(Z[i].x + a * pv.x), (T)(Z[i].y + a * pv.y)};
    r[i] = {(T)(r[i].x - a * qv.x), (T)(r[i].y - a * qv.y)};
  }
}

// per state b that moved (step_b != 0): p_b = s_b + beta_b p_b
template <typename T>
__global__ void k_zv_direction(cplx<T>* __restrict__ p, const cplx<T>* __restrict__ sv, const double* __restrict__ beta,
                               const double* __restrict__ step, long long len, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    if (step[i / len] == 0.0) continue;
    const double bt = beta[i / len];
    p[i] = {(T)(sv[i].x + bt * p[i].x), (T)(sv[i].y + bt * p[i].y)};
  }
}

// s = r / d, d = |G|^2/2 - eps_v with |d| clamped to >= 0.1 Ha (sign kept); rows [nb][nocc][npw]
template <typename T>
__global__ void k_zv_precondition(const cplx<T>* __restrict__ r, const T* __restrict__ g2h, const T* __restrict__ eps,
                                  int nocc, int npw, long long total, cplx<T>* __restrict__ sv) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / npw, g = i - row * npw;
    double d = (double)g2h[g] - (double)eps[row % nocc];
    if (fabs(d) < 0.1) d = d < 0.0 ? -0.1 : 0.1;
    sv[i] = {(T)(r[i].x / d), (T)(r[i].y / d)};
  }
}

template <typename T>
__global__ void k_negate(cplx<T>* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = {-x[i].x, -x[i].y};
}

// Terms of the exact Z-vector operator for the handle's Tamm-Dancoff mask: the
// K2 counterpart of every K1 term that is switched on.
static unsigned zvector_mask(unsigned m) {
  m &= TDDFT_TERMS_ALL;
  if (m & TDDFT_TERM_K1E_H) m |= TDDFT_TERM_K2E_H;
  if (m & TDDFT_TERM_K1E_XC) m |= TDDFT_TERM_K2E_XC;
  if (m & TDDFT_TERM_K1D) m |= TDDFT_TERM_K2D;
  return m;
}

template <typename T>
static tddft_status zvector_rhs_impl(tddft_system* h, int nb, const cplx<T>* X, cplx<T>* U, cudaStream_t st) {
  const long long len = (long long)h->d.nocc_src * h->npw;
  const double one = 1.0;
  for (int b = 0; b < nb; ++b) {
    STATUS_TRY(adjoint_impl<T>(h, 1, X + b * len, &one, h->b.wdev, U + b * len, nullptr, st));
    STATUS_TRY(project_rows<T>(h, (const cplx<T>*)h->b.phi_src_pw, h->d.nocc_src, U + b * len, h->d.nocc_src, st));
    { k_negate<T><<<grid_for(len, 256), 256, 0, st>>>(U + b * len, len); note_launch(); }
  }
  return check_launch("zvector rhs");
}

template <typename T>
static tddft_status zvector_impl(tddft_system* h, int nb, const cplx<T>* U, cplx<T>* Z, const tddft_zvector_opts& o,
                                 int* iters_out, int* exact_out, double* res_out, cudaStream_t st) {
  const long long len = (long long)h->d.nocc_src * h->npw, total = nb * len;
  const size_t bytes = (size_t)total * sizeof(cplx<T>);
  const unsigned m_exact = zvector_mask(h->d.term_mask), m_approx = m_exact & ~TDDFT_TERM_K2D;
  TempAllocs tmp;
  cplx<T> *r, *p, *q, *sv, *gin, *gout;
  double* dsc;  // [3][nb]: dots, steps, betas
  STATUS_TRY(tmp.get((void**)&r, bytes));
  STATUS_TRY(tmp.get((void**)&p, bytes));
  STATUS_TRY(tmp.get((void**)&q, bytes));
  STATUS_TRY(tmp.get((void**)&gin, bytes));
  STATUS_TRY(tmp.get((void**)&gout, bytes));
  if (o.precondition) STATUS_TRY(tmp.get((void**)&sv, bytes));
  else sv = r;
  STATUS_TRY(tmp.get((void**)&dsc, 3 * (size_t)nb * sizeof(double)));
  double* d_dot = dsc;
  double* d_step = dsc + nb;
  double* d_beta = dsc + 2 * nb;
  auto precond = [&]() -> tddft_status {
    if (!o.precondition) return TDDFT_OK;
    { k_zv_precondition<T><<<grid_for(total, 256), 256, 0, st>>>(r, (const T*)h->b.g2h, (const T*)h->b.eps,
                                                                 h->d.nocc_src, h->npw, total, sv); note_launch(); }
    return project_rows<T>(h, (const cplx<T>*)h->b.phi_tgt_pw, h->d.nocc_tgt, sv, nb * h->d.nocc_src, st);
  };
  // Re<x_b|y_b> for every b, to the host
  auto dots = [&](const cplx<T>* x, const cplx<T>* y, std::vector<double>& out) -> tddft_status {
    { k_bilinear<T><<<nb, 256, 0, st>>>(x, y, len, d_dot); note_launch(); }
    STATUS_TRY(check_launch("zvector dots"));
    out.resize(nb);
    CUDA_TRY(cudaMemcpyAsync(out.data(), d_dot, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDDFT_OK;
  };
  // q_b = L p_b for the states in `set` with the given terms (contiguous runs in place, others gathered)
  auto apply_set = [&](const std::vector<int>& set, unsigned mask) -> tddft_status {
    if (set.empty()) return TDDFT_OK;
    bool run = true;
    for (size_t j = 1; j < set.size(); ++j) run = run && set[j] == set[j - 1] + 1;
    if (run) return apply_impl<T>(h, (int)set.size(), p + set[0] * len, q + set[0] * len, mask, st);
    for (size_t j = 0; j < set.size(); ++j)
      CUDA_TRY(cudaMemcpyAsync(gin + j * len, p + set[j] * len, len * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st));
    STATUS_TRY(apply_impl<T>(h, (int)set.size(), gin, gout, mask, st));
    for (size_t j = 0; j < set.size(); ++j)
      CUDA_TRY(cudaMemcpyAsync(q + set[j] * len, gout + j * len, len * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st));
    return TDDFT_OK;
  };

  CUDA_TRY(cudaMemsetAsync(Z, 0, bytes, st));
  CUDA_TRY(cudaMemcpyAsync(r, U, bytes, cudaMemcpyDeviceToDevice, st));
  STATUS_TRY(precond());
  CUDA_TRY(cudaMemcpyAsync(p, sv, bytes, cudaMemcpyDeviceToDevice, st));
  std::vector<double> rs, rr, pq, rs_new;
  STATUS_TRY(dots(r, sv, rs));
  STATUS_TRY(dots(r, r, rr));
  std::vector<int> iters(nb, 0), n_exact(nb, 0);
  std::vector<double> step(nb), beta(nb);
  for (int it = 0; it < o.max_iter; ++it) {
    std::vector<int> ex, ap;
    for (int b = 0; b < nb; ++b) {
      const double rn = std::sqrt(std::max(rr[b], 0.0));
      if (!(rn >= o.tol)) continue;  // converged
      (rn >= o.lambda_thr ? ex : ap).push_back(b);
    }
    if (ex.empty() && ap.empty()) break;
    STATUS_TRY(apply_set(ex, m_exact));
    STATUS_TRY(apply_set(ap, m_approx));
    STATUS_TRY(dots(p, q, pq));
    std::fill(step.begin(), step.end(), 0.0);
    for (const std::vector<int>* set : {&ex, &ap})
      for (int b : *set) {
        if (!(pq[b] > 0.0))
          return fail(TDDFT_ENUMERIC, "the Z-vector operator is not positive definite on the search direction of state " +
                                          std::to_string(b));
        step[b] = rs[b] / pq[b];
        iters[b] += 1;
        n_exact[b] += set == &ex ? 1 : 0;
      }
    CUDA_TRY(cudaMemcpyAsync(d_step, step.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
    { k_zv_step<T><<<grid_for(total, 256), 256, 0, st>>>(Z, r, p, q, d_step, len, total); note_launch(); }
    STATUS_TRY(precond());
    STATUS_TRY(dots(r, sv, rs_new));
    STATUS_TRY(dots(r, r, rr));
    for (int b = 0; b < nb; ++b) {
      beta[b] = (step[b] != 0.0 && rs[b] > 0.0) ? rs_new[b] / rs[b] : 0.0;
      if (step[b] != 0.0) rs[b] = rs_new[b];
    }
    CUDA_TRY(cudaMemcpyAsync(d_beta, beta.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
    { k_zv_direction<T><<<grid_for(total, 256), 256, 0, st>>>(p, sv, d_beta, d_step, len, total); note_launch(); }
    STATUS_TRY(check_launch("zvector update"));
  }
  STATUS_TRY(check_device_flag(h, st));
  bool all = true;
  for (int b = 0; b < nb; ++b) {
    const double rn = std::sqrt(std::max(rr[b], 0.0));
    if (iters_out) iters_out[b] = iters[b];
    if (exact_out) exact_out[b] = n_exact[b];
    if (res_out) res_out[b] = rn;
    all = all && rn < o.tol;
  }
  if (!all) return fail(TDDFT_ENOTCONV, "the Z-vector CG did not reach the tolerance within max_iter");
  return TDDFT_OK;
}

extern "C" {

tddft_status tddft_zvector_rhs(tddft_handle h, int nb, const void* X, void* U, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h) return fail(TDDFT_EINVAL, "null handle");
    if (h->sf()) return fail(TDDFT_ENOTSUP, "the Z-vector equation is implemented for spin-conserving systems");
    if (h->ace_on) return fail(TDDFT_ENOTSUP, "the right-hand side differentiates the exact exchange; disable ACE first");
    if (h->loc_on) return fail(TDDFT_ENOTSUP, "the right-hand side differentiates the exact K1d; disable the localised frame first");
    if (nb < 1 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [1, nb_max]");
    if (!X || !U) return fail(TDDFT_EINVAL, "null buffer");
    if (X == U) return fail(TDDFT_EINVAL, "X and U must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d.precision == TDDFT_PREC_FP64)
      return zvector_rhs_impl<double>(h, nb, (const cplx<double>*)X, (cplx<double>*)U, st);
    return zvector_rhs_impl<float>(h, nb, (const cplx<float>*)X, (cplx<float>*)U, st);
  });
}

tddft_status tddft_zvector_solve(tddft_handle h, int nb, const void* U, void* Z, const tddft_zvector_opts* opts,
                                 int* iterations, int* exact_iterations, double* residual, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !opts) return fail(TDDFT_EINVAL, "null argument");
    if (h->sf()) return fail(TDDFT_ENOTSUP, "the Z-vector equation is implemented for spin-conserving systems");
    if (nb < 1 || nb > h->d.nb_max) return fail(TDDFT_EINVAL, "nb outside [1, nb_max]");
    if (!U || !Z) return fail(TDDFT_EINVAL, "null buffer");
    if (U == Z) return fail(TDDFT_EINVAL, "U and Z must not alias");
    if (!(opts->tol > 0.0) || !(opts->lambda_thr >= 0.0) || opts->max_iter < 0 || opts->precondition < 0 ||
        opts->precondition > 1)
      return fail(TDDFT_EINVAL, "need tol > 0, lambda_thr >= 0, max_iter >= 0, precondition 0 or 1");
    if ((h->d.term_mask & TDDFT_TERM_PROJ) == 0) return fail(TDDFT_EINVAL, "the Z-vector solve needs the projector term");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d.precision == TDDFT_PREC_FP64)
      return zvector_impl<double>(h, nb, (const cplx<double>*)U, (cplx<double>*)Z, *opts, iterations, exact_iterations,
                                  residual, st);
    return zvector_impl<float>(h, nb, (const cplx<float>*)U, (cplx<float>*)Z, *opts, iterations, exact_iterations,
                               residual, st);
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Davidson: block scheme with FP64 basis, orthogonalisation and Rayleigh-Ritz
// ---------------------------------------------------------------------------

// Hermitian eigenproblem of a small dense matrix (row-major, n x n) by cyclic
// complex Jacobi rotations. Eigenvalues ascending in w, eigenvectors in the
// columns of V (row-major). Returns false if the sweeps do not converge.
static bool herm_eig(int n, std::vector<std::complex<double>> A, std::vector<double>& w,
                     std::vector<std::complex<double>>& V) {
  using C = std::complex<double>;
  V.assign((size_t)n * n, C(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> C& { return A[(size_t)i * n + j]; };
  double fro = 0.0;
  for (auto& z : A) fro += std::norm(z);
  bool ok = false;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(at(p, q));
    if (off <= 1e-30 * std::max(fro, 1e-300)) {
      ok = true;
      break;
    }
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const C apq = at(p, q);
        const double r = std::abs(apq);
        if (r < 1e-300) continue;
        const C ph = apq / r;  // exp(i phi)
        const double app = at(p, p).real(), aqq = at(q, q).real();
        const double tau = (aqq - app) / (2.0 * r);
        const double t = tau == 0.0 ? 1.0 : (tau > 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        // U = diag(1, conj(ph)) [[c, sn], [-sn, c]] acting on (p, q)
        const C upp = c, upq = sn, uqp = -sn * std::conj(ph), uqq = c * std::conj(ph);
        for (int k = 0; k < n; ++k) {  // A <- A U
          const C akp = at(k, p), akq = at(k, q);
          at(k, p) = akp * upp + akq * uqp;
          at(k, q) = akp * upq + akq * uqq;
        }
        for (int k = 0; k < n; ++k) {  // A <- U^H A
          const C apk = at(p, k), aqk = at(q, k);
          at(p, k) = std::conj(upp) * apk + std::conj(uqp) * aqk;
          at(q, k) = std::conj(upq) * apk + std::conj(uqq) * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V U
          const C vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = vkp * upp + vkq * uqp;
          V[(size_t)k * n + q] = vkp * upq + vkq * uqq;
        }
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return at(x, x).real() < at(y, y).real(); });
  std::vector<std::complex<double>> Vs((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = at(idx[j], idx[j]).real();
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + j] = V[(size_t)k * n + idx[j]];
  }
  V.swap(Vs);
  return ok;
}

// nrm[b] = ||x_b||_2 (one block per row of length len)
__global__ void k_row_norms(const cplx<double>* __restrict__ x, long long len, double* __restrict__ nrm) {
  __shared__ double red[256];
  const long long b = blockIdx.x;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    const cplx<double> u = x[b * len + i];
    acc += u.x * u.x + u.y * u.y;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) nrm[b] = sqrt(red[0]);
}

// x /= max(||x||, tiny) with the norm from k_row_norms
__global__ void k_normalize(cplx<double>* __restrict__ x, const double* __restrict__ nrm, long long len) {
  const double s = 1.0 / fmax(nrm[0], 1e-300);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    x[i] = {x[i].x * s, x[i].y * s};
}

// t = r / d with d = |G|^2/2 - eps_v - theta, |d| clamped to >= 0.1 Ha (sign kept)
// (t may equal r: element-wise, in place)
__global__ void k_precondition(const cplx<double>* r, const double* __restrict__ g2h,
                               const double* __restrict__ eps, double theta, int npw, long long len,
                               cplx<double>* t) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / npw, g = i - v * npw;
    double d = g2h[g] - eps[v] - theta;
    if (fabs(d) < 0.1) d = d < 0.0 ? -0.1 : 0.1;
    t[i] = {r[i].x / d, r[i].y / d};
  }
}

// theta-shifted residuals of nr Ritz pairs: y_i = a_i - theta_i x_i (theta on the device)
__global__ void k_residuals(const cplx<double>* __restrict__ a, const cplx<double>* __restrict__ x,
                            const double* __restrict__ theta, cplx<double>* __restrict__ y, long long len, int nr) {
  const long long n = len * nr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double t = theta[i / len];
    y[i] = {a[i].x - t * x[i].x, a[i].y - t * x[i].y};
  }
}

// FP64 Hermitian eigensolver of the Rayleigh-Ritz matrix on the device: cyclic
// complex Jacobi rotations in the round-robin (tournament) order, so that the M/2
// rotations of a round act on disjoint index pairs and are applied together; one
// CTA. A [m][m] row-major is overwritten (its Hermitian part is taken first),
// V [m][m] is workspace. Writes theta[0..nr) ascending, S [m][nr] row-major (column
// j = eigenvector of theta[j]) and flag[0] = 1 when the off-diagonal norm fell
// below 1e-15 of the Frobenius norm within 100 sweeps (else 0; outputs then hold
// the last iterate).
constexpr int JACOBI_THREADS = 256;
constexpr int JACOBI_MAX_N = 1024;
__global__ void __launch_bounds__(JACOBI_THREADS)
    k_herm_jacobi(cplx<double>* A, cplx<double>* V, int m, int nr, double* theta, cplx<double>* S, double* flag) {
  __shared__ double rc[JACOBI_MAX_N / 2], rs[JACOBI_MAX_N / 2];
  __shared__ cplx<double> rph[JACOBI_MAX_N / 2];
  __shared__ int rp[JACOBI_MAX_N / 2], rq[JACOBI_MAX_N / 2];
  __shared__ double red[JACOBI_THREADS];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M = m + (m & 1), np = M / 2;
  auto block_sum = [&](double v) {
    red[tid] = v;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
  };
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    V[e] = {i == j ? 1.0 : 0.0, 0.0};
    if (i < j) {
      const cplx<double> a = A[e], b = A[(long long)j * m + i];
      const cplx<double> h = {0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
      A[e] = h;
      A[(long long)j * m + i] = {h.x, -h.y};
    } else if (i == j) {
      A[e].y = 0.0;
    }
  }
  __syncthreads();
  double f = 0.0;
  for (int e = tid; e < m * m; e += nt) f += A[e].x * A[e].x + A[e].y * A[e].y;
  const double fro = block_sum(f);
  bool conv = false;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double o = 0.0;
    for (int e = tid; e < m * m; e += nt) {
      const int i = e / m, j = e - i * m;
      if (i < j) o += A[e].x * A[e].x + A[e].y * A[e].y;
    }
    if (block_sum(o) <= 1e-30 * fmax(fro, 1e-300)) {
      conv = true;
      break;
    }
    for (int r = 0; r < M - 1; ++r) {
      for (int k = tid; k < np; k += nt) {
        int p = k == 0 ? M - 1 : (r + k) % (M - 1);
        int q = k == 0 ? r : (r - k + (M - 1)) % (M - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, sn = 0.0;
        cplx<double> ph = {1.0, 0.0};
        if (q < m) {
          const cplx<double> apq = A[(long long)p * m + q];
          const double rr = sqrt(apq.x * apq.x + apq.y * apq.y);
          if (rr >= 1e-300) {
            ph = {apq.x / rr, apq.y / rr};
            const double tau = (A[(long long)q * m + q].x - A[(long long)p * m + p].x) / (2.0 * rr);
            const double t = tau == 0.0 ? 1.0 : (tau > 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        rc[k] = c;
        rs[k] = sn;
        rph[k] = ph;
        rp[k] = p;
        rq[k] = q;
      }
      __syncthreads();
      // U = diag(1, conj(ph)) [[c, sn], [-sn, c]] on (p, q):  A <- A U,  V <- V U
      for (int e = tid; e < np * m; e += nt) {
        const int k = e / m, i = e - k * m;
        const int p = rp[k], q = rq[k];
        if (q >= m || rs[k] == 0.0) continue;
        const double c = rc[k], sn = rs[k];
        const cplx<double> cph = {rph[k].x, -rph[k].y};
        const cplx<double> uqp = cscale(cph, -sn), uqq = cscale(cph, c);
        cplx<double>* ai = A + (long long)i * m;
        const cplx<double> aip = ai[p], aiq = ai[q];
        ai[p] = cadd(cscale(aip, c), cmul(aiq, uqp));
        ai[q] = cadd(cscale(aip, sn), cmul(aiq, uqq));
        cplx<double>* vi = V + (long long)i * m;
        const cplx<double> vip = vi[p], viq = vi[q];
        vi[p] = cadd(cscale(vip, c), cmul(viq, uqp));
        vi[q] = cadd(cscale(vip, sn), cmul(viq, uqq));
      }
      __syncthreads();
      // A <- U^H A
      for (int e = tid; e < np * m; e += nt) {
        const int k = e / m, j = e - k * m;
        const int p = rp[k], q = rq[k];
        if (q >= m || rs[k] == 0.0) continue;
        const double c = rc[k], sn = rs[k];
        const cplx<double> cph = {rph[k].x, -rph[k].y};
        const cplx<double> uqp = cscale(cph, -sn), uqq = cscale(cph, c);
        const cplx<double> apj = A[(long long)p * m + j], aqj = A[(long long)q * m + j];
        A[(long long)p * m + j] = cadd(cscale(apj, c), cmulc(uqp, aqj));
        A[(long long)q * m + j] = cadd(cscale(apj, sn), cmulc(uqq, aqj));
      }
      __syncthreads();
    }
  }
  // ascending order: rank of each diagonal entry (ties by index)
  for (int i = tid; i < m; i += nt) {
    const double di = A[(long long)i * m + i].x;
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double dj = A[(long long)j * m + j].x;
      rank += (dj < di) || (dj == di && j < i);
    }
    if (rank < nr) {
      theta[rank] = di;
      for (int k = 0; k < m; ++k) S[(long long)k * nr + rank] = V[(long long)k * m + i];
    }
  }
  if (tid == 0) flag[0] = conv ? 1.0 : 0.0;
}

// info[slot] = the handle's device-wait error flag (0 when the handle has none)
__global__ void k_copy_flag(const int* __restrict__ err, double* __restrict__ info) {
  info[0] = err ? (double)err[0] : 0.0;
}

struct tddft_davidson {
  tddft_system* h = nullptr;
  int nroots = 0, max_basis = 0, m = 0;
  long long len = 0;  // nocc_src * npw
  std::vector<void*> allocs;
  cplx<double>* V = nullptr;   // [max_basis][len]
  cplx<double>* LV = nullptr;  // [max_basis][len]
  cplx<double>* X = nullptr;   // [nroots][len] Ritz vectors
  cplx<double>* W = nullptr;   // [nroots][len] L applied to the Ritz vectors
  cplx<double>* R = nullptr;   // [nroots][len] residuals, then corrections
  void* tin = nullptr;         // [nroots][len] working precision
  void* tout = nullptr;
  cplx<double>* part = nullptr;   // split-K partials [nsplit][max_basis][max_basis]
  cplx<double>* small = nullptr;  // [max_basis][max_basis]
  double* g2h = nullptr;          // [npw]
  double* eps = nullptr;          // [nocc_src]
  double* nrm = nullptr;          // [max_basis]
  cplx<double>* evec = nullptr;   // [max_basis][max_basis] eigenvector workspace of the Rayleigh-Ritz solve
  cplx<double>* ritz = nullptr;   // [max_basis][nroots] lowest Ritz coefficient vectors
  double* info = nullptr;         // [2 nroots + 2]: Ritz values, residual norms, eigensolver flag, wait flag
  int nsplit = 1;
  std::vector<double> theta;
  ~tddft_davidson() {
    for (void* p : allocs) cudaFree(p);
  }
};

static tddft_status dav_alloc(tddft_davidson* d, void** p, size_t bytes) {
  cudaError_t e = lib_malloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TDDFT_ENOMEM, alloc_error(bytes, e));
  }
  d->allocs.push_back(*p);
  return TDDFT_OK;
}

// C[i][j] = <A_i|B_j> over rows of length len (i < ma, j < mb) into d->small
static void dav_overlap(tddft_davidson* d, const cplx<double>* A, int ma, const cplx<double>* B, int mb,
                        cudaStream_t st) {
  const int kchunk = (int)(((d->len + d->nsplit - 1) / d->nsplit + 15) / 16 * 16);
  dim3 g1((ma + 31) / 32, (mb + 31) / 32, d->nsplit);
  { k_overlap<double><<<g1, 256, 0, st>>>(A, ma, B, mb, (int)d->len, kchunk, d->part); note_launch(); }
  { k_reduce_split<double><<<grid_for((long long)ma * mb, 256), 256, 0, st>>>(d->part, d->nsplit, (long long)ma * mb,
                                                                             d->small); note_launch(); }
}

// Y[n] += s * sum_m A[m] C[m][n]  (rows of length len, C is [ma][nn] in d->small or given)
static void dav_combine(tddft_davidson* d, const cplx<double>* A, int ma, const cplx<double>* C, int nn, double s,
                        cplx<double>* Y, cudaStream_t st) {
  dim3 g2((unsigned)((d->len + 63) / 64), (nn + 31) / 32);
  { k_update<double><<<g2, 256, 0, st>>>(A, ma, C, nn, (int)d->len, s, Y); note_launch(); }
}

// Orthogonalise t against the target orbitals (each of its nocc_src rows) and
// the current basis, twice; normalise; append to the basis.
static tddft_status dav_append(tddft_davidson* d, cplx<double>* t, cudaStream_t st) {
  tddft_system* h = d->h;
  for (int pass = 0; pass < 2; ++pass) {
    STATUS_TRY(project_rows<double>(h, h->b.phi_tgt_pw64, h->d.nocc_tgt, t, h->d.nocc_src, st));
    if (d->m > 0) {
      dav_overlap(d, d->V, d->m, t, 1, st);
      dav_combine(d, d->V, d->m, d->small, 1, -1.0, t, st);
    }
  }
  { k_row_norms<<<1, 256, 0, st>>>(t, d->len, d->nrm); note_launch(); }
  { k_normalize<<<grid_for(d->len, 256), 256, 0, st>>>(t, d->nrm, d->len); note_launch(); }
  cplx<double>* dst = d->V + (long long)d->m * d->len;
  if (dst != t) CUDA_TRY(cudaMemcpyAsync(dst, t, d->len * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, st));
  d->m += 1;
  return check_launch("davidson append");
}

// LV[m0 .. m) = L V[m0 .. m) through the handle's apply (working precision)
template <typename T>
static tddft_status dav_apply_new(tddft_davidson* d, int m0, cudaStream_t st) {
  tddft_system* h = d->h;
  for (int b0 = m0; b0 < d->m; b0 += d->h->d.nb_max) {
    const int nb = std::min(d->h->d.nb_max, d->m - b0);
    const long long cnt = (long long)nb * d->len;
    { k_cast<T><<<grid_for(cnt, 256), 256, 0, st>>>(d->V + (long long)b0 * d->len, (cplx<T>*)d->tin, cnt); note_launch(); }
    STATUS_TRY(apply_impl<T>(h, nb, (const cplx<T>*)d->tin, (cplx<T>*)d->tout, h->d.term_mask, st));
    { k_widen<T><<<grid_for(cnt, 256), 256, 0, st>>>((const cplx<T>*)d->tout, d->LV + (long long)b0 * d->len, cnt); note_launch(); }
  }
  return check_launch("davidson apply");
}

static tddft_status dav_apply(tddft_davidson* d, int m0, cudaStream_t st) {
  return d->h->d.precision == TDDFT_PREC_FP64 ? dav_apply_new<double>(d, m0, st) : dav_apply_new<float>(d, m0, st);
}

extern "C" {

tddft_status tddft_davidson_create(tddft_handle h, int nroots, int nguess, const double* X0, int max_basis,
                                   void* stream, tddft_dav_handle* out) {
  return abi_guard([&]() -> tddft_status {
    if (!h || !X0 || !out) return fail(TDDFT_EINVAL, "null argument");
    *out = nullptr;
    if (nroots < 1 || nguess < nroots) return fail(TDDFT_EINVAL, "need 1 <= nroots <= nguess");
    if (max_basis < 2 * nroots || max_basis < nguess) return fail(TDDFT_EINVAL, "max_basis must be >= 2*nroots and >= nguess");
    if (max_basis > JACOBI_MAX_N)
      return fail(TDDFT_EINVAL, "max_basis above the Rayleigh-Ritz solver's limit of " + std::to_string(JACOBI_MAX_N));
    if (h->d.nb_max < nroots) return fail(TDDFT_EINVAL, "the handle's nb_max must be >= nroots");
    if ((h->d.term_mask & TDDFT_TERM_PROJ) == 0) return fail(TDDFT_EINVAL, "Davidson needs the projector term");
    if (h->d.term_mask & ~TDDFT_TERMS_ALL)
      return fail(TDDFT_EINVAL, "Davidson diagonalises the Tamm-Dancoff operator: no K2 terms");
    cudaStream_t st = (cudaStream_t)stream;
    tddft_davidson* d = new tddft_davidson();
    d->h = h;
    d->nroots = nroots;
    d->max_basis = max_basis;
    d->len = (long long)h->d.nocc_src * h->npw;
    d->nsplit = (int)std::max<long long>(1, std::min<long long>(64, d->len / 4096));
    const size_t vb = (size_t)d->len * sizeof(cplx<double>);
    tddft_status s = TDDFT_OK;
    auto A = [&](void** p, size_t b) {
      if (s == TDDFT_OK) s = dav_alloc(d, p, b);
    };
    A((void**)&d->V, vb * max_basis);
    A((void**)&d->LV, vb * max_basis);
    A((void**)&d->X, vb * nroots);
    A((void**)&d->W, vb * nroots);
    A((void**)&d->R, vb * std::max(nroots, nguess));
    A(&d->tin, (size_t)d->len * h->esz() * h->d.nb_max);
    A(&d->tout, (size_t)d->len * h->esz() * h->d.nb_max);
    A((void**)&d->part, sizeof(cplx<double>) * d->nsplit * max_basis * max_basis);
    A((void**)&d->small, sizeof(cplx<double>) * max_basis * max_basis);
    A((void**)&d->g2h, sizeof(double) * h->npw);
    A((void**)&d->eps, sizeof(double) * h->d.nocc_src);
    A((void**)&d->nrm, sizeof(double) * max_basis);
    A((void**)&d->evec, sizeof(cplx<double>) * max_basis * max_basis);
    A((void**)&d->ritz, sizeof(cplx<double>) * max_basis * nroots);
    A((void**)&d->info, sizeof(double) * (2 * nroots + 2));
    if (s != TDDFT_OK) {
      delete d;
      return s;
    }
    // FP64 preconditioner tables
    std::vector<Miller> sph;
    tddft_status sb = build_sphere(h->n, h->d.a, h->d.ecut, sph);
    if (sb != TDDFT_OK) {
      delete d;
      return sb;
    }
    const double tpiba = 2.0 * M_PI / h->d.a, tpiba2 = tpiba * tpiba;
    std::vector<double> g2h(h->npw);
    for (int i = 0; i < h->npw; ++i) g2h[i] = 0.5 * (tpiba2 * (double)sph[i].m2);
    // the preconditioner's eigenvalues in FP64: the values given at set-up (the handle's
    // device copy is in the working precision)
    const std::vector<double>& eps = h->eps64;
    cudaMemcpyAsync(d->g2h, g2h.data(), g2h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d->eps, eps.data(), eps.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d->R, X0, vb * nguess, cudaMemcpyHostToDevice, st);
    for (int i = 0; i < nguess && s == TDDFT_OK; ++i) s = dav_append(d, d->R + (long long)i * d->len, st);
    if (s == TDDFT_OK) s = dav_apply(d, 0, st);
    if (s == TDDFT_OK) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = fail(TDDFT_ECUDA, std::string("davidson create: ") + cudaGetErrorString(e));
    }
    if (s != TDDFT_OK) {
      delete d;
      return s;
    }
    *out = d;
    return TDDFT_OK;
  });
}

tddft_status tddft_davidson_step(tddft_dav_handle d, double tol, int* n_converged, double* ritz_values,
                                 double* residual_norms, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!d || !n_converged || !ritz_values) return fail(TDDFT_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int m = d->m, nr = d->nroots;
    // Rayleigh-Ritz on the device: H = V^H L V (FP64), its lowest nr eigenpairs by Jacobi rotations
    dav_overlap(d, d->V, m, d->LV, m, st);
    { k_herm_jacobi<<<1, JACOBI_THREADS, 0, st>>>(d->small, d->evec, m, nr, d->info, d->ritz, d->info + 2 * nr);
      note_launch(); }
    // Ritz vectors X = V S, W = L V S, residuals R = W - theta X and their norms
    const size_t vb = (size_t)d->len * sizeof(cplx<double>);
    CUDA_TRY(cudaMemsetAsync(d->X, 0, vb * nr, st));
    CUDA_TRY(cudaMemsetAsync(d->W, 0, vb * nr, st));
    dav_combine(d, d->V, m, d->ritz, nr, 1.0, d->X, st);
    dav_combine(d, d->LV, m, d->ritz, nr, 1.0, d->W, st);
    { k_residuals<<<grid_for(d->len * nr, 256), 256, 0, st>>>(d->W, d->X, d->info, d->R, d->len, nr); note_launch(); }
    { k_row_norms<<<nr, 256, 0, st>>>(d->R, d->len, d->info + nr); note_launch(); }
    { k_copy_flag<<<1, 1, 0, st>>>(d->h->b.dev_err, d->info + 2 * nr + 1); note_launch(); }
    STATUS_TRY(check_launch("davidson step"));
    // the one host synchronisation: Ritz values, residual norms and both flags in one copy
    std::vector<double> info(2 * nr + 2);
    CUDA_TRY(cudaMemcpyAsync(info.data(), d->info, info.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (fault_take_wait())
      return fail(TDDFT_ETIMEOUT, "a bounded device wait ran out (injected fault); results of the call are invalid");
    if (info[2 * nr + 1] != 0.0) {
      CUDA_TRY(cudaMemsetAsync(d->h->b.dev_err, 0, sizeof(int), st));
      return fail(TDDFT_ETIMEOUT, "a bounded device wait (tensor-core projector) ran out; results of the call are invalid");
    }
    if (info[2 * nr] != 1.0) return fail(TDDFT_ENUMERIC, "subspace eigensolver did not converge");
    d->theta.assign(info.begin(), info.begin() + nr);
    int nconv = 0;
    for (int i = 0; i < nr; ++i) {
      const double rn = info[nr + i];
      nconv += rn < tol;
      ritz_values[i] = d->theta[i];
      if (residual_norms) residual_norms[i] = rn;
    }
    *n_converged = nconv;
    if (nconv == nr) return TDDFT_OK;
    // corrections for the unconverged roots
    std::vector<int> todo;
    for (int i = 0; i < nr; ++i)
      if (!(info[nr + i] < tol)) todo.push_back(i);
    for (int i : todo)
      { k_precondition<<<grid_for(d->len, 256), 256, 0, st>>>(d->R + (long long)i * d->len, d->g2h, d->eps, d->theta[i],
                                                             d->h->npw, d->len, d->R + (long long)i * d->len); note_launch(); }
    // restart on the Ritz vectors when the basis would overflow
    if (d->m + (int)todo.size() > d->max_basis) {
      CUDA_TRY(cudaMemcpyAsync(d->V, d->X, vb * nr, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(d->LV, d->W, vb * nr, cudaMemcpyDeviceToDevice, st));
      d->m = nr;
    }
    const int m0 = d->m;
    for (int i : todo) STATUS_TRY(dav_append(d, d->R + (long long)i * d->len, st));
    STATUS_TRY(dav_apply(d, m0, st));
    return TDDFT_OK;
  });
}

tddft_status tddft_davidson_vectors(tddft_dav_handle d, double* X_host, void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!d || !X_host) return fail(TDDFT_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(X_host, d->X, (size_t)d->nroots * d->len * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDDFT_OK;
  });
}

tddft_status tddft_davidson_destroy(tddft_dav_handle d) {
  return abi_guard([&]() -> tddft_status {
    delete d;
    return TDDFT_OK;
  });
}
}

// ---------------------------------------------------------------------------
// Allocation-free exchange pair term.
//
// For callers that cannot allocate device memory themselves and therefore
// cannot create a handle (for example a code that hands all device memory to
// its own pool allocator, so that a library cudaMalloc would fail or break the
// pool). All working memory lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int NOALLOC_MAX_N = 48;
constexpr size_t NOALLOC_N3 = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N;
// layout: twiddles | kernel table | sphere positions | orbital field | trial field | reciprocal-space field
constexpr size_t NA_TW = 0;       // up to 3 * NOALLOC_MAX_N twiddles
constexpr size_t NA_KERN = 2048;
constexpr size_t NA_POS = NA_KERN + NOALLOC_N3 * sizeof(float);
constexpr size_t NA_PHI = NA_POS + NOALLOC_N3 * sizeof(int);
constexpr size_t NA_A = NA_PHI + NOALLOC_N3 * sizeof(cplx<float>);
constexpr size_t NA_G = NA_A + NOALLOC_N3 * sizeof(cplx<float>);
constexpr size_t NOALLOC_BYTES = NA_G + NOALLOC_N3 * sizeof(cplx<float>);  // 3.5 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
constexpr int NOALLOC_MAX_DEVICES = 64;
// per device: the scratch array's device address, the grid sizes whose launchers are
// prepared, and the geometry whose tables the array holds now
struct NoallocDevice {
  unsigned char* ptr = nullptr;
  std::vector<int> prepared;
  bool tables = false;
  int n = 0;
  double a = 0.0, ecut = 0.0, kx_g0 = 0.0;
  int npw = 0;
};
NoallocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" tddft_status tddft_exchange_pair_noalloc(int n, double a, double ecut, double alpha, double kx_g0,
                                                     const void* phi_pw, const void* a_pw, void* out_pw,
                                                     void* stream) {
  return abi_guard([&]() -> tddft_status {
    if (!phi_pw || !a_pw || !out_pw) return fail(TDDFT_EINVAL, "null buffer");
    if (n > NOALLOC_MAX_N)
      return fail(TDDFT_EINVAL, "grid size " + std::to_string(n) + " exceeds the allocation-free limit of " +
                                    std::to_string(NOALLOC_MAX_N));
    if (!supported_n(n, TDDFT_PREC_FP32)) return fail(TDDFT_EINVAL, "unsupported grid size " + std::to_string(n));
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(TDDFT_EINVAL, "device index out of range");
    NoallocDevice& D = g_noalloc_dev[dev];
    if (!D.ptr) {
      // set-up, once per device: the device address of the scratch array
      void* p = nullptr;
      CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      D.ptr = (unsigned char*)p;
    }
    unsigned char* base = D.ptr;
    PlaneOps<float> o = plane_ops_for<float>(n);
    if (o.n != n) return fail(TDDFT_EINVAL, "unsupported grid size");
    if (std::find(D.prepared.begin(), D.prepared.end(), n) == D.prepared.end()) {
      // set-up, once per device and grid size: launch attributes and constant twiddles
      CUDA_TRY(o.prepare());
      D.prepared.push_back(n);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long n3 = (long long)n * n * n;
    cplx<float>* tw = (cplx<float>*)(base + NA_TW);
    float* kern = (float*)(base + NA_KERN);
    int* pos = (int*)(base + NA_POS);
    cplx<float>* phi_r = (cplx<float>*)(base + NA_PHI);
    cplx<float>* a_r = (cplx<float>*)(base + NA_A);
    cplx<float>* gbuf = (cplx<float>*)(base + NA_G);

    if (!(D.tables && D.n == n && D.a == a && D.ecut == ecut && D.kx_g0 == kx_g0)) {
      // tables of this geometry (the same host arithmetic as a handle's set-up), uploaded
      // only when the geometry differs from the one the array holds
      std::vector<Miller> sph;
      STATUS_TRY(build_sphere(n, a, ecut, sph));
      const int npw_new = (int)sph.size();
      std::vector<int> radices = plan_radices(n), rev(n);
      for (int k = 0; k < n; ++k) rev[k] = dif_position(k, radices, n);
      std::vector<cplx<float>> twh = host_twiddles<float>(n, radices);
      if (twh.size() * sizeof(cplx<float>) > NA_KERN - NA_TW)
        return fail(TDDFT_EINVAL, "twiddle table of grid " + std::to_string(n) + " exceeds its scratch region");
      const double tpiba = 2.0 * M_PI / a, tpiba2 = tpiba * tpiba;
      auto mof = [n](int k) { return k < n - n / 2 ? k : k - n; };
      std::vector<float> kh(n3);
      for (int kz = 0; kz < n; ++kz)
        for (int ky = 0; ky < n; ++ky)
          for (int kxx = 0; kxx < n; ++kxx) {
            const long long m2 =
                (long long)mof(kz) * mof(kz) + (long long)mof(ky) * mof(ky) + (long long)mof(kxx) * mof(kxx);
            const double vx = m2 == 0 ? kx_g0 : 4.0 * M_PI / (tpiba2 * (double)m2);
            kh[((long long)rev[kz] * n + rev[ky]) * n + rev[kxx]] = (float)(vx / (double)n3);
          }
      std::vector<int> posh(npw_new);
      for (int i = 0; i < npw_new; ++i)
        posh[i] = (rev[(sph[i].z % n + n) % n] * n + rev[(sph[i].y % n + n) % n]) * n + rev[(sph[i].x % n + n) % n];
      D.tables = false;
      CUDA_TRY(cudaMemcpyAsync(tw, twh.data(), twh.size() * sizeof(cplx<float>), cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(kern, kh.data(), n3 * sizeof(float), cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(pos, posh.data(), npw_new * sizeof(int), cudaMemcpyHostToDevice, st));
      D.tables = true;
      D.n = n;
      D.a = a;
      D.ecut = ecut;
      D.kx_g0 = kx_g0;
      D.npw = npw_new;
    }
    const int npw = D.npw;

    // both orbitals to real space (cube cleared first: it keeps the previous call's contents)
    const float s_in = (float)(1.0 / std::sqrt(a * a * a));
    const cplx<float>* srcs[2] = {(const cplx<float>*)phi_pw, (const cplx<float>*)a_pw};
    cplx<float>* dsts[2] = {phi_r, a_r};
    for (int i = 0; i < 2; ++i) {
      CUDA_TRY(cudaMemsetAsync(gbuf, 0, n3 * sizeof(cplx<float>), st));
      { k_scatter<float><<<grid_for(npw, 256), 256, 0, st>>>(srcs[i], gbuf, pos, npw, 1, s_in, n3); note_launch(); }
      o.z(Z_INV, gbuf, 1, nullptr, 1.f, tw, st);
      PairMap pm{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
      o.xy_inv(INV_WRITE, gbuf, dsts[i], nullptr, pm, 1, 1.f, tw, st);
    }
    // -alpha phi Conv_x[conj(phi) a], accumulated into the cleared trial field
    PairMap pp{1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1};
    o.xy_fwd(XY_PRODUCT, phi_r, a_r, pp, 1, gbuf, tw, st);
    o.z(Z_CONV, gbuf, 1, kern, 1.f, tw, st);
    CUDA_TRY(cudaMemsetAsync(a_r, 0, n3 * sizeof(cplx<float>), st));
    o.xy_inv(INV_ACCUM, gbuf, a_r, phi_r, pp, 1, (float)(-alpha), tw, st);
    // back to plane waves on the sphere
    PairMap pl{1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0};
    o.xy_fwd(XY_LOAD, nullptr, a_r, pl, 1, gbuf, tw, st);
    o.z(Z_FWD, gbuf, 1, nullptr, 1.f, tw, st);
    const float s_out = (float)(std::sqrt(a * a * a) / (double)n3);
    { k_gather<float><<<grid_for(npw, 256), 256, 0, st>>>(gbuf, pos, npw, 1, s_out, nullptr, nullptr, nullptr, 1, 0,
                                                           (cplx<float>*)out_pw, n3); note_launch(); }
    return check_launch("tddft_exchange_pair_noalloc");
  });
}

// ---------------------------------------------------------------------------
// host-only test entry points of the small dense routines
// ---------------------------------------------------------------------------
extern "C" {

tddft_status tddft_testing_herm_eig(int n, const double* A, double* w, double* V) {
  return abi_guard([&]() -> tddft_status {
    if (n < 1 || !A || !w || !V) return fail(TDDFT_EINVAL, "n >= 1 and non-null arrays required");
    const std::complex<double>* a = reinterpret_cast<const std::complex<double>*>(A);
    std::vector<std::complex<double>> M(a, a + (size_t)n * n), vecs;
    std::vector<double> vals;
    const bool ok = herm_eig(n, M, vals, vecs);
    std::copy(vals.begin(), vals.end(), w);
    std::copy(vecs.begin(), vecs.end(), reinterpret_cast<std::complex<double>*>(V));
    return ok ? TDDFT_OK : fail(TDDFT_ENUMERIC, "Jacobi sweeps did not converge");
  });
}

tddft_status tddft_testing_herm_eig_device(int n, int nr, const double* A, double* w, double* V) {
  return abi_guard([&]() -> tddft_status {
    if (n < 1 || nr < 1 || nr > n || !A || !w || !V) return fail(TDDFT_EINVAL, "1 <= nr <= n and non-null arrays required");
    if (n > JACOBI_MAX_N) return fail(TDDFT_EINVAL, "n above the device solver's limit of " + std::to_string(JACOBI_MAX_N));
    TempAllocs tmp;
    void *dA = nullptr, *dV = nullptr, *dS = nullptr, *dw = nullptr;
    const size_t nn = (size_t)n * n * sizeof(cplx<double>);
    STATUS_TRY(tmp.get(&dA, nn));
    STATUS_TRY(tmp.get(&dV, nn));
    STATUS_TRY(tmp.get(&dS, (size_t)n * nr * sizeof(cplx<double>)));
    STATUS_TRY(tmp.get(&dw, (size_t)(nr + 1) * sizeof(double)));
    CUDA_TRY(cudaMemcpy(dA, A, nn, cudaMemcpyHostToDevice));
    k_herm_jacobi<<<1, JACOBI_THREADS>>>((cplx<double>*)dA, (cplx<double>*)dV, n, nr, (double*)dw, (cplx<double>*)dS,
                                         (double*)dw + nr);
    note_launch();
    STATUS_TRY(check_launch("device Jacobi"));
    std::vector<double> wf(nr + 1);
    CUDA_TRY(cudaMemcpy(wf.data(), dw, wf.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(V, dS, (size_t)n * nr * sizeof(cplx<double>), cudaMemcpyDeviceToHost));
    std::copy(wf.begin(), wf.begin() + nr, w);
    return wf[nr] == 1.0 ? TDDFT_OK : fail(TDDFT_ENUMERIC, "Jacobi sweeps did not converge");
  });
}

tddft_status tddft_testing_cholesky(int n, double* A) {
  return abi_guard([&]() -> tddft_status {
    if (n < 1 || !A) return fail(TDDFT_EINVAL, "n >= 1 and a non-null array required");
    std::complex<double>* a = reinterpret_cast<std::complex<double>*>(A);
    std::vector<std::complex<double>> M(a, a + (size_t)n * n);
    if (!cholesky_lower(n, M)) return fail(TDDFT_ENUMERIC, "matrix is not positive definite");
    std::copy(M.begin(), M.end(), a);
    return TDDFT_OK;
  });
}

tddft_status tddft_testing_lower_inverse(int n, const double* L, double* X) {
  return abi_guard([&]() -> tddft_status {
    if (n < 1 || !L || !X) return fail(TDDFT_EINVAL, "n >= 1 and non-null arrays required");
    const std::complex<double>* l = reinterpret_cast<const std::complex<double>*>(L);
    for (int i = 0; i < n; ++i)
      if (l[(size_t)i * n + i] == 0.0) return fail(TDDFT_EINVAL, "zero on the diagonal");
    const std::vector<std::complex<double>> inv = lower_inverse(n, std::vector<std::complex<double>>(l, l + (size_t)n * n));
    std::copy(inv.begin(), inv.end(), reinterpret_cast<std::complex<double>*>(X));
    return TDDFT_OK;
  });
}

tddft_status tddft_testing_inject_fault(int kind, int after) {
  return abi_guard([&]() -> tddft_status {
    if (after < 0) return fail(TDDFT_EINVAL, "after must be >= 0");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    switch (kind) {
      case TDDFT_FAULT_NONE:
        g_fault_alloc = -1;
        g_fault_wait = false;
        break;
      case TDDFT_FAULT_ALLOC:
        g_fault_alloc = after;
        break;
      case TDDFT_FAULT_DEVICE_WAIT:
        g_fault_wait = true;
        break;
      default:
        return fail(TDDFT_EINVAL, "unknown fault kind " + std::to_string(kind));
    }
    fault_rearm_locked();
    return TDDFT_OK;
  });
}

tddft_status tddft_testing_fault_state(int* alloc_after, int* wait) {
  return abi_guard([&]() -> tddft_status {
    if (!alloc_after || !wait) return fail(TDDFT_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    *alloc_after = g_fault_alloc;
    *wait = g_fault_wait ? 1 : 0;
    return TDDFT_OK;
  });
}

}  // extern "C"
