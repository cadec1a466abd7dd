/*
 * C ABI of the B300 library for the Tamm-Dancoff Liouville operator of hybrid
 * linear-response TDDFT in plane waves at the Gamma point (spin-conserving and
 * spin-flip), after Jin, Yu, Govoni, Xu, Galli, arXiv:2309.03513.
 *
 * Conventions (all calls)
 * -----------------------
 * Cubic cell of side a (bohr), Omega = a^3, FFT grid n^3, r_j = a j / n,
 * G_m = (2 pi / a) m with m_i in [-n/2, n/2) (n even).
 * Wavefunction sphere S = {m : (1/2)|G_m|^2 < ecut} with |G|^2 computed in
 * FP64 as ((2 pi / a)^2) * |m|^2; its npw points are ordered by
 * (|m|^2, m_x, m_y, m_z) ascending. An orbital is
 *   phi(r_j) = Omega^{-1/2} sum_{G in S} c(G) exp(i G.r_j).
 * Plane-wave arrays are row-major [rows][npw] of interleaved complex numbers:
 * complex128 (two doubles) for TDDFT_PREC_FP64 and for every host input of
 * tddft_init_system, complex64 (two floats) for device buffers of TDDFT_PREC_FP32.
 * Real-space arrays are [n][n][n] indexed [j_z][j_y][j_x] (x fastest).
 * Coulomb kernels: kappa(G) = 4 pi / |G|^2 for G != 0; at G = 0 the exchange
 * kernel takes desc.kx_g0 (e.g. 2 pi R_c^2) and the Hartree kernel 0.
 * Periodic convolution: Conv_kappa[rho] = F^{-1}[kappa N_r^{-1} F[rho]].
 *
 * Errors: every call returns a tddft_status; no exception crosses the ABI.
 * tddft_last_error() gives a thread-local message for the last failure.
 * Streams are passed as void* (a cudaStream_t, NULL for the legacy stream).
 * Calls on one handle must not overlap: a handle owns one workspace.
 */
#ifndef TDDFT_H
#define TDDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tddft_status {
  TDDFT_OK = 0,
  TDDFT_EINVAL = 1,   /* bad argument, unsupported size, non-orthonormal orbitals */
  TDDFT_ENOMEM = 2,   /* device or host allocation failed */
  TDDFT_ECUDA = 3,    /* a CUDA runtime call failed */
  TDDFT_ETIMEOUT = 4, /* a bounded device wait ran out */
  TDDFT_ENUMERIC = 5, /* a small dense eigen/Cholesky step failed */
  TDDFT_ENOTCONV = 6, /* Davidson hit the caller's iteration cap */
  TDDFT_ENOTSUP = 7   /* combination not implemented */
} tddft_status;

/* Terms of L (Eq. 9 / Eq. 21 of the paper); a call applies the terms of the
 * handle's mask. */
#define TDDFT_TERM_D_KIN 1u   /* (1/2|G|^2 - eps_v) a_v            (Eq. 3, kinetic part of H^KS) */
#define TDDFT_TERM_D_VLOC 2u  /* V_loc(r) a_v(r)                    (Eq. 3, local part of H^KS) */
#define TDDFT_TERM_D_EXX 4u   /* +alpha V_X a_v, V_X a = -sum_w phi_w Conv_x[phi_w^* a]
                                 (Eq. 3 with the exchange operator of Sec. 3.1) */
#define TDDFT_TERM_K1E_H 8u   /* phi_v Conv_H[Delta rho]            (Eq. 4; absent for spin-flip, Sec. 2.3) */
#define TDDFT_TERM_K1E_XC 16u /* phi_v f_xc Delta rho               (Eq. 4; f_xc^SF for spin-flip) */
#define TDDFT_TERM_K1D 32u    /* -alpha sum_v' a_v' Conv_x[phi_v'^* phi_v]  (Eq. 6, Sec. 3.2) */
#define TDDFT_TERM_PROJ 64u   /* P^c = 1 - sum_u |phi_u><phi_u| of the target spin (after Eq. 7) */
#define TDDFT_TERMS_ALL 127u  /* the Tamm-Dancoff operator L = D + K1e - K1d (Eq. 9 / Eq. 21) */
/* Terms of the full operator of the Z-vector equation (Eq. 19), spin-conserving
 * handles only (TDDFT_ENOTSUP on spin-flip handles). They act on the complex
 * conjugate of the trial vectors, so with them the operator is linear over the
 * reals only (it is self-adjoint for Re<x|y>); Davidson rejects them. */
#define TDDFT_TERM_K2E_H 128u  /* phi_v Conv_H[sum_v' a_v'^* phi_v']          (Eq. 5) */
#define TDDFT_TERM_K2E_XC 256u /* phi_v f_xc sum_v' a_v'^* phi_v'             (Eq. 5) */
#define TDDFT_TERM_K2D 512u    /* -alpha sum_v' phi_v' Conv_x[a_v'^* phi_v]   (Eq. 7) */
#define TDDFT_TERMS_ZVEC 1023u /* D + K1e - K1d + K2e - K2d */

#define TDDFT_SPIN_CONSERVING 0
#define TDDFT_SPIN_FLIP 1 /* source spin up -> target spin down (Eq. 21) */

#define TDDFT_PREC_FP64 0 /* every step in FP64 (the plain path) */
#define TDDFT_PREC_FP32 1 /* pair products, FFTs, kernel multiplies in complex FP32 */

typedef struct tddft_desc {
  int n;              /* FFT points per axis; supported: 8 12 16 24 32 36 48 64 72 80 96 108 (FP32 also 128) */
  double a;           /* cubic cell side (bohr) */
  double ecut;        /* wavefunction cutoff (Ha) */
  int spin_mode;      /* TDDFT_SPIN_CONSERVING or TDDFT_SPIN_FLIP */
  int nocc_src;       /* occupied orbitals of the source spin: index v of a_v, pairs of K1e/K1d */
  int nocc_tgt;       /* occupied orbitals of the target spin: P^c and V_X inside D (= nocc_src for SC) */
  double alpha;       /* exact-exchange fraction alpha_EXX (Sec. 2.1) */
  double kx_g0;       /* exchange kernel at G = 0 */
  int precision;      /* TDDFT_PREC_FP64 or TDDFT_PREC_FP32 */
  unsigned term_mask; /* TDDFT_TERM_* bits */
  int nb_max;         /* largest batch of trial vectors one call may pass */
} tddft_desc;

/* Inputs of tddft_init_system, all FP64, each in host or device memory (the
 * library copies them with cudaMemcpyDefault). The library keeps its own copies;
 * the caller may free the inputs when the call returns. */
typedef struct tddft_inputs {
  const double* phi_src; /* complex128 [nocc_src][npw], orthonormal */
  const double* phi_tgt; /* complex128 [nocc_tgt][npw], orthonormal; spin-flip only (NULL for SC) */
  const double* eps_src; /* [nocc_src] eigenvalues of the source spin (Eq. 3; Eq. 21 for SF) */
  const double* vloc;    /* [n^3] local potential of the target spin, or NULL (= 0) */
  const double* fxc;     /* [n^3] f_xc(r) (SC) or f_xc^SF(r) (SF), or NULL (= 0) */
} tddft_inputs;

typedef struct tddft_info {
  int npw;                 /* sphere size */
  int n;                   /* grid points per axis */
  int nb_chunk;            /* trial vectors processed per internal pass */
  int precision;
  size_t device_bytes;     /* device memory owned by the handle */
  int n_exchange;          /* grid points per axis of the pair-convolution terms (tuning.exchange_grid) */
} tddft_info;

typedef struct tddft_system* tddft_handle;

/* Size of the sphere S for (n, a, ecut). Host only. EINVAL if S does not fit
 * strictly inside the grid (|m_i| < n/2). */
tddft_status tddft_sphere_size(int n, double a, double ecut, int* npw);

/* Miller indices of S in the library's order: miller[3*i + {0,1,2}] =
 * (m_x, m_y, m_z) of point i. The caller provides npw*3 ints. Host only. */
tddft_status tddft_sphere_miller(int n, double a, double ecut, int* miller);

/* Grid (points per axis) on which tddft_init_system runs the pair-convolution terms
 * when tuning.exchange_grid is on: the smallest supported N_x < n with N_x > 4 M,
 * M = max |m_i| over the sphere S (on such a grid those terms equal the n-grid ones up
 * to rounding, see tddft_tuning.exchange_grid), else n. Host only. EINVAL for an
 * unsupported (n, precision) or when S does not fit the grid. */
tddft_status tddft_exchange_grid(int n, double a, double ecut, int precision, int* n_exchange);

/* Local exchange-correlation kernels of the operator from a ground-state spin density, in the
 * local density approximation (the paper's LDA: Slater exchange and the Perdew-Zunger 1981
 * correlation with its spin interpolation). Host only, FP64, point by point.
 * rho_up, rho_dn: HOST [npts] spin densities (bohr^-3, finite and >= 0, else EINVAL).
 * Optional HOST [npts] outputs (NULL skips one):
 *   vxc_up, vxc_dn: the potentials V_xc,sigma = d(rho eps_xc)/d rho_sigma (Ha);
 *   fxc: the adiabatic local kernel of the spin-up channel, d V_xc,up / d rho_up (Ha bohr^3),
 *     in closed form: the f_xc array of a spin-conserving handle (Eq. 4 with one spin channel);
 *   fxc_sf: the spin-flip kernel (V_xc,up - V_xc,dn) / (rho_up - rho_dn) of Sec. 2.3, set to 0
 *     where |rho_up - rho_dn| < sf_cutoff (the paper uses 1e-3, Supporting Information Sec. S2)
 *     or where the two densities are equal: the f_xc array of a spin-flip handle.
 * Points where the density vanishes get zero potentials and kernels, and fxc is 0 where rho_up
 * vanishes (it diverges like rho_up^(-2/3) there). Near rs = 1 the two branches of the
 * correlation fit meet with a small mismatch of value and slope, as published. */
tddft_status tddft_lda_kernels(long long npts, const double* rho_up, const double* rho_dn, double sf_cutoff,
                               double* vxc_up, double* vxc_dn, double* fxc, double* fxc_sf);

/* Build a system: the inputs of the operator of Eq. 9 (spin-flip: Eq. 21) --
 * the occupied orbitals phi_v and eigenvalues eps_v of Eq. 3 (both spins for
 * spin-flip, Sec. 2.3), the local part of H^KS (Eq. 3), the local kernel f_xc of
 * Eq. 4 (f_xc^SF for spin-flip), the exact-exchange fraction alpha of the hybrid
 * functional (Sec. 2.1) and the Coulomb kernel of the exchange terms (Eqs. 3, 6
 * and Sec. 3.1) at G = 0. It copies the inputs to the device, builds the sphere
 * map and kernel tables, transforms the orbitals to real space and allocates
 * the workspace for nb_max trial vectors. The orbitals are checked orthonormal
 * in FP64 (max |Phi^dagger Phi - I| <= 1e-10) -> else TDDFT_EINVAL.
 * When tddft_exchange_grid gives a smaller grid, the handle also builds the
 * same system on that grid for the pair-convolution terms (tuning.exchange_grid);
 * if there is no room for it, every term runs on the n grid (same result).
 * The handle owns all device memory until tddft_destroy. Synchronises the
 * stream before returning. */
tddft_status tddft_init_system(const tddft_desc* desc, const tddft_inputs* in, void* stream,
                               tddft_handle* out);

/* Sizes of the handle. Also synchronises the legacy stream and reports
 * TDDFT_ETIMEOUT if a bounded device wait of the library ran out since the
 * last check (the flag is then cleared). */
tddft_status tddft_query(tddft_handle h, tddft_info* info);

/* Change the term mask of the handle (TDDFT_TERM_* bits; K2 bits on a
 * spin-flip handle -> TDDFT_ENOTSUP). */
tddft_status tddft_set_terms(tddft_handle h, unsigned term_mask);

/* Schedule of the pair-convolution passes (results agree to rounding for
 * every choice). A batch convolves `targets` x `sources` pairs at once
 * (bounded by batch_fields, the intermediate buffer of the handle); K1d
 * builds tau for k1d_block x k1d_block orbital pairs at a time and shares it
 * by every trial vector. accumulate = 0: one CTA per (target, plane) sums its
 * sources in a fixed order; 1: one CTA per pair with atomic accumulation
 * (order not fixed). In set_tuning, 0 (or -1 for accumulate) keeps a value and
 * batch_fields is ignored. Host only. */
typedef struct tddft_tuning {
  int targets;
  int sources;
  int k1d_block;    /* 1..16 */
  int accumulate;   /* 0 or 1 */
  int batch_fields; /* read-only */
  int graph;        /* 1: tddft_apply_liouville captures its launches into a CUDA
                       graph on first use for a given (nb, A, LA, term mask) and
                       replays it on the caller's stream; 0: plain launches */
  int prune;        /* 1 (default): pair convolutions of the exchange terms and the
                       Hartree convolution keep, after the xy transform, only the
                       (k_x, k_y) columns inside the disc of radius 2 G_max, stored
                       densely: the others are exactly zero for products of two sphere
                       functions when the grid does not alias them (checked at set-up;
                       otherwise full planes are used). The z pass and the
                       intermediate's memory traffic shrink by the share of columns
                       outside the disc (44% on an alias-free 72^3 grid at 25 Ha).
                       Register-resident z pass only. 0: full planes. -1 keeps the
                       value in set_tuning */
  int z_kernel;     /* z pass: 0 shared-memory radix stages; 1 register-resident columns
                       (FP32, n <= 80); 2 (default where it exists: FP32, n = 16, 24,
                       32, 48, 64, 72, 96) as 1, with the compact pair-density
                       convolutions on two threads per column (at n = 96 only those; its
                       other z passes are the shared-memory ones). -1 keeps the value in
                       set_tuning */
  int projector;    /* FP32 handles: projector (and ACE) GEMMs on tcgen05 tensor cores with
                       split-precision TF32 products (hi*hi + hi*lo + lo*hi, FP32
                       accumulation in tensor memory): 1 (default) the operands are first
                       packed as TF32 high / low tiles in the layout of the MMA (a device
                       buffer of at most 1 GiB, grown outside stream capture) and brought
                       into shared memory by bulk copies in a three-stage pipeline; where
                       the packed operands do not fit, as 2; 2 every CTA stages its
                       operands through registers; 0 SIMT FP32. FP64 handles always use
                       SIMT FP64. -1 keeps the value in set_tuning */
  int k1d_sparse;   /* K1d in the localised frame with truncated pairs
                       (tddft_set_localization): 1 only the kept pairs, from a pair
                       list; 0 blocks of k1d_block x k1d_block pairs, blocks without a
                       kept pair skipped; 2 automatic (pair list when fewer than half
                       of the pairs are kept). -1 keeps the value in set_tuning */
  int k1d_cache;    /* 1: K1d reads tau_vv' = Conv_x[phi_v'^* phi_v] (Eq. 6) of every
                       unordered pair from device memory instead of convolving the
                       pairs in every application. The tau depend on the occupied
                       orbitals only; setting 1 builds them once (synchronises; the
                       rows of the diagonal 16 x 16 blocks are stored in both orders:
                       about nocc (nocc + 16) / 2 fields of n^3 points, 27.5 GB for 128
                       orbitals on 72^3 in FP32) and fails with TDDFT_ENOMEM when they
                       do not fit, or with TDDFT_ENOTSUP while the localised frame is on
                       (the truncated K1d of that frame recomputes its pairs; the stored
                       tau serve again once it is switched off). Where the one-pass contraction
                       of k1d_all applies (FP32, at most 128 orbitals, compact intermediates with
                       the register-line passes) the tau are stored point-tiled and contracted by
                       it, whatever k1d_all says. The result equals that
                       of the recomputing path up to rounding. 0 (default): recompute;
                       releases the stored tau. -1 keeps the value in set_tuning */
  int exchange_grid; /* 1 (default): the pair-convolution terms (D_EXX, K1d, K2d) run on the
                       smallest supported grid N_x < n with N_x > 4 max|m_i| over the
                       sphere, when there is one (64^3 for a 72^3 grid at a = 13.48 bohr,
                       25 Ha). On any grid with N > 4 max|m_i| a pair density never folds
                       onto itself and its products with the orbitals fold only onto
                       plane waves outside the sphere, so these terms are the same as on
                       the n grid up to rounding; the local terms (V_loc, K1e, the
                       diagonal) stay on the n grid. tddft_info.n_exchange reports the grid
                       in use. 0: every term on the n grid. -1 keeps the value */
  int xy_kernel;    /* xy passes of the compact pair-density convolutions, where the
                       register-line kernels exist (FP32, n = 32, 48, 64; the shared-memory
                       radix stages elsewhere). Register-line passes transpose the plane once
                       through shared memory and hold each line either in one thread (the
                       whole line transform in registers) or in two lanes (radix-2 butterfly
                       by warp shuffle, the rest in registers). 1 (default): one thread per
                       line in both passes; 2: two lanes per line in both; 3: forward pass
                       one thread per line, inverse pass two lanes per line; 0: the
                       shared-memory radix stages. -1 keeps the value */
  int k1d_all;      /* K1d of the recomputing path (k1d_cache 0) for FP32 handles with at most
                       128 source orbitals whose pair convolutions use compact intermediates
                       and the register-line xy passes (n = 32, 48, 64 after the exchange
                       grid): 1 (default) the tau_vv' of every pair are convolved into a
                       point-tiled device scratch buffer (the size of the stored tau: 19.3 GB
                       for 128 orbitals on 64^3; allocated at the first K1d outside stream
                       capture when it takes at most a quarter of the free device memory)
                       and contracted in one pass that reads each of them once; 0 (and
                       wherever the above does not hold) by k1d_block x k1d_block blocks of
                       pairs. 0 releases the scratch. -1 keeps the value */
} tddft_tuning;
tddft_status tddft_set_tuning(tddft_handle h, const tddft_tuning* t);
tddft_status tddft_get_tuning(tddft_handle h, tddft_tuning* t);

/* Time a fixed set of schedules (batch shapes, accumulate mode, K1d block) on
 * nb trial vectors A (device, handle precision; LA is scratch output), keep
 * the fastest on the handle and return it in *best (may be NULL). Synchronises. */
tddft_status tddft_autotune(tddft_handle h, int nb, const void* A, void* LA, void* stream, tddft_tuning* best);

/* LA = L A for nb trial vectors (Eq. 9 for SC, Eq. 21 for SF).
 * A, LA: device buffers [nb][nocc_src][npw] (complex128 for FP64 handles,
 * complex64 for FP32 handles). They must not alias. Each A_b is assumed
 * orthogonal to the target-spin orbitals (the operator is defined on that
 * space). Asynchronous and stream-ordered; no host synchronisation.
 * nb = 0 is a no-op; nb > nb_max -> TDDFT_EINVAL. */
tddft_status tddft_apply_liouville(tddft_handle h, int nb, const void* A, void* LA, void* stream);

/* Same as tddft_apply_liouville with HOST buffers of the same layout: the call
 * copies A to the device, applies L and copies LA back, then synchronises
 * the stream. */
tddft_status tddft_apply_liouville_host(tddft_handle h, int nb, const void* A_host, void* LA_host, void* stream);

/* Several independent systems (any sizes, spin modes, precisions) in one CUDA
 * graph launch: system i applies L_i to nb[i] trial vectors A[i] -> LA[i]
 * (device buffers, layouts as in tddft_apply_liouville). Each system runs as
 * its own branch of the graph, so uneven systems overlap on the GPU. The graph
 * is captured on the first call and replayed while the argument lists are
 * unchanged (process-wide cache of one graph; not thread-safe). A handle may
 * appear once. Stream-ordered on `stream`. */
tddft_status tddft_apply_liouville_multi(int nsys, const tddft_handle* hs, const int* nb, const void* const* A,
                                         void* const* LA, void* stream);

/* Density responses of the force expression (Secs. 2.2 and 2.3), summed
 * over states with weights w (HOST [nb]):
 *   Delta rho^(x)(r) = sum_v |a_v(r)|^2 - sum_vv' phi_v^*(r) phi_v'(r) <a_v|a_v'>
 *   Delta rho^(Z)(r) = sum_v [Z_v^*(r) phi_v(r) + phi_v^*(r) Z_v(r)]
 * X (and Z, optional): device [nb][nocc_src][npw], handle precision.
 * drho: device double, written. Spin-conserving: [n^3] = Delta rho^(x) (+
 * Delta rho^(Z) when Z is given). Spin-flip (no Z): [2][n^3], channel 0 the
 * target spin (sum_v |a_v|^2), channel 1 the source spin
 * (-sum_vv' phi_v^* phi_v' <a_v|a_v'>). TDDFT_ENOTSUP for Z on a spin-flip
 * handle or while the localised frame is on. One host sync per state. */
tddft_status tddft_relaxed_density(tddft_handle h, int nb, const void* X, const void* Z, const double* w, double* drho,
                                   void* stream);

/* Z-vector equation (Eq. 19): (D + K1e - K1d + K2e - K2d) Z_s = U_s, solved
 * for each state s by conjugate gradients (Sec. 3.3). Spin-conserving handles
 * with the projector term (else TDDFT_ENOTSUP / TDDFT_EINVAL).
 * The operator is the handle's Tamm-Dancoff mask plus the K2 counterpart of
 * every K1 term in it (K1e_H -> K2e_H, K1e_XC -> K2e_XC, K1d -> K2d). With the
 * K2 terms it acts on conj(Z) too: it is linear over the reals and
 * self-adjoint for Re<x|y>, so CG uses that inner product and real steps.
 * Inexact Krylov switch: a state's search direction gets the exact operator
 * while its residual norm ||r_s||_2 (recursively updated, all v and G) is at
 * least lambda_thr, afterwards the operator without K2d. lambda_thr = 0: always
 * exact. A state stops once ||r_s|| < tol; Z starts at 0. precondition = 1:
 * s = P^c [r_v / (1/2|G|^2 - eps_v)], |denominator| clamped to >= 0.1 Ha.
 * U, Z: device [nb][nocc_src][npw] in the handle's precision (nb <= nb_max, no
 * aliasing); Z is written. iterations, exact_iterations, residual: optional
 * host arrays [nb] (CG steps per state, steps with the exact operator, final
 * ||r_s||). Host-driven: two small device->host reads per iteration.
 * TDDFT_ENOTCONV if a state has not reached tol after max_iter steps (Z holds
 * the last iterate); TDDFT_ENUMERIC if <p|L p> <= 0 (the operator is not
 * positive definite on the search space). */
typedef struct {
  double lambda_thr;
  double tol;
  int max_iter;
  int precondition;
} tddft_zvector_opts;
tddft_status tddft_zvector_solve(tddft_handle h, int nb, const void* U, void* Z, const tddft_zvector_opts* opts,
                                 int* iterations, int* exact_iterations, double* residual, void* stream);

/* Right-hand sides of Eq. 19 for nb states X (device [nb][nocc_src][npw]):
 * U_s = -P^c u_s with u_s = d omega_s / d phi^* from the adjoint
 * (tddft_apply_liouville_adjoint with weight 1 on state s alone; Eq. 20,
 * without the parts that come from H^KS, eps and V_xc depending on the
 * ground-state density, which are inputs here). U: device, same layout,
 * written. Spin-conserving handles with ACE off (else TDDFT_ENOTSUP). */
tddft_status tddft_zvector_rhs(tddft_handle h, int nb, const void* X, void* U, void* stream);

/* Localised frame and pair truncation of K1d (Sec. 3.2, Eq. 31).
 * U: HOST complex128 [nocc_src][nocc_src], unitary (max |U^H U - I| <= 1e-10,
 * else TDDFT_EINVAL), relating the handle's given source orbitals to localised
 * ones: phi_v = sum_n U_vn phi~_n (e.g. the rotation to maximally localised
 * Wannier functions, computed elsewhere). The handle then computes in the
 * localised frame: every term of L except the eigenvalue part of D is
 * covariant under the rotation, so L A = U [L~ (U^dagger A) - eps~ U^dagger A]
 * with eps~ = U^dagger diag(eps) U, and in L~ the K1d integrals
 * tau~_mn = Conv_x[phi~_n^* phi~_m] of pairs whose overlap function
 * S_mn = int |phi~_m|^2 |phi~_n|^2 / sqrt(int |phi~_m|^4 int |phi~_n|^4)
 * is below s_thr are taken as zero (whole blocks of such pairs are not
 * computed). s_thr = 0 keeps every pair (the exact operator, in the other frame).
 * Trial vectors and results stay in the given (canonical) frame.
 * S: optional HOST [nocc_src][nocc_src] output of S_mn (evaluated in FP64 from
 * the handle's real-space orbitals); kept_pairs: optional HOST count of ordered
 * pairs (m, n) kept. U = NULL goes back to the given orbitals. The adjoint and
 * tddft_zvector_rhs return TDDFT_ENOTSUP while the frame is on. Synchronises
 * the stream. */
tddft_status tddft_set_localization(tddft_handle h, const double* U, double s_thr, double* S, int* kept_pairs,
                                    void* stream);

/* Maximally localised orbitals at the Gamma point: the unitary U of the localised frame
 * that tddft_set_localization takes (Sec. 3.2: the pair truncation of Eq. 31 works on
 * maximally localised Wannier functions). Host only, FP64; no handle and no GPU needed.
 * phi_pw: HOST complex128 [nocc][npw], the orbitals on the sphere of (n, a, ecut) in the
 * library's order (tddft_sphere_miller), orthonormal. Minimises the spread of a cubic cell
 * Omega = (a/2pi)^2 sum_alpha sum_n (1 - |Z^alpha_nn|^2), Z^alpha_mn = <phi~_m| exp(i 2 pi r_alpha/a)
 * |phi~_n> (evaluated exactly on the plane-wave basis), over unitary rotations: complex
 * Jacobi sweeps over all pairs (m, n), each rotation the closed-form optimum of the joint
 * diagonalisation of the six Hermitian parts of Z^x, Z^y, Z^z (Cardoso and Souloumiac 1996;
 * used for Wannier functions by Gygi, Fattebert and Schwegler 2003), until the largest
 * rotation of a sweep is below tol or max_sweeps sweeps have run.
 * U: HOST complex128 [nocc][nocc] output with phi_v = sum_n U_vn phi~_n (the convention of
 * tddft_set_localization). spread: optional HOST [2], Omega before and after (bohr^2);
 * sweeps: optional HOST count of sweeps run. EINVAL for bad arguments; ENOTCONV when
 * max_sweeps ran out first (U then holds the last iterate, still unitary). The result is a
 * local maximum of sum |Z_nn|^2 reached from the given orbitals. */
tddft_status tddft_localize(int n, double a, double ecut, int nocc, const double* phi_pw, int max_sweeps, double tol,
                            double* U, double* spread, int* sweeps);

/* Adaptively compressed exchange (ACE, Sec. 3.1, Eqs. 29-30) for the exchange
 * term inside D: V_X^ACE = -sum_k |xi_k><xi_k| with xi = W L^{-dagger},
 * W = V_X Psi (exact pair convolutions), -Psi^dagger W = L L^dagger (FP64
 * Cholesky on the host). Psi = the target-spin occupied orbitals followed by
 * n_extra HOST complex128 rows extra[n_extra][npw] (orthonormal and orthogonal
 * to the orbitals; max deviation 1e-10, else TDDFT_EINVAL; NULL if n_extra = 0),
 * e.g. low unoccupied orbitals (the paper uses N_ACE = N_occ + 20 up to
 * 4 N_occ). V_X^ACE equals V_X on span(Psi) and approaches it as the set grows;
 * elsewhere it is an approximation. After a successful build the handle's
 * exchange term uses V_X^ACE: two GEMMs in plane waves (tensor cores for FP32)
 * instead of N_b N_occ N_occ,tgt pair convolutions. TDDFT_ENUMERIC if
 * -Psi^dagger W is not positive definite. Synchronises the stream. */
tddft_status tddft_ace_build(tddft_handle h, int n_extra, const double* extra, void* stream);

/* Switch the built ACE operator on (1) or back to the exact exchange (0). */
tddft_status tddft_ace_enable(tddft_handle h, int enable);

/* Bilinear form omega_b = <P^c X_b | M | P^c X_b> (M = L without the outer
 * P^c; equal to <X_b|L X_b> for X_b orthogonal to the orbitals) and the
 * gradient of E = sum_b w_b omega_b.
 * X: device [nb][nocc_src][npw] (handle precision). w: HOST [nb].
 * omega: device double [nb].
 * grad_phi: device, handle precision, the Wirtinger derivative dE/dc_u^*(G)
 *   with X, eps, V_loc, f_xc and the kernels held fixed and P^c taken on the
 *   handle's orbitals (the part of u_v of the Supporting Information, Sec. S1,
 *   that does not come from the ground-state density). Spin-conserving:
 *   [nocc][npw]. Spin-flip: [nocc_src + nocc_tgt][npw], the source-spin
 *   orbitals first (terms of K1e^SF and K1d^SF), then the target-spin ones
 *   (terms of V_X in D and of P^c).
 * grad_vloc: device double [n^3], dE/dV_loc(r_j) (target spin); may be NULL.
 * Pair convolutions are recomputed, not stored. Written, not accumulated.
 * TDDFT_ENOTSUP while ACE or the localised frame is switched on (the
 * gradient is of the exact operator). */
tddft_status tddft_apply_liouville_adjoint(tddft_handle h, int nb, const void* X, const double* w, double* omega,
                                           void* grad_phi, double* grad_vloc, void* stream);

/* Davidson solver for the lowest eigenpairs of L (Sec. 4 names Davidson's
 * method; block scheme, FP64 orthogonalisation and Rayleigh-Ritz). */
typedef struct tddft_davidson* tddft_dav_handle;

/* Start a solve for nroots roots from nguess >= nroots guess vectors
 * X0 (HOST complex128 [nguess][nocc_src][npw]); 2*nroots <= max_basis <= 1024
 * bounds the basis before a restart (EINVAL outside). Applies L to the guess
 * and synchronises the stream. */
tddft_status tddft_davidson_create(tddft_handle h, int nroots, int nguess, const double* X0, int max_basis,
                                   void* stream, tddft_dav_handle* out);

/* One Davidson iteration (Sec. 4 names Davidson's method for L; the block
 * scheme is this library's): Rayleigh-Ritz on the current basis (H = V^H L V
 * and its Hermitian eigenproblem, both FP64 on the device), Ritz vectors,
 * residuals and their norms, then preconditioned corrections r_i/(|G|^2/2 -
 * eps_v - theta_i) (|denominator| clamped >= 0.1 Ha, eps_v the FP64 values
 * given at set-up), FP64 orthogonalisation against the target orbitals and the
 * basis, and L applied to the new vectors. Writes the current Ritz values
 * (HOST double [nroots]), optionally the residual norms (HOST double [nroots]),
 * and the number of roots with residual norm < tol. One host synchronisation
 * per call (the Ritz values, residual norms and status flags come back in one
 * copy). TDDFT_ENUMERIC if the subspace eigensolver does not converge;
 * TDDFT_ETIMEOUT if a bounded device wait of the projector ran out. */
tddft_status tddft_davidson_step(tddft_dav_handle d, double tol, int* n_converged, double* ritz_values,
                                 double* residual_norms, void* stream);

/* Copy the current Ritz vectors to HOST complex128 [nroots][nocc_src][npw]. */
tddft_status tddft_davidson_vectors(tddft_dav_handle d, double* X_host, void* stream);

tddft_status tddft_davidson_destroy(tddft_dav_handle d);

tddft_status tddft_destroy(tddft_handle h);

/* Instrumentation (process-wide, not thread-safe). With the profiler enabled
 * every launch of the three FFT plane kernels is bracketed by CUDA events on
 * its stream. tddft_profile_read synchronises on those events and returns, per
 * class (0: forward xy pass with the pair product, 1: z pass with the kernel
 * multiply, 2: inverse xy pass with the re-multiply and accumulation), the
 * summed device time in ms, the launch count and the algorithmic bytes (each
 * operand read once, each output written once; the z pass counts the kernel
 * table once per launch). total_launches counts every kernel launch of the
 * library since it was loaded. Enabling resets the per-class records. */
#define TDDFT_PROFILE_CLASSES 3
tddft_status tddft_profile_enable(int enable);
tddft_status tddft_profile_read(double* ms, long long* launches, double* bytes, long long* total_launches);

/* Allocation-free exchange pair term (no counterpart in the paper; a service
 * for callers that cannot allocate device memory and so cannot create a
 * handle, e.g. codes that give all device memory to their own pool allocator).
 *
 * Computes, for one occupied orbital phi and one trial orbital a given as
 * plane-wave coefficients on the sphere of (n, a, ecut):
 *   out = PW[ -alpha * phi(r) * Conv_x[conj(phi) a](r) ]
 * (the exchange term alpha V_X a of Sec. 3.1 for a single occupied orbital),
 * in complex FP32 with the same kernels as tddft_apply_liouville.
 * phi_pw, a_pw, out_pw: device complex64 [npw]; the caller owns them.
 * The call allocates nothing: its working memory is one file-scope device
 * array of 3.5 MiB that every GPU which loads the library keeps until the
 * process exits, which limits n to <= 48 (larger n -> TDDFT_EINVAL with a
 * message naming the limit). Set-up: the first call on a device looks up the
 * array's device address, and the first call with a given n on a device sets
 * the launch attributes and constant twiddles of that grid (synchronous);
 * make such first calls before any stream capture. The array also holds the
 * tables of one geometry (twiddles, Coulomb kernel, sphere map): a call whose
 * (n, a, ecut, kx_g0) differs from the geometry the array holds rebuilds them
 * on the host and copies them in with cudaMemcpyAsync on `stream` (the host
 * buffers are pageable and released on return); a call with the same geometry
 * launches kernels only. Every call uses the same array and leaves its
 * contents behind (the fields it needs at zero are cleared by the call itself);
 * calls whose work overlaps on the GPU (different streams, or several host
 * threads) race on it and must be serialised by the caller. Stream-ordered
 * on `stream`. */
tddft_status tddft_exchange_pair_noalloc(int n, double a, double ecut, double alpha, double kx_g0,
                                         const void* phi_pw, const void* a_pw, void* out_pw, void* stream);

const char* tddft_status_string(tddft_status s);
const char* tddft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TDDFT_H */
