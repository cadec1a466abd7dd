/*
 * Test entry points to the library's small dense FP64 routines. They are the routines that
 * the Davidson step uses for its Rayleigh-Ritz problem (Hermitian eigenproblem, solved on
 * the device) and that the ACE build uses for -M = L L^dagger and L^{-1} (Sec. 3.1); they
 * are not part of the operator's interface. Also the measured arithmetic peaks and the
 * host-side fault injector.
 *
 * Matrices are row-major n x n arrays of interleaved complex128 (2n^2 doubles), owned by
 * the caller, in host memory. Only tddft_testing_herm_eig_device touches the GPU.
 */
#ifndef TDDFT_TESTING_H
#define TDDFT_TESTING_H

#include "tddft.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Eigenvalues (ascending, w[n]) and eigenvectors (columns of V) of the Hermitian matrix A,
 * by cyclic complex Jacobi rotations. EINVAL for n < 1 or a null pointer; ENUMERIC when the
 * sweeps do not converge (w and V then hold the last iterate). */
tddft_status tddft_testing_herm_eig(int n, const double* A, double* w, double* V);

/* The device solver of the Davidson step's Rayleigh-Ritz matrix (one-CTA cyclic Jacobi in the
 * round-robin order, FP64) on the current device: the nr lowest eigenvalues (ascending, w[nr])
 * and their eigenvectors (V [n][nr] row-major, column j for w[j]) of the Hermitian part of A.
 * Allocates and frees its own device buffers and synchronises. EINVAL unless 1 <= nr <= n <=
 * 1024; ENUMERIC when the sweeps do not converge. */
tddft_status tddft_testing_herm_eig_device(int n, int nr, const double* A, double* w, double* V);

/* Measured arithmetic peak of the current device, for roofline denominators: which = 0 FP32
 * FMA throughput of the CUDA cores (16 independent FMA chains per thread, 8 CTAs of 256
 * threads per SM); which = 1 TF32 tensor-core throughput (tcgen05.mma kind::tf32, M = 128,
 * N = 256, K = 8, one issuing thread per SM, operands in shared memory, accumulator in tensor
 * memory). Writes TFLOP/s (2 flops per multiply-add) of the fastest of three timed launches
 * after a warm-up, and optionally that launch's ms. Synchronises; EINVAL for another which;
 * ETIMEOUT if a bounded wait of the tensor-core kernel ran out. */
tddft_status tddft_testing_peak(int which, double* tflops, double* ms);

/* In place: the lower Cholesky factor L of a Hermitian positive definite A (A = L L^dagger,
 * real positive diagonal, zeros above it). ENUMERIC when a pivot is not positive. */
tddft_status tddft_testing_cholesky(int n, double* A);

/* X = L^{-1} for a lower-triangular L with non-zero diagonal. */
tddft_status tddft_testing_lower_inverse(int n, const double* L, double* X);

/* Host-side fault injection, for testing how callers handle the library's failure statuses
 * (failure detection; the paper has no counterpart). Nothing fails on
 * the GPU: the library reports an allocation or a bounded device wait as failed.
 *   TDDFT_FAULT_NONE: disarm every fault.
 *   TDDFT_FAULT_ALLOC: the library's device allocation number `after` from now (0 = the next one;
 *     every cudaMalloc the library makes counts) fails as cudaMalloc does when memory runs out.
 *     The entry point that made it returns TDDFT_ENOMEM after releasing what it had allocated
 *     ("(injected fault)" in tddft_last_error), or, where the allocation is optional (the
 *     all-pairs K1d scratch, the packed projector operands), takes its fallback path.
 *   TDDFT_FAULT_DEVICE_WAIT: the next check of a handle's device-wait flag (tddft_query,
 *     tddft_apply_liouville_host, the Davidson step, the Z-vector solve) reports that a bounded
 *     device wait ran out: TDDFT_ETIMEOUT ("results of the call are invalid"); `after` is not used.
 * Each armed fault fires once. The environment variable TDDFT_FAULT ("alloc", "alloc:N" or
 * "wait"), read when the library is loaded, arms the same faults. Process-wide and thread-safe;
 * host only. EINVAL for an unknown kind or after < 0. */
#define TDDFT_FAULT_NONE 0
#define TDDFT_FAULT_ALLOC 1
#define TDDFT_FAULT_DEVICE_WAIT 2
tddft_status tddft_testing_inject_fault(int kind, int after);

/* The armed faults: *alloc_after = allocations still let through before the injected failure
 * (-1: none armed), *wait = 1 while a device-wait fault is armed. Host only. */
tddft_status tddft_testing_fault_state(int* alloc_after, int* wait);

#ifdef __cplusplus
}
#endif

#endif /* TDDFT_TESTING_H */
