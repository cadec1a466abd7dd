/* A plain C99 client of the library's C ABI (include/tddft.h, include/tddft_testing.h), for the
 * entry points that need no GPU: sphere size, exchange grid, status strings and the last error,
 * the maximally localised frame, the LDA kernels, the fault injector and a dense FP64 routine. Built and run by
 * tests/test_c_client_cpu.py.
 *
 *   host_client ORBITALS U_OUT
 * ORBITALS: int32 nocc, int32 npw, then nocc * npw complex128 (re, im) rows of the 72^3 cell
 * (a = 13.48 bohr, 25 Ha); U_OUT receives nocc * nocc complex128 of tddft_localize. */
#include <stdio.h>
#include <stdlib.h>

#include "tddft.h"
#include "tddft_testing.h"

static int check(tddft_status s, const char* what) {
  if (s != TDDFT_OK) {
    fprintf(stderr, "%s: %s: %s\n", what, tddft_status_string(s), tddft_last_error());
    return 1;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: host_client ORBITALS U_OUT\n");
    return 2;
  }
  int npw = 0, nx = 0;
  if (check(tddft_sphere_size(72, 13.48, 25.0, &npw), "tddft_sphere_size")) return 1;
  printf("sphere_size %d\n", npw);
  if (check(tddft_exchange_grid(72, 13.48, 25.0, TDDFT_PREC_FP32, &nx), "tddft_exchange_grid")) return 1;
  printf("exchange_grid %d\n", nx);

  /* an invalid argument: a status, its string and the detail of the last error */
  tddft_status s = tddft_sphere_size(7, 5.0, 1.0, &npw);
  printf("invalid %d %s\n", (int)s, tddft_status_string(s));
  printf("last_error %s\n", tddft_last_error());

  /* the localised frame of the given orbitals */
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int hdr[2];
  if (fread(hdr, sizeof(int), 2, f) != 2) return 1;
  const int nocc = hdr[0], n_pw = hdr[1];
  double* phi = malloc(sizeof(double) * 2 * (size_t)nocc * n_pw);
  double* U = malloc(sizeof(double) * 2 * (size_t)nocc * nocc);
  if (!phi || !U) return 1;
  if (fread(phi, sizeof(double) * 2, (size_t)nocc * n_pw, f) != (size_t)nocc * n_pw) return 1;
  fclose(f);
  double spread[2];
  int sweeps = 0;
  if (check(tddft_localize(72, 13.48, 25.0, nocc, phi, 200, 1e-10, U, spread, &sweeps), "tddft_localize")) return 1;
  printf("localize %.17g %.17g %d\n", spread[0], spread[1], sweeps);
  f = fopen(argv[2], "wb");
  if (!f || fwrite(U, sizeof(double) * 2, (size_t)nocc * nocc, f) != (size_t)nocc * nocc) return 1;
  fclose(f);
  free(phi);
  free(U);

  /* the fault injector: arm, read back, disarm */
  int after = 0, wait = 0;
  if (check(tddft_testing_inject_fault(TDDFT_FAULT_ALLOC, 3), "inject")) return 1;
  if (check(tddft_testing_inject_fault(TDDFT_FAULT_DEVICE_WAIT, 0), "inject")) return 1;
  if (check(tddft_testing_fault_state(&after, &wait), "fault_state")) return 1;
  printf("fault %d %d\n", after, wait);
  if (check(tddft_testing_inject_fault(TDDFT_FAULT_NONE, 0), "inject")) return 1;

  /* LDA kernels of two spin densities */
  const double ru[3] = {0.1, 0.3, 0.02}, rd[3] = {0.1, 0.05, 0.02 + 5e-4};
  double vu[3], vd[3], fx[3], fsf[3];
  if (check(tddft_lda_kernels(3, ru, rd, 1e-3, vu, vd, fx, fsf), "lda")) return 1;
  printf("lda %.17g %.17g %.17g %.17g %.17g %.17g\n", vu[1], vd[1], fx[1], fsf[1], fsf[0], fsf[2]);

  /* Cholesky of [[4, 2+i], [2-i, 3]] (row-major interleaved complex128) */
  double A[8] = {4.0, 0.0, 2.0, 1.0, 2.0, -1.0, 3.0, 0.0};
  if (check(tddft_testing_cholesky(2, A), "cholesky")) return 1;
  printf("cholesky %.17g %.17g %.17g %.17g\n", A[0], A[4], A[5], A[6]);
  return 0;
}
