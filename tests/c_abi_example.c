/*
 * The C ABI driven from plain C (no C++, no Python): a square duct along z
 * (solid walls at x = 0, nx-1 and y = 0, ny-1, periodic in z), body force
 * along z, stepped in the FP64-storage form.  Prints the fluid-cell count,
 * the mass and the mean axial velocity of the last step, then checks that a
 * bad argument is refused with a message.  tests/test_c_abi_example.py
 * compiles it with a C compiler and compares its output with the oracle.
 *
 * usage: c_abi_example nx ny nz steps
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "lbm.h"

static int check(int rc, const char* what) {
  if (rc != LBM_OK) {
    fprintf(stderr, "%s failed: %d %s\n", what, rc, lbm_last_error());
    exit(2);
  }
  return rc;
}

int main(int argc, char** argv) {
  if (argc != 5) {
    fprintf(stderr, "usage: %s nx ny nz steps\n", argv[0]);
    return 1;
  }
  const int32_t dims[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
  const int32_t steps = atoi(argv[4]);
  const size_t box = (size_t)dims[0] * dims[1] * dims[2];
  uint8_t* flags = (uint8_t*)malloc(box);
  for (int32_t z = 0; z < dims[2]; ++z)
    for (int32_t y = 0; y < dims[1]; ++y)
      for (int32_t x = 0; x < dims[0]; ++x)
        flags[x + (size_t)dims[0] * (y + (size_t)dims[1] * z)] =
            (x == 0 || y == 0 || x == dims[0] - 1 || y == dims[1] - 1) ? 1 : 0;

  lbm_ordering ord;
  ord.kind = LBM_ORDER_LEX;
  ord.block[0] = ord.block[1] = ord.block[2] = 1;
  ord.periodic = 4u; /* z */
  lbm_sparse* sp = NULL;
  lbm_state* st = NULL;
  /* host flags: the library copies them to the device itself */
  check(lbm_build_sparse(flags, dims, ord, NULL, &sp), "lbm_build_sparse");
  int64_t n = 0;
  check(lbm_sparse_info(sp, &n, NULL, NULL, NULL), "lbm_sparse_info");
  check(lbm_state_create(sp, LBM_F64X, 0, &st), "lbm_state_create");

  const double omega_plus = 1.0 / 0.8;
  const double omega_minus = 1.0 / (0.5 + (3.0 / 16.0) / (1.0 / omega_plus - 0.5));
  const double force[3] = {0.0, 0.0, 1e-5};
  check(lbm_step(st, steps, omega_plus, omega_minus, force), "lbm_step");
  double mass = 0.0, flux = 0.0;
  check(lbm_reduce_flux(st, 2, &mass, &flux), "lbm_reduce_flux");
  printf("%lld %.17g %.17g\n", (long long)n, mass, flux);

  /* a refused call: negative step count */
  const int rc = lbm_step(st, -1, omega_plus, omega_minus, force);
  if (rc != LBM_EINVAL || lbm_last_error()[0] == '\0') {
    fprintf(stderr, "a negative step count was not refused (%d)\n", rc);
    return 3;
  }

  lbm_free(st);
  lbm_free(sp);
  free(flags);
  return 0;
}
