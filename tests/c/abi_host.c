/* A plain C11 program against include/lbs.h and include/lbs_serve.h: the
 * headers compile as C, the library links, and its host-side entry points
 * answer without a GPU.  Prints "ok" and exits 0, else names the check. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "lbs.h"
#include "lbs_serve.h"

#define CHECK(cond)                            \
  do {                                         \
    if (!(cond)) {                             \
      printf("failed: %s\n", #cond);           \
      return 1;                                \
    }                                          \
  } while (0)

int main(void) {
  lbs_lattice lat;
  memset(&lat, 0, sizeof(lat));
  lat.nx = 64;
  lat.ny = 32;
  lat.dx = 1.0 / 32;
  lat.tau = 0.55;
  lat.precision = LBS_FP32;
  lat.wall_extrap = LBS_EXTRAP_OWN;
  lbs_material mat = {LBS_NH, 1.0, 0.25, 1.0, {0.0, 0.0}};

  /* plane strain at nu = 1/4: lam = mu; c = sqrt(3) c_s; dt = dx / c */
  double p[5];
  CHECK(lbs_params(&lat, &mat, p) == LBS_OK);
  CHECK(fabs(p[1] / p[0] - 1.0) < 1e-14);
  CHECK(fabs(p[3] / p[2] - sqrt(3.0)) < 1e-14);
  CHECK(fabs(p[4] - lat.dx / p[3]) < 1e-15);

  /* the linear wall reading adds a second side-array layer to both buffers */
  const size_t own = lbs_footprint(&lat);
  lat.wall_extrap = LBS_EXTRAP_LINEAR;
  CHECK(own > 0 && lbs_footprint(&lat) == own + 2 * 4 * 64 * 4 * sizeof(float));
  lat.wall_extrap = LBS_EXTRAP_OWN;

  /* the kernels' constitutive forms: H = 0 gives P = N = 0 */
  double H[4] = {0, 0, 0, 0}, P[4], N[4];
  CHECK(lbs_constitutive(LBS_SVK, p[1], p[0], H, P, N) == LBS_OK);
  CHECK(P[0] == 0.0 && P[1] == 0.0 && P[2] == 0.0 && P[3] == 0.0 && N[0] == 0.0 && N[3] == 0.0);

  int32_t count = 0, tx[64], ty[64];
  CHECK(lbs_tile_variants(LBS_FP32, &count, tx, ty) == LBS_OK && count >= 2 && count <= 64);

  /* invalid configurations are refused before any device work */
  lbs_handle *h = NULL;
  lat.nx = 2;
  CHECK(lbs_create(&lat, &mat, NULL, &h) == LBS_EINVAL && h == NULL);
  lat.nx = 64;
  lat.wall_extrap = 7;
  CHECK(lbs_create(&lat, &mat, NULL, &h) == LBS_EINVAL);
  CHECK(lbs_strerror(LBS_EINVAL) != NULL && strlen(lbs_strerror(LBS_EINVAL)) > 0);
  CHECK(lbs_destroy(NULL) == LBS_OK);
  printf("ok\n");
  return 0;
}
