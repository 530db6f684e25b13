/* The C ABI from a plain C11 program: include/bvc.h compiles with -pedantic
 * -Werror as C, and host-side calls behave as declared (argument errors are
 * returned synchronously, before any device work). */
#include <stdio.h>
#include <string.h>

#include "bvc.h"

int main(void) {
  int bad = 0;
  const float v[4] = {0.0f, 0.0f, 1.0f, 0.0f};
  const int32_t f[2] = {0, 1};
  bvc_geometry g = NULL;
  bvc_mixed m = NULL;
  if (bvc_version() <= 0) ++bad;
  if (bvc_geometry_create(2, NULL, 2, f, 1, NULL, &g) != BVC_ERR_INVALID_ARG || g != NULL) ++bad;
  if (bvc_geometry_create(4, v, 2, f, 1, NULL, &g) != BVC_ERR_INVALID_ARG) ++bad;
  if (bvc_geometry_destroy(NULL) != BVC_ERR_INVALID_ARG) ++bad;
  if (bvc_mixed_set_silhouette_gap(m, 0.1) != BVC_ERR_INVALID_ARG) ++bad;
  if (bvc_status_string(BVC_OK) == NULL || strlen(bvc_status_string(BVC_ERR_INVALID_ARG)) == 0) ++bad;
  printf("version %d, bad %d, invalid-arg string: %s\n", (int)bvc_version(), bad,
         bvc_status_string(BVC_ERR_INVALID_ARG));
  return bad == 0 ? 0 : 1;
}
