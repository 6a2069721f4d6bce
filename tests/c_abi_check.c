/* A plain C caller of the library (no Python, no torch): calls that need no device.
 * Exit status = number of failed checks. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "hub.h"

static int failures = 0;

static void expect(int ok, const char *what) {
  if (!ok) {
    ++failures;
    printf("FAIL %s (%s)\n", what, hub_last_error());
  }
}

int main(void) {
  int64_t r = 0, c = 0, d = 0;
  int32_t perm[4] = {1, 2, 3, 0}, chi[1] = {1};
  expect(hub_set_symmetry(NULL, HUB_SYM_K0) == HUB_ERR_ARG, "hub_set_symmetry(NULL)");
  expect(hub_set_translations(NULL, 1, perm, chi) == HUB_ERR_ARG, "hub_set_translations(NULL)");
  expect(hub_k_dims(NULL, &r, &c, &d) == HUB_ERR_ARG, "hub_k_dims(NULL)");
  expect(hub_apply(NULL, NULL, NULL, NULL) == HUB_ERR_ARG, "hub_apply(NULL)");
  expect(hub_last_error() != NULL && hub_last_error()[0] != '\0', "hub_last_error message");
  hub_free(NULL);

  /* one-coefficient continued fraction: G(z) = n2 / (z - s (a0 - E0)); with n2 = 3, a0 = 2,
     E0 = 0.5, s = +1, z = 1 + 0.5i: 3 / (-0.5 + 0.5i) = -3 - 3i */
  double a[1] = {2.0}, b[1] = {0.0}, zr[1] = {1.0}, zi[1] = {0.5}, gr[1] = {0.0}, gi[1] = {0.0};
  expect(hub_green_eval(1, a, b, 3.0, 0.5, 1, 1, zr, zi, gr, gi) == HUB_OK, "hub_green_eval");
  expect(fabs(gr[0] + 3.0) < 1e-14 && fabs(gi[0] + 3.0) < 1e-14, "hub_green_eval value");
  /* hole term (s = -1): 3 / (1 + 0.5i + 1.5) = 3 (2.5 - 0.5i) / 6.5 */
  expect(hub_green_eval(1, a, b, 3.0, 0.5, -1, 1, zr, zi, gr, gi) == HUB_OK, "hub_green_eval hole");
  expect(fabs(gr[0] - 7.5 / 6.5) < 1e-14 && fabs(gi[0] + 1.5 / 6.5) < 1e-14, "hub_green_eval hole value");
  expect(hub_green_eval(1, a, b, 3.0, 0.5, 2, 1, zr, zi, gr, gi) == HUB_ERR_ARG, "hub_green_eval bad sign");

  printf("%s: %d failure(s)\n", failures ? "FAIL" : "ok", failures);
  return failures;
}
