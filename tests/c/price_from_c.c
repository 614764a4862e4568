/* The C ABI used from plain C99: price three strikes with host buffers.
 * Exit status 0 with one line per strike, or 2 with the library's message when
 * no context can be created (for example, on a machine without a GPU). */
#include <stdio.h>

#include "simr.h"

int main(void) {
  simr_ctx* ctx = NULL;
  int rc = simr_create(&ctx, 0);
  if (rc != SIMR_OK) {
    printf("no context: %d %s\n", rc, simr_last_error());
    return 2;
  }
  const simr_heston model = {100.0, 0.05, 1.0, 0.04, 1.5, 0.04, 0.3, -0.7}; /* S0 r T v0 kappa theta sigma rho */
  const double strikes[3] = {90.0, 100.0, 110.0};
  double price[3], stderr_[3];
  rc = simr_price(ctx, &model, strikes, 3, 0, 64, 65536, 1, 0, price, stderr_, NULL);
  if (rc != SIMR_OK) {
    printf("simr_price: %d %s\n", rc, simr_last_error());
    simr_destroy(ctx);
    return 1;
  }
  for (int i = 0; i < 3; ++i) printf("K=%.1f price=%.10f stderr=%.3e\n", strikes[i], price[i], stderr_[i]);
  simr_destroy(ctx);
  return 0;
}
