/* Plain-C client of the library's C ABI: host-only calls (no device needed). */
#include <stdio.h>

#include "mg.h"

int main(void) {
  mg_options o;
  mg_default_options(&o);
  printf("%d %d %d %d %d %.3f %d %d %d %g %d %d %d\n", o.transfer, o.coarse, o.precision, o.nu1, o.nu2, o.omega,
         o.coarsest_level, o.use_graphs, o.persistent, o.eps_mf, o.smoother, o.gs_sweeps, o.cycle);
  mg_grid* g = NULL;
  if (mg_create_grid(2, 3, NULL, &g) != MG_OK) {
    printf("create failed: %s\n", mg_last_error());
    return 1;
  }
  mg_level_info info;
  if (mg_grid_info(g, 3, &info) != MG_OK) return 2;
  printf("%lld %lld %d\n", (long long)info.n_dofs, (long long)info.n_slots, info.brick_edge);
  size_t bytes = 0;
  if (mg_hier_footprint(g, &o, &bytes) != MG_OK || bytes == 0) return 3;
  o.cycle = MG_CYCLE_ADDITIVE;
  o.precision = MG_PREC_MIXED_BF16;
  mg_hier* h = NULL;
  const mg_status st = mg_hier_create(g, &o, &h);  /* rejected before any device call */
  printf("%d %s\n", (int)st, h == NULL ? "null" : "handle");
  mg_destroy_grid(g);
  return 0;
}
