// Host helpers shared by the library's translation units.
#pragma once
#include "coupledmg.h"

namespace cmg {
// Records the calling thread's error message (read by mg_last_error) and
// returns the status.
mg_status set_error(mg_status s, const char *msg);

// Checks a grid on its own (dimensions, spacing, boundary kinds and values):
// every entry point that takes an mg_grid applies the same rules.  Returns
// MG_OK or MG_ERR_INVALID_ARG with the message set.
mg_status check_grid_geom(const mg_grid *g);
}  // namespace cmg
