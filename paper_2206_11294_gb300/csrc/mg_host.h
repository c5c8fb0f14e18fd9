// Host helpers shared by the library's translation units.
#pragma once
#include "coupledmg.h"

namespace cmg {
// Records the calling thread's error message (read by mg_last_error) and
// returns the status.
mg_status set_error(mg_status s, const char *msg);
}  // namespace cmg
