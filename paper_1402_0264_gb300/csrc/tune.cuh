// The autotuner's cache (tune.cu): measured choices per device model and size class.
#pragma once

#include <stdint.h>

#include "polymul.h"

namespace pm {

struct TuneChoice {
    int s;        // block parameter
    int64_t q;    // unit size of the warp-level batched schedule (0: the default)
    float ms;     // the time it was chosen with (informational)
};

// The cached choice for the current device and this size class (form PM_TUNE_PLAIN:
// x = n, y = m; PM_TUNE_BATCHED: x = max_deg + 1, y = batch); false if none.
bool tune_get(int form, uint32_t p, int64_t x, int64_t y, TuneChoice* out);
void tune_put(int form, uint32_t p, int64_t x, int64_t y, const TuneChoice& v);

}  // namespace pm
