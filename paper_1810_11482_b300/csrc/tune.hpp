// Tuning registry: launch-shape and work-split knobs of the built-in kernels.
// No knob changes a result (every kernel evaluates the same canonical
// expression for any value); they only change speed.  Values come from the
// defaults below, then from a JSON cache written by the autotuner
// (paper_1810_11482_b300/autotune.py), then from hxc_tune_set.
#pragma once

#include <cstdint>

#include "hxc.h"

namespace hxc {
namespace tune {

// Value of a knob (its default if never set).  Unknown keys return dflt.
int64_t get(const char *key);
// Sets a known knob (clamped to its range); false for an unknown key.
bool set(const char *key, int64_t value);
bool known(const char *key);
// Incremented by every change of a knob's value (set or cache load); part
// of the key of every cached CUDA graph, so that a graph captured before a
// change (with other launch shapes or kernel variants) is not replayed.
uint64_t generation();
// Loads {"sm_<major><minor>": {"key": int, ...}, ...} for the given
// architecture (or a flat {"key": int} object).  Returns HXC_E_INVALID on a
// malformed file, HXC_OK when the file is absent is not an error for the
// automatic load (see load_default).
hxc_status load_file(const char *path, int major, int minor);
// Once per process: HXC_TUNE_CACHE if set, else tune_cache.json next to the
// library, if present.
void load_default(int major, int minor);

}  // namespace tune
}  // namespace hxc
