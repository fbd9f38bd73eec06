// Helpers shared by the C entry points.
#pragma once

#include <stddef.h>

#include "bsrht.h"

namespace bsrht {

// Device scratch from the library pool of the current device.
int pool_get(size_t bytes, void** out);
// Caller workspace if given (checked against need), else the pool.
int workspace_for(const bsrht_opts* o, size_t need, void** out);
// *o, or the defaults of bsrht_opts_init when o is NULL.
bsrht_opts opts_or_default(const bsrht_opts* o);

}  // namespace bsrht
