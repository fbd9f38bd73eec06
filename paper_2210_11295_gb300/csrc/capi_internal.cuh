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

// Element-type code of the sketch plan for opts: opts.dtype, or
// kDtypeF32AsF64 for FP32 data with precision BSRHT_PREC_F64; EUNSUP for
// that precision on 16-bit data, EINVAL for an unknown precision.
int plan_dtype(const bsrht_opts& o, int* dt);

// BSRHT_OK for calls without an FP64-arithmetic form on FP32 storage when
// opts asks for none (precision AUTO, or F64 on FP64 data).
int precision_auto_only(const bsrht_opts& o);

}  // namespace bsrht
