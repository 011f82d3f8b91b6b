// lgt_api_internal.h -- helpers shared by the C ABI translation units.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/lgt.h"
#include "lgt_device.cuh"

void lgt_set_error(const char *fmt, ...);
lgt_status lgt_validate_params(const lgt_params *p);
lgt::Geom lgt_make_geom(const int32_t dims[4]);
// device bytes a context with these parameters allocates
size_t lgt_ctx_device_bytes(const lgt_params *p);
// threads per block of the sweep kernel for these parameters
int lgt_pick_block(const lgt_params *p);
int lgt_autotuned_block(const lgt_params *p);
