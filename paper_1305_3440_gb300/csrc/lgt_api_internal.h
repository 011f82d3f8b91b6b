// lgt_api_internal.h -- helpers shared by the C ABI translation units.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/lgt.h"
#include "lgt_device.cuh"
#include "lgt_internal.h"

void lgt_set_error(const char *fmt, ...);
// true if the LGT_FAULT environment list names `what` (host-side fault injection)
bool lgt_fault_injected(const char *what);
lgt_status lgt_validate_params(const lgt_params *p);
lgt::Geom lgt_make_geom(const int32_t dims[4]);
// device bytes a context with these parameters allocates
size_t lgt_ctx_device_bytes(const lgt_params *p);
// Launch configuration of the half-sweep kernel of format fmt: the fastest of
// the compiled configurations, timed on `links` (overwritten with unit links)
// and cached per (format, gauge, algorithm, dims, GPU).
int lgt_tune_sweep(const lgt::Geom &g, int fmt, const lgt::SweepCfg &cfg, void *links, void *G,
                   const lgt::Workspace &ws, cudaStream_t st, cudaError_t *err, void *aux = nullptr);
