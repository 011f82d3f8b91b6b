// lgt_internal.h -- host-side launchers of the kernels (used by the C ABI layer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgt_device.cuh"

namespace lgt {

// Number of doubles each measurement block reduces:
//   0: sum_mu=0..3 Re tr U_mu(x)     1: sum_mu=1..3 Re tr U_mu(x)
//   2: tr Delta Delta^dag (4-D)      3: tr Delta_s Delta_s^dag (spatial)
//   4: sum of the six plaquettes Re tr U_P
constexpr int MEAS_NV = 5;

// totals[] written by the measurement kernel's final block
enum {
  TOT_F_LANDAU = 0,
  TOT_THETA_LANDAU = 1,
  TOT_PLAQ = 2,
  TOT_F_COULOMB = 3,
  TOT_THETA_COULOMB_MAX = 4,
  TOT_THETA_COULOMB_MEAN = 5,
  TOT_ACTIVE_SLICES = 6,
  TOT_N = 8
};

// Device workspace of one lattice (one allocation, carved up).
struct Workspace {
  double *sweep_partial;    // [nt][gx_max][2]
  unsigned *sweep_counter;  // [nt]
  double *fused;            // [2][nt][2]  Re tr K, tr Delta^2 per parity and slice
  double *meas_partial;     // [nt][2][gx_max][MEAS_NV]
  unsigned *meas_counter;   // [nt]
  unsigned *glob_counter;   // [1]
  double *slice_sum;        // [nt][MEAS_NV]
  double *slice_F;          // [nt]
  double *slice_theta;      // [nt]
  double *totals;           // [TOT_N]
  uint8_t *active;          // [nt]
  int *err;                 // [1]
};

size_t workspace_bytes(const Geom &g, int min_block);
void workspace_carve(void *base, const Geom &g, int min_block, Workspace *w);

struct SweepCfg {
  int gauge;                 // GAUGE_*
  int algo;                  // ALGO_*
  double omega;
  unsigned long long sr_thr;
  unsigned long long seed;
  int transform_temporal;
};

// One half-sweep of parity p on a field of format fmt.  G (nullable) is
// multiplied by g at every updated site.  use_mask: skip inactive slices.
cudaError_t launch_half_sweep(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                              int parity, unsigned long long sweep, int reunit, int use_mask, int block,
                              cudaStream_t st);

// Exact measurement of a field of format fmt (FP64 arithmetic) into
// w.totals / w.slice_F / w.slice_theta.  If coulomb_target >= 0 the slice
// mask is set to (theta_t >= coulomb_target).  with_plaq: also plaquettes.
cudaError_t launch_measure(int fmt, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                           double coulomb_target, int block, cudaStream_t st);

// AoS complex128 (device) -> SoA of format fmt, with SU(3) / finiteness check
// (err bit 1 set on failure).
cudaError_t launch_ingest(int fmt, const Geom &g, const double *aos, void *soa, int *err, cudaStream_t st);

// SoA of format fmt -> AoS complex128 (device)
cudaError_t launch_egress(int fmt, const Geom &g, const void *soa, double *aos, cudaStream_t st);

// G <- identity
cudaError_t launch_g_identity(const Geom &g, void *G, cudaStream_t st);

// U(x,mu) <- G(x) U(x,mu) G(x+mu)^dagger in FP64 with G reunitarised in FP64.
// Writes to u64_out (SoA FP64, may equal u64_in) or, if aos_out != NULL,
// to AoS.  skip_temporal: leave mu = 0 untouched.
cudaError_t launch_apply_G(const Geom &g, const void *G, const void *u64_in, void *u64_out, double *aos_out,
                           int skip_temporal, cudaStream_t st);

// In-place conversion of an FP64 field to FP32-pair storage (to_pair = 1)
// or back (to_pair = 0).
cudaError_t launch_convert_pair(const Geom &g, void *u, int to_pair, cudaStream_t st);

}  // namespace lgt
