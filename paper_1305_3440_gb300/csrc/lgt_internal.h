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
  double2 *warp_part;       // [2][nt][wps] per 8-site group (Re tr K, tr Delta^2) of each parity's last half-sweep
  int wps;                  // group slots per timeslice (stride of warp_part)
  double *fused_slice;      // [nt][2] per-slice fused sums (parity-0 Re tr K, both parities' tr Delta^2)
  unsigned *fused_counter;  // [1]
  double *fused_totals;     // [TOT_N] fused estimate, layout of totals
  double *meas_partial;     // [nt][2][gx_max][MEAS_NV]
  unsigned *meas_counter;   // [nt]
  unsigned *glob_counter;   // [1]
  double *slice_sum;        // [nt][MEAS_NV]
  double *slice_F;          // [nt]
  double *slice_theta;      // [nt]
  double *totals;           // [TOT_N]
  uint8_t *active;          // [nt]
  int *err;                 // [1] bit 0: ingest check failed, bit 1: a streaming sweep's wait timed out
  unsigned *stream_ctr;     // [2 + nt] streaming sweeps: ticket, abort flag, tiles done per slice
  unsigned *stream_order;   // [LGT_STREAM_MAX_HALF * nt] rolling-band order of configuration 12 (h << 16 | k)
};

size_t workspace_bytes(const Geom &g, int min_block);
void workspace_carve(void *base, const Geom &g, int min_block, Workspace *w);

// Arguments of one lattice's half-sweep (also one row of a batched launch).
// Ladder rules shared by lgt_fix, its device loop and the server.
// The bulk phase also ends when the estimate stops improving for
// LGT_STALL_CHECKS checks in a row -- the FP32 rounding floor -- but only
// counts such checks below LGT_STALL_CEILING: far above any FP32 floor the
// overrelaxed iteration's estimate may wander for a few checks without a
// floor being near (seen on Coulomb lattices, where theta is a max over
// slices), and promoting there would leave the polish a large transformation.
constexpr int LGT_STALL_CHECKS = 3;
constexpr double LGT_STALL_CEILING = 1e-8;
// The anchored polish forms its field and re-anchors after this many sweeps
// without a measurement: the FP32 correction C ~ |D| 2^-24 must stay small
// against the violations being removed, so D is not left to grow.
constexpr int LGT_REANCHOR_SWEEPS = 500;

// State of a device-side sweep loop (lgt_fix's chunks of check_every sweeps run
// as a CUDA graph with a conditional while node): the decide kernel updates it
// after each chunk's fused estimate, the sweep kernels read the sweep counters.
struct LoopState {
  unsigned long long sweep;  // number of the next sweep (RNG counter)
  long long count;           // sweeps of this phase so far (reunitarisation schedule)
  long long remaining;       // sweeps the caller still allows
  long long site_updates;    // site updates done by the loop
  double target;             // theta_switch (bulk) or theta_tol (polish)
  double best;               // bulk: smallest estimate so far
  double theta;              // last estimate
  int stall;                 // bulk: checks without improvement
  int bulk;                  // 1: bulk rules (target, stall), 0: polish rules (target)
  int active;                // slices the next sweeps update
  int iters, max_iters;      // chunks run by this launch, and their cap
  // omega schedule: the sweeps' OR parameter (read by the sweep kernels), and,
  // while omega_switch is set, the check that moves it to omega_late once the
  // estimate drops below theta_omega
  double omega, omega_late, theta_omega;
  int omega_switch;
};

struct SweepArgs {
  Geom g;
  void *links;
  void *G;
  const void *aux;  // anchored polish: K0
  // device loop: sweep = loop->sweep + sweep, omega = loop->omega, reunitarise when
  // (loop->count + sweep + 1) % reunit_every == 0 (sweep holds the offset in the chunk)
  const LoopState *loop;

  const uint8_t *active;
  double2 *warp_part;  // [2][nt][wps]
  int wps;
  double omega;
  unsigned long long sr_thr;
  unsigned long long seed;
  unsigned long long sweep;
  double beta;  // ALGO_SA
  int transform_temporal;
  int reunit;
  // batched launches only: reunitarise when (count_base + s + 1) % reunit_every == 0
  int reunit_every;
  long long count_base;
  // streaming launches (one kernel for n_half half-sweeps): their counters and error word
  unsigned *stream;
  int *err;
  int n_half;
  int stream_tiles;  // tiles (of blockDim.x sites) per scheduled item
  // snake order: a half-sweep of parity 1 visits the (slice, tile) list from
  // its end, so it starts on the links the parity-0 half-sweep touched last
  int snake;
  // streaming launches: the bound on one wait, and the first ticket (0 in a
  // normal run; > 0 leaves the first items of the launch undone, which makes the
  // bounded waits expire: fault injection for tests)
  unsigned long long stream_wait_ns;
  unsigned stream_skip;
  // streaming launches: the (half-sweep h, position k) pair of each scheduled
  // slice in ticket order (h << 16 | k; nullptr: half-sweep after half-sweep),
  // and the start slice of half-sweep h, h * stream_shift mod nt
  const unsigned *stream_order;
  int stream_shift;
  // global timeslice of local slice 0 (a temporal slab's offset): the random
  // streams of stochastic relaxation and annealing are counted by the global site
  int t_offset;
  // the slices the launch covers: t_first .. t_first + t_count - 1 (all by default)
  int t_first, t_count;
};

// Arguments of one lattice's exact measurement.
struct MeasArgs {
  Geom g;
  const void *links;
  double *partial;      // [nt][2][gridDim.x][MEAS_NV]
  unsigned *counter;    // [nt]
  unsigned *glob;       // [1]
  double *slice_sum;    // [nt][MEAS_NV]
  double *slice_F;      // [nt]
  double *slice_theta;  // [nt]
  double *totals;       // [TOT_N]
  uint8_t *active;      // [nt]
  double coulomb_target;
  int with_plaq;
  int mag;  // maximally Abelian gauge: slot 0 sums |U_aa|^2, slot 2 tr Delta_MAG^2
};

// Arguments of the fused estimate's finishing reduction (one block per slice).
struct FusedArgs {
  Geom g;
  const double2 *warp_part;
  int wps;
  int nw;  // warps per slice that wrote in the last half-sweeps
  int gauge;
  double *slice;
  unsigned *counter;
  double *totals;
  uint8_t *active;
  double coulomb_target;
};

// One row of a batched launch: a lattice's arguments and its block range.
struct BatchSweep {
  SweepArgs a;
  int block_begin;  // first block of this lattice in the batched grid
  int nbx;          // blocks per timeslice
};
struct BatchMeas {
  MeasArgs a;
  int block_begin;
  int nbx;
};
struct BatchFused {
  FusedArgs a;
  int block_begin;  // one block per timeslice
  int nbx;          // unused
};

struct SweepCfg {
  int gauge;                 // GAUGE_*
  int algo;                  // ALGO_*
  double omega;
  unsigned long long sr_thr;
  unsigned long long seed;
  int transform_temporal;
  double beta = 0.0;         // ALGO_SA: inverse temperature of the sweep
  // streaming launches: wait bound (0: LGT_STREAM_WAIT_NS) and first ticket (see SweepArgs)
  unsigned long long stream_wait_ns = 0;
  unsigned stream_skip = 0;
  int t_offset = 0;  // temporal slab: global slice of local slice 0
  int t_first = 0, t_count = 0;  // slices a launch covers (t_count 0: all)
};

// Single-lattice half-sweep kernels, one per (format, gauge, algorithm,
// launch configuration).  A launch configuration is a block size with a
// register budget (__launch_bounds__(threads, min blocks per SM)), i.e. an
// occupancy/spill trade-off, and a site layout; the autotuner times them.
//   one thread per site (every format):
//     0: 128 threads, <= 255 registers     1: 128 threads, <= 170 registers
//     2: 256 threads, <= 255 registers     3:  64 threads, <= 128 registers
//   four threads per site, one per direction (FP32 formats only):
//     4: 128 threads (32 sites), <= 128 registers
//     5: 256 threads (64 sites), <= 128 registers
//     6: 128 threads (32 sites), <= 80 registers
//   one thread per site, pipelined (FP32-12 only): persistent blocks, the next
//   site's links and G staged in shared memory by cp.async during the update:
//     7: 128 threads, <= 255 registers, 2 blocks per SM (108 KB shared each)
//   one thread per site, lean (FP32 formats): K(x) streamed, links loaded again
//   for the write-back:
//     8: 128 threads, <= 128 registers     9: 128 threads, <= 96 registers
//   one thread per site, streaming (FP32-12 only): one persistent launch runs
//   several half-sweeps; its blocks take (half-sweep, slice, tile) items in
//   order from a ticket counter and start an item as soon as the previous
//   half-sweep has finished the item's slice and its two neighbours, so the
//   pipeline does not drain between half-sweeps; staging as configuration 7:
//    10: 128 threads, <= 255 registers, 2 blocks per SM (108 KB shared each)
//   one thread per site, lean as 8 and 9, more warps per SM:
//    11: 128 threads, <= 80 registers (6 blocks, 24 warps per SM); also the
//        anchored polish's update at that budget (no spills)
//   one thread per site, streaming in a rolling band (FP32-12 only): as 10, but
//   the launch's half-sweeps overlap in time -- half-sweep h starts D waves
//   after h - 1, S slices further on -- so a few of them sweep the lattice
//   together a few slices apart and each link comes back to L2-resident lines:
//    12: 128 threads, <= 255 registers, 2 blocks per SM (108 KB shared each)
//   one thread per site, staged (FP32-12 only): the site's links and G copied
//   into shared memory by one batch of cp.async, then the lean body from there:
//    13: 128 threads, <= 128 registers, 4 blocks per SM (54 KB shared each)
//    14:  64 threads, <= 128 registers, 8 blocks per SM (27 KB shared each)
//    15:  64 threads, <= 112 registers, 9 blocks per SM: the links only in
//         shared memory (24 KB), G loaded into registers beside the copies
// The one-thread and four-thread layouts form K(x) in the same order, the lean
// ones link by link; every configuration groups the fused estimate by the same
// 8 sites; results differ only in FP32 rounding (the order of K's sums and
// where the compiler fuses multiply-adds).  The maximally Abelian gauge has
// kernels in configurations 0-3, 13 and 14.
constexpr int LGT_NCFG = 16;
__host__ __device__ constexpr int lgt_cfg_threads(int c) { return (c == 2 || c == 5) ? 256 : ((c == 3 || c == 14 || c == 15) ? 64 : 128); }
__host__ __device__ constexpr int lgt_cfg_minblocks(int c) {
  return c == 1 ? 3
                : (c == 3 ? 8
                          : (c == 4 ? 4
                                    : (c == 5 ? 2
                                              : (c == 6 ? 6 : (c == 7 || c == 10 || c == 12 ? 2 : (c == 8 || c == 13 ? 4 : (c == 9 ? 5 : (c == 11 ? 6 : (c == 14 ? 8 : (c == 15 ? 9 : 1))))))))));
}
__host__ __device__ constexpr bool lgt_cfg_quad(int c) { return c >= 4 && c <= 6; }
__host__ __device__ constexpr bool lgt_cfg_pipe(int c) { return c == 7; }
__host__ __device__ constexpr bool lgt_cfg_lean(int c) { return c == 8 || c == 9 || c == 11; }
__host__ __device__ constexpr bool lgt_cfg_stream(int c) { return c == 10 || c == 12; }
__host__ __device__ constexpr bool lgt_cfg_band(int c) { return c == 12; }
__host__ __device__ constexpr bool lgt_cfg_staged(int c) { return c == 13 || c == 14 || c == 15; }
// 16-byte chunks a staged configuration keeps per thread: 8 links x 3, and G x 3 unless 15
__host__ __device__ constexpr int lgt_cfg_stage_chunks(int c) { return c == 15 ? 24 : 27; }
// sites covered by one block (per tile for the pipelined configuration)
__host__ __device__ constexpr int lgt_cfg_sites(int c) { return lgt_cfg_quad(c) ? lgt_cfg_threads(c) / 4 : lgt_cfg_threads(c); }
// whether a storage format has kernels for a configuration
__host__ __device__ constexpr bool lgt_cfg_supported(int fmt, int c) {
  return c >= 0 && c < LGT_NCFG &&
         (!(lgt_cfg_quad(c) || lgt_cfg_lean(c)) || fmt == FMT_F32_18 || fmt == FMT_F32_12 || (fmt == FMT_ANCHOR && c == 11)) &&
         (!(lgt_cfg_pipe(c) || lgt_cfg_stream(c) || lgt_cfg_staged(c)) || fmt == FMT_F32_12);
}
// the maximally Abelian gauge has kernels in the one-thread-per-site
// configurations 0-3 and, on FP32-12 links, the staged ones
__host__ __device__ constexpr bool lgt_cfg_mag(int c) { return (c >= 0 && c <= 3) || c == 13 || c == 14; }
// whether a (format, gauge) pair has kernels for a configuration
__host__ __device__ constexpr bool lgt_cfg_supported_gauge(int fmt, int gauge, int c) {
  return lgt_cfg_supported(fmt, c) &&
         (gauge != GAUGE_MAG || (lgt_cfg_mag(c) && (fmt == FMT_F64 || fmt == FMT_F32_18 || fmt == FMT_F32_12)));
}
// dynamic shared memory of the pipelined and streaming configurations: 2 buffers x 27 chunks x 16 B per thread
constexpr int LGT_PIPE_SMEM_PER_THREAD = 2 * 27 * 16;
// streaming configuration: half-sweeps per launch at most, the bound on one
// wait for a neighbouring slice (after it the launch gives up, sets bit 1 of
// the error word and ends), and the error bit
constexpr int LGT_STREAM_MAX_HALF = 64;
constexpr int LGT_STREAM_TILES = 8;  // tiles (of 128 sites) per scheduled item (LGT_STREAM_TILES in the environment)
constexpr unsigned long long LGT_STREAM_WAIT_NS = 2000000000ull;
// rolling band (configuration 12): half-sweeps active at once, the gap in
// slices between consecutive ones, and tiles per item (LGT_STREAM_BAND="B,G"
// and LGT_STREAM_BAND_TILES in the environment)
constexpr int LGT_BAND_ACTIVE = 4;
constexpr int LGT_BAND_GAP = 2;
constexpr int LGT_BAND_TILES = 2;

// Rolling-band order.  Half-sweep h of a launch of n_half visits position k
// (slice h * S + k mod nt) at wave D h + k; tickets go wave by wave and, within
// a wave, by increasing h.  Item (h + 1, k) needs half-sweep h at positions
// S + k - 1 .. S + k + 1 (mod nt), whose waves are at most D h + S + k + 1 <=
// D (h + 1) + k when 1 <= S <= D - 1 (equal only with S = D - 1, and then h + 1
// comes later in the wave): every item's dependencies hold smaller tickets.
// Returns the ticket slot of (h, k): the pairs of earlier waves, then those of
// the same wave with smaller h.
__host__ __device__ inline unsigned stream_band_rank(int h, int k, int nt, int n_half, int D) {
  const long long w = (long long)D * h + k;
  unsigned r = 0;
  for (int j = 0; j < n_half; j++) {
    const long long c = w - (long long)D * j;  // positions of half-sweep j before wave w
    r += (unsigned)(c < 0 ? 0 : (c > nt ? nt : c));
    if (j < h && c < nt) r++;  // half-sweep j < h is in wave w too (c > 0 here)
  }
  return r;
}
constexpr int LGT_ERR_STREAM_WAIT = 2;
// configuration for a requested block size (lgt_params.block_size)
inline int lgt_cfg_of_block(int block) { return block == 256 ? 2 : (block == 64 ? 3 : 0); }
// fused-estimate slots: one per 8 consecutive sites of a slice
constexpr int LGT_FUSED_GROUP = 8;
typedef void (*sweep_fn)(SweepArgs, int);
sweep_fn pick_sweep_f32(int fmt, int gauge, int algo, int cfg);  // FP32-18, FP32-12
sweep_fn pick_sweep_hi(int fmt, int gauge, int algo, int cfg);   // FP64, FP32-pair

// One half-sweep of parity p on a field of format fmt with launch
// configuration cfg.  G (nullable) is multiplied by g at every updated site.
// use_mask: skip inactive slices.
// loop / reunit_every: a device loop's sweep (SweepArgs.loop; sweep is then the
// offset within the chunk).
cudaError_t launch_half_sweep(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                              int parity, unsigned long long sweep, int reunit, int use_mask, int cfg,
                              cudaStream_t st, const void *aux = nullptr, const LoopState *loop = nullptr,
                              int reunit_every = 0);

// n_half consecutive half-sweeps, the first of parity p0: half-sweep h has
// parity (p0 + h) & 1 and belongs to sweep s = (p0 + h) / 2 of the run, whose
// number is sweep0 + s (with a device loop: loop->sweep + sweep0 + s) and which
// reunitarises when reunit_every > 0 and (count_base + s + 1) % reunit_every
// == 0 (with a device loop: loop->count + sweep0 + s + 1).  The streaming
// configuration runs them in launches of up to LGT_STREAM_MAX_HALF half-sweeps,
// the others one launch each.  *launches (nullable) receives the kernel launches.
cudaError_t launch_half_sweeps(int fmt, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                               int p0, int n_half, unsigned long long sweep0, long long count_base, int reunit_every,
                               int use_mask, int cfg, cudaStream_t st, const void *aux = nullptr,
                               const LoopState *loop = nullptr, int *launches = nullptr);

// Fused estimate of F and theta from the last two half-sweeps (each sweep
// kernel leaves per-warp sums of Re tr K and tr Delta^2 computed from the K it
// used, so theta is lagged by half a sweep).  Reduced in fixed order into
// w.fused_totals; if coulomb_target >= 0 the slice mask is set to
// (theta_t >= coulomb_target).  sweep_sites: sites per block of those sweeps.
cudaError_t launch_fused_finish(const Geom &g, const Workspace &w, int gauge, int sweep_sites, double coulomb_target,
                                cudaStream_t st);
void fill_fused_args(FusedArgs *a, const Geom &g, const Workspace &w, int gauge, int sweep_sites,
                     double coulomb_target);
cudaError_t launch_fused_finish_batch(const BatchFused *jobs, int n, int total_blocks, cudaStream_t st);

// Exact measurement of a field of format fmt (FP64 arithmetic) into
// w.totals / w.slice_F / w.slice_theta.  If coulomb_target >= 0 the slice
// mask is set to (theta_t >= coulomb_target).  with_plaq: also plaquettes.
cudaError_t launch_measure(int fmt, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                           double coulomb_target, int block, cudaStream_t st, int mag = 0);

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

// Temporal slabs: active[t] = (lo <= t < hi) for the nt slices.
cudaError_t launch_slice_mask(uint8_t *active, int nt, int lo, int hi, cudaStream_t st);
// n links of public AoS layout (18 doubles each) set to the unit matrix.
cudaError_t launch_fill_unit_aos(double *aos, long long n, cudaStream_t st);

// Every link of a field of format fmt set to the unit matrix.
cudaError_t launch_fill_unit(int fmt, const Geom &g, void *soa, cudaStream_t st);

// In-place conversion of an FP64 field to FP32-pair storage (to_pair = 1)
// or back (to_pair = 0).
// Device loop: one thread advances the LoopState after a chunk of k sweeps and
// sets the while node's condition (another chunk or not).
cudaError_t launch_loop_decide(LoopState *L, const double *fused_totals, int gauge, int k, int vs_half,
                               cudaGraphConditionalHandle h, cudaStream_t st);
// Anchored polish: G = 1 + D (pairs) applied in FP64 (as launch_apply_G).
cudaError_t launch_apply_D(const Geom &g, const void *D, const void *u64_in, void *u64_out, double *aos_out,
                           int skip_temporal, cudaStream_t st);
// Anchored polish set-up from the FP64 field u64: K0 (pairs), the FP32-12 copy
// in u32, D = 0.
cudaError_t launch_anchor_setup(const Geom &g, const void *u64, void *u32, void *K0, void *D, int gauge,
                                cudaStream_t st);
// bytes of K0 and of D (hi and lo arrays) for vh sites per parity
inline size_t k0_bytes(int vh) { return (size_t)vh * 2 * 144; }
inline size_t d_bytes(int vh) { return (size_t)vh * 2 * 96; }
cudaError_t launch_convert_pair(const Geom &g, void *u, int to_pair, cudaStream_t st);

// Batched half-sweep over n lattices of one kernel variant (fmt, gauge,
// algo): blocks [jobs[k].block_begin, jobs[k+1].block_begin) belong to
// lattice k; total_blocks in all.  s: sweep offset within the batch (SR
// counter and reunitarisation schedule: jobs[k].a.sweep + s, count_base + s).
cudaError_t launch_half_sweep_batch(int fmt, int gauge, int algo, const BatchSweep *jobs, int n, int total_blocks,
                                    int parity, int s, int block, cudaStream_t st);
// Batched exact measurement over n lattices of one storage format.
cudaError_t launch_measure_batch(int fmt, const BatchMeas *jobs, int n, int total_blocks, int block, cudaStream_t st);
// Fill the batch row of a lattice (pointers into its workspace).
void fill_sweep_args(SweepArgs *a, const Geom &g, void *links, void *G, const Workspace &w, const SweepCfg &c,
                     unsigned long long sweep, int reunit, int use_mask);
void fill_meas_args(MeasArgs *a, const Geom &g, const void *links, const Workspace &w, int with_plaq,
                    double coulomb_target);

}  // namespace lgt
