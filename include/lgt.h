/*
 * lgt.h -- C ABI of liblgt: SU(3) lattice gauge fixing (Landau gauge, and
 * Coulomb gauge one timeslice at a time) by checkerboard relaxation on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method is that of Schroeck & Vogt, "Gauge fixing in lattice QCD with
 * multi-GPUs" (Excited QCD 2013):
 *   - Sec. 2 defines the gauge functional F, the transformation
 *     U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger, the violation Delta(x) and the
 *     precision theta = 1/(N_c V) sum_x tr[Delta Delta^dagger];
 *   - Sec. 3 the relaxation: for all sites of one parity at once maximise
 *     Re tr[g(x) K(x)] with K(x) built from the 8 adjacent links, through the
 *     three SU(2) subgroups (Cabibbo-Marinari) and the closed-form SU(2)
 *     maximum g = K^dagger / sqrt(det K^dagger);
 *   - Sec. 3.1 overrelaxation (g -> g^omega to first order, omega in [1,2));
 *   - Sec. 3.2 stochastic relaxation (g -> g^2 with probability p);
 *   - Sec. 4 the driver: both parities in turn until theta reaches the
 *     requested precision.
 *
 * Conventions used by every call
 * ------------------------------
 * Lattice: dims = {N_t, N_3, N_2, N_1} (slowest to fastest), each even and
 *   >= 2, periodic.  Site index x1 + N1*(x2 + N2*(x3 + N3*t)).  Direction
 *   mu = 0 is t (the paper's U_0), mu = 1, 2, 3 are x1, x2, x3.  Parity of a
 *   site is (x1+x2+x3+t) mod 2; the even sites are updated first.
 * Links (public layout): complex128 interleaved (re, im), array-of-structs
 *   links[((site*4 + mu)*9 + 3*row + col)*2 + {0: re, 1: im}],
 *   i.e. a C array double[N_t][N_3][N_2][N_1][4][3][3][2].  Each link must be
 *   in SU(3) (checked on input to 1e-10).
 * A_mu(x) (left undefined by the paper) is the traceless part of
 *   (U_mu(x) - U_mu(x)^dagger) / (2i); theta is quoted in that normalisation.
 * Coulomb gauge: per timeslice t, spatial directions only (N_d = 3, V -> V_s);
 *   F_t and theta_t per slice; the result's F is the mean of F_t and its
 *   theta the maximum of theta_t.  By default g(x) is also applied to the
 *   temporal links so the output remains a gauge transform of the input.
 * Ownership: the library copies what it is given and never frees caller
 *   memory.  It owns all device state of a context until lgt_destroy.
 * Errors: every call returns an lgt_status; no exception crosses the ABI.
 *   lgt_last_error() returns a message for the calling thread's last error.
 *   Calls on one context are not thread-safe; a server is.
 * Streams: a context runs on the CUDA stream given at creation (NULL = the
 *   legacy default stream); every call that returns data synchronises it.
 */
#ifndef LGT_H
#define LGT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LGT_API __attribute__((visibility("default")))
#else
#define LGT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgt_ctx lgt_ctx;       /* one gauge-fixing job on one lattice */
typedef struct lgt_server lgt_server; /* continuous-batching job server */

typedef enum {
  LGT_OK = 0,
  LGT_EINVAL = 1,     /* bad argument (dims, params, non-SU(3) or non-finite input) */
  LGT_ENOMEM = 2,     /* device or host allocation failed / over budget */
  LGT_ECUDA = 3,      /* CUDA runtime error (message in lgt_last_error) */
  LGT_ENOTCONV = 4,   /* max_sweeps reached before theta < theta_tol (state kept) */
  LGT_EAGAIN = 5,     /* job still queued or running */
  LGT_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  LGT_EBUSY = 7,      /* resource in use */
  LGT_ECANCELLED = 8, /* job cancelled */
  LGT_ENOTFOUND = 9   /* unknown job id */
} lgt_status;

/* LGT_MAG: the maximally Abelian gauge, which the paper's abstract names
 * beside Landau and Coulomb gauge without giving its functional.  Reading:
 * F_MAG = 1/(N_c 4 V) sum_{x,mu} sum_a |U_mu(x)_aa|^2, maximised; theta_MAG =
 * 1/(N_c V) sum_x tr[Delta Delta^dagger], Delta the traceless part of
 * (X - X^dagger)/(2i), X(x) = sum_mu (U_mu(x) D_mu(x)^dagger -
 * D_mu(x-mu)^dagger U_mu(x-mu)), D = diagonal part (F_MAG is stationary iff
 * theta_MAG = 0).  The local update maximises the site's F_MAG over each SU(2)
 * subgroup in closed form (of the circle of maximisers, the element nearest
 * the identity), then overrelaxation or stochastic relaxation as for Landau
 * gauge.  lgt_result.F / theta and lgt_measure report F_MAG / theta_MAG.
 * Launch configurations 0-3, and 13-14 on FP32-12 links (others fall back to
 * 0); after promotion it
 * polishes in FP64 whatever `polish` says; no simulated annealing; not
 * served (lgt_submit: LGT_EINVAL). */
typedef enum { LGT_LANDAU = 0, LGT_COULOMB = 1, LGT_MAG = 2 } lgt_gauge;
typedef enum { LGT_OR = 0, LGT_SR = 1 } lgt_algo; /* Sec. 3.1 / Sec. 3.2 */
/* lgt_params.polish_algo: the relaxation of the sweeps after promotion */
typedef enum { LGT_POLISH_SAME = 0, LGT_POLISH_OR = 1 } lgt_polish_algo;
typedef enum {
  LGT_FP64 = 0,    /* all sweeps in FP64 */
  LGT_FP32_18 = 1, /* bulk sweeps on FP32 links (18 reals), then FP64 polish */
  LGT_FP32_12 = 2  /* bulk sweeps on FP32 links stored as rows 0,1 (12 reals) */
} lgt_prec;

/* Precision of the polishing sweeps that follow an FP32 bulk phase.
 * PAIR: links held as FP32 pairs (hi + lo, ~48-bit significand, converted
 *   in place from the promoted FP64 field); K(x) accumulated in pair
 *   arithmetic; the SU(2) rotation angles chosen in FP32; each rotation
 *   formed unitary to second order and applied to the links in pair
 *   arithmetic, so every update is a gauge transformation to ~2^-48.
 *   Runs on the FP32 pipe.
 * FP64: every operation in FP64.
 * ANCHOR: the promoted field U' (FP64) is kept fixed as an anchor and the
 *   sweeps relax the gauge transformation G = 1 + D alone: the local update
 *   at x sees K(x) = G(x) [K0(x) + C(x)], the K(x) of the same sweep on the
 *   transformed links G U' G^+ (Sec. 3), with the constant
 *   K0 = sum_mu U'_mu(x) + U'_mu(x-mu)^+ stored once as FP32 pairs and the
 *   small C = sum_mu U'_mu(x) D(x+mu)^+ + U'_mu(x-mu)^+ D(x-mu)^+ formed in
 *   FP32; rotation angles, SU(2) elements and delta = g - 1 in FP32 from the
 *   small quantities; D accumulated as FP32 pairs.  Only D is written (768
 *   bytes of compulsory traffic per site update against 2304 for PAIR).
 *   Measurements and output form G U' G^+ in FP64 with G orthonormalised in
 *   FP64 (an exact gauge transform); a measurement makes it the new anchor.
 * With bulk = LGT_FP64 every sweep uses the FP64 kernel. */
typedef enum { LGT_POLISH_PAIR = 0, LGT_POLISH_FP64 = 1, LGT_POLISH_ANCHOR = 2 } lgt_polish;

typedef struct {
  int32_t dims[4];            /* N_t, N_3, N_2, N_1 */
  int32_t gauge;              /* lgt_gauge */
  int32_t algo;               /* lgt_algo */
  int32_t bulk;               /* lgt_prec of the bulk sweeps */
  int32_t transform_temporal; /* Coulomb: also transform U_0 (default 1) */
  double omega;               /* overrelaxation parameter, [1, 2) (OR only) */
  double p;                   /* stochastic relaxation probability, [0, 1] (SR only) */
  uint64_t seed;              /* key of the SR random stream */
  uint64_t sweep_offset;      /* index of the first sweep (RNG counter; resume) */
  double theta_tol;           /* requested precision, e.g. 1e-14 */
  double theta_switch;        /* bulk FP32 -> FP64 switch threshold (ignored for FP64) */
  int32_t max_sweeps;         /* cap on sweeps of one lgt_fix call (all phases) */
  int32_t check_every;        /* exact theta check every k sweeps */
  int32_t reunit_every;       /* reunitarise FP32 links / G every n sweeps (0: never) */
  int32_t block_size;         /* threads per block of the sweep kernels, 64/128/256, one thread per
                                 site (0: autotuned over block sizes, register budgets and site
                                 layouts) */
  int32_t polish;             /* lgt_polish (FP64 phase after an FP32 bulk phase) */
  int32_t launch_config;      /* 0: as block_size says; k = 1..16: launch configuration k-1 of the
                                 sweep kernels (overrides block_size; see below) */
  double omega_polish;        /* OR parameter of the sweeps after promotion, [1, 2); 0: omega */
  int32_t sa_sweeps;          /* simulated-annealing sweeps lgt_fix runs first (0: none) */
  int32_t polish_algo;        /* relaxation after promotion: LGT_POLISH_SAME (0, default) keeps
                                 algo; LGT_POLISH_OR (1) switches a stochastic-relaxation job to
                                 overrelaxation at omega_polish (0: omega) once its field is
                                 promoted -- the ladder's last decade, where Sec. 3.2's squared
                                 steps converge slowly */
  double sa_beta0, sa_beta1;  /* inverse temperature of the first and the last annealing sweep,
                                 0 < sa_beta0 <= sa_beta1 (geometric in between) */
  double omega_late;          /* omega schedule (OR): the relaxation sweeps before promotion (all
                                 sweeps when bulk = LGT_FP64) run at omega until a check of theta
                                 (every check_every sweeps, on the sweeps' estimate) finds theta <
                                 theta_omega, and at omega_late from then on; [1, 2), 0: no
                                 schedule.  Sweeps after promotion run at omega_polish. */
  double theta_omega;         /* switch point of the omega schedule, >= 0 */
} lgt_params;

typedef struct {
  double F;             /* final F (Landau) or mean F_t (Coulomb), exact FP64 measurement */
  double theta;         /* final theta (Landau) or max theta_t (Coulomb) */
  double plaquette;     /* average plaquette Re tr U_P / 3 (gauge invariant) */
  double seconds;       /* wall time of the call */
  int64_t sweeps_bulk;  /* sweeps run in the bulk FP32 precision */
  int64_t sweeps_fp64;  /* sweeps run after promotion (FP64 or FP32-pair polish) */
  int32_t status;       /* lgt_status of the job */
  int32_t reserved;
} lgt_result;

/* Simulated annealing (Sec. 1 names it as a preconditioner that lowers the
 * chance of ending in a poor Gribov copy; its details are in a reference this
 * text lacks).  Read as sa_sweeps sweeps before the relaxation, each subgroup
 * element drawn from exp(beta Re tr[r M]) with respect to Haar measure (an
 * SU(2) heat bath, Kennedy-Pendleton draws from Philox streams keyed by seed),
 * beta rising geometrically from sa_beta0 to sa_beta1.  They run in the bulk
 * precision (launch configuration 0) and count as bulk sweeps; in FP32 every
 * annealing sweep reunitarises the links and G it writes, whatever
 * reunit_every says.  lgt_fix runs them once per loaded field.  Not served
 * (lgt_submit: LGT_EINVAL). */

/* Launch configurations of the sweep kernels (lgt_params.launch_config - 1):
 *   one thread per site:  0: 128 threads, <= 255 registers; 1: 128, <= 170;
 *                         2: 256, <= 255; 3: 64, <= 128;
 *   four threads per site (one per direction; FP32 bulk sweeps only):
 *                         4: 128 threads, <= 128 registers; 5: 256, <= 128;
 *                         6: 128, <= 80;
 *   one thread per site, pipelined (FP32-12 bulk sweeps only):
 *                         7: 128 threads, <= 255 registers, persistent blocks
 *                            (2 per SM) that stage the next site's links and G
 *                            in shared memory (cp.async) during the update;
 *   one thread per site, lean (FP32 bulk sweeps only): K(x) accumulated link by
 *   link, links loaded again for the write-back:
 *                         8: 128 threads, <= 128 registers; 9: 128, <= 96;
 *                        11: 128, <= 80 (24 warps per SM);
 *   one thread per site, streaming (FP32-12 bulk sweeps only):
 *                        10: as 7, but one launch runs up to 64 half-sweeps:
 *                            blocks take (half-sweep, slice, 8 tiles) items
 *                            in order from a counter and start an item once
 *                            the previous half-sweep has finished its slice
 *                            and both neighbours (bounded waits: a wait over
 *                            2 s fails the call with LGT_ETIMEOUT);
 *                        12: as 10, items of 2 tiles taken in a rolling band:
 *                            half-sweep h starts D = ceil(N_t / 4) slices of
 *                            work after h - 1, at a slice D - 2 further on,
 *                            so about four half-sweeps sweep the lattice
 *                            together two slices apart and a slice's links
 *                            return to the next half-sweep while L2 still
 *                            holds them (same bounded waits);
 *   one thread per site, staged (FP32-12 bulk sweeps only): one batch of
 *   cp.async copies brings the site's links and G into shared memory, then
 *   the lean configurations' update runs from there:
 *                        13: 128 threads, <= 128 registers (4 blocks per SM);
 *                        14: 64 threads, <= 128 registers (8 blocks per SM);
 *                        15: 64 threads, <= 112 registers (9 blocks per SM),
 *                            the links staged and G loaded into registers.
 * The anchored polish (the default after promotion) runs in 0-3 and in 11
 * (<= 80 registers, 24 warps per SM).  A configuration that a phase's kernel
 * lacks (4-15 after promotion, except 11 for the anchored polish; 7, 10 and
 * 12-15 on FP32-18 links; all but 0-3, 13 and 14 in the maximally Abelian
 * gauge) falls back to configuration 0 for that phase.  Every
 * configuration groups the fused estimate by the same 8 sites; results differ
 * only in FP32 rounding (the lean configurations sum K(x) link by link, the
 * others pairwise; and where the compiler fuses multiply-adds), converged F
 * within 1e-10. */

/* Fill *p with defaults: Landau, OR, omega 1.7, FP64, tol 1e-14,
 * theta_switch 1e-13, max_sweeps 10000, check_every 10, reunit_every 50,
 * transform_temporal 1, block_size 0, launch_config 0, polish LGT_POLISH_ANCHOR, omega_polish 1.3,
 * sa_sweeps 0, sa_beta0 1, sa_beta1 100, omega_late 0 (no omega schedule), theta_omega 0
 * (after promotion the residual is short-wavelength noise, which a smaller
 * omega removes fastest).  dims are zeroed.  Never fails for p != NULL. */
LGT_API lgt_status lgt_params_default(lgt_params *p);

/* Create a context for one lattice (Sec. 2 problem statement).
 * links: the field in the public layout above, either host memory
 *   (links_on_device = 0) or device memory of the current device
 *   (links_on_device = 1); copied, never retained.
 * cuda_stream: cudaStream_t to run on (NULL: default stream).
 * *out receives the context on LGT_OK, NULL otherwise.
 * Errors: LGT_EINVAL for odd/too-small dims, bad params, non-SU(3) or
 * non-finite links; LGT_ENOMEM when device memory is short; LGT_ECUDA. */
LGT_API lgt_status lgt_create(const lgt_params *params, const double *links, int links_on_device, void *cuda_stream,
                      lgt_ctx **out);

/* Run n full sweeps (even half then odd half, Sec. 3 and Sec. 4) in the
 * context's current phase (bulk precision until promoted, FP64 after), with no
 * convergence test.  Coulomb: every slice is updated.  n >= 0. */
LGT_API lgt_status lgt_sweep(lgt_ctx *ctx, int32_t n);

/* One half-sweep: every site of `parity` (0 even, 1 odd) gets its local
 * update (Sec. 3: all sites of one parity subset at once; Sec. 4: one parity
 * per kernel launch).  The SR counter is the current sweep number; it and the
 * sweep count advance after parity 1.  Coulomb: every slice is updated. */
LGT_API lgt_status lgt_half_sweep(lgt_ctx *ctx, int32_t parity);

/* Exact measurement of the current working field, FP64 arithmetic and
 * fixed-order FP64 sums (Sec. 2: F and theta; plus the average plaquette).
 * In the bulk phase the working field is the FP32 links (widened).
 * Any output pointer may be NULL. */
LGT_API lgt_status lgt_measure(lgt_ctx *ctx, double *F, double *theta, double *plaquette);

/* Per-timeslice F_t and theta_t of the current working field (Coulomb
 * normalisation: spatial directions, N_d = 3, V_s).  Host arrays of N_t. */
LGT_API lgt_status lgt_measure_slices(lgt_ctx *ctx, double *F_t, double *theta_t);

/* The sweeps' own estimate of F and theta (Sec. 4 checks the precision after
 * every few sweeps; here the sweep kernels form it from the K(x) every site
 * update already has in registers, and lgt_fix's checks read it).  After a
 * full sweep (parity 0, then parity 1) it describes that sweep:
 *   F from Re tr K(x) of the even sites before their update: every link
 *     counted once, so this is the F of the field the sweep started from;
 *   theta from tr[Delta Delta^dagger] of every site's K(x), Delta the
 *     traceless part of (K - K^dagger)/(2i) (the Sec. 2 violation at a site
 *     whose neighbours carry g = 1): the even sites on the field the sweep
 *     started from, the odd sites on the field after its even half (lagging
 *     the field by half a sweep).
 * Maximally Abelian gauge: F_MAG from sum_a |U_aa|^2 of the even sites' links
 * and theta_MAG from X(x), likewise.  Sums in FP64 (per site in the sweep's
 * precision).  F, theta: as lgt_measure reports them (Coulomb: mean F_t, max
 * theta_t).  F_t, theta_t (nullable): host arrays of N_t, per timeslice in the
 * Coulomb normalisation (Landau: the slice's share in that normalisation).
 * Slices masked off as converged report theta_t = 0.  Meaningless before the
 * first full sweep after lgt_create / lgt_load. */
LGT_API lgt_status lgt_estimate(lgt_ctx *ctx, double *F, double *theta, double *F_t, double *theta_t);

/* Gauge-fix to theta < theta_tol (Sec. 4 driver) through the precision
 * ladder: bulk FP32 sweeps until the exact working-field theta drops below
 * theta_switch, then promotion (the accumulated gauge transformation G,
 * reunitarised in FP64, applied to the retained FP64 input), then FP64
 * sweeps, checking the exact theta every check_every sweeps.  Coulomb: a
 * slice stops being updated once its theta_t is below the phase's target.
 * res (nullable) receives the outcome.  Returns LGT_OK when converged,
 * LGT_ENOTCONV after max_sweeps (state kept, may be continued). */
LGT_API lgt_status lgt_fix(lgt_ctx *ctx, lgt_result *res);

/* Leave the bulk phase now: G (reunitarised in FP64) is applied to the FP64
 * input, U <- G(x) U(x) G(x+mu)^dagger, and later sweeps run in FP64.
 * No-op in the FP64 phase. */
LGT_API lgt_status lgt_promote(lgt_ctx *ctx);

/* The current field in the public layout, FP64.  In the bulk phase this is
 * G U G^dagger of the FP64 input (the phase is not changed).  out: host
 * (out_on_device = 0) or device memory of V*4*9*2 doubles. */
LGT_API lgt_status lgt_get_links(lgt_ctx *ctx, double *out, int out_on_device);

/* The working links as stored (bulk phase: FP32 widened to FP64, 12-real
 * storage with its third row rebuilt; FP64 phase: as lgt_get_links). */
LGT_API lgt_status lgt_get_working_links(lgt_ctx *ctx, double *out, int out_on_device);

/* Sweeps run so far (bulk FP32; after promotion) and the phase: 0 bulk
 * FP32, 1 FP64 storage, 2 FP32-pair polish. */
LGT_API lgt_status lgt_get_progress(lgt_ctx *ctx, int64_t *sweeps_bulk, int64_t *sweeps_fp64, int32_t *phase);

/* Replace the context's field with new links (same dims and params) and
 * restart: bulk phase (or FP64 for LGT_FP64), G = 1, sweep counters zero,
 * RNG counter back to sweep_offset, every slice active.  Reuses the
 * context's device memory (host links are staged through a device buffer
 * allocated on first use and kept).  Errors as lgt_create. */
LGT_API lgt_status lgt_load(lgt_ctx *ctx, const double *links, int links_on_device);

typedef struct {
  double sweep_ms[2];        /* device time of the sweep kernels: [0] bulk FP32, [1] FP64 */
  int64_t sweep_launches[2]; /* half-sweeps run by the sweep kernels in each precision
                                (one per launch, except the streaming configuration's) */
  int64_t site_updates[2];   /* site updates done in each precision (converged Coulomb slices excluded) */
  int64_t launches;          /* every kernel launch of this context */
  double measure_ms;         /* device time of exact measurements */
  int64_t measure_launches;
  int32_t launch_config[2];  /* launch configuration of the bulk / polish sweep kernels
                                (the table above lgt_params_default) */
  int64_t loop_launches;     /* lgt_fix device loops: CUDA graph launches, each running
                                chunks of check_every sweeps and their checks on the
                                device until a check stops it */
  int64_t loop_chunks;       /* chunks those launches ran */
} lgt_stats;

/* Counters since creation (or the last lgt_load).  Sweep-kernel times come
 * from CUDA events recorded on the context's stream around each batch of
 * consecutive half-sweep launches (nothing else runs inside a batch). */
LGT_API lgt_status lgt_get_stats(lgt_ctx *ctx, lgt_stats *out);

/* ------------------------------------------------- temporal slabs (Sec. 5) */
/* The paper's multi-GPU method (Sec. 5): the lattice is cut along t into
 * slabs, one per device; in every half-sweep each slab needs the temporal links
 * U_0(t_min - 1) of the inactive parity from the slab before it, and the
 * update of its first slice changes them, so they go back.  A slab context
 * holds the owned slices and a halo for those links; a driver moves them
 * between slabs (the package's slab module: its steps follow the paper's
 * list, with the return transfer overlapped with the interior slices).
 *
 * lgt_slab_create: params->dims[0] = L, the slab's owned slices (even, >= 2);
 * they are the global slices t0 .. t0 + L - 1 of a lattice of nt_global
 * slices (t0 even, so a site's parity is that of the whole lattice).  links:
 * the owned slices in the public layout (L * N_3 * N_2 * N_1 sites), host or
 * device memory.  Landau or Coulomb gauge, OR or SR (random streams counted by
 * the global site, so slabs reproduce the whole lattice's sweeps bit for bit),
 * no annealing; the field stays in its bulk precision (no promotion).  The
 * context holds L + 2 slices: two halo slices, the second receiving
 * U_0(t_min - 1).  lgt_load takes owned slices as well; lgt_get_links and
 * lgt_get_working_links return the owned slices of the working field
 * (FP64-widened); lgt_estimate reports the owned slices (F_t, theta_t: L
 * entries; F, theta: their mean, Coulomb: max theta_t).  lgt_sweep,
 * lgt_half_sweep, lgt_measure, lgt_measure_slices, lgt_fix and lgt_promote
 * return LGT_EINVAL on a slab.  Errors as lgt_create. */
LGT_API lgt_status lgt_slab_create(const lgt_params *params, int32_t nt_global, int32_t t0, const double *links,
                                   int links_on_device, void *cuda_stream, lgt_ctx **out);

/* Half-sweep of `parity` (Sec. 3: all sites of one parity at once) over the
 * owned slices first .. first + count - 1 (0-based within the slab) of a slab.
 * Enqueued on the context's stream, not synchronised (lgt_slab_sync).  The
 * sweep counter (SR stream, reunitarisation schedule) advances after a parity-1
 * call that covers the last owned slice.  The links U_0(t_min - 1) must be in
 * the halo when the first owned slice is updated. */
LGT_API lgt_status lgt_slab_half_sweep(lgt_ctx *ctx, int32_t parity, int32_t first, int32_t count);

/* Bytes of one boundary transfer of a slab: the temporal links of one parity
 * of one slice in the working storage format (FP64: 144 B per link, FP32-18:
 * 72 B, FP32-12: 48 B). */
LGT_API lgt_status lgt_slab_boundary_bytes(lgt_ctx *ctx, size_t *bytes);

/* Copy the temporal links U_0 of `parity` on owned slice `slice` (-1: the
 * halo, U_0(t_min - 1)) between the slab and buf (device memory of
 * lgt_slab_boundary_bytes bytes): into the slab if into_slab != 0, out of it
 * otherwise.  Layout of buf: the storage chunks one after the other, each the
 * slice's sites of that parity in within-parity order.  Enqueued on the
 * context's stream, not synchronised. */
LGT_API lgt_status lgt_slab_boundary(lgt_ctx *ctx, int32_t slice, int32_t parity, void *buf, int32_t into_slab);

/* Synchronise the context's stream (and report a failure of what it ran). */
LGT_API lgt_status lgt_slab_sync(lgt_ctx *ctx);

/* Exact per-timeslice sums of the working field, FP64 (Sec. 2), in host
 * memory sums[N_t][5] (a slab: its L owned slices): sum over the slice's sites
 * of [0] sum_mu Re tr U_mu(x), [1] the same over mu = 1..3, [2] tr[Delta
 * Delta^dagger] (all four directions), [3] the same over mu = 1..3, [4] the six
 * plaquettes Re tr U_P.  F = sum [0] / (3 * 4 * V), theta = sum [2] / (3 V),
 * Coulomb F_t = [1] / (9 V_s), theta_t = [3] / (3 V_s).  On a slab, [2] needs
 * both parities of the halo current and [4] of the last owned slice reads
 * the slice after the slab (not held: invalid there). */
LGT_API lgt_status lgt_measure_slice_sums(lgt_ctx *ctx, double *sums);

/* Test support; the paper has no counterpart.  Fault injection for the bounded
 * waits of the streaming launch configuration (10), so that their error path
 * can be exercised on a GPU without any device fault.  Until the next
 * lgt_load, every streaming launch that lgt_sweep / lgt_half_sweep issue on
 * this context (lgt_fix's device loops are not affected) waits at most wait_ns
 * nanoseconds for a neighbouring slice (0: the built-in 2 s; larger values:
 * LGT_EINVAL) and takes its first work item at ticket skip_items instead of 0,
 * so the first skip_items items of its first half-sweep never run (0: none).
 * The slices those items cover then never become ready for the next
 * half-sweep: its items wait until the limit, a block raises the launch's
 * abort flag and the context's error word, every block ends, and the call
 * returns LGT_ETIMEOUT -- as does every later synchronisation of the context
 * until lgt_load clears the error.  The field is then invalid.  Every wait is
 * bounded and every block exits; a launch with fewer than two half-sweeps
 * never waits. */
LGT_API lgt_status lgt_inject_stream_stall(lgt_ctx *ctx, uint64_t wait_ns, uint32_t skip_items);

/* Release every resource of the context.  NULL is ignored. */
LGT_API void lgt_destroy(lgt_ctx *ctx);

/* Exact measurement that allocates nothing: F, theta and the average
 * plaquette (as lgt_measure) and the per-timeslice F_t, theta_t (as
 * lgt_measure_slices) of links given directly in the public layout in device
 * memory.  The paper has no counterpart; it exists for callers that cannot
 * allocate device memory -- an application that hands out every byte of HBM
 * through its own memory plan or pool, or code that must measure where no
 * allocation may happen -- and so cannot create a context.
 * links_device: V*4*9*2 doubles, device memory of the current device.
 * out_device: at least 8 + 2*N_t doubles of device memory, receiving
 *   [0] F, [1] theta, [2] plaquette, [3] mean F_t, [4] max theta_t,
 *   [5] mean theta_t, [6..7] 0, [8 .. 8+N_t) F_t, [8+N_t .. 8+2N_t) theta_t.
 * cuda_stream: stream to run on (NULL: default stream).  The call is
 *   asynchronous: synchronise the stream before reading out_device.
 * Scratch: one fixed array of about 700 KB in device memory, compiled into the
 *   library (every GPU that loads the library holds it until exit), which
 *   limits N_t to at most 1024 (larger N_t: LGT_EINVAL).  Every call shares
 *   it and it keeps the last call's contents; the call clears what must start
 *   at zero.  Calls that overlap on the GPU (on different streams or devices
 *   sharing nothing else) race on it on the same device: run them in order.
 * Set-up: the first call on a device looks up the device address of the
 *   scratch with that device current; make that first call before any
 *   stream capture.
 * Errors: LGT_EINVAL for NULL pointers, odd or too-small dims, N_t > 1024;
 *   LGT_ECUDA for launch or set-up failures.  Calls no allocator. */
LGT_API lgt_status lgt_measure_noalloc(const int32_t dims[4], const double *links_device, double *out_device,
                                       void *cuda_stream);

/* ---------------------------------------------------------------- serving */
/* A continuous-batching server: jobs are admitted while the device memory
 * they need fits hbm_budget_bytes, their lattices stay resident, and one
 * worker thread advances every live job through the sweep kernels, checking
 * each job's exact theta every check_every sweeps and retiring it when
 * converged (Sec. 4 driver, per job).  device: CUDA device ordinal.
 * One tick = up to check_every sweeps of every live job (one batched launch
 * per sweep, parity and kernel variant) plus one batched theta check.  A tick
 * whose launch shape repeats the previous tick's is captured once into a CUDA
 * graph and replayed for as long as the shape lasts (at most 16 shapes kept);
 * the environment variable LGT_SERVER_GRAPHS=0, read at creation, issues
 * every tick's launches directly instead.  Results do not depend on it. */
LGT_API lgt_status lgt_server_create(size_t hbm_budget_bytes, int device, lgt_server **out);

/* Queue a job; links (host, public layout) are copied before return.
 * *job_id receives its id.  LGT_EINVAL for bad params/links, LGT_ENOMEM when
 * the job alone exceeds the budget. */
LGT_API lgt_status lgt_submit(lgt_server *s, const lgt_params *params, const double *links, uint64_t *job_id);

/* Job state: LGT_EAGAIN while queued or running; otherwise the job's final
 * status, with *res filled and, if links_out != NULL, the fixed field written
 * there (host, public layout).  A finished job is released by this call. */
LGT_API lgt_status lgt_poll(lgt_server *s, uint64_t job_id, lgt_result *res, double *links_out);

/* Cancel a queued or running job (it finishes with LGT_ECANCELLED). */
LGT_API lgt_status lgt_cancel(lgt_server *s, uint64_t job_id);

/* Server counters: jobs done, jobs live, device bytes in use. */
LGT_API lgt_status lgt_server_stats(lgt_server *s, uint64_t *jobs_done, uint64_t *jobs_live, size_t *bytes_in_use);

/* Worker counters since creation: ticks run, ticks replayed from a captured
 * graph, graphs captured, and kernel launches the ticks issued (directly or
 * inside graphs).  Any pointer may be NULL. */
LGT_API lgt_status lgt_server_counters(lgt_server *s, uint64_t *ticks, uint64_t *graph_launches,
                                       uint64_t *graph_captures, uint64_t *kernel_launches);

/* Stop the worker (queued jobs are cancelled) and release everything. */
LGT_API void lgt_server_destroy(lgt_server *s);

/* Message of the calling thread's most recent error ("" if none). */
LGT_API const char *lgt_last_error(void);

/* Library version string. */
LGT_API const char *lgt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LGT_H */
