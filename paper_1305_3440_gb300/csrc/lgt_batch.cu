// lgt_batch.cu -- batched launches: one grid covers the blocks of many
// lattices (a device job table; block b belongs to the last row whose
// block_begin <= b).  Every row runs the same bodies as the single-lattice
// kernels, so a lattice's arithmetic and reduction order do not depend on
// what else is in the batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lgt_measure.cuh"
#include "lgt_sweep.cuh"

namespace lgt {

// Block b of a batched grid belongs to the last row k with
// jobs[k].block_begin <= b (rows sorted by block_begin).
__device__ __forceinline__ int batch_row(const int *begins, int stride_bytes, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int beg = *reinterpret_cast<const int *>(reinterpret_cast<const char *>(begins) + (size_t)mid * stride_bytes);
    if (beg <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Snake order over the whole batched grid (as the single-lattice sweeps): a
// half-sweep of parity 1 visits the blocks from the last, so it starts on the
// lattices and slices the parity-0 half-sweep finished last.  Every row of a
// batch is filled with the same order setting.
__device__ __forceinline__ int batch_block(const BatchSweep *jobs, int p) {
  return (jobs[0].a.snake && (p & 1)) ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
}

template <int FMT, int GAUGE, int ALGO>
__global__ void __launch_bounds__(256) k_sweep_batch(const BatchSweep *jobs, int n, int p, int s) {
  const int b = batch_block(jobs, p);
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchSweep), n, b);
  const BatchSweep &J = jobs[k];
  SweepArgs a = J.a;
  a.sweep += (unsigned long long)s;
  a.reunit = a.reunit_every > 0 && ((a.count_base + s + 1) % a.reunit_every) == 0;
  const int local = b - J.block_begin;
  const int t = local / J.nbx;
  sweep_dispatch<FMT, GAUGE, ALGO>(a, p, t, local - t * J.nbx, J.nbx);
}

template <int FMT>
__global__ void __launch_bounds__(256) k_measure_batch(const BatchMeas *jobs, int n) {
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchMeas), n, blockIdx.x);
  const BatchMeas &J = jobs[k];
  const int local = blockIdx.x - J.block_begin;
  const int per_t = 2 * J.nbx;
  const int t = local / per_t;
  const int rem = local - t * per_t;
  const int p = rem / J.nbx;
  measure_body<FMT>(J.a, t, p, rem - p * J.nbx, J.nbx);
}

// FP32-18 bulk sweeps of the batch: the lean one-thread layout (K streamed,
// links reloaded for the write-back; <= 128 registers, 4 blocks of 128 threads
// per SM), as launch configuration 8 of the single-lattice kernels.
template <int FMT, int GAUGE, int ALGO>
__global__ void __launch_bounds__(128, 4) k_sweep_batch_lean(const BatchSweep *jobs, int n, int p, int s) {
  const int b = batch_block(jobs, p);
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchSweep), n, b);
  const BatchSweep &J = jobs[k];
  SweepArgs a = J.a;
  a.sweep += (unsigned long long)s;
  a.reunit = a.reunit_every > 0 && ((a.count_base + s + 1) % a.reunit_every) == 0;
  const int local = b - J.block_begin;
  const int t = local / J.nbx;
  sweep_body_f32_lean<FMT, GAUGE, ALGO>(a, p, t, local - t * J.nbx);
}

// FP32-12 bulk sweeps of the batch: the staged one-thread layout (each site's
// links and G copied into shared memory by one batch of cp.async, then the
// lean update from there; 4 blocks of 128 threads per SM), as launch
// configuration 13 of the single-lattice kernels.
template <int GAUGE, int ALGO>
__global__ void __launch_bounds__(128, 4) k_sweep_batch_staged(const BatchSweep *jobs, int n, int p, int s) {
  const int b = batch_block(jobs, p);
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchSweep), n, b);
  const BatchSweep &J = jobs[k];
  SweepArgs a = J.a;
  a.sweep += (unsigned long long)s;
  a.reunit = a.reunit_every > 0 && ((a.count_base + s + 1) % a.reunit_every) == 0;
  const int local = b - J.block_begin;
  const int t = local / J.nbx;
  sweep_body_f32_staged<GAUGE, ALGO>(a, p, t, local - t * J.nbx);
}

// Anchored polish sweeps of the batch at <= 80 registers (6 blocks of 128
// threads = 24 warps per SM, as launch configuration 11 of the single-lattice
// polish kernels): the update is issue-bound, so the extra warps pay.
template <int GAUGE, int ALGO>
__global__ void __launch_bounds__(128, 6) k_sweep_batch_anchor(const BatchSweep *jobs, int n, int p, int s) {
  const int b = batch_block(jobs, p);
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchSweep), n, b);
  const BatchSweep &J = jobs[k];
  SweepArgs a = J.a;
  a.sweep += (unsigned long long)s;
  a.reunit = a.reunit_every > 0 && ((a.count_base + s + 1) % a.reunit_every) == 0;
  const int local = b - J.block_begin;
  const int t = local / J.nbx;
  sweep_body_anchor<GAUGE, ALGO>(a, p, t, local - t * J.nbx, J.nbx);
}

typedef void (*batch_fn)(const BatchSweep *, int, int, int);

static batch_fn pick_batch_anchor(int gauge, int algo) {
  if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_batch_anchor<GAUGE_LANDAU, ALGO_SR> : k_sweep_batch_anchor<GAUGE_LANDAU, ALGO_OR>;
  return algo == ALGO_SR ? k_sweep_batch_anchor<GAUGE_COULOMB, ALGO_SR> : k_sweep_batch_anchor<GAUGE_COULOMB, ALGO_OR>;
}

// the staged kernel's shared memory (27 chunks of 16 B per thread), opted in once per kernel
static cudaError_t staged_smem(batch_fn fn, int block, int *smem) {
  *smem = LGT_PIPE_SMEM_PER_THREAD / 2 * block;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

static batch_fn pick_batch_staged(int gauge, int algo) {
  if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_batch_staged<GAUGE_LANDAU, ALGO_SR> : k_sweep_batch_staged<GAUGE_LANDAU, ALGO_OR>;
  return algo == ALGO_SR ? k_sweep_batch_staged<GAUGE_COULOMB, ALGO_SR> : k_sweep_batch_staged<GAUGE_COULOMB, ALGO_OR>;
}

template <int FMT>
static batch_fn pick_batch_lean(int gauge, int algo) {
  if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_batch_lean<FMT, GAUGE_LANDAU, ALGO_SR> : k_sweep_batch_lean<FMT, GAUGE_LANDAU, ALGO_OR>;
  return algo == ALGO_SR ? k_sweep_batch_lean<FMT, GAUGE_COULOMB, ALGO_SR> : k_sweep_batch_lean<FMT, GAUGE_COULOMB, ALGO_OR>;
}

template <int FMT>
static batch_fn pick_batch_fmt(int gauge, int algo) {
  if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_batch<FMT, GAUGE_LANDAU, ALGO_SR> : k_sweep_batch<FMT, GAUGE_LANDAU, ALGO_OR>;
  return algo == ALGO_SR ? k_sweep_batch<FMT, GAUGE_COULOMB, ALGO_SR> : k_sweep_batch<FMT, GAUGE_COULOMB, ALGO_OR>;
}

cudaError_t launch_half_sweep_batch(int fmt, int gauge, int algo, const BatchSweep *jobs, int n, int total_blocks,
                                    int parity, int s, int block, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  batch_fn fn = nullptr;
  int smem = 0;
  if (fmt == FMT_F64) fn = pick_batch_fmt<FMT_F64>(gauge, algo);
  else if (fmt == FMT_F32_18) fn = block == 128 ? pick_batch_lean<FMT_F32_18>(gauge, algo) : pick_batch_fmt<FMT_F32_18>(gauge, algo);
  else if (fmt == FMT_F32_12 && block == 128 && (gauge == GAUGE_LANDAU || gauge == GAUGE_COULOMB) &&
           (algo == ALGO_OR || algo == ALGO_SR)) {
    fn = pick_batch_staged(gauge, algo);
    cudaError_t e = staged_smem(fn, block, &smem);
    if (e != cudaSuccess) return e;
  }
  else if (fmt == FMT_F32_12) fn = block == 128 ? pick_batch_lean<FMT_F32_12>(gauge, algo) : pick_batch_fmt<FMT_F32_12>(gauge, algo);
  else if (fmt == FMT_PAIR) fn = pick_batch_fmt<FMT_PAIR>(gauge, algo);
  else if (fmt == FMT_ANCHOR && block == 128 && (gauge == GAUGE_LANDAU || gauge == GAUGE_COULOMB) &&
           (algo == ALGO_OR || algo == ALGO_SR))
    fn = pick_batch_anchor(gauge, algo);
  else if (fmt == FMT_ANCHOR) fn = pick_batch_fmt<FMT_ANCHOR>(gauge, algo);
  if (!fn) return cudaErrorInvalidValue;
  fn<<<total_blocks, block, smem, st>>>(jobs, n, parity & 1, s);
  return cudaGetLastError();
}

cudaError_t launch_measure_batch(int fmt, const BatchMeas *jobs, int n, int total_blocks, int block, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  if (fmt == FMT_F64) k_measure_batch<FMT_F64><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_F32_18) k_measure_batch<FMT_F32_18><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_F32_12) k_measure_batch<FMT_F32_12><<<total_blocks, block, 0, st>>>(jobs, n);
  else if (fmt == FMT_PAIR) k_measure_batch<FMT_PAIR><<<total_blocks, block, 0, st>>>(jobs, n);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_fused_finish_batch(const BatchFused *jobs, int n) {
  const int k = batch_row(&jobs[0].block_begin, (int)sizeof(BatchFused), n, blockIdx.x);
  fused_finish_body(jobs[k].a, blockIdx.x - jobs[k].block_begin);
}

cudaError_t launch_fused_finish_batch(const BatchFused *jobs, int n, int total_blocks, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  k_fused_finish_batch<<<total_blocks, 256, 0, st>>>(jobs, n);
  return cudaGetLastError();
}

}  // namespace lgt
