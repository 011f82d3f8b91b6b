// lgt_sweep_hi.cu -- the higher-precision half-sweep kernels: FP64 (every
// operation in FP64), FP32-pair and anchored (the polishing sweeps), one
// instantiation per gauge, algorithm and launch configuration.
#include "lgt_sweep.cuh"

namespace lgt {

template <int GAUGE, int ALGO, int CFG>
__global__ void __launch_bounds__(lgt_cfg_threads(CFG), lgt_cfg_minblocks(CFG)) k_sweep_f64(SweepArgs in, int p) {
  pdl_enter();
  const SweepArgs a = resolve_loop(in);
  int t, bx;
  sweep_block_tile(a, p, t, bx);
  if constexpr (GAUGE == GAUGE_MAG) {
    sweep_body_mag<FMT_F64, double, ALGO>(a, p, t, bx);
  } else {
    sweep_body_f64<GAUGE, ALGO>(a, p, t, bx, gridDim.x);
  }
}

template <int GAUGE, int ALGO, int CFG>
__global__ void __launch_bounds__(lgt_cfg_threads(CFG), lgt_cfg_minblocks(CFG)) k_sweep_pair(SweepArgs in, int p) {
  pdl_enter();
  const SweepArgs a = resolve_loop(in);
  int t, bx;
  sweep_block_tile(a, p, t, bx);
  sweep_body_pair<GAUGE, ALGO>(a, p, t, bx, gridDim.x);
}

template <int GAUGE, int ALGO, int CFG>
__global__ void __launch_bounds__(lgt_cfg_threads(CFG), lgt_cfg_minblocks(CFG)) k_sweep_anchor(SweepArgs in, int p) {
  pdl_enter();
  const SweepArgs a = resolve_loop(in);
  int t, bx;
  sweep_block_tile(a, p, t, bx);
  sweep_body_anchor<GAUGE, ALGO>(a, p, t, bx, gridDim.x);
}

template <int CFG>
static sweep_fn pick_cfg(int fmt, int gauge, int algo) {
  if constexpr (CFG == 11) {  // 24 warps per SM at <= 80 registers: the anchored polish only
    if (fmt != FMT_ANCHOR || algo == ALGO_SA || gauge == GAUGE_MAG) return nullptr;
    if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_anchor<GAUGE_LANDAU, ALGO_SR, CFG> : k_sweep_anchor<GAUGE_LANDAU, ALGO_OR, CFG>;
    return algo == ALGO_SR ? k_sweep_anchor<GAUGE_COULOMB, ALGO_SR, CFG> : k_sweep_anchor<GAUGE_COULOMB, ALGO_OR, CFG>;
  }
  if (gauge == GAUGE_MAG) {  // maximally Abelian gauge: FP64 only here, configurations 0-3
    if constexpr (lgt_cfg_mag(CFG)) {
      if (fmt == FMT_F64 && algo == ALGO_OR) return k_sweep_f64<GAUGE_MAG, ALGO_OR, CFG>;
      if (fmt == FMT_F64 && algo == ALGO_SR) return k_sweep_f64<GAUGE_MAG, ALGO_SR, CFG>;
    }
    return nullptr;
  }
  if (fmt == FMT_F64) {
    if constexpr (CFG == 0) {  // the annealing sweeps run in configuration 0 only
      if (algo == ALGO_SA)
        return gauge == GAUGE_LANDAU ? k_sweep_f64<GAUGE_LANDAU, ALGO_SA, CFG> : k_sweep_f64<GAUGE_COULOMB, ALGO_SA, CFG>;
    }
    if (algo == ALGO_SA) return nullptr;
    if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_f64<GAUGE_LANDAU, ALGO_SR, CFG> : k_sweep_f64<GAUGE_LANDAU, ALGO_OR, CFG>;
    return algo == ALGO_SR ? k_sweep_f64<GAUGE_COULOMB, ALGO_SR, CFG> : k_sweep_f64<GAUGE_COULOMB, ALGO_OR, CFG>;
  }
  if (algo == ALGO_SA) return nullptr;
  if (fmt == FMT_PAIR) {
    if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_pair<GAUGE_LANDAU, ALGO_SR, CFG> : k_sweep_pair<GAUGE_LANDAU, ALGO_OR, CFG>;
    return algo == ALGO_SR ? k_sweep_pair<GAUGE_COULOMB, ALGO_SR, CFG> : k_sweep_pair<GAUGE_COULOMB, ALGO_OR, CFG>;
  }
  if (fmt == FMT_ANCHOR) {
    if (gauge == GAUGE_LANDAU) return algo == ALGO_SR ? k_sweep_anchor<GAUGE_LANDAU, ALGO_SR, CFG> : k_sweep_anchor<GAUGE_LANDAU, ALGO_OR, CFG>;
    return algo == ALGO_SR ? k_sweep_anchor<GAUGE_COULOMB, ALGO_SR, CFG> : k_sweep_anchor<GAUGE_COULOMB, ALGO_OR, CFG>;
  }
  return nullptr;
}

sweep_fn pick_sweep_hi(int fmt, int gauge, int algo, int cfg) {
  switch (cfg) {
    case 0: return pick_cfg<0>(fmt, gauge, algo);
    case 1: return pick_cfg<1>(fmt, gauge, algo);
    case 2: return pick_cfg<2>(fmt, gauge, algo);
    case 3: return pick_cfg<3>(fmt, gauge, algo);
    case 11: return pick_cfg<11>(fmt, gauge, algo);
  }
  return nullptr;
}

}  // namespace lgt
