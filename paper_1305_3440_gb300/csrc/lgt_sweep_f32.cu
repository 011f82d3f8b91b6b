// lgt_sweep_f32.cu -- FP32 bulk half-sweep kernels (FP32-18 and FP32-12 link
// storage), one instantiation per gauge, algorithm and launch configuration
// (one or four threads per site; pipelined or staged through shared memory;
// streaming several half-sweeps per launch); the maximally Abelian gauge in the
// one-thread-per-site configurations 0-3 and the staged ones (13, 14).
#include "lgt_sweep.cuh"

namespace lgt {

template <int FMT, int GAUGE, int ALGO, int CFG>
__global__ void __launch_bounds__(lgt_cfg_threads(CFG), lgt_cfg_minblocks(CFG)) k_sweep_f32(SweepArgs in, int p) {
  pdl_enter();
  if constexpr (lgt_cfg_stream(CFG)) {  // sweep numbers per item, from the loop state or the arguments
    if constexpr (FMT == FMT_F32_12)
      sweep_body_f32_stream<GAUGE, ALGO>(in, p, (in.g.vs_half + (int)blockDim.x - 1) / (int)blockDim.x);
    return;
  }
  const SweepArgs a = resolve_loop(in);
  if constexpr (lgt_cfg_pipe(CFG)) {
    if constexpr (FMT == FMT_F32_12 && GAUGE != GAUGE_MAG)
      sweep_body_f32_pipe<GAUGE, ALGO>(a, p, (a.g.vs_half + (int)blockDim.x - 1) / (int)blockDim.x);
    return;
  }
  int t, bx;
  sweep_block_tile(a, p, t, bx);
  if constexpr (lgt_cfg_staged(CFG)) {
    if constexpr (FMT == FMT_F32_12 && GAUGE == GAUGE_MAG) sweep_body_mag<FMT, float, ALGO, true>(a, p, t, bx);
    else if constexpr (FMT == FMT_F32_12) sweep_body_f32_staged<GAUGE, ALGO, lgt_cfg_stage_chunks(CFG) == 27>(a, p, t, bx);
    return;
  }
  if constexpr (GAUGE == GAUGE_MAG) {
    sweep_body_mag<FMT, float, ALGO>(a, p, t, bx);
  } else if constexpr (lgt_cfg_quad(CFG)) {
    sweep_body_f32_quad<FMT, GAUGE, ALGO>(a, p, t, bx);
  } else if constexpr (lgt_cfg_lean(CFG)) {
    sweep_body_f32_lean<FMT, GAUGE, ALGO>(a, p, t, bx);
  } else {
    sweep_body_f32<FMT, GAUGE, ALGO>(a, p, t, bx, gridDim.x);
  }
}

template <int CFG>
static sweep_fn pick_cfg(int fmt, int gauge, int algo) {
#define LGT_PICK(F, G, A) \
  if (fmt == F && gauge == G && algo == A) return k_sweep_f32<F, G, A, CFG>;
  if (!lgt_cfg_supported(fmt, CFG)) return nullptr;
  LGT_PICK(FMT_F32_18, GAUGE_LANDAU, ALGO_OR)
  LGT_PICK(FMT_F32_18, GAUGE_LANDAU, ALGO_SR)
  LGT_PICK(FMT_F32_18, GAUGE_COULOMB, ALGO_OR)
  LGT_PICK(FMT_F32_18, GAUGE_COULOMB, ALGO_SR)
  LGT_PICK(FMT_F32_12, GAUGE_LANDAU, ALGO_OR)
  LGT_PICK(FMT_F32_12, GAUGE_LANDAU, ALGO_SR)
  LGT_PICK(FMT_F32_12, GAUGE_COULOMB, ALGO_OR)
  LGT_PICK(FMT_F32_12, GAUGE_COULOMB, ALGO_SR)
  if constexpr (lgt_cfg_mag(CFG)) {  // maximally Abelian gauge: one thread per site, plain layouts
    LGT_PICK(FMT_F32_18, GAUGE_MAG, ALGO_OR)
    LGT_PICK(FMT_F32_18, GAUGE_MAG, ALGO_SR)
    LGT_PICK(FMT_F32_12, GAUGE_MAG, ALGO_OR)
    LGT_PICK(FMT_F32_12, GAUGE_MAG, ALGO_SR)
  }
  if constexpr (CFG == 0) {  // the annealing sweeps run in configuration 0 only
    LGT_PICK(FMT_F32_18, GAUGE_LANDAU, ALGO_SA)
    LGT_PICK(FMT_F32_18, GAUGE_COULOMB, ALGO_SA)
    LGT_PICK(FMT_F32_12, GAUGE_LANDAU, ALGO_SA)
    LGT_PICK(FMT_F32_12, GAUGE_COULOMB, ALGO_SA)
  }
#undef LGT_PICK
  return nullptr;
}

sweep_fn pick_sweep_f32(int fmt, int gauge, int algo, int cfg) {
  switch (cfg) {
    case 0: return pick_cfg<0>(fmt, gauge, algo);
    case 1: return pick_cfg<1>(fmt, gauge, algo);
    case 2: return pick_cfg<2>(fmt, gauge, algo);
    case 3: return pick_cfg<3>(fmt, gauge, algo);
    case 4: return pick_cfg<4>(fmt, gauge, algo);
    case 5: return pick_cfg<5>(fmt, gauge, algo);
    case 6: return pick_cfg<6>(fmt, gauge, algo);
    case 7: return pick_cfg<7>(fmt, gauge, algo);
    case 8: return pick_cfg<8>(fmt, gauge, algo);
    case 9: return pick_cfg<9>(fmt, gauge, algo);
    case 10: return pick_cfg<10>(fmt, gauge, algo);
    case 11: return pick_cfg<11>(fmt, gauge, algo);
    case 12: return pick_cfg<12>(fmt, gauge, algo);
    case 13: return pick_cfg<13>(fmt, gauge, algo);
    case 14: return pick_cfg<14>(fmt, gauge, algo);
    case 15: return pick_cfg<15>(fmt, gauge, algo);
  }
  return nullptr;
}

}  // namespace lgt
