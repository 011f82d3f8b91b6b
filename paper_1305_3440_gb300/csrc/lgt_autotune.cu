// lgt_autotune.cu -- block-size choice for the sweep kernel.
#include "lgt_api_internal.h"

int lgt_autotuned_block(const lgt_params *p) {
  (void)p;
  return 128;
}
