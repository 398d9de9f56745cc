// Spread kernels of the 16 x 8 x 16 brick (one of the shapes the brick autotuner
// chooses among; the kernel is the template of spread_impl.cuh).
#include "spread_impl.cuh"

namespace gbpme {

int launch_spread_16x8x16(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho,
                          const float* theta) {
  return launch_spread_shape<Shape<16, 8, 16>>(p, s, mode, mesh, keep_rho, theta);
}

GBPME_BOUNDS_READER(bounds_hit_spread_16x8x16)

}  // namespace gbpme
