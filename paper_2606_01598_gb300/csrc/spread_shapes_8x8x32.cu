// Spread kernels of the 8 x 8 x 32 brick (one of the shapes the brick autotuner
// chooses among; the kernel is the template of spread_impl.cuh).
#include "spread_impl.cuh"

namespace gbpme {

int launch_spread_8x8x32(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho,
                         const float* theta) {
  return launch_spread_shape<Shape<8, 8, 32>>(p, s, mode, mesh, keep_rho, theta);
}

GBPME_BOUNDS_READER(bounds_hit_spread_8x8x32)

}  // namespace gbpme
