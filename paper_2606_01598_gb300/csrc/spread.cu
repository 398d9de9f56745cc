// Spread of charges and dipoles onto the mesh (Section 2.3.2, Eq. charge_dipole_assign).
//
// Owner-computes design: one CTA owns one brick of BX x BY x BZ mesh points of one frame and
// is the only writer of those points, so the mesh needs no zeroing and no global atomics.
// One launch covers every brick of every frame of one spline order. Each of the 128 threads
// owns one z-segment of ZS points of one (X, Y) column of the brick and keeps it in registers.
//
// The CTA (1) lists the few source bricks whose ions' stencils can reach it (ions are sorted by
// the brick of their first stencil point), one thread per source brick; (2) walks their ions
// 256 at a time and keeps, in order, those whose p^3 stencil overlaps the brick (ballot
// compaction); (3) stages per kept ion, two threads to an ion, what a visit needs in shared
// memory: for each brick column X the coefficient combinations times the x weights (the
// density at a point is a sum over the weight-derivative orders of x, y and z, and the x and
// coefficient factors of every term are folded per column), for each row Y the y weights,
// and for each z-segment the aligned window of the z weights its 8 points see (zeros where
// the stencil does not reach); (4) builds separable coverage bitmasks -- bit l of xmask[X] is
// set when staged ion l's stencil covers plane X, likewise for Y and for each z-segment -- so
// that each thread visits only the ions whose stencil touches its segment
// (xmask[X] & ymask[Y] & zmask[seg]), in staged order; a visit is two table reads, a few
// multiply-adds for the y combination, vector window reads and the 8-point updates; (5)
// writes its points once. Every sum runs in a fixed order, so the result is bitwise
// reproducible.
//
// Tangent mode (backward pass) spreads, in the same sweep, the tangent density
//   d rho = sum_i [dq_i + (dmu_i + q_i dr_i) . grad + (mu_i . grad)(dr_i . grad)] W(x_i - m)
// (gradients with respect to the source position), the directional derivative of rho_mesh
// along the cotangent direction.
//
// Quadrupole mode spreads rho of charges, dipoles and point quadrupoles Theta_i (the rank-2
// channel), sum_i [q_i + mu_i . grad + Theta_i : grad grad] W(x_i - m): the tangent mode's
// record layout with (q, mu, Theta) in place of (dq, d', mu (x) dr), written to rho.
#include "spread_impl.cuh"

namespace gbpme {

// default brick 8 x 8 x 16 (measured faster than 8 x 8 x 32 and 8 x 8 x 8 on the 32768-ion
// frame); the other shapes live in spread_shapes_*.cu
int launch_spread_8x8x16(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho,
                         const float* theta) {
  return launch_spread_shape<Shape<8, 8, 16>>(p, s, mode, mesh, keep_rho, theta);
}

void spread_brick_shape(int shape[3]) {
  shape[0] = 8;
  shape[1] = 8;
  shape[2] = 16;
}

bool spread_shape_supported(const int shape[3]) {
  for (int k = 0; k < kNumSpreadShapes; ++k)
    if (kSpreadShapes[k][0] == shape[0] && kSpreadShapes[k][1] == shape[1] && kSpreadShapes[k][2] == shape[2])
      return true;
  return false;
}

static int dispatch(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho, const float* theta) {
  const int* b = p->g.brick;
  if (b[0] == 8 && b[1] == 8 && b[2] == 16) return launch_spread_8x8x16(p, s, mode, mesh, keep_rho, theta);
  if (b[0] == 8 && b[1] == 8 && b[2] == 32) return launch_spread_8x8x32(p, s, mode, mesh, keep_rho, theta);
  if (b[0] == 16 && b[1] == 8 && b[2] == 16) return launch_spread_16x8x16(p, s, mode, mesh, keep_rho, theta);
  if (b[0] == 16 && b[1] == 16 && b[2] == 16) return launch_spread_16x16x16(p, s, mode, mesh, keep_rho, theta);
  if (b[0] == 4 && b[1] == 8 && b[2] == 16) return launch_spread_4x8x16(p, s, mode, mesh, keep_rho, theta);
  return set_error(p, PME_ERR_UNSUPPORTED, "brick shape not supported");
}

int launch_spread(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep_rho) {
  return dispatch(p, s, tangent ? 1 : 0, mesh, keep_rho, nullptr);
}

int launch_spread_quad(pme_plan_t p, cudaStream_t s, const float* theta, float* mesh) {
  return dispatch(p, s, 2, mesh, nullptr, theta);
}

int launch_spread_quad_tangent(pme_plan_t p, cudaStream_t s, const float* theta, float* mesh) {
  return dispatch(p, s, 3, mesh, nullptr, theta);
}

GBPME_BOUNDS_READER(bounds_hit_spread)

}  // namespace gbpme
