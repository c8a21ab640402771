// Equilibrium populations of one colour, shared by the initialisation
// kernels of the two-buffer context and of the in-place step.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Equilibrium of one colour: Eq. 18 with the high-order term coefficient 3
// (improved) or Eq. 6 (original).  phi_i^k of Eq. 13, c = 1.
__device__ __forceinline__ void equilibrium(float rho, float alpha, float ux,
                                            float uy, float uz, int improved,
                                            float* fe) {
  const float cs2 = 0.5f * (1.f - alpha);
  const float uu = ux * ux + uy * uy + uz * uz;
  const float ph[3] = {alpha, (1.f - alpha) * (1.0f / 12.0f),
                       (1.f - alpha) * (1.0f / 24.0f)};
  const float w[3] = {1.0f / 3.0f, 1.0f / 18.0f, 1.0f / 36.0f};
  const float hk = improved ? 3.f * (3.f * cs2 - 1.f) : 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const float eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
    const int s = shell(i);
    const float ee = (float)s;  // |e|^2 = 0, 1, 2
    float br = 3.f * eu + 4.5f * eu * eu - 1.5f * uu + hk * eu * (3.f * ee - 5.f);
    fe[i] = rho * (ph[s] + w[s] * br);
  }
}

}  // namespace lbm
