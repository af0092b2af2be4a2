// The D1Q3 step of one site, shared by the per-step kernel (lb_step.cu) and the fused
// multi-step kernel (lb_d1q3_fused.cu).
//
// D1Q3: v = (0, +1, -1), w = (2/3, 1/6, 1/6), moments 1, sqrt3 v, (3 v^2 - 1)/sqrt2 (the
// projection of the D2Q9 basis).  Pull streaming (Eq. 1) from src, relaxation of the one
// non-conserved moment M^2 towards its equilibrium (Eqs. 5, 10) plus the noise of Eq. 8
// (noise mode 2: with the local density), back transform into dst; src and dst hold the
// populations as [3][nx].  With SAMPLE the pre-collision fields (moment minus its
// reference, or u - u0) of the replica's slots go to fields[slot * nx + x].
#pragma once
#include "flb_internal.cuh"

namespace flb {

template <typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void d1q3_site(const ReplicaDesc& d, const R* __restrict__ src, R* __restrict__ dst,
                                          R* __restrict__ fields, int nx, int x, uint32_t step) {
  if (!FLB_INB(x >= 0 && x < nx, 111)) return;
  const R g0 = src[x];
  const R g1 = src[nx + (x == 0 ? nx - 1 : x - 1)];
  const R g2 = src[2 * nx + (x == nx - 1 ? 0 : x + 1)];
  const R sum = g0 + (g1 + g2);
  const R rho = DEV ? coef<R>(d, kCoRho0) + sum : sum;
  const R j = g1 - g2;
  const R u = j / rho;
  const R S2 = (R)1.4142135623730950488, IS2 = (R)0.70710678118654752440;
  const R M2 = S2 * (g1 + g2) - IS2 * g0;
  const R E2 = (R)3 * IS2 * rho * u * u;
  if constexpr (SAMPLE) {
    const R mom[3] = {sum, (R)1.7320508075688772935 * j, M2};
    for (int slot = 0; slot < (int)d.n_fields; ++slot) {
      if (!FLB_INB(slot < kMaxFields, 111)) break;
      const int fid = d.field_id[slot];
      const R val = fid < 3 ? mom[fid] - coef<R>(d, kCoMref + fid) : u - coef<R>(d, kCoU0x);
      fields[(int64_t)slot * nx + x] = val;
    }
  }
  R D2 = (E2 - M2) * coef<R>(d, kCoInvTau + 2);
  if (d.noise_mask) {
    const uint4 w = philox4x32_10((uint32_t)x, step, 0u, d.stream, d.seed_lo, d.seed_hi);
    R n0, n1;
    box_muller(w.x, w.y, n0, n1);
    if (d.noise_mode == 2) n0 *= sqrt(rho / coef<R>(d, kCoRho0));    // local density in Eq. 8
    D2 += coef<R>(d, kCoAmp + 2) * n0;
  }
  dst[x] = g0 - (R)(2.0 / 3.0) * IS2 * D2;
  const R side = (R)(1.0 / 6.0) * S2 * D2;
  dst[nx + x] = g1 + side;
  dst[2 * nx + x] = g2 + side;
}

}  // namespace flb
