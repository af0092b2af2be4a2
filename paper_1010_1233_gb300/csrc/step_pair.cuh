// The FP32 D2Q9 site update for two sites at once with the packed FP32 instructions of
// sm_100-class GPUs (fma.rn.f32x2 and friends: one instruction, two lanes of FP32
// arithmetic).  A thread that owns two neighbouring sites (x, x + 1) runs density and
// velocity, the relaxation of the non-conserved moments (Eqs. 5, 9, 10), the noise of
// Eq. 8 and the back transform with half the instructions of two scalar updates: these
// are step_common.cuh's macro_site / relax_site / apply_site on the float2 lane type,
// whose explicitly rounded operations give the scalar update's results bit for bit
// (lane x of every float2 is the first site, lane y the second).
#pragma once
#include "step_common.cuh"

namespace flb {

__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }

template <bool SAMPLE>
__device__ __forceinline__ void relax_pair(const ReplicaDesc& d, const float2 (&g)[9], float2 sum, float2 ux, float2 uy,
                                           float2 (&D)[6], float2 (&fld)[kMaxFields]) {
  relax_site<float2, true, SAMPLE>(d, g, sum, ux, uy, D, fld);
}

template <bool GEN>
__device__ __forceinline__ void apply_pair(const ReplicaDesc& d, float2 (&g)[9], float2 sum, bool noisy,
                                           const float2 (&n)[6], const float2 (&sc)[6], const float2 (&Drel)[6]) {
  apply_site<float2, true, GEN>(d, g, sum, noisy, n, sc, Drel);
}

__device__ __forceinline__ void macro_pair(const float2 (&g)[9], float rho0, float2& sum, float2& ux, float2& uy) {
  macro_site<float2, true>(g, rho0, sum, ux, uy);
}

// Box-Muller (FP32, as box_muller) on word pairs of the two sites: (wa0, wb0) -> the
// first site's normals (n0.x, n1.x), (wa1, wb1) -> the second's.
__device__ __forceinline__ void box_muller_pair(uint32_t wa0, uint32_t wb0, uint32_t wa1, uint32_t wb1, float2& n0,
                                                float2& n1) {
  using A = Lane<float2>;
  const float2 ua = A::fma(p2(__uint2float_rn(wa0), __uint2float_rn(wa1)), A::splat(0x1p-32f), A::splat(0x1p-33f));
  const float2 l = A::mul(p2(lg2_approx(ua.x), lg2_approx(ua.y)), A::splat(kBmLn4));
  const float2 y = p2(fminf(l.x, -1e-30f), fminf(l.y, -1e-30f));
  const float2 nr = A::mul(y, p2(rsqrt_approx(-y.x), rsqrt_approx(-y.y)));
  const float2 th = A::fma(p2(__uint2float_rn(wb0), __uint2float_rn(wb1)), A::splat(kBmAngScale), A::splat(kBmAngShift));
  n0 = A::mul(nr, p2(cos_approx(th.x), cos_approx(th.y)));
  n1 = A::mul(nr, p2(sin_approx(th.x), sin_approx(th.y)));
}

// the six normals of each of the two sites from their Philox words (w0, w1: calls 0, 1)
__device__ __forceinline__ void normals_pair(const uint4& w0a, const uint4& w1a, const uint4& w0b, const uint4& w1b,
                                             float2 (&n)[6]) {
  box_muller_pair(w0a.x, w0a.y, w0b.x, w0b.y, n[0], n[1]);
  box_muller_pair(w0a.z, w0a.w, w0b.z, w0b.w, n[2], n[3]);
  box_muller_pair(w1a.x, w1a.y, w1b.x, w1b.y, n[4], n[5]);
}

}  // namespace flb
