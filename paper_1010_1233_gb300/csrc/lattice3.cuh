// Tables of the three-dimensional lattices (D3Q15, D3Q19) shared by their kernels
// (lb_3d.cu) and the host (api.cu): velocities, weights and the rows of the moment basis
// orthonormal in the weighted norm of Eq. 4 (the Gram-Schmidt construction and the
// closed forms are described in lb_3d.cu).
#pragma once
#include "flb_internal.cuh"

namespace flb {

// velocity components of population i of the Q-velocity lattice: 2 bits per population,
// value + 1
template <int Q> __host__ __device__ constexpr int v3x(int i) {
  return (int)(((Q == 15 ? 0x20889549ull : 0x1548889549ull) >> (2 * i)) & 3u) - 1;
}
template <int Q> __host__ __device__ constexpr int v3y(int i) {
  return (int)(((Q == 15 ? 0x0a089495ull : 0x895609495ull) >> (2 * i)) & 3u) - 1;
}
template <int Q> __host__ __device__ constexpr int v3z(int i) {
  return (int)(((Q == 15 ? 0x08a08955ull : 0x20a0954955ull) >> (2 * i)) & 3u) - 1;
}
static_assert(v3x<15>(7) == 1 && v3y<15>(7) == 1 && v3z<15>(7) == 1, "corner (1,1,1)");
static_assert(v3x<15>(13) == -1 && v3y<15>(13) == 1 && v3z<15>(13) == 1, "corner (-1,1,1)");
static_assert(v3x<15>(6) == 0 && v3y<15>(6) == 0 && v3z<15>(6) == -1, "axis -z");
static_assert(v3x<19>(9) == 1 && v3y<19>(9) == -1 && v3z<19>(9) == 0, "edge (1,-1,0)");
static_assert(v3x<19>(14) == -1 && v3y<19>(14) == 0 && v3z<19>(14) == 1, "edge (-1,0,1)");
static_assert(v3x<19>(18) == 0 && v3y<19>(18) == -1 && v3z<19>(18) == 1, "edge (0,-1,1)");

template <int Q> __host__ __device__ constexpr double w3(int i) {
  return Q == 15 ? (i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0))
                 : (i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0));
}
// noise normals (non-conserved moments) and Philox calls of the step; calls of the thermal start
template <int Q> struct Lat3 {
  static constexpr int kNC = Q - 4, kCalls = (Q - 4 + 3) / 4, kThermalCalls = (Q + 3) / 4;
};

// m_i^a of the basis above at velocity (vx, vy, vz)
template <int Q>
__host__ __device__ inline double moment_row3(int a, int vx, int vy, int vz) {
  const double S2 = 1.4142135623730950488, S3 = 1.7320508075688772935, S6 = 2.4494897427831780982;
  const double v2 = vx * vx + vy * vy + vz * vz;
  switch (a) {
    case 0: return 1.0;
    case 1: return S3 * vx;
    case 2: return S3 * vy;
    case 3: return S3 * vz;
    case 4: return 1.5 * (vx * vx - vy * vy);
    case 5: return 0.5 * S3 * (vx * vx + vy * vy - 2.0 * vz * vz);
    case 6: return 3.0 * vx * vy;
    case 7: return 3.0 * vy * vz;
    case 8: return 3.0 * vz * vx;
    case 9: return 0.5 * S6 * (v2 - 1.0);
    default: break;
  }
  if (Q == 15) {
    switch (a) {
      case 10: return 0.25 * S6 * vx * (3.0 * v2 - 5.0);
      case 11: return 0.25 * S6 * vy * (3.0 * v2 - 5.0);
      case 12: return 0.25 * S6 * vz * (3.0 * v2 - 5.0);
      case 13: return 3.0 * vx * vy * vz;
      default: return 0.25 * S2 * (3.0 * v2 * v2 - 9.0 * v2 + 4.0);
    }
  }
  switch (a) {
    case 10: return 0.5 * S6 * vx * (3.0 * v2 - 5.0);
    case 11: return 0.5 * S6 * vy * (3.0 * v2 - 5.0);
    case 12: return 0.5 * S6 * vz * (3.0 * v2 - 5.0);
    case 13: return 1.5 * S2 * vx * (vy * vy - vz * vz);
    case 14: return 1.5 * S2 * vy * (vz * vz - vx * vx);
    case 15: return 1.5 * S2 * vz * (vx * vx - vy * vy);
    case 16: return 0.5 * S2 * (3.0 * v2 * v2 - 6.0 * v2 + 1.0);
    case 17: return 1.5 * (vx * vx - vy * vy) * (2.0 * v2 - 3.0);
    default: return 0.5 * S3 * (vx * vx + vy * vy - 2.0 * vz * vz) * (2.0 * v2 - 3.0);
  }
}

}  // namespace flb
