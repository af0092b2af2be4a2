// Pieces of the D2Q9 step shared by the step kernels (lb_step.cu, lb_step_tc.cu):
// pull streaming with vector loads and warp shuffles, density/momentum, the
// collision with noise in the Hermite moment basis, and the stores.
//
// Population order (Sec. 3): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
// 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
#pragma once
#include "flb_internal.cuh"

namespace flb {

// Per-site noise-scale network parameters, FP32 copies of the bfloat16 values.
struct MlpWeights {
  float W1[kMlpHidden * 3];
  float W2[kMlpHidden * kMlpHidden];
  float W3[kMlpOut * kMlpHidden];
  float b1[kMlpHidden], b2[kMlpHidden], b3[kMlpOut];
};

__device__ __forceinline__ int find_replica(const int64_t* vb_begin, int n_reps, int64_t vb) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {                       // last r with vb_begin[r] <= vb
    const int mid = (lo + hi + 1) >> 1;
    if (vb_begin[mid] <= vb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Deterministic block reduction of kNumSums sums: each block writes its partial sums
// (fixed site set, fixed shuffle tree) to partial[kNumSums * blockIdx.x + k]; k_finish_sums
// (lb_step.cu) adds the partials in block order.
constexpr int kNumSums = 4;
__device__ __forceinline__ void block_sums(double (&acc)[kNumSums], double* __restrict__ partial) {
  __shared__ double red[32][kNumSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < kNumSums; ++k) {
      double v = 0.0;
      for (int w = 0; w < nw; ++w) v += red[w][k];
      partial[kNumSums * blockIdx.x + k] = v;
    }
  }
}

template <typename R, int VEC> struct VecIO;
template <> struct VecIO<float, 1> {
  static __device__ __forceinline__ void ld(const float* p, float (&v)[1]) { v[0] = __ldg(p); }
  static __device__ __forceinline__ void st(float* p, const float (&v)[1]) { *p = v[0]; }
};
template <> struct VecIO<float, 2> {
  static __device__ __forceinline__ void ld(const float* p, float (&v)[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p)); v[0] = t.x; v[1] = t.y; }
  static __device__ __forceinline__ void st(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
};
template <> struct VecIO<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
  static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct VecIO<double, 1> {
  static __device__ __forceinline__ void ld(const double* p, double (&v)[1]) { v[0] = __ldg(p); }
  static __device__ __forceinline__ void st(double* p, const double (&v)[1]) { *p = v[0]; }
};
template <> struct VecIO<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&v)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p)); v[0] = t.x; v[1] = t.y; }
  static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]); }
};

// Where a thread's VEC sites are: row y, first column x0 = VEC * xq of its unit.
struct UnitPos {
  int y, xq, x0;
  bool active, left_in_warp, right_in_warp;
};

__device__ __forceinline__ UnitPos unit_position(const ReplicaDesc& d, int64_t vb, int64_t vb0, int tid, int nthreads,
                                                 int vec) {
  // per-replica unit counts stay below 2^31 (sites < 2^32, at least 2 sites per unit or
  // VEC = 1 on lattices of < 2^31 sites), so the index arithmetic is 32-bit
  const int n_units = (int)d.n_units, upr = d.units_per_row;
  const int lane = tid & 31;
  const int unit_raw = (int)(vb - vb0) * nthreads + tid;
  UnitPos u;
  u.active = unit_raw < n_units;
  const int unit = u.active ? unit_raw : n_units - 1;
  u.y = (int)(((uint64_t)(uint32_t)unit * d.upr_magic) >> d.upr_shift);
  u.xq = unit - u.y * upr;
  u.x0 = u.xq * vec;
  // do the neighbour lanes hold the adjacent unit of the same row?
  u.left_in_warp = lane > 0 && u.xq > 0;
  u.right_in_warp = lane < 31 && (u.xq + 1) < upr && (unit_raw + 1) < n_units;
  return u;
}

// Pull streaming f_i(x) = f*_i(x - v_i), periodic (Eq. 1), in two halves so that a
// kernel can issue the loads of its next sites early: pull_issue loads the thread's
// own VEC values of each population and, at warp and row edges, the one value past
// the edge; pull_finish takes the +-x neighbours from the adjacent lane by shuffle.
template <typename R, int VEC>
struct PullRaw {
  R v[9][VEC];
  R e[9];                       // the value past the edge (used for v_ix != 0 only)
};

__host__ __device__ constexpr int vel_x(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int vel_y(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }

template <typename R, int VEC>
__device__ __forceinline__ void pull_issue(const R* __restrict__ src, int64_t plane, int nx, int ny, const UnitPos& u,
                                           PullRaw<R, VEC>& raw) {
  const int x0 = u.x0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int ys = u.y - vel_y(i);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    const R* row = src + i * plane + (int64_t)ys * nx;
    VecIO<R, VEC>::ld(row + x0, raw.v[i]);
    raw.e[i] = (R)0;
    if (vel_x(i) == 1) {                          // needs x0 - 1
      if (!u.left_in_warp) raw.e[i] = __ldg(row + (x0 == 0 ? nx - 1 : x0 - 1));
    } else if (vel_x(i) == -1) {                  // needs x0 + VEC
      if (!u.right_in_warp) raw.e[i] = __ldg(row + (x0 + VEC == nx ? 0 : x0 + VEC));
    }
  }
}

// Every lane of the warp must call it (the shuffles are warp-wide).
template <typename R, int VEC>
__device__ __forceinline__ void pull_finish(const PullRaw<R, VEC>& raw, const UnitPos& u, R (&f)[9][VEC]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (vel_x(i) == 0) {
#pragma unroll
      for (int s = 0; s < VEC; ++s) f[i][s] = raw.v[i][s];
    } else if (vel_x(i) == 1) {
      const R left = __shfl_up_sync(0xffffffffu, raw.v[i][VEC - 1], 1);
      f[i][0] = u.left_in_warp ? left : raw.e[i];
#pragma unroll
      for (int s = 1; s < VEC; ++s) f[i][s] = raw.v[i][s - 1];
    } else {
      const R right = __shfl_down_sync(0xffffffffu, raw.v[i][0], 1);
#pragma unroll
      for (int s = 0; s < VEC - 1; ++s) f[i][s] = raw.v[i][s + 1];
      f[i][VEC - 1] = u.right_in_warp ? right : raw.e[i];
    }
  }
}

template <typename R, int VEC>
__device__ __forceinline__ void pull_d2q9(const R* __restrict__ src, int64_t plane, int nx, int ny, const UnitPos& u,
                                          R (&f)[9][VEC]) {
  PullRaw<R, VEC> raw;
  pull_issue<R, VEC>(src, plane, nx, ny, u, raw);
  pull_finish<R, VEC>(raw, u, f);
}

// Density (as the sum of the stored values) and velocity of one site (Sec. 2).  In
// deviation storage sum_i w_i rho0 = rho0 and sum_i w_i rho0 v_i = 0.
template <typename R, bool DEV>
__device__ __forceinline__ void macro_d2q9(const R (&g)[9], R rho0, R& sum, R& ux, R& uy) {
  sum = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
  const R jx = (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
  const R jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
  const R irho = (R)1 / (DEV ? rho0 + sum : sum);
  ux = jx * irho;
  uy = jy * irho;
}

// The six unit normals of a site (Philox counter: site, step, call 0/1, stream), in two
// parts so that a kernel can spread them over independent work: the counter-based words,
// then the Box-Muller transform of three word pairs.
__device__ __forceinline__ void philox_words_d2q9(const ReplicaDesc& d, uint32_t site, uint32_t step, uint4& w0,
                                                  uint4& w1) {
  w0 = philox4x32_10(site, step, 0u, d.stream, d.seed_lo, d.seed_hi);
  w1 = philox4x32_10(site, step, 1u, d.stream, d.seed_lo, d.seed_hi);
}

template <typename R>
__device__ __forceinline__ void normals_from_words(const uint4& w0, const uint4& w1, R (&n)[6]) {
  box_muller(w0.x, w0.y, n[0], n[1]);
  box_muller(w0.z, w0.w, n[2], n[3]);
  box_muller(w1.x, w1.y, n[4], n[5]);
}

template <typename R>
__device__ __forceinline__ void normals_d2q9(const ReplicaDesc& d, uint32_t site, uint32_t step, R (&n)[6]) {
  uint4 w0, w1;
  philox_words_d2q9(d, site, step, w0, w1);
  normals_from_words<R>(w0, w1, n);
}

// Collision of one site (Eqs. 5, 8, 10), in two parts.  collide_relax: the non-conserved
// moments M^3..M^8 of Eq. 9, relaxed towards the equilibrium moments of Eq. 10 at rates
// 1/tau^a: D[a - 3] = Delta M^a (and the sampled fields of the pre-collision state when
// SAMPLE).  collide_apply: add xi^a = s_a amp_a N^a (noise mode 2: amp_a with the local
// density rho in place of rho0; mode 1, correlated noise: xi^a = s_a sum_c R_ac N^c) and
// the back transform
// sum_a n_i^a (Delta M^a + xi^a) with n_i^a = w_i m_i^a, in place.
template <typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void collide_relax(const ReplicaDesc& d, const R (&g)[9], R sum, R ux, R uy, R (&D)[6],
                                              R (&fld)[kMaxFields]) {
  const R S3 = (R)1.7320508075688772935, S32 = (R)1.2247448713915890491, S6 = (R)2.4494897427831780982;
  const R g0 = g[0], g1 = g[1], g2 = g[2], g3 = g[3], g4 = g[4], g5 = g[5], g6 = g[6], g7 = g[7], g8 = g[8];
  const R rho = DEV ? coef<R>(d, kCoRho0) + sum : sum;
  // non-conserved moments of Eq. 9 (identical for f and f - w rho0)
  const R ax = g1 + g3, ay = g2 + g4, dg = (g5 + g7) + (g6 + g8);
  const R M3 = (R)1.5 * (ax - ay);
  const R M4 = (R)3 * ((g5 + g7) - (g6 + g8));
  const R M5 = (R)0.5 * (ax + ay) + (R)2 * dg - g0;
  const R M6 = S32 * (g3 - g1) + S6 * ((g5 - g7) + (g8 - g6));
  const R M7 = S32 * (g4 - g2) + S6 * ((g5 - g7) + (g6 - g8));
  const R M8 = (R)0.5 * g0 - (ax + ay) + (R)2 * dg;
  // equilibrium moments, Eq. 10
  const R ux2 = ux * ux, uy2 = uy * uy;
  const R E3 = (R)1.5 * rho * (ux2 - uy2);
  const R E4 = (R)3 * rho * ux * uy;
  const R E5 = (R)1.5 * rho * (ux2 + uy2);
  if constexpr (SAMPLE) {
    const R jx = ux * rho, jy = uy * rho;
    const R mom[9] = {sum, S3 * jx, S3 * jy, M3, M4, M5, M6, M7, M8};
#pragma unroll
    for (int a = 0; a < 9; ++a) fld[a] = mom[a] - coef<R>(d, kCoMref + a);
    fld[9] = ux - coef<R>(d, kCoU0x);
    fld[10] = uy - coef<R>(d, kCoU0y);
  }
  // relaxation (Eq. 5)
  D[0] = (E3 - M3) * coef<R>(d, kCoInvTau + 3);
  D[1] = (E4 - M4) * coef<R>(d, kCoInvTau + 4);
  D[2] = (E5 - M5) * coef<R>(d, kCoInvTau + 5);
  D[3] = -M6 * coef<R>(d, kCoInvTau + 6);
  D[4] = -M7 * coef<R>(d, kCoInvTau + 7);
  D[5] = -M8 * coef<R>(d, kCoInvTau + 8);
}

// GEN: the replica may use noise modes 1 and 2 (branch on d.noise_mode); without it only
// mode 0 is compiled (the common case keeps its registers and instruction count).
template <typename R, bool DEV, bool GEN>
__device__ __forceinline__ void collide_apply(const ReplicaDesc& d, R (&g)[9], R sum, bool noisy, const R (&n)[6],
                                              const R (&sc)[6], const R (&Drel)[6]) {
  const R S32 = (R)1.2247448713915890491, S6 = (R)2.4494897427831780982;
  R D3 = Drel[0], D4 = Drel[1], D5 = Drel[2], D6 = Drel[3], D7 = Drel[4], D8 = Drel[5];
  if (GEN && noisy && d.noise_mode == 1) {              // correlated noise xi = R N (Eqs. 6-7 at u0), scaled by s
    R z[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      R acc = coef<R>(d, kCoNoiseR + 6 * c) * n[0];
#pragma unroll
      for (int e = 1; e < 6; ++e) acc += coef<R>(d, kCoNoiseR + 6 * c + e) * n[e];
      z[c] = acc;
    }
    D3 += sc[0] * z[0];
    D4 += sc[1] * z[1];
    D5 += sc[2] * z[2];
    D6 += sc[3] * z[3];
    D7 += sc[4] * z[4];
    D8 += sc[5] * z[5];
  } else if (noisy) {                            // Eq. 8, scaled per moment by s
    R s0 = sc[0], s1 = sc[1], s2 = sc[2], s3 = sc[3], s4 = sc[4], s5 = sc[5];
    if (GEN && d.noise_mode == 2) {              // local density in Eq. 8: amp * sqrt(rho / rho0)
      const R rho0 = coef<R>(d, kCoRho0);
      const R fac = sqrt((DEV ? rho0 + sum : sum) / rho0);
      s0 *= fac; s1 *= fac; s2 *= fac; s3 *= fac; s4 *= fac; s5 *= fac;
    }
    D3 += s0 * coef<R>(d, kCoAmp + 3) * n[0];
    D4 += s1 * coef<R>(d, kCoAmp + 4) * n[1];
    D5 += s2 * coef<R>(d, kCoAmp + 5) * n[2];
    D6 += s3 * coef<R>(d, kCoAmp + 6) * n[3];
    D7 += s4 * coef<R>(d, kCoAmp + 7) * n[4];
    D8 += s5 * coef<R>(d, kCoAmp + 8) * n[5];
  }
  // back transform of the moment change, n_i^a = w_i m_i^a
  const R w1 = (R)1 / (R)9, w5 = (R)1 / (R)36;
  const R c0 = (R)(4.0 / 9.0) * ((R)0.5 * D8 - D5);
  const R ax5 = (R)0.5 * D5 - D8;                   // common to the axis populations
  const R hx = (R)1.5 * D3;
  const R p6 = S32 * D6, p7 = S32 * D7;
  const R dcom = (R)2 * (D5 + D8);                  // common to the diagonal populations
  const R q6 = S6 * D6, q7 = S6 * D7, q4 = (R)3 * D4;
  g[0] = g[0] + c0;
  g[1] = g[1] + w1 * (ax5 + hx - p6);
  g[3] = g[3] + w1 * (ax5 + hx + p6);
  g[2] = g[2] + w1 * (ax5 - hx - p7);
  g[4] = g[4] + w1 * (ax5 - hx + p7);
  g[5] = g[5] + w5 * (dcom + q4 + q6 + q7);
  g[6] = g[6] + w5 * (dcom - q4 - q6 + q7);
  g[7] = g[7] + w5 * (dcom + q4 - q6 - q7);
  g[8] = g[8] + w5 * (dcom - q4 + q6 - q7);
}

template <typename R, bool DEV, bool SAMPLE, bool GEN>
__device__ __forceinline__ void collide_d2q9(const ReplicaDesc& d, R (&g)[9], R sum, R ux, R uy, bool noisy,
                                             const R (&n)[6], const R (&sc)[6], R (&fld)[kMaxFields]) {
  R D[6];
  collide_relax<R, DEV, SAMPLE>(d, g, sum, ux, uy, D, fld);
  collide_apply<R, DEV, GEN>(d, g, sum, noisy, n, sc, D);
}

// Store the post-collision populations (and the sampled fields) of a thread's sites.
template <typename R, int VEC, bool SAMPLE>
__device__ __forceinline__ void store_d2q9(const ReplicaDesc& d, char* __restrict__ ws, R* __restrict__ dst,
                                           int64_t plane, const UnitPos& u, const R (&f)[9][VEC],
                                           const R (&fld)[kMaxFields][VEC]) {
  if (!u.active) return;
  const int64_t off = (int64_t)u.y * d.nx + u.x0;
#pragma unroll
  for (int i = 0; i < 9; ++i) VecIO<R, VEC>::st(dst + i * plane + off, f[i]);
  if constexpr (SAMPLE) {
    R* fields = reinterpret_cast<R*>(ws + d.off_fields);
    for (int slot = 0; slot < (int)d.n_fields; ++slot) {
      const int fid = d.field_id[slot];
      R v[VEC];
#pragma unroll
      for (int s = 0; s < VEC; ++s) {
        R val = fld[0][s];
#pragma unroll
        for (int a = 1; a < kMaxFields; ++a) val = (fid == a) ? fld[a][s] : val;
        v[s] = val;
      }
      VecIO<R, VEC>::st(fields + slot * plane + off, v);
    }
  }
}

}  // namespace flb
