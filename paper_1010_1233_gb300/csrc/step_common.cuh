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
    if (FLB_INB(ys >= 0 && ys < ny && x0 >= 0 && x0 + VEC <= nx, 101)) VecIO<R, VEC>::ld(row + x0, raw.v[i]);
#ifdef FLB_CHECK_BOUNDS
    else for (int s = 0; s < VEC; ++s) raw.v[i][s] = (R)0;
#endif
    raw.e[i] = (R)0;
    if (vel_x(i) == 1) {                          // needs x0 - 1
      const int xe = x0 == 0 ? nx - 1 : x0 - 1;
      if (!u.left_in_warp && FLB_INB(xe >= 0 && xe < nx, 102)) raw.e[i] = __ldg(row + xe);
    } else if (vel_x(i) == -1) {                  // needs x0 + VEC
      const int xe = x0 + VEC == nx ? 0 : x0 + VEC;
      if (!u.right_in_warp && FLB_INB(xe >= 0 && xe < nx, 102)) raw.e[i] = __ldg(row + xe);
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

// Explicitly rounded arithmetic on one "lane type": a float, a double, or a float2 that
// carries two sites in the packed FP32 instructions of sm_100-class GPUs (fma.rn.f32x2,
// add, mul).  The site update below is written once on these operations, so no
// multiply-add is left for the compiler to contract: every kernel, vector width and
// launch flavour computes bit-identical results, one site or two at a time.
template <typename T> struct Lane;
template <> struct Lane<float> {
  using S = float;
  static __device__ __forceinline__ float splat(float c) { return c; }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.f, a); }   // hardware reciprocal, 2 ulp
  static __device__ __forceinline__ float sqrt_ratio(float a, float b) { return sqrtf(a / b); }
};
template <> struct Lane<double> {
  using S = double;
  static __device__ __forceinline__ double splat(double c) { return c; }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ double sqrt_ratio(double a, double b) { return sqrt(a / b); }
};
// Packed operations as inline PTX with the rounding mode spelled out (.rn): an operation
// with an explicit rounding mode is never fused with another, so a product that feeds a
// sum stays rounded on its own, as in the scalar operations above.
__device__ __forceinline__ uint64_t f2bits(float2 a) {
  return (uint64_t)__float_as_uint(a.x) | ((uint64_t)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 bitsf2(uint64_t v) {
  return make_float2(__uint_as_float((uint32_t)v), __uint_as_float((uint32_t)(v >> 32)));
}
template <> struct Lane<float2> {
  using S = float;
  static __device__ __forceinline__ float2 splat(float c) { return make_float2(c, c); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bitsf2(d);
  }
  // a - b = fma(b, -1, a): one rounding, the same value as a scalar subtraction
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return fma(b, make_float2(-1.f, -1.f), a); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bitsf2(d);
  }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(f2bits(c)));
    return bitsf2(d);
  }
  static __device__ __forceinline__ float2 rcp(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
  static __device__ __forceinline__ float2 sqrt_ratio(float2 a, float2 b) {
    return make_float2(sqrtf(a.x / b.x), sqrtf(a.y / b.y));
  }
};

// Density (as the sum of the stored values) and velocity (Sec. 2).  In deviation storage
// sum_i w_i rho0 = rho0 and sum_i w_i rho0 v_i = 0.
template <typename T, bool DEV>
__device__ __forceinline__ void macro_site(const T (&g)[9], typename Lane<T>::S rho0, T& sum, T& ux, T& uy) {
  using A = Lane<T>;
  const T ax = A::add(g[1], g[3]), ay = A::add(g[2], g[4]);
  const T dg = A::add(A::add(g[5], g[7]), A::add(g[6], g[8]));
  sum = A::add(A::add(A::add(g[0], ax), ay), dg);
  const T d57 = A::sub(g[5], g[7]), d86 = A::sub(g[8], g[6]);
  const T jx = A::add(A::sub(g[1], g[3]), A::add(d57, d86));
  const T jy = A::add(A::sub(g[2], g[4]), A::sub(d57, d86));
  const T irho = A::rcp(DEV ? A::add(A::splat(rho0), sum) : sum);
  ux = A::mul(jx, irho);
  uy = A::mul(jy, irho);
}

template <typename R, bool DEV>
__device__ __forceinline__ void macro_d2q9(const R (&g)[9], R rho0, R& sum, R& ux, R& uy) {
  macro_site<R, DEV>(g, rho0, sum, ux, uy);
}

// The six unit normals of a site, in two parts so that a kernel can spread them over
// independent work: the counter-based words, then the Box-Muller transform of three word
// pairs.  Sites 2q and 2q + 1 (the same row: nx is even) share the Philox counter
// (q, step, call, stream): calls 0, 1, 2 give twelve words W0..W11, and site 2q + h takes
// W_{6h}..W_{6h+5}, whose pairs (W_{6h+2m}, W_{6h+2m+1}) give normals 2m, 2m + 1.
// philox_words_d2q9: one site (two calls); on return its six words are w0.x..w0.w, w1.x,
// w1.y in pair order.
__device__ __forceinline__ void philox_words_d2q9(const ReplicaDesc& d, uint32_t site, uint32_t step, uint4& w0,
                                                  uint4& w1) {
  const uint32_t q = site >> 1, h = site & 1u;
  const uint4 a = philox4x32_10_rk(q, step, h, d.stream, d.rkey);         // call h
  const uint4 b = philox4x32_10_rk(q, step, h + 1u, d.stream, d.rkey);    // call h + 1
  w0 = h ? make_uint4(a.z, a.w, b.x, b.y) : a;
  w1 = h ? make_uint4(b.z, b.w, 0u, 0u) : make_uint4(b.x, b.y, 0u, 0u);
}

// Both sites of a pair (site_even even): three calls; the words of each site as above.
__device__ __forceinline__ void philox_words_pair(const ReplicaDesc& d, uint32_t site_even, uint32_t step, uint4& w0a,
                                                  uint4& w1a, uint4& w0b, uint4& w1b) {
  const uint32_t q = site_even >> 1;
  const uint4 c0 = philox4x32_10_rk(q, step, 0u, d.stream, d.rkey);
  const uint4 c1 = philox4x32_10_rk(q, step, 1u, d.stream, d.rkey);
  const uint4 c2 = philox4x32_10_rk(q, step, 2u, d.stream, d.rkey);
  w0a = c0;
  w1a = make_uint4(c1.x, c1.y, 0u, 0u);
  w0b = make_uint4(c1.z, c1.w, c2.x, c2.y);
  w1b = make_uint4(c2.z, c2.w, 0u, 0u);
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

// Collision (Eqs. 5, 8, 10), in two parts.  relax_site: the non-conserved moments
// M^3..M^8 of Eq. 9, relaxed towards the equilibrium moments of Eq. 10 at rates 1/tau^a:
// D[a - 3] = Delta M^a (and the sampled fields of the pre-collision state when SAMPLE).
// apply_site: add xi^a = s_a amp_a N^a (noise mode 2: amp_a with the local density rho in
// place of rho0; mode 1, correlated noise: xi^a = s_a sum_c R_ac N^c) and the back
// transform sum_a n_i^a (Delta M^a + xi^a) with n_i^a = w_i m_i^a, in place.
//
// No rounded product feeds a sum here unless the product is exact (a power of two) or
// the sum is written as a fused multiply-add: a code generator that fuses a packed
// multiply into the following packed add would otherwise round differently from the
// scalar operations.
template <typename T, bool DEV, bool SAMPLE>
__device__ __forceinline__ void relax_site(const ReplicaDesc& d, const T (&g)[9], T sum, T ux, T uy, T (&D)[6],
                                           T (&fld)[kMaxFields]) {
  using A = Lane<T>;
  using S = typename Lane<T>::S;
  const S S3 = (S)1.7320508075688772935, S32 = (S)1.2247448713915890491, S6 = (S)2.4494897427831780982;
  const T rho = DEV ? A::add(A::splat(coef<S>(d, kCoRho0)), sum) : sum;
  // non-conserved moments of Eq. 9 (identical for f and f - w rho0)
  const T ax = A::add(g[1], g[3]), ay = A::add(g[2], g[4]);
  const T s57 = A::add(g[5], g[7]), s68 = A::add(g[6], g[8]);
  const T dg = A::add(s57, s68), axy = A::add(ax, ay), dg2 = A::mul(A::splat((S)2), dg);
  const T d57 = A::sub(g[5], g[7]), d86 = A::sub(g[8], g[6]);
  const T axmy = A::sub(ax, ay), s57m = A::sub(s57, s68);
  //   M3 = 3/2 axmy, M4 = 3 s57m; M5 and M8 with the exact 2 dg
  const T M5 = A::fma(A::splat((S)0.5), axy, A::sub(dg2, g[0]));
  const T M6 = A::fma(A::splat(S6), A::add(d57, d86), A::mul(A::splat(S32), A::sub(g[3], g[1])));
  const T M7 = A::fma(A::splat(S6), A::sub(d57, d86), A::mul(A::splat(S32), A::sub(g[4], g[2])));
  const T M8 = A::fma(A::splat((S)0.5), g[0], A::sub(dg2, axy));
  // equilibrium moments of Eq. 10 minus the moments: E3 - M3, E4 - M4, E5 - M5
  const T nuy = A::mul(uy, A::splat((S)-1));
  const T u2d = A::fma(ux, ux, A::mul(uy, nuy));           // u_x^2 - u_y^2
  const T u2s = A::fma(ux, ux, A::mul(uy, uy));            // u_x^2 + u_y^2
  const T r15 = A::mul(A::splat((S)1.5), rho);
  const T t3 = A::fma(r15, u2d, A::mul(A::splat((S)-1.5), axmy));
  const T t4 = A::fma(A::mul(A::splat((S)3), rho), A::mul(ux, uy), A::mul(A::splat((S)-3), s57m));
  const T nM5 = A::fma(A::splat((S)-0.5), axy, A::sub(g[0], dg2));   // -M5 exactly
  const T t5 = A::fma(r15, u2s, nM5);
  if constexpr (SAMPLE) {
    const T jx = A::add(A::sub(g[1], g[3]), A::add(d57, d86));
    const T jy = A::add(A::sub(g[2], g[4]), A::sub(d57, d86));
    const T irho = A::rcp(rho);
    fld[0] = A::sub(sum, A::splat(coef<S>(d, kCoMref + 0)));
    fld[1] = A::fma(A::splat(S3), jx, A::splat(-coef<S>(d, kCoMref + 1)));
    fld[2] = A::fma(A::splat(S3), jy, A::splat(-coef<S>(d, kCoMref + 2)));
    fld[3] = A::fma(A::splat((S)1.5), axmy, A::splat(-coef<S>(d, kCoMref + 3)));
    fld[4] = A::fma(A::splat((S)3), s57m, A::splat(-coef<S>(d, kCoMref + 4)));
    fld[5] = A::sub(M5, A::splat(coef<S>(d, kCoMref + 5)));
    fld[6] = A::sub(M6, A::splat(coef<S>(d, kCoMref + 6)));
    fld[7] = A::sub(M7, A::splat(coef<S>(d, kCoMref + 7)));
    fld[8] = A::sub(M8, A::splat(coef<S>(d, kCoMref + 8)));
    fld[9] = A::fma(jx, irho, A::splat(-coef<S>(d, kCoU0x)));      // u - u0
    fld[10] = A::fma(jy, irho, A::splat(-coef<S>(d, kCoU0y)));
  }
  // relaxation (Eq. 5)
  D[0] = A::mul(t3, A::splat(coef<S>(d, kCoInvTau + 3)));
  D[1] = A::mul(t4, A::splat(coef<S>(d, kCoInvTau + 4)));
  D[2] = A::mul(t5, A::splat(coef<S>(d, kCoInvTau + 5)));
  D[3] = A::mul(M6, A::splat(-coef<S>(d, kCoInvTau + 6)));
  D[4] = A::mul(M7, A::splat(-coef<S>(d, kCoInvTau + 7)));
  D[5] = A::mul(M8, A::splat(-coef<S>(d, kCoInvTau + 8)));
}

// GEN: the replica may use noise modes 1 and 2 (branch on d.noise_mode); without it only
// mode 0 is compiled (the common case keeps its registers and instruction count).
template <typename T, bool DEV, bool GEN>
__device__ __forceinline__ void apply_site(const ReplicaDesc& d, T (&g)[9], T sum, bool noisy, const T (&n)[6],
                                           const T (&sc)[6], const T (&Drel)[6]) {
  using A = Lane<T>;
  using S = typename Lane<T>::S;
  const S S32 = (S)1.2247448713915890491, S6 = (S)2.4494897427831780982;
  T D[6] = {Drel[0], Drel[1], Drel[2], Drel[3], Drel[4], Drel[5]};
  if (GEN && noisy && d.noise_mode == 1) {              // correlated noise xi = R N (Eqs. 6-7 at u0), scaled by s
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T z = A::mul(A::splat(coef<S>(d, kCoNoiseR + 6 * c)), n[0]);
#pragma unroll
      for (int e = 1; e < 6; ++e) z = A::fma(A::splat(coef<S>(d, kCoNoiseR + 6 * c + e)), n[e], z);
      D[c] = A::fma(sc[c], z, D[c]);
    }
  } else if (noisy) {                            // Eq. 8, scaled per moment by s
    T fac = A::splat((S)1);
    if (GEN && d.noise_mode == 2) {              // local density in Eq. 8: amp * sqrt(rho / rho0)
      const T rho0 = A::splat(coef<S>(d, kCoRho0));
      fac = A::sqrt_ratio(DEV ? A::add(rho0, sum) : sum, rho0);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      T s = A::mul(sc[c], A::splat(coef<S>(d, kCoAmp + 3 + c)));
      if (GEN && d.noise_mode == 2) s = A::mul(s, fac);
      D[c] = A::fma(s, n[c], D[c]);
    }
  }
  // back transform of the moment change, n_i^a = w_i m_i^a (D[a - 3] = Delta M^a + xi^a)
  const T w1 = A::splat((S)1 / (S)9), w5 = A::splat((S)1 / (S)36);
  const T ax5 = A::sub(A::mul(A::splat((S)0.5), D[2]), D[5]);   // common to the axis populations
  const T Ap = A::fma(A::splat((S)1.5), D[0], ax5), Bm = A::fma(A::splat((S)-1.5), D[0], ax5);
  const T dcom = A::mul(A::splat((S)2), A::add(D[2], D[5]));      // common to the diagonal populations
  const T P = A::fma(A::splat((S)3), D[1], dcom), Q = A::fma(A::splat((S)-3), D[1], dcom);
  const T Rp = A::fma(A::splat(S6), D[3], A::mul(A::splat(S6), D[4]));      // q6 + q7
  const T Rm = A::fma(A::splat(S6), D[3], A::mul(A::splat(-S6), D[4]));     // q6 - q7
  g[0] = A::fma(A::splat((S)(4.0 / 9.0)), A::sub(A::mul(A::splat((S)0.5), D[5]), D[2]), g[0]);
  g[1] = A::fma(w1, A::fma(A::splat(-S32), D[3], Ap), g[1]);
  g[3] = A::fma(w1, A::fma(A::splat(S32), D[3], Ap), g[3]);
  g[2] = A::fma(w1, A::fma(A::splat(-S32), D[4], Bm), g[2]);
  g[4] = A::fma(w1, A::fma(A::splat(S32), D[4], Bm), g[4]);
  g[5] = A::fma(w5, A::add(P, Rp), g[5]);
  g[6] = A::fma(w5, A::sub(Q, Rm), g[6]);
  g[7] = A::fma(w5, A::sub(P, Rp), g[7]);
  g[8] = A::fma(w5, A::add(Q, Rm), g[8]);
}

template <typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void collide_relax(const ReplicaDesc& d, const R (&g)[9], R sum, R ux, R uy, R (&D)[6],
                                              R (&fld)[kMaxFields]) {
  relax_site<R, DEV, SAMPLE>(d, g, sum, ux, uy, D, fld);
}

template <typename R, bool DEV, bool GEN>
__device__ __forceinline__ void collide_apply(const ReplicaDesc& d, R (&g)[9], R sum, bool noisy, const R (&n)[6],
                                              const R (&sc)[6], const R (&Drel)[6]) {
  apply_site<R, DEV, GEN>(d, g, sum, noisy, n, sc, Drel);
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
  if (!FLB_INB(u.y >= 0 && u.y < d.ny && u.x0 >= 0 && u.x0 + VEC <= d.nx && plane == (int64_t)d.nx * d.ny, 103))
    return;
  const int64_t off = (int64_t)u.y * d.nx + u.x0;
#pragma unroll
  for (int i = 0; i < 9; ++i) VecIO<R, VEC>::st(dst + i * plane + off, f[i]);
  if constexpr (SAMPLE) {
    R* fields = reinterpret_cast<R*>(ws + d.off_fields);
    for (int slot = 0; slot < (int)d.n_fields; ++slot) {
      if (!FLB_INB(slot < kMaxFields && d.field_id[slot] >= 0 && d.field_id[slot] < kMaxFields, 104)) continue;
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
