// Fused pull-stream / collide / noise kernels (Eqs. 1, 3, 5, 8) and the
// initial-state and conservation kernels of libflb.
//
// One step reads the post-collision populations f*_i(x - v_i) of the previous
// step (pull streaming, periodic), forms density, momentum and the
// non-conserved Hermite moments M^a = sum_i m_i^a f_i of Eq. 9 in closed form,
// relaxes them towards the equilibrium moments of Eq. 10 at rate 1/tau^a,
// adds the noise of Eq. 8 drawn from Philox4x32-10, and writes
// f*_i = f_i + sum_{a non-conserved} n_i^a (Delta M^a + xi^a), n_i^a = w_i m_i^a.
// Density and momentum are untouched, so they are conserved up to rounding.
#include <cstdio>
#include "flb_internal.cuh"

namespace flb {

// Per-site noise-scale network weights, FP32 copies of the bfloat16 weights.
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

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// s_c = 1 + o_c(u_x, u_y, rho - rho0) with bfloat16 operands and FP32 accumulation.
__device__ __forceinline__ void mlp_scales(const MlpWeights& w, float ux, float uy, float drho,
                                           float (&s)[kMlpOut]) {
  const float x0 = bf16_round(ux), x1 = bf16_round(uy), x2 = bf16_round(drho);
  float h1[kMlpHidden];
#pragma unroll
  for (int h = 0; h < kMlpHidden; ++h) {
    float z = w.b1[h];
    z = fmaf(w.W1[3 * h + 0], x0, z);
    z = fmaf(w.W1[3 * h + 1], x1, z);
    z = fmaf(w.W1[3 * h + 2], x2, z);
    h1[h] = bf16_round(fmaxf(z, 0.f));
  }
  float o[kMlpOut];
#pragma unroll
  for (int c = 0; c < kMlpOut; ++c) o[c] = w.b3[c];
#pragma unroll 4
  for (int h = 0; h < kMlpHidden; ++h) {
    float z = w.b2[h];
#pragma unroll
    for (int k = 0; k < kMlpHidden; ++k) z = fmaf(w.W2[h * kMlpHidden + k], h1[k], z);
    const float h2 = bf16_round(fmaxf(z, 0.f));
#pragma unroll
    for (int c = 0; c < kMlpOut; ++c) o[c] = fmaf(w.W3[c * kMlpHidden + h], h2, o[c]);
  }
#pragma unroll
  for (int c = 0; c < kMlpOut; ++c) s[c] = 1.f + o[c];
}

// ---------------------------------------------------------------------------
// D2Q9.  Population order (Sec. 3): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
// 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
__device__ __constant__ int c_vx9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ int c_vy9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename R, bool DEV, int VEC, bool SAMPLE, bool MLP>
__global__ void __launch_bounds__(256)
k_step_d2q9(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
            int64_t n_vblocks, char* __restrict__ ws, int parity, uint32_t step,
            const MlpWeights* __restrict__ mlp_w) {
  constexpr int VX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int VY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  __shared__ MlpWeights sw;
  if constexpr (MLP) {
    const float* src = reinterpret_cast<const float*>(mlp_w);
    float* dst = reinterpret_cast<float*>(&sw);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpWeights) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int nx = d.nx, ny = d.ny;
    const int64_t unit_raw = (vb - vb_begin[r]) * blockDim.x + threadIdx.x;
    const bool active = unit_raw < d.n_units;
    const int64_t unit = active ? unit_raw : d.n_units - 1;
    const int y = (int)(unit / d.units_per_row);
    const int xq = (int)(unit - (int64_t)y * d.units_per_row);
    const int x0 = xq * VEC;
    const int64_t plane = (int64_t)nx * ny;
    const R* __restrict__ src = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    // neighbour lanes hold the adjacent unit of the same row?
    const bool left_in_warp = lane > 0 && xq > 0;
    const bool right_in_warp = lane < 31 && (xq + 1) < d.units_per_row && (unit_raw + 1) < d.n_units;

    // ---- pull streaming: f_i(x) = f*_i(x - v_i) -------------------------
    R f[9][VEC];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int ys = y - VY[i];
      ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
      const R* row = src + i * plane + (int64_t)ys * nx;
      R v[VEC];
      VecIO<R, VEC>::ld(row + x0, v);
      if (VX[i] == 0) {
#pragma unroll
        for (int s = 0; s < VEC; ++s) f[i][s] = v[s];
      } else if (VX[i] == 1) {                    // needs x0-1 .. x0+VEC-2
        R left = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
        if (!left_in_warp) left = __ldg(row + (x0 == 0 ? nx - 1 : x0 - 1));
        f[i][0] = left;
#pragma unroll
        for (int s = 1; s < VEC; ++s) f[i][s] = v[s - 1];
      } else {                                   // needs x0+1 .. x0+VEC
        R right = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (!right_in_warp) right = __ldg(row + (x0 + VEC == nx ? 0 : x0 + VEC));
#pragma unroll
        for (int s = 0; s < VEC - 1; ++s) f[i][s] = v[s + 1];
        f[i][VEC - 1] = right;
      }
    }

    const R rho0 = (R)d.rho0;
    const R it3 = (R)d.inv_tau[3], it4 = (R)d.inv_tau[4], it5 = (R)d.inv_tau[5];
    const R it6 = (R)d.inv_tau[6], it7 = (R)d.inv_tau[7], it8 = (R)d.inv_tau[8];
    const R a3 = (R)d.amp[3], a4 = (R)d.amp[4], a5 = (R)d.amp[5];
    const R a6 = (R)d.amp[6], a7 = (R)d.amp[7], a8 = (R)d.amp[8];
    const bool noisy = d.noise_mask != 0;
    const R S3 = (R)1.7320508075688772935, S32 = (R)1.2247448713915890491,
            S6 = (R)2.4494897427831780982;
    R fld[kMaxFields][VEC];

#pragma unroll
    for (int s = 0; s < VEC; ++s) {
      const R g0 = f[0][s], g1 = f[1][s], g2 = f[2][s], g3 = f[3][s], g4 = f[4][s];
      const R g5 = f[5][s], g6 = f[6][s], g7 = f[7][s], g8 = f[8][s];
      // density and momentum (Sec. 2); in deviation storage sum_i w_i rho0 = rho0, sum w v = 0
      const R sum = ((g0 + (g1 + g3)) + (g2 + g4)) + ((g5 + g7) + (g6 + g8));
      const R rho = DEV ? rho0 + sum : sum;
      const R jx = (g1 - g3) + ((g5 - g7) + (g8 - g6));
      const R jy = (g2 - g4) + ((g5 - g7) + (g6 - g8));
      const R irho = (R)1 / rho;
      const R ux = jx * irho, uy = jy * irho;
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
        const R mom[9] = {sum, S3 * jx, S3 * jy, M3, M4, M5, M6, M7, M8};
#pragma unroll
        for (int a = 0; a < 9; ++a) fld[a][s] = mom[a] - (R)d.mref[a];
        fld[9][s] = ux - (R)d.u0x;
        fld[10][s] = uy - (R)d.u0y;
      }
      // relaxation (Eq. 5)
      R D3 = (E3 - M3) * it3, D4 = (E4 - M4) * it4, D5 = (E5 - M5) * it5;
      R D6 = -M6 * it6, D7 = -M7 * it7, D8 = -M8 * it8;
      if (noisy) {
        const uint32_t site = (uint32_t)y * (uint32_t)nx + (uint32_t)(x0 + s);
        const uint4 w0 = philox4x32_10(site, step, 0u, d.stream, d.seed_lo, d.seed_hi);
        const uint4 w1 = philox4x32_10(site, step, 1u, d.stream, d.seed_lo, d.seed_hi);
        R n0, n1, n2, n3, n4, n5;
        box_muller(w0.x, w0.y, n0, n1);
        box_muller(w0.z, w0.w, n2, n3);
        box_muller(w1.x, w1.y, n4, n5);
        R sc[6] = {(R)1, (R)1, (R)1, (R)1, (R)1, (R)1};
        if constexpr (MLP) {
          float sf[kMlpOut];
          mlp_scales(sw, (float)ux, (float)uy, (float)(rho - rho0), sf);
#pragma unroll
          for (int c = 0; c < 6; ++c) sc[c] = (R)sf[c];
        }
        D3 += sc[0] * a3 * n0; D4 += sc[1] * a4 * n1; D5 += sc[2] * a5 * n2;
        D6 += sc[3] * a6 * n3; D7 += sc[4] * a7 * n4; D8 += sc[5] * a8 * n5;
      }
      // back transform of the moment change, n_i^a = w_i m_i^a
      const R w1 = (R)1 / (R)9, w5 = (R)1 / (R)36;
      const R c0 = (R)(4.0 / 9.0) * ((R)0.5 * D8 - D5);
      const R ax5 = (R)0.5 * D5 - D8;                   // common to the axis populations
      const R hx = (R)1.5 * D3;
      const R p6 = S32 * D6, p7 = S32 * D7;
      const R dcom = (R)2 * (D5 + D8);                  // common to the diagonal populations
      const R q6 = S6 * D6, q7 = S6 * D7, q4 = (R)3 * D4;
      f[0][s] = g0 + c0;
      f[1][s] = g1 + w1 * (ax5 + hx - p6);
      f[3][s] = g3 + w1 * (ax5 + hx + p6);
      f[2][s] = g2 + w1 * (ax5 - hx - p7);
      f[4][s] = g4 + w1 * (ax5 - hx + p7);
      f[5][s] = g5 + w5 * (dcom + q4 + q6 + q7);
      f[6][s] = g6 + w5 * (dcom - q4 - q6 + q7);
      f[7][s] = g7 + w5 * (dcom + q4 - q6 - q7);
      f[8][s] = g8 + w5 * (dcom - q4 + q6 - q7);
    }

    if (active) {
      const int64_t off = (int64_t)y * nx + x0;
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
  }
}

// ---------------------------------------------------------------------------
// D1Q3: v = (0, +1, -1), w = (2/3, 1/6, 1/6), moments 1, sqrt3 v, (3 v^2 - 1)/sqrt2.
template <typename R, bool DEV, bool SAMPLE>
__global__ void __launch_bounds__(256)
k_step_d1q3(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
            int64_t n_vblocks, char* __restrict__ ws, int parity, uint32_t step) {
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int nx = d.nx;
    const int64_t x64 = (vb - vb_begin[r]) * blockDim.x + threadIdx.x;
    if (x64 >= d.n_units) continue;
    const int x = (int)x64;
    const R* src = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
    R* dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    const R g0 = src[x];
    const R g1 = src[nx + (x == 0 ? nx - 1 : x - 1)];
    const R g2 = src[2 * nx + (x == nx - 1 ? 0 : x + 1)];
    const R sum = g0 + (g1 + g2);
    const R rho = DEV ? (R)d.rho0 + sum : sum;
    const R j = g1 - g2;
    const R u = j / rho;
    const R S2 = (R)1.4142135623730950488, IS2 = (R)0.70710678118654752440;
    const R M2 = S2 * (g1 + g2) - IS2 * g0;
    const R E2 = (R)3 * IS2 * rho * u * u;
    if constexpr (SAMPLE) {
      R* fields = reinterpret_cast<R*>(ws + d.off_fields);
      const R mom[3] = {sum, (R)1.7320508075688772935 * j, M2};
      for (int slot = 0; slot < (int)d.n_fields; ++slot) {
        const int fid = d.field_id[slot];
        const R val = fid < 3 ? mom[fid] - (R)d.mref[fid] : u - (R)d.u0x;
        fields[(int64_t)slot * nx + x] = val;
      }
    }
    R D2 = (E2 - M2) * (R)d.inv_tau[2];
    if (d.noise_mask) {
      const uint4 w = philox4x32_10((uint32_t)x, step, 0u, d.stream, d.seed_lo, d.seed_hi);
      R n0, n1;
      box_muller(w.x, w.y, n0, n1);
      D2 += (R)d.amp[2] * n0;
    }
    dst[x] = g0 - (R)(2.0 / 3.0) * IS2 * D2;
    const R side = (R)(1.0 / 6.0) * S2 * D2;
    dst[nx + x] = g1 + side;
    dst[2 * nx + x] = g2 + side;
  }
}

// ---------------------------------------------------------------------------
// Initial state.  mode 0: f^0(rho0, u0).  mode 1: f^0 + sum_a n_i^a dM^a with
// dM^a = sqrt(mu rho0) N_a (Philox tag 1, step 0) and the lattice mean of the
// density and momentum fluctuations removed (pass 1 sums, pass 2 writes).
__device__ __forceinline__ void thermal_normals(const ReplicaDesc& d, uint32_t site, int q,
                                                double (&N)[12]) {
  const int calls = (q + 3) / 4;
  for (int c = 0; c < calls; ++c) {
    const uint4 w = philox4x32_10(site, 0u, (uint32_t)c | (1u << 8), d.stream, d.seed_lo, d.seed_hi);
    box_muller(w.x, w.y, N[4 * c + 0], N[4 * c + 1]);
    box_muller(w.z, w.w, N[4 * c + 2], N[4 * c + 3]);
  }
}

// Deterministic block reduction of three sums: each block writes its partial sums
// (fixed site set, fixed shuffle tree); k_finish_sums adds the partials in order.
__device__ __forceinline__ void block_sum3(double (&acc)[3], double* __restrict__ partial) {
  __shared__ double red[32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
      for (int w = 0; w < nw; ++w) v += red[w][k];
      partial[3 * blockIdx.x + k] = v;
    }
  }
}

__global__ void k_finish_sums(const double* __restrict__ partial, int nblocks, double* __restrict__ sums,
                              DevStatus* status, int r) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < 3; ++k) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[3 * b + k];
    sums[k] = v;
    if (status && !isfinite(v) && status->error == 0) { status->error = FLB_EUNSTABLE; status->replica = r; }
  }
}

__global__ void k_thermal_sum(const ReplicaDesc* __restrict__ descs, int r, double* __restrict__ partial) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny;
  double acc[3] = {0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double N[12];
    thermal_normals(d, (uint32_t)s, d.q, N);
    acc[0] += N[0]; acc[1] += N[1];
    if (d.q == 9) acc[2] += N[2];
  }
  block_sum3(acc, partial);
}

template <typename R, bool DEV>
__global__ void k_init(const ReplicaDesc* __restrict__ descs, int r, char* __restrict__ ws, int mode,
                       const double* __restrict__ feq0, const double* __restrict__ sums) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny;
  R* dst = reinterpret_cast<R*>(ws + d.off_pop[0]);
  const double sm = sqrt(d.mu * d.rho0);
  const double S3 = 1.7320508075688772935, S32 = 1.2247448713915890491, S6 = 2.4494897427831780982;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double f[9];
    for (int i = 0; i < d.q; ++i) f[i] = feq0[i];
    if (mode == 1) {
      double N[12];
      thermal_normals(d, (uint32_t)s, d.q, N);
      double M[9];
      for (int a = 0; a < d.q; ++a) M[a] = sm * N[a];
      const int nc = d.q == 9 ? 3 : 2;
      for (int a = 0; a < nc; ++a) M[a] -= sm * sums[a] / (double)V;
      if (d.q == 9) {
        // f_i += w_i sum_a m_i^a M^a, Eq. 9 rows
        const double wa = 1.0 / 9.0, wd = 1.0 / 36.0;
        f[0] += (4.0 / 9.0) * (M[0] - M[5] + 0.5 * M[8]);
        const double base = M[0] + 0.5 * M[5] - M[8];
        f[1] += wa * (base + S3 * M[1] + 1.5 * M[3] - S32 * M[6]);
        f[3] += wa * (base - S3 * M[1] + 1.5 * M[3] + S32 * M[6]);
        f[2] += wa * (base + S3 * M[2] - 1.5 * M[3] - S32 * M[7]);
        f[4] += wa * (base - S3 * M[2] - 1.5 * M[3] + S32 * M[7]);
        const double db = M[0] + 2.0 * M[5] + 2.0 * M[8];
        f[5] += wd * (db + S3 * (M[1] + M[2]) + 3.0 * M[4] + S6 * (M[6] + M[7]));
        f[6] += wd * (db + S3 * (-M[1] + M[2]) - 3.0 * M[4] + S6 * (-M[6] + M[7]));
        f[7] += wd * (db - S3 * (M[1] + M[2]) + 3.0 * M[4] - S6 * (M[6] + M[7]));
        f[8] += wd * (db + S3 * (M[1] - M[2]) - 3.0 * M[4] + S6 * (M[6] - M[7]));
      } else {
        const double IS2 = 0.70710678118654752440;
        f[0] += (2.0 / 3.0) * (M[0] - IS2 * M[2]);
        f[1] += (1.0 / 6.0) * (M[0] + S3 * M[1] + 2.0 * IS2 * M[2]);
        f[2] += (1.0 / 6.0) * (M[0] - S3 * M[1] + 2.0 * IS2 * M[2]);
      }
    }
    for (int i = 0; i < d.q; ++i) {
      double v = f[i];
      if (DEV) v -= feq0[9 + i];          // w_i rho0
      dst[i * V + s] = (R)v;
    }
  }
}

// FP64 lattice sums of rho, j_x, j_y of the stored state (per-block partials).
template <typename R, bool DEV>
__global__ void k_conserved(const ReplicaDesc* __restrict__ descs, int r, const char* __restrict__ ws,
                            int parity, double* __restrict__ partial) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny;
  const R* p = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
  double acc[3] = {0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    if (d.q == 9) {
      double fv[9];
      for (int i = 0; i < 9; ++i) fv[i] = (double)p[i * V + s];
      double rho = 0;
      for (int i = 0; i < 9; ++i) rho += fv[i];
      acc[0] += DEV ? rho + d.rho0 : rho;
      acc[1] += fv[1] - fv[3] + fv[5] - fv[6] - fv[7] + fv[8];
      acc[2] += fv[2] - fv[4] + fv[5] + fv[6] - fv[7] - fv[8];
    } else {
      const double a = p[s], b = p[V + s], c = p[2 * V + s];
      acc[0] += DEV ? a + b + c + d.rho0 : a + b + c;
      acc[1] += b - c;
    }
  }
  block_sum3(acc, partial);
}

// Diagnostics: the generator exactly as the step kernels call it.
__global__ void k_philox(const uint32_t* site, int n, uint32_t step, uint32_t call, uint32_t tag,
                         uint32_t stream, uint32_t klo, uint32_t khi, int fp32, uint32_t* words,
                         double* normals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 w = philox4x32_10(site[i], step, call | (tag << 8), stream, klo, khi);
  if (words) { words[4 * i] = w.x; words[4 * i + 1] = w.y; words[4 * i + 2] = w.z; words[4 * i + 3] = w.w; }
  if (normals) {
    if (fp32) {
      float a, b, c, e;
      box_muller(w.x, w.y, a, b);
      box_muller(w.z, w.w, c, e);
      normals[4 * i] = a; normals[4 * i + 1] = b; normals[4 * i + 2] = c; normals[4 * i + 3] = e;
    } else {
      double a, b, c, e;
      box_muller(w.x, w.y, a, b);
      box_muller(w.z, w.w, c, e);
      normals[4 * i] = a; normals[4 * i + 1] = b; normals[4 * i + 2] = c; normals[4 * i + 3] = e;
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers (called from api.cu).

template <typename R, bool DEV, int VEC>
static void launch_d2q9_vec(const StepLaunch& L, bool sample, bool mlp, cudaStream_t st) {
  auto w = reinterpret_cast<const MlpWeights*>(L.mlp);
#define FLB_L(S, M) k_step_d2q9<R, DEV, VEC, S, M><<<L.grid, L.block, 0, st>>>( \
      L.descs, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w)
  if (sample) { if (mlp) FLB_L(true, true); else FLB_L(true, false); }
  else { if (mlp) FLB_L(false, true); else FLB_L(false, false); }
#undef FLB_L
}

void launch_step(int lattice, int precision, int vec, const StepLaunch& L, bool sample, bool mlp,
                 cudaStream_t st) {
  if (lattice == FLB_D2Q9) {
    if (precision == FLB_FP64) launch_d2q9_vec<double, false, 1>(L, sample, mlp, st);
    else if (vec == 4) launch_d2q9_vec<float, true, 4>(L, sample, mlp, st);
    else if (vec == 2) launch_d2q9_vec<float, true, 2>(L, sample, mlp, st);
    else launch_d2q9_vec<float, true, 1>(L, sample, mlp, st);
  } else {
#define FLB_L1(R, DEV, S) k_step_d1q3<R, DEV, S><<<L.grid, L.block, 0, st>>>( \
      L.descs, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step)
    if (precision == FLB_FP64) { if (sample) FLB_L1(double, false, true); else FLB_L1(double, false, false); }
    else { if (sample) FLB_L1(float, true, true); else FLB_L1(float, true, false); }
#undef FLB_L1
  }
}

void launch_init(int precision, const ReplicaDesc* descs, int r, char* ws, int mode, const double* feq0,
                 double* sums, double* partial, int64_t V, cudaStream_t st) {
  const int block = 256;
  const int grid = (int)((V + block - 1) / block < kReduceBlocks ? (V + block - 1) / block : kReduceBlocks);
  if (mode == 1) {
    k_thermal_sum<<<grid, block, 0, st>>>(descs, r, partial);
    k_finish_sums<<<1, 32, 0, st>>>(partial, grid, sums, nullptr, r);
  }
  if (precision == FLB_FP64) k_init<double, false><<<grid, block, 0, st>>>(descs, r, ws, mode, feq0, sums);
  else k_init<float, true><<<grid, block, 0, st>>>(descs, r, ws, mode, feq0, sums);
}

void launch_conserved(int precision, const ReplicaDesc* descs, int r, const char* ws, int parity,
                      double* sums, double* partial, DevStatus* status, int64_t V, cudaStream_t st) {
  const int block = 256;
  const int grid = (int)((V + block - 1) / block < kReduceBlocks ? (V + block - 1) / block : kReduceBlocks);
  if (precision == FLB_FP64) k_conserved<double, false><<<grid, block, 0, st>>>(descs, r, ws, parity, partial);
  else k_conserved<float, true><<<grid, block, 0, st>>>(descs, r, ws, parity, partial);
  k_finish_sums<<<1, 32, 0, st>>>(partial, grid, sums, status, r);
}

void launch_philox(const uint32_t* site, int n, uint32_t step, uint32_t call, uint32_t tag, uint32_t stream,
                   uint64_t seed, int fp32, uint32_t* words, double* normals, cudaStream_t st) {
  if (n <= 0) return;
  k_philox<<<(n + 255) / 256, 256, 0, st>>>(site, n, step, call, tag, stream, (uint32_t)seed,
                                            (uint32_t)(seed >> 32), fp32, words, normals);
}

size_t mlp_weights_bytes() { return sizeof(MlpWeights); }

}  // namespace flb
