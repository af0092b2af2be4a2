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

#ifndef FLB_MMA_VOLATILE
#define FLB_MMA_VOLATILE 1   // keep the MMA chains in program order (the compiler may not interleave tiles)
#endif
#if FLB_MMA_VOLATILE
#define FLB_MMA_ASM asm volatile
#else
#define FLB_MMA_ASM asm
#endif
#ifndef FLB_STEP_MINB
#define FLB_STEP_MINB 2        // minimum resident blocks per SM (network variants: <= 128 registers)
#endif
#ifndef FLB_STEP_MINB_PLAIN
#define FLB_STEP_MINB_PLAIN 3  // minimum resident blocks per SM (plain variants: caps registers at 85)
#endif



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

// ---------------------------------------------------------------------------
// Noise-scale network on the tensor cores (warp-level mma.sync m16n8k16, bfloat16
// operands, FP32 accumulation).  The sites of a warp are the M dimension: tile m
// holds warp sites 16m .. 16m+15, thread (g = lane/4, q = lane%4) owns rows g and
// g+8 of the accumulator and columns 2q, 2q+1.  The accumulator layout of two
// adjacent 8-column tiles is exactly the A-operand layout of the next layer, so
// h1 and h2 never leave registers; ReLU and the bfloat16 rounding are one cvt.
// Biases enter as the FP32 C operand.
// One lane's share of the network (176 B, 16-B aligned, so a lane reads it with
// 128-bit shared loads and the 32 lanes hit distinct banks): B-fragment words of
// layer 1 (per n-tile; the second word is 0 since K = 3), layer 2 ([n-tile][k-tile][2])
// and layer 3 ([k-tile][2]); bias pairs (b[8j+2q], b[8j+2q+1]) per n-tile.
struct __align__(16) MlpLane {
  uint4 b1;
  uint4 b2[4];
  uint4 b3;
  float4 c1[2], c2[2];
  float4 c3;
};
struct MlpFrags {
  MlpLane lanes[32];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// relu, round to bfloat16 and pack (lo in the low half)
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// d = a b + (c0, c1, c0, c1)
__device__ __forceinline__ void mma_bias(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1,
                                         float2 c) {
  FLB_MMA_ASM(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%10,%11};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c.x), "f"(c.y));
}

// d += a b
__device__ __forceinline__ void mma_acc(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  FLB_MMA_ASM(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void build_mlp_frags(const MlpWeights& w, MlpFrags& F) {
  for (int i = threadIdx.x; i < 32 * 4; i += blockDim.x) {
    const int lane = i >> 2, j = i & 3, g = lane >> 2, q = lane & 3, n = 8 * j + g;
    MlpLane& M = F.lanes[lane];
    uint32_t* b1 = reinterpret_cast<uint32_t*>(&M.b1);
    uint32_t* b2 = reinterpret_cast<uint32_t*>(M.b2);
    uint32_t* b3 = reinterpret_cast<uint32_t*>(&M.b3);
    float* c1 = reinterpret_cast<float*>(M.c1);
    float* c2 = reinterpret_cast<float*>(M.c2);
    float lo = 0.f, hi = 0.f;                       // B1[k][n] = W1[n][k], k < 3
    if (q == 0) { lo = w.W1[3 * n]; hi = w.W1[3 * n + 1]; }
    if (q == 1) { lo = w.W1[3 * n + 2]; }
    b1[j] = pack_bf16(lo, hi);
    c1[2 * j] = w.b1[8 * j + 2 * q]; c1[2 * j + 1] = w.b1[8 * j + 2 * q + 1];
    c2[2 * j] = w.b2[8 * j + 2 * q]; c2[2 * j + 1] = w.b2[8 * j + 2 * q + 1];
    for (int t = 0; t < 2; ++t)
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * t + 8 * h + 2 * q;
        b2[(j * 2 + t) * 2 + h] = pack_bf16(w.W2[n * kMlpHidden + k], w.W2[n * kMlpHidden + k + 1]);
      }
    if (j < 2) {
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * j + 8 * h + 2 * q;
        b3[j * 2 + h] = g < kMlpOut ? pack_bf16(w.W3[g * kMlpHidden + k], w.W3[g * kMlpHidden + k + 1]) : 0u;
      }
    }
    if (j == 0) M.c3 = q < 3 ? make_float4(w.b3[2 * q], w.b3[2 * q + 1], 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// One 16-site tile: feature words of rows g and g+8 (x0 = (u_x, u_y), x1 = (rho - rho0, 0)),
// outputs o_c for c in {2q, 2q+1} of both rows.  The lane's fragments come from shared memory.
__device__ __forceinline__ void mlp_tile(const MlpLane& M, int q, uint2 f0, uint2 f1, float (&o)[4]) {
  uint32_t a[4] = {0u, 0u, 0u, 0u};
  if (q == 0) { a[0] = f0.x; a[1] = f1.x; }
  if (q == 1) { a[0] = f0.y; a[1] = f1.y; }
  const uint4 b1 = M.b1;
  const float4 c1a = M.c1[0], c1b = M.c1[1];
  float h[4][4];
  mma_bias(h[0], a, b1.x, 0u, make_float2(c1a.x, c1a.y));                         // layer 1
  mma_bias(h[1], a, b1.y, 0u, make_float2(c1a.z, c1a.w));
  mma_bias(h[2], a, b1.z, 0u, make_float2(c1b.x, c1b.y));
  mma_bias(h[3], a, b1.w, 0u, make_float2(c1b.z, c1b.w));
  uint32_t a2[2][4];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    a2[t][0] = relu_pack(h[2 * t][0], h[2 * t][1]);
    a2[t][1] = relu_pack(h[2 * t][2], h[2 * t][3]);
    a2[t][2] = relu_pack(h[2 * t + 1][0], h[2 * t + 1][1]);
    a2[t][3] = relu_pack(h[2 * t + 1][2], h[2 * t + 1][3]);
  }
  const float4 c2a = M.c2[0], c2b = M.c2[1];
  const float2 c2[4] = {make_float2(c2a.x, c2a.y), make_float2(c2a.z, c2a.w), make_float2(c2b.x, c2b.y),
                        make_float2(c2b.z, c2b.w)};
#pragma unroll
  for (int j = 0; j < 4; ++j) {                                                    // layer 2
    const uint4 b = M.b2[j];                       // (k-tile 0: w0 w1, k-tile 1: w0 w1)
    mma_bias(h[j], a2[0], b.x, b.y, c2[j]);
    mma_acc(h[j], a2[1], b.z, b.w);
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    a2[t][0] = relu_pack(h[2 * t][0], h[2 * t][1]);
    a2[t][1] = relu_pack(h[2 * t][2], h[2 * t][3]);
    a2[t][2] = relu_pack(h[2 * t + 1][0], h[2 * t + 1][1]);
    a2[t][3] = relu_pack(h[2 * t + 1][2], h[2 * t + 1][3]);
  }
  const uint4 b3 = M.b3;
  const float4 c3 = M.c3;
  mma_bias(o, a2[0], b3.x, b3.y, make_float2(c3.x, c3.y));                         // layer 3
  mma_acc(o, a2[1], b3.z, b3.w);
}

// Two independent 16-site tiles with their instruction streams interleaved by hand,
// so the tensor pipe always has a second MMA chain to work on while one waits.
__device__ __forceinline__ void mlp_tile2(const MlpLane& M, int q, uint2 fa0, uint2 fa1, uint2 fb0, uint2 fb1,
                                          float (&oa)[4], float (&ob)[4]) {
  uint32_t a[4] = {0u, 0u, 0u, 0u}, b[4] = {0u, 0u, 0u, 0u};
  if (q == 0) { a[0] = fa0.x; a[1] = fa1.x; b[0] = fb0.x; b[1] = fb1.x; }
  if (q == 1) { a[0] = fa0.y; a[1] = fa1.y; b[0] = fb0.y; b[1] = fb1.y; }
  const uint4 b1 = M.b1;
  const float4 c1a = M.c1[0], c1b = M.c1[1];
  const float2 c1[4] = {make_float2(c1a.x, c1a.y), make_float2(c1a.z, c1a.w), make_float2(c1b.x, c1b.y),
                        make_float2(c1b.z, c1b.w)};
  const uint32_t b1w[4] = {b1.x, b1.y, b1.z, b1.w};
  float ha[4][4], hb[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {                                                    // layer 1
    mma_bias(ha[j], a, b1w[j], 0u, c1[j]);
    mma_bias(hb[j], b, b1w[j], 0u, c1[j]);
  }
  uint32_t pa[2][4], pb[2][4];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    pa[t][0] = relu_pack(ha[2 * t][0], ha[2 * t][1]);         pb[t][0] = relu_pack(hb[2 * t][0], hb[2 * t][1]);
    pa[t][1] = relu_pack(ha[2 * t][2], ha[2 * t][3]);         pb[t][1] = relu_pack(hb[2 * t][2], hb[2 * t][3]);
    pa[t][2] = relu_pack(ha[2 * t + 1][0], ha[2 * t + 1][1]); pb[t][2] = relu_pack(hb[2 * t + 1][0], hb[2 * t + 1][1]);
    pa[t][3] = relu_pack(ha[2 * t + 1][2], ha[2 * t + 1][3]); pb[t][3] = relu_pack(hb[2 * t + 1][2], hb[2 * t + 1][3]);
  }
  const float4 c2a = M.c2[0], c2b = M.c2[1];
  const float2 c2[4] = {make_float2(c2a.x, c2a.y), make_float2(c2a.z, c2a.w), make_float2(c2b.x, c2b.y),
                        make_float2(c2b.z, c2b.w)};
#pragma unroll
  for (int j = 0; j < 4; ++j) {                                                    // layer 2
    const uint4 w = M.b2[j];
    mma_bias(ha[j], pa[0], w.x, w.y, c2[j]);
    mma_bias(hb[j], pb[0], w.x, w.y, c2[j]);
    mma_acc(ha[j], pa[1], w.z, w.w);
    mma_acc(hb[j], pb[1], w.z, w.w);
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    pa[t][0] = relu_pack(ha[2 * t][0], ha[2 * t][1]);         pb[t][0] = relu_pack(hb[2 * t][0], hb[2 * t][1]);
    pa[t][1] = relu_pack(ha[2 * t][2], ha[2 * t][3]);         pb[t][1] = relu_pack(hb[2 * t][2], hb[2 * t][3]);
    pa[t][2] = relu_pack(ha[2 * t + 1][0], ha[2 * t + 1][1]); pb[t][2] = relu_pack(hb[2 * t + 1][0], hb[2 * t + 1][1]);
    pa[t][3] = relu_pack(ha[2 * t + 1][2], ha[2 * t + 1][3]); pb[t][3] = relu_pack(hb[2 * t + 1][2], hb[2 * t + 1][3]);
  }
  const uint4 b3 = M.b3;
  const float4 c3 = M.c3;
  mma_bias(oa, pa[0], b3.x, b3.y, make_float2(c3.x, c3.y));                       // layer 3
  mma_bias(ob, pb[0], b3.x, b3.y, make_float2(c3.x, c3.y));
  mma_acc(oa, pa[1], b3.z, b3.w);
  mma_acc(ob, pb[1], b3.z, b3.w);
}

// ---------------------------------------------------------------------------
// D2Q9.  Population order (Sec. 3): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
// 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
// Network modes of the D2Q9 step kernel: kMlpOff (s = 1) or kMlpWarp (each warp evaluates
// the network for its own sites between the loads and the collision, two 16-site tiles at
// a time).  A warp-specialised variant (separate network warps, block barriers) measured
// slower on GB300: its register union halves the resident blocks.
constexpr int kMlpOff = 0, kMlpWarp = 1;

template <typename R, bool DEV, int VEC, bool SAMPLE, int NET>
__global__ void __launch_bounds__(kStepThreads, NET == kMlpOff ? FLB_STEP_MINB_PLAIN : FLB_STEP_MINB)
k_step_d2q9(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
            int64_t n_vblocks, char* __restrict__ ws, int parity, uint32_t step,
            const MlpWeights* __restrict__ mlp_w, const uint64_t* __restrict__ step_dev) {
  if (step_dev) {                  // graph replay: step = device base + offset
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  constexpr int VX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int VY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  constexpr bool MLP = NET != kMlpOff;
  static_assert(!MLP || sizeof(R) == 4, "the network runs on the FP32 path");
  __shared__ MlpFrags sfr;
  __shared__ uint2 s_feat[MLP ? kStepThreads * VEC : 1];
  __shared__ float2 s_out[MLP ? kStepThreads * VEC * 4 : 1];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if constexpr (MLP) {
    build_mlp_frags(*mlp_w, sfr);
    __syncthreads();
  }
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = n_reps == 1 ? 0 : find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int nx = d.nx, ny = d.ny;
    // per-replica unit counts stay below 2^31 (sites < 2^32, at least 2 sites per unit or VEC = 1
    // on lattices of < 2^31 sites), so the index arithmetic is 32-bit
    const int n_units = (int)d.n_units, upr = d.units_per_row;
    const int tid = (int)threadIdx.x;
    const int unit_raw = (int)(vb - vb_begin[r]) * kStepThreads + tid;
    const bool active = unit_raw < n_units;
    const int unit = unit_raw < n_units ? unit_raw : n_units - 1;
    const int y = (int)((unsigned)unit / (unsigned)upr);
    const int xq = unit - y * upr;
    const int x0 = xq * VEC;
    const int64_t plane = (int64_t)nx * ny;
    const R* __restrict__ src = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    // neighbour lanes hold the adjacent unit of the same row?
    const bool left_in_warp = lane > 0 && xq > 0;
    const bool right_in_warp = lane < 31 && (xq + 1) < upr && (unit_raw + 1) < n_units;
    const R rho0 = coef<R>(d, kCoRho0);
    const bool noisy = d.noise_mask != 0;

    R f[9][VEC];
    R sum[VEC], ux[VEC], uy[VEC];
    {
      // ---- pull streaming: f_i(x) = f*_i(x - v_i) -------------------------
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
      // ---- density, momentum, velocity (Sec. 2) ----------------------------
      // deviation storage: sum_i w_i rho0 = rho0 and sum_i w_i rho0 v_i = 0
#pragma unroll
      for (int s = 0; s < VEC; ++s) {
        sum[s] = ((f[0][s] + (f[1][s] + f[3][s])) + (f[2][s] + f[4][s])) + ((f[5][s] + f[7][s]) + (f[6][s] + f[8][s]));
        const R jx = (f[1][s] - f[3][s]) + ((f[5][s] - f[7][s]) + (f[8][s] - f[6][s]));
        const R jy = (f[2][s] - f[4][s]) + ((f[5][s] - f[7][s]) + (f[6][s] - f[8][s]));
        const R irho = (R)1 / (DEV ? rho0 + sum[s] : sum[s]);
        ux[s] = jx * irho;
        uy[s] = jy * irho;
      }
      if constexpr (MLP) {
#pragma unroll
        for (int s = 0; s < VEC; ++s)
          s_feat[tid * VEC + s] = make_uint2(pack_bf16((float)ux[s], (float)uy[s]),
                                             pack_bf16((float)(DEV ? sum[s] : sum[s] - rho0), 0.f));
      }
    }

    // ---- per-site noise scales from the network (tensor cores) --------------
    // warp sites w = tid * VEC + s; 16-site tile m covers w in [16m, 16m + 16)
    if constexpr (NET == kMlpWarp) {
      __syncwarp();
      const int g = lane >> 2, q = lane & 3;
      const uint2* feat = s_feat + warp * 32 * VEC;
      float2* outw = s_out + warp * 32 * VEC * 4;
#pragma unroll 1
      for (int m = 0; m < 2 * VEC; m += 2) {
        float oa[4], ob[4];
        mlp_tile2(sfr.lanes[lane], q, feat[16 * m + g], feat[16 * m + g + 8], feat[16 * m + 16 + g],
                  feat[16 * m + 24 + g], oa, ob);
        if (q < 3) {
          outw[(16 * m + g) * 4 + q] = make_float2(oa[0], oa[1]);
          outw[(16 * m + g + 8) * 4 + q] = make_float2(oa[2], oa[3]);
          outw[(16 * m + 16 + g) * 4 + q] = make_float2(ob[0], ob[1]);
          outw[(16 * m + 24 + g) * 4 + q] = make_float2(ob[2], ob[3]);
        }
      }
      __syncwarp();
    }

    const R it3 = coef<R>(d, kCoInvTau + 3), it4 = coef<R>(d, kCoInvTau + 4), it5 = coef<R>(d, kCoInvTau + 5);
    const R it6 = coef<R>(d, kCoInvTau + 6), it7 = coef<R>(d, kCoInvTau + 7), it8 = coef<R>(d, kCoInvTau + 8);
    const R a3 = coef<R>(d, kCoAmp + 3), a4 = coef<R>(d, kCoAmp + 4), a5 = coef<R>(d, kCoAmp + 5);
    const R a6 = coef<R>(d, kCoAmp + 6), a7 = coef<R>(d, kCoAmp + 7), a8 = coef<R>(d, kCoAmp + 8);
    const R S3 = (R)1.7320508075688772935, S32 = (R)1.2247448713915890491,
            S6 = (R)2.4494897427831780982;
    R fld[kMaxFields][VEC];

#pragma unroll
    for (int s = 0; s < VEC; ++s) {
      const R g0 = f[0][s], g1 = f[1][s], g2 = f[2][s], g3 = f[3][s], g4 = f[4][s];
      const R g5 = f[5][s], g6 = f[6][s], g7 = f[7][s], g8 = f[8][s];
      const R rho = DEV ? rho0 + sum[s] : sum[s];
      // non-conserved moments of Eq. 9 (identical for f and f - w rho0)
      const R ax = g1 + g3, ay = g2 + g4, dg = (g5 + g7) + (g6 + g8);
      const R M3 = (R)1.5 * (ax - ay);
      const R M4 = (R)3 * ((g5 + g7) - (g6 + g8));
      const R M5 = (R)0.5 * (ax + ay) + (R)2 * dg - g0;
      const R M6 = S32 * (g3 - g1) + S6 * ((g5 - g7) + (g8 - g6));
      const R M7 = S32 * (g4 - g2) + S6 * ((g5 - g7) + (g6 - g8));
      const R M8 = (R)0.5 * g0 - (ax + ay) + (R)2 * dg;
      // equilibrium moments, Eq. 10
      const R ux2 = ux[s] * ux[s], uy2 = uy[s] * uy[s];
      const R E3 = (R)1.5 * rho * (ux2 - uy2);
      const R E4 = (R)3 * rho * ux[s] * uy[s];
      const R E5 = (R)1.5 * rho * (ux2 + uy2);
      if constexpr (SAMPLE) {
        const R jx = ux[s] * rho, jy = uy[s] * rho;
        const R mom[9] = {sum[s], S3 * jx, S3 * jy, M3, M4, M5, M6, M7, M8};
#pragma unroll
        for (int a = 0; a < 9; ++a) fld[a][s] = mom[a] - coef<R>(d, kCoMref + a);
        fld[9][s] = ux[s] - coef<R>(d, kCoU0x);
        fld[10][s] = uy[s] - coef<R>(d, kCoU0y);
      }
      // relaxation (Eq. 5)
      R D3 = (E3 - M3) * it3, D4 = (E4 - M4) * it4, D5 = (E5 - M5) * it5;
      R D6 = -M6 * it6, D7 = -M7 * it7, D8 = -M8 * it8;
      if (noisy) {
        R nrm[6];
        {
          const uint32_t site = (uint32_t)y * (uint32_t)nx + (uint32_t)(x0 + s);
          const uint4 w0 = philox4x32_10(site, step, 0u, d.stream, d.seed_lo, d.seed_hi);
          const uint4 w1 = philox4x32_10(site, step, 1u, d.stream, d.seed_lo, d.seed_hi);
          box_muller(w0.x, w0.y, nrm[0], nrm[1]);
          box_muller(w0.z, w0.w, nrm[2], nrm[3]);
          box_muller(w1.x, w1.y, nrm[4], nrm[5]);
        }
        R sc[6] = {(R)1, (R)1, (R)1, (R)1, (R)1, (R)1};
        if constexpr (MLP) {
          const float2* o = s_out + (tid * VEC + s) * 4;
          const float2 o01 = o[0], o23 = o[1], o45 = o[2];
          sc[0] = (R)1 + (R)o01.x; sc[1] = (R)1 + (R)o01.y; sc[2] = (R)1 + (R)o23.x;
          sc[3] = (R)1 + (R)o23.y; sc[4] = (R)1 + (R)o45.x; sc[5] = (R)1 + (R)o45.y;
        }
        D3 += sc[0] * a3 * nrm[0]; D4 += sc[1] * a4 * nrm[1]; D5 += sc[2] * a5 * nrm[2];
        D6 += sc[3] * a6 * nrm[3]; D7 += sc[4] * a7 * nrm[4]; D8 += sc[5] * a8 * nrm[5];
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
            int64_t n_vblocks, char* __restrict__ ws, int parity, uint32_t step,
            const uint64_t* __restrict__ step_dev) {
  if (step_dev) {
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
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
    const R rho = DEV ? coef<R>(d, kCoRho0) + sum : sum;
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
        const R val = fid < 3 ? mom[fid] - coef<R>(d, kCoMref + fid) : u - coef<R>(d, kCoU0x);
        fields[(int64_t)slot * nx + x] = val;
      }
    }
    R D2 = (E2 - M2) * coef<R>(d, kCoInvTau + 2);
    if (d.noise_mask) {
      const uint4 w = philox4x32_10((uint32_t)x, step, 0u, d.stream, d.seed_lo, d.seed_hi);
      R n0, n1;
      box_muller(w.x, w.y, n0, n1);
      D2 += coef<R>(d, kCoAmp + 2) * n0;
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
#define FLB_L(S, N, B) k_step_d2q9<R, DEV, VEC, S, N><<<L.grid, B, 0, st>>>( \
      L.descs, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w, L.step_dev)
  if constexpr (sizeof(R) == 4) {
    if (mlp) {
      if (sample) FLB_L(true, kMlpWarp, kStepThreads); else FLB_L(false, kMlpWarp, kStepThreads);
      return;
    }
  }
  if (sample) FLB_L(true, kMlpOff, kStepThreads); else FLB_L(false, kMlpOff, kStepThreads);
#undef FLB_L
}

void launch_step(int lattice, int precision, int vec, const StepLaunch& L, bool sample, bool mlp,
                 cudaStream_t st) {
  if (lattice == FLB_D2Q9) {
    if (precision == FLB_FP64) launch_d2q9_vec<double, false, 1>(L, sample, false, st);
    else if (vec == 4) launch_d2q9_vec<float, true, 4>(L, sample, mlp, st);
    else if (vec == 2) launch_d2q9_vec<float, true, 2>(L, sample, mlp, st);
    else launch_d2q9_vec<float, true, 1>(L, sample, mlp, st);
  } else {
#define FLB_L1(R, DEV, S) k_step_d1q3<R, DEV, S><<<L.grid, L.block, 0, st>>>( \
      L.descs, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, L.step_dev)
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

__global__ void k_set_step(uint64_t* s, uint64_t v) { *s = v; }
__global__ void k_advance_step(uint64_t* s, uint64_t n) { *s += n; }

void launch_set_step(uint64_t* s, uint64_t v, cudaStream_t st) { k_set_step<<<1, 1, 0, st>>>(s, v); }
void launch_advance_step(uint64_t* s, uint64_t n, cudaStream_t st) { k_advance_step<<<1, 1, 0, st>>>(s, n); }

}  // namespace flb
