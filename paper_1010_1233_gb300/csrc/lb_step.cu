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
// The variant with the noise-scale network is in lb_step_tc.cu.
#include <cstdio>
#include "step_common.cuh"
#include "d1q3_common.cuh"

#ifndef FLB_STEP_MINB_PLAIN
#define FLB_STEP_MINB_PLAIN 3  // minimum resident blocks per SM (caps the registers at 85)
#endif

namespace flb {

// ---------------------------------------------------------------------------
// D2Q9 step without the network (s = 1).  One thread = VEC consecutive sites of a row;
// a persistent grid loops over virtual blocks of kStepThreads units, each within one replica.
// ONE: a single replica, whose description is the kernel argument `one` (read through
// the constant bank) instead of descs[0] in global memory.
template <typename R, bool DEV, int VEC, bool SAMPLE, int FL>
__global__ void __launch_bounds__(kStepThreads, FLB_STEP_MINB_PLAIN)
k_step_d2q9(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
            const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_vblocks, char* __restrict__ ws, int parity,
            uint32_t step, const uint64_t* __restrict__ step_dev) {
  constexpr bool ONE = Flavor<FL>::kOne;
  if (step_dev) {                  // graph replay: step = device base + offset
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = ONE ? 0 : find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = ONE ? one : descs[r];
    const UnitPos u = unit_position(d, vb, ONE ? 0 : vb_begin[r], (int)threadIdx.x, kStepThreads, VEC);
    const int64_t plane = (int64_t)d.nx * d.ny;
    const R* __restrict__ src = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    R f[9][VEC];
    pull_d2q9<R, VEC>(src, plane, d.nx, d.ny, u, f);
    const R rho0 = coef<R>(d, kCoRho0);
    const bool noisy = d.noise_mask != 0;
    R fld[kMaxFields][VEC];
#pragma unroll
    for (int s = 0; s < VEC; ++s) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][s];
      R sum, ux, uy;
      macro_d2q9<R, DEV>(g, rho0, sum, ux, uy);
      R n[6] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
      const R one[6] = {(R)1, (R)1, (R)1, (R)1, (R)1, (R)1};
      if (noisy) normals_d2q9<R>(d, (uint32_t)u.y * (uint32_t)d.nx + (uint32_t)(u.x0 + s), step, n);
      R fl[kMaxFields];
      collide_d2q9<R, DEV, SAMPLE, Flavor<FL>::kGen>(d, g, sum, ux, uy, noisy, n, one, fl);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][s] = g[i];
      if constexpr (SAMPLE) {
#pragma unroll
        for (int a = 0; a < kMaxFields; ++a) fld[a][s] = fl[a];
      }
    }
    store_d2q9<R, VEC, SAMPLE>(d, ws, dst, plane, u, f, fld);
  }
}

// ---------------------------------------------------------------------------
// D1Q3, one step (d1q3_common.cuh) per launch.
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
    d1q3_site<R, DEV, SAMPLE>(d, reinterpret_cast<const R*>(ws + d.off_pop[parity]),
                              reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]),
                              SAMPLE ? reinterpret_cast<R*>(ws + d.off_fields) : nullptr, nx, x, step);
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

// Adds the per-block partials of block_sums in block order.
__global__ void k_finish_sums(const double* __restrict__ partial, int nblocks, double* __restrict__ sums,
                              DevStatus* status, int r) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < kNumSums; ++k) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[kNumSums * b + k];
    sums[k] = v;
    if (status && !isfinite(v) && status->error == 0) { status->error = FLB_EUNSTABLE; status->replica = r; }
  }
}

__global__ void k_thermal_sum(const ReplicaDesc* __restrict__ descs, int r, double* __restrict__ partial) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny;
  double acc[kNumSums] = {0, 0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double N[12];
    thermal_normals(d, (uint32_t)s, d.q, N);
    acc[0] += N[0]; acc[1] += N[1];
    if (d.q == 9) acc[2] += N[2];
  }
  block_sums(acc, partial);
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
    for (int i = 0; i < d.q && FLB_INB(d.q <= 9, 191); ++i) {
      double v = f[i];
      if (DEV) v -= feq0[kFeqW + i];      // w_i rho0
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
  double acc[kNumSums] = {0, 0, 0, 0};
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
  block_sums(acc, partial);
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

void launch_step_tc(int vec, const StepLaunch& L, bool sample, cudaStream_t st);
void launch_step_wn(int vec, const StepLaunch& L, bool sample, cudaStream_t st);

template <typename R, bool DEV, int VEC>
static void launch_d2q9_vec(const StepLaunch& L, bool sample, bool mlp, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (mlp) {
      if (L.net_engine == FLB_NET_TCGEN05) launch_step_tc(VEC, L, sample, st);
      else launch_step_wn(VEC, L, sample, st);
      return;
    }
  }
#define FLB_L(S, F) k_step_d2q9<R, DEV, VEC, S, F><<<L.grid, kStepThreads, 0, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, L.step_dev)
#define FLB_LF(F) { if (sample) FLB_L(true, F); else FLB_L(false, F); }
  const int fl = L.flavor();
  if (fl == 0) FLB_LF(0) else if (fl == 1) FLB_LF(1) else FLB_LF(2)
#undef FLB_LF
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

void launch_finish_sums(const double* partial, int nblocks, double* sums, DevStatus* status, int r,
                        cudaStream_t st) {
  k_finish_sums<<<1, 32, 0, st>>>(partial, nblocks, sums, status, r);
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
