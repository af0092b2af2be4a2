// D2Q9 step with the per-site noise-scale network on the fifth-generation tensor
// cores (tcgen05 MMA, operand A and the accumulators in tensor memory).
//
// The step is that of lb_step.cu (pull streaming, Eqs. 3, 5, 8, 10), with the
// Eq. 8 amplitude of moment 3 + c scaled by s_c = 1 + o_c(u_x, u_y, rho - rho0),
// o = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (3 -> 32 -> 32 -> 6; learned extension,
// not in the paper).  bfloat16 operands (inputs, weights, biases, activations),
// FP32 accumulation.
//
// LDG variant (any even nx): each thread's VEC sites are consecutive in a row, loaded
// with vector loads; the populations of the thread's next sites are loaded while the
// network of the current ones runs, and the Philox normals are drawn while layer 1
// runs.  The network itself (tc_common.cuh) keeps its operands in tensor memory.
// Every mbarrier wait is bounded; on a timeout the kernel records FLB_ETIMEOUT and
// carries on (no hang), and tensor memory is always freed.
#include <algorithm>
#include "tc_common.cuh"

namespace flb {

// ONE: a single replica, whose description is the kernel argument `one` (read through
// the constant bank) instead of descs[0] in global memory.
template <int VEC, bool SAMPLE, int FL>
__global__ void __launch_bounds__(kStepThreads, TcOcc<VEC>::kMinBlocks)
k_step_d2q9_tc(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
               const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_vblocks, char* __restrict__ ws, int parity,
               uint32_t step, const MlpWeights* __restrict__ mlp_w, const uint64_t* __restrict__ step_dev,
               DevStatus* status) {
  using R = float;
  constexpr bool DEV = true, ONE = Flavor<FL>::kOne;
  static_assert(kStepThreads == 256, "two warpgroups per block");
  constexpr uint32_t kCols = 2 * VEC * kTileCols;                    // 128, 256 or 512 columns
  __shared__ __align__(128) unsigned char sb[kBBytes];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  unsigned char* sb1 = sb;
  unsigned char* sb2 = sb1 + kB1Bytes;
  unsigned char* sb3 = sb2 + kB2Bytes;

  if (step_dev) {
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  const int tid = (int)threadIdx.x, warp = tid >> 5;
  build_b_tiles(*mlp_w, sb1, sb2, sb3);
  if (warp == 0) tmem_alloc<kCols>(&tmem_slot);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  TcNet<VEC> net;
  net.init(tmem_slot, sb1, sb2, sb3, &mbar[tid >> 7]);

  int64_t vb = blockIdx.x;
  PullRaw<R, VEC> raw;
  int r = 0;
  UnitPos u{};
  if (vb < n_vblocks) {
    r = ONE ? 0 : find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = ONE ? one : descs[r];
    u = unit_position(d, vb, ONE ? 0 : vb_begin[r], tid, kStepThreads, VEC);
    pull_issue<R, VEC>(reinterpret_cast<const R*>(ws + d.off_pop[parity]), (int64_t)d.nx * d.ny, d.nx, d.ny, u, raw);
  }
  for (; vb < n_vblocks; vb += gridDim.x) {
    const ReplicaDesc& d = ONE ? one : descs[r];
    const int64_t plane = (int64_t)d.nx * d.ny;
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    R f[9][VEC];
    pull_finish<R, VEC>(raw, u, f);
    const UnitPos uc = u;
    // the next sites' loads, in flight while the network runs
    const int64_t vbn = vb + gridDim.x;
    if (vbn < n_vblocks) {
      r = ONE ? 0 : find_replica(vb_begin, n_reps, vbn);
      const ReplicaDesc& dn = ONE ? one : descs[r];
      u = unit_position(dn, vbn, ONE ? 0 : vb_begin[r], tid, kStepThreads, VEC);
      pull_issue<R, VEC>(reinterpret_cast<const R*>(ws + dn.off_pop[parity]), (int64_t)dn.nx * dn.ny, dn.nx, dn.ny,
                         u, raw);
    }
    const R rho0 = coef<R>(d, kCoRho0);
    const bool noisy = d.noise_mask != 0;
    R sum[VEC], ux[VEC], uy[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      macro_d2q9<R, DEV>(g, rho0, sum[v], ux[v], uy[v]);
    }
    // independent work fills the three MMA round trips: the Philox words while layer 1
    // runs, the Box-Muller transform during layer 2, the relaxation during layer 3
    net.start(ux, uy, sum);
    uint4 w0[VEC], w1[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (noisy) philox_words_d2q9(d, (uint32_t)uc.y * (uint32_t)d.nx + (uint32_t)(uc.x0 + v), step, w0[v], w1[v]);
    net.template next_layer<2>();
    R nrm[VEC][6];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
#pragma unroll
      for (int c = 0; c < 6; ++c) nrm[v][c] = (R)0;
      if (noisy) normals_from_words<R>(w0[v], w1[v], nrm[v]);
    }
    net.template next_layer<3>();
    R Drel[VEC][6];
    R fld[kMaxFields][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      R fl[kMaxFields];
      collide_relax<R, DEV, SAMPLE>(d, g, sum[v], ux[v], uy[v], Drel[v], fl);
      if constexpr (SAMPLE) {
#pragma unroll
        for (int a = 0; a < kMaxFields; ++a) fld[a][v] = fl[a];
      }
    }
    R sc[VEC][6];
    net.scales(sc);
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      collide_apply<R, DEV, Flavor<FL>::kGen>(d, g, sum[v], noisy, nrm[v], sc[v], Drel[v]);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][v] = g[i];
    }
    store_d2q9<R, VEC, SAMPLE>(d, ws, dst, plane, uc, f, fld);
  }
  if (!net.ok && atomicCAS(&status->error, 0, FLB_ETIMEOUT) == 0) status->replica = -1;
  net.drain();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) tmem_free<kCols>(tmem_slot);
}

template <int VEC>
static void launch_tc_vec(const StepLaunch& L, bool sample, cudaStream_t st) {
  // no more blocks than the tensor memory of the SMs holds at once (blocks beyond that
  // would wait in tcgen05.alloc for a resident one to finish)
  int grid = L.grid;
  if (L.sms > 0) grid = (int)std::min<int64_t>((int64_t)grid, (int64_t)L.sms * TcOcc<VEC>::kBlocks);
  auto w = reinterpret_cast<const MlpWeights*>(L.mlp);
#define FLB_L(S, F) k_step_d2q9_tc<VEC, S, F><<<grid, kStepThreads, 0, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w, L.step_dev, L.status)
#define FLB_LF(F) { if (sample) FLB_L(true, F); else FLB_L(false, F); }
  const int fl = L.flavor();
  if (fl == 0) FLB_LF(0) else if (fl == 1) FLB_LF(1) else FLB_LF(2)
#undef FLB_LF
#undef FLB_L
}

// Diagnostic: one bounded wait (the network kernels' mbar_wait, with a shorter limit) on
// an mbarrier that nothing arrives at, reported through the status word the way a step
// kernel reports an MMA or a copy that never completed.  No asynchronous operation is
// involved, so giving up leaves nothing in flight.
__global__ void k_wait_probe(DevStatus* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit) && atomicCAS(&status->error, 0, FLB_ETIMEOUT) == 0)
    status->replica = -2;
}

void launch_wait_probe(DevStatus* status, long long limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, limit);
}

void launch_step_tc(int vec, const StepLaunch& L, bool sample, cudaStream_t st) {
  if (vec == 4) launch_tc_vec<4>(L, sample, st);
  else if (vec == 2) launch_tc_vec<2>(L, sample, st);
  else launch_tc_vec<1>(L, sample, st);
}

}  // namespace flb
