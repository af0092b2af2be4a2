// D2Q9 step with the per-site noise-scale network evaluated by each warp on the tensor
// cores with warp-level MMAs (warp_net.cuh).
//
// The step is that of lb_step.cu (pull streaming, Eqs. 3, 5, 8, 10), with the Eq. 8
// amplitude of moment 3 + c scaled by s_c = 1 + o_c(u_x, u_y, rho - rho0) (learned
// extension, not in the paper).  Each thread owns VEC consecutive sites of a row
// (vector loads and stores); the populations of its next sites are loaded while the
// current ones are collided.  The network runs on pairs of the thread's sites: one pass
// per pair evaluates 64 sites of the warp (56 MMAs).  No block-level synchronisation
// and no tensor memory in the loop, so the warps of an SM never wait for one another.
#include <algorithm>
#include "warp_net.cuh"
#include "step_pair.cuh"

namespace flb {

// Launch shape per vector width (measured at 16384^2): the kernel keeps the network's
// weight fragments, the next sites' loads and the site-pair arithmetic in registers, so
// it runs best with the full register file per thread: vec 4 as one block of 256 threads
// per SM, vec 1 and 2 as two blocks of 128.  A block of 128 threads takes half of a
// 256-unit virtual block.
template <int VEC> struct WnShape {
  static constexpr int kThreads = VEC == 4 ? 256 : 128;
  static constexpr int kMinBlocks = VEC == 4 ? 1 : 2;
  static constexpr int kSplit = kStepThreads / kThreads;       // blocks per virtual block
};

template <int VEC, bool SAMPLE, int FL>
__global__ void __launch_bounds__(WnShape<VEC>::kThreads, WnShape<VEC>::kMinBlocks)
k_step_d2q9_wn(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
               const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_vblocks, char* __restrict__ ws, int parity,
               uint32_t step, const MlpWeights* __restrict__ mlp_w, const uint64_t* __restrict__ step_dev) {
  constexpr int kWnThreads = WnShape<VEC>::kThreads, kWnSplit = WnShape<VEC>::kSplit;
  using R = float;
  constexpr bool DEV = true, ONE = Flavor<FL>::kOne;
  __shared__ __align__(16) float scr_all[kWnThreads / 32][kWarpNetScratch];
  float* scr = scr_all[threadIdx.x >> 5];

  if (step_dev) {
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  WarpNet net;
  net.load(*mlp_w);

  // work item h: virtual block h / kWnSplit, its threads from (h % kWnSplit) kWnThreads on
  const int64_t n_items = n_vblocks * kWnSplit;
  int64_t h = blockIdx.x;
  PullRaw<R, VEC> raw;
  int r = 0;
  UnitPos u{};
  if (h < n_items) {
    const int64_t vb = h / kWnSplit;
    const int tid = (int)(h % kWnSplit) * kWnThreads + (int)threadIdx.x;
    r = ONE ? 0 : find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = ONE ? one : descs[r];
    u = unit_position(d, vb, ONE ? 0 : vb_begin[r], tid, kStepThreads, VEC);
    pull_issue<R, VEC>(reinterpret_cast<const R*>(ws + d.off_pop[parity]), (int64_t)d.nx * d.ny, d.nx, d.ny, u, raw);
  }
  for (; h < n_items; h += gridDim.x) {
    const ReplicaDesc& d = ONE ? one : descs[r];
    const int64_t plane = (int64_t)d.nx * d.ny;
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    R f[9][VEC];
    pull_finish<R, VEC>(raw, u, f);
    const UnitPos uc = u;
    // the next sites' loads, in flight while these sites are collided
    const int64_t hn = h + gridDim.x;
    if (hn < n_items) {
      const int64_t vbn = hn / kWnSplit;
      const int tid = (int)(hn % kWnSplit) * kWnThreads + (int)threadIdx.x;
      r = ONE ? 0 : find_replica(vb_begin, n_reps, vbn);
      const ReplicaDesc& dn = ONE ? one : descs[r];
      u = unit_position(dn, vbn, ONE ? 0 : vb_begin[r], tid, kStepThreads, VEC);
      pull_issue<R, VEC>(reinterpret_cast<const R*>(ws + dn.off_pop[parity]), (int64_t)dn.nx * dn.ny, dn.nx, dn.ny,
                         u, raw);
    }
    const R rho0 = coef<R>(d, kCoRho0);
    const bool noisy = d.noise_mask != 0;
    R fld[kMaxFields][VEC];
    if constexpr (VEC >= 2) {
      // site pairs (2p, 2p + 1) on the packed FP32 instructions (step_pair.cuh)
      constexpr int NP = VEC / 2;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float2 g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = make_float2(f[i][2 * p], f[i][2 * p + 1]);
        float2 sum, ux, uy;
        macro_pair(g, rho0, sum, ux, uy);
        // the Philox words of both sites: three calls (independent integer work the
        // scheduler can place between the network's dependent MMAs; drawn even without
        // noise, then unused)
        const uint32_t site = (uint32_t)uc.y * (uint32_t)d.nx + (uint32_t)(uc.x0 + 2 * p);
        uint4 w0a, w1a, w0b, w1b;
        philox_words_pair(d, site, step, w0a, w1a, w0b, w1b);
        const uint32_t x[4] = {wn_pack2(ux.x, uy.x), wn_pack2(ux.y, uy.y), wn_pack2(sum.x, 1.f), wn_pack2(sum.y, 1.f)};
        float s0[6], s1[6];
        net.forward(x, scr, s0, s1);
        float2 sc[6], nrm[6], D[6], fl[kMaxFields];
#pragma unroll
        for (int c = 0; c < 6; ++c) sc[c] = make_float2(s0[c], s1[c]);
        normals_pair(w0a, w1a, w0b, w1b, nrm);
        relax_pair<SAMPLE>(d, g, sum, ux, uy, D, fl);
        apply_pair<Flavor<FL>::kGen>(d, g, sum, noisy, nrm, sc, D);
#pragma unroll
        for (int i = 0; i < 9; ++i) { f[i][2 * p] = g[i].x; f[i][2 * p + 1] = g[i].y; }
        if constexpr (SAMPLE) {
#pragma unroll
          for (int a = 0; a < kMaxFields; ++a) { fld[a][2 * p] = fl[a].x; fld[a][2 * p + 1] = fl[a].y; }
        }
      }
    } else {
      // one site: the second row of the network's tile repeats it
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][0];
      R sum, ux, uy;
      macro_d2q9<R, DEV>(g, rho0, sum, ux, uy);
      uint4 w0, w1;
      philox_words_d2q9(d, (uint32_t)uc.y * (uint32_t)d.nx + (uint32_t)uc.x0, step, w0, w1);
      const uint32_t x[4] = {wn_pack2(ux, uy), wn_pack2(ux, uy), wn_pack2(sum, 1.f), wn_pack2(sum, 1.f)};
      float sc[6], s1[6];
      net.forward(x, scr, sc, s1);
      R nrm[6], Drel[6], fl[kMaxFields];
      normals_from_words<R>(w0, w1, nrm);
      collide_relax<R, DEV, SAMPLE>(d, g, sum, ux, uy, Drel, fl);
      collide_apply<R, DEV, Flavor<FL>::kGen>(d, g, sum, noisy, nrm, sc, Drel);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][0] = g[i];
      if constexpr (SAMPLE) {
#pragma unroll
        for (int a = 0; a < kMaxFields; ++a) fld[a][0] = fl[a];
      }
    }
    store_d2q9<R, VEC, SAMPLE>(d, ws, dst, plane, uc, f, fld);
  }
}

template <int VEC>
static void launch_wn_vec(const StepLaunch& L, bool sample, cudaStream_t st) {
  auto w = reinterpret_cast<const MlpWeights*>(L.mlp);
  // the grid counts 256-thread blocks; kSplit blocks of kThreads take each one's place
  constexpr int kSplit = WnShape<VEC>::kSplit;
  const int grid = (int)std::min<int64_t>((int64_t)L.grid * kSplit, L.n_vblocks * kSplit);
#define FLB_L(S, F) k_step_d2q9_wn<VEC, S, F><<<grid, WnShape<VEC>::kThreads, 0, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w, L.step_dev)
#define FLB_LF(F) { if (sample) FLB_L(true, F); else FLB_L(false, F); }
  const int fl = L.flavor();
  if (fl == 0) FLB_LF(0) else if (fl == 1) FLB_LF(1) else FLB_LF(2)
#undef FLB_LF
#undef FLB_L
}

void launch_step_wn(int vec, const StepLaunch& L, bool sample, cudaStream_t st) {
  if (vec == 4) launch_wn_vec<4>(L, sample, st);
  else if (vec == 2) launch_wn_vec<2>(L, sample, st);
  else launch_wn_vec<1>(L, sample, st);
}

}  // namespace flb
