// Staged FP32 D2Q9 step: the populations move between HBM and shared memory by TMA
// bulk copies (cp.async.bulk), so the threads only touch shared memory.
//
// The step is that of lb_step.cu (pull streaming, Eqs. 1, 3, 5, 8, 10), optionally
// with the per-site noise-scale network of tc_common.cuh (NET).
//
// Work unit: a tile = row y, columns [x0, x0 + Wt) of one replica, Wt <= W = 256 VEC
// (nx a multiple of 4).  Pull streaming takes population i from row y - v_iy only, at
// columns x - v_ix, so a tile needs, per population, one row segment plus a 4-column
// halo on the side v_ix points away from (16-byte copies; periodic in x and y):
// 9 segment copies and 6 halo copies, all 16-byte aligned.  A persistent block
// walks its tiles through kStages input stages (full/empty mbarriers; warp 0 issues
// the copies kStages - 1 tiles ahead, one copy per lane).  Warpgroup g owns the sites [g W/2, (g+1) W/2)
// of a tile (thread t: sites g W/2 + 128 v + t, v < VEC), writes its post-collision
// populations to its own double-buffered output area, and its lanes 0..8 store them
// back with bulk copies (lane i: population i; one bulk group per lane and tile).  Shared-memory reads and writes
// are consecutive across a warp (no bank conflicts); global memory sees only bulk
// copies, except the sampled fields, which are stored directly.
//
// Every mbarrier wait is bounded (the first one to give up makes the thread skip
// the rest, so a lost copy cannot stall the launch), and a timeout is reported as
// FLB_ETIMEOUT; tensor memory is always freed and all bulk stores are waited for.
#include <algorithm>
#include "tc_common.cuh"

namespace flb {

constexpr int kStages = 3;

template <int VEC>
struct BulkGeom {
  static constexpr int W = 256 * VEC;                      // sites per tile
  static constexpr int SEG = W + 8;                        // floats per population segment (4-float halos)
  static constexpr int HALF = 128 * VEC;                   // sites per warpgroup
  static constexpr uint32_t kInBytes = 9u * SEG * 4;       // one input stage
  static constexpr uint32_t kOutBytes = 9u * HALF * 4;     // one output buffer of one warpgroup
  static constexpr uint32_t kBOff = 1024;                  // [0, 1024): mbarriers, tensor-memory slot
  static constexpr uint32_t kInOff = kBOff + ((kBBytes + 127) / 128) * 128;
  static constexpr uint32_t kOutOff = kInOff + kStages * kInBytes;
  static constexpr uint32_t kSmem = kOutOff + 4 * kOutBytes;   // 2 warpgroups x 2 buffers
};

// Resident blocks per SM: tensor memory (network), shared memory (228 KB per SM, 1 KB
// reserved per block), and at most 3 (85 registers a thread).
template <int VEC, bool NET>
struct BulkOcc {
  static constexpr int kSmemBlocks = 233472 / (BulkGeom<VEC>::kSmem + 1024);
  static constexpr int kTmemBlocks = NET ? TcOcc<VEC>::kBlocks : 8;
  static constexpr int kA = kSmemBlocks < kTmemBlocks ? kSmemBlocks : kTmemBlocks;
  static constexpr int kBlocks = kA < 3 ? kA : 3;
};

// 16-byte aligned global -> shared bulk copy completing on an mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// shared -> global bulk copy in the thread's current bulk group
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(dst), "r"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" :: "n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

struct TilePos {
  int r, y, x0, wt;
};

template <int VEC, bool ONE>
__device__ __forceinline__ TilePos tile_position(const ReplicaDesc* descs, const ReplicaDesc& one,
                                                 const int64_t* vb_begin, int n_reps, int64_t T) {
  TilePos p;
  p.r = ONE ? 0 : find_replica(vb_begin, n_reps, T);
  const ReplicaDesc& d = ONE ? one : descs[p.r];
  const uint32_t unit = (uint32_t)(T - (ONE ? 0 : vb_begin[p.r]));
  p.y = (int)(((uint64_t)unit * d.upr_magic) >> d.upr_shift);
  p.x0 = (int)(unit - (uint32_t)p.y * (uint32_t)d.units_per_row) * BulkGeom<VEC>::W;
  p.wt = min(BulkGeom<VEC>::W, d.nx - p.x0);
  return p;
}

// Warp 0: the copies of a tile into input stage `in`, all completing on `full`, one per
// lane (a bulk copy takes long to issue, so the lanes issue them side by side).  Lanes
// 0..8: population i = lane, row y - v_iy, columns [x0, x0 + wt) -> segment i at 4;
// lanes 9..11: the left halo (columns x0 - 4 .. x0 - 1) of i = 1, 5, 8 (v_ix = +1) ->
// segment i at 0; lanes 12..14: the right halo (x0 + wt .. x0 + wt + 3) of i = 3, 6, 7.
template <int VEC>
__device__ __forceinline__ void issue_tile(const ReplicaDesc& d, const TilePos& p, const char* ws, int parity,
                                           float* in, uint64_t* full, int lane) {
  using G = BulkGeom<VEC>;
  const int nx = d.nx, ny = d.ny, x0 = p.x0, wt = p.wt;
  if (lane == 0) mbar_expect_tx(full, 9u * (uint32_t)wt * 4u + 6u * 16u);
  __syncwarp();
  if (lane < 15) {
    const int i = lane < 9 ? lane : (lane < 12 ? (lane == 9 ? 1 : (lane == 10 ? 5 : 8)) : (lane == 12 ? 3 : (lane == 13 ? 6 : 7)));
    int ys = p.y - vel_y(i);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    const float* row = reinterpret_cast<const float*>(ws + d.off_pop[parity]) + i * ((int64_t)nx * ny) + (int64_t)ys * nx;
    const uint32_t seg = smem_u32(in + i * G::SEG);
    if (lane < 9) bulk_g2s(seg + 16u, row + x0, (uint32_t)wt * 4u, full);
    else if (lane < 12) bulk_g2s(seg, row + (x0 == 0 ? nx - 4 : x0 - 4), 16u, full);
    else bulk_g2s(seg + 16u + (uint32_t)wt * 4u, row + (x0 + wt == nx ? 0 : x0 + wt), 16u, full);
  }
}

template <int VEC, bool SAMPLE, int FL, bool NET>
__global__ void __launch_bounds__(kStepThreads, (BulkOcc<VEC, NET>::kBlocks))
k_step_d2q9_bulk(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
                 const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_tiles, char* __restrict__ ws,
                 int parity, uint32_t step, const MlpWeights* __restrict__ mlp_w,
                 const uint64_t* __restrict__ step_dev, DevStatus* status) {
  using G = BulkGeom<VEC>;
  using R = float;
  constexpr bool ONE = Flavor<FL>::kOne;
  static_assert(kStepThreads == 256, "two warpgroups per block");
  constexpr uint32_t kCols = 2 * VEC * kTileCols;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);          // [kStages]
  uint64_t* empty = full + kStages;                              // [kStages]
  uint64_t* mma_bar = empty + kStages;                           // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 256);
  unsigned char* sb1 = smem + G::kBOff;
  unsigned char* sb2 = sb1 + kB1Bytes;
  unsigned char* sb3 = sb2 + kB2Bytes;
  float* in_base = reinterpret_cast<float*>(smem + G::kInOff);
  float* out_base = reinterpret_cast<float*>(smem + G::kOutOff);

  if (step_dev) {
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  const int tid = (int)threadIdx.x, warp = tid >> 5, wg = tid >> 7, tw = tid & 127;
  if constexpr (NET) {
    build_b_tiles(*mlp_w, sb1, sb2, sb3);
    if (warp == 0) tmem_alloc<kCols>(tmem_slot);
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kStepThreads);
    }
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  TcNet<VEC> net;
  if constexpr (NET) net.init(*tmem_slot, sb1, sb2, sb3, &mma_bar[wg]);
  bool ok = true;

  const int64_t T0 = blockIdx.x, stride = gridDim.x;
  if (warp == 0) {                       // prologue: the first kStages - 1 tiles
    for (int k = 0; k < kStages - 1; ++k) {
      const int64_t T = T0 + k * stride;
      if (T < n_tiles) {
        const TilePos p = tile_position<VEC, ONE>(descs, one, vb_begin, n_reps, T);
        issue_tile<VEC>(ONE ? one : descs[p.r], p, ws, parity, in_base + k * 9 * G::SEG, &full[k], tid);
      }
    }
  }
  int k = 0;
  for (int64_t T = T0; T < n_tiles; T += stride, ++k) {
    const int s = k % kStages;
    const uint32_t use = (uint32_t)(k / kStages);
    if (warp == 0) {                     // producer: tile k + kStages - 1 into the stage tile k - 1 used
      const int64_t Tn = T + (int64_t)(kStages - 1) * stride;
      if (Tn < n_tiles) {
        const int kn = k + kStages - 1, sn = kn % kStages;
        if (ok) ok = mbar_wait(&empty[sn], (uint32_t)(kn / kStages - 1) & 1u);
        const TilePos pn = tile_position<VEC, ONE>(descs, one, vb_begin, n_reps, Tn);
        issue_tile<VEC>(ONE ? one : descs[pn.r], pn, ws, parity, in_base + sn * 9 * G::SEG, &full[sn], tid);
      }
    }
    const TilePos p = tile_position<VEC, ONE>(descs, one, vb_begin, n_reps, T);
    const ReplicaDesc& d = ONE ? one : descs[p.r];
    const int nx = d.nx;
    // ---- read the pulled populations of this thread's sites ------------------
    if (tw < 32 && ok) ok = mbar_wait(&full[s], use & 1u);    // one warp polls, the others wait for it
    wg_barrier(wg);
    const float* in = in_base + s * 9 * G::SEG;
    R f[9][VEC];
    int lx[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      lx[v] = wg * G::HALF + 128 * v + tw;
      const int l = min(lx[v], p.wt - 1);            // idle lanes of a short tile read a valid site
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][v] = in[i * G::SEG + 4 + l - vel_x(i)];
    }
    mbar_arrive(&empty[s]);
    const R rho0 = coef<R>(d, kCoRho0);
    const bool noisy = d.noise_mask != 0;
    R sum[VEC], ux[VEC], uy[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      macro_d2q9<R, true>(g, rho0, sum[v], ux[v], uy[v]);
    }
    if constexpr (NET) net.start(ux, uy, sum);
    R nrm[VEC][6];
    const uint32_t site0 = (uint32_t)p.y * (uint32_t)nx + (uint32_t)p.x0;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
#pragma unroll
      for (int c = 0; c < 6; ++c) nrm[v][c] = (R)0;
      if (noisy) normals_d2q9<R>(d, site0 + (uint32_t)lx[v], step, nrm[v]);
    }
    // this tile's output buffer is free once the bulk stores of tile k - 2 have read it
    R sc[VEC][6];
    if constexpr (NET) {
      net.finish(sc, [&] { if (tw < 9) bulk_wait_read<1>(); });
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int c = 0; c < 6; ++c) sc[v][c] = (R)1;
      if (tw < 9) bulk_wait_read<1>();
      wg_barrier(wg);
    }
    // ---- collide, write the populations to the output buffer ----------------
    float* out = out_base + (wg * 2 + (k & 1)) * 9 * G::HALF;
    const int64_t plane = (int64_t)nx * d.ny;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      R fl[kMaxFields];
      collide_d2q9<R, true, SAMPLE, Flavor<FL>::kGen>(d, g, sum[v], ux[v], uy[v], noisy, nrm[v], sc[v], fl);
#pragma unroll
      for (int i = 0; i < 9; ++i) out[i * G::HALF + 128 * v + tw] = g[i];
      if constexpr (SAMPLE) {
        if (lx[v] < p.wt) {
          R* fields = reinterpret_cast<R*>(ws + d.off_fields) + (int64_t)p.y * nx + p.x0 + lx[v];
          for (int slot = 0; slot < (int)d.n_fields; ++slot) {
            const int fid = d.field_id[slot];
            R val = fl[0];
#pragma unroll
            for (int a = 1; a < kMaxFields; ++a) val = (fid == a) ? fl[a] : val;
            fields[slot * plane] = val;
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    wg_barrier(wg);
    if (tw < 9) {                        // this warpgroup's part of the tile: lane i stores population i
      const int n = min(G::HALF, p.wt - wg * G::HALF);
      if (n > 0) {
        R* dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]) + tw * plane + (int64_t)p.y * nx + p.x0 + wg * G::HALF;
        bulk_s2g(dst, smem_u32(out + tw * G::HALF), (uint32_t)n * 4u);
      }
      bulk_commit();                     // one bulk group per lane and tile
    }
  }
  if (tw < 9) bulk_wait_all();
  const bool bad = __syncthreads_or(!ok);
  if (tid == 0 && bad) {                 // after a timeout: wait (bounded) for copies still in flight
    // (every issued tile was walked by the loop; the last kStages may not have landed)
    for (int j = k > kStages ? k - kStages : 0; j < k; ++j) mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
  }
  if (!(ok && (!NET || net.ok)) && atomicCAS(&status->error, 0, FLB_ETIMEOUT) == 0) status->replica = -1;
  if constexpr (NET) {
    net.drain();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) tmem_free<kCols>(*tmem_slot);
  }
}

template <int VEC, bool NET>
static void launch_bulk_vec(const StepLaunch& L, bool sample, cudaStream_t st) {
  using G = BulkGeom<VEC>;
  static bool attr = false;
  if (!attr) {
#define FLB_A(S, F) cudaFuncSetAttribute(k_step_d2q9_bulk<VEC, S, F, NET>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmem)
    FLB_A(false, 0); FLB_A(true, 0); FLB_A(false, 1); FLB_A(true, 1); FLB_A(false, 2); FLB_A(true, 2);
#undef FLB_A
    attr = true;
  }
  // a persistent grid of resident blocks
  int grid = L.grid;
  if (L.sms > 0) grid = (int)std::min<int64_t>((int64_t)grid, (int64_t)L.sms * BulkOcc<VEC, NET>::kBlocks);
  auto w = reinterpret_cast<const MlpWeights*>(L.mlp);
#define FLB_L(S, F) k_step_d2q9_bulk<VEC, S, F, NET><<<grid, kStepThreads, G::kSmem, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w, L.step_dev, L.status)
#define FLB_LF(F) { if (sample) FLB_L(true, F); else FLB_L(false, F); }
  const int fl = L.flavor();
  if (fl == 0) FLB_LF(0) else if (fl == 1) FLB_LF(1) else FLB_LF(2)
#undef FLB_LF
#undef FLB_L
}

void launch_step_bulk(int vec, const StepLaunch& L, bool sample, bool mlp, cudaStream_t st) {
  if (mlp) {
    if (vec == 4) launch_bulk_vec<4, true>(L, sample, st);
    else if (vec == 2) launch_bulk_vec<2, true>(L, sample, st);
    else launch_bulk_vec<1, true>(L, sample, st);
  } else {
    if (vec == 4) launch_bulk_vec<4, false>(L, sample, st);
    else if (vec == 2) launch_bulk_vec<2, false>(L, sample, st);
    else launch_bulk_vec<1, false>(L, sample, st);
  }
}

}  // namespace flb
