// D2Q9 step with the per-site noise-scale network on the fifth-generation tensor
// cores (tcgen05 MMA, operand A and the accumulators in tensor memory).
//
// The step is that of lb_step.cu (pull streaming, Eqs. 3, 5, 8, 10), with the
// Eq. 8 amplitude of moment 3 + c scaled by s_c = 1 + o_c(u_x, u_y, rho - rho0),
// o = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (3 -> 32 -> 32 -> 6; learned extension,
// not in the paper).  bfloat16 operands (inputs, weights, biases, activations),
// FP32 accumulation.
//
// Mapping: each warpgroup (128 threads) owns tensor-memory lanes 0..127; thread t
// of the warpgroup and its v-th site (v < VEC) form row t of tile v.  A tile has 64
// tensor-memory columns: D (32 FP32 columns) and A (24 columns = 48 bfloat16 of K,
// packed two per column).  Per layer the threads write their rows of A with
// tcgen05.st, one thread issues the MMAs (B, the weights, in shared memory) and
// commits them to the warpgroup's mbarrier, and every thread reads its row of D
// back with tcgen05.ld, applies relu and rounds to bfloat16 into A for the next
// layer.  Biases enter through a constant-1 column of A (K index 3 in layer 1, 32
// in layers 2 and 3; columns 16..23 of A are written once).  The populations of the
// thread's next sites are loaded while the network of the current ones runs, and
// the Philox normals are drawn while layer 1 runs.  Every mbarrier wait is bounded;
// on a timeout the kernel records FLB_ETIMEOUT and carries on (no hang), and tensor
// memory is always freed.
#include <algorithm>
#include "step_common.cuh"

namespace flb {

constexpr int kTcK1 = 16;                 // layer 1: x0, x1, x2, 1, zeros
constexpr int kTcK = 48;                  // layers 2, 3: 32 activations, 1, zeros
constexpr uint32_t kTileCols = 64;        // tensor-memory columns per tile
constexpr uint32_t kB1Bytes = 32 * kTcK1 * 2, kB2Bytes = 32 * kTcK * 2, kB3Bytes = 16 * kTcK * 2;
constexpr uint32_t kBBytes = kB1Bytes + kB2Bytes + kB3Bytes;   // 5632
constexpr int kWaitHintNs = 1000000;       // suspend-time hint of one mbarrier poll

// byte offset of element (row, k) in a K-major tile of K columns built from 8x8 core matrices
__host__ __device__ constexpr uint32_t core_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle; LBO = stride between core matrices along K,
// SBO = stride between 8-row groups; bits 46-48 = 0b001
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  return (uint32_t)*reinterpret_cast<const unsigned short*>(&h);
}

// round to bfloat16 and pack (lo in the low half)
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// relu, round to bfloat16 and pack
__device__ __forceinline__ uint32_t relu_pack2(uint32_t lo, uint32_t hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
  return d;
}

// D[tmem_d] (+)= A[tmem_a] B[desc_b]
__device__ __forceinline__ void mma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
               :: "r"(tmem_d), "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(bar)));
}

// bounded wait for the mbarrier phase with the given parity; false on timeout
// (each try_wait may suspend the thread for up to kWaitHintNs until the phase completes;
// the whole wait gives up after 2^32 SM clocks, about two seconds)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "n"(kWaitHintNs));
    if (done) return true;
    if (clock64() - t0 > (1LL << 32)) return false;
  }
}

__device__ __forceinline__ void wg_barrier(int wg) { asm volatile("bar.sync %0, 128;" :: "r"(1 + wg)); }

__device__ __forceinline__ void tmem_st8(uint32_t a, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                         uint32_t r5, uint32_t r6, uint32_t r7) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "r"(a), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(r4), "r"(r5), "r"(r6), "r"(r7));
}

__device__ __forceinline__ void tmem_st16(uint32_t a, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               :: "r"(a), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                  "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}

// load and wait in one statement, so the outputs are complete when the compiler sees them
__device__ __forceinline__ void tmem_ld16(uint32_t a, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(a));
}

__device__ __forceinline__ void tmem_ld8(uint32_t a, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(a));
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }

// D row (32 FP32 columns at tmem address d) -> relu -> bfloat16 -> A row columns 0..15
__device__ __forceinline__ void hidden_to_a(uint32_t d, uint32_t a) {
  uint32_t p[16];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t h[16];
    tmem_ld16(d + 16 * half, h);
#pragma unroll
    for (int j = 0; j < 8; ++j) p[8 * half + j] = relu_pack2(h[2 * j], h[2 * j + 1]);
  }
  tmem_st16(a, p);
}

// B operands (weights with the bias in the constant-1 column), bfloat16, K-major.
__device__ void build_b_tiles(const MlpWeights& w, unsigned char* b1, unsigned char* b2, unsigned char* b3) {
  for (int i = threadIdx.x; i < 32 * kTcK1; i += blockDim.x) {
    const int n = i / kTcK1, k = i % kTcK1;
    const float v = k < 3 ? w.W1[3 * n + k] : (k == 3 ? w.b1[n] : 0.f);
    *reinterpret_cast<unsigned short*>(b1 + core_off(n, k, kTcK1)) = (unsigned short)bf16_bits(v);
  }
  for (int i = threadIdx.x; i < 32 * kTcK; i += blockDim.x) {
    const int n = i / kTcK, k = i % kTcK;
    const float v = k < 32 ? w.W2[kMlpHidden * n + k] : (k == 32 ? w.b2[n] : 0.f);
    *reinterpret_cast<unsigned short*>(b2 + core_off(n, k, kTcK)) = (unsigned short)bf16_bits(v);
  }
  for (int i = threadIdx.x; i < 16 * kTcK; i += blockDim.x) {
    const int n = i / kTcK, k = i % kTcK;
    const float v = n < kMlpOut ? (k < 32 ? w.W3[kMlpHidden * n + k] : (k == 32 ? w.b3[n] : 0.f)) : 0.f;
    *reinterpret_cast<unsigned short*>(b3 + core_off(n, k, kTcK)) = (unsigned short)bf16_bits(v);
  }
}

// Resident blocks per SM: tensor memory (512 columns) holds 2 * VEC tiles of 64 per block.
template <int VEC> struct TcOcc {
  static constexpr int kBlocks = 512 / (2 * VEC * (int)kTileCols);
  static constexpr int kMinBlocks = kBlocks < 3 ? kBlocks : 3;      // register cap of the launch bounds
};

// ONE: a single replica, whose description is the kernel argument `one` (read through
// the constant bank) instead of descs[0] in global memory.
template <int VEC, bool SAMPLE, bool ONE>
__global__ void __launch_bounds__(kStepThreads, TcOcc<VEC>::kMinBlocks)
k_step_d2q9_tc(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
               const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_vblocks, char* __restrict__ ws, int parity,
               uint32_t step, const MlpWeights* __restrict__ mlp_w, const uint64_t* __restrict__ step_dev,
               DevStatus* status) {
  using R = float;
  constexpr bool DEV = true;
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
  const int tid = (int)threadIdx.x, warp = tid >> 5, wg = tid >> 7, tw = tid & 127;
  build_b_tiles(*mlp_w, sb1, sb2, sb3);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_slot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  // tile v of this warpgroup: D at columns [64 v, 64 v + 32), A at [64 v + 32, 64 v + 56)
  const uint32_t tbase = tmem_slot + (uint32_t)(wg * VEC) * kTileCols;
  const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's lanes
#pragma unroll
  for (int v = 0; v < VEC; ++v)        // constant columns 16..23 of A: (1, 0), zeros
    tmem_st8(trow + v * kTileCols + 32 + 16, 0x3F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u);
  tmem_wait_st();
  constexpr uint32_t id32 = instr_desc(128, 32), id16 = instr_desc(128, 16);
  const uint64_t db1 = smem_desc(smem_u32(sb1), kTcK1 / 8 * 128);
  const uint64_t db2 = smem_desc(smem_u32(sb2), kTcK / 8 * 128);
  const uint64_t db3 = smem_desc(smem_u32(sb3), kTcK / 8 * 128);
  uint32_t ph = 0;
  bool ok = true;

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
      // layer-1 row of A: (u_x, u_y, rho - rho0, 1, 0, ...)
      tmem_st8(trow + v * kTileCols + 32, pack2(ux[v], uy[v]), pack2(sum[v], 1.f), 0u, 0u, 0u, 0u, 0u, 0u);
    }
    tmem_wait_st();
    // ---- layer 1 -----------------------------------------------------------
    asm volatile("tcgen05.fence::before_thread_sync;");
    wg_barrier(wg);
    if (tw == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int v = 0; v < VEC; ++v) mma_ts(tbase + v * kTileCols, tbase + v * kTileCols + 32, db1, id32, 0u);
      mma_commit(&mbar[wg]);
    }
    // the normals meanwhile
    R nrm[VEC][6];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
#pragma unroll
      for (int c = 0; c < 6; ++c) nrm[v][c] = (R)0;
      if (noisy) normals_d2q9<R>(d, (uint32_t)uc.y * (uint32_t)d.nx + (uint32_t)(uc.x0 + v), step, nrm[v]);
    }
    if (ok) ok = mbar_wait(&mbar[wg], ph);
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
    for (int v = 0; v < VEC; ++v) hidden_to_a(trow + v * kTileCols, trow + v * kTileCols + 32);
    tmem_wait_st();
    // ---- layer 2 -----------------------------------------------------------
    asm volatile("tcgen05.fence::before_thread_sync;");
    wg_barrier(wg);
    if (tw == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk)     // K step: 16 bf16 = 256 B of B, 8 columns of A
          mma_ts(tbase + v * kTileCols, tbase + v * kTileCols + 32 + 8 * kk, db2 + (uint64_t)(kk * 256 >> 4), id32,
                 kk > 0 ? 1u : 0u);
      mma_commit(&mbar[wg]);
    }
    if (ok) ok = mbar_wait(&mbar[wg], ph);
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
    for (int v = 0; v < VEC; ++v) hidden_to_a(trow + v * kTileCols, trow + v * kTileCols + 32);
    tmem_wait_st();
    // ---- layer 3 -----------------------------------------------------------
    asm volatile("tcgen05.fence::before_thread_sync;");
    wg_barrier(wg);
    if (tw == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk)
          mma_ts(tbase + v * kTileCols, tbase + v * kTileCols + 32 + 8 * kk, db3 + (uint64_t)(kk * 256 >> 4), id16,
                 kk > 0 ? 1u : 0u);
      mma_commit(&mbar[wg]);
    }
    if (ok) ok = mbar_wait(&mbar[wg], ph);
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- collision with the scales -----------------------------------------
    R fld[kMaxFields][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      uint32_t o[8];
      tmem_ld8(trow + v * kTileCols, o);
      R sc[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) sc[c] = (R)1 + __uint_as_float(o[c]);
      R g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = f[i][v];
      R fl[kMaxFields];
      collide_d2q9<R, DEV, SAMPLE>(d, g, sum[v], ux[v], uy[v], noisy, nrm[v], sc, fl);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][v] = g[i];
      if constexpr (SAMPLE) {
#pragma unroll
        for (int a = 0; a < kMaxFields; ++a) fld[a][v] = fl[a];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    store_d2q9<R, VEC, SAMPLE>(d, ws, dst, plane, uc, f, fld);
  }
  if (!ok && atomicCAS(&status->error, 0, FLB_ETIMEOUT) == 0) status->replica = -1;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_slot), "r"(kCols));
}

template <int VEC>
static void launch_tc_vec(const StepLaunch& L, bool sample, cudaStream_t st) {
  // no more blocks than the tensor memory of the SMs holds at once (blocks beyond that
  // would wait in tcgen05.alloc for a resident one to finish)
  int grid = L.grid;
  if (L.sms > 0) grid = (int)std::min<int64_t>((int64_t)grid, (int64_t)L.sms * TcOcc<VEC>::kBlocks);
  auto w = reinterpret_cast<const MlpWeights*>(L.mlp);
#define FLB_L(S, O) k_step_d2q9_tc<VEC, S, O><<<grid, kStepThreads, 0, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, w, L.step_dev, L.status)
  if (L.n_reps == 1) { if (sample) FLB_L(true, true); else FLB_L(false, true); }
  else { if (sample) FLB_L(true, false); else FLB_L(false, false); }
#undef FLB_L
}

void launch_step_tc(int vec, const StepLaunch& L, bool sample, cudaStream_t st) {
  if (vec == 4) launch_tc_vec<4>(L, sample, st);
  else if (vec == 2) launch_tc_vec<2>(L, sample, st);
  else launch_tc_vec<1>(L, sample, st);
}

}  // namespace flb
