// tcgen05 pieces of the per-site noise-scale network shared by the step kernels with
// the network (lb_step_tc.cu, lb_step_bulk.cu): tensor-memory loads and stores, MMA
// issue and commit, bounded mbarrier waits, the bfloat16 weight tiles, and TcNet,
// which runs the three layers for the VEC tiles of one warpgroup.
//
// Tile layout: each warpgroup (128 threads) owns tensor-memory lanes 0..127; thread t
// of the warpgroup and its v-th site (v < VEC) form row t of tile v.  A tile has 64
// tensor-memory columns: D (32 FP32 columns) and A (24 columns = 48 bfloat16 of K,
// packed two per column).  Per layer the threads write their rows of A with
// tcgen05.st, one thread issues the MMAs (B, the weights, in shared memory) and
// commits them to the warpgroup's mbarrier, and every thread reads its row of D back
// with tcgen05.ld, applies relu and rounds to bfloat16 into A for the next layer.
// Biases enter through a constant-1 column of A (K index 3 in layer 1, 32 in layers 2
// and 3; columns 16..23 of A are written once).
#pragma once
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
// the clock is read every 16 polls and the wait gives up after `limit` SM clocks, by
// default 2^32, about two seconds)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = 1LL << 32) {
  const long long t0 = clock64();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 16; ++i) {
      uint32_t done;
      asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                   : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "n"(kWaitHintNs));
      if (done) return true;
    }
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void wg_barrier(int wg) { asm volatile("bar.sync %0, 128;" :: "r"(1 + wg)); }

// the warpgroup barrier that also ANDs a flag over its 128 threads
__device__ __forceinline__ bool wg_barrier_and(int wg, bool v) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.and.pred p, %2, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(r) : "r"((uint32_t)v), "r"(1 + wg));
  return r != 0;
}

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

// D row (32 FP32 columns at tmem address d) -> relu -> bfloat16 -> A row columns 0..15,
// in two halves of 16 values (8 packed columns each)
__device__ __forceinline__ void hidden_to_a(uint32_t d, uint32_t a) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t h[16];
    tmem_ld16(d + 16 * half, h);
    tmem_st8(a + 8 * half, relu_pack2(h[0], h[1]), relu_pack2(h[2], h[3]), relu_pack2(h[4], h[5]),
             relu_pack2(h[6], h[7]), relu_pack2(h[8], h[9]), relu_pack2(h[10], h[11]), relu_pack2(h[12], h[13]),
             relu_pack2(h[14], h[15]));
  }
}

// B operands (weights with the bias in the constant-1 column), bfloat16, K-major.
static __device__ void build_b_tiles(const MlpWeights& w, unsigned char* b1, unsigned char* b2, unsigned char* b3) {
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


// Resident blocks per SM allowed by tensor memory (512 columns, 2 * VEC tiles of 64 per block).
template <int VEC> struct TcOcc {
  static constexpr int kBlocks = 512 / (2 * VEC * (int)kTileCols);
  static constexpr int kMinBlocks = kBlocks < 3 ? kBlocks : 3;      // register cap of the launch bounds
};

// The three layers for the VEC tiles of one warpgroup.  start() writes the layer-1 rows
// and issues layer 1; the caller can do independent work (the Philox normals) before
// finish(), which runs layers 2 and 3 and returns the scales s = 1 + o.
template <int VEC>
struct TcNet {
  uint32_t tbase, trow;          // the warpgroup's first column; the same with this warp's lane base
  uint64_t db1, db2, db3;        // B descriptors
  uint64_t* bar;                 // the warpgroup's MMA mbarrier
  int wg, tw;
  uint32_t ph = 0;
  bool ok = true;                // false (in every thread of the warpgroup) once a wait gave up
  uint32_t pend = 2u;            // parity of the commit whose wait gave up (2: none)

  // Called by all threads after the block has built the B tiles, allocated tensor memory
  // (base `tmem`) and initialised `bar`, and synchronised.
  __device__ void init(uint32_t tmem, unsigned char* sb1, unsigned char* sb2, unsigned char* sb3, uint64_t* wg_bar) {
    const int tid = (int)threadIdx.x, warp = tid >> 5;
    wg = tid >> 7;
    tw = tid & 127;
    tbase = tmem + (uint32_t)(wg * VEC) * kTileCols;
    trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    db1 = smem_desc(smem_u32(sb1), kTcK1 / 8 * 128);
    db2 = smem_desc(smem_u32(sb2), kTcK / 8 * 128);
    db3 = smem_desc(smem_u32(sb3), kTcK / 8 * 128);
    bar = wg_bar;
    ph = 0;
    ok = true;
    pend = 2u;
#pragma unroll
    for (int v = 0; v < VEC; ++v)        // constant columns 16..23 of A: (1, 0), zeros
      tmem_st8(trow + v * kTileCols + 32 + 16, 0x3F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u);
    tmem_wait_st();
  }

  // the first warp of the warpgroup polls the mbarrier, the other three wait for it at
  // the warpgroup barrier (polling costs issue slots the other warps of the SM could use).
  // A wait that gives up clears ok in the whole warpgroup (the barrier ANDs it): from then
  // on no MMA is issued and no wait is made; drain() waits once more for that commit
  // before the tensor memory is freed.
  __device__ void wait_mma() {
    bool done = true;
    if (tw < 32 && ok) done = mbar_wait(bar, ph);
    const bool was_ok = ok;
    ok = wg_barrier_and(wg, ok && done);
    if (was_ok && !ok) pend = ph;
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
  }

  // after a wait gave up: one more bounded wait for the commit still pending, so that no
  // MMA is left writing tensor memory when it is freed (the caller synchronises the block
  // and frees it afterwards)
  __device__ void drain() {
    if (pend != 2u && tw < 32) mbar_wait(bar, pend);
  }

  // layer-1 rows of A: (u_x, u_y, rho - rho0, 1, 0, ...), then issue layer 1
  __device__ void start(const float (&ux)[VEC], const float (&uy)[VEC], const float (&drho)[VEC]) {
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      tmem_st8(trow + v * kTileCols + 32, pack2(ux[v], uy[v]), pack2(drho[v], 1.f), 0u, 0u, 0u, 0u, 0u, 0u);
    tmem_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;");
    wg_barrier(wg);
    if (tw == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int v = 0; v < VEC; ++v) mma_ts(tbase + v * kTileCols, tbase + v * kTileCols + 32, db1, instr_desc(128, 32), 0u);
      mma_commit(bar);
    }
  }

  // wait for layer L - 1, turn its output into the rows of A, issue layer L (2 or 3);
  // `hook` runs on the first warp of the warpgroup just before the issue
  template <int L, typename F>
  __device__ void next_layer(F&& hook) {
    wait_mma();
#pragma unroll
    for (int v = 0; v < VEC; ++v) hidden_to_a(trow + v * kTileCols, trow + v * kTileCols + 32);
    tmem_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;");
    wg_barrier(wg);
    if (tw < 32) hook();
    if (tw == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t db = L == 2 ? db2 : db3;
      constexpr uint32_t idesc = instr_desc(128, L == 2 ? 32 : 16);
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk)     // K step: 16 bf16 = 256 B of B, 8 columns of A
          mma_ts(tbase + v * kTileCols, tbase + v * kTileCols + 32 + 8 * kk, db + (uint64_t)(kk * 256 >> 4), idesc,
                 kk > 0 ? 1u : 0u);
      mma_commit(bar);
    }
  }
  template <int L>
  __device__ void next_layer() { next_layer<L>([] {}); }

  // wait for layer 3 and read the scales s = 1 + o
  __device__ void scales(float (&sc)[VEC][6]) {
    wait_mma();
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      uint32_t o[8];
      tmem_ld8(trow + v * kTileCols, o);
#pragma unroll
      for (int c = 0; c < 6; ++c) sc[v][c] = 1.f + __uint_as_float(o[c]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }

  template <typename F>
  __device__ void finish(float (&sc)[VEC][6], F&& before_l2) {
    next_layer<2>(before_l2);
    next_layer<3>();
    scales(sc);
  }
  __device__ void finish(float (&sc)[VEC][6]) { finish(sc, [] {}); }
};

// tensor-memory allocation by warp 0 (the slot receives the base address)
template <uint32_t kCols>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(slot)), "r"(kCols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
template <uint32_t kCols>
__device__ __forceinline__ void tmem_free(uint32_t base) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(base), "r"(kCols));
}

}  // namespace flb
