// The per-site noise-scale network (3 -> 32 -> 32 -> 6, bfloat16 operands, FP32
// accumulation; learned extension, not in the paper) evaluated by one warp on the
// tensor cores with warp-level MMAs (mma.sync m16n8k16), every operand in registers.
//
// Why a warp-level form: the network is three dependent layers with a relu between
// them, ~3 kflop per site, inside a step that moves 72 bytes per site.  The tensor
// work is small (at 70 % of the HBM rate the tensor pipes are ~40 % busy); what costs
// is moving activations between layers and synchronising.  Here a warp needs no
// barrier, no tensor memory and no shared memory between the layers: the accumulator
// fragment of one layer is, register for register, the A fragment of the next.
//
// Site -> fragment mapping.  Lane (g, c) = (lane / 4, lane % 4) holds two sites: s0 and
// s1 (the thread's sites v and v + 1).  They are rows g and g + 8 of "slot" c.  The
// layer-1 input row of slot c is k = 2c, 2c+1: (u_x, u_y); k = 8+2c, 9+2c: (drho, 1).
// So the A fragment of lane (g, c) is exactly its own inputs and no data moves.  For
// slot c the other lanes' inputs are masked to zero, and one weight tile (each slot's
// k rows equal) gives W1 x + b1 for the 16 sites of that slot.  Layers 2 and 3 then run
// per slot on 16-row tiles.  The layer-3 accumulators of site (row, slot) end up in lanes
// (row % 8, 0..2), two outputs each.  One shared-memory transpose per pass (8 two-float
// stores, 3 four-float loads per lane) returns them to the site's own lane.
#pragma once
#include "step_common.cuh"

namespace flb {

// round to bfloat16 and pack (lo in the low half, the lower k index)
__device__ __forceinline__ uint32_t wn_pack2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// relu, round to bfloat16 and pack
__device__ __forceinline__ uint32_t wn_relu_pack2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ float wn_bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// d = a b + c for one 16x8x16 tile (A row-major, B column-major, FP32 accumulators)
__device__ __forceinline__ void wn_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1, float c0,
                                       float c1, float c2, float c3) {
  // not volatile: the compiler may interleave the independent chains of the four slots
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

// Weight and bias fragments of one lane (38 registers), built once per kernel from the
// FP32 copies of the bfloat16 weights.  Biases are rounded to bfloat16, as in the
// tensor-memory form of the network (where they are weights of a constant-1 input).
struct WarpNet {
  uint32_t b1[4][2];      // layer 1, n-tile h (hidden 8h..8h+7): (W1[n][0], W1[n][1]), (W1[n][2], b1[n]), n = 8h + g
  uint32_t b2[2][4][2];   // layer 2, k-tile t, n-tile h: W2[n][16t + 2c ..], W2[n][16t + 8 + 2c ..]
  float c2[4][2];         // layer 2 bias at the lane's accumulator columns 8h + 2c, 8h + 2c + 1
  uint32_t b3[2][2];      // layer 3, k-tile t (outputs 0..7; 6 and 7 are zero)
  float c3[2];            // 1 + b3 at columns 2c, 2c + 1 (zero for c = 3): s = 1 + o

  __device__ void load(const MlpWeights& w) {
    const int lane = (int)(threadIdx.x & 31), g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int n = 8 * h + g;
      b1[h][0] = wn_pack2(w.W1[3 * n], w.W1[3 * n + 1]);
      b1[h][1] = wn_pack2(w.W1[3 * n + 2], w.b1[n]);
      c2[h][0] = wn_bf16_round(w.b2[8 * h + 2 * c]);
      c2[h][1] = wn_bf16_round(w.b2[8 * h + 2 * c + 1]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float* row = w.W2 + kMlpHidden * (8 * h + g) + 16 * t + 2 * c;
        b2[t][h][0] = wn_pack2(row[0], row[1]);
        b2[t][h][1] = wn_pack2(row[8], row[9]);
      }
      const float* row = w.W3 + kMlpHidden * (g < kMlpOut ? g : 0) + 16 * t + 2 * c;
      b3[t][0] = g < kMlpOut ? wn_pack2(row[0], row[1]) : 0u;
      b3[t][1] = g < kMlpOut ? wn_pack2(row[8], row[9]) : 0u;
    }
    c3[0] = 2 * c < kMlpOut ? 1.f + wn_bf16_round(w.b3[2 * c]) : 0.f;
    c3[1] = 2 * c + 1 < kMlpOut ? 1.f + wn_bf16_round(w.b3[2 * c + 1]) : 0.f;
  }

  // Scales s = 1 + o of the lane's two sites.  x = (pack(u_x, u_y) of s0, of s1,
  // pack(drho, 1) of s0, of s1).  scr: this warp's 384 floats of shared memory.  Every
  // lane of the warp must call it (warp-synchronous MMAs).
  __device__ __forceinline__ void forward(const uint32_t (&x)[4], float* scr, float (&s0)[6], float (&s1)[6]) const {
    const int lane = (int)(threadIdx.x & 31), g = lane >> 2, c = lane & 3;
    __syncwarp();                         // the previous pass's reads of scr are done
#pragma unroll
    for (int slot = 0; slot < 4; ++slot) {
      const bool mine = c == slot;
      const uint32_t a1[4] = {mine ? x[0] : 0u, mine ? x[1] : 0u, mine ? x[2] : 0u, mine ? x[3] : 0u};
      float d1[4][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) wn_mma(d1[h], a1, b1[h][0], b1[h][1], 0.f, 0.f, 0.f, 0.f);
      uint32_t a2[2][4];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        a2[t][0] = wn_relu_pack2(d1[2 * t][0], d1[2 * t][1]);
        a2[t][1] = wn_relu_pack2(d1[2 * t][2], d1[2 * t][3]);
        a2[t][2] = wn_relu_pack2(d1[2 * t + 1][0], d1[2 * t + 1][1]);
        a2[t][3] = wn_relu_pack2(d1[2 * t + 1][2], d1[2 * t + 1][3]);
      }
      // layer 2 with the bias as the first MMA's accumulator input (rows g and g + 8 take
      // the same bias columns), so no FP32 adds follow the MMAs: 20 fewer instructions per
      // site, 4.54 -> 4.41 ms per 16384^2 step, without spills in the single-replica kernels
      float d2[4][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        wn_mma(d2[h], a2[0], b2[0][h][0], b2[0][h][1], c2[h][0], c2[h][1], c2[h][0], c2[h][1]);
        wn_mma(d2[h], a2[1], b2[1][h][0], b2[1][h][1], d2[h][0], d2[h][1], d2[h][2], d2[h][3]);
      }
      uint32_t a3[2][4];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int h = 2 * t + e;
          a3[t][2 * e] = wn_relu_pack2(d2[h][0], d2[h][1]);       // row g
          a3[t][2 * e + 1] = wn_relu_pack2(d2[h][2], d2[h][3]);   // row g + 8
        }
      }
      float d3[4];                          // the scales 1 + o, the bias term likewise
      wn_mma(d3, a3[0], b3[0][0], b3[0][1], c3[0], c3[1], c3[0], c3[1]);
      wn_mma(d3, a3[1], b3[1][0], b3[1][1], d3[0], d3[1], d3[2], d3[3]);
      const float2 o0 = make_float2(d3[0], d3[1]);
      const float2 o1 = make_float2(d3[2], d3[3]);
      // site (row g, slot) -> scr[slot][g][0][...], site (row g + 8, slot) -> scr[slot][g][1][...]
      if (c < 3 && FLB_INB((slot * 8 + g) * 12 + 2 * c + 7 < 4 * 8 * 12, 121)) {
        float* p = scr + (slot * 8 + g) * 12 + 2 * c;
        *reinterpret_cast<float2*>(p) = o0;
        *reinterpret_cast<float2*>(p + 6) = o1;
      }
    }
    __syncwarp();
    const int qi = FLB_INB((c * 8 + g) * 12 + 12 <= 4 * 8 * 12, 122) ? (c * 8 + g) * 12 : 0;
    const float4* q = reinterpret_cast<const float4*>(scr + qi);
    const float4 q0 = q[0], q1 = q[1], q2 = q[2];
    s0[0] = q0.x; s0[1] = q0.y; s0[2] = q0.z; s0[3] = q0.w; s0[4] = q1.x; s0[5] = q1.y;
    s1[0] = q1.z; s1[1] = q1.w; s1[2] = q2.x; s1[3] = q2.y; s1[4] = q2.z; s1[5] = q2.w;
  }
};

constexpr int kWarpNetScratch = 4 * 8 * 12;     // floats of shared memory per warp

}  // namespace flb
