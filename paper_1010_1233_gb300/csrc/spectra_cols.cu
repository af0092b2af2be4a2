// Column passes of the correlator sampling (Eqs. 11-12) in FP32 for column transforms
// of length L = 16 B (B = 1, 2, 4, 8, 16): register-resident counterparts of
// k_fft_cols_a and k_fft_cols_acc (spectra.cu) with the same tiles, the same in-place
// spectrum and the same pair sums.  One kernel per B; each takes the blocks of the
// replicas whose columns have its length and skips the others (which the kernel of
// their own length, or the shared-memory kernel, takes), so a replica's results do not
// depend on the batch it runs in.
//
// Element n = r + B j of a length-L sequence (r < B, j < 16) is loaded by thread r of
// the sequence.  With k = q + 16 p (q < 16, p < B),
//   W_L^(n k) = W_L^(r q) W_B^(r p) W_16^(j q),
// so X(q + 16 p) = sum_r W_B^(r p) [W_L^(r q) sum_j x(r + B j) W_16^(j q)].
// Stage 1: the 16-point transform over j in registers, then the twiddle W_L^(r q); the
// results go to shared memory, sequence (f, c) row at s + (f ncol + c)(L + 1), V_r(q) at
// q B + r.  Stage 2: for each of its 16 / B values of q, a thread reads the B values
// V_r(q) (slots q B .. q B + B - 1) and transforms over r; X(q + 16 p) goes back to slot
// q B + p, the slots the thread read, so stage 2 works in place.
//
// Against the shared-memory radix-2 passes this does one shared-memory round trip per
// element instead of three and needs no bit reversal or per-stage index arithmetic:
// every twiddle of the 16- and B-point transforms is a compile-time constant.
#include <algorithm>
#include "fft_reg.cuh"
#include "spectra_acc.cuh"

namespace flb {

constexpr int kCols16Block = 256;

template <int B> constexpr int log2_ct() { return B == 1 ? 0 : 1 + log2_ct<B / 2>(); }

// W_L^m for m < L from the length-ny table tw (exp(-2 pi i m' / ny), m' < ny / 2):
// W_L^m = W_ny^(m ny / L)
__device__ __forceinline__ void fill_wl(float2* wl, int L, const float2* __restrict__ tw, int ny) {
  const int step = ny / L, hn = ny >> 1;
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    const int e = m * step;
    float2 w = tw[e < hn ? e : e - hn];
    if (e >= hn) { w.x = -w.x; w.y = -w.y; }
    wl[m] = w;
  }
}

// Stage 1 for the work item (f, c, r) whose 16 inputs are at src + j jstride (zero when
// !in), results into its shared-memory row e (already offset by r).
template <int B>
__device__ __forceinline__ void stage1(const float2* __restrict__ src, int64_t jstride, bool in, float2* e,
                                       const float2* wl, int r) {
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = in ? src[j * jstride] : make_float2(0.f, 0.f);
  dft_reg<float, 16>(v);
  e[0] = v[0];
#pragma unroll
  for (int q = 1; q < 16; ++q) e[q * B] = B > 1 ? cmul<float>(v[q], wl[r * q]) : v[q];
}

// Pass 2a tile (four-step, N1 = L) of one field f: the columns kx0 .. kx0 + ncl - 1 of
// the rows N2 y1 + y2, transformed over y1, times W_ny^(y2 k1), back to rows N2 k1 + y2.
// (Pass 2a needs no field pairs, so a block takes one field: a quarter of the shared
// memory of an all-field tile, and four times the blocks per SM.)  All threads call it;
// it ends with a barrier.
template <int B>
__device__ __forceinline__ void cols_a16_tile(const ReplicaDesc& d, char* __restrict__ ws, float2* s, int f, int y2,
                                              int kx0, int ncl, int ncol, int slot) {
  constexpr int L = 16 * B, SS = L + 1, QN = 16 / B, LB = log2_ct<B>();
  const int lc = 31 - __clz(ncol);
  const int n2 = d.ny >> d.log2n1, hn = d.ny >> 1;
  const float2* tw = reinterpret_cast<const float2*>(ws + d.off_tw_y);
  float2* spec = reinterpret_cast<float2*>(ws + d.off_spec + slot * d.spec_slot) + f * (int64_t)d.ny * d.wpitch;
  float2* wl = s + ncol * SS;
  fill_wl(wl, L, tw, d.ny);
  __syncthreads();
  const int items = 1 << (lc + LB);
  // stage 1: rows y = N2 (r + B j) + y2
  const int64_t jstride = (int64_t)n2 * B * d.wpitch;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it & (ncol - 1), r = it >> lc;
    const bool in = c < ncl && FLB_INB(f < (int)d.n_fields && n2 * (r + B * 15) + y2 < d.ny && kx0 + c < d.half_nx, 201);
    stage1<B>(spec + (int64_t)(n2 * r + y2) * d.wpitch + kx0 + c, jstride, in, s + c * SS + r, wl, r);
  }
  __syncthreads();
  // stage 2, then the twiddle W_ny^(y2 k1) and the store to row N2 k1 + y2
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it & (ncol - 1), t = it >> lc;
    const float2* e = s + c * SS;
    float2* dst = spec + (int64_t)y2 * d.wpitch + kx0 + c;
#pragma unroll
    for (int qi = 0; qi < QN; ++qi) {
      const int q = t * QN + qi;
      float2 u[B];
#pragma unroll
      for (int r = 0; r < B; ++r) u[r] = e[q * B + r];
      dft_reg<float, B>(u);
      if (c >= ncl) continue;
#pragma unroll
      for (int p = 0; p < B; ++p) {
        const int k1 = q + 16 * p;
        const int ex = y2 * k1;                     // < ny
        float2 w = tw[ex < hn ? ex : ex - hn];
        if (ex >= hn) { w.x = -w.x; w.y = -w.y; }
        if (FLB_INB(f < (int)d.n_fields && n2 * k1 + y2 < d.ny && kx0 + c < d.half_nx, 203))
          dst[(int64_t)n2 * k1 * d.wpitch] = cmul<float>(u[p], w);
      }
    }
  }
  __syncthreads();
}

// Pass 2b tile (N2 = L; one-pass columns are N1 = 1): the rows N2 k1 + y2 of the tile
// transformed over y2, X(k2) left at slot out_slot<B>(k2), then the pair products added
// to the FP64 sums.  All threads call it; it ends with a barrier.
template <int B>
__device__ __forceinline__ void cols_acc16_tile(const ReplicaDesc& d, char* __restrict__ ws, float2* s, int rep,
                                                int k1, int kx0, int ncl, int ncol, int tiles, const TimeCorr& tc,
                                                int nslots) {
  constexpr int L = 16 * B, SS = L + 1, QN = 16 / B, LB = log2_ct<B>();
  const int lc = 31 - __clz(ncol);
  const int n2 = d.ny >> d.log2n1, F = (int)d.n_fields;
  const int64_t fplane = (int64_t)d.ny * d.wpitch;
  const int slot_elems = F * ncol * SS;                 // shared-memory rows of one sample
  float2* wl = s + nslots * slot_elems;
  fill_wl(wl, L, reinterpret_cast<const float2*>(ws + d.off_tw_y), d.ny);
  __syncthreads();
  // work items (sample slot k, field f, row r or thread t of the sequence, column c)
  const int per_slot = F << (lc + LB), items = nslots * per_slot;
  // stage 1: rows y = N2 k1 + r + B j
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int k = it >= per_slot, i = it - k * per_slot;
    const int c = i & (ncol - 1), r = (i >> lc) & (B - 1), f = i >> (lc + LB);
    const float2* spec = reinterpret_cast<const float2*>(ws + d.off_spec + k * d.spec_slot);
    const bool in = c < ncl && FLB_INB(f < F && n2 * k1 + r + B * 15 < d.ny && kx0 + c < d.half_nx, 211);
    if (!FLB_INB((f * ncol + c + 1) * SS <= slot_elems, 212)) continue;
    stage1<B>(spec + f * fplane + (int64_t)(n2 * k1 + r) * d.wpitch + kx0 + c, (int64_t)B * d.wpitch, in,
              s + k * slot_elems + (f * ncol + c) * SS + r, wl, r);
  }
  __syncthreads();
  // stage 2 in place
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int k = it >= per_slot, i = it - k * per_slot;
    const int c = i & (ncol - 1), t = (i >> lc) & (B - 1), f = i >> (lc + LB);
    if (!FLB_INB((f * ncol + c + 1) * SS <= slot_elems, 212)) continue;
    float2* e = s + k * slot_elems + (f * ncol + c) * SS;
#pragma unroll
    for (int qi = 0; qi < QN; ++qi) {
      const int q = t * QN + qi;
      float2 u[B];
#pragma unroll
      for (int r = 0; r < B; ++r) u[r] = e[q * B + r];
      dft_reg<float, B>(u);
#pragma unroll
      for (int p = 0; p < B; ++p) e[q * B + p] = u[p];
    }
  }
  __syncthreads();
  accumulate_points<B>(d, ws, s, SS, k1, kx0, ncl, ncol, tiles, nslots, slot_elems);
  tile_tail<float, B>(d, ws, s, SS, rep, k1, kx0, ncl, ncol, tc, nslots, slot_elems);
  __syncthreads();
}

// One block per (replica, field, y2, tile of kColsA16 columns).
template <int B>
__global__ void __launch_bounds__(kCols16Block, 4)
k_fft_cols_a16(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
               int64_t n_vblocks, char* __restrict__ ws, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  constexpr int ncol = kColsA16, lc = log2_ct<kColsA16>();
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int rp = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[rp];
    if (cols16_b(1 << d.log2n1) != B) continue;
    const int tiles = (d.half_nx + ncol - 1) >> lc;
    const int64_t per_field = (int64_t)tiles * (d.ny >> d.log2n1);
    const int64_t local = vb - vb_begin[rp];
    const int f = (int)(local / per_field);
    const int64_t lf = local - f * per_field;
    const int y2 = (int)(lf / tiles);
    const int kx0 = (int)(lf - (int64_t)y2 * tiles) << lc;
    cols_a16_tile<B>(d, ws, s, f, y2, kx0, min(ncol, d.half_nx - kx0), ncol, slot);
  }
}

#ifndef FLB_ACC16_MIN_BLOCKS
#define FLB_ACC16_MIN_BLOCKS 4
#endif
template <int B>
__global__ void __launch_bounds__(kCols16Block, FLB_ACC16_MIN_BLOCKS)
k_fft_cols_acc16(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
                 int64_t n_vblocks, char* __restrict__ ws, int ncol, TimeCorr tc, int nslots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int lc = 31 - __clz(ncol);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int rp = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[rp];
    const int n2 = d.ny >> d.log2n1;
    if (cols16_b(n2) != B) continue;
    const int tiles = (d.half_nx + ncol - 1) >> lc;
    const int64_t local = vb - vb_begin[rp];
    const int k1 = (int)(local / tiles);
    const int kx0 = (int)(local - (int64_t)k1 * tiles) << lc;
    // blocked pair sums: this block's sums of every pair are one contiguous range, pulled
    // into L2 by bulk prefetches while the columns are loaded and transformed
    if (d.acc_ncol && threadIdx.x < d.n_pairs) {
      const int pr = threadIdx.x;
      const int64_t el = d.pair_a[pr] == d.pair_b[pr] ? 8 : 16;
      const int64_t first = (int64_t)(k1 * tiles + (kx0 >> lc)) * n2 * ncol;
      const char* base = ws + d.pair_off[pr] + first * el;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(base), "r"((uint32_t)(n2 * ncol * el)) : "memory");
    }
    cols_acc16_tile<B>(d, ws, s, rp, k1, kx0, min(ncol, d.half_nx - kx0), ncol, tiles, tc, nslots);
  }
}

cudaError_t set_fft16_smem_limits() {
  const int maxb = 227 * 1024, carve = (int)cudaSharedmemCarveoutMaxShared;
  cudaError_t e = cudaSuccess;
#define FLB_ATTR(K)                                                                                    \
  if (!e) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);              \
  if (!e) e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  FLB_ATTR(k_fft_cols_a16<1>) FLB_ATTR(k_fft_cols_a16<2>) FLB_ATTR(k_fft_cols_a16<4>)
  FLB_ATTR(k_fft_cols_a16<8>) FLB_ATTR(k_fft_cols_a16<16>)
  FLB_ATTR(k_fft_cols_acc16<1>) FLB_ATTR(k_fft_cols_acc16<2>) FLB_ATTR(k_fft_cols_acc16<4>)
  FLB_ATTR(k_fft_cols_acc16<8>) FLB_ATTR(k_fft_cols_acc16<16>)
#undef FLB_ATTR
  return e;
}

// one launch per B in the mask (bits 1, 2, 4, 8, 16); kColsA16 B threads (at least a warp,
// at most kCols16Block) and the shared memory of one field's tile
void launch_fft_cols_a16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                         char* ws, int grid, cudaStream_t st, int slot) {
#define FLB_L(B)                                                                                         \
  if (mask & B)                                                                                          \
    k_fft_cols_a16<B><<<grid, std::max(32, std::min(kCols16Block, kColsA16 * B)),                        \
                        (kColsA16 * (16 * B + 1) + 16 * B) * (int)sizeof(float2), st>>>(descs, vb_begin, \
                                                                                         n_reps, n_vblocks, ws, slot);
  FLB_L(1) FLB_L(2) FLB_L(4) FLB_L(8) FLB_L(16)
#undef FLB_L
}

// nslots = 2: the tiles of the samples in spectrum slots 0 and 1 in one pass (smem for both)
void launch_fft_cols_acc16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                           char* ws, int ncol, int grid, int smem, cudaStream_t st, const TimeCorr& tc, int nslots) {
#define FLB_L(B)                                                                                            \
  if (mask & B)                                                                                             \
    k_fft_cols_acc16<B><<<grid, kCols16Block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol, tc, nslots);
  FLB_L(1) FLB_L(2) FLB_L(4) FLB_L(8) FLB_L(16)
#undef FLB_L
}

}  // namespace flb
