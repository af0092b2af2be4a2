// Column passes of the correlator sampling (Eqs. 11-12) in FP32 for column transforms
// of length L = 16 B (B = 1, 2, 4, 8, 16): register-resident counterparts of
// k_fft_cols_a and k_fft_cols_acc (spectra.cu), on the same spectrum (in either of its
// layouts, spec_index) and the same pair sums; pass 2b keeps their tiles, pass 2a takes
// tiles of one field.  One kernel per B; each takes the blocks of the replicas whose
// columns have its length and skips the others (which the kernel of their own length,
// or the shared-memory kernel, takes), so a replica's results do not depend on the
// batch it runs in.
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

// Pass 2a (four-step, N1 = L): one unit per (replica, field f, y2, tile of kColsA16
// columns); pass 2a needs no field pairs, so a tile holds one field.  A block loads the
// columns kx0 .. kx0 + 15 of the rows N2 y1 + y2 (y1 < L), transforms over y1,
// multiplies by W_ny^(y2 k1) and stores back to rows N2 k1 + y2.  The loads go through
// shared memory by asynchronous 16-byte copies (cp.async) issued units ahead, so a
// block keeps its next units' copies in flight while it transforms (the copies are the
// block's only reads of the spectrum).
struct A16Unit {
  int rep, f, y2, kx0;
};

__device__ __forceinline__ A16Unit a16_unit(const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                                            int64_t vb) {
  A16Unit u;
  u.rep = find_rep(vb_begin, n_reps, vb);
  const ReplicaDesc& d = descs[u.rep];
  const int tiles = (d.half_nx + kColsA16 - 1) / kColsA16;
  const int64_t per_field = (int64_t)tiles * (d.ny >> d.log2n1);
  const int64_t local = vb - vb_begin[u.rep];
  u.f = (int)(local / per_field);
  const int64_t lf = local - u.f * per_field;
  if (d.spec_tiled) {               // y2 fastest: neighbouring units, neighbouring rows of a slab
    const int n2 = d.ny >> d.log2n1;
    const int t = (int)(lf / n2);
    u.y2 = (int)(lf - (int64_t)t * n2);
    u.kx0 = t * kColsA16;
  } else {                          // tile fastest: neighbouring units, neighbouring columns of rows
    u.y2 = (int)(lf / tiles);
    u.kx0 = (int)(lf - (int64_t)u.y2 * tiles) * kColsA16;
  }
  return u;
}

// the block's next unit of this kernel (blocks of replicas with other column lengths
// are skipped), or n_vblocks
template <int B>
__device__ __forceinline__ int64_t a16_next(const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                                            int64_t n_vblocks, int64_t vb) {
  for (; vb < n_vblocks; vb += gridDim.x)
    if (cols16_b(1 << descs[find_rep(vb_begin, n_reps, vb)].log2n1) == B) break;
  return vb;
}

// the asynchronous copies of a unit's L x kColsA16 complex values into a staging
// buffer [L][kColsA16]: 16-byte chunks (two columns), chunks past the row pitch skipped
template <int B>
__device__ __forceinline__ void a16_issue(const ReplicaDesc& d, const A16Unit& u, const char* ws, int slot,
                                          float2* buf) {
  constexpr int L = 16 * B, CH = kColsA16 / 2;          // chunks per row
  const int n2 = d.ny >> d.log2n1;
  const float2* spec = reinterpret_cast<const float2*>(ws + d.off_spec + slot * d.spec_slot) +
                       spec_index(d, u.f, 0, u.kx0);
  const int rs = spec_row_stride(d), cols = d.spec_tiled ? kSpecTile : d.wpitch - u.kx0;   // columns present
  for (int i = threadIdx.x; i < L * CH; i += blockDim.x) {
    const int y1 = i / CH, ch = i - y1 * CH;
    if (2 * ch >= cols) continue;
    if (!FLB_INB(u.f < (int)d.n_fields && n2 * y1 + u.y2 < d.ny, 204)) continue;
    const float2* src = spec + (int64_t)(n2 * y1 + u.y2) * rs + 2 * ch;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf + y1 * kColsA16 + 2 * ch);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
  }
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
  const int rs = spec_row_stride(d);
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
    stage1<B>(spec + spec_index(d, f, n2 * k1 + r, kx0) + c, (int64_t)B * rs, in,
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

// kA16Stages staging buffers of (L + 1) kColsA16 complex values: a unit's copies land in
// one as [y1][c]; once its values are in registers the same buffer takes the exchange
// rows [c][L + 1], so every buffer serves one unit from its copies to its stores and
// the copies of the next kA16Stages - 1 units are in flight meanwhile.
constexpr int kA16Stages = 3;

template <int B>
__global__ void __launch_bounds__(kColsA16 * 16, 64 / kColsA16)     // 64 registers a thread
k_fft_cols_a16(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
               int64_t n_vblocks, char* __restrict__ ws, int slot) {
  constexpr int L = 16 * B, SS = L + 1, QN = 16 / B, ncol = kColsA16, lc = log2_ct<kColsA16>();
  constexpr int BUF = ncol * SS;                         // >= L ncol
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* stage = reinterpret_cast<float2*>(smem_raw);   // [kA16Stages][BUF]
  float2* wl = stage + kA16Stages * BUF;                 // [L]: W_L^m
  float2* wy = wl + L;                                   // [L]: W_ny^(y2 k1) of the current unit
  // the block's units: the current one (u0, buffer cb) and the next two (u1, u2), whose
  // copies are in flight; vb: the unit after u2
  static_assert(kA16Stages == 3, "the current unit and two ahead");
  A16Unit u0{}, u1{}, u2{};
  int64_t v0 = a16_next<B>(descs, vb_begin, n_reps, n_vblocks, blockIdx.x);
  int64_t v1 = v0 < n_vblocks ? a16_next<B>(descs, vb_begin, n_reps, n_vblocks, v0 + gridDim.x) : n_vblocks;
  int64_t vb = v1 < n_vblocks ? a16_next<B>(descs, vb_begin, n_reps, n_vblocks, v1 + gridDim.x) : n_vblocks;
  if (v0 < n_vblocks) {
    u0 = a16_unit(descs, vb_begin, n_reps, v0);
    a16_issue<B>(descs[u0.rep], u0, ws, slot, stage);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (v1 < n_vblocks) {
    u1 = a16_unit(descs, vb_begin, n_reps, v1);
    a16_issue<B>(descs[u1.rep], u1, ws, slot, stage + BUF);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int cb = 0; v0 < n_vblocks; cb = cb == kA16Stages - 1 ? 0 : cb + 1) {
    const A16Unit cur = u0;
    const ReplicaDesc& d = descs[cur.rep];
    // the unit two ahead into the buffer the previous unit left
    const int nb = cb == 0 ? kA16Stages - 1 : cb - 1;
    const int64_t v2 = vb;
    if (v2 < n_vblocks) {
      u2 = a16_unit(descs, vb_begin, n_reps, v2);
      a16_issue<B>(descs[u2.rep], u2, ws, slot, stage + nb * BUF);
      vb = a16_next<B>(descs, vb_begin, n_reps, n_vblocks, v2 + gridDim.x);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const float2* tw = reinterpret_cast<const float2*>(ws + d.off_tw_y);
    const int n2 = d.ny >> d.log2n1, hn = d.ny >> 1;
    fill_wl(wl, L, tw, d.ny);
    for (int k1 = threadIdx.x; k1 < L; k1 += blockDim.x) {   // the unit's twiddles, y2 k1 < ny
      const int ex = cur.y2 * k1;
      float2 w = tw[ex < hn ? ex : ex - hn];
      if (ex >= hn) { w.x = -w.x; w.y = -w.y; }
      wy[k1] = w;
    }
    asm volatile("cp.async.wait_group %0;" :: "n"(kA16Stages - 1) : "memory");
    __syncthreads();
    const int ncl = min(ncol, d.half_nx - cur.kx0);
    float2* buf = stage + cb * BUF;
    // stage 1: thread (c, r) transforms y1 = r + B j, j < 16
    const int it0 = threadIdx.x, c0 = it0 & (ncol - 1), r0 = it0 >> lc;
    const bool act = it0 < ncol * B;                      // blockDim.x >= ncol B
    float2 v[16];
    if (act) {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = buf[(r0 + B * j) * ncol + c0];
      dft_reg<float, 16>(v);
    }
    __syncthreads();                                     // the copied values are all in registers
    if (act) {
      float2* e = buf + c0 * SS + r0;
      e[0] = v[0];
#pragma unroll
      for (int q = 1; q < 16; ++q) e[q * B] = B > 1 ? cmul<float>(v[q], wl[r0 * q]) : v[q];
    }
    __syncthreads();
    // stage 2, then the twiddle W_ny^(y2 k1) and the store to row N2 k1 + y2
    float2* spec = reinterpret_cast<float2*>(ws + d.off_spec + slot * d.spec_slot);
    const int rs = spec_row_stride(d);
    if (act) {
      const int c = c0, t = r0;
      const float2* e = buf + c * SS;
      float2* dst = spec + spec_index(d, cur.f, cur.y2, cur.kx0) + c;
#pragma unroll
      for (int qi = 0; qi < QN; ++qi) {
        const int q = t * QN + qi;
        float2 w8[B];
#pragma unroll
        for (int r = 0; r < B; ++r) w8[r] = e[q * B + r];
        dft_reg<float, B>(w8);
        if (c >= ncl) continue;
#pragma unroll
        for (int p = 0; p < B; ++p) {
          const int k1 = q + 16 * p;
          if (FLB_INB(cur.f < (int)d.n_fields && n2 * k1 + cur.y2 < d.ny && cur.kx0 + c < d.half_nx, 203))
            dst[(int64_t)n2 * k1 * rs] = cmul<float>(w8[p], wy[k1]);
        }
      }
    }
    __syncthreads();                                     // buffer cb free for a new unit
    u0 = u1; v0 = v1;
    u1 = u2; v1 = v2;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Pass 2b (N2 = L): one block per (replica, k1, tile of ncol columns), all fields and
// the nslots samples of the tile; four blocks per SM (measured against three, with 80
// registers and no spills: 10.08 against 10.50 ms per 16384^2 sample).
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

// shared memory of the pass-2a kernel: the staging buffers and two twiddle tables
static int a16_smem(int B) {
  const int L = 16 * B;
  return (kA16Stages * kColsA16 * (L + 1) + 2 * L) * (int)sizeof(float2);
}

// one launch per B in the mask (bits 1, 2, 4, 8, 16); kColsA16 B threads (at least a warp)
// and the shared memory of one field's tiles
void launch_fft_cols_a16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                         char* ws, int grid, cudaStream_t st, int slot) {
#define FLB_L(B)                                                                                         \
  if (mask & B)                                                                                          \
    k_fft_cols_a16<B><<<grid, std::max(32, kColsA16 * B), a16_smem(B), st>>>(                                \
        descs, vb_begin, n_reps, n_vblocks, ws, slot);
  FLB_L(1) FLB_L(2) FLB_L(4) FLB_L(8) FLB_L(16)
#undef FLB_L
}

// nslots = 2: the tiles of the samples in spectrum slots 0 and 1 in one pass; each launch
// with the shared memory of its column length (max_fields: the most fields of a replica)
void launch_fft_cols_acc16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                           char* ws, int ncol, int grid, int max_fields, cudaStream_t st, const TimeCorr& tc,
                           int nslots) {
#define FLB_L(B)                                                                                            \
  if (mask & B)                                                                                             \
    k_fft_cols_acc16<B><<<grid, kCols16Block, fft_cols16_smem(max_fields, 16 * B, ncol, nslots), st>>>(     \
        descs, vb_begin, n_reps, n_vblocks, ws, ncol, tc, nslots);
  FLB_L(1) FLB_L(2) FLB_L(4) FLB_L(8) FLB_L(16)
#undef FLB_L
}

}  // namespace flb
