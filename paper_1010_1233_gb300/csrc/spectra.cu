// Correlator sampling (Eqs. 11-12): 2D discrete Fourier transform of the
// sampled real fields with a hand-written radix-2 FFT, and FP64 accumulation
// of X_a(k) X_b(k)^* for every sampled field pair on the half spectrum
// kx in [0, nx/2] (the other half follows from X(-k) = X(k)^* for real fields).
//
// Pass 1 (rows): two real rows (consecutive (field, row) units) are packed as one
// complex row z = X_a + i X_b, transformed along x in shared memory, and unpacked
// into the transforms of both rows, X_a(kx) = (Z(kx) + Z(-kx)^*)/2,
// X_b(kx) = (Z(kx) - Z(-kx)^*)/(2i).
// Pass 2 (columns): tiles of columns of every field are transformed along y in
// shared memory and the pair products are added to the FP64 sums.  Columns too
// long for shared memory use the four-step split ny = N1 N2, y = N2 y1 + y2,
// ky = k1 + N1 k2:  X(ky) = sum_y2 W_N2^(y2 k2) W_N^(y2 k1) sum_y1 W_N1^(y1 k1) x(y);
// pass 2a does the inner length-N1 transforms and the W_N^(y2 k1) twiddle in
// place (rows N2 y1 + y2 -> N2 k1 + y2), pass 2b the outer length-N2 transforms.
#include <algorithm>
#include "spectra_acc.cuh"

namespace flb {

// Pass 1: one block per (replica, packed pair of row units).
template <typename R>
__global__ void __launch_bounds__(kRowsBlockMax)
k_fft_rows(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                           int n_reps, int64_t n_vblocks, char* __restrict__ ws, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* z = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    if (sizeof(R) == 4 && rows16_nx(d.nx)) continue;   // k_fft_rows16's row
    // block vb packs the row units u = 2 local and u + 1 (unit u: field u / ny, row u % ny;
    // ny is a power of two), so an odd field count leaves at most one half-empty transform
    const int64_t ua = 2 * (vb - vb_begin[r]), ub = ua + 1;
    const bool has_b = ub < (int64_t)d.n_fields << d.log2ny;
    const int fa = (int)(ua >> d.log2ny), ya = (int)(ua & (d.ny - 1));
    const int fb = (int)(ub >> d.log2ny), yb = (int)(ub & (d.ny - 1));
    const int nx = d.nx, logn = d.log2nx;
    const int64_t plane = (int64_t)nx * d.ny;
    const R* fields = reinterpret_cast<const R*>(ws + d.off_fields);
    const R* xa = fields + fa * plane + (int64_t)ya * nx;
    const R* xb = fields + fb * plane + (int64_t)yb * nx;
    const int ps = logn > 5 ? logn - 5 : 31;        // 32 pad slots per row
    const C<R>* tw = reinterpret_cast<const C<R>*>(ws + d.off_tw_x);
    // the rows of this block's next pair into L2 while this pair is transformed
    if (threadIdx.x == 0 && vb + gridDim.x < n_vblocks) {
      const int64_t vbn = vb + gridDim.x;
      const int rn = find_rep(vb_begin, n_reps, vbn);
      const ReplicaDesc& dn = descs[rn];
      const int64_t un = 2 * (vbn - vb_begin[rn]);
      const R* fn = reinterpret_cast<const R*>(ws + dn.off_fields);
      const uint32_t bytes = (uint32_t)(dn.nx * sizeof(R));
      if (bytes % 16 == 0) {         // unit u starts at u nx (the fields are contiguous rows)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(fn + un * dn.nx), "r"(bytes) : "memory");
        if (un + 1 < (int64_t)dn.n_fields << dn.log2ny)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(fn + (un + 1) * dn.nx), "r"(bytes)
                       : "memory");
      }
    }
    if (logn >= 3) {
      // thread x0 < nx/8 loads x0 + j nx/8 (j < 8, coalesced): after bit reversal these are
      // elements t = brev3(j) of the group m = brev(x0) of the first three stages, which
      // run in registers before the group is stored
      const int n8 = nx >> 3;
      for (int x0 = threadIdx.x; x0 < n8; x0 += blockDim.x) {
        C<R> v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int x = x0 + (((t & 1) << 2) | (t & 2) | ((t >> 2) & 1)) * n8;
          const bool in = FLB_INB(x >= 0 && x < nx, 131);
          v[t].x = in ? xa[x] : (R)0;
          v[t].y = has_b && in ? xb[x] : (R)0;
        }
        dit_group<R, 3>(v, logn, 0, 0, tw, 1);
        const int i0 = brev(x0, logn - 3) << 3;
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (FLB_INB(i0 + t < nx, 132)) z[i0 + t + ((i0 + t) >> ps)] = v[t];
      }
      __syncthreads();
      dit_fft<R, sizeof(R) == 4 ? 4 : 3>(z, logn, 1, 0, tw, 1, ps, 3);   // FP32: four stages per pass
    } else {
      for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        C<R> v; v.x = xa[x]; v.y = has_b ? xb[x] : (R)0;
        const int i = brev(x, logn);
        if (FLB_INB(i < nx, 132)) z[i + (i >> ps)] = v;
      }
      __syncthreads();
      dit_fft<R>(z, logn, 1, 0, tw, 1, ps);
    }
    C<R>* spec = reinterpret_cast<C<R>*>(ws + d.off_spec + slot * d.spec_slot);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    C<R>* ra = spec + fa * fplane + (int64_t)ya * d.wpitch;
    C<R>* rb = spec + fb * fplane + (int64_t)yb * d.wpitch;
    const int hn = nx >> 1;
    const bool rows_ok = FLB_INB(fa < (int)d.n_fields && ya < d.ny && (!has_b || (fb < (int)d.n_fields && yb < d.ny)) &&
                                 hn < d.wpitch, 133);
    for (int k = threadIdx.x; k <= hn && rows_ok; k += blockDim.x) {
      const int km = (nx - k) & (nx - 1);
      const C<R> Z = z[k + (k >> ps)];
      const C<R> Zm = z[km + (km >> ps)];
      C<R> A; A.x = (R)0.5 * (Z.x + Zm.x); A.y = (R)0.5 * (Z.y - Zm.y);
      ra[k] = A;
      if (has_b) {            // (Z - conj(Zm)) / (2i)
        C<R> B; B.x = (R)0.5 * (Z.y + Zm.y); B.y = (R)0.5 * (Zm.x - Z.x);
        rb[k] = B;
      }
    }
    __syncthreads();
  }
}

// Pass 2a (four-step only): one block per (replica, y2, tile of ncol columns).
template <typename R>
__global__ void __launch_bounds__(kColsBlock, sizeof(R) == 4 ? 4 : 2)
k_fft_cols_a(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                             int n_reps, int64_t n_vblocks, char* __restrict__ ws, int ncol, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* s = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    if (sizeof(R) == 4 && cols16_b(1 << d.log2n1)) continue;        // a register-resident kernel's block
    const int lc = 31 - __clz(ncol);                    // ncol is a power of two
    const int tiles = (d.half_nx + ncol - 1) >> lc;
    const int64_t local = vb - vb_begin[r];
    const int y2 = (int)(local / tiles);
    const int kx0 = (int)(local - (int64_t)y2 * tiles) << lc;
    const int ncl = min(ncol, d.half_nx - kx0);
    const int logn1 = d.log2n1, n1 = 1 << logn1, n2 = d.ny >> logn1, F = (int)d.n_fields;
    C<R>* spec = reinterpret_cast<C<R>*>(ws + d.off_spec + slot * d.spec_slot);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    const int total = F * n1 * ncol;
    // the next tile of this block into L2 (one bulk prefetch per (field, y1) segment)
    if (vb + gridDim.x < n_vblocks) {
      const int64_t vbn = vb + gridDim.x;
      const int rn = find_rep(vb_begin, n_reps, vbn);
      const ReplicaDesc& dn = descs[rn];
      const int tn = (dn.half_nx + ncol - 1) >> lc;
      const int64_t ln = vbn - vb_begin[rn];
      const int y2n = (int)(ln / tn);
      const int kxn = (int)(ln - (int64_t)y2n * tn) << lc;
      const int ncn = min(ncol, dn.half_nx - kxn);
      const int l1n = dn.log2n1, n2n = dn.ny >> l1n;
      const uint32_t bytes = (uint32_t)(((ncn * (int)sizeof(C<R>)) + 15) & ~15);
      const C<R>* sp = reinterpret_cast<const C<R>*>(ws + dn.off_spec + slot * dn.spec_slot);
      const int64_t fpn = (int64_t)dn.ny * dn.wpitch;
      const int segs = (int)dn.n_fields << l1n;
      for (int i = threadIdx.x; i < segs; i += blockDim.x) {
        const int f = i >> l1n, y1 = i & ((1 << l1n) - 1);
        const C<R>* a = sp + f * fpn + (int64_t)(n2n * y1 + y2n) * dn.wpitch + kxn;
        if ((reinterpret_cast<uintptr_t>(a) & 15) == 0)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a), "r"(bytes) : "memory");
      }
    }
    // gather, four loads in flight per thread
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {
      C<R> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const int c = i & (ncol - 1), y1 = (i >> lc) & (n1 - 1), f = i >> (lc + logn1);
        v[u].x = (R)0; v[u].y = (R)0;
        if (i < total && c < ncl && FLB_INB(f < F && n2 * y1 + y2 < d.ny && kx0 + c < d.half_nx, 151))
          v[u] = spec[f * fplane + (int64_t)(n2 * y1 + y2) * d.wpitch + kx0 + c];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const int c = i & (ncol - 1), y1 = (i >> lc) & (n1 - 1), f = i >> (lc + logn1);
        if (i < total && FLB_INB(f < F && c < ncol && brev(y1, logn1) < n1, 152))
          s[(f * ncol + c) * (n1 + 1) + brev(y1, logn1)] = v[u];
      }
    }
    __syncthreads();
    const C<R>* tw = reinterpret_cast<const C<R>*>(ws + d.off_tw_y);
    dit_fft<R>(s, logn1, F * ncol, n1 + 1, tw, n2);
    const int hn = d.ny >> 1;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int c = i & (ncol - 1);
      const int k1 = (i >> lc) & (n1 - 1);
      const int f = i >> (lc + logn1);
      if (c >= ncl || !FLB_INB(f < F && n2 * k1 + y2 < d.ny && kx0 + c < d.half_nx, 151)) continue;
      const int e = y2 * k1;                       // < ny
      C<R> w = tw[e < hn ? e : e - hn];
      if (e >= hn) { w.x = -w.x; w.y = -w.y; }
      spec[f * fplane + (int64_t)(n2 * k1 + y2) * d.wpitch + kx0 + c] = cmul<R>(s[(f * ncol + c) * (n1 + 1) + k1], w);
    }
    __syncthreads();
  }
}

// Pass 2b: one block per (replica, k1, tile of ncol columns); all fields of the tile.
// One-pass columns are the case N1 = 1.
template <typename R>
__global__ void __launch_bounds__(kColsBlock, sizeof(R) == 4 ? 4 : 2)     // FP32: four blocks per SM
k_fft_cols_acc(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                               int n_reps, int64_t n_vblocks, char* __restrict__ ws, int ncol, TimeCorr tc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* s = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    if (sizeof(R) == 4 && cols16_b(d.ny >> d.log2n1)) continue;     // a register-resident kernel's block
    const int lc = 31 - __clz(ncol);                    // ncol is a power of two
    const int tiles = (d.half_nx + ncol - 1) >> lc;
    const int64_t local = vb - vb_begin[r];
    const int k1 = (int)(local / tiles);
    const int kx0 = (int)(local - (int64_t)k1 * tiles) << lc;
    const int logn1 = d.log2n1, n1 = 1 << logn1, logn2 = d.log2ny - logn1, n2 = d.ny >> logn1;
    const int F = (int)d.n_fields;
    const int ncl = min(ncol, d.half_nx - kx0);
    const C<R>* spec = reinterpret_cast<const C<R>*>(ws + d.off_spec);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    // blocked pair sums: this block's sums of every pair are one contiguous range, pulled
    // into L2 by bulk prefetches while the columns are loaded and transformed
    if (d.acc_ncol && threadIdx.x < d.n_pairs) {
      const int pr = threadIdx.x;
      const int64_t el = d.pair_a[pr] == d.pair_b[pr] ? 8 : 16;
      const int64_t first = (int64_t)(k1 * tiles + (kx0 >> lc)) * n2 * ncol;
      const char* base = ws + d.pair_off[pr] + first * el;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(base), "r"((uint32_t)(n2 * ncol * el)) : "memory");
    }
    // smem layout: [field][column][n2]
    const int total = F * n2 * ncol;
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {   // four loads in flight
      C<R> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const int c = i & (ncol - 1), y2 = (i >> lc) & (n2 - 1), f = i >> (lc + logn2);
        v[u].x = (R)0; v[u].y = (R)0;
        if (i < total && c < ncl && FLB_INB(f < F && n2 * k1 + y2 < d.ny && kx0 + c < d.half_nx, 161))
          v[u] = spec[f * fplane + (int64_t)(n2 * k1 + y2) * d.wpitch + kx0 + c];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const int c = i & (ncol - 1), y2 = (i >> lc) & (n2 - 1), f = i >> (lc + logn2);
        if (i < total && FLB_INB(f < F && c < ncol && brev(y2, logn2) < n2, 162))
          s[(f * ncol + c) * (n2 + 1) + brev(y2, logn2)] = v[u];
      }
    }
    __syncthreads();
    dit_fft<R>(s, logn2, F * ncol, n2 + 1, reinterpret_cast<const C<R>*>(ws + d.off_tw_y), n1);
    accumulate_tile<R, 0>(d, ws, s, n2 + 1, r, k1, kx0, ncl, ncol, tiles, tc);
    __syncthreads();
  }
}

// Time correlators, after the column pass of a sample: sums[tau][a][b][j] +=
// X_a(k_j, s) X_b(k_j, s - tau)^* for every lag with a sample s - tau in the ring
// (s = count), then (k_time_corr_advance) count += 1.  One item per (tau, a, b, j);
// blockIdx.y is the replica.
__global__ void k_time_corr(const ReplicaDesc* __restrict__ descs, TimeCorr tc) {
  const int r = blockIdx.y;
  const ReplicaDesc& d = descs[r];
  const int F = (int)d.n_fields, T = tc.n_lags, nk = tc.n_k;
  const uint64_t cnt = tc.count[r];
  const int slot = (int)(cnt % (uint64_t)T);
  const double2* ring = reinterpret_cast<const double2*>(tc.base + d.off_tc_ring);
  double2* sums = reinterpret_cast<double2*>(tc.base + d.off_tc_sums);
  const int64_t items = (int64_t)T * F * F * nk;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(it % nk);
    const int64_t rest = it / nk;
    const int b = (int)(rest % F), a = (int)((rest / F) % F), tau = (int)(rest / ((int64_t)F * F));
    if ((uint64_t)tau > cnt) continue;                         // no sample s - tau yet
    const int old = (slot - tau + T) % T;
    const double2 xa = ring[((int64_t)slot * F + a) * nk + j];
    const double2 xb = ring[((int64_t)old * F + b) * nk + j];
    double2 v = sums[it];
    v.x += xa.x * xb.x + xa.y * xb.y;                          // X_a X_b^*
    v.y += xa.y * xb.x - xa.x * xb.y;
    sums[it] = v;
  }
}

__global__ void k_time_corr_advance(TimeCorr tc, int n_reps) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_reps) tc.count[r] += 1;
}

template <typename R>
__global__ void k_twiddles(C<R>* tw, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n / 2) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)n, &sn, &cs);
  C<R> v; v.x = (R)cs; v.y = (R)(-sn);
  tw[m] = v;
}

// ---------------------------------------------------------------------------
void launch_fft_cols_a16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                         char* ws, int grid, cudaStream_t st, int slot);
void launch_fft_cols_acc16(int mask, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks,
                           char* ws, int ncol, int grid, int max_fields, cudaStream_t st, const TimeCorr& tc,
                           int nslots);
cudaError_t set_fft16_smem_limits();
void launch_fft_rows16(const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks, char* ws,
                       int grid, int nx, cudaStream_t st, int slot);
cudaError_t set_rows16_smem_limits();

void launch_twiddles(int precision, void* tw, int n, cudaStream_t st) {
  if (n < 2) return;
  const int half = n / 2;
  if (precision == FLB_FP64)
    k_twiddles<double><<<(half + 255) / 256, 256, 0, st>>>(reinterpret_cast<double2*>(tw), n);
  else
    k_twiddles<float><<<(half + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2*>(tw), n);
}

// shared memory of the row pass for rows of nx: k_fft_rows16 holds nx / 2 complex values
// (one pad slot per 16), k_fft_rows nx plus 32 pad slots
int fft_rows_smem(int precision, int nx) {
  if (rows16(precision, nx)) return (nx / 2 + nx / 32) * 8;
  return (nx + 32) * (precision == FLB_FP64 ? 16 : 8);
}
// the columns of every field of a tile, plus a table of up to 256 roots of unity
// (the register-resident passes of spectra_cols.cu)
int fft_cols_smem(int precision, int F, int ny, int ncol) { return (F * (ny + 1) * ncol + 256) * (precision == FLB_FP64 ? 16 : 8); }

cudaError_t set_fft_smem_limits() {
  cudaError_t e;
  const int maxb = 227 * 1024;
  // the transforms want shared memory, not L1 (a preference the CUDA runtime rounds to a supported split)
  const int carve = (int)cudaSharedmemCarveoutMaxShared;
  if ((e = cudaFuncSetAttribute(k_fft_rows<float>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_a<float>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_acc<float>, cudaFuncAttributePreferredSharedMemoryCarveout, carve))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_acc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_a<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_a<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_acc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = set_rows16_smem_limits())) return e;
  return set_fft16_smem_limits();
}

// slot: the spectrum slot (0 or 1) the sample's transforms go to.  paths: kColsGeneric
// for the shared-memory kernel, bit b for k_fft_rows16 on rows of nx = 4096 << b (FP32).
// grid: blocks of the shared-memory kernel; the Stockham kernel takes at most two blocks
// per SM of the sms SMs (its blocks loop over their rows)
void launch_fft_rows(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int grid, int block, int smem, cudaStream_t st, int slot,
                     int paths, int sms) {
  if (precision == FLB_FP64) {
    k_fft_rows<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, slot);
    return;
  }
  if (paths & kColsGeneric) k_fft_rows<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, slot);
  const int g16 = (int)std::min<int64_t>((int64_t)grid, 2 * (int64_t)sms);
  for (int b = 0; b < 4; ++b)
    if (paths & (1 << b)) launch_fft_rows16(descs, vb_begin, n_reps, n_vblocks, ws, g16, 4096 << b, st, slot);
}

// paths: kColsGeneric for the shared-memory kernel, bit B for the register-resident
// kernel of columns of 16 B (FP32 only; see cols16_b).  The register-resident pass-2a
// kernel takes one block per field of a (y2, tile) unit (cols_a_units), tiles of kColsA16
// columns; the shared-memory kernel tiles of ncol.
void launch_fft_cols_a(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                       int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st,
                       int paths, int slot, int sms) {
  if (precision == FLB_FP64) {
    k_fft_cols_a<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol, slot);
    return;
  }
  if (paths & kColsGeneric)
    k_fft_cols_a<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol, slot);
  // the pipelined kernel: its resident blocks (4 per SM) loop over their units
  launch_fft_cols_a16(paths & (kColsGeneric - 1), descs, vb_begin, n_reps, n_vblocks, ws,
                      (int)std::min<int64_t>((int64_t)grid, 4 * (int64_t)sms), st, slot);
}

void launch_fft_cols(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st,
                     const TimeCorr& tc, int paths, int nslots, int max_fields) {
  if (precision == FLB_FP64) {
    k_fft_cols_acc<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol, tc);
    return;
  }
  if (paths & kColsGeneric)         // one slot (the host folds samples only without this kernel)
    k_fft_cols_acc<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol, tc);
  launch_fft_cols_acc16(paths & (kColsGeneric - 1), descs, vb_begin, n_reps, n_vblocks, ws, ncol, grid, max_fields, st,
                        tc, nslots);
}

void launch_time_corr(const ReplicaDesc* descs, int n_reps, int max_fields, const TimeCorr& tc, cudaStream_t st) {
  const int64_t items = (int64_t)tc.n_lags * max_fields * max_fields * tc.n_k;
  const int gx = (int)std::min<int64_t>((items + 255) / 256, 4096);
  k_time_corr<<<dim3(gx, n_reps), 256, 0, st>>>(descs, tc);
  k_time_corr_advance<<<(n_reps + 127) / 128, 128, 0, st>>>(tc, n_reps);
}

}  // namespace flb
