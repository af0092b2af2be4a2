// The accumulation step of the correlator sampling (Eq. 12), shared by the column
// kernels of spectra.cu and spectra_cols.cu: once a block holds the full 2D transforms
// X_f(kx, ky) of its tile (all fields, columns kx0 .. kx0 + ncl - 1, ky = k1 + N1 k2 for
// k2 < N2) in shared memory, add X_a X_b^* of every field pair to the FP64 sums, record
// the time-correlator ring entries of the tile's selected wave vectors, and add the
// k = 0 values to the mean sums.  The block may hold the transforms of two consecutive
// samples (nslots = 2, the second slot_elems elements after the first): each sum is then
// read once, gets the first sample's product added and then the second's (the same
// FP64 operations in the same order as two single-sample passes, so the same result),
// and is written once.
#pragma once
#include "fft_common.cuh"

namespace flb {

// Slot of output k2 in a sequence's shared-memory row: k2 itself (PB = 0), or, for the
// register-resident transforms of B = PB threads per sequence, q PB + p for
// k2 = q + 16 p (the slot stage 2 of that transform writes).
template <int PB>
__device__ __forceinline__ int out_slot(int k2) {
  if constexpr (PB == 0) return k2;
  else return ((k2 & 15) * PB) | (k2 >> 4);
}

// The time-correlator ring entries of the tile's selected wave vectors (one sample per
// pass) and the k = 0 values added to the mean sums.
template <typename R, int PB>
__device__ __forceinline__ void tile_tail(const ReplicaDesc& d, char* __restrict__ ws, const C<R>* s, int ss, int rep,
                                          int k1, int kx0, int ncl, int ncol, const TimeCorr& tc, int nslots,
                                          int slot_elems) {
  const int logn1 = d.log2n1, n1 = 1 << logn1, n2 = d.ny >> logn1;
  const int F = (int)d.n_fields;
  // time correlators (one sample per pass): this sample's X_f(k_j) of the selected wave
  // vectors in this tile
  if (tc.base) {
    const int slot = (int)(tc.count[rep] % (uint64_t)tc.n_lags);
    double2* ring = reinterpret_cast<double2*>(tc.base + d.off_tc_ring);
    for (int i = threadIdx.x; i < tc.n_k * F; i += blockDim.x) {
      const int j = i % tc.n_k, f = i / tc.n_k;
      const int kx = tc.kx[j], ky = tc.ky[j];
      if ((ky & (n1 - 1)) != k1 || kx < kx0 || kx >= kx0 + ncl) continue;
      if (!FLB_INB(slot >= 0 && slot < tc.n_lags && (ky >> logn1) < n2, 164)) continue;
      const C<R> X = s[(f * ncol + (kx - kx0)) * ss + out_slot<PB>(ky >> logn1)];
      ring[((int64_t)slot * F + f) * tc.n_k + j] = make_double2((double)X.x, (double)X.y);
    }
  }
  // k = 0 sums for the mean subtraction
  if (k1 == 0 && kx0 == 0 && threadIdx.x == 0) {
    double* m0 = reinterpret_cast<double*>(ws + d.off_mean0);
    for (int f = 0; f < F; ++f)
      for (int k = 0; k < nslots; ++k) m0[f] += (double)s[k * slot_elems + (f * ncol) * ss].x;
  }
}

// Pair sums of a tile, one thread per point (register-resident pass 2b): the point's
// shared-memory slot and its pair-sum index are computed once, each pair's sum is read
// once for the nslots samples, three pairs' reads in flight.
template <int PB>
__device__ __forceinline__ void accumulate_points(const ReplicaDesc& d, char* __restrict__ ws, const float2* s, int ss,
                                                  int k1, int kx0, int ncl, int ncol, int tiles, int nslots,
                                                  int slot_elems) {
  const int lc = 31 - __clz(ncol);
  const int logn1 = d.log2n1, n1 = 1 << logn1, n2 = d.ny >> logn1;
  const int npts = n2 << lc, fstride = ncol * ss, np = d.n_pairs, F = (int)d.n_fields;
  // blocked layout: the tile's points are one contiguous range of every pair's sums
  const int64_t first = (int64_t)(k1 * tiles + (kx0 >> lc)) * n2 * ncol;
  const int64_t limit = d.acc_ncol ? (int64_t)d.ny * tiles * ncol : (int64_t)d.ny * d.half_nx;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) {
    const int c = i & (ncol - 1), k2 = i >> lc;
    if (c >= ncl) continue;
    const int64_t pt = d.acc_ncol ? first + i : (int64_t)(k1 + n1 * k2) * d.half_nx + kx0 + c;
    if (!FLB_INB(pt < limit && c * ss + out_slot<PB>(k2) < fstride, 165)) continue;
    const float2* sp = s + c * ss + out_slot<PB>(k2);
    for (int p0 = 0; p0 < np; p0 += 3) {
      double2 acc[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int pr = p0 + u;
        if (pr >= np) break;
        if (d.pair_a[pr] == d.pair_b[pr]) acc[u].x = reinterpret_cast<const double*>(ws + d.pair_off[pr])[pt];
        else acc[u] = reinterpret_cast<const double2*>(ws + d.pair_off[pr])[pt];
      }
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int pr = p0 + u;
        if (pr >= np) break;
        const int a = d.pair_a[pr], b = d.pair_b[pr];
        if (!FLB_INB(a < F && b < F, 166)) continue;
        // the product in FP32 (exact to its rounding), the sum in FP64, sample by sample
        for (int k = 0; k < nslots; ++k) {
          const float2 Xa = sp[k * slot_elems + a * fstride];
          const float2 Xb = sp[k * slot_elems + b * fstride];
          if (a == b) {
            acc[u].x += widen(Xa.x * Xa.x + Xa.y * Xa.y);
          } else {
            acc[u].x += widen(Xa.x * Xb.x + Xa.y * Xb.y);     // X_a X_b^*
            acc[u].y += widen(Xa.y * Xb.x - Xa.x * Xb.y);
          }
        }
        if (a == b) reinterpret_cast<double*>(ws + d.pair_off[pr])[pt] = acc[u].x;
        else reinterpret_cast<double2*>(ws + d.pair_off[pr])[pt] = acc[u];
      }
    }
  }
}

// s: the tile's transforms, sequence (f, c) at s + (f ncol + c) ss; all threads call it.
template <typename R, int PB>
__device__ __forceinline__ void accumulate_tile(const ReplicaDesc& d, char* __restrict__ ws, const C<R>* s, int ss,
                                                int rep, int k1, int kx0, int ncl, int ncol, int tiles,
                                                const TimeCorr& tc, int nslots = 1, int slot_elems = 0) {
  const int lc = 31 - __clz(ncol);
  const int logn1 = d.log2n1, n1 = 1 << logn1, logn2 = d.log2ny - logn1, n2 = d.ny >> logn1;
  const int F = (int)d.n_fields;
  // pair products in FP64: one work item per (pair, point) of the block, pair-major so
  // that a warp works on one pair (uniform auto/cross branch) and 32 consecutive points;
  // four items per thread are loaded before any is stored
  const int lp = lc + logn2, npts = 1 << lp;
  const int items = d.n_pairs << lp;
  for (int it0 = threadIdx.x; it0 < items; it0 += 4 * blockDim.x) {
    double2 acc[4];
    int64_t pt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int it = it0 + u * blockDim.x;
      const int pr = it >> lp, i = it & (npts - 1);
      const int c = i & (ncol - 1), k2 = i >> lc;
      pt[u] = -1;
      if (it >= items || c >= ncl) continue;
      pt[u] = d.acc_ncol ? ((int64_t)(k1 * tiles + (kx0 >> lc)) * n2 + k2) * ncol + c   // contiguous per block
                         : (int64_t)(k1 + n1 * k2) * d.half_nx + kx0 + c;
      if (!FLB_INB(pr < d.n_pairs && d.pair_a[pr] < F && d.pair_b[pr] < F &&
                   pt[u] < (d.acc_ncol ? (int64_t)d.ny * tiles * ncol : (int64_t)d.ny * d.half_nx), 163)) {
        pt[u] = -1;
        continue;
      }
      if (d.pair_a[pr] == d.pair_b[pr]) acc[u].x = reinterpret_cast<const double*>(ws + d.pair_off[pr])[pt[u]];
      else acc[u] = reinterpret_cast<const double2*>(ws + d.pair_off[pr])[pt[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (pt[u] < 0) continue;
      const int it = it0 + u * blockDim.x;
      const int pr = it >> lp, i = it & (npts - 1);
      const int c = i & (ncol - 1), k2 = i >> lc;
      const int a = d.pair_a[pr], b = d.pair_b[pr];
      // the product in the transform's precision (exact to its rounding), the sum in FP64
      for (int k = 0; k < nslots; ++k) {
        const C<R> Xa = s[k * slot_elems + (a * ncol + c) * ss + out_slot<PB>(k2)];
        const C<R> Xb = s[k * slot_elems + (b * ncol + c) * ss + out_slot<PB>(k2)];
        if (a == b) {
          acc[u].x += widen(Xa.x * Xa.x + Xa.y * Xa.y);
        } else {
          acc[u].x += widen(Xa.x * Xb.x + Xa.y * Xb.y);     // X_a X_b^*
          acc[u].y += widen(Xa.y * Xb.x - Xa.x * Xb.y);
        }
      }
      if (a == b) reinterpret_cast<double*>(ws + d.pair_off[pr])[pt[u]] = acc[u].x;
      else reinterpret_cast<double2*>(ws + d.pair_off[pr])[pt[u]] = acc[u];
    }
  }
  tile_tail<R, PB>(d, ws, s, ss, rep, k1, kx0, ncl, ncol, tc, nslots, slot_elems);
}

}  // namespace flb
