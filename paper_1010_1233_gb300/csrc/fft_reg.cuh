// Discrete Fourier transforms of 1, 2, 4, 8 or 16 points held in registers, for the
// register-resident column passes of the correlator sampling (spectra_cols.cu).  The
// transform runs as radix-2 decimation in time on a compile-time index set: the input
// permutation is a renaming of registers, every twiddle is a sixteenth root of unity
// known at compile time (a multiplication by 1 or -i costs nothing, one by (1 - i)/sqrt2
// two multiplications), and no shared memory is touched.
#pragma once
#include "fft_common.cuh"

namespace flb {

// x * exp(-2 pi i m / 16), m in [0, 8); m is a constant after unrolling, so the switch
// folds away
template <typename R>
__device__ __forceinline__ C<R> mul_w16(C<R> x, int m) {
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
  C<R> r;
  switch (m) {
    case 0: r = x; break;
    case 1: r.x = x.x * c1 + x.y * s1; r.y = x.y * c1 - x.x * s1; break;      // (c1, -s1)
    case 2: r.x = h * (x.x + x.y); r.y = h * (x.y - x.x); break;              // (h, -h)
    case 3: r.x = x.x * s1 + x.y * c1; r.y = x.y * s1 - x.x * c1; break;      // (s1, -c1)
    case 4: r.x = x.y; r.y = -x.x; break;                                     // -i
    case 5: r.x = x.y * c1 - x.x * s1; r.y = -(x.x * c1 + x.y * s1); break;   // (-s1, -c1)
    case 6: r.x = h * (x.y - x.x); r.y = -h * (x.x + x.y); break;             // (-h, -h)
    default: r.x = x.y * s1 - x.x * c1; r.y = -(x.x * s1 + x.y * c1); break;  // (-c1, -s1)
  }
  return r;
}

template <int N>
__host__ __device__ constexpr int brev_ct(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
  return r;
}

// In place: v[k] <- sum_n v[n] exp(-2 pi i n k / N), natural order in and out.
// Stage h (half-size h = 1, 2, .., N/2) pairs a[k + j] with a[k + j + h] under the
// twiddle W_2h^j = W_16^(8 j / h).
template <typename R, int N>
__device__ __forceinline__ void dft_reg(C<R> (&v)[N]) {
  static_assert(N == 1 || N == 2 || N == 4 || N == 8 || N == 16, "1 to 16 points");
  if constexpr (N > 1) {
    C<R> a[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = v[brev_ct<N>(i)];
#pragma unroll
    for (int h = 1; h < N; h <<= 1) {
#pragma unroll
      for (int k = 0; k < N; k += 2 * h) {
#pragma unroll
        for (int j = 0; j < h; ++j) {
          const C<R> t = mul_w16<R>(a[k + j + h], j * (8 / h));
          const C<R> u = a[k + j];
          a[k + j].x = u.x + t.x; a[k + j].y = u.y + t.y;
          a[k + j + h].x = u.x - t.x; a[k + j + h].y = u.y - t.y;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = a[i];
  }
}

}  // namespace flb
