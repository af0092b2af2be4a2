// Radix-2 FFT building blocks shared by the correlator sampling kernels (spectra.cu)
// and the fused D1Q3 kernel (lb_d1q3_fused.cu): complex helpers, exact FP32 -> FP64
// widening, and in-place decimation-in-time transforms in shared memory.
#pragma once
#include "flb_internal.cuh"

namespace flb {

template <typename R> using C = typename vec2_of<R>::type;

// the replica of virtual block vb (vb_begin: each replica's first block, ascending)
__device__ __forceinline__ int find_rep(const int64_t* vb_begin, int n_reps, int64_t vb) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (vb_begin[mid] <= vb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Exact widening to FP64 with integer operations (GB300's FP64 pipe is slow, and the
// accumulation pass is bound by it), on the two 32-bit halves of the double: the high
// word takes the sign, the exponent rebiased by 1023 - 127 = 896 (0x380 << 20; 0x7FF for
// infinities and NaN) and the top 20 significand bits, the low word the last 3.  Zero
// and subnormal floats give a signed zero (a subnormal product is below 1.2e-38 and
// cannot change an FP64 sum of such correlators).
__device__ __forceinline__ double widen(float x) {
  const uint32_t b = __float_as_uint(x), a = b & 0x7FFFFFFFu;
  uint32_t hi = (a >> 3) + (a >= 0x7F800000u ? 0x70000000u : 0x38000000u);
  uint32_t lo = b << 29;
  if (a < 0x00800000u) { hi = 0u; lo = 0u; }
  hi |= b & 0x80000000u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double x) { return x; }

template <typename R> __device__ __forceinline__ C<R> cmul(C<R> a, C<R> b) {
  C<R> r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// w * exp(-2 pi i u / 2^(st+1)) for st <= 2 (u < 2^st): multiplication by an eighth
// root of unity (exact for 1 and -i)
template <typename R>
__device__ __forceinline__ C<R> rot8(C<R> w, int st, int u) {
  const int e = u << (2 - st);                        // exponent in units of -2 pi i / 8
  C<R> r = w;
  if (e == 2) { r.x = w.y; r.y = -w.x; }              // * (-i)
  else if (e == 1 || e == 3) {
    const R h = (R)0.70710678118654752440;            // * (1 - i)/sqrt2, * (-1 - i)/sqrt2
    if (e == 1) { r.x = h * (w.x + w.y); r.y = h * (w.y - w.x); }
    else { r.x = h * (w.y - w.x); r.y = -h * (w.x + w.y); }
  }
  return r;
}

// w * exp(-2 pi i u / 2^(st+1)) for st <= 3 (u < 2^st): odd sixteenth roots of unity
// by a complex multiplication with cos(pi/8), sin(pi/8), the others through rot8
template <typename R>
__device__ __forceinline__ C<R> rot16(C<R> w, int st, int u) {
  if (st < 3) return rot8<R>(w, st, u);
  if ((u & 1) == 0) return rot8<R>(w, 2, u >> 1);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
  C<R> z;                                             // exp(-2 pi i u / 16), u = 1, 3, 5, 7
  z.x = u == 1 ? c1 : (u == 3 ? s1 : (u == 5 ? -s1 : -c1));
  z.y = u == 1 ? -s1 : (u == 3 ? -c1 : (u == 5 ? -c1 : -s1));
  return cmul<R>(w, z);
}

// The butterflies of RS consecutive radix-2 decimation-in-time stages s .. s + RS - 1
// on a group of 2^RS elements held in registers: v[t] is element i0 + t 2^s of the
// sequence, where i0 has bits s .. s+RS-1 clear and low = i0 mod 2^s.  Stage S = s + st
// pairs t with t + 2^st and multiplies by exp(-2 pi i pos / 2^(S+1)),
// pos = low + (t mod 2^st) 2^s, i.e. the base twiddle exp(-2 pi i low / 2^(S+1)) (one
// table read per stage) times an eighth (sixteenth for RS = 4) root of unity.
template <typename R, int RS>
__device__ __forceinline__ void dit_group(C<R> (&v)[1 << RS], int logn, int s, int low,
                                          const C<R>* __restrict__ tw, int tw_stride) {
#pragma unroll
  for (int st = 0; st < RS; ++st) {
    const C<R> base = __ldg(&tw[(low << (logn - 1 - s - st)) * tw_stride]);
#pragma unroll
    for (int t = 0; t < (1 << RS); ++t) {
      if (t & (1 << st)) continue;
      const C<R> w = rot16<R>(base, st, t & ((1 << st) - 1));
      const C<R> a = v[t];
      const C<R> tt = cmul<R>(v[t + (1 << st)], w);
      v[t].x = a.x + tt.x; v[t].y = a.y + tt.y;
      v[t + (1 << st)].x = a.x - tt.x; v[t + (1 << st)].y = a.y - tt.y;
    }
  }
}

// RS consecutive stages in one pass through shared memory: each thread takes groups of
// 2^RS elements closed under those stages, keeps them in registers through the RS stages
// and writes them back (one barrier per RS stages).  Work item g = q n_fft + k (group q of
// sequence k): neighbouring threads take the same group of neighbouring sequences, so with
// an odd seq_stride their accesses fall in distinct banks and they share the twiddles.
template <typename R, int RS>
__device__ __forceinline__ void dit_pass(C<R>* data, int logn, int n_fft, int seq_stride,
                                         const C<R>* __restrict__ tw, int tw_stride, int pad_shift, int s) {
  constexpr int G = 1 << RS;
  const int lg = logn - RS;                          // log2 of the groups per sequence
  const int groups = 1 << lg;
  int q = (int)threadIdx.x / n_fft, k = (int)threadIdx.x - q * n_fft;
  const int dq = (int)blockDim.x / n_fft, dk = (int)blockDim.x - dq * n_fft;
  for (; q < groups;) {
    const int low = q & ((1 << s) - 1);
    const int i0 = ((q >> s) << (s + RS)) | low;
    C<R>* d = data + k * seq_stride;
    C<R> v[G];
    // (checked build: the group's last element inside the sequence, a valid sequence)
    const bool ok = FLB_INB(k < n_fft && i0 + ((G - 1) << s) < (1 << logn), 141);
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int e = i0 + (t << s);
      v[t] = ok ? d[e + (e >> pad_shift)] : C<R>{};
    }
    dit_group<R, RS>(v, logn, s, low, tw, tw_stride);
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int e = i0 + (t << s);
      if (ok) d[e + (e >> pad_shift)] = v[t];
    }
    q += dq;                                         // g += blockDim.x
    k += dk;
    if (k >= n_fft) { k -= n_fft; ++q; }
  }
}

// In-place radix-2 decimation-in-time FFTs on n_fft sequences of length 2^logn in
// shared memory, sequence k at data + k * seq_stride, already in bit-reversed order.
// tw[m * tw_stride] = exp(-2 pi i m / 2^logn), m < 2^(logn-1).  Element i of a sequence is
// stored at i + (i >> pad_shift) (one pad slot per 2^pad_shift elements, so that the
// bit-reversed scatter does not hit one bank).  Stages s0 .. logn - 1 run MAXRS at a
// time (dit_pass).  All threads of the block call it.
template <typename R, int MAXRS = 3>
__device__ void dit_fft(C<R>* data, int logn, int n_fft, int seq_stride, const C<R>* __restrict__ tw,
                        int tw_stride, int pad_shift = 31, int s0 = 0) {
  static_assert(MAXRS == 3 || MAXRS == 4, "three or four stages per pass");
  for (int s = s0; s < logn;) {
    const int rs = logn - s >= MAXRS ? MAXRS : logn - s;
    if (rs == 4) dit_pass<R, (MAXRS == 4 ? 4 : 3)>(data, logn, n_fft, seq_stride, tw, tw_stride, pad_shift, s);
    else if (rs == 3) dit_pass<R, 3>(data, logn, n_fft, seq_stride, tw, tw_stride, pad_shift, s);
    else if (rs == 2) dit_pass<R, 2>(data, logn, n_fft, seq_stride, tw, tw_stride, pad_shift, s);
    else dit_pass<R, 1>(data, logn, n_fft, seq_stride, tw, tw_stride, pad_shift, s);
    s += rs;
    __syncthreads();
  }
}

__device__ __forceinline__ int brev(int i, int logn) {
  return logn == 0 ? 0 : (int)(__brev((unsigned)i) >> (32 - logn));
}

}  // namespace flb
