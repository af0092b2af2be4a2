// Correlator sampling (Eqs. 11-12): 2D discrete Fourier transform of the
// sampled real fields with a hand-written radix-2 FFT, and FP64 accumulation
// of X_a(k) X_b(k)^* for every sampled field pair on the half spectrum
// kx in [0, nx/2] (the other half follows from X(-k) = X(k)^* for real fields).
//
// Pass 1 (rows): two real fields are packed as one complex row z = X_a + i X_b,
// transformed along x in shared memory, and unpacked into the row transforms
// of both fields, X_a(kx) = (Z(kx) + Z(-kx)^*)/2, X_b(kx) = (Z(kx) - Z(-kx)^*)/(2i).
// Pass 2 (columns): tiles of columns of every field are transformed along y in
// shared memory and the pair products are added to the FP64 sums.  Columns too
// long for shared memory use the four-step split ny = N1 N2, y = N2 y1 + y2,
// ky = k1 + N1 k2:  X(ky) = sum_y2 W_N2^(y2 k2) W_N^(y2 k1) sum_y1 W_N1^(y1 k1) x(y);
// pass 2a does the inner length-N1 transforms and the W_N^(y2 k1) twiddle in
// place (rows N2 y1 + y2 -> N2 k1 + y2), pass 2b the outer length-N2 transforms.
#include "flb_internal.cuh"

namespace flb {

template <typename R> using C = typename vec2_of<R>::type;

template <typename R> __device__ __forceinline__ C<R> cmul(C<R> a, C<R> b) {
  C<R> r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// In-place radix-2 decimation-in-time FFTs on n_fft sequences of length 2^logn in
// shared memory, sequence k at data + k * seq_stride, already in bit-reversed order.
// tw[m * tw_stride] = exp(-2 pi i m / 2^logn), m < 2^(logn-1).  Element i of a sequence is
// stored at i + (i >> pad_shift) (one pad slot per 2^pad_shift elements, so that the
// bit-reversed scatter does not hit one bank).  All threads of the block call it.
template <typename R>
__device__ void dit_fft(C<R>* data, int logn, int n_fft, int seq_stride, const C<R>* __restrict__ tw,
                        int tw_stride, int pad_shift = 31) {
  if (logn == 0) return;
  const int half_n = 1 << (logn - 1);
  const int total = n_fft * half_n;
  for (int s = 0; s < logn; ++s) {
    const int half = 1 << s;
    const int tshift = logn - 1 - s;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int k = b >> (logn - 1);
      const int j = b & (half_n - 1);
      const int pos = j & (half - 1);
      const int i0 = ((j >> s) << (s + 1)) + pos;
      C<R>* d = data + k * seq_stride;
      const C<R> w = tw[(pos << tshift) * tw_stride];
      const int p0 = i0 + (i0 >> pad_shift), p1 = i0 + half + ((i0 + half) >> pad_shift);
      const C<R> a = d[p0];
      const C<R> t = cmul<R>(d[p1], w);
      C<R> u, v;
      u.x = a.x + t.x; u.y = a.y + t.y;
      v.x = a.x - t.x; v.y = a.y - t.y;
      d[p0] = u; d[p1] = v;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev(int i, int logn) {
  return logn == 0 ? 0 : (int)(__brev((unsigned)i) >> (32 - logn));
}

__device__ __forceinline__ int find_rep(const int64_t* vb_begin, int n_reps, int64_t vb) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (vb_begin[mid] <= vb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pass 1: one block per (replica, packed field pair, row).
template <typename R>
__global__ void k_fft_rows(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                           int n_reps, int64_t n_vblocks, char* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* z = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int64_t local = vb - vb_begin[r];
    const int y = (int)(local % d.ny);
    const int p = (int)(local / d.ny);
    const int fa = 2 * p, fb = 2 * p + 1;
    const bool has_b = fb < (int)d.n_fields;
    const int nx = d.nx, logn = d.log2nx;
    const int64_t plane = (int64_t)nx * d.ny;
    const R* fields = reinterpret_cast<const R*>(ws + d.off_fields);
    const R* xa = fields + fa * plane + (int64_t)y * nx;
    const R* xb = fields + fb * plane + (int64_t)y * nx;
    const int ps = logn > 5 ? logn - 5 : 31;        // 32 pad slots per row
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      C<R> v; v.x = xa[x]; v.y = has_b ? xb[x] : (R)0;
      const int i = brev(x, logn);
      z[i + (i >> ps)] = v;
    }
    __syncthreads();
    dit_fft<R>(z, logn, 1, 0, reinterpret_cast<const C<R>*>(ws + d.off_tw_x), 1, ps);
    C<R>* spec = reinterpret_cast<C<R>*>(ws + d.off_spec);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    C<R>* ra = spec + fa * fplane + (int64_t)y * d.wpitch;
    C<R>* rb = spec + fb * fplane + (int64_t)y * d.wpitch;
    const int hn = nx >> 1;
    for (int k = threadIdx.x; k <= hn; k += blockDim.x) {
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
__global__ void k_fft_cols_a(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                             int n_reps, int64_t n_vblocks, char* __restrict__ ws, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* s = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int tiles = (d.half_nx + ncol - 1) / ncol;
    const int64_t local = vb - vb_begin[r];
    const int y2 = (int)(local / tiles);
    const int kx0 = (int)(local % tiles) * ncol;
    const int ncl = min(ncol, d.half_nx - kx0);
    const int logn1 = d.log2n1, n1 = 1 << logn1, n2 = d.ny >> logn1, F = (int)d.n_fields;
    C<R>* spec = reinterpret_cast<C<R>*>(ws + d.off_spec);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    const int total = F * n1 * ncol;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int c = i % ncol;
      const int y1 = (i / ncol) % n1;
      const int f = i / (ncol * n1);
      C<R> v; v.x = (R)0; v.y = (R)0;
      if (c < ncl) v = spec[f * fplane + (int64_t)(n2 * y1 + y2) * d.wpitch + kx0 + c];
      s[(f * ncol + c) * (n1 + 1) + brev(y1, logn1)] = v;
    }
    __syncthreads();
    const C<R>* tw = reinterpret_cast<const C<R>*>(ws + d.off_tw_y);
    dit_fft<R>(s, logn1, F * ncol, n1 + 1, tw, n2);
    const int hn = d.ny >> 1;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int c = i % ncol;
      const int k1 = (i / ncol) % n1;
      const int f = i / (ncol * n1);
      if (c >= ncl) continue;
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
__global__ void k_fft_cols_acc(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin,
                               int n_reps, int64_t n_vblocks, char* __restrict__ ws, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* s = reinterpret_cast<C<R>*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[r];
    const int tiles = (d.half_nx + ncol - 1) / ncol;
    const int64_t local = vb - vb_begin[r];
    const int k1 = (int)(local / tiles);
    const int kx0 = (int)(local % tiles) * ncol;
    const int logn1 = d.log2n1, n1 = 1 << logn1, logn2 = d.log2ny - logn1, n2 = d.ny >> logn1;
    const int F = (int)d.n_fields;
    const int ncl = min(ncol, d.half_nx - kx0);
    const C<R>* spec = reinterpret_cast<const C<R>*>(ws + d.off_spec);
    const int64_t fplane = (int64_t)d.ny * d.wpitch;
    // smem layout: [field][column][n2]
    const int total = F * n2 * ncol;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int c = i % ncol;
      const int y2 = (i / ncol) % n2;
      const int f = i / (ncol * n2);
      C<R> v; v.x = (R)0; v.y = (R)0;
      if (c < ncl) v = spec[f * fplane + (int64_t)(n2 * k1 + y2) * d.wpitch + kx0 + c];
      s[(f * ncol + c) * (n2 + 1) + brev(y2, logn2)] = v;
    }
    __syncthreads();
    dit_fft<R>(s, logn2, F * ncol, n2 + 1, reinterpret_cast<const C<R>*>(ws + d.off_tw_y), n1);
    // accumulate pair products in FP64; k = 0 sums for the mean subtraction
    const int npts = n2 * ncol;
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
      const int c = i % ncol;
      const int k2 = i / ncol;
      if (c >= ncl) continue;
      const int kx = kx0 + c;
      const int ky = k1 + n1 * k2;
      const int64_t pt = (int64_t)ky * d.half_nx + kx;
      for (int pr = 0; pr < d.n_pairs; ++pr) {
        const int a = d.pair_a[pr], b = d.pair_b[pr];
        const C<R> Xa = s[(a * ncol + c) * (n2 + 1) + k2];
        const C<R> Xb = s[(b * ncol + c) * (n2 + 1) + k2];
        // the product in the transform's precision (exact to its rounding), the sum in FP64
        if (a == b) {
          double* acc = reinterpret_cast<double*>(ws + d.pair_off[pr]);
          acc[pt] += (double)(Xa.x * Xa.x + Xa.y * Xa.y);
        } else {
          double2* acc = reinterpret_cast<double2*>(ws + d.pair_off[pr]);
          double2 v = acc[pt];
          v.x += (double)(Xa.x * Xb.x + Xa.y * Xb.y);          // X_a X_b^*
          v.y += (double)(Xa.y * Xb.x - Xa.x * Xb.y);
          acc[pt] = v;
        }
      }
      if (kx == 0 && ky == 0) {
        double* m0 = reinterpret_cast<double*>(ws + d.off_mean0);
        for (int f = 0; f < F; ++f) m0[f] += (double)s[(f * ncol + c) * (n2 + 1)].x;
      }
    }
    __syncthreads();
  }
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
void launch_twiddles(int precision, void* tw, int n, cudaStream_t st) {
  if (n < 2) return;
  const int half = n / 2;
  if (precision == FLB_FP64)
    k_twiddles<double><<<(half + 255) / 256, 256, 0, st>>>(reinterpret_cast<double2*>(tw), n);
  else
    k_twiddles<float><<<(half + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2*>(tw), n);
}

int fft_rows_smem(int precision, int nx) { return (nx + 32) * (precision == FLB_FP64 ? 16 : 8); }
int fft_cols_smem(int precision, int F, int ny, int ncol) { return F * (ny + 1) * ncol * (precision == FLB_FP64 ? 16 : 8); }

cudaError_t set_fft_smem_limits() {
  cudaError_t e;
  const int maxb = 227 * 1024;
  if ((e = cudaFuncSetAttribute(k_fft_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_acc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_a<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  if ((e = cudaFuncSetAttribute(k_fft_cols_a<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb))) return e;
  return cudaFuncSetAttribute(k_fft_cols_acc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
}

void launch_fft_rows(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int grid, int block, int smem, cudaStream_t st) {
  if (precision == FLB_FP64)
    k_fft_rows<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws);
  else
    k_fft_rows<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws);
}

void launch_fft_cols_a(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                       int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st) {
  if (precision == FLB_FP64)
    k_fft_cols_a<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol);
  else
    k_fft_cols_a<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol);
}

void launch_fft_cols(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st) {
  if (precision == FLB_FP64)
    k_fft_cols_acc<double><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol);
  else
    k_fft_cols_acc<float><<<grid, block, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, ncol);
}

}  // namespace flb
