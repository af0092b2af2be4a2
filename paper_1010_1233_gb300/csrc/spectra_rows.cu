// Row pass of the correlator sampling (Eq. 11) in FP32 for rows of nx = 2 M points,
// M = 2048 .. 16384: one real row per block.  The row is transformed as the complex
// sequence z(n) = x(2n) + i x(2n + 1) of length M, then split into the half spectrum
// X(k), k = 0 .. M, of the real row: with E(k) = (Z(k) + Z(M - k)^*) / 2 (the transform
// of the even samples) and O(k) = (Z(k) - Z(M - k)^*) / (2i) (the odd ones),
//   X(k) = E(k) + W_nx^k O(k),   X(M - k) = (E(k) - W_nx^k O(k))^*.
// The length-M transform runs as Stockham passes in shared memory, natural order in and
// out: with sub-transforms of length Ns (1, 16, 256, ..) combined R at a time, work item
// j < M / R takes v(r) = S(j + r M / R), multiplies by W_(R Ns)^((j mod Ns) r), transforms
// over r in registers (fft_reg.cuh) and writes S((j - j mod Ns) R + j mod Ns + r Ns).
// Passes of R = 16, then one of 2, 4 or 8 for the remaining factor.  A work item reads
// the twiddle table four times (W^e, W^2e, W^4e, W^8e) and forms the other powers by
// complex products.  M / 16 threads, 16 values each; every pass reads all its values
// before the barrier and writes after it, so one buffer serves (element i at i + i / 16,
// which keeps the stride-16 writes of the first pass off a single bank).  The first
// pass reads the row from global memory; the split writes the half spectrum in the
// replica's spectrum layout (spec_index).
#include "fft_reg.cuh"

namespace flb {

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// W_nx^e for e < nx from the half table tw (exp(-2 pi i m / nx), m < nx / 2)
__device__ __forceinline__ float2 tw_full(const float2* __restrict__ tw, int nx, int e) {
  const int h = nx >> 1;
  float2 w = __ldg(&tw[e < h ? e : e - h]);
  if (e >= h) { w.x = -w.x; w.y = -w.y; }
  return w;
}

// w[r] = W^(e r), r < R, from the table values of W^e, W^2e, W^4e, W^8e (as many as R
// needs) and products of them: at most three roundings on top of the table's
template <int R>
__device__ __forceinline__ void twiddle_powers(const float2* __restrict__ tw, int nx, int e, float2 (&w)[R]) {
  w[0] = make_float2(1.f, 0.f);
  if constexpr (R > 1) w[1] = tw_full(tw, nx, e);
  if constexpr (R > 2) { w[2] = tw_full(tw, nx, 2 * e); w[3] = cmul<float>(w[2], w[1]); }
  if constexpr (R > 4) {
    w[4] = tw_full(tw, nx, 4 * e);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul<float>(w[4], w[r - 4]);
  }
  if constexpr (R > 8) {
    w[8] = tw_full(tw, nx, 8 * e);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul<float>(w[8], w[r - 8]);
  }
}

// one Stockham pass of radix R over sub-transforms of length Ns (Ns > 1)
template <int R>
__device__ __forceinline__ void stockham_pass(float2* S, int M, int Ns, const float2* __restrict__ tw, int nx) {
  constexpr int G = 16 / R;                            // work items per thread
  const int T = blockDim.x, step = nx / (R * Ns);
  float2 v[G][R];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = threadIdx.x + g * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[g][r] = S[pad16(j + r * (M / R))];
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = threadIdx.x + g * T;
    const int jm = j & (Ns - 1);
    float2 w[R];
    twiddle_powers<R>(tw, nx, jm * step, w);            // W_(R Ns)^(jm r); jm r step < nx
#pragma unroll
    for (int r = 1; r < R; ++r) v[g][r] = cmul<float>(v[g][r], w[r]);
    dft_reg<float, R>(v[g]);
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (FLB_INB(base + r * Ns < M, 221)) S[pad16(base + r * Ns)] = v[g][r];
  }
  __syncthreads();
}

// One block per (replica, field, row) unit; blockDim.x = M / 16.
__global__ void __launch_bounds__(1024, 1)
k_fft_rows16(const ReplicaDesc* __restrict__ descs, const int64_t* __restrict__ vb_begin, int n_reps,
             int64_t n_vblocks, char* __restrict__ ws, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int rp = find_rep(vb_begin, n_reps, vb);
    const ReplicaDesc& d = descs[rp];
    const int nx = d.nx, M = nx >> 1;
    if (!rows16_nx(nx) || (M >> 4) != (int)blockDim.x) continue;   // another launch's row
    const int64_t u = vb - vb_begin[rp];
    const int f = (int)(u >> d.log2ny), y = (int)(u & (d.ny - 1));
    if (!FLB_INB(f < (int)d.n_fields, 222)) continue;
    const float* x = reinterpret_cast<const float*>(ws + d.off_fields) + ((int64_t)f * d.ny + y) * nx;
    const float2* tw = reinterpret_cast<const float2*>(ws + d.off_tw_x);
    // the block's next row into L2 while this one is transformed
    if (threadIdx.x == 0 && vb + gridDim.x < n_vblocks) {
      const int64_t vn = vb + gridDim.x;
      const int rn = find_rep(vb_begin, n_reps, vn);
      const ReplicaDesc& dn = descs[rn];
      const int64_t un = vn - vb_begin[rn];
      if (un < (int64_t)dn.n_fields << dn.log2ny)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     :: "l"(reinterpret_cast<const float*>(ws + dn.off_fields) + un * dn.nx), "r"((uint32_t)dn.nx * 4u)
                     : "memory");
    }
    // first pass (Ns = 1, R = 16) straight from the row
    {
      const int j = threadIdx.x;
      const float2* z = reinterpret_cast<const float2*>(x);
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = z[j + r * (M >> 4)];
      dft_reg<float, 16>(v);
#pragma unroll
      for (int r = 0; r < 16; ++r) S[pad16(j * 16 + r)] = v[r];
      __syncthreads();
    }
    int Ns = 16;
    for (; Ns * 16 <= M; Ns *= 16) stockham_pass<16>(S, M, Ns, tw, nx);
    if (M / Ns == 8) stockham_pass<8>(S, M, Ns, tw, nx);
    else if (M / Ns == 4) stockham_pass<4>(S, M, Ns, tw, nx);
    else if (M / Ns == 2) stockham_pass<2>(S, M, Ns, tw, nx);
    // the half spectrum of the real row
    float2* out = reinterpret_cast<float2*>(ws + d.off_spec + slot * d.spec_slot);
    const bool ok = FLB_INB(spec_index(d, f, y, M) < spec_elems(d), 223);
    for (int k = threadIdx.x; k <= (M >> 1) && ok; k += blockDim.x) {
      const float2 A = S[pad16(k)], Bv = S[pad16((M - k) & (M - 1))];
      const float2 E = make_float2(0.5f * (A.x + Bv.x), 0.5f * (A.y - Bv.y));
      const float2 O = make_float2(0.5f * (A.y + Bv.y), 0.5f * (Bv.x - A.x));   // (A - Bv^*) / (2i)
      const float2 WO = cmul<float>(__ldg(&tw[k]), O);                          // k <= nx / 4
      out[spec_index(d, f, y, k)] = make_float2(E.x + WO.x, E.y + WO.y);
      if (k != M - k) out[spec_index(d, f, y, M - k)] = make_float2(E.x - WO.x, WO.y - E.y);
    }
    __syncthreads();
  }
}

void launch_fft_rows16(const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps, int64_t n_vblocks, char* ws,
                       int grid, int nx, cudaStream_t st, int slot) {
  const int M = nx / 2;
  const int smem = (M + M / 16) * (int)sizeof(float2);     // fft_rows_smem
  k_fft_rows16<<<grid, M / 16, smem, st>>>(descs, vb_begin, n_reps, n_vblocks, ws, slot);
}

// Shared memory for two blocks of 8192-point rows (2 x 69.6 KB) and the rest as L1, which
// then holds the twiddle table of a 16384-point row (64 KB) that the passes read.
cudaError_t set_rows16_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_rows16, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (!e) e = cudaFuncSetAttribute(k_fft_rows16, cudaFuncAttributePreferredSharedMemoryCarveout, 64);
  return e;
}

}  // namespace flb
