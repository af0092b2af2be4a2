// D1Q3 steps and their correlator sampling fused into one launch.
//
// The one-dimensional lattices are small (L = 64 in the D1Q3 workload): as separate
// launches per step (step, row transform, pair accumulation) they are bound by launch
// latency, not by the GPU.  Here one block per replica keeps the populations (both
// buffers), the sampled fields and the row transforms in shared memory for a run of
// steps and touches global memory only for the FP64 pair sums (Eqs. 11-12), the final
// state and the fields of the last sample.  Each step is d1q3_site (d1q3_common.cuh) and each sample the packed row
// transform of k_fft_rows and the pair products of k_fft_cols_acc (spectra.cu) with the
// same building blocks (fft_common.cuh) in the same order, so the results match the
// separate launches.
#include <algorithm>
#include "d1q3_common.cuh"
#include "fft_common.cuh"

namespace flb {

constexpr int kD1q3FusedThreads = 256;

__host__ __device__ constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory of one block: populations [2][3][nx], fields [F][nx], the packed row
// [nx + 32] (complex), the row transforms [F][nx/2 + 1] (complex).
size_t d1q3_fused_smem(int precision, int nx, int F) {
  const size_t rs = precision == FLB_FP64 ? 8 : 4, cs = 2 * rs;
  return a16(6 * (size_t)nx * rs) + a16((size_t)F * nx * rs) + a16(((size_t)nx + 32) * cs) +
         a16((size_t)F * (nx / 2 + 1) * cs);
}

// Steps t0 .. t0 + n_steps - 1 of every replica (block r = replica r), sampling at the
// steps with t % every == 0 (every = 0: none).  Reads the state from the population
// buffer of parity t0 & 1 and leaves it in the buffer of parity (t0 + n_steps) & 1.
template <typename R, bool DEV>
__global__ void __launch_bounds__(kD1q3FusedThreads)
k_d1q3_fused(const ReplicaDesc* __restrict__ descs, char* __restrict__ ws, uint64_t t0, uint32_t n_steps,
             uint32_t every) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ReplicaDesc& d = descs[blockIdx.x];
  const int nx = d.nx, F = (int)d.n_fields, tid = (int)threadIdx.x, nt = (int)blockDim.x;
  unsigned char* sp = smem_raw;
  R* pop = reinterpret_cast<R*>(sp);
  sp += a16(6 * (size_t)nx * sizeof(R));
  R* fld = reinterpret_cast<R*>(sp);
  sp += a16((size_t)F * nx * sizeof(R));
  C<R>* z = reinterpret_cast<C<R>*>(sp);
  sp += a16(((size_t)nx + 32) * sizeof(C<R>));
  C<R>* X = reinterpret_cast<C<R>*>(sp);
  const int hn1 = nx / 2 + 1;                    // half spectrum kx = 0 .. nx/2

  const R* g_src = reinterpret_cast<const R*>(ws + d.off_pop[(int)(t0 & 1)]);
  for (int i = tid; i < 3 * nx; i += nt) pop[i] = g_src[i];
  __syncthreads();

  bool sampled = false;
  for (uint32_t s = 0; s < n_steps; ++s) {
    const uint64_t t = t0 + s;
    const bool sample = every != 0 && F > 0 && t % every == 0;
    sampled = sampled || sample;
    const R* src = pop + (s & 1) * 3 * nx;
    R* dst = pop + ((s & 1) ^ 1) * 3 * nx;
    if (sample) {
      for (int x = tid; x < nx; x += nt) d1q3_site<R, DEV, true>(d, src, dst, fld, nx, x, (uint32_t)t);
    } else {
      for (int x = tid; x < nx; x += nt) d1q3_site<R, DEV, false>(d, src, dst, nullptr, nx, x, (uint32_t)t);
    }
    __syncthreads();
    if (!sample) continue;

    // row transforms of the fields, two per complex transform (k_fft_rows with ny = 1)
    const int logn = d.log2nx;
    const int ps = logn > 5 ? logn - 5 : 31;
    const C<R>* tw = reinterpret_cast<const C<R>*>(ws + d.off_tw_x);
    for (int fa = 0; fa < F; fa += 2) {
      const int fb = fa + 1;
      const bool has_b = fb < F;
      const R* xa = fld + (size_t)fa * nx;
      const R* xb = fld + (size_t)(has_b ? fb : fa) * nx;
      if (logn >= 3) {
        const int n8 = nx >> 3;
        for (int x0 = tid; x0 < n8; x0 += nt) {
          C<R> v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int x = x0 + (((q & 1) << 2) | (q & 2) | ((q >> 2) & 1)) * n8;
            v[q].x = xa[x];
            v[q].y = has_b ? xb[x] : (R)0;
          }
          dit_group<R, 3>(v, logn, 0, 0, tw, 1);
          const int i0 = brev(x0, logn - 3) << 3;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (FLB_INB(i0 + q < nx, 181)) z[i0 + q + ((i0 + q) >> ps)] = v[q];
        }
        __syncthreads();
        dit_fft<R, sizeof(R) == 4 ? 4 : 3>(z, logn, 1, 0, tw, 1, ps, 3);
      } else {
        for (int x = tid; x < nx; x += nt) {
          C<R> v;
          v.x = xa[x];
          v.y = has_b ? xb[x] : (R)0;
          const int i = brev(x, logn);
          if (FLB_INB(i < nx, 181)) z[i + (i >> ps)] = v;
        }
        __syncthreads();
        dit_fft<R>(z, logn, 1, 0, tw, 1, ps);
      }
      for (int k = tid; k < hn1; k += nt) {
        const int km = (nx - k) & (nx - 1);
        const C<R> Zk = z[k + (k >> ps)];
        const C<R> Zm = z[km + (km >> ps)];
        C<R> A;
        A.x = (R)0.5 * (Zk.x + Zm.x);
        A.y = (R)0.5 * (Zk.y - Zm.y);
        X[(size_t)fa * hn1 + k] = A;
        if (has_b) {            // (Z - conj(Zm)) / (2i)
          C<R> B;
          B.x = (R)0.5 * (Zk.y + Zm.y);
          B.y = (R)0.5 * (Zm.x - Zk.x);
          X[(size_t)fb * hn1 + k] = B;
        }
      }
      __syncthreads();          // z is reused by the next pair; X is complete after the last
    }

    // FP64 pair sums (k_fft_cols_acc with ny = 1: the column transform is the identity)
    const int items = (int)d.n_pairs * hn1;
    for (int it = tid; it < items; it += nt) {
      const int pr = it / hn1, kx = it - pr * hn1;
      const int a = d.pair_a[pr], b = d.pair_b[pr];
      if (!FLB_INB(pr < d.n_pairs && a < F && b < F, 182)) continue;
      const C<R> Xa = X[(size_t)a * hn1 + kx];
      const C<R> Xb = X[(size_t)b * hn1 + kx];
      if (a == b) {
        double* acc = reinterpret_cast<double*>(ws + d.pair_off[pr]) + kx;
        *acc += widen(Xa.x * Xa.x + Xa.y * Xa.y);
      } else {
        double2* acc = reinterpret_cast<double2*>(ws + d.pair_off[pr]) + kx;
        double2 v = *acc;
        v.x += widen(Xa.x * Xb.x + Xa.y * Xb.y);       // X_a X_b^*
        v.y += widen(Xa.y * Xb.x - Xa.x * Xb.y);
        *acc = v;
      }
    }
    if (tid == 0) {             // k = 0 sums for the mean subtraction
      double* m0 = reinterpret_cast<double*>(ws + d.off_mean0);
      for (int f = 0; f < F; ++f) m0[f] += (double)X[(size_t)f * hn1].x;
    }
    __syncthreads();            // the next sample's products follow this one's in every sum
  }

  R* g_dst = reinterpret_cast<R*>(ws + d.off_pop[(int)((t0 + n_steps) & 1)]);
  const R* fin = pop + (n_steps & 1) * 3 * nx;
  for (int i = tid; i < 3 * nx; i += nt) g_dst[i] = fin[i];
  if (sampled) {                // the fields of the last sample, as the per-step kernel leaves them
    R* g_fld = reinterpret_cast<R*>(ws + d.off_fields);
    for (int i = tid; i < F * nx; i += nt) g_fld[i] = fld[i];
  }
}

cudaError_t launch_d1q3_fused(int precision, const ReplicaDesc* descs, int n_reps, char* ws, uint64_t t0,
                              uint32_t n_steps, uint32_t every, size_t smem, cudaStream_t st) {
  cudaError_t e;
  if (precision == FLB_FP64) {
    if ((e = cudaFuncSetAttribute(k_d1q3_fused<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    k_d1q3_fused<double, false><<<n_reps, kD1q3FusedThreads, smem, st>>>(descs, ws, t0, n_steps, every);
  } else {
    if ((e = cudaFuncSetAttribute(k_d1q3_fused<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
      return e;
    k_d1q3_fused<float, true><<<n_reps, kD1q3FusedThreads, smem, st>>>(descs, ws, t0, n_steps, every);
  }
  return cudaGetLastError();
}

}  // namespace flb
