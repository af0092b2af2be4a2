// Device-pointer entry point of the correlator sampler (Eqs. 11-12): FFT and FP64
// pair accumulation of caller-provided real fields, without a simulation context.
// Uses the kernels of spectra.cu; the per-call plan (descriptor, block tables,
// twiddles, row-transformed spectra) lives in caller-provided scratch memory.
#include <algorithm>
#include <cstring>

#include "flb_internal.cuh"
#include "spectra_plan.cuh"

namespace flb {

void launch_twiddles(int precision, void* tw, int n, cudaStream_t st);
int fft_rows_smem(int precision, int nx);
int fft_cols_smem(int precision, int F, int ny, int ncol);
cudaError_t set_fft_smem_limits();
void launch_fft_rows(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int grid, int block, int smem, cudaStream_t st, int slot,
                     int paths, int sms);
void launch_fft_cols(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                     int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st,
                     const TimeCorr& tc, int paths, int nslots, int max_fields);
void launch_fft_cols_a(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                       int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st,
                       int paths, int slot, int sms);

static inline int64_t a256(int64_t x) { return (x + 255) & ~int64_t(255); }

int spectra_plan(int precision, int nx, int ny, int F, SpectraPlan& P) {
  memset(&P, 0, sizeof P);
  if (precision != FLB_FP64 && precision != FLB_FP32_DEV) return set_error(FLB_EINVAL, "unknown precision %d", precision);
  if (F < 1 || F > kMaxFields) return set_error(FLB_EINVAL, "n_fields must be in 1..%d", kMaxFields);
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(nx) || !pow2(ny) || nx < 2) return set_error(FLB_EINVAL, "nx, ny must be powers of two, nx >= 2");
  if (fft_rows_smem(precision, nx) > 227 * 1024) return set_error(FLB_EINVAL, "nx = %d too long for the row FFT", nx);
  const int l1 = column_split(precision, F, ny);
  int ly = 0;
  while ((1 << ly) < ny) ++ly;
  int lx = 0;
  while ((1 << lx) < nx) ++lx;
  const int len = std::max(1 << l1, ny >> l1);
  if (fft_cols_smem(precision, F, len, 1) > kColsSmemBudget)
    return set_error(FLB_EINVAL, "ny = %d too long for the column FFT with %d fields", ny, F);
  const int64_t rs = precision == FLB_FP64 ? 8 : 4;
  const int cs = (int)(2 * rs);
  ReplicaDesc& d = P.desc;
  d.nx = nx; d.ny = ny; d.log2nx = lx; d.log2ny = ly; d.q = 9;
  d.n_fields = F;
  for (int f = 0; f < F; ++f) d.field_id[f] = f;
  int np = 0;
  for (int a = 0; a < F; ++a)
    for (int b = a; b < F; ++b) { d.pair_a[np] = a; d.pair_b[np] = b; ++np; }
  d.n_pairs = np;
  d.half_nx = nx / 2 + 1;
  d.wpitch = (d.half_nx + 1) & ~1;
  d.log2n1 = l1;
  P.ncol = kColsMax;
  while (P.ncol > 1 && fft_cols_smem(precision, F, len, P.ncol) > kColsSmemBudget) P.ncol >>= 1;
  P.rows_smem = fft_rows_smem(precision, nx);
  P.rows_block = std::max(32, std::min(kRowsBlockMax, nx / 2));
  P.cols_smem = fft_cols_smem(precision, F, len, P.ncol);
  const int64_t tiles = (d.half_nx + P.ncol - 1) / P.ncol;
  P.n_vb_rows = rows_blocks(precision, nx, F, ny);
  P.n_vb_cols = tiles << l1;
  P.n_vb_cols_a = cols_a_blocks(precision, l1, F, d.half_nx, ny, P.ncol);
  int64_t off = 0;
  P.off_desc = off; off = a256(off + (int64_t)sizeof(ReplicaDesc));
  P.off_vb = off; off = a256(off + 8 * 3);
  P.off_tw_x = off; off = a256(off + (int64_t)(nx / 2) * cs + 16);
  P.off_tw_y = off; off = a256(off + (int64_t)(ny / 2) * cs + 16);
  d.spec_tiled = spec_tiled_ok(precision, nx, ny, l1) ? 1 : 0;
  P.off_spec = off; off = a256(off + spec_elems(d) * cs);
  P.scratch_bytes = (size_t)off;
  int64_t sums = 0;
  for (int pr = 0; pr < np; ++pr) sums += (int64_t)ny * d.half_nx * (d.pair_a[pr] == d.pair_b[pr] ? 1 : 2);
  P.n_sum_doubles = sums;
  return FLB_OK;
}

// One thread stores the plan's descriptor and block tables into device memory, so no
// host-to-device copy (and no host staging buffer) is involved.
__global__ void k_store_plan(ReplicaDesc d, ReplicaDesc* dst, int64_t* vb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *dst = d;
    vb[0] = 0; vb[1] = 0; vb[2] = 0;
  }
}

int spectra_launch(int precision, SpectraPlan& P, char* scratch, const void* fields, double* pair_sums,
                   double* mean0, cudaStream_t st) {
  ReplicaDesc& d = P.desc;
  // offsets are relative to the scratch base
  const uintptr_t base = (uintptr_t)scratch;
  d.off_fields = (int64_t)((uintptr_t)fields - base);
  d.off_spec = P.off_spec;
  d.off_tw_x = P.off_tw_x;
  d.off_tw_y = P.off_tw_y;
  d.off_mean0 = (int64_t)((uintptr_t)mean0 - base);
  int64_t doff = 0;
  for (int pr = 0; pr < d.n_pairs; ++pr) {
    d.pair_off[pr] = (int64_t)((uintptr_t)(pair_sums + doff) - base);
    doff += (int64_t)d.ny * d.half_nx * (d.pair_a[pr] == d.pair_b[pr] ? 1 : 2);
  }
  cudaError_t e = set_fft_smem_limits();
  if (e != cudaSuccess) return set_error(FLB_ECUDA, "smem limits: %s", cudaGetErrorString(e));
  ReplicaDesc* ddesc = reinterpret_cast<ReplicaDesc*>(scratch + P.off_desc);
  int64_t* vb = reinterpret_cast<int64_t*>(scratch + P.off_vb);
  k_store_plan<<<1, 32, 0, st>>>(d, ddesc, vb);
  launch_twiddles(precision, scratch + P.off_tw_x, d.nx, st);
  launch_twiddles(precision, scratch + P.off_tw_y, d.ny, st);
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gr = (int)std::min<int64_t>(P.n_vb_rows, (int64_t)sms * 8);
  launch_fft_rows(precision, ddesc, vb, 1, P.n_vb_rows, scratch, gr, P.rows_block, P.rows_smem, st, 0,
                  rows16(precision, d.nx) ? 1 << (d.log2nx - 12) : kColsGeneric, sms);
  if (P.n_vb_cols_a) {
    const int ga = (int)std::min<int64_t>(P.n_vb_cols_a, (int64_t)sms * 8);
    launch_fft_cols_a(precision, ddesc, vb + 1, 1, P.n_vb_cols_a, scratch, P.ncol, ga, kColsBlock, P.cols_smem, st,
                      cols16_b(1 << d.log2n1) ? cols16_b(1 << d.log2n1) : kColsGeneric, 0, sms);
  }
  const int gc = (int)std::min<int64_t>(P.n_vb_cols, (int64_t)sms * 8);
  launch_fft_cols(precision, ddesc, vb + 2, 1, P.n_vb_cols, scratch, P.ncol, gc, kColsBlock, P.cols_smem, st,
                  TimeCorr{}, cols16_b(d.ny >> d.log2n1) ? cols16_b(d.ny >> d.log2n1) : kColsGeneric, 1, (int)d.n_fields);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FLB_ECUDA, "spectra launch: %s", cudaGetErrorString(e));
  return FLB_OK;
}

}  // namespace flb

using namespace flb;

extern "C" {

int flb_spectra_scratch_bytes(int precision, int nx, int ny, int n_fields, size_t* bytes_out, size_t* n_sums_out) {
  SpectraPlan P;
  const int rc = spectra_plan(precision, nx, ny, n_fields, P);
  if (rc) return rc;
  if (bytes_out) *bytes_out = P.scratch_bytes;
  if (n_sums_out) *n_sums_out = (size_t)P.n_sum_doubles;
  return FLB_OK;
}

int flb_spectra_accumulate(int precision, int nx, int ny, int n_fields, const void* fields_dev,
                           double* pair_sums_dev, double* mean0_dev, void* scratch_dev, size_t scratch_bytes,
                           void* cuda_stream) {
  SpectraPlan P;
  int rc = spectra_plan(precision, nx, ny, n_fields, P);
  if (rc) return rc;
  if (!fields_dev || !pair_sums_dev || !mean0_dev || !scratch_dev) return set_error(FLB_EINVAL, "NULL pointer");
  if (((uintptr_t)scratch_dev) & 255) return set_error(FLB_EINVAL, "scratch must be 256-byte aligned");
  if (scratch_bytes < P.scratch_bytes)
    return set_error(FLB_ENOMEM, "scratch %zu bytes < required %zu", scratch_bytes, P.scratch_bytes);
  return spectra_launch(precision, P, static_cast<char*>(scratch_dev), fields_dev, pair_sums_dev, mean0_dev,
                        static_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"
