// Host side of the C ABI declared in include/flb.h: validation, workspace
// layout, launch sequencing and host I/O.  All compute runs in the kernels of
// lb_step.cu and spectra.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <complex>

#include <nvtx3/nvToolsExt.h>

#include "flb_internal.cuh"
#include "lattice3.cuh"

namespace flb {

// launchers (lb_step.cu, spectra.cu)
void launch_step(int lattice, int precision, int vec, const StepLaunch& L, bool sample, bool mlp, cudaStream_t st);
void launch_step_bulk(int vec, const StepLaunch& L, bool sample, bool mlp, cudaStream_t st);
void launch_init(int precision, const ReplicaDesc* descs, int r, char* ws, int mode, const double* feq0,
                 double* sums, double* partial, int64_t V, cudaStream_t st);
void launch_conserved(int precision, const ReplicaDesc* descs, int r, const char* ws, int parity,
                      double* sums, double* partial, DevStatus* status, int64_t V, cudaStream_t st);
void launch_philox(const uint32_t* site, int n, uint32_t step, uint32_t call, uint32_t tag, uint32_t stream,
                   uint64_t seed, int fp32, uint32_t* words, double* normals, cudaStream_t st);
size_t mlp_weights_bytes();
void launch_set_step(uint64_t* s, uint64_t v, cudaStream_t st);
void launch_advance_step(uint64_t* s, uint64_t n, cudaStream_t st);
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
void launch_time_corr(const ReplicaDesc* descs, int n_reps, int max_fields, const TimeCorr& tc, cudaStream_t st);
void launch_fft_cols_a(int precision, const ReplicaDesc* descs, const int64_t* vb_begin, int n_reps,
                       int64_t n_vblocks, char* ws, int ncol, int grid, int block, int smem, cudaStream_t st,
                       int paths, int slot, int sms);
void launch_wait_probe(DevStatus* status, long long limit, cudaStream_t st);   // lb_step_tc.cu
// D1Q3 runs of steps with their sampling in one launch (lb_d1q3_fused.cu)
size_t d1q3_fused_smem(int precision, int nx, int F);
cudaError_t launch_d1q3_fused(int precision, const ReplicaDesc* descs, int n_reps, char* ws, uint64_t t0,
                              uint32_t n_steps, uint32_t every, size_t smem, cudaStream_t st);
// D3Q15 / D3Q19 (lb_3d.cu), q = 15 or 19
void launch_step3(int q, int precision, int vec, const StepLaunch& L, bool sample, cudaStream_t st);
void launch_init3(int q, int precision, const ReplicaDesc* descs, int r, char* ws, int mode, const double* feq0,
                  double* sums, double* partial, int64_t V, cudaStream_t st);
void launch_conserved3(int q, int precision, const ReplicaDesc* descs, int r, const char* ws, int parity, double* sums,
                       double* partial, DevStatus* status, int64_t V, cudaStream_t st);
size_t point_dft_smem(int precision, int nx, int ny, int nz, int items, int items2);
size_t point_tables_bytes(int precision, int nx, int ny, int nz);
void launch_point_tables(int precision, const ReplicaDesc* descs, int n_reps, char* base, cudaStream_t st);
cudaError_t set_point_dft_smem(int precision, size_t bytes);
void launch_point_dft(int precision, const ReplicaDesc* descs, int n_reps, int max_items, const char* ws,
                      const TimeCorr& tc, size_t smem, cudaStream_t st);

static thread_local std::string g_last_error;

// NVTX range on the host timeline around a library call (no cost without an attached tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

static int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FLB_OK;
  return set_error(FLB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static inline int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }
static inline bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
static inline int ilog2(int64_t x) { int l = 0; while ((int64_t(1) << l) < x) ++l; return l; }

static const double kW9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int kVx9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int kVy9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double kW3[3] = {2.0 / 3, 1.0 / 6, 1.0 / 6};
static const int kVx3[3] = {0, 1, -1};
// D3Q15: rest, +-x, +-y, +-z, then the corners in +- pairs (1,1,1), (1,1,-1), (1,-1,1), (-1,1,1)
static const int kVx15[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
static const int kVy15[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
static const int kVz15[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1};
// D3Q19: rest, +-x, +-y, +-z, then the edges in +- pairs (1,1,0), (1,-1,0), (1,0,1), (1,0,-1),
// (0,1,1), (0,1,-1)
static const int kVx19[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int kVy19[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int kVz19[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static double lattice_weight(int q, int i) {
  if (q == 9) return kW9[i];
  if (q == 3) return kW3[i];
  if (q == 19) return i == 0 ? 1.0 / 3 : (i < 7 ? 1.0 / 18 : 1.0 / 36);
  return i == 0 ? 2.0 / 9 : (i < 7 ? 1.0 / 9 : 1.0 / 72);
}
static inline int64_t volume(const ReplicaDesc& d) { return (int64_t)d.nx * d.ny * d.nz; }
static inline bool is3d(int lat) { return lat == FLB_D3Q15 || lat == FLB_D3Q19; }
static inline int lattice_q(int lat) {
  return lat == FLB_D3Q19 ? 19 : (lat == FLB_D3Q15 ? 15 : (lat == FLB_D2Q9 ? 9 : 3));
}
static inline int first_nonconserved(int lat) { return is3d(lat) ? 4 : (lat == FLB_D2Q9 ? 3 : 2); }
static constexpr int kMaxPointItems = 2048;    // 3D direct transforms: fields x wave vectors

static constexpr int kStepBlock = 256;

struct Layout {
  std::vector<ReplicaDesc> desc;
  int64_t off_descs = 0, off_vb_step = 0, off_vb_rows = 0, off_vb_cols = 0, off_vb_cols_a = 0;
  int64_t off_status = 0, off_sums = 0, off_partial = 0, off_feq0 = 0, off_mlp = 0, off_stepdev = 0;
  int64_t total = 0;
  int64_t n_vb_step = 0, n_vb_rows = 0, n_vb_cols = 0, n_vb_cols_a = 0;
  std::vector<int64_t> vb_step, vb_rows, vb_cols, vb_cols_a;
  int vec = 1, q = 9, ncol = 0, rows_block = 32, rows_smem = 0, cols_smem = 0;
  int cols_a_paths = 0, cols_paths = 0;   // column-pass kernels the replicas need (cols16_b)
  int rows_paths = 0;                     // row-pass kernels (launch_fft_rows)
  int fold = 1;               // 2: two spectrum slots, two samples per accumulation pass
  int max_fields = 0;         // the most sampled fields of a replica with pair sums
  int staged = 0;             // 1: the step kernel of lb_step_bulk.cu (tiles of 256 vec sites)
  bool any_fields = false;
};

static int field_valid(int lattice, int f) {
  if (is3d(lattice)) return f >= 0 && f < lattice_q(lattice);
  if (lattice == FLB_D2Q9) return f >= 0 && f <= 10;
  return f == 0 || f == 1 || f == 2 || f == FLB_FIELD_UX;
}

static int validate(int precision, const flb_replica* reps, int n) {
  if (precision != FLB_FP64 && precision != FLB_FP32_DEV) return set_error(FLB_EINVAL, "unknown precision %d", precision);
  if (!reps || n <= 0) return set_error(FLB_EINVAL, "need at least one replica");
  const int lat = reps[0].lattice;
  if (lat != FLB_D1Q3 && lat != FLB_D2Q9 && !is3d(lat)) return set_error(FLB_EINVAL, "unknown lattice %d", lat);
  for (int r = 0; r < n; ++r) {
    const flb_replica& p = reps[r];
    if (p.lattice != lat) return set_error(FLB_EINVAL, "replica %d: all replicas must share the lattice type", r);
    const int q = lattice_q(lat);
    if (p.nx < 2 || p.nx % 2) return set_error(FLB_EINVAL, "replica %d: nx must be even and >= 2", r);
    if (lat == FLB_D1Q3 && p.ny != 1) return set_error(FLB_EINVAL, "replica %d: D1Q3 needs ny = 1", r);
    if (lat != FLB_D1Q3 && p.ny < 1) return set_error(FLB_EINVAL, "replica %d: ny must be >= 1", r);
    if (is3d(lat) ? p.nz < 1 : (p.nz < 0 || p.nz > 1))
      return set_error(FLB_EINVAL, "replica %d: nz = %d (D3Q15, D3Q19: >= 1; otherwise 0 or 1)", r, p.nz);
    const int64_t V = (int64_t)p.nx * p.ny * (is3d(lat) ? p.nz : 1);
    if (V >= (int64_t(1) << 32)) return set_error(FLB_EINVAL, "replica %d: lattice too large", r);
    if (precision == FLB_FP64 && V >= (int64_t(1) << 31))
      return set_error(FLB_EINVAL, "replica %d: lattice too large for the FP64 path", r);
    if (!(p.rho0 > 0) || !std::isfinite(p.rho0)) return set_error(FLB_EINVAL, "replica %d: rho0 must be > 0", r);
    if (!(p.kT >= 0) || !std::isfinite(p.kT)) return set_error(FLB_EINVAL, "replica %d: kT must be >= 0", r);
    if (!std::isfinite(p.u0[0]) || !std::isfinite(p.u0[1]) || !std::isfinite(p.u0[2]))
      return set_error(FLB_EINVAL, "replica %d: u0 not finite", r);
    const int nc0 = first_nonconserved(lat);
    for (int a = nc0; a < q; ++a)
      if (!(p.tau[a] > 0.5) || !std::isfinite(p.tau[a]))
        return set_error(FLB_EINVAL, "replica %d: tau[%d] = %g must be > 1/2", r, a, p.tau[a]);
    if (p.noise_mask & ((1u << nc0) - 1)) return set_error(FLB_EINVAL, "replica %d: noise on a conserved moment", r);
    if (p.noise_mask >> q) return set_error(FLB_EINVAL, "replica %d: noise_mask has bits beyond moment %d", r, q - 1);
    if (p.init_mode > 1) return set_error(FLB_EINVAL, "replica %d: init_mode must be 0 or 1", r);
    if (p.noise_mode > 2) return set_error(FLB_EINVAL, "replica %d: noise_mode must be 0, 1 or 2", r);
    if (is3d(lat) && p.noise_mode != 0) return set_error(FLB_EINVAL, "replica %d: 3D lattices have noise_mode 0 only", r);
    for (int f = 0; f < 32; ++f)
      if (((p.field_mask >> f) & 1) && !field_valid(lat, f))
        return set_error(FLB_EINVAL, "replica %d: field %d not available on this lattice", r, f);
    if (p.field_mask && is3d(lat)) {
      if (__builtin_popcount(p.field_mask) > kMaxFields)
        return set_error(FLB_EINVAL, "replica %d: at most %d sampled fields", r, kMaxFields);
      if (p.nx > 4096 || p.ny > 4096 || p.nz > 4096)
        return set_error(FLB_EINVAL, "replica %d: sampling needs nx, ny, nz <= 4096", r);
    } else if (p.field_mask) {
      if (!is_pow2(p.nx) || !is_pow2(p.ny)) return set_error(FLB_EINVAL, "replica %d: sampling needs power-of-two nx, ny", r);
      if (fft_rows_smem(precision, p.nx) > 227 * 1024) return set_error(FLB_EINVAL, "replica %d: nx too large for the row FFT", r);
      const int F = __builtin_popcount(p.field_mask);
      const int l1 = column_split(precision, F, p.ny);
      const int len = std::max(1 << l1, p.ny >> l1);
      if (fft_cols_smem(precision, F, len, 1) > kColsSmemBudget)
        return set_error(FLB_EINVAL, "replica %d: ny = %d too long for the column FFT with %d fields", r, p.ny, F);
    }
    if (p.init_mode == 1 && p.kT > 0 && V < 2) return set_error(FLB_EINVAL, "thermal init needs V >= 2");
  }
  return FLB_OK;
}

// ---------------------------------------------------------------------------
// Correlated noise (noise_mode 1).  Moment rows of Eq. 9 (D2Q9) and of the D1Q3
// projection, the discrete Maxwellian of Eq. 2, the moment covariance of Eq. 7 at
// f^0(rho0, u0), the noise covariance of Eq. 6, and the principal square root of its
// positive part.

static double moment_row(bool d2, int a, double vx, double vy) {
  const double v2 = vx * vx + vy * vy, s3 = std::sqrt(3.0);
  if (!d2) {
    const double m[3] = {1.0, s3 * vx, (3.0 * vx * vx - 1.0) / std::sqrt(2.0)};
    return m[a];
  }
  switch (a) {
    case 0: return 1.0;
    case 1: return s3 * vx;
    case 2: return s3 * vy;
    case 3: return 1.5 * (vx * vx - vy * vy);
    case 4: return 3.0 * vx * vy;
    case 5: return 1.5 * v2 - 1.0;
    case 6: return std::sqrt(1.5) * vx * (3.0 * v2 - 4.0);
    case 7: return std::sqrt(1.5) * vy * (3.0 * v2 - 4.0);
    default: return 2.25 * v2 * v2 - 3.75 * v2 + 0.5;
  }
}

// Eigen-decomposition of a symmetric n x n matrix (n <= 6) by cyclic Jacobi rotations
// (Golub & Van Loan, Matrix Computations, Sec. 8.5): A = V diag(w) V^T.
static void jacobi_eigen(int n, double A[6][6], double V[6][6], double w[6]) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) { tot += A[i][j] * A[i][j]; if (i != j) off += A[i][j] * A[i][j]; }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (A[p][q] == 0.0) continue;
        // rotation that zeroes A[p][q]: t = tan(theta), theta = (A_qq - A_pp) / (2 A_pq)
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {            // A <- A J (columns p, q)
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {            // A <- J^T A (rows p, q)
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {            // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i][i];
}

// R (n_nc x n_nc, row-major in out) for replica p; returns n_nc.
static int correlated_root(const flb_replica& p, double* out) {
  const bool d2 = p.lattice == FLB_D2Q9;
  const int q = d2 ? 9 : 3, nc0 = d2 ? 3 : 2, n = q - nc0;
  const double mu = 3.0 * p.kT, ux = p.u0[0], uy = d2 ? p.u0[1] : 0.0, uu = ux * ux + uy * uy;
  double C[9][9] = {};
  for (int i = 0; i < q; ++i) {
    const double vx = d2 ? kVx9[i] : kVx3[i], vy = d2 ? kVy9[i] : 0.0, w = d2 ? kW9[i] : kW3[i];
    const double vu = vx * ux + vy * uy;
    const double f0 = w * p.rho0 * (1.0 + 3.0 * vu + 4.5 * vu * vu - 1.5 * uu);     // Eq. 2
    double m[9];
    for (int a = 0; a < q; ++a) m[a] = moment_row(d2, a, vx, vy);
    for (int a = 0; a < q; ++a)
      for (int b = 0; b < q; ++b) C[a][b] += mu * m[a] * m[b] * f0;             // Eq. 7 at u0
  }
  double A[6][6] = {}, V[6][6], w[6];
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      const int ma = nc0 + a, mc = nc0 + c;
      if (!((p.noise_mask >> ma) & 1) || !((p.noise_mask >> mc) & 1)) continue;
      A[a][c] = (p.tau[ma] + p.tau[mc] - 1.0) / (p.tau[ma] * p.tau[mc]) * C[ma][mc];   // Eq. 6
    }
  jacobi_eigen(n, A, V, w);
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      double r = 0.0;
      for (int k = 0; k < n; ++k) r += V[a][k] * std::sqrt(w[k] > 0.0 ? w[k] : 0.0) * V[c][k];
      out[a * n + c] = r;
    }
  return n;
}

static void fill_desc(int precision, const flb_replica& p, ReplicaDesc& d) {
  memset(&d, 0, sizeof d);
  const bool d2 = p.lattice == FLB_D2Q9, d3 = is3d(p.lattice);
  d.nx = p.nx; d.ny = p.ny; d.log2nx = ilog2(p.nx); d.log2ny = ilog2(p.ny);
  d.nz = d3 ? p.nz : 1;
  d.q = lattice_q(p.lattice);
  d.seed_lo = (uint32_t)p.seed; d.seed_hi = (uint32_t)(p.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    d.rkey[2 * r] = d.seed_lo + (uint32_t)r * 0x9E3779B9u;
    d.rkey[2 * r + 1] = d.seed_hi + (uint32_t)r * 0xBB67AE85u;
  }
  d.stream = p.stream; d.noise_mask = p.noise_mask; d.field_mask = p.field_mask;
  d.rho0 = p.rho0; d.kT = p.kT; d.mu = 3.0 * p.kT; d.u0x = p.u0[0]; d.u0y = (d2 || d3) ? p.u0[1] : 0.0;
  d.u0z = d3 ? p.u0[2] : 0.0;
  const int nc0 = first_nonconserved(p.lattice);
  for (int a = nc0; a < d.q; ++a) {
    d.inv_tau[a] = 1.0 / p.tau[a];
    d.amp[a] = ((p.noise_mask >> a) & 1) ? std::sqrt(d.mu * p.rho0 * (2.0 * p.tau[a] - 1.0)) / p.tau[a] : 0.0;
  }
  // field reference values M^{a,0}(rho0, u0) (Eq. 10), minus rho0 on the density
  // moment in deviation storage, where the stored moment is that of f - w rho0
  const double ux = d.u0x, uy = d.u0y, uz = d.u0z, r0 = p.rho0, s3 = std::sqrt(3.0);
  if (d3) {
    // the equilibrium moments of the D3Q15 / D3Q19 bases (lb_3d.cu) at (rho0, u0); ghosts 0
    const double m[10] = {r0, s3 * r0 * ux, s3 * r0 * uy, s3 * r0 * uz, 1.5 * r0 * (ux * ux - uy * uy),
                          0.5 * s3 * r0 * (ux * ux + uy * uy - 2 * uz * uz), 3 * r0 * ux * uy, 3 * r0 * uy * uz,
                          3 * r0 * uz * ux, 0.5 * std::sqrt(6.0) * r0 * (ux * ux + uy * uy + uz * uz)};
    for (int a = 0; a < 10; ++a) d.mref[a] = m[a];
  } else if (d2) {
    const double m[9] = {r0, s3 * r0 * ux, s3 * r0 * uy, 1.5 * r0 * (ux * ux - uy * uy), 3 * r0 * ux * uy,
                         1.5 * r0 * (ux * ux + uy * uy), 0, 0, 0};
    for (int a = 0; a < 9; ++a) d.mref[a] = m[a];
  } else {
    d.mref[0] = r0; d.mref[1] = s3 * r0 * ux; d.mref[2] = 3.0 * r0 * ux * ux / std::sqrt(2.0);
  }
  if (precision == FLB_FP32_DEV) d.mref[0] -= r0;
  int F = 0;
  for (int f = 0; f < 32 && F < kMaxFields; ++f)
    if ((p.field_mask >> f) & 1) d.field_id[F++] = f;
  d.n_fields = F;
  int np = 0;
  if (!d3)                     // pair sums on the FFT grid (D1Q3, D2Q9)
    for (int a = 0; a < F; ++a)
      for (int b = a; b < F; ++b) { d.pair_a[np] = a; d.pair_b[np] = b; ++np; }
  d.n_pairs = np;
  d.half_nx = p.nx / 2 + 1;
  d.wpitch = (d.half_nx + 1) & ~1;
  d.log2n1 = (F && !d3) ? column_split(precision, F, p.ny) : 0;
  d.noise_mode = (int32_t)p.noise_mode;
  if (p.noise_mode == 1) {
    double R[36];
    const int nr = correlated_root(p, R);
    if (d2) {
      for (int i = 0; i < 36; ++i) d.dco[kCoNoiseR + i] = R[i];
    } else {
      d.amp[2] = R[0];            // one non-conserved moment: the root is its amplitude
      d.noise_mode = 0;
    }
    (void)nr;
  }
  d.dco[kCoRho0] = d.rho0; d.dco[kCoU0x] = d.u0x; d.dco[kCoU0y] = d.u0y; d.dco[kCoU0z] = d.u0z;
  for (int a = 0; a < kMaxQ; ++a) { d.dco[kCoInvTau + a] = d.inv_tau[a]; d.dco[kCoAmp + a] = d.amp[a]; }
  for (int f = 0; f < kMaxQ; ++f) d.dco[kCoMref + f] = d.mref[f];
  for (int i = 0; i < kNumCoef; ++i) d.fco[i] = (float)d.dco[i];
}

// Step-launch tables.  Direct kernels: a unit is VEC consecutive sites (one thread),
// a virtual block is kStepBlock units of one replica.  Staged kernel: a unit is a row
// tile of up to 256 VEC sites, and a virtual block is one tile.
static void plan_step(int lattice, int vec, int staged, Layout& L) {
  L.vec = vec;
  L.staged = staged;
  L.n_vb_step = 0;
  L.vb_step.resize(L.desc.size());
  for (size_t r = 0; r < L.desc.size(); ++r) {
    ReplicaDesc& d = L.desc[r];
    const int tile = kStepBlock * vec;
    d.units_per_row = staged ? (d.nx + tile - 1) / tile : d.nx / (lattice == FLB_D1Q3 ? 1 : vec);
    // m = ceil(2^(31+l) / upr), l = ceil(log2 upr): floor(u m / 2^(31+l)) = floor(u / upr) for u < 2^31
    int l = 0;
    while ((1LL << l) < d.units_per_row) ++l;
    const uint64_t p2 = 1ULL << (31 + l);
    d.upr_magic = (uint32_t)((p2 + (uint64_t)d.units_per_row - 1) / (uint64_t)d.units_per_row);
    d.upr_shift = 31 + l;
    d.n_units = (int64_t)d.units_per_row * d.ny * d.nz;      // rows (y, z)
    L.vb_step[r] = L.n_vb_step;
    d.block_begin = L.n_vb_step;
    L.n_vb_step += staged ? d.n_units : (d.n_units + kStepBlock - 1) / kStepBlock;
  }
}

static int plan(int precision, const flb_replica* reps, int n, Layout& L) {
  int rc = validate(precision, reps, n);
  if (rc) return rc;
  const int lat = reps[0].lattice;
  const int64_t rs = precision == FLB_FP64 ? 8 : 4;
  L.q = lattice_q(lat);
  // vector width of the step kernel: all replicas share one launch
  L.vec = 1;
  if (precision == FLB_FP32_DEV && lat == FLB_D2Q9) {
    bool all4 = true;
    for (int r = 0; r < n; ++r) all4 = all4 && reps[r].nx % 4 == 0;
    L.vec = all4 ? 4 : 2;
  } else if (precision == FLB_FP32_DEV && is3d(lat)) {
    bool all4 = lat == FLB_D3Q15;                // nx is even; D3Q19 at vec 4 spills registers
    for (int r = 0; r < n; ++r) all4 = all4 && reps[r].nx % 4 == 0;
    L.vec = all4 ? 4 : 2;
  }
  L.desc.resize(n);
  int64_t off = 0;
  int maxF = 0, maxlen = 1;
  for (int r = 0; r < n; ++r) {
    ReplicaDesc& d = L.desc[r];
    fill_desc(precision, reps[r], d);
    if (d.n_fields) L.any_fields = true;
    if (d.n_pairs) {
      maxF = std::max(maxF, (int)d.n_fields);
      maxlen = std::max(maxlen, std::max(1 << d.log2n1, d.ny >> d.log2n1));
    }
  }
  // column tile width of the sampling passes (it fixes the blocked layout of the pair sums)
  L.max_fields = maxF;
  if (maxF) {
    L.ncol = kColsMax;
    while (L.ncol > 1 && fft_cols_smem(precision, maxF, maxlen, L.ncol) > kColsSmemBudget) L.ncol >>= 1;
    // the column-pass kernels: register-resident ones for FP32 columns of 16 .. 256
    int maxn2 = 1;
    for (const ReplicaDesc& d : L.desc) {
      if (!d.n_pairs) continue;
      L.rows_paths |= rows16(precision, d.nx) ? 1 << (ilog2(d.nx) - 12) : kColsGeneric;
      const int b2 = precision == FLB_FP64 ? 0 : cols16_b(d.ny >> d.log2n1);
      L.cols_paths |= b2 ? b2 : kColsGeneric;
      maxn2 = std::max(maxn2, d.ny >> d.log2n1);
      if (d.log2n1) {
        const int b1 = precision == FLB_FP64 ? 0 : cols16_b(1 << d.log2n1);
        L.cols_a_paths |= b1 ? b1 : kColsGeneric;
      }
    }
    // two samples per pass over the FP32 sums when every sampled replica has register-
    // resident columns and the two samples' tiles of at least 4 columns fit 4 blocks per SM
    if (!(L.cols_paths & kColsGeneric)) {
      int nc = L.ncol;
      while (nc >= 4 && fft_cols16_smem(maxF, maxn2, nc, 2) > kFoldSmemBudget) nc >>= 1;
      if (nc >= 4) { L.fold = 2; L.ncol = nc; }
    }
  }
  for (int r = 0; r < n; ++r) {
    ReplicaDesc& d = L.desc[r];
    const int64_t V = volume(d);
    d.off_pop[0] = off; off = align256(off + L.q * V * rs);
    d.off_pop[1] = off; off = align256(off + L.q * V * rs);
    if (d.n_fields) { d.off_fields = off; off = align256(off + (int64_t)d.n_fields * V * rs); }
    if (d.n_pairs) {
      d.spec_tiled = spec_tiled_ok(precision, d.nx, d.ny, d.log2n1) ? 1 : 0;
      const int64_t spec_bytes = align256(spec_elems(d) * 2 * rs);
      d.off_spec = off; off += L.fold * spec_bytes;
      d.spec_slot = L.fold == 2 ? spec_bytes : 0;
      d.acc_ncol = L.ncol;
      const int64_t padded_kx = (d.half_nx + L.ncol - 1) / L.ncol * L.ncol;
      for (int pr = 0; pr < d.n_pairs; ++pr) {
        d.pair_off[pr] = off;
        const int64_t el = d.pair_a[pr] == d.pair_b[pr] ? 8 : 16;
        off = align256(off + (int64_t)d.ny * padded_kx * el);
      }
      d.off_mean0 = off; off = align256(off + 8 * (int64_t)d.n_fields);
      d.off_tw_x = off; off = align256(off + (int64_t)(d.nx / 2) * 2 * rs + 16);
      d.off_tw_y = off; off = align256(off + (int64_t)(d.ny / 2) * 2 * rs + 16);
    }
  }
  // virtual-block prefixes of the three launches
  L.vb_step.resize(n); L.vb_rows.resize(n); L.vb_cols.resize(n); L.vb_cols_a.resize(n);
  if (maxF) {
    // the shared-memory row kernel's launch (replicas the Stockham kernel does not take)
    int gnx = 2;
    for (const ReplicaDesc& d : L.desc)
      if (d.n_pairs && !rows16(precision, d.nx)) gnx = std::max(gnx, d.nx);
    L.rows_smem = fft_rows_smem(precision, gnx);
    L.rows_block = std::max(32, std::min(kRowsBlockMax, gnx / 2));
    L.cols_smem = fft_cols_smem(precision, maxF, maxlen, L.ncol);
    if (L.fold == 2) L.cols_smem = std::max(L.cols_smem, fft_cols16_smem(maxF, maxlen, L.ncol, 2));
  }
  plan_step(lat, L.vec, 0, L);
  for (int r = 0; r < n; ++r) {
    ReplicaDesc& d = L.desc[r];
    L.vb_rows[r] = L.n_vb_rows;
    L.vb_cols[r] = L.n_vb_cols;
    L.vb_cols_a[r] = L.n_vb_cols_a;
    if (d.n_pairs) {
      const int64_t tiles = (d.half_nx + L.ncol - 1) / L.ncol;
      L.n_vb_rows += rows_blocks(precision, d.nx, (int)d.n_fields, d.ny);
      L.n_vb_cols += tiles << d.log2n1;                       // (k1, tile)
      L.n_vb_cols_a += cols_a_blocks(precision, d.log2n1, (int)d.n_fields, d.half_nx, d.ny, L.ncol);
    }
  }
  L.off_descs = off; off = align256(off + n * (int64_t)sizeof(ReplicaDesc));
  L.off_vb_step = off; off = align256(off + 8 * (int64_t)n);
  L.off_vb_rows = off; off = align256(off + 8 * (int64_t)n);
  L.off_vb_cols = off; off = align256(off + 8 * (int64_t)n);
  L.off_vb_cols_a = off; off = align256(off + 8 * (int64_t)n);
  L.off_status = off; off = align256(off + (int64_t)sizeof(DevStatus));
  L.off_sums = off; off = align256(off + 8 * 4 * (int64_t)n);
  L.off_partial = off; off = align256(off + 8 * 4 * (int64_t)kReduceBlocks);
  L.off_feq0 = off; off = align256(off + 8 * kFeqStride * (int64_t)n);
  L.off_mlp = off; off = align256(off + (int64_t)mlp_weights_bytes());
  L.off_stepdev = off; off = align256(off + 8);
  L.total = off;
  return FLB_OK;
}

// ---------------------------------------------------------------------------
// Linear stability of the noise-free dynamics about the uniform state f^0(rho0, u0).
// At wave vector k one step acts as A_k = P_k J: P_k = diag(exp(-i k.v_i)) (pull
// streaming, Eq. 1) and J the Jacobian of the collision (Eq. 5),
//   J = I + N Lambda (M E - M),   E_ij = d f^0_i / d f_j  (Eq. 2 through rho and j),
// with M the moment rows, N = (w_i m_i^a) the back transform and Lambda = diag(1/tau^a)
// on the non-conserved moments.  f^0_i = w_i (rho + 3 v.j + 9/2 (v.j)^2 / rho - 3/2 j^2 / rho)
// gives d f^0_i / d rho = w_i (1 - 9/2 (v.u)^2 + 3/2 u^2) and
// d f^0_i / d j_a = w_i (3 v_a + 9 (v.u) v_a - 3 u_a).

static int lattice_tables(int lat, int v[20][3], double w[20], double m[20][20]) {
  const int q = lattice_q(lat);
  for (int i = 0; i < q; ++i) {
    if (lat == FLB_D2Q9) { v[i][0] = kVx9[i]; v[i][1] = kVy9[i]; v[i][2] = 0; }
    else if (lat == FLB_D1Q3) { v[i][0] = kVx3[i]; v[i][1] = 0; v[i][2] = 0; }
    else if (lat == FLB_D3Q15) { v[i][0] = v3x<15>(i); v[i][1] = v3y<15>(i); v[i][2] = v3z<15>(i); }
    else { v[i][0] = v3x<19>(i); v[i][1] = v3y<19>(i); v[i][2] = v3z<19>(i); }
    w[i] = lattice_weight(q, i);
    for (int a = 0; a < q; ++a)
      m[a][i] = is3d(lat) ? (lat == FLB_D3Q15 ? moment_row3<15>(a, v[i][0], v[i][1], v[i][2])
                                              : moment_row3<19>(a, v[i][0], v[i][1], v[i][2]))
                          : moment_row(lat == FLB_D2Q9, a, v[i][0], v[i][1]);
  }
  return q;
}

// rho(A) = lim ||A^n||^(1/n) (Gelfand), n = 2^40 by repeated squaring with the norm
// factored out at every step
static double spectral_radius_of(int q, std::complex<double> A[20][20]) {
  typedef std::complex<double> cd;
  cd B[20][20], T[20][20];
  double nrm = 0.0;
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) nrm = std::max(nrm, std::abs(A[i][j]));
  if (nrm == 0.0) return 0.0;
  double logc = std::log(nrm);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) B[i][j] = A[i][j] / nrm;
  const int kSquarings = 40;
  for (int t = 0; t < kSquarings; ++t) {
    double mx = 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        cd acc = 0.0;
        for (int l = 0; l < q; ++l) acc += B[i][l] * B[l][j];
        T[i][j] = acc;
        mx = std::max(mx, std::abs(acc));
      }
    if (mx == 0.0) return 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) B[i][j] = T[i][j] / mx;
    logc = 2.0 * logc + std::log(mx);
  }
  return std::exp(std::ldexp(logc, -kSquarings));
}

}  // namespace flb

using namespace flb;

static constexpr uint32_t kGraphChunk = 32;      // at least this many steps per captured chunk
static constexpr uint32_t kMaxGraphChunk = 4096;  // longer sampling periods are issued directly
static constexpr uint32_t kFusedChunk = 4096;     // D1Q3 steps per fused launch
static constexpr size_t kFusedSmemMax = 200 * 1024;

struct flb_ctx {
  int precision = 0, lattice = 0, n = 0;
  std::vector<flb_replica> reps;
  Layout L;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  uint64_t step = 0, n_samples = 0;
  int pending = 0;            // samples in spectrum slots whose products are not yet in the sums
  int sms = 1;
  int step_grid = 0;          // 0: min(virtual blocks, 16 x SMs)
  bool mlp_on = false;
  int net_engine = FLB_NET_WARP;   // network of the direct D2Q9 kernels
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t copy_streams[4] = {nullptr, nullptr, nullptr, nullptr};   // checkpoint copies
  struct Graph { uint32_t len, every; cudaGraphExec_t exec; uint64_t kernels; };
  uint64_t launches = 0;      // kernels flb_run has issued (a replayed graph counts its kernels)
  bool capturing = false;     // issue_step / flush_samples are being captured into a graph
  uint64_t captured = 0;      // kernels in the graph being captured
  std::vector<Graph> graphs;
  std::vector<float> mlp_host;
  TimeCorr tc;                                 // time correlators (off: tc.base == nullptr)
  int64_t tc_off_sums0 = 0, tc_bytes = 0;      // start of the sums (first replica) and buffer size
  size_t tc_smem = 0;                          // 3D direct transforms: dynamic shared memory
  size_t fused_smem = 0;                       // D1Q3: shared memory of the fused kernel (0: not used)
};

static ReplicaDesc* descs_dev(flb_ctx* c) { return reinterpret_cast<ReplicaDesc*>(c->ws + c->L.off_descs); }
static DevStatus* status_dev(flb_ctx* c) { return reinterpret_cast<DevStatus*>(c->ws + c->L.off_status); }

static void feq0_host(const flb_replica& p, double out[kFeqStride]) {
  // Eq. 2 (c = 1) at (rho0, u0) at [i], and w_i rho0 at [kFeqW + i]
  const bool d2 = p.lattice == FLB_D2Q9, d3 = is3d(p.lattice), q19 = p.lattice == FLB_D3Q19;
  const int q = lattice_q(p.lattice);
  const double ux = p.u0[0], uy = (d2 || d3) ? p.u0[1] : 0.0, uz = d3 ? p.u0[2] : 0.0;
  for (int i = 0; i < kFeqStride; ++i) out[i] = 0.0;
  for (int i = 0; i < q; ++i) {
    const double w = lattice_weight(q, i);
    const double cu = q19 ? kVx19[i] * ux + kVy19[i] * uy + kVz19[i] * uz
                    : d3  ? kVx15[i] * ux + kVy15[i] * uy + kVz15[i] * uz
                          : (d2 ? kVx9[i] * ux + kVy9[i] * uy : kVx3[i] * ux);
    out[i] = p.rho0 * w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy + uz * uz));
    out[kFeqW + i] = w * p.rho0;
  }
}

static int reset_stats_async(flb_ctx* c) {
  for (int r = 0; r < c->n; ++r) {
    const ReplicaDesc& d = c->L.desc[r];
    if (!d.n_pairs) continue;
    const int64_t a0 = d.pair_off[0];
    const int64_t a1 = d.off_mean0 + 8 * (int64_t)d.n_fields;
    int rc = cuda_check(cudaMemsetAsync(c->ws + a0, 0, a1 - a0, c->stream), "reset stats");
    if (rc) return rc;
  }
  if (c->tc.base) {            // time-correlator sample counts and sums (the rings need no reset)
    int rc = cuda_check(cudaMemsetAsync(c->tc.count, 0, 8 * (size_t)c->n, c->stream), "reset stats");
    if (!rc) rc = cuda_check(cudaMemsetAsync(c->tc.base + c->tc_off_sums0, 0, (size_t)(c->tc_bytes - c->tc_off_sums0),
                                             c->stream), "reset stats");
    if (rc) return rc;
  }
  c->n_samples = 0;
  return FLB_OK;
}

// Blocks of the 3D direct transforms: FLB_POINT_BPS per SM at most, no more than the
// rows, and partial sums of at most 64 MB per replica.
#ifndef FLB_POINT_BPS
#define FLB_POINT_BPS 8
#endif
static int point_blocks(const flb_ctx* c, int n_k) {
  int64_t rows = 1, maxF = 1;
  for (const ReplicaDesc& d : c->L.desc) {
    rows = std::max<int64_t>(rows, (int64_t)d.ny * d.nz);
    maxF = std::max<int64_t>(maxF, d.n_fields);
  }
  int64_t g = std::min<int64_t>((int64_t)FLB_POINT_BPS * c->sms, rows);
  g = std::min<int64_t>(g, std::max<int64_t>(1, (int64_t(1) << 22) / (maxF * n_k)));
  return (int)std::max<int64_t>(g, 1);
}

// Time-correlator buffer layout: counts [n] u64 | kx [n_k] | ky [n_k] | kz [n_k] |
// kx index [n_k] | distinct kx [n_k] | rings
// of every replica | 3D block partials and phase tables of every replica | sums of
// every replica (contiguous, so a reset is one memset).
static int64_t time_corr_layout(const flb_ctx* c, int n_lags, int n_k, std::vector<int64_t>* ring,
                                std::vector<int64_t>* sums, int64_t* sums0, std::vector<int64_t>* part = nullptr,
                                std::vector<int64_t>* tab = nullptr) {
  int64_t off = align256(8 * (int64_t)c->n);
  for (int a = 0; a < 5; ++a) off = align256(off + 4 * (int64_t)n_k);
  for (int r = 0; r < c->n; ++r) {
    if (ring) (*ring)[r] = off;
    off = align256(off + 16 * (int64_t)n_lags * c->L.desc[r].n_fields * n_k);
  }
  if (is3d(c->lattice)) {
    const int G = point_blocks(c, n_k);
    for (int r = 0; r < c->n; ++r) {
      const ReplicaDesc& d = c->L.desc[r];
      if (part) (*part)[r] = off;
      off = align256(off + 16 * (int64_t)G * d.n_fields * n_k);
      if (tab) (*tab)[r] = off;
      off = align256(off + (int64_t)point_tables_bytes(c->precision, d.nx, d.ny, d.nz));
    }
  }
  if (sums0) *sums0 = off;
  for (int r = 0; r < c->n; ++r) {
    const int64_t F = c->L.desc[r].n_fields;
    if (sums) (*sums)[r] = off;
    off = align256(off + 16 * (int64_t)n_lags * F * F * n_k);
  }
  return off;
}

// Registry of the bounds-check counters of the translation units (checked build only).
namespace flb {
struct OobEntry { OobRead read; OobClear clear; };
static std::vector<OobEntry>& oob_registry() {
  static std::vector<OobEntry> v;
  return v;
}
bool register_oob_counter(OobRead read, OobClear clear) {
  oob_registry().push_back({read, clear});
  return true;
}
}  // namespace flb

extern "C" {

static void drop_graphs(flb_ctx* c);

int flb_time_correlator_bytes(flb_ctx* c, int n_lags, int n_k, size_t* bytes_out) {
  if (!c || !bytes_out) return set_error(FLB_EINVAL, "NULL argument");
  if (n_lags < 1 || n_k < 1) return set_error(FLB_EINVAL, "n_lags and n_k must be >= 1");
  *bytes_out = (size_t)time_corr_layout(c, n_lags, n_k, nullptr, nullptr, nullptr);
  return FLB_OK;
}

int flb_set_time_correlator(flb_ctx* c, int n_lags, int n_k, const int32_t* kx, const int32_t* ky, void* buf_dev,
                            size_t bytes) {
  return flb_set_time_correlator3(c, n_lags, n_k, kx, ky, nullptr, buf_dev, bytes);
}

int flb_set_time_correlator3(flb_ctx* c, int n_lags, int n_k, const int32_t* kx, const int32_t* ky,
                             const int32_t* kz, void* buf_dev, size_t bytes) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "time correlator");
  if (rc) return rc;
  drop_graphs(c);
  if (n_lags == 0) {                           // off
    c->tc = TimeCorr{};
    return FLB_OK;
  }
  if (n_lags < 1 || n_lags > 65536) return set_error(FLB_EINVAL, "n_lags must be in 1..65536 (0 = off)");
  if (n_k < 1 || n_k > 4096 || !kx || !ky) return set_error(FLB_EINVAL, "need 1..4096 wave vectors");
  if (!buf_dev || (reinterpret_cast<uintptr_t>(buf_dev) & 255)) return set_error(FLB_EINVAL, "buf_dev must be 256-B aligned");
  const bool d3 = is3d(c->lattice);
  std::vector<int32_t> kzv(n_k, 0);
  if (kz) kzv.assign(kz, kz + n_k);
  // distinct kx values (the row sums of the 3D direct transforms depend on kx only)
  std::vector<int32_t> kxl(kx, kx + n_k), kxi(n_k, 0);
  std::sort(kxl.begin(), kxl.end());
  kxl.erase(std::unique(kxl.begin(), kxl.end()), kxl.end());
  for (int j = 0; j < n_k; ++j) kxi[j] = (int32_t)(std::lower_bound(kxl.begin(), kxl.end(), kx[j]) - kxl.begin());
  const int n_kx = (int)kxl.size();
  kxl.resize(n_k, 0);
  size_t smem = 0;
  for (int r = 0; r < c->n; ++r) {
    const ReplicaDesc& d = c->L.desc[r];
    if (!d.n_fields) return set_error(FLB_EINVAL, "replica %d samples no fields", r);
    for (int j = 0; j < n_k; ++j) {
      if (d3) {
        if (kx[j] < 0 || kx[j] >= d.nx || ky[j] < 0 || ky[j] >= d.ny || kzv[j] < 0 || kzv[j] >= d.nz)
          return set_error(FLB_EINVAL, "wave vector %d = (%d, %d, %d) outside replica %d's lattice", j, kx[j], ky[j],
                           kzv[j], r);
      } else {
        if (kx[j] < 0 || kx[j] > d.nx / 2 || ky[j] < 0 || ky[j] >= d.ny)
          return set_error(FLB_EINVAL, "wave vector %d = (%d, %d) outside replica %d's half spectrum", j, kx[j], ky[j], r);
        if (kzv[j] != 0) return set_error(FLB_EINVAL, "wave vector %d: kz = %d on a lattice without z", j, kzv[j]);
      }
      if (kx[j] == 0 && ky[j] == 0 && kzv[j] == 0) return set_error(FLB_EINVAL, "wave vector %d is k = 0", j);
    }
    if (d3) {
      const int items = (int)d.n_fields * n_k;
      if (items > kMaxPointItems)
        return set_error(FLB_EINVAL, "fields x wave vectors = %d > %d", items, kMaxPointItems);
      smem = std::max(smem, point_dft_smem(c->precision, d.nx, d.ny, d.nz, items, (int)d.n_fields * n_kx));
    }
  }
  if (d3) {
    if (smem > 200 * 1024) return set_error(FLB_EINVAL, "direct transform needs %zu bytes of shared memory", smem);
    rc = cuda_check(set_point_dft_smem(c->precision, smem), "transform smem");
    if (rc) return rc;
  }
  std::vector<int64_t> ring(c->n), sums(c->n), part(c->n), tab(c->n);
  int64_t sums0 = 0;
  const int64_t need = time_corr_layout(c, n_lags, n_k, &ring, &sums, &sums0, &part, &tab);
  if ((int64_t)bytes < need) return set_error(FLB_EINVAL, "buffer of %zu bytes, need %lld", bytes, (long long)need);
  char* base = static_cast<char*>(buf_dev);
  const int64_t okx = align256(8 * (int64_t)c->n), oky = align256(okx + 4 * (int64_t)n_k);
  const int64_t okz = align256(oky + 4 * (int64_t)n_k);
  const int64_t okxi = align256(okz + 4 * (int64_t)n_k), okxl = align256(okxi + 4 * (int64_t)n_k);
  rc = cuda_check(cudaMemcpy(base + okx, kx, 4 * (size_t)n_k, cudaMemcpyHostToDevice), "copy wave vectors");
  if (!rc) rc = cuda_check(cudaMemcpy(base + oky, ky, 4 * (size_t)n_k, cudaMemcpyHostToDevice), "copy wave vectors");
  if (!rc) rc = cuda_check(cudaMemcpy(base + okz, kzv.data(), 4 * (size_t)n_k, cudaMemcpyHostToDevice),
                           "copy wave vectors");
  if (!rc) rc = cuda_check(cudaMemcpy(base + okxi, kxi.data(), 4 * (size_t)n_k, cudaMemcpyHostToDevice),
                           "copy wave vectors");
  if (!rc) rc = cuda_check(cudaMemcpy(base + okxl, kxl.data(), 4 * (size_t)n_k, cudaMemcpyHostToDevice),
                           "copy wave vectors");
  if (!rc) rc = cuda_check(cudaMemset(base, 0, 8 * (size_t)c->n), "zero counts");
  if (!rc) rc = cuda_check(cudaMemset(base + sums0, 0, (size_t)(need - sums0)), "zero sums");
  if (rc) return rc;
  for (int r = 0; r < c->n; ++r) {
    c->L.desc[r].off_tc_ring = ring[r];
    c->L.desc[r].off_tc_sums = sums[r];
    c->L.desc[r].off_tc_part = d3 ? part[r] : 0;
    c->L.desc[r].off_tc_tab = d3 ? tab[r] : 0;
  }
  rc = cuda_check(cudaMemcpy(c->ws + c->L.off_descs, c->L.desc.data(), c->n * sizeof(ReplicaDesc),
                             cudaMemcpyHostToDevice), "copy descriptors");
  if (rc) return rc;
  if (d3) {
    launch_point_tables(c->precision, descs_dev(c), c->n, base, c->stream);
    rc = cuda_check(cudaGetLastError(), "phase tables");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "phase tables");
    if (rc) return rc;
  }
  c->tc.base = base;
  c->tc.n_lags = n_lags;
  c->tc.n_k = n_k;
  c->tc.kx = reinterpret_cast<const int32_t*>(base + okx);
  c->tc.ky = reinterpret_cast<const int32_t*>(base + oky);
  c->tc.kz = reinterpret_cast<const int32_t*>(base + okz);
  c->tc.kxi = reinterpret_cast<const int32_t*>(base + okxi);
  c->tc.kxl = reinterpret_cast<const int32_t*>(base + okxl);
  c->tc.n_kx = n_kx;
  c->tc.count = reinterpret_cast<uint64_t*>(base);
  c->tc.part_blocks = d3 ? point_blocks(c, n_k) : 0;
  c->tc_smem = smem;
  c->tc_off_sums0 = sums0;
  c->tc_bytes = need;
  return FLB_OK;
}

int flb_get_time_correlator(flb_ctx* c, int replica, int fa, int fb, double* host_out, uint64_t* n_samples) {
  if (!c || !host_out) return set_error(FLB_EINVAL, "NULL argument");
  if (!c->tc.base) return set_error(FLB_ESTATE, "time correlators are off");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  const ReplicaDesc& d = c->L.desc[replica];
  int sa = -1, sb = -1;
  for (int s = 0; s < (int)d.n_fields; ++s) { if (d.field_id[s] == fa) sa = s; if (d.field_id[s] == fb) sb = s; }
  if (sa < 0 || sb < 0) return set_error(FLB_EINVAL, "fields %d, %d are not both sampled", fa, fb);
  int rc = flb_sync(c);
  if (rc) return rc;
  uint64_t cnt = 0;
  rc = cuda_check(cudaMemcpy(&cnt, c->tc.count + replica, 8, cudaMemcpyDeviceToHost), "read count");
  if (rc) return rc;
  const int T = c->tc.n_lags, nk = c->tc.n_k, F = (int)d.n_fields;
  std::vector<double> sums((size_t)T * F * F * nk * 2);
  rc = cuda_check(cudaMemcpy(sums.data(), c->tc.base + d.off_tc_sums, sums.size() * 8, cudaMemcpyDeviceToHost),
                  "read sums");
  if (rc) return rc;
  // moments: mu rho0; velocities (D2Q9, D1Q3 field ids 9, 10): kT / rho0
  auto var = [&](int f) { return (f < 9 || is3d(c->lattice)) ? d.mu * d.rho0 : d.kT / d.rho0; };
  const double vv = var(fa) * var(fb);
  const double V = (double)volume(d);
  const double norm = vv > 0 ? 1.0 / (V * std::sqrt(vv)) : 1.0 / V;
  for (int tau = 0; tau < T; ++tau)
    for (int j = 0; j < nk; ++j) {
      const size_t i = (((size_t)tau * F + sa) * F + sb) * nk + j;
      const double n_tau = cnt > (uint64_t)tau ? (double)(cnt - (uint64_t)tau) : 0.0;
      host_out[2 * ((size_t)tau * nk + j)] = n_tau > 0 ? sums[2 * i] / n_tau * norm : NAN;
      host_out[2 * ((size_t)tau * nk + j) + 1] = n_tau > 0 ? sums[2 * i + 1] / n_tau * norm : NAN;
    }
  if (n_samples) *n_samples = cnt;
  return FLB_OK;
}


const char* flb_last_error(void) { return g_last_error.c_str(); }

int flb_workspace_bytes(int precision, const flb_replica* reps, int n_replicas, size_t* bytes_out) {
  if (!bytes_out) return set_error(FLB_EINVAL, "bytes_out is NULL");
  Layout L;
  const int rc = plan(precision, reps, n_replicas, L);
  if (rc) return rc;
  *bytes_out = (size_t)L.total;
  return FLB_OK;
}

int flb_create(int precision, const flb_replica* reps, int n_replicas, void* dev_workspace,
               size_t workspace_bytes, void* cuda_stream, flb_ctx** out) {
  NvtxRange range("flb_create");
  if (!out) return set_error(FLB_EINVAL, "out is NULL");
  *out = nullptr;
  Layout L;
  int rc = plan(precision, reps, n_replicas, L);
  if (rc) return rc;
  if (!dev_workspace) return set_error(FLB_EINVAL, "workspace is NULL");
  if (((uintptr_t)dev_workspace) & 255) return set_error(FLB_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < (size_t)L.total)
    return set_error(FLB_ENOMEM, "workspace %zu bytes < required %lld", workspace_bytes, (long long)L.total);
  flb_ctx* c = new flb_ctx();
  c->precision = precision; c->lattice = reps[0].lattice; c->n = n_replicas;
  c->reps.assign(reps, reps + n_replicas);
  c->L = std::move(L);
  c->ws = static_cast<char*>(dev_workspace);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if ((rc = cuda_check(set_fft_smem_limits(), "smem limits"))) { delete c; return rc; }
  if (c->lattice == FLB_D1Q3) {      // the fused kernel holds a replica in one block's shared memory
    size_t smem = 0;
    for (const ReplicaDesc& d : c->L.desc)
      smem = std::max(smem, d1q3_fused_smem(precision, d.nx, (int)d.n_fields));
    c->fused_smem = smem <= kFusedSmemMax ? smem : 0;
  }
  cudaStream_t st = c->stream;
  const Layout& Lc = c->L;
  rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_descs, Lc.desc.data(), n_replicas * sizeof(ReplicaDesc),
                                  cudaMemcpyHostToDevice, st), "copy descriptors");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_vb_step, Lc.vb_step.data(), 8 * n_replicas, cudaMemcpyHostToDevice, st), "copy vb");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_vb_rows, Lc.vb_rows.data(), 8 * n_replicas, cudaMemcpyHostToDevice, st), "copy vb");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_vb_cols, Lc.vb_cols.data(), 8 * n_replicas, cudaMemcpyHostToDevice, st), "copy vb");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_vb_cols_a, Lc.vb_cols_a.data(), 8 * n_replicas, cudaMemcpyHostToDevice, st), "copy vb");
  std::vector<double> feq(kFeqStride * (size_t)n_replicas);
  for (int r = 0; r < n_replicas; ++r) feq0_host(reps[r], &feq[kFeqStride * (size_t)r]);
  if (!rc) rc = cuda_check(cudaMemcpyAsync(c->ws + Lc.off_feq0, feq.data(), feq.size() * 8, cudaMemcpyHostToDevice, st), "copy feq0");
  if (!rc) rc = cuda_check(cudaMemsetAsync(c->ws + Lc.off_status, 0, sizeof(DevStatus), st), "status");
  if (!rc) rc = cuda_check(cudaMemsetAsync(c->ws + Lc.off_mlp, 0, mlp_weights_bytes(), st), "mlp");
  for (int r = 0; r < n_replicas && !rc; ++r) {
    const ReplicaDesc& d = Lc.desc[r];
    const int64_t V = volume(d);
    double* sums = reinterpret_cast<double*>(c->ws + Lc.off_sums) + 4 * r;
    rc = cuda_check(cudaMemsetAsync(sums, 0, 32, st), "sums");
    if (rc) break;
    const double* feq0 = reinterpret_cast<const double*>(c->ws + Lc.off_feq0) + kFeqStride * r;
    double* partial = reinterpret_cast<double*>(c->ws + Lc.off_partial);
    if (is3d(c->lattice))
      launch_init3(d.q, precision, descs_dev(c), r, c->ws, (int)reps[r].init_mode, feq0, sums, partial, V, st);
    else launch_init(precision, descs_dev(c), r, c->ws, (int)reps[r].init_mode, feq0, sums, partial, V, st);
    if (d.n_pairs) {
      launch_twiddles(precision, c->ws + d.off_tw_x, d.nx, st);
      launch_twiddles(precision, c->ws + d.off_tw_y, d.ny, st);
    }
  }
  if (!rc) rc = reset_stats_async(c);
  if (!rc) rc = cuda_check(cudaGetLastError(), "init launch");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "init sync");
  if (rc) { delete c; return rc; }
  *out = c;
  return FLB_OK;
}

// Issue one step (and its sampling) on stream st.  With S.step_dev set, S.step is the
// offset from the device step counter (graph capture); otherwise the absolute step.
// kernels issued on behalf of flb_run: counted, or, during a capture, added to the graph's count
static void count_kernels(flb_ctx* c, uint64_t n) {
  if (c->capturing) c->captured += n;
  else c->launches += n;
}
// launches of a multi-path pass: one per bit of the path mask (FP64: the one kernel)
static int path_launches(int precision, int paths) { return precision == FLB_FP64 ? 1 : __builtin_popcount(paths); }

static void launch_step_any(flb_ctx* c, int vec, int staged, const StepLaunch& S, bool sample, cudaStream_t st) {
  if (is3d(c->lattice)) launch_step3(c->L.q, c->precision, vec, S, sample, st);
  else if (staged) launch_step_bulk(vec, S, sample, c->mlp_on, st);
  else launch_step(c->lattice, c->precision, vec, S, sample, c->mlp_on, st);
}

// The accumulation pass (pass 2b and the pair sums, then the time correlators) over the
// samples waiting in the spectrum slots, slot 0 first; nothing when none is waiting.
static void flush_samples(flb_ctx* c, const StepLaunch& S, cudaStream_t st) {
  const Layout& L = c->L;
  if (!c->pending) return;
  const int cols_grid = (int)std::min<int64_t>(L.n_vb_cols, (int64_t)c->sms * 8);
  launch_fft_cols(c->precision, S.descs, reinterpret_cast<const int64_t*>(c->ws + L.off_vb_cols), c->n,
                  L.n_vb_cols, c->ws, L.ncol, cols_grid, kColsBlock, L.cols_smem, st, c->tc, L.cols_paths,
                  c->pending, L.max_fields);
  count_kernels(c, path_launches(c->precision, L.cols_paths));
  c->pending = 0;
  if (c->tc.base) {
    int maxF = 0;
    for (const ReplicaDesc& d : L.desc) maxF = std::max(maxF, (int)d.n_fields);
    launch_time_corr(S.descs, c->n, maxF, c->tc, st);
    count_kernels(c, 2);
  }
}

static void issue_step(flb_ctx* c, StepLaunch& S, bool sample, cudaStream_t st) {
  NvtxRange range(sample ? "flb step + sample" : "flb step");
  const Layout& L = c->L;
  launch_step_any(c, L.vec, L.staged, S, sample, st);
  count_kernels(c, 1);
  if (sample && is3d(c->lattice)) {
    // direct transforms at the chosen wave vectors, then the time correlators
    if (c->tc.base) {
      int maxF = 0;
      for (const ReplicaDesc& d : L.desc) maxF = std::max(maxF, (int)d.n_fields);
      launch_point_dft(c->precision, S.descs, c->n, maxF * c->tc.n_k, c->ws, c->tc, c->tc_smem, st);
      launch_time_corr(S.descs, c->n, maxF, c->tc, st);
      count_kernels(c, 4);              // point transforms, their finishing pass, lagged products, ring advance
    }
  } else if (sample) {
    // the row and inner column transforms into the free spectrum slot; the accumulation
    // pass once both slots hold a sample (or right away without folding: one slot, or
    // time correlators, which take their ring entries one sample at a time)
    const bool fold = L.fold == 2 && !c->tc.base;
    const int slot = fold ? c->pending : 0;
    const int rows_grid = (int)std::min<int64_t>(L.n_vb_rows, (int64_t)c->sms * 8);
    const int cols_a_grid = (int)std::min<int64_t>(L.n_vb_cols_a, (int64_t)c->sms * 8);
    launch_fft_rows(c->precision, S.descs, reinterpret_cast<const int64_t*>(c->ws + L.off_vb_rows), c->n,
                    L.n_vb_rows, c->ws, rows_grid, L.rows_block, L.rows_smem, st, slot, L.rows_paths, c->sms);
    if (L.n_vb_cols_a)
      launch_fft_cols_a(c->precision, S.descs, reinterpret_cast<const int64_t*>(c->ws + L.off_vb_cols_a), c->n,
                        L.n_vb_cols_a, c->ws, L.ncol, cols_a_grid, kColsBlock, L.cols_smem, st,
                        L.cols_a_paths, slot, c->sms);
    count_kernels(c, path_launches(c->precision, L.rows_paths) +
                         (L.n_vb_cols_a ? path_launches(c->precision, L.cols_a_paths) : 0));
    c->pending = slot + 1;
    if (!fold || c->pending == 2) flush_samples(c, S, st);
  }
}

static StepLaunch step_launch(flb_ctx* c) {
  const Layout& L = c->L;
  StepLaunch S;
  S.descs = descs_dev(c);
  S.vb_begin = reinterpret_cast<const int64_t*>(c->ws + L.off_vb_step);
  S.n_reps = c->n;
  S.n_vblocks = L.n_vb_step;
  S.ws = c->ws;
  S.mlp = c->ws + L.off_mlp;
  S.block = kStepBlock;
  S.grid = (int)std::min<int64_t>(L.n_vb_step, c->step_grid > 0 ? (int64_t)c->step_grid : (int64_t)c->sms * 16);
  S.parity = 0;
  S.step = 0;
  S.status = status_dev(c);
  S.sms = c->sms;
  S.desc0 = &L.desc[0];
  S.net_engine = c->net_engine;
  for (const ReplicaDesc& d : L.desc) S.noise_general = S.noise_general || d.noise_mode != 0;
  return S;
}

static void drop_graphs(flb_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// A chunk of `len` steps starting at a step that is a multiple of len, sampling at its
// steps o with o % every == 0 (every = 0: no sampling; len is a multiple of every); it
// ends by advancing the device step counter by len.
static int chunk_graph(flb_ctx* c, uint32_t len, uint32_t every, cudaGraphExec_t* out, uint64_t* kernels) {
  for (auto& g : c->graphs)
    if (g.len == len && g.every == every) { *out = g.exec; *kernels = g.kernels; return FLB_OK; }
  if (!c->cap_stream) {
    int rc = cuda_check(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (rc) return rc;
  }
  StepLaunch S = step_launch(c);
  S.step_dev = reinterpret_cast<const uint64_t*>(c->ws + c->L.off_stepdev);
  int rc = cuda_check(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc) return rc;
  c->capturing = true;
  c->captured = 0;
  for (uint32_t o = 0; o < len; ++o) {
    S.step = o;
    issue_step(c, S, every && o % every == 0, c->cap_stream);
  }
  flush_samples(c, S, c->cap_stream);           // a chunk leaves no sample waiting
  launch_advance_step(reinterpret_cast<uint64_t*>(c->ws + c->L.off_stepdev), len, c->cap_stream);
  count_kernels(c, 1);
  c->capturing = false;
  cudaGraph_t graph = nullptr;
  rc = cuda_check(cudaStreamEndCapture(c->cap_stream, &graph), "end capture");
  if (rc) return rc;
  cudaGraphExec_t exec = nullptr;
  rc = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "instantiate graph");
  cudaGraphDestroy(graph);
  if (rc) return rc;
  c->graphs.push_back({len, every, exec, c->captured});
  *kernels = c->captured;
  *out = exec;
  return FLB_OK;
}

int flb_run(flb_ctx* c, uint64_t n_steps, uint32_t sample_every) {
  NvtxRange range("flb_run");
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  const Layout& L = c->L;
  const bool sampling = sample_every && L.any_fields;
  if (c->fused_smem && c->use_graphs && !c->tc.base) {
    // D1Q3: runs of up to kFusedChunk steps with their sampling in one launch
    NvtxRange fused_range("flb fused D1Q3 steps");
    const uint32_t every = sampling ? sample_every : 0;
    for (uint64_t i = 0; i < n_steps;) {
      const uint32_t n = (uint32_t)std::min<uint64_t>(n_steps - i, kFusedChunk);
      int rc = cuda_check(launch_d1q3_fused(c->precision, descs_dev(c), c->n, c->ws, c->step, n, every,
                                            c->fused_smem, c->stream), "fused D1Q3 launch");
      if (rc) return rc;
      count_kernels(c, 1);
      if (every) {               // samples at the steps t in [step, step + n) with t % every == 0
        const uint64_t first = (c->step + every - 1) / every * every;
        if (first < c->step + n) c->n_samples += (c->step + n - 1 - first) / every + 1;
      }
      c->step += n;
      i += n;
    }
    return FLB_OK;
  }
  StepLaunch S = step_launch(c);
  auto plain = [&]() {
    const uint64_t t = c->step;
    const bool sample = sampling && (t % sample_every) == 0;
    S.parity = (int)(t & 1);
    S.step = (uint32_t)t;
    issue_step(c, S, sample, c->stream);
    if (sample) ++c->n_samples;
    ++c->step;
  };
  // chunks of `len` steps (whole sampling periods, at least kGraphChunk steps) replay a
  // captured graph; steps before the first aligned chunk and after the last one are
  // issued directly
  const uint32_t every = sampling ? sample_every : 0;
  // samples per chunk: enough for kGraphChunk steps, even when samples are folded in pairs
  uint64_t per_chunk = sampling ? (kGraphChunk + sample_every - 1) / sample_every : 0;
  if (sampling && c->L.fold == 2 && !c->tc.base) per_chunk += per_chunk & 1;
  const uint64_t len64 = sampling ? per_chunk * sample_every : kGraphChunk;
  uint64_t i = 0;
  if (c->use_graphs && len64 <= kMaxGraphChunk && n_steps >= 2 * len64) {
    const uint32_t len = (uint32_t)len64;
    while (i < n_steps && (c->step % len) != 0) { plain(); ++i; }
    const uint64_t chunks = (n_steps - i) / len;
    if (chunks) {
      flush_samples(c, S, c->stream);            // the chunks start with no sample waiting
      cudaGraphExec_t exec = nullptr;
      uint64_t per_chunk_kernels = 0;
      int rc = chunk_graph(c, len, every, &exec, &per_chunk_kernels);
      if (rc) return rc;
      launch_set_step(reinterpret_cast<uint64_t*>(c->ws + L.off_stepdev), c->step, c->stream);
      count_kernels(c, 1 + chunks * per_chunk_kernels);
      NvtxRange chunks_range(sampling ? "flb graph chunks (sampling)" : "flb graph chunks");
      for (uint64_t k = 0; k < chunks; ++k) {
        rc = cuda_check(cudaGraphLaunch(exec, c->stream), "graph launch");
        if (rc) return rc;
      }
      c->step += chunks * len;
      if (sampling) c->n_samples += chunks * (len / every);
      i += chunks * len;
    }
  }
  while (i < n_steps) { plain(); ++i; }
  flush_samples(c, S, c->stream);                // a run leaves no sample waiting
  return cuda_check(cudaGetLastError(), "flb_run launch");
}

int flb_probe_wait_timeout(flb_ctx* c, uint64_t limit_clocks) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  if (limit_clocks < 1 || limit_clocks > (1ull << 32))
    return set_error(FLB_EINVAL, "limit_clocks must be in 1 .. 2^32");
  launch_wait_probe(status_dev(c), (long long)limit_clocks, c->stream);
  return cuda_check(cudaGetLastError(), "wait probe launch");
}

int flb_kernel_launches(flb_ctx* c, uint64_t* count) {
  if (!c || !count) return set_error(FLB_EINVAL, "NULL argument");
  *count = c->launches;
  return FLB_OK;
}

int flb_set_graphs(flb_ctx* c, int enable) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  c->use_graphs = enable != 0;
  if (!enable) {
    int rc = cuda_check(cudaStreamSynchronize(c->stream), "graphs");
    if (rc) return rc;
    drop_graphs(c);
  }
  return FLB_OK;
}

int flb_sync(flb_ctx* c) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "flb_sync");
  if (rc) return rc;
  DevStatus s;
  rc = cuda_check(cudaMemcpy(&s, status_dev(c), sizeof s, cudaMemcpyDeviceToHost), "status read");
  if (rc) return rc;
  if (s.error) return set_error(s.error, "device reported status %d on replica %d", s.error, s.replica);
  return FLB_OK;
}

int flb_reset_stats(flb_ctx* c) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  return reset_stats_async(c);
}

int flb_get_step(flb_ctx* c, uint64_t* step_out) {
  if (!c || !step_out) return set_error(FLB_EINVAL, "NULL argument");
  *step_out = c->step;
  return FLB_OK;
}

int flb_get_correlator(flb_ctx* c, int replica, int fa, int fb, double* host_out, uint64_t* n_samples) {
  if (!c || !host_out) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  const ReplicaDesc& d = c->L.desc[replica];
  if (is3d(c->lattice))
    return set_error(FLB_EINVAL, "3D correlators are taken at chosen wave vectors (flb_set_time_correlator3)");
  int sa = -1, sb = -1;
  for (int s = 0; s < (int)d.n_fields; ++s) { if (d.field_id[s] == fa) sa = s; if (d.field_id[s] == fb) sb = s; }
  if (sa < 0 || sb < 0) return set_error(FLB_EINVAL, "fields %d, %d are not both sampled", fa, fb);
  if (c->n_samples == 0) return set_error(FLB_ESTATE, "no samples accumulated");
  int rc = flb_sync(c);
  if (rc) return rc;
  const bool swap = sa > sb;
  const int lo = swap ? sb : sa, hi = swap ? sa : sb;
  int pr = -1;
  for (int k = 0; k < d.n_pairs; ++k) if (d.pair_a[k] == lo && d.pair_b[k] == hi) pr = k;
  const int nx = d.nx, ny = d.ny, hn = d.half_nx;
  const bool autoc = lo == hi;
  const int bc = d.acc_ncol;                              // blocked layout (see ReplicaDesc)
  const int n1 = 1 << d.log2n1, n2 = ny >> d.log2n1, tiles = (hn + bc - 1) / bc;
  std::vector<double> acc((size_t)ny * tiles * bc * (autoc ? 1 : 2));
  rc = cuda_check(cudaMemcpy(acc.data(), c->ws + d.pair_off[pr], acc.size() * 8, cudaMemcpyDeviceToHost), "read sums");
  if (rc) return rc;
  std::vector<double> m0(d.n_fields);
  rc = cuda_check(cudaMemcpy(m0.data(), c->ws + d.off_mean0, 8 * d.n_fields, cudaMemcpyDeviceToHost), "read means");
  if (rc) return rc;
  const double ns = (double)c->n_samples;
  const double V = (double)nx * ny;
  auto var = [&](int f) { return f < 9 ? d.mu * d.rho0 : d.kT / d.rho0; };
  const double vv = var(fa) * var(fb);
  const double norm = vv > 0 ? 1.0 / (V * std::sqrt(vv)) : 1.0 / V;
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nx; ++kx) {
      double re, im;
      int hy = ky, hx = kx;
      bool conj = false;
      if (kx > nx / 2) { hx = nx - kx; hy = (ny - ky) % ny; conj = true; }
      const size_t idx = ((size_t)((hy & (n1 - 1)) * tiles + hx / bc) * n2 + (hy >> d.log2n1)) * bc + hx % bc;
      if (autoc) { re = acc[idx]; im = 0.0; }
      else { re = acc[2 * idx]; im = acc[2 * idx + 1]; }
      if (conj) im = -im;
      if (swap) im = -im;
      re /= ns; im /= ns;
      if (kx == 0 && ky == 0) re -= (m0[sa] / ns) * (m0[sb] / ns);
      host_out[2 * ((size_t)ky * nx + kx)] = re * norm;
      host_out[2 * ((size_t)ky * nx + kx) + 1] = im * norm;
    }
  if (n_samples) *n_samples = c->n_samples;
  return FLB_OK;
}

int flb_get_populations(flb_ctx* c, int replica, double* host_out) {
  if (!c || !host_out) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  int rc = flb_sync(c);
  if (rc) return rc;
  const ReplicaDesc& d = c->L.desc[replica];
  const int64_t V = volume(d);
  const char* src = c->ws + d.off_pop[c->step & 1];
  if (c->precision == FLB_FP64)
    return cuda_check(cudaMemcpy(host_out, src, d.q * V * 8, cudaMemcpyDeviceToHost), "read populations");
  std::vector<float> tmp((size_t)d.q * V);
  rc = cuda_check(cudaMemcpy(tmp.data(), src, tmp.size() * 4, cudaMemcpyDeviceToHost), "read populations");
  if (rc) return rc;
  for (int i = 0; i < d.q; ++i) {
    const double wr = lattice_weight(d.q, i) * d.rho0;
    for (int64_t s = 0; s < V; ++s) host_out[i * V + s] = wr + (double)tmp[i * V + s];
  }
  return FLB_OK;
}

int flb_get_populations_window(flb_ctx* c, int replica, int x0, int y0, int w, int h, double* host_out) {
  if (!c || !host_out) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  const ReplicaDesc& d = c->L.desc[replica];
  if (is3d(c->lattice)) return set_error(FLB_EINVAL, "windows are read from D1Q3 / D2Q9 lattices");
  if (w <= 0 || h <= 0 || x0 < 0 || y0 < 0 || x0 + w > d.nx || y0 + h > d.ny)
    return set_error(FLB_EINVAL, "window [%d,%d)x[%d,%d) outside the %dx%d lattice", x0, x0 + w, y0, y0 + h, d.nx, d.ny);
  int rc = flb_sync(c);
  if (rc) return rc;
  const int64_t V = (int64_t)d.nx * d.ny;
  const size_t rs = c->precision == FLB_FP64 ? 8 : 4;
  const char* src = c->ws + d.off_pop[c->step & 1];
  std::vector<char> tmp((size_t)d.q * w * h * rs);
  for (int i = 0; i < d.q; ++i) {
    rc = cuda_check(cudaMemcpy2D(tmp.data() + (size_t)i * w * h * rs, w * rs,
                                 src + ((size_t)i * V + (size_t)y0 * d.nx + x0) * rs, (size_t)d.nx * rs,
                                 w * rs, h, cudaMemcpyDeviceToHost), "read window");
    if (rc) return rc;
  }
  for (int i = 0; i < d.q; ++i) {
    const double wr = c->precision == FLB_FP64 ? 0.0 : (d.q == 9 ? kW9[i] : kW3[i]) * d.rho0;
    for (size_t s = 0; s < (size_t)w * h; ++s) {
      const size_t k = (size_t)i * w * h + s;
      host_out[k] = rs == 8 ? reinterpret_cast<const double*>(tmp.data())[k]
                            : wr + (double)reinterpret_cast<const float*>(tmp.data())[k];
    }
  }
  return FLB_OK;
}

int flb_get_fields(flb_ctx* c, int replica, double* host_out) {
  if (!c || !host_out) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  const ReplicaDesc& d = c->L.desc[replica];
  if (!d.n_fields) return set_error(FLB_EINVAL, "replica %d samples no fields", replica);
  if (c->n_samples == 0) return set_error(FLB_ESTATE, "no samples taken");
  int rc = flb_sync(c);
  if (rc) return rc;
  const size_t n = (size_t)d.n_fields * volume(d);
  if (c->precision == FLB_FP64)
    return cuda_check(cudaMemcpy(host_out, c->ws + d.off_fields, n * 8, cudaMemcpyDeviceToHost), "read fields");
  std::vector<float> tmp(n);
  rc = cuda_check(cudaMemcpy(tmp.data(), c->ws + d.off_fields, n * 4, cudaMemcpyDeviceToHost), "read fields");
  if (rc) return rc;
  for (size_t i = 0; i < n; ++i) host_out[i] = tmp[i];
  return FLB_OK;
}

int flb_set_populations(flb_ctx* c, int replica, const double* host_in) {
  if (!c || !host_in) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  int rc = flb_sync(c);
  if (rc) return rc;
  const ReplicaDesc& d = c->L.desc[replica];
  const int64_t V = volume(d);
  char* dst = c->ws + d.off_pop[c->step & 1];
  if (c->precision == FLB_FP64)
    return cuda_check(cudaMemcpy(dst, host_in, d.q * V * 8, cudaMemcpyHostToDevice), "write populations");
  std::vector<float> tmp((size_t)d.q * V);
  for (int i = 0; i < d.q; ++i) {
    const double wr = lattice_weight(d.q, i) * d.rho0;
    for (int64_t s = 0; s < V; ++s) tmp[i * V + s] = (float)(host_in[i * V + s] - wr);
  }
  return cuda_check(cudaMemcpy(dst, tmp.data(), tmp.size() * 4, cudaMemcpyHostToDevice), "write populations");
}

int flb_get_conserved(flb_ctx* c, int replica, double* out4) {
  if (!c || !out4) return set_error(FLB_EINVAL, "NULL argument");
  if (replica < 0 || replica >= c->n) return set_error(FLB_EINVAL, "replica %d out of range", replica);
  const ReplicaDesc& d = c->L.desc[replica];
  double* sums = reinterpret_cast<double*>(c->ws + c->L.off_sums) + 4 * replica;
  double* partial = reinterpret_cast<double*>(c->ws + c->L.off_partial);
  if (is3d(c->lattice))
    launch_conserved3(d.q, c->precision, descs_dev(c), replica, c->ws, (int)(c->step & 1), sums, partial, status_dev(c),
                      volume(d), c->stream);
  else
    launch_conserved(c->precision, descs_dev(c), replica, c->ws, (int)(c->step & 1), sums, partial, status_dev(c),
                     volume(d), c->stream);
  int rc = cuda_check(cudaGetLastError(), "conserved launch");
  if (rc) return rc;
  rc = flb_sync(c);
  if (rc) return rc;
  return cuda_check(cudaMemcpy(out4, sums, 32, cudaMemcpyDeviceToHost), "read sums");
}

int flb_set_mlp(flb_ctx* c, const uint16_t* w_bf16, const float* biases, int enable) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  if (c->lattice != FLB_D2Q9) return set_error(FLB_EINVAL, "the noise-scale network is D2Q9 only");
  if (c->precision != FLB_FP32_DEV) return set_error(FLB_EINVAL, "the noise-scale network runs on the FP32 path");
  if (enable && (!w_bf16 || !biases)) return set_error(FLB_EINVAL, "NULL weights");
  if (enable) {
    const size_t nf = mlp_weights_bytes() / 4;
    c->mlp_host.assign(nf, 0.f);
    for (int i = 0; i < kMlpWeights; ++i) {
      const uint32_t bits = (uint32_t)w_bf16[i] << 16;
      float v;
      memcpy(&v, &bits, 4);
      c->mlp_host[i] = v;
    }
    for (int i = 0; i < kMlpBiases; ++i) c->mlp_host[kMlpWeights + i] = biases[i];
    int rc = cuda_check(cudaMemcpyAsync(c->ws + c->L.off_mlp, c->mlp_host.data(), nf * 4, cudaMemcpyHostToDevice,
                                        c->stream), "copy mlp");
    if (rc) return rc;
    rc = cuda_check(cudaStreamSynchronize(c->stream), "copy mlp");
    if (rc) return rc;
  }
  if ((enable != 0) != c->mlp_on) {
    int rc = cuda_check(cudaStreamSynchronize(c->stream), "set mlp");
    if (rc) return rc;
    drop_graphs(c);
  }
  c->mlp_on = enable != 0;
  return FLB_OK;
}

// Checkpoint copies between host memory and the workspace: the regions are cut into
// 64 MiB pieces issued round-robin on four streams (one cudaMemcpyAsync each), so that
// several copy engines work at once, then all four streams are waited for.
struct CopyStripe {
  static constexpr size_t kPiece = 64ull << 20;
  flb_ctx* c;
  int next = 0;
  int rc = FLB_OK;
  void copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    for (size_t o = 0; o < bytes && rc == FLB_OK; o += kPiece) {
      cudaStream_t& s = c->copy_streams[next];
      next = (next + 1) % 4;
      if (!s && (rc = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "copy stream"))) return;
      rc = cuda_check(cudaMemcpyAsync(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o,
                                      std::min(kPiece, bytes - o), kind, s), "checkpoint copy");
    }
  }
  int finish() {
    for (cudaStream_t s : c->copy_streams) {
      if (!s) continue;
      const int e = cuda_check(cudaStreamSynchronize(s), "checkpoint copy");
      if (!rc) rc = e;
    }
    return rc;
  }
};

int flb_save(flb_ctx* c, void* host_buf, size_t* bytes_inout) {
  NvtxRange range("flb_save");
  if (!c || !bytes_inout) return set_error(FLB_EINVAL, "NULL argument");
  const int64_t rs = c->precision == FLB_FP64 ? 8 : 4;
  size_t need = 64;
  for (int r = 0; r < c->n; ++r) {
    const ReplicaDesc& d = c->L.desc[r];
    need += d.q * (size_t)volume(d) * rs;
    if (d.n_pairs) need += (size_t)(d.off_mean0 + 8 * d.n_fields - d.pair_off[0]);
  }
  if (!host_buf) { *bytes_inout = need; return FLB_OK; }
  if (*bytes_inout < need) return set_error(FLB_EINVAL, "buffer of %zu bytes < %zu", *bytes_inout, need);
  int rc = flb_sync(c);
  if (rc) return rc;
  char* p = static_cast<char*>(host_buf);
  uint64_t hdr[8] = {0x464c4243484b5031ull, (uint64_t)c->precision, (uint64_t)c->n, c->step, c->n_samples,
                     (uint64_t)need, (uint64_t)c->lattice, 0};
  memcpy(p, hdr, 64);
  p += 64;
  CopyStripe cs{c};
  for (int r = 0; r < c->n; ++r) {
    const ReplicaDesc& d = c->L.desc[r];
    const size_t pb = d.q * (size_t)volume(d) * rs;
    cs.copy(p, c->ws + d.off_pop[c->step & 1], pb, cudaMemcpyDeviceToHost);
    p += pb;
    if (d.n_pairs) {
      const size_t ab = (size_t)(d.off_mean0 + 8 * d.n_fields - d.pair_off[0]);
      cs.copy(p, c->ws + d.pair_off[0], ab, cudaMemcpyDeviceToHost);
      p += ab;
    }
  }
  rc = cs.finish();
  if (rc) return rc;
  *bytes_inout = need;
  return FLB_OK;
}

int flb_load(flb_ctx* c, const void* host_buf, size_t bytes) {
  NvtxRange range("flb_load");
  if (!c || !host_buf) return set_error(FLB_EINVAL, "NULL argument");
  size_t need = 0;
  int rc = flb_save(c, nullptr, &need);
  if (rc) return rc;
  if (bytes != need) return set_error(FLB_EINVAL, "checkpoint has %zu bytes, context needs %zu", bytes, need);
  const char* p = static_cast<const char*>(host_buf);
  uint64_t hdr[8];
  memcpy(hdr, p, 64);
  if (hdr[0] != 0x464c4243484b5031ull || hdr[1] != (uint64_t)c->precision || hdr[2] != (uint64_t)c->n ||
      hdr[6] != (uint64_t)c->lattice)
    return set_error(FLB_EINVAL, "checkpoint does not match this context");
  rc = cuda_check(cudaStreamSynchronize(c->stream), "load");
  if (rc) return rc;
  p += 64;
  const uint64_t step = hdr[3];
  const int64_t rs = c->precision == FLB_FP64 ? 8 : 4;
  CopyStripe cs{c};
  for (int r = 0; r < c->n; ++r) {
    const ReplicaDesc& d = c->L.desc[r];
    const size_t pb = d.q * (size_t)volume(d) * rs;
    cs.copy(c->ws + d.off_pop[step & 1], p, pb, cudaMemcpyHostToDevice);
    p += pb;
    if (d.n_pairs) {
      const size_t ab = (size_t)(d.off_mean0 + 8 * d.n_fields - d.pair_off[0]);
      cs.copy(c->ws + d.pair_off[0], p, ab, cudaMemcpyHostToDevice);
      p += ab;
    }
  }
  rc = cs.finish();
  if (rc) return rc;
  c->step = step;
  c->n_samples = hdr[4];
  return FLB_OK;
}

static bool staged_ok(const flb_ctx* c) {
  if (c->precision != FLB_FP32_DEV || c->lattice != FLB_D2Q9) return false;
  for (int r = 0; r < c->n; ++r)
    if (c->L.desc[r].nx % 4) return false;
  return true;
}

int flb_set_step_config(flb_ctx* c, int vec, int grid_blocks, int staged) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  if (vec != 1 && vec != 2 && vec != 4) return set_error(FLB_EINVAL, "vec must be 1, 2 or 4");
  if (staged != 0 && staged != 1) return set_error(FLB_EINVAL, "staged must be 0 or 1");
  if (staged && !staged_ok(c)) return set_error(FLB_EINVAL, "the staged kernel needs the FP32 D2Q9 path, every nx a multiple of 4");
  if (vec > 1 && (c->precision != FLB_FP32_DEV || c->lattice == FLB_D1Q3))
    return set_error(FLB_EINVAL, "vec > 1 needs the FP32 D2Q9, D3Q15 or D3Q19 path");
  for (int r = 0; r < c->n && !staged; ++r) {
    if (c->L.desc[r].nx % vec) return set_error(FLB_EINVAL, "replica %d: nx not a multiple of vec = %d", r, vec);
    // one thread per site: unit indices are 32-bit
    if (vec == 1 && volume(c->L.desc[r]) >= (int64_t(1) << 31))
      return set_error(FLB_EINVAL, "replica %d: vec = 1 needs fewer than 2^31 sites", r);
  }
  if (grid_blocks < 0) return set_error(FLB_EINVAL, "grid_blocks must be >= 0");
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "step config");
  if (rc) return rc;
  drop_graphs(c);
  plan_step(c->lattice, vec, staged, c->L);
  rc = cuda_check(cudaMemcpy(c->ws + c->L.off_descs, c->L.desc.data(), c->n * sizeof(ReplicaDesc),
                             cudaMemcpyHostToDevice), "copy descriptors");
  if (!rc) rc = cuda_check(cudaMemcpy(c->ws + c->L.off_vb_step, c->L.vb_step.data(), 8 * (size_t)c->n,
                                      cudaMemcpyHostToDevice), "copy vb");
  if (!rc) c->step_grid = grid_blocks;
  return rc;
}

int flb_get_step_config(flb_ctx* c, int* vec, int* grid_blocks, int* staged) {
  if (!c || !vec || !grid_blocks || !staged) return set_error(FLB_EINVAL, "NULL argument");
  *vec = c->L.vec;
  *staged = c->L.staged;
  *grid_blocks = (int)std::min<int64_t>(c->L.n_vb_step, c->step_grid > 0 ? (int64_t)c->step_grid : (int64_t)c->sms * 16);
  return FLB_OK;
}

int flb_debug_bounds(uint64_t* violations, uint32_t* first_site, int clear) {
  if (!violations || !first_site) return set_error(FLB_EINVAL, "NULL argument");
  *violations = 0;
  *first_site = 0;
  if (oob_registry().empty())
    return set_error(FLB_ESTATE, "this library was built without bounds checks (build with --checked)");
  int rc = cuda_check(cudaDeviceSynchronize(), "bounds counters");
  if (rc) return rc;
  for (const OobEntry& e : oob_registry()) {
    unsigned int v[2] = {0u, 0u};
    rc = cuda_check((cudaError_t)e.read(v), "read bounds counters");
    if (rc) return rc;
    *violations += v[0];
    if (!*first_site && v[1]) *first_site = v[1];
    if (clear) {
      rc = cuda_check((cudaError_t)e.clear(), "clear bounds counters");
      if (rc) return rc;
    }
  }
  return FLB_OK;
}

int flb_set_network_engine(flb_ctx* c, int engine) {
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  if (engine != FLB_NET_WARP && engine != FLB_NET_TCGEN05)
    return set_error(FLB_EINVAL, "engine must be FLB_NET_WARP or FLB_NET_TCGEN05");
  if (engine == c->net_engine) return FLB_OK;
  int rc = cuda_check(cudaStreamSynchronize(c->stream), "network engine");
  if (rc) return rc;
  drop_graphs(c);
  c->net_engine = engine;
  return FLB_OK;
}

int flb_get_network_engine(flb_ctx* c, int* engine) {
  if (!c || !engine) return set_error(FLB_EINVAL, "NULL argument");
  *engine = c->net_engine;
  return FLB_OK;
}

int flb_autotune(flb_ctx* c, int trials, int* vec_out, int* grid_out, int* staged_out, double* ms_out) {
  NvtxRange range("flb_autotune");
  if (!c) return set_error(FLB_EINVAL, "ctx is NULL");
  if (trials < 1) return set_error(FLB_EINVAL, "trials must be >= 1");
  cudaEvent_t e0, e1;
  int rc = cuda_check(cudaEventCreate(&e0), "event");
  if (rc) return rc;
  rc = cuda_check(cudaEventCreate(&e1), "event");
  if (rc) { cudaEventDestroy(e0); return rc; }
  const int vecs[3] = {1, 2, 4};
  int best_vec = c->L.vec, best_grid = c->step_grid, best_staged = c->L.staged, best_engine = c->net_engine;
  float best = 1e30f;
  // direct kernels with either network engine (when the network is on), then the staged kernel
  const bool two_engines = c->mlp_on && c->lattice == FLB_D2Q9;
  for (int cfg = 0; cfg < 9 && !rc; ++cfg) {
    const int vec = vecs[cfg % 3], staged = cfg / 3 == 2 ? 1 : 0;
    const int engine = cfg / 3 == 1 ? FLB_NET_TCGEN05 : FLB_NET_WARP;
    if (engine == FLB_NET_TCGEN05 && !two_engines) continue;
    if (vec > 1 && (c->precision != FLB_FP32_DEV || c->lattice == FLB_D1Q3)) continue;
    if (staged && !staged_ok(c)) continue;
    bool ok = true;
    for (int r = 0; r < c->n && !staged; ++r)
      ok = ok && c->L.desc[r].nx % vec == 0 && (vec > 1 || volume(c->L.desc[r]) < (int64_t(1) << 31));
    if (!ok) continue;
    // the staged kernel is persistent (its launcher caps the grid at the resident blocks)
    const int mults[5] = {2, 4, 8, 16, 0};
    for (int mi = staged ? 4 : 0; mi < 5 && !rc; ++mi) {
      const int grid = mults[mi] ? mults[mi] * c->sms : 0;
      rc = flb_set_step_config(c, vec, grid ? grid : INT32_MAX, staged);
      if (rc) break;
      // dry runs: the same step (same input buffer, same step index) launched
      // repeatedly; it only rewrites the buffer the next real step overwrites.
      StepLaunch S;
      S.descs = descs_dev(c);
      S.vb_begin = reinterpret_cast<const int64_t*>(c->ws + c->L.off_vb_step);
      S.n_reps = c->n;
      S.n_vblocks = c->L.n_vb_step;
      S.ws = c->ws;
      S.mlp = c->ws + c->L.off_mlp;
      S.block = kStepBlock;
      S.grid = (int)std::min<int64_t>(c->L.n_vb_step, c->step_grid);
      S.parity = (int)(c->step & 1);
      S.step = (uint32_t)c->step;
      S.status = status_dev(c);
      S.sms = c->sms;
      S.desc0 = &c->L.desc[0];
      S.net_engine = engine;
      for (const ReplicaDesc& d : c->L.desc) S.noise_general = S.noise_general || d.noise_mode != 0;
      auto launch = [&] { launch_step_any(c, vec, staged, S, false, c->stream); };
      launch();
      cudaEventRecord(e0, c->stream);
      for (int t = 0; t < trials; ++t) launch();
      cudaEventRecord(e1, c->stream);
      rc = cuda_check(cudaEventSynchronize(e1), "autotune");
      if (rc) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= trials;
      if (ms < best) { best = ms; best_vec = vec; best_grid = S.grid; best_staged = staged; best_engine = engine; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = flb_set_step_config(c, best_vec, best_grid, best_staged);
  if (rc) return rc;
  if (two_engines) {
    rc = flb_set_network_engine(c, best_engine);
    if (rc) return rc;
  }
  if (vec_out) *vec_out = best_vec;
  if (grid_out) *grid_out = best_grid;
  if (staged_out) *staged_out = best_staged;
  if (ms_out) *ms_out = best;
  return FLB_OK;
}

void flb_destroy(flb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaStream_t s : c->copy_streams)
    if (s) cudaStreamDestroy(s);
  delete c;
}

int flb_stability(const flb_replica* rep, int max_k, double* radius_out, int32_t* k_out) {
  if (!rep || !radius_out) return set_error(FLB_EINVAL, "NULL argument");
  if (max_k < 1) return set_error(FLB_EINVAL, "max_k must be >= 1");
  int rc = validate(FLB_FP64, rep, 1);
  if (rc) return rc;
  const flb_replica& p = *rep;
  const int lat = p.lattice, q = lattice_q(lat), nc0 = first_nonconserved(lat);
  int v[20][3];
  double w[20], m[20][20];
  lattice_tables(lat, v, w, m);
  const double u[3] = {p.u0[0], lat == FLB_D1Q3 ? 0.0 : p.u0[1], is3d(lat) ? p.u0[2] : 0.0};
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  // E = d f^0 / d f, then J = I + N Lambda (M E - M)
  double E[20][20], ME[20][20], J[20][20];
  for (int i = 0; i < q; ++i) {
    const double vu = v[i][0] * u[0] + v[i][1] * u[1] + v[i][2] * u[2];
    const double drho = w[i] * (1.0 - 4.5 * vu * vu + 1.5 * uu);
    double dj[3];
    for (int a = 0; a < 3; ++a) dj[a] = w[i] * (3.0 * v[i][a] + 9.0 * vu * v[i][a] - 3.0 * u[a]);
    for (int j = 0; j < q; ++j) E[i][j] = drho + dj[0] * v[j][0] + dj[1] * v[j][1] + dj[2] * v[j][2];
  }
  for (int a = 0; a < q; ++a)
    for (int j = 0; j < q; ++j) {
      double acc = 0.0;
      for (int i = 0; i < q; ++i) acc += m[a][i] * E[i][j];
      ME[a][j] = acc;
    }
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double acc = i == j ? 1.0 : 0.0;
      for (int a = nc0; a < q; ++a) acc += w[i] * m[a][i] / p.tau[a] * (ME[a][j] - m[a][j]);
      J[i][j] = acc;
    }
  // the k-grid: N points per lattice dimension, N = min(n, max_k), k = 2 pi j / N
  const int N[3] = {std::min(p.nx, max_k), lat == FLB_D1Q3 ? 1 : std::min(p.ny, max_k),
                    is3d(lat) ? std::min(p.nz, max_k) : 1};
  const double two_pi = 6.283185307179586477;
  double best = 0.0;
  int bk[3] = {0, 0, 0};
  std::complex<double> A[20][20];
  for (int kz = 0; kz < N[2]; ++kz)
    for (int ky = 0; ky < N[1]; ++ky)
      for (int kx = 0; kx < N[0]; ++kx) {
        const double k[3] = {two_pi * kx / N[0], two_pi * ky / N[1], two_pi * kz / N[2]};
        for (int i = 0; i < q; ++i) {
          const double ph = -(k[0] * v[i][0] + k[1] * v[i][1] + k[2] * v[i][2]);
          const std::complex<double> e(std::cos(ph), std::sin(ph));
          for (int j = 0; j < q; ++j) A[i][j] = e * J[i][j];
        }
        const double r = spectral_radius_of(q, A);
        if (r > best) { best = r; bk[0] = kx; bk[1] = ky; bk[2] = kz; }
      }
  *radius_out = best;
  if (k_out) { k_out[0] = bk[0]; k_out[1] = bk[1]; k_out[2] = bk[2]; }
  return FLB_OK;
}

int flb_philox(const uint32_t* site_dev, int n, uint32_t step, uint32_t call, uint32_t tag, uint32_t stream,
               uint64_t seed, int fp32, uint32_t* words_out_dev, double* normals_out_dev, void* cuda_stream) {
  if (n < 0 || (n > 0 && !site_dev)) return set_error(FLB_EINVAL, "bad site array");
  if (call > 255 || tag > 0xFFFFFF) return set_error(FLB_EINVAL, "call must be < 256");
  launch_philox(site_dev, n, step, call, tag, stream, seed, fp32, words_out_dev, normals_out_dev,
                static_cast<cudaStream_t>(cuda_stream));
  return cuda_check(cudaGetLastError(), "flb_philox launch");
}

}  // extern "C"
