// Internal definitions shared by the CUDA translation units of libflb.
// Device code for sm_103a; host code plain C++17.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/flb.h"

namespace flb {

constexpr int kMaxFields = FLB_MAX_FIELDS;
constexpr int kMaxPairs = kMaxFields * (kMaxFields + 1) / 2;
constexpr int kStepThreads = 256;     // threads per block of the step kernels
constexpr int kReduceBlocks = 2048;   // partial sums of the deterministic reductions
constexpr int kMlpHidden = 32;
constexpr int kMlpOut = 6;
constexpr int kMlpWeights = kMlpHidden * 3 + kMlpHidden * kMlpHidden + kMlpOut * kMlpHidden;  // 1312
constexpr int kMlpBiases = kMlpHidden + kMlpHidden + kMlpOut;                               // 70

constexpr int kMaxQ = 20;                    // moments per site (D3Q19: 19)
constexpr int kFeqW = 24, kFeqStride = 48;   // per replica: f^0_i(rho0, u0) at [i], w_i rho0 at [kFeqW + i]
constexpr int kCoRho0 = 0, kCoU0x = 1, kCoU0y = 2, kCoU0z = 3;
constexpr int kCoInvTau = 4, kCoAmp = kCoInvTau + kMaxQ, kCoMref = kCoAmp + kMaxQ;
constexpr int kCoNoiseR = kCoMref + kMaxQ;   // 6 x 6 correlated-noise root (noise_mode 1), row-major
constexpr int kNumCoef = kCoNoiseR + 36;

// Per-replica description, resident in device memory (one array per context).
// Offsets are byte offsets from the workspace base.
struct ReplicaDesc {
  int32_t nx, ny, log2nx, log2ny;
  int32_t nz;                   // 3D depth (1 otherwise); a row is (y, z), row = z ny + y
  int32_t q;
  int32_t units_per_row;        // nx / VEC of the step launch
  uint32_t upr_magic;           // row of a unit u < 2^31: (u * upr_magic) >> upr_shift
  int32_t upr_shift;            //   (Granlund & Montgomery, PLDI'94, round-up multiplier)
  int64_t n_units;              // units_per_row * ny * nz
  int64_t block_begin;          // first virtual block of this replica in the step launch
  uint32_t seed_lo, seed_hi, stream, noise_mask;
  uint32_t rkey[20];            // Philox round keys (k0 + r W0, k1 + r W1), r = 0..9, of the key (seed_lo, seed_hi)
  int32_t noise_mode;           // 0: independent noise (Eq. 8); 1: correlated (root in kCoNoiseR)
  uint32_t field_mask, n_fields;
  int32_t field_id[kMaxFields];     // slot -> field id
  int32_t n_pairs;
  int32_t pair_a[kMaxPairs], pair_b[kMaxPairs];   // slot indices, a <= b
  int64_t pair_off[kMaxPairs];      // byte offset of the pair's accumulator plane
  double rho0, kT, mu, u0x, u0y, u0z;
  double inv_tau[kMaxQ];
  double amp[kMaxQ];                // (1/tau) sqrt(mu rho0 (2 tau - 1)), 0 when masked
  double mref[kMaxQ];               // reference value subtracted from each field id
  int64_t off_pop[2];               // population buffers (ping-pong)
  int64_t off_fields;               // [n_fields][nz][ny][nx] Real
  int64_t off_spec;                 // [n_fields][ny][wpitch] complex Real (row-transformed)
  int64_t spec_slot;                // bytes from spectrum slot 0 to slot 1 (two samples folded
                                    // into one accumulation pass; 0: one slot)
  int32_t spec_tiled;               // spectrum layout: 0 = [n_fields][ny][wpitch]; 1 = column tiles
                                    // [n_fields][ceil(half_nx / 16)][ny][16] (kSpecTile)
  int64_t off_mean0;                // [n_fields] double: sum over samples of X(k=0)
  int64_t off_tw_x, off_tw_y;       // twiddles exp(-2 pi i m / n), m < n/2, complex Real
  int32_t half_nx;                  // nx / 2 + 1
  int32_t wpitch;                   // pitch (complex elements) of spec rows
  int32_t log2n1;                   // column FFT split ny = N1 * N2 (0: one pass of length ny)
  int64_t off_tc_ring, off_tc_sums; // time correlators: offsets in the TimeCorr buffer (see TimeCorr)
  int64_t off_tc_part;              // 3D lattices: per-block partial transforms [blocks][F][n_k] double2
  int64_t off_tc_tab;               // 3D lattices: phase tables of the direct transforms (lb_3d.cu)
  int32_t acc_ncol;                 // pair-sum layout: 0 = [ky][kx]; c > 0 = blocked in the order
                                    // the column pass produces the points: [k1][kx / c][k2][kx % c]
                                    // (ky = k1 + N1 k2; kx padded to a multiple of c)
  // the per-replica coefficients in the arithmetic type of the path (host-filled),
  // so the FP32 kernels never convert from FP64: [kCoRho0], [kCoU0x .. kCoU0z],
  // [kCoInvTau + a], [kCoAmp + a], [kCoMref + field], [kCoNoiseR + 6 c + c'] (c, c' index
  // the non-conserved moments 3..8)
  float fco[kNumCoef];
  double dco[kNumCoef];
};

template <typename R> __device__ __forceinline__ R coef(const ReplicaDesc& d, int i);
template <> __device__ __forceinline__ float coef<float>(const ReplicaDesc& d, int i) { return d.fco[i]; }
template <> __device__ __forceinline__ double coef<double>(const ReplicaDesc& d, int i) { return d.dco[i]; }

struct DevStatus {
  int32_t error;        // 0 ok; FLB_EUNSTABLE / FLB_ETIMEOUT set by kernels
  int32_t replica;      // first replica that raised it
  uint64_t n_samples;   // samples accumulated
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 128-bit counter, 64-bit key.
__host__ __device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                                      uint32_t& c3, uint32_t k0, uint32_t k1) {
  // 32 x 32 -> 64-bit products: one wide multiply gives both halves
  const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c0, c1, c2, c3, k0, k1);
    k0 += W0; k1 += W1;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The same with the round keys precomputed (rk[2r], rk[2r + 1] = the keys of round r), so
// that a kernel reading them from its constant bank spends no instruction on the schedule.
__host__ __device__ __forceinline__ uint4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                           const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, rk[2 * r], rk[2 * r + 1]);
  return make_uint4(c0, c1, c2, c3);
}

// The hardware approximations (single MUFU operations, inputs flushed to zero below the
// normal range, which these inputs never reach): log2 (absolute error <= 2^-22 on
// [1/2, 2]), reciprocal square root (relative error <= 2^-22.9), sine and cosine (absolute
// error <= 2^-20.9 on [-pi, pi]).
__device__ __forceinline__ float lg2_approx(float x) { float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rsqrt_approx(float x) { float y; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sin_approx(float x) { float y; asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float cos_approx(float x) { float y; asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

// Box-Muller on a word pair: N0 = r cos(2 pi ub), N1 = r sin(2 pi ub), r = sqrt(-2 ln ua).
// FP64: u = (w + 1/2) 2^-32 (exact).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& n0, double& n1) {
  const double ua = ((double)wa + 0.5) * 0x1p-32;
  const double ub = ((double)wb + 0.5) * 0x1p-32;
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  n0 = r * c; n1 = r * s;
}

// FP32: ua = RN(wa) 2^-32 + 2^-33 (relative error <= 2^-24 for every ua, small ua
// included, where the log is sensitive; ua rounds up to 1 only where r is ~1e-4 anyway);
// 2 ln ua = log2(ua) * 2 ln 2 with the hardware log2, so r is within a few ulp for typical
// ua and within ~7e-4 absolute in the worst case (ua within 1e-7 of 1, r below ~5e-4).
// -r = y / sqrt(-y), y = 2 ln ua <= 0 (clamped below 0).  The angle theta =
// 2 pi (ub - 1/2) in [-pi, pi], the range of the hardware sine and cosine, is one
// multiply-add of RN(wb); (cos, sin)(2 pi ub) = -(cos, sin)(theta), and the two signs
// cancel: N = (-r) (cos, sin)(theta).
constexpr float kBmLn4 = 1.38629436111989061883f;                  // 2 ln 2
constexpr float kBmAngScale = (float)(6.283185307179586476925 / 4294967296.0);
constexpr float kBmAngShift = (float)(6.283185307179586476925 * (1.0 / 8589934592.0 - 0.5));
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const float ua = fmaf(__uint2float_rn(wa), 0x1p-32f, 0x1p-33f);
  const float y = fminf(lg2_approx(ua) * kBmLn4, -1e-30f);
  const float nr = y * rsqrt_approx(-y);
  const float th = fmaf(__uint2float_rn(wb), kBmAngScale, kBmAngShift);
  n0 = nr * cos_approx(th);
  n1 = nr * sin_approx(th);
}

template <typename T> struct cplx { T x, y; };
template <typename T> struct vec2_of;
template <> struct vec2_of<float> { using type = float2; };
template <> struct vec2_of<double> { using type = double2; };

// Time correlators at selected wave vectors (caller-owned device buffer; base = nullptr
// when off).  Per replica r with F sampled fields: the last n_lags samples of X_f(k_j)
// in a ring [n_lags][F][n_k] (double2) at base + off_tc_ring, slot = sample % n_lags, and
// the sums of X_a(k, s) X_b(k, s - tau)^* at base + off_tc_sums, [n_lags][F][F][n_k].
struct TimeCorr {
  char* base = nullptr;
  int n_lags = 0, n_k = 0;
  const int32_t* kx = nullptr;      // [n_k], 0 <= kx <= nx/2
  const int32_t* ky = nullptr;      // [n_k], 0 <= ky < ny
  const int32_t* kz = nullptr;      // [n_k], 0 <= kz < nz (3D lattices; 0 otherwise)
  const int32_t* kxi = nullptr;     // 3D: [n_k] index of kx[j] in kxl
  const int32_t* kxl = nullptr;     // 3D: [n_kx] the distinct kx values
  int n_kx = 0;
  uint64_t* count = nullptr;        // [n_replicas]: samples written so far
  int part_blocks = 0;              // 3D lattices: blocks of the direct transform (partials per replica)
};

// Arguments of one step launch (lb_step.cu).
struct StepLaunch {
  const ReplicaDesc* descs; const int64_t* vb_begin; int n_reps; int64_t n_vblocks;
  char* ws; int parity; uint32_t step; const void* mlp; int grid; int block;
  const uint64_t* step_dev = nullptr;   // non-NULL (graph replay): step = *step_dev + step
  DevStatus* status = nullptr;          // where a kernel reports a bounded wait that gave up
  int sms = 0;                          // multiprocessors of the device
  const ReplicaDesc* desc0 = nullptr;   // host copy of descs[0] (kernel argument of one-replica launches)
  bool noise_general = false;           // some replica uses noise mode 1 or 2
  int net_engine = FLB_NET_WARP;        // direct D2Q9 kernels with the network: FLB_NET_WARP or FLB_NET_TCGEN05
  // kernel flavour: 0 = one replica, noise mode 0; 1 = one replica, any mode; 2 = batched
  int flavor() const { return n_reps > 1 ? 2 : (noise_general ? 1 : 0); }
};
// flavour -> (descriptor in the constant bank, noise modes 1/2 compiled)
template <int FL> struct Flavor { static constexpr bool kOne = FL != 2, kGen = FL != 0; };

// Shared-memory budget of the column transforms and their split rule: one pass of
// length ny when F columns of 4 fit the budget, else ny = N1 * N2 with
// N1 = 2^floor(log2(ny)/2) (four-step).
constexpr int kColsSmemBudget = 200 * 1024;
constexpr int kRowsBlockMax = 1024;      // threads of a row-FFT block (at most nx / 2)
constexpr int kColsBlock = 256;
#ifndef FLB_COLS_MAX
#define FLB_COLS_MAX 16
#endif
constexpr int kColsMax = FLB_COLS_MAX;   // widest column tile (halved until it fits the budget)
// B of the register-resident FP32 column pass (spectra_cols.cu) for a column of length
// len = 16 B, B = 1, 2, 4, 8, 16; 0 if there is none (the shared-memory pass of spectra.cu).
// The launches take a mask of the passes they need: bit B for each B, kColsGeneric for
// the shared-memory pass.
__host__ __device__ __forceinline__ int cols16_b(int len) {
  return (len >= 16 && len <= 256 && (len & (len - 1)) == 0) ? len >> 4 : 0;
}
constexpr int kColsGeneric = 32;
// The FP32 row pass of spectra_rows.cu (one real row per block, Stockham radix-16) for
// nx = 4096 .. 32768; the shared-memory radix-2 pass of spectra.cu (two rows per block)
// otherwise.  Virtual blocks of the row pass of a replica:
__host__ __device__ __forceinline__ bool rows16_nx(int nx) {
  return nx >= 4096 && nx <= 32768 && (nx & (nx - 1)) == 0;
}
inline bool rows16(int precision, int nx) { return precision != FLB_FP64 && rows16_nx(nx); }
inline int64_t rows_blocks(int precision, int nx, int n_fields, int ny) {
  return rows16(precision, nx) ? (int64_t)n_fields * ny : ((int64_t)n_fields * ny + 1) / 2;
}
// The register-resident pass-2a kernel takes tiles of kColsA16 columns of one field
// (pass 2a needs no field pairs); the shared-memory kernel tiles of the layout's ncol
// columns of all fields.  Virtual blocks of pass 2a of a replica:
constexpr int kColsA16 = 16;
// Column-tiled spectrum (ReplicaDesc::spec_tiled): the row transforms of a field are
// stored in tiles of kSpecTile columns, each tile [ny][kSpecTile], so that a column pass
// reading the rows of a tile reads one contiguous slab instead of 128-byte pieces of
// rows a whole row apart.  Used when every pass of the replica runs on the
// register-resident / Stockham kernels (FP32 rows of 4096 .. 32768, columns of 16 ..
// 256); the shared-memory kernels keep the row-major layout.
constexpr int kSpecTile = 16;
static_assert(kColsA16 == kSpecTile, "a pass-2a tile is one spectrum tile");
// element (f, y, kx) of a spectrum slot, the distance between rows y, y + 1, and the
// complex elements of a slot
__host__ __device__ __forceinline__ int64_t spec_index(const ReplicaDesc& d, int f, int y, int kx) {
  if (d.spec_tiled) {
    const int nt = (d.half_nx + kSpecTile - 1) / kSpecTile;
    return (((int64_t)f * nt + kx / kSpecTile) * d.ny + y) * kSpecTile + kx % kSpecTile;
  }
  return ((int64_t)f * d.ny + y) * d.wpitch + kx;
}
__host__ __device__ __forceinline__ int spec_row_stride(const ReplicaDesc& d) {
  return d.spec_tiled ? kSpecTile : d.wpitch;
}
inline bool spec_tiled_ok(int precision, int nx, int ny, int log2n1) {
  return rows16(precision, nx) && cols16_b(ny >> log2n1) && (log2n1 == 0 || cols16_b(1 << log2n1));
}
__host__ __device__ __forceinline__ int64_t spec_elems(const ReplicaDesc& d) {
  if (d.spec_tiled) return (int64_t)d.n_fields * ((d.half_nx + kSpecTile - 1) / kSpecTile) * d.ny * kSpecTile;
  return (int64_t)d.n_fields * d.ny * d.wpitch;
}
// shared memory of the register-resident pass 2b: nslots samples' tiles of F fields x
// ncol columns of length L (rows padded to L + 1) and a table of L roots of unity
inline int fft_cols16_smem(int F, int L, int ncol, int nslots) {
  return (nslots * F * ncol * (L + 1) + L) * 8;
}
constexpr int kFoldSmemBudget = 56 * 1024;   // four blocks per SM
inline int64_t cols_a_blocks(int precision, int log2n1, int n_fields, int half_nx, int ny, int ncol) {
  if (!log2n1) return 0;
  const bool reg = precision != FLB_FP64 && cols16_b(1 << log2n1);
  const int w = reg ? kColsA16 : ncol;
  return (int64_t)((half_nx + w - 1) / w) * (ny >> log2n1) * (reg ? n_fields : 1);
}
inline int column_split(int precision, int F, int ny) {
  const int cs = precision == FLB_FP64 ? 16 : 8;
  if ((int64_t)F * (ny + 1) * 4 * cs <= kColsSmemBudget) return 0;
  int l = 0;
  while ((1 << l) < ny) ++l;
  return l / 2;
}

// host-side helpers (api.cu)
int set_error(int code, const char* fmt, ...);

// ---------------------------------------------------------------------------
// Bounds-checked debug build (compiled with -DFLB_CHECK_BOUNDS, python -m
// paper_1010_1233_gb300.build --checked): at every global and shared-memory access
// whose index the kernels compute, FLB_INB(condition, site) checks the index against
// its array; a violation is counted, the first violating site's code is kept, and the
// access is skipped (no trap, no fault).  Each translation unit has its own counters
// (the library is compiled without relocatable device code); they register a reader
// with api.cu, and flb_debug_bounds adds them up.  In the normal build FLB_INB is the
// constant true and costs nothing.
using OobRead = int (*)(unsigned int* out2);
using OobClear = int (*)();
bool register_oob_counter(OobRead read, OobClear clear);

#ifdef FLB_CHECK_BOUNDS
static __device__ unsigned int g_flb_oob[2];          // violations, first site code
__device__ __forceinline__ bool flb_inb(bool ok, int site) {
  if (!ok) {
    atomicAdd(&g_flb_oob[0], 1u);
    atomicCAS(&g_flb_oob[1], 0u, (unsigned int)site);
  }
  return ok;
}
static int flb_oob_read(unsigned int* out2) { return (int)cudaMemcpyFromSymbol(out2, g_flb_oob, sizeof(g_flb_oob)); }
static int flb_oob_clear() {
  const unsigned int z[2] = {0u, 0u};
  return (int)cudaMemcpyToSymbol(g_flb_oob, z, sizeof(z));
}
static const bool flb_oob_registered = register_oob_counter(flb_oob_read, flb_oob_clear);
#define FLB_INB(cond, site) flb_inb((cond), (site))
#else
#define FLB_INB(cond, site) true
#endif

}  // namespace flb
