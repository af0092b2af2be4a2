/*
 * flb.h -- C ABI of the GB300 fluctuating lattice Boltzmann library (libflb.so).
 *
 * The method (Kaehler & Wagner, "Cross Correlators and Galilean Invariance in
 * Fluctuating Ideal Gas Lattice Boltzmann Simulations"): the lattice Boltzmann
 * equation with a diagonal collision in the Hermite-orthonormal moment basis
 * (Eqs. 1, 3-5), Gaussian noise with the fluctuation-dissipation amplitude of
 * Eq. 8 on every non-conserved moment (stress and ghost moments, Sec. 2), and
 * the equal-time structure factors and cross correlators of Eqs. 11-12.
 *
 * Conventions for every entry point:
 *   - Return value: FLB_OK (0) or a negative FLB_E* code; flb_last_error()
 *     returns a thread-local message describing the last failure.  No C++
 *     exception crosses this boundary.
 *   - Device memory is owned by the caller (a single workspace block, sized by
 *     flb_workspace_bytes); the library never calls cudaMalloc.  The opaque
 *     flb_ctx is host memory owned by the library (flb_destroy frees it).
 *   - Work is issued on the caller's CUDA stream and is stream-ordered;
 *     asynchronous kernel errors surface at the next flb_sync / flb_get_*.
 *   - An invalid argument returns FLB_EINVAL before any work is issued and
 *     leaves the context unchanged.
 *   - Host arrays are plain FP64 in C order; a lattice field is [ny][nx]
 *     (x fastest), populations are [q][ny][nx].
 */
#ifndef FLB_H
#define FLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FLB_OK         0
#define FLB_EINVAL    (-1)  /* invalid argument or unsupported configuration */
#define FLB_ENOMEM    (-2)  /* workspace smaller than flb_workspace_bytes     */
#define FLB_ECUDA     (-3)  /* CUDA launch or runtime error                   */
#define FLB_EUNSTABLE (-4)  /* non-finite state detected                      */
#define FLB_ETIMEOUT  (-5)  /* a bounded device wait gave up                  */
#define FLB_ESTATE    (-6)  /* call not valid in the context's current state  */

/* ---- lattices and storage precisions --------------------------------- */
#define FLB_D1Q3 1          /* v = (0, +1, -1); moments rho, sqrt3 j, (3v^2-1)/sqrt2 */
#define FLB_D2Q9 2          /* Sec. 3 velocity set and the moment matrix of Eq. 9   */
#define FLB_D3Q15 3         /* tested in Sec. 3, tables not printed: standard D3Q15
                               velocities and weights (2/9, 1/9, 1/72) and the
                               orthonormal basis (Eq. 4) obtained by Gram-Schmidt of
                               1, vx, vy, vz, vx^2 - vy^2, vx^2 + vy^2 - 2 vz^2,
                               vx vy, vy vz, vz vx, v^2, vx v^2, vy v^2, vz v^2,
                               vx vy vz, v^4 (moments 0-3 conserved, 4-8 shear,
                               9 bulk, 10-14 ghosts).  Velocity order: rest,
                               +x, -x, +y, -y, +z, -z, (1,1,1), (-1,-1,-1),
                               (1,1,-1), (-1,-1,1), (1,-1,1), (-1,1,-1), (-1,1,1),
                               (1,-1,-1).  Noise normals 0..10 (Philox calls 0..2)
                               drive moments 4..14.                                  */
#define FLB_D3Q19 4         /* the other standard 3D lattice (not in the paper): rest,
                               +-x, +-y, +-z, then the edges (1,1,0), (-1,-1,0),
                               (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1),
                               (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1);
                               weights 1/3, 1/18, 1/36; Gram-Schmidt basis (Eq. 4
                               norm) of the D3Q15 list up to v^2, then vx v^2, vy v^2,
                               vz v^2, vx (vy^2 - vz^2), vy (vz^2 - vx^2),
                               vz (vx^2 - vy^2), v^4, (vx^2 - vy^2) v^2,
                               (vx^2 + vy^2 - 2 vz^2) v^2 (moments 0-3 conserved, 4-8
                               shear, 9 bulk, 10-18 ghosts).  Noise normals 0..14
                               (Philox calls 0..3) drive moments 4..18.              */
#define FLB_FP64     0      /* full f_i in FP64, all arithmetic FP64                 */
#define FLB_FP32_DEV 1      /* f_i - w_i rho0 stored and processed in FP32;
                               correlators accumulated in FP64                      */

/* ---- sampled fields (bit f of flb_replica.field_mask) -----------------
 * f = 0..q-1 : moment M^a - M^{a,0}(rho0, u0)   (M^0 = rho, M^1,2 = sqrt3 j)
 * f = 9, 10  : u_x - u0_x, u_y - u0_y           (u = j / rho; D1Q3, D2Q9)
 * Fields are taken from the pre-collision (post-streaming) state.  The 3D
 * lattices (D3Q15, D3Q19) sample moments only (f < q, at most FLB_MAX_FIELDS
 * of them) and accumulate correlators at chosen wave vectors
 * (flb_set_time_correlator3), not on the full FFT grid.                    */
#define FLB_FIELD_UX 9
#define FLB_FIELD_UY 10
#define FLB_MAX_FIELDS 11

/* One independent periodic lattice (a replica).  Several replicas with the
 * same lattice type and precision can run in one context (batched launch). */
typedef struct {
  int32_t  lattice;     /* FLB_D1Q3, FLB_D2Q9, FLB_D3Q15 or FLB_D3Q19            */
  int32_t  nx, ny;      /* lattice size; ny = 1 for D1Q3.  nx even.  Sampling
                           needs powers of two: 2 <= nx <= 16384, ny <= 16384  */
  double   tau[20];     /* relaxation time per moment a (Eq. 5), a < q; entries of
                           the conserved moments are ignored, the others must be
                           > 1/2                                                 */
  double   rho0;        /* mean density rho-bar (> 0)                            */
  double   kT;          /* temperature; mu = 3 kT scales the noise of Eq. 8      */
  double   u0[3];       /* mean velocity of the initial state (u0[2]: 3D only)   */
  uint64_t seed;        /* Philox key                                            */
  uint32_t stream;      /* Philox counter word 3 (replica stream id)             */
  uint32_t noise_mask;  /* bit a = noise on moment a; bits of conserved moments
                           must be 0.  All non-conserved bits = the scheme of
                           Sec. 2; D2Q9 without bits 6..8 = the Ladd scheme    */
  uint32_t init_mode;   /* 0: f^0(rho0, u0) on every site; 1: thermal (moment
                           fluctuations N(0, mu rho0), mean of rho and j removed) */
  uint32_t field_mask;  /* fields to sample (see above); 0 = no sampling         */
  uint32_t noise_mode;  /* 0: independent noise per non-conserved moment (Eq. 8).
                           1: correlated noise for a fluid moving at u0 (the
                           extension the paper points to after Eq. 7): the
                           noise covariance of Eq. 6 with the moment covariance
                           mu sum_i m_i^a m_i^b f^0_i(rho0, u0) of Eq. 7 on the
                           masked non-conserved moments; xi = R N with R the
                           principal square root of its positive part (computed
                           once per replica on the host).  At u0 = 0 it equals
                           mode 0.
                           2: Eq. 8 with the local density rho(x) of the site in
                           place of rho-bar (the amplitude times sqrt(rho/rho0)).
                           D3Q15, D3Q19: mode 0 only                            */
  int32_t  nz;          /* D3Q15, D3Q19: lattice depth (>= 1); 0 or 1 otherwise.  The
                           populations are [q][nz][ny][nx], site index
                           (z ny + y) nx + x                                    */
} flb_replica;

typedef struct flb_ctx flb_ctx;

/* Bytes of device workspace a context needs (alignment 256 B).
 * precision: FLB_FP64 / FLB_FP32_DEV.  reps: n_replicas host descriptors. */
int flb_workspace_bytes(int precision, const flb_replica* reps, int n_replicas,
                        size_t* bytes_out);

/* Create a context on the current CUDA device.  dev_workspace: caller-owned
 * device memory of at least flb_workspace_bytes bytes, 256-B aligned, kept
 * alive until flb_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default).
 * Initialises every replica's populations (init_mode) and zeroes the
 * correlator sums; global step counter = 0. */
int flb_create(int precision, const flb_replica* reps, int n_replicas,
               void* dev_workspace, size_t workspace_bytes, void* cuda_stream,
               flb_ctx** out);

/* Advance every replica by n_steps (Eq. 1 with the collision of Eq. 5 and the
 * noise of Eq. 8).  A step whose global index t satisfies sample_every != 0 and
 * t % sample_every == 0 first samples the fields of its pre-collision state and
 * adds X_a(k) X_b(k)^* of every field pair to FP64 sums (Eqs. 11-12).
 * Asynchronous: returns after issuing the work. */
int flb_run(flb_ctx* ctx, uint64_t n_steps, uint32_t sample_every);

/* Wait for the context's stream and report any asynchronous error, including a
 * non-finite state detected by the conservation check (FLB_EUNSTABLE). */
int flb_sync(flb_ctx* ctx);

/* Zero the correlator sums, the k = 0 means and the sample count. */
int flb_reset_stats(flb_ctx* ctx);

/* Normalised correlator C_ab(k) = N^ab (<X_a(k) X_b(k)^*> - delta_k0 <X_a(0)><X_b(0)>^*)
 * on the full grid: host_out[(ky*nx + kx)*2 + {0,1}] = {Re, Im}, with
 * k = 2 pi (kx/nx, ky/ny).  N^ab = 1/(V sqrt(var_a var_b)), var = mu rho0 for a
 * moment field, kT/rho0 for a velocity field (both fields must be sampled).
 * n_samples (may be NULL) receives the number of samples.  D1Q3 and D2Q9 only: the
 * 3D lattices accumulate correlators at chosen wave vectors (flb_set_time_correlator3,
 * flb_get_time_correlator; FLB_EINVAL here).  Synchronises. */
int flb_get_correlator(flb_ctx* ctx, int replica, int field_a, int field_b,
                       double* host_out, uint64_t* n_samples);

/* Copy the stored (post-collision) populations f_i of a replica to / from host
 * FP64 [q][ny][nx] ([q][nz][ny][nx] on the 3D lattices).  For FLB_FP32_DEV they
 * are converted from / to f - w rho0 in FP32.  Synchronises. */
int flb_get_populations(flb_ctx* ctx, int replica, double* host_out);
int flb_set_populations(flb_ctx* ctx, int replica, const double* host_in);

/* Copy the populations of a rectangular window [x0, x0+w) x [y0, y0+h) of a replica
 * (no wrap-around: the window must lie inside the lattice) to host FP64 [q][h][w].
 * For sampling outputs of large lattices without copying the whole state.  D1Q3 and
 * D2Q9 only (FLB_EINVAL on the 3D lattices).  Synchronises. */
int flb_get_populations_window(flb_ctx* ctx, int replica, int x0, int y0, int w, int h,
                               double* host_out);

/* The fields of the most recent sample of a replica (Eq. 11 inputs, before the
 * transform): host FP64 [n_fields][ny][nx] ([n_fields][nz][ny][nx] on the 3D
 * lattices), fields in increasing id order.
 * FLB_ESTATE before the first sample.  Synchronises. */
int flb_get_fields(flb_ctx* ctx, int replica, double* host_out);

/* FP64 sums over the lattice of rho, j_x, j_y, j_z (zero for the components
 * a lattice does not have) of the stored state; out[4].  Synchronises. */
int flb_get_conserved(flb_ctx* ctx, int replica, double* out4);

/* Global step counter (number of steps taken). */
int flb_get_step(flb_ctx* ctx, uint64_t* step_out);

/* Noise-scale network (learned extension, not in the paper): D2Q9 only.
 * s_a = 1 + o_a(u_x, u_y, rho - rho0) multiplies the Eq. 8 amplitude of moment
 * a = 3..8, o = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with W1 32x3, W2 32x32,
 * W3 6x32 (row-major, bfloat16 bit patterns, 96 + 1024 + 192 values in that
 * order) and biases b1(32) b2(32) b3(6) given in FP32.  Evaluated on the tensor
 * cores (flb_set_network_engine) with bfloat16 operands and FP32 accumulation:
 * the inputs, the biases and the hidden activations are rounded to bfloat16.  FP32 D2Q9 path only.  enable = 0 switches it off (s = 1,
 * bit-identical to the plain method).  Copies the weights. */
int flb_set_mlp(flb_ctx* ctx, const uint16_t* w_bf16, const float* biases, int enable);

/* Checkpoint: the state is the populations, the step counter and the
 * correlator sums.  flb_save with host_buf = NULL reports the size.  Both
 * calls return when the copies are complete (host_buf: host memory, pinned
 * for full copy speed; the copies run as 64 MiB pieces on four streams). */
int flb_save(flb_ctx* ctx, void* host_buf, size_t* bytes_inout);
int flb_load(flb_ctx* ctx, const void* host_buf, size_t bytes);

/* Time correlators at selected wave vectors (an extension: the paper's correlators
 * are equal-time ones, Sec. 3, Eqs. 11-12):
 *   F_ab(k, tau) = N^ab (1/n_tau) sum_s X_a(k, s) X_b(k, s - tau)^*
 * over the samples s taken by flb_run (every sample_every steps), lags
 * tau = 0 .. n_lags-1 in samples, n_tau = n_samples - tau, every ordered pair of
 * the sampled fields, with the normalisation N^ab of flb_get_correlator (so
 * F_ab(k, 0) = C_ab(k)).  The same n_k wave vectors for every replica: 0 <= kx_j
 * <= nx/2, 0 <= ky_j < ny, k != 0; every replica must sample fields.
 * flb_time_correlator_bytes: size of the caller-owned device buffer.
 * flb_set_time_correlator: buf_dev 256-B aligned, at least that size, kept alive
 * while enabled; zeroes the time-correlator sums (flb_reset_stats does too);
 * n_lags = 0 switches them off.  Synchronises; captured graphs are dropped.
 * flb_get_time_correlator: host_out [n_lags][n_k] complex (re, im), NaN for lags
 * without a pair of samples; n_samples (may be NULL) the samples taken.  The
 * time-correlator state is not part of flb_save checkpoints. */
int flb_time_correlator_bytes(flb_ctx* ctx, int n_lags, int n_k, size_t* bytes_out);
int flb_set_time_correlator(flb_ctx* ctx, int n_lags, int n_k, const int32_t* kx, const int32_t* ky,
                            void* buf_dev, size_t bytes);
/* Same with a third component kz (0 <= kz < nz) for D3Q15 / D3Q19, whose transforms are
 * direct sums over the lattice at the chosen wave vectors (no FFT grid); for
 * D1Q3 / D2Q9 kz must be 0.  With n_lags = 1 these are the equal-time correlators
 * C_ab(k) of Eqs. 11-12. */
int flb_set_time_correlator3(flb_ctx* ctx, int n_lags, int n_k, const int32_t* kx, const int32_t* ky,
                             const int32_t* kz, void* buf_dev, size_t bytes);
int flb_get_time_correlator(flb_ctx* ctx, int replica, int field_a, int field_b, double* host_out,
                            uint64_t* n_samples);

/* Launch configuration of the step kernel.  staged = 0: direct kernels, vec
 * consecutive sites per thread (1, 2 or 4; > 1 only on the FP32 D2Q9 path,
 * every nx a multiple of vec), grid_blocks persistent blocks (0 = 16 per SM).
 * staged = 1 (FP32 D2Q9 path, every nx a multiple of 4): row tiles of 256 vec
 * sites staged through shared memory by TMA bulk copies, one persistent block
 * per resident slot (grid_blocks caps it).  Results agree to rounding across
 * configurations (kernels may contract multiply-adds differently).
 * Synchronises. */
int flb_set_step_config(flb_ctx* ctx, int vec, int grid_blocks, int staged);
int flb_get_step_config(flb_ctx* ctx, int* vec, int* grid_blocks, int* staged);

/* How the direct D2Q9 step kernels (staged = 0) evaluate the noise-scale
 * network (flb_set_mlp); the arithmetic is the same (bfloat16 operands, FP32
 * accumulation), results agree to the rounding of the accumulation order.
 * FLB_NET_WARP (default): each warp runs the three layers for 64 sites with
 * warp-level tensor-core MMAs (m16n8k16), all operands in registers, no
 * barrier between warps.  FLB_NET_TCGEN05: each warpgroup runs them for 128
 * sites per tile with tcgen05 MMAs, operand A and the accumulators in tensor
 * memory, warpgroup barriers between the layers.  The staged kernel always
 * uses the tcgen05 form.  flb_autotune tries both.  Synchronises. */
#define FLB_NET_WARP    0
#define FLB_NET_TCGEN05 1
int flb_set_network_engine(flb_ctx* ctx, int engine);
int flb_get_network_engine(flb_ctx* ctx, int* engine);

/* Linear stability of one replica's parameters, on the host (no GPU, no context):
 * the largest modulus of the eigenvalues of the one-step operator A_k = P_k J of the
 * noise-free dynamics linearised about f^0(rho0, u0) (P_k the pull-streaming phases of
 * Eq. 1, J the Jacobian of the collision of Eq. 5 with the equilibrium of Eq. 2), over
 * the wave vectors k = 2 pi j / N, N = min(n, max_k) per lattice dimension, k = 0
 * included (where the conserved moments give exactly 1).  A radius above 1 (beyond
 * rounding) means some fluctuation grows every step: the run will diverge.  Spectral
 * radius by Gelfand's formula (2^40-th power by normalised squaring).  radius_out: the
 * maximum; k_out[3] (may be NULL): its (jx, jy, jz).  Validates the replica as
 * flb_workspace_bytes does. */
int flb_stability(const flb_replica* rep, int max_k, double* radius_out, int32_t* k_out);

/* Autotuner: times `trials` launches of the step kernel (current network
 * setting, no sampling) for every valid configuration: direct kernels with
 * every vec and grid size in {2,4,8,16} x SMs and all-blocks (with the network
 * on: with each network engine), and the staged kernel with every vec; keeps
 * the fastest, engine included, and reports it (ms_out: time per launch).  The timing launches recompute the next step from the current state
 * without advancing it, so the simulation is unchanged.  Synchronises. */
int flb_autotune(flb_ctx* ctx, int trials, int* vec_out, int* grid_out, int* staged_out, double* ms_out);

/* CUDA graphs (default on): flb_run replays a captured graph for every aligned
 * chunk of whole sampling periods (at least 32 steps; 32 steps without
 * sampling), which removes the per-kernel launch cost on small lattices.  D1Q3
 * contexts (without time correlators) instead run up to 4096 steps and their
 * samples per launch of one fused kernel, one block per replica with its state
 * in shared memory.  Results are identical to direct launches up to the
 * contraction of multiply-adds.  The captured graphs are dropped when the
 * launch configuration or the network switch changes.  enable = 0 issues every
 * kernel of every step directly. */
int flb_set_graphs(flb_ctx* ctx, int enable);

/* Kernels flb_run has issued on this context so far (a library bookkeeping value,
 * no counterpart in the paper): every kernel launched directly, and for a
 * replayed CUDA graph the kernels captured in it.  count: host uint64_t. */
int flb_kernel_launches(flb_ctx* ctx, uint64_t* count);

/* Failure-detection check: launches on the context's stream one bounded
 * mbarrier wait that nothing completes (the wait the network step kernels use
 * for their MMAs and copies, here limited to limit_clocks SM clocks, 1 .. 2^32)
 * and records its timeout in the context's status word, as a step kernel whose
 * MMA never completed would.  The next synchronising call (flb_sync) returns
 * FLB_ETIMEOUT; the status stays set for the life of the context.  No
 * asynchronous operation is left in flight and the device stays usable.
 * FLB_EINVAL for a limit out of range.  Asynchronous. */
int flb_probe_wait_timeout(flb_ctx* ctx, uint64_t limit_clocks);

/* Bounds-checked debug build only (built with python -m paper_1010_1233_gb300.build
 * --checked, which compiles every kernel with -DFLB_CHECK_BOUNDS): every global and
 * shared-memory index the step, sampling and 3D kernels compute is checked against its
 * array, and a violating access is counted and skipped (no trap).  Synchronises the
 * device, then returns in *violations the count since the last clear and in *first_site
 * the code of the first violating site (0: none; the codes are listed with FLB_INB in
 * the sources).  clear != 0 resets the counters.  FLB_ESTATE from a library built
 * without the checks. */
int flb_debug_bounds(uint64_t* violations, uint32_t* first_site, int clear);

/* Destroy the context (does not free the caller's workspace). */
void flb_destroy(flb_ctx* ctx);

/* Message of the last error on this thread ("" if none). */
const char* flb_last_error(void);

/* ---- device-pointer entry points (diagnostics and training) ----------- */

/* Philox4x32-10 words and unit normals exactly as the step kernels draw them.
 * For i < n: counter = (site[i], step, call | tag << 8, stream), key = seed.
 * words_out: device uint32[4*n] (may be NULL); normals_out: device double[n*2*...]:
 * if normals_out != NULL it receives, per i, the 2 Box-Muller normals of the
 * pair (w0, w1) and (w2, w3) of that call: 4 doubles, in FP64 (fp32 = 0) or in
 * the FP32 recipe (fp32 = 1, stored as double).  site: device uint32[n]. */
int flb_philox(const uint32_t* site_dev, int n, uint32_t step, uint32_t call, uint32_t tag,
               uint32_t stream, uint64_t seed, int fp32, uint32_t* words_out_dev,
               double* normals_out_dev, void* cuda_stream);

/* ---- correlator sampling of caller-provided fields (Eqs. 11-12) ------- */

/* Scratch bytes and output length for flb_spectra_accumulate on n_fields real
 * fields of nx x ny (powers of two, nx <= 16384 FP32 / 8192 FP64, n_fields <= 11).
 * n_sums_out receives the number of doubles of the pair-sum array (see below).
 * Either output pointer may be NULL.  Pure host call. */
int flb_spectra_scratch_bytes(int precision, int nx, int ny, int n_fields,
                              size_t* bytes_out, size_t* n_sums_out);

/* Add, for every field pair a <= b in the order (0,0),(0,1),..,(0,F-1),(1,1),..,
 * the products X_a(k) X_b(k)^* of the discrete Fourier transforms
 * X(k) = sum_x X(x) exp(-i k.x) (Eq. 11) to FP64 sums on the half spectrum
 * kx in [0, nx/2], all ky: an auto pair occupies ny*(nx/2+1) doubles
 * [ky][kx], a cross pair ny*(nx/2+1) complex values (re, im interleaved).
 * mean0_dev[a] += X_a(0).  fields_dev: device [n_fields][ny][nx], float for
 * FLB_FP32_DEV (FP32 transforms) or double for FLB_FP64.  pair_sums_dev,
 * mean0_dev: device FP64, accumulated in place (zero them to start).
 * scratch_dev: caller-owned device memory of flb_spectra_scratch_bytes bytes,
 * 256-B aligned; its contents are overwritten.  Asynchronous on cuda_stream. */
int flb_spectra_accumulate(int precision, int nx, int ny, int n_fields, const void* fields_dev,
                           double* pair_sums_dev, double* mean0_dev, void* scratch_dev,
                           size_t scratch_bytes, void* cuda_stream);

/* Same as flb_spectra_accumulate, for callers that cannot allocate device memory
 * (a framework that owns the whole device memory budget through its own pool, a
 * service under a fixed memory cap, a latency-critical loop that must not pay
 * for cudaMalloc / cudaFree and their device-wide synchronisation).  The paper
 * has no counterpart: this is a deployment variant.  Its scratch is a fixed
 * 8 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits; sizes whose plan needs more return
 * FLB_EINVAL with a message.  Each call outside a stream capture looks up the
 * array's device address (cudaGetSymbolAddress) with the device current, so the
 * address stays right after a cudaDeviceReset; a call made while its stream is
 * being captured uses the address found by the last such call on that device, so
 * make the first call on a device (and the first after a reset) before any
 * capture.  Calls allocate nothing (the array's memory is taken when the library's
 * module is loaded on the device, at the latest by the first call).  All calls on
 * a device share the array, which keeps the last call's contents (each call
 * rewrites what it reads); calls whose GPU work overlaps race on it and must be
 * serialised.  Outputs and semantics as flb_spectra_accumulate. */
int flb_spectra_accumulate_static(int precision, int nx, int ny, int n_fields, const void* fields_dev,
                                  double* pair_sums_dev, double* mean0_dev, void* cuda_stream);

/* ---- training of the noise-scale network (learned extension) -------------
 * Weight vector (FP32, 1382 values): W1 (32x3) | W2 (32x32) | W3 (6x32) | b1 (32)
 * | b2 (32) | b3 (6), row-major; the order flb_set_mlp takes (weights, biases).
 * Loss over R training runs, K included wave vectors and the P = 6 hydrodynamic
 * pairs (rho rho, rho u_x, rho u_y, u_x u_x, u_x u_y, u_y u_y):
 *   L = 1/(R P K) sum_{r,p,k} |S^plain_rp(k) + sum_c (m_rc - 1) G^c_rp(k) - delta_p|^2,
 *   m_rc = mean over the run's B inputs of s_c(x)^2, s = 1 + network(x),
 * with S^plain the plain method's correlators and G^c those of runs with only
 * the noise of moment 3 + c (linear response of the equal-time covariance). */
int flb_mlp_param_count(void);

/* Per-run Gram terms of the loss: gram_dev[R][43] = (sum |D|^2, Re sum D^* G^c
 * (6), Re sum G^c* G^c' (36)), D = S^plain - delta_p.  splain_dev: device FP64
 * [R][P][K][2] (re, im); g_dev: [R][6][P][K][2].  P must be 6.  Asynchronous. */
int flb_mlp_gram(const double* splain_dev, const double* g_dev, int R, int P, int K,
                 double* gram_dev, void* cuda_stream);

/* Scratch bytes of flb_mlp_train_step for R runs of B inputs. */
int flb_mlp_scratch_bytes(int R, int B, size_t* bytes);

/* One training step: FP32 forward of all inputs x_dev [R][B][3] = (u_x, u_y,
 * rho - rho0), loss and m (written to loss_dev[1], m_dev[R][6], FP64), backward,
 * gradient (written to grad_dev[1382] if not NULL; summed in a fixed order), and
 * when lr > 0 an Adam update of w_dev with moments adam_m/v_dev and step t >= 1
 * (bias-corrected).  lr = 0: gradient only, weights unchanged.  Asynchronous. */
int flb_mlp_train_step(float* w_dev, float* adam_m_dev, float* adam_v_dev, int t, float lr,
                       float beta1, float beta2, float eps, const float* x_dev, int R, int B,
                       const double* gram_dev, int P, int K, double* loss_dev, double* m_dev,
                       float* grad_dev, void* scratch_dev, size_t scratch_bytes, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FLB_H */
