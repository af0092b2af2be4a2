// Three-dimensional fluctuating lattice Boltzmann: the scheme of Sec. 2 (pull streaming,
// Eq. 1; relaxation of the non-conserved moments, Eq. 5; noise of Eq. 8 on each of them) on
// D3Q15, the lattice that Sec. 3 reports testing without printing its tables, and on D3Q19.
//
// D3Q15 velocities (order of the population index i): rest, +x, -x, +y, -y, +z, -z,
// (1,1,1), (-1,-1,-1), (1,1,-1), (-1,-1,1), (1,-1,1), (-1,1,-1), (-1,1,1), (1,-1,-1); weights
// 2/9, 1/9 (axes), 1/72 (corners).
// D3Q19 velocities: rest, +x, -x, +y, -y, +z, -z, then the edges (1,1,0), (-1,-1,0),
// (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1),
// (0,-1,1); weights 1/3, 1/18 (axes), 1/36 (edges).  Both give sum_i w_i v_i v_i = 1/3 as
// Eq. 2 needs.
//
// Moments: the basis orthonormal in the weighted norm of Eq. 4 that Gram-Schmidt gives
// from the polynomials 1, vx, vy, vz, vx^2 - vy^2, vx^2 + vy^2 - 2 vz^2, vx vy, vy vz,
// vz vx, v^2 and then the ghosts (D3Q15: vx v^2, vy v^2, vz v^2, vx vy vz, v^4; D3Q19:
// vx v^2, vy v^2, vz v^2, vx (vy^2 - vz^2), vy (vz^2 - vx^2), vz (vx^2 - vy^2), v^4,
// (vx^2 - vy^2) v^2, (vx^2 + vy^2 - 2 vz^2) v^2).  Written out (moment_row3), both share
//   m^0 = 1, m^{1,2,3} = sqrt3 v, m^4 = 3/2 (vx^2 - vy^2), m^5 = sqrt3/2 (vx^2 + vy^2 - 2 vz^2),
//   m^6 = 3 vx vy, m^7 = 3 vy vz, m^8 = 3 vz vx, m^9 = sqrt6/2 (v^2 - 1);
// D3Q15 ghosts: m^{10,11,12} = sqrt6/4 v_a (3 v^2 - 5), m^13 = 3 vx vy vz,
//   m^14 = sqrt2/4 (3 v^4 - 9 v^2 + 4);
// D3Q19 ghosts: m^{10,11,12} = sqrt6/2 v_a (3 v^2 - 5), m^13 = 3/sqrt2 vx (vy^2 - vz^2),
//   m^14 = 3/sqrt2 vy (vz^2 - vx^2), m^15 = 3/sqrt2 vz (vx^2 - vy^2),
//   m^16 = sqrt2/2 (3 v^4 - 6 v^2 + 1), m^17 = 3/2 (vx^2 - vy^2)(2 v^2 - 3),
//   m^18 = sqrt3/2 (vx^2 + vy^2 - 2 vz^2)(2 v^2 - 3).
// The equilibrium moments (Eq. 10 in three dimensions) are those of f^0 of Eq. 2, the same
// on both lattices:
//   M^{4..9,0} = rho (3/2 (ux^2 - uy^2), sqrt3/2 (ux^2 + uy^2 - 2 uz^2), 3 ux uy, 3 uy uz,
//                     3 uz ux, sqrt6/2 u^2), and 0 for the ghosts (f^0 / w is a polynomial
//   of degree 2 in v, to which the ghost rows are orthogonal).
// Noise: normals 0, 1, ... of Philox calls 0, 1, ... (counter site, step, call, stream)
// drive moments 4, 5, ... (11 normals from 3 calls on D3Q15, 15 from 4 calls on D3Q19).
// Site index (z ny + y) nx + x; populations [q][nz][ny][nx].
//
// Sampling: the step writes the moment fields (pre-collision state, minus M^{a,0}(rho0,
// u0)); k_point_dft forms X_f(k) = sum_x X_f(x) exp(-i k.x) (Eq. 11) at the chosen wave
// vectors by direct summation, and the time-correlator kernels of spectra.cu accumulate
// X_a(k, s) X_b(k, s - tau)^*.
#include <algorithm>
#include "step_common.cuh"
#include "lattice3.cuh"

#ifndef FLB_STEP3_MINB
#define FLB_STEP3_MINB 2       // minimum resident blocks of 256 threads per SM (128 registers)
#endif

namespace flb {

// ---------------------------------------------------------------------------
// Pull streaming f_i(x) = f*_i(x - v_i) on the periodic box: the source row of population
// i is (y - v_iy, z - v_iz); the x shift is taken by warp shuffle from the adjacent lane,
// with one extra load at warp and row edges (as in the D2Q9 kernels).
template <int Q, typename R, int VEC>
__device__ __forceinline__ void pull_3d(const R* __restrict__ src, int64_t vol, int nx, int ny, int nz, int y, int z,
                                        const UnitPos& u, R (&f)[Q][VEC]) {
  R v[Q][VEC], e[Q];
  const int x0 = u.x0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int ys = y - v3y<Q>(i), zs = z - v3z<Q>(i);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
    const R* row = src + i * vol + ((int64_t)zs * ny + ys) * nx;
    if (FLB_INB(ys >= 0 && ys < ny && zs >= 0 && zs < nz && x0 >= 0 && x0 + VEC <= nx, 171))
      VecIO<R, VEC>::ld(row + x0, v[i]);
#ifdef FLB_CHECK_BOUNDS
    else for (int s = 0; s < VEC; ++s) v[i][s] = (R)0;
#endif
    e[i] = (R)0;
    if (v3x<Q>(i) == 1) {
      const int xe = x0 == 0 ? nx - 1 : x0 - 1;
      if (!u.left_in_warp && FLB_INB(xe >= 0 && xe < nx, 172)) e[i] = __ldg(row + xe);
    } else if (v3x<Q>(i) == -1) {
      const int xe = x0 + VEC == nx ? 0 : x0 + VEC;
      if (!u.right_in_warp && FLB_INB(xe >= 0 && xe < nx, 172)) e[i] = __ldg(row + xe);
    }
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (v3x<Q>(i) == 0) {
#pragma unroll
      for (int s = 0; s < VEC; ++s) f[i][s] = v[i][s];
    } else if (v3x<Q>(i) == 1) {
      const R left = __shfl_up_sync(0xffffffffu, v[i][VEC - 1], 1);
      f[i][0] = u.left_in_warp ? left : e[i];
#pragma unroll
      for (int s = 1; s < VEC; ++s) f[i][s] = v[i][s - 1];
    } else {
      const R right = __shfl_down_sync(0xffffffffu, v[i][0], 1);
#pragma unroll
      for (int s = 0; s < VEC - 1; ++s) f[i][s] = v[i][s + 1];
      f[i][VEC - 1] = u.right_in_warp ? right : e[i];
    }
  }
}

// D3Q15 collision of one site in place (Eqs. 5, 8): moments in closed form, relaxation of
// M^4..M^14 towards the equilibrium moments, noise amp_a N_{a-4}, and the back transform
// f*_i = f_i + w_i sum_a m_i^a Delta M^a.  fld: the 15 moments minus their reference
// values (SAMPLE).  DEV: g holds f - w rho0 (the non-conserved moments are the same).
template <typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void collide_d3q15(const ReplicaDesc& d, R (&g)[15], bool noisy, const R (&n)[11],
                                              R (&fld)[15]) {
  const R S2 = (R)1.4142135623730950488, S3 = (R)1.7320508075688772935, S6 = (R)2.4494897427831780982;
  const R hS2 = (R)0.70710678118654752440, hS3 = (R)0.86602540378443864676, hS6 = (R)1.2247448713915890491;
  // density and momentum
  const R s1 = g[7] + g[8], s2 = g[9] + g[10], s3 = g[11] + g[12], s4 = g[13] + g[14];
  const R d1 = g[7] - g[8], d2 = g[9] - g[10], d3 = g[11] - g[12], d4 = g[13] - g[14];
  const R ax = g[1] + g[2], ay = g[3] + g[4], az = g[5] + g[6];
  const R C = (s1 + s2) + (s3 + s4);
  const R sum = g[0] + ((ax + ay) + az) + C;
  const R cx = (d1 + d2) + (d3 - d4), cy = (d1 + d2) - (d3 - d4), cz = (d1 - d2) + (d3 + d4);
  const R jx = (g[1] - g[2]) + cx, jy = (g[3] - g[4]) + cy, jz = (g[5] - g[6]) + cz;
  const R rho = DEV ? coef<R>(d, kCoRho0) + sum : sum;
  const R irho = (R)1 / rho;
  const R ux = jx * irho, uy = jy * irho, uz = jz * irho;
  // non-conserved moments
  const R M4 = (R)1.5 * (ax - ay);
  const R M5 = hS3 * ((ax + ay) - (R)2 * az);
  const R M6 = (R)3 * ((s1 + s2) - (s3 + s4));
  const R M7 = (R)3 * ((s1 + s4) - (s2 + s3));
  const R M8 = (R)3 * ((s1 + s3) - (s2 + s4));
  const R M9 = S6 * (C - (R)0.5 * g[0]);
  const R M10 = S6 * ((R)0.5 * (g[2] - g[1]) + cx);
  const R M11 = S6 * ((R)0.5 * (g[4] - g[3]) + cy);
  const R M12 = S6 * ((R)0.5 * (g[6] - g[5]) + cz);
  const R M13 = (R)3 * ((d1 - d2) - (d3 + d4));
  const R M14 = S2 * ((g[0] - (R)0.5 * ((ax + ay) + az)) + C);
  // equilibrium moments
  const R E4 = (R)1.5 * (jx * ux - jy * uy);
  const R E5 = hS3 * ((jx * ux + jy * uy) - (R)2 * jz * uz);
  const R E6 = (R)3 * jx * uy, E7 = (R)3 * jy * uz, E8 = (R)3 * jz * ux;
  const R E9 = hS6 * ((jx * ux + jy * uy) + jz * uz);
  if constexpr (SAMPLE) {
    const R mom[15] = {sum, S3 * jx, S3 * jy, S3 * jz, M4, M5, M6, M7, M8, M9, M10, M11, M12, M13, M14};
#pragma unroll
    for (int a = 0; a < 15; ++a) fld[a] = mom[a] - coef<R>(d, kCoMref + a);
  }
  // relaxation (Eq. 5) and noise (Eq. 8)
  R D[11] = {E4 - M4, E5 - M5, E6 - M6, E7 - M7, E8 - M8, E9 - M9, -M10, -M11, -M12, -M13, -M14};
#pragma unroll
  for (int c = 0; c < 11; ++c) {
    D[c] *= coef<R>(d, kCoInvTau + 4 + c);
    if (noisy) D[c] += coef<R>(d, kCoAmp + 4 + c) * n[c];
  }
  const R D4 = D[0], D5 = D[1], D6 = D[2], D7 = D[3], D8 = D[4], D9 = D[5];
  const R D10 = D[6], D11 = D[7], D12 = D[8], D13 = D[9], D14 = D[10];
  // back transform, n_i^a = w_i m_i^a
  const R wa = (R)1 / (R)9, wc = (R)1 / (R)72;
  g[0] = g[0] + (R)(2.0 / 9.0) * (S2 * D14 - hS6 * D9);
  const R base = hS3 * D5 - hS2 * D14;             // common to the axis populations
  const R hx = (R)1.5 * D4;
  const R tx = hS6 * D10, ty = hS6 * D11, tz = hS6 * D12;
  g[1] = g[1] + wa * ((base + hx) - tx);
  g[2] = g[2] + wa * ((base + hx) + tx);
  g[3] = g[3] + wa * ((base - hx) - ty);
  g[4] = g[4] + wa * ((base - hx) + ty);
  const R bz = -S3 * D5 - hS2 * D14;
  g[5] = g[5] + wa * (bz - tz);
  g[6] = g[6] + wa * (bz + tz);
  // corners: w (G + E(v) +- O(v)), E even and O odd in v
  const R G = S6 * D9 + S2 * D14;
  const R p6 = (R)3 * D6, p7 = (R)3 * D7, p8 = (R)3 * D8, p13 = (R)3 * D13;
  const R q10 = S6 * D10, q11 = S6 * D11, q12 = S6 * D12;
  {
    const R E = G + ((p6 + p7) + p8), O = ((q10 + q11) + q12) + p13;       // (1,1,1)
    g[7] = g[7] + wc * (E + O);
    g[8] = g[8] + wc * (E - O);
  }
  {
    const R E = G + ((p6 - p7) - p8), O = ((q10 + q11) - q12) - p13;       // (1,1,-1)
    g[9] = g[9] + wc * (E + O);
    g[10] = g[10] + wc * (E - O);
  }
  {
    const R E = G + ((p8 - p6) - p7), O = ((q10 - q11) + q12) - p13;       // (1,-1,1)
    g[11] = g[11] + wc * (E + O);
    g[12] = g[12] + wc * (E - O);
  }
  {
    const R E = G + ((p7 - p6) - p8), O = ((q11 + q12) - q10) - p13;       // (-1,1,1)
    g[13] = g[13] + wc * (E + O);
    g[14] = g[14] + wc * (E - O);
  }
}

// D3Q19 collision of one site in place: as collide_d3q15, on the 19 populations grouped
// into the rest population and nine +-v pairs (sums e, differences o): the even moments
// (0, 4-9, 16-18) are sums of e, the odd ones (1-3, 10-15) sums of o.
template <typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void collide_d3q19(const ReplicaDesc& d, R (&g)[19], bool noisy, const R (&n)[15],
                                              R (&fld)[19]) {
  const R S2 = (R)1.4142135623730950488, S3 = (R)1.7320508075688772935, S6 = (R)2.4494897427831780982;
  const R hS2 = (R)0.70710678118654752440, hS3 = (R)0.86602540378443864676, hS6 = (R)1.2247448713915890491;
  const R t2 = (R)2.1213203435596425732;           // 3 / sqrt2
  // pair sums and differences: axes x, y, z; edges A (1,1,0), B (1,-1,0), C (1,0,1),
  // D (1,0,-1), E (0,1,1), F (0,1,-1) (first member of each pair)
  const R ax = g[1] + g[2], ay = g[3] + g[4], az = g[5] + g[6];
  const R ox = g[1] - g[2], oy = g[3] - g[4], oz = g[5] - g[6];
  const R eA = g[7] + g[8], eB = g[9] + g[10], eC = g[11] + g[12], eD = g[13] + g[14], eE = g[15] + g[16],
          eF = g[17] + g[18];
  const R dA = g[7] - g[8], dB = g[9] - g[10], dC = g[11] - g[12], dD = g[13] - g[14], dE = g[15] - g[16],
          dF = g[17] - g[18];
  const R Sxy = eA + eB, Sxz = eC + eD, Syz = eE + eF, S = (Sxy + Sxz) + Syz;
  const R aa = (ax + ay) + az;
  const R sum = (g[0] + aa) + S;
  const R cx = (dA + dB) + (dC + dD), cy = (dA - dB) + (dE + dF), cz = (dC - dD) + (dE - dF);
  const R jx = ox + cx, jy = oy + cy, jz = oz + cz;
  const R rho = DEV ? coef<R>(d, kCoRho0) + sum : sum;
  const R irho = (R)1 / rho;
  const R ux = jx * irho, uy = jy * irho, uz = jz * irho;
  // non-conserved moments
  const R dxy = ax - ay, sxz = Sxz - Syz, pxy = ax + ay, t5 = (R)2 * Sxy - (Sxz + Syz);
  const R M4 = (R)1.5 * (dxy + sxz);
  const R M5 = hS3 * ((pxy - (R)2 * az) + t5);
  const R M6 = (R)3 * (eA - eB), M7 = (R)3 * (eE - eF), M8 = (R)3 * (eC - eD);
  const R M9 = hS6 * (S - g[0]);
  const R M10 = hS6 * (cx - (R)2 * ox), M11 = hS6 * (cy - (R)2 * oy), M12 = hS6 * (cz - (R)2 * oz);
  const R M13 = t2 * ((dA + dB) - (dC + dD));
  const R M14 = t2 * ((dB - dA) + (dE + dF));
  const R M15 = t2 * ((dC - dD) + (dF - dE));
  const R M16 = hS2 * ((g[0] - (R)2 * aa) + S);
  const R M17 = (R)1.5 * (sxz - dxy);
  const R M18 = hS3 * (((R)2 * az - pxy) + t5);
  // equilibrium moments
  const R E4 = (R)1.5 * (jx * ux - jy * uy);
  const R E5 = hS3 * ((jx * ux + jy * uy) - (R)2 * jz * uz);
  const R E6 = (R)3 * jx * uy, E7 = (R)3 * jy * uz, E8 = (R)3 * jz * ux;
  const R E9 = hS6 * ((jx * ux + jy * uy) + jz * uz);
  if constexpr (SAMPLE) {
    const R mom[19] = {sum, S3 * jx, S3 * jy, S3 * jz, M4, M5, M6, M7, M8, M9, M10, M11, M12, M13, M14, M15, M16,
                       M17, M18};
#pragma unroll
    for (int a = 0; a < 19; ++a) fld[a] = mom[a] - coef<R>(d, kCoMref + a);
  }
  // relaxation (Eq. 5) and noise (Eq. 8)
  R D[15] = {E4 - M4, E5 - M5, E6 - M6, E7 - M7, E8 - M8, E9 - M9, -M10, -M11, -M12, -M13, -M14, -M15, -M16,
             -M17, -M18};
#pragma unroll
  for (int c = 0; c < 15; ++c) {
    D[c] *= coef<R>(d, kCoInvTau + 4 + c);
    if (noisy) D[c] += coef<R>(d, kCoAmp + 4 + c) * n[c];
  }
  const R D4 = D[0], D5 = D[1], D6 = D[2], D7 = D[3], D8 = D[4], D9 = D[5], D10 = D[6], D11 = D[7], D12 = D[8];
  const R D13 = D[9], D14 = D[10], D15 = D[11], D16 = D[12], D17 = D[13], D18 = D[14];
  // back transform, n_i^a = w_i m_i^a: f(+-v) += w (E(v) +- O(v))
  const R wr = (R)1 / (R)3, wa = (R)1 / (R)18, we = (R)1 / (R)36;
  g[0] = g[0] + wr * (hS2 * D16 - hS6 * D9);
  const R p417 = (R)1.5 * (D4 - D17), p518 = D5 - D18, q16 = S2 * D16;
  {
    const R E = (p417 + hS3 * p518) - q16, O = -S6 * D10;                   // x
    g[1] = g[1] + wa * (E + O);
    g[2] = g[2] + wa * (E - O);
  }
  {
    const R E = (hS3 * p518 - p417) - q16, O = -S6 * D11;                   // y
    g[3] = g[3] + wa * (E + O);
    g[4] = g[4] + wa * (E - O);
  }
  {
    const R E = -S3 * p518 - q16, O = -S6 * D12;                            // z
    g[5] = g[5] + wa * (E + O);
    g[6] = g[6] + wa * (E - O);
  }
  const R G = hS6 * D9 + hS2 * D16;                  // common to the edges
  const R s518 = D5 + D18, s417 = (R)1.5 * (D4 + D17);
  const R Gxy = G + S3 * s518, Gxz = (G + s417) - hS3 * s518, Gyz = (G - s417) - hS3 * s518;
  const R h10 = hS6 * D10, h11 = hS6 * D11, h12 = hS6 * D12;
  const R k13 = t2 * D13, k14 = t2 * D14, k15 = t2 * D15;
  {
    const R E = Gxy + (R)3 * D6, O = (h10 + h11) + (k13 - k14);          // A (1,1,0)
    g[7] = g[7] + we * (E + O);
    g[8] = g[8] + we * (E - O);
  }
  {
    const R E = Gxy - (R)3 * D6, O = (h10 - h11) + (k13 + k14);          // B (1,-1,0)
    g[9] = g[9] + we * (E + O);
    g[10] = g[10] + we * (E - O);
  }
  {
    const R E = Gxz + (R)3 * D8, O = (h10 + h12) + (k15 - k13);          // C (1,0,1)
    g[11] = g[11] + we * (E + O);
    g[12] = g[12] + we * (E - O);
  }
  {
    const R E = Gxz - (R)3 * D8, O = (h10 - h12) - (k13 + k15);          // D (1,0,-1)
    g[13] = g[13] + we * (E + O);
    g[14] = g[14] + we * (E - O);
  }
  {
    const R E = Gyz + (R)3 * D7, O = (h11 + h12) + (k14 - k15);          // E (0,1,1)
    g[15] = g[15] + we * (E + O);
    g[16] = g[16] + we * (E - O);
  }
  {
    const R E = Gyz - (R)3 * D7, O = (h11 - h12) + (k14 + k15);          // F (0,1,-1)
    g[17] = g[17] + we * (E + O);
    g[18] = g[18] + we * (E - O);
  }
}

template <int Q, typename R, bool DEV, bool SAMPLE>
__device__ __forceinline__ void collide_3d(const ReplicaDesc& d, R (&g)[Q], bool noisy, const R (&n)[Q - 4],
                                           R (&fld)[Q]) {
  if constexpr (Q == 15) collide_d3q15<R, DEV, SAMPLE>(d, g, noisy, n, fld);
  else collide_d3q19<R, DEV, SAMPLE>(d, g, noisy, n, fld);
}

// The Q - 4 unit normals of a site (Philox calls 0, 1, ...; the rest of the last call's
// words are not used).
template <int Q, typename R>
__device__ __forceinline__ void normals_3d(const ReplicaDesc& d, uint32_t site, uint32_t step, R (&n)[Q - 4]) {
  constexpr int NC = Q - 4;
#pragma unroll
  for (int c = 0; c < Lat3<Q>::kCalls; ++c) {
    const uint4 w = philox4x32_10(site, step, (uint32_t)c, d.stream, d.seed_lo, d.seed_hi);
    R a, b, e, h;
    box_muller(w.x, w.y, a, b);
    box_muller(w.z, w.w, e, h);
    const R v[4] = {a, b, e, h};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (4 * c + k < NC) n[4 * c + k] = v[k];
  }
}

// One thread = VEC consecutive sites of a row (y, z); a persistent grid loops over virtual
// blocks of kStepThreads units, each within one replica.  ONE: a single replica whose
// description is the kernel argument (constant bank).
template <int Q, typename R, bool DEV, int VEC, bool SAMPLE, bool ONE>
__global__ void __launch_bounds__(kStepThreads, FLB_STEP3_MINB)
k_step_3d(const ReplicaDesc* __restrict__ descs, const __grid_constant__ ReplicaDesc one,
          const int64_t* __restrict__ vb_begin, int n_reps, int64_t n_vblocks, char* __restrict__ ws, int parity,
          uint32_t step, const uint64_t* __restrict__ step_dev) {
  if (step_dev) {
    const uint64_t t = *step_dev + step;
    step = (uint32_t)t;
    parity = (int)(t & 1);
  }
  for (int64_t vb = blockIdx.x; vb < n_vblocks; vb += gridDim.x) {
    const int r = ONE ? 0 : find_replica(vb_begin, n_reps, vb);
    const ReplicaDesc& d = ONE ? one : descs[r];
    const UnitPos u = unit_position(d, vb, ONE ? 0 : vb_begin[r], (int)threadIdx.x, kStepThreads, VEC);
    const int row = u.y;                       // z ny + y
    const int z = row / d.ny, y = row - z * d.ny;
    const int64_t vol = (int64_t)d.nx * d.ny * d.nz;
    const R* __restrict__ src = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
    R* __restrict__ dst = reinterpret_cast<R*>(ws + d.off_pop[parity ^ 1]);
    R f[Q][VEC];
    pull_3d<Q, R, VEC>(src, vol, d.nx, d.ny, d.nz, y, z, u, f);
    const bool noisy = d.noise_mask != 0;
    const int64_t off = (int64_t)row * d.nx + u.x0;
    R* fields = SAMPLE ? reinterpret_cast<R*>(ws + d.off_fields) : nullptr;
#pragma unroll
    for (int s = 0; s < VEC; ++s) {
      R g[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = f[i][s];
      R n[Q - 4];
#pragma unroll
      for (int c = 0; c < Q - 4; ++c) n[c] = (R)0;
      if (noisy) normals_3d<Q, R>(d, (uint32_t)row * (uint32_t)d.nx + (uint32_t)(u.x0 + s), step, n);
      R fl[Q];
      collide_3d<Q, R, DEV, SAMPLE>(d, g, noisy, n, fl);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i][s] = g[i];
      if constexpr (SAMPLE) {
        // the site's sampled fields, stored at once (scalar stores; the lanes of a warp
        // cover contiguous rows of each field plane)
        if (u.active && FLB_INB(off + s < vol, 174))
          for (int slot = 0; slot < (int)d.n_fields; ++slot) {
            const int fid = d.field_id[slot];
            R val = fl[0];
#pragma unroll
            for (int a = 1; a < Q; ++a) val = (fid == a) ? fl[a] : val;
            fields[slot * vol + off + s] = val;
          }
      }
    }
    if (!u.active || !FLB_INB(off >= 0 && off + VEC <= vol, 173)) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) VecIO<R, VEC>::st(dst + i * vol + off, f[i]);
  }
}

// ---------------------------------------------------------------------------
// Initial state.  mode 0: f^0(rho0, u0).  mode 1: f^0 + sum_a n_i^a dM^a with dM^a =
// sqrt(mu rho0) N_a (Q normals: Philox tag 1, step 0, calls 0, 1, ...) and the lattice mean
// of the density and momentum fluctuations removed (k_thermal_sum3 sums them first).
template <int Q>
__device__ __forceinline__ void thermal_normals3(const ReplicaDesc& d, uint32_t site, double (&N)[4 * Lat3<Q>::kThermalCalls]) {
#pragma unroll
  for (int c = 0; c < Lat3<Q>::kThermalCalls; ++c) {
    const uint4 w = philox4x32_10(site, 0u, (uint32_t)c | (1u << 8), d.stream, d.seed_lo, d.seed_hi);
    box_muller(w.x, w.y, N[4 * c + 0], N[4 * c + 1]);
    box_muller(w.z, w.w, N[4 * c + 2], N[4 * c + 3]);
  }
}

template <int Q>
__global__ void k_thermal_sum3(const ReplicaDesc* __restrict__ descs, int r, double* __restrict__ partial) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny * d.nz;
  double acc[kNumSums] = {0, 0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double N[4 * Lat3<Q>::kThermalCalls];
    thermal_normals3<Q>(d, (uint32_t)s, N);
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] += N[a];
  }
  block_sums(acc, partial);
}

// feq0: f^0_i(rho0, u0) at [i], w_i rho0 at [kFeqW + i]
template <int Q, typename R, bool DEV>
__global__ void k_init3(const ReplicaDesc* __restrict__ descs, int r, char* __restrict__ ws, int mode,
                        const double* __restrict__ feq0, const double* __restrict__ sums) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny * d.nz;
  R* dst = reinterpret_cast<R*>(ws + d.off_pop[0]);
  const double sm = sqrt(d.mu * d.rho0);
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double M[Q];
    if (mode == 1) {
      double N[4 * Lat3<Q>::kThermalCalls];
      thermal_normals3<Q>(d, (uint32_t)s, N);
#pragma unroll
      for (int a = 0; a < Q; ++a) M[a] = sm * N[a];
#pragma unroll
      for (int a = 0; a < 4; ++a) M[a] -= sm * sums[a] / (double)V;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double v = feq0[i];
      if (mode == 1) {
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < Q; ++a) acc += moment_row3<Q>(a, v3x<Q>(i), v3y<Q>(i), v3z<Q>(i)) * M[a];
        v += w3<Q>(i) * acc;
      }
      if (DEV) v -= feq0[kFeqW + i];
      dst[i * V + s] = (R)v;
    }
  }
}

// FP64 lattice sums of rho, j_x, j_y, j_z of the stored state (per-block partials).
template <int Q, typename R, bool DEV>
__global__ void k_conserved3(const ReplicaDesc* __restrict__ descs, int r, const char* __restrict__ ws, int parity,
                             double* __restrict__ partial) {
  const ReplicaDesc& d = descs[r];
  const int64_t V = (int64_t)d.nx * d.ny * d.nz;
  const R* p = reinterpret_cast<const R*>(ws + d.off_pop[parity]);
  double acc[kNumSums] = {0, 0, 0, 0};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    double rho = DEV ? d.rho0 : 0.0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fv = (double)p[i * V + s];
      rho += fv;
      jx += v3x<Q>(i) * fv; jy += v3y<Q>(i) * fv; jz += v3z<Q>(i) * fv;
    }
    acc[0] += rho; acc[1] += jx; acc[2] += jy; acc[3] += jz;
  }
  block_sums(acc, partial);
}

// ---------------------------------------------------------------------------
// Direct transforms at the time-correlator wave vectors.  Block b of replica blockIdx.y
// takes the row groups b, b + G, ... (G = gridDim.x) of R consecutive rows.  The x sum
// of a row depends on the field and on k_x only, so it is formed once per (row, field,
// distinct k_x): thread (q, part) sums x = part, part + P, ... with the phase
// exp(-2 pi i (kx x mod nx) / nx) from a table, in the path's precision; then each item
// (field f, wave vector j) adds, row by row, its row sum times the row phase
// exp(-2 pi i (ky y / ny + kz z / nz)) (FP64 tables) to its FP64 accumulator.  The
// block's sums go to partial [G][F n_k].
// The phase tables are made once per replica (k_point_tables, at configuration) in the
// correlator buffer at off_tc_tab: x table (nx complex R, 16-byte padded) | y, z tables
// (ny + nz complex double); each block copies them to shared memory, followed by the
// per-part row sums [P][R F n_kx] (complex R) and the accumulators [F n_k] (complex double).
// Shape of one pass: R consecutive rows at a time, P parts per (row, field, k_x) item,
// R * items2 * P <= kStepThreads.
__host__ __device__ inline void point_dft_shape(int items2, int& R, int& P) {
  R = kStepThreads / (4 * items2);
  R = R < 1 ? 1 : (R > 8 ? 8 : R);
  P = 1;
  while (R * items2 * P * 2 <= kStepThreads) P *= 2;
}

size_t point_tables_bytes(int precision, int nx, int ny, int nz) {
  const size_t cs = precision == FLB_FP64 ? 16 : 8;
  return ((nx * cs + 15) & ~size_t(15)) + (size_t)(ny + nz) * 16;
}

// items = F n_k, items2 = F n_kx
size_t point_dft_smem(int precision, int nx, int ny, int nz, int items, int items2) {
  const size_t cs = precision == FLB_FP64 ? 16 : 8;
  int R, P;
  point_dft_shape(items2, R, P);
  const size_t red = ((size_t)P * R * items2 * cs + 15) & ~size_t(15);
  return point_tables_bytes(precision, nx, ny, nz) + red + (size_t)items * 16;
}

template <typename R>
__global__ void k_point_tables(const ReplicaDesc* __restrict__ descs, char* __restrict__ base) {
  const ReplicaDesc& d = descs[blockIdx.y];
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  cplx<R>* tx = reinterpret_cast<cplx<R>*>(base + d.off_tc_tab);
  double2* tyz = reinterpret_cast<double2*>(base + d.off_tc_tab + ((nx * sizeof(cplx<R>) + 15) & ~size_t(15)));
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nx + ny + nz; m += gridDim.x * blockDim.x) {
    double s, c;
    if (m < nx) {
      sincospi(-2.0 * (double)m / (double)nx, &s, &c);
      tx[m].x = (R)c; tx[m].y = (R)s;
    } else {
      const int k = m - nx;
      sincospi(k < ny ? -2.0 * (double)k / (double)ny : -2.0 * (double)(k - ny) / (double)nz, &s, &c);
      tyz[k] = make_double2(c, s);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kStepThreads)
k_point_dft(const ReplicaDesc* __restrict__ descs, const char* __restrict__ ws, TimeCorr tc) {
  extern __shared__ __align__(16) unsigned char psm[];
  const ReplicaDesc& d = descs[blockIdx.y];
  const int F = (int)d.n_fields, nk = tc.n_k, nkx = tc.n_kx;
  const int items = F * nk, items2 = F * nkx;
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int64_t vol = (int64_t)nx * ny * nz;
  const size_t txb = (nx * sizeof(cplx<R>) + 15) & ~size_t(15);
  {
    const int4* src = reinterpret_cast<const int4*>(tc.base + d.off_tc_tab);
    int4* dst = reinterpret_cast<int4*>(psm);
    const int n16 = (int)((txb + (size_t)(ny + nz) * 16) / 16);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
  }
  const cplx<R>* tx = reinterpret_cast<const cplx<R>*>(psm);
  const double2* tyz = reinterpret_cast<const double2*>(psm + txb);
  int RR, P;
  point_dft_shape(items2, RR, P);
  const int q2n = RR * items2;                        // (row in pass, field, k_x) items
  cplx<R>* red = reinterpret_cast<cplx<R>*>(psm + txb + (size_t)(ny + nz) * 16);               // [P][q2n]
  double2* acc = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(red) +
                                            (((size_t)P * q2n * sizeof(cplx<R>) + 15) & ~size_t(15)));
  for (int it = threadIdx.x; it < items; it += blockDim.x) acc[it] = make_double2(0.0, 0.0);
  const int part = (int)threadIdx.x % P, qbase = (int)threadIdx.x / P, qstride = (int)blockDim.x / P;
  const R* fields = reinterpret_cast<const R*>(ws + d.off_fields);
  const int rows = ny * nz;
  const uint32_t unx = (uint32_t)nx, uny = (uint32_t)ny, unz = (uint32_t)nz;
  __syncthreads();
  for (int row0 = blockIdx.x * RR; row0 < rows; row0 += gridDim.x * RR) {
    // row sums per (row, field, distinct k_x); all index products stay below 2^24
    for (int q2 = qbase; q2 < q2n; q2 += qstride) {
      const int rr = q2 / items2, q = q2 - rr * items2;
      const int row = row0 + rr;
      cplx<R> sv;
      sv.x = (R)0; sv.y = (R)0;
      if (row < rows) {
        const int f = q / nkx;
        const uint32_t kx = (uint32_t)tc.kxl[q - f * nkx];
        const R* xr = fields + f * vol + (int64_t)row * nx;
        const int dm = (int)((kx * (uint32_t)P) % unx);
        int m0 = (int)((kx * (uint32_t)part) % unx);
        R sr0 = (R)0, si0 = (R)0, sr1 = (R)0, si1 = (R)0;
        int x = part;
        for (; x + 3 * P < nx; x += 4 * P) {
          const R v0 = xr[x], v1 = xr[x + P], v2 = xr[x + 2 * P], v3 = xr[x + 3 * P];
          int m1 = m0 + dm; m1 -= m1 >= nx ? nx : 0;
          int m2 = m1 + dm; m2 -= m2 >= nx ? nx : 0;
          int m3 = m2 + dm; m3 -= m3 >= nx ? nx : 0;
          const cplx<R> c0 = tx[m0], c1 = tx[m1], c2 = tx[m2], c3 = tx[m3];
          sr0 += v0 * c0.x; si0 += v0 * c0.y;
          sr1 += v1 * c1.x; si1 += v1 * c1.y;
          sr0 += v2 * c2.x; si0 += v2 * c2.y;
          sr1 += v3 * c3.x; si1 += v3 * c3.y;
          m0 = m3 + dm; m0 -= m0 >= nx ? nx : 0;
        }
        for (; x < nx; x += P) {
          const R v = xr[x];
          sr0 += v * tx[m0].x; si0 += v * tx[m0].y;
          m0 += dm; m0 -= m0 >= nx ? nx : 0;
        }
        sv.x = sr0 + sr1; sv.y = si0 + si1;
      }
      red[part * q2n + q2] = sv;
    }
    __syncthreads();
    // each wave vector: its field's row sums at its k_x times the row phases, in FP64,
    // rows in order
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int f = it / nk, j = it - f * nk;
      const int q = f * nkx + tc.kxi[j];
      const uint32_t ky = (uint32_t)tc.ky[j], kz = (uint32_t)tc.kz[j];
      double2 a = acc[it];
      for (int rr = 0; rr < RR; ++rr) {
        const int row = row0 + rr;
        if (row >= rows) break;
        const int q2 = rr * items2 + q;
        R sr = red[q2].x, si = red[q2].y;
        for (int p = 1; p < P; ++p) { sr += red[p * q2n + q2].x; si += red[p * q2n + q2].y; }
        const uint32_t z = (uint32_t)row / uny, y = (uint32_t)row - z * uny;
        const double2 py = tyz[(ky * y) % uny];
        const double2 pz = tyz[ny + (kz * z) % unz];
        const double pr = py.x * pz.x - py.y * pz.y, pi = py.x * pz.y + py.y * pz.x;
        a.x += (double)sr * pr - (double)si * pi;
        a.y += (double)sr * pi + (double)si * pr;
      }
      acc[it] = a;
    }
    __syncthreads();
  }
  double2* out = reinterpret_cast<double2*>(tc.base + d.off_tc_part) + (int64_t)blockIdx.x * items;
  for (int it = threadIdx.x; it < items; it += blockDim.x) out[it] = acc[it];
}

// Adds the G block partials of one item (blockIdx.x) into the replica's ring slot
// count % n_lags: thread t sums blocks t, t + 256, ... in order, then a fixed tree adds
// the 256 partial sums (the same order every time).
__global__ void __launch_bounds__(256) k_point_finish(const ReplicaDesc* __restrict__ descs, TimeCorr tc) {
  __shared__ double2 sred[256];
  const int r = blockIdx.y;
  const ReplicaDesc& d = descs[r];
  const int items = (int)d.n_fields * tc.n_k;
  const int it = blockIdx.x;
  if (it >= items) return;                      // uniform over the block
  const double2* part = reinterpret_cast<const double2*>(tc.base + d.off_tc_part);
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < tc.part_blocks; b += blockDim.x) {
    const double2 v = part[(int64_t)b * items + it];
    s.x += v.x; s.y += v.y;
  }
  sred[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sred[threadIdx.x].x += sred[threadIdx.x + h].x;
      sred[threadIdx.x].y += sred[threadIdx.x + h].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int slot = (int)(tc.count[r] % (uint64_t)tc.n_lags);
    reinterpret_cast<double2*>(tc.base + d.off_tc_ring)[(int64_t)slot * items + it] = sred[0];
  }
}

// ---------------------------------------------------------------------------
// Host launchers (called from api.cu).

void launch_finish_sums(const double* partial, int nblocks, double* sums, DevStatus* status, int r,
                        cudaStream_t st);

template <int Q>
static void launch_step3_q(int precision, int vec, const StepLaunch& L, bool sample, cudaStream_t st) {
  const bool one = L.n_reps == 1;
#define FLB_L3(R, DEV, V, S, O) k_step_3d<Q, R, DEV, V, S, O><<<L.grid, kStepThreads, 0, st>>>( \
      L.descs, *L.desc0, L.vb_begin, L.n_reps, L.n_vblocks, L.ws, L.parity, L.step, L.step_dev)
#define FLB_LS(R, DEV, V) { \
    if (one) { if (sample) FLB_L3(R, DEV, V, true, true); else FLB_L3(R, DEV, V, false, true); } \
    else { if (sample) FLB_L3(R, DEV, V, true, false); else FLB_L3(R, DEV, V, false, false); } }
  if (precision == FLB_FP64) FLB_LS(double, false, 1)
  else if (vec == 4) FLB_LS(float, true, 4)
  else if (vec == 2) FLB_LS(float, true, 2)
  else FLB_LS(float, true, 1)
#undef FLB_LS
#undef FLB_L3
}

void launch_step3(int q, int precision, int vec, const StepLaunch& L, bool sample, cudaStream_t st) {
  if (q == 15) launch_step3_q<15>(precision, vec, L, sample, st);
  else launch_step3_q<19>(precision, vec, L, sample, st);
}

template <int Q>
static void launch_init3_q(int precision, const ReplicaDesc* descs, int r, char* ws, int mode, const double* feq0,
                           double* sums, double* partial, int64_t V, cudaStream_t st) {
  const int block = 256;
  const int grid = (int)std::min<int64_t>((V + block - 1) / block, kReduceBlocks);
  if (mode == 1) {
    k_thermal_sum3<Q><<<grid, block, 0, st>>>(descs, r, partial);
    launch_finish_sums(partial, grid, sums, nullptr, r, st);
  }
  if (precision == FLB_FP64) k_init3<Q, double, false><<<grid, block, 0, st>>>(descs, r, ws, mode, feq0, sums);
  else k_init3<Q, float, true><<<grid, block, 0, st>>>(descs, r, ws, mode, feq0, sums);
}

void launch_init3(int q, int precision, const ReplicaDesc* descs, int r, char* ws, int mode, const double* feq0,
                  double* sums, double* partial, int64_t V, cudaStream_t st) {
  if (q == 15) launch_init3_q<15>(precision, descs, r, ws, mode, feq0, sums, partial, V, st);
  else launch_init3_q<19>(precision, descs, r, ws, mode, feq0, sums, partial, V, st);
}

template <int Q>
static void launch_conserved3_q(int precision, const ReplicaDesc* descs, int r, const char* ws, int parity,
                                double* sums, double* partial, DevStatus* status, int64_t V, cudaStream_t st) {
  const int block = 256;
  const int grid = (int)std::min<int64_t>((V + block - 1) / block, kReduceBlocks);
  if (precision == FLB_FP64) k_conserved3<Q, double, false><<<grid, block, 0, st>>>(descs, r, ws, parity, partial);
  else k_conserved3<Q, float, true><<<grid, block, 0, st>>>(descs, r, ws, parity, partial);
  launch_finish_sums(partial, grid, sums, status, r, st);
}

void launch_conserved3(int q, int precision, const ReplicaDesc* descs, int r, const char* ws, int parity, double* sums,
                       double* partial, DevStatus* status, int64_t V, cudaStream_t st) {
  if (q == 15) launch_conserved3_q<15>(precision, descs, r, ws, parity, sums, partial, status, V, st);
  else launch_conserved3_q<19>(precision, descs, r, ws, parity, sums, partial, status, V, st);
}

cudaError_t set_point_dft_smem(int precision, size_t bytes) {
  if (precision == FLB_FP64)
    return cudaFuncSetAttribute(k_point_dft<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(k_point_dft<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_point_tables(int precision, const ReplicaDesc* descs, int n_reps, char* base, cudaStream_t st) {
  const dim3 grid(16, n_reps);
  if (precision == FLB_FP64) k_point_tables<double><<<grid, 256, 0, st>>>(descs, base);
  else k_point_tables<float><<<grid, 256, 0, st>>>(descs, base);
}

void launch_point_dft(int precision, const ReplicaDesc* descs, int n_reps, int max_items, const char* ws,
                      const TimeCorr& tc, size_t smem, cudaStream_t st) {
  const dim3 grid(tc.part_blocks, n_reps);
  if (precision == FLB_FP64) k_point_dft<double><<<grid, kStepThreads, smem, st>>>(descs, ws, tc);
  else k_point_dft<float><<<grid, kStepThreads, smem, st>>>(descs, ws, tc);
  k_point_finish<<<dim3(max_items, n_reps), 256, 0, st>>>(descs, tc);
}

}  // namespace flb
