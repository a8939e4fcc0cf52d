// The fused coupled PF-LB step kernel (one launch per time step).
//
// Each block owns a tile of TA x TB cells across the fast axes and marches a
// chunk of cells along the slow axis (z in 3D, y in 2D). The order parameter
// of the planes around the current one lives in a shared-memory ring (radius
// 1 for the Allen-Cahn families, 2 for Cahn-Hilliard, whose chemical
// potential needs its own Laplacian and lives in a second ring). Each new
// plane's phi is recomputed from the incoming g populations of the tile and
// its halo, so phi is never written to device memory.
//
// Streaming: g uses two arrays (read one, push into the other), which keeps
// the g read by a neighbouring block's halo unmodified during the step; f
// uses the AA pattern in place (even steps read and write the cell's own
// slots, reversed; odd steps read from and write to the neighbours).
// Halfway bounce-back walls (2D, y ends) reflect into the cell's own slots.
#pragma once

#include <type_traits>

#include "pflb_args.h"
#include "pflb_mrt.cuh"
#include "pflb_symsum.cuh"
#include "pflb_tma.cuh"

namespace pflb {

template <int FAM, int DIM, typename T, int LAT = 0>
struct Geom {
  static constexpr int STORAGE = std::is_same<T, float>::value ? 0 : 1;
  static constexpr int TA = tile_shape(FAM, DIM, STORAGE, LAT).ta;
  static constexpr int TB = tile_shape(FAM, DIM, STORAGE, LAT).tb;
  static constexpr int MINB = tile_shape(FAM, DIM, STORAGE, LAT).minb;
};



// Kernel-space offsets of a physical lattice velocity: (a, b, c) = (x, y, z)
// in 3D and (x, -, y) in 2D.
template <int DIM, typename L>
__device__ __forceinline__ constexpr int da_of(int q) { return L::ex(q); }
template <int DIM, typename L>
__device__ __forceinline__ constexpr int db_of(int q) { return DIM == 3 ? L::ey(q) : 0; }
template <int DIM, typename L>
__device__ __forceinline__ constexpr int dc_of(int q) { return DIM == 3 ? L::ez(q) : L::ey(q); }

// Physical component k of a velocity.
template <typename L>
__device__ __forceinline__ constexpr int ecomp(int q, int k) {
  return k == 0 ? L::ex(q) : (k == 1 ? L::ey(q) : L::ez(q));
}

__device__ __forceinline__ int wrap_mod(int v, int n) {
  int m = v % n;
  return m < 0 ? m + n : m;
}

// Kinematic viscosity, Eqs. (fakhari_mu_update), (mu_linear), (mu_inverse), (mu_log).
__device__ __forceinline__ float viscosity(const DevParams& P, float phi, float rho) {
  const float t = (phi - P.phiL) * P.inv_dphi;
  switch (P.visc_interp) {
    case 0: return P.nuL + (P.nuH - P.nuL) * t;
    case 1: return (P.muL + (P.muH - P.muL) * t) / rho;
    case 2: return P.muH * P.muL / (t * P.muL + (1.0f - t) * P.muH) / rho;
    default: return expf(t * logf(P.muH) + (1.0f - t) * logf(P.muL)) / rho;
  }
}

// phi from phi* = sum g: identity for Fakhari2017/Liang2014; for
// Chai2018/Hu2019 phi = phi* + (1 - lambda) R(phi*)/2 (Eq. chai2018_phi_update,
// evaluated at phi*).
template <int FAM>
__device__ __forceinline__ float nonlocal_R(const DevParams& P, float ps, float gamma) {
  return P.M * (-P.four_beta_over_kappa * (ps - P.phiH) * (ps - P.phiL) * (ps - P.phi0) +
                gamma * (P.phiH - ps) * (ps - P.phiL));
}
template <int FAM>
__device__ __forceinline__ float finish_phi(const DevParams& P, float ps, float gamma) {
  if constexpr (FAM == FAM_CHAI) return ps + 0.5f * nonlocal_R<FAM>(P, ps, gamma);
  else if constexpr (FAM == FAM_HU) return ps + 0.5f * (1.0f - P.lambda) * nonlocal_R<FAM>(P, ps, gamma);
  else return ps;
}

// phi* = sum_a g_a (mirror-exact; the D3Q7 rest slot of the Allen-Cahn
// families is identically zero and left out).
template <typename LG, bool NO_REST, typename V>
__device__ __forceinline__ float phi_star(const V& g) {
  if constexpr (NO_REST) return Sym<LG>::moving(g);
  else return g[0] + Sym<LG>::moving(g);
}

// ---------------------------------------------------------------------------
// Collision of one cell. Inputs: pre-collision g, f; phi, phi*, grad phi,
// lap phi (and for Cahn-Hilliard mu, lap mu, phi*u of the previous step).
// Outputs: post-collision g*, f*, u, p, rho.
// ---------------------------------------------------------------------------
template <int FAM, int DIM, int LAT = 0>
struct Cell {
  using LG = typename Lattices<DIM, LAT>::G;
  using LF = typename Lattices<DIM, LAT>::F;
  static constexpr int QG = LG::Q, QF = LF::Q;
  // Size of the MRT work array: 27 on D3Q27 (the collision has an MRT form), 1 otherwise.
  static constexpr int MRT_Q = (QF == 27) ? 27 : 1;

  // Liu2023 is Liang2018 with the local weight lamx of its G (Eq. Liu_G).
  static constexpr bool L18 = (FAM == FAM_LIANG18 || FAM == FAM_LIU);

  __device__ __forceinline__ static void collide(
      const DevParams& P, float (&g)[QG], float (&f)[QF], float phi, float phis,
      const float (&gp)[DIM], float lp, float mu_in, float lmu, float (&phiu)[DIM],
      float gamma, float (&u)[DIM], float& rho, float& p, float lamx = 1.0f) {
    constexpr float cs2 = 1.0f / 3.0f;
    rho = P.rhoL + P.drho_dphi * (phi - P.phiL);
    const float nu = viscosity(P, phi, rho);
    const float itau = 1.0f / (3.0f * nu + 0.5f);
    const float fw = 1.0f - 0.5f * itau;
    const float inv_rho = 1.0f / rho;
    float grho[DIM], Fs[DIM], Fb[DIM], mom[DIM];
    const float sum_nz = Sym<LF>::moving(f);
    const float sumf = f[0] + sum_nz;
#pragma unroll
    for (int k = 0; k < DIM; ++k) mom[k] = Sym<LF>::first(f, k);
    const float mu = (FAM == FAM_LIANG) ? mu_in
        : P.beta4 * (phi - P.phiH) * (phi - P.phiL) * (phi - P.phi0) - P.kappa * lp;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      grho[k] = P.drho_dphi * gp[k];
      Fs[k] = mu * gp[k];
      Fb[k] = rho * P.grav[k] + P.fdens[k];
    }
    const float A = P.lundA;
    float F[DIM];

    if constexpr (L18) {
      // Liang2018: rho u = sum e f + F/2 with F = F_s + F_b (Eq.
      // liang_velocity_update); the linear forcing A rho u is solved for.
      const float den = inv_rho / (1.0f - 0.5f * A);
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        u[k] = (mom[k] + 0.5f * (Fs[k] + Fb[k])) * den;
        F[k] = Fs[k] + Fb[k] + A * rho * u[k];
      }
    } else if constexpr (FAM != FAM_LIANG) {
      // Pressure p = rho c_s^2 sum f (Eq. fakhari_p_update); F_p = -(p/rho) grad rho.
      p = rho * cs2 * sumf;
      float Fo[DIM];
      const float inv_1mA = 1.0f / (1.0f - 0.5f * A);
#pragma unroll
      for (int k = 0; k < DIM; ++k) Fo[k] = Fs[k] + Fb[k] - cs2 * sumf * grho[k];
      if (P.drho_dphi != 0.0f) {
        // F_mu = nu [grad u + grad u^T] . grad rho with the strain rate from the
        // local non-equilibrium second moment (Reading R3):
        // S_ij = -3 (Pi_ij - sum f/3 d_ij - u'_i u'_j) / tau.
        float u1[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) u1[k] = (mom[k] + 0.5f * inv_rho * Fo[k]) * inv_1mA;
        float Pi[DIM][DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = i; j < DIM; ++j) Pi[i][j] = Sym<LF>::second(f, i, j);
        const float c = -3.0f * nu * itau;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          float s = 0.0f;
#pragma unroll
          for (int j = 0; j < DIM; ++j) {
            const float pij = (i <= j ? Pi[i][j] : Pi[j][i]) - (i == j ? cs2 * sumf : 0.0f) - u1[i] * u1[j];
            s += pij * grho[j];
          }
          Fo[i] += c * s;
        }
      }
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        u[k] = (mom[k] + 0.5f * inv_rho * Fo[k]) * inv_1mA;  // Eq. (fakhari_velocity_update)
        F[k] = Fo[k] + A * rho * u[k];
      }
    } else {
      // Liang2014: u from Eq. (liang2014_velocity_update); F_a = drho/dphi div(M grad mu) u.
      const float acoef = P.drho_dphi * P.M * lmu;
      const float den = 1.0f / (rho - 0.5f * acoef - 0.5f * A * rho);
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        u[k] = (mom[k] + 0.5f * (Fs[k] + Fb[k])) * den;
        F[k] = Fs[k] + Fb[k] + (acoef + A * rho) * u[k];
      }
    }
    float usq = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) usq += u[k] * u[k];

    // ---------------- phase field ----------------
    // Equilibria whose zeroth moment is phi carry it exactly: where the rest
    // population is stored it is phi minus the moving ones; weights multiply
    // as hi + lo pairs (wmul), so no moment carries the bias of the FP32
    // weights.
    constexpr bool REST = (LG::w(0) > 0.0f) || (FAM == FAM_LIANG);
    float geq[QG], G[QG];
    if constexpr (FAM == FAM_LIANG) {
      // Eq. (liang2_geq) and Eq. (liang2_G) with the backward-Euler d_t(phi u).
      const float emu = P.eta * mu;
      float pu[DIM], dpu[DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        pu[k] = phi * u[k];
        dpu[k] = pu[k] - phiu[k];
        phiu[k] = pu[k];
      }
      geq[0] = 0.0f;
      G[0] = 0.0f;
#pragma unroll
      for (int q = 1; q < QG; ++q) {
        float epu = 0.0f, edpu = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (ecomp<LG>(q, k) != 0) {
            epu += (float)ecomp<LG>(q, k) * pu[k];
            edpu += (float)ecomp<LG>(q, k) * dpu[k];
          }
        geq[q] = wmul<LG>(q, emu + 3.0f * epu);
        G[q] = wmul<LG>(q, 3.0f * edpu);
      }
      geq[0] = phi - Sym<LG>::moving(geq);   // = phi + (w_0 - 1) eta mu
    } else {
      float flux[DIM];
      constexpr bool has_cons = (FAM == FAM_FAKHARI || FAM == FAM_HU || L18);
      if (has_cons) {
        // Conservative counter term, Eq. (fakhari_G_modified), with the
        // normal regularised as grad phi / sqrt(|grad phi|^2 + eps^2) (R6).
        float g2 = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) g2 += gp[k] * gp[k];
        const float sc = P.counter_k * (P.phiH - phi) * (phi - P.phiL) * rsqrtf(g2 + P.eps2);
#pragma unroll
        for (int k = 0; k < DIM; ++k) flux[k] = sc * gp[k];
      }
      // Liang2018: backward-Euler d_t(phi u) (Sec. III B) for Eq. (liang_G_final).
      float dpu[DIM];
      if constexpr (L18) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          const float pu = phi * u[k];
          dpu[k] = pu - phiu[k];
          phiu[k] = pu;
        }
      }
      float Rw = 0.0f, lam = 1.0f;
      if constexpr (FAM == FAM_CHAI || FAM == FAM_HU) {
        Rw = nonlocal_R<FAM>(P, phis, gamma);
        if constexpr (FAM == FAM_HU) { lam = P.lambda; Rw *= (1.0f - lam); }
      }
      if constexpr (FAM == FAM_LIU) {
        lam = lamx;
        Rw = (1.0f - lam) * nonlocal_R<FAM>(P, phis, gamma);
      }
      geq[0] = 0.0f;
      G[0] = 0.0f;
#pragma unroll
      for (int q = 1; q < QG; ++q) {
        float eu = 0.0f, ef = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (ecomp<LG>(q, k) != 0) {
            eu += (float)ecomp<LG>(q, k) * u[k];
            if constexpr (has_cons) ef += (float)ecomp<LG>(q, k) * flux[k];
            if constexpr (L18) ef += (float)ecomp<LG>(q, k) * (3.0f * dpu[k]);
          }
        if constexpr (FAM == FAM_FAKHARI)
          geq[q] = wmul<LG>(q, phi * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * usq));  // Eq. (fakhari_geq)
        else
          geq[q] = wmul<LG>(q, phi * (1.0f + 3.0f * eu));                   // Eqs. (Chai_geq), (liang_geq)
        if constexpr (FAM == FAM_FAKHARI || FAM == FAM_LIANG18) G[q] = wmul<LG>(q, ef);  // Eq. (liang_G_final)
        else if constexpr (FAM == FAM_CHAI) G[q] = wmul<LG>(q, Rw);
        else G[q] = wmul<LG>(q, lam * ef + Rw);                          // Eqs. (Hu_G), (Liu_G)
      }
      if constexpr (REST) {
        geq[0] = phi - Sym<LG>::moving(geq);
        if constexpr (FAM == FAM_CHAI || FAM == FAM_HU || FAM == FAM_LIU) G[0] = wmul<LG>(0, Rw);
      }
      if constexpr (FAM == FAM_FAKHARI && QG == 7) {
        // D3Q7 has no rest population to absorb the rounding of the
        // second-order equilibrium (w_0 = 0), and the FP32 terms
        // 4.5 (e.u)^2 - 1.5 u.u of the six did not sum to zero: phi drifted
        // by ~3e-9 per step. The z pair takes the even part that makes the
        // six sum to phi (one rounding), h = (phi - x and y pairs) / 2, and
        // keeps its odd part w phi 3 u_z; exact arithmetic gives the same
        // values, and every reflection still maps the update onto itself.
        const float S = (geq[1] + geq[2]) + (geq[3] + geq[4]);
        const float h = 0.5f * (phi - S);
        const float o = wmul<LG>(5, phi * (3.0f * u[DIM - 1]));
        geq[5] = h + o;
        geq[6] = h - o;
      }
    }
#pragma unroll
    for (int q = 0; q < QG; ++q) g[q] = g[q] - (g[q] - geq[q]) * P.inv_tau_phi + P.src_w_phi * G[q];

    // ---------------- hydrodynamics ----------------
    if constexpr (fam_phiu(FAM)) {
      // p by Eq. (liang_p_update); pressure-based f_eq (Eqs. liang2_feq,
      // liang_feq) and forcing of Eqs. (liang2_F), (Gamma_beta) for Liang2014,
      // of Eq. (liang_F_final) for Liang2018.
      float udg = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) udg += u[k] * grho[k];
      // 3p = X / (1 - w_0) with 1 - w_0 = 5/9 (D2Q9) or 2/3 (D3Q19), formed
      // without a biased FP32 constant so the p -> f_eq -> p round trip is
      // unbiased.
      const float Xp = sum_nz + 0.5f * udg - wmul<LF>(0, rho * 1.5f * usq);
      // 1 - w_0 = 5/9 (D2Q9), 2/3 (D3Q19), 19/27 (D3Q27)
      const float p3 = (LF::Q == 9) ? (Xp * 9.0f) / 5.0f : (LF::Q == 19 ? Xp * 1.5f : (Xp * 27.0f) / 19.0f);
      p = p3 / 3.0f;
      float uF = 0.0f, ua = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        uF += u[k] * F[k];
        ua += u[k] * cs2 * grho[k];
      }
      float nq[MRT_Q];   // f - f_eq + F_b/2 (MRT, D3Q27)
#pragma unroll
      for (int q = 0; q < QF; ++q) {
        float eu = 0.0f, eF = 0.0f, ea = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (ecomp<LF>(q, k) != 0) {
            const float e = (float)ecomp<LF>(q, k);
            eu += e * u[k];
            eF += e * F[k];
            ea += e * cs2 * grho[k];
          }
        const float Gam = wmul<LF>(q, 3.0f * eu + 4.5f * eu * eu - 1.5f * usq);
        const float feq = (q == 0) ? wmul<LF>(q, p3) - p3 + wmul<LF>(q, rho * (-1.5f * usq))
                                   : wmul<LF>(q, p3) + rho * Gam;
        float Fq;
        if constexpr (FAM == FAM_LIANG)
          Fq = 3.0f * ((ea - ua) * Gam + (eF - uF) * Gam + wmul<LF>(q, eF - uF));
        else
          // w [u.grad rho + 3 e.F + 3 ((e.u)(e.grad rho) - c_s^2 u.grad rho)]: the
          // u.grad rho terms cancel, leaving w (3 e.F + 3 (e.u)(e.grad rho)),
          // with ea = c_s^2 e.grad rho.
          Fq = wmul<LF>(q, 3.0f * eF + 9.0f * eu * ea);
        if constexpr (MRT_Q == QF) nq[q] = (f[q] - feq) + 0.5f * Fq;
        f[q] = f[q] - (f[q] - feq) * itau + fw * Fq;
      }
      if constexpr (MRT_Q == QF)
        if (P.mrt) mrt_correct(f, nq, itau, P.mrt_sb, P.mrt_sh);
    } else {
      // f* = f - (f - f_eq) itau + fw F_b = f (1 - itau) + w (itau X + fw Y), with
      // f_eq = w X, X = sum f + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u   Eq. (fakhari_feq),
      // F_b = w Y, Y = 3 e.F~ (Eq. fakhari_F) or
      //       3 e.F~ + 9 (e.u)(e.F~) - 3 u.F~ (Eq. chai_F, Reading R2), F~ = F/rho.
      // A velocity and its opposite share everything but the sign of e: with
      // e.u and e.F~ of the first, itau X + fw Y = E + O for it and E - O for
      // the opposite, E = itau (sum f - 1.5 u.u + 4.5 (e.u)^2) + fw Y_even,
      // O = 3 (itau e.u + fw e.F~). Every operation is sign-symmetric, so the
      // mirror image of a cell still gets the mirror image of its update.
      float Ft[DIM], uFt = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        Ft[k] = F[k] * inv_rho;
        uFt += u[k] * Ft[k];
      }
      const float s0 = sumf - 1.5f * usq;
      const float omi = 1.0f - itau;
      const float itau3 = 3.0f * itau, fw3 = 3.0f * fw;
      const float ye0 = (FAM == FAM_FAKHARI) ? 0.0f : -3.0f * uFt;   // even part of Y at e = 0
      // MRT (D3Q27): n = f - f_eq + F_b/2 = f - w (X - Y/2), collected before the update.
      float nq[MRT_Q];
      if constexpr (MRT_Q == QF) nq[0] = f[0] - wmul<LF>(0, s0 - 0.5f * ye0);
      f[0] = fmaf(f[0], omi, wmul<LF>(0, fmaf(itau, s0, fw * ye0)));
#pragma unroll
      for (int q = 1; q < QF; ++q) {
        const int qo = LF::opp(q);
        if (qo < q) continue;   // each pair once, from its first member
        float eu = 0.0f, eF = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (ecomp<LF>(q, k) != 0) {
            const float e = (float)ecomp<LF>(q, k);
            eu += e * u[k];
            eF += e * Ft[k];
          }
        float E;
        if constexpr (FAM == FAM_FAKHARI) E = itau * fmaf(4.5f * eu, eu, s0);
        else E = fmaf(itau, fmaf(4.5f * eu, eu, s0), fw * fmaf(9.0f * eu, eF, ye0));
        const float O = fmaf(itau3, eu, fw3 * eF);
        if constexpr (MRT_Q == QF) {
          // X - Y/2 = (s0 + 4.5 (e.u)^2 - Y_even/2) +- (3 e.u - 1.5 e.F~)
          const float xe = fmaf(4.5f * eu, eu, s0) - ((FAM == FAM_FAKHARI) ? 0.0f : 0.5f * fmaf(9.0f * eu, eF, ye0));
          const float xo = fmaf(3.0f, eu, -1.5f * eF);
          nq[q] = f[q] - wmul<LF>(q, xe + xo);
          nq[qo] = f[qo] - wmul<LF>(qo, xe - xo);
        }
        f[q] = fmaf(f[q], omi, wmul<LF>(q, E + O));
        f[qo] = fmaf(f[qo], omi, wmul<LF>(qo, E - O));
      }
      if constexpr (MRT_Q == QF)
        if (P.mrt) mrt_correct(f, nq, itau, P.mrt_sb, P.mrt_sh);
    }
  }
};

// Number of velocities of a lattice with e_x != 0 (their odd-step f reads
// cross the tile's x edge).
template <typename L>
__host__ __device__ constexpr int nsx() {
  int n = 0;
  for (int q = 0; q < L::Q; ++q) n += L::ex(q) != 0 ? 1 : 0;
  return n;
}

// Rank of velocity q among those with e_x != 0.
template <typename L>
__host__ __device__ constexpr int side_rank(int q) {
  int n = 0;
  for (int a = 0; a < q; ++a) n += L::ex(a) != 0 ? 1 : 0;
  return n;
}

// Number of 16-byte f chunks a block stages per plane (cooperative staging):
// per velocity and tile row TA / CE chunks, one more on odd steps where e_x != 0.
template <typename LF, int PAR, int TB, int NCH0>
__host__ __device__ constexpr int coop_items() {
  int n = 0;
  for (int q = 0; q < LF::Q; ++q) n += TB * (NCH0 + ((PAR == 1 && LF::ex(q) != 0) ? 1 : 0));
  return n;
}

// ---------------------------------------------------------------------------
// Shared-memory footprint of one tile march.
// ---------------------------------------------------------------------------
template <int FAM, int DIM, typename T, int TA, int TB, bool COOP = false, int LAT = 0, bool TMA = false, int PAR = 0>
struct TileSmem {
  static constexpr bool CH = (FAM == FAM_LIANG);
  static constexpr int H = CH ? 2 : 1;
  static constexpr int HB = (DIM == 3) ? H : 0;
  static constexpr int NT = TA * TB;
  static constexpr int PLANE = (TA + 2 * H) * (TB + 2 * HB);
  static constexpr int NSLOT = CH ? 8 : 4;
  static constexpr int PHI = NSLOT * PLANE;
  static constexpr int MU = CH ? 4 * (TA + 2) * (TB + 2 * ((DIM == 3) ? 1 : 0)) : 1;
  // The populations of the next planes are staged asynchronously: NST stages
  // of f and g (Q_g words per cell of the tile and halo); a 16-bit g is
  // staged as the aligned 32-bit word holding it. f is staged either per
  // thread (Q_f words per cell) or, with COOP, by the whole block in 16-byte
  // chunks: per velocity and tile row, TA + CE elements of the storage type
  // (CE = 16 bytes of elements; the extra chunk holds the neighbour cell an
  // odd AA step reads across the tile's x edge).
  static constexpr bool STAGED = true;
  static constexpr int CE = 16 / (int)sizeof(T);
  static constexpr int FROW = TA + CE;
  static constexpr int FST = COOP ? Lattices<DIM, LAT>::F::Q * TB * FROW * (int)sizeof(T) / 4
                                  : Lattices<DIM, LAT>::F::Q * NT;
  static constexpr int GST = Lattices<DIM, LAT>::G::Q * PLANE;
  // COOP refills a stage only after the next plane's barrier, so a fourth
  // stage keeps one more plane in flight. The FP32 tiles take three stages
  // instead, which lets one more block fit per SM (D3Q19: four blocks of 53
  // KB, 16 warps, 24.96 -> 25.27 GLUPS at 512^3; D3Q27: three of 67 KB);
  // Cahn-Hilliard tiles have no room for a fourth stage.
  static constexpr int NST = (COOP && !CH && sizeof(T) < 4) ? 4 : 3;
  // TMA staging (3D, rows aligned to the population blocks, Allen-Cahn
  // halo): NST stages in the box layout of TmaStage, 128-byte aligned (plus
  // 128 bytes of slack to align the dynamic base), then NST mbarriers.
  using TS = TmaStage<TB, (DIM == 3 && !CH) ? Lattices<DIM, LAT>::G::Q - 1 : Lattices<DIM, LAT>::G::Q,
                      Lattices<DIM, LAT>::F::Q, nsx<typename Lattices<DIM, LAT>::F>(), (int)sizeof(T), PAR>;
  // TMA: the stages, 128 bytes of alignment slack, NST stage barriers and
  // one barrier of the wait-timeout test hook
  static constexpr int STAGE = TMA ? (NST * TS::BYTES + 128 + 8 * (NST + 1)) / 4 : (STAGED ? NST * (FST + GST) : 0);
  static_assert(!COOP || (FST % 4 == 0 && GST % 4 == 0), "16-byte aligned stages");
  static constexpr size_t BYTES = (size_t)(STAGE + PHI + MU) * sizeof(float);
};

// ---------------------------------------------------------------------------
// One tile: the cells [a0, a0+TA) x [b0, b0+TB) marched over planes
// [c0, min(c0+chunk, NC)) of the slow axis. Called by the single-domain
// kernel (one tile per block) and by the persistent batch kernel (tiles of
// many domains claimed in turn). Accumulates the observables into obs.
// ---------------------------------------------------------------------------
template <int FAM, int DIM, typename T, int TA, int TB, int PAR = -1, int ROW = -1, int LAT = 0, bool TMA = false>
__device__ __forceinline__ void step_tile(const StepArgs& args, int a0, int b0, int c0, int chunk,
                                          float* __restrict__ s_phi, float* __restrict__ s_mu,
                                          float* __restrict__ s_stage, ObsPartial& obs,
                                          const TmaMaps* tm = nullptr) {
  using LG = typename Lattices<DIM, LAT>::G;
  using LF = typename Lattices<DIM, LAT>::F;
  using LS = typename Lattices<DIM, LAT>::S;
  constexpr int QG = LG::Q, QF = LF::Q, QS = LS::Q;
  constexpr int NT = TA * TB;
  constexpr bool CH = (FAM == FAM_LIANG);
  constexpr int H = CH ? 2 : 1;                 // phi halo
  constexpr int HB = (DIM == 3) ? H : 0;
  constexpr int RA = TA + 2 * H, RB = TB + 2 * HB, PLANE = RA * RB;
  constexpr int NSLOT = CH ? 8 : 4;             // power of two >= 2H + 2
  constexpr int NHALO = PLANE - NT;
  constexpr int KH = (NHALO + NT - 1) / NT;
  constexpr int MHB = (DIM == 3) ? 1 : 0;       // mu region halo (CH)
  constexpr int MRA = TA + 2, MRB = TB + 2 * MHB, MPLANE = MRA * MRB;
  constexpr int MSLOT = 4;
  constexpr int MHALO = MPLANE - NT;
  constexpr int KM = (MHALO + NT - 1) / NT;
  // COOP: the block stages f together in 16-byte chunks (3D, rows aligned to
  // the population blocks, AA parity known at compile time).
  constexpr bool COOP = (DIM == 3) && (ROW == 1) && (PAR >= 0);
  // TMA: the block-staged geometry with its copies made by the tensor
  // memory accelerator (the host guarantees ny % TB == 0 for it).
  constexpr bool TMAS = TMA && COOP && !CH && TA == 32;
  static_assert(!TMA || TMAS, "TMA staging needs the row-aligned 3D Allen-Cahn tile");
  using SMEM = TileSmem<FAM, DIM, T, TA, TB, COOP, LAT, TMAS, (PAR == 1 ? 1 : 0)>;
  constexpr bool STAGED = SMEM::STAGED;
  constexpr int FST = SMEM::FST, GST = SMEM::GST;
  constexpr int NST = SMEM::NST;
  constexpr int CE = SMEM::CE, FROW = SMEM::FROW;
  constexpr bool SKIP0 = (DIM == 3 && !CH);   // D3Q7 rest slot of the AC families: w_0 = 0, g_0 = 0
  (void)RB;

  const DevParams& P = args.p;
  const int NA = P.nx, NB = (DIM == 3) ? P.ny : 1, NC = (DIM == 3) ? P.nz : P.ny;
  // Element offsets into one population array, q*N + cell, fit in 32 bits
  // (the host rejects Q*N >= 2^32).
  const unsigned N = (unsigned)args.N;
  const int NAB = NA * NB;
  const int c1 = min(c0 + chunk, NC);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TA * ty;
  const int a = a0 + tx, b = b0 + ty;
  const bool active = (a < NA) && (b < NB);
  const bool walls = DIM == 2 && P.walls != 0;   // walls are a 2D feature
  // AA parity of this step: a compile-time constant for the single-domain
  // kernel (one instantiation per parity), read from the arguments otherwise.
  const int parity = PAR >= 0 ? PAR : args.parity;

  float gamma = 0.0f;
  if constexpr (FAM == FAM_CHAI || FAM == FAM_HU) {
    const double I2 = args.gamma_acc[1];
    gamma = (I2 != 0.0) ? (float)(args.gamma_acc[0] / I2) : 0.0f;
  }

  const T* gsrc = static_cast<const T*>(args.g_src);
  T* gdst = static_cast<T*>(args.g_dst);
  T* fb = static_cast<T*>(args.f);

  // Ring cells of this thread: its own cell and KH halo cells (constant
  // across the march). Offsets are wrapped (a, b) linear offsets.
  const int own_ab = wrap_mod(a, NA) + NA * wrap_mod(b, NB);
  const int own_slot = (ty + HB) * RA + (tx + H);
  int halo_ab[KH], halo_pos[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    int hk = tid + k * NT;
    halo_pos[k] = -1;
    halo_ab[k] = 0;
    if (hk < NHALO) {
      int ra, rb;
      if (hk < HB * RA) { rb = hk / RA; ra = hk % RA; }
      else {
        hk -= HB * RA;
        if (hk < HB * RA) { rb = HB + TB + hk / RA; ra = hk % RA; }
        else {
          hk -= HB * RA;
          rb = HB + hk / (2 * H);
          const int j = hk % (2 * H);
          ra = (j < H) ? j : TA + j;
        }
      }
      halo_pos[k] = rb * RA + ra;
      halo_ab[k] = wrap_mod(a0 - H + ra, NA) + NA * wrap_mod(b0 - HB + rb, NB);
    }
  }

  // Plane index along the marching axis: periodic wrap, or mirror at walls.
  auto map_c = [&](int c) -> int {
    if (walls) {
      if (c < 0) return -1 - c;
      if (c >= NC) return 2 * NC - 1 - c;
      return c;
    }
    return wrap_mod(c, NC);
  };

  auto load_g = [&](unsigned idx, float (&gv)[QG]) -> float {
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      if (DIM == 3 && !CH && q == 0) { gv[q] = 0.0f; continue; }  // D3Q7 rest slot: w_0 = 0, g_0 = 0
      gv[q] = pop_load<T, LG>(gsrc + pop_ix<LG>(q, idx), q, P.gref);
    }
    return phi_star<LG, (DIM == 3 && !CH)>(gv);
  };

  auto ring = [&](int c) -> float* { return s_phi + (c & (NSLOT - 1)) * PLANE; };

  // Compute phi of logical plane c into ring slot; keep the own cell's g.
  auto produce = [&](int c, float (&gown)[QG]) {
    const unsigned pofs = (unsigned)(NAB * map_c(c));
    float* slot = ring(c);
    const float ps = load_g(own_ab + pofs, gown);
    slot[own_slot] = finish_phi<FAM>(P, ps, gamma);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      if (halo_pos[k] >= 0) {
        float tmp[QG];
        const float hs = load_g(halo_ab[k] + pofs, tmp);
        slot[halo_pos[k]] = finish_phi<FAM>(P, hs, gamma);
      }
    }
  };

  // Value at stencil offset q around ring position pos, with the three
  // plane pointers of c-1, c, c+1 (compile-time offsets after unrolling).
  auto ring_nb = [&](const float* pm, const float* p0, const float* pp, int pos, int q) -> float {
    const int dc = dc_of<DIM, LS>(q);
    const float* pl = dc < 0 ? pm : (dc > 0 ? pp : p0);
    return pl[pos + db_of<DIM, LS>(q) * RA + da_of<DIM, LS>(q)];
  };

  // Cahn-Hilliard: mu of logical plane c over the tile + 1 region.
  auto make_mu = [&](int c) {
    float* mslot = s_mu + (c & (MSLOT - 1)) * MPLANE;
    const float *pm = ring(c - 1), *p0 = ring(c), *pp = ring(c + 1);
    auto one = [&](int ma, int mb) {
      const int pos = (mb + HB - MHB) * RA + (ma + H - 1);
      const float pc = p0[pos];
      float nb[QS];
      nb[0] = pc;
#pragma unroll
      for (int q = 1; q < QS; ++q) nb[q] = ring_nb(pm, p0, pp, pos, q);
      const float lap = Sym<LS>::lap(nb, pc);
      mslot[mb * MRA + ma] = P.beta4 * (pc - P.phiH) * (pc - P.phiL) * (pc - P.phi0) - P.kappa * lap;
    };
    one(tx + 1, ty + MHB);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      int hk = tid + k * NT;
      if (hk < MHALO) {
        int ma, mb;
        if (hk < MHB * MRA) { mb = hk / MRA; ma = hk % MRA; }
        else {
          hk -= MHB * MRA;
          if (hk < MHB * MRA) { mb = MHB + TB + hk / MRA; ma = hk % MRA; }
          else {
            hk -= MHB * MRA;
            mb = MHB + hk / 2;
            ma = (hk % 2 == 0) ? 0 : TA + 1;
          }
        }
        one(ma, mb);
      }
    }
  };

  // Own-cell neighbour coordinates along the fast axes (constant).
  const int aw = (a < NA) ? a : 0, bw = (b < NB) ? b : 0;
  const int am = aw == 0 ? NA - 1 : aw - 1, ap = aw == NA - 1 ? 0 : aw + 1;
  const int bm = bw == 0 ? NB - 1 : bw - 1, bp = bw == NB - 1 ? 0 : bw + 1;
  const int rbm = bm * NA, rbw = bw * NA, rbp = bp * NA;
  auto A_of = [&](int d) { return d < 0 ? am : (d > 0 ? ap : aw); };
  auto RB_of = [&](int d) { return d < 0 ? rbm : (d > 0 ? rbp : rbw); };

  // Element offsets in the block layout (pop_ix): population q of a cell
  // sits 32 q elements after its population 0, so every access below forms
  // one pointer per cell (population 0) and reaches the populations by
  // compile-time offsets. When nx is a multiple of the block width, shifting
  // a cell by whole rows or planes moves its population 0 by a multiple of
  // the block stride, so the population-0 offset of the neighbour
  // (x + da, y + db) on plane cs is
  //   E0 + D_x(da) + D_y(db) + cs * Q * nx * ny
  // with per-thread constants E0, D_x, D_y (periodic wrap included).
  // Otherwise the cell index is formed and mapped (pop_ix) per cell.
  // ROW: 1 = nx is a multiple of the block width, 0 = it is not, -1 = test here.
  const bool rowal = ROW >= 0 ? ROW == 1 : (NA % (int)kPopBlock) == 0;
  const unsigned cell0 = (unsigned)(aw + rbw);
  const unsigned fE0 = pop_ix<LF>(0, cell0), gE0 = pop_ix<LG>(0, cell0);
  const unsigned fdxm = pop_ix<LF>(0, (unsigned)(am + rbw)) - fE0, fdxp = pop_ix<LF>(0, (unsigned)(ap + rbw)) - fE0;
  const unsigned fdym = pop_ix<LF>(0, (unsigned)(aw + rbm)) - fE0, fdyp = pop_ix<LF>(0, (unsigned)(aw + rbp)) - fE0;
  const unsigned gdxm = pop_ix<LG>(0, (unsigned)(am + rbw)) - gE0, gdxp = pop_ix<LG>(0, (unsigned)(ap + rbw)) - gE0;
  const unsigned gdym = pop_ix<LG>(0, (unsigned)(aw + rbm)) - gE0, gdyp = pop_ix<LG>(0, (unsigned)(aw + rbp)) - gE0;
  const unsigned fplane = (unsigned)NAB * (unsigned)QF, gplane = (unsigned)NAB * (unsigned)QG;
  // Population 0 of the cell (x + da, y + db) on plane cs (cs already wrapped).
  auto f_cell = [&](int da, int db, int cs) -> unsigned {
    if (rowal)
      return fE0 + (da < 0 ? fdxm : (da > 0 ? fdxp : 0u)) + (db < 0 ? fdym : (db > 0 ? fdyp : 0u)) +
             (unsigned)cs * fplane;
    return pop_ix<LF>(0, (unsigned)(A_of(da) + RB_of(db) + cs * NAB));
  };
  auto g_cell = [&](int da, int db, int cs) -> unsigned {
    if (rowal)
      return gE0 + (da < 0 ? gdxm : (da > 0 ? gdxp : 0u)) + (db < 0 ? gdym : (db > 0 ? gdyp : 0u)) +
             (unsigned)cs * gplane;
    return pop_ix<LG>(0, (unsigned)(A_of(da) + RB_of(db) + cs * NAB));
  };
  // Plane reached from c by dc (periodic, or c itself at a wall).
  auto plane_of = [&](int c, int dc) -> int {
    return dc < 0 ? (c == 0 ? NC - 1 : c - 1) : (dc > 0 ? (c == NC - 1 ? 0 : c + 1) : c);
  };
  // AA pattern, f population q the own cell reads at plane c: even steps its
  // own slot q; odd steps slot opp(q) of x - e_q, or its own slot q where
  // x - e_q lies beyond a wall.
  auto f_read_crosses = [&](int c, int dc) { return walls && ((dc > 0 && c == 0) || (dc < 0 && c == NC - 1)); };
  // Own and halo g of plane cm (mapped): the halo cells' offsets relative to
  // their plane are per-thread constants in the row-aligned case.
  unsigned gHalo0[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) gHalo0[k] = pop_ix<LG>(0, (unsigned)halo_ab[k]);
  const unsigned gOwn0 = pop_ix<LG>(0, (unsigned)own_ab);
  auto g_src_cell = [&](int k, int cm) -> unsigned {   // k < 0: own cell
    if (rowal) return (k < 0 ? gOwn0 : gHalo0[k]) + (unsigned)cm * gplane;
    return pop_ix<LG>(0, (unsigned)((k < 0 ? own_ab : halo_ab[k]) + NAB * cm));
  };

  // The incoming g of plane cg (own cell and this thread's halo cells) and
  // the own cell's f of plane cf are copied asynchronously into this
  // thread's slots of stage s a plane before they are used. Each thread
  // reads back only its own slots, so completing its own copies
  // (cp.async.wait_group) is all the synchronisation needed. cp.async moves
  // at least 4 aligned bytes: a 16-bit population is fetched as the aligned
  // word that contains it (its neighbour's half is ignored; the arrays are
  // allocated with padding so the last word is in bounds), and a bit of
  // gm/fm records which half is ours. Populations of one cell are 32
  // elements apart, an even count, so they all sit in the same half.
  constexpr bool WIDE = sizeof(T) == 4;
  constexpr long long TSZ = (long long)sizeof(T);
  constexpr long long PSTRIDE = (long long)kPopBlock * TSZ;   // bytes between populations of a cell
  static_assert((1 + KH) * QG <= 32, "half-select bits of the staged g");
  auto stage_f = [&](int s) { return s_stage + s * (FST + GST); };
  auto stage_g = [&](int s) { return s_stage + s * (FST + GST) + FST; };
  const unsigned s_stage_u32 = (unsigned)__cvta_generic_to_shared(s_stage);
  // Address of the aligned word holding element e of base; its half in hb.
  auto word_at = [&](const T* base, unsigned e, unsigned& hb) -> const void* {
    if constexpr (WIDE) {
      hb = 0u;
      return base + e;
    } else {
      hb = e & 1u;
      return base + (e & ~1u);
    }
  };
  // COOP f items: the stage of one plane is QF x TB rows of FROW elements;
  // row (q, r) holds the slot f reads for velocity q on tile row r, chunk j
  // (CE elements) at element CE j. Even steps read the own cells (slot q);
  // odd steps slot opp(q) of x - e_q, so a velocity with e_x != 0 needs one
  // cell beyond the tile: for e_x = +1 the row starts at x0 - CE, otherwise
  // at x0, and it has TA / CE + 1 chunks. Items are numbered velocity-major
  // and dealt to the threads in turn; each thread keeps its items' element
  // offsets (plane term excluded, z neighbour included) and stage offsets.
  constexpr int NCH0 = TA / CE;
  constexpr int NFI = coop_items<LF, PAR, TB, NCH0>();
  constexpr int KF = (COOP && !TMAS) ? (NFI + NT - 1) / NT : 1;
  unsigned fsrc[KF] = {}, fdst[KF] = {};
  unsigned fmz = 0u, fpz = 0u;   // items reading plane c - 1 / c + 1
  if constexpr (COOP && !TMAS) {
#pragma unroll
    for (int k = 0; k < KF; ++k) {
      fsrc[k] = 0u;
      fdst[k] = 0u;
      const int i = tid + k * NT;
      int base = 0;
      static_for<0, QF>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int nch = NCH0 + ((PAR == 1 && LF::ex(q) != 0) ? 1 : 0);
        if (i >= base && i < base + TB * nch) {
          const int r = (i - base) / nch, j = (i - base) % nch;
          constexpr int slot = PAR == 0 ? q : LF::opp(q);
          constexpr int dx = PAR == 0 ? 0 : -LF::ex(q), dy = PAR == 0 ? 0 : -LF::ey(q);
          constexpr int dz = PAR == 0 ? 0 : -LF::ez(q);
          const int x = wrap_mod(a0 + CE * j - (dx < 0 ? CE : 0), NA);
          const int y = wrap_mod(b0 + r + dy, NB);
          fsrc[k] = pop_ix<LF>(slot, (unsigned)(x + NA * y)) + (unsigned)(dz * (int)fplane);
          fdst[k] = (unsigned)(((q * TB + r) * FROW + CE * j) * (int)sizeof(T));
          if (dz < 0) fmz |= 1u << k;
          if (dz > 0) fpz |= 1u << k;
        }
        base += TB * nch;
      });
    }
  }

  auto issue = [&](int cg, int cf, int s, unsigned& gm, unsigned& fm) {
    gm = 0u;
    fm = 0u;
    const int cm = map_c(cg);
    const unsigned sg = s_stage_u32 + (unsigned)(s * (FST + GST) + FST + tid) * 4u;
    {
      unsigned hb;
      const void* w = word_at(gsrc, g_src_cell(-1, cm), hb);
      static_for<SKIP0 ? 1 : 0, QG>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cp_async4_at<q * PLANE * 4, q * PSTRIDE>(sg, w);
        gm |= hb << q;
      });
    }
    static_for<0, KH>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if (halo_pos[k] >= 0) {
        unsigned hb;
        const void* w = word_at(gsrc, g_src_cell(k, cm), hb);
        static_for<SKIP0 ? 1 : 0, QG>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          cp_async4_at<(q * PLANE + NT + k * NT) * 4, q * PSTRIDE>(sg, w);
          gm |= hb << ((1 + k) * QG + q);
        });
      }
    });
    if constexpr (COOP) {
      // The block's f chunks of plane cf (this thread's share, fixed per
      // thread; items that read plane cf -+ 1 wrap at the domain's z ends).
      const unsigned sf = s_stage_u32 + (unsigned)(s * (FST + GST)) * 4u;
      const unsigned cbase = (unsigned)cf * fplane;
      const bool zwrap = (cf == 0) || (cf == NC - 1);
      static_for<0, KF>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if ((k + 1) * NT <= NFI || tid + k * NT < NFI) {
          unsigned e = fsrc[k] + cbase;
          if (zwrap) {
            if (cf == 0 && ((fmz >> k) & 1u)) e += (unsigned)NC * fplane;
            if (cf == NC - 1 && ((fpz >> k) & 1u)) e -= (unsigned)NC * fplane;
          }
          cp_async16(sf + fdst[k], fb + e);
        }
      });
    } else if (active) {
      const unsigned sf = s_stage_u32 + (unsigned)(s * (FST + GST) + tid) * 4u;
      static_for<0, QF>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr int da = da_of<DIM, LF>(q), db = db_of<DIM, LF>(q), dc = dc_of<DIM, LF>(q);
        unsigned hb;
        if (parity == 0 || f_read_crosses(cf, dc)) {
          const void* w = word_at(fb, f_cell(0, 0, cf), hb);
          cp_async4_at<q * NT * 4, q * PSTRIDE>(sf, w);
        } else {
          const void* w = word_at(fb, f_cell(-da, -db, plane_of(cf, -dc)), hb);
          cp_async4_at<q * NT * 4, LF::opp(q) * PSTRIDE>(sf, w);
        }
        fm |= hb << q;
      });
    }
  };
  // Decode one staged population.
  auto staged = [&](float word, unsigned bits, int bit, int q, bool is_g) -> float {
    if constexpr (WIDE) {
      (void)bits;
      (void)bit;
      (void)q;
      (void)is_g;
      return word;
    } else {
      const unsigned hi = (bits >> bit) & 1u;
      return is_g ? pop_from_word<T, LG>(word, hi, q, P.gref) : pop_from_word<T, LF>(word, hi, q, 0.0f);
    }
  };
  // phi of logical plane c from stage s into the ring; keeps the own cell's g.
  auto produce_staged = [&](int c, int s, unsigned gm, float (&gown)[QG]) {
    const float* gs = stage_g(s);
    float* slot = ring(c);
#pragma unroll
    for (int q = 0; q < QG; ++q) gown[q] = (SKIP0 && q == 0) ? 0.0f : staged(gs[q * PLANE + tid], gm, q, q, true);
    slot[own_slot] = finish_phi<FAM>(P, phi_star<LG, SKIP0>(gown), gamma);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      if (halo_pos[k] >= 0) {
        float tmp[QG];
#pragma unroll
        for (int q = 0; q < QG; ++q)
          tmp[q] = (SKIP0 && q == 0) ? 0.0f : staged(gs[q * PLANE + NT + tid + k * NT], gm, (1 + k) * QG + q, q, true);
        slot[halo_pos[k]] = finish_phi<FAM>(P, phi_star<LG, SKIP0>(tmp), gamma);
      }
    }
  };

  // ------------------------------------------------------------------ TMA
  // Stage s holds plane c's g (the tile's rows and both halo rows; the x
  // halo in two side boxes) and its f, in the box layout of TmaStage; the
  // copies of stage s complete on barrier s. Warp 0 issues them, one box per
  // lane: item 0 the g main box, 1 and 2 the g side boxes, then the f boxes
  // (even steps: one box of every slot; odd steps: one box per velocity,
  // slot opp(q) of the rows shifted by -e_q, then one 16-byte side box per
  // velocity with e_x != 0). A box whose rows cross the domain's y edge is
  // zero-filled there by the TMA unit; the threads that need such a wrapped
  // row (a halo row of g, one row of f for e_y != 0) read it from global
  // memory instead.
  using TS = typename SMEM::TS;
  static_assert(!TMAS || TS::ALIGNED, "TMA boxes must land 128-byte aligned");
  constexpr int QGS = SKIP0 ? QG - 1 : QG;   // staged g slots (Q0 .. QG - 1)
  constexpr int Q0 = SKIP0 ? 1 : 0;
  constexpr int SL = TS::SL;
  constexpr int ES = (int)sizeof(T);
  constexpr int NITEMS = 3 + (PAR == 1 ? QF + nsx<LF>() : 1);
  constexpr int KI = TMAS ? (NITEMS + 31) / 32 : 1;
  unsigned tstage = 0u, tbar = 0u;   // shared addresses of stage 0 and barrier 0
  const char* tgen = nullptr;        // generic address of stage 0
  unsigned tphase = 0u;              // parity of each stage's next completion (bit s)
  bool tmo = false;                  // a bounded wait ran out
  int cstop = c1;
  int it_map[KI], it_c0[KI], it_c1[KI], it_dxb[KI], it_dy[KI], it_dz[KI], it_dst[KI];
  bool it_g[KI];
  int hoff[KH], hqs[KH];             // halo cell: byte offset of its first staged g slot, slot stride
  bool hglob[KH];                    // halo cell in a row beyond the y edge: read from global memory
  int own_goff = 0;
  const int NXB = NA / 32, xb0 = a0 / 32;
  if constexpr (TMAS) {
    tstage = (smem_u32(s_stage) + 127u) & ~127u;
    tbar = tstage + (unsigned)(NST * TS::BYTES);
    tgen = reinterpret_cast<const char*>(s_stage) + (tstage - smem_u32(s_stage));
    own_goff = TS::G_MAIN + ((ty + 1) * QGS * 32 + tx) * ES;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      hoff[k] = 0;
      hqs[k] = 0;
      hglob[k] = false;
      if (halo_pos[k] >= 0) {
        const int rb = halo_pos[k] / RA, ra = halo_pos[k] % RA;
        hglob[k] = (rb == 0 && b0 == 0) || (rb == TB + 1 && b0 + TB >= NB);
        if (ra == 0) { hoff[k] = TS::G_LEFT + (rb * QGS * SL + SL - 1) * ES; hqs[k] = SL * ES; }
        else if (ra == TA + 1) { hoff[k] = TS::G_RIGHT + (rb * QGS * SL) * ES; hqs[k] = SL * ES; }
        else { hoff[k] = TS::G_MAIN + (rb * QGS * 32 + ra - 1) * ES; hqs[k] = 32 * ES; }
      }
    }
    const int lane = tid & 31;
#pragma unroll
    for (int ki = 0; ki < KI; ++ki) {
      const int i = lane + 32 * ki;
      it_map[ki] = -1;
      it_c0[ki] = it_c1[ki] = it_dxb[ki] = it_dy[ki] = it_dz[ki] = it_dst[ki] = 0;
      it_g[ki] = false;
      if (i < 3) {
        it_g[ki] = true;
        it_map[ki] = i == 0 ? TM_G_MAIN : TM_G_SIDE;
        it_c0[ki] = i == 1 ? 32 - SL : 0;
        it_c1[ki] = Q0;
        it_dxb[ki] = i == 0 ? 0 : (i == 1 ? -1 : 1);
        it_dy[ki] = -1;
        it_dst[ki] = i == 0 ? TS::G_MAIN : (i == 1 ? TS::G_LEFT : TS::G_RIGHT);
      } else if (PAR == 0 && i == 3) {
        it_map[ki] = TM_F_ALL;
        it_dst[ki] = TS::F;
      } else if (PAR == 1 && i < NITEMS) {
        const bool side = i >= 3 + QF;
        // velocity q of the item: i - 3, or for a side item the
        // (i - 3 - QF)-th velocity with e_x != 0 (selected at compile time)
        int q = 0, ex = 0, ey = 0, ez = 0, oq = 0;
        static_for<0, QF>([&](auto qc) {
          constexpr int qq = decltype(qc)::value;
          const bool hit = side ? (LF::ex(qq) != 0 && side_rank<LF>(qq) == i - 3 - QF) : (qq == i - 3);
          if (hit) {
            q = qq;
            ex = LF::ex(qq);
            ey = LF::ey(qq);
            ez = LF::ez(qq);
            oq = LF::opp(qq);
          }
        });
        it_map[ki] = side ? TM_F_SIDE : TM_F_MAIN;
        it_c0[ki] = side && ex > 0 ? 32 - SL : 0;
        it_c1[ki] = oq;
        it_dxb[ki] = side ? (ex > 0 ? -1 : 1) : 0;
        it_dy[ki] = -ey;
        it_dz[ki] = -ez;
        it_dst[ki] = side ? TS::F_SIDE + (i - 3 - QF) * TS::F_SIDE_STRIDE : TS::F + q * TB * 32 * ES;
        (void)ex;
      }
    }
    if (tid == 0) {
      for (int k = 0; k < NST + 1; ++k) mbar_init(tbar + 8u * k, 1u);
      mbar_init_fence();
    }
    __syncthreads();
    if (args.test_wait_polls > 0) {
      // Test hook for the bounded waits: wait on barrier NST, which no
      // thread and no copy ever completes, give up after the given number
      // of polls and report it as a timed-out wait; the step then proceeds
      // unchanged (no copy is in flight yet).
      if (!mbar_wait_bounded(tbar + 8u * NST, 0u, args.test_wait_polls)) obs.bad |= kStatusTimeout;
    }
  }
  // Warp 0: the copies of g of plane cg and f of plane cf into stage s.
  auto tma_issue = [&](int cg, int cf, int s) {
    const unsigned bar = tbar + 8u * (unsigned)s, base = tstage + (unsigned)(s * TS::BYTES);
    if ((tid & 31) == 0) mbar_arrive_expect_tx(bar, TS::TX);
    __syncwarp();
    const int pg = wrap_mod(cg, NC);
#pragma unroll
    for (int ki = 0; ki < KI; ++ki) {
      if (it_map[ki] < 0) continue;
      const int z = wrap_mod((it_g[ki] ? pg : cf) + it_dz[ki], NC);
      const int xb = wrap_mod(xb0 + it_dxb[ki], NXB);
      // y may be -1 or run past ny - 1: those rows are zero-filled
      tma_load5(base + (unsigned)it_dst[ki], &tm->m[it_map[ki]], it_c0[ki], it_c1[ki], xb, b0 + it_dy[ki], z, bar);
    }
  };
  // phi of logical plane c from TMA stage s into the ring; keeps the own cell's g.
  auto produce_tma = [&](int c, int s, float (&gown)[QG]) {
    const char* base = tgen + s * TS::BYTES;
    float* slot = ring(c);
#pragma unroll
    for (int q = 0; q < QG; ++q)
      gown[q] = (q < Q0) ? 0.0f
                         : Codec<T>::dec(*reinterpret_cast<const T*>(base + own_goff + (q - Q0) * 32 * ES),
                                         pow2_scale<LG>(q), wprime<LG>(q) * P.gref);
    slot[own_slot] = finish_phi<FAM>(P, phi_star<LG, SKIP0>(gown), gamma);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      if (halo_pos[k] >= 0) {
        float tmp[QG];
        float hs;
        if (hglob[k]) {   // a wrapped halo row: from global memory
          hs = load_g(halo_ab[k] + (unsigned)(NAB * map_c(c)), tmp);
        } else {
#pragma unroll
          for (int q = 0; q < QG; ++q)
            tmp[q] = (q < Q0) ? 0.0f
                              : Codec<T>::dec(*reinterpret_cast<const T*>(base + hoff[k] + (q - Q0) * hqs[k]),
                                              pow2_scale<LG>(q), wprime<LG>(q) * P.gref);
          hs = phi_star<LG, SKIP0>(tmp);
        }
        slot[halo_pos[k]] = finish_phi<FAM>(P, hs, gamma);
      }
    }
  };

  float g0[QG], g1[QG], g2[QG];
  // Prologue: planes c0-H .. c0+H-1.
  {
    float tmp[QG];
#pragma unroll
    for (int h = H; h >= 1; --h) produce(c0 - h, tmp);
    produce(c0, g0);
    if constexpr (CH) produce(c0 + 1, g1);
  }
  // Half-select bits of the staged planes c, c+1, ..., c+NST-1 (index 0 is
  // the plane being collided; rotated every plane, compile-time indices).
  unsigned gmq[NST], fmq[NST];
  int st = 0;   // stage holding plane c
  // Planes in flight ahead of the current one: NST per-thread stages are
  // refilled at the end of the plane that consumed them; COOP stages only
  // after the next plane's first barrier, so one of the NST is always being
  // drained.
  constexpr int AHEAD = COOP ? NST - 1 : NST;
  if constexpr (TMAS) {
#pragma unroll
    for (int k = 0; k < NST; ++k) gmq[k] = fmq[k] = 0u;
    if (tid < 32) {
      for (int k = 0; k < AHEAD; ++k)
        if (c0 + k < c1) tma_issue(c0 + k + H, c0 + k, k);
    }
  } else if constexpr (STAGED) {
#pragma unroll
    for (int k = 0; k < NST; ++k) {
      gmq[k] = fmq[k] = 0u;
      if (k < AHEAD && c0 + k < c1) issue(c0 + k + H, c0 + k, k, gmq[k], fmq[k]);
      if (k < AHEAD) cp_async_commit();
    }
  }
  if constexpr (CH) {
    __syncthreads();
    make_mu(c0 - 1);
    make_mu(c0);
  }

  for (int c = c0; c < c1; ++c) {
    const unsigned gms = gmq[0], fms = fmq[0];
    bool landed = true;
    if constexpr (TMAS) {
      landed = mbar_wait_bounded(tbar + 8u * (unsigned)st, (tphase >> st) & 1u);   // plane c's copies
      tphase ^= 1u << st;
    } else if constexpr (STAGED) {
      cp_async_wait<AHEAD - 1>();   // plane c has landed; the later ones may be in flight
    }
    if constexpr (CH) {
      if constexpr (STAGED) produce_staged(c + 2, st, gms, g2);
      else produce(c + 2, g2);
      __syncthreads();
      make_mu(c + 1);
      __syncthreads();
    } else {
      if constexpr (TMAS) {
        produce_tma(c + 1, st, g1);
        // this thread's reads of the stage of plane c - 1 come before the
        // copies that refill it (generic -> async proxy)
        fence_proxy_async();
        if (__syncthreads_or(landed ? 0 : 1)) {
          tmo = true;
          cstop = c;
          break;
        }
      } else {
        if constexpr (STAGED) produce_staged(c + 1, st, gms, g1);
        else produce(c + 1, g1);
        __syncthreads();
      }
    }
    if constexpr (COOP) {
      // Every thread is past plane c - 1: refill its stage with plane c + NST - 1.
      const int sn = (st == 0) ? NST - 1 : st - 1;
      if constexpr (TMAS) {
        if (tid < 32 && c + NST - 1 < c1) tma_issue(c + NST - 1 + H, c + NST - 1, sn);
      } else {
        unsigned gnext = 0u, fnext = 0u;
        if (c + NST - 1 < c1) issue(c + NST - 1 + H, c + NST - 1, sn, gnext, fnext);
        cp_async_commit();
        gmq[NST - 1] = gnext;
        fmq[NST - 1] = fnext;
      }
    }

    if (active) {
      // Stencils of Sec. III on the ring (stencil lattice weights). Both are
      // formed from differences phi(x + e) - phi(x) (the gradient's sum of
      // w e phi(x) vanishes), which are exact in FP32 for nearby values.
      const float *pm = ring(c - 1), *p0 = ring(c), *pp = ring(c + 1);
      const float pc = p0[own_slot];
      float gp[DIM], lp;
      {
        float nb[QS];
        nb[0] = pc;
#pragma unroll
        for (int q = 1; q < QS; ++q) nb[q] = ring_nb(pm, p0, pp, own_slot, q);
        lp = Sym<LS>::lap(nb, pc);
#pragma unroll
        for (int k = 0; k < DIM; ++k) gp[k] = Sym<LS>::grad(nb, k);
      }

      float mu_c = 0.0f, lmu = 0.0f;
      if constexpr (CH) {
        const float* mm = s_mu + ((c - 1) & (MSLOT - 1)) * MPLANE;
        const float* m0 = s_mu + (c & (MSLOT - 1)) * MPLANE;
        const float* mp = s_mu + ((c + 1) & (MSLOT - 1)) * MPLANE;
        const int mpos = (ty + MHB) * MRA + (tx + 1);
        mu_c = m0[mpos];
        float nb[QS];
        nb[0] = mu_c;
#pragma unroll
        for (int q = 1; q < QS; ++q) {
          const int dc = dc_of<DIM, LS>(q);
          const float* ml = dc < 0 ? mm : (dc > 0 ? mp : m0);
          nb[q] = ml[mpos + db_of<DIM, LS>(q) * MRA + da_of<DIM, LS>(q)];
        }
        lmu = Sym<LS>::lap(nb, mu_c);
      }

      const bool lo_wall = walls && c == 0, hi_wall = walls && c == NC - 1;
      auto crosses = [&](int dcv) { return (dcv < 0 && lo_wall) || (dcv > 0 && hi_wall); };
      const unsigned idx = (unsigned)(aw + rbw + c * NAB);

      // Pre-collision f (AA pattern).
      float f[QF];
      if constexpr (TMAS) {
        // Even steps: row ty of the all-slot box. Odd steps: row ty of
        // velocity q's box holds the cells x0 - e_x .. x0 + 31 - e_x shifted
        // into lanes; the one lane whose source lies beyond the tile's x edge
        // reads the side box (lane SL - 1 of the left block for e_x = +1,
        // lane 0 of the right block for e_x = -1).
        const char* fst = tgen + st * TS::BYTES;
        static_for<0, QF>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          T v;
          if constexpr (PAR == 0) {
            v = *reinterpret_cast<const T*>(fst + TS::F + ((ty * QF + q) * 32 + tx) * ES);
          } else {
            constexpr int ex = LF::ex(q), ey = LF::ey(q);
            // the box's row ty lies beyond the y edge (wrapped): global memory
            const bool wrapped = (ey > 0 && ty == 0 && b0 == 0) || (ey < 0 && ty == TB - 1 && b0 + TB >= NB);
            if (wrapped) {
              constexpr int dc = dc_of<DIM, LF>(q);
              v = Codec<T>::ldc(fb + f_cell(-ex, -ey, plane_of(c, -dc)) + LF::opp(q) * kPopBlock);
            } else {
              const char* mainp = fst + TS::F + ((q * TB + ty) * 32 + tx - ex) * ES;
              if constexpr (ex == 0) {
                v = *reinterpret_cast<const T*>(mainp);
              } else {
                constexpr int sidx = side_rank<LF>(q);
                const char* sidep = fst + TS::F_SIDE + sidx * TS::F_SIDE_STRIDE + (ty * SL + (ex > 0 ? SL - 1 : 0)) * ES;
                const bool out = ex > 0 ? (tx == 0) : (tx == TA - 1);
                v = *reinterpret_cast<const T*>(out ? sidep : mainp);
              }
            }
          }
          f[q] = Codec<T>::dec(v, pow2_scale<LF>(q), 0.0f);
        });
      } else if constexpr (COOP) {
        // Row (q, ty) of the stage; an odd step's x - e_q sits at tx - e_x
        // from the row's x0 (+ CE where the row starts at x0 - CE).
        const T* fs = reinterpret_cast<const T*>(stage_f(st)) + ty * FROW + tx;
        static_for<0, QF>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          constexpr int ex = LF::ex(q);
          constexpr int off = PAR == 0 ? 0 : (ex > 0 ? CE - 1 : (ex < 0 ? 1 : 0));
          f[q] = Codec<T>::dec(fs[q * TB * FROW + off], pow2_scale<LF>(q), 0.0f);
        });
      } else if constexpr (STAGED) {
        const float* fs = stage_f(st);
#pragma unroll
        for (int q = 0; q < QF; ++q) f[q] = staged(fs[q * NT + tid], fms, q, q, false);
      } else {
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          const int da = da_of<DIM, LF>(q), db = db_of<DIM, LF>(q), dc = dc_of<DIM, LF>(q);
          const T* src = (parity == 0 || f_read_crosses(c, dc))
                             ? fb + f_cell(0, 0, c) + q * kPopBlock
                             : fb + f_cell(-da, -db, plane_of(c, -dc)) + LF::opp(q) * kPopBlock;
          f[q] = pop_loadc<T, LF>(src, q, 0.0f);
        }
      }
      float phiu[DIM];
      if constexpr (fam_phiu(FAM)) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) phiu[k] = args.phiu[k * N + idx];
      }
      const float phis = phi_star<LG, (DIM == 3 && !CH)>(g0);

      float u[DIM], rho, p;
      float gnew[QG];
#pragma unroll
      for (int q = 0; q < QG; ++q) gnew[q] = g0[q];
      Cell<FAM, DIM, LAT>::collide(P, gnew, f, pc, phis, gp, lp, mu_c, lmu, phiu, gamma, u, rho, p);

      // Observables of the pre-collision state.
      {
        comp_add(obs.s_hi, obs.s_lo, pc);
        const float fr = (pc - P.phiL) * P.inv_dphi;
        float usq = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) usq += u[k] * u[k];
        obs.vs += fr;
        obs.ke += 0.5f * rho * usq;
        // The fast-axis coordinates are fixed per thread: their moments are
        // aw (and bw in 3D) times the thread's volume sum, formed at the end.
        if constexpr (DIM == 3) obs.cz += (float)c * fr;
        else obs.cy += (float)c * fr;
        obs.count += (pc > P.phi0) ? 1u : 0u;
        obs.mx = fmaxf(obs.mx, pc);
        obs.mn = fminf(obs.mn, pc);
        // Instability (rho <= 0, non-finite phi or u) is judged once per thread
        // after the march: a non-finite value propagates into the sums.
      }

      if (args.macro) {
        args.out_phi[idx] = pc;
#pragma unroll
        for (int k = 0; k < DIM; ++k) args.out_u[k * N + idx] = u[k];
        args.out_p[idx] = p;
      } else {
        if constexpr (fam_phiu(FAM)) {
#pragma unroll
          for (int k = 0; k < DIM; ++k) args.phiu[k * N + idx] = phiu[k];
        }
        // g: two-array push, bounce-back into the own cell at walls.
        const float uw_lo = P.moving ? P.wall_u[0] : 0.0f, uw_hi = P.moving ? P.wall_u[1] : 0.0f;
        const unsigned rng = WIDE ? 0u : dither_seed(idx, args.seed);   // 16-bit storage: stochastic rounding
#pragma unroll
        for (int q = 0; q < QG; ++q) {
          if (DIM == 3 && !CH && q == 0) continue;
          const int da = da_of<DIM, LG>(q), db = db_of<DIM, LG>(q), dc = dc_of<DIM, LG>(q);
          if (P.freeze) {
            pop_store_sr<T, LG>(gdst + g_cell(0, 0, c) + q * kPopBlock, q, g0[q], P.gref, rng);
          } else if (crosses(dc)) {
            const float uw = dc < 0 ? uw_lo : uw_hi;
            const float v = gnew[q] - 6.0f * LG::w(q) * pc * (float)LG::ex(q) * uw;
            pop_store_sr<T, LG>(gdst + g_cell(0, 0, c) + LG::opp(q) * kPopBlock, q, v, P.gref, rng);
          } else {
            pop_store_sr<T, LG>(gdst + g_cell(da, db, plane_of(c, dc)) + q * kPopBlock, q, gnew[q], P.gref, rng);
          }
        }
        // f: AA pattern.
        const float sc = fam_phiu(FAM) ? rho : 1.0f;   // first-order f_eq scale: rho for the pressure-based forms
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          const int da = da_of<DIM, LF>(q), db = db_of<DIM, LF>(q), dc = dc_of<DIM, LF>(q);
          float v = f[q];
          const bool cr = crosses(dc);
          if (cr) {
            const float uw = dc < 0 ? uw_lo : uw_hi;
            v -= 6.0f * LF::w(q) * sc * (float)LF::ex(q) * uw;
          }
          if (parity == 0 || cr) {
            pop_store_sr<T, LF>(fb + f_cell(0, 0, c) + LF::opp(q) * kPopBlock, q, v, 0.0f, rng);
          } else {
            pop_store_sr<T, LF>(fb + f_cell(da, db, plane_of(c, dc)) + q * kPopBlock, q, v, 0.0f, rng);
          }
        }
      }
    }

    // Refill the stage just consumed with plane c + NST (issued here, where
    // the fewest values are live), and rotate the half-select bits.
    if constexpr (STAGED) {
      unsigned gnext = 0u, fnext = 0u;
      if constexpr (!COOP) {
        if (c + NST < c1) issue(c + NST + H, c + NST, st, gnext, fnext);
        cp_async_commit();
      } else {
        gnext = gmq[NST - 1];
        fnext = fmq[NST - 1];
      }
#pragma unroll
      for (int k = 0; k + 1 < NST; ++k) {
        gmq[k] = gmq[k + 1];
        fmq[k] = fmq[k + 1];
      }
      gmq[NST - 1] = gnext;
      fmq[NST - 1] = fnext;
      st = (st + 1 == NST) ? 0 : st + 1;
    }

    // Rotate the own-cell g pipeline.
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      g0[q] = g1[q];
      if constexpr (CH) g1[q] = g2[q];
    }
  }

  if constexpr (TMAS) {
    if (tmo) {
      // A stage's copies did not land within the poll limit: report it and
      // wait (bounded again) for the copies still in flight -- those of the
      // planes cstop .. cstop + NST - 2 -- before the block exits.
      obs.bad |= kStatusTimeout;
      for (int j = 0; j + 1 < NST; ++j) {
        if (cstop + j >= c1) break;
        const int s = (st + j) % NST;
        const unsigned par = ((tphase >> s) & 1u) ^ (j == 0 ? 1u : 0u);
        (void)mbar_wait_bounded(tbar + 8u * (unsigned)s, par);
      }
    }
  }
  (void)cstop;
  (void)tmo;
  // Centroid moments along the fast axes, whose coordinates are fixed per
  // thread (inactive threads added nothing to vs).
  obs.cx += (float)aw * obs.vs;
  if constexpr (DIM == 3) obs.cy += (float)bw * obs.vs;
  // A non-finite phi or u at any cell makes the phi or kinetic-energy sum
  // non-finite; rho is linear in phi, so its minimum over the cells is
  // attained at phi_min or phi_max (mn <= mx once a cell was visited).
  if (obs.mn <= obs.mx) {
    const float r1 = P.rhoL + P.drho_dphi * (obs.mn - P.phiL), r2 = P.rhoL + P.drho_dphi * (obs.mx - P.phiL);
    if (!(isfinite(obs.s_hi) && isfinite(obs.ke) && r1 > 0.0f && r2 > 0.0f)) obs.bad |= 1u;
  }
}

// ---------------------------------------------------------------------------
// The single-domain kernel: one tile per block.
// ---------------------------------------------------------------------------
template <int FAM, int DIM, typename T, int PAR, int ROW, int LAT>
__global__ void __launch_bounds__(Geom<FAM, DIM, T, LAT>::TA * Geom<FAM, DIM, T, LAT>::TB, Geom<FAM, DIM, T, LAT>::MINB)
step_kernel(const StepArgs args) {
  constexpr int TA = Geom<FAM, DIM, T, LAT>::TA, TB = Geom<FAM, DIM, T, LAT>::TB;
  using SM = TileSmem<FAM, DIM, T, TA, TB, (DIM == 3) && (ROW == 1) && (PAR >= 0), LAT>;
  extern __shared__ __align__(16) float dyn_smem[];
  float* s_stage = dyn_smem;
  float* s_phi = dyn_smem + SM::STAGE;
  float* s_mu = s_phi + SM::PHI;
  __shared__ double s_red[(TA * TB / 32) * 10];
  const int NA = args.p.nx, NB = (DIM == 3) ? args.p.ny : 1;
  const int tiles_a = (NA + TA - 1) / TA, tiles_b = (NB + TB - 1) / TB;
  int bid = blockIdx.x;
  const int ti = bid % tiles_a;
  bid /= tiles_a;
  const int tj = bid % tiles_b;
  bid /= tiles_b;
  if (args.obs_zero != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    obs_zero_slot(args.obs_zero);
  ObsPartial obs;
  obs_init(obs);
  step_tile<FAM, DIM, T, TA, TB, PAR, ROW, LAT>(args, ti * TA, tj * TB, bid * args.chunk, args.chunk, s_phi, s_mu,
                                                s_stage, obs);
  obs_block_commit(obs, args.obs_slot, s_red);
}

// The single-domain kernel with TMA staging (3D, nx a multiple of 32, ny a
// multiple of TB, Allen-Cahn halo): the tensor maps of this step's arrays
// come by value in parameter space.
template <int FAM, int DIM, typename T, int PAR, int LAT>
__global__ void __launch_bounds__(Geom<FAM, DIM, T, LAT>::TA * Geom<FAM, DIM, T, LAT>::TB, Geom<FAM, DIM, T, LAT>::MINB)
step_kernel_tma(const StepArgs args, const __grid_constant__ TmaMaps tm) {
  constexpr int TA = Geom<FAM, DIM, T, LAT>::TA, TB = Geom<FAM, DIM, T, LAT>::TB;
  using SM = TileSmem<FAM, DIM, T, TA, TB, true, LAT, true, PAR>;
  extern __shared__ __align__(128) float dyn_smem_tma[];
  float* s_stage = dyn_smem_tma;
  float* s_phi = dyn_smem_tma + SM::STAGE;
  float* s_mu = s_phi + SM::PHI;
  __shared__ double s_red[(TA * TB / 32) * 10];
  const int NA = args.p.nx, NB = args.p.ny;
  const int tiles_a = (NA + TA - 1) / TA, tiles_b = (NB + TB - 1) / TB;
  int bid = blockIdx.x;
  const int ti = bid % tiles_a;
  bid /= tiles_a;
  const int tj = bid % tiles_b;
  bid /= tiles_b;
  if (args.obs_zero != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    obs_zero_slot(args.obs_zero);
  ObsPartial obs;
  obs_init(obs);
  step_tile<FAM, DIM, T, TA, TB, PAR, 1, LAT, true>(args, ti * TA, tj * TB, bid * args.chunk, args.chunk, s_phi, s_mu,
                                                    s_stage, obs, &tm);
  obs_block_commit(obs, args.obs_slot, s_red);
}

template <int FAM, int DIM, typename T, int PAR, int ROW, int LAT>
void launch_step_par(const StepArgs& args, cudaStream_t stream) {
  constexpr int TA = Geom<FAM, DIM, T, LAT>::TA, TB = Geom<FAM, DIM, T, LAT>::TB;
  if constexpr (DIM == 3 && ROW == 1 && FAM != FAM_LIANG && TA == 32) {
    if (args.tma != nullptr && args.p.ny % TB == 0) {
      constexpr size_t smem = TileSmem<FAM, DIM, T, TA, TB, true, LAT, true, PAR>::BYTES;
      static const cudaError_t attr = cudaFuncSetAttribute(
          step_kernel_tma<FAM, DIM, T, PAR, LAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      (void)attr;
      const long long tiles = (long long)(args.p.nx / TA) * (args.p.ny / TB);
      const long long chunks = (args.p.nz + args.chunk - 1) / args.chunk;
      step_kernel_tma<FAM, DIM, T, PAR, LAT><<<(unsigned)(tiles * chunks), dim3(TA, TB, 1), smem, stream>>>(
          args, *args.tma);
      return;
    }
  }
  constexpr size_t smem = TileSmem<FAM, DIM, T, TA, TB, (DIM == 3) && (ROW == 1) && (PAR >= 0), LAT>::BYTES;
  static const cudaError_t attr = cudaFuncSetAttribute(
      step_kernel<FAM, DIM, T, PAR, ROW, LAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  (void)attr;
  const int NA = args.p.nx, NB = (DIM == 3) ? args.p.ny : 1, NC = (DIM == 3) ? args.p.nz : args.p.ny;
  const long long tiles = (long long)((NA + TA - 1) / TA) * ((NB + TB - 1) / TB);
  const long long chunks = (NC + args.chunk - 1) / args.chunk;
  dim3 block(TA, TB, 1);
  step_kernel<FAM, DIM, T, PAR, ROW, LAT><<<(unsigned)(tiles * chunks), block, smem, stream>>>(args);
}

template <int FAM, int DIM, typename T, int LAT = 0>
void launch_step(const StepArgs& args, cudaStream_t stream) {
  const bool row = args.p.nx % (int)kPopBlock == 0;
  if (args.parity) {
    if (row) launch_step_par<FAM, DIM, T, 1, 1, LAT>(args, stream);
    else launch_step_par<FAM, DIM, T, 1, 0, LAT>(args, stream);
  } else {
    if (row) launch_step_par<FAM, DIM, T, 0, 1, LAT>(args, stream);
    else launch_step_par<FAM, DIM, T, 0, 0, LAT>(args, stream);
  }
}

}  // namespace pflb
