// Bao2024 (Sec. II D 3): Cahn-Hilliard with singular mobility (Eq.
// bao_singular_mobility), a lattice kinetic scheme (Eqs. bao_g_eq, bao_f_eq,
// bao_Mphi, bao_v) and the quasi-incompressible sources and updates of
// Yang2016 (Eqs. Yang_G, Yang_F, yang_update); constants of Reading R21.
//
// Its equilibria need the gradients of u, p and mu at the current time, i.e.
// macroscopic fields of the neighbours, so the step runs as four grid-stride
// passes over the domain (periodic, FP32 storage, same population layout and
// AA / push streaming as the fused step):
//   1. phi = sum g                                   -> work[phi]
//   2. mu = 4 beta (...) - kappa lap phi             -> work[mu]
//   3. u (Eq. yang_u_update), p (Eq. yang_p_update)  -> work[u], work[p];
//      observables of the state
//   4. collision of g and f with the stencils of phi, mu, M(phi), u, p;
//      streaming.
// The work buffer holds (3 + d) fields: phi, mu, p, u_x, u_y[, u_z]. Every
// pass walks the domain as (x, y) tiles marching in z (pflb_pass.cuh).
#include "pflb_init.cuh"
#include "pflb_pass.cuh"

namespace pflb {
namespace {

constexpr int kThreads = kPassThreads;

// Field values at the stencil neighbours x + e_q of the stencil lattice.
template <int DIM, typename LS>
__device__ __forceinline__ void gather(const float* fld, const PassCell& cl, float (&v)[LS::Q]) {
#pragma unroll
  for (int q = 0; q < LS::Q; ++q) v[q] = fld[cl.nb(LS::ex(q), LS::ey(q), LS::ez(q))];
}

// Singular mobility M(phi), Eq. (bao_singular_mobility); M_0 = P.M.
__device__ __forceinline__ float bao_M(const DevParams& P, float phi) {
  return 4.0f * P.M * fabsf(phi - P.phiH) * fabsf(phi - P.phiL) * P.inv_dphi * P.inv_dphi;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_phi_kernel(const StepArgs a, PassGeo<DIM> G) {
  using LG = typename Lattices<DIM>::G;
  const float* g = static_cast<const float*>(a.g_src);
  float* phi = a.work;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    float v[LG::Q];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) v[q] = g[pop_ix<LG>(q, cl.c)];
    phi[cl.c] = v[0] + Sym<LG>::moving(v);   // Eq. (fakhari_phi_update)
  });
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_mu_kernel(const StepArgs a, PassGeo<DIM> G) {
  using LS = typename Lattices<DIM>::S;
  const DevParams& P = a.p;
  const float* phi = a.work;
  float* mu = a.work + a.N;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    float v[LS::Q];
    gather<DIM, LS>(phi, cl, v);
    const float pc = v[0];
    mu[cl.c] = P.beta4 * (pc - P.phiH) * (pc - P.phiL) * (pc - P.phi0) - P.kappa * Sym<LS>::lap(v, pc);  // Eq. (chemical_potential)
  });
}

// grad mu, lap mu and div(M grad mu) = M lap mu + grad M . grad mu (Reading R21),
// from phi at the stencil neighbours (vp, already gathered by the caller)
template <int DIM>
__device__ __forceinline__ void bao_flux(const DevParams& P, const float (&vp)[Lattices<DIM>::S::Q], const float* mu,
                                         const PassCell& cl, float phic, float (&gmu)[DIM], float& divJ) {
  using LS = typename Lattices<DIM>::S;
  float vm[LS::Q];
  gather<DIM, LS>(mu, cl, vm);
  float vM[LS::Q];
#pragma unroll
  for (int q = 0; q < LS::Q; ++q) vM[q] = bao_M(P, vp[q]);
  const float lmu = Sym<LS>::lap(vm, vm[0]);
  float gdot = 0.0f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    gmu[k] = Sym<LS>::grad(vm, k);
    gdot += Sym<LS>::grad(vM, k) * gmu[k];
  }
  divJ = bao_M(P, phic) * lmu + gdot;
}

// Pass 3: u, p and the observables of the state.
template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_macro_kernel(const StepArgs a, PassGeo<DIM> G) {
  using LF = typename Lattices<DIM>::F;
  using LS = typename Lattices<DIM>::S;
  constexpr float cs2 = 1.0f / 3.0f;
  const DevParams& P = a.p;
  const float* phi = a.work;
  const float* mu = a.work + a.N;
  float* pf = a.work + 2 * a.N;
  float* uf = a.work + 3 * a.N;
  const float* fb = static_cast<const float*>(a.f);
  __shared__ double s_red[(kThreads / 32) * 10];
  if (a.obs_zero != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    obs_zero_slot(a.obs_zero);
  ObsPartial obs;
  obs_init(obs);
  const float theta = P.theta;   // quasi-incompressible theta, Eq. (quasi_incomp_system)
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    const int x = cl.x, y = cl.y, z = cl.z;
    // next plane: the f lines, then the phi and mu rows
    const long long rn = next_plane_row<DIM>(G, cl);
    if (rn >= 0) {
      const int l = threadIdx.x;
      if (l < LF::Q) prefetch_l2(group_line<LF>(fb, rn, l));
      else if (l < LF::Q + 2) prefetch_l2(a.work + (size_t)(l - LF::Q) * a.N + rn);
    }
    // incoming f (AA): even steps slot q of the own cell, odd steps slot opp(q) of x - e_q
    float f[LF::Q];
#pragma unroll
    for (int q = 0; q < LF::Q; ++q)
      f[q] = a.parity == 0 ? fb[pop_ix<LF>(q, (unsigned)c)]
                           : fb[pop_ix<LF>(LF::opp(q), cl.nb(-LF::ex(q), -LF::ey(q), -LF::ez(q)))];
    float vp[LS::Q];
    gather<DIM, LS>(phi, cl, vp);
    const float pc = vp[0];
    float gp[DIM], gmu[DIM], divJ;
    bao_flux<DIM>(P, vp, mu, cl, pc, gmu, divJ);
    const float rho = P.rhoL + P.drho_dphi * (pc - P.phiL);
    const float muc = mu[c];
    float u[DIM], Fs[DIM], Fb[DIM];
    const float A = P.lundA;
    float usq = 0.0f, ugr = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      gp[k] = Sym<LS>::grad(vp, k);
      Fs[k] = muc * gp[k];
      Fb[k] = rho * P.grav[k] + P.fdens[k];
      // Eq. (yang_u_update): rho c_s^2 u = sum e f + c_s^2 F / 2 (linear forcing solved for)
      u[k] = (Sym<LF>::first(f, k) + 0.5f * cs2 * (Fs[k] + Fb[k])) / (rho * cs2 * (1.0f - 0.5f * A));
      usq += u[k] * u[k];
      ugr += u[k] * P.drho_dphi * gp[k];
    }
    // Eq. (yang_p_update)
    const float p = (f[0] + Sym<LF>::moving(f)) + 0.5f * cs2 * (ugr - theta * rho * divJ);
    if (a.macro) {
      a.out_phi[c] = pc;
#pragma unroll
      for (int k = 0; k < DIM; ++k) a.out_u[k * a.N + c] = u[k];
      a.out_p[c] = p;
    } else {
      pf[c] = p;
#pragma unroll
      for (int k = 0; k < DIM; ++k) uf[k * a.N + c] = u[k];
    }
    comp_add(obs.s_hi, obs.s_lo, pc);
    const float fr = (pc - P.phiL) * P.inv_dphi;
    obs.vs += fr;
    obs.ke += 0.5f * rho * usq;
    obs.cx += (float)x * fr;
    obs.cy += (float)y * fr;
    if (DIM == 3) obs.cz += (float)z * fr;
    obs.count += (pc > P.phi0) ? 1u : 0u;
    obs.mx = fmaxf(obs.mx, pc);
    obs.mn = fminf(obs.mn, pc);
  });
  if (obs.mn <= obs.mx) {
    const float r1 = P.rhoL + P.drho_dphi * (obs.mn - P.phiL), r2 = P.rhoL + P.drho_dphi * (obs.mx - P.phiL);
    if (!(isfinite(obs.s_hi) && isfinite(obs.ke) && r1 > 0.0f && r2 > 0.0f)) obs.bad = 1u;
  }
  obs_block_commit(obs, a.obs_slot, s_red);
}

// Gamma_a(u) / w_a = e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2), Eq. (Gamma_beta)
template <typename L, int DIM>
__device__ __forceinline__ float gam_w(int q, const float (&u)[DIM], float usq) {
  float eu = 0.0f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) eu += (float)ecomp<L>(q, k) * u[k];
  return 3.0f * eu + 4.5f * eu * eu - 1.5f * usq;
}

// Pass 4: collision and streaming.
template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_collide_kernel(const StepArgs a, PassGeo<DIM> G) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  using LS = typename Lattices<DIM>::S;
  constexpr float cs2 = 1.0f / 3.0f;
  const DevParams& P = a.p;
  const float* phi = a.work;
  const float* mu = a.work + a.N;
  const float* pf = a.work + 2 * a.N;
  const float* uf = a.work + 3 * a.N;
  const float* gs = static_cast<const float*>(a.g_src);
  float* gd = static_cast<float*>(a.g_dst);
  float* fb = static_cast<float*>(a.f);
  const float theta = P.theta;
  const float itp = P.inv_tau_phi, swp = P.src_w_phi;   // constant tau_phi (Reading R21)
  const float itau = P.lks_itau, fwt = 1.0f - 0.5f * P.lks_itau;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    // next plane: lanes 0..QG-1 the g lines, then the f lines, then the
    // field rows (phi, mu, p, u)
    const long long rn = next_plane_row<DIM>(G, cl);
    if (rn >= 0) {
      const int l = threadIdx.x;
      if (l < LG::Q) prefetch_l2(group_line<LG>(gs, rn, l));
      else if (l < LG::Q + LF::Q) prefetch_l2(group_line<LF>(fb, rn, l - LG::Q));
      else if (l < LG::Q + LF::Q + 3 + DIM) prefetch_l2(a.work + (size_t)(l - LG::Q - LF::Q) * a.N + rn);
    }
    float vp[LS::Q], vpr[LS::Q];
    gather<DIM, LS>(phi, cl, vp);
    gather<DIM, LS>(pf, cl, vpr);
    const float pc = vp[0], p = vpr[0], muc = mu[c];
    float gmu[DIM], divJ;
    bao_flux<DIM>(P, vp, mu, cl, pc, gmu, divJ);
    const float rho = P.rhoL + P.drho_dphi * (pc - P.phiL);
    const float nu = viscosity(P, pc, rho);
    const float A_lks = (1.0f / itp) - 0.5f - bao_M(P, pc) * 3.0f / P.eta;   // Eq. (bao_Mphi)
    const float B_lks = (1.0f / itau) - 0.5f - 3.0f * nu;                      // Eq. (bao_v)
    float u[DIM], gp[DIM], gpr[DIM], F[DIM], S[DIM][DIM];
    float usq = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      u[k] = uf[k * a.N + c];
      usq += u[k] * u[k];
      gp[k] = Sym<LS>::grad(vp, k);
      gpr[k] = Sym<LS>::grad(vpr, k);
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[k] = muc * gp[k] + rho * P.grav[k] + P.fdens[k] + P.lundA * rho * u[k];
    // S = grad u + (grad u)^T by the stencils of the u fields
    float du[DIM][DIM];   // du[k][i] = d_i u_k
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      float vu[LS::Q];
      gather<DIM, LS>(uf + k * a.N, cl, vu);
#pragma unroll
      for (int i = 0; i < DIM; ++i) du[k][i] = Sym<LS>::grad(vu, i);
    }
    float trS = 0.0f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
#pragma unroll
      for (int j = 0; j < DIM; ++j) S[i][j] = du[j][i] + du[i][j];
      trS += S[i][i];
    }
    // ---- phase field: Eqs. (bao_g_eq), (Yang_G)
    float g[LG::Q], geq[LG::Q], Gs[LG::Q];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) g[q] = gs[pop_ix<LG>(q, c)];
    float V[DIM], uV = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      V[k] = gpr[k] - F[k];
      uV += u[k] * V[k];
    }
    const float gcoef = -pc / (cs2 * rho);
    float sumeq = 0.0f, sumG = 0.0f;
#pragma unroll
    for (int q = 1; q < LG::Q; ++q) {
      const float w = LG::w(q);
      float egm = 0.0f, eV = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        egm += (float)ecomp<LG>(q, k) * gmu[k];
        eV += (float)ecomp<LG>(q, k) * V[k];
      }
      const float gw = gam_w<LG, DIM>(q, u, usq);
      geq[q] = w * (P.eta * muc + pc * gw + A_lks * P.eta * egm);
      Gs[q] = gcoef * (eV - uV) * w * (1.0f + gw);
      sumeq += geq[q];
      sumG += Gs[q];
    }
    geq[0] = pc - sumeq;   // = phi - (1 - w_0) eta mu + phi Gamma_0: zeroth moment phi exactly
    Gs[0] = -sumG;         // sum G = 0 exactly
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) g[q] = g[q] - (g[q] - geq[q]) * itp + swp * Gs[q];
    // ---- hydrodynamics: Eqs. (bao_f_eq), (Yang_F)
    float f[LF::Q];
#pragma unroll
    for (int q = 0; q < LF::Q; ++q)
      f[q] = a.parity == 0 ? fb[pop_ix<LF>(q, (unsigned)c)]
                           : fb[pop_ix<LF>(LF::opp(q), cl.nb(-LF::ex(q), -LF::ey(q), -LF::ez(q)))];
    float uF = 0.0f, ugr = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      uF += u[k] * F[k];
      ugr += u[k] * P.drho_dphi * gp[k];
    }
#pragma unroll
    for (int q = 0; q < LF::Q; ++q) {
      const float w = LF::w(q);
      float eF = 0.0f, eg = 0.0f, SS = 0.0f;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        eF += (float)ecomp<LF>(q, i) * F[i];
        eg += (float)ecomp<LF>(q, i) * P.drho_dphi * gp[i];
#pragma unroll
        for (int j = 0; j < DIM; ++j) SS += (float)(ecomp<LF>(q, i) * ecomp<LF>(q, j)) * S[i][j];
      }
      const float gw = gam_w<LF, DIM>(q, u, usq);
      const float feq = w * (p + cs2 * rho * gw + 0.5f * rho * B_lks * (SS - cs2 * trS));
      const float Fq = (eF - uF) * w * (1.0f + gw) + w * gw * cs2 * (eg - ugr) - w * cs2 * rho * theta * divJ;
      f[q] = f[q] - (f[q] - feq) * itau + fwt * Fq;
    }
    // ---- streaming: g pushed to x + e into the other array; f AA
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) gd[pop_ix<LG>(q, cl.nb(LG::ex(q), LG::ey(q), LG::ez(q)))] = g[q];
#pragma unroll
    for (int q = 0; q < LF::Q; ++q) {
      if (a.parity == 0) fb[pop_ix<LF>(LF::opp(q), c)] = f[q];
      else fb[pop_ix<LF>(q, cl.nb(LF::ex(q), LF::ey(q), LF::ez(q)))] = f[q];
    }
  });
}

// Initial state: mu of phi0 into work[mu], then the equilibria of Eqs.
// (bao_g_eq), (bao_f_eq) with p = 0 and S of u0 (Reading R8).
template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_init_mu_kernel(const InitArgs a, PassGeo<DIM> G) {
  using LS = typename Lattices<DIM>::S;
  const DevParams& P = a.p;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    float v[LS::Q];
    gather<DIM, LS>(a.phi0, cl, v);
    const float pc = v[0];
    a.work[a.N + cl.c] = P.beta4 * (pc - P.phiH) * (pc - P.phiL) * (pc - P.phi0) - P.kappa * Sym<LS>::lap(v, pc);
  });
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) bao_init_kernel(const InitArgs a, PassGeo<DIM> G) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  using LS = typename Lattices<DIM>::S;
  constexpr float cs2 = 1.0f / 3.0f;
  const DevParams& P = a.p;
  const float* mu = a.work + a.N;
  float* g = static_cast<float*>(a.g);
  float* f = static_cast<float*>(a.f);
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    const float pc = a.phi0[c], muc = mu[c];
    const float rho = P.rhoL + P.drho_dphi * (pc - P.phiL);
    const float nu = viscosity(P, pc, rho);
    const float A_lks = (1.0f / P.inv_tau_phi) - 0.5f - bao_M(P, pc) * 3.0f / P.eta;
    const float B_lks = (1.0f / P.lks_itau) - 0.5f - 3.0f * nu;
    float vm[LS::Q];
    gather<DIM, LS>(mu, cl, vm);
    float u[DIM], gmu[DIM], du[DIM][DIM], S[DIM][DIM];
    float usq = 0.0f, trS = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      u[k] = a.u0 ? a.u0[k * a.N + c] : 0.0f;
      usq += u[k] * u[k];
      gmu[k] = Sym<LS>::grad(vm, k);
      float vu[LS::Q];
      if (a.u0) gather<DIM, LS>(a.u0 + k * a.N, cl, vu);
#pragma unroll
      for (int i = 0; i < DIM; ++i) du[k][i] = a.u0 ? Sym<LS>::grad(vu, i) : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
#pragma unroll
      for (int j = 0; j < DIM; ++j) S[i][j] = du[j][i] + du[i][j];
      trS += S[i][i];
    }
    float sumeq = 0.0f;
#pragma unroll
    for (int q = 1; q < LG::Q; ++q) {
      float egm = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) egm += (float)ecomp<LG>(q, k) * gmu[k];
      const float geq = LG::w(q) * (P.eta * muc + pc * gam_w<LG, DIM>(q, u, usq) + A_lks * P.eta * egm);
      g[pop_ix<LG>(q, c)] = geq;
      sumeq += geq;
    }
    g[pop_ix<LG>(0, c)] = pc - sumeq;
#pragma unroll
    for (int q = 0; q < LF::Q; ++q) {
      float SS = 0.0f;
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) SS += (float)(ecomp<LF>(q, i) * ecomp<LF>(q, j)) * S[i][j];
      f[pop_ix<LF>(q, c)] =
          LF::w(q) * (cs2 * rho * gam_w<LF, DIM>(q, u, usq) + 0.5f * rho * B_lks * (SS - cs2 * trS));
    }
  });
}

template <int DIM>
void bao_step_dim(const StepArgs& a, cudaStream_t s) {
  const PassGeo<DIM> G = pass_geo<DIM>(a.p.nx, a.p.ny, a.p.nz, num_sms());
  const dim3 grid = G.grid(), block(kPassTX, kPassTY);
  bao_phi_kernel<DIM><<<grid, block, 0, s>>>(a, G);
  bao_mu_kernel<DIM><<<grid, block, 0, s>>>(a, G);
  bao_macro_kernel<DIM><<<grid, block, 0, s>>>(a, G);
  if (!a.macro) bao_collide_kernel<DIM><<<grid, block, 0, s>>>(a, G);
}

template <int DIM>
void bao_init_dim(const InitArgs& a, cudaStream_t s) {
  const PassGeo<DIM> G = pass_geo<DIM>(a.p.nx, a.p.ny, a.p.nz, num_sms());
  const dim3 grid = G.grid(), block(kPassTX, kPassTY);
  bao_init_mu_kernel<DIM><<<grid, block, 0, s>>>(a, G);
  bao_init_kernel<DIM><<<grid, block, 0, s>>>(a, G);
}

}  // namespace

void step_bao2024(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  (void)storage;   // FP32 only (validated by the API)
  if (dim == 2) bao_step_dim<2>(a, s);
  else bao_step_dim<3>(a, s);
}

void init_bao2024(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  (void)storage;
  if (dim == 2) bao_init_dim<2>(a, s);
  else bao_init_dim<3>(a, s);
}

}  // namespace pflb
