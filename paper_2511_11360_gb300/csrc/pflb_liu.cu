// Liu2023 (Sec. II C 5): hybrid Allen-Cahn whose weight lambda(x) is 1 within
// d_min = 3 xi of the interface and 0 elsewhere, with Liang2018's equilibria,
// forcing and updates (Eqs. Liu_G, Liu_F); Reading R22 for the reconstruction.
//
// lambda needs a signed distance of the whole field before any collision, so
// the step runs as grid-stride passes over the domain (periodic, FP32, same
// population layout and AA / push streaming as the fused step):
//   1. phi* = sum g; predictor psi0 = -(xi/4) ln((phi_H - phi_L)/(phi* - phi_L) - 1)
//      (phi* clamped to [phi_L + 0.01, phi_H - 0.01])
//   2. ceil(2 d_min) pseudo-time steps (dt' = 1/2) of the reinitialisation
//      equation d psi/dt' + S(psi0)(|grad psi| - 1) = 0, first-order Godunov
//      upwinding, S(psi0) = psi0 / sqrt(psi0^2 + 1) (formed once by the
//      predictor)
//   3. lambda = [|psi| < d_min]; the (1 - lambda)-weighted integrals of Eq.
//      (lagrange_multiplier) in FP64
//   4. phi = phi* + (1 - lambda) R(phi*) / 2
//   5. collision (the Liang2018 update of the fused step with Eq. Liu_G's
//      mix), streaming, observables.
// Work fields (N floats each): phi*, S(psi0), psi_a, psi_b, lambda, phi.
// Every pass walks the domain as (x, y) tiles marching in z (pflb_pass.cuh).
#include <algorithm>

#include "pflb_init.cuh"
#include "pflb_pass.cuh"

namespace pflb {
namespace {

constexpr int kThreads = kPassThreads;

struct LiuWork {
  float *phis, *s0, *psia, *psib, *lam, *phi;
};
__host__ __device__ inline LiuWork liu_work(float* w, long long N) {
  return LiuWork{w, w + N, w + 2 * N, w + 3 * N, w + 4 * N, w + 5 * N};
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) liu_predict_kernel(const StepArgs a, PassGeo<DIM> G) {
  using LG = typename Lattices<DIM>::G;
  constexpr bool SKIP0 = DIM == 3;   // D3Q7 rest population of the Allen-Cahn families is zero
  const DevParams& P = a.p;
  const LiuWork W = liu_work(a.work, a.N);
  const float* g = static_cast<const float*>(a.g_src);
  const float lo = P.phiL + 0.01f, hi = P.phiH - 0.01f, dphi = P.phiH - P.phiL;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    float v[LG::Q];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) v[q] = (SKIP0 && q == 0) ? 0.0f : g[pop_ix<LG>(q, (unsigned)c)];
    const float ps = phi_star<LG, SKIP0>(v);
    W.phis[c] = ps;
    const float pc = fminf(fmaxf(ps, lo), hi);
    const float psi = -0.25f * P.W_xi * logf(dphi / (pc - P.phiL) - 1.0f);
    W.s0[c] = psi * rsqrtf(psi * psi + 1.0f);
    W.psia[c] = psi;
  });
}

// One first-order Godunov step (dt' = 1/2) of the reinitialisation equation
// at a cell from its value p, its axis neighbours (minus, plus) and
// S = S(psi0) (Reading R22). Upwinding per axis: for S > 0,
// max(max(D-, 0)^2, min(D+, 0)^2), for S <= 0, max(min(D-, 0)^2, max(D+, 0)^2)
// with D- = p - p(x - e), D+ = p(x + e) - p; with sg = sign(S) both read
// max(max(sg D-, 0)^2, max(-sg D+, 0)^2) (the squares lose the sign exactly).
template <int DIM>
__device__ __forceinline__ float liu_godunov(float p, const float (&nm)[DIM], const float (&np)[DIM], float S) {
  const float sg = S > 0.0f ? 1.0f : -1.0f;
  float g2 = 0.0f;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    // a, b >= 0 and rounding is monotonic: max(a, b)^2 == max(a^2, b^2) exactly
    const float a = fmaxf(sg * (p - nm[ax]), 0.0f), b = fmaxf(sg * (p - np[ax]), 0.0f);
    const float m = fmaxf(a, b);
    g2 = fmaf(m, m, g2);
  }
  return p - 0.5f * S * (sqrtf(g2) - 1.0f);
}

// One pseudo-time step over the domain: the (x, y)-tile walk of the other
// passes, with psi of the z neighbours carried in registers along the march.
template <int DIM>
__global__ void __launch_bounds__(kThreads) liu_reinit_kernel(const float* __restrict__ psi_in,
                                                              float* __restrict__ psi_out,
                                                              const float* __restrict__ s0, PassGeo<DIM> G) {
  const int x = (int)(blockIdx.x * kPassTX + threadIdx.x), y = (int)(blockIdx.y * kPassTY + threadIdx.y);
  if (x >= G.nx || y >= G.ny) return;
  const unsigned nx = (unsigned)G.nx;
  const unsigned xm = (unsigned)(x == 0 ? G.nx - 1 : x - 1), xp = (unsigned)(x == G.nx - 1 ? 0 : x + 1);
  const unsigned ym = nx * (unsigned)(y == 0 ? G.ny - 1 : y - 1), yp = nx * (unsigned)(y == G.ny - 1 ? 0 : y + 1);
  const unsigned xc = (unsigned)x, yc = nx * (unsigned)y;
  if constexpr (DIM == 2) {
    const unsigned c = xc + yc;
    const float nm[2] = {psi_in[xm + yc], psi_in[xc + ym]};
    const float np[2] = {psi_in[xp + yc], psi_in[xc + yp]};
    psi_out[c] = liu_godunov<2>(psi_in[c], nm, np, s0[c]);
  } else {
    const unsigned nxy = nx * (unsigned)G.ny;
    const int z0 = (int)blockIdx.z * G.zc, z1 = min(G.nz, z0 + G.zc);
    float pzm = psi_in[xc + yc + nxy * (unsigned)(z0 == 0 ? G.nz - 1 : z0 - 1)];
    float pzc = psi_in[xc + yc + nxy * (unsigned)z0];
    // U planes per round, all of their loads issued before any update (the
    // update is cheap, so the march is bound by how many loads are in flight;
    // at 512^3 U = 2 measured best: 8 cost occupancy); planes past the run
    // repeat its last plane and are not stored
    constexpr int U = 2;
    for (int z = z0; z < z1; z += U) {
      float zn[U], vxm[U], vxp[U], vym[U], vyp[U], sv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int zz = min(z + u, z1 - 1);
        const unsigned oz = nxy * (unsigned)zz, ozp = nxy * (unsigned)(zz == G.nz - 1 ? 0 : zz + 1);
        zn[u] = psi_in[xc + yc + ozp];
        vxm[u] = psi_in[xm + yc + oz];
        vxp[u] = psi_in[xp + yc + oz];
        vym[u] = psi_in[xc + ym + oz];
        vyp[u] = psi_in[xc + yp + oz];
        sv[u] = s0[xc + yc + oz];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (z + u < z1) {
          const float nm[3] = {vxm[u], vym[u], pzm};
          const float np[3] = {vxp[u], vyp[u], zn[u]};
          psi_out[xc + yc + nxy * (unsigned)(z + u)] = liu_godunov<3>(pzc, nm, np, sv[u]);
          pzm = pzc;
          pzc = zn[u];
        }
      }
    }
  }
}

// The same sweep in 3D with four consecutive x cells per thread (nx a
// multiple of 4): psi rows and S(psi0) as 16-byte loads, the two x
// neighbours outside the four as scalar loads, the same update per cell.
// The sweep is bound by instruction issue (~100 instructions per cell, most
// of them loads and their addressing); this form has a quarter of the loads
// and address arithmetic per cell. Block: 32 x 8 threads = 128 x 8 cells.
constexpr int kR4X = 4 * kPassTX;

struct Reinit4Geo {
  int nx, ny, nz, zc;
  __host__ dim3 grid() const {
    return dim3((unsigned)((nx + kR4X - 1) / kR4X), (unsigned)((ny + kPassTY - 1) / kPassTY),
                (unsigned)((nz + zc - 1) / zc));
  }
};

__host__ inline Reinit4Geo reinit4_geo(int nx, int ny, int nz, int sms) {
  Reinit4Geo G{nx, ny, nz, 1};
  const long long tiles = (long long)((nx + kR4X - 1) / kR4X) * ((ny + kPassTY - 1) / kPassTY);
  const long long target = 32LL * sms;   // blocks, as for the other passes
  long long zc = (tiles * nz + target - 1) / target;
  G.zc = (int)std::min<long long>(std::max<long long>(zc, 1), std::min(32, nz));
  return G;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__global__ void __launch_bounds__(kThreads) liu_reinit4_kernel(const float* __restrict__ psi_in,
                                                               float* __restrict__ psi_out,
                                                               const float* __restrict__ s0, Reinit4Geo G) {
  const int x = (int)(blockIdx.x * kPassTX + threadIdx.x) * 4, y = (int)(blockIdx.y * kPassTY + threadIdx.y);
  if (x >= G.nx || y >= G.ny) return;
  const unsigned nx = (unsigned)G.nx, nxy = nx * (unsigned)G.ny;
  const unsigned xm = (unsigned)(x == 0 ? G.nx - 1 : x - 1), xp = (unsigned)(x + 4 == G.nx ? 0 : x + 4);
  const unsigned ym = nx * (unsigned)(y == 0 ? G.ny - 1 : y - 1), yp = nx * (unsigned)(y == G.ny - 1 ? 0 : y + 1);
  const unsigned xc = (unsigned)x, yc = nx * (unsigned)y;
  const int z0 = (int)blockIdx.z * G.zc, z1 = min(G.nz, z0 + G.zc);
  float4 pzm = ld4(psi_in + xc + yc + nxy * (unsigned)(z0 == 0 ? G.nz - 1 : z0 - 1));
  float4 pzc = ld4(psi_in + xc + yc + nxy * (unsigned)z0);
  // two planes per round, all loads issued before any update (planes past
  // the run repeat its last plane and are not stored)
  constexpr int U = 2;
  for (int z = z0; z < z1; z += U) {
    float4 zn[U], vym[U], vyp[U], sv[U];
    float lx[U], rx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int zz = min(z + u, z1 - 1);
      const unsigned oz = nxy * (unsigned)zz, ozp = nxy * (unsigned)(zz == G.nz - 1 ? 0 : zz + 1);
      zn[u] = ld4(psi_in + xc + yc + ozp);
      vym[u] = ld4(psi_in + xc + ym + oz);
      vyp[u] = ld4(psi_in + xc + yp + oz);
      sv[u] = ld4(s0 + xc + yc + oz);
      lx[u] = psi_in[xm + yc + oz];
      rx[u] = psi_in[xp + yc + oz];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (z + u < z1) {
        float4 o;
        {
          const float nm[3] = {lx[u], vym[u].x, pzm.x}, np[3] = {pzc.y, vyp[u].x, zn[u].x};
          o.x = liu_godunov<3>(pzc.x, nm, np, sv[u].x);
        }
        {
          const float nm[3] = {pzc.x, vym[u].y, pzm.y}, np[3] = {pzc.z, vyp[u].y, zn[u].y};
          o.y = liu_godunov<3>(pzc.y, nm, np, sv[u].y);
        }
        {
          const float nm[3] = {pzc.y, vym[u].z, pzm.z}, np[3] = {pzc.w, vyp[u].z, zn[u].z};
          o.z = liu_godunov<3>(pzc.z, nm, np, sv[u].z);
        }
        {
          const float nm[3] = {pzc.z, vym[u].w, pzm.w}, np[3] = {rx[u], vyp[u].w, zn[u].w};
          o.w = liu_godunov<3>(pzc.w, nm, np, sv[u].w);
        }
        *reinterpret_cast<float4*>(psi_out + xc + yc + nxy * (unsigned)(z + u)) = o;
        pzm = pzc;
        pzc = zn[u];
      }
    }
  }
}

// lambda and the (1 - lambda)-weighted integrals I1, I2 (compensated FP32 per
// thread, FP64 across threads, one atomic per block into acc).
template <int DIM>
__global__ void __launch_bounds__(kThreads) liu_gamma_kernel(const StepArgs a, const float* psi, double* acc,
                                                             PassGeo<DIM> G) {
  const DevParams& P = a.p;
  const LiuWork W = liu_work(a.work, a.N);
  const float dmin = 3.0f * P.W_xi;
  float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;   // per-thread compensated FP32 sums
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    const float lam = fabsf(psi[c]) < dmin ? 1.0f : 0.0f;
    W.lam[c] = lam;
    if (lam == 0.0f) {
      const float ps = W.phis[c];
      comp_add(h1, l1, P.four_beta_over_kappa * (ps - P.phiH) * (ps - P.phiL) * (ps - P.phi0));
      comp_add(h2, l2, (P.phiH - ps) * (ps - P.phiL));
    }
  });
  const double s1 = warp_sum((double)h1 + (double)l1);
  const double s2 = warp_sum((double)h2 + (double)l2);
  __shared__ double sh[2 * (kThreads / 32)];
  const int tid = threadIdx.x + kPassTX * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    sh[2 * warp] = s1;
    sh[2 * warp + 1] = s2;
  }
  __syncthreads();
  if (tid == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t1 += sh[2 * w];
      t2 += sh[2 * w + 1];
    }
    atomicAdd(acc, t1);
    atomicAdd(acc + 1, t2);
  }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) liu_phi_kernel(const StepArgs a, const double* acc, PassGeo<DIM> G) {
  const DevParams& P = a.p;
  const LiuWork W = liu_work(a.work, a.N);
  const double I2 = acc[1];
  const float gamma = I2 != 0.0 ? (float)(acc[0] / I2) : 0.0f;
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const float ps = W.phis[cl.c];
    W.phi[cl.c] = ps + 0.5f * (1.0f - W.lam[cl.c]) * nonlocal_R<FAM_LIU>(P, ps, gamma);
  });
}

// Collision (Liang2018 with Eq. Liu_G's mix), streaming and observables.
template <int DIM>
__global__ void __launch_bounds__(kThreads) liu_collide_kernel(const StepArgs a, const double* acc, PassGeo<DIM> G) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  using LS = typename Lattices<DIM>::S;
  constexpr bool SKIP0 = DIM == 3;
  const DevParams& P = a.p;
  const LiuWork W = liu_work(a.work, a.N);
  const float* gs = static_cast<const float*>(a.g_src);
  float* gd = static_cast<float*>(a.g_dst);
  float* fb = static_cast<float*>(a.f);
  const double I2 = acc[1];
  const float gamma = I2 != 0.0 ? (float)(acc[0] / I2) : 0.0f;
  __shared__ double s_red[(kThreads / 32) * 10];
  if (a.obs_zero != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    obs_zero_slot(a.obs_zero);
  ObsPartial obs;
  obs_init(obs);
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const unsigned c = cl.c;
    const int x = cl.x, y = cl.y, z = cl.z;
    // next plane: lanes 0..QG-1 the g lines, then the f lines, then the
    // rows of phi, lambda, phi* and phi u
    const long long rn = next_plane_row<DIM>(G, cl);
    if (rn >= 0) {
      const int l = threadIdx.x;
      if (l < LG::Q) prefetch_l2(group_line<LG>(gs, rn, l));
      else if (l < LG::Q + LF::Q) prefetch_l2(group_line<LF>(fb, rn, l - LG::Q));
      else if (l == LG::Q + LF::Q) prefetch_l2(W.phi + rn);
      else if (l == LG::Q + LF::Q + 1) prefetch_l2(W.lam + rn);
      else if (l == LG::Q + LF::Q + 2) prefetch_l2(W.phis + rn);
      else if (l < LG::Q + LF::Q + 3 + DIM) prefetch_l2(a.phiu + (size_t)(l - LG::Q - LF::Q - 3) * a.N + rn);
    }
    float nb[LS::Q];
#pragma unroll
    for (int q = 0; q < LS::Q; ++q) nb[q] = W.phi[cl.nb(LS::ex(q), LS::ey(q), LS::ez(q))];
    const float pc = nb[0];
    float gp[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) gp[k] = Sym<LS>::grad(nb, k);
    const float lp = Sym<LS>::lap(nb, pc);
    float g[LG::Q], f[LF::Q], phiu[DIM];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) g[q] = (SKIP0 && q == 0) ? 0.0f : gs[pop_ix<LG>(q, (unsigned)c)];
#pragma unroll
    for (int q = 0; q < LF::Q; ++q)
      f[q] = a.parity == 0 ? fb[pop_ix<LF>(q, (unsigned)c)]
                           : fb[pop_ix<LF>(LF::opp(q), cl.nb(-LF::ex(q), -LF::ey(q), -LF::ez(q)))];
#pragma unroll
    for (int d = 0; d < DIM; ++d) phiu[d] = a.phiu[d * a.N + c];
    float u[DIM], rho, p;
    const float lam = W.lam[c];
    Cell<FAM_LIU, DIM>::collide(P, g, f, pc, W.phis[c], gp, lp, 0.0f, 0.0f, phiu, gamma, u, rho, p, lam);
    {
      comp_add(obs.s_hi, obs.s_lo, pc);
      const float fr = (pc - P.phiL) * P.inv_dphi;
      float usq = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) usq += u[k] * u[k];
      obs.vs += fr;
      obs.ke += 0.5f * rho * usq;
      obs.cx += (float)x * fr;
      obs.cy += (float)y * fr;
      if (DIM == 3) obs.cz += (float)z * fr;
      obs.count += (pc > P.phi0) ? 1u : 0u;
      obs.mx = fmaxf(obs.mx, pc);
      obs.mn = fminf(obs.mn, pc);
    }
    if (a.macro) {
      a.out_phi[c] = pc;
#pragma unroll
      for (int k = 0; k < DIM; ++k) a.out_u[k * a.N + c] = u[k];
      a.out_p[c] = p;
      return;
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) a.phiu[k * a.N + c] = phiu[k];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q)
      if (!(SKIP0 && q == 0)) gd[pop_ix<LG>(q, cl.nb(LG::ex(q), LG::ey(q), LG::ez(q)))] = g[q];
#pragma unroll
    for (int q = 0; q < LF::Q; ++q) {
      if (a.parity == 0) fb[pop_ix<LF>(LF::opp(q), (unsigned)c)] = f[q];
      else fb[pop_ix<LF>(q, cl.nb(LF::ex(q), LF::ey(q), LF::ez(q)))] = f[q];
    }
  });
  if (obs.mn <= obs.mx) {
    const float r1 = P.rhoL + P.drho_dphi * (obs.mn - P.phiL), r2 = P.rhoL + P.drho_dphi * (obs.mx - P.phiL);
    if (!(isfinite(obs.s_hi) && isfinite(obs.ke) && r1 > 0.0f && r2 > 0.0f)) obs.bad = 1u;
  }
  obs_block_commit(obs, a.obs_slot, s_red);
}

template <int DIM>
void liu_step_dim(const StepArgs& a, cudaStream_t s) {
  const PassGeo<DIM> G = pass_geo<DIM>(a.p.nx, a.p.ny, a.p.nz, num_sms());
  const dim3 grid = G.grid(), block(kPassTX, kPassTY);
  const LiuWork W = liu_work(a.work, a.N);
  liu_predict_kernel<DIM><<<grid, block, 0, s>>>(a, G);
  const int nit = (int)ceilf(2.0f * 3.0f * a.p.W_xi);
  const float* in = W.psia;
  float* out = W.psib;
  auto swap = [&] {
    const float* t = out;
    out = const_cast<float*>(in);
    in = t;
  };
  // the four-cells-per-thread sweep where rows are whole 16-byte groups
  const bool four = DIM == 3 && a.p.nx % 4 == 0;
  const Reinit4Geo G4 = reinit4_geo(a.p.nx, a.p.ny, a.p.nz, num_sms());
  for (int it = 0; it < nit; ++it) {
    if (four) liu_reinit4_kernel<<<G4.grid(), block, 0, s>>>(in, out, W.s0, G4);
    else liu_reinit_kernel<DIM><<<grid, block, 0, s>>>(in, out, W.s0, G);
    swap();
  }
  // gamma_acc holds this step's (I1, I2) pair, zeroed here
  double* acc = const_cast<double*>(a.gamma_acc);
  cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
  liu_gamma_kernel<DIM><<<grid, block, 0, s>>>(a, in, acc, G);
  liu_phi_kernel<DIM><<<grid, block, 0, s>>>(a, acc, G);
  liu_collide_kernel<DIM><<<grid, block, 0, s>>>(a, acc, G);
}

}  // namespace

void step_liu2023(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  (void)storage;   // FP32 only (validated by the API)
  if (dim == 2) liu_step_dim<2>(a, s);
  else liu_step_dim<3>(a, s);
}

void init_liu2023(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_LIU>(dim, storage, a, s);
}

}  // namespace pflb
