// Reverse-mode (adjoint) kernels of the conservative Allen-Cahn step
// (Fakhari2017, Sec. II C 1) on a periodic grid at density ratio 1.
//
// Forward step, per cell x, from the post-streaming populations g_a, f_b:
//   phi = sum g;  grad phi, lap phi by the Sec. III stencils;
//   nu(phi) linear, itau = 1/(3 nu + 1/2), fw = 1 - itau/2;
//   mu = 4 beta (phi-phi_H)(phi-phi_L)(phi-phi_0) - kappa lap phi;
//   F_o = mu grad phi + F_b,  u = (sum e f + F_o/(2 rho)) / (1 - A/2),
//   F = F_o + A rho u                          Eq. (fakhari_velocity_update);
//   g*_a = g_a - (g_a - g_eq,a)/tau_phi + (1 - 1/(2 tau_phi)) G_a,
//     g_eq,a = w_a phi (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u)     Eq. (fakhari_geq),
//     G_a = w_a e_a . [k (phi_H-phi)(phi-phi_L) grad phi / sqrt(|grad phi|^2 + eps^2)]
//                                          Eq. (fakhari_G_modified), Reading R6;
//   f*_b = f_b - (f_b - f_eq,b) itau + fw 3 w_b e_b.F/rho,
//     f_eq,b = w_b (sum f + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u)     Eq. (fakhari_feq);
//   push streaming g_a(x + e_a) <- g*_a(x), f likewise.
// At density ratio 1 the pressure and viscous forces vanish (grad rho = 0).
//
// Reverse sweep of one step, given the adjoints lambda of the next state:
//   1. adj_local: pull lambda* = lambda(x + e), differentiate the local
//      update of x, write the direct part of lambda_g (through g_a itself),
//      all of lambda_f, and the cell's sensitivities to phi(x), grad phi(x)
//      and lap phi(x); add the parameter sensitivities (tau_phi <- M;
//      beta, kappa <- sigma, W; k = 4/(W dphi) <- W) to FP64 accumulators.
//   2. adj_stencil: phi(y) enters grad phi and lap phi of the cells
//      y - e_q; apply the transposed stencils and add the total phi
//      sensitivity to every lambda_g,a(y) (phi = sum g).
// Arithmetic is FP32; the parameter sums are FP64.
#pragma once

#include "pflb_pass.cuh"
#include "pflb_step.cuh"

namespace pflb {

struct AdjArgs {
  DevParams p;
  int nx, ny, nz;
  int zc;                 // planes per block of the (x, y)-tile walk
  long long N;
  const float* state;     // canonical state of step n: g (QG x N) then f (QF x N)
  const float* phi;       // phi of that state (N)
  const float* lam_in;    // adjoint of step n+1 (QG + QF) x N
  float* lam_out;         // adjoint of step n   (QG + QF) x N
  float* aux;             // (d + 2) x N: d phi, d grad phi, d lap phi of each cell
  double* acc;            // dJ/dM, dJ/dsigma, dJ/dW accumulators
  float dbeta4_dsigma, dkappa_dsigma;  // beta4 and kappa are linear in sigma
  float W;
};

template <typename L>
__device__ __forceinline__ float edot(int q, const float* v, int dim) {
  float s = 0.0f;
  if (L::ex(q)) s += (float)L::ex(q) * v[0];
  if (dim > 1 && L::ey(q)) s += (float)L::ey(q) * v[1];
  if (dim > 2 && L::ez(q)) s += (float)L::ez(q) * v[2];
  return s;
}

template <typename L>
__device__ __forceinline__ int ecomp_adj(int q, int k) {
  return k == 0 ? L::ex(q) : (k == 1 ? L::ey(q) : L::ez(q));
}

__device__ __forceinline__ void block_add3(double a, double b, double c, double* acc) {
  __shared__ double s[3 * 32];
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nthreads = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    s[3 * warp] = a;
    s[3 * warp + 1] = b;
    s[3 * warp + 2] = c;
  }
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (nthreads >> 5); ++w) {
      t0 += s[3 * w];
      t1 += s[3 * w + 1];
      t2 += s[3 * w + 2];
    }
    atomicAdd(&acc[0], t0);
    atomicAdd(&acc[1], t1);
    atomicAdd(&acc[2], t2);
  }
  __syncthreads();
}

// phi = sum g of a canonical state.
template <int DIM>
__global__ void adj_phi_kernel(const float* __restrict__ state, float* __restrict__ phi, long long N) {
  using LG = typename Lattices<DIM>::G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float g[LG::Q];
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) g[q] = state[q * N + i];
    phi[i] = phi_star<LG, (DIM == 3)>(g);
  }
}

template <int DIM>
__global__ void __launch_bounds__(256, 2) adj_local_kernel(const AdjArgs a) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  using LS = typename Lattices<DIM>::S;
  constexpr int QG = LG::Q, QF = LF::Q, QS = LS::Q;
  const DevParams& P = a.p;
  const long long N = a.N;
  double accM = 0.0, accS = 0.0, accW = 0.0;
  const PassGeo<DIM> G{a.nx, a.ny, a.nz, a.zc};
  const int lane = threadIdx.x;   // the x lane: a warp covers 32 consecutive cells of one row
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const long long i = cl.c;
    // The cell is latency-bound (one cell per thread, many dependent loads):
    // ask L2 for the rows of the next plane now. Lane q < QG + QF takes the
    // row of array q of the state and of lambda_in (the pulled lambda of the
    // next plane mostly lies in that row).
    if (DIM == 3 && cl.z + 1 < a.nz && lane < QG + QF) {
      const long long rn = (long long)(cl.c - (unsigned)lane) + (long long)a.nx * a.ny + (long long)lane * N;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.state + rn));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.lam_in + rn));
    }
    // ---- forward recomputation at the cell
    const float phi = a.phi[i];
    float gp[3] = {0.0f, 0.0f, 0.0f}, lp = 0.0f;
#pragma unroll
    for (int q = 1; q < QS; ++q) {
      const float nb = a.phi[cl.nb(LS::ex(q), LS::ey(q), LS::ez(q))];
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        if (ecomp_adj<LS>(q, k)) gp[k] += LS::w(q) * (float)ecomp_adj<LS>(q, k) * nb;
      lp += LS::w(q) * (nb - phi);
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) gp[k] *= 3.0f;
    lp *= 6.0f;
    float sumf = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      const float fq = a.state[(QG + q) * N + i];
      sumf += fq;
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        if (ecomp_adj<LF>(q, k)) mom[k] += (float)ecomp_adj<LF>(q, k) * fq;
    }
    const float rho = P.rhoL;
    const float inv_rho = 1.0f / rho;
    const float nu = P.nuL + (P.nuH - P.nuL) * (phi - P.phiL) * P.inv_dphi;
    const float itau = 1.0f / (3.0f * nu + 0.5f);
    const float fw = 1.0f - 0.5f * itau;
    const float d1 = phi - P.phiH, d2 = phi - P.phiL, d3 = phi - P.phi0;
    const float P3 = d1 * d2 * d3;
    const float dP3 = d2 * d3 + d1 * d3 + d1 * d2;
    const float mu = P.beta4 * P3 - P.kappa * lp;
    const float A = P.lundA;
    const float inv_1mA = 1.0f / (1.0f - 0.5f * A);
    float Fo[3], u[3], F[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      Fo[k] = mu * gp[k] + rho * P.grav[k] + P.fdens[k];
      u[k] = (mom[k] + 0.5f * inv_rho * Fo[k]) * inv_1mA;
      F[k] = Fo[k] + A * rho * u[k];
    }
    float usq = 0.0f, g2 = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      usq += u[k] * u[k];
      g2 += gp[k] * gp[k];
    }
    const float r = rsqrtf(g2 + P.eps2);
    const float Pp = (P.phiH - phi) * (phi - P.phiL);
    const float kk = P.counter_k;
    const float s = kk * Pp * r;
    float flux[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) flux[k] = s * gp[k];
    const float itp = P.inv_tau_phi, sw = P.src_w_phi;

    // ---- reverse
    float phibar = 0.0f, ubar[3] = {0.0f, 0.0f, 0.0f}, fluxbar[3] = {0.0f, 0.0f, 0.0f};
    float gpbar[3] = {0.0f, 0.0f, 0.0f};
    float tphibar = 0.0f;
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      const long long src = cl.nb(LG::ex(q), LG::ey(q), LG::ez(q));
      const float ls = a.lam_in[q * N + src];          // lambda of g*_q(x)
      const float w = LG::w(q);
      const float gq = a.state[q * N + i];
      const float eu = edot<LG>(q, u, DIM);
      const float Aq = 1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * usq;
      const float geq = w * phi * Aq;
      const float Gq = w * edot<LG>(q, flux, DIM);
      a.lam_out[q * N + i] = ls * (1.0f - itp);
      const float geqbar = ls * itp;
      const float Gbar = ls * sw;
      phibar += geqbar * w * Aq;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const float e = (float)ecomp_adj<LG>(q, k);
        ubar[k] += geqbar * w * phi * (3.0f * e + 9.0f * eu * e - 3.0f * u[k]);
        fluxbar[k] += Gbar * w * e;
      }
      tphibar += ls * ((gq - geq) + 0.5f * Gq) * itp * itp;
    }
    float itaubar = 0.0f, sumfbar = 0.0f, Ftbar[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      const long long src = cl.nb(LF::ex(q), LF::ey(q), LF::ez(q));
      const float ls = a.lam_in[(QG + q) * N + src];   // lambda of f*_q(x)
      const float w = LF::w(q);
      const float eu = edot<LF>(q, u, DIM);
      const float feq = w * (sumf + 3.0f * eu + 4.5f * eu * eu - 1.5f * usq);
      const float Fq = 3.0f * w * edot<LF>(q, F, DIM) * inv_rho;
      const float feqbar = ls * itau;
      const float Fqbar = ls * fw;
      sumfbar += feqbar * w;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const float e = (float)ecomp_adj<LF>(q, k);
        ubar[k] += feqbar * w * (3.0f * e + 9.0f * eu * e - 3.0f * u[k]);
        Ftbar[k] += Fqbar * 3.0f * w * e;
      }
      // f_q read again (cached) rather than held in registers across the cell
      itaubar += ls * (-(a.state[(QG + q) * N + i] - feq) - 0.5f * Fq);
    }
    // F = F_o + A rho u; u = (mom + F_o/(2 rho)) / (1 - A/2)
    float Fobar[3], mombar[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const float Fbar = Ftbar[k] * inv_rho;
      ubar[k] += A * rho * Fbar;
      mombar[k] = ubar[k] * inv_1mA;
      Fobar[k] = Fbar + ubar[k] * inv_1mA * 0.5f * inv_rho;
    }
    // F_o = mu grad phi + F_b
    float mubar = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      mubar += Fobar[k] * gp[k];
      gpbar[k] += Fobar[k] * mu;
    }
    phibar += mubar * P.beta4 * dP3;
    const float lpbar = -P.kappa * mubar;
    const float beta4bar = mubar * P3;
    const float kappabar = -mubar * lp;
    // flux = s grad phi, s = k Pp r, r = (|grad phi|^2 + eps^2)^(-1/2)
    float sbar = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      sbar += fluxbar[k] * gp[k];
      gpbar[k] += fluxbar[k] * s;
    }
    phibar += sbar * kk * r * (P.phiH + P.phiL - 2.0f * phi);
    const float rbar = sbar * kk * Pp;
    const float r3 = r * r * r;
#pragma unroll
    for (int k = 0; k < DIM; ++k) gpbar[k] -= rbar * gp[k] * r3;
    const float kbar = sbar * Pp * r;
    // itau = 1/(3 nu + 1/2), nu linear in phi
    phibar += itaubar * (-itau * itau) * 3.0f * (P.nuH - P.nuL) * P.inv_dphi;
    // f: through sum f and sum e f
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      // lambda of f*_q(x) read again (cached) rather than held in registers
      const float ls = a.lam_in[(QG + q) * N + cl.nb(LF::ex(q), LF::ey(q), LF::ez(q))];
      float v = ls * (1.0f - itau) + sumfbar;
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        if (ecomp_adj<LF>(q, k)) v += (float)ecomp_adj<LF>(q, k) * mombar[k];
      a.lam_out[(QG + q) * N + i] = v;
    }
    a.aux[i] = phibar;
#pragma unroll
    for (int k = 0; k < DIM; ++k) a.aux[(1 + k) * N + i] = gpbar[k];
    a.aux[(1 + DIM) * N + i] = lpbar;
    // parameters: tau_phi = 3 M + 1/2; beta4, kappa linear in sigma;
    // beta4 ~ 1/W, kappa ~ W, k ~ 1/W.
    accM += 3.0 * (double)tphibar;
    accS += (double)beta4bar * a.dbeta4_dsigma + (double)kappabar * a.dkappa_dsigma;
    accW += ((double)(-beta4bar * P.beta4) + (double)(kappabar * P.kappa) - (double)(kbar * kk)) / (double)a.W;
  });
  block_add3(accM, accS, accW, a.acc);
}

// Transposed stencils: phi(y) feeds grad phi and lap phi of y - e_q.
template <int DIM>
__global__ void __launch_bounds__(256) adj_stencil_kernel(const AdjArgs a) {
  using LG = typename Lattices<DIM>::G;
  using LS = typename Lattices<DIM>::S;
  constexpr int QG = LG::Q, QS = LS::Q;
  const long long N = a.N;
  const float wrest = 1.0f - LS::w(0);
  const PassGeo<DIM> G{a.nx, a.ny, a.nz, a.zc};
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const long long i = cl.c;
    float t = a.aux[i] - 6.0f * wrest * a.aux[(1 + DIM) * N + i];
#pragma unroll
    for (int q = 1; q < QS; ++q) {
      const long long y = cl.nb(-LS::ex(q), -LS::ey(q), -LS::ez(q));
      float eg = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        if (ecomp_adj<LS>(q, k)) eg += (float)ecomp_adj<LS>(q, k) * a.aux[(1 + k) * N + y];
      t += LS::w(q) * (3.0f * eg + 6.0f * a.aux[(1 + DIM) * N + y]);
    }
#pragma unroll
    for (int q = 0; q < QG; ++q) a.lam_out[q * N + i] += t;
  });
}

// Objective pieces of a phi field: sum phi, sum x_k phi, smooth volume.
__global__ void __launch_bounds__(256) adj_objective_kernel(const float* __restrict__ phi, long long N, int nx,
                                                             int ny, float phi0, float inv_eps, double* out) {
  double s = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double p = (double)phi[i];
    const long long x = i % nx, r = i / nx, y = r % ny, z = r / ny;
    s += p;
    sx += (double)x * p;
    sy += (double)y * p;
    sz += (double)z * p;
    v += 0.5 * (1.0 + tanh(((double)phi[i] - (double)phi0) * (double)inv_eps));
  }
  __shared__ double sh[5 * 32];
  double vals[5] = {s, sx, sy, sz, v};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    vals[k] = warp_sum(vals[k]);
    if (lane == 0) sh[5 * warp + k] = vals[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[5 * w + k];
      atomicAdd(&out[k], t);
    }
  }
}

// lambda of the final state: dJ/dphi for every g population, 0 for f
// (phi = sum g of the final state, Reading R13 objective).
template <int DIM>
__global__ void adj_seed_kernel(const float* __restrict__ phi, float* __restrict__ lam, long long N, int nx, int ny,
                                float phi0, float inv_eps, float w_vol, float wx, float wy, float wz, float inv_S,
                                float shift) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const long long x = i % nx, r = i / nx, y = r % ny, z = r / ny;
    const float t = tanhf((phi[i] - phi0) * inv_eps);
    // d/dphi of w_vol V_s + sum_k w_k c_k, with c_k = sum x_k phi / S:
    // w_k (x_k - c_k) / S; shift = -sum_k w_k c_k / S.
    const float d = w_vol * 0.5f * (1.0f - t * t) * inv_eps
                  + (wx * (float)x + wy * (float)y + wz * (float)z) * inv_S + shift;
#pragma unroll
    for (int q = 0; q < LG::Q; ++q) lam[q * N + i] = d;
#pragma unroll
    for (int q = 0; q < LF::Q; ++q) lam[(LG::Q + q) * N + i] = 0.0f;
  }
}

// dJ/du0 from the adjoint of the initial state (g = g_eq(phi0, u0),
// f = f_eq(0, u0), Reading R8); phi0 = sum g and u0 = sum e f of that state.
template <int DIM>
__global__ void adj_du0_kernel(const float* __restrict__ state, const float* __restrict__ lam, float* __restrict__ du0,
                               long long N) {
  using LG = typename Lattices<DIM>::G;
  using LF = typename Lattices<DIM>::F;
  constexpr int QG = LG::Q, QF = LF::Q;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float g[QG];
    for (int q = 0; q < QG; ++q) g[q] = state[q * N + i];
    const float phi = phi_star<LG, (DIM == 3)>(g);
    float u[3] = {0.0f, 0.0f, 0.0f};
    for (int q = 0; q < QF; ++q)
      for (int k = 0; k < DIM; ++k) u[k] += (float)ecomp_adj<LF>(q, k) * state[(QG + q) * N + i];
    float ub[3] = {0.0f, 0.0f, 0.0f};
    for (int q = 0; q < QG; ++q) {
      const float l = lam[q * N + i], w = LG::w(q), eu = edot<LG>(q, u, DIM);
      for (int k = 0; k < DIM; ++k) {
        const float e = (float)ecomp_adj<LG>(q, k);
        ub[k] += l * w * phi * (3.0f * e + 9.0f * eu * e - 3.0f * u[k]);
      }
    }
    for (int q = 0; q < QF; ++q) {
      const float l = lam[(QG + q) * N + i], w = LF::w(q), eu = edot<LF>(q, u, DIM);
      for (int k = 0; k < DIM; ++k) {
        const float e = (float)ecomp_adj<LF>(q, k);
        ub[k] += l * w * (3.0f * e + 9.0f * eu * e - 3.0f * u[k]);
      }
    }
    for (int k = 0; k < DIM; ++k) du0[k * N + i] = ub[k];
  }
}

}  // namespace pflb
