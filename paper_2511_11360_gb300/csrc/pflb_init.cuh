// Initial state: equilibrium populations for given phi and u with p = 0.
#pragma once

#include "pflb_step.cuh"

namespace pflb {

// One thread per cell (grid-stride). g goes to the source array in the
// canonical slot order; f goes to the AA array in the even-step layout
// (slot q of the cell holds f_q); Liang2014 and Liang2018 also store phi*u.
template <int FAM, int DIM, typename T, int LAT = 0>
__global__ void init_kernel(const InitArgs args) {
  using LG = typename Lattices<DIM, LAT>::G;
  using LF = typename Lattices<DIM, LAT>::F;
  using LS = typename Lattices<DIM, LAT>::S;
  constexpr int QG = LG::Q, QF = LF::Q, QS = LS::Q;
  const DevParams& P = args.p;
  const long long N = args.N;
  const int nx = P.nx, ny = P.ny, nz = (DIM == 3) ? P.nz : 1;
  T* g = static_cast<T*>(args.g);
  T* f = static_cast<T*>(args.f);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx);
    const int y = (int)((idx / nx) % ny);
    const int z = (int)(idx / ((long long)nx * ny));
    const float phi = args.phi0[idx];
    float u[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) u[k] = args.u0 ? args.u0[(long long)k * N + idx] : 0.0f;
    const float rho = P.rhoL + P.drho_dphi * (phi - P.phiL);
    float usq = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) usq += u[k] * u[k];

    float mu = 0.0f;
    if constexpr (FAM == FAM_LIANG) {
      // Chemical potential of phi0, Eq. (chemical_potential), Sec. III stencil.
      float nb[QS];
      nb[0] = phi;
#pragma unroll
      for (int q = 1; q < QS; ++q) {
        int xn = x + LS::ex(q), yn = y + LS::ey(q), zn = z + LS::ez(q);
        xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
        if (P.walls) yn = yn < 0 ? -1 - yn : (yn >= ny ? 2 * ny - 1 - yn : yn);
        else yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
        zn = zn < 0 ? zn + nz : (zn >= nz ? zn - nz : zn);
        nb[q] = args.phi0[xn + (long long)nx * (yn + (long long)ny * zn)];
      }
      mu = P.beta4 * (phi - P.phiH) * (phi - P.phiL) * (phi - P.phi0) - P.kappa * Sym<LS>::lap(nb, phi);
    }

#pragma unroll
    for (int q = 0; q < QG; ++q) {
      float eu = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) eu += (float)ecomp<LG>(q, k) * u[k];
      const float w = LG::w(q);
      float geq;
      if constexpr (FAM == FAM_FAKHARI) geq = w * phi * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * usq);
      else if constexpr (FAM == FAM_LIANG) geq = (q == 0) ? phi + (w - 1.0f) * P.eta * mu : w * (P.eta * mu + 3.0f * phi * eu);
      else geq = w * phi * (1.0f + 3.0f * eu);
      pop_store<T, LG>(g + pop_ix<LG>(q, (unsigned)idx), q, geq, P.gref);
    }
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      float eu = 0.0f;
#pragma unroll
      for (int k = 0; k < DIM; ++k) eu += (float)ecomp<LF>(q, k) * u[k];
      const float w = LF::w(q);
      float feq;
      if constexpr (fam_phiu(FAM))   // pressure-based f_eq with p = 0 (Eqs. liang_feq, liang2_feq)
        feq = (q == 0) ? rho * w * (-1.5f * usq) : rho * w * (3.0f * eu + 4.5f * eu * eu - 1.5f * usq);
      else
        feq = w * (3.0f * eu + 4.5f * eu * eu - 1.5f * usq);
      pop_store<T, LF>(f + pop_ix<LF>(q, (unsigned)idx), q, feq, 0.0f);
    }
    if constexpr (fam_phiu(FAM)) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) args.phiu[(long long)k * N + idx] = phi * u[k];
    }
  }
}

template <int FAM, int DIM, typename T, int LAT = 0>
void launch_init(const InitArgs& a, cudaStream_t s) {
  const long long blocks = (a.N + 255) / 256;
  init_kernel<FAM, DIM, T, LAT><<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(a);
}

// Per-family dispatch over dimension and storage (instantiated once per
// family translation unit).
template <int FAM>
void step_dispatch(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  if (dim == 2) {
    if (storage == 0) launch_step<FAM, 2, float>(a, s);
    else if (storage == 1) launch_step<FAM, 2, __half>(a, s);
    else launch_step<FAM, 2, __nv_bfloat16>(a, s);
  } else if (a.p.lat == 0) {
    if (storage == 0) launch_step<FAM, 3, float>(a, s);
    else if (storage == 1) launch_step<FAM, 3, __half>(a, s);
    else launch_step<FAM, 3, __nv_bfloat16>(a, s);
  } else {
    if (storage == 0) launch_step<FAM, 3, float, 1>(a, s);
    else if (storage == 1) launch_step<FAM, 3, __half, 1>(a, s);
    else launch_step<FAM, 3, __nv_bfloat16, 1>(a, s);
  }
}

template <int FAM>
void init_dispatch(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  if (dim == 2) {
    if (storage == 0) launch_init<FAM, 2, float>(a, s);
    else if (storage == 1) launch_init<FAM, 2, __half>(a, s);
    else launch_init<FAM, 2, __nv_bfloat16>(a, s);
  } else if (a.p.lat == 0) {
    if (storage == 0) launch_init<FAM, 3, float>(a, s);
    else if (storage == 1) launch_init<FAM, 3, __half>(a, s);
    else launch_init<FAM, 3, __nv_bfloat16>(a, s);
  } else {
    if (storage == 0) launch_init<FAM, 3, float, 1>(a, s);
    else if (storage == 1) launch_init<FAM, 3, __half, 1>(a, s);
    else launch_init<FAM, 3, __nv_bfloat16, 1>(a, s);
  }
}

}  // namespace pflb
