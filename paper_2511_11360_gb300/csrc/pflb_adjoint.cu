// C ABI of the adjoint (declared in include/pflb.h): gradients of a droplet
// objective of the final state with respect to M, sigma, W and the initial
// velocity, by a reverse sweep with sqrt(N) checkpointing and recomputation.
#include <cmath>
#include <cstring>
#include <vector>

#include "pflb_adjoint_kernels.cuh"
#include "pflb_internal.h"

using namespace pflb;

namespace {

#define ACU(h, call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      rc = handle_fail((h), PFLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
      goto done;                                                                              \
    }                                                                                         \
  } while (0)

int grid_for(long long N) {
  const long long want = (N + 255) / 256;
  const long long cap = 8LL * num_sms();
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int DIM>
void launch_reverse_step(const AdjArgs& a, cudaStream_t s) {
  const int grid = grid_for(a.N);
  const PassGeo<DIM> G{a.nx, a.ny, a.nz, a.zc};
  const dim3 wgrid = G.grid(), wblock(kPassTX, kPassTY);
  adj_phi_kernel<DIM><<<grid, 256, 0, s>>>(a.state, const_cast<float*>(a.phi), a.N);
  adj_local_kernel<DIM><<<wgrid, wblock, 0, s>>>(a);
  adj_stencil_kernel<DIM><<<wgrid, wblock, 0, s>>>(a);
}

}  // namespace

extern "C" int pflb_adjoint(pflb_handle* h, int64_t nsteps, int32_t checkpoint_every, const pflb_obs_weights* w,
                            pflb_grads* out, float* du0) {
  if (!h || !w || !out || nsteps < 1 || checkpoint_every < 0)
    return handle_fail(h, PFLB_EINVAL, "pflb_adjoint: invalid argument");
  if (h->status != PFLB_OK && h->status != PFLB_EUNSTABLE) return h->status;
  const pflb_params& p = h->prm;
  if (h->family != PFLB_CAC_FAKHARI2017)
    return handle_fail(h, PFLB_EINVAL, "pflb_adjoint covers the Fakhari2017 family");
  if (h->QF != (h->dim == 2 ? 9 : 19))
    return handle_fail(h, PFLB_EINVAL, "pflb_adjoint covers the D2Q9 and D3Q19 hydrodynamic lattices (BGK)");
  if (p.bc_y != 0) return handle_fail(h, PFLB_EINVAL, "pflb_adjoint covers periodic domains");
  if (h->storage != PFLB_FP32) return handle_fail(h, PFLB_EINVAL, "pflb_adjoint needs FP32 storage");
  if (p.rho_H != p.rho_L) return handle_fail(h, PFLB_EINVAL, "pflb_adjoint covers density ratio 1");
  if (p.visc_interp != 0) return handle_fail(h, PFLB_EINVAL, "pflb_adjoint covers the linear viscosity interpolation");
  if (p.freeze_phi) return handle_fail(h, PFLB_EINVAL, "pflb_adjoint: freeze_phi is not differentiated");
  if (!h->initialized || h->step != 0)
    return handle_fail(h, PFLB_EINVAL, "pflb_adjoint starts from the state pflb_init made (step 0)");
  if (!(w->eps_v > 0.0)) return handle_fail(h, PFLB_EINVAL, "eps_v must be > 0");
  const NvtxRange range("pflb_adjoint");

  const long long N = h->N;
  const int dim = h->dim, QG = h->QG, QF = h->QF;
  const long long S = (long long)(QG + QF) * N;      // canonical state floats
  long long K = checkpoint_every > 0 ? checkpoint_every : (long long)std::ceil(std::sqrt((double)nsteps));
  if (K > nsteps) K = nsteps;
  const long long nck = (nsteps + K - 1) / K;        // checkpoints at 0, K, 2K, ...
  cudaStream_t st = h->stream;
  int rc = PFLB_OK;
  float *ck = nullptr, *seg = nullptr, *fin = nullptr, *lam0 = nullptr, *lam1 = nullptr, *phi = nullptr,
        *aux = nullptr, *du = nullptr;
  double* acc = nullptr;
  DevObs* ring = nullptr;   // the forward sweep's observables records, restored at the end
  const size_t ring_bytes = (size_t)(h->obs_cap + 1) * sizeof(DevObs);
  double hacc[8];
  AdjArgs a;
  const bool du_dev = du0 != nullptr && [&] {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, du0) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  }();
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = handle_fail(h, PFLB_ENOMEM, "pflb_adjoint: cudaMalloc of %zu bytes failed", bytes);
      return false;
    }
    return true;
  };
  if (!alloc((void**)&ck, (size_t)(nck * S) * sizeof(float)) || !alloc((void**)&seg, (size_t)(K * S) * sizeof(float)) ||
      !alloc((void**)&fin, (size_t)S * sizeof(float)) || !alloc((void**)&lam0, (size_t)S * sizeof(float)) ||
      !alloc((void**)&lam1, (size_t)S * sizeof(float)) || !alloc((void**)&phi, (size_t)N * sizeof(float)) ||
      !alloc((void**)&aux, (size_t)(dim + 2) * N * sizeof(float)) || !alloc((void**)&acc, 8 * sizeof(double)) ||
      !alloc((void**)&ring, ring_bytes))
    goto done;
  if (du0 && !du_dev && !alloc((void**)&du, (size_t)dim * N * sizeof(float))) goto done;
  ACU(h, cudaMemsetAsync(acc, 0, 8 * sizeof(double), st));

  // ---- forward sweep, keeping every K-th state
  for (long long c = 0; c < nck; ++c) {
    if ((rc = handle_canon(h, ck + c * S, 1))) goto done;
    const long long n = (c + 1) * K < nsteps ? K : nsteps - c * K;
    if ((rc = pflb_step(h, n)) != PFLB_OK && rc != PFLB_EUNSTABLE) goto done;
    rc = PFLB_OK;
  }
  if ((rc = handle_canon(h, fin, 1))) goto done;
  ACU(h, cudaMemcpyAsync(ring, h->obs, ring_bytes, cudaMemcpyDeviceToDevice, st));

  // ---- objective of the final state and the seed adjoint
  {
    const float phi0 = (float)(0.5 * (p.phi_H + p.phi_L));
    const float inv_eps = (float)(1.0 / w->eps_v);
    const int grid = grid_for(N);
    if (dim == 2) adj_phi_kernel<2><<<grid, 256, 0, st>>>(fin, phi, N);
    else adj_phi_kernel<3><<<grid, 256, 0, st>>>(fin, phi, N);
    adj_objective_kernel<<<grid, 256, 0, st>>>(phi, N, p.nx, p.ny, phi0, inv_eps, acc + 3);
    ACU(h, cudaGetLastError());
    ACU(h, cudaMemcpyAsync(hacc, acc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACU(h, cudaStreamSynchronize(st));
    const double Ssum = hacc[3];
    if (!(std::fabs(Ssum) > 0.0) || !std::isfinite(Ssum)) {
      rc = handle_fail(h, PFLB_EUNSTABLE, "pflb_adjoint: sum of phi of the final state is %g", Ssum);
      goto done;
    }
    double cen[3] = {hacc[4] / Ssum, hacc[5] / Ssum, hacc[6] / Ssum};
    out->vol_smooth = hacc[7];
    double J = w->w_vol * hacc[7], shift = 0.0;
    for (int k = 0; k < 3; ++k) {
      out->centroid[k] = k < dim ? cen[k] : 0.0;
      if (k < dim) {
        J += w->w_cen[k] * cen[k];
        shift -= w->w_cen[k] * cen[k];
      }
    }
    out->J = J;
    const float wz = dim == 3 ? (float)w->w_cen[2] : 0.0f;
    if (dim == 2)
      adj_seed_kernel<2><<<grid, 256, 0, st>>>(phi, lam0, N, p.nx, p.ny, phi0, inv_eps, (float)w->w_vol,
                                               (float)w->w_cen[0], (float)w->w_cen[1], 0.0f, (float)(1.0 / Ssum),
                                               (float)(shift / Ssum));
    else
      adj_seed_kernel<3><<<grid, 256, 0, st>>>(phi, lam0, N, p.nx, p.ny, phi0, inv_eps, (float)w->w_vol,
                                               (float)w->w_cen[0], (float)w->w_cen[1], wz, (float)(1.0 / Ssum),
                                               (float)(shift / Ssum));
    ACU(h, cudaGetLastError());
  }

  // ---- reverse sweep, segment by segment from the last checkpoint
  memset(&a, 0, sizeof(a));
  a.p = h->dp;
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = dim == 3 ? p.nz : 1;
  a.zc = dim == 3 ? pass_geo<3>(p.nx, p.ny, p.nz, num_sms()).zc : 1;
  a.N = N;
  a.phi = phi;
  a.aux = aux;
  a.acc = acc;
  {
    const double dphi = p.phi_H - p.phi_L;
    a.dbeta4_dsigma = (float)(48.0 / (p.W * std::pow(std::fabs(dphi), 4)));
    a.dkappa_dsigma = (float)(3.0 * p.W / (2.0 * dphi * dphi));
    a.W = (float)p.W;
  }
  {
    float* lin = lam0;
    float* lout = lam1;
    for (long long c = nck - 1; c >= 0; --c) {
      const long long n0 = c * K, n1 = (c + 1) * K < nsteps ? (c + 1) * K : nsteps;
      // Recompute the states n0 .. n1-1 of this segment from its checkpoint.
      h->step = n0;
      if ((rc = handle_canon(h, ck + c * S, 0))) goto done;
      for (long long n = n0; n < n1; ++n) {
        if ((rc = handle_canon(h, seg + (n - n0) * S, 1))) goto done;
        if (n + 1 < n1) {
          if ((rc = pflb_step(h, 1)) != PFLB_OK && rc != PFLB_EUNSTABLE) goto done;
          rc = PFLB_OK;
        }
      }
      for (long long n = n1 - 1; n >= n0; --n) {
        a.state = seg + (n - n0) * S;
        a.lam_in = lin;
        a.lam_out = lout;
        if (dim == 2) launch_reverse_step<2>(a, st);
        else launch_reverse_step<3>(a, st);
        ACU(h, cudaGetLastError());
        float* t = lin;
        lin = lout;
        lout = t;
      }
    }
    // lin now holds the adjoint of the initial state.
    if (du0) {
      float* dst = du_dev ? du0 : du;
      const int grid = grid_for(N);
      if (dim == 2) adj_du0_kernel<2><<<grid, 256, 0, st>>>(ck, lin, dst, N);
      else adj_du0_kernel<3><<<grid, 256, 0, st>>>(ck, lin, dst, N);
      ACU(h, cudaGetLastError());
      if (!du_dev)
        ACU(h, cudaMemcpyAsync(du0, du, (size_t)dim * N * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
  }
  ACU(h, cudaMemcpyAsync(hacc, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  // Leave the handle at the final state, as pflb_step(h, nsteps) would.
  h->step = nsteps;
  if ((rc = handle_canon(h, fin, 0))) goto done;
  ACU(h, cudaMemcpyAsync(h->obs, ring, ring_bytes, cudaMemcpyDeviceToDevice, st));
  ACU(h, cudaStreamSynchronize(st));
  out->dJ_dM = hacc[0];
  out->dJ_dsigma = hacc[1];
  out->dJ_dW = hacc[2];
  out->steps = nsteps;
  out->checkpoint_every = (int32_t)K;
  out->checkpoints = (int32_t)nck;

done:
  cudaStreamSynchronize(st);
  cudaFree(ck);
  cudaFree(seg);
  cudaFree(fin);
  cudaFree(lam0);
  cudaFree(lam1);
  cudaFree(phi);
  cudaFree(aux);
  cudaFree(acc);
  cudaFree(du);
  cudaFree(ring);
  return rc;
}
