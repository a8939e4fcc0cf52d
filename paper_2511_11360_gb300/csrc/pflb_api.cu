// C ABI of the coupled PF-LB step (declared in include/pflb.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pflb.h"
#include "pflb_internal.h"

using namespace pflb;

namespace pflb {

int handle_fail(pflb_handle* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
    if (h->status == PFLB_OK || code == PFLB_EUNSTABLE) h->status = code;
  }
  return code;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

bool handle_nonlocal(const pflb_handle* h) { return h->family == 1 || h->family == 2; }

}  // namespace pflb

namespace {

#define CU(h, call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return handle_fail((h), PFLB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

int default_chunk(const pflb_handle* h, int parity, bool tma) {
  const TileShape ts = tile_shape(h->family, h->dim, h->storage);
  const int ta = ts.ta, tb = ts.tb;
  const int NA = h->prm.nx, NB = h->dim == 3 ? h->prm.ny : 1, NC = h->dim == 3 ? h->prm.nz : h->prm.ny;
  const long long tiles = (long long)((NA + ta - 1) / ta) * ((NB + tb - 1) / tb);
  const long long target = 8LL * num_sms();
  long long c = (tiles * NC + target - 1) / target;
  // Longer marches amortise the prologue (two planes of phi) and keep each
  // block's reads on fewer DRAM pages; 128 planes measured best at 512^3
  // (FP32 24.9 vs 24.8 GLUPS at 64, FP16 31.3 vs 30.7), with at least ~8
  // blocks per SM still in the grid.
  if (c < 4) c = 4;
  if (c > 128) c = 128;
  // TMA-staged steps: the even AA step (f read and written at the own cell)
  // runs faster in short marches, 4.66 -> 4.09 ms from 128 to 32 planes at
  // 512^3 (Fakhari2017; Chai2018 5.17 -> 4.57), while the odd step (f from
  // and to the neighbours) runs slower in them (5.40 -> 5.55 ms): 32 planes
  // on even steps, the default on odd ones. Liang2018, which also carries
  // phi*u, gains nothing from short marches (5.34 -> 5.43 ms) and keeps the
  // default.
  // D3Q27 (27 f slots per plane, three blocks per SM): 64 planes measured
  // best on its TMA-staged even steps (5.49 ms against 5.67 at 32 and 5.60
  // at 128).
  const long long cap = h->QF == 27 ? 64 : 32;
  if (tma && parity == 0 && !fam_phiu(h->family) && c > cap) c = cap;
  if (c > NC) c = NC;
  return (int)c;
}

double tau_of(double nu) { return 3.0 * nu + 0.5; }

int validate(const pflb_params* p, char* msg, size_t n) {
  if (p->dim != 2 && p->dim != 3) return snprintf(msg, n, "dim must be 2 or 3"), PFLB_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return snprintf(msg, n, "sizes must be >= 1"), PFLB_EINVAL;
  if (p->dim == 2 && p->nz != 1) return snprintf(msg, n, "nz must be 1 in 2D"), PFLB_EINVAL;
  const long long N = (long long)p->nx * p->ny * p->nz;
  // Population offsets (pop_ix, cells rounded up to blocks of 32) are 32-bit
  // in the kernels.
  const long long qmax = p->dim == 2 ? 9 : 19;
  if (((N + 31) / 32) * 32 * qmax >= (1LL << 32))
    return snprintf(msg, n, "Q * cells must be < 2^32 (%lld cells max)", ((1LL << 32) - 1) / qmax / 32 * 32), PFLB_EINVAL;
  if (p->family < 0 || p->family > 6) return snprintf(msg, n, "unknown family %d", p->family), PFLB_EINVAL;
  if (p->family >= PFLB_CH_BAO2024 && (p->storage != PFLB_FP32 || p->bc_y != 0 || p->lattice_f == 27 ||
                                       p->collision != 0))
    return snprintf(msg, n, "Bao2024 and Liu2023 run on periodic domains with FP32 storage and BGK on D2Q9 / D3Q19"),
           PFLB_EINVAL;
  if (p->storage < 0 || p->storage > 2) return snprintf(msg, n, "unknown storage %d", p->storage), PFLB_EINVAL;
  if (p->bc_y < 0 || p->bc_y > 2) return snprintf(msg, n, "bc_y must be 0, 1 or 2"), PFLB_EINVAL;
  if (p->bc_y != 0 && p->dim != 2) return snprintf(msg, n, "walls are supported in 2D only"), PFLB_EINVAL;
  // Mirrored ghost planes reach 2 cells beyond a wall (Cahn-Hilliard halo).
  if (p->bc_y != 0 && p->ny < 4) return snprintf(msg, n, "walls need ny >= 4"), PFLB_EINVAL;
  if (p->visc_interp < 0 || p->visc_interp > 3) return snprintf(msg, n, "unknown visc_interp"), PFLB_EINVAL;
  if (p->obs_capacity < 1) return snprintf(msg, n, "obs_capacity must be >= 1"), PFLB_EINVAL;
  if (!(p->phi_H != p->phi_L)) return snprintf(msg, n, "phi_H must differ from phi_L"), PFLB_EINVAL;
  if (!(p->W > 0.0)) return snprintf(msg, n, "W must be > 0"), PFLB_EINVAL;
  if (!(p->sigma >= 0.0)) return snprintf(msg, n, "sigma must be >= 0"), PFLB_EINVAL;
  if (!(p->rho_H > 0.0 && p->rho_L > 0.0)) return snprintf(msg, n, "densities must be > 0"), PFLB_EINVAL;
  if (!(tau_of(p->nu_H) > 0.5 && tau_of(p->nu_L) > 0.5))
    return snprintf(msg, n, "tau = 3 nu + 1/2 must exceed 1/2 in both phases"), PFLB_EINVAL;
  const double eta = (p->family == 3 || p->family == 5) ? p->eta_ch : 1.0;
  if (!(eta > 0.0)) return snprintf(msg, n, "eta must be > 0"), PFLB_EINVAL;
  if (!(3.0 * p->M / eta + 0.5 > 0.5)) return snprintf(msg, n, "tau_phi must exceed 1/2 (M > 0)"), PFLB_EINVAL;
  if (!(p->lundgren_A < 2.0)) return snprintf(msg, n, "lundgren_A must be < 2"), PFLB_EINVAL;
  const int lf = p->lattice_f;
  if (p->dim == 2 ? !(lf == 0 || lf == 9) : !(lf == 0 || lf == 19 || lf == 27))
    return snprintf(msg, n, "lattice_f must be 9 in 2D and 19 or 27 in 3D (0: default)"), PFLB_EINVAL;
  if (p->collision != 0 && p->collision != 1) return snprintf(msg, n, "collision must be 0 (BGK) or 1 (MRT)"), PFLB_EINVAL;
  if (p->collision == 1) {
    if (lf != 27) return snprintf(msg, n, "the MRT collision is defined on D3Q27 (lattice_f = 27)"), PFLB_EINVAL;
    if (!(p->mrt_s_bulk > 0.0 && p->mrt_s_bulk < 2.0 && p->mrt_s_ho > 0.0 && p->mrt_s_ho < 2.0))
      return snprintf(msg, n, "MRT rates must lie in (0, 2)"), PFLB_EINVAL;
  }
  return PFLB_OK;
}

// Derived constants (Sec. II A, II B), computed in double, used in FP32.
DevParams derive(const pflb_params* p) {
  DevParams d;
  memset(&d, 0, sizeof(d));
  d.nx = p->nx;
  d.ny = p->ny;
  d.nz = p->nz;
  d.dim = p->dim;
  d.family = p->family;
  d.walls = p->bc_y != 0;
  d.moving = p->bc_y == 2;
  d.visc_interp = p->visc_interp;
  d.freeze = p->freeze_phi != 0;
  const double dphi = p->phi_H - p->phi_L;
  const double beta = 12.0 * p->sigma / (p->W * std::pow(std::fabs(dphi), 4));   // Eq. (coefficient1)
  const double kappa = 3.0 * p->sigma * p->W / (2.0 * dphi * dphi);              // Eq. (coefficients)
  d.phiH = (float)p->phi_H;
  d.phiL = (float)p->phi_L;
  d.phi0 = (float)(0.5 * (p->phi_H + p->phi_L));
  d.inv_dphi = (float)(1.0 / dphi);
  d.rhoL = (float)p->rho_L;
  d.drho_dphi = (float)((p->rho_H - p->rho_L) / dphi);
  d.nuH = (float)p->nu_H;
  d.nuL = (float)p->nu_L;
  d.muH = (float)(p->rho_H * p->nu_H);
  d.muL = (float)(p->rho_L * p->nu_L);
  d.beta4 = (float)(4.0 * beta);
  d.kappa = (float)kappa;
  d.four_beta_over_kappa = (float)(kappa > 0 ? 4.0 * beta / kappa : 32.0 / (p->W * p->W * dphi * dphi));
  d.counter_k = (float)(4.0 / (p->W * std::fabs(dphi)));  // sqrt(2 beta / kappa)
  d.M = (float)p->M;
  const double eta = (p->family == 3 || p->family == 5) ? p->eta_ch : 1.0;
  const double tau_phi = 3.0 * p->M / eta + 0.5;                                   // Eq. (fakhari_tau_model)
  d.inv_tau_phi = (float)(1.0 / tau_phi);
  d.src_w_phi = (float)(1.0 - 0.5 / tau_phi);
  d.lambda = (float)p->lambda_hybrid;
  d.eta = (float)eta;
  for (int k = 0; k < 3; ++k) {
    d.grav[k] = (float)p->gravity[k];
    d.fdens[k] = (float)p->force_density[k];
  }
  d.lundA = (float)p->lundgren_A;
  d.wall_u[0] = (float)p->wall_u[0];
  d.wall_u[1] = (float)p->wall_u[1];
  d.eps2 = (float)(p->grad_eps * p->grad_eps);
  d.gref = (float)(0.5 * (p->phi_H + p->phi_L));
  d.lat = (p->dim == 3 && p->lattice_f == 27) ? 1 : 0;
  d.mrt = p->collision == 1 ? 1 : 0;
  d.mrt_sb = (float)p->mrt_s_bulk;
  d.mrt_sh = (float)p->mrt_s_ho;
  // Bao2024 (Reading R21): theta of Eq. (quasi_incomp_system), constant tau.
  const double r = p->rho_H / p->rho_L;
  d.theta = (float)((r - 1.0) / (p->phi_H - p->phi_L * r));
  d.lks_itau = (float)(1.0 / (3.0 * (p->nu_H > p->nu_L ? p->nu_H : p->nu_L) + 0.5));
  d.W_xi = (float)p->W;
  return d;
}

void step_launch(int fam, int dim, int storage, const StepArgs& a, cudaStream_t s) {
  switch (fam) {
    case 0: step_fakhari(dim, storage, a, s); break;
    case 1: step_chai(dim, storage, a, s); break;
    case 2: step_hu(dim, storage, a, s); break;
    case 3: step_liang2014(dim, storage, a, s); break;
    case 4: step_liang2018(dim, storage, a, s); break;
    case 5: step_bao2024(dim, storage, a, s); break;
    default: step_liu2023(dim, storage, a, s); break;
  }
}

void init_launch(int fam, int dim, int storage, const InitArgs& a, cudaStream_t s) {
  switch (fam) {
    case 0: init_fakhari(dim, storage, a, s); break;
    case 1: init_chai(dim, storage, a, s); break;
    case 2: init_hu(dim, storage, a, s); break;
    case 3: init_liang2014(dim, storage, a, s); break;
    case 4: init_liang2018(dim, storage, a, s); break;
    case 5: init_bao2024(dim, storage, a, s); break;
    default: init_liu2023(dim, storage, a, s); break;
  }
}

int ensure_scratch(pflb_handle* h) {
  if (h->scratch) return PFLB_OK;
  const long long n = h->N * (h->dim + 2);
  CU(h, cudaMalloc(&h->scratch, (size_t)n * sizeof(float)));
  return PFLB_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

void pflb::obs_to_host(const DevObs& d, long long step, pflb_obs* o) {
  o->step = step;
  o->sum_phi = d.sum_phi;
  o->vol_smooth = d.vol_smooth;
  o->vol_count = (int64_t)d.vol_count;
  o->ke = d.ke;
  o->phi_max = key_float(d.phi_max_key);
  o->phi_min = key_float(d.phi_min_key);
  for (int k = 0; k < 3; ++k) o->centroid[k] = d.vol_smooth != 0.0 ? d.cen[k] / d.vol_smooth : 0.0;
  o->status = (d.status & kStatusTimeout) ? PFLB_ETIMEOUT : (d.status ? PFLB_EUNSTABLE : PFLB_OK);
  o->pad = 0;
}

StepArgs pflb::handle_step_args(const pflb_handle* h) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.p = h->dp;
  a.g_src = h->g[h->cur];
  a.g_dst = h->g[1 - h->cur];
  a.f = h->f;
  a.phiu = h->phiu;
  a.work = h->work;
  a.parity = (int)(h->step & 1);
  a.N = h->N;
  a.tma = handle_tma_step(h, a.parity) ? h->tma[h->cur] : nullptr;
  a.chunk = h->chunk > 0 ? h->chunk : default_chunk(h, a.parity, a.tma != nullptr);
  a.seed = (unsigned)h->step;
  a.test_wait_polls = h->test_wait_polls;
  return a;
}

namespace {

// A read-only pass over the current state: fields to device buffers and the
// observables into the extra ring slot.
int macro_pass(pflb_handle* h, float* phi, float* u, float* p) {
  DevObs* slot = h->obs + h->obs_cap;
  // Sums start at zero, the max key below every key, the min key above.
  static DevObs init = [] {
    DevObs o;
    memset(&o, 0, sizeof(o));
    o.phi_min_key = 0xffffffffu;
    return o;
  }();
  CU(h, cudaMemcpyAsync(slot, &init, sizeof(DevObs), cudaMemcpyHostToDevice, h->stream));
  StepArgs a = handle_step_args(h);
  a.obs_slot = slot;
  a.obs_zero = nullptr;
  a.macro = 1;
  a.out_phi = phi;
  a.out_u = u;
  a.out_p = p;
  if (handle_nonlocal(h)) {
    double* acc = h->gamma_acc + 4;
    CU(h, cudaMemsetAsync(acc, 0, 2 * sizeof(double), h->stream));
    GammaArgs ga;
    ga.p = h->dp;
    ga.g_src = h->g[h->cur];
    ga.acc = acc;
    ga.zero = nullptr;
    ga.N = h->N;
    gamma_sums(h->dim, h->storage, ga, h->stream);
    a.gamma_acc = acc;
  }
  if (h->family == PFLB_HAC_LIU2023) a.gamma_acc = h->gamma_acc + 4;
  step_launch(h->family, h->dim, h->storage, a, h->stream);
  CU(h, cudaGetLastError());
  return PFLB_OK;
}


}  // namespace

int pflb::handle_canon(pflb_handle* h, float* state_dev, int to_canon) {
  CanonArgs a;
  a.p = h->dp;
  a.g = h->g[h->cur];
  a.f = h->f;
  a.phiu = h->phiu;
  a.state = state_dev;
  a.parity = (int)(h->step & 1);
  a.to_canon = to_canon;
  a.ch = h->family == 3 || h->family == 5;   // Cahn-Hilliard: the D3Q7 rest population is stored
  a.N = h->N;
  canon_copy(h->dim, h->storage, a, h->stream);
  CU(h, cudaGetLastError());
  return PFLB_OK;
}

extern "C" {

int pflb_create(const pflb_params* params, void* cuda_stream, pflb_handle** out) {
  if (!params || !out) return PFLB_EINVAL;
  *out = nullptr;
  pflb_handle* h = new (std::nothrow) pflb_handle();
  if (!h) return PFLB_ENOMEM;
  int rc = validate(params, h->err, sizeof(h->err));
  if (rc != PFLB_OK) {
    // Hand back the handle so the caller can read the message, then destroy it.
    h->status = rc;
    *out = h;
    return rc;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    h->status = PFLB_ECUDA;
    snprintf(h->err, sizeof(h->err), "no CUDA device");
    *out = h;
    return PFLB_ECUDA;
  }
  h->prm = *params;
  h->dp = derive(params);
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->dim = params->dim;
  h->QG = params->dim == 2 ? 9 : 7;
  h->QF = params->dim == 2 ? 9 : (params->lattice_f == 27 ? 27 : 19);
  h->storage = params->storage;
  h->family = params->family;
  h->N = (long long)params->nx * params->ny * params->nz;
  h->elem = params->storage == 0 ? 4 : 2;
  h->obs_cap = params->obs_capacity < 2 ? 2 : params->obs_capacity;
  *out = h;
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return handle_fail(h, PFLB_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    return PFLB_OK;
  };
  // Populations in blocks of kPopBlock cells (pop_ix), plus 16 bytes of
  // padding: the step kernel fetches 16-bit populations as the aligned
  // 32-bit words that contain them.
  const size_t npad = (size_t)((h->N + kPopBlock - 1) / kPopBlock) * kPopBlock;
  if ((rc = alloc(&h->g[0], (size_t)h->QG * npad * h->elem + 16))) return rc;
  if ((rc = alloc(&h->g[1], (size_t)h->QG * npad * h->elem + 16))) return rc;
  if ((rc = alloc(&h->f, (size_t)h->QF * npad * h->elem + 16))) return rc;
  if (fam_phiu(h->family) && (rc = alloc((void**)&h->phiu, (size_t)h->dim * h->N * sizeof(float)))) return rc;
  if (h->family == PFLB_CH_BAO2024 && (rc = alloc((void**)&h->work, (size_t)(3 + h->dim) * h->N * sizeof(float))))
    return rc;
  if (h->family == PFLB_HAC_LIU2023 && (rc = alloc((void**)&h->work, (size_t)6 * h->N * sizeof(float)))) return rc;
  if ((rc = alloc((void**)&h->obs, (size_t)(h->obs_cap + 1) * sizeof(DevObs)))) return rc;
  if ((rc = alloc((void**)&h->gamma_acc, 6 * sizeof(double)))) return rc;
  handle_build_tma(h);
  return PFLB_OK;
}

int pflb_init(pflb_handle* h, const float* phi0, const float* u0) {
  if (!h || !phi0) return handle_fail(h, PFLB_EINVAL, "null argument");
  if (h->status != PFLB_OK && h->status != PFLB_EUNSTABLE) return h->status;
  int rc = ensure_scratch(h);
  if (rc) return rc;
  const size_t nb = (size_t)h->N * sizeof(float);
  CU(h, cudaMemcpyAsync(h->scratch, phi0, nb, cudaMemcpyDefault, h->stream));
  if (u0) CU(h, cudaMemcpyAsync(h->scratch + h->N, u0, nb * h->dim, cudaMemcpyDefault, h->stream));
  InitArgs a;
  a.p = h->dp;
  a.phi0 = h->scratch;
  a.u0 = u0 ? h->scratch + h->N : nullptr;
  a.g = h->g[0];
  a.f = h->f;
  a.phiu = h->phiu;
  a.N = h->N;
  a.work = h->work;
  init_launch(h->family, h->dim, h->storage, a, h->stream);
  CU(h, cudaGetLastError());
  // Zero every observables slot and the nonlocal accumulators.
  std::vector<DevObs> z(h->obs_cap + 1);
  for (auto& o : z) {
    memset(&o, 0, sizeof(o));
    o.phi_min_key = 0xffffffffu;
  }
  CU(h, cudaMemcpyAsync(h->obs, z.data(), z.size() * sizeof(DevObs), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaMemsetAsync(h->gamma_acc, 0, 6 * sizeof(double), h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  h->cur = 0;
  h->step = 0;
  h->initialized = 1;
  h->status = PFLB_OK;
  h->err[0] = 0;
  return PFLB_OK;
}

int pflb_step(pflb_handle* h, int64_t nsteps) {
  if (!h || nsteps < 0) return handle_fail(h, PFLB_EINVAL, "invalid argument");
  if (h->status != PFLB_OK && h->status != PFLB_EUNSTABLE) return h->status;
  const NvtxRange range("pflb_step");
  for (int64_t i = 0; i < nsteps; ++i) {
    StepArgs a = handle_step_args(h);
    a.obs_slot = h->obs + (h->step % h->obs_cap);
    a.obs_zero = h->obs + ((h->step + 1) % h->obs_cap);
    if (handle_nonlocal(h)) {
      double* acc = h->gamma_acc + 2 * (h->step & 1);
      GammaArgs ga;
      ga.p = h->dp;
      ga.g_src = h->g[h->cur];
      ga.acc = acc;
      ga.zero = h->gamma_acc + 2 * ((h->step + 1) & 1);
      ga.N = h->N;
      gamma_sums(h->dim, h->storage, ga, h->stream);
      a.gamma_acc = acc;
    }
    if (h->family == PFLB_HAC_LIU2023) a.gamma_acc = h->gamma_acc + 2 * (h->step & 1);
    step_launch(h->family, h->dim, h->storage, a, h->stream);
    h->cur ^= 1;
    h->step += 1;
  }
  CU(h, cudaGetLastError());
  return h->status;
}

int pflb_sync(pflb_handle* h) {
  if (!h) return PFLB_EINVAL;
  CU(h, cudaStreamSynchronize(h->stream));
  if (h->step > 0) {
    // Check the per-step status words of the recorded steps.
    const long long n = h->step < h->obs_cap ? h->step : h->obs_cap;
    std::vector<DevObs> o(h->obs_cap);
    CU(h, cudaMemcpy(o.data(), h->obs, h->obs_cap * sizeof(DevObs), cudaMemcpyDeviceToHost));
    for (long long i = 0; i < n; ++i) {
      const long long s = h->step - 1 - i;
      const unsigned st = o[s % h->obs_cap].status;
      if (st & kStatusTimeout)
        return handle_fail(h, PFLB_ETIMEOUT, "step %lld: a staging copy did not complete in time", s);
      if (st) return handle_fail(h, PFLB_EUNSTABLE, "step %lld produced rho <= 0 or non-finite phi/u", s);
    }
  }
  return h->status;
}

int pflb_observables(pflb_handle* h, pflb_obs* out) {
  if (!h || !out) return handle_fail(h, PFLB_EINVAL, "null argument");
  int rc = ensure_scratch(h);
  if (rc) return rc;
  rc = macro_pass(h, h->scratch, h->scratch + h->N, h->scratch + (long long)(h->dim + 1) * h->N);
  if (rc) return rc;
  DevObs d;
  CU(h, cudaMemcpyAsync(&d, h->obs + h->obs_cap, sizeof(DevObs), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  obs_to_host(d, h->step, out);
  if (out->status == PFLB_ETIMEOUT) handle_fail(h, PFLB_ETIMEOUT, "a staging copy did not complete in time");
  else if (out->status != PFLB_OK) handle_fail(h, PFLB_EUNSTABLE, "state has rho <= 0 or non-finite phi/u");
  return h->status;
}

int pflb_obs_history(pflb_handle* h, pflb_obs* out, int32_t n, int32_t* written) {
  if (!h || !out || n < 0) return handle_fail(h, PFLB_EINVAL, "invalid argument");
  long long m = n;
  if (m > h->step) m = h->step;
  if (m > h->obs_cap - 1) m = h->obs_cap - 1;  // the newest slot may be in flight-zeroed
  std::vector<DevObs> o(h->obs_cap);
  CU(h, cudaStreamSynchronize(h->stream));
  CU(h, cudaMemcpy(o.data(), h->obs, h->obs_cap * sizeof(DevObs), cudaMemcpyDeviceToHost));
  for (long long i = 0; i < m; ++i) {
    const long long s = h->step - m + i;
    obs_to_host(o[s % h->obs_cap], s, &out[i]);
  }
  if (written) *written = (int32_t)m;
  return PFLB_OK;
}

int pflb_get_fields(pflb_handle* h, float* phi, float* u, float* p) {
  if (!h) return PFLB_EINVAL;
  int rc = ensure_scratch(h);
  if (rc) return rc;
  const long long N = h->N;
  float* dphi = (phi && is_device_ptr(phi)) ? phi : h->scratch;
  float* du = (u && is_device_ptr(u)) ? u : h->scratch + N;
  float* dp = (p && is_device_ptr(p)) ? p : h->scratch + (long long)(h->dim + 1) * N;
  rc = macro_pass(h, dphi, du, dp);
  if (rc) return rc;
  const size_t nb = (size_t)N * sizeof(float);
  if (phi && dphi != phi) CU(h, cudaMemcpyAsync(phi, dphi, nb, cudaMemcpyDefault, h->stream));
  if (u && du != u) CU(h, cudaMemcpyAsync(u, du, nb * h->dim, cudaMemcpyDefault, h->stream));
  if (p && dp != p) CU(h, cudaMemcpyAsync(p, dp, nb, cudaMemcpyDefault, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return PFLB_OK;
}

int64_t pflb_state_floats(const pflb_handle* h) {
  if (!h) return -1;
  return (int64_t)(h->QG + h->QF + (fam_phiu(h->family) ? h->dim : 0)) * h->N;
}


int pflb_save(pflb_handle* h, float* state) {
  if (!h || !state) return handle_fail(h, PFLB_EINVAL, "null argument");
  const size_t nb = (size_t)pflb_state_floats(h) * sizeof(float);
  if (is_device_ptr(state)) {
    int rc = handle_canon(h, state, 1);
    if (rc) return rc;
  } else {
    float* tmp = nullptr;
    CU(h, cudaMalloc(&tmp, nb));
    int rc = handle_canon(h, tmp, 1);
    if (rc == PFLB_OK) {
      cudaError_t e = cudaMemcpyAsync(state, tmp, nb, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) rc = handle_fail(h, PFLB_ECUDA, "copy of the state failed: %s", cudaGetErrorString(e));
    }
    cudaFree(tmp);
    if (rc) return rc;
  }
  CU(h, cudaStreamSynchronize(h->stream));
  return PFLB_OK;
}

int pflb_load(pflb_handle* h, const float* state) {
  if (!h || !state) return handle_fail(h, PFLB_EINVAL, "null argument");
  const size_t nb = (size_t)pflb_state_floats(h) * sizeof(float);
  float* src = const_cast<float*>(state);
  float* tmp = nullptr;
  if (!is_device_ptr(state)) {
    CU(h, cudaMalloc(&tmp, nb));
    cudaError_t e = cudaMemcpyAsync(tmp, state, nb, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return handle_fail(h, PFLB_ECUDA, "copy of the state failed: %s", cudaGetErrorString(e));
    }
    src = tmp;
  }
  int rc = handle_canon(h, src, 0);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (tmp) cudaFree(tmp);
  if (rc) return rc;
  if (e != cudaSuccess) return handle_fail(h, PFLB_ECUDA, "load failed: %s", cudaGetErrorString(e));
  return PFLB_OK;
}

int64_t pflb_step_count(const pflb_handle* h) { return h ? h->step : -1; }

double pflb_bytes_per_update(const pflb_handle* h) {
  if (!h) return 0.0;
  // Stored populations read once and written once (the D3Q7 rest slot of the
  // Allen-Cahn families is identically zero and never touched).
  const int qg = (h->dim == 3 && h->family != 3 && h->family != 5) ? h->QG - 1 : h->QG;
  double b = 2.0 * (qg + h->QF) * (double)h->elem;
  if (h->family == PFLB_CH_BAO2024) {
    // the passes: g read for phi, phi and mu written and read by the mu,
    // macroscopic and collision passes, f read for u and p, u and p written
    // and read (field words of 4 bytes)
    b += 4.0 * (qg + 1) + 8.0 + 4.0 * h->QF + 8.0 + 4.0 * (h->dim + 1) + 4.0 * (3 + h->dim);
  }
  if (h->family == PFLB_HAC_LIU2023) {
    // the passes: g read for phi*, phi* S(psi0) psi written; per
    // reinitialisation step psi and S(psi0) read and psi written; lambda
    // written, phi* read twice, lambda read twice, phi written and read
    // (field words of 4 bytes)
    const double nit = std::ceil(6.0 * h->prm.W);
    b += 4.0 * qg + 12.0 + 12.0 * nit + 12.0 + 12.0 + 12.0;
  }
  if (fam_phiu(h->family)) b += 2.0 * h->dim * 4.0;  // phi*u read + write
  if (handle_nonlocal(h)) b += (double)qg * h->elem;         // g read by the gamma reduction
  return b;
}

int pflb_set_chunk(pflb_handle* h, int32_t chunk) {
  if (!h || chunk < 0) return handle_fail(h, PFLB_EINVAL, "chunk must be >= 0");
  h->chunk = chunk;
  return PFLB_OK;
}

int pflb_lattice(int32_t dim, int32_t which, int32_t* q, int32_t* e, double* w) {
  if ((dim != 2 && dim != 3) || which < 0 || which > 2 || (which == 2 && dim != 3)) return PFLB_EINVAL;
  auto put = [&](auto L) {
    using Lt = decltype(L);
    if (q) *q = Lt::Q;
    for (int a = 0; a < Lt::Q; ++a) {
      if (e) {
        e[3 * a] = Lt::ex(a);
        e[3 * a + 1] = Lt::ey(a);
        e[3 * a + 2] = Lt::ez(a);
      }
      if (w) w[a] = Lt::wx(a);
    }
  };
  if (dim == 2) put(D2Q9{});
  else if (which == 0) put(D3Q7{});
  else if (which == 1) put(D3Q19{});
  else put(D3Q27{});
  return PFLB_OK;
}

int pflb_destroy(pflb_handle* h) {
  if (!h) return PFLB_OK;
  cudaFree(h->g[0]);
  cudaFree(h->g[1]);
  cudaFree(h->f);
  cudaFree(h->phiu);
  cudaFree(h->work);
  cudaFree(h->obs);
  cudaFree(h->gamma_acc);
  cudaFree(h->scratch);
  delete h->tma[0];
  delete h->tma[1];
  delete h;
  return PFLB_OK;
}

const char* pflb_last_error(const pflb_handle* h) { return h ? h->err : "null handle"; }

}  // extern "C"
