// Device-side definitions shared by the PF-LB kernels: lattice tables,
// derived parameters, 16-bit storage codec, observables accumulators.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace pflb {

constexpr int FAM_FAKHARI = 0;
constexpr int FAM_CHAI = 1;
constexpr int FAM_HU = 2;
constexpr int FAM_LIANG = 3;

// ---------------------------------------------------------------------------
// Lattices (c_s^2 = 1/3 for all three, Sec. III and Sec. IV), in the
// canonical velocity order documented by pflb_lattice().
//   D2Q9 : rest, +x, +y, -x, -y, (1,1), (-1,1), (-1,-1), (1,-1)
//   D3Q7 : rest, +x, -x, +y, -y, +z, -z          (w_0 = 0: Sec. IV c_s^2 = 1/3)
//   D3Q19: D3Q7's seven, then (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1)
//          (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
// ---------------------------------------------------------------------------
struct D2Q9 {
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int ex(int a) {
    constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return t[a];
  }
  __host__ __device__ static constexpr int ey(int a) {
    constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return t[a];
  }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr float w(int a) {
    return a == 0 ? 4.0f / 9.0f : (a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr int opp(int a) {
    constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return t[a];
  }
};

struct D3Q7 {
  static constexpr int Q = 7;
  __host__ __device__ static constexpr int ex(int a) {
    constexpr int t[7] = {0, 1, -1, 0, 0, 0, 0};
    return t[a];
  }
  __host__ __device__ static constexpr int ey(int a) {
    constexpr int t[7] = {0, 0, 0, 1, -1, 0, 0};
    return t[a];
  }
  __host__ __device__ static constexpr int ez(int a) {
    constexpr int t[7] = {0, 0, 0, 0, 0, 1, -1};
    return t[a];
  }
  __host__ __device__ static constexpr float w(int a) { return a == 0 ? 0.0f : 1.0f / 6.0f; }
  __host__ __device__ static constexpr int opp(int a) {
    constexpr int t[7] = {0, 2, 1, 4, 3, 6, 5};
    return t[a];
  }
};

struct D3Q19 {
  static constexpr int Q = 19;
  __host__ __device__ static constexpr int ex(int a) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[a];
  }
  __host__ __device__ static constexpr int ey(int a) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[a];
  }
  __host__ __device__ static constexpr int ez(int a) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[a];
  }
  __host__ __device__ static constexpr float w(int a) {
    return a == 0 ? 1.0f / 3.0f : (a < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr int opp(int a) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    return t[a];
  }
};

// Lattice triple per dimension: phase field g, hydrodynamics f, stencil.
template <int DIM> struct Lattices;
template <> struct Lattices<2> { using G = D2Q9; using F = D2Q9; using S = D2Q9; };
template <> struct Lattices<3> { using G = D3Q7; using F = D3Q19; using S = D3Q19; };

// ---------------------------------------------------------------------------
// Parameters in the form the kernels use (host-derived, FP32).
// ---------------------------------------------------------------------------
struct DevParams {
  int32_t nx, ny, nz;       // physical sizes
  int32_t dim, family;
  int32_t walls, moving;    // bounce-back walls at the y ends (2D)
  int32_t visc_interp, freeze;
  float phiH, phiL, phi0, inv_dphi;
  float rhoL, drho_dphi;    // rho = rhoL + drho_dphi (phi - phiL)
  float nuH, nuL, muH, muL; // bulk kinematic / dynamic viscosities
  float beta4;              // 4 beta
  float kappa;
  float four_beta_over_kappa;
  float counter_k;          // sqrt(2 beta / kappa)
  float M;
  float inv_tau_phi;        // 1 / tau_phi
  float src_w_phi;          // 1 - 1/(2 tau_phi)
  float lambda, eta;
  float grav[3], fdens[3];
  float lundA;
  float wall_u[2];          // bottom, top
  float eps2;               // grad_eps^2
  float gref;               // rest-state offset of g in 16-bit storage
};

// Observables accumulated by one pass (one slot of the per-step ring).
struct DevObs {
  double sum_phi, vol_smooth, ke, cen[3];
  unsigned long long vol_count;
  unsigned int phi_max_key, phi_min_key;
  unsigned int status;
  unsigned int pad;
};

// Order-preserving map float -> uint32 for atomicMax / atomicMin.
__device__ __forceinline__ unsigned int float_key(float v) {
  unsigned int u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_float(unsigned int k) {
  unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

// ---------------------------------------------------------------------------
// Storage codec: FP32 pass-through, or 16-bit deviation from the rest state
// scaled by the weight: stored = (x - w c) / w (w = 1 where the weight is 0).
// ---------------------------------------------------------------------------
template <typename T> struct Codec;
template <> struct Codec<float> {
  __device__ __forceinline__ static float load(const float* p, float, float) { return __ldg(p); }
  __device__ __forceinline__ static float loadc(const float* p, float, float) { return *p; }
  __device__ __forceinline__ static void store(float* p, float v, float, float) { *p = v; }
};
template <> struct Codec<__half> {
  __device__ __forceinline__ static float load(const __half* p, float w, float c) {
    return fmaf(__half2float(__ldg(p)), w, w * c);
  }
  __device__ __forceinline__ static float loadc(const __half* p, float w, float c) {
    return fmaf(__half2float(*p), w, w * c);
  }
  __device__ __forceinline__ static void store(__half* p, float v, float w, float c) {
    *p = __float2half_rn((v - w * c) / w);
  }
};
template <> struct Codec<__nv_bfloat16> {
  __device__ __forceinline__ static float load(const __nv_bfloat16* p, float w, float c) {
    return fmaf(__bfloat162float(__ldg(p)), w, w * c);
  }
  __device__ __forceinline__ static float loadc(const __nv_bfloat16* p, float w, float c) {
    return fmaf(__bfloat162float(*p), w, w * c);
  }
  __device__ __forceinline__ static void store(__nv_bfloat16* p, float v, float w, float c) {
    *p = __float2bfloat16_rn((v - w * c) / w);
  }
};

// Normaliser of slot a for the 16-bit codec (the weight, or 1 where it is 0).
template <typename L>
__host__ __device__ constexpr float norm_w(int a) {
  return L::w(a) > 0.0f ? L::w(a) : 1.0f;
}

// ---------------------------------------------------------------------------
// Block-level reduction of the observables into one ring slot.
// ---------------------------------------------------------------------------
struct ObsPartial {
  float s_hi, s_lo;  // compensated sum of phi
  float vs, ke, cx, cy, cz;
  unsigned int count;
  float mx, mn;
  unsigned int bad;
};

__device__ __forceinline__ void obs_init(ObsPartial& o) {
  o.s_hi = o.s_lo = o.vs = o.ke = o.cx = o.cy = o.cz = 0.0f;
  o.count = 0u;
  o.mx = -3.0e38f;
  o.mn = 3.0e38f;
  o.bad = 0u;
}

// Neumaier-compensated FP32 accumulation of phi.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float v) {
  float t = hi + v;
  if (fabsf(hi) >= fabsf(v)) lo += (hi - t) + v;
  else lo += (v - t) + hi;
  hi = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned int warp_usum(unsigned int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// All threads of the block call this; `scratch` holds >= 8 doubles per warp.
__device__ inline void obs_block_commit(const ObsPartial& o, DevObs* slot, double* scratch) {
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
  double v[6] = {(double)o.s_hi + (double)o.s_lo, (double)o.vs, (double)o.ke,
                 (double)o.cx, (double)o.cy, (double)o.cz};
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = warp_sum(v[k]);
  unsigned int cnt = warp_usum(o.count);
  float mx = warp_max(o.mx), mn = warp_min(o.mn);
  unsigned int bad = __any_sync(0xffffffffu, o.bad != 0u) ? 1u : 0u;
  if (lane == 0) {
    double* s = scratch + warp * 10;
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = v[k];
    s[6] = (double)cnt;
    s[7] = (double)mx;
    s[8] = (double)mn;
    s[9] = (double)bad;
  }
  __syncthreads();
  if (tid == 0) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double c = 0.0, smx = -3.0e38, smn = 3.0e38, sbad = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      const double* s = scratch + w * 10;
      for (int k = 0; k < 6; ++k) acc[k] += s[k];
      c += s[6];
      smx = fmax(smx, s[7]);
      smn = fmin(smn, s[8]);
      sbad += s[9];
    }
    atomicAdd(&slot->sum_phi, acc[0]);
    atomicAdd(&slot->vol_smooth, acc[1]);
    atomicAdd(&slot->ke, acc[2]);
    atomicAdd(&slot->cen[0], acc[3]);
    atomicAdd(&slot->cen[1], acc[4]);
    atomicAdd(&slot->cen[2], acc[5]);
    atomicAdd(&slot->vol_count, (unsigned long long)c);
    atomicMax(&slot->phi_max_key, float_key((float)smx));
    atomicMin(&slot->phi_min_key, float_key((float)smn));
    if (sbad > 0.0) atomicOr(&slot->status, 1u);
  }
}

__device__ __forceinline__ void obs_zero_slot(DevObs* slot) {
  slot->sum_phi = slot->vol_smooth = slot->ke = 0.0;
  slot->cen[0] = slot->cen[1] = slot->cen[2] = 0.0;
  slot->vol_count = 0ull;
  slot->phi_max_key = 0u;            // below every key
  slot->phi_min_key = 0xffffffffu;   // above every key
  slot->status = 0u;
}

}  // namespace pflb
