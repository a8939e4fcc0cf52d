// Device-side definitions shared by the PF-LB kernels: lattice tables,
// derived parameters, 16-bit storage codec, observables accumulators.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace pflb {

constexpr int FAM_FAKHARI = 0;
constexpr int FAM_CHAI = 1;
constexpr int FAM_HU = 2;
constexpr int FAM_LIANG = 3;     // Liang2014 (Cahn-Hilliard)
constexpr int FAM_LIANG18 = 4;   // Liang2018 (conservative Allen-Cahn, conservative NS form)
constexpr int FAM_BAO = 5;       // Bao2024 (Cahn-Hilliard, singular mobility, multi-pass step)
constexpr int FAM_LIU = 6;       // Liu2023 (hybrid AC, lambda(x) from a signed distance, multi-pass step)

// Families that keep phi*u of the previous step for d_t(phi u) (Sec. III B)
// and use the pressure-based hydrodynamic equilibrium (Eq. liang2_feq).
__host__ __device__ constexpr bool fam_phiu(int fam) {
  return fam == FAM_LIANG || fam == FAM_LIANG18 || fam == FAM_LIU;
}

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
  __host__ __device__ static constexpr double wx(int a) {
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr float w(int a) { return (float)wx(a); }
  __host__ __device__ static constexpr float wlo(int a) { return (float)(wx(a) - (double)w(a)); }
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
  __host__ __device__ static constexpr double wx(int a) { return a == 0 ? 0.0 : 1.0 / 6.0; }
  __host__ __device__ static constexpr float w(int a) { return (float)wx(a); }
  __host__ __device__ static constexpr float wlo(int a) { return (float)(wx(a) - (double)w(a)); }
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
  __host__ __device__ static constexpr double wx(int a) {
    return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr float w(int a) { return (float)wx(a); }
  __host__ __device__ static constexpr float wlo(int a) { return (float)(wx(a) - (double)w(a)); }
  __host__ __device__ static constexpr int opp(int a) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    return t[a];
  }
};

// D3Q27 (Sec. IV: the paper's 3D hydrodynamic lattice): D3Q19's nineteen,
// then the corners (1,1,1) (-1,-1,-1) (1,1,-1) (-1,-1,1) (1,-1,1) (-1,1,-1)
// (-1,1,1) (1,-1,-1); weights 8/27, 2/27, 1/54, 1/216.
struct D3Q27 {
  static constexpr int Q = 27;
  __host__ __device__ static constexpr int ex(int a) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
    return t[a];
  }
  __host__ __device__ static constexpr int ey(int a) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
    return t[a];
  }
  __host__ __device__ static constexpr int ez(int a) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
    return t[a];
  }
  __host__ __device__ static constexpr double wx(int a) {
    return a == 0 ? 8.0 / 27.0 : (a < 7 ? 2.0 / 27.0 : (a < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
  __host__ __device__ static constexpr float w(int a) { return (float)wx(a); }
  __host__ __device__ static constexpr float wlo(int a) { return (float)(wx(a) - (double)w(a)); }
  __host__ __device__ static constexpr int opp(int a) {
    return a == 0 ? 0 : ((a % 2 == 1) ? a + 1 : a - 1);
  }
};

// w_a * x with the weight carried as hi + lo (w = w_hi + w_lo to ~1e-16):
// the FP32 weights alone have sum_a w_a e_a e_a = (1 + 7.45e-9) I / 3 on D2Q9
// and D3Q19, which biases every equilibrium moment and made the momentum grow
// by ~1e-8 per relaxation.
template <typename L>
__device__ __forceinline__ float wmul(int a, float x) {
  return fmaf(L::w(a), x, L::wlo(a) * x);
}

// Population layout in device memory (AoSoA): the linear cell index is cut
// into blocks of 32 consecutive cells, and each block holds its Q velocity
// planes one after another, so population q of cell i sits at element
// ((i / 32) Q + q) 32 + i % 32. A warp over 32 aligned cells of a row then
// reads or writes one contiguous 32 Q-element span instead of Q scattered
// rows. Arrays hold Q x (N rounded up to 32) elements.
constexpr unsigned kPopBlock = 32u;
template <typename L>
__host__ __device__ __forceinline__ unsigned pop_ix(int q, unsigned cell) {
  return ((cell >> 5) * (unsigned)L::Q + (unsigned)q) * kPopBlock + (cell & (kPopBlock - 1u));
}

// Lattice triple per dimension: phase field g, hydrodynamics f, stencil.
// LAT = 1 selects the D3Q27 hydrodynamic lattice in 3D; the stencils keep
// the D3Q19 weights.
template <int DIM, int LAT = 0> struct Lattices;
template <> struct Lattices<2, 0> { using G = D2Q9; using F = D2Q9; using S = D2Q9; };
template <> struct Lattices<3, 0> { using G = D3Q7; using F = D3Q19; using S = D3Q19; };
template <> struct Lattices<3, 1> { using G = D3Q7; using F = D3Q27; using S = D3Q19; };

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
  float eps2;               // grad_eps^2 (normal regularisation)
  float gref;               // rest-state offset of g in 16-bit storage
  int32_t lat;              // 3D hydrodynamic lattice: 0 D3Q19, 1 D3Q27
  int32_t mrt;              // 1: multiple-relaxation-time collision (D3Q27)
  float mrt_sb, mrt_sh;     // MRT rates: trace of the second moments, orders >= 3
  float theta;              // Bao2024: quasi-incompressible theta (Eq. quasi_incomp_system)
  float lks_itau;           // Bao2024: 1 / tau of the lattice kinetic scheme (constant)
  float W_xi;               // interface thickness xi (Liu2023: d_min = 3 xi, predictor scale)
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
// Storage codec: FP32 pass-through, or a 16-bit deviation from the rest state,
//   stored = (x - w' c) / s,   x = stored * s + w' c,
// with c the rest-state constant (phi_0 for g, 0 for f), w' the weight (1
// where the weight is 0) and s the power of two nearest w' -- a scale that is
// exact in both directions, so encode/decode adds no bias, only the 16-bit
// rounding of the deviation.
// ---------------------------------------------------------------------------
template <typename L>
__host__ __device__ constexpr float wprime(int a) {
  return L::w(a) > 0.0f ? L::w(a) : 1.0f;
}
template <typename L>
__host__ __device__ constexpr float pow2_scale(int a) {
  // nearest power of two to w' in log scale: 2^k with 2^(k-1/2) < w' <= 2^(k+1/2)
  float s = 1.0f;
  const float w = wprime<L>(a);
  while (w < s * 0.70710678f) s *= 0.5f;
  while (w > s * 1.41421356f) s *= 2.0f;
  return s;
}

// Stochastic rounding of the per-step 16-bit stores. Round-to-nearest of a
// value that repeats step after step (quasi-steady regions) repeats its
// error, and the errors add up coherently -- linearly in the step count,
// and in the sum of phi, which the populations carry. Rounding up with
// probability equal to the dropped fraction makes each error zero-mean, so
// they add up as a random walk. The random threshold comes from a
// counter-based integer hash of (cell, step), one per cell and step, shared
// by that cell's stores: every store is still unbiased, and the g that
// meet at a cell after push streaming come from different cells, so their
// thresholds are independent where phi sums them. The result depends only
// on (cell, step), not on the launch shape or the staging.
__device__ __forceinline__ unsigned dither_seed(unsigned cell, unsigned step) {
  unsigned x = (cell ^ (step * 0x85EBCA6Bu)) * 0x9E3779B9u;
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  return x;
}

template <typename T> struct Codec;
template <> struct Codec<float> {
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float ldc(const float* p) { return *p; }
  __device__ __forceinline__ static float dec(float x, float, float) { return x; }
  __device__ __forceinline__ static void st(float* p, float v, float, float) { *p = v; }
  __device__ __forceinline__ static void st_sr(float* p, float v, float, float, unsigned) { *p = v; }
};
template <> struct Codec<__half> {
  __device__ __forceinline__ static __half ld(const __half* p) { return __ldg(p); }
  __device__ __forceinline__ static __half ldc(const __half* p) { return *p; }
  __device__ __forceinline__ static float dec(__half x, float s, float off) { return fmaf(__half2float(x), s, off); }
  __device__ __forceinline__ static __half from_bits(unsigned short b) { return __ushort_as_half(b); }
  __device__ __forceinline__ static void st(__half* p, float v, float inv_s, float off) {
    *p = __float2half_rn((v - off) * inv_s);
  }
  // Stochastic rounding: 13 random bits added below the last FP16 mantissa
  // bit of the FP32 value's magnitude, then truncation toward zero (exact in
  // the FP16 normal range; FP16 subnormals, below 6.1e-5 of the scale, keep
  // a bias toward zero of at most one subnormal step).
  __device__ __forceinline__ static void st_sr(__half* p, float v, float inv_s, float off, unsigned r) {
    const unsigned b = __float_as_uint((v - off) * inv_s) + (r >> 19);
    *p = __float2half_rz(__uint_as_float(b));
  }
};
template <> struct Codec<__nv_bfloat16> {
  __device__ __forceinline__ static __nv_bfloat16 ld(const __nv_bfloat16* p) { return __ldg(p); }
  __device__ __forceinline__ static __nv_bfloat16 ldc(const __nv_bfloat16* p) { return *p; }
  __device__ __forceinline__ static float dec(__nv_bfloat16 x, float s, float off) {
    return fmaf(__bfloat162float(x), s, off);
  }
  __device__ __forceinline__ static __nv_bfloat16 from_bits(unsigned short b) { return __ushort_as_bfloat16(b); }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v, float inv_s, float off) {
    *p = __float2bfloat16_rn((v - off) * inv_s);
  }
  // Stochastic rounding: 16 random bits added to the FP32 value's magnitude,
  // then its upper half kept (BF16 shares the FP32 exponent range).
  __device__ __forceinline__ static void st_sr(__nv_bfloat16* p, float v, float inv_s, float off, unsigned r) {
    const unsigned b = __float_as_uint((v - off) * inv_s) + (r >> 16);
    *p = __ushort_as_bfloat16((unsigned short)(b >> 16));
  }
};

// Population slot q of lattice L at p, rest-state constant c.
// Asynchronous 4-byte global -> shared copies (cp.async, L1-allocating),
// completed per thread by cp.async.wait_group.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// The same copy with both addresses given as a register plus a compile-time
// byte offset ([reg+imm] operands), so a run of copies from one cell's
// populations to one thread's slots needs no address arithmetic per copy.
template <int SOFF, long long GOFF>
__device__ __forceinline__ void cp_async4_at(unsigned sbase, const void* gbase) {
  asm volatile("cp.async.ca.shared.global [%0+%2], [%1+%3], 4;\n" ::"r"(sbase), "l"(gbase), "n"(SOFF), "n"(GOFF)
               : "memory");
}
// 16-byte global -> shared copy cached in L2 only (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(unsigned saddr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Compile-time loop: fn(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, typename Fn>
__device__ __forceinline__ void static_for(Fn&& fn) {
  if constexpr (B < E) {
    fn(std::integral_constant<int, B>{});
    static_for<B + 1, E>(fn);
  }
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

template <typename T, typename L>
__device__ __forceinline__ float pop_load(const T* p, int q, float c) {  // read-only data
  return Codec<T>::dec(Codec<T>::ld(p), pow2_scale<L>(q), wprime<L>(q) * c);
}
template <typename T, typename L>
__device__ __forceinline__ float pop_loadc(const T* p, int q, float c) { // data written in this kernel
  return Codec<T>::dec(Codec<T>::ldc(p), pow2_scale<L>(q), wprime<L>(q) * c);
}
// A 16-bit population staged as the aligned 32-bit word that holds it:
// hi selects the upper half.
template <typename T, typename L>
__device__ __forceinline__ float pop_from_word(float word, unsigned hi, int q, float c) {
  const unsigned w = __float_as_uint(word);
  const unsigned short b = (unsigned short)(hi ? (w >> 16) : (w & 0xffffu));
  return Codec<T>::dec(Codec<T>::from_bits(b), pow2_scale<L>(q), wprime<L>(q) * c);
}
template <typename T, typename L>
__device__ __forceinline__ void pop_store(T* p, int q, float v, float c) {
  Codec<T>::st(p, v, 1.0f / pow2_scale<L>(q), wprime<L>(q) * c);
}
// The per-step store: stochastically rounded in 16-bit storage with the
// cell's threshold r (dither_seed), exact in FP32.
template <typename T, typename L>
__device__ __forceinline__ void pop_store_sr(T* p, int q, float v, float c, unsigned r) {
  if constexpr (std::is_same<T, float>::value) {
    *p = v;
  } else {
    Codec<T>::st_sr(p, v, 1.0f / pow2_scale<L>(q), wprime<L>(q) * c, r);
  }
}

// ---------------------------------------------------------------------------
// Block-level reduction of the observables into one ring slot.
// ---------------------------------------------------------------------------
struct ObsPartial {
  float s_hi, s_lo;  // compensated sum of phi
  float vs, ke, cx, cy, cz;
  unsigned int count;
  float mx, mn;
  unsigned int bad;  // status bits: 1 unstable, 2 a bounded wait ran out
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
  // status bits: 1 unstable state, 2 a bounded wait ran out
  unsigned int bad = __reduce_or_sync(0xffffffffu, o.bad);
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
    double c = 0.0, smx = -3.0e38, smn = 3.0e38;
    unsigned int sbad = 0u;
    for (int w = 0; w < nwarps; ++w) {
      const double* s = scratch + w * 10;
      for (int k = 0; k < 6; ++k) acc[k] += s[k];
      c += s[6];
      smx = fmax(smx, s[7]);
      smn = fmin(smn, s[8]);
      sbad |= (unsigned int)s[9];
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
    if (sbad) atomicOr(&slot->status, sbad);
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
