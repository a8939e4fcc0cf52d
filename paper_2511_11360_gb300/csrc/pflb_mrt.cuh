// Multiple-relaxation-time collision on D3Q27 (Sec. IV: the paper's 3D
// hydrodynamics), as a correction of the BGK update.
//
// Moments are the raw ones, m_ijk = sum_a e_ax^i e_ay^j e_az^k f_a with
// i, j, k in {0, 1, 2}. The relaxation matrix S relaxes the conserved and
// first-order moments and the traceless part of the second-order moments at
// w = 1/tau (so the shear viscosity is the BGK one), the trace
// m_200 + m_020 + m_002 at s_b and every moment of order >= 3 at s_h. With the
// forcing in moment space, f* = f - M^-1 S M (f - f_eq) + M^-1 (I - S/2) M F_b.
// Writing f_bgk for the BGK update (all rates w) and n = f - f_eq + F_b/2,
//   f* = f_bgk + M^-1 D M n,
// where D is nonzero only on the trace ((w - s_b)/3 on each diagonal second
// moment, applied to the trace of M n) and on the orders >= 3 (w - s_h). M
// factorises over the axes (D3Q27 is the cube of D1Q3): along one axis a
// triple (f_-, f_0, f_+) has moments (f_- + f_+ + f_0, f_+ - f_-, f_+ + f_-),
// and back f_0 = k_0 - k_2, f_+- = (k_2 +- k_1)/2. Both passes are
// sign-symmetric, so the mirror image of a cell gets the mirror image of the
// correction.
#pragma once

#include "pflb_common.cuh"

namespace pflb {

// Velocity slot of D3Q27 for e = (a, b, c), each in {-1, 0, 1}.
__host__ __device__ constexpr int q27_of(int a, int b, int c) {
  int q = 0;
  for (int k = 0; k < 27; ++k)
    if (D3Q27::ex(k) == a && D3Q27::ey(k) == b && D3Q27::ez(k) == c) q = k;
  return q;
}

// One axis pass of the forward transform on the 3 x 3 x 3 array t[a][b][c]
// (index 0, 1, 2 for e = -1, 0, +1; after the pass, index = moment order).
template <int AXIS>
__device__ __forceinline__ void m_pass(float (&t)[27]) {
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const int i0 = AXIS == 0 ? 0 * 9 + u * 3 + v : (AXIS == 1 ? u * 9 + 0 * 3 + v : u * 9 + v * 3 + 0);
      const int st = AXIS == 0 ? 9 : (AXIS == 1 ? 3 : 1);
      const float fm = t[i0], f0 = t[i0 + st], fp = t[i0 + 2 * st];
      t[i0] = (fm + fp) + f0;
      t[i0 + st] = fp - fm;
      t[i0 + 2 * st] = fp + fm;
    }
}
template <int AXIS>
__device__ __forceinline__ void m_pass_inv(float (&t)[27]) {
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const int i0 = AXIS == 0 ? 0 * 9 + u * 3 + v : (AXIS == 1 ? u * 9 + 0 * 3 + v : u * 9 + v * 3 + 0);
      const int st = AXIS == 0 ? 9 : (AXIS == 1 ? 3 : 1);
      const float k0 = t[i0], k1 = t[i0 + st], k2 = t[i0 + 2 * st];
      t[i0] = 0.5f * (k2 - k1);
      t[i0 + st] = k0 - k2;
      t[i0 + 2 * st] = 0.5f * (k2 + k1);
    }
}

// f += M^-1 D M n for the rates (w, s_b, s_h) above; n is consumed.
__device__ __forceinline__ void mrt_correct(float (&f)[27], const float (&n)[27], float w, float sb, float sh) {
  float t[27];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) t[a * 9 + b * 3 + c] = n[q27_of(a - 1, b - 1, c - 1)];
  m_pass<0>(t);
  m_pass<1>(t);
  m_pass<2>(t);
  // t[i*9 + j*3 + k] = m_ijk. Keep only the relaxed-differently parts.
  const float trc = (w - sb) * (1.0f / 3.0f) * ((t[18] + t[6]) + t[2]);   // m_200, m_020, m_002
  const float dh = w - sh;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int o = i + j + k, idx = i * 9 + j * 3 + k;
        if (o >= 3) t[idx] *= dh;
        else if (o == 2 && (i == 2 || j == 2 || k == 2)) t[idx] = trc;
        else t[idx] = 0.0f;
      }
  m_pass_inv<2>(t);
  m_pass_inv<1>(t);
  m_pass_inv<0>(t);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) f[q27_of(a - 1, b - 1, c - 1)] += t[a * 9 + b * 3 + c];
}

}  // namespace pflb
