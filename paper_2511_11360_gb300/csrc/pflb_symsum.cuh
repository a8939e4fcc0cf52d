// Mirror-exact velocity sums.
//
// A plain loop over the velocities adds the same terms in a different order
// for a cell and for its mirror image, so FP32 rounding breaks the mirror
// symmetry of the step by an ulp per sum. Where a flow has a neutral mode (a
// droplet's position, the phase of a standing interface wave) or a symmetric
// unstable one, that systematic asymmetry drives it coherently. Here every sum
// over velocities adds opposite pairs first, then adds the pair sums that a
// mirror (x, y or z) exchanges as commutative pairs; reflecting the inputs
// then reflects every result bit for bit (addition is commutative, negation
// exact). Used for the population moments and the Sec. III stencils.
#pragma once

#include "pflb_common.cuh"

namespace pflb {

template <typename L> struct Sym;

// D2Q9: 1 +x, 2 +y, 3 -x, 4 -y, 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
template <> struct Sym<D2Q9> {
  template <typename V>
  __device__ __forceinline__ static float moving(const V& v) {  // sum over q >= 1
    return ((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
  }
  template <typename V>
  __device__ __forceinline__ static float first(const V& v, int k) {  // sum e_k v
    return k == 0 ? (v[1] - v[3]) + ((v[5] - v[7]) + (v[8] - v[6]))
                  : (v[2] - v[4]) + ((v[5] - v[7]) + (v[6] - v[8]));
  }
  template <typename V>
  __device__ __forceinline__ static float second(const V& v, int i, int j) {  // sum e_i e_j v
    const float d = (v[5] + v[7]) + (v[6] + v[8]);
    if (i != j) return (v[5] + v[7]) - (v[6] + v[8]);
    return (i == 0 ? (v[1] + v[3]) : (v[2] + v[4])) + d;
  }
  // Sec. III stencils from neighbour values n[q] = phi(x + e_q) and centre c.
  template <typename V>
  __device__ __forceinline__ static float grad(const V& n, int k) {  // sum w e_k n / c_s^2
    return k == 0 ? 3.0f * ((1.0f / 9.0f) * (n[1] - n[3]) + (1.0f / 36.0f) * ((n[5] - n[7]) + (n[8] - n[6])))
                  : 3.0f * ((1.0f / 9.0f) * (n[2] - n[4]) + (1.0f / 36.0f) * ((n[5] - n[7]) + (n[6] - n[8])));
  }
  template <typename V>
  __device__ __forceinline__ static float lap(const V& n, float c) {  // 2 sum w (n - c) / c_s^2
    const float ax = ((n[1] - c) + (n[3] - c)) + ((n[2] - c) + (n[4] - c));
    const float dg = ((n[5] - c) + (n[7] - c)) + ((n[6] - c) + (n[8] - c));
    return 6.0f * ((1.0f / 9.0f) * ax + (1.0f / 36.0f) * dg);
  }
};

// D3Q7: 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z.
template <> struct Sym<D3Q7> {
  template <typename V>
  __device__ __forceinline__ static float moving(const V& v) {
    return ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
  }
  template <typename V>
  __device__ __forceinline__ static float first(const V& v, int k) {
    return k == 0 ? v[1] - v[2] : (k == 1 ? v[3] - v[4] : v[5] - v[6]);
  }
};

// D3Q19: faces 1..6 as D3Q7; edges 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0)
// 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1)
// 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1).
template <> struct Sym<D3Q19> {
  template <typename V>
  __device__ __forceinline__ static float edges_xy(const V& v) { return (v[7] + v[8]) + (v[9] + v[10]); }
  template <typename V>
  __device__ __forceinline__ static float edges_xz(const V& v) { return (v[11] + v[12]) + (v[13] + v[14]); }
  template <typename V>
  __device__ __forceinline__ static float edges_yz(const V& v) { return (v[15] + v[16]) + (v[17] + v[18]); }
  template <typename V>
  __device__ __forceinline__ static float moving(const V& v) {
    const float faces = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
    return faces + ((edges_xy(v) + edges_xz(v)) + edges_yz(v));
  }
  template <typename V>
  __device__ __forceinline__ static float first(const V& v, int k) {
    if (k == 0) return (v[1] - v[2]) + (((v[7] - v[8]) + (v[9] - v[10])) + ((v[11] - v[12]) + (v[13] - v[14])));
    if (k == 1) return (v[3] - v[4]) + (((v[7] - v[8]) + (v[10] - v[9])) + ((v[15] - v[16]) + (v[17] - v[18])));
    return (v[5] - v[6]) + (((v[11] - v[12]) + (v[14] - v[13])) + ((v[15] - v[16]) + (v[18] - v[17])));
  }
  template <typename V>
  __device__ __forceinline__ static float second(const V& v, int i, int j) {
    if (i == j) {
      if (i == 0) return (v[1] + v[2]) + (edges_xy(v) + edges_xz(v));
      if (i == 1) return (v[3] + v[4]) + (edges_xy(v) + edges_yz(v));
      return (v[5] + v[6]) + (edges_xz(v) + edges_yz(v));
    }
    const int a = i < j ? i : j, b = i < j ? j : i;
    if (a == 0 && b == 1) return (v[7] + v[8]) - (v[9] + v[10]);
    if (a == 0 && b == 2) return (v[11] + v[12]) - (v[13] + v[14]);
    return (v[15] + v[16]) - (v[17] + v[18]);
  }
  template <typename V>
  __device__ __forceinline__ static float grad(const V& n, int k) {
    float face, e1, e2;
    if (k == 0) { face = n[1] - n[2]; e1 = (n[7] - n[8]) + (n[9] - n[10]); e2 = (n[11] - n[12]) + (n[13] - n[14]); }
    else if (k == 1) { face = n[3] - n[4]; e1 = (n[7] - n[8]) + (n[10] - n[9]); e2 = (n[15] - n[16]) + (n[17] - n[18]); }
    else { face = n[5] - n[6]; e1 = (n[11] - n[12]) + (n[14] - n[13]); e2 = (n[15] - n[16]) + (n[18] - n[17]); }
    return 3.0f * ((1.0f / 18.0f) * face + (1.0f / 36.0f) * (e1 + e2));
  }
  template <typename V>
  __device__ __forceinline__ static float lap(const V& n, float c) {
    auto d = [&](int q) { return n[q] - c; };
    const float faces = ((d(1) + d(2)) + (d(3) + d(4))) + (d(5) + d(6));
    const float exy = (d(7) + d(8)) + (d(9) + d(10));
    const float exz = (d(11) + d(12)) + (d(13) + d(14));
    const float eyz = (d(15) + d(16)) + (d(17) + d(18));
    return 6.0f * ((1.0f / 18.0f) * faces + (1.0f / 36.0f) * ((exy + exz) + eyz));
  }
};

// D3Q27: D3Q19's nineteen, then corners 19 (1,1,1) 20 (-1,-1,-1) 21 (1,1,-1)
// 22 (-1,-1,1) 23 (1,-1,1) 24 (-1,1,-1) 25 (-1,1,1) 26 (1,-1,-1). With the
// opposite-pair sums P1..P4 (19+20, 21+22, 23+24, 25+26), each mirror swaps
// them in pairs (x: P1<->P4, P2<->P3; y: P1<->P3, P2<->P4; z: P1<->P2,
// P3<->P4), all of which leave ((P1 + P2) + (P3 + P4)) bit for bit intact;
// the first and mixed second moments use the matching pairings.
template <> struct Sym<D3Q27> {
  using B = Sym<D3Q19>;
  template <typename V>
  __device__ __forceinline__ static float corners(const V& v) {
    return ((v[19] + v[20]) + (v[21] + v[22])) + ((v[23] + v[24]) + (v[25] + v[26]));
  }
  template <typename V>
  __device__ __forceinline__ static float moving(const V& v) {
    return B::moving(v) + corners(v);
  }
  template <typename V>
  __device__ __forceinline__ static float first(const V& v, int k) {
    float c;
    if (k == 0) c = ((v[19] - v[20]) + (v[21] - v[22])) + ((v[23] - v[24]) + (v[26] - v[25]));
    else if (k == 1) c = ((v[19] - v[20]) + (v[21] - v[22])) + ((v[24] - v[23]) + (v[25] - v[26]));
    else c = ((v[19] - v[20]) + (v[22] - v[21])) + ((v[23] - v[24]) + (v[25] - v[26]));
    return B::first(v, k) + c;
  }
  template <typename V>
  __device__ __forceinline__ static float second(const V& v, int i, int j) {
    if (i == j) return B::second(v, i, j) + corners(v);
    const int a = i < j ? i : j, b = i < j ? j : i;
    const float P1 = v[19] + v[20], P2 = v[21] + v[22], P3 = v[23] + v[24], P4 = v[25] + v[26];
    float c;
    if (a == 0 && b == 1) c = (P1 + P2) - (P3 + P4);
    else if (a == 0 && b == 2) c = (P1 + P3) - (P2 + P4);
    else c = (P1 + P4) - (P2 + P3);
    return B::second(v, i, j) + c;
  }
};

}  // namespace pflb
