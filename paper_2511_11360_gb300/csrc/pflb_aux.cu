// Auxiliary kernels: the domain integrals of the nonlocal Lagrange
// multiplier and the copy between storage and the canonical FP32 state.
#include "pflb_pass.cuh"
#include "pflb_step.cuh"

namespace pflb {

// I1 = sum (4 beta/kappa)(phi-phi_H)(phi-phi_L)(phi-phi_0) and
// I2 = sum (phi_H - phi)(phi - phi_L) over all cells with phi = sum g
// (Eq. lagrange_multiplier; Reading R1 takes phi* = sum g). Per-thread
// compensated FP32 sums, FP64 across threads and blocks.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) gamma_kernel(const GammaArgs a) {
  using LG = typename Lattices<DIM>::G;
  constexpr int QG = LG::Q;
  const DevParams& P = a.p;
  const T* g = static_cast<const T*>(a.g_src);
  if (a.zero != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    a.zero[0] = 0.0;
    a.zero[1] = 0.0;
  }
  float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < a.N;
       idx += (long long)gridDim.x * blockDim.x) {
    // phi* exactly as the step kernel forms it (the nonlocal families are
    // Allen-Cahn: on D3Q7 the rest slot is zero and not read).
    float gv[QG];
#pragma unroll
    for (int q = 0; q < QG; ++q)
      gv[q] = (DIM == 3 && q == 0) ? 0.0f : pop_load<T, LG>(g + pop_ix<LG>(q, (unsigned)idx), q, P.gref);
    const float ps = phi_star<LG, DIM == 3>(gv);
    comp_add(h1, l1, P.four_beta_over_kappa * (ps - P.phiH) * (ps - P.phiL) * (ps - P.phi0));
    comp_add(h2, l2, (P.phiH - ps) * (ps - P.phiL));
  }
  double v1 = warp_sum((double)h1 + (double)l1);
  double v2 = warp_sum((double)h2 + (double)l2);
  __shared__ double s[2 * 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s[2 * warp] = v1;
    s[2 * warp + 1] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t1 += s[2 * w];
      t2 += s[2 * w + 1];
    }
    atomicAdd(&a.acc[0], t1);
    atomicAdd(&a.acc[1], t2);
  }
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int DIM, typename T>
static void launch_gamma(const GammaArgs& a, cudaStream_t s) {
  long long want = (a.N + 255) / 256;
  long long cap = 4LL * sm_count();
  gamma_kernel<DIM, T><<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(a);
}

void gamma_sums(int dim, int storage, const GammaArgs& a, cudaStream_t s) {
  if (dim == 2) {
    if (storage == 0) launch_gamma<2, float>(a, s);
    else if (storage == 1) launch_gamma<2, __half>(a, s);
    else launch_gamma<2, __nv_bfloat16>(a, s);
  } else {
    if (storage == 0) launch_gamma<3, float>(a, s);
    else if (storage == 1) launch_gamma<3, __half>(a, s);
    else launch_gamma<3, __nv_bfloat16>(a, s);
  }
}

// Canonical state <-> storage. The canonical f_q(x) is what the next step
// reads: slot q of x before an even step; before an odd step slot opp(q) of
// x - e_q, or slot q of x itself where x - e_q lies beyond a wall.
template <int DIM, typename T, int LAT>
__global__ void __launch_bounds__(kPassThreads) canon_kernel(const CanonArgs a, const PassGeo<DIM> G) {
  using LG = typename Lattices<DIM, LAT>::G;
  using LF = typename Lattices<DIM, LAT>::F;
  constexpr int QG = LG::Q, QF = LF::Q;
  const DevParams& P = a.p;
  const long long N = a.N;
  const int nx = P.nx, ny = P.ny, nz = (DIM == 3) ? P.nz : 1;
  T* g = static_cast<T*>(a.g);
  T* f = static_cast<T*>(a.f);
  pass_walk<DIM>(G, [&](const PassCell& cl) {
    const long long idx = cl.c;
    const int x = cl.x, y = cl.y, z = cl.z;
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      float* sp = a.state + (long long)q * N + idx;
      T* gp = g + pop_ix<LG>(q, (unsigned)idx);
      const bool skip = (DIM == 3 && !a.ch && q == 0);
      if (a.to_canon) *sp = skip ? 0.0f : pop_loadc<T, LG>(gp, q, P.gref);
      else if (!skip) pop_store<T, LG>(gp, q, *sp, P.gref);
    }
#pragma unroll
    for (int q = 0; q < QF; ++q) {
      long long src;
      int slot;
      if (a.parity == 0) {
        src = idx;
        slot = q;
      } else {
        int xs = x - LF::ex(q), ys = y - LF::ey(q), zs = z - LF::ez(q);
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        bool beyond = false;
        if (P.walls) beyond = (ys < 0 || ys >= ny);
        else ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
        if (beyond) {
          src = idx;
          slot = q;
        } else {
          src = xs + (long long)nx * (ys + (long long)ny * zs);
          slot = LF::opp(q);
        }
      }
      float* sp = a.state + (long long)(QG + q) * N + idx;
      T* fp = f + pop_ix<LF>(slot, (unsigned)src);
      if (a.to_canon) *sp = pop_loadc<T, LF>(fp, q, 0.0f);
      else pop_store<T, LF>(fp, q, *sp, 0.0f);
    }
    if (a.phiu) {
      for (int k = 0; k < DIM; ++k) {
        float* sp = a.state + (long long)(QG + QF + k) * N + idx;
        float* pp = a.phiu + (long long)k * N + idx;
        if (a.to_canon) *sp = *pp;
        else *pp = *sp;
      }
    }
  });
}

template <int DIM, typename T>
static void launch_canon(const CanonArgs& a, cudaStream_t s) {
  const PassGeo<DIM> G = pass_geo<DIM>(a.p.nx, a.p.ny, a.p.nz, sm_count());
  const dim3 grid = G.grid(), block(kPassTX, kPassTY);
  if (DIM == 3 && a.p.lat == 1) canon_kernel<DIM, T, (DIM == 3 ? 1 : 0)><<<grid, block, 0, s>>>(a, G);
  else canon_kernel<DIM, T, 0><<<grid, block, 0, s>>>(a, G);
}

void canon_copy(int dim, int storage, const CanonArgs& a, cudaStream_t s) {
  if (dim == 2) {
    if (storage == 0) launch_canon<2, float>(a, s);
    else if (storage == 1) launch_canon<2, __half>(a, s);
    else launch_canon<2, __nv_bfloat16>(a, s);
  } else {
    if (storage == 0) launch_canon<3, float>(a, s);
    else if (storage == 1) launch_canon<3, __half>(a, s);
    else launch_canon<3, __nv_bfloat16>(a, s);
  }
}

}  // namespace pflb
