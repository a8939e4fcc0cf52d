// Kernels of the batched step: many 2D domains of uneven size, family and
// parameters advanced by one persistent launch per family (FP32 storage).
//
// The tile work list holds every (domain, x-tile, y-chunk) of the batch,
// grouped by family. Resident blocks claim tiles of their family from an
// atomic counter until that range is exhausted; each tile runs the same per-cell update as the single-domain
// kernel (step_tile), so a domain advanced in a batch is bitwise identical
// to the same domain advanced alone (its observables differ only in the
// order of the FP64 sums). The counter of the next step is reset by the
// current one, so consecutive launches (or a replayed graph of them) need
// no host work in between.
#include "pflb_step.cuh"

namespace pflb {

template <int TA>
struct BatchGeom {
  // Registers are capped at 128 per thread, as for the single-domain 2D kernel.
  static constexpr int MINB = 512 / TA;
};

// One family's tiles: the resident blocks of this kernel claim the tiles of
// one family (a contiguous range of the work list) from that family's
// counter, so each kernel holds one family's code and shared-memory
// footprint. The families' kernels of one step run as concurrent branches
// (the host forks them on separate streams), so one family's last tiles
// overlap the next family's first ones.
template <int TA, int FAM>
__global__ void __launch_bounds__(TA, BatchGeom<TA>::MINB) batch_step_kernel(const BatchArgs ba) {
  using SMX = TileSmem<FAM, 2, float, TA, 1>;
  extern __shared__ __align__(16) float dyn_smem[];
  float* s_stage = dyn_smem;
  float* s_phi = dyn_smem + SMX::STAGE;
  float* s_mu = s_phi + SMX::PHI;
  __shared__ double s_red[(TA / 32) * 10];
  __shared__ __align__(16) StepArgs s_args;
  __shared__ int s_tile;
  static_assert(sizeof(StepArgs) % 4 == 0, "StepArgs is copied as 32-bit words");
  const int tid = threadIdx.x;

  if (blockIdx.x == 0 && tid == 0) *ba.counter_next = 0u;
  // the next step's observables slot of this family's domains
  for (int i = blockIdx.x * TA + tid; i < ba.ninst; i += gridDim.x * TA) {
    DevObs* z = ba.args[i].obs_zero;
    if (z != nullptr && ba.args[i].p.family == FAM) obs_zero_slot(z);
  }

  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(ba.counter, 1u);
    __syncthreads();
    const int t = s_tile;
    if (t >= ba.ntiles) break;
    const BatchTile e = ba.tiles[t];
    {
      const int* src = reinterpret_cast<const int*>(ba.args + e.inst);
      int* dst = reinterpret_cast<int*>(&s_args);
      for (int k = tid; k < (int)(sizeof(StepArgs) / 4); k += TA) dst[k] = src[k];
    }
    __syncthreads();
    ObsPartial obs;
    obs_init(obs);
    // Widths that are a multiple of the population block take the
    // constant-offset addressing (the sweep's widths all are).
    if (s_args.p.nx % (int)kPopBlock == 0)
      step_tile<FAM, 2, float, TA, 1, -1, 1>(s_args, e.a0, 0, e.c0, ba.chunk, s_phi, s_mu, s_stage, obs);
    else
      step_tile<FAM, 2, float, TA, 1, -1, 0>(s_args, e.a0, 0, e.c0, ba.chunk, s_phi, s_mu, s_stage, obs);
    obs_block_commit(obs, s_args.obs_slot, s_red);
    __syncthreads();  // s_tile, s_args and the rings are rewritten by the next tile
  }
}

// Batched form of the nonlocal pre-pass (Eq. lagrange_multiplier, Reading
// R1): each entry is a cell range of one nonlocal/hybrid domain; the block
// adds its range's (I1, I2) to that domain's pair for this step. The first
// threads also zero every domain's pair of the next step.
__global__ void __launch_bounds__(256) batch_gamma_kernel(const BatchGammaArgs ga) {
  using LG = D2Q9;
  __shared__ double s[2 * 8];
  const int tid = threadIdx.x;
  for (int i = blockIdx.x * 256 + tid; i < ga.ninst; i += gridDim.x * 256) {
    double* z = ga.args[i].gamma_next;
    if (z != nullptr) {
      z[0] = 0.0;
      z[1] = 0.0;
    }
  }
  for (int k = blockIdx.x; k < ga.nent; k += gridDim.x) {
    const BatchGammaEntry e = ga.ent[k];
    const StepArgs& A = ga.args[e.inst];
    const float* g = static_cast<const float*>(A.g_src);
    const float fbk = A.p.four_beta_over_kappa, pH = A.p.phiH, pL = A.p.phiL, p0 = A.p.phi0;
    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    for (int idx = e.begin + tid; idx < e.end; idx += 256) {
      float gv[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) gv[q] = g[pop_ix<LG>(q, (unsigned)idx)];
      const float ps = phi_star<LG, false>(gv);
      comp_add(h1, l1, fbk * (ps - pH) * (ps - pL) * (ps - p0));
      comp_add(h2, l2, (pH - ps) * (ps - pL));
    }
    double v1 = warp_sum((double)h1 + (double)l1);
    double v2 = warp_sum((double)h2 + (double)l2);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
      s[2 * warp] = v1;
      s[2 * warp + 1] = v2;
    }
    __syncthreads();
    if (tid == 0) {
      double t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < 8; ++w) {
        t1 += s[2 * w];
        t2 += s[2 * w + 1];
      }
      double* acc = const_cast<double*>(A.gamma_acc);
      atomicAdd(&acc[0], t1);
      atomicAdd(&acc[1], t2);
    }
    __syncthreads();
  }
}

__global__ void obs_gather_kernel(const DevObs* const* src, DevObs* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = *src[i];
}

bool batch_tile_supported(int tile_a) { return tile_a == 64 || tile_a == 128 || tile_a == 256; }

template <int TA, int FAM>
static size_t batch_smem() {
  constexpr size_t smem = TileSmem<FAM, 2, float, TA, 1>::BYTES;
  static const cudaError_t attr =
      cudaFuncSetAttribute(batch_step_kernel<TA, FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  (void)attr;
  return smem;
}

template <int TA, int FAM>
static int max_blocks() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_step_kernel<TA, FAM>, TA, batch_smem<TA, FAM>()) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b > 0 ? b : 1;
}

template <int TA>
static int max_blocks_ta(int fam) {
  switch (fam) {
    case FAM_FAKHARI: return max_blocks<TA, FAM_FAKHARI>();
    case FAM_CHAI: return max_blocks<TA, FAM_CHAI>();
    case FAM_HU: return max_blocks<TA, FAM_HU>();
    case FAM_LIANG: return max_blocks<TA, FAM_LIANG>();
    default: return max_blocks<TA, FAM_LIANG18>();
  }
}

int batch_max_blocks_per_sm(int tile_a, int fam) {
  switch (tile_a) {
    case 64: return max_blocks_ta<64>(fam);
    case 128: return max_blocks_ta<128>(fam);
    default: return max_blocks_ta<256>(fam);
  }
}

template <int TA>
static void step_ta(int fam, const BatchArgs& a, int grid, cudaStream_t s) {
  switch (fam) {
    case FAM_FAKHARI:
      batch_step_kernel<TA, FAM_FAKHARI><<<grid, TA, batch_smem<TA, FAM_FAKHARI>(), s>>>(a);
      break;
    case FAM_CHAI: batch_step_kernel<TA, FAM_CHAI><<<grid, TA, batch_smem<TA, FAM_CHAI>(), s>>>(a); break;
    case FAM_HU: batch_step_kernel<TA, FAM_HU><<<grid, TA, batch_smem<TA, FAM_HU>(), s>>>(a); break;
    case FAM_LIANG: batch_step_kernel<TA, FAM_LIANG><<<grid, TA, batch_smem<TA, FAM_LIANG>(), s>>>(a); break;
    default: batch_step_kernel<TA, FAM_LIANG18><<<grid, TA, batch_smem<TA, FAM_LIANG18>(), s>>>(a); break;
  }
}

void batch_step(int tile_a, int fam, const BatchArgs& a, int grid, cudaStream_t s) {
  switch (tile_a) {
    case 64: step_ta<64>(fam, a, grid, s); break;
    case 128: step_ta<128>(fam, a, grid, s); break;
    default: step_ta<256>(fam, a, grid, s); break;
  }
}

void batch_gamma(const BatchGammaArgs& a, int grid, cudaStream_t s) {
  batch_gamma_kernel<<<grid, 256, 0, s>>>(a);
}

void batch_obs_gather(const DevObs* const* src, DevObs* dst, int n, cudaStream_t s) {
  if (n > 0) obs_gather_kernel<<<(n + 127) / 128, 128, 0, s>>>(src, dst, n);
}

}  // namespace pflb
