// Launch arguments of the PF-LB kernels and the host-side entry points of
// each translation unit (no kernel code here).
#pragma once

#include "pflb_common.cuh"
#include "pflb_tma.cuh"

namespace pflb {

// Tile of the single-domain step kernel: cells per block along the two fast
// axes (ta x tb) and the resident blocks per SM its register budget is sized
// for. The 3D Allen-Cahn tiles fit 128 registers a thread without spills and
// run four blocks per SM (16 warps; FP32 with three f stages so that four
// blocks fit in shared memory): 16-bit storage, bound by instruction issue,
// went from 31.3 to 32.5 GLUPS at 512^3 against three blocks, FP32 from 24.7
// to 25.3. D3Q27 and Cahn-Hilliard tiles run three and two blocks per SM at
// up to 168 registers.
struct TileShape {
  int ta, tb, minb;
};
__host__ __device__ constexpr TileShape tile_shape(int family, int dim, int storage, int lat = 0) {
  // D3Q27 holds 27 populations (and with MRT their moments) a thread: three
  // blocks per SM at 168 registers (no spills).
  return (void)storage, dim == 2 ? TileShape{128, 1, 4}
         : family == 3 ? TileShape{32, 6, 2}
         : lat == 1 ? TileShape{32, 4, 3} : TileShape{32, 4, 4};
}

struct StepArgs {
  DevParams p;
  const void* g_src;
  void* g_dst;
  void* f;
  float* phiu;            // Liang2014/Liang2018: phi*u of the previous step (d x N), in place
  DevObs* obs_slot;       // accumulate the observables here
  DevObs* obs_zero;       // zero this slot (the next step's), may be null
  const double* gamma_acc;// nonlocal/hybrid: (I1, I2) of this step
  int parity;             // 0: even step, 1: odd step (AA pattern)
  int macro;              // 1: write fields, no populations
  float* out_phi;
  float* out_u;
  float* out_p;
  int chunk;              // cells per block along the marching axis
  long long N;
  double* gamma_next;     // nonlocal/hybrid: the next step's pair (zeroed by the batched pre-pass)
  float* work;            // Bao2024: phi, mu, p, u fields ((3 + d) x N); Liu2023: 6 x N
  const TmaMaps* tma = nullptr;  // host copy of this step's tensor maps (TMA staging), or null
  unsigned seed = 0u;     // step counter: seeds the stochastic rounding of 16-bit stores
  int test_wait_polls = 0;  // > 0: TMA-staged blocks first run out a wait of this many polls (test hook)
};

struct InitArgs {
  DevParams p;
  const float* phi0;
  const float* u0;        // may be null (rest)
  void* g;
  void* f;
  float* phiu;
  long long N;
  float* work;            // Bao2024: (3 + d) x N work fields
};

struct GammaArgs {
  DevParams p;
  const void* g_src;
  double* acc;            // (I1, I2) accumulated here
  double* zero;           // zeroed (the next step's pair), may be null
  long long N;
};

struct CanonArgs {
  DevParams p;
  void* g;                // current source g
  void* f;                // AA buffer
  float* phiu;
  float* state;           // canonical FP32 state
  int parity;             // parity of the next step
  int to_canon;           // 1: storage -> state (save); 0: state -> storage (load)
  int ch;                 // Cahn-Hilliard (g_0 stored in 3D); the phi*u block is present when phiu != null
  long long N;
};

// One tile of the batched step: instance, first cell along x, first row of
// the chunk along y, family of the instance.
struct BatchTile {
  int inst, a0, c0, fam;
};

// A contiguous cell range of one nonlocal/hybrid instance for the batched
// gamma pre-pass.
struct BatchGammaEntry {
  int inst, begin, end, pad;
};

struct BatchArgs {
  const StepArgs* args;     // per instance: this step's arguments
  const BatchTile* tiles;   // this family's tiles
  int ntiles;
  int ninst;
  int chunk;                // rows per tile along y
  unsigned* counter;        // tile claims of this step (zero at launch)
  unsigned* counter_next;   // the next step's counter, reset here
};

struct BatchGammaArgs {
  const StepArgs* args;
  const BatchGammaEntry* ent;
  int nent;
  int ninst;
};

// Per-family translation units.
void step_fakhari(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_chai(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_hu(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_liang2014(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_liang2018(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_bao2024(int dim, int storage, const StepArgs& a, cudaStream_t s);
void step_liu2023(int dim, int storage, const StepArgs& a, cudaStream_t s);
void init_fakhari(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_chai(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_hu(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_liang2014(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_liang2018(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_bao2024(int dim, int storage, const InitArgs& a, cudaStream_t s);
void init_liu2023(int dim, int storage, const InitArgs& a, cudaStream_t s);
// pflb_aux.cu
void gamma_sums(int dim, int storage, const GammaArgs& a, cudaStream_t s);
void canon_copy(int dim, int storage, const CanonArgs& a, cudaStream_t s);
// pflb_batch_kernels.cu (2D, FP32 storage)
bool batch_tile_supported(int tile_a);
int batch_max_blocks_per_sm(int tile_a, int fam);
void batch_step(int tile_a, int fam, const BatchArgs& a, int grid, cudaStream_t s);
void batch_gamma(const BatchGammaArgs& a, int grid, cudaStream_t s);
void batch_obs_gather(const DevObs* const* src, DevObs* dst, int n, cudaStream_t s);

}  // namespace pflb
