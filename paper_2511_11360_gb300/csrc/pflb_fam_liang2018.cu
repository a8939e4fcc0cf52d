// Step and init kernels of Liang2018 (conservative Allen-Cahn with the
// conservative form of the Navier-Stokes equations), Sec. II C 2: every
// dimension and storage form, instantiated in their own translation unit so
// the families compile in parallel.
#include "pflb_init.cuh"

namespace pflb {

void step_liang2018(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  step_dispatch<FAM_LIANG18>(dim, storage, a, s);
}

void init_liang2018(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_LIANG18>(dim, storage, a, s);
}

}  // namespace pflb
