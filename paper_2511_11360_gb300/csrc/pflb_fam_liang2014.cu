// Step and init kernels of the Cahn-Hilliard (Liang2014), Sec. II D 1: every dimension and
// storage form, instantiated in their own translation unit so the families
// compile in parallel.
#include "pflb_init.cuh"

namespace pflb {

void step_liang2014(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  step_dispatch<FAM_LIANG>(dim, storage, a, s);
}

void init_liang2014(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_LIANG>(dim, storage, a, s);
}

}  // namespace pflb
