// Step and init kernels of the conservative Allen-Cahn (Fakhari2017), Sec. II C 1: every dimension and
// storage form, instantiated in their own translation unit so the families
// compile in parallel.
#include "pflb_init.cuh"

namespace pflb {

void step_fakhari(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  step_dispatch<FAM_FAKHARI>(dim, storage, a, s);
}

void init_fakhari(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_FAKHARI>(dim, storage, a, s);
}

}  // namespace pflb
