// Step and init kernels of the hybrid Allen-Cahn (Hu2019), Sec. II C 4: every dimension and
// storage form, instantiated in their own translation unit so the families
// compile in parallel.
#include "pflb_init.cuh"

namespace pflb {

void step_hu(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  step_dispatch<FAM_HU>(dim, storage, a, s);
}

void init_hu(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_HU>(dim, storage, a, s);
}

}  // namespace pflb
