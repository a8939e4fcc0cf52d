// Step and init kernels of the nonlocal Allen-Cahn (Chai2018), Sec. II C 3: every dimension and
// storage form, instantiated in their own translation unit so the families
// compile in parallel.
#include "pflb_init.cuh"

namespace pflb {

void step_chai(int dim, int storage, const StepArgs& a, cudaStream_t s) {
  step_dispatch<FAM_CHAI>(dim, storage, a, s);
}

void init_chai(int dim, int storage, const InitArgs& a, cudaStream_t s) {
  init_dispatch<FAM_CHAI>(dim, storage, a, s);
}

}  // namespace pflb
