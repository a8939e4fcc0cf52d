// Host-side state shared by the translation units of the C ABI: the handle of
// one domain and the helpers the batch entry points reuse.
#pragma once

#include <nvtx3/nvToolsExt.h>   // header-only NVTX v3 (no link dependency)

#include "../../include/pflb.h"
#include "pflb_args.h"

// NVTX range over one C ABI call (a host-side range around the launches it
// enqueues: profilers can filter kernels by it, e.g. ncu --nvtx).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct pflb_handle {
  pflb_params prm;
  pflb::DevParams dp;
  cudaStream_t stream = nullptr;
  int dim = 2, QG = 9, QF = 9, storage = 0, family = 0;
  long long N = 0;
  size_t elem = 4;
  void* g[2] = {nullptr, nullptr};
  void* f = nullptr;
  float* phiu = nullptr;
  float* work = nullptr;        // work fields: Bao2024 (3 + d) x N, Liu2023 6 x N
  pflb::DevObs* obs = nullptr;  // ring of obs_cap slots + 1 slot for read-only passes
  int obs_cap = 2;
  double* gamma_acc = nullptr;  // 3 pairs: step ring (2) + read-only pass (1)
  float* scratch = nullptr;     // N*(d+2) floats, for host-side transfers
  long long step = 0;
  int cur = 0;                  // index of the source g array
  int chunk = 0;
  int initialized = 0;         // set by pflb_init
  int status = PFLB_OK;
  char err[512] = {0};
  pflb::TmaMaps* tma[2] = {nullptr, nullptr};  // tensor maps per g source buffer (TMA staging), or null
  int test_wait_polls = 0;      // wait-timeout test hook (pflb_inject_wait_timeout)
  int staging = 2;              // 0 cp.async staging; 1 TMA where the geometry allows it; 2 TMA where it measured faster
};

namespace pflb {

int num_sms();
// Nonlocal or hybrid Allen-Cahn (needs the global gamma pre-pass).
bool handle_nonlocal(const pflb_handle* h);
// Launch arguments of the next step of h (no observables slots set).
StepArgs handle_step_args(const pflb_handle* h);
// Copy between the handle's storage and a canonical FP32 state in device
// memory (to_canon = 1: storage -> state), asynchronously on its stream.
int handle_canon(pflb_handle* h, float* state_dev, int to_canon);
// Host form of a device observables record.
void obs_to_host(const DevObs& d, long long step, pflb_obs* o);
// TMA staging: whether the handle's geometry and family allow it, and the
// tensor maps of its arrays (returns 1 when built; 0 leaves the cp.async path).
bool handle_tma_eligible(const pflb_handle* h);
int handle_build_tma(pflb_handle* h);
// Whether a step of the given AA parity is staged by TMA under the handle's
// staging mode (pflb_set_staging), given that its tensor maps were built.
bool handle_tma_step(const pflb_handle* h, int parity);
// Records a message and a sticky status on h; returns code.
int handle_fail(pflb_handle* h, int code, const char* fmt, ...);

}  // namespace pflb
