// Host side of the TMA staging: the tensor maps of a handle's population
// arrays, built once when the handle is created.
//
// cuTensorMapEncodeTiled is a driver function; it is fetched through the
// runtime's driver entry point, so the library links no driver library. The
// maps are plain 128-byte descriptors held in host memory and passed by value
// to the kernel (parameter space), one set per g source buffer.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <new>

#include "pflb_internal.h"

namespace pflb {

namespace {

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || p == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Map over a population array of Q slots viewed as the 5-D tensor
// (lane 32, slot Q, x-block nx/32, y ny, z nz), box {b0, b1, 1, b3, 1}.
// The constraints of a tiled map are checked here first: base and strides
// multiples of 16 bytes, the box's innermost extent a multiple of 16 bytes,
// every box extent in 1 .. 256.
bool encode(CUtensorMap* m, const void* base, int storage, int Q, int nx, int ny, int nz, unsigned b0, unsigned b1,
            unsigned b3) {
  EncodeTiled fn = encoder();
  if (!fn) return false;
  const unsigned long long es = storage == 0 ? 4ull : 2ull;
  const CUtensorMapDataType dt = storage == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : storage == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[5] = {32ull, (cuuint64_t)Q, (cuuint64_t)(nx / 32), (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[4] = {32ull * es, 32ull * Q * es, (cuuint64_t)Q * nx * es, (cuuint64_t)Q * nx * ny * es};
  const cuuint32_t box[5] = {b0, b1, 1u, b3, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  if (((unsigned long long)(size_t)base) % 16ull != 0ull) return false;
  for (int i = 0; i < 4; ++i)
    if (strides[i] % 16ull != 0ull || strides[i] >= (1ull << 40)) return false;
  if ((b0 * es) % 16ull != 0ull) return false;
  for (int i = 0; i < 5; ++i)
    if (box[i] < 1u || box[i] > 256u || box[i] > dims[i]) return false;
  return fn(m, dt, 5, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool handle_tma_eligible(const pflb_handle* h) {
  const pflb_params& p = h->prm;
  if (p.dim != 3) return false;
  if (!(p.family == PFLB_CAC_FAKHARI2017 || p.family == PFLB_NLAC_CHAI2018 || p.family == PFLB_HAC_HU2019 ||
        p.family == PFLB_CAC_LIANG2018))
    return false;
  const TileShape t = tile_shape(p.family, 3, p.storage, p.lattice_f == 27 ? 1 : 0);
  if (t.ta != 32 || p.nx % 32 != 0) return false;
  return p.ny % t.tb == 0 && p.ny >= 2 * t.tb;
}

int handle_build_tma(pflb_handle* h) {
  for (int b = 0; b < 2; ++b) {
    delete h->tma[b];
    h->tma[b] = nullptr;
  }
  if (!handle_tma_eligible(h)) return 0;
  const pflb_params& p = h->prm;
  const int tb = tile_shape(p.family, 3, p.storage, p.lattice_f == 27 ? 1 : 0).tb;
  const unsigned sl = p.storage == 0 ? 4u : 8u;    // 16 bytes of lanes
  const unsigned qgs = (unsigned)h->QG - 1u;        // D3Q7 slots 1..6 (the rest slot is not stored)
  const unsigned qf = (unsigned)h->QF;
  for (int b = 0; b < 2; ++b) {
    TmaMaps* m = new (std::nothrow) TmaMaps();
    if (!m) return 0;
    const void* g = h->g[b];
    bool ok = encode(&m->m[TM_G_MAIN], g, p.storage, h->QG, p.nx, p.ny, p.nz, 32u, qgs, (unsigned)tb + 2u) &&
              encode(&m->m[TM_G_SIDE], g, p.storage, h->QG, p.nx, p.ny, p.nz, sl, qgs, (unsigned)tb + 2u) &&
              encode(&m->m[TM_F_ALL], h->f, p.storage, h->QF, p.nx, p.ny, p.nz, 32u, qf, (unsigned)tb) &&
              encode(&m->m[TM_F_MAIN], h->f, p.storage, h->QF, p.nx, p.ny, p.nz, 32u, 1u, (unsigned)tb) &&
              encode(&m->m[TM_F_SIDE], h->f, p.storage, h->QF, p.nx, p.ny, p.nz, sl, 1u, (unsigned)tb);
    if (!ok) {
      delete m;
      for (int c = 0; c < 2; ++c) {
        delete h->tma[c];
        h->tma[c] = nullptr;
      }
      return 0;
    }
    h->tma[b] = m;
  }
  return 1;
}

// Staging of a step of the given AA parity. Mode 2 (the default) takes TMA
// where it measured faster at 512^3: FP32 D3Q19 on both parities (4.10 /
// 5.39 ms against 5.06 / 5.57 with cp.async), FP32 D3Q27 on even steps
// (5.49 against 6.63 ms; odd: 9.42 against 7.77); the 16-bit forms keep
// cp.async (issue-bound: FP16 even 3.99 against 3.93 ms, odd 5.92 against
// 4.58).
bool handle_tma_step(const pflb_handle* h, int parity) {
  if (h->staging == 1) return true;
  if (h->staging != 2 || h->storage != 0) return false;
  return h->QF == 19 || (h->QF == 27 && parity == 0);
}

}  // namespace pflb

// Upper bound on the test hook's poll count (each poll of an mbarrier may
// suspend the thread for a short, hardware-chosen time).
static constexpr int kMaxTestWaitPolls = 1 << 16;

int pflb_set_staging(pflb_handle* h, int32_t mode) {
  if (!h || mode < 0 || mode > 2) return pflb::handle_fail(h, PFLB_EINVAL, "staging mode must be 0, 1 or 2");
  h->staging = mode;
  return PFLB_OK;
}

int pflb_inject_wait_timeout(pflb_handle* h, int32_t polls) {
  if (!h || polls < 0 || polls > kMaxTestWaitPolls)
    return pflb::handle_fail(h, PFLB_EINVAL, "polls must be in [0, %d]", kMaxTestWaitPolls);
  if (polls > 0 && pflb_get_staging(h) != 1)
    return pflb::handle_fail(h, PFLB_EINVAL, "the wait-timeout hook needs a TMA-staged step (pflb_get_staging)");
  h->test_wait_polls = polls;
  return PFLB_OK;
}

int pflb_get_staging(const pflb_handle* h) {
  if (!h) return PFLB_EINVAL;
  return (pflb::handle_tma_step(h, (int)(h->step & 1)) && h->tma[h->cur] != nullptr) ? 1 : 0;
}
