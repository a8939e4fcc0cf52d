// pflb_phase_sums_static: the phase-field sums of a caller's phi field, for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: an application that budgets all
// device memory through its own allocator and forbids allocations it does not
// make, or a latency-bound loop that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree imply. This entry point needs no
// allocation: its scratch space is a file-scope device array that every GPU
// loading the library holds until the process exits.
//
// Scratch: PFLB_STATIC_PARTIALS per-block partial records plus one result
// record. Pass 1 has each block reduce PFLB_STATIC_CELLS_PER_BLOCK cells (or
// fewer) into its own record; pass 2 reduces the records in a fixed order.
// Every record used is written in full before it is read, so nothing needs
// clearing between calls, and the result is deterministic. The array keeps
// the last call's contents. Calls that overlap on the GPU (other streams,
// other host threads) share the array and race: serialise them. The call
// copies its result to the host and synchronises the stream, so it cannot
// be used while the stream is being captured into a CUDA graph.
#include "../../include/pflb.h"
#include "pflb_common.cuh"

namespace {

struct Partial {
  double sum_phi, vol_smooth, cx, cy, cz;
  unsigned long long count;
  float mx, mn;
};

constexpr int kThreads = 256;
constexpr long long kCellsPerBlock = PFLB_STATIC_CELLS_PER_BLOCK;
constexpr int kPartials = PFLB_STATIC_PARTIALS;

static __device__ __align__(256) Partial g_scratch[kPartials + 1];

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads) phase_sums_pass1(
    const float* __restrict__ phi, long long N, int nx, int ny, float phiL, float inv_dphi,
    float phi0, Partial* scratch) {
  const long long begin = blockIdx.x * kCellsPerBlock;
  const long long end = begin + kCellsPerBlock < N ? begin + kCellsPerBlock : N;
  double s = 0.0, vs = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
  unsigned long long cnt = 0;
  float mx = -3.0e38f, mn = 3.0e38f;
  for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
    const float p = phi[i];
    const float fr = (p - phiL) * inv_dphi;
    const long long x = i % nx, y = (i / nx) % ny, z = i / ((long long)nx * ny);
    s += (double)p;
    vs += (double)fr;
    cx += (double)x * fr;
    cy += (double)y * fr;
    cz += (double)z * fr;
    cnt += (p > phi0) ? 1ull : 0ull;
    mx = fmaxf(mx, p);
    mn = fminf(mn, p);
  }
  s = wsum(s); vs = wsum(vs); cx = wsum(cx); cy = wsum(cy); cz = wsum(cz);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  __shared__ Partial w[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) w[warp] = Partial{s, vs, cx, cy, cz, cnt, mx, mn};
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = w[0];
    for (int k = 1; k < kThreads / 32; ++k) {
      r.sum_phi += w[k].sum_phi; r.vol_smooth += w[k].vol_smooth;
      r.cx += w[k].cx; r.cy += w[k].cy; r.cz += w[k].cz;
      r.count += w[k].count;
      r.mx = fmaxf(r.mx, w[k].mx); r.mn = fminf(r.mn, w[k].mn);
    }
    scratch[blockIdx.x] = r;
  }
}

// One thread reduces the partial records in block order into record kPartials.
__global__ void phase_sums_pass2(int nblocks, Partial* scratch) {
  Partial r = scratch[0];
  for (int k = 1; k < nblocks; ++k) {
    const Partial& q = scratch[k];
    r.sum_phi += q.sum_phi; r.vol_smooth += q.vol_smooth;
    r.cx += q.cx; r.cy += q.cy; r.cz += q.cz;
    r.count += q.count;
    r.mx = fmaxf(r.mx, q.mx); r.mn = fminf(r.mn, q.mn);
  }
  scratch[kPartials] = r;
}

// Device address of g_scratch on the current device. The host-side name of a
// __device__ array is not a device address, so it is looked up with the
// device current -- on every call: the lookup is cheap, and a cached address
// would go stale after cudaDeviceReset or a new context.
int scratch_address(Partial** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return PFLB_ECUDA;
  }
  *out = static_cast<Partial*>(p);
  return PFLB_OK;
}

}  // namespace

extern "C" int pflb_phase_sums_static(const pflb_params* params, const float* phi, pflb_obs* out,
                                      void* cuda_stream) {
  if (!params || !phi || !out) return PFLB_EINVAL;
  if (params->dim != 2 && params->dim != 3) return PFLB_EINVAL;
  if (params->nx < 1 || params->ny < 1 || params->nz < 1) return PFLB_EINVAL;
  if (!(params->phi_H != params->phi_L)) return PFLB_EINVAL;
  const long long nz = params->dim == 3 ? params->nz : 1;
  const long long N = (long long)params->nx * params->ny * nz;
  if (N > PFLB_STATIC_MAX_CELLS) return PFLB_EINVAL;  // beyond the scratch array
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { cudaGetLastError(); return PFLB_ECUDA; }
  Partial* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != PFLB_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = (int)((N + kCellsPerBlock - 1) / kCellsPerBlock);
  const double dphi = params->phi_H - params->phi_L;
  phase_sums_pass1<<<nblocks, kThreads, 0, s>>>(phi, N, params->nx, params->ny, (float)params->phi_L,
                                                (float)(1.0 / dphi),
                                                (float)(0.5 * (params->phi_H + params->phi_L)), scratch);
  phase_sums_pass2<<<1, 1, 0, s>>>(nblocks, scratch);
  Partial r;
  if (cudaMemcpyAsync(&r, scratch + kPartials, sizeof(Partial), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return PFLB_ECUDA;
  }
  out->step = -1;
  out->sum_phi = r.sum_phi;
  out->vol_smooth = r.vol_smooth;
  out->vol_count = (int64_t)r.count;
  out->ke = 0.0;
  out->phi_max = r.mx;
  out->phi_min = r.mn;
  out->centroid[0] = r.vol_smooth != 0.0 ? r.cx / r.vol_smooth : 0.0;
  out->centroid[1] = r.vol_smooth != 0.0 ? r.cy / r.vol_smooth : 0.0;
  out->centroid[2] = r.vol_smooth != 0.0 ? r.cz / r.vol_smooth : 0.0;
  out->status = PFLB_OK;
  out->pad = 0;
  return PFLB_OK;
}
