// Cell walk of the per-cell pass kernels (the Bao2024 and Liu2023 passes,
// the adjoint's reverse sweep, the canonical copy): blocks of 32 x 8 threads
// over (x, y), each marching over a run of z planes. Coordinates are
// known from the launch, so no cell index is ever divided; the periodic
// neighbour offsets of the x and y axes are built once per thread and those
// of z once per plane. A warp covers 32 consecutive x of one row, i.e. one
// 32-cell group of the block-interleaved population layout when nx is a
// multiple of 32.
#pragma once

#include "pflb_common.cuh"

namespace pflb {

constexpr int kPassTX = 32, kPassTY = 8, kPassThreads = kPassTX * kPassTY;

int num_sms();   // SMs of the current device (pflb_api.cu)

template <int DIM>
struct PassGeo {
  int nx, ny, nz;
  int zc;   // planes per block (1 in 2D)

  __host__ dim3 grid() const {
    return dim3((unsigned)((nx + kPassTX - 1) / kPassTX), (unsigned)((ny + kPassTY - 1) / kPassTY),
                DIM == 3 ? (unsigned)((nz + zc - 1) / zc) : 1u);
  }
};

// Planes per block: about 32 blocks per SM over the grid (several waves of
// resident blocks), runs of at most 32 planes, long enough that a block's
// neighbour planes are still in its L1 when it reaches them.
template <int DIM>
__host__ inline PassGeo<DIM> pass_geo(int nx, int ny, int nz, int sms) {
  PassGeo<DIM> G{nx, ny, DIM == 3 ? nz : 1, 1};
  if (DIM == 3) {
    const long long tiles = (long long)((nx + kPassTX - 1) / kPassTX) * ((ny + kPassTY - 1) / kPassTY);
    const long long target = 32LL * sms;
    long long zc = (tiles * nz + target - 1) / target;
    if (zc < 1) zc = 1;
    if (zc > 32) zc = 32;
    if (zc > nz) zc = nz;
    G.zc = (int)zc;
  }
  return G;
}

// One cell of the walk: its coordinates, index and the offsets that give the
// index of any neighbour x + e (|e_i| <= 1) as ox[ex+1] + oy[ey+1] + oz[ez+1].
struct PassCell {
  int x, y, z;
  unsigned c;
  unsigned ox[3], oy[3], oz[3];
  __device__ __forceinline__ unsigned nb(int ex, int ey, int ez) const { return ox[ex + 1] + oy[ey + 1] + oz[ez + 1]; }
};

// Calls fn(const PassCell&) for every cell of this block's run. Threads
// outside the domain call nothing but return normally (kernels that reduce
// over the block afterwards need every thread).
template <int DIM, typename Fn>
__device__ __forceinline__ void pass_walk(const PassGeo<DIM>& G, Fn&& fn) {
  PassCell k;
  k.x = (int)(blockIdx.x * kPassTX + threadIdx.x);
  k.y = (int)(blockIdx.y * kPassTY + threadIdx.y);
  if (k.x >= G.nx || k.y >= G.ny) return;
  const unsigned nx = (unsigned)G.nx, nxy = (unsigned)G.nx * (unsigned)G.ny;
  k.ox[0] = (unsigned)(k.x == 0 ? G.nx - 1 : k.x - 1);
  k.ox[1] = (unsigned)k.x;
  k.ox[2] = (unsigned)(k.x == G.nx - 1 ? 0 : k.x + 1);
  k.oy[0] = nx * (unsigned)(k.y == 0 ? G.ny - 1 : k.y - 1);
  k.oy[1] = nx * (unsigned)k.y;
  k.oy[2] = nx * (unsigned)(k.y == G.ny - 1 ? 0 : k.y + 1);
  const int z0 = DIM == 3 ? (int)blockIdx.z * G.zc : 0;
  const int z1 = DIM == 3 ? min(G.nz, z0 + G.zc) : 1;
  for (int z = z0; z < z1; ++z) {
    k.z = z;
    if (DIM == 3) {
      k.oz[0] = nxy * (unsigned)(z == 0 ? G.nz - 1 : z - 1);
      k.oz[1] = nxy * (unsigned)z;
      k.oz[2] = nxy * (unsigned)(z == G.nz - 1 ? 0 : z + 1);
    } else {
      k.oz[0] = k.oz[1] = k.oz[2] = 0u;
    }
    k.c = k.ox[1] + k.oy[1] + k.oz[1];
    fn(k);
  }
}

// L2 prefetch hint for the 128-byte line holding *p (callers pass addresses
// inside their buffers; nothing is returned).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Row start of the warp's 32 cells in the next plane (x lane = threadIdx.x),
// or -1 when the cell is in the last plane. The per-cell passes are bound by
// the latency of their many dependent loads; asking L2 for the next plane's
// rows one plane ahead overlaps it with the current cell.
template <int DIM>
__device__ __forceinline__ long long next_plane_row(const PassGeo<DIM>& G, const PassCell& cl) {
  if (DIM != 3 || cl.z + 1 >= G.nz) return -1;
  return (long long)(cl.c - threadIdx.x) + (long long)G.nx * G.ny;
}

// Line q of the population group (32 cells, Q values each) that holds cell r.
template <typename L>
__device__ __forceinline__ const float* group_line(const float* pops, long long r, int q) {
  return pops + ((size_t)(r >> 5) * L::Q + q) * 32;
}

}  // namespace pflb
