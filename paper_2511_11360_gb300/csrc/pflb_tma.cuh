// Tensor-memory-accelerator (TMA) staging of the fused step's populations:
// the tensor maps the host builds over the population arrays, and the
// mbarrier / bulk-tensor-copy primitives the kernel uses (inline PTX).
//
// View of a population array. Population q of cell (x, y, z) sits at element
// ((i / 32) Q + q) 32 + i % 32 with i = x + nx (y + ny z) (pop_ix). When nx
// is a multiple of 32 that is a dense 5-D tensor, innermost first:
//   lane (32) x slot (Q) x x-block (nx / 32) x y (ny) x z (nz),
// strides 32, 32 Q, Q nx, Q nx ny elements. A tile of 32 x TB cells of one
// plane is one box {32, slots, 1, rows, 1}; the one-cell x halo lies in the
// neighbouring x-blocks, so it comes as a box of SL lanes (16 bytes: lanes
// 32 - SL .. 31 of the block to the left, 0 .. SL - 1 of the block to the
// right). Periodic wraps in x and z are coordinates taken modulo the extent
// by the issuing thread. A box whose rows cross the domain's y edge starts at
// row -1 or ends at row ny: the TMA unit fills the rows outside the tensor
// with zeros, and the threads that need those (wrapped) rows read them from
// global memory instead. Every box lands at a 128-byte-aligned shared-memory
// address, as bulk tensor copies require.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the driver function is fetched at run time)

#include "pflb_common.cuh"

namespace pflb {

// The maps of one step: the g source array (MAIN: the tile's rows plus the
// two halo rows; SIDE: the 16-byte x-halo boxes of the same rows) and the f
// array (ALL: every slot of the tile's rows, even AA steps; MAIN, SIDE: one
// slot of the tile's rows and of its x halo, odd AA steps).
enum TmaMap : int { TM_G_MAIN = 0, TM_G_SIDE, TM_F_ALL, TM_F_MAIN, TM_F_SIDE, TM_COUNT };
struct TmaMaps {   // CUtensorMap carries its own (64-byte or wider) alignment
  CUtensorMap m[TM_COUNT];
};

// Bounded waits: a wait that has not seen its phase complete after this
// many polls gives up and reports PFLB_ETIMEOUT through the observables
// status (each poll may suspend the thread for a short, hardware-chosen time).
constexpr int kTmaWaitPolls = 1 << 22;
constexpr unsigned kStatusTimeout = 2u;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
// Make the initialised barriers visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Order this thread's earlier generic accesses of shared memory before the
// async-proxy writes of the copies it issues next.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait for phase `parity` of the barrier; false if the poll limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, int polls = kTmaWaitPolls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Bulk tensor copy of one box of a rank-5 map into shared memory, completing
// its bytes on the barrier (a CTA is its own cluster here: no multicast).
__device__ __forceinline__ void tma_load5(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          int c4, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__host__ __device__ constexpr int align128(int b) { return (b + 127) / 128 * 128; }

// Byte layout of one TMA stage (every box at a 128-byte-aligned offset), for
// a tile of 32 x TB cells, QGS staged g slots, QF f slots, NSX velocities
// with e_x != 0, element size ES, PAR the AA parity:
//   g main [TB + 2 rows][QGS][32], g left / right [TB + 2][QGS][SL];
//   f (even) [TB][QF][32]; f (odd) main [QF][TB][32], side [NSX] slots of
//   F_SIDE_STRIDE bytes, each [TB][SL].
template <int TB, int QGS, int QF, int NSX, int ES, int PAR>
struct TmaStage {
  static constexpr int SL = 16 / ES;
  static constexpr int G_MAIN = 0;
  static constexpr int G_MAIN_B = (TB + 2) * QGS * 32 * ES;
  static constexpr int G_SIDE_B = (TB + 2) * QGS * SL * ES;
  static constexpr int G_LEFT = align128(G_MAIN_B);
  static constexpr int G_RIGHT = G_LEFT + align128(G_SIDE_B);
  static constexpr int F = G_RIGHT + align128(G_SIDE_B);
  static constexpr int F_MAIN_B = TB * QF * 32 * ES;
  static constexpr int F_SIDE = F + align128(F_MAIN_B);
  static constexpr int F_SIDE_BOX = TB * SL * ES;
  static constexpr int F_SIDE_STRIDE = align128(F_SIDE_BOX);
  static constexpr int F_SIDE_B = PAR == 1 ? NSX * F_SIDE_STRIDE : 0;
  static constexpr int BYTES = align128(F_SIDE + F_SIDE_B);
  // bytes the copies of one stage complete on its barrier (whole boxes,
  // zero-filled rows included)
  static constexpr unsigned TX =
      (unsigned)(G_MAIN_B + 2 * G_SIDE_B + F_MAIN_B + (PAR == 1 ? NSX * F_SIDE_BOX : 0));
  // every box starts 128-byte aligned (checked where the layout is used)
  static constexpr bool ALIGNED = G_MAIN_B % 128 == 0 && F_MAIN_B % 128 == 0 && (PAR == 0 || (TB * 32 * ES) % 128 == 0);
};

}  // namespace pflb
