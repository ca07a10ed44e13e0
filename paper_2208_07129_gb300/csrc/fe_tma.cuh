// Inline-PTX helpers for the Tensor Memory Accelerator: tiled bulk loads of
// a box of a tensor map into shared memory (completion counted in bytes on
// an mbarrier) and tiled bulk reduce-add stores of a shared-memory box into
// global memory (completion tracked in per-thread bulk groups).
//
// A box is described by the tensor map (created on the host with
// cuTensorMapEncodeTiled and passed as a __grid_constant__ kernel parameter);
// the shared-memory image of a box is dense, innermost dimension first.
// Elements of the box outside the tensor are read as zero by a load and
// skipped by a reduce.  The innermost coordinate times the element size must
// be a multiple of 16 bytes.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "fe_umma.cuh"

namespace fe {

// The mbarrier's current phase completes once `bytes` more bytes have arrived
// (and the one pending arrival, this one, has been made).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// Box at coordinates (c0, c1, c2, c3) of a 4-D tensor map -> dst.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(mbar))
      : "memory");
}

// Global box at (c0, c1, c2, c3) += src, element by element (the element type
// and rounding are those of the tensor map's type).
__device__ __forceinline__ void tma_reduce_add_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                                  int c3) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}

// Contiguous bytes src (global, 16-byte aligned, a multiple of 16 bytes) ->
// dst (shared), completion counted on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Every bulk group of this thread has finished reading its shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Every bulk group of this thread has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace fe
