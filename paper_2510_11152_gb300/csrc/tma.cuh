// tma.cuh -- tensor-memory-accelerator (TMA) tile loads into shared memory, completed on mbarriers
// whose waits are bounded in time.
//
// A tile of a global field is described on the host by a tensor map (cuTensorMapEncodeTiled through
// the runtime's driver entry point, so the library does not link libcuda) and loaded by one thread
// with cp.async.bulk.tensor into shared memory; the copy signals an mbarrier in shared memory with the
// number of bytes it wrote, and the threads that read the tile wait on that barrier's phase. A wait
// gives up after a deadline on the global nanosecond timer instead of spinning forever: the caller
// then records an error the host turns into FAS_ETIMEOUT. The innermost tile coordinate times the
// element size must be a multiple of 16 bytes; out-of-range elements of a load read as zero.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fasmg {

// Deadline of a bounded mbarrier wait: far above any tile load's latency (microseconds).
constexpr unsigned long long kTmaWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisations (generic proxy) visible to the copies (async proxy).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier shared-memory accesses before later copies into shared memory.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One arrival on the barrier, announcing `bytes` bytes the copies will deliver in this phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Tile load of a rank-3 tensor map at element coordinates (x, y, z) into dst (128-byte aligned),
// completing `bytes` on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of the given parity to complete; false when the deadline passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// Bulk reduction of `bytes` bytes (a multiple of 16; both addresses 16-byte aligned) of float64 values
// from shared memory into global memory: dst[i] += src[i], each sum rounded to nearest in the L2. The
// copy joins this thread's current bulk group (commit with bulk_commit).
__device__ __forceinline__ void bulk_reduce_add_f64(double* dst, const double* src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's bulk groups still read their shared-memory source.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Wait until every bulk group of this thread has completed (its writes are performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Host: a rank-3 tensor map of a dense float64 or float32 field (elem_bytes 8 or 4, x fastest) with
// box (bx, by, bz); out-of-range elements of a tile load read as zero. Returns cudaErrorInvalidValue
// when the driver rejects the description (alignment, sizes), cudaErrorNotSupported without the
// driver's entry point.
cudaError_t tensor_map_3d(CUtensorMap* map, const void* base, int elem_bytes, int nx, int ny, int nz, int bx, int by,
                          int bz);

}  // namespace fasmg
