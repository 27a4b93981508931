// Staged persistent variant of the two-vector hypercube passes (FE, R1, R2, R0; complex64).
//
// The per-tile kernels load a tile, transpose and rotate it, and store it; with 128 registers two
// CTAs share an SM and a tile's loads, its shared-memory transposes and its stores largely follow
// one another. Here each CTA walks tiles blockIdx.x, + gridDim.x, ... and, while it works on one,
// the Tensor Memory Accelerator lands the next tile's psi and lambda densely in a shared-memory
// stage (cp.async.bulk.tensor, completion counted on one mbarrier) and prefetches that tile's
// quality block into L2. Layout: 64 KiB stage (psi then lambda, slot = tile index) + one padded
// transpose buffer (the two vectors are transposed one after the other), so two CTAs fit an SM.
//
// The tile geometry becomes a 5-d tensor over the state vector: d0 = the low chunk bits (at most 8),
// d1 = chunk bits 8..s-1 (s > 8 only), d2 = the non-tile bits between the chunk and the high tile
// bits, d3 = the high tile bits, d4 = the non-tile bits above them. A tile is the box
// {d0, d1, 1, d3, 1} at coordinates (0, 0, mid, 0, top), where (mid, top) are the tile number's
// low and high bits; the box lands in shared memory with its elements in tile-index order.
//
// Every mbarrier wait is bounded (2 s of the global timer): on expiry the kernel sets the caller's
// error flag to 1, waits (again bounded) for its own copies in flight and returns; the host turns a
// set flag into QVS_ETIMEOUT. A stage that is not 128-byte aligned sets the flag to 2 before any copy.
#pragma once

#include <cuda.h>

#include "hc_pass.cuh"

namespace qvs {
namespace hc {

struct alignas(64) StageMaps {
  CUtensorMap psi;    // tile box over the pass's psi input
  CUtensorMap lam;    // over its lambda input (two-vector inputs only)
  CUtensorMap q;      // over q (4-byte elements) for the L2 prefetch
  int two;            // stage lambda as well
  int qpf;            // prefetch the quality block
  int mid_bits;       // width of the tile number's low field (d2)
  int top_bits;       // width of its high field (d4)
  int* err;           // set to 1 when a wait expires
};

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // a wait gives up after 2 s (global timer)
constexpr uint32_t kStageAlign = 1024;             // alignment of the stage in shared memory

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's (and, after a barrier, the CTA's) generic-proxy shared-memory accesses
// before the async proxy's next writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Poll the phase; a poll may suspend the thread for a system-dependent time, so the bound is in
// wall time, read from the global nanosecond timer.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c2, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %3, %4, %3, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(0), "r"(c2), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_l2_5d(const CUtensorMap* map, int c2, int c4) {
  asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %1, %2, %1, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(0), "r"(c2), "r"(c4)
               : "memory");
}

template <int SHAPE, int TH>
__global__ void __launch_bounds__(NT, 2)
staged_kernel(const __grid_constant__ PassArgs<float> a, const __grid_constant__ StageMaps m, uint32_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_fail;
  // the tensor copies land at 1024-byte boundaries: the dynamic region (which follows the static
  // shared variables) is over-allocated by kStageAlign bytes and the stage starts at the first
  // aligned address in it
  const uint32_t pad = (kStageAlign - (smem_u32(smem_raw) & (kStageAlign - 1u))) & (kStageAlign - 1u);
  float2* stage = reinterpret_cast<float2*>(smem_raw + pad);
  unsigned char* tsm = smem_raw + pad + (size_t)(m.two ? 2 : 1) * TILE * sizeof(float2);
  const int tid = threadIdx.x;
  if (smem_u32(stage) & 127u) {   // never expected: report instead of issuing a misaligned copy
    if (tid == 0) atomicExch(m.err, 2);
    return;
  }
  const uint32_t bytes = (uint32_t)((m.two ? 2 : 1) * TILE * sizeof(float2));
  const uint32_t mid_mask = (1u << m.mid_bits) - 1u;
  const uint32_t top_mask = (1u << m.top_bits) - 1u;
  auto issue = [&](uint32_t tile) {   // thread 0
    const int mid = (int)(tile & mid_mask), top = (int)(tile >> m.mid_bits);
    mbar_expect_tx(&bar, bytes);
    tma_load_5d(stage, &m.psi, &bar, mid, top);
    if (m.two) tma_load_5d(stage + TILE, &m.lam, &bar, mid, top);
    if (m.qpf) {   // the flipped frame reads q at complemented indices: the complemented tile
      const int qm = a.qx ? (int)(~(uint32_t)mid & mid_mask) : mid;
      const int qt = a.qx ? (int)(~(uint32_t)top & top_mask) : top;
      tma_prefetch_l2_5d(&m.q, qm, qt);
    }
  };
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  __syncthreads();
  uint32_t t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t);
  uint32_t parity = 0;
  for (; t < ntiles; t += gridDim.x) {
    if (!mbar_wait_bounded(&bar, parity)) s_fail = 1;
    __syncthreads();
    if (s_fail) {   // every thread sees it after the barrier: stop, after the copies in flight
      if (tid == 0) {
        atomicExch(m.err, 1);
        (void)mbar_wait_bounded(&bar, parity);
      }
      return;
    }
    parity ^= 1u;
    const uint32_t next = t + gridDim.x;
    auto consumed = [&]() {   // every thread has read the stage: land the next tile there
      if (tid == 0 && next < ntiles) {
        fence_proxy_async_smem();
        issue(next);
      }
    };
    run_pass<float, SHAPE, TH, false, true>(a, t, ntiles, tsm, stage, consumed);
    __syncthreads();   // the partial-sum scratch and the transpose buffer are reused by the next tile
  }
}

// Launch one staged pass over ntiles tiles with grid persistent CTAs (stream-ordered).
template <int TH>
int launch_staged(int shape, const PassArgs<float>& a, const StageMaps& m, uint32_t ntiles, uint32_t grid,
                  cudaStream_t st) {
  const size_t sm =
      kStageAlign + (size_t)(m.two ? 2 : 1) * TILE * sizeof(float2) + (size_t)SM_SLOTS * sizeof(float2);
  auto go = [&](auto kern, std::atomic<uint64_t>& configured) -> int {
    QVS_TRY(smem_limit_once(reinterpret_cast<const void*>(kern), configured, (int)sm));
    kern<<<grid, NT, sm, st>>>(a, m, ntiles);
    QVS_CUDA_TRY(cudaGetLastError());
    return QVS_OK;
  };
  static std::atomic<uint64_t> c_fe{0}, c_r1{0}, c_r2{0}, c_r0{0};   // per instantiation: devices set
  switch (shape) {
    case FE: return go(staged_kernel<FE, TH>, c_fe);
    case R1: return go(staged_kernel<R1, TH>, c_r1);
    case R2: return go(staged_kernel<R2, TH>, c_r2);
    case R0: return go(staged_kernel<R0, TH>, c_r0);
  }
  return QVS_EINVAL;
}

#define QVS_HC_STAGED_EXTERN(K) \
  extern template int launch_staged<K>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);
#ifndef QVS_HC_PASS_TU
QVS_HC_C64_THRESHOLDS(QVS_HC_STAGED_EXTERN)
#endif
#undef QVS_HC_STAGED_EXTERN

}  // namespace hc
}  // namespace qvs
