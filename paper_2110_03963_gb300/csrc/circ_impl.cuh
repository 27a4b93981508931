// Kernels and host driver of the circulant (QWOA) path, instantiated per transform size by the
// circ_n*.cu translation units (compiled in parallel).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <vector>

#include "fft_kernels.cuh"
#include "qvs_internal.h"

namespace qvs {
namespace cf {

using GRow = Geo<0, 4, 5, 5>;

enum ColMode : int { CF = 0, CM = 1, CL = 2, CV = 3, RCM = 4, RCF = 5 };
enum RowMode : int { RF = 0, RR = 1 };

struct CircArgs {
  int n;                       // log2 N
  const float2* in;            // pass input (natural positions)
  float2* out;                 // pass output
  const float2* psi0;          // explicit initial state (natural, normal form) or NULL
  float2* priv_out;            // stored vector for the adjoint (thread-major), or NULL
  const float2* priv_in;       // stored vector read by the adjoint (thread-major)
  const float* qT;             // q in column-pass thread-major order
  const float2* lamT;          // eigenvalues (hi, lo) in row-spectral thread-major order
  float ph_hi, ph_lo;          // phase: gamma / 2pi (float-float)
  float ph2_hi, ph2_lo;        // reverse passes: the phase to re-apply to the stored psi
  float ev_hi, ev_lo;          // eigenphase: t / 2pi (float-float)
  float init_amp;
  double* part;                // partial rows [row * gridDim.x + blockIdx.x]
  int row_a, row_b;
  int tma_store;               // 1: the layout-0 result leaves through one tensor store (out_map)
  int pf_ahead;                // > 0: prefetch into L2 the inputs of tile blockIdx.x + pf_ahead
  int pf_map;                  // 1: in_map describes `in` (column passes' state prefetch and load)
  int tma_load;                // 1: the layout-0 input arrives through one tensor load (in_map)
  int* err;                    // set to 1 when a tile copy did not arrive within the wait limit
  CUtensorMap out_map;         // 4-d view of `out` matching the shared-memory box (see box_word)
  CUtensorMap in_map;          // the same view of `in`
};

// ---------------------------------------------------------------- tensor copies of a column tile
//
// The column tile of Geo<2, 4, 4, 4> (4 adjacent columns x 4096 rows of a 2^26 state) is loaded by
// one tensor copy into the transpose buffer and stored by one from it, instead of 32 loads and 32
// stores per thread, whose burst at the end of every tile kept the LSU queue full (lg throttle was
// the top stall). The box is {4 columns, 4 (row bits 4-5), 16 (row bits 0-3), 64 (row bits 6-11)}:
// in shared memory a tile index lands at box_word, and a half-warp of layout 0 (lanes = tile bits
// 0, 1, 6, 7) reads or writes 16 consecutive 8-byte words, one per bank pair. The load completes on
// an mbarrier before the first transpose; the store reads the buffer after the last transpose, and
// the CTA waits only until the copy has read it.
template <class G>
struct TmaTile {
  static constexpr bool ok = false;
};
template <>
struct TmaTile<Geo<2, 4, 4, 4>> {
  static constexpr bool ok = true;
};
__host__ __device__ constexpr int box_word(int j) {
  return (j & 3) | (((j >> 6) & 3) << 2) | (((j >> 2) & 15) << 4) | ((j >> 8) << 8);
}
constexpr int kBoxAlign = 1024;   // the dynamic shared region is realigned to this (tensor copies: 128 B)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// L2 prefetch hints for the tile one wave later (one CTA per SM: tile blockIdx.x + SMs starts when
// this one ends), so its state loads find the data in L2. Only the state tile is prefetched:
// adding q, the eigenvalue table and the stored vectors made the passes slower overall (QWOA
// N=2^26: 15.3 ms without prefetch, 15.9 with all inputs, 15.0 with the state only).
// Contiguous blocks go in 32 KiB requests (16-byte aligned, multiples of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (uint32_t o = 0; o < bytes; o += 32768u) {
    const uint32_t n = bytes - o < 32768u ? bytes - o : 32768u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(n) : "memory");
  }
}
__device__ __forceinline__ void prefetch_l2_box(const CUtensorMap* m, int c0) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %2, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(m)),
               "r"(c0), "r"(0)
               : "memory");
}

// Tile loads through the tensor engine complete on an mbarrier. Every wait is bounded by 2 s of the
// global timer: on expiry the CTA sets the caller's error flag, waits (again bounded) for its own
// copy in flight and returns, and the host reports QVS_ETIMEOUT.
constexpr uint64_t kCopyWaitNs = 2000000000ull;
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_done(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_done(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_done(bar, parity)) return true;
    if (global_ns() - t0 > kCopyWaitNs) return false;
  }
}

// Thread-major private arrays (q in column-pass order, the stored vectors, the eigenvalue table):
// only these kernels read them, so they are interleaved by register pairs: registers 2m and 2m+1 of
// a thread sit side by side (one float4 of a complex array, one float2 of q), so one access serves
// two registers and a warp's access still covers consecutive bytes.
__device__ __forceinline__ size_t pair_idx(uint32_t blk, int m, int tid) {   // units of the pair
  return ((size_t)blk * (R / 2) + m) * NT + tid;
}
template <int C>
__device__ __forceinline__ float2 half4(const float4& x) {
  if constexpr (C == 0) return make_float2(x.x, x.y);
  else return make_float2(x.z, x.w);
}

// Compiler fence after every 8th register of a per-register loop: the loads of the next group are
// not hoisted above it, so at most 8 registers' side-vector loads (stored psi, q) are in flight at
// once instead of all 32 competing with the 64 state registers for the 128 a thread has.
template <int r, int GROUP = 8>
__device__ __forceinline__ void group_fence() {
  if constexpr ((r & (GROUP - 1)) == GROUP - 1) asm volatile("" ::: "memory");
}

// fractional turns of x * y for float-float x and y (|x y| well below 2^24)
__device__ __forceinline__ float ff_turns(float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  const float e = fmaf(xh, yh, -p) + fmaf(xh, yl, xl * yh);
  return (p - rintf(p)) + e;
}

// block sum (lanes in fp32, warps and CTAs in fp64, fixed order)
__device__ __forceinline__ void block_store2(float a, float b, double scale, double* part, int ra, int rb) {
  __shared__ double red[2][NT / 32];
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = scale * (double)a;
    red[1][tid >> 5] = scale * (double)b;
  }
  __syncthreads();
  if (tid < 2) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[tid][w];
    const int row = tid == 0 ? ra : rb;
    if (row >= 0) part[(size_t)row * gridDim.x + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------- column pass

template <class G, int MODE>
__global__ void __launch_bounds__(NT, 1) col_kernel(const __grid_constant__ CircArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the region is over-allocated by kBoxAlign bytes; the buffers start at the first aligned address
  const uint32_t pad = (kBoxAlign - (smem_addr(smem_raw) & (kBoxAlign - 1u))) & (kBoxAlign - 1u);
  float2* sm = reinterpret_cast<float2*>(smem_raw + pad);
  const uint32_t blk = blockIdx.x;
  if constexpr (TmaTile<G>::ok) {
    if (a.pf_ahead > 0 && threadIdx.x == 0 && blk + (uint32_t)a.pf_ahead < gridDim.x) {
      const uint32_t nb = blk + (uint32_t)a.pf_ahead;
      if (MODE != CF && a.pf_map) prefetch_l2_box(&a.in_map, (int)(4u * nb));
    }
  }
  constexpr int CB = G::dstart(0);
  const int tid = threadIdx.x;
  // global index of tile index j
  auto gidx = [&](int j) -> uint32_t {
    return (uint32_t)(j & ((1 << CB) - 1)) | (blk << CB) | ((uint32_t)(j >> CB) << TB);
  };
  // four-step twiddle omega_N^(+-j_low * k_col) on layout 0 (column-spectral positions). The
  // position-to-frequency map is a bit permutation, so it splits into a per-thread part and a
  // compile-time per-register part. The exponent is exact in 32-bit integers; shifted to the top of
  // a 32-bit word it is the turn e / N as a fixed-point fraction whose signed value is already
  // reduced to [-1/2, 1/2), so one hardware sine/cosine of its float conversion (relative error
  // 2^-24 of an angle of at most pi) replaces four table reads and three complex products.
  auto gtw = [&](float2(&v)[R], bool conj) {
    const int jt = G::template jthr<0>(tid_fresh());
    const uint32_t jlt = (uint32_t)(jt & ((1 << CB) - 1)) | (blk << CB);
    const uint32_t kt = (uint32_t)G::freq(jt >> CB);
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      constexpr int jr = G::jreg(0, r);
      constexpr uint32_t jlr = (uint32_t)(jr & ((1 << CB) - 1));
      constexpr uint32_t kr = (uint32_t)G::freq(jr >> CB);
      // e / N as a 32-bit fixed-point fraction; its signed value is the reduced turn in [-1/2, 1/2)
      const int32_t es = (int32_t)(((jlt | jlr) * (kt | kr)) << (32 - a.n));
      float sn, cs;
      __sincosf((float)es * 1.46291807926715968e-09f, &sn, &cs);   // 2 pi / 2^32
      const float2 w = make_float2(cs, -sn);
      v[r] = conj ? cmulc(v[r], w) : cmul(v[r], w);
    });
  };
  // layout-0 input; false when the tensor copy did not arrive (the error flag is then set)
  auto gload0 = [&](float2(&v)[R], const float2* src) -> bool {
    const int jt = G::template jthr<0>(tid_fresh());
    if constexpr (TmaTile<G>::ok) {
      // a.tma_load is uniform; the alignment test never fails (the region is realigned above)
      if (a.tma_load && (smem_addr(sm) & 127u) == 0u) {
        __shared__ __align__(8) uint64_t bar;
        if (threadIdx.x == 0) {
          asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
          asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)),
                       "r"((uint32_t)(TILE * sizeof(float2)))
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %3, %3}], [%4];" ::"r"(smem_addr(sm)),
              "l"(reinterpret_cast<uint64_t>(&a.in_map)), "r"((int)(4u * blk)), "r"(0), "r"(smem_addr(&bar))
              : "memory");
        }
        const bool failed = __syncthreads_or(mbar_wait_bounded(&bar, 0) ? 0 : 1) != 0;
        if (failed) {   // never expected: report, let the copy in flight finish, stop
          if (threadIdx.x == 0) {
            atomicExch(a.err, 1);
            (void)mbar_wait_bounded(&bar, 0);
          }
          return false;
        }
        const int bw = box_word(jt);
        static_for<R>([&](auto ri) {
          constexpr int r = decltype(ri)::value;
          constexpr int o = box_word(G::jreg(0, r));
          v[r] = sm[bw + o];
        });
        __syncthreads();   // the transposes reuse the buffer
        return true;
      }
    }
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      v[r] = __ldcs(src + gidx(jt | G::jreg(0, r)));
    });
    return true;
  };
  auto gstore0 = [&](const float2(&v)[R], float2* dst) {
    const int jt = G::template jthr<0>(tid_fresh());
    if constexpr (TmaTile<G>::ok) {
      // a.tma_store is uniform; the alignment test never fails (the region is realigned above)
      if (a.tma_store && (smem_addr(sm) & 127u) == 0u) {
        const int bw = box_word(jt);
        static_for<R>([&](auto ri) {
          constexpr int r = decltype(ri)::value;
          constexpr int o = box_word(G::jreg(0, r));
          sm[bw + o] = v[r];
        });
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the copy engine
        __syncthreads();
        if (threadIdx.x == 0) {
          asm volatile(
              "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %2, %2}], [%3];" ::"l"(
                  reinterpret_cast<uint64_t>(&a.out_map)),
              "r"((int)(4u * blk)), "r"(0), "r"(smem_addr(sm))
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        return;
      }
    }
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      __stcs(dst + gidx(jt | G::jreg(0, r)), v[r]);
    });
  };
  // exp(-i 2pi turns(q * g)) for the amplitude in register r of layout 2 (natural positions)
  auto phase_cs = [&](int r, float q, float gh, float gl, float& c, float& s) {
    __sincosf(6.28318530717958647692f * ff_turns(gh, gl, q, 0.0f), &s, &c);
  };
  // The side vectors never alias the stored-vector outputs: restrict-qualified copies let their
  // loads be issued ahead of the stores instead of one latency at a time.
  const float2* __restrict__ qT2 = reinterpret_cast<const float2*>(a.qT);
  // q of register r: one 8-byte load per pair of registers (r a compile-time index, loops unrolled;
  // 16-byte quads made the adjoint pass spill)
  float2 q2;
  auto qat = [&](auto ri) {
    constexpr int r = decltype(ri)::value;
    if constexpr ((r & 1) == 0) q2 = __ldcs(qT2 + pair_idx(blk, r >> 1, tid_fresh()));
    return (r & 1) ? q2.y : q2.x;
  };
  const float invL = 1.0f / (float)G::L;

  float2 v[R];
  if constexpr (MODE == CF) {
    const int jt = G::template jthr<2>(tid);
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      float2 x = a.psi0 ? __ldg(a.psi0 + gidx(jt | G::jreg(2, r))) : make_float2(a.init_amp, 0.0f);
      float c, s;
      phase_cs(r, qat(ri), a.ph_hi, a.ph_lo, c, s);
      v[r] = make_float2(c * x.x + s * x.y, c * x.y - s * x.x);
    });
    tile_fwd<G>(v, sm, tid);
    gtw(v, false);
    gstore0(v, a.out);
  } else {
    if (!gload0(v, a.in)) return;
    gtw(v, true);
    tile_inv<G>(v, sm, tid);
    // block barriers around the per-register step separate the inverse and forward transforms in
    // the schedule: fewer values held across them, fewer register spills (ptxas -v: RCM 820 -> 492,
    // CL 524 -> 376 bytes per thread at n = 26)
    __syncthreads();
    if constexpr (MODE == CM) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = make_float2(v[r].x * invL, v[r].y * invL);
      float4* __restrict__ po = reinterpret_cast<float4*>(a.priv_out);
      if (po) {   // stored for the adjoint
#pragma unroll
        for (int m = 0; m < R / 2; ++m)
          __stcs(po + pair_idx(blk, m, tid), make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y));
      }
      static_for<R>([&](auto ri) {
        constexpr int r = decltype(ri)::value;
        const float2 x = v[r];
        float c, s;
        phase_cs(r, qat(ri), a.ph_hi, a.ph_lo, c, s);
        v[r] = make_float2(c * x.x + s * x.y, c * x.y - s * x.x);
      });
      tile_fwd<G>(v, sm, tid);
      gtw(v, false);
      gstore0(v, a.out);
    } else if constexpr (MODE == CL || MODE == CV) {
      float e = 0.0f;
      if constexpr (MODE == CV) {
        const int jt = G::template jthr<2>(tid);
        static_for<R>([&](auto ri) {
          constexpr int r = decltype(ri)::value;
          const float2 x = make_float2(v[r].x * invL, v[r].y * invL);
          e += qat(ri) * (x.x * x.x + x.y * x.y);
          __stcs(a.out + gidx(jt | G::jreg(2, r)), x);
        });
      } else {
        static_for<R>([&](auto ri) {
          constexpr int r = decltype(ri)::value;
          const float q = qat(ri);
          const float2 x = make_float2(v[r].x * invL, v[r].y * invL);
          e += q * (x.x * x.x + x.y * x.y);
          v[r] = make_float2(q * x.x, q * x.y);
          group_fence<r>();
        });
        // the objective is reduced before the forward transform (its barrier also separates the
        // two in the schedule), so neither the sum nor its row and output pointers stay live
        // across the transform
        block_store2(e, 0.0f, 1.0, a.part, a.row_a, -1);
        tile_fwd<G>(v, sm, tid);
        gtw(v, false);
        gstore0(v, a.out);
        return;
      }
      block_store2(e, 0.0f, 1.0, a.part, a.row_a, -1);
    } else {   // RCM, RCF: v = lambda' after the adjoint mixer; gamma gradient, then phase^dagger
      const float4* __restrict__ pin = reinterpret_cast<const float4*>(a.priv_in);
      float g = 0.0f;
      const int jt = G::template jthr<2>(tid);
      float4 ps4;
      static_for<R>([&](auto ri) {
        constexpr int r = decltype(ri)::value;
        float2 ps;
        if constexpr (MODE == RCM) {
          if constexpr ((r & 1) == 0) ps4 = __ldcs(pin + pair_idx(blk, r >> 1, tid));
          ps = half4<r & 1>(ps4);
        } else {
          ps = a.psi0 ? __ldg(a.psi0 + gidx(jt | G::jreg(2, r))) : make_float2(a.init_amp, 0.0f);
        }
        const float q = qat(ri);
        float c, s;
        phase_cs(r, q, a.ph2_hi, a.ph2_lo, c, s);
        const float2 phi = make_float2(c * ps.x + s * ps.y, c * ps.y - s * ps.x);   // P psi
        const float2 l = make_float2(v[r].x * invL, v[r].y * invL);
        g += q * (l.x * phi.y - l.y * phi.x);
        v[r] = make_float2(c * l.x - s * l.y, c * l.y + s * l.x);                   // P^dagger lambda'
        group_fence<r>();
      });
      // gamma-gradient row reduced before the forward transform (see the last pass above)
      block_store2(g, 0.0f, 2.0, a.part, a.row_a, -1);
      if constexpr (MODE == RCM) {
        tile_fwd<G>(v, sm, tid);
        gtw(v, false);
        gstore0(v, a.out);
      }
    }
  }
}

// ---------------------------------------------------------------- row pass

template <int MODE>
__global__ void __launch_bounds__(NT, 1) row_kernel(const __grid_constant__ CircArgs a) {
  using G = GRow;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  const uint32_t blk = blockIdx.x;
  if (a.pf_ahead > 0 && tid == 0 && blk + (uint32_t)a.pf_ahead < gridDim.x) {
    const uint32_t nb = blk + (uint32_t)a.pf_ahead;
    prefetch_l2(a.in + ((size_t)nb << TB), (uint32_t)(TILE * sizeof(float2)));
  }
  const float2* src = a.in + ((size_t)blk << TB);
  float2* dst = a.out + ((size_t)blk << TB);
  float2 v[R];
  {
    const int jt = G::template jthr<2>(tid);
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      v[r] = __ldcs(src + (jt | G::jreg(2, r)));
    });
  }
  tile_fwd<G>(v, sm, tid);
  // restrict-qualified: the table and stored-vector loads are issued ahead of the stores
  const float4* __restrict__ lamT = reinterpret_cast<const float4*>(a.lamT);
  const float4* __restrict__ pin = reinterpret_cast<const float4*>(a.priv_in);
  float4* __restrict__ po = reinterpret_cast<float4*>(a.priv_out);
  float acc = 0.0f;
  float4 lam4, x4;
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    if constexpr ((r & 1) == 0) lam4 = __ldcs(lamT + pair_idx(blk, r >> 1, tid));
    const float2 lam = half4<r & 1>(lam4);
    float s, c;
    __sincosf(6.28318530717958647692f * ff_turns(lam.x, lam.y, a.ev_hi, a.ev_lo), &s, &c);
    if constexpr (MODE == RF) {
      v[r] = make_float2(c * v[r].x + s * v[r].y, c * v[r].y - s * v[r].x);   // exp(-i t lambda)
    } else {
      if constexpr ((r & 1) == 0) x4 = __ldcs(pin + pair_idx(blk, r >> 1, tid));
      const float2 x = half4<r & 1>(x4);
      acc += lam.x * (v[r].x * x.y - v[r].y * x.x);
      v[r] = make_float2(c * v[r].x - s * v[r].y, c * v[r].y + s * v[r].x);   // exp(+i t lambda)
    }
  });
  if constexpr (MODE == RF) {
    if (po) {
#pragma unroll
      for (int m = 0; m < R / 2; ++m)
        __stcs(po + pair_idx(blk, m, tid), make_float4(v[2 * m].x, v[2 * m].y, v[2 * m + 1].x, v[2 * m + 1].y));
    }
  }
  tile_inv<G>(v, sm, tid);
  const float invL = 1.0f / (float)TILE;
  {
    const int jt = G::template jthr<2>(tid);
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      __stcs(dst + (jt | G::jreg(2, r)), make_float2(v[r].x * invL, v[r].y * invL));
    });
  }
  if constexpr (MODE == RR) {
    block_store2(acc, 0.0f, 2.0 / (double)(1ull << a.n), a.part, a.row_a, -1);
  }
}

// ---------------------------------------------------------------- tables

// eigenvalues lambda_k = sum_s w_s (2 cos(2 pi s k / N), or (-1)^k for s = N/2), fp64, stored as
// float-float in the row-spectral thread-major order
template <class GC>
__global__ void __launch_bounds__(NT) lam_kernel(int n, int nofs, const int64_t* __restrict__ ofs,
                                                 const double* __restrict__ w, float2* lamT) {
  using G = GRow;
  const int tid = threadIdx.x;
  const uint32_t blk = blockIdx.x;
  const uint64_t N = 1ull << n;
  const int B = n - TB;
  const uint64_t kcol = (uint64_t)GC::freq((int)blk);
  const int jt = G::template jthr<0>(tid);
  for (int r = 0; r < R; ++r) {
    const int j = jt | G::jreg(0, r);
    const uint64_t k = kcol + ((uint64_t)G::freq(j) << B);
    double lam = 0.0;
    for (int i = 0; i < nofs; ++i) {
      const uint64_t s = (uint64_t)ofs[i];
      if (2 * s == N) lam += w[i] * ((k & 1) ? -1.0 : 1.0);
      else lam += 2.0 * w[i] * cospi(2.0 * (double)((s * k) & (N - 1)) / (double)N);
    }
    const float hi = (float)lam;
    lamT[pair_idx(blk, r >> 1, tid) * 2 + (r & 1)] = make_float2(hi, (float)(lam - (double)hi));
  }
}

template <class GC>
__global__ void __launch_bounds__(NT) qperm_kernel(const float* __restrict__ q, float* __restrict__ qT) {
  constexpr int CB = GC::dstart(0);
  const int tid = threadIdx.x;
  const uint32_t blk = blockIdx.x;
  const int jt = GC::template jthr<2>(tid);
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    const int j = jt | GC::jreg(2, r);
    const uint32_t g = (uint32_t)(j & ((1 << CB) - 1)) | (blk << CB) | ((uint32_t)(j >> CB) << TB);
    qT[pair_idx(blk, r >> 1, tid) * 2 + (r & 1)] = q[g];
  });
}

// ---------------------------------------------------------------- host driver

template <class GC>
struct Driver {
  static int set_mixer(qvs_ctx* h, const int64_t* ofs_dev, const double* w_dev, int nofs) {
    const uint32_t grid = (uint32_t)(h->dim >> TB);
    QVS_TRY(h->circ.lam.ensure(sizeof(float2) * (size_t)h->dim));
    lam_kernel<GC><<<grid, NT, 0, h->stream>>>(h->n, nofs, ofs_dev, w_dev, h->circ.lam.as<float2>());
    QVS_CUDA_TRY(cudaGetLastError());
    return QVS_OK;
  }

  static int run(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E,
                 double* dg, double* dt) {
    const int64_t dim = h->dim;
    const uint32_t grid = (uint32_t)(dim >> TB);
    const size_t vb = sizeof(float2) * (size_t)dim;
    const size_t smem = sizeof(float2) * SM_SLOTS + kBoxAlign;
    // q in column-pass order (rebuilt when q or the mixer changed)
    if (!h->circ.qT_valid) {
      QVS_TRY(h->circ.qT.ensure(sizeof(float) * (size_t)dim));
      qperm_kernel<GC><<<grid, NT, 0, h->stream>>>(h->q.as<float>(), h->circ.qT.as<float>());
      QVS_CUDA_TRY(cudaGetLastError());
      h->circ.qT_valid = true;
    }
    QVS_TRY(h->psi.ensure(vb));
    if (grad) {
      QVS_TRY(h->lam.ensure(vb));
      QVS_TRY(h->ckpt.ensure(vb * (size_t)(2 * p)));   // psi_1..psi_{p-1}, X_1..X_p
    }
    const int nslots = 1 + 2 * p;
    const int nrows = 2 * p + 1;   // 0: E; 1..p: dgamma_k; p+1..2p: dt_k
    QVS_TRY(h->flags.ensure(16));
    QVS_CUDA_TRY(cudaMemsetAsync(h->flags.ptr, 0, 16, h->stream));
    QVS_TRY(h->part.ensure(sizeof(double) * (size_t)nrows * grid));
    QVS_TRY(h->res.ensure(sizeof(double) * nslots));
    QVS_TRY(h->rowmap.ensure(sizeof(int) * 3 * nslots));
    std::vector<int> rowmap(3 * (size_t)nslots, -1);
    for (int s = 0; s < (grad ? nslots : 1); ++s) rowmap[3 * s] = s;
    QVS_CUDA_TRY(cudaMemcpyAsync(h->rowmap.ptr, rowmap.data(), sizeof(int) * rowmap.size(),
                                 cudaMemcpyHostToDevice, h->stream));
    for (auto f : {col_kernel<GC, CF>, col_kernel<GC, CM>, col_kernel<GC, CL>, col_kernel<GC, CV>,
                   col_kernel<GC, RCM>, col_kernel<GC, RCF>})
      QVS_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (auto f : {row_kernel<RF>, row_kernel<RR>})
      QVS_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));

    float2* W = h->psi.as<float2>();
    float2* Lb = grad ? h->lam.as<float2>() : nullptr;
    float2* S = grad ? h->ckpt.as<float2>() : nullptr;             // psi_k, k = 1..p-1
    float2* X = grad ? S + (size_t)p * dim : nullptr;             // X_k, k = 1..p
    auto Sk = [&](int k) { return S + (size_t)(k - 1) * dim; };
    auto Xk = [&](int k) { return X + (size_t)(k - 1) * dim; };

    CircArgs base{};
    base.n = h->n;
    base.psi0 = h->have_psi0 ? h->psi0.as<float2>() : nullptr;
    base.qT = h->circ.qT.as<float>();
    base.lamT = h->circ.lam.as<float2>();
    base.init_amp = (float)(1.0 / sqrt((double)dim));
    base.part = h->part.as<double>();
    base.row_a = base.row_b = -1;
    base.err = h->flags.as<int>();
    auto ph = [&](CircArgs& a, int k) { turns_split(gammas[k], &a.ph_hi, &a.ph_lo); };
    auto ev = [&](CircArgs& a, int k) { turns_split(ts[k], &a.ev_hi, &a.ev_lo); };
    const double colb = 16.0 + 4.0, rowb = 16.0 + 8.0;   // bytes per amplitude (state r+w, q / lambda)
    // tensor maps of the two state buffers for the tensor-store epilogue (box_word's order: columns,
    // row bits 4-5, row bits 0-3, row bits 6-11); per-thread stores when the driver has no encoder
    // or rejects the view
    CUtensorMap map_w, map_l;
    bool tma_w = false, tma_l = false;
    if constexpr (TmaTile<GC>::ok) {
      auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(hc::tensor_map_encode_fn());
      auto encode = [&](CUtensorMap* m, void* ptr) -> bool {
        if (!enc || !ptr) return false;
        const cuuint64_t C = (cuuint64_t)dim >> GC::B;   // columns: the index bits below the transform
        cuuint64_t dims[4] = {C, 4, 16, 64};
        cuuint64_t strides[3] = {16 * C * 8, C * 8, 64 * C * 8};
        cuuint32_t box[4] = {4, 4, 16, 64};
        cuuint32_t es[4] = {1, 1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
      };
      tma_w = h->staged && encode(&map_w, W);
      tma_l = h->staged && encode(&map_l, Lb);
    }
    int64_t launches = 0;
    // prefetch distance: the tile one wave later (one CTA per SM)
    const int pf = TmaTile<GC>::ok && h->staged ? h->sms : 0;
    auto launch_col = [&](int mode, const CircArgs& a0, double bytes) -> int {
      CircArgs a = a0;
      if (a.out == W && tma_w) {
        a.tma_store = 1;
        a.out_map = map_w;
      } else if (a.out == Lb && a.out && tma_l) {
        a.tma_store = 1;
        a.out_map = map_l;
      }
      a.pf_ahead = pf;
      if (a.in == W && tma_w) {
        a.pf_map = 1;
        a.in_map = map_w;
      } else if (a.in == Lb && a.in && tma_l) {
        a.pf_map = 1;
        a.in_map = map_l;
      }
      a.tma_load = a.pf_map;
      cudaEvent_t e0;
      QVS_TRY(prof_begin(h, &e0));
      switch (mode) {
        case CF: col_kernel<GC, CF><<<grid, NT, smem, h->stream>>>(a); break;
        case CM: col_kernel<GC, CM><<<grid, NT, smem, h->stream>>>(a); break;
        case CL: col_kernel<GC, CL><<<grid, NT, smem, h->stream>>>(a); break;
        case CV: col_kernel<GC, CV><<<grid, NT, smem, h->stream>>>(a); break;
        case RCM: col_kernel<GC, RCM><<<grid, NT, smem, h->stream>>>(a); break;
        case RCF: col_kernel<GC, RCF><<<grid, NT, smem, h->stream>>>(a); break;
      }
      QVS_CUDA_TRY(cudaGetLastError());
      ++launches;
      static const char* names[] = {"circ_col_first", "circ_col_mid", "circ_col_last", "circ_col_last_evolve",
                                    "circ_col_adjoint", "circ_col_adjoint_first"};
      return prof_end(h, names[mode], bytes * (double)dim, e0);
    };
    auto launch_row = [&](int mode, const CircArgs& a0, double bytes) -> int {
      CircArgs a = a0;
      a.pf_ahead = pf;
      cudaEvent_t e0;
      QVS_TRY(prof_begin(h, &e0));
      if (mode == RF) row_kernel<RF><<<grid, NT, smem, h->stream>>>(a);
      else row_kernel<RR><<<grid, NT, smem, h->stream>>>(a);
      QVS_CUDA_TRY(cudaGetLastError());
      ++launches;
      return prof_end(h, mode == RF ? "circ_row" : "circ_row_adjoint", bytes * (double)dim, e0);
    };

    // forward: C_0, R_1, C_1, ..., R_p, C_p
    {
      CircArgs a = base;
      ph(a, 0);
      a.out = W;
      QVS_TRY(launch_col(CF, a, 12.0 + (base.psi0 ? 8.0 : 0.0)));
    }
    for (int k = 1; k <= p; ++k) {
      CircArgs r = base;
      ev(r, k - 1);
      r.in = W;
      r.out = W;
      r.priv_out = grad ? Xk(k) : nullptr;
      QVS_TRY(launch_row(RF, r, rowb + (grad ? 8.0 : 0.0)));
      CircArgs c = base;
      c.in = W;
      if (k < p) {
        ph(c, k);
        c.out = W;
        c.priv_out = grad ? Sk(k) : nullptr;
        QVS_TRY(launch_col(CM, c, colb + (grad ? 8.0 : 0.0)));
      } else if (grad) {
        c.out = Lb;
        c.row_a = 0;
        QVS_TRY(launch_col(CL, c, colb));
      } else {
        c.out = W;
        c.row_a = 0;
        QVS_TRY(launch_col(CV, c, colb));
      }
    }
    // adjoint: R_p^dag, C_{p-1}^dag, ..., R_1^dag, C_0^dag
    if (grad) {
      for (int k = p; k >= 1; --k) {
        CircArgs r = base;
        ev(r, k - 1);
        r.in = Lb;
        r.out = Lb;
        r.priv_in = Xk(k);
        r.row_a = 1 + p + (k - 1);
        QVS_TRY(launch_row(RR, r, rowb + 8.0));
        CircArgs c = base;
        c.in = Lb;
        c.out = Lb;
        turns_split(gammas[k - 1], &c.ph2_hi, &c.ph2_lo);
        c.row_a = 1 + (k - 1);
        if (k >= 2) {
          c.priv_in = Sk(k - 1);
          QVS_TRY(launch_col(RCM, c, colb + 8.0));
        } else {
          QVS_TRY(launch_col(RCF, c, 12.0 + (base.psi0 ? 8.0 : 0.0)));
        }
      }
    }
    const int nout = grad ? nslots : 1;
    {
      cudaEvent_t e0;
      QVS_TRY(prof_begin(h, &e0));
      QVS_TRY(reduce_rows(h, h->part.as<double>(), grid, h->rowmap.as<int>(), nout, h->res.as<double>()));
      QVS_TRY(prof_end(h, "reduce_rows", 8.0 * grid * nout, e0));
      ++launches;
    }
    h->launches = launches;
    QVS_TRY(ensure_host_res(h, p));
    QVS_CUDA_TRY(cudaMemcpyAsync(h->host_res, h->res.ptr, sizeof(double) * nout, cudaMemcpyDeviceToHost,
                                 h->stream));
    int* host_flag = reinterpret_cast<int*>(h->host_res + 1 + 2 * (size_t)h->host_res_cap);
    QVS_CUDA_TRY(cudaMemcpyAsync(host_flag, h->flags.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    QVS_TRY(prof_flush(h));
    if (*host_flag != 0) return QVS_ETIMEOUT;   // a column pass gave up waiting for its tile copy
    *E = h->host_res[0];
    if (grad)
      for (int k = 0; k < p; ++k) {
        dg[k] = h->host_res[1 + k];
        dt[k] = h->host_res[1 + p + k];
      }
    return QVS_OK;
  }
};

}  // namespace cf
}  // namespace qvs
