// Device building blocks of the hypercube (QAOA) mixer passes.
//
// The QAOA mixer of Sec. 2.3.1, exp(-i t sum_j X_j), is the product over qubits of the commuting
// rotations exp(-i t X_j) = cos t I - i sin t X_j. A pass loads a tile of 2^TB amplitudes (all
// values of TB index bits for fixed values of the others), applies rotations on any of those bits,
// optionally the diagonal phase exp(-i gamma Q) of Sec. 3, and writes the tile back. Inside a
// tile each thread holds R = 2^RB amplitudes in registers; three register layouts (L0, L1, L2)
// cover the 12 tile bits, and shared memory transposes between them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qvs {
namespace hc {

constexpr int TB = 12;           // tile bits
constexpr int TILE = 1 << TB;    // amplitudes per tile
constexpr int RB = 4;            // register bits per layout
constexpr int R = 1 << RB;       // amplitudes per thread per vector
constexpr int NT = TILE / R;     // threads per CTA (256)

// Tile index j held in register r by thread tid, per layout:
//   L0: register bits {0, 9, 10, 11}, thread bits {1..8}   (global float4 loads/stores)
//   L1: register bits {1, 2, 3, 4},   thread bits {0, 5..11}
//   L2: register bits {5, 6, 7, 8},   thread bits {0..4, 9..11} (lanes = 32 consecutive j)
template <int L>
__host__ __device__ __forceinline__ constexpr int tj(int r, int tid) {
  return L == 0 ? ((r & 1) | (tid << 1) | ((r >> 1) << 9))
       : L == 1 ? ((tid & 1) | (r << 1) | ((tid >> 1) << 5))
                : ((tid & 31) | (r << 5) | ((tid >> 5) << 9));
}
// tile bit carried by register bit i in layout L
__host__ __device__ __forceinline__ constexpr int regbit(int L, int i) {
  return L == 0 ? (i == 0 ? 0 : 8 + i) : (L == 1 ? 1 + i : 5 + i);
}
// shared-memory slot of tile index j: XOR swizzle of bits 1..3 by bits 5..7 keeps the 16-lane
// phases of 8-byte accesses conflict-free in all three layouts and keeps pairs (j, j^1) adjacent.
__device__ __forceinline__ int spos(int j) { return j ^ ((j >> 4) & 0xE); }

// Tile geometry: global element offset of each tile bit, and the non-tile bit positions that
// the CTA index scatters into.
struct Tile {
  uint32_t bitoff[TB];
  uint8_t ntbit[32];
  int n_nt;
};

__device__ __forceinline__ uint32_t tile_base(const Tile& t, uint32_t bid) {
  uint32_t base = 0;
  for (int i = 0; i < t.n_nt; ++i)
    if ((bid >> i) & 1u) base |= 1u << t.ntbit[i];
  return base;
}

// global offset of tile index j (bit scatter through bitoff)
__device__ __forceinline__ uint32_t scatter(const Tile& t, int j) {
  uint32_t o = 0;
#pragma unroll
  for (int b = 0; b < TB; ++b)
    if ((j >> b) & 1) o += t.bitoff[b];
  return o;
}

template <class T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

// ---------------------------------------------------------------- complex helpers

// exp(-i t X) on the pair (a, b) with c = cos t, s = sin t:
//   a' = c a - i s b,  b' = c b - i s a   (the adjoint passes -s)
__device__ __forceinline__ void rot(float2& a, float2& b, float c, float s) {
  const float2 cc = make_float2(c, c);
  const float2 sp = make_float2(s, -s);
  const float2 na = __ffma2_rn(cc, a, __fmul2_rn(sp, make_float2(b.y, b.x)));
  const float2 nb = __ffma2_rn(cc, b, __fmul2_rn(sp, make_float2(a.y, a.x)));
  a = na;
  b = nb;
}
__device__ __forceinline__ void rot(double2& a, double2& b, double c, double s) {
  const double2 a0 = a;
  a.x = c * a.x + s * b.y;
  a.y = c * a.y - s * b.x;
  b.x = c * b.x + s * a0.y;
  b.y = c * b.y - s * a0.x;
}

// Im(conj(a) * b)
__device__ __forceinline__ float imdot(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ double imdot(double2 a, double2 b) { return a.x * b.y - a.y * b.x; }

// multiply v by (c - i s) (forward phase exp(-i theta) with c = cos theta, s = sin theta)
__device__ __forceinline__ float2 cmul_conj(float2 v, float c, float s) {
  return make_float2(c * v.x + s * v.y, c * v.y - s * v.x);
}
__device__ __forceinline__ double2 cmul_conj(double2 v, double c, double s) {
  return make_double2(c * v.x + s * v.y, c * v.y - s * v.x);
}

// Phase angle of exp(-i gamma q): the complex64 path carries gamma / 2pi as a float-float pair
// (hi, lo). The exact product error of hi*q (FMA two-product, Ogita-Rump-Oishi 2005) and the lo
// term give the fractional number of turns to ~1e-8; the rotation angle is then at most pi in
// magnitude and the hardware sine/cosine approximations are accurate to ~5e-7 there.
__device__ __forceinline__ void phase_cs(float q, float ghi, float glo, float& c, float& s) {
  const float p = ghi * q;
  const float e = fmaf(ghi, q, -p);
  const float r = p - rintf(p);
  const float f = r + fmaf(glo, q, e);
  __sincosf(6.28318530717958647692f * f, &s, &c);
}
__device__ __forceinline__ void phase_cs(double q, double gamma, double, double& c, double& s) {
  sincos(gamma * q, &s, &c);
}

// ---------------------------------------------------------------- register-layout operations

template <int L, class C, class T>
__device__ __forceinline__ void rot_layout(C (&v)[R], uint32_t mask, T c, T s) {
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    if (mask & (1u << regbit(L, i))) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!(r & (1 << i))) rot(v[r], v[r | (1 << i)], c, s);
    }
  }
}

// Adjoint rotations exp(+i t X_b) on psi and lam, accumulating Im<lam|X_b psi> for every bit b
// undone (X_b commutes with all rotations of the same layer, so the value is the one at the
// layer's output).
template <int L, class C, class T, class A>
__device__ __forceinline__ void unrot_layout_acc(C (&p)[R], C (&l)[R], uint32_t mask, T c, T s,
                                                 A& acc) {
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    if (mask & (1u << regbit(L, i))) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(r & (1 << i))) {
          const int r1 = r | (1 << i);
          acc += imdot(l[r], p[r1]) + imdot(l[r1], p[r]);
          rot(p[r], p[r1], c, -s);
          rot(l[r], l[r1], c, -s);
        }
      }
    }
  }
}

// shared-memory transpose from layout LF to layout LT
template <int LF, int LT, class C>
__device__ __forceinline__ void xchg(C (&v)[R], C* sm, int tid) {
  if constexpr (LF == 0 && sizeof(C) == 8) {
    float4* s4 = reinterpret_cast<float4*>(sm);
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float2 a = *reinterpret_cast<float2*>(&v[r]);
      const float2 b = *reinterpret_cast<float2*>(&v[r + 1]);
      s4[spos(tj<0>(r, tid)) >> 1] = make_float4(a.x, a.y, b.x, b.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) sm[spos(tj<LF>(r, tid))] = v[r];
  }
  __syncthreads();
  if constexpr (LT == 0 && sizeof(C) == 8) {
    const float4* s4 = reinterpret_cast<const float4*>(sm);
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 w = s4[spos(tj<0>(r, tid)) >> 1];
      *reinterpret_cast<float2*>(&v[r]) = make_float2(w.x, w.y);
      *reinterpret_cast<float2*>(&v[r + 1]) = make_float2(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sm[spos(tj<LT>(r, tid))];
  }
  __syncthreads();
}

template <int LF, int LT, class C>
__device__ __forceinline__ void xchg2(C (&a)[R], C (&b)[R], C* sm, int tid) {
  xchg<LF, LT>(a, sm, tid);
  xchg<LF, LT>(b, sm, tid);
}

// ---------------------------------------------------------------- global loads and stores

// offsets of the 16 registers of layout L relative to the thread's own offset
template <int L>
__device__ __forceinline__ void reg_offsets(const Tile& t, uint32_t (&ro)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) ro[r] = scatter(t, tj<L>(r, 0));
}

template <int L, class C>
__device__ __forceinline__ void gload(C (&v)[R], const C* __restrict__ g, uint32_t off,
                                      const uint32_t (&ro)[R]) {
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 w = __ldcs(reinterpret_cast<const float4*>(g + off + ro[r]));
      *reinterpret_cast<float2*>(&v[r]) = make_float2(w.x, w.y);
      *reinterpret_cast<float2*>(&v[r + 1]) = make_float2(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = __ldcs(g + off + ro[r]);
  }
}

template <int L, class C>
__device__ __forceinline__ void gstore(const C (&v)[R], C* __restrict__ g, uint32_t off,
                                       const uint32_t (&ro)[R]) {
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float2 a = *reinterpret_cast<const float2*>(&v[r]);
      const float2 b = *reinterpret_cast<const float2*>(&v[r + 1]);
      __stcs(reinterpret_cast<float4*>(g + off + ro[r]), make_float4(a.x, a.y, b.x, b.y));
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) __stcs(g + off + ro[r], v[r]);
  }
}

}  // namespace hc
}  // namespace qvs
