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
//   L3: register bits {4, 9, 10, 11}, thread bits {0..3, 5..8} (lanes = two runs of 16 j)
// L0, L1, L2 cover all twelve tile bits; L3 and L2 cover bits 4..11, all that a pass rotating only
// the tile bits >= 4 needs, with one transpose between them instead of two.
template <int L>
__host__ __device__ __forceinline__ constexpr int tj(int r, int tid) {
  return L == 0 ? ((r & 1) | (tid << 1) | ((r >> 1) << 9))
       : L == 1 ? ((tid & 1) | (r << 1) | ((tid >> 1) << 5))
       : L == 2 ? ((tid & 31) | (r << 5) | ((tid >> 5) << 9))
                : ((tid & 15) | ((r & 1) << 4) | ((tid >> 4) << 5) | ((r >> 1) << 9));
}
// tile bit carried by register bit i in layout L
__host__ __device__ __forceinline__ constexpr int regbit(int L, int i) {
  return L == 0 ? (i == 0 ? 0 : 8 + i) : (L == 1 ? 1 + i : (L == 2 ? 5 + i : (i == 0 ? 4 : 8 + i)));
}
// shared-memory slot of tile index j: two padding slots after every 32 amplitudes. The map is
// additive over disjoint index bits, so a register's slot is the thread's base slot plus a
// compile-time constant (no per-access index arithmetic); the 16-lane phases of 8-byte accesses
// (L1, L2) and the 8-lane phases of 16-byte accesses (L0) hit distinct banks, and pairs (j, j^1)
// stay adjacent and 16-byte aligned.
__host__ __device__ __forceinline__ constexpr int spos(int j) { return j + 2 * (j >> 5); }
constexpr int SM_SLOTS = TILE + 2 * (TILE >> 5);   // slots per shared buffer

// Tile geometry. Tile bits 0..s-1 are the low index bits 0..s-1 (a contiguous chunk of 2^s
// amplitudes); tile bits s..TB-1 are the consecutive index bits hfirst..hfirst+TB-s-1. The CTA
// index scatters into the remaining (non-tile) index bits.
struct Tile {
  uint32_t smask;     // (1 << s) - 1
  int hshift;         // hfirst - s
  uint8_t ntbit[32];  // non-tile index bit positions (ascending)
  int n_nt;
};

__device__ __forceinline__ uint32_t tile_base(const Tile& t, uint32_t bid) {
  uint32_t base = 0;
  for (int i = 0; i < t.n_nt; ++i)
    if ((bid >> i) & 1u) base |= 1u << t.ntbit[i];
  return base;
}

// global offset of tile index j (bits below s stay, bits from s up move by hshift); the map is
// bitwise, so offset(j1 | j2) = offset(j1) + offset(j2) for disjoint j1, j2
__device__ __forceinline__ uint32_t toff(const Tile& t, uint32_t j) {
  return (j & t.smask) + ((j & ~t.smask) << t.hshift);
}

template <class T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

// ---------------------------------------------------------------- storage form
//
// The private buffers of the tiled path (working state, adjoint vector, checkpoints) hold
// W_j = (-i)^popcount(j) psi_j (up to the frame below). In this gauge the single-qubit term -i X_b
// is the real map (W_a, W_b) -> (W_b, -W_a) on every pair a, b = a | 2^b, so
//     exp(-i t X_b) = cos t (I - i tan t X_b)   acts as   W_a += T W_b,  W_b -= T W_a   (T = tan t)
// up to the common real factor cos t: one paired-float FMA per amplitude and bit, with the same
// two constants (T, T) and (-T, -T) for every pair. Diagonal operators (phase, Q) are unchanged.
//
// |T| <= 1 is kept by a per-layer angle shift t = t' + pi/2 where |tan t| > 1:
// exp(-i t X)^{(x)n} = exp(-i t' X)^{(x)n} (-i)^n X_all, and (-i)^n X_all (X_all = all bits
// flipped) commutes with every mixer rotation, so the schedule carries it as a frame: the buffer
// holds W with state = k P^F W, P the gauge image of (-i)^n X_all, F in {0, 1} and k real. Under
// F = 1 the diagonal operators read q at the complemented index (q index XOR qx, qx = 2^n - 1).
// The host tracks k and F pass by pass (the cos t' factors, the frame toggles and the
// renormalisation folded into each phase) and hands every kernel its real scale factors.

__host__ __device__ __forceinline__ constexpr int cpop(int x) {
  int c = 0;
  while (x) {
    c += x & 1;
    x >>= 1;
  }
  return c;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
template <class C, class T> __device__ __forceinline__ C mk2(T x, T y);
template <> __device__ __forceinline__ float2 mk2<float2, float>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 mk2<double2, double>(double x, double y) { return make_double2(x, y); }

// multiply by i^m (m mod 4): edge conversions between the gauge and the plain amplitudes
template <class C>
__device__ __forceinline__ C mul_ipow(C v, uint32_t m) {
  C w = v;
  if (m & 1u) {
    w.x = -v.y;
    w.y = v.x;
  }
  if (m & 2u) {
    w.x = -w.x;
    w.y = -w.y;
  }
  return w;
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

// multiply an amplitude by (c - i s) (c = rho cos theta, s = rho sin theta: exp(-i theta) and a real
// scale rho)
template <class C, class T>
__device__ __forceinline__ C phase_mul(C v, T c, T s) {
  C w;
  w.x = c * v.x + s * v.y;
  w.y = c * v.y - s * v.x;
  return w;
}

// Im(conj(l) * p)
template <class C> __device__ __forceinline__ auto imdot_st(C l, C p) { return l.x * p.y - l.y * p.x; }
template <class C> __device__ __forceinline__ auto hsum(C z) { return z.x + z.y; }

// normal-form helpers (the single-CTA small-state kernel keeps amplitudes as (re, im))
__device__ __forceinline__ void rot_normal(float2& a, float2& b, float c, float s) {
  const float2 a0 = a;
  a.x = c * a.x + s * b.y;
  a.y = c * a.y - s * b.x;
  b.x = c * b.x + s * a0.y;
  b.y = c * b.y - s * a0.x;
}
__device__ __forceinline__ void rot_normal(double2& a, double2& b, double c, double s) {
  const double2 a0 = a;
  a.x = c * a.x + s * b.y;
  a.y = c * a.y - s * b.x;
  b.x = c * b.x + s * a0.y;
  b.y = c * b.y - s * a0.x;
}
__device__ __forceinline__ float imdot(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ double imdot(double2 a, double2 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ float2 cmul_conj(float2 v, float c, float s) {
  return make_float2(c * v.x + s * v.y, c * v.y - s * v.x);
}
__device__ __forceinline__ double2 cmul_conj(double2 v, double c, double s) {
  return make_double2(c * v.x + s * v.y, c * v.y - s * v.x);
}

// ---------------------------------------------------------------- register-layout operations
//
// The tile bits a pass rotates are "every tile bit >= TH" for a threshold TH fixed by the tile type
// (TH = 0: all twelve; TH = s: the group above the s low chunk bits). With TH a template argument
// the per-bit choice folds away after unrolling and each layout step is straight-line code.
// TH < 0 reads the bits from the runtime mask instead (batched kernel).
template <int L, int TH>
__device__ __forceinline__ bool bit_on(int i, uint32_t mask) {
  if constexpr (TH >= 0) return regbit(L, i) >= TH;
  else return (mask >> regbit(L, i)) & 1u;
}

// W_a += T W_b, W_b -= T W_a on the register pairs of the rotated bits (T < 0: the inverse map up
// to the real factor 1 + T^2). With a runtime mask every bit is rotated, the masked-out ones with
// tangent 0 (the identity): a per-bit branch would cost register moves at every join.
template <int L, int TH, class C, class T>
__device__ __forceinline__ void rot_layout(C (&v)[R], uint32_t mask, T tn) {
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    if (TH < 0 || bit_on<L, TH>(i, mask)) {
      const T ti = (TH >= 0 || bit_on<L, TH>(i, mask)) ? tn : T(0);
      const C tp = mk2<C, T>(ti, ti), tm = mk2<C, T>(-ti, -ti);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(r & (1 << i))) {
          const int r1 = r | (1 << i);
          const C a = v[r], b = v[r1];
          v[r] = fma2(tp, b, a);
          v[r1] = fma2(tm, a, b);
        }
      }
    }
  }
}

// Adjoint step on psi (p) and lambda (l): accumulate Re<l|Y_b|p> = Im<lam|X_b psi> for every
// rotated bit b of the layout at the step's entry point (X_b commutes with all rotations of the
// same layer, so any common point of the two vectors gives the layer's value), then undo the
// rotations (tangent -tn). acc += sc * sum; the step moves both vectors by the real factor
// cos t' per bit, so sc advances by c2 = cos^2 t' per rotated bit.
template <int L, int TH, class C, class T, class A>
__device__ __forceinline__ void unrot_layout_acc(C (&p)[R], C (&l)[R], uint32_t mask, T tn, T c2, T& sc,
                                                 A& acc) {
  C e1 = mk2<C, T>(0, 0), e2 = e1;
  T step = T(1);
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    if (bit_on<L, TH>(i, mask)) {
      step *= c2;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(r & (1 << i))) {
          const int r1 = r | (1 << i);
          e1 = fma2(l[r], p[r1], e1);
          e2 = fma2(l[r1], p[r], e2);
        }
      }
    }
  }
  rot_layout<L, TH>(p, mask, -tn);
  rot_layout<L, TH>(l, mask, -tn);
  acc += (A)(sc * (hsum(e1) - hsum(e2)));
  sc *= step;
}

// shared-memory transpose from layout LF to layout LT
template <int L, class C>
__device__ __forceinline__ void sput(const C (&v)[R], C* sm, int tid);
template <int L, class C>
__device__ __forceinline__ void sget(C (&v)[R], const C* sm, int tid);

template <int LF, int LT, class C>
__device__ __forceinline__ void xchg(C (&v)[R], C* sm, int tid) {
  sput<LF>(v, sm, tid);
  __syncthreads();
  sget<LT>(v, sm, tid);
  __syncthreads();
}

// ALT: transpose through buffer BUF of two (sm, sm + SM_SLOTS) with one barrier: a pass alternates
// the buffers, so the barrier of the next transpose already orders this one's reads before the
// transpose after it writes the same buffer again. Used where the CTA already holds two buffers
// (the batched kernel); the per-pass kernels keep one buffer, since a second one costs them L1
// capacity that their streaming loads need (F2 0.67 -> 0.86 ms at n=28 with two).
template <int LF, int LT, int BUF, bool ALT, class C>
__device__ __forceinline__ void xchg_alt(C (&v)[R], C* sm, int tid) {
  if constexpr (ALT) {
    C* b = sm + BUF * SM_SLOTS;
    sput<LF>(v, b, tid);
    __syncthreads();
    sget<LT>(v, b, tid);
  } else {
    xchg<LF, LT>(v, sm, tid);
  }
}

template <int L, class C>
__device__ __forceinline__ void sput(const C (&v)[R], C* sm, int tid) {
  C* b = sm + spos(tj<L>(0, tid));
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float2 x = *reinterpret_cast<const float2*>(&v[r]);
      const float2 y = *reinterpret_cast<const float2*>(&v[r + 1]);
      *reinterpret_cast<float4*>(b + spos(tj<0>(r, 0))) = make_float4(x.x, x.y, y.x, y.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) b[spos(tj<L>(r, 0))] = v[r];
  }
}

template <int L, class C>
__device__ __forceinline__ void sget(C (&v)[R], const C* sm, int tid) {
  const C* b = sm + spos(tj<L>(0, tid));
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 w = *reinterpret_cast<const float4*>(b + spos(tj<0>(r, 0)));
      *reinterpret_cast<float2*>(&v[r]) = make_float2(w.x, w.y);
      *reinterpret_cast<float2*>(&v[r + 1]) = make_float2(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[spos(tj<L>(r, 0))];
  }
}

// read layout L from a dense shared copy of the tile (slot = tile index, no padding): L0 reads
// 16-byte pairs at 16 (tid + 256 k) and L2 reads 8 bytes at 8 (lane + 32 (r + 16 warp)), so a warp's
// accesses are contiguous and conflict-free
template <int L, class C>
__device__ __forceinline__ void dget(C (&v)[R], const C* st, int tid) {
  const C* b = st + tj<L>(0, tid);
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 w = *reinterpret_cast<const float4*>(b + tj<0>(r, 0));
      *reinterpret_cast<float2*>(&v[r]) = make_float2(w.x, w.y);
      *reinterpret_cast<float2*>(&v[r + 1]) = make_float2(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = b[tj<L>(r, 0)];
  }
}

// two vectors through two shared buffers (sm and sm + SM_SLOTS) with one barrier pair
template <int LF, int LT, class C>
__device__ __forceinline__ void xchg2(C (&a)[R], C (&b)[R], C* sm, int tid) {
  sput<LF>(a, sm, tid);
  sput<LF>(b, sm + SM_SLOTS, tid);
  __syncthreads();
  sget<LT>(a, sm, tid);
  sget<LT>(b, sm + SM_SLOTS, tid);
  __syncthreads();
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- global loads and stores
// off = tile base + offset of the thread's own index bits in layout L. The tile map is additive
// over disjoint index bits, so the offset of register r is the sum of the offsets of its set
// register bits: four per-layout values, combined with at most three additions per access.

template <int L>
__device__ __forceinline__ void reg_bit_offsets(const Tile& t, uint32_t (&o)[RB]) {
#pragma unroll
  for (int i = 0; i < RB; ++i) o[i] = toff(t, 1u << regbit(L, i));
}

__device__ __forceinline__ uint32_t reg_off(const uint32_t (&o)[RB], int r) {
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < RB; ++i)
    if ((r >> i) & 1) x += o[i];
  return x;
}

template <int L, class C>
__device__ __forceinline__ void gload(C (&v)[R], const C* __restrict__ g, uint32_t off, const Tile& t) {
  uint32_t o[RB];
  reg_bit_offsets<L>(t, o);
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float4 w = __ldcs(reinterpret_cast<const float4*>(g + off + reg_off(o, r)));
      *reinterpret_cast<float2*>(&v[r]) = make_float2(w.x, w.y);
      *reinterpret_cast<float2*>(&v[r + 1]) = make_float2(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = __ldcs(g + off + reg_off(o, r));
  }
}

template <int L, class C>
__device__ __forceinline__ void gstore(const C (&v)[R], C* __restrict__ g, uint32_t off, const Tile& t) {
  uint32_t o[RB];
  reg_bit_offsets<L>(t, o);
  if constexpr (L == 0 && sizeof(C) == 8) {
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const float2 a = *reinterpret_cast<const float2*>(&v[r]);
      const float2 b = *reinterpret_cast<const float2*>(&v[r + 1]);
      __stcs(reinterpret_cast<float4*>(g + off + reg_off(o, r)), make_float4(a.x, a.y, b.x, b.y));
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) __stcs(g + off + reg_off(o, r), v[r]);
  }
}

// Caller-visible (plain) amplitudes to the gauge on load: W_j = (-i)^|j| psi_j. tpop = popcount
// of the tile base and the thread's own index bits in layout L.
template <int L, class C>
__device__ __forceinline__ void gload_plain(C (&v)[R], const C* __restrict__ g, uint32_t off,
                                            const Tile& t, uint32_t tpop) {
  gload<L>(v, g, off, t);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = mul_ipow(v[r], (0u - (tpop + (uint32_t)cpop(tj<L>(r, 0)))) & 3u);
}

// Gauge to plain amplitudes on store, with the frame: slot j holds the amplitude of index j ^ ox,
// psi_{j ^ ox} = k i^(|j| - F n) W_j (fm = F n mod 4); scalar stores at the XORed index.
template <int L, class C, class T>
__device__ __forceinline__ void gstore_plain(const C (&v)[R], C* __restrict__ g, uint32_t off,
                                             const Tile& t, uint32_t tpop, uint32_t ox, uint32_t fm, T k) {
  uint32_t o[RB];
  reg_bit_offsets<L>(t, o);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    C w = mul_ipow(v[r], (tpop + (uint32_t)cpop(tj<L>(r, 0)) - fm) & 3u);
    w.x *= k;
    w.y *= k;
    __stcs(g + ((off + reg_off(o, r)) ^ ox), w);
  }
}

// q at the element indices XOR qx (qx = 0, or 2^n - 1 under the flipped frame: the warp then reads
// the same segments in reverse lane order)
template <int L, class T>
__device__ __forceinline__ void qload(T (&qv)[R], const T* __restrict__ q, uint32_t off, const Tile& t,
                                      uint32_t qx) {
  uint32_t o[RB];
  reg_bit_offsets<L>(t, o);
#pragma unroll
  for (int r = 0; r < R; ++r) qv[r] = __ldcs(q + ((off + reg_off(o, r)) ^ qx));
}

}  // namespace hc
}  // namespace qvs
