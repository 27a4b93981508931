// Device building blocks of the circulant (QWOA) mixer passes: a 2^14-point tile DFT held in
// registers and shared memory.
//
// Sec. 3: a circulant W is diagonalised by the discrete Fourier transform, so
// exp(-i t W) psi = F^-1 exp(-i t Lambda) F psi. The N-point transform (N = 2^n) is split into a
// column transform over the high index bits and a row transform over the low 14 bits, with the
// twiddle omega_N^(j_low * k_col) between them (four-step). Each of those tile transforms is again
// a three-digit four-step transform: a small DFT over each digit (at most 32 points, in registers,
// radix-2 decimation in frequency with compile-time twiddles) and one computed twiddle per
// amplitude between digits. Outputs stay in the digit-reversed, bit-reversed order the steps produce; the
// eigenvalue table is stored in that order, and the inverse transform runs the same steps
// backwards, so no reordering pass is ever made.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace qvs {
namespace cf {

constexpr int TB = 14;            // tile bits
constexpr int TILE = 1 << TB;     // amplitudes per tile
constexpr int RB = 5;             // register bits per layout
constexpr int R = 1 << RB;        // amplitudes per thread
constexpr int NT = TILE / R;      // 512 threads

// e^{-2 pi i m / 32}, m < 16
constexpr float kCos32[16] = {1.0f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                              7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
                              0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
                              -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f};
constexpr float kSin32[16] = {0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
                              7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f,
                              1.0f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                              7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f};

template <int N, class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl<N>(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int bitrev(int x, int d) {
  int r = 0;
  for (int i = 0; i < d; ++i) r |= ((x >> i) & 1) << (d - 1 - i);
  return r;
}

// Geometry of a tile DFT over tile bits [CB, 14) with digits D1 (low), D2, D3 (high); tile bits
// below CB are spectator columns. Step layout k (0, 1, 2 for digits 1, 2, 3) holds digit k in
// register bits 0..d_k-1 and spectators in the rest; thread bits are the remaining tile bits in
// increasing order. Row tiles (CB = 0) take the lowest other tile bits as spectators. Column tiles
// take the other digits' bits, highest first, then the highest column bits, so that the lowest
// column bits (consecutive addresses) are lane bits: a warp's global load or store of one register
// then covers whole 32-byte sectors, where the lowest-bit choice spread it over two to four times
// as many partly used sectors.
template <int CB, int D1, int D2, int D3>
struct Geo {
  static_assert(CB + D1 + D2 + D3 == TB, "digits must cover the transform bits");
  static_assert(D1 <= RB && D2 <= RB && D3 <= RB, "a digit must fit in registers");
  static constexpr int B = D1 + D2 + D3;
  static constexpr int L = 1 << B;
  __host__ __device__ static constexpr int dstart(int k) { return k == 0 ? CB : (k == 1 ? CB + D1 : CB + D1 + D2); }
  __host__ __device__ static constexpr int dsize(int k) { return k == 0 ? D1 : (k == 1 ? D2 : D3); }
  __host__ __device__ static constexpr int regbit(int k, int i) {
    if (i < dsize(k)) return dstart(k) + i;
    int need = i - dsize(k);
    for (int m = 0; m < TB; ++m) {
      // candidate order: ascending for row tiles; descending for column tiles (the transform bits
      // from the top, then the column bits from the top)
      const int b = CB == 0 ? m : TB - 1 - m;
      if (b >= dstart(k) && b < dstart(k) + dsize(k)) continue;
      if (need == 0) return b;
      --need;
    }
    return -1;
  }
  __host__ __device__ static constexpr bool isreg(int k, int b) {
    for (int i = 0; i < RB; ++i)
      if (regbit(k, i) == b) return true;
    return false;
  }
  __host__ __device__ static constexpr int thrbit(int k, int i) {
    int c = 0;
    for (int b = 0; b < TB; ++b) {
      if (isreg(k, b)) continue;
      if (c == i) return b;
      ++c;
    }
    return -1;
  }
  __host__ __device__ static constexpr int jreg(int k, int r) {
    int j = 0;
    for (int i = 0; i < RB; ++i)
      if ((r >> i) & 1) j |= 1 << regbit(k, i);
    return j;
  }
  template <int K>
  __host__ __device__ static int jthr(int tid) {
    int j = 0;
#pragma unroll
    for (int i = 0; i < TB - RB; ++i)
      if ((tid >> i) & 1) j |= 1 << thrbit(K, i);
    return j;
  }
  // frequency produced at position p (the B transform bits of the tile index, shifted down by CB)
  __host__ __device__ static constexpr int freq(int p) {
    const int p1 = p & ((1 << D1) - 1);
    const int p2 = (p >> D1) & ((1 << D2) - 1);
    const int p3 = p >> (D1 + D2);
    return bitrev(p3, D3) + (bitrev(p2, D2) << D3) + (bitrev(p1, D1) << (D3 + D2));
  }
};

// threadIdx.x read through a volatile instruction: index arithmetic (and the loads that
// depend on it) is recomputed where it is used instead of being kept live, or reused, across the
// forward and inverse transforms of one pass
__device__ __forceinline__ int tid_fresh() {
  int t;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
  return t;
}

// shared-memory slot of tile index j: one padding slot after every 16 amplitudes and one more
// after every 256. The map is additive over disjoint index bits (a register's slot is the
// thread's base slot plus a compile-time constant) and keeps the 16-lane phases of the step layouts
// of the 14-bit row transform and the 12-bit column transform conflict-free.
__host__ __device__ __forceinline__ constexpr int spos(int j) { return j + (j >> 4) + (j >> 8); }
constexpr int SM_SLOTS = TILE + (TILE >> 4) + (TILE >> 8);

// complex add / subtract as one paired-float instruction each (same rounding as two scalar adds)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// small forward DFT (decimation in frequency, output bit-reversed) on digit k of layout k:
// registers r = u + 2^d * sp, d = digit size, u = digit-local index
template <class G, int K>
__device__ __forceinline__ void small_dft(float2 (&v)[R]) {
  constexpr int d = G::dsize(K);
  static_for<d>([&](auto si) {
    constexpr int s = d - 1 - decltype(si)::value;
    constexpr int h = 1 << s;
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      constexpr int u = r & ((1 << d) - 1);
      if constexpr (!(u & h)) {
        constexpr int m = (u & (h - 1)) << (4 - s);
        const float2 a = v[r], b = v[r | h];
        v[r] = cadd(a, b);
        const float2 t = csub(a, b);
        if constexpr (m == 0) {
          v[r | h] = t;
        } else if constexpr (m == 8) {
          v[r | h] = make_float2(t.y, -t.x);   // * (-i)
        } else {
          constexpr float wc = kCos32[m], ws = kSin32[m];
          v[r | h] = cmul(t, make_float2(wc, -ws));
        }
      }
    });
  });
}

// exact inverse of small_dft up to a factor 2^d (stages in reverse order)
template <class G, int K>
__device__ __forceinline__ void small_idft(float2 (&v)[R]) {
  constexpr int d = G::dsize(K);
  static_for<d>([&](auto si) {
    constexpr int s = decltype(si)::value;
    constexpr int h = 1 << s;
    static_for<R>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      constexpr int u = r & ((1 << d) - 1);
      if constexpr (!(u & h)) {
        constexpr int m = (u & (h - 1)) << (4 - s);
        const float2 a = v[r], b = v[r | h];
        float2 t;
        if constexpr (m == 0) {
          t = b;
        } else if constexpr (m == 8) {
          t = make_float2(-b.y, b.x);   // * (+i)
        } else {
          constexpr float wc = kCos32[m], ws = kSin32[m];
          t = cmul(b, make_float2(wc, ws));
        }
        v[r] = cadd(a, t);
        v[r | h] = csub(a, t);
      }
    });
  });
}

// shared-memory transpose from step layout KF to step layout KT
template <class G, int KF, int KT>
__device__ __forceinline__ void xchg(float2 (&v)[R], float2* sm, int tid) {
  float2* bf = sm + spos(G::template jthr<KF>(tid));
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    constexpr int o = spos(G::jreg(KF, r));
    bf[o] = v[r];
  });
  __syncthreads();
  const float2* bt = sm + spos(G::template jthr<KT>(tid));
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    constexpr int o = spos(G::jreg(KT, r));
    v[r] = bt[o];
  });
  __syncthreads();
}

// Inter-digit twiddles e^{-2 pi i e / 2^14}: the integer exponent shifted to the top of a 32-bit word
// is the turn e / 2^14 as a signed fixed-point fraction in [-1/2, 1/2), and one hardware
// sine/cosine of its float conversion gives the twiddle. A shared 4096-entry table of fp64-rounded
// roots (one read per twiddle, XOR-swizzled against bank conflicts) measured slower in every pass:
// QWOA N=2^26, p=6 14.2 ms computed against 15.0 ms with the table.
__device__ __forceinline__ float2 tw14(int e) {
  const int32_t es = (int32_t)((uint32_t)e << (32 - TB));
  float sn, cs;
  __sincosf((float)es * 1.46291807926715968e-09f, &sn, &cs);   // 2 pi / 2^32
  return make_float2(cs, -sn);
}

// Twiddle between digit 3 and digit 2 (in step layout 2): omega_L^((j1 + 2^D1 j2) * k3), and
// between digit 2 and digit 1 (in step layout 1): omega_L^(2^D3 * j1 * k2). conj = true applies
// the conjugate (inverse transform).
template <class G, bool CONJ>
__device__ __forceinline__ void twiddle32(float2 (&v)[R], int tid) {
  constexpr int D1 = G::dsize(0), D2 = G::dsize(1), D3 = G::dsize(2);
  const int jt = G::template jthr<2>(tid_fresh());
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    constexpr int k3 = bitrev(r & ((1 << D3) - 1), D3);
    if constexpr (k3 != 0) {
      const int jlow = ((jt | G::jreg(2, r)) >> G::dstart(0)) & ((1 << (D1 + D2)) - 1);
      const int e = (jlow * k3) & (G::L - 1);
      const float2 w = tw14(e << (TB - G::B));
      v[r] = CONJ ? cmulc(v[r], w) : cmul(v[r], w);
    }
  });
}
template <class G, bool CONJ>
__device__ __forceinline__ void twiddle21(float2 (&v)[R], int tid) {
  constexpr int D1 = G::dsize(0), D2 = G::dsize(1), D3 = G::dsize(2);
  const int jt = G::template jthr<1>(tid_fresh());
  static_for<R>([&](auto ri) {
    constexpr int r = decltype(ri)::value;
    constexpr int k2 = bitrev(r & ((1 << D2) - 1), D2);
    if constexpr (k2 != 0) {
      const int j1 = ((jt | G::jreg(1, r)) >> G::dstart(0)) & ((1 << D1) - 1);
      const int e = ((j1 * k2) << D3) & (G::L - 1);
      // the 14-bit row transform's digit-2 reads land 2-way on the banks: computed as well
      const float2 w = tw14(e << (TB - G::B));
      v[r] = CONJ ? cmulc(v[r], w) : cmul(v[r], w);
    }
  });
}

// forward tile DFT: from step layout 2 (natural order in the transform bits) to step layout 0
template <class G>
__device__ __forceinline__ void tile_fwd(float2 (&v)[R], float2* sm, int tid) {
  small_dft<G, 2>(v);
  twiddle32<G, false>(v, tid);
  xchg<G, 2, 1>(v, sm, tid);
  small_dft<G, 1>(v);
  twiddle21<G, false>(v, tid);
  xchg<G, 1, 0>(v, sm, tid);
  small_dft<G, 0>(v);
}

// inverse tile DFT (unscaled): from step layout 0 back to step layout 2
template <class G>
__device__ __forceinline__ void tile_inv(float2 (&v)[R], float2* sm, int tid) {
  small_idft<G, 0>(v);
  xchg<G, 0, 1>(v, sm, tid);
  twiddle21<G, true>(v, tid);
  small_idft<G, 1>(v);
  xchg<G, 1, 2>(v, sm, tid);
  twiddle32<G, true>(v, tid);
  small_idft<G, 2>(v);
}

}  // namespace cf
}  // namespace qvs
