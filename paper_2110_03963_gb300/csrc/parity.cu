// QAOAz parity-ring mixer path (Sec. 2.4.1): U_parity(t) = exp(-i t B_last) exp(-i t B_even)
// exp(-i t B_odd) on two rings of qubits (the even qubits and the odd qubits), over the full 2^n
// register. Each factor is a sum of XY terms on disjoint qubit pairs, so its exponential is one
// layer of Givens rotations: on the |01>, |10> amplitudes of a pair,
//     (a, b) -> (cos 2t a - i sin 2t b, cos 2t b - i sin 2t a),
// and the identity on |00>, |11>. No series is needed.
//
// Schedule. The gates of a layer (pairs of index bits, in the printed factor order) are packed on
// the host into passes: a pass is a tile of 12 index bits (the 4 lowest bits, so each tile row is
// 128 contiguous bytes, plus up to 8 others) and the gates whose two bits lie in the tile, taken in
// an order that respects every dependency (a gate follows every earlier gate sharing a bit with
// it; gates on disjoint bits commute). A CTA stages its 2^12-amplitude tile in shared memory,
// applies the pass's gates one after another (1024 pairs each) and writes the tile back. The
// phase of layer k is applied as the tile is loaded in the first pass of the layer. n = 24 needs
// three passes per layer.
//
// Chained sweeps. Consecutive gates of a pass are applied two at a time: each thread takes the
// amplitudes spanned by the two gates' bits (16 for gates on four distinct bits, 8 when they share
// one), loads those either gate moves, applies the first gate and then the second in registers, and
// writes them back. Against one sweep per gate this moves 12 amplitudes instead of 16 through shared
// memory per 16 and halves the barriers; a pass with an odd gate count ends with a one-gate sweep.
//
// Gradient. Every pass output of the forward sweep is stored. The reverse sweep runs the passes
// backwards on (psi, lambda): psi is re-read from the pass's stored output and both vectors are
// staged in shared memory; each gate is undone on both after its term
//     df/dt_k += 2 Im <lambda| (XX+YY)_g |psi>   (at the gate's output)
// is accumulated (one t per layer is shared by every gate, so the layer's derivative is the sum
// over its gates, in any order consistent with the dependencies); the first pass of a layer then
// adds df/dgamma_k = 2 Im <lambda|Q phi_k> and undoes the phase on lambda.
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "qvs_internal.h"

namespace qvs {
namespace pr {

constexpr int TB = 12;
constexpr int TILE = 1 << TB;
constexpr int NT = 256;
constexpr int EPT = TILE / NT;   // 16 amplitudes per thread when staging
constexpr int CHUNK = 4;         // lowest index bits, always in the tile
constexpr int MAXG = 40;         // gates per pass
constexpr int MAXNT = 32;        // non-tile bits

// Shared slot of tile index j: tile bits 4, 5, 6 and 7 XOR the classes 11, 12, 2 and 13 into the low
// four bits (the 8-byte bank class of a half-warp access). A sweep's 16 lanes of a half-warp take
// the first four tile bits its gates leave free, so they fall on 16 distinct classes whenever those
// bits' classes are independent: for the one- and two-gate sweeps of every schedule at n = 12..30
// that costs 1.02 times the conflict-free count of shared-memory wavefronts (1.27 with bits 4 and 5
// alone). Staging lanes (tile bits 0..3) are always conflict-free. The map is linear over XOR, so
// slot(j1 ^ j2) = slot(j1) ^ slot(j2), leaves bits 8..11 alone (slot(t + 256 m) = slot(t) + 256 m)
// and needs no padding slots.
__host__ __device__ __forceinline__ constexpr uint32_t swz(uint32_t j) {
  return j ^ (((j >> 4) & 1u) ? 11u : 0u) ^ (((j >> 5) & 1u) ? 12u : 0u) ^ (((j >> 6) & 1u) ? 2u : 0u) ^
         (((j >> 7) & 1u) ? 13u : 0u);
}
constexpr int SLOTS = TILE;

// combination c of a two-gate sweep on four distinct bits moves unless both gates see 00 or 11
__host__ __device__ constexpr bool moved4(int c) {
  return ((c & 3) == 1 || (c & 3) == 2) || ((c >> 2) == 1 || (c >> 2) == 2);
}

template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// kinds of a sweep: one gate (pairs); two gates on four distinct tile bits (combination bits 0, 1
// = the first gate's, 2, 3 = the second's); two gates sharing one bit (combination bit 1 = the shared
// bit, 0 = the first gate's other bit, 2 = the second's)
enum SweepKind : uint8_t { SW_ONE = 0, SW_DISJOINT = 1, SW_SHARED = 2 };

struct PassDesc {
  uint8_t pos[TB];       // index bit of tile bit i (pos[i] = i for i < CHUNK)
  uint8_t ga[MAXG];      // gate g couples tile bits ga[g] and gb[g]
  uint8_t gb[MAXG];
  uint16_t goff[MAXG][4];  // slot offsets of gate g: pair groups k = 1..3 (t + 256 k), and the pair mask
  uint8_t ntbit[MAXNT];  // non-tile index bits (the CTA index scatters into them)
  int ngates, nnt;
  int nsweeps;
  uint8_t skind[MAXG];       // SweepKind of sweep s
  uint8_t sgate[MAXG];       // its first gate (the second, if any, is sgate + 1)
  uint8_t sbits[MAXG][4];    // the tile bits it spans, ascending (3 or 4 of them)
  uint16_t soff[MAXG][16];   // slot offset of combination c of its bits (in the kind's bit order)
};

struct Args {
  PassDesc d;
  const float2* in;      // forward: pass input (NULL: uniform state); reverse: psi at the output
  float2* out;           // forward: pass output
  const float2* lam_in;  // reverse only
  float2* lam_out;
  const float* q;
  float c, s;            // cos 2t, sin 2t of the layer
  float ph0, ph1;        // phase gamma / 2pi as a float-float pair (first pass of a layer)
  int has_phase;
  float init_amp;
  double* part;          // partial rows part[row * gridDim.x + blockIdx.x]
  int row_t, row_g;
};

__device__ __forceinline__ uint32_t tile_base(const PassDesc& d, uint32_t bid) {
  uint32_t base = 0;
  for (int i = 0; i < d.nnt; ++i)
    if ((bid >> i) & 1u) base |= 1u << d.ntbit[i];
  return base;
}

// index offsets of the amplitudes thread t stages: element m (0..15) is tile index t + 256 m
__device__ __forceinline__ uint32_t thr_off(const PassDesc& d, uint32_t t) {
  uint32_t o = t & 15u;
#pragma unroll
  for (int i = 4; i < 8; ++i)
    if ((t >> i) & 1u) o |= 1u << d.pos[i];
  return o;
}
__device__ __forceinline__ uint32_t elem_off(const PassDesc& d, int m) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 8; i < 12; ++i)
    if ((m >> (i - 8)) & 1) o |= 1u << d.pos[i];
  return o;
}

// slot of pair 0 of thread t for a gate on tile bits (a, b): t's 8 bits spread over the tile bits
// other than a and b, bit a = 0, bit b = 1; pair k = t + 256 m is this slot XOR goff[m - 1]
__device__ __forceinline__ uint32_t pair_slot(uint32_t t, int a, int b) {
  const int p1 = a < b ? a : b, p2 = a < b ? b : a;
  uint32_t x = ((t >> p1) << (p1 + 1)) | (t & ((1u << p1) - 1u));
  x = ((x >> p2) << (p2 + 1)) | (x & ((1u << p2) - 1u));
  return swz(x | (1u << b));
}

// slot of the group base: g's bits spread over the tile bits other than the NB ascending bits b[]
template <int NB>
__device__ __forceinline__ uint32_t group_slot(uint32_t g, const uint8_t* b) {
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int p = b[i];
    g = ((g >> p) << (p + 1)) | (g & ((1u << p) - 1u));
  }
  return swz(g);
}

// paired-float arithmetic: one instruction for both components
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }

// exp(-i 2 pi f) with f = gamma / 2pi * q reduced exactly (float-float turns, FMA two-product)
__device__ __forceinline__ void phase_cs(float q, float ghi, float glo, float& c, float& s) {
  const float p = ghi * q;
  const float e = fmaf(ghi, q, -p);
  const float r = p - rintf(p);
  const float f = r + fmaf(glo, q, e);
  __sincosf(6.28318530717958647692f * f, &s, &c);
}

__device__ __forceinline__ void block_store2(float a, float b, double* part, int ra, int rb) {
  __shared__ double red[2][NT / 32];
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = (double)a;
    red[1][tid >> 5] = (double)b;
  }
  __syncthreads();
  if (tid < 2) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[tid][w];
    const int row = tid == 0 ? ra : rb;
    if (row >= 0) part[(size_t)row * gridDim.x + blockIdx.x] = s;
  }
}

// stage a tile into shared memory: input amplitudes (or the uniform state), the layer's phase
// applied on the way in; every load of the thread is issued before the first use
template <bool IN, bool PH>
__device__ __forceinline__ void stage_fwd(const Args& a, uint32_t base, uint32_t st, float2* sm) {
  float2 xv[EPT];
  float qv[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const uint32_t g = base | elem_off(a.d, m);
    xv[m] = IN ? __ldcs(a.in + g) : make_float2(a.init_amp, 0.f);
    if (PH) qv[m] = __ldcs(a.q + g);
  }
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    float2 x = xv[m];
    if (PH) {
      float c, s;
      phase_cs(qv[m], a.ph0, a.ph1, c, s);
      x = make_float2(c * x.x + s * x.y, c * x.y - s * x.x);   // exp(-i gamma q) x
    }
    sm[st + NT * m] = x;
  }
}

// forward pass: stage (phase), gates, write back
__global__ void __launch_bounds__(NT) fwd_kernel(const __grid_constant__ Args a) {
  __shared__ __align__(16) float2 sm[SLOTS];
  const uint32_t t = threadIdx.x;
  const uint32_t base = tile_base(a.d, blockIdx.x) | thr_off(a.d, t);
  const uint32_t st = swz(t);   // slot of tile index t + 256 m is st + 256 m
  if (a.in) {
    if (a.has_phase) stage_fwd<true, true>(a, base, st, sm);
    else stage_fwd<true, false>(a, base, st, sm);
  } else {
    if (a.has_phase) stage_fwd<false, true>(a, base, st, sm);
    else stage_fwd<false, false>(a, base, st, sm);
  }
  __syncthreads();
  const float2 cc = make_float2(a.c, a.c), sn = make_float2(a.s, -a.s);
  // c x - i s y = (c x.re + s y.im, c x.im - s y.re) and c y - i s x on a pair (x, y)
  auto givens = [&](float2& x, float2& y) {
    const float2 x0 = x;
    x = fma2(cc, x, mul2(sn, swp(y)));
    y = fma2(cc, y, mul2(sn, swp(x0)));
  };
  for (int sw = 0; sw < a.d.nsweeps; ++sw) {
    const int kind = a.d.skind[sw];
    const uint16_t* off = a.d.soff[sw];
    if (kind == SW_DISJOINT) {   // one group of 16 per thread; 12 of them move
      const uint32_t sb = group_slot<4>(t, a.d.sbits[sw]);
      float2 v[16];
      static_for<16>([&](auto ci) {
        constexpr int c = decltype(ci)::value;
        if constexpr (moved4(c)) v[c] = sm[sb ^ off[c]];
      });
      static_for<4>([&](auto ci) {   // first gate: combination bits 0, 1
        constexpr int h = decltype(ci)::value << 2;
        givens(v[h | 1], v[h | 2]);
      });
      static_for<4>([&](auto ci) {   // second gate: combination bits 2, 3
        constexpr int l = decltype(ci)::value;
        givens(v[l | 4], v[l | 8]);
      });
      static_for<16>([&](auto ci) {
        constexpr int c = decltype(ci)::value;
        if constexpr (moved4(c)) sm[sb ^ off[c]] = v[c];
      });
    } else if (kind == SW_SHARED) {   // two groups of 8 per thread; 6 of each move
#pragma unroll
      for (int hg = 0; hg < 2; ++hg) {
        const uint32_t sb = group_slot<3>(t + NT * hg, a.d.sbits[sw]);
        float2 v[8];
        static_for<8>([&](auto ci) {
          constexpr int c = decltype(ci)::value;
          if constexpr (c != 0 && c != 7) v[c] = sm[sb ^ off[c]];
        });
        givens(v[1], v[2]);   // first gate: combination bits 0, 1 (bit 2 = 0)
        givens(v[5], v[6]);   //                                  (bit 2 = 1)
        givens(v[2], v[4]);   // second gate: combination bits 1, 2 (bit 0 = 0)
        givens(v[3], v[5]);   //                                   (bit 0 = 1)
        static_for<8>([&](auto ci) {
          constexpr int c = decltype(ci)::value;
          if constexpr (c != 0 && c != 7) sm[sb ^ off[c]] = v[c];
        });
      }
    } else {
      const int gi = a.d.sgate[sw];
      const uint32_t s0 = pair_slot(t, a.d.ga[gi], a.d.gb[gi]), sm_ab = a.d.goff[gi][3];
#pragma unroll
      for (int k = 0; k < TILE / 4 / NT; ++k) {
        const uint32_t lo = k ? (s0 ^ a.d.goff[gi][k - 1]) : s0, hi = lo ^ sm_ab;
        float2 x = sm[lo], y = sm[hi];
        givens(x, y);
        sm[lo] = x;
        sm[hi] = y;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < EPT; ++m) __stcs(a.out + (base | elem_off(a.d, m)), sm[st + NT * m]);
}

// reverse pass on (psi, lambda)
__global__ void __launch_bounds__(NT) rev_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];   // 2 * SLOTS float2 (dynamic)
  float2* sp = reinterpret_cast<float2*>(smem_raw);
  float2* sl = sp + SLOTS;
  const uint32_t t = threadIdx.x;
  const uint32_t base = tile_base(a.d, blockIdx.x) | thr_off(a.d, t);
  const uint32_t st = swz(t);
  float qv[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const uint32_t g = base | elem_off(a.d, m);
    sp[st + NT * m] = __ldcs(a.in + g);
    sl[st + NT * m] = __ldcs(a.lam_in + g);
    qv[m] = a.has_phase ? __ldcs(a.q + g) : 0.f;   // read with the vectors, used after the gates
  }
  __syncthreads();
  float acc_g = 0.f;
  // Im(conj(l_lo) p_hi) + Im(conj(l_hi) p_lo) = <lambda|(XX+YY)|psi> / 2 on a pair, accumulated as
  // componentwise products (re*im, im*re) whose difference is taken once at the end
  float2 at = make_float2(0.f, 0.f);
  const float2 cc = make_float2(a.c, a.c), sn = make_float2(-a.s, a.s);
  // on a pair at the gate's output: accumulate the gradient term, then undo the gate on both
  // vectors: (a, b) -> (c a + i s b, c b + i s a) = (c a.re - s b.im, c a.im + s b.re)
  auto undo = [&](float2& x, float2& y, float2& u, float2& v) {
    at = fma2(u, swp(y), at);
    at = fma2(v, swp(x), at);
    const float2 x0 = x, u0 = u;
    x = fma2(cc, x, mul2(sn, swp(y)));
    y = fma2(cc, y, mul2(sn, swp(x0)));
    u = fma2(cc, u, mul2(sn, swp(v)));
    v = fma2(cc, v, mul2(sn, swp(u0)));
  };
  for (int sw = a.d.nsweeps - 1; sw >= 0; --sw) {
    const int kind = a.d.skind[sw];
    const uint16_t* off = a.d.soff[sw];
    if (kind == SW_DISJOINT) {
      const uint32_t sb = group_slot<4>(t, a.d.sbits[sw]);
      float2 x[16], l[16];
      static_for<16>([&](auto ci) {
        constexpr int c = decltype(ci)::value;
        if constexpr (moved4(c)) {
          x[c] = sp[sb ^ off[c]];
          l[c] = sl[sb ^ off[c]];
        }
      });
      static_for<4>([&](auto ci) {   // second gate first
        constexpr int lo = decltype(ci)::value;
        undo(x[lo | 4], x[lo | 8], l[lo | 4], l[lo | 8]);
      });
      static_for<4>([&](auto ci) {
        constexpr int h = decltype(ci)::value << 2;
        undo(x[h | 1], x[h | 2], l[h | 1], l[h | 2]);
      });
      static_for<16>([&](auto ci) {
        constexpr int c = decltype(ci)::value;
        if constexpr (moved4(c)) {
          sp[sb ^ off[c]] = x[c];
          sl[sb ^ off[c]] = l[c];
        }
      });
    } else if (kind == SW_SHARED) {
#pragma unroll
      for (int hg = 0; hg < 2; ++hg) {
        const uint32_t sb = group_slot<3>(t + NT * hg, a.d.sbits[sw]);
        float2 x[8], l[8];
        static_for<8>([&](auto ci) {
          constexpr int c = decltype(ci)::value;
          if constexpr (c != 0 && c != 7) {
            x[c] = sp[sb ^ off[c]];
            l[c] = sl[sb ^ off[c]];
          }
        });
        undo(x[2], x[4], l[2], l[4]);   // second gate first: combination bits 1, 2
        undo(x[3], x[5], l[3], l[5]);
        undo(x[1], x[2], l[1], l[2]);   // first gate: combination bits 0, 1
        undo(x[5], x[6], l[5], l[6]);
        static_for<8>([&](auto ci) {
          constexpr int c = decltype(ci)::value;
          if constexpr (c != 0 && c != 7) {
            sp[sb ^ off[c]] = x[c];
            sl[sb ^ off[c]] = l[c];
          }
        });
      }
    } else {
      const int gi = a.d.sgate[sw];
      const uint32_t s0 = pair_slot(t, a.d.ga[gi], a.d.gb[gi]), sm_ab = a.d.goff[gi][3];
#pragma unroll
      for (int k = 0; k < TILE / 4 / NT; ++k) {
        const uint32_t lo = k ? (s0 ^ a.d.goff[gi][k - 1]) : s0, hi = lo ^ sm_ab;
        float2 x = sp[lo], y = sp[hi], u = sl[lo], v = sl[hi];
        undo(x, y, u, v);
        sp[lo] = x;
        sp[hi] = y;
        sl[lo] = u;
        sl[hi] = v;
      }
    }
    __syncthreads();
  }
  const float acc_t = at.x - at.y;
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    const uint32_t g = base | elem_off(a.d, m);
    float2 l = sl[st + NT * m];
    if (a.has_phase) {
      const float2 p = sp[st + NT * m];
      acc_g += qv[m] * (l.x * p.y - l.y * p.x);
      float c, s;
      phase_cs(qv[m], a.ph0, a.ph1, c, s);
      l = make_float2(c * l.x - s * l.y, c * l.y + s * l.x);   // exp(+i gamma q) lambda
    }
    __stcs(a.lam_out + g, l);
  }
  // 2 Im<lambda|(XX+YY)|psi> = 4 * (accumulated half-sums); df/dgamma = 2 Im<lambda|Q phi>
  block_store2(4.f * acc_t, 2.f * acc_g, a.part, a.row_t, a.has_phase ? a.row_g : -1);
}

// E = sum q |psi|^2 and lambda = Q psi (elementwise over the register)
__global__ void __launch_bounds__(NT) elam_kernel(int64_t dim, const float2* __restrict__ psi,
                                                  const float* __restrict__ q, float2* __restrict__ lam,
                                                  double* part, int row) {
  float e = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < dim; i += (int64_t)gridDim.x * NT) {
    const float2 x = __ldcs(psi + i);
    const float qq = __ldcs(q + i);
    e += qq * (x.x * x.x + x.y * x.y);
    if (lam) __stcs(lam + i, make_float2(qq * x.x, qq * x.y));
  }
  block_store2(e, 0.f, part, row, -1);
}

// the paper's parity initial state (Sec. 6.2): asset a on qubits (2a, 2a+1); |01> for a < A,
// (|00> + |11>)/sqrt 2 otherwise (qubit u = index bit n-1-u)
__global__ void parity_state_kernel(int n, int A, double amp, float2* __restrict__ out) {
  const int64_t dim = (int64_t)1 << n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    bool ok = true;
    for (int a = 0; a < n / 2; ++a) {
      const int hi = (int)((i >> (n - 1 - 2 * a)) & 1), lo = (int)((i >> (n - 2 - 2 * a)) & 1);
      ok = ok && (a < A ? (hi == 0 && lo == 1) : (hi == lo));
    }
    out[i] = make_float2(ok ? (float)amp : 0.f, 0.f);
  }
}

// ---------------------------------------------------------------- host side

// qubit pairs of B_odd, B_even, B_last on the even-qubit ring and the odd-qubit ring (1-indexed
// ring positions k: B_odd (k, k+1) for odd k < N; B_even (k, k+1) for even k < N plus (N, 1) when
// N is even; B_last (N, 1) when N is odd), as index-bit pairs, in the printed factor order
static std::vector<std::pair<int, int>> layer_gates(int n) {
  std::vector<std::pair<int, int>> rounds[3];
  for (int start = 0; start < 2; ++start) {
    std::vector<int> ring;
    for (int qb = start; qb < n; qb += 2) ring.push_back(qb);
    const int N = (int)ring.size();
    for (int k = 1; k < N; ++k) rounds[(k % 2 == 1) ? 0 : 1].push_back({ring[k - 1], ring[k]});
    if (N >= 2) rounds[(N % 2 == 0) ? 1 : 2].push_back({ring[N - 1], ring[0]});
  }
  std::vector<std::pair<int, int>> gates;
  for (auto& r : rounds)
    for (auto& pq : r) gates.push_back({n - 1 - pq.first, n - 1 - pq.second});
  return gates;
}

struct Pass {
  PassDesc d;
};

// greedy packing of one layer's gates into passes (see the file comment)
static int plan_layer(int n, std::vector<Pass>& out) {
  const auto gates = layer_gates(n);
  const int G = (int)gates.size();
  std::vector<char> done(G, 0);
  int left = G;
  while (left > 0) {
    std::vector<int> tile;
    for (int b = 0; b < CHUNK; ++b) tile.push_back(b);
    auto in_tile = [&](int b) { return std::find(tile.begin(), tile.end(), b) != tile.end(); };
    std::vector<int> sel;
    for (int g = 0; g < G; ++g) {
      if (done[g]) continue;
      bool ok = true;
      for (int h = 0; h < g && ok; ++h) {
        const bool shares = gates[h].first == gates[g].first || gates[h].first == gates[g].second ||
                            gates[h].second == gates[g].first || gates[h].second == gates[g].second;
        if (shares && !done[h] && std::find(sel.begin(), sel.end(), h) == sel.end()) ok = false;
      }
      if (!ok) continue;
      const int need = (in_tile(gates[g].first) ? 0 : 1) + (in_tile(gates[g].second) ? 0 : 1);
      if ((int)tile.size() + need > TB || (int)sel.size() >= MAXG) continue;
      if (!in_tile(gates[g].first)) tile.push_back(gates[g].first);
      if (!in_tile(gates[g].second)) tile.push_back(gates[g].second);
      sel.push_back(g);
    }
    if (sel.empty()) return QVS_EUNSUPPORTED;
    // pad the tile to 12 bits with the lowest free index bits
    for (int b = CHUNK; (int)tile.size() < TB && b < n; ++b)
      if (!in_tile(b)) tile.push_back(b);
    if ((int)tile.size() != TB) return QVS_EUNSUPPORTED;
    std::sort(tile.begin() + CHUNK, tile.end());
    Pass P{};
    for (int i = 0; i < TB; ++i) P.d.pos[i] = (uint8_t)tile[i];
    auto tbit = [&](int b) { return (int)(std::find(tile.begin(), tile.end(), b) - tile.begin()); };
    P.d.ngates = (int)sel.size();
    for (int i = 0; i < P.d.ngates; ++i) {
      const int ta = tbit(gates[sel[i]].first), tb = tbit(gates[sel[i]].second);
      P.d.ga[i] = (uint8_t)ta;
      P.d.gb[i] = (uint8_t)tb;
      // pair group k (= bits 8, 9 of the pair index) spread past the gate's two tile bits
      const int p1 = std::min(ta, tb), p2 = std::max(ta, tb);
      for (int k = 1; k < 4; ++k) {
        uint32_t x = (uint32_t)k << 8;
        x = ((x >> p1) << (p1 + 1)) | (x & ((1u << p1) - 1u));
        x = ((x >> p2) << (p2 + 1)) | (x & ((1u << p2) - 1u));
        P.d.goff[i][k - 1] = (uint16_t)swz(x);
      }
      P.d.goff[i][3] = (uint16_t)swz((1u << ta) | (1u << tb));
      done[sel[i]] = 1;
    }
    left -= (int)sel.size();
    // sweeps: consecutive gates two at a time (the order within the pass is kept)
    P.d.nsweeps = 0;
    auto combo_offsets = [&](int s, const int* cb, int nb) {
      for (int c = 0; c < (1 << nb); ++c) {
        uint32_t x = 0;
        for (int i = 0; i < nb; ++i)
          if ((c >> i) & 1) x |= 1u << cb[i];
        P.d.soff[s][c] = (uint16_t)swz(x);
      }
      int sorted[4];
      for (int i = 0; i < nb; ++i) sorted[i] = cb[i];
      std::sort(sorted, sorted + nb);
      for (int i = 0; i < 4; ++i) P.d.sbits[s][i] = (uint8_t)(i < nb ? sorted[i] : 0);
    };
    for (int g = 0; g < P.d.ngates;) {
      const int s = P.d.nsweeps++;
      P.d.sgate[s] = (uint8_t)g;
      if (g + 1 < P.d.ngates) {
        const int a1 = P.d.ga[g], b1 = P.d.gb[g], a2 = P.d.ga[g + 1], b2 = P.d.gb[g + 1];
        const int shared = (a1 == a2) + (a1 == b2) + (b1 == a2) + (b1 == b2);
        if (shared == 0) {
          const int cb[4] = {a1, b1, a2, b2};
          P.d.skind[s] = SW_DISJOINT;
          combo_offsets(s, cb, 4);
          g += 2;
          continue;
        }
        if (shared == 1) {
          const int sh = (a1 == a2 || a1 == b2) ? a1 : b1;
          const int o1 = sh == a1 ? b1 : a1, o2 = sh == a2 ? b2 : a2;
          const int cb[3] = {o1, sh, o2};
          P.d.skind[s] = SW_SHARED;
          combo_offsets(s, cb, 3);
          g += 2;
          continue;
        }
      }
      P.d.skind[s] = SW_ONE;   // last gate of an odd count, or a gate repeated on the same pair
      g += 1;
    }
    P.d.nnt = 0;
    for (int b = 0; b < n; ++b)
      if (!in_tile(b)) P.d.ntbit[P.d.nnt++] = (uint8_t)b;
    out.push_back(P);
  }
  return QVS_OK;
}

static int run(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
               double* dt) {
  const int n = h->n;
  if (h->precision != QVS_C64) return QVS_EUNSUPPORTED;
  std::vector<Pass> layer;
  QVS_TRY(plan_layer(n, layer));
  const int L = (int)layer.size();
  const int F = L * p;                       // forward passes
  const int64_t dim = h->dim;
  const uint32_t grid = (uint32_t)(dim >> TB);
  const size_t vb = sizeof(float2) * (size_t)dim;
  // stored pass outputs (every pass), lambda
  QVS_TRY(h->ckpt.ensure(vb * (size_t)(grad ? F : 1)));
  if (grad) QVS_TRY(h->lam.ensure(vb));
  // rows: 0 = E; per layer k: 1 + k = dgamma_k, 1 + p + k = dt_k; one row per reverse pass for dt
  const int nslots = 1 + 2 * p;
  const int nrows = 1 + p + F;
  QVS_TRY(h->part.ensure(sizeof(double) * (size_t)nrows * grid));
  QVS_TRY(h->res.ensure(sizeof(double) * nslots));
  std::vector<int> rowmap;   // each slot sums its rows (reduce_rows takes up to 3 rows per slot)
  // dt_k collects L rows: chain them through extra slots when L > 3 (summed on the host below)
  const int dt_groups = (L + 2) / 3;
  const int nout = grad ? (1 + p + p * dt_groups) : 1;
  rowmap.assign(3 * (size_t)nout, -1);
  rowmap[0] = 0;
  if (grad) {
    for (int k = 0; k < p; ++k) rowmap[3 * (1 + k)] = 1 + k;
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < L; ++j) rowmap[3 * (1 + p + k * dt_groups + j / 3) + (j % 3)] = 1 + p + k * L + j;
  }
  QVS_TRY(h->rowmap.ensure(sizeof(int) * rowmap.size()));
  QVS_TRY(h->res.ensure(sizeof(double) * (size_t)nout));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->rowmap.ptr, rowmap.data(), sizeof(int) * rowmap.size(), cudaMemcpyHostToDevice,
                               h->stream));
  float2* S = h->ckpt.as<float2>();
  auto stored = [&](int j) { return S + (size_t)(grad ? j : 0) * dim; };   // output of forward pass j
  int64_t launches = 0;
  const double c = 8.0, qb = 4.0;
  for (int k = 0; k < p; ++k) {
    for (int j = 0; j < L; ++j) {
      const int f = k * L + j;
      Args a{};
      a.d = layer[j].d;
      a.in = f == 0 ? (h->have_psi0 ? h->psi0.as<float2>() : nullptr) : stored(f - 1);
      a.out = stored(f);
      a.q = h->q.as<float>();
      a.c = (float)cos(2.0 * ts[k]);
      a.s = (float)sin(2.0 * ts[k]);
      a.has_phase = j == 0;
      if (j == 0) turns_split(gammas[k], &a.ph0, &a.ph1);
      a.init_amp = (float)(1.0 / sqrt((double)dim));
      cudaEvent_t e0;
      QVS_TRY(prof_begin(h, &e0));
      fwd_kernel<<<grid, NT, 0, h->stream>>>(a);
      QVS_CUDA_TRY(cudaGetLastError());
      QVS_TRY(prof_end(h, "parity_pass", (double)dim * ((a.in ? c : 0.0) + c + (j == 0 ? qb : 0.0)), e0));
      ++launches;
    }
  }
  float2* psiF = stored(F - 1);
  {
    cudaEvent_t e0;
    QVS_TRY(prof_begin(h, &e0));
    elam_kernel<<<grid, NT, 0, h->stream>>>(dim, psiF, h->q.as<float>(), grad ? h->lam.as<float2>() : nullptr,
                                            h->part.as<double>(), 0);
    QVS_CUDA_TRY(cudaGetLastError());
    QVS_TRY(prof_end(h, "parity_elam", (double)dim * (c + qb + (grad ? c : 0.0)), e0));
    ++launches;
  }
  if (grad) {
    const size_t rsm = 2 * (size_t)SLOTS * sizeof(float2);
    QVS_CUDA_TRY(cudaFuncSetAttribute(rev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    for (int f = F - 1; f >= 0; --f) {
      const int k = f / L, j = f % L;
      Args a{};
      a.d = layer[j].d;
      a.in = stored(f);
      a.lam_in = h->lam.as<float2>();
      a.lam_out = h->lam.as<float2>();
      a.q = h->q.as<float>();
      a.c = (float)cos(2.0 * ts[k]);
      a.s = (float)sin(2.0 * ts[k]);
      a.has_phase = j == 0;
      if (j == 0) turns_split(gammas[k], &a.ph0, &a.ph1);
      a.part = h->part.as<double>();
      a.row_t = 1 + p + f;
      a.row_g = 1 + k;
      cudaEvent_t e0;
      QVS_TRY(prof_begin(h, &e0));
      rev_kernel<<<grid, NT, rsm, h->stream>>>(a);
      QVS_CUDA_TRY(cudaGetLastError());
      QVS_TRY(prof_end(h, "parity_pass_adjoint", (double)dim * (3 * c + (j == 0 ? qb : 0.0)), e0));
      ++launches;
    }
  }
  {
    cudaEvent_t e0;
    QVS_TRY(prof_begin(h, &e0));
    QVS_TRY(reduce_rows(h, h->part.as<double>(), grid, h->rowmap.as<int>(), nout, h->res.as<double>()));
    QVS_TRY(prof_end(h, "reduce_rows", 8.0 * grid * nrows, e0));
    ++launches;
  }
  h->launches = launches;
  QVS_TRY(ensure_host_res(h, (nout + 1) / 2 + 1));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->host_res, h->res.ptr, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  QVS_TRY(prof_flush(h));
  *E = h->host_res[0];
  if (grad) {
    for (int k = 0; k < p; ++k) {
      dg[k] = h->host_res[1 + k];
      double s = 0.0;
      for (int gi = 0; gi < dt_groups; ++gi) s += h->host_res[1 + p + k * dt_groups + gi];
      dt[k] = s;
    }
  } else {
    // evolve: the final state is the last pass output
    QVS_TRY(h->psi.ensure(vb));
    QVS_CUDA_TRY(cudaMemcpyAsync(h->psi.ptr, psiF, vb, cudaMemcpyDeviceToDevice, h->stream));
    QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  return QVS_OK;
}

}  // namespace pr

int parity_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d) {
  if (h->precision != QVS_C64) return QVS_EUNSUPPORTED;
  if (d->n_qubits < pr::TB || d->n_qubits > 30 || h->n != d->n_qubits) return QVS_EINVAL;
  std::vector<pr::Pass> layer;
  return pr::plan_layer(h->n, layer);
}

int parity_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts) {
  double E = 0.0;
  QVS_TRY(pr::run(h, p, gammas, ts, false, &E, nullptr, nullptr));
  h->E = E;
  h->have_E = true;
  return QVS_OK;
}

int parity_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg, double* dt) {
  return pr::run(h, p, gammas, ts, true, E, dg, dt);
}

}  // namespace qvs

extern "C" int qvs_state_parity(int n_qubits, int A, void* dst, void* stream) {
  if (n_qubits < 2 || n_qubits > 30 || (n_qubits & 1) || A < 0 || A > n_qubits / 2 || !dst) return QVS_EINVAL;
  const double amp = pow(sqrt(0.5), (double)(n_qubits / 2 - A));
  qvs::pr::parity_state_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(n_qubits, A, amp, static_cast<float2*>(dst));
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

static_assert(qvs::pr::TB == QVS_PARITY_TILE_BITS && qvs::pr::MAXG == QVS_PARITY_MAX_GATES,
              "the plan layout of qvs_parity_plan");

extern "C" int qvs_parity_plan(int n_qubits, int max_passes, int* n_passes, int32_t* ngates, int32_t* tile_bits,
                               int32_t* gate_bits, int32_t* nsweeps, int32_t* sweep_kind, int32_t* sweep_first) {
  using namespace qvs::pr;
  if (!n_passes || n_qubits < TB || n_qubits > 30 || max_passes < 0) return QVS_EINVAL;
  std::vector<Pass> layer;
  QVS_TRY(plan_layer(n_qubits, layer));
  *n_passes = (int)layer.size();
  if (!ngates) return QVS_OK;   // size query
  if ((int)layer.size() > max_passes || !tile_bits || !gate_bits || !nsweeps || !sweep_kind || !sweep_first)
    return QVS_EINVAL;
  for (size_t i = 0; i < layer.size(); ++i) {
    const PassDesc& d = layer[i].d;
    ngates[i] = d.ngates;
    nsweeps[i] = d.nsweeps;
    for (int b = 0; b < TB; ++b) tile_bits[i * TB + b] = d.pos[b];
    for (int g = 0; g < MAXG; ++g) {
      const size_t k = i * MAXG + g;
      gate_bits[2 * k] = g < d.ngates ? d.pos[d.ga[g]] : -1;
      gate_bits[2 * k + 1] = g < d.ngates ? d.pos[d.gb[g]] : -1;
      sweep_kind[k] = g < d.nsweeps ? d.skind[g] : -1;
      sweep_first[k] = g < d.nsweeps ? d.sgate[g] : -1;
    }
  }
  return QVS_OK;
}
