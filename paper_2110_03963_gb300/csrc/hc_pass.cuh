// Tiled passes of the QAOA hypercube-mixer path (Sec. 2.3.1): the per-tile body shared by the
// one-CTA-per-tile kernels and the batched persistent kernel, and the per-pass kernel launchers.
// The complex64 launchers are instantiated once per rotation threshold TH in hc_pass_th*.cu.
#pragma once

#include <type_traits>

#include "hc_kernels.cuh"
#include "qvs_internal.h"

namespace qvs {
namespace hc {

constexpr int TH_NONE = TB;   // no "before" rotations, all tile bits "after" (single-tile schedules)
constexpr int TH_RUNTIME = -1;
constexpr int TH_RUNTIME_HI = -2;   // runtime masks within tile bits 4..11: the two-layout form

enum Shape : int {
  F0 = 0,   // first pass: psi0 (generated or loaded), phase, rotations ("after")
  F1 = 1,   // rotations (before), phase, rotations (after)
  F2 = 2,   // rotations only
  FE = 3,   // last forward pass fused with its adjoint: rotations, E and lambda = Q psi, undo
  FV = 4,   // last forward pass for qvs_evolve: rotations, E, store psi
  R1 = 5,   // adjoint of F1
  R2 = 6,   // adjoint of F2
  R0 = 7,   // adjoint of F0 (gradient contributions only)
  R1X = 8,  // R1 / R0 of an ex-QAOA layer: also store g(x) for the per-term gradients (runtime
  R0X = 9   // masks only)
};
__host__ __device__ constexpr int base_shape(int s) { return s == R1X ? R1 : (s == R0X ? R0 : s); }
__host__ __device__ constexpr bool two_vector(int s) {
  return base_shape(s) == FE || base_shape(s) == R1 || base_shape(s) == R2 || base_shape(s) == R0;
}

// Scalars of one pass. Rotations use the tangent form of the gauge (see hc_kernels.cuh): the
// kernels never see cos t'; every real factor of the frame reaches them as a scale.
template <class T>
struct PassArgs {
  Tile tile;
  const typename Cx<T>::t* psi_in;
  typename Cx<T>::t* psi_out;
  const typename Cx<T>::t* lam_in;
  typename Cx<T>::t* lam_out;
  const T* q;
  uint32_t mask_bef, mask_aft;
  uint32_t qx;          // q is read at index XOR qx (frame F = 1: 2^n - 1)
  T tb, ta;             // tan t' of the "before" and "after" layers' rotations
  T c2b, c2a;           // cos^2 t' of those layers (adjoint accumulation scale per undone bit)
  T ph0, ph1;           // phase: complex64: gamma/2pi as hi, lo; complex128: gamma, 0
  T rho_p, rho_l;       // real factors folded into the phase of psi and of lambda (renormalisation)
  T sc_b, sc_a;         // real scale of the first adjoint accumulation step, before / after layers
  T sc_g, sc_E;         // real scale of the gamma term and of E
  // plain output (FV): psi_{j ^ ox} = out_k i^(|j| - out_fm) W_j
  uint32_t ox, out_fm;
  T out_k;
  double* part;         // partial-sum rows: part[row * gridDim.x + blockIdx.x]
  int row_bef, row_aft, row_gam, row_E;
  T init_amp;           // amplitude of the uniform initial state
  int gen_init;         // F0: 1 = generate psi0 = init_amp, 0 = load psi_in (plain amplitudes)
  // Quadratic quality evaluated in the pass (qcta != NULL; q is then not read): tables of this
  // pass's tile type and frame (see qgen2)
  const int* qcta;      // per tile: [16] = {constant, linear coefficient of tile bits 0..11}
  const int* qthr;      // per thread: [8] = {pair sum of its own bits, cross sums of bits 5..8}
  int qpp[R];           // per register r: pair sum of register bits 5..8
  T qscale;             // 2^-F (quality) or 2^-32 (ex-QAOA phase angle in turns)
  // ex-QAOA adjoint phase passes: g(x) = 2 Im(conj(lambda) phi)(x) stored at the physical index
  // (the per-term gradients are its moments); NULL otherwise
  T* gout;
};

// ---------------------------------------------------------------- per-pass scalars (host and device)
//
// Layer k's rotation angle t_k is applied as t' = t_k (|tan t_k| <= 1) or t' = t_k - pi/2 (flip: the
// remaining (-i)^n X_all becomes a frame toggle). Frame of a buffer: state = k P^F W (gauge form).
struct LayerRot {
  double tn, cp;   // tan t', cos t'
  int flip;
};
__host__ __device__ inline LayerRot layer_rot(double t) {
  const double s = sin(t), c = cos(t);
  if (fabs(s) > fabs(c)) return {-c / s, s, 1};
  return {s / c, c, 0};
}
struct Frame {
  double k;
  int f;
};
// P applied (forward) / P^-1 = (-1)^n P applied (adjoint); P^2 = (-1)^n
__host__ __device__ inline void fwd_toggle(Frame& fr, int n) {
  if (fr.f && (n & 1)) fr.k = -fr.k;
  fr.f ^= 1;
}
__host__ __device__ inline void bwd_toggle(Frame& fr, int n) {
  if (!fr.f && (n & 1)) fr.k = -fr.k;
  fr.f ^= 1;
}
__host__ __device__ inline double ipow(double x, int m) {
  double r = 1.0;
  for (int i = 0; i < m; ++i) r *= x;
  return r;
}
__host__ __device__ inline uint32_t all_bits(int n) { return n >= 32 ? 0xffffffffu : ((1u << n) - 1u); }

template <class T>
__host__ __device__ inline void set_phase(PassArgs<T>& a, double gamma) {
  if constexpr (sizeof(T) == 4) {
    float hi, lo;
    turns_split(gamma, &hi, &lo);
    a.ph0 = hi;
    a.ph1 = lo;
  } else {
    a.ph0 = gamma;
    a.ph1 = 0.0;
  }
}

// Scalars of forward pass (shape, lb, la, lg) rotating G tile bits per layer; fr: the psi frame,
// advanced from the pass's input boundary to its output (FE: to its input again, after the fused
// undo); FE also sets lf, the frame of the lambda it writes.
template <class T>
__host__ __device__ inline void fwd_scalars(PassArgs<T>& a, int shape, int lb, int la, int lg, int G, int n,
                                            int p, const double* gammas, const double* ts, Frame& fr,
                                            Frame& lf) {
  if (lb >= 0) {
    const LayerRot r = layer_rot(ts[lb]);
    a.tb = (T)r.tn;
    a.c2b = (T)(r.cp * r.cp);
    fr.k *= ipow(r.cp, G);
  }
  if (lg >= 0) {
    if (lg >= 1 && layer_rot(ts[lg - 1]).flip) fwd_toggle(fr, n);
    a.qx = fr.f ? all_bits(n) : 0u;
    a.rho_p = (T)fr.k;
    fr.k = 1.0;
    set_phase(a, gammas[lg]);
  }
  if (la >= 0) {
    const LayerRot r = layer_rot(ts[la]);
    a.ta = (T)r.tn;
    fr.k *= ipow(r.cp, G);
  }
  if (shape == FE || shape == FV) {
    const LayerRot r = layer_rot(ts[p - 1]);
    if (r.flip) fwd_toggle(fr, n);
    a.qx = fr.f ? all_bits(n) : 0u;
    a.sc_E = (T)(fr.k * fr.k);
    if (shape == FV) {
      a.ox = a.qx;
      a.out_fm = fr.f ? (uint32_t)(n & 3) : 0u;
      a.out_k = (T)fr.k;
    } else {
      lf = fr;   // lambda = Q psi at the end point
      if (r.flip) {
        bwd_toggle(fr, n);
        bwd_toggle(lf, n);
      }
      if (lb >= 0) {   // the pass undoes its "before" rotations (none in single-tile schedules)
        a.sc_b = (T)(fr.k * lf.k);
        fr.k *= ipow(r.cp, G);
        lf.k *= ipow(r.cp, G);
      }
    }
  }
}

// Scalars of adjoint pass (shape R0 / R1 / R2 of forward pass lb, la, lg); pf / lf: psi / lambda
// frames, advanced from the pass's output boundary back to its input.
template <class T>
__host__ __device__ inline void bwd_scalars(PassArgs<T>& a, int shape, int lb, int la, int lg, int G, int n,
                                            const double* gammas, const double* ts, Frame& pf, Frame& lf) {
  if (la >= 0) {
    const LayerRot r = layer_rot(ts[la]);
    a.ta = (T)r.tn;
    a.c2a = (T)(r.cp * r.cp);
    a.sc_a = (T)(pf.k * lf.k);
    pf.k *= ipow(r.cp, G);
    lf.k *= ipow(r.cp, G);
  }
  if (lg >= 0) {
    a.qx = pf.f ? all_bits(n) : 0u;
    a.sc_g = (T)(pf.k * lf.k);
    set_phase(a, gammas[lg]);
    if (shape == R1) {
      a.rho_p = (T)pf.k;
      a.rho_l = (T)lf.k;
      pf.k = lf.k = 1.0;
      if (lg >= 1 && layer_rot(ts[lg - 1]).flip) {
        bwd_toggle(pf, n);
        bwd_toggle(lf, n);
      }
    }
  }
  if (lb >= 0) {
    const LayerRot r = layer_rot(ts[lb]);
    a.tb = (T)r.tn;
    a.c2b = (T)(r.cp * r.cp);
    a.sc_b = (T)(pf.k * lf.k);
    pf.k *= ipow(r.cp, G);
    lf.k *= ipow(r.cp, G);
  }
}

// Block sum of up to three values, written to their partial rows (rows < 0 skipped). Lanes are
// summed in the thread's precision (a warp holds 512 amplitude contributions), warps and CTAs in
// fp64; the order is fixed, so results are reproducible run to run.
template <class T>
__device__ __forceinline__ void block_store3(T a, T b, T c, double* part, int ra, int rb, int rc,
                                             int tid, uint32_t bid, uint32_t nblk) {
  __shared__ double red[3][NT / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = (double)a;
    red[1][tid >> 5] = (double)b;
    red[2][tid >> 5] = (double)c;
  }
  __syncthreads();
  if (tid < 3) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += red[tid][w];
    const int row = tid == 0 ? ra : (tid == 1 ? rb : rc);
    if (row >= 0) part[(size_t)row * nblk + bid] = s;
  }
}

// One tile (index bid of nblk) of one pass; the CTA's shared memory is smem_raw. Used by the
// per-pass kernels (one CTA per tile) and by the batched persistent kernel (a CTA walks the tiles).
// TH: rotated tile bits are those >= TH (TH_RUNTIME: the runtime masks a.mask_bef / a.mask_aft).
// TBF / TAF are the thresholds of the "before" / "after" rotations: both TH, except for TH_NONE
// (single-tile schedules, whose passes have no "before" rotations and rotate every tile bit after).
// ALT: the single-vector passes alternate two shared buffers (one barrier per transpose); the CTA
// must hold 2 * SM_SLOTS elements.
// q of the amplitudes a thread holds in layout 2 from a quadratic form (exact int32 sums).
// Index bits split into the tile's non-tile bits (fixed per CTA), the thread's own tile bits
// TT = {0..4, 9..11} and the register bits 5..8; with x = the bit values read at index XOR qx,
//   q = [c + non-tile terms] + sum_{k in TT} x_k L_k + K_T + sum_{i} x_{5+i} (L_{5+i} + K_i) + PP(r),
// L_k = h_k + sum_{non-tile j} J_kj x_j (per tile, s_q[1 + k]; s_q[0] = the bracket), K_T / K_i the
// pair sums within TT / between TT and register bit 5+i (per thread, qthr), PP(r) the pairs among
// the register bits (per register, qpp). Flipped bits (qx != 0) read x = 1 - bit.
template <class T>
__device__ __forceinline__ void qgen2(T (&qv)[R], const PassArgs<T>& a, const int* s_q, int tid) {
  // sums modulo 2^32 (exact for qualities, which stay below 2^30; ex-QAOA angles wrap by design)
  const uint32_t fl = a.qx ? 0xFFFu : 0u;
  const uint32_t xt = (uint32_t)tj<2>(0, tid) ^ fl;
  const int4 k0 = *reinterpret_cast<const int4*>(a.qthr + 8 * tid);
  const uint32_t k4 = (uint32_t)a.qthr[8 * tid + 4];
  uint32_t qT = (uint32_t)s_q[0] + (uint32_t)k0.x;
#pragma unroll
  for (int k = 0; k < TB; ++k)
    if (k < 5 || k > 8)
      if ((xt >> k) & 1u) qT += (uint32_t)s_q[1 + k];
  uint32_t cc[RB] = {(uint32_t)s_q[6] + (uint32_t)k0.y, (uint32_t)s_q[7] + (uint32_t)k0.z,
                     (uint32_t)s_q[8] + (uint32_t)k0.w, (uint32_t)s_q[9] + k4};
  if (fl) {
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      qT += cc[i];
      cc[i] = 0u - cc[i];
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    uint32_t v = qT + (uint32_t)a.qpp[r];
#pragma unroll
    for (int i = 0; i < RB; ++i)
      if ((r >> i) & 1) v += cc[i];
    qv[r] = (T)(int32_t)v * a.qscale;
  }
}

struct NoHook {
  __device__ void operator()() const {}
};

// STG: the tile's input vectors were landed densely in shared memory (stg: psi at [0, TILE), lambda
// at [TILE, 2 TILE), index = tile index) by the staged persistent kernel; the transposes then go
// through the single buffer sm, one vector at a time. Once every thread has read the stage (a
// barrier after the loads), consumed() runs, which lands the next tile there.
template <class T, int SHAPE, int TH, bool ALT = false, bool STG = false, class Fn = NoHook>
__device__ __forceinline__ void run_pass(const PassArgs<T>& a, uint32_t bid, uint32_t nblk,
                                         unsigned char* smem_raw, const typename Cx<T>::t* stg = nullptr,
                                         Fn consumed = Fn{}) {
  constexpr int S = base_shape(SHAPE);
  constexpr bool EXG = SHAPE != S;
  using C = typename Cx<T>::t;
  C* sm = reinterpret_cast<C*>(smem_raw);
  constexpr int TBF = TH == TH_NONE ? TH_NONE : TH;   // threshold of the "before" rotations
  constexpr int TAF = TH == TH_NONE ? 0 : TH;         // threshold of the "after" rotations
  auto x2 = [&](auto lf, auto lt, C(&p)[R], C(&l)[R]) {
    constexpr int LF = decltype(lf)::value, LT = decltype(lt)::value;
    if constexpr (STG) {
      xchg<LF, LT>(p, sm, threadIdx.x);
      xchg<LF, LT>(l, sm, threadIdx.x);
    } else {
      xchg2<LF, LT>(p, l, sm, threadIdx.x);
    }
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  // which: 0 = psi, 1 = lambda (the staged copy's half)
  auto ld = [&](auto li, C(&v)[R], int which, const C* g, uint32_t off) {
    constexpr int L = decltype(li)::value;
    if constexpr (STG) dget<L>(v, stg + which * TILE, threadIdx.x);
    else gload<L>(v, g, off, a.tile);
  };
  auto loaded = [&]() {
    if constexpr (STG) {
      __syncthreads();
      consumed();
    }
  };
  const int tid = threadIdx.x;
  const uint32_t base = tile_base(a.tile, bid);
  const uint32_t off0 = base + toff(a.tile, tj<0>(0, tid));
  const uint32_t off2 = base + toff(a.tile, tj<2>(0, tid));
  T qv[R];
  // quadratic quality (one-CTA-per-tile kernels only; the batched kernel reads vectors): this
  // tile's row of the table, published by the first barrier below
  __shared__ int s_q[16];
  if constexpr (!ALT) {
    if (a.qcta && tid < 13) s_q[tid] = a.qcta[16 * (size_t)bid + tid];
  }
  auto qget = [&]() {
    if constexpr (!ALT) {
      if (a.qcta) {
        qgen2<T>(qv, a, s_q, tid);
        return;
      }
    }
    qload<2>(qv, a.q, off2, a.tile, a.qx);
  };
  // the vector's loads can be issued early; the in-pass quadratic form needs its table row, which
  // the first barrier publishes
  auto qget_early = [&]() {
    if constexpr (!ALT) {
      if (a.qcta) return;
    }
    qload<2>(qv, a.q, off2, a.tile, a.qx);
  };
  auto qget_late = [&]() {
    if constexpr (!ALT) {
      if (a.qcta) qgen2<T>(qv, a, s_q, tid);
    }
  };
  // Passes whose rotated tile bits all lie in 4..11 (TH >= 4: every tile type but the contiguous
  // one) go through layouts L3 and L2 only: one transpose per direction instead of two.
  constexpr bool TWO = (TH >= 4 && TH < TB) || TH == TH_RUNTIME_HI;
  const uint32_t off3 = base + toff(a.tile, tj<3>(0, tid));
  using I3 = std::integral_constant<int, 3>;

  // v <- (rho exp(-+i gamma q)) v on the amplitudes of layout 2 (dir = +1 forward, -1 adjoint)
  auto phase2 = [&](C (&v)[R], T dir, T rho) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T c, s;
      phase_cs(qv[r], a.ph0, a.ph1, c, s);
      v[r] = phase_mul(v[r], rho * c, dir * rho * s);
    }
  };
  // the same phase on psi and lambda with their own scales (one sine/cosine per amplitude)
  auto phase2x2 = [&](C (&v)[R], C (&l)[R], T dir) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T c, s;
      phase_cs(qv[r], a.ph0, a.ph1, c, s);
      s *= dir;
      v[r] = phase_mul(v[r], a.rho_p * c, a.rho_p * s);
      l[r] = phase_mul(l[r], a.rho_l * c, a.rho_l * s);
    }
  };

  C v[R];
  if constexpr (S == F0 && TWO) {   // the high tile types: one transpose (L2 -> L3)
    const uint32_t tpop = __popc(base) + __popc(tj<2>(0, tid));
    if (a.gen_init) {
#pragma unroll
      for (int r = 0; r < R; ++r) {   // W_j = amp (-i)^|j|
        C w;
        w.x = a.init_amp;
        w.y = T(0);
        v[r] = mul_ipow(w, (0u - (tpop + (uint32_t)cpop(tj<2>(r, 0)))) & 3u);
      }
    } else {
      gload_plain<2>(v, a.psi_in, off2, a.tile, tpop);
    }
    if constexpr (!ALT) {
      if (a.qcta) __syncthreads();
    }
    qget();
    phase2(v, T(1), a.rho_p);
    rot_layout<2, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<2, 3, 0, ALT>(v, sm, tid);
    rot_layout<3, TAF>(v, a.mask_aft, a.ta);
    gstore<3>(v, a.psi_out, off3, a.tile);
  } else if constexpr (S == F0) {
    const uint32_t tpop = __popc(base) + __popc(tj<2>(0, tid));
    if (a.gen_init) {
#pragma unroll
      for (int r = 0; r < R; ++r) {   // W_j = amp (-i)^|j|
        C w;
        w.x = a.init_amp;
        w.y = T(0);
        v[r] = mul_ipow(w, (0u - (tpop + (uint32_t)cpop(tj<2>(r, 0)))) & 3u);
      }
    } else {
      gload_plain<2>(v, a.psi_in, off2, a.tile, tpop);
    }
    if constexpr (!ALT) {
      if (a.qcta) __syncthreads();
    }
    qget();
    phase2(v, T(1), a.rho_p);
    rot_layout<2, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<2, 1, 0, ALT>(v, sm, tid);
    rot_layout<1, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<1, 0, 1, ALT>(v, sm, tid);
    rot_layout<0, TAF>(v, a.mask_aft, a.ta);
    gstore<0>(v, a.psi_out, off0, a.tile);
  } else if constexpr (S == F1 && TWO) {
    ld(I3{}, v, 0, a.psi_in, off3);
    rot_layout<3, TBF>(v, a.mask_bef, a.tb);
    qget_early();
    xchg_alt<3, 2, 0, ALT>(v, sm, tid);
    qget_late();
    rot_layout<2, TBF>(v, a.mask_bef, a.tb);
    phase2(v, T(1), a.rho_p);
    rot_layout<2, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<2, 3, 1, ALT>(v, sm, tid);
    rot_layout<3, TAF>(v, a.mask_aft, a.ta);
    gstore<3>(v, a.psi_out, off3, a.tile);
  } else if constexpr (S == F1) {
    ld(I0{}, v, 0, a.psi_in, off0);
    rot_layout<0, TBF>(v, a.mask_bef, a.tb);
    xchg_alt<0, 1, 0, ALT>(v, sm, tid);
    rot_layout<1, TBF>(v, a.mask_bef, a.tb);
    qget();
    xchg_alt<1, 2, 1, ALT>(v, sm, tid);
    rot_layout<2, TBF>(v, a.mask_bef, a.tb);
    phase2(v, T(1), a.rho_p);
    rot_layout<2, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<2, 1, 0, ALT>(v, sm, tid);
    rot_layout<1, TAF>(v, a.mask_aft, a.ta);
    xchg_alt<1, 0, 1, ALT>(v, sm, tid);
    rot_layout<0, TAF>(v, a.mask_aft, a.ta);
    gstore<0>(v, a.psi_out, off0, a.tile);
  } else if constexpr (S == F2 && TWO) {
    ld(I3{}, v, 0, a.psi_in, off3);
    rot_layout<3, TBF>(v, a.mask_bef, a.tb);
    xchg_alt<3, 2, 0, ALT>(v, sm, tid);
    rot_layout<2, TBF>(v, a.mask_bef, a.tb);
    gstore<2>(v, a.psi_out, off2, a.tile);
  } else if constexpr (S == F2) {
    ld(I0{}, v, 0, a.psi_in, off0);
    rot_layout<0, TBF>(v, a.mask_bef, a.tb);
    xchg_alt<0, 1, 0, ALT>(v, sm, tid);
    rot_layout<1, TBF>(v, a.mask_bef, a.tb);
    xchg_alt<1, 2, 1, ALT>(v, sm, tid);
    rot_layout<2, TBF>(v, a.mask_bef, a.tb);
    gstore<2>(v, a.psi_out, off2, a.tile);
  } else if constexpr (S == FE || S == FV) {
    if constexpr (TWO) {
      ld(I3{}, v, 0, a.psi_in, off3);
      loaded();
      rot_layout<3, TBF>(v, a.mask_bef, a.tb);
      qget_early();
      if constexpr (S == FV) xchg_alt<3, 2, 0, ALT>(v, sm, tid);
      else xchg<3, 2>(v, sm, tid);   // FE's second half writes both buffers: keep the trailing barrier
      qget_late();
    } else {
      ld(I0{}, v, 0, a.psi_in, off0);
      loaded();
      rot_layout<0, TBF>(v, a.mask_bef, a.tb);
      if constexpr (S == FV) xchg_alt<0, 1, 0, ALT>(v, sm, tid);
      else xchg<0, 1>(v, sm, tid);   // FE's second half writes both buffers: keep the trailing barrier
      rot_layout<1, TBF>(v, a.mask_bef, a.tb);
      qget();
      if constexpr (S == FV) xchg_alt<1, 2, 1, ALT>(v, sm, tid);
      else xchg<1, 2>(v, sm, tid);
    }
    rot_layout<2, TBF>(v, a.mask_bef, a.tb);
    T e = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) e += qv[r] * (v[r].x * v[r].x + v[r].y * v[r].y);
    e *= a.sc_E;
    if constexpr (S == FV) {
      const uint32_t tpop = __popc(base) + __popc(tj<2>(0, tid));
      gstore_plain<2>(v, a.psi_out, off2, a.tile, tpop, a.ox, a.out_fm, a.out_k);
      block_store3(e, T(0), T(0), a.part, a.row_E, -1, -1, tid, bid, nblk);
    } else {
      C l[R];
#pragma unroll
      for (int r = 0; r < R; ++r) { l[r].x = qv[r] * v[r].x; l[r].y = qv[r] * v[r].y; }
      T acc = T(0), sc = a.sc_b;
      unrot_layout_acc<2, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc);
      if constexpr (TWO) {
        x2(I2{}, I3{}, v, l);
        unrot_layout_acc<3, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc);
        gstore<3>(l, a.lam_out, off3, a.tile);
      } else {
        x2(I2{}, I1{}, v, l);
        unrot_layout_acc<1, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc);
        x2(I1{}, I0{}, v, l);
        unrot_layout_acc<0, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc);
        gstore<0>(l, a.lam_out, off0, a.tile);
      }
      block_store3(e, T(2) * acc, T(0), a.part, a.row_E, a.row_bef, -1, tid, bid, nblk);
    }
  } else if constexpr (S == R1 || S == R0) {
    C l[R];
    T acc_a = T(0), acc_b = T(0), acc_g = T(0), sc = a.sc_a;
    if constexpr (TWO) {
      ld(I3{}, v, 0, a.psi_in, off3);
      ld(I3{}, l, 1, a.lam_in, off3);
      loaded();
      unrot_layout_acc<3, TAF>(v, l, a.mask_aft, a.ta, a.c2a, sc, acc_a);
      qget_early();
      x2(I3{}, I2{}, v, l);
      qget_late();
    } else {
      ld(I0{}, v, 0, a.psi_in, off0);
      ld(I0{}, l, 1, a.lam_in, off0);
      loaded();
      unrot_layout_acc<0, TAF>(v, l, a.mask_aft, a.ta, a.c2a, sc, acc_a);
      x2(I0{}, I1{}, v, l);
      unrot_layout_acc<1, TAF>(v, l, a.mask_aft, a.ta, a.c2a, sc, acc_a);
      qget();
      x2(I1{}, I2{}, v, l);
    }
    unrot_layout_acc<2, TAF>(v, l, a.mask_aft, a.ta, a.c2a, sc, acc_a);
#pragma unroll
    for (int r = 0; r < R; ++r) acc_g += qv[r] * imdot_st(l[r], v[r]);
    acc_g *= a.sc_g;
    if constexpr (EXG) {
      {
        uint32_t o[RB];
        reg_bit_offsets<2>(a.tile, o);
#pragma unroll
        for (int r = 0; r < R; ++r)
          a.gout[(off2 + reg_off(o, r)) ^ a.qx] = T(2) * a.sc_g * imdot_st(l[r], v[r]);
      }
    }
    if constexpr (S == R1) {
      phase2x2(v, l, T(-1));
      sc = a.sc_b;
      unrot_layout_acc<2, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
      if constexpr (TWO) {
        x2(I2{}, I3{}, v, l);
        unrot_layout_acc<3, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
        gstore<3>(l, a.lam_out, off3, a.tile);
        if (a.psi_out) gstore<3>(v, a.psi_out, off3, a.tile);
      } else {
        x2(I2{}, I1{}, v, l);
        unrot_layout_acc<1, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
        x2(I1{}, I0{}, v, l);
        unrot_layout_acc<0, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
        gstore<0>(l, a.lam_out, off0, a.tile);
        if (a.psi_out) gstore<0>(v, a.psi_out, off0, a.tile);
      }
    }
    block_store3(T(2) * acc_b, T(2) * acc_a, T(2) * acc_g, a.part, a.row_bef, a.row_aft, a.row_gam, tid, bid, nblk);
  } else if constexpr (S == R2) {
    C l[R];
    ld(I2{}, v, 0, a.psi_in, off2);
    ld(I2{}, l, 1, a.lam_in, off2);
    loaded();
    T acc_b = T(0), sc = a.sc_b;
    unrot_layout_acc<2, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
    if constexpr (TWO) {
      x2(I2{}, I3{}, v, l);
      unrot_layout_acc<3, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
      gstore<3>(l, a.lam_out, off3, a.tile);
      if (a.psi_out) gstore<3>(v, a.psi_out, off3, a.tile);
    } else {
      x2(I2{}, I1{}, v, l);
      unrot_layout_acc<1, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
      x2(I1{}, I0{}, v, l);
      unrot_layout_acc<0, TBF>(v, l, a.mask_bef, a.tb, a.c2b, sc, acc_b);
      gstore<0>(l, a.lam_out, off0, a.tile);
      if (a.psi_out) gstore<0>(v, a.psi_out, off0, a.tile);
    }
    block_store3(T(2) * acc_b, T(0), T(0), a.part, a.row_bef, -1, -1, tid, bid, nblk);
  }
}

// CTAs per SM the complex64 kernels are compiled for (register budget 65536 / (256 x CTAs)): the
// single-vector passes 4 (64 registers); the last forward pass FE 3 (80 registers, no spills: at
// n=28 1.41 -> 1.22 ms per launch); the adjoint passes 2 (128 registers: R2 at 3 spills and runs
// 1.47 -> 1.72 ms, R1 and R0 spill more).
template <class T, int SHAPE>
__host__ __device__ constexpr int ctas_per_sm() {
  return sizeof(T) == 8 ? 1 : (!two_vector(SHAPE) ? 4 : (SHAPE == FE ? 3 : 2));
}

template <class T, int SHAPE, int TH>
__global__ void __launch_bounds__(NT, ctas_per_sm<T, SHAPE>())
pass_kernel(const __grid_constant__ PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  run_pass<T, SHAPE, TH>(a, blockIdx.x, gridDim.x, smem_raw);
}

template <class T, int SHAPE, int TH>
static int launch_one(const PassArgs<T>& a, uint32_t grid, cudaStream_t st) {
  constexpr bool two = two_vector(SHAPE);
  const size_t sm = (two ? 2 : 1) * (size_t)SM_SLOTS * sizeof(typename Cx<T>::t);
  static std::atomic<uint64_t> configured{0};   // per instantiation: devices already set
  QVS_TRY(smem_limit_once(reinterpret_cast<const void*>(pass_kernel<T, SHAPE, TH>), configured, (int)sm));
  pass_kernel<T, SHAPE, TH><<<grid, NT, sm, st>>>(a);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

// one pass of the given shape over grid tiles, rotated bits >= TH
template <class T, int TH>
int launch_pass(int shape, const PassArgs<T>& a, uint32_t grid, cudaStream_t st) {
  switch (shape) {
    case F0: return launch_one<T, F0, TH>(a, grid, st);
    case F1: return launch_one<T, F1, TH>(a, grid, st);
    case F2: return launch_one<T, F2, TH>(a, grid, st);
    case FE: return launch_one<T, FE, TH>(a, grid, st);
    case FV: return launch_one<T, FV, TH>(a, grid, st);
    case R1: return launch_one<T, R1, TH>(a, grid, st);
    case R2: return launch_one<T, R2, TH>(a, grid, st);
    case R0: return launch_one<T, R0, TH>(a, grid, st);
    case R1X:
    case R0X:
      if constexpr (TH == TH_RUNTIME)
        return shape == R1X ? launch_one<T, R1X, TH>(a, grid, st) : launch_one<T, R0X, TH>(a, grid, st);
      return QVS_EINVAL;
  }
  return QVS_EINVAL;
}

// complex64 launchers are compiled in their own translation units (hc_pass_th*.cu)
#define QVS_HC_C64_THRESHOLDS(X) X(0) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(-1)
#define QVS_HC_EXTERN(K) extern template int launch_pass<float, K>(int, const PassArgs<float>&, uint32_t, cudaStream_t);
#ifndef QVS_HC_PASS_TU
QVS_HC_C64_THRESHOLDS(QVS_HC_EXTERN)
#endif
#undef QVS_HC_EXTERN

}  // namespace hc
}  // namespace qvs
