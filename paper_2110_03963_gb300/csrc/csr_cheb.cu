// QAOAz sparse-mixer path (Sec. 2.4.1, Sec. 3): exp(-i t W) v for a real symmetric CSR matrix W
// by a Chebyshev expansion,
//     exp(-i t W) v = e^{-i t a} sum_m (2 - delta_m0) (-i)^m J_m(b t) T_m(W~) v,  W~ = (W - a) / b,
// with [a - b, a + b] enclosing the spectrum (estimated by Lanczos when no bounds are given). The series is
// cut at the first K whose tail bound sum_{m > K} 2 |J_m(b t)| falls below the tolerance (the
// truncation error in the 2-norm is at most that bound since |T_m| <= 1 on [-1, 1]). Coefficients
// are computed in fp64 on the host; each term is one fused kernel: a CSR SpMV of T_m (one lane per
// row, up to 16 index loads in flight before their gathers, which L1/L2 serve), the three-term
// recurrence and the accumulation into y.
//
// Gradient: the subspace vectors are small (C(24,12) complex64 amplitudes = 21.6 MB), so every
// phi_k and psi_k of the forward sweep is stored and the adjoint sweep moves only lambda:
//   df/dt_k     = 2 Im <lambda_k | W psi_k>      (one SpMV fused with the inner product)
//   df/dgamma_k = 2 Im <M_k^dag lambda_k | Q phi_k>.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "qvs_internal.h"

namespace qvs {
namespace cs {

constexpr int NT = 256;
constexpr int LPR = 1;                 // lanes per row
constexpr int ROWS_PER_CTA = NT / LPR;
constexpr int RED_GRID = 152 * 8;      // CTAs of the elementwise/reduction kernels

struct StepArgs {
  int64_t dim;
  const uint32_t* rowptr;
  const int32_t* colind;
  const float* values;        // NULL = implicit value
  float implicit_value;
  float inv_b, a_over_b;      // W~ = W / b - a / b
  float alpha, beta;          // T_next = alpha W~ T_cur - beta T_prev
  float2 c, c_lo;             // coefficient of T_next added to y: the fp64 value as hi + lo floats
  const float2* tcur;
  const float2* tprev;        // may be NULL when beta == 0
  float2* tnext;
  float2* y;                  // y += c * T_next
  int y_init;                 // 1: y = c0 * tcur + c * tnext (first term folded in)
  float2 c0, c0_lo;
};

// c * t for an fp64 coefficient carried as the float pair c_hi + c_lo (c_hi = float(c), c_lo =
// float(c - c_hi): the coefficient to about 2^-48 relative): both products in fp32, summed, so
// only the product is rounded to single precision, not the coefficient
__device__ __forceinline__ float2 cmul_ff(float2 chi, float2 clo, float2 t) {
  const float2 h = make_float2(fmaf(chi.x, t.x, -chi.y * t.y), fmaf(chi.x, t.y, chi.y * t.x));
  const float2 l = make_float2(fmaf(clo.x, t.x, -clo.y * t.y), fmaf(clo.x, t.y, clo.y * t.x));
  return make_float2(h.x + l.x, h.y + l.y);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// sum over the row's nonzeros of value * x[col], by LPR lanes. Every lane of the warp must call
// it (the lane sum uses full-warp shuffles); lanes past the last row pass valid = false. Each
// lane issues the index loads of up to UNR nonzeros before their gathers, so the
// row pointer -> column index -> vector chain is paid once per UNR*LPR nonzeros. The step is bound
// by that chain's latency, so the number of rows in flight is what matters: one lane per row with
// 16 loads in flight ran the C(24,12) step in 75 us, against 82 us at 2 lanes x 8 and 104 us at
// 4 lanes x 4.
constexpr int UNR = 16;

__device__ __forceinline__ float2 row_spmv(const uint32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                           const float* __restrict__ values, float iv,
                                           const float2* __restrict__ x, int64_t row, int lane, bool valid) {
  float2 acc = make_float2(0.f, 0.f);
  uint32_t b = 0, e = 0;
  if (valid) {
    b = __ldg(rowptr + row);
    e = __ldg(rowptr + row + 1);
  }
  for (uint32_t j0 = b + lane; j0 < e; j0 += UNR * LPR) {
    int32_t c[UNR];
    float v[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const uint32_t j = j0 + u * LPR;
      const bool in = j < e;
      c[u] = in ? __ldcs(colind + j) : -1;
      v[u] = in ? (values ? __ldcs(values + j) : iv) : 0.f;
    }
    float2 t[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) t[u] = c[u] >= 0 ? __ldg(x + c[u]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      acc.x = fmaf(v[u], t[u].x, acc.x);
      acc.y = fmaf(v[u], t[u].y, acc.y);
    }
  }
#pragma unroll
  for (int o = LPR / 2; o; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  return acc;
}

// The sparse operator W, applied one row at a time.
//
// CsrOp: an explicit CSR matrix (row_spmv above).
// XyRingOp: the XY ring sum_a (X_a X_{a+1} + Y_a Y_{a+1}) (a + 1 mod n) on the n-bit basis states of
// Hamming weight k in increasing order (the matrix qvs_xy_ring_csr writes), generated from the row's
// state bits instead of read: (XX + YY) maps |01> to 2 |10> on a pair of differing bits, and the
// rank of a weight-k state with set bits c_1 < ... < c_k in increasing order is sum_i C(c_i, i).
// Moving the set bit at position b (p of the set bits lie below it) to the free position b + 1
// changes the rank by +C(b, p) (Pascal's rule); moving it from b + 1 down to a free b changes it by
// -C(b, p). The ring's closing pair (bits 0 and n-1) moves the lowest set bit to the top or the
// highest to the bottom, which renumbers every set bit; that neighbour's rank is summed afresh once,
// when the mixer is set.
struct CsrOp {
  const uint32_t* rowptr;
  const int32_t* colind;
  const float* values;
  float iv;
  __device__ __forceinline__ float2 apply(const float2* __restrict__ x, int64_t row, int lane, bool valid) const {
    return row_spmv(rowptr, colind, values, iv, x, row, lane, valid);
  }
  __device__ __forceinline__ double apply_d(const double* __restrict__ x, int64_t r) const {
    double acc = 0.0;
    for (uint32_t j = rowptr[r]; j < rowptr[r + 1]; ++j) acc += (double)(values ? values[j] : iv) * x[colind[j]];
    return acc;
  }
};

constexpr int XY_BW = 33;   // binomial table row width: C(b, j) at binom[b * XY_BW + j], b, j <= 32

struct XyRingOp {
  const uint2* rows;        // per row: basis state, row of the closing-pair neighbour (-1: none)
  const int32_t* binom;     // C(b, j), b <= n, j <= k
  int n, k;
  // Row indices and rank steps are 32-bit: the largest space allowed, C(31, 15), is below 2^31.
  // The closing pair (bits 0 and n-1) moves the lowest set bit to the top or the highest to the
  // bottom, which renumbers every set bit; that neighbour's row is computed once, on the host, when
  // the mixer is set, and read with the state.
  template <class F>
  __device__ __forceinline__ void neighbours(uint2 rw, int32_t row, F&& visit) const {
    const uint32_t s = rw.x;
    uint32_t d = (s ^ (s >> 1)) & ((1u << (n - 1)) - 1u);   // bit b: bits b and b + 1 differ
    while (d) {
      const int b = __ffs(d) - 1;
      d &= d - 1u;
      const int32_t step = __ldg(binom + (b * XY_BW + __popc(s & ((1u << b) - 1u))));
      visit(((s >> b) & 1u) ? row + step : row - step);
    }
    if ((int32_t)rw.y >= 0) visit((int32_t)rw.y);
  }
  // the same neighbours in groups of 8 adjacent pairs: each group's ranks first, then its gathers,
  // so up to 8 loads are in flight instead of one per dependent step
  __device__ __forceinline__ float2 gather_sum(const float2* __restrict__ x, uint2 rw, int32_t row) const {
    const uint32_t s = rw.x;
    float2 acc = make_float2(0.f, 0.f);
    const uint32_t d = (s ^ (s >> 1)) & ((1u << (n - 1)) - 1u);
#pragma unroll
    for (int g = 0; g < 32; g += 8) {
      if ((d >> g) == 0u) break;
      int32_t nb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = g + u;
        const int32_t step = ((d >> b) & 1u) ? __ldg(binom + (b * XY_BW + __popc(s & ((1u << b) - 1u)))) : 0;
        nb[u] = ((s >> b) & 1u) ? row + step : row - step;
      }
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = ((d >> (g + u)) & 1u) ? __ldg(x + nb[u]) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = __fadd2_rn(acc, v[u]);
    }
    if ((int32_t)rw.y >= 0) acc = __fadd2_rn(acc, __ldg(x + (int32_t)rw.y));
    return acc;
  }
  __device__ __forceinline__ float2 apply(const float2* __restrict__ x, int64_t row, int, bool valid) const {
    if (!valid) return make_float2(0.f, 0.f);
    const float2 acc = gather_sum(x, __ldg(rows + row), (int32_t)row);
    return make_float2(2.f * acc.x, 2.f * acc.y);
  }
  __device__ __forceinline__ double apply_d(const double* __restrict__ x, int64_t r) const {
    double acc = 0.0;
    neighbours(rows[r], (int32_t)r, [&](int32_t nb) { acc += x[nb]; });
    return 2.0 * acc;
  }
};

// The operator is a __grid_constant__ parameter: read in place, not copied into registers (a copied
// CSR operator doubled the step's registers to 64 and halved the rows in flight that bound it).
template <class Op>
__global__ void __launch_bounds__(NT) cheb_step_kernel(const __grid_constant__ StepArgs a,
                                                       const __grid_constant__ Op op) {
  const int lane = threadIdx.x & (LPR - 1);
  const int64_t row = (int64_t)blockIdx.x * ROWS_PER_CTA + (threadIdx.x / LPR);
  const bool valid = row < a.dim;
  const float2 wx = op.apply(a.tcur, row, lane, valid);
  if (lane != 0 || !valid) return;
  const float2 tc = a.tcur[row];
  // W~ x = (W x) / b - (a / b) x
  float2 t = make_float2(a.alpha * (wx.x * a.inv_b - a.a_over_b * tc.x),
                         a.alpha * (wx.y * a.inv_b - a.a_over_b * tc.y));
  if (a.tprev) {
    const float2 tp = a.tprev[row];
    t.x -= a.beta * tp.x;
    t.y -= a.beta * tp.y;
  }
  a.tnext[row] = t;
  const float2 ct = cmul_ff(a.c, a.c_lo, t);
  if (a.y_init) {
    const float2 c0 = cmul_ff(a.c0, a.c0_lo, tc);
    a.y[row] = make_float2(c0.x + ct.x, c0.y + ct.y);
  } else {
    const float2 yo = a.y[row];
    a.y[row] = make_float2(yo.x + ct.x, yo.y + ct.y);
  }
}

// y = c0 * x (a single-term series, bt == 0); c0 as an fp64 value split into hi + lo floats
__global__ void scale_kernel(int64_t dim, float2 c0, float2 c0_lo, const float2* __restrict__ x,
                             float2* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cmul_ff(c0, c0_lo, x[i]);
}

// fractional turns of gamma q (gamma / 2pi as float-float, q exact in fp32)
__device__ __forceinline__ void phase_cs(float q, float gh, float gl, float& c, float& s) {
  const float p = gh * q;
  const float e = fmaf(gh, q, -p) + gl * q;
  __sincosf(6.28318530717958647692f * ((p - rintf(p)) + e), &s, &c);
}

__device__ __forceinline__ void block_store(float v, double scale, double* part, int row) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    part[(size_t)row * gridDim.x + blockIdx.x] = scale * s;
  }
}

enum EwMode : int { PH_FWD = 0, PH_REV = 1, E_LAM = 2, E_ONLY = 3 };

struct EwArgs {
  int64_t dim;
  const float* q;
  const float2* in;       // PH_FWD: psi; PH_REV: phi (stored); E_*: psi
  float2* out;            // PH_FWD: phi; PH_REV: lambda (in place); E_LAM: lambda
  float gh, gl;
  float init_amp;         // PH_FWD with in == NULL: uniform psi0
  double* part;
  int row;
};

template <int MODE>
__global__ void __launch_bounds__(NT) ew_kernel(const __grid_constant__ EwArgs a) {
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < a.dim; i += (int64_t)gridDim.x * NT) {
    const float q = a.q[i];
    if constexpr (MODE == PH_FWD) {
      const float2 v = a.in ? a.in[i] : make_float2(a.init_amp, 0.f);
      float c, s;
      phase_cs(q, a.gh, a.gl, c, s);
      a.out[i] = make_float2(c * v.x + s * v.y, c * v.y - s * v.x);
    } else if constexpr (MODE == PH_REV) {
      const float2 ph = a.in[i];
      const float2 l = a.out[i];
      acc += q * (l.x * ph.y - l.y * ph.x);
      float c, s;
      phase_cs(q, a.gh, a.gl, c, s);
      a.out[i] = make_float2(c * l.x - s * l.y, c * l.y + s * l.x);
    } else {
      const float2 v = a.in[i];
      acc += q * (v.x * v.x + v.y * v.y);
      if constexpr (MODE == E_LAM) a.out[i] = make_float2(q * v.x, q * v.y);
    }
  }
  if constexpr (MODE != PH_FWD) block_store(acc, MODE == PH_REV ? 2.0 : 1.0, a.part, a.row);
}

// df/dt partial: 2 Im sum_row conj(lambda_row) (W psi)_row
template <class Op>
__global__ void __launch_bounds__(NT) dt_kernel(int64_t dim, const __grid_constant__ Op op, const float2* __restrict__ psi,
                                                const float2* __restrict__ lam, double* part, int prow,
                                                int nchunks) {
  const int lane = threadIdx.x & (LPR - 1);
  float acc = 0.f;
  // CTA b handles row blocks b, b + gridDim.x, ...
  for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t row = (int64_t)chunk * ROWS_PER_CTA + (threadIdx.x / LPR);
    const bool valid = row < dim;
    const float2 wx = op.apply(psi, row, lane, valid);
    if (lane == 0 && valid) {
      const float2 l = lam[row];
      acc += l.x * wx.y - l.y * wx.x;
    }
  }
  block_store(acc, 2.0, part, prow);
}

__global__ void gershgorin_kernel(int64_t dim, const uint32_t* rowptr, const float* values, float iv,
                                  unsigned int* out_bits) {
  float m = 0.f;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (uint32_t j = rowptr[r]; j < rowptr[r + 1]; ++j) s += fabsf(values ? values[j] : iv);
    m = fmaxf(m, s);
  }
  atomicMax(out_bits, __float_as_uint(m));   // non-negative floats order like their bit patterns
}

__global__ void rowptr32_kernel(int64_t n1, const int64_t* __restrict__ in, uint32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)in[i];
}

// ---------------------------------------------------------------- spectral interval (Lanczos)
//
// A few dozen Lanczos steps in fp64 on the device give Ritz values inside the spectrum whose
// extremes converge to the extreme eigenvalues first; their residuals bound how far an eigenvalue
// lies from them. The interval used is the extreme Ritz values widened by those residuals and by 1 %
// of the width, capped by the Gershgorin interval (which always encloses the spectrum).

template <class Op>
__global__ void lz_spmv_kernel(int64_t dim, const __grid_constant__ Op op, const double* __restrict__ x,
                               double* __restrict__ y) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = op.apply_d(x, r);
}

// the CTA's partial sum into out[blockIdx.x] (the host adds the partials in a fixed order, so the
// interval does not depend on the order in which CTAs finish)
__device__ __forceinline__ void lz_block_add(double v, double* out) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < NT / 32; ++w) sum += red[w];
    out[blockIdx.x] = sum;
  }
}

// out[CTA] = partial sums of a . b
__global__ void __launch_bounds__(NT) lz_dot_kernel(int64_t dim, const double* __restrict__ a,
                                                    const double* __restrict__ b, double* out) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  lz_block_add(acc, out);
}

// w -= alpha v + beta vprev; out[CTA] = partial sums of |w|^2
__global__ void __launch_bounds__(NT) lz_update_kernel(int64_t dim, double alpha, double beta,
                                                       const double* __restrict__ v, const double* __restrict__ vprev,
                                                       double* __restrict__ w, double* out) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[i] - alpha * v[i] - beta * vprev[i];
    w[i] = x;
    acc += x * x;
  }
  lz_block_add(acc, out);
}

// y = s x, also in place (y may be x, so neither pointer is restrict-qualified)
__global__ void lz_scale_kernel(int64_t dim, double s, const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

// deterministic start vector: entries from a 64-bit mix of the index, in [-1, 1)
__global__ void lz_start_kernel(int64_t dim, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x2110039630ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x (Sturm sequence)
static int sturm_below(const std::vector<double>& al, const std::vector<double>& be, double x) {
  int c = 0;
  double d = 1.0;
  for (size_t i = 0; i < al.size(); ++i) {
    const double b2 = i ? be[i - 1] * be[i - 1] : 0.0;
    d = al[i] - x - (i ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++c;
  }
  return c;
}

// k-th smallest eigenvalue (0-based) of the tridiagonal, by bisection
static double tri_eig(const std::vector<double>& al, const std::vector<double>& be, int k) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < al.size(); ++i) {
    const double r = (i ? fabs(be[i - 1]) : 0.0) + (i + 1 < al.size() ? fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, fabs(hi) + fabs(lo)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(al, be, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of the tridiagonal for eigenvalue th (inverse iteration)
static double tri_last_component(const std::vector<double>& al, const std::vector<double>& be, double th) {
  const size_t k = al.size();
  std::vector<double> x(k, 1.0), c(k), d(k), y(k);
  const double shift = th + 1e-10 * std::max(1.0, fabs(th));
  for (int it = 0; it < 3; ++it) {
    // solve (T - shift) y = x by the Thomas algorithm
    for (size_t i = 0; i < k; ++i) {
      const double a = i ? be[i - 1] : 0.0;
      double m = al[i] - shift - (i ? a * c[i - 1] : 0.0);
      if (fabs(m) < 1e-300) m = 1e-300;
      c[i] = (i + 1 < k ? be[i] : 0.0) / m;
      d[i] = (x[i] - (i ? a * d[i - 1] : 0.0)) / m;
    }
    for (size_t i = k; i-- > 0;) y[i] = d[i] - (i + 1 < k ? c[i] * y[i + 1] : 0.0);
    double nrm = 0.0;
    for (double v : y) nrm += v * v;
    nrm = sqrt(nrm);
    for (size_t i = 0; i < k; ++i) x[i] = y[i] / nrm;
  }
  return fabs(x[k - 1]);
}

static CsrOp make_csr_op(const CsrData& C) {
  return CsrOp{C.rowptr.as<uint32_t>(), C.colind.as<int32_t>(), C.has_values ? C.values.as<float>() : nullptr,
               C.implicit_value};
}
static XyRingOp make_xy_op(const CsrData& C) {
  return XyRingOp{C.states.as<uint2>(), C.binom.as<int32_t>(), C.xy_n, C.xy_k};
}
// f(op) with the handle's operator type
template <class F>
static int with_op(const CsrData& C, F&& f) {
  if (C.xy) return f(make_xy_op(C));
  return f(make_csr_op(C));
}

static int lanczos_interval(qvs_ctx* h, int iters, double gersh, double* lo, double* hi) {
  const int64_t dim = h->dim;
  CsrData& C = h->csr;
  DevBuf buf;   // freed on every return (cudaFree waits for the kernels that use it)
  struct Release {
    DevBuf& b;
    ~Release() { b.release(); }
  } release{buf};
  QVS_TRY(buf.ensure(sizeof(double) * (3 * (size_t)dim + RED_GRID)));
  double* v = buf.as<double>();
  double* vp = v + dim;
  double* w = vp + dim;
  double* sc = w + dim;   // one partial sum per CTA of the reduction kernels
  cudaStream_t st = h->stream;
  std::vector<double> parts(RED_GRID);
  auto scalar = [&](double* out) -> int {
    QVS_CUDA_TRY(cudaMemcpyAsync(parts.data(), sc, sizeof(double) * RED_GRID, cudaMemcpyDeviceToHost, st));
    QVS_CUDA_TRY(cudaStreamSynchronize(st));
    double sum = 0.0;
    for (double x : parts) sum += x;
    *out = sum;
    return QVS_OK;
  };
  lz_start_kernel<<<RED_GRID, NT, 0, st>>>(dim, v);
  QVS_CUDA_TRY(cudaMemsetAsync(vp, 0, sizeof(double) * dim, st));
  lz_dot_kernel<<<RED_GRID, NT, 0, st>>>(dim, v, v, sc);
  QVS_CUDA_TRY(cudaGetLastError());
  double n2 = 0.0;
  QVS_TRY(scalar(&n2));
  if (!(n2 > 0.0)) return QVS_ENUMERIC;
  lz_scale_kernel<<<RED_GRID, NT, 0, st>>>(dim, 1.0 / sqrt(n2), v, v);
  std::vector<double> al, be;
  double beta = 0.0;
  const int kmax = (int)std::min<int64_t>(iters, dim);
  for (int j = 0; j < kmax; ++j) {
    QVS_TRY(with_op(C, [&](auto op) -> int {
      lz_spmv_kernel<<<RED_GRID, NT, 0, st>>>(dim, op, v, w);
      return QVS_OK;
    }));
    lz_dot_kernel<<<RED_GRID, NT, 0, st>>>(dim, v, w, sc);
    QVS_CUDA_TRY(cudaGetLastError());
    double alpha = 0.0;
    QVS_TRY(scalar(&alpha));
    al.push_back(alpha);
    lz_update_kernel<<<RED_GRID, NT, 0, st>>>(dim, alpha, beta, v, vp, w, sc);
    QVS_CUDA_TRY(cudaGetLastError());
    double b2 = 0.0;
    QVS_TRY(scalar(&b2));
    beta = sqrt(std::max(b2, 0.0));
    if (beta <= 1e-12 * (fabs(alpha) + gersh + 1e-300)) break;   // invariant subspace: T is exact
    be.push_back(beta);
    std::swap(vp, v);                                             // vprev <- v
    lz_scale_kernel<<<RED_GRID, NT, 0, st>>>(dim, 1.0 / beta, w, v);   // v <- w / beta
    QVS_CUDA_TRY(cudaGetLastError());
  }
  const int k = (int)al.size();
  be.resize(k - 1 > 0 ? k - 1 : 0);
  const double tlo = tri_eig(al, be, 0), thi = tri_eig(al, be, k - 1);
  const double rlast = (int)be.size() < k ? beta : 0.0;   // beta_k: residual factor of every Ritz pair
  const double rlo = rlast * tri_last_component(al, be, tlo);
  const double rhi = rlast * tri_last_component(al, be, thi);
  const double width = thi - tlo;
  *lo = std::max(-gersh, tlo - rlo - 0.01 * width);
  *hi = std::min(gersh, thi + rhi + 0.01 * width);
  if (!(*hi > *lo)) {
    *lo = -gersh;
    *hi = gersh;
  }
  return QVS_OK;
}

// ---------------------------------------------------------------- host side

// an fp64 complex value as hi + lo float pairs (hi = nearest float, lo = nearest float of the rest)
static void split_ff(double re, double im, float2* hi, float2* lo) {
  const float hr = (float)re, hi_ = (float)im;
  *hi = make_float2(hr, hi_);
  *lo = make_float2((float)(re - (double)hr), (float)(im - (double)hi_));
}

// Chebyshev coefficients c_m = (2 - delta_m0) (-i)^m J_m(b t) e^{-i t a}, cut where the tail bound
// sum_{m > K} 2 |J_m(b t)| < tol. Returns K + 1 coefficients, or an empty vector if none fits.
static std::vector<double> cheb_coeffs(double a, double b, double t, double tol, int kmax, double* tail_out) {
  const double x = b * t;
  const double ax = fabs(x);
  const int mmax = (int)std::min<double>(kmax + 64.0, ax + 60.0 + 8.0 * std::cbrt(ax + 1.0));
  std::vector<double> J(mmax + 1);
  for (int m = 0; m <= mmax; ++m) J[m] = std::cyl_bessel_j((double)m, ax) * ((x < 0 && (m & 1)) ? -1.0 : 1.0);
  // tail sums
  std::vector<double> tail(mmax + 2, 0.0);
  for (int m = mmax; m >= 0; --m) tail[m] = tail[m + 1] + 2.0 * fabs(J[m]);
  int K = -1;
  for (int m = 0; m < mmax; ++m)
    if (tail[m + 1] < tol) { K = m; break; }
  if (K < 0 || K > kmax) return {};
  if (tail_out) *tail_out = tail[K + 1];
  std::vector<double> c(2 * (size_t)(K + 1));
  const double ca = cos(t * a), sa = -sin(t * a);   // e^{-i t a}
  for (int m = 0; m <= K; ++m) {
    const double w = (m == 0 ? 1.0 : 2.0) * J[m];
    // (-i)^m
    double re, im;
    switch (m & 3) {
      case 0: re = w; im = 0; break;
      case 1: re = 0; im = -w; break;
      case 2: re = -w; im = 0; break;
      default: re = 0; im = w; break;
    }
    c[2 * m] = re * ca - im * sa;
    c[2 * m + 1] = re * sa + im * ca;
  }
  return c;
}

}  // namespace cs
}  // namespace qvs

extern "C" int qvs_chebyshev_coefficients(double a, double b, double t, double tol, int max_terms, double* c,
                                          int* n_terms, double* tail) {
  if (!n_terms || !isfinite(a) || !isfinite(b) || !isfinite(t) || !(b >= 0.0) || !(tol > 0.0) ||
      max_terms < 1 || max_terms > 20000)
    return QVS_EINVAL;
  double tl = 0.0;
  const std::vector<double> v = qvs::cs::cheb_coeffs(a, b, t, tol, max_terms - 1, &tl);
  if (v.empty()) return QVS_ENUMERIC;
  *n_terms = (int)(v.size() / 2);
  if (tail) *tail = tl;
  if (c) memcpy(c, v.data(), sizeof(double) * v.size());
  return QVS_OK;
}

namespace qvs {
namespace cs {

static int launch_prof(qvs_ctx* h, const char* name, double bytes, int64_t& launches,
                       const std::function<void()>& fn) {
  cudaEvent_t e0;
  QVS_TRY(prof_begin(h, &e0));
  fn();
  QVS_CUDA_TRY(cudaGetLastError());
  ++launches;
  return prof_end(h, name, bytes, e0);
}

// y = exp(-i t W) x (sign = +1) or exp(+i t W) x (sign = -1); uses three scratch vectors.
static int expmv(qvs_ctx* h, double t, const float2* x, float2* y, float2* s0, float2* s1, float2* s2,
                 int64_t& launches) {
  const int64_t dim = h->dim;
  const CsrData& C = h->csr;
  const double a = 0.5 * (C.spec_hi + C.spec_lo), b = 0.5 * (C.spec_hi - C.spec_lo);
  double tail = 0.0;
  const std::vector<double> c = cheb_coeffs(a, b, t, C.tol, 20000, &tail);
  if (c.empty()) return QVS_ENUMERIC;
  const int K = (int)(c.size() / 2) - 1;
  const uint32_t grid = (uint32_t)((dim + ROWS_PER_CTA - 1) / ROWS_PER_CTA);
  const double nnz = (double)C.nnz;
  // compulsory bytes per series term: the operator's index data (the CSR arrays, or one 8-byte
  // record per row: the state word and the closing-pair neighbour's rank), T_cur's own row, T_prev,
  // T_next and y (the neighbour gathers of T_cur hit in L2)
  const double step_bytes = C.xy ? (double)dim * (8.0 + 8 + 8 + 8 + 16)
                                 : nnz * 4.0 + (C.has_values ? nnz * 4.0 : 0.0) + (double)dim * (4.0 + 8 + 8 + 8 + 16);
  if (K == 0) {
    return launch_prof(h, "csr_scale", 16.0 * dim, launches, [&] {
      float2 c0, c0_lo;
      split_ff(c[0], c[1], &c0, &c0_lo);
      scale_kernel<<<RED_GRID, NT, 0, h->stream>>>(dim, c0, c0_lo, x, y);
    });
  }
  StepArgs s{};
  s.dim = dim;
  s.inv_b = (float)(1.0 / b);
  s.a_over_b = (float)(a / b);
  // T_0 = x, T_1 = W~ x, y = c0 T_0 + c1 T_1
  float2* bufs[3] = {s0, s1, s2};
  const float2* tprev = nullptr;
  const float2* tcur = x;
  for (int m = 1; m <= K; ++m) {
    float2* tnext = bufs[m % 3];
    if (tnext == tcur || tnext == tprev) tnext = bufs[(m + 1) % 3];
    s.alpha = m == 1 ? 1.f : 2.f;
    s.beta = m == 1 ? 0.f : 1.f;
    s.tcur = tcur;
    s.tprev = m == 1 ? nullptr : tprev;
    s.tnext = tnext;
    s.y = y;
    split_ff(c[2 * m], c[2 * m + 1], &s.c, &s.c_lo);
    s.y_init = m == 1 ? 1 : 0;
    split_ff(c[0], c[1], &s.c0, &s.c0_lo);
    QVS_TRY(launch_prof(h, C.xy ? "xy_cheb_step" : "csr_cheb_step", step_bytes, launches, [&] {
      with_op(C, [&](auto op) -> int {
        cheb_step_kernel<<<grid, NT, 0, h->stream>>>(s, op);
        return QVS_OK;
      });
    }));
    tprev = tcur;
    tcur = tnext;
  }
  return QVS_OK;
}

static int run(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
               double* dt) {
  const int64_t dim = h->dim;
  const size_t vb = sizeof(float2) * (size_t)dim;
  // vectors: work (psi / y), 3 recurrence buffers, lambda, and for the gradient phi_k, psi_k
  QVS_TRY(h->psi.ensure(vb));
  QVS_TRY(h->work.ensure(vb * 3));
  if (grad) {
    QVS_TRY(h->lam.ensure(vb * 2));
    QVS_TRY(h->ckpt.ensure(vb * (size_t)(2 * p)));
  }
  const int nslots = 1 + 2 * p;
  QVS_TRY(h->part.ensure(sizeof(double) * (size_t)nslots * RED_GRID));
  QVS_TRY(h->res.ensure(sizeof(double) * nslots));
  QVS_TRY(h->rowmap.ensure(sizeof(int) * 3 * nslots));
  std::vector<int> rowmap(3 * (size_t)nslots, -1);
  for (int s = 0; s < nslots; ++s) rowmap[3 * s] = s;
  QVS_CUDA_TRY(cudaMemcpyAsync(h->rowmap.ptr, rowmap.data(), sizeof(int) * rowmap.size(), cudaMemcpyHostToDevice,
                               h->stream));
  float2* W = h->psi.as<float2>();
  float2* S = h->work.as<float2>();
  float2* s0 = S;
  float2* s1 = S + dim;
  float2* s2 = S + 2 * dim;
  float2* phiK = grad ? h->ckpt.as<float2>() : nullptr;        // phi_k, k = 1..p
  float2* psiK = grad ? phiK + (size_t)p * dim : nullptr;      // psi_k, k = 1..p
  int64_t launches = 0;
  const float amp = (float)(1.0 / sqrt((double)dim));
  const float* q = h->q.as<float>();
  const float2* psi0 = h->have_psi0 ? h->psi0.as<float2>() : nullptr;
  auto ew = [&](int mode, EwArgs e, double bytes) -> int {
    static const char* names[] = {"csr_phase", "csr_phase_adjoint", "csr_expect_lambda", "csr_expect"};
    return launch_prof(h, names[mode], bytes * (double)dim, launches, [&] {
      switch (mode) {
        case PH_FWD: ew_kernel<PH_FWD><<<RED_GRID, NT, 0, h->stream>>>(e); break;
        case PH_REV: ew_kernel<PH_REV><<<RED_GRID, NT, 0, h->stream>>>(e); break;
        case E_LAM: ew_kernel<E_LAM><<<RED_GRID, NT, 0, h->stream>>>(e); break;
        case E_ONLY: ew_kernel<E_ONLY><<<RED_GRID, NT, 0, h->stream>>>(e); break;
      }
    });
  };
  // forward (evolve mode: phi in lam[0..dim), the state in W)
  if (!grad) QVS_TRY(h->lam.ensure(vb * 2));
  const float2* cur = psi0;   // NULL = uniform
  for (int k = 0; k < p; ++k) {
    float2* phi = grad ? phiK + (size_t)k * dim : h->lam.as<float2>();
    float2* out = grad ? psiK + (size_t)k * dim : W;
    EwArgs e{};
    e.dim = dim;
    e.q = q;
    e.in = cur;
    e.out = phi;
    turns_split(gammas[k], &e.gh, &e.gl);
    e.init_amp = amp;
    QVS_TRY(ew(PH_FWD, e, 4.0 + 8.0 + (cur ? 8.0 : 0.0)));
    QVS_TRY(expmv(h, ts[k], phi, out, s0, s1, s2, launches));
    cur = out;
  }
  {
    EwArgs e{};
    e.dim = dim;
    e.q = q;
    e.in = cur;
    e.part = h->part.as<double>();
    e.row = 0;
    if (grad) {
      e.out = h->lam.as<float2>();
      QVS_TRY(ew(E_LAM, e, 4.0 + 16.0));
    } else {
      QVS_TRY(ew(E_ONLY, e, 4.0 + 8.0));
    }
  }
  if (grad) {
    float2* lam = h->lam.as<float2>();
    float2* lam2 = lam + dim;
    const CsrData& C = h->csr;
    const int nchunks = (int)((dim + ROWS_PER_CTA - 1) / ROWS_PER_CTA);
    for (int k = p - 1; k >= 0; --k) {
      const float2* psik = psiK + (size_t)k * dim;
      QVS_TRY(launch_prof(h, "csr_dt", (C.xy ? 4.0 * dim : (double)C.nnz * 4.0) + (double)dim * 20.0, launches, [&] {
        with_op(C, [&](auto op) -> int {
          dt_kernel<<<RED_GRID, NT, 0, h->stream>>>(dim, op, psik, lam, h->part.as<double>(), 1 + p + k, nchunks);
          return QVS_OK;
        });
      }));
      QVS_TRY(expmv(h, -ts[k], lam, lam2, s0, s1, s2, launches));
      std::swap(lam, lam2);
      EwArgs e{};
      e.dim = dim;
      e.q = q;
      e.in = phiK + (size_t)k * dim;
      e.out = lam;
      turns_split(gammas[k], &e.gh, &e.gl);
      e.part = h->part.as<double>();
      e.row = 1 + k;
      QVS_TRY(ew(PH_REV, e, 4.0 + 8.0 + 16.0));
    }
  }
  const int nout = grad ? nslots : 1;
  QVS_TRY(launch_prof(h, "reduce_rows", 8.0 * RED_GRID * nout, launches, [&] {
    reduce_rows(h, h->part.as<double>(), RED_GRID, h->rowmap.as<int>(), nout, h->res.as<double>());
  }));
  h->launches = launches;
  QVS_TRY(ensure_host_res(h, p));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->host_res, h->res.ptr, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  QVS_TRY(prof_flush(h));
  *E = h->host_res[0];
  if (grad)
    for (int k = 0; k < p; ++k) {
      dg[k] = h->host_res[1 + k];
      dt[k] = h->host_res[1 + p + k];
    }
  return QVS_OK;
}

}  // namespace cs

int csr_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d) {
  using namespace cs;
  if (h->precision != QVS_C64) return QVS_EUNSUPPORTED;
  const int64_t dim = h->dim;
  if (!d->rowptr || !d->colind || d->nnz < 0 || d->nnz >= (int64_t(1) << 32)) return QVS_EINVAL;
  if (!(d->cheb_tol >= 0.0) || !isfinite(d->spec_lo) || !isfinite(d->spec_hi)) return QVS_EINVAL;
  CsrData& C = h->csr;
  C.xy = false;
  const int64_t nnz = d->nnz;
  const auto kind = d->csr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!d->csr_on_device) {
    if (d->rowptr[0] != 0 || d->rowptr[dim] != nnz) return QVS_EINVAL;
    for (int64_t r = 0; r < dim; ++r)
      if (d->rowptr[r + 1] < d->rowptr[r]) return QVS_EINVAL;
    for (int64_t j = 0; j < nnz; ++j)
      if (d->colind[j] < 0 || d->colind[j] >= dim) return QVS_EINVAL;
  }
  // rowptr: staged as int64 in work, narrowed to uint32 on the device
  QVS_TRY(h->work.ensure(sizeof(int64_t) * (size_t)(dim + 1)));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->work.ptr, d->rowptr, sizeof(int64_t) * (dim + 1), kind, h->stream));
  QVS_TRY(C.rowptr.ensure(sizeof(uint32_t) * (size_t)(dim + 1)));
  rowptr32_kernel<<<RED_GRID, NT, 0, h->stream>>>(dim + 1, h->work.as<int64_t>(), C.rowptr.as<uint32_t>());
  QVS_CUDA_TRY(cudaGetLastError());
  QVS_TRY(C.colind.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)));
  if (nnz) QVS_CUDA_TRY(cudaMemcpyAsync(C.colind.ptr, d->colind, sizeof(int32_t) * nnz, kind, h->stream));
  C.has_values = d->values != nullptr;
  if (C.has_values) {
    QVS_TRY(C.values.ensure(sizeof(float) * (size_t)std::max<int64_t>(nnz, 1)));
    if (nnz) QVS_CUDA_TRY(cudaMemcpyAsync(C.values.ptr, d->values, sizeof(float) * nnz, kind, h->stream));
  }
  C.implicit_value = d->implicit_value;
  C.nnz = nnz;
  C.tol = d->cheb_tol > 0 ? d->cheb_tol : 1e-7;
  if (d->spec_lo == 0.0 && d->spec_hi == 0.0) {
    // Gershgorin: every eigenvalue lies within the largest absolute row sum of zero (diagonal
    // included); the Lanczos estimate below is capped by it
    unsigned int* bits = nullptr;
    QVS_TRY(h->res.ensure(sizeof(double) * 8));
    bits = reinterpret_cast<unsigned int*>(h->res.ptr);
    QVS_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned int), h->stream));
    gershgorin_kernel<<<RED_GRID, NT, 0, h->stream>>>(dim, C.rowptr.as<uint32_t>(),
                                                      C.has_values ? C.values.as<float>() : nullptr,
                                                      C.implicit_value, bits);
    QVS_CUDA_TRY(cudaGetLastError());
    unsigned int hb = 0;
    QVS_CUDA_TRY(cudaMemcpyAsync(&hb, bits, sizeof(hb), cudaMemcpyDeviceToHost, h->stream));
    QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    float g;
    memcpy(&g, &hb, sizeof(g));
    const double G = (double)g * (1.0 + 1e-6) + 1e-30;
    C.gersh = G;
    QVS_TRY(lanczos_interval(h, 64, G, &C.spec_lo, &C.spec_hi));
  } else {
    if (!(d->spec_hi > d->spec_lo)) return QVS_EINVAL;
    C.spec_lo = d->spec_lo;
    C.spec_hi = d->spec_hi;
  }
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return QVS_OK;
}

int xy_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d) {
  using namespace cs;
  if (h->precision != QVS_C64) return QVS_EUNSUPPORTED;
  const int n = d->n_qubits, k = d->hamming_weight;
  if (n < 2 || n > 31 || k < 1 || k >= n) return QVS_EINVAL;
  if (!(d->cheb_tol >= 0.0) || !isfinite(d->spec_lo) || !isfinite(d->spec_hi)) return QVS_EINVAL;
  std::vector<int32_t> binom((size_t)XY_BW * XY_BW, 0);
  for (int b = 0; b < XY_BW; ++b) {
    binom[(size_t)b * XY_BW] = 1;
    for (int j = 1; j <= b && j < XY_BW; ++j) {
      const int64_t v = (int64_t)binom[(size_t)(b - 1) * XY_BW + j - 1] + (j < b ? binom[(size_t)(b - 1) * XY_BW + j] : 0);
      binom[(size_t)b * XY_BW + j] = v > INT32_MAX ? INT32_MAX : (int32_t)v;   // only C(b, j), b <= 31 used
    }
  }
  if ((int64_t)binom[(size_t)n * XY_BW + k] != h->dim) return QVS_EINVAL;
  // the weight-k states in increasing order (next state with the same popcount: Gosper's rule),
  // each with the row of its closing-pair neighbour: the rank sum_i C(c_i, i) of the state with bits
  // 0 and n-1 exchanged (set bits c_1 < ... < c_k), or -1 when the two bits agree
  auto rank = [&](uint32_t s) {
    int64_t r = 0;
    for (int i = 1; s; ++i) {
      const int c = __builtin_ctz(s);
      s &= s - 1u;
      r += binom[(size_t)c * XY_BW + i];
    }
    return r;
  };
  const uint32_t ends = 1u | (1u << (n - 1));
  std::vector<uint2> st((size_t)h->dim);
  uint32_t x = (1u << k) - 1u;
  for (int64_t r = 0; r < h->dim; ++r) {
    const bool differ = ((x & ends) != 0u) && ((x & ends) != ends);
    st[(size_t)r] = make_uint2(x, differ ? (uint32_t)rank(x ^ ends) : 0xffffffffu);
    const uint32_t c = x & (0u - x), rr = x + c;
    x = (((rr ^ x) >> 2) / c) | rr;
  }
  CsrData& C = h->csr;
  QVS_TRY(C.states.ensure(sizeof(uint2) * st.size()));
  QVS_TRY(C.binom.ensure(sizeof(int32_t) * binom.size()));
  QVS_CUDA_TRY(cudaMemcpyAsync(C.states.ptr, st.data(), sizeof(uint2) * st.size(), cudaMemcpyHostToDevice,
                               h->stream));
  QVS_CUDA_TRY(cudaMemcpyAsync(C.binom.ptr, binom.data(), sizeof(int32_t) * binom.size(), cudaMemcpyHostToDevice,
                               h->stream));
  C.xy = true;
  C.xy_n = n;
  C.xy_k = k;
  C.nnz = 0;
  C.tol = d->cheb_tol > 0 ? d->cheb_tol : 1e-7;
  if (d->spec_lo == 0.0 && d->spec_hi == 0.0) {
    // Gershgorin: a row has at most min(n, 2 min(k, n - k)) differing ring pairs, each entry 2
    const double G = 2.0 * std::min(n, 2 * std::min(k, n - k)) * (1.0 + 1e-12);
    C.gersh = G;
    QVS_TRY(lanczos_interval(h, 64, G, &C.spec_lo, &C.spec_hi));
  } else {
    if (!(d->spec_hi > d->spec_lo)) return QVS_EINVAL;
    C.spec_lo = d->spec_lo;
    C.spec_hi = d->spec_hi;
  }
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  st.clear();
  return QVS_OK;
}

int csr_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts) {
  double E = 0.0;
  QVS_TRY(cs::run(h, p, gammas, ts, false, &E, nullptr, nullptr));
  h->E = E;
  h->have_E = true;
  return QVS_OK;
}

int csr_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg, double* dt) {
  return cs::run(h, p, gammas, ts, true, E, dg, dt);
}

}  // namespace qvs
