// QAOA hypercube-mixer path (Sec. 2.3.1): forward evolution, objective and adjoint gradient.
//
// Schedule. The n index bits are split into g groups (g = 2 for n <= 20, g = 3 up to n = 32):
// group A = bits 0..11 (contiguous tile), groups B and C = higher bits, each tile padded with
// low "chunk" bits so every tile row is >= 128 contiguous bytes (s >= 4 for the default sizes).
// Because the rotations of different bits commute, one pass over a tile can finish the mixer of
// layer k on its group, apply the phase of layer k+1, and start the mixer of layer k+1 on the same
// group. With g groups a layer therefore costs g-1 passes instead of g: p+1 passes in total for
// g = 2 and 2p+1 for g = 3, each one read and one write of the state (plus q where a phase is
// applied). The last forward pass is fused with the first adjoint pass.
//
// Adjoint (gradient of f = <psi|Q|psi>, Sec. 2.1): with lambda = Q psi at the end, the reverse
// sweep undoes each pass on psi and lambda together and accumulates
//   df/dt_k     = 2 Im <lambda|X_b psi> summed over the bits b of layer k's mixer,
//   df/dgamma_k = 2 Im <lambda|Q phi_k> at the point just before phase k is undone.
// psi is either re-read from a stored checkpoint of the forward sweep or uncomputed by the
// inverse pass; checkpoints are kept every ckpt_layers layers (default ceil(sqrt(p))).
#include <math.h>

#include <string.h>

#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>

#include "hc_pass.cuh"
#include "hc_staged.cuh"
#include "hc_batch.h"

namespace qvs {
namespace hc {

// ---------------------------------------------------------------- small states (n <= TB)
//
// One CTA holds the whole state in shared memory and runs every layer, the objective and the
// adjoint sweep; the forward states psi_k are kept in global scratch for the adjoint.

template <class T>
struct SmallArgs {
  int n, p;
  const T* q;
  const typename Cx<T>::t* psi0;    // NULL = uniform
  typename Cx<T>::t* states;        // [p][dim] forward states psi_k (gradient) or NULL
  typename Cx<T>::t* psi_out;       // final state (evolve) or NULL
  const double* ang;                // [4p]: cos t_k, sin t_k, gamma_k, (unused)
  double* res;                      // [1 + 2p]: E, dgamma, dt
  int grad;
};

__device__ __forceinline__ double block_sum_all(double v, double* red) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

template <class T>
__device__ void small_rotate(typename Cx<T>::t* s, int n, T c, T sn) {
  const int dim = 1 << n;
  for (int b = 0; b < n; ++b) {
    const int h = 1 << b;
    for (int k = threadIdx.x; k < dim / 2; k += blockDim.x) {
      const int i = ((k >> b) << (b + 1)) | (k & (h - 1));
      rot_normal(s[i], s[i | h], c, sn);
    }
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(256) small_kernel(const __grid_constant__ SmallArgs<T> a) {
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int dim = 1 << a.n;
  C* ps = reinterpret_cast<C*>(smem_raw);
  C* ls = ps + dim;
  const T amp = (T)rsqrt((double)dim);
  for (int i = threadIdx.x; i < dim; i += blockDim.x) {
    if (a.psi0) ps[i] = a.psi0[i];
    else { ps[i].x = amp; ps[i].y = T(0); }
  }
  __syncthreads();
  for (int k = 0; k < a.p; ++k) {
    const double g = a.ang[4 * k + 2];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      double sd, cd;
      sincos(g * (double)a.q[i], &sd, &cd);
      ps[i] = cmul_conj(ps[i], (T)cd, (T)sd);
    }
    __syncthreads();
    small_rotate<T>(ps, a.n, (T)a.ang[4 * k], (T)a.ang[4 * k + 1]);
    if (a.grad)
      for (int i = threadIdx.x; i < dim; i += blockDim.x) a.states[(size_t)k * dim + i] = ps[i];
  }
  double e = 0.0;
  for (int i = threadIdx.x; i < dim; i += blockDim.x)
    e += (double)a.q[i] * ((double)ps[i].x * ps[i].x + (double)ps[i].y * ps[i].y);
  e = block_sum_all(e, red);
  if (threadIdx.x == 0) a.res[0] = e;
  if (!a.grad) {
    for (int i = threadIdx.x; i < dim; i += blockDim.x) a.psi_out[i] = ps[i];
    return;
  }
  for (int i = threadIdx.x; i < dim; i += blockDim.x) {
    ls[i].x = a.q[i] * ps[i].x;
    ls[i].y = a.q[i] * ps[i].y;
  }
  __syncthreads();
  for (int k = a.p - 1; k >= 0; --k) {
    // psi_k from the forward sweep
    for (int i = threadIdx.x; i < dim; i += blockDim.x) ps[i] = a.states[(size_t)k * dim + i];
    __syncthreads();
    // dt_k = 2 Im <lam | W psi>, W = sum_b X_b
    double acc = 0.0;
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      C w;
      w.x = T(0);
      w.y = T(0);
      for (int b = 0; b < a.n; ++b) {
        w.x += ps[i ^ (1 << b)].x;
        w.y += ps[i ^ (1 << b)].y;
      }
      acc += (double)imdot(ls[i], w);
    }
    acc = block_sum_all(acc, red);
    if (threadIdx.x == 0) a.res[1 + a.p + k] = 2.0 * acc;
    const T c = (T)a.ang[4 * k], s = (T)a.ang[4 * k + 1];
    small_rotate<T>(ps, a.n, c, -s);
    small_rotate<T>(ls, a.n, c, -s);
    double ag = 0.0;
    for (int i = threadIdx.x; i < dim; i += blockDim.x) ag += (double)a.q[i] * (double)imdot(ls[i], ps[i]);
    ag = block_sum_all(ag, red);
    if (threadIdx.x == 0) a.res[1 + k] = 2.0 * ag;
    const double g = a.ang[4 * k + 2];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      double sd, cd;
      sincos(g * (double)a.q[i], &sd, &cd);
      ls[i] = cmul_conj(ls[i], (T)cd, -(T)sd);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host-side plan

struct PassInfo {
  int type, shape;
  int lb, la, lg;   // layer of the before rotations, after rotations, phase (-1 = none)
};

struct Plan {
  int n = 0, g = 0, F = 0;
  Tile tile[3];
  uint32_t gmask[3];
  std::vector<PassInfo> pass;   // index 1..F (0 unused)
};

static Tile make_tile(int n, int s, int hfirst, int nh) {
  Tile t{};
  t.smask = (1u << s) - 1u;
  t.hshift = hfirst - s;
  int k = 0;
  for (int b = 0; b < n; ++b) {
    const bool in_tile = (b < s) || (b >= hfirst && b < hfirst + nh);
    if (!in_tile) t.ntbit[k++] = (uint8_t)b;
  }
  t.n_nt = k;
  return t;
}

// tile type of pass j (1-based) when a layer takes three types (see make_plan)
__host__ __device__ __forceinline__ int three_type(int j) { return (j & 1) ? 1 + ((j - 1) / 2) % 2 : 0; }

static int make_plan(int n, int p, Plan& pl) {
  pl = Plan{};
  pl.n = n;
  const int rest = n - TB;
  if (rest < 0) return QVS_EUNSUPPORTED;
  pl.tile[0] = make_tile(n, TB, TB, 0);
  pl.gmask[0] = (1u << TB) - 1;
  if (rest == 0) {
    // one tile holds the whole state: pass j applies phase j-1 and all of mixer j-1
    pl.g = 1;
    pl.F = p + 1;
    pl.pass.assign(pl.F + 1, PassInfo{});
    for (int j = 1; j <= pl.F; ++j) {
      PassInfo& q = pl.pass[j];
      if (j == 1) q = {0, F0, -1, 0, 0};
      else if (j <= p) q = {0, F1, -1, j - 1, j - 1};
      else q = {0, FE, -1, -1, -1};
    }
    return QVS_OK;
  }
  if (rest <= TB - 4) {
    pl.g = 2;
    const int s = TB - rest;
    pl.tile[1] = make_tile(n, s, TB, rest);
    pl.gmask[1] = ((1u << TB) - 1) & ~((1u << s) - 1);
  } else {
    const int r1 = (rest + 1) / 2, r2 = rest - r1;
    if (TB - r1 < 2) return QVS_EUNSUPPORTED;
    pl.g = 3;
    const int s1 = TB - r1, s2 = TB - r2;
    pl.tile[1] = make_tile(n, s1, TB, r1);
    pl.gmask[1] = ((1u << TB) - 1) & ~((1u << s1) - 1);
    pl.tile[2] = make_tile(n, s2, TB + r1, r2);
    pl.gmask[2] = ((1u << TB) - 1) & ~((1u << s2) - 1);
  }
  if (pl.g == 2) {
    pl.F = p + 1;
    pl.pass.assign(pl.F + 1, PassInfo{});
    for (int j = 1; j <= pl.F; ++j) {
      PassInfo& q = pl.pass[j];
      q.type = (j - 1) % 2;
      if (j == 1) q = {q.type, F0, -1, 0, 0};
      else if (j <= p) q = {q.type, F1, j - 2, j - 1, j - 1};
      else q = {q.type, FE, p - 1, -1, -1};
    }
  } else {
    // Passes alternate: odd j carries a phase (F0, F1, FE) and rotates one high tile type on both
    // of its sides, even j (F2) rotates the rest of a layer. Odd passes alternate types 1 and 2 and
    // every even pass takes type 0, so each layer rotates types {1, 0, 2} or {2, 0, 1}: the
    // arithmetic-heavy phase passes always use a high type (two register layouts), and the
    // contiguous type 0 (three layouts, one more transpose per direction) only the F2 / R2 passes.
    pl.F = 2 * p + 1;
    pl.pass.assign(pl.F + 1, PassInfo{});
    for (int j = 1; j <= pl.F; ++j) {
      PassInfo& q = pl.pass[j];
      q.type = three_type(j);
      if (j == 1) q = {q.type, F0, -1, 0, 0};
      else if (j == pl.F) q = {q.type, FE, p - 1, -1, -1};
      else if (j % 2 == 0) q = {q.type, F2, (j - 2) / 2, -1, -1};
      else q = {q.type, F1, (j - 3) / 2, (j - 1) / 2, (j - 1) / 2};
    }
  }
  return QVS_OK;
}


static const char* shape_name(int shape, bool dbl) {
  static const char* f[] = {"hc_pass_F0_c64", "hc_pass_F1_c64", "hc_pass_F2_c64", "hc_pass_FE_c64",
                            "hc_pass_FV_c64", "hc_pass_R1_c64", "hc_pass_R2_c64", "hc_pass_R0_c64",
                            "hc_pass_R1X_c64", "hc_pass_R0X_c64"};
  static const char* d[] = {"hc_pass_F0_c128", "hc_pass_F1_c128", "hc_pass_F2_c128", "hc_pass_FE_c128",
                            "hc_pass_FV_c128", "hc_pass_R1_c128", "hc_pass_R2_c128", "hc_pass_R0_c128",
                            "hc_pass_R1X_c128", "hc_pass_R0X_c128"};
  return dbl ? d[shape] : f[shape];
}

// compulsory bytes per amplitude of one pass (complex element size c, quality element size qb)
static double shape_bytes(int shape, const void* psi_in, const void* psi_out, double c, double qb) {
  switch (shape) {
    case F0: return qb + c + (psi_in ? c : 0.0);
    case F1: return 2 * c + qb;
    case F2: return 2 * c;
    case FE: return 2 * c + qb;
    case FV: return 2 * c + qb;
    case R1: return 3 * c + qb + (psi_out ? c : 0.0);
    case R2: return 3 * c + (psi_out ? c : 0.0);
    case R0: return 2 * c + qb;
    case R1X: return 3 * c + qb + (psi_out ? c : 0.0) + qb;   // + the stored g
    case R0X: return 2 * c + 2 * qb;
  }
  return 0.0;
}

// Rotation threshold of a pass from its masks: every used mask must be "tile bits >= TH" for one
// TH that has a compiled complex64 kernel (TH_NONE: no "before" bits, all "after" bits), else the
// runtime-mask kernel runs.
static int pass_threshold(int shape, uint32_t mask_bef, uint32_t mask_aft) {
  const bool ub = shape == F1 || shape == F2 || shape == FE || shape == FV || shape == R1 || shape == R2;
  const bool ua = shape == F0 || shape == F1 || shape == R1 || shape == R0;
  auto th = [](uint32_t m) -> int {
    if (m == 0) return -2;
    int t = 0;
    while (!((m >> t) & 1u)) ++t;
    return m == (((1u << TB) - 1u) & ~((1u << t) - 1u)) ? t : -3;
  };
  const int tb = ub ? th(mask_bef) : -4, ta = ua ? th(mask_aft) : -4;
  int t = TH_RUNTIME;
  if (ub && ua) {
    if (tb >= 0 && tb == ta) t = tb;
    else if (tb == -2 && ta == 0) t = TH_NONE;
  } else if (ub) {
    t = tb >= 0 ? tb : TH_RUNTIME;
  } else if (ua) {
    t = ta >= 0 ? ta : TH_RUNTIME;
  }
  return t;
}

static int launch_c64(int th, int shape, const PassArgs<float>& a, uint32_t grid, cudaStream_t st) {
  switch (th) {
#define QVS_HC_CASE(K) \
    case K: return launch_pass<float, K>(shape, a, grid, st);
    QVS_HC_C64_THRESHOLDS(QVS_HC_CASE)
#undef QVS_HC_CASE
    default: return launch_pass<float, TH_RUNTIME>(shape, a, grid, st);
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link to libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    (void)cudaGetLastError();
    return nullptr;
  }();   // initialised once, thread-safely
  return fn;
}

// the same lookup for the other mixer paths (NULL when the driver lacks the entry point)
void* tensor_map_encode_fn() { return reinterpret_cast<void*>(tensor_map_encoder()); }

// The tile box of tile geometry t over a 2^n-element vector (elem bytes per element): the packed
// 5-d view (low chunk bits up to 8 | chunk bits 8..s-1 | middle non-tile bits | high tile bits |
// top non-tile bits); a tile is {d0, d1, 1, d3, 1} at (0, 0, mid, 0, top).
static int encode_tile_map(CUtensorMap* map, const void* base, int elem, const Tile& t, int n, int* mid_bits,
                           int* top_bits) {
  auto enc = tensor_map_encoder();
  if (!enc) return QVS_EUNSUPPORTED;
  const int s = __builtin_popcount(t.smask), hfirst = s + t.hshift, nh = TB - s;
  const int top = n - hfirst - nh;
  const cuuint64_t d0 = s > 8 ? 256u : (1u << s), d1 = s > 8 ? (1u << (s - 8)) : 1u;
  cuuint64_t dims[5] = {d0, d1, (cuuint64_t)1 << (hfirst - s), (cuuint64_t)1 << nh, (cuuint64_t)1 << top};
  cuuint64_t strides[4] = {d0 * elem, ((cuuint64_t)1 << s) * elem, ((cuuint64_t)1 << hfirst) * elem,
                           ((cuuint64_t)1 << (hfirst + nh)) * elem};
  cuuint32_t box[5] = {(cuuint32_t)d0, (cuuint32_t)d1, 1u, (cuuint32_t)1u << nh, 1u};
  cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r =
      enc(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base),
          dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return QVS_ECUDA;
  *mid_bits = hfirst - s;
  *top_bits = top;
  return QVS_OK;
}

static int launch_staged_c64(int th, int shape, const PassArgs<float>& a, const StageMaps& m, uint32_t ntiles,
                             uint32_t grid, cudaStream_t st) {
  switch (th) {
#define QVS_HC_CASE(K) \
    case K: return launch_staged<K>(shape, a, m, ntiles, grid, st);
    QVS_HC_C64_THRESHOLDS(QVS_HC_CASE)
#undef QVS_HC_CASE
    default: return launch_staged<TH_RUNTIME>(shape, a, m, ntiles, grid, st);
  }
}

// Which complex64 passes run staged (persistent CTAs, TMA-fed): the last forward pass FE, whose
// single input vector leaves room for the stage beside two transpose buffers' worth of work (n=28:
// 1.41 -> 1.17 ms per launch). The adjoint passes measured no faster staged (R2 1.474 vs 1.479 ms,
// R1 2.215 vs 2.259 ms: their two vectors go through one transpose buffer one after the other), so
// they keep one CTA per tile. Also needed: the option on, the tensor-map encoder available, and the
// tile's high field within one box dimension (at most 256 elements: chunks of >= 4 bits, n <= 28).
static bool use_staged(const qvs_ctx* h, int shape, const Tile& t) {
  return h->staged && shape == FE && __builtin_popcount(t.smask) >= TB - 8 && tensor_map_encoder();
}

template <class T>
static int launch_shape(qvs_ctx* h, int shape, const PassArgs<T>& a, uint32_t grid) {
  cudaEvent_t ev;
  QVS_TRY(prof_begin(h, &ev));
  if constexpr (sizeof(T) == 4) {
    const int th = shape >= R1X ? TH_RUNTIME : pass_threshold(shape, a.mask_bef, a.mask_aft);
    if (use_staged(h, shape, a.tile)) {
      StageMaps m;
      memset(&m, 0, sizeof(m));
      m.two = shape != FE;
      QVS_TRY(encode_tile_map(&m.psi, a.psi_in, 8, a.tile, h->n, &m.mid_bits, &m.top_bits));
      if (m.two) QVS_TRY(encode_tile_map(&m.lam, a.lam_in, 8, a.tile, h->n, &m.mid_bits, &m.top_bits));
      m.qpf = shape != R2 && !a.qcta && a.q;
      if (m.qpf) QVS_TRY(encode_tile_map(&m.q, a.q, 4, a.tile, h->n, &m.mid_bits, &m.top_bits));
      m.err = h->flags.as<int>();
      const uint32_t ctas = std::min<uint32_t>(grid, 2u * (uint32_t)h->sms);
      QVS_TRY(launch_staged_c64(th, shape, a, m, grid, ctas, h->stream));
    } else {
      QVS_TRY(launch_c64(th, shape, a, grid, h->stream));
    }
  } else {
    QVS_TRY((launch_pass<T, TH_RUNTIME>(shape, a, grid, h->stream)));
  }
  // a quadratic quality reads one 64-byte table row per tile instead of q
  const double c = sizeof(typename Cx<T>::t), qb = a.qcta ? 64.0 / TILE : (double)sizeof(T);
  return prof_end(h, shape_name(shape, sizeof(T) == 8),
                  shape_bytes(shape, a.psi_in, a.psi_out, c, qb) * (double)grid * TILE, ev);
}

// ---------------------------------------------------------------- small-state driver

template <class T>
static int run_small(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad,
                     double* E, double* dg, double* dt) {
  using C = typename Cx<T>::t;
  const int64_t dim = h->dim;
  QVS_TRY(h->res.ensure(sizeof(double) * (size_t)(1 + 2 * p) + sizeof(double) * 4 * (size_t)p));
  double* res = h->res.as<double>();
  double* ang = res + 1 + 2 * p;
  std::vector<double> hang(4 * (size_t)p);
  for (int k = 0; k < p; ++k) {
    hang[4 * k] = cos(ts[k]);
    hang[4 * k + 1] = sin(ts[k]);
    hang[4 * k + 2] = gammas[k];
    hang[4 * k + 3] = 0.0;
  }
  QVS_CUDA_TRY(cudaMemcpyAsync(ang, hang.data(), sizeof(double) * 4 * p, cudaMemcpyHostToDevice,
                               h->stream));
  QVS_TRY(h->psi.ensure(dim * sizeof(C)));
  if (grad) QVS_TRY(h->ckpt.ensure((size_t)p * dim * sizeof(C)));
  SmallArgs<T> a{};
  a.n = h->n;
  a.p = p;
  a.q = h->q.as<T>();
  a.psi0 = h->have_psi0 ? h->psi0.as<C>() : nullptr;
  a.states = grad ? h->ckpt.as<C>() : nullptr;
  a.psi_out = h->psi.as<C>();
  a.ang = ang;
  a.res = res;
  a.grad = grad ? 1 : 0;
  const size_t sm = 2 * (size_t)dim * sizeof(C);
  QVS_CUDA_TRY(cudaFuncSetAttribute(small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm));
  small_kernel<T><<<1, 256, sm, h->stream>>>(a);
  QVS_CUDA_TRY(cudaGetLastError());
  h->launches = 1;
  QVS_TRY(ensure_host_res(h, p));
  const int nres = grad ? 1 + 2 * p : 1;
  QVS_CUDA_TRY(cudaMemcpyAsync(h->host_res, res, sizeof(double) * nres, cudaMemcpyDeviceToHost,
                               h->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  *E = h->host_res[0];
  if (grad) {
    for (int k = 0; k < p; ++k) {
      dg[k] = h->host_res[1 + k];
      dt[k] = h->host_res[1 + p + k];
    }
  }
  return QVS_OK;
}

// ---------------------------------------------------------------- quadratic-quality tables
//
// For a quadratic quality (qvs_set_quality_qubo) the phase passes compute q themselves (qgen2):
// per tile type and frame f (bits read at index XOR f (2^n - 1)) they need the per-tile rows
// {c + non-tile terms, L_0..L_11} and the per-thread rows {K_T, K_5..K_8}, plus the register pair
// sums PP(r) carried in the pass arguments.

static int tile_index_bit(const Tile& t, int k) {
  const int s = __builtin_popcount(t.smask);
  return k < s ? k : k + t.hshift;
}

// Rows of coefficient set blockIdx.y (sums mod 2^32: exact int32 qualities never wrap, ex-QAOA
// angles are turns in 32-bit fixed point and wrap by design).
__global__ void qubo_rows_kernel(const QuboCoef* __restrict__ Qs, Tile t, int flip, uint32_t ntiles,
                                 int* __restrict__ rows0, size_t cstride) {
  const uint32_t bid = blockIdx.x * blockDim.x + threadIdx.x;
  if (bid >= ntiles) return;
  const QuboCoef* Q = Qs + blockIdx.y;
  const uint32_t xb = tile_base(t, bid) ^ (flip ? all_bits(Q->n) : 0u);
  const int s = __popc(t.smask);
  uint32_t qU = (uint32_t)Q->c;
  for (int i = 0; i < t.n_nt; ++i) {
    const int j = t.ntbit[i];
    if (!((xb >> j) & 1u)) continue;
    qU += (uint32_t)Q->h[j];
    for (int i2 = 0; i2 < i; ++i2) {
      const int j2 = t.ntbit[i2];
      if ((xb >> j2) & 1u) qU += (uint32_t)Q->J[j][j2];
    }
  }
  int* row = rows0 + cstride * blockIdx.y + 16 * (size_t)bid;
  row[0] = (int)qU;
  for (int k = 0; k < TB; ++k) {
    const int pk = k < s ? k : k + t.hshift;
    uint32_t L = (uint32_t)Q->h[pk];
    for (int i = 0; i < t.n_nt; ++i) {
      const int j = t.ntbit[i];
      if ((xb >> j) & 1u) L += (uint32_t)Q->J[pk][j];
    }
    row[1 + k] = (int)L;
  }
  row[13] = row[14] = row[15] = 0;
}

static size_t qubo_block_ints(uint32_t grid) { return 16 * (size_t)grid + 8 * (size_t)NT; }

// Tables of ncoef quadratic forms: block (c * g + tau) * 2 + f of tab holds the CTA rows and thread
// rows of form c, tile type tau and frame f; pp[16 * block + r] its register pair sums.
static int build_tables(qvs_ctx* h, const Plan& pl, uint32_t grid, const QuboCoef* coefs, int ncoef,
                        DevBuf& dcoef, DevBuf& tab, std::vector<int32_t>& pp) {
  const size_t bi = qubo_block_ints(grid);
  const int nblk = ncoef * pl.g * 2;
  QVS_TRY(tab.ensure(sizeof(int) * bi * nblk));
  QVS_TRY(dcoef.ensure(sizeof(QuboCoef) * ncoef));
  QVS_CUDA_TRY(cudaMemcpyAsync(dcoef.ptr, coefs, sizeof(QuboCoef) * ncoef, cudaMemcpyHostToDevice, h->stream));
  pp.assign(16 * (size_t)nblk, 0);
  std::vector<int> thr(8 * (size_t)NT * nblk, 0);
  for (int tau = 0; tau < pl.g; ++tau) {
    const Tile& t = pl.tile[tau];
    int pk[TB];
    for (int k = 0; k < TB; ++k) pk[k] = tile_index_bit(t, k);
    for (int f = 0; f < 2; ++f) {
      int* rows0 = tab.as<int>() + bi * (size_t)(tau * 2 + f);
      dim3 gr((grid + 127) / 128, ncoef);
      qubo_rows_kernel<<<gr, 128, 0, h->stream>>>(dcoef.as<QuboCoef>(), t, f, grid, rows0, bi * pl.g * 2);
      QVS_CUDA_TRY(cudaGetLastError());
      const uint32_t fl = f ? 0xFFFu : 0u;
      for (int c = 0; c < ncoef; ++c) {
        const QuboCoef& Q = coefs[c];
        const int blk = (c * pl.g + tau) * 2 + f;
        for (int tid = 0; tid < NT; ++tid) {
          const uint32_t xt = (uint32_t)tj<2>(0, tid) ^ fl;
          uint32_t kt = 0, kc[RB] = {0, 0, 0, 0};
          for (int k = 0; k < TB; ++k) {
            if ((k >= 5 && k <= 8) || !((xt >> k) & 1u)) continue;
            for (int l = 0; l < k; ++l)
              if ((l < 5 || l > 8) && ((xt >> l) & 1u)) kt += (uint32_t)Q.J[pk[k]][pk[l]];
            for (int i = 0; i < RB; ++i) kc[i] += (uint32_t)Q.J[pk[5 + i]][pk[k]];
          }
          int* row = thr.data() + 8 * ((size_t)NT * blk + tid);
          row[0] = (int)kt;
          for (int i = 0; i < RB; ++i) row[1 + i] = (int)kc[i];
        }
        for (int r = 0; r < R; ++r) {
          const int x = r ^ (f ? R - 1 : 0);
          uint32_t v = 0;
          for (int i = 0; i < RB; ++i)
            for (int i2 = 0; i2 < i; ++i2)
              if (((x >> i) & 1) && ((x >> i2) & 1)) v += (uint32_t)Q.J[pk[5 + i]][pk[5 + i2]];
          pp[16 * (size_t)blk + r] = (int32_t)v;
        }
      }
    }
  }
  for (int blk = 0; blk < nblk; ++blk)
    QVS_CUDA_TRY(cudaMemcpyAsync(tab.as<int>() + bi * blk + 16 * (size_t)grid, thr.data() + 8 * (size_t)NT * blk,
                                 sizeof(int) * 8 * NT, cudaMemcpyHostToDevice, h->stream));
  // the host staging vector goes out of scope: finish the copies first
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return QVS_OK;
}

static int build_qubo_tables(qvs_ctx* h, const Plan& pl, uint32_t grid) {
  QVS_TRY(build_tables(h, pl, grid, &h->qubo.coef, 1, h->qubo.dcoef, h->qubo.tab, h->qubo.pp));
  h->qubo.tab_valid = true;
  return QVS_OK;
}

// point a pass at the tables of form c, its tile type and its frame
template <class T>
static void set_table_args(const int* tab, const std::vector<int32_t>& pp, int c, int g, int type, uint32_t grid,
                           T scale, PassArgs<T>& a) {
  const int blk = (c * g + type) * 2 + (a.qx ? 1 : 0);
  const int* base = tab + qubo_block_ints(grid) * blk;
  a.qcta = base;
  a.qthr = base + 16 * (size_t)grid;
  for (int r = 0; r < R; ++r) a.qpp[r] = pp[16 * (size_t)blk + r];
  a.qscale = scale;
}

template <class T>
static void set_qubo_args(const qvs_ctx* h, int g, int type, uint32_t grid, PassArgs<T>& a) {
  set_table_args<T>(h->qubo.tab.as<int>(), h->qubo.pp, 0, g, type, grid, (T)ldexp(1.0, -h->qubo.coef.F), a);
}

// ex-QAOA state of one solve: per-layer phase-angle tables, the g buffer and the term list of the
// moments kernel
struct ExRun {
  const int* tab;
  const std::vector<int32_t>* pp;
  float* g;
  int nterms;
  const int2* tbits;
  const float* tc;
  double* mpart;
  uint32_t mgrid;
};

// the phase of an ex-QAOA layer: its angle (turns, 32-bit fixed point) from the layer's tables
template <class T>
static void set_ex_phase(const ExRun* ex, int g, int layer, int type, uint32_t grid, PassArgs<T>& a) {
  set_table_args<T>(ex->tab, *ex->pp, layer, g, type, grid, (T)ldexp(1.0, -32), a);
  if constexpr (sizeof(T) == 4) {
    a.ph0 = 1.0f;   // phase_cs(q, 1, 0): exp(-i 2 pi q) with q in turns
    a.ph1 = 0.0f;
  } else {
    a.ph0 = 6.283185307179586476925286766559;   // complex128: sincos(2 pi q)
    a.ph1 = 0.0;
  }
}

// ---------------------------------------------------------------- ex-QAOA per-term gradients
//
// After the adjoint phase pass of layer k has stored g(x) = 2 Im(conj(lambda) phi)(x), the
// derivative by gamma_{k,j} is sum_x c_j s_j(x) g(x), with s_j = z_a z_b or z_a and z = 1 - 2x
// (Sec. 2.3.2). On a tile of 4096 consecutive amplitudes (index bits 0..11) a Walsh-Hadamard
// transform gives M[S] = sum_x prod_{k in S} z_k(x) g(x) for every subset S of the tile bits; term j
// takes M[S_j] (its bits inside the tile) times its z over the tile-index bits. Each CTA walks a
// fixed set of tiles, keeps its terms' sums in fp64 and writes them as partial rows; the rows are
// summed over CTAs in a fixed order (deterministic).
constexpr int MT_MAX = 1024;   // terms per solve
__device__ __forceinline__ int mslot(int j) { return j + (j >> 4); }

__device__ __forceinline__ void wht16(float (&v)[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (!((m >> i) & 1)) {
        const float x = v[m], y = v[m | (1 << i)];
        v[m] = x + y;
        v[m | (1 << i)] = x - y;
      }
}

__global__ void __launch_bounds__(256) exq_moments_kernel(const float* __restrict__ g, int n, int nterms,
                                                          const int2* __restrict__ tb, const float* __restrict__ tc,
                                                          double* __restrict__ part) {
  __shared__ float sm[4096 + 256];
  const int t = threadIdx.x;
  const uint32_t ntiles = 1u << (n - 12);
  double acc[MT_MAX / 256];
#pragma unroll
  for (int i = 0; i < MT_MAX / 256; ++i) acc[i] = 0.0;
  for (uint32_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
    float v[16];
    const float* src = g + ((size_t)T << 12);
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = __ldcs(src + t + 256 * m);   // register bits = tile bits 8..11
    wht16(v);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[mslot(t + 256 * m)] = v[m];
    __syncthreads();
    const int pb = (t & 15) | ((t >> 4) << 8);                        // register bits = tile bits 4..7
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sm[mslot(pb | (m << 4))];
    wht16(v);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[mslot(pb | (m << 4))] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sm[mslot(m | (t << 4))];     // register bits = tile bits 0..3
    wht16(v);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[mslot(m | (t << 4))] = v[m];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MT_MAX / 256; ++i) {
      const int j = t + 256 * i;
      if (j < nterms) {
        const int2 b = tb[j];
        int S = 0;
        float sg = tc[j];
        if (b.x < 12) S |= 1 << b.x;
        else if ((T >> (b.x - 12)) & 1u) sg = -sg;
        if (b.y >= 0) {
          if (b.y < 12) S |= 1 << b.y;
          else if ((T >> (b.y - 12)) & 1u) sg = -sg;
        }
        acc[i] += (double)(sg * sm[mslot(S)]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MT_MAX / 256; ++i) {
    const int j = t + 256 * i;
    if (j < nterms) part[(size_t)j * gridDim.x + blockIdx.x] = acc[i];
  }
}

static bool shape_reads_q(int shape) { return shape != F2 && shape != R2; }

// ---------------------------------------------------------------- tiled driver

template <class T>
static int run_tiled(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad,
                     double* E, double* dg, double* dt, const ExRun* ex = nullptr, double* dG = nullptr) {
  using C = typename Cx<T>::t;
  Plan pl;
  QVS_TRY(make_plan(h->n, p, pl));
  const int F = pl.F;
  const uint32_t grid = 1u << (h->n - TB);
  const size_t sbytes = (size_t)h->dim * sizeof(C);
  const bool qubo = h->qubo.on;
  if (qubo && !h->qubo.tab_valid) QVS_TRY(build_qubo_tables(h, pl, grid));

  // checkpoint placement: stored pass boundaries j = c, 2c, ... <= F-1
  int ckl = h->ckpt_layers > 0 ? h->ckpt_layers : (int)ceil(sqrt((double)p) - 1e-9);
  if (ckl < 1) ckl = 1;
  const int c = grad ? ckl * (pl.g - 1) : (F + 1);
  const int nck = grad ? (F - 1) / c : 0;
  QVS_TRY(h->psi.ensure(sbytes));
  if (grad) {
    QVS_TRY(h->lam.ensure(sbytes));
    if (nck > 0) QVS_TRY(h->ckpt.ensure((size_t)nck * sbytes));
  }
  const int nrows = 3 * F + 1;
  QVS_TRY(h->part.ensure(sizeof(double) * (size_t)nrows * grid));
  const int nslots = 1 + 2 * p;
  QVS_TRY(h->res.ensure(sizeof(double) * nslots));
  QVS_TRY(h->rowmap.ensure(sizeof(int) * 3 * nslots));
  C* W = h->psi.as<C>();
  C* K = h->ckpt.as<C>();
  auto loc = [&](int j) -> C* {
    if (j >= 1 && j <= F - 1 && j % c == 0 && (j / c) <= nck) return K + (size_t)(j / c - 1) * h->dim;
    return W;
  };
  const bool stored_ck = true;
  (void)stored_ck;
  auto is_stored = [&](int j) { return j >= 1 && j <= F - 1 && j % c == 0 && (j / c) <= nck; };

  // reduction row map: slot 0 = E; 1..p = dgamma_k; p+1..2p = dt_k
  std::vector<int> rowmap(3 * (size_t)nslots, -1);
  rowmap[0] = 3 * F;
  if (grad) {
    std::vector<int> fill(nslots, 0);
    auto add = [&](int slot, int row) { rowmap[3 * slot + fill[slot]++] = row; };
    for (int j = 1; j <= F; ++j) {
      const PassInfo& pi = pl.pass[j];
      if (pi.lg >= 0) add(1 + pi.lg, 3 * (j - 1) + 2);
      if (pi.lb >= 0) add(1 + p + pi.lb, 3 * (j - 1) + 0);
      if (pi.la >= 0) add(1 + p + pi.la, 3 * (j - 1) + 1);
    }
  }
  QVS_CUDA_TRY(cudaMemcpyAsync(h->rowmap.ptr, rowmap.data(), sizeof(int) * rowmap.size(),
                               cudaMemcpyHostToDevice, h->stream));
  QVS_TRY(h->flags.ensure(16));
  QVS_CUDA_TRY(cudaMemsetAsync(h->flags.ptr, 0, 16, h->stream));

  const T amp = (T)(1.0 / sqrt((double)h->dim));
  const int n = h->n;
  int64_t launches = 0;
  // Frames (scale k and flip F of the stored vector) at the pass boundaries, tracked on the host:
  // fw[j] = psi after forward pass j.
  std::vector<Frame> fw(F + 1, Frame{1.0, 0});
  Frame fr{1.0, 0}, lf{1.0, 0};
  // qvs_evolve under a flipped final frame writes the output at complemented indices: another
  // tile's input, so it goes to a second buffer
  C* out_buf = W;
  // forward
  for (int j = 1; j <= F; ++j) {
    const PassInfo& pi = pl.pass[j];
    const int G = __builtin_popcount(pl.gmask[pi.type]);
    PassArgs<T> a{};
    a.tile = pl.tile[pi.type];
    a.q = h->q.as<T>();
    a.part = h->part.as<double>();
    a.row_bef = a.row_aft = a.row_gam = -1;
    a.row_E = 3 * F;
    a.init_amp = amp;
    a.gen_init = h->have_psi0 ? 0 : 1;
    a.mask_bef = pi.lb >= 0 ? pl.gmask[pi.type] : 0u;
    a.mask_aft = pi.la >= 0 ? pl.gmask[pi.type] : 0u;
    a.psi_in = (j == 1) ? (h->have_psi0 ? h->psi0.as<C>() : nullptr) : loc(j - 1);
    int shape = pi.shape;
    if (j == F) shape = grad ? FE : FV;
    fwd_scalars<T>(a, shape, pi.lb, pi.la, pi.lg, G, n, p, gammas, ts, fr, lf);
    if (qubo && shape_reads_q(shape)) set_qubo_args<T>(h, pl.g, pi.type, grid, a);
    if (ex && pi.lg >= 0 && (shape == F0 || shape == F1)) set_ex_phase(ex, pl.g, pi.lg, pi.type, grid, a);
    if (j == F) {
      if (grad) {
        a.lam_out = h->lam.as<C>();
        a.row_bef = 3 * (j - 1) + 0;
      } else {
        if (a.ox) {
          QVS_TRY(h->lam.ensure(sbytes));
          out_buf = h->lam.as<C>();
        }
        a.psi_out = out_buf;
      }
    } else {
      a.psi_out = grad ? loc(j) : W;
      fw[j] = fr;
    }
    QVS_TRY(launch_shape<T>(h, shape, a, grid));
    ++launches;
  }
  if (out_buf != W) std::swap(h->psi, h->lam);
  // adjoint
  if (grad) {
    Frame pout{1.0, 0};
    for (int j = F - 1; j >= 1; --j) {
      const PassInfo& pi = pl.pass[j];
      const int G = __builtin_popcount(pl.gmask[pi.type]);
      PassArgs<T> a{};
      a.tile = pl.tile[pi.type];
      a.q = h->q.as<T>();
      a.part = h->part.as<double>();
      a.mask_bef = pi.lb >= 0 ? pl.gmask[pi.type] : 0u;
      a.mask_aft = pi.la >= 0 ? pl.gmask[pi.type] : 0u;
      a.psi_in = loc(j);
      a.lam_in = h->lam.as<C>();
      a.lam_out = h->lam.as<C>();
      a.psi_out = (j - 1 >= 1 && !is_stored(j - 1)) ? W : nullptr;
      a.row_bef = pi.lb >= 0 ? 3 * (j - 1) + 0 : -1;
      a.row_aft = pi.la >= 0 ? 3 * (j - 1) + 1 : -1;
      a.row_gam = pi.lg >= 0 ? 3 * (j - 1) + 2 : -1;
      a.row_E = -1;
      const int shape = pi.shape == F0 ? R0 : (pi.shape == F1 ? R1 : R2);
      // psi at boundary j: a checkpoint or the forward sweep's last write (frame fw[j]), else the
      // previous adjoint pass's uncompute
      Frame pf = (is_stored(j) || j == F - 1) ? fw[j] : pout;
      bwd_scalars<T>(a, shape, pi.lb, pi.la, pi.lg, G, n, gammas, ts, pf, lf);
      if (qubo && shape_reads_q(shape)) set_qubo_args<T>(h, pl.g, pi.type, grid, a);
      pout = pf;
      if (ex && pi.lg >= 0) {
        set_ex_phase(ex, pl.g, pi.lg, pi.type, grid, a);
        a.gout = reinterpret_cast<T*>(ex->g);
        a.row_gam = -1;
        QVS_TRY(launch_shape<T>(h, shape == R1 ? R1X : R0X, a, grid));
        cudaEvent_t ev;
        QVS_TRY(prof_begin(h, &ev));
        exq_moments_kernel<<<ex->mgrid, 256, 0, h->stream>>>(
            ex->g, n, ex->nterms, ex->tbits, ex->tc, ex->mpart + (size_t)pi.lg * ex->nterms * ex->mgrid);
        QVS_CUDA_TRY(cudaGetLastError());
        QVS_TRY(prof_end(h, "exq_moments", 4.0 * (double)h->dim, ev));
        launches += 2;
        continue;
      }
      QVS_TRY(launch_shape<T>(h, shape, a, grid));
      ++launches;
    }
  }
  const int nout = grad ? nslots : 1;
  {
    cudaEvent_t ev;
    QVS_TRY(prof_begin(h, &ev));
    QVS_TRY(reduce_rows(h, h->part.as<double>(), grid, h->rowmap.as<int>(), nout, h->res.as<double>()));
    QVS_TRY(prof_end(h, "reduce_rows", 8.0 * grid * (nout == 1 ? 1 : 3 * F), ev));
  }
  ++launches;
  h->launches = launches;
  QVS_TRY(ensure_host_res(h, p));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->host_res, h->res.ptr, sizeof(double) * nout,
                               cudaMemcpyDeviceToHost, h->stream));
  int* host_flag = reinterpret_cast<int*>(h->host_res + 1 + 2 * (size_t)h->host_res_cap);
  QVS_CUDA_TRY(cudaMemcpyAsync(host_flag, h->flags.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  QVS_TRY(prof_flush(h));
  if (*host_flag != 0) return QVS_ETIMEOUT;   // a staged pass gave up waiting for its tile copies
  *E = h->host_res[0];
  if (grad) {
    for (int k = 0; k < p; ++k) {
      dg[k] = h->host_res[1 + k];
      dt[k] = h->host_res[1 + p + k];
    }
  }
  if (ex && grad) {   // per-term sums over the moments kernel's CTAs
    const int ns = p * ex->nterms;
    ExData& X = h->ex;
    std::vector<int> rm(3 * (size_t)ns, -1);
    for (int s2 = 0; s2 < ns; ++s2) rm[3 * (size_t)s2] = s2;
    QVS_TRY(X.mrowmap.ensure(sizeof(int) * rm.size()));
    QVS_TRY(X.mres.ensure(sizeof(double) * ns));
    QVS_CUDA_TRY(cudaMemcpyAsync(X.mrowmap.ptr, rm.data(), sizeof(int) * rm.size(), cudaMemcpyHostToDevice,
                                 h->stream));
    QVS_TRY(reduce_rows(h, ex->mpart, ex->mgrid, X.mrowmap.as<int>(), ns, X.mres.as<double>()));
    QVS_CUDA_TRY(cudaMemcpyAsync(dG, X.mres.ptr, sizeof(double) * ns, cudaMemcpyDeviceToHost, h->stream));
    QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->launches += 1;
  }
  return QVS_OK;
}

}  // namespace hc

static int hc_run(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E,
                  double* dg, double* dt) {
  if (h->n < 1) return QVS_EINVAL;
  const bool small = h->n <= hc::TB;
  if (small) QVS_TRY(ensure_q_vector(h));   // the one-CTA kernel reads q from memory
  if (h->precision == QVS_C64)
    return small ? hc::run_small<float>(h, p, gammas, ts, grad, E, dg, dt)
                 : hc::run_tiled<float>(h, p, gammas, ts, grad, E, dg, dt);
  return small ? hc::run_small<double>(h, p, gammas, ts, grad, E, dg, dt)
               : hc::run_tiled<double>(h, p, gammas, ts, grad, E, dg, dt);
}

// ex-QAOA: per-layer phase-angle forms, their tables, the g buffer and the moments kernel's inputs
static int ex_prepare(qvs_ctx* h, int p, const double* G, bool grad, hc::ExRun& run) {
  using namespace hc;
  ExData& X = h->ex;
  const int n = h->n, J = (int)X.terms.size();
  Plan pl;
  QVS_TRY(make_plan(n, p, pl));
  const uint32_t grid = 1u << (n - TB);
  // angle of layer k in turns: sum_j gamma_kj c_j s_j / 2pi with s_j = z_a z_b = 1 - 2x_a - 2x_b + 4 x_a x_b
  // (or z_a = 1 - 2 x_a), each coefficient reduced mod 1 turn into 32-bit fixed point
  auto fx = [](double x) -> int32_t {
    const double f = x - floor(x);
    return (int32_t)(uint32_t)(int64_t)llround(f * 4294967296.0);
  };
  std::vector<QuboCoef> coefs(p);
  for (int k = 0; k < p; ++k) {
    double c = 0.0;
    std::vector<double> hh(n, 0.0), jj((size_t)n * n, 0.0);
    for (int j = 0; j < J; ++j) {
      const ExTerm& t = X.terms[j];
      const double w = G[(size_t)k * J + j] * t.c / 6.283185307179586476925286766559;
      c += w;
      hh[t.a] -= 2.0 * w;
      if (t.b >= 0) {
        hh[t.b] -= 2.0 * w;
        jj[(size_t)t.a * n + t.b] += 4.0 * w;
        jj[(size_t)t.b * n + t.a] += 4.0 * w;
      }
    }
    QuboCoef& Q = coefs[k];
    Q.n = n;
    Q.F = 32;
    Q.c = fx(c);
    for (int b = 0; b < n; ++b) Q.h[b] = fx(hh[b]);
    for (int b = 0; b < n; ++b)
      for (int b2 = 0; b2 < n; ++b2) Q.J[b][b2] = b == b2 ? 0 : fx(jj[(size_t)b * n + b2]);
  }
  QVS_TRY(build_tables(h, pl, grid, coefs.data(), p, X.coef, X.tab, X.pp));
  run = ExRun{};
  run.tab = X.tab.as<int>();
  run.pp = &X.pp;
  run.nterms = J;
  if (grad) {
    QVS_TRY(X.g.ensure(sizeof(float) * (size_t)h->dim));
    std::vector<int2> tb(J);
    std::vector<float> tc(J);
    for (int j = 0; j < J; ++j) {
      tb[j] = make_int2(X.terms[j].a, X.terms[j].b);
      tc[j] = (float)X.terms[j].c;
    }
    QVS_TRY(X.mterms.ensure((sizeof(int2) + sizeof(float)) * (size_t)J));
    QVS_CUDA_TRY(cudaMemcpyAsync(X.mterms.ptr, tb.data(), sizeof(int2) * J, cudaMemcpyHostToDevice, h->stream));
    float* tcd = reinterpret_cast<float*>(X.mterms.as<int2>() + J);
    QVS_CUDA_TRY(cudaMemcpyAsync(tcd, tc.data(), sizeof(float) * J, cudaMemcpyHostToDevice, h->stream));
    run.g = X.g.as<float>();
    run.tbits = X.mterms.as<int2>();
    run.tc = tcd;
    run.mgrid = std::min<uint32_t>((uint32_t)(h->dim >> 12), 512u);
    QVS_TRY(X.mpart.ensure(sizeof(double) * (size_t)p * J * run.mgrid));
    run.mpart = X.mpart.as<double>();
    QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));   // the host term arrays go out of scope
  }
  return QVS_OK;
}

static int ex_check(qvs_ctx* h) {
  if (h->precision != QVS_C64 || h->n <= hc::TB || h->n > 32) return QVS_EUNSUPPORTED;
  if (h->ex.terms.empty()) return QVS_ESTATE;
  return QVS_OK;
}

int hc_evolve_ex(qvs_ctx* h, int p, const double* gammas, const double* ts) {
  QVS_TRY(ex_check(h));
  hc::ExRun run;
  QVS_TRY(ex_prepare(h, p, gammas, false, run));
  std::vector<double> zg(p, 0.0);
  double E = 0.0;
  QVS_TRY(hc::run_tiled<float>(h, p, zg.data(), ts, false, &E, nullptr, nullptr, &run, nullptr));
  h->E = E;
  h->have_E = true;
  return QVS_OK;
}

int hc_gradient_ex(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dG,
                   double* dt) {
  QVS_TRY(ex_check(h));
  if ((int)h->ex.terms.size() > hc::MT_MAX) return QVS_EUNSUPPORTED;
  hc::ExRun run;
  QVS_TRY(ex_prepare(h, p, gammas, true, run));
  std::vector<double> zg(p, 0.0), dg(p, 0.0);
  h->have_E = false;
  return hc::run_tiled<float>(h, p, zg.data(), ts, true, E, dg.data(), dt, &run, dG);
}

int hc_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts) {
  double E = 0.0;
  QVS_TRY(hc_run(h, p, gammas, ts, false, &E, nullptr, nullptr));
  h->E = E;
  h->have_E = true;
  return QVS_OK;
}

int hc_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                double* dt) {
  h->have_E = false;
  return hc_run(h, p, gammas, ts, true, E, dg, dt);
}

}  // namespace qvs

// ================================================================ batched persistent solve
//
// Many independent QAOA instances (each with its own n >= 12, p and quality vector) are solved
// by one persistent kernel: every CTA owns a workspace slot and repeatedly takes the next
// instance from a device-side counter (instances pre-sorted by decreasing cost, so the longest
// start first), then runs that instance's whole pass schedule - forward sweep, fused adjoint,
// reductions - walking its tiles itself, with a block barrier between passes. Small instances stay
// in L2 for their whole solve.

namespace qvs {
namespace hc {

constexpr int BATCH_MAX_LAYERS = 64;

struct BInst {
  int n, p, F, g;
  uint32_t ntiles;
  int th0;            // offset of the instance's p parameters / gradient entries
  int ck_c, nck;      // checkpoint interval (passes) and count
  int64_t qoff;       // offset of the instance's q in the concatenated quality buffer
  Tile tile[3];
  uint32_t gmask[3];
};

struct BatchArgs {
  int count;
  const BInst* inst;
  const int* order;          // processing order (by decreasing cost)
  const float* q;            // concatenated qualities
  const double* gammas;      // concatenated parameters
  const double* ts;
  double* out_E;             // [count]
  double* out_dg;            // concatenated like gammas
  double* out_dt;
  int* counter;
  const int* active;         // per-instance flags (NULL: every instance); 0 = skip
  unsigned char* ws;         // workspace slots
  size_t slot_bytes;
  int64_t dim_max;
  int nck_max;
};

// pass j (1-based) of an instance's forward schedule (same rules as make_plan)
__host__ __device__ __forceinline__ void bpass_info(const BInst& I, int j, int& type, int& shape, int& lb, int& la,
                                           int& lg) {
  const int p = I.p;
  if (I.g == 1) {
    type = 0;
    if (j == 1) { shape = F0; lb = -1; la = 0; lg = 0; }
    else if (j <= p) { shape = F1; lb = -1; la = j - 1; lg = j - 1; }
    else { shape = FE; lb = -1; la = -1; lg = -1; }
  } else if (I.g == 2) {
    type = (j - 1) % 2;
    if (j == 1) { shape = F0; lb = -1; la = 0; lg = 0; }
    else if (j <= p) { shape = F1; lb = j - 2; la = j - 1; lg = j - 1; }
    else { shape = FE; lb = p - 1; la = -1; lg = -1; }
  } else {
    type = three_type(j);
    if (j == 1) { shape = F0; lb = -1; la = 0; lg = 0; }
    else if (j == I.F) { shape = FE; lb = p - 1; la = -1; lg = -1; }
    else if (j % 2 == 0) { shape = F2; lb = (j - 2) / 2; la = -1; lg = -1; }
    else { shape = F1; lb = (j - 3) / 2; la = (j - 1) / 2; lg = (j - 1) / 2; }
  }
}

// Cost model of one instance's solve in the batched kernel, per amplitude summed over its passes:
// compulsory global-memory bytes (8 per complex64 vector read or written, 4 per quality read) and
// fp32 fused multiply-adds. A pass on the contiguous tile type rotates all 12 tile bits of a layer
// (the runtime masks give the others tangent 0); the two-layout form of the high types rotates the
// 8 bits 4..11. Each rotated bit costs 2 FMAs per amplitude and vector, plus 2 per amplitude for
// the adjoint accumulation; a phase costs about 8 (argument reduction and the complex product).
struct PassCost {
  double bytes, fma;
};
static PassCost batch_instance_cost(const BInst& I) {
  auto stored = [&](int j) { return j >= 1 && j <= I.F - 1 && j % I.ck_c == 0 && (j / I.ck_c) <= I.nck; };
  double bytes = 0.0, fma = 0.0;
  auto bits = [&](int type) { return (I.gmask[type] & 0xFu) ? (double)TB : 8.0; };
  for (int j = 1; j <= I.F; ++j) {   // forward
    int type, shape, lb, la, lg;
    bpass_info(I, j, type, shape, lb, la, lg);
    const double rot = 2.0 * bits(type) * ((lb >= 0) + (la >= 0));
    switch (shape) {
      case F0: bytes += 12; fma += rot + 8; break;
      case F1: bytes += 20; fma += rot + 8; break;
      case F2: bytes += 16; fma += rot; break;
      case FE: bytes += 20; fma += (lb >= 0 ? 8.0 * bits(type) : 0.0) + 4; break;   // rotate, E, lambda, undo
    }
  }
  for (int j = I.F - 1; j >= 1; --j) {   // adjoint
    int type, shape, lb, la, lg;
    bpass_info(I, j, type, shape, lb, la, lg);
    const double unrot = 6.0 * bits(type) * ((lb >= 0) + (la >= 0));
    const double psi_w = (j - 1 >= 1 && !stored(j - 1)) ? 8.0 : 0.0;
    switch (shape) {
      case F0: bytes += 20; fma += unrot + 4; break;                  // R0
      case F1: bytes += 28 + psi_w; fma += unrot + 16; break;         // R1
      case F2: bytes += 24 + psi_w; fma += unrot; break;              // R2
    }
  }
  const double dim = (double)((int64_t)1 << I.n);
  return {bytes * dim, fma * dim};
}

template <int TH>
__device__ __forceinline__ void run_shape_th(int shape, const PassArgs<float>& a, uint32_t t, uint32_t nt,
                                             unsigned char* sm) {
  switch (shape) {
    case F0: run_pass<float, F0, TH, true>(a, t, nt, sm); break;
    case F1: run_pass<float, F1, TH, true>(a, t, nt, sm); break;
    case F2: run_pass<float, F2, TH, true>(a, t, nt, sm); break;
    case FE: run_pass<float, FE, TH, true>(a, t, nt, sm); break;
    case R1: run_pass<float, R1, TH, true>(a, t, nt, sm); break;
    case R2: run_pass<float, R2, TH, true>(a, t, nt, sm); break;
    case R0: run_pass<float, R0, TH, true>(a, t, nt, sm); break;
  }
}
// a pass whose masks leave tile bits 0..3 alone (every high tile type of n <= 20) takes the
// two-layout form: one transpose per direction, and no tangent-0 rotations of the low bits
__device__ __forceinline__ void run_shape(int shape, const PassArgs<float>& a, uint32_t t, uint32_t nt,
                                          unsigned char* sm) {
  if ((a.mask_bef | a.mask_aft) & 0xFu) run_shape_th<TH_RUNTIME>(shape, a, t, nt, sm);
  else run_shape_th<TH_RUNTIME_HI>(shape, a, t, nt, sm);
}

__global__ void __launch_bounds__(NT, 2) batch_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_inst;
  __shared__ PassArgs<float> s_pa;
  __shared__ Frame s_fw[2 * BATCH_MAX_LAYERS + 2];   // psi frame after forward pass j
  const int tid = threadIdx.x;
  unsigned char* slot = a.ws + (size_t)blockIdx.x * a.slot_bytes;
  float2* W = reinterpret_cast<float2*>(slot);
  float2* Lm = W + a.dim_max;
  float2* K = Lm + a.dim_max;
  double* part = reinterpret_cast<double*>(K + (size_t)a.nck_max * a.dim_max);
  for (;;) {
    if (tid == 0) s_inst = atomicAdd(a.counter, 1);
    __syncthreads();
    const int idx = s_inst;
    __syncthreads();
    if (idx >= a.count) return;
    const int i = a.order[idx];
    if (a.active && !a.active[i]) continue;   // uniform across the CTA: i comes from shared memory
    const BInst& I = a.inst[i];
    const int F = I.F;
    const int64_t dim = (int64_t)1 << I.n;
    auto is_stored = [&](int j) { return j >= 1 && j <= F - 1 && j % I.ck_c == 0 && (j / I.ck_c) <= I.nck; };
    auto loc = [&](int j) -> float2* {
      return is_stored(j) ? K + (size_t)(j / I.ck_c - 1) * dim : W;
    };
    // frames of psi / lambda (thread 0 only; see the host driver)
    Frame fr{1.0, 0}, lf{1.0, 0}, pout{1.0, 0};
    for (int step = 0; step < 2 * F - 1; ++step) {
      const bool fwd = step < F;
      const int j = fwd ? step + 1 : 2 * F - 1 - step;   // forward 1..F, then F-1..1
      int type, shape, lb, la, lg;
      bpass_info(I, j, type, shape, lb, la, lg);
      if (tid == 0) {
        PassArgs<float> pa{};
        pa.tile = I.tile[type];
        pa.q = a.q + I.qoff;
        pa.mask_bef = lb >= 0 ? I.gmask[type] : 0u;
        pa.mask_aft = la >= 0 ? I.gmask[type] : 0u;
        pa.part = part;
        pa.init_amp = (float)rsqrt((double)dim);
        pa.gen_init = 1;
        pa.row_bef = pa.row_aft = pa.row_gam = pa.row_E = -1;
        const int G = __popc(I.gmask[type]);
        const double* gs = a.gammas + I.th0;
        const double* ts = a.ts + I.th0;
        if (fwd) {
          fwd_scalars<float>(pa, shape, lb, la, lg, G, I.n, I.p, gs, ts, fr, lf);
          pa.psi_in = j == 1 ? nullptr : loc(j - 1);
          if (j == F) {
            pa.lam_out = Lm;
            pa.row_bef = lb >= 0 ? 3 * (j - 1) : -1;
            pa.row_E = 3 * F;
          } else {
            pa.psi_out = loc(j);
            s_fw[j] = fr;
          }
        } else {
          const int rshape = shape == F0 ? R0 : (shape == F1 ? R1 : R2);
          Frame pf = (is_stored(j) || j == F - 1) ? s_fw[j] : pout;
          bwd_scalars<float>(pa, rshape, lb, la, lg, G, I.n, gs, ts, pf, lf);
          pout = pf;
          pa.psi_in = loc(j);
          pa.lam_in = Lm;
          pa.lam_out = Lm;
          pa.psi_out = (j - 1 >= 1 && !is_stored(j - 1)) ? W : nullptr;
          pa.row_bef = lb >= 0 ? 3 * (j - 1) + 0 : -1;
          pa.row_aft = la >= 0 ? 3 * (j - 1) + 1 : -1;
          pa.row_gam = lg >= 0 ? 3 * (j - 1) + 2 : -1;
        }
        s_pa = pa;
      }
      __syncthreads();
      const PassArgs<float> pa = s_pa;
      if (!fwd) shape = shape == F0 ? R0 : (shape == F1 ? R1 : R2);
      for (uint32_t t = 0; t < I.ntiles; ++t) run_shape(shape, pa, t, I.ntiles, smem_raw);
      __syncthreads();   // every tile of this pass is written before the next pass reads it
    }
    // deterministic reduction of the partial rows into the outputs
    const int p = I.p;
    if (tid < 1 + 2 * p) {
      double sum = 0.0;
      for (int j = 1; j <= F; ++j) {
        int type, shape, lb, la, lg;
        bpass_info(I, j, type, shape, lb, la, lg);
        int rows[2] = {-1, -1};
        if (tid == 0) rows[0] = j == F ? 3 * F : -1;
        else if (tid <= p) rows[0] = (lg == tid - 1) ? 3 * (j - 1) + 2 : -1;
        else {
          rows[0] = (lb == tid - 1 - p) ? 3 * (j - 1) + 0 : -1;
          rows[1] = (la == tid - 1 - p) ? 3 * (j - 1) + 1 : -1;
        }
        for (int r = 0; r < 2; ++r)
          if (rows[r] >= 0)
            for (uint32_t t = 0; t < I.ntiles; ++t) sum += part[(size_t)rows[r] * I.ntiles + t];
      }
      if (tid == 0) a.out_E[i] = sum;
      else if (tid <= p) a.out_dg[I.th0 + tid - 1] = sum;
      else a.out_dt[I.th0 + tid - 1 - p] = sum;
    }
    __syncthreads();
  }
}

}  // namespace hc
}  // namespace qvs

namespace qvs {
namespace hc {

int batch_launch(qvs_batch_t b, int ctas_per_sm, const int* active) {
  BatchArgs a{};
  a.active = active;
  a.count = b->count;
  a.inst = b->inst.as<BInst>();
  a.order = b->order.as<int>();
  a.q = b->q.as<float>();
  a.gammas = b->theta.as<double>();
  a.ts = a.gammas + b->total_p;
  a.out_E = b->out.as<double>();
  a.out_dg = a.out_E + b->count;
  a.out_dt = a.out_dg + b->total_p;
  a.counter = b->counter.as<int>();
  a.ws = b->ws.as<unsigned char>();
  a.slot_bytes = b->slot_bytes;
  a.dim_max = b->dim_max;
  a.nck_max = b->nck_max;
  const int grid = std::min(b->nslots, b->sms * ctas_per_sm);
  QVS_CUDA_TRY(cudaMemsetAsync(b->counter.ptr, 0, sizeof(int), b->stream));
  batch_kernel<<<grid, NT, 2 * SM_SLOTS * sizeof(float2), b->stream>>>(a);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

// Switch the batch to checkpoint policy pol: its instance table, slot size and workspace. The
// captured graphs name the old workspace and slot size, so they are dropped.
int batch_configure(qvs_batch_t b, int pol) {
  const size_t ws_bytes = b->slot_bytes_pol[pol] * (size_t)b->nslots;
  QVS_TRY(b->ws.ensure(ws_bytes));
  QVS_CUDA_TRY(cudaMemcpyAsync(b->inst.ptr, b->host_inst[pol].data(), b->host_inst[pol].size(), cudaMemcpyHostToDevice,
                               b->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->ckpt_policy = pol;
  b->slot_bytes = b->slot_bytes_pol[pol];
  b->nck_max = b->nck_max_pol[pol];
  b->model_bytes = b->model_bytes_pol[pol];
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->opt_graph) cudaGraphExecDestroy(b->opt_graph);
  b->graph = nullptr;
  b->opt_graph = nullptr;
  return QVS_OK;
}

// ---- persistent cache of tuned schedules
//
// A JSON file (QVS_TUNE_CACHE, else $HOME/.cache/qvs/batch_tune.json) with one entry per line:
//   {"key": "<gpu>|<sms>|<count>|<hash of the (n, p) multiset>", "ctas_per_sm": c, "ckpt_policy": k, "ms": t}
// Unreadable or unwritable files are ignored (the batch is then tuned every time).
static std::string tune_cache_path() {
  if (const char* e = getenv("QVS_TUNE_CACHE")) return e;
  const char* home = getenv("HOME");
  if (!home) return "";
  const std::string dir = std::string(home) + "/.cache/qvs";
  mkdir((std::string(home) + "/.cache").c_str(), 0755);
  mkdir(dir.c_str(), 0755);
  return dir + "/batch_tune.json";
}

static std::string tune_key(qvs_batch_t b) {
  std::vector<uint32_t> np(b->count);
  for (int i = 0; i < b->count; ++i) np[i] = ((uint32_t)b->n[i] << 8) | (uint32_t)b->p[i];
  std::sort(np.begin(), np.end());
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the sorted (n, p) pairs
  for (uint32_t v : np)
    for (int k = 0; k < 4; ++k) {
      h ^= (v >> (8 * k)) & 0xFFu;
      h *= 1099511628211ull;
    }
  std::string name = b->gpu_name;
  for (char& c : name)
    if (c == '"' || c == '|' || c == '\\') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|%d|%d|%016llx", name.c_str(), b->sms, b->count, (unsigned long long)h);
  return buf;
}

static std::vector<std::string> tune_cache_lines(const std::string& path) {
  std::vector<std::string> out;
  if (path.empty()) return out;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    if (l.find("{\"key\": \"") != std::string::npos) {
      while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == ' ')) l.pop_back();
      out.push_back(l);
    }
  }
  fclose(f);
  return out;
}

static bool tune_cache_lookup(const std::string& key, int* ctas, int* pol) {
  const std::string needle = "{\"key\": \"" + key + "\",";
  for (const std::string& l : tune_cache_lines(tune_cache_path())) {
    if (l.compare(0, needle.size(), needle) != 0) continue;
    int c = 0, k = -1;
    if (sscanf(l.c_str() + needle.size(), " \"ctas_per_sm\": %d, \"ckpt_policy\": %d", &c, &k) == 2 && c >= 1 &&
        c <= 2 && (k == 0 || k == 1)) {
      *ctas = c;
      *pol = k;
      return true;
    }
  }
  return false;
}

static void tune_cache_store(const std::string& key, int ctas, int pol, double ms) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  std::vector<std::string> lines = tune_cache_lines(path);
  const std::string needle = "{\"key\": \"" + key + "\",";
  lines.erase(std::remove_if(lines.begin(), lines.end(),
                             [&](const std::string& l) { return l.compare(0, needle.size(), needle) == 0; }),
              lines.end());
  char buf[512];
  snprintf(buf, sizeof(buf), "{\"key\": \"%s\", \"ctas_per_sm\": %d, \"ckpt_policy\": %d, \"ms\": %.3f}", key.c_str(),
           ctas, pol, ms);
  lines.push_back(buf);
  const std::string tmp = path + ".tmp." + std::to_string((long long)getpid());   // one per process
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fputs("{\"batch_schedules\": [\n", f);
  for (size_t i = 0; i < lines.size(); ++i) fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
  fputs("]}\n", f);
  const bool ok = fclose(f) == 0;
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

// Choose the schedule on the first solve: a cached choice for the same GPU and instance mix, else
// one timed launch per candidate (CTAs per SM 1 or 2, checkpoint policy 0 or 1; a policy whose
// workspace cannot be allocated is skipped), keeping the fastest. Needs b->theta set.
int batch_autotune(qvs_batch_t b) {
  if (b->ctas_per_sm > 0) return QVS_OK;
  const std::string key = tune_key(b);
  int cc = 0, cp = 0;
  if (tune_cache_lookup(key, &cc, &cp) && batch_configure(b, cp) == QVS_OK) {
    b->ctas_per_sm = cc;
    b->from_cache = true;
    return QVS_OK;
  }
  (void)cudaGetLastError();
  cudaEvent_t e0, e1;
  QVS_CUDA_TRY(cudaEventCreate(&e0));
  QVS_CUDA_TRY(cudaEventCreate(&e1));
  double best = 1e30;
  int choice = 1, choice_pol = 0;
  for (int pol = 0; pol < 2; ++pol) {
    if (batch_configure(b, pol) != QVS_OK) {   // e.g. the larger workspace does not fit
      (void)cudaGetLastError();
      continue;
    }
    for (int c = 1; c <= 2; ++c) {
      int st = QVS_OK;
      if (cudaEventRecord(e0, b->stream) != cudaSuccess) st = QVS_ECUDA;
      if (st == QVS_OK) st = batch_launch(b, c, nullptr);
      if (st == QVS_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = QVS_ECUDA;
      float ms = 0.f;
      if (st == QVS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = QVS_ECUDA;
      if (st != QVS_OK) {
        (void)cudaGetLastError();
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      b->trial_ms4[2 * pol + c - 1] = ms;
      if (pol == 0) b->tuned_ms[c] = ms;
      if (ms < best) {
        best = ms;
        choice = c;
        choice_pol = pol;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e30) return QVS_ENOMEM;
  QVS_TRY(batch_configure(b, choice_pol));
  b->ctas_per_sm = choice;
  tune_cache_store(key, choice, choice_pol, best);
  return QVS_OK;
}

}  // namespace hc
}  // namespace qvs

static int qvs_batch_create_impl(qvs_batch_t* out, int count, const int32_t* n_qubits, const int32_t* layers,
                                 void* stream) {
  using namespace qvs;
  using namespace qvs::hc;
  if (!out || count < 1 || count > (1 << 20) || !n_qubits || !layers) return QVS_EINVAL;
  *out = nullptr;
  qvs_batch* b = new (std::nothrow) qvs_batch();
  if (!b) return QVS_ENOMEM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  std::vector<BInst> inst(count), inst_all(count);   // checkpoint policies 0 and 1
  std::vector<double> cost(count);
  int64_t qtot = 0;
  int ptot = 0;
  size_t max_rows_tiles = 0;
  for (int i = 0; i < count; ++i) {
    const int n = n_qubits[i], p = layers[i];
    if (n < TB || n > 28 || p < 1 || p > BATCH_MAX_LAYERS) {
      delete b;
      return n < TB ? QVS_EUNSUPPORTED : QVS_EINVAL;
    }
    Plan pl;
    const int st = make_plan(n, p, pl);
    if (st != QVS_OK) {
      delete b;
      return st;
    }
    BInst& I = inst[i];
    I.n = n;
    I.p = p;
    I.F = pl.F;
    I.g = pl.g;
    I.ntiles = 1u << (n - TB);
    I.th0 = ptot;
    const int ckl = (int)ceil(sqrt((double)p) - 1e-9);
    I.ck_c = std::max(1, ckl * std::max(1, pl.g - 1));
    I.nck = (pl.F - 1) / I.ck_c;
    I.qoff = qtot;
    for (int t = 0; t < 3; ++t) {
      I.tile[t] = pl.tile[t];
      I.gmask[t] = pl.gmask[t];
    }
    b->n.push_back(n);
    b->p.push_back(p);
    b->th0.push_back(ptot);
    b->qoff.push_back(qtot);
    BInst& A = inst_all[i];
    A = I;
    A.ck_c = 1;
    A.nck = pl.F - 1;
    b->dim_max = std::max<int64_t>(b->dim_max, (int64_t)1 << n);
    b->nck_max_pol[0] = std::max(b->nck_max_pol[0], I.nck);
    b->nck_max_pol[1] = std::max(b->nck_max_pol[1], A.nck);
    max_rows_tiles = std::max(max_rows_tiles, (size_t)(3 * pl.F + 1) * I.ntiles);
    cost[i] = (double)((int64_t)1 << n) * (2 * pl.F - 1);
    const PassCost pc = batch_instance_cost(I);
    b->model_bytes_pol[0] += pc.bytes;
    b->model_bytes_pol[1] += batch_instance_cost(A).bytes;
    b->model_fma += pc.fma;
    b->amp_layers += (double)((int64_t)1 << n) * p;
    qtot += (int64_t)1 << n;
    ptot += p;
  }
  b->total_q = qtot;
  b->total_p = ptot;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return QVS_ECUDA;
  }
  b->sms = prop.multiProcessorCount;
  b->gpu_name = prop.name;
  b->nslots = 2 * b->sms;
  for (int pol = 0; pol < 2; ++pol) {
    b->slot_bytes_pol[pol] =
        (sizeof(float2) * (size_t)b->dim_max * (2 + b->nck_max_pol[pol]) + sizeof(double) * max_rows_tiles + 255) &
        ~(size_t)255;
    const std::vector<BInst>& src = pol ? inst_all : inst;
    b->host_inst[pol].assign(reinterpret_cast<const unsigned char*>(src.data()),
                             reinterpret_cast<const unsigned char*>(src.data() + count));
  }
  b->ckpt_policy = 0;
  b->slot_bytes = b->slot_bytes_pol[0];
  b->nck_max = b->nck_max_pol[0];
  b->model_bytes = b->model_bytes_pol[0];
  int st = QVS_OK;
  if ((st = b->inst.ensure(sizeof(BInst) * count)) != QVS_OK || (st = b->order.ensure(sizeof(int) * count)) != QVS_OK ||
      (st = b->theta.ensure(sizeof(double) * 2 * (size_t)ptot)) != QVS_OK ||
      (st = b->out.ensure(sizeof(double) * ((size_t)count + 2 * (size_t)ptot))) != QVS_OK ||
      (st = b->counter.ensure(sizeof(int))) != QVS_OK ||
      (st = b->ws.ensure(b->slot_bytes * (size_t)b->nslots)) != QVS_OK) {
    qvs_batch_destroy(b);
    return st;
  }
  if (cudaMallocHost((void**)&b->host_theta, sizeof(double) * 2 * (size_t)ptot) != cudaSuccess ||
      cudaMallocHost((void**)&b->host_out, sizeof(double) * ((size_t)count + 2 * (size_t)ptot)) != cudaSuccess) {
    (void)cudaGetLastError();
    qvs_batch_destroy(b);
    return QVS_ENOMEM;
  }
  if (cudaMemcpyAsync(b->inst.ptr, inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->order.ptr, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(2 * SM_SLOTS * sizeof(float2))) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    qvs_batch_destroy(b);
    return QVS_ECUDA;
  }
  *out = b;
  return QVS_OK;
}

extern "C" int qvs_batch_create(qvs_batch_t* out, int count, const int32_t* n_qubits, const int32_t* layers,
                                void* stream) {
  return qvs::guarded([&] { return qvs_batch_create_impl(out, count, n_qubits, layers, stream); });
}

// Captured graphs hold the quality pointer: drop them when the buffer moves.
static int batch_ensure_q(qvs_batch_t b, size_t bytes) {
  void* before = b->q.ptr;
  QVS_TRY(b->q.ensure(bytes));
  if (b->q.ptr != before) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->opt_graph) cudaGraphExecDestroy(b->opt_graph);
    b->graph = nullptr;
    b->opt_graph = nullptr;
  }
  return QVS_OK;
}

// Point every instance's quality offset at its own segment (shared = false) or at the one
// shared vector (shared = true); the kernel reads the offsets from the device instance table.
static int batch_set_qoffsets(qvs_batch_t b, bool shared) {
  using namespace qvs::hc;
  if (b->shared_q == shared && b->have_q) return QVS_OK;
  for (int pol = 0; pol < 2; ++pol) {
    BInst* inst = reinterpret_cast<BInst*>(b->host_inst[pol].data());
    for (int i = 0; i < b->count; ++i) inst[i].qoff = shared ? 0 : b->qoff[i];
  }
  QVS_CUDA_TRY(cudaMemcpyAsync(b->inst.ptr, b->host_inst[b->ckpt_policy].data(), sizeof(BInst) * b->count,
                               cudaMemcpyHostToDevice, b->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->shared_q = shared;
  return QVS_OK;
}

extern "C" int qvs_batch_set_quality(qvs_batch_t b, const float* q, int on_device) {
  if (!b || !q) return QVS_EINVAL;
  QVS_TRY(batch_ensure_q(b, sizeof(float) * (size_t)b->total_q));
  QVS_CUDA_TRY(cudaMemcpyAsync(b->q.ptr, q, sizeof(float) * (size_t)b->total_q,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  QVS_TRY(batch_set_qoffsets(b, false));
  b->have_q = true;
  return QVS_OK;
}

extern "C" int qvs_batch_set_quality_shared(qvs_batch_t b, const float* q, int on_device) {
  if (!b || !q) return QVS_EINVAL;
  for (int i = 1; i < b->count; ++i)
    if (b->n[i] != b->n[0]) return QVS_EINVAL;
  const size_t dim = (size_t)1 << b->n[0];
  QVS_TRY(batch_ensure_q(b, sizeof(float) * dim));
  QVS_CUDA_TRY(cudaMemcpyAsync(b->q.ptr, q, sizeof(float) * dim,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  QVS_TRY(batch_set_qoffsets(b, true));
  b->have_q = true;
  return QVS_OK;
}

extern "C" int qvs_batch_gradient(qvs_batch_t b, const double* gammas, const double* ts, double* E, double* dgamma,
                                  double* dt) {
  using namespace qvs;
  if (!b || !gammas || !ts || !E || !dgamma || !dt) return QVS_EINVAL;
  if (!b->have_q) return QVS_ESTATE;
  const size_t P = (size_t)b->total_p;
  for (size_t k = 0; k < P; ++k)
    if (!isfinite(gammas[k]) || !isfinite(ts[k])) return QVS_EINVAL;
  memcpy(b->host_theta, gammas, sizeof(double) * P);
  memcpy(b->host_theta + P, ts, sizeof(double) * P);
  if (b->ctas_per_sm == 0) {
    QVS_CUDA_TRY(cudaMemcpyAsync(b->theta.ptr, b->host_theta, sizeof(double) * 2 * P, cudaMemcpyHostToDevice,
                                 b->stream));
    QVS_TRY(hc::batch_autotune(b));
  }
  if (!b->graph) {
    // capture the whole solve (parameters in, kernel, results out) as a CUDA graph
    cudaStream_t cs;
    QVS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const cudaStream_t keep = b->stream;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cs);
      (void)cudaGetLastError();
      return QVS_ECUDA;
    }
    b->stream = cs;
    int st = QVS_OK;
    if (cudaMemcpyAsync(b->theta.ptr, b->host_theta, sizeof(double) * 2 * P, cudaMemcpyHostToDevice, cs) != cudaSuccess)
      st = QVS_ECUDA;
    if (st == QVS_OK) st = hc::batch_launch(b, b->ctas_per_sm, nullptr);
    if (st == QVS_OK &&
        cudaMemcpyAsync(b->host_out, b->out.ptr, sizeof(double) * ((size_t)b->count + 2 * P), cudaMemcpyDeviceToHost,
                        cs) != cudaSuccess)
      st = QVS_ECUDA;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    b->stream = keep;
    cudaStreamDestroy(cs);
    if (st != QVS_OK || ce != cudaSuccess) {   // a failed capture leaves no graph behind
      if (ce == cudaSuccess && g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      return st != QVS_OK ? st : QVS_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    QVS_CUDA_TRY(ie);
  }
  QVS_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(b->stream));
  memcpy(E, b->host_out, sizeof(double) * b->count);
  memcpy(dgamma, b->host_out + b->count, sizeof(double) * P);
  memcpy(dt, b->host_out + b->count + P, sizeof(double) * P);
  return QVS_OK;
}

extern "C" int qvs_batch_set_schedule(qvs_batch_t b, int ctas_per_sm, int ckpt_policy) {
  if (!b || ctas_per_sm < 0 || ctas_per_sm > 2 || (ckpt_policy != 0 && ckpt_policy != 1)) return QVS_EINVAL;
  QVS_TRY(qvs::hc::batch_configure(b, ckpt_policy));
  b->ctas_per_sm = ctas_per_sm;   // 0: the autotuner chooses again on the next solve
  b->from_cache = false;
  return QVS_OK;
}

extern "C" int qvs_batch_info(qvs_batch_t b, qvs_batch_info_t* info) {
  if (!b || !info) return QVS_EINVAL;
  memset(info, 0, sizeof(*info));
  info->ctas_per_sm = b->ctas_per_sm;
  info->trial_ms[0] = b->tuned_ms[1];
  info->trial_ms[1] = b->tuned_ms[2];
  info->ckpt_policy = b->ckpt_policy;
  info->from_cache = b->from_cache ? 1 : 0;
  for (int k = 0; k < 4; ++k) info->trial_ms_all[k] = b->trial_ms4[k];
  info->bytes_per_solve = b->model_bytes;
  info->fma_per_solve = b->model_fma;
  info->amp_layers = b->amp_layers;
  info->shared_quality = b->shared_q ? 1 : 0;
  return QVS_OK;
}

extern "C" int qvs_batch_destroy(qvs_batch_t b) {
  if (!b) return QVS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->opt_graph) cudaGraphExecDestroy(b->opt_graph);
  b->opt_state.release();
  b->opt_vec.release();
  b->opt_H.release();
  b->opt_active.release();
  b->opt_nactive.release();
  if (b->host_nactive) cudaFreeHost(b->host_nactive);
  b->inst.release();
  b->order.release();
  b->q.release();
  b->theta.release();
  b->out.release();
  b->counter.release();
  b->ws.release();
  if (b->host_theta) cudaFreeHost(b->host_theta);
  if (b->host_out) cudaFreeHost(b->host_out);
  delete b;
  (void)cudaGetLastError();
  return QVS_OK;
}

extern "C" int qvs_hypercube_plan(int n_qubits, int p, int max_passes, int* n_passes, int32_t* shape, int32_t* type,
                                  uint32_t* rot_bits, int32_t* layer_before, int32_t* layer_after,
                                  int32_t* layer_phase) {
  using namespace qvs::hc;
  if (!n_passes || n_qubits < TB || n_qubits > 32 || p < 1 || p > 4096 || max_passes < 0) return QVS_EINVAL;
  Plan pl;
  QVS_TRY(make_plan(n_qubits, p, pl));
  *n_passes = pl.F;
  if (!shape) return QVS_OK;   // size query
  if (pl.F > max_passes || !type || !rot_bits || !layer_before || !layer_after || !layer_phase) return QVS_EINVAL;
  for (int j = 1; j <= pl.F; ++j) {
    const PassInfo& q = pl.pass[j];
    const Tile& t = pl.tile[q.type];
    const int s = __builtin_popcount(t.smask);
    uint32_t bits = 0;   // tile bit i is index bit i below s and index bit i + hshift above
    for (int i = 0; i < TB; ++i)
      if ((pl.gmask[q.type] >> i) & 1u) bits |= 1u << (i < s ? i : i + t.hshift);
    shape[j - 1] = q.shape;
    type[j - 1] = q.type;
    rot_bits[j - 1] = bits;
    layer_before[j - 1] = q.lb;
    layer_after[j - 1] = q.la;
    layer_phase[j - 1] = q.lg;
  }
  return QVS_OK;
}
