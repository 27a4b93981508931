// Internal declarations shared by the libqvs translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qvs.h"

#define QVS_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) {                       \
      (void)cudaGetLastError();                    \
      return _e == cudaErrorMemoryAllocation ? QVS_ENOMEM : QVS_ECUDA; \
    }                                              \
  } while (0)

#define QVS_TRY(expr)                 \
  do {                                \
    int _s = (expr);                  \
    if (_s != QVS_OK) return _s;      \
  } while (0)

namespace qvs {

// Run f() (an entry point's body) so that no C++ exception crosses the C ABI: a host allocation
// that fails (std::bad_alloc, or a size past std::vector's limit) becomes QVS_ENOMEM.
template <class F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return QVS_ENOMEM;
  } catch (const std::length_error&) {
    return QVS_ENOMEM;
  } catch (...) {
    return QVS_EINVAL;
  }
}

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device, once per device:
// the attribute belongs to the device, so a process that drives several GPUs sets it on each.
// `done` holds one bit per device index (devices >= 64 set it on every call).
inline int smem_limit_once(const void* fn, std::atomic<uint64_t>& done, int bytes) {
  int dev = 0;
  QVS_CUDA_TRY(cudaGetDevice(&dev));
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return QVS_OK;
  QVS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
  return QVS_OK;
}

// Device allocator of a handle: the alloc/dealloc hooks given to qvs_create (both NULL: the
// CUDA runtime's cudaMalloc / cudaFree).
struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*dealloc)(void*, void*) = nullptr;
  void* ctx = nullptr;
};

// The allocator DevBuf::ensure uses on the calling thread. Every public entry point that works on
// a handle sets it to the handle's allocator for the duration of the call (AllocScope); outside
// such a call it is NULL and buffers come from cudaMalloc (batched solves, generators).
const Allocator* current_allocator();
struct AllocScope {
  explicit AllocScope(const Allocator* a);
  ~AllocScope();
  AllocScope(const AllocScope&) = delete;
  AllocScope& operator=(const AllocScope&) = delete;
  const Allocator* prev;
};

// Device buffer owned by a handle. It remembers the allocator that made its block, so release()
// always returns the block to the same allocator.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  Allocator made_by;
  int ensure(size_t b) {
    if (b <= bytes && ptr) return QVS_OK;
    release();
    if (b == 0) return QVS_OK;
    const Allocator* a = current_allocator();
    if (a && a->alloc) {
      void* p = a->alloc(b, a->ctx);
      if (!p) return QVS_ENOMEM;
      if (reinterpret_cast<uintptr_t>(p) & 255u) {   // the hook must return 256-byte aligned blocks
        if (a->dealloc) a->dealloc(p, a->ctx);
        return QVS_EINVAL;
      }
      ptr = p;
      made_by = *a;
    } else {
      cudaError_t e = cudaMalloc(&ptr, b);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ptr = nullptr;
        return QVS_ENOMEM;
      }
      made_by = Allocator{};
    }
    bytes = b;
    return QVS_OK;
  }
  void release() {
    if (ptr) {
      if (made_by.alloc) {
        if (made_by.dealloc) made_by.dealloc(ptr, made_by.ctx);
      } else {
        cudaFree(ptr);
      }
    }
    ptr = nullptr;
    bytes = 0;
    made_by = Allocator{};
  }
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Quadratic quality in fixed point (qvs_set_quality_qubo): q(x) = 2^-F (c + sum_b h_b x_b +
// sum_{b<b'} J_bb' x_b x_b') over INDEX bits b (qubit u = bit n-1-u); J symmetric, zero diagonal.
// Every sum of these integers stays below 2^30 in magnitude.
struct QuboCoef {
  int n = 0, F = 0;
  int32_t c = 0;
  int32_t h[32] = {};
  int32_t J[32][32] = {};
};
// Round a qubit-indexed quadratic form to the fixed-point grid (quality.cu). QVS_EINVAL for n
// outside 1..32 or a non-finite coefficient.
int qubo_quantize(int n, double c, const double* hlin, const double* J, QuboCoef* out);
// Write q(i) = float(integer sum) * 2^-F for i < 2^n into out (F32 or F64), stream-ordered.
int qubo_generate(const QuboCoef& Q, int out_dtype, void* out, cudaStream_t stream);

struct QuboData {
  bool on = false;            // the handle's quality is this quadratic form
  bool materialized = false;  // h->q holds it as a vector (paths that read q from memory)
  QuboCoef coef;
  DevBuf dcoef;               // QuboCoef on the device (table builder)
  DevBuf tab;                 // hypercube tables: per tile type and frame, CTA rows + thread rows
  bool tab_valid = false;
  std::vector<int32_t> pp;    // per tile type and frame: 16 register pair sums
};

// ex-QAOA phase terms (qvs_set_phase_terms): Sigma_j = c_j Z_a Z_b (b < 0: c_j Z_a) over INDEX bits.
struct ExTerm {
  int32_t a, b;
  double c;
};
struct ExData {
  std::vector<ExTerm> terms;  // empty: plain QAOA phase
  DevBuf coef;                // per-layer QuboCoef of the phase angle in 2^-32 turns
  DevBuf tab;                 // per layer, tile type and frame: CTA rows + thread rows
  std::vector<int32_t> pp;    // per layer, tile type and frame: 16 register pair sums
  DevBuf g;                   // float[dim]: 2 Im(conj(lambda) phi) at one phase point
  DevBuf mterms;              // int2[nterms] index bits, float[nterms] coefficients
  DevBuf mpart;               // double[p * nterms * grid] moment partial rows
  DevBuf mrowmap, mres;       // identity row map and final per-term sums
};

// Circulant mixer data: eigenvalues in the order the FFT passes produce them.
struct CircData {
  DevBuf lam;           // float2[dim]: eigenvalues (hi, lo) in row-spectral thread-major order
  DevBuf qT;            // float[dim]: q in column-pass thread-major order
  bool qT_valid = false;
};

// CSR mixer data.
struct CsrData {
  DevBuf rowptr, colind, values;
  int64_t nnz = 0;
  bool has_values = false;
  float implicit_value = 0.f;
  double spec_lo = 0, spec_hi = 0, tol = 1e-7;
  double gersh = 0;         // Gershgorin radius (0 when the caller gave the interval)
  // matrix-free XY ring on the Hamming-weight-k states of n qubits (QVS_MIX_XY_RING)
  bool xy = false;
  int xy_n = 0, xy_k = 0;
  DevBuf states;            // uint2 per row: its basis state (rows in increasing state order) and the
                            // row of its closing-pair neighbour (-1: bits 0 and n-1 agree)
  DevBuf binom;             // int32 binomial table
};

}  // namespace qvs

struct qvs_ctx {
  int64_t dim = 0;
  qvs::Allocator allocator;   // qvs_create's hooks (default: cudaMalloc / cudaFree)
  int n = 0;                // log2(dim) when dim is a power of two, else -1
  int precision = QVS_C64;
  cudaStream_t stream = nullptr;
  int device = 0;

  bool have_q = false, have_mixer = false, have_psi0 = false;
  int mixer = 0;
  qvs::DevBuf q;            // float[dim] (C64) or double[dim] (C128)
  qvs::DevBuf psi0;         // explicit initial state
  qvs::DevBuf psi;          // working state / final state of qvs_evolve
  qvs::DevBuf lam;          // adjoint vector
  qvs::DevBuf ckpt;         // checkpoint states (contiguous slots)
  qvs::DevBuf part;         // per-CTA fp64 partial sums (reduction scratch)
  qvs::DevBuf res;          // double[1 + 2p] final reductions
  qvs::DevBuf rowmap;       // int[...] reduction row map
  qvs::DevBuf work;         // mixer-specific scratch
  qvs::DevBuf flags;        // int error flags written by bounded device waits
  bool staged = true;       // QVS_OPT_STAGED
  double* host_res = nullptr;   // pinned, 1 + 2 * host_res_cap doubles
  int host_res_cap = 0;

  int sms = 0;               // multiprocessors of the device (grid sizing of persistent kernels)
  int ckpt_layers = 0;
  bool have_E = false;
  double E = 0.0;
  int64_t launches = 0;

  qvs::CircData circ;
  qvs::CsrData csr;
  qvs::QuboData qubo;
  qvs::ExData ex;

  // QVS_OPT_PROFILE: per-kernel event timing
  struct KStat {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
  };
  struct Pending {
    int id;
    double bytes;
    cudaEvent_t a, b;
  };
  bool profile = false;
  std::vector<KStat> kstats;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> evpool;
};

namespace qvs {

// complex element size in bytes for the handle precision
inline size_t elem_bytes(const qvs_ctx* h) { return h->precision == QVS_C128 ? 16 : 8; }

int ensure_host_res(qvs_ctx* h, int p);

// Profiling: prof_begin records a start event (when QVS_OPT_PROFILE is on) and returns a token;
// prof_end records the end event for kernel `name` moving `bytes` algorithmic bytes; prof_flush
// (after the stream has been synchronised) folds the elapsed times into the statistics.
int prof_begin(qvs_ctx* h, cudaEvent_t* start);
int prof_end(qvs_ctx* h, const char* name, double bytes, cudaEvent_t start);
int prof_flush(qvs_ctx* h);
void prof_release(qvs_ctx* h);

// Materialise a quadratic quality into h->q (no-op for a vector quality); api.cu
int ensure_q_vector(qvs_ctx* h);

// hypercube (QAOA) path: hypercube.cu
int hc_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts);
int hc_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                double* dt);
// ex-QAOA on the tiled hypercube path: gammas / dG hold p * nterms values (layer-major)
int hc_evolve_ex(qvs_ctx* h, int p, const double* gammas, const double* ts);
int hc_gradient_ex(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dG,
                   double* dt);

// circulant (QWOA) path: circulant.cu
int circ_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d);
int circ_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts);
int circ_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                  double* dt);

// QAOAz parity-ring mixer path: parity.cu
int parity_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d);
int parity_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts);
int parity_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                    double* dt);

// CSR Chebyshev path: csr_cheb.cu
int csr_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d);
int xy_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d);
namespace hc {
void* tensor_map_encode_fn();   // cuTensorMapEncodeTiled from the driver, or NULL
}
int csr_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts);
int csr_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                 double* dt);

// Final deterministic reduction of per-CTA partial rows into result slots (reduce.cu).
// slot s = sum over rows rowmap[s*3 + 0..2] (-1 = unused) of part[row * nblk + b], b < nblk.
int reduce_rows(qvs_ctx* h, const double* part, int64_t nblk, const int* rowmap_dev, int nslots,
                double* out_dev);

// float-float turns of an angle gamma: gamma / (2 pi) split into hi + lo floats.
__host__ __device__ inline void turns_split(double gamma, float* hi, float* lo) {
  const double two_pi = 6.283185307179586476925286766559;
  double g = gamma / two_pi;
  float h = (float)g;
  *hi = h;
  *lo = (float)(g - (double)h);
}

}  // namespace qvs
