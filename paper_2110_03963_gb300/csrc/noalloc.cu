// Allocation-free variant of the small-state solve (objective + adjoint gradient of the QAOA
// hypercube ansatz for states of at most 2^12 amplitudes).
//
// Some callers cannot allocate device memory at the time they need a solve: code that runs inside
// an allocator or memory-pool callback, in a real-time loop whose memory budget is fixed up front,
// or in a host runtime that owns all device memory and forbids libraries from taking more. For them
// qvs_gradient_small_noalloc takes every input and output from the caller and keeps its only
// scratch - the forward states the adjoint sweep reads back - in one file-scope device array of
// fixed size, so it never calls cudaMalloc, cudaFree or any allocating routine.
#include <math.h>
#include <string.h>

#include <mutex>

#include "hc_kernels.cuh"
#include "qvs_internal.h"

namespace qvs {
namespace na {

constexpr size_t kScratchBytes = (size_t)QVS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxLayers = QVS_NOALLOC_MAX_LAYERS;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device (each device that loads the library holds its own copy
// until the process exits). Host code must not use this name as a device address: it resolves
// the address with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

template <class T>
struct Args {
  int n, p;
  const T* q;
  typename hc::Cx<T>::t* states;   // scratch: p forward states of 2^n amplitudes
  double* out;                     // caller's [1 + 2p]: E, dgamma, dt
  double ang[3 * kMaxLayers];      // cos t_k, sin t_k, gamma_k
};

template <class T>
__device__ __forceinline__ double block_sum(double v, double* red) {
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

template <class C, class T>
__device__ void rotate_all(C* s, int n, T c, T sn) {
  const int dim = 1 << n;
  for (int b = 0; b < n; ++b) {
    const int h = 1 << b;
    for (int k = threadIdx.x; k < dim / 2; k += blockDim.x) {
      const int i = ((k >> b) << (b + 1)) | (k & (h - 1));
      hc::rot_normal(s[i], s[i | h], c, sn);
    }
    __syncthreads();
  }
}

// One CTA: the whole state in shared memory, the forward states in the static scratch.
template <class T>
__global__ void __launch_bounds__(256) solve_kernel(const __grid_constant__ Args<T> a) {
  using C = typename hc::Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int dim = 1 << a.n;
  C* ps = reinterpret_cast<C*>(smem_raw);
  C* ls = ps + dim;
  const T amp = (T)rsqrt((double)dim);
  for (int i = threadIdx.x; i < dim; i += blockDim.x) {
    ps[i].x = amp;
    ps[i].y = T(0);
  }
  __syncthreads();
  for (int k = 0; k < a.p; ++k) {
    const double g = a.ang[3 * k + 2];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      double sd, cd;
      sincos(g * (double)a.q[i], &sd, &cd);
      ps[i] = hc::cmul_conj(ps[i], (T)cd, (T)sd);
    }
    __syncthreads();
    rotate_all<C, T>(ps, a.n, (T)a.ang[3 * k], (T)a.ang[3 * k + 1]);
    for (int i = threadIdx.x; i < dim; i += blockDim.x) a.states[(size_t)k * dim + i] = ps[i];
  }
  double e = 0.0;
  for (int i = threadIdx.x; i < dim; i += blockDim.x)
    e += (double)a.q[i] * ((double)ps[i].x * ps[i].x + (double)ps[i].y * ps[i].y);
  e = block_sum<T>(e, red);
  if (threadIdx.x == 0) a.out[0] = e;
  for (int i = threadIdx.x; i < dim; i += blockDim.x) {
    ls[i].x = a.q[i] * ps[i].x;
    ls[i].y = a.q[i] * ps[i].y;
  }
  __syncthreads();
  for (int k = a.p - 1; k >= 0; --k) {
    for (int i = threadIdx.x; i < dim; i += blockDim.x) ps[i] = a.states[(size_t)k * dim + i];
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      C w;
      w.x = T(0);
      w.y = T(0);
      for (int b = 0; b < a.n; ++b) {
        w.x += ps[i ^ (1 << b)].x;
        w.y += ps[i ^ (1 << b)].y;
      }
      acc += (double)hc::imdot(ls[i], w);
    }
    acc = block_sum<T>(acc, red);
    if (threadIdx.x == 0) a.out[1 + a.p + k] = 2.0 * acc;
    const T c = (T)a.ang[3 * k], s = (T)a.ang[3 * k + 1];
    rotate_all<C, T>(ps, a.n, c, -s);
    rotate_all<C, T>(ls, a.n, c, -s);
    double ag = 0.0;
    for (int i = threadIdx.x; i < dim; i += blockDim.x)
      ag += (double)a.q[i] * (double)hc::imdot(ls[i], ps[i]);
    ag = block_sum<T>(ag, red);
    if (threadIdx.x == 0) a.out[1 + k] = 2.0 * ag;
    const double g = a.ang[3 * k + 2];
    for (int i = threadIdx.x; i < dim; i += blockDim.x) {
      double sd, cd;
      sincos(g * (double)a.q[i], &sd, &cd);
      ls[i] = hc::cmul_conj(ls[i], (T)cd, -(T)sd);
    }
    __syncthreads();
  }
}

// Per-device set-up: the scratch address and the kernels' shared-memory limit.
struct DeviceState {
  bool ready = false;
  void* scratch = nullptr;
};
static DeviceState g_dev[kMaxDevices];
static std::mutex g_mutex;

static int setup(int dev, void** scratch) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    QVS_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
    const int max_smem = 2 * (1 << hc::TB) * (int)sizeof(double2);
    QVS_CUDA_TRY(cudaFuncSetAttribute(solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    QVS_CUDA_TRY(cudaFuncSetAttribute(solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    d.scratch = p;
    d.ready = true;
  }
  *scratch = d.scratch;
  return QVS_OK;
}

template <class T>
static int launch(int n, int p, const void* q, const double* gammas, const double* ts, double* out,
                  void* scratch, cudaStream_t st) {
  using C = typename hc::Cx<T>::t;
  Args<T> a;   // built on this thread's stack and copied into the launch
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.p = p;
  a.q = static_cast<const T*>(q);
  a.states = static_cast<C*>(scratch);
  a.out = out;
  for (int k = 0; k < p; ++k) {
    a.ang[3 * k] = cos(ts[k]);
    a.ang[3 * k + 1] = sin(ts[k]);
    a.ang[3 * k + 2] = gammas[k];
  }
  const size_t smem = 2 * ((size_t)1 << n) * sizeof(C);
  solve_kernel<T><<<1, 256, smem, st>>>(a);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

}  // namespace na
}  // namespace qvs

extern "C" int qvs_gradient_small_noalloc(int n, int precision, int p, const void* q, const double* gammas,
                                          const double* ts, double* out, void* stream) {
  using namespace qvs;
  if (n < 1 || n > hc::TB || p < 1 || p > na::kMaxLayers || !q || !gammas || !ts || !out) return QVS_EINVAL;
  if (precision != QVS_C64 && precision != QVS_C128) return QVS_EINVAL;
  for (int k = 0; k < p; ++k)
    if (!isfinite(gammas[k]) || !isfinite(ts[k])) return QVS_EINVAL;
  const size_t elem = precision == QVS_C64 ? 8 : 16;
  if ((size_t)p * ((size_t)1 << n) * elem > na::kScratchBytes) return QVS_EINVAL;
  int dev = 0;
  QVS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= na::kMaxDevices) return QVS_EUNSUPPORTED;
  void* scratch = nullptr;
  QVS_TRY(na::setup(dev, &scratch));
  const cudaStream_t st = (cudaStream_t)stream;
  return precision == QVS_C64 ? na::launch<float>(n, p, q, gammas, ts, out, scratch, st)
                              : na::launch<double>(n, p, q, gammas, ts, out, scratch, st);
}
