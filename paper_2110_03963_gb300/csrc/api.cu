// C ABI of libqvs: handle life cycle, argument checks and dispatch to the mixer paths.
// The call sequence mirrors the paper's Ansatz workflow (Sec. 5, Table of Ansatz methods):
// set the quality vector (observables), the unitaries (mixer), optionally the initial state,
// then evolve / evaluate the objective / its gradient.
#include <math.h>
#include <string.h>

#include <new>

#include <vector>

#include "qvs_internal.h"

namespace qvs {

static thread_local const Allocator* t_allocator = nullptr;

const Allocator* current_allocator() { return t_allocator; }

AllocScope::AllocScope(const Allocator* a) : prev(t_allocator) { t_allocator = a; }
AllocScope::~AllocScope() { t_allocator = prev; }

int ensure_host_res(qvs_ctx* h, int p) {
  if (h->host_res && h->host_res_cap >= p) return QVS_OK;
  if (h->host_res) cudaFreeHost(h->host_res);
  h->host_res = nullptr;
  h->host_res_cap = 0;
  const int cap = p < 64 ? 64 : p;
  // 1 + 2 cap result slots and one more for the device error flag
  QVS_CUDA_TRY(cudaMallocHost((void**)&h->host_res, sizeof(double) * (2 + 2 * (size_t)cap)));
  h->host_res_cap = cap;
  return QVS_OK;
}

static cudaEvent_t pool_get(qvs_ctx* h) {
  if (!h->evpool.empty()) {
    cudaEvent_t e = h->evpool.back();
    h->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

int prof_begin(qvs_ctx* h, cudaEvent_t* start) {
  *start = nullptr;
  if (!h->profile) return QVS_OK;
  *start = pool_get(h);
  if (!*start) return QVS_ECUDA;
  QVS_CUDA_TRY(cudaEventRecord(*start, h->stream));
  return QVS_OK;
}

int prof_end(qvs_ctx* h, const char* name, double bytes, cudaEvent_t start) {
  if (!h->profile || !start) return QVS_OK;
  cudaEvent_t end = pool_get(h);
  if (!end) return QVS_ECUDA;
  QVS_CUDA_TRY(cudaEventRecord(end, h->stream));
  int id = -1;
  for (size_t i = 0; i < h->kstats.size(); ++i)
    if (h->kstats[i].name == name) id = (int)i;
  if (id < 0) {
    h->kstats.push_back(qvs_ctx::KStat{});
    h->kstats.back().name = name;
    id = (int)h->kstats.size() - 1;
  }
  h->pending.push_back(qvs_ctx::Pending{id, bytes, start, end});
  return QVS_OK;
}

int prof_flush(qvs_ctx* h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    QVS_CUDA_TRY(cudaEventSynchronize(p.b));
    QVS_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
    auto& k = h->kstats[p.id];
    k.launches += 1;
    k.ms += ms;
    k.bytes += p.bytes;
    h->evpool.push_back(p.a);
    h->evpool.push_back(p.b);
  }
  h->pending.clear();
  return QVS_OK;
}

void prof_release(qvs_ctx* h) {
  for (auto& p : h->pending) {
    h->evpool.push_back(p.a);
    h->evpool.push_back(p.b);
  }
  h->pending.clear();
  for (auto e : h->evpool) cudaEventDestroy(e);
  h->evpool.clear();
}

static int log2_exact(int64_t d) {
  if (d < 1 || (d & (d - 1))) return -1;
  int n = 0;
  while ((int64_t(1) << n) < d) ++n;
  return n;
}

static bool params_ok(int p, const double* g, const double* t) {
  if (p < 1 || p > 4096 || !g || !t) return false;
  for (int k = 0; k < p; ++k)
    if (!isfinite(g[k]) || !isfinite(t[k])) return false;
  return true;
}

}  // namespace qvs

using namespace qvs;

extern "C" int qvs_create(qvs_t* out, int64_t dim, int precision, void* stream,
                          void* (*alloc)(size_t, void*), void (*dealloc)(void*, void*), void* alloc_ctx) {
  if (!out) return QVS_EINVAL;
  *out = nullptr;
  if (dim < 2 || dim > (int64_t(1) << 34)) return QVS_EINVAL;
  if (precision != QVS_C64 && precision != QVS_C128) return QVS_EINVAL;
  if ((alloc == nullptr) != (dealloc == nullptr)) return QVS_EINVAL;
  qvs_ctx* h = new (std::nothrow) qvs_ctx();
  if (!h) return QVS_ENOMEM;
  h->dim = dim;
  h->n = log2_exact(dim);
  h->precision = precision;
  h->stream = (cudaStream_t)stream;
  h->allocator.alloc = alloc;
  h->allocator.dealloc = dealloc;
  h->allocator.ctx = alloc_ctx;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return QVS_ECUDA;
  }

  *out = h;
  return QVS_OK;
}

extern "C" int qvs_destroy(qvs_t h) {
  if (!h) return QVS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  qvs::DevBuf* bufs[] = {&h->q, &h->psi0, &h->psi, &h->lam, &h->ckpt, &h->part, &h->res, &h->rowmap,
                         &h->work, &h->circ.lam, &h->circ.qT, &h->csr.rowptr,
                         &h->csr.colind, &h->csr.values, &h->csr.states, &h->csr.binom, &h->qubo.dcoef, &h->qubo.tab, &h->ex.coef,
                         &h->ex.tab, &h->ex.g, &h->ex.mterms, &h->ex.mpart, &h->ex.mrowmap, &h->ex.mres,
                         &h->flags};
  for (qvs::DevBuf* b : bufs) b->release();
  if (h->host_res) cudaFreeHost(h->host_res);
  prof_release(h);
  delete h;
  (void)cudaGetLastError();
  return QVS_OK;
}

template <class Dst, class Src>
__global__ void convert_kernel(Dst* __restrict__ d, const Src* __restrict__ s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (Dst)s[i];
}

template <class Dst, class Src>
static int convert_on_device(qvs_ctx* h, Dst* d, const Src* s, int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  convert_kernel<Dst, Src><<<(int)g, 256, 0, h->stream>>>(d, s, n);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

extern "C" int qvs_set_quality(qvs_t h, const void* q, int dtype, int on_device) {
  if (!h || !q) return QVS_EINVAL;
  AllocScope scope(&h->allocator);
  if (dtype != QVS_I32 && dtype != QVS_F32 && dtype != QVS_F64) return QVS_EINVAL;
  const int64_t n = h->dim;
  const size_t in_elem = dtype == QVS_F64 ? 8 : 4;
  const bool want_f32 = h->precision == QVS_C64;
  const size_t out_elem = want_f32 ? 4 : 8;
  QVS_TRY(h->q.ensure(out_elem * (size_t)n));
  h->have_q = false;
  const bool same = (want_f32 && dtype == QVS_F32) || (!want_f32 && dtype == QVS_F64);
  if (same) {
    QVS_CUDA_TRY(cudaMemcpyAsync(h->q.ptr, q, out_elem * n,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 h->stream));
  } else {
    // stage the raw input on the device, then convert there
    const void* src = q;
    if (!on_device) {
      QVS_TRY(h->work.ensure(in_elem * (size_t)n));
      QVS_CUDA_TRY(cudaMemcpyAsync(h->work.ptr, q, in_elem * n, cudaMemcpyHostToDevice, h->stream));
      src = h->work.ptr;
    }
    if (want_f32) {
      if (dtype == QVS_I32) QVS_TRY(convert_on_device(h, h->q.as<float>(), (const int32_t*)src, n));
      else QVS_TRY(convert_on_device(h, h->q.as<float>(), (const double*)src, n));
    } else {
      if (dtype == QVS_I32) QVS_TRY(convert_on_device(h, h->q.as<double>(), (const int32_t*)src, n));
      else QVS_TRY(convert_on_device(h, h->q.as<double>(), (const float*)src, n));
    }
  }
  h->have_q = true;
  h->have_E = false;
  h->circ.qT_valid = false;
  h->qubo.on = false;
  h->qubo.tab_valid = false;
  return QVS_OK;
}

extern "C" int qvs_set_quality_qubo(qvs_t h, int n_qubits, double c, const double* hlin, const double* J) {
  if (!h || !hlin || !J) return QVS_EINVAL;
  AllocScope scope(&h->allocator);
  if (h->n < 1 || n_qubits != h->n) return QVS_EINVAL;
  QVS_TRY(qubo_quantize(n_qubits, c, hlin, J, &h->qubo.coef));
  h->qubo.on = true;
  h->qubo.materialized = false;
  h->qubo.tab_valid = false;
  h->have_q = true;
  h->have_E = false;
  h->circ.qT_valid = false;
  return QVS_OK;
}

namespace qvs {
int ensure_q_vector(qvs_ctx* h) {
  if (!h->qubo.on || h->qubo.materialized) return QVS_OK;
  const bool f32 = h->precision == QVS_C64;
  QVS_TRY(h->q.ensure((f32 ? 4 : 8) * (size_t)h->dim));
  QVS_TRY(qubo_generate(h->qubo.coef, f32 ? QVS_F32 : QVS_F64, h->q.ptr, h->stream));
  h->qubo.materialized = true;
  return QVS_OK;
}
}  // namespace qvs

static int qvs_set_mixer_impl(qvs_t h, int kind, const qvs_mixer_desc* d) {
  if (!h || !d) return QVS_EINVAL;
  AllocScope scope(&h->allocator);
  h->have_mixer = false;
  h->have_E = false;
  if (kind == QVS_MIX_HYPERCUBE) {
    if (d->n_qubits < 1 || h->n != d->n_qubits) return QVS_EINVAL;
    if (h->n > 32) return QVS_EUNSUPPORTED;
  } else if (kind == QVS_MIX_CIRCULANT) {
    if (h->n < 1) return QVS_EINVAL;
    QVS_TRY(circ_set_mixer(h, d));
  } else if (kind == QVS_MIX_CSR) {
    QVS_TRY(csr_set_mixer(h, d));
  } else if (kind == QVS_MIX_XY_RING) {
    QVS_TRY(xy_set_mixer(h, d));
  } else if (kind == QVS_MIX_PARITY) {
    QVS_TRY(parity_set_mixer(h, d));
  } else {
    return QVS_EINVAL;
  }
  h->mixer = kind;
  h->have_mixer = true;
  return QVS_OK;
}

extern "C" int qvs_set_mixer(qvs_t h, int kind, const qvs_mixer_desc* d) {
  return qvs::guarded([&] { return qvs_set_mixer_impl(h, kind, d); });
}

extern "C" int qvs_set_initial_state(qvs_t h, int kind, const void* psi0, int on_device) {
  if (!h) return QVS_EINVAL;
  if (kind == QVS_INIT_UNIFORM) {
    if (psi0) return QVS_EINVAL;
    h->have_E = false;
    h->have_psi0 = false;
    return QVS_OK;
  }
  if (kind != QVS_INIT_EXPLICIT || !psi0) return QVS_EINVAL;
  AllocScope scope(&h->allocator);
  h->have_E = false;
  const size_t bytes = elem_bytes(h) * (size_t)h->dim;
  QVS_TRY(h->psi0.ensure(bytes));
  QVS_CUDA_TRY(cudaMemcpyAsync(h->psi0.ptr, psi0, bytes,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               h->stream));
  h->have_psi0 = true;
  return QVS_OK;
}

extern "C" int qvs_set_option(qvs_t h, int option, int64_t value) {
  if (!h) return QVS_EINVAL;
  if (option == QVS_OPT_CKPT_LAYERS) {
    if (value < 0 || value > 4096) return QVS_EINVAL;
    h->ckpt_layers = (int)value;
    return QVS_OK;
  }
  if (option == QVS_OPT_STAGED) {
    if (value != 0 && value != 1) return QVS_EINVAL;
    h->staged = value == 1;
    return QVS_OK;
  }
  if (option == QVS_OPT_PROFILE) {
    if (value != 0 && value != 1) return QVS_EINVAL;
    h->profile = value == 1;
    h->kstats.clear();
    return QVS_OK;
  }
  return QVS_EINVAL;
}

static int ready(qvs_t h) {
  if (!h) return QVS_EINVAL;
  if (!h->have_q || !h->have_mixer) return QVS_ESTATE;
  return QVS_OK;
}

extern "C" int qvs_evolve(qvs_t h, int p, const double* gammas, const double* ts) {
  QVS_TRY(ready(h));
  AllocScope scope(&h->allocator);
  if (!params_ok(p, gammas, ts)) return QVS_EINVAL;
  h->have_E = false;
  if (h->mixer != QVS_MIX_HYPERCUBE) QVS_TRY(ensure_q_vector(h));
  switch (h->mixer) {
    case QVS_MIX_HYPERCUBE: return hc_evolve(h, p, gammas, ts);
    case QVS_MIX_CIRCULANT: return circ_evolve(h, p, gammas, ts);
    case QVS_MIX_CSR:
    case QVS_MIX_XY_RING: return csr_evolve(h, p, gammas, ts);
    case QVS_MIX_PARITY: return parity_evolve(h, p, gammas, ts);
  }
  return QVS_ESTATE;
}

extern "C" int qvs_set_phase_terms(qvs_t h, int n_terms, const int32_t* u, const int32_t* v, const double* coef) {
  if (!h || h->n < 1 || n_terms < 0 || n_terms > 1024) return QVS_EINVAL;
  if (n_terms > 0 && (!u || !v || !coef)) return QVS_EINVAL;
  std::vector<ExTerm> t;
  for (int j = 0; j < n_terms; ++j) {
    if (u[j] < 0 || u[j] >= h->n || v[j] < -1 || v[j] >= h->n || v[j] == u[j] || !isfinite(coef[j]))
      return QVS_EINVAL;
    t.push_back({h->n - 1 - u[j], v[j] < 0 ? -1 : h->n - 1 - v[j], coef[j]});
  }
  h->ex.terms = t;
  h->have_E = false;
  return QVS_OK;
}

static bool ex_params_ok(qvs_t h, int p, const double* g, const double* t) {
  const size_t J = h->ex.terms.size();
  if (p < 1 || p > 4096 || !g || !t) return false;
  for (size_t i = 0; i < (size_t)p * J; ++i)
    if (!isfinite(g[i])) return false;
  for (int k = 0; k < p; ++k)
    if (!isfinite(t[k])) return false;
  return true;
}

extern "C" int qvs_evolve_ex(qvs_t h, int p, const double* gammas, const double* ts) {
  QVS_TRY(ready(h));
  AllocScope scope(&h->allocator);
  if (h->mixer != QVS_MIX_HYPERCUBE) return QVS_EUNSUPPORTED;
  if (h->ex.terms.empty()) return QVS_ESTATE;
  if (!ex_params_ok(h, p, gammas, ts)) return QVS_EINVAL;
  h->have_E = false;
  return hc_evolve_ex(h, p, gammas, ts);
}

extern "C" int qvs_gradient_ex(qvs_t h, int p, const double* gammas, const double* ts, double* E, double* dgamma,
                               double* dt) {
  QVS_TRY(ready(h));
  AllocScope scope(&h->allocator);
  if (h->mixer != QVS_MIX_HYPERCUBE) return QVS_EUNSUPPORTED;
  if (h->ex.terms.empty()) return QVS_ESTATE;
  if (!ex_params_ok(h, p, gammas, ts) || !E || !dgamma || !dt) return QVS_EINVAL;
  h->have_E = false;
  return hc_gradient_ex(h, p, gammas, ts, E, dgamma, dt);
}

extern "C" int qvs_expectation(qvs_t h, double* E) {
  if (!h || !E) return QVS_EINVAL;
  if (!h->have_E) return QVS_ESTATE;
  *E = h->E;
  return QVS_OK;
}

extern "C" int qvs_gradient(qvs_t h, int p, const double* gammas, const double* ts, double* E,
                            double* dgamma, double* dt) {
  QVS_TRY(ready(h));
  AllocScope scope(&h->allocator);
  if (!params_ok(p, gammas, ts) || !E || !dgamma || !dt) return QVS_EINVAL;
  h->have_E = false;
  if (h->mixer != QVS_MIX_HYPERCUBE) QVS_TRY(ensure_q_vector(h));
  switch (h->mixer) {
    case QVS_MIX_HYPERCUBE: return hc_gradient(h, p, gammas, ts, E, dgamma, dt);
    case QVS_MIX_CIRCULANT: return circ_gradient(h, p, gammas, ts, E, dgamma, dt);
    case QVS_MIX_CSR:
    case QVS_MIX_XY_RING: return csr_gradient(h, p, gammas, ts, E, dgamma, dt);
    case QVS_MIX_PARITY: return parity_gradient(h, p, gammas, ts, E, dgamma, dt);
  }
  return QVS_ESTATE;
}

extern "C" int qvs_get_state(qvs_t h, void* dst, int on_device) {
  if (!h || !dst) return QVS_EINVAL;
  if (!h->have_E || !h->psi.ptr) return QVS_ESTATE;
  const size_t bytes = elem_bytes(h) * (size_t)h->dim;
  QVS_CUDA_TRY(cudaMemcpyAsync(dst, h->psi.ptr, bytes,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               h->stream));
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return QVS_OK;
}

extern "C" int qvs_last_launch_count(qvs_t h, int64_t* count) {
  if (!h || !count) return QVS_EINVAL;
  *count = h->launches;
  return QVS_OK;
}

extern "C" int qvs_kernel_stats(qvs_t h, int slot, char* name, int name_len, int64_t* launches,
                                double* ms, double* bytes) {
  if (!h || slot < 0 || slot >= (int)h->kstats.size()) return QVS_EINVAL;
  const auto& k = h->kstats[slot];
  if (name && name_len > 0) {
    strncpy(name, k.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = k.launches;
  if (ms) *ms = k.ms;
  if (bytes) *bytes = k.bytes;
  return QVS_OK;
}

extern "C" const char* qvs_strerror(int s) {
  switch (s) {
    case QVS_OK: return "ok";
    case QVS_EINVAL: return "invalid argument";
    case QVS_ENOMEM: return "device allocation failed";
    case QVS_ECUDA: return "CUDA error";
    case QVS_ESTATE: return "call out of order (quality, mixer or evolve missing)";
    case QVS_ENUMERIC: return "numerical check failed";
    case QVS_ETIMEOUT: return "device wait timed out";
    case QVS_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}
