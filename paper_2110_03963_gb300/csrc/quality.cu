// Quality-vector generators (Sec. 2.2: q_i = C(s_i) on the basis states) and the XY-ring CSR
// builder for the constrained mixer (Sec. 2.4.1).
//
// Sums run in fp64 in the documented order with explicit round-to-nearest operations (no FMA
// contraction), and are rounded once to the output type, so an integer or fp32 quality vector is
// reproducible bit for bit from the same inputs.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "qvs_internal.h"

namespace qvs {

constexpr int kMaxEdges = 1024;

struct MaxcutArgs {
  int n, m, out_dtype, weighted;
  uint8_t eu[kMaxEdges], ev[kMaxEdges];
  double w[kMaxEdges];
};

__global__ void maxcut_kernel(const __grid_constant__ MaxcutArgs a, void* out, int64_t dim) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!a.weighted) {
      int cnt = 0;
      for (int e = 0; e < a.m; ++e)
        cnt += (((i >> (a.n - 1 - a.eu[e])) ^ (i >> (a.n - 1 - a.ev[e]))) & 1) == 0;
      if (a.out_dtype == QVS_I32) static_cast<int32_t*>(out)[i] = cnt;
      else if (a.out_dtype == QVS_F32) static_cast<float*>(out)[i] = (float)cnt;
      else static_cast<double*>(out)[i] = (double)cnt;
    } else {
      double s = 0.0;
      for (int e = 0; e < a.m; ++e)
        if ((((i >> (a.n - 1 - a.eu[e])) ^ (i >> (a.n - 1 - a.ev[e]))) & 1) == 0)
          s = __dadd_rn(s, a.w[e]);
      if (a.out_dtype == QVS_F32) static_cast<float*>(out)[i] = __double2float_rn(s);
      else static_cast<double*>(out)[i] = s;
    }
  }
}

struct SubsetArgs {
  int n, out_dtype;
  double w[64];
};

__global__ void subset_kernel(const __grid_constant__ SubsetArgs a, void* out, int64_t dim) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < a.n; ++b)
      if ((i >> (a.n - 1 - b)) & 1) s = __dadd_rn(s, a.w[b]);
    if (a.out_dtype == QVS_F32) static_cast<float*>(out)[i] = __double2float_rn(s);
    else static_cast<double*>(out)[i] = s;
  }
}

constexpr int kMaxAssets = 32;

struct PortArgs {
  int nq, M, out_dtype;
  double omega, one_minus_omega;
  double r[kMaxAssets];
  double cov[kMaxAssets * kMaxAssets];
};

__global__ void portfolio_kernel(const __grid_constant__ PortArgs a, const int64_t* states,
                                 void* out, int64_t dim) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = states[i];
    double z[kMaxAssets];
    for (int s = 0; s < a.M; ++s) {
      const int lng = (int)((x >> (a.nq - 1 - 2 * s)) & 1);
      const int sht = (int)((x >> (a.nq - 2 - 2 * s)) & 1);
      z[s] = (double)(lng - sht);
    }
    double q = 0.0;
    for (int u = 0; u < a.M; ++u)
      for (int v = 0; v < a.M; ++v) {
        double t = __dmul_rn(a.omega, a.cov[u * a.M + v]);
        t = __dmul_rn(t, z[u]);
        t = __dmul_rn(t, z[v]);
        q = __dadd_rn(q, t);
      }
    for (int u = 0; u < a.M; ++u) {
      double t = __dmul_rn(a.one_minus_omega, a.r[u]);
      t = __dmul_rn(t, z[u]);
      q = __dsub_rn(q, t);
    }
    if (a.out_dtype == QVS_F32) static_cast<float*>(out)[i] = __double2float_rn(q);
    else static_cast<double*>(out)[i] = q;
  }
}

static int grid_for(int64_t dim) {
  int64_t g = (dim + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------- quadratic qualities

int qubo_quantize(int n, double c, const double* hlin, const double* J, QuboCoef* out) {
  if (n < 1 || n > 32 || !hlin || !J || !out) return QVS_EINVAL;
  double S = fabs(c);
  if (!isfinite(c)) return QVS_EINVAL;
  for (int u = 0; u < n; ++u) {
    if (!isfinite(hlin[u])) return QVS_EINVAL;
    S += fabs(hlin[u]);
  }
  for (int u = 0; u < n; ++u)
    for (int v = u + 1; v < n; ++v) {
      if (!isfinite(J[u * n + v])) return QVS_EINVAL;
      S += fabs(J[u * n + v]);
    }
  int F = 40;
  while (F > -30 && ldexp(S, F) + 1024.0 > 1073741824.0) --F;
  // nearest multiple of 2^-F, halves away from zero (llround)
  auto rnd = [F](double x) -> int32_t { return (int32_t)llround(ldexp(x, F)); };
  QuboCoef Q;
  Q.n = n;
  Q.F = F;
  Q.c = rnd(c);
  for (int u = 0; u < n; ++u) Q.h[n - 1 - u] = rnd(hlin[u]);
  for (int u = 0; u < n; ++u)
    for (int v = u + 1; v < n; ++v) {
      const int32_t x = rnd(J[u * n + v]);
      Q.J[n - 1 - u][n - 1 - v] = x;
      Q.J[n - 1 - v][n - 1 - u] = x;
    }
  *out = Q;
  return QVS_OK;
}

__global__ void qubo_kernel(const __grid_constant__ QuboCoef Q, int out_dtype, void* out, int64_t dim) {
  const float sf = ldexpf(1.0f, -Q.F);
  const double sd = ldexp(1.0, -Q.F);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = Q.c;
    for (int b = 0; b < Q.n; ++b) {
      if (!((i >> b) & 1)) continue;
      v += Q.h[b];
      for (int b2 = 0; b2 < b; ++b2)
        if ((i >> b2) & 1) v += Q.J[b][b2];
    }
    if (out_dtype == QVS_F32) static_cast<float*>(out)[i] = (float)v * sf;
    else static_cast<double*>(out)[i] = (double)v * sd;
  }
}

int qubo_generate(const QuboCoef& Q, int out_dtype, void* out, cudaStream_t stream) {
  if (out_dtype != QVS_F32 && out_dtype != QVS_F64) return QVS_EINVAL;
  const int64_t dim = (int64_t)1 << Q.n;
  qubo_kernel<<<grid_for(dim), 256, 0, stream>>>(Q, out_dtype, out, dim);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

}  // namespace qvs

extern "C" int qvs_quality_maxcut(int n, int n_edges, const int32_t* eu, const int32_t* ev,
                                  const double* w, int out_dtype, void* q_out, void* stream) {
  using namespace qvs;
  if (n < 1 || n > 40 || n_edges < 0 || n_edges > kMaxEdges || !q_out) return QVS_EINVAL;
  if (n_edges > 0 && (!eu || !ev)) return QVS_EINVAL;
  if (out_dtype != QVS_I32 && out_dtype != QVS_F32 && out_dtype != QVS_F64) return QVS_EINVAL;
  if (out_dtype == QVS_I32 && w) return QVS_EINVAL;
  MaxcutArgs a;   // built on the host (one per call) and passed by value
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.m = n_edges;
  a.out_dtype = out_dtype;
  a.weighted = w ? 1 : 0;
  for (int e = 0; e < n_edges; ++e) {
    if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n || eu[e] == ev[e]) return QVS_EINVAL;
    a.eu[e] = (uint8_t)eu[e];
    a.ev[e] = (uint8_t)ev[e];
    a.w[e] = w ? w[e] : 1.0;
    if (w && !isfinite(w[e])) return QVS_EINVAL;
  }
  const int64_t dim = (int64_t)1 << n;
  maxcut_kernel<<<grid_for(dim), 256, 0, (cudaStream_t)stream>>>(a, q_out, dim);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

extern "C" int qvs_quality_subset(int n, const double* w, int out_dtype, void* q_out, void* stream) {
  using namespace qvs;
  if (n < 1 || n > 40 || !w || !q_out) return QVS_EINVAL;
  if (out_dtype != QVS_F32 && out_dtype != QVS_F64) return QVS_EINVAL;
  SubsetArgs a{};
  a.n = n;
  a.out_dtype = out_dtype;
  for (int b = 0; b < n; ++b) {
    if (!isfinite(w[b])) return QVS_EINVAL;
    a.w[b] = w[b];
  }
  const int64_t dim = (int64_t)1 << n;
  subset_kernel<<<grid_for(dim), 256, 0, (cudaStream_t)stream>>>(a, q_out, dim);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

extern "C" int qvs_quality_portfolio(int n_qubits, int64_t dim, const int64_t* states,
                                     const double* returns, const double* cov, double omega,
                                     int out_dtype, void* q_out, void* stream) {
  using namespace qvs;
  if (n_qubits < 2 || (n_qubits & 1) || n_qubits / 2 > kMaxAssets || n_qubits > 62) return QVS_EINVAL;
  if (dim < 1 || !states || !returns || !cov || !q_out || !isfinite(omega)) return QVS_EINVAL;
  if (out_dtype != QVS_F32 && out_dtype != QVS_F64) return QVS_EINVAL;
  PortArgs a;   // built on the host (one per call) and passed by value
  memset(&a, 0, sizeof(a));
  a.nq = n_qubits;
  a.M = n_qubits / 2;
  a.out_dtype = out_dtype;
  a.omega = omega;
  a.one_minus_omega = 1.0 - omega;
  for (int u = 0; u < a.M; ++u) {
    a.r[u] = returns[u];
    for (int v = 0; v < a.M; ++v) a.cov[u * a.M + v] = cov[u * a.M + v];
  }
  portfolio_kernel<<<grid_for(dim), 256, 0, (cudaStream_t)stream>>>(a, states, q_out, dim);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

// ------------------------------------------------------------------ XY-ring CSR (host)

static int qvs_xy_ring_csr_impl(int n, int k, int64_t* states, int64_t* rowptr, int32_t* colind,
                                int64_t* dim_out, int64_t* nnz_out) {
  if (n < 3 || n > 40 || k < 0 || k > n) return QVS_EINVAL;
  // binomial table for the combinatorial number system rank of a weight-k state
  std::vector<std::vector<int64_t>> C(n + 1, std::vector<int64_t>(n + 2, 0));
  for (int a = 0; a <= n; ++a) {
    C[a][0] = 1;
    for (int b = 1; b <= a; ++b) C[a][b] = C[a - 1][b - 1] + (b <= a - 1 ? C[a - 1][b] : 0);
  }
  const int64_t dim = C[n][k];
  if (dim > INT32_MAX) return QVS_EUNSUPPORTED;
  // nonzeros: every ring edge (a, a+1 mod n) whose two bits differ
  auto count_row = [&](uint64_t x) {
    int c = 0;
    for (int a = 0; a < n; ++a) {
      const int b = (a + 1) % n;
      c += (int)(((x >> a) ^ (x >> b)) & 1);
    }
    return c;
  };
  // enumerate weight-k states in increasing order (Gosper's hack)
  std::vector<uint64_t> st((size_t)dim);
  {
    uint64_t x = k == 0 ? 0 : ((1ull << k) - 1);
    for (int64_t r = 0; r < dim; ++r) {
      st[(size_t)r] = x;
      if (k == 0) break;
      const uint64_t c = x & (~x + 1);
      const uint64_t rr = x + c;
      x = (((rr ^ x) >> 2) / c) | rr;
    }
  }
  int64_t nnz = 0;
  for (int64_t r = 0; r < dim; ++r) nnz += count_row(st[(size_t)r]);
  if (dim_out) *dim_out = dim;
  if (nnz_out) *nnz_out = nnz;
  if (!states && !rowptr && !colind) return QVS_OK;
  if (!states || !rowptr || !colind) return QVS_EINVAL;
  auto rank = [&](uint64_t x) {
    // rank among weight-k states in increasing order: sum over the set bits (ascending,
    // j-th set bit at position c_j) of C(c_j, j+1)
    int64_t rk = 0;
    int j = 0;
    for (int b = 0; b < n; ++b)
      if ((x >> b) & 1) rk += C[b][++j];
    return rk;
  };
  rowptr[0] = 0;
  int64_t pos = 0;
  std::vector<int32_t> cols;
  cols.reserve(2 * n);
  for (int64_t r = 0; r < dim; ++r) {
    const uint64_t x = st[(size_t)r];
    states[r] = (int64_t)x;
    cols.clear();
    for (int a = 0; a < n; ++a) {
      const int b = (a + 1) % n;
      if (((x >> a) ^ (x >> b)) & 1) cols.push_back((int32_t)rank(x ^ ((1ull << a) | (1ull << b))));
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t c : cols) colind[pos++] = c;
    rowptr[r + 1] = pos;
  }
  return QVS_OK;
}

extern "C" int qvs_xy_ring_csr(int n, int k, int64_t* states, int64_t* rowptr, int32_t* colind,
                               int64_t* dim_out, int64_t* nnz_out) {
  return qvs::guarded([&] { return qvs_xy_ring_csr_impl(n, k, states, rowptr, colind, dim_out, nnz_out); });
}

extern "C" int qvs_quality_qubo(int n_qubits, double c, const double* hlin, const double* J, int out_dtype,
                                void* q_out, void* stream) {
  if (!q_out) return QVS_EINVAL;
  static qvs::QuboCoef Q;   // 4 KiB: kept off the stack
  QVS_TRY(qvs::qubo_quantize(n_qubits, c, hlin, J, &Q));
  return qvs::qubo_generate(Q, out_dtype, q_out, (cudaStream_t)stream);
}

extern "C" int qvs_qubo_fixed_point(int n_qubits, double c, const double* hlin, const double* J, int* F,
                                    int32_t* ci, int32_t* hi, int32_t* Ji) {
  if (!F || !ci || !hi || !Ji) return QVS_EINVAL;
  qvs::QuboCoef Q;
  QVS_TRY(qvs::qubo_quantize(n_qubits, c, hlin, J, &Q));
  const int n = n_qubits;
  *F = Q.F;
  *ci = Q.c;
  for (int u = 0; u < n; ++u) hi[u] = Q.h[n - 1 - u];
  for (int u = 0; u < n; ++u)
    for (int v = 0; v < n; ++v) Ji[u * n + v] = v > u ? Q.J[n - 1 - u][n - 1 - v] : 0;
  return QVS_OK;
}

extern "C" int qvs_qubo_from_maxcut(int n, int n_edges, const int32_t* eu, const int32_t* ev, const double* w,
                                    double* c, double* hlin, double* J) {
  if (n < 1 || n > 32 || n_edges < 0 || !c || !hlin || !J) return QVS_EINVAL;
  if (n_edges > 0 && (!eu || !ev)) return QVS_EINVAL;
  *c = 0.0;
  for (int u = 0; u < n; ++u) hlin[u] = 0.0;
  for (int u = 0; u < n * n; ++u) J[u] = 0.0;
  for (int e = 0; e < n_edges; ++e) {
    if (eu[e] < 0 || eu[e] >= n || ev[e] < 0 || ev[e] >= n || eu[e] == ev[e]) return QVS_EINVAL;
    const double we = w ? w[e] : 1.0;
    const int u = std::min(eu[e], ev[e]), v = std::max(eu[e], ev[e]);
    *c += we;
    hlin[u] -= we;
    hlin[v] -= we;
    J[u * n + v] += 2.0 * we;
  }
  return QVS_OK;
}
