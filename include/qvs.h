/*
 * qvs.h - C ABI of libqvs, a single-GPU (sm_103a) state-vector engine for quantum variational
 * algorithms (QAOA, QWOA, QAOAz) following Matwiejew & Wang, "QuOp_MPI: a framework for parallel
 * simulation of quantum variational algorithms" (arXiv 2110.03963).
 *
 * What the library computes (paper Sec. 2.1): for a quality vector q (the diagonal of Q), a mixing
 * operator W and parameters gamma_k, t_k (k = 1..p), the state
 *     |theta> = prod_{k=1..p} exp(-i t_k W) exp(-i gamma_k Q) |psi0>
 * (phase first, then mixer, within each layer - the interleaved order of Sec. 6.1.1), the
 * objective f = <theta|Q|theta> and its gradient with respect to every gamma_k and t_k.
 *
 * Conventions shared by every entry point:
 *   - All functions return an int status (QVS_OK = 0 or a negative QVS_E* code); none aborts,
 *     traps or prints. qvs_strerror() names a code. A CUDA failure is QVS_ECUDA and leaves the
 *     handle usable unless the CUDA context itself is lost.
 *   - A qvs_t handle owns every device buffer it allocates (state, adjoint vector, checkpoints,
 *     copies of q and of the mixer, reduction scratch), through the allocator hooks given to
 *     qvs_create (default cudaMalloc); qvs_destroy frees them. Inputs are always
 *     copied: the caller may free or reuse its buffers as soon as a call returns.
 *   - "on_device" arguments: 0 = the pointer is host memory, 1 = device memory of the handle's
 *     device. Host inputs may be pageable or pinned.
 *   - Every kernel is launched on the handle's stream (the one given to qvs_create, or the legacy
 *     default stream when NULL). Scalar outputs (E, gradients) are complete when the call returns;
 *     the call synchronises the stream for them.
 *   - Basis index i holds qubit u in bit (n-1-u) (most significant first).
 *   - Parameters arrive as two host arrays gammas[p], ts[p] (layer k uses gammas[k], ts[k]).
 *   - Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef QVS_H
#define QVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qvs_ctx* qvs_t;

/* status codes */
enum {
  QVS_OK = 0,
  QVS_EINVAL = -1,       /* bad argument: NULL pointer, size, dtype, non-finite parameter   */
  QVS_ENOMEM = -2,       /* device allocation failed                                         */
  QVS_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed                      */
  QVS_ESTATE = -4,       /* call out of order (e.g. evolve before quality and mixer are set) */
  QVS_ENUMERIC = -5,     /* numerical check failed (e.g. Chebyshev series did not converge)  */
  QVS_ETIMEOUT = -6,     /* a bounded device-side wait gave up                               */
  QVS_EUNSUPPORTED = -7  /* valid request outside what this build implements                  */
};

/* state precision */
enum { QVS_C64 = 1, QVS_C128 = 2 };
/* element type of quality vectors */
enum { QVS_I32 = 1, QVS_F32 = 2, QVS_F64 = 3 };
/* initial-state kinds of qvs_set_initial_state */
enum { QVS_INIT_UNIFORM = 0, QVS_INIT_EXPLICIT = 1 };
/* mixer kinds (paper Sec. 3: sparse, circulant, and the QAOA hypercube) */
enum { QVS_MIX_HYPERCUBE = 1, QVS_MIX_CIRCULANT = 2, QVS_MIX_CSR = 3, QVS_MIX_PARITY = 4, QVS_MIX_XY_RING = 5 };
/* options for qvs_set_option */
enum {
  QVS_OPT_CKPT_LAYERS = 1,  /* hypercube adjoint: store the forward state every this many
                               layers and uncompute in between; 0 = ceil(sqrt(p)) (default).
                               1 stores every layer boundary: up to 20 qubits a layer is one
                               pass, so nothing is uncomputed; from 21 qubits a layer is two
                               passes and the rotation-only pass of each layer is still
                               uncomputed.                                                    */
  QVS_OPT_PROFILE = 2,      /* 1: bracket every kernel launch with CUDA events on the handle's
                               stream and accumulate per-kernel statistics (qvs_kernel_stats);
                               0: off (default). Setting it resets the statistics.           */
  QVS_OPT_STAGED = 3        /* complex64 data movement through the Tensor Memory Accelerator;
                               1 (default), 0 = per-thread loads and stores, one CTA per tile.
                               Hypercube mixer, complex64, n > 12: the last forward pass of
                               qvs_gradient (fused with the adjoint seed) runs as a persistent
                               kernel whose next tile is copied into shared memory while the
                               current one is processed, when that pass's tile keeps at least 4
                               contiguous low index bits (every n <= 28). Circulant mixer,
                               N = 2^26: each column tile is loaded and stored by one tensor
                               copy, and every column and row pass prefetches the next wave's
                               state tile into L2. Results are identical either way. A pass
                               whose copy wait expires makes the call return QVS_ETIMEOUT.    */
};

/*
 * Mixer description (qvs_set_mixer). Only the fields of the chosen kind are read.
 *
 * QVS_MIX_HYPERCUBE (Sec. 2.3.1): W = sum_j X_j on n_qubits qubits; dim must equal 2^n_qubits.
 * QVS_MIX_CIRCULANT (Sec. 2.4.2, Sec. 3): W symmetric circulant of size dim = 2^n, 17 <= n <= 27,
 *     complex64 (other sizes: QVS_EUNSUPPORTED), given by n_offsets connection offsets s
 *     (0 < s < dim) with weights w_s (NULL = all 1): W[j][(j+s) mod dim] = W[j][(j-s) mod dim] = w_s
 *     (the offset dim/2 couples each j once).
 * QVS_MIX_CSR (Sec. 2.4.1, Sec. 3): W real symmetric sparse (rowptr int64[dim+1], colind
 *     int32[nnz]), values float[nnz] or NULL for a constant implicit_value; host or device arrays
 *     per csr_on_device. spec_lo/spec_hi bound the spectrum (both 0: the library estimates the
 *     interval once, here: 64 fp64 Lanczos steps, extreme Ritz values widened by their residuals
 *     and by 1 % of the width, capped by the Gershgorin bound); cheb_tol is the Chebyshev
 *     truncation tolerance (0: 1e-7).
 * QVS_MIX_PARITY (Sec. 2.4.1, QAOAz): U(t) = exp(-i t B_last) exp(-i t B_even) exp(-i t B_odd) on
 *     two rings of qubits, the even qubits (0, 2, ...) and the odd qubits (1, 3, ...), over the
 *     full register (dim = 2^n_qubits, 12 <= n_qubits <= 30, complex64). On a ring of N qubits
 *     (1-indexed positions k) B_odd couples (k, k+1) for odd k, B_even (k, k+1) for even k plus
 *     the closing pair (N, 1) when N is even, B_last the closing pair when N is odd; each coupling
 *     is X X + Y Y; one t per layer. Reads n_qubits only.
 * QVS_MIX_XY_RING (Sec. 2.4.1): the XY ring sum_a (X_a X_{a+1} + Y_a Y_{a+1}) (a+1 mod n) on the
 *     basis states of n_qubits qubits with hamming_weight ones (2 <= n <= 31, 1 <= k < n), in
 *     increasing integer order: the operator qvs_xy_ring_csr writes as CSR, applied without it (each
 *     row's neighbours are ranked from its state bits on the device). dim must equal C(n, k);
 *     complex64. spec_lo/spec_hi and cheb_tol as for QVS_MIX_CSR; the Gershgorin bound used to cap
 *     the estimated interval is 2 min(n, 2 min(k, n - k)).
 */
typedef struct {
  int n_qubits;
  int n_offsets;
  const int64_t* offsets;
  const double* offset_weights;
  const int64_t* rowptr;
  const int32_t* colind;
  const float* values;
  float implicit_value;
  int64_t nnz;
  int csr_on_device;
  double spec_lo, spec_hi;
  double cheb_tol;
  int hamming_weight;   /* QVS_MIX_XY_RING */
} qvs_mixer_desc;

/* Sec. 5 (the plan/destroy life cycle of the Unitary table): create a handle for states of
 * dimension dim (2 <= dim <= 2^34) at the given precision on the current CUDA device.
 *   stream     a cudaStream_t or NULL (legacy default stream); every kernel and copy of the
 *              handle is ordered on it.
 *   alloc, dealloc, alloc_ctx
 *              device-memory hooks, both NULL (cudaMalloc / cudaFree) or both set. Every device
 *              buffer the handle owns is then obtained as alloc(bytes, alloc_ctx) and returned as
 *              dealloc(ptr, alloc_ctx). alloc returns NULL when it cannot serve the request (the
 *              call that needed the memory returns QVS_ENOMEM) and must return blocks aligned to
 *              256 bytes (a misaligned block is handed back to dealloc and the call returns
 *              QVS_EINVAL). dealloc may be called while earlier work on the handle's stream still
 *              reads the block: the hooks must not reuse it before that work completes in stream
 *              order (a stream-ordered pool allocating on the handle's stream, such as the PyTorch
 *              caching allocator, satisfies this). The hooks are called on the thread of the
 *              qvs_* call that needs the memory, never from a device callback.
 * On success *out is set. QVS_EINVAL for NULL out, dim or precision out of range, or only one of
 * alloc/dealloc given; QVS_ECUDA when no CUDA device is usable. */
int qvs_create(qvs_t* out, int64_t dim, int precision, void* stream, void* (*alloc)(size_t, void*),
               void (*dealloc)(void*, void*), void* alloc_ctx);

/* Sec. 5 (destroy): wait for the handle's stream, then return every device buffer of the handle to
 * the allocator that made it (NULL is accepted). */
int qvs_destroy(qvs_t h);

/* Sec. 2.1: set the quality vector q (dim entries). I32 and F32 values are used as given
 * (the complex64 path computes phases from the fp32 value); F64 is kept in fp64 by the
 * complex128 path and rounded once to fp32 by the complex64 path. */
int qvs_set_quality(qvs_t h, const void* q, int dtype, int on_device);

/* Sec. 2.2 / Sec. 6: set a quality given as a quadratic form of the qubit values x_u in {0, 1}
 * (qubit u = index bit n-1-u):
 *     q(x) = c + sum_u hlin[u] x_u + sum_{u<v} J[u*n + v] x_u x_v
 * (J: n*n row-major host array, read above the diagonal only; hlin: n host values). The
 * max-cut, subset-sum and portfolio costs of Sec. 6 are all of this form.
 * Fixed point: S = |c| + sum_u |hlin[u]| + sum_{u<v} |J[u*n+v]| (fp64, in that order); F is the
 * largest integer in [-30, 40] with S 2^F + 1024 <= 2^30; every coefficient is rounded to the
 * nearest integer multiple of 2^-F (halves away from zero). q(x) is then summed exactly in 32-bit
 * integers and rounded once to the handle's quality type (fp32 for complex64, fp64 for
 * complex128): the same values qvs_quality_qubo writes.
 * The hypercube path for n > 12 evaluates q inside its phase passes from per-tile tables (no
 * q vector is stored or read); the other paths materialise the vector once on the device.
 * Needs dim = 2^n_qubits. QVS_EINVAL for a NULL argument, n_qubits not matching the handle, or a
 * non-finite coefficient. */
int qvs_set_quality_qubo(qvs_t h, int n_qubits, double c, const double* hlin, const double* J);

/* Sec. 3: set the mixing operator (copied). */
int qvs_set_mixer(qvs_t h, int kind, const qvs_mixer_desc* desc);

/* Sec. 2.1 / Sec. 5 (the Ansatz table's initial state): choose |psi0>.
 *   kind = QVS_INIT_UNIFORM   the equal superposition 1/sqrt(dim) over the simulated space (the
 *                             default; never stored: the first pass generates it); psi0 must be NULL.
 *   kind = QVS_INIT_EXPLICIT  psi0 holds dim complex values (interleaved re/im, in the handle's
 *                             precision), host or device memory per on_device; copied into the
 *                             handle (the caller may free it on return).
 * QVS_EINVAL for another kind, a NULL psi0 with QVS_INIT_EXPLICIT or a non-NULL one with
 * QVS_INIT_UNIFORM. */
int qvs_set_initial_state(qvs_t h, int kind, const void* psi0, int on_device);

/* Set an option (QVS_OPT_*). */
int qvs_set_option(qvs_t h, int option, int64_t value);

/* Sec. 6.2 (QAOAz initial state): write |01>^{(x)A} ((|00> + |11>)/sqrt 2)^{(x)(n/2 - A)} into the
 * complex64 device buffer dst (2^n_qubits amplitudes, normal form): asset a occupies qubits
 * (2a, 2a+1) (qubit u = index bit n-1-u), the first A assets are |01>. Stream-ordered on stream
 * (NULL: default stream). QVS_EINVAL for odd or out-of-range n_qubits, A outside [0, n/2], NULL dst.
 * Pass the buffer to qvs_set_initial_state. */
int qvs_state_parity(int n_qubits, int A, void* dst, void* stream);

/* Sec. 2.1: evolve |psi0> through p layers; the final state stays on the device and its
 * objective is available from qvs_expectation. gammas, ts: host arrays of length p. */
int qvs_evolve(qvs_t h, int p, const double* gammas, const double* ts);

/* Sec. 2.3.2 (ex-QAOA): the phase of layer k becomes prod_j exp(-i gamma_{k,j} Sigma_j) with one
 * parameter per term Sigma_j = coef[j] Z_{u[j]} Z_{v[j]} (v[j] = -1: coef[j] Z_{u[j]}), the non-identity
 * Pauli terms of the quality operator (Z = +1 on |0>; qubit u = index bit n-1-u). Host arrays of
 * n_terms entries (copied), 0 <= n_terms <= 1024; u in 0..n-1, v = -1 or in 0..n-1 with v != u.
 * Used by qvs_evolve_ex / qvs_gradient_ex only; the objective stays <psi|Q|psi> with the handle's
 * quality. QVS_EINVAL for an out-of-range index, a repeated qubit or a non-finite coefficient. */
int qvs_set_phase_terms(qvs_t h, int n_terms, const int32_t* u, const int32_t* v, const double* coef);

/* ex-QAOA forward evolution (Sec. 2.3.2): gammas[k * n_terms + j] = gamma_{k,j} (host, p * n_terms
 * values), ts[k]. Each layer's phase angle sum_j gamma_{k,j} Sigma_j(x) is evaluated in the phase
 * passes in 32-bit fixed-point turns (exact modulo one turn for the coefficients reduced to 2^-32
 * turn). Hypercube mixer, complex64, n_qubits > 12 (QVS_EUNSUPPORTED otherwise); QVS_ESTATE
 * without terms. */
int qvs_evolve_ex(qvs_t h, int p, const double* gammas, const double* ts);

/* ex-QAOA objective and gradient: E, dgamma[k * n_terms + j] = df/dgamma_{k,j}, dt[k] (host arrays).
 * The adjoint phase passes store g(x) = 2 Im(conj(lambda) phi)(x); a Walsh-Hadamard transform per
 * 4096-amplitude tile turns it into every term's derivative sum_x coef_j Z..(x) g(x). Same
 * conditions as qvs_evolve_ex. */
int qvs_gradient_ex(qvs_t h, int p, const double* gammas, const double* ts, double* E, double* dgamma,
                    double* dt);

/* Objective-and-gradient callback of qvs_bfgs_minimize: writes f(x) and g = grad f(x) (n values)
 * for the point x; returns QVS_OK or an error status, which stops the minimisation. */
typedef int (*qvs_fg_fn)(const double* x, double* f, double* g, void* user);

/* Sec. 4: BFGS minimisation (the paper's default optimiser), on the host: direction -H g with the
 * inverse-Hessian estimate H (identity at the start and after a non-descent direction),
 * backtracking line search from step 1 halving (at most 30 times) until
 * f(x + a d) <= f(x) + 1e-4 a g.d, inverse update H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
 * (rho = 1/y.s, skipped when y.s <= 0). It stops when max |g| <= gtol (*stop_out = 0), after
 * max_iter iterations (1), or when no step of the line search decreases f enough (2: the
 * objective's rounding hides further descent; x and f stay at the last accepted point). x (n host
 * values) is the start and receives the result; f_out, iters_out, evals_out, stop_out may be NULL.
 * QVS_EINVAL for n outside 1..8192, NULL x or fg, negative max_iter or gtol; a callback error is
 * returned as is. */
int qvs_bfgs_minimize(int n, double* x, qvs_fg_fn fg, void* user, double gtol, int max_iter,
                      double* f_out, int* iters_out, int* evals_out, int* stop_out);

/* Sec. 4: minimise f(theta) = <theta|Q|theta> over theta = (gamma_1, t_1, ..., gamma_p, t_p) with
 * qvs_bfgs_minimize, each evaluation one qvs_gradient on the handle (device objective and adjoint
 * gradient). gammas, ts (host, p values) hold the start and receive the result. */
int qvs_optimise(qvs_t h, int p, double* gammas, double* ts, double gtol, int max_iter, double* f_out,
                 int* iters_out, int* evals_out, int* stop_out);

/* Sec. 2.1: f = <theta|Q|theta> of the last qvs_evolve (fp64 reduction). */
int qvs_expectation(qvs_t h, double* E);

/* Sec. 2.1 / Sec. 4: objective and its gradient in one forward sweep and one adjoint sweep.
 * Writes E, dgamma[p], dt[p] (host arrays). Afterwards the handle's state is undefined
 * (qvs_get_state needs a fresh qvs_evolve). */
int qvs_gradient(qvs_t h, int p, const double* gammas, const double* ts,
                 double* E, double* dgamma, double* dt);

/* Copy the current state (dim interleaved complex values in the handle's precision) to dst. */
int qvs_get_state(qvs_t h, void* dst, int on_device);

/* Number of kernels the last qvs_evolve / qvs_gradient launched. */
int qvs_last_launch_count(qvs_t h, int64_t* count);

/* Per-kernel statistics gathered while QVS_OPT_PROFILE is on: for slot = 0, 1, ... returns the
 * kernel's name (NUL-terminated, truncated to name_len), its launch count, the summed
 * event-timed duration in milliseconds, and the summed algorithmic bytes it must move (compulsory
 * reads + writes of state, adjoint vector, quality and tables). QVS_EINVAL past the last slot. */
int qvs_kernel_stats(qvs_t h, int slot, char* name, int name_len, int64_t* launches, double* ms,
                     double* bytes);

/* ----------------------------------------------------------------- quality generators
 * Write a quality vector into the device buffer q_out (caller-owned, dim entries of out_dtype)
 * on the given stream, computed on the GPU.
 *
 * Sec. 6.1, max-cut: q_i = sum over edges e=(u,v) with x_u(i) == x_v(i) of w_e (w = NULL: 1),
 *   dim = 2^n; edge endpoints are qubit indices (host arrays). The sum runs over the edges in
 *   the given order in fp64 and is rounded once to out_dtype (QVS_I32 needs w == NULL).
 *   1 <= n <= 40, 0 <= n_edges <= 1024 (no edges: q = 0); QVS_EINVAL otherwise, for an endpoint
 *   outside 0..n-1, a self-loop or a non-finite weight.
 */
int qvs_quality_maxcut(int n, int n_edges, const int32_t* eu, const int32_t* ev, const double* w,
                       int out_dtype, void* q_out, void* stream);

/* Quadratic form of qvs_set_quality_qubo (same arguments, same fixed-point rule), written for
 * all 2^n_qubits basis states (1 <= n_qubits <= 32) as F32 or F64 into the device buffer q_out. */
int qvs_quality_qubo(int n_qubits, double c, const double* hlin, const double* J, int out_dtype,
                     void* q_out, void* stream);

/* The fixed-point form of qvs_set_quality_qubo / qvs_quality_qubo (host only, no GPU): *F and the
 * integer coefficients ci (for c), hi[u] (for hlin[u]) and Ji[u*n + v] (for J[u*n + v], u < v; zero
 * on and below the diagonal), each the nearest integer to the coefficient times 2^F (halves away
 * from zero). q(x) = 2^-F (ci + sum_u hi[u] x_u + sum_{u<v} Ji[u*n+v] x_u x_v) exactly. QVS_EINVAL as
 * qvs_quality_qubo, or for a NULL output. */
int qvs_qubo_fixed_point(int n_qubits, double c, const double* hlin, const double* J, int* F, int32_t* ci,
                         int32_t* hi, int32_t* Ji);

/* The max-cut cost of qvs_quality_maxcut as a quadratic form (host only): an edge (u, v) with
 * weight w (w = NULL: 1) adds w [x_u == x_v] = w (1 - x_u - x_v + 2 x_u x_v), i.e. w to *c, -w to
 * hlin[u] and hlin[v], 2w to J[min(u,v)*n + max(u,v)]. Outputs: *c, hlin[n], J[n*n] (zeroed
 * first). QVS_EINVAL for an endpoint outside 0..n-1 or a self-loop. */
int qvs_qubo_from_maxcut(int n, int n_edges, const int32_t* eu, const int32_t* ev, const double* w,
                         double* c, double* hlin, double* J);

/* QWOA subset sums: q_i = sum_b w_b x_b(i) over items b = 0..n-1 (qubit b selects item b),
 * fp64 in item order, rounded once to out_dtype (F32 or F64). w: host array of n weights,
 * 1 <= n <= 40. */
int qvs_quality_subset(int n, const double* w, int out_dtype, void* q_out, void* stream);

/* Sec. 6.2, portfolio cost on a list of basis states (device array states[dim], n_qubits
 * qubits, asset a = qubits (2a long, 2a+1 short)): q = omega sum_ij sigma_ij z_i z_j
 * - (1-omega) sum_i r_i z_i, z_a = x_{2a} - x_{2a+1}; fp64, rounded once to out_dtype.
 * returns[M], cov[M*M] (row-major): host arrays, M = n_qubits/2 <= 32. */
int qvs_quality_portfolio(int n_qubits, int64_t dim, const int64_t* states, const double* returns,
                          const double* cov, double omega, int out_dtype, void* q_out, void* stream);

/* Sec. 2.3.1 (the hypercube mixer as commuting single-bit rotations), host only: the forward pass
 * schedule QVS_MIX_HYPERCUBE runs for n_qubits (12..32) and p layers. Pass j (0-based, in order)
 * applies, on tiles of 2^12 amplitudes: the rotations of layer layer_before[j] on the index bits
 * rot_bits[j] (bit b set = index bit b), then the phase of layer layer_phase[j], then the rotations
 * of layer layer_after[j] on the same bits (-1: that part is absent). shape[j]: 0 = first pass (the
 * initial state is generated or loaded), 1 = rotations, phase, rotations, 2 = rotations only,
 * 3 = last pass (rotations, objective, adjoint seed). type[j] is the tile type (0 = the 12 lowest
 * index bits). The adjoint sweep runs the same passes backwards. Call with shape = NULL to get
 * *n_passes only; otherwise every array has room for max_passes entries. QVS_EINVAL for sizes out
 * of range, a NULL array or too small max_passes. */
int qvs_hypercube_plan(int n_qubits, int p, int max_passes, int* n_passes, int32_t* shape, int32_t* type,
                       uint32_t* rot_bits, int32_t* layer_before, int32_t* layer_after, int32_t* layer_phase);

/* Sec. 2.4.1 (the parity-ring mixer's factors as passes), host only: how QVS_MIX_PARITY splits one
 * layer's Givens gates (B_odd, B_even, B_last of both rings, in the printed order) into shared-memory
 * passes. Each pass stages a tile of QVS_PARITY_TILE_BITS index bits (index bit b = qubit n-1-b) and
 * applies its gates in order, two at a time where they chain ("sweeps"). Call with ngates = NULL to
 * get *n_passes only; otherwise every array has room for max_passes passes:
 *   ngates[i], nsweeps[i]              gates and sweeps of pass i;
 *   tile_bits[i*TILE_BITS + j]         the tile's index bits (the 4 lowest index bits first);
 *   gate_bits[2*(i*MAX_GATES + g) + e] the two index bits of gate g (-1 past ngates[i]);
 *   sweep_kind[i*MAX_GATES + s]        0 = one gate, 1 = two gates on four distinct bits, 2 = two
 *                                      gates sharing one bit (-1 past nsweeps[i]);
 *   sweep_first[i*MAX_GATES + s]       the sweep's first gate (the second, if any, follows it).
 * 12 <= n_qubits <= 30. QVS_EINVAL for other sizes, a NULL array or too small max_passes. */
#define QVS_PARITY_TILE_BITS 12
#define QVS_PARITY_MAX_GATES 40
int qvs_parity_plan(int n_qubits, int max_passes, int* n_passes, int32_t* ngates, int32_t* tile_bits,
                    int32_t* gate_bits, int32_t* nsweeps, int32_t* sweep_kind, int32_t* sweep_first);

/* Host only: the register layouts of the tiled kernels, for checks of their index maps without a
 * GPU. For thread t and register r of step layout `layout`, index[t * regs + r] is the tile index
 * that register holds; slot[j] is the shared-memory slot of tile index j (8-byte words) and
 * global[j] its offset in the state vector for the first tile. Families:
 *   QVS_LAYOUT_HYPERCUBE        log2n 0; layouts 0..3 of the 2^12-amplitude hypercube tiles (the
 *                               contiguous tile type: global[j] = j);
 *   QVS_LAYOUT_CIRCULANT_COLUMN log2n 17..27; layouts 0..2 (one per transform digit) of that
 *                               size's column pass over 2^14-amplitude tiles;
 *   QVS_LAYOUT_CIRCULANT_ROW    log2n 0; layouts 0..2 of the row pass (contiguous tiles);
 *   QVS_LAYOUT_CIRCULANT_BOX    log2n 26, layout 0: slot[j] is the word of the tensor-copy box.
 * index has room for threads * regs values, slot and global for the tile's amplitudes (4096 or
 * 16384); *threads, *regs and *column_bits (the tile bits that are consecutive index bits)
 * describe the layout. QVS_EINVAL for another family, size or layout, or a NULL pointer. */
enum { QVS_LAYOUT_HYPERCUBE = 1, QVS_LAYOUT_CIRCULANT_COLUMN = 2, QVS_LAYOUT_CIRCULANT_ROW = 3,
       QVS_LAYOUT_CIRCULANT_BOX = 4 };
int qvs_tile_layout(int family, int log2n, int layout, int32_t* index, int32_t* slot, int32_t* global,
                    int* threads, int* regs, int* column_bits);

/* Sec. 3 (the sparse mixer's series expansion), host only: the Chebyshev coefficients the library
 * uses for exp(-i t W) v when the spectrum of W lies in [a - b, a + b]:
 *     exp(-i t W) = sum_{m=0}^{K} c_m T_m((W - a) / b),
 *     c_m = (2 - delta_{m0}) (-i)^m J_m(b t) e^{-i t a}   (the Jacobi-Anger expansion),
 * with K the smallest index whose tail bound sum_{m>K} 2 |J_m(b t)| is below tol (fp64 Bessel values,
 * std::cyl_bessel_j). c (NULL: query only) receives the K + 1 coefficients as interleaved re/im
 * doubles, room for 2 max_terms values; *n_terms = K + 1; *tail (may be NULL) = the tail bound,
 * which bounds the series' error in the 2-norm for a normalised v. QVS_EINVAL for non-finite a, b, t,
 * b < 0, tol <= 0 or max_terms outside 1..20000; QVS_ENUMERIC when more than max_terms terms are
 * needed. */
int qvs_chebyshev_coefficients(double a, double b, double t, double tol, int max_terms, double* c,
                               int* n_terms, double* tail);

/* Sec. 2.4.1: the XY-ring mixer sum_{a} (X_a X_{a+1} + Y_a Y_{a+1}) (a+1 mod n) restricted to
 * the n-qubit basis states of Hamming weight k, as CSR over those states in increasing integer
 * order. Host arrays; pass NULL outputs to query the sizes (*dim_out, *nnz_out). Values are all 2
 * (use implicit_value = 2). */
int qvs_xy_ring_csr(int n, int k, int64_t* states, int64_t* rowptr, int32_t* colind,
                    int64_t* dim_out, int64_t* nnz_out);

/* ----------------------------------------------------------------- batched solves
 * Sec. 4 parallelises over gradient components with MPI sub-communicators; the GPU analogue here
 * is many independent instances solved by one persistent kernel. A batch holds `count` QAOA
 * max-cut-style instances with the hypercube mixer and the equal-superposition initial state:
 * instance i has n_qubits[i] qubits (12 <= n <= 28) and layers[i] layers (1 <= p <= 64), complex64
 * state, fp32 qualities. The kernel's CTAs pull instances (longest first) from a device counter and
 * run each one's forward sweep, objective and adjoint gradient to completion. The first solve
 * picks the schedule (qvs_batch_info): one timed launch per candidate of 1 or 2 CTAs per SM and
 * checkpoint policy 0 or 1, or the cached choice for the same GPU and instance mix, unless
 * qvs_batch_set_schedule pinned one. It then captures parameters-in, the kernel and results-out
 * as a CUDA graph that later solves replay.
 *
 * Layouts: qualities are concatenated in instance order (instance i at offset
 * sum_{j<i} 2^n_j); parameters and gradient entries are concatenated per instance (instance i at
 * offset sum_{j<i} p_j). The handle owns its device workspace (one slot per resident CTA).
 */
typedef struct qvs_batch* qvs_batch_t;

int qvs_batch_create(qvs_batch_t* out, int count, const int32_t* n_qubits, const int32_t* layers,
                     void* stream);
/* q: the concatenated fp32 qualities (host or device per on_device); copied. */
int qvs_batch_set_quality(qvs_batch_t b, const float* q, int on_device);
/* gammas, ts: concatenated host arrays; E[count], dgamma and dt concatenated host outputs. */
int qvs_batch_gradient(qvs_batch_t b, const double* gammas, const double* ts, double* E,
                       double* dgamma, double* dt);
/* Many parameter sets of ONE instance, evaluated at once (the GPU analogue of the paper's Sec. 4
 * parallel evaluation of gradient components): every instance of the batch reads the same 2^n fp32
 * qualities q (host or device per on_device; copied). All instances must have the same n (QVS_EINVAL otherwise); their
 * depths and parameters may differ. */
int qvs_batch_set_quality_shared(qvs_batch_t b, const float* q, int on_device);

/* Sec. 4 on the device: minimise every instance's objective f_i(theta_i) over theta_i =
 * (gamma_1, t_1, ..., gamma_p, t_p) with its own BFGS, all at once. Each iteration evaluates the
 * objective and adjoint gradient of every still-active instance at its trial point in one launch of
 * the batched kernel, then one small kernel advances every instance's BFGS state: the same rules as
 * qvs_bfgs_minimize (Armijo test with c1 = 1e-4, at most 30 halvings, the inverse update skipped
 * when y.s <= 0, a reset to steepest descent on a non-descent direction), the inverse-Hessian
 * estimate kept in fp64 on the device. Both steps and the read-back of the active count form one
 * CUDA graph, replayed until no instance is active. gammas, ts: concatenated host arrays (as for
 * qvs_batch_gradient) holding the start points, overwritten with the results. Per-instance host
 * outputs (count entries each, NULL allowed): f_out the final objective, iters_out the accepted
 * iterations, evals_out the evaluations, stop_out 0 = max|g| <= gtol, 1 = max_iter reached,
 * 2 = no line-search step lowered f. Needs 2p <= 128 per instance (QVS_EUNSUPPORTED otherwise);
 * QVS_ESTATE before the qualities are set; QVS_EINVAL for negative gtol, max_iter outside
 * 0..100000 or non-finite start values. */
int qvs_batch_optimise(qvs_batch_t b, double* gammas, double* ts, double gtol, int max_iter, double* f_out,
                       int* iters_out, int* evals_out, int* stop_out);

/* Sec. 5 (the Ansatz's benchmark method with param_persist): a depth sweep D = d_min..d_max of
 * `repeats` optimisations of ONE QAOA instance (hypercube mixer, n qubits with 12 <= n <= 28,
 * equal-superposition start, 2^n fp32 qualities q in host or device memory per on_device). Each
 * depth is one batch of `repeats` parameter sets sharing q, optimised together by
 * qvs_batch_optimise(gtol, max_iter). Start points (the random draws are the caller's):
 *   D = d_min: repeat r starts from init[r*2*d_min .. ]: gamma_1..gamma_dmin, then t_1..t_dmin;
 *   D > d_min: every repeat starts from the best optimum (lowest f, first repeat on ties) of depth
 *              D-1 for layers 1..D-1 and from its own new-layer values for layer D, taken in order
 *              from the rest of init: repeats * (gamma_D, t_D) per depth.
 * Outputs (host): f_out[(d_max - d_min + 1) * repeats] the optimised objectives, depth-major;
 * best_theta: per depth D (in order) its best parameters, gamma_1..gamma_D then t_1..t_D
 * (sum over D of 2D values). QVS_EINVAL for a NULL pointer or a size out of range (2 d_max <= 128). */
int qvs_benchmark(int n, const float* q, int on_device, int d_min, int d_max, int repeats,
                  const double* init, double gtol, int max_iter, double* f_out, double* best_theta,
                  void* stream);

/* Pin the batch's schedule instead of tuning it: ctas_per_sm 1 or 2 (0: let the autotuner choose
 * on the next solve) and ckpt_policy 0 (forward states stored every ceil(sqrt(p)) layers,
 * uncomputed in between) or 1 (every pass boundary stored). QVS_EINVAL for other values,
 * QVS_ENOMEM when the policy's workspace cannot be allocated. */
int qvs_batch_set_schedule(qvs_batch_t b, int ctas_per_sm, int ckpt_policy);

/* What a batch does per solve (qvs_batch_info):
 *   ctas_per_sm      the autotuner's choice (0 before the first solve or optimisation);
 *   trial_ms[2]      its timed launches at 1 and 2 CTAs per SM under checkpoint policy 0;
 *   bytes_per_solve  compulsory global-memory bytes of one solve, summed over every pass of every
 *                    instance (8 per complex64 vector element read or written, 4 per quality read;
 *                    the HBM roofline's numerator whether or not a pass hits in L2);
 *   fma_per_solve    fp32 fused multiply-adds of one solve (a model: 2 per amplitude, rotated bit
 *                    and vector, 2 more per amplitude and bit for the adjoint accumulations, about
 *                    8 per phase; passes on the contiguous tile type rotate all 12 tile bits, the
 *                    others the 8 bits 4..11; the FP32-pipe roofline's numerator);
 *   amp_layers       sum over instances of 2^n p (the throughput unit);
 *   shared_quality   1 when every instance reads one shared quality vector;
 *   ckpt_policy      the autotuner's checkpoint policy: 0 = store the forward state every
 *                    ceil(sqrt(p)) layers and uncompute in between, 1 = store every pass boundary
 *                    (no uncompute, larger workspace);
 *   from_cache       1 when the choice came from the schedule cache (no trial launches): a JSON
 *                    file, QVS_TUNE_CACHE or else $HOME/.cache/qvs/batch_tune.json, keyed by GPU
 *                    name, SM count, instance count and the (n, p) multiset;
 *   trial_ms_all[4]  the timed candidates: policy 0 at 1 and 2 CTAs/SM, then policy 1 (0 = not
 *                    timed). */
typedef struct {
  int ctas_per_sm;
  int shared_quality;
  double trial_ms[2];
  double bytes_per_solve;
  double fma_per_solve;
  double amp_layers;
  int ckpt_policy;
  int from_cache;
  double trial_ms_all[4];
} qvs_batch_info_t;
int qvs_batch_info(qvs_batch_t b, qvs_batch_info_t* info);
int qvs_batch_destroy(qvs_batch_t b);

/* ----------------------------------------------------------------- allocation-free small solve
 * The paper has no counterpart to this entry point. It is for callers that cannot allocate device
 * memory at the moment they need a solve: code inside an allocator or memory-pool callback, a
 * real-time loop whose device memory is fixed up front, or a host runtime that owns all device
 * memory and forbids libraries from taking more.
 *
 * It computes what qvs_gradient computes for a handle with the hypercube (QAOA) mixer, the
 * equal-superposition initial state and dim = 2^n with n <= 12, but takes every input and output
 * from the caller and keeps its only scratch (the p forward states that the adjoint sweep reads
 * back) in one file-scope device array of QVS_NOALLOC_SCRATCH_BYTES bytes, which every GPU that
 * loads the library holds until the process exits. It never calls cudaMalloc, cudaFree or any
 * allocating routine.
 *
 *   n          qubits, 1 <= n <= 12 (dim = 2^n);
 *   precision  QVS_C64 or QVS_C128;
 *   p          layers, 1 <= p <= QVS_NOALLOC_MAX_LAYERS, and p * 2^n * (8 for C64, 16 for C128)
 *              must not exceed QVS_NOALLOC_SCRATCH_BYTES (QVS_EINVAL otherwise);
 *   q          device array of 2^n qualities: float for QVS_C64, double for QVS_C128;
 *   gammas, ts host arrays of length p (read before the call returns);
 *   out        device array of 1 + 2p doubles, written with E, dgamma[0..p), dt[0..p);
 *   stream     cudaStream_t or NULL.
 * The call only enqueues one kernel on `stream` and returns; `out` is valid once the stream has
 * reached that point. The first call on a device (with that device current) resolves the scratch
 * address with cudaGetSymbolAddress and sets the kernel's shared-memory limit. Every call on a
 * device shares the one scratch array and overwrites it (it keeps the last call's contents;
 * nothing in it needs to start at zero), so calls whose kernels may overlap on the GPU - on
 * different streams without ordering between them - race.
 */
#define QVS_NOALLOC_SCRATCH_BYTES (4u << 20)
#define QVS_NOALLOC_MAX_LAYERS 128
int qvs_gradient_small_noalloc(int n, int precision, int p, const void* q, const double* gammas,
                               const double* ts, double* out, void* stream);

const char* qvs_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* QVS_H */
