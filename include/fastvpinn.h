/*
 * fastvpinn.h -- C ABI of the B300 (sm_103a) FastVPINNs loss library.
 *
 * The library evaluates the variational loss of FastVPINNs (arXiv 2404.12063)
 * and its gradient with respect to the parameters of a tanh MLP, on one GPU:
 *
 *   u_NN(x; theta)            tanh MLP, linear output            (Sec. 2.2, Eq. NN)
 *   G[e][c][j][q]             quadrature-weighted, Jacobian-mapped test-function
 *                             premultipliers stacked over elements
 *                             (Sec. 4.4, Algorithm 3; App. A.1 bilinear map; App. A.2)
 *   R[e][j] = eps sum_q (Gx u_x + Gy u_y) + sum_q Gv (bx u_x + by u_y) - F[e][j]
 *                             cell weak residual (Sec. 2.3, Eq. VPINNs_Bound_Loss,
 *                             Algorithm 3; convection term of Eq. CD2D_strong)
 *   L = Lv + tau Lb + gamma Ls
 *       Lv = (1/N_test) sum_{e,j} R^2   (Algorithm 3, default)  or
 *            (1/N_elem) sum_{e,j} R^2   (Eq. loss)
 *       Lb = mean over Dirichlet points of (u - g)^2          (Eq. PINNs_Loss_components)
 *       Ls = mean over sensor points of (u - u_obs)^2         (Sec. 4.7)
 *
 * Conventions
 *   - Every call returns an int status: FV_OK or one of the FV_ERR_* codes.
 *     On failure, fv_last_error() returns a message for the calling thread.
 *   - Handles (fv_ctx, fv_mesh, fv_forcing, fv_bc, fv_adam) are owned by the
 *     library; each has a *_destroy call.  Device buffers passed in (params,
 *     grads, outputs) are owned by the caller.
 *   - Evaluation calls are asynchronous on the context's stream: they enqueue
 *     kernels and return; results are valid once the stream reaches them.
 *     The first evaluation of a (mesh, network) pair may allocate workspace,
 *     so make it before capturing a stream into a CUDA graph.
 *   - Numbers: vertices, f, boundary data are FP64 on the host.  Parameters,
 *     gradients and Adam state are FP64 when the network precision is FV_FP64
 *     and FP32 otherwise.  Scalar outputs are FP64.
 *   - Parameter layout (flat): for each affine map i = 0..n_layers-1, W_i
 *     row-major [out][in] followed by b_i [out].
 *   - Reference-element conventions: cell vertices b0..b3 counter-clockwise,
 *     mapped from (-1,-1), (1,-1), (1,1), (-1,1); quadrature index
 *     q = a*Q + b with a along xi; test index j = (m-1)*T + (n-1) with m along xi;
 *     test functions v_n = P_{n+1} - P_{n-1} (Sec. 4.5), Gauss-Lobatto-Legendre
 *     quadrature (Sec. 4.5).
 */
#ifndef FASTVPINN_H
#define FASTVPINN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FV_OK = 0,
  FV_ERR_ARG = 1,                 /* invalid argument (null handle, bad size, mismatched handles) */
  FV_ERR_DEGENERATE_ELEMENT = 2,  /* Jacobian determinant <= 0 at a quadrature node; see fv_last_error */
  FV_ERR_UNSUPPORTED = 3,         /* order / width / precision outside what the kernels support */
  FV_ERR_OOM = 4,                 /* device allocation failed */
  FV_ERR_CUDA = 5,                /* CUDA runtime error */
  FV_ERR_TIMEOUT = 6              /* a bounded device-side wait gave up */
};

typedef enum { FV_FP64 = 0, FV_FP32 = 1, FV_TF32 = 2, FV_BF16 = 3, FV_FP16 = 4 } fv_precision;
typedef enum { FV_NORM_TEST = 0, FV_NORM_ELEM = 1 } fv_norm;

typedef struct fv_ctx_s* fv_ctx;
typedef struct fv_mesh_s* fv_mesh;
typedef struct fv_forcing_s* fv_forcing;
typedef struct fv_bc_s* fv_bc;
typedef struct fv_adam_s* fv_adam;

/* Network shape: widths[0] = 2 (x, y), widths[n_layers] = 1 (u) or 2 (u and
 * the diffusion coefficient eps(x, y), the space-dependent inverse problem of
 * Sec. 4.7.2: the second output is eps itself, linear, and replaces the scalar
 * eps of fv_eval_opts in the diffusion term at every quadrature point; such
 * networks run in FP64 / FP32 and use the matrix-free contraction), hidden
 * widths in [1, 128]; 2..12 affine maps (at least one hidden layer); tanh
 * after every map but the last (Sec. 2.2, Eq. NN).  The parameters (and, for
 * the reverse sweep, an FP64 copy of their gradient) must fit in one CTA's
 * shared memory; larger networks return FV_ERR_UNSUPPORTED.  The last map's
 * parameters are W_L (row-major [outputs][inputs]) then b_L, as for every map. */
typedef struct {
  int n_layers;
  const int* widths; /* host, n_layers + 1 entries */
} fv_mlp_desc;

/* Per-evaluation options. */
typedef struct {
  fv_precision mlp_precision; /* FV_FP64, FV_FP32: CUDA-core FMA.  FV_BF16, FV_FP16: tcgen05 tensor cores,
                                 16-bit operands, FP32 accumulation (FP16 scales the reverse-sweep
                                 adjoints by a power of two).  FV_TF32 returns FV_ERR_UNSUPPORTED. */
  double eps;                 /* diffusion coefficient (Eq. CD2D_strong); used when eps_dev is NULL */
  const double* eps_dev;      /* optional device scalar read by the kernels instead of eps */
  double bx, by;              /* convection velocity b */
  fv_norm norm;               /* FV_NORM_TEST (Algorithm 3) or FV_NORM_ELEM (Eq. loss) */
} fv_eval_opts;

/* ---------------------------------------------------------------- context */

/* Bind a context to CUDA device `device` and stream `stream` (a cudaStream_t,
 * NULL = legacy default stream).  The context owns the evaluation workspace. */
int fv_ctx_create(fv_ctx* out, int device, void* stream);
int fv_ctx_set_stream(fv_ctx ctx, void* stream);
int fv_ctx_destroy(fv_ctx ctx);

/* Message describing the last failing call made by this thread ("" if none). */
const char* fv_last_error(void);

/* Per-kernel timing: when enabled, every evaluation records CUDA events
 * around each kernel on the context's stream; fv_ctx_kernel_times
 * synchronises the stream and returns accumulated milliseconds and launch
 * counts per kernel kind (names: fv_kernel_name).  Off by default. */
int fv_ctx_enable_timing(fv_ctx ctx, int on);

/* Activation stash of the reverse sweep, on by default: the forward kernel
 * also writes each tile's hidden activations (value and both tangents) to the
 * context's workspace, and the reverse kernel reads them by bulk copies
 * instead of recomputing those maps (Sec. 4.4's tensor form of the loss; the
 * reverse sweep of the network in Eq. NN).
 *   FV_BF16 / FV_FP16 gradients of networks with 3 or 4 hidden layers: the
 *     layers below the last hidden map, 16-bit, per 128-point tile (384 bytes
 *     per point and layer at width 50).
 *   FV_FP32 / FV_FP64: every hidden layer, in the path's precision, per tile
 *     of the reverse kernel (about 2.5 KB per point in FP32 at width 50x4).
 * Off: the reverse kernel recomputes them.  Results are bitwise the same
 * either way.  A fixed scratch area too small for it (fv_loss_grad_noalloc)
 * or a workspace allocation that fails with it falls back to recomputing.
 * Errors: FV_ERR_ARG (null context). */
int fv_ctx_set_activation_stash(fv_ctx ctx, int on);
int fv_ctx_kernel_times(fv_ctx ctx, int max_kinds, double* ms, int64_t* launches, int* n_kinds);
const char* fv_kernel_name(int kind);
int fv_ctx_reset_kernel_times(fv_ctx ctx);

/* ---------------------------------------------------------------- mesh tensors (a1) */

/* Precompute, once per mesh, the stacked premultiplier tensors of Algorithm 3
 * (Sec. 4.4) with the bilinear map of App. A.1 and the assembly of App. A.2:
 *   Gx[e][j][q] = w_q * (y_eta dv_j/dxi - y_xi dv_j/deta)      (= w_q |J| dv_j/dx)
 *   Gy[e][j][q] = w_q * (-x_eta dv_j/dxi + x_xi dv_j/deta)     (= w_q |J| dv_j/dy)
 *   Gv[e][j][q] = w_q |J| v_j                                   (only if with_mass_term)
 * computed in FP64 on the GPU and stored in `g_storage` (FV_FP64, FV_FP32 or
 * FV_BF16), plus the mapped quadrature points X[e][q] (FP64).
 *   vertices: host [n_vertices][2];  cells: host [n_elements][4] vertex indices, b0..b3
 *   quad_order Q in [2, 32] GLL points per direction; test_order T in [1, 16]
 * Errors: FV_ERR_ARG (bad sizes / vertex index out of range), FV_ERR_UNSUPPORTED
 * (orders), FV_ERR_DEGENERATE_ELEMENT (|J| <= 0 at some node; the message names
 * the first such element), FV_ERR_OOM, FV_ERR_CUDA.  Synchronises the stream. */
int fv_build_mesh_tensors(fv_ctx ctx, int n_vertices, const double* vertices, int n_elements,
                          const int32_t* cells, int quad_order, int test_order, fv_precision g_storage,
                          int with_mass_term, fv_mesh* out);

/* info[0..7] = n_elements, Q*Q, T*T, n_points (= n_elements*Q*Q), n_components (2 or 3),
 * G bytes actually stored (with padding), G bytes without padding, storage precision. */
int fv_mesh_info(fv_mesh mesh, int64_t* info);

/* Copy the mapped quadrature points to the host: xy_host [n_elements*Q*Q][2],
 * element-major, q = a*Q + b.  Synchronises the stream. */
int fv_mesh_quad_points(fv_mesh mesh, double* xy_host);

/* Copy the stored G tensor (converted to FP64) to the host for inspection:
 * g_host [n_elements][n_components][T*T][Q*Q], components (x, y[, v]). */
int fv_mesh_copy_g(fv_mesh mesh, double* g_host);
int fv_mesh_destroy(fv_mesh mesh);

/* How evaluations with this mesh contract grad u against the premultipliers.
 * FV_G_STORED (default): stream the stored G tensor (Alg. 3, G precomputed as
 * in App. A.2).  FV_G_MATRIX_FREE: rebuild the premultipliers inside the
 * contraction from the element vertices and the reference tables and sum them
 * by sum factorisation over the tensor-product test functions; the stored G
 * is not read.  Both give the same loss, residuals and gradients up to
 * rounding (the matrix-free form rounds geometry in the evaluation precision
 * instead of rounding G to the storage precision).  The paper precomputes G
 * (Sec. 4.2); the matrix-free form is this library's extension.
 * FV_G_REGULAR: the regular-element form of Alg. 2 (Sec. 4.3, premultipliers
 * as in the appendix's assembly): every element must be an axis-aligned
 * rectangle, so its premultipliers are one reference matrix scaled by the
 * element's Jacobian terms, and a tile of 128 elements' residuals and seeds
 * are four GEMMs with N = elements on the tensor cores (BF16 / FP16
 * evaluations, Q*Q and T*T <= 128); other precisions and shapes use the
 * matrix-free kernel, which computes the same quantities.
 * Errors: FV_ERR_ARG (null mesh, mode not 0, 1 or 2; FV_G_REGULAR on a mesh
 * with an element that is not an axis-aligned rectangle, named in the
 * message), FV_ERR_CUDA. */
#define FV_G_STORED 0
#define FV_G_MATRIX_FREE 1
#define FV_G_REGULAR 2
int fv_mesh_set_g_mode(fv_mesh mesh, int mode);

/* Autotune the contraction of Alg. 3 for this mesh at evaluation precision
 * `mlp_precision`: times each candidate launch plan (one or two shared-memory
 * stages per CTA, each with the planner's element grouping and with 1 to 4
 * elements per stage; lane splits as the planner picks them) on zero-valued
 * inputs and keeps the fastest in the mesh handle.  Later evaluations with
 * this mesh and precision use it; without a call the planner's two-stage
 * plan is used.  Plans differ only in how sums are grouped, so a tuned and an
 * untuned evaluation agree to rounding, and each plan is deterministic.
 * ms_out (nullable, host, 2 doubles) receives the median times of the best
 * two-stage and the best one-stage candidate.
 * Errors: FV_ERR_ARG (null mesh, precision not 0..4), FV_ERR_OOM, FV_ERR_CUDA.
 * Synchronises the stream; not allowed during stream capture. */
int fv_autotune(fv_ctx ctx, fv_mesh mesh, fv_precision mlp_precision, double* ms_out);

/* F[e][j] = sum_q Gv[e][j][q] f(X[e][q]) (App. A.2, "Compute Forcing Matrix"),
 * assembled in FP64 from the caller's f at the quadrature points
 * (host [n_elements*Q*Q], the order of fv_mesh_quad_points). */
int fv_assemble_forcing(fv_mesh mesh, const double* f_at_quad_host, fv_forcing* out);
int fv_forcing_copy(fv_forcing forcing, double* F_host /* [n_elements][T*T] */);
int fv_forcing_destroy(fv_forcing forcing);

/* ---------------------------------------------------------------- boundary / sensor data (a4) */

/* Dirichlet points (xy, g) with weight tau and optional sensor points (xs,
 * u_obs) with weight gamma (Sec. 2.2 L_b; Sec. 4.7 L_s).  Host arrays,
 * [n][2] points.  n_bd or n_sensor may be 0. */
int fv_bc_create(fv_ctx ctx, int n_bd, const double* bd_xy, const double* bd_g, double tau, int n_sensor,
                 const double* s_xy, const double* s_u, double gamma, fv_bc* out);
int fv_bc_destroy(fv_bc bc);

/* ---------------------------------------------------------------- evaluation (a2-a6) */

/* Loss only.  out_dev: device double[4] = (L, Lv, Lb, Ls).  bc may be NULL. */
int fv_loss(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
            const void* params_dev, const fv_eval_opts* opts, double* out_dev);

/* Loss and gradient in one pass (forward + tangents, contraction, adjoint,
 * reverse sweep; Sec. 4.4 "single backpropagation").
 *   grad_dev: device [n_params] (FP64 or FP32 as params), overwritten
 *   out_dev:  device double[5] = (L, Lv, Lb, Ls, dL/deps) */
int fv_loss_grad(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                 const void* params_dev, const fv_eval_opts* opts, void* grad_dev, double* out_dev);

/* Size of the fixed scratch area used by fv_loss_grad_noalloc (32 MiB). */
#define FV_NOALLOC_SCRATCH_BYTES (32u << 20)

/* fv_loss_grad for callers that must not allocate device memory.  (This is a
 * service of the library; the paper has no counterpart.)  Some callers cannot
 * call cudaMalloc: programs whose device memory is owned by a framework pool
 * that forbids raw allocations, and latency-critical training loops that
 * cannot afford cudaMalloc's implicit device-wide synchronisation.  This entry
 * point computes exactly what fv_loss_grad computes, with the same arguments,
 * but keeps every temporary in one fixed area of FV_NOALLOC_SCRATCH_BYTES that
 * is compiled into the library: each device that loads the library holds that
 * area until the process exits.  Nothing is allocated per call.
 *   - Caller: ordinary host code.  The call itself makes CUDA runtime calls
 *     (cudaSetDevice, the area's address lookup, cudaMemsetAsync, kernel
 *     launches, event records), so it cannot be made where the CUDA API is
 *     not allowed, such as inside a host function enqueued on a stream.
 *   - Size limit: problems whose temporaries exceed the area (roughly a million
 *     quadrature points in FP32, fewer in FP64 or with large networks) are
 *     rejected with FV_ERR_UNSUPPORTED and a message giving both sizes.  For the
 *     16-bit tensor-core forms the activation stash is left out when it does not
 *     fit (the reverse sweep then recomputes the hidden layers; same results).
 *   - Set-up: the first call on a device looks up the area's device address
 *     (cudaGetSymbolAddress, once per device, cached); make that first call
 *     before any stream capture.  A device reset (cudaDeviceReset) unloads the
 *     library's module and leaves the cached address stale: do not call this
 *     entry point on a device after resetting it.
 *   - Sharing: every call on a device uses the same area, and the area keeps
 *     the last call's contents.  Calls whose kernels overlap on the GPU (for
 *     example on two streams, or from two contexts) race on it; issue them one
 *     after another.  The per-kernel timing of fv_ctx_enable_timing is not
 *     recorded for these calls.
 * Arguments, layout, outputs and other errors as for fv_loss_grad. */
int fv_loss_grad_noalloc(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                         const void* params_dev, const fv_eval_opts* opts, void* grad_dev, double* out_dev);

/* Inspection: one loss + gradient evaluation that also copies out its
 * intermediates (synchronises the stream):
 *   U_dev  [S][P_tot]   u, du/dx, du/dy (, eps(x, y)) at the quadrature points then the boundary and
 *                       sensor points; S = 3, or 4 for a two-output network
 *   UB_dev [S][P_tot]   adjoint seeds dL/du, dL/du_x, dL/du_y (, dL/deps(x, y)) at the same points
 *   R_dev  [n_elements][T*T] (double) element residuals R[e][j]
 * U_dev / UB_dev are in the network precision (FP64 or FP32); any of the three
 * may be NULL.  out_dev as for fv_loss_grad.  Allocates a temporary gradient. */
int fv_eval_intermediates(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                          const void* params_dev, const fv_eval_opts* opts, void* U_dev, void* UB_dev,
                          double* R_dev, double* out_dev);

/* Point values: u, du/dx, du/dy (and eps(x, y) for a two-output network) at
 * n points (device [n][2] FP64 in, device [S][n] out in the params' precision,
 * S = 3 or 4). */
int fv_mlp_eval(fv_ctx ctx, const fv_mlp_desc* mlp, const void* params_dev, fv_precision prec, int n,
                const double* xy_dev, void* out_dev);

/* ---------------------------------------------------------------- inverse problem (a7) */

/* Adam state for the parameters and, if with_eps, the scalar eps
 * (Kingma & Ba; paper Sec. 4.7.1 trains eps with the network). */
int fv_adam_create(fv_ctx ctx, int64_t n_params, fv_precision prec, double beta1, double beta2,
                   double adam_eps, int with_eps, fv_adam* out);
int fv_adam_destroy(fv_adam adam);

/* One inverse-problem step (Sec. 4.7.1): loss + gradient with respect to
 * (theta, eps) with eps read from eps_dev (device double), then, if lr > 0,
 * one Adam update of params_dev and *eps_dev in place.
 * grad_dev: device [n_params] scratch/output; out_dev: device double[5]. */
int fv_inverse_step(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                    void* params_dev, double* eps_dev, const fv_eval_opts* opts, fv_adam adam, double lr,
                    void* grad_dev, double* out_dev);

/* ---------------------------------------------------------------- batches */

typedef struct {
  fv_mesh mesh;
  fv_forcing forcing;
  fv_bc bc;              /* may be NULL */
  const void* params_dev;
  void* grad_dev;
  double* out_dev;       /* device double[5] */
} fv_instance;

/* Captured training steps: n_steps consecutive fv_inverse_step calls with the
 * same arguments (loss + gradient, then the Adam update when lr > 0; Sec. 4.5)
 * recorded once into a CUDA graph, replayed by fv_graph_launch with one host
 * call on the context's stream.  Small problems are bound by the host-side
 * cost of issuing each step's launches; a graph removes it.  The graph owns a
 * workspace sized at creation, and keeps the device pointers it was given
 * (params, eps_dev, grad, out and the Adam state are updated in place on every
 * replay; their contents may change between launches, the pointers may not).
 * Results equal those of n_steps fv_inverse_step calls bitwise.  The handles
 * (mesh, forcing, bc, adam) must outlive the graph.
 * Errors: FV_ERR_ARG, FV_ERR_UNSUPPORTED (as fv_inverse_step), FV_ERR_OOM,
 * FV_ERR_CUDA (capture or instantiation failed). */
typedef struct fv_graph_s* fv_graph;
int fv_step_graph_create(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                         void* params, double* eps_dev, const fv_eval_opts* opts, fv_adam adam, double lr,
                         void* grad, double* out, int n_steps, fv_graph* out_graph);
int fv_graph_launch(fv_graph graph);
int fv_graph_destroy(fv_graph graph);

/* Loss + gradient of n independent problems sharing one network shape and
 * options (each with its own mesh, forcing, boundary data, parameters and
 * outputs).  fv_batch_plan allocates a workspace per instance and captures
 * all the instances' evaluations once into a CUDA graph, spread over
 * n_streams forked streams (largest instance first, each on the least loaded
 * stream) so that small instances run side by side; n_streams = 0 captures
 * with 1, 2, 4 and 8 streams, times three replays of each and keeps the
 * fastest.  Planning synchronises the stream; do it outside any capture.
 * fv_batch_loss_grad enqueues the batch as one graph launch on the context's
 * stream; parameters are read from the instances' device buffers at replay
 * time, so they may change between launches (the buffers may not move).
 * Device eps (opts->eps_dev) is not supported in batches.  With more than
 * one stream each instance's tensor-core network kernels run at most one CTA
 * per SM (room for the other streams' kernels), so their gradient partials
 * cover other point tiles than in a single call and the FP16/BF16 results
 * agree with single calls to rounding; all other results are bitwise equal.
 * fv_batch_info: streams in use and the tuning replay times (ms) for
 * 1, 2, 4, 8 streams (0 where not measured). */
typedef struct fv_batch_s* fv_batch;
int fv_batch_plan(fv_ctx ctx, int n, const fv_instance* inst, const fv_mlp_desc* mlp, const fv_eval_opts* opts,
                  int n_streams, fv_batch* out);
int fv_batch_loss_grad(fv_batch batch);
int fv_batch_info(fv_batch batch, int* n_streams, double* tuned_ms);
int fv_batch_destroy(fv_batch batch);

#ifdef __cplusplus
}
#endif
#endif /* FASTVPINN_H */
