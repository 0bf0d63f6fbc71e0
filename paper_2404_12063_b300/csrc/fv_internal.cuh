// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fastvpinn.h"

namespace fv {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

#define FV_CUDA_TRY(call)                                                              \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::fv::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                       \
      return _e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;               \
    }                                                                                  \
  } while (0)

#define FV_CHECK_ARG(cond, ...)         \
  do {                                  \
    if (!(cond)) {                      \
      ::fv::set_error(__VA_ARGS__);     \
      return FV_ERR_ARG;                \
    }                                   \
  } while (0)

// ------------------------------------------------------------------ limits
constexpr int kMaxLayers = 12;     // affine maps
constexpr int kMaxWidth = 128;     // hidden width
constexpr int kMaxQ = 32;
constexpr int kMaxT = 16;

// Kernel kinds for the optional per-kernel event timing.
enum KernelKind {
  K_G_BUILD = 0, K_FORCING, K_MLP_FWD, K_CONTRACT, K_BC, K_MLP_BWD, K_FINALIZE, K_ADAM,
  K_MLP_FWD_TC, K_MLP_BWD_TC, K_BATCH, K_SEED_SCALE, K_NUM_KINDS
};

// Network shape passed to kernels by value.
struct MlpShape {
  int L = 0;                    // affine maps
  int w[kMaxLayers + 1] = {};   // widths
  int off[kMaxLayers] = {};     // flat offset of W_i (b_i follows at off + w[i+1]*w[i])
  int n_params = 0;
};

bool make_shape(const fv_mlp_desc* d, MlpShape* s);

// ------------------------------------------------------------------ handles
struct TimingRec { int kind; cudaEvent_t a, b; };

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace fv

struct fv_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_sm = 148;
  int tc_ctas_cap = 0;              // > 0: at most this many tensor-core MLP CTAs per SM (kernels sharing the GPU)
  bool tc_stash = true;             // reverse sweeps read stored activations (false: recompute them)
  size_t smem_optin = 227 * 1024;
  size_t smem_per_sm = 228 * 1024;
  fv::Workspace ws;
  int* err_dev = nullptr;           // device error word (bounded waits, degenerate elements)
  cudaStream_t side = nullptr;      // boundary terms concurrent with the contraction (null: serial)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool timing = false;
  std::vector<fv::TimingRec> recs;
  std::vector<cudaEvent_t> free_events;
  double kind_ms[fv::K_NUM_KINDS] = {0};
  int64_t kind_launches[fv::K_NUM_KINDS] = {0};
};

struct fv_mesh_s {
  fv_ctx ctx = nullptr;
  int n_e = 0, Q = 0, T = 0, Nq = 0, Nt = 0, n_comp = 2;
  int64_t P = 0;
  fv_precision storage = FV_FP32;
  void* G = nullptr;                // [n_e] blocks of g_stride_bytes
  size_t g_stride_bytes = 0;        // bytes per element block (16-byte multiple)
  size_t g_elem_bytes = 0;          // bytes per element without padding
  double* X = nullptr;              // [P][2]
  double* tables = nullptr;         // xi[Q], w[Q], v[T][Q], dv[T][Q]
  double* verts = nullptr;          // [n_v][2]
  int* cells = nullptr;             // [n_e][4]
  int n_v = 0;
  int contract_stages[2] = {0, 0};  // tuned stages per CTA (FP32 / FP64 evaluation); 0 = default
  int contract_elems[2] = {0, 0};   // tuned elements per stage (FP32 / FP64 evaluation); 0 = the planner's choice
  int g_mode = FV_G_STORED;         // contraction from the stored G or matrix-free
  float* jreg = nullptr;            // regular mode: per element y_eta, x_xi, |J| (FP32), [n_e][3]
  void* reg_ref[2] = {nullptr, nullptr};   // regular mode: FP16 / BF16 shared-memory images of the reference matrix
};

struct fv_forcing_s {
  fv_mesh mesh = nullptr;
  double* F = nullptr;              // [n_e][Nt]
  float* F32 = nullptr;             // FP32 copy for the FP32 / tensor-core paths
};

struct fv_bc_s {
  fv_ctx ctx = nullptr;
  int n_bd = 0, n_s = 0;
  double* xy = nullptr;             // [n_bd + n_s][2]
  double* val = nullptr;            // [n_bd + n_s]
  double tau = 0, gamma = 0;
};

struct fv_adam_s {
  fv_ctx ctx = nullptr;
  int64_t n = 0;
  fv_precision prec = FV_FP32;
  double beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
  int with_eps = 0;
  void* m = nullptr;                // [n] (+ eps slot in me)
  void* v = nullptr;
  double* me = nullptr;             // [2]: m, v of eps
  int* t = nullptr;                 // step count (device)
};

namespace fv {

// Workspace: grows on demand (synchronous cudaMalloc).
int ws_reserve(fv_ctx ctx, size_t bytes, void** out);

// Timing hooks around each launch (no-ops unless ctx->timing).
void time_begin(fv_ctx ctx, int kind, cudaEvent_t* a);
void time_end(fv_ctx ctx, int kind, cudaEvent_t a);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class T> struct Real;
template <> struct Real<double> { using type = double; };
template <> struct Real<float> { using type = float; };
template <> struct Real<__nv_bfloat16> { using type = float; };

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Neumaier-compensated accumulator (Kahan-Babuska), FP64.
struct KSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// Bilinear map of a quad element (App. A.1): x = x0 + x1 xi + x2 eta + x3 xi eta
// (likewise y) from its counter-clockwise vertices b0..b3.
struct Bilin { double x0, x1, x2, x3, y0, y1, y2, y3; };

__device__ __forceinline__ Bilin bilin_coeffs(const double* verts, const int* cell) {
  double vx[4], vy[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { vx[k] = verts[2 * cell[k]]; vy[k] = verts[2 * cell[k] + 1]; }
  Bilin c;
  c.x0 = 0.25 * (vx[0] + vx[1] + vx[2] + vx[3]);
  c.x1 = 0.25 * (-vx[0] + vx[1] + vx[2] - vx[3]);
  c.x2 = 0.25 * (-vx[0] - vx[1] + vx[2] + vx[3]);
  c.x3 = 0.25 * (vx[0] - vx[1] + vx[2] - vx[3]);
  c.y0 = 0.25 * (vy[0] + vy[1] + vy[2] + vy[3]);
  c.y1 = 0.25 * (-vy[0] + vy[1] + vy[2] - vy[3]);
  c.y2 = 0.25 * (-vy[0] - vy[1] + vy[2] + vy[3]);
  c.y3 = 0.25 * (vy[0] - vy[1] + vy[2] - vy[3]);
  return c;
}


// Compensated (Kahan) accumulator in the evaluation precision.
template <class R>
struct KahanR {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R x) {
    const R y = x - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Launch attributes queried once per device and kernel (the queries cost
// microseconds of host time each, which small problems would pay every call).
// Raises the kernel's dynamic shared-memory limit to at least `bytes`.
cudaError_t ensure_smem_attr(fv_ctx ctx, const void* kernel, size_t bytes);
// Resident CTAs per SM for (kernel, threads, dynamic shared memory); 0 on error.
int occupancy(fv_ctx ctx, const void* kernel, int threads, size_t smem);
// Resident CTAs per SM from the kernel's registers, shared memory and threads
// alone.  For the kernels that allocate tensor memory the occupancy query
// answers one whatever their resources; their callers cap this count by the
// tensor-memory columns each CTA allocates.
int resident_ctas(fv_ctx ctx, const void* kernel, int threads, size_t smem);

// ------------------------------------------------------------------ launchers
// Each returns FV_OK or an error code and enqueues on ctx->stream.
struct EvalPlan {
  MlpShape shape;
  fv_precision prec;        // network precision
  int64_t P_mesh = 0;       // quadrature points
  int n_bd = 0, n_s = 0;
  int64_t P_tot = 0;        // P_mesh + n_bd + n_s
  bool want_grad = false;
  float* seed_max = nullptr;  // FP16 reverse sweep: the kernels that write seeds raise this to max |seed|
};

// max(*word, v) for non-negative floats (their bit patterns order like the values)
__device__ __forceinline__ void atomic_max_nonneg(float* word, float v) {
  if (v > 0.f) atomicMax(reinterpret_cast<int*>(word), __float_as_int(v));
}

// A warp's largest value, then one atomic per warp (null word: nothing).
__device__ __forceinline__ void warp_max_to(float* word, float v) {
  if (!word) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(word, v);
}

// stash: null, or mlp_simt_stash_bytes(ctx, pl) bytes that the forward fills
// with the hidden layers (value and tangents) the reverse sweep then reads
// instead of recomputing them.
int launch_mlp_fwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xmesh, const double* Xextra,
                   void* U, void* stash = nullptr);
size_t mlp_simt_stash_bytes(fv_ctx ctx, const EvalPlan& pl);   // 0: no stash for this network
int autotune_contract(fv_ctx ctx, fv_mesh mesh, fv_precision prec, double* ms_out);
int launch_contract_mfree(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, const EvalPlan& pl, const void* U,
                          void* UB, double eps, const double* eps_dev, double bx, double by, double rscale,
                          double* partials, int* n_partials_out, double* R_out);
void mfree_grid(fv_ctx ctx, fv_mesh mesh, fv_precision prec, int* grid, int* warps_per_cta, size_t* smem);
bool regular_supported(fv_mesh mesh, fv_precision prec);
int regular_grid(fv_ctx ctx, fv_mesh mesh);
int check_regular_mesh(fv_mesh mesh, std::vector<float>* scales);
int build_regular_reference(fv_mesh mesh);
int launch_contract_regular(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, const EvalPlan& pl, const void* U,
                            void* UB, double eps, const double* eps_dev, double bx, double by, double rscale,
                            double* partials, int* n_partials_out, double* R_out);
int launch_contract(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, const EvalPlan& pl, const void* U, void* UB,
                    double eps, const double* eps_dev, double bx, double by, double rscale, double* partials,
                    int* n_partials_out, double* R_out = nullptr);
int contract_grid(fv_ctx ctx, fv_mesh mesh, fv_precision prec, int* grid, int* elems_per_stage, int* stages,
                  size_t* smem, bool matrix_free = false);
int launch_bc(fv_ctx ctx, fv_bc bc, const EvalPlan& pl, const void* U, void* UB, double* partial2);
int launch_mlp_bwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xmesh, const double* Xextra,
                   const void* UB, double* gpart, int* n_blocks_out, const void* stash = nullptr);
int mlp_bwd_blocks(fv_ctx ctx, const EvalPlan& pl);
int launch_finalize(fv_ctx ctx, const EvalPlan& pl, const double* cpart, int n_cpart, const double* bcpart,
                    const double* gpart, int n_gpart, double inv_norm, double tau, double gamma, int n_bd, int n_s,
                    void* grad, double* out);

// Tensor-core MLP paths (tcgen05).
// stash: null, or mlp_tc_stash_bytes(pl) bytes that the forward fills with the
// hidden activations the reverse sweep reads instead of recomputing them.
int launch_mlp_fwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xmesh,
                      const double* Xextra, void* U,
                      int* tile_counter, void* stash);
int launch_mlp_bwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xmesh,
                      const double* Xextra, const void* UB, double* gpart, int* n_blocks_out,
                      const float* seed_absmax, const void* stash);
size_t mlp_tc_stash_bytes(const EvalPlan& pl);   // 0: this network has no stash
bool tc_supported(const EvalPlan& pl);
int mlp_bwd_tc_blocks(fv_ctx ctx, const EvalPlan& pl);

}  // namespace fv
