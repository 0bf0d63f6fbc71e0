// C ABI: contexts, workspace, evaluation entry points, Adam, batches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include <map>
#include <tuple>
#include "fv_internal.cuh"

namespace fv {

namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_set;
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;
std::map<std::tuple<int, const void*, int, size_t>, int> g_res;
}  // namespace

cudaError_t ensure_smem_attr(fv_ctx ctx, const void* kernel, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t& have = g_smem_set[{ctx->device, kernel}];
  if (bytes <= have) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

int occupancy(fv_ctx ctx, const void* kernel, int threads, size_t smem) {
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_occ.find({ctx->device, kernel, threads, smem});
    if (it != g_occ.end()) return it->second;
  }
  if (ensure_smem_attr(ctx, kernel, smem) != cudaSuccess) { cudaGetLastError(); return 0; }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_attr_mu);
  g_occ[{ctx->device, kernel, threads, smem}] = n;
  return n;
}

int resident_ctas(fv_ctx ctx, const void* kernel, int threads, size_t smem) {
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_res.find({ctx->device, kernel, threads, smem});
    if (it != g_res.end()) return it->second;
  }
  cudaFuncAttributes fa;
  int regs_sm = 0, thr_sm = 0, smem_sm = 0, reserved = 0;
  if (ensure_smem_attr(ctx, kernel, smem) != cudaSuccess || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;     // allocated per warp in units of 256
  int n = std::min(thr_sm / (warps * 32), regs_sm / std::max(1, regs_warp * warps));
  n = std::min<int>(n, (int)(smem_sm / (smem + fa.sharedSizeBytes + reserved)));
  std::lock_guard<std::mutex> lk(g_attr_mu);
  g_res[{ctx->device, kernel, threads, smem}] = n;
  return n;
}


static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

bool make_shape(const fv_mlp_desc* d, MlpShape* s) {
  if (!d || !d->widths || d->n_layers < 2 || d->n_layers > kMaxLayers) return false;
  if (d->widths[0] != 2 || (d->widths[d->n_layers] != 1 && d->widths[d->n_layers] != 2)) return false;
  s->L = d->n_layers;
  int o = 0;
  for (int i = 0; i <= d->n_layers; ++i) {
    const int w = d->widths[i];
    if (i > 0 && i < d->n_layers && (w < 1 || w > kMaxWidth)) return false;
    s->w[i] = w;
  }
  for (int i = 0; i < d->n_layers; ++i) { s->off[i] = o; o += s->w[i + 1] * s->w[i] + s->w[i + 1]; }
  s->n_params = o;
  return true;
}

int ws_reserve(fv_ctx ctx, size_t bytes, void** out) {
  if (ctx->ws.bytes < bytes) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaFree(ctx->ws.ptr);
    ctx->ws.ptr = nullptr; ctx->ws.bytes = 0;
    const size_t want = std::max(bytes, (size_t)(1 << 20));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws.ptr, want);
    if (e != cudaSuccess) {
      set_error("workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
    }
    ctx->ws.bytes = want;
  }
  *out = ctx->ws.ptr;
  return FV_OK;
}

static cudaEvent_t get_event(fv_ctx ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void time_begin(fv_ctx ctx, int kind, cudaEvent_t* a) {
  (void)kind;
  *a = nullptr;
  if (!ctx->timing) return;
  *a = get_event(ctx);
  cudaEventRecord(*a, ctx->stream);
}

void time_end(fv_ctx ctx, int kind, cudaEvent_t a) {
  if (!ctx->timing || !a) return;
  cudaEvent_t b = get_event(ctx);
  cudaEventRecord(b, ctx->stream);
  ctx->recs.push_back({kind, a, b});
}

namespace {

constexpr size_t kAlign = 256;
inline size_t al(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Fixed-shape tree sum over a block of 256 threads (deterministic).
__device__ __forceinline__ double block_sum256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Boundary and sensor terms (Sec. 2.2 L_b, Sec. 4.7 L_s) and their seeds.
template <class R>
__global__ void __launch_bounds__(256) bc_kernel(const double* __restrict__ val, int n_bd, int n_s, double tau,
                                                 double gamma, const R* __restrict__ U, R* __restrict__ UB,
                                                 int64_t P_mesh, int64_t P_tot, double* __restrict__ partial2,
                                                 float* __restrict__ seed_max) {
  __shared__ double red[256];
  R lb = 0, ls = 0;
  float smx = 0.f;
  const R cb = (R)(2.0 * tau / (n_bd > 0 ? n_bd : 1)), cs = (R)(2.0 * gamma / (n_s > 0 ? n_s : 1));
  const int nd = n_bd + n_s;
  for (int d0 = threadIdx.x; d0 < nd; d0 += 4 * blockDim.x) {
    R uv[4];
    double gv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {          // loads of four points first, then their terms in order
      const int d = d0 + k * blockDim.x;
      uv[k] = d < nd ? U[P_mesh + d] : (R)0;
      gv[k] = d < nd ? val[d] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int d = d0 + k * blockDim.x;
      if (d >= nd) break;
      const int64_t gp = P_mesh + d;
      const R diff = uv[k] - (R)gv[k];
      R seed;
      if (d < n_bd) { lb += diff * diff; seed = cb * diff; }
      else { ls += diff * diff; seed = cs * diff; }
      smx = fmaxf(smx, fabsf((float)seed));
      if (UB) {
        UB[gp] = seed;
        UB[P_tot + gp] = (R)0;
        UB[2 * P_tot + gp] = (R)0;
      }
    }
  }
  warp_max_to(seed_max, smx);
  const double a = block_sum256((double)lb, red);
  const double b = block_sum256((double)ls, red);
  if (threadIdx.x == 0) { partial2[0] = a; partial2[1] = b; }
}

// Deterministic final sums: the gradient over per-CTA partials and the loss
// scalars, both as fixed-shape trees.  out = (L, Lv, Lb, Ls, dL/deps).
// Gradient (blocks 0 .. gridDim-2): 8 threads per parameter, each summing a
// strided subset of the partials in a fixed order (loads issued eight at a
// time), then a 3-level shuffle tree.  Loss scalars: the last block.
template <class R>
__global__ void __launch_bounds__(256) finalize_kernel(const double* __restrict__ cpart, int n_cpart,
                                                       const double* __restrict__ bcpart,
                                                       const double* __restrict__ gpart, int n_gpart, int n_params,
                                                       double inv_norm, double tau, double gamma, int n_bd, int n_s,
                                                       R* __restrict__ grad, double* __restrict__ out) {
  __shared__ double red[256];
  if (grad && blockIdx.x + 1 < gridDim.x) {
    const int sub = threadIdx.x & 7;
    const int i = blockIdx.x * 32 + (threadIdx.x >> 3);
    double s = 0.0;
    if (i < n_params)
      for (int b0 = sub; b0 < n_gpart; b0 += 64) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int b = b0 + 8 * u;
          t[u] = b < n_gpart ? gpart[(size_t)b * n_params + i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (b0 + 8 * u < n_gpart) s += t[u];
      }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (i < n_params && sub == 0) grad[i] = (R)s;
  }
  if (blockIdx.x + 1 == gridDim.x) {
    double l = 0.0, d = 0.0;
    for (int b = threadIdx.x; b < n_cpart; b += blockDim.x) { l += cpart[2 * b]; d += cpart[2 * b + 1]; }
    l = block_sum256(l, red);
    d = block_sum256(d, red);
    if (threadIdx.x == 0) {
      const double Lv = inv_norm * l;
      const double Lb = n_bd ? bcpart[0] / n_bd : 0.0;
      const double Ls = n_s ? bcpart[1] / n_s : 0.0;
      out[0] = Lv + tau * Lb + gamma * Ls;
      out[1] = Lv;
      out[2] = Lb;
      out[3] = Ls;
      out[4] = d;
    }
  }
}

// Adam (Kingma & Ba, bias-corrected) on theta and, when trained, eps.  The
// bias corrections are computed once, in FP64, by one thread; the element
// updates run in the parameters' precision (FP64 arithmetic is slow on this
// part, and FP32 parameters gain nothing from it).
template <class R>
__global__ void adam_kernel(R* __restrict__ p, const R* __restrict__ g, int64_t n, R* __restrict__ m,
                            R* __restrict__ v, double* eps_p, const double* dLde, double* me, int with_eps, int* t,
                            double lr, double b1, double b2, double ae) {
  __shared__ double s_c[2];
  const int tt = *t + 1;
  if (threadIdx.x == 0) {
    s_c[0] = 1.0 - pow(b1, (double)tt);
    s_c[1] = 1.0 - pow(b2, (double)tt);
  }
  __syncthreads();
  const double c1 = s_c[0], c2 = s_c[1];
  const R rb1 = (R)b1, rb2 = (R)b2, rc1 = (R)c1, rc2 = (R)c2, rlr = (R)lr, rae = (R)ae;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const R gi = g[i];
    const R mi = rb1 * m[i] + ((R)1 - rb1) * gi;
    const R vi = rb2 * v[i] + ((R)1 - rb2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = p[i] - rlr * (mi / rc1) / (sqrt(vi / rc2) + rae);
  }
  if (with_eps && threadIdx.x == 0) {
    const double gi = dLde[0];
    const double mi = b1 * me[0] + (1.0 - b1) * gi;
    const double vi = b2 * me[1] + (1.0 - b2) * gi * gi;
    me[0] = mi; me[1] = vi;
    eps_p[0] -= lr * (mi / c1) / (sqrt(vi / c2) + ae);
  }
  __syncthreads();
  if (threadIdx.x == 0) *t = tt;
}

int check_eval(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp, const void* params,
               const fv_eval_opts* opts, MlpShape* sh) {
  FV_CHECK_ARG(ctx && mesh && forcing && mlp && params && opts, "evaluation: null argument");
  FV_CHECK_ARG(forcing->mesh == mesh, "evaluation: forcing was assembled on a different mesh");
  FV_CHECK_ARG(mesh->ctx == ctx && (!bc || bc->ctx == ctx), "evaluation: handles belong to another context");
  FV_CHECK_ARG(opts->norm == FV_NORM_TEST || opts->norm == FV_NORM_ELEM, "evaluation: bad norm");
  if (!make_shape(mlp, sh)) {
    set_error("network shape unsupported: need widths[0]=2, widths[L]=1 or 2, 2..%d affine maps, hidden widths 1..%d",
              kMaxLayers, kMaxWidth);
    return FV_ERR_UNSUPPORTED;
  }
  const fv_precision p = opts->mlp_precision;
  if (p != FV_FP64 && p != FV_FP32 && p != FV_TF32 && p != FV_BF16 && p != FV_FP16) {
    set_error("evaluation: unknown precision");
    return FV_ERR_UNSUPPORTED;
  }
  if (p == FV_FP64 && mesh->storage != FV_FP64) {
    set_error("FP64 evaluation needs a mesh built with FV_FP64 storage");
    return FV_ERR_UNSUPPORTED;
  }
  if ((opts->bx != 0.0 || opts->by != 0.0) && mesh->n_comp != 3) {
    set_error("non-zero convection needs a mesh built with with_mass_term=1");
    return FV_ERR_ARG;
  }
  return FV_OK;
}

struct WsLayout {
  size_t U, UB, cpart, bcpart, gpart, smax, ctr, stash, total;
};

// The core evaluation shared by fv_loss, fv_loss_grad and fv_inverse_step.
// Restores a context's timing switch on scope exit.
struct TimingOff {
  fv_ctx ctx;
  bool saved;
  explicit TimingOff(fv_ctx c, bool off) : ctx(c), saved(c ? c->timing : false) { if (c && off) c->timing = false; }
  ~TimingOff() { if (ctx) ctx->timing = saved; }
};

// fixed_ws: when given, all temporaries go to this caller-supplied device area
// of fixed_ws_bytes (no workspace growth, no timing events).
int evaluate(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp, const void* params,
             const fv_eval_opts* opts, const double* eps_dev, bool want_grad, void* grad, double* out,
             void* U_copy = nullptr, void* UB_copy = nullptr, double* R_out = nullptr, void* fixed_ws = nullptr,
             size_t fixed_ws_bytes = 0, size_t* ws_bytes_only = nullptr) {
  TimingOff timing_guard(ctx, fixed_ws != nullptr);
  MlpShape sh;
  int rc = check_eval(ctx, mesh, forcing, bc, mlp, params, opts, &sh);
  if (rc) return rc;
  EvalPlan pl;
  pl.shape = sh;
  pl.prec = opts->mlp_precision;
  pl.P_mesh = mesh->P;
  pl.n_bd = bc ? bc->n_bd : 0;
  pl.n_s = bc ? bc->n_s : 0;
  pl.P_tot = pl.P_mesh + pl.n_bd + pl.n_s;
  pl.want_grad = want_grad;
  const bool tc = pl.prec == FV_TF32 || pl.prec == FV_BF16 || pl.prec == FV_FP16;
  if (tc && !tc_supported(pl)) {
    set_error("tensor-core path does not support this network shape");
    return FV_ERR_UNSUPPORTED;
  }
  const size_t rsz = pl.prec == FV_FP64 ? 8 : 4;
  int cgrid, E, S;
  size_t csmem;
  const int n_str = sh.w[sh.L] == 2 ? 4 : 3;        // value streams: u, u_x, u_y (, eps(x, y))
  contract_grid(ctx, mesh, pl.prec, &cgrid, &E, &S, &csmem, n_str == 4);
  int nb = 0;
  if (want_grad) {
    nb = tc ? mlp_bwd_tc_blocks(ctx, pl) : mlp_bwd_blocks(ctx, pl);
    if (nb <= 0) return nb < 0 ? -nb : FV_ERR_UNSUPPORTED;
  }
  WsLayout w;
  size_t o = 0;
  w.U = o; o += al(n_str * pl.P_tot * rsz);
  w.UB = o; o += want_grad ? al(n_str * pl.P_tot * rsz) : 0;
  w.cpart = o; o += al(2 * (size_t)cgrid * 8);
  w.bcpart = o; o += al(2 * 8);
  w.gpart = o; o += al((size_t)nb * sh.n_params * 8);
  w.smax = o; o += al(16);
  w.ctr = o; o += al(16);
  // activation stash of the reverse sweep; left out (the reverse
  // kernel recomputes) when a fixed scratch area has no room for it
  size_t stash_bytes = !want_grad || !ctx->tc_stash ? 0 : tc ? mlp_tc_stash_bytes(pl) : mlp_simt_stash_bytes(ctx, pl);
  if (fixed_ws && o + al(stash_bytes) > fixed_ws_bytes) stash_bytes = 0;
  w.stash = o; o += al(stash_bytes);
  w.total = o;
  if (ws_bytes_only) {          // size query only: nothing is launched
    *ws_bytes_only = w.total;
    return FV_OK;
  }
  void* base;
  if (fixed_ws) {
    if (w.total > fixed_ws_bytes) {
      set_error("this problem needs %zu bytes of scratch; the fixed scratch area holds %zu", w.total, fixed_ws_bytes);
      return FV_ERR_UNSUPPORTED;
    }
    base = fixed_ws;
  } else {
    rc = ws_reserve(ctx, w.total, &base);
    if (rc == FV_ERR_OOM && stash_bytes) {   // no room for the stash: the reverse sweep recomputes
      cudaGetLastError();
      w.total -= al(stash_bytes);
      stash_bytes = 0;
      rc = ws_reserve(ctx, w.total, &base);
    }
    if (rc) return rc;
  }
  char* b = static_cast<char*>(base);
  void* U = b + w.U;
  void* UB = want_grad ? b + w.UB : nullptr;
  double* cpart = reinterpret_cast<double*>(b + w.cpart);
  double* bcpart = reinterpret_cast<double*>(b + w.bcpart);
  double* gpart = reinterpret_cast<double*>(b + w.gpart);
  float* smax = reinterpret_cast<float*>(b + w.smax);
  int* tile_ctr = reinterpret_cast<int*>(b + w.ctr);
  void* stash = stash_bytes ? b + w.stash : nullptr;
  const double* Xe = bc ? bc->xy : nullptr;

  rc = tc ? launch_mlp_fwd_tc(ctx, pl, params, mesh->X, Xe, U, tile_ctr, stash)
          : launch_mlp_fwd(ctx, pl, params, mesh->X, Xe, U, stash);
  if (rc) return rc;
  const double inv_norm = 1.0 / (opts->norm == FV_NORM_TEST ? mesh->Nt : mesh->n_e);
  // Boundary and sensor terms read U and write the boundary points' seeds and
  // two partials, disjoint from the contraction's outputs: on the context's
  // side stream they run concurrently with it (serially when timing kernels).
  // FP16 reverse sweep: the kernels that write seeds (contraction, boundary
  // terms) raise *smax to max |seed|; the reverse sweep scales by it
  if (want_grad && pl.prec == FV_FP16) {
    FV_CUDA_TRY(cudaMemsetAsync(smax, 0, sizeof(float), ctx->stream));
    pl.seed_max = smax;
  }
  const bool has_bc = bc && pl.n_bd + pl.n_s > 0;
  const bool concurrent = has_bc && ctx->side && !ctx->timing;
  const cudaStream_t bst = concurrent ? ctx->side : ctx->stream;
  if (concurrent) {
    FV_CUDA_TRY(cudaEventRecord(ctx->ev_fork, ctx->stream));
    FV_CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  if (has_bc) {
    cudaEvent_t ta;
    time_begin(ctx, K_BC, &ta);
    if (pl.prec == FV_FP64)
      bc_kernel<double><<<1, 256, 0, bst>>>(bc->val, pl.n_bd, pl.n_s, bc->tau, bc->gamma, (const double*)U,
                                            (double*)UB, pl.P_mesh, pl.P_tot, bcpart, pl.seed_max);
    else
      bc_kernel<float><<<1, 256, 0, bst>>>(bc->val, pl.n_bd, pl.n_s, bc->tau, bc->gamma, (const float*)U,
                                           (float*)UB, pl.P_mesh, pl.P_tot, bcpart, pl.seed_max);
    time_end(ctx, K_BC, ta);
    FV_CUDA_TRY(cudaGetLastError());
    if (concurrent) FV_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->side));
  } else {
    FV_CUDA_TRY(cudaMemsetAsync(bcpart, 0, 16, ctx->stream));
  }
  int ncp = 0;
  rc = launch_contract(ctx, mesh, forcing, pl, U, UB, opts->eps, eps_dev ? eps_dev : opts->eps_dev, opts->bx, opts->by,
                       2.0 * inv_norm, cpart, &ncp, R_out);
  if (concurrent) FV_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));   // join before any return
  if (rc) return rc;
  if (n_str == 4 && UB && pl.P_tot > pl.P_mesh)       // boundary and sensor points: no eps(x, y) seed
    FV_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(UB) + (3 * pl.P_tot + pl.P_mesh) * rsz, 0,
                                (pl.P_tot - pl.P_mesh) * rsz, ctx->stream));
  if (U_copy) FV_CUDA_TRY(cudaMemcpyAsync(U_copy, U, n_str * pl.P_tot * rsz, cudaMemcpyDeviceToDevice, ctx->stream));
  if (UB_copy && UB)
    FV_CUDA_TRY(cudaMemcpyAsync(UB_copy, UB, n_str * pl.P_tot * rsz, cudaMemcpyDeviceToDevice, ctx->stream));
  int ngp = 0;
  if (want_grad) {
    rc = tc ? launch_mlp_bwd_tc(ctx, pl, params, mesh->X, Xe, UB, gpart, &ngp, smax, stash)
            : launch_mlp_bwd(ctx, pl, params, mesh->X, Xe, UB, gpart, &ngp, stash);
    if (rc) return rc;
  }
  cudaEvent_t ta;
  time_begin(ctx, K_FINALIZE, &ta);
  const double tau = bc ? bc->tau : 0.0, gamma = bc ? bc->gamma : 0.0;
  const int fgrid = (want_grad ? (sh.n_params + 31) / 32 : 0) + 1;     // gradient blocks + the loss block
  if (pl.prec == FV_FP64)
    finalize_kernel<double><<<fgrid, 256, 0, ctx->stream>>>(cpart, ncp, bcpart, gpart, ngp, sh.n_params, inv_norm, tau,
                                                            gamma, pl.n_bd, pl.n_s, (double*)grad, out);
  else
    finalize_kernel<float><<<fgrid, 256, 0, ctx->stream>>>(cpart, ncp, bcpart, gpart, ngp, sh.n_params, inv_norm, tau,
                                                           gamma, pl.n_bd, pl.n_s, (float*)grad, out);
  time_end(ctx, K_FINALIZE, ta);
  FV_CUDA_TRY(cudaGetLastError());
  return FV_OK;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" const char* fv_last_error(void) { return fv::g_err; }

extern "C" int fv_ctx_create(fv_ctx* out, int device, void* stream) {
  clear_error();
  FV_CHECK_ARG(out, "fv_ctx_create: null output");
  int n = 0;
  FV_CUDA_TRY(cudaGetDeviceCount(&n));
  FV_CHECK_ARG(device >= 0 && device < n, "fv_ctx_create: device %d out of range (%d devices)", device, n);
  FV_CUDA_TRY(cudaSetDevice(device));
  cudaDeviceProp prop;
  FV_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major < 10) {
    set_error("fv_ctx_create: device %d is sm_%d%d; this library is built for sm_103a", device, prop.major, prop.minor);
    return FV_ERR_UNSUPPORTED;
  }
  fv_ctx c = new fv_ctx_s();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->n_sm = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  c->smem_per_sm = prop.sharedMemPerMultiprocessor;
  cudaError_t e = cudaMalloc(&c->err_dev, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->err_dev, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFree(c->err_dev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    delete c;
    set_error("fv_ctx_create: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  *out = c;
  return FV_OK;
}

extern "C" int fv_ctx_set_stream(fv_ctx ctx, void* stream) {
  clear_error();
  FV_CHECK_ARG(ctx, "fv_ctx_set_stream: null context");
  ctx->stream = static_cast<cudaStream_t>(stream);
  return FV_OK;
}

extern "C" int fv_ctx_destroy(fv_ctx ctx) {
  clear_error();
  if (!ctx) return FV_OK;
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  cudaFree(ctx->ws.ptr);
  cudaFree(ctx->err_dev);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  delete ctx;
  return FV_OK;
}

extern "C" int fv_ctx_set_activation_stash(fv_ctx ctx, int on) {
  clear_error();
  FV_CHECK_ARG(ctx, "fv_ctx_set_activation_stash: null context");
  ctx->tc_stash = on != 0;
  return FV_OK;
}

extern "C" int fv_ctx_enable_timing(fv_ctx ctx, int on) {
  clear_error();
  FV_CHECK_ARG(ctx, "fv_ctx_enable_timing: null context");
  ctx->timing = on != 0;
  return FV_OK;
}

static void drain_times(fv_ctx ctx) {
  for (auto& r : ctx->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->kind_ms[r.kind] += ms;
      ctx->kind_launches[r.kind] += 1;
    }
    ctx->free_events.push_back(r.a);
    ctx->free_events.push_back(r.b);
  }
  ctx->recs.clear();
}

extern "C" int fv_ctx_kernel_times(fv_ctx ctx, int max_kinds, double* ms, int64_t* launches, int* n_kinds) {
  clear_error();
  FV_CHECK_ARG(ctx && ms && launches && n_kinds, "fv_ctx_kernel_times: null argument");
  FV_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  drain_times(ctx);
  const int n = std::min<int>(max_kinds, K_NUM_KINDS);
  for (int i = 0; i < n; ++i) { ms[i] = ctx->kind_ms[i]; launches[i] = ctx->kind_launches[i]; }
  *n_kinds = K_NUM_KINDS;
  return FV_OK;
}

extern "C" int fv_ctx_reset_kernel_times(fv_ctx ctx) {
  clear_error();
  FV_CHECK_ARG(ctx, "fv_ctx_reset_kernel_times: null context");
  FV_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  drain_times(ctx);
  for (int i = 0; i < K_NUM_KINDS; ++i) { ctx->kind_ms[i] = 0; ctx->kind_launches[i] = 0; }
  return FV_OK;
}

extern "C" const char* fv_kernel_name(int kind) {
  static const char* names[K_NUM_KINDS] = {"g_build", "forcing", "mlp_fwd", "contract", "bc_seed", "mlp_bwd",
                                           "finalize", "adam", "mlp_fwd_tc", "mlp_bwd_tc", "batch", "seed_scale"};
  return (kind >= 0 && kind < K_NUM_KINDS) ? names[kind] : "";
}

extern "C" int fv_loss(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                       const void* params, const fv_eval_opts* opts, double* out) {
  clear_error();
  FV_CHECK_ARG(out, "fv_loss: null output");
  if (ctx) FV_CUDA_TRY(cudaSetDevice(ctx->device));
  return evaluate(ctx, mesh, forcing, bc, mlp, params, opts, nullptr, false, nullptr, out);
}

extern "C" int fv_loss_grad(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                            const void* params, const fv_eval_opts* opts, void* grad, double* out) {
  clear_error();
  FV_CHECK_ARG(out && grad, "fv_loss_grad: null output");
  if (ctx) FV_CUDA_TRY(cudaSetDevice(ctx->device));
  return evaluate(ctx, mesh, forcing, bc, mlp, params, opts, nullptr, true, grad, out);
}

// ---------------------------------------------------------------- evaluation without allocation
// Scratch for fv_loss_grad_noalloc: a fixed area in the library's device
// image, present on every device that loads the library, until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FV_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current).
// In host code the array's name only stands in for the symbol, so the
// address is looked up once per device and cached; a device reset
// (cudaDeviceReset) unloads the module and leaves the cached address stale.
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("fv_loss_grad_noalloc: device %d out of range", device);
    return FV_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("fv_loss_grad_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FV_ERR_CUDA;
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return FV_OK;
}
}  // namespace

extern "C" int fv_loss_grad_noalloc(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                                    const void* params, const fv_eval_opts* opts, void* grad, double* out) {
  clear_error();
  FV_CHECK_ARG(ctx && out && grad, "fv_loss_grad_noalloc: null argument");
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  void* scratch = nullptr;
  int rc = noalloc_scratch(ctx->device, &scratch);
  if (rc) return rc;
  return evaluate(ctx, mesh, forcing, bc, mlp, params, opts, nullptr, true, grad, out, nullptr, nullptr, nullptr,
                  scratch, FV_NOALLOC_SCRATCH_BYTES);
}

extern "C" int fv_eval_intermediates(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                                     const void* params, const fv_eval_opts* opts, void* U_dev, void* UB_dev,
                                     double* R_dev, double* out_dev) {
  clear_error();
  FV_CHECK_ARG(out_dev, "fv_eval_intermediates: null output");
  if (ctx) FV_CUDA_TRY(cudaSetDevice(ctx->device));
  // the gradient goes to the workspace-backed scratch of a throw-away buffer
  MlpShape sh;
  if (!make_shape(mlp, &sh)) { set_error("fv_eval_intermediates: unsupported network shape"); return FV_ERR_UNSUPPORTED; }
  void* g = nullptr;
  FV_CUDA_TRY(cudaMalloc(&g, (size_t)sh.n_params * 8));
  int rc = evaluate(ctx, mesh, forcing, bc, mlp, params, opts, nullptr, true, g, out_dev, U_dev, UB_dev, R_dev);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cudaFree(g);
  if (rc) return rc;
  if (e != cudaSuccess) { set_error("fv_eval_intermediates: %s", cudaGetErrorString(e)); return FV_ERR_CUDA; }
  return FV_OK;
}

extern "C" int fv_mlp_eval(fv_ctx ctx, const fv_mlp_desc* mlp, const void* params, fv_precision prec, int n,
                           const double* xy, void* out) {
  clear_error();
  FV_CHECK_ARG(ctx && mlp && params && xy && out && n >= 0, "fv_mlp_eval: bad argument");
  MlpShape sh;
  if (!make_shape(mlp, &sh)) { set_error("fv_mlp_eval: unsupported network shape"); return FV_ERR_UNSUPPORTED; }
  if (prec != FV_FP64 && prec != FV_FP32) { set_error("fv_mlp_eval: FP64 or FP32 only"); return FV_ERR_UNSUPPORTED; }
  if (n == 0) return FV_OK;
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  EvalPlan pl;
  pl.shape = sh; pl.prec = prec; pl.P_mesh = n; pl.P_tot = n;
  return launch_mlp_fwd(ctx, pl, params, xy, nullptr, out);
}

extern "C" int fv_adam_create(fv_ctx ctx, int64_t n, fv_precision prec, double b1, double b2, double ae, int with_eps,
                              fv_adam* out) {
  clear_error();
  FV_CHECK_ARG(ctx && out && n > 0, "fv_adam_create: bad argument");
  FV_CHECK_ARG(prec == FV_FP64 || prec == FV_FP32 || prec == FV_TF32 || prec == FV_BF16 || prec == FV_FP16,
               "fv_adam_create: precision");
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  fv_adam a = new fv_adam_s();
  a->ctx = ctx; a->n = n; a->prec = prec == FV_FP64 ? FV_FP64 : FV_FP32;
  a->beta1 = b1; a->beta2 = b2; a->eps = ae; a->with_eps = with_eps;
  const size_t es = a->prec == FV_FP64 ? 8 : 4;
  cudaError_t e;
  if ((e = cudaMalloc(&a->m, es * n)) || (e = cudaMalloc(&a->v, es * n)) || (e = cudaMalloc(&a->me, 16)) ||
      (e = cudaMalloc(&a->t, sizeof(int))) || (e = cudaMemsetAsync(a->m, 0, es * n, ctx->stream)) ||
      (e = cudaMemsetAsync(a->v, 0, es * n, ctx->stream)) || (e = cudaMemsetAsync(a->me, 0, 16, ctx->stream)) ||
      (e = cudaMemsetAsync(a->t, 0, sizeof(int), ctx->stream)) || (e = cudaStreamSynchronize(ctx->stream))) {
    cudaFree(a->m); cudaFree(a->v); cudaFree(a->me); cudaFree(a->t);
    delete a;
    set_error("fv_adam_create: %s", cudaGetErrorString(e));
    return FV_ERR_OOM;
  }
  *out = a;
  return FV_OK;
}

extern "C" int fv_adam_destroy(fv_adam a) {
  clear_error();
  if (!a) return FV_OK;
  cudaFree(a->m); cudaFree(a->v); cudaFree(a->me); cudaFree(a->t);
  delete a;
  return FV_OK;
}

namespace fv {
// One Adam update of (theta, eps) on the context's stream (Sec. 4.5: Adam).
int launch_adam(fv_ctx ctx, fv_adam adam, void* params, const void* grad, double* eps_dev, double* out, double lr) {
  cudaEvent_t ta;
  time_begin(ctx, K_ADAM, &ta);
  if (adam->prec == FV_FP64)
    adam_kernel<double><<<1, 1024, 0, ctx->stream>>>((double*)params, (const double*)grad, adam->n, (double*)adam->m,
                                                     (double*)adam->v, eps_dev, out + 4, adam->me, adam->with_eps,
                                                     adam->t, lr, adam->beta1, adam->beta2, adam->eps);
  else
    adam_kernel<float><<<1, 1024, 0, ctx->stream>>>((float*)params, (const float*)grad, adam->n, (float*)adam->m,
                                                    (float*)adam->v, eps_dev, out + 4, adam->me, adam->with_eps,
                                                    adam->t, lr, adam->beta1, adam->beta2, adam->eps);
  time_end(ctx, K_ADAM, ta);
  FV_CUDA_TRY(cudaGetLastError());
  return FV_OK;
}
}  // namespace fv

extern "C" int fv_inverse_step(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                               void* params, double* eps_dev, const fv_eval_opts* opts, fv_adam adam, double lr,
                               void* grad, double* out) {
  clear_error();
  FV_CHECK_ARG(eps_dev && grad && out, "fv_inverse_step: null argument");
  FV_CHECK_ARG(lr <= 0.0 || adam, "fv_inverse_step: an Adam state is needed when lr > 0");
  if (ctx) FV_CUDA_TRY(cudaSetDevice(ctx->device));
  int rc = evaluate(ctx, mesh, forcing, bc, mlp, params, opts, eps_dev, true, grad, out);
  if (rc || lr <= 0.0) return rc;
  MlpShape sh;
  make_shape(mlp, &sh);
  FV_CHECK_ARG(adam->n == sh.n_params && adam->ctx == ctx, "fv_inverse_step: Adam state does not match");
  FV_CHECK_ARG((adam->prec == FV_FP64) == (opts->mlp_precision == FV_FP64), "fv_inverse_step: Adam precision");
  return launch_adam(ctx, adam, params, grad, eps_dev, out, lr);
}

// ---------------------------------------------------------------- captured training steps
// n_steps consecutive inverse steps (loss + gradient + Adam) captured once
// into a CUDA graph; a launch replays them with one host call.  The graph
// owns a workspace sized before capture, so nothing allocates inside it.
struct fv_graph_s {
  fv_ctx ctx = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* ws = nullptr;
  int n_steps = 0;
};

static void graph_release(fv_graph g) {
  if (!g) return;
  if (g->ctx) cudaStreamSynchronize(g->ctx->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->capture) cudaStreamDestroy(g->capture);
  if (g->ws) cudaFree(g->ws);
  delete g;
}

extern "C" int fv_step_graph_create(fv_ctx ctx, fv_mesh mesh, fv_forcing forcing, fv_bc bc, const fv_mlp_desc* mlp,
                                    void* params, double* eps_dev, const fv_eval_opts* opts, fv_adam adam, double lr,
                                    void* grad, double* out, int n_steps, fv_graph* out_graph) {
  clear_error();
  FV_CHECK_ARG(ctx && mesh && forcing && mlp && params && eps_dev && opts && grad && out && out_graph,
               "fv_step_graph_create: null argument");
  FV_CHECK_ARG(n_steps >= 1 && n_steps <= 100000, "fv_step_graph_create: n_steps %d outside 1..100000", n_steps);
  FV_CHECK_ARG(lr <= 0.0 || adam, "fv_step_graph_create: an Adam state is needed when lr > 0");
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  size_t need = 0;
  int rc = evaluate(ctx, mesh, forcing, bc, mlp, params, opts, eps_dev, true, grad, out, nullptr, nullptr, nullptr,
                    nullptr, 0, &need);
  if (rc) return rc;
  if (lr > 0.0) {
    MlpShape sh;
    make_shape(mlp, &sh);
    FV_CHECK_ARG(adam->n == sh.n_params && adam->ctx == ctx, "fv_step_graph_create: Adam state does not match");
    FV_CHECK_ARG((adam->prec == FV_FP64) == (opts->mlp_precision == FV_FP64), "fv_step_graph_create: Adam precision");
  }
  fv_graph g = new fv_graph_s();
  g->ctx = ctx;
  g->n_steps = n_steps;
  auto fail = [&](int code) { graph_release(g); return code; };
  cudaError_t e = cudaMalloc(&g->ws, std::max<size_t>(need, 256));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("fv_step_graph_create: %s", cudaGetErrorString(e));
    return fail(e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA);
  }
  fv_ctx_s cap_ctx;                           // same device, the capture stream, no timing
  cap_ctx.device = ctx->device;
  cap_ctx.stream = g->capture;
  cap_ctx.n_sm = ctx->n_sm;
  cap_ctx.smem_optin = ctx->smem_optin;
  cap_ctx.smem_per_sm = ctx->smem_per_sm;
  cap_ctx.tc_stash = ctx->tc_stash;
  cap_ctx.err_dev = ctx->err_dev;
  fv_mesh_s mesh_copy = *mesh;
  mesh_copy.ctx = &cap_ctx;
  fv_forcing_s forcing_copy = *forcing;
  forcing_copy.mesh = &mesh_copy;
  fv_bc_s bc_copy;
  if (bc) { bc_copy = *bc; bc_copy.ctx = &cap_ctx; }
  fv_adam_s adam_copy;
  if (adam) { adam_copy = *adam; adam_copy.ctx = &cap_ctx; }
  e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    set_error("fv_step_graph_create: capture failed to start (%s)", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  for (int k = 0; k < n_steps && rc == FV_OK; ++k) {
    rc = evaluate(&cap_ctx, &mesh_copy, &forcing_copy, bc ? &bc_copy : nullptr, mlp, params, opts, eps_dev, true, grad,
                  out, nullptr, nullptr, nullptr, g->ws, std::max<size_t>(need, 256));
    if (rc == FV_OK && lr > 0.0) rc = launch_adam(&cap_ctx, &adam_copy, params, grad, eps_dev, out, lr);
  }
  cap_ctx.ws.ptr = nullptr;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->capture, &graph);
  g->graph = graph;
  if (rc) return fail(rc);
  if (e != cudaSuccess) {
    set_error("fv_step_graph_create: capture failed (%s)", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    set_error("fv_step_graph_create: instantiation failed (%s)", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  *out_graph = g;
  return FV_OK;
}

extern "C" int fv_graph_launch(fv_graph g) {
  clear_error();
  FV_CHECK_ARG(g && g->exec, "fv_graph_launch: null graph");
  FV_CUDA_TRY(cudaSetDevice(g->ctx->device));
  FV_CUDA_TRY(cudaGraphLaunch(g->exec, g->ctx->stream));
  return FV_OK;
}

extern "C" int fv_graph_destroy(fv_graph g) {
  clear_error();
  graph_release(g);
  return FV_OK;
}

// ---------------------------------------------------------------- batches
// A batch of independent problems (one network shape and options) is
// captured once into a CUDA graph: the instances' evaluations are spread
// over n_streams forked capture streams (largest first, each on the least
// loaded stream) so that small instances run side by side, and every
// instance has its own workspace.  fv_batch_loss_grad is one graph launch.
struct fv_batch_s {
  fv_ctx ctx = nullptr;
  std::vector<fv_instance> inst;
  fv_mlp_desc mlp{};
  std::vector<int> widths;
  fv_eval_opts opts{};
  std::vector<void*> ws;
  std::vector<size_t> ws_bytes;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n_streams = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaStream_t capture = nullptr;   // capture origin (the context's stream may be the legacy default stream)
  double tuned_ms[8] = {0};
};

namespace {

void batch_free_graph(fv_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Capture all instances on S streams into b->graph / b->exec.
int batch_capture(fv_batch b, int S) {
  batch_free_graph(b);
  fv_ctx ctx = b->ctx;
  while ((int)b->streams.size() < S) {
    cudaStream_t st;
    FV_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->streams.push_back(st);
  }
  while ((int)b->events.size() < S + 1) {
    cudaEvent_t ev;
    FV_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->events.push_back(ev);
  }
  // largest instances first, each onto the least loaded stream
  std::vector<int> order(b->inst.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(),
            [&](int x, int y) { return b->inst[x].mesh->P > b->inst[y].mesh->P; });
  std::vector<int64_t> load(S, 0);
  std::vector<int> lane_of(b->inst.size(), 0);
  for (int i : order) {
    int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane_of[i] = s;
    load[s] += b->inst[i].mesh->P;
  }
  if (!b->capture) FV_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  cudaStream_t main = b->capture;
  FV_CUDA_TRY(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
  int rc = FV_OK;
  cudaError_t e = cudaEventRecord(b->events[S], main);
  for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->streams[s], b->events[S], 0);
  if (e != cudaSuccess) {
    set_error("batch capture fork failed: %s", cudaGetErrorString(e));
    rc = FV_ERR_CUDA;
  }
  for (int i : order) {
    if (rc) break;
    fv_ctx_s lane_ctx;                         // same device, the lane's stream, no timing
    lane_ctx.device = ctx->device;
    lane_ctx.stream = b->streams[lane_of[i]];
    lane_ctx.n_sm = ctx->n_sm;
    lane_ctx.tc_ctas_cap = S > 1 ? 1 : ctx->tc_ctas_cap;   // leave SM room for the other streams' kernels
    lane_ctx.smem_optin = ctx->smem_optin;
    lane_ctx.smem_per_sm = ctx->smem_per_sm;
    lane_ctx.tc_stash = ctx->tc_stash;
    lane_ctx.err_dev = ctx->err_dev;
    const fv_instance& in = b->inst[i];
    // the handles were created on ctx; evaluate them on the lane context
    fv_mesh_s mesh_copy = *in.mesh;
    mesh_copy.ctx = &lane_ctx;
    fv_forcing_s forcing_copy = *in.forcing;
    forcing_copy.mesh = &mesh_copy;
    fv_bc_s bc_copy;
    if (in.bc) { bc_copy = *in.bc; bc_copy.ctx = &lane_ctx; }
    rc = evaluate(&lane_ctx, &mesh_copy, &forcing_copy, in.bc ? &bc_copy : nullptr, &b->mlp, in.params_dev, &b->opts,
                  nullptr, true, in.grad_dev, in.out_dev, nullptr, nullptr, nullptr, b->ws[i], b->ws_bytes[i]);
    lane_ctx.ws.ptr = nullptr;
  }
  for (int s = 0; s < S && rc == FV_OK; ++s) {
    e = cudaEventRecord(b->events[s], b->streams[s]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, b->events[s], 0);
    if (e != cudaSuccess) {
      set_error("batch capture join failed: %s", cudaGetErrorString(e));
      rc = FV_ERR_CUDA;
    }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(main, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) {
    set_error("batch capture failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    set_error("batch graph instantiation failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  b->n_streams = S;
  return FV_OK;
}

}  // namespace

void batch_release(fv_batch b) {   // frees without touching the error message
  if (!b) return;
  if (b->ctx) cudaStreamSynchronize(b->ctx->stream);
  batch_free_graph(b);
  for (auto p : b->ws) cudaFree(p);
  for (auto st : b->streams) cudaStreamDestroy(st);
  for (auto ev : b->events) cudaEventDestroy(ev);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

extern "C" int fv_batch_plan(fv_ctx ctx, int n, const fv_instance* inst, const fv_mlp_desc* mlp,
                             const fv_eval_opts* opts, int n_streams, fv_batch* out) {
  clear_error();
  FV_CHECK_ARG(ctx && inst && mlp && opts && out && n >= 1, "fv_batch_plan: bad argument");
  FV_CHECK_ARG(n_streams >= 0 && n_streams <= 8, "fv_batch_plan: n_streams must be 0 (tune) .. 8");
  FV_CHECK_ARG(!opts->eps_dev, "fv_batch_plan: a device eps is not supported in batches");
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  MlpShape sh;
  for (int i = 0; i < n; ++i) {
    int rc = check_eval(ctx, inst[i].mesh, inst[i].forcing, inst[i].bc, mlp, inst[i].params_dev, opts, &sh);
    if (rc) return rc;
    FV_CHECK_ARG(inst[i].grad_dev && inst[i].out_dev, "fv_batch_plan: instance %d has no outputs", i);
  }
  fv_batch b = new fv_batch_s();
  b->ctx = ctx;
  b->inst.assign(inst, inst + n);
  b->widths.assign(mlp->widths, mlp->widths + mlp->n_layers + 1);
  b->mlp.n_layers = mlp->n_layers;
  b->mlp.widths = b->widths.data();
  b->opts = *opts;
  auto fail = [&](int rc) { batch_release(b); return rc; };
  for (int i = 0; i < n; ++i) {
    size_t bytes = 0;
    int rc = evaluate(ctx, inst[i].mesh, inst[i].forcing, inst[i].bc, &b->mlp, inst[i].params_dev, &b->opts, nullptr,
                      true, inst[i].grad_dev, inst[i].out_dev, nullptr, nullptr, nullptr, nullptr, 0, &bytes);
    if (rc) return fail(rc);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      set_error("fv_batch_plan: workspace allocation failed: %s", cudaGetErrorString(e));
      return fail(FV_ERR_OOM);
    }
    b->ws.push_back(p);
    b->ws_bytes.push_back(bytes);
  }
  if (n_streams > 0) {
    int rc = batch_capture(b, n_streams);
    if (rc) return fail(rc);
  } else {
    // tune: capture with 1, 2, 4, 8 streams and keep the fastest replay
    int best = 1;
    float best_ms = 1e30f;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    for (int S = 1; S <= 8; S *= 2) {
      int rc = batch_capture(b, S);
      if (rc) { cudaEventDestroy(t0); cudaEventDestroy(t1); return fail(rc); }
      cudaGraphLaunch(b->exec, ctx->stream);          // warm-up
      cudaEventRecord(t0, ctx->stream);
      for (int r = 0; r < 3; ++r) cudaGraphLaunch(b->exec, ctx->stream);
      cudaEventRecord(t1, ctx->stream);
      cudaError_t e = cudaEventSynchronize(t1);
      float ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
      if (e != cudaSuccess) {
        set_error("fv_batch_plan: tuning run failed: %s", cudaGetErrorString(e));
        cudaEventDestroy(t0); cudaEventDestroy(t1);
        return fail(FV_ERR_CUDA);
      }
      int k = 0;
      for (int t = S; t > 1; t >>= 1) ++k;
      b->tuned_ms[k] = ms / 3;
      if (ms < best_ms) { best_ms = ms; best = S; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (best != b->n_streams) {
      int rc = batch_capture(b, best);
      if (rc) return fail(rc);
    }
  }
  *out = b;
  return FV_OK;
}

extern "C" int fv_batch_loss_grad(fv_batch b) {
  clear_error();
  FV_CHECK_ARG(b && b->exec, "fv_batch_loss_grad: batch not planned");
  FV_CUDA_TRY(cudaSetDevice(b->ctx->device));
  FV_CUDA_TRY(cudaGraphLaunch(b->exec, b->ctx->stream));
  return FV_OK;
}

extern "C" int fv_batch_info(fv_batch b, int* n_streams, double* tuned_ms /* [4]: 1, 2, 4, 8 streams */) {
  clear_error();
  FV_CHECK_ARG(b, "fv_batch_info: null batch");
  if (n_streams) *n_streams = b->n_streams;
  if (tuned_ms) for (int k = 0; k < 4; ++k) tuned_ms[k] = b->tuned_ms[k];
  return FV_OK;
}

extern "C" int fv_batch_destroy(fv_batch b) {
  clear_error();
  batch_release(b);
  return FV_OK;
}

