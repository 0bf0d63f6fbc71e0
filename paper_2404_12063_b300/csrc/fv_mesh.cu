// Mesh tensors: reference-element tables, the stacked premultiplier tensor G
// (Algorithm 3, Sec. 4.4; bilinear map of App. A.1; assembly of App. A.2),
// the mapped quadrature points, the forcing matrix F, and boundary data.
#include <cmath>
#include <cstring>

#include "fv_internal.cuh"

namespace fv {
namespace {

// Legendre P_n(x) by the three-term recurrence; also returns P_{n-1}.
void leg(int n, double x, double* Pn, double* Pnm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) { *Pn = 1.0; *Pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b; b = c;
  }
  *Pn = b; *Pnm1 = a;
}

double legP(int n, double x) { double p, q; leg(n, x, &p, &q); return p; }

// Gauss-Lobatto-Legendre nodes: +-1 and the zeros of q(x) = P_{N+1} - P_{N-1}
// inside (-1, 1) (which are the zeros of P_N'), N = Q-1, by Newton's method
// with q'(x) = (2N+1) P_N(x).  Weights 2 / (N (N+1) P_N(x)^2).
void gll_nodes(int Q, double* x, double* w) {
  const int N = Q - 1;
  for (int i = 0; i <= N; ++i) {
    double t = -std::cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 200; ++it) {
        double q = legP(N + 1, t) - legP(N - 1, t);
        double dq = (2.0 * N + 1.0) * legP(N, t);
        double dt = q / dq;
        t -= dt;
        if (std::fabs(dt) <= 1e-16 * (1.0 + std::fabs(t))) break;
      }
    }
    x[i] = t;
  }
  // symmetrise (the rule is symmetric about 0)
  for (int i = 0; i < Q / 2; ++i) {
    double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s; x[N - i] = s;
  }
  if (Q % 2) x[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double p = legP(N, x[i]);
    w[i] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

// Reference tables: xi[Q], w[Q], v[T][Q], dv[T][Q] with v_m = P_{m+1} - P_{m-1}
// and v_m' = (2m+1) P_m  (Sec. 4.5 test functions).
void make_tables(int Q, int T, std::vector<double>& tab) {
  tab.assign(2 * Q + 2 * T * Q, 0.0);
  double* xi = tab.data();
  double* w = xi + Q;
  double* v = w + Q;
  double* dv = v + T * Q;
  gll_nodes(Q, xi, w);
  for (int m = 1; m <= T; ++m)
    for (int a = 0; a < Q; ++a) {
      v[(m - 1) * Q + a] = legP(m + 1, xi[a]) - legP(m - 1, xi[a]);
      dv[(m - 1) * Q + a] = (2.0 * m + 1.0) * legP(m, xi[a]);
    }
}

template <class Gt> __device__ __forceinline__ Gt cvt_g(double v);
template <> __device__ __forceinline__ double cvt_g<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt_g<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_g<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// One CTA per element (grid-stride).  FP64 throughout; the adjugate form
// w (y_eta v_xi - y_xi v_eta) = w |J| dv/dx needs no division by |J|.
template <class Gt>
__global__ void g_build_kernel(const double* __restrict__ verts, const int* __restrict__ cells, int n_e, int Q,
                               int T, const double* __restrict__ tab, int n_comp, Gt* __restrict__ G,
                               int64_t stride, double* __restrict__ X, int* __restrict__ bad_elem) {
  __shared__ double s_tab[2 * kMaxQ + 2 * kMaxT * kMaxQ];
  __shared__ Bilin s_c;
  const int Nq = Q * Q, Nt = T * T;
  for (int i = threadIdx.x; i < 2 * Q + 2 * T * Q; i += blockDim.x) s_tab[i] = tab[i];
  const double* xi = s_tab;
  const double* w = xi + Q;
  const double* v = w + Q;
  const double* dv = v + T * Q;
  for (int e = blockIdx.x; e < n_e; e += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) s_c = bilin_coeffs(verts, cells + 4 * (size_t)e);
    __syncthreads();
    const Bilin c = s_c;
    Gt* Ge = G + (size_t)e * stride;
    for (int idx = threadIdx.x; idx < Nt * Nq; idx += blockDim.x) {
      const int j = idx / Nq, q = idx - j * Nq;
      const int a = q / Q, b = q - a * Q;
      const int m = j / T, n = j - m * T;
      const double s = xi[a], t = xi[b];
      const double x_xi = c.x1 + c.x3 * t, x_eta = c.x2 + c.x3 * s;
      const double y_xi = c.y1 + c.y3 * t, y_eta = c.y2 + c.y3 * s;
      const double D = x_xi * y_eta - x_eta * y_xi;
      const double vm = v[m * Q + a], dvm = dv[m * Q + a], vn = v[n * Q + b], dvn = dv[n * Q + b];
      const double wq = w[a] * w[b];
      const double v_xi = dvm * vn, v_eta = vm * dvn;
      Ge[(size_t)j * Nq + q] = cvt_g<Gt>(wq * (y_eta * v_xi - y_xi * v_eta));
      Ge[(size_t)(Nt + j) * Nq + q] = cvt_g<Gt>(wq * (x_xi * v_eta - x_eta * v_xi));
      if (n_comp == 3) Ge[(size_t)(2 * Nt + j) * Nq + q] = cvt_g<Gt>(wq * D * vm * vn);
      if (j == 0) {
        X[((size_t)e * Nq + q) * 2] = c.x0 + c.x1 * s + c.x2 * t + c.x3 * s * t;
        X[((size_t)e * Nq + q) * 2 + 1] = c.y0 + c.y1 * s + c.y2 * t + c.y3 * s * t;
        if (!(D > 0.0)) atomicMin(bad_elem, e);
      }
    }
    for (int idx = n_comp * Nt * Nq + threadIdx.x; idx < stride; idx += blockDim.x) Ge[idx] = cvt_g<Gt>(0.0);
  }
}

// F[e][j] = sum_q w_q |J|_q v_j(q) f_q in FP64 (App. A.2).
__global__ void forcing_kernel(const double* __restrict__ verts, const int* __restrict__ cells, int n_e, int Q, int T,
                               const double* __restrict__ tab, const double* __restrict__ f, double* __restrict__ F) {
  __shared__ double s_tab[2 * kMaxQ + 2 * kMaxT * kMaxQ];
  __shared__ double s_wDf[kMaxQ * kMaxQ];
  const int Nq = Q * Q, Nt = T * T;
  for (int i = threadIdx.x; i < 2 * Q + 2 * T * Q; i += blockDim.x) s_tab[i] = tab[i];
  const double* xi = s_tab;
  const double* w = xi + Q;
  const double* v = w + Q;
  for (int e = blockIdx.x; e < n_e; e += gridDim.x) {
    __syncthreads();
    const Bilin c = bilin_coeffs(verts, cells + 4 * (size_t)e);
    for (int q = threadIdx.x; q < Nq; q += blockDim.x) {
      const int a = q / Q, b = q - a * Q;
      const double s = xi[a], t = xi[b];
      const double D = (c.x1 + c.x3 * t) * (c.y2 + c.y3 * s) - (c.x2 + c.x3 * s) * (c.y1 + c.y3 * t);
      s_wDf[q] = w[a] * w[b] * D * f[(size_t)e * Nq + q];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < Nt; j += blockDim.x) {
      const int m = j / T, n = j - m * T;
      double acc = 0.0;
      for (int a = 0; a < Q; ++a) {
        double inner = 0.0;
        for (int b = 0; b < Q; ++b) inner += s_wDf[a * Q + b] * v[n * Q + b];
        acc += v[m * Q + a] * inner;
      }
      F[(size_t)e * Nt + j] = acc;
    }
  }
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

template <class Gt>
__global__ void g_to_double_kernel(const Gt* __restrict__ G, int64_t stride, int n_e, int64_t per_elem,
                                   double* __restrict__ out) {
  const int64_t total = (int64_t)n_e * per_elem;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / per_elem, r = i - e * per_elem;
    out[i] = to_d(G[e * stride + r]);
  }
}

size_t storage_bytes(fv_precision p) {
  return p == FV_FP64 ? 8 : (p == FV_FP32 ? 4 : 2);
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" int fv_build_mesh_tensors(fv_ctx ctx, int n_vertices, const double* vertices, int n_elements,
                                     const int32_t* cells, int quad_order, int test_order, fv_precision g_storage,
                                     int with_mass_term, fv_mesh* out) {
  clear_error();
  FV_CHECK_ARG(ctx && out && vertices && cells, "fv_build_mesh_tensors: null argument");
  FV_CHECK_ARG(n_vertices >= 3 && n_elements >= 1, "fv_build_mesh_tensors: need >= 3 vertices and >= 1 element");
  if (quad_order < 2 || quad_order > kMaxQ || test_order < 1 || test_order > kMaxT) {
    set_error("fv_build_mesh_tensors: quad_order must be in [2,%d] and test_order in [1,%d]", kMaxQ, kMaxT);
    return FV_ERR_UNSUPPORTED;
  }
  if (g_storage != FV_FP64 && g_storage != FV_FP32 && g_storage != FV_BF16) {
    set_error("fv_build_mesh_tensors: G storage must be FV_FP64, FV_FP32 or FV_BF16");
    return FV_ERR_UNSUPPORTED;
  }
  for (int64_t i = 0; i < 4LL * n_elements; ++i)
    FV_CHECK_ARG(cells[i] >= 0 && cells[i] < n_vertices, "fv_build_mesh_tensors: cell %lld references vertex %d",
                 (long long)(i / 4), cells[i]);
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  fv_mesh m = new fv_mesh_s();
  m->ctx = ctx;
  m->n_e = n_elements; m->Q = quad_order; m->T = test_order;
  m->Nq = quad_order * quad_order; m->Nt = test_order * test_order;
  m->n_comp = with_mass_term ? 3 : 2;
  m->P = (int64_t)n_elements * m->Nq;
  m->storage = g_storage;
  m->n_v = n_vertices;
  const size_t es = storage_bytes(g_storage);
  m->g_elem_bytes = (size_t)m->n_comp * m->Nt * m->Nq * es;
  m->g_stride_bytes = (m->g_elem_bytes + 15) / 16 * 16;
  std::vector<double> tab;
  make_tables(m->Q, m->T, tab);
  auto fail = [&](int rc) {   // frees without touching the error message
    cudaFree(m->G); cudaFree(m->X); cudaFree(m->tables); cudaFree(m->verts); cudaFree(m->cells);
    delete m;
    return rc;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&m->G, m->g_stride_bytes * n_elements)) != cudaSuccess ||
      (e = cudaMalloc(&m->X, sizeof(double) * 2 * m->P)) != cudaSuccess ||
      (e = cudaMalloc(&m->tables, sizeof(double) * tab.size())) != cudaSuccess ||
      (e = cudaMalloc(&m->verts, sizeof(double) * 2 * n_vertices)) != cudaSuccess ||
      (e = cudaMalloc(&m->cells, sizeof(int) * 4 * n_elements)) != cudaSuccess) {
    set_error("fv_build_mesh_tensors: cudaMalloc failed (%s)", cudaGetErrorString(e));
    return fail(e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA);
  }
  cudaStream_t st = ctx->stream;
  if ((e = cudaMemcpyAsync(m->tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(m->verts, vertices, sizeof(double) * 2 * n_vertices, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(m->cells, cells, sizeof(int) * 4 * n_elements, cudaMemcpyHostToDevice, st))) {
    set_error("fv_build_mesh_tensors: copy failed (%s)", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  int big = 0x7fffffff;
  if ((e = cudaMemcpyAsync(ctx->err_dev, &big, sizeof(int), cudaMemcpyHostToDevice, st))) {
    set_error("fv_build_mesh_tensors: %s", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  const int grid = (int)std::min<int64_t>(n_elements, (int64_t)ctx->n_sm * 8);
  cudaEvent_t ta;
  time_begin(ctx, K_G_BUILD, &ta);
  if (g_storage == FV_FP64)
    g_build_kernel<double><<<grid, 256, 0, st>>>(m->verts, m->cells, n_elements, m->Q, m->T, m->tables, m->n_comp,
                                                  (double*)m->G, m->g_stride_bytes / 8, m->X, ctx->err_dev);
  else if (g_storage == FV_FP32)
    g_build_kernel<float><<<grid, 256, 0, st>>>(m->verts, m->cells, n_elements, m->Q, m->T, m->tables, m->n_comp,
                                                 (float*)m->G, m->g_stride_bytes / 4, m->X, ctx->err_dev);
  else
    g_build_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(m->verts, m->cells, n_elements, m->Q, m->T, m->tables,
                                                         m->n_comp, (__nv_bfloat16*)m->G, m->g_stride_bytes / 2, m->X,
                                                         ctx->err_dev);
  time_end(ctx, K_G_BUILD, ta);
  int bad = 0;
  if ((e = cudaGetLastError()) || (e = cudaMemcpyAsync(&bad, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st))) {
    set_error("fv_build_mesh_tensors: kernel failed (%s)", cudaGetErrorString(e));
    return fail(FV_ERR_CUDA);
  }
  if (bad != 0x7fffffff) {
    set_error("fv_build_mesh_tensors: element %d has a non-positive Jacobian determinant at a quadrature node "
              "(vertices must be counter-clockwise and the cell convex)", bad);
    return fail(FV_ERR_DEGENERATE_ELEMENT);
  }
  *out = m;
  return FV_OK;
}

extern "C" int fv_mesh_info(fv_mesh m, int64_t* info) {
  clear_error();
  FV_CHECK_ARG(m && info, "fv_mesh_info: null argument");
  info[0] = m->n_e; info[1] = m->Nq; info[2] = m->Nt; info[3] = m->P; info[4] = m->n_comp;
  info[5] = (int64_t)(m->g_stride_bytes * m->n_e);
  info[6] = (int64_t)(m->g_elem_bytes * m->n_e);
  info[7] = m->storage;
  return FV_OK;
}

extern "C" int fv_mesh_quad_points(fv_mesh m, double* xy) {
  clear_error();
  FV_CHECK_ARG(m && xy, "fv_mesh_quad_points: null argument");
  FV_CUDA_TRY(cudaMemcpyAsync(xy, m->X, sizeof(double) * 2 * m->P, cudaMemcpyDeviceToHost, m->ctx->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(m->ctx->stream));
  return FV_OK;
}

extern "C" int fv_mesh_copy_g(fv_mesh m, double* g_host) {
  clear_error();
  FV_CHECK_ARG(m && g_host, "fv_mesh_copy_g: null argument");
  const int64_t per = (int64_t)m->n_comp * m->Nt * m->Nq;
  double* tmp = nullptr;
  FV_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * per * m->n_e));
  cudaStream_t st = m->ctx->stream;
  const int grid = m->ctx->n_sm * 4;
  if (m->storage == FV_FP64)
    g_to_double_kernel<double><<<grid, 256, 0, st>>>((const double*)m->G, m->g_stride_bytes / 8, m->n_e, per, tmp);
  else if (m->storage == FV_FP32)
    g_to_double_kernel<float><<<grid, 256, 0, st>>>((const float*)m->G, m->g_stride_bytes / 4, m->n_e, per, tmp);
  else
    g_to_double_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)m->G, m->g_stride_bytes / 2,
                                                            m->n_e, per, tmp);
  cudaError_t e = cudaMemcpyAsync(g_host, tmp, sizeof(double) * per * m->n_e, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) { set_error("fv_mesh_copy_g: %s", cudaGetErrorString(e)); return FV_ERR_CUDA; }
  return FV_OK;
}

extern "C" int fv_mesh_destroy(fv_mesh m) {
  clear_error();
  if (!m) return FV_OK;
  cudaFree(m->G); cudaFree(m->X); cudaFree(m->tables); cudaFree(m->verts); cudaFree(m->cells); cudaFree(m->jreg);
  cudaFree(m->reg_ref[0]); cudaFree(m->reg_ref[1]);
  delete m;
  return FV_OK;
}

extern "C" int fv_mesh_set_g_mode(fv_mesh m, int mode) {
  clear_error();
  FV_CHECK_ARG(m, "fv_mesh_set_g_mode: null mesh");
  FV_CHECK_ARG(mode == FV_G_STORED || mode == FV_G_MATRIX_FREE || mode == FV_G_REGULAR,
               "fv_mesh_set_g_mode: mode %d is not 0, 1 or 2", mode);
  if (mode == FV_G_REGULAR) {
    FV_CUDA_TRY(cudaSetDevice(m->ctx->device));
    std::vector<float> scales;
    const int rc = check_regular_mesh(m, &scales);
    if (rc) return rc;
    if (!m->jreg) FV_CUDA_TRY(cudaMalloc(&m->jreg, sizeof(float) * 3 * (size_t)m->n_e));
    FV_CUDA_TRY(cudaMemcpy(m->jreg, scales.data(), sizeof(float) * scales.size(), cudaMemcpyHostToDevice));
    const int rb = build_regular_reference(m);
    if (rb) return rb;
  }
  m->g_mode = mode;
  return FV_OK;
}

extern "C" int fv_autotune(fv_ctx ctx, fv_mesh m, fv_precision prec, double* ms_out) {
  clear_error();
  FV_CHECK_ARG(ctx && m, "fv_autotune: null context or mesh");
  FV_CHECK_ARG(prec >= FV_FP64 && prec <= FV_FP16, "fv_autotune: precision %d out of range", (int)prec);
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  return autotune_contract(ctx, m, prec, ms_out);
}

extern "C" int fv_assemble_forcing(fv_mesh m, const double* f, fv_forcing* out) {
  clear_error();
  FV_CHECK_ARG(m && f && out, "fv_assemble_forcing: null argument");
  fv_ctx ctx = m->ctx;
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  double* fd = nullptr;
  fv_forcing fo = new fv_forcing_s();
  fo->mesh = m;
  cudaError_t e;
  if ((e = cudaMalloc(&fo->F, sizeof(double) * m->n_e * m->Nt)) ||
      (e = cudaMalloc(&fo->F32, sizeof(float) * m->n_e * m->Nt)) || (e = cudaMalloc(&fd, sizeof(double) * m->P))) {
    cudaFree(fo->F); cudaFree(fo->F32); cudaFree(fd); delete fo;
    set_error("fv_assemble_forcing: cudaMalloc failed (%s)", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
  }
  cudaStream_t st = ctx->stream;
  e = cudaMemcpyAsync(fd, f, sizeof(double) * m->P, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    cudaEvent_t ta;
    time_begin(ctx, K_FORCING, &ta);
    forcing_kernel<<<(int)std::min<int64_t>(m->n_e, ctx->n_sm * 8), 128, 0, st>>>(m->verts, m->cells, m->n_e, m->Q,
                                                                                  m->T, m->tables, fd, fo->F);
    to_float_kernel<<<ctx->n_sm, 256, 0, st>>>(fo->F, fo->F32, (int64_t)m->n_e * m->Nt);
    time_end(ctx, K_FORCING, ta);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(fd);
  if (e != cudaSuccess) {
    cudaFree(fo->F); cudaFree(fo->F32); delete fo;
    set_error("fv_assemble_forcing: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  *out = fo;
  return FV_OK;
}

extern "C" int fv_forcing_copy(fv_forcing fo, double* F) {
  clear_error();
  FV_CHECK_ARG(fo && F, "fv_forcing_copy: null argument");
  FV_CUDA_TRY(cudaMemcpyAsync(F, fo->F, sizeof(double) * fo->mesh->n_e * fo->mesh->Nt, cudaMemcpyDeviceToHost,
                              fo->mesh->ctx->stream));
  FV_CUDA_TRY(cudaStreamSynchronize(fo->mesh->ctx->stream));
  return FV_OK;
}

extern "C" int fv_forcing_destroy(fv_forcing fo) {
  clear_error();
  if (!fo) return FV_OK;
  cudaFree(fo->F);
  cudaFree(fo->F32);
  delete fo;
  return FV_OK;
}

extern "C" int fv_bc_create(fv_ctx ctx, int n_bd, const double* bd_xy, const double* bd_g, double tau, int n_s,
                            const double* s_xy, const double* s_u, double gamma, fv_bc* out) {
  clear_error();
  FV_CHECK_ARG(ctx && out && n_bd >= 0 && n_s >= 0, "fv_bc_create: bad argument");
  FV_CHECK_ARG(n_bd == 0 || (bd_xy && bd_g), "fv_bc_create: boundary arrays missing");
  FV_CHECK_ARG(n_s == 0 || (s_xy && s_u), "fv_bc_create: sensor arrays missing");
  FV_CUDA_TRY(cudaSetDevice(ctx->device));
  fv_bc bc = new fv_bc_s();
  bc->ctx = ctx; bc->n_bd = n_bd; bc->n_s = n_s; bc->tau = tau; bc->gamma = gamma;
  const int n = n_bd + n_s;
  if (n > 0) {
    cudaError_t e;
    if ((e = cudaMalloc(&bc->xy, sizeof(double) * 2 * n)) || (e = cudaMalloc(&bc->val, sizeof(double) * n))) {
      cudaFree(bc->xy); delete bc;
      set_error("fv_bc_create: cudaMalloc failed (%s)", cudaGetErrorString(e));
      return FV_ERR_OOM;
    }
    cudaStream_t st = ctx->stream;
    if (n_bd) {
      cudaMemcpyAsync(bc->xy, bd_xy, sizeof(double) * 2 * n_bd, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(bc->val, bd_g, sizeof(double) * n_bd, cudaMemcpyHostToDevice, st);
    }
    if (n_s) {
      cudaMemcpyAsync(bc->xy + 2 * n_bd, s_xy, sizeof(double) * 2 * n_s, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(bc->val + n_bd, s_u, sizeof(double) * n_s, cudaMemcpyHostToDevice, st);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(bc->xy); cudaFree(bc->val); delete bc;
      set_error("fv_bc_create: %s", cudaGetErrorString(e));
      return FV_ERR_CUDA;
    }
  }
  *out = bc;
  return FV_OK;
}

extern "C" int fv_bc_destroy(fv_bc bc) {
  clear_error();
  if (!bc) return FV_OK;
  cudaFree(bc->xy); cudaFree(bc->val);
  delete bc;
  return FV_OK;
}
