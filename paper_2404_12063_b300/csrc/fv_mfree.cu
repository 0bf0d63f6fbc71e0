// Matrix-free contraction: the same loss, residuals and adjoint seeds as the
// stored-G contraction (Alg. 3 with the premultipliers of App. A.2), but G is
// never read from memory.  Per element the kernel rebuilds what it needs from
// the four vertices (bilinear map, App. A.1) and the reference tables
// (GLL nodes and weights, v_m and v_m' at the nodes), and evaluates the
// element sums by sum factorisation over the tensor-product structure
// v_(m,n)(xi, eta) = v_m(xi) v_n(eta):
//
//   Gx u_x + Gy u_y summed over q  =  sum_(a,b) P_ab v_m'(xi_a) v_n(eta_b) + Qm_ab v_m(xi_a) v_n'(eta_b)
//     P  = w (y_eta u_x - x_eta u_y),  Qm = w (x_xi u_y - y_xi u_x)        (adjugate form, no 1/|J|)
//   Gv (bx u_x + by u_y) summed over q =  sum_(a,b) C_ab v_m(xi_a) v_n(eta_b),  C = w |J| (bx u_x + by u_y)
//
// so each element costs O(T Q^2) instead of O(T^2 Q^2) and reads about
// 2.3 KB (grad u in, seeds out, F, vertices) instead of its G block.
// One warp per element; the tables sit in shared memory once per CTA.
#include <algorithm>

#include <type_traits>

#include "fv_internal.cuh"

namespace fv {
namespace {

__device__ __forceinline__ void cp_async_val(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_val(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct MfArgs {
  const double* verts;
  const int* cells;
  const double* tables;     // xi[Q], w[Q], v[T][Q], dv[T][Q]
  int n_e, Q, T;
  const void* Fr;           // [n_e][T*T] in the evaluation precision
  const void* U;            // [3][P_tot]
  void* UB;                 // [3][P_tot] seeds, or null (loss only)
  int64_t P_tot;
  double eps_h;
  const double* eps_d;
  double bx, by, rscale;
  double* partials;         // [gridDim][2]
  double* R_out;            // optional [n_e][T*T]
  float* seed_max;          // optional: raised to max |seed| (FP16 reverse sweep)
};

// One element's inputs staged in shared memory: u_x, u_y (and eps(x, y)) at its
// nodes and its F row.
__host__ __device__ inline int mf_stage_values(int Q, int T) { return ((3 * Q * Q + T * T) + 1) & ~1; }
// Shared memory per warp (values of R): P, Qm(, C) over the Q x Q nodes, the
// half-contracted T x Q arrays T1, T2(, T3), the Rbar rows and two input stages.
__host__ __device__ inline int mf_warp_values(int Q, int T, int nc) {
  return (nc == 3 ? 3 : 2) * (Q * Q + T * Q) + T * T + 2 * mf_stage_values(Q, T);
}
__host__ __device__ inline int mf_table_values(int Q, int T) { return 2 * Q + 2 * T * Q; }

// EPSQ: eps(x, y) at every node (the second output of a two-output network,
// Sec. 4.7.2) instead of the scalar eps; the kernel then also writes the seed
// dL/deps(x_q) = u_x sum_j Rbar_j Gx[j][q] + u_y sum_j Rbar_j Gy[j][q].
// QC, TC > 0: the orders as compile-time constants (index arithmetic by
// constants, loops unrolled); 0: the runtime orders.
template <class R, int NC, bool EPSQ, int QC = 0, int TC = 0>
__global__ void __launch_bounds__(256) contract_mfree(MfArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Q = QC ? QC : a.Q, T = TC ? TC : a.T, Nq = Q * Q, Nt = T * T, TQ = T * Q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  R* xi = reinterpret_cast<R*>(smem);
  R* wq = xi + Q;
  R* v = wq + Q;           // v[m][a] = v_m(xi_a)
  R* dv = v + TQ;          // dv[m][a] = v_m'(xi_a)
  for (int i = threadIdx.x; i < mf_table_values(Q, T); i += blockDim.x) xi[i] = (R)a.tables[i];
  __syncthreads();
  R* P = dv + TQ + (size_t)warp * mf_warp_values(Q, T, NC);
  R* Qm = P + Nq;
  R* C = Qm + Nq;                              // NC == 3
  R* T1 = P + (NC == 3 ? 3 : 2) * Nq;
  R* T2 = T1 + TQ;
  R* T3 = T2 + TQ;                             // NC == 3
  R* Rb = T1 + (NC == 3 ? 3 : 2) * TQ;
  R* stage = Rb + Nt;                          // [2][u_x (Nq), u_y (Nq), F (Nt), eps (Nq)]
  const int SV = mf_stage_values(Q, T);

  const R eps = (R)(a.eps_d ? *a.eps_d : a.eps_h);
  const R bx = (R)a.bx, by = (R)a.by, rscale = (R)a.rscale;
  const R* U = reinterpret_cast<const R*>(a.U);
  R* UB = reinterpret_cast<R*>(a.UB);
  const R* F = reinterpret_cast<const R*>(a.Fr);
  KahanR<R> lsum, dsum;
  float smx = 0.f;                 // largest |seed| this thread wrote

  // the element's u_x, u_y and F rows go to a stage with cp.async, one element ahead
  auto fetch = [&](int e, R* st) {
    if (e < a.n_e) {
      const int64_t p0 = (int64_t)e * Nq;
      for (int q = lane; q < Nq; q += 32) {
        cp_async_val(st + q, U + a.P_tot + p0 + q);
        cp_async_val(st + Nq + q, U + 2 * a.P_tot + p0 + q);
      }
      for (int j = lane; j < Nt; j += 32) cp_async_val(st + 2 * Nq + j, F + (size_t)e * Nt + j);
      if (EPSQ)
        for (int q = lane; q < Nq; q += 32) cp_async_val(st + 2 * Nq + Nt + q, U + 3 * a.P_tot + p0 + q);
    }
    cp_async_commit();
  };
  const int e_first = blockIdx.x * nw + warp, e_step = gridDim.x * nw;
  fetch(e_first, stage);
  int buf = 0;
  for (int e = e_first; e < a.n_e; e += e_step, buf ^= 1) {
    const R* st = stage + buf * SV;
    fetch(e + e_step, stage + (buf ^ 1) * SV);
    // Jacobian coefficients of the bilinear map in the evaluation precision
    // (FP64 arithmetic runs at a small fraction of the FP32 rate on this part)
    R vx[4], vy[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = a.cells[4 * (size_t)e + k];
      vx[k] = (R)a.verts[2 * c];
      vy[k] = (R)a.verts[2 * c + 1];
    }
    const R x1 = (R)0.25 * (-vx[0] + vx[1] + vx[2] - vx[3]), x2 = (R)0.25 * (-vx[0] - vx[1] + vx[2] + vx[3]);
    const R x3 = (R)0.25 * (vx[0] - vx[1] + vx[2] - vx[3]);
    const R y1 = (R)0.25 * (-vy[0] + vy[1] + vy[2] - vy[3]), y2 = (R)0.25 * (-vy[0] - vy[1] + vy[2] + vy[3]);
    const R y3 = (R)0.25 * (vy[0] - vy[1] + vy[2] - vy[3]);
    const int64_t p0 = (int64_t)e * Nq;
    cp_async_wait1();
    __syncwarp();
    // point terms
    for (int q = lane; q < Nq; q += 32) {
      const int ia = q / Q, ib = q - ia * Q;
      const R s = xi[ia], t = xi[ib];
      const R x_xi = x1 + x3 * t, x_eta = x2 + x3 * s, y_xi = y1 + y3 * t, y_eta = y2 + y3 * s;
      const R w = wq[ia] * wq[ib];
      const R ux = st[q], uy = st[Nq + q];
      const R we = EPSQ ? w * st[2 * Nq + Nt + q] : w;      // eps(x_q) folded into the diffusion terms
      P[q] = we * (y_eta * ux - x_eta * uy);
      Qm[q] = we * (x_xi * uy - y_xi * ux);
      if (NC == 3) C[q] = w * (x_xi * y_eta - x_eta * y_xi) * (bx * ux + by * uy);
    }
    __syncwarp();
    // contract over xi: T1[m][b] = sum_a v_m'(xi_a) P_ab, T2 = sum_a v_m(xi_a) Qm_ab, T3 = sum_a v_m(xi_a) C_ab
    for (int o = lane; o < TQ; o += 32) {
      const int m = o / Q, ib = o - m * Q;
      R s1 = 0, s2 = 0, s3 = 0;
      #pragma unroll 4
      for (int ia = 0; ia < Q; ++ia) {
        s1 += dv[m * Q + ia] * P[ia * Q + ib];
        s2 += v[m * Q + ia] * Qm[ia * Q + ib];
        if (NC == 3) s3 += v[m * Q + ia] * C[ia * Q + ib];
      }
      T1[o] = s1;
      T2[o] = s2;
      if (NC == 3) T3[o] = s3;
    }
    __syncwarp();
    // contract over eta: residual of test (m, n), loss and the eps derivative
    for (int j = lane; j < Nt; j += 32) {
      const int m = j / T, n = j - m * T;
      R A = 0, B = 0;
      #pragma unroll 4
      for (int ib = 0; ib < Q; ++ib) {
        A += T1[m * Q + ib] * v[n * Q + ib] + T2[m * Q + ib] * dv[n * Q + ib];
        if (NC == 3) B += T3[m * Q + ib] * v[n * Q + ib];
      }
      const R Rv = (EPSQ ? A : eps * A) + B - st[2 * Nq + j];
      const R rb = rscale * Rv;
      Rb[j] = rb;
      lsum.add(Rv * Rv);
      if (!EPSQ) dsum.add(rb * A);
      if (a.R_out) a.R_out[(size_t)e * Nt + j] = (double)Rv;
    }
    __syncwarp();
    if (UB) {
      // adjoint over eta: U1[m][b] = sum_n Rbar_mn v_n(eta_b), U2[m][b] = sum_n Rbar_mn v_n'(eta_b)
      for (int o = lane; o < TQ; o += 32) {
        const int m = o / Q, ib = o - m * Q;
        R s1 = 0, s2 = 0;
        #pragma unroll 4
        for (int n = 0; n < T; ++n) {
          s1 += Rb[m * T + n] * v[n * Q + ib];
          s2 += Rb[m * T + n] * dv[n * Q + ib];
        }
        T1[o] = s1;
        T2[o] = s2;
      }
      __syncwarp();
      // over xi: S_xi = sum_j Rbar_j v_xi,j(q), S_eta likewise, S_v = sum_j Rbar_j v_j(q); then the seeds
      for (int q = lane; q < Nq; q += 32) {
        const int ia = q / Q, ib = q - ia * Q;
        R sxi = 0, seta = 0, sv = 0;
        #pragma unroll 4
        for (int m = 0; m < T; ++m) {
          sxi += dv[m * Q + ia] * T1[m * Q + ib];
          seta += v[m * Q + ia] * T2[m * Q + ib];
          if (NC == 3) sv += v[m * Q + ia] * T1[m * Q + ib];
        }
        const R s = xi[ia], t = xi[ib];
        const R x_xi = x1 + x3 * t, x_eta = x2 + x3 * s, y_xi = y1 + y3 * t, y_eta = y2 + y3 * s;
        const R w = wq[ia] * wq[ib];
        const R gx = w * (y_eta * sxi - y_xi * seta);          // sum_j Rbar_j Gx[j][q]
        const R gy = w * (x_xi * seta - x_eta * sxi);          // sum_j Rbar_j Gy[j][q]
        const R gv = NC == 3 ? w * (x_xi * y_eta - x_eta * y_xi) * sv : (R)0;
        const R eq = EPSQ ? st[2 * Nq + Nt + q] : eps;
        const R s1 = eq * gx + bx * gv, s2 = eq * gy + by * gv;
        UB[p0 + q] = (R)0;
        UB[a.P_tot + p0 + q] = s1;
        UB[2 * a.P_tot + p0 + q] = s2;
        smx = fmaxf(smx, fmaxf(fabsf((float)s1), fabsf((float)s2)));
        if (EPSQ) UB[3 * a.P_tot + p0 + q] = st[q] * gx + st[Nq + q] * gy;
      }
    }
    __syncwarp();
  }
  cp_async_wait0();
  warp_max_to(a.seed_max, smx);
  // loss partials: per-thread compensated sums, a fixed-order tree in FP64 per warp, warps in order
  __shared__ double s_red[8][2];
  double l = (double)lsum.s - (double)lsum.c, d = (double)dsum.s - (double)dsum.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if (lane == 0) {
    s_red[warp][0] = l;
    s_red[warp][1] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ls = 0.0, ds = 0.0;
    for (int w = 0; w < nw; ++w) {
      ls += s_red[w][0];
      ds += s_red[w][1];
    }
    a.partials[2 * blockIdx.x] = ls;
    a.partials[2 * blockIdx.x + 1] = ds;
  }
}

template <class R, int NC, bool EPSQ, int QC, int TC>
cudaError_t launch_mf_shape(fv_ctx ctx, const MfArgs& a, int grid, int wpb, size_t smem) {
  cudaError_t e = ensure_smem_attr(ctx, (const void*)contract_mfree<R, NC, EPSQ, QC, TC>, smem);
  if (e == cudaSuccess) contract_mfree<R, NC, EPSQ, QC, TC><<<grid, 32 * wpb, smem, ctx->stream>>>(a);
  return e;
}
// FP32 evaluations of the common orders use compile-time instantiations.
template <class R, int NC, bool EPSQ>
cudaError_t launch_mf(fv_ctx ctx, const MfArgs& a, int grid, int wpb, size_t smem) {
  if constexpr (std::is_same<R, float>::value) {
    if (a.Q == 10 && a.T == 8) return launch_mf_shape<R, NC, EPSQ, 10, 8>(ctx, a, grid, wpb, smem);
    if (a.Q == 8 && a.T == 6) return launch_mf_shape<R, NC, EPSQ, 8, 6>(ctx, a, grid, wpb, smem);
    if (a.Q == 5 && a.T == 5) return launch_mf_shape<R, NC, EPSQ, 5, 5>(ctx, a, grid, wpb, smem);
  }
  return launch_mf_shape<R, NC, EPSQ, 0, 0>(ctx, a, grid, wpb, smem);
}
template <class R, bool EPSQ>
cudaError_t launch_mf_nc(fv_ctx ctx, const MfArgs& a, int nc, int grid, int wpb, size_t smem) {
  return nc == 3 ? launch_mf<R, 3, EPSQ>(ctx, a, grid, wpb, smem) : launch_mf<R, 2, EPSQ>(ctx, a, grid, wpb, smem);
}

}  // namespace

template <class R, int NC>
int mf_blocks_per_sm(fv_ctx ctx, int wpb, size_t smem) {
  return std::max(1, occupancy(ctx, (const void*)contract_mfree<R, NC, true>, 32 * wpb, smem));
}

// Warps per CTA (up to 8) such that tables and per-warp scratch fit in about
// 96 KB; a persistent grid (resident CTAs per SM x SMs, at most one element
// per warp) so that every warp streams several elements through its stages.
void mfree_grid(fv_ctx ctx, fv_mesh m, fv_precision prec, int* grid, int* wpb, size_t* smem) {
  const size_t rsz = prec == FV_FP64 ? 8 : 4;
  const size_t per_warp = (size_t)mf_warp_values(m->Q, m->T, m->n_comp) * rsz;
  const size_t tables = (size_t)mf_table_values(m->Q, m->T) * rsz;
  int w = 8;
  while (w > 1 && tables + w * per_warp > 96 * 1024) --w;
  *wpb = w;
  *smem = tables + w * per_warp;
  int per_sm = 1;
  if (*smem <= ctx->smem_optin) {
    if (prec == FV_FP64)
      per_sm = m->n_comp == 3 ? mf_blocks_per_sm<double, 3>(ctx, w, *smem) : mf_blocks_per_sm<double, 2>(ctx, w, *smem);
    else
      per_sm = m->n_comp == 3 ? mf_blocks_per_sm<float, 3>(ctx, w, *smem) : mf_blocks_per_sm<float, 2>(ctx, w, *smem);
  }
  const int64_t blocks = (m->n_e + w - 1) / w;
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)ctx->n_sm * per_sm));
}

int launch_contract_mfree(fv_ctx ctx, fv_mesh m, fv_forcing f, const EvalPlan& pl, const void* U, void* UB,
                          double eps, const double* eps_dev, double bx, double by, double rscale, double* partials,
                          int* n_part, double* R_out) {
  int grid, wpb;
  size_t smem;
  mfree_grid(ctx, m, pl.prec, &grid, &wpb, &smem);
  if (smem > ctx->smem_optin) {
    set_error("matrix-free contraction: Q = %d, T = %d need %zu bytes of shared memory", m->Q, m->T, smem);
    return FV_ERR_UNSUPPORTED;
  }
  MfArgs a;
  a.verts = m->verts; a.cells = m->cells; a.tables = m->tables;
  a.n_e = m->n_e; a.Q = m->Q; a.T = m->T;
  a.Fr = pl.prec == FV_FP64 ? (const void*)f->F : (const void*)f->F32;
  a.U = U; a.UB = UB; a.P_tot = pl.P_tot;
  a.eps_h = eps; a.eps_d = eps_dev; a.bx = bx; a.by = by; a.rscale = rscale;
  a.partials = partials; a.R_out = R_out; a.seed_max = pl.seed_max;
  *n_part = grid;
  cudaEvent_t ta;
  time_begin(ctx, K_CONTRACT, &ta);
  cudaError_t e;
  const bool epsq = pl.shape.w[pl.shape.L] == 2;
  if (pl.prec == FV_FP64)
    e = epsq ? launch_mf_nc<double, true>(ctx, a, m->n_comp, grid, wpb, smem)
             : launch_mf_nc<double, false>(ctx, a, m->n_comp, grid, wpb, smem);
  else
    e = epsq ? launch_mf_nc<float, true>(ctx, a, m->n_comp, grid, wpb, smem)
             : launch_mf_nc<float, false>(ctx, a, m->n_comp, grid, wpb, smem);
  if (e == cudaSuccess) e = cudaGetLastError();
  time_end(ctx, K_CONTRACT, ta);
  if (e != cudaSuccess) {
    set_error("matrix-free contraction launch failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

}  // namespace fv
