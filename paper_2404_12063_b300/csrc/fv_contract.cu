// Contraction of the stacked premultiplier tensor with the network gradient,
// the variational loss and its adjoint (Algorithm 3, Sec. 4.4):
//
//   A[e][j]  = sum_q Gx[e][j][q] u_x[e][q] + Gy[e][j][q] u_y[e][q]
//   B[e][j]  = sum_q Gv[e][j][q] (bx u_x + by u_y)           (convection, Eq. CD2D_strong)
//   R[e][j]  = eps A + B - F[e][j]
//   Lv       = inv_norm sum R^2                               (Alg. 3: inv_norm = 1/N_test)
//   Rbar     = 2 inv_norm R
//   dL/du_x[e][q] = sum_j Rbar[e][j] (eps Gx[e][j][q] + bx Gv[e][j][q])   (likewise y)
//   dL/deps  = sum_{e,j} Rbar A
//
// G is streamed from HBM exactly once: each CTA pulls element groups into a
// ring of shared-memory stages with cp.async.bulk (TMA bulk copies completing
// on an mbarrier), then runs the row pass (residuals; warp-shuffle sums over
// q) and the column pass (adjoint seeds; one thread per quadrature point) on
// the same shared tile.
#include <algorithm>

#include "fv_internal.cuh"

namespace fv {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most ~limit_ns; false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

struct ContractArgs {
  const void* G;
  int64_t g_stride_bytes;
  int n_e, Nt, Nq, n_comp;
  const double* F;
  const void* U;        // [3][P_tot] (u, u_x, u_y) in R
  void* UB;             // [3][P_tot] seeds, or null (loss only)
  int64_t P_tot;
  double eps_h;
  const double* eps_d;
  double bx, by, rscale;
  int elems_per_stage, n_stages, n_groups;
  double* partials;     // [gridDim][2]
  int* err;
  double* R_out;        // optional [n_e][Nt] element residuals
};

template <class R, class Gt>
__global__ void __launch_bounds__(kThreads) contract_pipelined(ContractArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nt = a.Nt, Nq = a.Nq, Eg = a.elems_per_stage, S = a.n_stages;
  const size_t stage_bytes = (size_t)Eg * a.g_stride_bytes;
  unsigned char* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  R* s_ux = reinterpret_cast<R*>(full + S);
  R* s_uy = s_ux + (size_t)Eg * Nq;
  // 2*Eg*Nq values of R (4 or 8 bytes) keep s_R 8-byte aligned
  double* s_R = reinterpret_cast<double*>(s_uy + (size_t)Eg * Nq);
  double* s_red = s_R + (size_t)Eg * Nt;     // [kWarps][4]

  const double eps = a.eps_d ? *a.eps_d : a.eps_h;
  const R* U = reinterpret_cast<const R*>(a.U);
  R* UB = reinterpret_cast<R*>(a.UB);
  const unsigned char* Gb = reinterpret_cast<const unsigned char*>(a.G);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](int it) {
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp >= a.n_groups) return;
    const int s = it % S;
    const int e0 = grp * Eg;
    const int ne = min(Eg, a.n_e - e0);
    const uint32_t bytes = (uint32_t)(ne * a.g_stride_bytes);
    mbar_expect_tx(&full[s], bytes);
    bulk_g2s(stages + s * stage_bytes, Gb + (size_t)e0 * a.g_stride_bytes, bytes, &full[s]);
  };
  if (tid == 0)
    for (int it = 0; it < S; ++it) issue(it);

  KSum lsum, dsum;       // lane 0 of each warp accumulates
  const int ncomp = a.n_comp;
  for (int it = 0;; ++it) {
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp >= a.n_groups) break;
    const int s = it % S;
    const uint32_t parity = (uint32_t)((it / S) & 1);
    const int e0 = grp * Eg;
    const int ne = min(Eg, a.n_e - e0);
    // stage the gradient values of this group's points (contiguous in [3][P_tot])
    const int64_t p0 = (int64_t)e0 * Nq;
    for (int i = tid; i < ne * Nq; i += kThreads) {
      s_ux[i] = U[a.P_tot + p0 + i];
      s_uy[i] = U[2 * a.P_tot + p0 + i];
    }
    const bool ok = mbar_wait_bounded(&full[s], parity, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT);
      // drain: give the other issued copies a bounded chance to land before exiting
      if (tid == 0)
        for (int k = 1; k < S; ++k) {
          const int it2 = it + k;
          if (blockIdx.x + it2 * gridDim.x < a.n_groups)
            mbar_wait_bounded(&full[it2 % S], (uint32_t)((it2 / S) & 1), kWaitLimitNs / 4);
        }
      return;
    }
    const Gt* tile = reinterpret_cast<const Gt*>(stages + s * stage_bytes);
    const int64_t gstride = a.g_stride_bytes / (int64_t)sizeof(Gt);

    // ---- row pass: one warp per (element, test function) row
    for (int row = warp; row < ne * Nt; row += kWarps) {
      const int k = row / Nt, j = row - k * Nt;
      const Gt* gx = tile + k * gstride + (size_t)j * Nq;
      const Gt* gy = gx + (size_t)Nt * Nq;
      const R* ux = s_ux + k * Nq;
      const R* uy = s_uy + k * Nq;
      R accA = 0, accB = 0;
      if (ncomp == 3) {
        const Gt* gv = gy + (size_t)Nt * Nq;
        const R bx = (R)a.bx, by = (R)a.by;
        for (int q = lane; q < Nq; q += 32) {
          const R x = ux[q], y = uy[q];
          accA += (R)gx[q] * x + (R)gy[q] * y;
          accB += (R)gv[q] * (bx * x + by * y);
        }
        accB = warp_sum(accB);
      } else {
        for (int q = lane; q < Nq; q += 32) accA += (R)gx[q] * ux[q] + (R)gy[q] * uy[q];
      }
      accA = warp_sum(accA);
      if (lane == 0) {
        const double A = (double)accA;
        const double Rv = eps * A + (double)accB - a.F[(size_t)(e0 + k) * Nt + j];
        s_R[row] = Rv;
        if (a.R_out) a.R_out[(size_t)(e0 + k) * Nt + j] = Rv;
        lsum.add(Rv * Rv);
        dsum.add(a.rscale * Rv * A);
      }
    }
    __syncthreads();

    // ---- column pass: adjoint seeds at each quadrature point
    if (UB) {
      for (int col = tid; col < ne * Nq; col += kThreads) {
        const int k = col / Nq, q = col - k * Nq;
        const Gt* gx = tile + k * gstride + q;
        const Gt* gy = gx + (size_t)Nt * Nq;
        const double* Rk = s_R + k * Nt;
        R sx = 0, sy = 0, sv = 0;
        if (ncomp == 3) {
          const Gt* gv = gy + (size_t)Nt * Nq;
          for (int j = 0; j < Nt; ++j) {
            const R rb = (R)(a.rscale * Rk[j]);
            sx += rb * (R)gx[(size_t)j * Nq];
            sy += rb * (R)gy[(size_t)j * Nq];
            sv += rb * (R)gv[(size_t)j * Nq];
          }
        } else {
          for (int j = 0; j < Nt; ++j) {
            const R rb = (R)(a.rscale * Rk[j]);
            sx += rb * (R)gx[(size_t)j * Nq];
            sy += rb * (R)gy[(size_t)j * Nq];
          }
        }
        const int64_t p = p0 + col;
        UB[p] = (R)0;
        UB[a.P_tot + p] = (R)eps * sx + (R)a.bx * sv;
        UB[2 * a.P_tot + p] = (R)eps * sy + (R)a.by * sv;
      }
    }
    __syncthreads();
    if (tid == 0) issue(it + S);
  }
  // ---- CTA partials (loss sum and dL/deps), compensated
  if (lane == 0) {
    s_red[warp * 4 + 0] = lsum.s; s_red[warp * 4 + 1] = lsum.c;
    s_red[warp * 4 + 2] = dsum.s; s_red[warp * 4 + 3] = dsum.c;
  }
  __syncthreads();
  if (tid == 0) {
    KSum l, d;
    for (int w = 0; w < kWarps; ++w) {
      l.add(s_red[w * 4 + 0]); l.add(s_red[w * 4 + 1]);
      d.add(s_red[w * 4 + 2]); d.add(s_red[w * 4 + 3]);
    }
    a.partials[2 * blockIdx.x] = l.value();
    a.partials[2 * blockIdx.x + 1] = d.value();
  }
}

// Fallback for element blocks too large for a shared-memory stage: one CTA per
// element, G read straight from global memory in both passes.
template <class R, class Gt>
__global__ void __launch_bounds__(kThreads) contract_direct(ContractArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_R = reinterpret_cast<double*>(smem);     // [Nt]
  double* s_red = s_R + a.Nt;                         // [kWarps][4]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nt = a.Nt, Nq = a.Nq;
  const double eps = a.eps_d ? *a.eps_d : a.eps_h;
  const R* U = reinterpret_cast<const R*>(a.U);
  R* UB = reinterpret_cast<R*>(a.UB);
  const int64_t gstride = a.g_stride_bytes / (int64_t)sizeof(Gt);
  KSum lsum, dsum;
  for (int e = blockIdx.x; e < a.n_e; e += gridDim.x) {
    const Gt* Ge = reinterpret_cast<const Gt*>(a.G) + (size_t)e * gstride;
    const R* ux = U + a.P_tot + (int64_t)e * Nq;
    const R* uy = U + 2 * a.P_tot + (int64_t)e * Nq;
    for (int j = warp; j < Nt; j += kWarps) {
      const Gt* gx = Ge + (size_t)j * Nq;
      const Gt* gy = gx + (size_t)Nt * Nq;
      R accA = 0, accB = 0;
      for (int q = lane; q < Nq; q += 32) {
        accA += (R)gx[q] * ux[q] + (R)gy[q] * uy[q];
        if (a.n_comp == 3) accB += (R)gy[(size_t)Nt * Nq + q] * ((R)a.bx * ux[q] + (R)a.by * uy[q]);
      }
      accA = warp_sum(accA);
      accB = warp_sum(accB);
      if (lane == 0) {
        const double A = (double)accA;
        const double Rv = eps * A + (double)accB - a.F[(size_t)e * Nt + j];
        s_R[j] = Rv;
        if (a.R_out) a.R_out[(size_t)e * Nt + j] = Rv;
        lsum.add(Rv * Rv);
        dsum.add(a.rscale * Rv * A);
      }
    }
    __syncthreads();
    if (UB) {
      for (int q = tid; q < Nq; q += kThreads) {
        R sx = 0, sy = 0, sv = 0;
        for (int j = 0; j < Nt; ++j) {
          const R rb = (R)(a.rscale * s_R[j]);
          sx += rb * (R)Ge[(size_t)j * Nq + q];
          sy += rb * (R)Ge[(size_t)(Nt + j) * Nq + q];
          if (a.n_comp == 3) sv += rb * (R)Ge[(size_t)(2 * Nt + j) * Nq + q];
        }
        const int64_t p = (int64_t)e * Nq + q;
        UB[p] = (R)0;
        UB[a.P_tot + p] = (R)eps * sx + (R)a.bx * sv;
        UB[2 * a.P_tot + p] = (R)eps * sy + (R)a.by * sv;
      }
    }
    __syncthreads();
  }
  if (lane == 0) {
    s_red[warp * 4 + 0] = lsum.s; s_red[warp * 4 + 1] = lsum.c;
    s_red[warp * 4 + 2] = dsum.s; s_red[warp * 4 + 3] = dsum.c;
  }
  __syncthreads();
  if (tid == 0) {
    KSum l, d;
    for (int w = 0; w < kWarps; ++w) {
      l.add(s_red[w * 4 + 0]); l.add(s_red[w * 4 + 1]);
      d.add(s_red[w * 4 + 2]); d.add(s_red[w * 4 + 3]);
    }
    a.partials[2 * blockIdx.x] = l.value();
    a.partials[2 * blockIdx.x + 1] = d.value();
  }
}

size_t pipelined_smem(size_t stage_bytes, int S, int Eg, int Nq, int Nt, size_t rsz) {
  size_t b = S * stage_bytes + S * 8;
  b += 2 * (size_t)Eg * Nq * rsz;       // s_ux, s_uy
  b += (size_t)Eg * Nt * 8 + kWarps * 4 * 8;
  return b;
}

template <class R, class Gt>
int launch_t(fv_ctx ctx, const ContractArgs& a0, bool pipelined, int grid, size_t smem) {
  ContractArgs a = a0;
  cudaError_t e;
  if (pipelined) {
    e = cudaFuncSetAttribute(contract_pipelined<R, Gt>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) contract_pipelined<R, Gt><<<grid, kThreads, smem, ctx->stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(contract_direct<R, Gt>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) contract_direct<R, Gt><<<grid, kThreads, smem, ctx->stream>>>(a);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("contraction launch failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

}  // namespace

// Stage geometry: about 48 KB of G per stage, up to 4 stages within ~200 KB.
int contract_grid(fv_ctx ctx, fv_mesh m, fv_precision prec, int* grid, int* eg, int* stages, size_t* smem) {
  const size_t rsz = prec == FV_FP64 ? 8 : 4;
  const size_t budget = std::min<size_t>(ctx->smem_optin, 220 * 1024);
  const size_t gs = m->g_stride_bytes;
  int E = (int)std::max<size_t>(1, (48 * 1024) / gs);
  E = std::min(E, 32);
  int S = 4;
  while (S >= 2 && pipelined_smem(E * gs, S, E, m->Nq, m->Nt, rsz) > budget) {
    if (E > 1) E = std::max(1, E / 2); else --S;
  }
  if (S < 2 || E * gs > (1u << 20) - 16) {   // element block too large to stage: direct kernel
    *eg = 0; *stages = 0;
    *smem = (size_t)m->Nt * 8 + kWarps * 4 * 8;
    *grid = (int)std::min<int64_t>(m->n_e, (int64_t)ctx->n_sm * 8);
    return FV_OK;
  }
  const size_t sm = pipelined_smem(E * gs, S, E, m->Nq, m->Nt, rsz);
  const int per_sm = std::max<int>(1, (int)(std::min<size_t>(ctx->smem_optin, 228 * 1024) / (sm + 1024)));
  const int n_groups = (m->n_e + E - 1) / E;
  *eg = E; *stages = S; *smem = sm;
  *grid = std::min<int>(n_groups, ctx->n_sm * std::min(per_sm, 2));
  return FV_OK;
}

int launch_contract(fv_ctx ctx, fv_mesh m, fv_forcing f, const EvalPlan& pl, const void* U, void* UB, double eps,
                    const double* eps_dev, double bx, double by, double rscale, double* partials, int* n_part,
                    double* R_out) {
  int grid, E, S;
  size_t smem;
  contract_grid(ctx, m, pl.prec, &grid, &E, &S, &smem);
  ContractArgs a;
  a.G = m->G; a.g_stride_bytes = (int64_t)m->g_stride_bytes;
  a.n_e = m->n_e; a.Nt = m->Nt; a.Nq = m->Nq; a.n_comp = m->n_comp;
  a.F = f->F; a.U = U; a.UB = UB; a.P_tot = pl.P_tot;
  a.eps_h = eps; a.eps_d = eps_dev; a.bx = bx; a.by = by; a.rscale = rscale;
  a.elems_per_stage = E; a.n_stages = S; a.n_groups = E ? (m->n_e + E - 1) / E : m->n_e;
  a.partials = partials; a.err = ctx->err_dev; a.R_out = R_out;
  *n_part = grid;
  const bool pip = E > 0;
  cudaEvent_t ta;
  time_begin(ctx, K_CONTRACT, &ta);
  int rc;
  if (pl.prec == FV_FP64) {
    if (m->storage != FV_FP64) { set_error("FP64 evaluation needs FP64 G storage"); return FV_ERR_UNSUPPORTED; }
    rc = launch_t<double, double>(ctx, a, pip, grid, smem);
  } else if (m->storage == FV_FP32) {
    rc = launch_t<float, float>(ctx, a, pip, grid, smem);
  } else if (m->storage == FV_BF16) {
    rc = launch_t<float, __nv_bfloat16>(ctx, a, pip, grid, smem);
  } else {
    rc = launch_t<float, double>(ctx, a, pip, grid, smem);
  }
  time_end(ctx, K_CONTRACT, ta);
  return rc;
}

}  // namespace fv
