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
  const void* Fr;       // F in the evaluation precision (R)
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

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <class R> __device__ __forceinline__ void cp_async_r(R* dst, const R* src);
template <> __device__ __forceinline__ void cp_async_r<float>(float* d, const float* s) { cp_async4(d, s); }
template <> __device__ __forceinline__ void cp_async_r<double>(double* d, const double* s) { cp_async8(d, s); }

// Per-stage auxiliary data: u_x, u_y of the group's points and its F rows.
template <class R>
struct Aux {
  R* ux;
  R* uy;
  R* F;
};

constexpr int kPThreads = 512;                      // pipelined kernel: 16 warps
constexpr int kPWarps = kPThreads / 32;

// Row step over NR consecutive test rows (j .. j+NR-1) of one element: the
// lane's q-chunks of each G row are loaded from the stage once and used for
// both the residual (butterfly all-reduce over the warp) and the adjoint
// accumulation.
template <class R, class Gt, int KQ, int NC, int NR>
__device__ __forceinline__ void row_step(const Gt* __restrict__ tile_k, int j, int Nt, int Nq, int lane,
                                         const R (&gu)[KQ], const R (&gw)[KQ], R bx, R by, R eps, R rscale,
                                         const R* __restrict__ Fr, R (&ax)[KQ], R (&ay)[KQ], R (&av)[KQ],
                                         KahanR<R>& lsum, KahanR<R>& dsum, double* R_out_row) {
  R vx[NR][KQ], vy[NR][KQ], vv[NR][KQ];
  R A[NR], B[NR];
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    const Gt* gx = tile_k + (j + t) * Nq;
    const Gt* gy = gx + Nt * Nq;
    const Gt* gv = gy + Nt * Nq;
    A[t] = 0; B[t] = 0;
#pragma unroll
    for (int m = 0; m < KQ; ++m) {
      const int q = lane + 32 * m;
      const bool in = (KQ == 1 || m < KQ - 1) ? (q < Nq) : (q < Nq);
      vx[t][m] = in ? (R)gx[q] : (R)0;
      vy[t][m] = in ? (R)gy[q] : (R)0;
      A[t] += vx[t][m] * gu[m] + vy[t][m] * gw[m];
      if (NC == 3) {
        vv[t][m] = in ? (R)gv[q] : (R)0;
        B[t] += vv[t][m] * (bx * gu[m] + by * gw[m]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int t = 0; t < NR; ++t) {
      A[t] += __shfl_xor_sync(0xffffffffu, A[t], o);
      if (NC == 3) B[t] += __shfl_xor_sync(0xffffffffu, B[t], o);
    }
  }
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    const R Rv = eps * A[t] + B[t] - Fr[t];
    const R Rb = rscale * Rv;
    if (lane == 0) {
      lsum.add(Rv * Rv);
      dsum.add(Rb * A[t]);
      if (R_out_row) R_out_row[t] = (double)Rv;
    }
#pragma unroll
    for (int m = 0; m < KQ; ++m) {
      ax[m] += Rb * vx[t][m];
      ay[m] += Rb * vy[t][m];
      if (NC == 3) av[m] += Rb * vv[t][m];
    }
  }
}

// KQ = ceil(Nq / 32) quadrature chunks per lane (lane l owns q = l + 32 m);
// NC = 2 (diffusion only) or 3 (with the convection/mass component).
template <class R, class Gt, int KQ, int NC>
__global__ void __launch_bounds__(kPThreads) contract_pipelined(ContractArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nt = a.Nt, Nq = a.Nq, Eg = a.elems_per_stage, S = a.n_stages;
  const size_t stage_bytes = (size_t)Eg * a.g_stride_bytes;
  unsigned char* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  R* aux_base = reinterpret_cast<R*>(full + S);
  const int aux_n = 2 * Eg * Nq + Eg * Nt;          // R values per aux buffer
  auto aux_of = [&](int b) {
    Aux<R> x;
    x.ux = aux_base + b * aux_n;
    x.uy = x.ux + Eg * Nq;
    x.F = x.uy + Eg * Nq;
    return x;
  };
  // seed partial sums, one slot per (warp, element) segment: slot = warp + element
  R* s_seg = aux_base + 2 * aux_n;                    // [kPWarps + Eg - 1][3][Nq]
  const int n_seg = kPWarps + Eg - 1;
  double* s_red = reinterpret_cast<double*>(s_seg + ((3 * n_seg * Nq + 1) & ~1));   // [kPWarps][4]

  const R eps = (R)(a.eps_d ? *a.eps_d : a.eps_h);
  const R bx = (R)a.bx, by = (R)a.by, rscale = (R)a.rscale;
  const R* U = reinterpret_cast<const R*>(a.U);
  const R* Fsrc = reinterpret_cast<const R*>(a.Fr);
  R* UB = reinterpret_cast<R*>(a.UB);
  const unsigned char* Gb = reinterpret_cast<const unsigned char*>(a.G);
  const int gstride = (int)(a.g_stride_bytes / (int64_t)sizeof(Gt));

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
  auto prefetch_aux = [&](int it) {
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp < a.n_groups) {
      const Aux<R> x = aux_of(it & 1);
      const int e0 = grp * Eg;
      const int ne = min(Eg, a.n_e - e0);
      const int64_t p0 = (int64_t)e0 * Nq;
      for (int i = tid; i < ne * Nq; i += kPThreads) {
        cp_async_r<R>(x.ux + i, U + a.P_tot + p0 + i);
        cp_async_r<R>(x.uy + i, U + 2 * a.P_tot + p0 + i);
      }
      for (int i = tid; i < ne * Nt; i += kPThreads) cp_async_r<R>(x.F + i, Fsrc + (size_t)e0 * Nt + i);
    }
    cp_async_commit();
  };
  if (tid == 0)
    for (int it = 0; it < S; ++it) issue(it);
  prefetch_aux(0);

  KahanR<R> lsum, dsum;        // lane 0 of each warp
  for (int it = 0;; ++it) {
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp >= a.n_groups) break;
    const int s = it % S;
    const uint32_t parity = (uint32_t)((it / S) & 1);
    const int e0 = grp * Eg;
    const int ne = min(Eg, a.n_e - e0);
    prefetch_aux(it + 1);
    cp_async_wait1();
    const bool ok = mbar_wait_bounded(&full[s], parity, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, FV_ERR_TIMEOUT);
        for (int k = 1; k < S; ++k) {      // bounded drain of the other copies in flight
          const int it2 = it + k;
          if (blockIdx.x + it2 * gridDim.x < a.n_groups)
            mbar_wait_bounded(&full[it2 % S], (uint32_t)((it2 / S) & 1), kWaitLimitNs / 4);
        }
      }
      cp_async_wait0();
      return;
    }
    const Gt* tile = reinterpret_cast<const Gt*>(stages + s * stage_bytes);
    const Aux<R> x = aux_of(it & 1);

    // each warp takes a contiguous block of the group's (element, test) rows
    const int n_rows = ne * Nt;
    const int rpw = (n_rows + kPWarps - 1) / kPWarps;
    const int r0 = warp * rpw, r1 = min(n_rows, r0 + rpw);
    if (r0 < r1) {
      int k = r0 / Nt, j = r0 - k * Nt;
      R gu[KQ], gw[KQ], ax[KQ], ay[KQ], av[KQ];
      auto load_elem = [&](int kk) {
#pragma unroll
        for (int m = 0; m < KQ; ++m) {
          const int q = lane + 32 * m;
          gu[m] = q < Nq ? x.ux[kk * Nq + q] : (R)0;
          gw[m] = q < Nq ? x.uy[kk * Nq + q] : (R)0;
          ax[m] = ay[m] = av[m] = (R)0;
        }
      };
      auto flush = [&](int kk) {
        R* seg = s_seg + (warp + kk) * 3 * Nq;
#pragma unroll
        for (int m = 0; m < KQ; ++m) {
          const int q = lane + 32 * m;
          if (q < Nq) {
            seg[q] = ax[m];
            seg[Nq + q] = ay[m];
            if (NC == 3) seg[2 * Nq + q] = av[m];
          }
        }
      };
      load_elem(k);
      int r = r0;
      while (r < r1) {
        if (j == Nt) { flush(k); ++k; j = 0; load_elem(k); }
        const Gt* tile_k = tile + k * gstride;
        double* rout = a.R_out ? a.R_out + (size_t)(e0 + k) * Nt + j : nullptr;
        if (r + 1 < r1 && j + 1 < Nt) {
          row_step<R, Gt, KQ, NC, 2>(tile_k, j, Nt, Nq, lane, gu, gw, bx, by, eps, rscale, x.F + r, ax, ay, av,
                                     lsum, dsum, rout);
          r += 2; j += 2;
        } else {
          row_step<R, Gt, KQ, NC, 1>(tile_k, j, Nt, Nq, lane, gu, gw, bx, by, eps, rscale, x.F + r, ax, ay, av,
                                     lsum, dsum, rout);
          r += 1; j += 1;
        }
      }
      flush(k);
    }
    __syncthreads();
    // seeds dL/du = 0, dL/du_x = eps sum Rbar Gx + bx sum Rbar Gv, likewise y;
    // an element's segments are summed in warp order (deterministic)
    const int64_t p0 = (int64_t)e0 * Nq;
    for (int col = tid; col < ne * Nq; col += kPThreads) {
      const int k = col / Nq, q = col - k * Nq;
      const int w_lo = (k * Nt) / rpw, w_hi = min(kPWarps - 1, ((k + 1) * Nt - 1) / rpw);
      R sx = 0, sy = 0, sv = 0;
      for (int w = w_lo; w <= w_hi; ++w) {
        const R* seg = s_seg + (w + k) * 3 * Nq + q;
        sx += seg[0];
        sy += seg[Nq];
        if (NC == 3) sv += seg[2 * Nq];
      }
      if (UB) {
        UB[p0 + col] = (R)0;
        UB[a.P_tot + p0 + col] = eps * sx + bx * sv;
        UB[2 * a.P_tot + p0 + col] = eps * sy + by * sv;
      }
    }
    __syncthreads();
    if (tid == 0) issue(it + S);
  }
  cp_async_wait0();
  if (lane == 0) {
    s_red[warp * 4 + 0] = (double)lsum.s; s_red[warp * 4 + 1] = -(double)lsum.c;
    s_red[warp * 4 + 2] = (double)dsum.s; s_red[warp * 4 + 3] = -(double)dsum.c;
  }
  __syncthreads();
  if (tid == 0) {
    double l = 0.0, d = 0.0;
    for (int w = 0; w < kPWarps; ++w) {
      l += s_red[w * 4 + 0] + s_red[w * 4 + 1];
      d += s_red[w * 4 + 2] + s_red[w * 4 + 3];
    }
    a.partials[2 * blockIdx.x] = l;
    a.partials[2 * blockIdx.x + 1] = d;
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
  b += 2 * (size_t)(2 * Eg * Nq + Eg * Nt) * rsz;              // two aux buffers
  b += (size_t)((3 * (kPWarps + Eg - 1) * Nq + 1) & ~1) * rsz;  // seed segments
  b += kPWarps * 4 * 8 + 16;
  return b;
}

template <class R, class Gt, int KQ, int NC>
cudaError_t launch_pip(fv_ctx ctx, const ContractArgs& a, int grid, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(contract_pipelined<R, Gt, KQ, NC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) contract_pipelined<R, Gt, KQ, NC><<<grid, kPThreads, smem, ctx->stream>>>(a);
  return e;
}

template <class R, class Gt, int NC>
cudaError_t launch_pip_kq(fv_ctx ctx, const ContractArgs& a, int grid, size_t smem) {
  const int kq = (a.Nq + 31) / 32;
  return kq <= 1 ? launch_pip<R, Gt, 1, NC>(ctx, a, grid, smem)
       : kq == 2 ? launch_pip<R, Gt, 2, NC>(ctx, a, grid, smem)
       : kq == 3 ? launch_pip<R, Gt, 3, NC>(ctx, a, grid, smem)
                 : launch_pip<R, Gt, 4, NC>(ctx, a, grid, smem);
}

template <class R, class Gt>
int launch_t(fv_ctx ctx, const ContractArgs& a, bool pipelined, int grid, size_t smem) {
  cudaError_t e;
  if (pipelined) {
    e = a.n_comp == 3 ? launch_pip_kq<R, Gt, 3>(ctx, a, grid, smem) : launch_pip_kq<R, Gt, 2>(ctx, a, grid, smem);
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

// Stage geometry: about 96 KB of G per stage (several elements, so that the
// per-stage barriers are amortised over many rows), 2-4 stages within ~210 KB.
int contract_grid(fv_ctx ctx, fv_mesh m, fv_precision prec, int* grid, int* eg, int* stages, size_t* smem) {
  const size_t rsz = prec == FV_FP64 ? 8 : 4;
  const size_t budget = std::min<size_t>(ctx->smem_optin, 220 * 1024);
  const size_t gs = m->g_stride_bytes;
  // as many elements per stage as fit with two stages (up to ~96 KB), then add stages while they fit
  int E = (int)std::min<size_t>(32, std::max<size_t>(1, (96 * 1024 + gs - 1) / gs));
  while (E > 1 && pipelined_smem(E * gs, 2, E, m->Nq, m->Nt, rsz) > budget) --E;
  int S = pipelined_smem(E * gs, 2, E, m->Nq, m->Nt, rsz) <= budget ? 2 : 0;
  while (S >= 2 && S < 4 && pipelined_smem(E * gs, S + 1, E, m->Nq, m->Nt, rsz) <= budget) ++S;
  if (S < 2 || E * gs > (1u << 20) - 16 || m->Nq > 128) {   // too large to stage / > 4 q-chunks: direct kernel
    *eg = 0; *stages = 0;
    *smem = (size_t)m->Nt * 8 + kWarps * 4 * 8;
    *grid = (int)std::min<int64_t>(m->n_e, (int64_t)ctx->n_sm * 8);
    return FV_OK;
  }
  const size_t sm = pipelined_smem(E * gs, S, E, m->Nq, m->Nt, rsz);
  const int n_groups = (m->n_e + E - 1) / E;
  *eg = E; *stages = S; *smem = sm;
  *grid = std::min<int>(n_groups, ctx->n_sm);
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
  a.F = f->F; a.Fr = pl.prec == FV_FP64 ? (const void*)f->F : (const void*)f->F32; a.U = U; a.UB = UB; a.P_tot = pl.P_tot;
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
