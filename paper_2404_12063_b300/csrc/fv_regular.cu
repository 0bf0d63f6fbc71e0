// Regular-mesh contraction (Alg. 2, with the premultiplier assembly of the
// appendix): on a mesh of axis-aligned rectangles every element's
// premultipliers are one reference matrix scaled per element,
//
//   Gx[e][j][q] = J_x(e) Vxi[j][q],  Gy = J_y(e) Veta[j][q],  Gv = J(e) V[j][q]
//   Vxi = w v_xi,  Veta = w v_eta,  V = w v  (reference, shared by all elements)
//   J_x = |J| / (dx/dxi)... = h_y / 2,  J_y = h_x / 2,  J = h_x h_y / 4
//
// so the residuals of a tile of 128 elements are GEMMs with N = elements,
//
//   A [N_t x 128] = [Vxi | Veta] . [J_x u_x ; J_y u_y],   B = V . [J (b . grad u)]  (convection)
//   R = eps A + B - F^T,  Lv = inv_norm sum R^2,  Rbar = rscale R,  dL/deps = sum Rbar A
//
// and the adjoint seeds three more, D2_c [N_q x 128] = V_c^T . Rbar:
//
//   dL/du_x = eps J_x D2_xi + bx J D2_v,  dL/du_y = eps J_y D2_eta + by J D2_v.
//
// All of them run on the tensor cores (tcgen05, 16-bit operands, FP32
// accumulators in tensor memory).  The reference matrix is stored once in
// shared memory in the core-matrix layout and read K-major (rows = tests) by
// the residual GEMM and MN-major (rows = quadrature points) by the adjoint
// GEMMs.  Rbar is scaled by a per-tile power of two before it is rounded to
// 16 bits (exact to apply and undo).
#include <algorithm>
#include <cmath>
#include <vector>

#include "fv_internal.cuh"
#include "fv_tcgen05.cuh"

namespace fv {
namespace {

using namespace fv::tc;

constexpr int kRegTile = 128;         // elements per tile (the GEMMs' N)
constexpr int kRegThreads = 256;      // eight warps: two per TMEM lane quarter, each on half of the tile's elements

struct RegPlan {
  int Nq_pad;        // K-block width per component: Nq rounded up to 16
  int M2;            // adjoint GEMMs' M (64 or 128 >= Nq); reads may run into the next block (rows >= Nq unused)
  int Nt_blk, K1, nc;
  int o_A, o_B1, o_B2, o_J, o_red, o_bar, smem;
  int tmem_cols;
};

struct RegArgs {
  RegPlan pl;
  const float* J;         // [n_e][3]: y_eta, x_xi, |J| (rectangles)
  const uint4* ref;       // the reference matrix as its shared-memory image (Nt_blk x K1 16-bit values)
  const double* tables;   // xi[Q], w[Q], v[T][Q], dv[T][Q]
  int n_e, Q, T;
  const float* F;         // [n_e][T*T]
  const float* U;         // [3][P_tot]
  float* UB;              // [3][P_tot] or null
  int64_t P_tot;
  double eps_h;
  const double* eps_d;
  double bx, by, rscale;
  double* partials;       // [gridDim][2]
  double* R_out;          // optional [n_e][T*T]
  int* err;
  float* seed_max;        // optional: raised to max |seed| (FP16 reverse sweep)
};

bool make_reg_plan(int Q, int T, int nc, RegPlan* p) {
  const int Nq = Q * Q, Nt = T * T;
  if (Nq > 128 || Nt > 128 || nc < 2 || nc > 3) return false;
  p->nc = nc;
  p->Nq_pad = (Nq + 15) & ~15;
  p->M2 = Nq <= 64 ? 64 : 128;
  p->Nt_blk = Nt <= 64 ? 64 : 128;
  p->K1 = nc * p->Nq_pad;
  int o = 0;
  p->o_A = o; o += p->Nt_blk * p->K1 * 2;
  p->o_B1 = o; o += kRegTile * p->K1 * 2;          // B1 follows A: the adjoint reads past A's last block land here
  p->o_B2 = o; o += kRegTile * p->Nt_blk * 2;
  p->o_J = o; o += kRegTile * 3 * 4;                 // per element J_x, J_y, J
  o = (o + 15) & ~15;
  p->o_red = o; o += 64 * 8;                         // max |Rbar| bits, loss partials
  p->o_bar = o; o += 16;                             // mbarrier + TMEM base
  // D2_0 reuses D1's columns: 256 tensor-memory columns for two components (two CTAs per SM), 512 for
  // three (one per SM); the shared-memory request is padded so that no more CTAs than that share an SM
  p->tmem_cols = nc == 2 ? 256 : 512;
  const int min_smem = nc == 2 ? 77 * 1024 : 116 * 1024;
  p->smem = std::max((o + 127) & ~127, min_smem);
  return p->smem <= 227 * 1024;
}

// 16-bit element (row, k) of a core-matrix tile with Kb columns.
__device__ __forceinline__ uint32_t cm_off(int row, int k, int Kb) {
  return row_off(row, Kb) + (k >> 3) * 128 + (k & 7) * 2;
}

template <class OP>
__device__ __forceinline__ uint16_t to16(float v) {
  return (uint16_t)(OP::pack(v, 0.f) & 0xFFFFu);
}

// The reference matrix [Vxi | Veta (| V)] in the core-matrix image of the
// kernel's A operand: row j = (m, n) per CTA, columns c Nq_pad + q with q = (a, b);
// products of the one-dimensional tables in FP32, rounded to 16 bits.
template <class OP>
__global__ void __launch_bounds__(128) build_reference(const double* __restrict__ tables, int Q, int T, int Nqb,
                                                       int K1, uint16_t* __restrict__ out) {
  const int j = blockIdx.x, Nt = T * T, Nq = Q * Q;
  const double* w = tables + Q;
  const double* v = w + Q;
  const double* dv = v + T * Q;
  const bool jv = j < Nt;
  const int m = jv ? j / T : 0, n = jv ? j - m * T : 0;
  for (int k = threadIdx.x; k < K1; k += blockDim.x) {
    const int c = k / Nqb, q = k - c * Nqb;
    float val = 0.f;
    if (jv && q < Nq) {
      const int ia = q / Q, ib = q - ia * Q;
      const float r = c == 0 ? (float)dv[m * Q + ia] * (float)v[n * Q + ib]
                    : c == 1 ? (float)v[m * Q + ia] * (float)dv[n * Q + ib] : (float)v[m * Q + ia] * (float)v[n * Q + ib];
      val = ((float)w[ia] * (float)w[ib]) * r;
    }
    out[cm_off(j, k, K1) >> 1] = to16<OP>(val);
  }
}

template <class OP, int NC>
__global__ void __launch_bounds__(kRegThreads, 2) contract_regular_tc(RegArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const RegPlan& pl = a.pl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Q = a.Q, T = a.T, Nq = Q * Q, Nt = T * T, K1 = pl.K1, Nqb = pl.Nq_pad, Ntb = pl.Nt_blk, M2 = pl.M2;
  uint8_t* sA = sm + pl.o_A;
  uint8_t* sB1 = sm + pl.o_B1;
  uint8_t* sB2 = sm + pl.o_B2;
  float* sJ = reinterpret_cast<float*>(sm + pl.o_J);        // [128][3]
  uint32_t* s_max = reinterpret_cast<uint32_t*>(sm + pl.o_red);
  double* s_red = reinterpret_cast<double*>(sm + pl.o_red + 16);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + pl.o_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + pl.o_bar + 8);
  if (warp == 0) { tmem_alloc(s_tmem, pl.tmem_cols); tmem_relinquish(); }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the reference matrix, built once per mesh in its shared-memory image: 16-byte copies
  {
    const int n16 = Ntb * K1 * 2 / 16;
    for (int i = tid; i < n16; i += kRegThreads) reinterpret_cast<uint4*>(sA)[i] = a.ref[i];
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = *s_tmem;
  // D1 (diffusion residual A) at columns 0..127, the convection residual (three
  // components) at 384..511; D2_c at columns 128 c (D1 is dead by then)
  const uint32_t tD1 = tD, tD1c = tD + 3 * kRegTile, tD2 = tD;
  const float eps = (float)(a.eps_d ? *a.eps_d : a.eps_h);
  const float bx = (float)a.bx, by = (float)a.by, rscale = (float)a.rscale;
  uint32_t phase = 0;
  bool failed = false;
  double lsum = 0.0, dsum = 0.0;
  float smx = 0.f;                 // largest |seed| this thread wrote
  // TMEM lane quarter q4 of this warp and its half of the tile's elements (columns);
  // GEMM row of this thread: M = 128 -> row = lane 32 q4 + l; M = 64 -> row 16 q4 + l (l < 16)
  const int q4 = warp & 3, c_lo = (warp >> 2) * (kRegTile / 2), c_hi = c_lo + kRegTile / 2;
  const int row1 = Ntb == 128 ? q4 * 32 + lane : (lane < 16 ? q4 * 16 + lane : -1);
  const int row2 = M2 == 128 ? q4 * 32 + lane : (lane < 16 ? q4 * 16 + lane : -1);
  const uint32_t tRow = (uint32_t)(q4 * 32) << 16;
  const int n_tiles = (a.n_e + kRegTile - 1) / kRegTile;

  for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    const int e0 = tile * kRegTile;
    float lt = 0.f, dt = 0.f;            // this tile's loss and eps-derivative terms (FP32; FP64 across tiles)
    // ---- stage the scaled gradient field (B1) and the element scales; each warp takes
    //      four elements at a time and issues all their loads before converting
    for (int n0 = warp * 4; n0 < kRegTile; n0 += kRegThreads / 8) {
      float ux[4][4], uy[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t p0 = (int64_t)(e0 + n0 + t) * Nq;
        const bool ok_e = e0 + n0 + t < a.n_e;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int q = lane + 32 * r;
          const bool in = ok_e && q < Nq;
          ux[t][r] = in ? a.U[a.P_tot + p0 + q] : 0.f;
          uy[t][r] = in ? a.U[2 * a.P_tot + p0 + q] : 0.f;
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n = n0 + t, e = e0 + n;
        float jx = 0.f, jy = 0.f, jj = 0.f;    // y_eta = |J| / x_xi, x_xi, |J| on a rectangle
        if (e < a.n_e) { jx = a.J[3 * (size_t)e]; jy = a.J[3 * (size_t)e + 1]; jj = a.J[3 * (size_t)e + 2]; }
        if (lane == 0) { sJ[n * 3] = jx; sJ[n * 3 + 1] = jy; sJ[n * 3 + 2] = jj; }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int q = lane + 32 * r;
          if (q >= Nqb) continue;
          *reinterpret_cast<uint16_t*>(sB1 + cm_off(n, q, K1)) = to16<OP>(jx * ux[t][r]);
          *reinterpret_cast<uint16_t*>(sB1 + cm_off(n, Nqb + q, K1)) = to16<OP>(jy * uy[t][r]);
          if (NC == 3)
            *reinterpret_cast<uint16_t*>(sB1 + cm_off(n, 2 * Nqb + q, K1)) =
                to16<OP>(jj * (bx * ux[t][r] + by * uy[t][r]));
        }
      }
    }
    if (tid == 0) *s_max = 0u;
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- residual GEMM: D1 = A . B1 (M = Nt_blk, N = 128, K = K1)
    if (tid == 0) {
      tc_fence_after();
      const uint32_t id = idesc_f16(OP::fmt, Ntb, kRegTile, 0, 0);
      const int kd = 2 * Nqb / 16;                    // K steps of the two diffusion components
      for (int kk = 0; kk < K1 / 16; ++kk) {
        const uint64_t ad = sdesc(su32(sA) + kk * 256, 128, K1 * 16);
        const uint64_t bd = sdesc(su32(sB1) + kk * 256, 128, K1 * 16);
        if (kk < kd) mma_bf16(tD1, ad, bd, id, kk > 0);
        else mma_bf16(tD1c, ad, bd, id, kk > kd);
      }
      mma_commit(bar);
    }
    bool ok = mbar_wait(bar, phase);
    phase ^= 1;
    if (__syncthreads_or(!ok)) { failed = true; if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT); break; }
    tc_fence_after();
    // ---- epilogue 1: R = D1 - F^T, loss, max |Rbar| over the tile (pass A); 32 elements at a time,
    //      their F entries loaded together
    float rmax = 0.f;
    for (int c = c_lo; c < c_hi; c += 16) {
      float d[16], dc[16], fv[16];
      const bool rv = row1 >= 0 && row1 < Nt;
#pragma unroll
      for (int i = 0; i < 16; ++i) fv[i] = rv && e0 + c + i < a.n_e ? a.F[(size_t)(e0 + c + i) * Nt + row1] : 0.f;
#pragma unroll
      for (int i = 0; i < 16; i += 8) {
        tmem_ld8(tD1 + tRow + c + i, d + i);
        if (NC == 3) tmem_ld8(tD1c + tRow + c + i, dc + i);
      }
      tmem_wait_ld();
      if (rv) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int e = e0 + c + i;
          if (e < a.n_e) {
            const float R = fmaf(eps, d[i], (NC == 3 ? dc[i] : 0.f) - fv[i]);   // eps A + B - F
            lt = fmaf(R, R, lt);
            dt = fmaf(rscale * R, d[i], dt);                                       // Rbar A
            rmax = fmaxf(rmax, fabsf(rscale * R));
            if (a.R_out) a.R_out[(size_t)e * Nt + row1] = (double)R;
          }
        }
      }
    }
    atomicMax(s_max, __float_as_uint(rmax));
    __syncthreads();
    // power-of-two scale with max |Rbar| s <= 1 (exact)
    float sc = 1.f;
    {
      const float m = __uint_as_float(*s_max);
      if (m > 0.f && isfinite(m)) {
        int ex;
        frexpf(m, &ex);
        ex = max(-100, min(100, ex));
        sc = __int_as_float((127 - ex) << 23);
      }
    }
    // pass B: Rbar s into B2 (rows = elements, K = tests); invalid rows and columns are zero
    for (int c = c_lo; c < c_hi; c += 16) {
      float d[16], dc[16], fv[16];
      const bool rv = row1 >= 0 && row1 < Nt;
#pragma unroll
      for (int i = 0; i < 16; ++i) fv[i] = rv && e0 + c + i < a.n_e ? a.F[(size_t)(e0 + c + i) * Nt + row1] : 0.f;
#pragma unroll
      for (int i = 0; i < 16; i += 8) {
        tmem_ld8(tD1 + tRow + c + i, d + i);
        if (NC == 3) tmem_ld8(tD1c + tRow + c + i, dc + i);
      }
      tmem_wait_ld();
      if (row1 >= 0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int e = e0 + c + i;
          const float R = fmaf(eps, d[i], (NC == 3 ? dc[i] : 0.f) - fv[i]);
          const float rb = rv && e < a.n_e ? sc * rscale * R : 0.f;
          *reinterpret_cast<uint16_t*>(sB2 + cm_off(c + i, row1, Ntb)) = to16<OP>(rb);
        }
      }
    }
    if (!a.UB) {
      lsum += (double)lt;
      tc_fence_before();
      __syncthreads();
      continue;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ---- adjoint GEMMs: D2_c = V_c^T . Rbar (M = M2, N = 128, K = Nt_blk), A read MN-major
    if (tid == 0) {
      tc_fence_after();
      const uint32_t id = idesc_f16(OP::fmt, M2, kRegTile, 1, 0);
      for (int ks = 0; ks < Ntb / 16; ++ks)
        for (int cc = 0; cc < NC; ++cc) {
          const uint64_t ad = sdesc(su32(sA) + (cc * Nqb / 8) * 128 + ks * 2 * K1 * 16, K1 * 16, 128);
          const uint64_t bd = sdesc(su32(sB2) + ks * 256, 128, Ntb * 16);
          mma_bf16(tD2 + cc * kRegTile, ad, bd, id, ks > 0);
        }
      mma_commit(bar);
    }
    ok = mbar_wait(bar, phase);
    phase ^= 1;
    if (__syncthreads_or(!ok)) { failed = true; if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT); break; }
    tc_fence_after();
    // ---- epilogue 2: the seeds, 8 elements at a time
    const float inv = 1.f / sc;
    const bool qv = row2 >= 0 && row2 < Nq;
    for (int c = c_lo; c < c_hi; c += 8) {
      float dx[8], dy[8], dvv[8];
      tmem_ld8(tD2 + tRow + c, dx);
      tmem_ld8(tD2 + kRegTile + tRow + c, dy);
      if (NC == 3) tmem_ld8(tD2 + 2 * kRegTile + tRow + c, dvv);
      tmem_wait_ld();
      if (qv) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n = c + i, e = e0 + n;
          if (e >= a.n_e) continue;
          const float jx = sJ[n * 3], jy = sJ[n * 3 + 1], jj = sJ[n * 3 + 2];
          const float sx = dx[i] * inv, sy = dy[i] * inv, sv = NC == 3 ? dvv[i] * inv : 0.f;
          const int64_t p = (int64_t)e * Nq + row2;
          const float s1 = eps * jx * sx + bx * jj * sv, s2 = eps * jy * sy + by * jj * sv;
          a.UB[p] = 0.f;
          a.UB[a.P_tot + p] = s1;
          a.UB[2 * a.P_tot + p] = s2;
          smx = fmaxf(smx, fmaxf(fabsf(s1), fabsf(s2)));
        }
      }
    }
    lsum += (double)lt;
    dsum += (double)dt;
    tc_fence_before();
    __syncthreads();
  }
  warp_max_to(a.seed_max, smx);
  // loss and eps-derivative partials: per-thread sums, a fixed-order warp tree, warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  }
  if (lane == 0) { s_red[warp * 2] = lsum; s_red[warp * 2 + 1] = dsum; }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    double l = 0.0, d = 0.0;
    for (int w = 0; w < kRegThreads / 32; ++w) { l += s_red[w * 2]; d += s_red[w * 2 + 1]; }
    a.partials[2 * blockIdx.x] = failed ? 0.0 : l;
    a.partials[2 * blockIdx.x + 1] = failed ? 0.0 : d;
  }
  if (warp == 0) tmem_dealloc(tD, pl.tmem_cols);
}

template <class OP, int NC>
cudaError_t launch_reg(fv_ctx ctx, const RegArgs& a, int grid) {
  cudaError_t e = ensure_smem_attr(ctx, (const void*)contract_regular_tc<OP, NC>, a.pl.smem);
  if (e == cudaSuccess) contract_regular_tc<OP, NC><<<grid, kRegThreads, a.pl.smem, ctx->stream>>>(a);
  return e;
}

}  // namespace

bool regular_supported(fv_mesh m, fv_precision prec) {
  RegPlan p;
  return (prec == FV_BF16 || prec == FV_FP16) && make_reg_plan(m->Q, m->T, m->n_comp, &p);
}

int regular_grid(fv_ctx ctx, fv_mesh m) {
  const int n_tiles = (m->n_e + kRegTile - 1) / kRegTile;
  RegPlan p;
  const int per_sm = make_reg_plan(m->Q, m->T, m->n_comp, &p) && p.tmem_cols == 256 ? 2 : 1;
  return std::max(1, std::min(n_tiles, ctx->n_sm * per_sm));
}

// Every element an axis-aligned rectangle: x depends on xi only, y on eta only.
// Fills `scales` with each element's y_eta, x_xi and |J| = x_xi y_eta in FP32.
int check_regular_mesh(fv_mesh m, std::vector<float>* scales) {
  std::vector<double> v(2 * (size_t)m->n_v);
  std::vector<int> c(4 * (size_t)m->n_e);
  cudaError_t e = cudaMemcpy(v.data(), m->verts, v.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(c.data(), m->cells, c.size() * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error("fv_mesh_set_g_mode: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  for (int k = 0; k < m->n_e; ++k) {
    double vx[4], vy[4];
    for (int i = 0; i < 4; ++i) { vx[i] = v[2 * c[4 * k + i]]; vy[i] = v[2 * c[4 * k + i] + 1]; }
    const double x1 = 0.25 * (-vx[0] + vx[1] + vx[2] - vx[3]), x2 = 0.25 * (-vx[0] - vx[1] + vx[2] + vx[3]);
    const double x3 = 0.25 * (vx[0] - vx[1] + vx[2] - vx[3]);
    const double y1 = 0.25 * (-vy[0] + vy[1] + vy[2] - vy[3]), y2 = 0.25 * (-vy[0] - vy[1] + vy[2] + vy[3]);
    const double y3 = 0.25 * (vy[0] - vy[1] + vy[2] - vy[3]);
    const double scale = std::fabs(x1) + std::fabs(y2);
    if (std::fabs(x2) + std::fabs(x3) + std::fabs(y1) + std::fabs(y3) > 1e-12 * scale) {
      set_error("fv_mesh_set_g_mode: element %d is not an axis-aligned rectangle (Alg. 2 needs a constant, "
                "diagonal Jacobian)", k);
      return FV_ERR_ARG;
    }
    if (scales) {
      scales->push_back((float)y2);
      scales->push_back((float)x1);
      scales->push_back((float)(x1 * y2));
    }
  }
  return FV_OK;
}

// The FP16 and BF16 images of the reference matrix for this mesh's orders
// (nothing to build where the GEMM form does not apply).
int build_regular_reference(fv_mesh m) {
  RegPlan p;
  if (!make_reg_plan(m->Q, m->T, m->n_comp, &p)) return FV_OK;
  const size_t bytes = (size_t)p.Nt_blk * p.K1 * 2;
  for (int img = 0; img < 2; ++img) {
    if (!m->reg_ref[img]) {
      const cudaError_t e = cudaMalloc(&m->reg_ref[img], bytes);
      if (e != cudaSuccess) {
        set_error("fv_mesh_set_g_mode: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA;
      }
    }
    uint16_t* out = static_cast<uint16_t*>(m->reg_ref[img]);
    if (img == 0) build_reference<OpF16><<<p.Nt_blk, 128, 0, m->ctx->stream>>>(m->tables, m->Q, m->T, p.Nq_pad, p.K1, out);
    else build_reference<OpBF16><<<p.Nt_blk, 128, 0, m->ctx->stream>>>(m->tables, m->Q, m->T, p.Nq_pad, p.K1, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("fv_mesh_set_g_mode: reference build failed: %s", cudaGetErrorString(e));
      return FV_ERR_CUDA;
    }
  }
  const cudaError_t e = cudaStreamSynchronize(m->ctx->stream);
  if (e != cudaSuccess) {
    set_error("fv_mesh_set_g_mode: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

int launch_contract_regular(fv_ctx ctx, fv_mesh m, fv_forcing f, const EvalPlan& pl, const void* U, void* UB,
                            double eps, const double* eps_dev, double bx, double by, double rscale,
                            double* partials, int* n_part, double* R_out) {
  RegArgs a;
  if (!make_reg_plan(m->Q, m->T, m->n_comp, &a.pl)) {
    set_error("regular-mesh contraction: Q = %d, T = %d outside Q*Q, T*T <= 128", m->Q, m->T);
    return FV_ERR_UNSUPPORTED;
  }
  if (!m->jreg) {
    set_error("regular-mesh contraction: the mesh has no element scales (set FV_G_REGULAR first)");
    return FV_ERR_ARG;
  }
  const int img = pl.prec == FV_FP16 ? 0 : 1;
  if (!m->reg_ref[img]) {
    set_error("regular-mesh contraction: the mesh has no reference matrix (set FV_G_REGULAR first)");
    return FV_ERR_ARG;
  }
  a.J = m->jreg; a.tables = m->tables; a.ref = static_cast<const uint4*>(m->reg_ref[img]);
  a.n_e = m->n_e; a.Q = m->Q; a.T = m->T;
  a.F = f->F32;
  a.U = static_cast<const float*>(U); a.UB = static_cast<float*>(UB); a.P_tot = pl.P_tot;
  a.eps_h = eps; a.eps_d = eps_dev; a.bx = bx; a.by = by; a.rscale = rscale;
  a.partials = partials; a.R_out = R_out; a.err = ctx->err_dev; a.seed_max = pl.seed_max;
  const int grid = regular_grid(ctx, m);
  *n_part = grid;
  cudaEvent_t ta;
  time_begin(ctx, K_CONTRACT, &ta);
  cudaError_t e;
  if (pl.prec == FV_FP16)
    e = m->n_comp == 3 ? launch_reg<OpF16, 3>(ctx, a, grid) : launch_reg<OpF16, 2>(ctx, a, grid);
  else
    e = m->n_comp == 3 ? launch_reg<OpBF16, 3>(ctx, a, grid) : launch_reg<OpBF16, 2>(ctx, a, grid);
  if (e == cudaSuccess) e = cudaGetLastError();
  time_end(ctx, K_CONTRACT, ta);
  if (e != cudaSuccess) {
    set_error("regular-mesh contraction launch failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

}  // namespace fv
