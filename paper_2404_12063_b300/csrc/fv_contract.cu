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
// on an mbarrier), then runs the row pass (residuals; one row per lane group,
// vector loads of G and grad u) and the column pass (adjoint seeds; one
// q-chunk per lane group) on the same shared tile.
#include <algorithm>
#include <vector>
#include <cmath>
#include <type_traits>

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

// G is streamed once per evaluation: its lines are the first the L2 evicts,
// so that data the neighbouring kernels keep there (written activations
// still to be drained, u and its gradient) stays.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
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
  int sh1, sh2, nq_pad;  // staged kernel: log2 of the row-pass and column-pass splits, padded aux row
  double* partials;     // [gridDim][2]
  int* err;
  double* R_out;        // optional [n_e][Nt] element residuals
  float* seed_max;      // optional: raised to max |seed| (FP16 reverse sweep)
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

// Per-stage auxiliary data: u_x, u_y of the stage's points (each element's
// row padded to nq_pad values so that every q-chunk is vector aligned) and
// its F rows.
template <class R>
struct Aux {
  R* ux;
  R* uy;
  R* F;
};

constexpr int kCThreads = 128;                      // staged kernel: 4 warps, several CTAs per SM
constexpr int kCWarps = kCThreads / 32;

__host__ __device__ inline size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

// Values per element row of the staged u_x / u_y: N_q rounded up to the
// vector width (at least 4), so that every q-chunk load is aligned.
__host__ __device__ inline int aux_row(int Nq, int vec) {
  const int a = vec > 4 ? vec : 4;
  return (Nq + a - 1) / a * a;
}

// Shared-memory layout of the staged kernel (offsets in bytes); host and
// device evaluate the same function.
struct StagedLayout {
  size_t aux_n;            // R values per aux buffer
  size_t rb, red, bar, stage, total;
};
__host__ __device__ inline StagedLayout staged_layout(int Eg, int Nt, int nqp, int S, size_t stage_bytes,
                                                      size_t rsz) {
  StagedLayout L;
  const int ntp = (Nt + 7) & ~7;
  L.aux_n = (size_t)2 * Eg * nqp + (size_t)Eg * ntp;
  L.rb = round16(2 * L.aux_n * rsz);                  // two aux buffers at offset 0
  L.red = L.rb + round16((size_t)Eg * Nt * rsz);      // Rbar of the stage's rows
  L.bar = L.red + round16(kCWarps * 4 * 8);           // per-warp loss partials
  L.stage = L.bar + round16((size_t)S * 8);           // one barrier per stage; bulk copies land 16-byte aligned
  L.total = L.stage + (size_t)S * stage_bytes;
  return L;
}

// VEC consecutive values read from shared memory as one aligned access.
template <class T, int VEC>
struct alignas(sizeof(T) * VEC) VecT {
  T v[VEC];
};

template <class R, class T, int VEC>
__device__ __forceinline__ void lds_vec(const T* p, R (&out)[VEC]) {
  const VecT<T, VEC> t = *reinterpret_cast<const VecT<T, VEC>*>(p);
#pragma unroll
  for (int v = 0; v < VEC; ++v) out[v] = (R)t.v[v];
}

// BF16 -> FP32 is exact: the BF16 bits are the upper half of the FP32 word.
// Value 2i of a packed run sits in the low half of 32-bit word i.
template <int VEC>
__device__ __forceinline__ void lds_bf16(const __nv_bfloat16* p, float (&out)[VEC]) {
  if constexpr (VEC == 1) {
    out[0] = __uint_as_float((uint32_t)*reinterpret_cast<const unsigned short*>(p) << 16);
  } else {
    constexpr int W = VEC / 2;
    const VecT<uint32_t, W> t = *reinterpret_cast<const VecT<uint32_t, W>*>(p);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      out[2 * i] = __uint_as_float(t.v[i] << 16);
      out[2 * i + 1] = __uint_as_float(t.v[i] & 0xffff0000u);
    }
  }
}

// VEC values of G from shared memory, in the evaluation precision R.
template <class R, class Gt, int VEC>
__device__ __forceinline__ void gload(const Gt* p, R (&out)[VEC]) {
  if constexpr (std::is_same<Gt, __nv_bfloat16>::value) lds_bf16<VEC>(p, out);
  else lds_vec<R, Gt, VEC>(p, out);
}

// acc[v] += a[v] * b[v], v < VEC.  In FP32 adjacent lanes go through the
// packed FP32x2 FMA (two independent round-to-nearest FMAs per instruction).
template <int VEC>
__device__ __forceinline__ void fma_vec(float (&acc)[VEC], const float (&a)[VEC], const float (&b)[VEC]) {
  if constexpr (VEC % 2 == 0) {
#pragma unroll
    for (int i = 0; i < VEC; i += 2) {
      const float2 r = __ffma2_rn(make_float2(a[i], a[i + 1]), make_float2(b[i], b[i + 1]),
                                  make_float2(acc[i], acc[i + 1]));
      acc[i] = r.x;
      acc[i + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc[i] += a[i] * b[i];
  }
}
template <int VEC>
__device__ __forceinline__ void fma_vec(double (&acc)[VEC], const double (&a)[VEC], const double (&b)[VEC]) {
#pragma unroll
  for (int i = 0; i < VEC; ++i) acc[i] += a[i] * b[i];
}

// sum of acc[0..VEC) as a pairwise tree
template <class R, int VEC>
__device__ __forceinline__ R tree_sum(const R (&acc)[VEC]) {
  if constexpr (VEC == 1) {
    return acc[0];
  } else {
    R t[VEC / 2 + VEC % 2];
#pragma unroll
    for (int i = 0; i < VEC / 2; ++i) t[i] = acc[2 * i] + acc[2 * i + 1];
    if constexpr (VEC % 2) t[VEC / 2] = acc[VEC - 1];
    return tree_sum<R, VEC / 2 + VEC % 2>(t);
  }
}

// One CTA of 128 threads streams element groups through a ring of S shared
// stages (cp.async.bulk completing on an mbarrier per stage); several CTAs
// share an SM so that one CTA's copies overlap the others' arithmetic.  Each
// staged group is read twice from shared memory, never again from HBM:
//   pass 1 (residuals): a task is (row (e, j), split h of the row's
//     q-chunks).  Lane = h * (32 / H1) + r, so the lanes of one shared-memory
//     wavefront read consecutive rows at the same chunk (distinct banks when
//     the row length in chunks is odd; SKEW rotates each lane's chunk order
//     otherwise).  The H1 splits meet by shuffles.
//   pass 2 (seeds): a task is (element, q-chunk c, split h of the test rows
//     taken interleaved j = h, h + H2, ...); the H2 splits sit in adjacent
//     lanes and meet by shuffles.
// Every sum has a fixed order, so results are bitwise reproducible.
// NC = 2 (diffusion only) or 3 (with the convection/mass component); VEC
// divides Nq.  CNCH, CNT, CSH1, CSH2 fix the chunks per row, the test count
// and the two split exponents at compile time for common element shapes
// (0 / -1: taken from the arguments).
template <class R, class Gt, int NC, int VEC, bool SKEW, int CNCH = 0, int CNT = 0, int CSH1 = -1, int CSH2 = -1>
__global__ void __launch_bounds__(kCThreads) contract_staged(ContractArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nt = CNT ? CNT : a.Nt, Nq = CNCH ? CNCH * VEC : a.Nq, Eg = a.elems_per_stage, S = a.n_stages;
  const int sh1 = CSH1 >= 0 ? CSH1 : a.sh1, sh2 = CSH2 >= 0 ? CSH2 : a.sh2, H1 = 1 << sh1, H2 = 1 << sh2;
  const int nqp = CNCH ? aux_row(CNCH * VEC, VEC) : a.nq_pad;
  const int lg_rpw = 5 - sh1;                         // rows per warp and round: 32 / H1
  const int nch = Nq / VEC;
  const size_t stage_bytes = (size_t)Eg * a.g_stride_bytes;
  const StagedLayout L = staged_layout(Eg, Nt, nqp, S, stage_bytes, sizeof(R));
  R* aux_base = reinterpret_cast<R*>(smem);
  R* s_rb = reinterpret_cast<R*>(smem + L.rb);
  double* s_red = reinterpret_cast<double*>(smem + L.red);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar);
  unsigned char* stages = smem + L.stage;
  auto aux_of = [&](int b) {
    Aux<R> x;
    x.ux = aux_base + b * L.aux_n;
    x.uy = x.ux + Eg * nqp;
    x.F = x.uy + Eg * nqp;
    return x;
  };

  const R eps = (R)(a.eps_d ? *a.eps_d : a.eps_h);
  const R bx = (R)a.bx, by = (R)a.by, rscale = (R)a.rscale;
  const R* U = reinterpret_cast<const R*>(a.U);
  const R* Fsrc = reinterpret_cast<const R*>(a.Fr);
  R* UB = reinterpret_cast<R*>(a.UB);
  const unsigned char* Gb = reinterpret_cast<const unsigned char*>(a.G);
  const int gstride = (int)(a.g_stride_bytes / (int64_t)sizeof(Gt));
  const int plane = Nt * Nq;                          // values per component of one element

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
      for (int i = tid; i < ne * Nq; i += kCThreads) {
        const int k = i / Nq, q = i - k * Nq;
        cp_async_r<R>(x.ux + k * nqp + q, U + a.P_tot + p0 + i);
        cp_async_r<R>(x.uy + k * nqp + q, U + 2 * a.P_tot + p0 + i);
      }
      for (int i = tid; i < ne * Nt; i += kCThreads) cp_async_r<R>(x.F + i, Fsrc + (size_t)e0 * Nt + i);
    }
    cp_async_commit();
  };
  if (tid == 0)
    for (int it = 0; it < S; ++it) issue(it);
  prefetch_aux(0);

  // rounds of each pass: uniform over the CTA (whole warps take part in the shuffles)
  const int n1 = (Eg * Nt * H1 + kCThreads - 1) / kCThreads;
  const int n2 = (Eg * nch * H2 + kCThreads - 1) / kCThreads;
  KahanR<R> lsum, dsum;
  float smx = 0.f;                 // largest |seed| this thread wrote
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
    const int n_rows = ne * Nt;

    // pass 1: residual of every (element, test) row
    for (int r1 = 0; r1 < n1; ++r1) {
      const int row = ((r1 * kCWarps + warp) << lg_rpw) + (lane & ((1 << lg_rpw) - 1));
      const int h = lane >> lg_rpw;
      const bool valid = row < n_rows;
      R Ax = 0, Ay = 0, Bx = 0, By = 0;
      if (valid) {
        const int k = row / Nt, j = row - k * Nt;
        const int cb = (h * nch) >> sh1, n = (((h + 1) * nch) >> sh1) - cb;
        const Gt* px = tile + k * gstride + j * Nq + cb * VEC;
        const R* pu = x.ux + k * nqp + cb * VEC;
        const R* pw = pu + Eg * nqp;
        R ax[VEC], ay[VEC], bxa[VEC], bya[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) ax[v] = ay[v] = bxa[v] = bya[v] = (R)0;
        int c = SKEW ? row % n : 0;
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
          const int o = SKEW ? c * VEC : i * VEC;
          R vx[VEC], vy[VEC], wx[VEC], wy[VEC];
          gload<R, Gt, VEC>(px + o, vx);
          gload<R, Gt, VEC>(px + plane + o, vy);
          lds_vec<R, R, VEC>(pu + o, wx);
          lds_vec<R, R, VEC>(pw + o, wy);
          fma_vec<VEC>(ax, vx, wx);
          fma_vec<VEC>(ay, vy, wy);
          if (NC == 3) {
            R vv[VEC];
            gload<R, Gt, VEC>(px + 2 * plane + o, vv);
            fma_vec<VEC>(bxa, vv, wx);
            fma_vec<VEC>(bya, vv, wy);
          }
          if (SKEW) c = c + 1 == n ? 0 : c + 1;
        }
        Ax = tree_sum<R, VEC>(ax);
        Ay = tree_sum<R, VEC>(ay);
        if (NC == 3) {
          Bx = tree_sum<R, VEC>(bxa);
          By = tree_sum<R, VEC>(bya);
        }
      }
      for (int o = 16; o >= (1 << lg_rpw); o >>= 1) {
        Ax += __shfl_xor_sync(0xffffffffu, Ax, o);
        Ay += __shfl_xor_sync(0xffffffffu, Ay, o);
        if (NC == 3) {
          Bx += __shfl_xor_sync(0xffffffffu, Bx, o);
          By += __shfl_xor_sync(0xffffffffu, By, o);
        }
      }
      if (valid && h == 0) {
        const R A = Ax + Ay;
        const R Rv = eps * A + (NC == 3 ? bx * Bx + by * By : (R)0) - x.F[row];
        const R Rb = rscale * Rv;
        s_rb[row] = Rb;
        lsum.add(Rv * Rv);
        dsum.add(Rb * A);
        if (a.R_out) a.R_out[(size_t)e0 * Nt + row] = (double)Rv;
      }
    }
    __syncthreads();
    // pass 2: seeds dL/du = 0, dL/du_x = eps sum_j Rbar Gx + bx sum_j Rbar Gv, likewise y
    if (UB) {
      for (int r2 = 0; r2 < n2; ++r2) {
        const int task = r2 * kCThreads + tid;
        const int h = task & (H2 - 1), cc = task >> sh2;
        const int k = cc / nch, c = cc - k * nch;
        const bool valid = k < ne;
        R sx[VEC], sy[VEC], sv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) sx[v] = sy[v] = sv[v] = (R)0;
        if (valid) {
          const Gt* px = tile + k * gstride + h * Nq + c * VEC;
          const R* pr = s_rb + k * Nt + h;
          const int gstep = Nq << sh2;
          const int n = (Nt - h + H2 - 1) >> sh2;
#pragma unroll 4
          for (int i = 0; i < n; ++i) {
            const R r = pr[i << sh2];
            R rr[VEC], vx[VEC], vy[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) rr[v] = r;
            gload<R, Gt, VEC>(px + i * gstep, vx);
            gload<R, Gt, VEC>(px + plane + i * gstep, vy);
            fma_vec<VEC>(sx, rr, vx);
            fma_vec<VEC>(sy, rr, vy);
            if (NC == 3) {
              R vv[VEC];
              gload<R, Gt, VEC>(px + 2 * plane + i * gstep, vv);
              fma_vec<VEC>(sv, rr, vv);
            }
          }
        }
        for (int o = 1; o < H2; o <<= 1) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            sx[v] += __shfl_xor_sync(0xffffffffu, sx[v], o);
            sy[v] += __shfl_xor_sync(0xffffffffu, sy[v], o);
            if (NC == 3) sv[v] += __shfl_xor_sync(0xffffffffu, sv[v], o);
          }
        }
        if (valid && h == 0) {
          const int64_t p = (int64_t)(e0 + k) * Nq + c * VEC;
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const R s1 = eps * sx[v] + bx * sv[v], s2 = eps * sy[v] + by * sv[v];
            UB[p + v] = (R)0;
            UB[a.P_tot + p + v] = s1;
            UB[2 * a.P_tot + p + v] = s2;
            smx = fmaxf(smx, fmaxf(fabsf((float)s1), fabsf((float)s2)));
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0) issue(it + S);
  }
  cp_async_wait0();
  warp_max_to(a.seed_max, smx);
  // loss partials: per-thread compensated sums, then a fixed-order tree in FP64
  double l = (double)lsum.s - (double)lsum.c, d = (double)dsum.s - (double)dsum.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if (lane == 0) {
    s_red[warp * 2] = l;
    s_red[warp * 2 + 1] = d;
  }
  __syncthreads();
  if (tid == 0) {
    double ls = 0.0, ds = 0.0;
    for (int w = 0; w < kCWarps; ++w) {
      ls += s_red[w * 2];
      ds += s_red[w * 2 + 1];
    }
    a.partials[2 * blockIdx.x] = ls;
    a.partials[2 * blockIdx.x + 1] = ds;
  }
}

// Fallback for element blocks too large for a shared-memory stage: one CTA per
// element, G read straight from global memory in both passes.
template <class R, class Gt>
__global__ void __launch_bounds__(kThreads) contract_direct(ContractArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  double* s_R = reinterpret_cast<double*>(smem);     // [Nt]
  double* s_red = s_R + a.Nt;                         // [kWarps][4]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Nt = a.Nt, Nq = a.Nq;
  const double eps = a.eps_d ? *a.eps_d : a.eps_h;
  const R* U = reinterpret_cast<const R*>(a.U);
  R* UB = reinterpret_cast<R*>(a.UB);
  const int64_t gstride = a.g_stride_bytes / (int64_t)sizeof(Gt);
  KSum lsum, dsum;
  float smx = 0.f;
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
        const R s1 = (R)eps * sx + (R)a.bx * sv, s2 = (R)eps * sy + (R)a.by * sv;
        UB[p] = (R)0;
        UB[a.P_tot + p] = s1;
        UB[2 * a.P_tot + p] = s2;
        smx = fmaxf(smx, fmaxf(fabsf((float)s1), fabsf((float)s2)));
      }
    }
    __syncthreads();
  }
  warp_max_to(a.seed_max, smx);
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

template <class R, class Gt, int NC, int VEC, bool SKEW, int... Shape>
cudaError_t launch_staged1(fv_ctx ctx, const ContractArgs& a, int grid, size_t smem) {
  auto kern = contract_staged<R, Gt, NC, VEC, SKEW, Shape...>;
  cudaError_t e = ensure_smem_attr(ctx, (const void*)kern, smem);
  if (e == cudaSuccess) kern<<<grid, kCThreads, smem, ctx->stream>>>(a);
  return e;
}

// Compile-time element shapes: (chunks per row, tests, split exponents) of
// the Q = 10, T = 8 element with 4-wide chunks, as the planner splits it.
template <class R, class Gt, int NC, int VEC>
cudaError_t launch_staged(fv_ctx ctx, const ContractArgs& a, bool skew, int grid, size_t smem) {
  if (skew) return launch_staged1<R, Gt, NC, VEC, true>(ctx, a, grid, smem);
  if constexpr (VEC == 4 && NC == 2) {
    if (a.Nq == 100 && a.Nt == 64 && a.sh1 == 1 && a.sh2 == 2)
      return launch_staged1<R, Gt, NC, VEC, false, 25, 64, 1, 2>(ctx, a, grid, smem);
  }
  return launch_staged1<R, Gt, NC, VEC, false>(ctx, a, grid, smem);
}

template <class R, class Gt, int NC>
cudaError_t launch_staged_vec(fv_ctx ctx, const ContractArgs& a, int vec, bool skew, int grid, size_t smem) {
  switch (vec) {
    case 8: if constexpr (sizeof(Gt) * 8 <= 16) return launch_staged<R, Gt, NC, 8>(ctx, a, skew, grid, smem); break;
    case 4: if constexpr (sizeof(Gt) * 4 <= 16) return launch_staged<R, Gt, NC, 4>(ctx, a, skew, grid, smem); break;
    case 2: return launch_staged<R, Gt, NC, 2>(ctx, a, skew, grid, smem);
    default: break;
  }
  return launch_staged<R, Gt, NC, 1>(ctx, a, skew, grid, smem);
}

template <class R, class Gt>
int launch_t(fv_ctx ctx, const ContractArgs& a, bool staged, int vec, bool skew, int grid, size_t smem) {
  cudaError_t e;
  if (staged) {
    e = a.n_comp == 3 ? launch_staged_vec<R, Gt, 3>(ctx, a, vec, skew, grid, smem)
                      : launch_staged_vec<R, Gt, 2>(ctx, a, vec, skew, grid, smem);
  } else {
    e = ensure_smem_attr(ctx, (const void*)contract_direct<R, Gt>, smem);
    if (e == cudaSuccess) contract_direct<R, Gt><<<grid, kThreads, smem, ctx->stream>>>(a);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("contraction launch failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

// Launch geometry of the contraction.
struct ContractPlan {
  bool staged = false, skew = false;
  int vec = 1, E = 0, S = 0, sh1 = 0, sh2 = 0, nqp = 0, grid = 0;
  size_t smem = 0;
};

size_t g_value_bytes(fv_precision storage) {
  return storage == FV_FP64 ? 8 : storage == FV_BF16 ? 2 : 4;
}

int gcd_int(int a, int b) { return b ? gcd_int(b, a % b) : a; }

// Staged plan: the vector width is the widest shared-memory access (at most
// 16 bytes of G) whose width divides Nq.  Elements per stage E and the two
// split factors minimise a per-element cost model counted in CTA-wide vector
// steps (idle lanes included), preferring E small enough that four CTAs
// share an SM.  Stages per CTA: double-buffered by default; one stage with up
// to eight CTAs per SM where autotuning found that faster for the mesh, or
// where an element block is too large for two stages.  The row pass rotates each lane's
// chunk order when the row length in chunks shares a factor with the number
// of lanes that one shared-memory wavefront serves.
ContractPlan plan_contract(fv_ctx ctx, fv_mesh m, fv_precision prec, int stages = 0, int elems = 0) {
  ContractPlan P;
  const size_t rsz = prec == FV_FP64 ? 8 : 4;
  const size_t gsz = g_value_bytes(m->storage);
  const size_t gs = m->g_stride_bytes;
  int vec = 1;
  for (int v = 8; v >= 2; v >>= 1)
    if (v * gsz <= 16 && m->Nq % v == 0) { vec = v; break; }
  const int nch = m->Nq / vec;
  const int nqp = aux_row(m->Nq, vec);
  const int wave_lanes = (int)std::min<size_t>(32, std::max<size_t>(1, 128 / (vec * gsz)));
  const int slot = prec == FV_FP64 ? 1 : 0;
  const int tuned = m->contract_stages[slot];
  const int S = stages ? stages : tuned ? tuned : 2;
  const int Ef = stages ? elems : m->contract_elems[slot];     // forced elements per stage (0: by the model)
  const size_t max_ctas = S == 1 ? 8 : 4;
  double best = 1e300;
  for (int E = 1; E <= 16 && E <= m->n_e; ++E) {
    const StagedLayout L = staged_layout(E, m->Nt, nqp, S, E * gs, rsz);
    if (L.total > ctx->smem_optin || E * gs > (1u << 20) - 16) break;
    const int C = (int)std::min<size_t>(max_ctas, ctx->smem_per_sm / (L.total + 1024));
    if (C < 1) break;
    if (Ef && E != Ef) continue;
    double c1 = 1e300, c2 = 1e300;
    int s1 = 0, s2 = 0;
    for (int sh = 0; sh <= 3 && (1 << sh) <= nch; ++sh) {
      const int H = 1 << sh;
      const double rounds = std::ceil((double)E * m->Nt * H / kCThreads);
      const double c = rounds * (std::ceil((double)nch / H) + 2.0 * sh);
      if (c < c1) { c1 = c; s1 = sh; }
    }
    for (int sh = 0; sh <= 4 && (1 << sh) <= m->Nt; ++sh) {
      const int H = 1 << sh;
      const double rounds = std::ceil((double)E * nch * H / kCThreads);
      const double c = rounds * (std::ceil((double)m->Nt / H) + 0.5 * sh * vec);
      if (c < c2) { c2 = c; s2 = sh; }
    }
    const double occ = C >= 4 ? 1.0 : C == 3 ? 1.1 : C == 2 ? 1.3 : 2.0;
    const double cost = (c1 + c2) / E * occ;
    if (cost < best) {
      best = cost;
      P.staged = true; P.vec = vec; P.E = E; P.S = S; P.sh1 = s1; P.sh2 = s2; P.nqp = nqp; P.smem = L.total;
      P.skew = gcd_int(nch, wave_lanes) > 1;
      P.grid = std::min<int>((m->n_e + E - 1) / E, ctx->n_sm * C);
    }
  }
  if (!P.staged && S == 2 && !stages) return plan_contract(ctx, m, prec, 1, Ef);   // one stage per CTA
  if (!P.staged) {        // an element too large to stage: direct kernel
    P.smem = (size_t)m->Nt * 8 + kWarps * 4 * 8;
    P.grid = (int)std::min<int64_t>(m->n_e, (int64_t)ctx->n_sm * 8);
  }
  return P;
}

}  // namespace

int contract_grid(fv_ctx ctx, fv_mesh m, fv_precision prec, int* grid, int* eg, int* stages, size_t* smem,
                  bool matrix_free) {
  if (!matrix_free && m->g_mode == FV_G_REGULAR && regular_supported(m, prec)) {
    *grid = regular_grid(ctx, m);
    *eg = 0; *stages = 0; *smem = 0;
    return FV_OK;
  }
  if (matrix_free || m->g_mode != FV_G_STORED) {
    int wpb;
    mfree_grid(ctx, m, prec, grid, &wpb, smem);
    *eg = 0; *stages = 0;
    return FV_OK;
  }
  const ContractPlan P = plan_contract(ctx, m, prec);
  *grid = P.grid; *eg = P.E; *stages = P.S; *smem = P.smem;
  return FV_OK;
}

// Times candidate plans on zero-valued inputs (median of seven launches after
// two warm-up launches each) and keeps the fastest: one and two stages per CTA,
// each with the cost model's elements per stage and with 1 to 4 elements.
int autotune_contract(fv_ctx ctx, fv_mesh m, fv_precision prec, double* ms_out) {
  const int slot = prec == FV_FP64 ? 1 : 0;
  const size_t rsz = prec == FV_FP64 ? 8 : 4;
  if (ms_out) ms_out[0] = ms_out[1] = 0.0;
  if (m->g_mode != FV_G_STORED) return FV_OK;
  struct Cand { int S, E, grid; };
  std::vector<Cand> cands;
  for (int S = 2; S >= 1; --S)
    for (int E = 0; E <= 4; ++E) {
      const ContractPlan p = plan_contract(ctx, m, prec, S, E);
      if (!p.staged || p.S != S) continue;
      bool dup = false;
      for (const Cand& c : cands) dup |= c.S == S && c.E == p.E;
      if (!dup) cands.push_back({S, p.E, p.grid});
    }
  if (cands.size() < 2) return FV_OK;   // nothing to choose
  EvalPlan pl;
  pl.prec = prec;
  pl.P_mesh = pl.P_tot = m->P;
  pl.shape.L = 1;                       // a one-output network: scalar eps
  pl.shape.w[0] = 2;
  pl.shape.w[1] = 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  int max_grid = 1;
  for (const Cand& c : cands) max_grid = std::max(max_grid, c.grid);
  const size_t u_bytes = 3 * (size_t)m->P * rsz, nf = (size_t)m->n_e * m->Nt;
  const size_t o_ub = al(u_bytes), o_f = o_ub + al(u_bytes), o_f32 = o_f + al(nf * 8), o_part = o_f32 + al(nf * 4);
  const size_t total = o_part + al((size_t)max_grid * 16);
  char* buf = nullptr;
  if (cudaMalloc(&buf, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("autotune: cannot allocate %zu bytes of scratch", total);
    return FV_ERR_OOM;
  }
  fv_forcing_s fz;
  fz.mesh = m;
  fz.F = reinterpret_cast<double*>(buf + o_f);
  fz.F32 = reinterpret_cast<float*>(buf + o_f32);
  double* part = reinterpret_cast<double*>(buf + o_part);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FV_OK;
  auto fail = [&](cudaError_t e) {
    set_error("autotune: %s", cudaGetErrorString(e));
    rc = FV_ERR_CUDA;
  };
  cudaError_t ce = cudaMemsetAsync(buf, 0, total, ctx->stream);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) fail(ce);
  const int saved_s = m->contract_stages[slot], saved_e = m->contract_elems[slot];
  const bool timing = ctx->timing;
  ctx->timing = false;
  double best_ms = 1e300, best_s[3] = {0.0, 1e300, 1e300};
  int best = -1;
  for (size_t k = 0; k < cands.size() && rc == FV_OK; ++k) {
    m->contract_stages[slot] = cands[k].S;
    m->contract_elems[slot] = cands[k].E;
    float t[7] = {0};
    int n_part = 0;
    for (int r = 0; r < 9 && rc == FV_OK; ++r) {
      if (r >= 2 && (ce = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) { fail(ce); break; }
      rc = launch_contract(ctx, m, &fz, pl, buf, buf + o_ub, 1.0, nullptr, 0.0, 0.0, 1.0, part, &n_part, nullptr);
      if (rc || r < 2) continue;
      if ((ce = cudaEventRecord(e1, ctx->stream)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess ||
          (ce = cudaEventElapsedTime(&t[r - 2], e0, e1)) != cudaSuccess)
        fail(ce);
    }
    if (rc == FV_OK) {
      std::sort(t, t + 7);
      const double ms = t[3];
      best_s[cands[k].S] = std::min(best_s[cands[k].S], ms);
      if (ms < best_ms) { best_ms = ms; best = (int)k; }
    }
  }
  ctx->timing = timing;
  if (rc == FV_OK && (ce = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) fail(ce);
  m->contract_stages[slot] = rc == FV_OK && best >= 0 ? cands[best].S : saved_s;
  m->contract_elems[slot] = rc == FV_OK && best >= 0 ? cands[best].E : saved_e;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (ms_out && rc == FV_OK) {
    ms_out[0] = best_s[2] < 1e300 ? best_s[2] : 0.0;
    ms_out[1] = best_s[1] < 1e300 ? best_s[1] : 0.0;
  }
  return rc;
}

int launch_contract(fv_ctx ctx, fv_mesh m, fv_forcing f, const EvalPlan& pl, const void* U, void* UB, double eps,
                    const double* eps_dev, double bx, double by, double rscale, double* partials, int* n_part,
                    double* R_out) {
  // eps(x, y) from a two-output network (Sec. 4.7.2) needs the per-node form of the matrix-free kernel
  const bool eps_field = pl.shape.w[pl.shape.L] == 2;
  // regular meshes (Alg. 2): tensor-core GEMMs in the 16-bit forms, otherwise the matrix-free kernel
  if (m->g_mode == FV_G_REGULAR && !eps_field && regular_supported(m, pl.prec))
    return launch_contract_regular(ctx, m, f, pl, U, UB, eps, eps_dev, bx, by, rscale, partials, n_part, R_out);
  if (m->g_mode != FV_G_STORED || eps_field)
    return launch_contract_mfree(ctx, m, f, pl, U, UB, eps, eps_dev, bx, by, rscale, partials, n_part, R_out);
  const ContractPlan P = plan_contract(ctx, m, pl.prec);
  ContractArgs a;
  a.G = m->G; a.g_stride_bytes = (int64_t)m->g_stride_bytes;
  a.n_e = m->n_e; a.Nt = m->Nt; a.Nq = m->Nq; a.n_comp = m->n_comp;
  a.F = f->F; a.Fr = pl.prec == FV_FP64 ? (const void*)f->F : (const void*)f->F32; a.U = U; a.UB = UB; a.P_tot = pl.P_tot;
  a.eps_h = eps; a.eps_d = eps_dev; a.bx = bx; a.by = by; a.rscale = rscale;
  a.elems_per_stage = P.E; a.n_stages = P.S; a.n_groups = P.staged ? (m->n_e + P.E - 1) / P.E : m->n_e;
  a.sh1 = P.sh1; a.sh2 = P.sh2; a.nq_pad = P.nqp;
  a.partials = partials; a.err = ctx->err_dev; a.R_out = R_out; a.seed_max = pl.seed_max;
  *n_part = P.grid;
  cudaEvent_t ta;
  time_begin(ctx, K_CONTRACT, &ta);
  int rc;
  if (pl.prec == FV_FP64) {
    if (m->storage != FV_FP64) { set_error("FP64 evaluation needs FP64 G storage"); return FV_ERR_UNSUPPORTED; }
    rc = launch_t<double, double>(ctx, a, P.staged, P.vec, P.skew, P.grid, P.smem);
  } else if (m->storage == FV_FP32) {
    rc = launch_t<float, float>(ctx, a, P.staged, P.vec, P.skew, P.grid, P.smem);
  } else if (m->storage == FV_BF16) {
    rc = launch_t<float, __nv_bfloat16>(ctx, a, P.staged, P.vec, P.skew, P.grid, P.smem);
  } else {
    rc = launch_t<float, double>(ctx, a, P.staged, P.vec, P.skew, P.grid, P.smem);
  }
  time_end(ctx, K_CONTRACT, ta);
  return rc;
}

}  // namespace fv
