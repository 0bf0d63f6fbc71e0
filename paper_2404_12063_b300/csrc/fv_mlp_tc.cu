// tanh-MLP forward with tangents and its reverse sweep on the 5th-generation
// tensor cores (tcgen05, BF16 or FP16 operands, FP32 accumulation in tensor
// memory).
// Same mathematics as the CUDA-core kernels (Sec. 2.2 Eq. NN; forward-mode
// tangents d/dx, d/dy; reverse sweep through the tanh rule):
//
//   forward  map i:  Z_s = H_{i-1,s} W_i^T (+ b_i on the value stream)   s in {value, d/dx, d/dy}
//            t = tanh z, t'_s = (1 - t^2) z'_s
//   reverse  map i:  Zbar from Tbar and (t, t'_x, t'_y) (tanh rule),
//            Wbar_i += sum_s Zbar_s^T H_{i-1,s}     (bias gradient from a ones column)
//            Tbar_{i-1,s} = Zbar_s W_i
//
// A CTA of 128 x (HP/16) threads handles tiles of 128 points: point p is row
// p of every GEMM tile and lane p of tensor memory; warps w, w+4, ... share
// TMEM lane quarter w and each takes one 16-column group of the tile.  All three
// GEMMs read the same shared-memory tiles: activations are stored once in the
// no-swizzle core-matrix layout (8 rows x 16 bytes) and addressed as K-major
// operands (forward, Tbar) or as MN-major operands (weight gradient, and W_i
// for Tbar).  Layer 0 (two inputs) and the output layer (one output) run on
// CUDA cores.  The bias of each hidden map rides in an extra weight column
// that multiplies a constant-1 activation column, so the tensor core adds it
// and the weight-gradient GEMM returns the bias gradient in that column.
// When the reverse sweep follows (3 or 4 hidden layers), the forward kernel
// also stores the hidden layers below the last hidden map per tile (the
// activation stash) and the reverse kernel reads them back instead of
// recomputing those maps.
#include <algorithm>

#include "fv_internal.cuh"
#include "fv_tcgen05.cuh"

namespace fv {
namespace {

using namespace fv::tc;

constexpr int kTile = 128;
// 128 x (HP/16) threads: thread (quarter q, group g, lane l) owns point
// p = 32 q + l (TMEM lane p) and the 16 columns [16 g, 16 g + 16).
template <int HP> constexpr int tc_threads() { return kTile * (HP / 16); }

inline int ru16(int v) { return (v + 15) & ~15; }

// ------------------------------------------------------------------ plan
struct TcPlan {
  int L;
  int w[kMaxLayers + 1];
  int off[kMaxLayers];
  int n_params;
  int WP[kMaxLayers];       // padded width of the output of hidden map i: ru16(w[i+1] + 1)
  int HP;                   // max WP (32 or 64)
  int o_w[kMaxLayers];      // byte offset of BF16 W_i (maps 1..L-2): [WP_i rows][WP_{i-1} cols], bias in col w_i
  int o_small;              // FP32: w0x[HP], w0y[HP], b0[HP], wL[HP], bL
  int o_buf[2];             // activation tiles (3 streams x 128 x HP BF16)
  int o_z;                  // adjoint tile (reverse kernel)
  int o_x;                  // layer-0 input tile (reverse kernel): 3 streams x 128 x 16
  int o_red;                // FP32 scratch [128][4] (output-layer partial sums)
  int o_bar;                // MMA mbarrier (8 B) + TMEM base (4 B) + flags (4 B) + two upcoming tile indices
                            // (8 B, forward) or the activation-load mbarrier (8 B, reverse) + a failure word
  int o_tab;                // per-map constants copied to shared memory (TcTab)
  int smem;
  int tmem_cols;
  int c_wbar[kMaxLayers];   // TMEM column of the weight-gradient accumulator of map i (reverse)
  int c_part;               // reverse: partial weight-gradient accumulator (HP columns), 0: none
  // Activation stash (networks of 3 or 4 hidden layers): H_j for j = stash_lo ..
  // L-3, the stored layers below the last hidden map, written per tile by the
  // forward kernel and read by the reverse kernel instead of recomputing maps
  // 1 .. L-3; slot_bytes per tile and layer (3 streams x 128 rows x HP columns).
  int n_stash, stash_lo, slot_bytes;
};

struct TcArgs {
  TcPlan pl;
  const float* params;
  const double* Xm;
  int64_t P_mesh;
  const double* Xe;
  int64_t P_tot;
  float* U;                 // [3][P_tot] (forward)
  const float* UB;          // [3][P_tot] seeds (reverse)
  double* gpart;            // [grid][n_params] (reverse)
  const float* seed_absmax; // device max |seed| (FP16 reverse sweep) or null
  int* tile_ctr;            // forward: tiles handed out beyond the first one per CTA (zero at launch)
  uint8_t* stash;           // [n_tiles][n_stash][slot_bytes] activation tiles, or null (recompute)
  int* err;
};

// The plan's per-map arrays in shared memory.  Kernel parameters indexed with a
// run-time map index are loads from the constant bank at a computed address,
// which cost hundreds of cycles each on the MMA-issue path when they miss the
// constant cache; the copies in shared memory cost a shared-memory load.
struct TcTab {
  int w[kMaxLayers + 1], WP[kMaxLayers], o_w[kMaxLayers], c_wbar[kMaxLayers], off[kMaxLayers], o_buf[2];
};
__device__ __forceinline__ const TcTab* tc_tab_init(const TcPlan& pl, uint8_t* sm) {
  TcTab* t = reinterpret_cast<TcTab*>(sm + pl.o_tab);
  const int i = threadIdx.x;
  if (i <= kMaxLayers) {
    t->w[i] = pl.w[i];
    if (i < kMaxLayers) {
      t->WP[i] = pl.WP[i];
      t->o_w[i] = pl.o_w[i];
      t->c_wbar[i] = pl.c_wbar[i];
      t->off[i] = pl.off[i];
    }
    if (i < 2) t->o_buf[i] = pl.o_buf[i];
  }
  return t;
}

// Power-of-two scale 2^-e with max|seed| <= 2^e, so scaled seeds lie in [-1, 1]
// (exact to apply and to undo).
__device__ __forceinline__ float seed_scale(const float* absmax) {
  if (!absmax) return 1.f;
  const float m = *absmax;
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  int e;
  frexpf(m, &e);               // m = f 2^e, f in [0.5, 1)
  e = max(-100, min(100, e));
  return __int_as_float((127 - e) << 23);
}

// W_i (maps 1..L-2) as BF16 K-major core-matrix tiles, bias folded in column w_i;
// layer-0 and output-layer weights in FP32.
template <class OP>
__device__ void tc_load_weights(const TcPlan& pl, const float* __restrict__ P, uint8_t* sm) {
  const int L = pl.L;
  for (int i = 1; i <= L - 2; ++i) {
    const int in = pl.w[i], out = pl.w[i + 1], Kb = pl.WP[i - 1], Nr = pl.WP[i];
    const float* W = P + pl.off[i];
    uint16_t* dst = reinterpret_cast<uint16_t*>(sm + pl.o_w[i]);
    // eight entries per thread and pass, all loads issued before the first use
    constexpr int U = 8;
    for (int base = threadIdx.x; base < Nr * Kb; base += U * blockDim.x) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * blockDim.x;
        const int o = idx / Kb, k = idx - o * Kb;
        v[u] = 0.f;
        if (idx < Nr * Kb && o < out) v[u] = k < in ? W[o * in + k] : (k == in ? W[out * in + o] : 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx >= Nr * Kb) break;
        const int o = idx / Kb, k = idx - o * Kb;
        const uint32_t byte = row_off(o, Kb) + (k >> 3) * 128 + (k & 7) * 2;
        dst[byte >> 1] = (uint16_t)(OP::pack(v[u], 0.f) & 0xFFFFu);
      }
    }
  }
  float* s = reinterpret_cast<float*>(sm + pl.o_small);
  const int HP = pl.HP, w1 = pl.w[1];
  const float* W0 = P + pl.off[0];
  for (int o = threadIdx.x; o < HP; o += blockDim.x) {
    s[o] = o < w1 ? W0[o * 2] : 0.f;
    s[HP + o] = o < w1 ? W0[o * 2 + 1] : 0.f;
    s[2 * HP + o] = o < w1 ? W0[w1 * 2 + o] : 0.f;
    const int win = pl.w[L - 1];
    s[3 * HP + o] = o < win ? P[pl.off[L - 1] + o] : 0.f;
  }
  if (threadIdx.x == 0) s[4 * HP] = P[pl.off[L - 1] + pl.w[L - 1]];
}

// A point's coordinates and (reverse sweep) seeds as loaded from global memory;
// zero past the end.
struct PointIn {
  double x, y;
  float s[3];
};

__device__ __forceinline__ void point_fetch(const TcArgs& a, int64_t gp, PointIn& in) {
  in.x = 0.0; in.y = 0.0;
  if (gp < a.P_mesh) { in.x = a.Xm[2 * gp]; in.y = a.Xm[2 * gp + 1]; }
  else if (gp < a.P_tot) { in.x = a.Xe[2 * (gp - a.P_mesh)]; in.y = a.Xe[2 * (gp - a.P_mesh) + 1]; }
  const bool live = gp < a.P_tot && a.UB;
#pragma unroll
  for (int k = 0; k < 3; ++k) in.s[k] = live ? a.UB[k * a.P_tot + gp] : 0.f;
}

// Layer 0 on CUDA cores: H_0 row p (3 streams), this thread's 16 columns.
// Columns past the width have zero weights, so their tangents are 0; the bias
// column (index w1) is then set to (1, 0, 0) by the warps that hold it.
template <class OP>
__device__ __forceinline__ void layer0_store(const TcPlan& pl, const float* s_small, float x, float y, int p,
                                             int c0, uint8_t* buf) {
  const int K0 = pl.WP[0], w1 = pl.w[1], HP = pl.HP;
  if (c0 >= K0) return;
#pragma unroll
  for (int sc = 0; sc < 16; sc += 8) {
    const int cc = c0 + sc;
    float wx[8], wy[8], b0[8];
#pragma unroll
    for (int q = 0; q < 8; q += 4) {
      const float4 a = *reinterpret_cast<const float4*>(s_small + cc + q);
      const float4 b = *reinterpret_cast<const float4*>(s_small + HP + cc + q);
      const float4 c = *reinterpret_cast<const float4*>(s_small + 2 * HP + cc + q);
      wx[q] = a.x; wx[q + 1] = a.y; wx[q + 2] = a.z; wx[q + 3] = a.w;
      wy[q] = b.x; wy[q + 1] = b.y; wy[q + 2] = b.z; wy[q + 3] = b.w;
      b0[q] = c.x; b0[q + 1] = c.y; b0[q + 2] = c.z; b0[q + 3] = c.w;
    }
    uint32_t pv[4], px[4], py[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      float tv[2], tx[2], ty[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float t = tanh_fast(fmaf(wx[j + h], x, fmaf(wy[j + h], y, b0[j + h])));
        const float sd = fmaf(-t, t, 1.f);
        tv[h] = t;
        tx[h] = sd * wx[j + h];
        ty[h] = sd * wy[j + h];
      }
      pv[j >> 1] = OP::pack(tv[0], tv[1]);
      px[j >> 1] = OP::pack(tx[0], tx[1]);
      py[j >> 1] = OP::pack(ty[0], ty[1]);
    }
    if (w1 >= cc && w1 < cc + 8) set_bias_col<OP>(w1 - cc, pv, px, py);
    st8(buf, K0, p, cc, pv);
    st8(buf + 256 * K0, K0, p, cc, px);
    st8(buf + 512 * K0, K0, p, cc, py);
  }
}

// MMA issue.  One thread issues a tcgen05.mma about every 60 cycles, while the
// tensor core completes an M = 128, N = 64, K = 16 product in about 50 (M = 64:
// about 33), so the MMAs of a step are spread over the lane 0 of warps 0..3 (one
// per SM sub-partition), each writing its own accumulator; every step commits
// from all four threads to one mbarrier (arrival count 4; a thread with nothing
// to issue commits an empty set).  Descriptors are formed once per chain and
// advanced by adding the byte offset / 16 to the start-address field (shared
// memory below 256 KB keeps it inside its 14 bits).
constexpr uint32_t kIssuers = 4;

// A chain of n MMAs into D: operand descriptors advance by da / db per step.
__device__ __forceinline__ void mma_chain(uint32_t tD, uint64_t a, uint32_t da, uint64_t b, uint32_t db, uint32_t id,
                                          int n, bool first) {
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    mma_bf16(tD, a, b, id, (first && k == 0) ? 0u : 1u);
    a += da;
    b += db;
  }
}

// Forward MMAs of map i for stream s: D_s (columns s*HP) = H_{i-1,s} W_i^T, K = Kin, N = Nout.
__device__ __forceinline__ void issue_fwd_stream(uint32_t fmt, uint32_t tD, uint32_t abuf, uint32_t wbuf, int Kin,
                                                 int Nout, int HP, int s) {
  const uint32_t id = idesc_f16(fmt, 128, Nout, 0, 0);
  mma_chain(tD + s * HP, sdesc(abuf + s * 256 * Kin, 128, Kin * 16), 256 >> 4, sdesc(wbuf, 128, Kin * 16), 256 >> 4, id,
            Kin / 16, true);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float v[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Steps [k0, k1) of a weight-gradient chain (step k: stream k / 8, point block k % 8;
// 24 steps = K of 3 streams x 128 points) into accumulator tAcc.  Wbar_i reads
// H_{i-1} (Kin columns); Wbar_0 (w0) reads the layer-0 input: the value stream
// (x, y, 1) per point block and the constant tangent blocks.
__device__ __forceinline__ void wbar_chain_part(uint32_t fmt, uint32_t tAcc, uint32_t zbuf, int Nout, uint32_t bbuf,
                                                int Kin, bool w0, int k0, int k1, bool zero_first) {
  const uint32_t id = w0 ? idesc_f16(fmt, 64, 16, 1, 1) : idesc_f16(fmt, 64, Kin, 1, 1);
  for (int s = k0 >> 3; s <= (k1 - 1) >> 3; ++s) {
    const int p0 = s == (k0 >> 3) ? (k0 & 7) : 0;
    const int p1 = s == ((k1 - 1) >> 3) ? ((k1 - 1) & 7) + 1 : 8;
    const uint64_t a = sdesc(zbuf + s * 256 * Nout + p0 * 2 * Nout * 16, Nout * 16, 128);
    uint64_t b;
    uint32_t db;
    if (w0) {
      b = s ? sdesc(bbuf + 256 * 16 + (s - 1) * 512, 256, 128) : sdesc(bbuf + p0 * 2 * 16 * 16, 256, 128);
      db = s ? 0u : ((2 * 16 * 16) >> 4);
    } else {
      b = sdesc(bbuf + s * 256 * Kin + p0 * 2 * Kin * 16, Kin * 16, 128);
      db = (2 * Kin * 16) >> 4;
    }
    mma_chain(tAcc, a, (2 * Nout * 16) >> 4, b, db, id, p1 - p0, zero_first && s == (k0 >> 3));
  }
}

// Reverse step of map i >= 1:
//   Tbar_s (columns s*HP) = Zbar_s W_i: A = Zbar (K-major, K = Nout), B = W_i read
//     MN-major (N = Kin); stream s on issuer s (s = 0, 1, 2);
//   Wbar_i (M = 64 rows o, N = Kin) += sum over streams and points of Zbar^T B,
//     both read MN-major; K runs over 3 streams x 128 points.  With a partial
//     accumulator (tP) the chain is split: steps 0..11 into Wbar_i on issuer 3,
//     steps 12..23 into the partial on issuer 2, and the epilogue threads add
//     the partial into Wbar_i once both have completed; otherwise one chain on
//     issuer 3.
__device__ __forceinline__ void issue_reverse(uint32_t fmt, uint32_t tD, uint32_t tW, uint32_t tP, bool split,
                                              uint32_t zbuf, uint32_t wbuf, uint32_t bbuf, int Kin, int Nout, int HP,
                                              bool first, int issuer) {
  if (issuer < 3) {
    const int s = issuer;
    const uint32_t idt = idesc_f16(fmt, 128, Kin, 0, 1);
    mma_chain(tD + s * HP, sdesc(zbuf + s * 256 * Nout, 128, Nout * 16), 256 >> 4, sdesc(wbuf, Kin * 16, 128),
              (2 * Kin * 16) >> 4, idt, Nout / 16, true);
  }
  if (issuer == 3) wbar_chain_part(fmt, tW, zbuf, Nout, bbuf, Kin, false, 0, split ? 12 : 24, first);
  if (issuer == 2 && split) wbar_chain_part(fmt, tP, zbuf, Nout, bbuf, Kin, false, 12, 24, true);
}

// Reverse step of map 0 (inputs x, y, 1 in a 16-column tile): Wbar_0, split as above.
__device__ __forceinline__ void issue_wbar0(uint32_t fmt, uint32_t tW, uint32_t tP, bool split, uint32_t zbuf, int Kz,
                                            uint32_t xbuf, bool first, int issuer) {
  // the tangent streams of the layer-0 input tile are the full 128-point tiles of this kernel
  const uint32_t id = idesc_f16(fmt, 64, 16, 1, 1);
  auto part = [&](uint32_t tAcc, int k0, int k1, bool zero_first) {
    for (int s = k0 >> 3; s <= (k1 - 1) >> 3; ++s) {
      const int p0 = s == (k0 >> 3) ? (k0 & 7) : 0;
      const int p1 = s == ((k1 - 1) >> 3) ? ((k1 - 1) & 7) + 1 : 8;
      mma_chain(tAcc, sdesc(zbuf + s * 256 * Kz + p0 * 2 * Kz * 16, Kz * 16, 128), (2 * Kz * 16) >> 4,
                sdesc(xbuf + s * 256 * 16 + p0 * 2 * 16 * 16, 256, 128), (2 * 16 * 16) >> 4, id, p1 - p0,
                zero_first && s == (k0 >> 3));
    }
  };
  if (issuer == 3) part(tW, 0, split ? 12 : 24, first);
  if (issuer == 2 && split) part(tP, 12, 24, true);
}

// ------------------------------------------------------------------ forward kernel
// One activation tile, updated in place: once map i's MMAs have completed,
// H_{i-1} is dead and the epilogue overwrites it with H_i.
template <int HP, class OP>
__global__ void __launch_bounds__(tc_threads<HP>(), HP == 32 ? 3 : 2) mlp_fwd_tc(TcArgs a) {
  constexpr int NG = HP / 16;
  extern __shared__ __align__(1024) uint8_t sm[];
  const TcPlan& pl = a.pl;
  const TcTab* tb = tc_tab_init(pl, sm);       // read after the prologue barrier
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, grp = warp >> 2;
  const int p = q4 * 32 + lane;                 // point (row / TMEM lane)
  const int c0 = grp * 16;                      // this thread's 16 columns
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + pl.o_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + pl.o_bar + 8);
  const float* s_small = reinterpret_cast<const float*>(sm + pl.o_small);
  float* s_red = reinterpret_cast<float*>(sm + pl.o_red);        // [NG][128][3]
  uint8_t* buf = sm + pl.o_buf[0];
  if (warp == 0) { tmem_alloc(s_tmem, pl.tmem_cols); tmem_relinquish(); }
  if (tid == 0) {
    mbar_init(bar, kIssuers);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const bool issuer = lane == 0 && warp < (int)kIssuers;   // issues and commits this CTA's MMAs
  // Tiles: the first from the CTA index, the later ones from the launch's
  // counter (the outputs of a tile do not depend on which CTA computes it),
  // requested two ahead so that the atomic and the next tile's coordinate
  // loads are in flight during a tile; a ring of two shared slots.
  int* s_tl = reinterpret_cast<int*>(sm + pl.o_bar + 16);
  if (tid == 0) s_tl[0] = (int)gridDim.x + atomicAdd(a.tile_ctr, 1);
  const int64_t n_tiles = (a.P_tot + kTile - 1) / kTile;
  PointIn nxt;                                  // next tile's coordinates, loads in flight under the prologue
  if (blockIdx.x < n_tiles) point_fetch(a, blockIdx.x * kTile + p, nxt);
  tc_load_weights<OP>(pl, a.params, sm);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = *s_tmem;
  const uint32_t tRow = tD + ((uint32_t)(q4 * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;
  // this thread's MMA wait timed out; the threads agree on it at the barrier
  // that ends each map (a reduction barrier), so all leave the tile loop together
  bool tfail = false;
  const int L = pl.L;
  int64_t tile = blockIdx.x, next = s_tl[0];
  for (int it = 0; tile < n_tiles && !failed; ++it) {
    const int64_t gp = tile * kTile + p;
    const float x = (float)nxt.x, y = (float)nxt.y;
    if (next < n_tiles) point_fetch(a, next * kTile + p, nxt);
    if (tid == 0) s_tl[(it + 1) & 1] = (int)gridDim.x + atomicAdd(a.tile_ctr, 1);   // the tile after next
    float u = 0.f, ux = 0.f, uy = 0.f;          // output-layer partial sums over this thread's columns
    if (L == 2) {   // one hidden layer: output straight from layer 0
      for (int o = c0; o < min(tb->w[1], c0 + 16); ++o) {
        const float wx = s_small[o], wy = s_small[HP + o];
        const float t = tanh_fast(fmaf(wx, x, fmaf(wy, y, s_small[2 * HP + o])));
        const float sd = fmaf(-t, t, 1.f), wl = s_small[3 * HP + o];
        u = fmaf(wl, t, u); ux = fmaf(wl, sd * wx, ux); uy = fmaf(wl, sd * wy, uy);
      }
    } else {
      layer0_store<OP>(pl, s_small, x, y, p, c0, buf);
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      for (int i = 1; i <= L - 2; ++i) {
        const int Kin = tb->WP[i - 1], Nout = tb->WP[i];
        if (issuer) {
          tc_fence_after();
          if (warp < 3) issue_fwd_stream(OP::fmt, tD, su32(buf), su32(sm + tb->o_w[i]), Kin, Nout, HP, warp);
          mma_commit(bar);
        }
        __syncwarp();   // the issuer's warp-mates wait here, not in a polling loop beside it
        if (!mbar_wait(bar, phase)) {
          tfail = true;
          if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT);
        }
        phase ^= 1;
        tc_fence_after();
        const bool last = i == L - 2;
        const int wo = tb->w[i + 1];
        // H_i also goes to the stash (same tile layout, streaming stores) when the
        // reverse sweep reads it: this thread's row and first column chunk of the
        // value stream
        uint8_t* gst = nullptr;
        if (a.stash && i >= pl.stash_lo && i < pl.stash_lo + pl.n_stash && c0 < Nout)
          gst = a.stash + (tile * pl.n_stash + (i - pl.stash_lo)) * (int64_t)pl.slot_bytes + row_off(p, Nout) +
                (c0 >> 3) * 128;
        if (c0 < Nout) {
#pragma unroll
          for (int sc = 0; sc < 16; sc += 8) {
            const int cc = c0 + sc;
            float dv[8], dx[8], dy[8];
            tmem_ld8(tRow + cc, dv);
            tmem_ld8(tRow + HP + cc, dx);
            tmem_ld8(tRow + 2 * HP + cc, dy);
            tmem_wait_ld();
            uint32_t pv[4], px[4], py[4];
            if (last) {
              // output layer: the bias column and the padding carry zero output
              // weights, so no column needs patching here
              const float4 wa = *reinterpret_cast<const float4*>(s_small + 3 * HP + cc);
              const float4 wb = *reinterpret_cast<const float4*>(s_small + 3 * HP + cc + 4);
              const float wl[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float t = tanh_fast(dv[j]);
                const float sd = fmaf(-t, t, 1.f);
                u = fmaf(wl[j], t, u);
                ux = fmaf(wl[j] * sd, dx[j], ux);
                uy = fmaf(wl[j] * sd, dy[j], uy);
              }
              continue;
            }
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              float tv[2], tx[2], ty[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float t = tanh_fast(dv[j + h]);
                const float sd = fmaf(-t, t, 1.f);
                tv[h] = t;
                tx[h] = sd * dx[j + h];
                ty[h] = sd * dy[j + h];
              }
              pv[j >> 1] = OP::pack(tv[0], tv[1]);
              px[j >> 1] = OP::pack(tx[0], tx[1]);
              py[j >> 1] = OP::pack(ty[0], ty[1]);
            }
            if (wo >= cc && wo < cc + 8) set_bias_col<OP>(wo - cc, pv, px, py);
            {
              // H_{i-1} (the MMA's A operand) is dead: overwrite the tile with H_i
              st8(buf, Nout, p, cc, pv);
              st8(buf + 256 * Nout, Nout, p, cc, px);
              st8(buf + 512 * Nout, Nout, p, cc, py);
              if (gst) {
                __stcs(reinterpret_cast<uint4*>(gst + sc * 16), make_uint4(pv[0], pv[1], pv[2], pv[3]));
                __stcs(reinterpret_cast<uint4*>(gst + 256 * Nout + sc * 16), make_uint4(px[0], px[1], px[2], px[3]));
                __stcs(reinterpret_cast<uint4*>(gst + 512 * Nout + sc * 16), make_uint4(py[0], py[1], py[2], py[3]));
              }
            }
          }
        }
        if (!last) fence_proxy_async();
        tc_fence_before();
        if (__syncthreads_or(tfail)) { failed = true; break; }
      }
      if (failed) break;
    }
    // combine the column groups in fixed order: u = b_L + sum over groups
    s_red[(grp * kTile + p) * 3] = u;
    s_red[(grp * kTile + p) * 3 + 1] = ux;
    s_red[(grp * kTile + p) * 3 + 2] = uy;
    __syncthreads();
    if (grp == 0 && gp < a.P_tot) {
      float su = s_small[4 * HP], sx = 0.f, sy = 0.f;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        su += s_red[(g * kTile + p) * 3];
        sx += s_red[(g * kTile + p) * 3 + 1];
        sy += s_red[(g * kTile + p) * 3 + 2];
      }
      a.U[gp] = su;
      a.U[a.P_tot + gp] = sx;
      a.U[2 * a.P_tot + gp] = sy;
    }
    __syncthreads();
    tile = next;
    next = s_tl[(it + 1) & 1];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tD, pl.tmem_cols);
}

// ------------------------------------------------------------------ reverse kernel
template <int HP, class OP>
__global__ void __launch_bounds__(tc_threads<HP>(), HP == 32 ? 2 : 1) mlp_bwd_tc(TcArgs a) {
  constexpr int NT = tc_threads<HP>();
  extern __shared__ __align__(1024) uint8_t sm[];
  const TcPlan& pl = a.pl;
  const TcTab* tb = tc_tab_init(pl, sm);       // read after the prologue barrier
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, grp = warp >> 2;
  const int p = q4 * 32 + lane;                 // point (row / TMEM lane)
  const int c0 = grp * 16;                      // this thread's 16 columns
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + pl.o_bar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + pl.o_bar + 8);
  const float* s_small = reinterpret_cast<const float*>(sm + pl.o_small);
  uint8_t* xbuf = sm + pl.o_x;
  uint8_t* zb = sm + pl.o_z;
  // activation stash: the tile's stored layers arrive by bulk copies on ldbar
  // (one arrival per layer); the next tile's are requested as soon as their
  // buffers are dead in this tile
  uint64_t* ldbar = reinterpret_cast<uint64_t*>(sm + pl.o_bar + 24);
  // (read from the kernel parameters at each use rather than held in registers)
  auto stash_on = [&]() { return a.stash != nullptr && pl.n_stash > 0; };
  if (warp == 0) { tmem_alloc(s_tmem, pl.tmem_cols); tmem_relinquish(); }
  if (tid == 0) {
    mbar_init(bar, kIssuers);
    if (stash_on()) mbar_init(ldbar, pl.n_stash);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the first tile's stashed layers, in flight under the weight prologue
    // (before the barrier that publishes the shared table: kernel parameters here)
    if (stash_on() && blockIdx.x < (a.P_tot + kTile - 1) / kTile)
      for (int j = pl.stash_lo; j < pl.stash_lo + pl.n_stash; ++j) {
        const uint32_t bytes = 3u * 256u * (uint32_t)pl.WP[j];
        mbar_expect_tx(ldbar, bytes);
        bulk_load(sm + pl.o_buf[j & 1],
                  a.stash + ((int64_t)blockIdx.x * pl.n_stash + (j - pl.stash_lo)) * (int64_t)pl.slot_bytes, bytes,
                  ldbar, l2_evict_first());
      }
  }
  // this thread's point inputs for a tile (coordinates and seeds), kept as
  // loaded so that the loads of the next tile stay in flight until first use
  // (the first tile's under the weight prologue)
  const int64_t n_tiles = (a.P_tot + kTile - 1) / kTile;
  PointIn nxt;
  if (blockIdx.x < n_tiles) point_fetch(a, blockIdx.x * kTile + p, nxt);
  tc_load_weights<OP>(pl, a.params, sm);
  if (grp == 0) {  // layer-0 input tile: streams d/dx and d/dy are the constant unit vectors
    uint32_t ex[4] = {OP::pack(1.f, 0.f), 0, 0, 0};
    uint32_t ey[4] = {OP::pack(0.f, 1.f), 0, 0, 0};
    uint32_t zz[4] = {0, 0, 0, 0};
    st8(xbuf + 256 * 16, 16, p, 0, ex);
    st8(xbuf + 256 * 16, 16, p, 8, zz);
    st8(xbuf + 512 * 16, 16, p, 0, ey);
    st8(xbuf + 512 * 16, 16, p, 8, zz);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = *s_tmem;
  const uint32_t tRow = tD + ((uint32_t)(q4 * 32) << 16);
  uint32_t phase = 0;
  bool failed = false;
  const int L = pl.L;
  const bool issuer = lane == 0 && warp < (int)kIssuers;   // issues and commits this CTA's MMAs
  constexpr int kWbarWarp = 3;     // the issuer of the weight-gradient chains (their first half when split)
  const bool split = pl.c_part > 0;   // weight-gradient chains in two halves (a partial accumulator exists)
  // Wbar_i += partial, this thread's lane quarter (rows in lanes 0..15) and column group
  auto fold_part = [&](int i) {
    const int ncols = i >= 1 ? tb->WP[i - 1] : 16;
    for (int cb = c0; cb < c0 + 16 && cb < ncols; cb += 8) {
      float pv[8], wv[8];
      tmem_ld8(tRow + pl.c_part + cb, pv);
      tmem_ld8(tRow + tb->c_wbar[i] + cb, wv);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; ++j) wv[j] += pv[j];
      tmem_st8(tRow + tb->c_wbar[i] + cb, wv);
    }
    tmem_wait_st();
  };
  uint32_t wfirst = 0xFFFFFFFFu;   // bit i: Wbar_i accumulator not yet written (weight-gradient issuer)
  float accL[16];                  // output-layer weight gradient: this thread's columns, its points
#pragma unroll
  for (int k = 0; k < 16; ++k) accL[k] = 0.f;
  float accB = 0.f;                // output-bias gradient (the bias column's activation is 1): its points'
                                   // value seeds, summed in tile order
  int bufH0 = -1, bufH1 = -1;      // layer held by activation tile 0 / 1
  const float sc = seed_scale(a.seed_absmax);   // adjoint scale (1 for BF16)
  const double inv_sc = 1.0 / (double)sc;

  // wait for the committed MMAs (every thread for itself: the wait orders its
  // own tensor-memory reads); a time-out sets this thread's flag, which the
  // threads agree on at the reduction barrier that ends the step (the flag
  // stays set, so every later barrier agrees too)
  bool tfail = false;
  auto wait_mma = [&]() {
    if (!mbar_wait(bar, phase)) {
      tfail = true;
      if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT);
    }
    phase ^= 1;
    tc_fence_after();
  };
  // tid 0: request stash layers j of tile t whose buffer (j & 1) is in `bufs`
  auto stash_request = [&](int64_t t, int bufs) {
    for (int j = pl.stash_lo; j < pl.stash_lo + pl.n_stash; ++j) {
      if (!((bufs >> (j & 1)) & 1)) continue;
      const uint32_t bytes = 3u * 256u * (uint32_t)tb->WP[j];
      mbar_expect_tx(ldbar, bytes);
      bulk_load(sm + tb->o_buf[j & 1], a.stash + (t * pl.n_stash + (j - pl.stash_lo)) * (int64_t)pl.slot_bytes, bytes,
                ldbar, l2_evict_first());
    }
  };
  // make this thread's shared stores visible to the tensor core; true when
  // some thread's MMA wait has timed out
  auto publish = [&]() -> bool {
    fence_proxy_async();
    tc_fence_before();
    return __syncthreads_or(tfail) != 0;
  };
  auto issue_fwd_map = [&](int i) {
    if (issuer) {
      tc_fence_after();
      if (warp < 3)
        issue_fwd_stream(OP::fmt, tD, su32(sm + tb->o_buf[(i - 1) & 1]), su32(sm + tb->o_w[i]), tb->WP[i - 1], tb->WP[i],
                         HP, warp);
      mma_commit(bar);
    }
    __syncwarp();
  };
  // forward epilogue of hidden map i from D into activation tile `ob`
  auto fwd_epilogue_store = [&](int i, uint8_t* ob) {
    const int Nout = tb->WP[i], wo = tb->w[i + 1];
    if (c0 >= Nout) return;
#pragma unroll
    for (int sc8 = 0; sc8 < 16; sc8 += 8) {
      const int cc = c0 + sc8;
      float dv[8], dx[8], dy[8];
      tmem_ld8(tRow + cc, dv);
      tmem_ld8(tRow + HP + cc, dx);
      tmem_ld8(tRow + 2 * HP + cc, dy);
      tmem_wait_ld();
      uint32_t pv[4], px[4], py[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        float tv[2], tx[2], ty[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float t = tanh_fast(dv[j + h]);
          const float sd = fmaf(-t, t, 1.f);
          tv[h] = t;
          tx[h] = sd * dx[j + h];
          ty[h] = sd * dy[j + h];
        }
        pv[j >> 1] = OP::pack(tv[0], tv[1]);
        px[j >> 1] = OP::pack(tx[0], tx[1]);
        py[j >> 1] = OP::pack(ty[0], ty[1]);
      }
      if (wo >= cc && wo < cc + 8) set_bias_col<OP>(wo - cc, pv, px, py);
      st8(ob, Nout, p, cc, pv);
      st8(ob + 256 * Nout, Nout, p, cc, px);
      st8(ob + 512 * Nout, Nout, p, cc, py);
    }
  };
  // recompute H_0 .. H_upto into the two activation tiles (H_j -> buf[j & 1])
  auto recompute = [&](int upto, float x, float y) -> bool {
    layer0_store<OP>(pl, s_small, x, y, p, c0, sm + tb->o_buf[0]);
    if (publish()) return false;
    for (int j = 1; j <= upto; ++j) {
      issue_fwd_map(j);
      wait_mma();
      fwd_epilogue_store(j, sm + tb->o_buf[j & 1]);
      if (publish()) return false;
    }
    bufH0 = upto >= 1 ? ((upto & 1) == 0 ? upto : upto - 1) : 0;
    bufH1 = upto >= 1 ? ((upto & 1) == 1 ? upto : upto - 1) : -1;
    return true;
  };

  bool h0_ready = false;           // H_0 of this tile already in buf[0] (computed under the previous tile's MMAs)
  // with the stash, buf[0] takes a stashed layer (4 hidden layers) or H_0 (3)
  auto stash_buf0 = [&]() { return stash_on() && pl.n_stash == 2; };
  uint32_t ldstate = 0;            // bit 0: ldbar phase to wait for; bit 1: copies requested, not waited for
  if (stash_on() && blockIdx.x < n_tiles) ldstate |= 2u;   // the first tile's copies (requested above)
  for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
    const float x = (float)nxt.x, y = (float)nxt.y;
    const float su = sc * nxt.s[0], sx = sc * nxt.s[1], sy = sc * nxt.s[2];
    accB += su;
    const bool has_next = tile + gridDim.x < n_tiles;
    if (has_next) point_fetch(a, (tile + gridDim.x) * kTile + p, nxt);
    if (grp == 0) {
      uint32_t xr[4] = {OP::pack(x, y), OP::pack(1.f, 0.f), 0, 0};
      st8(xbuf, 16, p, 0, xr);
      uint32_t zz[4] = {0, 0, 0, 0};
      st8(xbuf, 16, p, 8, zz);
    }
    // ---- forward recompute; the last hidden map's epilogue applies the output
    //      layer and the seeds and writes Zbar_{L-2} (its H is never stored)
    const int last = L - 2;
    if (stash_on()) {
      // stored layers from the forward kernel; maps 1 .. last-1 are not recomputed
      if (!stash_buf0() && !h0_ready) layer0_store<OP>(pl, s_small, x, y, p, c0, sm + tb->o_buf[0]);
      const bool ok = mbar_wait(ldbar, ldstate & 1u);
      ldstate = (ldstate & 1u) ^ 1u;
      if (__syncthreads_or(!ok)) { if (tid == 0) atomicExch(a.err, FV_ERR_TIMEOUT); failed = true; break; }
      if (publish()) { failed = true; break; }
      issue_fwd_map(last);
      wait_mma();
    } else if (last >= 1) {
      if (!h0_ready) layer0_store<OP>(pl, s_small, x, y, p, c0, sm + tb->o_buf[0]);
      if (publish()) { failed = true; break; }
      for (int i = 1; i < last; ++i) {
        issue_fwd_map(i);
        wait_mma();
        fwd_epilogue_store(i, sm + tb->o_buf[i & 1]);
        if (publish()) { failed = true; break; }
      }
      if (failed) break;
      issue_fwd_map(last);
      wait_mma();
    }
    {
      const int Nout = tb->WP[last];
      if (c0 < Nout) {
#pragma unroll
        for (int sc8 = 0; sc8 < 16; sc8 += 8) {
          const int cc = c0 + sc8;
          float dv[8], dx[8], dy[8];
          if (last >= 1) {
            tmem_ld8(tRow + cc, dv);
            tmem_ld8(tRow + HP + cc, dx);
            tmem_ld8(tRow + 2 * HP + cc, dy);
            tmem_wait_ld();
          } else {      // single hidden layer: pre-activations from layer 0 on CUDA cores
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int o = cc + j;
              const float wx = s_small[o], wy = s_small[HP + o];
              dv[j] = fmaf(wx, x, fmaf(wy, y, s_small[2 * HP + o]));
              dx[j] = wx;
              dy[j] = wy;
            }
          }
          uint32_t pv[4], px[4], py[4];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            float zv[2], zx[2], zy[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // the bias column (o == w[last + 1]) has zero weights into it and a zero output
              // weight: its t, tangents and adjoints come out 0 here; only the
              // output-bias gradient needs its value 1, added below
              const int o = cc + j + h;
              const float t = tanh_fast(dv[j + h]);
              const float sd = fmaf(-t, t, 1.f);
              const float tx = sd * dx[j + h], ty = sd * dy[j + h];
              float& acc = accL[sc8 + j + h];
              acc = fmaf(su, t, fmaf(sx, tx, fmaf(sy, ty, acc)));
              const float wl = s_small[3 * HP + o];
              const float bv = wl * su, bx = wl * sx, by = wl * sy;
              zv[h] = sd * bv - 2.f * t * (tx * bx + ty * by);
              zx[h] = sd * bx;
              zy[h] = sd * by;
            }
            pv[j >> 1] = OP::pack(zv[0], zv[1]);
            px[j >> 1] = OP::pack(zx[0], zx[1]);
            py[j >> 1] = OP::pack(zy[0], zy[1]);
          }
          st8(zb, Nout, p, cc, pv);
          st8(zb + 256 * Nout, Nout, p, cc, px);
          st8(zb + 512 * Nout, Nout, p, cc, py);
        }
      }
    }
    if (publish()) { failed = true; break; }
    // tiles holding H after the forward: H_j in buf[j & 1] for the two highest stored j
    bufH0 = -1; bufH1 = -1;
    if (last - 1 >= 0) { if ((last - 1) & 1) bufH1 = last - 1; else bufH0 = last - 1; }
    if (last - 2 >= 0) { if ((last - 2) & 1) bufH1 = last - 2; else bufH0 = last - 2; }
    // ---- reverse, map by map from the top
    for (int i = last; i >= 0 && !failed; --i) {
      uint32_t bsrc;
      int Kb;
      if (i >= 1) {
        if ((((i - 1) & 1) ? bufH1 : bufH0) != i - 1) {
          if (!recompute(i - 1, x, y)) { failed = true; break; }
        }
        bsrc = su32(sm + tb->o_buf[(i - 1) & 1]);
        Kb = tb->WP[i - 1];
      } else {
        bsrc = su32(xbuf);
        Kb = 16;
      }
      if (issuer) {
        tc_fence_after();
        if (i >= 1)
          issue_reverse(OP::fmt, tD, tD + tb->c_wbar[i], tD + pl.c_part, split, su32(zb), su32(sm + tb->o_w[i]), bsrc,
                        tb->WP[i - 1], tb->WP[i], HP, (wfirst >> i) & 1u, warp);
        else
          issue_wbar0(OP::fmt, tD + tb->c_wbar[0], tD + pl.c_part, split, su32(zb), tb->WP[0], bsrc, (wfirst >> 0) & 1u,
                      warp);
        wfirst &= ~(1u << i);
        mma_commit(bar);
      }
      __syncwarp();
      if (tid == 0) {
        // the next tile's stashed layers into buffers this tile no longer reads:
        // buf[1] from step 1 on (only H_0 in buf[0] is left), buf[0] at step 0
        // (requesting buf[0] once step 1's MMAs are done, with epilogue 1
        // recomputing H_0, measured slower: 494 against 451 us)
        if (stash_on() && has_next && i <= 1) {
          fence_proxy_async();
          stash_request(tile + gridDim.x, i == 1 ? 2 : 1);
        }
      }
      if (stash_on() && has_next && i <= 1) ldstate |= 2u;
      // CUDA-core work on dead tiles while the tensor core runs: H_0 for map 1's
      // reverse step into buf[0] (H_2 there is dead once map 3's step is done),
      // and under map 0's step the next tile's H_0 (buf[0] held this tile's H_0,
      // read by map 1's step only)
      if (i == 2 && bufH0 != 0) {
        layer0_store<OP>(pl, s_small, x, y, p, c0, sm + tb->o_buf[0]);
        bufH0 = 0;
      }
      if (i == 0) {
        h0_ready = last >= 1 && has_next && !stash_buf0();
        if (h0_ready) layer0_store<OP>(pl, s_small, (float)nxt.x, (float)nxt.y, p, c0, sm + tb->o_buf[0]);
      }
      wait_mma();
      if (split) fold_part(i);
      if (i >= 1) {
        // Zbar_{i-1} from Tbar_{i-1} (tensor memory) and H_{i-1} (shared tile), tanh rule
        const int K = tb->WP[i - 1];
        const uint8_t* hb = sm + tb->o_buf[(i - 1) & 1];
        // this thread's 8 columns [cc, cc + 8) of H_{i-1}, 3 streams, as stored (16-bit pairs)
        auto h_packed = [&](int cc, uint32_t hv[4], uint32_t hx[4], uint32_t hy[4]) {
          const uint32_t ho = row_off(p, K) + (cc >> 3) * 128;
          const uint4 Hv = *reinterpret_cast<const uint4*>(hb + ho);
          const uint4 Hx = *reinterpret_cast<const uint4*>(hb + 256 * K + ho);
          const uint4 Hy = *reinterpret_cast<const uint4*>(hb + 512 * K + ho);
          hv[0] = Hv.x; hv[1] = Hv.y; hv[2] = Hv.z; hv[3] = Hv.w;
          hx[0] = Hx.x; hx[1] = Hx.y; hx[2] = Hx.z; hx[3] = Hx.w;
          hy[0] = Hy.x; hy[1] = Hy.y; hy[2] = Hy.z; hy[3] = Hy.w;
        };
        if (c0 < K && OP::fmt == OpF16::fmt) {
          // FP16: the tanh rule in packed half2 arithmetic on the FP16 activations as
          // stored (two columns per instruction); the adjoints from tensor memory are
          // rounded to FP16 first (they are stored in FP16 anyway)
#pragma unroll
          for (int sc8 = 0; sc8 < 16; sc8 += 8) {
            const int cc = c0 + sc8;
            float bv[8], bx[8], by[8];
            tmem_ld8(tRow + cc, bv);
            tmem_ld8(tRow + HP + cc, bx);
            tmem_ld8(tRow + 2 * HP + cc, by);
            uint32_t hv[4], hx[4], hy[4];
            h_packed(cc, hv, hx, hy);
            tmem_wait_ld();
            uint32_t pv[4], px[4], py[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const __half2 one = __float2half2_rn(1.f);
              const __half2 t = u32_h2(hv[w]), tx = u32_h2(hx[w]), ty = u32_h2(hy[w]);
              const __half2 gv = __floats2half2_rn(bv[2 * w], bv[2 * w + 1]);
              const __half2 gx = __floats2half2_rn(bx[2 * w], bx[2 * w + 1]);
              const __half2 gy = __floats2half2_rn(by[2 * w], by[2 * w + 1]);
              const __half2 sd = __hfma2(__hneg2(t), t, one);
              const __half2 q = __hfma2(ty, gy, __hmul2(tx, gx));
              pv[w] = h2_u32(__hfma2(sd, gv, __hneg2(__hmul2(__hadd2(t, t), q))));
              px[w] = h2_u32(__hmul2(sd, gx));
              py[w] = h2_u32(__hmul2(sd, gy));
            }
            st8(zb, K, p, cc, pv);
            st8(zb + 256 * K, K, p, cc, px);
            st8(zb + 512 * K, K, p, cc, py);
          }
        } else if (c0 < K) {
#pragma unroll
          for (int sc8 = 0; sc8 < 16; sc8 += 8) {
            const int cc = c0 + sc8;
            float bv[8], bx[8], by[8], hv[8], hx[8], hy[8];
            tmem_ld8(tRow + cc, bv);
            tmem_ld8(tRow + HP + cc, bx);
            tmem_ld8(tRow + 2 * HP + cc, by);
            {
              uint32_t uv[4], ux[4], uy[4];
              h_packed(cc, uv, ux, uy);
#pragma unroll
              for (int w = 0; w < 4; ++w) {
                hv[2 * w] = OP::lo(uv[w]); hv[2 * w + 1] = OP::hi(uv[w]);
                hx[2 * w] = OP::lo(ux[w]); hx[2 * w + 1] = OP::hi(ux[w]);
                hy[2 * w] = OP::lo(uy[w]); hy[2 * w + 1] = OP::hi(uy[w]);
              }
            }
            tmem_wait_ld();
            uint32_t pv[4], px[4], py[4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              float zv[2], zx[2], zy[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float t = hv[j + h], sd = fmaf(-t, t, 1.f);
                zv[h] = sd * bv[j + h] - 2.f * t * (hx[j + h] * bx[j + h] + hy[j + h] * by[j + h]);
                zx[h] = sd * bx[j + h];
                zy[h] = sd * by[j + h];
              }
              pv[j >> 1] = OP::pack(zv[0], zv[1]);
              px[j >> 1] = OP::pack(zx[0], zx[1]);
              py[j >> 1] = OP::pack(zy[0], zy[1]);
            }
            st8(zb, K, p, cc, pv);
            st8(zb + 256 * K, K, p, cc, px);
            st8(zb + 512 * K, K, p, cc, py);
          }
        }
        if (publish()) { failed = true; break; }
      } else {
        tc_fence_before();
        if (__syncthreads_or(tfail)) { failed = true; break; }
      }
    }
  }
  if (ldstate & 2u) mbar_wait(ldbar, ldstate & 1u);   // after a failure: let requested copies land
  // ---- write this CTA's gradient partials
  uint32_t* s_flags = reinterpret_cast<uint32_t*>(sm + pl.o_bar + 12);
  if (tid == kWbarWarp * 32) *s_flags = wfirst;   // accumulators never written by this CTA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t never_mask = *s_flags;
  double* g = a.gpart + (size_t)blockIdx.x * pl.n_params;
  if (!failed) {
    if (grp == 0) {
      // hidden maps 0..L-2 from tensor memory (M = 64 layout: row o in lane (o/16)*32 + o%16)
      const int o = q4 * 16 + lane;
      for (int i = 0; i <= L - 2; ++i) {
        const int Kb = i >= 1 ? tb->WP[i - 1] : 16;
        const int in = tb->w[i], out = tb->w[i + 1];
        const bool never = (never_mask >> i) & 1u;
        for (int cb = 0; cb < Kb; cb += 8) {
          float v[8];
          tmem_ld8(tRow + tb->c_wbar[i] + cb, v);
          tmem_wait_ld();

          if (lane < 16 && o < out) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int k = cb + j;
              const double val = never ? 0.0 : (double)v[j] * inv_sc;
              if (k < in) g[tb->off[i] + o * in + k] = val;
              else if (k == in) g[tb->off[i] + out * in + o] = val;
            }
          }
        }
      }
    }
  } else {
    for (int i = tid; i < pl.n_params; i += NT) g[i] = 0.0;
  }
  // output layer: reduce accL over the CTA's 128 points in fixed order
  tc_fence_before();
  __syncthreads();
  float* scratch = reinterpret_cast<float*>(sm + tb->o_buf[0]);   // [128][HP]
  const int win = tb->w[L - 1];
#pragma unroll
  for (int k = 0; k < 16; ++k) scratch[p * HP + c0 + k] = c0 + k == win ? accB : accL[k];
  __syncthreads();
  if (tid < HP) {
    double sum = 0.0;
    for (int t = 0; t < kTile; ++t) sum += (double)scratch[t * HP + tid];
    if (tid <= win) g[tb->off[L - 1] + tid] = failed ? 0.0 : sum * inv_sc;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tD, pl.tmem_cols);
}

// ------------------------------------------------------------------ host side
bool make_tc_plan(const EvalPlan& ep, bool reverse, TcPlan* p) {
  const MlpShape& s = ep.shape;
  if (ep.prec != FV_BF16 && ep.prec != FV_FP16) return false;
  if (s.L < 2 || s.w[s.L] != 1) return false;     // one output (u); eps(x, y) networks run on CUDA cores
  p->L = s.L;
  p->n_params = s.n_params;
  int HP = 16;
  for (int i = 0; i <= s.L; ++i) p->w[i] = s.w[i];
  for (int i = 0; i < s.L; ++i) p->off[i] = s.off[i];
  for (int i = 0; i + 1 < s.L; ++i) {
    p->WP[i] = ru16(s.w[i + 1] + 1);
    HP = std::max(HP, p->WP[i]);
  }
  if (HP > 64) return false;
  HP = HP <= 32 ? 32 : 64;
  p->HP = HP;
  int o = 0;
  for (int i = 1; i <= s.L - 2; ++i) {
    p->o_w[i] = o;
    o += p->WP[i] * p->WP[i - 1] * 2;
  }
  o = (o + 127) & ~127;
  p->o_small = o; o += (4 * HP + 4) * 4;
  o = (o + 127) & ~127;
  const int tile_bytes = 3 * kTile * HP * 2;
  p->o_buf[0] = o; o += tile_bytes;
  if (reverse) {
    p->o_buf[1] = o; o += tile_bytes;
    p->o_z = o; o += tile_bytes;
    p->o_x = o; o += 3 * kTile * 16 * 2;
    o += 512;   // the 64-row weight-gradient read of a 32-wide adjoint tile runs past its end
  } else {
    p->o_buf[1] = p->o_buf[0];
    p->o_z = p->o_x = 0;
  }
  p->o_red = o; o += kTile * (HP / 16) * 3 * 4;
  p->o_bar = o; o += 48;
  p->o_tab = o; o += (int)sizeof(TcTab);
  p->smem = (o + 127) & ~127;
  int cols = 3 * HP;
  if (reverse) {
    for (int i = 1; i <= s.L - 2; ++i) { p->c_wbar[i] = cols; cols += HP; }
    p->c_wbar[0] = cols; cols += 16;
  }
  auto alloc_cols = [](int c) { int t = 32; while (t < c) t *= 2; return t; };
  int t = alloc_cols(cols);
  // reverse: a partial weight-gradient accumulator (HP columns) splits each
  // weight-gradient chain in two; taken where it keeps the allocation (and the
  // CTAs per SM) unchanged
  p->c_part = 0;
  if (reverse && alloc_cols(cols + HP) == t) {
    p->c_part = cols;
    cols += HP;
    t = alloc_cols(cols);
  }
  if (t > 512) return false;
  p->tmem_cols = t;
  const int last = s.L - 2;
  p->stash_lo = std::max(1, last - 2);
  p->n_stash = (last == 2 || last == 3) ? last - p->stash_lo : 0;
  p->slot_bytes = 3 * kTile * HP * 2;
  return true;
}

// Resident CTAs per SM: registers, shared memory and threads, capped so that
// their tensor-memory allocations fit in 512 columns.
template <int HP, class OP>
int tc_ctas_per_sm(fv_ctx ctx, const TcPlan& p, bool reverse) {
  const int n = reverse ? resident_ctas(ctx, (const void*)mlp_bwd_tc<HP, OP>, tc_threads<HP>(), p.smem)
                        : resident_ctas(ctx, (const void*)mlp_fwd_tc<HP, OP>, tc_threads<HP>(), p.smem);
  return std::max(1, std::min(std::max(n, 1), 512 / p.tmem_cols));
}

int tc_grid(fv_ctx ctx, const TcPlan& p, bool reverse, bool fp16, int64_t P_tot) {
  const int64_t n_tiles = (P_tot + kTile - 1) / kTile;
  const int per = p.HP == 32 ? (fp16 ? tc_ctas_per_sm<32, OpF16>(ctx, p, reverse) : tc_ctas_per_sm<32, OpBF16>(ctx, p, reverse))
                             : (fp16 ? tc_ctas_per_sm<64, OpF16>(ctx, p, reverse) : tc_ctas_per_sm<64, OpBF16>(ctx, p, reverse));
  const int cap = ctx->tc_ctas_cap > 0 ? std::min(per, ctx->tc_ctas_cap) : per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)ctx->n_sm * cap));
}

template <int HP, class OP>
int launch_tc(fv_ctx ctx, const TcArgs& a, bool reverse, int grid) {
  cudaError_t e;
  if (reverse) {
    e = ensure_smem_attr(ctx, (const void*)mlp_bwd_tc<HP, OP>, a.pl.smem);
    if (e == cudaSuccess) mlp_bwd_tc<HP, OP><<<grid, tc_threads<HP>(), a.pl.smem, ctx->stream>>>(a);
  } else {
    e = ensure_smem_attr(ctx, (const void*)mlp_fwd_tc<HP, OP>, a.pl.smem);
    if (e == cudaSuccess) mlp_fwd_tc<HP, OP><<<grid, tc_threads<HP>(), a.pl.smem, ctx->stream>>>(a);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tensor-core MLP launch failed: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  return FV_OK;
}

int launch_tc_any(fv_ctx ctx, const TcArgs& a, bool reverse, bool fp16, int grid) {
  if (a.pl.HP == 32) return fp16 ? launch_tc<32, OpF16>(ctx, a, reverse, grid) : launch_tc<32, OpBF16>(ctx, a, reverse, grid);
  return fp16 ? launch_tc<64, OpF16>(ctx, a, reverse, grid) : launch_tc<64, OpBF16>(ctx, a, reverse, grid);
}

}  // namespace

bool tc_supported(const EvalPlan& pl) {
  TcPlan p;
  return make_tc_plan(pl, true, &p) && p.smem <= 227 * 1024;
}

int mlp_bwd_tc_blocks(fv_ctx ctx, const EvalPlan& pl) {
  TcPlan p;
  if (!make_tc_plan(pl, true, &p)) return -FV_ERR_UNSUPPORTED;
  return tc_grid(ctx, p, true, pl.prec == FV_FP16, pl.P_tot);
}

size_t mlp_tc_stash_bytes(const EvalPlan& pl) {
  TcPlan p;
  if (!make_tc_plan(pl, true, &p) || p.n_stash == 0) return 0;
  const int64_t n_tiles = (pl.P_tot + kTile - 1) / kTile;
  return (size_t)n_tiles * p.n_stash * p.slot_bytes;
}

int launch_mlp_fwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                      void* U, int* tile_counter, void* stash) {
  TcArgs a;
  if (!make_tc_plan(pl, false, &a.pl)) { set_error("tensor-core path: unsupported network"); return FV_ERR_UNSUPPORTED; }
  a.params = static_cast<const float*>(params);
  a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot;
  a.U = static_cast<float*>(U); a.UB = nullptr; a.gpart = nullptr; a.seed_absmax = nullptr; a.err = ctx->err_dev;
  a.tile_ctr = tile_counter;
  a.stash = static_cast<uint8_t*>(stash);
  const int grid = tc_grid(ctx, a.pl, false, pl.prec == FV_FP16, pl.P_tot);
  cudaError_t e = cudaMemsetAsync(tile_counter, 0, sizeof(int), ctx->stream);
  if (e != cudaSuccess) {
    set_error("tensor-core forward: %s", cudaGetErrorString(e));
    return FV_ERR_CUDA;
  }
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_FWD_TC, &ta);
  const int rc = launch_tc_any(ctx, a, false, pl.prec == FV_FP16, grid);
  time_end(ctx, K_MLP_FWD_TC, ta);
  return rc;
}

int launch_mlp_bwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                      const void* UB, double* gpart, int* nb, const float* seed_absmax, const void* stash) {
  TcArgs a;
  if (!make_tc_plan(pl, true, &a.pl)) { set_error("tensor-core path: unsupported network"); return FV_ERR_UNSUPPORTED; }
  a.params = static_cast<const float*>(params);
  a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot;
  a.U = nullptr; a.UB = static_cast<const float*>(UB); a.gpart = gpart; a.err = ctx->err_dev;
  a.seed_absmax = pl.prec == FV_FP16 ? seed_absmax : nullptr;
  a.tile_ctr = nullptr;
  a.stash = static_cast<uint8_t*>(const_cast<void*>(stash));
  const int grid = mlp_bwd_tc_blocks(ctx, pl);
  *nb = grid;
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_BWD_TC, &ta);
  const int rc = launch_tc_any(ctx, a, true, pl.prec == FV_FP16, grid);
  time_end(ctx, K_MLP_BWD_TC, ta);
  return rc;
}

}  // namespace fv
