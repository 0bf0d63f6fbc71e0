// tanh-MLP forward with forward-mode tangents and its reverse sweep on CUDA
// cores (FP64 and FP32 FMA paths).  Sec. 2.2 Eq. (NN): u = l o T^(h) o ... o T^(1).
//
// Forward, per hidden layer i and point p (three streams sharing W_i):
//   z = W h + b,  z'_x = W h'_x,  z'_y = W h'_y
//   t = tanh z,   t'_s = (1 - t^2) z'_s          (h_0 = (x, y), h'_x = (1,0), h'_y = (0,1))
// Output layer (linear): u = w.h, u_x = w.h'_x, u_y = w.h'_y (+ bias on u).
//
// Reverse, given seeds (ubar, u_xbar, u_ybar) per point and the stored
// (t, t'_x, t'_y) of each hidden layer:
//   zbar_s' = (1 - t^2) tbar'_s
//   zbar    = (1 - t^2) tbar - 2 t (t'_x tbar'_x + t'_y tbar'_y)
//   Wbar += zbar h^T + sum_s zbar'_s h'_s^T,  bbar += zbar,
//   hbar = W^T zbar,  hbar'_s = W^T zbar'_s
// (the identity (1-t^2) z'_s = t'_s removes z' from the stored state).
//
// A CTA handles tiles of TP points.  Activations live in shared memory as
// [stream][neuron][TPS] (TPS = TP padded so that TPS/4 is odd: consecutive
// rows fall in distinct bank groups); each hidden layer has one extra row, the
// constant 1, so that a bias is one more weight column.  Each map is a small
// GEMM on register tiles (4 rows x 4 points x 3 streams, or 4 x 4 weight
// entries over 4-point steps) whose lane pairs share one operand, updated by
// packed FP32 FMAs.  The forward kernel computes u, u_x, u_y per point and
// (for a gradient) stores every tile's hidden layers; the reverse kernel reads
// them back by bulk copies (or recomputes them), sweeps the maps top down with
// the adjoint GEMM and the weight-gradient GEMM running side by side on
// separate warps, and accumulates the weight gradient of all its tiles in
// shared memory, written out once per CTA (deterministic per-CTA partials).
#include <algorithm>

#include "fv_internal.cuh"
#include "fv_tcgen05.cuh"

namespace fv {
namespace {

constexpr int kThreads = 256;      // forward kernel
constexpr int kThreadsBwd = 512;   // reverse kernel: its shared memory allows one CTA per SM, so 16 warps

// Hidden layers are stored with one row more than their width (the constant
// 1 of the bias column), so a hidden map's padded input count and a hidden
// layer's padded row count are ru4(width + 1).
struct WLayout {
  int woff[kMaxLayers];  // padded W_i: rows x ld, row-major, zero padding
  int boff[kMaxLayers];  // padded b_i: rows
  int ld[kMaxLayers];    // ru4(in), ru4(in + 1) for i >= 1
  int rows[kMaxLayers];  // ru4(out + 1) for hidden outputs, ru4(out) for the output map
  int total;             // elements (multiple of 4)
};

inline int ru4(int v) { return (v + 3) & ~3; }

WLayout make_layout(const MlpShape& s) {
  WLayout l;
  int o = 0;
  for (int i = 0; i < s.L; ++i) {
    l.ld[i] = ru4(s.w[i] + (i >= 1 ? 1 : 0));
    l.rows[i] = ru4(s.w[i + 1] + (i + 1 < s.L ? 1 : 0));
    l.woff[i] = o; o += l.ld[i] * l.rows[i];
    l.boff[i] = o; o += l.rows[i];
  }
  l.total = o;
  return l;
}

int max_hidden_pad(const MlpShape& s) {
  int d = 4;
  for (int i = 1; i < s.L; ++i) d = std::max(d, ru4(s.w[i] + 1));
  return d;
}

int tps_for(int TP) {
  int t = TP;
  if (((t / 4) & 1) == 0) t += 4;
  return t;
}

struct FwdArgs {
  MlpShape sh;
  WLayout wl;
  int DP, TP, TPS;
  const void* params;
  const double* Xm;
  int64_t P_mesh;
  const double* Xe;
  int64_t P_tot;
  void* U;       // [3][P_tot]
  void* stash;   // null, or per tile the hidden layers in the reverse kernel's layout
};

struct BwdArgs {
  MlpShape sh;
  WLayout wl;
  int DP, TP, TPS;
  const void* params;
  const double* Xm;
  int64_t P_mesh;
  const double* Xe;
  int64_t P_tot;
  const void* UB;   // [3][P_tot] seeds
  double* gpart;    // [gridDim][n_params]
  const void* stash;   // null (recompute the forward), or the forward kernel's stored hidden layers
  int* err;            // FV_ERR_TIMEOUT when a bounded wait gives up
};

__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ld2(const double* p, double v[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void st2(double* p, const double v[2]) { *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]); }
// PP (4 or 2) consecutive values
template <int PP, class R> __device__ __forceinline__ void ldp(const R* p, R v[PP]) {
  if constexpr (PP == 4) ld4(p, v);
  else if constexpr (PP == 2) ld2(p, v);
  else v[0] = p[0];
}
template <int PP, class R> __device__ __forceinline__ void stp(R* p, const R v[PP]) {
  if constexpr (PP == 4) st4(p, v);
  else if constexpr (PP == 2) st2(p, v);
  else p[0] = v[0];
}
__device__ __forceinline__ float tanh_r(float v) { return tanhf(v); }
__device__ __forceinline__ double tanh_r(double v) { return tanh(v); }

// Value pairs for the GEMM inner loops.  In FP32 a pair is updated by one
// packed FMA instruction (two correctly rounded FP32 FMAs, the same results
// as two fmaf calls) so that the loops issue half as many FMA instructions;
// in FP64 a pair is two scalar FMAs.
template <class R> struct PairOf;
template <> struct PairOf<float> { using T = float2; };
template <> struct PairOf<double> { using T = double2; };
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pdup(float v) { return make_float2(v, v); }
__device__ __forceinline__ double2 pdup(double v) { return make_double2(v, v); }
template <class P> __device__ __forceinline__ P pzero() { P z; z.x = 0; z.y = 0; return z; }
// 2*NP consecutive values as NP pairs (16-byte aligned when 2*NP*sizeof >= 16)
template <int NP> __device__ __forceinline__ void ldpair(const float* p, float2* v) {
  if constexpr (NP == 2) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = make_float2(t.x, t.y); v[1] = make_float2(t.z, t.w);
  } else {
#pragma unroll
    for (int j = 0; j < NP; ++j) v[j] = reinterpret_cast<const float2*>(p)[j];
  }
}
template <int NP> __device__ __forceinline__ void ldpair(const double* p, double2* v) {
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = reinterpret_cast<const double2*>(p)[j];
}

// Per-CTA weight-gradient accumulator in shared memory, one entry per
// parameter in the path's precision: a tile's contribution is formed in
// registers over its 3 x TP point-streams and added once per tile, and the
// per-CTA partials are summed in FP64 across CTAs.  (A compensated FP32 pair
// per entry took twice the shared memory, and with it half the tile size.)
template <class R> struct GradAcc {
  R* a;
  __device__ __forceinline__ void zero(int i) { a[i] = (R)0; }
  __device__ __forceinline__ void add(int i, R v) { a[i] += v; }
  __device__ __forceinline__ double get(int i) const { return (double)a[i]; }
};

// Load the padded weights into shared memory (zero padding).
template <class R>
__device__ void load_weights(const MlpShape& sh, const WLayout& wl, const R* __restrict__ p, R* sW) {
  for (int i = 0; i < sh.L; ++i) {
    const int in = sh.w[i], out = sh.w[i + 1], ld = wl.ld[i], rows = wl.rows[i];
    const R* W = p + sh.off[i];
    for (int idx = threadIdx.x; idx < rows * ld; idx += blockDim.x) {
      const int o = idx / ld, k = idx - o * ld;
      sW[wl.woff[i] + idx] = (o < out && k < in) ? W[o * in + k] : (R)0;
    }
    for (int o = threadIdx.x; o < rows; o += blockDim.x) sW[wl.boff[i] + o] = o < out ? W[out * in + o] : (R)0;
  }
}

// Tile points: X (FP64) -> sX[2][TPS] in R; points past P_tot get (0,0).
template <class R>
__device__ void load_points(const double* __restrict__ Xm, int64_t P_mesh, const double* __restrict__ Xe,
                            int64_t P_tot, int64_t p_base, int TP, int TPS, R* sX) {
  for (int p = threadIdx.x; p < TP; p += blockDim.x) {
    const int64_t gp = p_base + p;
    double x = 0.0, y = 0.0;
    if (gp < P_mesh) { x = Xm[2 * gp]; y = Xm[2 * gp + 1]; }
    else if (gp < P_tot) { x = Xe[2 * (gp - P_mesh)]; y = Xe[2 * (gp - P_mesh) + 1]; }
    sX[p] = (R)x;
    sX[TPS + p] = (R)y;
  }
}

// Layer 0: inputs (x, y) with unit tangents; row `out` is the constant 1
// (tangents 0), the input that carries the next map's bias.  One thread per
// (row, group of PW points).
template <class R, int PW>
__device__ void fwd_layer0(const R* W, const R* b, int ld, int out, int rows, const R* sX, R* B, int TP, int TPS,
                           int plane) {
  const int n_pg = TP / PW;
  for (int mt = threadIdx.x; mt < rows * n_pg; mt += blockDim.x) {
    const int pg = mt % n_pg, o = mt / n_pg, p0 = pg * PW;
    R x[PW], y[PW], t4[PW], x4[PW], y4[PW];
    ldp<PW>(sX + p0, x);
    ldp<PW>(sX + TPS + p0, y);
    const R w0 = W[o * ld], w1 = W[o * ld + 1], bo = b[o];
    const bool one = o == out;
#pragma unroll
    for (int pp = 0; pp < PW; ++pp) {
      const R t = tanh_r(w0 * x[pp] + w1 * y[pp] + bo), sd = (R)1 - t * t;
      t4[pp] = one ? (R)1 : t;
      x4[pp] = one ? (R)0 : sd * w0;
      y4[pp] = one ? (R)0 : sd * w1;
    }
    stp<PW>(B + o * TPS + p0, t4);
    stp<PW>(B + plane + o * TPS + p0, x4);
    stp<PW>(B + 2 * plane + o * TPS + p0, y4);
  }
}

// ----------------------------------------------------------------------------- reverse kernel
// Per tile the reverse kernel recomputes the forward (keeping every hidden
// layer's (t, t'_x, t'_y) in shared memory), then sweeps the maps top down.
// Row `out` of each stored hidden layer holds the constant 1 (tangents 0), so
// the weight-gradient GEMM of the map above yields the bias gradient as one
// more column (b is W's column `in` against a constant input).  A sweep step
// runs two GEMMs that only read Zbar_i and S_{i-1}: the adjoint GEMM
// (hbar = W^T zbar, fused with the tanh-rule adjoint of layer i-1) on the
// first kTbarThreads threads and the weight-gradient GEMM on the rest.
constexpr int kTbarThreads = 128;
constexpr size_t kBwdStaticSmem = 1024;   // bound on the reverse kernel's static shared memory
constexpr int kWgThreads = kThreadsBwd - kTbarThreads;
constexpr int kWgBarrier = 1;   // named barrier of the weight-gradient threads

// Points per thread tile: four in FP32, two in FP64 (register budget).
template <class R> struct PointsPerTile { static constexpr int v = sizeof(R) == 4 ? 4 : 2; };

// Lane pairs.  A 16-byte shared-memory load whose even and odd lanes read the
// same addresses is served in two half-warp passes; otherwise it takes four
// quarter-warp passes (measured on this part: about 2.4 against 4 cycles per
// warp, more with bank conflicts).  The GEMM tiles below therefore give the
// two lanes of a pair the same point group (or output rows) and different
// row groups: the larger operand is read at the pair rate.  A pair index q
// maps to (row-group pair, point group) with the point group fastest, so the
// eight pairs of a half-warp read eight different 16-byte chunks of one row.

// Pair index q -> (row-group pair, point group).  Point groups go in blocks
// of eight (the eight pairs of a half-warp read eight chunks of one row, in
// distinct bank groups); the groups past the last full block of eight are
// spread over the row-group pairs on their own, so no half-warp reads two
// chunks eight apart (which share banks).
__device__ __forceinline__ void pair_split(int q, int n_pg, int n_rgp, int& pg, int& rgp) {
  const int full = n_pg & ~7, rem = n_pg - full;
  if (q < n_rgp * full || rem == 0) {
    pg = q % full;
    rgp = q / full;
  } else {
    const int r = q - n_rgp * full;
    pg = full + r % rem;
    rgp = r / rem;
  }
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Forward GEMM of hidden map i: B = tanh-rule(W A + b) for the three streams,
// row `out` of B set to the constant 1 (tangents 0).  Thread tile: rows
// o = og + n_og*oo (oo < 4), points p0..p0+PW-1, three streams; the lanes of
// a pair share the points (og = 2 x pair row group + lane parity); k runs
// over the padded inputs four at a time (padded weight columns are zero, so
// the constant row adds nothing).  SPLIT: point groups as in pair_split (the
// forward kernel: 3.5% faster), else point group fastest (the reverse
// kernel's recompute path; either gives each element the same arithmetic,
// only the thread that computes it differs).  The k range of a tile is split between
// two threads in different warps of one scheduler: the second leaves its
// partial sums in B at the tile's own places, and after a CTA barrier the
// first adds them and applies the tanh rule.  Every thread of the CTA calls
// this (barriers).
template <class R, int PW, bool SPLIT>
__device__ void fwd_gemm(const R* __restrict__ W, const R* __restrict__ b, int ld, int out, int rows,
                         const R* __restrict__ A, R* __restrict__ B, int TP, int TPS, int plane) {
  const int n_og = rows >> 2, n_pg = TP / PW, slots = 2 * ((n_og + 1) >> 1) * n_pg;
  const int T = blockDim.x >> 1, half = threadIdx.x >= T ? 1 : 0;
  const int kh = (((ld >> 2) + 1) >> 1) << 2;         // first k of the second half
  const int k0 = half ? kh : 0, k1 = half ? ld : kh;
  for (int base = 0; base < slots; base += T) {
    const int q2 = base + threadIdx.x - half * T, q = q2 >> 1;
    int pg, ogp;
    if (SPLIT) {
      pair_split(q, n_pg, (n_og + 1) >> 1, pg, ogp);
    } else {
      pg = q % n_pg;
      ogp = q / n_pg;
    }
    const int og = 2 * ogp + (q2 & 1), p0 = pg * PW;
    const bool active = q2 < slots && og < n_og;
    using P = typename PairOf<R>::T;
    constexpr int NP = PW / 2;
    P acc[3][4][NP];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[s][i][j] = pzero<P>();
    const int wst = n_og * ld;
    if (active) {
      const R* Wr = W + og * ld;
      const R* Ap = A + p0;
      for (int k = k0; k < k1; k += 4) {
        R w[4][4];
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) ld4(Wr + oo * wst + k, w[oo]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          P a0[NP], a1[NP], a2[NP];
          const R* ak = Ap + (k + kk) * TPS;
          ldpair<NP>(ak, a0);
          ldpair<NP>(ak + plane, a1);
          ldpair<NP>(ak + 2 * plane, a2);
#pragma unroll
          for (int oo = 0; oo < 4; ++oo) {
            const P wd = pdup(w[oo][kk]);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
              acc[0][oo][j] = pfma(wd, a0[j], acc[0][oo][j]);
              acc[1][oo][j] = pfma(wd, a1[j], acc[1][oo][j]);
              acc[2][oo][j] = pfma(wd, a2[j], acc[2][oo][j]);
            }
          }
        }
      }
    }
    if constexpr (SPLIT) {
      // each half finishes two of the four row groups (adds the other half's
      // partial sums and applies the tanh rule), sharing the epilogue's tanh
      // work; a row's value is (first half + second half) + bias as below
      auto finishes = [&](int oo) { return (oo >> 1) == half; };
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
        if (active && !finishes(oo)) {
          R* Bo = B + (og + oo * n_og) * TPS + p0;
#pragma unroll
          for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int j = 0; j < NP; ++j) reinterpret_cast<P*>(Bo + s * plane)[j] = acc[s][oo][j];
        }
      __syncthreads();
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
        if (active && finishes(oo)) {
          const int o = og + oo * n_og;
          R* Bo = B + o * TPS + p0;
          R q0[PW], q1[PW], qq2[PW];
          ldp<PW>(Bo, q0);
          ldp<PW>(Bo + plane, q1);
          ldp<PW>(Bo + 2 * plane, qq2);
          const R bo = b[o];
          const bool one = o == out;
          R t4[PW], x4[PW], y4[PW];
#pragma unroll
          for (int pp = 0; pp < PW; ++pp) {
            const P c0 = acc[0][oo][pp >> 1], c1 = acc[1][oo][pp >> 1], c2 = acc[2][oo][pp >> 1];
            const R t = tanh_r(((pp & 1) ? c0.y : c0.x) + q0[pp] + bo), sd = (R)1 - t * t;
            t4[pp] = one ? (R)1 : t;
            x4[pp] = one ? (R)0 : sd * (((pp & 1) ? c1.y : c1.x) + q1[pp]);
            y4[pp] = one ? (R)0 : sd * (((pp & 1) ? c2.y : c2.x) + qq2[pp]);
          }
          stp<PW>(Bo, t4);
          stp<PW>(Bo + plane, x4);
          stp<PW>(Bo + 2 * plane, y4);
        }
    } else {
      if (active && half == 1)
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) {
          R* Bo = B + (og + oo * n_og) * TPS + p0;
#pragma unroll
          for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int j = 0; j < NP; ++j) reinterpret_cast<P*>(Bo + s * plane)[j] = acc[s][oo][j];
        }
      __syncthreads();
      if (active && half == 0)
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) {
          const int o = og + oo * n_og;
          R* Bo = B + o * TPS + p0;
          R q0[PW], q1[PW], qq2[PW];
          ldp<PW>(Bo, q0);
          ldp<PW>(Bo + plane, q1);
          ldp<PW>(Bo + 2 * plane, qq2);
          const R bo = b[o];
          const bool one = o == out;
          R t4[PW], x4[PW], y4[PW];
#pragma unroll
          for (int pp = 0; pp < PW; ++pp) {
            const P c0 = acc[0][oo][pp >> 1], c1 = acc[1][oo][pp >> 1], c2 = acc[2][oo][pp >> 1];
            const R t = tanh_r(((pp & 1) ? c0.y : c0.x) + q0[pp] + bo), sd = (R)1 - t * t;
            t4[pp] = one ? (R)1 : t;
            x4[pp] = one ? (R)0 : sd * (((pp & 1) ? c1.y : c1.x) + q1[pp]);
            y4[pp] = one ? (R)0 : sd * (((pp & 1) ? c2.y : c2.x) + qq2[pp]);
          }
          stp<PW>(Bo, t4);
          stp<PW>(Bo + plane, x4);
          stp<PW>(Bo + 2 * plane, y4);
        }
    }
    tc::fence_proxy_async();   // B may be read next by a bulk copy
    __syncthreads();
  }
}

// tanh-rule adjoint of a stored layer (t, t'_x, t'_y) applied to (tbar, tbar'_x, tbar'_y).
template <class R>
__device__ __forceinline__ void tanh_adjoint(R t, R tx, R ty, R bt, R bx, R by, R& z0, R& z1, R& z2) {
  const R s = (R)1 - t * t;
  z0 = s * bt - (R)2 * t * (tx * bx + ty * by);
  z1 = s * bx;
  z2 = s * by;
}

// Adjoint GEMM of hidden map i fused with the tanh-rule adjoint of layer i-1:
//   Tb[s][k][p] = sum_{o < out} W[o][k] Zin[s][o][p], then Zout = adjoint(S, Tb)
// with S the stored layer i-1 (its constant row and padding give Zout = 0).
// Thread tile: k = 4kg..4kg+3 (one 16-byte load of W per o), points
// p0..p0+PW-1 shared by the lanes of a pair (kg = 2 x pair group + lane
// parity), three streams.  Threads tid < nthr of the CTA take part.
template <class R, int PW>
__device__ void tbar_gemm(const R* __restrict__ W, int ld, int out, int krows, const R* __restrict__ Zin,
                          const R* __restrict__ S, R* __restrict__ Zout, int TP, int TPS, int plane, int tid,
                          int nthr) {
  const int n_kg = krows >> 2, n_pg = TP / PW, n_pairs = ((n_kg + 1) >> 1) * n_pg;
  for (int q2 = tid; q2 < 2 * n_pairs; q2 += nthr) {
    // (point group fastest; the split of pair_split measured no faster here)
    const int q = q2 >> 1, pg = q % n_pg, kg = 2 * (q / n_pg) + (q2 & 1), p0 = pg * PW, k0 = kg << 2;
    if (kg >= n_kg) continue;
    using P = typename PairOf<R>::T;
    constexpr int NP = PW / 2;
    P acc[3][4][NP];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[s][i][j] = pzero<P>();
    const R* Wc = W + k0;
    const R* Zp = Zin + p0;
#pragma unroll 2
    for (int o = 0; o < out; ++o) {
      R w[4];
      P z0[NP], z1[NP], z2[NP];
      ld4(Wc + o * ld, w);
      ldpair<NP>(Zp + o * TPS, z0);
      ldpair<NP>(Zp + plane + o * TPS, z1);
      ldpair<NP>(Zp + 2 * plane + o * TPS, z2);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const P wd = pdup(w[kk]);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          acc[0][kk][j] = pfma(wd, z0[j], acc[0][kk][j]);
          acc[1][kk][j] = pfma(wd, z1[j], acc[1][kk][j]);
          acc[2][kk][j] = pfma(wd, z2[j], acc[2][kk][j]);
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int r = (k0 + kk) * TPS + p0;
      R t[PW], tx[PW], ty[PW], z0[PW], z1[PW], z2[PW];
      ldp<PW>(S + r, t);
      ldp<PW>(S + plane + r, tx);
      ldp<PW>(S + 2 * plane + r, ty);
#pragma unroll
      for (int pp = 0; pp < PW; ++pp) {
        const P c0 = acc[0][kk][pp >> 1], c1 = acc[1][kk][pp >> 1], c2 = acc[2][kk][pp >> 1];
        tanh_adjoint<R>(t[pp], tx[pp], ty[pp], (pp & 1) ? c0.y : c0.x, (pp & 1) ? c1.y : c1.x,
                        (pp & 1) ? c2.y : c2.x, z0[pp], z1[pp], z2[pp]);
      }
      stp<PW>(Zout + r, z0);
      stp<PW>(Zout + plane + r, z1);
      stp<PW>(Zout + 2 * plane + r, z2);
    }
  }
}

// Gradient entry of W[o][k] (k < in) or of b[o] (k == in, the constant column).
__device__ __forceinline__ int wgrad_index(int off, int out, int in, int o, int k) {
  return k < in ? off + o * in + k : off + out * in + o;
}

// Weight-gradient GEMM of map i: G[o][k] += sum over streams s and points p of
// Zin[s][o][p] H[s][k][p], o < out, k <= in (k == in: the bias, H's constant
// row).  4 x 4 (o, k) tiles with interleaved rows o = og + n_og*oo,
// k = kg + n_kg*kk; the lanes of a pair share og (kg = 2 x pair group + lane
// parity).  The (stream, 4-point) steps of a tile are split between two
// threads: the second leaves its sum in `scratch`, and after a barrier of the
// nthr weight-gradient threads the first adds it and accumulates into G (a
// fixed order).  Every weight-gradient thread calls this (barriers).
template <class R>
__device__ void wgrad_gemm(const R* __restrict__ Zin, const R* __restrict__ H, int out, int in, int TP, int TPS,
                           int plane, GradAcc<R> G, int off, R* __restrict__ scratch, int tid, int nthr) {
  const int n_og = (out + 3) >> 2, n_kg = (in + 4) >> 2, n_kgp = (n_kg + 1) >> 1;
  const int slots = 2 * n_og * n_kgp;                 // thread slots of one half (pairs x 2)
  const int n_p4 = TP >> 2, n_steps = 3 * n_p4;
  const int T = nthr >> 1, half = tid >= T ? 1 : 0;
  for (int base = 0; base < slots; base += T) {
    const int q2 = base + tid - half * T, q = q2 >> 1;
    const int og = q / n_kgp, kg = 2 * (q - og * n_kgp) + (q2 & 1);
    const bool active = q2 < slots && og < n_og && kg < n_kg;
    const int m = og * n_kg + kg;
    using P = typename PairOf<R>::T;
    P acc2[4][4];                                     // (even-point, odd-point) partial sums
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc2[i][j] = pzero<P>();
    if (active) {
      const int s0 = half ? n_steps / 2 : 0, s1 = half ? n_steps : n_steps / 2;
      int s = s0 / n_p4, p = (s0 - s * n_p4) << 2;
      const R* Zr = Zin + og * TPS;
      const R* Hr = H + kg * TPS;
      const int zst = n_og * TPS, hst = n_kg * TPS;
      for (int st = s0; st < s1; ++st) {
        const int base = s * plane + p;
        P z[4][2], h[4][2];
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) ldpair<2>(Zr + base + oo * zst, z[oo]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) ldpair<2>(Hr + base + kk * hst, h[kk]);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int oo = 0; oo < 4; ++oo)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) acc2[oo][kk] = pfma(z[oo][j], h[kk][j], acc2[oo][kk]);
        p += 4;
        if (p == TP) { p = 0; ++s; }
      }
    }
    R acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = acc2[i][j].x + acc2[i][j].y;
    if (active && half == 1)
#pragma unroll
      for (int i = 0; i < 4; ++i) st4(scratch + m * 16 + 4 * i, acc[i]);
    named_sync(kWgBarrier, nthr);
    if (active && half == 0) {
#pragma unroll
      for (int oo = 0; oo < 4; ++oo) {
        R o4[4];
        ld4(scratch + m * 16 + 4 * oo, o4);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int o = og + oo * n_og, k = kg + kk * n_kg;
          if (o < out && k <= in) G.add(wgrad_index(off, out, in, o, k), acc[oo][kk] + o4[kk]);
        }
      }
    }
    named_sync(kWgBarrier, nthr);
  }
}

// Output map (linear) from the seeds (ubar, u_xbar, u_ybar[, epsbar]) per point:
//   Tb[s][k][p] = w_u[k] seed_s[p] (+ w_e[k] epsbar[p] on the value stream),
//   Zout = tanh-rule adjoint of the last hidden layer S applied to Tb,
//   w_ubar[k] = sum_p (ubar t + u_xbar t'_x + u_ybar t'_y)[k][p],
//   w_ebar[k] = sum_p epsbar t[k][p]   (row k == in of S is 1: the biases).
// One thread per (k, point group) leaves its partial sums in scratch[k][pg][2];
// after a barrier they are summed in a fixed order.
template <class R, int PW>
__device__ void out_adjoint(const R* __restrict__ Wl, int ld, int in, bool two, int krows, const R* __restrict__ sSeed,
                            const R* __restrict__ S, R* __restrict__ Zout, int TP, int TPS, int plane, GradAcc<R> G,
                            int off, R* __restrict__ scratch) {
  const int n_pg = TP / PW;
  for (int mt = threadIdx.x; mt < krows * n_pg; mt += blockDim.x) {
    const int pg = mt % n_pg, k = mt / n_pg, p0 = pg * PW, r = k * TPS + p0;
    const R w = Wl[k], we = two ? Wl[ld + k] : (R)0;
    R t[PW], tx[PW], ty[PW], su[PW], sx[PW], sy[PW], se[PW], z0[PW], z1[PW], z2[PW];
    ldp<PW>(S + r, t);
    ldp<PW>(S + plane + r, tx);
    ldp<PW>(S + 2 * plane + r, ty);
    ldp<PW>(sSeed + p0, su);
    ldp<PW>(sSeed + TPS + p0, sx);
    ldp<PW>(sSeed + 2 * TPS + p0, sy);
    if (two) ldp<PW>(sSeed + 3 * TPS + p0, se);
    R gu = 0, ge = 0;
#pragma unroll
    for (int pp = 0; pp < PW; ++pp) {
      const R e = two ? se[pp] : (R)0;
      tanh_adjoint<R>(t[pp], tx[pp], ty[pp], w * su[pp] + we * e, w * sx[pp], w * sy[pp], z0[pp], z1[pp], z2[pp]);
      gu += su[pp] * t[pp] + sx[pp] * tx[pp] + sy[pp] * ty[pp];
      ge += e * t[pp];
    }
    stp<PW>(Zout + r, z0);
    stp<PW>(Zout + plane + r, z1);
    stp<PW>(Zout + 2 * plane + r, z2);
    scratch[2 * mt] = gu;
    scratch[2 * mt + 1] = ge;
  }
  __syncthreads();
  const int nout = two ? 2 : 1;
  for (int idx = threadIdx.x; idx < nout * (in + 1); idx += blockDim.x) {
    const int j = idx / (in + 1), k = idx - j * (in + 1);
    R acc = 0;
    for (int pg = 0; pg < n_pg; ++pg) acc += scratch[2 * (k * n_pg + pg) + j];
    G.add(wgrad_index(off, nout, in, j, k), acc);
  }
}

// Map 0 (inputs (x, y), tangents (1, 0) and (0, 1)):
//   W0bar[o][0] = sum_p Z0[o][p] x_p + Z1[o][p],  W0bar[o][1] = sum_p Z0[o][p] y_p + Z2[o][p],
//   b0bar[o] = sum_p Z0[o][p].
// Partial sums per (o, point group) in scratch[o][pg][3], then a fixed-order sum.
template <class R, int PW>
__device__ void wgrad_map0(const R* __restrict__ Zin, const R* __restrict__ sX, int out, int TP, int TPS, int plane,
                           GradAcc<R> G, int off, R* __restrict__ scratch) {
  const int n_pg = TP / PW;
  for (int mt = threadIdx.x; mt < out * n_pg; mt += blockDim.x) {
    const int pg = mt % n_pg, o = mt / n_pg, p0 = pg * PW, r = o * TPS + p0;
    R z0[PW], z1[PW], z2[PW], x[PW], y[PW];
    ldp<PW>(Zin + r, z0);
    ldp<PW>(Zin + plane + r, z1);
    ldp<PW>(Zin + 2 * plane + r, z2);
    ldp<PW>(sX + p0, x);
    ldp<PW>(sX + TPS + p0, y);
    R g0 = 0, g1 = 0, gb = 0;
#pragma unroll
    for (int pp = 0; pp < PW; ++pp) {
      g0 += z0[pp] * x[pp] + z1[pp];
      g1 += z0[pp] * y[pp] + z2[pp];
      gb += z0[pp];
    }
    scratch[3 * mt] = g0;
    scratch[3 * mt + 1] = g1;
    scratch[3 * mt + 2] = gb;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * out; idx += blockDim.x) {
    const int o = idx / 3, c = idx - 3 * o;
    R acc = 0;
    for (int pg = 0; pg < n_pg; ++pg) acc += scratch[3 * (o * n_pg + pg) + c];
    G.add(wgrad_index(off, out, 2, o, c), acc);
  }
}

// ----------------------------------------------------------------------------- forward kernel
// Per tile of TP points: layer 0, the hidden maps (the same GEMM as the
// reverse kernel's recompute, two activation buffers alternating), then the
// output map with one thread per (point, output stream).
template <class R>
__global__ void __launch_bounds__(kThreads) mlp_fwd_simt(FwdArgs a) {
  constexpr int PW = PointsPerTile<R>::v;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sW = reinterpret_cast<R*>(smem);
  const int plane = a.DP * a.TPS;
  R* bufA = sW + a.wl.total;
  R* bufB = bufA + 3 * plane;
  R* sX = bufB + 3 * plane;
  const MlpShape& sh = a.sh;
  const WLayout& wl = a.wl;
  load_weights<R>(sh, wl, reinterpret_cast<const R*>(a.params), sW);
  R* U = reinterpret_cast<R*>(a.U);
  const int64_t n_tiles = (a.P_tot + a.TP - 1) / a.TP;
  const int L = sh.L, TP = a.TP, TPS = a.TPS;
  const int in = sh.w[L - 1], nout = sh.w[L];     // a second output eps(x, y) (Sec. 4.7.2)
  // stash: each hidden layer of the tile leaves by one bulk copy issued by
  // thread 0 once the layer is complete; a buffer is overwritten only after
  // the copy that reads it has finished reading
  const uint32_t slot_bytes = (uint32_t)(3 * (size_t)plane * sizeof(R));
  char* stash = static_cast<char*>(a.stash);
  const bool lead = threadIdx.x == 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p_base = tile * TP;
    char* st_tile = stash ? stash + (size_t)tile * (L - 1) * slot_bytes : nullptr;
    if (stash && lead) tc::bulk_wait_read<0>();
    __syncthreads();
    load_points<R>(a.Xm, a.P_mesh, a.Xe, a.P_tot, p_base, TP, TPS, sX);
    __syncthreads();
    R* A = bufA;
    R* B = bufB;
    fwd_layer0<R, PW>(sW + wl.woff[0], sW + wl.boff[0], wl.ld[0], sh.w[1], wl.rows[0], sX, A, TP, TPS, plane);
    tc::fence_proxy_async();
    __syncthreads();
    if (stash && lead) tc::bulk_store(st_tile, A, slot_bytes);
    for (int i = 1; i < L - 1; ++i) {
      if (stash) {                 // B's previous layer (two maps down) has left
        if (lead) tc::bulk_wait_read<1>();
        __syncthreads();
      }
      fwd_gemm<R, PW, true>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i + 1], wl.rows[i], A, B, TP, TPS,
                            plane);
      if (stash && lead) tc::bulk_store(st_tile + (size_t)i * slot_bytes, B, slot_bytes);
      R* t = A; A = B; B = t;
    }
    // output map: stream 0 of output 0 is u, streams 1, 2 its tangents; output 1 is eps (value only)
    const R* Wl = sW + wl.woff[L - 1];
    const int ldl = wl.ld[L - 1];
    for (int idx = threadIdx.x; idx < (nout == 2 ? 4 : 3) * TP; idx += blockDim.x) {
      const int j = idx / TP, p = idx - j * TP;
      const int64_t gp = p_base + p;
      if (gp >= a.P_tot) continue;
      const R* w = Wl + (j == 3 ? ldl : 0);
      const R* h = A + (j == 3 ? 0 : j) * plane + p;
      R acc0 = j == 0 ? sW[wl.boff[L - 1]] : j == 3 ? sW[wl.boff[L - 1] + 1] : (R)0, acc1 = 0;
      int k = 0;
      for (; k + 1 < in; k += 2) {
        acc0 = fma(w[k], h[k * TPS], acc0);
        acc1 = fma(w[k + 1], h[(k + 1) * TPS], acc1);
      }
      if (k < in) acc0 = fma(w[k], h[k * TPS], acc0);
      U[(int64_t)j * a.P_tot + gp] = acc0 + acc1;
    }
  }
  if (stash && lead) tc::bulk_wait_all();
}

template <class R>
__global__ void __launch_bounds__(kThreadsBwd) mlp_bwd_simt(BwdArgs a) {
  constexpr int PW = PointsPerTile<R>::v;
  extern __shared__ __align__(16) unsigned char smem[];
  const MlpShape& sh = a.sh;
  const WLayout& wl = a.wl;
  const int L = sh.L, TP = a.TP, TPS = a.TPS;
  const int plane = a.DP * TPS;
  GradAcc<R> G;
  G.a = reinterpret_cast<R*>(smem);                               // [n_params] (rounded up to 4)
  R* sW = G.a + ((sh.n_params + 3) & ~3);
  R* S = sW + wl.total;                                           // [L-1][3][DP][TPS]
  R* Z = S + (size_t)(L - 1) * 3 * plane;                         // [2][3][DP][TPS]: zbar of two layers
  R* sX = Z + 6 * plane;                                          // [2][TPS]
  R* sSeed = sX + 2 * TPS;                                        // [4][TPS]: u, u_x, u_y (, eps) seeds
  R* sScr = sSeed + 4 * TPS;                                      // partial sums
  const bool two = sh.w[L] == 2;
  const int64_t n_tiles = (a.P_tot + TP - 1) / TP;
  // stash: hidden layer i of a tile arrives in its slot S_i by one bulk copy
  // on barrier sbar[i]; the copy for the CTA's next tile is issued as soon as
  // the current tile has finished with the slot
  __shared__ uint64_t sbar[kMaxLayers];
  static_assert(sizeof(sbar) <= kBwdStaticSmem, "static shared memory exceeds the reserve");
  const char* stash = static_cast<const char*>(a.stash);
  const uint32_t slot_bytes = (uint32_t)(3 * (size_t)plane * sizeof(R));
  const size_t tile_bytes = (size_t)(L - 1) * slot_bytes;
  uint32_t sphase = 0;                 // parity to wait for, per slot
  uint32_t pending = 0;                // slots with a copy in flight (thread 0)
  const uint64_t pol = stash ? tc::l2_evict_first() : 0;
  auto issue = [&](int i, int64_t t) {
    if (threadIdx.x != 0 || t >= n_tiles) return;
    tc::fence_proxy_async();
    tc::mbar_expect_tx(&sbar[i], slot_bytes);
    tc::bulk_load(S + (size_t)i * 3 * plane, stash + (size_t)t * tile_bytes + (size_t)i * slot_bytes, slot_bytes,
                  &sbar[i], pol);
    pending |= 1u << i;
  };
  bool failed = false;
  auto arrive = [&](int i) {           // every thread: slot i holds the current tile's layer i
    const bool ok = tc::mbar_wait(&sbar[i], (sphase >> i) & 1u);
    if (ok) {                          // a copy that did not arrive stays pending (waited for at exit)
      sphase ^= 1u << i;
      if (threadIdx.x == 0) pending &= ~(1u << i);
    }
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, FV_ERR_TIMEOUT);
      failed = true;
    }
    return !failed;
  };
  if (stash) {
    if (threadIdx.x == 0)
      for (int i = 0; i < L - 1; ++i) tc::mbar_init(&sbar[i], 1);
    tc::fence_proxy_async();
    __syncthreads();
    for (int i = 0; i < L - 1; ++i) issue(i, blockIdx.x);
  }
  for (int i = threadIdx.x; i < sh.n_params; i += blockDim.x) G.zero(i);
  load_weights<R>(sh, wl, reinterpret_cast<const R*>(a.params), sW);
  const R* UB = reinterpret_cast<const R*>(a.UB);
  // point and seeds of thread p < TP for the next tile, fetched a tile ahead
  double px = 0.0, py = 0.0;
  R sd[4] = {(R)0, (R)0, (R)0, (R)0};
  auto fetch = [&](int64_t t) {
    const int64_t gp = t * TP + threadIdx.x;
    px = 0.0; py = 0.0;
    sd[0] = sd[1] = sd[2] = sd[3] = (R)0;
    if (threadIdx.x >= TP || t >= n_tiles) return;
    if (gp < a.P_mesh) { px = a.Xm[2 * gp]; py = a.Xm[2 * gp + 1]; }
    else if (gp < a.P_tot) { px = a.Xe[2 * (gp - a.P_mesh)]; py = a.Xe[2 * (gp - a.P_mesh) + 1]; }
    if (gp < a.P_tot) {
      sd[0] = UB[gp];
      sd[1] = UB[a.P_tot + gp];
      sd[2] = UB[2 * a.P_tot + gp];
      if (two) sd[3] = UB[3 * a.P_tot + gp];
    }
  };
  fetch(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < TP) {
      const int p = threadIdx.x;
      sX[p] = (R)px;
      sX[TPS + p] = (R)py;
#pragma unroll
      for (int j = 0; j < 4; ++j) sSeed[j * TPS + p] = sd[j];
    }
    fetch(tile + gridDim.x);
    __syncthreads();
    if (!stash) {
      // forward recompute, keeping every hidden layer's (t, t'_x, t'_y)
      fwd_layer0<R, PW>(sW + wl.woff[0], sW + wl.boff[0], wl.ld[0], sh.w[1], wl.rows[0], sX, S, TP, TPS, plane);
      __syncthreads();
      for (int i = 1; i < L - 1; ++i) {
        fwd_gemm<R, PW, false>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i + 1], wl.rows[i],
                        S + (size_t)(i - 1) * 3 * plane, S + (size_t)i * 3 * plane, TP, TPS, plane);
        __syncthreads();
      }
    } else if (!arrive(L - 2)) {
      break;
    }
    // output map: its gradient and zbar of the last hidden layer
    out_adjoint<R, PW>(sW + wl.woff[L - 1], wl.ld[L - 1], sh.w[L - 1], two, wl.rows[L - 2], sSeed,
                       S + (size_t)(L - 2) * 3 * plane, Z, TP, TPS, plane, G, sh.off[L - 1], sScr);
    __syncthreads();
    if (stash) issue(L - 2, tile + gridDim.x);
    // hidden maps, top down: adjoint GEMM and weight-gradient GEMM side by side
    int cur = 0;
    for (int i = L - 2; i >= 1; --i) {
      if (stash && !arrive(i - 1)) break;
      const R* Zi = Z + (size_t)cur * 3 * plane;
      const R* H = S + (size_t)(i - 1) * 3 * plane;
      if (threadIdx.x < kTbarThreads)
        tbar_gemm<R, PW>(sW + wl.woff[i], wl.ld[i], sh.w[i + 1], wl.ld[i], Zi, H, Z + (size_t)(cur ^ 1) * 3 * plane,
                         TP, TPS, plane, threadIdx.x, kTbarThreads);
      else
        wgrad_gemm<R>(Zi, H, sh.w[i + 1], sh.w[i], TP, TPS, plane, G, sh.off[i], sScr, threadIdx.x - kTbarThreads,
                      kWgThreads);
      __syncthreads();
      if (stash) issue(i - 1, tile + gridDim.x);
      cur ^= 1;
    }
    if (failed) break;
    wgrad_map0<R, PW>(Z + (size_t)cur * 3 * plane, sX, sh.w[1], TP, TPS, plane, G, sh.off[0], sScr);
  }
  // a CTA that gave up waits (bounded) for its copies still in flight
  if (threadIdx.x == 0)
    for (int i = 0; i < L - 1; ++i)
      if (pending & (1u << i)) tc::mbar_wait(&sbar[i], (sphase >> i) & 1u);
  __syncthreads();
  double* dst = a.gpart + (size_t)blockIdx.x * sh.n_params;
  for (int i = threadIdx.x; i < sh.n_params; i += blockDim.x) dst[i] = failed ? 0.0 : G.get(i);
}

size_t fwd_smem(const MlpShape& sh, const WLayout& wl, int DP, int TP, size_t rsz) {
  const int TPS = tps_for(TP);
  return rsz * ((size_t)wl.total + 6 * (size_t)DP * TPS + 2 * TPS);
}

// Partial-sum scratch of the reverse kernel: weight-gradient halves, the output
// map's and map 0's per-point-group sums.
size_t bwd_scratch(const MlpShape& sh, const WLayout& wl, int TP, size_t rsz) {
  const int n_pg = TP / (rsz == 4 ? 4 : 2);
  size_t n = (size_t)wl.rows[sh.L - 2] * n_pg * 2;
  n = std::max(n, (size_t)sh.w[1] * n_pg * 3);
  for (int i = 1; i < sh.L - 1; ++i) n = std::max(n, (size_t)((sh.w[i + 1] + 3) / 4) * ((sh.w[i] + 4) / 4) * 16);
  return (n + 3) & ~(size_t)3;
}

size_t bwd_smem(const MlpShape& sh, const WLayout& wl, int DP, int TP, size_t rsz) {
  const int TPS = tps_for(TP);
  size_t b = rsz * (size_t)((sh.n_params + 3) & ~3);
  b += rsz * ((size_t)wl.total + (size_t)(sh.L - 1) * 3 * DP * TPS + 6 * (size_t)DP * TPS + 6 * TPS);
  b += rsz * bwd_scratch(sh, wl, TP, rsz);
  return b;
}

// Largest point tile that fits, preferring adjoint-GEMM tiles that all fit
// the adjoint threads at once (on the annulus in FP32: 36 points, nine point
// groups; 36 measured 6% faster per step than 32, whose eight point groups
// keep a half-warp's lane pairs in distinct banks).
int pick_tp_bwd(fv_ctx ctx, const MlpShape& sh, const WLayout& wl, int DP, size_t rsz) {
  // the per-block limit covers the kernel's static shared memory (the stash
  // barriers) as well as the dynamic part sized here
  const size_t budget = std::min<size_t>(ctx->smem_optin, 227 * 1024) - kBwdStaticSmem;
  const int PW = rsz == 4 ? 4 : 2;
  int n_kg = 1;
  for (int i = 1; i < sh.L - 1; ++i) n_kg = std::max(n_kg, wl.ld[i] / 4);
  int best = 0, best_fit = 0;
  for (int TP = 4; TP <= 64; TP += 4) {
    if (bwd_smem(sh, wl, DP, TP, rsz) > budget) continue;
    best = TP;
    if (2 * ((n_kg + 1) / 2) * (TP / PW) <= kTbarThreads) best_fit = TP;
  }
  return best_fit ? best_fit : best;
}

template <class R>
int launch_fwd_t(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe, void* U,
                 void* stash) {
  FwdArgs a;
  a.sh = pl.shape;
  a.wl = make_layout(pl.shape);
  a.DP = max_hidden_pad(pl.shape);
  // the reverse kernel's tile (a stash must use it); eight point groups when
  // the reverse kernel does not fit
  a.TP = pick_tp_bwd(ctx, a.sh, a.wl, a.DP, sizeof(R));
  if (a.TP == 0 && !stash) a.TP = 8 * PointsPerTile<R>::v;
  size_t smem = fwd_smem(a.sh, a.wl, a.DP, a.TP, sizeof(R));
  while (!stash && smem > ctx->smem_optin && a.TP > 4) { a.TP -= 4; smem = fwd_smem(a.sh, a.wl, a.DP, a.TP, sizeof(R)); }
  if (a.TP == 0 || smem > ctx->smem_optin) { set_error("network too large for the shared-memory forward kernel"); return FV_ERR_UNSUPPORTED; }
  a.TPS = tps_for(a.TP);
  a.params = params; a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot; a.U = U; a.stash = stash;
  const int64_t n_tiles = (pl.P_tot + a.TP - 1) / a.TP;
  const int per_sm = std::max<int>(1, (int)(std::min<size_t>(ctx->smem_optin, 228 * 1024) / (smem + 1024)));
  const int grid = (int)std::min<int64_t>(n_tiles, (int64_t)ctx->n_sm * std::min(per_sm, 4));
  cudaError_t e = ensure_smem_attr(ctx, (const void*)mlp_fwd_simt<R>, smem);
  if (e == cudaSuccess) {
    mlp_fwd_simt<R><<<grid, kThreads, smem, ctx->stream>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { set_error("mlp forward launch failed: %s", cudaGetErrorString(e)); return FV_ERR_CUDA; }
  return FV_OK;
}

template <class R>
int bwd_config(fv_ctx ctx, const EvalPlan& pl, BwdArgs* a, size_t* smem, int* grid) {
  a->sh = pl.shape;
  a->wl = make_layout(pl.shape);
  a->DP = max_hidden_pad(pl.shape);
  a->TP = pick_tp_bwd(ctx, a->sh, a->wl, a->DP, sizeof(R));
  if (a->TP == 0) { set_error("network too large for the shared-memory reverse kernel"); return FV_ERR_UNSUPPORTED; }
  a->TPS = tps_for(a->TP);
  *smem = bwd_smem(a->sh, a->wl, a->DP, a->TP, sizeof(R));
  const int64_t n_tiles = (pl.P_tot + a->TP - 1) / a->TP;
  const int per_sm = std::max<int>(1, (int)(std::min<size_t>(ctx->smem_optin, 228 * 1024) / (*smem + 1024)));
  *grid = (int)std::min<int64_t>(n_tiles, (int64_t)ctx->n_sm * std::min(per_sm, 2));
  return FV_OK;
}

template <class R>
int launch_bwd_t(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                 const void* UB, double* gpart, int* nb, const void* stash) {
  BwdArgs a;
  size_t smem;
  int grid;
  int rc = bwd_config<R>(ctx, pl, &a, &smem, &grid);
  if (rc) return rc;
  a.params = params; a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot; a.UB = UB; a.gpart = gpart;
  a.stash = stash; a.err = ctx->err_dev;
  *nb = grid;
  cudaError_t e = ensure_smem_attr(ctx, (const void*)mlp_bwd_simt<R>, smem);
  if (e == cudaSuccess) {
    mlp_bwd_simt<R><<<grid, kThreadsBwd, smem, ctx->stream>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { set_error("mlp reverse launch failed: %s", cudaGetErrorString(e)); return FV_ERR_CUDA; }
  return FV_OK;
}

}  // namespace

int launch_mlp_fwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe, void* U,
                   void* stash) {
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_FWD, &ta);
  const int rc = pl.prec == FV_FP64 ? launch_fwd_t<double>(ctx, pl, params, Xm, Xe, U, stash)
                                    : launch_fwd_t<float>(ctx, pl, params, Xm, Xe, U, stash);
  time_end(ctx, K_MLP_FWD, ta);
  return rc;
}

size_t mlp_simt_stash_bytes(fv_ctx ctx, const EvalPlan& pl) {
  const size_t rsz = pl.prec == FV_FP64 ? 8 : 4;
  const MlpShape& sh = pl.shape;
  if (sh.L < 2) return 0;
  const WLayout wl = make_layout(sh);
  const int DP = max_hidden_pad(sh);
  const int TP = pick_tp_bwd(ctx, sh, wl, DP, rsz);
  if (TP == 0 || fwd_smem(sh, wl, DP, TP, rsz) > ctx->smem_optin) return 0;
  const int64_t n_tiles = (pl.P_tot + TP - 1) / TP;
  return (size_t)n_tiles * (size_t)(sh.L - 1) * 3 * (size_t)DP * tps_for(TP) * rsz;
}

int mlp_bwd_blocks(fv_ctx ctx, const EvalPlan& pl) {
  BwdArgs a;
  size_t smem;
  int grid = 0;
  int rc = pl.prec == FV_FP64 ? bwd_config<double>(ctx, pl, &a, &smem, &grid) : bwd_config<float>(ctx, pl, &a, &smem, &grid);
  return rc ? -rc : grid;
}

int launch_mlp_bwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                   const void* UB, double* gpart, int* nb, const void* stash) {
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_BWD, &ta);
  const int rc = pl.prec == FV_FP64 ? launch_bwd_t<double>(ctx, pl, params, Xm, Xe, UB, gpart, nb, stash)
                                    : launch_bwd_t<float>(ctx, pl, params, Xm, Xe, UB, gpart, nb, stash);
  time_end(ctx, K_MLP_BWD, ta);
  return rc;
}

}  // namespace fv
