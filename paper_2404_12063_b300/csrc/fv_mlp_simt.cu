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
// [stream][neuron][TPS] (TPS = TP padded so that TPS/4 is odd: rows of a
// micro-tile fall in distinct bank groups).  Each layer is a small GEMM done
// as 4x4 register micro-tiles.  The reverse kernel recomputes the forward for
// its tile, keeps every hidden layer's (t, t'_x, t'_y) on chip, and
// accumulates the weight gradient of all its tiles in a shared-memory buffer
// (FP64, or compensated FP32 pairs on the FP32 path) that it writes out once
// (deterministic per-CTA partials).
#include <algorithm>

#include "fv_internal.cuh"

namespace fv {
namespace {

constexpr int kThreads = 256;      // forward kernel
constexpr int kThreadsBwd = 512;   // reverse kernel: its shared memory allows one CTA per SM, so 16 warps

struct WLayout {
  int woff[kMaxLayers];  // padded W_i: rows ru4(out) x ld ru4(in), row-major
  int boff[kMaxLayers];  // padded b_i: ru4(out)
  int ld[kMaxLayers];
  int rows[kMaxLayers];
  int total;             // elements (multiple of 4)
};

inline int ru4(int v) { return (v + 3) & ~3; }

WLayout make_layout(const MlpShape& s) {
  WLayout l;
  int o = 0;
  for (int i = 0; i < s.L; ++i) {
    l.ld[i] = ru4(s.w[i]);
    l.rows[i] = ru4(s.w[i + 1]);
    l.woff[i] = o; o += l.ld[i] * l.rows[i];
    l.boff[i] = o; o += l.rows[i];
  }
  l.total = o;
  return l;
}

int max_hidden_pad(const MlpShape& s) {
  int d = 4;
  for (int i = 1; i < s.L; ++i) d = std::max(d, ru4(s.w[i]));
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
  int inplace;   // one activation buffer (every micro-tile is one thread's)
  const void* params;
  const double* Xm;
  int64_t P_mesh;
  const double* Xe;
  int64_t P_tot;
  void* U;       // [3][P_tot]
};

struct BwdArgs {
  MlpShape sh;
  WLayout wl;
  int DP, TP, TPS;
  int pp;        // points per micro-tile of the forward and adjoint GEMMs (4, 2 or 1: small point tiles)
  int wsplit;    // threads sharing one weight-gradient micro-tile (1 or 2)
  const void* params;
  const double* Xm;
  int64_t P_mesh;
  const double* Xe;
  int64_t P_tot;
  const void* UB;   // [3][P_tot] seeds
  double* gpart;    // [gridDim][n_params]
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
__device__ __forceinline__ void ld2(const float* p, float v[2]) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ld2(const double* p, double v[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void st2(float* p, const float v[2]) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
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

// Layer 0: inputs (x, y) with unit tangents.
template <class R>
__device__ void fwd_layer0(const R* W, const R* b, int ld, int rows, const R* sX, R* B, int TP, int TPS, int plane) {
  for (int idx = threadIdx.x; idx < rows * TP; idx += blockDim.x) {
    const int o = idx / TP, p = idx - o * TP;
    const R w0 = W[o * ld], w1 = W[o * ld + 1];
    const R z = w0 * sX[p] + w1 * sX[TPS + p] + b[o];
    const R t = tanh_r(z), s = (R)1 - t * t;
    B[o * TPS + p] = t;
    B[plane + o * TPS + p] = s * w0;
    B[2 * plane + o * TPS + p] = s * w1;
  }
}

// Hidden layer: B = tanh-rule(W A + b) for the three streams; 4 x PP (o, p)
// micro-tiles (PP = 2 or 1 multiplies the micro-tiles of a small point tile).
template <class R, int PP = 4>
__device__ void fwd_layer(const R* __restrict__ W, const R* __restrict__ b, int ld, int in, int rows,
                          const R* __restrict__ A, R* __restrict__ B, int TP, int TPS, int plane) {
  const int n_pg = TP / PP, n_og = rows >> 2;
  for (int mt = threadIdx.x; mt < n_og * n_pg; mt += blockDim.x) {
    const int pg = mt % n_pg, og = mt / n_pg, p0 = pg * PP;
    R acc[3][4][PP];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < PP; ++j) acc[s][i][j] = (R)0;
    for (int k = 0; k < in; ++k) {
      R a0[PP], a1[PP], a2[PP], w[4];
      ldp<PP>(A + k * TPS + p0, a0);
      ldp<PP>(A + plane + k * TPS + p0, a1);
      ldp<PP>(A + 2 * plane + k * TPS + p0, a2);
#pragma unroll
      for (int oo = 0; oo < 4; ++oo) w[oo] = W[(og + oo * n_og) * ld + k];
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
          acc[0][oo][pp] = fma(w[oo], a0[pp], acc[0][oo][pp]);
          acc[1][oo][pp] = fma(w[oo], a1[pp], acc[1][oo][pp]);
          acc[2][oo][pp] = fma(w[oo], a2[pp], acc[2][oo][pp]);
        }
    }
#pragma unroll
    for (int oo = 0; oo < 4; ++oo) {
      const int o = og + oo * n_og;
      const R bo = b[o];
      R t4[PP], x4[PP], y4[PP];
#pragma unroll
      for (int pp = 0; pp < PP; ++pp) {
        const R t = tanh_r(acc[0][oo][pp] + bo), s = (R)1 - t * t;
        t4[pp] = t; x4[pp] = s * acc[1][oo][pp]; y4[pp] = s * acc[2][oo][pp];
      }
      stp<PP>(B + o * TPS + p0, t4);
      stp<PP>(B + plane + o * TPS + p0, x4);
      stp<PP>(B + 2 * plane + o * TPS + p0, y4);
    }
  }
}

// Hidden layer in place: every micro-tile of the CTA is one thread's (the
// caller checks rows/4 x TP/4 <= blockDim), so each thread holds its results
// in registers across a barrier and then overwrites A with B.
template <class R>
__device__ void fwd_layer_inplace(const R* __restrict__ W, const R* __restrict__ b, int ld, int in, int rows, R* A,
                                  int TP, int TPS, int plane) {
  const int n_pg = TP >> 2, n_og = rows >> 2;
  const int mt = threadIdx.x;
  const bool active = mt < n_og * n_pg;
  const int pg = active ? mt % n_pg : 0, og = active ? mt / n_pg : 0, p0 = pg << 2;
  R acc[3][4][4];
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[s][i][j] = (R)0;
  if (active) {
    for (int k = 0; k < in; ++k) {
      R a0[4], a1[4], a2[4], w[4];
      ld4(A + k * TPS + p0, a0);
      ld4(A + plane + k * TPS + p0, a1);
      ld4(A + 2 * plane + k * TPS + p0, a2);
#pragma unroll
      for (int oo = 0; oo < 4; ++oo) w[oo] = W[(og + oo * n_og) * ld + k];
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          acc[0][oo][pp] = fma(w[oo], a0[pp], acc[0][oo][pp]);
          acc[1][oo][pp] = fma(w[oo], a1[pp], acc[1][oo][pp]);
          acc[2][oo][pp] = fma(w[oo], a2[pp], acc[2][oo][pp]);
        }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int oo = 0; oo < 4; ++oo) {
      const int o = og + oo * n_og;
      const R bo = b[o];
      R t4[4], x4[4], y4[4];
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) {
        const R t = tanh_r(acc[0][oo][pp] + bo), s = (R)1 - t * t;
        t4[pp] = t; x4[pp] = s * acc[1][oo][pp]; y4[pp] = s * acc[2][oo][pp];
      }
      st4(A + o * TPS + p0, t4);
      st4(A + plane + o * TPS + p0, x4);
      st4(A + 2 * plane + o * TPS + p0, y4);
    }
  }
}

// ----------------------------------------------------------------------------- forward kernel
// inplace: one activation buffer, updated layer by layer (fwd_layer_inplace);
// otherwise two, alternating.
template <class R>
__global__ void __launch_bounds__(kThreads) mlp_fwd_simt(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sW = reinterpret_cast<R*>(smem);
  const int plane = a.DP * a.TPS;
  R* bufA = sW + a.wl.total;
  R* bufB = a.inplace ? bufA : bufA + 3 * plane;
  R* sX = bufB + 3 * plane;
  const MlpShape& sh = a.sh;
  const WLayout& wl = a.wl;
  load_weights<R>(sh, wl, reinterpret_cast<const R*>(a.params), sW);
  R* U = reinterpret_cast<R*>(a.U);
  const int64_t n_tiles = (a.P_tot + a.TP - 1) / a.TP;
  const int L = sh.L;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p_base = tile * a.TP;
    __syncthreads();
    load_points<R>(a.Xm, a.P_mesh, a.Xe, a.P_tot, p_base, a.TP, a.TPS, sX);
    __syncthreads();
    R* A = bufA;
    R* B = bufB;
    fwd_layer0<R>(sW + wl.woff[0], sW + wl.boff[0], wl.ld[0], wl.rows[0], sX, A, a.TP, a.TPS, plane);
    __syncthreads();
    for (int i = 1; i < L - 1; ++i) {
      if (a.inplace) {
        fwd_layer_inplace<R>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i], wl.rows[i], A, a.TP, a.TPS, plane);
        __syncthreads();
      } else {
        fwd_layer<R>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i], wl.rows[i], A, B, a.TP, a.TPS, plane);
        __syncthreads();
        R* t = A; A = B; B = t;
      }
    }
    const R* Wl = sW + wl.woff[L - 1];
    const R bl = sW[wl.boff[L - 1]];
    const int in = sh.w[L - 1];
    const bool two = sh.w[L] == 2;                 // second output eps(x, y) (Sec. 4.7.2)
    const R* We = Wl + wl.ld[L - 1];
    const R be = sW[wl.boff[L - 1] + 1];
    for (int p = threadIdx.x; p < a.TP; p += blockDim.x) {
      const int64_t gp = p_base + p;
      if (gp >= a.P_tot) continue;
      R u = bl, ux = 0, uy = 0, e = be;
      for (int k = 0; k < in; ++k) {
        const R w = Wl[k];
        u = fma(w, A[k * a.TPS + p], u);
        ux = fma(w, A[plane + k * a.TPS + p], ux);
        uy = fma(w, A[2 * plane + k * a.TPS + p], uy);
        if (two) e = fma(We[k], A[k * a.TPS + p], e);
      }
      U[gp] = u;
      U[a.P_tot + gp] = ux;
      U[2 * a.P_tot + gp] = uy;
      if (two) U[3 * a.P_tot + gp] = e;
    }
  }
}

// ----------------------------------------------------------------------------- reverse kernel
// Zb <- tanh-rule adjoint of the stored layer S from Tb (rows x TP)
template <class R>
__device__ void bwd_elementwise(const R* __restrict__ S, const R* __restrict__ Tb, R* __restrict__ Zb, int rows,
                                int TP, int TPS, int plane) {
  for (int idx = threadIdx.x; idx < rows * TP; idx += blockDim.x) {
    const int k = idx / TP, p = idx - k * TP;
    const int o = k * TPS + p;
    const R t = S[o], tx = S[plane + o], ty = S[2 * plane + o];
    const R bt = Tb[o], bx = Tb[plane + o], by = Tb[2 * plane + o];
    const R s = (R)1 - t * t;
    Zb[o] = s * bt - (R)2 * t * (tx * bx + ty * by);
    Zb[plane + o] = s * bx;
    Zb[2 * plane + o] = s * by;
  }
}

// gW[o][k] += sum_s sum_p Zb[s][o][p] H[s][k][p]; 4x4 (o, k) micro-tiles with
// interleaved rows (o = og + n_og*oo, k = kg + n_kg*kk).  With split = 2 each
// micro-tile's sum over the 3 x TP point-streams is shared by two threads (the
// first and second halves of the 4-point steps); the second leaves its part in
// `scratch` ([micro-tile][16]) and the first adds it, then its own sum goes to
// the accumulator: a fixed order.  Every thread of the CTA takes part (barrier).
template <class R>
__device__ void wgrad_layer(const R* __restrict__ Zb, const R* __restrict__ H, int out, int in, int rows_o,
                            int rows_k, int TP, int TPS, int plane, GradAcc<R> G, int off, int split,
                            R* __restrict__ scratch) {
  const int n_og = rows_o >> 2, n_kg = rows_k >> 2, n_micro = n_og * n_kg;
  const int n_steps = 3 * (TP >> 2);                  // (stream, 4-point group) steps
  const int rounds = (n_micro * split + blockDim.x - 1) / blockDim.x;
  for (int r = 0; r < rounds; ++r) {
    const int mt = r * blockDim.x + threadIdx.x;
    const bool active = mt < n_micro * split;
    const int half = active ? mt / n_micro : 0, m = active ? mt % n_micro : 0;
    const int kg = m % n_kg, og = m / n_kg;
    const int s0 = half * n_steps / split, s1 = (half + 1) * n_steps / split;
    R acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (R)0;
    if (active)
      for (int st = s0; st < s1; ++st) {
        const int sstream = st / (TP >> 2), p = (st % (TP >> 2)) << 2;
        const R* Zs = Zb + sstream * plane;
        const R* Hs = H + sstream * plane;
        R z[4][4], h[4][4];
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) ld4(Zs + (og + oo * n_og) * TPS + p, z[oo]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) ld4(Hs + (kg + kk * n_kg) * TPS + p, h[kk]);
#pragma unroll
        for (int oo = 0; oo < 4; ++oo)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) acc[oo][kk] = fma(z[oo][pp], h[kk][pp], acc[oo][kk]);
      }
    if (split > 1) {
      if (active && half == 1)
#pragma unroll
        for (int i = 0; i < 16; ++i) scratch[m * 16 + i] = acc[i >> 2][i & 3];
      __syncthreads();
      if (active && half == 0)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i >> 2][i & 3] += scratch[m * 16 + i];
      __syncthreads();
    }
    if (active && half == 0)
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int o = og + oo * n_og, k = kg + kk * n_kg;
          if (o < out && k < in) G.add(off + o * in + k, acc[oo][kk]);
        }
  }
}

// Layer-0 weight gradient: inputs (x, y), tangents (1,0) and (0,1).
template <class R>
__device__ void wgrad_layer0(const R* __restrict__ Zb, const R* __restrict__ sX, int out, int TP, int TPS,
                             int plane, GradAcc<R> G, int off) {
  for (int idx = threadIdx.x; idx < 2 * out; idx += blockDim.x) {
    const int o = idx >> 1, c = idx & 1;
    R acc = 0;
    for (int p = 0; p < TP; ++p) acc += Zb[o * TPS + p] * sX[c * TPS + p] + Zb[(1 + c) * plane + o * TPS + p];
    G.add(off + o * 2 + c, acc);
  }
}

template <class R>
__device__ void bgrad(const R* __restrict__ Zb, int out, int TP, int TPS, GradAcc<R> G, int off) {
  for (int o = threadIdx.x; o < out; o += blockDim.x) {
    R acc = 0;
    for (int p = 0; p < TP; ++p) acc += Zb[o * TPS + p];
    G.add(off + o, acc);
  }
}

// Tb[s][k][p] = sum_o W[o][k] Zb[s][o][p]; 4 x PP (k, p) micro-tiles.
template <class R, int PP = 4>
__device__ void tbar_layer(const R* __restrict__ W, int ld, int out, int rows_k, const R* __restrict__ Zb,
                           R* __restrict__ Tb, int TP, int TPS, int plane) {
  const int n_pg = TP / PP, n_kg = rows_k >> 2;
  for (int mt = threadIdx.x; mt < n_kg * n_pg; mt += blockDim.x) {
    const int pg = mt % n_pg, kg = mt / n_pg, p0 = pg * PP, k0 = kg << 2;
    R acc[3][4][PP];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < PP; ++j) acc[s][i][j] = (R)0;
    for (int o = 0; o < out; ++o) {
      R w[4], z0[PP], z1[PP], z2[PP];
      ld4(W + o * ld + k0, w);
      ldp<PP>(Zb + o * TPS + p0, z0);
      ldp<PP>(Zb + plane + o * TPS + p0, z1);
      ldp<PP>(Zb + 2 * plane + o * TPS + p0, z2);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
          acc[0][kk][pp] = fma(w[kk], z0[pp], acc[0][kk][pp]);
          acc[1][kk][pp] = fma(w[kk], z1[pp], acc[1][kk][pp]);
          acc[2][kk][pp] = fma(w[kk], z2[pp], acc[2][kk][pp]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      stp<PP>(Tb + (k0 + kk) * TPS + p0, acc[0][kk]);
      stp<PP>(Tb + plane + (k0 + kk) * TPS + p0, acc[1][kk]);
      stp<PP>(Tb + 2 * plane + (k0 + kk) * TPS + p0, acc[2][kk]);
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kThreadsBwd) mlp_bwd_simt(BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const MlpShape& sh = a.sh;
  const WLayout& wl = a.wl;
  const int L = sh.L, TP = a.TP, TPS = a.TPS;
  const int plane = a.DP * TPS;
  GradAcc<R> G;
  G.a = reinterpret_cast<R*>(smem);                               // [n_params] (rounded up to 4)
  R* sW = G.a + ((sh.n_params + 3) & ~3);
  R* S = sW + wl.total;                                           // [L-1][3][DP][TPS]
  R* Zb = S + (size_t)(L - 1) * 3 * plane;
  R* Tb = Zb + 3 * plane;
  R* sX = Tb + 3 * plane;                                         // [2][TPS]
  R* sSeed = sX + 2 * TPS;                                        // [4][TPS]: u, u_x, u_y (, eps) seeds
  R* sScr = sSeed + 4 * TPS;                                      // weight-gradient halves [micro-tiles][16]
  const bool two = sh.w[L] == 2;
  for (int i = threadIdx.x; i < sh.n_params; i += blockDim.x) G.zero(i);
  load_weights<R>(sh, wl, reinterpret_cast<const R*>(a.params), sW);
  const R* UB = reinterpret_cast<const R*>(a.UB);
  const int64_t n_tiles = (a.P_tot + TP - 1) / TP;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t p_base = tile * TP;
    __syncthreads();
    load_points<R>(a.Xm, a.P_mesh, a.Xe, a.P_tot, p_base, TP, TPS, sX);
    for (int p = threadIdx.x; p < TP; p += blockDim.x) {
      const int64_t gp = p_base + p;
      const bool in = gp < a.P_tot;
      sSeed[p] = in ? UB[gp] : (R)0;
      sSeed[TPS + p] = in ? UB[a.P_tot + gp] : (R)0;
      sSeed[2 * TPS + p] = in ? UB[2 * a.P_tot + gp] : (R)0;
      if (two) sSeed[3 * TPS + p] = in ? UB[3 * a.P_tot + gp] : (R)0;
    }
    __syncthreads();
    // forward recompute, keeping every hidden layer's (t, t'_x, t'_y)
    fwd_layer0<R>(sW + wl.woff[0], sW + wl.boff[0], wl.ld[0], wl.rows[0], sX, S, TP, TPS, plane);
    __syncthreads();
    for (int i = 1; i < L - 1; ++i) {
      if (a.pp == 1)
        fwd_layer<R, 1>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i], wl.rows[i],
                        S + (size_t)(i - 1) * 3 * plane, S + (size_t)i * 3 * plane, TP, TPS, plane);
      else if (a.pp == 2)
        fwd_layer<R, 2>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i], wl.rows[i],
                        S + (size_t)(i - 1) * 3 * plane, S + (size_t)i * 3 * plane, TP, TPS, plane);
      else
        fwd_layer<R>(sW + wl.woff[i], sW + wl.boff[i], wl.ld[i], sh.w[i], wl.rows[i], S + (size_t)(i - 1) * 3 * plane,
                     S + (size_t)i * 3 * plane, TP, TPS, plane);
      __syncthreads();
    }
    // output layer: gradient of w_L, b_L and seeds for the last hidden layer; a
    // second output eps(x, y) takes a value seed only (it has no tangents)
    {
      const int in = sh.w[L - 1], nout = sh.w[L];
      const R* H = S + (size_t)(L - 2) * 3 * plane;
      const R* Wl = sW + wl.woff[L - 1];
      const R* We = Wl + wl.ld[L - 1];
      const int goff = sh.off[L - 1];
      for (int k = threadIdx.x; k < in; k += blockDim.x) {
        R acc = 0, acce = 0;
        for (int p = 0; p < TP; ++p) {
          acc += sSeed[p] * H[k * TPS + p] + sSeed[TPS + p] * H[plane + k * TPS + p] +
                 sSeed[2 * TPS + p] * H[2 * plane + k * TPS + p];
          if (two) acce += sSeed[3 * TPS + p] * H[k * TPS + p];
        }
        G.add(goff + k, acc);
        if (two) G.add(goff + in + k, acce);
      }
      if (threadIdx.x == 0) {
        R acc = 0, acce = 0;
        for (int p = 0; p < TP; ++p) {
          acc += sSeed[p];
          if (two) acce += sSeed[3 * TPS + p];
        }
        G.add(goff + nout * in, acc);
        if (two) G.add(goff + nout * in + 1, acce);
      }
      const int rows = wl.rows[L - 2];
      for (int idx = threadIdx.x; idx < rows * TP; idx += blockDim.x) {
        const int k = idx / TP, p = idx - k * TP;
        const R w = k < in ? Wl[k] : (R)0;
        const R we = two && k < in ? We[k] : (R)0;
        Tb[k * TPS + p] = w * sSeed[p] + (two ? we * sSeed[3 * TPS + p] : (R)0);
        Tb[plane + k * TPS + p] = w * sSeed[TPS + p];
        Tb[2 * plane + k * TPS + p] = w * sSeed[2 * TPS + p];
      }
    }
    __syncthreads();
    // hidden layers, top down
    for (int i = L - 2; i >= 0; --i) {
      const int out = sh.w[i + 1], in = sh.w[i];
      const R* Si = S + (size_t)i * 3 * plane;
      bwd_elementwise<R>(Si, Tb, Zb, wl.rows[i], TP, TPS, plane);
      __syncthreads();
      const int goff = sh.off[i];
      if (i >= 1)
        wgrad_layer<R>(Zb, S + (size_t)(i - 1) * 3 * plane, out, in, wl.rows[i], wl.ld[i], TP, TPS, plane, G, goff,
                       a.wsplit, sScr);
      else
        wgrad_layer0<R>(Zb, sX, out, TP, TPS, plane, G, goff);
      bgrad<R>(Zb, out, TP, TPS, G, goff + out * in);
      if (i >= 1) {
        if (a.pp == 1) tbar_layer<R, 1>(sW + wl.woff[i], wl.ld[i], out, wl.ld[i], Zb, Tb, TP, TPS, plane);
        else if (a.pp == 2) tbar_layer<R, 2>(sW + wl.woff[i], wl.ld[i], out, wl.ld[i], Zb, Tb, TP, TPS, plane);
        else tbar_layer<R>(sW + wl.woff[i], wl.ld[i], out, wl.ld[i], Zb, Tb, TP, TPS, plane);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  double* dst = a.gpart + (size_t)blockIdx.x * sh.n_params;
  for (int i = threadIdx.x; i < sh.n_params; i += blockDim.x) dst[i] = G.get(i);
}

size_t fwd_smem(const MlpShape& sh, const WLayout& wl, int DP, int TP, size_t rsz, bool inplace = false) {
  const int TPS = tps_for(TP);
  return rsz * ((size_t)wl.total + (inplace ? 3 : 6) * (size_t)DP * TPS + 2 * TPS);
}

size_t bwd_smem(const MlpShape& sh, const WLayout& wl, int DP, int TP, size_t rsz) {
  const int TPS = tps_for(TP);
  size_t b = rsz * (size_t)((sh.n_params + 3) & ~3);
  b += rsz * ((size_t)wl.total + (size_t)(sh.L - 1) * 3 * DP * TPS + 6 * (size_t)DP * TPS + 6 * TPS);
  b += rsz * (size_t)(DP / 4) * (DP / 4) * 16;   // weight-gradient halves
  return b;
}

int pick_tp_bwd(fv_ctx ctx, const MlpShape& sh, const WLayout& wl, int DP, size_t rsz) {
  const size_t budget = std::min<size_t>(ctx->smem_optin, 227 * 1024);
  int best = 0;
  for (int TP = 4; TP <= 64; TP += 4)
    if (bwd_smem(sh, wl, DP, TP, rsz) <= budget) best = TP;
  // prefer TP that fills the micro-tile grid without huge tiles
  return std::min(best, 40);
}

template <class R>
int launch_fwd_t(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe, void* U) {
  FwdArgs a;
  a.sh = pl.shape;
  a.wl = make_layout(pl.shape);
  a.DP = max_hidden_pad(pl.shape);
  a.TP = sizeof(R) == 8 ? 32 : 64;
  // in place when every hidden map's micro-tiles fit one per thread
  int max_micro = 0;
  for (int i = 1; i < a.sh.L - 1; ++i) max_micro = std::max(max_micro, (a.wl.rows[i] / 4) * (a.TP / 4));
  a.inplace = max_micro <= kThreads;
  size_t smem = fwd_smem(a.sh, a.wl, a.DP, a.TP, sizeof(R), a.inplace);
  while (smem > ctx->smem_optin && a.TP > 4) { a.TP -= 4; smem = fwd_smem(a.sh, a.wl, a.DP, a.TP, sizeof(R), a.inplace); }
  if (smem > ctx->smem_optin) { set_error("network too large for the shared-memory forward kernel"); return FV_ERR_UNSUPPORTED; }
  a.TPS = tps_for(a.TP);
  a.params = params; a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot; a.U = U;
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
  // micro-tile shapes that keep most of the CTA's threads busy
  const int n_og = a->DP / 4;
  a->pp = 4;
  if (n_og * (a->TP / 4) * 2 <= kThreadsBwd && a->TP % 2 == 0) a->pp = 2;
  if (n_og * (a->TP / 2) * 2 <= kThreadsBwd) a->pp = 1;
  a->wsplit = n_og * n_og * 2 <= kThreadsBwd ? 2 : 1;
  *smem = bwd_smem(a->sh, a->wl, a->DP, a->TP, sizeof(R));
  const int64_t n_tiles = (pl.P_tot + a->TP - 1) / a->TP;
  const int per_sm = std::max<int>(1, (int)(std::min<size_t>(ctx->smem_optin, 228 * 1024) / (*smem + 1024)));
  *grid = (int)std::min<int64_t>(n_tiles, (int64_t)ctx->n_sm * std::min(per_sm, 2));
  return FV_OK;
}

template <class R>
int launch_bwd_t(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                 const void* UB, double* gpart, int* nb) {
  BwdArgs a;
  size_t smem;
  int grid;
  int rc = bwd_config<R>(ctx, pl, &a, &smem, &grid);
  if (rc) return rc;
  a.params = params; a.Xm = Xm; a.P_mesh = pl.P_mesh; a.Xe = Xe; a.P_tot = pl.P_tot; a.UB = UB; a.gpart = gpart;
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

int launch_mlp_fwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe, void* U) {
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_FWD, &ta);
  const int rc = pl.prec == FV_FP64 ? launch_fwd_t<double>(ctx, pl, params, Xm, Xe, U)
                                    : launch_fwd_t<float>(ctx, pl, params, Xm, Xe, U);
  time_end(ctx, K_MLP_FWD, ta);
  return rc;
}

int mlp_bwd_blocks(fv_ctx ctx, const EvalPlan& pl) {
  BwdArgs a;
  size_t smem;
  int grid = 0;
  int rc = pl.prec == FV_FP64 ? bwd_config<double>(ctx, pl, &a, &smem, &grid) : bwd_config<float>(ctx, pl, &a, &smem, &grid);
  return rc ? -rc : grid;
}

int launch_mlp_bwd(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                   const void* UB, double* gpart, int* nb) {
  cudaEvent_t ta;
  time_begin(ctx, K_MLP_BWD, &ta);
  const int rc = pl.prec == FV_FP64 ? launch_bwd_t<double>(ctx, pl, params, Xm, Xe, UB, gpart, nb)
                                    : launch_bwd_t<float>(ctx, pl, params, Xm, Xe, UB, gpart, nb);
  time_end(ctx, K_MLP_BWD, ta);
  return rc;
}

}  // namespace fv
