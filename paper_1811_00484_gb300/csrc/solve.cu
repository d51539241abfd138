// GMRES solve of the J-block system (Section VI.C: restarted GMRES) with FP64
// iterative refinement.
//
// Outer loop (FP64):  r = b - A x with the FP64 operator; stop when
//   ||r_b|| / ||b_b|| <= tol for every right-hand side b; otherwise solve
//   A d = r / ||r|| with FP32 GMRES and update x += ||r|| d.
// Inner loop (FP32 vectors): restarted GMRES(m), B right-hand sides at once.
//   Arnoldi by classical Gram-Schmidt (one pass, or a second pass where the
//   DGKS test asks for it) with FP32 products and FP64 sums, FP64 Hessenberg
//   matrix and complex Givens rotations, FP64 triangular solve.  Each restart
//   cycle (m Arnoldi steps, the update of the iterate and the next cycle's
//   true residual) is one CUDA graph: kernels read their state (active flags,
//   iteration counts) from device memory, so converged right-hand sides drop
//   out without host synchronisation; the host synchronises once per cycle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "vie_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 4;                       // elements per thread in the BLAS kernels
constexpr int kChunk = kThreads * kPer;       // elements per CTA

__device__ __forceinline__ double2 wsum(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Krylov basis storage.  Basis vector j of right-hand side b is kept
// unnormalised, V_j = sig[b][j] * Vraw_j, with sig[b][j] = 1 / h_{j,j-1}
// (1 / beta for j = 0): the matvec writes A V_k straight into slot k+1 (its
// x-stage prologue applies sig[b][k] to the input and its epilogue to the
// subtracted input), Gram-Schmidt orthogonalises slot k+1 in place, and the
// factor of every basis vector is folded into the coefficients that read it.
// No pass over the data only to normalise a vector.
//
// The two long kernels of a Gram-Schmidt pass read the basis with 16-byte
// loads (two complex values) when every vector starts on a 16-byte boundary
// (N even), with several basis vectors' loads in flight per thread.
template <int W> struct Pack { float2 c[W]; };

template <int W> __device__ __forceinline__ Pack<W> ldp(const float2* p);
template <> __device__ __forceinline__ Pack<1> ldp<1>(const float2* p) {
  Pack<1> r;
  r.c[0] = *p;
  return r;
}
template <> __device__ __forceinline__ Pack<2> ldp<2>(const float2* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  Pack<2> r;
  r.c[0] = make_float2(v.x, v.y);
  r.c[1] = make_float2(v.z, v.w);
  return r;
}
template <int W> __device__ __forceinline__ void stp(float2* p, const Pack<W>& v);
template <> __device__ __forceinline__ void stp<1>(float2* p, const Pack<1>& v) { *p = v.c[0]; }
template <> __device__ __forceinline__ void stp<2>(float2* p, const Pack<2>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.c[0].x, v.c[0].y, v.c[1].x, v.c[1].y);
}
template <int W> __device__ __forceinline__ Pack<W> zpack() {
  Pack<W> r;
#pragma unroll
  for (int j = 0; j < W; ++j) r.c[j] = make_float2(0.f, 0.f);
  return r;
}

__device__ __forceinline__ float2 shfl_xor32(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ float2 wsum32(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// dots: a tile is kDotThreads x kDotPacks packs; basis vectors kDotBlock at a time
constexpr int kDotThreads = 128;
constexpr int kDotPacks = 4;
constexpr int kDotBlock = 4;
constexpr int kMaxDotCtas = 4096;             // per right-hand side (bounds the partials)
// update: one pack per thread, basis vectors kUpdBlock at a time
constexpr int kUpdThreads = 256;
constexpr int kUpdBlock = 4;

// partial[b][i][cta] = sum over the CTA's tiles of conj(Vraw_i[b]) w[b], i = 0..k.
// Products and warp sums in FP32 (the data are FP32); sums across tiles, warps
// and CTAs in FP64 (GB300's FP64 rate is far below its FP32 rate, so FP64
// stays out of per-element work).
template <int W>
__global__ void __launch_bounds__(kDotThreads) dots_kernel(const float2* __restrict__ V,
                                                           const float2* __restrict__ w, int k, int B,
                                                           long long N, int G, int ps, double2* partial,
                                                           const int* active,
                                                           unsigned long long* prof,
                                                           unsigned long long prof_bytes) {
  constexpr int NW = kDotThreads / 32;
  constexpr int TILE = kDotThreads * kDotPacks * W;
  const int b = blockIdx.y, cta = blockIdx.x;
  __shared__ double2 red[NW][129];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = lane; i <= k; i += 32) red[warp][i] = make_double2(0.0, 0.0);
  __syncwarp();
  pdl_trigger();
  pdl_wait();
  if (!active[b]) return;
  if (prof != nullptr && cta == 0 && threadIdx.x == 0) atomicAdd(prof, prof_bytes);
  const long long ntile = (N + TILE - 1) / TILE;
  const float2* wb = w + (long long)b * N;
  for (long long t = cta; t < ntile; t += G) {
    Pack<W> wv[kDotPacks];
    long long off[kDotPacks];
#pragma unroll
    for (int e = 0; e < kDotPacks; ++e) {
      const long long j = t * TILE + (long long)(e * kDotThreads + threadIdx.x) * W;
      const bool in = j < N;                     // N % W == 0: a pack is all in or all out
      off[e] = in ? j : 0;                       // loads stay in bounds; the product is zeroed
      wv[e] = in ? ldp<W>(wb + j) : zpack<W>();
    }
    for (int i0 = 0; i0 <= k; i0 += kDotBlock) {
      float2 acc[kDotBlock];
#pragma unroll
      for (int u = 0; u < kDotBlock; ++u) {
        const int i = min(i0 + u, k);            // repeats vector k past the end; not stored
        const float2* vi = V + ((long long)i * B + b) * N;
        float ax = 0.f, ay = 0.f;
#pragma unroll
        for (int e = 0; e < kDotPacks; ++e) {
          const Pack<W> v = ldp<W>(vi + off[e]);
#pragma unroll
          for (int q = 0; q < W; ++q) {
            ax = fmaf(v.c[q].x, wv[e].c[q].x, fmaf(v.c[q].y, wv[e].c[q].y, ax));
            ay = fmaf(v.c[q].x, wv[e].c[q].y, fmaf(-v.c[q].y, wv[e].c[q].x, ay));
          }
        }
        acc[u] = make_float2(ax, ay);
      }
      // warp sums of the four accumulators in one butterfly (12 shuffles, not 40):
      // halve the values each lane holds at xor 16 and 8, then finish at 4, 2, 1;
      // lanes 8u .. 8u+7 end with the sum of acc[u]
      static_assert(kDotBlock == 4, "butterfly below reduces four accumulators");
      const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
      float2 k0 = h16 ? acc[2] : acc[0], k1 = h16 ? acc[3] : acc[1];
      const float2 s0 = h16 ? acc[0] : acc[2], s1 = h16 ? acc[1] : acc[3];
      k0 = k0 + shfl_xor32(s0, 16);
      k1 = k1 + shfl_xor32(s1, 16);
      float2 kv = h8 ? k1 : k0;
      kv = kv + shfl_xor32(h8 ? k0 : k1, 8);
      kv = kv + shfl_xor32(kv, 4);
      kv = kv + shfl_xor32(kv, 2);
      kv = kv + shfl_xor32(kv, 1);
      const int u = lane >> 3;
      if ((lane & 7) == 0 && i0 + u <= k)
        red[warp][i0 + u] = red[warp][i0 + u] + make_double2(kv.x, kv.y);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= k; i += kDotThreads) {
    double2 s = red[0][i];
    for (int q = 1; q < NW; ++q) s = s + red[q][i];
    partial[((long long)b * ps + i) * G + cta] = s;
  }
}

// coef[b][i] = h_{i,k} = sig[b][i] sum_cta partial; H[b][k][i] (+)= coef.
// One CTA of kReduceThreads per (i, b).
constexpr int kReduceThreads = 128;
__global__ void __launch_bounds__(kReduceThreads) reduce_dots_kernel(const double2* partial, int k,
                                                                     int G, int ps, const double* sig,
                                                                     double2* coef, double2* H,
                                                                     int m, int accumulate,
                                                                     const int* active) {
  const int b = blockIdx.y, i = blockIdx.x;
  pdl_trigger();
  pdl_wait();
  if (!active[b]) return;
  __shared__ double2 red[kReduceThreads / 32];
  const double2* p = partial + ((long long)b * ps + i) * G;
  double2 s = make_double2(0.0, 0.0);
  for (int c = threadIdx.x; c < G; c += kReduceThreads) s = s + p[c];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    s = red[0];
    for (int q = 1; q < kReduceThreads / 32; ++q) s = s + red[q];
    s = sig[(long long)b * (m + 1) + i] * s;
    coef[(long long)b * 129 + i] = s;
    double2* h = H + ((long long)b * m + k) * (m + 1) + i;
    *h = accumulate ? (*h + s) : s;
  }
}

enum { UPD_FINAL = 0, UPD_DGKS = 1 };

// w[b] -= sum_i coef[b][i] sig[b][i] Vraw_i[b], then ||w[b]||.  The last CTA
// of right-hand side b to finish (an atomic ticket) sums the norm partials:
//   UPD_FINAL: nrm[b] = h_{k+1,k} = ||w||, sig[b][k+1] = 1 / h_{k+1,k};
//   UPD_DGKS:  the DGKS test (re-orthogonalise only where the projection
//              removed most of w, ||w'||^2 < (1/2)(||w'||^2 + ||h||^2)), and
//              the UPD_FINAL results where no second pass is needed.
template <int W>
__global__ void __launch_bounds__(kUpdThreads) update_kernel(const float2* __restrict__ V, float2* w,
                                                             const double2* coef, double* sig,
                                                             int k, int m, int B, long long N, int G,
                                                             double* nrm_partial, int* ticket,
                                                             int mode, double* nrm_out, int* again,
                                                             const int* mask,
                                                             unsigned long long* prof,
                                                             unsigned long long prof_bytes) {
  const int b = blockIdx.y, cta = blockIdx.x;
  pdl_trigger();
  pdl_wait();
  if (!mask[b]) return;
  if (prof != nullptr && cta == 0 && threadIdx.x == 0) atomicAdd(prof, prof_bytes);
  __shared__ float2 c[129];
  __shared__ double red[kUpdThreads / 32];
  __shared__ int last;
  for (int i = threadIdx.x; i <= k; i += kUpdThreads) {
    const double2 v = sig[(long long)b * (m + 1) + i] * coef[(long long)b * 129 + i];
    c[i] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const long long j = ((long long)cta * kUpdThreads + threadIdx.x) * W;
  const bool in = j < N;
  const long long off = in ? j : 0;
  float2* wb = w + (long long)b * N;
  Pack<W> acc = in ? ldp<W>(wb + j) : zpack<W>();
  // basis vectors from k down to 0: the dots kernel just read them from 0 up
  // to k, so the most recent ones are still in L2
  int i = k;
  for (; i + 1 >= kUpdBlock; i -= kUpdBlock) {
    Pack<W> v[kUpdBlock];
#pragma unroll
    for (int u = 0; u < kUpdBlock; ++u) v[u] = ldp<W>(V + ((long long)(i - u) * B + b) * N + off);
#pragma unroll
    for (int u = 0; u < kUpdBlock; ++u) {
      const float2 ci = c[i - u];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        acc.c[q].x -= ci.x * v[u].c[q].x - ci.y * v[u].c[q].y;
        acc.c[q].y -= ci.x * v[u].c[q].y + ci.y * v[u].c[q].x;
      }
    }
  }
  for (; i >= 0; --i) {
    const float2 ci = c[i];
    const Pack<W> v = ldp<W>(V + ((long long)i * B + b) * N + off);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      acc.c[q].x -= ci.x * v.c[q].x - ci.y * v.c[q].y;
      acc.c[q].y -= ci.x * v.c[q].y + ci.y * v.c[q].x;
    }
  }
  float nrm32 = 0.f;
  if (in) {
    stp<W>(wb + j, acc);
#pragma unroll
    for (int q = 0; q < W; ++q) nrm32 = fmaf(acc.c[q].x, acc.c[q].x, fmaf(acc.c[q].y, acc.c[q].y, nrm32));
  }
  double nrm = (double)nrm32;
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kUpdThreads / 32; ++q) s += red[q];
    nrm_partial[(long long)b * G + cta] = s;
    __threadfence();
    last = (atomicAdd(&ticket[b], 1) == G - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  // last CTA of right-hand side b: every other CTA's partial is visible
  __threadfence();
  double s = 0.0;
  for (int q = threadIdx.x; q < G; q += kUpdThreads) s += __ldcg(nrm_partial + (long long)b * G + q);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();                               // red[] reuse
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double w2 = 0.0;
  for (int q = 0; q < kUpdThreads / 32; ++q) w2 += red[q];
  bool fin = true;
  if (mode == UPD_DGKS) {
    double hh = 0.0;
    for (int q = lane; q <= k; q += 32) hh += abs2(coef[(long long)b * 129 + q]);
    for (int o = 16; o > 0; o >>= 1) hh += __shfl_xor_sync(0xffffffffu, hh, o);
    const bool redo = w2 < 0.5 * (w2 + hh);
    if (lane == 0) again[b] = redo ? 1 : 0;
    fin = !redo;
  }
  if (lane == 0) {
    ticket[b] = 0;                               // ready for the next launch
    if (fin) {
      const double h = sqrt(w2);
      nrm_out[b] = h;
      sig[(long long)b * (m + 1) + k + 1] = h > 1e-300 ? 1.0 / h : 0.0;
    }
  }
}

// One Givens step per right-hand side (one warp each): finish column k
// (h_{k+1,k} = nrm), apply the k earlier rotations, form the new one, update
// g and test convergence.  The column and the rotations are staged in shared
// memory so the sequential rotation chain does not wait on global memory.  It
// runs beside the next matvec (which needs only sig[b][k+1]); its FP64 chain,
// a few microseconds on a part with GB300's FP64 latency, is then off the
// critical path.
__global__ void __launch_bounds__(128) givens_kernel(double2* H, double2* cs, double2* sn, double2* g,
                                                     const double* nrm, int k, int m, int B,
                                                     int* active, int* again, int* iters,
                                                     const double* tol_abs, int* count) {
  __shared__ double2 sh[4][130], sc[4][128], ss[4][128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * 4 + warp;
  if (b >= B || !active[b]) return;            // warp-uniform; no block barrier below
  double2* h = H + ((long long)b * m + k) * (m + 1);
  double2* c = cs + (long long)b * m;
  double2* s = sn + (long long)b * m;
  for (int i = lane; i <= k; i += 32) sh[warp][i] = h[i];
  for (int i = lane; i < k; i += 32) {
    sc[warp][i] = c[i];
    ss[warp][i] = s[i];
  }
  __syncwarp();
  if (lane == 0) {
    count[b] += 1;
    double2* hh = sh[warp];
    const double hk1 = nrm[b];
    hh[k + 1] = make_double2(hk1, 0.0);
    for (int i = 0; i < k; ++i) {
      const double2 ci = sc[warp][i], si = ss[warp][i];
      const double2 t = ci * hh[i] + si * hh[i + 1];
      hh[i + 1] = (-1.0) * (conjg(si) * hh[i]) + conjg(ci) * hh[i + 1];
      hh[i] = t;
    }
    const double2 x = hh[k], y = hh[k + 1];
    const double den = sqrt(abs2(x) + abs2(y));
    double2 ck, sk;
    if (den == 0.0) {
      ck = make_double2(1.0, 0.0);
      sk = make_double2(0.0, 0.0);
    } else {
      ck = (1.0 / den) * conjg(x);
      sk = (1.0 / den) * conjg(y);
    }
    c[k] = ck;
    s[k] = sk;
    hh[k] = ck * x + sk * y;
    hh[k + 1] = make_double2(0.0, 0.0);
    double2* gb = g + (long long)b * (m + 1);
    const double2 gk = gb[k];
    gb[k + 1] = (-1.0) * (conjg(sk) * gk);
    gb[k] = ck * gk;
    iters[b] = k + 1;
    const double res2 = abs2(gb[k + 1]);
    const double tol = tol_abs[b];
    const bool breakdown = !(hk1 > 1e-300) || !(abs2(hh[k]) > 0.0);
    if (res2 <= tol * tol || breakdown || k + 1 == m || !(res2 == res2)) {
      active[b] = 0;
      again[b] = 0;
    }
  }
  __syncwarp();
  for (int i = lane; i <= k + 1; i += 32) h[i] = sh[warp][i];
}

// out[b] = sqrt(sum_chunk partial[b][chunk])
__global__ void reduce_norm_kernel(const double* partial, int nchunk, double* out, const int* active) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += 32) s += partial[(long long)b * nchunk + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[b] = sqrt(s);
}

// partial norms of an FP32 vector batch
__global__ void __launch_bounds__(kThreads) norm32_kernel(const float2* v, long long N, int nchunk,
                                                          double* partial, const int* active) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (active && !active[b]) return;
  __shared__ double red[kThreads / 32];
  float s32 = 0.f;
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)chunk * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      const float2 x = v[(long long)b * N + idx];
      s32 = fmaf(x.x, x.x, fmaf(x.y, x.y, s32));
    }
  }
  double s = (double)s32;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[(long long)b * nchunk + chunk] = t;
  }
}

// y = R^-1 g over the iters[b] columns of the rotated Hessenberg matrix, one
// warp per right-hand side: the reciprocals of the diagonal are formed in
// parallel first (an FP64 division is slow on GB300), then column by column
// y_i = r_i / R_ii and the lanes update r_j -= R_ji y_i for j < i.
__global__ void __launch_bounds__(128) backsolve_kernel(const double2* __restrict__ H,
                                                        const double2* g, double2* y, int m, int B,
                                                        const int* iters) {
  __shared__ double2 r[4][129], rinv[4][128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * 4 + warp;
  if (b >= B) return;                          // warp-uniform; no block barrier below
  const int kk = iters[b];
  const double2* gb = g + (long long)b * (m + 1);
  const double2* Hb = H + (long long)b * m * (m + 1);   // column j at Hb + j (m + 1)
  double2* yb = y + (long long)b * 129;
  for (int i = lane; i < kk; i += 32) {
    r[warp][i] = gb[i];
    const double2 d = Hb[(long long)i * (m + 1) + i];
    const double dd = abs2(d);
    rinv[warp][i] = dd > 0.0 ? (1.0 / dd) * conjg(d) : make_double2(0.0, 0.0);
  }
  __syncwarp();
  for (int i = kk - 1; i >= 0; --i) {
    const double2 yi = r[warp][i] * rinv[warp][i];
    if (lane == 0) yb[i] = yi;
    const double2* col = Hb + (long long)i * (m + 1);
    for (int jj = lane; jj < i; jj += 32) r[warp][jj] = r[warp][jj] - col[jj] * yi;
    __syncwarp();
  }
}

// d[b] += sum_{j < iters[b]} y[b][j] V_j[b]  (V_j = sig[b][j] Vraw_j)
__global__ void __launch_bounds__(kThreads) combine_kernel(const float2* V, float2* d, const double2* y,
                                                           const double* sig, int m, int B,
                                                           long long N, const int* iters) {
  const int b = blockIdx.y;
  const int kk = iters[b];
  if (kk == 0) return;
  __shared__ float2 c[129];
  for (int i = threadIdx.x; i < kk; i += kThreads) {
    const double2 v = sig[(long long)b * (m + 1) + i] * y[(long long)b * 129 + i];
    c[i] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)blockIdx.x * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      float2 acc = d[(long long)b * N + idx];
      for (int j = 0; j < kk; ++j) {
        const float2 v = V[((long long)j * B + b) * N + idx];
        acc.x += c[j].x * v.x - c[j].y * v.y;
        acc.y += c[j].x * v.y + c[j].y * v.x;
      }
      d[(long long)b * N + idx] = acc;
    }
  }
}

// r = rhs - Ad (FP32), for RHS still to be solved; partial norms of r
__global__ void __launch_bounds__(kThreads) residual32_kernel(const float2* rhs, const float2* ad,
                                                              float2* r, long long N, int nchunk,
                                                              double* partial, const int* want) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (!want[b]) return;
  __shared__ double red[kThreads / 32];
  float s32 = 0.f;
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)chunk * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      const long long o = (long long)b * N + idx;
      const float2 v = make_float2(rhs[o].x - ad[o].x, rhs[o].y - ad[o].y);
      r[o] = v;
      s32 = fmaf(v.x, v.x, fmaf(v.y, v.y, s32));
    }
  }
  double s = (double)s32;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[(long long)b * nchunk + chunk] = t;
  }
}

// start of a cycle: beta = ||r||, g = (beta, 0, ...), iters = 0, active = want && beta > tol,
// and basis vector 0 = r / beta (slot 0 holds r, its factor is 1 / beta)
__global__ void cycle_start_kernel(const double* beta, double2* g, double* sig, int m, int B,
                                   const int* want, int* active, int* again, int* iters,
                                   const double* tol_abs, int* count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  iters[b] = 0;
  if (count && want[b]) count[b] += 1;   // the residual matvec that produced beta
  const bool go = want[b] && beta[b] > tol_abs[b] && beta[b] == beta[b];
  active[b] = go ? 1 : 0;
  again[b] = 0;
  double2* gb = g + (long long)b * (m + 1);
  for (int i = 0; i <= m; ++i) gb[i] = make_double2(0.0, 0.0);
  gb[0] = make_double2(go ? beta[b] : 0.0, 0.0);
  sig[(long long)b * (m + 1)] = go ? 1.0 / beta[b] : 0.0;
}

// ---------------------------------------------------------------------------
// FP64 vector kernels of the refinement loop (templated on the I/O precision)
// ---------------------------------------------------------------------------
template <typename Tin>
__global__ void load_rhs_kernel(const cx<Tin>* rhs, const cx<Tin>* chi, double2* b, long long nvox,
                                int B, int incident) {
  const long long total = 3LL * nvox * B;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double2 v = make_double2((double)rhs[i].x, (double)rhs[i].y);
    if (incident) {
      const cx<Tin> c = chi[i % nvox];
      v = make_double2((double)c.x, (double)c.y) * v;
    }
    b[i] = v;
  }
}

template <typename Tout>
__global__ void convert_kernel(const double2* x, cx<Tout>* out, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    cx<Tout> o;
    o.x = (Tout)x[i].x;
    o.y = (Tout)x[i].y;
    out[i] = o;
  }
}

template <typename Tin>
__global__ void load_x_kernel(const cx<Tin>* in, double2* x, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = make_double2((double)in[i].x, (double)in[i].y);
}

// r = b - Ax and partial ||r||^2, ||b||^2 (FP64)
__global__ void __launch_bounds__(kThreads) residual64_kernel(const double2* b, const double2* ax,
                                                              double2* r, long long N, int nchunk,
                                                              double* pr, double* pb, int have_ax) {
  const int rb = blockIdx.y, chunk = blockIdx.x;
  __shared__ double red[2][kThreads / 32];
  double sr = 0.0, sb = 0.0;
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)chunk * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      const long long o = (long long)rb * N + idx;
      const double2 bv = b[o];
      const double2 v = have_ax ? bv - ax[o] : bv;
      r[o] = v;
      sr += abs2(v);
      sb += abs2(bv);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) {
      t0 += red[0][q];
      t1 += red[1][q];
    }
    pr[(long long)rb * nchunk + chunk] = t0;
    pb[(long long)rb * nchunk + chunk] = t1;
  }
}

// r32 = r / scale (FP32), d = 0, for RHS that still need work
__global__ void __launch_bounds__(kThreads) to_inner_kernel(const double2* r, const double* scale,
                                                            float2* r32, float2* d, long long N,
                                                            const int* want) {
  const int b = blockIdx.y;
  if (!want[b]) return;
  const double s = scale[b] > 0.0 ? 1.0 / scale[b] : 0.0;
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)blockIdx.x * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      const long long o = (long long)b * N + idx;
      r32[o] = make_float2((float)(s * r[o].x), (float)(s * r[o].y));
      d[o] = make_float2(0.f, 0.f);
    }
  }
}

// x += scale * d  (FP64), for RHS that were worked on
__global__ void __launch_bounds__(kThreads) accumulate_kernel(double2* x, const float2* d,
                                                              const double* scale, long long N,
                                                              const int* want) {
  const int b = blockIdx.y;
  if (!want[b]) return;
  const double s = scale[b];
  for (int e = 0; e < kPer; ++e) {
    const long long idx = (long long)blockIdx.x * kChunk + e * kThreads + threadIdx.x;
    if (idx < N) {
      const long long o = (long long)b * N + idx;
      x[o] = x[o] + make_double2(s * d[o].x, s * d[o].y);
    }
  }
}

__global__ void reduce_norm2_kernel(const double* partial, int nchunk, double* out, int B) {
  const int b = blockIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += 32) s += partial[(long long)b * nchunk + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[b] = sqrt(s);
}

int grid1(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(b, 152 * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// solver state, cached on the operator
// ---------------------------------------------------------------------------
struct SolverState {
  int B = 0, m = 0, path = -1;
  long long N = 0;
  int nchunk = 0;
  int G = 0, Gu = 0;                // CTAs per RHS of the dots and update kernels
  int wide = 0;                     // 16-byte loads in dots / update (N even)
  size_t bytes = 0;
  char* base = nullptr;
  float2 *V, *W, *d, *r32;
  double2 *H, *cs, *sn, *g, *coef, *partial;
  double *nrm_partial, *nrm, *sig, *beta, *tol_abs, *rnorm, *bnorm, *pb;
  int *active, *iters, *want, *count_it, *count_mv, *again, *ticket;
  int* mv_active;                   // the matvec's copy of `active` (see arnoldi_step)
  double2 *x, *b64, *r64, *ax64;
  float2* chi32;
  double2* chi64;
  // graph of one restart cycle
  // the solve runs on its own stream (graphs cannot be captured on the legacy
  // default stream), ordered after and before the caller's stream by events
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // the Givens step runs on a side stream beside the next matvec
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool givens_pending = false;
  cudaGraphExec_t exec = nullptr;
  const void* graph_chi = nullptr;
  const void* graph_ws = nullptr;
  cudaStream_t graph_stream = nullptr;
  int graph_adjoint = -1;
  int graph_prof = -1;                        // profiler epoch the graph was captured in
  int graph_passes = -1;                      // Gram-Schmidt passes baked into the graph
  unsigned graph_cp_epoch = ~0u;              // Tucker+CP model the graph's rebuilds read
  std::vector<ProfEventPair> graph_events;    // event nodes of the captured graph
  bool graph_pending = false;                 // a replay ran since the last harvest
};

static void drop_graph(SolverState* st) {
  if (st->exec) cudaGraphExecDestroy(st->exec);
  st->exec = nullptr;
  prof_release_pairs(st->graph_events);
}

static void release_state(SolverState* st) {
  if (!st) return;
  if (st->stream) cudaStreamSynchronize(st->stream);
  drop_graph(st);
  if (st->stream) {
    cudaStreamSynchronize(st->stream);
    cudaStreamDestroy(st->stream);
  }
  if (st->aux) {
    cudaStreamSynchronize(st->aux);
    cudaStreamDestroy(st->aux);
  }
  if (st->ev_in) cudaEventDestroy(st->ev_in);
  if (st->ev_out) cudaEventDestroy(st->ev_out);
  if (st->ev_fork) cudaEventDestroy(st->ev_fork);
  if (st->ev_join) cudaEventDestroy(st->ev_join);
  cudaFree(st->base);
  delete st;
}

void solver_release(vie_op* op) {
  release_state(static_cast<SolverState*>(op->solver));
  op->solver = nullptr;
}

template <typename T> static T* carve(char*& p, size_t count) {
  T* r = reinterpret_cast<T*>(p);
  p += ((count * sizeof(T) + 255) / 256) * 256;
  return r;
}

static size_t carve_bytes(int B, int m, long long N, int nchunk, int G, int Gu) {
  char* p = nullptr;
  carve<float2>(p, (size_t)(m + 1) * B * N);          // V
  carve<float2>(p, (size_t)B * N);                    // W
  carve<float2>(p, (size_t)B * N);                    // d
  carve<float2>(p, (size_t)B * N);                    // r32
  carve<double2>(p, (size_t)B * m * (m + 1));         // H
  carve<double2>(p, (size_t)B * m);                   // cs
  carve<double2>(p, (size_t)B * m);                   // sn
  carve<double2>(p, (size_t)B * (m + 1));             // g
  carve<double2>(p, (size_t)B * 129);                 // coef / y
  carve<double2>(p, (size_t)B * (m + 1) * G);         // partial dots
  carve<double>(p, (size_t)B * std::max(nchunk, Gu)); // norm partials
  for (int i = 0; i < 7; ++i) carve<double>(p, B);    // nrm beta tol_abs rnorm bnorm
  carve<double>(p, (size_t)B * (m + 1));              // sig
  carve<double>(p, (size_t)B * nchunk);               // pb
  for (int i = 0; i < 8; ++i) carve<int>(p, B);       // active iters want counters again ticket mv_active
  for (int i = 0; i < 4; ++i) carve<double2>(p, (size_t)B * N);   // x b64 r64 ax64
  carve<float2>(p, (size_t)N / 3);                    // chi32
  carve<double2>(p, (size_t)N / 3);                   // chi64
  return (size_t)(p - (char*)nullptr);
}

static int get_state(vie_op* op, int B, int m, SolverState** out) {
  SolverState* st = static_cast<SolverState*>(op->solver);
  const long long N = 3LL * op->n[0] * op->n[1] * op->n[2];
  if (st && st->B == B && st->m == m) {
    *out = st;
    return VIE_OK;
  }
  const int wide = (N % 2 == 0) ? 1 : 0;
  const int W = wide ? 2 : 1;
  const long long dtile = (long long)kDotThreads * kDotPacks * W;
  // tiles per CTA: as few as the cap on CTAs allows, and the same for every CTA
  const long long ntile = (N + dtile - 1) / dtile;
  const long long per = (ntile + kMaxDotCtas - 1) / kMaxDotCtas;
  const int G = (int)((ntile + per - 1) / per);
  const int Gu = (int)((N + (long long)kUpdThreads * W - 1) / ((long long)kUpdThreads * W));
  release_state(st);
  op->solver = nullptr;
  op->solve_ws.bytes = 0;
  st = new SolverState();
  st->B = B;
  st->m = m;
  st->N = N;
  st->nchunk = (int)((N + kChunk - 1) / kChunk);
  st->G = G;
  st->Gu = Gu;
  st->wide = wide;
  st->bytes = carve_bytes(B, m, N, st->nchunk, st->G, st->Gu);
  cudaError_t e = cudaMalloc(&st->base, st->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete st;
    set_error("solver workspace of %zu bytes could not be allocated", st->bytes);
    return VIE_ERR_OOM;
  }
  if ((e = cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&st->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&st->aux, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming)) != cudaSuccess) {
    release_state(st);
    return cuda_status(e, "solver stream");
  }
  char* p = st->base;
  const int nc = st->nchunk;
  st->V = carve<float2>(p, (size_t)(m + 1) * B * N);
  st->W = carve<float2>(p, (size_t)B * N);
  st->d = carve<float2>(p, (size_t)B * N);
  st->r32 = carve<float2>(p, (size_t)B * N);
  st->H = carve<double2>(p, (size_t)B * m * (m + 1));
  st->cs = carve<double2>(p, (size_t)B * m);
  st->sn = carve<double2>(p, (size_t)B * m);
  st->g = carve<double2>(p, (size_t)B * (m + 1));
  st->coef = carve<double2>(p, (size_t)B * 129);
  st->partial = carve<double2>(p, (size_t)B * (m + 1) * st->G);
  st->nrm_partial = carve<double>(p, (size_t)B * std::max(nc, st->Gu));
  st->nrm = carve<double>(p, B);
  carve<double>(p, B);
  st->beta = carve<double>(p, B);
  st->tol_abs = carve<double>(p, B);
  st->rnorm = carve<double>(p, B);
  st->bnorm = carve<double>(p, B);
  carve<double>(p, B);
  st->sig = carve<double>(p, (size_t)B * (m + 1));
  st->pb = carve<double>(p, (size_t)B * nc);
  st->active = carve<int>(p, B);
  st->iters = carve<int>(p, B);
  st->want = carve<int>(p, B);
  st->count_it = carve<int>(p, B);
  st->count_mv = carve<int>(p, B);
  st->again = carve<int>(p, B);
  st->ticket = carve<int>(p, B);
  st->mv_active = carve<int>(p, B);
  st->x = carve<double2>(p, (size_t)B * N);
  st->b64 = carve<double2>(p, (size_t)B * N);
  st->r64 = carve<double2>(p, (size_t)B * N);
  st->ax64 = carve<double2>(p, (size_t)B * N);
  st->chi32 = carve<float2>(p, (size_t)N / 3);
  st->chi64 = carve<double2>(p, (size_t)N / 3);
  // tickets start at zero; each use returns its counter to zero
  if ((e = cudaMemset(st->ticket, 0, B * sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(st->again, 0, B * sizeof(int))) != cudaSuccess) {
    release_state(st);
    return cuda_status(e, "solver workspace");
  }
  op->solver = st;
  op->solve_ws.bytes = st->bytes;
  *out = st;
  return VIE_OK;
}

// Wait on stream s for the Givens step running on the side stream.
static int join_givens(SolverState* st, cudaStream_t s) {
  if (!st->givens_pending) return VIE_OK;
  VIE_CUDA(cudaStreamWaitEvent(s, st->ev_join, 0));
  st->givens_pending = false;
  return VIE_OK;
}

// One Arnoldi step k for all active RHS: w = A V_k into basis slot k+1, one
// or two classical Gram-Schmidt passes (the second where the DGKS test asks
// for it), then the Givens step on the side stream, joined before the next
// step's Gram-Schmidt (the next matvec needs only sig[b][k+1]; a right-hand
// side that the Givens step retires meanwhile is skipped from then on and
// its extra matvec output is never read).
static int arnoldi_step(const vie_op* op, SolverState* st, const float2* chi, int k, int path,
                        int adjoint, int passes, cudaStream_t s) {
  const int B = st->B, m = st->m, G = st->G, Gu = st->Gu;
  const long long N = st->N;
  const float2* vk = st->V + (long long)k * B * N;
  float2* w = st->V + (long long)(k + 1) * B * N;
  const size_t flag_bytes = (size_t)B * sizeof(int);
  // The matvec skips right-hand sides by a copy of the active flags taken
  // before the previous step's Givens step was forked: that step may retire a
  // right-hand side while the matvec runs, and every thread of every stage
  // (the producer and consumers of a persistent kernel alike) must take the
  // same decision for it.  A right-hand side retired meanwhile is still
  // multiplied; its output is never read.
  if (k == 0)
    VIE_CUDA(cudaMemcpyAsync(st->mv_active, st->active, flag_bytes, cudaMemcpyDeviceToDevice, s));
  // w = A (sig_k Vraw_k); the rebuild for the next matvec (the next step's or
  // the cycle tail's) starts beside this step's Gram-Schmidt work
  if (!adjoint)
    VIE_TRY(matvec_impl<float>(op, vk, w, B, path, 0, EPI_SUB | EPI_CHI, chi, vk, st->mv_active, s,
                               st->sig + k, m + 1));
  else
    VIE_TRY(matvec_impl<float>(op, vk, w, B, path, PRO_CONJ | PRO_CHI, EPI_CONJ | EPI_SUB, chi, vk,
                               st->mv_active, s, st->sig + k, m + 1));
  VIE_TRY(join_givens(st, s));
  const unsigned long long vec = (unsigned long long)N * sizeof(float2);
  for (int pass = 0; pass < passes; ++pass) {
    const int* mask = pass == 0 ? st->active : st->again;
    const int mode = (pass == 0 && passes > 1) ? UPD_DGKS : UPD_FINAL;
    {
      ProfScope ps(PF_DOTS, s);
      launch_pdl(st->wide ? dots_kernel<2> : dots_kernel<1>, dim3(G, B), dim3(kDotThreads), 0, s,
                 (const float2*)st->V, (const float2*)w, k, B, N, G, m + 1, st->partial, mask,
                 prof_bytes(PF_DOTS), (k + 2) * vec);
    }
    // the next matvec's rebuild, beside the rest of this step's Gram-Schmidt work
    if (pass == 0 && (path == VIE_PATH_TUCKER || path == VIE_PATH_TUCKER_CP))
      VIE_TRY(prefetch_rebuild(op, s, path == VIE_PATH_TUCKER_CP));
    {
      ProfScope ps(PF_SMALL, s);
      launch_pdl(reduce_dots_kernel, dim3(k + 1, B), dim3(kReduceThreads), 0, s,
                 (const double2*)st->partial, k, G, m + 1, (const double*)st->sig, st->coef, st->H, m,
                 pass, mask);
    }
    {
      ProfScope ps(PF_UPDATE, s);
      launch_pdl(st->wide ? update_kernel<2> : update_kernel<1>, dim3(Gu, B), dim3(kUpdThreads), 0,
                 s, (const float2*)st->V, w, (const double2*)st->coef, st->sig, k, m, B, N, Gu,
                 st->nrm_partial, st->ticket, mode, st->nrm, st->again, mask,
                 prof_bytes(PF_UPDATE), (k + 3) * vec);
    }
  }
  // the Givens step beside the next matvec (which reads the flags as they are now)
  if (k + 1 < m)
    VIE_CUDA(cudaMemcpyAsync(st->mv_active, st->active, flag_bytes, cudaMemcpyDeviceToDevice, s));
  VIE_CUDA(cudaEventRecord(st->ev_fork, s));
  VIE_CUDA(cudaStreamWaitEvent(st->aux, st->ev_fork, 0));
  {
    ProfScope ps(PF_SMALL, st->aux);
    givens_kernel<<<(B + 3) / 4, 128, 0, st->aux>>>(st->H, st->cs, st->sn, st->g, st->nrm, k, m, B,
                                                    st->active, st->again, st->iters, st->tol_abs,
                                                    st->count_it);
  }
  VIE_CUDA(cudaEventRecord(st->ev_join, st->aux));
  st->givens_pending = true;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "arnoldi");
  return VIE_OK;
}

// End of a cycle: d += V y, then the true residual r = r32 - A d and the next cycle's start.
static int cycle_tail(const vie_op* op, SolverState* st, const float2* chi, int path, int adjoint,
                      cudaStream_t s) {
  const int B = st->B, m = st->m, nc = st->nchunk;
  const long long N = st->N;
  dim3 grid(nc, B);
  VIE_TRY(join_givens(st, s));
  {
    ProfScope ps(PF_SMALL, s);
    backsolve_kernel<<<(B + 3) / 4, 128, 0, s>>>(st->H, st->g, st->coef, m, B, st->iters);
    combine_kernel<<<grid, kThreads, 0, s>>>(st->V, st->d, st->coef, st->sig, m, B, N, st->iters);
  }
  // W = A d for the RHS still wanted
  if (!adjoint)
    VIE_TRY(matvec_impl<float>(op, st->d, st->W, B, path, 0, EPI_SUB | EPI_CHI, chi, st->d, st->want, s));
  else
    VIE_TRY(matvec_impl<float>(op, st->d, st->W, B, path, PRO_CONJ | PRO_CHI, EPI_CONJ | EPI_SUB, chi,
                               st->d, st->want, s));
  {
    ProfScope ps(PF_SMALL, s);
    residual32_kernel<<<grid, kThreads, 0, s>>>(st->r32, st->W, st->V, N, nc, st->nrm_partial,
                                                st->want);
    reduce_norm_kernel<<<B, 32, 0, s>>>(st->nrm_partial, nc, st->beta, st->want);
    cycle_start_kernel<<<(B + 63) / 64, 64, 0, s>>>(st->beta, st->g, st->sig, m, B, st->want,
                                                   st->active, st->again, st->iters, st->tol_abs,
                                                   st->count_mv);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "cycle tail");
  return VIE_OK;
}

static int run_cycle(const vie_op* op, SolverState* st, const float2* chi, int path, int adjoint,
                     int passes, bool use_graph, cudaStream_t s) {
  st->givens_pending = false;                 // every cycle ends joined
  const_cast<vie_op*>(op)->rb_pending = false;   // (both side streams)
  if (!use_graph) {
    for (int k = 0; k < st->m; ++k) VIE_TRY(arnoldi_step(op, st, chi, k, path, adjoint, passes, s));
    return cycle_tail(op, st, chi, path, adjoint, s);
  }
  // the graph bakes in every pointer it touches: rebuild it when any changes
  if (st->exec && (st->graph_chi != chi || st->graph_stream != s || st->path != path ||
                   st->graph_adjoint != adjoint || st->graph_ws != op->ws.ptr ||
                   st->graph_prof != prof_epoch() || st->graph_passes != passes ||
                   st->graph_cp_epoch != op->cp.epoch)) {
    drop_graph(st);
  }
  if (!st->exec) {
    cudaGraph_t graph;
    VIE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof_set_capture_sink(&st->graph_events);
    int rc = VIE_OK;
    for (int k = 0; k < st->m && rc == VIE_OK; ++k)
      rc = arnoldi_step(op, st, chi, k, path, adjoint, passes, s);
    if (rc == VIE_OK) rc = cycle_tail(op, st, chi, path, adjoint, s);
    prof_set_capture_sink(nullptr);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != VIE_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_status(e, "graph capture");
    e = cudaGraphInstantiate(&st->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      st->exec = nullptr;
      return cuda_status(e, "graph instantiate");
    }
    st->graph_chi = chi;
    st->graph_stream = s;
    st->path = path;
    st->graph_adjoint = adjoint;
    st->graph_ws = op->ws.ptr;
    st->graph_prof = prof_epoch();
    st->graph_passes = passes;
    st->graph_cp_epoch = op->cp.epoch;
  }
  VIE_CUDA(cudaGraphLaunch(st->exec, s));
  st->graph_pending = true;
  return VIE_OK;
}

// after a synchronisation: read the event nodes of the graph replay that just ran
static void harvest_graph(SolverState* st) {
  if (st->graph_pending) prof_harvest_graph(st->graph_events);
  st->graph_pending = false;
}

// A kernel whose bounded wait gave up has set the operator's error word: report
// it (and clear it) after a synchronisation.
static int check_device_error(const vie_op* op, cudaStream_t s) {
  int h = 0;
  VIE_CUDA(cudaMemcpyAsync(&h, op->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  if (h != 0) {
    VIE_CUDA(cudaMemsetAsync(op->dev_err, 0, sizeof(int), s));
    set_error("a bounded device wait gave up (an asynchronous copy did not complete)");
    return VIE_ERR_TIMEOUT;
  }
  return VIE_OK;
}

// FP32 GMRES on r32 (unit-norm rows) to relative tolerance `tol` for the RHS in `want`.
static int inner_gmres(const vie_op* op, SolverState* st, int path, int adjoint, double tol,
                       int max_outer, int passes, bool use_graph, const std::vector<int>& want,
                       cudaStream_t s) {
  const int B = st->B, nc = st->nchunk;
  const long long N = st->N;
  dim3 grid(nc, B);
  std::vector<double> tolv(B, tol);
  VIE_CUDA(cudaMemcpyAsync(st->tol_abs, tolv.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
  VIE_CUDA(cudaMemcpyAsync(st->want, want.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
  // first cycle: d = 0, so the residual is r32 itself
  norm32_kernel<<<grid, kThreads, 0, s>>>(st->r32, N, nc, st->nrm_partial, st->want);
  reduce_norm_kernel<<<B, 32, 0, s>>>(st->nrm_partial, nc, st->beta, st->want);
  cycle_start_kernel<<<(B + 63) / 64, 64, 0, s>>>(st->beta, st->g, st->sig, st->m, B, st->want,
                                                 st->active, st->again, st->iters, st->tol_abs,
                                                 nullptr);
  // basis slot 0 = r32, with factor 1 / beta
  VIE_CUDA(cudaMemcpyAsync(st->V, st->r32, (size_t)B * N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  VIE_CUDA(cudaGetLastError());
  std::vector<int> act(B);
  for (int cycle = 0; cycle < max_outer; ++cycle) {
    VIE_CUDA(cudaMemcpyAsync(act.data(), st->active, B * sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    harvest_graph(st);
    VIE_TRY(check_device_error(op, s));
    int nact = 0;
    for (int b = 0; b < B; ++b) nact += act[b];
    if (nact == 0) return VIE_OK;
    VIE_TRY(run_cycle(op, st, st->chi32, path, adjoint, passes, use_graph, s));
  }
  VIE_CUDA(cudaStreamSynchronize(s));
  harvest_graph(st);
  return VIE_OK;
}

template <typename Tio>
static void load_inputs(SolverState* st, const void* chi, const void* rhs, void* w, int B, long long nvox,
                        int flags, cudaStream_t s) {
  const long long total = 3LL * nvox * B;
  const cx<Tio>* c = static_cast<const cx<Tio>*>(chi);
  load_x_kernel<Tio><<<grid1(nvox), 256, 0, s>>>(c, st->chi64, nvox);
  convert_kernel<float><<<grid1(nvox), 256, 0, s>>>(st->chi64, st->chi32, nvox);
  load_rhs_kernel<Tio><<<grid1(total), 256, 0, s>>>(static_cast<const cx<Tio>*>(rhs), c, st->b64, nvox, B,
                                                   (flags & VIE_SOLVE_RHS_INCIDENT) ? 1 : 0);
  if (flags & VIE_SOLVE_X0)
    load_x_kernel<Tio><<<grid1(total), 256, 0, s>>>(static_cast<const cx<Tio>*>(w), st->x, total);
  else
    cudaMemsetAsync(st->x, 0, total * sizeof(double2), s);
}

static int solve_on(vie_op* op, SolverState* st, const void* chi, const void* rhs, void* w, int B,
                    int flags, int precision, const vie_solve_opts* o, vie_solve_info* info,
                    cudaStream_t s);

int solve_impl(const vie_op* op_c, const void* chi, const void* rhs, void* w, int B, int flags,
               int precision, const vie_solve_opts* o, vie_solve_info* info, cudaStream_t caller) {
  vie_op* op = const_cast<vie_op*>(op_c);
  std::memset(info, 0, sizeof(*info));
  const int m = o->restart;
  const int path = o->path;
  const int adjoint = (flags & VIE_SOLVE_ADJOINT) ? 1 : 0;
  // matvec scratch: the FP32 inner matvecs take all B right-hand sides at once;
  // the FP64 residual matvecs go in as many right-hand sides as fit in it
  VIE_TRY(ensure_workspace_bytes(op, std::max(workspace_bytes_for(op, B, sizeof(float2)),
                                              workspace_bytes_for(op, 1, sizeof(double2)))));
  SolverState* st = nullptr;
  VIE_TRY(get_state(op, B, m, &st));
  (void)path;
  (void)adjoint;
  VIE_CUDA(cudaEventRecord(st->ev_in, caller));
  VIE_CUDA(cudaStreamWaitEvent(st->stream, st->ev_in, 0));
  const int rc = solve_on(op, st, chi, rhs, w, B, flags, precision, o, info, st->stream);
  cudaEventRecord(st->ev_out, st->stream);
  cudaStreamWaitEvent(caller, st->ev_out, 0);
  return rc;
}

static int solve_on(vie_op* op, SolverState* st, const void* chi, const void* rhs, void* w, int B,
                    int flags, int precision, const vie_solve_opts* o, vie_solve_info* info,
                    cudaStream_t s) {
  const int path = o->path;
  // Tucker+CP is an FP32 model: FP64 residuals use the Tucker model it approximates
  const int path64 = path == VIE_PATH_TUCKER_CP ? VIE_PATH_TUCKER : path;
  const int adjoint = (flags & VIE_SOLVE_ADJOINT) ? 1 : 0;
  const long long nvox = (long long)op->n[0] * op->n[1] * op->n[2];
  const long long N = st->N, total = N * B;
  const int nc = st->nchunk;
  dim3 grid(nc, B);
  VIE_CUDA(cudaMemsetAsync(st->count_it, 0, B * sizeof(int), s));
  VIE_CUDA(cudaMemsetAsync(st->count_mv, 0, B * sizeof(int), s));
  if (precision == VIE_C64) load_inputs<float>(st, chi, rhs, w, B, nvox, flags, s);
  else load_inputs<double>(st, chi, rhs, w, B, nvox, flags, s);
  VIE_CUDA(cudaGetLastError());

  std::vector<double> bn(B), rn(B);
  std::vector<int> want(B, 1);
  bool have_x = (flags & VIE_SOLVE_X0) != 0;
  long long mv64 = 0;
  int status = VIE_OK;
  int step = 0;
  for (;; ++step) {
    if (have_x) {
      // A x in FP64, in groups of right-hand sides that fit the matvec scratch
      const int sub = (int)std::max<size_t>(
          1, std::min<size_t>(B, op->ws.bytes / workspace_bytes_for(op, 1, sizeof(double2))));
      for (int b0 = 0; b0 < B; b0 += sub) {
        const int nb = std::min(sub, B - b0);
        const double2* xb = st->x + (long long)b0 * N;
        double2* ab = st->ax64 + (long long)b0 * N;
        if (!adjoint)
          VIE_TRY(matvec_impl<double>(op, xb, ab, nb, path64, 0, EPI_SUB | EPI_CHI, st->chi64, xb,
                                      nullptr, s));
        else
          VIE_TRY(matvec_impl<double>(op, xb, ab, nb, path64, PRO_CONJ | PRO_CHI, EPI_CONJ | EPI_SUB,
                                      st->chi64, xb, nullptr, s));
      }
      mv64 += B;
    }
    {
      ProfScope ps(PF_FP64, s);
      residual64_kernel<<<grid, kThreads, 0, s>>>(st->b64, st->ax64, st->r64, N, nc, st->nrm_partial,
                                                  st->pb, have_x ? 1 : 0);
      reduce_norm2_kernel<<<B, 32, 0, s>>>(st->nrm_partial, nc, st->rnorm, B);
      reduce_norm2_kernel<<<B, 32, 0, s>>>(st->pb, nc, st->bnorm, B);
    }
    VIE_CUDA(cudaGetLastError());
    VIE_CUDA(cudaMemcpyAsync(rn.data(), st->rnorm, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaMemcpyAsync(bn.data(), st->bnorm, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    VIE_TRY(check_device_error(op, s));
    double worst = 0.0;
    bool finite = true;
    for (int b = 0; b < B; ++b) {
      // a non-finite norm (NaN or Inf in the inputs or the iterate) is an error,
      // never a zero right-hand side
      if (!std::isfinite(rn[b]) || !std::isfinite(bn[b])) finite = false;
      const double rel = bn[b] > 0.0 ? rn[b] / bn[b] : 0.0;
      if (!std::isfinite(rel)) finite = false;
      want[b] = rel > o->tol ? 1 : 0;
      worst = std::max(worst, rel);
    }
    if (step < 65) info->history[step] = worst;
    info->relres = worst;
    if (!finite) {
      set_error("non-finite residual in refinement step %d", step);
      status = VIE_ERR_NUMERIC;
      break;
    }
    if (worst <= o->tol) {
      info->converged = 1;
      break;
    }
    if (step >= o->max_refine || (!o->refine && step >= 1)) {
      set_error("relative residual %.3e above %.3e after %d refinement steps", worst, o->tol, step);
      status = VIE_ERR_NO_CONVERGENCE;
      break;
    }
    VIE_CUDA(cudaMemcpyAsync(st->want, want.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    {
      ProfScope ps(PF_FP64, s);
      to_inner_kernel<<<grid, kThreads, 0, s>>>(st->r64, st->rnorm, st->r32, st->d, N, st->want);
    }
    // each refinement step only needs to bring the residual from `worst` to `tol`
    // (with a factor 4 of headroom), never tighter than inner_tol or FP32 allows
    const double need = 0.25 * o->tol / std::max(worst, 1e-300);
    const double itol = o->refine ? std::min(0.5, std::max({o->inner_tol, need, 1e-7})) : o->tol;
    VIE_TRY(inner_gmres(op, st, path, adjoint, itol, o->max_outer, o->orth == 1 ? 1 : 2,
                        o->use_graph != 0, want, s));
    {
      ProfScope ps(PF_FP64, s);
      accumulate_kernel<<<grid, kThreads, 0, s>>>(st->x, st->d, st->rnorm, N, st->want);
    }
    VIE_CUDA(cudaGetLastError());
    have_x = true;
  }
  info->refine_steps = step;
  std::vector<int> ci(B), cm(B);
  VIE_CUDA(cudaMemcpyAsync(ci.data(), st->count_it, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaMemcpyAsync(cm.data(), st->count_mv, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (precision == VIE_C64)
    convert_kernel<float><<<grid1(total), 256, 0, s>>>(st->x, static_cast<float2*>(w), total);
  else
    VIE_CUDA(cudaMemcpyAsync(w, st->x, total * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  long long it = 0, mv = mv64;
  for (int b = 0; b < B; ++b) {
    it += ci[b];
    mv += ci[b] + cm[b];
  }
  info->iterations = (int)std::min<long long>(it, 2147483647LL);
  info->matvecs = (int)std::min<long long>(mv, 2147483647LL);
  return status;
}
