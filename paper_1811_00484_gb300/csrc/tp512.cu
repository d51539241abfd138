// Length-512 transforms of the matvec (Section V.B) for 256-voxel grid edges
// (P = 512): the x and y line stages and the fused z stage (zero-padded
// forward z-FFT, voxel-wise product with the rebuilt or stored spectra,
// cropped inverse z-FFT).
//
// Three radix-8 passes, 64 threads per line, 8 values per thread.  With
// n = a + 64 b (a < 64, b < 8), a = e + 8 f and k = c + 8 g + 64 h,
//   X[c + 8g + 64h] = sum_e w8^{eh} w64^{eg} sum_f w8^{fg} w512^{ac}
//                     sum_b w8^{bc} x[a + 64 b],
// so
//   pass 1 (thread a):      DFT-8 over b, twiddle w512^{a c}, store X1[c][a]
//   pass 2 (thread (c, e)): DFT-8 over f (a = e + 8f), twiddle w64^{e g},
//                           store X2[c][g][e]
//   pass 3 (thread (c, g)): DFT-8 over e, giving X[c + 8g + 64h] in register h.
// The inverse runs the three passes backwards (inverse DFT-8s, conjugate
// twiddles), from the register layout where the forward one ends to the
// layout where it starts, so a forward / product / inverse sequence never
// reorders data.  Zero padding (x[n] = 0 for n >= 256: b >= 4) and cropping
// (outputs n < 256) prune the first and last passes.
//
// Exchange layouts (float2 units): X1[c][a] at c LA + a, X2[c][g][e] at
// c 72 + 9 g + e.  Each half-warp's 64-bit accesses of every pass fall in 16
// different bank pairs (checked for both thread layouts below).
#include <algorithm>

#include "stages.cuh"
#include "tma.cuh"

namespace vie {

namespace tp {

constexpr int kN = 512;
constexpr int kM = 64;            // threads per line
constexpr int kX2 = 576;          // 8 x 72 per line

template <typename C>
__device__ __forceinline__ C root(const C* roots, int e, bool inv) {
  const C w = __ldg(roots + e);
  return inv ? conjg(w) : w;
}

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

// DFT-8 of x[0..3] with x[4..7] = 0: X[2k] = DFT4(x)[k], X[2k+1] = DFT4(x_n w8^n)[k]
template <typename C>
__device__ __forceinline__ void dft8_half_in(C* v, bool inv) {
  using T = typename RealOf<C>::type;
  const T r = (T)0.70710678118654752440;
  C e0 = v[0], e1 = v[1], e2 = v[2], e3 = v[3];
  C o0 = v[0], o1, o2, o3;
  if (!inv) {
    o1 = mk(r * (v[1].x + v[1].y), r * (v[1].y - v[1].x));
    o2 = mul_mi(v[2]);
    o3 = mk(r * (v[3].y - v[3].x), -r * (v[3].x + v[3].y));
  } else {
    o1 = mk(r * (v[1].x - v[1].y), r * (v[1].x + v[1].y));
    o2 = mul_i(v[2]);
    o3 = mk(-r * (v[3].x + v[3].y), r * (v[3].x - v[3].y));
  }
  dft4(e0, e1, e2, e3, inv);
  dft4(o0, o1, o2, o3, inv);
  v[0] = e0; v[2] = e1; v[4] = e2; v[6] = e3;
  v[1] = o0; v[3] = o1; v[5] = o2; v[7] = o3;
}

// pass 1 in thread a: v[b] = x[a + 64 b]  ->  X1[c][a]
template <bool INV, bool HALF_IN, typename C>
__device__ __forceinline__ void pass1(C (&v)[8], int a, const C* roots, C* x1, int la) {
  if (HALF_IN) dft8_half_in(v, INV); else dft8<C, typename RealOf<C>::type>(v, INV);
#pragma unroll
  for (int c = 1; c < 8; ++c) v[c] = v[c] * root(roots, a * c, INV);
#pragma unroll
  for (int c = 0; c < 8; ++c) x1[c * la + a] = v[c];
}

// pass 2 in thread (c, e): X1[c][e + 8f]  ->  X2[c][g][e]
template <bool INV, typename C>
__device__ __forceinline__ void pass2(int c, int e, const C* x1, int la, C* x2, const C* roots) {
  C u[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) u[f] = x1[c * la + e + 8 * f];
  dft8<C, typename RealOf<C>::type>(u, INV);
#pragma unroll
  for (int g = 1; g < 8; ++g) u[g] = u[g] * root(roots, 8 * e * g, INV);
#pragma unroll
  for (int g = 0; g < 8; ++g) x2[c * 72 + 9 * g + e] = u[g];
}

// pass 3 in thread (c, g): X2[c][g][e]  ->  w[h] = X[c + 8 g + 64 h]
template <bool INV, typename C>
__device__ __forceinline__ void pass3(int c, int g, const C* x2, C (&w)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) w[e] = x2[c * 72 + 9 * g + e];
  dft8<C, typename RealOf<C>::type>(w, INV);
}

// inverse of pass 3 in thread (c, g): w[h] = Y[c + 8g + 64h]  ->  X2[c][g][e]
__device__ __forceinline__ void ipass3(int c, int g, float2 (&w)[8], float2* x2, const float2* roots) {
  dft8<float2, float>(w, true);
#pragma unroll
  for (int e = 1; e < 8; ++e) w[e] = w[e] * root(roots, 8 * e * g, true);
#pragma unroll
  for (int e = 0; e < 8; ++e) x2[c * 72 + 9 * g + e] = w[e];
}

// inverse of pass 2 in thread (c, e): X2[c][g][e]  ->  X1[c][e + 8f]
__device__ __forceinline__ void ipass2(int c, int e, const float2* x2, float2* x1, int la,
                                       const float2* roots) {
  float2 u[8];
#pragma unroll
  for (int g = 0; g < 8; ++g) u[g] = x2[c * 72 + 9 * g + e];
  dft8<float2, float>(u, true);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const int a = e + 8 * f;
    x1[c * la + a] = (c == 0) ? u[f] : u[f] * root(roots, a * c, true);
  }
}

// inverse of pass 1 in thread a: X1[c][a]  ->  v[b] = 512 x[a + 64 b]
__device__ __forceinline__ void ipass1(int a, const float2* x1, int la, float2 (&v)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = x1[c * la + a];
  dft8<float2, float>(v, true);
}

// Per-slot twiddle table in shared memory, [22][64] (row j, slot t):
//   rows 0..6   w512^{t c},             c = 1..7        (pass 1)
//   rows 7..13  w64^{(t mod 8) x},      x = 1..7        (pass 2, inverse pass 3)
//   rows 14..21 w512^{(t mod 8 + 8 f) (t div 8)}, f = 0..7   (inverse pass 2)
// The same for every line, tile and right-hand side a thread handles.
constexpr int kTwRows = 22;
__device__ __forceinline__ void fill_twiddles(float2* tw, const float2* roots, int tid, int nth) {
  for (int i = tid; i < kTwRows * kM; i += nth) {
    const int j = i / kM, t = i % kM;
    int e;
    if (j < 7) e = t * (j + 1);
    else if (j < 14) e = 8 * (t & 7) * (j - 6);
    else e = ((t & 7) + 8 * (j - 14)) * (t >> 3);
    tw[i] = roots[e];
  }
}
__device__ __forceinline__ float2 twv(const float2* tw, int row, int t, bool inv) {
  const float2 w = tw[row * kM + t];
  return inv ? conjg(w) : w;
}

template <bool INV, bool HALF_IN>
__device__ __forceinline__ void pass1t(float2 (&v)[8], int a, const float2* tw, float2* x1, int la) {
  if (HALF_IN) dft8_half_in(v, INV); else dft8<float2, float>(v, INV);
#pragma unroll
  for (int c = 1; c < 8; ++c) v[c] = v[c] * twv(tw, c - 1, a, INV);
#pragma unroll
  for (int c = 0; c < 8; ++c) x1[c * la + a] = v[c];
}

// pass 2 up to its twiddles (the caller stores u[g] at X2[c][g][e]); slot t = 8 c + e
template <bool INV>
__device__ __forceinline__ void pass2t_load(float2 (&u)[8], int t, const float2* x1, int la,
                                            const float2* tw) {
  const int c = t >> 3, e = t & 7;
#pragma unroll
  for (int f = 0; f < 8; ++f) u[f] = x1[c * la + e + 8 * f];
  dft8<float2, float>(u, INV);
#pragma unroll
  for (int g = 1; g < 8; ++g) u[g] = u[g] * twv(tw, 6 + g, t, INV);
}

// inverse of pass 3 in slot t = 8 c + g
__device__ __forceinline__ void ipass3t(int t, float2 (&w)[8], float2* x2, const float2* tw) {
  const int c = t >> 3, g = t & 7;
  dft8<float2, float>(w, true);
#pragma unroll
  for (int e = 1; e < 8; ++e) w[e] = w[e] * twv(tw, 6 + e, t, true);
#pragma unroll
  for (int e = 0; e < 8; ++e) x2[c * 72 + 9 * g + e] = w[e];
}

// inverse of pass 2 in slot t = 8 c + e
__device__ __forceinline__ void ipass2t(int t, const float2* x2, float2* x1, int la, const float2* tw) {
  const int c = t >> 3, e = t & 7;
  float2 u[8];
#pragma unroll
  for (int g = 0; g < 8; ++g) u[g] = x2[c * 72 + 9 * g + e];
  dft8<float2, float>(u, true);
#pragma unroll
  for (int f = 0; f < 8; ++f) x1[c * la + e + 8 * f] = u[f] * twv(tw, 14 + f, t, true);
}

// ---------------------------------------------------------------------------
// x / y line stage: 8 adjacent columns per CTA, 64 threads per column.
// Thread tid: column col = tid & 7, slot t = tid >> 3.  A warp's global
// accesses are 4 rows x 64 contiguous bytes.  X1 column stride 514, X2 578
// (both 2 mod 16 in float2 units).
// ---------------------------------------------------------------------------
constexpr int kLineCols = 8;
constexpr int kCS1 = 514, kCS2 = 578;
constexpr size_t kLineSmem = (size_t)kLineCols * (kCS1 + kCS2) * sizeof(float2);

// INV: inverse transform (conjugate roots); HALF: forward from x[n < 256]
// (the rest zero padding) or inverse cropped to outputs n < 256
template <bool INV, bool HALF>
__global__ void __launch_bounds__(512, 3) line_tp_kernel(const LineArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x, col = tid & 7, t = tid >> 3;
  float2* x1 = sm + col * kCS1;
  float2* x2 = sm + kLineCols * kCS1 + col * kCS2;
  const int c0 = blockIdx.x * kLineCols, o = blockIdx.y, bb = blockIdx.z;
  pdl_trigger();
  pdl_wait();
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // block-uniform
  if (a.prof != nullptr && blockIdx.x == 0 && o == 0 && tid == 0) atomicAdd(a.prof, a.prof_batch_bytes);
  const bool col_ok = c0 + col < a.ncol;
  const float rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                       ? (float)a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                       : 1.f;
  const float2* in = a.in + bb * a.in_bs + o * a.in_os + (long long)(c0 + col);
  float2 v[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int p = t + kM * b;
    float2 x = make_float2(0.f, 0.f);
    if ((INV || !HALF || b < 4) && col_ok && p < a.lin) {
      x = in[(long long)p * a.in_ls];
      if (!INV) {
        if (a.flags & PRO_RSCALE) x = rs * x;
        if (a.flags & PRO_CONJ) x = conjg(x);
        if (a.flags & PRO_CHI) x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * x;
      }
    }
    v[b] = x;
  }
  pass1<INV, !INV && HALF>(v, t, a.roots, x1, 64);
  __syncthreads();
  pass2<INV>(t >> 3, t & 7, x1, 64, x2, a.roots);
  __syncthreads();
  const int c = t >> 3, g = t & 7;
  pass3<INV>(c, g, x2, v);
  float2* out = a.out + bb * a.out_bs + o * a.out_os + (long long)(c0 + col);
  if (!col_ok) return;
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    if (INV && HALF && h >= 4) continue;
    const int p = c + 8 * g + kM * h;
    if (p >= a.lout) continue;
    float2 x = v[h];
    if (INV) {
      x = a.scale * x;
      if (a.flags & EPI_CONJ) x = conjg(x);
      if (a.flags & (EPI_SUB | EPI_ADD)) {
        if (a.flags & EPI_CHI) x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * x;
        float2 w = a.addend[bb * a.out_bs + o * a.out_os + (long long)(c0 + col) + (long long)p * a.out_ls];
        if (a.flags & EPI_RSCALE) w = rs * w;
        x = (a.flags & EPI_SUB) ? (w - x) : (w + x);
      }
    }
    out[(long long)p * a.out_ls] = x;
  }
}

// ---------------------------------------------------------------------------
// The same line stage as a persistent kernel whose input tiles arrive by TMA:
// each CTA walks its tiles (8 columns x one line position range) through a
// ring of `nstage` input buffers, so that the next tiles' copies are in
// flight while the current one is transformed; one exchange buffer serves
// as X1 and then as X2.  A tile is one or two boxes of 256 rows x 8 columns,
// stored [row][column].
// ---------------------------------------------------------------------------
constexpr size_t kPipeX = (size_t)kLineCols * kCS2 * sizeof(float2);   // X1 / X2 (37 KB)
constexpr size_t kTwBytes = (size_t)kTwRows * kM * sizeof(float2);       // 11 KB
constexpr unsigned long long kWaitNs = 1000000000ull;     // 1 s per bounded wait
constexpr int kMaxStages = 4;

struct PipeTiles {
  int ncg;              // column groups
  int ntiles;           // ncg * nother * nbatch
  int rows;             // input rows per tile (256 or 512)
  int p_dim;            // tensor-map dimension of the line position (1 or 2; the other is `o`)
  int nstage;           // ring depth (2 .. kMaxStages)
};

__host__ __device__ constexpr size_t pipe_stage_bytes(int rows) {
  return (size_t)rows * kLineCols * sizeof(float2);
}
__host__ __device__ constexpr size_t pipe_smem(int rows, int nstage) {
  return (size_t)nstage * pipe_stage_bytes(rows) + kPipeX + kTwBytes + kMaxStages * sizeof(uint64_t) +
         1024;
}

// Position of a tile (column group, other index, batch index) of the CTA's
// sequence blockIdx.x, blockIdx.x + G, ...: stepped by G with carries, no
// divisions.
struct TilePos {
  int cg, o, bb;
};
struct TileStep {
  int cg, o, bb;        // G split into the three digits (cg fastest)
};

template <bool INV, bool HALF, bool FLAGS>
__global__ void __launch_bounds__(512, 2) line_tpp_kernel(const LineArgs<float> a,
                                                        const __grid_constant__ CUtensorMap map,
                                                        const PipeTiles pt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int sbytes = (int)pipe_stage_bytes(pt.rows);
  const int NS = pt.nstage;
  auto stage = [&](int s) { return reinterpret_cast<float2*>(base + s * sbytes); };
  float2* xb = reinterpret_cast<float2*>(base + NS * sbytes);
  float2* tw = reinterpret_cast<float2*>(base + NS * sbytes + kPipeX);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + NS * sbytes + kPipeX + kTwBytes);
  const int tid = threadIdx.x, col = tid & 7, t = tid >> 3;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  fill_twiddles(tw, a.roots, tid, blockDim.x);
  __syncthreads();
  pdl_trigger();
  pdl_wait();
  const int ncg = pt.ncg, nother = a.nother, nbatch = a.nbatch;
  TileStep st;
  {
    const int G = gridDim.x;
    st.cg = G % ncg;
    const int r = G / ncg;
    st.o = r % nother;
    st.bb = r / nother;
  }
  auto advance = [&](TilePos& q) {
    q.cg += st.cg;
    int carry = q.cg >= ncg;
    if (carry) q.cg -= ncg;
    q.o += st.o + carry;
    carry = q.o >= nother;
    if (carry) q.o -= nother;
    q.bb += st.bb + carry;
  };
  // the next tile at or after q (in steps of G) whose right-hand side is active
  auto settle = [&](TilePos& q) {
    if (a.active == nullptr) return;
    while (q.bb < nbatch && a.active[q.bb / 3] == 0) advance(q);
  };
  const int box_rows = pt.rows < 256 ? pt.rows : 256;
  auto issue = [&](const TilePos& q, int s) {
    mbar_arrive_expect_tx(&bar[s], (unsigned)sbytes);
    for (int p0 = 0; p0 < pt.rows; p0 += box_rows) {
      const int c1 = pt.p_dim == 1 ? p0 : q.o, c2 = pt.p_dim == 1 ? q.o : p0;
      tma_load_4d(stage(s) + p0 * kLineCols, &map, q.cg * kLineCols, c1, c2, q.bb, &bar[s]);
    }
  };
  TilePos cur;
  {
    const int b0 = blockIdx.x;
    cur.cg = b0 % ncg;
    const int r = b0 / ncg;
    cur.o = r % nother;
    cur.bb = r / nother;
  }
  settle(cur);
  // the ring holds the tile cur and the next NS - 1 ones (ahead is the newest)
  TilePos ahead = cur;
  if (tid == 0 && cur.bb < nbatch) issue(cur, 0);
  for (int q = 1; q < NS; ++q) {
    if (ahead.bb < nbatch) {
      advance(ahead);
      settle(ahead);
    }
    if (tid == 0 && ahead.bb < nbatch) issue(ahead, q);
  }
  if (a.prof != nullptr && blockIdx.x == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int bb = 0; bb < nbatch; ++bb) nb += (a.active == nullptr || a.active[bb / 3]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_batch_bytes);
  }
  const int c = t >> 3, g = t & 7;
  const long long out_step = (long long)kM * a.out_ls;
  int s = 0;
  unsigned phase_bits = 0;                        // bit q: parity of the next wait on stage q
  while (cur.bb < nbatch) {
    const bool ok = mbar_wait_bounded(&bar[s], (phase_bits >> s) & 1u, kWaitNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.err != nullptr) atomicExch(a.err, VIE_ERR_TIMEOUT);
      for (int q = 0; q < NS; ++q) mbar_wait_bounded(&bar[q], (phase_bits >> q) & 1u, kWaitNs);
      return;
    }
    phase_bits ^= 1u << s;
    const int o = cur.o, bb = cur.bb;
    const int c0 = cur.cg * kLineCols;
    const bool col_ok = c0 + col < a.ncol;
    float rs = 1.f;
    if (FLAGS && (a.flags & (PRO_RSCALE | EPI_RSCALE)))
      rs = (float)a.rscale[(long long)(bb / 3) * a.rscale_stride];
    const float2* S = stage(s) + col;
    float2 v[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int p = t + kM * b;
      float2 x = make_float2(0.f, 0.f);
      if (INV || !HALF || b < 4) {
        x = S[p * kLineCols];
        if (FLAGS && !INV) {
          if (a.flags & PRO_RSCALE) x = rs * x;
          if (a.flags & PRO_CONJ) x = conjg(x);
          if ((a.flags & PRO_CHI) && col_ok)
            x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * x;
        }
      }
      v[b] = x;
    }
    __syncthreads();                       // stage s read; the exchange buffer is free
    if (ahead.bb < nbatch) {
      advance(ahead);
      settle(ahead);
    }
    if (tid == 0 && ahead.bb < nbatch) {
      fence_proxy_async_smem();
      issue(ahead, s);
    }
    float2* x1 = xb + col * kCS1;
    float2* x2 = xb + col * kCS2;
    pass1t<INV, !INV && HALF>(v, t, tw, x1, 64);
    __syncthreads();
    {
      float2 u[8];
      pass2t_load<INV>(u, t, x1, 64, tw);
      __syncthreads();                     // X1 read: X2 overwrites the same buffer
#pragma unroll
      for (int q = 0; q < 8; ++q) x2[c * 72 + 9 * q + g] = u[q];
    }
    __syncthreads();
    pass3<INV>(c, g, x2, v);
    if (col_ok) {
      float2* out = a.out + bb * a.out_bs + o * a.out_os + (long long)(c0 + col) +
                    (long long)(c + 8 * g) * a.out_ls;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        if (INV && HALF && h >= 4) continue;
        float2 x = v[h];
        if (INV) {
          x = a.scale * x;
          if (FLAGS) {
            const int p = c + 8 * g + kM * h;
            if (a.flags & EPI_CONJ) x = conjg(x);
            if (a.flags & (EPI_SUB | EPI_ADD)) {
              if (a.flags & EPI_CHI)
                x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * x;
              float2 w = a.addend[bb * a.out_bs + o * a.out_os + (long long)(c0 + col) +
                                  (long long)p * a.out_ls];
              if (a.flags & EPI_RSCALE) w = rs * w;
              x = (a.flags & EPI_SUB) ? (w - x) : (w + x);
            }
          }
        }
        out[h * out_step] = x;
      }
    }
    s = (s + 1 == NS) ? 0 : s + 1;
    advance(cur);
    settle(cur);
  }
}

// ---------------------------------------------------------------------------
// FP64 line stage (the refinement residuals): 4 adjacent columns per CTA, 64
// threads per column (col = tid & 3, slot t = tid >> 2; a warp's global
// accesses are 8 rows x 64 contiguous bytes), one exchange buffer per column
// used as X1 and then X2, twiddles read from the root table.  Bound by FP64
// arithmetic.
// ---------------------------------------------------------------------------
constexpr int kCols64 = 4;
constexpr int kX64 = 580;
constexpr size_t kLine64Smem = (size_t)kCols64 * kX64 * sizeof(double2);

template <bool INV, bool HALF>
__global__ void __launch_bounds__(256, 3) line_tp64_kernel(const LineArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, col = tid & 3, t = tid >> 2;
  double2* x = reinterpret_cast<double2*>(smem_raw) + col * kX64;
  const int c0 = blockIdx.x * kCols64, o = blockIdx.y, bb = blockIdx.z;
  pdl_trigger();
  pdl_wait();
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // block-uniform
  const bool col_ok = c0 + col < a.ncol;
  const double rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                        ? a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                        : 1.0;
  const double2* in = a.in + bb * a.in_bs + o * a.in_os + (long long)(c0 + col);
  double2 v[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int p = t + kM * b;
    double2 xv = make_double2(0.0, 0.0);
    if ((INV || !HALF || b < 4) && col_ok && p < a.lin) {
      xv = in[(long long)p * a.in_ls];
      if (!INV) {
        if (a.flags & PRO_RSCALE) xv = rs * xv;
        if (a.flags & PRO_CONJ) xv = conjg(xv);
        if (a.flags & PRO_CHI) xv = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * xv;
      }
    }
    v[b] = xv;
  }
  pass1<INV, !INV && HALF>(v, t, a.roots, x, 64);
  __syncthreads();
  const int c = t >> 3, g = t & 7;
  {
    double2 u[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) u[f] = x[c * 64 + g + 8 * f];
    dft8<double2, double>(u, INV);
#pragma unroll
    for (int q = 1; q < 8; ++q) u[q] = u[q] * root(a.roots, 8 * g * q, INV);
    __syncthreads();                       // X1 read: X2 overwrites the same buffer
#pragma unroll
    for (int q = 0; q < 8; ++q) x[c * 72 + 9 * q + g] = u[q];
  }
  __syncthreads();
  pass3<INV>(c, g, x, v);
  if (!col_ok) return;
  double2* out = a.out + bb * a.out_bs + o * a.out_os + (long long)(c0 + col);
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    if (INV && HALF && h >= 4) continue;
    const int p = c + 8 * g + kM * h;
    if (p >= a.lout) continue;
    double2 xv = v[h];
    if (INV) {
      xv = a.scale * xv;
      if (a.flags & EPI_CONJ) xv = conjg(xv);
      if (a.flags & (EPI_SUB | EPI_ADD)) {
        if (a.flags & EPI_CHI) xv = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + col)] * xv;
        double2 w = a.addend[bb * a.out_bs + o * a.out_os + (long long)(c0 + col) + (long long)p * a.out_ls];
        if (a.flags & EPI_RSCALE) w = rs * w;
        xv = (a.flags & EPI_SUB) ? (w - xv) : (w + xv);
      }
    }
    out[(long long)p * a.out_ls] = xv;
  }
}

// ---------------------------------------------------------------------------
// Fused z stage: one CTA of 256 threads per (k1, k2) mirror group, 64 threads
// per mirror line (thread tid: line l = tid >> 6, slot t = tid & 63).  Each
// thread carries the three Cartesian components of its line through the
// forward passes (one after another, sharing the line's exchange buffers),
// holds their spectra at the eight frequencies c + 8g + 64h in registers,
// forms Y = D G D J there (G the rebuilt half fibre with mirror signs D, or
// the stored spectra), and runs the inverse passes.  The line's 256 outputs
// overwrite its 256 inputs.
// ---------------------------------------------------------------------------
constexpr int kGS = 256 + 32 + 1;     // ghalf_slot(256) + 1
constexpr int kLA = 72;               // X1 row stride of the fused layout
constexpr size_t kFusedSmem = (size_t)(6 * kGS + 4 * kX2 + 4 * kX2 + kTwRows * kM) * sizeof(float2);

template <bool STORED>
__global__ void __launch_bounds__(256, STORED ? 2 : 3) fused_tp_kernel(const FusedArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ghalf = reinterpret_cast<float2*>(smem_raw);   // [6][kGS]
  const int tid = threadIdx.x, l = tid >> 6, t = tid & 63;
  float2* x1 = ghalf + 6 * kGS + l * kX2;
  float2* x2 = ghalf + 6 * kGS + 4 * kX2 + l * kX2;
  float2* tw = ghalf + 6 * kGS + 8 * kX2;
  const int grp = a.g0 + blockIdx.x;
  const int k1 = grp / a.H2, k2 = grp % a.H2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const bool valid = l < nx * ny;                          // warp-uniform
  const int ix = valid ? l / ny : 0, iy = valid ? l % ny : 0;
  const int kx = ix ? a.P1 - k1 : k1, ky = iy ? a.P2 - k2 : k2;
  const long long line_off = ((long long)kx * a.P2 + ky) * a.n3;
  const int n3 = a.n3;
  fill_twiddles(tw, a.roots, tid, 256);
  pdl_trigger();
  pdl_wait();
  if (a.prof != nullptr && grp == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }
  if (!STORED) {
    const float2* src = a.octant + ((long long)(k1 - a.oct_k1a) * a.H2 + k2) * 6 * a.H3;
    for (int it = tid; it < 6 * a.H3; it += 256) {
      const int cc = it / a.H3, kk = it - cc * a.H3;
      ghalf[cc * kGS + ghalf_slot(kk)] = src[it];
    }
  }
  const float sx = (STORED || !ix) ? 1.f : -1.f, sy = (STORED || !iy) ? 1.f : -1.f;
  const int c = t >> 3, g = t & 7;
  __syncthreads();
  for (int b = 0; b < a.B; ++b) {
    if (a.active != nullptr && a.active[b] == 0) continue;   // block-uniform
    float2 s[3][8];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float2* line = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int p = t + kM * m;
        v[m] = (m < 4 && valid && p < n3) ? line[p] : make_float2(0.f, 0.f);
      }
      pass1t<false, true>(v, t, tw, x1, kLA);
      __syncthreads();
      {
        float2 u[8];
        pass2t_load<false>(u, t, x1, kLA, tw);
#pragma unroll
        for (int q = 0; q < 8; ++q) x2[c * 72 + 9 * q + (t & 7)] = u[q];
      }
      __syncthreads();
      pass3<false>(c, g, x2, s[comp]);
    }
    // Y = D G D J at f = c + 8 g + 64 h
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int f = c + 8 * g + kM * h;
      float2 G[6];
      float sz = 1.f;
      if (STORED) {
        const long long off = ((long long)kx * a.P2 + ky) * kN + f;
#pragma unroll
        for (int q = 0; q < 6; ++q) G[q] = __ldg(a.spec + q * a.spec_stride + off);
      } else {
        const bool zm = 2 * f > kN;
        const int fold = zm ? kN - f : f;
        sz = zm ? -1.f : 1.f;
        const float2* gp = ghalf + ghalf_slot(fold);
#pragma unroll
        for (int q = 0; q < 6; ++q) G[q] = gp[q * kGS];
      }
      // D G D with the mirror signs folded into the off-diagonal entries
      const float sxy = sx * sy, sxz = sx * sz, syz = sy * sz;
      const float2 gxy = sxy * G[1], gxz = sxz * G[2], gyz = syz * G[4];
      const float2 jx = s[0][h], jy = s[1][h], jz = s[2][h];
      s[0][h] = cmadd(G[0], jx, cmadd(gxy, jy, gxz * jz));
      s[1][h] = cmadd(gxy, jx, cmadd(G[3], jy, gyz * jz));
      s[2][h] = cmadd(gxz, jx, cmadd(gyz, jy, G[5] * jz));
    }
    // inverse passes: the first writes X1 (in the X2 layout), which the forward
    // passes last read before the barrier that preceded pass 3, the second
    // reads X1 and writes X2 (layout of X1), the third reads X2
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      float2* line = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
      ipass3t(t, s[comp], x1, tw);
      __syncthreads();
      ipass2t(t, x1, x2, kLA, tw);
      __syncthreads();
      float2 v[8];
      ipass1(t, x2, kLA, v);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int p = t + kM * m;
        if (valid && p < n3) line[p] = v[m];
      }
    }
    // the next right-hand side's pass 1 writes X1, last read by the inverse pass
    // 2 above before the barrier that preceded the inverse pass 1
  }
}

}  // namespace tp

static int g_sms = 0;

// the TMA-pipelined persistent form: input rows 256 or 512, strides of 16-byte
// multiples, 16-byte aligned input
static bool launch_line_tpp(LineArgs<float> a, bool half, cudaStream_t s) {
  const int rows = a.lin;
  if (rows != 256 && rows != 512) return false;
  // every tile's rows are loaded and, inverse and halved, its first 256 outputs
  // stored: the kernel relies on lin = N (inverse) or N / 2 (forward halved)
  // and lout = N / 2 (inverse halved) or N (forward)
  if (a.inverse ? (rows != 512 || a.lout != (half ? 256 : 512)) : (a.lout != 512 || rows != (half ? 256 : 512)))
    return false;
  if (a.batch_per_rhs != 3) return false;
  if (((uintptr_t)a.in & 15u) != 0 || a.in_os % 2 || a.in_ls % 2 || a.in_bs % 2) return false;
  tp::PipeTiles pt;
  pt.ncg = (a.ncol + tp::kLineCols - 1) / tp::kLineCols;
  if ((long long)pt.ncg * a.nother * a.nbatch >= (1LL << 31)) return false;
  pt.ntiles = pt.ncg * a.nother * a.nbatch;
  pt.rows = rows;
  pt.p_dim = a.in_ls < a.in_os ? 1 : 2;
  const unsigned long long dp = (unsigned long long)rows, doth = (unsigned long long)a.nother;
  const unsigned long long dims[4] = {(unsigned long long)a.ncol, pt.p_dim == 1 ? dp : doth,
                                      pt.p_dim == 1 ? doth : dp, (unsigned long long)a.nbatch};
  const unsigned long long strides[3] = {(unsigned long long)(pt.p_dim == 1 ? a.in_ls : a.in_os),
                                         (unsigned long long)(pt.p_dim == 1 ? a.in_os : a.in_ls),
                                         (unsigned long long)a.in_bs};
  pt.nstage = rows == 256 ? 4 : 2;
  const unsigned box_rows = rows < 256 ? rows : 256;
  const unsigned box[4] = {(unsigned)tp::kLineCols, pt.p_dim == 1 ? box_rows : 1u,
                           pt.p_dim == 1 ? 1u : box_rows, 1u};
  CUtensorMap map;
  if (encode_tensor_map_c64(&map, a.in, 4, dims, strides, box) != VIE_OK) return false;
  if (g_sms == 0) g_sms = device_sms();
  const long long grid = std::min<long long>(pt.ntiles, 2LL * g_sms);
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  const size_t smem = tp::pipe_smem(rows, pt.nstage);
  using K = void (*)(LineArgs<float>, CUtensorMap, tp::PipeTiles);
  static const K kernels[2][2][2] = {
      {{tp::line_tpp_kernel<false, false, false>, tp::line_tpp_kernel<false, false, true>},
       {tp::line_tpp_kernel<false, true, false>, tp::line_tpp_kernel<false, true, true>}},
      {{tp::line_tpp_kernel<true, false, false>, tp::line_tpp_kernel<true, false, true>},
       {tp::line_tpp_kernel<true, true, false>, tp::line_tpp_kernel<true, true, true>}}};
  const K k = kernels[a.inverse ? 1 : 0][half ? 1 : 0][a.flags != 0 ? 1 : 0];
  launch_pdl(k, dim3((unsigned)grid), dim3(512), smem, s, a, map, pt);
  return true;
}

// x / y stage of a length-512 line (columns contiguous in memory)
bool launch_line_tp(LineArgs<float> a, cudaStream_t s) {
  if (a.plan.N != tp::kN || a.in_cs != 1 || a.out_cs != 1) return false;
  if ((a.flags & (PRO_CHI | EPI_CHI)) && a.chi_cs != 1) return false;
  if (a.nother > 65535 || a.nbatch > 65535) return false;
  const bool half = a.inverse ? (2 * a.lout == tp::kN) : (2 * a.lin == tp::kN);
  if (launch_line_tpp(a, half, s)) return true;
  dim3 grid((a.ncol + tp::kLineCols - 1) / tp::kLineCols, a.nother, a.nbatch);
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  if (a.inverse)
    launch_pdl(half ? tp::line_tp_kernel<true, true> : tp::line_tp_kernel<true, false>, grid,
               dim3(512), tp::kLineSmem, s, a);
  else
    launch_pdl(half ? tp::line_tp_kernel<false, true> : tp::line_tp_kernel<false, false>, grid,
               dim3(512), tp::kLineSmem, s, a);
  return true;
}

// FP64 x / y stage of a length-512 line (columns contiguous in memory)
bool launch_line_tp64(LineArgs<double> a, cudaStream_t s) {
  if (a.plan.N != tp::kN || a.in_cs != 1 || a.out_cs != 1) return false;
  if ((a.flags & (PRO_CHI | EPI_CHI)) && a.chi_cs != 1) return false;
  if (a.nother > 65535 || a.nbatch > 65535) return false;
  const bool half = a.inverse ? (2 * a.lout == tp::kN) : (2 * a.lin == tp::kN);
  dim3 grid((a.ncol + tp::kCols64 - 1) / tp::kCols64, a.nother, a.nbatch);
  a.prof = nullptr;
  ProfScope ps(a.prof_family, s);
  if (a.inverse)
    launch_pdl(half ? tp::line_tp64_kernel<true, true> : tp::line_tp64_kernel<true, false>, grid,
               dim3(256), tp::kLine64Smem, s, a);
  else
    launch_pdl(half ? tp::line_tp64_kernel<false, true> : tp::line_tp64_kernel<false, false>, grid,
               dim3(256), tp::kLine64Smem, s, a);
  return true;
}

// fused z stage over the mirror groups [a.g0, a.g0 + groups) (P3 = 512, n3 <= 256)
bool fused_tp_supported(const FusedArgs<float>& a, bool stored) {
  return a.P3 == tp::kN && 2 * a.n3 <= tp::kN && (stored || a.octant != nullptr);
}

void launch_fused_tp(const FusedArgs<float>& a, int groups, bool stored, cudaStream_t s) {
  if (stored)
    launch_pdl(tp::fused_tp_kernel<true>, dim3(groups), dim3(256), tp::kFusedSmem, s, a);
  else
    launch_pdl(tp::fused_tp_kernel<false>, dim3(groups), dim3(256), tp::kFusedSmem, s, a);
}

}  // namespace vie

int tp_init_attributes() {
  cudaError_t e = cudaSuccess;
  const int ls = (int)vie::tp::kLineSmem, fs = (int)vie::tp::kFusedSmem;
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::line_tp_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ls);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::line_tp_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ls);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::line_tp_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ls);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::line_tp_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ls);
  const int ps = (int)std::max(vie::tp::pipe_smem(256, 4), vie::tp::pipe_smem(512, 2));
#define VIE_TPP_ATTR(I, H, F) \
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::line_tpp_kernel<I, H, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps)
  VIE_TPP_ATTR(false, false, false); VIE_TPP_ATTR(false, false, true);
  VIE_TPP_ATTR(false, true, false); VIE_TPP_ATTR(false, true, true);
  VIE_TPP_ATTR(true, false, false); VIE_TPP_ATTR(true, false, true);
  VIE_TPP_ATTR(true, true, false); VIE_TPP_ATTR(true, true, true);
#undef VIE_TPP_ATTR
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::fused_tp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::tp::fused_tp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "length-512 kernel attributes");
}

// Host: tiled tensor map of 8-byte elements through the driver entry point
// (looked up once; the library links only the runtime).
int encode_tensor_map_c64(CUtensorMap* map, const void* base, int rank, const unsigned long long* dims,
                          const unsigned long long* strides, const unsigned* box) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Encode>(p);
    else
      cudaGetLastError();
    looked = true;
  }
  if (fn == nullptr || rank < 1 || rank > 5) return VIE_ERR_ARG;
  cuuint64_t gd[5], gs[4];
  cuuint32_t bd[5], es[5];
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bd[i] = box[i];
    es[i] = 1;
    if (i > 0) gs[i - 1] = strides[i - 1] * 8ull;
  }
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void*>(base), gd,
                        gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? VIE_OK : VIE_ERR_ARG;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: one thread waits on a shared-memory mbarrier
// for at most `limit_ns`; with arrive = 1 the barrier's single arrival is
// made first (the wait completes), with arrive = 0 nothing arrives and the
// wait must give up.  status: 1 completed, 2 gave up.
// ---------------------------------------------------------------------------
namespace vie {
__global__ void bounded_wait_selftest_kernel(int arrive, unsigned long long limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  mbar_fence_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  *status = mbar_wait_bounded(&bar, 0, limit_ns) ? 1 : 2;
}
}  // namespace vie

int grid_barrier_selftest(bool all_arrive, double seconds, cudaStream_t s);

extern "C" int vie_selftest_bounded_wait(int arrive, double seconds, void* stream) {
  clear_error();
  if (seconds <= 0.0 || seconds > 10.0 || arrive < 0 || arrive > 3) {
    set_error("wait limit %g s outside (0, 10] or unknown kind %d", seconds, arrive);
    return VIE_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (arrive >= 2) return grid_barrier_selftest(arrive == 3, seconds, s);
  int* d = nullptr;
  VIE_CUDA(cudaMalloc(&d, sizeof(int)));
  int h = 0;
  vie::bounded_wait_selftest_kernel<<<1, 1, 0, s>>>(arrive ? 1 : 0,
                                                      (unsigned long long)(seconds * 1e9), d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(e, "bounded-wait self-test");
  if (h == 2) {
    set_error("the bounded wait gave up after %g s", seconds);
    return VIE_ERR_TIMEOUT;
  }
  return h == 1 ? VIE_OK : VIE_ERR_CUDA;
}
