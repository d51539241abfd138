// Device bodies of the register-path (N = 32 R) matvec stages, shared by the
// per-operator kernels (lines.cu, fused.cu) and the multi-grid kernels
// (multi.cu): one x/y line tile, one fused z-line group, one slab-core block.
#pragma once

#include "warpfft.cuh"

namespace vie {

// sign of component c (xx, xy, xz, yy, yz, zz) under k_q -> P_q - k_q: the
// dyad (k0^2 delta_ab + d_a d_b) g is odd in coordinate q once per index equal to q
__device__ __forceinline__ int parity_sign(int c, int axis) {
  const int a = c < 3 ? 0 : (c < 5 ? 1 : 2);
  const int b = c == 0 ? 0 : (c == 1 || c == 3) ? 1 : 2;
  return (((a == axis) + (b == axis)) & 1) ? -1 : 1;
}

template <typename T> struct SlabArgs {
  const cx<T>* core[6];
  const cx<T>* U1[6];
  int r1[6], r2[6], r3[6];
  cx<T>* slab;
  long long slab_stride;
  int r2max, r3max;
  unsigned long long* prof;
  unsigned long long prof_launch_bytes;
};

template <typename T> struct FusedArgs {
  cx<T>* data;                 // [B*3][P1][P2][n3], transformed in place
  const cx<T>* roots;          // P3-th roots of unity
  FftPlan plan;
  int n3, P1, P2, P3, H1, H2, H3;
  int B;
  long long comp_stride;       // P1 * P2 * n3
  const CompMeta<T>* meta;     // [6] (Tucker)
  int r2max, r3max;
  const cx<T>* spec;           // [6][P1][P2][P3] (stored)
  long long spec_stride;       // P1 * P2 * P3
  const int* active;           // per RHS, nullptr = all
  const cx<T>* octant;         // rebuilt half fibres [k1 - oct_k1a][H2][6][H3] (nullptr: rebuild here)
  int oct_k1a;                 // first k1 held in `octant`
  int oct_chunk;               // k1 values per fill of `octant`
  bool oct_first_ready;        // host: chunk 0 already rebuilt on the side stream (joined)
  const vie_op* op;            // host: the operator (rebuild launches of later chunks)
  bool oct_cp;                 // host: rebuild from the Tucker+CP model (eq. (17))
  int g0;                      // group of the first CTA (k1 chunks)
  int lines_per_round;         // z-lines (x3 components) held in shared memory at once
  int ld;                      // shared-memory line stride
  unsigned long long* prof;    // profiler byte counter (nullptr = off)
  unsigned long long prof_rhs_bytes, prof_launch_bytes;
};

// S_c[k1] = core_c x1 U1_c[k1, :] for one (k1, c): the first stage of eq. (13)
template <typename T>
__device__ __forceinline__ void slab_core_block(const SlabArgs<T>& a, int k1, int c) {
  using C = cx<T>;
  const int r1 = a.r1[c], r2 = a.r2[c], r3 = a.r3[c];
  const C* core = a.core[c];
  const C* u1 = a.U1[c] + (long long)k1 * r1;
  C* S = a.slab + c * a.slab_stride + (long long)k1 * a.r2max * a.r3max;
  for (int it = threadIdx.x; it < r2 * r3; it += blockDim.x) {
    const int b = it / r3, g = it % r3;
    C acc = czero<C>();
    for (int al = 0; al < r1; ++al) acc = cmadd(u1[al], core[(al * r2 + b) * r3 + g], acc);
    S[b * a.r3max + g] = acc;
  }
}

// Tile slot of element (row p, column c): rows of 16 columns with the
// column index XOR-swizzled by (p ^ p>>4 ^ p>>6) mod 16.  Row-wise loads and
// stores stay conflict-free (a permutation within the row), and so do the
// warps' column accesses at natural rows lane + 32 j and at bit-reversed rows
// k1 + R brev5(lane) for every power-of-two R (at most 3-way otherwise).
__device__ __forceinline__ int tile_slot(int p, int c) {
  return p * 16 + (c ^ ((p ^ (p >> 4) ^ (p >> 6)) & 15));
}

constexpr int kLineTile = 16;      // columns per line tile

__host__ __device__ constexpr size_t line_warp_smem(int R) {
  return (size_t)(32 * R * kLineTile + 32 * R) * sizeof(float2);
}

// One tile of 16 contiguous columns of strided lines (an x or y stage), for
// batch index bb and outer index o.  The CTA stages the tile in shared
// memory (coalesced rows), each warp pulls whole columns into registers,
// transforms them with the lane FFT and writes them back; forward transforms
// write the bit-reversed lane layout to natural rows, inverse transforms read
// it from natural rows.  HALF: forward from N/2 loaded points, or inverse
// cropped to N/2 stored points.  Every thread of the block must call it.
template <int R, bool HALF>
__device__ __forceinline__ void line_warp_tile(const LineArgs<float>& a, int c0, int o, int bb,
                                               float2* smem) {
  using C = float2;
  constexpr int N = 32 * R;
  constexpr int TW = kLineTile;
  C* tile = smem;                  // element (row p, column c) at tile_slot(p, c)
  C* roots = smem + N * TW;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  // prologue (tables only), then the preceding kernel's results
  for (int m = tid; m < N; m += nth) roots[m] = a.roots[m];
  pdl_trigger();
  pdl_wait();
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // block-uniform
  if (a.prof != nullptr && c0 == 0 && o == 0 && tid == 0) atomicAdd(a.prof, a.prof_batch_bytes);
  const int ncols = min(TW, a.ncol - c0);
  const float rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                       ? (float)a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                       : 1.f;
  const C* in = a.in + bb * a.in_bs + o * a.in_os + (long long)c0;
  for (int e = tid; e < a.lin * TW; e += nth) {
    const int c = e % TW, p = e / TW;
    if (c < ncols) {
      C v = in[p * a.in_ls + c];
      if (a.flags & PRO_RSCALE) v = rs * v;
      if (a.flags & PRO_CONJ) v = conjg(v);
      if (a.flags & PRO_CHI) v = a.chi[o * a.chi_os + p * a.chi_ls + (long long)(c0 + c)] * v;
      tile[tile_slot(p, c)] = v;
    }
  }
  __syncthreads();

  const int br = brev5(lane);
  LaneConsts<C, float, R> lc;
  lc.init(lane, roots, N);
  for (int c = warp; c < ncols; c += nwarp) {
    C v[R];
    if (!a.inverse) {
#pragma unroll
      for (int j = 0; j < (HALF ? (R + 1) / 2 : R); ++j) {
        const int p = lane + 32 * j;
        v[j] = p < a.lin ? tile[tile_slot(p, c)] : make_float2(0.f, 0.f);
      }
      warp_fft_fwd<C, float, R, HALF>(v, lc, roots, N);
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) {
        const int p = k1 + R * br;
        if (p < a.lout) tile[tile_slot(p, c)] = v[k1];
      }
    } else {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) v[k1] = tile[tile_slot(k1 + R * br, c)];
      warp_fft_inv<C, float, R, HALF>(v, lane, lc, roots, N);
#pragma unroll
      for (int j = 0; j < (HALF ? (R + 1) / 2 : R); ++j) {
        const int p = lane + 32 * j;
        if (p < a.lout) tile[tile_slot(p, c)] = v[j];
      }
    }
  }
  __syncthreads();

  const long long obase = bb * a.out_bs + o * a.out_os + (long long)c0;
  C* out = a.out + obase;
  for (int e = tid; e < a.lout * TW; e += nth) {
    const int c = e % TW, p = e / TW;
    if (c >= ncols) continue;
    C v = a.scale * tile[tile_slot(p, c)];
    if (a.flags & EPI_CONJ) v = conjg(v);
    const long long oi = p * a.out_ls + c;
    if (a.flags & (EPI_SUB | EPI_ADD)) {
      if (a.flags & EPI_CHI) v = a.chi[o * a.chi_os + p * a.chi_ls + (long long)(c0 + c)] * v;
      C w = a.addend[obase + oi];
      if (a.flags & EPI_RSCALE) w = rs * w;
      v = (a.flags & EPI_SUB) ? (w - v) : (w + v);
    }
    out[oi] = v;
  }
}

// Columns per warp of the register-direct line stage: four c64 columns are one
// 32-byte sector of a row.
constexpr int kRegCols = 4;

// One group of kRegCols adjacent columns of strided lines (an x or y stage),
// transformed by one warp straight from and to global memory, no shared
// memory: lane l holds rows l + 32 j (natural order) of every column, or rows
// k1 + R brev5(l) (the lane FFT's bit-reversed order) on the frequency side.
// Each row access moves the group's 32 contiguous bytes, two 16-byte accesses
// when `vec` (the caller has checked that every row of the group starts on a
// 16-byte boundary), one 8-byte access per column otherwise.  HALF: forward
// from N/2 loaded points, or inverse cropped to N/2 stored points.
template <int R, bool HALF>
__device__ __forceinline__ void line_reg_group(const LineArgs<float>& a, int c0, int o, int bb,
                                               bool vec, int lane) {
  using C = float2;
  constexpr int N = 32 * R;
  constexpr int NC = kRegCols;
  constexpr int NH = HALF ? (R + 1) / 2 : R;     // natural-order rows held per lane
  // prologue (tables only), then the preceding kernel's results
  LaneConsts<C, float, R> lc;
  lc.init(lane, a.roots, N);
  pdl_trigger();
  pdl_wait();
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // warp-uniform
  if (a.prof != nullptr && c0 == 0 && o == 0 && lane == 0) atomicAdd(a.prof, a.prof_batch_bytes);
  const int ncols = min(NC, a.ncol - c0);
  const bool v4 = vec && ncols == NC;
  const float rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                       ? (float)a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                       : 1.f;
  const int br = brev5(lane);
  C v[NC][R];
  const C* in = a.in + bb * a.in_bs + o * a.in_os + (long long)c0;
  C* out = a.out + bb * a.out_bs + o * a.out_os + (long long)c0;
  auto load_row = [&](int p, int j) {
    const C* src = in + (long long)p * a.in_ls;
    if (v4) {
      const float4 x0 = *reinterpret_cast<const float4*>(src);
      const float4 x1 = *reinterpret_cast<const float4*>(src + 2);
      v[0][j] = make_float2(x0.x, x0.y);
      v[1][j] = make_float2(x0.z, x0.w);
      v[2][j] = make_float2(x1.x, x1.y);
      v[3][j] = make_float2(x1.z, x1.w);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c][j] = c < ncols ? src[c] : make_float2(0.f, 0.f);
    }
  };
  // kRegCols values of an array laid out like a row of the group (chi, addend)
  auto load4 = [&](const C* src, bool wide, C* x) {
    if (wide) {
      const float4 x0 = *reinterpret_cast<const float4*>(src);
      const float4 x1 = *reinterpret_cast<const float4*>(src + 2);
      x[0] = make_float2(x0.x, x0.y);
      x[1] = make_float2(x0.z, x0.w);
      x[2] = make_float2(x1.x, x1.y);
      x[3] = make_float2(x1.z, x1.w);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = c < ncols ? src[c] : make_float2(0.f, 0.f);
    }
  };
  const bool chi4 = v4 && a.chi_vec;
  auto store_row = [&](int p, int j) {
    C* dst = out + (long long)p * a.out_ls;
    if (v4) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0][j].x, v[0][j].y, v[1][j].x, v[1][j].y);
      *reinterpret_cast<float4*>(dst + 2) = make_float4(v[2][j].x, v[2][j].y, v[3][j].x, v[3][j].y);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < ncols) dst[c] = v[c][j];
    }
  };
  if (!a.inverse) {
#pragma unroll
    for (int j = 0; j < NH; ++j) {
      const int p = lane + 32 * j;
      if (p < a.lin) {
        load_row(p, j);
        if (a.flags & (PRO_RSCALE | PRO_CONJ | PRO_CHI)) {
          C ch[NC];
          if (a.flags & PRO_CHI) load4(a.chi + o * a.chi_os + (long long)p * a.chi_ls + c0, chi4, ch);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            C x = v[c][j];
            if (a.flags & PRO_RSCALE) x = rs * x;
            if (a.flags & PRO_CONJ) x = conjg(x);
            if (a.flags & PRO_CHI) x = ch[c] * x;
            v[c][j] = x;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c][j] = make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) warp_fft_fwd<C, float, R, HALF>(v[c], lc, a.roots, N);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const int p = k1 + R * br;
      if (p < a.lout) store_row(p, k1);
    }
  } else {
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) load_row(k1 + R * br, k1);
#pragma unroll
    for (int c = 0; c < NC; ++c) warp_fft_inv<C, float, R, HALF>(v[c], lane, lc, a.roots, N);
#pragma unroll
    for (int j = 0; j < NH; ++j) {
      const int p = lane + 32 * j;
      if (p < a.lout) {
        if (a.flags & (EPI_CONJ | EPI_SUB | EPI_ADD)) {
          C ch[NC], ad[NC];
          if (a.flags & (EPI_SUB | EPI_ADD)) {
            if (a.flags & EPI_CHI) load4(a.chi + o * a.chi_os + (long long)p * a.chi_ls + c0, chi4, ch);
            load4(a.addend + bb * a.out_bs + o * a.out_os + (long long)c0 + (long long)p * a.out_ls,
                  v4 && a.addend_vec, ad);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            C x = a.scale * v[c][j];
            if (a.flags & EPI_CONJ) x = conjg(x);
            if (a.flags & (EPI_SUB | EPI_ADD)) {
              if (a.flags & EPI_CHI) x = ch[c] * x;
              C w = ad[c];
              if (a.flags & EPI_RSCALE) w = rs * w;
              x = (a.flags & EPI_SUB) ? (w - x) : (w + x);
            }
            v[c][j] = x;
          }
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c][j] = a.scale * v[c][j];
        }
        store_row(p, j);
      }
    }
  }
}

// Two-pass (four-step) variant for N = 8 V, V a multiple of 8: a warp owns
// kRegCols adjacent columns and eight lanes per column, lane = 4 j + c.
//   pass 1 (registers): lane (j, c) holds x[j + 8 m], m < V, of column c, takes
//          the length-V DFT over m and multiplies by w_N^{j k1};
//   exchange (shared memory, one write and one read per value);
//   pass 2 (registers): for k1 = j + 8 t, the length-8 DFT over j gives
//          X[k1 + V k2], k2 < 8.
// The inverse runs the same steps with conjugate roots (unscaled).  For a
// fixed register index the warp's 32 lanes touch 8 rows x 4 columns, i.e.
// whole 32-byte sectors.  No shuffles.  HALF: forward from x[n < N/2] (m < V/2
// nonzero), or inverse cropped to n < N/2 (k2 < 4).
// Exchange layout per warp: [c][j][k1], row stride V+1, column stride
// 8(V+1)+4 (both passes conflict-free within each half-warp).
__host__ __device__ constexpr int fs_col_stride(int V) { return 8 * (V + 1) + 4; }
__host__ __device__ constexpr size_t line_fs_smem(int V, int warps) {
  return (size_t)warps * kRegCols * fs_col_stride(V) * sizeof(float2);
}

template <int V, bool HALF>
__device__ __forceinline__ void line_fs_group(const LineArgs<float>& a, int c0, int o, int bb,
                                              int lane, float2* xs) {
  using C = float2;
  constexpr int N = 8 * V;
  constexpr int S = fs_col_stride(V);
  const int j = lane >> 2, c = lane & 3;
  C* xc = xs + c * S;
  pdl_trigger();
  pdl_wait();
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // warp-uniform
  if (a.prof != nullptr && c0 == 0 && o == 0 && lane == 0) atomicAdd(a.prof, a.prof_batch_bytes);
  const bool col_ok = c0 + c < a.ncol;
  const float rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                       ? (float)a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                       : 1.f;
  const C* in = a.in + bb * a.in_bs + o * a.in_os + (long long)(c0 + c);
  C* out = a.out + bb * a.out_bs + o * a.out_os + (long long)(c0 + c);
  const bool inv = a.inverse != 0;
  C v[V];
  // pass 1: rows j + 8 m
  constexpr int M1 = HALF ? V / 2 : V;         // forward: rows loaded (the rest is padding)
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int p = j + 8 * m;
    C x = make_float2(0.f, 0.f);
    if ((inv || m < M1) && col_ok && p < a.lin) {
      x = in[(long long)p * a.in_ls];
      if (!inv) {
        if (a.flags & PRO_RSCALE) x = rs * x;
        if (a.flags & PRO_CONJ) x = conjg(x);
        if (a.flags & PRO_CHI) x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + c)] * x;
      }
    }
    v[m] = x;
  }
  if (!inv) {
#pragma unroll
    for (int m = M1; m < V; ++m) v[m] = make_float2(0.f, 0.f);   // zero padding, compile-time
  }
  reg_dft<C, float, V>(v, a.roots, N, inv);
#pragma unroll
  for (int k1 = 1; k1 < V; ++k1) {
    const C w = a.roots[j * k1];
    v[k1] = v[k1] * (inv ? conjg(w) : w);
  }
  // exchange: [c][j][k1]
#pragma unroll
  for (int k1 = 0; k1 < V; ++k1) xc[j * (V + 1) + k1] = v[k1];
  __syncwarp();
  // pass 2: k1 = j + 8 t, DFT over the eight j
  constexpr int K2 = (HALF ? 4 : 8);           // inverse: outputs kept (cropped to N/2)
#pragma unroll
  for (int t = 0; t < V / 8; ++t) {
    const int k1 = j + 8 * t;
    C u[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) u[l] = xc[l * (V + 1) + k1];
    reg_dft<C, float, 8>(u, a.roots, N, inv);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      if (inv && k2 >= K2) continue;
      const int p = k1 + V * k2;
      if (!col_ok || p >= a.lout) continue;
      C x = u[k2];
      if (inv) {
        x = a.scale * x;
        if (a.flags & EPI_CONJ) x = conjg(x);
        if (a.flags & (EPI_SUB | EPI_ADD)) {
          if (a.flags & EPI_CHI)
            x = a.chi[o * a.chi_os + (long long)p * a.chi_ls + (long long)(c0 + c)] * x;
          C w = a.addend[bb * a.out_bs + o * a.out_os + (long long)(c0 + c) + (long long)p * a.out_ls];
          if (a.flags & EPI_RSCALE) w = rs * w;
          x = (a.flags & EPI_SUB) ? (w - x) : (w + x);
        }
      }
      out[(long long)p * a.out_ls] = x;
    }
  }
}

// Slot of z-frequency k in a row of the rebuilt half fibre: one padding slot
// every 8 entries, so the lanes' folded, bit-reversed frequencies (stride R)
// fall in different banks (at most 2-way for the radices used, 4-way at R=10).
__device__ __forceinline__ int ghalf_slot(int k) { return k + (k >> 3); }

__host__ __device__ constexpr size_t fused_warp_smem(int R, int H3, int r2max, int r3max) {
  (void)r2max;
  return (size_t)(32 * R + 6 * ((H3 - 1) + ((H3 - 1) >> 3) + 1) + 6 * r3max) * sizeof(float2);
}

// One (k1, k2) mirror group of the fused stage on the register path (P3 = 32 R):
// the four warps of the CTA take one mirror z-line each, hold the three
// components of every right-hand side in registers, and do the forward lane
// FFT, the voxel-wise product with the rebuilt (or stored) components in the
// bit-reversed lane layout, and the inverse lane FFT.  The rebuild of the
// half fibre (k3 <= P3/2) is shared by the CTA.  Every thread must call it.
template <int R, bool STORED>
__device__ __forceinline__ void fused_warp_group(const FusedArgs<float>& a, int g, float2* smem) {
  using C = float2;
  constexpr int P3 = 32 * R;
  constexpr int NLOAD = (R + 1) / 2;               // points lane + 32 j < P3 / 2 + 16
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int n3 = a.n3, H3 = a.H3;
  const int k1 = g / a.H2, k2 = g % a.H2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const int nl = nx * ny;
  const bool has_line = warp < nl;                 // this warp's mirror line
  const int ix = has_line ? warp / ny : 0, iy = has_line ? warp % ny : 0;
  const int kx = ix ? a.P1 - k1 : k1, ky = iy ? a.P2 - k2 : k2;
  const long long line_off = ((long long)kx * a.P2 + ky) * n3;

  const int GS = ghalf_slot(H3 - 1) + 1;   // padded row length of the half fibre
  C* roots = smem;
  C* ghalf = roots + P3;               // [6][GS]
  C* wv = ghalf + 6 * GS;              // [6][r3max]
  // prologue: tables and factors only (no earlier kernel writes them)
  for (int m = tid; m < P3; m += nth) roots[m] = a.roots[m];
  const bool rebuild_here = !STORED && a.octant == nullptr;
  if (rebuild_here) {
    for (int it = tid; it < 6 * a.r3max; it += nth) {
      const int c = it / a.r3max, gm = it % a.r3max;
      const CompMeta<float> m = a.meta[c];
      C acc = make_float2(0.f, 0.f);
      if (gm < m.r3) {
        const C* S = m.slab + (long long)k1 * a.r2max * a.r3max;
        const C* u2 = m.U2 + (long long)k2 * m.r2;
        for (int b = 0; b < m.r2; ++b) acc = cmadd(u2[b], S[b * a.r3max + gm], acc);
      }
      wv[it] = acc;
    }
    __syncthreads();
    for (int it = tid; it < 6 * H3; it += nth) {
      const int c = it / H3, kk = it % H3;
      const CompMeta<float>& m = a.meta[c];
      const C* u3t = m.U3t + kk;              // U3_c[kk, q] at u3t[q * H3]: coalesced
      const C* w = wv + c * a.r3max;
      C acc = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int q = 0; q < m.r3; ++q) acc = cmadd(w[q], u3t[(long long)q * H3], acc);
      ghalf[c * GS + ghalf_slot(kk)] = acc;
    }
  }
  pdl_trigger();
  pdl_wait();

  if (a.prof != nullptr && g == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }
  // the first active right-hand side's lines are loaded before the half fibres
  // are copied, so the two latencies overlap
  int b0 = 0;
  if (a.active != nullptr)
    while (b0 < a.B && a.active[b0] == 0) ++b0;
  C v[3][R];
  auto load_lines = [&](int b) {
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const C* src = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
#pragma unroll
      for (int j = 0; j < NLOAD; ++j) {
        const int p = lane + 32 * j;
        v[comp][j] = p < n3 ? src[p] : make_float2(0.f, 0.f);
      }
    }
  };
  if (has_line && b0 < a.B) load_lines(b0);
  if (!STORED && !rebuild_here) {
    // the group's half fibres, rebuilt for this matvec into the scratch
    const C* src = a.octant + ((long long)(k1 - a.oct_k1a) * a.H2 + k2) * 6 * H3;
    for (int it = tid; it < 6 * H3; it += nth) {
      const int c = it / H3, kk = it - c * H3;
      ghalf[c * GS + ghalf_slot(kk)] = src[it];
    }
  }
  __syncthreads();
  if (!has_line) return;                   // no block barrier follows

  const int br = brev5(lane);
  LaneConsts<C, float, R> lc;
  lc.init(lane, roots, P3);
  // mirror signs: the component (a, b) of the spectrum at the mirror point is
  // s_a s_b times its half-fibre value, s_q = -1 along each mirrored axis, so
  // Y = D G D J with D = diag(s_x, s_y, s_z)
  const float sx = ix ? -1.f : 1.f, sy = iy ? -1.f : 1.f;
  for (int b = b0; b < a.B; ++b) {
    if (a.active != nullptr && a.active[b] == 0) continue;   // warp-uniform
    if (b != b0) load_lines(b);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) warp_fft_fwd<C, float, R, true>(v[comp], lc, roots, P3);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int kk = q + R * br;                       // z-frequency held in register q
      C gc[6];
      C jx = v[0][q], jy = v[1][q], jz = v[2][q];
      float sz = 1.f;
      if (STORED) {
        const long long off = ((long long)kx * a.P2 + ky) * P3 + kk;
#pragma unroll
        for (int c = 0; c < 6; ++c) gc[c] = a.spec[c * a.spec_stride + off];
      } else {
        const bool zm = 2 * kk > P3;
        const int fold = zm ? P3 - kk : kk;
        sz = zm ? -1.f : 1.f;
        const C* gp = ghalf + ghalf_slot(fold);
#pragma unroll
        for (int c = 0; c < 6; ++c) gc[c] = gp[c * GS];
        jx = sx * jx;
        jy = sy * jy;
        jz = sz * jz;
      }
      // Y_a = sum_b G_ab J_b with G symmetric: xx xy xz / xy yy yz / xz yz zz
      const C yx = gc[0] * jx + gc[1] * jy + gc[2] * jz;
      const C yy = gc[1] * jx + gc[3] * jy + gc[4] * jz;
      const C yz = gc[2] * jx + gc[4] * jy + gc[5] * jz;
      if (STORED) {
        v[0][q] = yx;
        v[1][q] = yy;
        v[2][q] = yz;
      } else {
        v[0][q] = sx * yx;
        v[1][q] = sy * yy;
        v[2][q] = sz * yz;
      }
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      warp_fft_inv<C, float, R, true>(v[comp], lane, lc, roots, P3);
      C* dst = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
#pragma unroll
      for (int j = 0; j < NLOAD; ++j) {
        const int p = lane + 32 * j;
        if (p < n3) dst[p] = v[comp][j];
      }
    }
  }
}

// Fused z stage with the four-step transform (P3 = 8 V): one CTA of three warps
// per (k1, k2) mirror group, warp = Cartesian component of J and Y, lane =
// 4 j + l with l the mirror line (up to four) and j the eighth of the line.
//   forward: pass 1 / exchange / pass 2 as in line_fs_group, then the
//            component's spectrum goes to a shared buffer spec[comp][l][f];
//   product: each lane forms Y_comp[l][f] = s_comp sum_b G_comp,b[fold f] s_b J_b[l][f]
//            (D G D, with G the rebuilt half fibre, or the stored spectra) for
//            the frequencies f = j + 8 m its inverse pass 1 needs;
//   inverse: pass 1 / exchange / pass 2 cropped to n3 outputs, written in place.
// Every thread must call it.
__host__ __device__ constexpr int fused_fs_spec_stride(int V) { return 8 * V + 4; }
__host__ __device__ constexpr size_t fused_fs_smem(int V, int H3) {
  return (size_t)(6 * ((H3 - 1) + ((H3 - 1) >> 3) + 1) + 3 * 4 * fused_fs_spec_stride(V) +
                  3 * kRegCols * fs_col_stride(V)) *
         sizeof(float2);
}

template <int V, bool STORED>
__device__ __forceinline__ void fused_fs_group(const FusedArgs<float>& a, int g, float2* smem) {
  using C = float2;
  constexpr int N = 8 * V;                     // P3
  constexpr int XS = fs_col_stride(V);
  constexpr int SS = fused_fs_spec_stride(V);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, comp = tid >> 5;  // three warps (a fourth, if any, only helps copy)
  const bool act = comp < 3;
  const int j = lane >> 2, ln = lane & 3;
  const int n3 = a.n3, H3 = a.H3;
  const int k1 = g / a.H2, k2 = g % a.H2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const bool valid = ln < nx * ny;
  const int ix = valid ? ln / ny : 0, iy = valid ? ln % ny : 0;
  const int kx = ix ? a.P1 - k1 : k1, ky = iy ? a.P2 - k2 : k2;
  const long long line_off = ((long long)kx * a.P2 + ky) * n3;
  const int GS = ghalf_slot(H3 - 1) + 1;
  C* ghalf = smem;                              // [6][GS]
  C* spec = ghalf + 6 * GS;                     // [3][4][SS]
  C* xw = spec + 3 * 4 * SS + (act ? comp : 0) * kRegCols * XS;   // this warp's exchange buffer
  C* xc = xw + ln * XS;
  pdl_trigger();
  pdl_wait();
  if (a.prof != nullptr && g == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }
  if (!STORED) {
    // the group's half fibres, rebuilt for this matvec into the scratch
    const C* src = a.octant + ((long long)(k1 - a.oct_k1a) * a.H2 + k2) * 6 * H3;
    for (int it = tid; it < 6 * H3; it += nth) {
      const int c = it / H3, kk = it - c * H3;
      ghalf[c * GS + ghalf_slot(kk)] = src[it];
    }
  }
  // rows of G used by this warp's component: x: xx xy xz, y: xy yy yz, z: xz yz zz
  const int g0 = comp == 0 ? 0 : (comp == 1 ? 1 : 2);
  const int g1 = comp == 0 ? 1 : (comp == 1 ? 3 : 4);
  const int g2 = comp == 0 ? 2 : (comp == 1 ? 4 : 5);
  const float sx = ix ? -1.f : 1.f, sy = iy ? -1.f : 1.f;
  const float sc = comp == 0 ? sx : (comp == 1 ? sy : 1.f);
  __syncthreads();
  for (int b = 0; b < a.B; ++b) {
    if (a.active != nullptr && a.active[b] == 0) continue;   // block-uniform
    C* line = a.data + (long long)(b * 3 + (act ? comp : 0)) * a.comp_stride + line_off;
    C v[V];
    if (act) {
      // forward pass 1: x[j + 8 m], m < V/2 (the rest is zero padding)
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const int p = j + 8 * m;
        v[m] = (m < V / 2 && valid && p < n3) ? line[p] : make_float2(0.f, 0.f);
      }
      reg_dft<C, float, V>(v, a.roots, N, false);
#pragma unroll
      for (int q = 1; q < V; ++q) v[q] = v[q] * a.roots[j * q];
#pragma unroll
      for (int q = 0; q < V; ++q) xc[j * (V + 1) + q] = v[q];
      __syncwarp();
      // forward pass 2 -> spec[comp][ln][q + V k2]
      C* sp = spec + (comp * 4 + ln) * SS;
#pragma unroll
      for (int t = 0; t < V / 8; ++t) {
        const int q = j + 8 * t;
        C u[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) u[l] = xc[l * (V + 1) + q];
        reg_dft<C, float, 8>(u, a.roots, N, false);
#pragma unroll
        for (int k = 0; k < 8; ++k) sp[q + V * k] = u[k];
      }
    }
    __syncthreads();
    if (act) {
      // product at f = j + 8 m, straight into the inverse pass 1 registers
      const C* s0 = spec + (0 * 4 + ln) * SS;
      const C* s1 = spec + (1 * 4 + ln) * SS;
      const C* s2 = spec + (2 * 4 + ln) * SS;
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const int f = j + 8 * m;
        C G0, G1, G2;
        float sz = 1.f;
        if (STORED) {
          const long long off = ((long long)kx * a.P2 + ky) * N + f;
          G0 = a.spec[g0 * a.spec_stride + off];
          G1 = a.spec[g1 * a.spec_stride + off];
          G2 = a.spec[g2 * a.spec_stride + off];
        } else {
          const bool zm = 2 * f > N;
          const int fold = zm ? N - f : f;
          sz = zm ? -1.f : 1.f;
          const C* gp = ghalf + ghalf_slot(fold);
          G0 = gp[g0 * GS];
          G1 = gp[g1 * GS];
          G2 = gp[g2 * GS];
        }
        // stored spectra are complete: no mirror signs
        const float ex = STORED ? 1.f : sx, ey = STORED ? 1.f : sy;
        C y = G0 * (ex * s0[f]) + G1 * (ey * s1[f]) + G2 * (sz * s2[f]);
        if (!STORED) y = (comp == 2 ? sz : sc) * y;
        v[m] = y;
      }
      // inverse pass 1 (exchange buffer free: pass 2 read it before the barrier)
      reg_dft<C, float, V>(v, a.roots, N, true);
#pragma unroll
      for (int q = 1; q < V; ++q) v[q] = v[q] * conjg(a.roots[j * q]);
#pragma unroll
      for (int q = 0; q < V; ++q) xc[j * (V + 1) + q] = v[q];
      __syncwarp();
      // inverse pass 2, cropped: n = q + V k2 < N / 2
#pragma unroll
      for (int t = 0; t < V / 8; ++t) {
        const int q = j + 8 * t;
        C u[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) u[l] = xc[l * (V + 1) + q];
        reg_dft<C, float, 8>(u, a.roots, N, true);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int n = q + V * k;
          if (valid && n < n3) line[n] = u[k];
        }
      }
    }
    __syncthreads();                           // spec and xw reused by the next right-hand side
  }
}

// Length-512 kernels (tp512.cu): x / y line stages and the fused z stage
bool launch_line_tp(LineArgs<float> a, cudaStream_t s);
bool launch_line_tp64(LineArgs<double> a, cudaStream_t s);
bool fused_tp_supported(const FusedArgs<float>& a, bool stored);
void launch_fused_tp(const FusedArgs<float>& a, int groups, bool stored, cudaStream_t s);
// P3 = 128 (64-voxel z edges): 16 threads per line, radix 8, 4, 4 (t128.cu)
bool fused_t128_supported(const FusedArgs<float>& a, bool stored);
void launch_fused_t128(const FusedArgs<float>& a, int groups, bool stored, cudaStream_t s);

}  // namespace vie
