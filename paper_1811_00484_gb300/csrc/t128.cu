// Fused z stage for 64-voxel z edges (P3 = 128): z-FFT of the zero-padded
// lines, voxel-wise product with the six Green's components (Section V.B,
// Table II), inverse z-FFT cropped to the 64 outputs; the same product as
// fused_fs_kernel, laid out like the length-512 kernel.
//
// One CTA of 64 threads per (k1, k2) mirror group, 16 threads per mirror
// line (thread tid: line l = tid >> 4, slot t = tid & 15), two lines per warp,
// so every exchange is inside a warp.  With n = t + 16 b, f = c + 8 k,
// t = e + 4 f', k = g + 4 h:
//   X[c + 8 k] = sum_e w4^{e h} w16^{e g} sum_{f'} w4^{f' g}
//                [ w128^{t c} sum_b x[t + 16 b] w8^{b c} ]
//   pass 1 (thread t):      DFT-8 over b (inputs b >= 4 are the zero padding),
//                           twiddle w128^{t c};                 -> X1[t][c]
//   exchange through shared memory;
//   pass 2 (thread (c, p)): DFT-4 over f' for e = 2p, 2p + 1, twiddle w16^{e g}
//   exchange with the partner thread (c, 1 - p) by shuffles;
//   pass 3 (thread (c, p)): DFT-4 over e for g = 2p, 2p + 1
// leaves frequency c + 8 (2p + gamma) + 32 h in register [gamma][h] of thread
// (c, p) = (tid >> 1, tid & 1).  Each thread carries the three Cartesian
// components of its line through the forward passes, forms Y = D G D J at its
// eight frequencies in registers (G the rebuilt half fibre with the mirror
// signs D folded into its off-diagonal entries, or the stored spectra), and
// runs the passes backwards; the inverse pass 1 computes only the outputs
// b < 4 (the crop).  The line's 64 outputs overwrite its inputs.
#include "stages.cuh"

namespace vie {
namespace t128 {

constexpr int kN = 128;
constexpr int kThreads = 64;
constexpr int kGS = 64 + 8 + 1;             // ghalf_slot(64) + 1
// shared memory: half fibres [6][kGS], w128^m [128], per-slot pass-1 twiddles
// [7][16], and each line's X1 [8][16]
constexpr size_t kSmem = (size_t)(6 * kGS + kN + 7 * 16 + 4 * 8 * 16) * sizeof(float2);

// X1[t][c] lives at c * 16 + (t ^ swz(c)): pass 1 writes a row c from 16
// consecutive t, pass 2 reads t = e + 4 f' with e = 2p + eps across (c, p), and
// the XOR with swz(c) (bits c0, c1, c2 to bits 0, 2, 3) spreads both over the
// 16 float2 bank pairs
__device__ __forceinline__ int xslot(int c, int t) { return c * 16 + (t ^ ((c & 1) | ((c & 6) << 1))); }

__device__ __forceinline__ float2 shfl1(float2 v) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}

// DFT-8 of (v0, v1, v2, v3, 0, 0, 0, 0) (forward), natural order out
__device__ __forceinline__ void dft8_lower_half(const float2 (&v)[4], float2 (&o)[8]) {
  const float r = 0.70710678118654752440f;
  // even part: DFT-4 of (v0, v2, 0, 0); odd part: DFT-4 of (v1, v3, 0, 0)
  const float2 e0 = v[0] + v[2], e2 = v[0] - v[2];
  const float2 e1 = v[0] + mul_mi(v[2]), e3 = v[0] + mul_i(v[2]);
  const float2 p0 = v[1] + v[3], p2 = v[1] - v[3];
  const float2 p1 = v[1] + mul_mi(v[3]), p3 = v[1] + mul_i(v[3]);
  // odd part times exp(-i pi k / 4)
  const float2 t1 = make_float2(r * (p1.x + p1.y), r * (p1.y - p1.x));
  const float2 t2 = mul_mi(p2);
  const float2 t3 = make_float2(r * (p3.y - p3.x), -r * (p3.x + p3.y));
  o[0] = e0 + p0;
  o[4] = e0 - p0;
  o[1] = e1 + t1;
  o[5] = e1 - t1;
  o[2] = e2 + t2;
  o[6] = e2 - t2;
  o[3] = e3 + t3;
  o[7] = e3 - t3;
}

// outputs 0..3 of the inverse DFT-8 of v (exp(+2 pi i b c / 8))
__device__ __forceinline__ void idft8_first_half(const float2 (&v)[8], float2 (&o)[4]) {
  const float r = 0.70710678118654752440f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 p0 = v[1], p1 = v[3], p2 = v[5], p3 = v[7];
  dft4(e0, e1, e2, e3, true);
  dft4(p0, p1, p2, p3, true);
  const float2 t1 = make_float2(r * (p1.x - p1.y), r * (p1.x + p1.y));
  const float2 t2 = mul_i(p2);
  const float2 t3 = make_float2(-r * (p3.x + p3.y), r * (p3.x - p3.y));
  o[0] = e0 + p0;
  o[1] = e1 + t1;
  o[2] = e2 + t2;
  o[3] = e3 + t3;
}

template <bool STORED>
__global__ void __launch_bounds__(kThreads, 8) fused_t128_kernel(const FusedArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ghalf = reinterpret_cast<float2*>(smem_raw);   // [6][kGS]
  float2* roots = ghalf + 6 * kGS;                       // w128^m
  float2* tw1 = roots + kN;                               // [q - 1][t] = w128^{t q}, q = 1..7
  const int tid = threadIdx.x, l = tid >> 4, t = tid & 15;
  float2* xb = tw1 + 7 * 16 + l * 8 * 16;                 // this line's X1
  const int c = t >> 1, p = t & 1;                        // pass 2 / 3 slot
  const int grp = a.g0 + blockIdx.x;
  const int k1 = grp / a.H2, k2 = grp % a.H2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const bool valid = l < nx * ny;
  const int ix = valid ? l / ny : 0, iy = valid ? l % ny : 0;
  const int kx = ix ? a.P1 - k1 : k1, ky = iy ? a.P2 - k2 : k2;
  const long long line_off = ((long long)kx * a.P2 + ky) * 64;
  for (int m = tid; m < kN; m += kThreads) roots[m] = a.roots[m];
  for (int m = tid; m < 7 * 16; m += kThreads) tw1[m] = a.roots[(m & 15) * ((m >> 4) + 1)];
  pdl_trigger();
  pdl_wait();
  if (a.prof != nullptr && grp == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }
  // x[t + 16 q] (q < 4) of component comp of right-hand side b
  auto load_line = [&](int b, int comp, float2 (&x)[4]) {
    const float2* line = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = valid ? line[t + 16 * q] : make_float2(0.f, 0.f);
  };
  auto next_active = [&](int b) {
    if (a.active != nullptr)
      while (b < a.B && a.active[b] == 0) ++b;
    return b;
  };
  // the first active right-hand side's first line is loaded before the half
  // fibres are copied, so the two latencies overlap; later lines are loaded one
  // component ahead
  float2 vc[4];
  int b = next_active(0);
  if (b < a.B) load_line(b, 0, vc);
  if (!STORED) {
    const float2* src = a.octant + ((long long)(k1 - a.oct_k1a) * a.H2 + k2) * 6 * a.H3;
    for (int it = tid; it < 6 * a.H3; it += kThreads) {
      const int cc = it / a.H3, kk = it - cc * a.H3;
      ghalf[cc * kGS + ghalf_slot(kk)] = src[it];
    }
  }
  const float sx = (STORED || !ix) ? 1.f : -1.f, sy = (STORED || !iy) ? 1.f : -1.f;
  __syncthreads();
  bool first = true;
  for (; b < a.B; b = next_active(b + 1)) {   // block-uniform
    if (!first) load_line(b, 0, vc);
    first = false;
    float2 s[3][2][4];                     // [component][gamma][h]: f = c + 8 (2p + gamma) + 32 h
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      float2 vn[4];
      if (comp < 2) load_line(b, comp + 1, vn);
      // pass 1: DFT-8 over b of x[t + 16 b] (b < 4), twiddle w128^{t c}
      float2 x1[8];
      dft8_lower_half(vc, x1);
      if (comp < 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) vc[q] = vn[q];
      }
#pragma unroll
      for (int q = 1; q < 8; ++q) x1[q] = x1[q] * tw1[(q - 1) * 16 + t];
#pragma unroll
      for (int q = 0; q < 8; ++q) xb[xslot(q, t)] = x1[q];
      __syncwarp();
      // pass 2: for e = 2p + eps, DFT-4 over f' of X1[e + 4 f'][c], twiddle w16^{e g}
      float2 u[2][4];
#pragma unroll
      for (int eps = 0; eps < 2; ++eps) {
        const int e = 2 * p + eps;
#pragma unroll
        for (int f = 0; f < 4; ++f) u[eps][f] = xb[xslot(c, e + 4 * f)];
        dft4(u[eps][0], u[eps][1], u[eps][2], u[eps][3], false);
#pragma unroll
        for (int g = 1; g < 4; ++g) u[eps][g] = u[eps][g] * roots[8 * e * g];
      }
      __syncwarp();                         // X1 read: the next component may overwrite it
      // exchange: keep g = 2p + gamma, send the partner's g = 2 (1 - p) + gamma
      float2 r[2][2];
#pragma unroll
      for (int eps = 0; eps < 2; ++eps)
#pragma unroll
        for (int gm = 0; gm < 2; ++gm) r[eps][gm] = shfl1(p ? u[eps][gm] : u[eps][2 + gm]);
      // pass 3: DFT-4 over e for g = 2p + gamma
#pragma unroll
      for (int gm = 0; gm < 2; ++gm) {
        float2 w0 = p ? r[0][gm] : u[0][gm];
        float2 w1 = p ? r[1][gm] : u[1][gm];
        float2 w2 = p ? u[0][2 + gm] : r[0][gm];
        float2 w3 = p ? u[1][2 + gm] : r[1][gm];
        dft4(w0, w1, w2, w3, false);
        s[comp][gm][0] = w0;
        s[comp][gm][1] = w1;
        s[comp][gm][2] = w2;
        s[comp][gm][3] = w3;
      }
    }
    // Y = D G D J at the thread's frequencies
#pragma unroll
    for (int gm = 0; gm < 2; ++gm) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int f = c + 8 * (2 * p + gm) + 32 * h;
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
        const float sxy = sx * sy, sxz = sx * sz, syz = sy * sz;
        const float2 gxy = sxy * G[1], gxz = sxz * G[2], gyz = syz * G[4];
        const float2 jx = s[0][gm][h], jy = s[1][gm][h], jz = s[2][gm][h];
        s[0][gm][h] = cmadd(G[0], jx, cmadd(gxy, jy, gxz * jz));
        s[1][gm][h] = cmadd(gxy, jx, cmadd(G[3], jy, gyz * jz));
        s[2][gm][h] = cmadd(gxz, jx, cmadd(gyz, jy, G[5] * jz));
      }
    }
    // inverse passes, cropped to the 64 outputs
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      float2* line = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
      // inverse pass 3: for g = 2p + gamma, inverse DFT-4 over h -> e, twiddle w16^{-e g}
      float2 z[2][4];
#pragma unroll
      for (int gm = 0; gm < 2; ++gm) {
        const int g = 2 * p + gm;
        float2 w0 = s[comp][gm][0], w1 = s[comp][gm][1], w2 = s[comp][gm][2], w3 = s[comp][gm][3];
        dft4(w0, w1, w2, w3, true);
        z[gm][0] = w0;
        z[gm][1] = w1 * conjg(roots[8 * g]);
        z[gm][2] = w2 * conjg(roots[16 * g]);
        z[gm][3] = w3 * conjg(roots[24 * g]);
      }
      // exchange back: keep e = 2p + eps, send the partner's e = 2 (1 - p) + eps
      float2 r[2][2];
#pragma unroll
      for (int gm = 0; gm < 2; ++gm)
#pragma unroll
        for (int eps = 0; eps < 2; ++eps) r[gm][eps] = shfl1(p ? z[gm][eps] : z[gm][2 + eps]);
      // inverse pass 2: for e = 2p + eps, inverse DFT-4 over g -> f', X1[e + 4 f'][c]
#pragma unroll
      for (int eps = 0; eps < 2; ++eps) {
        const int e = 2 * p + eps;
        float2 w0 = p ? r[0][eps] : z[0][eps];
        float2 w1 = p ? r[1][eps] : z[1][eps];
        float2 w2 = p ? z[0][2 + eps] : r[0][eps];
        float2 w3 = p ? z[1][2 + eps] : r[1][eps];
        dft4(w0, w1, w2, w3, true);
        xb[xslot(c, e)] = w0;
        xb[xslot(c, e + 4)] = w1;
        xb[xslot(c, e + 8)] = w2;
        xb[xslot(c, e + 12)] = w3;
      }
      __syncwarp();
      // inverse pass 1: twiddle w128^{-t c}, inverse DFT-8 over c, outputs b < 4
      float2 x1[8], o[4];
      x1[0] = xb[xslot(0, t)];
#pragma unroll
      for (int q = 1; q < 8; ++q) x1[q] = xb[xslot(q, t)] * conjg(tw1[(q - 1) * 16 + t]);
      idft8_first_half(x1, o);
      if (valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q) line[t + 16 * q] = o[q];
      }
      __syncwarp();                         // X1 read: the next component may overwrite it
    }
  }
}

}  // namespace t128

bool fused_t128_supported(const FusedArgs<float>& a, bool stored) {
  return a.P3 == t128::kN && a.n3 == t128::kN / 2 && (stored || a.octant != nullptr);
}

void launch_fused_t128(const FusedArgs<float>& a, int groups, bool stored, cudaStream_t s) {
  if (stored)
    launch_pdl(t128::fused_t128_kernel<true>, dim3(groups), dim3(t128::kThreads), t128::kSmem, s, a);
  else
    launch_pdl(t128::fused_t128_kernel<false>, dim3(groups), dim3(t128::kThreads), t128::kSmem, s, a);
}

}  // namespace vie
