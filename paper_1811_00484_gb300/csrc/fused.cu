// Fused z-axis FFT, voxel-wise product and inverse z-FFT: the element-wise
// product of the matvec (Section V.B, Table II) with the components rebuilt
// from their Tucker form at every matvec.
//
// The rebuild follows eq. (13) in three stages:
//   slab cores   S_c[k1] = core_c x1 U1_c[k1, :]            (r2 x r3, once, at setup)
//   one fibre    G_c[k1, k2, k3] = sum_g ( U2_c[k2, :] S_c[k1] )[g] U3_c[k3, g]
// The spectrum of every component is even or odd along each axis
// (G_c[P - k] = s G_c[k], s = -1 when the component is odd in that
// coordinate), and so are the HOSVD factors of its unfoldings.  Only the half
// fibres k3 <= P3/2 of the octant k1 <= P1/2, k2 <= P2/2 are rebuilt, and
// each serves, with signs, the up-to-four z-lines (k1 | P1-k1, k2 | P2-k2)
// of every right-hand side.  On the register path the half fibres of a chunk
// of k1 are rebuilt into an FP32 scratch (one k1 chunk at a time, so the
// scratch stays a small fraction of the uncompressed spectra) by
// octant_tc_kernel on the tensor cores (or octant_kernel with FP32 FMAs, or,
// for the Tucker+CP model of eq. (17), octant_cp_kernel), and one CTA per
// (k1, k2) mirror group copies its 6 x (P3/2 + 1) values to shared memory;
// the multi-grid and shared-memory variants rebuild the fibre in the CTA.
// The stored (uncompressed) variant reads the six spectra from memory instead.
#include <algorithm>

#include "stages.cuh"

namespace vie {

template <typename T>
__global__ void __launch_bounds__(256) slab_core_kernel(const SlabArgs<T> a) {
  if (a.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(a.prof, a.prof_launch_bytes);
  slab_core_block<T>(a, blockIdx.x, blockIdx.y);
}

template <typename T, bool STORED>
__global__ void __launch_bounds__(256, 3) fused_z_kernel(const FusedArgs<T> a) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nth = blockDim.x;
  if (a.prof != nullptr && blockIdx.x == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }
  const int P3 = a.P3, n3 = a.n3, ld = a.ld, H3 = a.H3;
  const int g = blockIdx.x;
  const int k1 = g / a.H2, k2 = g % a.H2;
  const int xs0 = k1, xs1 = a.P1 - k1;
  const int ys0 = k2, ys1 = a.P2 - k2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const int nl = nx * ny;
  const int LR = a.lines_per_round;

  C* roots = reinterpret_cast<C*>(smem_raw);
  C* ghalf = roots + P3;               // [6][H3]
  C* wv = ghalf + 6 * H3;              // [6][r3max]
  C* buf0 = wv + 6 * a.r3max;          // [LR*3][ld]
  C* buf1 = buf0 + LR * 3 * ld;

  for (int m = tid; m < P3; m += nth) roots[m] = a.roots[m];

  if (!STORED) {
    for (int it = tid; it < 6 * a.r3max; it += nth) {
      const int c = it / a.r3max, gm = it % a.r3max;
      const CompMeta<T> m = a.meta[c];
      C acc = czero<C>();
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
      const CompMeta<T> m = a.meta[c];
      const C* u3 = m.U3 + (long long)kk * m.r3;
      const C* w = wv + c * a.r3max;
      C acc = czero<C>();
      for (int q = 0; q < m.r3; ++q) acc = cmadd(w[q], u3[q], acc);
      ghalf[it] = acc;
    }
  }
  __syncthreads();

  for (int b = 0; b < a.B; ++b) {
    if (a.active != nullptr && a.active[b] == 0) continue;   // block-uniform
    for (int l0 = 0; l0 < nl; l0 += LR) {
      const int nlr = min(LR, nl - l0);
      const int nlines = nlr * 3;
      for (int e = tid; e < nlines * P3; e += nth) {
        const int line = e / P3, p = e % P3;
        const int l = l0 + line / 3, comp = line % 3;
        const int kx = (l / ny) ? xs1 : xs0, ky = (l % ny) ? ys1 : ys0;
        C v = czero<C>();
        if (p < n3)
          v = a.data[(long long)(b * 3 + comp) * a.comp_stride + ((long long)kx * a.P2 + ky) * n3 + p];
        buf0[line * ld + p] = v;
      }
      __syncthreads();
      C* F = fft_lines<T, false>(buf0, buf1, a.plan, nlines, ld, 1, roots, false, tid, nth);
      C* Fo = (F == buf0) ? buf1 : buf0;

      for (int e = tid; e < nlr * P3; e += nth) {
        const int lr = e / P3, kk = e % P3;
        const int l = l0 + lr;
        const int ix = l / ny, iy = l % ny;
        C* base = F + lr * 3 * ld + kk;
        const C jx = base[0], jy = base[ld], jz = base[2 * ld];
        C gc[6];
        if (STORED) {
          const int kx = ix ? xs1 : xs0, ky = iy ? ys1 : ys0;
          const long long off = ((long long)kx * a.P2 + ky) * P3 + kk;
#pragma unroll
          for (int c = 0; c < 6; ++c) gc[c] = a.spec[c * a.spec_stride + off];
        } else {
          const bool zm = 2 * kk > P3;
          const int fold = zm ? P3 - kk : kk;
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            int s = 1;
            if (ix) s *= parity_sign(c, 0);
            if (iy) s *= parity_sign(c, 1);
            if (zm) s *= parity_sign(c, 2);
            const C v = ghalf[c * H3 + fold];
            gc[c] = (s > 0) ? v : mk(-v.x, -v.y);
          }
        }
        // Y_a = sum_b G_ab J_b with G symmetric: xx xy xz / xy yy yz / xz yz zz
        base[0] = gc[0] * jx + gc[1] * jy + gc[2] * jz;
        base[ld] = gc[1] * jx + gc[3] * jy + gc[4] * jz;
        base[2 * ld] = gc[2] * jx + gc[4] * jy + gc[5] * jz;
      }
      __syncthreads();
      C* R = fft_lines<T, false>(F, Fo, a.plan, nlines, ld, 1, roots, true, tid, nth);

      for (int e = tid; e < nlines * n3; e += nth) {
        const int line = e / n3, p = e % n3;
        const int l = l0 + line / 3, comp = line % 3;
        const int kx = (l / ny) ? xs1 : xs0, ky = (l % ny) ? ys1 : ys0;
        a.data[(long long)(b * 3 + comp) * a.comp_stride + ((long long)kx * a.P2 + ky) * n3 + p] =
            R[line * ld + p];
      }
      __syncthreads();
    }
  }
}

// Register-resident variant for P3 = 32 R: one CTA of four warps per (k1, k2)
// mirror group, see fused_warp_group.
// Resident CTAs per SM the register budget is sized for (up to radix 4: 96
// registers, five CTAs of four warps; radix 5-6: 128; radix 8: 168).
__host__ __device__ constexpr int fused_min_blocks(int R) {
  return R <= 4 ? 5 : (R <= 6 ? 4 : (R <= 8 ? 3 : 2));
}

template <int R, bool STORED>
__global__ void __launch_bounds__(128, fused_min_blocks(R)) fused_warp_kernel(const FusedArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fused_warp_group<R, STORED>(a, a.g0 + blockIdx.x, reinterpret_cast<float2*>(smem_raw));
}

// Rebuild of the half fibres of eq. (13) for k1 in [k1a, k1a + gridDim.y), every
// k2 and k3 <= P3/2, into out[k1 - k1a][k2][c][k3]:
//   W_c[k2, q]      = sum_b U2_c[k2, b] S_c[k1][b, q]          (S = slab core)
//   G_c[k1, k2, k3] = sum_q W_c[k2, q] U3_c[k3, q]
// One CTA per (k1, kOctK2 values of k2).  Each thread keeps the kOctK2 values
// of one (c, q) or (c, k3) in registers, so every factor entry it loads serves
// kOctK2 independent multiply-adds; U3 is read transposed (consecutive k3 at
// consecutive addresses) and the output rows (k3 fastest) are written
// contiguously.
constexpr int kOctK2 = kOctantK2;
__host__ __device__ constexpr size_t octant_smem(int r2max, int r3max) {
  return octant_smem_bytes(r2max, r3max);
}

struct OctArgs {
  const CompMeta<float>* meta;
  int r2max, r3max, H2, H3;
  int k1a;
  float2* out;
};

__global__ void __launch_bounds__(256) octant_kernel(const OctArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* W = reinterpret_cast<float2*>(smem_raw);     // [6][r3max][kOctK2]
  float2* Ss = W + 6 * a.r3max * kOctK2;               // [6][r2max][r3max]  slab cores of k1
  float2* U2s = Ss + 6 * a.r2max * a.r3max;            // [6][kOctK2][r2max] U2 rows k2_0 ..
  __shared__ CompMeta<float> meta[6];
  if (threadIdx.x < 6) meta[threadIdx.x] = a.meta[threadIdx.x];
  __syncthreads();
  const int k1l = blockIdx.y, k1 = a.k1a + k1l;
  const int k2_0 = blockIdx.x * kOctK2;
  const int nk2 = min(kOctK2, a.H2 - k2_0);
  const int r23 = a.r2max * a.r3max;
  // stage the slab cores of k1 and the U2 rows of this CTA's k2 (all loads in flight)
  for (int it = threadIdx.x; it < 6 * r23; it += blockDim.x) {
    const int c = it / r23;
    Ss[it] = meta[c].slab[(long long)k1 * r23 + (it - c * r23)];
  }
  for (int it = threadIdx.x; it < 6 * kOctK2 * a.r2max; it += blockDim.x) {
    const int b = it % a.r2max, ct = it / a.r2max, t = ct % kOctK2, c = ct / kOctK2;
    const CompMeta<float>& m = meta[c];
    U2s[it] = (t < nk2 && b < m.r2) ? m.U2[(long long)(k2_0 + t) * m.r2 + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // W[c][q][t] = sum_b U2_c[k2_0 + t, b] S_c[k1][b, q]: one (c, q) per thread, all t
  for (int it = threadIdx.x; it < 6 * a.r3max; it += blockDim.x) {
    const int c = it / a.r3max, q = it - c * a.r3max;
    const int r2 = meta[c].r2;
    const float2* S = Ss + c * r23 + q;
    const float2* u2 = U2s + c * kOctK2 * a.r2max;
    float2 acc[kOctK2];
#pragma unroll
    for (int t = 0; t < kOctK2; ++t) acc[t] = make_float2(0.f, 0.f);
    for (int b = 0; b < r2; ++b) {
      const float2 sv = S[b * a.r3max];
#pragma unroll
      for (int t = 0; t < kOctK2; ++t) acc[t] = cmadd(u2[t * a.r2max + b], sv, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < kOctK2; ++t) W[it * kOctK2 + t] = acc[t];
  }
  __syncthreads();
  // G_c[k1, k2_0 + t, kk] = sum_q W[c][q][t] U3_c[kk, q]: two kk per thread, all t
  float2* out = a.out + ((long long)k1l * a.H2 + k2_0) * 6 * a.H3;
  const int hk = (a.H3 + 1) / 2;                       // kk pairs per component
  for (int it = threadIdx.x; it < 6 * hk; it += blockDim.x) {
    const int c = it / hk, kp = it - c * hk;
    const int kk0 = 2 * kp, kk1 = min(2 * kp + 1, a.H3 - 1);
    const CompMeta<float>& m = meta[c];
    const float2* u3t = m.U3t;                         // U3_c[kk, q] at u3t[q * H3 + kk]
    const float4* w = reinterpret_cast<const float4*>(W + c * a.r3max * kOctK2);
    float2 acc0[kOctK2], acc1[kOctK2];
#pragma unroll
    for (int t = 0; t < kOctK2; ++t) acc0[t] = acc1[t] = make_float2(0.f, 0.f);
    for (int q = 0; q < m.r3; ++q) {
      const float2 u0 = u3t[(long long)q * a.H3 + kk0];
      const float2 u1 = u3t[(long long)q * a.H3 + kk1];
#pragma unroll
      for (int t2 = 0; t2 < kOctK2 / 2; ++t2) {
        const float4 wv = w[q * (kOctK2 / 2) + t2];     // W[c][q][2 t2], W[c][q][2 t2 + 1]
        const float2 wa = make_float2(wv.x, wv.y), wb = make_float2(wv.z, wv.w);
        acc0[2 * t2] = cmadd(wa, u0, acc0[2 * t2]);
        acc1[2 * t2] = cmadd(wa, u1, acc1[2 * t2]);
        acc0[2 * t2 + 1] = cmadd(wb, u0, acc0[2 * t2 + 1]);
        acc1[2 * t2 + 1] = cmadd(wb, u1, acc1[2 * t2 + 1]);
      }
    }
#pragma unroll
    for (int t = 0; t < kOctK2; ++t) {
      if (t < nk2) {
        float2* o = out + ((long long)t * 6 + c) * a.H3;
        o[kk0] = acc0[t];
        if (kk1 != kk0) o[kk1] = acc1[t];
      }
    }
  }
}

// The same rebuild on the tensor cores (warp-level mma.sync m16n8k8, TF32
// operands, FP32 accumulation).  A complex product C = A B is one real GEMM
// C' = A' B': A' is A read as interleaved (re, im) floats (M x 2K), B' puts the
// 2x2 block [[Re b, Im b], [-Im b, Re b]] in place of every entry b of B
// (2K x 2N), and C' is C as interleaved floats.  Each operand is split into a
// TF32 value and a TF32 remainder and the product is accumulated as
// lo*hi + hi*lo + hi*hi (3xTF32), which keeps the rebuilt values at FP32
// accuracy (one TF32 product alone is ~3e-4 relative).
//
// One warp per (component c, k1, 16 consecutive k2), two GEMMs back to back:
//   W'  = U2_c'[k2 rows] S_c[k1]'          (M = 16, K = 2 r2, N = 2 r3)
//   G'  = W' (U3_c^T)'                     (M = 16, K = 2 r3, N = 2 H3)
// The accumulators of the first are the A fragments of the second, without a
// shuffle or a trip through shared memory: inside every block of 8 the second
// GEMM's K index is permuted (slot s < 4 is column 2s of the block, slot s >= 4
// column 2(s-4)+1), which is exactly where a lane holds W' in its accumulator.
// (U3_c^T)' is stored with the same permutation in fragment order, split at
// setup (u3frag_kernel): one 16-byte shared load per lane per (k-step, n-tile)
// gives the TF32 value and remainder of both B elements.
//
// The last k2 tile holds H2 mod 16 rows (one, the Nyquist row, when P2 is a
// multiple of 32); up to kTcSimtRows such rows are rebuilt with FP32 FMAs by
// one warp instead of a mostly empty mma tile.
//
// One CTA per SM: a CTA takes an equal, contiguous range of (k1, k2-tile)
// units of one component (and one range of n-tiles), so the slab cores it
// needs are a few consecutive k1; it stages them, the U2 rows and the U3
// fragments with cp.async in one round trip, then each warp runs its units
// from shared memory.
constexpr int kTcThreads = 512;
constexpr int kTcSimtRows = 4;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcMaxKs = 8;                           // r3 <= 32
constexpr size_t kTcFragMax = 72u << 10;              // U3 fragments per CTA

struct OctTcArgs {
  OctArgs o;
  const uint4* frag;  // [6][nsplit][KS][ntc][32]
  int nk1;            // k1 values in the chunk
  int mt;             // 16-row tiles of k2: ceil(H2 / 16)
  int nt2;            // 8-column tiles of G': ceil(H3 / 4)
  int nsplit;         // CTAs of a component split the n-tiles into nsplit ranges
  int ntc;            // n-tiles per range (even)
  int per;            // units per CTA
  int kspan;          // k1 rows of slab cores a CTA stages
  int la;             // row stride (floats) of the staged U2 rows
  int ks1m;           // k-steps of GEMM 1 for r2max: ceil(r2max / 4)
};

__host__ __device__ constexpr int tc_ks(int r) { return (r + 3) / 4; }

// n-tile ranges per component and n-tiles per range for KS k-steps
inline void tc_split(int KS, int nt2, int* nsplit, int* ntc) {
  for (int s = 1;; ++s) {
    int c = (nt2 + s - 1) / s;
    c += c & 1;
    if ((size_t)KS * c * 32 * sizeof(uint4) <= kTcFragMax || c <= 2) {
      *nsplit = s;
      *ntc = c;
      return;
    }
  }
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi, lo TF32 (lo carries the bits hi dropped)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(x);
  lo = tf32_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// (U3_c^T)' fragments: k-step j, slot t is Re W[q], slot t + 4 is Im W[q]
// (q = 4 j + t); column 8 nt + g is Re (even) or Im (odd) of G[., n],
// n = 4 nt + g / 2; entries past r3 or H3 are zero.  uint4 = (hi b0, hi b1,
// lo b0, lo b1).
__global__ void u3frag_kernel(const CompMeta<float>* meta, int KS, int nsplit, int ntc, int H3,
                              uint4* out) {
  const long long blk = (long long)KS * ntc * 32, per = nsplit * blk;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * per) return;
  const int c = (int)(i / per);
  long long r = i - c * per;
  const int sp = (int)(r / blk);
  r -= sp * blk;
  const int ln = (int)(r & 31), jt = (int)(r >> 5);
  const int j = jt / ntc, ntl = jt - j * ntc;
  const CompMeta<float> m = meta[c];
  const int q = 4 * j + (ln & 3);
  const int col = 8 * (sp * ntc + ntl) + (ln >> 2), n = col >> 1;
  float2 u = make_float2(0.f, 0.f);
  if (q < m.r3 && n < H3) u = m.U3t[(long long)q * H3 + n];
  const float b0 = (col & 1) ? u.y : u.x;            // row Re W[q]: (U3r, U3i)
  const float b1 = (col & 1) ? u.x : -u.y;           // row Im W[q]: (-U3i, U3r)
  uint4 v;
  tf32_split(b0, v.x, v.z);
  tf32_split(b1, v.y, v.w);
  out[i] = v;
}

// GEMM 2 of one unit and its store: the 16 rows of G' for this CTA's n-tiles,
// two n-tiles at a time, the hi*hi products and the two correction products
// in separate accumulators (four independent chains).  C' columns 8 nt + 2 t
// and + 1 are (Re, Im) of G[k2][4 nt + t].
template <int KS>
__device__ __forceinline__ void tc_gemm2_store(const uint32_t (&a2h)[KS][4], const uint32_t (&a2l)[KS][4],
                                               const uint4* B2, int ntc, int nt_lo, int nt_n, int lane,
                                               float2* o0, float2* o1, bool in0, bool in1, int H3) {
  const int t = lane & 3;
  for (int ntl = 0; ntl < nt_n; ntl += 2) {
    float hh0[4] = {0.f, 0.f, 0.f, 0.f}, cr0[4] = {0.f, 0.f, 0.f, 0.f};
    float hh1[4] = {0.f, 0.f, 0.f, 0.f}, cr1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < KS; ++j) {
      const uint4 p = B2[(j * ntc + ntl) * 32 + lane];
      const uint4 r = B2[(j * ntc + ntl + 1) * 32 + lane];
      mma_tf32(cr0, a2l[j], p.x, p.y);
      mma_tf32(cr1, a2l[j], r.x, r.y);
      mma_tf32(cr0, a2h[j], p.z, p.w);
      mma_tf32(cr1, a2h[j], r.z, r.w);
      mma_tf32(hh0, a2h[j], p.x, p.y);
      mma_tf32(hh1, a2h[j], r.x, r.y);
    }
    const int n0 = 4 * (nt_lo + ntl) + t, n1 = n0 + 4;
    if (in0) {
      if (n0 < H3) o0[n0] = make_float2(hh0[0] + cr0[0], hh0[1] + cr0[1]);
      if (n1 < H3) o0[n1] = make_float2(hh1[0] + cr1[0], hh1[1] + cr1[1]);
    }
    if (in1) {
      if (n0 < H3) o1[n0] = make_float2(hh0[2] + cr0[2], hh0[3] + cr0[3]);
      if (n1 < H3) o1[n1] = make_float2(hh1[2] + cr1[2], hh1[3] + cr1[3]);
    }
  }
}

// One row of a partial k2 tile with FP32 FMAs: lane q holds w[q] (q < rq),
// G[n] = sum_q w[q] F[n, q] for n in [nb, ne), F staged as [q][n - nb].
__device__ __forceinline__ void fma_row(float2 w, int rq, const float2* Fs, int ncols, int nb, int ne,
                                        float2* orow, int lane) {
  for (int n0 = nb; n0 < ne; n0 += 32) {
    const int n = n0 + lane;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < rq; ++q) {
      const float2 wq = make_float2(__shfl_sync(0xffffffffu, w.x, q), __shfl_sync(0xffffffffu, w.y, q));
      if (n < ne) acc = cmadd(wq, Fs[q * ncols + (n - nb)], acc);
    }
    if (n < ne) orow[n] = acc;
  }
}

template <int KS>
__global__ void __launch_bounds__(kTcThreads, 1) octant_tc_kernel(const OctTcArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x / a.nsplit, sp = blockIdx.x - c * a.nsplit;
  const CompMeta<float> m = a.o.meta[c];
  const int H2 = a.o.H2, H3 = a.o.H3, r2 = m.r2, r3 = m.r3, r2m = a.o.r2max, r3m = a.o.r3max;
  const int units = a.nk1 * a.mt;
  const int u0 = blockIdx.y * a.per, u1 = min(units, u0 + a.per);
  if (u0 >= u1) return;
  const int k1lo = u0 / a.mt, kspan = (u1 - 1) / a.mt - k1lo + 1;
  const int LA = a.la, rows = a.mt * 16, ks1m = a.ks1m, ncols = 4 * a.ntc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int nt_lo = sp * a.ntc, nt_n = min(a.ntc, a.nt2 - nt_lo);
  uint4* B2 = reinterpret_cast<uint4*>(smem_raw);                // [KS][ntc][32]
  uint4* B1 = B2 + KS * a.ntc * 32;                               // [kspan][ks1m][KS][32]
  float* U2s = reinterpret_cast<float*>(B1 + a.kspan * ks1m * KS * 32);   // [mt 16][LA]
  float2* Ss = reinterpret_cast<float2*>(U2s + rows * LA);       // [kspan][r2max][r3max]
  float2* U3s = Ss + a.kspan * r2m * r3m;                        // [r3max][4 ntc]: U3[n0 + i, q]
  {
    const uint4* fr = a.frag + ((long long)c * a.nsplit + sp) * KS * a.ntc * 32;
    for (int i = threadIdx.x; i < KS * a.ntc * 32; i += kTcThreads) cp_async16(B2 + i, fr + i);
    const float2* U2 = m.U2;                                      // [H2][r2]
    const int half = LA / 2;                                      // float2 per staged row
    for (int i = threadIdx.x; i < rows * half; i += kTcThreads) {
      const int k2 = i / half, b = i - k2 * half;
      float2* d = reinterpret_cast<float2*>(U2s + k2 * LA) + b;
      if (k2 < H2 && b < r2) cp_async8(d, U2 + (long long)k2 * r2 + b);
      else *d = make_float2(0.f, 0.f);
    }
    const float2* S = m.slab + (long long)(a.o.k1a + k1lo) * r2m * r3m;
    for (int i = threadIdx.x; i < kspan * r2m * r3m; i += kTcThreads) cp_async8(Ss + i, S + i);
    for (int i = threadIdx.x; i < r3m * ncols; i += kTcThreads) {
      const int q = i / ncols, n = 4 * nt_lo + (i - q * ncols);
      if (q < r3 && n < H3) cp_async8(U3s + i, m.U3t + (long long)q * H3 + n);
      else U3s[i] = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  // S' fragments of GEMM 1 for every staged k1: rows kc0 = 8 k + t and
  // kc1 = kc0 + 4 (b = kc >> 1, parity e = t & 1), column 8 nt + g (q =
  // 4 nt + g / 2, parity f = g & 1): (e, f) = (0,0) Re s, (0,1) Im s,
  // (1,0) -Im s, (1,1) Re s.  uint4 = (hi v0, hi v1, lo v0, lo v1).
  for (int i = threadIdx.x; i < kspan * ks1m * KS * 32; i += kTcThreads) {
    const int ln = i & 31, r = i >> 5;
    const int nt = r % KS, k = (r / KS) % ks1m, kk = r / (KS * ks1m);
    const int tt = ln & 3, gg = ln >> 2;
    const int b0 = (8 * k + tt) >> 1, b1 = b0 + 2, e = tt & 1, f = gg & 1;
    const int q = 4 * nt + (gg >> 1);
    const float2* Sk = Ss + kk * r2m * r3m;
    float2 s0 = make_float2(0.f, 0.f), s1 = s0;
    if (q < r3) {
      if (b0 < r2) s0 = Sk[b0 * r3m + q];
      if (b1 < r2) s1 = Sk[b1 * r3m + q];
    }
    const float v0 = e == f ? s0.x : (e ? -s0.y : s0.y);
    const float v1 = e == f ? s1.x : (e ? -s1.y : s1.y);
    uint4 v;
    tf32_split(v0, v.x, v.z);
    tf32_split(v1, v.y, v.w);
    B1[i] = v;
  }
  __syncthreads();
  const int ks1 = (2 * r2 + 7) / 8;
  const int rem = H2 - 16 * (H2 / 16);                 // rows of the last, partial tile
  for (int u = u0 + warp; u < u1; u += kTcWarps) {
    const int k1l = u / a.mt, mt = u - k1l * a.mt;
    if (rem > 0 && rem <= kTcSimtRows && mt == a.mt - 1) {
      // W[q] = sum_b U2[k2, b] S[b, q] with q = lane, then G[k2, n] =
      // sum_q W[q] U3[n, q] for this CTA's n range, W broadcast by shuffles
      const float2* S = Ss + (k1l - k1lo) * r2m * r3m;
      const int nb = 4 * nt_lo, ne = min(H3, 4 * (nt_lo + nt_n));
      for (int k2 = 16 * mt; k2 < H2; ++k2) {
        const float2* u2 = reinterpret_cast<const float2*>(U2s + k2 * LA);
        float2 w = make_float2(0.f, 0.f);
        if (lane < r3)
          for (int b = 0; b < r2; ++b) w = cmadd(u2[b], S[b * r3m + lane], w);
        fma_row(w, r3, U3s, ncols, nb, ne, a.o.out + (((long long)k1l * H2 + k2) * 6 + c) * H3, lane);
      }
      continue;
    }
    const uint4* B1k = B1 + (k1l - k1lo) * ks1m * KS * 32 + lane;
    const int row0 = mt * 16 + g, row1 = row0 + 8;
    const float* A0 = U2s + row0 * LA;
    const float* A1 = A0 + 8 * LA;
    // GEMM 1: W' = U2' S', K index kc = 2 b + e (e: Re/Im of U2[k2, b])
    float acc1[KS][4];
#pragma unroll
    for (int nt = 0; nt < KS; ++nt) acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.f;
    for (int k = 0; k < ks1; ++k) {
      const int kc0 = 8 * k + t, kc1 = kc0 + 4;
      uint32_t ah[4], al[4];
      tf32_split(A0[kc0], ah[0], al[0]);
      tf32_split(A1[kc0], ah[1], al[1]);
      tf32_split(A0[kc1], ah[2], al[2]);
      tf32_split(A1[kc1], ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < KS; ++nt) {
        const uint4 bv = B1k[(k * KS + nt) * 32];
        mma_tf32(acc1[nt], al, bv.x, bv.y);
        mma_tf32(acc1[nt], ah, bv.z, bv.w);
        mma_tf32(acc1[nt], ah, bv.x, bv.y);
      }
    }
    // GEMM 2's A fragments: slot t <- W'[., 8 j + 2 t] (c0, c2), slot t + 4 <-
    // W'[., 8 j + 2 t + 1] (c1, c3)
    uint32_t a2h[KS][4], a2l[KS][4];
#pragma unroll
    for (int j = 0; j < KS; ++j) {
      tf32_split(acc1[j][0], a2h[j][0], a2l[j][0]);
      tf32_split(acc1[j][2], a2h[j][1], a2l[j][1]);
      tf32_split(acc1[j][1], a2h[j][2], a2l[j][2]);
      tf32_split(acc1[j][3], a2h[j][3], a2l[j][3]);
    }
    float2* o0 = a.o.out + (((long long)k1l * H2 + row0) * 6 + c) * H3;
    tc_gemm2_store<KS>(a2h, a2l, B2, a.ntc, nt_lo, nt_n, lane, o0, o0 + 8ll * 6 * H3, row0 < H2,
                       row1 < H2, H3);
  }
}

// Tucker+CP rebuild, eq. (17): G_c[k1, k2, k3] = sum_l W1[k1, l] W2[k2, l] W3[k3, l]
// for the half fibres of a chunk of k1.  The same units and second GEMM as
// octant_tc_kernel; the first GEMM becomes a Hadamard product: the A
// fragments of a unit are A[k2][l] = W1[k1, l] W2[k2, l] (slot t of k-step j
// is Re A[., 4 j + t], slot t + 4 its Im), and B is W3's real form in the same
// fragment order (u3frag_kernel applied to W3).
struct CpMeta {
  const float2* W1;    // [H1][R]
  const float2* W2;    // [H2][R]
  const float2* W3t;   // [R][H3]
};

struct OctCpArgs {
  const CpMeta* meta;
  const uint4* frag;   // [6][nsplit][KS][ntc][32]
  float2* out;         // [chunk][H2][6][H3]
  int R, H2, H3, k1a, nk1, mt, nt2, nsplit, ntc, per, kspan;
};

template <int KS>
__global__ void __launch_bounds__(kTcThreads, 1) octant_cp_kernel(const OctCpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x / a.nsplit, sp = blockIdx.x - c * a.nsplit;
  const CpMeta m = a.meta[c];
  const int H2 = a.H2, H3 = a.H3, R = a.R;
  const int units = a.nk1 * a.mt;
  const int u0 = blockIdx.y * a.per, u1 = min(units, u0 + a.per);
  if (u0 >= u1) return;
  const int k1lo = u0 / a.mt, kspan = (u1 - 1) / a.mt - k1lo + 1;
  const int rows = a.mt * 16, ncols = 4 * a.ntc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int nt_lo = sp * a.ntc, nt_n = min(a.ntc, a.nt2 - nt_lo);
  uint4* B2 = reinterpret_cast<uint4*>(smem_raw);                 // [KS][ntc][32]
  float2* W2s = reinterpret_cast<float2*>(B2 + KS * a.ntc * 32);  // [mt 16][R]
  float2* W1s = W2s + rows * R;                                   // [kspan][R]
  float2* W3s = W1s + a.kspan * R;                                // [R][4 ntc]: W3[n0 + i, l]
  {
    const uint4* fr = a.frag + ((long long)c * a.nsplit + sp) * KS * a.ntc * 32;
    for (int i = threadIdx.x; i < KS * a.ntc * 32; i += kTcThreads) cp_async16(B2 + i, fr + i);
    for (int i = threadIdx.x; i < rows * R; i += kTcThreads) {
      if (i < H2 * R) cp_async8(W2s + i, m.W2 + i);
      else W2s[i] = make_float2(0.f, 0.f);
    }
    const float2* w1 = m.W1 + (long long)(a.k1a + k1lo) * R;
    for (int i = threadIdx.x; i < kspan * R; i += kTcThreads) cp_async8(W1s + i, w1 + i);
    for (int i = threadIdx.x; i < R * ncols; i += kTcThreads) {
      const int l = i / ncols, n = 4 * nt_lo + (i - l * ncols);
      if (n < H3) cp_async8(W3s + i, m.W3t + (long long)l * H3 + n);
      else W3s[i] = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const int rem = H2 - 16 * (H2 / 16);
  for (int u = u0 + warp; u < u1; u += kTcWarps) {
    const int k1l = u / a.mt, mt = u - k1l * a.mt;
    const float2* w1 = W1s + (k1l - k1lo) * R;
    if (rem > 0 && rem <= kTcSimtRows && mt == a.mt - 1) {
      const int nb = 4 * nt_lo, ne = min(H3, 4 * (nt_lo + nt_n));
      for (int k2 = 16 * mt; k2 < H2; ++k2) {
        const float2 w = lane < R ? w1[lane] * W2s[k2 * R + lane] : make_float2(0.f, 0.f);
        fma_row(w, R, W3s, ncols, nb, ne, a.out + (((long long)k1l * H2 + k2) * 6 + c) * H3, lane);
      }
      continue;
    }
    const int row0 = mt * 16 + g, row1 = row0 + 8;
    uint32_t a2h[KS][4], a2l[KS][4];
#pragma unroll
    for (int j = 0; j < KS; ++j) {
      const int l = 4 * j + t;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (l < R) {
        v0 = w1[l] * W2s[row0 * R + l];
        v1 = w1[l] * W2s[row1 * R + l];
      }
      tf32_split(v0.x, a2h[j][0], a2l[j][0]);
      tf32_split(v1.x, a2h[j][1], a2l[j][1]);
      tf32_split(v0.y, a2h[j][2], a2l[j][2]);
      tf32_split(v1.y, a2h[j][3], a2l[j][3]);
    }
    float2* o0 = a.out + (((long long)k1l * H2 + row0) * 6 + c) * H3;
    tc_gemm2_store<KS>(a2h, a2l, B2, a.ntc, nt_lo, nt_n, lane, o0, o0 + 8ll * 6 * H3, row0 < H2,
                       row1 < H2, H3);
  }
}

int launch_octant_args(const vie_op* op, int k1a, cudaStream_t s, bool cp);

// Four-step variant (fused_fs_group) for P3 = 8 V, V = 4 R with R even.
__host__ __device__ constexpr int fused_fs_min_blocks(int V) { return V <= 8 ? 8 : (V <= 16 ? 5 : 4); }

template <int V, bool STORED>
__global__ void __launch_bounds__(96, fused_fs_min_blocks(V)) fused_fs_kernel(const FusedArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fused_fs_group<V, STORED>(a, a.g0 + blockIdx.x, reinterpret_cast<float2*>(smem_raw));
}

template <int R, bool STORED>
static void launch_fused_warp_r(FusedArgs<float> a, cudaStream_t s) {
  const size_t smem = fused_warp_smem(R, a.H3, a.r2max, a.r3max);
  const int fam = STORED ? PF_FUSED_STORED : PF_FUSED_TUCKER;
  a.prof = prof_bytes(fam);
  a.prof_rhs_bytes = 12ull * a.comp_stride * sizeof(float2);     // 48 B per padded voxel
  a.prof_launch_bytes = STORED ? 6ull * a.spec_stride * sizeof(float2) : 0ull;
  // the four-step kernel when R is even (and, on the Tucker path, the half
  // fibres come from the rebuild scratch)
  constexpr bool kFs = (R == 2 || R == 4 || R == 6);
  const bool fs = kFs && (STORED || a.octant != nullptr);
  const size_t fs_smem = fused_fs_smem(4 * R, a.H3);
  // P3 = 512: the three-pass radix-8 kernel (tp512.cu); P3 = 128: radix 8, 4, 4 (t128.cu)
  const bool tp = (R == 16) && fused_tp_supported(a, STORED);
  const bool t128 = (R == 4) && fused_t128_supported(a, STORED);
  if (STORED || a.octant == nullptr) {
    ProfScope ps(fam, s);
    a.g0 = 0;
    if (tp) {
      launch_fused_tp(a, a.H1 * a.H2, STORED, s);
      return;
    }
    if (t128) {
      launch_fused_t128(a, a.H1 * a.H2, STORED, s);
      return;
    }
    if constexpr (kFs) {
      if (fs) {
        launch_pdl(fused_fs_kernel<4 * R, STORED>, dim3(a.H1 * a.H2), dim3(96), fs_smem, s, a);
        return;
      }
    }
    launch_pdl(fused_warp_kernel<R, STORED>, dim3(a.H1 * a.H2), dim3(128), smem, s, a);
    return;
  }
  // Tucker path: per chunk of k1, rebuild the half fibres (chunk 0 may already be
  // rebuilt, see matvec_run), then the groups of the chunk
  const int chunk = a.oct_chunk;
  for (int k1a = 0; k1a < a.H1; k1a += chunk) {
    const int nk1 = std::min(chunk, a.H1 - k1a);
    if (k1a > 0 || !a.oct_first_ready) launch_octant_args(a.op, k1a, s, a.oct_cp);
    a.oct_k1a = k1a;
    a.g0 = k1a * a.H2;
    ProfScope ps(fam, s);
    bool done = false;
    if (tp) {
      launch_fused_tp(a, nk1 * a.H2, STORED, s);
      done = true;
    }
    if (t128) {
      launch_fused_t128(a, nk1 * a.H2, STORED, s);
      done = true;
    }
    if constexpr (kFs) {
      if (fs && !done) {
        launch_pdl(fused_fs_kernel<4 * R, STORED>, dim3(nk1 * a.H2), dim3(96), fs_smem, s, a);
        done = true;
      }
    }
    if (!done) launch_pdl(fused_warp_kernel<R, STORED>, dim3(nk1 * a.H2), dim3(128), smem, s, a);
  }
}

template <bool STORED>
static bool launch_fused_warp(const FusedArgs<float>& a, cudaStream_t s) {
  if (a.P3 % 32 != 0) return false;
  switch (a.P3 / 32) {
    case 1: launch_fused_warp_r<1, STORED>(a, s); return true;
    case 2: launch_fused_warp_r<2, STORED>(a, s); return true;
    case 3: launch_fused_warp_r<3, STORED>(a, s); return true;
    case 4: launch_fused_warp_r<4, STORED>(a, s); return true;
    case 5: launch_fused_warp_r<5, STORED>(a, s); return true;
    case 6: launch_fused_warp_r<6, STORED>(a, s); return true;
    case 8: launch_fused_warp_r<8, STORED>(a, s); return true;
    case 10: launch_fused_warp_r<10, STORED>(a, s); return true;
    case 12: launch_fused_warp_r<12, STORED>(a, s); return true;
    case 16: launch_fused_warp_r<16, STORED>(a, s); return true;
    default: return false;
  }
}

template <typename T>
static size_t fused_smem(const FusedArgs<T>& a, int LR) {
  return (size_t)(a.P3 + 6 * a.H3 + 6 * a.r3max + 2 * LR * 3 * a.ld) * sizeof(cx<T>);
}

template <typename T, bool STORED>
static int launch_fused_impl(FusedArgs<T> a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (launch_fused_warp<STORED>(a, s)) return VIE_OK;
  }
  const size_t limit = 227 * 1024;
  int LR = 4;
  while (LR > 1 && fused_smem(a, LR) > limit) LR /= 2;
  if (fused_smem(a, LR) > limit) {
    set_error("fused kernel: line length %d needs more shared memory than available", a.P3);
    return VIE_ERR_ARG;
  }
  a.lines_per_round = LR;
  const int fam = sizeof(T) == 8 ? PF_MATVEC64 : (STORED ? PF_FUSED_STORED : PF_FUSED_TUCKER);
  a.prof = sizeof(T) == 8 ? nullptr : prof_bytes(fam);
  a.prof_rhs_bytes = 12ull * a.comp_stride * sizeof(cx<T>);      // 48 B per padded voxel
  a.prof_launch_bytes = STORED ? 6ull * a.spec_stride * sizeof(cx<T>) : 0ull;
  ProfScope ps(fam, s);
  fused_z_kernel<T, STORED><<<a.H1 * a.H2, 256, fused_smem(a, LR), s>>>(a);
  return VIE_OK;
}

}  // namespace vie

// ---------------------------------------------------------------------------
// host launchers used by matvec.cu
// ---------------------------------------------------------------------------
template <typename T>
vie::SlabArgs<T> make_slab_args(const vie_op* op) {
  vie::SlabArgs<T> a;
  for (int c = 0; c < 6; ++c) {
    const TuckerComp& tc = op->comp[c];
    if constexpr (sizeof(T) == 4) {
      a.core[c] = tc.core32;
      a.U1[c] = tc.U32[0];
    } else {
      a.core[c] = tc.core64;
      a.U1[c] = tc.U64[0];
    }
    a.r1[c] = tc.r[0];
    a.r2[c] = tc.r[1];
    a.r3[c] = tc.r[2];
  }
  if constexpr (sizeof(T) == 4) a.slab = op->slab32; else a.slab = op->slab64;
  a.slab_stride = (long long)op->slab_stride;
  a.r2max = op->rmax[1];
  a.r3max = op->rmax[2];
  a.prof = prof_bytes(PF_REBUILD);
  a.prof_launch_bytes = 6ull * op->slab_stride * sizeof(cx<T>);
  return a;
}

template <typename T>
int launch_slab_cores(const vie_op* op, cudaStream_t s) {
  vie::SlabArgs<T> a = make_slab_args<T>(op);
  dim3 grid(op->H[0], 6);
  ProfScope ps(PF_REBUILD, s);
  vie::slab_core_kernel<T><<<grid, 256, 0, s>>>(a);
  return VIE_OK;
}

template <typename T>
vie::FusedArgs<T> make_fused_args(const vie_op* op, cx<T>* data, int B, bool stored,
                                  const int* active) {
  vie::FusedArgs<T> a = {};
  a.data = data;
  if constexpr (sizeof(T) == 4) {
    a.roots = op->roots32[2];
    a.spec = op->spec32;
    a.meta = reinterpret_cast<const CompMeta<T>*>(op->meta);
  } else {
    a.roots = op->roots64[2];
    a.spec = op->spec64;
    a.meta = reinterpret_cast<const CompMeta<T>*>(static_cast<char*>(op->meta) +
                                                  6 * sizeof(CompMeta<float>));
  }
  a.plan = op->plan[2];
  a.n3 = op->n[2];
  a.P1 = op->P[0];
  a.P2 = op->P[1];
  a.P3 = op->P[2];
  a.H1 = op->H[0];
  a.H2 = op->H[1];
  a.H3 = op->H[2];
  a.B = B;
  a.comp_stride = (long long)op->P[0] * op->P[1] * op->n[2];
  a.r2max = op->rmax[1];
  a.r3max = op->rmax[2];
  a.spec_stride = (long long)op->P[0] * op->P[1] * op->P[2];
  a.active = active;
  a.ld = op->P[2];
  a.lines_per_round = 4;
  const int fam = stored ? PF_FUSED_STORED : PF_FUSED_TUCKER;
  a.prof = prof_bytes(fam);
  // algorithmic bytes of the voxel-wise product (read J^, write Y^): 48 B per
  // padded voxel and right-hand side; the fused kernel itself moves half of
  // that (n3 of P3 z-points in and out), the zero padding never leaving chip
  a.prof_rhs_bytes = 12ull * a.comp_stride * sizeof(cx<T>);
  a.prof_launch_bytes = stored ? 6ull * a.spec_stride * sizeof(cx<T>) : 0ull;
  (void)stored;
  return a;
}

int launch_octant(const vie_op* op, int k1a, cudaStream_t s, bool cp) {
  return vie::launch_octant_args(op, k1a, s, cp);
}

bool octant_uses_tc(const vie_op* op) { return op->u3frag != nullptr; }

bool tc_rebuild_eligible(const vie_op* op) {
  return op->oct32 != nullptr && !(op->flags & VIE_REBUILD_SIMT) &&
         vie::tc_ks(op->rmax[2]) <= vie::kTcMaxKs;
}

namespace vie {
template <int KS>
static void launch_tc(const OctTcArgs& t, int gy, size_t smem, cudaStream_t s) {
  octant_tc_kernel<KS><<<dim3(6 * t.nsplit, gy), kTcThreads, smem, s>>>(t);
}

constexpr size_t kTcSmemLimit = 227u << 10;

// launch shape of octant_tc_kernel for nk1 values of k1; returns its shared memory
static size_t tc_plan(const vie_op* op, const OctArgs& o, int nk1, OctTcArgs* t) {
  t->o = o;
  t->frag = op->u3frag;
  t->nk1 = nk1;
  t->mt = (o.H2 + 15) / 16;
  t->nt2 = (o.H3 + 3) / 4;
  t->nsplit = op->tc_nsplit;
  t->ntc = op->tc_ntc;
  t->la = 8 * tc_ks(o.r2max) + 4;                     // >= 2 r2max, 4 mod 8: no bank conflicts
  t->ks1m = tc_ks(o.r2max);
  // one CTA per SM with equal unit ranges; more, smaller ranges when the
  // staged slab cores would not fit
  const int units = nk1 * t->mt;
  int gy = std::max(1, std::min(units, device_sms() / (6 * t->nsplit)));
  for (;;) {
    t->per = (units + gy - 1) / gy;
    t->kspan = (t->per + t->mt - 1) / t->mt + 1;
    const size_t smem = (size_t)op->tc_ks * t->ntc * 32 * sizeof(uint4) +
                        (size_t)t->kspan * t->ks1m * op->tc_ks * 32 * sizeof(uint4) +
                        (size_t)t->mt * 16 * t->la * sizeof(float) +
                        (size_t)t->kspan * o.r2max * o.r3max * sizeof(float2) +
                        (size_t)o.r3max * 4 * t->ntc * sizeof(float2);
    if (smem <= kTcSmemLimit || t->per == 1) return smem;
    gy = std::min(units, 2 * gy);
  }
}

static OctArgs octant_args(const vie_op* op, int k1a) {
  OctArgs o;
  o.meta = reinterpret_cast<const CompMeta<float>*>(op->meta);
  o.r2max = op->rmax[1];
  o.r3max = op->rmax[2];
  o.H2 = op->H[1];
  o.H3 = op->H[2];
  o.k1a = k1a;
  o.out = op->oct32;
  return o;
}

template <int KS>
static void launch_cp(const OctCpArgs& t, int gy, size_t smem, cudaStream_t s) {
  octant_cp_kernel<KS><<<dim3(6 * t.nsplit, gy), kTcThreads, smem, s>>>(t);
}

// launch shape of octant_cp_kernel for nk1 values of k1; returns its shared memory
static size_t cp_plan(const vie_op* op, int k1a, int nk1, OctCpArgs* t) {
  t->meta = reinterpret_cast<const CpMeta*>(op->cp.meta);
  t->frag = op->cp.frag;
  t->out = op->oct32;
  t->R = op->cp.R;
  t->H2 = op->H[1];
  t->H3 = op->H[2];
  t->k1a = k1a;
  t->nk1 = nk1;
  t->mt = (t->H2 + 15) / 16;
  t->nt2 = (t->H3 + 3) / 4;
  t->nsplit = op->cp.nsplit;
  t->ntc = op->cp.ntc;
  const int units = nk1 * t->mt;
  int gy = std::max(1, std::min(units, device_sms() / (6 * t->nsplit)));
  for (;;) {
    t->per = (units + gy - 1) / gy;
    t->kspan = (t->per + t->mt - 1) / t->mt + 1;
    const size_t smem = (size_t)op->cp.ks * t->ntc * 32 * sizeof(uint4) +
                        ((size_t)t->mt * 16 + t->kspan + 4 * t->ntc) * t->R * sizeof(float2);
    if (smem <= kTcSmemLimit || t->per == 1) return smem;
    gy = std::min(units, 2 * gy);
  }
}

// the rebuild of chunk [k1a, k1a + oct_k1): from the Tucker+CP model (cp), or
// from the Tucker model on the tensor cores, through tcgen05 (op->umma) or
// warp-level mma.sync when the operator holds the U3 fragments (r3 <= 32, no
// VIE_REBUILD_SIMT), else with FMAs
int launch_octant_args(const vie_op* op, int k1a, cudaStream_t s, bool cp) {
  const OctArgs o = octant_args(op, k1a);
  const int nk1 = std::min(op->oct_k1, op->H[0] - k1a);
  ProfScope ps(PF_REBUILD, s);
  if (cp) {
    OctCpArgs t;
    const size_t smem = cp_plan(op, k1a, nk1, &t);
    const int gy = (nk1 * t.mt + t.per - 1) / t.per;
    switch (op->cp.ks) {
      case 1: launch_cp<1>(t, gy, smem, s); break;
      case 2: launch_cp<2>(t, gy, smem, s); break;
      case 3: launch_cp<3>(t, gy, smem, s); break;
      case 4: launch_cp<4>(t, gy, smem, s); break;
      case 5: launch_cp<5>(t, gy, smem, s); break;
      case 6: launch_cp<6>(t, gy, smem, s); break;
      case 7: launch_cp<7>(t, gy, smem, s); break;
      default: launch_cp<8>(t, gy, smem, s); break;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VIE_OK : cuda_status(e, "Tucker+CP rebuild launch");
  }
  if (op->umma) return launch_octant_umma(op, k1a, nk1, s);
  OctTcArgs t;
  const size_t smem = op->u3frag != nullptr ? tc_plan(op, o, nk1, &t) : 0;
  if (op->u3frag != nullptr && smem <= kTcSmemLimit) {
    const int KS = op->tc_ks;
    const int gy = (nk1 * t.mt + t.per - 1) / t.per;   // every CTA has a unit
    switch (KS) {
      case 1: launch_tc<1>(t, gy, smem, s); break;
      case 2: launch_tc<2>(t, gy, smem, s); break;
      case 3: launch_tc<3>(t, gy, smem, s); break;
      case 4: launch_tc<4>(t, gy, smem, s); break;
      case 5: launch_tc<5>(t, gy, smem, s); break;
      case 6: launch_tc<6>(t, gy, smem, s); break;
      case 7: launch_tc<7>(t, gy, smem, s); break;
      default: launch_tc<8>(t, gy, smem, s); break;
    }
  } else {
    const size_t osmem = octant_smem(o.r2max, o.r3max);
    octant_kernel<<<dim3((o.H2 + kOctK2 - 1) / kOctK2, nk1), 256, osmem, s>>>(o);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "rebuild launch");
}
}  // namespace vie

void tc_layout(int r3max, int H3, int* ks, int* nsplit, int* ntc) {
  *ks = vie::tc_ks(r3max);
  vie::tc_split(*ks, (H3 + 3) / 4, nsplit, ntc);
}

// the largest chunk's launch fits in shared memory (op->tc_* already set)
bool tc_rebuild_fits(const vie_op* op) {
  vie::OctTcArgs t;
  return vie::tc_plan(op, vie::octant_args(op, 0), op->oct_k1, &t) <= vie::kTcSmemLimit;
}

int launch_u3_fragments(const vie_op* op, cudaStream_t s) {
  const long long n = 6ll * op->tc_nsplit * op->tc_ks * op->tc_ntc * 32;
  vie::u3frag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const CompMeta<float>*>(op->meta), op->tc_ks, op->tc_nsplit, op->tc_ntc,
      op->H[2], op->u3frag);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "U3 fragment launch");
}

// Operands of the Tucker+CP rebuild once the factors W^q exist: W3's real form
// in fragment order (u3frag_kernel reads W3 through a CompMeta whose U3t and
// r3 are W3t and R) and the per-component pointer records.
int build_cp_rebuild(vie_op* op, cudaStream_t s) {
  const int R = op->cp.R;
  tc_layout(R, op->H[2], &op->cp.ks, &op->cp.nsplit, &op->cp.ntc);
  CompMeta<float> m[6] = {};
  vie::CpMeta cm[6];
  for (int c = 0; c < 6; ++c) {
    m[c].U3t = op->cp.W3t32[c];
    m[c].r3 = R;
    cm[c] = vie::CpMeta{op->cp.W32[c][0], op->cp.W32[c][1], op->cp.W3t32[c]};
  }
  const size_t nfrag = 6ull * op->cp.nsplit * op->cp.ks * op->cp.ntc * 32;
  CompMeta<float>* dm = nullptr;
  cudaError_t e = cudaMalloc(&op->cp.frag, nfrag * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMalloc(&op->cp.meta, sizeof(cm));
  if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(m));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dm);
    set_error("out of device memory for the Tucker+CP rebuild operands");
    return VIE_ERR_OOM;
  }
  e = cudaMemcpy(op->cp.meta, cm, sizeof(cm), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dm, m, sizeof(m), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    vie::u3frag_kernel<<<(unsigned)((nfrag + 255) / 256), 256, 0, s>>>(dm, op->cp.ks, op->cp.nsplit,
                                                                      op->cp.ntc, op->H[2], op->cp.frag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dm);
  if (e != cudaSuccess) return cuda_status(e, "Tucker+CP rebuild operands");
  vie::OctCpArgs t;
  if (vie::cp_plan(op, 0, op->oct_k1, &t) > vie::kTcSmemLimit) {
    set_error("the Tucker+CP rebuild of rank %d does not fit in shared memory", R);
    return VIE_ERR_ARG;
  }
  return VIE_OK;
}


template <typename T>
int launch_fused(const vie_op* op, cx<T>* data, int B, bool stored, const int* active,
                 cudaStream_t s, bool first_chunk_ready, bool cp) {
  vie::FusedArgs<T> a = make_fused_args<T>(op, data, B, stored, active);
  if constexpr (sizeof(T) == 4) {
    if (!stored && op->oct32 != nullptr) {
      a.octant = op->oct32;
      a.oct_chunk = op->oct_k1;
      a.op = op;
      a.oct_first_ready = first_chunk_ready;
      a.oct_cp = cp;
    }
  }
  if (stored) {
    if (a.spec == nullptr) {
      set_error("operator was built without VIE_STORE_UNCOMPRESSED");
      return VIE_ERR_ARG;
    }
    return vie::launch_fused_impl<T, true>(a, s);
  }
  return vie::launch_fused_impl<T, false>(a, s);
}

int fused_init_attributes() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaSuccess;
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_z_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_z_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_z_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_z_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<24, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::fused_fs_kernel<24, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_cp_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  // octant_kernel also holds the six metadata records in static shared memory
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "fused kernel attributes");
}

template vie::SlabArgs<float> make_slab_args<float>(const vie_op*);
template vie::FusedArgs<float> make_fused_args<float>(const vie_op*, float2*, int, bool, const int*);
template int launch_slab_cores<float>(const vie_op*, cudaStream_t);
template int launch_slab_cores<double>(const vie_op*, cudaStream_t);
template int launch_fused<float>(const vie_op*, float2*, int, bool, const int*, cudaStream_t, bool, bool);
template int launch_fused<double>(const vie_op*, double2*, int, bool, const int*, cudaStream_t, bool, bool);
