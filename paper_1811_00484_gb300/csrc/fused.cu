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
// of k1 are rebuilt by octant_kernel into an FP32 scratch (one k1 chunk at a
// time, so the scratch stays a small fraction of the uncompressed spectra),
// and one CTA per (k1, k2) mirror group copies its 6 x (P3/2 + 1) values to
// shared memory; the multi-grid and shared-memory variants rebuild the fibre
// in the CTA.  The stored (uncompressed) variant reads the six spectra from
// memory instead.
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
  a.prof_rhs_bytes = 6ull * a.comp_stride * sizeof(float2);
  a.prof_launch_bytes = STORED ? 6ull * a.spec_stride * sizeof(float2) : 0ull;
  // the four-step kernel when R is even (and, on the Tucker path, the half
  // fibres come from the rebuild scratch)
  constexpr bool kFs = (R == 2 || R == 4 || R == 6);
  const bool fs = kFs && (STORED || a.octant != nullptr);
  const size_t fs_smem = fused_fs_smem(4 * R, a.H3);
  if (STORED || a.octant == nullptr) {
    ProfScope ps(fam, s);
    a.g0 = 0;
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
  OctArgs o;
  o.meta = a.meta;
  o.r2max = a.r2max;
  o.r3max = a.r3max;
  o.H2 = a.H2;
  o.H3 = a.H3;
  o.out = const_cast<float2*>(a.octant);
  const size_t osmem = octant_smem(a.r2max, a.r3max);
  for (int k1a = 0; k1a < a.H1; k1a += chunk) {
    const int nk1 = std::min(chunk, a.H1 - k1a);
    o.k1a = k1a;
    if (k1a > 0 || !a.oct_first_ready) {
      ProfScope ps(PF_REBUILD, s);
      octant_kernel<<<dim3((a.H2 + kOctK2 - 1) / kOctK2, nk1), 256, osmem, s>>>(o);
    }
    a.oct_k1a = k1a;
    a.g0 = k1a * a.H2;
    ProfScope ps(fam, s);
    bool done = false;
    if constexpr (kFs) {
      if (fs) {
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
  const int fam = STORED ? PF_FUSED_STORED : PF_FUSED_TUCKER;
  a.prof = prof_bytes(fam);
  a.prof_rhs_bytes = 6ull * a.comp_stride * sizeof(cx<T>);       // 3 components read + written
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
  a.prof_rhs_bytes = 6ull * a.comp_stride * sizeof(cx<T>);
  a.prof_launch_bytes = stored ? 6ull * a.spec_stride * sizeof(cx<T>) : 0ull;
  (void)stored;
  return a;
}

int launch_octant(const vie_op* op, int k1a, cudaStream_t s) {
  vie::OctArgs o;
  o.meta = reinterpret_cast<const CompMeta<float>*>(op->meta);
  o.r2max = op->rmax[1];
  o.r3max = op->rmax[2];
  o.H2 = op->H[1];
  o.H3 = op->H[2];
  o.k1a = k1a;
  o.out = op->oct32;
  const int nk1 = std::min(op->oct_k1, op->H[0] - k1a);
  const size_t osmem = vie::octant_smem(o.r2max, o.r3max);
  ProfScope ps(PF_REBUILD, s);
  vie::octant_kernel<<<dim3((o.H2 + vie::kOctK2 - 1) / vie::kOctK2, nk1), 256, osmem, s>>>(o);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "rebuild launch");
}

template <typename T>
int launch_fused(const vie_op* op, cx<T>* data, int B, bool stored, const int* active,
                 cudaStream_t s, bool first_chunk_ready) {
  vie::FusedArgs<T> a = make_fused_args<T>(op, data, B, stored, active);
  if constexpr (sizeof(T) == 4) {
    if (!stored && op->oct32 != nullptr) {
      a.octant = op->oct32;
      a.oct_chunk = op->oct_k1;
      a.oct_first_ready = first_chunk_ready;
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
  // octant_kernel also holds the six metadata records in static shared memory
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::octant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 1024);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "fused kernel attributes");
}

template vie::SlabArgs<float> make_slab_args<float>(const vie_op*);
template vie::FusedArgs<float> make_fused_args<float>(const vie_op*, float2*, int, bool, const int*);
template int launch_slab_cores<float>(const vie_op*, cudaStream_t);
template int launch_slab_cores<double>(const vie_op*, cudaStream_t);
template int launch_fused<float>(const vie_op*, float2*, int, bool, const int*, cudaStream_t, bool);
template int launch_fused<double>(const vie_op*, double2*, int, bool, const int*, cudaStream_t, bool);
