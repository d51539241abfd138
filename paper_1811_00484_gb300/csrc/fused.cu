// Fused z-axis FFT, Tucker rebuild, voxel-wise product and inverse z-FFT:
// the element-wise product of the matvec (Section V.B, Table II) done with
// the components decompressed on chip instead of into a buffer.
//
// The rebuild follows eq. (13) in two stages:
//   slab cores   S_c[k1] = core_c x1 U1_c[k1, :]            (r2 x r3)
//   one fibre    G_c[k1, k2, k3] = sum_g ( U2_c[k2, :] S_c[k1] )[g] U3_c[k3, g]
// The spectrum of every component is even or odd along each axis
// (G_c[P - k] = s G_c[k], s = -1 when the component is odd in that
// coordinate), and so are the HOSVD factors of its unfoldings.  One CTA
// therefore rebuilds the fibre of (k1, k2) once, for k3 <= P3/2, and uses it,
// with signs, for the up-to-four z-lines (k1 | P1-k1, k2 | P2-k2) of every
// right-hand side.  The stored (uncompressed) variant reads the six spectra
// from memory instead.
#include "warpfft.cuh"

namespace vie {

// sign of component c (xx, xy, xz, yy, yz, zz) under k_q -> P_q - k_q
__constant__ int kParity[6][3] = {
    {1, 1, 1}, {-1, -1, 1}, {-1, 1, -1}, {1, 1, 1}, {1, -1, -1}, {1, 1, 1}};

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

template <typename T>
__global__ void __launch_bounds__(256) slab_core_kernel(const SlabArgs<T> a) {
  if (a.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(a.prof, a.prof_launch_bytes);
  using C = cx<T>;
  const int k1 = blockIdx.x, c = blockIdx.y;
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
  int lines_per_round;         // z-lines (x3 components) held in shared memory at once
  int ld;                      // shared-memory line stride
  unsigned long long* prof;    // profiler byte counter (nullptr = off)
  unsigned long long prof_rhs_bytes, prof_launch_bytes;
};

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
            if (ix) s *= kParity[c][0];
            if (iy) s *= kParity[c][1];
            if (zm) s *= kParity[c][2];
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
// group, one warp per mirror z-line holding the three components of every
// right-hand side in registers.  Forward lane FFT, voxel-wise product in the
// bit-reversed lane layout, inverse lane FFT: no shared-memory round trips
// and no block barriers after the rebuild.
// Slot of z-frequency k in a row of the rebuilt half fibre: one padding slot
// every 8 entries, so the lanes' folded, bit-reversed frequencies (stride R)
// fall in different banks (at most 2-way for the radices used, 4-way at R=10).
__device__ __forceinline__ int ghalf_slot(int k) { return k + (k >> 3); }

template <int R, bool STORED>
__global__ void __launch_bounds__(128) fused_warp_kernel(const FusedArgs<float> a) {
  using C = float2;
  constexpr int P3 = 32 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int n3 = a.n3, H3 = a.H3;
  const int g = blockIdx.x;
  const int k1 = g / a.H2, k2 = g % a.H2;
  const int nx = (k1 == 0 || 2 * k1 == a.P1) ? 1 : 2;
  const int ny = (k2 == 0 || 2 * k2 == a.P2) ? 1 : 2;
  const int nl = nx * ny;
  if (a.prof != nullptr && blockIdx.x == 0 && tid == 0) {
    unsigned long long nb = 0;
    for (int b = 0; b < a.B; ++b) nb += (a.active == nullptr || a.active[b]) ? 1 : 0;
    atomicAdd(a.prof, nb * a.prof_rhs_bytes + a.prof_launch_bytes);
  }

  const int GS = ghalf_slot(H3 - 1) + 1;   // padded row length of the half fibre
  C* roots = reinterpret_cast<C*>(smem_raw);
  C* ghalf = roots + P3;               // [6][GS]
  C* wv = ghalf + 6 * GS;              // [6][r3max]
  for (int m = tid; m < P3; m += nth) roots[m] = a.roots[m];
  if (!STORED) {
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
      const CompMeta<float> m = a.meta[c];
      const C* u3 = m.U3 + (long long)kk * m.r3;
      const C* w = wv + c * a.r3max;
      C acc = make_float2(0.f, 0.f);
      for (int q = 0; q < m.r3; ++q) acc = cmadd(w[q], u3[q], acc);
      ghalf[c * GS + ghalf_slot(kk)] = acc;
    }
  }
  __syncthreads();
  if (warp >= nl) return;                  // no block barrier follows

  const int ix = warp / ny, iy = warp % ny;
  const int kx = ix ? a.P1 - k1 : k1, ky = iy ? a.P2 - k2 : k2;
  const int br = brev5(lane);
  LaneConsts<C, float, R> lc;
  lc.init(lane, roots, P3);
  const long long line_off = ((long long)kx * a.P2 + ky) * n3;
  for (int b = 0; b < a.B; ++b) {
    if (a.active != nullptr && a.active[b] == 0) continue;   // warp-uniform
    C v[3][R];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const C* src = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
#pragma unroll
      for (int j = 0; j < (R + 1) / 2; ++j) {
        const int p = lane + 32 * j;
        v[comp][j] = p < n3 ? src[p] : make_float2(0.f, 0.f);
      }
      warp_fft_fwd<C, float, R, true>(v[comp], lc, roots, P3);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int kk = q + R * br;                       // z-frequency held in register q
      C gc[6];
      if (STORED) {
        const long long off = ((long long)kx * a.P2 + ky) * P3 + kk;
#pragma unroll
        for (int c = 0; c < 6; ++c) gc[c] = a.spec[c * a.spec_stride + off];
      } else {
        const bool zm = 2 * kk > P3;
        const int fold = zm ? P3 - kk : kk;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          int s = 1;
          if (ix) s *= kParity[c][0];
          if (iy) s *= kParity[c][1];
          if (zm) s *= kParity[c][2];
          const C gv = ghalf[c * GS + ghalf_slot(fold)];
          gc[c] = (s > 0) ? gv : make_float2(-gv.x, -gv.y);
        }
      }
      const C jx = v[0][q], jy = v[1][q], jz = v[2][q];
      v[0][q] = gc[0] * jx + gc[1] * jy + gc[2] * jz;
      v[1][q] = gc[1] * jx + gc[3] * jy + gc[4] * jz;
      v[2][q] = gc[2] * jx + gc[4] * jy + gc[5] * jz;
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      warp_fft_inv<C, float, R, true>(v[comp], lane, lc, roots, P3);
      C* dst = a.data + (long long)(b * 3 + comp) * a.comp_stride + line_off;
#pragma unroll
      for (int j = 0; j < (R + 1) / 2; ++j) {
        const int p = lane + 32 * j;
        if (p < n3) dst[p] = v[comp][j];
      }
    }
  }
}

template <int R, bool STORED>
static void launch_fused_warp_r(FusedArgs<float> a, cudaStream_t s) {
  const int GS = (a.H3 - 1) + ((a.H3 - 1) >> 3) + 1;
  const size_t smem = (size_t)(32 * R + 6 * GS + 6 * a.r3max) * sizeof(float2);
  const int fam = STORED ? PF_FUSED_STORED : PF_FUSED_TUCKER;
  a.prof = prof_bytes(fam);
  a.prof_rhs_bytes = 6ull * a.comp_stride * sizeof(float2);
  a.prof_launch_bytes = STORED ? 6ull * a.spec_stride * sizeof(float2) : 0ull;
  ProfScope ps(fam, s);
  fused_warp_kernel<R, STORED><<<a.H1 * a.H2, 128, smem, s>>>(a);
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
int launch_slab_cores(const vie_op* op, cudaStream_t s) {
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
  a.prof = prof_bytes(PF_SLAB);
  a.prof_launch_bytes = 6ull * op->slab_stride * sizeof(cx<T>);
  dim3 grid(op->H[0], 6);
  ProfScope ps(PF_SLAB, s);
  vie::slab_core_kernel<T><<<grid, 256, 0, s>>>(a);
  return VIE_OK;
}

template <typename T>
int launch_fused(const vie_op* op, cx<T>* data, int B, bool stored, const int* active,
                 cudaStream_t s) {
  vie::FusedArgs<T> a;
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
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "fused kernel attributes");
}

template int launch_slab_cores<float>(const vie_op*, cudaStream_t);
template int launch_slab_cores<double>(const vie_op*, cudaStream_t);
template int launch_fused<float>(const vie_op*, float2*, int, bool, const int*, cudaStream_t);
template int launch_fused<double>(const vie_op*, double2*, int, bool, const int*, cudaStream_t);
