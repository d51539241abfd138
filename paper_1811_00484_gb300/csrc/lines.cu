// Strided line FFTs: the x- and y-axis stages of the zero-padded forward
// FFT and of the cropped inverse FFT of the matvec (Section V.B), and the
// full 3-D FFT of the FP64 spectrum assembly (Section V.A).
//
// One CTA transforms TW lines that sit next to each other in memory (a tile
// of TW consecutive columns), so that every global load and store of a
// line position is a contiguous run of TW complex numbers.  Zero padding
// (points lin..N-1 read as zero), cropping (only points < lout stored),
// conjugation, the contrast product and the final scale/subtract of the
// system operator are fused into the load and store loops.
#include <cstdint>

#include "stages.cuh"

namespace vie {

template <typename T, int TW>
__global__ void __launch_bounds__(256, 3) line_fft_kernel(const LineArgs<T> a) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.plan.N;
  C* buf0 = reinterpret_cast<C*>(smem_raw);   // element (col c, pos p) at p*TW + c
  C* buf1 = buf0 + N * TW;
  C* roots = buf1 + N * TW;

  const int c0 = blockIdx.x * TW;
  const int o = blockIdx.y;
  const int bb = blockIdx.z;
  if (a.active != nullptr && a.active[bb / a.batch_per_rhs] == 0) return;   // block-uniform
  const int tid = threadIdx.x, nth = blockDim.x;
  if (a.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0)
    atomicAdd(a.prof, a.prof_batch_bytes);
  const int ncols = min(TW, a.ncol - c0);

  for (int m = tid; m < N; m += nth) roots[m] = a.roots[m];
  const T rs = (a.flags & (PRO_RSCALE | EPI_RSCALE))
                   ? (T)a.rscale[(long long)(bb / a.batch_per_rhs) * a.rscale_stride]
                   : (T)1;

  const C* in = a.in + bb * a.in_bs + o * a.in_os + (long long)c0 * a.in_cs;
  const bool col_fast_in = (a.in_cs == 1);
  for (int e = tid; e < N * TW; e += nth) {
    int p, c;
    if (col_fast_in) { c = e % TW; p = e / TW; } else { p = e % N; c = e / N; }
    C v = czero<C>();
    if (p < a.lin && c < ncols) {
      v = in[p * a.in_ls + c * a.in_cs];
      if (a.flags & PRO_RSCALE) v = rs * v;
      if (a.flags & PRO_CONJ) v = conjg(v);
      if (a.flags & PRO_CHI) v = a.chi[o * a.chi_os + p * a.chi_ls + (long long)(c0 + c) * a.chi_cs] * v;
    }
    buf0[p * TW + c] = v;
  }
  __syncthreads();

  C* res = fft_lines<T, true>(buf0, buf1, a.plan, TW, 1, TW, roots, a.inverse != 0, tid, nth);

  const long long obase = bb * a.out_bs + o * a.out_os + (long long)c0 * a.out_cs;
  C* out = a.out + obase;
  const bool col_fast_out = (a.out_cs == 1);
  for (int e = tid; e < a.lout * TW; e += nth) {
    int p, c;
    if (col_fast_out) { c = e % TW; p = e / TW; } else { p = e % a.lout; c = e / a.lout; }
    if (c >= ncols) continue;
    C v = a.scale * res[p * TW + c];
    if (a.flags & EPI_CONJ) v = conjg(v);
    const long long oi = p * a.out_ls + c * a.out_cs;
    if (a.flags & (EPI_SUB | EPI_ADD)) {
      if (a.flags & EPI_CHI) v = a.chi[o * a.chi_os + p * a.chi_ls + (long long)(c0 + c) * a.chi_cs] * v;
      C w = a.addend[obase + oi];
      if (a.flags & EPI_RSCALE) w = rs * w;
      v = (a.flags & EPI_SUB) ? (w - v) : (w + v);
    }
    out[oi] = v;
  }
}

// Register-resident variant for N = 32 R (columns contiguous in memory): one
// 16-column tile per CTA, see line_warp_tile.
// Resident CTAs per SM the register budget is sized for: up to radix 4 the
// kernel fits 40 registers without spills (six 256-thread CTAs per SM), up to
// radix 8 64 registers; larger radices get more registers than that.
__host__ __device__ constexpr int line_min_blocks(int R) { return R <= 4 ? 6 : (R <= 8 ? 4 : 2); }

template <int R, bool HALF>
__global__ void __launch_bounds__(256, line_min_blocks(R)) line_warp_kernel(const LineArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  line_warp_tile<R, HALF>(a, blockIdx.x * kLineTile, blockIdx.y, blockIdx.z,
                          reinterpret_cast<float2*>(smem_raw));
}

// Register-direct variant (no shared memory): one warp per kRegCols adjacent
// columns, see line_reg_group.  Used for radix <= 6.
__host__ __device__ constexpr int line_reg_min_blocks(int R) { return R <= 4 ? 8 : 5; }

template <int R, bool HALF>
__global__ void __launch_bounds__(128, line_reg_min_blocks(R)) line_reg_kernel(const LineArgs<float> a,
                                                                             int vec) {
  const int lane = threadIdx.x & 31;
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int ncg = (a.ncol + kRegCols - 1) / kRegCols;
  if (w >= (long long)ncg * a.nother * a.nbatch) return;        // warp-uniform; no barriers
  const int cg = (int)(w % ncg);
  const int o = (int)((w / ncg) % a.nother);
  const int bb = (int)(w / ((long long)ncg * a.nother));
  line_reg_group<R, HALF>(a, cg * kRegCols, o, bb, vec != 0, lane);
}

// Four-step variant (see line_fs_group) for N = 8 V with V = 4 R, R even.
__host__ __device__ constexpr int line_fs_min_blocks(int V) { return V <= 16 ? 8 : 4; }

template <int V, bool HALF>
__global__ void __launch_bounds__(128, line_fs_min_blocks(V)) line_fs_kernel(const LineArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* xs = reinterpret_cast<float2*>(smem_raw) + (size_t)warp * kRegCols * fs_col_stride(V);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const int ncg = (a.ncol + kRegCols - 1) / kRegCols;
  if (w >= (long long)ncg * a.nother * a.nbatch) return;        // warp-uniform; no barriers
  const int cg = (int)(w % ncg);
  const int o = (int)((w / ncg) % a.nother);
  const int bb = (int)(w / ((long long)ncg * a.nother));
  line_fs_group<V, HALF>(a, cg * kRegCols, o, bb, lane, xs);
}

template <int V>
static void launch_fs_v(LineArgs<float> a, cudaStream_t s) {
  const int ncg = (a.ncol + kRegCols - 1) / kRegCols;
  const long long warps = (long long)ncg * a.nother * a.nbatch;
  const int threads = a.threads > 0 && a.threads <= 128 ? a.threads : 128;
  const unsigned grid = (unsigned)((warps + threads / 32 - 1) / (threads / 32));
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  const bool half = a.inverse ? (2 * a.lout == a.plan.N) : (2 * a.lin == a.plan.N);
  launch_pdl(half ? line_fs_kernel<V, true> : line_fs_kernel<V, false>, dim3(grid), dim3(threads),
             line_fs_smem(V, threads / 32), s, a);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int R>
static void launch_reg_r(LineArgs<float> a, cudaStream_t s) {
  const int ncg = (a.ncol + kRegCols - 1) / kRegCols;
  const long long warps = (long long)ncg * a.nother * a.nbatch;
  const int threads = a.threads > 0 && a.threads <= 128 ? a.threads : 128;
  const unsigned grid = (unsigned)((warps + threads / 32 - 1) / (threads / 32));
  // 16-byte row accesses: every row start of every group is a multiple of 16 bytes
  const bool even = a.in_bs % 2 == 0 && a.in_os % 2 == 0 && a.in_ls % 2 == 0 &&
                    a.out_bs % 2 == 0 && a.out_os % 2 == 0 && a.out_ls % 2 == 0;
  const int vec = even && aligned16(a.in) && aligned16(a.out) ? 1 : 0;
  a.chi_vec = a.chi != nullptr && aligned16(a.chi) && a.chi_os % 2 == 0 && a.chi_ls % 2 == 0;
  a.addend_vec = a.addend != nullptr && aligned16(a.addend);
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  const bool half = a.inverse ? (2 * a.lout == a.plan.N) : (2 * a.lin == a.plan.N);
  launch_pdl(half ? line_reg_kernel<R, true> : line_reg_kernel<R, false>, dim3(grid), dim3(threads), 0,
             s, a, vec);
}

template <int R>
static void launch_warp_r(LineArgs<float> a, cudaStream_t s) {
  const size_t smem = line_warp_smem(R);
  dim3 grid((a.ncol + kLineTile - 1) / kLineTile, a.nother, a.nbatch);
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  const int threads = a.threads > 0 ? a.threads : 256;
  // half-length lines: forward from n = N/2 points, or inverse cropped to N/2
  const bool half = a.inverse ? (2 * a.lout == a.plan.N) : (2 * a.lin == a.plan.N);
  launch_pdl(half ? line_warp_kernel<R, true> : line_warp_kernel<R, false>, grid, dim3(threads), smem,
             s, a);
}

static bool launch_warp(const LineArgs<float>& a, cudaStream_t s) {
  const int N = a.plan.N;
  if (N % 32 != 0 || a.in_cs != 1 || a.out_cs != 1) return false;
  if ((a.flags & (PRO_CHI | EPI_CHI)) && a.chi_cs != 1) return false;
  switch (N / 32) {
    case 1: launch_reg_r<1>(a, s); return true;
    case 2: launch_fs_v<8>(a, s); return true;
    case 3: launch_reg_r<3>(a, s); return true;
    case 4: launch_fs_v<16>(a, s); return true;
    case 5: launch_reg_r<5>(a, s); return true;
    case 6: launch_fs_v<24>(a, s); return true;
    case 8: launch_warp_r<8>(a, s); return true;
    case 10: launch_warp_r<10>(a, s); return true;
    case 12: launch_warp_r<12>(a, s); return true;
    case 16: if (!launch_line_tp(a, s)) launch_warp_r<16>(a, s); return true;
    default: return false;
  }
}

template <typename T, int TW>
static void launch_tw(LineArgs<T> a, size_t smem, cudaStream_t s) {
  dim3 grid((a.ncol + TW - 1) / TW, a.nother, a.nbatch);
  a.prof = prof_bytes(a.prof_family);
  ProfScope ps(a.prof_family, s);
  line_fft_kernel<T, TW><<<grid, 256, smem, s>>>(a);
}

// Widest tile (16, 8 or 4 lines; 128 bytes per row for c64 at 16) whose two
// ping-pong buffers and root table fit in 227 KB of shared memory.
template <typename T>
void launch_line_fft(const LineArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (launch_warp(a, s)) return;
  } else {
    if (a.plan.N == 512 && launch_line_tp64(a, s)) return;
  }
  const int N = a.plan.N;
  auto bytes = [&](int tw) { return (size_t)(2 * N * tw + N) * sizeof(cx<T>); };
  const size_t limit = 227 * 1024;
  if constexpr (sizeof(T) == 4) {
    if (bytes(16) <= limit) {
      launch_tw<T, 16>(a, bytes(16), s);
      return;
    }
  }
  if (bytes(8) <= limit) launch_tw<T, 8>(a, bytes(8), s);
  else launch_tw<T, 4>(a, bytes(4), s);
}

}  // namespace vie

template <typename T>
void launch_line_fft(const LineArgs<T>& a, cudaStream_t s) {
  vie::launch_line_fft<T>(a, s);
}
template void launch_line_fft<float>(const LineArgs<float>&, cudaStream_t);
template void launch_line_fft<double>(const LineArgs<double>&, cudaStream_t);

// Opt every line kernel into the full 227 KB of dynamic shared memory (once
// per device, before any launch or graph capture).
int line_fft_init_attributes() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaSuccess;
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_fft_kernel<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_fft_kernel<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_fft_kernel<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_fft_kernel<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_fft_kernel<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<10, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<10, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<12, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<12, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  e = e != cudaSuccess ? e : cudaFuncSetAttribute(vie::line_warp_kernel<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "line kernel attributes");
}

bool make_plan(int N, FftPlan* plan) {
  plan->N = N;
  plan->npass = 0;
  if (N < 1 || N > VIE_MAX_N) return false;
  int m = N;
  static const int order[] = {8, 4, 2, 3, 5, 7};
  for (int r : order) {
    while (m % r == 0) {
      if (plan->npass == VIE_MAX_PASSES) return false;
      plan->radix[plan->npass++] = r;
      m /= r;
    }
  }
  return m == 1;
}
