// Several operators (grids of different sizes, each with its own batch of
// right-hand sides) through one persistent launch or one launch per matvec
// stage, and the autotuner that picks the line stages' CTA size and the
// tcgen05 rebuild's tiles.
//
// Each multi-grid kernel gets a table of per-problem arguments as a kernel
// parameter, with the prefix sums of the problems' work-item counts; a CTA
// finds its problem from the item index and runs the device body the
// per-operator kernels run for that problem's FFT length P = 32 R: for a line
// item (16 adjacent columns) each of the four warps transforms four columns
// with the four-step body (R even) or the register lane FFT (R odd), or the
// CTA runs the shared-memory tile (R = 8); a fused item is one mirror group,
// four-step (R even, half fibres from the operator's rebuild scratch) or lane
// FFT.
#include <algorithm>
#include <mutex>
#include <vector>

#include "stages.cuh"

template <typename T>
vie::FusedArgs<T> make_fused_args(const vie_op* op, cx<T>* data, int B, bool stored,
                                  const int* active);

namespace vie {

constexpr int kMaxMulti = 8;

struct MultiLine {
  int count;
  int R[kMaxMulti];
  int vec[kMaxMulti];          // lane FFT rows are 16-byte aligned (two 16-byte accesses per row)
  long long start[kMaxMulti + 1];
  LineArgs<float> a[kMaxMulti];
};
struct MultiFused {
  int count;
  int R[kMaxMulti];
  int fs[kMaxMulti];           // four-step body, half fibres from the rebuild scratch
  long long start[kMaxMulti + 1];
  FusedArgs<float> a[kMaxMulti];
};

constexpr int kMultiThreads = 128;     // 4 warps x 4 columns = one 16-column line item

// shared memory of a line item of length 32 R (4 warps), and of a fused item
__host__ __device__ constexpr size_t multi_line_smem(int R) {
  return R == 8 ? line_warp_smem(8) : (R % 2 == 0 ? line_fs_smem(4 * R, kMultiThreads / 32) : 0);
}

__device__ __forceinline__ int find_problem(const long long* start, int count, long long b) {
  int p = 0;
  while (p + 1 < count && b >= start[p + 1]) ++p;
  return p;
}

// radices the multi-grid kernels carry (P = 32 R <= 256)
__host__ __device__ constexpr bool multi_radix(int R) {
  return R == 1 || R == 2 || R == 3 || R == 4 || R == 5 || R == 6 || R == 8;
}

// One line item: columns [c0, c0 + 16) of line o of batch entry bb.
template <int RMAX>
__device__ __forceinline__ void multi_line_body(const MultiLine& ml, long long b, float2* smem) {
  const int p = find_problem(ml.start, ml.count, b);
  const LineArgs<float>& a = ml.a[p];
  const long long t = b - ml.start[p];
  const int ntc = (a.ncol + kLineTile - 1) / kLineTile;
  const int ct = (int)(t % ntc);
  const int o = (int)((t / ntc) % a.nother);
  const int bb = (int)(t / ((long long)ntc * a.nother));
  const int R = ml.R[p];
  if (R == 8) {
    if constexpr (RMAX >= 8) line_warp_tile<8, true>(a, ct * kLineTile, o, bb, smem);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = ct * kLineTile + warp * kRegCols;
  if (c0 >= a.ncol) return;                           // warp-uniform; no block barrier here
  float2* xs = smem + (size_t)warp * kRegCols * fs_col_stride(4 * R);
  switch (R) {
    case 1: line_reg_group<1, true>(a, c0, o, bb, ml.vec[p] != 0, lane); break;
    case 2: line_fs_group<8, true>(a, c0, o, bb, lane, xs); break;
    case 3: line_reg_group<3, true>(a, c0, o, bb, ml.vec[p] != 0, lane); break;
    case 4: line_fs_group<16, true>(a, c0, o, bb, lane, xs); break;
    case 5: if constexpr (RMAX >= 5) line_reg_group<5, true>(a, c0, o, bb, ml.vec[p] != 0, lane); break;
    case 6: if constexpr (RMAX >= 6) line_fs_group<24, true>(a, c0, o, bb, lane, xs); break;
    default: break;
  }
}

// One fused item: mirror group g of its problem.
template <int RMAX>
__device__ __forceinline__ void multi_fused_body(const MultiFused& mf, long long b, float2* smem) {
  const int p = find_problem(mf.start, mf.count, b);
  const int g = (int)(b - mf.start[p]);
  const FusedArgs<float>& a = mf.a[p];
  if (mf.fs[p]) {
    switch (mf.R[p]) {
      case 2: fused_fs_group<8, false>(a, g, smem); break;
      case 4: fused_fs_group<16, false>(a, g, smem); break;
      case 6: if constexpr (RMAX >= 6) fused_fs_group<24, false>(a, g, smem); break;
      default: break;
    }
    return;
  }
  switch (mf.R[p]) {
    case 1: fused_warp_group<1, false>(a, g, smem); break;
    case 2: fused_warp_group<2, false>(a, g, smem); break;
    case 3: fused_warp_group<3, false>(a, g, smem); break;
    case 4: fused_warp_group<4, false>(a, g, smem); break;
    case 5: if constexpr (RMAX >= 5) fused_warp_group<5, false>(a, g, smem); break;
    case 6: if constexpr (RMAX >= 6) fused_warp_group<6, false>(a, g, smem); break;
    case 8: if constexpr (RMAX >= 8) fused_warp_group<8, false>(a, g, smem); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kMultiThreads) line_multi_kernel(const __grid_constant__ MultiLine m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  multi_line_body<8>(m, blockIdx.x, reinterpret_cast<float2*>(smem_raw));
}

__global__ void __launch_bounds__(kMultiThreads) fused_multi_kernel(const __grid_constant__ MultiFused m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  multi_fused_body<8>(m, blockIdx.x, reinterpret_cast<float2*>(smem_raw));
}

// ---------------------------------------------------------------------------
// The whole matvec of several operators as one persistent cooperative launch:
// the five stages (x, y, fused z with the rebuild in each CTA, inverse y,
// inverse x) run one after another, each CTA taking the stage's work items
// (line tiles or mirror groups of any problem) in steps of the grid, with a
// grid-wide barrier between stages.  Every CTA of a cooperative launch is
// resident, so the barrier is met; its wait is still bounded by the device
// timer, and a CTA that gives up sets the error word and returns.
// ---------------------------------------------------------------------------
struct MultiAll {
  MultiLine line[4];        // x, y, inverse y, inverse x
  MultiFused fused;
};

struct GridBarrier {
  unsigned count;
  unsigned gen;
};

__device__ __forceinline__ unsigned long long global_ns_multi() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// false (in every thread of the CTA) if the other CTAs did not arrive within budget_ns
__device__ bool grid_barrier(GridBarrier* gb, unsigned nblocks, unsigned long long budget_ns) {
  __syncthreads();
  int bad = 0;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gb->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns_multi();
      while (*vgen == g) {
        if (global_ns_multi() - t0 > budget_ns) {
          bad = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  return __syncthreads_or(bad) == 0;
}

// RMAX: the largest radix the launch carries (the register budget follows it)
template <int RMAX>
__global__ void __launch_bounds__(kMultiThreads, 4) matvec_multi_persistent_kernel(const __grid_constant__ MultiAll m,
                                                                      GridBarrier* gb, int* err,
                                                                      unsigned long long budget_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* smem = reinterpret_cast<float2*>(smem_raw);
  for (int st = 0; st < 5; ++st) {
    if (st == 2) {
      const long long total = m.fused.start[m.fused.count];
      for (long long b = blockIdx.x; b < total; b += gridDim.x) {
        multi_fused_body<RMAX>(m.fused, b, smem);
        __syncthreads();                       // shared tables reused by the next item
      }
    } else {
      const MultiLine& ml = m.line[st < 2 ? st : st - 1];
      const long long total = ml.start[ml.count];
      for (long long b = blockIdx.x; b < total; b += gridDim.x) {
        multi_line_body<RMAX>(ml, b, smem);
        __syncthreads();
      }
    }
    if (st < 4 && !grid_barrier(gb, gridDim.x, budget_ns)) {
      if (threadIdx.x == 0 && err != nullptr) atomicExch(err, VIE_ERR_TIMEOUT);
      return;
    }
  }
}

// self-test of the grid barrier: every CTA but (when skip_last) the last one
// arrives; status[cta] = 1 if the barrier completed for it, 2 if it gave up
__global__ void grid_barrier_selftest_kernel(GridBarrier* gb, int skip_last, unsigned long long budget_ns,
                                             int* status) {
  if (skip_last && blockIdx.x == gridDim.x - 1) {
    if (threadIdx.x == 0) status[blockIdx.x] = 0;
    return;
  }
  const bool ok = grid_barrier(gb, gridDim.x, budget_ns);
  if (threadIdx.x == 0) status[blockIdx.x] = ok ? 1 : 2;
}

}  // namespace vie

using namespace vie;

// Two co-resident CTAs meet at a grid barrier (all_arrive) or one of them never
// comes: VIE_OK when the barrier completed, VIE_ERR_TIMEOUT when the waiting
// CTA gave up after `seconds`.  Its own barrier state, freed afterwards.
int grid_barrier_selftest(bool all_arrive, double seconds, cudaStream_t s) {
  GridBarrier* gb = nullptr;
  int* st = nullptr;
  int h[2] = {0, 0};
  cudaError_t e = cudaMalloc(&gb, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMalloc(&st, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(gb, 0, sizeof(GridBarrier), s);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(64);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, grid_barrier_selftest_kernel, gb, all_arrive ? 0 : 1,
                           (unsigned long long)(seconds * 1e9), st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, st, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(gb);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_status(e, "grid-barrier self-test");
  if (h[0] == 2) {
    set_error("the grid barrier gave up after %g s", seconds);
    return VIE_ERR_TIMEOUT;
  }
  return h[0] == 1 && (!all_arrive || h[1] == 1) ? VIE_OK : VIE_ERR_CUDA;
}

static bool multi_eligible(const vie_op* op) {
  for (int q = 0; q < 3; ++q)
    if (op->P[q] % 32 != 0 || !multi_radix(op->P[q] / 32)) return false;
  return true;
}

int multi_init_attributes() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(line_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(matvec_multi_persistent_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(matvec_multi_persistent_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(matvec_multi_persistent_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "multi kernel attributes");
}

// Grid barrier state of the persistent launch, one per device, allocated once
// and zeroed (each use leaves the count at zero and advances the generation).
static int multi_grid_barrier(GridBarrier** out) {
  static std::mutex mu;
  static GridBarrier* ptr[64] = {};
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device %d outside the supported range", dev);
    return VIE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!ptr[dev]) {
    GridBarrier* p = nullptr;
    VIE_CUDA(cudaMalloc(&p, sizeof(GridBarrier)));
    VIE_CUDA(cudaMemset(p, 0, sizeof(GridBarrier)));
    ptr[dev] = p;
  }
  *out = ptr[dev];
  return VIE_OK;
}

// The matvec of up to kMaxMulti operators: one persistent cooperative launch, or
// one launch per stage.  VIE_ERR_ARG from the persistent form means it cannot be
// made co-resident (the caller then uses the staged form).
static int matvec_multi_chunk(const vie_op* const* ops, const float2* const* J, float2* const* Y,
                              const int* B, int count, bool persistent, cudaStream_t s) {
  std::vector<LineStages<float>> lines(count);
  std::vector<char> prebuilt(count, 0);
  MultiLine ml[4];
  MultiFused mf;
  size_t smem_line = 0, smem_fused = 0;
  for (int st = 0; st < 4; ++st) ml[st].count = count;
  mf.count = count;
  long long lstart[4] = {0, 0, 0, 0}, fstart = 0;
  for (int p = 0; p < count; ++p) {
    const vie_op* op = ops[p];
    VIE_TRY(ensure_workspace(const_cast<vie_op*>(op), B[p], sizeof(float2)));
    lines[p] = make_line_stages<float>(op, op->ws.ptr, J[p], Y[p], B[p], 0, 0, nullptr, nullptr,
                                       nullptr);
    for (int st = 0; st < 4; ++st) {
      LineArgs<float> a = lines[p].s[st];
      a.prof = prof_bytes(a.prof_family);
      ml[st].a[p] = a;
      ml[st].R[p] = a.plan.N / 32;
      // 16-byte row accesses of the lane FFT: every row of every group starts
      // on a 16-byte boundary
      ml[st].vec[p] = a.in_bs % 2 == 0 && a.in_os % 2 == 0 && a.in_ls % 2 == 0 && a.out_bs % 2 == 0 &&
                      a.out_os % 2 == 0 && a.out_ls % 2 == 0 && ((uintptr_t)a.in & 15u) == 0 &&
                      ((uintptr_t)a.out & 15u) == 0;
      ml[st].start[p] = lstart[st];
      lstart[st] += (long long)((a.ncol + kLineTile - 1) / kLineTile) * a.nother * a.nbatch;
      smem_line = std::max(smem_line, multi_line_smem(a.plan.N / 32));
    }
    float2* T2 = lines[p].s[1].out;
    mf.a[p] = make_fused_args<float>(op, T2, B[p], false, nullptr);
    // An operator whose rebuild scratch holds every k1 has its half fibres
    // rebuilt once by its own rebuild kernel (on its side stream, after the
    // work already on s) and shared by all its right-hand sides; the fused
    // items then copy them instead of rebuilding them in each CTA.
    if (op->oct32 != nullptr && op->rb_stream != nullptr && op->oct_k1 >= op->H[0]) {
      if (!(op->rb_pending && !op->rb_cp)) {
        VIE_CUDA(cudaEventRecord(op->rb_fork, s));
        VIE_CUDA(cudaStreamWaitEvent(op->rb_stream, op->rb_fork, 0));
        VIE_TRY(launch_octant(op, 0, op->rb_stream, false));
        VIE_CUDA(cudaEventRecord(op->rb_join, op->rb_stream));
      }
      const_cast<vie_op*>(op)->rb_pending = false;
      prebuilt[p] = true;
      mf.a[p].octant = op->oct32;
      mf.a[p].oct_k1a = 0;
      mf.a[p].oct_chunk = op->oct_k1;
    }
    mf.R[p] = op->P[2] / 32;
    mf.fs[p] = prebuilt[p] && mf.R[p] % 2 == 0 && mf.R[p] <= 6;
    mf.start[p] = fstart;
    fstart += (long long)op->H[0] * op->H[1];
    smem_fused = std::max(smem_fused, mf.fs[p] ? fused_fs_smem(4 * mf.R[p], op->H[2])
                                               : fused_warp_smem(op->P[2] / 32, op->H[2], op->rmax[1],
                                                                 op->rmax[2]));
  }
  for (int st = 0; st < 4; ++st) ml[st].start[count] = lstart[st];
  mf.start[count] = fstart;
  if (persistent) {
    MultiAll* all = new MultiAll;
    for (int st = 0; st < 4; ++st) {
      all->line[st] = ml[st];
      for (int p = 0; p < count; ++p) all->line[st].a[p].prof = nullptr;
    }
    all->fused = mf;
    for (int p = 0; p < count; ++p) all->fused.a[p].prof = nullptr;
    const size_t smem = std::max(smem_line, smem_fused);
    int rmax = 1;
    for (int p = 0; p < count; ++p)
      for (int q = 0; q < 3; ++q) rmax = std::max(rmax, ops[p]->P[q] / 32);
    using PK = void (*)(MultiAll, GridBarrier*, int*, unsigned long long);
    const PK kern = rmax <= 4 ? matvec_multi_persistent_kernel<4>
                              : (rmax <= 6 ? matvec_multi_persistent_kernel<6> : matvec_multi_persistent_kernel<8>);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMultiThreads, smem);
    long long work = fstart;
    for (int st = 0; st < 4; ++st) work = std::max(work, lstart[st]);
    GridBarrier* gb = nullptr;
    int rc = VIE_OK;
    if (e != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      rc = VIE_ERR_ARG;   // not co-resident: the caller falls back to the staged launches
    } else if ((rc = multi_grid_barrier(&gb)) == VIE_OK) {
      const unsigned grid = (unsigned)std::min<long long>(work, (long long)per_sm * device_sms());
      for (int p = 0; p < count && rc == VIE_OK; ++p)
        if (prebuilt[p] && cudaStreamWaitEvent(s, ops[p]->rb_join, 0) != cudaSuccess)
          rc = cuda_status(cudaGetLastError(), "rebuild join");
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(kMultiThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (rc == VIE_OK) {
        ProfScope ps(PF_FUSED_TUCKER, s);
        e = cudaLaunchKernelEx(&cfg, kern, *all, gb, ops[0]->dev_err, (unsigned long long)1000000000ull);
        if (e != cudaSuccess) rc = cuda_status(e, "persistent multi-grid matvec launch");
      }
    }
    delete all;
    return rc;
  }
  static const int fam[4] = {PF_LINE_X, PF_LINE_Y, PF_LINE_IY, PF_LINE_IX};
  for (int st = 0; st < 4; ++st) {
    if (st == 2) {
      for (int p = 0; p < count; ++p)
        if (prebuilt[p]) VIE_CUDA(cudaStreamWaitEvent(s, ops[p]->rb_join, 0));
      ProfScope ps(PF_FUSED_TUCKER, s);
      fused_multi_kernel<<<(unsigned)fstart, kMultiThreads, smem_fused, s>>>(mf);
    }
    ProfScope ps(fam[st], s);
    // every stage of every operator is a half-length transform (zero pad or crop)
    line_multi_kernel<<<(unsigned)lstart[st], kMultiThreads, smem_line, s>>>(ml[st]);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "multi-grid matvec launch");
  return VIE_OK;
}

extern "C" int vie_matvec_multi_ex(const vie_op* const* ops, const void* const* J, void* const* Y,
                                   const int* B, int count, int mode, void* stream) {
  clear_error();
  if (mode != VIE_MULTI_PERSISTENT && mode != VIE_MULTI_STAGED) {
    set_error("unknown multi-grid mode %d", mode);
    return VIE_ERR_ARG;
  }
  if (!ops || !J || !Y || !B || count < 1) {
    set_error("NULL argument or empty problem list");
    return VIE_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool all = true;
  for (int p = 0; p < count; ++p) {
    if (!ops[p] || !J[p] || !Y[p] || B[p] < 1 || B[p] > 4096) {
      set_error("problem %d: NULL operator/array or batch outside [1, 4096]", p);
      return VIE_ERR_ARG;
    }
    all = all && multi_eligible(ops[p]);
  }
  if (!all) {
    // a grid edge that is not 32 R (R <= 8): one matvec per operator
    for (int p = 0; p < count; ++p)
      VIE_TRY(matvec_impl<float>(ops[p], static_cast<const float2*>(J[p]), static_cast<float2*>(Y[p]),
                                 B[p], VIE_PATH_TUCKER, 0, 0, nullptr, nullptr, nullptr, s));
    return VIE_OK;
  }
  for (int p0 = 0; p0 < count; p0 += kMaxMulti) {
    const int c = std::min(kMaxMulti, count - p0);
    const float2* const* Jc = reinterpret_cast<const float2* const*>(J) + p0;
    float2* const* Yc = reinterpret_cast<float2* const*>(Y) + p0;
    int rc = VIE_ERR_ARG;
    if (mode == VIE_MULTI_PERSISTENT) rc = matvec_multi_chunk(ops + p0, Jc, Yc, B + p0, c, true, s);
    if (rc == VIE_ERR_ARG) rc = matvec_multi_chunk(ops + p0, Jc, Yc, B + p0, c, false, s);
    VIE_TRY(rc);
  }
  return VIE_OK;
}

extern "C" int vie_matvec_multi(const vie_op* const* ops, const void* const* J, void* const* Y,
                                const int* B, int count, void* stream) {
  return vie_matvec_multi_ex(ops, J, Y, B, count, VIE_MULTI_PERSISTENT, stream);
}

// Time the per-matvec rebuild (every k1 chunk) of a tcgen05 operator with each
// tile shape: N ranges per component (the accepted counts) x CTAs per
// (component, range) (half, one and two times the one-per-SM default); keep
// the fastest in op->tune.  The tiles change only the speed of the rebuild.
static int tune_rebuild_tiles(vie_op* op, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  int opts[16];
  const int nopt = umma_split_options(op, opts, 16);
  float best = 1e30f;
  int best_split = 0, best_ctas = 0;
  for (int i = 0; i < nopt; ++i) {
    const int d = umma_default_ctas(op, opts[i]);
    const int ctas[3] = {std::max(1, d / 2), d, 2 * d};
    for (int ci = 0; ci < 3; ++ci) {
      op->tune.rb_nsplit = opts[i];
      op->tune.rb_ctas = ctas[ci];
      float total = 0.f;
      for (int rep = 0; rep < 4; ++rep) {              // rep 0 warms up
        VIE_CUDA(cudaEventRecord(e0, s));
        for (int k1a = 0; k1a < op->H[0]; k1a += op->oct_k1)
          VIE_TRY(launch_octant(op, k1a, s, false));
        VIE_CUDA(cudaEventRecord(e1, s));
        VIE_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        VIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) total += ms;
      }
      if (total < best) {
        best = total;
        best_split = opts[i];
        best_ctas = ctas[ci];
      }
    }
  }
  op->tune.rb_nsplit = best_split;
  op->tune.rb_ctas = best_ctas;
  return VIE_OK;
}

// Time the FP32 Tucker matvec at batch B with each candidate CTA size of each
// line stage (the other stages at their current choice) and keep the fastest;
// then the tile shape of the tcgen05 rebuild.
extern "C" int vie_autotune(vie_op* op, int B, void* stream) {
  if (!op || B < 1 || B > 4096) {
    set_error("bad operator or batch");
    return VIE_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  VIE_TRY(ensure_workspace(op, B, sizeof(float2)));
  const size_t n = (size_t)B * 3 * op->n[0] * op->n[1] * op->n[2];
  float2 *J = nullptr, *Y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = VIE_OK;
  if (cudaMalloc(&J, n * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&Y, n * sizeof(float2)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    set_error("autotune scratch allocation failed");
    rc = VIE_ERR_OOM;
  }
  if (rc == VIE_OK) {
    cudaMemsetAsync(J, 0, n * sizeof(float2), s);
    static const int cand[3] = {64, 128, 256};
    for (int st = 0; st < 4 && rc == VIE_OK; ++st) {
      float best = 1e30f;
      int best_t = op->tune.line_threads[st];
      for (int t : cand) {
        op->tune.line_threads[st] = t;
        float total = 0.f;
        for (int rep = 0; rep < 4 && rc == VIE_OK; ++rep) {   // rep 0 warms up
          cudaEventRecord(e0, s);
          rc = matvec_impl<float>(op, J, Y, B, VIE_PATH_TUCKER, 0, 0, nullptr, nullptr, nullptr, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) total += ms;
        }
        if (total < best) {
          best = total;
          best_t = t;
        }
      }
      op->tune.line_threads[st] = best_t;
    }
    // the rebuild's scratch is free here: no matvec of this operator is in
    // flight on another stream while the caller tunes it
    if (rc == VIE_OK && op->umma && !op->rb_pending) rc = tune_rebuild_tiles(op, s, e0, e1);
    op->tune.tuned_batch = B;
  }
  cudaFree(J);
  cudaFree(Y);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
