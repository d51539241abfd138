// Internal declarations of libvie (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "vie.h"

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cx = typename cplx<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

#define VIE_CX_OPS(C, T)                                                                  \
  __host__ __device__ __forceinline__ C operator+(C a, C b) { return mk(a.x + b.x, a.y + b.y); } \
  __host__ __device__ __forceinline__ C operator-(C a, C b) { return mk(a.x - b.x, a.y - b.y); } \
  __host__ __device__ __forceinline__ C operator*(C a, C b) {                               \
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                 \
  }                                                                                         \
  __host__ __device__ __forceinline__ C operator*(T s, C a) { return mk(s * a.x, s * a.y); } \
  __host__ __device__ __forceinline__ C conjg(C a) { return mk(a.x, -a.y); }                \
  __host__ __device__ __forceinline__ C mul_i(C a) { return mk(-a.y, a.x); }               \
  __host__ __device__ __forceinline__ C mul_mi(C a) { return mk(a.y, -a.x); }              \
  __host__ __device__ __forceinline__ C cmadd(C a, C b, C c) { /* a*b + c */               \
    return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));      \
  }                                                                                         \
  __host__ __device__ __forceinline__ C conj_madd(C a, C b, C c) { /* conj(a)*b + c */     \
    return mk(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));      \
  }                                                                                         \
  __host__ __device__ __forceinline__ T abs2(C a) { return a.x * a.x + a.y * a.y; }
VIE_CX_OPS(float2, float)
VIE_CX_OPS(double2, double)
#undef VIE_CX_OPS

template <typename C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------------------
// FFT plan: mixed-radix Stockham, radices 8, 4, 2, 3, 5, 7.
// ---------------------------------------------------------------------------
#define VIE_MAX_PASSES 12
#define VIE_MAX_N 1024
struct FftPlan {
  int N;
  int npass;
  int radix[VIE_MAX_PASSES];
};
bool make_plan(int N, FftPlan* plan);   // false if N has a prime factor > 7

// ---------------------------------------------------------------------------
// Line-FFT stage parameters (strided lines along one axis of a 3-D array).
// Element (batch bb, other o, line position p, tile column c) lives at
//   bb*bs + o*os + p*ls + c*cs   (separately for input and output).
// ---------------------------------------------------------------------------
enum {
  PRO_CONJ = 1,      // conjugate the input
  PRO_CHI = 2,       // multiply the input by chi[p, o, c] (scalar field)
  EPI_CONJ = 4,      // conjugate the (scaled) result
  EPI_SUB = 8,       // out = addend - (chi?) result
  EPI_ADD = 16,      // out = addend + result
  EPI_CHI = 32,      // multiply the result by chi before EPI_SUB
  PRO_RSCALE = 64,   // multiply the input by the real per-RHS factor rscale[rhs * rscale_stride]
  EPI_RSCALE = 128   // multiply the addend by that factor (EPI_SUB / EPI_ADD)
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with launch_pdl may start
// while the kernel before it on the stream is still running, as soon as every
// CTA of that kernel has executed pdl_trigger(); everything it does before
// pdl_wait() must only read data that no earlier kernel writes (tables,
// factors) and only write on-chip storage.  pdl_wait() returns once the
// preceding kernel has completed and its memory is visible (immediately for a
// kernel launched without the attribute).  Both are no-ops for the driver
// outside such a launch, and neither waits on memory written by other CTAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// kernel-family profiler (profiler.cu)
// ---------------------------------------------------------------------------
enum {
  PF_LINE_X = 0, PF_LINE_Y, PF_FUSED_TUCKER, PF_FUSED_STORED, PF_LINE_IY, PF_LINE_IX, PF_REBUILD,
  PF_DOTS, PF_UPDATE, PF_SMALL, PF_FP64, PF_SETUP, PF_MATVEC64, VIE_PROF_FAMILIES
};
struct ProfEventPair {
  cudaEvent_t a, b;
  int family;
};
unsigned long long* prof_bytes(int family);     // device counter, nullptr when off
int prof_epoch();                               // -1 when off
int prof_begin(int family, cudaStream_t s);     // handle for prof_end (or -1)
void prof_end(int handle, cudaStream_t s);
void prof_set_capture_sink(std::vector<ProfEventPair>* sink);
void prof_harvest_graph(std::vector<ProfEventPair>& pairs);
void prof_release_pairs(std::vector<ProfEventPair>& pairs);

// RAII bracket of one launch
struct ProfScope {
  int h;
  cudaStream_t s;
  ProfScope(int family, cudaStream_t st) : h(prof_begin(family, st)), s(st) {}
  ~ProfScope() { prof_end(h, s); }
};

template <typename T> struct LineArgs {
  const cx<T>* in;
  cx<T>* out;
  const cx<T>* roots;      // N-th roots of unity exp(-2 pi i m / N), m < N
  const cx<T>* chi;        // scalar field (PRO_CHI / EPI_CHI)
  const cx<T>* addend;     // EPI_SUB / EPI_ADD, laid out like `out`
  const double* rscale;    // PRO_RSCALE / EPI_RSCALE: per-RHS real factor
  long long rscale_stride;
  FftPlan plan;
  int lin, lout;           // points loaded (rest zero) / points stored
  int inverse;
  T scale;
  int flags;
  int nbatch, nother, ncol;            // grid extents
  long long in_bs, in_os, in_ls, in_cs;
  long long out_bs, out_os, out_ls, out_cs;
  long long chi_os, chi_ls, chi_cs;    // chi index = o*chi_os + p*chi_ls + c*chi_cs
  int chi_vec, addend_vec;             // chi / addend rows allow 16-byte accesses
  int batch_per_rhs;                   // batches per RHS (3 components) for `active`
  const int* active;                   // per-RHS flag (nullptr = all active)
  int threads;                         // CTA size of the register-path kernel (0 = 256)
  int prof_family;                     // profiler family of this launch
  unsigned long long* prof;            // profiler byte counter (nullptr = off)
  unsigned long long prof_batch_bytes; // algorithmic bytes per active batch index
  int* err;                            // device word set when a bounded wait gives up (or nullptr)
};

template <typename T> void launch_line_fft(const LineArgs<T>& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Operator state
// ---------------------------------------------------------------------------
struct TuckerComp {
  int r[3];            // multilinear ranks
  int s[3];            // parity sign of the spectrum along each axis
  float2* core32 = nullptr;  double2* core64 = nullptr;   // [r1][r2][r3]
  float2* U32[3] = {};       double2* U64[3] = {};        // half factors [H_q][r_q]
  float2* U3t32 = nullptr;                                 // U3 half factor transposed [r3][H3]
  std::vector<double> sigma[3];                            // H_q singular values
};

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Launch shapes chosen by vie_autotune (defaults until it runs).
struct Tuning {
  int line_threads[4] = {256, 256, 256, 256};   // x, y, inverse y, inverse x stages
  int tuned_batch = 0;                          // batch the choice was timed at (0 = default)
  // tcgen05 rebuild tiles: N ranges per component (k3 columns per CTA =
  // (P3/2) / rb_nsplit) and CTAs per (component, range); 0 = the default plan
  int rb_nsplit = 0, rb_ctas = 0;
};

// Tucker+CP model (Algorithm 2, eq. (17)), formed by vie_tucker_cp: factors
// W^q = U^q V^q for the stored half rows ([H_q][R]; rows P_q - k follow by the
// parity sign of U^q), and the operands of the per-matvec rebuild.
constexpr int kCpMaxRank = 32;
struct CpModel {
  int R = 0;                               // 0: no model
  double err[6] = {};                      // relative core error ||G - CP|| / ||G||
  int sweeps[6] = {};
  double2* W64[6][3] = {};
  float2* W32[6][3] = {};
  float2* W3t32[6] = {};                   // W3 transposed [R][H3]
  void* meta = nullptr;                    // device records of the rebuild kernel
  uint4* frag = nullptr;                   // W3 in fragment order [6][nsplit][ks][ntc][32]
  int ks = 0, nsplit = 0, ntc = 0;
  unsigned epoch = 0;                      // bumped whenever the model's buffers change
};

struct vie_op {
  vie_grid grid;
  int n[3], P[3], H[3];
  double k0;
  int flags;
  TuckerComp comp[6];
  int rmax[3];
  // slab cores S_c[k1] = core_c x1 U1_c[k1, :] (mode 1 of eq. (13)), formed at setup
  float2* slab32 = nullptr;  double2* slab64 = nullptr;
  size_t slab_stride;        // elements per component: H1 * rmax2 * rmax3
  // per-matvec rebuild of the half fibres (FP32 Tucker path): scratch for
  // oct_k1 values of k1 at a time, [oct_k1][H2][6][H3], rewritten by every matvec
  float2* oct32 = nullptr;
  int oct_k1 = 0;
  // the first chunk's rebuild does not depend on J: it runs on this stream
  // beside the x and y stages and is joined before the fused kernel
  cudaStream_t rb_stream = nullptr;
  cudaEvent_t rb_fork = nullptr, rb_join = nullptr;
  // host-side, in launch order: chunk 0 of the next matvec's rebuild is already
  // enqueued on rb_stream (started by the previous matvec, see MV_PREFETCH_REBUILD)
  bool rb_pending = false;
  bool rb_cp = false;        // the pending (or last) rebuild used the Tucker+CP model
  // tensor-core rebuild: the real form of U3^T, split into TF32 value and
  // remainder, in mma fragment order [6][tc_nsplit][tc_ks][tc_ntc][32]
  uint4* u3frag = nullptr;
  int tc_ks = 0, tc_nsplit = 0, tc_ntc = 0;
  // the rebuild runs on tcgen05 (octant_umma_kernel, umma.cu) instead
  bool umma = false;
  CpModel cp;
  // stored spectra (optional)
  float2* spec32 = nullptr;  double2* spec64 = nullptr;
  FftPlan plan[3];
  float2* roots32[3] = {};   double2* roots64[3] = {};
  // device copy of per-component metadata for the fused kernel
  void* meta = nullptr;
  // device word that kernels with bounded waits set when a wait gives up
  // (VIE_ERR_TIMEOUT, reported by vie_solve); zero otherwise
  int* dev_err = nullptr;
  // device scratch the setup held while compressing (spectrum or Toeplitz octant,
  // Gram matrices, eigenvectors); released before the operator is returned
  size_t setup_scratch_bytes = 0;
  Workspace ws;
  int ws_batch = 0;
  Tuning tune;
  // solver scratch
  Workspace solve_ws;
  void* solver = nullptr;    // cached solver state (graphs), see solve.cu
};

// Per-component data read by the fused kernel (device copy in op->meta).
template <typename T> struct CompMeta {
  const cx<T>* U2;   // [H2][r2]
  const cx<T>* U3;   // [H3][r3]
  const cx<T>* U3t;  // [r3][H3] (FP32 only: coalesced rebuild reads; nullptr in FP64)
  const cx<T>* slab; // [H1][r2][r3] (row stride rmax)
  int r2, r3;
  int s1, s2, s3;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
int cuda_status(cudaError_t e, const char* what);
#define VIE_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return cuda_status(e__, #call);     \
  } while (0)
#define VIE_TRY(call)                        \
  do {                                       \
    int st__ = (call);                       \
    if (st__ != VIE_OK) return st__;         \
  } while (0)

int check_grid(const vie_grid* g);
int component_parity(int c, int axis);     // +1 / -1
void component_axes(int c, int* a, int* b);
double wavenumber(double freq_hz);

// matvec internals (matvec.cu)
// matvec_impl / matvec_run option: after the fused kernel, start rebuilding the
// half fibres for the next FP32 Tucker matvec on the operator's side stream (the
// next matvec joins it); the caller must make another Tucker matvec follow
enum { MV_PREFETCH_REBUILD = 1 };
// start that rebuild now (after the work already on s); the next matvec joins it
int prefetch_rebuild(const vie_op* op, cudaStream_t s, bool cp = false);
template <typename T>
int matvec_impl(const vie_op* op, const cx<T>* in, cx<T>* out, int B, int path, int pro_flags,
                int epi_flags, const cx<T>* chi, const cx<T>* addend, const int* active,
                cudaStream_t s, const double* rscale = nullptr, long long rscale_stride = 0,
                int mv_flags = 0);
// matvec scratch T1 + T2 for B right-hand sides of `elem`-byte complex values
// (8: FP32 path, 16: FP64 path); ensure_* grows op->ws to at least that size
int ensure_workspace(vie_op* op, int B, size_t elem);
int ensure_workspace_bytes(vie_op* op, size_t bytes);
// The four line-stage launches of one matvec (x, y, inverse y, inverse x).
template <typename T> struct LineStages {
  LineArgs<T> s[4];
};
template <typename T>
LineStages<T> make_line_stages(const vie_op* op, void* ws, const cx<T>* in, cx<T>* out, int B,
                               int pro_flags, int epi_flags, const cx<T>* chi, const cx<T>* addend,
                               const int* active, const double* rscale = nullptr,
                               long long rscale_stride = 0);
// the same stages with an explicit scratch buffer of at least matvec_scratch_bytes() bytes
template <typename T>
int matvec_run(const vie_op* op, void* ws, const cx<T>* in, cx<T>* out, int B, int path,
               int pro_flags, int epi_flags, const cx<T>* chi, const cx<T>* addend,
               const int* active, cudaStream_t s, const double* rscale = nullptr,
               long long rscale_stride = 0, int mv_flags = 0);
size_t workspace_bytes_for(const vie_op* op, int B, size_t elem);

template <typename T> int launch_slab_cores(const vie_op* op, cudaStream_t s);
// rebuild of the half fibres of k1 in [k1a, k1a + oct_k1) into op->oct32 (fused.cu);
// its dynamic shared memory holds W [6][r3][8], the slab cores of k1 [6][r2][r3]
// and eight U2 rows [6][8][r2]; operators whose ranks make that exceed
// kOctantSmemMax keep the in-CTA rebuild instead
constexpr int kOctantK2 = 8;
constexpr size_t kOctantSmemMax = 200u << 10;
__host__ __device__ constexpr size_t octant_smem_bytes(int r2max, int r3max) {
  return (size_t)(6 * r3max * kOctantK2 + 6 * r2max * r3max + 6 * kOctantK2 * r2max) * sizeof(float2);
}
int launch_octant(const vie_op* op, int k1a, cudaStream_t s, bool cp = false);
// the rebuild runs on the tensor cores (octant_tc_kernel, when the operator
// holds the U3 fragments), else on the FP32-FMA octant_kernel
bool octant_uses_tc(const vie_op* op);
bool tc_rebuild_eligible(const vie_op* op);
void tc_layout(int r3max, int H3, int* ks, int* nsplit, int* ntc);
bool tc_rebuild_fits(const vie_op* op);
int launch_u3_fragments(const vie_op* op, cudaStream_t s);
// the same rebuild on tcgen05 with TMEM accumulators (umma.cu): whether the
// operator's sizes fit it, and the launch for nk1 values of k1 from k1a
bool umma_rebuild_eligible(const vie_op* op);
int launch_octant_umma(const vie_op* op, int k1a, int nk1, cudaStream_t s);
// the N-range counts the tcgen05 rebuild accepts for this operator (at most
// `cap`), and the default CTAs per (component, range) for nsplit ranges
int umma_split_options(const vie_op* op, int* out, int cap);
int umma_default_ctas(const vie_op* op, int nsplit);
// the tiles the tcgen05 rebuild launches with (k3 columns per range, CTAs per
// (component, range)); zeros when the operator does not use it
void umma_tiles(const vie_op* op, int out[2]);
int umma_init_attributes();
int build_cp_rebuild(vie_op* op, cudaStream_t s);
void free_cp(vie_op* op);

// setup internals (setup.cu)
int build_operator(const vie_grid* grid, double tol, int rank_rule, int flags, cudaStream_t s,
                   vie_op** out);
int assemble_spectrum(const vie_op* op, int c, double2* out, cudaStream_t s);
int op_tables(vie_op* op);   // FFT plans and root tables of op->P
int line_fft_init_attributes();
// persistent grid size for `kernel` with `threads` threads and `smem` bytes of
// dynamic shared memory: resident CTAs per SM x SMs, capped by `work`
int device_sms();
int persistent_grid(const void* kernel, int threads, size_t smem, long long work);
int fused_init_attributes();
int multi_init_attributes();
int tp_init_attributes();

// solver (solve.cu)
int solve_impl(const vie_op* op, const void* chi, const void* rhs, void* w, int B, int flags,
               int precision, const vie_solve_opts* opts, vie_solve_info* info, cudaStream_t s);
void solver_release(vie_op* op);

// elementwise kernels (blas.cu)
template <typename T>
int launch_gradient(const cx<T>* lam, const cx<T>* E, cx<T>* grad, int B, double scale,
                    long long nvox, cudaStream_t s);
template <typename T>
int launch_dipole(const vie_op* op, const double* src_dev, int B, cx<T>* out, cudaStream_t s);
