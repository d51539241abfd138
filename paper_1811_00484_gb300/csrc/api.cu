// C ABI entry points of libvie (declared in include/vie.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "vie_internal.cuh"

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return VIE_ERR_OOM;
  return VIE_ERR_CUDA;
}

double wavenumber(double freq_hz) { return 2.0 * 3.14159265358979323846 * freq_hz / 299792458.0; }

// components in the order xx, xy, xz, yy, yz, zz
void component_axes(int c, int* a, int* b) {
  static const int A[6] = {0, 0, 0, 1, 1, 2}, Bv[6] = {0, 1, 2, 1, 2, 2};
  *a = A[c];
  *b = Bv[c];
}

// The kernel (k0^2 delta_ab + d_a d_b) g is odd in coordinate q once for each
// of a, b equal to q; so is its circulant embedding and its DFT.
int component_parity(int c, int axis) {
  int a, b;
  component_axes(c, &a, &b);
  return ((a == axis) + (b == axis)) % 2 ? -1 : 1;
}

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    sms = v;
  }
  return sms;
}

int persistent_grid(const void* kernel, int threads, size_t smem, long long work) {
  const int sms = device_sms();
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm <= 0) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long g = (long long)per_sm * sms;
  return (int)(work < g ? (work > 0 ? work : 1) : g);
}

int check_grid(const vie_grid* g) {
  if (!g) { set_error("grid is NULL"); return VIE_ERR_ARG; }
  const int n[3] = {g->n1, g->n2, g->n3};
  for (int q = 0; q < 3; ++q) {
    if (n[q] < 1 || n[q] > 512) {
      set_error("grid edge n%d = %d outside [1, 512]", q + 1, n[q]);
      return VIE_ERR_ARG;
    }
    FftPlan p;
    if (!make_plan(2 * n[q], &p)) {
      set_error("padded edge %d has a prime factor above 7", 2 * n[q]);
      return VIE_ERR_ARG;
    }
  }
  if (!(g->h > 0.0) || !std::isfinite(g->h)) { set_error("voxel edge h must be > 0"); return VIE_ERR_ARG; }
  if (!(g->freq_hz >= 0.0) || !std::isfinite(g->freq_hz)) {
    set_error("frequency must be >= 0");
    return VIE_ERR_ARG;
  }
  return VIE_OK;
}

static int check_op(const vie_op* op, int B) {
  if (!op) { set_error("operator is NULL"); return VIE_ERR_ARG; }
  if (B < 1 || B > 4096) { set_error("batch %d outside [1, 4096]", B); return VIE_ERR_ARG; }
  return VIE_OK;
}

static int check_prec_path(int precision, int path, const vie_op* op) {
  if (precision != VIE_C64 && precision != VIE_C128) {
    set_error("precision must be VIE_C64 or VIE_C128");
    return VIE_ERR_ARG;
  }
  if (path != VIE_PATH_TUCKER && path != VIE_PATH_UNCOMPRESSED && path != VIE_PATH_TUCKER_CP) {
    set_error("path must be VIE_PATH_TUCKER, VIE_PATH_UNCOMPRESSED or VIE_PATH_TUCKER_CP");
    return VIE_ERR_ARG;
  }
  if (path == VIE_PATH_UNCOMPRESSED && op->spec32 == nullptr) {
    set_error("operator was built without VIE_STORE_UNCOMPRESSED");
    return VIE_ERR_ARG;
  }
  if (path == VIE_PATH_TUCKER_CP && op->cp.R == 0) {
    set_error("no Tucker+CP model: call vie_tucker_cp first");
    return VIE_ERR_ARG;
  }
  return VIE_OK;
}

// Operator applications with the Tucker+CP model exist in FP32 only.
static int check_cp_precision(int precision, int path) {
  if (path == VIE_PATH_TUCKER_CP && precision != VIE_C64) {
    set_error("VIE_PATH_TUCKER_CP applies the FP32 model: use VIE_C64");
    return VIE_ERR_ARG;
  }
  return VIE_OK;
}

void clear_error() { g_last_error.clear(); }

#define CLEAR_ERROR() g_last_error.clear()

template <typename T>
static int matvec_dispatch(const vie_op* op, const void* in, void* out, int B, int path, int pro,
                           int epi, const void* chi, const void* addend, cudaStream_t s) {
  return matvec_impl<T>(op, static_cast<const cx<T>*>(in), static_cast<cx<T>*>(out), B, path, pro,
                        epi, static_cast<const cx<T>*>(chi), static_cast<const cx<T>*>(addend),
                        nullptr, s);
}

static int run_matvec(const vie_op* op, const void* in, void* out, int B, int path, int precision,
                      int pro, int epi, const void* chi, const void* addend, void* stream) {
  VIE_TRY(check_op(op, B));
  VIE_TRY(check_prec_path(precision, path, op));
  VIE_TRY(check_cp_precision(precision, path));
  if (!in || !out) { set_error("NULL array"); return VIE_ERR_ARG; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == VIE_C64) return matvec_dispatch<float>(op, in, out, B, path, pro, epi, chi, addend, s);
  return matvec_dispatch<double>(op, in, out, B, path, pro, epi, chi, addend, s);
}

extern "C" {

int vie_tucker_compress(const vie_grid* grid, double tol, int rank_rule, int flags, void* stream,
                        vie_op** out) {
  CLEAR_ERROR();
  if (!out) { set_error("out is NULL"); return VIE_ERR_ARG; }
  *out = nullptr;
  VIE_TRY(check_grid(grid));
  if (!(tol > 0.0 && tol < 1.0)) { set_error("tol must lie in (0, 1)"); return VIE_ERR_ARG; }
  if (rank_rule != VIE_RANK_TAIL && rank_rule != VIE_RANK_SIGMA_MAX) {
    set_error("unknown rank rule %d", rank_rule);
    return VIE_ERR_ARG;
  }
  if (flags & ~(VIE_STORE_UNCOMPRESSED | VIE_SELF_TERM_PV | VIE_REBUILD_SIMT | VIE_REBUILD_TCGEN05 |
                VIE_SETUP_FACTORWISE)) {
    set_error("unknown flags 0x%x", flags);
    return VIE_ERR_ARG;
  }
  return build_operator(grid, tol, rank_rule, flags, static_cast<cudaStream_t>(stream), out);
}

int vie_op_info(const vie_op* op, vie_op_info_t* info) {
  CLEAR_ERROR();
  if (!op || !info) { set_error("NULL argument"); return VIE_ERR_ARG; }
  vie_op_info_t r = {};
  size_t half = 0, fullf = 0;
  for (int q = 0; q < 3; ++q) {
    r.n[q] = op->n[q];
    r.P[q] = op->P[q];
  }
  for (int c = 0; c < 6; ++c) {
    const TuckerComp& tc = op->comp[c];
    const size_t core = (size_t)tc.r[0] * tc.r[1] * tc.r[2];
    half += core;
    fullf += core;
    for (int q = 0; q < 3; ++q) {
      r.ranks[c][q] = tc.r[q];
      half += (size_t)op->H[q] * tc.r[q];
      fullf += (size_t)op->P[q] * tc.r[q];
    }
  }
  r.tucker_bytes = half * sizeof(float2);
  r.tucker_bytes_full = fullf * sizeof(float2);
  r.slab_bytes = 6 * op->slab_stride * sizeof(float2);
  r.rebuild_scratch_bytes = (size_t)op->oct_k1 * op->H[1] * 6 * op->H[2] * sizeof(float2);
  r.uncompressed_bytes = 6ull * op->P[0] * op->P[1] * op->P[2] * sizeof(float2);
  r.workspace_bytes = op->ws.bytes + op->solve_ws.bytes;
  r.has_uncompressed = op->spec32 != nullptr;
  r.max_batch = op->ws_batch;
  for (int i = 0; i < 4; ++i) r.line_threads[i] = op->tune.line_threads[i];
  r.tuned_batch = op->tune.tuned_batch;
  r.rebuild_kernel = op->oct32 == nullptr ? 0 : op->umma ? 3 : (octant_uses_tc(op) ? 2 : 1);
  r.cp_rank = op->cp.R;
  for (int c = 0; c < 6; ++c) {
    r.cp_rel_err[c] = op->cp.err[c];
    r.cp_sweeps[c] = op->cp.sweeps[c];
  }
  r.cp_bytes = op->cp.R == 0 ? 0 : (size_t)6 * (op->H[0] + op->H[1] + op->H[2]) * op->cp.R * sizeof(float2);
  // device memory held for the Tucker path: cores and half factors in both
  // precisions, the transposed FP32 U3, slab cores in both precisions, the U3
  // fragments and rebuild scratch of the FP32 rebuild, metadata, root tables
  size_t tb = 0;
  for (int c = 0; c < 6; ++c) {
    const TuckerComp& tc = op->comp[c];
    tb += (size_t)tc.r[0] * tc.r[1] * tc.r[2] * (sizeof(float2) + sizeof(double2));
    for (int q = 0; q < 3; ++q) tb += (size_t)op->H[q] * tc.r[q] * (sizeof(float2) + sizeof(double2));
    if (tc.U3t32) tb += (size_t)op->H[2] * tc.r[2] * sizeof(float2);
  }
  tb += 6 * op->slab_stride * (sizeof(float2) + sizeof(double2));
  if (op->u3frag) tb += 6ull * op->tc_nsplit * op->tc_ks * op->tc_ntc * 32 * sizeof(uint4);
  tb += r.rebuild_scratch_bytes;
  tb += 12 * sizeof(CompMeta<float>);
  for (int q = 0; q < 3; ++q) tb += (size_t)op->P[q] * (sizeof(float2) + sizeof(double2));
  if (op->cp.R > 0) {
    tb += r.cp_bytes * 3;                                          // W32 and W64
    tb += 6ull * op->H[2] * op->cp.R * sizeof(float2);             // W3 transposed
    tb += 6ull * op->cp.nsplit * op->cp.ks * op->cp.ntc * 32 * sizeof(uint4);
  }
  r.device_bytes_tucker = tb;
  r.device_bytes_spectra = op->spec32 ? 6ull * op->P[0] * op->P[1] * op->P[2] *
                                            (sizeof(float2) + sizeof(double2))
                                      : 0;
  r.matvec_workspace_bytes = op->ws.bytes;
  r.solver_workspace_bytes = op->solve_ws.bytes;
  r.setup_scratch_bytes = op->setup_scratch_bytes;
  umma_tiles(op, r.rebuild_tiles);
  *info = r;
  return VIE_OK;
}

int vie_op_export(const vie_op* op, int c, double* core, double* U1, double* U2, double* U3,
                  double* sigma1, double* sigma2, double* sigma3, void* stream) {
  CLEAR_ERROR();
  if (!op || c < 0 || c > 5) { set_error("bad operator or component"); return VIE_ERR_ARG; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const TuckerComp& tc = op->comp[c];
  VIE_CUDA(cudaStreamSynchronize(s));
  if (core) {
    const size_t n = (size_t)tc.r[0] * tc.r[1] * tc.r[2];
    VIE_CUDA(cudaMemcpy(core, tc.core64, n * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  double* U[3] = {U1, U2, U3};
  double* sg[3] = {sigma1, sigma2, sigma3};
  for (int q = 0; q < 3; ++q) {
    const int H = op->H[q], P = op->P[q], r = tc.r[q];
    if (U[q]) {
      std::vector<double2> half((size_t)H * r);
      VIE_CUDA(cudaMemcpy(half.data(), tc.U64[q], half.size() * sizeof(double2),
                          cudaMemcpyDeviceToHost));
      double2* dst = reinterpret_cast<double2*>(U[q]);
      for (int k = 0; k < P; ++k) {
        const bool mirror = 2 * k > P;
        const int src = mirror ? P - k : k;
        const double sg_ = mirror ? (double)tc.s[q] : 1.0;
        for (int j = 0; j < r; ++j) {
          const double2 v = half[(size_t)src * r + j];
          dst[(size_t)k * r + j] = make_double2(sg_ * v.x, sg_ * v.y);
        }
      }
    }
    if (sg[q])
      for (int j = 0; j < H; ++j) sg[q][j] = tc.sigma[q][j];
  }
  return VIE_OK;
}

int vie_green_spectrum(const vie_grid* grid, int c, int flags, void* out, void* stream) {
  CLEAR_ERROR();
  VIE_TRY(check_grid(grid));
  if (c < 0 || c > 5 || !out) { set_error("bad component or NULL output"); return VIE_ERR_ARG; }
  vie_op tmp;
  tmp.grid = *grid;
  tmp.flags = flags;
  tmp.k0 = wavenumber(grid->freq_hz);
  const int nn[3] = {grid->n1, grid->n2, grid->n3};
  for (int q = 0; q < 3; ++q) {
    tmp.n[q] = nn[q];
    tmp.P[q] = 2 * nn[q];
    tmp.H[q] = nn[q] + 1;
  }
  int st = op_tables(&tmp);
  if (st == VIE_OK) st = assemble_spectrum(&tmp, c, static_cast<double2*>(out),
                                           static_cast<cudaStream_t>(stream));
  if (st == VIE_OK) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) st = cuda_status(e, "spectrum");
  }
  for (int q = 0; q < 3; ++q) {
    cudaFree(tmp.roots32[q]);
    cudaFree(tmp.roots64[q]);
    tmp.roots32[q] = nullptr;
    tmp.roots64[q] = nullptr;
  }
  return st;
}

int vie_reserve(vie_op* op, int max_batch) {
  CLEAR_ERROR();
  VIE_TRY(check_op(op, max_batch));
  return ensure_workspace(op, max_batch, sizeof(double2));
}

int vie_matvec(const vie_op* op, const void* J, void* Y, int B, int path, int precision,
               void* stream) {
  CLEAR_ERROR();
  return run_matvec(op, J, Y, B, path, precision, 0, 0, nullptr, nullptr, stream);
}

int vie_matvec_adjoint(const vie_op* op, const void* Y, void* X, int B, int path, int precision,
                       void* stream) {
  CLEAR_ERROR();
  return run_matvec(op, Y, X, B, path, precision, PRO_CONJ, EPI_CONJ, nullptr, nullptr, stream);
}

int vie_apply_system(const vie_op* op, const void* chi, const void* w, void* out, int B,
                     int adjoint, int path, int precision, void* stream) {
  CLEAR_ERROR();
  if (!chi) { set_error("chi is NULL"); return VIE_ERR_ARG; }
  if (!adjoint)
    return run_matvec(op, w, out, B, path, precision, 0, EPI_SUB | EPI_CHI, chi, w, stream);
  return run_matvec(op, w, out, B, path, precision, PRO_CONJ | PRO_CHI, EPI_CONJ | EPI_SUB, chi, w,
                    stream);
}

int vie_total_field(const vie_op* op, const void* einc, const void* w, void* E, int B, int path,
                    int precision, void* stream) {
  CLEAR_ERROR();
  if (!einc) { set_error("einc is NULL"); return VIE_ERR_ARG; }
  return run_matvec(op, w, E, B, path, precision, 0, EPI_ADD, nullptr, einc, stream);
}

int vie_solve(const vie_op* op, const void* chi, const void* rhs, void* w, int B, int flags,
              int precision, const vie_solve_opts* opts, vie_solve_info* info, void* stream) {
  CLEAR_ERROR();
  VIE_TRY(check_op(op, B));
  if (!chi || !rhs || !w || !opts) { set_error("NULL argument"); return VIE_ERR_ARG; }
  VIE_TRY(check_prec_path(precision, opts->path, op));
  if (flags & ~(VIE_SOLVE_ADJOINT | VIE_SOLVE_RHS_INCIDENT | VIE_SOLVE_X0)) {
    set_error("unknown solve flags 0x%x", flags);
    return VIE_ERR_ARG;
  }
  if (opts->restart < 1 || opts->restart > 128 || opts->max_outer < 1 || opts->max_refine < 0 ||
      opts->max_refine > 64 || !(opts->tol > 0.0) || !(opts->inner_tol > 0.0) ||
      (opts->orth != 1 && opts->orth != 2)) {
    set_error("invalid solve options");
    return VIE_ERR_ARG;
  }
  vie_solve_info local;
  return solve_impl(op, chi, rhs, w, B, flags, precision, opts, info ? info : &local,
                    static_cast<cudaStream_t>(stream));
}

int vie_solve_multi(const vie_op* const* ops, const void* const* chi, const void* const* rhs,
                    void* const* w, const int* B, int count, int flags, int precision,
                    const vie_solve_opts* opts, vie_solve_info* info, void* stream) {
  CLEAR_ERROR();
  if (!ops || !chi || !rhs || !w || !B || count < 1 || !opts) {
    set_error("NULL argument or empty problem list");
    return VIE_ERR_ARG;
  }
  for (int p = 0; p < count; ++p) {
    for (int q = 0; q < p; ++q)
      if (ops[q] == ops[p]) {
        set_error("problems %d and %d share an operator", q, p);
        return VIE_ERR_ARG;
      }
  }
  if (count == 1)
    return vie_solve(ops[0], chi[0], rhs[0], w[0], B[0], flags, precision, opts,
                     info ? &info[0] : nullptr, stream);
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::vector<int> status(count, VIE_OK);
  std::vector<std::string> message(count);
  std::vector<std::thread> threads;
  threads.reserve(count);
  for (int p = 0; p < count; ++p) {
    threads.emplace_back([&, p]() {
      cudaSetDevice(dev);
      status[p] = vie_solve(ops[p], chi[p], rhs[p], w[p], B[p], flags, precision, opts,
                            info ? &info[p] : nullptr, stream);
      if (status[p] != VIE_OK) message[p] = vie_last_error();
    });
  }
  for (std::thread& t : threads) t.join();
  for (int p = 0; p < count; ++p) {
    if (status[p] != VIE_OK) {
      set_error("problem %d: %s", p, message[p].c_str());
      return status[p];
    }
  }
  return VIE_OK;
}

int vie_contrast_gradient(const vie_op* op, const void* lam, const void* E, void* grad, int B,
                          double scale, int precision, void* stream) {
  CLEAR_ERROR();
  VIE_TRY(check_op(op, B));
  if (!lam || !E || !grad) { set_error("NULL array"); return VIE_ERR_ARG; }
  const long long nvox = (long long)op->n[0] * op->n[1] * op->n[2];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == VIE_C64)
    return launch_gradient<float>(static_cast<const float2*>(lam), static_cast<const float2*>(E),
                                  static_cast<float2*>(grad), B, scale, nvox, s);
  if (precision == VIE_C128)
    return launch_gradient<double>(static_cast<const double2*>(lam), static_cast<const double2*>(E),
                                   static_cast<double2*>(grad), B, scale, nvox, s);
  set_error("precision must be VIE_C64 or VIE_C128");
  return VIE_ERR_ARG;
}

int vie_incident_dipole(const vie_op* op, const double* sources, int B, void* out, int precision,
                        void* stream) {
  CLEAR_ERROR();
  VIE_TRY(check_op(op, B));
  if (!sources || !out) { set_error("NULL argument"); return VIE_ERR_ARG; }
  // a source exactly at a voxel centre would divide by zero
  const double h = op->grid.h;
  for (int b = 0; b < B; ++b) {
    bool at_centre = true;
    for (int q = 0; q < 3; ++q) {
      const double u = sources[3 * b + q] / h + 0.5 * op->n[q] - 0.5;   // voxel index if integral
      const double ui = std::nearbyint(u);
      if (std::fabs(u - ui) > 1e-9 || ui < 0 || ui >= op->n[q]) at_centre = false;
    }
    if (at_centre) {
      set_error("dipole %d sits at a voxel centre", b);
      return VIE_ERR_ARG;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dsrc = nullptr;
  VIE_CUDA(cudaMallocAsync(&dsrc, 3 * B * sizeof(double), s));
  VIE_CUDA(cudaMemcpyAsync(dsrc, sources, 3 * B * sizeof(double), cudaMemcpyHostToDevice, s));
  int st;
  if (precision == VIE_C64)
    st = launch_dipole<float>(op, dsrc, B, static_cast<float2*>(out), s);
  else if (precision == VIE_C128)
    st = launch_dipole<double>(op, dsrc, B, static_cast<double2*>(out), s);
  else {
    set_error("precision must be VIE_C64 or VIE_C128");
    st = VIE_ERR_ARG;
  }
  cudaFreeAsync(dsrc, s);
  cudaError_t e = cudaStreamSynchronize(s);   // the host `sources` may be released on return
  if (st == VIE_OK && e != cudaSuccess) st = cuda_status(e, "dipole");
  return st;
}

void vie_destroy(vie_op* op) {
  if (!op) return;
  solver_release(op);
  if (op->rb_stream) {
    cudaStreamSynchronize(op->rb_stream);
    cudaStreamDestroy(op->rb_stream);
  }
  if (op->rb_fork) cudaEventDestroy(op->rb_fork);
  if (op->rb_join) cudaEventDestroy(op->rb_join);
  for (int c = 0; c < 6; ++c) {
    TuckerComp& tc = op->comp[c];
    cudaFree(tc.core32);
    cudaFree(tc.core64);
    for (int q = 0; q < 3; ++q) {
      cudaFree(tc.U32[q]);
      cudaFree(tc.U64[q]);
    }
    cudaFree(tc.U3t32);
  }
  cudaFree(op->slab32);
  cudaFree(op->slab64);
  cudaFree(op->oct32);
  cudaFree(op->u3frag);
  free_cp(op);
  cudaFree(op->spec32);
  cudaFree(op->spec64);
  for (int q = 0; q < 3; ++q) {
    cudaFree(op->roots32[q]);
    cudaFree(op->roots64[q]);
  }
  cudaFree(op->meta);
  cudaFree(op->dev_err);
  cudaFree(op->ws.ptr);
  cudaFree(op->solve_ws.ptr);
  delete op;
}

const char* vie_status_string(int status) {
  switch (status) {
    case VIE_OK: return "ok";
    case VIE_ERR_ARG: return "invalid argument";
    case VIE_ERR_CUDA: return "CUDA error";
    case VIE_ERR_OOM: return "out of memory";
    case VIE_ERR_NO_CONVERGENCE: return "no convergence";
    case VIE_ERR_NUMERIC: return "numerical failure";
    case VIE_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* vie_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
