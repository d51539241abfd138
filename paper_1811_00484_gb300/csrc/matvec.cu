// Host orchestration of the FFT-based matvec (Section V.B):
//
//   J [B][3][n1][n2][n3]
//     -- x-FFT, zero-padded n1 -> P1 -->            T1 [B][3][P1][n2][n3]
//     -- y-FFT, zero-padded n2 -> P2 -->            T2 [B][3][P1][P2][n3]
//     -- fused: z-FFT n3 -> P3, rebuild + product,
//        inverse z-FFT cropped P3 -> n3 -->         T2 (in place)
//     -- inverse y-FFT, cropped P2 -> n2 -->        T1
//     -- inverse x-FFT, cropped P1 -> n1, scaled
//        by 1/(P1 P2 P3), optional epilogue -->    Y [B][3][n1][n2][n3]
//
// Lines that are entirely zero padding are never transformed: the x stage
// runs n2 n3 lines, the y stage P1 n3 lines.
#include "vie_internal.cuh"

template <typename T>
int launch_fused(const vie_op* op, cx<T>* data, int B, bool stored, const int* active,
                 cudaStream_t s, bool first_chunk_ready, bool cp);

size_t workspace_bytes_for(const vie_op* op, int B, size_t elem) {
  const size_t n1 = op->n[0], n2 = op->n[1], n3 = op->n[2];
  const size_t P1 = op->P[0], P2 = op->P[1];
  (void)n1;
  const size_t per = 3 * (P1 * n2 * n3 + P1 * P2 * n3);   // T1 + T2 elements per RHS
  return per * (size_t)B * elem;
}

int ensure_workspace_bytes(vie_op* op, size_t need) {
  if (op->ws.bytes >= need) return VIE_OK;
  if (op->ws.ptr) {
    cudaDeviceSynchronize();
    cudaFree(op->ws.ptr);
    op->ws.ptr = nullptr;
    op->ws.bytes = 0;
    op->ws_batch = 0;
  }
  cudaError_t e = cudaMalloc(&op->ws.ptr, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("workspace allocation of %zu bytes failed", need);
    return VIE_ERR_OOM;
  }
  op->ws.bytes = need;
  op->ws_batch = (int)(need / workspace_bytes_for(op, 1, sizeof(float2)));
  return VIE_OK;
}

int ensure_workspace(vie_op* op, int B, size_t elem) {
  return ensure_workspace_bytes(op, workspace_bytes_for(op, B, elem));
}

// Arguments of the four line stages for one operator and batch, T1 then T2 in `ws`.
template <typename T>
LineStages<T> make_line_stages(const vie_op* op, void* ws, const cx<T>* in, cx<T>* out, int B,
                               int pro_flags, int epi_flags, const cx<T>* chi, const cx<T>* addend,
                               const int* active, const double* rscale, long long rscale_stride) {
  using C = cx<T>;
  const long long n1 = op->n[0], n2 = op->n[1], n3 = op->n[2];
  const long long P1 = op->P[0], P2 = op->P[1], P3 = op->P[2];
  C* T1 = static_cast<C*>(ws);
  C* T2 = T1 + (size_t)B * 3 * P1 * n2 * n3;
  const C* r[3];
  for (int q = 0; q < 3; ++q) {
    if constexpr (sizeof(T) == 4) r[q] = op->roots32[q]; else r[q] = op->roots64[q];
  }
  LineStages<T> st = {};
  // x stage: J -> T1
  {
    LineArgs<T>& a = st.s[0];
    a.in = in;
    a.out = T1;
    a.roots = r[0];
    a.chi = chi;
    a.plan = op->plan[0];
    a.lin = (int)n1;
    a.lout = (int)P1;
    a.inverse = 0;
    a.scale = (T)1;
    a.flags = pro_flags & (PRO_CONJ | PRO_CHI);
    if (rscale) a.flags |= PRO_RSCALE;
    a.nbatch = 3 * B;
    a.nother = (int)n2;
    a.ncol = (int)n3;
    a.in_bs = n1 * n2 * n3; a.in_os = n3; a.in_ls = n2 * n3; a.in_cs = 1;
    a.out_bs = P1 * n2 * n3; a.out_os = n3; a.out_ls = n2 * n3; a.out_cs = 1;
    a.chi_os = n3; a.chi_ls = n2 * n3; a.chi_cs = 1;
    a.prof_family = PF_LINE_X;
    a.prof_batch_bytes = (unsigned long long)((n1 + P1) * n2 * n3 * sizeof(C)) +
                         ((a.flags & PRO_CHI) ? (unsigned long long)(n1 * n2 * n3 * sizeof(C)) : 0ull);
  }
  // y stage: T1 -> T2
  {
    LineArgs<T>& a = st.s[1];
    a.in = T1;
    a.out = T2;
    a.roots = r[1];
    a.plan = op->plan[1];
    a.lin = (int)n2;
    a.lout = (int)P2;
    a.scale = (T)1;
    a.nbatch = 3 * B;
    a.nother = (int)P1;
    a.ncol = (int)n3;
    a.in_bs = P1 * n2 * n3; a.in_os = n2 * n3; a.in_ls = n3; a.in_cs = 1;
    a.out_bs = P1 * P2 * n3; a.out_os = P2 * n3; a.out_ls = n3; a.out_cs = 1;
    a.prof_family = PF_LINE_Y;
    a.prof_batch_bytes = (unsigned long long)((n2 + P2) * P1 * n3 * sizeof(C));
  }
  // inverse y stage: T2 -> T1 (crop)
  {
    LineArgs<T>& a = st.s[2];
    a.in = T2;
    a.out = T1;
    a.roots = r[1];
    a.plan = op->plan[1];
    a.lin = (int)P2;
    a.lout = (int)n2;
    a.inverse = 1;
    a.scale = (T)1;
    a.nbatch = 3 * B;
    a.nother = (int)P1;
    a.ncol = (int)n3;
    a.in_bs = P1 * P2 * n3; a.in_os = P2 * n3; a.in_ls = n3; a.in_cs = 1;
    a.out_bs = P1 * n2 * n3; a.out_os = n2 * n3; a.out_ls = n3; a.out_cs = 1;
    a.prof_family = PF_LINE_IY;
    a.prof_batch_bytes = (unsigned long long)((n2 + P2) * P1 * n3 * sizeof(C));
  }
  // inverse x stage: T1 -> out (crop, scale, epilogue)
  {
    LineArgs<T>& a = st.s[3];
    a.in = T1;
    a.out = out;
    a.roots = r[0];
    a.chi = chi;
    a.addend = addend;
    a.plan = op->plan[0];
    a.lin = (int)P1;
    a.lout = (int)n1;
    a.inverse = 1;
    a.scale = (T)(1.0 / ((double)P1 * (double)P2 * (double)P3));
    a.flags = epi_flags & (EPI_CONJ | EPI_SUB | EPI_ADD | EPI_CHI);
    if (rscale && (a.flags & (EPI_SUB | EPI_ADD))) a.flags |= EPI_RSCALE;
    a.nbatch = 3 * B;
    a.nother = (int)n2;
    a.ncol = (int)n3;
    a.in_bs = P1 * n2 * n3; a.in_os = n3; a.in_ls = n2 * n3; a.in_cs = 1;
    a.out_bs = n1 * n2 * n3; a.out_os = n3; a.out_ls = n2 * n3; a.out_cs = 1;
    a.chi_os = n3; a.chi_ls = n2 * n3; a.chi_cs = 1;
    a.prof_family = PF_LINE_IX;
    a.prof_batch_bytes = (unsigned long long)((P1 + n1) * n2 * n3 * sizeof(C)) +
                         ((a.flags & (EPI_SUB | EPI_ADD)) ? (unsigned long long)(n1 * n2 * n3 * sizeof(C)) : 0ull) +
                         ((a.flags & EPI_CHI) ? (unsigned long long)(n1 * n2 * n3 * sizeof(C)) : 0ull);
  }
  for (int i = 0; i < 4; ++i) {
    st.s[i].batch_per_rhs = 3;
    st.s[i].active = active;
    st.s[i].threads = op->tune.line_threads[i];
    st.s[i].rscale = rscale;
    st.s[i].rscale_stride = rscale_stride;
    st.s[i].err = op->dev_err;
    // the FP64 stages (refinement residuals) form one family of their own: they
    // are bound by FP64 arithmetic, and count no algorithmic bytes
    if constexpr (sizeof(T) == 8) {
      st.s[i].prof_family = PF_MATVEC64;
      st.s[i].prof_batch_bytes = 0;
    }
  }
  return st;
}

// Rebuild the scratch for the next FP32 Tucker matvec on the side stream, ordered
// after the work already on s (the fused kernel that last read the scratch).
int prefetch_rebuild(const vie_op* op, cudaStream_t s, bool cp) {
  if (op->oct32 == nullptr || op->rb_stream == nullptr) return VIE_OK;
  VIE_CUDA(cudaEventRecord(op->rb_fork, s));
  VIE_CUDA(cudaStreamWaitEvent(op->rb_stream, op->rb_fork, 0));
  VIE_TRY(launch_octant(op, 0, op->rb_stream, cp));
  VIE_CUDA(cudaEventRecord(op->rb_join, op->rb_stream));
  vie_op* opm = const_cast<vie_op*>(op);
  opm->rb_pending = true;
  opm->rb_cp = cp;
  return VIE_OK;
}

// The stages of one matvec with the caller-chosen scratch `ws` (T1 then T2).
template <typename T>
int matvec_run(const vie_op* op, void* ws, const cx<T>* in, cx<T>* out, int B, int path,
               int pro_flags, int epi_flags, const cx<T>* chi, const cx<T>* addend,
               const int* active, cudaStream_t s, const double* rscale, long long rscale_stride,
               int mv_flags) {
  using C = cx<T>;
  const bool stored = (path == VIE_PATH_UNCOMPRESSED);
  const bool cp = (path == VIE_PATH_TUCKER_CP);
  const LineStages<T> st = make_line_stages<T>(op, ws, in, out, B, pro_flags, epi_flags, chi,
                                               addend, active, rscale, rscale_stride);
  C* T2 = const_cast<C*>(st.s[1].out);
  // FP32 Tucker path on the register kernels: the first k1 chunk of the rebuild
  // does not read J, so it runs on the operator's side stream beside the x and
  // y stages and is joined before the fused kernel
  // (or it was started after the previous matvec's fused kernel: rb_pending)
  vie_op* opm = const_cast<vie_op*>(op);
  bool pre = false;
  const bool side = !stored && op->oct32 != nullptr && op->rb_stream != nullptr;
  if constexpr (sizeof(T) == 4) {
    // a pending rebuild of the other model is overwritten (same stream, in order)
    if (side && !(op->rb_pending && op->rb_cp == cp)) {
      VIE_CUDA(cudaEventRecord(op->rb_fork, s));
      VIE_CUDA(cudaStreamWaitEvent(op->rb_stream, op->rb_fork, 0));
      VIE_TRY(launch_octant(op, 0, op->rb_stream, cp));
      VIE_CUDA(cudaEventRecord(op->rb_join, op->rb_stream));
    }
    pre = side;
    if (side) opm->rb_pending = false;
  }
  launch_line_fft<T>(st.s[0], s);
  launch_line_fft<T>(st.s[1], s);
  if (pre) VIE_CUDA(cudaStreamWaitEvent(s, op->rb_join, 0));
  VIE_TRY(launch_fused<T>(op, T2, B, stored, active, s, pre, cp));
  launch_line_fft<T>(st.s[2], s);
  launch_line_fft<T>(st.s[3], s);
  if (pre && (mv_flags & MV_PREFETCH_REBUILD)) VIE_TRY(prefetch_rebuild(op, s, cp));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "matvec launch");
  return VIE_OK;
}

template <typename T>
int matvec_impl(const vie_op* op, const cx<T>* in, cx<T>* out, int B, int path, int pro_flags,
                int epi_flags, const cx<T>* chi, const cx<T>* addend, const int* active,
                cudaStream_t s, const double* rscale, long long rscale_stride, int mv_flags) {
  if (workspace_bytes_for(op, B, sizeof(cx<T>)) > op->ws.bytes) {
    VIE_TRY(ensure_workspace(const_cast<vie_op*>(op), B, sizeof(cx<T>)));
  }
  return matvec_run<T>(op, op->ws.ptr, in, out, B, path, pro_flags, epi_flags, chi, addend, active,
                       s, rscale, rscale_stride, mv_flags);
}

template int matvec_run<float>(const vie_op*, void*, const float2*, float2*, int, int, int, int,
                               const float2*, const float2*, const int*, cudaStream_t,
                               const double*, long long, int);
template LineStages<float> make_line_stages<float>(const vie_op*, void*, const float2*, float2*, int,
                                                   int, int, const float2*, const float2*,
                                                   const int*, const double*, long long);
template int matvec_impl<float>(const vie_op*, const float2*, float2*, int, int, int, int,
                                const float2*, const float2*, const int*, cudaStream_t,
                                const double*, long long, int);
template int matvec_impl<double>(const vie_op*, const double2*, double2*, int, int, int, int,
                                 const double2*, const double2*, const int*, cudaStream_t,
                                 const double*, long long, int);
