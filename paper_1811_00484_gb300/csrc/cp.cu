// Tucker+CP (Algorithm 2, eq. (17)) on the device.
//
// A CP model with R terms, core_c ~ sum_l V1[:, l] o V2[:, l] o V3[:, l], is
// fitted to each of the six HOSVD cores by alternating least squares, in FP64
// with one CTA per component.  A sweep updates V1, V2, V3 in turn; the update
// of mode q solves the normal equations of its linear least-squares problem,
//   (P^H P) V_q[i, :]^T = P^H G_(q)[i, :]^T,   P = Khatri-Rao of the other two,
// where P^H P = (Vx^H Vx) o (Vy^H Vy) (Hadamard) and P^H G_(q)^T is the
// "matricised tensor times Khatri-Rao product", by a Cholesky factorisation.
// The relative error ||G - CP||_F / ||G||_F is evaluated entry by entry after
// every sweep; the sweeps stop when it changes by less than `tol`.
//
// The Tucker+CP factors W^q = U^q V^q are then formed for the stored half
// factors (rows P_q - k follow from row k by the same parity sign as U^q), in
// FP64 and FP32, with W3 transposed and in the tensor cores' fragment order
// for the per-matvec rebuild (octant_cp_kernel).
#include <cmath>
#include <cstring>
#include <vector>

#include "vie_internal.cuh"

namespace {

constexpr int kAlsThreads = 256;
constexpr int kMaxTucker = 64;          // Tucker ranks the ALS kernel stages

struct AlsArgs {
  const double2* core[6];               // [r1][r2][r3]
  int r[6][3];
  int R, max_iter;
  double tol;
  unsigned long long seed;
  double2* V;                           // [6][3][kMaxTucker][R]
  double* err;                          // [6] final relative error
  int* sweeps;                          // [6]
};

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// seeded start: re and im uniform in [-1, 1)
__device__ double2 start_value(unsigned long long seed, int c, int q, int i, int l) {
  const unsigned long long key =
      seed ^ ((unsigned long long)c << 56) ^ ((unsigned long long)q << 48) ^ ((unsigned long long)i << 24) ^
      (unsigned long long)l;
  const unsigned long long a = splitmix64(key), b = splitmix64(a);
  return make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kAlsThreads / 32; ++w) s += red[w];
  return s;
}

// Gram matrix V^H V of a [rows][R] factor
__device__ void gram(const double2* V, int rows, int R, double2* out) {
  for (int o = threadIdx.x; o < R * R; o += kAlsThreads) {
    const int l = o / R, m = o - l * R;
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < rows; ++i) s = conj_madd(V[i * R + l], V[i * R + m], s);
    out[o] = s;
  }
}

__global__ void __launch_bounds__(kAlsThreads) cp_als_kernel(const AlsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x, R = a.R;
  const int r[3] = {a.r[c][0], a.r[c][1], a.r[c][2]};
  const int st[3] = {r[1] * r[2], r[2], 1};        // strides of core[a][b][c]
  const int total = r[0] * r[1] * r[2];
  const double2* G = a.core[c];
  double2* V[3];
  V[0] = reinterpret_cast<double2*>(smem_raw);
  V[1] = V[0] + kMaxTucker * R;
  V[2] = V[1] + kMaxTucker * R;
  double2* Gm[3] = {V[2] + kMaxTucker * R, nullptr, nullptr};
  Gm[1] = Gm[0] + R * R;
  Gm[2] = Gm[1] + R * R;
  double2* A = Gm[2] + R * R;                       // normal matrix, then its Cholesky factor
  double2* N = A + R * R;                           // right-hand sides [r_q][R]
  __shared__ double red[kAlsThreads / 32];
  __shared__ double s_prev;
  __shared__ int s_stop;
  for (int q = 0; q < 3; ++q)
    for (int o = threadIdx.x; o < r[q] * R; o += kAlsThreads)
      V[q][o] = start_value(a.seed, c, q, o / R, o % R);
  double g2 = 0.0;
  for (int o = threadIdx.x; o < total; o += kAlsThreads) g2 += abs2(G[o]);
  g2 = block_sum(g2, red);
  for (int q = 0; q < 3; ++q) gram(V[q], r[q], R, Gm[q]);
  if (threadIdx.x == 0) {
    s_prev = -1.0;
    s_stop = 0;
  }
  __syncthreads();
  int sweep = 0;
  double err = 1.0;
  for (; sweep < a.max_iter && !s_stop; ++sweep) {
    for (int q = 0; q < 3; ++q) {
      const int x = q == 0 ? 1 : 0, y = q == 2 ? 1 : 2;
      // A = (Vx^H Vx) o (Vy^H Vy) + delta I
      for (int o = threadIdx.x; o < R * R; o += kAlsThreads) A[o] = Gm[x][o] * Gm[y][o];
      __syncthreads();
      if (threadIdx.x == 0) {
        double dmax = 0.0;
        for (int l = 0; l < R; ++l) dmax = fmax(dmax, A[l * R + l].x);
        const double delta = 1e-13 * dmax + 1e-300;
        for (int l = 0; l < R; ++l) A[l * R + l].x += delta;
      }
      // N[i][l] = sum_{x, y} G_(q)[i, (x, y)] conj(Vx[x, l] Vy[y, l])
      for (int o = threadIdx.x; o < r[q] * R; o += kAlsThreads) {
        const int i = o / R, l = o - i * R;
        double2 acc = make_double2(0.0, 0.0);
        for (int xi = 0; xi < r[x]; ++xi) {
          const double2* g = G + i * st[q] + xi * st[x];
          double2 t = make_double2(0.0, 0.0);
          for (int yi = 0; yi < r[y]; ++yi) t = conj_madd(V[y][yi * R + l], g[yi * st[y]], t);
          acc = conj_madd(V[x][xi * R + l], t, acc);
        }
        N[o] = acc;
      }
      __syncthreads();
      // Cholesky A = L L^H in place (lower triangle)
      for (int j = 0; j < R; ++j) {
        if (threadIdx.x == 0) {
          double d = A[j * R + j].x;
          for (int k = 0; k < j; ++k) d -= abs2(A[j * R + k]);
          A[j * R + j] = make_double2(sqrt(fmax(d, 1e-300)), 0.0);
        }
        __syncthreads();
        const double ljj = A[j * R + j].x;
        for (int i = j + 1 + threadIdx.x; i < R; i += kAlsThreads) {
          double2 s = A[i * R + j];
          for (int k = 0; k < j; ++k) s = s - A[i * R + k] * conjg(A[j * R + k]);
          A[i * R + j] = (1.0 / ljj) * s;
        }
        __syncthreads();
      }
      // each row i: L z = N[i, :]^T, L^H v = z, V_q[i, :] = v^T
      for (int i = threadIdx.x; i < r[q]; i += kAlsThreads) {
        double2* z = N + i * R;
        for (int k = 0; k < R; ++k) {
          double2 s = z[k];
          for (int m = 0; m < k; ++m) s = s - A[k * R + m] * z[m];
          z[k] = (1.0 / A[k * R + k].x) * s;
        }
        for (int k = R - 1; k >= 0; --k) {
          double2 s = z[k];
          for (int m = k + 1; m < R; ++m) s = s - conjg(A[m * R + k]) * z[m];
          z[k] = (1.0 / A[k * R + k].x) * s;
        }
        for (int k = 0; k < R; ++k) V[q][i * R + k] = z[k];
      }
      __syncthreads();
      // unit columns for the first two factors (the third carries the scale)
      if (q < 2) {
        for (int l = threadIdx.x; l < R; l += kAlsThreads) {
          double s = 0.0;
          for (int i = 0; i < r[q]; ++i) s += abs2(V[q][i * R + l]);
          const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
          for (int i = 0; i < r[q]; ++i) V[q][i * R + l] = inv * V[q][i * R + l];
        }
        __syncthreads();
      }
      gram(V[q], r[q], R, Gm[q]);
      __syncthreads();
    }
    // ||G - CP||^2, entry by entry
    double e2 = 0.0;
    for (int o = threadIdx.x; o < total; o += kAlsThreads) {
      const int ia = o / st[0], ib = (o - ia * st[0]) / st[1], ic = o - ia * st[0] - ib * st[1];
      double2 m = make_double2(0.0, 0.0);
      for (int l = 0; l < R; ++l) m = cmadd(V[0][ia * R + l] * V[1][ib * R + l], V[2][ic * R + l], m);
      e2 += abs2(G[o] - m);
    }
    e2 = block_sum(e2, red);
    err = g2 > 0.0 ? sqrt(e2 / g2) : 0.0;
    if (threadIdx.x == 0) {
      if (!(err == err) || (s_prev >= 0.0 && fabs(s_prev - err) < a.tol)) s_stop = 1;
      s_prev = err;
    }
    __syncthreads();
  }
  for (int q = 0; q < 3; ++q)
    for (int o = threadIdx.x; o < r[q] * R; o += kAlsThreads)
      a.V[((long long)c * 3 + q) * kMaxTucker * R + o] = V[q][o];
  if (threadIdx.x == 0) {
    a.err[c] = err;
    a.sweeps[c] = sweep;
  }
}

// W^q = U^q V^q for the stored half rows, FP64 and FP32; W3 also transposed
// ([R][H3], FP32).  One CTA per (component, mode).
__global__ void cp_factor_kernel(const double2* const* U64, const int* rq, const double2* V, int R,
                                 const int* H, double2* const* W64, float2* const* W32,
                                 float2* const* W3t) {
  const int c = blockIdx.x / 3, q = blockIdx.x % 3;
  const int h = H[q], r = rq[c * 3 + q];
  const double2* U = U64[c * 3 + q];
  const double2* Vq = V + ((long long)c * 3 + q) * kMaxTucker * R;
  for (int o = threadIdx.x; o < h * R; o += blockDim.x) {
    const int k = o / R, l = o - k * R;
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < r; ++j) s = cmadd(U[(long long)k * r + j], Vq[j * R + l], s);
    W64[c * 3 + q][o] = s;
    const float2 f = make_float2((float)s.x, (float)s.y);
    W32[c * 3 + q][o] = f;
    if (q == 2) W3t[c][(long long)l * h + k] = f;
  }
}

}  // namespace

void free_cp(vie_op* op) {
  for (int c = 0; c < 6; ++c)
    for (int q = 0; q < 3; ++q) {
      cudaFree(op->cp.W64[c][q]);
      cudaFree(op->cp.W32[c][q]);
      op->cp.W64[c][q] = nullptr;
      op->cp.W32[c][q] = nullptr;
    }
  for (int c = 0; c < 6; ++c) {
    cudaFree(op->cp.W3t32[c]);
    op->cp.W3t32[c] = nullptr;
  }
  cudaFree(op->cp.meta);
  cudaFree(op->cp.frag);
  op->cp.meta = nullptr;
  op->cp.frag = nullptr;
  op->cp.R = 0;
  ++op->cp.epoch;          // solver graphs captured with the old buffers are rebuilt
}

template <typename P> static int cp_alloc(P** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("out of device memory (%zu bytes)", bytes);
    return VIE_ERR_OOM;
  }
  return VIE_OK;
}

static int tucker_cp_impl(vie_op* op, int R, double tol, int max_iter, unsigned long long seed,
                          cudaStream_t s) {
  for (int c = 0; c < 6; ++c)
    for (int q = 0; q < 3; ++q)
      if (op->comp[c].r[q] > kMaxTucker) {
        set_error("Tucker rank %d above %d (component %d): the ALS kernel stages at most %d rows",
                  op->comp[c].r[q], kMaxTucker, c, kMaxTucker);
        return VIE_ERR_ARG;
      }
  // work of any stream may still read the model being replaced
  VIE_CUDA(cudaDeviceSynchronize());
  free_cp(op);
  // ALS
  AlsArgs a;
  for (int c = 0; c < 6; ++c) {
    a.core[c] = op->comp[c].core64;
    for (int q = 0; q < 3; ++q) a.r[c][q] = op->comp[c].r[q];
  }
  a.R = R;
  a.max_iter = max_iter;
  a.tol = tol;
  a.seed = seed;
  double2* V = nullptr;
  double* err = nullptr;
  int* sweeps = nullptr;
  int arc = cp_alloc(&V, (size_t)6 * 3 * kMaxTucker * R * sizeof(double2));
  if (arc == VIE_OK) arc = cp_alloc(&err, 6 * sizeof(double));
  if (arc == VIE_OK) arc = cp_alloc(&sweeps, 6 * sizeof(int));
  if (arc != VIE_OK) {
    cudaFree(V);
    cudaFree(err);
    return arc;
  }
  VIE_CUDA(cudaMemsetAsync(V, 0, (size_t)6 * 3 * kMaxTucker * R * sizeof(double2), s));
  a.V = V;
  a.err = err;
  a.sweeps = sweeps;
  const size_t smem = ((size_t)3 * kMaxTucker * R + 4 * R * R + (size_t)kMaxTucker * R) * sizeof(double2);
  int rc = VIE_OK;
  cudaError_t e = cudaFuncSetAttribute(cp_als_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    cp_als_kernel<<<6, kAlsThreads, smem, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = cuda_status(e, "CP-ALS");
  double herr[6] = {};
  int hsw[6] = {};
  if (rc == VIE_OK) {
    e = cudaMemcpy(herr, err, sizeof(herr), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hsw, sweeps, sizeof(hsw), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_status(e, "CP-ALS results");
  }
  for (int c = 0; c < 6 && rc == VIE_OK; ++c)
    if (!(herr[c] == herr[c])) {
      set_error("CP-ALS of component %d did not stay finite", c);
      rc = VIE_ERR_NUMERIC;
    }
  // W^q = U^q V^q
  if (rc == VIE_OK) {
    for (int c = 0; c < 6 && rc == VIE_OK; ++c)
      for (int q = 0; q < 3 && rc == VIE_OK; ++q) {
        rc = cp_alloc(&op->cp.W64[c][q], (size_t)op->H[q] * R * sizeof(double2));
        if (rc == VIE_OK) rc = cp_alloc(&op->cp.W32[c][q], (size_t)op->H[q] * R * sizeof(float2));
      }
    for (int c = 0; c < 6 && rc == VIE_OK; ++c)
      rc = cp_alloc(&op->cp.W3t32[c], (size_t)op->H[2] * R * sizeof(float2));
  }
  if (rc == VIE_OK) {
    std::vector<const double2*> U(18);
    std::vector<int> rq(18), H(3);
    std::vector<double2*> w64(18);
    std::vector<float2*> w32(18), w3t(6);
    for (int c = 0; c < 6; ++c) {
      for (int q = 0; q < 3; ++q) {
        U[c * 3 + q] = op->comp[c].U64[q];
        rq[c * 3 + q] = op->comp[c].r[q];
        w64[c * 3 + q] = op->cp.W64[c][q];
        w32[c * 3 + q] = op->cp.W32[c][q];
      }
      w3t[c] = op->cp.W3t32[c];
    }
    for (int q = 0; q < 3; ++q) H[q] = op->H[q];
    // one staging buffer for the pointer and size tables
    const size_t bytes = 18 * sizeof(void*) * 3 + 6 * sizeof(void*) + 21 * sizeof(int);
    char* tab = nullptr;
    rc = cp_alloc(&tab, bytes);
    if (rc == VIE_OK) {
      std::vector<char> host(bytes);
      char* p = host.data();
      memcpy(p, U.data(), 18 * sizeof(void*));
      memcpy(p + 18 * sizeof(void*), w64.data(), 18 * sizeof(void*));
      memcpy(p + 36 * sizeof(void*), w32.data(), 18 * sizeof(void*));
      memcpy(p + 54 * sizeof(void*), w3t.data(), 6 * sizeof(void*));
      memcpy(p + 60 * sizeof(void*), rq.data(), 18 * sizeof(int));
      memcpy(p + 60 * sizeof(void*) + 18 * sizeof(int), H.data(), 3 * sizeof(int));
      e = cudaMemcpy(tab, host.data(), bytes, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        cp_factor_kernel<<<18, 256, 0, s>>>(
            reinterpret_cast<const double2* const*>(tab), reinterpret_cast<const int*>(tab + 60 * sizeof(void*)),
            V, R, reinterpret_cast<const int*>(tab + 60 * sizeof(void*) + 18 * sizeof(int)),
            reinterpret_cast<double2* const*>(tab + 18 * sizeof(void*)),
            reinterpret_cast<float2* const*>(tab + 36 * sizeof(void*)),
            reinterpret_cast<float2* const*>(tab + 54 * sizeof(void*)));
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_status(e, "Tucker+CP factors");
      cudaFree(tab);
    }
  }
  if (rc == VIE_OK) {
    op->cp.R = R;
    for (int c = 0; c < 6; ++c) {
      op->cp.err[c] = herr[c];
      op->cp.sweeps[c] = hsw[c];
    }
    rc = build_cp_rebuild(op, s);
  }
  cudaFree(V);
  cudaFree(err);
  cudaFree(sweeps);
  if (rc != VIE_OK) free_cp(op);
  return rc;
}

extern "C" int vie_tucker_cp(vie_op* op, int rank, double tol, int max_iter, unsigned long long seed,
                             void* stream) {
  clear_error();
  if (!op) { set_error("operator is NULL"); return VIE_ERR_ARG; }
  if (rank < 1 || rank > kCpMaxRank) {
    set_error("CP rank %d outside [1, %d]", rank, kCpMaxRank);
    return VIE_ERR_ARG;
  }
  if (!(tol >= 0.0) || max_iter < 1 || max_iter > 100000) {
    set_error("tol must be >= 0 and max_iter in [1, 100000]");
    return VIE_ERR_ARG;
  }
  if (op->oct32 == nullptr) {
    set_error("Tucker+CP needs the rebuild scratch (grid edge P3 = 32 R with a four-step or "
              "register FFT)");
    return VIE_ERR_ARG;
  }
  return tucker_cp_impl(op, rank, tol, max_iter, seed, static_cast<cudaStream_t>(stream));
}

extern "C" int vie_cp_export(const vie_op* op, int c, double* W1, double* W2, double* W3,
                             double* rel_err, int* sweeps, void* stream) {
  clear_error();
  if (!op || c < 0 || c > 5) { set_error("bad operator or component"); return VIE_ERR_ARG; }
  if (op->cp.R == 0) { set_error("no Tucker+CP model: call vie_tucker_cp first"); return VIE_ERR_ARG; }
  VIE_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  const int R = op->cp.R;
  double* W[3] = {W1, W2, W3};
  for (int q = 0; q < 3; ++q) {
    if (!W[q]) continue;
    const int H = op->H[q], P = op->P[q];
    std::vector<double2> half((size_t)H * R);
    VIE_CUDA(cudaMemcpy(half.data(), op->cp.W64[c][q], half.size() * sizeof(double2),
                        cudaMemcpyDeviceToHost));
    double2* dst = reinterpret_cast<double2*>(W[q]);
    for (int k = 0; k < P; ++k) {
      const bool mirror = 2 * k > P;
      const int src = mirror ? P - k : k;
      const double sg = mirror ? (double)op->comp[c].s[q] : 1.0;
      for (int l = 0; l < R; ++l) {
        const double2 v = half[(size_t)src * R + l];
        dst[(size_t)k * R + l] = make_double2(sg * v.x, sg * v.y);
      }
    }
  }
  if (rel_err) *rel_err = op->cp.err[c];
  if (sweeps) *sweeps = op->cp.sweeps[c];
  return VIE_OK;
}
