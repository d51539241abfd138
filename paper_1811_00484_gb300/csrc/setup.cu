// Setup of the compressed operator, all in FP64 on the device:
//   assembly of a defining tensor (eqs. (5)-(6)) directly in its circulant
//   embedding (Section V.A), 3-D FFT, and truncated HOSVD (Algorithm 1).
//
// HOSVD on the weighted octant.  The spectrum A of every component obeys
// A[.., P-k, ..] = s A[.., k, ..] along each axis (s = +-1), so row P-k of a
// mode unfolding is s times row k.  With E the P x H map that copies the H =
// P/2 + 1 distinct rows into all P rows (with signs) and D = diag(w),
// w_k = sqrt(2) for 0 < k < P/2 and 1 otherwise (E^H E = D^2):
//   * the unfolding of A has the same singular values as that of the
//     weighted octant A_w = A[0:H1, 0:H2, 0:H3] x1 D1 x2 D2 x3 D3;
//   * its left singular vectors are U = E D^-1 Y, Y those of A_w;
//   * the core A x1 U1^* x2 U2^* x3 U3^* equals A_w x1 Y1^* x2 Y2^* x3 Y3^*.
// So Algorithm 1 runs on an (P/2+1)^3 tensor, exactly, and only the H_q
// rows D^-1 Y of each factor are stored (the others follow by the sign).
//
// The singular vectors come from the Hermitian Gram matrix of each
// unfolding, diagonalised by parallel cyclic Jacobi.  Because forming the
// Gram matrix squares the singular values, a second pass re-forms the Gram
// matrix of Y^* A_w^(q) (rows nearly orthogonal, norms sigma_j) and
// diagonalises it again; Jacobi on that graded, nearly diagonal matrix
// gives the small singular values to high relative accuracy, which the
// 1e-8 truncation threshold needs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "vie_internal.cuh"
#include "warpfft.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ int circulant_offset(int i, int n, int P, bool* zero) {
  if (i < n) return i;
  if (i == n) { *zero = true; return 0; }
  return i - P;
}

// One component of h^3 (k0^2 delta_ab + d_a d_b) g at the voxel-centre offset,
// or the equivalent-sphere self term at zero offset, at every circulant index.
__global__ void assemble_kernel(double2* out, int ca, int cb, int n1, int n2, int n3, int P1,
                                int P2, int P3, double h, double k0, double2 self) {
  const long long total = (long long)P1 * P2 * P3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(idx % P3);
    const int i2 = (int)((idx / P3) % P2);
    const int i1 = (int)(idx / ((long long)P2 * P3));
    bool zero = false;
    const int o1 = circulant_offset(i1, n1, P1, &zero);
    const int o2 = circulant_offset(i2, n2, P2, &zero);
    const int o3 = circulant_offset(i3, n3, P3, &zero);
    double2 v = make_double2(0.0, 0.0);
    if (!zero) {
      if (o1 == 0 && o2 == 0 && o3 == 0) {
        if (ca == cb) v = self;
      } else {
        const double R[3] = {o1 * h, o2 * h, o3 * h};
        const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
        double sn, cs;
        sincos(k0 * r, &sn, &cs);
        const double inv4pir = 1.0 / (4.0 * kPi * r);
        const double2 g = make_double2(cs * inv4pir, -sn * inv4pir);   // exp(-i k0 r)/(4 pi r)
        const double ir = 1.0 / r;
        const double2 diag = make_double2(k0 * k0 - ir * ir, -k0 * ir);
        const double2 dyad = make_double2(-k0 * k0 + 3.0 * ir * ir, 3.0 * k0 * ir);
        const double rr = (R[ca] * ir) * (R[cb] * ir);
        double2 f = make_double2(dyad.x * rr, dyad.y * rr);
        if (ca == cb) f = f + diag;
        v = (h * h * h) * (g * f);
      }
    }
    out[idx] = v;
  }
}

// max |A[mirror] - s A| and max |A| over the tensor (non-negative doubles
// compare like their bit patterns).
__global__ void parity_check_kernel(const double2* A, int P1, int P2, int P3, int s1, int s2, int s3,
                                    unsigned long long* out) {
  const long long total = (long long)P1 * P2 * P3;
  double dev = 0.0, mx = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(idx % P3);
    const int i2 = (int)((idx / P3) % P2);
    const int i1 = (int)(idx / ((long long)P2 * P3));
    const double2 a = A[idx];
    const double s = (double)(s1 * s2 * s3);
    const int m1 = (P1 - i1) % P1, m2 = (P2 - i2) % P2, m3 = (P3 - i3) % P3;
    const double2 b = A[((long long)m1 * P2 + m2) * P3 + m3];
    dev = fmax(dev, sqrt(abs2(b - s * a)));
    mx = fmax(mx, sqrt(abs2(a)));
    // single-axis mirrors
    const double2 bx = A[((long long)m1 * P2 + i2) * P3 + i3];
    dev = fmax(dev, sqrt(abs2(bx - (double)s1 * a)));
    const double2 by = A[((long long)i1 * P2 + m2) * P3 + i3];
    dev = fmax(dev, sqrt(abs2(by - (double)s2 * a)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_down_sync(0xffffffffu, dev, o));
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __double_as_longlong(dev));
    atomicMax(out + 1, __double_as_longlong(mx));
  }
}

__global__ void octant_kernel(const double2* A, double2* Aw, int P1, int P2, int P3, int H1, int H2,
                              int H3) {
  const long long total = (long long)H1 * H2 * H3;
  const double r2 = 1.41421356237309504880;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k3 = (int)(idx % H3);
    const int k2 = (int)((idx / H3) % H2);
    const int k1 = (int)(idx / ((long long)H2 * H3));
    double w = 1.0;
    if (k1 != 0 && 2 * k1 != P1) w *= r2;
    if (k2 != 0 && 2 * k2 != P2) w *= r2;
    if (k3 != 0 && 2 * k3 != P3) w *= r2;
    Aw[idx] = w * A[((long long)k1 * P2 + k2) * P3 + k3];
  }
}

// Factor-wise route (Section V.A): the weighted octant of the Toeplitz defining
// tensor itself, T_w[i1, i2, i3] = w(i1) w(i2) w(i3) T_ab(i1 h, i2 h, i3 h) for
// offsets 0 <= i_q < n_q, w(0) = 1, w(i > 0) = sqrt(2) (offsets +i and -i
// hold the same entry up to the component's parity sign).
__global__ void toeplitz_octant_kernel(double2* out, int ca, int cb, int n1, int n2, int n3, double h,
                                       double k0, double2 self) {
  const long long total = (long long)n1 * n2 * n3;
  const double r2 = 1.41421356237309504880;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int o3 = (int)(idx % n3);
    const int o2 = (int)((idx / n3) % n2);
    const int o1 = (int)(idx / ((long long)n2 * n3));
    double2 v = make_double2(0.0, 0.0);
    if (o1 == 0 && o2 == 0 && o3 == 0) {
      if (ca == cb) v = self;
    } else {
      const double R[3] = {o1 * h, o2 * h, o3 * h};
      const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
      double sn, cs;
      sincos(k0 * r, &sn, &cs);
      const double inv4pir = 1.0 / (4.0 * kPi * r);
      const double2 g = make_double2(cs * inv4pir, -sn * inv4pir);
      const double ir = 1.0 / r;
      const double2 diag = make_double2(k0 * k0 - ir * ir, -k0 * ir);
      const double2 dyad = make_double2(-k0 * k0 + 3.0 * ir * ir, 3.0 * k0 * ir);
      const double rr = (R[ca] * ir) * (R[cb] * ir);
      double2 f = make_double2(dyad.x * rr, dyad.y * rr);
      if (ca == cb) f = f + diag;
      v = (h * h * h) * (g * f);
    }
    double w = 1.0;
    if (o1 != 0) w *= r2;
    if (o2 != 0) w *= r2;
    if (o3 != 0) w *= r2;
    out[idx] = w * v;
  }
}

// Rows k = 0 .. P/2 of the embedded, DFT'd factor, normalised to orthonormal
// columns: out[k][j] = P^-1/2 sum_{|i| < n} U[i][j] exp(-2 pi i k i / P), with
// U[-i] = s U[i] and the stored rows U[i], i = 0..n-1 (Uh [n][r]):
//   out[k][j] = P^-1/2 (U[0][j] + sum_{i >= 1} U[i][j] (w^{ki} + s conj(w^{ki}))).
__global__ void factor_dft_kernel(const double2* Uh, double2* out, const double2* roots, int n, int P,
                                  int r, int s) {
  const int total = (P / 2 + 1) * r;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int k = idx / r, j = idx % r;
    double2 acc = Uh[j];
    for (int i = 1; i < n; ++i) {
      const double2 w = roots[(int)(((long long)k * i) % P)];
      const double2 c = make_double2(w.x + s * w.x, w.y - s * w.y);
      acc = cmadd(Uh[(long long)i * r + j], c, acc);
    }
    const double sc = 1.0 / sqrt((double)P);
    out[idx] = make_double2(sc * acc.x, sc * acc.y);
  }
}

__global__ void to_c64_kernel(const double2* a, float2* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// element (i, m) of the mode-q unfolding of a D0 x D1 x D2 tensor
__device__ __forceinline__ long long unfold_index(int q, int i, long long m, int D1, int D2) {
  if (q == 0) return (long long)i * D1 * D2 + m;
  if (q == 1) return (m / D2) * (long long)D1 * D2 + (long long)i * D2 + (m % D2);
  return m * D2 + i;
}

// G = X X^* for the mode-q unfolding X (Dq x M), one 16 x 16 tile per CTA.
__global__ void __launch_bounds__(256) gram_kernel(const double2* X, double2* G, int q, int D0, int D1,
                                                   int D2) {
  __shared__ double2 Ai[16][17], Aj[16][17];
  const int Dq = q == 0 ? D0 : (q == 1 ? D1 : D2);
  const long long M = ((long long)D0 * D1 * D2) / Dq;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  double2 acc = make_double2(0.0, 0.0);
  for (long long m0 = 0; m0 < M; m0 += 16) {
    const long long m = m0 + tx;
    Ai[ty][tx] = (i0 + ty < Dq && m < M) ? X[unfold_index(q, i0 + ty, m, D1, D2)] : make_double2(0, 0);
    Aj[ty][tx] = (j0 + ty < Dq && m < M) ? X[unfold_index(q, j0 + ty, m, D1, D2)] : make_double2(0, 0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = acc + Ai[ty][k] * conjg(Aj[tx][k]);
    __syncthreads();
  }
  if (i0 + ty < Dq && j0 + tx < Dq) G[(long long)(i0 + ty) * Dq + j0 + tx] = acc;
}

// out = in x_q M with M(i, t) = Mat[t * ld + i] (conjugated if cj):
// out[p, i, r] = sum_t in[p, t, r] M(i, t); in is Dpre x Dm x Dpost.
__global__ void mode_product_kernel(const double2* in, double2* out, const double2* Mat, int ld,
                                    int cj, long long Dpre, int Dm, long long Dpost, int Rm) {
  const long long total = Dpre * Rm * Dpost;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx % Dpost;
    const int i = (int)((idx / Dpost) % Rm);
    const long long p = idx / (Dpost * Rm);
    const double2* src = in + p * Dm * Dpost + r;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < Dm; ++t) {
      double2 mv = Mat[(long long)t * ld + i];
      if (cj) mv = conjg(mv);
      acc = cmadd(src[(long long)t * Dpost], mv, acc);
    }
    out[idx] = acc;
  }
}

struct JacobiJob {
  double2* A;     // m x m Hermitian, overwritten (diagonal = eigenvalues)
  double2* V;     // m x m eigenvectors (columns)
  int m;
};

#define JACOBI_MAX_PAIRS 257

// Parallel cyclic Jacobi (round-robin pairing, all disjoint rotations of a
// step applied at once), one CTA per matrix.  A pair (p, q) is rotated when
// |a_pq| > tol sqrt(|a_pp a_qq|); the sweep loop stops after a sweep without
// rotations or after max_sweeps (status -1).
__global__ void __launch_bounds__(1024) jacobi_kernel(const JacobiJob* jobs, int max_sweeps,
                                                      double tol, int* status) {
  const JacobiJob job = jobs[blockIdx.x];
  const int m = job.m;
  const int mm = m + (m & 1);
  const int M = mm - 1;
  const int npair = mm / 2;
  double2* A = job.A;
  double2* V = job.V;
  __shared__ double cs[JACOBI_MAX_PAIRS];
  __shared__ double2 se[JACOBI_MAX_PAIRS];
  __shared__ int pp[JACOBI_MAX_PAIRS], qq[JACOBI_MAX_PAIRS];
  __shared__ double dpp[JACOBI_MAX_PAIRS], dqq[JACOBI_MAX_PAIRS];
  __shared__ int rotated;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (long long e = tid; e < (long long)m * m; e += nth)
    V[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  int sweep = 0;
  bool done = (m <= 1);
  for (; sweep < max_sweeps && !done; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < M; ++step) {
      for (int i = tid; i < npair; i += nth) {
        int p, q;
        if (i == 0) { p = 0; q = 1 + step; }
        else { p = 1 + (step + i) % M; q = 1 + (step - i + M) % M; }
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0;
        double2 sv = make_double2(0.0, 0.0);
        double np_ = 0.0, nq_ = 0.0;
        if (q < m) {
          const double app = A[(long long)p * m + p].x, aqq = A[(long long)q * m + q].x;
          const double2 apq = A[(long long)p * m + q];
          const double mag = sqrt(abs2(apq));
          if (mag > tol * sqrt(fabs(app * aqq)) && mag > 0.0) {
            const double th = (aqq - app) / (2.0 * mag);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            const double s = t * c;
            sv = make_double2(s * apq.x / mag, s * apq.y / mag);   // s e^{i phi}
            np_ = app - t * mag;                                    // rotated diagonal
            nq_ = aqq + t * mag;
            rotated = 1;
          }
        }
        cs[i] = c; se[i] = sv; pp[i] = p; qq[i] = q < m ? q : -1;
        dpp[i] = np_; dqq[i] = nq_;
      }
      __syncthreads();
      // A <- J^* A (rows p, q)
      for (long long it = tid; it < (long long)npair * m; it += nth) {
        const int i = (int)(it / m), k = (int)(it % m);
        if (qq[i] < 0 || (se[i].x == 0.0 && se[i].y == 0.0)) continue;
        const long long ip = (long long)pp[i] * m + k, iq = (long long)qq[i] * m + k;
        const double2 ap = A[ip], aq = A[iq];
        A[ip] = cs[i] * ap - se[i] * aq;
        A[iq] = conjg(se[i]) * ap + cs[i] * aq;
      }
      __syncthreads();
      // A <- A J, V <- V J (columns p, q)
      for (long long it = tid; it < (long long)npair * m; it += nth) {
        const int i = (int)(it / m), k = (int)(it % m);
        if (qq[i] < 0 || (se[i].x == 0.0 && se[i].y == 0.0)) continue;
        const long long ip = (long long)k * m + pp[i], iq = (long long)k * m + qq[i];
        const double2 ap = A[ip], aq = A[iq];
        A[ip] = cs[i] * ap - conjg(se[i]) * aq;
        A[iq] = se[i] * ap + cs[i] * aq;
        const double2 vp = V[ip], vq = V[iq];
        V[ip] = cs[i] * vp - conjg(se[i]) * vq;
        V[iq] = se[i] * vp + cs[i] * vq;
      }
      __syncthreads();
      // the rotation annihilates a_pq exactly and moves t|a_pq| between a_pp and a_qq;
      // writing those values (instead of the rounded updates) lets the relative
      // stopping test be met on graded matrices
      for (int i = tid; i < npair; i += nth) {
        if (qq[i] < 0 || (se[i].x == 0.0 && se[i].y == 0.0)) continue;
        const long long p = pp[i], q = qq[i];
        A[p * m + q] = make_double2(0.0, 0.0);
        A[q * m + p] = make_double2(0.0, 0.0);
        A[p * m + p] = make_double2(dpp[i], 0.0);
        A[q * m + q] = make_double2(dqq[i], 0.0);
      }
      __syncthreads();
    }
    done = (rotated == 0);
    __syncthreads();
  }
  if (tid == 0) status[blockIdx.x] = done ? sweep : -1;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

void make_roots(int N, std::vector<double2>& r64, std::vector<float2>& r32) {
  r64.resize(N);
  r32.resize(N);
  for (int m = 0; m < N; ++m) {
    const double a = -2.0 * kPi * (double)m / (double)N;
    r64[m] = make_double2(std::cos(a), std::sin(a));
    r32[m] = make_float2((float)r64[m].x, (float)r64[m].y);
  }
}

template <typename P> int dalloc(P** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed", bytes);
    return VIE_ERR_OOM;
  }
  return VIE_OK;
}

struct DeviceBuffers {
  double2* full = nullptr;    // P1 P2 P3
  double2* aw = nullptr;      // H1 H2 H3
  double2* tmp = nullptr;     // H1 H2 H3
  double2* gram[3] = {};      // Hq x Hq
  double2* vec[3] = {};       // Hq x Hq
  double2* vec2[3] = {};      // Hq x Hq
  double2* ytr = nullptr;     // truncated Y, max Hq x Hq
  JacobiJob* jobs = nullptr;
  int* jstatus = nullptr;
  unsigned long long* red = nullptr;
  ~DeviceBuffers() {
    cudaFree(full); cudaFree(aw); cudaFree(tmp);
    for (int q = 0; q < 3; ++q) { cudaFree(gram[q]); cudaFree(vec[q]); cudaFree(vec2[q]); }
    cudaFree(ytr); cudaFree(jobs); cudaFree(jstatus); cudaFree(red);
  }
};

}  // namespace

// 3-D FFT of a P1 x P2 x P3 FP64 array in place (three line stages).
static void fft3d_f64(const vie_op* op, double2* a, cudaStream_t s) {
  const long long P1 = op->P[0], P2 = op->P[1], P3 = op->P[2];
  for (int axis = 0; axis < 3; ++axis) {
    LineArgs<double> L = {};
    L.in = a;
    L.out = a;
    L.roots = op->roots64[axis];
    L.plan = op->plan[axis];
    L.lin = L.lout = op->P[axis];
    L.scale = 1.0;
    L.nbatch = 1;
    L.batch_per_rhs = 1;
    L.prof_family = PF_SETUP;
    if (axis == 0) {          // lines along x, columns z, other y
      L.nother = (int)P2; L.ncol = (int)P3;
      L.in_os = L.out_os = P3; L.in_ls = L.out_ls = P2 * P3; L.in_cs = L.out_cs = 1;
    } else if (axis == 1) {   // lines along y, columns z, other x
      L.nother = (int)P1; L.ncol = (int)P3;
      L.in_os = L.out_os = P2 * P3; L.in_ls = L.out_ls = P3; L.in_cs = L.out_cs = 1;
    } else {                  // lines along z (contiguous), columns y, other x
      L.nother = (int)P1; L.ncol = (int)P2;
      L.in_os = L.out_os = P2 * P3; L.in_ls = L.out_ls = 1; L.in_cs = L.out_cs = P3;
    }
    launch_line_fft<double>(L, s);
  }
}

// (2/3)(1 + i k0 a) exp(-i k0 a) - 1 (or without the -1/3 part), a = h (3/4pi)^(1/3)
static double2 self_term_value(const vie_op* op) {
  const double h = op->grid.h, k0 = op->k0;
  const double a = h * std::cbrt(3.0 / (4.0 * kPi));
  const double ca_ = std::cos(k0 * a), sa_ = std::sin(k0 * a);
  double2 self = make_double2((2.0 / 3.0) * (ca_ + k0 * a * sa_) - 1.0,
                              (2.0 / 3.0) * (k0 * a * ca_ - sa_));
  if (op->flags & VIE_SELF_TERM_PV) self.x += 1.0 / 3.0;
  return self;
}

int assemble_spectrum(const vie_op* op, int c, double2* out, cudaStream_t s) {
  int ca, cb;
  component_axes(c, &ca, &cb);
  const double h = op->grid.h, k0 = op->k0;
  const double2 self = self_term_value(op);
  const long long total = (long long)op->P[0] * op->P[1] * op->P[2];
  assemble_kernel<<<grid_for(total), 256, 0, s>>>(out, ca, cb, op->n[0], op->n[1], op->n[2],
                                                   op->P[0], op->P[1], op->P[2], h, k0, self);
  fft3d_f64(op, out, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "assemble/fft");
  return VIE_OK;
}

static int init_tables(vie_op* op) {
  VIE_TRY(line_fft_init_attributes());
  VIE_TRY(fused_init_attributes());
  VIE_TRY(multi_init_attributes());
  VIE_TRY(tp_init_attributes());
  VIE_TRY(umma_init_attributes());
  for (int q = 0; q < 3; ++q) {
    const int N = op->P[q];
    if (!make_plan(N, &op->plan[q])) {
      set_error("padded size %d has a prime factor above 7", N);
      return VIE_ERR_ARG;
    }
    std::vector<double2> r64;
    std::vector<float2> r32;
    make_roots(N, r64, r32);
    VIE_TRY(dalloc(&op->roots64[q], N * sizeof(double2)));
    VIE_TRY(dalloc(&op->roots32[q], N * sizeof(float2)));
    VIE_CUDA(cudaMemcpy(op->roots64[q], r64.data(), N * sizeof(double2), cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(op->roots32[q], r32.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
  }
  return VIE_OK;
}

static int run_jacobi(DeviceBuffers& d, double2* const* A, double2* const* V, const int* m, int njobs,
                      cudaStream_t s) {
  JacobiJob jobs[3];
  for (int j = 0; j < njobs; ++j) jobs[j] = JacobiJob{A[j], V[j], m[j]};
  VIE_CUDA(cudaMemcpyAsync(d.jobs, jobs, njobs * sizeof(JacobiJob), cudaMemcpyHostToDevice, s));
  jacobi_kernel<<<njobs, 1024, 0, s>>>(d.jobs, 60, 1e-15, d.jstatus);
  VIE_CUDA(cudaGetLastError());
  int st[3];
  VIE_CUDA(cudaMemcpyAsync(st, d.jstatus, njobs * sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < njobs; ++j) {
    if (st[j] < 0) {
      set_error("Jacobi eigen-solver did not converge (matrix %d, size %d)", j, m[j]);
      return VIE_ERR_NUMERIC;
    }
  }
  return VIE_OK;
}

static size_t rank_from_sigma2(const std::vector<double>& s2, double tol, int rule, double norm2) {
  const size_t H = s2.size();
  if (H == 0 || s2[0] <= 0.0) return 1;
  if (rule == VIE_RANK_SIGMA_MAX) {
    const double thr = tol / std::sqrt(3.0) * std::sqrt(s2[0]);
    size_t r = 0;
    for (size_t j = 0; j < H; ++j)
      if (std::sqrt(s2[j]) >= thr) ++r;
    return std::max<size_t>(r, 1);
  }
  const double bound = tol / std::sqrt(3.0) * std::sqrt(norm2);
  std::vector<double> tail(H + 1, 0.0);
  for (size_t j = H; j-- > 0;) tail[j] = tail[j + 1] + s2[j];
  for (size_t r = 1; r <= H; ++r)
    if (std::sqrt(tail[r]) <= bound) return r;
  return H;
}

// Compress one component; fills op->comp[c].  Spectrum route: Algorithm 1 on
// the weighted octant of the FFT'd circulant component.  Factor-wise route
// (VIE_SETUP_FACTORWISE, Section V.A): Algorithm 1 on the weighted octant of
// the Toeplitz defining tensor, then the embedding and DFT of each factor
// column; F_q E_q / sqrt(P_q) is an isometry, so both routes give the same
// ranks and the same truncated model (core scaled by sqrt(P1 P2 P3)).
static int compress_component(vie_op* op, int c, double tol, int rule, DeviceBuffers& d,
                              cudaStream_t s, bool factorwise) {
  const int P1 = op->P[0], P2 = op->P[1], P3 = op->P[2];
  // dimensions of the weighted octant the HOSVD runs on
  const int H[3] = {factorwise ? op->n[0] : op->H[0], factorwise ? op->n[1] : op->H[1],
                    factorwise ? op->n[2] : op->H[2]};
  const long long full = (long long)P1 * P2 * P3;
  const long long oct = (long long)H[0] * H[1] * H[2];
  TuckerComp& tc = op->comp[c];
  for (int q = 0; q < 3; ++q) tc.s[q] = component_parity(c, q);
  const bool need_spectrum = !factorwise || op->spec64 != nullptr;

  if (need_spectrum) {
    VIE_TRY(assemble_spectrum(op, c, d.full, s));

    // the symmetry every later step relies on
    VIE_CUDA(cudaMemsetAsync(d.red, 0, 2 * sizeof(unsigned long long), s));
    parity_check_kernel<<<grid_for(full), 256, 0, s>>>(d.full, P1, P2, P3, tc.s[0], tc.s[1], tc.s[2],
                                                        d.red);
    unsigned long long red[2];
    VIE_CUDA(cudaMemcpyAsync(red, d.red, sizeof(red), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    double dev, mx;
    std::memcpy(&dev, &red[0], 8);
    std::memcpy(&mx, &red[1], 8);
    if (!(dev <= 1e-9 * mx + 1e-300) || !std::isfinite(mx)) {
      set_error("component %d spectrum breaks its mirror symmetry (%.3e of %.3e)", c, dev, mx);
      return VIE_ERR_NUMERIC;
    }

    if (op->spec64) {
      VIE_CUDA(cudaMemcpyAsync(op->spec64 + c * full, d.full, full * sizeof(double2),
                               cudaMemcpyDeviceToDevice, s));
      to_c64_kernel<<<grid_for(full), 256, 0, s>>>(d.full, op->spec32 + c * full, full);
    }
  }

  if (!factorwise) {
    octant_kernel<<<grid_for(oct), 256, 0, s>>>(d.full, d.aw, P1, P2, P3, H[0], H[1], H[2]);
  } else {
    int ca, cb;
    component_axes(c, &ca, &cb);
    toeplitz_octant_kernel<<<grid_for(oct), 256, 0, s>>>(d.aw, ca, cb, H[0], H[1], H[2], op->grid.h,
                                                          op->k0, self_term_value(op));
  }

  // pass 1: Gram matrices of the three unfoldings and their eigenvectors Y
  for (int q = 0; q < 3; ++q) {
    dim3 g((H[q] + 15) / 16, (H[q] + 15) / 16);
    gram_kernel<<<g, 256, 0, s>>>(d.aw, d.gram[q], q, H[0], H[1], H[2]);
  }
  VIE_CUDA(cudaGetLastError());
  VIE_TRY(run_jacobi(d, d.gram, d.vec, H, 3, s));

  // pass 2: Gram of Y^* A_w^(q), eigenvectors V2; final vectors Y V2
  for (int q = 0; q < 3; ++q) {
    const long long Dpre = q == 0 ? 1 : (q == 1 ? H[0] : (long long)H[0] * H[1]);
    const long long Dpost = q == 0 ? (long long)H[1] * H[2] : (q == 1 ? H[2] : 1);
    mode_product_kernel<<<grid_for(oct), 256, 0, s>>>(d.aw, d.tmp, d.vec[q], H[q], 1, Dpre, H[q],
                                                      Dpost, H[q]);
    dim3 g((H[q] + 15) / 16, (H[q] + 15) / 16);
    gram_kernel<<<g, 256, 0, s>>>(d.tmp, d.gram[q], q, H[0], H[1], H[2]);
  }
  VIE_CUDA(cudaGetLastError());
  VIE_TRY(run_jacobi(d, d.gram, d.vec2, H, 3, s));

  // sort pass-2 eigenvalues, pick ranks, form Y V2 restricted to the kept columns
  double norm2 = 0.0;
  std::vector<double2> Ytr[3];
  for (int q = 0; q < 3; ++q) {
    const int h = H[q];
    std::vector<double2> G2((size_t)h * h), YV((size_t)h * h);
    VIE_CUDA(cudaMemcpyAsync(G2.data(), d.gram[q], G2.size() * sizeof(double2),
                             cudaMemcpyDeviceToHost, s));
    // Y V2: view Y as [h][h][1] and contract its second index with V2
    mode_product_kernel<<<grid_for((long long)h * h), 256, 0, s>>>(d.vec[q], d.ytr, d.vec2[q], h,
                                                                   0, h, h, 1, h);
    VIE_CUDA(cudaGetLastError());
    VIE_CUDA(cudaMemcpyAsync(YV.data(), d.ytr, YV.size() * sizeof(double2), cudaMemcpyDeviceToHost,
                             s));
    VIE_CUDA(cudaStreamSynchronize(s));
    std::vector<double> lam(h);
    for (int j = 0; j < h; ++j) lam[j] = std::max(G2[(size_t)j * h + j].x, 0.0);
    std::vector<int> order(h);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    std::vector<double> s2(h);
    for (int j = 0; j < h; ++j) s2[j] = lam[order[j]];
    double sum = 0.0;
    for (double v : s2) sum += v;
    if (q == 0) norm2 = sum;
    // singular values of the spectrum's unfolding (P_q / 2 + 1 of them); the
    // factor-wise route has those of the Toeplitz tensor's, sqrt(P1 P2 P3) times smaller
    const double sig_scale = factorwise ? std::sqrt((double)P1 * P2 * P3) : 1.0;
    tc.sigma[q].assign(op->H[q], 0.0);
    for (int j = 0; j < h && j < op->H[q]; ++j) tc.sigma[q][j] = sig_scale * std::sqrt(s2[j]);
    // every mode sees the same ||A||_F; use mode 1's sum for all three
    const int r = (int)rank_from_sigma2(s2, tol, rule, norm2);
    tc.r[q] = r;
    Ytr[q].resize((size_t)h * r);
    for (int i = 0; i < h; ++i)
      for (int j = 0; j < r; ++j) Ytr[q][(size_t)i * r + j] = YV[(size_t)i * h + order[j]];
  }
  if (!(norm2 > 0.0) || !std::isfinite(norm2)) {
    set_error("component %d has zero or non-finite norm", c);
    return VIE_ERR_NUMERIC;
  }

  // core = A_w x1 Y1^* x2 Y2^* x3 Y3^*  (the truncated Y's go to d.vec2)
  const int r1 = tc.r[0], r2 = tc.r[1], r3 = tc.r[2];
  for (int q = 0; q < 3; ++q)
    VIE_CUDA(cudaMemcpy(d.vec2[q], Ytr[q].data(), Ytr[q].size() * sizeof(double2),
                        cudaMemcpyHostToDevice));
  mode_product_kernel<<<grid_for((long long)r1 * H[1] * H[2]), 256, 0, s>>>(
      d.aw, d.tmp, d.vec2[0], r1, 1, 1, H[0], (long long)H[1] * H[2], r1);
  mode_product_kernel<<<grid_for((long long)r1 * r2 * H[2]), 256, 0, s>>>(
      d.tmp, d.aw, d.vec2[1], r2, 1, r1, H[1], H[2], r2);
  mode_product_kernel<<<grid_for((long long)r1 * r2 * r3), 256, 0, s>>>(
      d.aw, d.tmp, d.vec2[2], r3, 1, (long long)r1 * r2, H[2], 1, r3);
  VIE_CUDA(cudaGetLastError());
  const size_t ncore = (size_t)r1 * r2 * r3;
  VIE_TRY(dalloc(&tc.core64, ncore * sizeof(double2)));
  VIE_TRY(dalloc(&tc.core32, ncore * sizeof(float2)));
  if (factorwise) {
    // the spectrum's core: the Toeplitz tensor's times sqrt(P1 P2 P3)
    const double sc = std::sqrt((double)P1 * P2 * P3);
    std::vector<double2> hc(ncore);
    VIE_CUDA(cudaMemcpyAsync(hc.data(), d.tmp, ncore * sizeof(double2), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    for (auto& v : hc) v = make_double2(sc * v.x, sc * v.y);
    VIE_CUDA(cudaMemcpy(d.tmp, hc.data(), ncore * sizeof(double2), cudaMemcpyHostToDevice));
  }
  VIE_CUDA(cudaMemcpyAsync(tc.core64, d.tmp, ncore * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  to_c64_kernel<<<grid_for(ncore), 256, 0, s>>>(tc.core64, tc.core32, (long long)ncore);

  // stored factor rows: U_half = D^-1 Y (rows 0..P/2 of the full factor); on the
  // factor-wise route D^-1 Y are the Toeplitz factor's rows at offsets 0..n-1, which
  // are embedded and DFT'd into rows 0..P/2 of the spectrum's factor
  for (int q = 0; q < 3; ++q) {
    const int h = op->H[q], r = tc.r[q];
    std::vector<double2> u64((size_t)h * r);
    std::vector<float2> u32((size_t)h * r);
    if (!factorwise) {
      for (int i = 0; i < h; ++i) {
        const double w = (i == 0 || 2 * i == op->P[q]) ? 1.0 : 1.0 / std::sqrt(2.0);
        for (int j = 0; j < r; ++j) {
          const double2 v = Ytr[q][(size_t)i * r + j];
          u64[(size_t)i * r + j] = make_double2(w * v.x, w * v.y);
        }
      }
    } else {
      const int n = op->n[q];
      std::vector<double2> ut((size_t)n * r);
      for (int i = 0; i < n; ++i) {
        const double w = i == 0 ? 1.0 : 1.0 / std::sqrt(2.0);
        for (int j = 0; j < r; ++j) {
          const double2 v = Ytr[q][(size_t)i * r + j];
          ut[(size_t)i * r + j] = make_double2(w * v.x, w * v.y);
        }
      }
      VIE_CUDA(cudaMemcpy(d.ytr, ut.data(), ut.size() * sizeof(double2), cudaMemcpyHostToDevice));
      factor_dft_kernel<<<grid_for((long long)h * r), 256, 0, s>>>(d.ytr, d.tmp, op->roots64[q], n,
                                                                    op->P[q], r, tc.s[q]);
      VIE_CUDA(cudaGetLastError());
      VIE_CUDA(cudaMemcpyAsync(u64.data(), d.tmp, u64.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
      VIE_CUDA(cudaStreamSynchronize(s));
    }
    for (size_t i = 0; i < u64.size(); ++i) u32[i] = make_float2((float)u64[i].x, (float)u64[i].y);
    VIE_TRY(dalloc(&tc.U64[q], u64.size() * sizeof(double2)));
    VIE_TRY(dalloc(&tc.U32[q], u32.size() * sizeof(float2)));
    VIE_CUDA(cudaMemcpy(tc.U64[q], u64.data(), u64.size() * sizeof(double2), cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(tc.U32[q], u32.data(), u32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if (q == 2) {
      // transposed copy: a warp rebuilding consecutive k3 reads consecutive addresses
      std::vector<float2> t((size_t)r * h);
      for (int i = 0; i < h; ++i)
        for (int j = 0; j < r; ++j) t[(size_t)j * h + i] = u32[(size_t)i * r + j];
      VIE_TRY(dalloc(&tc.U3t32, t.size() * sizeof(float2)));
      VIE_CUDA(cudaMemcpy(tc.U3t32, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
  }
  VIE_CUDA(cudaStreamSynchronize(s));
  return VIE_OK;
}

static int finish_operator(vie_op* op) {
  for (int q = 0; q < 3; ++q) {
    op->rmax[q] = 1;
    for (int c = 0; c < 6; ++c) op->rmax[q] = std::max(op->rmax[q], op->comp[c].r[q]);
  }
  op->slab_stride = (size_t)op->H[0] * op->rmax[1] * op->rmax[2];
  VIE_TRY(dalloc(&op->slab32, 6 * op->slab_stride * sizeof(float2)));
  VIE_TRY(dalloc(&op->slab64, 6 * op->slab_stride * sizeof(double2)));
  CompMeta<float> m32[6];
  CompMeta<double> m64[6];
  for (int c = 0; c < 6; ++c) {
    const TuckerComp& tc = op->comp[c];
    m32[c] = CompMeta<float>{tc.U32[1], tc.U32[2], tc.U3t32, op->slab32 + c * op->slab_stride,
                             tc.r[1], tc.r[2], tc.s[0], tc.s[1], tc.s[2]};
    m64[c] = CompMeta<double>{tc.U64[1], tc.U64[2], nullptr, op->slab64 + c * op->slab_stride,
                              tc.r[1], tc.r[2], tc.s[0], tc.s[1], tc.s[2]};
  }
  static_assert(sizeof(CompMeta<float>) == sizeof(CompMeta<double>), "meta layout");
  VIE_TRY(dalloc(&op->dev_err, sizeof(int)));
  VIE_CUDA(cudaMemset(op->dev_err, 0, sizeof(int)));
  VIE_TRY(dalloc((char**)&op->meta, sizeof(m32) + sizeof(m64)));
  VIE_CUDA(cudaMemcpy(op->meta, m32, sizeof(m32), cudaMemcpyHostToDevice));
  VIE_CUDA(cudaMemcpy(static_cast<char*>(op->meta) + sizeof(m32), m64, sizeof(m64),
                      cudaMemcpyHostToDevice));
  // slab cores S_c[k1] = core_c x1 U1_c[k1, :]: the first stage of eq. (13), fixed
  // for the operator, so formed once here rather than at every matvec
  VIE_TRY(launch_slab_cores<float>(op, 0));
  VIE_TRY(launch_slab_cores<double>(op, 0));
  // FP32 scratch for the per-matvec rebuild of the half fibres (register-path
  // fused kernel): whole k1 planes of [H2][6][H3], as many as fit in kOctBudget
  if (op->P[2] % 32 == 0 && vie::warp_fft_supported(op->P[2] / 32) &&
      octant_smem_bytes(op->rmax[1], op->rmax[2]) <= kOctantSmemMax) {
    constexpr size_t kOctBudget = 64u << 20;
    const size_t plane = (size_t)op->H[1] * 6 * op->H[2] * sizeof(float2);
    op->oct_k1 = (int)std::max<size_t>(1, std::min<size_t>(op->H[0], kOctBudget / plane));
    VIE_TRY(dalloc(&op->oct32, (size_t)op->oct_k1 * plane));
    VIE_CUDA(cudaStreamCreateWithFlags(&op->rb_stream, cudaStreamNonBlocking));
    VIE_CUDA(cudaEventCreateWithFlags(&op->rb_fork, cudaEventDisableTiming));
    VIE_CUDA(cudaEventCreateWithFlags(&op->rb_join, cudaEventDisableTiming));
    if ((op->flags & VIE_REBUILD_TCGEN05) && !(op->flags & VIE_REBUILD_SIMT) && umma_rebuild_eligible(op)) {
      op->umma = true;
    } else if (tc_rebuild_eligible(op)) {
      tc_layout(op->rmax[2], op->H[2], &op->tc_ks, &op->tc_nsplit, &op->tc_ntc);
    }
    if (op->tc_ks > 0 && tc_rebuild_fits(op)) {
      VIE_TRY(dalloc(&op->u3frag, 6ull * op->tc_nsplit * op->tc_ks * op->tc_ntc * 32 * sizeof(uint4)));
      VIE_TRY(launch_u3_fragments(op, 0));
    }
  }
  VIE_CUDA(cudaDeviceSynchronize());
  return VIE_OK;
}

int op_tables(vie_op* op) { return init_tables(op); }

int build_operator(const vie_grid* grid, double tol, int rank_rule, int flags, cudaStream_t s,
                   vie_op** out) {
  vie_op* op = new (std::nothrow) vie_op();
  if (!op) {
    set_error("host allocation failed");
    return VIE_ERR_OOM;
  }
  op->grid = *grid;
  op->flags = flags;
  op->k0 = wavenumber(grid->freq_hz);
  const int nn[3] = {grid->n1, grid->n2, grid->n3};
  for (int q = 0; q < 3; ++q) {
    op->n[q] = nn[q];
    op->P[q] = 2 * nn[q];
    op->H[q] = nn[q] + 1;
  }
  int st = init_tables(op);
  if (st != VIE_OK) { vie_destroy(op); return st; }
  const long long full = (long long)op->P[0] * op->P[1] * op->P[2];
  const long long oct = (long long)op->H[0] * op->H[1] * op->H[2];
  if (flags & VIE_STORE_UNCOMPRESSED) {
    if ((st = dalloc(&op->spec64, 6 * full * sizeof(double2))) != VIE_OK ||
        (st = dalloc(&op->spec32, 6 * full * sizeof(float2))) != VIE_OK) {
      vie_destroy(op);
      return st;
    }
  }
  {
    DeviceBuffers d;
    const int hmax = std::max(op->H[0], std::max(op->H[1], op->H[2]));
    const bool factorwise = (flags & VIE_SETUP_FACTORWISE) != 0;
    // the P1 P2 P3 spectrum is formed only on the spectrum route or to be stored
    const bool need_full = !factorwise || (flags & VIE_STORE_UNCOMPRESSED);
    if ((need_full && (st = dalloc(&d.full, full * sizeof(double2))) != VIE_OK) ||
        (st = dalloc(&d.aw, oct * sizeof(double2))) != VIE_OK ||
        (st = dalloc(&d.tmp, std::max(oct, (long long)hmax * hmax) * sizeof(double2))) != VIE_OK ||
        (st = dalloc(&d.ytr, (size_t)hmax * hmax * sizeof(double2))) != VIE_OK ||
        (st = dalloc(&d.jobs, 3 * sizeof(JacobiJob))) != VIE_OK ||
        (st = dalloc(&d.jstatus, 3 * sizeof(int))) != VIE_OK ||
        (st = dalloc(&d.red, 2 * sizeof(unsigned long long))) != VIE_OK) {
      vie_destroy(op);
      return st;
    }
    op->setup_scratch_bytes =
        (need_full ? full * sizeof(double2) : 0) + oct * sizeof(double2) +
        std::max(oct, (long long)hmax * hmax) * sizeof(double2) + (size_t)hmax * hmax * sizeof(double2);
    for (int q = 0; q < 3; ++q) op->setup_scratch_bytes += 3 * (size_t)op->H[q] * op->H[q] * sizeof(double2);
    for (int q = 0; q < 3 && st == VIE_OK; ++q) {
      const size_t hh = (size_t)op->H[q] * op->H[q] * sizeof(double2);
      if ((st = dalloc(&d.gram[q], hh)) != VIE_OK || (st = dalloc(&d.vec[q], hh)) != VIE_OK ||
          (st = dalloc(&d.vec2[q], hh)) != VIE_OK)
        break;
    }
    for (int c = 0; c < 6 && st == VIE_OK; ++c)
      st = compress_component(op, c, tol, rank_rule, d, s, factorwise);
    if (st == VIE_OK) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_status(e, "compress");
    }
  }
  if (st == VIE_OK) st = finish_operator(op);
  if (st != VIE_OK) {
    vie_destroy(op);
    return st;
  }
  *out = op;
  return VIE_OK;
}
