// Shared-memory mixed-radix Stockham FFT used by every transform of the
// matvec (zero-padded forward FFT and cropped inverse FFT, Section V.B) and
// by the FP64 spectrum assembly of the setup (Section V.A).
//
// A length-N line is transformed in passes of radix R; with Ns the product
// of the radices already applied, butterfly j (0 <= j < N/R) reads
// x[j + t N/R] (t < R), multiplies element t by w^(t k N/(Ns R)) where
// k = j mod Ns and w = exp(-2 pi i / N), applies a length-R DFT and writes
// y[(j / Ns) Ns R + k + t Ns].  Radices 2, 3, 4, 5, 8 have hand-written
// butterflies; 7 uses a direct length-R sum.
#pragma once

#include "vie_internal.cuh"

namespace vie {

template <typename C>
__device__ __forceinline__ C twiddle(const C* roots, int e, bool inv) {
  C w = roots[e];
  return inv ? conjg(w) : w;
}

// forward: exp(-2 pi i t k / R); inverse: exp(+2 pi i t k / R)
template <typename C>
__device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3, bool inv) {
  C a = v0 + v2, b = v0 - v2, c = v1 + v3, d = v1 - v3;
  C id = inv ? mul_i(d) : mul_mi(d);
  v0 = a + c;
  v2 = a - c;
  v1 = b + id;
  v3 = b - id;
}

template <typename C, typename T>
__device__ __forceinline__ void dft8(C* v, bool inv) {
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3, inv);
  dft4(o0, o1, o2, o3, inv);
  const T r = (T)0.70710678118654752440;
  // o_k *= exp(-/+ i pi k / 4)
  C t1, t2, t3;
  if (!inv) {
    t1 = mk(r * (o1.x + o1.y), r * (o1.y - o1.x));
    t2 = mul_mi(o2);
    t3 = mk(r * (o3.y - o3.x), -r * (o3.x + o3.y));
  } else {
    t1 = mk(r * (o1.x - o1.y), r * (o1.x + o1.y));
    t2 = mul_i(o2);
    t3 = mk(-r * (o3.x + o3.y), r * (o3.x - o3.y));
  }
  v[0] = e0 + o0;
  v[4] = e0 - o0;
  v[1] = e1 + t1;
  v[5] = e1 - t1;
  v[2] = e2 + t2;
  v[6] = e2 - t2;
  v[3] = e3 + t3;
  v[7] = e3 - t3;
}

// v * w16^e with w16 = exp(-/+ 2 pi i / 16), e in {1, 2, 3, 4, 6, 9} (compile time)
template <typename C, typename T, int E>
__device__ __forceinline__ C w16mul(C v, bool inv) {
  const T c = (T)0.92387953251128675613, s = (T)0.38268343236508977173;   // cos, sin(pi/8)
  const T r = (T)0.70710678118654752440;
  T wr, wi;                                            // forward root
  if (E == 1) { wr = c; wi = -s; }
  else if (E == 2) { wr = r; wi = -r; }
  else if (E == 3) { wr = s; wi = -c; }
  else if (E == 4) { wr = 0; wi = -1; }
  else if (E == 6) { wr = -r; wi = -r; }
  else { wr = -c; wi = s; }                            // E == 9
  if (inv) wi = -wi;
  if (E == 4) return inv ? mul_i(v) : mul_mi(v);
  return mk(v.x * wr - v.y * wi, v.x * wi + v.y * wr);
}

// length-16 DFT in registers, natural order in and out: 4 x 4 with in-place
// radix-4 butterflies (n = 4 n1 + n2, k = k1 + 4 k2) and constant twiddles
template <typename C, typename T>
__device__ __forceinline__ void dft16(C* v, bool inv) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[4 + n2], v[8 + n2], v[12 + n2], inv);
  // v[4 k1 + n2] *= w16^{n2 k1}
  v[5] = w16mul<C, T, 1>(v[5], inv);
  v[6] = w16mul<C, T, 2>(v[6], inv);
  v[7] = w16mul<C, T, 3>(v[7], inv);
  v[9] = w16mul<C, T, 2>(v[9], inv);
  v[10] = w16mul<C, T, 4>(v[10], inv);
  v[11] = w16mul<C, T, 6>(v[11], inv);
  v[13] = w16mul<C, T, 3>(v[13], inv);
  v[14] = w16mul<C, T, 6>(v[14], inv);
  v[15] = w16mul<C, T, 9>(v[15], inv);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3], inv);
  // X[k1 + 4 k2] sits in v[4 k1 + k2]: transpose (a register permutation)
  C t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <typename C, typename T>
__device__ __forceinline__ void dft3(C* v, bool inv) {
  const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
  C t1 = v[1] + v[2], t2 = v[1] - v[2];
  C m = v[0] - (T)0.5 * t1;
  C u = h * t2;
  C iu = inv ? mul_i(u) : mul_mi(u);
  v[0] = v[0] + t1;
  v[1] = m + iu;
  v[2] = m - iu;
}

template <typename C, typename T>
__device__ __forceinline__ void dft5(C* v, bool inv) {
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
  const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
  C t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  C a1 = v[0] + c1 * t1 + c2 * t2;
  C a2 = v[0] + c2 * t1 + c1 * t2;
  C b1 = s1 * t3 + s2 * t4;
  C b2 = s2 * t3 - s1 * t4;
  C ib1 = inv ? mul_i(b1) : mul_mi(b1);
  C ib2 = inv ? mul_i(b2) : mul_mi(b2);
  v[0] = v[0] + t1 + t2;
  v[1] = a1 + ib1;
  v[4] = a1 - ib1;
  v[2] = a2 + ib2;
  v[3] = a2 - ib2;
}

// direct length-R DFT using the N-th roots (w_R^m = roots[m N / R])
template <typename C, int R>
__device__ __forceinline__ void dft_direct(C* v, const C* roots, int N, bool inv) {
  C out[R];
  const int step = N / R;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    C acc = v[0];
#pragma unroll
    for (int t = 1; t < R; ++t) acc = cmadd(v[t], twiddle(roots, ((t * k) % R) * step, inv), acc);
    out[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

// One Stockham pass of radix R over `nlines` lines.  Element (line, p) is at
// line * lstride + p * pstride.  COLS: consecutive threads take consecutive
// lines (lines interleaved in memory); otherwise consecutive butterflies.
template <typename T, int R, bool COLS>
__device__ __forceinline__ void fft_pass_r(const cx<T>* __restrict__ x, cx<T>* __restrict__ y,
                                           int N, int Ns, int nlines, int lstride, int pstride,
                                           const cx<T>* roots, bool inv, int tid, int nth) {
  using C = cx<T>;
  const int nb = N / R;
  const int total = nb * nlines;
  const int twstep = N / (Ns * R);
  for (int item = tid; item < total; item += nth) {
    int line, j;
    if (COLS) {
      line = item % nlines;
      j = item / nlines;
    } else {
      j = item % nb;
      line = item / nb;
    }
    const int k = j % Ns;
    const C* xl = x + line * lstride;
    C v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = xl[(j + t * nb) * pstride];
    if (k != 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) v[t] = v[t] * twiddle(roots, t * k * twstep, inv);
    }
    if (R == 2) dft2(v);
    else if (R == 4) dft4(v[0], v[1], v[2], v[3], inv);
    else if (R == 8) dft8<C, T>(v, inv);
    else if (R == 3) dft3<C, T>(v, inv);
    else if (R == 5) dft5<C, T>(v, inv);
    else dft_direct<C, R>(v, roots, N, inv);
    const int base = (j / Ns) * Ns * R + k;
    C* yl = y + line * lstride;
#pragma unroll
    for (int t = 0; t < R; ++t) yl[(base + t * Ns) * pstride] = v[t];
  }
}

template <typename T, bool COLS>
__device__ __forceinline__ void fft_pass(const cx<T>* x, cx<T>* y, int N, int R, int Ns, int nlines,
                                         int lstride, int pstride, const cx<T>* roots, bool inv,
                                         int tid, int nth) {
  switch (R) {
    case 8: fft_pass_r<T, 8, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    case 4: fft_pass_r<T, 4, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    case 2: fft_pass_r<T, 2, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    case 3: fft_pass_r<T, 3, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    case 5: fft_pass_r<T, 5, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    case 7: fft_pass_r<T, 7, COLS>(x, y, N, Ns, nlines, lstride, pstride, roots, inv, tid, nth); break;
    default: break;
  }
}

// Full transform of `nlines` lines held in `a`, using `b` as the ping-pong
// buffer.  Returns the buffer that holds the result.  Every thread of the
// block must call it (it synchronises between passes).
template <typename T, bool COLS>
__device__ __forceinline__ cx<T>* fft_lines(cx<T>* a, cx<T>* b, const FftPlan& plan, int nlines,
                                            int lstride, int pstride, const cx<T>* roots, bool inv,
                                            int tid, int nth) {
  int Ns = 1;
  cx<T>* src = a;
  cx<T>* dst = b;
  for (int p = 0; p < plan.npass; ++p) {
    const int R = plan.radix[p];
    fft_pass<T, COLS>(src, dst, plan.N, R, Ns, nlines, lstride, pstride, roots, inv, tid, nth);
    __syncthreads();
    Ns *= R;
    cx<T>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

}  // namespace vie
