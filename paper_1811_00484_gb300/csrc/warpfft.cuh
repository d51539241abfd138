// Register-resident FFTs of length N = 32 R, one warp per line.
//
// Lane l holds x[l + 32 j], j < R.  With n = l + 32 j and k = k1 + R k2,
//   X[k1 + R k2] = sum_l w_32^{l k2} w_N^{l k1} sum_j x[l + 32 j] w_R^{j k1},
// so the forward transform is a length-R DFT in registers, a twiddle by
// w_N^{l k1}, and a 32-point decimation-in-frequency FFT across the lanes
// (shuffles) that leaves X[k1 + R brev5(l)] in register k1 of lane l.  The
// inverse runs the same steps backwards with a decimation-in-time lane FFT,
// which takes exactly that bit-reversed layout and returns natural order, so
// a forward / voxel-wise product / inverse sequence never reorders data.
// w_M^m = exp(-2 pi i m / M) is read from the table of N-th roots.
#pragma once

#include "fft.cuh"

namespace vie {

__device__ __forceinline__ float2 shfl_xor(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ int brev5(int l) { return __brev((unsigned)l) >> 27; }

template <typename C, typename T, int R> struct RegDft;

// length-R DFT of v[0..R) in registers, natural order in and out
template <typename C, typename T, int R>
__device__ __forceinline__ void reg_dft(C* v, const C* roots, int N, bool inv) {
  RegDft<C, T, R>::run(v, roots, N, inv);
}

template <typename C, typename T> struct RegDft<C, T, 1> {
  static __device__ __forceinline__ void run(C*, const C*, int, bool) {}
};
template <typename C, typename T> struct RegDft<C, T, 2> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool) { dft2(v); }
};
template <typename C, typename T> struct RegDft<C, T, 3> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool inv) { dft3<C, T>(v, inv); }
};
template <typename C, typename T> struct RegDft<C, T, 4> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool inv) {
    dft4(v[0], v[1], v[2], v[3], inv);
  }
};
template <typename C, typename T> struct RegDft<C, T, 5> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool inv) { dft5<C, T>(v, inv); }
};
template <typename C, typename T> struct RegDft<C, T, 8> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool inv) { dft8<C, T>(v, inv); }
};

// R = R1 R2: x[R2 n1 + n2] -> DFT_R1 over n1, twiddle w_R^{n2 k1}, DFT_R2 over n2,
// X[k1 + R1 k2]
template <typename C, typename T, int R1, int R2> struct RegDftSplit {
  static __device__ __forceinline__ void run(C* v, const C* roots, int N, bool inv) {
    constexpr int R = R1 * R2;
    C a[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      C t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
      reg_dft<C, T, R1>(t, roots, N, inv);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        C x = t[k1];
        if (n2 * k1 != 0) x = x * twiddle(roots, n2 * k1 * (N / R), inv);
        a[n2 * R1 + k1] = x;
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C t[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) t[n2] = a[n2 * R1 + k1];
      reg_dft<C, T, R2>(t, roots, N, inv);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[k2];
    }
  }
};
template <typename C, typename T> struct RegDft<C, T, 6> : RegDftSplit<C, T, 2, 3> {};
template <typename C, typename T> struct RegDft<C, T, 10> : RegDftSplit<C, T, 2, 5> {};
template <typename C, typename T> struct RegDft<C, T, 12> : RegDftSplit<C, T, 4, 3> {};
template <typename C, typename T> struct RegDft<C, T, 16> : RegDftSplit<C, T, 4, 4> {};

// forward: v[j] = x[lane + 32 j]  ->  v[k1] = X[k1 + R brev5(lane)]
template <typename C, typename T, int R>
__device__ __forceinline__ void warp_fft_fwd(C* v, int lane, const C* roots, int N) {
  reg_dft<C, T, R>(v, roots, N, false);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * roots[lane * k1];
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const int i = lane & (h - 1);
    const bool upper = (lane & h) != 0;
    const C w = roots[i * (N / (2 * h))];
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const C p = shfl_xor(v[k1], h);
      v[k1] = upper ? (p - v[k1]) * w : v[k1] + p;
    }
  }
}

// inverse (unscaled): v[k1] = X[k1 + R brev5(lane)]  ->  v[j] = N x[lane + 32 j]
template <typename C, typename T, int R>
__device__ __forceinline__ void warp_fft_inv(C* v, int lane, const C* roots, int N) {
#pragma unroll
  for (int h = 1; h <= 16; h <<= 1) {
    const int i = lane & (h - 1);
    const bool upper = (lane & h) != 0;
    const C w = conjg(roots[i * (N / (2 * h))]);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const C p = shfl_xor(v[k1], h);
      v[k1] = upper ? (p - w * v[k1]) : (v[k1] + w * p);
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * conjg(roots[lane * k1]);
  reg_dft<C, T, R>(v, roots, N, true);
}

// radices handled by the register path (N = 32 R <= 512)
__host__ __device__ constexpr bool warp_fft_supported(int R) {
  return R == 1 || R == 2 || R == 3 || R == 4 || R == 5 || R == 6 || R == 8 || R == 10 || R == 12 ||
         R == 16;
}

}  // namespace vie
