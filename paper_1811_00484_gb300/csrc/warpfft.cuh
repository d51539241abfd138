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
template <typename C, typename T> struct RegDft<C, T, 16> {
  static __device__ __forceinline__ void run(C* v, const C*, int, bool inv) { dft16<C, T>(v, inv); }
};
template <typename C, typename T> struct RegDft<C, T, 24> : RegDftSplit<C, T, 3, 8> {};
template <typename C, typename T> struct RegDft<C, T, 32> : RegDftSplit<C, T, 4, 8> {};

// Per-lane constants of the lane transforms, computed once per kernel:
//   tw[k1]  = w_N^{lane k1}                       (twiddle between the stages)
//   fw[s]   = upper ? w_{2h}^i : 1, fs[s] = upper ? -1 : 1   (DIF stage s, h = 16 >> s)
//   iw[s]   = (upper ? -1 : 1) conj(w_{2h}^i)                (DIT stage s, h = 1 << s)
// with i = lane mod h and `upper` = bit h of the lane.
template <typename C, typename T, int R> struct LaneConsts {
  C tw[R > 1 ? R : 1];
  C fw[5];
  T fs[5];
  C iw[5];
  __device__ __forceinline__ void init(int lane, const C* roots, int N) {
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) tw[k1] = roots[lane * k1];
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int h = 16 >> st;
      const bool up = (lane & h) != 0;
      const C w = roots[(lane & (h - 1)) * (N / (2 * h))];
      fw[st] = up ? w : mk((T)1, (T)0);
      fs[st] = up ? (T)-1 : (T)1;
    }
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int h = 1 << st;
      const bool up = (lane & h) != 0;
      const C w = conjg(roots[(lane & (h - 1)) * (N / (2 * h))]);
      iw[st] = up ? mk(-w.x, -w.y) : w;
    }
  }
};

// forward: v[j] = x[lane + 32 j]  ->  v[k1] = X[k1 + R brev5(lane)].
// HALF: only x[0 .. N/2) can be nonzero (zero-padded input): v[j] for
// j >= (R+1)/2 (points lane + 32 j >= N/2 + 16) is set to zero here, so the
// caller only loads j < (R+1)/2.
template <typename C, typename T, int R, bool HALF = false>
__device__ __forceinline__ void warp_fft_fwd(C* v, const LaneConsts<C, T, R>& lc, const C* roots,
                                             int N) {
  if (HALF) {
#pragma unroll
    for (int j = (R + 1) / 2; j < R; ++j) v[j] = mk((T)0, (T)0);
  }
  reg_dft<C, T, R>(v, roots, N, false);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * lc.tw[k1];
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 16 >> st;
    const T sg = lc.fs[st];
    const C w = lc.fw[st];
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const C p = shfl_xor(v[k1], h);
      // lower lane: v + p; upper lane: (p - v) w
      const C t = mk(fma(sg, v[k1].x, p.x), fma(sg, v[k1].y, p.y));
      v[k1] = t * w;
    }
  }
}

// inverse (unscaled): v[k1] = X[k1 + R brev5(lane)]  ->  v[j] = N x[lane + 32 j].
// HALF: only x[0 .. N/2) is wanted (cropped output): the caller stores only
// j < (R+1)/2.
template <typename C, typename T, int R, bool HALF = false>
__device__ __forceinline__ void warp_fft_inv(C* v, int lane, const LaneConsts<C, T, R>& lc,
                                             const C* roots, int N) {
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 1 << st;
    const bool upper = (lane & h) != 0;
    const C w = lc.iw[st];
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const C p = shfl_xor(v[k1], h);
      // lower lane: v + w p; upper lane: p - w v  (w carries the sign)
      const C a = upper ? p : v[k1];
      const C b = upper ? v[k1] : p;
      v[k1] = cmadd(w, b, a);
    }
  }
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) v[k1] = v[k1] * conjg(lc.tw[k1]);
  reg_dft<C, T, R>(v, roots, N, true);
  (void)HALF;
}

// the original forms (per-call constants), kept for the FP64 and non-template users
template <typename C, typename T, int R>
__device__ __forceinline__ void warp_fft_fwd(C* v, int lane, const C* roots, int N) {
  LaneConsts<C, T, R> lc;
  lc.init(lane, roots, N);
  warp_fft_fwd<C, T, R, false>(v, lc, roots, N);
}
template <typename C, typename T, int R>
__device__ __forceinline__ void warp_fft_inv(C* v, int lane, const C* roots, int N) {
  LaneConsts<C, T, R> lc;
  lc.init(lane, roots, N);
  warp_fft_inv<C, T, R, false>(v, lane, lc, roots, N);
}

// radices handled by the register path (N = 32 R <= 512)
__host__ __device__ constexpr bool warp_fft_supported(int R) {
  return R == 1 || R == 2 || R == 3 || R == 4 || R == 5 || R == 6 || R == 8 || R == 10 || R == 12 ||
         R == 16;
}

}  // namespace vie
