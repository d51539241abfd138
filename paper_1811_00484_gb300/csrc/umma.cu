// The per-matvec rebuild of the half fibres, eq. (13), on the fifth-generation
// tensor cores: tcgen05.mma with operands in shared memory and the
// accumulator in tensor memory (TMEM).
//
//   G_c[k1, k2, k3] = sum_q W[k2, q] U3_c[k3, q],   W = U2_c S_c[k1]
//
// for k1 in a chunk, k2 <= P2/2 and k3 <= P3/2, into the same FP32 scratch
// [chunk][H2][6][H3] that octant_tc_kernel (warp-level mma.sync) fills.
//
// Complex GEMM as one real GEMM (the 4M form): row k2 of A is W[k2, :] read as
// interleaved (re, im) floats (K = 2 r3, padded to a multiple of 8); row j of
// B (N rows, K-major) is, for output column j = 2 k3 + s,
//   s = 0 (Re G):  ( Re U3[k3, q], -Im U3[k3, q] )  over q
//   s = 1 (Im G):  ( Im U3[k3, q],  Re U3[k3, q] )
// so that D[k2, j] is G[k2, k3] as interleaved floats, written out directly.
// Operands are split into TF32 value and remainder and three MMAs per k-step
// accumulate hi*hi + hi*lo + lo*hi (3xTF32) into the same FP32 accumulator:
// one TF32 product (~3e-4 relative) would break the 1e-5 matvec tolerance.
//
// CTA = 256 threads, one per SM (shared memory), persistent over the units
// (k1, 128-row tile of k2) of one component and one range of N columns:
//   - once: B (hi, lo) for the CTA's columns into shared memory;
//   - per unit: all threads form W for the 128 rows (FP32 FMAs, W = U2 S,
//     two threads per row) into one of two A buffers, one thread issues the
//     K/8 x 3 MMAs into one of two TMEM accumulators and commits them to an
//     mbarrier, and while they run, all threads drain the previous unit's
//     accumulator (tcgen05.ld, staged per warp through shared memory so that
//     each row segment is stored by consecutive lanes).
// The column k3 = P3/2 (the Nyquist column, outside the N ranges) is formed
// from the A tile with FMAs by the CTA of the last range; rows k2 >= H2 of the
// last tile are zero in A and not stored.
//
// Shared-memory operand layout (no swizzle, K-major): core matrices of 8 rows
// x 16 bytes stored contiguously; core matrices adjacent in K are 128 bytes
// apart (leading byte offset), 8-row groups 32 K bytes apart (stride byte
// offset); a k-step of 8 TF32 values spans two core matrices, so its
// descriptor starts 256 bytes after the previous one.
#include <algorithm>

#include "tma.cuh"

namespace vie {

constexpr int kUmThreads = 256;
constexpr int kUmRows = 128;              // M of every MMA (one TMEM lane per row)
constexpr int kUmMaxR3 = 32;              // K = 2 r3 <= 64
constexpr int kUmStage = 32 * 17;         // floats per warp: 32 rows x 16 columns (+1 pad)
constexpr unsigned long long kUmWaitNs = 1000000000ull;   // 1 s per bounded wait
// dynamic shared memory: the 227 KB a CTA may hold, less the kernel's static barriers
constexpr size_t kUmSmemLimit = (227u << 10) - 256;

struct OctUmmaArgs {
  const CompMeta<float>* meta;
  float2* out;       // [nk1][H2][6][H3]
  int H2, H3;
  int r2max, r3max;  // slab cores [H1][r2max][r3max]
  int r23;           // r2max * r3max
  int k1a, nk1;
  int mt;            // 128-row tiles of k2
  int nsplit, NC;    // N ranges per component, NC complex columns each (N = 2 NC)
  int per;           // units per CTA
  int kp;            // K of the operand buffers (>= every component's K)
  int tmem_cols;     // power of two >= 2 N
  int* err;          // device word set to VIE_ERR_TIMEOUT when a wait gives up
};

__host__ __device__ constexpr int um_k(int r3) { return (2 * r3 + 7) & ~7; }

// U2 rows staged with an odd float2 stride: the A-build's row-per-thread
// reads are then free of bank conflicts
__host__ __device__ constexpr int um_r2p(int r2max) { return r2max | 1; }

__host__ __device__ constexpr size_t um_smem(int N, int kp, int H2, int r2max, int r3max) {
  return (size_t)2 * N * kp * sizeof(float) +                  // B hi, lo
         (size_t)4 * kUmRows * kp * sizeof(float) +            // A [2 buffers][hi, lo]
         (size_t)(kUmThreads / 32) * kUmStage * sizeof(float) + // epilogue staging
         ((size_t)H2 * um_r2p(r2max) +                          // U2 of the component
          (size_t)r2max * r3max + r3max) * sizeof(float2) +     // S[k1], U3[P3/2, :]
         1024;                                                  // alignment slack
}

// float offset of element (row, k) in the K-major core-matrix layout with K columns
__device__ __forceinline__ int um_off(int row, int k, int K) {
  return (row >> 3) * (8 * K) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint32_t um_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: no swizzle, descriptor version 1
__device__ __forceinline__ uint64_t um_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void um_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void um_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void um_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void um_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void um_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kUmThreads, 1) octant_umma_kernel(const OctUmmaArgs a) {
  extern __shared__ __align__(16) unsigned char um_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x / a.nsplit, sp = blockIdx.x - c * a.nsplit;
  const int units = a.nk1 * a.mt;
  const int u0 = blockIdx.y * a.per, u1 = min(units, u0 + a.per);
  if (u0 >= u1) return;                                   // uniform: before any allocation
  const CompMeta<float> m = a.meta[c];
  const int r2 = m.r2, r3 = m.r3, H2 = a.H2, H3 = a.H3;
  const int K = um_k(r3), N = 2 * a.NC, kp = a.kp;
  // 1024-byte aligned operand buffers
  const uint32_t raw_s = smem_u32(um_raw);
  float* base = reinterpret_cast<float*>(um_raw + ((1024u - (raw_s & 1023u)) & 1023u));
  float* Bhi = base;
  float* Blo = Bhi + (size_t)N * kp;
  float* Abuf = Blo + (size_t)N * kp;                     // [buffer][hi, lo][128 kp]
  float* stage = Abuf + (size_t)4 * kUmRows * kp + warp * kUmStage;
  const int r2p = um_r2p(a.r2max);
  float2* U2s = reinterpret_cast<float2*>(Abuf + (size_t)4 * kUmRows * kp + (kUmThreads / 32) * kUmStage);
  float2* Ss = U2s + (size_t)H2 * r2p;                    // [r2][r3max] of the unit's k1
  float2* U3n = Ss + (size_t)a.r2max * a.r3max;           // U3[H3 - 1, q]

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)), "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  // B (hi, lo) of this CTA's columns, eight loads in flight per thread; the U2
  // rows and U3[P3/2, :] of the component; A buffers zeroed (K padding stays 0)
  for (int i0 = tid; i0 < N * K; i0 += 8 * kUmThreads) {
    float2 u[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e * kUmThreads;
      const int j = i / K, k = i - j * K, q = k >> 1;
      u[e] = (i < N * K && q < r3) ? __ldg(m.U3t + (long long)q * H3 + sp * a.NC + (j >> 1))
                                   : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e * kUmThreads;
      if (i < N * K) {
        const int j = i / K, k = i - j * K;
        const float v = (j & 1) ? ((k & 1) ? u[e].x : u[e].y) : ((k & 1) ? -u[e].y : u[e].x);
        const uint32_t hi = um_tf32(v);
        const int o = um_off(j, k, K);
        Bhi[o] = __uint_as_float(hi);
        Blo[o] = __uint_as_float(um_tf32(v - __uint_as_float(hi)));
      }
    }
  }
  for (int i0 = tid; i0 < H2 * r2; i0 += 8 * kUmThreads) {
    float2 u[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e * kUmThreads;
      u[e] = i < H2 * r2 ? __ldg(m.U2 + i) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e * kUmThreads;
      if (i < H2 * r2) {
        const int k2 = i / r2;
        U2s[k2 * r2p + (i - k2 * r2)] = u[e];
      }
    }
  }
  if (tid < r3) U3n[tid] = __ldg(m.U3t + (long long)tid * H3 + (H3 - 1));
  for (int i = tid; i < 4 * kUmRows * kp; i += kUmThreads) Abuf[i] = 0.f;
  fence_proxy_async_smem();
  um_fence_before();
  __syncthreads();
  um_fence_after();
  const uint32_t tmem = tmem_sh;

  // instruction descriptor: D F32, A and B TF32, both K-major, N, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                         ((uint32_t)(kUmRows >> 4) << 24);
  const uint32_t sbo = 32u * K;
  const int row = tid & (kUmRows - 1), qh = tid >> 7;
  const int qa = qh ? (r3 + 1) / 2 : 0, qb = qh ? r3 : (r3 + 1) / 2;
  const bool nyq = sp == a.nsplit - 1;
  int fail_it = -1, fail_u = -1;

  for (int u = u0, it = 0; u <= u1; ++u, ++it) {
    const int b = it & 1;
    float* Ahi = Abuf + (size_t)(2 * b) * kUmRows * kp;
    float* Alo = Ahi + (size_t)kUmRows * kp;
    const int k1l = u / a.mt, k2 = (u - k1l * a.mt) * kUmRows + row;
    if (u < u1) {
      // the slab core S[k1] of the unit (the previous unit's readers passed
      // the barrier after its A-build)
      {
        const float2* S = m.slab + (long long)(a.k1a + k1l) * a.r23;
        for (int i = tid; i < r2 * a.r3max; i += kUmThreads) Ss[i] = __ldg(S + i);
      }
      __syncthreads();
      // W[k2, q] = sum_b U2[k2, b] S[k1][b, q] for this thread's half of q
      float2 w[kUmMaxR3 / 2];
#pragma unroll
      for (int j = 0; j < kUmMaxR3 / 2; ++j) w[j] = make_float2(0.f, 0.f);
      if (k2 < H2) {
        const float2* S = Ss + qa;
        const float2* u2 = U2s + k2 * r2p;
        for (int bb = 0; bb < r2; ++bb) {
          const float2 uv = u2[bb];
          const float2* Sb = S + bb * a.r3max;
#pragma unroll
          for (int j = 0; j < kUmMaxR3 / 2; ++j)
            if (qa + j < qb) w[j] = cmadd(uv, Sb[j], w[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kUmMaxR3 / 2; ++j) {
        if (qa + j < qb) {
          const int o = um_off(row, 2 * (qa + j), K);
          const uint32_t hr = um_tf32(w[j].x), hi = um_tf32(w[j].y);
          *reinterpret_cast<float2*>(Ahi + o) = make_float2(__uint_as_float(hr), __uint_as_float(hi));
          *reinterpret_cast<float2*>(Alo + o) = make_float2(__uint_as_float(um_tf32(w[j].x - __uint_as_float(hr))),
                                                            __uint_as_float(um_tf32(w[j].y - __uint_as_float(hi))));
        }
      }
      fence_proxy_async_smem();
    }
    __syncthreads();
    if (u < u1) {
      if (tid == 0) {
        um_fence_after();
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo);
        const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Blo);
        const uint32_t d = tmem + (uint32_t)(b * N);
        for (int s = 0; s < K / 8; ++s) {
          const uint32_t off = 256u * s;
          const uint64_t dah = um_desc(ah + off, 128, sbo), dal = um_desc(al + off, 128, sbo);
          const uint64_t dbh = um_desc(bh + off, 128, sbo), dbl = um_desc(bl + off, 128, sbo);
          um_mma(d, dah, dbh, idesc, s > 0 ? 1u : 0u);
          um_mma(d, dah, dbl, idesc, 1u);
          um_mma(d, dal, dbh, idesc, 1u);
        }
        um_commit(&mbar[b]);
      }
      // the Nyquist column k3 = H3 - 1 from the A tile (hi + lo is W to ~2^-22)
      if (nyq && tid < kUmRows && k2 < H2) {
        float2 acc = make_float2(0.f, 0.f);
        for (int q = 0; q < r3; ++q) {
          const int o = um_off(row, 2 * q, K);
          const float2 h = *reinterpret_cast<const float2*>(Ahi + o);
          const float2 l = *reinterpret_cast<const float2*>(Alo + o);
          acc = cmadd(make_float2(h.x + l.x, h.y + l.y), U3n[q], acc);
        }
        a.out[(((long long)k1l * H2 + k2) * 6 + c) * H3 + (H3 - 1)] = acc;
      }
    }
    if (it > 0) {
      // drain the previous unit's accumulator (buffer b ^ 1)
      const int pb = b ^ 1, pu = u - 1;
      const bool ok = mbar_wait_bounded(&mbar[pb], (unsigned)((it - 1) >> 1) & 1u, kUmWaitNs);
      if (__syncthreads_or(!ok)) {
        if (tid == 0 && a.err != nullptr) atomicExch(a.err, VIE_ERR_TIMEOUT);
        fail_it = it;
        fail_u = u;
        break;
      }
      um_fence_after();
      const int pk1 = pu / a.mt, prow0 = (pu - pk1 * a.mt) * kUmRows + 32 * (warp & 3);
      const int half = warp >> 2;                         // columns [half NC, (half + 1) NC)
      const uint32_t tw = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(pb * N + half * a.NC);
      for (int ch = 0; ch < a.NC / 16; ++ch) {
        float v[16];
        um_ld16(tw + 16u * ch, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) stage[lane * 17 + i] = v[i];
        __syncwarp();
        // 8 complex per row: lanes 8 r + e store element e of row 4 i + r
        const int e = lane & 7;
        const int kc = sp * a.NC + (half * a.NC + 16 * ch) / 2 + e;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = 4 * i + (lane >> 3), k2o = prow0 + rr;
          if (k2o < H2)
            a.out[(((long long)pk1 * H2 + k2o) * 6 + c) * H3 + kc] =
                make_float2(stage[rr * 17 + 2 * e], stage[rr * 17 + 2 * e + 1]);
        }
        __syncwarp();
      }
      um_fence_before();
    }
  }
  if (fail_it >= 0) {
    // give the MMAs still in flight (the unit waited for, and the one issued
    // after it) their time before the accumulator is freed
    mbar_wait_bounded(&mbar[(fail_it - 1) & 1], (unsigned)((fail_it - 1) >> 1) & 1u, kUmWaitNs);
    if (fail_u < u1) mbar_wait_bounded(&mbar[fail_it & 1], (unsigned)(fail_it >> 1) & 1u, kUmWaitNs);
  }
  __syncthreads();
  if (warp == 0) {
    um_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                 : "memory");
  }
}

}  // namespace vie

// N ranges of the tcgen05 rebuild: nsplit divides P3/2 into NC = (P3/2) /
// nsplit k3 columns per CTA with NC a multiple of 16 and at most 128 (N = 2 NC
// accumulator columns, two accumulators in at most 512 TMEM columns), and the
// operands fit in shared memory.
static bool umma_split_ok(const vie_op* op, int nsplit) {
  using namespace vie;
  const int H3m = op->H[2] - 1;
  if (nsplit < 1 || H3m % nsplit) return false;
  const int NC = H3m / nsplit;
  return NC % 16 == 0 && NC <= 128 &&
         um_smem(2 * NC, um_k(op->rmax[2]), op->H[1], op->rmax[1], op->rmax[2]) <= kUmSmemLimit;
}

int umma_split_options(const vie_op* op, int* out, int cap) {
  int n = 0;
  if (op->rmax[2] > vie::kUmMaxR3 || op->oct32 == nullptr || op->H[2] < 2) return 0;
  for (int s = 1; s <= 16 && n < cap; ++s)
    if (umma_split_ok(op, s)) out[n++] = s;
  return n;
}

int umma_default_ctas(const vie_op* op, int nsplit) {
  return std::max(1, device_sms() / (6 * nsplit));
}

// Launch plan of the tcgen05 rebuild for chunks of nk1 values of k1: the
// autotuner's tiles when it chose some, else the fewest N ranges that fit and
// one CTA per SM; false when the operator's sizes do not fit the kernel.
static bool umma_plan(const vie_op* op, int k1a, int nk1, vie::OctUmmaArgs* a, size_t* smem) {
  using namespace vie;
  int opts[16];
  const int nopt = umma_split_options(op, opts, 16);
  if (nopt == 0) return false;
  int nsplit = opts[0];
  if (op->tune.rb_nsplit > 0 && umma_split_ok(op, op->tune.rb_nsplit)) nsplit = op->tune.rb_nsplit;
  const int H3m = op->H[2] - 1, kp = um_k(op->rmax[2]);
  a->meta = reinterpret_cast<const CompMeta<float>*>(op->meta);
  a->out = op->oct32;
  a->H2 = op->H[1];
  a->H3 = op->H[2];
  a->r2max = op->rmax[1];
  a->r3max = op->rmax[2];
  a->r23 = op->rmax[1] * op->rmax[2];
  a->k1a = k1a;
  a->nk1 = nk1;
  a->mt = (op->H[1] + kUmRows - 1) / kUmRows;
  a->nsplit = nsplit;
  a->NC = H3m / nsplit;
  a->kp = kp;
  int cols = 32;
  while (cols < 4 * a->NC) cols *= 2;                     // two accumulators of N = 2 NC columns
  a->tmem_cols = cols;
  a->err = op->dev_err;
  const int units = nk1 * a->mt;
  const int ctas = op->tune.rb_ctas > 0 ? op->tune.rb_ctas : umma_default_ctas(op, nsplit);
  const int gy = std::max(1, std::min(units, ctas));
  a->per = (units + gy - 1) / gy;
  *smem = um_smem(2 * a->NC, kp, op->H[1], op->rmax[1], op->rmax[2]);
  return true;
}

void umma_tiles(const vie_op* op, int out[2]) {
  vie::OctUmmaArgs a;
  size_t smem = 0;
  out[0] = out[1] = 0;
  if (!op->umma || !umma_plan(op, 0, op->oct_k1, &a, &smem)) return;
  out[0] = a.NC;
  out[1] = (a.nk1 * a.mt + a.per - 1) / a.per;
}

bool umma_rebuild_eligible(const vie_op* op) {
  vie::OctUmmaArgs a;
  size_t smem = 0;
  return umma_plan(op, 0, op->oct_k1, &a, &smem);
}

int launch_octant_umma(const vie_op* op, int k1a, int nk1, cudaStream_t s) {
  vie::OctUmmaArgs a;
  size_t smem = 0;
  if (!umma_plan(op, k1a, nk1, &a, &smem)) {
    set_error("the tcgen05 rebuild does not support this operator's sizes");
    return VIE_ERR_ARG;
  }
  const int gy = (nk1 * a.mt + a.per - 1) / a.per;
  vie::octant_umma_kernel<<<dim3(6 * a.nsplit, gy), vie::kUmThreads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "tcgen05 rebuild launch");
}

int umma_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(vie::octant_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)vie::kUmSmemLimit);
  return e == cudaSuccess ? VIE_OK : cuda_status(e, "tcgen05 rebuild attributes");
}
