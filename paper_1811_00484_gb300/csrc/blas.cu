// Element-wise kernels: the contrast gradient of the field misfit and the
// incident field of z-directed point dipoles.
#include "vie_internal.cuh"

namespace {

// grad[v] = scale sum_b sum_a lam[b, a, v] conj(E[b, a, v])
template <typename T>
__global__ void gradient_kernel(const cx<T>* lam, const cx<T>* E, cx<T>* grad, int B, T scale,
                                long long nvox) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
       v += (long long)gridDim.x * blockDim.x) {
    cx<T> acc = czero<cx<T>>();
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < 3; ++a) {
        const long long i = ((long long)b * 3 + a) * nvox + v;
        acc = conj_madd(E[i], lam[i], acc);      // lam * conj(E)
      }
    grad[v] = scale * acc;
  }
}

// e_a(r) = (k0^2 delta_az + d_a d_z) g(r - r_s), g = exp(-i k0 R)/(4 pi R), at voxel centres
template <typename T>
__global__ void dipole_kernel(const double* src, int B, cx<T>* out, int n1, int n2, int n3, double h,
                              double k0) {
  const long long nvox = (long long)n1 * n2 * n3;
  const long long total = nvox * B;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / nvox);
    const long long v = idx % nvox;
    const int i3 = (int)(v % n3), i2 = (int)((v / n3) % n2), i1 = (int)(v / ((long long)n2 * n3));
    const double R[3] = {(i1 + 0.5 - 0.5 * n1) * h - src[3 * b], (i2 + 0.5 - 0.5 * n2) * h - src[3 * b + 1],
                         (i3 + 0.5 - 0.5 * n3) * h - src[3 * b + 2]};
    const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    const double ir = 1.0 / r;
    double sn, cs;
    sincos(k0 * r, &sn, &cs);
    const double2 g = make_double2(cs * ir * (0.25 / 3.14159265358979323846),
                                   -sn * ir * (0.25 / 3.14159265358979323846));
    const double2 diag = make_double2(k0 * k0 - ir * ir, -k0 * ir);
    const double2 dyad = make_double2(-k0 * k0 + 3.0 * ir * ir, 3.0 * k0 * ir);
    for (int a = 0; a < 3; ++a) {
      const double rr = (R[a] * ir) * (R[2] * ir);
      double2 f = make_double2(dyad.x * rr, dyad.y * rr);
      if (a == 2) f = f + diag;
      const double2 e = g * f;
      cx<T> o;
      o.x = (T)e.x;
      o.y = (T)e.y;
      out[((long long)b * 3 + a) * nvox + v] = o;
    }
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

template <typename T>
int launch_gradient(const cx<T>* lam, const cx<T>* E, cx<T>* grad, int B, double scale,
                    long long nvox, cudaStream_t s) {
  gradient_kernel<T><<<blocks_for(nvox), 256, 0, s>>>(lam, E, grad, B, (T)scale, nvox);
  VIE_CUDA(cudaGetLastError());
  return VIE_OK;
}

template <typename T>
int launch_dipole(const vie_op* op, const double* src_dev, int B, cx<T>* out, cudaStream_t s) {
  const long long total = (long long)op->n[0] * op->n[1] * op->n[2] * B;
  dipole_kernel<T><<<blocks_for(total), 256, 0, s>>>(src_dev, B, out, op->n[0], op->n[1], op->n[2],
                                                     op->grid.h, op->k0);
  VIE_CUDA(cudaGetLastError());
  return VIE_OK;
}

template int launch_gradient<float>(const float2*, const float2*, float2*, int, double, long long, cudaStream_t);
template int launch_gradient<double>(const double2*, const double2*, double2*, int, double, long long, cudaStream_t);
template int launch_dipole<float>(const vie_op*, const double*, int, float2*, cudaStream_t);
template int launch_dipole<double>(const vie_op*, const double*, int, double2*, cudaStream_t);
