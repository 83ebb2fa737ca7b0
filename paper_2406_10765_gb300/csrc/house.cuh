// Device helpers of the blocked Householder reduction shared by its kernels
// (dense.cu: the chained column kernels and the cooperative FP64 panel;
// hemv_tc.cu: the tensor-core Hermitian product and the cooperative
// tensor-core panel): warp and block sums, complex multiply-adds written as
// four FMAs, the panel's alpha, the reflector entries, programmatic
// dependent launch.
#pragma once
#include "pw_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// block-wide sum of one double (blockDim.x multiple of 32, <= 1024)
__device__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// s += a b and s += conj(a) b, four FMAs each
__device__ __forceinline__ void cmac(double2 &s, double2 a, double2 b) {
  s.x = fma(a.x, b.x, s.x);
  s.x = fma(-a.y, b.y, s.x);
  s.y = fma(a.x, b.y, s.y);
  s.y = fma(a.y, b.x, s.y);
}
__device__ __forceinline__ void cmacc(double2 &s, double2 a, double2 b) {
  s.x = fma(a.x, b.x, s.x);
  s.x = fma(a.y, b.y, s.x);
  s.y = fma(a.x, b.y, s.y);
  s.y = fma(-a.y, b.x, s.y);
}

// alpha = -1/2 tau (p^H v) from the per-block partial dots (block-wide sum)
// (stride: the partial sums run over `stride` threads, blockDim.x by default;
// the cooperative panel kernel uses k_pcol's 128 to reproduce its sums)
__device__ double2 panel_alpha(const double2 *dotpart, int ndot, double2 t, double *sh, int stride = 0) {
  double sr = 0.0, si = 0.0;
  const int st = stride > 0 ? stride : (int)blockDim.x;
  for (int q = threadIdx.x; q < ndot && (int)threadIdx.x < st; q += st) {
    const double2 v = __ldcg(&dotpart[q]);
    sr += v.x;
    si += v.y;
  }
  sr = block_sum(sr, sh);
  si = block_sum(si, sh);
  return cmul(make_double2(-0.5 * t.x, -0.5 * t.y), make_double2(sr, si));
}

// v_c entry x (x = row - (c+1)) from the stored column and the scale
__device__ __forceinline__ double2 refl_entry(const double2 *xcol, int x, double2 scal) {
  return x == 0 ? make_double2(1.0, 0.0) : cmul(xcol[x], scal);
}

// Reflector of x = (alpha, x_2..) with ||x_2..||^2 = xn2: beta, tau and the
// scale s of v = x s below its unit head (tau = 0 and s = 0 when x is
// already a multiple of the first unit vector with a real head)
__device__ __forceinline__ void reflector_scalars(double xn2, double2 alpha, double &beta, double2 &tk,
                                                  double2 &scal) {
  if (xn2 == 0.0 && alpha.y == 0.0) {
    beta = alpha.x;
    tk = make_double2(0.0, 0.0);
    scal = make_double2(0.0, 0.0);
  } else {
    beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
    tk = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
    const double2 den = make_double2(alpha.x - beta, alpha.y);
    const double qq = 1.0 / (den.x * den.x + den.y * den.y);
    scal = make_double2(den.x * qq, -den.y * qq);
  }
}

}  // namespace
