// Register-resident line FFTs for the local part of H psi (Sec. II-B), used
// when every grid dimension is N = L * R with L a power of two up to 32 lanes
// and R = N / L <= 18 values per lane (N = 2^a 3^b).
//
// A line x[0..N) is held by a group of L lanes, lane l owning x[l + L r],
// r < R.  With n = l + L r and k = k2 + R k1:
//   1. in-lane DFT of length R over r            -> Y[l][k2]
//   2. twiddle Y[l][k2] *= w_N^(l k2)
//   3. DFT of length L across the lanes for each k2 (radix-2 decimation in
//      frequency with warp shuffles), which leaves X[k2 + R k1] in lane
//      bitrev(k1).
// Each pass loads a line from shared memory in the strided order above and
// stores the result at its natural position, so a whole 1-D transform is one
// shared-memory read and one write, with no block barrier inside it.
//
// The kernels mirror the generic Stockham path (k_sphere_to_z, k_plane,
// k_z_to_sphere): same data layout, same sign and scaling conventions.
//
// A plan is one factorisation N = L R; several plans exist per grid size
// (fewer lanes: fewer shuffle stages, longer in-lane DFTs) and the cell picks
// one (default: the first listed, or the autotuner's choice).  Each
// fft_reg_*.cu instantiates the kernels of a few plans, so the translation
// units compile in parallel.
#pragma once
#include <string.h>

#include <algorithm>

#include "pw_internal.cuh"

namespace {

constexpr int log2c(int x) { return x <= 1 ? 0 : 1 + log2c(x / 2); }

template <typename C> __device__ __forceinline__ C czero_r() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> __device__ __forceinline__ C conj_if(C w, bool inv) {
  if (inv) w.y = -w.y;
  return w;
}
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}
__device__ __forceinline__ double2 shfl_xor2(double2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// ---- in-lane DFTs: y_q = sum_p x_p exp(s 2 pi i p q / R), s = -1 forward, +1 inverse
template <typename C, int R, int N> struct LaneDFT;

template <typename C, int N> struct LaneDFT<C, 1, N> {
  static __device__ __forceinline__ void run(C (&)[1], const C *, bool) {}
};
template <typename C, int N> struct LaneDFT<C, 2, N> {
  static __device__ __forceinline__ void run(C (&v)[2], const C *, bool) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <typename C, int N> struct LaneDFT<C, 3, N> {
  static __device__ __forceinline__ void run(C (&v)[3], const C *, bool inv) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.86602540378443864676;   // sqrt(3)/2
    const C a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m, t;
    m.x = a.x - (T)0.5 * s.x;
    m.y = a.y - (T)0.5 * s.y;
    if (inv) { t.x = -h * d.y; t.y = h * d.x; } else { t.x = h * d.y; t.y = -h * d.x; }
    v[0] = cadd(a, s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
  }
};
template <typename C, int N> struct LaneDFT<C, 4, N> {
  static __device__ __forceinline__ void run(C (&v)[4], const C *, bool inv) {
    const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    C jd;   // -i d13 (forward) or +i d13 (inverse)
    if (inv) { jd.x = -d13.y; jd.y = d13.x; } else { jd.x = d13.y; jd.y = -d13.x; }
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, jd);
    v[3] = csub(d02, jd);
  }
};
// composite R = P Q: index r = p + P q, output k = kq + Q kp; tw holds w_N^m
template <typename C, int R, int N> struct LaneDFT {
  static constexpr int P = (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 3;
  static constexpr int Q = R / P;
  static __device__ __forceinline__ void run(C (&v)[R], const C *tw, bool inv) {
    C t[P][Q];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      C u[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) u[q] = v[p + P * q];
      LaneDFT<C, Q, N>::run(u, tw, inv);
#pragma unroll
      for (int kq = 0; kq < Q; ++kq) {
        C x = u[kq];
        if (p > 0 && kq > 0) x = cmul(x, conj_if(tw[p * kq * (N / R)], inv));
        t[p][kq] = x;
      }
    }
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) {
      C u[P];
#pragma unroll
      for (int p = 0; p < P; ++p) u[p] = t[p][kq];
      LaneDFT<C, P, N>::run(u, tw, inv);
#pragma unroll
      for (int kp = 0; kp < P; ++kp) v[kq + Q * kp] = u[kp];
    }
  }
};

// per-lane twiddles of a line: w_N^(l k2) and the shuffle-stage factors
template <typename C, int L, int R> struct LineTw {
  static constexpr int N = L * R, LG = log2c(L);
  C lt[R > 1 ? R - 1 : 1];
  C st[LG > 0 ? LG : 1];
  __device__ __forceinline__ void init(const C *tw, int l) {
#pragma unroll
    for (int k2 = 1; k2 < R; ++k2) lt[k2 - 1] = tw[l * k2];
    int s = 0;
#pragma unroll
    for (int h = L / 2; h >= 1; h >>= 1, ++s) st[s] = tw[(l & (h - 1)) * (N / (2 * h))];
  }
  // natural index of register k2 of lane l after line_fft
  __device__ __forceinline__ int out_index(int k2, int l) const {
    if (LG == 0) return k2;
    return k2 + R * (int)(__brev((unsigned)l) >> (32 - LG));
  }
};

template <typename C, int L, int R>
__device__ __forceinline__ void line_fft(C (&v)[R], const LineTw<C, L, R> &t, const C *tw, int l,
                                         bool inv) {
  LaneDFT<C, R, L * R>::run(v, tw, inv);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], conj_if(t.lt[k2 - 1], inv));
  int s = 0;
#pragma unroll
  for (int h = L / 2; h >= 1; h >>= 1, ++s) {
    const C w = conj_if(t.st[s], inv);
    const bool upper = (l & h) != 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const C p = shfl_xor2(v[r], h);
      v[r] = upper ? cmul(csub(p, v[r]), w) : cadd(v[r], p);
    }
  }
}

template <typename C> __device__ __forceinline__ C from64r(double2 a);
template <> __device__ __forceinline__ double2 from64r<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from64r<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

constexpr int ZCB = 16;          // z-lines per block in K1 / K3
constexpr int ZTHREADS = 256;
// threads of the plane kernels: 512 for FP32 lines of up to 9 values per
// lane; 256 (twice the registers per thread) for longer FP32 lines and FP64
template <typename C, int R> struct RegPlaneThreads { static constexpr int value = R >= 12 ? 256 : 512; };
template <int R> struct RegPlaneThreads<double2, R> { static constexpr int value = 256; };

// FFT of `nlines` lines held in shared memory (line i at buf + i * ls, element
// e at e * es), all warps of the block; lines are processed G = 32 / L at a
// time per warp, every lane taking part in the shuffles
template <typename C, int L, int R>
__device__ __forceinline__ void fft_lines_reg(C *buf, int nlines, int ls, int es, const C *tw,
                                              const LineTw<C, L, R> &t, bool inv) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gid = lane / L, l = lane % L;
  for (int base = warp * G; base < nlines; base += nw * G) {
    const int line = base + gid;
    const bool act = line < nlines;
    C *p = buf + (long)(act ? line : 0) * ls;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = act ? p[(l + L * r) * es] : czero_r<C>();
    line_fft<C, L, R>(v, t, tw, l, inv);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) p[t.out_index(r, l) * es] = v[r];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- K1 ----
// z-columns bx*ZCB.. of one band: scatter the sphere into the z-lines,
// inverse FFT along z, store the z-pencils Zb[z][column]
template <typename C, int L, int R>
__device__ __forceinline__ void sphere_to_z_body(int bx, const double2 *__restrict__ p,
                                                 const int *__restrict__ colstart, const int *__restrict__ gcol,
                                                 const int *__restrict__ gz, int ncol, const C *__restrict__ twz,
                                                 C *__restrict__ Zb) {
  constexpr int Nz = L * R, ls = Nz + 1;
  __shared__ C lines[ZCB * ls];
  const int c0 = bx * ZCB;
  const int nc = min(ZCB, ncol - c0);
  LineTw<C, L, R> t;
  t.init(twz, (threadIdx.x & 31) % L);
  for (int i = threadIdx.x; i < nc * ls; i += blockDim.x) lines[i] = czero_r<C>();
  __syncthreads();
  const int g0 = colstart[c0], g1 = colstart[c0 + nc];
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x)
    lines[(gcol[g] - c0) * ls + gz[g]] = from64r<C>(p[g]);
  __syncthreads();
  fft_lines_reg<C, L, R>(lines, nc, ls, 1, twz, t, true);
  __syncthreads();
  for (int i = threadIdx.x; i < nc * Nz; i += blockDim.x) {
    const int z = i / nc, cl = i % nc;
    Zb[(long)z * ncol + c0 + cl] = lines[cl * ls + z];
  }
}

template <typename C, int L, int R>
__global__ void __launch_bounds__(ZTHREADS) k_sphere_to_z_reg(const double2 *__restrict__ psi, int ld,
                                                              const int *__restrict__ colstart,
                                                              const int *__restrict__ gcol,
                                                              const int *__restrict__ gz, int ncol,
                                                              const C *__restrict__ twz,
                                                              C *__restrict__ Z) {
  const int b = blockIdx.y;
  sphere_to_z_body<C, L, R>(blockIdx.x, psi + (long)b * ld, colstart, gcol, gz, ncol, twz,
                            Z + (long)b * (L * R) * ncol);
}

// ---------------------------------------------------------------- K2 ----
// Plane layouts in shared memory: full, the N x N plane with row stride N + 1;
// compact (CP), only the x-columns that meet the sphere (x in [-mxmax,
// mxmax], column x + mxmax) with an odd row stride, plus one N-point row
// buffer per line group of each warp for the x transforms.  After the y
// transforms the other x-columns are zero, and after the x transforms only
// the sphere's x-columns are read again, so the compact plane holds
// everything the pass needs (an FP64 plane of 128 x 85 instead of 128 x 129).
__host__ __device__ inline int compact_stride(int mxmax) { return (2 * mxmax + 1) | 1; }
template <typename C, int L, int R>
__host__ __device__ inline size_t plane_smem_bytes(int mxmax, bool cp, int nthreads) {
  constexpr int N = L * R;
  if (!cp) return (size_t)N * (N + 1) * sizeof(C);
  return ((size_t)N * compact_stride(mxmax) + (size_t)(nthreads / 32) * (32 / L) * N) * sizeof(C);
}

// plane z of one band: its z-pencils Zp[column] through the y and x
// transforms, V(r), and back (P: the block's dynamic shared memory)
template <typename C, typename T, int L, int R, bool CP>
__device__ __forceinline__ void plane_body(C *P, int z, C *__restrict__ Zp, int ncol, const int *__restrict__ colxy,
                                           int mxmax, const C *__restrict__ twx, const T *__restrict__ V) {
  constexpr int N = L * R, G = 32 / L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gid = lane / L, l = lane % L;
  const int nxe = 2 * mxmax + 1;
  const int ps = CP ? compact_stride(mxmax) : N + 1;
  // plane column of x in [0, N): the x index itself, or its place in the
  // compact sphere extent (valid for x <= mxmax or x >= N - mxmax)
  auto pcol = [&](int x) { return CP ? (x <= mxmax ? x + mxmax : x - N + mxmax) : x; };
  auto in_ext = [&](int x) { return !CP || x <= mxmax || x >= N - mxmax; };
  C *rowbuf = P + (long)N * ps + (long)(warp * G + gid) * N;   // compact only
  LineTw<C, L, R> t;
  t.init(twx, l);
  for (int i = threadIdx.x; i < N * ps; i += blockDim.x) P[i] = czero_r<C>();
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int xy = colxy[c];
    P[(xy / N) * ps + pcol(xy % N)] = Zp[c];
  }
  __syncthreads();
  // inverse FFT along y on the x-columns that meet the sphere (x in [-mxmax, mxmax])
  for (int base = warp * G; base < nxe; base += nw * G) {
    const int xi = base + gid;
    const bool act = xi < nxe;
    int x = xi - mxmax;
    if (x < 0) x += N;
    C *col = P + (act ? pcol(x) : 0);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = act ? col[(l + L * r) * ps] : czero_r<C>();
    line_fft<C, L, R>(v, t, twx, l, true);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) col[t.out_index(r, l) * ps] = v[r];
    }
  }
  __syncthreads();
  // each row: inverse FFT along x, V(r), forward FFT along x
  const T *Vz = V + (long)z * N * N;
  for (int base = warp * G; base < N; base += nw * G) {
    const int y = base + gid;
    const bool act = y < N;
    C *row = P + (long)(act ? y : 0) * ps;
    C *mid = CP ? rowbuf : row;               // the row between the two transforms, natural x order
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int x = l + L * r;
      v[r] = act && in_ext(x) ? row[pcol(x)] : czero_r<C>();
    }
    line_fft<C, L, R>(v, t, twx, l, true);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int x = t.out_index(r, l);
        const T vv = Vz[(long)y * N + x];
        C e = v[r];
        e.x *= vv;
        e.y *= vv;
        mid[x] = e;
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = act ? mid[l + L * r] : czero_r<C>();
    line_fft<C, L, R>(v, t, twx, l, false);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int x = t.out_index(r, l);
        if (in_ext(x)) row[pcol(x)] = v[r];
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // forward FFT along y on the same x-columns
  for (int base = warp * G; base < nxe; base += nw * G) {
    const int xi = base + gid;
    const bool act = xi < nxe;
    int x = xi - mxmax;
    if (x < 0) x += N;
    C *col = P + (act ? pcol(x) : 0);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = act ? col[(l + L * r) * ps] : czero_r<C>();
    line_fft<C, L, R>(v, t, twx, l, false);
    if (act) {
#pragma unroll
      for (int r = 0; r < R; ++r) col[t.out_index(r, l) * ps] = v[r];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int xy = colxy[c];
    Zp[c] = P[(xy / N) * ps + pcol(xy % N)];
  }
}

template <typename C, typename T, int L, int R, bool CP>
__global__ void __launch_bounds__(RegPlaneThreads<C, R>::value) k_plane_reg(C *__restrict__ Z, int ncol,
                                                                         const int *__restrict__ colxy,
                                                                         int mxmax, const C *__restrict__ twx,
                                                                         int Nz, const T *__restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int z = blockIdx.x, b = blockIdx.y;
  plane_body<C, T, L, R, CP>(reinterpret_cast<C *>(smem_raw), z, Z + ((long)b * Nz + z) * ncol, ncol, colxy,
                             mxmax, twx, V);
}

// ---------------------------------------------------------------- K3 ----
// z-columns bx*ZCB.. of one band: forward FFT along z, gather onto the
// sphere, hpsi = kin psi + scale (V psi)
template <typename C, int L, int R>
__device__ __forceinline__ void z_to_sphere_body(int bx, const C *__restrict__ Zb, int ncol,
                                                 const C *__restrict__ twz, const int *__restrict__ colstart,
                                                 const int *__restrict__ gcol, const int *__restrict__ gz,
                                                 const double *__restrict__ kin, const double2 *__restrict__ p,
                                                 double2 *__restrict__ h, double scale) {
  constexpr int Nz = L * R, ls = Nz + 1;
  __shared__ C lines[ZCB * ls];
  const int c0 = bx * ZCB;
  const int nc = min(ZCB, ncol - c0);
  LineTw<C, L, R> t;
  t.init(twz, (threadIdx.x & 31) % L);
  for (int i = threadIdx.x; i < nc * Nz; i += blockDim.x) {
    const int z = i / nc, cl = i % nc;
    lines[cl * ls + z] = Zb[(long)z * ncol + c0 + cl];
  }
  __syncthreads();
  fft_lines_reg<C, L, R>(lines, nc, ls, 1, twz, t, false);
  __syncthreads();
  const int g0 = colstart[c0], g1 = colstart[c0 + nc];
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const C v = lines[(gcol[g] - c0) * ls + gz[g]];
    const double k = kin[g];
    const double2 x = p[g];
    h[g] = make_double2(k * x.x + scale * (double)v.x, k * x.y + scale * (double)v.y);
  }
}

template <typename C, int L, int R>
__global__ void __launch_bounds__(ZTHREADS) k_z_to_sphere_reg(const C *__restrict__ Z, int ncol,
                                                              const C *__restrict__ twz,
                                                              const int *__restrict__ colstart,
                                                              const int *__restrict__ gcol,
                                                              const int *__restrict__ gz,
                                                              const double *__restrict__ kin,
                                                              const double2 *__restrict__ psi, int ld,
                                                              double2 *__restrict__ hpsi, double scale) {
  const int b = blockIdx.y;
  z_to_sphere_body<C, L, R>(blockIdx.x, Z + (long)b * (L * R) * ncol, ncol, twz, colstart, gcol, gz, kin,
                            psi + (long)b * ld, hpsi + (long)b * ld, scale);
}

// ------------------------------------------------- several cells at once ----
// The local part of H psi for bands of several cells (requests) that share
// the grid size and plan, in one launch per kernel: blockIdx.y runs over the
// bands of all cells, each block finds its cell in the job table (passed by
// value) and runs the same body as the one-cell kernels, so every band's
// arithmetic is that of the one-cell launch.
template <typename C, typename T> struct RegJob {
  const double2 *psi;
  double2 *hpsi;
  C *Z;
  const T *V;
  const double *kin;
  const int *colstart, *gcol, *gz, *colxy;
  const C *twz, *twx;
  int ld, nb, b0, ncol, mxmax, pad;
  double scale;
};
template <typename C, typename T> struct RegJobs {
  int n, pad;
  RegJob<C, T> j[PW_FFT_BATCH_MAX];
};
template <typename C, typename T>
__device__ __forceinline__ int job_of(const RegJobs<C, T> &J, int band) {
  int j = 0;
  while (j + 1 < J.n && band >= J.j[j + 1].b0) ++j;
  return j;
}

template <typename C, typename T, int L, int R>
__global__ void __launch_bounds__(ZTHREADS) k_sphere_to_z_multi(const __grid_constant__ RegJobs<C, T> J) {
  const RegJob<C, T> &q = J.j[job_of(J, blockIdx.y)];
  if ((int)blockIdx.x * ZCB >= q.ncol) return;
  const int b = blockIdx.y - q.b0;
  sphere_to_z_body<C, L, R>(blockIdx.x, q.psi + (long)b * q.ld, q.colstart, q.gcol, q.gz, q.ncol, q.twz,
                            q.Z + (long)b * (L * R) * q.ncol);
}
template <typename C, typename T, int L, int R, bool CP>
__global__ void __launch_bounds__(RegPlaneThreads<C, R>::value) k_plane_multi(const __grid_constant__ RegJobs<C, T> J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RegJob<C, T> &q = J.j[job_of(J, blockIdx.y)];
  const int z = blockIdx.x, b = blockIdx.y - q.b0;
  plane_body<C, T, L, R, CP>(reinterpret_cast<C *>(smem_raw), z, q.Z + ((long)b * (L * R) + z) * q.ncol, q.ncol,
                             q.colxy, q.mxmax, q.twx, q.V);
}
template <typename C, typename T, int L, int R>
__global__ void __launch_bounds__(ZTHREADS) k_z_to_sphere_multi(const __grid_constant__ RegJobs<C, T> J) {
  const RegJob<C, T> &q = J.j[job_of(J, blockIdx.y)];
  if ((int)blockIdx.x * ZCB >= q.ncol) return;
  const int b = blockIdx.y - q.b0;
  z_to_sphere_body<C, L, R>(blockIdx.x, q.Z + (long)b * (L * R) * q.ncol, q.ncol, q.twz, q.colstart, q.gcol,
                            q.gz, q.kin, q.psi + (long)b * q.ld, q.hpsi + (long)b * q.ld, q.scale);
}

template <typename C> __host__ __device__ inline const C *twtab(const pw_fft_axis &a);
template <> inline const double2 *twtab<double2>(const pw_fft_axis &a) { return a.tw64; }
template <> inline const float2 *twtab<float2>(const pw_fft_axis &a) { return a.tw32; }

template <typename C, typename T, int L, int R, bool CP>
pw_status run_batch(pw_cell *c, const double2 *psi, int ld, int nbb, double2 *hpsi, C *Z, const T *V,
                    double scale, cudaStream_t st) {
  constexpr int N = L * R;
  if (2 * c->mxmax + 1 > N) return PW_ERR_ARG;
  const size_t plane_bytes = plane_smem_bytes<C, L, R>(c->mxmax, CP, RegPlaneThreads<C, R>::value);
  if (plane_bytes > 227 * 1024) return PW_ERR_ARG;
  // the opt-in is set to the largest size (threads launching this plan for
  // cells of different sphere extents then never lower it under each other)
  if (plane_bytes > 48 * 1024)
    PW_CUDA(cudaFuncSetAttribute(k_plane_reg<C, T, L, R, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
  const dim3 gcols((c->ncol + ZCB - 1) / ZCB, nbb);
  pw_count_launch();
  k_sphere_to_z_reg<C, L, R><<<gcols, ZTHREADS, 0, st>>>(psi, ld, c->d_colstart, c->d_gcol, c->d_gz,
                                                         c->ncol, twtab<C>(c->ax[2]), Z);
  pw_count_launch();
  k_plane_reg<C, T, L, R, CP><<<dim3(N, nbb), RegPlaneThreads<C, R>::value, plane_bytes, st>>>(
      Z, c->ncol, c->d_colxy, c->mxmax, twtab<C>(c->ax[0]), N, V);
  pw_count_launch();
  k_z_to_sphere_reg<C, L, R><<<gcols, ZTHREADS, 0, st>>>(Z, c->ncol, twtab<C>(c->ax[2]), c->d_colstart,
                                                         c->d_gcol, c->d_gz, c->d_kin, psi, ld, hpsi,
                                                         scale);
  return pw_check_launch("local part (register FFT)");
}

// ------------------------------------------------------------ density ----
// Per z-plane and band group: psi_j(r) of the plane by inverse FFTs along y
// and x (as in K2), then acc += w_j |psi_j(r)|^2.  Each thread owns fixed
// plane points, so the sum over the group's bands runs in a fixed order in
// registers; part[g][z][y][x] holds each group's sum.
template <typename C, int L, int R>
__global__ void __launch_bounds__(RegPlaneThreads<C, R>::value) k_density_reg(const C *__restrict__ Z, int ncol,
                                                                           const int *__restrict__ colxy,
                                                                           int mxmax, const C *__restrict__ twx,
                                                                           int nbb, const double *__restrict__ occ,
                                                                           double *__restrict__ part) {
  typedef decltype(Z[0].x) T;
  constexpr int N = L * R, pxs = N + 1, G = 32 / L;
  constexpr int NT = RegPlaneThreads<C, R>::value;
  constexpr int ACC = (N * N + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *P = reinterpret_cast<C *>(smem_raw);
  const int z = blockIdx.x, grp = blockIdx.y, ngroups = gridDim.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gid = lane / L, l = lane % L;
  LineTw<C, L, R> t;
  t.init(twx, l);
  T acc[ACC];
#pragma unroll
  for (int k = 0; k < ACC; ++k) acc[k] = 0;
  const int nxe = 2 * mxmax + 1;
  for (int j = grp; j < nbb; j += ngroups) {
    const T w = occ ? (T)occ[j] : (T)1;
    const C *Zp = Z + ((long)j * N + z) * ncol;
    for (int i = threadIdx.x; i < N * pxs; i += blockDim.x) P[i] = czero_r<C>();
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      const int xy = colxy[c];
      P[(xy / N) * pxs + (xy % N)] = Zp[c];
    }
    __syncthreads();
    for (int base = warp * G; base < nxe; base += nw * G) {
      const int xi = base + gid;
      const bool act = xi < nxe;
      int x = xi - mxmax;
      if (x < 0) x += N;
      C *col = P + (act ? x : 0);
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = act ? col[(l + L * r) * pxs] : czero_r<C>();
      line_fft<C, L, R>(v, t, twx, l, true);
      if (act) {
#pragma unroll
        for (int r = 0; r < R; ++r) col[t.out_index(r, l) * pxs] = v[r];
      }
    }
    __syncthreads();
    for (int base = warp * G; base < N; base += nw * G) {
      const int y = base + gid;
      const bool act = y < N;
      C *row = P + (long)(act ? y : 0) * pxs;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = act ? row[l + L * r] : czero_r<C>();
      line_fft<C, L, R>(v, t, twx, l, true);
      if (act) {
#pragma unroll
        for (int r = 0; r < R; ++r) row[t.out_index(r, l)] = v[r];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ACC; ++k) {
      const int i = threadIdx.x + k * NT;
      if (i < N * N) {
        const C e = P[(i / N) * pxs + (i % N)];
        acc[k] += w * (e.x * e.x + e.y * e.y);
      }
    }
    __syncthreads();
  }
  double *out = part + ((long)grp * N + z) * N * N;
#pragma unroll
  for (int k = 0; k < ACC; ++k) {
    const int i = threadIdx.x + k * NT;
    if (i < N * N) out[i] = (double)acc[k];
  }
}

template <typename C, int L, int R>
pw_status density_batch(pw_cell *c, const double2 *psi, int ld, int nbb, C *Z, const double *occ, int ngroups,
                        double *part, cudaStream_t st) {
  constexpr int N = L * R;
  const size_t plane_bytes = (size_t)N * (N + 1) * sizeof(C);
  if (plane_bytes > 227 * 1024) return PW_ERR_ARG;
  if (plane_bytes > 48 * 1024)
    PW_CUDA(cudaFuncSetAttribute(k_density_reg<C, L, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
  const dim3 gcols((c->ncol + ZCB - 1) / ZCB, nbb);
  pw_count_launch();
  k_sphere_to_z_reg<C, L, R><<<gcols, ZTHREADS, 0, st>>>(psi, ld, c->d_colstart, c->d_gcol, c->d_gz,
                                                         c->ncol, twtab<C>(c->ax[2]), Z);
  pw_count_launch();
  k_density_reg<C, L, R><<<dim3(N, ngroups), RegPlaneThreads<C, R>::value, plane_bytes, st>>>(
      Z, c->ncol, c->d_colxy, c->mxmax, twtab<C>(c->ax[0]), nbb, occ, part);
  return pw_check_launch("density (register FFT)");
}

// several cells' bands in one launch per kernel (the cells share this plan)
template <typename C, typename T, int L, int R, bool CP>
pw_status run_multi(const pw_fft_job *jobs, int n, cudaStream_t st) {
  constexpr int N = L * R;
  if (n < 1 || n > PW_FFT_BATCH_MAX) return PW_ERR_ARG;
  RegJobs<C, T> J;
  memset(&J, 0, sizeof J);
  J.n = n;
  int bands = 0, colblocks = 0;
  size_t plane_bytes = 0;
  for (int i = 0; i < n; ++i) {
    pw_cell *c = jobs[i].c;
    if (c->N[0] != N || c->N[1] != N || c->N[2] != N || 2 * c->mxmax + 1 > N) return PW_ERR_ARG;
    RegJob<C, T> &q = J.j[i];
    q.psi = jobs[i].psi;
    q.hpsi = jobs[i].hpsi;
    q.Z = (C *)jobs[i].Z;
    q.V = (const T *)(sizeof(C) == sizeof(float2) ? (const void *)c->d_Vf : (const void *)c->d_V);
    q.kin = c->d_kin;
    q.colstart = c->d_colstart;
    q.gcol = c->d_gcol;
    q.gz = c->d_gz;
    q.colxy = c->d_colxy;
    q.twz = twtab<C>(c->ax[2]);
    q.twx = twtab<C>(c->ax[0]);
    q.ld = jobs[i].ld;
    q.nb = jobs[i].nb;
    q.b0 = bands;
    q.ncol = c->ncol;
    q.mxmax = c->mxmax;
    q.scale = jobs[i].scale;
    bands += jobs[i].nb;
    colblocks = std::max(colblocks, (c->ncol + ZCB - 1) / ZCB);
    plane_bytes = std::max(plane_bytes, plane_smem_bytes<C, L, R>(c->mxmax, CP, RegPlaneThreads<C, R>::value));
  }
  if (plane_bytes > 227 * 1024) return PW_ERR_ARG;
  if (plane_bytes > 48 * 1024)
    PW_CUDA(cudaFuncSetAttribute(k_plane_multi<C, T, L, R, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024));
  pw_count_launch();
  k_sphere_to_z_multi<C, T, L, R><<<dim3(colblocks, bands), ZTHREADS, 0, st>>>(J);
  pw_count_launch();
  k_plane_multi<C, T, L, R, CP><<<dim3(N, bands), RegPlaneThreads<C, R>::value, plane_bytes, st>>>(J);
  pw_count_launch();
  k_z_to_sphere_multi<C, T, L, R><<<dim3(colblocks, bands), ZTHREADS, 0, st>>>(J);
  return pw_check_launch("local part of several cells (register FFT)");
}

template <int L, int R, bool CP>
pw_status reg_multi64(const pw_fft_job *jobs, int n, cudaStream_t st) {
  return run_multi<double2, double, L, R, CP>(jobs, n, st);
}
template <int L, int R, bool CP>
pw_status reg_multi32(const pw_fft_job *jobs, int n, cudaStream_t st) {
  return run_multi<float2, float, L, R, CP>(jobs, n, st);
}

// entry points of one plan, as stored in the plan tables
template <int L, int R, bool CP>
pw_status reg_run64(pw_cell *c, const double2 *psi, int ld, int nbb, double2 *hpsi, void *Z, double scale,
                    cudaStream_t st) {
  return run_batch<double2, double, L, R, CP>(c, psi, ld, nbb, hpsi, (double2 *)Z, c->d_V, scale, st);
}
template <int L, int R, bool CP>
pw_status reg_run32(pw_cell *c, const double2 *psi, int ld, int nbb, double2 *hpsi, void *Z, double scale,
                    cudaStream_t st) {
  return run_batch<float2, float, L, R, CP>(c, psi, ld, nbb, hpsi, (float2 *)Z, c->d_Vf, scale, st);
}
// shared memory of the plane kernel for a cell (full or compact layout)
template <int L, int R>
size_t reg_smem(const pw_cell *c, int fp32, int compact) {
  return fp32 ? plane_smem_bytes<float2, L, R>(c->mxmax, compact != 0, RegPlaneThreads<float2, R>::value)
              : plane_smem_bytes<double2, L, R>(c->mxmax, compact != 0, RegPlaneThreads<double2, R>::value);
}
template <int L, int R>
pw_status reg_dens64(pw_cell *c, const double2 *psi, int ld, int nbb, void *Z, const double *occ, int ngroups,
                     double *part, cudaStream_t st) {
  return density_batch<double2, L, R>(c, psi, ld, nbb, (double2 *)Z, occ, ngroups, part, st);
}
template <int L, int R>
pw_status reg_dens32(pw_cell *c, const double2 *psi, int ld, int nbb, void *Z, const double *occ, int ngroups,
                     double *part, cudaStream_t st) {
  return density_batch<float2, L, R>(c, psi, ld, nbb, (float2 *)Z, occ, ngroups, part, st);
}

}  // namespace

#define PW_REG_PLAN(LL, RR)                                                                           \
  { (LL) * (RR), LL, RR, {reg_run64<LL, RR, false>, reg_run64<LL, RR, true>},                          \
    {reg_run32<LL, RR, false>, reg_run32<LL, RR, true>}, reg_dens64<LL, RR>, reg_dens32<LL, RR>,         \
    reg_smem<LL, RR>, {reg_multi64<LL, RR, false>, reg_multi64<LL, RR, true>},                           \
    {reg_multi32<LL, RR, false>, reg_multi32<LL, RR, true>} }
