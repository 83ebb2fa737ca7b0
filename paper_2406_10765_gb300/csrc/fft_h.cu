// Local part of H psi through the FFT grid (Sec. II-B: each band is
// transformed whole, as in the paper's column-partition H*Psi), fused with the
// sphere scatter / gather, the V_loc(r) multiply and the kinetic term.
//
//   K1  k_sphere_to_z : scatter the sphere columns of each band onto z-lines
//                       of the grid and inverse-FFT them along z.
//   K2  k_plane       : per z-plane: inverse FFT along y (only the x-columns
//                       that meet the sphere), inverse FFT along x, multiply by
//                       V(r), forward x, forward y, keep the sphere columns.
//   K3  k_z_to_sphere : forward FFT along z, gather the sphere, scale by
//                       N^-3 and add 1/2|G|^2 psi.
//
// The FFTs are Stockham autosort passes of radix 4, 2 and 3 on data held in
// shared memory; each pass reads all its inputs into registers, synchronises,
// then writes, so passes run in place.  Bands go through K1-K3 in batches
// whose z-pencil buffer stays resident in the 126 MB L2.
//
// Convention: psi(r_j) = sum_G c_G exp(+i G.r_j); (V psi)_G =
// N^-3 sum_j V(r_j) psi(r_j) exp(-i G.r_j).
#include <stdio.h>

#include "pw_internal.cuh"

namespace {

template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

template <typename C, int R> __device__ __forceinline__ void dft_small(C *v, bool inv);

template <typename C> __device__ __forceinline__ void dft2(C *v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <> __device__ __forceinline__ void dft_small<double2, 2>(double2 *v, bool) { dft2(v); }
template <> __device__ __forceinline__ void dft_small<float2, 2>(float2 *v, bool) { dft2(v); }

// radix 4, sign s = -1 (forward) or +1 (inverse): y_q = sum_p x_p exp(s 2 pi i p q / 4)
template <typename C> __device__ __forceinline__ void dft4(C *v, bool inv) {
  C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
  // j * d13 with j = -i (forward) or +i (inverse)
  C jd;
  if (inv) { jd.x = -d13.y; jd.y = d13.x; } else { jd.x = d13.y; jd.y = -d13.x; }
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, jd);
  v[3] = csub(d02, jd);
}
template <> __device__ __forceinline__ void dft_small<double2, 4>(double2 *v, bool inv) { dft4(v, inv); }
template <> __device__ __forceinline__ void dft_small<float2, 4>(float2 *v, bool inv) { dft4(v, inv); }

// radix 3: w = exp(s 2 pi i / 3) = -1/2 + i s sqrt(3)/2
template <typename C> __device__ __forceinline__ void dft3(C *v, bool inv) {
  typedef decltype(v[0].x) T;
  const T h = (T)0.86602540378443864676;  // sqrt(3)/2
  C a = v[0], b = v[1], c = v[2];
  C sbc = cadd(b, c), dbc = csub(b, c);
  C m;
  m.x = a.x - (T)0.5 * sbc.x;
  m.y = a.y - (T)0.5 * sbc.y;
  // t = i s h (b - c)
  C t;
  if (inv) { t.x = -h * dbc.y; t.y = h * dbc.x; } else { t.x = h * dbc.y; t.y = -h * dbc.x; }
  v[0] = cadd(a, sbc);
  v[1] = cadd(m, t);
  v[2] = csub(m, t);
}
template <> __device__ __forceinline__ void dft_small<double2, 3>(double2 *v, bool inv) { dft3(v, inv); }
template <> __device__ __forceinline__ void dft_small<float2, 3>(float2 *v, bool inv) { dft3(v, inv); }

// Lines: element e of line l sits at buf[((l - lshift) mod lmod) * ls + e * es].
struct LineMap {
  int ls, es, lshift, lmod;
  __device__ __forceinline__ int base(int l) const {
    int q = l - lshift;
    if (q < 0) q += lmod;
    return q * ls;
  }
};

template <typename C, int R>
__device__ void stockham_pass(C *buf, int nlines, const LineMap &lm, int N, int Ns, const C *tw,
                              bool inv) {
  constexpr int MAXB = 16 / R;   // at most 16 complex values in registers per thread
  const int nbl = N / R;                     // butterflies per line
  const int cap = MAXB * blockDim.x;
  int lpg = cap / nbl;
  if (lpg < 1) lpg = 1;
  const int step = N / (Ns * R);
  for (int l0 = 0; l0 < nlines; l0 += lpg) {
    const int l1 = min(nlines, l0 + lpg);
    const int cnt = (l1 - l0) * nbl;
    C v[MAXB][R];
#pragma unroll
    for (int q = 0; q < MAXB; ++q) {
      const int idx = threadIdx.x + q * blockDim.x;
      if (idx < cnt) {
        const int l = l0 + idx / nbl, j = idx % nbl;
        const C *line = buf + lm.base(l);
        const int k = j % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          C x = line[(j + r * nbl) * lm.es];
          if (r > 0 && k > 0) {
            C w = tw[k * r * step];
            if (inv) w.y = -w.y;
            x = cmul(x, w);
          }
          v[q][r] = x;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXB; ++q) {
      const int idx = threadIdx.x + q * blockDim.x;
      if (idx < cnt) {
        const int l = l0 + idx / nbl, j = idx % nbl;
        C *line = buf + lm.base(l);
        const int k = j % Ns;
        dft_small<C, R>(v[q], inv);
        const int d0 = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) line[(d0 + r * Ns) * lm.es] = v[q][r];
      }
    }
    __syncthreads();
  }
}

template <typename C> __device__ __forceinline__ const C *tw_of(const pw_fft_axis &a);
template <> __device__ __forceinline__ const double2 *tw_of<double2>(const pw_fft_axis &a) { return a.tw64; }
template <> __device__ __forceinline__ const float2 *tw_of<float2>(const pw_fft_axis &a) { return a.tw32; }

template <typename C>
__device__ void fft_lines(C *buf, int nlines, const LineMap &lm, const pw_fft_axis &ax, bool inv) {
  int Ns = 1;
  const C *tw = tw_of<C>(ax);
  for (int p = 0; p < ax.npass; ++p) {
    const int R = ax.radix[p];
    if (R == 4) stockham_pass<C, 4>(buf, nlines, lm, ax.n, Ns, tw, inv);
    else if (R == 2) stockham_pass<C, 2>(buf, nlines, lm, ax.n, Ns, tw, inv);
    else stockham_pass<C, 3>(buf, nlines, lm, ax.n, Ns, tw, inv);
    Ns *= R;
  }
}

template <typename C> __device__ __forceinline__ C from64(double2 a);
template <> __device__ __forceinline__ double2 from64<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from64<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// ---------------------------------------------------------------- K1 ----
template <typename C>
__global__ void __launch_bounds__(256) k_sphere_to_z(const double2 *__restrict__ psi, int ld,
                                                     const int *__restrict__ colstart,
                                                     const int *__restrict__ gcol,
                                                     const int *__restrict__ gz, int ncol, int cb,
                                                     pw_fft_axis az, C *__restrict__ Z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *lines = reinterpret_cast<C *>(smem_raw);
  const int Nz = az.n, ls = Nz + 1;
  const int c0 = blockIdx.x * cb;
  const int nc = min(cb, ncol - c0);
  const int b = blockIdx.y;
  const double2 *p = psi + (long)b * ld;
  for (int i = threadIdx.x; i < nc * ls; i += blockDim.x) lines[i] = czero<C>();
  __syncthreads();
  const int g0 = colstart[c0], g1 = colstart[c0 + nc];
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x)
    lines[(gcol[g] - c0) * ls + gz[g]] = from64<C>(p[g]);
  __syncthreads();
  LineMap lm{ls, 1, 0, 1 << 30};
  fft_lines<C>(lines, nc, lm, az, true);
  C *Zb = Z + (long)b * Nz * ncol;
  for (int i = threadIdx.x; i < nc * Nz; i += blockDim.x) {
    const int z = i / nc, cl = i % nc;
    Zb[(long)z * ncol + c0 + cl] = lines[cl * ls + z];
  }
}

// ---------------------------------------------------------------- K2 ----
// FP64 planes run 256 threads (the FP64 pipe, not latency, bounds them and
// 16 complex doubles per thread need the registers); FP32 planes run 512.
template <typename C> struct kPlaneThreads { static constexpr int value = 512; };
template <> struct kPlaneThreads<double2> { static constexpr int value = 256; };

template <typename C, typename T>
__global__ void __launch_bounds__(kPlaneThreads<C>::value) k_plane(C *__restrict__ Z, int ncol,
                                               const int *__restrict__ colxy, int mxmax,
                                               pw_fft_axis ax, pw_fft_axis ay, int Nz,
                                               const T *__restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *P = reinterpret_cast<C *>(smem_raw);
  const int Nx = ax.n, Ny = ay.n, pxs = Nx + 1;
  const int z = blockIdx.x, b = blockIdx.y;
  C *Zp = Z + ((long)b * Nz + z) * ncol;
  for (int i = threadIdx.x; i < Ny * pxs; i += blockDim.x) P[i] = czero<C>();
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int xy = colxy[c];
    P[(xy / Nx) * pxs + (xy % Nx)] = Zp[c];
  }
  __syncthreads();
  const int nxe = 2 * mxmax + 1;
  LineMap ycols{1, pxs, mxmax, Nx};
  LineMap xrows{pxs, 1, 0, 1 << 30};
  fft_lines<C>(P, nxe, ycols, ay, true);
  fft_lines<C>(P, Ny, xrows, ax, true);
  const T *Vz = V + (long)z * Ny * Nx;
  for (int i = threadIdx.x; i < Ny * Nx; i += blockDim.x) {
    const int y = i / Nx, x = i % Nx;
    C &e = P[y * pxs + x];
    const T v = Vz[i];
    e.x *= v;
    e.y *= v;
  }
  __syncthreads();
  fft_lines<C>(P, Ny, xrows, ax, false);
  fft_lines<C>(P, nxe, ycols, ay, false);
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int xy = colxy[c];
    Zp[c] = P[(xy / Nx) * pxs + (xy % Nx)];
  }
}

// ---------------------------------------------------------------- K3 ----
template <typename C>
__global__ void __launch_bounds__(256) k_z_to_sphere(const C *__restrict__ Z, int ncol, int cb,
                                                     pw_fft_axis az,
                                                     const int *__restrict__ colstart,
                                                     const int *__restrict__ gcol,
                                                     const int *__restrict__ gz,
                                                     const double *__restrict__ kin,
                                                     const double2 *__restrict__ psi, int ld,
                                                     double2 *__restrict__ hpsi, double scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *lines = reinterpret_cast<C *>(smem_raw);
  const int Nz = az.n, ls = Nz + 1;
  const int c0 = blockIdx.x * cb;
  const int nc = min(cb, ncol - c0);
  const int b = blockIdx.y;
  const C *Zb = Z + (long)b * Nz * ncol;
  for (int i = threadIdx.x; i < nc * Nz; i += blockDim.x) {
    const int z = i / nc, cl = i % nc;
    lines[cl * ls + z] = Zb[(long)z * ncol + c0 + cl];
  }
  __syncthreads();
  LineMap lm{ls, 1, 0, 1 << 30};
  fft_lines<C>(lines, nc, lm, az, false);
  const int g0 = colstart[c0], g1 = colstart[c0 + nc];
  const double2 *p = psi + (long)b * ld;
  double2 *h = hpsi + (long)b * ld;
  for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const C v = lines[(gcol[g] - c0) * ls + gz[g]];
    const double t = kin[g];
    const double2 x = p[g];
    h[g] = make_double2(t * x.x + scale * (double)v.x, t * x.y + scale * (double)v.y);
  }
}

// ------------------------------------------------------------ density ----
// Stockham counterpart of k_density_reg (grids without a register FFT):
// inverse y and x FFTs of each band's plane, acc += w |psi(r)|^2 in fixed
// per-thread points (at most DENS_ACC per thread).
constexpr int DENS_ACC = 32;
template <typename C>
__global__ void __launch_bounds__(kPlaneThreads<C>::value) k_density_plane(const C *__restrict__ Z, int ncol,
                                                                           const int *__restrict__ colxy,
                                                                           int mxmax, pw_fft_axis ax, pw_fft_axis ay,
                                                                           int Nz, int nbb,
                                                                           const double *__restrict__ occ,
                                                                           double *__restrict__ part) {
  typedef decltype(Z[0].x) T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *P = reinterpret_cast<C *>(smem_raw);
  const int Nx = ax.n, Ny = ay.n, pxs = Nx + 1, np = Nx * Ny;
  const int z = blockIdx.x, grp = blockIdx.y, ngroups = gridDim.y;
  T acc[DENS_ACC];
#pragma unroll
  for (int k = 0; k < DENS_ACC; ++k) acc[k] = 0;
  const int nxe = 2 * mxmax + 1;
  LineMap ycols{1, pxs, mxmax, Nx};
  LineMap xrows{pxs, 1, 0, 1 << 30};
  for (int j = grp; j < nbb; j += ngroups) {
    const T w = occ ? (T)occ[j] : (T)1;
    const C *Zp = Z + ((long)j * Nz + z) * ncol;
    for (int i = threadIdx.x; i < Ny * pxs; i += blockDim.x) P[i] = czero<C>();
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      const int xy = colxy[c];
      P[(xy / Nx) * pxs + (xy % Nx)] = Zp[c];
    }
    __syncthreads();
    fft_lines<C>(P, nxe, ycols, ay, true);
    fft_lines<C>(P, Ny, xrows, ax, true);
#pragma unroll
    for (int k = 0; k < DENS_ACC; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < np) {
        const C e = P[(i / Nx) * pxs + (i % Nx)];
        acc[k] += w * (e.x * e.x + e.y * e.y);
      }
    }
    __syncthreads();
  }
  double *out = part + ((long)grp * Nz + z) * np;
#pragma unroll
  for (int k = 0; k < DENS_ACC; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < np) out[i] = (double)acc[k];
  }
}

// ------------------------------------------------------ full-grid FFT ----
// One axis of a 3-D transform of a complex grid g[(z N1 + y) N0 + x]
// (x fastest): each block gathers 16 lines of the axis into shared memory,
// runs the Stockham passes in place and writes them back.  Unscaled; sign -1
// forward, +1 inverse.
constexpr int GL = 16;
__global__ void __launch_bounds__(256) k_grid_fft_axis(double2 *__restrict__ g, int N0, int N1, int N2,
                                                       int axis, pw_fft_axis ax, int inv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *lines = reinterpret_cast<double2 *>(smem_raw);
  const int n = ax.n, ls = n + 1;
  const long nlines = (long)N0 * N1 * N2 / n;
  const long l0 = (long)blockIdx.x * GL;
  const int nl = (int)min((long)GL, nlines - l0);
  // line q -> (first element, stride)
  auto base = [&](long q, long *stride) -> long {
    if (axis == 0) { *stride = 1; return q * N0; }
    if (axis == 1) { *stride = N0; const long z = q / N0, x = q % N0; return z * (long)N0 * N1 + x; }
    *stride = (long)N0 * N1;
    return q;                                            // q = y N0 + x
  };
  for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
    const int e = i / nl, q = i % nl;                    // consecutive threads: consecutive lines
    long st;
    const long b = base(l0 + q, &st);
    lines[q * ls + e] = g[b + e * st];
  }
  __syncthreads();
  LineMap lm{ls, 1, 0, 1 << 30};
  fft_lines<double2>(lines, nl, lm, ax, inv != 0);
  for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
    const int e = i / nl, q = i % nl;
    long st;
    const long b = base(l0 + q, &st);
    g[b + e * st] = lines[q * ls + e];
  }
}

// shared-memory opt-in for a kernel whose launches need `bytes`: set to the
// largest size, so threads launching it for different grids never lower it
// under each other
template <typename K> static pw_status allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    PW_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  return PW_OK;
}

template <typename C, typename T>
pw_status apply_local_t(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                        const T *V, cudaStream_t st) {
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  constexpr int fp32 = sizeof(C) == sizeof(float2);
  const pw_reg_plan *reg = pw_reg_plan_at(pw_cell_fft_plan(c, fp32));
  const int cp = pw_cell_fft_compact(c, fp32);
  // the Stockham passes hold the whole x-y plane in shared memory
  const size_t plane_bytes = (size_t)Ny * (Nx + 1) * sizeof(C);
  if (!reg && plane_bytes > 227 * 1024) return PW_ERR_ARG;
  const int cb = 16;
  const size_t line_bytes = (size_t)cb * (Nz + 1) * sizeof(C);
  const size_t per_band = (size_t)Nz * c->ncol * sizeof(C);
  // batch of bands whose z-pencils stay L2-resident (default ~64 MB)
  int batch = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, pw_cell_fft_batch_bytes(c, fp32) / per_band));
  PW_TRY(pw_ensure(&c->d_z, &c->z_bytes, per_band * batch));
  C *Z = reinterpret_cast<C *>(c->d_z);
  if (!reg) {
    PW_TRY(allow_smem(k_sphere_to_z<C>, line_bytes));
    PW_TRY(allow_smem(k_plane<C, T>, plane_bytes));
    PW_TRY(allow_smem(k_z_to_sphere<C>, line_bytes));
  }
  const double scale = 1.0 / ((double)Nx * Ny * Nz);
  for (int b0 = 0; b0 < nb; b0 += batch) {
    const int nbb = std::min(batch, nb - b0);
    if (reg && c->fft_hook) {
      // serving: this batch of bands joins a launch shared with other cells
      const pw_fft_job job{c, psi + (long)b0 * ld, hpsi + (long)b0 * ld, ld, nbb, Z, scale};
      PW_TRY(c->fft_hook(c->fft_hook_ctx, job, reg, fp32, cp, st));
      continue;
    }
    if (reg) {
      PW_TRY((fp32 ? reg->run32[cp] : reg->run64[cp])(c, psi + (long)b0 * ld, ld, nbb, hpsi + (long)b0 * ld, Z,
                                                      scale, st));
      continue;
    }
    dim3 gcols((c->ncol + cb - 1) / cb, nbb);
    pw_count_launch();
    k_sphere_to_z<C><<<gcols, 256, line_bytes, st>>>(psi + (long)b0 * ld, ld, c->d_colstart,
                                                     c->d_gcol, c->d_gz, c->ncol, cb, c->ax[2], Z);
    pw_count_launch();
    k_plane<C, T><<<dim3(Nz, nbb), kPlaneThreads<C>::value, plane_bytes, st>>>(Z, c->ncol, c->d_colxy, c->mxmax,
                                                           c->ax[0], c->ax[1], Nz, V);
    pw_count_launch();
    k_z_to_sphere<C><<<gcols, 256, line_bytes, st>>>(Z, c->ncol, cb, c->ax[2], c->d_colstart,
                                                     c->d_gcol, c->d_gz, c->d_kin,
                                                     psi + (long)b0 * ld, ld,
                                                     hpsi + (long)b0 * ld, scale);
  }
  return pw_check_launch("apply_local");
}

// FP64 local part with a caller-provided z-pencil buffer of `zbytes` bytes
// (no allocation); bands are processed in batches that fit the buffer
pw_status apply_local_into(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                           void *zbuf, size_t zbytes, cudaStream_t st) {
  typedef double2 C;
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  const pw_reg_plan *reg = pw_reg_plan_at(pw_cell_fft_plan(c, 0));
  const int cp = pw_cell_fft_compact(c, 0);
  const size_t plane_bytes = (size_t)Ny * (Nx + 1) * sizeof(C);
  if (!reg && plane_bytes > 227 * 1024) return PW_ERR_ARG;
  const int cb = 16;
  const size_t line_bytes = (size_t)cb * (Nz + 1) * sizeof(C);
  const size_t per_band = (size_t)Nz * c->ncol * sizeof(C);
  const int batch = (int)std::min<size_t>((size_t)nb, zbytes / per_band);
  if (batch < 1) return PW_ERR_ARG;
  C *Z = reinterpret_cast<C *>(zbuf);
  if (!reg) {
    PW_TRY(allow_smem(k_sphere_to_z<C>, line_bytes));
    PW_TRY(allow_smem(k_plane<C, double>, plane_bytes));
    PW_TRY(allow_smem(k_z_to_sphere<C>, line_bytes));
  }
  const double scale = 1.0 / ((double)Nx * Ny * Nz);
  for (int b0 = 0; b0 < nb; b0 += batch) {
    const int nbb = std::min(batch, nb - b0);
    if (reg) {
      PW_TRY(reg->run64[cp](c, psi + (long)b0 * ld, ld, nbb, hpsi + (long)b0 * ld, Z, scale, st));
      continue;
    }
    dim3 gcols((c->ncol + cb - 1) / cb, nbb);
    pw_count_launch();
    k_sphere_to_z<C><<<gcols, 256, line_bytes, st>>>(psi + (long)b0 * ld, ld, c->d_colstart,
                                                     c->d_gcol, c->d_gz, c->ncol, cb, c->ax[2], Z);
    pw_count_launch();
    k_plane<C, double><<<dim3(Nz, nbb), kPlaneThreads<C>::value, plane_bytes, st>>>(
        Z, c->ncol, c->d_colxy, c->mxmax, c->ax[0], c->ax[1], Nz, c->d_V);
    pw_count_launch();
    k_z_to_sphere<C><<<gcols, 256, line_bytes, st>>>(Z, c->ncol, cb, c->ax[2], c->d_colstart,
                                                     c->d_gcol, c->d_gz, c->d_kin,
                                                     psi + (long)b0 * ld, ld,
                                                     hpsi + (long)b0 * ld, scale);
  }
  return pw_check_launch("apply_local_into");
}

template <typename C>
pw_status density_batch_t(pw_cell *c, const double2 *psi, int ld, int nbb, C *Z, const double *occ,
                          int ngroups, double *part, cudaStream_t st) {
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  const size_t plane_bytes = (size_t)Ny * (Nx + 1) * sizeof(C);
  if (plane_bytes > 227 * 1024 || (long)Nx * Ny > (long)DENS_ACC * kPlaneThreads<C>::value) return PW_ERR_ARG;
  const int cb = 16;
  const size_t line_bytes = (size_t)cb * (Nz + 1) * sizeof(C);
  PW_TRY(allow_smem(k_sphere_to_z<C>, line_bytes));
  PW_TRY(allow_smem(k_density_plane<C>, plane_bytes));
  dim3 gcols((c->ncol + cb - 1) / cb, nbb);
  pw_count_launch();
  k_sphere_to_z<C><<<gcols, 256, line_bytes, st>>>(psi, ld, c->d_colstart, c->d_gcol, c->d_gz, c->ncol, cb,
                                                   c->ax[2], Z);
  pw_count_launch();
  k_density_plane<C><<<dim3(Nz, ngroups), kPlaneThreads<C>::value, plane_bytes, st>>>(
      Z, c->ncol, c->d_colxy, c->mxmax, c->ax[0], c->ax[1], Nz, nbb, occ, part);
  return pw_check_launch("density");
}

}  // namespace

size_t pw_local_zbytes_per_band(const pw_cell *c) { return (size_t)c->N[2] * c->ncol * sizeof(double2); }

pw_status pw_apply_local_fp64_into(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                                   void *zbuf, size_t zbytes, cudaStream_t st) {
  return apply_local_into(c, psi, ld, nb, hpsi, zbuf, zbytes, st);
}

pw_status pw_apply_local(pw_cell *c, const double2 *psi, int ld, int nb, double2 *hpsi,
                         int precision, cudaStream_t st) {
  if (precision == PW_MIXED) return apply_local_t<float2, float>(c, psi, ld, nb, hpsi, c->d_Vf, st);
  return apply_local_t<double2, double>(c, psi, ld, nb, hpsi, c->d_V, st);
}

pw_status pw_fft_density_batch(pw_cell *c, const double2 *psi, int ld, int nbb, void *Z, int fp32,
                               const double *occ, int ngroups, double *part, cudaStream_t st) {
  if (fp32) return density_batch_t<float2>(c, psi, ld, nbb, (float2 *)Z, occ, ngroups, part, st);
  return density_batch_t<double2>(c, psi, ld, nbb, (double2 *)Z, occ, ngroups, part, st);
}

pw_status pw_grid_fft(pw_cell *c, double2 *g, int inverse, cudaStream_t st) {
  const long npts = (long)c->N[0] * c->N[1] * c->N[2];
  for (int a = 0; a < 3; ++a) {
    const int n = c->N[a];
    const size_t bytes = (size_t)GL * (n + 1) * sizeof(double2);
    PW_TRY(allow_smem(k_grid_fft_axis, bytes));
    const long nlines = npts / n;
    pw_count_launch();
    k_grid_fft_axis<<<(unsigned)((nlines + GL - 1) / GL), 256, bytes, st>>>(g, c->N[0], c->N[1], c->N[2], a,
                                                                          c->ax[a], inverse);
  }
  return pw_check_launch("grid fft");
}
