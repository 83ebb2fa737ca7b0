// Cell setup: plane-wave sphere, FFT grid and plans, kinetic table, local
// potential on the grid and the Kleinman-Bylander projector matrix.
//
// The eigenproblem is H X = X Lambda (Sec. II-A, Eq. 1).  The sphere holds
// the plane waves with 1/2|G|^2 <= Ecut and the FFT grid follows the
// Ecut -> grid rule of Sec. II-A (times 1.5, rounded up to 2^a 3^b).  Per-atom
// data lives in flat arrays indexed by atom (the map-to-array rule of
// Sec. III-F); no lookup structures are used on the device.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "oz_gemm.cuh"
#include "pw_internal.cuh"
#include "tc_gemm.cuh"

#include <atomic>

static thread_local char g_err[256];
static std::atomic<unsigned long long> g_launches{0};

static thread_local unsigned long long g_thread_launches = 0;

void pw_count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++g_thread_launches;
}
// a replayed graph runs the kernels its capture counted
void pw_count_launches(uint64_t n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  g_thread_launches += n;
}
uint64_t pw_thread_launches() { return g_thread_launches; }
extern "C" uint64_t pw_kernel_launches(void) { return g_launches.load(); }

void pw_last_cuda_error(cudaError_t e, const char *file, int line) {
  snprintf(g_err, sizeof g_err, "%s at %s:%d", cudaGetErrorString(e), file, line);
  fprintf(stderr, "pw: CUDA error %s\n", g_err);
}

pw_status pw_check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
    fprintf(stderr, "pw: launch failed %s\n", g_err);
    return PW_ERR_CUDA;
  }
  return PW_OK;
}

pw_status pw_ensure(void **ptr, size_t *cur, size_t need) {
  if (need <= *cur && *ptr) return PW_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cur = 0;
  if (need == 0) return PW_OK;
  if (cudaMalloc(ptr, need) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return PW_ERR_OOM;
  }
  *cur = need;
  return PW_OK;
}

extern "C" const char *pw_strerror(pw_status s) {
  switch (s) {
    case PW_OK: return "ok";
    case PW_ERR_ARG: return "invalid argument";
    case PW_ERR_OOM: return "out of device memory";
    case PW_ERR_CUDA: return "CUDA error";
    case PW_ERR_CHOL: return "overlap matrix not positive definite";
    case PW_ERR_NOCONV: return "not converged";
    case PW_ERR_TIMEOUT: return "device wait timed out";
    case PW_ERR_BUSY: return "busy: not enough device memory to admit";
    case PW_ERR_NUMERIC: return "NaN or Inf met";
  }
  return "unknown status";
}

// --------------------------------------------------------------------------
// host helpers
// --------------------------------------------------------------------------
static int smooth_at_least(double target) {
  long best = -1;
  for (long p2 = 1; p2 < 1L << 20; p2 *= 2)
    for (long p = p2; p < 1L << 20; p *= 3)
      if (p >= target && (best < 0 || p < best)) best = p;
  return (int)best;
}

static bool fft_plan(int n, pw_fft_axis &ax) {
  ax.n = n;
  ax.npass = 0;
  int r = n;
  while (r % 4 == 0) { ax.radix[ax.npass++] = 4; r /= 4; if (ax.npass >= PW_MAX_PASSES) return false; }
  while (r % 2 == 0) { ax.radix[ax.npass++] = 2; r /= 2; if (ax.npass >= PW_MAX_PASSES) return false; }
  while (r % 3 == 0) { ax.radix[ax.npass++] = 3; r /= 3; if (ax.npass >= PW_MAX_PASSES) return false; }
  return r == 1 && n >= 2;
}

// Host tables to the device, ordered on the caller's stream: a plain
// cudaMemcpy from pageable memory may return before its DMA has landed, and
// kernels on a non-blocking stream are not ordered after it
static pw_status upload(void **dst, const void *src, size_t bytes, size_t *acc, cudaStream_t st) {
  if (bytes == 0) { *dst = nullptr; return PW_OK; }
  if (cudaMalloc(dst, bytes) != cudaSuccess) { cudaGetLastError(); *dst = nullptr; return PW_ERR_OOM; }
  *acc += bytes;
  PW_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
  return PW_OK;
}

// --------------------------------------------------------------------------
// device kernels
// --------------------------------------------------------------------------

// V[z][y][x] = sum_a d_a fx[a][x] fy[a][y] fz[a][z]: the periodic Gaussian
// sum factorises over the three axes (fx etc. are 1-D periodic sums).
__global__ void k_vloc(double *V, float *Vf, const double *fx, const double *fy, const double *fz,
                       const double *depth, int natom, int Nx, int Ny, int Nz) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long tot = (long)Nx * Ny * Nz;
  if (idx >= tot) return;
  int x = (int)(idx % Nx);
  int y = (int)((idx / Nx) % Ny);
  int z = (int)(idx / ((long)Nx * Ny));
  double acc = 0.0;
  for (int a = 0; a < natom; ++a)
    acc += depth[a] * fx[(long)a * Nx + x] * fy[(long)a * Ny + y] * fz[(long)a * Nz + z];
  V[idx] = acc;
  Vf[idx] = (float)acc;
}

// beta[g + p*npw] for p = 4a + (s, px, py, pz).  The structure factor
// exp(-i G.tau_a) is the product of three per-axis phases from host tables
// ph[axis][a][m + M_axis].
__global__ void k_beta(double2 *beta, const int *mvec, const double2 *phx, const double2 *phy,
                       const double2 *phz, int Mx, int My, int Mz, int npw, int natom, int a0,
                       double gx, double gy, double gz, double ns, double np, double rp2,
                       double inv_sqrt_omega) {
  // atom a0 + blockIdx.y into columns 4 blockIdx.y .. (chunks of atoms)
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int al = blockIdx.y, a = a0 + al;
  if (g >= npw || al >= natom) return;
  int mx = mvec[3 * g], my = mvec[3 * g + 1], mz = mvec[3 * g + 2];
  double Gx = gx * mx, Gy = gy * my, Gz = gz * mz;
  double g2 = Gx * Gx + Gy * Gy + Gz * Gz;
  double rad = exp(-0.5 * g2 * rp2) * inv_sqrt_omega;
  double2 p = cmul(cmul(phx[(long)a * (2 * Mx + 1) + mx + Mx], phy[(long)a * (2 * My + 1) + my + My]),
                   phz[(long)a * (2 * Mz + 1) + mz + Mz]);
  double2 *col = beta + (long)(4 * al) * npw + g;
  col[0] = make_double2(ns * rad * p.x, ns * rad * p.y);
  // (-i) * G_k * rad * p  ->  (G_k rad) * (p.y, -p.x)
  double f = np * rad;
  col[(long)npw] = make_double2(f * Gx * p.y, -f * Gx * p.x);
  col[(long)2 * npw] = make_double2(f * Gy * p.y, -f * Gy * p.x);
  col[(long)3 * npw] = make_double2(f * Gz * p.y, -f * Gz * p.x);
}

// beta rows g0 .. g0 + ng - 1 for all projectors, in FP32 arithmetic
// (for the split-FP16 products, which keep ~22 bits): out[(g - g0) + p ng]
__global__ void k_beta_rows_f32(double2 *out, const int *mvec, const double2 *phx, const double2 *phy,
                                const double2 *phz, int Mx, int My, int Mz, int g0, int ng, int natom,
                                float gx, float gy, float gz, float ns, float np, float rp2,
                                float inv_sqrt_omega) {
  const int gl = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (gl >= ng || a >= natom) return;
  const int g = g0 + gl;
  const int mx = mvec[3 * g], my = mvec[3 * g + 1], mz = mvec[3 * g + 2];
  const float Gx = gx * mx, Gy = gy * my, Gz = gz * mz;
  const float g2 = Gx * Gx + Gy * Gy + Gz * Gz;
  const float rad = expf(-0.5f * g2 * rp2) * inv_sqrt_omega;
  const double2 px = phx[(long)a * (2 * Mx + 1) + mx + Mx], py = phy[(long)a * (2 * My + 1) + my + My],
                pz = phz[(long)a * (2 * Mz + 1) + mz + Mz];
  const float2 qx = make_float2((float)px.x, (float)px.y), qy = make_float2((float)py.x, (float)py.y),
               qz = make_float2((float)pz.x, (float)pz.y);
  const float2 p = cmul(cmul(qx, qy), qz);
  double2 *col = out + (long)(4 * a) * ng + gl;
  col[0] = make_double2(ns * rad * p.x, ns * rad * p.y);
  const float f = np * rad;
  col[(long)ng] = make_double2(f * Gx * p.y, -f * Gx * p.x);
  col[(long)2 * ng] = make_double2(f * Gy * p.y, -f * Gy * p.x);
  col[(long)3 * ng] = make_double2(f * Gz * p.y, -f * Gz * p.x);
}

pw_status pw_beta_rows_f32(pw_cell *c, int g0, int ng, double2 *out, cudaStream_t st) {
  if (ng <= 0) return PW_OK;
  const double twopi = 2.0 * M_PI;
  const double omega = c->L[0] * c->L[1] * c->L[2];
  dim3 grid((ng + 127) / 128, c->natom);
  pw_count_launch();
  k_beta_rows_f32<<<grid, 128, 0, st>>>(out, c->d_m, c->d_ph[0], c->d_ph[1], c->d_ph[2], c->Mext[0],
                                        c->Mext[1], c->Mext[2], g0, ng, c->natom, (float)(twopi / c->L[0]),
                                        (float)(twopi / c->L[1]), (float)(twopi / c->L[2]), (float)c->proj_ns,
                                        (float)c->proj_np, (float)(c->pwidth * c->pwidth),
                                        (float)(1.0 / sqrt(omega)));
  return pw_check_launch("k_beta_rows_f32");
}

pw_status pw_beta_chunk(pw_cell *c, int a0, int na, double2 *out, cudaStream_t st) {
  if (na <= 0) return PW_OK;
  const double twopi = 2.0 * M_PI;
  const double omega = c->L[0] * c->L[1] * c->L[2];
  dim3 grid((c->npw + 127) / 128, na);
  pw_count_launch();
  k_beta<<<grid, 128, 0, st>>>(out, c->d_m, c->d_ph[0], c->d_ph[1], c->d_ph[2], c->Mext[0], c->Mext[1],
                               c->Mext[2], c->npw, na, a0, twopi / c->L[0], twopi / c->L[1],
                               twopi / c->L[2], c->proj_ns, c->proj_np, c->pwidth * c->pwidth,
                               1.0 / sqrt(omega));
  return pw_check_launch("k_beta");
}

// --------------------------------------------------------------------------
// entry points
// --------------------------------------------------------------------------
extern "C" void pw_destroy_cell(pw_cell *c) {
  if (!c) return;
  pw_tc_operand **ops[] = {&c->op_beta_rows, &c->op_beta_t, &c->op_psi, &c->op_db, &c->op_bc_rows,
                           &c->op_bc_t, &c->op_psi_c};
  for (pw_tc_operand **o : ops)
    if (*o) { pw_tc_operand_free(*o); delete *o; *o = nullptr; }
  if (c->d_rmax) cudaFree(c->d_rmax);
  if (c->d_tc_err) cudaFree(c->d_tc_err);
  if (c->oz) { pw_oz_free(c->oz); delete c->oz; c->oz = nullptr; }
  void *ptrs[] = {c->d_gcol, c->d_gz, c->d_colstart, c->d_colxy, c->d_kin, c->d_V, c->d_Vf,
                  c->d_beta, c->d_D, c->d_z, c->d_dpart, c->d_V0, c->d_grid, c->d_B, c->d_gemm_ws, c->d_beta_split,
                  c->d_m, c->d_ph[0], c->d_ph[1], c->d_ph[2], c->d_bchunk,
                  c->ax[0].tw64, c->ax[0].tw32, c->ax[1].tw64, c->ax[1].tw32,
                  c->ax[2].tw64, c->ax[2].tw32};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

extern "C" pw_status pw_setup_cell(const pw_cell_desc *d, void *stream, pw_cell **out) {
  if (!out) return PW_ERR_ARG;
  *out = nullptr;
  if (!d || d->natom < 0 || !(d->ecut > 0) || (d->natom > 0 && (!d->tau || !d->vdepth || !d->dkb)))
    return PW_ERR_ARG;
  if (d->precision != PW_FP64 && d->precision != PW_MIXED) return PW_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j && d->lattice[3 * j + i] != 0.0) return PW_ERR_ARG;
  double L[3] = {d->lattice[0], d->lattice[4], d->lattice[8]};
  for (int i = 0; i < 3; ++i)
    if (!(L[i] > 0)) return PW_ERR_ARG;
  if (d->natom > 0 && !(d->vwidth > 0 && d->pwidth > 0)) return PW_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;

  pw_cell *c = new pw_cell();
  c->precision = d->precision;
  c->ecut = d->ecut;
  c->vwidth = d->vwidth;
  c->pwidth = d->pwidth;
  c->natom = d->natom;
  c->nproj = 4 * d->natom;
  for (int i = 0; i < 3; ++i) c->L[i] = L[i];
  for (int i = 0; i < 3; ++i) c->ax[i] = pw_fft_axis{};

  // ---- sphere (lexicographic mx, my, mz; each (mx, my) column contiguous)
  const double twopi = 2.0 * M_PI;
  int M[3];
  for (int i = 0; i < 3; ++i) M[i] = (int)floor(sqrt(2.0 * d->ecut) * L[i] / twopi) + 1;
  std::vector<int> gcol, gz, colstart, colxy;
  std::vector<double> kin;
  std::vector<int> colmx, colmy;
  int mabs[3] = {0, 0, 0};
  for (int mx = -M[0]; mx <= M[0]; ++mx)
    for (int my = -M[1]; my <= M[1]; ++my) {
      bool opened = false;
      for (int mz = -M[2]; mz <= M[2]; ++mz) {
        double gxv = twopi * mx / L[0], gyv = twopi * my / L[1], gzv = twopi * mz / L[2];
        double t = 0.5 * (gxv * gxv + gyv * gyv + gzv * gzv);
        if (fabs(t - d->ecut) < 1e-9) { pw_destroy_cell(c); return PW_ERR_ARG; }
        if (t > d->ecut) continue;
        if (!opened) {
          colstart.push_back((int)kin.size());
          colmx.push_back(mx);
          colmy.push_back(my);
          opened = true;
        }
        c->m_host.push_back(mx);
        c->m_host.push_back(my);
        c->m_host.push_back(mz);
        gcol.push_back((int)colstart.size() - 1);
        gz.push_back(mz);
        kin.push_back(t);
        mabs[0] = std::max(mabs[0], abs(mx));
        mabs[1] = std::max(mabs[1], abs(my));
        mabs[2] = std::max(mabs[2], abs(mz));
      }
    }
  c->npw = (int)kin.size();
  c->ncol = (int)colstart.size();
  colstart.push_back(c->npw);
  c->mxmax = mabs[0];

  // ---- grid
  for (int i = 0; i < 3; ++i) {
    int n = d->grid[i] > 0 ? d->grid[i] : smooth_at_least(1.5 * sqrt(2.0 * d->ecut) * L[i] / M_PI);
    if (n < 2 * mabs[i] + 1 || !fft_plan(n, c->ax[i])) { pw_destroy_cell(c); return PW_ERR_ARG; }
    c->N[i] = n;
  }
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  for (int g = 0; g < c->npw; ++g) gz[g] = ((gz[g] % Nz) + Nz) % Nz;
  colxy.resize(c->ncol);
  for (int k = 0; k < c->ncol; ++k)
    colxy[k] = (((colmy[k] % Ny) + Ny) % Ny) * Nx + (((colmx[k] % Nx) + Nx) % Nx);

  size_t acc = 0;
  pw_status s;
#define UP(dst, vec)                                                                           \
  s = upload((void **)&(dst), (vec).data(), (vec).size() * sizeof((vec)[0]), &acc, st);        \
  if (s != PW_OK) { pw_destroy_cell(c); return s; }
  UP(c->d_gcol, gcol);
  UP(c->d_gz, gz);
  UP(c->d_colstart, colstart);
  UP(c->d_colxy, colxy);
  UP(c->d_kin, kin);

  // ---- FFT twiddles exp(-2 pi i k / n)
  for (int i = 0; i < 3; ++i) {
    int n = c->N[i];
    std::vector<double2> t64(n);
    std::vector<float2> t32(n);
    for (int k = 0; k < n; ++k) {
      double a = twopi * (double)k / (double)n;
      t64[k] = make_double2(cos(a), -sin(a));
      t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
    }
    UP(c->ax[i].tw64, t64);
    UP(c->ax[i].tw32, t32);
  }

  // ---- local potential: 1-D periodic Gaussian sums per atom and axis
  c->tau_host.assign(d->tau, d->tau + 3 * (size_t)d->natom);
  c->depth_host.assign(d->vdepth, d->vdepth + d->natom);
  c->dkb_host.assign(d->dkb, d->dkb + 4 * (size_t)d->natom);
  {
    const long ng = (long)Nx * Ny * Nz;
    if (cudaMalloc(&c->d_V, ng * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_Vf, ng * sizeof(float)) != cudaSuccess) {
      cudaGetLastError(); pw_destroy_cell(c); return PW_ERR_OOM;
    }
    acc += ng * (sizeof(double) + sizeof(float));
    if (d->natom == 0) {
      PW_CUDA(cudaMemsetAsync(c->d_V, 0, ng * sizeof(double), st));
      PW_CUDA(cudaMemsetAsync(c->d_Vf, 0, ng * sizeof(float), st));
    } else {
      std::vector<double> f[3];
      const double s2 = 2.0 * d->vwidth * d->vwidth;
      for (int ax = 0; ax < 3; ++ax) {
        int n = c->N[ax];
        f[ax].assign((size_t)d->natom * n, 0.0);
        for (int a = 0; a < d->natom; ++a)
          for (int j = 0; j < n; ++j) {
            double dd = L[ax] * j / n - d->tau[3 * a + ax];
            dd -= L[ax] * floor(dd / L[ax] + 0.5);        // nearest image in [-L/2, L/2)
            double sum = 0.0;
            for (int im = -2; im <= 2; ++im) {
              double e = dd - im * L[ax];
              sum += exp(-e * e / s2);
            }
            f[ax][(size_t)a * n + j] = sum;
          }
      }
      double *dfx, *dfy, *dfz, *ddep;
      size_t tmp = 0;
      if ((s = upload((void **)&dfx, f[0].data(), f[0].size() * 8, &tmp, st)) != PW_OK ||
          (s = upload((void **)&dfy, f[1].data(), f[1].size() * 8, &tmp, st)) != PW_OK ||
          (s = upload((void **)&dfz, f[2].data(), f[2].size() * 8, &tmp, st)) != PW_OK ||
          (s = upload((void **)&ddep, d->vdepth, (size_t)d->natom * 8, &tmp, st)) != PW_OK) {
        pw_destroy_cell(c); return s;
      }
      pw_count_launch();
      k_vloc<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(c->d_V, c->d_Vf, dfx, dfy, dfz, ddep,
                                                         d->natom, Nx, Ny, Nz);
      s = pw_check_launch("k_vloc");
      cudaStreamSynchronize(st);
      cudaFree(dfx); cudaFree(dfy); cudaFree(dfz); cudaFree(ddep);
      if (s != PW_OK) { pw_destroy_cell(c); return s; }
    }
  }

  // ---- projectors
  if (d->natom > 0) {
    std::vector<double> D(d->dkb, d->dkb + 4 * (size_t)d->natom);
    UP(c->d_D, D);
    size_t nbeta = (size_t)c->npw * c->nproj;
    if (cudaMalloc(&c->d_beta, nbeta * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError(); pw_destroy_cell(c); return PW_ERR_OOM;
    }
    acc += nbeta * sizeof(double2);
    std::vector<double2> ph[3];
    for (int ax = 0; ax < 3; ++ax) {
      int w = 2 * M[ax] + 1;
      ph[ax].resize((size_t)d->natom * w);
      for (int a = 0; a < d->natom; ++a)
        for (int m = -M[ax]; m <= M[ax]; ++m) {
          double th = twopi * m * d->tau[3 * a + ax] / L[ax];
          ph[ax][(size_t)a * w + m + M[ax]] = make_double2(cos(th), -sin(th));
        }
    }
    // tables stay with the cell (projector regeneration); uploaded straight
    // into it, so a failure part-way is released by pw_destroy_cell
    size_t tmp = 0;
    if ((s = upload((void **)&c->d_m, c->m_host.data(), c->m_host.size() * 4, &tmp, st)) != PW_OK ||
        (s = upload((void **)&c->d_ph[0], ph[0].data(), ph[0].size() * 16, &tmp, st)) != PW_OK ||
        (s = upload((void **)&c->d_ph[1], ph[1].data(), ph[1].size() * 16, &tmp, st)) != PW_OK ||
        (s = upload((void **)&c->d_ph[2], ph[2].data(), ph[2].size() * 16, &tmp, st)) != PW_OK) {
      pw_destroy_cell(c); return s;
    }
    double rp = d->pwidth;
    c->proj_ns = sqrt(8.0 * pow(M_PI, 1.5) * rp * rp * rp);
    c->proj_np = sqrt(16.0 * pow(M_PI, 1.5) * rp * rp * rp * rp * rp);
    for (int ax = 0; ax < 3; ++ax) c->Mext[ax] = M[ax];
    acc += tmp;
    s = pw_beta_chunk(c, 0, d->natom, c->d_beta, st);
    cudaStreamSynchronize(st);
    if (s != PW_OK) { pw_destroy_cell(c); return s; }
  }
#undef UP
  c->bytes = acc;
  if (cudaStreamSynchronize(st) != cudaSuccess) { pw_destroy_cell(c); return PW_ERR_CUDA; }
  *out = c;
  return PW_OK;
}

extern "C" pw_status pw_cell_info(const pw_cell *c, int *npw, int grid[3], const int **mvec) {
  if (!c) return PW_ERR_ARG;
  if (npw) *npw = c->npw;
  if (grid) for (int i = 0; i < 3; ++i) grid[i] = c->N[i];
  if (mvec) *mvec = c->m_host.data();
  return PW_OK;
}

extern "C" pw_status pw_cell_sizes(const pw_cell *c, int *nproj, size_t *bytes) {
  if (!c) return PW_ERR_ARG;
  if (nproj) *nproj = c->nproj;
  if (bytes) *bytes = c->bytes + c->z_bytes + c->B_elems * 16 + c->gemm_ws_elems * 16 +
                      c->beta_split_bytes;
  return PW_OK;
}

extern "C" pw_status pw_cell_set_precision(pw_cell *c, int p) {
  if (!c || (p != PW_FP64 && p != PW_MIXED)) return PW_ERR_ARG;
  c->precision = p;
  return PW_OK;
}

extern "C" pw_status pw_cell_set_projectors(pw_cell *c, int onthefly, void *stream) {
  if (!c || (onthefly != 0 && onthefly != 1)) return PW_ERR_ARG;
  if (c->natom == 0 || onthefly == c->proj_onthefly) return PW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  PW_CUDA(cudaStreamSynchronize(st));
  // the stored split operands of beta go either way (rebuilt on first use)
  pw_tc_operand **ops[] = {&c->op_beta_rows, &c->op_beta_t};
  for (pw_tc_operand **o : ops)
    if (*o) { pw_tc_operand_free(*o); delete *o; *o = nullptr; }
  if (onthefly) {
    cudaFree(c->d_beta);
    c->d_beta = nullptr;
    c->proj_onthefly = 1;
    return PW_OK;
  }
  if (cudaMalloc(&c->d_beta, (size_t)c->npw * c->nproj * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    c->d_beta = nullptr;
    return PW_ERR_OOM;
  }
  PW_TRY(pw_beta_chunk(c, 0, c->natom, c->d_beta, st));
  PW_CUDA(cudaStreamSynchronize(st));
  cudaFree(c->d_bchunk);
  c->d_bchunk = nullptr;
  c->bchunk_bytes = 0;
  c->proj_onthefly = 0;
  return PW_OK;
}
