// One-time tables of a geometry, computed in FP64 on the device and stored
// as complex64: the spectrum of the circulant embedding of G (Sec. II, Eq. 3,
// made a pointwise product by the FFT, Sec. III-A), the sensing matrix H
// (Eq. 2), the incident plane waves and the FFT twiddles.
//
// Discretisation (readings of points the paper leaves open):
//  * g(r) = +(j/4) H0^(1)(k_b r) in 2D.  Eq. 1 prints -(j/4); only +j/4
//    agrees with the 3D kernel's sign and with u = u_in + k^2 int g f u.
//    In 3D g(r) = e^{j k_b r} / (4 pi r) as Eq. 1 prints it.
//  * G_ij = k^2 delta^d g(|r_i - r_j|) (midpoint rule, as the 3D
//    discretisation of Appendix A writes delta^3 sum g).
//  * G_ii (g is singular at 0): k^2 times the integral of g over the disk
//    (ball) of the pixel's area (voxel's volume):
//        2D, a = delta / sqrt(pi):       G_ii = k^2 [ (j pi a / (2 k_b)) H1^(1)(k_b a) - 1 / k_b^2 ]
//        3D, a = delta (3 / 4 pi)^(1/3): G_ii = (k / k_b)^2 [ (1 - j k_b a) e^{j k_b a} - 1 ]
// Bessel functions are CUDA's double-precision j0/y0/j1/y1.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "regfft.cuh"

namespace cisor {

__global__ void twiddle_kernel(float2* tw32, double2* tw64, int P) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= P) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)P, &s, &c);
  tw32[m] = make_float2((float)c, (float)s);
  tw64[m] = make_double2(c, s);
}

__device__ __forceinline__ double2 green2d_scaled(double r, double k, double kb, double delta) {
  // k^2 delta^2 (j/4) (J0 + j Y0)(kb r)
  double x = kb * r;
  double s = k * k * delta * delta * 0.25;
  return make_double2(-s * y0(x), s * j0(x));
}

__device__ __forceinline__ double2 self_term2d(double k, double kb, double delta) {
  const double a = delta * 0.56418958354775628695;  // delta / sqrt(pi)
  const double x = kb * a;
  const double c = 3.14159265358979323846 * a / (2.0 * kb);
  // (j c)(J1 + j Y1) - 1/kb^2
  return make_double2(k * k * (-c * y1(x) - 1.0 / (kb * kb)), k * k * c * j1(x));
}

__device__ __forceinline__ double2 green3d_scaled(double r, double k, double kb, double delta) {
  // k^2 delta^3 e^{j kb r} / (4 pi r)
  double sn, cs;
  sincos(kb * r, &sn, &cs);
  const double s = k * k * delta * delta * delta / (4.0 * 3.14159265358979323846 * r);
  return make_double2(s * cs, s * sn);
}

__device__ __forceinline__ double2 self_term3d(double k, double kb, double delta) {
  const double a = delta * 0.62035049089940001667;  // delta (3 / (4 pi))^(1/3)
  const double x = kb * a;
  double sn, cs;
  sincos(x, &sn, &cs);
  // (1 - j x)(cs + j sn) - 1
  const double s = (k * k) / (kb * kb);
  return make_double2(s * (cs + x * sn - 1.0), s * (sn - x * cs));
}

// First column of the P^3 circulant embedding of the 3D block-Toeplitz G.
__global__ void green_column3d_kernel(double2* cbuf, int n, int P, double delta, double k, double kb) {
  const int jx = blockIdx.x * blockDim.x + threadIdx.x;
  const int jy = blockIdx.y, jz = blockIdx.z;
  if (jx >= P) return;
  const int mx = jx < n ? jx : jx - P;
  const int my = jy < n ? jy : jy - P;
  const int mz = jz < n ? jz : jz - P;
  const bool used = (jx < n || jx > P - n) && (jy < n || jy > P - n) && (jz < n || jz > P - n);
  double2 v = make_double2(0.0, 0.0);
  if (used) {
    if (mx == 0 && my == 0 && mz == 0) {
      v = self_term3d(k, kb, delta);
    } else {
      const double r = delta * sqrt((double)mx * mx + (double)my * my + (double)mz * mz);
      v = green3d_scaled(r, k, kb, delta);
    }
  }
  cbuf[((size_t)jz * P + jy) * P + jx] = v;
}

// First column of the P x P circulant embedding: axis index j holds offset
// j (j < n), j - P (j > P - n), and nothing in between.
__global__ void green_column_kernel(double2* cbuf, int n, int P, double delta, double k, double kb) {
  int jx = blockIdx.x * blockDim.x + threadIdx.x;
  int jy = blockIdx.y;
  if (jx >= P) return;
  int mx = jx < n ? jx : jx - P;
  int my = jy < n ? jy : jy - P;
  bool used = (jx < n || jx > P - n) && (jy < n || jy > P - n);
  double2 v = make_double2(0.0, 0.0);
  if (used) {
    if (mx == 0 && my == 0) {
      v = self_term2d(k, kb, delta);
    } else {
      double r = delta * sqrt((double)mx * mx + (double)my * my);
      v = green2d_scaled(r, k, kb, delta);
    }
  }
  cbuf[(size_t)jy * P + jx] = v;
}

template <int P>
__global__ void fft64_rows_kernel(double2* data, const double2* tw_g) {
  extern __shared__ double2 sm64[];
  double2* tw = sm64;
  double2* a = tw + P;
  double2* b = a + P;
  const int tid = threadIdx.x, nthr = blockDim.x;
  double2* row = data + (size_t)blockIdx.x * P;
  for (int i = tid; i < P; i += nthr) {
    tw[i] = tw_g[i];
    a[i] = row[i];
  }
  __syncthreads();
  double2* res = block_fft<P, false, false>(a, b, 1, P, 1, tw, tid, nthr);
  for (int i = tid; i < P; i += nthr) row[i] = res[i];
}

// FFT of the columns c0 .. c0 + W - 1 (element stride es) of slab blockIdx.y
// (offset blockIdx.y * slab): in place in FP64, or into out32 scaled.
template <int P>
__global__ void fft64_cols_kernel(double2* data, const double2* tw_g, size_t es, size_t slab, float2* out32,
                                  double scale) {
  constexpr int W = 2;
  extern __shared__ double2 sm64[];
  double2* tw = sm64;
  double2* a = tw + P;
  double2* b = a + P * W;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const size_t c0 = blockIdx.y * slab + (size_t)blockIdx.x * W;
  for (int i = tid; i < P; i += nthr) tw[i] = tw_g[i];
  for (int e = tid; e < P * W; e += nthr) {
    int i = e / W, w = e % W;
    a[e] = data[i * es + c0 + w];
  }
  __syncthreads();
  double2* res = block_fft<P, false, true>(a, b, W, 1, W, tw, tid, nthr);
  for (int e = tid; e < P * W; e += nthr) {
    int i = e / W, w = e % W;
    double2 v = res[e];
    if (out32)
      out32[i * es + c0 + w] = make_float2((float)(v.x * scale), (float)(v.y * scale));
    else
      data[i * es + c0 + w] = v;
  }
}

__global__ void sensing_kernel(float2* H, const double* rx, int M, int n, double delta, double k, double kb) {
  long long N = (long long)n * n;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  int m = (int)(idx / N);
  int p = (int)(idx % N);
  int ix = p % n, iy = p / n;
  double x = (ix - n / 2.0 + 0.5) * delta, y = (iy - n / 2.0 + 0.5) * delta;
  double dx = rx[2 * m] - x, dy = rx[2 * m + 1] - y;
  double2 g = green2d_scaled(sqrt(dx * dx + dy * dy), k, kb, delta);
  H[idx] = make_float2((float)g.x, (float)g.y);
}

__global__ void sensing3d_kernel(float2* H, const double* rx, int M, int n, double delta, double k, double kb) {
  const long long N = (long long)n * n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int m = (int)(idx / N);
  const long long p = idx % N;
  const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / ((long long)n * n));
  const double h = n / 2.0 - 0.5;
  const double dx = rx[3 * m] - (ix - h) * delta, dy = rx[3 * m + 1] - (iy - h) * delta,
               dz = rx[3 * m + 2] - (iz - h) * delta;
  const double2 g = green3d_scaled(sqrt(dx * dx + dy * dy + dz * dz), k, kb, delta);
  H[idx] = make_float2((float)g.x, (float)g.y);
}

// exp(j kb d_t . r) for unit directions d_t (3D plane waves)
__global__ void plane_wave3d_kernel(float2* u, const double* dir, int T, int n, double delta, double kb) {
  const long long N = (long long)n * n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)T * N) return;
  const int t = (int)(idx / N);
  const long long p = idx % N;
  const int ix = (int)(p % n), iy = (int)((p / n) % n), iz = (int)(p / ((long long)n * n));
  const double h = n / 2.0 - 0.5;
  const double ph = kb * (dir[3 * t] * (ix - h) * delta + dir[3 * t + 1] * (iy - h) * delta +
                          dir[3 * t + 2] * (iz - h) * delta);
  double s, c;
  sincos(ph, &s, &c);
  u[idx] = make_float2((float)c, (float)s);
}

// Field of a unit point (3D) or line (2D) source at src_t: g(|r - src_t|) of
// Eq. 1 without the quadrature weight k^2 delta^d.  Sources lie outside the grid.
__global__ void point_source_kernel(float2* u, const double* src, int T, int n, int dim, double delta, double kb) {
  const long long N = dim == 3 ? (long long)n * n * n : (long long)n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)T * N) return;
  const int t = (int)(idx / N);
  const long long p = idx % N;
  const double h = n / 2.0 - 0.5;
  const double x = ((int)(p % n) - h) * delta, y = ((int)((p / n) % n) - h) * delta;
  const double z = dim == 3 ? ((int)(p / ((long long)n * n)) - h) * delta : 0.0;
  const double dx = src[dim * t] - x, dy = src[dim * t + 1] - y, dz = dim == 3 ? src[3 * t + 2] - z : 0.0;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double2 g;
  if (dim == 3) {
    double sn, cs;
    sincos(kb * r, &sn, &cs);
    const double s = 1.0 / (4.0 * 3.14159265358979323846 * r);
    g = make_double2(s * cs, s * sn);
  } else {
    g = make_double2(-0.25 * y0(kb * r), 0.25 * j0(kb * r));  // (j/4)(J0 + j Y0)
  }
  u[idx] = make_float2((float)g.x, (float)g.y);
}

__global__ void plane_wave_kernel(float2* u, const double* ang, int T, int n, double delta, double kb) {
  long long N = (long long)n * n;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)T * N) return;
  int t = (int)(idx / N);
  int p = (int)(idx % N);
  int ix = p % n, iy = p / n;
  double x = (ix - n / 2.0 + 0.5) * delta, y = (iy - n / 2.0 + 0.5) * delta;
  double s, c, sa, ca;
  sincos(ang[t], &sa, &ca);
  sincos(kb * (ca * x + sa * y), &s, &c);
  u[idx] = make_float2((float)c, (float)s);
}

// Stage twiddle tables of the forward plan (slot 0) and the reversed plan (slot 1).
template <int P, bool REV>
__global__ void stage_twiddle_kernel(float2* out) {
  typedef TwTable<P, REV> TT;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= TT::SIZE) return;
  int ns, R, off;
  if (e < TT::OFF2 || RPlan<P>::NSTAGE == 2) {
    ns = TT::R0;
    R = TT::R1;
    off = TT::OFF1;
  } else {
    ns = TT::R0 * TT::R1;
    R = TT::R2;
    off = TT::OFF2;
  }
  const int r = (e - off) / ns + 1, k = (e - off) % ns;
  double s, c;
  sincospi(-2.0 * (double)r * k / ((double)ns * R), &s, &c);
  out[e] = make_float2((float)c, (float)s);
}

template <int P>
static cisor_status stage_twiddles(cisor_ctx* c) {
  stage_twiddle_kernel<P, false><<<(TW_STRIDE + 127) / 128, 128, 0, c->stream>>>(c->twst);
  CISOR_CUDA(cudaGetLastError());
  stage_twiddle_kernel<P, true><<<(TW_STRIDE + 127) / 128, 128, 0, c->stream>>>(c->twst + TW_STRIDE);
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

cisor_status make_stage_twiddles(cisor_ctx* c) {
  switch (c->P) {
    case 64: return stage_twiddles<64>(c);
    case 128: return stage_twiddles<128>(c);
    case 256: return stage_twiddles<256>(c);
    case 512: return stage_twiddles<512>(c);
  }
  set_error("unsupported FFT size %d", c->P);
  return CISOR_ERR_INVALID_ARG;
}

// FP64 FFT of the P^d circulant column (x rows, then y, then z columns),
// stored complex64 scaled by 1/P^d.
template <int P>
static cisor_status spectrum_fft(cisor_ctx* c, double2* cbuf, const double2* tw64) {
  size_t sm_rows = 3 * P * sizeof(double2);
  size_t sm_cols = (P + 2 * P * 2) * sizeof(double2);
  const size_t PP = (size_t)P * P;
  CISOR_CUDA(cudaFuncSetAttribute(fft64_cols_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_cols));
  if (c->dim == 3) {
    fft64_rows_kernel<P><<<(unsigned)PP, 128, sm_rows, c->stream>>>(cbuf, tw64);
    CISOR_CUDA(cudaGetLastError());
    fft64_cols_kernel<P><<<dim3(P / 2, P), 128, sm_cols, c->stream>>>(cbuf, tw64, P, PP, nullptr, 1.0);
    CISOR_CUDA(cudaGetLastError());
    fft64_cols_kernel<P><<<dim3((unsigned)(PP / 2), 1), 128, sm_cols, c->stream>>>(cbuf, tw64, PP, 0, c->ghat,
                                                                                  1.0 / ((double)PP * P));
  } else {
    fft64_rows_kernel<P><<<P, 128, sm_rows, c->stream>>>(cbuf, tw64);
    CISOR_CUDA(cudaGetLastError());
    fft64_cols_kernel<P><<<P / 2, 128, sm_cols, c->stream>>>(cbuf, tw64, P, 0, c->ghat, 1.0 / ((double)PP));
  }
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

cisor_status build_tables(cisor_ctx* c) {
  const int P = c->P, n = c->n, d = c->dim;
  const size_t cells = d == 3 ? (size_t)P * P * P : (size_t)P * P;
  double2* cbuf = nullptr;
  double2* tw64 = nullptr;
  double* d_rx = nullptr;
  double* d_ang = nullptr;
  CISOR_CUDA(cudaMallocAsync((void**)&cbuf, sizeof(double2) * cells, c->stream));
  CISOR_CUDA(cudaMallocAsync((void**)&tw64, sizeof(double2) * P, c->stream));
  CISOR_CUDA(cudaMallocAsync((void**)&d_rx, sizeof(double) * c->rx_pos.size(), c->stream));
  CISOR_CUDA(cudaMallocAsync((void**)&d_ang, sizeof(double) * c->tx_angles.size(), c->stream));
  CISOR_CUDA(cudaMemcpyAsync(d_rx, c->rx_pos.data(), sizeof(double) * c->rx_pos.size(), cudaMemcpyHostToDevice,
                             c->stream));
  CISOR_CUDA(cudaMemcpyAsync(d_ang, c->tx_angles.data(), sizeof(double) * c->tx_angles.size(), cudaMemcpyHostToDevice,
                             c->stream));

  twiddle_kernel<<<(P + 127) / 128, 128, 0, c->stream>>>(c->tw, tw64, P);
  CISOR_CUDA(cudaGetLastError());
  if (d == 3)
    green_column3d_kernel<<<dim3((P + 127) / 128, P, P), 128, 0, c->stream>>>(cbuf, n, P, c->delta, c->k, c->kb);
  else
    green_column_kernel<<<dim3((P + 127) / 128, P), 128, 0, c->stream>>>(cbuf, n, P, c->delta, c->k, c->kb);
  CISOR_CUDA(cudaGetLastError());
  switch (P) {
    case 64: CISOR_TRY(spectrum_fft<64>(c, cbuf, tw64)); CISOR_TRY(stage_twiddles<64>(c)); break;
    case 128: CISOR_TRY(spectrum_fft<128>(c, cbuf, tw64)); CISOR_TRY(stage_twiddles<128>(c)); break;
    case 256: CISOR_TRY(spectrum_fft<256>(c, cbuf, tw64)); CISOR_TRY(stage_twiddles<256>(c)); break;
    case 512: CISOR_TRY(spectrum_fft<512>(c, cbuf, tw64)); CISOR_TRY(stage_twiddles<512>(c)); break;
    default: set_error("unsupported FFT size %d", P); return CISOR_ERR_INVALID_ARG;
  }
  long long MN = (long long)c->M * c->N;
  long long TN = (long long)c->T * c->N;
  if (c->ncomp == 3) {  // vectorial model: dyadic sensing row and polarised plane waves
    CISOR_TRY(vec_tables(c, d_ang, d_rx));
  } else if (d == 3)
    sensing3d_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, c->stream>>>(c->H, d_rx, c->M, n, c->delta, c->k, c->kb);
  else
    sensing_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, c->stream>>>(c->H, d_rx, c->M, n, c->delta, c->k, c->kb);
  CISOR_CUDA(cudaGetLastError());
  CISOR_TRY(sense_tc_prepare(c));
  const unsigned gT = (unsigned)((TN + 255) / 256);
  if (c->ncomp == 3)
    ;  // incident fields written by vec_tables
  else if (c->tx_kind == 1)
    point_source_kernel<<<gT, 256, 0, c->stream>>>(c->u_in, d_ang, c->T, n, d, c->delta, c->kb);
  else if (d == 3)
    plane_wave3d_kernel<<<gT, 256, 0, c->stream>>>(c->u_in, d_ang, c->T, n, c->delta, c->kb);
  else
    plane_wave_kernel<<<gT, 256, 0, c->stream>>>(c->u_in, d_ang, c->T, n, c->delta, c->kb);
  CISOR_CUDA(cudaGetLastError());
  CISOR_CUDA(cudaFreeAsync(cbuf, c->stream));
  CISOR_CUDA(cudaFreeAsync(tw64, c->stream));
  CISOR_CUDA(cudaFreeAsync(d_rx, c->stream));
  CISOR_CUDA(cudaFreeAsync(d_ang, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  return CISOR_OK;
}

}  // namespace cisor
