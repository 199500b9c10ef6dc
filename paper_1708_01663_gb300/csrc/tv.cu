// prox of gamma R, R = tau TV_iso + chi_C (Eq. 8), by the fast gradient
// projection (FGP) method of Beck and Teboulle (IEEE TIP 2009), which the
// paper cites for this prox (Sec. III-A) without restating it.  On the dual
// p = (p_x, p_y), with lam = gamma tau, D the forward difference (zero at the
// last index) and P_C the box clamp:
//     x(r)    = P_C(z - lam D^T r)
//     p_k     = Pi_unit-disk(r_k + D x(r_k) / (8 lam))
//     t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
//     r_{k+1} = p_k + ((t_k - 1) / t_{k+1}) (p_k - p_{k-1})
// from r_1 = p_0 = 0, t_1 = 1; output x(p_K).  One kernel per FGP iteration
// (r ping-pongs between two buffers; p is updated in place per pixel); the
// right neighbour's x comes from the next lane by warp shuffle.  Complex f
// takes the separable prox: Re and Im planes, each with its own box.
// The last kernel also applies the relaxed-FISTA momentum of Eq. 11,
// s_{k+1} = f_k + beta (f_k - f_{k-1}).
// 3D volumes take the same iteration with p = (p_x, p_y, p_z), the unit-ball
// projection in R^3 and the dual step 1 / (12 lam) (||D||^2 <= 4 d).
//
// Anisotropic TV (tv_kind 1): R = tau sum_d sum_n |[D_d x]_n| + chi_C, the
// alternative Sec. III-A points to (Kamilov, IEEE TIP 2017).  Along each axis
// the differences split into pairs (i, i+1) with i even and with i odd; each
// parity is a sum over disjoint pairs whose prox keeps the pair's mean and
// soft-thresholds its difference by 2c.  With the box, m = 2d + 1 pieces f_j,
// and prox_{sum f_j}(z) comes from the parallel Dykstra-like proximal
// iteration (Combettes and Pesquet 2011): z_j = z; repeat p_j = prox_{m f_j}(z_j),
// x = mean_j p_j, z_j += x - p_j.  Every step is pointwise (a pixel needs its
// pair partner along each axis), so one kernel per iteration, ping-ponging the
// 2d + 1 auxiliary images between two buffers.
#include <math.h>

#include "common.cuh"

namespace cisor {

// Dual planes: component k of plane c at (dim * c + k) * N.
__global__ void tv_split_kernel(const float2* __restrict__ z, float* __restrict__ zp, float* __restrict__ r,
                                float* __restrict__ p, long long N, int ncomp, int dim) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float2 v = z[i];
  zp[i] = v.x;
  if (ncomp == 2) zp[N + i] = v.y;
  for (int k = 0; k < dim * ncomp; ++k) {
    r[k * N + i] = 0.f;
    p[k * N + i] = 0.f;
  }
}

// (D^T r)(iy, ix) for the forward difference with zero difference at the last index
__device__ __forceinline__ float dt_at(const float* __restrict__ rx, const float* __restrict__ ry, int iy, int ix,
                                       int n) {
  const int i = iy * n + ix;
  float v = 0.f;
  if (ix < n - 1) v -= rx[i];
  if (ix > 0) v += rx[i - 1];
  if (iy < n - 1) v -= ry[i];
  if (iy > 0) v += ry[i - n];
  return v;
}

__global__ void tv_iter_kernel(const float* __restrict__ zp, const float* __restrict__ rin, float* __restrict__ rout,
                               float* __restrict__ p, int n, float lam, float step, float beta, float lo0, float hi0,
                               float lo1, float hi1) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y, c = blockIdx.z;
  const long long N = (long long)n * n;
  const float lo = c ? lo1 : lo0, hi = c ? hi1 : hi0;
  const float* z = zp + c * N;
  const float* rx = rin + 2 * c * N;
  const float* ry = rx + N;
  const bool valid = ix < n;
  const int xi = valid ? ix : n - 1;
  const int i = iy * n + xi;
  const float x0 = fminf(fmaxf(z[i] - lam * dt_at(rx, ry, iy, xi, n), lo), hi);
  // right neighbour from the next lane; the last lane of a warp computes it itself
  float xr = __shfl_down_sync(0xffffffffu, x0, 1);
  const int lane = threadIdx.x & 31;
  if (lane == 31 && xi < n - 1) xr = fminf(fmaxf(z[i + 1] - lam * dt_at(rx, ry, iy, xi + 1, n), lo), hi);
  if (!valid) return;
  const float dx = (ix < n - 1) ? xr - x0 : 0.f;
  float dy = 0.f;
  if (iy < n - 1) dy = fminf(fmaxf(z[i + n] - lam * dt_at(rx, ry, iy + 1, ix, n), lo), hi) - x0;
  const float qx = rx[i] + step * dx, qy = ry[i] + step * dy;
  const float nrm = fmaxf(1.f, sqrtf(qx * qx + qy * qy));
  const float px = qx / nrm, py = qy / nrm;
  float* pc = p + 2 * c * N;
  const float pox = pc[i], poy = pc[N + i];
  pc[i] = px;
  pc[N + i] = py;
  float* ro = rout + 2 * c * N;
  ro[i] = px + beta * (px - pox);
  ro[N + i] = py + beta * (py - poy);
}

// (D^T r) at voxel (iz, iy, ix) of an n^3 volume
__device__ __forceinline__ float dt3_at(const float* __restrict__ rx, const float* __restrict__ ry,
                                        const float* __restrict__ rz, int iz, int iy, int ix, int n) {
  const long long nn = (long long)n * n;
  const long long i = iz * nn + (long long)iy * n + ix;
  float v = 0.f;
  if (ix < n - 1) v -= rx[i];
  if (ix > 0) v += rx[i - 1];
  if (iy < n - 1) v -= ry[i];
  if (iy > 0) v += ry[i - n];
  if (iz < n - 1) v -= rz[i];
  if (iz > 0) v += rz[i - nn];
  return v;
}

__global__ void tv_iter3_kernel(const float* __restrict__ zp, const float* __restrict__ rin, float* __restrict__ rout,
                                float* __restrict__ p, int n, float lam, float step, float beta, float lo0, float hi0,
                                float lo1, float hi1) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y, iz = blockIdx.z % n, c = blockIdx.z / n;
  const long long nn = (long long)n * n, N = nn * n;
  const float lo = c ? lo1 : lo0, hi = c ? hi1 : hi0;
  const float* z = zp + c * N;
  const float* rx = rin + 3 * c * N;
  const float* ry = rx + N;
  const float* rz = ry + N;
  const bool valid = ix < n;
  const int xi = valid ? ix : n - 1;
  const long long i = iz * nn + (long long)iy * n + xi;
  auto xat = [&](int zz, int yy, int xx, long long j) {
    return fminf(fmaxf(z[j] - lam * dt3_at(rx, ry, rz, zz, yy, xx, n), lo), hi);
  };
  const float x0 = xat(iz, iy, xi, i);
  // right neighbour from the next lane; the last lane of a warp computes it itself
  float xr = __shfl_down_sync(0xffffffffu, x0, 1);
  const int lane = threadIdx.x & 31;
  if (lane == 31 && xi < n - 1) xr = xat(iz, iy, xi + 1, i + 1);
  if (!valid) return;
  const float dx = (ix < n - 1) ? xr - x0 : 0.f;
  const float dy = (iy < n - 1) ? xat(iz, iy + 1, ix, i + n) - x0 : 0.f;
  const float dz = (iz < n - 1) ? xat(iz + 1, iy, ix, i + nn) - x0 : 0.f;
  const float qx = rx[i] + step * dx, qy = ry[i] + step * dy, qz = rz[i] + step * dz;
  const float nrm = fmaxf(1.f, sqrtf(qx * qx + qy * qy + qz * qz));
  const float px = qx / nrm, py = qy / nrm, pz = qz / nrm;
  float* pc = p + 3 * c * N;
  const float pox = pc[i], poy = pc[N + i], poz = pc[2 * N + i];
  pc[i] = px;
  pc[N + i] = py;
  pc[2 * N + i] = pz;
  float* ro = rout + 3 * c * N;
  ro[i] = px + beta * (px - pox);
  ro[N + i] = py + beta * (py - poy);
  ro[2 * N + i] = pz + beta * (pz - poz);
}

__global__ void tv_final_kernel(const float* __restrict__ zp, const float* __restrict__ p, int n, int dim, float lam,
                                float lo0, float hi0, float lo1, float hi1, int ncomp, float2* x, const float2* fprev,
                                float beta_mom, float2* __restrict__ s_out) {
  const long long N = dim == 3 ? (long long)n * n * n : (long long)n * n;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((long long)n * n));
  float xv[2] = {0.f, 0.f};
  for (int c = 0; c < ncomp; ++c) {
    const float lo = c ? lo1 : lo0, hi = c ? hi1 : hi0;
    const float* pc = p + dim * c * N;
    float d = 0.f;
    if (lam > 0.f) d = dim == 3 ? dt3_at(pc, pc + N, pc + 2 * N, iz, iy, ix, n) : dt_at(pc, pc + N, iy, ix, n);
    xv[c] = fminf(fmaxf(zp[c * N + i] - lam * d, lo), hi);
  }
  const float2 xo = make_float2(xv[0], xv[1]);
  if (s_out) {
    const float2 fp = fprev[i];  // read before x (x may alias fprev)
    s_out[i] = make_float2(xo.x + beta_mom * (xo.x - fp.x), xo.y + beta_mom * (xo.y - fp.y));
  }
  x[i] = xo;
}

// z_j = z for every piece j of every plane: layout (plane * m + j) * N
__global__ void tv_ppa_init_kernel(const float2* __restrict__ z, float* __restrict__ zs, long long N, int m,
                                   int ncomp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float2 v = z[i];
  for (int c = 0; c < ncomp; ++c)
    for (int j = 0; j < m; ++j) zs[((long long)c * m + j) * N + i] = c ? v.y : v.x;
}

__device__ __forceinline__ float soft(float d, float t) { return copysignf(fmaxf(fabsf(d) - t, 0.f), d); }

template <int D>
__global__ void __launch_bounds__(256) tv_ppa_kernel(const float* __restrict__ zin, float* __restrict__ zout, int n,
                                                     float cthr, float lo0, float hi0, float lo1, float hi1, int ncomp,
                                                     int last, float2* x_out, const float2* fprev, float beta_mom,
                                                     float2* __restrict__ s_out) {
  constexpr int M = 2 * D + 1;
  const long long nn = (long long)n * n;
  const long long N = D == 3 ? nn * n : nn;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int coord[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / nn)};
  const long long stride[3] = {1, n, nn};
  float xv[2] = {0.f, 0.f};
  for (int c = 0; c < ncomp; ++c) {
    const float* zc = zin + (long long)c * M * N;
    float zj[M], p[M];
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) {
      const int a = j >> 1, par = j & 1, pos = coord[a];
      const float* zp = zc + (long long)j * N;
      const float v = zp[i];
      zj[j] = v;
      const int rel = pos - par;
      float pj = v;
      if (rel >= 0 && (rel & 1) == 0 && pos + 1 < n) {  // first of the pair (pos, pos + 1)
        const float w = zp[i + stride[a]];
        pj = 0.5f * (v + w) - 0.5f * soft(w - v, 2.f * cthr);
      } else if (rel >= 1 && (rel & 1) == 1) {          // second of the pair (pos - 1, pos)
        const float w = zp[i - stride[a]];
        pj = 0.5f * (w + v) + 0.5f * soft(v - w, 2.f * cthr);
      }
      p[j] = pj;
      acc += pj;
    }
    const float lo = c ? lo1 : lo0, hi = c ? hi1 : hi0;
    zj[2 * D] = zc[(long long)(2 * D) * N + i];
    p[2 * D] = fminf(fmaxf(zj[2 * D], lo), hi);
    acc += p[2 * D];
    const float x = acc * (1.f / M);
    xv[c] = x;
    if (!last) {
      float* zo = zout + (long long)c * M * N;
#pragma unroll
      for (int j = 0; j < M; ++j) zo[(long long)j * N + i] = x + zj[j] - p[j];
    }
  }
  if (last) {
    const float2 xo = make_float2(xv[0], xv[1]);
    if (s_out) {
      const float2 fp = fprev[i];  // read before x (x may alias fprev)
      s_out[i] = make_float2(xo.x + beta_mom * (xo.x - fp.x), xo.y + beta_mom * (xo.y - fp.y));
    }
    x_out[i] = xo;
  }
}

cisor_status tv_prox_aniso(cisor_ctx* c, const float2* z, float2* x, double lam, int iters, double lo, double hi,
                           double lo_im, double hi_im, int complex_f, const float2* f_prev, double beta_mom,
                           float2* s_out) {
  if (!(lam > 0.0) || iters < 1)  // the prox of the box alone is the clamp (the FGP path's last kernel)
    return tv_prox(c, z, x, 0.0, 0, lo, hi, lo_im, hi_im, complex_f, f_prev, beta_mom, s_out);
  const long long N = c->N;
  const int ncomp = complex_f ? 2 : 1;
  const int m = 2 * c->dim + 1;
  const unsigned gN = (unsigned)((N + 255) / 256);
  tv_ppa_init_kernel<<<gN, 256, 0, c->stream>>>(z, c->tva0, N, m, ncomp);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  float* zin = c->tva0;
  float* zout = c->tva1;
  const float cthr = (float)(m * lam);
  for (int k = 0; k < iters; ++k) {
    const int last = k == iters - 1;
    if (c->dim == 3)
      tv_ppa_kernel<3><<<gN, 256, 0, c->stream>>>(zin, zout, c->n, cthr, (float)lo, (float)hi, (float)lo_im,
                                                  (float)hi_im, ncomp, last, x, f_prev, (float)beta_mom, s_out);
    else
      tv_ppa_kernel<2><<<gN, 256, 0, c->stream>>>(zin, zout, c->n, cthr, (float)lo, (float)hi, (float)lo_im,
                                                  (float)hi_im, ncomp, last, x, f_prev, (float)beta_mom, s_out);
    CISOR_CUDA(cudaGetLastError());
    c->launches += 1;
    float* t = zin;
    zin = zout;
    zout = t;
  }
  return CISOR_OK;
}

cisor_status tv_prox(cisor_ctx* c, const float2* z, float2* x, double lam, int iters, double lo, double hi,
                     double lo_im, double hi_im, int complex_f, const float2* f_prev, double beta_mom,
                     float2* s_out) {
  const int n = c->n;
  const long long N = c->N;
  const int ncomp = complex_f ? 2 : 1;
  const unsigned gN = (unsigned)((N + 255) / 256);
  const int dim = c->dim;
  tv_split_kernel<<<gN, 256, 0, c->stream>>>(z, c->tv_z, c->tv_r0, c->tv_p, N, ncomp, dim);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  if (lam > 0.0 && iters > 0) {
    const int bx = ((n + 31) / 32) * 32 > 256 ? 256 : ((n + 31) / 32) * 32;
    dim3 g((n + bx - 1) / bx, n, dim == 3 ? n * ncomp : ncomp);
    double t = 1.0;
    float* rin = c->tv_r0;
    float* rout = c->tv_r1;
    const float step = (float)(1.0 / (4.0 * dim * lam));
    for (int k = 0; k < iters; ++k) {
      const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
      const float beta = (float)((t - 1.0) / tn);
      if (dim == 3)
        tv_iter3_kernel<<<g, bx, 0, c->stream>>>(c->tv_z, rin, rout, c->tv_p, n, (float)lam, step, beta, (float)lo,
                                                 (float)hi, (float)lo_im, (float)hi_im);
      else
        tv_iter_kernel<<<g, bx, 0, c->stream>>>(c->tv_z, rin, rout, c->tv_p, n, (float)lam, step, beta, (float)lo,
                                                (float)hi, (float)lo_im, (float)hi_im);
      CISOR_CUDA(cudaGetLastError());
      c->launches += 1;
      float* tmp = rin;
      rin = rout;
      rout = tmp;
      t = tn;
    }
  }
  const float lam_f = (lam > 0.0 && iters > 0) ? (float)lam : 0.f;
  tv_final_kernel<<<gN, 256, 0, c->stream>>>(c->tv_z, c->tv_p, n, dim, lam_f, (float)lo, (float)hi, (float)lo_im,
                                             (float)hi_im, ncomp, x, f_prev, (float)beta_mom, s_out);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

}  // namespace cisor
