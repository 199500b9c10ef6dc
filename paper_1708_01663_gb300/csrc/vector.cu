// The 3D vectorial model of the appendix ("3D Diffractive Imaging").
//
// Fields are E = (E^(1), E^(2), E^(3)) stored [T, 3, N] (component-major per
// transmitter), so the three components of a transmitter are three
// consecutive transforms of the scalar FFT convolution (ConvOp::tx_div = 3).
// With C = k^2 B = conv_G(f E) (G the k^2-weighted scalar matrix of Eq. 3, so
// B = G~ (f E) of the appendix):
//     A x   = x - C - D C / k^2                        (discrete constraint)
//     A^H x = x - conj(f) conv_{G^H}(x + D x / k^2)    (D real and symmetric)
// D is the appendix's finite-difference grad-div operator: the 3-point second
// difference for d^2/dx_c^2 and the 4-point diagonal stencil / (4 delta^2)
// for the mixed derivatives, acting on grid values only (neighbours outside
// the grid count as zero).  The forward matvec runs the stencil as the
// epilogue of the convolution (A x, b - A x and the dot slots of the Krylov
// solver); the adjoint runs it before the convolution, whose inverse-row
// epilogue then forms the result.  Dot partials of both land in
// [T][3 nblk][DOT_SLOTS] (component-major), the layout the solver's scalar
// step sums.
//
// Tables: H~ [M, 3N] = delta^3 times row 3 of the dyadic Green's function
//     G(r) = k^2 [ (3/(kd)^2 - 3j/(kd) - 1) r^ r^T + (1 + j/(kd) - 1/(kd)^2) I ] g(d)
// (the receivers measure the z component), and polarised plane waves
// E_in,t = p_t exp(j k d_t . r).
#include <math.h>

#include "common.cuh"
#include "dots.cuh"

namespace cisor {

// (D F)^(C) at voxel v = (ix, iy, iz) of the 3-component field F (component stride N)
template <int C>
__device__ __forceinline__ float2 graddiv_at(const float2* __restrict__ F, int N, int n, int ix, int iy, int iz, int v,
                                            float inv_d2) {
  const int coord[3] = {ix, iy, iz};
  const int stride[3] = {1, n, n * n};
  const float2* Fc = F + C * N;
  float2 acc = c_scale(Fc[v], -2.f);
  if (coord[C] > 0) acc = c_add(acc, Fc[v - stride[C]]);
  if (coord[C] < n - 1) acc = c_add(acc, Fc[v + stride[C]]);
  acc = c_scale(acc, inv_d2);
  float2 mix = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j == C) continue;
    const float2* Fj = F + j * N;
#pragma unroll
    for (int sc = -1; sc <= 1; sc += 2)
#pragma unroll
      for (int sj = -1; sj <= 1; sj += 2) {
        const int qc = coord[C] + sc, qj = coord[j] + sj;
        if (qc < 0 || qc >= n || qj < 0 || qj >= n) continue;
        const float2 val = Fj[v + sc * stride[C] + sj * stride[j]];
        mix = (sc * sj > 0) ? c_add(mix, val) : c_sub(mix, val);
      }
  }
  return c_add(acc, c_scale(mix, 0.25f * inv_d2));
}

struct VecEpiArgs {
  const float2* C;      // conv output [ntx, 3, N] (forward) or the field x (pre-pass)
  const float2* x;      // the x of A x
  const float2* aux;
  float2* out;
  float2* out2;
  int epi;              // EPI_MATVEC, EPI_RESID; -1: pre-pass w = x + D x / k^2
  int dot_a[DOT_SLOTS], dot_b[DOT_SLOTS];
  const int* active;
  float* part;
  int n, RB, nblk;
  long long N;
  float inv_k2, inv_d2;
};

// RB x rows (RB n voxels) of component C of transmitter blockIdx.z (N < 2^31: n <= 64).
template <int C>
__device__ __forceinline__ void vec_stencil_body(const VecEpiArgs& a) {
  const int rb = blockIdx.x, t = blockIdx.z;
  const int N = (int)a.N, n = a.n;
  const long long base = (long long)t * 3 * N;
  const float2* F = a.C + base;
  const int v0 = rb * a.RB * n;
  const int v1 = min(N, v0 + a.RB * n);
  const bool any_dot = a.epi >= 0 && (a.dot_a[0] | a.dot_a[1] | a.dot_a[2]) != 0;
  const bool need_aux = a.epi == EPI_RESID || a.dot_a[0] == OP_AUX || a.dot_b[0] == OP_AUX ||
                        a.dot_a[1] == OP_AUX || a.dot_b[1] == OP_AUX || a.dot_a[2] == OP_AUX || a.dot_b[2] == OP_AUX;
  float2 acc[DOT_SLOTS];
#pragma unroll
  for (int s = 0; s < DOT_SLOTS; ++s) acc[s] = make_float2(0.f, 0.f);
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const int row = v / n, ix = v - row * n, iz = row / n, iy = row - iz * n;
    const float2 dc = graddiv_at<C>(F, N, n, ix, iy, iz, v, a.inv_d2);
    const long long idx = base + (long long)C * N + v;
    if (a.epi < 0) {  // pre-pass of the adjoint: w = x + D x / k^2
      a.out[idx] = c_add(F[C * N + v], c_scale(dc, a.inv_k2));
      continue;
    }
    const float2 xv = a.x[idx];
    float2 y = c_sub(c_sub(xv, F[C * N + v]), c_scale(dc, a.inv_k2));
    const float2 av = need_aux ? a.aux[idx] : make_float2(0.f, 0.f);
    if (a.epi == EPI_RESID) y = c_sub(av, y);
    a.out[idx] = y;
    if (a.out2) a.out2[idx] = y;
    if (any_dot) {
#pragma unroll
      for (int s = 0; s < DOT_SLOTS; ++s)
        if (a.dot_a[s]) acc[s] = c_add(acc[s], c_cjmul(pick(a.dot_a[s], y, xv, av), pick(a.dot_b[s], y, xv, av)));
    }
  }
  if (any_dot)
    block_dots<256>(acc, reinterpret_cast<float2*>(a.part) + (((size_t)t * 3 + C) * a.nblk + rb) * DOT_SLOTS);
}

// One CTA: RB x rows of component blockIdx.y of transmitter blockIdx.z.
__global__ void __launch_bounds__(256) vec_stencil_kernel(const VecEpiArgs a) {
  if (a.active && !a.active[blockIdx.z]) return;
  switch (blockIdx.y) {
    case 0: vec_stencil_body<0>(a); break;
    case 1: vec_stencil_body<1>(a); break;
    default: vec_stencil_body<2>(a); break;
  }
}

static VecEpiArgs stencil_args(cisor_ctx* c) {
  VecEpiArgs a{};
  a.n = c->n;
  a.N = c->N;
  a.RB = conv_rows_per_block(c->P);
  a.nblk = c->nblk;
  a.part = c->part;
  a.inv_k2 = (float)(1.0 / (c->k * c->k));
  a.inv_d2 = (float)(1.0 / (c->delta * c->delta));
  return a;
}

static cisor_status launch_stencil(cisor_ctx* c, const VecEpiArgs& a, int ntx) {
  dim3 g(c->nblk, 3, ntx);
  vec_stencil_kernel<<<g, 256, 0, c->stream>>>(a);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

cisor_status vec_matvec(cisor_ctx* c, const VecOp& op) {
  if (!op.adjoint) {
    ConvOp co{};
    co.mul_f = 1;
    co.prologue = PRO_COPY;
    co.src = op.x;
    co.epilogue = EPI_CONV_ADD;
    co.out = c->vbuf;
    co.f = c->f;
    co.ntx = 3 * op.ntx;
    co.tx_div = 3;
    co.active = op.active;
    CISOR_TRY(conv_pass(c, co));
    VecEpiArgs a = stencil_args(c);
    a.C = c->vbuf;
    a.x = op.x;
    a.aux = op.aux;
    a.out = op.out;
    a.out2 = op.out2;
    a.epi = op.epilogue;
    for (int s = 0; s < DOT_SLOTS; ++s) {
      a.dot_a[s] = op.dot_a[s];
      a.dot_b[s] = op.dot_b[s];
    }
    a.active = op.active;
    return launch_stencil(c, a, op.ntx);
  }
  VecEpiArgs a = stencil_args(c);
  a.C = op.x;
  a.out = c->vbuf;
  a.epi = -1;
  a.active = op.active;
  CISOR_TRY(launch_stencil(c, a, op.ntx));
  ConvOp co{};
  co.adjoint = 1;
  co.mul_f = 1;
  co.prologue = PRO_COPY;
  co.src = c->vbuf;
  co.epilogue = op.epilogue;
  co.esrc = op.x;
  co.aux = op.aux;
  co.out = op.out;
  co.out2 = op.out2;
  for (int s = 0; s < DOT_SLOTS; ++s) {
    co.dot_a[s] = op.dot_a[s];
    co.dot_b[s] = op.dot_b[s];
  }
  co.part = c->part;
  co.f = c->f;
  co.ntx = 3 * op.ntx;
  co.tx_div = 3;
  co.active = op.active;
  return conv_pass(c, co);
}

cisor_status vec_gz(cisor_ctx* c) {
  VecEpiArgs a = stencil_args(c);
  a.C = c->vadj;
  a.out = c->vbuf;
  a.epi = -1;
  CISOR_TRY(launch_stencil(c, a, c->T));
  ConvOp co{};
  co.adjoint = 1;
  co.prologue = PRO_COPY;
  co.src = c->vbuf;
  co.epilogue = EPI_CONV_ADD;
  co.aux = c->z;
  co.out = c->gz;
  co.f = c->f;
  co.ntx = 3 * c->T;
  co.tx_div = 3;
  return conv_pass(c, co);
}

// p = r + beta (p - omega v) (p = r when beta = 0) and s = r - alpha v over [ntx, Nf]
__global__ void __launch_bounds__(256) vec_pupdate_kernel(long long Nf, const int* __restrict__ active,
                                                          const double* __restrict__ scal, const float2* __restrict__ r,
                                                          float2* __restrict__ p, const float2* __restrict__ v) {
  const int t = blockIdx.y;
  if (!active[t]) return;
  const double2* sc = reinterpret_cast<const double2*>(scal) + (size_t)t * SC_STRIDE;
  const float2 beta = z_to_c(sc[SC_BETA]), omega = z_to_c(sc[SC_OMEGA]);
  const bool fresh = beta.x == 0.f && beta.y == 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nf; i += (long long)gridDim.x * blockDim.x) {
    const long long k = (long long)t * Nf + i;
    p[k] = fresh ? r[k] : c_add(r[k], c_mul(beta, c_sub(p[k], c_mul(omega, v[k]))));
  }
}

__global__ void __launch_bounds__(256) vec_axpy_kernel(long long Nf, const int* __restrict__ active,
                                                       const double* __restrict__ scal, const float2* __restrict__ r,
                                                       const float2* __restrict__ v, float2* __restrict__ s) {
  const int t = blockIdx.y;
  if (!active[t]) return;
  const float2 alpha = z_to_c(reinterpret_cast<const double2*>(scal)[(size_t)t * SC_STRIDE + SC_ALPHA]);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nf; i += (long long)gridDim.x * blockDim.x) {
    const long long k = (long long)t * Nf + i;
    s[k] = c_sub(r[k], c_mul(alpha, v[k]));
  }
}

static unsigned vec_blocks(long long Nf) {
  const long long b = (Nf + 1023) / 1024;
  return (unsigned)(b < 1 ? 1 : b);
}

cisor_status vec_pupdate(cisor_ctx* c, int ntx) {
  vec_pupdate_kernel<<<dim3(vec_blocks(c->Nf), ntx), 256, 0, c->stream>>>(c->Nf, c->active, c->scal, c->r, c->p, c->v);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

cisor_status vec_axpy(cisor_ctx* c, int ntx) {
  vec_axpy_kernel<<<dim3(vec_blocks(c->Nf), ntx), 256, 0, c->stream>>>(c->Nf, c->active, c->scal, c->r, c->v, c->s);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

// ---------------------------------------------------------------- tables (FP64)
__global__ void dyadic_sensing_kernel(float2* H, const double* rx, int M, int n, double delta, double k) {
  const long long N = (long long)n * n * n, K = 3 * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * K) return;
  const int m = (int)(idx / K);
  const long long rem = idx % K;
  const int c = (int)(rem / N);
  const long long p = rem % N;
  const double h = n / 2.0 - 0.5;
  const double dx = rx[3 * m] - ((int)(p % n) - h) * delta;
  const double dy = rx[3 * m + 1] - ((int)((p / n) % n) - h) * delta;
  const double dz = rx[3 * m + 2] - ((int)(p / ((long long)n * n)) - h) * delta;
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  const double rh[3] = {dx / d, dy / d, dz / d};
  const double kd = k * d;
  double sn, cs;
  sincos(kd, &sn, &cs);
  const double2 g = make_double2(cs / (4.0 * 3.14159265358979323846 * d), sn / (4.0 * 3.14159265358979323846 * d));
  // a = 3/(kd)^2 - 1 - 3j/(kd), b = 1 - 1/(kd)^2 + j/(kd)
  const double2 av = make_double2(3.0 / (kd * kd) - 1.0, -3.0 / kd);
  const double2 bv = make_double2(1.0 - 1.0 / (kd * kd), 1.0 / kd);
  double2 coef = make_double2(av.x * rh[2] * rh[c], av.y * rh[2] * rh[c]);
  if (c == 2) coef = z_add(coef, bv);
  const double s = k * k * delta * delta * delta;
  const double2 v = z_mul(coef, g);
  H[idx] = make_float2((float)(s * v.x), (float)(s * v.y));
}

__global__ void polarised_wave_kernel(float2* u, const double* tx, int T, int n, double delta, double k) {
  const long long N = (long long)n * n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)T * 3 * N) return;
  const int t = (int)(idx / (3 * N));
  const long long rem = idx % (3 * N);
  const int c = (int)(rem / N);
  const long long p = rem % N;
  const double h = n / 2.0 - 0.5;
  const double* d = tx + 6 * t;
  const double ph = k * delta * (d[0] * ((int)(p % n) - h) + d[1] * ((int)((p / n) % n) - h) +
                                 d[2] * ((int)(p / ((long long)n * n)) - h));
  double sn, cs;
  sincos(ph, &sn, &cs);
  const double pol = d[3 + c];
  u[idx] = make_float2((float)(pol * cs), (float)(pol * sn));
}

cisor_status vec_tables(cisor_ctx* c, const double* d_tx, const double* d_rx) {
  const long long MK = (long long)c->M * c->Nf, TK = (long long)c->T * c->Nf;
  dyadic_sensing_kernel<<<(unsigned)((MK + 255) / 256), 256, 0, c->stream>>>(c->H, d_rx, c->M, c->n, c->delta, c->k);
  CISOR_CUDA(cudaGetLastError());
  polarised_wave_kernel<<<(unsigned)((TK + 255) / 256), 256, 0, c->stream>>>(c->u_in, d_tx, c->T, c->n, c->delta, c->k);
  CISOR_CUDA(cudaGetLastError());
  return CISOR_OK;
}

}  // namespace cisor
