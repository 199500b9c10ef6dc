// Batched field solves A u_t = u_in,t and A^H v_t = b_t (Eq. 13).
//
// The paper solves both "by the conjugate gradient method" (Sec. III-A,
// after Eq. 13); A = I - G diag(f) is complex and not Hermitian, so this
// build reads that as a Krylov solver for non-Hermitian systems and uses
// BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992), one
// independent recurrence per transmitter, all transmitters in every launch.
// Vectors are complex64; inner products are FP32 per thread and FP64 across
// threads and blocks; the scalars (rho, alpha, omega, beta) are FP64.
//
// One iteration is 10 kernels:
//   conv(p = r + beta (p - omega v) ; v = A p ; <rhat, v>)     3 kernels
//   alpha = rho / <rhat, v>                                     scalar
//   conv(s = r - alpha v ; t = A s ; <t, s>, <t, t>)            3 kernels
//   omega = <t, s> / <t, t>                                     scalar
//   x += alpha p + omega s ; r = s - omega t ; <rhat,r>, <r,r>  update
//   rho' , beta, convergence / iteration cap / breakdown         scalar
// A transmitter whose recursive residual reaches tol is masked off (its CTAs
// exit at once).  Chunks of iterations are captured once into a CUDA graph
// and replayed; the host reads one counter per chunk.  At the end the true
// residual ||b - A x|| / ||b|| is recomputed with an explicit matvec and any
// transmitter above tol restarts from its current iterate (the stopping rule
// is always on the true residual of the paper's system).
#include <math.h>

#include "common.cuh"

namespace cisor {

enum { SCM_INIT = 0, SCM_ALPHA = 1, SCM_OMEGA = 2, SCM_RHO = 3, SCM_TRUE = 4 };

__global__ void bicg_scalar_kernel(int mode, int ntx, int nblk, const double* __restrict__ part,
                                   double* __restrict__ scal, int* __restrict__ active, int* __restrict__ iters,
                                   int* __restrict__ txflag, int* __restrict__ n_active,
                                   const double* __restrict__ params) {
  const int t = threadIdx.x;
  int act = 0;
  if (t < ntx) {
    const double tol = params[0];
    const int max_iter = (int)params[1];
    double2 d[DOT_SLOTS];
    for (int s = 0; s < DOT_SLOTS; ++s) d[s] = make_double2(0.0, 0.0);
    const double2* pp = reinterpret_cast<const double2*>(part) + (size_t)t * nblk * DOT_SLOTS;
    for (int b = 0; b < nblk; ++b)
      for (int s = 0; s < DOT_SLOTS; ++s) d[s] = z_add(d[s], pp[b * DOT_SLOTS + s]);
    double2* sc = reinterpret_cast<double2*>(scal) + (size_t)t * SC_STRIDE;
    act = active[t];
    if (mode == SCM_INIT) {
      const double bn2 = d[0].x, rn2 = d[2].x;
      const double rel = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
      sc[SC_NORMS] = make_double2(bn2, rn2);
      sc[SC_RHO] = make_double2(rn2, 0.0);
      sc[SC_ALPHA] = make_double2(1.0, 0.0);
      sc[SC_OMEGA] = make_double2(1.0, 0.0);
      sc[SC_BETA] = make_double2(0.0, 0.0);
      sc[SC_REL] = make_double2(rel, rel);
      iters[t] = 0;
      txflag[t] = TX_OK;
      act = (rel > tol && isfinite(rel)) ? 1 : 0;
    } else if (mode == SCM_ALPHA) {
      if (act) {
        const double2 den = d[0];
        const double m = den.x * den.x + den.y * den.y;
        if (!(m > 0.0) || !isfinite(m)) {
          txflag[t] = TX_BREAKDOWN;
          act = 0;
        } else {
          sc[SC_ALPHA] = z_div(sc[SC_RHO], den);
        }
      }
    } else if (mode == SCM_OMEGA) {
      if (act) {
        const double tt = d[2].x;
        sc[SC_OMEGA] = tt > 0.0 ? make_double2(d[1].x / tt, d[1].y / tt) : make_double2(0.0, 0.0);
      }
    } else if (mode == SCM_RHO) {
      if (act) {
        const double2 rho_new = d[0];
        const double rn2 = d[2].x;
        const double bn2 = sc[SC_NORMS].x;
        const int it = iters[t] + 1;
        iters[t] = it;
        const double rel = sqrt(rn2 / bn2);
        sc[SC_NORMS].y = rn2;
        sc[SC_REL].x = rel;
        const double2 om = sc[SC_OMEGA];
        const double rm = rho_new.x * rho_new.x + rho_new.y * rho_new.y;
        const double omm = om.x * om.x + om.y * om.y;
        if (rel <= tol) {
          act = 0;
        } else if (!isfinite(rel)) {
          txflag[t] = TX_BREAKDOWN;
          act = 0;
        } else if (it >= max_iter) {
          txflag[t] = TX_MAXITER;
          act = 0;
        } else if (!(rm > 0.0) || !(omm > 0.0)) {
          txflag[t] = TX_BREAKDOWN;
          act = 0;
        } else {
          sc[SC_BETA] = z_mul(z_div(rho_new, sc[SC_RHO]), z_div(sc[SC_ALPHA], om));
          sc[SC_RHO] = rho_new;
        }
      }
    } else {  // SCM_TRUE: r = b - A x and rhat = r were just recomputed
      const double rn2 = d[2].x;
      const double bn2 = sc[SC_NORMS].x;
      const double rel = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
      sc[SC_REL].y = rel;
      act = 0;
      if (rel > tol && isfinite(rel) && iters[t] < max_iter && txflag[t] != TX_MAXITER) {
        // restart from the current iterate with a fresh shadow residual
        sc[SC_NORMS].y = rn2;
        sc[SC_RHO] = make_double2(rn2, 0.0);
        sc[SC_ALPHA] = make_double2(1.0, 0.0);
        sc[SC_OMEGA] = make_double2(1.0, 0.0);
        sc[SC_BETA] = make_double2(0.0, 0.0);
        txflag[t] = TX_OK;
        act = 1;
      }
    }
    active[t] = act;
  }
  const int total = __syncthreads_count(act);
  if (threadIdx.x == 0) *n_active = total;
}

// x += alpha p + omega s ; r = s - omega t ; partials <rhat, r> (slot 0), <r, r> (slot 2)
__global__ void __launch_bounds__(256) bicg_update_kernel(int n, int RB, int nblk, const int* __restrict__ active,
                                                          const double* __restrict__ scal, float2* __restrict__ x,
                                                          const float2* __restrict__ p, const float2* __restrict__ s,
                                                          const float2* __restrict__ tv, float2* __restrict__ r,
                                                          const float2* __restrict__ rhat, double* __restrict__ part) {
  const int t = blockIdx.y;
  if (!active[t]) return;
  const double2* sc = reinterpret_cast<const double2*>(scal) + (size_t)t * SC_STRIDE;
  const float2 alpha = z_to_c(sc[SC_ALPHA]), omega = z_to_c(sc[SC_OMEGA]);
  const long long N = (long long)n * n;
  const int row0 = blockIdx.x * RB;
  const int rows = min(RB, n - row0);
  const long long base = t * N + (long long)row0 * n;
  float2 a0 = make_float2(0.f, 0.f), a2 = a0;
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const long long i = base + e;
    const float2 pv = p[i], sv = s[i], tv_ = tv[i];
    float2 xv = x[i];
    xv = c_add(xv, c_add(c_mul(alpha, pv), c_mul(omega, sv)));
    x[i] = xv;
    const float2 rv = c_sub(sv, c_mul(omega, tv_));
    r[i] = rv;
    a0 = c_add(a0, c_cjmul(rhat[i], rv));
    a2.x += rv.x * rv.x + rv.y * rv.y;
  }
  // block reduction in FP64
  __shared__ double red[8][4];
  double v[4] = {a0.x, a0.y, a2.x, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 3; ++k) red[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[w][0];
      s1 += red[w][1];
      s2 += red[w][2];
    }
    double2* out = reinterpret_cast<double2*>(part) + ((size_t)t * nblk + blockIdx.x) * DOT_SLOTS;
    out[0] = make_double2(s0, s1);
    out[1] = make_double2(0.0, 0.0);
    out[2] = make_double2(s2, 0.0);
  }
}

static cisor_status scalar_step(cisor_ctx* c, int mode, int ntx) {
  const int thr = ((ntx + 31) / 32) * 32;
  bicg_scalar_kernel<<<1, thr, 0, c->stream>>>(mode, ntx, c->nblk, c->part, c->scal, c->active, c->iters,
                                               c->txflag, c->n_active, c->sparams);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return CISOR_OK;
}

static ConvOp base_op(cisor_ctx* c, int adjoint, int ntx) {
  ConvOp op{};
  op.adjoint = adjoint;
  op.mul_f = 1;
  op.f = c->f;
  op.scal = c->scal;
  op.part = c->part;
  op.ntx = ntx;
  return op;
}

// r = b - A x ; rhat = r ; partials <b,b> (slot 0) and <r,r> (slot 2)
static cisor_status residual_pass(cisor_ctx* c, int adjoint, const float2* b, const float2* x, int ntx) {
  ConvOp op = base_op(c, adjoint, ntx);
  op.prologue = PRO_COPY;
  op.src = x;
  op.epilogue = EPI_RESID;
  op.esrc = x;
  op.aux = b;
  op.out = c->r;
  op.out2 = c->rhat;
  op.dot_a[0] = OP_AUX;
  op.dot_b[0] = OP_AUX;
  op.dot_a[2] = OP_Y;
  op.dot_b[2] = OP_Y;
  return conv_pass(c, op);
}

static cisor_status enqueue_iteration(cisor_ctx* c, int adjoint, float2* x, int ntx) {
  // p = r + beta (p - omega v) ; v = A p ; <rhat, v>
  ConvOp op = base_op(c, adjoint, ntx);
  op.active = c->active;
  op.prologue = PRO_PUPDATE;
  op.src = c->r;
  op.pvec = c->p;
  op.vvec = c->v;
  op.epilogue = EPI_MATVEC;
  op.esrc = c->p;
  op.out = c->v;
  op.aux = c->rhat;
  op.dot_a[0] = OP_AUX;
  op.dot_b[0] = OP_Y;
  CISOR_TRY(conv_pass(c, op));
  CISOR_TRY(scalar_step(c, SCM_ALPHA, ntx));
  // s = r - alpha v ; t = A s ; <t, s>, <t, t>
  ConvOp op2 = base_op(c, adjoint, ntx);
  op2.active = c->active;
  op2.prologue = PRO_AXPY;
  op2.src = c->r;
  op2.vvec = c->v;
  op2.svec = c->s;
  op2.epilogue = EPI_MATVEC;
  op2.esrc = c->s;
  op2.out = c->tv;
  op2.dot_a[1] = OP_Y;
  op2.dot_b[1] = OP_SRC;
  op2.dot_a[2] = OP_Y;
  op2.dot_b[2] = OP_Y;
  CISOR_TRY(conv_pass(c, op2));
  CISOR_TRY(scalar_step(c, SCM_OMEGA, ntx));
  const int RB = conv_rows_per_block(c->P);
  dim3 g(c->nblk, ntx);
  bicg_update_kernel<<<g, 256, 0, c->stream>>>(c->n, RB, c->nblk, c->active, c->scal, x, c->p, c->s, c->tv, c->r,
                                               c->rhat, c->part);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return scalar_step(c, SCM_RHO, ntx);
}

static cisor_status get_graph(cisor_ctx* c, int adjoint, float2* x, int ntx, cudaGraphExec_t* out) {
  if (c->graph[adjoint] && c->graph_ntx[adjoint] == ntx && c->graph_x[adjoint] == x) {
    *out = c->graph[adjoint];
    return CISOR_OK;
  }
  if (c->graph[adjoint]) {
    cudaGraphExecDestroy(c->graph[adjoint]);
    c->graph[adjoint] = nullptr;
  }
  cudaGraph_t g = nullptr;
  const long long l0 = c->launches;
  CISOR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cisor_status st = CISOR_OK;
  for (int i = 0; i < c->graph_chunk && st == CISOR_OK; ++i) st = enqueue_iteration(c, adjoint, x, ntx);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->graph_kernels[adjoint] = c->launches - l0;  // captured, not launched
  c->launches = l0;
  if (st != CISOR_OK) {
    if (e == cudaSuccess && g) cudaGraphDestroy(g);
    return st;
  }
  CISOR_CUDA(e);
  cudaError_t e2 = cudaGraphInstantiate(&c->graph[adjoint], g, 0);
  cudaGraphDestroy(g);
  CISOR_CUDA(e2);
  c->graph_ntx[adjoint] = ntx;
  c->graph_x[adjoint] = x;
  *out = c->graph[adjoint];
  return CISOR_OK;
}

static cisor_status read_active(cisor_ctx* c, int* n_active) {
  CISOR_CUDA(cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  *n_active = *c->h_n_active;
  return CISOR_OK;
}

cisor_status solve_batch(cisor_ctx* c, int adjoint, const float2* f, const float2* b, float2* x, int ntx, double tol,
                         int max_iter, int* iters_max, double* iters_mean, double* resid_max, int* n_bad) {
  (void)f;  // the operator always reads the context's copy of f (c->f), baked into the graphs
  const size_t vb = sizeof(float2) * (size_t)ntx * c->N;
  double hp[2] = {tol, (double)max_iter};
  CISOR_CUDA(cudaMemcpyAsync(c->sparams, hp, sizeof(hp), cudaMemcpyHostToDevice, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->p, 0, vb, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->v, 0, vb, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->active, 0, sizeof(int) * ntx, c->stream));
  CISOR_TRY(residual_pass(c, adjoint, b, x, ntx));
  CISOR_TRY(scalar_step(c, SCM_INIT, ntx));
  int nact = 0;
  CISOR_TRY(read_active(c, &nact));
  cudaGraphExec_t ge = nullptr;
  int done = 0;
  for (int restart = 0; restart < 6 && nact > 0; ++restart) {
    CISOR_TRY(get_graph(c, adjoint, x, ntx, &ge));
    while (nact > 0 && done < max_iter + c->graph_chunk) {
      CISOR_CUDA(cudaGraphLaunch(ge, c->stream));
      c->launches += c->graph_kernels[adjoint];
      done += c->graph_chunk;
      CISOR_TRY(read_active(c, &nact));
    }
    CISOR_TRY(residual_pass(c, adjoint, b, x, ntx));
    CISOR_TRY(scalar_step(c, SCM_TRUE, ntx));
    CISOR_TRY(read_active(c, &nact));
  }
  if (nact == 0) {
    // every transmitter ended: refresh the true residuals of those that never iterated
  }
  // statistics
  std::vector<int> it(ntx), fl(ntx);
  std::vector<double> sc((size_t)ntx * SC_STRIDE * 2);
  CISOR_CUDA(cudaMemcpyAsync(it.data(), c->iters, sizeof(int) * ntx, cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaMemcpyAsync(fl.data(), c->txflag, sizeof(int) * ntx, cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaMemcpyAsync(sc.data(), c->scal, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  int imax = 0, bad = 0;
  double isum = 0.0, rmax = 0.0;
  for (int t = 0; t < ntx; ++t) {
    imax = it[t] > imax ? it[t] : imax;
    isum += it[t];
    const double rel = sc[((size_t)t * SC_STRIDE + SC_REL) * 2 + 1];
    rmax = (rel > rmax || !(rel == rel)) ? rel : rmax;
    if (!(rel <= tol)) ++bad;
  }
  if (iters_max) *iters_max = imax;
  if (iters_mean) *iters_mean = isum / (ntx > 0 ? ntx : 1);
  if (resid_max) *resid_max = rmax;
  if (n_bad) *n_bad = bad;
  if (bad) {
    int brk = 0;
    for (int t = 0; t < ntx; ++t) brk |= (fl[t] == TX_BREAKDOWN);
    set_error("%d of %d field solves above tol %.3g (max true residual %.3g)%s", bad, ntx, tol, rmax,
              brk ? ", Krylov breakdown" : "");
    return brk ? CISOR_ERR_BREAKDOWN : CISOR_ERR_NOT_CONVERGED;
  }
  return CISOR_OK;
}

}  // namespace cisor
