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

// One 32-thread block per transmitter: the lanes sum the per-CTA partials of
// the three dot slots (FP32 tree), lane 0 advances that transmitter's
// recurrence in FP64.  (FP64 arithmetic runs at a small fraction of the FP32
// rate on this part, so FP64 is kept to these few scalar operations.)
__global__ void __launch_bounds__(32) bicg_scalar_kernel(int mode, int nblk, const float* __restrict__ part,
                                                         double* __restrict__ scal, int* __restrict__ active,
                                                         int* __restrict__ iters, int* __restrict__ txflag,
                                                         const double* __restrict__ params) {
  pdl_trigger();
  pdl_wait();
  const int t = blockIdx.x, lane = threadIdx.x;
  float d[2 * DOT_SLOTS];
#pragma unroll
  for (int k = 0; k < 2 * DOT_SLOTS; ++k) d[k] = 0.f;
  const float* pp = part + (size_t)t * nblk * DOT_SLOTS * 2;
  for (int b = lane; b < nblk; b += 32)
#pragma unroll
    for (int k = 0; k < 2 * DOT_SLOTS; ++k) d[k] += pp[b * DOT_SLOTS * 2 + k];
#pragma unroll
  for (int k = 0; k < 2 * DOT_SLOTS; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
  if (lane != 0) return;
  const double tol = params[0];
  const int max_iter = (int)params[1];
  const double2 d0 = make_double2(d[0], d[1]), d1 = make_double2(d[2], d[3]), d2 = make_double2(d[4], d[5]);
  double2* sc = reinterpret_cast<double2*>(scal) + (size_t)t * SC_STRIDE;
  int act = active[t];
  if (mode == SCM_INIT) {
    const double bn2 = d0.x, rn2 = d2.x;
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
      const double m = d0.x * d0.x + d0.y * d0.y;
      if (!(m > 0.0) || !isfinite(m)) {
        txflag[t] = TX_BREAKDOWN;
        act = 0;
      } else {
        sc[SC_ALPHA] = z_div(sc[SC_RHO], d0);
      }
    }
  } else if (mode == SCM_OMEGA) {
    if (act) {
      const double tt = d2.x;
      sc[SC_OMEGA] = tt > 0.0 ? make_double2(d1.x / tt, d1.y / tt) : make_double2(0.0, 0.0);
    }
  } else if (mode == SCM_RHO) {
    if (act) {
      const double rn2 = d2.x;
      const double bn2 = sc[SC_NORMS].x;
      const int it = iters[t] + 1;
      iters[t] = it;
      const double rel = sqrt(rn2 / bn2);
      sc[SC_NORMS].y = rn2;
      sc[SC_REL].x = rel;
      const double2 om = sc[SC_OMEGA];
      const double rm = d0.x * d0.x + d0.y * d0.y;
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
        sc[SC_BETA] = z_mul(z_div(d0, sc[SC_RHO]), z_div(sc[SC_ALPHA], om));
        sc[SC_RHO] = d0;
      }
    }
  } else {  // SCM_TRUE: r = b - A x and rhat = r were just recomputed
    const double rn2 = d2.x;
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

// x += alpha p + omega s ; r = s - omega t ; partials <rhat, r> (slot 0), <r, r> (slot 2).
// Each CTA covers the RB rows of one transmitter that a row-pass CTA covers,
// so its partial lands in the same slot layout; two complex values per
// 16-byte access when the row length is even.
__global__ void __launch_bounds__(256) bicg_update_kernel(int n, int nrows, int RB, int nblk,
                                                          const int* __restrict__ active,
                                                          const double* __restrict__ scal, float2* __restrict__ x,
                                                          const float2* __restrict__ p, const float2* __restrict__ s,
                                                          const float2* __restrict__ tv, float2* __restrict__ r,
                                                          const float2* __restrict__ rhat, float* __restrict__ part) {
  pdl_trigger();
  pdl_wait();
  const int t = blockIdx.y;
  if (!active[t]) return;
  const double2* sc = reinterpret_cast<const double2*>(scal) + (size_t)t * SC_STRIDE;
  const float2 alpha = z_to_c(sc[SC_ALPHA]), omega = z_to_c(sc[SC_OMEGA]);
  const long long N = (long long)nrows * n;
  const int row0 = blockIdx.x * RB;
  const int rows = min(RB, nrows - row0);
  const long long base = t * N + (long long)row0 * n;
  const int cnt = rows * n;
  float2 a0 = make_float2(0.f, 0.f);
  float a2 = 0.f;
  auto one = [&](long long i, float2 pv, float2 sv, float2 tv_, float2 xv, float2 rh, float2& xo, float2& ro) {
    xo = c_add(xv, c_add(c_mul(alpha, pv), c_mul(omega, sv)));
    ro = c_sub(sv, c_mul(omega, tv_));
    a0 = c_add(a0, c_cjmul(rh, ro));
    a2 += ro.x * ro.x + ro.y * ro.y;
  };
  if ((n & 1) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p + base);
    const float4* s4 = reinterpret_cast<const float4*>(s + base);
    const float4* t4 = reinterpret_cast<const float4*>(tv + base);
    const float4* h4 = reinterpret_cast<const float4*>(rhat + base);
    float4* x4 = reinterpret_cast<float4*>(x + base);
    float4* r4 = reinterpret_cast<float4*>(r + base);
    for (int e = threadIdx.x; e < cnt / 2; e += blockDim.x) {
      const float4 pv = p4[e], sv = s4[e], tq = t4[e], hv = h4[e], xv = x4[e];
      float2 xo0, ro0, xo1, ro1;
      one(0, make_float2(pv.x, pv.y), make_float2(sv.x, sv.y), make_float2(tq.x, tq.y), make_float2(xv.x, xv.y),
          make_float2(hv.x, hv.y), xo0, ro0);
      one(0, make_float2(pv.z, pv.w), make_float2(sv.z, sv.w), make_float2(tq.z, tq.w), make_float2(xv.z, xv.w),
          make_float2(hv.z, hv.w), xo1, ro1);
      x4[e] = make_float4(xo0.x, xo0.y, xo1.x, xo1.y);
      r4[e] = make_float4(ro0.x, ro0.y, ro1.x, ro1.y);
    }
  } else {
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const long long i = base + e;
      float2 xo, ro;
      one(i, p[i], s[i], tv[i], x[i], rhat[i], xo, ro);
      x[i] = xo;
      r[i] = ro;
    }
  }
  // block reduction, FP32 tree
  __shared__ float red[3][8];
  float v[3] = {a0.x, a0.y, a2};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 3; ++k) red[k][wid] = v[k];
  __syncthreads();
  if (threadIdx.x < 3) {
    float* rr = red[threadIdx.x];
    for (int w = 4; w > 0; w >>= 1)
      for (int i = 0; i < w; ++i) rr[i] += rr[i + w];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2* out = reinterpret_cast<float2*>(part) + ((size_t)t * nblk + blockIdx.x) * DOT_SLOTS;
    out[0] = make_float2(red[0][0], red[1][0]);
    out[1] = make_float2(0.f, 0.f);
    out[2] = make_float2(red[2][0], 0.f);
  }
}

static cisor_status scalar_step(cisor_ctx* c, int mode, int ntx) {
  (void)launch_pdl(bicg_scalar_kernel, dim3(ntx), dim3(32), 0, c->stream, mode, c->nblk * c->ncomp,
                   (const float*)c->part, c->scal, c->active, c->iters, c->txflag, (const double*)c->sparams);
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
  if (c->ncomp == 3) {
    VecOp vo{};
    vo.adjoint = adjoint;
    vo.epilogue = EPI_RESID;
    vo.x = x;
    vo.aux = b;
    vo.out = c->r;
    vo.out2 = c->rhat;
    vo.dot_a[0] = OP_AUX;
    vo.dot_b[0] = OP_AUX;
    vo.dot_a[2] = OP_Y;
    vo.dot_b[2] = OP_Y;
    vo.ntx = ntx;
    return vec_matvec(c, vo);
  }
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

// x += alpha p + omega s ; r = s - omega t ; <rhat, r>, <r, r>, then rho', beta, convergence
static cisor_status update_step(cisor_ctx* c, float2* x, int ntx) {
  const int RB = conv_rows_per_block(c->P);
  dim3 g(c->nblk * c->ncomp, ntx);
  (void)launch_pdl(bicg_update_kernel, g, dim3(256), 0, c->stream, c->n, c->nrows * c->ncomp, RB, c->nblk * c->ncomp,
                   (const int*)c->active, (const double*)c->scal, x, (const float2*)c->p, (const float2*)c->s,
                   (const float2*)c->tv, c->r, (const float2*)c->rhat, c->part);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  return scalar_step(c, SCM_RHO, ntx);
}

// The vectorial model: the same recurrence with the vector updates in their
// own kernels around the stencil-plus-convolution matvec.
static cisor_status enqueue_iteration_vec(cisor_ctx* c, int adjoint, float2* x, int ntx) {
  CISOR_TRY(vec_pupdate(c, ntx));
  VecOp op{};
  op.adjoint = adjoint;
  op.epilogue = EPI_MATVEC;
  op.x = c->p;
  op.aux = c->rhat;
  op.out = c->v;
  op.dot_a[0] = OP_AUX;
  op.dot_b[0] = OP_Y;
  op.active = c->active;
  op.ntx = ntx;
  CISOR_TRY(vec_matvec(c, op));
  CISOR_TRY(scalar_step(c, SCM_ALPHA, ntx));
  CISOR_TRY(vec_axpy(c, ntx));
  VecOp op2{};
  op2.adjoint = adjoint;
  op2.epilogue = EPI_MATVEC;
  op2.x = c->s;
  op2.out = c->tv;
  op2.dot_a[1] = OP_Y;
  op2.dot_b[1] = OP_SRC;
  op2.dot_a[2] = OP_Y;
  op2.dot_b[2] = OP_Y;
  op2.active = c->active;
  op2.ntx = ntx;
  CISOR_TRY(vec_matvec(c, op2));
  CISOR_TRY(scalar_step(c, SCM_OMEGA, ntx));
  return update_step(c, x, ntx);
}

static cisor_status enqueue_iteration(cisor_ctx* c, int adjoint, float2* x, int ntx) {
  if (c->ncomp == 3) return enqueue_iteration_vec(c, adjoint, x, ntx);
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
  return update_step(c, x, ntx);
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

// ---------------------------------------------------------------- whole-solve graphs
// A solve's iterations run as ONE graph launch: a WHILE conditional node
// whose body is a chunk of BiCGSTAB iterations (of every problem, forked to
// their streams) followed by loop_cond_kernel, which keeps the loop going
// while any transmitter of any problem is active and the body has run fewer
// than ceil(max_iter / chunk) + 2 times (so the loop always ends, whatever
// the flags).  The host only waits for the graph, not for every chunk.
__global__ void loop_cond_kernel(const cisor_loop_item* __restrict__ items, int nitems,
                                 const double* __restrict__ params, int chunk, int* __restrict__ count,
                                 cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int a = 0;
  for (int p = 0; p < nitems; ++p)
    for (int t = threadIdx.x; t < items[p].ntx; t += blockDim.x) a |= items[p].active[t];
  if (a) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int cap = (int)(params[1] / chunk) + 2;
    const int k = *count + 1;
    *count = k;
    cudaGraphSetConditional(h, (any && k < cap) ? 1u : 0u);
  }
}

// Builds a graph [WHILE { body ; loop_cond_kernel }]: `body` enqueues the
// iterations on `st` (forking to other streams and joining back is allowed).
template <class Body>
static cudaError_t build_while_graph(cudaStream_t st, Body body, const cisor_loop_item* items, int nitems,
                                     const double* params, int chunk, int* count, cudaGraphExec_t* out,
                                     cisor_status* body_status) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    *body_status = body();
    loop_cond_kernel<<<1, 256, 0, st>>>(items, nitems, params, chunk, count, h);
    cudaError_t el = cudaGetLastError();
    cudaGraph_t cap = nullptr;
    e = cudaStreamEndCapture(st, &cap);
    if (e == cudaSuccess) e = el;
  }
  if (e == cudaSuccess && *body_status == CISOR_OK) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// The whole-solve graph of one context (built on first use, rebuilt when x or
// the transmitter count changes); false when the WHILE graph cannot be built
// here (the caller then runs the host-driven chunk loop).
static cisor_status get_while_graph(cisor_ctx* c, int adjoint, float2* x, int ntx, cudaGraphExec_t* out, bool* ok) {
  *ok = false;
  if (!c->use_while) return CISOR_OK;
  if (c->wgraph[adjoint] && c->wgraph_ntx[adjoint] == ntx && c->wgraph_x[adjoint] == x) {
    *out = c->wgraph[adjoint];
    *ok = true;
    return CISOR_OK;
  }
  if (c->wgraph[adjoint]) {
    cudaGraphExecDestroy(c->wgraph[adjoint]);
    c->wgraph[adjoint] = nullptr;
  }
  if (!c->loop_item) {
    CISOR_CUDA(cudaMalloc((void**)&c->loop_item, sizeof(cisor_loop_item)));
    CISOR_CUDA(cudaMalloc((void**)&c->loop_count, sizeof(int)));
    CISOR_CUDA(cudaMallocHost((void**)&c->h_loop_count, sizeof(int)));
  }
  const cisor_loop_item it{c->active, ntx};
  CISOR_CUDA(cudaMemcpyAsync(c->loop_item, &it, sizeof(it), cudaMemcpyHostToDevice, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  const long long l0 = c->launches;
  cisor_status bs = CISOR_OK;
  auto body = [&]() {
    cisor_status s2 = CISOR_OK;
    for (int i = 0; i < c->graph_chunk && s2 == CISOR_OK; ++i) s2 = enqueue_iteration(c, adjoint, x, ntx);
    return s2;
  };
  cudaError_t e = build_while_graph(c->stream, body, c->loop_item, 1, c->sparams, c->graph_chunk, c->loop_count,
                                    &c->wgraph[adjoint], &bs);
  c->graph_kernels[adjoint] = c->launches - l0 + 1;  // captured per body execution (+ the condition)
  c->launches = l0;
  if (bs != CISOR_OK) return bs;
  if (e != cudaSuccess) {  // conditional graphs unavailable: keep the host-driven loop
    cudaGetLastError();
    c->wgraph[adjoint] = nullptr;
    c->use_while = 0;
    return CISOR_OK;
  }
  c->wgraph_ntx[adjoint] = ntx;
  c->wgraph_x[adjoint] = x;
  *out = c->wgraph[adjoint];
  *ok = true;
  return CISOR_OK;
}

static cisor_status read_active(cisor_ctx* c, int ntx, int* n_active) {
  CISOR_CUDA(cudaMemcpyAsync(c->h_active, c->active, sizeof(int) * ntx, cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  int s = 0;
  for (int t = 0; t < ntx; ++t) s += c->h_active[t];
  *n_active = s;
  return CISOR_OK;
}

// Sets the solve parameters, zeroes p and v, forms r = b - A x0, rhat = r and
// runs the INIT scalar step (all on c->stream).
static cisor_status init_solve(cisor_ctx* c, int adjoint, const float2* b, float2* x, int ntx, double tol,
                               int max_iter) {
  const size_t vb = sizeof(float2) * (size_t)ntx * c->Nf;
  // pageable source: the copy is staged before cudaMemcpyAsync returns, so the stack array may go
  const double hp[2] = {tol, (double)max_iter};
  CISOR_CUDA(cudaMemcpyAsync(c->sparams, hp, sizeof(hp), cudaMemcpyHostToDevice, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->p, 0, vb, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->v, 0, vb, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->active, 0, sizeof(int) * ntx, c->stream));
  CISOR_TRY(residual_pass(c, adjoint, b, x, ntx));
  return scalar_step(c, SCM_INIT, ntx);
}

// True residual r = b - A x and the restart decision (SCM_TRUE).
static cisor_status true_residual(cisor_ctx* c, int adjoint, const float2* b, float2* x, int ntx) {
  CISOR_TRY(residual_pass(c, adjoint, b, x, ntx));
  return scalar_step(c, SCM_TRUE, ntx);
}

// Per-transmitter statistics of the last solve; the status reports any
// transmitter above tol (breakdown or iteration cap).
static cisor_status collect_stats(cisor_ctx* c, int adjoint, int ntx, double tol, int* iters_max,
                                  double* iters_mean, double* resid_max, int* n_bad) {
  std::vector<int> it(ntx), fl(ntx);
  std::vector<double> sc((size_t)ntx * SC_STRIDE * 2);
  CISOR_CUDA(cudaMemcpyAsync(it.data(), c->iters, sizeof(int) * ntx, cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaMemcpyAsync(fl.data(), c->txflag, sizeof(int) * ntx, cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaMemcpyAsync(sc.data(), c->scal, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  c->last_iters[adjoint ? 1 : 0] = it;
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

cisor_status solve_batch(cisor_ctx* c, int adjoint, const float2* f, const float2* b, float2* x, int ntx, double tol,
                         int max_iter, int* iters_max, double* iters_mean, double* resid_max, int* n_bad) {
  (void)f;  // the operator always reads the context's copy of f (c->f), baked into the graphs
  CISOR_TRY(init_solve(c, adjoint, b, x, ntx, tol, max_iter));
  int nact = 0;
  CISOR_TRY(read_active(c, ntx, &nact));
  cudaGraphExec_t ge = nullptr;
  int done = 0;
  for (int restart = 0; restart < 6 && nact > 0; ++restart) {
    bool whole = false;
    CISOR_TRY(get_while_graph(c, adjoint, x, ntx, &ge, &whole));
    if (whole) {  // all chunks in one launch; the device decides when to stop
      CISOR_CUDA(cudaMemsetAsync(c->loop_count, 0, sizeof(int), c->stream));
      CISOR_CUDA(cudaGraphLaunch(ge, c->stream));
      CISOR_CUDA(cudaMemcpyAsync(c->h_loop_count, c->loop_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CISOR_CUDA(cudaStreamSynchronize(c->stream));
      c->launches += c->graph_kernels[adjoint] * (long long)c->h_loop_count[0];
    } else {
      CISOR_TRY(get_graph(c, adjoint, x, ntx, &ge));
      while (nact > 0 && done < max_iter + c->graph_chunk) {
        CISOR_CUDA(cudaGraphLaunch(ge, c->stream));
        c->launches += c->graph_kernels[adjoint];
        done += c->graph_chunk;
        CISOR_TRY(read_active(c, ntx, &nact));
      }
    }
    CISOR_TRY(true_residual(c, adjoint, b, x, ntx));
    CISOR_TRY(read_active(c, ntx, &nact));
  }
  return collect_stats(c, adjoint, ntx, tol, iters_max, iters_mean, resid_max, n_bad);
}

// ---------------------------------------------------------------- several problems in one graph
// The problems' BiCGSTAB iterations are captured into ONE graph per chunk:
// fork from ms.main to every context's stream, each context's chunk of
// iterations on its own stream, join back.  One cudaGraphLaunch advances all
// problems; converged transmitters and finished problems exit their CTAs at once.
cisor_status solve_multi(cisor_ctx* const* cs, int np, int adjoint, const float2* const* b, double tol, int max_iter,
                         MultiSolve& ms, SolveStat* st) {
  auto xof = [&](cisor_ctx* c) { return adjoint ? c->vadj : c->u; };
  for (int i = 0; i < np; ++i) CISOR_TRY(init_solve(cs[i], adjoint, b[i], xof(cs[i]), cs[i]->T, tol, max_iter));
  auto count = [&](int* total) -> cisor_status {
    for (int i = 0; i < np; ++i)
      CISOR_CUDA(cudaMemcpyAsync(cs[i]->h_active, cs[i]->active, sizeof(int) * cs[i]->T, cudaMemcpyDeviceToHost,
                                 cs[i]->stream));
    int s = 0;
    for (int i = 0; i < np; ++i) {
      CISOR_CUDA(cudaStreamSynchronize(cs[i]->stream));
      for (int t = 0; t < cs[i]->T; ++t) s += cs[i]->h_active[t];
    }
    *total = s;
    return CISOR_OK;
  };
  int nact = 0;
  CISOR_TRY(count(&nact));
  // the forked chunk of iterations of every problem (captured into either kind of graph)
  auto fork_body = [&]() -> cisor_status {
    cisor_status s = CISOR_OK;
    cudaError_t e = cudaEventRecord(ms.fork, ms.main);
    for (int i = 0; i < np && s == CISOR_OK && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(cs[i]->stream, ms.fork, 0);
      for (int k = 0; k < cs[i]->graph_chunk && s == CISOR_OK && e == cudaSuccess; ++k)
        s = enqueue_iteration(cs[i], adjoint, xof(cs[i]), cs[i]->T);
      if (e == cudaSuccess) e = cudaEventRecord(ms.join[i], cs[i]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ms.main, ms.join[i], 0);
    }
    if (s == CISOR_OK && e != cudaSuccess) return cuda_fail(e, "batch graph fork", __FILE__, __LINE__);
    return s;
  };
  if (nact > 0 && ms.use_while && !ms.wgraph[adjoint]) {
    std::vector<cisor_loop_item> items(np);
    for (int i = 0; i < np; ++i) items[i] = cisor_loop_item{cs[i]->active, cs[i]->T};
    CISOR_CUDA(cudaMemcpyAsync(ms.items, items.data(), sizeof(cisor_loop_item) * np, cudaMemcpyHostToDevice, ms.main));
    CISOR_CUDA(cudaStreamSynchronize(ms.main));
    std::vector<long long> l0(np);
    for (int i = 0; i < np; ++i) l0[i] = cs[i]->launches;
    cisor_status bs = CISOR_OK;
    cudaError_t e = build_while_graph(ms.main, fork_body, ms.items, np, cs[0]->sparams, cs[0]->graph_chunk,
                                      ms.loop_count, &ms.wgraph[adjoint], &bs);
    for (int i = 0; i < np; ++i) {
      ms.kernels[adjoint][i] = cs[i]->launches - l0[i];
      cs[i]->launches = l0[i];
    }
    if (bs != CISOR_OK) return bs;
    if (e != cudaSuccess) {
      cudaGetLastError();
      ms.wgraph[adjoint] = nullptr;
      ms.use_while = 0;
    }
  }
  if (nact > 0 && ms.use_while && ms.wgraph[adjoint]) {
    for (int restart = 0; restart < 6 && nact > 0; ++restart) {
      CISOR_CUDA(cudaMemsetAsync(ms.loop_count, 0, sizeof(int), ms.main));
      CISOR_CUDA(cudaGraphLaunch(ms.wgraph[adjoint], ms.main));
      CISOR_CUDA(cudaMemcpyAsync(ms.h_loop_count, ms.loop_count, sizeof(int), cudaMemcpyDeviceToHost, ms.main));
      CISOR_CUDA(cudaStreamSynchronize(ms.main));
      for (int i = 0; i < np; ++i) cs[i]->launches += ms.kernels[adjoint][i] * (long long)ms.h_loop_count[0];
      for (int i = 0; i < np; ++i) CISOR_TRY(true_residual(cs[i], adjoint, b[i], xof(cs[i]), cs[i]->T));
      CISOR_TRY(count(&nact));
    }
    nact = 0;  // the stats below report any transmitter still above tol
  }
  if (nact > 0 && !ms.graph[adjoint]) {
    std::vector<long long> l0(np);
    for (int i = 0; i < np; ++i) l0[i] = cs[i]->launches;
    cudaGraph_t g = nullptr;
    CISOR_CUDA(cudaStreamBeginCapture(ms.main, cudaStreamCaptureModeThreadLocal));
    cisor_status s = fork_body();
    cudaError_t e = cudaSuccess;
    cudaError_t e2 = cudaStreamEndCapture(ms.main, &g);
    for (int i = 0; i < np; ++i) {
      ms.kernels[adjoint][i] = cs[i]->launches - l0[i];
      cs[i]->launches = l0[i];
    }
    if (s != CISOR_OK) {
      if (e2 == cudaSuccess && g) cudaGraphDestroy(g);
      return s;
    }
    CISOR_CUDA(e);
    CISOR_CUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&ms.graph[adjoint], g, 0);
    cudaGraphDestroy(g);
    CISOR_CUDA(e3);
  }
  int done = 0;
  const int chunk = cs[0]->graph_chunk;
  for (int restart = 0; restart < 6 && nact > 0; ++restart) {
    while (nact > 0 && done < max_iter + chunk) {
      CISOR_CUDA(cudaGraphLaunch(ms.graph[adjoint], ms.main));
      for (int i = 0; i < np; ++i) cs[i]->launches += ms.kernels[adjoint][i];
      done += chunk;
      CISOR_CUDA(cudaStreamSynchronize(ms.main));
      CISOR_TRY(count(&nact));
    }
    for (int i = 0; i < np; ++i) CISOR_TRY(true_residual(cs[i], adjoint, b[i], xof(cs[i]), cs[i]->T));
    CISOR_TRY(count(&nact));
  }
  cisor_status worst = CISOR_OK;
  for (int i = 0; i < np; ++i) {
    st[i].status = collect_stats(cs[i], adjoint, cs[i]->T, tol, &st[i].iters_max, &st[i].iters_mean, &st[i].resid_max,
                                 &st[i].n_bad);
    if (st[i].status == CISOR_ERR_CUDA || st[i].status == CISOR_ERR_OOM) return st[i].status;
    if (st[i].status != CISOR_OK) worst = st[i].status;
  }
  return worst;
}

}  // namespace cisor
