// C ABI entry points (include/cisor.h).  Arguments are copied into the
// context's device buffers with cudaMemcpyDefault (unified addressing: host
// or device pointers), work runs on the context's own non-blocking stream,
// ordered after and before the caller's stream with events, and results are
// copied out; a call that writes host memory synchronises before returning.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "common.cuh"

namespace cisor {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

cisor_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? CISOR_ERR_OOM : CISOR_ERR_CUDA;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void scale_copy_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long n, float s) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2(in[i].x * s, in[i].y * s);
}

// Orders the call after the caller's stream on entry and the caller's stream
// after the call on exit; synchronises if host memory was written.
struct Call {
  cisor_ctx* c;
  bool host_out = false;
  explicit Call(cisor_ctx* ctx) : c(ctx) {}
  cisor_status enter() {
    CISOR_CUDA(cudaEventRecord(c->ev_a, c->user_stream));
    CISOR_CUDA(cudaStreamWaitEvent(c->stream, c->ev_a, 0));
    return CISOR_OK;
  }
  cisor_status in(void* dst, const void* src, size_t bytes) {
    CISOR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return CISOR_OK;
  }
  cisor_status out(void* dst, const void* src, size_t bytes) {
    if (!dst) return CISOR_OK;
    if (!is_device_ptr(dst)) host_out = true;
    CISOR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return CISOR_OK;
  }
  cisor_status leave() {
    CISOR_CUDA(cudaEventRecord(c->ev_b, c->stream));
    CISOR_CUDA(cudaStreamWaitEvent(c->user_stream, c->ev_b, 0));
    if (host_out) CISOR_CUDA(cudaStreamSynchronize(c->stream));
    return sense_tc_check(c, host_out);
  }
};

static bool check_opts(const cisor_solve_opts* o) {
  if (!o) {
    set_error("solve options are NULL");
    return false;
  }
  if (!(o->tol > 0.0) || o->max_iter < 1 || o->x0_mode < 0 || o->x0_mode > 2) {
    set_error("invalid solve options (tol %g, max_iter %d, x0_mode %d)", o->tol, o->max_iter, o->x0_mode);
    return false;
  }
  return true;
}

static cisor_status worse(cisor_status a, cisor_status b) {
  if (a == CISOR_ERR_CUDA || b == CISOR_ERR_CUDA || a == CISOR_ERR_OOM || b == CISOR_ERR_OOM)
    return (a == CISOR_ERR_CUDA || a == CISOR_ERR_OOM) ? a : b;
  if (a == CISOR_ERR_BREAKDOWN || b == CISOR_ERR_BREAKDOWN) return CISOR_ERR_BREAKDOWN;
  if (a == CISOR_ERR_NOT_CONVERGED || b == CISOR_ERR_NOT_CONVERGED) return CISOR_ERR_NOT_CONVERGED;
  return a != CISOR_OK ? a : b;
}

static bool solve_ok(cisor_status s) {
  return s == CISOR_OK || s == CISOR_ERR_NOT_CONVERGED || s == CISOR_ERR_BREAKDOWN;
}

// Forward half of the gradient machinery on c->f (the point) and c->yobs
// (the data): forward solve into c->u (kept: the fields are the checkpoint the
// backward half needs), Z, w = Z - y and D.
static cisor_status data_core(cisor_ctx* c, const cisor_solve_opts* o, double* D, cisor_solve_info* li) {
  const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
  if (o->x0_mode != 2 || !c->have_u) CISOR_CUDA(cudaMemcpyAsync(c->u, c->u_in, vb, cudaMemcpyDeviceToDevice, c->stream));
  int nb1 = 0;
  c->have_w = 0;
  cisor_status s1 = solve_batch(c, 0, c->f, c->u_in, c->u, c->T, o->tol, o->max_iter, &li->iters_max, &li->iters_mean,
                                &li->resid_max, &nb1);
  if (!solve_ok(s1)) return s1;
  c->have_u = 1;
  li->n_not_converged = nb1;
  CISOR_TRY(residual_and_D(c, c->f, c->u, c->yobs, c->Y, c->w, c->T));
  CISOR_CUDA(cudaMemcpyAsync(c->h_dsum, c->dsum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CISOR_CUDA(cudaStreamSynchronize(c->stream));
  if (D) *D = c->h_dsum[0];
  return s1;
}

// Backward half: adjoint RHS, adjoint solve into c->vadj, gz = z + G^H v,
// g = sum_t conj(u_t) gz_t into c->grad and, when zstep is given,
// zstep = s - gamma g.  Needs data_core's u and w.
static cisor_status adjoint_core(cisor_ctx* c, const cisor_solve_opts* o, double gamma, const float2* s,
                                 float2* zstep, cisor_solve_info* li) {
  const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
  CISOR_TRY(sense_adjoint(c, c->f, c->w, c->z, c->b, c->T));
  if (o->x0_mode != 2 || !c->have_v) CISOR_CUDA(cudaMemsetAsync(c->vadj, 0, vb, c->stream));
  int nb2 = 0;
  cisor_status s2 = solve_batch(c, 1, c->f, c->b, c->vadj, c->T, o->tol, o->max_iter, &li->adj_iters_max,
                                &li->adj_iters_mean, &li->adj_resid_max, &nb2);
  if (!solve_ok(s2)) return s2;
  c->have_v = 1;
  li->n_not_converged += nb2;
  if (c->ncomp == 3) {
    CISOR_TRY(vec_gz(c));  // z + conv_{G^H}(v + D v / k^2)
  } else {
    ConvOp op{};
    op.adjoint = 1;
    op.mul_f = 0;
    op.prologue = PRO_COPY;
    op.src = c->vadj;
    op.epilogue = EPI_CONV_ADD;
    op.aux = c->z;
    op.out = c->gz;
    op.f = c->f;
    op.ntx = c->T;
    CISOR_TRY(conv_pass(c, op));
  }
  CISOR_TRY(grad_assemble(c, c->u, c->gz, s, gamma, c->grad, zstep, c->T));
  return s2;
}

// Prop. 1's backward half needs the u, w and f of the forward half.  f is
// checkpointed by cisor_data_term in c->f_ck; u and w live in buffers that
// cisor_forward, cisor_sense_adjoint, cisor_grad, cisor_step and the batch
// solves overwrite, so those entry points drop the held state and a later
// cisor_data_backward is refused instead of differentiating at another point.
static void drop_data_term(cisor_ctx* c) { c->have_w = 0; }

static cisor_status grad_core(cisor_ctx* c, const cisor_solve_opts* o, double gamma, const float2* s, float2* zstep,
                              double* D, cisor_solve_info* info) {
  cisor_solve_info li{};
  cisor_status s1 = data_core(c, o, D, &li);
  if (!solve_ok(s1)) return s1;
  cisor_status s2 = adjoint_core(c, o, gamma, s, zstep, &li);
  if (!solve_ok(s2)) return s2;
  if (info) *info = li;
  return worse(s1, s2);
}

// Captured graphs hold the kernel variants and launch sequence they were built with.
static cisor_status drop_graphs(cisor_ctx* c) {
  for (int i = 0; i < 2; ++i) {
    if (c->graph[i]) CISOR_CUDA(cudaGraphExecDestroy(c->graph[i]));
    if (c->wgraph[i]) CISOR_CUDA(cudaGraphExecDestroy(c->wgraph[i]));
    c->graph[i] = nullptr;
    c->wgraph[i] = nullptr;
  }
  return CISOR_OK;
}

static void free_ctx(cisor_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int i = 0; i < 2; ++i) {
    if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    if (c->wgraph[i]) cudaGraphExecDestroy(c->wgraph[i]);
  }
  if (c->loop_item) cudaFree(c->loop_item);
  if (c->loop_count) cudaFree(c->loop_count);
  if (c->h_loop_count) cudaFreeHost(c->h_loop_count);
  void* dev[] = {c->ghat, c->tw, c->twst, c->H, c->u_in, c->R, c->r, c->rhat, c->p, c->v, c->s, c->tv, c->b, c->u,
                 c->vadj, c->z, c->gz, c->f, c->fz, c->grad, c->work_n, c->Y, c->w, c->yobs, c->sense_part,
                 c->part, c->scal, c->active, c->iters, c->txflag, c->dsum, c->sparams, c->tv_z,
                 c->tv_r0, c->tv_r1, c->tv_p, c->rx_mask, c->tva0, c->tva1, c->vbuf, c->f_ck, c->Ht};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (c->h_active) cudaFreeHost(c->h_active);
  if (c->h_dsum) cudaFreeHost(c->h_dsum);
  if (c->h_tc_err) cudaFreeHost(c->h_tc_err);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace cisor

using namespace cisor;

extern "C" {

const char* cisor_last_error(void) { return g_err; }

const char* cisor_version(void) { return "cisor-gb300 0.1 (sm_103a)"; }

cisor_status cisor_create(cisor_ctx** out, const cisor_geometry* g, void* stream) {
  if (!out || !g) {
    set_error("cisor_create: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (g->dim != 2 && g->dim != 3) {
    set_error("dim must be 2 or 3 (got %d)", g->dim);
    return CISOR_ERR_INVALID_ARG;
  }
  const int nmax = g->dim == 3 ? 128 : 256, pmax = g->dim == 3 ? 256 : 512;
  if (g->n < 8 || g->n > nmax || !(g->delta > 0) || !(g->wavelength > 0) || !(g->eps_b > 0) || g->T < 1 ||
      g->T > 1024 || g->M < 1 || !g->tx_angles || !g->rx_pos) {
    set_error("invalid geometry (n %d, T %d, M %d, delta %g, wavelength %g, eps_b %g)", g->n, g->T, g->M, g->delta,
              g->wavelength, g->eps_b);
    return CISOR_ERR_INVALID_ARG;
  }
  if (g->vectorial && (g->dim != 3 || g->tx_kind != 0 || g->eps_b != 1.0 || g->n > 64)) {
    set_error("the vectorial model needs dim 3, polarised plane waves (tx_kind 0), eps_b = 1 and n <= 64");
    return CISOR_ERR_INVALID_ARG;
  }
  if (g->vectorial) {  // [T, 6]: unit direction d_t, unit polarisation p_t, p_t . d_t = 0
    for (int t = 0; t < g->T; ++t) {
      const double* q = g->tx_angles + 6 * t;
      const double dd = q[0] * q[0] + q[1] * q[1] + q[2] * q[2], pp = q[3] * q[3] + q[4] * q[4] + q[5] * q[5];
      const double dp = q[0] * q[3] + q[1] * q[4] + q[2] * q[5];
      if (fabs(dd - 1.0) > 1e-6 || fabs(pp - 1.0) > 1e-6 || fabs(dp) > 1e-6) {
        set_error("transmitter %d: direction and polarisation must be orthogonal unit vectors", t);
        return CISOR_ERR_INVALID_ARG;
      }
    }
  }
  if (g->tx_kind != 0 && g->tx_kind != 1) {
    set_error("tx_kind must be 0 (plane waves) or 1 (point sources), got %d", g->tx_kind);
    return CISOR_ERR_INVALID_ARG;
  }
  if (g->tx_kind == 1) {  // sources outside the grid's bounding box: g is never evaluated at r = 0
    const double half = 0.5 * g->n * g->delta;
    for (int t = 0; t < g->T; ++t) {
      bool outside = false;
      for (int a = 0; a < g->dim; ++a) outside |= fabs(g->tx_angles[(size_t)g->dim * t + a]) > half;
      if (!outside) {
        set_error("point source %d lies inside the grid's bounding box (half-width %g)", t, half);
        return CISOR_ERR_INVALID_ARG;
      }
    }
  }
  int P = g->pad;
  if (P == 0) {
    P = 64;
    while (P < 2 * g->n - 1) P *= 2;
  }
  if ((P & (P - 1)) != 0 || P < 64 || P > pmax || P < 2 * g->n - 1) {
    set_error("FFT side %d must be a power of two in [64, %d] and >= 2n - 1 = %d", P, pmax, 2 * g->n - 1);
    return CISOR_ERR_INVALID_ARG;
  }
  cisor_ctx* c = new (std::nothrow) cisor_ctx();
  if (!c) {
    set_error("out of host memory");
    return CISOR_ERR_OOM;
  }
  c->dim = g->dim;
  c->n = g->n;
  c->P = P;
  c->T = g->T;
  c->M = g->M;
  c->complex_f = g->complex_f ? 1 : 0;
  c->N = (long long)g->n * g->n * (g->dim == 3 ? g->n : 1);
  c->ncomp = g->vectorial ? 3 : 1;
  c->Nf = c->N * c->ncomp;
  c->delta = g->delta;
  c->wavelength = g->wavelength;
  c->eps_b = g->eps_b;
  c->k = 2.0 * 3.14159265358979323846 / g->wavelength;
  c->kb = c->k * sqrt(g->eps_b);
  const int d = g->dim;
  c->tx_kind = g->tx_kind;
  const size_t per_tx = g->vectorial ? 6 : (g->tx_kind == 1 ? (size_t)d : (d == 3 ? 3 : 1));
  c->tx_angles.assign(g->tx_angles, g->tx_angles + per_tx * g->T);
  c->rx_pos.assign(g->rx_pos, g->rx_pos + (size_t)d * g->M);
  c->user_stream = (cudaStream_t)stream;
  c->graph_chunk = 4;
  c->use_while = 0;  // host-driven chunks by default: profilers list the kernels of these graphs
  c->cols_nt = 512;
  conv_geometry(c);
  {
    // split-K of the forward sensing GEMM: about 4 CTAs per SM, chunks of >= 256 pixels
    const int tiles = sense_tiles(c->M, c->T);
    int ks = (4 * 152 + tiles - 1) / tiles;
    const int kmax = (int)((c->Nf + 255) / 256);
    c->ksplit = ks < 1 ? 1 : (ks > kmax ? kmax : ks);
  }
  cisor_status st = CISOR_OK;
  auto fail = [&](cisor_status s) {
    free_ctx(c);
    return s;
  };
#define ALLOC(ptr, bytes)                                              \
  do {                                                                 \
    cudaError_t e__ = cudaMalloc((void**)&(ptr), (bytes));             \
    if (e__ != cudaSuccess) return fail(cuda_fail(e__, "cudaMalloc " #ptr, __FILE__, __LINE__)); \
  } while (0)
  {
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_fail(e, "stream/event setup", __FILE__, __LINE__));
  }
  const size_t TN = (size_t)c->T * c->Nf * sizeof(float2);
  const size_t Nb = (size_t)c->N * sizeof(float2);
  const size_t TM = (size_t)c->T * c->M * sizeof(float2);
  const size_t Pd = (size_t)P * P * (d == 3 ? P : 1);
  ALLOC(c->ghat, sizeof(float2) * Pd);
  ALLOC(c->tw, sizeof(float2) * P);
  ALLOC(c->twst, sizeof(float2) * 2 * 512);
  ALLOC(c->H, (size_t)c->M * c->Nf * sizeof(float2));
  ALLOC(c->u_in, TN);
  ALLOC(c->R, (size_t)c->T * c->ncomp * c->rtstride * sizeof(float2));
  ALLOC(c->r, TN);
  ALLOC(c->rhat, TN);
  ALLOC(c->p, TN);
  ALLOC(c->v, TN);
  ALLOC(c->s, TN);
  ALLOC(c->tv, TN > sizeof(float2) * Pd ? TN : sizeof(float2) * Pd);
  ALLOC(c->b, TN);
  ALLOC(c->u, TN);
  ALLOC(c->vadj, TN);
  ALLOC(c->z, TN);
  ALLOC(c->gz, TN);
  ALLOC(c->f, Nb);
  ALLOC(c->fz, Nb);
  ALLOC(c->f_ck, Nb);
  ALLOC(c->grad, Nb);
  ALLOC(c->work_n, Nb);
  ALLOC(c->Y, TM);
  ALLOC(c->w, TM);
  ALLOC(c->yobs, TM);
  {
    int ks = c->ksplit;
    if (sense_tc_ok(c)) {  // tensor-core sensing: the transposed matrix, the timeout flag, its split-K partials
      ALLOC(c->Ht, (size_t)c->M * c->Nf * sizeof(float2));
      cudaError_t e = cudaHostAlloc((void**)&c->h_tc_err, sizeof(int), cudaHostAllocMapped);
      if (e == cudaSuccess) {
        *c->h_tc_err = 0;
        e = cudaHostGetDevicePointer((void**)&c->tc_err, c->h_tc_err, 0);
      }
      if (e != cudaSuccess) return fail(cuda_fail(e, "mapped flag", __FILE__, __LINE__));
      st = sense_tc_setup(c);
      if (st != CISOR_OK) return fail(st);
      const int s = sense_tc_splits(c, nullptr);
      if (s > ks) ks = s;
    }
    ALLOC(c->sense_part, TM * ks);
  }
  ALLOC(c->part, sizeof(float) * 2 * DOT_SLOTS * (size_t)c->T * c->nblk * c->ncomp);
  if (c->ncomp == 3) ALLOC(c->vbuf, TN);
  ALLOC(c->scal, sizeof(double) * 2 * SC_STRIDE * (size_t)c->T);
  ALLOC(c->active, sizeof(int) * c->T);
  ALLOC(c->iters, sizeof(int) * c->T);
  ALLOC(c->txflag, sizeof(int) * c->T);
  ALLOC(c->dsum, sizeof(double) * 4);
  ALLOC(c->sparams, sizeof(double) * 2);
  ALLOC(c->tv_z, sizeof(float) * 2 * c->N);
  ALLOC(c->tv_r0, sizeof(float) * 2 * d * c->N);
  ALLOC(c->tv_r1, sizeof(float) * 2 * d * c->N);
  ALLOC(c->tv_p, sizeof(float) * 2 * d * c->N);
  ALLOC(c->tva0, sizeof(float) * 2 * (2 * d + 1) * c->N);
  ALLOC(c->tva1, sizeof(float) * 2 * (2 * d + 1) * c->N);
#undef ALLOC
  {
    cudaError_t e = cudaMallocHost((void**)&c->h_active, sizeof(int) * c->T);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_dsum, sizeof(double) * 4);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__));
  }
  st = conv_init(P);
  if (st != CISOR_OK) return fail(st);
  st = build_tables(c);
  if (st != CISOR_OK) return fail(st);
  *out = c;
  return CISOR_OK;
}

cisor_status cisor_destroy(cisor_ctx* ctx) {
  free_ctx(ctx);
  return CISOR_OK;
}

cisor_status cisor_sizes(const cisor_ctx* c, int* n, int* P, int* T, int* M, long long* N) {
  if (!c) {
    set_error("NULL context");
    return CISOR_ERR_INVALID_ARG;
  }
  if (n) *n = c->n;
  if (P) *P = c->P;
  if (T) *T = c->T;
  if (M) *M = c->M;
  if (N) *N = c->N;
  return CISOR_OK;
}

cisor_status cisor_green_spectrum(cisor_ctx* c, void* out) {
  if (!c || !out) {
    set_error("cisor_green_spectrum: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  const long long PP = (long long)c->P * c->P * (c->dim == 3 ? c->P : 1);
  scale_copy_kernel<<<(unsigned)((PP + 255) / 256), 256, 0, c->stream>>>(c->ghat, c->tv, PP, (float)PP);
  CISOR_CUDA(cudaGetLastError());
  c->launches += 1;
  CISOR_TRY(call.out(out, c->tv, sizeof(float2) * PP));
  return call.leave();
}

cisor_status cisor_sensing_matrix(cisor_ctx* c, void* out) {
  if (!c || !out) {
    set_error("cisor_sensing_matrix: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.out(out, c->H, sizeof(float2) * (size_t)c->M * c->Nf));
  return call.leave();
}

cisor_status cisor_incident(cisor_ctx* c, void* out) {
  if (!c || !out) {
    set_error("cisor_incident: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.out(out, c->u_in, sizeof(float2) * (size_t)c->T * c->Nf));
  return call.leave();
}

// y = A x (or A^H x) for nvec fields, no dot products
static cisor_status matvec_once(cisor_ctx* c, int adjoint, int nvec, const float2* x, float2* y) {
  if (c->ncomp == 3) {
    VecOp vo{};
    vo.adjoint = adjoint ? 1 : 0;
    vo.epilogue = EPI_MATVEC;
    vo.x = x;
    vo.out = y;
    vo.ntx = nvec;
    return vec_matvec(c, vo);
  }
  ConvOp op{};
  op.adjoint = adjoint ? 1 : 0;
  op.mul_f = 1;
  op.prologue = PRO_COPY;
  op.src = x;
  op.epilogue = EPI_MATVEC;
  op.esrc = x;
  op.out = y;
  op.f = c->f;
  op.ntx = nvec;
  return conv_pass(c, op);
}

cisor_status cisor_apply_A(cisor_ctx* c, const void* f, const void* x, void* y, int adjoint, int nvec) {
  if (!c || !f || !x || !y || nvec < 1 || nvec > (c ? c->T : 0)) {
    set_error("cisor_apply_A: NULL argument or nvec outside [1, T]");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  const size_t vb = sizeof(float2) * (size_t)nvec * c->Nf;
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_TRY(call.in(c->s, x, vb));
  CISOR_TRY(matvec_once(c, adjoint, nvec, c->s, c->tv));
  CISOR_TRY(call.out(y, c->tv, vb));
  return call.leave();
}

cisor_status cisor_forward(cisor_ctx* c, const void* f, const void* u_in, const void* x0, void* u_out, void* y_out,
                           const cisor_solve_opts* o, cisor_solve_info* info) {
  if (!c || !f) {
    set_error("cisor_forward: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!check_opts(o)) return CISOR_ERR_INVALID_ARG;
  if (o->x0_mode == 1 && !x0) {
    set_error("cisor_forward: x0_mode 1 needs x0");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  drop_data_term(c);  // the solve overwrites c->u
  const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  const float2* b = c->u_in;
  if (u_in) {
    CISOR_TRY(call.in(c->b, u_in, vb));
    b = c->b;
  }
  if (o->x0_mode == 1) {
    CISOR_TRY(call.in(c->u, x0, vb));
  } else if (o->x0_mode == 0 || !c->have_u) {
    CISOR_CUDA(cudaMemcpyAsync(c->u, b, vb, cudaMemcpyDeviceToDevice, c->stream));
  }
  cisor_solve_info li{};
  int nb = 0;
  cisor_status st = solve_batch(c, 0, c->f, b, c->u, c->T, o->tol, o->max_iter, &li.iters_max, &li.iters_mean,
                                &li.resid_max, &nb);
  if (!solve_ok(st)) return st;
  li.n_not_converged = nb;
  c->have_u = 1;
  if (u_out) CISOR_TRY(call.out(u_out, c->u, vb));
  if (y_out) {
    CISOR_TRY(sense_forward(c, c->f, c->u, c->Y, c->T));
    CISOR_TRY(call.out(y_out, c->Y, sizeof(float2) * (size_t)c->T * c->M));
  }
  if (info) *info = li;
  CISOR_TRY(call.leave());
  return st;
}

cisor_status cisor_sense(cisor_ctx* c, const void* f, const void* u, void* Z_out) {
  if (!c || !f || !u || !Z_out) {
    set_error("cisor_sense: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_TRY(call.in(c->s, u, sizeof(float2) * (size_t)c->T * c->Nf));
  CISOR_TRY(sense_forward(c, c->f, c->s, c->Y, c->T));
  CISOR_TRY(call.out(Z_out, c->Y, sizeof(float2) * (size_t)c->T * c->M));
  return call.leave();
}

cisor_status cisor_sense_adjoint(cisor_ctx* c, const void* f, const void* w, void* z_out, void* b_out) {
  if (!c || !f || !w) {
    set_error("cisor_sense_adjoint: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  drop_data_term(c);  // c->w is overwritten
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_TRY(call.in(c->w, w, sizeof(float2) * (size_t)c->T * c->M));
  CISOR_TRY(sense_adjoint(c, c->f, c->w, c->z, c->b, c->T));
  const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
  CISOR_TRY(call.out(z_out, c->z, vb));
  CISOR_TRY(call.out(b_out, c->b, vb));
  return call.leave();
}

cisor_status cisor_grad(cisor_ctx* c, const void* f, const void* y, void* grad_out, double* D_out,
                        const cisor_solve_opts* o, cisor_solve_info* info) {
  if (!c || !f || !y || !grad_out) {
    set_error("cisor_grad: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!check_opts(o)) return CISOR_ERR_INVALID_ARG;
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_TRY(call.in(c->yobs, y, sizeof(float2) * (size_t)c->T * c->M));
  drop_data_term(c);  // u and w are recomputed at this f
  double D = 0.0;
  cisor_status st = grad_core(c, o, 0.0, nullptr, nullptr, &D, info);
  if (!solve_ok(st)) return st;
  CISOR_TRY(call.out(grad_out, c->grad, sizeof(float2) * c->N));
  if (D_out) *D_out = D;
  CISOR_TRY(call.leave());
  return st;
}

cisor_status cisor_data_term(cisor_ctx* c, const void* f, const void* y, double* D_out, const cisor_solve_opts* o,
                             cisor_solve_info* info) {
  if (!c || !f || !y) {
    set_error("cisor_data_term: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!check_opts(o)) return CISOR_ERR_INVALID_ARG;
  Call call(c);
  CISOR_TRY(call.enter());
  drop_data_term(c);
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_CUDA(cudaMemcpyAsync(c->f_ck, c->f, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  CISOR_TRY(call.in(c->yobs, y, sizeof(float2) * (size_t)c->T * c->M));
  double D = 0.0;
  cisor_solve_info li{};
  cisor_status st = data_core(c, o, &D, &li);
  if (!solve_ok(st)) return st;
  c->have_w = 1;
  if (D_out) *D_out = D;
  if (info) *info = li;
  CISOR_TRY(call.leave());
  return st;
}

cisor_status cisor_data_backward(cisor_ctx* c, void* grad_out, const cisor_solve_opts* o, cisor_solve_info* info) {
  if (!c || !grad_out) {
    set_error("cisor_data_backward: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!check_opts(o)) return CISOR_ERR_INVALID_ARG;
  if (!c->have_w) {
    set_error("cisor_data_backward: no preceding cisor_data_term on this context");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  // other entry points may have written c->f since cisor_data_term (apply_A, sense, autotune, time_matvec)
  CISOR_CUDA(cudaMemcpyAsync(c->f, c->f_ck, sizeof(float2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  cisor_solve_info li{};
  cisor_status st = adjoint_core(c, o, 0.0, nullptr, nullptr, &li);
  if (!solve_ok(st)) return st;
  CISOR_TRY(call.out(grad_out, c->grad, sizeof(float2) * c->N));
  if (info) {
    info->adj_iters_max = li.adj_iters_max;
    info->adj_iters_mean = li.adj_iters_mean;
    info->adj_resid_max = li.adj_resid_max;
    info->n_not_converged = li.n_not_converged;
  }
  CISOR_TRY(call.leave());
  return st;
}

static cisor_status tv_prox_entry(cisor_ctx* c, const void* z, void* x, double gamma_tau, int iters, double lo,
                                  double hi, double lo_im, double hi_im, int aniso) {
  if (!c || !z || !x || iters < 0 || !(lo <= hi) || (c && c->complex_f && !(lo_im <= hi_im))) {
    set_error("cisor_tv_prox: NULL argument, negative iteration count or empty box");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.in(c->fz, z, sizeof(float2) * c->N));
  auto prox = aniso ? tv_prox_aniso : tv_prox;
  CISOR_TRY(prox(c, c->fz, c->work_n, gamma_tau, iters, lo, hi, lo_im, hi_im, c->complex_f, nullptr, 0.0, nullptr));
  CISOR_TRY(call.out(x, c->work_n, sizeof(float2) * c->N));
  return call.leave();
}

cisor_status cisor_tv_prox(cisor_ctx* c, const void* z, void* x, double gamma_tau, int iters, double lo, double hi,
                           double lo_im, double hi_im) {
  return tv_prox_entry(c, z, x, gamma_tau, iters, lo, hi, lo_im, hi_im, 0);
}

cisor_status cisor_tv_prox_aniso(cisor_ctx* c, const void* z, void* x, double gamma_tau, int iters, double lo,
                                 double hi, double lo_im, double hi_im) {
  return tv_prox_entry(c, z, x, gamma_tau, iters, lo, hi, lo_im, hi_im, 1);
}

static bool state_ok(const cisor_ctx* c, const cisor_fista_state* st, const char* who) {
  if (!(st->alpha >= 0.0 && st->alpha <= 1.0) || !(st->gamma > 0.0) || !(st->tau >= 0.0) || st->tv_iters < 0 ||
      !(st->lo <= st->hi) || (c->complex_f && !(st->lo_im <= st->hi_im)) || !(st->t >= 1.0) ||
      (st->tv_kind != 0 && st->tv_kind != 1)) {
    set_error("%s: invalid state (alpha %g, gamma %g, tau %g, t %g)", who, st->alpha, st->gamma, st->tau, st->t);
    return false;
  }
  return true;
}

// f_k = prox(z) into work_n and s_{k+1} into c->f, from z in c->fz and f_{k-1} in work_n (Eqs. 9-11)
static cisor_status prox_and_momentum(cisor_ctx* c, cisor_fista_state* st, double* tn_out) {
  const double t = st->t;
  const double tn = (sqrt(4.0 * t * t + 1.0) + 1.0) / 2.0;
  const double beta = st->alpha * (t - 1.0) / tn;
  auto prox = st->tv_kind == 1 ? tv_prox_aniso : tv_prox;
  CISOR_TRY(prox(c, c->fz, c->work_n, st->gamma * st->tau, st->tv_iters, st->lo, st->hi, st->lo_im, st->hi_im,
                 c->complex_f, c->work_n, beta, c->f));
  *tn_out = tn;
  return CISOR_OK;
}

cisor_status cisor_step_update(cisor_ctx* c, cisor_fista_state* st, const void* grad, double D) {
  if (!c || !st || !st->f || !st->s || !grad) {
    set_error("cisor_step_update: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!state_ok(c, st, "cisor_step_update")) return CISOR_ERR_INVALID_ARG;
  Call call(c);
  CISOR_TRY(call.enter());
  const size_t nb = sizeof(float2) * c->N;
  CISOR_TRY(call.in(c->f, st->s, nb));       // s_k
  CISOR_TRY(call.in(c->work_n, st->f, nb));  // f_{k-1}
  CISOR_TRY(call.in(c->grad, grad, nb));
  CISOR_TRY(gradient_step(c, c->f, c->grad, st->gamma, c->fz));
  double tn = 0.0;
  CISOR_TRY(prox_and_momentum(c, st, &tn));
  CISOR_TRY(call.out(st->f, c->work_n, nb));
  CISOR_TRY(call.out(st->s, c->f, nb));
  CISOR_TRY(call.leave());
  st->t = tn;
  st->k += 1;
  st->D = D;
  return CISOR_OK;
}

cisor_status cisor_step(cisor_ctx* c, cisor_fista_state* st, const void* y, const cisor_solve_opts* o,
                        cisor_solve_info* info) {
  if (!c || !st || !st->f || !st->s || !y) {
    set_error("cisor_step: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!check_opts(o)) return CISOR_ERR_INVALID_ARG;
  if (!state_ok(c, st, "cisor_step")) return CISOR_ERR_INVALID_ARG;
  Call call(c);
  CISOR_TRY(call.enter());
  const size_t nb = sizeof(float2) * c->N;
  CISOR_TRY(call.in(c->yobs, y, sizeof(float2) * (size_t)c->T * c->M));
  CISOR_TRY(call.in(c->f, st->s, nb));       // gradient at s_k
  CISOR_TRY(call.in(c->work_n, st->f, nb));  // f_{k-1}
  drop_data_term(c);  // u and w are recomputed at s_k
  double D = 0.0;
  cisor_status s1 = grad_core(c, o, st->gamma, c->f, c->fz, &D, info);
  if (!solve_ok(s1)) return s1;
  double tn = 0.0;
  CISOR_TRY(prox_and_momentum(c, st, &tn));
  CISOR_TRY(call.out(st->f, c->work_n, nb));
  CISOR_TRY(call.out(st->s, c->f, nb));
  CISOR_TRY(call.leave());
  st->t = tn;
  st->k += 1;
  st->D = D;
  return s1;
}

cisor_status cisor_set_rx_mask(cisor_ctx* c, const void* mask) {
  if (!c) {
    set_error("cisor_set_rx_mask: NULL context");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!mask) {
    if (c->rx_mask) CISOR_CUDA(cudaFree(c->rx_mask));
    c->rx_mask = nullptr;
    return CISOR_OK;
  }
  if (!c->rx_mask) CISOR_CUDA(cudaMalloc((void**)&c->rx_mask, (size_t)c->T * c->M));
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.in(c->rx_mask, mask, (size_t)c->T * c->M));
  return call.leave();
}

static bool two_stage_ok(const cisor_ctx* c) { return c->P == 128 || c->P == 256 || (c->dim == 2 && c->P == 512); }

cisor_status cisor_set_cols_cta(cisor_ctx* c, int cols_nt) {
  if (!c || (cols_nt != 512 && cols_nt != 256 && cols_nt != COLS_TWO_STAGE && cols_nt != COLS_CLUSTER)) {
    set_error("cisor_set_cols_cta: NULL context or cols_nt not 512 / 256 / %d / %d", COLS_TWO_STAGE, COLS_CLUSTER);
    return CISOR_ERR_INVALID_ARG;
  }
  if (cols_nt == COLS_CLUSTER && !conv_fused_ok(c)) {
    set_error("cisor_set_cols_cta: the cluster pass (%d) needs a scalar 2D grid with P = 512", COLS_CLUSTER);
    return CISOR_ERR_INVALID_ARG;
  }
  if (cols_nt == COLS_TWO_STAGE && !two_stage_ok(c)) {
    set_error("cisor_set_cols_cta: the two-stage column shape (%d) needs P = 128 or 256, or P = 512 in 2D "
              "(this grid: %dD, P = %d)", COLS_TWO_STAGE, c->dim, c->P);
    return CISOR_ERR_INVALID_ARG;
  }
  if (cols_nt != c->cols_nt) {
    c->cols_nt = cols_nt;
    CISOR_TRY(drop_graphs(c));
  }
  return CISOR_OK;
}

cisor_status cisor_set_tx_chunk(cisor_ctx* c, int tx_chunk) {
  if (!c || tx_chunk < 0) {
    set_error("cisor_set_tx_chunk: NULL context or negative chunk");
    return CISOR_ERR_INVALID_ARG;
  }
  if (tx_chunk != c->tx_chunk) {
    c->tx_chunk = tx_chunk;
    CISOR_TRY(drop_graphs(c));
  }
  return CISOR_OK;
}

cisor_status cisor_set_solve_loop(cisor_ctx* c, int device_loop) {
  if (!c || (device_loop != 0 && device_loop != 1)) {
    set_error("cisor_set_solve_loop: NULL context or mode not 0 / 1");
    return CISOR_ERR_INVALID_ARG;
  }
  c->use_while = device_loop;
  return drop_graphs(c);
}

cisor_status cisor_tuning(const cisor_ctx* c, int* cols_nt, int* tx_chunk) {
  if (!c) {
    set_error("cisor_tuning: NULL context");
    return CISOR_ERR_INVALID_ARG;
  }
  if (cols_nt) *cols_nt = c->cols_nt;
  if (tx_chunk) *tx_chunk = c->tx_chunk;
  return CISOR_OK;
}

cisor_status cisor_solve_iterations(const cisor_ctx* c, int adjoint, int* iters_out, int* count) {
  if (!c || !count) {
    set_error("cisor_solve_iterations: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  const std::vector<int>& it = c->last_iters[adjoint ? 1 : 0];
  *count = (int)it.size();
  if (iters_out)
    for (size_t i = 0; i < it.size(); ++i) iters_out[i] = it[i];
  return CISOR_OK;
}

cisor_status cisor_autotune(cisor_ctx* c, int reps, int* cols_nt_out) {
  if (!c || reps < 1) {
    set_error("cisor_autotune: NULL context or reps < 1");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_CUDA(cudaMemcpyAsync(c->s, c->u_in, sizeof(float2) * (size_t)c->T * c->Nf, cudaMemcpyDeviceToDevice, c->stream));
  CISOR_CUDA(cudaMemsetAsync(c->f, 0, sizeof(float2) * c->N, c->stream));
  cudaEvent_t e0, e1;
  CISOR_CUDA(cudaEventCreate(&e0));
  CISOR_CUDA(cudaEventCreate(&e1));
  int variants[4] = {512, 256, 0, 0};
  int nvar = 2;
  if (two_stage_ok(c)) variants[nvar++] = COLS_TWO_STAGE;
  if (conv_fused_ok(c)) variants[nvar++] = COLS_CLUSTER;
  // transmitter chunks whose FFT intermediate takes about 16, 32 or 48 MB (L2 is 126 MB), and no chunking
  const int ntr = c->T * c->ncomp;
  const long long rbytes = (long long)c->rtstride * (long long)sizeof(float2);
  int chunks[4] = {0, 0, 0, 0};
  int nch = 1;
  for (int mb = 16; mb <= 48; mb += 16) {
    const long long k = ((long long)mb << 20) / rbytes;
    if (k >= 1 && k < ntr && (nch == 1 || k != chunks[nch - 1])) chunks[nch++] = (int)k;
  }
  int best = 512, best_chunk = 0;
  float best_ms = 1e30f;
  cisor_status st = CISOR_OK;
  for (int v = 0; v < nvar && st == CISOR_OK; ++v)
    for (int h = 0; h < nch && st == CISOR_OK; ++h) {
      c->cols_nt = variants[v];
      c->tx_chunk = chunks[h];
      st = matvec_once(c, 0, c->T, c->s, c->tv);  // warm-up
      CISOR_CUDA(cudaEventRecord(e0, c->stream));
      for (int i = 0; i < reps && st == CISOR_OK; ++i) st = matvec_once(c, 0, c->T, c->s, c->tv);
      CISOR_CUDA(cudaEventRecord(e1, c->stream));
      CISOR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CISOR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = variants[v];
        best_chunk = chunks[h];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CISOR_TRY(st);
  c->cols_nt = best;
  c->tx_chunk = best_chunk;
  CISOR_TRY(drop_graphs(c));
  if (cols_nt_out) *cols_nt_out = best;
  return call.leave();
}

cisor_status cisor_launch_count(const cisor_ctx* c, long long* count) {
  if (!c || !count) {
    set_error("cisor_launch_count: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  *count = c->launches;
  return CISOR_OK;
}

cisor_status cisor_device_info(int device, int* sm_count, int* max_clock_khz, int* fp32_lanes, int* cc) {
  int sms = 0, clk = 0, ma = 0, mi = 0;
  CISOR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  CISOR_CUDA(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device));
  CISOR_CUDA(cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, device));
  CISOR_CUDA(cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, device));
  if (sm_count) *sm_count = sms;
  if (max_clock_khz) *max_clock_khz = clk;
  if (fp32_lanes) *fp32_lanes = (ma == 10 || ma == 12) ? 128 : ((ma == 9 || (ma == 8 && mi == 0)) ? 64 : 0);
  if (cc) *cc = 10 * ma + mi;
  return CISOR_OK;
}

cisor_status cisor_time_matvec(cisor_ctx* c, const void* f, int adjoint, int reps, double* ms_per_pass) {
  if (!c || !f || reps < 1 || !ms_per_pass) {
    set_error("cisor_time_matvec: NULL argument or reps < 1");
    return CISOR_ERR_INVALID_ARG;
  }
  Call call(c);
  CISOR_TRY(call.enter());
  CISOR_TRY(call.in(c->f, f, sizeof(float2) * c->N));
  CISOR_CUDA(cudaMemcpyAsync(c->s, c->u_in, sizeof(float2) * (size_t)c->T * c->Nf, cudaMemcpyDeviceToDevice, c->stream));
  CISOR_TRY(matvec_once(c, adjoint, c->T, c->s, c->tv));
  cudaEvent_t e0, e1;
  CISOR_CUDA(cudaEventCreate(&e0));
  CISOR_CUDA(cudaEventCreate(&e1));
  CISOR_CUDA(cudaEventRecord(e0, c->stream));
  cisor_status st = CISOR_OK;
  for (int i = 0; i < reps && st == CISOR_OK; ++i) st = matvec_once(c, adjoint, c->T, c->s, c->tv);
  CISOR_CUDA(cudaEventRecord(e1, c->stream));
  CISOR_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  CISOR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CISOR_TRY(st);
  *ms_per_pass = ms / reps;
  return call.leave();
}

}  // extern "C"
