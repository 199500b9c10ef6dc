// Several imaging problems of uneven size (grid side, transmitter count,
// receivers) solved together.  Each problem keeps its own context (tables,
// workspace, stream, FFT-size-specialised kernels); the field solves of all
// problems advance in ONE CUDA-graph launch per chunk of BiCGSTAB iterations
// (fork to every problem's stream, join back), so small problems fill the GPU
// together instead of one after another.  Sensing, gradient assembly and the
// table set-up run per problem on the problems' own streams, concurrently.
#include <new>
#include <vector>

#include "common.cuh"

struct cisor_batch {
  std::vector<cisor_ctx*> ctx;
  cudaStream_t user_stream = nullptr;
  cudaEvent_t ev_in = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<long long> kern[2];
  cisor::MultiSolve ms{};
};

using namespace cisor;

namespace {

void free_batch(cisor_batch* b) {
  if (!b) return;
  if (b->ms.main) cudaStreamSynchronize(b->ms.main);
  for (int d = 0; d < 2; ++d) {
    if (b->ms.graph[d]) cudaGraphExecDestroy(b->ms.graph[d]);
    if (b->ms.wgraph[d]) cudaGraphExecDestroy(b->ms.wgraph[d]);
  }
  if (b->ms.items) cudaFree(b->ms.items);
  if (b->ms.loop_count) cudaFree(b->ms.loop_count);
  if (b->ms.h_loop_count) cudaFreeHost(b->ms.h_loop_count);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->ms.fork) cudaEventDestroy(b->ms.fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ms.main) cudaStreamDestroy(b->ms.main);
  for (cisor_ctx* c : b->ctx) cisor_destroy(c);
  delete b;
}

bool opts_ok(const cisor_solve_opts* o) {
  if (!o || !(o->tol > 0.0) || o->max_iter < 1 || o->x0_mode < 0 || o->x0_mode > 2 || o->x0_mode == 1) {
    set_error("batch: invalid solve options (x0_mode must be 0 or 2)");
    return false;
  }
  return true;
}

// caller's stream -> every problem stream
cisor_status enter(cisor_batch* b) {
  CISOR_CUDA(cudaEventRecord(b->ev_in, b->user_stream));
  for (cisor_ctx* c : b->ctx) CISOR_CUDA(cudaStreamWaitEvent(c->stream, b->ev_in, 0));
  return CISOR_OK;
}

// every problem stream -> caller's stream; synchronise when host memory was written
cisor_status leave(cisor_batch* b, bool host_out) {
  for (cisor_ctx* c : b->ctx) {
    CISOR_CUDA(cudaEventRecord(c->ev_b, c->stream));
    CISOR_CUDA(cudaStreamWaitEvent(b->user_stream, c->ev_b, 0));
  }
  if (host_out)
    for (cisor_ctx* c : b->ctx) CISOR_CUDA(cudaStreamSynchronize(c->stream));
  for (cisor_ctx* c : b->ctx) CISOR_TRY(sense_tc_check(c, host_out));
  return CISOR_OK;
}

bool is_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

void fill_info(cisor_solve_info* info, const SolveStat& fw, const SolveStat* ad) {
  if (!info) return;
  cisor_solve_info li{};
  li.iters_max = fw.iters_max;
  li.iters_mean = fw.iters_mean;
  li.resid_max = fw.resid_max;
  li.n_not_converged = fw.n_bad + (ad ? ad->n_bad : 0);
  if (ad) {
    li.adj_iters_max = ad->iters_max;
    li.adj_iters_mean = ad->iters_mean;
    li.adj_resid_max = ad->resid_max;
  }
  *info = li;
}

cisor_status worst_of(cisor_status a, cisor_status b) {
  if (a == CISOR_ERR_BREAKDOWN || b == CISOR_ERR_BREAKDOWN) return CISOR_ERR_BREAKDOWN;
  if (a == CISOR_ERR_NOT_CONVERGED || b == CISOR_ERR_NOT_CONVERGED) return CISOR_ERR_NOT_CONVERGED;
  return a != CISOR_OK ? a : b;
}

bool solve_ok(cisor_status s) { return s == CISOR_OK || s == CISOR_ERR_NOT_CONVERGED || s == CISOR_ERR_BREAKDOWN; }

}  // namespace

extern "C" {

cisor_status cisor_batch_create(cisor_batch** out, const cisor_geometry* geoms, int nprob, void* stream,
                                int autotune) {
  if (!out || !geoms || nprob < 1 || nprob > 256) {
    set_error("cisor_batch_create: NULL argument or nprob outside [1, 256]");
    return CISOR_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cisor_batch* b = new (std::nothrow) cisor_batch();
  if (!b) {
    set_error("out of host memory");
    return CISOR_ERR_OOM;
  }
  b->user_stream = (cudaStream_t)stream;
  for (int i = 0; i < nprob; ++i) {
    cisor_ctx* c = nullptr;
    cisor_status st = cisor_create(&c, &geoms[i], stream);
    if (st != CISOR_OK) {
      free_batch(b);
      return st;
    }
    b->ctx.push_back(c);
    if (autotune) {
      st = cisor_autotune(c, 5, nullptr);
      if (st != CISOR_OK) {
        free_batch(b);
        return st;
      }
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->ms.main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ms.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  b->join.assign(nprob, nullptr);
  for (int i = 0; i < nprob && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ms.items, sizeof(cisor_loop_item) * nprob);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->ms.loop_count, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->ms.h_loop_count, sizeof(int));
  b->ms.use_while = 1;
  if (e != cudaSuccess) {
    cisor_status st = cuda_fail(e, "batch stream/event setup", __FILE__, __LINE__);
    free_batch(b);
    return st;
  }
  b->ms.join = b->join.data();
  for (int d = 0; d < 2; ++d) {
    b->kern[d].assign(nprob, 0);
    b->ms.kernels[d] = b->kern[d].data();
  }
  *out = b;
  return CISOR_OK;
}

cisor_status cisor_batch_set_solve_loop(cisor_batch* b, int device_loop) {
  if (!b || (device_loop != 0 && device_loop != 1)) {
    set_error("cisor_batch_set_solve_loop: NULL batch or mode not 0 / 1");
    return CISOR_ERR_INVALID_ARG;
  }
  if (b->ms.main) CISOR_CUDA(cudaStreamSynchronize(b->ms.main));
  for (int d = 0; d < 2; ++d) {
    if (b->ms.wgraph[d]) CISOR_CUDA(cudaGraphExecDestroy(b->ms.wgraph[d]));
    b->ms.wgraph[d] = nullptr;
  }
  b->ms.use_while = device_loop;
  return CISOR_OK;
}

cisor_status cisor_batch_destroy(cisor_batch* b) {
  free_batch(b);
  return CISOR_OK;
}

cisor_status cisor_batch_context(cisor_batch* b, int i, cisor_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= (int)b->ctx.size()) {
    set_error("cisor_batch_context: bad argument");
    return CISOR_ERR_INVALID_ARG;
  }
  *ctx = b->ctx[i];
  return CISOR_OK;
}

cisor_status cisor_batch_forward(cisor_batch* b, const void* const* f, void* const* u_out,
                                 const cisor_solve_opts* o, cisor_solve_info* info) {
  if (!b || !f) {
    set_error("cisor_batch_forward: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!opts_ok(o)) return CISOR_ERR_INVALID_ARG;
  const int np = (int)b->ctx.size();
  for (int i = 0; i < np; ++i)
    if (!f[i]) {
      set_error("cisor_batch_forward: f[%d] is NULL", i);
      return CISOR_ERR_INVALID_ARG;
    }
  CISOR_TRY(enter(b));
  std::vector<const float2*> rhs(np);
  for (int i = 0; i < np; ++i) {
    cisor_ctx* c = b->ctx[i];
    const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
    c->have_w = 0;  // this solve overwrites the u a cisor_data_term on the problem's context left
    CISOR_CUDA(cudaMemcpyAsync(c->f, f[i], sizeof(float2) * c->N, cudaMemcpyDefault, c->stream));
    if (o->x0_mode == 0 || !c->have_u)
      CISOR_CUDA(cudaMemcpyAsync(c->u, c->u_in, vb, cudaMemcpyDeviceToDevice, c->stream));
    rhs[i] = c->u_in;
  }
  std::vector<SolveStat> st(np);
  cisor_status s = solve_multi(b->ctx.data(), np, 0, rhs.data(), o->tol, o->max_iter, b->ms, st.data());
  if (!solve_ok(s)) return s;
  bool host_out = false;
  for (int i = 0; i < np; ++i) {
    cisor_ctx* c = b->ctx[i];
    c->have_u = 1;
    if (u_out && u_out[i]) {
      host_out |= is_host(u_out[i]);
      CISOR_CUDA(cudaMemcpyAsync(u_out[i], c->u, sizeof(float2) * (size_t)c->T * c->Nf, cudaMemcpyDefault,
                                 c->stream));
    }
    if (info) fill_info(&info[i], st[i], nullptr);
  }
  CISOR_TRY(leave(b, host_out));
  return s;
}

cisor_status cisor_batch_grad(cisor_batch* b, const void* const* f, const void* const* y, void* const* grad_out,
                              double* D_out, const cisor_solve_opts* o, cisor_solve_info* info) {
  if (!b || !f || !y || !grad_out) {
    set_error("cisor_batch_grad: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (!opts_ok(o)) return CISOR_ERR_INVALID_ARG;
  const int np = (int)b->ctx.size();
  for (int i = 0; i < np; ++i)
    if (!f[i] || !y[i] || !grad_out[i]) {
      set_error("cisor_batch_grad: NULL entry %d", i);
      return CISOR_ERR_INVALID_ARG;
    }
  CISOR_TRY(enter(b));
  std::vector<const float2*> rhs(np);
  for (int i = 0; i < np; ++i) {
    cisor_ctx* c = b->ctx[i];
    const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
    c->have_w = 0;  // u and w of the problem's context are overwritten
    CISOR_CUDA(cudaMemcpyAsync(c->f, f[i], sizeof(float2) * c->N, cudaMemcpyDefault, c->stream));
    CISOR_CUDA(cudaMemcpyAsync(c->yobs, y[i], sizeof(float2) * (size_t)c->T * c->M, cudaMemcpyDefault, c->stream));
    if (o->x0_mode == 0 || !c->have_u)
      CISOR_CUDA(cudaMemcpyAsync(c->u, c->u_in, vb, cudaMemcpyDeviceToDevice, c->stream));
    rhs[i] = c->u_in;
  }
  std::vector<SolveStat> fw(np), ad(np);
  cisor_status s1 = solve_multi(b->ctx.data(), np, 0, rhs.data(), o->tol, o->max_iter, b->ms, fw.data());
  if (!solve_ok(s1)) return s1;
  for (int i = 0; i < np; ++i) {
    cisor_ctx* c = b->ctx[i];
    const size_t vb = sizeof(float2) * (size_t)c->T * c->Nf;
    c->have_u = 1;
    CISOR_TRY(residual_and_D(c, c->f, c->u, c->yobs, c->Y, c->w, c->T));
    CISOR_TRY(sense_adjoint(c, c->f, c->w, c->z, c->b, c->T));
    if (o->x0_mode == 0 || !c->have_v) CISOR_CUDA(cudaMemsetAsync(c->vadj, 0, vb, c->stream));
    rhs[i] = c->b;
  }
  cisor_status s2 = solve_multi(b->ctx.data(), np, 1, rhs.data(), o->tol, o->max_iter, b->ms, ad.data());
  if (!solve_ok(s2)) return s2;
  bool host_out = false;
  for (int i = 0; i < np; ++i) {
    cisor_ctx* c = b->ctx[i];
    c->have_v = 1;
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
    CISOR_TRY(grad_assemble(c, c->u, c->gz, nullptr, 0.0, c->grad, nullptr, c->T));
    host_out |= is_host(grad_out[i]);
    CISOR_CUDA(cudaMemcpyAsync(grad_out[i], c->grad, sizeof(float2) * c->N, cudaMemcpyDefault, c->stream));
    CISOR_CUDA(cudaMemcpyAsync(c->h_dsum, c->dsum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  for (int i = 0; i < np; ++i) {
    CISOR_CUDA(cudaStreamSynchronize(b->ctx[i]->stream));
    if (D_out) D_out[i] = b->ctx[i]->h_dsum[0];
    if (info) fill_info(&info[i], fw[i], &ad[i]);
  }
  CISOR_TRY(leave(b, host_out));
  return worst_of(s1, s2);
}

}  // extern "C"
