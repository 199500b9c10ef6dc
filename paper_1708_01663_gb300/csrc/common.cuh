// Internal declarations shared by the translation units of libcisor.
//
// Device data layout (all row-major, x index fastest):
//   fields      [T, n, n] (2D) / [T, n, n, n] (3D)   complex64 (float2), transmitter-major
//   f           [n, n] / [n, n, n]                   complex64
//   R (scratch) [T, n, P] (2D): the padded field after the x FFT; only the n
//               non-zero rows of the P x P padded image are kept.
//               [T, n, P, P] (3D): z slabs of the padded field after the x
//               and y FFTs; only the n non-zero z slabs are kept.
//   ghat        [P^d]    complex64: spectrum of the circulant embedding of
//               G (Sec. II, Eq. 3), pre-scaled by 1/P^d for the inverse FFTs
//   H           [M, N]      complex64 (Eq. 2)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/cisor.h"

namespace cisor {

// ---------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// conj(a) * b
__host__ __device__ __forceinline__ float2 c_cjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc + a * b and acc + conj(a) * b as four FMAs (a product formed first and
// then added would take an extra rounding and two more instructions)
__host__ __device__ __forceinline__ float2 c_fma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ float2 c_cjfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ double2 z_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 z_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 z_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 z_div(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__host__ __device__ __forceinline__ double2 z_conj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 z_to_c(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------- per-transmitter Krylov scalars
// scal[t * SC_STRIDE + i], double2 each
enum {
  SC_RHO = 0,     // <rhat, r>
  SC_ALPHA = 1,
  SC_OMEGA = 2,
  SC_BETA = 3,
  SC_NORMS = 4,   // (||b||^2, ||r||^2)
  SC_REL = 5,     // (recursive rel. residual, true rel. residual)
  SC_STRIDE = 8
};

// dot-product slots written by epilogues: partial sums [T][nblk][3] float2
// (FP32 pairwise tree within a CTA; the per-transmitter sum over CTAs is a
// second FP32 tree; the Krylov scalars built from them are FP64)
enum { DOT_SLOTS = 3 };
// operand codes for epilogue dot products
enum { OP_NONE = 0, OP_Y = 1, OP_SRC = 2, OP_AUX = 3 };

// Solver status flags per transmitter
enum { TX_OK = 0, TX_BREAKDOWN = 1, TX_MAXITER = 2 };

}  // namespace cisor

struct cisor_ctx {
  // geometry
  int dim, n, P, T, M, complex_f;
  long long N;
  int ncomp;              // field components: 1 (scalar), 3 (vectorial model of the appendix)
  long long Nf;           // field length per transmitter: ncomp * N
  int nrows;              // x rows per field: n (2D), n^2 (3D)
  long long rslab;        // R offset between z slabs (3D: P^2)
  long long rtstride;     // R elements per transmitter
  double delta, wavelength, eps_b, k, kb;
  std::vector<double> tx_angles, rx_pos;  // 2D: [T] angles, [M, 2]; 3D: [T, 3] directions, [M, 3];
                                          // point sources (tx_kind 1): [T, d] positions
  int tx_kind;                            // 0 plane waves, 1 point / line sources
  int device;
  cudaStream_t stream;  // internal non-blocking stream; ordered against the caller's via events
  cudaStream_t user_stream;
  cudaEvent_t ev_a, ev_b;
  // tables
  float2* ghat;   // [P^d], scaled by 1/P^d
  float2* tw;     // [P] exp(-2 pi i m / P)
  float2* twst;   // [2][512] stage twiddle tables of the forward / reversed FFT plans
  float2* H;      // [M, N]
  float2* u_in;   // [T, N]
  // Krylov workspace, [T, N] each
  float2 *R, *r, *rhat, *p, *v, *s, *tv, *b;
  float2 *u, *vadj;   // last forward / adjoint solutions (warm starts)
  int have_u, have_v;  // warm starts held
  int have_w;          // 1 from cisor_data_term until an entry point overwrites the u or w it left
  float2* f_ck;        // [N] the point of the last cisor_data_term (its backward half's f)
  float2 *z, *gz;     // H^H w and z + G^H v
  float2 *f, *fz, *grad, *work_n;  // [N]
  float2 *Y, *w, *yobs;          // [T, M]
  unsigned char* rx_mask;        // [T, M] active receivers (NULL: all), set by cisor_set_rx_mask
  float2* sense_part;            // [ksplit, T, M]
  int ksplit;
  float2* Ht;                    // [Nf, M] transposed sensing matrix of the tensor-core adjoint (null: FP32 GEMMs)
  int* tc_err;                   // device alias of h_tc_err
  int* h_tc_err;                 // mapped host flag, set by a sensing kernel whose bounded MMA wait gave up
  bool tc_used;                  // a tensor-core sensing kernel ran in the current call
  int sms;                       // multiprocessors of the device
  int sense_tc_occ;              // resident CTAs per SM of the tensor-core forward sensing kernel
  float* part;     // [T, nblk, DOT_SLOTS] float2
  int nblk;        // dot partials per transmitter
  double* scal;    // [T, SC_STRIDE] double2
  int *active, *iters, *txflag;
  int* h_active;    // pinned [T]
  double* dsum;     // device scalar accumulators [4]
  double* h_dsum;   // pinned [4]
  // TV workspace (d dual components x N floats per plane, up to 2 planes)
  float *tv_z, *tv_r0, *tv_r1, *tv_p;
  float *tva0, *tva1;  // anisotropic TV: (2d + 1) auxiliary images per plane, ping-pong
  float2* vbuf;        // vectorial model: conv output / grad-div pre-pass [T, 3, N]
  // whole-solve graphs: a device-side WHILE loop over chunks of BiCGSTAB iterations
  cudaGraphExec_t wgraph[2];
  int wgraph_ntx[2];
  float2* wgraph_x[2];
  int* loop_count;            // device: loop-body executions of the current launch
  int* h_loop_count;          // pinned copy
  struct cisor_loop_item* loop_item;  // device [1]: this context's active flags for the loop condition
  int use_while;              // 1 until building a WHILE graph fails (then the host-driven chunk loop)
  // graphs of a chunk of BiCGSTAB iterations (host-driven loop)
  cudaGraphExec_t graph[2];
  int graph_ntx[2];
  float2* graph_x[2];
  double* sparams;  // device [2]: solve tolerance, iteration cap (read by the captured graphs)
  int graph_chunk;
  long long launches;       // kernels launched (graph replays add their kernel count)
  int cols_nt;              // column-FFT kernel shape (512 or 256 threads of the three-stage kernel, or
                            // COLS_TWO_STAGE), set by the autotuner
  int tx_chunk;             // transforms per convolution launch (0: all at once); every chunk reuses the
                            // start of R, so a chunk's intermediate can stay in L2 between its kernels
  long long graph_kernels[2];
  std::vector<int> last_iters[2];  // per-transmitter iterations of the last forward / adjoint solve
};

// One problem's per-transmitter active flags, read by the device-side loop
// condition of a whole-solve graph.
struct cisor_loop_item {
  const int* active;
  int ntx;
};

namespace cisor {

// thread-local last error message
void set_error(const char* fmt, ...);
cisor_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CISOR_CUDA(call)                                                      \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess) return cisor::cuda_fail(e__, #call, __FILE__, __LINE__); \
  } while (0)

#define CISOR_TRY(call)                        \
  do {                                         \
    cisor_status s__ = (call);                 \
    if (s__ != CISOR_OK) return s__;           \
  } while (0)

// tables.cu
cisor_status build_tables(cisor_ctx* c);
cisor_status make_stage_twiddles(cisor_ctx* c);  // stage twiddles of P into c->twst, on c->stream

// conv.cu: one batched FFT convolution pass on ntx transmitters.
struct ConvOp {
  int adjoint;            // 0: G (prologue multiplies by f); 1: G^H (epilogue multiplies by conj f)
  int mul_f;              // apply the f factor (A / A^H); 0 gives the bare convolution
  int prologue;           // PRO_*
  int epilogue;           // EPI_*
  const float2* src;      // prologue input: the vector convolved (PRO_COPY), or r (PRO_AXPY / PRO_PUPDATE)
  const float2* esrc;     // epilogue: the x of A x (EPI_MATVEC, EPI_RESID)
  float2* pvec;           // p (PRO_PUPDATE, read-write)
  const float2* vvec;     // v (PRO_PUPDATE, PRO_AXPY)
  float2* svec;           // s written by PRO_AXPY
  const float2* f;        // [N]
  const float2* aux;      // epilogue auxiliary vector (rhat, b, z)
  float2* out;            // epilogue output
  float2* out2;           // second epilogue output (copy of out), may be null
  int dot_a[DOT_SLOTS], dot_b[DOT_SLOTS];  // operand codes per dot slot
  const int* active;      // may be null
  const double* scal;     // per-transmitter scalars (alpha, beta, omega)
  float* part;            // dot partials [T, nblk, DOT_SLOTS] float2
  int ntx;
  int tx_div;             // transforms per transmitter (3: the field components of the vectorial
                          // model run as consecutive transforms; 0 or 1: one)
  int tx0;                // first transform of this launch (set by conv_pass when it splits a pass
                          // into transmitter chunks; R is indexed from the chunk's start)
};
enum { PRO_COPY = 0, PRO_PUPDATE = 1, PRO_AXPY = 2 };
// Programmatic dependent launch (sm_90 and later): the solver chain's kernels
// are launched with programmatic stream serialization, so a kernel's CTAs may
// become resident while its predecessor's last CTAs still run.  Each such
// kernel calls pdl_trigger() (its own dependents may launch once all of its
// CTAs have started) and then pdl_wait(), which returns once the predecessor
// grid has completed and its memory operations are visible, before touching
// any global memory.  Both are no-ops for a kernel launched without the
// attribute.  The wait is the hardware's grid dependency, not a spin loop, and
// a predecessor never waits on its dependent.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#ifndef CISOR_PDL
#define CISOR_PDL 1
#endif
// launch kernel k with programmatic stream serialization (see pdl_wait)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = CISOR_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
}

// column shape code of the two-stage column kernels (P = 128, 256; P = 512 in 2D)
constexpr int COLS_TWO_STAGE = 16;
// shape code of the one-kernel pass by 8-CTA clusters (2D, P = 512, scalar fields; conv_cluster.cu)
constexpr int COLS_CLUSTER = 8;
cisor_status conv_fused_init();
bool conv_fused_ok(const cisor_ctx* c);
int conv_fused_pass(cisor_ctx* c, const ConvOp& op, int dk, cudaError_t* e);
// EPI_MATVEC: out = src - m .* conv ; EPI_RESID: out = aux - (src - m .* conv);
// EPI_CONV_ADD: out = conv + aux (aux may be null)
enum { EPI_MATVEC = 0, EPI_RESID = 1, EPI_CONV_ADD = 2 };
cisor_status conv_pass(cisor_ctx* c, const ConvOp& op);
cisor_status conv_init(int P);
int conv_rows_per_block(int P);
// Fills nrows, rslab, rtstride and nblk from dim, n, P.
void conv_geometry(cisor_ctx* c);
long long conv_scratch_elems(int dim, int n, int P);  // R elements per transmitter
int conv_kernels_per_pass(int dim);

// solver.cu
cisor_status solve_batch(cisor_ctx* c, int adjoint, const float2* f, const float2* b, float2* x,
                         int ntx, double tol, int max_iter, int* iters_max, double* iters_mean,
                         double* resid_max, int* n_bad);

struct SolveStat {
  int iters_max, n_bad;
  double iters_mean, resid_max;
  cisor_status status;
};
// Graph cache and streams of a multi-problem solve (owned by a cisor_batch).
struct MultiSolve {
  cudaStream_t main;
  cudaEvent_t fork;
  cudaEvent_t* join;            // [np]
  cudaGraphExec_t graph[2];     // forward / adjoint chunk graphs (host-driven loop)
  cudaGraphExec_t wgraph[2];    // forward / adjoint whole-solve graphs (device-side WHILE loop)
  long long* kernels[2];        // [np] kernels per problem in one replay
  struct cisor_loop_item* items;  // device [np]: every problem's active flags
  int* loop_count;              // device
  int* h_loop_count;            // pinned
  int use_while;
};
cisor_status solve_multi(cisor_ctx* const* cs, int np, int adjoint, const float2* const* b, double tol, int max_iter,
                         MultiSolve& ms, SolveStat* st);

// vector.cu: the vectorial model (appendix).  Matvec over [ntx, 3, N] fields:
// A x = x - C - D C / k^2 (C = conv_G(f x)) or A^H x = x - conj(f) conv_{G^H}(x + D x / k^2),
// with the epilogue (MATVEC / RESID, dot slots) of a ConvOp; partials land in
// [T][3 nblk][DOT_SLOTS].
struct VecOp {
  int adjoint, epilogue;  // EPI_MATVEC or EPI_RESID
  const float2* x;        // input (and the x of A x)
  const float2* aux;      // b of EPI_RESID, dot operand
  float2* out;
  float2* out2;
  int dot_a[DOT_SLOTS], dot_b[DOT_SLOTS];
  const int* active;
  int ntx;
};
cisor_status vec_matvec(cisor_ctx* c, const VecOp& op);
cisor_status vec_pupdate(cisor_ctx* c, int ntx);   // p = r + beta (p - omega v), per transmitter
cisor_status vec_axpy(cisor_ctx* c, int ntx);      // s = r - alpha v
cisor_status vec_gz(cisor_ctx* c);                 // gz = z + conv_{G^H}(v + D v / k^2)
cisor_status vec_tables(cisor_ctx* c, const double* d_tx, const double* d_rx);  // H~, E_in

// sense.cu
int sense_tiles(int M, int T);  // CTA tiles of the forward sensing GEMM (before split-K)
cisor_status sense_forward(cisor_ctx* c, const float2* f, const float2* u, float2* Y, int ntx);
cisor_status residual_and_D(cisor_ctx* c, const float2* f, const float2* u, const float2* y, float2* Z, float2* w,
                            int ntx);
cisor_status sense_adjoint(cisor_ctx* c, const float2* f, const float2* w, float2* z, float2* b, int ntx);
// tensor-core sensing GEMMs (sense_tc.cu): available when sense_tc_ok; sense_tc_prepare builds Ht from H
bool sense_tc_ok(const cisor_ctx* c);
int sense_tc_splits(const cisor_ctx* c, long long* KS);
cisor_status sense_tc_setup(cisor_ctx* c);
cisor_status sense_tc_prepare(cisor_ctx* c);
cisor_status sense_tc_forward(cisor_ctx* c, const float2* f, const float2* u, int ntx, int* splits);
cisor_status sense_tc_adjoint(cisor_ctx* c, const float2* f, const float2* w, float2* z, float2* b, int ntx);
cisor_status sense_tc_check(cisor_ctx* c, bool synced);
cisor_status grad_assemble(cisor_ctx* c, const float2* u, const float2* gz, const float2* s, double gamma,
                           float2* grad, float2* zstep, int ntx);
cisor_status gradient_step(cisor_ctx* c, const float2* s, const float2* g, double gamma, float2* z);

// tv.cu
cisor_status tv_prox(cisor_ctx* c, const float2* z, float2* x, double lam, int iters, double lo, double hi,
                     double lo_im, double hi_im, int complex_f, const float2* f_prev, double beta_mom,
                     float2* s_out);
cisor_status tv_prox_aniso(cisor_ctx* c, const float2* z, float2* x, double lam, int iters, double lo, double hi,
                           double lo_im, double hi_im, int complex_f, const float2* f_prev, double beta_mom,
                           float2* s_out);

}  // namespace cisor
