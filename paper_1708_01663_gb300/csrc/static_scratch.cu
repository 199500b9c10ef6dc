// Batched matvec y = A x (or A^H x) that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host
// framework that owns every device allocation (a custom allocator, a
// sandboxed plug-in, a runtime that forbids allocation after start-up), or
// code that must not allocate while a CUDA graph is being captured.  For
// them this entry point runs the same three FFT-convolution kernels as
// cisor_apply_A, with its scratch in the file-scope array below instead of
// context-owned memory: the two stage-twiddle tables (2 x 512 complex64)
// followed by the row-FFT intermediate [nvec, n, P] complex64.  Every GPU
// that loads the library holds this array until the process exits.
#include <mutex>

#include "common.cuh"

namespace cisor {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kStaticTwiddleFloats2 = 2 * 512;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices];  // device address of g_static_scratch, per device

// Device address of the scratch array on the current device, looked up once
// per device; the same first call raises the convolution kernels' dynamic
// shared-memory limits for every supported FFT size.  A stream of another
// device is rejected: the address and the kernel attributes are per device.
static cisor_status static_scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  CISOR_CUDA(cudaGetDevice(&dev));
  if (stream) {
    int sdev = -1;
    CISOR_CUDA(cudaStreamGetDevice(stream, &sdev));
    if (sdev != dev) {
      set_error("cisor_apply_A_static: the stream belongs to device %d but device %d is current", sdev, dev);
      return CISOR_ERR_INVALID_ARG;
    }
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d outside the %d devices this entry point supports", dev, kMaxDevices);
    return CISOR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    CISOR_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    for (int P = 64; P <= 512; P *= 2) CISOR_TRY(conv_init(P));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return CISOR_OK;
}

}  // namespace cisor

using namespace cisor;

extern "C" cisor_status cisor_apply_A_static(const void* ghat_scaled, const void* f, const void* x, void* y, int n,
                                             int P, int nvec, int adjoint, void* stream) {
  if (!ghat_scaled || !f || !x || !y) {
    set_error("cisor_apply_A_static: NULL argument");
    return CISOR_ERR_INVALID_ARG;
  }
  if (n < 8 || n > 256 || (P & (P - 1)) != 0 || P < 64 || P > 512 || P < 2 * n - 1 || nvec < 1) {
    set_error("cisor_apply_A_static: unsupported sizes (n %d, P %d, nvec %d)", n, P, nvec);
    return CISOR_ERR_INVALID_ARG;
  }
  const size_t need = sizeof(float2) * ((size_t)kStaticTwiddleFloats2 + (size_t)nvec * n * P);
  if (need > kStaticScratchBytes) {
    set_error("cisor_apply_A_static: %zu bytes of scratch needed (nvec %d x n %d x P %d), the maximum is %zu",
              need, nvec, n, P, kStaticScratchBytes);
    return CISOR_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  CISOR_TRY(static_scratch_address((cudaStream_t)stream, &base));
  // Host-side descriptor of the launch; nothing in it is allocated.
  cisor_ctx c{};
  c.n = n;
  c.P = P;
  c.N = (long long)n * n;
  c.T = nvec;
  c.stream = (cudaStream_t)stream;
  c.twst = reinterpret_cast<float2*>(base);
  c.R = reinterpret_cast<float2*>(base) + kStaticTwiddleFloats2;
  c.ghat = reinterpret_cast<float2*>(const_cast<void*>(ghat_scaled));
  c.dim = 2;
  c.ncomp = 1;
  c.Nf = c.N;
  c.cols_nt = 512;
  conv_geometry(&c);
  CISOR_TRY(make_stage_twiddles(&c));
  ConvOp op{};
  op.adjoint = adjoint ? 1 : 0;
  op.mul_f = 1;
  op.prologue = PRO_COPY;
  op.src = reinterpret_cast<const float2*>(x);
  op.epilogue = EPI_MATVEC;
  op.esrc = reinterpret_cast<const float2*>(x);
  op.out = reinterpret_cast<float2*>(y);
  op.f = reinterpret_cast<const float2*>(f);
  op.ntx = nvec;
  return conv_pass(&c, op);
}
