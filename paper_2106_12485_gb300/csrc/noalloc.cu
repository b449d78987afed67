// noalloc.cu -- field energies computed without allocating any device memory.
//
// Some callers cannot allocate device memory at the moment they want this
// diagnostic: real-time loops that must never stall on an allocator, and
// host applications that give this library a fixed memory budget or their
// own pool and forbid it to grow.  zpic_field_energy_noalloc_f32 serves
// them: it runs the same reduction as zpic_field_energy, on device arrays
// the caller already owns, and keeps its scratch space in an array compiled
// into the library.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/zpic.h"
#include "zpic_kernels.h"

namespace zp {
int set_last_error(int code, const char *msg);  // zpic_api.cu
}

namespace {

// Rows the built-in scratch can take: two partial sums per row plus the two
// results, 2 * 65536 + 2 doubles (1 MiB + 16 bytes).  Every GPU that loads
// the library holds this array until the process exits.
constexpr int kMaxRows = 65536;
static __device__ __align__(256) double g_energy_scratch[2 * kMaxRows + 2];

// Device address of g_energy_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up with the
// device current and cached here, together with the id of the context it
// belongs to: after cudaDeviceReset (or when the host makes another context
// current on the device) the array lives at a new address, and the lookup
// runs again.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  double *p = nullptr;
  unsigned long long ctx_id = 0;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Id of the calling thread's current context (0 when none is current yet),
// through the driver entry points the runtime hands out (no link against
// the driver library).
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000,
                                         cudaEnableDefault, &qa) ==
            cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000,
                                         cudaEnableDefault, &qb) ==
            cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      get_current = (GetCurrent)a;
      get_id = (GetId)b;
    }
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_for_current_device(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return zp::set_last_error(ZPIC_ECUDA, "no CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return zp::set_last_error(ZPIC_ENOTSUP, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchAddr &a = g_scratch_addr[dev];
  const unsigned long long ctx = current_context_id();
  if (!a.p || ctx == 0 || ctx != a.ctx_id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return zp::set_last_error(
          ZPIC_ECUDA, "cudaGetSymbolAddress of the built-in scratch failed");
    }
    a.p = (double *)p;
    a.ctx_id = current_context_id();  // current now, if it was not before
  }
  *out = a.p;
  return ZPIC_OK;
}

}  // namespace

extern "C" int zpic_field_energy_noalloc_f32(
    const float *ex, const float *ey, const float *ez, const float *bx,
    const float *by, const float *bz, int nx, int ny, int ld, double dx,
    double dy, double *out, void *stream) {
  if (!ex || !ey || !ez || !bx || !by || !bz || !out)
    return zp::set_last_error(ZPIC_EINVAL, "NULL field or output pointer");
  if (nx < 1 || ny < 1 || ld < nx)
    return zp::set_last_error(ZPIC_EINVAL, "need nx >= 1, ny >= 1, ld >= nx");
  if (ny > kMaxRows)
    return zp::set_last_error(
        ZPIC_EINVAL, "ny exceeds the 65536 rows of the built-in scratch");
  if (!(dx > 0) || !(dy > 0))
    return zp::set_last_error(ZPIC_EINVAL, "dx and dy must be positive");
  double *scratch = nullptr;
  int r = scratch_for_current_device(&scratch);
  if (r != ZPIC_OK) return r;
  zp::FieldPtrs<float> f;
  f.e[0] = ex;
  f.e[1] = ey;
  f.e[2] = ez;
  f.b[0] = bx;
  f.b[1] = by;
  f.b[2] = bz;
  cudaStream_t s = (cudaStream_t)stream;
  // every scratch value is written before it is read: nothing to clear
  cudaError_t e = zp::launch_field_energy<float>(f, nx, ny, ld, dx, dy,
                                                 scratch, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + 2 * (size_t)ny, 2 * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return zp::set_last_error(ZPIC_ECUDA, cudaGetErrorString(e));
  }
  return ZPIC_OK;
}
