// fcm_cell_apply_noalloc: y = sum_c P_c^T K_c P_c x from caller-owned cell
// matrices, without allocating device memory.
//
// Who needs this: host applications that own the whole device heap and do
// not allow allocation once they run (solver services that carve a fixed
// arena at start-up, real-time loops that must never enter the allocator's
// synchronising paths, plug-ins living inside another framework's memory
// pool).  They cannot call fcm_setup, which allocates the hierarchy, but
// they can hold cell matrices and vectors in their own memory.  The apply
// kernels need one scratch buffer (the per-cell products that the DOF
// gather sums, plus the list of cell ids); here it is a fixed array compiled
// into the library instead of a cudaMalloc.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes (4 MiB).
// Every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress while that
// device is current and caches it; make that first call before any stream
// capture.  The cached address belongs to the device's current context: after
// the host application calls cudaDeviceReset the module is loaded again and
// the cache is stale, so this entry point must not be used across a device
// reset.  Every call synchronizes its stream before it returns.  All calls on
// a device share the array: calls whose kernels overlap on the GPU (for
// example on two streams) race on it.  Each call writes every scratch entry
// it reads before reading it, so nothing needs to start at zero.
#include <mutex>

#include "fcm_internal.h"

namespace {

constexpr long long kNoAllocBytes = 4LL << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void iota_kernel(int* ids, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    ids[i] = i;
}

}  // namespace

extern "C" fcm_status fcm_cell_apply_noalloc(int dim, const int* cells, int p, const double* K_dev,
                                             const double* x_dev, double* y_dev, void* stream) {
  if (!cells || !K_dev || !x_dev || !y_dev || dim < 2 || dim > 3 || p < 1 || p > fcm::kMaxP) {
    fcm::set_last_error("fcm_cell_apply_noalloc: invalid argument");
    return FCM_E_INVALID;
  }
  int C[3] = {1, 1, 1};
  long long ncells = 1;
  for (int a = 0; a < dim; ++a) {
    if (cells[a] < 1 || cells[a] > 4096) {
      fcm::set_last_error("fcm_cell_apply_noalloc: cells per axis must be in [1, 4096]");
      return FCM_E_INVALID;
    }
    C[a] = cells[a];
    ncells *= cells[a];
  }
  if (ncells * 8 > kNoAllocBytes) {
    fcm::set_last_error(
        "fcm_cell_apply_noalloc: cells x (p+1)^d too large for the 4 MiB scratch array "
        "(at most about 520,000 per-cell products)");
    return FCM_E_INVALID;
  }
  fcm::LevelGeom g = fcm::make_geom(dim, 1, p, C);
  if (g.nloc > 128) {
    fcm::set_last_error("fcm_cell_apply_noalloc: (p+1)^d must be <= 128");
    return FCM_E_INVALID;
  }
  const long long id_bytes = ((long long)g.ncells * (long long)sizeof(int) + 255) / 256 * 256;
  const long long need = id_bytes + (long long)g.ncells * g.nloc * (long long)sizeof(double);
  if (need > kNoAllocBytes) {
    fcm::set_last_error(
        "fcm_cell_apply_noalloc: cells x (p+1)^d too large for the 4 MiB scratch array "
        "(at most about 520,000 per-cell products)");
    return FCM_E_INVALID;
  }
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    fcm::set_last_error(cudaGetErrorString(e));
    return FCM_E_CUDA;
  }
  int* ids = reinterpret_cast<int*>(base);
  double* Y = reinterpret_cast<double*>(base + id_bytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int blocks = (g.ncells + 255) / 256;
  iota_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(ids, g.ncells);
  fcm::OpData<double> op;
  op.ld = g.nloc;  // caller matrices are unpadded n x n
  op.own.n = g.ncells;
  op.own.cells = ids;
  op.own.mats = const_cast<double*>(K_dev);
  fcm::launch_cell_op<double>(g, op, x_dev, Y, s);
  fcm::launch_gather<double>(g, fcm::GATHER_SET, Y, nullptr, y_dev, 1.0, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  // The streaming kernel (stored matrices with more than 16 rows) bounds its
  // waits on bulk copies; an expired wait leaves stale products in y.
  int timed_out = 0;
  if (e == cudaSuccess) e = fcm::read_and_clear_timeout(&timed_out, s);
  if (e != cudaSuccess) {
    fcm::set_last_error(cudaGetErrorString(e));
    return FCM_E_CUDA;
  }
  if (timed_out) {
    fcm::set_last_error("fcm_cell_apply_noalloc: a bounded device wait on a bulk copy expired");
    return FCM_E_TIMEOUT;
  }
  return FCM_OK;
}
