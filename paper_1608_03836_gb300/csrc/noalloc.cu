// wadg_energy_noalloc: the energy reduction without any allocation.
//
// Some callers cannot call cudaMalloc at the moment they need a diagnostic:
// code inside a framework whose caching allocator already owns the device
// memory budget (a cudaMalloc behind its back can fail or evict its cache),
// and real-time loops that must not block on the driver's allocator.  This
// entry point gives them the energy of a field without allocating: the
// per-column partial sums go to a fixed array in device memory that is part
// of the library image, instead of the scratch that wadg_set_operators
// allocates for wadg_energy.  Like wadg_energy, it returns the value on the
// host, so it synchronises the caller's stream before it returns.
#include <cmath>
#include <mutex>

#include "aux_kernels.h"
#include "wadg_internal.h"

namespace {

// Largest number of columns (elements x shots) one call can reduce.  The
// array holds one partial sum per column plus the total: 8 MiB + 8 bytes,
// resident on every GPU that loads the library until the process exits.
constexpr int64_t kMaxColumns = int64_t(1) << 20;

static __device__ __align__(256) double g_energy_scratch[kMaxColumns + 1];

// Host-side device addresses of g_energy_scratch, one per device, taken with
// that device current on the first call that uses it.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

int set_error(wadg_mesh* m, int status, const char* msg) {
  if (m) m->last_error = msg;
  return status;
}

}  // namespace

extern "C" int wadg_energy_noalloc(wadg_mesh* m, const void* Q, double* E, wadg_stream stream) {
  const int ready = wadg_mesh_ready(m);  // the same checks, status and message as wadg_energy
  if (ready != WADG_OK) return ready;
  if (!Q || !E) return set_error(m, WADG_EINVAL, "null pointer");
  const int64_t ncols = m->K * m->S;
  if (ncols > kMaxColumns)
    return set_error(m, WADG_EINVAL,
                     "wadg_energy_noalloc: K*S exceeds the 1048576 columns of its fixed scratch; use wadg_energy");
  if (m->device < 0 || m->device >= kMaxDevices) return set_error(m, WADG_EINVAL, "device index out of range");

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_error(m, WADG_ECUDA, "cudaGetDevice failed");
  if (prev != m->device && cudaSetDevice(m->device) != cudaSuccess)
    return set_error(m, WADG_ECUDA, "cudaSetDevice failed");
  auto restore = [&](int status) {
    if (prev != m->device) cudaSetDevice(prev);
    return status;
  };

  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[m->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
      if (e != cudaSuccess) {
        m->last_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return restore(WADG_ECUDA);
      }
      g_scratch_ptr[m->device] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[m->device];
  }

  // Same reduction kernels and operator tables as wadg_energy.  Every slot
  // read (partial sums 0..ncols-1 and the total at ncols) is written earlier
  // in the same call, so nothing needs clearing between calls.
  const wadg::RefOps& o = m->ref;
  const double* dVq = m->d_ref64;
  const double* dwq = dVq + 5 * (size_t)o.Nq * o.Np + (size_t)4 * 3 * o.Nfq * o.Np;
  double* partial = scratch;
  double* total = scratch + ncols;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = m->precision == WADG_FP64
                      ? wadg::launch_reduce<double>(0, ncols, m->S, o.Np, o.Nq, (const double*)Q, dVq, dwq, m->d_J,
                                                    m->d_c2, nullptr, 0, partial, total, s)
                      : wadg::launch_reduce<float>(0, ncols, m->S, o.Np, o.Nq, (const float*)Q, dVq, dwq, m->d_J,
                                                   m->d_c2, nullptr, 0, partial, total, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(E, total, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    m->last_error = std::string("wadg_energy_noalloc: ") + cudaGetErrorString(e);
    return restore(WADG_ECUDA);
  }
  if (!std::isfinite(*E)) return restore(set_error(m, WADG_EUNSTABLE, "energy is not finite"));
  return restore(WADG_OK);
}
