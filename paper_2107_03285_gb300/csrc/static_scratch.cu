// sgn_assemble_static: sgn_assemble with its per-element scratch in a
// file-scope device array instead of the caller's bound buffer.
//
// Who needs this: code that may not allocate device memory at the point where
// it assembles, e.g. a solver loop inside a real-time or memory-capped
// service whose allocator is frozen, or a host that has handed all device
// memory to another runtime, and that would rather not size or keep the
// element-state part of the workspace itself.  The array below is a fixed
// part of the library image: every GPU that loads libsgn.so holds it (16 MB)
// until the process exits.
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace {

// element state: (3 + (d+1) d) doubles per element, at most 15 (tetrahedra)
constexpr int64_t kStaticScratchDoubles = 2 * 1024 * 1024;  // 16 MB
static __device__ __align__(256) double g_assemble_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" sgn_status sgn_assemble_static(sgn_t h, const double *x_d, const double *p_d) {
  if (!h || !x_d || !p_d) return SGN_EINVAL;
  sgn::Ctx &c = *h;
  if (!c.bound || !c.have_objective) return SGN_ESTATE;
  const int64_t need = (int64_t)(3 + (c.S.dim + 1) * c.S.dim) * c.S.n_elem;
  if (need > kStaticScratchDoubles) {
    c.last_error = "sgn_assemble_static: mesh needs more element scratch than the 16 MB static array";
    return SGN_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SGN_ECUDA;
  double *scratch = nullptr;
  {
    // first call on this device (with it current): resolve the device address
    // of the array; host code must not use the symbol itself as a pointer
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_assemble_scratch);
      if (e != cudaSuccess || !ptr) {
        c.last_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return SGN_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<double *>(ptr);
    }
    scratch = g_scratch_ptr[dev];
  }
  // the element state is written for every element before it is read, so
  // nothing in the array needs clearing between calls
  sgn::launch_elem_state_into(c, x_d, p_d, scratch);
  sgn::launch_slot_gather_from(c, scratch);
  sgn::launch_objective_terms(c, x_d, p_d);
  c.assembled = true;
  c.kkt64.factored = c.kkt32.factored = c.kf.factored = c.kf32.factored = false;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c.last_error = std::string("kernel launch: ") + cudaGetErrorString(e);
    return SGN_ECUDA;
  }
  return SGN_OK;
}
