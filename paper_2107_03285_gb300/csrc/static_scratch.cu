// sgn_assemble_static: sgn_assemble with its per-element scratch in a
// file-scope device array instead of the caller's bound buffer.
//
// Who needs this: code that may not allocate device memory at the point where
// it assembles, e.g. a solver loop inside a real-time or memory-capped
// service whose allocator is frozen after start-up, or a host that has handed
// all device memory to another runtime.  The array below is a fixed part of
// the library's device image: every GPU that loads libsgn.so holds it (16 MB)
// until the process exits.  Under CUDA's lazy module loading the array's
// memory is taken when the module is first used; sgn_bind resolves the
// array's address (static_scratch_bind below), so that happens at bind time,
// where the caller provides memory anyway, and never inside an assembly.
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

namespace sgn {

// Called by sgn_bind with the handle's device current: looks up (once per
// device) the device address of the array.  Host code must never use the
// symbol itself as a pointer: on the host it names a stand-in object.
cudaError_t static_scratch_bind(int device) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[device]) return cudaSuccess;
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_assemble_scratch);
  if (e != cudaSuccess) return e;
  if (!ptr) return cudaErrorInvalidSymbol;
  g_scratch_ptr[device] = static_cast<double *>(ptr);
  return cudaSuccess;
}

}  // namespace sgn

extern "C" sgn_status sgn_assemble_static(sgn_t h, const double *x_d, const double *p_d) {
  if (!h || !x_d || !p_d) {
    sgn::set_error(nullptr, "sgn_assemble_static: null argument");
    return SGN_EINVAL;
  }
  sgn::Ctx &c = *h;
  if (!c.bound || !c.have_objective) return SGN_ESTATE;
  const int64_t need = (int64_t)(3 + (c.S.dim + 1) * c.S.dim) * c.S.n_elem;
  if (need > kStaticScratchDoubles) {
    sgn::set_error(&c, "sgn_assemble_static: the mesh needs more element scratch than the 16 MB static array "
                       "((3 + (dim+1) dim) n_elem must be <= 2^21 doubles)");
    return SGN_EINVAL;
  }
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    scratch = (c.device >= 0 && c.device < kMaxDevices) ? g_scratch_ptr[c.device] : nullptr;
  }
  if (!scratch) {  // sgn_bind resolves it; without that the handle is not usable here
    sgn::set_error(&c, "sgn_assemble_static: the static array's address was not resolved at sgn_bind");
    return SGN_ESTATE;
  }
  // the element state is written for every element before it is read, so
  // nothing in the array needs clearing between calls
  {
    sgn::ProfScope ps(c, SGN_PROF_ELEMENTS);
    sgn::launch_elem_state_into(c, x_d, p_d, scratch);
    sgn::launch_slot_gather_from(c, scratch);
  }
  {
    sgn::ProfScope ps(c, SGN_PROF_VECTOR);
    sgn::launch_objective_terms(c, x_d, p_d);
  }
  c.assembled = true;
  c.kkt64.factored = c.kkt32.factored = c.kf.factored = c.kf32.factored = false;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sgn::set_error(&c, std::string("sgn_assemble_static: kernel launch: ") + cudaGetErrorString(e));
    return SGN_ECUDA;
  }
  return SGN_OK;
}
