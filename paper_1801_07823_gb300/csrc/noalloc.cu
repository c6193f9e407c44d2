// sw_dslash_schur_noalloc: the Schur operator of sw_dslash (SW_OP_S) for
// callers that must not allocate device memory -- for instance a host
// application or framework that owns every device allocation and forbids
// others, or a real-time loop that may not call into the allocator.
// sw_dslash allocates its work buffers and the B^-1 table on first use; this
// entry point instead keeps all of its scratch in one file-scope device array
// of fixed size.
//
// Scratch layout for N = L0 L1 <= kNoAllocMaxSites (complex128 units):
//   [0, N)      input packed to parity-split order
//   [N, 2N)     output in parity-split order (odd half cleared every call)
//   [2N, 3N)    intermediate vectors of the Schur operator
//   [3N, 7N)    B^-1 table for the requested mass (rebuilt every call)
#include <cmath>
#include <mutex>
#include <string>

#include "sw_internal.h"

namespace {

constexpr long kNoAllocMaxSites = 65536;  // e.g. 256 x 256; 7.3 MB of device memory
static __device__ __align__(256) double2 g_noalloc_scratch[7 * kNoAllocMaxSites];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double2* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the name g_noalloc_scratch is only a host-side stand-in).
double2* noalloc_scratch(int device) {
  SW_REQUIRE(device >= 0 && device < kMaxDevices, SW_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    SW_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[device] = (double2*)p;
  }
  return g_noalloc_ptr[device];
}

}  // namespace

extern "C" int sw_dslash_schur_noalloc(sw_gauge* g, double mass, const void* in, void* out) {
  if (!g || !in || !out) return SW_ERR_ARG;
  sw_ctx* c = g->ctx;
  return guarded(c, [&] {
    SW_REQUIRE((long)g->N <= kNoAllocMaxSites, SW_ERR_SHAPE,
               "sw_dslash_schur_noalloc: lattice has " + std::to_string(g->N) +
                   " sites, the fixed scratch holds at most " +
                   std::to_string(kNoAllocMaxSites));
    SW_REQUIRE(std::isfinite(mass) && mass > 0.0, SW_ERR_ARG, "mass must be > 0");
    cudaStream_t s = c->stream;
    long N = g->N;
    double2* base = noalloc_scratch(c->device);
    double2* a = base;
    double2* b = base + N;
    double2* w = base + 2 * N;
    double2* binv = base + 3 * N;
    launch_binv_build(g, mass, binv, s);
    launch_pack(g, (const double2*)in, a, s);
    fine_apply_S(g, binv, a, b, w, s);
    SW_CUDA(cudaMemsetAsync(b + N / 2, 0, N / 2 * sizeof(double2), s));
    launch_unpack(g, b, (double2*)out, s);
    return SW_OK;
  });
}
