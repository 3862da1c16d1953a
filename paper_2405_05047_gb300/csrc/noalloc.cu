// Allocation-free variant of the residual + restriction level operator.
//
// mg_apply(MG_OP_RESTRICT) keeps the intermediate residual r = b - A_l x in a
// buffer of the hierarchy's workspace.  mg_restrict_static computes the same
// d = R_l (b - A_l x) with r held in a fixed device array compiled into the
// library instead, so a call makes no allocation of any kind.  That serves
// callers that cannot allocate device memory: applications whose device memory
// is owned up front by another allocator or a fixed pool (they hand the
// library inputs and outputs, but have no allocation to give it for
// temporaries), and real-time loops that must not enter the CUDA allocator
// at all.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device.h"

namespace {

// Residual scratch shared by every call in the process, on every device that
// loads the library (each such device holds it until the process exits).
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 20;   // 8 MiB
__device__ __align__(256) double g_restrict_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a host-side stand-in for the symbol).
int scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (device < 0 || device >= kMaxDevices) return mgi::fail(MG_ERR_INVALID, "device index out of range");
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_restrict_scratch);
    if (e != cudaSuccess) return mgi::fail(MG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return MG_OK;
}

}  // namespace

extern "C" int mg_restrict_static(mg_hier* h, int level, const void* x, const void* b, void* d, int prec) {
  using namespace mgi;
  if (!h || !x || !b || !d || level < 1 || level >= h->nlev) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  const int64_t rows = h->L[level].n * h->nc;
  const int64_t cap = prec == MG_FP64 ? kStaticScratchDoubles : 2 * kStaticScratchDoubles;
  if (rows > cap)
    return fail(MG_ERR_INVALID, "level has " + std::to_string(rows) + " dofs; the static residual scratch holds " +
                                    std::to_string(cap) + " at this precision");
  if (cudaSetDevice(h->ctx->device) != cudaSuccess) return fail(MG_ERR_CUDA, "cudaSetDevice");
  void* scratch = nullptr;
  if ((rc = scratch_address(h->ctx->device, &scratch))) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  const LevelMats& L = h->L[level];
  const int nc = h->nc;
  // the residual is written in full before it is read: nothing to clear
  if (prec == MG_FP64) {
    launch_residual<double>(L.A64.v, nc, (const double*)x, (const double*)b, (double*)scratch, nullptr, s);
    launch_restrict<double>(L.R.t, nc, (const double*)scratch, (double*)d, nullptr, nullptr, 0.0, nullptr, s);
  } else {
    launch_residual<float>(prec == MG_MIXED_BF16 ? L.A16.v : L.A32.v, nc, (const float*)x, (const float*)b,
                           (float*)scratch, nullptr, s);
    launch_restrict<float>(L.R.t, nc, (const float*)scratch, (float*)d, nullptr, nullptr, 0.0, nullptr, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
  return MG_OK;
}
