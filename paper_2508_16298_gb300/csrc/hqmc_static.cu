// M^dagger M apply for callers that cannot allocate device memory.
//
// hqmc_apply_MdagM needs a config, and hqmc_make_config allocates the config's
// workspace with cudaMalloc.  Some callers cannot do that: code that runs while
// another component owns the device allocator (a memory pool that must not be
// bypassed, or a budget that is already fully handed out), plug-ins that are
// only given device pointers, or code that must not synchronise the device the
// way cudaMalloc and cudaFree may.  hqmc_apply_MdagM_static serves them: the
// only scratch the fused apply needs, the FP64 link table of the gauge field,
// lives in a fixed file-scope device array, so the call allocates nothing.
//
// Limits and sharing (also stated in include/hqmc.h):
//   * at most kStaticMaxSites = 262144 lattice sites (Ntau * L * L), which
//     sizes the array at 8 MiB; every device that loads the library holds that
//     array until the process exits;
//   * the link table is rebuilt completely by every call before it is read, so
//     nothing has to start at zero, but every call on a device shares the one
//     array: calls whose executions overlap on the GPU (different streams, no
//     ordering between them) race and give wrong results.  Order them on one
//     stream, or with events;
//   * the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make
//     that first call before any stream capture on the device.
#include <cmath>
#include <mutex>

#include "hqmc.h"
#include "kernels.h"

using namespace hqmc;

namespace {

constexpr long long kStaticMaxSites = 262144;
constexpr int kStaticMaxDevices = 64;

// Two complex-double links per site: 32 bytes x 262144 sites = 8 MiB.
static __device__ __align__(256) double2 g_static_links[2 * kStaticMaxSites];

std::mutex g_static_mutex;
double2* g_static_links_dev[kStaticMaxDevices] = {};  // device address per device, once looked up
size_t g_static_smem_set[kStaticMaxDevices] = {};     // largest dynamic shared memory opted into
int g_static_major[kStaticMaxDevices] = {};           // compute capability major, once queried (0: not yet)

}  // namespace

extern "C" int hqmc_apply_MdagM_static(const hqmc_params* p, const double* theta, const void* x, void* y,
                                       void* stream) {
  if (!p || !theta || !x || !y) return HQMC_EINVAL;
  if (((uintptr_t)theta | (uintptr_t)x | (uintptr_t)y) & 15u) return HQMC_EINVAL;
  if (p->L < 4 || (p->L & 1) || p->L > 68 || p->Ntau < 2 || !(p->dtau > 0)) return HQMC_EINVAL;
  // the link factors are tanh and cosh of dtau * t: a non-finite or non-positive
  // product would give NaN or a non-physical operator without any other error
  if (!std::isfinite(p->dtau) || !std::isfinite(p->t) || !(p->dtau * p->t > 0.0)) return HQMC_EINVAL;
  const long long n = (long long)p->L * p->L * p->Ntau;
  if (n > kStaticMaxSites) return HQMC_EUNSUPPORTED;  // beyond the fixed scratch array
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  if (xb < yb + 16 * n && yb < xb + 16 * n) return HQMC_EINVAL;  // x and y overlap

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return HQMC_ECUDA;

  const int L = p->L, V = L * L;
  Geo g{L, V, L / 2, p->Ntau};
  const int bonds = V / 2;
  const int rounds = (bonds + 1023) / 1024;
  int threads = ((bonds + rounds - 1) / rounds + 31) / 32 * 32;
  if (threads < 64) threads = 64;
  // generic fused kernel, links re-read from the table, one slice per cluster
  SliceLaunch sl{g, threads, 1, p->Ntau, 0, 0};
  const size_t smem = (size_t)3 * V * sizeof(double2);

  double2* links = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_major[dev]) {
      int major = 0;
      if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) {
        cudaGetLastError();
        return HQMC_ECUDA;
      }
      g_static_major[dev] = major;
    }
    if (g_static_major[dev] != 10) return HQMC_EUNSUPPORTED;  // the kernels are built for sm_103a only
    if (!g_static_links_dev[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_static_links) != cudaSuccess || !addr) {
        cudaGetLastError();
        return HQMC_ECUDA;
      }
      g_static_links_dev[dev] = (double2*)addr;
    }
    if (smem > g_static_smem_set[dev]) {
      if (prepare_mdagm<double, MODE_APPLY>(sl) != cudaSuccess) {
        cudaGetLastError();
        return HQMC_ECUDA;
      }
      g_static_smem_set[dev] = smem;
    }
    links = g_static_links_dev[dev];
  }

  const double a = p->dtau * p->t;
  cudaStream_t s = (cudaStream_t)stream;
  if (launch_links(g, theta, std::tanh(a), std::tanh(a / 2), links, nullptr, nullptr, s) != cudaSuccess)
    return HQMC_ECUDA;
  MdagmArgs<double> args{};
  args.g = g;
  args.cB = std::cosh(a) * std::pow(std::cosh(a / 2), 6);
  args.U = links;
  args.x = (const double2*)x;
  args.y = (double2*)y;
  if (launch_mdagm<double, MODE_APPLY>(sl, args, s) != cudaSuccess) return HQMC_ECUDA;
  return HQMC_OK;
}
