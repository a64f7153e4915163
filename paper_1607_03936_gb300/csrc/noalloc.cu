// A context-free, allocation-free form of the weighted pressure-Poisson apply
// y = B C^-1 B^T p, for callers that cannot allocate device memory: code that
// runs inside another framework's memory pool or allocator hooks, embedded or
// real-time hosts that forbid cudaMalloc after start-up (it can synchronise the
// device and fragments memory), and library code that may only touch
// caller-provided buffers.  Every temporary lives in file-scope __device__
// arrays that each GPU loading this library holds until the process exits.
#include <mutex>

#include "kernels.h"
#include "wbfbt.h"

namespace {

constexpr int kMaxNodes = WBFBT_NOALLOC_MAX_NODES;

// [0, n): C^-1 per node (0 on Dirichlet nodes); [n, 4n): B^T p, component-major.
static __device__ __align__(256) double g_noalloc_scratch[4 * (size_t)kMaxNodes];
// reference tables for k = 2, 3, 4
static __device__ __align__(256) RefTables g_noalloc_tabs[3];

struct DeviceSlot {
  bool ready = false;
  double* scratch = nullptr;   // device address of g_noalloc_scratch on this device
  RefTables* tabs = nullptr;   // device address of g_noalloc_tabs on this device
};

std::mutex g_mutex;
DeviceSlot g_slots[64];

// Once per device, with that device current: resolve the device addresses of the static
// arrays (host code cannot use the symbols as pointers) and fill the reference tables.
int ensure_slot(DeviceSlot** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WBFBT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return WBFBT_ERR_CUDA;
    s.scratch = static_cast<double*>(p);
    if (cudaGetSymbolAddress(&p, g_noalloc_tabs) != cudaSuccess) return WBFBT_ERR_CUDA;
    s.tabs = static_cast<RefTables*>(p);
    RefTables t[3];
    for (int k = 2; k <= 4; ++k)
      if (!build_ref_tables(k, &t[k - 2])) return WBFBT_ERR_INVALID;
    if (cudaMemcpyToSymbol(g_noalloc_tabs, t, sizeof(t)) != cudaSuccess) return WBFBT_ERR_CUDA;
    s.ready = true;
  }
  *out = &s;
  return WBFBT_OK;
}

__global__ void k_invert_interior(Grid g, double* __restrict__ c) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  c[n] = on_boundary(g, ix, iy, iz) ? 0.0 : 1.0 / c[n];
}

}  // namespace

extern "C" int wbfbt_apply_Kw_noalloc(const wbfbt_mesh* mesh, int k, const double* mu_nodes, double a,
                                      const double* p, double* y, void* stream) {
  if (!mesh || !mu_nodes || !p || !y || k < 2 || k > 4 || !(a >= 1.0)) return WBFBT_ERR_INVALID;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->lx > 0) || !(mesh->ly > 0) || !(mesh->lz > 0))
    return WBFBT_ERR_INVALID;
  // node counts per axis in 64-bit arithmetic: each must fit the static scratch on its own
  // before the product is formed, so no multiplication below can overflow
  const long long NX = (long long)k * mesh->nx + 1, NY = (long long)k * mesh->ny + 1, NZ = (long long)k * mesh->nz + 1;
  if (NX > kMaxNodes || NY > kMaxNodes || NZ > kMaxNodes) return WBFBT_ERR_INVALID;
  const long long nn = NX * NY * NZ;
  if (nn > kMaxNodes) return WBFBT_ERR_INVALID;   // beyond the static scratch
  DeviceSlot* slot = nullptr;
  int st = ensure_slot(&slot);
  if (st != WBFBT_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Grid g = make_grid(mesh->nx, mesh->ny, mesh->nz, k, mesh->lx, mesh->ly, mesh->lz);
  const RefTables* tab = slot->tabs + (k - 2);
  double* cinv = slot->scratch;
  double* bt = slot->scratch + nn;
  // C = M~_u(a sqrt(mu)) per node, then its inverse with zeros on the Dirichlet nodes
  if (launch_lumped_weight(g, k, tab, mu_nodes, a, cinv, s) != cudaSuccess) return WBFBT_ERR_CUDA;
  wb_launch(k_invert_interior, (unsigned)((nn + 255) / 256), 256, 0, s, g, cinv);
  // B^T p into the scratch velocity (the launcher zeroes it first), then B (C^-1 .)
  if (launch_stokes<double>(g, k, tab, OP_BT, nullptr, nullptr, p, nullptr, 0, bt, nullptr, s) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  if (launch_stokes<double>(g, k, tab, OP_B, bt, cinv, nullptr, nullptr, 0, nullptr, y, s) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
}
