// Shared device-side definitions: mesh geometry, index maps, error checks.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <utility>

#include "tables.h"

// Structured brick of nx x ny x nz affine hexahedra carrying Q_k nodes.
struct Grid {
  int nx, ny, nz;       // elements per axis
  int NX, NY, NZ;       // nodes per axis, k * n + 1
  int nn;               // nodes
  int ne;               // elements
  double h[3];          // element sizes
  double s[3];          // 2 / h: reference-to-physical derivative scale per axis
  double detJ;          // hx hy hz / 8
  int rowk;             // 1: k = 2 element passes use the row-segment kernels
  int kern;             // the element-kernel option (0 automatic, 1 per point, 2 per element)
};

inline Grid make_grid(int nx, int ny, int nz, int k, double lx, double ly, double lz) {
  Grid g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.NX = k * nx + 1; g.NY = k * ny + 1; g.NZ = k * nz + 1;
  g.nn = g.NX * g.NY * g.NZ;
  g.ne = nx * ny * nz;
  g.h[0] = lx / nx; g.h[1] = ly / ny; g.h[2] = lz / nz;
  g.s[0] = 2.0 / g.h[0]; g.s[1] = 2.0 / g.h[1]; g.s[2] = 2.0 / g.h[2];
  g.detJ = g.h[0] * g.h[1] * g.h[2] / 8.0;
  g.rowk = 0;
  g.kern = 0;
  return g;
}

__host__ __device__ inline bool on_boundary(const Grid& g, int ix, int iy, int iz) {
  return ix == 0 || iy == 0 || iz == 0 || ix == g.NX - 1 || iy == g.NY - 1 || iz == g.NZ - 1;
}

// Elements of one of the 8 parity colours (ex % 2, ey % 2, ez % 2) = (c & 1, (c >> 1) & 1, c >> 2).
// Two elements of the same colour share no node, so scatter-adds within one colour never collide.
__host__ __device__ inline int colour_count(const Grid& g, int c) {
  int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
  return ((g.nx - cx + 1) / 2) * ((g.ny - cy + 1) / 2) * ((g.nz - cz + 1) / 2);
}

__device__ inline void colour_element(const Grid& g, int c, int t, int& ex, int& ey, int& ez) {
  if (c < 0) {
    ex = t % g.nx; t /= g.nx; ey = t % g.ny; ez = t / g.ny;
    return;
  }
  int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
  int ncx = (g.nx - cx + 1) / 2, ncy = (g.ny - cy + 1) / 2;
  int ix = t % ncx; t /= ncx;
  int iy = t % ncy; int iz = t / ncy;
  ex = 2 * ix + cx; ey = 2 * iy + cy; ez = 2 * iz + cz;
}

// Process-wide count of kernel launches issued by this library (one shared instance:
// inline-function statics are merged across translation units).
inline std::atomic<long long>& wb_launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}
inline void wb_count_launch() { wb_launch_counter().fetch_add(1, std::memory_order_relaxed); }

// Programmatic dependent launch.  Every kernel of this library is launched by wb_launch with
// programmatic stream serialisation, so the next kernel of a stream is set up while the current
// one drains (its blocks are released as the current kernel's blocks exit), and pdl_entry() is
// the first statement of every kernel: it waits until the previous grid has completed with its
// memory visible.  Ordering is therefore exactly that of plain stream launches; only launch
// latency overlaps.  (Releasing the next grid at kernel entry instead measured slower: its
// waiting blocks hold registers and shared memory during long kernels.)
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t wb_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  wb_count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define WB_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return WBFBT_ERR_CUDA;          \
  } while (0)
