// Device side of the fused epilogues declared in fused.h: the update applied to an operator
// output v at entry i (node `node`) by the node pass.
#pragma once

#include "fused.h"

namespace wb {

template <typename T>
__device__ inline void epi_apply(const Epi<T>& E, size_t i, int node, T v) {
  switch (E.mode) {
    case EPI_STORE: E.y[i] = v; break;
    case EPI_SCALE: E.y[i] = v * E.sc[node]; break;
    case EPI_DINV: E.y[i] = E.dinv[i] * v; break;
    case EPI_BMINUS: E.y[i] = E.b[i] - v; break;
    case EPI_SUB: E.r[i] -= v; break;
    case EPI_CHEB_INIT1: {
      const T rv = E.b[i] - v;
      const T dv = E.dinv[i] * rv * E.inv_theta;
      E.r[i] = rv;
      E.d[i] = dv;
      E.x[i] += dv;
    } break;
    case EPI_CHEB_STEP: {
      const T rv = E.r[i] - v;
      const T dv = E.a * E.d[i] + E.bc * (E.dinv[i] * rv);
      E.r[i] = rv;
      E.d[i] = dv;
      E.x[i] += dv;
    } break;
    default: break;
  }
}

}  // namespace wb
