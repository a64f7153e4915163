// Device side of the fused epilogues declared in fused.h: the update applied to an operator
// output v at entry i (node `node`) by the node pass.
#pragma once

#include <type_traits>

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

// The same update split in two for a mode known at compile time: epi_pre loads the operands
// (so a kernel can issue them before the loads that form v), epi_post combines and stores.
// Arithmetic and its order are those of epi_apply.
template <typename T>
struct EpiOps {
  T a0, a1, a2, a3;
};

template <int MODE, typename T>
__device__ inline EpiOps<T> epi_pre(const Epi<T>& E, size_t i, int node) {
  EpiOps<T> o{T(0), T(0), T(0), T(0)};
  if (MODE == EPI_SCALE) o.a0 = E.sc[node];
  if (MODE == EPI_DINV) o.a0 = E.dinv[i];
  if (MODE == EPI_BMINUS) o.a0 = E.b[i];
  if (MODE == EPI_SUB) o.a0 = E.r[i];
  if (MODE == EPI_CHEB_INIT1) {
    o.a0 = E.b[i];
    o.a1 = E.dinv[i];
    o.a2 = E.x[i];
  }
  if (MODE == EPI_CHEB_STEP) {
    o.a0 = E.r[i];
    o.a1 = E.d[i];
    o.a2 = E.dinv[i];
    o.a3 = E.x[i];
  }
  return o;
}

template <int MODE, typename T>
__device__ inline void epi_post(const Epi<T>& E, size_t i, const EpiOps<T>& o, T v) {
  if (MODE == EPI_STORE) E.y[i] = v;
  if (MODE == EPI_SCALE) E.y[i] = v * o.a0;
  if (MODE == EPI_DINV) E.y[i] = o.a0 * v;
  if (MODE == EPI_BMINUS) E.y[i] = o.a0 - v;
  if (MODE == EPI_SUB) E.r[i] = o.a0 - v;
  if (MODE == EPI_CHEB_INIT1) {
    const T rv = o.a0 - v;
    const T dv = o.a1 * rv * E.inv_theta;
    E.r[i] = rv;
    E.d[i] = dv;
    E.x[i] = o.a2 + dv;
  }
  if (MODE == EPI_CHEB_STEP) {
    const T rv = o.a0 - v;
    const T dv = E.a * o.a1 + E.bc * (o.a2 * rv);
    E.r[i] = rv;
    E.d[i] = dv;
    E.x[i] = o.a3 + dv;
  }
}

// Launch helper: calls f(std::integral_constant<int, MODE>) for the runtime mode m.
template <typename F>
inline cudaError_t epi_dispatch(int m, F f) {
  switch (m) {
    case EPI_STORE: return f(std::integral_constant<int, EPI_STORE>());
    case EPI_CHEB_STEP: return f(std::integral_constant<int, EPI_CHEB_STEP>());
    case EPI_SUB: return f(std::integral_constant<int, EPI_SUB>());
    case EPI_CHEB_INIT1: return f(std::integral_constant<int, EPI_CHEB_INIT1>());
    case EPI_SCALE: return f(std::integral_constant<int, EPI_SCALE>());
    case EPI_DINV: return f(std::integral_constant<int, EPI_DINV>());
    case EPI_BMINUS: return f(std::integral_constant<int, EPI_BMINUS>());
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wb
